// tm_internal.h -- host-side structures and launcher declarations shared by
// the library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "tm_device.cuh"
#include "tmhop.h"

struct tm_ctx {
    int device = 0;
    std::string err;
    void *scratch = nullptr;       // odd-parity temporaries of Q_tm and friends
    size_t scratch_bytes = 0;
    int sm_count = 0;
    std::vector<cudaEvent_t> trace;  // events recorded at kernel boundaries (tm_ctx_trace)
    void *ws = nullptr;              // solver workspace (grow-only)
    size_t ws_bytes = 0;
    void *red = nullptr;             // partial sums of tm_spinor_dot (grow-only)
    size_t red_bytes = 0;
    int autotune = 1;                // time launch configurations on first use
    int batch_code = -1;             // forced batched-hop configuration (tm_ctx_set_batch_config), -1 = tuned
    unsigned batch_cap = 0;          // and its persistent CTA cap (0: one CTA per work item)
    std::map<std::string, std::pair<int, unsigned>> tuned;  // batched hop: key -> (pass width, CTA cap)
    std::map<std::string, float> tuned_ms;                  // and the winner's time for 3 launches
    std::map<std::string, int> tuned_band;                  // and its tile order (1 banded, 0 lexicographic)
    std::map<std::string, std::string> tuned_maps;          // single-lattice hop: key -> chosen map (tm_gauge_tune)
    std::string tune_cache;          // autotune cache file ("" = none; TMHOP_TUNE_CACHE at creation)
    void *stage = nullptr;           // device staging slots of tm_Qtm_host (grow-only)
    size_t stage_bytes = 0;
    cudaStream_t copy_in = nullptr;  // copy streams of tm_Qtm_host (created on first use)
    cudaStream_t copy_out = nullptr;
    // tm_Qtm_batch: its tables and odd temporaries (grow-only), and the batch
    // they were built for, so that a repeated call only launches
    void *bq = nullptr;
    size_t bq_bytes = 0;
    std::vector<uintptr_t> bq_sig;
    cudaStream_t bq_stream = nullptr;
    struct {
        int nrb = 1, ngroups = 0;
        unsigned grid = 0, nitems = 0;
        void *dsys = nullptr, *dgrp = nullptr;
        const void *smaps = nullptr, *lmaps = nullptr;  // tensor maps of the staged hop, if built
    } bq_tab;
    int *dev_status = nullptr;       // set by a kernel whose bounded wait ran out (tm_ctx_check)
};

// Records msg as the context's last error (tm_last_error) and returns st.
inline tm_status tm_fail(tm_ctx *ctx, tm_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

// n rounded up to a multiple of 256 bytes, the alignment of every
// sub-buffer carved out of a workspace.
constexpr size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Records trace event k of ctx on stream s, if tracing is on.
// A device pointer that the kernels may read or write with 16-byte vector
// accesses: non-null and 16-byte aligned (a misaligned vector access would
// fault on the device, so the host rejects it first).
inline bool bad_ptr(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

inline void tm_trace_mark(tm_ctx *ctx, size_t k, cudaStream_t s)
{
    if (k < ctx->trace.size()) cudaEventRecord(ctx->trace[k], s);
}

// The reliable-update threshold of a mixed-precision solve: the caller's
// value, or for a negative one the square root of the unit roundoff of the
// inner storage format, at least 1e-3 (FP32 1e-3, FP16 0.022).  Measured on
// 32^3x64: FP32 inner solves need no more iterations down to 1e-3 and take
// the fewest reliable updates there; FP16 ones start to need more
// iterations below about 0.01.
inline double reliable_delta_for(double delta, int inner_prec)
{
    if (delta >= 0.0) return delta;
    const double u = inner_prec == TM_F16 ? 0x1p-11 : 0x1p-24;
    const double d = __builtin_sqrt(u);
    return d > 1e-3 ? d : 1e-3;
}

// Grows the context's scratch buffer to at least `bytes` and returns it.
tm_status tm_ctx_scratch(tm_ctx *ctx, size_t bytes, void **ptr);
// Grows the context's solver workspace to at least `bytes` and returns it.
tm_status tm_ctx_workspace(tm_ctx *ctx, size_t bytes, void **ptr);
// Grows the context's reduction buffer (partials of tm_spinor_dot) and returns it.
tm_status tm_ctx_reduce_buffer(tm_ctx *ctx, size_t bytes, void **ptr);

struct tm_gauge {
    tm_ctx *ctx = nullptr;
    int dims[4] = {0, 0, 0, 0};
    int bc[4] = {1, 1, 1, 1};
    int prec = 0;
    int recon = 18;
    twm::Geom geom{};
    void *links = nullptr;
    size_t bytes = 0;
    twm::SiteMap map{};   // site-to-thread map of this lattice's hop launches (tm_gauge_tune)
    std::string map_name = "linear128";
    mutable void *links8 = nullptr;  // site-complete link copy of the staged batched hop (built on first use)
};

// Gives U the site map its lattice has in the context's tune cache, if any.
void tm_apply_cached_map(tm_ctx *ctx, tm_gauge *U);

namespace twm {
// The tune cache file (tm_tune.cu): lines "<key> <value> <ms>", the last
// entry of a key wins; keys start with the GPU's name.
std::string tune_cache_gpu(const tm_ctx *ctx);
bool tune_cache_lookup(const std::string &path, const std::string &key, std::string &value, double &ms);
void tune_cache_store(const std::string &path, const std::string &key, const std::string &value, double ms);
}  // namespace twm

namespace twm {

// Fills the geometry of a lattice; returns false if the extents are invalid.
bool make_geom(const int dims[4], const int bc[4], Geom &g);

// Launchers (tm_kernels.cu).  All enqueue on `s` and return the launch status.
// Q_tm of an FP64 handle on fields in the canonical layout: launch A
// (in_can -> tmp, an odd packed FP64 field) or launch B (tmp -> out_can,
// in_can re-read), with coefficients k.
cudaError_t launch_qtm_canonical(bool stage_b, const Geom &g, int recon, const SiteMap &m, const void *links,
                                 const double *in_can, void *tmp, double *out_can, const Coef &k, cudaStream_t s);
// The hop with the given site-to-thread map, or with the linear map of
// `block` threads per CTA.
cudaError_t launch_hop(const Geom &g, int prec, int recon, bool dag, int out_parity, const void *links,
                       const void *in, void *out, const void *x, const Coef &k, cudaStream_t s, const SiteMap &m);
cudaError_t launch_hop(const Geom &g, int prec, int recon, bool dag, int out_parity, const void *links,
                       const void *in, void *out, const void *x, const Coef &k, cudaStream_t s, int block);
cudaError_t launch_pack_gauge(const Geom &g, int prec, int recon, const double *U, void *links, cudaStream_t s);
cudaError_t launch_pack_spinor(unsigned vh, int prec, const double *in, void *out, cudaStream_t s);
cudaError_t launch_unpack_spinor(unsigned vh, int prec, const void *in, double *out, cudaStream_t s);
size_t link_chunk_bytes(int prec, int recon);
int link_nchunk(int prec, int recon);

// Coefficients of the two Q_tm launches (see tm_Qtm): kernel A gives
// (1 + i mut gamma5)^-1 H_oe in, kernel B gives
// gamma5 [ (1 + i mut gamma5) in - kappa^2 H_eo tmp ].
Coef coef_plain();
Coef coef_qtm_a(double mut);
Coef coef_qtm_b(double kappa, double mut);
Coef coef_qtm_a_scaled(double kappa, double mut);
Coef coef_qtm_b_unit(double mut);
// gamma5 (1 + i mut gamma5) / (1 + mut^2): the odd field B of the force
Coef coef_force_b(double mut);

}  // namespace twm
