// tm_batch.cu -- the operator and the solver over many systems at once:
// several right-hand sides on one lattice and several lattices of uneven
// volume, each step of the iteration one launch over all of them.
//
// Systems that share a gauge handle form a group.  A launch walks a work
// list of tiles of all groups; its CTAs are persistent (each takes items
// blockIdx.x, blockIdx.x + gridDim.x, ...), so one launch covers every
// lattice whatever their sizes.  The links are most of the bytes of a hop,
// so a group's n right-hand sides should read them once, not n times.  Two
// ways, both measured: (a) a CTA copies the 8 links of each tile site into
// shared memory once and applies them to all right-hand sides in passes;
// (b) consecutive work items are the right-hand sides of one tile, so the
// CTAs that need the same links run back to back and share them through L2
// (default-cached loads).  With one right-hand side per group links are
// streamed from global memory (evict-first).
// Tile size (right-hand sides processed together) and the number of
// persistent CTAs are picked by timing candidates on first use.
//
// Every system keeps its own CG scalars; reductions write one partial per
// (system, tile) and a small finishing launch sums them in index order.
// Kernels of finished systems, and reliable-update stages not due, exit at
// once, so a whole segment of iterations replays as one CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "tm_stage.cuh"
#include "tm_stage_host.h"

namespace twm {

// Maps a vector-kernel item to (system, tile of BLA sites) by the prefix
// table item0[nsys+1]; `staged` is its copy in shared memory (or null).
__device__ __forceinline__ int find_sys(const unsigned *item0, const unsigned *staged, int nsys, unsigned item)
{
    if (staged) return find_first(staged, nsys, item);
    int k = 0;
    while (k + 1 < nsys && item >= item0[k + 1]) ++k;
    return k;
}

// Stages item0[0 .. nsys) in `buf` (shared memory of STAGE_MAX entries) when
// it fits; every thread of the block must call it.  Returns the staged copy
// or null.
__device__ __forceinline__ const unsigned *stage_item0(const unsigned *item0, int nsys, unsigned *buf)
{
    if (nsys > STAGE_MAX) return nullptr;
    for (int k = threadIdx.x; k < nsys; k += blockDim.x) buf[k] = item0[k];
    __syncthreads();
    return buf;
}

// Block sum of v over BLA threads in a fixed order (warp sums, then the
// BLA / 32 warp results in order); the result is valid in thread 0.  Every
// thread of the block must call it.
__device__ __forceinline__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < BLA / 32; ++w) r += red[w];
    __syncthreads();  // red is reused by the caller's next item
    return r;
}

// p = r + beta p (restart: p = r)
template <int P>
__global__ void __launch_bounds__(BLA, P == F64 ? 3 : 4) k_batch_pupdate(const BSys *__restrict__ sys, const unsigned *item0, int nsys,
                                                       unsigned nitems, int gate, int restart)
{
    using R = typename SpinorIO<P>::R;
    __shared__ unsigned item0_s[STAGE_MAX];
    const unsigned *staged = stage_item0(item0, nsys, item0_s);
    for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int k = find_sys(item0, staged, nsys, item);
        const BSys &S = sys[k];
        if (gated(S.s, gate)) continue;
        const unsigned i = (item - item0[k]) * BLA + threadIdx.x;
        if (i >= S.vh) continue;
        Spinor<R> rv, pv;
        SpinorIO<P>::load(S.f[R_R], S.vh, i, rv);
        if (!restart) {
            const R b = to_R<R>(S.s->rr_new / S.s->rr);
            SpinorIO<P>::load(S.f[R_P], S.vh, i, pv);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rv[sp][c].re += b * pv[sp][c].re;
                    rv[sp][c].im += b * pv[sp][c].im;
                }
        }
        SpinorIO<P>::store(S.f[R_P], S.vh, i, rv);
    }
}

// x += y (FP64), y = 0
template <int PY>
__global__ void __launch_bounds__(BLA, 4) k_batch_accum(const BSys *__restrict__ sys, const unsigned *item0, int nsys,
                                                     unsigned nitems, int gate)
{
    using RY = typename SpinorIO<PY>::R;
    __shared__ unsigned item0_s[STAGE_MAX];
    const unsigned *staged = stage_item0(item0, nsys, item0_s);
    for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int k = find_sys(item0, staged, nsys, item);
        const BSys &S = sys[k];
        if (gated(S.s, gate)) continue;
        const unsigned i = (item - item0[k]) * BLA + threadIdx.x;
        if (i >= S.vh) continue;
        Spinor<double> xv;
        Spinor<RY> yv, z;
        SpinorIO<F64>::load(S.f[R_X], S.vh, i, xv);
        SpinorIO<PY>::load(S.f[R_Y], S.vh, i, yv);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xv[sp][c].re += double(yv[sp][c].re);
                xv[sp][c].im += double(yv[sp][c].im);
                z[sp][c] = {RY(0), RY(0)};
            }
        SpinorIO<F64>::store(S.f[R_X], S.vh, i, xv);
        SpinorIO<PY>::store(S.f[R_Y], S.vh, i, z);
    }
}

// r_lo = b - Ax in precision P (FP64 arithmetic), partial |b - Ax|^2
template <int P>
__global__ void __launch_bounds__(BLA, 3) k_batch_residual(const BSys *__restrict__ sys, const unsigned *item0, int nsys,
                                                        unsigned nitems, int gate)
{
    using R = typename SpinorIO<P>::R;
    __shared__ double red[BLA / 32];
    __shared__ unsigned item0_s[STAGE_MAX];
    const unsigned *staged = stage_item0(item0, nsys, item0_s);
    for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int k = find_sys(item0, staged, nsys, item);
        const BSys &S = sys[k];
        if (gated(S.s, gate)) continue;
        const unsigned tno = item - item0[k], i = tno * BLA + threadIdx.x;
        double nrm = 0.0;
        if (i < S.vh) {
            Spinor<double> bv, av;
            SpinorIO<F64>::load(S.f[R_B], S.vh, i, bv);
            SpinorIO<F64>::load(S.f[R_AX], S.vh, i, av);
            Spinor<R> lo;
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    bv[sp][c].re -= av[sp][c].re;
                    bv[sp][c].im -= av[sp][c].im;
                    lo[sp][c] = {to_R<R>(bv[sp][c].re), to_R<R>(bv[sp][c].im)};
                }
            SpinorIO<P>::store(S.f[R_R], S.vh, i, lo);
            nrm = norm2(bv);
        }
        double sum = block_sum(nrm, red);
        if (threadIdx.x == 0) S.partials[tno] = sum;
    }
}

// partial |f|^2 of an FP64 field
__global__ void __launch_bounds__(BLA, 4) k_batch_norm(const BSys *__restrict__ sys, const unsigned *item0, int nsys,
                                                    unsigned nitems, int role)
{
    __shared__ double red[BLA / 32];
    __shared__ unsigned item0_s[STAGE_MAX];
    const unsigned *staged = stage_item0(item0, nsys, item0_s);
    for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int k = find_sys(item0, staged, nsys, item);
        const BSys &S = sys[k];
        const unsigned tno = item - item0[k], i = tno * BLA + threadIdx.x;
        double nrm = 0.0;
        if (i < S.vh) {
            Spinor<double> v;
            SpinorIO<F64>::load(S.f[role], S.vh, i, v);
            nrm = norm2(v);
        }
        double sum = block_sum(nrm, red);
        if (threadIdx.x == 0) S.partials[tno] = sum;
    }
}

template <int P>
__global__ void __launch_bounds__(BLA, 4) k_batch_zero(const BSys *__restrict__ sys, const unsigned *item0, int nsys,
                                                    unsigned nitems, int role)
{
    using R = typename SpinorIO<P>::R;
    __shared__ unsigned item0_s[STAGE_MAX];
    const unsigned *staged = stage_item0(item0, nsys, item0_s);
    for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int k = find_sys(item0, staged, nsys, item);
        const BSys &S = sys[k];
        const unsigned i = (item - item0[k]) * BLA + threadIdx.x;
        if (i >= S.vh) continue;
        Spinor<R> z;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) z[sp][c] = {R(0), R(0)};
        SpinorIO<P>::store(S.f[role], S.vh, i, z);
    }
}

// One CTA per system: sums its partials (tiles of tile_sites sites) in index
// order and finishes `op`.
__global__ void __launch_bounds__(BLA, 4) k_batch_finish(const BSys *__restrict__ sys, int nsys, unsigned tile_sites, int op,
                                                      int gate)
{
    __shared__ double red[BLA / 32];
    const BSys &S = sys[blockIdx.x];
    if (gated(S.s, gate)) return;
    const unsigned n = (S.vh + tile_sites - 1) / tile_sites;
    double acc = 0.0;
    for (unsigned t = threadIdx.x; t < n; t += BLA) acc += S.partials[t];
    double sum = block_sum(acc, red);
    if (threadIdx.x == 0) cg_finish(op, sum, S.s);
}

// ------------------------------------------------------------------ host side
namespace {

struct Batch {
    int nsys = 0, ngroups = 0;
    int P = F64, recon_lo = 18, recon_hi = 18, PY = F64;
    std::vector<BGroup> groups_lo, groups_hi;   // host templates (links set per precision)
    std::vector<int> order;                     // batch position -> caller's system index
    BSys *sys = nullptr;                        // device array
    unsigned *la_item0 = nullptr;               // device prefix table of vector-kernel items
    unsigned la_items = 0, la_grid = 0;
    HopTable lo, hi;
};

unsigned cdiv(unsigned a, unsigned b) { return (a + b - 1) / b; }

cudaError_t bhop(int prec, int recon, const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx,
                 const Coef &k, int mode, int gate, cudaStream_t st)
{
    if (t.nitems == 0) return cudaSuccess;
    switch (prec * 100 + recon) {
    case F64 * 100 + 18: return batch_hop_f64(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    case F64X * 100 + 18: return batch_hop_f64x(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    case F32 * 100 + 12: return batch_hop_f32_12(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    case F32 * 100 + 18: return batch_hop_f32_18(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    case F16 * 100 + 12: return batch_hop_f16(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    }
    return cudaErrorInvalidValue;
}

// Candidate link-sharing modes for a storage format (static shared memory <= 48 KB),
// and the staged hop where its tensor maps were built (`staged`).
std::vector<int> nrb_candidates(int prec, int recon, int nrhs_max, bool staged = false)
{
    std::vector<int> c{1};
    if (staged) c.push_back(STAGE_CODE);
    if (nrhs_max <= 1) return c;
    c.push_back(0);
    if (prec != F64 && prec != F64X) c.push_back(2);
    c.push_back(4);
    if (prec == F32 || prec == F16) {   // two right-hand sides per thread
        c.push_back(10);
        c.push_back(12);
        c.push_back(14);
    }
    (void)recon;
    return c;
}

// z planes per band of the gather hops' tile order (tile_of) on lattice g
// with tiles of ts sites: the largest divisor of Lz whose band slab holds at
// most TM_BATCH_BAND_SITES sites and whole tiles; 0 (lexicographic) if none.
#ifndef TM_BATCH_BAND_SITES
#define TM_BATCH_BAND_SITES 8192
#endif
int zband_for(const Geom &g, unsigned ts)
{
    const unsigned plane = unsigned(g.hx) * unsigned(g.ly);
    int best = 0;
    for (int b = 1; b < g.lz; ++b)
        if (g.lz % b == 0 && (plane * unsigned(b)) % ts == 0 && plane * unsigned(b) <= TM_BATCH_BAND_SITES) best = b;
    return best;
}

// Whether the gather hops of a storage format walk their tiles in z bands.
// Measured on 32^3x64 with 12 right-hand sides (tuned configuration, Q_tm
// per call): FP32-12 1.87 ms banded against 1.91 lexicographic (launch B
// 0.99 against 1.02 ms: fewer neighbour re-reads from memory), FP16-12 1.743
// against 1.721.  Timing both orders in the tuner did not separate them (its
// launches differ by less than their spread), so the order is fixed per format.
bool band_order(int prec) { return prec != F16; }

// Fills a hop table for pass width nrb and uploads it to `dev` (capacity ngroups).
cudaError_t build_table(const std::vector<BGroup> &tmpl, int nrb, unsigned grid_cap, HopTable &t, BGroup *dev,
                        cudaStream_t st, std::vector<BGroup> &host, const StageArgs &sa = StageArgs{},
                        bool band = true)
{
    host = tmpl;
    const int w = code_nrb(nrb), rpt = code_rpt(nrb);
    const unsigned ts = w > 1 ? BT / w : BT;
    unsigned item = 0;
    for (auto &g : host) {
        g.item0 = item;
        if (nrb == STAGE_CODE) {   // boxes of STS sites, all right-hand sides of a box in one item
            g.ntiles = g.g.vh / STS;
            g.sbz = stage_zblock(g.g);
            item += g.ntiles;
            continue;
        }
        g.ntiles = cdiv(g.g.vh, ts);
        g.zband = band && g.nrhs > 1 ? zband_for(g.g, ts) : 0;
        item += w <= 1 ? g.ntiles * cdiv(unsigned(g.nrhs), unsigned(rpt)) : g.ntiles;
    }
    t.sa = sa;
    t.nrb = nrb;
    t.nitems = item;
    t.grid = std::max(1u, std::min(item, grid_cap));
    t.ngroups = int(host.size());
    t.dev = dev;
    return cudaMemcpyAsync(dev, host.data(), sizeof(BGroup) * host.size(), cudaMemcpyHostToDevice, st);
}

// Times a candidate hop table with (parity 1, rin -> rout) launches; returns
// ms.  rin and rout must be fields of the table's precision.  The time of
// three launches is the median of three rounds, so that one disturbed round
// (clock ramp, another process's work) can neither hide a slow configuration
// nor discard a fast one.  A round is two launches without and one with the
// second input stream of Q_tm's second hop (rout read as x before each
// thread overwrites its own site: the traffic, not the meaning), the mix of
// a Q_tm application.
float time_table(int prec, int recon, const HopTable &t, const BSys *sys, int rin, int rout, cudaStream_t st)
{
    cudaEvent_t ev[4];
    for (auto &e : ev) cudaEventCreate(&e);
    Coef k = coef_plain();
    bhop(prec, recon, t, sys, 1, rin, rout, -1, k, BH_PLAIN, 0, st);
    float ms[3] = {0.f, 0.f, 0.f};
    cudaEventRecord(ev[0], st);
    for (int round = 0; round < 3; ++round) {
        for (int r = 0; r < 3; ++r) bhop(prec, recon, t, sys, 1, rin, rout, r == 2 ? rout : -1, k, BH_PLAIN, 0, st);
        cudaEventRecord(ev[round + 1], st);
    }
    cudaEventSynchronize(ev[3]);
    for (int round = 0; round < 3; ++round) cudaEventElapsedTime(&ms[round], ev[round], ev[round + 1]);
    for (auto &e : ev) cudaEventDestroy(e);
    if (cudaGetLastError() != cudaSuccess) return 1e30f;
    std::sort(ms, ms + 3);
    return ms[1];
}

}  // namespace

// Picks the pass width and persistent grid of a batched hop by timing, with a
// per-context cache keyed by precision and the shape of the batch.
cudaError_t tune_hop_table(tm_ctx *ctx, int prec, int recon, const std::vector<BGroup> &tmpl, BGroup *dev,
                           const BSys *sys, int rin, int rout, HopTable &out, cudaStream_t st,
                           const StageArgs *sa = nullptr)
{
    const StageArgs no_stage{};
    const StageArgs &sta = sa ? *sa : no_stage;
    int nrhs_max = 0;
    std::string key = "bhop/" + std::to_string(prec) + "/" + std::to_string(recon);
    for (auto &g : tmpl) {
        nrhs_max = std::max(nrhs_max, g.nrhs);
        key += "/" + std::to_string(g.g.vh) + "x" + std::to_string(g.nrhs);
    }
    const unsigned sms = unsigned(std::max(1, ctx->sm_count));
    std::vector<BGroup> host;
    if (ctx->batch_code >= 0) {   // a configuration set by the caller, where this format has it
        const std::vector<int> ok = nrb_candidates(prec, recon, std::max(nrhs_max, 2), sa != nullptr);
        if (std::find(ok.begin(), ok.end(), ctx->batch_code) != ok.end()) {
            const unsigned dcap = ctx->batch_code == STAGE_CODE ? sms : 1u << 30;
            cudaError_t e = build_table(tmpl, ctx->batch_code, ctx->batch_cap ? ctx->batch_cap : dcap, out, dev,
                                        st, host, sta, band_order(prec));
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            return e;
        }
    }
    if (sa) key += "/staged";
    auto it = ctx->tuned.find(key);
    // a choice persisted by an earlier process (tm_ctx_set_tune_cache), if its code is a candidate here
    const std::string ckey = tune_cache_gpu(ctx) + "|" + key;
    if (it == ctx->tuned.end() && ctx->autotune && !ctx->tune_cache.empty()) {
        std::string val;
        double cms = 0;
        int code = -1;
        unsigned cap = 0;
        if (tune_cache_lookup(ctx->tune_cache, ckey, val, cms) && sscanf(val.c_str(), "code%d-cap%u", &code, &cap) == 2) {
            const std::vector<int> ok = nrb_candidates(prec, recon, nrhs_max, sa != nullptr);
            if (std::find(ok.begin(), ok.end(), code) != ok.end() && cap > 0) {
                ctx->tuned[key] = {code, cap};
                ctx->tuned_ms[key] = float(cms);
                ctx->tuned_band[key] = band_order(prec) ? 1 : 0;
                it = ctx->tuned.find(key);
            }
        }
    }
    if (it != ctx->tuned.end()) {
        cudaError_t e = build_table(tmpl, it->second.first, it->second.second, out, dev, st, host, sta,
                                    band_order(prec));
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e;
    }
    float best = 1e30f;
    int best_nrb = 1;
    unsigned best_cap = 1u << 30;
    const unsigned caps[] = {sms * 4, sms * 8, sms * 16, 1u << 30};
    for (int nrb : nrb_candidates(prec, recon, nrhs_max, sa != nullptr)) {
        for (unsigned cap : caps) {
            if (nrb == STAGE_CODE && cap != caps[0]) break;   // one CTA per SM, persistent
            HopTable t;
            cudaError_t e = build_table(tmpl, nrb, nrb == STAGE_CODE ? sms : cap, t, dev, st, host, sta,
                                        band_order(prec));
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            float ms = ctx->autotune ? time_table(prec, recon, t, sys, rin, rout, st) : 0.f;
            if (ms < best) {
                best = ms;
                best_nrb = nrb;
                best_cap = nrb == STAGE_CODE ? sms : cap;
            }
            if (!ctx->autotune) break;
        }
        if (!ctx->autotune) {
            best_nrb = nrhs_max > 1 ? 4 : 1;
            break;
        }
    }
    ctx->tuned[key] = {best_nrb, best_cap};
    ctx->tuned_ms[key] = best;
    ctx->tuned_band[key] = band_order(prec) ? 1 : 0;
    if (ctx->autotune && !ctx->tune_cache.empty())
        tune_cache_store(ctx->tune_cache, ckey, "code" + std::to_string(best_nrb) + "-cap" + std::to_string(best_cap),
                         best);
    cudaError_t e = build_table(tmpl, best_nrb, best_cap, out, dev, st, host, sta, band_order(prec));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace twm

using namespace twm;

namespace {


tm_status bcuda(tm_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    return TM_ERR_CUDA;
}


// Groups the systems by gauge handle (first appearance order) and fills the
// group templates; order[k] is the caller's index of batch position k.
tm_status group_systems(tm_ctx *ctx, int nsys, const tm_gauge *const *U, std::vector<const tm_gauge *> &handles,
                        std::vector<std::vector<int>> &members)
{
    for (int k = 0; k < nsys; ++k) {
        if (!U[k]) return tm_fail(ctx, TM_ERR_ARG, "batch: null gauge handle");
        size_t g = 0;
        while (g < handles.size() && handles[g] != U[k]) ++g;
        if (g == handles.size()) {
            handles.push_back(U[k]);
            members.emplace_back();
        }
        members[g].push_back(k);
    }
    return TM_OK;
}

}  // namespace

extern "C" tm_status tm_ctx_set_batch_config(tm_ctx *ctx, int code, unsigned cap)
{
    if (!ctx) return TM_ERR_ARG;
    if (code != -1 && code != 0 && code != 1 && code != 2 && code != 4 && code != 10 && code != 12 && code != 14 &&
        code != STAGE_CODE)
        return tm_fail(ctx, TM_ERR_ARG, "tm_ctx_set_batch_config: code must be -1, 0, 1, 2, 4, 10, 12, 14 or 100");
    ctx->batch_code = code;
    ctx->batch_cap = cap;
    return TM_OK;
}

extern "C" tm_status tm_Qtm_batch(tm_ctx *ctx, int nsys, const tm_gauge *const *U, void *const *out_e,
                                  const void *const *in_e, double kappa, double mu, int sign, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (nsys < 1 || !U || !out_e || !in_e) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_batch: bad arguments");
    if (sign != 1 && sign != -1) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_batch: sign must be +1 or -1");
    std::vector<const tm_gauge *> handles;
    std::vector<std::vector<int>> members;
    tm_status st = group_systems(ctx, nsys, U, handles, members);
    if (st != TM_OK) return st;
    const int prec = handles[0]->prec, recon = handles[0]->recon;
    for (auto *h : handles)
        if (h->prec != prec || h->recon != recon)
            return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_Qtm_batch: all gauge handles need the same precision and reconstruction");
    for (int k = 0; k < nsys; ++k) {
        if (bad_ptr(out_e[k]) || bad_ptr(in_e[k]) || out_e[k] == in_e[k]) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_batch: bad field pointer");
    }
    {   // every output is written by one system and read by none (inputs may repeat)
        std::set<const void *> outs(out_e, out_e + nsys), ins(in_e, in_e + nsys);
        if (int(outs.size()) != nsys) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_batch: an output field appears twice");
        for (const void *o : outs)
            if (ins.count(o)) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_batch: an output field is also an input");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // The staged hop is a candidate where every lattice is tiled by its boxes
    // and some lattice has several right-hand sides (its links are shared).
    bool staged = stage_supported(prec, recon) && stage_available();
    size_t nrhs_max = 0;
    for (size_t g = 0; g < handles.size(); ++g) {
        nrhs_max = std::max(nrhs_max, members[g].size());
        staged = staged && stage_geometry_ok(handles[g]->geom);
    }
    staged = staged && nrhs_max >= 2;
    cudaError_t e = cudaSuccess;
    if (staged) {
        // the staged hop is an optional candidate: without memory for its link
        // copies the batch runs with the gather hops alone
        for (auto *h : handles)
            if (e == cudaSuccess) e = stage_links8(h, s);
        if (e == cudaSuccess && !ctx->dev_status) {
            e = cudaMalloc(&ctx->dev_status, sizeof(int));
            if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), s);
            else ctx->dev_status = nullptr;
        }
        if (e == cudaErrorMemoryAllocation) {
            (void)cudaGetLastError();   // not sticky: clear it and go on without the staged hop
            staged = false;
            e = cudaSuccess;
        }
        if (e != cudaSuccess) return bcuda(ctx, e, "tm_Qtm_batch: staged-hop links");
    }
    // The batch as the device tables describe it: handles (with their links
    // and sizes), fields, precision and stream.  A repeated call with the same
    // batch finds its tables and temporaries in place and only launches.
    std::vector<uintptr_t> sig{uintptr_t(prec), uintptr_t(recon), uintptr_t(nsys), uintptr_t(s),
                               uintptr_t(ctx->batch_code + 1), uintptr_t(ctx->batch_cap), uintptr_t(staged)};
    for (int k = 0; k < nsys; ++k) {
        sig.push_back(uintptr_t(U[k]));
        sig.push_back(uintptr_t(U[k]->links));
        sig.push_back(uintptr_t(U[k]->links8));
        const Geom &gk = U[k]->geom;   // a handle re-created at the same address may describe another lattice
        sig.push_back((uintptr_t(gk.lx) << 48) | (uintptr_t(gk.ly) << 32) | (uintptr_t(gk.lz) << 16) | uintptr_t(gk.lt));
        sig.push_back(uintptr_t(gk.anti[0]) | uintptr_t(gk.anti[1]) << 1 | uintptr_t(gk.anti[2]) << 2 |
                      uintptr_t(gk.anti[3]) << 3);
        sig.push_back(uintptr_t(out_e[k]));
        sig.push_back(uintptr_t(in_e[k]));
    }
    HopTable t;
    BSys *dsys = nullptr;
    if (ctx->bq && sig == ctx->bq_sig) {
        t.nrb = ctx->bq_tab.nrb;
        t.grid = ctx->bq_tab.grid;
        t.nitems = ctx->bq_tab.nitems;
        t.ngroups = ctx->bq_tab.ngroups;
        t.dev = static_cast<BGroup *>(ctx->bq_tab.dgrp);
        t.sa.smaps = static_cast<const CUtensorMap *>(ctx->bq_tab.smaps);
        t.sa.lmaps = static_cast<const CUtensorMap *>(ctx->bq_tab.lmaps);
        t.sa.status = ctx->dev_status;
        t.sa.roles = t.sa.smaps ? (1u << R_IN) | (1u << R_T) : 0u;
        dsys = static_cast<BSys *>(ctx->bq_tab.dsys);
    } else {
        // the previous batch's launches may still read the buffer on another stream
        if (ctx->bq && ctx->bq_stream != s) {
            e = cudaStreamSynchronize(ctx->bq_stream);
            if (e != cudaSuccess) return bcuda(ctx, e, "tm_Qtm_batch: previous batch");
        }
        ctx->bq_sig.clear();
        // buffer: odd temporaries, system table, group table
        size_t need = 0;
        for (int k = 0; k < nsys; ++k) need += align256(spinor_bytes(U[k]->geom.vh, prec));
        need += align256(sizeof(BSys) * nsys) + align256(sizeof(BGroup) * handles.size());
        const size_t nsmap = size_t(nsys) * NROLE * 2 * NSH;   // [system][role][shape] field maps
        if (staged) need += align256(sizeof(CUtensorMap) * nsmap) + align256(sizeof(CUtensorMap) * handles.size());
        if (ctx->bq_bytes < need) {
            if (ctx->bq) cudaFree(ctx->bq);
            ctx->bq = nullptr;
            ctx->bq_bytes = 0;
            e = cudaMalloc(&ctx->bq, need);
            if (e != cudaSuccess) return bcuda(ctx, e, "tm_Qtm_batch: cudaMalloc");
            ctx->bq_bytes = need;
        }
        char *c = static_cast<char *>(ctx->bq);
        std::vector<BSys> hs;
        std::vector<BGroup> tmpl;
        std::vector<void *> tmp(nsys);
        for (int k = 0; k < nsys; ++k) {
            tmp[k] = c;
            c += align256(spinor_bytes(U[k]->geom.vh, prec));
        }
        for (size_t g = 0; g < handles.size(); ++g) {
            BGroup G{};
            G.g = handles[g]->geom;
            G.links = handles[g]->links;
            G.nrhs = int(members[g].size());
            G.sys0 = int(hs.size());
            tmpl.push_back(G);
            for (int k : members[g]) {
                BSys S{};
                S.f[R_IN] = const_cast<void *>(in_e[k]);
                S.f[R_OUT] = out_e[k];
                S.f[R_T] = tmp[k];
                S.vh = U[k]->geom.vh;
                hs.push_back(S);
            }
        }
        dsys = reinterpret_cast<BSys *>(c);
        c += align256(sizeof(BSys) * nsys);
        BGroup *dgrp = reinterpret_cast<BGroup *>(c);
        c += align256(sizeof(BGroup) * handles.size());
        // pageable source: the copy has taken the data when the call returns
        e = cudaMemcpyAsync(dsys, hs.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, s);
        StageArgs sa{};
        if (staged && e == cudaSuccess) {
            // tensor maps of the two hop inputs of every system and of every group's links
            std::vector<CUtensorMap> hm(nsmap), hl(handles.size());
            memset(hm.data(), 0, sizeof(CUtensorMap) * nsmap);
            bool ok = true;
            for (int q = 0; q < nsys && ok; ++q) {
                const Geom &gq = tmpl[size_t(std::upper_bound(tmpl.begin(), tmpl.end(), q,
                                                              [](int v, const BGroup &G) { return v < G.sys0; }) -
                                             tmpl.begin()) - 1].g;
                for (int role : {int(R_IN), int(R_T)})
                    ok = ok && stage_field_maps(prec, gq, hs[size_t(q)].f[role], &hm[(size_t(q) * NROLE + role) * 2 * NSH]);
            }
            for (size_t g = 0; g < handles.size() && ok; ++g) ok = stage_link_map(handles[g], hl[g]);
            if (ok) {
                CUtensorMap *dsm = reinterpret_cast<CUtensorMap *>(c);
                c += align256(sizeof(CUtensorMap) * nsmap);
                CUtensorMap *dlm = reinterpret_cast<CUtensorMap *>(c);
                e = cudaMemcpyAsync(dsm, hm.data(), sizeof(CUtensorMap) * nsmap, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(dlm, hl.data(), sizeof(CUtensorMap) * hl.size(), cudaMemcpyHostToDevice, s);
                sa.smaps = dsm;
                sa.lmaps = dlm;
                sa.status = ctx->dev_status;
                sa.roles = (1u << R_IN) | (1u << R_T);
            }
        }
        if (e == cudaSuccess)
            e = tune_hop_table(ctx, prec, recon, tmpl, dgrp, dsys, R_IN, R_T, t, s, sa.smaps ? &sa : nullptr);
        if (e != cudaSuccess) return bcuda(ctx, e, "tm_Qtm_batch: setup");
        ctx->bq_sig = sig;
        ctx->bq_stream = s;
        ctx->bq_tab.nrb = t.nrb;
        ctx->bq_tab.grid = t.grid;
        ctx->bq_tab.nitems = t.nitems;
        ctx->bq_tab.ngroups = t.ngroups;
        ctx->bq_tab.dsys = dsys;
        ctx->bq_tab.dgrp = dgrp;
        ctx->bq_tab.smaps = t.sa.smaps;
        ctx->bq_tab.lmaps = t.sa.lmaps;
    }
    const double mut = 2.0 * kappa * mu * sign;
    tm_trace_mark(ctx, 0, s);
    e = bhop(prec, recon, t, dsys, 1, R_IN, R_T, -1, coef_qtm_a_scaled(kappa, mut), BH_PLAIN, 0, s);
    tm_trace_mark(ctx, 1, s);
    if (e == cudaSuccess) e = bhop(prec, recon, t, dsys, 0, R_T, R_OUT, R_IN, coef_qtm_b_unit(mut), BH_PLAIN, 0, s);
    tm_trace_mark(ctx, 2, s);
    if (e != cudaSuccess) return bcuda(ctx, e, "tm_Qtm_batch: launch");
    return TM_OK;
}

extern "C" tm_status tm_cg_QdagQ_batch(tm_ctx *ctx, int nsys, const tm_gauge *const *U_hi, const tm_gauge *const *U_lo,
                                       void *const *x_dev, const void *const *b_dev, const tm_cg_params *prm,
                                       tm_cg_info *info, void *stream)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!ctx) return TM_ERR_ARG;
    if (nsys < 1 || !U_hi || !x_dev || !b_dev || !prm) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: bad arguments");
    if (!(prm->tol > 0.0) || prm->maxiter < 0 || prm->reliable_every < 1 || !(prm->reliable_delta < 1.0))
        return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: bad solver parameters");
    std::vector<const tm_gauge *> handles;
    std::vector<std::vector<int>> members;
    tm_status st = group_systems(ctx, nsys, U_hi, handles, members);
    if (st != TM_OK) return st;
    // inner handles: one per group, same precision everywhere
    std::vector<const tm_gauge *> lo(handles.size());
    for (size_t g = 0; g < handles.size(); ++g) {
        if (handles[g]->prec != TM_F64) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: U_hi must be FP64 handles");
        for (int k : members[g]) {
            const tm_gauge *l = (U_lo && U_lo[k]) ? U_lo[k] : U_hi[k];
            if (lo[g] && lo[g] != l) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: systems sharing U_hi need the same U_lo");
            lo[g] = l;
            if (memcmp(l->dims, handles[g]->dims, sizeof l->dims) || memcmp(l->bc, handles[g]->bc, sizeof l->bc))
                return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: U_hi and U_lo describe different lattices");
            if (bad_ptr(x_dev[k]) || bad_ptr(b_dev[k]) || x_dev[k] == b_dev[k]) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: bad field pointer");
        }
    }
    {   // every solution is written by one system and read by none (sources may repeat)
        std::set<const void *> xs(x_dev, x_dev + nsys), bs(b_dev, b_dev + nsys);
        if (int(xs.size()) != nsys) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: a solution field appears twice");
        for (const void *x : xs)
            if (bs.count(x)) return tm_fail(ctx, TM_ERR_ARG, "tm_cg_QdagQ_batch: a solution field is also a source");
    }
    for (size_t g = 0; g < handles.size(); ++g)
        if (lo[g]->prec != lo[0]->prec || lo[g]->recon != lo[0]->recon || handles[g]->recon != handles[0]->recon)
            return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_cg_QdagQ_batch: all systems need the same storage formats");
    if (lo[0]->prec == TM_F64X)
        return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_cg_QdagQ_batch: TM_F64X inner handles are not supported");

    Batch B;
    B.nsys = nsys;
    B.ngroups = int(handles.size());
    B.P = lo[0]->prec;
    B.recon_lo = lo[0]->recon;
    B.recon_hi = handles[0]->recon;
    B.PY = B.P == F16 ? F32 : B.P;

    // workspace per system: inner r, p, q, t; y; FP64 ax, t_hi, q_hi; partials; scalars
    std::vector<size_t> sys_bytes(nsys);
    size_t need = 0;
    for (int k = 0; k < nsys; ++k) {
        unsigned vh = U_hi[k]->geom.vh;
        size_t fl = align256(spinor_bytes(vh, B.P)), fy = align256(spinor_bytes(vh, B.PY)), f64 = align256(spinor_bytes(vh, F64));
        sys_bytes[k] = 4 * fl + fy + 3 * f64 + align256(sizeof(double) * (vh / 16 + 2)) + align256(sizeof(CgScalars));
        need += sys_bytes[k];
    }
    need += align256(sizeof(BSys) * nsys) + 2 * align256(sizeof(BGroup) * handles.size()) + align256(sizeof(unsigned) * (nsys + 1));
    void *base = nullptr;
    st = tm_ctx_workspace(ctx, need, &base);
    if (st != TM_OK) return st;
    char *c = static_cast<char *>(base);
    auto take = [&](size_t n) { void *p = c; c += align256(n); return p; };

    std::vector<BSys> hs;
    std::vector<BGroup> tl, th;
    std::vector<unsigned> item0;
    unsigned la_items = 0;
    for (size_t g = 0; g < handles.size(); ++g) {
        BGroup G{};
        G.g = handles[g]->geom;
        G.nrhs = int(members[g].size());
        G.sys0 = int(hs.size());
        G.links = lo[g]->links;
        tl.push_back(G);
        G.links = handles[g]->links;
        th.push_back(G);
        for (int k : members[g]) {
            unsigned vh = G.g.vh;
            BSys S{};
            S.vh = vh;
            S.f[R_X] = x_dev[k];
            S.f[R_B] = const_cast<void *>(b_dev[k]);
            S.f[R_R] = take(spinor_bytes(vh, B.P));
            S.f[R_P] = take(spinor_bytes(vh, B.P));
            S.f[R_Q] = take(spinor_bytes(vh, B.P));
            S.f[R_T] = take(spinor_bytes(vh, B.P));
            S.f[R_Y] = take(spinor_bytes(vh, B.PY));
            S.f[R_AX] = take(spinor_bytes(vh, F64));
            S.f[R_THI] = take(spinor_bytes(vh, F64));
            S.f[R_QHI] = take(spinor_bytes(vh, F64));
            S.partials = static_cast<double *>(take(sizeof(double) * (vh / 16 + 2)));
            S.s = static_cast<CgScalars *>(take(sizeof(CgScalars)));
            hs.push_back(S);
            B.order.push_back(k);
            item0.push_back(la_items);
            la_items += cdiv(vh, BLA);
        }
    }
    item0.push_back(la_items);
    B.sys = static_cast<BSys *>(take(sizeof(BSys) * nsys));
    BGroup *dlo = static_cast<BGroup *>(take(sizeof(BGroup) * handles.size()));
    BGroup *dhi = static_cast<BGroup *>(take(sizeof(BGroup) * handles.size()));
    B.la_item0 = static_cast<unsigned *>(take(sizeof(unsigned) * (nsys + 1)));
    B.la_items = la_items;
    B.la_grid = std::min(la_items, unsigned(std::max(1, ctx->sm_count)) * 8u);

    cudaStream_t s = (cudaStream_t)stream;
    std::vector<CgScalars> hsc(nsys);
    for (auto &h : hsc) {
        h = CgScalars{};
        h.tol2 = prm->tol * prm->tol;
        h.maxiter = prm->maxiter;
        const double d = reliable_delta_for(prm->reliable_delta, B.P);
        h.delta2 = d * d;
        h.every = prm->reliable_every;
        h.mixed = 1;
    }
    cudaError_t e = cudaMemcpyAsync(B.sys, hs.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, s);
    for (int k = 0; k < nsys && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(hs[k].s, &hsc[k], sizeof(CgScalars), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.la_item0, item0.data(), sizeof(unsigned) * (nsys + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // tuning launches read whatever the work fields hold and write scratch fields of the same precision
    if (e == cudaSuccess) e = tune_hop_table(ctx, B.P, B.recon_lo, tl, dlo, B.sys, R_P, R_T, B.lo, s);
    if (e == cudaSuccess) e = tune_hop_table(ctx, F64, B.recon_hi, th, dhi, B.sys, R_AX, R_THI, B.hi, s);
    if (e != cudaSuccess) return bcuda(ctx, e, "tm_cg_QdagQ_batch: setup");

    const double kappa = prm->kappa, mut = 2.0 * prm->kappa * prm->mu;
    const unsigned G = B.la_grid, NI = B.la_items;
    BSys *SY = B.sys;
    unsigned *I0 = B.la_item0;
    auto finish = [&](unsigned tile_sites, int op, int gate, cudaStream_t q) {
        k_batch_finish<<<nsys, BLA, 0, q>>>(SY, nsys, tile_sites, op, gate);
        return cudaGetLastError();
    };
    auto hop_tile = [&](const HopTable &t) { return unsigned(code_nrb(t.nrb) > 1 ? BT / code_nrb(t.nrb) : BT); };
    // ax = Q^dag Q x in FP64 for the systems the gate lets through
    auto qdagq_hi = [&](int gate, cudaStream_t q) {
        cudaError_t r = bhop(F64, B.recon_hi, B.hi, SY, 1, R_X, R_THI, -1, coef_qtm_a_scaled(kappa, mut), BH_PLAIN, gate, q);
        if (r == cudaSuccess) r = bhop(F64, B.recon_hi, B.hi, SY, 0, R_THI, R_QHI, R_X, coef_qtm_b_unit(mut), BH_PLAIN, gate, q);
        if (r == cudaSuccess) r = bhop(F64, B.recon_hi, B.hi, SY, 1, R_QHI, R_THI, -1, coef_qtm_a_scaled(kappa, -mut), BH_PLAIN, gate, q);
        if (r == cudaSuccess) r = bhop(F64, B.recon_hi, B.hi, SY, 0, R_THI, R_AX, R_QHI, coef_qtm_b_unit(-mut), BH_PLAIN, gate, q);
        return r;
    };
    auto residual = [&](int gate, cudaStream_t q) {
        if (B.P == F64) k_batch_residual<F64><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, gate);
        else if (B.P == F32) k_batch_residual<F32><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, gate);
        else k_batch_residual<F16><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, gate);
        cudaError_t r = cudaGetLastError();
        if (r == cudaSuccess) r = finish(BLA, FIN_RR_TRUE, gate, q);
        return r;
    };
    auto pupdate = [&](int gate, int restart, cudaStream_t q) {
        if (B.P == F64) k_batch_pupdate<F64><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, gate, restart);
        else if (B.P == F32) k_batch_pupdate<F32><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, gate, restart);
        else k_batch_pupdate<F16><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, gate, restart);
        cudaError_t r = cudaGetLastError();
        if (r == cudaSuccess) r = finish(BLA, FIN_ROLL, gate, q);
        return r;
    };
    auto iteration = [&](cudaStream_t q) {
        cudaError_t r = bhop(B.P, B.recon_lo, B.lo, SY, 1, R_P, R_T, -1, coef_qtm_a_scaled(kappa, mut), BH_PLAIN, 1, q);
        if (r == cudaSuccess) r = bhop(B.P, B.recon_lo, B.lo, SY, 0, R_T, R_Q, R_P, coef_qtm_b_unit(mut), BH_NORM, 1, q);
        if (r == cudaSuccess) r = finish(hop_tile(B.lo), FIN_PAP, 1, q);
        if (r == cudaSuccess) r = bhop(B.P, B.recon_lo, B.lo, SY, 1, R_Q, R_T, -1, coef_qtm_a_scaled(kappa, -mut), BH_PLAIN, 1, q);
        // the last hop of Q^dag Q p applies y += alpha p, r -= alpha Ap itself (Ap is not stored)
        if (r == cudaSuccess) r = bhop(B.P, B.recon_lo, B.lo, SY, 0, R_T, -1, R_Q, coef_qtm_b_unit(-mut), BH_UPDATE, 1, q);
        if (r == cudaSuccess) r = finish(hop_tile(B.lo), FIN_RR_UPDATE, 1, q);
        // reliable update where due: x += y, r = b - Q^dag Q x in FP64
        if (r == cudaSuccess) {
            if (B.PY == F64) k_batch_accum<F64><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, 2);
            else k_batch_accum<F32><<<G, BLA, 0, q>>>(SY, I0, nsys, NI, 2);
            r = cudaGetLastError();
        }
        if (r == cudaSuccess) r = qdagq_hi(2, q);
        if (r == cudaSuccess) r = residual(2, q);
        if (r == cudaSuccess) r = pupdate(1, 0, q);
        return r;
    };

    // setup: |b|^2, r = b - Q^dag Q x, p = r, y = 0
    k_batch_norm<<<G, BLA, 0, s>>>(SY, I0, nsys, NI, R_B);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = finish(BLA, FIN_BB, 0, s);
    if (e == cudaSuccess) e = qdagq_hi(0, s);
    if (e == cudaSuccess) e = residual(0, s);
    if (e == cudaSuccess) e = pupdate(0, 1, s);
    if (e == cudaSuccess) {
        if (B.PY == F64) k_batch_zero<F64><<<G, BLA, 0, s>>>(SY, I0, nsys, NI, R_Y);
        else k_batch_zero<F32><<<G, BLA, 0, s>>>(SY, I0, nsys, NI, R_Y);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bcuda(ctx, e, "tm_cg_QdagQ_batch: setup launches");

    const int K = prm->reliable_every;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    if (prm->use_graph) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaSuccess;
            for (int j = 0; j < K && e1 == cudaSuccess; ++j) e1 = iteration(cap);
            e = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            if (exec) cudaGraphExecDestroy(exec);
            if (cap) cudaStreamDestroy(cap);
            return bcuda(ctx, e, "tm_cg_QdagQ_batch: graph capture");
        }
    }

    int stalled = 0;
    for (;;) {
        for (int k = 0; k < nsys && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(&hsc[k], hs[k].s, sizeof(CgScalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        bool all_done = true;
        for (auto &h : hsc) all_done = all_done && (h.done || h.status != TM_OK);
        if (all_done) break;
        int before = 0;
        for (auto &h : hsc) before += h.iters;
        e = exec ? cudaGraphLaunch(exec, s) : cudaSuccess;
        for (int j = 0; !exec && j < K && e == cudaSuccess; ++j) e = iteration(s);
        if (e != cudaSuccess) break;
        for (int k = 0; k < nsys && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(&hsc[k], hs[k].s, sizeof(CgScalars), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        int after = 0;
        for (auto &h : hsc) after += h.iters;
        stalled = after == before ? stalled + 1 : 0;
        if (stalled >= 2) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) return bcuda(ctx, e, "tm_cg_QdagQ_batch: iteration");

    tm_status result = TM_OK;
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    for (int pos = 0; pos < nsys; ++pos) {
        const CgScalars &h = hsc[pos];
        tm_cg_info inf{};
        const double target = h.tol2 * h.bb;
        tm_status r = TM_OK;
        if (h.status != TM_OK || !std::isfinite(h.rr_true)) r = TM_ERR_NONFINITE;
        else if (h.rr_true > target) r = TM_ERR_NOT_CONVERGED;
        inf.iters = h.iters;
        inf.reliable_updates = h.nreliable;
        inf.true_relres = h.bb > 0 ? std::sqrt(h.rr_true / h.bb) : 0.0;
        inf.seconds = secs;
        inf.status = r;
        if (info) info[B.order[pos]] = inf;
        if (r == TM_ERR_NONFINITE) result = r;
        else if (r == TM_ERR_NOT_CONVERGED && result == TM_OK) result = r;
    }
    if (result != TM_OK) ctx->err = result == TM_ERR_NONFINITE ? "tm_cg_QdagQ_batch: non-finite residual"
                                                               : "tm_cg_QdagQ_batch: maxiter reached";
    return result;
}
