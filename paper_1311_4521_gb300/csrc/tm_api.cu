// tm_api.cu -- the C ABI of include/tmhop.h: contexts, gauge handles,
// packed fields, the hopping matrix and Q_tm.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "tm_internal.h"

using namespace twm;

namespace {

tm_status fail(tm_ctx *ctx, tm_status st, const char *fmt, const char *detail = "")
{
    if (ctx) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, detail);
        ctx->err = buf;
    }
    return st;
}

tm_status cuda_fail(tm_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    return TM_ERR_CUDA;
}

#define TM_CUDA(ctx, call)                                     \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

bool valid_prec(int p) { return p == TM_F64 || p == TM_F32 || p == TM_F16 || p == TM_F64X; }

}  // namespace

tm_status tm_ctx_scratch(tm_ctx *ctx, size_t bytes, void **ptr)
{
    if (ctx->scratch_bytes < bytes) {
        if (ctx->scratch) {
            cudaError_t e = cudaFree(ctx->scratch);
            ctx->scratch = nullptr;
            ctx->scratch_bytes = 0;
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(scratch)");
        }
        TM_CUDA(ctx, cudaMalloc(&ctx->scratch, bytes));
        ctx->scratch_bytes = bytes;
    }
    *ptr = ctx->scratch;
    return TM_OK;
}

tm_status tm_ctx_reduce_buffer(tm_ctx *ctx, size_t bytes, void **ptr)
{
    if (ctx->red_bytes < bytes) {
        if (ctx->red) {
            cudaError_t e = cudaFree(ctx->red);
            ctx->red = nullptr;
            ctx->red_bytes = 0;
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(reduce buffer)");
        }
        TM_CUDA(ctx, cudaMalloc(&ctx->red, bytes));
        ctx->red_bytes = bytes;
    }
    *ptr = ctx->red;
    return TM_OK;
}

extern "C" {

const char *tm_status_string(tm_status s)
{
    switch (s) {
    case TM_OK: return "ok";
    case TM_ERR_ARG: return "invalid argument";
    case TM_ERR_CUDA: return "CUDA error";
    case TM_ERR_NOT_CONVERGED: return "solver did not converge";
    case TM_ERR_NONFINITE: return "non-finite residual";
    case TM_ERR_TIMEOUT: return "device wait timed out";
    case TM_ERR_UNSUPPORTED: return "unsupported combination";
    }
    return "unknown status";
}

tm_status tm_ctx_create(tm_ctx **out, int device)
{
    if (!out) return TM_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TM_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return TM_ERR_CUDA;
    tm_ctx *ctx = new tm_ctx;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (const char *cache = getenv("TMHOP_TUNE_CACHE")) ctx->tune_cache = cache;
    *out = ctx;
    return TM_OK;
}

void tm_ctx_destroy(tm_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->bq) cudaFree(ctx->bq);
    if (ctx->red) cudaFree(ctx->red);
    if (ctx->dev_status) cudaFree(ctx->dev_status);
    if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
    if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
    delete ctx;
}

const char *tm_last_error(const tm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tm_status tm_ctx_check(tm_ctx *ctx)
{
    if (!ctx) return TM_ERR_ARG;
    if (!ctx->dev_status) return TM_OK;
    int v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemset(ctx->dev_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tm_ctx_check");
    if (v) return fail(ctx, TM_ERR_CUDA, "tm_ctx_check: a bounded wait of the staged batched hop ran out");
    return TM_OK;
}

tm_status tm_ctx_set_autotune(tm_ctx *ctx, int on)
{
    if (!ctx) return TM_ERR_ARG;
    ctx->autotune = on ? 1 : 0;
    return TM_OK;
}

size_t tm_ctx_tune_report(const tm_ctx *ctx, char *buf, size_t size)
{
    if (!ctx) return 0;
    std::string rep;
    for (const auto &kv : ctx->tuned) {
        char line[256];
        auto ms = ctx->tuned_ms.find(kv.first);
        auto band = ctx->tuned_band.find(kv.first);
        snprintf(line, sizeof line, "%s nrb=%d cap=%u ms3=%.4f band=%d\n", kv.first.c_str(), kv.second.first,
                 kv.second.second, ms == ctx->tuned_ms.end() ? 0.0 : double(ms->second),
                 band == ctx->tuned_band.end() ? 1 : band->second);
        rep += line;
    }
    for (const auto &kv : ctx->tuned_maps) rep += "hop/" + kv.first + " " + kv.second + "\n";
    if (buf && size > 0) {
        const size_t n = rep.size() < size - 1 ? rep.size() : size - 1;
        memcpy(buf, rep.data(), n);
        buf[n] = '\0';
    }
    return rep.size() + 1;
}

tm_status tm_ctx_trace(tm_ctx *ctx, void *const *events, int nevents)
{
    if (!ctx) return TM_ERR_ARG;
    ctx->trace.clear();
    if (!events) return TM_OK;
    if (nevents < 3) return fail(ctx, TM_ERR_ARG, "tm_ctx_trace: need at least 3 events");
    for (int k = 0; k < nevents; ++k) {
        if (!events[k]) {
            ctx->trace.clear();
            return fail(ctx, TM_ERR_ARG, "tm_ctx_trace: null event");
        }
        ctx->trace.push_back(static_cast<cudaEvent_t>(events[k]));
    }
    return TM_OK;
}

size_t tm_spinor_bytes(long vh, int prec)
{
    if (vh < 0 || !valid_prec(prec)) return 0;
    return spinor_bytes(unsigned(vh), prec);
}

tm_status tm_spinor_pack(tm_ctx *ctx, long vh, const double *in_dev, void *out_dev, int prec, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (vh < 0 || vh >= (1L << 31)) return fail(ctx, TM_ERR_ARG, "tm_spinor_pack: bad site count");
    if (!valid_prec(prec)) return fail(ctx, TM_ERR_ARG, "tm_spinor_pack: bad precision");
    if (vh > 0 && (bad_ptr(in_dev) || bad_ptr(out_dev))) return fail(ctx, TM_ERR_ARG, "tm_spinor_pack: null or misaligned pointer");
    TM_CUDA(ctx, launch_pack_spinor(unsigned(vh), prec, in_dev, out_dev, (cudaStream_t)stream));
    return TM_OK;
}

tm_status tm_spinor_unpack(tm_ctx *ctx, long vh, const void *in_dev, double *out_dev, int prec, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (vh < 0 || vh >= (1L << 31)) return fail(ctx, TM_ERR_ARG, "tm_spinor_unpack: bad site count");
    if (!valid_prec(prec)) return fail(ctx, TM_ERR_ARG, "tm_spinor_unpack: bad precision");
    if (vh > 0 && (bad_ptr(in_dev) || bad_ptr(out_dev))) return fail(ctx, TM_ERR_ARG, "tm_spinor_unpack: null or misaligned pointer");
    TM_CUDA(ctx, launch_unpack_spinor(unsigned(vh), prec, in_dev, out_dev, (cudaStream_t)stream));
    return TM_OK;
}

tm_status tm_gauge_create(tm_ctx *ctx, const int dims[4], const double *U_dev, int prec, int reconstruct,
                          const int bc[4], void *stream, tm_gauge **out)
{
    if (!ctx) return TM_ERR_ARG;
    if (!out || !dims || bad_ptr(U_dev) || !bc) return fail(ctx, TM_ERR_ARG, "tm_gauge_create: null or misaligned pointer");
    *out = nullptr;
    if (!valid_prec(prec)) return fail(ctx, TM_ERR_ARG, "tm_gauge_create: bad precision");
    if (reconstruct != 12 && reconstruct != 18) return fail(ctx, TM_ERR_ARG, "tm_gauge_create: reconstruct must be 12 or 18");
    if (prec == TM_F16 && reconstruct != 12) return fail(ctx, TM_ERR_UNSUPPORTED, "tm_gauge_create: TM_F16 links need reconstruct 12");
    for (int m = 0; m < 4; ++m)
        if (bc[m] != 1 && bc[m] != -1) return fail(ctx, TM_ERR_ARG, "tm_gauge_create: bc entries must be +1 or -1");
    Geom g;
    if (!make_geom(dims, bc, g)) return fail(ctx, TM_ERR_ARG, "tm_gauge_create: extents must be even, >= 2, volume < 2^31");
    tm_gauge *h = new tm_gauge;
    h->ctx = ctx;
    memcpy(h->dims, dims, sizeof h->dims);
    memcpy(h->bc, bc, sizeof h->bc);
    h->prec = prec;
    h->recon = reconstruct;
    h->geom = g;
    h->bytes = size_t(8) * link_nchunk(prec, reconstruct) * link_chunk_bytes(prec, reconstruct) * g.vh;
    cudaError_t e = cudaMalloc(&h->links, h->bytes);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(ctx, e, "cudaMalloc(links)");
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = launch_pack_gauge(g, prec, reconstruct, U_dev, h->links, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(h->links);
        delete h;
        return cuda_fail(ctx, e, "tm_gauge_create: pack");
    }
    tm_apply_cached_map(ctx, h);
    *out = h;
    return TM_OK;
}

void tm_gauge_destroy(tm_gauge *g)
{
    if (!g) return;
    if (g->links) cudaFree(g->links);
    if (g->links8) cudaFree(g->links8);
    delete g;
}

size_t tm_gauge_bytes(const tm_gauge *g) { return g ? g->bytes : 0; }

tm_status tm_hopping_eo(tm_ctx *ctx, const tm_gauge *U, void *out_dev, const void *in_dev, int dir, int dagger,
                        void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(out_dev) || bad_ptr(in_dev)) return fail(ctx, TM_ERR_ARG, "tm_hopping_eo: null or misaligned pointer");
    if (dir != TM_EO && dir != TM_OE) return fail(ctx, TM_ERR_ARG, "tm_hopping_eo: dir must be TM_EO or TM_OE");
    if (out_dev == in_dev) return fail(ctx, TM_ERR_ARG, "tm_hopping_eo: out and in must not overlap");
    TM_CUDA(ctx, launch_hop(U->geom, U->prec, U->recon, dagger != 0, dir, U->links, in_dev, out_dev, nullptr,
                            coef_plain(), (cudaStream_t)stream, U->map));
    return TM_OK;
}

tm_status tm_Qtm(tm_ctx *ctx, const tm_gauge *U, void *out_e_dev, const void *in_e_dev, double kappa, double mu,
                 int sign, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(out_e_dev) || bad_ptr(in_e_dev)) return fail(ctx, TM_ERR_ARG, "tm_Qtm: null or misaligned pointer");
    if (sign != 1 && sign != -1) return fail(ctx, TM_ERR_ARG, "tm_Qtm: sign must be +1 or -1");
    if (out_e_dev == in_e_dev) return fail(ctx, TM_ERR_ARG, "tm_Qtm: out and in must not overlap");
    void *tmp = nullptr;
    tm_status st = tm_ctx_scratch(ctx, spinor_bytes(U->geom.vh, U->prec), &tmp);
    if (st != TM_OK) return st;
    double mut = 2.0 * kappa * mu * sign;
    cudaStream_t s = (cudaStream_t)stream;
    tm_trace_mark(ctx, 0, s);
    TM_CUDA(ctx, launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, in_e_dev, tmp, nullptr,
                            coef_qtm_a_scaled(kappa, mut), s, U->map));
    tm_trace_mark(ctx, 1, s);
    TM_CUDA(ctx, launch_hop(U->geom, U->prec, U->recon, false, TM_EO, U->links, tmp, out_e_dev, in_e_dev,
                            coef_qtm_b_unit(mut), s, U->map));
    tm_trace_mark(ctx, 2, s);
    return TM_OK;
}

}  // extern "C"
