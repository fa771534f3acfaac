// tm_host.cu -- Q_tm on spinor fields that live in host memory.
//
// A caller whose fields are in host memory (a host-side application, a
// service that receives right-hand sides from elsewhere) pays, per
// application, a host-to-device copy of the input, the operator and a
// device-to-host copy of the result.  tm_Qtm_host takes a list of such
// fields and pipelines them through two device staging slots: while the
// operator of field k runs on the compute stream, field k+1 is copied in
// and packed on one copy stream and field k-1 unpacked and copied out on
// another.  For FP64 handles the operator's two launches read the input
// and write the result in the caller's canonical layout directly (the
// component-major packing only pays for itself when a field is used many
// times), so only the copies run beside it; the other formats pack and
// unpack on the copy streams.  Every copy is one cudaMemcpyAsync of one
// contiguous field.
#include <set>
#include <string>

#include "tm_internal.h"

using namespace twm;

namespace {

tm_status grow_stage(tm_ctx *ctx, size_t bytes)
{
    if (ctx->stage_bytes >= bytes) return TM_OK;
    if (ctx->stage) {
        cudaError_t e = cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("cudaFree(stage): ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&ctx->stage, bytes);
    if (e != cudaSuccess) {
        ctx->stage = nullptr;
        return tm_fail(ctx, TM_ERR_CUDA, std::string("cudaMalloc(stage): ") + cudaGetErrorString(e));
    }
    ctx->stage_bytes = bytes;
    return TM_OK;
}

// The events of one call, per slot: "packed" (copy-in stream -> compute),
// "multiplied" (compute -> both copy streams), "unpacked" (copy-out stream
// -> compute).
struct SlotEvents {
    cudaEvent_t packed[2] = {}, multiplied[2] = {}, unpacked[2] = {};
    cudaError_t create()
    {
        for (int k = 0; k < 2; ++k)
            for (cudaEvent_t *e : {&packed[k], &multiplied[k], &unpacked[k]}) {
                cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
                if (r != cudaSuccess) return r;
            }
        return cudaSuccess;
    }
    ~SlotEvents()
    {
        for (int k = 0; k < 2; ++k)
            for (cudaEvent_t e : {packed[k], multiplied[k], unpacked[k]})
                if (e) cudaEventDestroy(e);
    }
};

}  // namespace

extern "C" tm_status tm_Qtm_host(tm_ctx *ctx, const tm_gauge *U, int n, double *const *out_host,
                                 const double *const *in_host, double kappa, double mu, int sign, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || n < 1 || !out_host || !in_host) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_host: bad arguments");
    if (sign != 1 && sign != -1) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_host: sign must be +1 or -1");
    std::set<const void *> ins;
    for (int k = 0; k < n; ++k) {
        if (!out_host[k] || !in_host[k]) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_host: null field pointer");
        ins.insert(in_host[k]);
    }
    for (int k = 0; k < n; ++k)
        if (ins.count(out_host[k])) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_host: an output buffer is also an input");

    const unsigned vh = U->geom.vh;
    const size_t cb = size_t(vh) * 24 * sizeof(double);  // canonical complex double [Vh][4][3]
    const size_t cba = align256(cb), pba = align256(spinor_bytes(vh, U->prec));
    tm_status st = grow_stage(ctx, 2 * (2 * cba + 2 * pba));
    if (st != TM_OK) return st;
    void *tmp = nullptr;  // tm_Qtm's scratch, grown now so that no call below reallocates it
    st = tm_ctx_scratch(ctx, spinor_bytes(vh, U->prec), &tmp);
    if (st != TM_OK) return st;
    char *base = static_cast<char *>(ctx->stage);
    double *can_in[2], *can_out[2];
    void *p_in[2], *p_out[2];
    for (int k = 0; k < 2; ++k) {
        char *b = base + size_t(k) * (2 * cba + 2 * pba);
        can_in[k] = reinterpret_cast<double *>(b);
        can_out[k] = reinterpret_cast<double *>(b + cba);
        p_in[k] = b + 2 * cba;
        p_out[k] = b + 2 * cba + pba;
    }
    cudaError_t e = cudaSuccess;
    if (!ctx->copy_in) e = cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->copy_out) e = cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking);
    SlotEvents ev;
    if (e == cudaSuccess) e = ev.create();
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_Qtm_host: ") + cudaGetErrorString(e));

    cudaStream_t s = (cudaStream_t)stream, ci = ctx->copy_in, co = ctx->copy_out;
    st = TM_OK;
    if (U->prec == F64) {
        // FP64: the operator reads and writes the canonical staging slots
        // itself (no pack or unpack launches competing with it for the SMs).
        // Events per slot: packed = copied in, unpacked = copied out.
        const double mut = 2.0 * kappa * mu * sign;
        const Coef ka = coef_qtm_a_scaled(kappa, mut), kb = coef_qtm_b_unit(mut);
        for (int k = 0; k < n && e == cudaSuccess; ++k) {
            const int q = k & 1;
            // copy-in stream: once the operator of field k-2 has read this slot, field k
            e = cudaStreamWaitEvent(ci, ev.multiplied[q], 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(can_in[q], in_host[k], cb, cudaMemcpyHostToDevice, ci);
            if (e == cudaSuccess) e = cudaEventRecord(ev.packed[q], ci);
            // compute stream: once field k is in and field k-2's result has left the slot
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev.packed[q], 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev.unpacked[q], 0);
            if (e == cudaSuccess) {
                tm_trace_mark(ctx, 0, s);
                e = launch_qtm_canonical(false, U->geom, U->recon, U->map, U->links, can_in[q], tmp, can_out[q], ka, s);
                tm_trace_mark(ctx, 1, s);
                if (e == cudaSuccess)
                    e = launch_qtm_canonical(true, U->geom, U->recon, U->map, U->links, can_in[q], tmp, can_out[q], kb,
                                             s);
                tm_trace_mark(ctx, 2, s);
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev.multiplied[q], s);
            // copy-out stream: field k back to the host
            if (e == cudaSuccess) e = cudaStreamWaitEvent(co, ev.multiplied[q], 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(out_host[k], can_out[q], cb, cudaMemcpyDeviceToHost, co);
            if (e == cudaSuccess) e = cudaEventRecord(ev.unpacked[q], co);
        }
    }
    for (int k = 0; U->prec != F64 && k < n && e == cudaSuccess && st == TM_OK; ++k) {
        const int q = k & 1;
        // copy-in stream: field k to the device, then (once the operator of
        // field k-2 has read this slot's packed input) its pack
        e = cudaMemcpyAsync(can_in[q], in_host[k], cb, cudaMemcpyHostToDevice, ci);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ci, ev.multiplied[q], 0);
        if (e == cudaSuccess) e = launch_pack_spinor(vh, U->prec, can_in[q], p_in[q], ci);
        if (e == cudaSuccess) e = cudaEventRecord(ev.packed[q], ci);
        // compute stream: the operator, once field k is packed and the unpack
        // of field k-2 has read this slot's packed output
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev.packed[q], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev.unpacked[q], 0);
        if (e == cudaSuccess) st = tm_Qtm(ctx, U, p_out[q], p_in[q], kappa, mu, sign, s);
        if (e == cudaSuccess && st == TM_OK) e = cudaEventRecord(ev.multiplied[q], s);
        // copy-out stream: unpack and copy field k back to the host
        if (e == cudaSuccess && st == TM_OK) e = cudaStreamWaitEvent(co, ev.multiplied[q], 0);
        if (e == cudaSuccess && st == TM_OK) e = launch_unpack_spinor(vh, U->prec, p_out[q], can_out[q], co);
        if (e == cudaSuccess && st == TM_OK) e = cudaEventRecord(ev.unpacked[q], co);
        if (e == cudaSuccess && st == TM_OK) e = cudaMemcpyAsync(out_host[k], can_out[q], cb, cudaMemcpyDeviceToHost, co);
    }
    // drain every stream before the events go away, whatever happened
    cudaError_t e1 = cudaStreamSynchronize(ci);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaError_t e3 = cudaStreamSynchronize(co);
    if (st != TM_OK) return st;
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_Qtm_host: ") + cudaGetErrorString(e));
    return TM_OK;
}
