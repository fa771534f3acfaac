// tm_noalloc.cu -- Q_tm for callers that cannot allocate device memory.
//
// tm_Qtm needs one odd-parity temporary field between its two launches and
// takes it from the context's scratch buffer, which it grows with
// cudaMalloc on first use.  Some callers cannot let a library allocate:
// code running inside a host framework that owns all device memory through
// its own pool and forbids outside cudaMalloc calls, plugins held to a fixed
// memory budget, and latency-critical loops that cannot afford the implicit
// device synchronisation cudaMalloc/cudaFree may cause.  tm_Qtm_noalloc
// gives them the same operator with the temporary held in a statically
// sized device array that the CUDA runtime reserves when it loads this
// library's code onto a device; the call itself allocates nothing.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it.  Nothing in it has to start at zero: launch A writes the
// temporary at every odd site before launch B reads it.  Calls whose work
// overlaps on the GPU (different streams, or different host threads without
// ordering) race on the array and give wrong results.
#include <cstdio>
#include <mutex>

#include "tm_internal.h"

using namespace twm;

namespace {

// The scratch array.  In host code its name is only a stand-in for the
// device symbol, never a device address: kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_qtm_scratch[TM_QTM_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_qtm_scratch on the context's device, looked up once
// per device with that device current (the caller's current device is
// restored afterwards) and kept for the life of the process.  It belongs to
// the device's primary context: a cudaDeviceReset destroys that context and
// with it every allocation of this library (contexts' buffers, gauge
// handles), so after a reset the library is not used again on that device
// and the stale address is never read.
tm_status scratch_address(tm_ctx *ctx, void **addr)
{
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return tm_fail(ctx, TM_ERR_UNSUPPORTED, "tm_Qtm_noalloc: device index out of range");
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[ctx->device]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e == cudaSuccess && cur != ctx->device) e = cudaSetDevice(ctx->device);
        void *p = nullptr;
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_qtm_scratch);
        if (cur >= 0 && cur != ctx->device) {
            cudaError_t e2 = cudaSetDevice(cur);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess)
            return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_Qtm_noalloc: cudaGetSymbolAddress: ") +
                                                      cudaGetErrorString(e));
        g_scratch_addr[ctx->device] = p;
    }
    *addr = g_scratch_addr[ctx->device];
    return TM_OK;
}

}  // namespace

extern "C" tm_status tm_Qtm_noalloc(tm_ctx *ctx, const tm_gauge *U, void *out_e_dev, const void *in_e_dev,
                                    double kappa, double mu, int sign, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || bad_ptr(out_e_dev) || bad_ptr(in_e_dev)) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_noalloc: null or misaligned pointer");
    if (sign != 1 && sign != -1) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_noalloc: sign must be +1 or -1");
    if (out_e_dev == in_e_dev) return tm_fail(ctx, TM_ERR_ARG, "tm_Qtm_noalloc: out and in must not overlap");
    size_t need = spinor_bytes(U->geom.vh, U->prec);
    if (need > size_t(TM_QTM_NOALLOC_MAX_BYTES)) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "tm_Qtm_noalloc: the odd temporary needs %zu bytes, more than the %zu-byte static scratch "
                 "array; use tm_Qtm for this lattice and precision",
                 need, size_t(TM_QTM_NOALLOC_MAX_BYTES));
        return tm_fail(ctx, TM_ERR_ARG, buf);
    }
    void *tmp = nullptr;
    tm_status st = scratch_address(ctx, &tmp);
    if (st != TM_OK) return st;
    double mut = 2.0 * kappa * mu * sign;
    cudaStream_t s = (cudaStream_t)stream;
    tm_trace_mark(ctx, 0, s);
    cudaError_t e = launch_hop(U->geom, U->prec, U->recon, false, TM_OE, U->links, in_e_dev, tmp, nullptr,
                               coef_qtm_a_scaled(kappa, mut), s, 128);
    if (e == cudaSuccess) {
        tm_trace_mark(ctx, 1, s);
        e = launch_hop(U->geom, U->prec, U->recon, false, TM_EO, U->links, tmp, out_e_dev, in_e_dev,
                       coef_qtm_b_unit(mut), s, 128);
    }
    if (e == cudaSuccess) tm_trace_mark(ctx, 2, s);
    if (e != cudaSuccess)
        return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_Qtm_noalloc: launch: ") + cudaGetErrorString(e));
    return TM_OK;
}
