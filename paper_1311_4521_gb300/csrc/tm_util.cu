// tm_util.cu -- measurement and field utilities of the C ABI: the FMA
// throughput probe that gives the FP64 (and FP32) arithmetic peak the
// operator is measured against, a deterministic inner product of packed
// fields, and an in-place scale of complex arrays by a device scalar.
#include <cstring>
#include <string>

#include "tm_internal.h"

using namespace twm;

namespace {

// Sink of the probe: written only if the chains reach a value they cannot
// reach, so the compiler keeps every FMA.
__device__ double g_probe_sink;
// The multiplier and addend of the chains, read from device memory into
// registers once per thread.  As kernel parameters (constant-bank operands)
// they were measured to hold FP64 FMA issue at 1.68 of the 2 lanes per SM
// and clock that register operands reach on GB300, which would understate
// the peak.
__device__ double g_probe_f64[2] = {0.9999999, 1e-7};
__device__ float g_probe_f32[2] = {0.9999f, 1e-4f};

constexpr int kProbeChains = 8;     // independent FMA chains per thread
constexpr int kProbeThreads = 256;

// x <- x a + b on kProbeChains independent chains for `iters` iterations:
// 2 flop per FMA.  a < 1 and b > 0 keep every value near b / (1 - a) = 1,
// away from overflow and subnormals.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, const T *ab)
{
    const T a = ab[0], b = ab[1];
    T x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = T(threadIdx.x * 1e-6) + T(k);
#pragma unroll 4
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], a, b);
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    if (s == T(-12345.0)) g_probe_sink = double(s);
}

// Inner product <a, b> = sum over sites and components of conj(a) b, FP64
// accumulation.  Block k sums sites k, k + grid, ... (per thread, then in a
// fixed tree), so the result depends only on the field size and the grid,
// never on scheduling.
constexpr int kDotThreads = 256;

template <int P>
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(unsigned vh, const void *__restrict__ a,
                                                              const void *__restrict__ b, double2 *partial)
{
    using R = typename SpinorIO<P>::R;
    __shared__ double2 red[kDotThreads];
    double re = 0.0, im = 0.0;
    for (unsigned i = blockIdx.x * kDotThreads + threadIdx.x; i < vh; i += gridDim.x * kDotThreads) {
        Spinor<R> x, y;
        SpinorIO<P>::load(a, vh, i, x);
        SpinorIO<P>::load(b, vh, i, y);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double xr = double(x[s][c].re), xi = double(x[s][c].im);
                const double yr = double(y[s][c].re), yi = double(y[s][c].im);
                re += xr * yr + xi * yi;
                im += xr * yi - xi * yr;
            }
    }
    red[threadIdx.x] = make_double2(re, im);
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x].x += red[threadIdx.x + w].x;
            red[threadIdx.x].y += red[threadIdx.x + w].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kDotThreads) k_dot_final(int n, const double2 *__restrict__ partial, double *out)
{
    __shared__ double2 red[kDotThreads];
    double re = 0.0, im = 0.0;
    for (int k = threadIdx.x; k < n; k += kDotThreads) {
        re += partial[k].x;
        im += partial[k].y;
    }
    red[threadIdx.x] = make_double2(re, im);
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x].x += red[threadIdx.x + w].x;
            red[threadIdx.x].y += red[threadIdx.x + w].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0].x;
        out[1] = red[0].y;
    }
}

// z[k] <- c * alpha * z[k] for n complex doubles (alpha = *alpha_dev, or 1
// when alpha_dev is null).
__global__ void k_scale_complex(size_t n, double2 *z, const double *alpha_dev, double c)
{
    const double f = c * (alpha_dev ? *alpha_dev : 1.0);
    for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n; k += size_t(gridDim.x) * blockDim.x) {
        double2 v = z[k];
        z[k] = make_double2(f * v.x, f * v.y);
    }
}

bool valid_prec(int p) { return p == TM_F64 || p == TM_F32 || p == TM_F16 || p == TM_F64X; }

}  // namespace

extern "C" {

tm_status tm_probe_fma(tm_ctx *ctx, int prec, double *tflops, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!tflops) return tm_fail(ctx, TM_ERR_ARG, "tm_probe_fma: null result pointer");
    if (prec != TM_F64 && prec != TM_F32) return tm_fail(ctx, TM_ERR_ARG, "tm_probe_fma: prec must be TM_F64 or TM_F32");
    cudaStream_t s = (cudaStream_t)stream;
    // 8 CTAs of 256 threads per SM (64 warps: every scheduler has 16 warps
    // of 8 independent chains to hide the FMA latency).  Iterations sized
    // for about 10 ms at the nominal rates (FP64 ~1.3, FP32 ~80 TFLOP/s).
    const unsigned grid = unsigned(ctx->sm_count > 0 ? ctx->sm_count : 1) * 8u;
    const int iters = prec == TM_F64 ? 2048 : 131072;
    const double *ab64 = nullptr;
    const float *ab32 = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&ab64, g_probe_f64);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ab32, g_probe_f32);
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_probe_fma: ") + cudaGetErrorString(e));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best_ms = 1e30;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first launch warms up
        e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) break;
        if (prec == TM_F64) k_fma_probe<double><<<grid, kProbeThreads, 0, s>>>(iters, ab64);
        else k_fma_probe<float><<<grid, kProbeThreads, 0, s>>>(iters, ab32);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_probe_fma: ") + cudaGetErrorString(e));
    const double flops = double(grid) * kProbeThreads * double(iters) * kProbeChains * 2.0;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return TM_OK;
}

tm_status tm_spinor_dot(tm_ctx *ctx, long vh, const void *a_dev, const void *b_dev, int prec, double *out_dev,
                        void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (vh < 0 || vh >= (1L << 31)) return tm_fail(ctx, TM_ERR_ARG, "tm_spinor_dot: bad site count");
    if (!valid_prec(prec)) return tm_fail(ctx, TM_ERR_ARG, "tm_spinor_dot: bad precision");
    if (!out_dev || (reinterpret_cast<uintptr_t>(out_dev) & 7u))
        return tm_fail(ctx, TM_ERR_ARG, "tm_spinor_dot: null or misaligned result pointer");
    if (vh > 0 && (bad_ptr(a_dev) || bad_ptr(b_dev))) return tm_fail(ctx, TM_ERR_ARG, "tm_spinor_dot: null or misaligned pointer");
    const int grid = 2 * (ctx->sm_count > 0 ? ctx->sm_count : 1);
    void *part = nullptr;
    tm_status st = tm_ctx_reduce_buffer(ctx, size_t(grid) * sizeof(double2), &part);
    if (st != TM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double2 *p = static_cast<double2 *>(part);
    const unsigned n = unsigned(vh);
    if (prec == TM_F64) k_dot_partial<F64><<<grid, kDotThreads, 0, s>>>(n, a_dev, b_dev, p);
    else if (prec == TM_F64X) k_dot_partial<F64X><<<grid, kDotThreads, 0, s>>>(n, a_dev, b_dev, p);
    else if (prec == TM_F32) k_dot_partial<F32><<<grid, kDotThreads, 0, s>>>(n, a_dev, b_dev, p);
    else k_dot_partial<F16><<<grid, kDotThreads, 0, s>>>(n, a_dev, b_dev, p);
    k_dot_final<<<1, kDotThreads, 0, s>>>(grid, p, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_spinor_dot: ") + cudaGetErrorString(e));
    return TM_OK;
}

tm_status tm_scale_complex(tm_ctx *ctx, size_t n, double *z_dev, const double *alpha_dev, double c, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (n == 0) return TM_OK;
    if (bad_ptr(z_dev)) return tm_fail(ctx, TM_ERR_ARG, "tm_scale_complex: null or misaligned pointer");
    if (alpha_dev && (reinterpret_cast<uintptr_t>(alpha_dev) & 7u))
        return tm_fail(ctx, TM_ERR_ARG, "tm_scale_complex: misaligned scalar pointer");
    const unsigned grid = unsigned(ctx->sm_count > 0 ? ctx->sm_count : 1) * 4u;
    k_scale_complex<<<grid, 256, 0, (cudaStream_t)stream>>>(n, reinterpret_cast<double2 *>(z_dev), alpha_dev, c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_scale_complex: ") + cudaGetErrorString(e));
    return TM_OK;
}

size_t tm_ctx_device_bytes(const tm_ctx *ctx)
{
    if (!ctx) return 0;
    return ctx->scratch_bytes + ctx->ws_bytes + ctx->stage_bytes + ctx->bq_bytes + ctx->red_bytes;
}

}  // extern "C"
