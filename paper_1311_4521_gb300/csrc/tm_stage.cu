// tm_stage.cu -- host side of the staged batched hop (tm_stage.cuh): the
// site-complete link copy of a gauge handle and the tensor maps that
// describe fields and links to the Tensor Memory Accelerator.
#include <cudaTypedefs.h>

#include <cstring>
#include <string>
#include <vector>

#include "tm_stage.cuh"
#include "tm_stage_host.h"

namespace twm {

namespace {

// For parity p and site i the 8 links the hop of that site multiplies:
// U_mu(x) (direction mu, storage block 4p + mu) and U_mu(x - mu) (block
// 4(1-p) + mu at the backward neighbour), as blocks 8p + mu and 8p + 4 + mu.
template <class V, int NCH>
__global__ void k_links8(Geom g, const V *__restrict__ links, V *__restrict__ out)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = int(blockIdx.y);
    if (i >= g.vh) return;
    Nbrs n;
    neighbours(g, p, i, n);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            out[(size_t(8 * p + mu) * NCH + c) * g.vh + i] = links[(size_t(4 * p + mu) * NCH + c) * g.vh + i];
            out[(size_t(8 * p + 4 + mu) * NCH + c) * g.vh + i] =
                links[(size_t(4 * (1 - p) + mu) * NCH + c) * g.vh + n.bwd[mu]];
        }
}

// The same for 12-real FP32 storage, written with all 18 reals (row 2 rebuilt once here).
__global__ void k_links8_expand(Geom g, const float4 *__restrict__ links, float2 *__restrict__ out)
{
    using L12 = LinkIO<F32, 12>;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = int(blockIdx.y);
    if (i >= g.vh) return;
    Nbrs n;
    neighbours(g, p, i, n);
    for (int d = 0; d < 8; ++d) {
        const int mu = d & 3;
        const int blk = d < 4 ? 4 * p + mu : 4 * (1 - p) + mu;
        Link<float> u;
        L12::load(links + size_t(blk) * 3 * g.vh, g.vh, d < 4 ? i : n.bwd[mu], u);
        for (int k = 0; k < 9; ++k)
            out[(size_t(8 * p + d) * 9 + k) * g.vh + i] = make_float2(u[k / 3][k % 3].re, u[k / 3][k % 3].im);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 lookup_encode()
{
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = lookup_encode();   // thread-safe once
    return fn;
}

// A tensor map of `rank` dimensions over 8-byte (u64) or 4-byte (f32)
// elements; dims innermost first, strides in bytes of dimensions 1..rank-1.
bool encode(CUtensorMap &m, bool u64, int rank, const void *base, const cuuint64_t *dims, const cuuint64_t *strides,
            const cuuint32_t *box)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(&m, u64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, cuuint32_t(rank),
                          const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Box extents (x in half-sites, y, z, t) of the five shapes.
void shape_box(int sh, cuuint32_t &bx, cuuint32_t &by, cuuint32_t &bz, cuuint32_t &bt)
{
    bx = sh == SH_X ? 1 : SBX;
    by = sh == SH_Y ? 1 : 2;
    bz = sh == SH_Z ? 1 : 2;
    bt = sh == SH_T ? 1 : 2;
}

}  // namespace

bool stage_supported(int prec, int recon)
{
    return (prec == F32 && (recon == 12 || recon == 18)) || (prec == F16 && recon == 12);
}

bool stage_geometry_ok(const Geom &g) { return g.hx % SBX == 0 && g.ly % 2 == 0 && g.lz % 2 == 0 && g.lt % 2 == 0; }

bool stage_available() { return encode_fn() != nullptr; }

#ifndef TM_STAGE_ZBLOCK
#define TM_STAGE_ZBLOCK 128   // boxes per time layer pair of a z block
#endif

int stage_zblock(const Geom &g)
{
    const int plane = (g.hx / SBX) * (g.ly / 2), nbz = g.lz / 2;
    int best = 1;
    for (int b = 1; b <= nbz; ++b)
        if (nbz % b == 0 && plane * b <= TM_STAGE_ZBLOCK) best = b;
    return best;
}

cudaError_t stage_links8(const tm_gauge *U, cudaStream_t s)
{
    if (U->links8) return cudaSuccess;
    void *p = nullptr;
    const Geom &g = U->geom;
    const size_t bytes = U->prec == F32 ? size_t(16) * 9 * 8 * g.vh : 2 * U->bytes;   // FP32: 18 reals per link
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.vh + 255) / 256, 2);
    if (U->prec == F32 && U->recon == 12)
        k_links8_expand<<<grid, 256, 0, s>>>(g, static_cast<const float4 *>(U->links), static_cast<float2 *>(p));
    else if (U->prec == F32 && U->recon == 18)
        k_links8<float2, 9><<<grid, 256, 0, s>>>(g, static_cast<const float2 *>(U->links), static_cast<float2 *>(p));
    else if (U->prec == F16 && U->recon == 12)
        k_links8<uint2, 3><<<grid, 256, 0, s>>>(g, static_cast<const uint2 *>(U->links), static_cast<uint2 *>(p));
    else {
        cudaFree(p);
        return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    // complete before the handle publishes it: later calls may use it from any stream
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(p);
        return e;
    }
    U->links8 = p;
    return cudaSuccess;
}

bool stage_field_maps(int prec, const Geom &g, const void *field, CUtensorMap *maps)
{
    const cuuint64_t hx = cuuint64_t(g.hx), ly = cuuint64_t(g.ly), lz = cuuint64_t(g.lz), lt = cuuint64_t(g.lt);
    const int ch = prec == F16 ? 3 : 6;
    const cuuint64_t dims[5] = {2 * hx, ly, lz, lt, cuuint64_t(ch)};
    const cuuint64_t str[4] = {hx * 16, hx * ly * 16, hx * ly * lz * 16, cuuint64_t(g.vh) * 16};
    for (int sh = 0; sh < NSH; ++sh) {
        cuuint32_t bx, by, bz, bt;
        shape_box(sh, bx, by, bz, bt);
        const cuuint32_t box[5] = {2 * bx, by, bz, bt, cuuint32_t(ch)};
        if (!encode(maps[sh], true, 5, field, dims, str, box)) return false;
    }
    if (prec == F16) {   // the site norms: one float per site after the three component arrays
        const char *nb = static_cast<const char *>(field) + size_t(48) * g.vh;
        const cuuint64_t nd[4] = {hx, ly, lz, lt};
        const cuuint64_t ns[3] = {hx * 4, hx * ly * 4, hx * ly * lz * 4};
        for (int sh = 0; sh < NSH; ++sh) {
            cuuint32_t bx, by, bz, bt;
            shape_box(sh, bx, by, bz, bt);
            const cuuint32_t box[4] = {sh == SH_X ? 4u : bx, by, bz, bt};
            if (!encode(maps[NSH + sh], false, 4, nb, nd, ns, box)) return false;
        }
    }
    return true;
}

bool stage_link_map(const tm_gauge *U, CUtensorMap &m)
{
    const Geom &g = U->geom;
    const int recon = U->prec == F32 ? 18 : U->recon;   // the FP32 copy holds 18 reals per link
    const int nch = link_nchunk(U->prec, recon);
    const cuuint64_t w = cuuint64_t(link_chunk_bytes(U->prec, recon) / 8);
    const cuuint64_t hx = cuuint64_t(g.hx), ly = cuuint64_t(g.ly), lz = cuuint64_t(g.lz), lt = cuuint64_t(g.lt);
    const cuuint64_t dims[5] = {w * hx, ly, lz, lt, cuuint64_t(16 * nch)};
    const cuuint64_t str[4] = {w * hx * 8, w * hx * ly * 8, w * hx * ly * lz * 8, cuuint64_t(g.vh) * w * 8};
    const cuuint32_t box[5] = {cuuint32_t(w * SBX), 2, 2, 2, cuuint32_t(8 * nch)};
    return U->links8 && encode(m, true, 5, U->links8, dims, str, box);
}

namespace {

// One thread waits on a barrier that nothing arrives at: the wait runs out
// after its limit and records that in *status (the path every staged-hop
// wait takes when a copy never completes).
__global__ void k_wait_selftest(int *status)
{
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) (void)mbar_wait(b, 0, status);
}

}  // namespace

}  // namespace twm

using namespace twm;

extern "C" tm_status tm_ctx_selftest_wait(tm_ctx *ctx, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!ctx->dev_status) {
        e = cudaMalloc(&ctx->dev_status, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), s);
        else ctx->dev_status = nullptr;
    }
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, s>>>(ctx->dev_status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_ctx_selftest_wait: ") + cudaGetErrorString(e));
    return TM_OK;
}
