// tm_batch.cuh -- shared definitions of the batched operator and solver:
// the system and group tables, the batched hop kernel and its launchers.
#pragma once

#include <cuda.h>   // CUtensorMap (the staged hop's tensor maps)

#include "tm_cg.cuh"
#include "tm_internal.h"

namespace twm {

enum Role { R_X, R_B, R_R, R_P, R_Q, R_T, R_Y, R_AX, R_THI, R_QHI, R_IN, R_OUT, NROLE };

struct BSys {
    void *f[NROLE];
    double *partials;  // one slot per work tile of the system's lattice
    CgScalars *s;
    unsigned vh;
};

struct BGroup {
    Geom g;
    const void *links;  // gauge storage in the launch's precision
    int nrhs, sys0;     // systems sys0 .. sys0 + nrhs - 1
    unsigned item0;     // first work item of the group
    unsigned ntiles;    // tiles covering the group's Vh sites
    int sbz = 1;        // staged hop: boxes per z block of its traversal order
    int zband = 0;      // gather hops: z planes per band of the tile order (0: lexicographic)
};

// The tile order of the gather hops.  Lexicographic tiles reach a site's t
// neighbours two time slices later; with 12 right-hand sides that is more
// traffic than L2 keeps, and a third of the neighbour reads went to memory
// again.  With bands of zband z planes the order is band, t, tile within the
// band's slab, so the t neighbours are one band slab (a few thousand sites)
// away; only the z neighbours across band edges are read twice.
TM_HD unsigned tile_of(const BGroup &G, unsigned tno, unsigned ts)
{
    if (G.zband == 0) return tno;
    const unsigned plane = unsigned(G.g.hx) * unsigned(G.g.ly);
    const unsigned tpb = plane * unsigned(G.zband) / ts;   // tiles per band slab
    const unsigned per_band = tpb * unsigned(G.g.lt);
    const unsigned band = tno / per_band, rem = tno - band * per_band;
    const unsigned t = rem / tpb, k = rem - t * tpb;
    return (t * unsigned(G.g.lz) + band * unsigned(G.zband)) * plane / ts + k;
}

constexpr int BT = 128;   // threads per CTA of the batched hop
// Resident CTAs per SM the batched hop is compiled for, with one and with two
// right-hand sides per thread (registers per thread <= 65536 / (128 x this)).
#ifndef TM_BATCH_MINB
#define TM_BATCH_MINB 4
#endif
#ifndef TM_BATCH_MINB_RPT2
#define TM_BATCH_MINB_RPT2 4
#endif

// What the batched hop does with its result: store it (PLAIN), store it and
// reduce |out|^2 per (system, tile) (NORM), or, as the last hop of
// Q^dag Q p in the CG, apply y += alpha p, r -= alpha out and reduce |r|^2
// per (system, tile) without storing out (UPDATE).
enum { BH_PLAIN = 0, BH_NORM = 1, BH_UPDATE = 2 };
constexpr int BLA = 256;  // threads per CTA of the batched vector kernels

// Sum of v over the 32 lanes of a warp in a fixed order (valid in lane 0).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// The first work item of every group (or system), staged once per CTA in
// shared memory so that mapping an item to its group is a short binary
// search there instead of a chain of dependent global loads.  Tables longer
// than STAGE_MAX entries stay in global memory.
constexpr int STAGE_MAX = 256;

// Largest k < n with first[k] <= item (first[] strictly increasing, first[0] = 0).
__device__ __forceinline__ int find_first(const unsigned *first, int n, unsigned item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_group(const BGroup *gr, int ng, const unsigned *staged, unsigned item)
{
    if (staged) return find_first(staged, ng, item);
    int gi = 0;
    while (gi + 1 < ng && item >= gr[gi + 1].item0) ++gi;
    return gi;
}


// Arguments of the staged hop (tm_stage.cuh) beyond those of the batched hop.
struct StageArgs {
    const CUtensorMap *smaps = nullptr;  // [system][role][2 * 5]: field boxes, then FP16 norm boxes
    const CUtensorMap *lmaps = nullptr;  // [group]: the group's site-complete links
    int *status = nullptr;               // set to 1 when a wait of the kernel runs out
    unsigned roles = 0;                  // bit r: the maps of hop-input role r are encoded
};

struct HopTable {
    int nrb = 1;            // configuration code: pass width (code % 10; <= 1: no link staging) and
                            // right-hand sides per thread (code / 10 + 1)
    unsigned grid = 0;      // persistent CTAs
    unsigned nitems = 0;
    BGroup *dev = nullptr;  // device copy of the groups
    int ngroups = 0;
    StageArgs sa{};         // tensor maps of the staged hop (configuration code 100)
};

// Launches of the batched hop for one storage format (tm_batch_hop_*.cu).
cudaError_t batch_hop_f64(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                          int mode, int gate, cudaStream_t st);
cudaError_t batch_hop_f64x(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                           int mode, int gate, cudaStream_t st);
cudaError_t batch_hop_f32_12(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                             int mode, int gate, cudaStream_t st);
cudaError_t batch_hop_f32_18(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                             int mode, int gate, cudaStream_t st);
cudaError_t batch_hop_f16(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                          int mode, int gate, cudaStream_t st);

// Configuration codes of the batched hop: code % 10 is the pass width NRB,
// code / 10 + 1 the right-hand sides each thread computes (RPT).
__host__ __device__ constexpr int code_nrb(int code) { return code % 10; }
__host__ __device__ constexpr int code_rpt(int code) { return code / 10 + 1; }

// The output of one site for one system: the epilogue, then either the store
// (and |out|^2 for BH_NORM) or the solver update of BH_UPDATE; returns the
// site's contribution to the system's partial.
template <int P, int MODE>
__device__ __forceinline__ double batch_site_out(const BSys *S, unsigned vh, unsigned i,
                                                 const Spinor<typename SpinorIO<P>::R> &acc, const Coef &k, int rout,
                                                 int rx)
{
    using R = typename SpinorIO<P>::R;
    Spinor<R> o;
    if (rx >= 0) {
        Spinor<R> xs;
        SpinorIO<P>::load(S->f[rx], vh, i, xs);
        epilogue(k, acc, &xs, o);
    } else {
        epilogue(k, acc, static_cast<const Spinor<R> *>(nullptr), o);
    }
    if (MODE == BH_UPDATE) {
        constexpr int PY = P == F16 ? F32 : P;
        using RY = typename SpinorIO<PY>::R;
        const double alpha = S->s->alpha;
        Spinor<R> pv, rv;
        Spinor<RY> yv;
        SpinorIO<P>::load(S->f[R_P], vh, i, pv);
        SpinorIO<P>::load(S->f[R_R], vh, i, rv);
        SpinorIO<PY>::load(S->f[R_Y], vh, i, yv);
        const R a = to_R<R>(alpha);
        const RY ay = to_R<RY>(alpha);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                yv[sp][c].re += ay * RY(pv[sp][c].re);
                yv[sp][c].im += ay * RY(pv[sp][c].im);
                rv[sp][c].re -= a * o[sp][c].re;
                rv[sp][c].im -= a * o[sp][c].im;
            }
        SpinorIO<PY>::store(S->f[R_Y], vh, i, yv);
        SpinorIO<P>::store(S->f[R_R], vh, i, rv);
        return norm2(rv);
    }
    SpinorIO<P>::store(S->f[rout], vh, i, o);
    return MODE == BH_NORM ? norm2(o) : 0.0;
}

// NRB: 1 streams links, items (tile, rhs) with the right-hand side fastest;
// 0 the same with default-cached links (L2 sharing); >= 2 stages the tile's
// links in shared memory and sweeps the right-hand sides NRB at a time.
// RPT = 2: each thread computes two right-hand sides of its site with one
// load of each link (items (tile, pair of rhs) for NRB <= 1; NRB pairs per
// pass otherwise), which doubles the neighbour loads it has in flight.
template <int P, int RECON, int NRB, int MODE, int RPT>
__global__ void __launch_bounds__(BT, RPT == 1 ? TM_BATCH_MINB : TM_BATCH_MINB_RPT2) k_batch_hop(const BGroup *__restrict__ groups, int ngroups, unsigned nitems,
                                                  const BSys *__restrict__ sys, int parity, int rin, int rout, int rx,
                                                  Coef k, int gate)
{
    using L = LinkIO<P, RECON>;
    using V = typename L::V;
    using R = typename SpinorIO<P>::R;
    constexpr int TS = NRB > 1 ? BT / NRB : BT;
    __shared__ V tile[NRB > 1 ? 8 * L::NCHUNK * TS : 1];
    __shared__ unsigned bwd_idx[NRB > 1 ? 4 * TS : 1];
    __shared__ double red[RPT][BT / 32];
    __shared__ unsigned first[STAGE_MAX];
    const unsigned tx = threadIdx.x % TS, ty = threadIdx.x / TS;
    const unsigned *staged = ngroups <= STAGE_MAX ? first : nullptr;
    if (staged) {
        for (int g = threadIdx.x; g < ngroups; g += BT) first[g] = groups[g].item0;
        __syncthreads();
    }

    for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
        const BGroup &G = groups[find_group(groups, ngroups, staged, item)];
        const unsigned rel = item - G.item0;
        const unsigned nsets = (unsigned(G.nrhs) + RPT - 1) / RPT;   // items per tile for NRB <= 1
        const unsigned tno = NRB <= 1 ? rel / nsets : rel;
        const unsigned ptile = tile_of(G, tno, TS);   // the tile's place in the lattice
        const unsigned i = ptile * TS + tx;
        const V *links = static_cast<const V *>(G.links);
        if (NRB > 1) {
            // skip the tile (and its link traffic) when no system of the group is active
            bool any = false;
            for (int r = 0; r < G.nrhs && !any; ++r) any = !gated(sys[G.sys0 + r].s, gate);
            if (!any) continue;   // uniform over the block
            __syncthreads();  // readers of the previous tile are done
            if (ty == 0) {
                unsigned site = ptile * TS + tx;
                if (site < G.g.vh) {
                    Nbrs n;
                    neighbours(G.g, parity, site, n);
                    for (int m = 0; m < 4; ++m) bwd_idx[m * TS + tx] = n.bwd[m];
                }
            }
            __syncthreads();
            for (unsigned e = threadIdx.x; e < 8u * L::NCHUNK * TS; e += BT) {
                const unsigned s = e % TS, dc = e / TS, c = dc % L::NCHUNK, d = dc / L::NCHUNK;
                const unsigned site = ptile * TS + s;
                V v{};
                if (site < G.g.vh) {
                    const unsigned idx = d < 4 ? site : bwd_idx[(d - 4) * TS + s];
                    const unsigned blk = d < 4 ? 4 * parity + d : 4 * (1 - parity) + (d - 4);
                    v = ld_stream(links + (size_t(blk) * L::NCHUNK + c) * G.g.vh + idx);
                }
                tile[e] = v;
            }
            __syncthreads();
        }
        const int passes = NRB <= 1 ? 1 : (G.nrhs + NRB * RPT - 1) / (NRB * RPT);
        for (int q = 0; q < passes; ++q) {
            // right-hand sides r0 + j * step, j < RPT
            const int r0 = NRB <= 1 ? int(rel % nsets) * RPT : q * NRB * RPT + int(ty);
            const int step = NRB <= 1 ? 1 : NRB;
            const BSys *S[RPT];
            bool act[RPT], any = false;
            double nrm[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const int r = r0 + j * step;
                S[j] = r < G.nrhs ? &sys[G.sys0 + r] : nullptr;
                act[j] = S[j] && !gated(S[j]->s, gate);
                any = any || act[j];
                nrm[j] = 0.0;
            }
            if (any && i < G.g.vh) {
                Nbrs n;
                neighbours(G.g, parity, i, n);
                if constexpr (RPT == 1) {
                    Spinor<R> acc;
                    if (NRB > 1) {
                        StagedLinks<P, RECON> src{tile, TS, tx};
                        hop_site_src<P, false>(G.g, n, src, S[0]->f[rin], acc);
                    } else {
                        GlobalLinks<P, RECON, NRB == 1> src{links, G.g.vh, i, parity};
                        hop_site_src<P, false>(G.g, n, src, S[0]->f[rin], acc);
                    }
                    nrm[0] = batch_site_out<P, MODE>(S[0], G.g.vh, i, acc, k, rout, rx);
                } else {
                    // an inactive partner reads the active one's input; its result is dropped
                    const void *in0 = act[0] ? S[0]->f[rin] : S[1]->f[rin];
                    const void *in1 = act[1] ? S[1]->f[rin] : in0;
                    Spinor<R> acc0, acc1;
                    if (NRB > 1) {
                        StagedLinks<P, RECON> src{tile, TS, tx};
                        hop_site_src_pair<P, false>(G.g, n, src, in0, in1, acc0, acc1);
                    } else {
                        GlobalLinks<P, RECON, NRB == 1> src{links, G.g.vh, i, parity};
                        hop_site_src_pair<P, false>(G.g, n, src, in0, in1, acc0, acc1);
                    }
                    if (act[0]) nrm[0] = batch_site_out<P, MODE>(S[0], G.g.vh, i, acc0, k, rout, rx);
                    if (act[1]) nrm[1] = batch_site_out<P, MODE>(S[1], G.g.vh, i, acc1, k, rout, rx);
                }
            }
            if (MODE != BH_PLAIN) {
                // one partial per (system, tile): each warp sums its lanes, then the
                // TS / 32 warps of each right-hand side are added in order
                static_assert(TS % 32 == 0, "a warp must not span two right-hand sides");
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const double ws = warp_sum(nrm[j]);
                    if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = ws;
                }
                __syncthreads();
                if (tx == 0) {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) {
                        if (!act[j]) continue;
                        double sum = 0.0;
                        for (int w = 0; w < TS / 32; ++w) sum += red[j][(ty * TS) / 32 + w];
                        S[j]->partials[tno] = sum;
                    }
                }
                __syncthreads();
            }
        }
    }
}

template <int P, int RECON, int NRB, int RPT, bool WITH_NORM = true>
inline cudaError_t hop_nrb(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k, int mode,
                    int gate, cudaStream_t st)
{
    if (mode != BH_PLAIN) {
        if constexpr (WITH_NORM) {
            if (mode == BH_NORM)
                k_batch_hop<P, RECON, NRB, BH_NORM, RPT><<<t.grid, BT, 0, st>>>(t.dev, t.ngroups, t.nitems, sys, parity, rin, rout, rx, k, gate);
            else
                k_batch_hop<P, RECON, NRB, BH_UPDATE, RPT><<<t.grid, BT, 0, st>>>(t.dev, t.ngroups, t.nitems, sys, parity, rin, rout, rx, k, gate);
        } else {
            return cudaErrorInvalidValue;
        }
    } else {
        k_batch_hop<P, RECON, NRB, BH_PLAIN, RPT><<<t.grid, BT, 0, st>>>(t.dev, t.ngroups, t.nitems, sys, parity, rin, rout, rx, k, gate);
    }
    return cudaGetLastError();
}

// Two right-hand sides per thread are built for the memory-latency-bound
// formats only (FP32, FP16); the FP64 formats are bound by arithmetic.
template <int P> constexpr bool has_rpt2() { return P == F32 || P == F16; }

template <int P, int RECON, bool WITH_NORM = true>
inline cudaError_t hop_pr(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k, int mode,
                   int gate, cudaStream_t st)
{
    switch (t.nrb) {
    case 0: return hop_nrb<P, RECON, 0, 1, WITH_NORM>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    case 1: return hop_nrb<P, RECON, 1, 1, WITH_NORM>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    case 2:
        // 8-byte-per-real tiles of 64 sites would exceed 48 KB of static shared memory
        if constexpr (P != F64 && P != F64X) return hop_nrb<P, RECON, 2, 1, WITH_NORM>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
        return cudaErrorInvalidValue;
    case 4: return hop_nrb<P, RECON, 4, 1, WITH_NORM>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    case 10:
        if constexpr (has_rpt2<P>()) return hop_nrb<P, RECON, 0, 2, WITH_NORM>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
        return cudaErrorInvalidValue;
    case 12:
        if constexpr (has_rpt2<P>()) return hop_nrb<P, RECON, 2, 2, WITH_NORM>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
        return cudaErrorInvalidValue;
    case 14:
        if constexpr (has_rpt2<P>()) return hop_nrb<P, RECON, 4, 2, WITH_NORM>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

}  // namespace twm
