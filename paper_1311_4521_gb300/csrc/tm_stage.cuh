// tm_stage.cuh -- the batched multi-right-hand-side hop with its operands
// staged in shared memory by the Tensor Memory Accelerator (TMA).
//
// A work tile is a box of 64 output sites: 8 half-sites in x (16 sites of the
// full lattice, one parity) by 2 in each of y, z and t.  The hop of the box
// reads, per right-hand side, the box's own sites (the x and inner y, z, t
// neighbours) and eight faces around it: the half-site columns just left and
// right of it in x and the layers just outside it in y, z and t, 272 sites
// in all (4.25 per output site).  Each is one rectangular box of the
// component-major field seen as a tensor (x, y, z, t, component), so a stage
// is nine `cp.async.bulk.tensor` loads (eighteen for FP16: the site norms
// are a second tensor), at wrapped coordinates for the periodic lattice.
// The links of the tile, in a site-complete copy of the gauge field (for
// every site its 4 forward links and the 4 backward ones U_mu(x-mu)^dag
// needs), are one more box, loaded once per tile and used by all its
// right-hand sides.  This is the shared-memory analogue of the paper's
// precomputed hopping order (Sec. 2.2): every neighbour a thread reads has
// been brought next to the SM in one bulk transfer, instead of eight
// independent gathers through L1 per site and right-hand side.
//
// Warp roles: NPROD producer threads (lane 0 of their warps) issue the
// copies, each for its own stage buffers; consumer groups of two warps (one
// thread per site of the box) compute the hop of one right-hand side each.
// (Issuing the copies from one lane each, 9 or 18 at once, was measured
// slower: 1.19 against 1.07 ms for FP32 launch B.)  A ring of NSTAGE stage buffers carries the
// right-hand sides (stage j serves consumer group j mod NG, so every group
// has two stages: one it computes on while the other fills) with a full and
// an empty mbarrier each; the link tile is double-buffered on its own pair of
// barriers.  Every wait is bounded (about one second of SM clock): a wait
// that runs out sets the status word of the launch and its thread returns,
// so no failure leaves the GPU waiting.
#pragma once

#include <atomic>

#include "tm_batch.cuh"

namespace twm {

constexpr int SBX = 8;           // half-sites of a box in x
constexpr int STS = 64;          // sites of a box (8 x 2 x 2 x 2)
constexpr int STAGE_CODE = 100;  // configuration code of the staged hop

// Tensor-map shapes: the own box, an x column, a y, z or t layer.
enum { SH_OWN = 0, SH_X = 1, SH_Y = 2, SH_Z = 3, SH_T = 4, NSH = 5 };
// The boxes of one stage: own, x-, x+, y-, y+, z-, z+, t-, t+.
enum { B_OWN = 0, B_XM, B_XP, B_YM, B_YP, B_ZM, B_ZP, B_TM, B_TP, NBOX };
TM_HD constexpr int box_shape(int b) { return b == 0 ? SH_OWN : (b + 1) / 2; }
TM_HD constexpr int box_sites(int b) { return b == 0 ? 64 : b <= 2 ? 8 : 32; }
TM_HD constexpr int box_first(int b) { return b == 0 ? 0 : b <= 2 ? 64 + 8 * (b - 1) : 80 + 32 * (b - 3); }
constexpr int STAGE_SITES = 272;
// FP16 site norms: x columns are loaded 4 half-sites wide (16 bytes, the
// smallest row a tensor copy moves), so every norm box holds 32 or 64 floats.
TM_HD constexpr int nbox_first(int b) { return b == 0 ? 0 : 64 + 32 * (b - 1); }
constexpr int NORM_SLOTS = 320;

template <int P> struct StageFmt;
template <> struct StageFmt<F32> {
    static constexpr int CH = 6;  // 16-byte components per site
    static constexpr int NORM = 0;
};
// FP16 site norms: staged like the components (0: nine more tensor copies per
// stage, for 1280 bytes) or read by the consumers from memory (1, the
// default: one 4-byte load per neighbour, issued before the stage is waited
// for).  The single producer thread is on the critical path, so the nine
// copies cost more than the loads: launch B 1.40 -> 1.13 ms on 32^3x64 with
// 12 right-hand sides (and six consumer groups, which the smaller stages fit).
#ifndef TM_STAGE_F16_NORM_GLOBAL
#define TM_STAGE_F16_NORM_GLOBAL 1
#endif
template <> struct StageFmt<F16> {
    static constexpr int CH = 3;
    static constexpr int NORM = TM_STAGE_F16_NORM_GLOBAL ? 0 : 1;
};

// Consumer groups and stage buffers per group (one computed on, the others
// filling) of the FP32 and FP16 formats.  Measured on 32^3x64 with 12
// right-hand sides, FP16 launch B: with staged norms 1.65, 1.39, 1.49, 1.55
// ms for 2, 3, 4, 6 groups; with norms from memory 1.38 (3 groups of 2
// stages), 1.20 (4 of 3), 1.13 ms (6 of 2).  FP32 (26 KB per stage): 3
// groups of 2 stages 1.02 ms, 4 groups of 1 stage 0.955 ms, 6 of 1 (128
// registers, spills) 1.03 ms: with two producers refilling, a group needs no
// second stage of its own, and the fourth group hides more latency.
#ifndef TM_STAGE_NG_F32
#define TM_STAGE_NG_F32 4
#endif
// Producer threads, each in its own warp: stage buffer j is always filled by
// producer j mod NPROD, so every buffer's uses are armed in order by one
// thread (a parity wait can tell phase k from k+1, not from k+2).  Measured
// on 32^3x64 with 12 right-hand sides, launch B: 1 producer 1.06-1.11 ms, 2
// 1.01 ms (FP32-12); FP16 1.16 -> 1.07 ms.
#ifndef TM_STAGE_NPROD
#define TM_STAGE_NPROD 2
#endif
#ifndef TM_STAGE_K_F32
#define TM_STAGE_K_F32 1
#endif
#ifndef TM_STAGE_NG_F16
#define TM_STAGE_NG_F16 6
#endif
#ifndef TM_STAGE_K_F16
#define TM_STAGE_K_F16 2
#endif

// Shared-memory plan of one storage format.  FP32 links are staged with all
// 18 reals (the site-complete copy of a 12-real handle is expanded once, so
// that row 2 is not rebuilt for every right-hand side).
template <int P, int RECON> struct StageCfg {
    static constexpr int LRECON = P == F32 ? 18 : RECON;
    using L = LinkIO<P, LRECON>;
    static constexpr int CH = StageFmt<P>::CH;
    static constexpr int NORM_OFF = STAGE_SITES * CH * 16;
    static constexpr int SBYTES = NORM_OFF + StageFmt<P>::NORM * NORM_SLOTS * 4;   // one right-hand side
    static constexpr int LBYTES = STS * 8 * L::NCHUNK * int(sizeof(typename L::V));  // one link tile
    static constexpr int NG = P == F16 ? TM_STAGE_NG_F16 : TM_STAGE_NG_F32;   // consumer groups (two warps each)
    static constexpr int NSTAGE = (P == F16 ? TM_STAGE_K_F16 : TM_STAGE_K_F32) * NG;   // stages per group
    static constexpr int NCW = 2 * NG;            // consumer warps
    static constexpr int NPROD = TM_STAGE_NPROD;  // producer warps (one issuing thread each)
    static constexpr int NT = 32 * (NCW + NPROD);
    static_assert(NSTAGE % NPROD == 0, "every stage buffer belongs to one producer");
    static constexpr int NBAR = 2 * NSTAGE + 4;
    static constexpr int SMEM = NSTAGE * SBYTES + 2 * LBYTES + NBAR * 8;
    static_assert(SBYTES % 128 == 0 && LBYTES % 128 == 0, "stage buffers keep 128-byte alignment");
    static_assert(SMEM + 4 * STAGE_MAX <= 227 * 1024, "shared memory per CTA");
};

// ---------------------------------------------------------------- PTX
__device__ __forceinline__ unsigned smem_addr(const void *p) { return unsigned(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase of the given parity has completed.  Gives up after
// 2^31 SM clock cycles (about a second): sets *status and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int *status)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicExch(status, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load5(unsigned dst, const CUtensorMap *m, int c0, int c1, int c2, int c3, int c4,
                                          unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load4(unsigned dst, const CUtensorMap *m, int c0, int c1, int c2, int c3,
                                          unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// The tensor maps are written to global memory by host copies: make them
// visible to this thread's tensor copies.
__device__ __forceinline__ void tmap_acquire(const CUtensorMap *m)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

// ---------------------------------------------------------------- consumers
// Where a neighbour lies in the stage: box and position inside the box.
struct SPos {
    int box, pos;
};

// The projected half-spinor of a staged site and its weight (FP16 site norm, else 1).
template <int P, int MU, int S>
__device__ __forceinline__ typename SpinorIO<P>::R stage_project(const unsigned char *st, SPos q,
                                                                 Half<typename SpinorIO<P>::R> &h)
{
    const int cs = box_sites(q.box);
#if defined(__CUDA_ARCH__)
    if constexpr (P == F16) {
        const uint4 *b = reinterpret_cast<const uint4 *>(st) + box_first(q.box) * 3 + q.pos;
        unsigned w[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 v = b[k * cs];
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        }
        project_h2<MU, S>(w, h);
        if constexpr (StageFmt<F16>::NORM == 0) return 1.f;   // the caller multiplies by the site norm
        const int np = q.box == B_XM ? 4 * q.pos + 3 : q.box == B_XP ? 4 * q.pos : q.pos;
        return reinterpret_cast<const float *>(st + StageCfg<F16, 12>::NORM_OFF)[nbox_first(q.box) + np];
    } else
#endif
    {
        const float4 *b = reinterpret_cast<const float4 *>(st) + box_first(q.box) * 6 + q.pos;
        Spinor<float> s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = b[k * cs];
            s[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
            s[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
        }
        project<MU, S>(s, h);
        return 1.f;
    }
}

// Direction mu of the hop from the stage, in the order of hop_dir; bit mu
// (forward) and 4 + mu (backward) of neg mark the hops that cross an
// antiperiodic boundary.
template <int P, int RECON, int MU>
__device__ __forceinline__ void stage_dir(const Nbrs &n, const StagedLinks<P, RECON> &src, const unsigned char *st,
                                          SPos qf, SPos qb, unsigned neg, Spinor<typename SpinorIO<P>::R> &acc,
                                          typename SpinorIO<P>::R nf = 1, typename SpinorIO<P>::R nb = 1)
{
    using R = typename SpinorIO<P>::R;
    Half<R> h, r;
    Link<R> u;
    R w = nf * stage_project<P, MU, -1>(st, qf, h);
    src.template fwd<MU>(n, u);
    link_mul<false>(u, h, r);
    if (neg & (1u << MU)) w = -w;
    accumulate<MU, -1>(r, w, acc);
    w = nb * stage_project<P, MU, +1>(st, qb, h);
    src.template bwd<MU>(n, u);
    link_mul<true>(u, h, r);
    if (neg & (16u << MU)) w = -w;
    accumulate<MU, +1>(r, w, acc);
}

// Box coordinates of work tile tno of a lattice: x fastest, then y, z
// within a block of sbz boxes, t, and the z blocks (stage_zblock).
struct TileBox {
    int xh0, y0, z0, t0;
};
TM_HD TileBox tile_box(const Geom &g, int sbz, unsigned tno)
{
    const unsigned nbx = unsigned(g.hx) / SBX, nby = unsigned(g.ly) / 2, nbt = unsigned(g.lt) / 2;
    unsigned q = tno;
    TileBox b;
    b.xh0 = int(q % nbx) * SBX;
    q /= nbx;
    b.y0 = int(q % nby) * 2;
    q /= nby;
    const unsigned zl = q % unsigned(sbz);
    q /= unsigned(sbz);
    b.t0 = int(q % nbt) * 2;
    b.z0 = int((q / nbt) * unsigned(sbz) + zl) * 2;
    return b;
}

// Even-odd index of site s (0..63: x-half fastest, then y, z, t) of box B.
TM_HD unsigned box_site_index(const Geom &g, const TileBox &B, int s)
{
    const int a = s & 7, b = (s >> 3) & 1, c = (s >> 4) & 1, d = s >> 5;
    return ((unsigned(B.t0 + d) * unsigned(g.lz) + unsigned(B.z0 + c)) * unsigned(g.ly) + unsigned(B.y0 + b)) *
               unsigned(g.hx) + unsigned(B.xh0 + a);
}

// Origin (x-half, y, z, t) of stage box b of tile B: the own box, or the
// layer / column just outside it, wrapped onto the periodic lattice.
struct BoxOrigin {
    int x, y, z, t;
};
TM_HD BoxOrigin stage_box_origin(const Geom &g, const TileBox &B, int b)
{
    BoxOrigin o{B.xh0, B.y0, B.z0, B.t0};
    if (b == B_XM) o.x = (B.xh0 - 1 + g.hx) % g.hx;
    if (b == B_XP) o.x = (B.xh0 + SBX) % g.hx;
    if (b == B_YM) o.y = (B.y0 - 1 + g.ly) % g.ly;
    if (b == B_YP) o.y = (B.y0 + 2) % g.ly;
    if (b == B_ZM) o.z = (B.z0 - 1 + g.lz) % g.lz;
    if (b == B_ZP) o.z = (B.z0 + 2) % g.lz;
    if (b == B_TM) o.t = (B.t0 - 1 + g.lt) % g.lt;
    if (b == B_TP) o.t = (B.t0 + 2) % g.lt;
    return o;
}

// Where the 8 neighbours of box site s (even-odd index i, neighbours n)
// lie in the stage: q[2 mu] forward, q[2 mu + 1] backward.
TM_HD void stage_neighbour_slots(const TileBox &B, int s, unsigned i, const Nbrs &n, SPos (&q)[8])
{
    const int a = s & 7, b = (s >> 3) & 1, c = (s >> 4) & 1, d = s >> 5;
    const unsigned row = i - unsigned(B.xh0 + a);
    const int af = n.wf[1] ? SBX : int(n.fwd[1] - row) - B.xh0;
    const int ab = n.wb[1] ? -1 : int(n.bwd[1] - row) - B.xh0;
    const int xcol = (d * 2 + c) * 2 + b;
    q[0] = d == 0 ? SPos{B_OWN, s + 32} : SPos{B_TP, (c * 2 + b) * 8 + a};
    q[1] = d == 1 ? SPos{B_OWN, s - 32} : SPos{B_TM, (c * 2 + b) * 8 + a};
    q[2] = af >= SBX ? SPos{B_XP, xcol} : SPos{B_OWN, s - a + af};
    q[3] = ab < 0 ? SPos{B_XM, xcol} : SPos{B_OWN, s - a + ab};
    q[4] = b == 0 ? SPos{B_OWN, s + 8} : SPos{B_YP, (d * 2 + c) * 8 + a};
    q[5] = b == 1 ? SPos{B_OWN, s - 8} : SPos{B_YM, (d * 2 + c) * 8 + a};
    q[6] = c == 0 ? SPos{B_OWN, s + 16} : SPos{B_ZP, (d * 2 + b) * 8 + a};
    q[7] = c == 1 ? SPos{B_OWN, s - 16} : SPos{B_ZM, (d * 2 + b) * 8 + a};
}

template <int P, int RECON, int MODE>
__global__ void __launch_bounds__(StageCfg<P, RECON>::NT, 1)
    k_stage_hop(const BGroup *__restrict__ groups, int ngroups, unsigned nitems, const BSys *__restrict__ sys,
                int parity, int rin, int rout, int rx, Coef k, int gate, StageArgs sa)
{
    using C = StageCfg<P, RECON>;
    using R = typename SpinorIO<P>::R;
    using V = typename C::L::V;
    static_assert(MODE == BH_PLAIN, "the staged hop stores its result");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned first[STAGE_MAX];
    unsigned char *stages = smem;
    unsigned char *ltiles = smem + C::NSTAGE * C::SBYTES;
    const unsigned bar0 = smem_addr(ltiles + 2 * C::LBYTES);
    auto full = [&](int j) { return bar0 + 8u * unsigned(j); };
    auto empty = [&](int j) { return bar0 + 8u * unsigned(C::NSTAGE + j); };
    auto lfull = [&](int j) { return bar0 + 8u * unsigned(2 * C::NSTAGE + j); };
    auto lempty = [&](int j) { return bar0 + 8u * unsigned(2 * C::NSTAGE + 2 + j); };

    const int warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    const unsigned *staged = ngroups <= STAGE_MAX ? first : nullptr;
    if (staged)
        for (int g = threadIdx.x; g < ngroups; g += C::NT) first[g] = groups[g].item0;
    if (threadIdx.x == 0) {
        for (int j = 0; j < C::NSTAGE; ++j) {
            mbar_init(full(j), 1);
            mbar_init(empty(j), 2);   // the two warps of the stage's consumer group
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(lfull(j), 1);
            mbar_init(lempty(j), C::NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (warp >= C::NCW) {
        // ---------------- producers: lane 0 of each producer warp issues the copies
        // of the stage buffers j = pi (mod NPROD) and, producer 0, of the link tiles
        const int pi = warp - C::NCW;
        if (lane != 0) return;
        // the last use of each of this producer's buffers and of the link tiles
        // armed so far: on a wait that runs out, the copies still in flight are
        // waited for (bounded) before the thread leaves, so none lands in the
        // shared memory of a finished CTA
        int armed[C::NSTAGE];
#pragma unroll
        for (int j = 0; j < C::NSTAGE; ++j) armed[j] = -1;
        int larmed[2] = {-1, -1};
        auto drain = [&]() {
#pragma unroll
            for (int j = 0; j < C::NSTAGE; ++j)
                if (armed[j] >= 0) (void)mbar_wait(full(j), unsigned(armed[j]) & 1, sa.status);
            for (int j = 0; j < 2; ++j)
                if (larmed[j] >= 0) (void)mbar_wait(lfull(j), unsigned(larmed[j]) & 1, sa.status);
        };
        const int nmap = StageFmt<P>::NORM ? 2 * NSH : NSH;
        for (int gi = 0; gi < ngroups; ++gi) {
            tmap_acquire(sa.lmaps + gi);
            const BGroup &G = groups[gi];
            for (int r = 0; r < G.nrhs; ++r)
                for (int m = 0; m < nmap; ++m) tmap_acquire(sa.smaps + (size_t(G.sys0 + r) * NROLE + rin) * (2 * NSH) + m);
        }
        constexpr int W = int(sizeof(V)) / 8;   // 8-byte elements per link chunk
        constexpr int LCH = 8 * C::L::NCHUNK;
        unsigned u = 0, tl = 0;
        for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
            const int gi = find_group(groups, ngroups, staged, item);
            const BGroup &G = groups[gi];
            bool any = false;
            for (int r = 0; r < G.nrhs && !any; ++r) any = !gated(sys[G.sys0 + r].s, gate);
            if (!any) continue;
            const TileBox B = tile_box(G.g, G.sbz, item - G.item0);
            const int ls = int(tl & 1);
            if (pi == 0) {   // the links of the tile: producer 0
                if (tl >= 2 && !mbar_wait(lempty(ls), ((tl - 2) >> 1) & 1, sa.status)) {
                    drain();
                    return;
                }
                mbar_expect_tx(lfull(ls), C::LBYTES);
                larmed[ls] = int(tl >> 1);
                tma_load5(smem_addr(ltiles + ls * C::LBYTES), sa.lmaps + gi, W * B.xh0, B.y0, B.z0, B.t0,
                          parity * LCH, lfull(ls));
            }
            const int hx = G.g.hx;
            BoxOrigin org[NBOX];   // once per tile: the producer issues every copy, keep its loop short
#pragma unroll
            for (int b = 0; b < NBOX; ++b) org[b] = stage_box_origin(G.g, B, b);
            const int xnm = (B.xh0 - 4 + hx) % hx;
            for (int r = 0; r < G.nrhs; ++r) {
                if (gated(sys[G.sys0 + r].s, gate)) continue;
                const int slot = int(u % C::NSTAGE);
                const unsigned use = u / C::NSTAGE;
                ++u;
                if (slot % C::NPROD != pi) continue;
                if (use >= 1 && !mbar_wait(empty(slot), (use - 1) & 1, sa.status)) {
                    drain();
                    return;
                }
                const unsigned fb = full(slot);
                mbar_expect_tx(fb, C::SBYTES);
                armed[slot] = int(use);
                unsigned char *st = stages + slot * C::SBYTES;
                const CUtensorMap *m = sa.smaps + (size_t(G.sys0 + r) * NROLE + rin) * (2 * NSH);
#pragma unroll
                for (int b = 0; b < NBOX; ++b) {
                    const BoxOrigin &o = org[b];
                    tma_load5(smem_addr(st + box_first(b) * C::CH * 16), m + box_shape(b), 2 * o.x, o.y, o.z, o.t, 0,
                              fb);
                    if constexpr (StageFmt<P>::NORM) {   // FP16 site norms; x columns 4 wide at 16-byte boundaries
                        const int xn = b == B_XM ? xnm : o.x;
                        tma_load4(smem_addr(st + C::NORM_OFF + nbox_first(b) * 4), m + NSH + box_shape(b), xn, o.y,
                                  o.z, o.t, fb);
                    }
                }
            }
            ++tl;
        }
        return;
    }

    // ---------------- consumers: group warp/2 computes the stages j = group (mod NG)
    const int grp = warp >> 1;
    const int s = (warp & 1) * 32 + lane;   // site of the box
    unsigned u = 0, tl = 0;
    for (unsigned item = blockIdx.x; item < nitems; item += gridDim.x) {
        const BGroup &G = groups[find_group(groups, ngroups, staged, item)];
        bool any = false;
        for (int r = 0; r < G.nrhs && !any; ++r) any = !gated(sys[G.sys0 + r].s, gate);
        if (!any) continue;
        const TileBox B = tile_box(G.g, G.sbz, item - G.item0);
        const int ls = int(tl & 1);
        const unsigned vh = G.g.vh;
        const unsigned i = box_site_index(G.g, B, s);
        Nbrs n;
        neighbours(G.g, parity, i, n);
        unsigned neg = 0;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            if (G.g.anti[mu] && n.wf[mu]) neg |= 1u << mu;
            if (G.g.anti[mu] && n.wb[mu]) neg |= 16u << mu;
        }
        SPos q[8];   // positions of the 8 neighbours in the stage
        stage_neighbour_slots(B, s, i, n, q);
        const StagedLinks<P, C::LRECON> src{reinterpret_cast<const V *>(ltiles + ls * C::LBYTES), STS, unsigned(s)};
        if (!mbar_wait(lfull(ls), (tl >> 1) & 1, sa.status)) return;
        const int nrhs = G.nrhs, sys0 = G.sys0;
        for (int r = 0; r < nrhs; ++r) {
            const BSys *S = &sys[sys0 + r];
            if (gated(S->s, gate)) continue;
            const int slot = int(u % C::NSTAGE);
            const unsigned use = u / C::NSTAGE;
            ++u;
            if (slot % C::NG != grp) continue;
            void *outp = S->f[rout];   // loaded now, used after the hop
            Spinor<R> xs;
            if (rx >= 0) SpinorIO<P>::load(S->f[rx], vh, i, xs);   // in flight during the hop
            R nw[8];   // neighbour site norms read from memory (FP16 without staged norms), else 1
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) nw[kk] = R(1);
            if constexpr (P == F16 && StageFmt<F16>::NORM == 0) {
                const float *nrm = reinterpret_cast<const float *>(static_cast<const char *>(S->f[rin]) + size_t(48) * vh);
#pragma unroll
                for (int mu = 0; mu < 4; ++mu) {
                    nw[2 * mu] = ld_keep(nrm + n.fwd[mu]);
                    nw[2 * mu + 1] = ld_keep(nrm + n.bwd[mu]);
                }
            }
            if (!mbar_wait(full(slot), use & 1, sa.status)) return;
            const unsigned char *st = stages + slot * C::SBYTES;
            Spinor<R> acc;
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) acc[sp][cc] = {R(0), R(0)};
            stage_dir<P, C::LRECON, 0>(n, src, st, q[0], q[1], neg, acc, nw[0], nw[1]);
            stage_dir<P, C::LRECON, 1>(n, src, st, q[2], q[3], neg, acc, nw[2], nw[3]);
            stage_dir<P, C::LRECON, 2>(n, src, st, q[4], q[5], neg, acc, nw[4], nw[5]);
            stage_dir<P, C::LRECON, 3>(n, src, st, q[6], q[7], neg, acc, nw[6], nw[7]);
            __syncwarp();
            if (lane == 0) mbar_arrive(empty(slot));   // the stage may be refilled
            Spinor<R> o;
            if (rx >= 0) epilogue(k, acc, &xs, o);
            else epilogue(k, acc, static_cast<const Spinor<R> *>(nullptr), o);
            SpinorIO<P>::store(outp, vh, i, o);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(lempty(ls));   // this warp is done with the tile's links
        ++tl;
    }
}

template <int P, int RECON>
inline cudaError_t stage_hop(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                             int mode, int gate, cudaStream_t st)
{
    using C = StageCfg<P, RECON>;
    // only inputs whose tensor maps were encoded (a zero map must never reach a tensor copy)
    if (mode != BH_PLAIN || !t.sa.smaps || !t.sa.lmaps || !t.sa.status || rin < 0 || rin >= NROLE ||
        !(t.sa.roles & (1u << rin)))
        return cudaErrorInvalidValue;
    // the shared-memory opt-in is a per-device function attribute: set once per device
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        e = cudaFuncSetAttribute(k_stage_hop<P, RECON, BH_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit);
    }
    k_stage_hop<P, RECON, BH_PLAIN><<<t.grid, C::NT, C::SMEM, st>>>(t.dev, t.ngroups, t.nitems, sys, parity, rin,
                                                                     rout, rx, k, gate, t.sa);
    return cudaGetLastError();
}

}  // namespace twm
