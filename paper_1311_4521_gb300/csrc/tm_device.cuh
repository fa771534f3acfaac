// tm_device.cuh -- per-site building blocks of the hopping matrix on sm_103a.
//
// One output site per thread, pull form: every site gathers its eight
// neighbours, so no two threads write the same memory and no atomics are
// needed (the race-free alternative to the push loops with "critical",
// "atomic" or per-site "halo memory" discussed in Sec. 2.4 of the paper).
// Neighbour indices are computed arithmetically from the even-odd index
// instead of being read from the g_iup/g_idn/g_hi tables of Sec. 2.2, so
// index lookups cost no memory traffic at all.
//
// The spin structure uses the half-spinor ("Weyl-type") form that the
// paper's introduction names for tmLQCD's Hopping_Matrix:
// in the chiral basis gamma_mu = [[0, A_mu], [A_mu^dag, 0]] with A_0 = -1,
// A_k = -i sigma_k, and
//     (1 + s gamma_mu) psi = ( h , s A_mu^dag h ),   h = u + s A_mu l,
// where u, l are the upper and lower spin pairs of psi.  Each hop projects
// to the two-spin h (12 reals), multiplies by the link, and rebuilds the
// lower pair from the upper one.
//
// Everything here is __host__ __device__ so that the same code can be
// instantiated for a host-side check of the index arithmetic.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "tm_dd.cuh"

#define TM_HD __host__ __device__ __forceinline__

// Resident CTAs per SM the hop kernels are compiled for (registers per
// thread <= 65536 / (128 x this)).  Measured on GB300 at 32^3x64 (sweep of
// 4, 5, 6, 8): FP32 storage is fastest at 4 (more registers, more loads in
// flight per thread), FP16 at 5; FP64 hops are bound by the FP64 pipe.
#ifndef TM_HOP_MINB_F32
#define TM_HOP_MINB_F32 4
#endif
#ifndef TM_HOP_MINB_F16
#define TM_HOP_MINB_F16 5
#endif
#ifndef TM_HOP_MINB_F64X
#define TM_HOP_MINB_F64X 3
#endif
#ifndef TM_HOP_MINB_F64
#define TM_HOP_MINB_F64 2
#endif
#ifndef TM_F64X_UNROLL
#define TM_F64X_UNROLL 2  // hops per iteration of the double-float stencil loop (sweep of 1, 2, 4)
#endif
#define TM_HOP_MINB(P) ((P) == 0 ? TM_HOP_MINB_F64 : (P) == 3 ? TM_HOP_MINB_F64X : (P) == 1 ? TM_HOP_MINB_F32 : TM_HOP_MINB_F16)

namespace twm {

// Storage precisions: FP64; FP32; FP16 with a per-site norm; F64X, each
// FP64 value stored as a double-float pair (FP32 hi, lo) and computed on with
// double-float arithmetic (tm_dd.cuh).
enum { F64 = 0, F32 = 1, F16 = 2, F64X = 3 };
// Not a storage format of a handle: FP64 spinors in the caller's canonical
// layout ([site][spin][colour] complex double), read and written in place by
// the host-field operator (tm_Qtm_host) instead of being packed first.
enum { F64C = 4 };

// Conversions between double and the compute type of a storage precision.
template <typename R> TM_HD R to_R(double x) { return R(x); }
template <> TM_HD dd to_R<dd>(double x) { return dd_from_double(x); }

// Conversion between compute types (double, float, double-float).
template <typename To> TM_HD To cvt(double x) { return to_R<To>(x); }
template <typename To> TM_HD To cvt(float x) { return To(x); }
template <typename To> TM_HD To cvt(dd x);
template <> TM_HD dd cvt<dd>(dd x) { return x; }
template <> TM_HD double cvt<double>(dd x) { return double(x); }
template <> TM_HD float cvt<float>(dd x) { return x.hi; }

// ---------------------------------------------------------------- complex
template <typename R>
struct cpx {
    R re, im;
};

template <typename R> TM_HD cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> TM_HD cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> TM_HD cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <typename R> TM_HD cpx<R> operator*(cpx<R> a, cpx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> TM_HD cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> TM_HD cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
// i*a and -i*a
template <typename R> TM_HD cpx<R> ti(cpx<R> a) { return {-a.im, a.re}; }
template <typename R> TM_HD cpx<R> tmi(cpx<R> a) { return {a.im, -a.re}; }
// acc + a*b and acc + conj(a)*b
template <typename R> TM_HD cpx<R> cmadd(cpx<R> a, cpx<R> b, cpx<R> acc)
{
    acc.re += a.re * b.re;
    acc.re -= a.im * b.im;
    acc.im += a.re * b.im;
    acc.im += a.im * b.re;
    return acc;
}
template <typename R> TM_HD cpx<R> cjmadd(cpx<R> a, cpx<R> b, cpx<R> acc)
{
    acc.re += a.re * b.re;
    acc.re += a.im * b.im;
    acc.im += a.re * b.im;
    acc.im -= a.im * b.re;
    return acc;
}

template <typename R> using Spinor = cpx<R>[4][3];
template <typename R> using Half = cpx<R>[2][3];
template <typename R> using Link = cpx<R>[3][3];

// ---------------------------------------------------------------- geometry
// Division by a divisor fixed on the host: q = (umulhi(n, m) + n) >> s with
// s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1, exact for every
// n < 2^31 (the "round-up" method of Granlund and Montgomery, PLDI 1994).
struct FastDiv {
    unsigned d = 1, m = 0, s = 0;
    FastDiv() = default;
    explicit FastDiv(unsigned div) : d(div)
    {
        while ((1ull << s) < d) ++s;
        m = unsigned(((1ull << 32) * ((1ull << s) - d)) / d + 1);
    }
    TM_HD unsigned div(unsigned n) const
    {
#if defined(__CUDA_ARCH__)
        const unsigned hi = __umulhi(n, m);
#else
        const unsigned hi = unsigned((static_cast<unsigned long long>(n) * m) >> 32);
#endif
        return (hi + n) >> s;
    }
};

// Extents and the even-odd strides.  A one-parity field stores site lex at
// index lex/2; with Lx even, moving by one in y, z or t moves the index by
// sy = Lx/2, sz = sy*Ly, st = sz*Lz.  The divisions that recover a site's
// coordinates from its index use the invariant-divisor form (three integer
// operations instead of a division routine).
struct Geom {
    int lx, ly, lz, lt;
    int hx;                 // lx / 2
    unsigned vh;            // sites per parity
    unsigned sy, sz, st;    // index strides of y, z, t
    int anti[4];            // 1 if a wrapping hop in direction mu (0=t,1=x,2=y,3=z) takes a minus sign
    FastDiv dhx, dly, dlz;  // division by hx, ly, lz
};

// Fills the divisors of a geometry whose extents are set.
inline void geom_set_divisors(Geom &g)
{
    g.dhx = FastDiv(unsigned(g.hx));
    g.dly = FastDiv(unsigned(g.ly));
    g.dlz = FastDiv(unsigned(g.lz));
}

// Neighbour indices (other parity) and wrap flags of output site i of parity p.
struct Nbrs {
    unsigned fwd[4], bwd[4];
    bool wf[4], wb[4];
};

TM_HD void neighbours(const Geom &g, int p, unsigned i, Nbrs &n)
{
    const unsigned q1 = g.dhx.div(i), xh = i - q1 * unsigned(g.hx);
    const unsigned q2 = g.dly.div(q1), y = q1 - q2 * unsigned(g.ly);
    const unsigned t = g.dlz.div(q2), z = q2 - t * unsigned(g.lz);
    unsigned x = 2 * xh + ((y + z + t + p) & 1);
    unsigned row = i - xh;
    // x
    n.wf[1] = x == unsigned(g.lx - 1);
    n.wb[1] = x == 0;
    n.fwd[1] = row + ((n.wf[1] ? 0u : x + 1) >> 1);
    n.bwd[1] = row + ((n.wb[1] ? unsigned(g.lx - 1) : x - 1) >> 1);
    // y
    n.wf[2] = y == unsigned(g.ly - 1);
    n.wb[2] = y == 0;
    n.fwd[2] = n.wf[2] ? i - (g.ly - 1) * g.sy : i + g.sy;
    n.bwd[2] = n.wb[2] ? i + (g.ly - 1) * g.sy : i - g.sy;
    // z
    n.wf[3] = z == unsigned(g.lz - 1);
    n.wb[3] = z == 0;
    n.fwd[3] = n.wf[3] ? i - (g.lz - 1) * g.sz : i + g.sz;
    n.bwd[3] = n.wb[3] ? i + (g.lz - 1) * g.sz : i - g.sz;
    // t
    n.wf[0] = t == unsigned(g.lt - 1);
    n.wb[0] = t == 0;
    n.fwd[0] = n.wf[0] ? i - (g.lt - 1) * g.st : i + g.st;
    n.bwd[0] = n.wb[0] ? i + (g.lt - 1) * g.st : i - g.st;
}

// ---------------------------------------------------------------- site maps
// Which output site (even-odd index) thread k of CTA b handles.  Linear:
// site b * block + k (a CTA covers consecutive sites: with Lx/2 sites per
// half-row, whole y rows at one z, t).  Tiled: a CTA covers a box of
// 2^lg[0] x 2^lg[1] x 2^lg[2] x 2^lg[3] sites in (x-half, y, z, t), every
// extent dividing the lattice's, and the boxes are numbered x-half fastest.
// A box keeps more of each site's 8 neighbours inside the CTA's own sites
// than a run of whole rows (e.g. 16x2x2x2 against 16x8x1x1: 62 % against
// 47 % of the neighbour loads), so more of them may hit in L1.  Every map
// covers every site exactly once and the per-site arithmetic does not
// depend on the map, so all maps give bit-identical results.
struct SiteMap {
    int tiled = 0;
    unsigned block = 128;           // threads per CTA
    unsigned lg[4] = {0, 0, 0, 0};  // log2 of the box extents (tiled)
    FastDiv nbx, nby, nbz;          // boxes along x-half, y, z (tiled)
};

TM_HD unsigned map_site(const Geom &g, const SiteMap &m, unsigned b, unsigned k)
{
    if (!m.tiled) return b * m.block + k;
    const unsigned kx = k & ((1u << m.lg[0]) - 1);
    const unsigned ky = (k >> m.lg[0]) & ((1u << m.lg[1]) - 1);
    const unsigned kz = (k >> (m.lg[0] + m.lg[1])) & ((1u << m.lg[2]) - 1);
    const unsigned kt = k >> (m.lg[0] + m.lg[1] + m.lg[2]);
    const unsigned r1 = m.nbx.div(b), bx = b - r1 * m.nbx.d;
    const unsigned r2 = m.nby.div(r1), by = r1 - r2 * m.nby.d;
    const unsigned bt = m.nbz.div(r2), bz = r2 - bt * m.nbz.d;
    const unsigned x = (bx << m.lg[0]) + kx, y = (by << m.lg[1]) + ky;
    const unsigned z = (bz << m.lg[2]) + kz, t = (bt << m.lg[3]) + kt;
    return x + unsigned(g.hx) * (y + unsigned(g.ly) * (z + unsigned(g.lz) * t));
}

// CTAs a map needs; the linear map of `block` threads; a tiled map with box
// extents 2^lg[d] (false if they do not divide the lattice or the box has
// fewer than 32 or more than 128 sites, the most the hop kernels are
// compiled for).
inline unsigned map_grid(const Geom &g, const SiteMap &m)
{
    if (!m.tiled) return (g.vh + m.block - 1) / m.block;
    return m.nbx.d * m.nby.d * m.nbz.d * (unsigned(g.lt) >> m.lg[3]);
}

inline SiteMap linear_map(unsigned block)
{
    SiteMap m;
    m.block = block;
    return m;
}

inline bool tiled_map(const Geom &g, const unsigned lg[4], SiteMap &m)
{
    const unsigned ext[4] = {unsigned(g.hx), unsigned(g.ly), unsigned(g.lz), unsigned(g.lt)};
    unsigned threads = 1;
    for (int d = 0; d < 4; ++d) {
        if (lg[d] > 10 || ext[d] % (1u << lg[d])) return false;
        threads <<= lg[d];
    }
    if (threads < 32 || threads > 128) return false;
    m = SiteMap();
    m.tiled = 1;
    m.block = threads;
    for (int d = 0; d < 4; ++d) m.lg[d] = lg[d];
    m.nbx = FastDiv(ext[0] >> lg[0]);
    m.nby = FastDiv(ext[1] >> lg[1]);
    m.nbz = FastDiv(ext[2] >> lg[2]);
    return true;
}

// ---------------------------------------------------------------- loads
#if defined(__CUDA_ARCH__)
template <typename T> __device__ __forceinline__ T ld_keep(const T *p) { return __ldg(p); }
template <typename T> __device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }
template <typename T> __device__ __forceinline__ void st_stream(T *p, T v) { __stcs(p, v); }
#else
template <typename T> inline T ld_keep(const T *p) { return *p; }
template <typename T> inline T ld_stream(const T *p) { return *p; }
template <typename T> inline void st_stream(T *p, T v) { *p = v; }
#endif
// Link loads: streaming (evict-first) from global memory, or plain (e.g. from
// a tile staged in shared memory).
template <bool STREAM, typename T> TM_HD T ld_link(const T *p)
{
    if (STREAM) return ld_stream(p);
    return *p;
}

// Spinor storage of one parity (component-major, Vh sites per array).
template <int P> struct SpinorIO;

template <> struct SpinorIO<F64> {
    using R = double;
    // load without the site scale; returns the factor the values must be multiplied by
    TM_HD static R load_raw(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        load(base, vh, i, s);
        return R(1);
    }
    TM_HD static void load(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        const double2 *b = static_cast<const double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 v = ld_keep(b + size_t(c) * vh + i);
            s[c / 3][c % 3] = {v.x, v.y};
        }
    }
    TM_HD static void store(void *base, unsigned vh, unsigned i, const Spinor<R> &s)
    {
        double2 *b = static_cast<double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) st_stream(b + size_t(c) * vh + i, make_double2(s[c / 3][c % 3].re, s[c / 3][c % 3].im));
    }
};

template <> struct SpinorIO<F32> {
    using R = float;
    TM_HD static R load_raw(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        load(base, vh, i, s);
        return R(1);
    }
    TM_HD static void load(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        const float4 *b = static_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = ld_keep(b + size_t(k) * vh + i);
            s[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
            s[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
        }
    }
    TM_HD static void store(void *base, unsigned vh, unsigned i, const Spinor<R> &s)
    {
        float4 *b = static_cast<float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const cpx<R> &a = s[(2 * k) / 3][(2 * k) % 3];
            const cpx<R> &c = s[(2 * k + 1) / 3][(2 * k + 1) % 3];
            st_stream(b + size_t(k) * vh + i, make_float4(a.re, a.im, c.re, c.im));
        }
    }
};

// The canonical layout: site i's 12 complex components at [12 i, 12 i + 12).
template <> struct SpinorIO<F64C> {
    using R = double;
    TM_HD static R load_raw(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        load(base, vh, i, s);
        return R(1);
    }
    TM_HD static void load(const void *base, unsigned, unsigned i, Spinor<R> &s)
    {
        const double2 *b = static_cast<const double2 *>(base) + size_t(i) * 12;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 v = ld_keep(b + c);
            s[c / 3][c % 3] = {v.x, v.y};
        }
    }
    TM_HD static void store(void *base, unsigned, unsigned i, const Spinor<R> &s)
    {
        double2 *b = static_cast<double2 *>(base) + size_t(i) * 12;
#pragma unroll
        for (int c = 0; c < 12; ++c) st_stream(b + c, make_double2(s[c / 3][c % 3].re, s[c / 3][c % 3].im));
    }
};

// Half precision: each site stores its 24 reals divided by the site norm
// (the largest |re| or |im|), so every stored value lies in [-1, 1], and the
// norm itself as a float after the three component arrays.
template <> struct SpinorIO<F16> {
    using R = float;
    // the stored values (in [-1, 1]) and, as return value, the site norm they are scaled by
    TM_HD static R load_raw(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        const uint4 *b = static_cast<const uint4 *>(base);
        const float *nrm = reinterpret_cast<const float *>(b + size_t(3) * vh);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = ld_keep(b + size_t(k) * vh + i);
            unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __half2 h = *reinterpret_cast<__half2 *>(&w[q]);
                float2 f = __half22float2(h);
                int c = 4 * k + q;
                s[c / 3][c % 3] = {f.x, f.y};
            }
        }
        return ld_keep(nrm + i);
    }
    TM_HD static void load(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        const R n = load_raw(base, vh, i, s);
#pragma unroll
        for (int c = 0; c < 12; ++c) s[c / 3][c % 3] = n * s[c / 3][c % 3];
    }
    TM_HD static void store(void *base, unsigned vh, unsigned i, const Spinor<R> &s)
    {
        uint4 *b = static_cast<uint4 *>(base);
        float *nrm = reinterpret_cast<float *>(b + size_t(3) * vh);
        float n = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) n = fmaxf(n, fmaxf(fabsf(s[c / 3][c % 3].re), fabsf(s[c / 3][c % 3].im)));
        float inv = n > 0.f ? 1.f / n : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            unsigned w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int c = 4 * k + q;
                __half2 h = __floats2half2_rn(s[c / 3][c % 3].re * inv, s[c / 3][c % 3].im * inv);
                w[q] = *reinterpret_cast<unsigned *>(&h);
            }
            st_stream(b + size_t(k) * vh + i, make_uint4(w[0], w[1], w[2], w[3]));
        }
        st_stream(nrm + i, n);
    }
};

// Double-float storage: 12 arrays of Vh float4 = (re.hi, re.lo, im.hi, im.lo).
template <> struct SpinorIO<F64X> {
    using R = dd;
    TM_HD static R load_raw(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        load(base, vh, i, s);
        return R(1.f);
    }
    TM_HD static void load(const void *base, unsigned vh, unsigned i, Spinor<R> &s)
    {
        const float4 *b = static_cast<const float4 *>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            float4 v = ld_keep(b + size_t(c) * vh + i);
            s[c / 3][c % 3] = {dd{v.x, v.y}, dd{v.z, v.w}};
        }
    }
    TM_HD static void store(void *base, unsigned vh, unsigned i, const Spinor<R> &s)
    {
        float4 *b = static_cast<float4 *>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const cpx<R> &a = s[c / 3][c % 3];
            st_stream(b + size_t(c) * vh + i, make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo));
        }
    }
};

// Bytes of one packed parity field.
TM_HD size_t spinor_bytes(unsigned vh, int prec)
{
    return prec == F64 || prec == F64X ? size_t(192) * vh : prec == F32 ? size_t(96) * vh
                                        : prec == F16 ? size_t(52) * vh : 0;
}

// Link storage: for each origin parity p and direction mu a block of NCHUNK
// arrays of Vh vectors, block index 4p + mu.  Reconstruct 12 keeps rows 0
// and 1; row 2 of an SU(3) matrix is conj(row0 x row1).
template <typename R> TM_HD void reconstruct_row2(Link<R> &u)
{
    u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
}

template <int P, int RECON> struct LinkIO;

template <> struct LinkIO<F64, 18> {
    using R = double;
    using V = double2;
    static constexpr int NCHUNK = 9;
    template <bool STREAM = true> TM_HD static void load(const V *blk, unsigned vh, unsigned i, Link<R> &u)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            V v = ld_link<STREAM>(blk + size_t(k) * vh + i);
            u[k / 3][k % 3] = {v.x, v.y};
        }
    }
    TM_HD static void store(V *blk, unsigned vh, unsigned i, const double *m)
    {
        for (int k = 0; k < 9; ++k) blk[size_t(k) * vh + i] = make_double2(m[2 * k], m[2 * k + 1]);
    }
};

template <> struct LinkIO<F64, 12> {
    using R = double;
    using V = double2;
    static constexpr int NCHUNK = 6;
    template <bool STREAM = true> TM_HD static void load(const V *blk, unsigned vh, unsigned i, Link<R> &u)
    {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            V v = ld_link<STREAM>(blk + size_t(k) * vh + i);
            u[k / 3][k % 3] = {v.x, v.y};
        }
        reconstruct_row2(u);
    }
    TM_HD static void store(V *blk, unsigned vh, unsigned i, const double *m)
    {
        for (int k = 0; k < 6; ++k) blk[size_t(k) * vh + i] = make_double2(m[2 * k], m[2 * k + 1]);
    }
};

template <> struct LinkIO<F32, 18> {
    using R = float;
    using V = float2;
    static constexpr int NCHUNK = 9;
    template <bool STREAM = true> TM_HD static void load(const V *blk, unsigned vh, unsigned i, Link<R> &u)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            V v = ld_link<STREAM>(blk + size_t(k) * vh + i);
            u[k / 3][k % 3] = {v.x, v.y};
        }
    }
    TM_HD static void store(V *blk, unsigned vh, unsigned i, const double *m)
    {
        for (int k = 0; k < 9; ++k) blk[size_t(k) * vh + i] = make_float2(float(m[2 * k]), float(m[2 * k + 1]));
    }
};

template <> struct LinkIO<F32, 12> {
    using R = float;
    using V = float4;
    static constexpr int NCHUNK = 3;
    template <bool STREAM = true> TM_HD static void load(const V *blk, unsigned vh, unsigned i, Link<R> &u)
    {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V v = ld_link<STREAM>(blk + size_t(k) * vh + i);
            u[(2 * k) / 3][(2 * k) % 3] = {v.x, v.y};
            u[(2 * k + 1) / 3][(2 * k + 1) % 3] = {v.z, v.w};
        }
        reconstruct_row2(u);
    }
    TM_HD static void store(V *blk, unsigned vh, unsigned i, const double *m)
    {
        for (int k = 0; k < 3; ++k)
            blk[size_t(k) * vh + i] = make_float4(float(m[4 * k]), float(m[4 * k + 1]), float(m[4 * k + 2]), float(m[4 * k + 3]));
    }
};

// Half-precision links: entries of an SU(3) matrix lie in [-1, 1], so no scale is stored.
template <> struct LinkIO<F16, 12> {
    using R = float;
    using V = uint2;
    static constexpr int NCHUNK = 3;
    template <bool STREAM = true> TM_HD static void load(const V *blk, unsigned vh, unsigned i, Link<R> &u)
    {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V v = ld_link<STREAM>(blk + size_t(k) * vh + i);
            float2 a = __half22float2(*reinterpret_cast<__half2 *>(&v.x));
            float2 b = __half22float2(*reinterpret_cast<__half2 *>(&v.y));
            u[(2 * k) / 3][(2 * k) % 3] = {a.x, a.y};
            u[(2 * k + 1) / 3][(2 * k + 1) % 3] = {b.x, b.y};
        }
        reconstruct_row2(u);
    }
    TM_HD static void store(V *blk, unsigned vh, unsigned i, const double *m)
    {
        for (int k = 0; k < 3; ++k) {
            __half2 a = __floats2half2_rn(float(m[4 * k]), float(m[4 * k + 1]));
            __half2 b = __floats2half2_rn(float(m[4 * k + 2]), float(m[4 * k + 3]));
            blk[size_t(k) * vh + i] = make_uint2(*reinterpret_cast<unsigned *>(&a), *reinterpret_cast<unsigned *>(&b));
        }
    }
};

// Double-float links: each complex entry one float4 (re.hi, re.lo, im.hi, im.lo).
template <> struct LinkIO<F64X, 18> {
    using R = dd;
    using V = float4;
    static constexpr int NCHUNK = 9;
    template <bool STREAM = true> TM_HD static void load(const V *blk, unsigned vh, unsigned i, Link<R> &u)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            V v = ld_link<STREAM>(blk + size_t(k) * vh + i);
            u[k / 3][k % 3] = {dd{v.x, v.y}, dd{v.z, v.w}};
        }
    }
    TM_HD static void store(V *blk, unsigned vh, unsigned i, const double *m)
    {
        for (int k = 0; k < 9; ++k) {
            dd re = dd_from_double(m[2 * k]), im = dd_from_double(m[2 * k + 1]);
            blk[size_t(k) * vh + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
};

template <> struct LinkIO<F64X, 12> {
    using R = dd;
    using V = float4;
    static constexpr int NCHUNK = 6;
    template <bool STREAM = true> TM_HD static void load(const V *blk, unsigned vh, unsigned i, Link<R> &u)
    {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            V v = ld_link<STREAM>(blk + size_t(k) * vh + i);
            u[k / 3][k % 3] = {dd{v.x, v.y}, dd{v.z, v.w}};
        }
        reconstruct_row2(u);
    }
    TM_HD static void store(V *blk, unsigned vh, unsigned i, const double *m)
    {
        for (int k = 0; k < 6; ++k) {
            dd re = dd_from_double(m[2 * k]), im = dd_from_double(m[2 * k + 1]);
            blk[size_t(k) * vh + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
};

// ---------------------------------------------------------------- spin algebra
// h = u + s A_mu l  (the upper pair of (1 + s gamma_mu) psi), s = +1 or -1.
template <int MU, int S, typename R> TM_HD void project(const Spinor<R> &p, Half<R> &h)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) {  // A_0 l = (-l0, -l1)
            h[0][c] = S > 0 ? p[0][c] - p[2][c] : p[0][c] + p[2][c];
            h[1][c] = S > 0 ? p[1][c] - p[3][c] : p[1][c] + p[3][c];
        } else if (MU == 1) {  // A_1 l = (-i l1, -i l0)
            h[0][c] = S > 0 ? p[0][c] + tmi(p[3][c]) : p[0][c] + ti(p[3][c]);
            h[1][c] = S > 0 ? p[1][c] + tmi(p[2][c]) : p[1][c] + ti(p[2][c]);
        } else if (MU == 2) {  // A_2 l = (-l1, l0)
            h[0][c] = S > 0 ? p[0][c] - p[3][c] : p[0][c] + p[3][c];
            h[1][c] = S > 0 ? p[1][c] + p[2][c] : p[1][c] - p[2][c];
        } else {  // A_3 l = (-i l0, i l1)
            h[0][c] = S > 0 ? p[0][c] + tmi(p[2][c]) : p[0][c] + ti(p[2][c]);
            h[1][c] = S > 0 ? p[1][c] + ti(p[3][c]) : p[1][c] + tmi(p[3][c]);
        }
    }
}

// acc += w (h, s A_mu^dag h), the full spinor rebuilt from its upper pair.
// w carries the boundary sign of the hop and the site scale of the input
// (1 except for half-precision storage); it rides on fused multiply-adds.
template <typename R> TM_HD cpx<R> fmadd(R w, cpx<R> a, cpx<R> acc) { return {acc.re + w * a.re, acc.im + w * a.im}; }

// Double-float storage has no site scale, so w is +1 or -1: a sign flip and
// an addition instead of a double-float product.
TM_HD cpx<dd> fmadd(dd w, cpx<dd> a, cpx<dd> acc)
{
    const float s = w.hi;
    return {acc.re + dd{s * a.re.hi, s * a.re.lo}, acc.im + dd{s * a.im.hi, s * a.im.lo}};
}

template <int MU, int S, typename R> TM_HD void accumulate(const Half<R> &h, R w, Spinor<R> &a)
{
    const R ws = S > 0 ? w : -w;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[0][c] = fmadd(w, h[0][c], a[0][c]);
        a[1][c] = fmadd(w, h[1][c], a[1][c]);
        if (MU == 0) {  // s A_0^dag h = -s (h0, h1)
            a[2][c] = fmadd(-ws, h[0][c], a[2][c]);
            a[3][c] = fmadd(-ws, h[1][c], a[3][c]);
        } else if (MU == 1) {  // s A_1^dag h = s (i h1, i h0)
            a[2][c] = fmadd(ws, ti(h[1][c]), a[2][c]);
            a[3][c] = fmadd(ws, ti(h[0][c]), a[3][c]);
        } else if (MU == 2) {  // s A_2^dag h = s (h1, -h0)
            a[2][c] = fmadd(ws, h[1][c], a[2][c]);
            a[3][c] = fmadd(-ws, h[0][c], a[3][c]);
        } else {  // s A_3^dag h = s (i h0, -i h1)
            a[2][c] = fmadd(ws, ti(h[0][c]), a[2][c]);
            a[3][c] = fmadd(-ws, ti(h[1][c]), a[3][c]);
        }
    }
}

// r = U h (dag = false) or U^dag h (dag = true) on both spin components.
template <bool DAG, typename R> TM_HD void link_mul(const Link<R> &u, const Half<R> &h, Half<R> &r)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cpx<R> acc = {R(0), R(0)};
#pragma unroll
            for (int b = 0; b < 3; ++b) acc = DAG ? cjmadd(u[b][a], h[s][b], acc) : cmadd(u[a][b], h[s][b], acc);
            r[s][a] = acc;
        }
}

// Double-float link multiply: each output component is a dot product of six
// real terms, summed with the compensated accumulator instead of six
// double-float multiply-adds.
template <bool DAG> TM_HD void link_mul(const Link<dd> &u, const Half<dd> &h, Half<dd> &r)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dot2 re, im;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cpx<dd> w = DAG ? u[b][a] : u[a][b];
                const cpx<dd> x = h[s][b];
                if (DAG) {  // conj(w) x
                    re.add(w.re, x.re);
                    re.add(w.im, x.im);
                    im.add(w.re, x.im);
                    im.sub(w.im, x.re);
                } else {  // w x
                    re.add(w.re, x.re);
                    re.sub(w.im, x.im);
                    im.add(w.re, x.im);
                    im.add(w.im, x.re);
                }
            }
            r[s][a] = {re.result(), im.result()};
        }
}

// Where the hop finds its links.  GlobalLinks reads the forward link
// U_mu(x) at the output site's index and the backward link U_mu(x-mu) at
// the neighbour's index from the packed gauge field; StagedLinks reads both
// from a tile [8 directions][NCHUNK][ts sites] that the block has copied to
// shared memory (forward mu at 0..3, backward at 4..7).
// STREAM: evict-first loads (each link is used once); otherwise default
// caching, for launches in which several CTAs read the same links.
template <int P, int RECON, bool STREAM = true> struct GlobalLinks {
    using L = LinkIO<P, RECON>;
    const typename L::V *links;
    unsigned vh, i;
    int p;
    template <int MU> TM_HD void fwd(const Nbrs &, Link<typename SpinorIO<P>::R> &u) const
    {
        L::template load<STREAM>(links + size_t(4 * p + MU) * L::NCHUNK * vh, vh, i, u);
    }
    template <int MU> TM_HD void bwd(const Nbrs &n, Link<typename SpinorIO<P>::R> &u) const
    {
        L::template load<STREAM>(links + size_t(4 * (1 - p) + MU) * L::NCHUNK * vh, vh, n.bwd[MU], u);
    }
};

template <int P, int RECON> struct StagedLinks {
    using L = LinkIO<P, RECON>;
    const typename L::V *tile;
    unsigned ts, s;
    template <int MU> TM_HD void fwd(const Nbrs &, Link<typename SpinorIO<P>::R> &u) const
    {
        L::template load<false>(tile + size_t(MU) * L::NCHUNK * ts, ts, s, u);
    }
    template <int MU> TM_HD void bwd(const Nbrs &, Link<typename SpinorIO<P>::R> &u) const
    {
        L::template load<false>(tile + size_t(4 + MU) * L::NCHUNK * ts, ts, s, u);
    }
};

// The projected half-spinor h = (1 + S gamma_mu)-upper pair of the input at
// site j, and the weight its components carry (the FP16 site norm, else 1).
// Half-precision storage projects the packed half2 values before converting
// them: 6 half2 additions and 12 conversions instead of 24 conversions and
// 12 FP32 additions.  The sums round to FP16 (relative 2^-11 of each sum,
// the order of the storage rounding itself).
#if defined(__CUDA_ARCH__)
// h from the 12 packed half2 words of an FP16 site (component 3 s + c)
template <int MU, int S> __device__ __forceinline__ void project_h2(const unsigned (&w)[12], Half<float> &h)
{
    auto p = [&](int sp, int c) { return *reinterpret_cast<const __half2 *>(&w[3 * sp + c]); };
    const __half2 pm = __floats2half2_rn(1.f, -1.f), mp = __floats2half2_rn(-1.f, 1.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        __half2 h0, h1;
        if (MU == 0) {  // A_0 l = (-l0, -l1)
            h0 = S > 0 ? __hsub2(p(0, c), p(2, c)) : __hadd2(p(0, c), p(2, c));
            h1 = S > 0 ? __hsub2(p(1, c), p(3, c)) : __hadd2(p(1, c), p(3, c));
        } else if (MU == 1) {  // A_1 l = (-i l1, -i l0); -i a = swap(a) (1, -1)
            h0 = __hfma2(__lowhigh2highlow(p(3, c)), S > 0 ? pm : mp, p(0, c));
            h1 = __hfma2(__lowhigh2highlow(p(2, c)), S > 0 ? pm : mp, p(1, c));
        } else if (MU == 2) {  // A_2 l = (-l1, l0)
            h0 = S > 0 ? __hsub2(p(0, c), p(3, c)) : __hadd2(p(0, c), p(3, c));
            h1 = S > 0 ? __hadd2(p(1, c), p(2, c)) : __hsub2(p(1, c), p(2, c));
        } else {  // A_3 l = (-i l0, i l1)
            h0 = __hfma2(__lowhigh2highlow(p(2, c)), S > 0 ? pm : mp, p(0, c));
            h1 = __hfma2(__lowhigh2highlow(p(3, c)), S > 0 ? mp : pm, p(1, c));
        }
        const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
        h[0][c] = {f0.x, f0.y};
        h[1][c] = {f1.x, f1.y};
    }
}
#endif

template <int P, int MU, int S>
TM_HD typename SpinorIO<P>::R load_project(const void *in, unsigned vh, unsigned j, Half<typename SpinorIO<P>::R> &h)
{
    using R = typename SpinorIO<P>::R;
#if defined(__CUDA_ARCH__)
    if constexpr (P == F16) {
        const uint4 *b = static_cast<const uint4 *>(in);
        unsigned w[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 v = ld_keep(b + size_t(k) * vh + j);
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        }
        project_h2<MU, S>(w, h);
        return ld_keep(reinterpret_cast<const float *>(b + size_t(3) * vh) + j);
    } else
#endif
    {
        Spinor<R> s;
        const R w = SpinorIO<P>::load_raw(in, vh, j, s);
        project<MU, S>(s, h);
        return w;
    }
}

// One direction mu of the hop at output site i, added into acc.  Forward:
// (1 - gamma_mu) U_mu(x) psi(x+mu); backward (1 + gamma_mu) U_mu(x-mu)^dag
// psi(x-mu).  DAG swaps the two projectors, which gives the adjoint hop
// gamma5 Dhop gamma5 = Dhop^dag.
template <int P, bool DAG, int MU, class Src>
TM_HD void hop_fwd(const Geom &g, const Nbrs &n, const Src &src, const void *in, Spinor<typename SpinorIO<P>::R> &acc)
{
    using R = typename SpinorIO<P>::R;
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma_mu
    Half<R> h, r;
    Link<R> u;
    R w = load_project<P, MU, SF>(in, g.vh, n.fwd[MU], h);
    src.template fwd<MU>(n, u);
    link_mul<false>(u, h, r);
    if (n.wf[MU] && g.anti[MU]) w = -w;
    accumulate<MU, SF>(r, w, acc);
}

template <int P, bool DAG, int MU, class Src>
TM_HD void hop_bwd(const Geom &g, const Nbrs &n, const Src &src, const void *in, Spinor<typename SpinorIO<P>::R> &acc)
{
    using R = typename SpinorIO<P>::R;
    constexpr int SB = DAG ? -1 : +1;  // backward projector 1 + SB gamma_mu
    Half<R> h, r;
    Link<R> u;
    R w = load_project<P, MU, SB>(in, g.vh, n.bwd[MU], h);
    src.template bwd<MU>(n, u);
    link_mul<true>(u, h, r);
    if (n.wb[MU] && g.anti[MU]) w = -w;
    accumulate<MU, SB>(r, w, acc);
}

template <int P, bool DAG, int MU, class Src>
TM_HD void hop_dir(const Geom &g, const Nbrs &n, const Src &src, const void *in, Spinor<typename SpinorIO<P>::R> &acc)
{
    hop_fwd<P, DAG, MU>(g, n, src, in, acc);
    hop_bwd<P, DAG, MU>(g, n, src, in, acc);
}

// ---------------------------------------------------------------- FP64 pairs
// FP64 runs at 1/64 of the FP32 rate here, so the FP64 hop is bound by its
// FP64 operation count, not by memory.  The two hops of one direction share
// their spin reconstruction: with rf = w_f U_mu(x) h_f and
// rb = w_b U_mu(x-mu)^dag h_b (w the boundary signs), the direction adds
// rf + rb to the upper spins and SF A_mu^dag (rf - rb) to the lower ones.
// The boundary signs are folded into h by flipping sign bits (integer
// operations), the backward product's sums start from -rf so that
// d = rb - rf comes out of the same fused multiply-adds, and then
// upper += 2 rf + d, lower += SB A_mu^dag d: 36 FP64 operations per
// direction for reconstruction and accumulation instead of 48 (24 for the
// first direction, while the accumulator is still zero).
TM_HD double flip_sign(double x, unsigned long long m)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)m);
#else
    unsigned long long b;
    memcpy(&b, &x, 8);
    b ^= m;
    memcpy(&x, &b, 8);
    return x;
#endif
}

TM_HD void flip_sign(Half<double> &h, bool neg)
{
    const unsigned long long m = neg ? 0x8000000000000000ull : 0ull;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) h[s][c] = {flip_sign(h[s][c].re, m), flip_sign(h[s][c].im, m)};
}

// r = U h - sub (dag = false) or U^dag h - sub (dag = true)
template <bool DAG, typename R>
TM_HD void link_mul_minus(const Link<R> &u, const Half<R> &h, const Half<R> &sub, Half<R> &r)
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cpx<R> acc = {-sub[s][a].re, -sub[s][a].im};
#pragma unroll
            for (int b = 0; b < 3; ++b) acc = DAG ? cjmadd(u[b][a], h[s][b], acc) : cmadd(u[a][b], h[s][b], acc);
            r[s][a] = acc;
        }
}

// the lower-spin term S A_mu^dag d for lower spin 2 + k
template <int MU, int S, typename R> TM_HD cpx<R> lower_term(const Half<R> &d, int k, int c)
{
    cpx<R> v;
    if (MU == 0) v = -d[k][c];                      // A_0^dag d = -(d0, d1)
    else if (MU == 1) v = ti(d[1 - k][c]);          // A_1^dag d = (i d1, i d0)
    else if (MU == 2) v = k == 0 ? d[1][c] : -d[0][c];  // A_2^dag d = (d1, -d0)
    else v = k == 0 ? ti(d[0][c]) : -ti(d[1][c]);   // A_3^dag d = (i d0, -i d1)
    return S > 0 ? v : -v;
}

template <int P, bool DAG, int MU, bool FIRST, class Src>
TM_HD void hop_dir_pair(const Geom &g, const Nbrs &n, const Src &src, const void *in, Spinor<double> &acc)
{
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma_mu
    constexpr int SB = -SF;
    Half<double> rf, d;
    {
        Spinor<double> s;
        Half<double> h;
        Link<double> u;
        SpinorIO<P>::load_raw(in, g.vh, n.fwd[MU], s);
        project<MU, SF>(s, h);
        flip_sign(h, n.wf[MU] && g.anti[MU]);
        src.template fwd<MU>(n, u);
        link_mul<false>(u, h, rf);
    }
    {
        Spinor<double> s;
        Half<double> h;
        Link<double> u;
        SpinorIO<P>::load_raw(in, g.vh, n.bwd[MU], s);
        project<MU, SB>(s, h);
        flip_sign(h, n.wb[MU] && g.anti[MU]);
        src.template bwd<MU>(n, u);
        link_mul_minus<true>(u, h, rf, d);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cpx<double> lo = lower_term<MU, SB>(d, k, c);
            if (FIRST) {
                acc[k][c] = {2.0 * rf[k][c].re + d[k][c].re, 2.0 * rf[k][c].im + d[k][c].im};
                acc[2 + k][c] = lo;
            } else {
                acc[k][c] = {(acc[k][c].re + 2.0 * rf[k][c].re) + d[k][c].re,
                             (acc[k][c].im + 2.0 * rf[k][c].im) + d[k][c].im};
                acc[2 + k][c] = acc[2 + k][c] + lo;
            }
        }
}

// The 8 hops as a loop unrolled only by TM_F64X_UNROLL, for double-float
// storage: its arithmetic expands to so many FP32 instructions that the
// fully unrolled stencil overflows the instruction cache (ncu: warps stalled
// on "no instruction"); two hops per iteration were measured 2 % faster
// than one, four slower.  Each link multiply is instantiated once; the
// direction-dependent spin algebra is selected by small switches, and all
// register arrays keep static indices.
template <int P, bool DAG, class Src>
TM_HD void hop_site_rolled(const Geom &g, const Nbrs &n, const Src &src, const void *in,
                           Spinor<typename SpinorIO<P>::R> &acc)
{
    using R = typename SpinorIO<P>::R;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    constexpr int kUnroll = TM_F64X_UNROLL;
#pragma unroll kUnroll
    for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1;
        const bool fwd = (k & 1) == 0;
        unsigned j;
        bool wrap;
        switch (k) {
        case 0: j = n.fwd[0]; wrap = n.wf[0]; break;
        case 1: j = n.bwd[0]; wrap = n.wb[0]; break;
        case 2: j = n.fwd[1]; wrap = n.wf[1]; break;
        case 3: j = n.bwd[1]; wrap = n.wb[1]; break;
        case 4: j = n.fwd[2]; wrap = n.wf[2]; break;
        case 5: j = n.bwd[2]; wrap = n.wb[2]; break;
        case 6: j = n.fwd[3]; wrap = n.wf[3]; break;
        default: j = n.bwd[3]; wrap = n.wb[3]; break;
        }
        Spinor<R> s;
        Half<R> h, r;
        Link<R> u;
        R w = SpinorIO<P>::load_raw(in, g.vh, j, s);
        if (wrap && g.anti[mu]) w = -w;
        switch (k) {
        case 0: project<0, SF>(s, h); src.template fwd<0>(n, u); break;
        case 1: project<0, SB>(s, h); src.template bwd<0>(n, u); break;
        case 2: project<1, SF>(s, h); src.template fwd<1>(n, u); break;
        case 3: project<1, SB>(s, h); src.template bwd<1>(n, u); break;
        case 4: project<2, SF>(s, h); src.template fwd<2>(n, u); break;
        case 5: project<2, SB>(s, h); src.template bwd<2>(n, u); break;
        case 6: project<3, SF>(s, h); src.template fwd<3>(n, u); break;
        default: project<3, SB>(s, h); src.template bwd<3>(n, u); break;
        }
        if (fwd) link_mul<false>(u, h, r);
        else link_mul<true>(u, h, r);
        switch (k) {
        case 0: accumulate<0, SF>(r, w, acc); break;
        case 1: accumulate<0, SB>(r, w, acc); break;
        case 2: accumulate<1, SF>(r, w, acc); break;
        case 3: accumulate<1, SB>(r, w, acc); break;
        case 4: accumulate<2, SF>(r, w, acc); break;
        case 5: accumulate<2, SB>(r, w, acc); break;
        case 6: accumulate<3, SF>(r, w, acc); break;
        default: accumulate<3, SB>(r, w, acc); break;
        }
    }
}

template <int P, bool DAG, class Src>
TM_HD void hop_site_src(const Geom &g, const Nbrs &n, const Src &src, const void *in, Spinor<typename SpinorIO<P>::R> &acc)
{
    using R = typename SpinorIO<P>::R;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[s][c] = {R(0), R(0)};
    if constexpr (P == F64X) {
        hop_site_rolled<P, DAG>(g, n, src, in, acc);
    } else if constexpr (P == F64 || P == F64C) {
        hop_dir_pair<P, DAG, 0, true>(g, n, src, in, acc);
        hop_dir_pair<P, DAG, 1, false>(g, n, src, in, acc);
        hop_dir_pair<P, DAG, 2, false>(g, n, src, in, acc);
        hop_dir_pair<P, DAG, 3, false>(g, n, src, in, acc);
    } else {
        hop_dir<P, DAG, 0>(g, n, src, in, acc);
        hop_dir<P, DAG, 1>(g, n, src, in, acc);
        hop_dir<P, DAG, 2>(g, n, src, in, acc);
        hop_dir<P, DAG, 3>(g, n, src, in, acc);
    }
}

// The hop of one site for two input fields at once (two right-hand sides on
// one lattice): each link is loaded once and applied to both, and the two
// fields' neighbour loads are independent, so a thread has twice the loads
// in flight (per-hop form; for the storage formats whose hop is bound by
// memory latency, not by FP64 arithmetic).
template <int P, bool DAG, int MU, class Src>
TM_HD void hop_dir2(const Geom &g, const Nbrs &n, const Src &src, const void *in0, const void *in1,
                    Spinor<typename SpinorIO<P>::R> &a0, Spinor<typename SpinorIO<P>::R> &a1)
{
    using R = typename SpinorIO<P>::R;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    {
        Half<R> h0, h1, r;
        Link<R> u;
        R w0 = load_project<P, MU, SF>(in0, g.vh, n.fwd[MU], h0);
        R w1 = load_project<P, MU, SF>(in1, g.vh, n.fwd[MU], h1);
        src.template fwd<MU>(n, u);
        if (n.wf[MU] && g.anti[MU]) {
            w0 = -w0;
            w1 = -w1;
        }
        link_mul<false>(u, h0, r);
        accumulate<MU, SF>(r, w0, a0);
        link_mul<false>(u, h1, r);
        accumulate<MU, SF>(r, w1, a1);
    }
    {
        Half<R> h0, h1, r;
        Link<R> u;
        R w0 = load_project<P, MU, SB>(in0, g.vh, n.bwd[MU], h0);
        R w1 = load_project<P, MU, SB>(in1, g.vh, n.bwd[MU], h1);
        src.template bwd<MU>(n, u);
        if (n.wb[MU] && g.anti[MU]) {
            w0 = -w0;
            w1 = -w1;
        }
        link_mul<true>(u, h0, r);
        accumulate<MU, SB>(r, w0, a0);
        link_mul<true>(u, h1, r);
        accumulate<MU, SB>(r, w1, a1);
    }
}

template <int P, bool DAG, class Src>
TM_HD void hop_site_src_pair(const Geom &g, const Nbrs &n, const Src &src, const void *in0, const void *in1,
                             Spinor<typename SpinorIO<P>::R> &a0, Spinor<typename SpinorIO<P>::R> &a1)
{
    using R = typename SpinorIO<P>::R;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) a0[s][c] = a1[s][c] = {R(0), R(0)};
    hop_dir2<P, DAG, 0>(g, n, src, in0, in1, a0, a1);
    hop_dir2<P, DAG, 1>(g, n, src, in0, in1, a0, a1);
    hop_dir2<P, DAG, 2>(g, n, src, in0, in1, a0, a1);
    hop_dir2<P, DAG, 3>(g, n, src, in0, in1, a0, a1);
}

// The hop at output site i of parity p with links read from the packed gauge field.
template <int P, int RECON, bool DAG>
TM_HD void hop_site(const Geom &g, int p, unsigned i, const typename LinkIO<P, RECON>::V *links, const void *in,
                    Spinor<typename SpinorIO<P>::R> &acc)
{
    Nbrs n;
    neighbours(g, p, i, n);
    GlobalLinks<P, RECON> src{links, g.vh, i, p};
    hop_site_src<P, DAG>(g, n, src, in, acc);
}

// Site-local epilogue: out_u = a_u hop_u + b_u x_u, out_l = a_l hop_l + b_l x_l
// (u = spins 0,1; l = spins 2,3).  With gamma5 = diag(1,1,-1,-1) this covers
// the twisted-mass factors (1 +- i mut gamma5)^(+-1) and the final gamma5.
// With `unit` set the hop term enters as +hop_u, -hop_l (no multiply).
struct Coef {
    double d[8];  // au_re, au_im, al_re, al_im, bu_re, bu_im, bl_re, bl_im
    float f[8];   // the same, rounded once on the host for single-precision kernels
    float xh[8], xl[8];  // and as double-float pairs
    int unit;            // a_u = 1, a_l = -1 exactly: the hop term is applied as a sign
    Coef() = default;
    __host__ __device__ Coef(double au_re, double au_im, double al_re, double al_im, double bu_re, double bu_im,
                             double bl_re, double bl_im)
        : d{au_re, au_im, al_re, al_im, bu_re, bu_im, bl_re, bl_im}, unit(0)
    {
        for (int k = 0; k < 8; ++k) {
            f[k] = float(d[k]);
            dd x = dd_from_double(d[k]);
            xh[k] = x.hi;
            xl[k] = x.lo;
        }
    }
    TM_HD double get(int k, double) const { return d[k]; }
    TM_HD float get(int k, float) const { return f[k]; }
    TM_HD dd get(int k, dd) const { return dd{xh[k], xl[k]}; }
};

// out_u = a_u hop_u + b_u x_u, out_l = a_l hop_l + b_l x_l per spin half;
// with `unit` the hop term enters as +hop_u, -hop_l (no multiply).
template <typename R>
TM_HD void epilogue_with(cpx<R> au, cpx<R> al, cpx<R> bu, cpx<R> bl, bool unit, const Spinor<R> &hop,
                         const Spinor<R> *x, Spinor<R> &out)
{
    if (unit) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cpx<R> v = s < 2 ? hop[s][c] : -hop[s][c];
                if (x) v = cmadd(s < 2 ? bu : bl, (*x)[s][c], v);
                out[s][c] = v;
            }
        return;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cpx<R> a = s < 2 ? au : al;
            cpx<R> v = a * hop[s][c];
            if (x) v = cmadd(s < 2 ? bu : bl, (*x)[s][c], v);
            out[s][c] = v;
        }
}

template <typename R> TM_HD void epilogue(const Coef &k, const Spinor<R> &hop, const Spinor<R> *x, Spinor<R> &out)
{
    const R z = R(0);
    cpx<R> au = {k.get(0, z), k.get(1, z)}, al = {k.get(2, z), k.get(3, z)};
    cpx<R> bu = {k.get(4, z), k.get(5, z)}, bl = {k.get(6, z), k.get(7, z)};
    epilogue_with(au, al, bu, bl, k.unit != 0, hop, x, out);
}

// The same with the x coefficients multiplied by xs: for half-precision
// storage x is passed as its stored values and xs is its site norm, one
// multiply per coefficient instead of one per component.
TM_HD void epilogue(const Coef &k, const Spinor<float> &hop, const Spinor<float> *x, Spinor<float> &out, float xs)
{
    const float z = 0.f;
    cpx<float> au = {k.get(0, z), k.get(1, z)}, al = {k.get(2, z), k.get(3, z)};
    cpx<float> bu = {xs * k.get(4, z), xs * k.get(5, z)}, bl = {xs * k.get(6, z), xs * k.get(7, z)};
    epilogue_with(au, al, bu, bl, k.unit != 0, hop, x, out);
}

}  // namespace twm
