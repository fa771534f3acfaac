// Host-side check of the batched hops' work orders (compiled with nvcc as a
// host program; no GPU needed):
//  * the banded tile order of the gather hops (tile_of) is a permutation of
//    the tiles for every band width that divides the lattice, at tiles of
//    128, 64 and 32 sites;
//  * the staged hop's boxes (tile_box, box_site_index) cover every even-odd
//    site exactly once for every z block size;
//  * for every site of every box and both output parities, each of the 8
//    stage slots the consumer reads (stage_neighbour_slots) holds, by the
//    content the producer's tensor copies put there (stage_box_origin and
//    the box extents), exactly the neighbour that neighbours() names.
#include <cstdio>
#include <vector>

#include "tm_stage.cuh"

using namespace twm;

static Geom geom(int lx, int ly, int lz, int lt)
{
    Geom g{};
    g.lx = lx, g.ly = ly, g.lz = lz, g.lt = lt, g.hx = lx / 2;
    g.vh = unsigned(lx) * ly * lz * lt / 2;
    g.sy = g.hx, g.sz = g.sy * ly, g.st = g.sz * lz;
    geom_set_divisors(g);
    return g;
}

static int check_bands(const Geom &g)
{
    int bad = 0, tried = 0;
    const unsigned plane = unsigned(g.hx) * unsigned(g.ly);
    for (unsigned ts : {128u, 64u, 32u}) {
        if (g.vh % ts) continue;
        for (int zb = 1; zb < g.lz; ++zb) {
            if (g.lz % zb || (plane * unsigned(zb)) % ts) continue;
            BGroup G{};
            G.g = g;
            G.zband = zb;
            const unsigned nt = g.vh / ts;
            std::vector<int> hits(nt, 0);
            for (unsigned t = 0; t < nt; ++t) {
                const unsigned p = tile_of(G, t, ts);
                if (p >= nt) {
                    printf("FAIL bands %dx%dx%dx%d ts=%u zband=%d: tile %u -> %u out of range\n", g.lx, g.ly, g.lz,
                           g.lt, ts, zb, t, p);
                    return 1;
                }
                ++hits[p];
            }
            for (unsigned t = 0; t < nt; ++t)
                if (hits[t] != 1) ++bad;
            ++tried;
        }
    }
    if (bad) printf("FAIL bands %dx%dx%dx%d: %d tiles not hit once\n", g.lx, g.ly, g.lz, g.lt, bad);
    return bad ? 1 : 0;
}

// The even-odd index the tensor copy of stage box b puts at position pos.
static unsigned slot_site(const Geom &g, const TileBox &B, int b, int pos)
{
    const int bx = b == B_XM || b == B_XP ? 1 : SBX;
    const int by = b == B_YM || b == B_YP ? 1 : 2;
    const int bz = b == B_ZM || b == B_ZP ? 1 : 2;
    const BoxOrigin o = stage_box_origin(g, B, b);
    const int lx = pos % bx, ly = (pos / bx) % by, lz = (pos / (bx * by)) % bz, lt = pos / (bx * by * bz);
    return ((unsigned(o.t + lt) * unsigned(g.lz) + unsigned(o.z + lz)) * unsigned(g.ly) + unsigned(o.y + ly)) *
               unsigned(g.hx) + unsigned(o.x + lx);
}

static int check_stage(const Geom &g)
{
    if (!(g.hx % SBX == 0 && g.ly % 2 == 0 && g.lz % 2 == 0 && g.lt % 2 == 0)) return 0;
    const unsigned nbox = g.vh / STS;
    for (int sbz = 1; sbz <= g.lz / 2; ++sbz) {
        if ((g.lz / 2) % sbz) continue;
        std::vector<int> hits(g.vh, 0);
        for (unsigned t = 0; t < nbox; ++t) {
            const TileBox B = tile_box(g, sbz, t);
            for (int s = 0; s < STS; ++s) {
                const unsigned i = box_site_index(g, B, s);
                if (i >= g.vh) {
                    printf("FAIL boxes %dx%dx%dx%d sbz=%d: site out of range\n", g.lx, g.ly, g.lz, g.lt, sbz);
                    return 1;
                }
                ++hits[i];
                if (sbz != 1) continue;   // the slots do not depend on the order
                for (int p = 0; p < 2; ++p) {
                    Nbrs n;
                    neighbours(g, p, i, n);
                    SPos q[8];
                    stage_neighbour_slots(B, s, i, n, q);
                    for (int k = 0; k < 8; ++k) {
                        const int mu = k >> 1;
                        const unsigned want = (k & 1) ? n.bwd[mu] : n.fwd[mu];
                        if (q[k].pos < 0 || q[k].pos >= box_sites(q[k].box)) {
                            printf("FAIL slots %dx%dx%dx%d: slot outside its box\n", g.lx, g.ly, g.lz, g.lt);
                            return 1;
                        }
                        const unsigned got = slot_site(g, B, q[k].box, q[k].pos);
                        if (got != want) {
                            printf("FAIL slots %dx%dx%dx%d p=%d site %u hop %d: slot holds %u, neighbour is %u\n",
                                   g.lx, g.ly, g.lz, g.lt, p, i, k, got, want);
                            return 1;
                        }
                    }
                }
            }
        }
        for (unsigned i = 0; i < g.vh; ++i)
            if (hits[i] != 1) {
                printf("FAIL boxes %dx%dx%dx%d sbz=%d: site %u covered %d times\n", g.lx, g.ly, g.lz, g.lt, sbz, i,
                       hits[i]);
                return 1;
            }
    }
    return 0;
}

int main()
{
    const int shapes[][4] = {{16, 2, 2, 2},  {16, 2, 2, 4},  {32, 4, 6, 8},   {16, 4, 4, 4},   {32, 2, 2, 2},
                             {16, 16, 16, 32}, {48, 6, 4, 10}, {8, 8, 8, 8},  {32, 32, 32, 64}, {12, 12, 12, 24},
                             {6, 4, 2, 10},  {64, 2, 4, 2}};
    int fails = 0;
    for (const auto &d : shapes) {
        const Geom g = geom(d[0], d[1], d[2], d[3]);
        fails += check_bands(g);
        fails += check_stage(g);
    }
    if (fails) {
        printf("%d failures\n", fails);
        return 1;
    }
    printf("OK\n");
    return 0;
}
