// Host-side check of the hop's index arithmetic (compiled with nvcc as a
// host program; no GPU needed): every linear and box map of several lattice
// shapes covers every even-odd site exactly once, the division by
// invariant integers used for the boxes and the site coordinates is exact,
// and every site's 8 neighbour indices and wrap flags agree with plain
// coordinate arithmetic.
#include <cstdio>
#include <vector>

#include "tm_device.cuh"

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

static int check_map(const Geom &g, const SiteMap &m, const char *what)
{
    std::vector<int> hits(g.vh, 0);
    const unsigned grid = map_grid(g, m);
    for (unsigned b = 0; b < grid; ++b)
        for (unsigned k = 0; k < m.block; ++k) {
            const unsigned i = map_site(g, m, b, k);
            if (i < g.vh) ++hits[i];
            else if (m.tiled) {
                printf("FAIL %s %dx%dx%dx%d: box map leaves the lattice (b=%u k=%u i=%u)\n", what, g.lx, g.ly, g.lz,
                       g.lt, b, k, i);
                return 1;
            }
        }
    for (unsigned i = 0; i < g.vh; ++i)
        if (hits[i] != 1) {
            printf("FAIL %s %dx%dx%dx%d: site %u covered %d times\n", what, g.lx, g.ly, g.lz, g.lt, i, hits[i]);
            return 1;
        }
    return 0;
}

// neighbours() against coordinates decoded by plain division and the
// neighbour indices recomputed from them, for both parities and all sites.
static int check_neighbours(const Geom &g)
{
    for (int p = 0; p < 2; ++p)
        for (unsigned i = 0; i < g.vh; ++i) {
            Nbrs n;
            neighbours(g, p, i, n);
            const unsigned xh = i % g.hx, y = (i / g.hx) % g.ly, z = (i / g.hx / g.ly) % g.lz,
                           t = i / g.hx / g.ly / g.lz;
            const unsigned x = 2 * xh + ((y + z + t + p) & 1);
            const int ext[4] = {g.lt, g.lx, g.ly, g.lz};
            const unsigned c[4] = {t, x, y, z};
            for (int mu = 0; mu < 4; ++mu)
                for (int step = -1; step <= 1; step += 2) {
                    unsigned cc[4] = {c[0], c[1], c[2], c[3]};
                    cc[mu] = unsigned((int(cc[mu]) + step + ext[mu]) % ext[mu]);
                    const unsigned lex = cc[1] + g.lx * (cc[2] + g.ly * (cc[3] + g.lz * cc[0]));
                    const bool wrap = int(c[mu]) + step < 0 || int(c[mu]) + step >= ext[mu];
                    const unsigned got = step > 0 ? n.fwd[mu] : n.bwd[mu];
                    const bool gotw = step > 0 ? n.wf[mu] : n.wb[mu];
                    if (got != lex / 2 || gotw != wrap) {
                        printf("FAIL neighbours %dx%dx%dx%d p=%d i=%u mu=%d step=%d\n", g.lx, g.ly, g.lz, g.lt, p, i,
                               mu, step);
                        return 1;
                    }
                }
        }
    return 0;
}

int main()
{
    int fails = 0, maps = 0;
    // exact division for every divisor up to 4096 on a sweep of numerators
    for (unsigned d = 1; d <= 4096; ++d) {
        const FastDiv f(d);
        for (unsigned n = 0; n < 70000; n += (n < 5000 ? 1 : 97))
            if (f.div(n) != n / d) {
                printf("FAIL FastDiv %u / %u\n", n, d);
                return 1;
            }
        for (unsigned n = 0x7fffffffu; n > 0x7fff0000u; n -= 4099)
            if (f.div(n) != n / d) {
                printf("FAIL FastDiv %u / %u\n", n, d);
                return 1;
            }
    }
    const int shapes[][4] = {{4, 4, 4, 8},   {8, 8, 8, 16},  {16, 8, 4, 8},  {32, 32, 32, 64},
                             {48, 8, 12, 16}, {24, 24, 8, 8}, {6, 4, 8, 10},  {8, 2, 2, 2}};
    for (const auto &s : shapes) {
        const Geom g = geom(s[0], s[1], s[2], s[3]);
        fails += check_neighbours(g);
        for (unsigned b : {32u, 64u, 96u, 128u}) {
            fails += check_map(g, linear_map(b), "linear");
            ++maps;
        }
        for (unsigned l0 = 0; l0 <= 5; ++l0)
            for (unsigned l1 = 0; l1 <= 3; ++l1)
                for (unsigned l2 = 0; l2 <= 3; ++l2)
                    for (unsigned l3 = 0; l3 <= 3; ++l3) {
                        const unsigned lg[4] = {l0, l1, l2, l3};
                        SiteMap m;
                        if (!tiled_map(g, lg, m)) continue;
                        fails += check_map(g, m, "box");
                        ++maps;
                    }
    }
    printf("%d maps checked, %d failures\n", maps, fails);
    return fails ? 1 : 0;
}
