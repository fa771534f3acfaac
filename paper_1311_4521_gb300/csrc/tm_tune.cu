// tm_tune.cu -- the autotuner of the single-lattice hop: which output sites
// each CTA computes (a run of whole rows, or a box of the lattice) and how
// many threads it has, chosen per lattice and storage format by timing every
// candidate, and kept in a cache file keyed by (GPU, lattice, storage,
// reconstruction, right-hand sides) so that later processes skip the timing.
//
// The paper measured how to distribute the hopping matrix's sites over
// threads and processes (Sec. 2.3, the threads-per-process study; Sec. 2.2,
// the hopping-order index g_hi that fixed the memory access order): the best
// decomposition was found by measurement.  Here the candidates are site-to-
// thread maps of one launch; all of them compute every site with the same
// arithmetic, so the choice changes the time and never the result.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "tm_internal.h"

using namespace twm;

namespace {

std::string map_name(const SiteMap &m)
{
    char b[64];
    if (!m.tiled) snprintf(b, sizeof b, "linear%u", m.block);
    else snprintf(b, sizeof b, "box%ux%ux%ux%u", 1u << m.lg[0], 1u << m.lg[1], 1u << m.lg[2], 1u << m.lg[3]);
    return b;
}

// Parses a name written by map_name for lattice g; false if it does not apply.
bool parse_map(const Geom &g, const std::string &name, SiteMap &m)
{
    unsigned a, b, c, d;
    if (sscanf(name.c_str(), "linear%u", &a) == 1 && name == "linear" + std::to_string(a)) {
        if (a < 32 || a > 128 || a % 32) return false;
        m = linear_map(a);
        return true;
    }
    if (sscanf(name.c_str(), "box%ux%ux%ux%u", &a, &b, &c, &d) == 4) {
        unsigned ext[4] = {a, b, c, d}, lg[4];
        for (int k = 0; k < 4; ++k) {
            if (ext[k] == 0 || (ext[k] & (ext[k] - 1))) return false;
            lg[k] = 0;
            while ((1u << lg[k]) < ext[k]) ++lg[k];
        }
        return tiled_map(g, lg, m);
    }
    return false;
}

// Candidate maps: linear with 128 and 64 threads, and every box of 64 or 128
// sites with at least 4 sites along the x half-row (coalesced runs) and at
// most 8 along each other direction that divides the lattice.
std::vector<SiteMap> candidates(const Geom &g)
{
    std::vector<SiteMap> c{linear_map(128), linear_map(64)};
    for (unsigned total = 7; total >= 6; --total)
        for (unsigned l0 = 5; l0 >= 2; --l0)
            for (unsigned l1 = 0; l1 <= 3; ++l1)
                for (unsigned l2 = 0; l2 <= 3; ++l2) {
                    if (l0 + l1 + l2 > total) continue;
                    const unsigned l3 = total - l0 - l1 - l2;
                    if (l3 > 3) continue;
                    const unsigned lg[4] = {l0, l1, l2, l3};
                    SiteMap m;
                    if (!tiled_map(g, lg, m)) continue;
                    // a box as wide as the half-row and stacked only along y is a linear map
                    if (l2 == 0 && l3 == 0 && (1u << l0) == unsigned(g.hx)) continue;
                    c.push_back(m);
                }
    return c;
}

std::string gpu_name(int device)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return "unknown-gpu";
    std::string n = p.name;
    for (char &ch : n)
        if (ch == ' ' || ch == '|') ch = '_';
    return n;
}

std::string cache_key(const tm_ctx *ctx, const tm_gauge *U)
{
    char b[256];
    snprintf(b, sizeof b, "%s|%dx%dx%dx%d|prec%d|recon%d|nrhs1", gpu_name(ctx->device).c_str(), U->dims[0], U->dims[1],
             U->dims[2], U->dims[3], U->prec, U->recon);
    return b;
}

// The map name and time stored for key in the cache file (last entry wins).
bool cache_lookup(const std::string &path, const std::string &key, std::string &name, double &ms)
{
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream ls(line);
        std::string k, n;
        double t = 0;
        if (!(ls >> k >> n >> t)) continue;
        if (k == key) {
            name = n;
            ms = t;
            found = true;
        }
    }
    return found;
}

void cache_store(const std::string &path, const std::string &key, const std::string &name, double ms)
{
    std::ofstream f(path, std::ios::app);
    if (f) f << key << ' ' << name << ' ' << ms << '\n';
}

// Median of three rounds of two launch-B-like hops (even output, fused
// update with x) with map m; ms per launch.
float time_map(const tm_gauge *U, const SiteMap &m, const void *in, void *out, const void *x, cudaStream_t s,
               cudaError_t &err)
{
    cudaEvent_t ev[4];
    for (auto &e : ev) cudaEventCreate(&e);
    const Coef k = coef_qtm_b_unit(0.01);
    err = launch_hop(U->geom, U->prec, U->recon, false, TM_EO, U->links, in, out, x, k, s, m);
    cudaEventRecord(ev[0], s);
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
        for (int q = 0; q < 2 && err == cudaSuccess; ++q)
            err = launch_hop(U->geom, U->prec, U->recon, false, TM_EO, U->links, in, out, x, k, s, m);
        cudaEventRecord(ev[r + 1], s);
    }
    float ms[3] = {1e30f, 1e30f, 1e30f};
    if (err == cudaSuccess) err = cudaEventSynchronize(ev[3]);
    if (err == cudaSuccess)
        for (int r = 0; r < 3; ++r) cudaEventElapsedTime(&ms[r], ev[r], ev[r + 1]);
    for (auto &e : ev) cudaEventDestroy(e);
    std::sort(ms, ms + 3);
    return ms[1] / 2;
}

}  // namespace

namespace twm {

std::string tune_cache_gpu(const tm_ctx *ctx) { return gpu_name(ctx->device); }

bool tune_cache_lookup(const std::string &path, const std::string &key, std::string &value, double &ms)
{
    return cache_lookup(path, key, value, ms);
}

void tune_cache_store(const std::string &path, const std::string &key, const std::string &value, double ms)
{
    cache_store(path, key, value, ms);
}

}  // namespace twm

// Applies the cached map of U's lattice, if the context has a cache file
// with an entry for it (called by tm_gauge_create).
void tm_apply_cached_map(tm_ctx *ctx, tm_gauge *U)
{
    if (!ctx->autotune || ctx->tune_cache.empty()) return;
    std::string name;
    double ms = 0;
    if (!cache_lookup(ctx->tune_cache, cache_key(ctx, U), name, ms)) return;
    SiteMap m;
    if (!parse_map(U->geom, name, m)) return;
    U->map = m;
    U->map_name = name;
}

extern "C" {

tm_status tm_ctx_set_tune_cache(tm_ctx *ctx, const char *path)
{
    if (!ctx) return TM_ERR_ARG;
    ctx->tune_cache = path ? path : "";
    return TM_OK;
}

tm_status tm_gauge_set_map(tm_ctx *ctx, tm_gauge *U, const char *name)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U || !name) return tm_fail(ctx, TM_ERR_ARG, "tm_gauge_set_map: null argument");
    SiteMap m;
    if (!parse_map(U->geom, name, m))
        return tm_fail(ctx, TM_ERR_ARG, std::string("tm_gauge_set_map: '") + name + "' is not a map of this lattice");
    U->map = m;
    U->map_name = map_name(m);
    return TM_OK;
}

size_t tm_gauge_map(const tm_gauge *U, char *buf, size_t size)
{
    if (!U) return 0;
    const std::string &n = U->map_name;
    if (buf && size > 0) {
        const size_t k = std::min(n.size(), size - 1);
        memcpy(buf, n.data(), k);
        buf[k] = '\0';
    }
    return n.size() + 1;
}

tm_status tm_gauge_tune(tm_ctx *ctx, tm_gauge *U, void *stream)
{
    if (!ctx) return TM_ERR_ARG;
    if (!U) return tm_fail(ctx, TM_ERR_ARG, "tm_gauge_tune: null gauge handle");
    const std::string key = cache_key(ctx, U);
    if (!ctx->tune_cache.empty()) {
        std::string name;
        double ms = 0;
        SiteMap m;
        if (cache_lookup(ctx->tune_cache, key, name, ms) && parse_map(U->geom, name, m)) {
            U->map = m;
            U->map_name = name;
            ctx->tuned_maps[key] = "map=" + name + " (cache)";
            return TM_OK;
        }
    }
    if (!ctx->autotune) {
        U->map = linear_map(128);
        U->map_name = "linear128";
        return TM_OK;
    }
    // three fields of the lattice in the context's workspace: input, output, x
    const size_t fb = align256(spinor_bytes(U->geom.vh, U->prec));
    void *base = nullptr;
    tm_status st = tm_ctx_workspace(ctx, 3 * fb, &base);
    if (st != TM_OK) return st;
    char *c = static_cast<char *>(base);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(c, 0x3c, 3 * fb, s);   // finite values in every format
    if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_gauge_tune: ") + cudaGetErrorString(e));
    const std::vector<SiteMap> cand = candidates(U->geom);
    float best = 1e30f, base_ms = 0.f;
    size_t best_k = 0;
    for (size_t k = 0; k < cand.size(); ++k) {
        const float ms = time_map(U, cand[k], c, c + fb, c + 2 * fb, s, e);
        if (e != cudaSuccess) return tm_fail(ctx, TM_ERR_CUDA, std::string("tm_gauge_tune: ") + cudaGetErrorString(e));
        if (k == 0) base_ms = ms;
        if (ms < best) {
            best = ms;
            best_k = k;
        }
    }
    U->map = cand[best_k];
    U->map_name = map_name(cand[best_k]);
    char line[160];
    snprintf(line, sizeof line, "map=%s ms=%.4f linear128_ms=%.4f gain=%.3f candidates=%zu", U->map_name.c_str(), best,
             base_ms, base_ms / best, cand.size());
    ctx->tuned_maps[key] = line;
    if (!ctx->tune_cache.empty()) cache_store(ctx->tune_cache, key, U->map_name, best);
    return TM_OK;
}

}  // extern "C"
