// gom_ims.cu -- the Interleaved Multi-start Scheme (Sec. 6.3) on the batched
// path: populations P_0, P_1, ... of base_pop * 2^i individuals, where one
// generation of P_i is made each time P_{i-1} has made c more generations.
// The populations are independent, so an advance of the scheme by `steps`
// generations of P_0 is one batched launch in which P_i makes its share of
// generations; the generation at which the scheme first reaches a target is
// recovered from the populations' counters in the scheme's own order.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "gom_ctx.h"
#include "gom_internal.h"

struct gom_ims {
    std::vector<gom_ctx_t *> pops; // P_0 .. P_{L-1}
    gom_batch_t *batch = nullptr;
    int32_t c = 4;
    int64_t steps = 0; // generations made by P_0
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int32_t num_populations(int32_t base_pop, int32_t max_pop)
{
    int32_t L = 0;
    for (int64_t p = base_pop; p <= max_pop; p *= 2) ++L;
    return L;
}

// Generations population i has made when P_0 has made T: floor(T / c^i).
int64_t gens_at(int64_t T, int32_t c, int32_t i)
{
    for (int32_t q = 0; q < i; ++q) T /= c;
    return T;
}

} // namespace

extern "C" {

size_t gom_ims_workspace_bytes(const gom_graph_t *g, const gom_fos_t *fos, int32_t base_pop, int32_t max_pop)
{
    if (!g || !fos || base_pop < 2 || max_pop < base_pop || max_pop > GOM_MAX_POPULATION) return 0;
    const int32_t L = num_populations(base_pop, max_pop);
    size_t total = 0;
    for (int32_t i = 0; i < L; ++i) {
        const size_t b = gom_workspace_bytes(g, fos, base_pop << i);
        if (!b) return 0;
        total += align_up(b);
    }
    return total + align_up(gom_batch_workspace_bytes(L));
}

int gom_ims_create(const gom_graph_t *g, const gom_fos_t *fos, int32_t base_pop, int32_t c, int32_t max_pop,
                   uint64_t seed, void *d_workspace, size_t ws_bytes, void *cuda_stream, gom_ims_t **out)
{
    if (!g || !fos || !out || base_pop < 2 || c < 1 || max_pop < base_pop) return GOM_E_ARG;
    if (max_pop > GOM_MAX_POPULATION) return GOM_E_LIMIT;
    const size_t need = gom_ims_workspace_bytes(g, fos, base_pop, max_pop);
    if (!need || !d_workspace || ws_bytes < need || reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
        return GOM_E_WORKSPACE;
    std::unique_ptr<gom_ims> ims(new (std::nothrow) gom_ims());
    if (!ims) return GOM_E_ARG;
    ims->c = c;
    const int32_t L = num_populations(base_pop, max_pop);
    char *base = static_cast<char *>(d_workspace);
    size_t off = 0;
    int rc = GOM_OK;
    for (int32_t i = 0; i < L && rc == GOM_OK; ++i) {
        const size_t b = gom_workspace_bytes(g, fos, base_pop << i);
        gom_ctx_t *ctx = nullptr;
        rc = gom_init_population(g, fos, base_pop << i, seed + static_cast<uint64_t>(i), base + off, b, cuda_stream,
                                 &ctx);
        if (rc == GOM_OK) ims->pops.push_back(ctx);
        off += align_up(b);
    }
    if (rc == GOM_OK)
        rc = gom_batch_create(ims->pops.data(), L, nullptr, base + off, ws_bytes - off, cuda_stream, &ims->batch);
    if (rc) {
        for (gom_ctx_t *ctx : ims->pops) gom_destroy(ctx);
        return rc;
    }
    *out = ims.release();
    return GOM_OK;
}

int gom_ims_run(gom_ims_t *ims, int32_t steps, int64_t target, gom_ims_result_t *res)
{
    if (!ims || steps < 0 || steps > kStatsCap) return GOM_E_ARG;
    const int32_t L = static_cast<int32_t>(ims->pops.size());
    const int64_t T0 = ims->steps, T1 = T0 + steps;
    std::vector<int32_t> gens(L);
    std::vector<int64_t> targets(L, target);
    for (int32_t i = 0; i < L; ++i)
        gens[i] = static_cast<int32_t>(gens_at(T1, ims->c, i) - gens_at(T0, ims->c, i));
    std::vector<int32_t> run(L, 0);
    int rc = gom_batch_generation_each(ims->batch, gens.data(), targets.data(), run.data());
    if (rc) return rc;
    ims->steps = T1;
    if (!res) return GOM_OK;
    std::memset(res, 0, sizeof(*res));
    res->steps = T1;
    res->reached_population = -1;
    res->best_fitness = INT64_MIN;
    // the first reach in the scheme's order: P_i's r-th generation of this call
    // happens at step (gens_at(T0) + r) c^i, and within one step P_0 goes first
    int64_t first_step = INT64_MAX;
    std::vector<gom_gen_stats_t> st(kStatsCap);
    for (int32_t i = 0; i < L; ++i) {
        int32_t n = 0;
        rc = ctx_read_stats(ims->pops[i], run[i], st.data(), &n);
        if (rc) return rc;
        int64_t cpow = 1;
        for (int32_t q = 0; q < i; ++q) cpow *= ims->c;
        for (int32_t r = 0; r < n; ++r) {
            res->best_fitness = std::max(res->best_fitness, st[r].best_fitness);
            if (st[r].reached_target) {
                const int64_t at = (gens_at(T0, ims->c, i) + r + 1) * cpow;
                if (at < first_step) {
                    first_step = at;
                    res->reached_population = i;
                    res->reached_generation = st[r].generation;
                }
                break;
            }
        }
    }
    if (res->reached_population >= 0) {
        res->reached = 1;
        res->reached_step = first_step;
    }
    return GOM_OK;
}

int gom_ims_population(gom_ims_t *ims, int32_t i, gom_ctx_t **ctx)
{
    if (!ims || !ctx || i < 0 || i >= static_cast<int32_t>(ims->pops.size())) return GOM_E_ARG;
    *ctx = ims->pops[i];
    return GOM_OK;
}

int32_t gom_ims_num_populations(const gom_ims_t *ims) { return ims ? static_cast<int32_t>(ims->pops.size()) : 0; }

void gom_ims_destroy(gom_ims_t *ims)
{
    if (!ims) return;
    gom_batch_destroy(ims->batch);
    for (gom_ctx_t *ctx : ims->pops) gom_destroy(ctx);
    delete ims;
}

} // extern "C"
