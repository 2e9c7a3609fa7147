// gom_api.cu -- the C ABI declared in include/gom.h: handles, workspace
// layout, uploads, the per-generation CUDA graph and the exports.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "gom_ctx.h"
#include "gom_internal.h"
#include "gom_kernels.cuh"

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxMixBlocks = 8192;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int words_for(int32_t p)
{
    int wv = (p + 31) / 32, w = 1;
    while (w < wv) w <<= 1;
    return w;
}

// Byte offsets of every device array inside the workspace.
struct Layout {
    size_t O, P, f, eqw, xe, st, bar, trace, stats, order, work;
    size_t fi_accw, fi_eq, fi_act0, fi_imp, fi_stale, fi_f0;
    size_t row_ptr, col, wgt, hdr, fv, wout, wabs, seg, dep, cptr;
    size_t total;
};

Layout make_layout(int64_t n, int32_t p, int64_t nadj, int64_t m, int64_t total_vars, int64_t ndeps,
                   int32_t k)
{
    const int64_t W = words_for(p);
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + std::max<size_t>(bytes, 1));
        return at;
    };
    L.O = take(sizeof(uint32_t) * n * W);
    L.P = take(sizeof(uint32_t) * n * W);
    L.f = take(sizeof(int64_t) * 32 * W);
    L.eqw = take(sizeof(uint32_t) * 2 * W);
    L.xe = take(n);
    L.st = take(sizeof(GomDevState));
    L.bar = take(sizeof(GomBarrier));
    L.trace = take(sizeof(unsigned long long) * (5 + 2 * static_cast<size_t>(std::max<int32_t>(k, 1))));
    L.stats = take(sizeof(GomDevStats) * kStatsCap);
    L.order = take(sizeof(int32_t) * std::max<int32_t>(k, 1));
    L.work = take(sizeof(uint32_t) * std::max<int32_t>(k, 1));
    L.fi_accw = take(sizeof(uint32_t) * W);
    L.fi_eq = take(sizeof(uint32_t) * W);
    L.fi_act0 = take(sizeof(uint32_t) * W);
    L.fi_imp = take(sizeof(uint32_t) * W * std::max<int32_t>(k, 1));
    L.fi_stale = take(sizeof(int32_t) * 32 * W);
    L.fi_f0 = take(sizeof(int64_t) * 32 * W);
    L.row_ptr = take(sizeof(int64_t) * (n + 1));
    L.col = take(sizeof(int32_t) * nadj);
    L.wgt = take(sizeof(int32_t) * nadj);
    L.hdr = take(sizeof(int32_t) * 8 * m);
    L.fv = take(sizeof(int32_t) * total_vars);
    L.wout = take(sizeof(int64_t) * total_vars);
    L.wabs = take(sizeof(int32_t) * total_vars);
    L.seg = take(sizeof(uint32_t) * (total_vars + m));
    L.dep = take(sizeof(int32_t) * 2 * ndeps);
    L.cptr = take(sizeof(int32_t) * (std::max<int32_t>(k, 0) + 1));
    L.total = off;
    return L;
}

template <class T>
cudaError_t upload(void *base, size_t off, const std::vector<T> &v, cudaStream_t s)
{
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(static_cast<char *>(base) + off, v.data(), sizeof(T) * v.size(),
                           cudaMemcpyHostToDevice, s);
}

cudaError_t upload_raw(void *base, size_t off, const void *src, size_t bytes, cudaStream_t s)
{
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(static_cast<char *>(base) + off, src, bytes, cudaMemcpyHostToDevice, s);
}

// Adds a kernel node after `dep` (may be null) and returns it.
cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t *node, cudaGraphNode_t dep, const void *fn,
                       int grid, int block, size_t smem, void **args)
{
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(fn);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = static_cast<unsigned>(smem);
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

// One generation as a chain of nodes: gen_start, order, k mixing launches,
// gen_end.  With `timed`, event records bracket every mixing launch.
int build_graph(gom_ctx *ctx, bool timed, cudaGraph_t *out_graph, cudaGraphExec_t *out_exec)
{
    cudaGraph_t g;
    GOM_CUDA(ctx, cudaGraphCreate(&g, 0));
    GomParams prm = ctx->prm;
    void *args1[] = {&prm};
    cudaGraphNode_t last = nullptr, node;
    cudaError_t e = add_kernel(g, &node, last, (const void *)k_gen_start, ctx->grid_start, 256, 0, args1);
    if (e == cudaSuccess) {
        last = node;
        e = add_kernel(g, &node, last, (const void *)k_order, ctx->grid_order, 256, ctx->order_smem, args1);
    }
    // the learned filter's select phase: decisions, and for the bit-sliced
    // path while it skips, the compacted list of the elements to run
    int compact = prm.learn == 2 && prm.flt.compact ? 1 : 0;
    int sel_warps = 0;
    const int sel_grid = std::max(1, ctx->sms * 8); // 64 warps per SM: the size of the count array
    if (e == cudaSuccess && prm.learn) {
        void *argsS[] = {&prm, &compact};
        last = node;
        e = add_kernel(g, &node, last, (const void *)k_filter_select, sel_grid, 256, 0, argsS);
        sel_warps = sel_grid * 8;
        if (e == cudaSuccess && compact) {
            void *argsC[] = {&prm, &sel_warps};
            last = node;
            e = add_kernel(g, &node, last, (const void *)k_filter_scan, 1, 1024, 0, argsC);
            if (e == cudaSuccess) {
                last = node;
                e = add_kernel(g, &node, last, (const void *)k_filter_compact, sel_grid, 256, 0, args1);
            }
        }
    }
    std::vector<int> ts(ctx->k);
    for (int t = 0; t < ctx->k && e == cudaSuccess; ++t) {
        last = node;
        if (timed) {
            e = cudaGraphAddEventRecordNode(&node, g, &last, 1, ctx->events[2 * t]);
            if (e != cudaSuccess) break;
            last = node;
        }
        ts[t] = t;
        void *args2[] = {&prm, &ts[t]};
        if (use_bs(ctx))
            e = add_kernel(g, &node, last, ctx->mix_bs_fn, ctx->bs_grid_mix, ctx->bs_threads, ctx->bs_smem, args2);
        else
            e = add_kernel(g, &node, last, ctx->mix_fn, ctx->grid_mix, ctx->mix_threads, ctx->mix_smem, args2);
        if (e == cudaSuccess && timed) {
            last = node;
            e = cudaGraphAddEventRecordNode(&node, g, &last, 1, ctx->events[2 * t + 1]);
        }
    }
    std::vector<int> fts(ctx->prm.fi.on ? ctx->k : 0);
    if (e == cudaSuccess && ctx->prm.fi.on) { // Forced Improvement after the mixing
        last = node;
        e = add_kernel(g, &node, last, gom_fi_kernel(0, ctx->fi_r), 1, 1024, 0, args1);
        if (e == cudaSuccess) {
            last = node;
            e = add_kernel(g, &node, last, gom_fi_kernel(1, ctx->fi_r), ctx->grid_start, 256, 0, args1);
        }
        for (int t = 0; t < ctx->k && e == cudaSuccess; ++t) {
            last = node;
            fts[t] = t;
            void *args3[] = {&prm, &fts[t]};
            e = add_kernel(g, &node, last, gom_fi_kernel(2, ctx->fi_r), ctx->fi_grid, 256, 0, args3);
        }
        if (e == cudaSuccess) {
            last = node;
            e = add_kernel(g, &node, last, gom_fi_kernel(3, ctx->fi_r), ctx->grid_start, 256, 0, args1);
        }
    }
    if (e == cudaSuccess) {
        last = node;
        e = add_kernel(g, &node, last, (const void *)k_gen_end, 1, 1024, 0, args1);
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e);
    }
    *out_graph = g;
    *out_exec = ex;
    return GOM_OK;
}



int accumulate_timing(gom_ctx *ctx)
{
    if (!ctx->timing_pending) return GOM_OK;
    ctx->timing_pending = false;
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int t = 0; t < ctx->k; ++t) {
        float ms = 0.f;
        GOM_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->events[2 * t], ctx->events[2 * t + 1]));
        ctx->mix_ms += ms;
    }
    return GOM_OK;
}

} // namespace

// Rebuilds the per-generation graphs after a change of the parameters they
// copy (the timed variant only if it exists).  Waits for the stream.
int rebuild_graphs(gom_ctx *ctx)
{
    // the learned filter's counting unit and list mode follow the mixing path in use
    ctx->prm.flt.compact = use_bs(ctx) ? 1 : 0;
    ctx->prm.flt.items_per_elem =
        use_bs(ctx) || !ctx->prm.split ? 1 : (ctx->prm.Wv + ctx->wpi - 1) / std::max(ctx->wpi, 1);
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const bool had_timed = ctx->texec != nullptr;
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->texec) cudaGraphExecDestroy(ctx->texec);
    if (ctx->tgraph) cudaGraphDestroy(ctx->tgraph);
    ctx->exec = ctx->texec = nullptr;
    ctx->graph = ctx->tgraph = nullptr;
    int rc = build_graph(ctx, false, &ctx->graph, &ctx->exec);
    if (rc == GOM_OK && had_timed) rc = build_graph(ctx, true, &ctx->tgraph, &ctx->texec);
    return rc;
}

// The counters of the generations of the context's last call (host_stats
// may be null), and their number.  Waits for the stream.
int ctx_read_stats(gom_ctx *ctx, int32_t num, gom_gen_stats_t *host_stats, int32_t *run_out)
{
    GomDevState st;
    GOM_CUDA(ctx, cudaMemcpyAsync(&st, ctx->prm.st, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (st.err) return GOM_E_TIMEOUT;
    const int32_t run = static_cast<int32_t>(st.g - st.call_g0);
    if (run_out) *run_out = run;
    if (host_stats) {
        std::memset(host_stats, 0, sizeof(gom_gen_stats_t) * num);
        std::vector<GomDevStats> ring(kStatsCap);
        GOM_CUDA(ctx, cudaMemcpyAsync(ring.data(), ctx->prm.stats, sizeof(GomDevStats) * kStatsCap,
                                      cudaMemcpyDeviceToHost, ctx->stream));
        GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int32_t q = 0; q < run && q < num; ++q) {
            const GomDevStats &S = ring[(st.call_g0 + q) % kStatsCap];
            gom_gen_stats_t &H = host_stats[q];
            H.generation = S.generation;
            H.best_fitness = S.best;
            H.elite_fitness = S.elite;
            H.trials = S.trials;
            H.donorless = S.donorless;
            H.accepted = S.accepted;
            H.improving = S.improving;
            H.reached_target = S.reached;
            H.fi_individuals = S.fi_individuals;
            H.fi_trials = S.fi_trials;
            H.fi_accepted = S.fi_accepted;
            H.fi_improving = S.fi_improving;
            H.fi_replaced = S.fi_replaced;
        }
    }
    return GOM_OK;
}

extern "C" {

const char *gom_strerror(int code)
{
    switch (code) {
    case GOM_OK: return "ok";
    case GOM_E_ARG: return "invalid argument";
    case GOM_E_GRAPH: return "graph is not a simple symmetric CSR with sorted rows";
    case GOM_E_NOT_COLORED: return "FOS has not been coloured";
    case GOM_E_WORKSPACE: return "workspace missing, misaligned or too small";
    case GOM_E_CUDA: return "CUDA call failed";
    case GOM_E_TIMEOUT: return "bounded device wait gave up";
    case GOM_E_STATE: return "call not valid in this state";
    case GOM_E_LIMIT: return "size beyond the library's limits";
    case GOM_E_FOS: return "FOS incomplete, out of range or for another graph";
    default: return "unknown error";
    }
}

int gom_build_fos(const gom_graph_t *g, int32_t kind, int32_t param, gom_fos_t **out)
{
    if (!g || !out) return GOM_E_ARG;
    if (kind == GOM_FOS_BFLT ? param < 1 : param != 0) return GOM_E_ARG;
    if (kind != GOM_FOS_NEIGHBOURHOOD && kind != GOM_FOS_SINGLETON && kind != GOM_FOS_BFLT) return GOM_E_ARG;
    int rc = gomh::validate_graph(g);
    if (rc) return rc;
    std::unique_ptr<gom_fos> fos(new (std::nothrow) gom_fos());
    if (!fos) return GOM_E_ARG;
    rc = kind == GOM_FOS_BFLT ? gomh::build_bflt(g, param, fos.get()) : gomh::build_fos(g, kind, fos.get());
    if (rc) return rc;
    *out = fos.release();
    return GOM_OK;
}

int gom_fos_create(int32_t num_vars, int64_t m, const int64_t *elem_ptr, const int32_t *elem_vars,
                   gom_fos_t **out)
{
    if (!out || num_vars < 0 || m < 0 || !elem_ptr || (m > 0 && !elem_vars)) return GOM_E_ARG;
    std::unique_ptr<gom_fos> fos(new (std::nothrow) gom_fos());
    if (!fos) return GOM_E_ARG;
    fos->n = num_vars;
    fos->m = m;
    fos->eptr.assign(elem_ptr, elem_ptr + m + 1);
    if (fos->eptr[0] != 0 || fos->eptr[m] < 0) return GOM_E_FOS;
    for (int64_t j = 0; j < m; ++j)
        if (fos->eptr[j + 1] < fos->eptr[j]) return GOM_E_FOS;
    fos->evars.assign(elem_vars, elem_vars + fos->eptr[m]);
    int rc = gomh::check_fos(num_vars, *fos);
    if (rc) return rc;
    *out = fos.release();
    return GOM_OK;
}

int gom_color_fos(const gom_graph_t *g, gom_fos_t *fos, int32_t *num_colors)
{
    if (!g || !fos) return GOM_E_ARG;
    int rc = gomh::validate_graph(g);
    if (rc) return rc;
    if (fos->n != g->num_vertices) return GOM_E_FOS;
    rc = gomh::color_fos(g, fos);
    if (rc) return rc;
    if (num_colors) *num_colors = fos->k;
    return GOM_OK;
}

int gom_fos_sizes(const gom_fos_t *fos, int64_t *m, int64_t *total_vars, int32_t *k)
{
    if (!fos) return GOM_E_ARG;
    if (m) *m = fos->m;
    if (total_vars) *total_vars = static_cast<int64_t>(fos->evars.size());
    if (k) *k = fos->k;
    return GOM_OK;
}

int gom_fos_export(const gom_fos_t *fos, int64_t *elem_ptr, int32_t *elem_vars, int32_t *color_of_elem,
                   int64_t *color_ptr, int32_t *color_elems)
{
    if (!fos) return GOM_E_ARG;
    if ((color_of_elem || color_ptr || color_elems) && fos->k < 0) return GOM_E_NOT_COLORED;
    if (elem_ptr) std::copy(fos->eptr.begin(), fos->eptr.end(), elem_ptr);
    if (elem_vars) std::copy(fos->evars.begin(), fos->evars.end(), elem_vars);
    if (color_of_elem) std::copy(fos->color_of.begin(), fos->color_of.end(), color_of_elem);
    if (color_ptr) std::copy(fos->cptr.begin(), fos->cptr.end(), color_ptr);
    if (color_elems) std::copy(fos->celems.begin(), fos->celems.end(), color_elems);
    return GOM_OK;
}

void gom_fos_destroy(gom_fos_t *fos) { delete fos; }

size_t gom_workspace_bytes(const gom_graph_t *g, const gom_fos_t *fos, int32_t pop)
{
    if (!g || !fos || pop < 2 || pop > GOM_MAX_POPULATION || g->num_vertices < 0) return 0;
    if (fos->n != g->num_vertices || !g->row_ptr) return 0;
    const int64_t ndeps = gomh::count_deps(g, *fos);
    return make_layout(g->num_vertices, pop, g->num_adj, fos->m, static_cast<int64_t>(fos->evars.size()),
                       ndeps, std::max<int32_t>(fos->k, 1))
        .total;
}

int gom_init_population(const gom_graph_t *g, const gom_fos_t *fos, int32_t pop, uint64_t seed,
                        void *d_workspace, size_t ws_bytes, void *cuda_stream, gom_ctx_t **out)
{
    if (!g || !fos || !out) return GOM_E_ARG;
    if (pop < 2) return GOM_E_ARG;
    if (pop > GOM_MAX_POPULATION) return GOM_E_LIMIT;
    int rc = gomh::validate_graph(g);
    if (rc) return rc;
    if (fos->n != g->num_vertices) return GOM_E_FOS;
    if (fos->k < 0) return GOM_E_NOT_COLORED;
    if (fos->k > GOM_MAX_COLORS) return GOM_E_LIMIT;
    if (static_cast<int64_t>(fos->evars.size()) + fos->m >= INT_MAX || fos->m >= INT_MAX) return GOM_E_LIMIT;
    for (int64_t j = 0; j < fos->m; ++j)
        if (fos->eptr[j + 1] - fos->eptr[j] > GOM_MAX_ELEMENT) return GOM_E_LIMIT;
    const int64_t ndeps_bound = gomh::count_deps(g, *fos);
    const Layout L = make_layout(g->num_vertices, pop, g->num_adj, fos->m,
                                 static_cast<int64_t>(fos->evars.size()), ndeps_bound, fos->k);
    if (!d_workspace || ws_bytes < L.total || reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
        return GOM_E_WORKSPACE;

    gomh::ElemTables tabs;
    rc = gomh::build_elem_tables(g, *fos, &tabs);
    if (rc) return rc;
    if (static_cast<int64_t>(g->num_vertices) * words_for(pop) >= INT_MAX) return GOM_E_LIMIT;

    std::unique_ptr<gom_ctx> ctx(new (std::nothrow) gom_ctx());
    if (!ctx) return GOM_E_ARG;
    gom_ctx *c = ctx.get();
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->n = g->num_vertices;
    c->p = pop;
    c->W = words_for(pop);
    c->m = fos->m;
    c->k = fos->k;

    // kernel instance: words per item, mask and delta widths
    const int32_t variant = kernel_variant(tabs.max_s, tabs.max_abs_w);
    int64_t max_group = 1;
    for (int32_t q = 0; q < fos->k; ++q) max_group = std::max(max_group, fos->cptr[q + 1] - fos->cptr[q]);
    int dev = 0;
    GOM_CUDA(c, cudaGetDevice(&dev));
    GOM_CUDA(c, cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
    // Work split for the whole grid (~24 resident warps per SM).
    const int wv = (pop + 31) / 32;
    int wpi = 1, split = 0;
    item_split(c->W, pop, max_group, static_cast<int64_t>(c->sms) * 24, variant, &wpi, &split);
    // Block mode (the 128-bit instances, 4 or more word groups per element):
    // the warps of a block stage each element once, together, and share its
    // word groups -- rather than every (element, word group) item staging the
    // element's rows and pattern table (both grow with the population) on its own.
    const bool blk = variant == kVarHuge && (wv + wpi - 1) / wpi >= 4;
    if (blk) split = 0;
    const int nwg = (wv + wpi - 1) / wpi;
    const int per = split ? nwg : 1;
    c->mix_fn = gom_mix_kernel(wpi, variant, false);
    const SliceLayout SL = slice_layout(tabs.max_s, tabs.max_edges, c->W, wpi, variant, split != 0, nwg);
    const int64_t off_fv = SL.off_fv, off_seg = SL.off_seg, off_wout = SL.off_wout, off_pr = SL.off_pr;
    const int64_t off_pat = SL.off_pat, off_rs = SL.off_rs, off_ds = SL.off_ds;
    const int64_t base_words = SL.base_words;
    const int64_t all_words = SL.all_words;
    const int64_t xw_words = SL.off_ds - SL.off_xw; // one warp's region of outside neighbours' words
    constexpr int64_t kSmemBudget = 200 * 1024;
    int warps_per_block = 0;
    if (blk) { // one slice per block plus a region of outside words per further warp
        warps_per_block = std::min(kMixThreads / 32, nwg);
        while (warps_per_block > 1 && (base_words + (warps_per_block - 1) * xw_words) * 4 > kSmemBudget)
            --warps_per_block;
        if (base_words * 4 > kSmemBudget) warps_per_block = 0;
    } else {
        warps_per_block = static_cast<int>(std::min<int64_t>(kMixThreads / 32, kSmemBudget / (base_words * 4)));
    }
    if (warps_per_block < 1) return GOM_E_LIMIT;
    c->mix_threads = 32 * warps_per_block;
    // shared-memory words of a block's staging outside stage-all mode
    const int64_t block_words =
        blk ? base_words + (warps_per_block - 1) * xw_words : base_words * warps_per_block;
    // one warp per item (a block per element in block mode) of the largest group, at most a full wave
    const int64_t need_blocks = blk ? max_group : (max_group * per + warps_per_block - 1) / warps_per_block;

    // persistent path: one cooperative kernel, grid limited to co-resident blocks
    c->run_fn = gom_run_kernel(wpi, variant, false);
    const size_t keys_smem = sizeof(unsigned long long) * static_cast<size_t>(std::max(c->k, 1));
    int coop = 0;
    GOM_CUDA(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    auto run_grid = [&](size_t smem_bytes, int *out_grid) -> cudaError_t {
        *out_grid = 0;
        if (smem_bytes > static_cast<size_t>(kSmemBudget)) return cudaSuccess;
        cudaError_t e = raise_smem_limit(c->run_fn, smem_bytes);
        if (e != cudaSuccess) return e;
        int occ_run = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_run, c->run_fn, c->mix_threads, smem_bytes);
        if (e != cudaSuccess) return e;
        *out_grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(c->sms) * occ_run,
                                                       std::max<int64_t>(need_blocks, 1)));
        return cudaSuccess;
    };
    int64_t warp_words = base_words;
    if (coop) {
        // stage_all: every warp stages its item of every colour group at the
        // start of a generation -- when each group fits in one wave of warps,
        // the k slices per warp fit in shared memory and k is small enough
        // for every block to hold the group order
        const size_t all_smem = static_cast<size_t>(c->k) * all_words * 4 * warps_per_block;
        int grid_all = 0;
        if (c->k <= kStageAllMaxK && !blk) GOM_CUDA(c, run_grid(all_smem, &grid_all));
        if (grid_all > 0 && max_group * per <= static_cast<int64_t>(grid_all) * warps_per_block) {
            c->run_smem = all_smem;
            c->grid_run = grid_all;
            c->prm.stage_all = 1;
            c->can_persist = true;
            warp_words = all_words;
        } else {
            const size_t one_smem = std::max(keys_smem, static_cast<size_t>(block_words * 4));
            int grid_one = 0;
            GOM_CUDA(c, run_grid(one_smem, &grid_one));
            if (grid_one > 0) {
                c->run_smem = one_smem;
                c->grid_run = grid_one;
                c->prm.stage_all = 0;
                c->can_persist = true;
            }
        }
    }
    c->mix_smem = static_cast<size_t>(c->prm.stage_all ? all_words * 4 * warps_per_block : block_words * 4);
    if (blk) warp_words = block_words; // the block's one slice
    GOM_CUDA(c, raise_smem_limit(c->mix_fn, c->mix_smem));
    int occ = 0;
    GOM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->mix_fn, c->mix_threads, c->mix_smem));
    occ = std::max(occ, 1);
    int64_t grid = std::min<int64_t>(static_cast<int64_t>(c->sms) * occ, need_blocks);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxMixBlocks));
    c->grid_mix = static_cast<int>(grid);
    c->persistent = c->can_persist;
    c->wpi = wpi;
    c->variant = variant;
    c->max_items = std::max<int64_t>(1, max_group * per);
    c->max_group = max_group;
    c->celems.assign(fos->celems.begin(), fos->celems.end());
    c->max_s = tabs.max_s;
    c->max_edges = tabs.max_edges;
    for (int64_t q = 0; q < c->m; ++q) {
        const int32_t *h = tabs.hdr.data() + 8 * q;
        c->sum_se += (h[3] & 0xFF) + (h[3] >> 8) + h[4];
    }
    // the bit-sliced path: elements of <= 32 variables, |w| <= 255, element
    // sums of |w| below 2^16 (R-bit plane accumulators, R = 12 or 16); an item
    // is E = 32 / W elements, one pair (element, word) per lane
    int64_t max_w = 0;
    for (int64_t x = 0; x < g->num_adj; ++x) max_w = std::max<int64_t>(max_w, std::llabs(g->weight[x]));
    // Forced Improvement works on bit-planes too: |w| <= 255 and element sums of |w| below 2^16
    c->fi_ok = max_w <= 255 && tabs.max_abs_w < (int64_t(1) << 16);
    c->fi_r = tabs.max_abs_w < (int64_t(1) << 12) ? 12 : 16;
    if (c->fi_ok) {
        int occ_f = 0;
        GOM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, gom_fi_kernel(2, c->fi_r), 256, 0));
        c->fi_grid = std::max(1, c->sms * std::max(occ_f, 1));
    }
    {
        const int R = tabs.max_abs_w < (int64_t(1) << 12) ? 12 : 16;
        if (coop && variant == kVarNarrow && max_w <= 255 && tabs.max_abs_w < (int64_t(1) << 16)) {
            const int sm = static_cast<int>(std::max<int64_t>(tabs.max_s, 1) | 1); // odd row stride: no bank conflicts
            const int S = static_cast<int>(std::max<int64_t>(tabs.max_s, 1));
            const int epw = 32 / S, E0 = 32 / c->W;
            const int nc = (E0 + epw - 1) / epw;
            const int64_t ww = gom_bs_warp_words(sm, nc, c->W);
            const int wpb = static_cast<int>(std::min<int64_t>(kBsThreads / 32, kSmemBudget / (ww * 4)));
            // the block's fitness accumulators (32 W int64), then the warps' regions
            const size_t smem = std::max(static_cast<size_t>(256 * c->W + ww * 4 * wpb), keys_smem);
            // the kernels without the learned filter's code, and with it (same grids)
            const void *rf = gom_run_bs_kernel(R, false), *mf = gom_mix_bs_kernel(R, false);
            const void *rfl = gom_run_bs_kernel(R, true), *mfl = gom_mix_bs_kernel(R, true);
            if (wpb >= 1 && smem <= static_cast<size_t>(kSmemBudget) && rf && mf && rfl && mfl) {
                const int E = 32 / c->W;
                const int64_t items = (max_group + E - 1) / E;
                const int64_t need = std::max<int64_t>(1, (items + wpb - 1) / wpb);
                for (const void *fn : {rf, mf, rfl, mfl}) GOM_CUDA(c, raise_smem_limit(fn, smem));
                int occ_r = 0, occ_m = 0, occ_rl = 0, occ_ml = 0;
                GOM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_r, rf, 32 * wpb, smem));
                GOM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_m, mf, 32 * wpb, smem));
                GOM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_rl, rfl, 32 * wpb, smem));
                GOM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ml, mfl, 32 * wpb, smem));
                occ_r = std::min(occ_r, occ_rl);
                occ_m = std::min(occ_m, occ_ml);
                if (occ_r > 0 && occ_m > 0) {
                    c->bs_r = R;
                    c->bs_ok = true;
                    c->run_bs_fn = rf;
                    c->mix_bs_fn = mf;
                    c->bs_smem = smem;
                    c->bs_threads = 32 * wpb;
                    c->bs_grid_run = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(c->sms) * occ_r, need));
                    c->bs_grid_mix = static_cast<int>(std::min<int64_t>(
                        std::min<int64_t>(static_cast<int64_t>(c->sms) * occ_m, need), kMaxMixBlocks));
                    c->prm.bs_sm = sm;
                    c->prm.bs_S = S;
                    c->prm.bs_epw = epw;
                    c->prm.bs_nc = nc;
                    c->prm.bs_words = static_cast<int32_t>(ww);
                    // the default where the largest group gives at least a quarter of the
                    // resident warps an item, and a variable row has at most 16 words: with
                    // fewer items the per-lane path's finer items win, and with 32 words
                    // (one element per item) its scalar trials do (measured on the torus,
                    // 3D torus and random regular workloads, p = 64 to 1024)
                    c->bs_on = c->W <= 16 && 4 * items >= static_cast<int64_t>(c->sms) * occ_r * wpb;
                }
            }
        }
    }
    // dynamic item claims: faster warps take more items (in stage-all mode
    // every warp has at most one item per group and the schedule is moot)
    c->prm.dyn = 1;
    const int blk_mult = std::max(1, c->W / 8);
    c->grid_fit = std::max(blk_mult, c->sms * 4 / blk_mult * blk_mult);
    c->grid_start = c->sms * 4;
    c->grid_io = c->sms * 4;
    c->grid_order = (c->k + 255) / 256;
    c->order_smem = sizeof(unsigned long long) * std::max(c->k, 1);
    if (c->order_smem > 48 * 1024)
        GOM_CUDA(c, raise_smem_limit((const void *)k_order, c->order_smem));

    char *base = static_cast<char *>(d_workspace);
    c->base = base;
    c->state_bytes = L.row_ptr;
    GomParams &P = c->prm;
    P.n = c->n;
    P.p = pop;
    P.W = c->W;
    P.Wv = (pop + 31) / 32;
    P.m = static_cast<int32_t>(fos->m);
    P.k = fos->k;
    P.seed = seed;
    for (int r = 0; r < 10; ++r) { // Philox4x32-10 round keys (the published Weyl increments)
        P.rk[2 * r] = static_cast<uint32_t>(seed) + static_cast<uint32_t>(r) * 0x9E3779B9u;
        P.rk[2 * r + 1] = static_cast<uint32_t>(seed >> 32) + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
    P.split = split;
    P.blk = blk ? 1 : 0;
    P.xw_words = static_cast<int32_t>(xw_words);
    P.warp_smem = static_cast<int32_t>(warp_words);
    P.off_fv = static_cast<int32_t>(off_fv);
    P.off_seg = static_cast<int32_t>(off_seg);
    P.off_wout = static_cast<int32_t>(off_wout);
    P.off_pr = static_cast<int32_t>(off_pr);
    P.off_pat = static_cast<int32_t>(off_pat);
    P.off_rs = static_cast<int32_t>(off_rs);
    P.off_cw = static_cast<int32_t>(SL.off_cw);
    P.off_xw = static_cast<int32_t>(SL.off_xw);
    P.off_ds = static_cast<int32_t>(off_ds);
    P.O = reinterpret_cast<uint32_t *>(base + L.O);
    P.P = reinterpret_cast<uint32_t *>(base + L.P);
    P.f = reinterpret_cast<int64_t *>(base + L.f);
    P.eqw = reinterpret_cast<uint32_t *>(base + L.eqw);
    P.xe = reinterpret_cast<uint8_t *>(base + L.xe);
    P.st = reinterpret_cast<GomDevState *>(base + L.st);
    P.bar = reinterpret_cast<GomBarrier *>(base + L.bar);
    c->trace_buf = reinterpret_cast<unsigned long long *>(base + L.trace);
    P.trace = nullptr;
    P.stats = reinterpret_cast<GomDevStats *>(base + L.stats);
    P.order = reinterpret_cast<int32_t *>(base + L.order);
    P.work = reinterpret_cast<uint32_t *>(base + L.work);
    P.fi.on = 0;
    P.fi.nis = 0;
    P.fi.accw = reinterpret_cast<uint32_t *>(base + L.fi_accw);
    P.fi.eq = reinterpret_cast<uint32_t *>(base + L.fi_eq);
    P.fi.act0 = reinterpret_cast<uint32_t *>(base + L.fi_act0);
    P.fi.imp = reinterpret_cast<uint32_t *>(base + L.fi_imp);
    P.fi.stale = reinterpret_cast<int32_t *>(base + L.fi_stale);
    P.fi.f0 = reinterpret_cast<int64_t *>(base + L.fi_f0);
    P.row_ptr = reinterpret_cast<const int64_t *>(base + L.row_ptr);
    P.col = reinterpret_cast<const int32_t *>(base + L.col);
    P.wgt = reinterpret_cast<const int32_t *>(base + L.wgt);
    P.hdr = reinterpret_cast<const int4 *>(base + L.hdr);
    P.fv = reinterpret_cast<const int32_t *>(base + L.fv);
    P.wout = reinterpret_cast<const int64_t *>(base + L.wout);
    P.wabs = reinterpret_cast<const int32_t *>(base + L.wabs);
    P.seg = reinterpret_cast<const uint32_t *>(base + L.seg);
    P.dep = reinterpret_cast<const int2 *>(base + L.dep);
    P.cptr = reinterpret_cast<const int32_t *>(base + L.cptr);

    // uploads (host vectors outlive the copies: the stream is synchronised below)
    std::vector<int32_t> cptr32(fos->cptr.begin(), fos->cptr.end());
    cudaStream_t s = c->stream;
    GOM_CUDA(c, cudaMemsetAsync(base, 0, L.row_ptr, s)); // all state arrays
    GOM_CUDA(c, upload_raw(base, L.row_ptr, g->row_ptr, sizeof(int64_t) * (c->n + 1), s));
    GOM_CUDA(c, upload_raw(base, L.col, g->col, sizeof(int32_t) * g->num_adj, s));
    GOM_CUDA(c, upload_raw(base, L.wgt, g->weight, sizeof(int32_t) * g->num_adj, s));
    GOM_CUDA(c, upload(base, L.hdr, tabs.hdr, s));
    GOM_CUDA(c, upload(base, L.fv, tabs.fv, s));
    GOM_CUDA(c, upload(base, L.wout, tabs.wout, s));
    GOM_CUDA(c, upload(base, L.wabs, tabs.wabs, s));
    GOM_CUDA(c, upload(base, L.seg, tabs.seg, s));
    GOM_CUDA(c, upload(base, L.dep, tabs.dep, s));
    GOM_CUDA(c, upload(base, L.cptr, cptr32, s));

    k_init_pop<<<c->grid_io, 256, 0, s>>>(P);
    GOM_CUDA(c, cudaGetLastError());
    k_fitness<<<c->grid_fit, 256, 0, s>>>(P, P.f);
    GOM_CUDA(c, cudaGetLastError());
    k_elite_init<<<1, 1024, 0, s>>>(P);
    GOM_CUDA(c, cudaGetLastError());

    c->events.resize(2 * static_cast<size_t>(std::max(c->k, 1)), nullptr);
    for (auto &ev : c->events) GOM_CUDA(c, cudaEventCreate(&ev));
    rc = build_graph(c, false, &c->graph, &c->exec);
    if (rc) {
        gom_destroy(ctx.release());
        return rc;
    }
    GOM_CUDA(c, cudaStreamSynchronize(s));
    *out = ctx.release();
    return GOM_OK;
}

int gom_generation(gom_ctx_t *ctx, int32_t num_generations, int64_t target_fitness,
                   gom_gen_stats_t *host_stats, int32_t *generations_run)
{
    if (!ctx || num_generations < 0) return GOM_E_ARG;
    int32_t done_total = 0;
    int32_t remaining = num_generations;
    gom_gen_stats_t *stats_out = host_stats;
    const bool want = host_stats || generations_run;
    do {
        // with host statistics the device ring bounds one chunk
        const int32_t chunk = want ? std::min<int32_t>(remaining, kStatsCap) : remaining;
        if (ctx->persistent && !ctx->timing) {
            GomParams prm = ctx->prm;
            int gens = chunk;
            int64_t target = target_fitness;
            void *args[] = {&prm, &gens, &target};
            if (use_bs(ctx))
                GOM_CUDA(ctx, cudaLaunchCooperativeKernel(ctx->run_bs_fn, dim3(ctx->bs_grid_run), dim3(ctx->bs_threads),
                                                          args, ctx->bs_smem, ctx->stream));
            else
                GOM_CUDA(ctx, cudaLaunchCooperativeKernel(ctx->run_fn, dim3(ctx->grid_run), dim3(ctx->mix_threads),
                                                          args, ctx->run_smem, ctx->stream));
        } else {
            k_begin_call<<<1, 1, 0, ctx->stream>>>(ctx->prm, target_fitness);
            GOM_CUDA(ctx, cudaGetLastError());
        }
        for (int32_t q = 0; q < chunk && !(ctx->persistent && !ctx->timing); ++q) {
            if (ctx->timing) {
                // the events of the previous timed generation are read first
                int rc = accumulate_timing(ctx);
                if (rc) return rc;
                GOM_CUDA(ctx, cudaGraphLaunch(ctx->texec, ctx->stream));
                ctx->timing_pending = true;
            } else {
                GOM_CUDA(ctx, cudaGraphLaunch(ctx->exec, ctx->stream));
            }
        }
        remaining -= chunk;
        if (want) {
            int32_t run = 0;
            int rc = ctx_read_stats(ctx, chunk, stats_out, &run);
            if (rc) return rc;
            done_total += run;
            if (stats_out) stats_out += chunk;
            if (run < chunk) { // target reached: zero the rest
                if (stats_out) std::memset(stats_out, 0, sizeof(gom_gen_stats_t) * remaining);
                break;
            }
        }
    } while (remaining > 0);
    if (generations_run) *generations_run = done_total;
    return GOM_OK;
}

int gom_fitness(gom_ctx_t *ctx, int64_t *d_fitness_out)
{
    if (!ctx || !d_fitness_out) return GOM_E_ARG;
    GOM_CUDA(ctx, cudaMemsetAsync(d_fitness_out, 0, sizeof(int64_t) * ctx->p, ctx->stream));
    k_fitness<<<ctx->grid_fit, 256, 0, ctx->stream>>>(ctx->prm, d_fitness_out);
    GOM_CUDA(ctx, cudaGetLastError());
    return GOM_OK;
}

int gom_get_population(gom_ctx_t *ctx, uint8_t *d_pop, int64_t *d_fit, int64_t *elite_f)
{
    if (!ctx) return GOM_E_ARG;
    if (d_pop) {
        k_export_pop<<<ctx->grid_io, 256, 0, ctx->stream>>>(ctx->prm, d_pop);
        GOM_CUDA(ctx, cudaGetLastError());
    }
    if (d_fit)
        GOM_CUDA(ctx, cudaMemcpyAsync(d_fit, ctx->prm.f, sizeof(int64_t) * ctx->p, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    if (elite_f) {
        GomDevState st;
        GOM_CUDA(ctx, cudaMemcpyAsync(&st, ctx->prm.st, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
        GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        *elite_f = st.fe;
    }
    return GOM_OK;
}

int gom_get_elite(gom_ctx_t *ctx, uint8_t *d_elite, int64_t *elite_f)
{
    if (!ctx) return GOM_E_ARG;
    if (d_elite) {
        k_export_elite<<<ctx->grid_io, 256, 0, ctx->stream>>>(ctx->prm, d_elite);
        GOM_CUDA(ctx, cudaGetLastError());
    }
    return gom_get_population(ctx, nullptr, nullptr, elite_f);
}

int gom_set_population(gom_ctx_t *ctx, const uint8_t *d_pop, const uint8_t *d_elite, int64_t elite_f,
                       int64_t generation)
{
    if (!ctx || !d_pop || !d_elite || generation < 0 || generation > UINT32_MAX) return GOM_E_ARG;
    k_import_pop<<<ctx->grid_io, 256, 0, ctx->stream>>>(ctx->prm, d_pop, d_elite);
    GOM_CUDA(ctx, cudaGetLastError());
    GOM_CUDA(ctx, cudaMemsetAsync(ctx->prm.f, 0, sizeof(int64_t) * 32 * ctx->W, ctx->stream));
    k_fitness<<<ctx->grid_fit, 256, 0, ctx->stream>>>(ctx->prm, ctx->prm.f);
    GOM_CUDA(ctx, cudaGetLastError());
    k_set_state<<<1, 256, 0, ctx->stream>>>(ctx->prm, elite_f, generation);
    GOM_CUDA(ctx, cudaGetLastError());
    return GOM_OK;
}

int gom_get_generation(gom_ctx_t *ctx, int64_t *generation)
{
    if (!ctx || !generation) return GOM_E_ARG;
    GomDevState st;
    GOM_CUDA(ctx, cudaMemcpyAsync(&st, ctx->prm.st, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (st.err) return GOM_E_TIMEOUT;
    *generation = st.g;
    return GOM_OK;
}

int gom_set_timing(gom_ctx_t *ctx, int32_t enable)
{
    if (!ctx) return GOM_E_ARG;
    if (enable && !ctx->texec) {
        int rc = build_graph(ctx, true, &ctx->tgraph, &ctx->texec);
        if (rc) return rc;
    }
    int rc = accumulate_timing(ctx);
    if (rc) return rc;
    if (enable && !ctx->timing) {
        ctx->mix_ms = 0.0;
        rc = gom_get_generation(ctx, &ctx->timing_g0);
        if (rc) return rc;
    }
    ctx->timing = enable != 0;
    return GOM_OK;
}

int gom_read_timing(gom_ctx_t *ctx, double *mix_ms, int64_t *mix_launches)
{
    if (!ctx) return GOM_E_ARG;
    int rc = accumulate_timing(ctx);
    if (rc) return rc;
    int64_t g = 0;
    rc = gom_get_generation(ctx, &g);
    if (rc) return rc;
    if (mix_ms) *mix_ms = ctx->mix_ms;
    if (mix_launches) *mix_launches = (g - ctx->timing_g0) * ctx->k;
    ctx->mix_ms = 0.0;
    ctx->timing_g0 = g;
    return GOM_OK;
}

int gom_launches_per_generation(gom_ctx_t *ctx, int64_t *launches)
{
    if (!ctx || !launches) return GOM_E_ARG;
    *launches = (ctx->persistent && !ctx->timing)
                    ? 1
                    : 3 + static_cast<int64_t>(ctx->k) + (ctx->prm.fi.on ? 3 + static_cast<int64_t>(ctx->k) : 0);
    return GOM_OK;
}

int gom_set_option(gom_ctx_t *ctx, int32_t option, int64_t value)
{
    if (!ctx) return GOM_E_ARG;
    if (option == GOM_OPT_PERSISTENT) {
        if (value && !ctx->can_persist) return GOM_E_STATE;
        ctx->persistent = value != 0;
        return GOM_OK;
    }
    if (option == GOM_OPT_PHASE_TRACE) {
        ctx->prm.trace = value ? ctx->trace_buf : nullptr;
        return GOM_OK;
    }
    if (option == GOM_OPT_DYNAMIC) {
        if (value != 0 && value != 1) return GOM_E_ARG;
        if (ctx->prm.dyn == value) return GOM_OK;
        ctx->prm.dyn = static_cast<int32_t>(value);
        return rebuild_graphs(ctx); // the graphs hold a copy of the parameters
    }
    if (option == GOM_OPT_BITSLICED) {
        if (value != 0 && value != 1) return GOM_E_ARG;
        if (value && !ctx->bs_ok) return GOM_E_STATE;
        ctx->bs_set = static_cast<int>(value); // batched launches follow it too
        if (ctx->bs_on == (value != 0)) return GOM_OK;
        ctx->bs_on = value != 0;
        return rebuild_graphs(ctx); // the graphs hold the mixing kernel
    }
    if (option == GOM_OPT_FORCED_IMPROVEMENT) {
        if (value != 0 && value != 1) return GOM_E_ARG;
        if (value && !ctx->fi_ok) return GOM_E_LIMIT;
        if (ctx->prm.fi.on == value) return GOM_OK;
        if (value) // no generation without improvement counted yet
            GOM_CUDA(ctx, cudaMemsetAsync(ctx->prm.fi.stale, 0, sizeof(int32_t) * 32 * ctx->W, ctx->stream));
        ctx->prm.fi.on = static_cast<int32_t>(value);
        return rebuild_graphs(ctx); // the graphs hold the parameters and the FI nodes
    }
    if (option == GOM_OPT_FI_NIS) {
        if (value < 0 || value > INT32_MAX) return GOM_E_ARG;
        ctx->prm.fi.nis = static_cast<int32_t>(value);
        return rebuild_graphs(ctx);
    }
    if (option == GOM_OPT_FILTER_LABEL) {
        if (value < 0 || value > 1) return GOM_E_ARG;
        ctx->prm.flt.label = static_cast<int32_t>(value);
        return rebuild_graphs(ctx);
    }
    return GOM_E_ARG;
}

int gom_get_option(gom_ctx_t *ctx, int32_t option, int64_t *value)
{
    if (!ctx || !value) return GOM_E_ARG;
    if (option == GOM_OPT_PERSISTENT) {
        *value = ctx->persistent ? 1 : 0;
        return GOM_OK;
    }
    if (option == GOM_OPT_PHASE_TRACE) {
        *value = ctx->prm.trace ? 1 : 0;
        return GOM_OK;
    }
    if (option == GOM_OPT_DYNAMIC) {
        *value = ctx->prm.dyn;
        return GOM_OK;
    }
    if (option == GOM_OPT_BITSLICED) {
        *value = ctx->bs_on ? 1 : 0;
        return GOM_OK;
    }
    if (option == GOM_OPT_FORCED_IMPROVEMENT) {
        *value = ctx->prm.fi.on;
        return GOM_OK;
    }
    if (option == GOM_OPT_FI_NIS) {
        *value = ctx->prm.fi.nis;
        return GOM_OK;
    }
    if (option == GOM_OPT_FILTER_LABEL) {
        *value = ctx->prm.flt.label;
        return GOM_OK;
    }
    return GOM_E_ARG;
}

int gom_read_phase_trace(gom_ctx_t *ctx, int64_t *ns, int32_t capacity, int32_t *count)
{
    if (!ctx || capacity < 0) return GOM_E_ARG;
    const int32_t n = 5 + 2 * ctx->k;
    if (count) *count = n;
    if (!ns || capacity < n) return GOM_E_ARG;
    GOM_CUDA(ctx, cudaMemcpyAsync(ns, ctx->trace_buf, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    GOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GOM_OK;
}

int gom_selftest_barrier(void *d_scratch, int32_t blocks, int32_t extra, int64_t limit_ns, void *cuda_stream,
                         int32_t *timed_out)
{
    if (!d_scratch || blocks < 1 || extra < 0 || limit_ns <= 0 || !timed_out) return GOM_E_ARG;
    if (reinterpret_cast<uintptr_t>(d_scratch) % 16) return GOM_E_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, coop = 0;
    GOM_CUDA(nullptr, cudaGetDevice(&dev));
    GOM_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GOM_CUDA(nullptr, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return GOM_E_STATE;
    if (blocks > sms) return GOM_E_LIMIT;
    GomBarrier *bar = static_cast<GomBarrier *>(d_scratch);
    int *err = reinterpret_cast<int *>(static_cast<char *>(d_scratch) + sizeof(GomBarrier));
    GOM_CUDA(nullptr, cudaMemsetAsync(d_scratch, 0, sizeof(GomBarrier) + sizeof(int), s));
    unsigned long long lim = static_cast<unsigned long long>(limit_ns);
    int ex = extra;
    void *args[] = {&bar, &err, &ex, &lim};
    GOM_CUDA(nullptr, cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(blocks), dim3(32), args, 0, s));
    int herr = 0;
    GOM_CUDA(nullptr, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GOM_CUDA(nullptr, cudaStreamSynchronize(s));
    *timed_out = herr != 0;
    return GOM_OK;
}

int gom_last_cuda_error(gom_ctx_t *ctx) { return ctx ? ctx->last_cuda : 0; }

void gom_destroy(gom_ctx_t *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->texec) cudaGraphExecDestroy(ctx->texec);
    if (ctx->tgraph) cudaGraphDestroy(ctx->tgraph);
    for (auto ev : ctx->events)
        if (ev) cudaEventDestroy(ev);
    delete ctx;
}

} // extern "C"
