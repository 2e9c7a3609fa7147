// gom_ctx.h -- the context handle behind gom_ctx_t and the CUDA error
// helper, shared by the C ABI's translation units (gom_api.cu, gom_batch.cu).
#pragma once

#include <vector>

#include <cuda_runtime.h>

#include "gom_internal.h"

struct gom_ctx {
    GomParams prm{};
    cudaStream_t stream = nullptr;
    int32_t n = 0, p = 0, W = 0, k = 0;
    int64_t m = 0;
    int sms = 0;
    int grid_mix = 0, grid_fit = 0, grid_start = 0, grid_order = 0, grid_io = 0;
    const void *mix_fn = nullptr; // k_mix instance for this population and FOS
    size_t mix_smem = 0;          // its dynamic shared memory per block
    int mix_threads = kMixThreads; // its block size (fewer warps for very large elements)
    const void *run_fn = nullptr; // persistent generation kernel (same instance parameters)
    size_t run_smem = 0;          // its dynamic shared memory (staging or the k group keys)
    int grid_run = 0;             // its grid: co-resident blocks only
    bool can_persist = false;     // cooperative launch available and the sizes fit
    bool persistent = false;      // current path: k_run (true) or the per-generation graph
    // the bit-sliced mixing path (gom_bs.cu), where the FOS and weights allow it
    bool bs_ok = false;           // available for this context
    bool bs_on = false;           // selected (GOM_OPT_BITSLICED)
    int bs_set = -1;              // GOM_OPT_BITSLICED as the caller set it (-1: never set; batched launches
                                  //   then choose by the instance's share of warps)
    const void *run_bs_fn = nullptr, *mix_bs_fn = nullptr; // the instances for the learned filter's mode
    int bs_r = 0;                 // their accumulator width R
    size_t bs_smem = 0;           // dynamic shared memory of both (warp regions, group keys)
    int bs_threads = 0;           // their block size
    int bs_grid_run = 0, bs_grid_mix = 0;
    // Forced Improvement (GOM_OPT_FORCED_IMPROVEMENT)
    bool fi_ok = false;           // available: |w| <= 255, element sums of |w| below 2^16
    int fi_r = 16;                // bit-plane width of its accumulators
    int fi_grid = 0;              // grid of its per-group kernel on the per-launch path
    unsigned long long *trace_buf = nullptr; // workspace slot of the phase trace
    size_t order_smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t tgraph = nullptr; // variant with event records around each mixing launch
    cudaGraphExec_t texec = nullptr;
    std::vector<cudaEvent_t> events;
    bool timing = false;
    bool timing_pending = false; // the events hold a generation not yet added to mix_ms
    double mix_ms = 0.0;
    int64_t timing_g0 = 0;       // generation counter when timing was (re)started
    int last_cuda = 0;
    // for batched launches (gom_batch_*)
    int wpi = 1;                 // words per mixing item
    int32_t variant = kVarNarrow; // kernel variant (mask and delta widths)
    int64_t max_items = 1;       // mixing items of the largest colour group
    double sum_se = 0.0;         // sum over elements of (variables + edges)
    int64_t max_group = 1;       // elements of the largest colour group
    int64_t max_s = 0;           // variables of the largest element
    int64_t max_edges = 0;       // most edges of one element
    std::vector<int32_t> celems; // element index at each colour-order position
    char *filter_base = nullptr; // learned-filter workspace (gom_filter_attach), or null
    int64_t filter_cap = 0;      // its training-log capacity
    char *base = nullptr;        // the workspace
    size_t state_bytes = 0;      // its state arrays: [0, state_bytes) (population, fitness, elitist, ...)
};


// The bit-sliced path runs the context's generations (selected and
// available; the learned filter works on either path).
inline bool use_bs(const gom_ctx *ctx) { return ctx->bs_on; }

inline int cuda_fail(gom_ctx *ctx, cudaError_t e)
{
    if (ctx) ctx->last_cuda = static_cast<int>(e);
    return GOM_E_CUDA;
}

// One staging slice (one mixing item) in shared memory -- the one definition
// of its layout; the kernels take these offsets (32-bit words): an 8-word
// item header, the element's variables, their outside-edge starts (s+1),
// their outside weight sums (int64), the rows of P on the element (W words
// each), the pattern table (32 W masks of 4, 8 or 16 bytes), its run starts (W
// words), each edge's {code, weight} (two words), each outside edge's parent
// words (WPI words), and in stage-all mode the item's donor start positions
// (one int per individual of its words).  Every offset is a multiple of 4
// words.
struct SliceLayout {
    int64_t off_fv, off_seg, off_wout, off_pr, off_pat, off_rs, off_cw, off_xw, off_ds;
    int64_t base_words; // a slice without the donor starts
    int64_t all_words;  // with them (stage-all mode)
};

inline SliceLayout slice_layout(int64_t max_s, int64_t max_edges, int W, int wpi, int32_t variant, bool split,
                                int nwg)
{
    auto round4 = [](int64_t x) { return (x + 3) & ~int64_t(3); };
    SliceLayout L{};
    L.off_fv = 8;
    L.off_seg = L.off_fv + round4(max_s);
    L.off_wout = L.off_seg + round4(max_s + 1);
    L.off_pr = L.off_wout + round4(2 * max_s);
    L.off_pat = L.off_pr + round4(max_s * W);
    L.off_rs = L.off_pat + int64_t(32) * W * (variant == kVarNarrow ? 1 : variant == kVarWide ? 2 : 4);
    L.off_cw = L.off_rs + round4(W);
    L.off_xw = L.off_cw + round4(2 * max_edges);
    L.off_ds = L.off_xw + round4(max_edges * wpi);
    L.base_words = L.off_ds;
    L.all_words = L.off_ds + int64_t(32) * wpi * (split ? 1 : nwg);
    return L;
}

// Words per item and split mode for p individuals when `warps` warps share
// the items of the largest colour group of `max_group` elements: one warp per
// element walking all its words in groups of min(W, 4) words, or, with fewer
// than about 4 elements per warp, one warp per (element, word group) so that
// the warps stay busy (then single words if the population has only one
// group of min(W, 4) words).  The kernel variant for elements of more than
// 64 variables has instances for groups of at most 2 words.
inline void item_split(int W, int32_t p, int64_t max_group, int64_t warps, int32_t variant, int *wpi, int *split)
{
    const int wv = (p + 31) / 32;
    const int most = variant == kVarHuge ? 2 : 4;
    *wpi = W < most ? W : most;
    *split = 0;
    if (max_group < 4 * warps && wv > 1) {
        *split = 1;
        if ((wv + *wpi - 1) / *wpi == 1) *wpi = 1;
    }
}

// Raises a kernel's dynamic shared memory limit to at least `bytes`, never
// lowers it: kernel instances are shared by every context (and batch), and a
// limit lowered below what an existing context launches with would make its
// launches fail.
inline cudaError_t raise_smem_limit(const void *fn, size_t bytes)
{
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

#define GOM_CUDA(ctx, call)                               \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_); \
    } while (0)

// The counters of the generations of the context's last call into
// host_stats[0..num) (may be null) and their number (*run_out).  Waits for
// the stream.  GOM_E_TIMEOUT if the context's device error word is set.
int ctx_read_stats(gom_ctx *ctx, int32_t num, gom_gen_stats_t *host_stats, int32_t *run_out);

// Rebuilds the per-generation graphs after a change of the parameters they
// copy (the timed variant only if it exists).  Waits for the stream.
int rebuild_graphs(gom_ctx *ctx);
