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
    bool narrow = true;          // 32-bit masks and deltas
    int64_t max_items = 1;       // mixing items of the largest colour group
    double work = 0.0;           // cost estimate of one generation (trial-weighted element sizes)
    char *base = nullptr;        // the workspace
    size_t state_bytes = 0;      // its state arrays: [0, state_bytes) (population, fitness, elitist, ...)
};


inline int cuda_fail(gom_ctx *ctx, cudaError_t e)
{
    if (ctx) ctx->last_cuda = static_cast<int>(e);
    return GOM_E_CUDA;
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
