// gom_kernels.cuh -- declarations of the kernels in gom_kernels.cu for the
// host code that launches them and builds the per-generation CUDA graph.
#pragma once

#include <cuda_runtime.h>

#include "gom_internal.h"

__global__ void k_init_pop(GomParams P);
__global__ void k_fitness(GomParams P, int64_t *out);
__global__ void k_elite_init(GomParams P);
__global__ void k_set_state(GomParams P, int64_t fe, int64_t g);
__global__ void k_begin_call(GomParams P, int64_t target);
__global__ void k_gen_start(GomParams P);
__global__ void k_order(GomParams P);
// The mixing kernel instance for WPI words per warp item (1, 2 or 4) and
// variant (kVarNarrow: 32-bit masks and deltas; kVarWide: 64-bit masks and
// deltas; kVarHuge: 128-bit masks and 64-bit deltas, WPI <= 2, no learned
// filter), with or without the learned filter's bookkeeping; a host-stub
// address usable as a graph-node function, or null for a combination that
// has no instance.
const void *gom_mix_kernel(int wpi, int variant, bool learn);
// The persistent generation kernel k_run<WPI, mask, delta, learn>(GomParams,
// int G, int64_t target), with the same instances (null where none).
const void *gom_run_kernel(int wpi, int variant, bool learn);
// The bit-sliced path (gom_bs.cu): the persistent generation kernel
// k_run_bs<R, learn>(GomParams, int G, int64_t target) and the per-group
// mixing kernel k_mix_bs<R, learn>(GomParams, int t) for bit-plane
// accumulators of R bits (12 or 16; null beyond), with or without the learned
// filter's select phase and bookkeeping, and the shared-memory words of one warp's region
// for staged row blocks of `sm` words, `nc` packed pattern words per
// individual and `w` population words per variable row.
const void *gom_run_bs_kernel(int r, bool learn);
const void *gom_mix_bs_kernel(int r, bool learn);
int gom_bs_warp_words(int sm, int nc, int w);
// Forced Improvement on the per-launch path: which = 0 k_fi_elite(GomParams)
// (one block of 1024), 1 k_fi_start(GomParams), 2 k_fi_group<R>(GomParams,
// int t) (256 threads), 3 k_fi_finish(GomParams).
const void *gom_fi_kernel(int which, int r);
// Batched path: instances on block ranges of one cooperative launch.
// k_batch<MINB>(const GomParams *Ps, const GomBatchInst *inst, GomBarrier *bars, int B, int G, int f_words),
// registers cut for MINB (2 or 3) resident blocks of 256 threads.
const void *gom_batch_kernel(int minb);
__global__ void k_batch_collect(const GomParams *Ps, GomBatchInst *inst, int B);
__global__ void k_barrier_selftest(GomBarrier *bar, int *err, int extra, unsigned long long limit_ns);
__global__ void k_gen_end(GomParams P);
// The learned filter's select phase on the graph path: decisions (and with
// `compact` each warp's count of elements to run; 256 threads), the scan of
// the counts over `nwarps` warps (one block of up to 1024 threads), and the
// compacted list (the decision kernel's grid).
__global__ void k_filter_select(GomParams P, int compact);
__global__ void k_filter_scan(GomParams P, int nwarps);
__global__ void k_filter_compact(GomParams P);
__global__ void k_export_pop(GomParams P, uint8_t *out);
__global__ void k_export_elite(GomParams P, uint8_t *out);
__global__ void k_import_pop(GomParams P, const uint8_t *in, const uint8_t *elite);
