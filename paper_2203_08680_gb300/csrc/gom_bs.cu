// gom_bs.cu -- the kernels of the bit-sliced mixing path (gom_bs.cuh): the
// persistent generation kernel, the per-group mixing kernel of the
// per-generation graph, and the Forced Improvement kernels of that graph.
#include <climits>
#include <cuda_runtime.h>

#include "gom_bs.cuh"
#include "gom_internal.h"
#include "gom_kernels.cuh"

namespace {

// Persistent path on the bit-sliced phase: up to G generations in one
// cooperative launch (bs_generations on the whole grid).  The dynamic shared
// memory holds the block's fitness accumulators, then the warps' regions (the
// k group keys of the order phase overlay them).
template <int R, bool LEARN>
__global__ void __launch_bounds__(kBsThreads, 5) k_run_bs(GomParams P, int G, int64_t target)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    __shared__ unsigned long long s_cnt[4], s_fc[4];
    bs_generations<R, LEARN>(P, whole_grid(), P.bar, G, target, reinterpret_cast<unsigned long long *>(s_dyn),
                             bs_warp_region(P, s_dyn), reinterpret_cast<long long *>(s_dyn), s_cnt, s_fc);
}

// Per-launch path: the mixing of the group at position t (one launch per
// group in the per-generation CUDA graph).
template <int R, bool LEARN>
__global__ void __launch_bounds__(kBsThreads, 5) k_mix_bs(GomParams P, int t)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    __shared__ unsigned long long s_cnt[4], s_fc[4];
    long long *s_f = reinterpret_cast<long long *>(s_dyn);
    if (P.st->done) return;
    fc_zero(s_fc);
    acc_zero(P, s_f, s_cnt);
    BsLane L;
    bs_lane_zero(L);
    uint32_t *wsm = bs_warp_region(P, s_dyn);
    phase_mix_bs<R, LEARN>(P, whole_grid(), t, P.order[t], P.st->g, wsm, L, s_f, s_fc);
    bs_finish_generation(P, L, s_f, s_cnt);
    acc_flush(P, s_f, s_cnt);
    if (LEARN) fc_flush(P, s_fc);
}

// Forced Improvement on the per-launch path (one CUDA graph per
// generation): the elitist update of its start (one block), the start
// (flags, x_e, the set of individuals in FI), one launch per group, the end.
__global__ void __launch_bounds__(1024) k_fi_elite(GomParams P)
{
    if (P.st->done) return;
    int64_t best;
    int arg;
    block_argmax(P.f, P.p, &best, &arg);
    if (threadIdx.x == 0) {
        const bool newel = best > P.st->fe;
        if (newel) {
            P.st->fe = best;
            P.st->argmax = arg;
            P.st->improved = 1;
        }
        P.st->fi_newel = newel ? 1 : 0;
    }
}

__global__ void k_fi_start(GomParams P)
{
    if (P.st->done) return;
    fi_start(P, whole_grid(), P.st->fi_newel != 0, P.st->argmax >> 5, P.st->argmax & 31, blockIdx.x == 0);
}

template <int R>
__global__ void __launch_bounds__(kMixThreads, 2) k_fi_group(GomParams P, int t)
{
    __shared__ long long s_f[1024];
    __shared__ unsigned long long s_cnt[4];
    __shared__ uint32_t s_act[32];
    if (P.st->done) return;
    if (threadIdx.x < 32) {
        uint32_t done = 0;
        if ((int)threadIdx.x < P.W)
            for (int t2 = 0; t2 < t; ++t2) done |= P.fi.imp[(int64_t)t2 * P.W + threadIdx.x];
        s_act[threadIdx.x] = (int)threadIdx.x < P.W ? P.fi.act0[threadIdx.x] & ~done : 0u;
    }
    acc_zero(P, s_f, s_cnt);
    BsLane L;
    bs_lane_zero(L);
    unsigned cnt[3] = {0, 0, 0};
    fi_group<R>(P, whole_grid(), t, P.order[t], s_act, L, cnt, s_f);
    bs_flush(P, L, s_f);
    fi_count_flush(P, cnt);
    acc_flush(P, s_f, s_cnt);
}

__global__ void k_fi_finish(GomParams P)
{
    __shared__ uint32_t s_rep[32];
    if (P.st->done) return;
    if (threadIdx.x < 32) {
        uint32_t done = 0;
        if ((int)threadIdx.x < P.W)
            for (int t2 = 0; t2 < P.k; ++t2) done |= P.fi.imp[(int64_t)t2 * P.W + threadIdx.x];
        s_rep[threadIdx.x] = (int)threadIdx.x < P.W ? P.fi.act0[threadIdx.x] & ~done : 0u;
    }
    __syncthreads();
    fi_finish(P, whole_grid(), s_rep, P.st->fe, blockIdx.x == 0);
}

} // namespace

const void *gom_fi_kernel(int which, int r)
{
    switch (which) {
    case 0: return (const void *)k_fi_elite;
    case 1: return (const void *)k_fi_start;
    case 2: return r <= 12 ? (const void *)k_fi_group<12> : (const void *)k_fi_group<16>;
    default: return (const void *)k_fi_finish;
    }
}

int gom_bs_warp_words(int sm, int nc, int w) { return bs_warp_words(sm, nc, w); }

const void *gom_run_bs_kernel(int r, bool learn)
{
    if (learn) return r <= 12 ? (const void *)k_run_bs<12, true> : r <= 16 ? (const void *)k_run_bs<16, true> : nullptr;
    return r <= 12 ? (const void *)k_run_bs<12, false> : r <= 16 ? (const void *)k_run_bs<16, false> : nullptr;
}

const void *gom_mix_bs_kernel(int r, bool learn)
{
    if (learn) return r <= 12 ? (const void *)k_mix_bs<12, true> : r <= 16 ? (const void *)k_mix_bs<16, true> : nullptr;
    return r <= 12 ? (const void *)k_mix_bs<12, false> : r <= 16 ? (const void *)k_mix_bs<16, false> : nullptr;
}
