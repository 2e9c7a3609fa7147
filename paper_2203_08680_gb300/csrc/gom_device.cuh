// gom_device.cuh -- device code shared by the kernel translation units:
// Philox4x32-10, the virtual grid of one problem, the bounded grid barrier,
// and the generation-level phases of Alg. 3 (generation start with the
// elitist flags, the random group order, the generation end with the
// elitist update and counters), plus the block accumulators of fitness
// deltas and counters.  Everything is in an anonymous namespace, so each
// translation unit that includes it compiles its own copy.
#pragma once

#include <climits>
#include <cuda_runtime.h>

#include "gom_internal.h"

namespace {


constexpr uint32_t kFull = 0xFFFFFFFFu;

// Per-individual mask of an element's variables in the instances for elements
// of 65 to 128 variables.
using Mask128 = unsigned __int128;

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the published multipliers, the key bumped by the
// published Weyl constants between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same generator with the ten round keys precomputed (rk[2r], rk[2r+1]:
// the key after r bumps), e.g. from the kernel parameters.
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x; // one 32x32 -> 64-bit product each
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                       (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint32_t pick(uint4 r, int q)
{
    return (q & 2) ? ((q & 1) ? r.w : r.z) : ((q & 1) ? r.y : r.x);
}

__device__ __forceinline__ int64_t gthread() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gthreads() { return (int64_t)gridDim.x * blockDim.x; }

// The blocks that run one problem: the whole grid, or, in a batched launch,
// the range of blocks given to one instance (block `blk` of `nblk`).
struct VGrid {
    int blk, nblk;
    __device__ __forceinline__ int64_t thread() const { return (int64_t)blk * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int64_t threads() const { return (int64_t)nblk * blockDim.x; }
};
__device__ __forceinline__ VGrid whole_grid() { return VGrid{(int)blockIdx.x, (int)gridDim.x}; }

// Lowest index of the maximum of f[0..p) over one block (blockDim <= 1024);
// every thread of the block receives the result.
__device__ void block_argmax(const int64_t *f, int p, int64_t *best_out, int *arg_out)
{
    __shared__ long long s_best[32];
    __shared__ int s_arg[32];
    long long best = LLONG_MIN;
    int arg = INT_MAX;
    for (int i = threadIdx.x; i < p; i += blockDim.x)
        if (f[i] > best) {
            best = f[i];
            arg = i;
        }
    for (int off = 16; off; off >>= 1) {
        const long long ob = __shfl_down_sync(kFull, best, off);
        const int oa = __shfl_down_sync(kFull, arg, off);
        if (ob > best || (ob == best && oa < arg)) {
            best = ob;
            arg = oa;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_best[wid] = best;
        s_arg[wid] = arg;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        best = lane < nw ? s_best[lane] : LLONG_MIN;
        arg = lane < nw ? s_arg[lane] : INT_MAX;
        for (int off = 16; off; off >>= 1) {
            const long long ob = __shfl_down_sync(kFull, best, off);
            const int oa = __shfl_down_sync(kFull, arg, off);
            if (ob > best || (ob == best && oa < arg)) {
                best = ob;
                arg = oa;
            }
        }
    }
    __syncthreads(); // every warp has read s_best / s_arg
    if (threadIdx.x == 0) {
        s_best[0] = best;
        s_arg[0] = arg;
    }
    __syncthreads();
    *best_out = s_best[0];
    *arg_out = s_arg[0];
    __syncthreads(); // s_best / s_arg may be reused by the next call
}


// ----------------------------------------------------------------------------
// Grid-wide barrier of the persistent generation kernel (all blocks are
// co-resident: cooperative launch).  One monotonic 64-bit arrival counter:
// a block adds 1 with release semantics (a reduction: nothing comes back)
// and waits, with acquire loads, until the counter reaches the end of the
// barrier's epoch; each block's thread 0 keeps the next epoch end (`next`),
// which starts at the multiple of the block count that follows the counter's
// value at kernel start (the counter is a multiple of the block count between
// launches: every launch either passes each barrier with all blocks or stops
// on the sticky error word).  Nothing is ever reset.  A block that waits
// longer than kBarrierNs (wall clock, %globaltimer) or sees the error word set
// stops waiting, sets the error word and returns false; every block then
// leaves the kernel, so a failure ends as an error status, never a hang.
constexpr unsigned long long kBarrierNs = 2000000000ull; // 2 s

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// End of the first barrier epoch of this launch (thread 0 of each block).
__device__ __forceinline__ unsigned long long barrier_first(const unsigned long long *count, unsigned nblk)
{
    return ld_acquire_u64(count) / nblk * nblk + nblk;
}

__device__ bool grid_barrier(unsigned long long *count, int *err, unsigned nblk, unsigned long long &next,
                             unsigned long long limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int *verr = err;
        red_add_release_u64(count, 1ull);
        const unsigned long long target = next;
        next += nblk;
        int ok = 1;
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u64(count) < target) {
            if (*verr || global_ns() - t0 > limit_ns) {
                ok = 0;
                atomicExch(err, 1);
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok;
}

// Generation start (Alg. 3): P <- O (skipped with copy = false, when every
// item's generation-start data is staged from O before anything is written;
// with the learned filter on, the change marks of the generation before),
// the new elitist copied out of O[argmax] when it changed, the elitist flags
// eqw[g mod 2] (P[i] == x_e over all variables), the other buffer set for
// generation g+1, and the item claim counters zeroed.
__device__ void phase_gen_start(const GomParams &P, const VGrid &V, int improved, int argmax, uint32_t g, bool copy)
{
    __shared__ uint32_t s_eq[32];
    const int aw = argmax >> 5, ab = argmax & 31;
    const int W = P.W;
    const int lw = __ffs(W) - 1;
    const int64_t total = (int64_t)P.n * W;
    const int64_t tid = V.thread(), nth = V.threads();
    const int w = (int)(tid & (W - 1));
    uint32_t *eqw = P.eqw + (g & 1) * W;
    if (tid < W) P.eqw[((g + 1) & 1) * W + tid] = kFull;
    for (int64_t t = tid; t < P.k; t += nth) P.work[t] = 0;
    if (P.fi.on) { // Forced Improvement: the generation's accepted steps, FI's elitist flags, the fitness at its start
        if (tid < W) {
            P.fi.accw[tid] = 0;
            P.fi.eq[tid] = kFull;
        }
        for (int64_t i = tid; i < 32 * W; i += nth) P.fi.f0[i] = P.f[i];
    }
    if (P.learn) { // the learned filter's history and skip marks of generation g, and its counters
        uint32_t *cur = P.flt.hist + (size_t)(g & 1) * 3 * (size_t)P.m;
        for (int64_t x = tid; x < 3 * (int64_t)P.m; x += nth) cur[x] = 0;
        for (int64_t x = tid; x < P.m; x += nth) P.flt.skipped[x] = 0;
        if (tid < FC_N) P.flt.st->cnt[tid] = 0;
    }
    uint32_t eq = kFull;
    // the learned filter's change marks: variable v changed in some individual
    // during generation g - 1 (O now against P, its start; none before the
    // first generation).  The W words of v sit in W consecutive lanes of one
    // warp, and a warp's active lanes in the last round are whole such groups.
    const bool marks = P.learn && copy;
    for (int64_t idx = tid; idx < total; idx += nth) {
        const int64_t v = idx >> lw;
        const uint32_t word = P.O[idx];
        if (marks) {
            uint32_t ch = g > 0 ? word ^ P.P[idx] : 0u;
            const unsigned am = __activemask();
            for (int off = 1; off < W; off <<= 1) ch |= __shfl_xor_sync(am, ch, off);
            if (w == 0) P.flt.dirty[v] = ch != 0;
        }
        if (copy) P.P[idx] = word;
        uint32_t xb;
        if (improved) {
            xb = (P.O[v * W + aw] >> ab) & 1u;
            if (w == 0) P.xe[v] = (uint8_t)xb;
        } else {
            xb = P.xe[v];
        }
        eq &= ~(word ^ (0u - xb));
    }
    for (int off = 16; off >= W; off >>= 1) eq &= __shfl_xor_sync(kFull, eq, off);
    if (threadIdx.x < 32) s_eq[threadIdx.x] = kFull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (lane < W) atomicAnd(&s_eq[lane], eq);
    __syncthreads();
    if (threadIdx.x < W && threadIdx.x < 32 && s_eq[threadIdx.x] != kFull)
        atomicAnd(&eqw[threadIdx.x], s_eq[threadIdx.x]);
}

// Group order of generation g (Alg. 3 visits the groups in random order):
// colours sorted by their 64-bit Philox key, ties by colour index.  Every
// block draws all k keys into shared memory s_key[k]; rank_of gives the
// position of colour c.
__device__ __forceinline__ void order_keys(const GomParams &P, unsigned long long *s_key, uint32_t g)
{
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    for (int c = threadIdx.x; c < P.k; c += blockDim.x) {
        const uint4 r = philox10(make_uint4((uint32_t)c, 0u, g, kTagOrder), k0, k1);
        s_key[c] = ((unsigned long long)r.x << 32) | r.y;
    }
    __syncthreads();
}

__device__ __forceinline__ int rank_of(const unsigned long long *s_key, int k, int c)
{
    const unsigned long long kc = s_key[c];
    int rank = 0;
    for (int c2 = 0; c2 < k; ++c2) {
        const unsigned long long k2 = s_key[c2];
        rank += (k2 < kc) || (k2 == kc && c2 < c);
    }
    return rank;
}

// The order into P.order, the colours ranked in a grid-strided share per block.
__device__ void phase_order(const GomParams &P, const VGrid &V, unsigned long long *s_key, uint32_t g)
{
    order_keys(P, s_key, g);
    for (int c = (int)V.thread(); c < P.k; c += (int)V.threads()) P.order[rank_of(s_key, P.k, c)] = c;
    __syncthreads();
}

// The whole order in every block, into shared memory (k <= kStageAllMaxK).
__device__ void phase_order_block(const GomParams &P, unsigned long long *s_key, int *s_order, uint32_t g)
{
    order_keys(P, s_key, g);
    for (int c = threadIdx.x; c < P.k; c += blockDim.x) s_order[rank_of(s_key, P.k, c)] = c;
    __syncthreads();
}

// Generation end: the elitist update (strict improvement, lowest index of
// the best; Sec. 4), the counters, the target check and g += 1.  Every block
// that calls it computes the same values from the fitness array; block 0
// (write_state) records them: the state, and the counters of generation g in
// the statistics ring.  `improved` tells the next generation start to copy the
// elitist out of O.  Returns the target check.
struct GenEnd {
    int64_t fe;
    int improved, argmax;
};

// The learned filter at the end of generation g (one thread): the counters
// into last/total, then, with at least 16 audits, the recall estimate --
// useful items run / (useful items run + skipped items x the useful fraction
// of the audited ones).  The threshold steps down (skip less) while the
// estimate is under target_recall and up while it is well over it, and up
// too while the filter skips too little to be audited 16 times; two
// generations in a row under min_recall turn the filter off, and the run goes
// on as plain GOM.
__device__ void filter_generation_end(const GomParams &P, uint32_t g)
{
    GomFilterState *st = P.flt.st;
    for (int x = 0; x < FC_N; ++x) {
        st->last[x] = st->cnt[x];
        st->total[x] += st->cnt[x];
    }
    if (P.learn == 2 && st->enabled && st->last[FC_AUDITED] >= 16) {
        const double miss = (double)st->last[FC_AUDITED_USEFUL] / (double)st->last[FC_AUDITED];
        const double found = (double)st->last[FC_RUN_USEFUL];
        const double lost = (double)st->last[FC_SKIPPED] * miss;
        const double recall = found + lost > 0.0 ? found / (found + lost) : 1.0;
        if (recall < (double)st->target_recall)
            st->threshold -= 0.25f;
        else if (recall > (double)st->target_recall + 0.03)
            st->threshold += 0.125f;
        st->low_streak = recall < (double)st->min_recall ? st->low_streak + 1 : 0;
        if (st->low_streak >= 2) {
            st->enabled = 0;
            st->disabled_at = (int32_t)g;
        }
    } else if (P.learn == 2 && st->enabled) {
        st->threshold += 0.125f; // too few audits to estimate the recall: skip a little more
    }
}

__device__ bool phase_gen_end(const GomParams &P, int64_t target, uint32_t g, GenEnd &e, bool write_state)
{
    int64_t best;
    int arg;
    block_argmax(P.f, P.p, &best, &arg);
    e.improved = best > e.fe;
    if (e.improved) {
        e.fe = best;
        e.argmax = arg;
    }
    const bool reached = best >= target;
    if (write_state && threadIdx.x == 0) {
        GomDevState *st = P.st;
        st->fe = e.fe;
        st->argmax = e.argmax;
        st->improved = e.improved;
        st->best = best;
        GomDevStats &S = P.stats[g % kStatsCap];
        S.generation = g;
        S.best = best;
        S.elite = e.fe;
        S.trials = (int64_t)P.p * P.m - st->cnt[3]; // minus the trials a learned filter skipped
        S.donorless = st->cnt[0];
        S.accepted = st->cnt[1];
        S.improving = st->cnt[2];
        S.reached = reached;
        S.fi_individuals = st->fi_cnt[0];
        S.fi_trials = st->fi_cnt[1];
        S.fi_accepted = st->fi_cnt[2];
        S.fi_improving = st->fi_cnt[3];
        S.fi_replaced = st->fi_cnt[4];
        st->cnt[0] = st->cnt[1] = st->cnt[2] = st->cnt[3] = 0;
        st->fi_cnt[0] = st->fi_cnt[1] = st->fi_cnt[2] = st->fi_cnt[3] = st->fi_cnt[4] = 0;
        st->done = reached;
        st->g = g + 1;
        if (P.learn) filter_generation_end(P, g);
    }
    __syncthreads();
    return reached;
}

// First position after d, in cyclic order over [0, p), whose bit is set in
// rs[0..Wv) (bits >= p are zero); -1 if no bit is set.
__device__ __forceinline__ int next_set_cyclic(const uint32_t *rs, int Wv, int p, int d)
{
    int x = d + 1;
    if (x >= p) x = 0;
    int w = x >> 5;
    uint32_t m = rs[w] & (kFull << (x & 31));
    for (int step = 0; step <= Wv; ++step) {
        if (m) return 32 * w + __ffs(m) - 1;
        if (++w == Wv) w = 0;
        m = rs[w];
    }
    return -1;
}

// Asynchronous global -> shared copies (cp.async): they do not hold registers
// or stall the warp until cp_wait(), so many can be in flight together.
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// Waits for this thread's copies, then makes the warp's copies visible to the warp.
__device__ __forceinline__ void cp_wait_warp()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
}

// Zeroes the block's fitness and counter accumulators.
__device__ __forceinline__ void acc_zero(const GomParams &P, long long *s_f, unsigned long long *s_cnt)
{
    for (int q = threadIdx.x; q < 32 * P.W; q += blockDim.x) s_f[q] = 0;
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();
}

// Adds the block's accumulators into the fitness array and the generation's
// counters: one atomic per individual (and per counter), integer adds, so
// the result does not depend on their order.
__device__ __forceinline__ void acc_flush(const GomParams &P, long long *s_f, unsigned long long *s_cnt)
{
    __syncthreads();
    for (int q = threadIdx.x; q < 32 * P.W; q += blockDim.x) {
        const long long v = s_f[q];
        if (v) atomicAdd((unsigned long long *)&P.f[q], (unsigned long long)v);
    }
    if (threadIdx.x < 3 && s_cnt[threadIdx.x])
        atomicAdd((unsigned long long *)&P.st->cnt[threadIdx.x], s_cnt[threadIdx.x]);
    __syncthreads();
}

// Adds a warp's per-lane counters into the block's counters.
__device__ __forceinline__ void count_flush(unsigned long long *s_cnt, unsigned n_dl, unsigned n_acc, unsigned n_imp)
{
    n_dl = __reduce_add_sync(kFull, n_dl);
    n_acc = __reduce_add_sync(kFull, n_acc);
    n_imp = __reduce_add_sync(kFull, n_imp);
    if ((threadIdx.x & 31) == 0 && (n_dl | n_acc | n_imp)) {
        atomicAdd(&s_cnt[0], (unsigned long long)n_dl);
        atomicAdd(&s_cnt[1], (unsigned long long)n_acc);
        atomicAdd(&s_cnt[2], (unsigned long long)n_imp);
    }
}

} // namespace
