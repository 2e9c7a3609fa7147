// gom_fi.cuh -- Forced Improvement (Sec. 4, Alg. 1) after a generation's
// mixing, in the library's parallel reading.  The paper's FI is serial: it
// walks one individual's linkage sets with the elitist as donor and stops at
// the first improving step; its parallel GOMEA leaves FI out and names a
// parallel-friendly variant as future work (Sec. 5.4).  Here:
//   - the elitist is first updated from the population after mixing
//     (strict improvement, lowest index), and copied into x_e;
//   - FI applies to the individuals with no accepted GOM step in the
//     generation, and, with a threshold nis > 0, to those whose fitness has
//     not improved for nis generations (this one included);
//   - those individuals take GOM steps with x_e as donor on every element of
//     each colour group, the groups in this generation's order; a step is
//     accepted as in Alg. 2 (delta > 0, or delta = 0 and the individual not
//     equal to the elitist, that flag taken at the start of FI);
//   - an individual leaves FI after the first group in which a step improved
//     its fitness (the elements of one group share no variable and no edge,
//     so their order within the group does not matter);
//   - an individual that no step improved becomes a copy of the elitist.
// With one donor for everyone, a step's flip planes are (O_a ^ x_e,a) on the
// individuals still in FI, so every (element, word) pair is one lane doing
// the bit-plane partial evaluation of gom_bitplane.cuh, reading its rows
// from global memory (elements of up to 128 variables).  Anonymous
// namespace: each translation unit that includes it compiles its own copy.
#pragma once

#include <cuda_runtime.h>

#include "gom_bitplane.cuh"
#include "gom_device.cuh"
#include "gom_internal.h"

namespace {

// FI counters: individuals, trials, accepted, improving, replaced.
enum : int { FIC_IND = 0, FIC_TRIALS = 1, FIC_ACC = 2, FIC_IMP = 3, FIC_REP = 4 };

// Start of FI, part 1 (every block of the problem, after the barrier that
// closes the mixing; `newel`, `aw`, `ab`: whether the elitist changed at this
// point and the word and bit of the individual now holding it): x_e copied
// out of O when it changed, the flags "equal to the elitist" (into fi.eq,
// set to all ones at generation start), the per-group improvement words and
// the group claim counters zeroed.  Block `lead` also writes the set of
// individuals in FI (fi.act0) and counts them.
__device__ void fi_start(const GomParams &P, const VGrid &V, bool newel, int aw, int ab, bool lead)
{
    __shared__ uint32_t s_eq[32];
    const int W = P.W;
    const int lw = __ffs(W) - 1;
    const int64_t tid = V.thread(), nth = V.threads();
    const int w = (int)(tid & (W - 1));
    uint32_t eq = 0xFFFFFFFFu;
    for (int64_t idx = tid; idx < (int64_t)P.n * W; idx += nth) {
        const int64_t v = idx >> lw;
        const uint32_t word = P.O[idx];
        uint32_t xb;
        if (newel) {
            xb = (P.O[v * W + aw] >> ab) & 1u;
            if (w == 0) P.xe[v] = (uint8_t)xb;
        } else {
            xb = P.xe[v];
        }
        eq &= ~(word ^ (0u - xb));
    }
    for (int off = 16; off >= W; off >>= 1) eq &= __shfl_xor_sync(0xFFFFFFFFu, eq, off);
    if (threadIdx.x < 32) s_eq[threadIdx.x] = 0xFFFFFFFFu;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (lane < W) atomicAnd(&s_eq[lane], eq);
    __syncthreads();
    if (threadIdx.x < W && threadIdx.x < 32 && s_eq[threadIdx.x] != 0xFFFFFFFFu)
        atomicAnd(&P.fi.eq[threadIdx.x], s_eq[threadIdx.x]);
    for (int64_t x = tid; x < (int64_t)P.k * W; x += nth) P.fi.imp[x] = 0;
    for (int64_t t = tid; t < P.k; t += nth) P.work[t] = 0;
    if (lead && threadIdx.x < 32) { // the individuals in FI, word by word (warp 0 of the lead block)
        unsigned long long cnt = 0;
        for (int ww = 0; ww < W; ++ww) {
            const int i = 32 * ww + lane;
            bool in = false;
            if (i < P.p) {
                const bool acc = (P.fi.accw[ww] >> lane) & 1u;
                const bool stale =
                    P.fi.nis > 0 && (P.f[i] > P.fi.f0[i] ? 0 : P.fi.stale[i] + 1) >= P.fi.nis;
                in = !acc || stale;
            }
            const uint32_t mk = __ballot_sync(0xFFFFFFFFu, in);
            if (lane == 0) P.fi.act0[ww] = mk;
            cnt += __popc(mk);
        }
        if (lane == 0 && cnt) atomicAdd((unsigned long long *)&P.st->fi_cnt[FIC_IND], cnt);
    }
}

// The FI steps of one item: elements [q0, q1) of the group at position t,
// lane = (element slot, word); s_act[w] the individuals of word w still in FI.
template <int R>
__device__ __forceinline__ void fi_item(const GomParams &P, int t, int q0, int q1, const uint32_t *s_act, BsLane &L,
                                        unsigned (&cnt)[3], long long *s_f)
{
    const int lane = threadIdx.x & 31;
    const int W = P.W, Wv = P.Wv;
    const int lw = __ffs(W) - 1;
    const int e = lane >> lw, w = lane & (W - 1);
    const int q = q0 + e;
    if (L.since_flush >= (1 << (kFitPlanes - R))) bs_flush(P, L, s_f);
    ++L.since_flush;
    if (q >= q1 || w >= Wv) return;
    const uint32_t act = s_act[w];
    if (!act) return;
    const int4 h0 = __ldg(P.hdr + 2 * q), h1 = __ldg(P.hdr + 2 * q + 1);
    const int f0 = h0.y, d0 = h0.z, s = h0.w & 0xFF, n_in = h0.w >> 8, n_out = h1.x;
    uint32_t D[R + 1]; // the trials' deltas, two's complement (|partial sums| < 2^R)
#pragma unroll
    for (int x = 0; x <= R; ++x) D[x] = 0;
    uint32_t hd = 0;
    for (int a = 0; a < s; ++a) {
        const int64_t v = __ldg(P.fv + f0 + a);
        const uint32_t Xa = P.O[v * W + w];
        const uint32_t Fa = (Xa ^ (0u - (uint32_t)P.xe[v])) & act;
        hd |= Fa;
        if (!Fa) continue;
        const int xb = (int)__ldg(P.seg + f0 + q + a), xe = (int)__ldg(P.seg + f0 + q + a + 1);
        for (int x = xb; x < xe; ++x) {
            const int2 ed = __ldg(P.dep + d0 + x);
            const uint32_t Xv = P.O[(int64_t)ed.x * W + w];
            const uint32_t cut = Xa ^ Xv ^ (uint32_t)(ed.y >> 31);
            add_signed<R + 1, kWeightBits>(D, Fa & ~cut, Fa & cut, (uint32_t)(ed.y < 0 ? -ed.y : ed.y));
        }
    }
    for (int x = n_out; x < n_out + n_in; ++x) {
        const int2 ed = __ldg(P.dep + d0 + x);
        const int64_t va = __ldg(P.fv + f0 + (ed.x & 0xFF)), vb = __ldg(P.fv + f0 + (ed.x >> 8));
        const uint32_t Xa = P.O[va * W + w], Xb = P.O[vb * W + w];
        const uint32_t Fa = (Xa ^ (0u - (uint32_t)P.xe[va])) & act, Fb = (Xb ^ (0u - (uint32_t)P.xe[vb])) & act;
        const uint32_t tg = Fa ^ Fb;
        if (!tg) continue;
        const uint32_t cut = Xa ^ Xb ^ (uint32_t)(ed.y >> 31);
        add_signed<R + 1, kWeightBits>(D, tg & ~cut, tg & cut, (uint32_t)(ed.y < 0 ? -ed.y : ed.y));
    }
    uint32_t nz = 0;
#pragma unroll
    for (int x = 0; x <= R; ++x) nz |= D[x];
    const uint32_t neg = D[R];
    const uint32_t pos = nz & ~neg;
    const uint32_t acc = hd & act & (pos | (~nz & ~P.fi.eq[w]));
    cnt[0] += __popc(act);
    cnt[1] += __popc(acc);
    cnt[2] += __popc(acc & pos);
    if (acc & pos) atomicOr(&P.fi.imp[(int64_t)t * W + w], acc & pos);
    if (acc) {
        for (int a = 0; a < s; ++a) {
            const int64_t v = __ldg(P.fv + f0 + a);
            const uint32_t Xa = P.O[v * W + w];
            const uint32_t m = (Xa ^ (0u - (uint32_t)P.xe[v])) & acc;
            if (m) P.O[v * W + w] = Xa ^ m;
        }
        fit_add<R>(L, D, acc);
    }
}

// The FI steps of the group at position t (colour c): items of E = 32 / W
// consecutive elements, warp x takes items x, x + nwarps, ...  The fitness
// deltas go to the lanes' accumulators L, the counters to cnt.
template <int R>
__device__ void fi_group(const GomParams &P, const VGrid &V, int t, int c, const uint32_t *s_act, BsLane &L,
                         unsigned (&cnt)[3], long long *s_f)
{
    const int gwarp = (int)(V.thread() >> 5), nwarps = (int)(V.threads() >> 5);
    const int E = 32 / P.W;
    const int qa = P.cptr[c], qz = P.cptr[c + 1];
    const int items = (qz - qa + E - 1) / E;
    for (int it = gwarp; it < items; it += nwarps) {
        const int q0 = qa + it * E;
        fi_item<R>(P, t, q0, min(q0 + E, qz), s_act, L, cnt, s_f);
        __syncwarp();
    }
}

// Adds a warp's FI counters into the generation's (one atomic per counter).
__device__ __forceinline__ void fi_count_flush(const GomParams &P, unsigned (&cnt)[3])
{
    const unsigned a = __reduce_add_sync(0xFFFFFFFFu, cnt[0]), b = __reduce_add_sync(0xFFFFFFFFu, cnt[1]),
                   c = __reduce_add_sync(0xFFFFFFFFu, cnt[2]);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd((unsigned long long *)&P.st->fi_cnt[FIC_TRIALS], (unsigned long long)a);
        if (b) atomicAdd((unsigned long long *)&P.st->fi_cnt[FIC_ACC], (unsigned long long)b);
        if (c) atomicAdd((unsigned long long *)&P.st->fi_cnt[FIC_IMP], (unsigned long long)c);
    }
    cnt[0] = cnt[1] = cnt[2] = 0;
}

// End of FI (every block, after the fitness deltas of all groups are in f):
// the individuals FI did not improve (s_rep[w]) become copies of x_e with
// the elitist's fitness fe; every individual's count of generations without
// improvement is updated (fitness at its end against fi.f0).  Block `lead`
// counts the replacements.
__device__ void fi_finish(const GomParams &P, const VGrid &V, const uint32_t *s_rep, int64_t fe, bool lead)
{
    const int W = P.W;
    const int lw = __ffs(W) - 1;
    const int64_t tid = V.thread(), nth = V.threads();
    for (int64_t idx = tid; idx < (int64_t)P.n * W; idx += nth) {
        const uint32_t rep = s_rep[idx & (W - 1)];
        if (!rep) continue;
        const int64_t v = idx >> lw;
        P.O[idx] = (P.O[idx] & ~rep) | (P.xe[v] ? rep : 0u);
    }
    for (int64_t i = tid; i < P.p; i += nth) {
        const bool r = (s_rep[i >> 5] >> (i & 31)) & 1u;
        const int64_t f = r ? fe : P.f[i];
        if (r) P.f[i] = fe;
        P.fi.stale[i] = f > P.fi.f0[i] ? 0 : P.fi.stale[i] + 1;
    }
    if (lead && threadIdx.x == 0) {
        unsigned long long n = 0;
        for (int w = 0; w < W; ++w) n += __popc(s_rep[w]);
        if (n) atomicAdd((unsigned long long *)&P.st->fi_cnt[FIC_REP], n);
    }
}

// FI on the persistent path, between the barrier that closes the mixing and
// the generation end; `order` holds the generation's group order, e the
// generation-end state (the elitist update of FI's start goes into it, as in
// every block), s_f / s_cnt the block's accumulators.  Returns false when a
// barrier gave up (the kernel then leaves).  Not inlined: one copy per bit
// width serves every kernel instance of a translation unit.
template <int R>
__device__ __noinline__ bool fi_generation(const GomParams &P, const VGrid V, unsigned long long *bar_count,
                                           unsigned nblk, unsigned long long &bnext, GenEnd &e, const int *order,
                                           long long *s_f, unsigned long long *s_cnt)
{
    __shared__ uint32_t s_act0[32], s_done[32];
    const bool lead = V.blk == 0;
    int64_t best;
    int arg;
    block_argmax(P.f, P.p, &best, &arg);
    const bool newel = best > e.fe;
    if (newel) {
        e.fe = best;
        e.argmax = arg;
        e.improved = 1;
    }
    fi_start(P, V, newel, e.argmax >> 5, e.argmax & 31, lead);
    acc_zero(P, s_f, s_cnt);
    if (!grid_barrier(bar_count, &P.st->err, nblk, bnext, kBarrierNs)) return false;
    if (threadIdx.x < 32) {
        s_act0[threadIdx.x] = threadIdx.x < P.W ? P.fi.act0[threadIdx.x] : 0u;
        s_done[threadIdx.x] = 0;
    }
    __syncthreads();
    __shared__ uint32_t s_act[32];
    BsLane L;
    bs_lane_zero(L);
    unsigned cnt[3] = {0, 0, 0};
    for (int t = 0; t < P.k; ++t) {
        if (t > 0) {
            if (!grid_barrier(bar_count, &P.st->err, nblk, bnext, kBarrierNs)) return false;
            if (threadIdx.x < P.W) s_done[threadIdx.x] |= P.fi.imp[(int64_t)(t - 1) * P.W + threadIdx.x];
            __syncthreads();
        }
        if (threadIdx.x < 32) s_act[threadIdx.x] = s_act0[threadIdx.x] & ~s_done[threadIdx.x];
        __syncthreads();
        fi_group<R>(P, V, t, order[t], s_act, L, cnt, s_f);
        __syncthreads(); // every warp has read s_act
    }
    bs_flush(P, L, s_f);
    fi_count_flush(P, cnt);
    acc_flush(P, s_f, s_cnt);
    if (!grid_barrier(bar_count, &P.st->err, nblk, bnext, kBarrierNs)) return false;
    if (threadIdx.x < P.W) s_done[threadIdx.x] |= P.fi.imp[(int64_t)(P.k - 1) * P.W + threadIdx.x];
    __syncthreads();
    if (threadIdx.x < 32) s_act[threadIdx.x] = s_act0[threadIdx.x] & ~s_done[threadIdx.x];
    __syncthreads();
    fi_finish(P, V, s_act, e.fe, lead);
    return grid_barrier(bar_count, &P.st->err, nblk, bnext, kBarrierNs);
}

} // namespace
