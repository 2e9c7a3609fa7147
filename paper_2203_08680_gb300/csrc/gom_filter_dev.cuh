// gom_filter_dev.cuh -- device side of the learned trial filter, shared by
// the per-lane and the bit-sliced mixing paths: the 16 features of an
// element, the MLP's logit, the sampling and audit hashes, and the select
// phase that runs after each generation start -- it updates the elements'
// history, takes the filter's decision for every element before any group
// runs, and (bit-sliced path) compacts the elements to run into one ordered
// list, so that a skipped element costs its mixing nothing.
//
// The paper's GOM (Sec. 4, Alg. 2) has no filter: it is an addition beside
// the method, and every change it lets through is still decided by the exact
// integer partial evaluation.  Anonymous namespace: each translation unit
// that includes it compiles its own copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gom_device.cuh"
#include "gom_internal.h"

namespace {

// The select phase's decision for an element: run its trials, skip them, or
// run them although the filter would skip them (an audit of its recall).
enum : uint8_t { DEC_RUN = 0, DEC_SKIP = 1, DEC_AUDIT = 2 };
constexpr int32_t kActAudit = INT32_MIN; // flag of an audited element in the compacted list

__device__ __forceinline__ float bf16_bits_to_f32(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// Element q's variables (dF) and outside edges (dN, counted by edge) whose
// variable changed in some individual during the previous generation.
// Warp-wide: every lane receives both counts.
__device__ __forceinline__ void filter_dirty_counts(const GomParams &P, int q, int *dF, int *dN)
{
    const int lane = threadIdx.x & 31;
    const int4 a = P.hdr[2 * q], b = P.hdr[2 * q + 1];
    const int f0 = a.y, d0 = a.z, s = a.w & 0xFF, n_out = b.x;
    int cf = 0, cn = 0;
    for (int x = lane; x < s; x += 32) cf += P.flt.dirty[P.fv[f0 + x]];
    for (int x = lane; x < n_out; x += 32) cn += P.flt.dirty[P.dep[d0 + x].x];
    *dF = (int)__reduce_add_sync(kFull, (unsigned)cf);
    *dN = (int)__reduce_add_sync(kFull, (unsigned)cn);
}

// Features of the element at position q for generation g, given its change
// counts and its quiet count (the same in every lane): its size and edge
// counts, its accepted / donor-less / improving trials of the previous
// generation (as fractions of p), whether it accepted nothing or had no donor
// at all, the generation, the population's accept / improve / donor-less
// rates of the previous generation, a constant, the fractions of its
// variables and of its outside edges that changed during the previous
// generation, and how many generations in a row (up to 16) it has been quiet
// -- no accepted trial and no change in its variables or outside neighbours.
__device__ __forceinline__ void filter_features_from(const GomParams &P, int q, uint32_t g, int dF, int dN,
                                                     unsigned quiet, float (&x)[kFilterIn])
{
    const int4 a = P.hdr[2 * q], b = P.hdr[2 * q + 1];
    const int s = a.w & 0xFF, n_in = a.w >> 8, n_out = b.x;
    const float inv_p = 1.f / (float)P.p;
    const uint32_t *prev = P.flt.hist + (size_t)((g + 1) & 1) * 3 * (size_t)P.m;
    const uint32_t acc = prev[q], dl = prev[P.m + q], imp = prev[2 * (size_t)P.m + q];
    x[0] = (float)s / 16.f;
    x[1] = (float)n_out / 64.f;
    x[2] = (float)n_in / 32.f;
    x[3] = (float)acc * inv_p;
    x[4] = (float)dl * inv_p;
    x[5] = (float)imp * inv_p;
    x[6] = acc == 0 ? 1.f : 0.f;
    x[7] = dl >= (uint32_t)P.p ? 1.f : 0.f;
    x[8] = log2f(1.f + (float)g) / 16.f;
    x[9] = x[10] = x[11] = 0.f;
    if (g > 0) {
        const GomDevStats &S = P.stats[(g - 1) % kStatsCap];
        const float tr = (float)S.trials;
        x[9] = (float)S.accepted / tr;
        x[10] = (float)S.improving / tr;
        x[11] = (float)S.donorless / tr;
    }
    x[12] = 1.f;
    x[13] = (float)dF / (float)s;
    x[14] = n_out > 0 ? (float)dN / (float)n_out : 0.f;
    x[15] = (float)min(quiet, 16u) / 16.f;
}

// The features as the select phase computed them (warp-wide): the change
// counts again (the change marks are constant during a generation) and the
// quiet count the select phase stored.
__device__ __forceinline__ void filter_features(const GomParams &P, int q, uint32_t g, float (&x)[kFilterIn])
{
    int dF, dN;
    filter_dirty_counts(P, q, &dF, &dN);
    filter_features_from(P, q, g, dF, dN, P.flt.quiet[q], x);
}

// The MLP's output (logit) for one element, in one lane: 64 ReLU units over
// the 16 features (rounded to bf16, as logged), bf16 weights, fp32
// accumulation in a fixed order -- unit h's sum over k = 0..15 from its bias,
// then the output's sum over h = 0..63 from zero, plus the output bias (the
// order of the training code's evaluation).  The weights are read with the
// same address in every lane (broadcast loads), eight bf16 values at a time.
__device__ __forceinline__ float filter_logit(const GomParams &P, const float (&x0)[kFilterIn])
{
    float x[kFilterIn];
#pragma unroll
    for (int k = 0; k < kFilterIn; ++k) x[k] = __bfloat162float(__float2bfloat16_rn(x0[k]));
    const uint4 *w1 = reinterpret_cast<const uint4 *>(P.flt.w1); // row h: w1[2h], w1[2h + 1]
    float out = 0.f;
#pragma unroll 4
    for (int h = 0; h < kFilterHidden; ++h) {
        const uint4 r0 = __ldg(w1 + 2 * h), r1 = __ldg(w1 + 2 * h + 1);
        const uint32_t wd[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        float z = __ldg(P.flt.b1 + h);
#pragma unroll
        for (int k = 0; k < kFilterIn; ++k) {
            const uint32_t word = wd[k >> 1];
            z = fmaf(__uint_as_float((k & 1) ? (word & 0xFFFF0000u) : (word << 16)), x[k], z);
        }
        out = fmaf(bf16_bits_to_f32(__ldg(P.flt.w2 + h)), fmaxf(z, 0.f), out);
    }
    return out + __ldg(P.flt.b2);
}

// One in 16 elements of a generation whose trials the filter would skip is run
// anyway (an audit), to estimate how many useful elements it skips.
__device__ __forceinline__ bool filter_audit(int q, uint32_t g)
{
    uint32_t h = (uint32_t)q * 0x9E3779B1u ^ (g * 0x85EBCA77u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    return (h & 15u) == 0;
}

// One in 32 elements of a generation gives a training sample.
__device__ __forceinline__ bool filter_sample(int q, uint32_t g)
{
    uint32_t h = (uint32_t)q * 0xCC9E2D51u ^ (g * 0x1B873593u);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    return (h & 31u) == 0;
}

// A deterministic offset in [-0.5, 0.5) per (element position, generation),
// added to the logit before the threshold: elements with equal features have
// equal logits, and without it a threshold would skip all or none of them.
__device__ __forceinline__ float filter_jitter(int q, uint32_t g)
{
    uint32_t h = (uint32_t)q * 0x27D4EB2Fu ^ (g * 0x165667B1u);
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    h ^= h >> 13;
    return (float)(h >> 8) * (1.f / 16777216.f) - 0.5f;
}

// Appends one training sample (the element's features and its label) to the
// log ring.  Warp-wide.
__device__ __forceinline__ void filter_log_sample(const GomParams &P, const float (&x)[kFilterIn], bool useful)
{
    const int lane = threadIdx.x & 31;
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(&P.flt.st->log_count, 1ull);
    idx = __shfl_sync(kFull, idx, 0);
    if (P.flt.log_cap > 0) { // a ring: the log keeps the latest log_cap samples
        idx %= (unsigned long long)P.flt.log_cap;
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < kFilterIn; ++k) v = lane == k ? x[k] : v;
        if (lane < kFilterIn) P.flt.log_x[idx * kFilterIn + lane] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        if (lane == 0) P.flt.log_y[idx] = useful ? 1 : 0;
    }
}

// Positions [qa, qz) of the contiguous chunk that warp `gwarp` of `nwarps`
// owns in the select phase.
__device__ __forceinline__ void filter_chunk(const GomParams &P, int gwarp, int nwarps, int *qa, int *qz)
{
    const int C = (P.m + nwarps - 1) / nwarps;
    *qa = min(P.m, gwarp * C);
    *qz = min(P.m, *qa + C);
}

// filter_dirty_counts for one lane's own element (the same counts).
__device__ __forceinline__ void filter_dirty_counts_lane(const GomParams &P, int q, int *dF, int *dN)
{
    const int4 a = P.hdr[2 * q], b = P.hdr[2 * q + 1];
    const int f0 = a.y, d0 = a.z, s = a.w & 0xFF, n_out = b.x;
    int cf = 0, cn = 0;
    for (int x = 0; x < s; x += 4) { // four loads in flight, then their marks
        int v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = x + u < s ? __ldg(P.fv + f0 + x + u) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) cf += v[u] >= 0 ? P.flt.dirty[v[u]] : 0;
    }
    for (int x = 0; x < n_out; x += 8) {
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = x + u < n_out ? __ldg(P.dep + d0 + x + u).x : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u) cn += v[u] >= 0 ? P.flt.dirty[v[u]] : 0;
    }
    *dF = cf;
    *dN = cn;
}

// Select, step 1 (every warp, its chunk of positions, 32 at a time, lane =
// element): the element's quiet count, then -- while the filter skips -- its
// features, logit and decision (DEC_SKIP when logit + jitter is below the
// threshold, DEC_AUDIT for the audited ones among those).  Skipped
// elements are marked (for a replay) and counted, in items_per_elem items
// each and p trials.  With `compact`, each warp's count of elements to run
// goes to wcnt.
__device__ void filter_select_decide(const GomParams &P, const VGrid &V, uint32_t g, bool compact)
{
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)(V.thread() >> 5), nwarps = (int)(V.threads() >> 5);
    int qa, qz;
    filter_chunk(P, gwarp, nwarps, &qa, &qz);
    // (block mode stages elements without reading the decisions: nothing is skipped there)
    const bool decide = P.learn == 2 && P.flt.st->enabled && !P.blk;
    const float thr = P.flt.st->threshold;
    const uint32_t *prev = P.flt.hist + (size_t)((g + 1) & 1) * 3 * (size_t)P.m;
    unsigned kept = 0, nskip = 0;
    for (int q0 = qa; q0 < qz; q0 += 32) {
        const int q = q0 + lane;
        const bool v = q < qz;
        float x[kFilterIn];
#pragma unroll
        for (int k = 0; k < kFilterIn; ++k) x[k] = 0.f;
        unsigned quiet = 0;
        if (v) {
            int dF, dN;
            filter_dirty_counts_lane(P, q, &dF, &dN);
            quiet = P.flt.quiet[q];
            quiet = (prev[q] == 0 && dF == 0 && dN == 0) ? min(quiet + 1u, 255u) : 0u;
            if (decide) filter_features_from(P, q, g, dF, dN, quiet, x);
        }
        uint8_t d = DEC_RUN;
        if (decide && v && filter_logit(P, x) + filter_jitter(q, g) < thr) d = filter_audit(q, g) ? DEC_AUDIT : DEC_SKIP;
        if (v) {
            P.flt.quiet[q] = (uint8_t)quiet;
            P.flt.dec[q] = d;
            if (d == DEC_SKIP) P.flt.skipped[q] = 1;
        }
        kept += __popc(__ballot_sync(kFull, v && d != DEC_SKIP));
        nskip += __popc(__ballot_sync(kFull, v && d == DEC_SKIP));
    }
    if (lane == 0) {
        if (compact) P.flt.wcnt[gwarp] = kept;
        if (nskip) {
            atomicAdd(&P.flt.st->cnt[FC_SKIPPED], (unsigned long long)nskip * (unsigned)P.flt.items_per_elem);
            atomicAdd((unsigned long long *)&P.st->cnt[3], (unsigned long long)nskip * (unsigned)P.p);
        }
    }
}

// Select, step 2 (one block): wcnt[0 .. nwarps) becomes its exclusive prefix
// sum (in place) -- each warp's first slot in the compacted list.
__device__ void filter_select_scan(const GomParams &P, int nwarps)
{
    __shared__ unsigned s_warp[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (nwarps + nt - 1) / nt, a = min(nwarps, tid * per), b = min(nwarps, a + per);
    unsigned sum = 0;
    for (int x = a; x < b; ++x) sum += P.flt.wcnt[x];
    // inclusive scan of the per-thread sums across the block
    const int lane = tid & 31, wid = tid >> 5;
    unsigned v = sum;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v += y;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        unsigned w = lane < (nt >> 5) ? s_warp[lane] : 0u;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, w, off);
            if (lane >= off) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    unsigned run = v - sum + (wid > 0 ? s_warp[wid - 1] : 0u); // exclusive prefix of this thread's range
    for (int x = a; x < b; ++x) {
        const unsigned c = P.flt.wcnt[x];
        P.flt.wcnt[x] = run;
        run += c;
    }
    __syncthreads();
}

// Select, step 3 (every warp, its chunk again, 32 positions at a time): the
// elements to run in position order, act[r] = q (kActAudit set for an
// audited one), and for each colour c whose first position lies in the
// chunk, act_ptr[c] = the number of elements to run before it (act_ptr[k] =
// all of them; empty colours share their successor's value).
__device__ void filter_select_compact(const GomParams &P, const VGrid &V)
{
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)(V.thread() >> 5), nwarps = (int)(V.threads() >> 5);
    int qa, qz;
    filter_chunk(P, gwarp, nwarps, &qa, &qz);
    unsigned base = P.flt.wcnt[gwarp];
    // the first colour whose first position is at or after qa
    int c = 0;
    {
        int lo = 0, hi = P.k + 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (P.cptr[mid] < qa) lo = mid + 1;
            else hi = mid;
        }
        c = lo;
    }
    for (int q0 = qa; q0 < qz; q0 += 32) {
        const int q = q0 + lane;
        const uint8_t d = q < qz ? P.flt.dec[q] : DEC_SKIP;
        const unsigned run = __ballot_sync(kFull, d != DEC_SKIP);
        if (d != DEC_SKIP) P.flt.act[base + __popc(run & ((1u << lane) - 1u))] = d == DEC_AUDIT ? (q | kActAudit) : q;
        for (; c <= P.k && P.cptr[c] < min(q0 + 32, qz); ++c)
            if (lane == 0) P.flt.act_ptr[c] = (int32_t)(base + __popc(run & ((1u << (P.cptr[c] - q0)) - 1u)));
        base += __popc(run);
    }
    // colours starting at position m (the last boundary, and empty colours at the end)
    // (the last warp's chunk ends at m, so its base is now the total)
    if (gwarp == nwarps - 1 && lane == 0)
        for (int c2 = 0; c2 <= P.k; ++c2)
            if (P.cptr[c2] >= P.m) P.flt.act_ptr[c2] = (int32_t)base;
}

// The block's item counters of the learned filter on the bit-sliced path
// (run, run with an acceptance, audited, audited with an acceptance): zeroed
// before the barrier of acc_zero, added into the generation's counters after
// acc_flush (whose barriers order the block's counts before the read).
__device__ __forceinline__ void fc_zero(unsigned long long *s_fc)
{
    if (threadIdx.x < 4) s_fc[threadIdx.x] = 0;
}

__device__ __forceinline__ void fc_flush(const GomParams &P, const unsigned long long *s_fc)
{
    if (P.learn && threadIdx.x < 4 && s_fc[threadIdx.x]) {
        const int x = threadIdx.x < 2 ? FC_RUN + threadIdx.x : FC_AUDITED + (threadIdx.x - 2);
        atomicAdd(&P.flt.st->cnt[x], s_fc[threadIdx.x]);
    }
}

// The select phase inside a persistent launch, right after the barrier that
// follows the generation start: decisions, then (with compaction) the scan by
// block 0 and the compacted list, each step closed by a grid barrier; the
// last barrier also opens group 0.  False if a barrier timed out.
__device__ __noinline__ bool phase_filter_select(const GomParams &P, const VGrid &V, uint32_t g, unsigned long long *count,
                                    unsigned nblk, unsigned long long &bnext, bool compact)
{
    filter_select_decide(P, V, g, compact);
    if (!grid_barrier(count, &P.st->err, nblk, bnext, kBarrierNs)) return false;
    if (!compact) return true;
    if (V.blk == 0) filter_select_scan(P, (int)(V.threads() >> 5));
    if (!grid_barrier(count, &P.st->err, nblk, bnext, kBarrierNs)) return false;
    filter_select_compact(P, V);
    return grid_barrier(count, &P.st->err, nblk, bnext, kBarrierNs);
}

} // namespace
