// gom_bs.cuh -- the bit-sliced mixing path of parallel GOM for weighted Max-Cut:
// its device code, shared by its own kernels (gom_bs.cu) and the batched
// kernel (gom_kernels.cu).  Anonymous namespace: each translation unit that
// includes it compiles its own copy.
//
// Same generations as the per-lane path of gom_kernels.cu (Alg. 3; every
// trial of Alg. 2 decided by the exact integer delta), with the partial
// evaluation, the acceptance and the fitness bookkeeping done on bit-planes:
// one 32-bit register holds one bit of 32 individuals, so one logic
// instruction works on 32 trials at once.
//
// A warp takes an item of E = 32 / W elements of the colour group (W = words
// per variable row); lane k owns the pair (element slot k / W, word k mod W),
// i.e. 32 individuals of one element.  Per item:
//   phase 0  (lane = pair) the parent's current rows on F_j and the
//            generation-start rows of P on F_j into shared memory, the run
//            starts of P's patterns on F_j, and the Philox donor starts of
//            all 1024 trials (one Philox call per 4 individuals); then, by
//            32 x 32 bit transposes, the patterns of P and of the parents on
//            the item's elements packed side by side per individual
//   phase 1  (lane = individual, one word after the other) the donor search
//            of Sec. 4.2: one lookup of the start candidate's packed pattern
//            and of the next run start after it, the run-start walk and the
//            word-parallel scan for the rare rest; the packed flips (donor ^
//            parent) go back through transposes into flip planes F_a (bit b:
//            individual b flips variable a)
//   phase 2  (lane = pair) the partial evaluation (Sec. 2.2, Alg. 4) as
//            bit-plane arithmetic: an edge e that a trial toggles (t_e = F_a
//            for an edge leaving F_j, F_a ^ F_b inside) changes the cut by
//            +|w_e| if it was uncut and -|w_e| if it was cut (its cut plane
//            c_e taken with the weight's sign folded in), so
//              delta = sum_e |w_e| (t_e & ~c_e) - |w_e| (t_e & c_e),
//            one signed ripple-carry chain per edge on R + 1 two's-complement
//            planes (each edge counted once); then the accept plane (Alg. 2:
//            delta > 0, or delta = 0 and not the elitist), counters by
//            popcount, the accepted flips XORed into the rows, and the
//            accepted deltas into a bit-sliced per-lane fitness accumulator,
//            flushed into the block's accumulators once per generation (or
//            before it could overflow).
// With the learned trial filter on, a select phase after the generation start
// (gom_filter_dev.cuh) decides which elements run and lists them in order, the
// groups run only the listed elements, and each item records its elements'
// history and training samples.
// Elements of one colour group share no variable and no edge (LMIG
// colouring), so the rows a pair reads and writes belong to it alone during
// the group.
//
// The path takes elements of at most 32 variables, |w| <= 255, and elements
// whose sum of |w| over their edges is below 2^R (R = 12 or 16, the width of
// the bit-plane accumulators); the host selects it only then.
#pragma once

#include <climits>
#include <cuda_runtime.h>

#include "gom_bitplane.cuh"
#include "gom_device.cuh"
#include "gom_fi.cuh"
#include "gom_filter_dev.cuh"
#include "gom_internal.h"

namespace {

// Four independent 32 x 32 bit-matrix transposes across the warp, interleaved
// step by step (their shuffles and logic overlap instead of waiting on one
// another): lane r holds row r of each matrix (bit c = entry (r, c)) on entry
// and column r (bit c = entry (c, r)) on return.  Five steps; step j swaps
// the off-diagonal j x j blocks of each 2j x 2j block between lanes l and
// l ^ j, branch-free: a lane keeps its own half of each block (mask `keep`)
// and takes the partner's other half rotated into place (left by j for the
// lower lane of a pair, right by j for the upper one).
__device__ __forceinline__ void transpose32x4(uint32_t (&x)[4])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 16; j; j >>= 1) {
        const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu : j == 2 ? 0x33333333u
                                                                                                  : 0x55555555u;
        const uint32_t up = 0u - (uint32_t)((lane >> (31 - __clz(j))) & 1);
        const uint32_t keep = m ^ up;
        const int sh = up ? 32 - j : j;
        uint32_t y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) y[q] = __shfl_xor_sync(0xFFFFFFFFu, x[q], j);
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = (x[q] & keep) | (__funnelshift_l(y[q], y[q], sh) & ~keep);
    }
}

// Brings the 128-byte line holding *ptr into L2 (a hint: no data returned).
__device__ __forceinline__ void prefetch_l2(const void *ptr)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// Word-parallel donor scan over the staged rows (32 candidates per step):
// the first individual in cyclic order from `start`, skipping `self`, whose
// generation-start bits on F_j differ from the parent's bits xf; -1 if none.
__device__ int scan_rows(const uint32_t *sP, int SM, int e, int W, int Wv, int p, int s, uint32_t xf, int start,
                         int self)
{
    const int ws = start >> 5, bs = start & 31;
    for (int step = 0; step <= Wv; ++step) {
        int wc = ws + step;
        if (wc >= Wv) wc -= Wv;
        const uint32_t *row = sP + (e * W + wc) * SM;
        uint32_t diff = 0;
        for (int a = 0; a < s; ++a) diff |= row[a] ^ (0u - ((xf >> a) & 1u));
        const int lim = p - 32 * wc;
        uint32_t mk = diff & (lim >= 32 ? 0xFFFFFFFFu : ((1u << lim) - 1u));
        if (wc == (self >> 5)) mk &= ~(1u << (self & 31));
        if (step == 0)
            mk &= 0xFFFFFFFFu << bs;
        else if (step == Wv)
            mk &= ~(0xFFFFFFFFu << bs);
        if (mk) return 32 * wc + __ffs(mk) - 1;
    }
    return -1;
}

// First position at or after x, in cyclic order over [0, p), whose bit is set
// in the run starts rs[0..Wv); nz has bit w set iff rs[w] != 0 (so the next
// non-empty word is one bit scan away).  -1 if no bit is set.
__device__ __forceinline__ int next_run_start(const uint32_t *rs, uint32_t nz, int x)
{
    const int w = x >> 5;
    const uint32_t m = rs[w] & (0xFFFFFFFFu << (x & 31));
    if (m) return 32 * w + __ffs(m) - 1;
    const uint32_t later = nz & ~((2u << w) - 1u); // words after w
    const uint32_t any = later ? later : nz;        // else wrap round (word w's low bits included)
    if (!any) return -1;
    const int w2 = __ffs(any) - 1;
    return 32 * w2 + __ffs(rs[w2]) - 1;
}

// The donor of individual `self` (Sec. 4.2): the first candidate in cyclic
// order from `start`, skipping self, whose generation-start bits on F_j
// differ from the parent's current bits xf, or -1.  The search resumes at
// candidate `cur`, whose pattern is known to equal xf (start, or the one
// after it).  Candidates' patterns come from the packed table tc of P (the
// element's field at offset `off`); rs are the run starts of the element's
// patterns (bit d: pattern d differs from pattern d - 1, cyclically), so the
// candidates strictly inside a run equal to the parent are passed in one
// step (a run start after such a run differs from xf); after a few steps the
// word-parallel scan over the staged rows finishes the search.  *pd receives
// the donor's pattern.  Divergent code.
__device__ int find_donor_packed(const uint32_t *tc, int off, uint32_t fmask, const uint32_t *sP, const uint32_t *rs,
                                 uint32_t nz, int SM, int e, int W, int Wv, int p, int s, uint32_t xf, int start,
                                 int cur, int self, uint32_t *pd)
{
    int d = cur; // pattern d == xf here
    for (int it = 0; it < 4; ++it) {
        const int d2 = next_run_start(rs, nz, d + 1 == p ? 0 : d + 1);
        if (d2 < 0) return -1; // one run: every candidate equals the parent
        const int dist_d = d - start + (d < start ? p : 0);
        const int dist_2 = d2 - start + (d2 < start ? p : 0);
        if (dist_2 <= dist_d) return -1; // the jump passed the start
        if (d2 != self) {
            *pd = (tc[d2] >> off) & fmask;
            return d2;
        }
        d = d2 + 1 == p ? 0 : d2 + 1; // skip the parent's own column
        if (d == start) return -1;
        const uint32_t pat = (tc[d] >> off) & fmask;
        if (pat != xf) {
            *pd = pat;
            return d;
        }
    }
    const int d3 = d + 1 == p ? 0 : d + 1;
    if (d3 == start) return -1;
    const int r = scan_rows(sP, SM, e, W, Wv, p, s, xf, d3, self);
    if (r >= 0) *pd = (tc[r] >> off) & fmask;
    return r;
}

// Shared-memory words of one warp's region (SM = P.bs_sm, odd, so that the
// 32 lanes reading word a of their own rows hit 32 different banks; NC
// chunks of packed patterns): rows of O on F_j [32 pairs][SM], rows of P
// [32][SM], flip planes [32][SM], donor starts [32 pairs][32 individuals] as
// 16-bit values, run starts [32 pairs], packed patterns of P [NC][W][32],
// packed patterns of O [NC][W][32] (their slots reused for the packed flips),
// the item's element sizes [32] and the masks of their non-empty run-start
// words [32].
__host__ __device__ __forceinline__ int bs_warp_words(int SM, int NC, int W)
{
    return 96 * SM + 16 * 32 + 32 + 64 * NC * W + 64;
}

// The dynamic shared memory of the bit-sliced kernels: the block's fitness
// accumulators (32 W int64, i.e. 64 W words) first, then the warps' regions.
__device__ __forceinline__ uint32_t *bs_warp_region(const GomParams &P, uint32_t *s_dyn)
{
    return s_dyn + 64 * P.W + (threadIdx.x >> 5) * P.bs_words;
}

// Learned filter bookkeeping after a bit-sliced item (warp-wide): each
// element's accepted, donor-less and improving trials (summed over its W
// lanes) into this generation's history, the block's item counters s_fc (run,
// useful, audited, audited and useful; one item per element on this path),
// and for the elements the sampling hash picks a training sample -- the
// features as the select phase saw them, label: the element was useful (an
// accepted trial, or with P.flt.label an improving one).
__device__ __noinline__ void bs_record(const GomParams &P, int q, bool ke, bool audited, uint32_t g, unsigned acc,
                                       unsigned dl, unsigned imp, unsigned long long *s_fc)
{
    const int lane = threadIdx.x & 31;
    const int W = P.W, lw = __ffs(W) - 1, E = 32 >> lw;
    for (int off = 1; off < W; off <<= 1) {
        acc += __shfl_xor_sync(kFull, acc, off);
        dl += __shfl_xor_sync(kFull, dl, off);
        imp += __shfl_xor_sync(kFull, imp, off);
    }
    const bool useful = P.flt.label ? imp != 0 : acc != 0;
    if (ke && (lane & (W - 1)) == 0) {
        uint32_t *cur = P.flt.hist + (size_t)(g & 1) * 3 * (size_t)P.m;
        cur[q] = acc;
        cur[P.m + q] = dl;
        cur[2 * (size_t)P.m + q] = imp;
        atomicAdd(&s_fc[0], 1ull);
        if (useful) atomicAdd(&s_fc[1], 1ull);
        if (audited) atomicAdd(&s_fc[2], 1ull);
        if (audited && useful) atomicAdd(&s_fc[3], 1ull);
    }
    for (int e2 = 0; e2 < E; ++e2) {
        const int src = e2 << lw;
        const int q2 = __shfl_sync(kFull, q, src);
        const bool ok = __shfl_sync(kFull, ke ? 1 : 0, src) != 0;
        const bool u2 = __shfl_sync(kFull, useful ? 1 : 0, src) != 0;
        if (ok && filter_sample(q2, g)) {
            float x[kFilterIn];
            filter_features(P, q2, g, x);
            filter_log_sample(P, x, u2);
        }
    }
    __syncwarp();
}

// One item of colour group c at position t: entries [k0, k1) (at most E) of
// the group's elements -- positions k0 .. k1 - 1, or with the learned filter
// skipping, the positions qlist[k0 .. k1) of the compacted list -- with every
// word, all trials of Alg. 2.
template <int R, bool LEARN>
__device__ __forceinline__ void bs_item(const GomParams &P, const int32_t *qlist, int k0, int k1, uint32_t g,
                                        uint32_t *wsm, BsLane &L, long long *s_f, unsigned long long *s_fc)
{
    const int lane = threadIdx.x & 31;
    const int W = P.W, Wv = P.Wv, p = P.p, SM = P.bs_sm;
    const int lw = __ffs(W) - 1;
    const int e = lane >> lw, w = lane & (W - 1);
    const bool ke = k0 + e < k1; // this lane's element exists
    int q = k0 + e;
    bool audited = false;
    if (LEARN && qlist && ke) {
        const int32_t en = qlist[k0 + e];
        q = en & 0x7FFFFFFF;
        audited = en < 0;
    }
    const bool kv = ke && w < Wv; // this lane's pair exists
    uint32_t *sO = wsm, *sP = wsm + 32 * SM, *sD = wsm + 64 * SM;
    uint16_t *sStart = reinterpret_cast<uint16_t *>(wsm + 96 * SM); // p <= 1024: a start fits 16 bits
    uint32_t *sRS = wsm + 96 * SM + 16 * 32;

    // ---- phase 0: the pair's rows, run starts, donor starts
    int j = 0, s = 0, f0 = 0, d0 = 0, n_in = 0, n_out = 0;
    if (ke) {
        const int4 a = __ldg(P.hdr + 2 * q), b = __ldg(P.hdr + 2 * q + 1);
        j = a.x;
        f0 = a.y;
        d0 = a.z;
        s = a.w & 0xFF;
        n_in = a.w >> 8;
        n_out = b.x;
        // the element's edge list and segment offsets are read in phase 2:
        // ask for their lines in L2 now (the W lanes of the element take every
        // W-th line; the arrays start on 256-byte boundaries, so every line
        // named here holds bytes of the array)
        const uintptr_t d_at = reinterpret_cast<uintptr_t>(P.dep + d0), d_end = d_at + 8u * (uint32_t)(n_out + n_in);
        for (uintptr_t at = (d_at & ~uintptr_t(127)) + 128u * (uint32_t)w; at < d_end; at += 128u * (uint32_t)W)
            prefetch_l2(reinterpret_cast<const void *>(at));
        if (w == 0) {
            prefetch_l2(P.seg + f0 + q);
            prefetch_l2(P.seg + f0 + q + s);
        }
    }
    for (int a4 = 0; a4 < SM; a4 += 4) {
        uint32_t xo[4], xp[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            xo[c] = xp[c] = 0;
            if (kv && a4 + c < s) {
                const int64_t v = __ldg(P.fv + f0 + a4 + c);
                xo[c] = P.O[v * W + w];
                xp[c] = P.P[v * W + w];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (a4 + c < SM) {
                sO[lane * SM + a4 + c] = xo[c];
                sP[lane * SM + a4 + c] = xp[c];
            }
    }
    __syncwarp();
    {   // run starts of the element's patterns in word w: bit b set iff the
        // pattern of individual 32 w + b differs from the one before it (cyclically)
        uint32_t rsw = 0;
        if (kv) {
            const uint32_t *cur = sP + lane * SM;
            const uint32_t *prev = sP + (e * W + (w == 0 ? Wv - 1 : w - 1)) * SM;
            const int pb = w == 0 ? (p - 1) & 31 : 31;
            for (int a = 0; a < s; ++a) {
                const uint32_t x = cur[a];
                rsw |= x ^ ((x << 1) | ((prev[a] >> pb) & 1u));
            }
            const int lim = p - 32 * w;
            rsw &= lim >= 32 ? 0xFFFFFFFFu : ((1u << lim) - 1u);
        }
        sRS[lane] = rsw;
        // element e's words with a run start: bits e W .. e W + W - 1 of the ballot
        const uint32_t nzb = __ballot_sync(0xFFFFFFFFu, rsw != 0);
        if (w == 0)
            wsm[96 * SM + 16 * 32 + 32 + 64 * P.bs_nc * W + 32 + e] = W == 32 ? nzb : (nzb >> (e * W)) & ((1u << W) - 1u);
    }
    {   // donor starts: call (pair k2, c) covers individuals 32 w2 + 4c .. + 3
#pragma unroll 1
        for (int r = 0; r < 8; ++r) {
            const int k2 = 4 * r + (lane >> 3), c = lane & 7;
            const int w2 = k2 & (W - 1);
            const int j2 = __shfl_sync(0xFFFFFFFFu, j, k2);
            const bool v2 = __shfl_sync(0xFFFFFFFFu, kv ? 1 : 0, k2) && 32 * w2 + 4 * c < p;
            if (v2) {
                const uint4 r4 = philox10_rk(make_uint4((uint32_t)j2, (uint32_t)(8 * w2 + c), g, kTagDonor), P.rk);
                const int i0 = 32 * w2 + 4 * c;
                int st[4];
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int d = i0 + cc + 1 + (int)__umulhi(pick(r4, cc), (uint32_t)(p - 1));
                    st[cc] = d >= p ? d - p : d;
                }
                *reinterpret_cast<uint2 *>(sStart + k2 * 32 + 4 * c) =
                    make_uint2((uint32_t)st[0] | ((uint32_t)st[1] << 16), (uint32_t)st[2] | ((uint32_t)st[3] << 16));
            }
        }
    }
    // packed patterns: for chunk c (elements c EPW .. c EPW + EPW - 1 of the
    // item) and word w2, lane b receives the bits of individual 32 w2 + b on
    // the chunk's elements side by side (element e_c at bit offset e_c S), by
    // one transpose of the rows (row r = variable r mod S of element r / S);
    // four words at a time, interleaved
    const int S = P.bs_S, EPW = P.bs_epw, NC = P.bs_nc;
    const int E = 32 >> lw;
    uint32_t *tabP = wsm + 96 * SM + 16 * 32 + 32, *tabO = tabP + 32 * NC * W;
    uint32_t *sFM = tabO; // a lane reads its entry of tabO before it writes the same entry of sFM
    int *sS = reinterpret_cast<int *>(tabO + 32 * NC * W);
    const uint32_t *sNZ = tabO + 32 * NC * W + 32; // per element slot: its non-empty run-start words
    const uint32_t fmask = S >= 32 ? 0xFFFFFFFFu : ((1u << S) - 1u);
    if (w == 0) sS[e] = s; // the item's element sizes, by slot
    const int er = lane / S, ar = lane - er * S; // this lane's row in a transpose: element er of a chunk, variable ar
    for (int c = 0; c < NC; ++c) {
        const int e3 = c * EPW + er;
        const bool row = er < EPW && e3 < E;
        for (int w2 = 0; w2 < Wv; w2 += 4) {
            uint32_t tp[4], to[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int at = (e3 * W + w2 + j) * SM + ar;
                const bool ok = row && w2 + j < Wv;
                tp[j] = ok ? sP[at] : 0u;
                to[j] = ok ? sO[at] : 0u;
            }
            transpose32x4(tp);
            transpose32x4(to);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (w2 + j < Wv) {
                    tabP[(c * W + w2 + j) * 32 + lane] = tp[j];
                    tabO[(c * W + w2 + j) * 32 + lane] = to[j];
                }
        }
    }
    __syncwarp();

    // ---- phase 1: donors, lane = individual.  Pass A checks every pair's
    // start candidate (one table lookup) and, when it equals the parent on
    // F_j, takes the first run start after it (one more); pass B searches
    // again from the start for the rare individuals whose run start is their
    // own column (run starts, then the word-parallel scan).  Each word's
    // flips of a chunk are packed like the patterns into sFM.
    for (int w2 = 0; w2 < Wv; ++w2) {
        const int i = 32 * w2 + lane;
        const bool vi = i < p;
        for (int c = 0; c < NC; ++c) {
            const uint32_t xo = tabO[(c * W + w2) * 32 + lane]; // the parents' current patterns
            const int ne = min(EPW, min(E, k1 - k0) - c * EPW); // elements of this chunk in the item
            const uint32_t *tc = tabP + c * W * 32;             // chunk c's patterns, by individual
            const uint16_t *sc = sStart + (c * EPW * W + w2) * 32 + lane;
            uint32_t fmw = 0, fails = 0;
#pragma unroll 4
            for (int el = 0; el < ne; ++el) {
                const int e2 = c * EPW + el;
                // the element's field of the packed words: its flips are (donor ^ parent) & field
                const uint32_t field = fmask << (el * S);
                // starts exist for individuals < p only (others read candidate 0, and are dropped below)
                const int st = vi ? sc[el * W * 32] : 0;
                // every candidate from st up to the next run start d2 has st's pattern; when
                // that is the parent's, d2 differs from it and is the donor -- unless it is
                // the parent's own column (pass B); no run start: no donor.  d2 is found
                // whatever st's pattern (branch-free, all loads issued together)
                const int x = st + 1 == p ? 0 : st + 1, wx = x >> 5;
                const uint32_t *rs = sRS + e2 * W;
                const uint32_t nzm = sNZ[e2];
                const uint32_t later = nzm & ~((2u << wx) - 1u); // run-start words after wx
                const uint32_t any = later ? later : nzm;          // else wrap round
                const int wy = any ? __ffs(any) - 1 : 0;
                const uint32_t t1 = tc[st], r1 = rs[wx], r2 = rs[wy];
                const uint32_t m = r1 & (0xFFFFFFFFu << (x & 31));
                const int d2 = m ? 32 * wx + __ffs(m) - 1 : any ? 32 * wy + __ffs(r2) - 1 : -1;
                const uint32_t t2 = tc[d2 < 0 ? 0 : d2];
                const uint32_t f1 = (t1 ^ xo) & field;
                const uint32_t f2 = d2 >= 0 && d2 != i ? (t2 ^ xo) & field : 0u;
                fmw |= f1 ? f1 : f2;
                fails |= !f1 && d2 == i ? 1u << el : 0u;
            }
            if (!vi) fmw = fails = 0;
            for (uint32_t f = fails; f; f &= f - 1) { // pass B, divergent
                const int el = __ffs(f) - 1, off = el * S, e2 = c * EPW + el;
                const uint32_t xf = (xo >> off) & fmask;
                const int st = sStart[(e2 * W + w2) * 32 + lane];
                uint32_t pd = 0;
                const int d = find_donor_packed(tabP + c * W * 32, off, fmask, sP, sRS + e2 * W, sNZ[e2], SM, e2, W, Wv, p,
                                                sS[e2], xf, st, st, i, &pd);
                if (d >= 0) fmw |= (pd ^ xf) << off;
            }
            sFM[(c * W + w2) * 32 + lane] = fmw;
        }
    }
    __syncwarp();
    // the flip planes: lane r of the transpose of a word's packed flips gets
    // variable r mod S of element r / S of the chunk (bit b: individual 32 w2 + b
    // flips it); four words at a time
    for (int c = 0; c < NC; ++c) {
        const int e3 = c * EPW + er;
        const bool row = er < EPW && e3 < E;
        for (int w2 = 0; w2 < Wv; w2 += 4) {
            uint32_t tf[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) tf[j] = w2 + j < Wv ? sFM[(c * W + w2 + j) * 32 + lane] : 0u;
            transpose32x4(tf);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (row && w2 + j < Wv) sD[(e3 * W + w2 + j) * SM + ar] = tf[j];
        }
    }
    __syncwarp();

    // ---- phase 2: bit-plane partial evaluation, acceptance, write, lane = pair
    unsigned i_acc = 0, i_dl = 0, i_imp = 0; // this pair's accepted, donor-less and improving trials
    // each item adds less than 2^R to an individual's sum: flush before it could pass 2^kFitPlanes
    if (L.since_flush >= (1 << (kFitPlanes - R))) bs_flush(P, L, s_f);
    if (kv) {
        const uint32_t *myD = sD + lane * SM, *myO = sO + lane * SM;
        // the delta of every trial, R + 1 planes two's complement: an edge that
        // a trial toggles adds |w| if it was uncut (with its sign folded into
        // the cut bit), -|w| if it was cut (Eq. 1); no partial sum leaves
        // (-2^R, 2^R) since the element's sum of |w| is below 2^R
        uint32_t D[R + 1];
#pragma unroll
        for (int t = 0; t <= R; ++t) D[t] = 0;
        uint32_t hd = 0;
        for (int a = 0; a < s; ++a) {
            const uint32_t Fa = myD[a];
            hd |= Fa;
            if (!Fa) continue; // no trial flips variable a: none of its edges changes
            const uint32_t Xa = myO[a];
            const int xb = (int)__ldg(P.seg + f0 + q + a), xe = (int)__ldg(P.seg + f0 + q + a + 1);
            for (int x = xb; x < xe; x += 4) { // four edges' loads issued before their arithmetic
                int2 ed[4];
                uint32_t Xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) ed[u] = x + u < xe ? __ldg(P.dep + d0 + x + u) : make_int2(0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) Xv[u] = x + u < xe ? P.O[(int64_t)ed[u].x * W + w] : 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // an outgoing edge toggles wherever a flips
                    const uint32_t cut = Xa ^ Xv[u] ^ (uint32_t)(ed[u].y >> 31);
                    if (x + u < xe)
                        add_signed<R + 1, kWeightBits>(D, Fa & ~cut, Fa & cut, (uint32_t)(ed[u].y < 0 ? -ed[u].y : ed[u].y));
                }
            }
        }
        for (int x = n_out; x < n_out + n_in; ++x) {
            const int2 ed = __ldg(P.dep + d0 + x);
            const int a = ed.x & 0xFF, b = ed.x >> 8;
            const uint32_t tg = myD[a] ^ myD[b];
            if (!tg) continue; // the edge toggles for no individual
            const uint32_t cut = myO[a] ^ myO[b] ^ (uint32_t)(ed.y >> 31);
            add_signed<R + 1, kWeightBits>(D, tg & ~cut, tg & cut, (uint32_t)(ed.y < 0 ? -ed.y : ed.y));
        }
        uint32_t nz = 0;
#pragma unroll
        for (int t = 0; t <= R; ++t) nz |= D[t];
        const uint32_t neg = D[R];
        const uint32_t pos = nz & ~neg;
        const int lim = p - 32 * w;
        const uint32_t vm = lim >= 32 ? 0xFFFFFFFFu : ((1u << lim) - 1u);
        const uint32_t eqv = P.eqw[(g & 1) * W + w];
        const uint32_t acc = hd & vm & (pos | (~nz & ~eqv));
        i_acc = __popc(acc);
        i_imp = __popc(acc & pos);
        i_dl = __popc(vm & ~hd);
        L.n_acc += i_acc;
        L.n_imp += i_imp;
        L.n_dl += i_dl;
        if (P.fi.on && acc) atomicOr(&P.fi.accw[w], acc); // Forced Improvement: who had an accepted step
        if (acc) {
            for (int a = 0; a < s; ++a) {
                const uint32_t m = myD[a] & acc;
                if (m) {
                    const int64_t v = __ldg(P.fv + f0 + a);
                    P.O[v * W + w] = myO[a] ^ m;
                }
            }
            fit_add<R>(L, D, acc); // the accepted deltas (>= 0, below 2^R)
        }
    }
    ++L.since_flush;
    __syncwarp();
    if (LEARN && P.learn) bs_record(P, q, ke, audited, g, i_acc, i_dl, i_imp, s_fc);
}

// One colour group (position t, colour c) on the bit-sliced path: items of
// E = 32 / W consecutive elements of the group -- of the compacted list of the
// elements to run while the learned filter skips elements; warp x takes item
// x, then items nwarps + the claims it draws from work[t] (P.dyn), one ahead,
// or x + nwarps, x + 2 nwarps, ... (static stride).
template <int R, bool LEARN>
__device__ void phase_mix_bs(const GomParams &P, const VGrid &V, int t, int c, uint32_t g, uint32_t *wsm, BsLane &L,
                             long long *s_f, unsigned long long *s_fc)
{
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)(V.thread() >> 5), nwarps = (int)(V.threads() >> 5);
    const int E = 32 / P.W;
    const bool cl = LEARN && P.learn == 2 && P.flt.compact;
    const int32_t *qlist = cl ? P.flt.act : nullptr;
    const int ka = cl ? P.flt.act_ptr[c] : P.cptr[c], kz = cl ? P.flt.act_ptr[c + 1] : P.cptr[c + 1];
    const int items = (kz - ka + E - 1) / E;
    unsigned claim = 0;
    if (P.dyn && lane == 0) claim = atomicAdd(&P.work[t], 1u);
    for (int it = gwarp, next = gwarp + nwarps; it < items;) {
        const int k0 = ka + it * E;
        bs_item<R, LEARN>(P, qlist, k0, min(k0 + E, kz), g, wsm, L, s_f, s_fc);
        if (P.dyn) {
            it = nwarps + (int)__shfl_sync(0xFFFFFFFFu, claim, 0);
            if (it < items && lane == 0) claim = atomicAdd(&P.work[t], 1u);
        } else {
            it = next;
            next += nwarps;
        }
    }
}

// Adds the warp's counters and the lanes' fitness sums into the block's
// accumulators.
__device__ __forceinline__ void bs_finish_generation(const GomParams &P, BsLane &L, long long *s_f,
                                                     unsigned long long *s_cnt)
{
    bs_flush(P, L, s_f);
    count_flush(s_cnt, L.n_dl, L.n_acc, L.n_imp);
    L.n_dl = L.n_acc = L.n_imp = 0;
}

// Up to G generations of one context on the bit-sliced phase, on the blocks
// of the (virtual) grid V, the phases separated by grid barriers on `bar`:
// [generation start + group order] | group 0 | ... | group k-1 | and again;
// every block computes a generation's end from the fitness array after the
// barrier that closes its last group (block 0 of V records it).  s_keys: room
// for the k group keys of the order phase (it may overlay wsm and s_f, which
// are set up after it); wsm: this warp's region; s_f, s_cnt: the block's
// fitness accumulators and counters; s_fc: the learned filter's block
// counters (LEARN only).
template <int R, bool LEARN>
__device__ __forceinline__ void bs_generations(const GomParams &P, const VGrid &V, GomBarrier *bar, int G,
                                               int64_t target, unsigned long long *s_keys, uint32_t *wsm,
                                               long long *s_f, unsigned long long *s_cnt, unsigned long long *s_fc)
{
    const unsigned nblk = (unsigned)V.nblk;
    const bool lead = V.blk == 0;
    uint32_t g = P.st->g;
    GenEnd e{P.st->fe, P.st->improved, P.st->argmax};
    unsigned long long bnext = 0;
    if (threadIdx.x == 0) bnext = barrier_first(&bar->count, nblk);
    if (lead && threadIdx.x == 0) {
        P.st->call_g0 = g;
        P.st->target = target;
    }
    const bool tr = P.trace != nullptr && lead && threadIdx.x == 0;
    BsLane L;
    bs_lane_zero(L);
    for (int qg = 0; qg < G; ++qg) {
        if (qg > 0 && phase_gen_end(P, target, g - 1, e, lead)) return;
        if (tr) P.trace[0] = global_ns();
        phase_gen_start(P, V, e.improved, e.argmax, g, true);
        phase_order(P, V, s_keys, g);
        if (LEARN) fc_zero(s_fc);
        acc_zero(P, s_f, s_cnt);
        if (tr) P.trace[1] = P.trace[2] = global_ns();
        if (!grid_barrier(&bar->count, &P.st->err, nblk, bnext, kBarrierNs)) return;
        if (LEARN && P.learn && !phase_filter_select(P, V, g, &bar->count, nblk, bnext, P.learn == 2 && P.flt.compact))
            return;
        if (tr) P.trace[3] = global_ns();
        for (int t = 0; t < P.k; ++t) {
            if (t > 0 && !grid_barrier(&bar->count, &P.st->err, nblk, bnext, kBarrierNs)) return;
            if (tr) P.trace[4 + 2 * t] = global_ns();
            phase_mix_bs<R, LEARN>(P, V, t, P.order[t], g, wsm, L, s_f, s_fc);
            if (tr) P.trace[5 + 2 * t] = global_ns();
        }
        bs_finish_generation(P, L, s_f, s_cnt);
        acc_flush(P, s_f, s_cnt);
        if (LEARN) fc_flush(P, s_fc);
        if (!grid_barrier(&bar->count, &P.st->err, nblk, bnext, kBarrierNs)) return;
        if (P.fi.on && !fi_generation<R>(P, V, &bar->count, nblk, bnext, e, P.order, s_f, s_cnt)) return;
        if (tr) P.trace[4 + 2 * P.k] = global_ns();
        ++g;
    }
    if (G > 0 && lead) phase_gen_end(P, target, g - 1, e, true);
}

} // namespace
