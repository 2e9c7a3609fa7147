// gom_kernels.cu -- sm_103a kernels of parallel GOM for weighted Max-Cut.
//
// Population layout (bit-sliced, variable-major): O[v*W + w] holds variable v
// of individuals 32w .. 32w+31, one bit each.  W is a power of two; words and
// bits past the population size stay zero.  A warp therefore reads one
// variable of 32 individuals with a single broadcast load, and the writes of
// one GOM trial batch (32 individuals x one element) are whole words.
//
// Kernels of one generation (Alg. 3):
//   gen start  Clone (P <- O), copy of the new elitist, elitist flags
//   order      random order of the colour groups
//   mix        one phase per colour group: every (individual, element) trial
//              of the group -- donor, partial evaluation, accept, write
//   gen end    elitist update, counters, target check
// Two ways to run them: one kernel per phase in a per-generation CUDA graph
// (k_gen_start, k_order, k_mix, k_gen_end), or one persistent cooperative
// kernel (k_run) that runs many generations with grid barriers between the
// phases.  Plus initialisation, full evaluation and import/export kernels.
#include <climits>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gom_bs.cuh"
#include "gom_device.cuh"
#include "gom_fi.cuh"
#include "gom_filter_dev.cuh"
#include "gom_internal.h"
#include "gom_kernels.cuh"


// ----------------------------------------------------------------------------
// InitializePopulation (Alg. 3): one Philox call gives 128 variables of one
// individual; a warp covers 32 individuals and turns each variable into one
// word with a ballot.
__global__ void k_init_pop(GomParams P)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = gthread() >> 5, nwarps = gthreads() >> 5;
    const int64_t nq = (P.n + 127) / 128;
    const int64_t items = nq * P.W;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    for (int64_t it = warp; it < items; it += nwarps) {
        const int64_t q = it / P.W;
        const int w = (int)(it - q * P.W);
        const int i = 32 * w + lane;
        const bool valid = i < P.p;
        const uint4 r = philox10(make_uint4((uint32_t)q, (uint32_t)i, 0u, kTagInit), k0, k1);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t word = pick(r, t);
            uint32_t mine = 0;
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                const uint32_t mk = __ballot_sync(kFull, valid && ((word >> b) & 1u));
                if (lane == b) mine = mk;
            }
            const int64_t v = 128 * q + 32 * t + lane;
            if (v < P.n) P.O[v * P.W + w] = mine;
        }
    }
}

// Full evaluation (Sec. 6.2): f[i] = sum over edges {u<v} of w_uv [x_u != x_v].
// A warp takes chunks of 32 vertices for one word; lane = individual.
// The number of warps in the grid is a multiple of W.
__global__ void k_fitness(GomParams P, int64_t *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = gthread() >> 5, nwarps = gthreads() >> 5;
    const int w = (int)(warp & (P.W - 1));
    if (w >= P.Wv) return;
    const int64_t nchunks = (P.n + 31) / 32;
    long long acc = 0;
    for (int64_t ch = warp / P.W; ch < nchunks; ch += nwarps / P.W) {
        const int64_t uend = min((int64_t)P.n, 32 * ch + 32);
        for (int64_t u = 32 * ch; u < uend; ++u) {
            const uint32_t xu = P.O[u * P.W + w];
            for (int64_t e = P.row_ptr[u]; e < P.row_ptr[u + 1]; ++e) {
                const int64_t v = P.col[e];
                if (v > u && (((xu ^ P.O[v * P.W + w]) >> lane) & 1u)) acc += P.wgt[e];
            }
        }
    }
    const int i = 32 * w + lane;
    if (i < P.p && acc) atomicAdd((unsigned long long *)&out[i], (unsigned long long)acc);
}

// Elitist of a fresh population: lowest index of maximal fitness.
__global__ void k_elite_init(GomParams P)
{
    int64_t best;
    int arg;
    block_argmax(P.f, P.p, &best, &arg);
    if (threadIdx.x == 0) {
        P.st->fe = best;
        P.st->best = best;
        P.st->argmax = arg;
        P.st->improved = 1;
        P.st->done = 0;
    }
    for (int w = threadIdx.x; w < 2 * P.W; w += blockDim.x) P.eqw[w] = kFull;
}

// State after an import: given elitist fitness and generation counter.
__global__ void k_set_state(GomParams P, int64_t fe, int64_t g)
{
    if (threadIdx.x == 0) {
        P.st->fe = fe;
        P.st->best = fe;
        P.st->argmax = 0;
        P.st->improved = 0;
        P.st->done = 0;
        P.st->g = (uint32_t)g;
        P.st->cnt[0] = P.st->cnt[1] = P.st->cnt[2] = P.st->cnt[3] = 0;
    }
    for (int w = threadIdx.x; w < 2 * P.W; w += blockDim.x) P.eqw[w] = kFull;
}

__global__ void k_begin_call(GomParams P, int64_t target)
{
    P.st->done = 0;
    P.st->target = target;
    P.st->call_g0 = P.st->g; // first generation of this call
}


// Loads WPI consecutive 32-bit words (16/8/4-byte aligned by construction);
// works on global and shared memory.
template <int WPI>
__device__ __forceinline__ void load_words(const uint32_t *p, uint32_t (&x)[WPI])
{
    if constexpr (WPI == 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else if constexpr (WPI == 2) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        x[0] = v.x; x[1] = v.y;
    } else {
        x[0] = *p;
    }
}

// Stores WPI consecutive 32-bit words (aligned as in load_words).
template <int WPI>
__device__ __forceinline__ void store_words(uint32_t *p, const uint32_t (&x)[WPI])
{
    if constexpr (WPI == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(x[0], x[1], x[2], x[3]);
    } else if constexpr (WPI == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(x[0], x[1]);
    } else {
        *p = x[0];
    }
}

// First individual, scanning cyclically upwards from `start` and skipping
// `self`, whose generation-start bits on F differ from the parent's bits
// `xf`; 32 candidates per step from the staged rows sP[a*W + word] of P on
// F.  -1 if none.  Called from divergent code: no warp collectives.
template <typename MaskT>
__device__ int scan_donor(const uint32_t *sP, int W, int Wv, int p, int s, MaskT xf, int start, int self)
{
    const int ws = start >> 5, bs = start & 31;
    for (int step = 0; step <= Wv; ++step) {
        int wc = ws + step;
        if (wc >= Wv) wc -= Wv;
        uint32_t diff = 0;
        for (int a = 0; a < s; ++a) diff |= sP[a * W + wc] ^ (0u - (uint32_t)((xf >> a) & 1u));
        const int lim = p - 32 * wc;
        uint32_t mk = diff & (lim >= 32 ? kFull : ((1u << lim) - 1u));
        if (wc == (self >> 5)) mk &= ~(1u << (self & 31));
        if (step == 0)
            mk &= kFull << bs;
        else if (step == Wv)
            mk &= ~(kFull << bs);
        if (mk) return 32 * wc + __ffs(mk) - 1;
    }
    return -1;
}

// Value held by lane (a mod 32) of X[a / 32][r]: per-variable registers of
// elements with up to 32 NQ variables, lane l holding variables l, l + 32,
// ...  Warp-uniform a.
template <int NQ, int WPI>
__device__ __forceinline__ uint32_t lane_get(const uint32_t (&X)[NQ][WPI], int r, int a)
{
    if constexpr (NQ == 1) {
        return __shfl_sync(kFull, X[0][r], a);
    } else {
        uint32_t v = X[0][r];
#pragma unroll
        for (int h = 1; h < NQ; ++h) v = (a >> 5) == h ? X[h][r] : v;
        return __shfl_sync(kFull, v, a & 31);
    }
}


// The donor of individual `self` (Sec. 4.2, reading 6): the first candidate in
// cyclic order from `start`, skipping self, whose generation-start bits on F_j
// (patP) differ from the parent's bits xf; -1 if there is none.  rs marks the
// starts of runs of equal patterns (bit d: patP[d] != patP[d-1], cyclically),
// so a run of candidates equal to the parent is passed in one step.  After a
// few steps (only possible when the parent's own column interrupts runs)
// the word-parallel scan over the staged rows finishes the search.  Divergent
// code: no warp collectives.
template <typename MaskT>
__device__ int find_donor(const MaskT *patP, const uint32_t *rs, const uint32_t *sP, int W, int Wv, int p, int s,
                          MaskT xf, int start, int self)
{
    if (patP[start] != xf) return start;
    int d = start; // patP[d] == xf here
    for (int it = 0; it < 4; ++it) {
        const int d2 = next_set_cyclic(rs, Wv, p, d);
        if (d2 < 0) return -1; // one run: every candidate equals the parent
        // candidates strictly between d and d2 equal patP[d] == xf; stop if the jump passed start
        const int dist_d = d - start + (d < start ? p : 0);
        const int dist_2 = d2 - start + (d2 < start ? p : 0);
        if (dist_2 <= dist_d) return -1;
        if (d2 != self) return d2;
        d = d2 + 1 == p ? 0 : d2 + 1; // skip the parent's own column
        if (d == start) return -1;
        if (patP[d] != xf) return d;
    }
    // no donor between start and d: continue with a full scan from the next position
    const int d3 = d + 1 == p ? 0 : d + 1;
    if (d3 == start) return -1;
    return scan_donor<MaskT>(sP, W, Wv, p, s, xf, d3, self);
}


// A staging slice (one mixing item: an element and a range of its words):
//  hdr[8] = {valid, q, sub, n_out, j, f0, d0, s | n_in << 8}
//  fv[s] variables, seg[s+1] their outside-edge starts, wout[s] their outside
//  weight sums (int64), rows of P on F_j [s][W], patP[32 W] every individual's
//  bits on F_j, rs[W] run starts of patP, cw[E] each edge's {code, weight},
//  xw[E_out][WPI] the outside edges' parent words, and in stage-all mode the
//  donor start positions of the item's individuals.
// Offsets come from the host (the one definition of the layout).

// Slice header words: validity, element position q, word group, outside
// edges, then the element header {j, f0, d0, s | n_in << 8}.
enum : int { H_VALID = 0, H_Q = 1, H_SUB = 2, H_NOUT = 3, H_J = 4, H_F0 = 5, H_D0 = 6, H_SN = 7 };

// Header of item (element at position q, word group sub), written by one lane.
__device__ __forceinline__ void write_item_header(const GomParams &P, int q, int sub, int *h)
{
    const int4 a = P.hdr[2 * q], b = P.hdr[2 * q + 1];
    h[H_Q] = q;
    h[H_SUB] = sub;
    h[H_NOUT] = b.x;
    h[H_J] = a.x;
    h[H_F0] = a.y;
    h[H_D0] = a.z;
    h[H_SN] = a.w;
}

// Decodes item `it` of colour c into the slice header (lane 0 writes).
// Returns validity.  A warp-uniform result.
__device__ __forceinline__ bool decode_item(const GomParams &P, int c, int it, int WPI_, uint32_t *sl)
{
    const int q0 = P.cptr[c], ne = P.cptr[c + 1] - q0;
    const int nwg = (P.Wv + WPI_ - 1) / WPI_;
    const int per = P.split ? nwg : 1;
    const bool valid = it < ne * per;
    if ((threadIdx.x & 31) == 0) {
        int *h = reinterpret_cast<int *>(sl);
        h[H_VALID] = valid;
        if (valid) write_item_header(P, q0 + it / per, it % per, h);
    }
    return valid;
}

// Level-1 copies of a decoded item: variables, their edge starts and weight
// sums, and the edge list (code, weight).
template <int WPI>
__device__ __forceinline__ void stage_lists(const GomParams &P, uint32_t *sl)
{
    const int lane = threadIdx.x & 31;
    const int *h = reinterpret_cast<const int *>(sl);
    const int q = h[H_Q], d0 = h[H_D0], s = h[H_SN] & 0xFF, n_in = h[H_SN] >> 8, n_out = h[H_NOUT], f0 = h[H_F0];
    for (int a = lane; a < s; a += 32) {
        cp_async4(sl + P.off_fv + a, P.fv + f0 + a);
        cp_async8(sl + P.off_wout + 2 * a, P.wout + f0 + a);
    }
    for (int a = lane; a <= s; a += 32) cp_async4(sl + P.off_seg + a, P.seg + f0 + q + a);
    for (int x = lane; x < n_out + n_in; x += 32) cp_async8(sl + P.off_cw + 2 * x, P.dep + d0 + x);
}

// Level-2 copies: the rows of the generation-start population on F_j (all W
// words), from the staged variables; src is P, or O before anything of the
// generation is written.
__device__ __forceinline__ void stage_rows(const GomParams &P, uint32_t *sl, const uint32_t *src)
{
    const int lane = threadIdx.x & 31;
    const int *h = reinterpret_cast<const int *>(sl);
    const int s = h[H_SN] & 0xFF, W = P.W;
    const int *fv = reinterpret_cast<const int *>(sl + P.off_fv);
    uint32_t *sP = sl + P.off_pr;
    if (W >= 4) {
        const int n4 = (s * W) >> 2, lw4 = __ffs(W >> 2) - 1;
        for (int x = lane; x < n4; x += 32) {
            const int a = x >> lw4, w4 = x & ((W >> 2) - 1);
            cp_async16(sP + 4 * x, src + fv[a] * W + 4 * w4);
        }
    } else {
        const int lw = __ffs(W) - 1;
        for (int x = lane; x < (s << lw); x += 32) cp_async4(sP + x, src + fv[x >> lw] * W + (x & (W - 1)));
    }
}

// Pattern table and its run starts, from the staged rows (no global memory).
template <typename MaskT>
__device__ __forceinline__ void stage_patterns(const GomParams &P, uint32_t *sl)
{
    const int lane = threadIdx.x & 31;
    const int *h = reinterpret_cast<const int *>(sl);
    const int s = h[H_SN] & 0xFF, W = P.W, Wv = P.Wv, p = P.p;
    const uint32_t *sP = sl + P.off_pr;
    MaskT *patP = reinterpret_cast<MaskT *>(sl + P.off_pat);
    uint32_t *rs = sl + P.off_rs;
    // lane l builds the bits on F_j of individuals 32 wc + l
    for (int wc = 0; wc < Wv; ++wc) {
        MaskT pat = 0;
        for (int a = 0; a < s; ++a) pat |= (MaskT)((sP[a * W + wc] >> lane) & 1u) << a;
        patP[32 * wc + lane] = pat;
    }
    __syncwarp();
    for (int wc = 0; wc < Wv; ++wc) {
        const int d = 32 * wc + lane;
        const bool start = d < p && patP[d] != patP[d == 0 ? p - 1 : d - 1];
        const uint32_t b = __ballot_sync(kFull, start);
        if (lane == 0) rs[wc] = b;
    }
    __syncwarp();
}

// Donor start positions of the item's individuals (Sec. 4.2, reading 6):
// individual i of element j starts its cyclic scan at
// i + 1 + mulhi(r, p - 1) mod p, r word i mod 4 of Philox(j, i / 4, g, DONR).
// Lane c makes the call of individuals 4c .. 4c+3 of a word group and stores
// their four starts together, so the start of individual 32 (w0 + r) + l sits
// at int (wg - wg0) 32 WPI + 32 r + l of the region.
template <int WPI>
__device__ __forceinline__ void stage_draws(const GomParams &P, uint32_t *sl, uint32_t g)
{
    const int lane = threadIdx.x & 31;
    const int *h = reinterpret_cast<const int *>(sl);
    const int j = h[H_J], sub = h[H_SUB];
    const int nwg = (P.Wv + WPI - 1) / WPI;
    const int wg0 = P.split ? sub : 0, wg1 = P.split ? sub + 1 : nwg;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const int p = P.p;
    int4 *ds = reinterpret_cast<int4 *>(sl + P.off_ds);
    for (int wg = wg0; wg < wg1; ++wg) {
        const int w0 = wg * WPI;
        if (lane < 8 * WPI) {
            const uint4 r4 = philox10(make_uint4((uint32_t)j, (uint32_t)(8 * w0 + lane), g, kTagDonor), k0, k1);
            const int i0 = 32 * w0 + 4 * lane;
            int st[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int d = i0 + c + 1 + (int)__umulhi(pick(r4, c), (uint32_t)(p - 1));
                st[c] = d >= p ? d - p : d;
            }
            ds[(wg - wg0) * 8 * WPI + lane] = make_int4(st[0], st[1], st[2], st[3]);
        }
    }
}

// ----------------------------------------------------------------------------
// Learned trial filter: features, logit, hashes and the select phase are in
// gom_filter_dev.cuh; the decision of each element is taken there, after the
// generation start, and read here when an item is staged.

// Slice validity states: no item, staged, skipped by the filter, staged for an audit.
enum : int { IT_NONE = 0, IT_STAGED = 1, IT_SKIPPED = 2, IT_AUDIT = 3 };

// The filter's decision on a decoded item (warp-wide), as the select phase
// took it for its element: IT_STAGED, IT_SKIPPED or IT_AUDIT; written to the
// slice header.
__device__ __forceinline__ int filter_decide(const GomParams &P, uint32_t *sl)
{
    const int q = reinterpret_cast<const int *>(sl)[H_Q];
    const uint8_t d = P.flt.dec[q];
    const int state = d == DEC_SKIP ? IT_SKIPPED : d == DEC_AUDIT ? IT_AUDIT : IT_STAGED;
    __syncwarp();
    if ((threadIdx.x & 31) == 0) sl[H_VALID] = (uint32_t)state;
    __syncwarp();
    return state;
}

// Stages one item of colour c (item index `it`) into a slice: decode, then
// two levels of asynchronous copies, then the pattern table.  Only
// generation-constant data: it may run before the barrier that opens the
// group.  With the learned filter on, an element predicted to accept nothing
// is not staged (IT_SKIPPED) unless it is audited.  Returns the slice state.
template <int WPI, typename MaskT, bool LEARN>
__device__ __forceinline__ int stage_item(const GomParams &P, int c, int it, uint32_t *sl, uint32_t g)
{
    __syncwarp();
    const bool valid = decode_item(P, c, it, WPI, sl);
    if (!valid) return IT_NONE;
    __syncwarp();
    int state = IT_STAGED;
    if (LEARN && P.learn == 2) {
        state = filter_decide(P, sl);
        if (state == IT_SKIPPED) return state;
    }
    stage_lists<WPI>(P, sl);
    cp_wait_warp();
    stage_rows(P, sl, P.P);
    cp_wait_warp();
    stage_patterns<MaskT>(P, sl);
    return state;
}

// Stage-all mode: this warp's item of every colour (one item per colour at
// most), slice c for colour c, staged at generation start from O (equal to
// P then) and overlapping the copies of all of them.  The decoded headers and
// the lists (first level) stay valid for the whole launch and are copied on
// its first generation only (`lists`); the rows, pattern tables and donor
// starts are made every generation.
template <int WPI, typename MaskT>
__device__ void stage_all_items(const GomParams &P, int gwarp, uint32_t *slices, uint32_t g, bool lists)
{
    const int lane = threadIdx.x & 31;
    const int k = P.k;
    if (lists) {
        const int nwg = (P.Wv + WPI - 1) / WPI;
        const int per = P.split ? nwg : 1;
        __syncwarp();
        for (int c = lane; c < k; c += 32) { // lane c decodes colour c
            int *h = reinterpret_cast<int *>(slices + c * P.warp_smem);
            const int q0 = P.cptr[c], ne = P.cptr[c + 1] - q0;
            const bool valid = gwarp < ne * per;
            h[H_VALID] = valid;
            if (valid) write_item_header(P, q0 + gwarp / per, gwarp % per, h);
        }
        __syncwarp();
        for (int c = 0; c < k; ++c) {
            uint32_t *sl = slices + c * P.warp_smem;
            if (sl[0]) stage_lists<WPI>(P, sl);
        }
        cp_wait_warp();
    }
    for (int c = 0; c < k; ++c) {
        uint32_t *sl = slices + c * P.warp_smem;
        if (sl[0]) stage_rows(P, sl, P.O);
    }
    for (int c = 0; c < k; ++c) { // while the rows are in flight
        uint32_t *sl = slices + c * P.warp_smem;
        if (sl[0]) stage_draws<WPI>(P, sl, g);
    }
    cp_wait_warp();
    for (int c = 0; c < k; ++c) {
        uint32_t *sl = slices + c * P.warp_smem;
        if (sl[0]) stage_patterns<MaskT>(P, sl);
    }
}

// Learned filter bookkeeping after an item ran: the element's accepted,
// donor-less and improving trials into this generation's history, and for
// sampled elements a training sample (the features as at the decision,
// label: the item was useful, see GomFilter::label).  Returns the item's counter increments
// (bits: run, useful, audited, audited and useful) for the caller to sum.
__device__ __forceinline__ unsigned item_record(const GomParams &P, const int *h, uint32_t g, unsigned acc, unsigned dl,
                                            unsigned imp)
{
    const int lane = threadIdx.x & 31;
    acc = __reduce_add_sync(kFull, acc);
    dl = __reduce_add_sync(kFull, dl);
    imp = __reduce_add_sync(kFull, imp);
    const int q = h[H_Q];
    const bool audited = h[H_VALID] == IT_AUDIT, first = h[H_SUB] == 0;
    if (lane == 0) {
        uint32_t *cur = P.flt.hist + (size_t)(g & 1) * 3 * (size_t)P.m;
        if (acc) atomicAdd(&cur[q], acc);
        if (dl) atomicAdd(&cur[P.m + q], dl);
        if (imp) atomicAdd(&cur[2 * (size_t)P.m + q], imp);
    }
    const bool useful = P.flt.label ? imp != 0 : acc != 0;
    if (first && filter_sample(q, g)) {
        float x[kFilterIn];
        filter_features(P, q, g, x);
        filter_log_sample(P, x, useful);
    }
    // the item's counter increments: run, useful, audited, audited and useful
    return 1u | (useful ? 2u : 0u) | (audited ? 4u : 0u) | (audited && useful ? 8u : 0u);
}

// All trials of a staged item (Alg. 2 for each individual of its words):
//  loads:   every global load of a word group is issued together: the
//           parent's rows on F_j, its outside neighbours' words and the
//           elitist flags
//  draws:   the staged donor starts (pre), or one Philox call per lane: lane
//           c holds the call of individuals 4c..4c+3 of the word group,
//           fetched by shuffles
//  donor:   find_donor over patP and its run starts; flips = patP[d] ^ parent
//  delta:   per variable a of F_j, the weighted count S of its outside
//           neighbours set in the parent gives the cut change of its outside
//           edges if a flips (x_a ? 2S - W_a : W_a - 2S); edges inside F_j are
//           evaluated directly, once each (Sec. 2.2, Alg. 4)
//  accept:  delta > 0, or delta == 0 and P[i] is not the elitist (Alg. 2)
//  write:   one ballot per (variable, word) when anything was accepted; lane a
//           XORs the accepted flips into row F_j[a]
// Fitness deltas go to the block's shared accumulators s_f; counters to
// per-lane counts.
// In block mode the caller names the one word group to run (wg_only) and
// gives the warp's own region for the outside neighbours' words (xw_own).
template <int WPI, typename MaskT, typename AccT, bool LEARN>
__device__ __forceinline__ unsigned run_item(const GomParams &P, uint32_t *sl, uint32_t g, bool pre, long long *s_f,
                                         unsigned &n_dl, unsigned &n_acc, unsigned &n_imp, int wg_only = -1,
                                         uint32_t *xw_own = nullptr)
{
    constexpr int NQ = sizeof(MaskT) / 4; // 32-variable quarters of a mask: 1, 2 or 4
    const int lane = threadIdx.x & 31;
    const int W = P.W, Wv = P.Wv, p = P.p;
    const int *h = reinterpret_cast<const int *>(sl);
    const int j = h[H_J], s = h[H_SN] & 0xFF, n_in = h[H_SN] >> 8, n_out = h[H_NOUT], sub = h[H_SUB];
    const int nwg = (Wv + WPI - 1) / WPI;
    const int wg0 = wg_only >= 0 ? wg_only : P.split ? sub : 0;
    const int wg1 = wg_only >= 0 ? wg_only + 1 : P.split ? sub + 1 : nwg;
    const int *fv = reinterpret_cast<const int *>(sl + P.off_fv);
    const uint32_t *sseg = sl + P.off_seg;
    const int64_t *swout = reinterpret_cast<const int64_t *>(sl + P.off_wout);
    const uint32_t *sP = sl + P.off_pr;
    const MaskT *patP = reinterpret_cast<const MaskT *>(sl + P.off_pat);
    const uint32_t *rs = sl + P.off_rs;
    const int *sds = reinterpret_cast<const int *>(sl + P.off_ds);
    const int2 *cw = reinterpret_cast<const int2 *>(sl + P.off_cw);
    uint32_t *xw = xw_own ? xw_own : sl + P.off_xw;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const int ne_tot = n_out + n_in;
    const unsigned acc0 = n_acc, dl0 = n_dl, imp0 = n_imp; // this item's counts, for the learned filter
    int fl[NQ]; // lane l: variables l, l + 32, ... of F_j
#pragma unroll
    for (int q = 0; q < NQ; ++q) fl[q] = lane + 32 * q < s ? fv[lane + 32 * q] : 0;

    for (int wg = wg0; wg < wg1; ++wg) {
        const int w0 = wg * WPI;
        // global loads: the parent's rows on F_j (lane a loads row F_j[a]),
        // the elitist flags, the outside neighbours' words (to shared memory)
        uint32_t Xa[NQ][WPI], eqv[WPI];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
#pragma unroll
            for (int r = 0; r < WPI; ++r) Xa[q][r] = 0;
            if (lane + 32 * q < s) load_words<WPI>(P.O + fl[q] * W + w0, Xa[q]);
        }
        load_words<WPI>(P.eqw + (g & 1) * W + w0, eqv);
        __syncwarp();
        for (int x = lane; x < n_out; x += 32) {
            uint32_t X[WPI];
            load_words<WPI>(P.O + cw[x].x * W + w0, X);
            store_words<WPI>(xw + x * WPI, X);
        }
        // parent bits on F_j: a shuffle transpose of the rows
        MaskT xf[WPI];
#pragma unroll
        for (int r = 0; r < WPI; ++r) xf[r] = 0;
        for (int a = 0; a < s; ++a) {
#pragma unroll
            for (int r = 0; r < WPI; ++r)
                xf[r] |= (MaskT)((lane_get<NQ, WPI>(Xa, r, a) >> lane) & 1u) << a;
        }
        __syncwarp();

        // donor start positions, then the donors
        int dstart[WPI];
        if (pre) {
#pragma unroll
            for (int r = 0; r < WPI; ++r) dstart[r] = sds[(wg - wg0) * 32 * WPI + 32 * r + lane];
        } else {
            // Philox call (j, 8 w0 + lane) covers individuals 32 w0 + 4 lane .. + 3
            const uint4 r4 = philox10(make_uint4((uint32_t)j, (uint32_t)(8 * w0 + lane), g, kTagDonor), k0, k1);
#pragma unroll
            for (int r = 0; r < WPI; ++r) {
                const int src = 8 * r + (lane >> 2);
                const uint32_t x = __shfl_sync(kFull, r4.x, src), y = __shfl_sync(kFull, r4.y, src);
                const uint32_t z = __shfl_sync(kFull, r4.z, src), w = __shfl_sync(kFull, r4.w, src);
                const int cc = lane & 3;
                const uint32_t draw = cc == 0 ? x : cc == 1 ? y : cc == 2 ? z : w;
                const int i = 32 * (w0 + r) + lane;
                int ds = i + 1 + (int)__umulhi(draw, (uint32_t)(p - 1));
                dstart[r] = ds >= p ? ds - p : ds;
            }
        }
        int donor[WPI];
        MaskT fm[WPI];
#pragma unroll
        for (int r = 0; r < WPI; ++r) {
            const int i = 32 * (w0 + r) + lane;
            donor[r] = -1;
            fm[r] = 0;
            if (i < p) {
                const int d = find_donor<MaskT>(patP, rs, sP, W, Wv, p, s, xf[r], dstart[r], i);
                if (d >= 0) {
                    donor[r] = d;
                    fm[r] = patP[d] ^ xf[r];
                }
            }
        }

        // partial evaluation
        AccT dl[WPI];
#pragma unroll
        for (int r = 0; r < WPI; ++r) dl[r] = 0;
        for (int a = 0; a < s; ++a) {
            const int qb = (int)sseg[a], qe = (int)sseg[a + 1];
            const AccT Wa = (AccT)swout[a];
            AccT S[WPI];
#pragma unroll
            for (int r = 0; r < WPI; ++r) S[r] = 0;
            for (int x = qb; x < qe; ++x) {
                uint32_t X[WPI];
                load_words<WPI>(xw + x * WPI, X);
                const AccT wx = (AccT)cw[x].y;
#pragma unroll
                for (int r = 0; r < WPI; ++r) S[r] += wx * (AccT)((X[r] >> lane) & 1u);
            }
#pragma unroll
            for (int r = 0; r < WPI; ++r) {
                const AccT gain = Wa - 2 * S[r];                      // if x_a = 0
                const AccT sx = -(AccT)((xf[r] >> a) & 1u);          // 0 or -1
                const AccT sf = -(AccT)((fm[r] >> a) & 1u);
                dl[r] += ((gain ^ sx) - sx) & sf;
            }
        }
        for (int x = n_out; x < ne_tot; ++x) {
            const int2 e = cw[x];
            const uint32_t code = (uint32_t)e.x;
            const AccT wx = (AccT)e.y;
            const int a = code & 0xFF, b = code >> 8;
#pragma unroll
            for (int r = 0; r < WPI; ++r) {
                const AccT tg = (AccT)(((fm[r] >> a) ^ (fm[r] >> b)) & 1u); // edge toggles
                const AccT sc = -(AccT)(((xf[r] >> a) ^ (xf[r] >> b)) & 1u); // cut before
                dl[r] += ((wx ^ sc) - sc) & -tg;
            }
        }

        // accept, fitness, write
        MaskT afm[WPI]; // accepted flips
        bool anyacc = false;
#pragma unroll
        for (int r = 0; r < WPI; ++r) {
            const int i = 32 * (w0 + r) + lane;
            const bool eq = (eqv[r] >> lane) & 1u;
            const bool acc = donor[r] >= 0 && (dl[r] > 0 || (dl[r] == 0 && !eq));
            afm[r] = acc ? fm[r] : (MaskT)0;
            anyacc |= acc;
            if (acc) {
                atomicAdd((unsigned long long *)&s_f[i], (unsigned long long)(long long)dl[r]);
                ++n_acc;
                if (dl[r] > 0) ++n_imp;
            }
            if (i < p && donor[r] < 0) ++n_dl;
        }
        if (P.fi.on) { // Forced Improvement: the individuals with an accepted step in the generation
#pragma unroll
            for (int r = 0; r < WPI; ++r) {
                const uint32_t mk = __ballot_sync(kFull, afm[r] != (MaskT)0);
                if (lane == 0 && mk) atomicOr(&P.fi.accw[w0 + r], mk);
            }
        }
        if (__any_sync(kFull, anyacc)) {
            uint32_t mine[NQ][WPI]; // lane l: accepted flips of variables l, l + 32, ...
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
#pragma unroll
                for (int r = 0; r < WPI; ++r) mine[q][r] = 0;
            }
            for (int a = 0; a < s; ++a) {
#pragma unroll
                for (int r = 0; r < WPI; ++r) {
                    const uint32_t mk = __ballot_sync(kFull, (unsigned)((afm[r] >> a) & 1u));
#pragma unroll
                    for (int q = 0; q < NQ; ++q) mine[q][r] = lane + 32 * q == a ? mk : mine[q][r];
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (lane + 32 * q < s) {
                    uint32_t *row = P.O + fl[q] * W + w0;
#pragma unroll
                    for (int r = 0; r < WPI; ++r)
                        if (mine[q][r]) row[r] ^= mine[q][r];
                }
            }
        }
    }
    unsigned flags = 0;
    if (LEARN && P.learn) flags = item_record(P, h, g, n_acc - acc0, n_dl - dl0, n_imp - imp0);
    __syncwarp();
    return flags;
}


// One colour group: all (individual, element) GOM trials (Alg. 2) of the
// group at position t, colour c.  Items (an element, or an element's word
// group when P.split is set) go to warps: warp w takes item w first (it may
// already be staged in its slice: `first_staged`), then items w + nwarps,
// w + 2 nwarps, ... (static stride), or, with P.dyn, items nwarps + x for
// the claims x it draws from the counter work[t] -- each claim issued one
// item ahead, so its latency hides behind the item being run.  In stage-all
// mode (`single`) the staged item, with its precomputed donor starts, is the
// warp's only item of the group.  Elements of one group share no variable and no edge (LMIG
// colouring), so a warp owns its element's rows for its words and nothing
// else in the group touches the closure it reads.  MaskT holds one bit per
// variable of F_j (uint32_t: s <= 32, uint64_t: s <= 64); AccT is the delta
// type (int32_t when every element's sum of |w| is < 2^30).  Counters
// accumulate per lane.
template <int WPI, typename MaskT, typename AccT, bool LEARN>
__device__ __forceinline__ void phase_mix(const GomParams &P, const VGrid &V, int t, int c, uint32_t g, uint32_t *sl,
                                          bool first_staged, bool single, long long *s_f, unsigned &n_dl,
                                          unsigned &n_acc, unsigned &n_imp)
{
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)(V.thread() >> 5), nwarps = (int)(V.threads() >> 5);
    int state = first_staged ? (int)sl[H_VALID] : stage_item<WPI, MaskT, LEARN>(P, c, gwarp, sl, g);
    if (state == IT_NONE) return;
    // one call site of run_item and of stage_item (the loop body is the hot code)
    const bool dyn = P.dyn && !single;
    unsigned claim = 0;
    unsigned fc[FC_N] = {}; // learned filter: this warp's counters of the group
    if (dyn && lane == 0) claim = atomicAdd(&P.work[t], 1u);
    for (int next = gwarp + nwarps;; next += nwarps) {
        if (state != IT_SKIPPED) {
            const unsigned f = run_item<WPI, MaskT, AccT, LEARN>(P, sl, g, single, s_f, n_dl, n_acc, n_imp);
            if (LEARN) {
                fc[FC_RUN] += f & 1u;
                fc[FC_RUN_USEFUL] += (f >> 1) & 1u;
                fc[FC_AUDITED] += (f >> 2) & 1u;
                fc[FC_AUDITED_USEFUL] += (f >> 3) & 1u;
            }
        } // a skipped element was counted by the select phase
        // stage-all mode: the staged item is the warp's only one, its slice stays as it is
        if (single) break;
        // stop on the first item past the group (items are numbered densely)
        const int it = dyn ? nwarps + (int)__shfl_sync(kFull, claim, 0) : next;
        state = stage_item<WPI, MaskT, LEARN>(P, c, it, sl, g);
        if (state == IT_NONE) break;
        if (dyn && lane == 0) claim = atomicAdd(&P.work[t], 1u);
    }
    if (LEARN && P.learn && lane == 0) {
        for (int x = 0; x < FC_N; ++x)
            if (fc[x]) atomicAdd(&P.flt.st->cnt[x], (unsigned long long)fc[x]);
    }
}

// Block mode (only in the 128-bit instances, for elements with 4 or more
// word groups): the warps of a block stage one element together into the
// block's one slice and share its word groups, so an element's rows and
// pattern table are made once, not once per (element, word group) item.
// Staging: the header and lists by warp 0, then P's rows, the pattern table
// and its run starts split over the warps.  Called by every thread of the
// block with the same `it`; it first waits until every warp has left the
// slice's previous contents.  Returns the item's validity (block-uniform).
template <typename MaskT>
__device__ bool stage_item_block(const GomParams &P, int c, int it, uint32_t *sl)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    __syncthreads(); // every thread has read the previous header and runs no item any more
    if (wib == 0 && decode_item(P, c, it, 1, sl)) { // P.split is 0: items are elements
        __syncwarp();
        stage_lists<1>(P, sl);
        cp_wait_warp();
    }
    __syncthreads();
    const int *h = reinterpret_cast<const int *>(sl);
    if (!h[H_VALID]) return false;
    const int s = h[H_SN] & 0xFF, W = P.W, Wv = P.Wv, p = P.p;
    const int *fv = reinterpret_cast<const int *>(sl + P.off_fv);
    uint32_t *sP = sl + P.off_pr;
    if (W >= 4) {
        const int n4 = (s * W) >> 2, lw4 = __ffs(W >> 2) - 1;
        for (int x = threadIdx.x; x < n4; x += blockDim.x)
            cp_async16(sP + 4 * x, P.P + fv[x >> lw4] * W + 4 * (x & ((W >> 2) - 1)));
    } else {
        const int lw = __ffs(W) - 1;
        for (int x = threadIdx.x; x < (s << lw); x += blockDim.x) cp_async4(sP + x, P.P + fv[x >> lw] * W + (x & (W - 1)));
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    MaskT *patP = reinterpret_cast<MaskT *>(sl + P.off_pat);
    uint32_t *rs = sl + P.off_rs;
    for (int wc = wib; wc < Wv; wc += nwb) { // warp wib: the patterns of words wib, wib + nwb, ...
        MaskT pat = 0;
        for (int a = 0; a < s; ++a) pat |= (MaskT)((sP[a * W + wc] >> lane) & 1u) << a;
        patP[32 * wc + lane] = pat;
    }
    __syncthreads();
    for (int wc = wib; wc < Wv; wc += nwb) {
        const int d = 32 * wc + lane;
        const bool start = d < p && patP[d] != patP[d == 0 ? p - 1 : d - 1];
        const uint32_t b = __ballot_sync(kFull, start);
        if (lane == 0) rs[wc] = b;
    }
    __syncthreads();
    return true;
}

// One colour group in block mode: block b of the (virtual) grid takes
// element b first (already staged when `first_staged`), then elements
// nblk + x for the claims x it draws from work[t] (P.dyn) or b + nblk,
// b + 2 nblk, ...; warp w runs word groups w, w + nwarps, ... of each, with
// its own region for the outside neighbours' words.
template <int WPI, typename MaskT, typename AccT>
__device__ void phase_mix_block(const GomParams &P, const VGrid &V, int t, int c, uint32_t g, uint32_t *sl,
                                bool first_staged, long long *s_f, unsigned &n_dl, unsigned &n_acc, unsigned &n_imp)
{
    __shared__ int s_next[1];
    const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int nwg = (P.Wv + WPI - 1) / WPI;
    uint32_t *xw = sl + P.off_xw + wib * P.xw_words;
    bool valid = first_staged ? sl[H_VALID] != 0 : stage_item_block<MaskT>(P, c, V.blk, sl);
    for (int next = V.blk + V.nblk; valid; next += V.nblk) {
        if (threadIdx.x == 0) s_next[0] = P.dyn ? V.nblk + (int)atomicAdd(&P.work[t], 1u) : next;
        for (int wg = wib; wg < nwg; wg += nwb)
            run_item<WPI, MaskT, AccT, false>(P, sl, g, false, s_f, n_dl, n_acc, n_imp, wg, xw);
        __syncthreads(); // the claim is visible (thread 0 writes the next one only after the staging's barriers)
        const int it = s_next[0];
        valid = stage_item_block<MaskT>(P, c, it, sl);
    }
}

// Shared-memory words of one warp's staging: k slices in stage-all mode, else one.
__device__ __forceinline__ int warp_words(const GomParams &P, bool all)
{
    return all ? P.k * P.warp_smem : P.warp_smem;
}


// ----------------------------------------------------------------------------
// Kernels of the per-launch path (one CUDA graph per generation).

__global__ void k_gen_start(GomParams P)
{
    if (P.st->done) return;
    phase_gen_start(P, whole_grid(), P.st->improved, P.st->argmax, P.st->g, true);
}

__global__ void k_order(GomParams P)
{
    extern __shared__ unsigned long long s_key[];
    if (P.st->done) return;
    phase_order(P, whole_grid(), s_key, P.st->g);
}

template <int WPI, typename MaskT, typename AccT, bool LEARN>
__global__ void __launch_bounds__(kMixThreads, 3) k_mix(GomParams P, int t)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    __shared__ long long s_f[1024];
    __shared__ unsigned long long s_cnt[4];
    if (P.st->done) return;
    acc_zero(P, s_f, s_cnt);
    unsigned n_dl = 0, n_acc = 0, n_imp = 0;
    if (sizeof(MaskT) == 16 && P.blk)
        phase_mix_block<WPI, MaskT, AccT>(P, whole_grid(), t, P.order[t], P.st->g, s_dyn, false, s_f, n_dl, n_acc,
                                          n_imp);
    else
        phase_mix<WPI, MaskT, AccT, LEARN>(P, whole_grid(), t, P.order[t], P.st->g,
                                    s_dyn + (threadIdx.x >> 5) * warp_words(P, false), false, false, s_f, n_dl, n_acc,
                                    n_imp);
    count_flush(s_cnt, n_dl, n_acc, n_imp);
    acc_flush(P, s_f, s_cnt);
}

// The learned filter's select phase on the per-generation graph path: the
// decisions (with `compact`, each warp's count of elements to run), the scan
// of the counts (one block) and the compacted list, each a node of its own,
// launched on the same grid for the first and the last.
__global__ void __launch_bounds__(256) k_filter_select(GomParams P, int compact)
{
    if (P.st->done) return;
    filter_select_decide(P, whole_grid(), P.st->g, compact != 0);
}

__global__ void __launch_bounds__(1024) k_filter_scan(GomParams P, int nwarps)
{
    if (P.st->done) return;
    filter_select_scan(P, nwarps);
}

__global__ void __launch_bounds__(256) k_filter_compact(GomParams P)
{
    if (P.st->done) return;
    filter_select_compact(P, whole_grid());
}

__global__ void __launch_bounds__(1024) k_gen_end(GomParams P)
{
    if (P.st->done) return;
    GenEnd e{P.st->fe, 0, P.st->argmax};
    phase_gen_end(P, P.st->target, P.st->g, e, true);
}

// Persistent path: up to G generations in one cooperative launch, the phases
// separated by grid barriers: [generation start + group order] | group 0 |
// ... | group k-1 | and again.  A generation's end is computed by every block
// from the fitness array right after the barrier that closes its last group
// (the same values everywhere; block 0 records them), so it needs no phase
// of its own, and every block takes the same stop decision.
// Staging: in stage-all mode every block computes the whole group order and
// every warp stages its item of every colour from O before the barrier that
// opens the generation (P itself is then never read, so it is not copied);
// otherwise every warp stages its first item of group t before the barrier
// that opens the group.  The block's fitness accumulators and the warps'
// counters span all groups of a generation and are flushed once, before the
// closing barrier.  V is the set of blocks that run this problem (the whole
// grid, or one instance's blocks in a batched launch); `bar` is their
// barrier counter.
struct RunShared {
    uint32_t *dyn;              // staging slices (and the group keys outside stage-all mode)
    long long *f;               // [32 W] the block's fitness accumulators
    unsigned long long *cnt;    // [4] the block's counters
    unsigned long long *okey;   // [kStageAllMaxK] stage-all group keys
    int *order;                 // [kStageAllMaxK] stage-all group order
};

template <int WPI, typename MaskT, typename AccT, bool LEARN>
__device__ void run_generations(const GomParams &P, const VGrid V, GomBarrier *bar, int G, int64_t target,
                                const RunShared &S)
{
    const unsigned nblk = (unsigned)V.nblk;
    const int gwarp = (int)(V.thread() >> 5);
    const bool all = P.stage_all != 0;
    const bool lead = V.blk == 0;
    // block mode: one slice for the whole block (the 128-bit instances only)
    const bool blkm = sizeof(MaskT) == 16 && P.blk;
    // this warp's staging: one slice, or one per colour with stage_all
    uint32_t *slices = S.dyn + (blkm ? 0 : (threadIdx.x >> 5) * warp_words(P, all));
    uint32_t g = P.st->g;
    GenEnd e{P.st->fe, P.st->improved, P.st->argmax};
    unsigned long long bnext = 0; // next barrier epoch end (thread 0)
    if (threadIdx.x == 0) bnext = barrier_first(&bar->count, nblk);
    if (lead && threadIdx.x == 0) {
        P.st->call_g0 = g; // read by the host after the kernel only
        P.st->target = target;
    }
    // optional phase trace (block 0, thread 0): wall-clock stamps of the last
    // generation of the call, see gom_read_phase_trace
    const bool tr = P.trace != nullptr && lead && threadIdx.x == 0;
    for (int q = 0; q < G; ++q) {
        if (q > 0 && phase_gen_end(P, target, g - 1, e, lead)) return;
        if (tr) P.trace[0] = global_ns();
        phase_gen_start(P, V, e.improved, e.argmax, g, !all);
        if (all)
            phase_order_block(P, S.okey, S.order, g);
        else
            phase_order(P, V, reinterpret_cast<unsigned long long *>(S.dyn), g);
        acc_zero(P, S.f, S.cnt);
        if (tr) P.trace[1] = global_ns();
        if (all) stage_all_items<WPI, MaskT>(P, gwarp, slices, g, q == 0);
        if (tr) P.trace[2] = global_ns();
        if (!grid_barrier(&bar->count, &P.st->err, nblk, bnext, kBarrierNs)) return;
        // the learned filter's decisions, before the first item is staged
        if (LEARN && P.learn && !phase_filter_select(P, V, g, &bar->count, nblk, bnext, false)) return;
        if (tr) P.trace[3] = global_ns();
        unsigned n_dl = 0, n_acc = 0, n_imp = 0;
        for (int t = 0; t < P.k; ++t) {
            const int c = all ? S.order[t] : P.order[t];
            uint32_t *sl = all ? slices + c * P.warp_smem : slices;
            // without stage_all: stage the first item of group t before its barrier
            if (blkm)
                stage_item_block<MaskT>(P, c, V.blk, sl);
            else if (!all)
                stage_item<WPI, MaskT, LEARN>(P, c, gwarp, sl, g);
            if (t > 0 && !grid_barrier(&bar->count, &P.st->err, nblk, bnext, kBarrierNs)) return;
            if (tr) P.trace[4 + 2 * t] = global_ns();
            if (blkm)
                phase_mix_block<WPI, MaskT, AccT>(P, V, t, c, g, sl, true, S.f, n_dl, n_acc, n_imp);
            else
                phase_mix<WPI, MaskT, AccT, LEARN>(P, V, t, c, g, sl, true, all, S.f, n_dl, n_acc, n_imp);
            if (tr) P.trace[5 + 2 * t] = global_ns();
        }
        count_flush(S.cnt, n_dl, n_acc, n_imp);
        acc_flush(P, S.f, S.cnt);
        if (!grid_barrier(&bar->count, &P.st->err, nblk, bnext, kBarrierNs)) return;
        if (P.fi.on && !fi_generation<16>(P, V, &bar->count, nblk, bnext, e, all ? S.order : P.order, S.f, S.cnt))
            return;
        if (tr) P.trace[4 + 2 * P.k] = global_ns();
        ++g;
    }
    if (G > 0 && lead) phase_gen_end(P, target, g - 1, e, true);
}

template <int WPI, typename MaskT, typename AccT, bool LEARN>
__global__ void __launch_bounds__(kMixThreads, 3) k_run(GomParams P, int G, int64_t target)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    __shared__ long long s_f[1024];
    __shared__ unsigned long long s_cnt[4];
    __shared__ unsigned long long s_okey[kStageAllMaxK];
    __shared__ int s_order[kStageAllMaxK];
    const RunShared S{s_dyn, s_f, s_cnt, s_okey, s_order};
    run_generations<WPI, MaskT, AccT, LEARN>(P, whole_grid(), P.bar, G, target, S);
}

// One kernel variant of the batched path, compiled as its own function so
// that each variant gets its own register allocation.
template <int WPI, typename MaskT, typename AccT>
__device__ __noinline__ void batch_variant(const GomParams &P, const VGrid V, GomBarrier *bar, int G, int64_t target,
                                           const RunShared &S)
{
    run_generations<WPI, MaskT, AccT, false>(P, V, bar, G, target, S);
}

// The bit-sliced variant of the batched path: the instance's generations on
// the bit-sliced phase (gom_bs.cuh), warp w of the block in the w-th region
// of P.bs_words words after the fitness accumulators.
template <int R>
__device__ __noinline__ void batch_variant_bs(const GomParams &P, const VGrid V, GomBarrier *bar, int G,
                                              int64_t target, const RunShared &S)
{
    bs_generations<R, false>(P, V, bar, G, target, reinterpret_cast<unsigned long long *>(S.dyn),
                             S.dyn + (threadIdx.x >> 5) * P.bs_words, S.f, S.cnt, nullptr);
}

// Batched path: many independent instances in one cooperative launch.  Each
// instance owns a range of blocks and runs its own generations on them, with
// its own barrier counter and its own stop decision, exactly as its
// persistent kernel would; instances never wait for one another.  Ps[b] is
// instance b's parameter block (one-slice staging), inst[b] its blocks,
// kernel variant, target and generation count (at most G).  The dynamic shared memory holds the block's
// fitness accumulators (f_words 32-bit words, 32 W of the widest instance)
// and then the warps' staging slices.
// MINB: resident blocks of 256 threads the register budget is cut for (2: no
// spills, 3: more warps per SM).
template <int MINB>
__global__ void __launch_bounds__(kMixThreads, MINB)
    k_batch(const GomParams *Ps, const GomBatchInst *inst, GomBarrier *bars, int B, int G, int f_words)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    __shared__ GomParams sP;
    __shared__ unsigned long long s_cnt[4];
    __shared__ int s_b;
    if (threadIdx.x == 0) {
        // the instance of this block: the last b with blk0 <= blockIdx.x
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst[mid].blk0 <= (int)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_b = lo;
        sP = Ps[lo];
    }
    __syncthreads();
    const int b = s_b;
    const GomBatchInst I = inst[b];
    if ((int)blockIdx.x >= I.blk0 + I.nblk) return; // a block past every range (none by construction)
    const VGrid V{(int)blockIdx.x - I.blk0, I.nblk};
    const RunShared S{s_dyn + f_words, reinterpret_cast<long long *>(s_dyn), s_cnt, nullptr, nullptr};
    GomBarrier *bar = bars + b;
    G = min(G, I.gens);
    if (MINB == 2 && I.variant == kVarBits) { // the bit-sliced phase needs the larger register budget
        if constexpr (MINB == 2) {
            if (I.bs_r <= 12)
                batch_variant_bs<12>(sP, V, bar, G, I.target, S);
            else
                batch_variant_bs<16>(sP, V, bar, G, I.target, S);
        }
    } else if (I.variant == kVarNarrow || I.variant == kVarBits) {
        if (I.wpi == 4)
            batch_variant<4, uint32_t, int32_t>(sP, V, bar, G, I.target, S);
        else if (I.wpi == 2)
            batch_variant<2, uint32_t, int32_t>(sP, V, bar, G, I.target, S);
        else
            batch_variant<1, uint32_t, int32_t>(sP, V, bar, G, I.target, S);
    } else if (I.variant == kVarHuge) {
        if (I.wpi == 2)
            batch_variant<2, Mask128, long long>(sP, V, bar, G, I.target, S);
        else
            batch_variant<1, Mask128, long long>(sP, V, bar, G, I.target, S);
    } else {
        if (I.wpi == 4)
            batch_variant<4, uint64_t, long long>(sP, V, bar, G, I.target, S);
        else if (I.wpi == 2)
            batch_variant<2, uint64_t, long long>(sP, V, bar, G, I.target, S);
        else
            batch_variant<1, uint64_t, long long>(sP, V, bar, G, I.target, S);
    }
}

const void *gom_batch_kernel(int minb)
{
    return minb >= 3 ? (const void *)k_batch<3> : (const void *)k_batch<2>;
}

// After a batched call: each instance's generation count and error word.
__global__ void k_batch_collect(const GomParams *Ps, GomBatchInst *inst, int B)
{
    for (int b = (int)gthread(); b < B; b += (int)gthreads()) {
        const GomDevState *st = Ps[b].st;
        inst[b].gens_run = (int32_t)(st->g - st->call_g0);
        inst[b].err = st->err;
    }
}

// Self-test of the grid barrier's bounded wait: `blocks` co-resident blocks
// meet at a barrier that expects `blocks + extra` arrivals; with extra > 0 no
// block is ever released and every block must give up after limit_ns.
__global__ void k_barrier_selftest(GomBarrier *bar, int *err, int extra, unsigned long long limit_ns)
{
    const unsigned expected = gridDim.x + (unsigned)extra;
    unsigned long long next = 0;
    if (threadIdx.x == 0) next = barrier_first(&bar->count, expected);
    grid_barrier(&bar->count, err, expected, next, limit_ns);
}

template <bool LEARN>
const void *mix_kernel(int wpi, int variant)
{
    if (variant == kVarNarrow)
        return wpi == 4 ? (const void *)k_mix<4, uint32_t, int32_t, LEARN>
             : wpi == 2 ? (const void *)k_mix<2, uint32_t, int32_t, LEARN>
                        : (const void *)k_mix<1, uint32_t, int32_t, LEARN>;
    if (variant == kVarHuge) // no filter instances, at most two words per item
        return LEARN || wpi > 2 ? nullptr
             : wpi == 2         ? (const void *)k_mix<2, Mask128, long long, false>
                                : (const void *)k_mix<1, Mask128, long long, false>;
    return wpi == 4 ? (const void *)k_mix<4, uint64_t, long long, LEARN>
         : wpi == 2 ? (const void *)k_mix<2, uint64_t, long long, LEARN>
                    : (const void *)k_mix<1, uint64_t, long long, LEARN>;
}

template <bool LEARN>
const void *run_kernel(int wpi, int variant)
{
    if (variant == kVarNarrow)
        return wpi == 4 ? (const void *)k_run<4, uint32_t, int32_t, LEARN>
             : wpi == 2 ? (const void *)k_run<2, uint32_t, int32_t, LEARN>
                        : (const void *)k_run<1, uint32_t, int32_t, LEARN>;
    if (variant == kVarHuge)
        return LEARN || wpi > 2 ? nullptr
             : wpi == 2         ? (const void *)k_run<2, Mask128, long long, false>
                                : (const void *)k_run<1, Mask128, long long, false>;
    return wpi == 4 ? (const void *)k_run<4, uint64_t, long long, LEARN>
         : wpi == 2 ? (const void *)k_run<2, uint64_t, long long, LEARN>
                    : (const void *)k_run<1, uint64_t, long long, LEARN>;
}

const void *gom_mix_kernel(int wpi, int variant, bool learn)
{
    return learn ? mix_kernel<true>(wpi, variant) : mix_kernel<false>(wpi, variant);
}

const void *gom_run_kernel(int wpi, int variant, bool learn)
{
    return learn ? run_kernel<true>(wpi, variant) : run_kernel<false>(wpi, variant);
}

// ----------------------------------------------------------------------------
// uint8 rows out[i*n + v] of the population.
__global__ void k_export_pop(GomParams P, uint8_t *out)
{
    const int64_t total = (int64_t)P.p * P.n;
    for (int64_t idx = gthread(); idx < total; idx += gthreads()) {
        const int64_t i = idx / P.n, v = idx - i * P.n;
        out[idx] = (uint8_t)((P.O[v * P.W + (i >> 5)] >> (i & 31)) & 1u);
    }
}

__global__ void k_export_elite(GomParams P, uint8_t *out)
{
    const int improved = P.st->improved;
    const int aw = P.st->argmax >> 5, ab = P.st->argmax & 31;
    for (int64_t v = gthread(); v < P.n; v += gthreads())
        out[v] = improved ? (uint8_t)((P.O[v * P.W + aw] >> ab) & 1u) : P.xe[v];
}

// Packs uint8 rows in[i*n + v] into the bit-sliced O and copies the elitist.
__global__ void k_import_pop(GomParams P, const uint8_t *in, const uint8_t *elite)
{
    const int64_t total = (int64_t)P.n * P.W;
    for (int64_t idx = gthread(); idx < total; idx += gthreads()) {
        const int64_t v = idx / P.W;
        const int w = (int)(idx - v * P.W);
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t i = 32 * w + b;
            if (i < P.p && in[i * P.n + v]) word |= 1u << b;
        }
        P.O[idx] = word;
        if (w == 0) P.xe[v] = elite[v] ? 1 : 0;
    }
}
