// gom_kernels.cu -- sm_103a kernels of parallel GOM for weighted Max-Cut.
//
// Population layout (bit-sliced, variable-major): O[v*W + w] holds variable v
// of individuals 32w .. 32w+31, one bit each.  W is a power of two; words and
// bits past the population size stay zero.  A warp therefore reads one
// variable of 32 individuals with a single broadcast load, and the writes of
// one GOM trial batch (32 individuals x one element) are whole words.
//
// Kernels of one generation (Alg. 3):
//   k_gen_start  Clone (P <- O), copy of the new elitist, elitist flags
//   k_order      random order of the colour groups
//   k_mix        one launch per colour group: every (individual, element)
//                trial of the group -- donor, partial evaluation, accept, write
//   k_gen_end    fitness fold, elitist update, counters, target check
// plus initialisation, full evaluation and import/export kernels.
#include <climits>
#include <cuda_runtime.h>

#include "gom_internal.h"
#include "gom_kernels.cuh"

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

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

__device__ __forceinline__ uint32_t pick(uint4 r, int q)
{
    return (q & 2) ? ((q & 1) ? r.w : r.z) : ((q & 1) ? r.y : r.x);
}

__device__ __forceinline__ int64_t gthread() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gthreads() { return (int64_t)gridDim.x * blockDim.x; }

// Lowest index of the maximum of f[0..p) over one block (blockDim <= 1024).
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
        if (lane == 0) {
            *best_out = best;
            *arg_out = arg;
        }
    }
    __syncthreads();
}

} // namespace

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
    for (int w = threadIdx.x; w < P.W; w += blockDim.x) P.eqw[w] = kFull;
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
        P.st->cnt[0] = P.st->cnt[1] = P.st->cnt[2] = 0;
    }
    for (int w = threadIdx.x; w < P.W; w += blockDim.x) P.eqw[w] = kFull;
}

__global__ void k_begin_call(GomParams P, int64_t target)
{
    P.st->done = 0;
    P.st->target = target;
    P.st->call_g0 = P.st->g; // first generation of this call
}

// Generation start (Alg. 3 Clone): P <- O.  If the elitist changed in the last
// generation, its bits are taken from column `argmax` of O (O has not changed
// since).  eqw[w] bit b ends as 1 iff individual 32w+b equals the elitist on
// every variable (the flag of the acceptance rule, fixed for the generation).
// Thread idx handles word idx = v*W + w; the grid stride is a multiple of W.
__global__ void k_gen_start(GomParams P)
{
    __shared__ uint32_t s_eq[32];
    if (P.st->done) return;
    const int improved = P.st->improved;
    const int aw = P.st->argmax >> 5, ab = P.st->argmax & 31;
    const int W = P.W;
    const int lw = __ffs(W) - 1;
    const int64_t total = (int64_t)P.n * W;
    const int64_t tid = gthread(), nth = gthreads();
    const int w = (int)(tid & (W - 1));
    uint32_t eq = kFull;
    for (int64_t idx = tid; idx < total; idx += nth) {
        const int64_t v = idx >> lw;
        const uint32_t word = P.O[idx];
        P.P[idx] = word;
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
    if (threadIdx.x < W && threadIdx.x < 32) atomicAnd(&P.eqw[threadIdx.x], s_eq[threadIdx.x]);
}

// Group order of generation g (Alg. 3, "random order"): colours sorted by
// their 64-bit Philox key, ties by colour index.  Every block draws all k keys
// into shared memory and ranks blockDim colours.
__global__ void k_order(GomParams P)
{
    extern __shared__ unsigned long long s_key[];
    if (P.st->done) return;
    const uint32_t g = P.st->g;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    for (int c = threadIdx.x; c < P.k; c += blockDim.x) {
        const uint4 r = philox10(make_uint4((uint32_t)c, 0u, g, kTagOrder), k0, k1);
        s_key[c] = ((unsigned long long)r.x << 32) | r.y;
    }
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < P.k) {
        const unsigned long long kc = s_key[c];
        int rank = 0;
        for (int c2 = 0; c2 < P.k; ++c2) {
            const unsigned long long k2 = s_key[c2];
            rank += (k2 < kc) || (k2 == kc && c2 < c);
        }
        P.order[rank] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) P.st->improved = 0; // x_e copied by k_gen_start
}

// Loads WPI consecutive 32-bit words (16/8/4-byte aligned by construction).
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

// First individual, scanning cyclically upwards from `start` and skipping
// `self`, whose generation-start bits on F differ from the parent's bits
// `xf`; 32 candidates per step (one word of each of F's rows of P).  -1 if
// none.  Called from divergent code: no warp collectives.
template <typename MaskT>
__device__ int scan_donor(const GomParams &P, const int32_t *F, int s, MaskT xf, int start, int self)
{
    const int W = P.W, Wv = P.Wv, p = P.p;
    const int ws = start >> 5, bs = start & 31;
    for (int step = 0; step <= Wv; ++step) {
        int wc = ws + step;
        if (wc >= Wv) wc -= Wv;
        uint32_t diff = 0;
        for (int a = 0; a < s; ++a)
            diff |= P.P[F[a] * W + wc] ^ (0u - (uint32_t)((xf >> a) & 1u));
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

// One colour group: all (individual, element) GOM trials (Alg. 2) of group
// order[t].  A warp item is (element, WPI consecutive words); lane l works on
// the individuals 32w + l of those words.  Elements of one group share no
// variable and no edge (LMIG colouring), so the warp owns its element's rows
// for its words and nothing else in the group touches the closure it reads.
//  draws:   one Philox call per lane gives 4 words: lane c holds the call
//           of individuals 4c..4c+3 of the item, fetched with shuffles
//  donor:   the start candidate's bits on F_j first; if equal to the
//           parent's, the word-parallel cyclic scan (scan_donor)
//  delta:   per variable a of F_j that flips, the weighted count S of its
//           outside neighbours set in the parent gives the cut change of its
//           outside edges (x_a ? 2S - W_a : W_a - 2S); edges inside F_j are
//           evaluated directly, once each (Sec. 2.2, Alg. 4)
//  accept:  delta > 0, or delta == 0 and P[i] is not the elitist (Alg. 2)
//  write:   one ballot per variable and word; lane 0 XORs the accepted flips
// MaskT holds one bit per variable of F_j (uint32_t or uint64_t); AccT is
// the delta type (int32_t when every element's sum of |w| is < 2^30).
// Fitness deltas and counters are summed per block in shared memory, then
// added with one atomic per individual (and per counter) per block: integer
// adds, so the result does not depend on their order.
template <int WPI, typename MaskT, typename AccT>
__global__ void __launch_bounds__(kMixThreads) k_mix(GomParams P, int t)
{
    __shared__ long long s_f[1024];
    __shared__ unsigned long long s_cnt[4];
    if (P.st->done) return;
    const int lane = threadIdx.x & 31;
    const int W = P.W;
    const int np = 32 * W;
    for (int q = threadIdx.x; q < np; q += blockDim.x) s_f[q] = 0;
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();

    const int c = P.order[t];
    const int q0 = P.cptr[c], ne = P.cptr[c + 1] - q0;
    const int G = W / WPI; // word groups per element; the warp count is a multiple of G
    const int gwarp = (int)(gthread() >> 5), nwarps = (int)(gthreads() >> 5);
    const int w0 = (gwarp % G) * WPI;
    const int p = P.p;
    const uint32_t g = P.st->g;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);

    int iv[WPI];
    bool eqf[WPI];
    long long facc[WPI];
#pragma unroll
    for (int r = 0; r < WPI; ++r) {
        iv[r] = 32 * (w0 + r) + lane;
        eqf[r] = (P.eqw[w0 + r] >> lane) & 1u;
        facc[r] = 0;
    }
    unsigned n_dl = 0, n_acc = 0, n_imp = 0;

    if (w0 < P.Wv) {
        for (int e = gwarp / G; e < ne; e += nwarps / G) {
            const int q = q0 + e;
            const int4 h = P.hdr[q];
            const int j = h.x, f0 = h.y, d0 = h.z;
            const int s = h.w & 0xFF, n_in = h.w >> 8;
            const int32_t *F = P.fv + f0;
            const int fl = lane < s ? F[lane] : 0; // lane a holds F_j[a] (s <= 32 here)

            // parent bits on F_j
            MaskT xf[WPI];
#pragma unroll
            for (int r = 0; r < WPI; ++r) xf[r] = 0;
            for (int a = 0; a < s; ++a) {
                const int fa = s <= 32 ? __shfl_sync(kFull, fl, a) : F[a];
                uint32_t X[WPI];
                load_words<WPI>(P.O + fa * W + w0, X);
#pragma unroll
                for (int r = 0; r < WPI; ++r) xf[r] |= (MaskT)((X[r] >> lane) & 1u) << a;
            }

            // Philox draws: call (j, 8 w0 + lane) covers individuals 32 w0 + 4 lane .. + 3
            const uint4 r4 = philox10(make_uint4((uint32_t)j, (uint32_t)(8 * w0 + lane), g, kTagDonor), k0, k1);
            uint32_t draw[WPI];
#pragma unroll
            for (int r = 0; r < WPI; ++r) {
                const int src = 8 * r + (lane >> 2);
                const uint32_t x = __shfl_sync(kFull, r4.x, src), y = __shfl_sync(kFull, r4.y, src);
                const uint32_t z = __shfl_sync(kFull, r4.z, src), w = __shfl_sync(kFull, r4.w, src);
                const int cc = lane & 3;
                draw[r] = cc == 0 ? x : cc == 1 ? y : cc == 2 ? z : w;
            }

            // donors: start candidate, then the scan
            int donor[WPI];
            MaskT fm[WPI];
#pragma unroll
            for (int r = 0; r < WPI; ++r) {
                const uint32_t u = __umulhi(draw[r], (uint32_t)(p - 1));
                int ds = iv[r] + 1 + (int)u;
                if (ds >= p) ds -= p;
                if (iv[r] >= p) ds = 0;
                const int dw = ds >> 5, db = ds & 31;
                MaskT pat = 0;
                for (int a = 0; a < s; ++a) {
                    const int fa = s <= 32 ? __shfl_sync(kFull, fl, a) : F[a];
                    pat |= (MaskT)((P.P[fa * W + dw] >> db) & 1u) << a;
                }
                donor[r] = -1;
                fm[r] = 0;
                if (iv[r] < p) {
                    if (pat != xf[r]) {
                        donor[r] = ds;
                        fm[r] = pat ^ xf[r];
                    } else {
                        const int d = scan_donor<MaskT>(P, F, s, xf[r], ds, iv[r]);
                        if (d >= 0) {
                            MaskT pd = 0;
                            for (int a = 0; a < s; ++a)
                                pd |= (MaskT)((P.P[F[a] * W + (d >> 5)] >> (d & 31)) & 1u) << a;
                            donor[r] = d;
                            fm[r] = pd ^ xf[r];
                        }
                    }
                }
            }

            // partial evaluation
            AccT dl[WPI];
#pragma unroll
            for (int r = 0; r < WPI; ++r) dl[r] = 0;
            bool any = false;
#pragma unroll
            for (int r = 0; r < WPI; ++r) any |= donor[r] >= 0;
            if (__any_sync(kFull, any)) {
                const uint16_t *seg = P.seg + f0 + q;
                const int2 *dep = P.dep + d0;
                int qb = 0;
                for (int a = 0; a < s; ++a) {
                    const int qe = seg[a + 1];
                    bool flips = false;
#pragma unroll
                    for (int r = 0; r < WPI; ++r) flips |= (fm[r] >> a) & 1u;
                    if (__any_sync(kFull, flips)) {
                        AccT S[WPI];
#pragma unroll
                        for (int r = 0; r < WPI; ++r) S[r] = 0;
                        for (int x = qb; x < qe; ++x) {
                            const int2 d = dep[x];
                            uint32_t X[WPI];
                            load_words<WPI>(P.O + d.x * W + w0, X);
#pragma unroll
                            for (int r = 0; r < WPI; ++r) S[r] += (AccT)d.y * (AccT)((X[r] >> lane) & 1u);
                        }
                        const AccT Wa = (AccT)P.wout[f0 + a];
#pragma unroll
                        for (int r = 0; r < WPI; ++r)
                            if ((fm[r] >> a) & 1u) dl[r] += ((xf[r] >> a) & 1u) ? 2 * S[r] - Wa : Wa - 2 * S[r];
                    }
                    qb = qe;
                }
                for (int x = qb; x < qb + n_in; ++x) {
                    const int2 d = dep[x];
                    const int a = d.x & 0xFF, b = d.x >> 8;
#pragma unroll
                    for (int r = 0; r < WPI; ++r) {
                        const MaskT y = xf[r] ^ fm[r];
                        const int cn = (int)(((y >> a) ^ (y >> b)) & 1u);
                        const int co = (int)(((xf[r] >> a) ^ (xf[r] >> b)) & 1u);
                        dl[r] += (AccT)d.y * (AccT)(cn - co);
                    }
                }
            }

            bool acc[WPI];
#pragma unroll
            for (int r = 0; r < WPI; ++r)
                acc[r] = donor[r] >= 0 && (dl[r] > 0 || (dl[r] == 0 && !eqf[r]));
            for (int a = 0; a < s; ++a) {
                const int fa = s <= 32 ? __shfl_sync(kFull, fl, a) : F[a];
                uint32_t mk[WPI];
                bool anym = false;
#pragma unroll
                for (int r = 0; r < WPI; ++r) {
                    mk[r] = __ballot_sync(kFull, acc[r] && ((fm[r] >> a) & 1u));
                    anym |= mk[r] != 0;
                }
                if (lane == 0 && anym) {
                    uint32_t *row = P.O + fa * W + w0;
#pragma unroll
                    for (int r = 0; r < WPI; ++r)
                        if (mk[r]) row[r] ^= mk[r];
                }
            }
#pragma unroll
            for (int r = 0; r < WPI; ++r) {
                if (acc[r]) {
                    facc[r] += dl[r];
                    ++n_acc;
                    if (dl[r] > 0) ++n_imp;
                }
                if (iv[r] < p && donor[r] < 0) ++n_dl;
            }
        }
    }

#pragma unroll
    for (int r = 0; r < WPI; ++r)
        if (facc[r]) atomicAdd((unsigned long long *)&s_f[iv[r]], (unsigned long long)facc[r]);
    n_dl = __reduce_add_sync(kFull, n_dl);
    n_acc = __reduce_add_sync(kFull, n_acc);
    n_imp = __reduce_add_sync(kFull, n_imp);
    if (lane == 0 && (n_dl | n_acc | n_imp)) {
        atomicAdd(&s_cnt[0], (unsigned long long)n_dl);
        atomicAdd(&s_cnt[1], (unsigned long long)n_acc);
        atomicAdd(&s_cnt[2], (unsigned long long)n_imp);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const long long v = s_f[q];
        if (v) atomicAdd((unsigned long long *)&P.f[q], (unsigned long long)v);
    }
    if (threadIdx.x < 3 && s_cnt[threadIdx.x])
        atomicAdd((unsigned long long *)&P.st->cnt[threadIdx.x], s_cnt[threadIdx.x]);
}

const void *gom_mix_kernel(int wpi, bool narrow)
{
    if (narrow)
        return wpi == 4 ? (const void *)k_mix<4, uint32_t, int32_t>
             : wpi == 2 ? (const void *)k_mix<2, uint32_t, int32_t>
                        : (const void *)k_mix<1, uint32_t, int32_t>;
    return wpi == 4 ? (const void *)k_mix<4, uint64_t, long long>
         : wpi == 2 ? (const void *)k_mix<2, uint64_t, long long>
                    : (const void *)k_mix<1, uint64_t, long long>;
}

// Generation end: elitist update (strict improvement, lowest index; Sec. 4),
// counters, target check, g += 1.
__global__ void __launch_bounds__(1024) k_gen_end(GomParams P)
{
    if (P.st->done) return;
    int64_t best;
    int arg;
    block_argmax(P.f, P.p, &best, &arg);
    if (threadIdx.x == 0) {
        GomDevState *st = P.st;
        if (best > st->fe) {
            st->fe = best;
            st->improved = 1;
            st->argmax = arg;
        }
        st->best = best;
        GomDevStats &S = P.stats[st->g % kStatsCap];
        S.generation = st->g;
        S.best = best;
        S.elite = st->fe;
        S.trials = (int64_t)P.p * P.m;
        S.donorless = st->cnt[0];
        S.accepted = st->cnt[1];
        S.improving = st->cnt[2];
        S.reached = best >= st->target;
        st->cnt[0] = st->cnt[1] = st->cnt[2] = 0;
        st->done = best >= st->target;
        st->g += 1;
    }
    for (int w = threadIdx.x; w < P.W; w += blockDim.x) P.eqw[w] = kFull;
}

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
