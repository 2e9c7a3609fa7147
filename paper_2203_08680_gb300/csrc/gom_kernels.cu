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

// One colour group: all (individual, element) GOM trials (Alg. 2) of group
// order[t].  Warp = (element, word w), lane = individual 32w+lane.  Elements of
// one group share no variable and no edge (LMIG colouring), so each warp owns
// the rows of its element for its word and nothing else of this group touches
// the closure it reads.
//  donor:    Philox start, cyclic scan over 32 candidates per step, comparing
//            P's words on F_j against the parent's bits (word-parallel)
//  delta:    sum over the element's dependency list of the change of each
//            edge's cut contribution (Sec. 2.2; edges inside F_j listed once)
//  accept:   delta > 0, or delta == 0 and P[i] is not the elitist (Alg. 2)
//  write:    one ballot per variable of F_j; lane 0 XORs the accepted flips
// Fitness deltas and counters are summed per block in shared memory, then one
// atomic add per individual (and per counter) per block: integer adds, so the
// result does not depend on their order.
__global__ void __launch_bounds__(kMixThreads) k_mix(GomParams P, int t)
{
    __shared__ long long s_f[1024];
    __shared__ unsigned long long s_cnt[4];
    if (P.st->done) return;
    const int lane = threadIdx.x & 31;
    const int np = 32 * P.W;
    for (int q = threadIdx.x; q < np; q += blockDim.x) s_f[q] = 0;
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();

    const int c = P.order[t];
    const int e0 = P.cptr[c], ne = P.cptr[c + 1] - e0;
    const int W = P.W;
    const int64_t gwarp = gthread() >> 5, nwarps = gthreads() >> 5;
    const int w = (int)(gwarp & (W - 1));
    const int i = 32 * w + lane;
    const bool valid = i < P.p;
    const bool eqflag = (P.eqw[w] >> lane) & 1u;
    const uint32_t g = P.st->g;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const int p = P.p, Wv = P.Wv;
    long long facc = 0;
    unsigned n_dl = 0, n_acc = 0, n_imp = 0;

    if (w < Wv) {
        for (int64_t e = gwarp / W; e < ne; e += nwarps / W) {
            const int j = P.celems[e0 + e];
            const int f0 = P.eptr[j];
            const int s = P.eptr[j + 1] - f0;
            const int32_t *F = P.evars + f0;

            // parent bits on F_j
            uint64_t xf = 0;
            for (int a = 0; a < s; ++a) {
                const uint32_t word = P.O[(int64_t)F[a] * W + w];
                xf |= (uint64_t)((word >> lane) & 1u) << a;
            }

            // SelectDonorFromPopulation
            const uint4 r4 = philox10(make_uint4((uint32_t)j, (uint32_t)i >> 2, g, kTagDonor), k0, k1);
            const uint32_t u = __umulhi(pick(r4, i & 3), (uint32_t)(p - 1));
            int dstart = i + 1 + (int)u;
            if (dstart >= p) dstart -= p;
            int donor = -1;
            if (valid) {
                const int ws = dstart >> 5, bs = dstart & 31;
                for (int step = 0; step <= Wv && donor < 0; ++step) {
                    int wc = ws + step;
                    if (wc >= Wv) wc -= Wv;
                    uint32_t diff = 0;
                    for (int a = 0; a < s; ++a)
                        diff |= P.P[(int64_t)F[a] * W + wc] ^ (0u - (uint32_t)((xf >> a) & 1u));
                    const int lim = p - 32 * wc;
                    uint32_t mk = lim >= 32 ? kFull : ((1u << lim) - 1u);
                    mk &= diff;
                    if (wc == w) mk &= ~(1u << lane);
                    if (step == 0)
                        mk &= kFull << bs;
                    else if (step == Wv)
                        mk &= ~(kFull << bs);
                    if (mk) donor = 32 * wc + __ffs(mk) - 1;
                }
            }

            // flips: the donor's bits on F_j that differ from the parent's
            uint64_t fm = 0;
            if (donor >= 0) {
                const int dw = donor >> 5, db = donor & 31;
                for (int a = 0; a < s; ++a) {
                    const uint32_t word = P.P[(int64_t)F[a] * W + dw];
                    fm |= (uint64_t)(((word >> db) & 1u) ^ (uint32_t)((xf >> a) & 1u)) << a;
                }
            }

            // PartialEvaluation over the element's dependency list
            long long delta = 0;
            const int2 *dep = P.dep + P.dep_ptr[j];
            const uint16_t *seg = P.seg + f0 + j;
            for (int a = 0; a < s; ++a) {
                const uint32_t fa = (uint32_t)(fm >> a) & 1u, xa = (uint32_t)(xf >> a) & 1u;
                const int q1 = seg[a + 1];
                for (int q = seg[a]; q < q1; ++q) {
                    const int2 d = dep[q];
                    uint32_t xb, fb;
                    if (d.x >= 0) {
                        xb = (P.O[(int64_t)d.x * W + w] >> lane) & 1u;
                        fb = 0;
                    } else {
                        const int b = -1 - d.x;
                        xb = (uint32_t)(xf >> b) & 1u;
                        fb = (uint32_t)(fm >> b) & 1u;
                    }
                    if (fa ^ fb) delta += (xa ^ xb) ? -(long long)d.y : (long long)d.y;
                }
            }

            const bool acc = donor >= 0 && (delta > 0 || (delta == 0 && !eqflag));
            for (int a = 0; a < s; ++a) {
                const uint32_t mk = __ballot_sync(kFull, acc && ((fm >> a) & 1u));
                if (lane == 0 && mk) P.O[(int64_t)F[a] * W + w] ^= mk;
            }
            if (acc) {
                facc += delta;
                ++n_acc;
                if (delta > 0) ++n_imp;
            }
            if (valid && donor < 0) ++n_dl;
        }
    }

    if (facc) atomicAdd((unsigned long long *)&s_f[i], (unsigned long long)facc);
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
