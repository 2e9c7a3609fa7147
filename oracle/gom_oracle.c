/*
 * gom_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU statement of parallel Gene-pool Optimal
 * Mixing (GOM) for weighted Max-Cut, written from Bouter & Bosman, "GPU-Accelerated
 * Parallel Gene-pool Optimal Mixing in a Gray-Box Optimization Setting"
 * (arXiv 2203.08680).  It is the checker of the CUDA library, not part of it:
 * only the test suite, the smoke check and the benchmark's CPU-baseline arm may
 * load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Everything is integer (int32 weights, int64 fitness), so every result is
 * exact and must be matched bit for bit.
 *
 * Population storage is the plainest possible: uint8 x[i*n + v] in {0,1}.
 *
 * Single-threaded, except orc_generation_par: the same generation with the
 * individuals of each colour group split over threads (OpenMP, when built
 * with it), which must give the identical state; it times the CPU baseline
 * on all host cores.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *  R1 objective: f(x) = sum over undirected edges {u,v} of w_uv [x_u != x_v];
 *     this is the Max-Cut formula of Sec. 6.2 with x in {-1,1} mapped from {0,1}.
 *  R2 FOS: neighbourhood F_j = {j} u adj(j) (sorted), or singleton F_j = {j}.
 *  R3 LMIG (Sec. 5.2): F_i ~ F_j iff they intersect or a VIG edge joins them.
 *  R4 Welsh-Powell (Sec. 5.2): visit elements by LMIG degree descending, ties
 *     by ascending index; give each the smallest colour unused by its
 *     already-coloured neighbours.  Groups list their elements ascending.
 *  R5 group order (Alg. 3 visits the groups in random order): colours sorted ascending by a
 *     64-bit Philox key per (colour, generation), ties by colour index.
 *  R6 donor (Sec. 4, SelectDonorFromPopulation): a uniform random start in the
 *     other p-1 individuals of the generation-start population P, then a
 *     cyclic scan to the first whose bits on F_j differ from the parent's
 *     current bits; no such individual means the trial is skipped.
 *  R7 partial evaluation (Sec. 2.2, Alg. 4): delta = sum over the set union of
 *     edges incident to F_j (each edge once) of new minus old contribution.
 *  R8 acceptance (Alg. 2, Sec. 5.3): accept iff delta > 0, or delta == 0 and
 *     the individual's generation-start genotype P[i] differs from the elitist.
 *  R9 elitist: after each generation, if max f > f_e the elitist becomes the
 *     lowest-index individual attaining max f.
 *  R10 random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *     (seed low, seed high), counters as in the functions below.
 *  R11 bounded fixed linkage tree (Sec. 4.1): UPGMA on the edge weights, linked
 *     pairs only, merges above the bound never made, ties by creation ids
 *     (orc_build_bflt).
 *  R12 Forced Improvement (Sec. 4, Alg. 1; off unless orc_set_fi switches it
 *     on -- the paper's parallel GOMEA runs without it, Sec. 5.4, and names a
 *     parallel-friendly variant as future work).  After the generation's
 *     mixing the elitist is updated as in R9; FI then applies to every
 *     individual with no accepted GOM step in the generation (or, with a
 *     threshold nis > 0, whose fitness has not improved for nis generations,
 *     this one included).  Such an individual takes GOM steps with the
 *     elitist as donor on the elements of each colour group, the groups in
 *     this generation's order; a step is accepted as in R8 with the flag
 *     "equal to the elitist" taken at the start of FI; FI stops after the
 *     first group in which a step improved its fitness (the elements of one
 *     group are independent of each other, so their order does not matter);
 *     if no step improved it, the individual becomes a copy of the elitist.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TAG_INIT 0x494E4954u  /* 'INIT' */
#define ORC_TAG_DONOR 0x444F4E52u /* 'DONR' */
#define ORC_TAG_ORDER 0x4F524452u /* 'ORDR' */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (SC'11, Sec. 4 and Table 2). */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t tag, int word)
{
    uint32_t ctr[4] = {a, b, c, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* floor(r * n / 2^32): maps a uniform 32-bit word onto [0, n). */
static uint32_t bounded(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* The graph (the Max-Cut instance, which is also the VIG, Sec. 2.3). */

/* 0 if the CSR is a simple undirected graph: rows sorted strictly ascending,
 * no self-loops, every (u,v,w) mirrored by (v,u,w).  -1 otherwise. */
int orc_check_graph(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *w)
{
    if (n < 0 || rp[0] != 0) return -1;
    for (int32_t u = 0; u < n; ++u) {
        if (rp[u + 1] < rp[u]) return -1;
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t v = col[e];
            if (v < 0 || v >= n || v == u) return -1;
            if (e > rp[u] && col[e - 1] >= v) return -1;
            /* find the mirror entry by a plain linear search */
            int found = 0;
            for (int64_t q = rp[v]; q < rp[v + 1]; ++q)
                if (col[q] == u) { found = (w[q] == w[e]); break; }
            if (!found) return -1;
        }
    }
    return 0;
}

/* R1: the cut weight of one assignment x[0..n). */
int64_t orc_cut_value(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                      const uint8_t *x)
{
    int64_t f = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t v = col[e];
            if (u < v && x[u] != x[v]) f += w[e];
        }
    return f;
}

/* Exhaustive maximum cut for n <= 26, fixing x_0 = 0 (a cut and its
 * complement have equal weight); each assignment evaluated from scratch. */
int64_t orc_brute_force_maxcut(int32_t n, const int64_t *rp, const int32_t *col,
                               const int32_t *w, uint8_t *best_x)
{
    if (n <= 0) return 0;
    if (n > 26) return -1;
    uint8_t *x = (uint8_t *)calloc((size_t)n, 1);
    int64_t best = INT64_MIN;
    uint64_t total = 1ull << (n - 1);
    for (uint64_t code = 0; code < total; ++code) {
        for (int32_t v = 1; v < n; ++v) x[v] = (uint8_t)((code >> (v - 1)) & 1u);
        x[0] = 0;
        int64_t f = orc_cut_value(n, rp, col, w, x);
        if (f > best) {
            best = f;
            if (best_x) memcpy(best_x, x, (size_t)n);
        }
    }
    free(x);
    return best;
}

/* ------------------------------------------------------------------------ */
/* FOS (Sec. 4.1), R2.  kind 0 = neighbourhood, 1 = singleton. */

int64_t orc_fos_total(int32_t n, const int64_t *rp, int32_t kind)
{
    if (kind == 1) return n;
    return rp[n] + n;
}

void orc_build_fos(int32_t n, const int64_t *rp, const int32_t *col, int32_t kind,
                   int64_t *eptr, int32_t *evars)
{
    int64_t pos = 0;
    for (int32_t j = 0; j < n; ++j) {
        eptr[j] = pos;
        if (kind == 1) {
            evars[pos++] = j;
            continue;
        }
        /* merge j into its (sorted) neighbour list */
        int placed = 0;
        for (int64_t e = rp[j]; e < rp[j + 1]; ++e) {
            if (!placed && j < col[e]) { evars[pos++] = j; placed = 1; }
            evars[pos++] = col[e];
        }
        if (!placed) evars[pos++] = j;
    }
    eptr[n] = pos;
}

/* ------------------------------------------------------------------------ */
/* Bounded fixed linkage tree (Sec. 4.1), R11: UPGMA on the Max-Cut graph with
 * the edge weights as similarity (Sec. 6.1 uses it for every GOMEA version).
 * Starting from the n singletons, repeatedly merge the pair of clusters with
 * the highest average pairwise similarity, sum of w_uv over u in A, v in B,
 * divided by |A||B|.  Readings: only clusters joined by at least one edge are
 * candidates (non-adjacent pairs have no dependence to link); a merge whose
 * result would exceed `bound` variables is never made, and the tree stops
 * when no candidate remains; a cluster holding all n variables is not a
 * linkage set (Sec. 4.1); ties go to the pair with the smaller first id,
 * then the smaller second id, ids numbering clusters in creation order
 * (singletons 0..n-1).  Elements: the singletons, then the merged clusters in
 * creation order, variables ascending.  Plain O(c^2) rescans per merge: for
 * the small graphs of the tests.  eptr[2n], evars[n * bound] (upper bounds);
 * returns the number of elements m. */

/* weight of edge {u,v}, and whether it exists */
static int edge_weight(const int64_t *rp, const int32_t *col, const int32_t *w, int32_t u, int32_t v,
                       int64_t *out)
{
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
        if (col[e] == v) { *out = w[e]; return 1; }
    return 0;
}

int64_t orc_build_bflt(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *w, int32_t bound,
                       int64_t *eptr, int32_t *evars)
{
    int64_t cap = 2 * (int64_t)n;
    int32_t *size = (int32_t *)calloc((size_t)cap + 1, sizeof(int32_t));
    uint8_t *alive = (uint8_t *)calloc((size_t)cap + 1, 1);
    int64_t *mptr = (int64_t *)calloc((size_t)cap + 2, sizeof(int64_t)); /* members of cluster c */
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n * (size_t)(bound > 0 ? bound : 1) + 1));
    int64_t nc = 0, nm = 0;
    for (int32_t v = 0; v < n; ++v) {
        mptr[nc] = nm;
        mem[nm++] = v;
        size[nc] = 1;
        alive[nc] = 1;
        ++nc;
    }
    mptr[nc] = nm;
    for (;;) {
        int64_t ba = -1, bb = -1, bs = 0, bn = 1;
        for (int64_t a = 0; a < nc; ++a) {
            if (!alive[a]) continue;
            for (int64_t b = a + 1; b < nc; ++b) {
                if (!alive[b] || size[a] + size[b] > bound) continue;
                int64_t S = 0;
                int linked = 0;
                for (int64_t x = mptr[a]; x < mptr[a + 1]; ++x)
                    for (int64_t y = mptr[b]; y < mptr[b + 1]; ++y) {
                        int64_t wv;
                        if (edge_weight(rp, col, w, mem[x], mem[y], &wv)) { S += wv; linked = 1; }
                    }
                if (!linked) continue;
                int64_t N = (int64_t)size[a] * size[b];
                /* S / N > bs / bn, exactly (128-bit products) */
                if (ba < 0 || (__int128)S * bn > (__int128)bs * N) { ba = a; bb = b; bs = S; bn = N; }
            }
        }
        if (ba < 0 || size[ba] + size[bb] >= n) break; /* nothing to merge, or the root */
        /* the new cluster: members of both, ascending */
        int64_t i = mptr[ba], j = mptr[bb];
        mptr[nc] = nm;
        while (i < mptr[ba + 1] || j < mptr[bb + 1]) {
            if (j >= mptr[bb + 1] || (i < mptr[ba + 1] && mem[i] < mem[j])) mem[nm++] = mem[i++];
            else mem[nm++] = mem[j++];
        }
        size[nc] = size[ba] + size[bb];
        alive[nc] = 1;
        alive[ba] = alive[bb] = 0;
        ++nc;
        mptr[nc] = nm;
    }
    for (int64_t c = 0; c <= nc; ++c) eptr[c] = mptr[c];
    memcpy(evars, mem, sizeof(int32_t) * (size_t)nm);
    free(size); free(alive); free(mptr); free(mem);
    return nc;
}

/* ------------------------------------------------------------------------ */
/* LMIG (Sec. 5.2), R3, and its Welsh-Powell colouring, R4. */

typedef struct {
    int64_t m;
    int64_t *nptr;   /* [m+1] */
    int32_t *nbr;    /* LMIG neighbours of each element, ascending */
} lmig_t;

/* The elements containing each variable (an inverted index of the FOS). */
static void invert_fos(int32_t n, int64_t m, const int64_t *eptr, const int32_t *evars,
                       int64_t **vptr_out, int32_t **velems_out)
{
    int64_t *vptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t q = 0; q < eptr[m]; ++q) vptr[evars[q] + 1]++;
    for (int32_t v = 0; v < n; ++v) vptr[v + 1] += vptr[v];
    int32_t *velems = (int32_t *)malloc(sizeof(int32_t) * (size_t)(eptr[m] > 0 ? eptr[m] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    memcpy(fill, vptr, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t j = 0; j < m; ++j)
        for (int64_t q = eptr[j]; q < eptr[j + 1]; ++q) velems[fill[evars[q]]++] = (int32_t)j;
    free(fill);
    *vptr_out = vptr;
    *velems_out = velems;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* F_j' is an LMIG neighbour of F_j iff F_j' shares a variable with
 * F_j u adj(F_j): that covers both the intersection and the edge case of R3. */
static lmig_t build_lmig(int32_t n, const int64_t *rp, const int32_t *col, int64_t m,
                         const int64_t *eptr, const int32_t *evars)
{
    int64_t *vptr;
    int32_t *velems;
    invert_fos(n, m, eptr, evars, &vptr, &velems);
    int64_t *seen = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) seen[j] = -1;
    int64_t cap = 1024, cnt = 0;
    int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int64_t *nptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    for (int64_t j = 0; j < m; ++j) {
        nptr[j] = cnt;
        for (int64_t q = eptr[j]; q < eptr[j + 1]; ++q) {
            int32_t u = evars[q];
            /* u itself, then every VIG neighbour of u */
            for (int64_t e = rp[u] - 1; e < rp[u + 1]; ++e) {
                int32_t v = (e < rp[u]) ? u : col[e];
                for (int64_t r = vptr[v]; r < vptr[v + 1]; ++r) {
                    int32_t jj = velems[r];
                    if (jj == j || seen[jj] == j) continue;
                    seen[jj] = j;
                    if (cnt == cap) {
                        cap *= 2;
                        nbr = (int32_t *)realloc(nbr, sizeof(int32_t) * (size_t)cap);
                    }
                    nbr[cnt++] = jj;
                }
            }
        }
        qsort(nbr + nptr[j], (size_t)(cnt - nptr[j]), sizeof(int32_t), cmp_i32);
    }
    nptr[m] = cnt;
    free(seen);
    free(vptr);
    free(velems);
    lmig_t L = {m, nptr, nbr};
    return L;
}

static void free_lmig(lmig_t *L)
{
    free(L->nptr);
    free(L->nbr);
}

/* Number of LMIG edges; writes up to cap (a<b) pairs into out_pairs. */
int64_t orc_lmig_edges(int32_t n, const int64_t *rp, const int32_t *col, int64_t m,
                       const int64_t *eptr, const int32_t *evars, int32_t *out_pairs, int64_t cap)
{
    lmig_t L = build_lmig(n, rp, col, m, eptr, evars);
    int64_t cnt = 0;
    for (int64_t a = 0; a < m; ++a)
        for (int64_t q = L.nptr[a]; q < L.nptr[a + 1]; ++q) {
            int32_t b = L.nbr[q];
            if (a < b) {
                if (cnt < cap) {
                    out_pairs[2 * cnt] = (int32_t)a;
                    out_pairs[2 * cnt + 1] = b;
                }
                ++cnt;
            }
        }
    free_lmig(&L);
    return cnt;
}

static const int64_t *g_sort_deg;
static int cmp_wp(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_sort_deg[x] != g_sort_deg[y]) return g_sort_deg[x] > g_sort_deg[y] ? -1 : 1;
    return (x > y) - (x < y);
}

/* Calls of the neighbour enumeration below: every LMIG neighbour jj != j of
 * element j, through the variables of F_j and of their VIG neighbours and the
 * elements holding each such variable; seen[] (stamped with j) makes each
 * neighbour appear once.  The LMIG itself is never stored. */
typedef struct {
    int32_t n;
    const int64_t *rp;
    const int32_t *col;
    const int64_t *eptr;
    const int32_t *evars;
    int64_t *vptr;
    int32_t *velems;
    int64_t *seen;
} lmig_walk;

static int64_t lmig_degree(lmig_walk *L, int64_t j)
{
    int64_t deg = 0;
    for (int64_t q = L->eptr[j]; q < L->eptr[j + 1]; ++q) {
        int32_t u = L->evars[q];
        for (int64_t e = L->rp[u] - 1; e < L->rp[u + 1]; ++e) {
            int32_t v = (e < L->rp[u]) ? u : L->col[e];
            for (int64_t r = L->vptr[v]; r < L->vptr[v + 1]; ++r) {
                int32_t jj = L->velems[r];
                if (jj == j || L->seen[jj] == j) continue;
                L->seen[jj] = j;
                ++deg;
            }
        }
    }
    return deg;
}

/* R4.  Returns the number of colours k; color_of_elem[j] in [0,k). */
int32_t orc_color(int32_t n, const int64_t *rp, const int32_t *col, int64_t m,
                  const int64_t *eptr, const int32_t *evars, int32_t *color_of_elem)
{
    lmig_walk L = {n, rp, col, eptr, evars, NULL, NULL, NULL};
    invert_fos(n, m, eptr, evars, &L.vptr, &L.velems);
    L.seen = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) L.seen[j] = -1;
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) {
        deg[j] = lmig_degree(&L, j);
        order[j] = (int32_t)j;
        color_of_elem[j] = -1;
    }
    g_sort_deg = deg;
    qsort(order, (size_t)m, sizeof(int32_t), cmp_wp);
    int32_t k = 0;
    int64_t *used = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    for (int64_t c = 0; c <= m; ++c) used[c] = -1;
    for (int64_t t = 0; t < m; ++t) {
        int32_t j = order[t];
        /* colours of the coloured LMIG neighbours of j */
        for (int64_t q = eptr[j]; q < eptr[j + 1]; ++q) {
            int32_t u = evars[q];
            for (int64_t e = rp[u] - 1; e < rp[u + 1]; ++e) {
                int32_t v = (e < rp[u]) ? u : col[e];
                for (int64_t r = L.vptr[v]; r < L.vptr[v + 1]; ++r) {
                    int32_t jj = L.velems[r];
                    if (jj != j && color_of_elem[jj] >= 0) used[color_of_elem[jj]] = j;
                }
            }
        }
        int32_t c = 0;
        while (used[c] == j) ++c;
        color_of_elem[j] = c;
        if (c + 1 > k) k = c + 1;
    }
    free(used);
    free(order);
    free(deg);
    free(L.seen);
    free(L.vptr);
    free(L.velems);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Partial evaluation (Sec. 2.2 and Alg. 4), R7. */

/* in_f[v] == stamp marks the variables of F.  x is the parent; y_on_f[q] is
 * the new value of F[q].  Returns new minus old over the union of the edges
 * incident to F, each edge counted once. */
static int64_t partial_delta(const int64_t *rp, const int32_t *col, const int32_t *w,
                             const uint8_t *x, const int32_t *F, int32_t sz, const uint8_t *y_on_f,
                             const int32_t *pos_in_f, const int64_t *in_f, int64_t stamp)
{
    int64_t d = 0;
    for (int32_t q = 0; q < sz; ++q) {
        int32_t u = F[q];
        uint8_t xu = x[u], yu = y_on_f[q];
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t v = col[e];
            uint8_t xv = x[v], yv = x[v];
            if (in_f[v] == stamp) {
                if (v < u) continue; /* counted from v's side */
                yv = y_on_f[pos_in_f[v]];
            }
            int64_t cut_new = (yu != yv), cut_old = (xu != xv);
            d += (int64_t)w[e] * (cut_new - cut_old);
        }
    }
    return d;
}

/* Exposed for the pins: delta of setting x on F[0..sz) to y_on_f. */
int64_t orc_partial_delta(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                          const uint8_t *x, const int32_t *F, int32_t sz, const uint8_t *y_on_f)
{
    int64_t *in_f = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) in_f[v] = -1;
    for (int32_t q = 0; q < sz; ++q) { in_f[F[q]] = 1; pos[F[q]] = q; }
    int64_t d = partial_delta(rp, col, w, x, F, sz, y_on_f, pos, in_f, 1);
    free(in_f);
    free(pos);
    return d;
}

/* ------------------------------------------------------------------------ */
/* Parallel GOMEA state (Alg. 3). */

typedef struct {
    int64_t generation;   /* index of the generation these counters describe */
    int64_t best;         /* max_i f[i] after the generation */
    int64_t elite;        /* f_e after the generation */
    int64_t trials;       /* (individual, element) pairs, donor-less included */
    int64_t donorless;
    int64_t accepted;
    int64_t improving;
    int64_t reached;      /* 1 if best >= target */
    int64_t fi_individuals; /* R12: individuals that entered FI */
    int64_t fi_trials;    /* their (individual, element) steps, those without variation included */
    int64_t fi_accepted;
    int64_t fi_improving;
    int64_t fi_replaced;  /* individuals replaced by a copy of the elitist */
} orc_stats;

/* Scratch of one trial: the element's membership stamps and donor bits. */
typedef struct {
    int64_t *in_f;    /* [n] stamp of the trial whose element holds v */
    int32_t *pos_in_f;/* [n] position of v in that element */
    int64_t stamp;
    uint8_t *ybuf;    /* [max element size] */
} orc_scratch;

typedef struct {
    int32_t n;
    int64_t *rp;
    int32_t *col, *w;
    int64_t m;
    int64_t *eptr;
    int32_t *evars;
    int32_t k;
    int64_t *cptr;   /* colour -> elements, ascending */
    int32_t *celems;
    int32_t p;
    uint64_t seed;
    uint8_t *O, *P;  /* [p][n] */
    int64_t *f;
    uint8_t *xe;
    int64_t fe;
    uint32_t g;
    uint8_t *eq;     /* [p] P[i] == x_e at generation start */
    int32_t fi_on;   /* R12 */
    int32_t fi_nis;  /* R12 threshold, 0 = condition off */
    uint8_t *acc_any;/* [p] an accepted GOM step in this generation */
    int32_t *nis;    /* [p] generations in a row without improvement */
    int64_t *f_start;/* [p] fitness at generation start */
    int32_t *ecnt;   /* [3][m] per element: accepted, donor-less and improving trials of the last
                        generation (NULL: not kept; single-threaded generations only) */
    int64_t max_s;   /* largest element */
    orc_scratch sc;  /* scratch of the single-threaded path */
} orc_state;

static void *dup_mem(const void *src, size_t bytes)
{
    void *d = malloc(bytes ? bytes : 1);
    if (bytes) memcpy(d, src, bytes);
    return d;
}

static void elitist_from_scratch(orc_state *s)
{
    int64_t best = INT64_MIN;
    int32_t arg = 0;
    for (int32_t i = 0; i < s->p; ++i)
        if (s->f[i] > best) { best = s->f[i]; arg = i; }
    memcpy(s->xe, s->O + (size_t)arg * s->n, (size_t)s->n);
    s->fe = best;
}

/* InitializePopulation (Alg. 3): bit v of individual i is bit (v mod 32) of
 * word (v/32 mod 4) of Philox(ctr = (v/128, i, 0, TAG_INIT)). */
void orc_init_individual(uint64_t seed, int32_t i, int32_t n, uint8_t *x)
{
    for (int32_t v = 0; v < n; ++v) {
        uint32_t r = draw(seed, (uint32_t)v >> 7, (uint32_t)i, 0u, ORC_TAG_INIT, (v >> 5) & 3);
        x[v] = (uint8_t)((r >> (v & 31)) & 1u);
    }
}

static void scratch_init(orc_scratch *sc, int32_t n, int64_t max_s)
{
    sc->in_f = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    sc->pos_in_f = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t v = 0; v < n; ++v) sc->in_f[v] = -1;
    sc->stamp = 0;
    sc->ybuf = (uint8_t *)malloc((size_t)max_s);
}

static void scratch_free(orc_scratch *sc)
{
    free(sc->in_f);
    free(sc->pos_in_f);
    free(sc->ybuf);
}

/* With init = 0 the population is left zero (for orc_load). */
orc_state *orc_new_ex(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                      int64_t m, const int64_t *eptr, const int32_t *evars,
                      const int32_t *color_of_elem, int32_t k, int32_t p, uint64_t seed, int32_t init)
{
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    s->n = n;
    s->rp = (int64_t *)dup_mem(rp, sizeof(int64_t) * ((size_t)n + 1));
    s->col = (int32_t *)dup_mem(col, sizeof(int32_t) * (size_t)rp[n]);
    s->w = (int32_t *)dup_mem(w, sizeof(int32_t) * (size_t)rp[n]);
    s->m = m;
    s->eptr = (int64_t *)dup_mem(eptr, sizeof(int64_t) * ((size_t)m + 1));
    s->evars = (int32_t *)dup_mem(evars, sizeof(int32_t) * (size_t)eptr[m]);
    s->k = k;
    s->cptr = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    s->celems = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) s->cptr[color_of_elem[j] + 1]++;
    for (int32_t c = 0; c < k; ++c) s->cptr[c + 1] += s->cptr[c];
    {
        int64_t *fill = (int64_t *)dup_mem(s->cptr, sizeof(int64_t) * ((size_t)k + 1));
        for (int64_t j = 0; j < m; ++j) s->celems[fill[color_of_elem[j]]++] = (int32_t)j;
        free(fill);
    }
    s->p = p;
    s->seed = seed;
    s->O = (uint8_t *)malloc((size_t)p * (size_t)n + 1);
    s->P = (uint8_t *)malloc((size_t)p * (size_t)n + 1);
    s->f = (int64_t *)malloc(sizeof(int64_t) * (size_t)p);
    s->xe = (uint8_t *)malloc((size_t)n + 1);
    s->eq = (uint8_t *)malloc((size_t)p);
    s->acc_any = (uint8_t *)calloc((size_t)p, 1);
    s->nis = (int32_t *)calloc((size_t)p, sizeof(int32_t));
    s->f_start = (int64_t *)calloc((size_t)p, sizeof(int64_t));
    s->fi_on = 0;
    s->fi_nis = 0;
    s->g = 0;
    if (!init) {
        memset(s->O, 0, (size_t)p * (size_t)n);
        memset(s->f, 0, sizeof(int64_t) * (size_t)p);
        memset(s->xe, 0, (size_t)n);
        s->fe = 0;
    }
    s->max_s = 1;
    for (int64_t j = 0; j < m; ++j)
        if (eptr[j + 1] - eptr[j] > s->max_s) s->max_s = eptr[j + 1] - eptr[j];
    scratch_init(&s->sc, n, s->max_s);
    if (!init) return s;
    for (int32_t i = 0; i < p; ++i) orc_init_individual(seed, i, n, s->O + (size_t)i * n);
    for (int32_t i = 0; i < p; ++i) s->f[i] = orc_cut_value(n, rp, col, w, s->O + (size_t)i * n);
    elitist_from_scratch(s);
    return s;
}

orc_state *orc_new(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                   int64_t m, const int64_t *eptr, const int32_t *evars,
                   const int32_t *color_of_elem, int32_t k, int32_t p, uint64_t seed)
{
    return orc_new_ex(n, rp, col, w, m, eptr, evars, color_of_elem, k, p, seed, 1);
}

void orc_free(orc_state *s)
{
    if (!s) return;
    free(s->rp); free(s->col); free(s->w); free(s->eptr); free(s->evars);
    free(s->cptr); free(s->celems); free(s->O); free(s->P); free(s->f); free(s->xe);
    free(s->eq);
    free(s->acc_any);
    free(s->nis);
    free(s->f_start);
    free(s->ecnt);
    scratch_free(&s->sc);
    free(s);
}

/* Overwrite the state (used to resume from, or replay, a given point). */
void orc_load(orc_state *s, const uint8_t *pop, const int64_t *f, const uint8_t *xe, int64_t fe,
              uint32_t g)
{
    memcpy(s->O, pop, (size_t)s->p * s->n);
    memcpy(s->f, f, sizeof(int64_t) * (size_t)s->p);
    memcpy(s->xe, xe, (size_t)s->n);
    s->fe = fe;
    s->g = g;
}

void orc_get(const orc_state *s, uint8_t *pop, int64_t *f, uint8_t *xe, int64_t *fe, uint32_t *g)
{
    if (pop) memcpy(pop, s->O, (size_t)s->p * s->n);
    if (f) memcpy(f, s->f, sizeof(int64_t) * (size_t)s->p);
    if (xe) memcpy(xe, s->xe, (size_t)s->n);
    if (fe) *fe = s->fe;
    if (g) *g = s->g;
}

/* R5: the order of the colour groups in generation g. */
static uint64_t order_key(uint64_t seed, int32_t c, uint32_t g)
{
    uint32_t ctr[4] = {(uint32_t)c, 0u, g, ORC_TAG_ORDER};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return ((uint64_t)out[0] << 32) | out[1];
}

void orc_group_order(uint64_t seed, int32_t k, uint32_t g, int32_t *order)
{
    /* selection of the smallest remaining (key, colour) pair, k times */
    uint8_t *taken = (uint8_t *)calloc((size_t)k + 1, 1);
    for (int32_t t = 0; t < k; ++t) {
        int32_t best = -1;
        uint64_t bk = 0;
        for (int32_t c = 0; c < k; ++c) {
            if (taken[c]) continue;
            uint64_t key = order_key(seed, c, g);
            if (best < 0 || key < bk) { best = c; bk = key; }
        }
        taken[best] = 1;
        order[t] = best;
    }
    free(taken);
}

/* One GOM trial (Alg. 2) of individual i with element j. */
static void gom_trial(orc_state *s, orc_scratch *sc, int32_t i, int32_t j, orc_stats *st)
{
    const int32_t n = s->n, p = s->p;
    const int32_t *F = s->evars + s->eptr[j];
    const int32_t sz = (int32_t)(s->eptr[j + 1] - s->eptr[j]);
    uint8_t *o = s->O + (size_t)i * n;

    /* SelectDonorFromPopulation, R6 */
    uint32_t r = draw(s->seed, (uint32_t)j, (uint32_t)i >> 2, s->g, ORC_TAG_DONOR, i & 3);
    uint32_t u = bounded(r, (uint32_t)(p - 1));
    int32_t donor = -1;
    for (int32_t t = 0; t <= p - 2 && donor < 0; ++t) {
        int32_t d = (int32_t)((i + 1 + (int64_t)((u + (uint32_t)t) % (uint32_t)(p - 1))) % p);
        const uint8_t *pd = s->P + (size_t)d * n;
        for (int32_t q = 0; q < sz; ++q)
            if (pd[F[q]] != o[F[q]]) { donor = d; break; }
    }
    st->trials++;
    if (donor < 0) {
        st->donorless++;
        if (s->ecnt) s->ecnt[s->m + j]++;
        return;
    }

    /* PartialEvaluation, R7 */
    const uint8_t *pd = s->P + (size_t)donor * n;
    uint8_t *y = sc->ybuf;
    sc->stamp++;
    for (int32_t q = 0; q < sz; ++q) {
        y[q] = pd[F[q]];
        sc->in_f[F[q]] = sc->stamp;
        sc->pos_in_f[F[q]] = q;
    }
    int64_t d = partial_delta(s->rp, s->col, s->w, o, F, sz, y, sc->pos_in_f, sc->in_f, sc->stamp);

    /* acceptance, R8 */
    if (d > 0 || (d == 0 && !s->eq[i])) {
        for (int32_t q = 0; q < sz; ++q) o[F[q]] = y[q];
        s->f[i] += d;
        st->accepted++;
        if (d > 0) st->improving++;
        s->acc_any[i] = 1;
        if (s->ecnt) {
            s->ecnt[j]++;
            if (d > 0) s->ecnt[2 * s->m + j]++;
        }
    }
}

/* Keeps (on != 0) or stops keeping the per-element counters of each
 * generation: accepted, donor-less and improving trials of element j. */
void orc_keep_element_counts(orc_state *s, int32_t on)
{
    free(s->ecnt);
    s->ecnt = on ? (int32_t *)calloc(3 * (size_t)(s->m > 0 ? s->m : 1), sizeof(int32_t)) : NULL;
}

/* The per-element counters of the last generation (each [m], may be NULL). */
void orc_element_counts(const orc_state *s, int32_t *acc, int32_t *dl, int32_t *imp)
{
    if (!s->ecnt) return;
    if (acc) memcpy(acc, s->ecnt, sizeof(int32_t) * (size_t)s->m);
    if (dl) memcpy(dl, s->ecnt + s->m, sizeof(int32_t) * (size_t)s->m);
    if (imp) memcpy(imp, s->ecnt + 2 * s->m, sizeof(int32_t) * (size_t)s->m);
}

/* R12: switches Forced Improvement on or off, with its no-improvement
 * threshold (0: only individuals without an accepted step enter FI). */
void orc_set_fi(orc_state *s, int32_t on, int32_t nis)
{
    s->fi_on = on ? 1 : 0;
    s->fi_nis = nis > 0 ? nis : 0;
}

/* One FI step (R12) of individual i on element j: the elitist as donor,
 * accepted as in R8 with the flag eq_fi.  Returns 1 if it improved f[i]. */
static int fi_trial(orc_state *s, orc_scratch *sc, int32_t i, int32_t j, uint8_t eq_fi, orc_stats *st)
{
    const int32_t n = s->n;
    const int32_t *F = s->evars + s->eptr[j];
    const int32_t sz = (int32_t)(s->eptr[j + 1] - s->eptr[j]);
    uint8_t *o = s->O + (size_t)i * n;
    st->fi_trials++;
    int differs = 0;
    for (int32_t q = 0; q < sz; ++q)
        if (s->xe[F[q]] != o[F[q]]) differs = 1;
    if (!differs) return 0; /* no variation: GOM is not performed */
    uint8_t *y = sc->ybuf;
    sc->stamp++;
    for (int32_t q = 0; q < sz; ++q) {
        y[q] = s->xe[F[q]];
        sc->in_f[F[q]] = sc->stamp;
        sc->pos_in_f[F[q]] = q;
    }
    int64_t d = partial_delta(s->rp, s->col, s->w, o, F, sz, y, sc->pos_in_f, sc->in_f, sc->stamp);
    if (d > 0 || (d == 0 && !eq_fi)) {
        for (int32_t q = 0; q < sz; ++q) o[F[q]] = y[q];
        s->f[i] += d;
        st->fi_accepted++;
        if (d > 0) st->fi_improving++;
        return d > 0;
    }
    return 0;
}

/* R12: Forced Improvement after the generation's mixing, groups in `order`. */
static void forced_improvement(orc_state *s, const int32_t *order, orc_stats *st)
{
    const int32_t n = s->n, p = s->p;
    /* the elitist of the population as it is now (R9's rule) */
    int64_t best = INT64_MIN;
    int32_t arg = 0;
    for (int32_t i = 0; i < p; ++i)
        if (s->f[i] > best) { best = s->f[i]; arg = i; }
    if (best > s->fe) {
        s->fe = best;
        memcpy(s->xe, s->O + (size_t)arg * n, (size_t)n);
    }
    for (int32_t i = 0; i < p; ++i) {
        const int stale = s->fi_nis > 0 && (s->f[i] > s->f_start[i] ? 0 : s->nis[i] + 1) >= s->fi_nis;
        if (s->acc_any[i] && !stale) continue;
        st->fi_individuals++;
        const uint8_t eq_fi = memcmp(s->O + (size_t)i * n, s->xe, (size_t)n) == 0;
        int improved = 0;
        for (int32_t t = 0; t < s->k && !improved; ++t) {
            const int32_t c = order[t];
            for (int64_t q = s->cptr[c]; q < s->cptr[c + 1]; ++q)
                improved |= fi_trial(s, &s->sc, i, s->celems[q], eq_fi, st);
        }
        if (!improved) {
            memcpy(s->O + (size_t)i * n, s->xe, (size_t)n);
            s->f[i] = s->fe;
            st->fi_replaced++;
        }
    }
}

/* R12 bookkeeping at generation end: generations without improvement. */
static void fi_count_stale(orc_state *s)
{
    for (int32_t i = 0; i < s->p; ++i) s->nis[i] = s->f[i] > s->f_start[i] ? 0 : s->nis[i] + 1;
}

/* Small deterministic generator used only to permute the trials of one group
 * in the order-invariance test (it is not one of the method's random draws). */
static uint64_t splitmix_next(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Generation start (Alg. 3): Clone P <- O; R8 flags. */
static void generation_start(orc_state *s)
{
    const int32_t n = s->n, p = s->p;
    memcpy(s->P, s->O, (size_t)p * n);
    /* R8: the elitist flag of each individual is fixed at generation start */
    for (int32_t i = 0; i < p; ++i) s->eq[i] = memcmp(s->P + (size_t)i * n, s->xe, (size_t)n) == 0;
    memset(s->acc_any, 0, (size_t)p);
    memcpy(s->f_start, s->f, sizeof(int64_t) * (size_t)p);
    if (s->ecnt) memset(s->ecnt, 0, sizeof(int32_t) * 3 * (size_t)s->m);
}

/* Generation end: R9 elitist update, the target check, g += 1. */
static void generation_end(orc_state *s, int64_t target, orc_stats *st)
{
    int64_t best = INT64_MIN;
    int32_t arg = 0;
    for (int32_t i = 0; i < s->p; ++i)
        if (s->f[i] > best) { best = s->f[i]; arg = i; }
    if (best > s->fe) {
        s->fe = best;
        memcpy(s->xe, s->O + (size_t)arg * s->n, (size_t)s->n);
    }
    st->best = best;
    st->elite = s->fe;
    st->reached = best >= target;
}

/* One generation of Par-GOMEA (Alg. 3).  `shuffle` != 0 visits the trials of
 * each group in a permuted order; `only`/`n_only` restricts the trials to a
 * subset of individuals (the elitist update is then skipped, since it needs the
 * whole population).  A run stops once a generation ends with max f >= target;
 * that stop is the caller's loop, st->reached reports it. */
static int32_t generation_impl(orc_state *s, int64_t target, uint64_t shuffle, const int32_t *only,
                               int32_t n_only, const uint8_t *skip_elem, orc_stats *st);

int32_t orc_generation_ex(orc_state *s, int64_t target, uint64_t shuffle, const int32_t *only,
                          int32_t n_only, orc_stats *st)
{
    return generation_impl(s, target, shuffle, only, n_only, NULL, st);
}

/* The generation with the trials of the elements marked in skip_elem[j] left
 * out (a replay of a run whose learned filter skipped them); everything else
 * is the plain generation. */
int32_t orc_generation_skip(orc_state *s, int64_t target, const uint8_t *skip_elem, orc_stats *st)
{
    return generation_impl(s, target, 0, NULL, 0, skip_elem, st);
}

static int32_t generation_impl(orc_state *s, int64_t target, uint64_t shuffle, const int32_t *only,
                               int32_t n_only, const uint8_t *skip_elem, orc_stats *st)
{
    memset(st, 0, sizeof(*st));
    const int32_t p = s->p;
    generation_start(s);

    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s->k > 0 ? s->k : 1));
    orc_group_order(s->seed, s->k, s->g, order);

    int32_t n_ind = only ? n_only : p;
    for (int32_t t = 0; t < s->k; ++t) {
        int32_t c = order[t];
        int64_t gsz = s->cptr[c + 1] - s->cptr[c];
        int64_t ntr = gsz * n_ind;
        int64_t *perm = NULL;
        uint64_t sm = shuffle;
        if (shuffle) {
            perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ntr > 0 ? ntr : 1));
            for (int64_t q = 0; q < ntr; ++q) perm[q] = q;
            for (int64_t q = ntr - 1; q > 0; --q) {
                int64_t r = (int64_t)(splitmix_next(&sm) % (uint64_t)(q + 1));
                int64_t tmp = perm[q]; perm[q] = perm[r]; perm[r] = tmp;
            }
        }
        for (int64_t q = 0; q < ntr; ++q) {
            int64_t id = perm ? perm[q] : q;
            int32_t j = s->celems[s->cptr[c] + id / n_ind];
            int32_t ii = (int32_t)(id % n_ind);
            int32_t i = only ? only[ii] : ii;
            if (skip_elem && skip_elem[j]) continue;
            gom_trial(s, &s->sc, i, j, st);
        }
        free(perm);
    }
    if (s->fi_on && !only) {
        forced_improvement(s, order, st);
        fi_count_stale(s);
    }
    free(order);

    st->generation = s->g;
    if (!only) generation_end(s, target, st);
    s->g++;
    return 0;
}

/* Threads the multi-threaded generation can use (1 without OpenMP). */
int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The same generation with the individuals of each colour group split over
 * `threads` threads (OpenMP).  The trials of one group are independent of
 * one another -- its elements share no variable and no edge (LMIG colouring),
 * donors come from the frozen P, the elitist flags are fixed -- so any order,
 * and this parallel one, gives the single-threaded result (checked by the
 * test suite).  Each thread has its own scratch and counters. */
int32_t orc_generation_par_ex(orc_state *s, int64_t target, int32_t threads, const int32_t *only, int32_t n_only,
                              orc_stats *st);

int32_t orc_generation_par(orc_state *s, int64_t target, int32_t threads, orc_stats *st)
{
    return orc_generation_par_ex(s, target, threads, NULL, 0, st);
}

/* The multi-threaded generation for the individuals only[0..n_only) (all if
 * only is NULL); with a subset the elitist update is skipped, as in
 * orc_generation_ex. */
int32_t orc_generation_par_ex(orc_state *s, int64_t target, int32_t threads, const int32_t *only, int32_t n_only,
                              orc_stats *st)
{
    memset(st, 0, sizeof(*st));
    if (s->ecnt) return -1; /* per-element counters: single-threaded generations only */
    const int32_t p = only ? n_only : s->p;
    if (threads < 1) threads = 1;
    generation_start(s);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s->k > 0 ? s->k : 1));
    orc_group_order(s->seed, s->k, s->g, order);
    orc_scratch *sc = (orc_scratch *)malloc(sizeof(orc_scratch) * (size_t)threads);
    orc_stats *ts = (orc_stats *)calloc((size_t)threads, sizeof(orc_stats));
    for (int32_t th = 0; th < threads; ++th) scratch_init(&sc[th], s->n, s->max_s);
    for (int32_t t = 0; t < s->k; ++t) {
        const int32_t c = order[t];
        const int64_t e0 = s->cptr[c], e1 = s->cptr[c + 1];
#pragma omp parallel for num_threads(threads) schedule(static)
        for (int32_t ii = 0; ii < p; ++ii) {
#ifdef _OPENMP
            const int th = omp_get_thread_num();
#else
            const int th = 0;
#endif
            const int32_t i = only ? only[ii] : ii;
            for (int64_t q = e0; q < e1; ++q) gom_trial(s, &sc[th], i, s->celems[q], &ts[th]);
        }
    }
    for (int32_t th = 0; th < threads; ++th) {
        st->trials += ts[th].trials;
        st->donorless += ts[th].donorless;
        st->accepted += ts[th].accepted;
        st->improving += ts[th].improving;
        scratch_free(&sc[th]);
    }
    free(sc);
    free(ts);
    if (s->fi_on && !only) {
        forced_improvement(s, order, st);
        fi_count_stale(s);
    }
    free(order);
    st->generation = s->g;
    if (!only) generation_end(s, target, st);
    s->g++;
    return 0;
}

int32_t orc_generation(orc_state *s, int64_t target, orc_stats *st)
{
    return orc_generation_ex(s, target, 0, NULL, 0, st);
}
