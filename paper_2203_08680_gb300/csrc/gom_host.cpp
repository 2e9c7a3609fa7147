// gom_host.cpp -- one-time host set-up of parallel GOM: graph validation, the
// linkage model (FOS, Sec. 4.1), the Welsh-Powell colouring of the linkage
// model interaction graph (LMIG, Sec. 5.2) and the per-element dependency
// tables (the edges incident to each element, Alg. 4, in colour order).
//
// Large instances (10^6 elements) are handled without materialising the LMIG:
// the neighbours of an element are enumerated on the fly through a
// variable -> elements index, and the degree pass runs on all host threads.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <queue>
#include <thread>
#include <utility>
#include <vector_types.h>

#include "gom_internal.h"

namespace gomh {

namespace {

int num_threads()
{
    unsigned t = std::thread::hardware_concurrency();
    return t == 0 ? 1 : static_cast<int>(std::min(t, 64u));
}

// Runs body(begin, end) over [0, count) split into contiguous ranges.
template <class F>
void parallel_ranges(int64_t count, F body)
{
    int nt = num_threads();
    if (count < 4096 || nt == 1) {
        body(int64_t(0), count);
        return;
    }
    std::vector<std::thread> pool;
    int64_t chunk = (count + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        int64_t b = t * chunk, e = std::min(count, b + chunk);
        if (b >= e) break;
        pool.emplace_back([=] { body(b, e); });
    }
    for (auto &th : pool) th.join();
}

} // namespace

int validate_graph(const gom_graph_t *g)
{
    if (!g || g->num_vertices < 0 || g->num_adj < 0) return GOM_E_ARG;
    const int32_t n = g->num_vertices;
    if (!g->row_ptr) return GOM_E_ARG;
    if (g->num_adj > 0 && (!g->col || !g->weight)) return GOM_E_ARG;
    if (g->row_ptr[0] != 0 || g->row_ptr[n] != g->num_adj) return GOM_E_GRAPH;
    for (int32_t u = 0; u < n; ++u)
        if (g->row_ptr[u + 1] < g->row_ptr[u]) return GOM_E_GRAPH;
    std::atomic<int> bad{0};
    parallel_ranges(n, [&](int64_t b, int64_t e) {
        for (int64_t u = b; u < e && !bad.load(std::memory_order_relaxed); ++u) {
            const int64_t r0 = g->row_ptr[u], r1 = g->row_ptr[u + 1];
            for (int64_t q = r0; q < r1; ++q) {
                const int32_t v = g->col[q];
                if (v < 0 || v >= n || v == u || (q > r0 && g->col[q - 1] >= v)) {
                    bad = 1;
                    break;
                }
                // the mirror entry (v, u) with the same weight, by binary search
                const int32_t *lo = g->col + g->row_ptr[v], *hi = g->col + g->row_ptr[v + 1];
                const int32_t *it = std::lower_bound(lo, hi, static_cast<int32_t>(u));
                if (it == hi || *it != u || g->weight[it - g->col] != g->weight[q]) {
                    bad = 1;
                    break;
                }
            }
        }
    });
    return bad ? GOM_E_GRAPH : GOM_OK;
}

int build_fos(const gom_graph_t *g, int32_t kind, gom_fos *out)
{
    const int32_t n = g->num_vertices;
    out->n = n;
    out->m = n;
    out->k = -1;
    out->eptr.assign(static_cast<size_t>(n) + 1, 0);
    if (kind == GOM_FOS_SINGLETON) {
        out->evars.resize(n);
        for (int32_t j = 0; j < n; ++j) {
            out->eptr[j + 1] = j + 1;
            out->evars[j] = j;
        }
        return GOM_OK;
    }
    if (kind != GOM_FOS_NEIGHBOURHOOD) return GOM_E_ARG;
    for (int32_t j = 0; j < n; ++j)
        out->eptr[j + 1] = out->eptr[j] + (g->row_ptr[j + 1] - g->row_ptr[j]) + 1;
    out->evars.resize(out->eptr[n]);
    parallel_ranges(n, [&](int64_t b, int64_t e) {
        for (int64_t j = b; j < e; ++j) {
            int32_t *dst = out->evars.data() + out->eptr[j];
            const int32_t *nb = g->col + g->row_ptr[j];
            const int64_t d = g->row_ptr[j + 1] - g->row_ptr[j];
            // the row is sorted: j goes before the first larger neighbour
            int64_t split = std::lower_bound(nb, nb + d, static_cast<int32_t>(j)) - nb;
            std::memcpy(dst, nb, sizeof(int32_t) * split);
            dst[split] = static_cast<int32_t>(j);
            std::memcpy(dst + split + 1, nb + split, sizeof(int32_t) * (d - split));
        }
    });
    return GOM_OK;
}

int build_bflt(const gom_graph_t *g, int32_t bound, gom_fos *out)
{
    if (bound < 1) return GOM_E_ARG;
    const int32_t n = g->num_vertices;
    // candidate merge: clusters a < b joined by at least one edge, summed weight S, N = |a| |b|
    struct Cand {
        int64_t S, N;
        int32_t a, b;
    };
    // lower priority: smaller average S/N (exact, 128-bit products), then larger a, then larger b
    auto lower = [](const Cand &x, const Cand &y) {
        const __int128 lx = static_cast<__int128>(x.S) * y.N, ly = static_cast<__int128>(y.S) * x.N;
        if (lx != ly) return lx < ly;
        if (x.a != y.a) return x.a > y.a;
        return x.b > y.b;
    };
    std::priority_queue<Cand, std::vector<Cand>, decltype(lower)> pq(lower);
    std::vector<int32_t> size(n, 1);
    std::vector<uint8_t> alive(n, 1);
    std::vector<std::vector<std::pair<int32_t, int64_t>>> adj(n); // neighbour cluster -> weight sum, ascending
    std::vector<std::vector<int32_t>> members(n);
    for (int32_t v = 0; v < n; ++v) {
        members[v] = {v};
        for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
            adj[v].push_back({g->col[e], g->weight[e]});
            if (v < g->col[e] && bound >= 2) pq.push({g->weight[e], 1, v, g->col[e]});
        }
    }
    while (!pq.empty()) {
        const Cand top = pq.top();
        pq.pop();
        if (!alive[top.a] || !alive[top.b]) continue; // stale: a cluster was merged since
        const int32_t a = top.a, b = top.b;
        if (size[a] + size[b] >= n) break; // the set of all variables is no linkage set
        const int32_t c = static_cast<int32_t>(size.size());
        size.push_back(size[a] + size[b]);
        alive.push_back(1);
        alive[a] = alive[b] = 0;
        std::vector<int32_t> mc(members[a].size() + members[b].size());
        std::merge(members[a].begin(), members[a].end(), members[b].begin(), members[b].end(), mc.begin());
        members.push_back(std::move(mc));
        // neighbours of the new cluster: those of a and b (summed), without a and b
        std::vector<std::pair<int32_t, int64_t>> ac;
        {
            const auto &A = adj[a], &Bv = adj[b];
            size_t i = 0, j = 0;
            while (i < A.size() || j < Bv.size()) {
                std::pair<int32_t, int64_t> x;
                if (j >= Bv.size() || (i < A.size() && A[i].first < Bv[j].first))
                    x = A[i++];
                else if (i >= A.size() || Bv[j].first < A[i].first)
                    x = Bv[j++];
                else {
                    x = {A[i].first, A[i].second + Bv[j].second};
                    ++i;
                    ++j;
                }
                if (x.first != a && x.first != b) ac.push_back(x);
            }
        }
        for (const auto &xs : ac) {
            auto &ax = adj[xs.first];
            ax.erase(std::remove_if(ax.begin(), ax.end(),
                                    [&](const std::pair<int32_t, int64_t> &y) { return y.first == a || y.first == b; }),
                     ax.end());
            ax.push_back({c, xs.second}); // c is the largest id: the list stays ascending
            if (size[c] + size[xs.first] <= bound)
                pq.push({xs.second, static_cast<int64_t>(size[c]) * size[xs.first], xs.first, c});
        }
        adj.push_back(std::move(ac));
        adj[a].clear();
        adj[a].shrink_to_fit();
        adj[b].clear();
        adj[b].shrink_to_fit();
    }
    out->n = n;
    out->m = static_cast<int64_t>(members.size());
    out->k = -1;
    out->eptr.assign(static_cast<size_t>(out->m) + 1, 0);
    for (int64_t j = 0; j < out->m; ++j) out->eptr[j + 1] = out->eptr[j] + static_cast<int64_t>(members[j].size());
    out->evars.resize(static_cast<size_t>(out->eptr[out->m]));
    for (int64_t j = 0; j < out->m; ++j)
        std::copy(members[j].begin(), members[j].end(), out->evars.begin() + out->eptr[j]);
    return GOM_OK;
}

int check_fos(int32_t n, const gom_fos &fos)
{
    if (fos.eptr.size() != static_cast<size_t>(fos.m) + 1 || fos.eptr[0] != 0) return GOM_E_FOS;
    std::vector<uint8_t> covered(n, 0);
    for (int64_t j = 0; j < fos.m; ++j) {
        if (fos.eptr[j + 1] <= fos.eptr[j]) return GOM_E_FOS; // empty element
        for (int64_t q = fos.eptr[j]; q < fos.eptr[j + 1]; ++q) {
            const int32_t v = fos.evars[q];
            if (v < 0 || v >= n) return GOM_E_FOS;
            if (q > fos.eptr[j] && fos.evars[q - 1] >= v) return GOM_E_FOS;
            covered[v] = 1;
        }
    }
    for (int32_t v = 0; v < n; ++v)
        if (!covered[v]) return GOM_E_FOS; // FOS must be complete (Sec. 4.1)
    return GOM_OK;
}

namespace {

// variable -> elements containing it
struct Inverted {
    std::vector<int64_t> ptr;
    std::vector<int32_t> elems;
};

Inverted invert(int32_t n, const gom_fos &fos)
{
    Inverted inv;
    inv.ptr.assign(static_cast<size_t>(n) + 1, 0);
    for (int32_t v : fos.evars) inv.ptr[v + 1]++;
    for (int32_t v = 0; v < n; ++v) inv.ptr[v + 1] += inv.ptr[v];
    inv.elems.resize(fos.evars.size());
    std::vector<int64_t> fill(inv.ptr.begin(), inv.ptr.end() - 1);
    for (int64_t j = 0; j < fos.m; ++j)
        for (int64_t q = fos.eptr[j]; q < fos.eptr[j + 1]; ++q)
            inv.elems[fill[fos.evars[q]]++] = static_cast<int32_t>(j);
    return inv;
}

// Calls visit(j2) for every LMIG neighbour j2 of element j: the elements
// holding a variable of F_j or of adj(F_j).  vmark (one entry per variable)
// makes each such variable's element list scanned once per j.  With a mark
// array each neighbour is visited once; without one (mark == nullptr) a
// neighbour may be visited several times, which is enough for first-fit
// colouring.
template <class V>
void for_each_lmig_neighbour(const gom_graph_t *g, const gom_fos &fos, const Inverted &inv,
                             int64_t j, int32_t *mark, int32_t *vmark, V visit)
{
    auto touch_var = [&](int32_t v) {
        if (vmark[v] == j) return;
        vmark[v] = static_cast<int32_t>(j);
        for (int64_t r = inv.ptr[v]; r < inv.ptr[v + 1]; ++r) {
            const int32_t j2 = inv.elems[r];
            if (j2 == j) continue;
            if (mark) {
                if (mark[j2] == j) continue;
                mark[j2] = static_cast<int32_t>(j);
            }
            visit(j2);
        }
    };
    for (int64_t q = fos.eptr[j]; q < fos.eptr[j + 1]; ++q) {
        const int32_t u = fos.evars[q];
        touch_var(u);
        for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) touch_var(g->col[e]);
    }
}

} // namespace

int color_fos(const gom_graph_t *g, gom_fos *fos)
{
    const int64_t m = fos->m;
    const Inverted inv = invert(fos->n, *fos);

    // LMIG degree of every element
    std::vector<int64_t> deg(m, 0);
    parallel_ranges(m, [&](int64_t b, int64_t e) {
        std::vector<int32_t> mark(m, -1), vmark(fos->n, -1);
        for (int64_t j = b; j < e; ++j) {
            int64_t d = 0;
            for_each_lmig_neighbour(g, *fos, inv, j, mark.data(), vmark.data(), [&](int32_t) { ++d; });
            deg[j] = d;
        }
    });

    // Welsh-Powell order: degree descending, index ascending
    std::vector<int32_t> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return deg[a] > deg[b]; });

    // first fit in that order.  The colours taken by j's LMIG neighbours are
    // the colours of the coloured elements that hold a variable of C_j = F_j
    // united with adj(F_j); cset[v] keeps, as a bitset, the colours of the
    // coloured elements holding v, so j's forbidden colours are the union of
    // cset over C_j (each variable once), and colouring j with c adds c to
    // cset[v] for v in F_j.  Same colours as visiting the neighbours one by one.
    std::vector<int32_t> color(m, -1);
    int32_t k = 0;
    int64_t words = 1; // 64-bit words per variable's bitset, doubled when the colours outgrow it
    std::vector<uint64_t> cset(static_cast<size_t>(fos->n) * words, 0), forbid;
    std::vector<int32_t> vmark(fos->n, -1);
    for (int64_t t = 0; t < m; ++t) {
        const int32_t j = order[t];
        forbid.assign(words, 0);
        auto take = [&](int32_t v) {
            if (vmark[v] == j) return;
            vmark[v] = j;
            const uint64_t *cs = cset.data() + static_cast<size_t>(v) * words;
            for (int64_t x = 0; x < words; ++x) forbid[x] |= cs[x];
        };
        for (int64_t q = fos->eptr[j]; q < fos->eptr[j + 1]; ++q) {
            const int32_t u = fos->evars[q];
            take(u);
            for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; ++e) take(g->col[e]);
        }
        int32_t c = 0;
        while (c < k && ((forbid[c >> 6] >> (c & 63)) & 1u)) ++c;
        if (c == k) ++k;
        if (k > 64 * words) { // re-stride the bitsets to twice the words
            std::vector<uint64_t> wider(static_cast<size_t>(fos->n) * 2 * words, 0);
            for (int64_t v = 0; v < fos->n; ++v)
                for (int64_t x = 0; x < words; ++x) wider[static_cast<size_t>(v) * 2 * words + x] = cset[v * words + x];
            cset.swap(wider);
            words *= 2;
        }
        color[j] = c;
        for (int64_t q = fos->eptr[j]; q < fos->eptr[j + 1]; ++q)
            cset[static_cast<size_t>(fos->evars[q]) * words + (c >> 6)] |= uint64_t(1) << (c & 63);
    }

    fos->k = k;
    fos->color_of = std::move(color);
    fos->cptr.assign(static_cast<size_t>(k) + 1, 0);
    for (int64_t j = 0; j < m; ++j) fos->cptr[fos->color_of[j] + 1]++;
    for (int32_t c = 0; c < k; ++c) fos->cptr[c + 1] += fos->cptr[c];
    fos->celems.resize(m);
    std::vector<int64_t> fill(fos->cptr.begin(), fos->cptr.end() - 1);
    for (int64_t j = 0; j < m; ++j) fos->celems[fill[fos->color_of[j]]++] = static_cast<int32_t>(j);
    return GOM_OK;
}

int64_t count_deps(const gom_graph_t *g, const gom_fos &fos)
{
    int64_t total = 0;
    for (int32_t v : fos.evars) total += g->row_ptr[v + 1] - g->row_ptr[v];
    return total;
}

int build_elem_tables(const gom_graph_t *g, const gom_fos &fos, ElemTables *out)
{
    const int64_t m = fos.m;
    if (fos.k < 0 || static_cast<int64_t>(fos.celems.size()) != m) return GOM_E_NOT_COLORED;
    // offsets in colour order
    std::vector<int64_t> f0(m + 1, 0);
    for (int64_t q = 0; q < m; ++q) {
        const int32_t j = fos.celems[q];
        f0[q + 1] = f0[q] + (fos.eptr[j + 1] - fos.eptr[j]);
    }
    const size_t total = static_cast<size_t>(f0[m]);
    out->hdr.assign(8 * static_cast<size_t>(m), 0);
    out->fv.assign(total, 0);
    out->wout.assign(total, 0);
    out->wabs.assign(total, 0);
    out->seg.assign(total + static_cast<size_t>(m), 0);
    std::vector<int64_t> d0(m + 1, 0);
    std::atomic<int> too_big{0};
    std::vector<int32_t> smax(m, 0);
    std::vector<int64_t> wabs(m, 0);
    std::vector<int64_t> nedges(m, 0);

    // pass 1: counts, segment offsets, outside weight sums
    parallel_ranges(m, [&](int64_t b, int64_t e) {
        std::vector<int32_t> pos(fos.n, -1);
        for (int64_t q = b; q < e; ++q) {
            const int32_t j = fos.celems[q];
            const int64_t e0 = fos.eptr[j], s = fos.eptr[j + 1] - e0;
            for (int64_t a = 0; a < s; ++a) pos[fos.evars[e0 + a]] = static_cast<int32_t>(a);
            uint32_t *seg = out->seg.data() + f0[q] + q;
            int64_t n_out = 0, n_in = 0, sum_abs = 0;
            for (int64_t a = 0; a < s; ++a) {
                const int32_t u = fos.evars[e0 + a];
                out->fv[f0[q] + a] = u;
                seg[a] = static_cast<uint32_t>(n_out);
                int64_t wsum = 0, wab = 0;
                for (int64_t x = g->row_ptr[u]; x < g->row_ptr[u + 1]; ++x) {
                    const int32_t bb = pos[g->col[x]];
                    const int64_t w = g->weight[x];
                    if (bb < 0) {
                        ++n_out;
                        wsum += w;
                        wab += w < 0 ? -w : w;
                        sum_abs += w < 0 ? -w : w;
                    } else if (bb > a) {
                        ++n_in;
                        sum_abs += w < 0 ? -w : w;
                    }
                }
                out->wout[f0[q] + a] = wsum;
                out->wabs[f0[q] + a] = static_cast<int32_t>(std::min<int64_t>(wab, INT32_MAX));
                if (n_out > 65535) too_big = 1;
            }
            seg[s] = static_cast<uint32_t>(n_out);
            d0[q + 1] = n_out + n_in;
            int32_t *h = out->hdr.data() + 8 * q;
            h[0] = j;
            h[1] = static_cast<int32_t>(f0[q]);
            h[3] = static_cast<int32_t>(s | (n_in << 8));
            h[4] = static_cast<int32_t>(n_out);
            smax[q] = static_cast<int32_t>(s);
            wabs[q] = sum_abs;
            nedges[q] = n_out + n_in;
            for (int64_t a = 0; a < s; ++a) pos[fos.evars[e0 + a]] = -1;
        }
    });
    if (too_big) return GOM_E_LIMIT;
    for (int64_t q = 0; q < m; ++q) d0[q + 1] += d0[q];
    if (d0[m] >= (int64_t(1) << 31)) return GOM_E_LIMIT;
    out->dep.assign(2 * static_cast<size_t>(d0[m]), 0);
    out->max_s = m ? *std::max_element(smax.begin(), smax.end()) : 0;
    out->max_abs_w = m ? *std::max_element(wabs.begin(), wabs.end()) : 0;
    out->max_edges = m ? *std::max_element(nedges.begin(), nedges.end()) : 0;

    // pass 2: the edge lists
    parallel_ranges(m, [&](int64_t b, int64_t e) {
        std::vector<int32_t> pos(fos.n, -1);
        for (int64_t q = b; q < e; ++q) {
            const int32_t j = fos.celems[q];
            const int64_t e0 = fos.eptr[j], s = fos.eptr[j + 1] - e0;
            for (int64_t a = 0; a < s; ++a) pos[fos.evars[e0 + a]] = static_cast<int32_t>(a);
            out->hdr[8 * q + 2] = static_cast<int32_t>(d0[q]);
            int32_t *dst = out->dep.data() + 2 * d0[q];
            for (int64_t a = 0; a < s; ++a) { // outside edges, grouped by a
                const int32_t u = fos.evars[e0 + a];
                for (int64_t x = g->row_ptr[u]; x < g->row_ptr[u + 1]; ++x)
                    if (pos[g->col[x]] < 0) {
                        *dst++ = g->col[x];
                        *dst++ = g->weight[x];
                    }
            }
            for (int64_t a = 0; a < s; ++a) { // inside edges, once each (a < b)
                const int32_t u = fos.evars[e0 + a];
                for (int64_t x = g->row_ptr[u]; x < g->row_ptr[u + 1]; ++x) {
                    const int32_t bb = pos[g->col[x]];
                    if (bb > a) {
                        *dst++ = static_cast<int32_t>(a | (bb << 8));
                        *dst++ = g->weight[x];
                    }
                }
            }
            for (int64_t a = 0; a < s; ++a) pos[fos.evars[e0 + a]] = -1;
        }
    });
    return GOM_OK;
}

} // namespace gomh
