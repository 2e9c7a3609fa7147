// gom_internal.h -- data structures shared by the library's translation units
// (host set-up code, kernels and the C ABI).  Not installed; include/gom.h is
// the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <vector_types.h>

#include "../../include/gom.h"

// Linkage model (FOS, Sec. 4.1) and its colouring (Sec. 5.2), host side.
struct gom_fos {
    int32_t n = 0;                 // variables (graph vertices)
    int64_t m = 0;                 // elements
    std::vector<int64_t> eptr;     // [m+1]
    std::vector<int32_t> evars;    // ascending within each element
    int32_t k = -1;                // colours, -1 until coloured
    std::vector<int32_t> color_of; // [m]
    std::vector<int64_t> cptr;     // [k+1]
    std::vector<int32_t> celems;   // elements of each colour, ascending
};

namespace gomh {

// Host set-up steps (gom_host.cpp).
int validate_graph(const gom_graph_t *g);
int build_fos(const gom_graph_t *g, int32_t kind, gom_fos *out);
int check_fos(int32_t n, const gom_fos &fos);
int color_fos(const gom_graph_t *g, gom_fos *fos);

// Per-element dependency lists: the edges incident to F_j (Alg. 4's
// dependent subfunctions), grouped by the F-local index a of the endpoint in
// F_j, each edge listed once.  Entry = {code, weight}: code >= 0 is the other
// endpoint (outside F_j); code < 0 is -1 - b with b the F-local index of the
// other endpoint (inside F_j, b > a).  seg holds, per element, s+1 offsets
// (relative to dep_ptr[j]) at seg[eptr[j] + j + a].
struct DepTables {
    std::vector<int64_t> dep_ptr; // [m+1]
    std::vector<int32_t> dep;     // 2 ints per entry: code, weight
    std::vector<uint16_t> seg;    // [total_vars + m]
};
int64_t count_deps(const gom_graph_t *g, const gom_fos &fos); // upper bound of entries
int build_deps(const gom_graph_t *g, const gom_fos &fos, DepTables *out);

} // namespace gomh

// ----------------------------------------------------------------------------
// Device-side state and parameters.

struct GomDevState {
    uint32_t g;        // generation counter
    int32_t done;      // a generation of the current call reached the target
    int64_t target;    // target fitness of the current call
    int64_t fe;        // elitist fitness
    int32_t improved;  // elitist changed; x_e still to be copied from O[argmax]
    int32_t argmax;    // individual holding the new elitist
    int64_t best;      // best fitness after the last generation
    int32_t err;       // device-side error word (0 = none)
    uint32_t call_g0;  // generation counter at the start of the current call
    int64_t cnt[4];    // counters of the running generation: donorless, accepted, improving
};

struct GomDevStats { // mirrors gom_gen_stats_t
    int64_t generation, best, elite, trials, donorless, accepted, improving, reached;
};

constexpr int kStatsCap = 1024;    // per-generation counters kept on the device
constexpr int kMixThreads = 256;   // mixing kernel block size (8 warps)
constexpr uint32_t kTagInit = 0x494E4954u;
constexpr uint32_t kTagDonor = 0x444F4E52u;
constexpr uint32_t kTagOrder = 0x4F524452u;

struct GomParams {
    int32_t n;         // variables
    int32_t p;         // individuals
    int32_t W;         // words per variable row (power of two >= ceil(p/32))
    int32_t Wv;        // words holding valid individuals, ceil(p/32)
    int32_t m;         // FOS elements
    int32_t k;         // colours
    int32_t pad0, pad1;
    uint64_t seed;
    uint32_t *O;       // [n][W] offspring, bit-sliced: bit b of O[v][w] = x_v of 32w+b
    uint32_t *P;       // [n][W] generation-start population
    int64_t *f;        // [32W] fitness
    uint32_t *eqw;     // [W] generation-start flags P[i] == x_e
    uint8_t *xe;       // [n] elitist
    GomDevState *st;
    GomDevStats *stats;  // [kStatsCap] ring indexed by generation
    int32_t *order;      // [k] colour visited at position t
    const int64_t *row_ptr;
    const int32_t *col;
    const int32_t *wgt;
    const int32_t *eptr;   // [m+1]
    const int32_t *evars;
    const int64_t *dep_ptr;  // [m+1]
    const int2 *dep;         // {code, weight}
    const uint16_t *seg;     // [total_vars + m]
    const int32_t *cptr;     // [k+1]
    const int32_t *celems;   // [m]
};
