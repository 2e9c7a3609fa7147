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
int build_bflt(const gom_graph_t *g, int32_t bound, gom_fos *out);
int check_fos(int32_t n, const gom_fos &fos);
int color_fos(const gom_graph_t *g, gom_fos *fos);

// Per-element tables in colour order (position q = rank of the element in
// the colour-sorted element list, so a colour group is one contiguous range
// [cptr[c], cptr[c+1])).  For the element j at position q with s variables:
//   hdr[8q .. 8q+8)  = {j, f0, d0, s | (n_in << 8), n_out, 0, 0, 0}
//   fv[f0 + a]       = a-th variable of F_j (ascending)
//   wout[f0 + a]     = sum of the weights of the edges from F_j[a] to
//                      variables outside F_j
//   wabs[f0 + a]     = the same sum of their absolute values
//   seg[f0 + q + a]  = start of F_j[a]'s outside edges in dep[d0 ..], a = 0..s
//                      (seg[f0 + q + s] = n_out)
//   dep[d0 + x]      = {v, w} for the n_out outside edges grouped by a, then
//                      {a | (b << 8), w} for the n_in edges inside F_j (a < b)
// These are the dependent subfunctions of Alg. 4, each edge listed once.
struct ElemTables {
    std::vector<int32_t> hdr;     // 8 ints per element (32 bytes)
    std::vector<int32_t> fv;      // [total_vars]
    std::vector<int64_t> wout;    // [total_vars]
    std::vector<int32_t> wabs;    // [total_vars] sum of |w| over F_j[a]'s outside edges (saturated at INT32_MAX)
    std::vector<uint32_t> seg;    // [total_vars + m]
    std::vector<int32_t> dep;     // 2 ints per entry
    int32_t max_s = 0;            // largest element
    int64_t max_edges = 0;        // most edges (outside + inside) of one element
    int64_t max_abs_w = 0;        // largest sum of |w| over one element's edges
};
int64_t count_deps(const gom_graph_t *g, const gom_fos &fos); // upper bound of entries
int build_elem_tables(const gom_graph_t *g, const gom_fos &fos, ElemTables *out);

} // namespace gomh

// ----------------------------------------------------------------------------
// Device-side state and parameters.

// Kernel variants by the largest element and the element weight sums:
// narrow = elements of <= 32 variables with sums of |w| below 2^30 (32-bit
// masks and deltas), wide = <= 64 variables (64-bit masks and deltas), huge =
// 65 to GOM_MAX_ELEMENT variables (128-bit masks, 64-bit deltas; at most two
// population words per item, no learned filter).
enum : int32_t { kVarNarrow = 0, kVarWide = 1, kVarHuge = 2, kVarBits = 3 }; // kVarBits: batched instances on
                                                                          // the bit-sliced phase
inline int32_t kernel_variant(int64_t max_s, int64_t max_abs_w)
{
    if (max_s <= 32 && max_abs_w < (int64_t(1) << 30)) return kVarNarrow;
    return max_s <= 64 ? kVarWide : kVarHuge;
}

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
    int64_t cnt[4];    // counters of the running generation: donorless, accepted, improving, trials skipped
    int64_t fi_cnt[5]; // Forced Improvement counters of the running generation: individuals, trials,
                       //   accepted, improving, replaced
    int32_t fi_newel;  // per-launch path: the elitist changed at the start of FI
    int32_t pad_;
};

struct GomBarrier { // grid barrier of the persistent kernel: monotonic arrival count
    unsigned long long count;
    unsigned long long pad;
};

// One instance of a batched launch (gom_batch_*): its blocks, kernel variant
// and target; gens_run and err are filled after each call.
struct GomBatchInst {
    int32_t blk0, nblk; // its blocks [blk0, blk0 + nblk) of the launch
    int32_t wpi;        // words per item of its mixing (1, 2, 4)
    int32_t variant;    // kernel variant (kVarNarrow, kVarWide, kVarHuge; kVarBits: the bit-sliced phase)
    int64_t target;     // target fitness of the current call
    int32_t gens;       // generations of the current call for this instance
    int32_t bs_r;       // kVarBits: the width R of its plane accumulators (12 or 16)
    int32_t gens_run;   // generations run by the last call
    int32_t err;        // the instance's device error word after the last call
};

// Learned trial filter (gom_filter_*): a 16 -> 64 -> 1 MLP with bf16 weights
// that skips the trials of elements predicted to accept nothing, with
// per-element history of the last two generations and audit counters.
constexpr int kFilterIn = 16;
constexpr int kFilterHidden = 64;
enum : int { FC_RUN = 0, FC_RUN_USEFUL = 1, FC_SKIPPED = 2, FC_AUDITED = 3, FC_AUDITED_USEFUL = 4, FC_N = 5 };

struct GomFilterState {
    int32_t enabled;                   // 1 while the filter skips elements
    int32_t disabled_at;               // generation at which it turned itself off, -1 never
    float threshold;                   // skip when the logit is below it
    float min_recall;                  // estimated recall under which (two generations running) the
                                       // filter turns itself off
    float target_recall;               // the threshold follows the audits towards this recall
    int32_t low_streak;                // generations in a row below min_recall
    unsigned long long log_count;      // samples offered to the log (those past its capacity are dropped)
    unsigned long long cnt[FC_N];      // items of the running generation: run, run with an acceptance,
                                       // skipped, audited, audited with an acceptance
    unsigned long long last[FC_N];     // the same for the last finished generation
    unsigned long long total[FC_N];    // since the filter was attached
};

struct GomFilter {
    GomFilterState *st;
    uint32_t *hist;       // [2][3][m] accepted, donor-less and improving trials per element position, by g mod 2
    uint8_t *skipped;     // [m] elements (by position) skipped in the last generation
    const uint16_t *w1;   // [64][16] bf16 bits
    const float *b1;      // [64]
    const uint16_t *w2;   // [64] bf16 bits
    const float *b2;      // [1]
    uint16_t *log_x;      // [cap][16] bf16 features
    uint8_t *log_y;       // [cap] label: the item was useful (see label)
    int64_t log_cap;
    uint8_t *dirty;       // [n] 1: the variable changed in some individual during the previous generation
    uint8_t *quiet;       // [m] generations in a row (saturating at 255) an element had no accepted trial
                          //   and no change in its variables or outside neighbours
    uint8_t *dec;         // [m] the select phase's decision per position (DEC_RUN / DEC_SKIP / DEC_AUDIT)
    int32_t *act;         // [m] positions to run, in order (bit 31: audited); bit-sliced path
    int32_t *act_ptr;     // [k + 1] colour c's part of act: [act_ptr[c], act_ptr[c + 1])
    uint32_t *wcnt;       // [select warps] elements to run per select warp, then their first slots
    int32_t items_per_elem; // mixing items of one element (the unit of the filter's item counters)
    int32_t compact;      // 1: the bit-sliced mixing runs the compacted list while the filter skips
    int32_t label;        // what makes an element useful (its training label): 0 an accepted trial, 1 an
                          //   improving trial
};

struct GomDevStats { // mirrors gom_gen_stats_t
    int64_t generation, best, elite, trials, donorless, accepted, improving, reached;
    int64_t fi_individuals, fi_trials, fi_accepted, fi_improving, fi_replaced;
};

// Forced Improvement (Sec. 4, Alg. 1) after each generation's mixing, in the
// parallel reading of the library (gom_fi.cuh); arrays in the workspace.
struct GomFI {
    int32_t on;        // 1: FI after each generation's mixing
    int32_t nis;       // also individuals not improved for nis generations (0: that condition off)
    uint32_t *accw;    // [W] individuals with an accepted GOM step in the generation
    uint32_t *eq;      // [W] individuals equal to the elitist at the start of FI
    uint32_t *act0;    // [W] individuals in FI
    uint32_t *imp;     // [k][W] individuals FI improved in the group at position t
    int32_t *stale;    // [32W] generations in a row without improvement
    int64_t *f0;       // [32W] fitness at generation start
};

constexpr int kStatsCap = 1024;    // per-generation counters kept on the device
constexpr int kMixThreads = 256;   // mixing kernel block size (8 warps)
constexpr int kBsThreads = 128;    // bit-sliced kernels' block size (4 warps; 5 blocks per SM)
constexpr int kStageAllMaxK = 128; // most colour groups of the stage-all mode (group order held per block)
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
    int32_t split;      // mixing items: 0 = one warp per element, 1 = one per (element, word group)
    int32_t stage_all;  // 1: each warp stages its items of all k groups at generation start
    int32_t warp_smem;  // 32-bit words of one staging slice (one item) in the mixing phase:
    int32_t off_fv;     //   [0, 8) item header, [off_fv, ..) the element's variables,
    int32_t off_seg;    //   [off_seg, ..) their outside-edge starts (s+1), [off_wout, ..)
    int32_t off_wout;   //   their outside weight sums (int64), [off_pr, ..) the rows of P
    int32_t off_pr;     //   on F_j, [off_pat, ..) the pattern table (32 W masks),
    int32_t off_pat;    //   [off_rs, ..) its run starts (W words), [off_cw, ..) each edge's
    int32_t off_rs;     //   {code, weight}, [off_xw, ..) each outside edge's WPI parent words
    int32_t off_cw;
    int32_t off_xw;
    int32_t off_ds;     //   [off_ds, ..) donor start positions (stage-all mode only)
    int32_t dyn;        // 1: after its first item, a warp (a block in block mode) claims items from work[t]
    int32_t blk;        // block mode (128-bit instances): a block stages one element at a time into one
                        //   slice and its warps share the element's word groups
    int32_t xw_words;   // block mode: words of one warp's region of outside neighbours' words, the
                        //   regions of warps 0, 1, ... following each other from off_xw
    int32_t learn;      // learned filter: 0 off, 1 history and training log, 2 also skip elements
    GomFI fi;
    int32_t bs_sm;      // bit-sliced path: words per staged row block of one pair (>= the largest
                        //   element, odd: a lane-strided row access is free of bank conflicts)
    int32_t bs_S;       //   field width of one element in a packed pattern (the largest element)
    int32_t bs_epw;     //   elements per packed pattern word (32 / bs_S)
    int32_t bs_nc;      //   packed words per individual for one item (ceil(E / bs_epw), E = 32 / W)
    int32_t bs_words;   //   shared-memory words of one warp's region
    GomFilter flt;
    uint64_t seed;
    uint32_t rk[20];   // Philox round keys of the seed: rk[2r], rk[2r+1] = the key after r bumps
    uint32_t *O;       // [n][W] offspring, bit-sliced: bit b of O[v][w] = x_v of 32w+b
    uint32_t *P;       // [n][W] generation-start population
    int64_t *f;        // [32W] fitness
    uint32_t *eqw;     // [2][W] flags P[i] == x_e of generation g in buffer g mod 2
    uint8_t *xe;       // [n] elitist
    GomDevState *st;
    GomBarrier *bar;
    unsigned long long *trace; // [5 + 2k] phase stamps of k_run, or null (off)
    GomDevStats *stats;  // [kStatsCap] ring indexed by generation
    int32_t *order;      // [k] colour visited at position t
    uint32_t *work;      // [k] item claim counters of the colour-group positions
    const int64_t *row_ptr;
    const int32_t *col;
    const int32_t *wgt;
    const int4 *hdr;         // [2m] element headers in colour order: {j, f0, d0, s | n_in << 8}, {n_out, 0, 0, 0}
    const int32_t *fv;       // [total_vars]
    const int64_t *wout;     // [total_vars]
    const int32_t *wabs;     // [total_vars] sum of |w| over each variable's outside edges
    const uint32_t *seg;     // [total_vars + m]
    const int2 *dep;         // outside edges {v, w}, then inside edges {a | b << 8, w}
    const int32_t *cptr;     // [k+1] colour -> positions
};
