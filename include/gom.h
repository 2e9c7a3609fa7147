/*
 * gom.h -- C ABI of the GB300 parallel Gene-pool Optimal Mixing (GOM) library
 * for weighted Max-Cut.
 *
 * The method is parallel GOMEA of Bouter & Bosman, "GPU-Accelerated Parallel
 * Gene-pool Optimal Mixing in a Gray-Box Optimization Setting" (arXiv
 * 2203.08680): a population of binary solutions is improved generation by
 * generation; in each generation the elements of the linkage model (FOS,
 * Sec. 4.1) are split into colour groups of mutually independent elements
 * (Sec. 5.2), the groups are visited in random order (Alg. 3), and every
 * (individual, element) pair of a group is one GOM trial (Alg. 2): copy a
 * donor's bits on the element, take the cut-weight change by partial
 * evaluation (Sec. 2.2, Alg. 4) and keep the change unless it makes the
 * solution worse.
 *
 * Conventions for every call:
 *  - Return value: GOM_OK (0) or a negative GOM_E_* code; gom_strerror() names it.
 *  - Host pointers are read during the call only and stay owned by the caller.
 *  - Device memory is never allocated by the library: the caller passes one
 *    device workspace (sized by gom_workspace_bytes) to gom_init_population
 *    and device output buffers to the export calls.
 *  - Device work is enqueued on the caller's CUDA stream given at
 *    gom_init_population; a call returns before that work finishes unless it
 *    says otherwise.  Handles are not thread-safe.
 *  - Integer arithmetic throughout: int32 edge weights, int64 fitness.  Results
 *    are bit-exact and reproducible from (graph, FOS, population size, seed).
 *
 * Random numbers are Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) with
 * key (seed low 32 bits, seed high 32 bits) and these counters:
 *  - initial bit v of individual i: bit (v mod 32) of word (v/32 mod 4) of
 *    ctr (v/128, i, 0, 0x494E4954);
 *  - group order of generation g: colours sorted ascending by the 64-bit key
 *    (word0 << 32 | word1) of ctr (colour, 0, g, 0x4F524452), ties by colour;
 *  - donor of trial (individual i, element j) in generation g: r = word (i mod 4)
 *    of ctr (j, i/4, g, 0x444F4E52); start = (i + 1 + floor(r (p-1) / 2^32)) mod p;
 *    the donor is the first individual, scanning cyclically upwards from start
 *    and skipping i, whose generation-start bits on the element differ from
 *    the parent's current bits (no such individual: the trial is skipped).
 */
#ifndef GOM_H_
#define GOM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define GOM_OK 0
#define GOM_E_ARG (-1)          /* null pointer, population < 2, unknown kind, ... */
#define GOM_E_GRAPH (-2)        /* CSR not a simple symmetric graph with sorted rows */
#define GOM_E_NOT_COLORED (-3)  /* gom_color_fos has not run on this FOS */
#define GOM_E_WORKSPACE (-4)    /* workspace null, misaligned or too small */
#define GOM_E_CUDA (-5)         /* a CUDA call failed; gom_last_cuda_error has it */
#define GOM_E_TIMEOUT (-6)      /* a bounded device wait gave up; the population is then undefined
                                   until gom_set_population or a new gom_init_population */
#define GOM_E_STATE (-7)        /* call not valid in the handle's state */
#define GOM_E_LIMIT (-8)        /* size beyond what the library supports */
#define GOM_E_FOS (-9)          /* FOS incomplete, out of range or for another graph */

/* FOS kinds for gom_build_fos. */
#define GOM_FOS_NEIGHBOURHOOD 0 /* F_j = {j} u adj(j), one element per vertex */
#define GOM_FOS_SINGLETON 1     /* F_j = {j} */
#define GOM_FOS_BFLT 2          /* bounded fixed linkage tree: UPGMA on the edge weights, sets of
                                   at most `param` variables (Sec. 4.1) */

/* Options for gom_set_option / gom_get_option. */
#define GOM_OPT_PERSISTENT 1 /* 1: each gom_generation call is one persistent cooperative
                                kernel that runs all its generations, phases separated by
                                bounded grid barriers (default where the device supports
                                cooperative launch); 0: one CUDA graph per generation with one
                                kernel per phase and per colour group */

#define GOM_OPT_PHASE_TRACE 2 /* 1: the persistent kernel records wall-clock stamps (ns) of
                                 the phase boundaries of each generation, read with
                                 gom_read_phase_trace; 0 (default): off */

#define GOM_OPT_DYNAMIC 3 /* item schedule inside a colour group: 0 = static stride (warp w
                             takes items w, w + nwarps, ...); 1 = each warp takes item w,
                             then claims further items from a per-group counter (faster
                             warps take more; the default).  Same results either way */

#define GOM_OPT_BITSLICED 4 /* mixing on bit-planes: each lane owns 32 individuals of one element and
                               takes the partial evaluation, the acceptance and the fitness
                               bookkeeping as bit-plane arithmetic on them (one logic instruction
                               works on 32 trials); the donor search stays per individual.
                               Available for elements of at most 32 variables, |w| <= 255 and
                               element weight sums (of |w| over their edges) below 2^16; the
                               default where available, a variable row has at most 16 words
                               (p <= 512) and the largest colour group gives at least a quarter
                               of the resident warps an item (GOM_E_STATE when set to 1 where
                               unavailable).  Same results either way; the learned filter works
                               on both.  A batched launch follows the value the caller set for
                               the context, else the same rule on the warps the instance gets
                               (bit-sliced instances only with min_blocks 2) */

#define GOM_OPT_FORCED_IMPROVEMENT 5 /* 1: Forced Improvement (Sec. 4, Alg. 1) after each generation's
                                        mixing, in this library's parallel reading (the paper's
                                        parallel GOMEA runs without it, Sec. 5.4): the elitist is
                                        first updated from the population; every individual without
                                        an accepted GOM step in the generation (see GOM_OPT_FI_NIS)
                                        then takes GOM steps with the elitist as donor on the
                                        elements of each colour group, groups in the generation's
                                        order, accepted as in Alg. 2 with "equal to the elitist"
                                        taken at the start of FI; it leaves FI after the first group
                                        in which a step improved its fitness, and one that no step
                                        improved becomes a copy of the elitist.  0 (default): off.
                                        GOM_E_LIMIT where |w| > 255 or an element's sum of |w| over
                                        its edges reaches 2^16; not available in batched launches */

#define GOM_OPT_FI_NIS 6 /* Forced Improvement also for individuals whose fitness has not improved
                            for this many generations, the current one included (0, the default:
                            only individuals without an accepted step) */

#define GOM_OPT_FILTER_LABEL 7 /* learned trial filter: what makes an element's trials of a
                                  generation useful -- its training label and the unit of its
                                  recall estimate: 0 (default) an accepted trial, 1 an improving
                                  trial (a strictly better fitness) */

/* Supported maxima of the library. */
#define GOM_MAX_POPULATION 1024 /* individuals */
#define GOM_MAX_ELEMENT 128     /* variables in one FOS element (the paper's largest
                                   linkage-tree bound, Sec. 6.1, is 100) */
#define GOM_MAX_COLORS 28000    /* colour groups */

/*
 * Weighted undirected graph in symmetric CSR form (Sec. 6.2: the Max-Cut
 * instance, which is also the variable interaction graph of Sec. 2.3).
 * row_ptr[num_vertices+1] (int64, row_ptr[0] = 0, row_ptr[n] = num_adj),
 * col[num_adj] and weight[num_adj]; each undirected edge {u,v} appears as
 * (u,v,w) and (v,u,w); rows sorted strictly ascending; no self-loops.  Host
 * memory, caller-owned, read during the call.  Any int32 weight is allowed.
 */
typedef struct gom_graph {
    int32_t num_vertices;
    int64_t num_adj;
    const int64_t *row_ptr;
    const int32_t *col;
    const int32_t *weight;
} gom_graph_t;

typedef struct gom_fos gom_fos_t; /* linkage model + colouring (host, library-owned) */
typedef struct gom_ctx gom_ctx_t; /* one population on one GPU (library-owned) */

/* Counters of one generation. */
typedef struct gom_gen_stats {
    int64_t generation;     /* index g of the generation (0 = first after init) */
    int64_t best_fitness;   /* max_i f[i] at its end */
    int64_t elite_fitness;  /* fitness of the elitist at its end */
    int64_t trials;         /* (individual, element) trials made: p * m, less those a learned
                               filter skipped; donor-less ones included */
    int64_t donorless;      /* trials with no donor differing on the element */
    int64_t accepted;       /* trials whose change was kept */
    int64_t improving;      /* accepted trials with a positive delta */
    int64_t reached_target; /* 1 if best_fitness >= the call's target */
    /* Forced Improvement (GOM_OPT_FORCED_IMPROVEMENT; zero while off): */
    int64_t fi_individuals; /* individuals that entered FI */
    int64_t fi_trials;      /* their (individual, element) steps, those without variation included */
    int64_t fi_accepted;    /* FI steps whose change was kept */
    int64_t fi_improving;   /* accepted FI steps with a positive delta */
    int64_t fi_replaced;    /* individuals FI did not improve, replaced by a copy of the elitist */
} gom_gen_stats_t;

/*
 * Builds the linkage model (FOS, Sec. 4.1) of a graph.  kind is
 * GOM_FOS_NEIGHBOURHOOD (element j = {j} u adj(j), variables ascending),
 * GOM_FOS_SINGLETON (param 0 for both), or GOM_FOS_BFLT with param = the
 * largest linkage set (>= 1).  GOM_FOS_BFLT is the paper's model (Sec. 4.1,
 * used for every GOMEA version in Sec. 6.1): a fixed linkage tree learned once
 * by UPGMA with the edge weights as similarity -- from the singletons,
 * repeatedly merge the two clusters of highest average pairwise weight,
 * sum over u in A, v in B of w_uv divided by |A||B| -- bounded: a merge above
 * param variables is never made.  Readings: only clusters joined by an edge
 * are merged (the tree stops when none fits the bound), the set of all
 * variables is left out (Sec. 4.1), ties go to the pair of smaller creation
 * ids (singletons 0..n-1, then merges in order).  Elements: the n
 * singletons, then the merged sets in creation order, variables ascending.
 * The mixing kernels take elements of up to GOM_MAX_ELEMENT variables (the
 * paper's bounds of 10 and 100 both fit).  Validates the graph (GOM_E_GRAPH).  *out receives a handle to free with
 * gom_fos_destroy.
 */
int gom_build_fos(const gom_graph_t *g, int32_t kind, int32_t param, gom_fos_t **out);

/*
 * Wraps a caller-given FOS over num_vars variables: m elements, element j =
 * elem_vars[elem_ptr[j] .. elem_ptr[j+1]), each ascending without repeats.  The
 * FOS must be complete (Sec. 4.1: every variable in some element), else
 * GOM_E_FOS.  Arrays are copied.  Elements above GOM_MAX_ELEMENT variables are
 * accepted here and rejected by gom_init_population with GOM_E_LIMIT.
 */
int gom_fos_create(int32_t num_vars, int64_t m, const int64_t *elem_ptr,
                   const int32_t *elem_vars, gom_fos_t **out);

/*
 * Colours the linkage-model interaction graph (LMIG, Sec. 5.2: elements i and j
 * are joined iff they share a variable or a graph edge joins them) with the
 * greedy Welsh-Powell algorithm: elements by LMIG degree descending, ties by
 * ascending index, each given the smallest colour unused by its coloured
 * neighbours.  The LMIG is never materialised.  Stores the colouring in fos
 * and writes the number of colours k to *num_colors.  Host-only work.
 */
int gom_color_fos(const gom_graph_t *g, gom_fos_t *fos, int32_t *num_colors);

/* Sizes of a FOS: elements m, total variables over all elements, colours k
 * (-1 if not coloured).  Any output pointer may be NULL. */
int gom_fos_sizes(const gom_fos_t *fos, int64_t *m, int64_t *total_vars, int32_t *k);

/*
 * Copies a FOS and its colouring into caller-sized host arrays (any may be
 * NULL): elem_ptr[m+1], elem_vars[total_vars], color_of_elem[m],
 * color_ptr[k+1], color_elems[m] (the elements of colour c, ascending, are
 * color_elems[color_ptr[c] .. color_ptr[c+1])).  Colour arrays need a coloured
 * FOS (GOM_E_NOT_COLORED).
 */
int gom_fos_export(const gom_fos_t *fos, int64_t *elem_ptr, int32_t *elem_vars,
                   int32_t *color_of_elem, int64_t *color_ptr, int32_t *color_elems);

void gom_fos_destroy(gom_fos_t *fos);

/*
 * Bytes of device workspace gom_init_population needs for this graph, FOS
 * and population size (0 on invalid arguments).  The workspace must be
 * 256-byte aligned.
 */
size_t gom_workspace_bytes(const gom_graph_t *g, const gom_fos_t *fos, int32_t pop);

/*
 * InitializePopulation (Alg. 3): validates and uploads the graph, the coloured
 * FOS and its per-element dependency lists (the edges incident to each
 * element, Alg. 4) into d_workspace, draws the population uniformly at random
 * with Philox (counters above), evaluates it fully (Sec. 6.2) and takes the
 * elitist (lowest index of maximal fitness).  pop in [2, GOM_MAX_POPULATION].
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).  d_workspace
 * (caller-owned device memory of ws_bytes >= gom_workspace_bytes) must outlive
 * the handle.  Synchronises the stream before returning.
 */
int gom_init_population(const gom_graph_t *g, const gom_fos_t *fos, int32_t pop, uint64_t seed,
                        void *d_workspace, size_t ws_bytes, void *cuda_stream, gom_ctx_t **out);

/*
 * Runs up to num_generations generations of parallel GOMEA (Alg. 3): P <- O;
 * the elitist flag of each individual (P[i] equals the elitist); the colour
 * groups in random order, each group one mixing launch over all its
 * (individual, element) trials (donor, partial evaluation, accept, write);
 * then the fitness fold, the elitist update (if max f beats it) and the
 * counters.  Stops after the first generation whose best fitness is >=
 * target_fitness (INT64_MAX: never).  With host_stats (an array of
 * num_generations entries) or generations_run non-NULL the call waits for the
 * stream and fills them (entries past the stop are zeroed); otherwise it only
 * enqueues.  The generation counter lives in the handle, so split calls
 * reproduce one long call exactly.
 */
int gom_generation(gom_ctx_t *ctx, int32_t num_generations, int64_t target_fitness,
                   gom_gen_stats_t *host_stats, int32_t *generations_run);

/* Full re-evaluation (Sec. 6.2) of the current population into the caller's
 * device buffer d_fitness_out[pop] (int64).  Enqueued only. */
int gom_fitness(gom_ctx_t *ctx, int64_t *d_fitness_out);

/*
 * Exports the current population as uint8 {0,1} rows d_pop[pop][num_vertices]
 * and its fitness d_fit[pop] (device buffers, either may be NULL), and writes
 * the elitist's fitness to *elite_f (host, may be NULL; waits for the stream).
 */
int gom_get_population(gom_ctx_t *ctx, uint8_t *d_pop, int64_t *d_fit, int64_t *elite_f);

/* Exports the elitist solution as uint8 d_elite[num_vertices] (device) and its
 * fitness (host, may be NULL; waits for the stream). */
int gom_get_elite(gom_ctx_t *ctx, uint8_t *d_elite, int64_t *elite_f);

/*
 * Replaces the state (checkpoint resume): population d_pop[pop][num_vertices]
 * (uint8 {0,1}, device), elitist d_elite[num_vertices] (device) with fitness
 * elite_f, and the generation counter.  Fitness is re-evaluated on the device.
 */
int gom_set_population(gom_ctx_t *ctx, const uint8_t *d_pop, const uint8_t *d_elite,
                       int64_t elite_f, int64_t generation);

/* Current generation counter (generations run since init or the last set). */
int gom_get_generation(gom_ctx_t *ctx, int64_t *generation);

/*
 * Kernel timing.  gom_set_timing(ctx, 1) makes each following generation
 * run on the per-generation graph path and record a CUDA event pair around
 * every mixing launch (event-record nodes in the graph; off by default).  A timed generation's events are
 * read when the next timed generation is enqueued or by gom_read_timing,
 * which waits for the stream and returns the summed mixing-kernel
 * milliseconds and the number of mixing launches run since timing was enabled
 * or last read.
 */
int gom_set_timing(gom_ctx_t *ctx, int32_t enable);
int gom_read_timing(gom_ctx_t *ctx, double *mix_ms, int64_t *mix_launches);

/* Kernel launches one generation makes on the current path (for launch
 * accounting; the persistent path counts its one launch per call as one). */
int gom_launches_per_generation(gom_ctx_t *ctx, int64_t *launches);

/* Sets or reads an option (GOM_OPT_*).  GOM_OPT_PERSISTENT = 1 is refused
 * with GOM_E_STATE where the persistent path is unavailable.  Both paths give
 * identical results. */
int gom_set_option(gom_ctx_t *ctx, int32_t option, int64_t value);
int gom_get_option(gom_ctx_t *ctx, int32_t option, int64_t *value);

/*
 * Phase trace of the last generation run on the persistent path with
 * GOM_OPT_PHASE_TRACE on: 5 + 2k wall-clock stamps (%globaltimer, ns), taken
 * by block 0: [0] generation start, [1] end of the start/order phase, [2]
 * end of the staging of every group's items (stage-all mode, used when every
 * colour group fits one wave of warps; otherwise no staging happens there),
 * [3] after the barrier that opens the generation (and, with the learned
 * filter on, after its select phase), then for each
 * colour-group position t: [4+2t] when the group starts (after its barrier
 * for t > 0), [5+2t] when block 0 finished its share of the group; [4+2k]
 * after the barrier that closes the generation.  ns[capacity] host array; *count receives 5 + 2k (GOM_E_ARG if
 * capacity is smaller).  Waits for the stream.
 */
int gom_read_phase_trace(gom_ctx_t *ctx, int64_t *ns, int32_t capacity, int32_t *count);

/*
 * Self-test of the bounded wait in the persistent kernel's grid barrier
 * (failure detection without a hang): `blocks` co-resident blocks meet at a
 * barrier that expects blocks + extra arrivals.  With extra = 0 they pass;
 * with extra > 0 no block is released, each gives up after limit_ns
 * nanoseconds of wall clock and the kernel returns.  *timed_out reports
 * whether the error word was set.  d_scratch: caller-owned device memory of
 * at least 64 bytes, 16-byte aligned.  Waits for cuda_stream.
 */
int gom_selftest_barrier(void *d_scratch, int32_t blocks, int32_t extra, int64_t limit_ns, void *cuda_stream,
                         int32_t *timed_out);

/*
 * Largest problem of gom_fitness_noalloc: num_vertices * W words, W the
 * smallest power of two with 32 W >= pop.  The scratch array behind it,
 * 4 Mi words = 16 MiB, is held by every GPU that loads this library until
 * the process exits.
 */
#define GOM_NOALLOC_MAX_WORDS (4 * 1024 * 1024)

/*
 * Full fitness (cut weight) of every individual of a caller-given population,
 * without allocating any device memory -- for callers that must not allocate:
 * cudaMalloc can synchronise the device and can fail under memory pressure,
 * and some host programs hand out all device memory through their own
 * allocator.  It does the same evaluation as gom_fitness but needs no handle
 * or workspace: its scratch (the population packed 32 individuals per word)
 * is a fixed array inside the library.  The paper has no counterpart; it is
 * an interface convenience.
 *   d_row_ptr[num_vertices+1] (int64), d_col, d_weight (int32): the graph's
 *     symmetric CSR in device memory, as in gom_graph_t (not validated here);
 *   d_pop[pop][num_vertices]: uint8 {0,1} rows, device;
 *   d_fitness_out[pop]: int64, device, overwritten.
 * Enqueued on cuda_stream (NULL = legacy default stream).  Returns
 * GOM_E_LIMIT if num_vertices * W > GOM_NOALLOC_MAX_WORDS or
 * pop > GOM_MAX_POPULATION, GOM_E_ARG if any pointer is null (d_col and
 * d_weight included, even for a graph without edges) or a size is not
 * positive.  The first call in a CUDA context (once per device in the usual
 * case of its primary context; again after cudaDeviceReset, or in a context
 * the caller made current itself) looks up the scratch array's device
 * address in that context; make that first call before any stream capture.
 * With no context current on the calling thread, the current device's
 * primary context is made current.  All calls share the one scratch array,
 * which keeps the last call's contents (every call rewrites the part it
 * reads): calls that overlap on the GPU, on different streams or threads,
 * race.
 */
int gom_fitness_noalloc(const int64_t *d_row_ptr, const int32_t *d_col, const int32_t *d_weight,
                        int32_t num_vertices, const uint8_t *d_pop, int32_t pop, int64_t *d_fitness_out,
                        void *cuda_stream);

/* Last CUDA error code seen by the handle (0 if none). */
int gom_last_cuda_error(gom_ctx_t *ctx);

/* ---------------------------------------------------------------------------
 * Batched GOM: many independent instances in one persistent launch.
 *
 * The paper runs one problem at a time (Sec. 6); a small instance then leaves
 * most of the GPU idle, and its experiments show the GPU gaining little on
 * small graphs (Sec. 6.3).  A batch runs several contexts made by
 * gom_init_population in one cooperative launch: each instance gets its own
 * range of blocks, its own grid barrier and its own target, and goes through
 * exactly the generations (Alg. 3) that gom_generation would run for it --
 * the same population, fitness, elitist and counters bit for bit, whatever
 * the batch configuration.  Instances never wait for one another.  The paper
 * has no batched form.
 */
typedef struct gom_batch gom_batch_t;

typedef struct gom_batch_config {
    int32_t warps_per_block; /* 1, 2, 4 or 8 */
    int32_t min_blocks;      /* register budget: 2 (128 registers a thread, no spills) or 3 (85) */
    int32_t max_blocks;      /* most blocks of the launch (0: every block that can be resident) */
    int32_t item_cost;       /* block allocation: a warp's time for one element is taken as
                                item_cost + (population words) x (variables + edges), so
                                item_cost is the fixed cost of an item (staging, draws,
                                memory round trips); 0 means 300 */
} gom_batch_config_t;

/* Device bytes of a batch of `num` instances (their parameter blocks, the
 * instance table and one barrier counter each). */
size_t gom_batch_workspace_bytes(int32_t num);

/*
 * A batch over ctxs[0..num) (num >= 1, each context at most once), all made
 * on cuda_stream on the current device; cfg NULL means {4, 3, 0, 0}.  Blocks go
 * to instances in proportion to their estimated time per generation (the
 * item_cost model; at least one each, at most what their largest colour group
 * can use).  d_workspace:
 * caller-owned device memory of gom_batch_workspace_bytes(num) bytes,
 * 256-byte aligned.  The contexts stay the caller's, must outlive the batch
 * and can still be used on their own.  GOM_E_LIMIT if the device cannot hold
 * one block per instance at once or an element does not fit the
 * configuration's shared memory; GOM_E_STATE without cooperative launch.
 */
int gom_batch_create(gom_ctx_t *const *ctxs, int32_t num, const gom_batch_config_t *cfg, void *d_workspace,
                     size_t ws_bytes, void *cuda_stream, gom_batch_t **out);

/*
 * Up to num_generations generations of every instance in one launch;
 * instance b stops after the first generation whose best fitness reaches
 * targets[b] (host array, or NULL for no target).  generations_run (host
 * [num], or NULL for an asynchronous call) receives the generations each
 * instance ran; the call then waits for the stream.  GOM_E_TIMEOUT if the
 * grid-barrier wait of any instance timed out (that context's error is
 * sticky).
 */
int gom_batch_generation(gom_batch_t *batch, int32_t num_generations, const int64_t *targets,
                         int32_t *generations_run);

/* As gom_batch_generation, with a generation count per instance:
 * num_generations[b] (host [num], each >= 0) for instance b. */
int gom_batch_generation_each(gom_batch_t *batch, const int32_t *num_generations, const int64_t *targets,
                              int32_t *generations_run);

/* ---------------------------------------------------------------------------
 * Learned trial filter (not in the paper).  A small MLP -- 16 features of an
 * FOS element, 64 ReLU units, one logit; bf16 weights, fp32 accumulation --
 * trained on accept/reject samples that GOM itself logs, skips the trials of
 * elements predicted to accept nothing.  Every change that is kept is still
 * decided by the exact integer partial evaluation of Alg. 2; skipping only
 * removes trials.  One in 16 elements the filter would skip is run anyway (an
 * audit).  From the audits each generation estimates the recall (useful
 * elements run / all useful ones); the skip threshold steps down while the
 * estimate is under target_recall and up while it is well over it, and when
 * it stays under min_recall for two generations the filter turns itself off
 * and the run goes on as plain GOM.  Features of element j in generation g: its size,
 * outside and inside edge counts, its accepted, donor-less and improving
 * trials of generation g-1 (fractions of p), whether it accepted none or had no
 * donor at all, log2(1+g), the population's accept, improve and donor-less
 * rates of generation g-1, and a constant.
 *
 * Modes: 0 off (plain GOM); 1 history and training log (results identical to
 * plain GOM); 2 also skip.  Mode 2 is not available to a context whose
 * persistent path stages all groups at once (small problems): GOM_E_STATE.
 */
typedef struct gom_filter_train {
    int64_t samples;      /* logged samples trained on */
    int64_t useful;       /* of which accepted at least one trial */
    double loss;          /* mean weighted logistic loss of the last epoch */
    float threshold;      /* logit below which an element is skipped */
    double skip_fraction; /* of the logged samples below the threshold */
    double recall;        /* useful logged samples at or above the threshold */
} gom_filter_train_t;

typedef struct gom_filter_stats {
    int32_t mode, enabled, disabled_at; /* disabled_at: generation the filter turned itself off, -1 never */
    float threshold;
    int64_t log_count;                  /* samples offered to the log */
    int64_t last[5];                    /* last generation's items: run, run useful, skipped, audited, audited useful */
    int64_t total[5];                   /* the same since attach */
} gom_filter_stats_t;

/* Device bytes of the filter state: per-element history (24 bytes per element),
 * the MLP and its optimiser, and a training log of log_capacity samples (38 bytes each). */
size_t gom_filter_workspace_bytes(gom_ctx_t *ctx, int64_t log_capacity);

/* Attaches caller-owned device memory (256-byte aligned) as the filter state; mode 0. */
int gom_filter_attach(gom_ctx_t *ctx, void *d_workspace, size_t ws_bytes, int64_t log_capacity);

/* Mode 0, 1 or 2 (above).  Waits for the stream.  GOM_E_LIMIT for modes 1
 * and 2 when the FOS has an element of more than 64 variables (the filter's
 * kernel instances take elements of up to 64). */
int gom_filter_set_mode(gom_ctx_t *ctx, int32_t mode);

/* Skip threshold (logit), the recall the threshold follows, and the recall
 * under which the filter turns itself off (defaults after attach: none, 0.9, 0.5). */
int gom_filter_configure(gom_ctx_t *ctx, float threshold, float target_recall, float min_recall);

/*
 * Trains the MLP from scratch on the logged samples: `epochs` full-batch Adam
 * steps on the logistic loss with positive samples weighted by pos_weight
 * (hand-written kernels; weights initialised from `seed`), then sets the
 * threshold to the largest logit that keeps target_recall of the useful
 * logged samples (and target_recall as the recall the threshold follows).
 * The log is a ring: it holds the latest log_capacity samples.  *out (may be
 * NULL) reports it.  GOM_E_STATE with an empty
 * log.  Waits.
 */
int gom_filter_train(gom_ctx_t *ctx, int32_t epochs, float learning_rate, float pos_weight, float target_recall,
                     uint64_t seed, gom_filter_train_t *out);

int gom_filter_stats(gom_ctx_t *ctx, gom_filter_stats_t *out);

/* ---- Inspection and stepwise training of the filter's MLP.
 * Parameters, as one fp32 vector theta of GOM_FILTER_PARAMS values: W1 [64][16]
 * (unit h, feature k at 16 h + k), b1 [64], W2 [64], b2 [1], in that order.
 * The mixing kernels and the logits read W1 and W2 rounded to bf16. */
#define GOM_FILTER_PARAMS 1153

/* Copies theta, the Adam moments and the gradient of the last training step
 * (each GOM_FILTER_PARAMS floats, host; any may be NULL).  Waits. */
int gom_filter_get_params(gom_ctx_t *ctx, float *theta, float *adam_m, float *adam_v, float *grad);

/* Sets theta (and the Adam moments; NULL = zero) from host arrays, and the
 * bf16 copies of W1 and W2 the kernels read.  Waits. */
int gom_filter_set_params(gom_ctx_t *ctx, const float *theta, const float *adam_m, const float *adam_v);

/* One training step on the logged samples: the full-batch gradient of the
 * mean weighted logistic loss (the forward pass with bf16-rounded W1 and
 * W2, fp32 sums; positive samples weighted pos_weight), then one Adam step
 * (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8, bias correction of
 * step `step` >= 1, learning rate lr).  *loss (may be NULL) receives the mean
 * loss at the parameters before the step.  GOM_E_STATE with an empty log.
 * Waits. */
int gom_filter_epoch(gom_ctx_t *ctx, float learning_rate, float pos_weight, int32_t step, double *loss);

/* The training log: *n = samples held (the latest min(offered, capacity));
 * copies the first min(*n, max) of them, features as bf16 bits [.][16] (x) and
 * labels [.] (y), into host arrays (either may be NULL).  Waits. */
int gom_filter_log(gom_ctx_t *ctx, int64_t max, uint16_t *x, uint8_t *y, int64_t *n);

/* Logits of the first n logged samples with the current parameters, as the
 * mixing kernels compute them (bf16 W1 and W2, fp32 sums: two units per lane,
 * a fixed-order warp sum), into host logits[n].  Waits. */
int gom_filter_logits(gom_ctx_t *ctx, int64_t n, float *logits);

/* The elements skipped in the last generation: host_mask[j] = 1 (host, [m]). */
int gom_filter_skipped(gom_ctx_t *ctx, uint8_t *host_mask);

/* ---------------------------------------------------------------------------
 * Interleaved Multi-start Scheme (Sec. 6.3): populations P_0, P_1, ... of
 * base_pop * 2^i individuals (up to max_pop), P_i seeded with seed + i; one
 * generation of P_i is made each time P_{i-1} has made c more generations (the
 * paper's default c = 4).  All populations are made at creation (a population
 * made later would be the same: its initialisation depends on its seed only)
 * and run together on the batched path.
 */
typedef struct gom_ims gom_ims_t;

typedef struct gom_ims_result {
    int64_t steps;              /* generations made by P_0 so far */
    int64_t best_fitness;       /* best fitness of any generation of this call */
    int32_t reached;            /* 1 if a generation of this call reached the target */
    int32_t reached_population; /* the first to reach it in the scheme's order, -1 if none */
    int64_t reached_step;       /* the P_0 generation count at which that happened */
    int64_t reached_generation; /* that population's generation index */
} gom_ims_result_t;

/* Device bytes for gom_ims_create (every population's workspace and the batch). */
size_t gom_ims_workspace_bytes(const gom_graph_t *g, const gom_fos_t *fos, int32_t base_pop, int32_t max_pop);

/* The scheme on a coloured FOS; base_pop >= 2, c >= 1, max_pop <= GOM_MAX_POPULATION.
 * d_workspace: caller-owned, gom_ims_workspace_bytes bytes, 256-byte aligned. */
int gom_ims_create(const gom_graph_t *g, const gom_fos_t *fos, int32_t base_pop, int32_t c, int32_t max_pop,
                   uint64_t seed, void *d_workspace, size_t ws_bytes, void *cuda_stream, gom_ims_t **out);

/*
 * Advances the scheme by `steps` generations of P_0 (0..1024), every other
 * population by its share, in one batched launch.  A population that reaches
 * `target` stops there; res (host, may be NULL) reports the first reach in the
 * scheme's own order -- P_i's r-th generation comes at P_0's generation
 * r * c^i, after those of the smaller populations -- and the best fitness.
 * The scheme as stated stops every population at that first reach; here the
 * other populations run on to their own share or target.  Waits.
 */
int gom_ims_run(gom_ims_t *ims, int32_t steps, int64_t target, gom_ims_result_t *res);

/* Population i of the scheme (owned by it), for export or inspection. */
int gom_ims_population(gom_ims_t *ims, int32_t i, gom_ctx_t **ctx);
int32_t gom_ims_num_populations(const gom_ims_t *ims);
void gom_ims_destroy(gom_ims_t *ims);

/* Counters of the generations instance b ran in the last call, into
 * host_stats[0..capacity); *count receives their number.  Waits. */
int gom_batch_stats(gom_batch_t *batch, int32_t b, gom_gen_stats_t *host_stats, int32_t capacity, int32_t *count);

/* The blocks of instance b ([*blk0, *blk0 + *nblk)) and the launch's grid. */
int gom_batch_layout(const gom_batch_t *batch, int32_t b, int32_t *blk0, int32_t *nblk, int32_t *grid);

void gom_batch_destroy(gom_batch_t *batch);

/*
 * Autotuner of the batch configuration: for each of cfgs[0..num_cfg) it
 * builds the batch and times `generations` generations of every instance
 * (CUDA events), all from the same starting state -- the instances' states
 * are saved to d_scratch first and restored after every trial, so tuning
 * changes no result.  *best receives the index of the fastest configuration,
 * ms[c] (host, may be NULL) the milliseconds per generation of each (a
 * configuration that cannot be built gets a negative value).  d_scratch:
 * gom_batch_scratch_bytes(ctxs, num) bytes of device memory, 256-byte
 * aligned.  Waits for cuda_stream.
 */
size_t gom_batch_scratch_bytes(gom_ctx_t *const *ctxs, int32_t num);
int gom_batch_autotune(gom_ctx_t *const *ctxs, int32_t num, const gom_batch_config_t *cfgs, int32_t num_cfg,
                       int32_t generations, void *d_scratch, size_t scratch_bytes, void *cuda_stream,
                       int32_t *best, double *ms);

void gom_destroy(gom_ctx_t *ctx);

const char *gom_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GOM_H_ */
