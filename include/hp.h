/*
 * hp.h -- C ABI of the GB300 (sm_103a) constrained multilevel hypergraph
 * partitioner.
 *
 * The operation is the one of Ronzani & Silvano, "Hypergraph Partitioning on
 * GPU with Distinct Incident Hyperedges and Size Constraints":
 *   Sec. II-A  a directed, weighted hypergraph: each hyperedge e has source
 *              pins src(e) and destination pins dst(e); in(n) is the set of
 *              hyperedges that hold n as a destination.
 *   Sec. II-B  find a partitioning rho that minimises the connectivity
 *              Conn = sum_e w(e) * (lambda(e) - 1)   (Eq. 1)
 *              subject to |p| <= Omega and |U_{n in p} in(n)| <= Delta for
 *              every part p.
 *   Sec. III   by multilevel coarsening (Sec. V) and refinement (Sec. VI).
 *
 * Conventions (all calls):
 *   - ids are 0-based int32; a hypergraph has num_nodes nodes and num_hedges
 *     hyperedges in CSR form: offsets[num_hedges + 1] (offsets[0] = 0,
 *     strictly increasing, so every hyperedge has at least one pin) and
 *     pins[offsets[num_hedges]]; pins within a hyperedge are distinct; the
 *     first src_counts[e] pins of hyperedge e are its sources (Sec. IV-B
 *     stores sources first), the rest its destinations.  src_counts == NULL
 *     means exactly one source per hyperedge, its first pin.
 *   - weights == NULL means w(e) = 1; otherwise 1 <= w(e) <= 65536 and
 *     sum_e w(e) <= 2^37.
 *   - Omega >= 1, Delta >= 0.  A node with |in(n)| > Delta makes the problem
 *     infeasible (HP_ERR_INFEASIBLE).
 *   - The caller owns every buffer it passes; the library never frees caller
 *     memory and releases all of its own device memory before returning.
 *   - Outputs are written only when the call returns HP_OK.
 *   - Results are deterministic: the same inputs, Omega, Delta, seed and
 *     options give the same part vector on every run, and it is the part
 *     vector of the method as specified by the readings listed with
 *     hp_options below.
 *   - A call is synchronous with respect to the host (it returns after the
 *     results are in place); calls on different streams may run from
 *     different host threads.
 */
#ifndef HP_H
#define HP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HP_API __attribute__((visibility("default")))
#else
#define HP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HP_OK = 0,
    HP_ERR_INVALID_ARG = 1,  /* bad scalar argument, option, weight or NULL pointer */
    HP_ERR_BAD_CSR = 2,      /* offsets not strictly increasing from 0, pin out of range,
                                src count outside [0, |e|], duplicate pin in a hyperedge */
    HP_ERR_INFEASIBLE = 3,   /* some node alone exceeds Delta */
    HP_ERR_OOM = 4,          /* device allocation failed */
    HP_ERR_CUDA = 5,         /* CUDA runtime error (see hp_last_error) */
    HP_ERR_TIMEOUT = 6,      /* a bounded device loop ran out of iterations */
    HP_ERR_INTERNAL = 7      /* an internal consistency check failed */
} hp_status;

typedef enum {
    HP_COUNT_INBOUND = 0,   /* Delta bounds distinct inbound hyperedges (Sec. II-B) */
    HP_COUNT_INCIDENT = 1   /* Delta bounds distinct incident hyperedges (Sec. II-B, last
                               paragraph): every pin counts as a destination */
} hp_count_kind;

/*
 * Options (hp_default_options gives the paper's defaults):
 *   pi             candidates per node and matching rounds per level (Sec. V-D, 4)
 *   theta          refinement repetitions per level (Sec. VI-A, 16); repetitions
 *                  in the second half only propose moves that keep the
 *                  destination within Omega (Sec. VI-B)
 *   chain_window   successor candidates a chain end examines (Sec. VI-C, 256)
 *   chain_rounds   chaining rounds (Sec. VI-C, 16)
 *   noise_permille pairing noise cap in permille of the mean fixed-point
 *                  hyperedge weight (Sec. V-C, 100 = 10%)
 *   count_kind     hp_count_kind
 *   max_levels     coarsening levels at most (256)
 *   debug_table_cap  0 in normal use; a positive power of two caps the shared-
 *                  memory neighbour table of the proposal kernel so that tests
 *                  can force its overflow path on small inputs (result-neutral)
 *   debug_walk_cap 0 in normal use; a positive value bounds each tree walk of
 *                  the matching (Sec. V-D) to that many steps instead of the
 *                  level's node count, so that a test can make the bounded
 *                  loop give up: the call then returns HP_ERR_TIMEOUT before
 *                  the level is contracted
 *   learned_k      0 (default): C(n) is the top-pi valid neighbours by
 *                  (eta, id), as in the paper.  pi..16: the learned merge
 *                  priority below ranks each node's top-learned_k list.
 *   merge_model    host pointer to the model of the learned priority (read
 *                  during the call; required when learned_k > 0, else ignored)
 *   learned_levels 0 (default): with learned_k > 0 the learned priority ranks
 *                  the candidates of every coarsening level; n > 0: of the first n
 *                  levels only, deeper levels taking the paper's (eta, id) order
 *                  (the model is trained on level-0 pairs)
 *   node_batch     0 (default): every node of a level at once.  n > 0: the
 *                  learned priority scores the pairs of n nodes per pass, so
 *                  its per-pair rows (24 B per listed pair) take n*learned_k
 *                  rows instead of one per listed pair of the level (the
 *                  node-batched coarsening of Sec. VII-C; result-neutral)
 */
typedef struct hp_merge_model hp_merge_model;
typedef struct {
    int32_t pi;
    int32_t theta;
    int32_t chain_window;
    int32_t chain_rounds;
    int32_t noise_permille;
    int32_t count_kind;
    int32_t max_levels;
    int32_t debug_table_cap;
    int32_t learned_k;
    int32_t debug_walk_cap;
    const hp_merge_model *merge_model;
    int32_t node_batch;
    int32_t learned_levels;
} hp_options;

/*
 * Learned merge priority -- a growth of Sec. V-C that the paper does not
 * have.  Each node keeps its top-K valid neighbours by (eta, id) (Eq. 5-6
 * with K in place of pi); a pair stays a candidate only when each end is in
 * the other's list; C(n) is then the top pi of the node's candidates by
 * (s, eta, id), descending, where s is the score of the MLP below on sixteen
 * features of the pair, each in 0..255 and symmetric in the two ends.  The
 * matching of Sec. V-D keeps eta as its weight and the best-effort pairing
 * still takes the nodes with no valid neighbour.  Because s and the candidate
 * relation are symmetric, the proposal graph keeps only 2-cycles, so the
 * matching stays exact.
 *
 * Features, with L(x) = 0 for x = 0, else min(255, 1 + 4 floor(log2 x) + the
 * two bits that follow the leading one), for the pair (v, m):
 *   0 L(eta)  1 L(|I(v) & I(m)|)  2 L(inter = |in(v) & in(m)|)
 *   3,4 L(min, max of the sizes)  5,6 L(min, max of |in|)  7,8 L(min, max of |I|)
 *   9 floor(255 (size(v)+size(m)) / Omega)  10 floor(255 |in(v) U in(m)| / Delta)
 *   11 min(level, 255)  12 floor(255 inter / |in(v) U in(m)|) (0 if empty)
 *   13,14 min, max of the two list positions  15 L(|in(v)| + |in(m)|)
 * MLP, integers throughout (floor shifts; every product and partial sum is
 * an integer below 2^21, so bf16 operands with fp32 accumulation compute it
 * exactly):
 *   a1 = clamp((b1 + W1 f) >> shift1, 0, 255)     W1 [64][16]
 *   a2 = clamp((b2 + W2 a1) >> shift2, 0, 255)    W2 [64][64]
 *   s  = b3 + w3 . a2                              w3 [64]
 * Weight codes lie in [-127, 127], biases in [-2^30, 2^30], shifts in 0..30;
 * anything else is HP_ERR_INVALID_ARG.
 */
struct hp_merge_model {
    int8_t w1[64][16];
    int8_t w2[64][64];
    int8_t w3[64];
    int32_t b1[64];
    int32_t b2[64];
    int32_t b3;
    int32_t shift1;
    int32_t shift2;
};

/* Per-call statistics (host struct filled on HP_OK). */
typedef struct {
    int64_t connectivity;      /* Eq. 1 of the returned part vector */
    int64_t cut_net;           /* Eq. 16 */
    int32_t num_parts;
    int32_t max_part_size;
    int32_t max_part_distinct; /* max over parts of distinct inbound (or incident) hyperedges */
    int32_t violations;        /* parts over Omega or Delta (0 on success) */
    int32_t levels;            /* hypergraphs in the hierarchy, level 0 included */
    int32_t reserved0;
    int64_t moves_applied;     /* refinement moves applied over all levels */
    int64_t pin_visits;        /* sum over coarsening levels of sum_e |e|^2 (proposal traversal) */
    double ms_total;           /* device time of the call, input checks included */
    double ms_coarsen;
    double ms_refine;
    int64_t kernel_launches;   /* CUDA kernels this call launched */
    int64_t l0_pin_visits;     /* sum_e |e|^2 of level 0: pins read by the level-0 proposal */
    int64_t l0_neighbours;     /* sum over nodes of |N(n)| at level 0 */
    double ms_propose_l0;      /* CUDA-event time of the level-0 candidate proposal (Sec. V-C) */
    int64_t alg_bytes;         /* algorithmic bytes of the whole call: per coarsening level the
                                  proposal traversal (4 B per pin visit, 8 B per distinct
                                  neighbour, 12 B per incidence entry, 12*pi+4 B per node), the
                                  matching (48 B per node per round) and the contraction (12 B per
                                  pin, 8 B per coarse pin, 16 B per node); per refinement
                                  repetition the pins lists when rebuilt (12 B per pin + 12 B per
                                  list entry), the cut entries and their list entries (4 B + 12 B),
                                  and 48 B per proposed move */
} hp_stats;

/* Per-level trace record (optional output of hp_partition_ex). */
typedef struct {
    int32_t n;             /* nodes of the level */
    int32_t pairs;         /* clusters of two formed at this level (0 at the coarsest) */
    int32_t iso_pairs;     /* of which by the best-effort pairing of Sec. V-C */
    int32_t reps;          /* refinement repetitions run at this level */
    int64_t pins;          /* sum_e |e| of the level */
    int64_t conn;          /* connectivity after refining this level */
    int64_t moves;         /* moves applied at this level */
    /* how the level paired (Sec. V-C, V-D; 0 at the coarsest level): */
    int32_t valid;         /* nodes with at least one valid neighbour */
    int32_t iso_list;      /* nodes without one: the best-effort pairing's list */
    int32_t targets_r1;    /* distinct targets of the first proposal graph */
    int32_t max_indeg_r1;  /* largest number of nodes targeting one node in it */
    int32_t pairs_r1;      /* pairs formed by the first matching round */
    int32_t reserved;
} hp_level_trace;

HP_API void hp_default_options(hp_options *opt);

/*
 * hp_partition -- partition a hypergraph held in device memory.
 *   pins, offsets, src_counts, weights: device pointers, layout above.
 *   part_out: device int32[num_nodes]; part ids compacted to
 *             0..num_parts-1 in ascending order of the internal id.
 *   stats:    host pointer or NULL.
 *   stream:   cudaStream_t (NULL = legacy default stream).
 * Errors: see hp_status; on error nothing is written.
 * Kernels on levels of up to 32,768 nodes are launched with programmatic
 *   dependent launch (each may be scheduled while its predecessor on
 *   `stream` runs, and waits for it at entry); the environment variable
 *   HP_PDL=0, read at the first launch, turns that off.  Results do not
 *   depend on it.
 */
HP_API hp_status hp_partition(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                       const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta,
                       uint64_t seed, const hp_options *opt, int32_t *part_out, hp_stats *stats,
                       void *stream);

/*
 * hp_partition_ex -- hp_partition plus an optional per-level trace:
 *   trace: host array of trace_cap records or NULL; levels beyond trace_cap
 *          are not recorded (hp_stats.levels tells how many exist).
 */
HP_API hp_status hp_partition_ex(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                          const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta,
                          uint64_t seed, const hp_options *opt, int32_t *part_out, hp_stats *stats,
                          hp_level_trace *trace, int32_t trace_cap, void *stream);

/*
 * One hypergraph of a batch: the arguments of hp_partition, device pointers.
 */
typedef struct {
    const int32_t *pins, *offsets, *src_counts, *weights;
    int32_t num_hedges, num_nodes, omega, delta;
    uint64_t seed;
    int32_t *part_out;
} hp_instance;

/*
 * hp_partition_batch -- partitions count independent hypergraphs (each one
 *   exactly as hp_partition would, same part vector and stats) with up to
 *   `concurrency` (1..64) of them in flight at once, largest first, each on a
 *   stream of its own; the paper partitions one hypergraph per call, this
 *   is the batched form for many small ones.
 *   concurrency 0: autotuned.  Instances are grouped into size classes by
 *   nodes + hyperedges ([0, 2^12), then factors of 4), largest class first;
 *   the first instances of a class not tuned yet on this device run in
 *   groups of 2c at c = 4, 8, 16, 32, 64 in flight, and the rest of the class
 *   (and that class in later calls) at the c with the most nodes + hyperedges
 *   per second.  Only the schedule is tuned: every instance is partitioned
 *   once, with the result hp_partition gives.
 *   inst: host array [count]; opt: shared options (NULL = defaults);
 *   stats_out, status_out: host arrays [count] or NULL, filled per instance.
 *   The work starts after the work already queued on `stream`, and `stream`
 *   waits for all of it.  Returns HP_OK when every instance succeeded, else
 *   the status of the first failing instance (by index), whose message
 *   hp_last_error gives; the other instances are still partitioned.
 *   Synchronous with respect to the host.
 */
HP_API hp_status hp_partition_batch(const hp_instance *inst, int32_t count, const hp_options *opt,
                                    int32_t concurrency, hp_stats *stats_out, int32_t *status_out, void *stream);

/*
 * hp_batch_tuned_concurrency -- the concurrency the autotuner of
 *   hp_partition_batch settled on for size class `size_class` (0..5) on CUDA
 *   device `device`, or 0 when that class has not been tuned there.
 */
HP_API int32_t hp_batch_tuned_concurrency(int32_t device, int32_t size_class);

/*
 * hp_partition_host -- the same with every array in host memory: the call
 * copies the hypergraph to the device once and the part vector back once
 * (the two transfers of Sec. VII-C).  part_out is host int32[num_nodes].
 */
HP_API hp_status hp_partition_host(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                            const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta,
                            uint64_t seed, const hp_options *opt, int32_t *part_out, hp_stats *stats,
                            void *stream);

/*
 * hp_set_allocator -- route the library's device workspace through a caller
 * allocator (e.g. a framework's caching allocator).  alloc(bytes, ctx) returns
 * a device pointer aligned to 256 bytes or NULL; free(ptr, ctx) releases it.
 * Passing NULL functions restores stream-ordered cudaMallocAsync/cudaFreeAsync.
 * Process-wide; not to be changed while a call is running.
 */
HP_API hp_status hp_set_allocator(void *(*alloc_fn)(size_t bytes, void *ctx), void (*free_fn)(void *ptr, void *ctx),
                           void *ctx);

/* Static description of a status code. */
HP_API const char *hp_status_string(hp_status status);

/* Message of the last error raised on the calling host thread ("" if none). */
HP_API const char *hp_last_error(void);

/*
 * hp_connectivity -- Eq. 1 and Eq. 16 of a given part vector, on the device.
 *   pins, offsets, weights (nullable), part: device pointers; num_parts > max part id.
 *   conn_out, cutnet_out: host pointers.
 */
HP_API hp_status hp_connectivity(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, const int32_t *weights,
                          const int32_t *part, int32_t num_nodes, int32_t num_parts, int64_t *conn_out,
                          int64_t *cutnet_out, void *stream);

/*
 * hp_connectivity_noalloc -- the same two numbers as hp_connectivity,
 *   computed without allocating any device memory.  The paper has no
 *   counterpart: this is a service call for callers that cannot let the
 *   library allocate at the moment they need the number (an allocator hook
 *   that refuses requests while the caller's own step runs, a process whose
 *   free device memory belongs to another pool, a monitoring thread that must
 *   not take or wait on an allocator lock).
 *   Arguments, layouts and ownership as for hp_connectivity.
 *   Scratch: a fixed area inside the loaded library, one per device (256 B of
 *   result words, zeroed by each call on `stream` before use, and an 8 MiB
 *   hash table that is zero at load and that every call returns to zero).
 *   The area is device memory of the library, placed on a device when the
 *   library's kernels are loaded there.  The first call on a device of this
 *   function, hp_partition, hp_partition_ex, hp_partition_host or
 *   hp_connectivity loads them (and looks up the area's device address with
 *   the device current), so a caller that hands all free device memory to
 *   another pool makes one such call on each device first; make that first
 *   call before any stream capture too.  The looked-up address belongs to the
 *   device's context: do not call the library on a device after
 *   cudaDeviceReset.  Calls that can overlap on one device (two streams, two
 *   host threads) share the area and race: serialise them.
 *   Limit: a hyperedge of more than 262,144 pins returns HP_ERR_INVALID_ARG
 *   (hp_last_error names the size), with nothing written.
 *   Errors: HP_ERR_BAD_CSR for offsets that are not strictly increasing from
 *   0 or a pin out of range (duplicate pins are not detected: they leave
 *   lambda(e) unchanged); HP_ERR_INVALID_ARG for a part id outside
 *   [0, num_parts), a weight outside 1..65536, or a bad scalar/pointer.
 *   Synchronises `stream` before returning.
 */
HP_API hp_status hp_connectivity_noalloc(const int32_t *pins, const int32_t *offsets, int32_t num_hedges,
                                         const int32_t *weights, const int32_t *part, int32_t num_nodes,
                                         int32_t num_parts, int64_t *conn_out, int64_t *cutnet_out, void *stream);

/*
 * hp_merge_scores -- the MLP of the learned merge priority on `count` feature
 *   rows: feat is device uint8[count][16], score_out device int32[count],
 *   model a host pointer.  HP_ERR_INVALID_ARG for a model out of range, a
 *   negative count or a NULL pointer (count 0 needs none).  Synchronises
 *   `stream` before returning.
 */
HP_API hp_status hp_merge_scores(const uint8_t *feat, int64_t count, const hp_merge_model *model,
                                 int32_t *score_out, void *stream);

/*
 * Training the learned merge priority.  The trainable form is the same
 * network in fp32 on scaled features x = f / 256:
 *   z1 = W1 x + b1, h1 = max(z1, 0), z2 = W2 h1 + b2, h2 = max(z2, 0),
 *   o = w3 . h2 + b3, loss = mean over rows of BCE(sigmoid(o), y).
 * Its parameters are one fp32 array of HP_MERGE_NPARAM values, in this order:
 * W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.
 */
#define HP_MERGE_NPARAM 5313

/*
 * hp_merge_features -- the level-0 training rows of one hypergraph: the
 *   proposal's top-K lists (K = opt->learned_k, pi <= K <= 16; no model
 *   needed) and the sixteen features of every listed pair, exactly as the
 *   partitioner computes them at level 0.  Inputs as for hp_partition (device
 *   pointers).  Device outputs of num_nodes*K entries: cand_out[v*K+j] the
 *   j-th candidate of v (-1 padded), rank_out the position of v in that
 *   candidate's list (-1 when the pair is not mutual), feat_out 16 bytes per
 *   entry (zero unless mutual).  Synchronises `stream` before returning.
 */
HP_API hp_status hp_merge_features(const int32_t *pins, const int32_t *offsets, int32_t num_hedges, int32_t num_nodes,
                                   const int32_t *src_counts, const int32_t *weights, int32_t omega, int32_t delta,
                                   uint64_t seed, const hp_options *opt, int32_t *cand_out, int32_t *rank_out,
                                   uint8_t *feat_out, void *stream);

/*
 * hp_merge_grad -- loss and gradient of the trainable form over `count` rows
 *   (device: feat uint8[count][16], label float[count] in [0, 1], params
 *   float[HP_MERGE_NPARAM]; grad_out float[HP_MERGE_NPARAM] is overwritten).
 *   *loss_out (host, optional): the mean loss.  fp32 arithmetic; the
 *   reduction over rows has a fixed order, so results repeat bit for bit.
 *   Synchronises `stream` before returning.
 */
HP_API hp_status hp_merge_grad(const uint8_t *feat, const float *label, int64_t count, const float *params,
                               float *grad_out, double *loss_out, void *stream);

/*
 * hp_merge_adam -- one Adam step (Kingma & Ba 2015) with decoupled weight
 *   decay on params, using grad; m and v are the moment arrays (device,
 *   HP_MERGE_NPARAM each, zero before step 1); step counts from 1.
 */
HP_API hp_status hp_merge_adam(float *params, const float *grad, float *m, float *v, int64_t step, float lr,
                               float beta1, float beta2, float eps, float weight_decay, void *stream);

/*
 * hp_merge_quantize -- the integer model (hp_merge_model) of trained
 *   parameters (host float[HP_MERGE_NPARAM]).  Each layer's weights are
 *   scaled so that their largest magnitude becomes 127 and rounded; biases
 *   are carried into the integer scale; each shift is the smallest one that
 *   keeps the layer's largest activation over the `count` calibration rows
 *   (host uint8[count][16]) within 255.  The score is then, up to rounding, a
 *   positive multiple of the float output o, so it ranks pairs the same way.
 *   Host only.
 */
HP_API hp_status hp_merge_quantize(const float *params, const uint8_t *calib, int64_t count, hp_merge_model *out);

/*
 * Step-level entry points (test hooks) on one level graph given in device
 * memory: num_nodes, num_hedges, offsets, pins, src_counts (required, one
 * count per hyperedge), weights (required) and node sizes.  They run one step
 * of the method exactly as hp_partition runs it inside its level loop.
 *
 * hp_debug_coarsen_level -- one coarsening level (Sec. V-C, V-D): the top-pi
 *   candidates of every node (cand_out[n*pi], -1 padded; score_out[n*pi] the
 *   fixed-point eta plus noise of Eq. 5, noise keyed by seed and level), then
 *   best-effort pairing and pi rounds of matching; mate_out[n] is the
 *   partner or -1; *pairs_out (host) counts the pairs.  With learned_k set,
 *   cand_out/score_out hold C(n) of the learned priority and eta.
 */
HP_API hp_status hp_debug_coarsen_level(int32_t num_nodes, int32_t num_hedges, const int32_t *offsets,
                                        const int32_t *pins, const int32_t *src_counts, const int32_t *weights,
                                        const int32_t *size, int32_t omega, int32_t delta, uint64_t seed,
                                        int32_t level, const hp_options *opt, int32_t *cand_out, uint64_t *score_out,
                                        int32_t *mate_out, int64_t *pairs_out, void *stream);

/*
 * hp_debug_refine_rep -- one refinement repetition (Sec. VI) of part vector
 *   rho (device int32[n], ids < num_parts, updated in place).  Device outputs
 *   of n entries: the proposed moves sorted by (p_s asc, gain desc, node asc)
 *   (move_node/src/dst/gain, Eq. 13), seq[k] = index of the k-th move of the
 *   chained sequence (Sec. VI-C), gseq[k] its in-sequence gain (Eq. 14-15).
 *   Host outputs: *num_moves, *applied (moves of the best valid prefix,
 *   Sec. VI-D) and *best_gain (its cumulative gain; 0 when none is applied).
 */
HP_API hp_status hp_debug_refine_rep(int32_t num_nodes, int32_t num_hedges, const int32_t *offsets,
                                     const int32_t *pins, const int32_t *src_counts, const int32_t *weights,
                                     const int32_t *size, int32_t *rho, int32_t num_parts, int32_t second_half,
                                     int32_t omega, int32_t delta, const hp_options *opt, int32_t *move_node,
                                     int32_t *move_src, int32_t *move_dst, int64_t *move_gain, int32_t *seq,
                                     int64_t *gseq, int32_t *num_moves, int32_t *applied, int64_t *best_gain,
                                     void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HP_H */
