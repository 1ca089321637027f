/*
 * kc.h -- C ABI of the GB300 (sm_103a) implementation of the 2-forest /
 * tree-to-forest (TTF) Kemeny-constant estimator of Li, Liao, Li and Wang,
 * "Scalable and Provable Kemeny Constant Computation on Static and Dynamic
 * Graphs: A 2-Forest Sampling Approach".
 *
 * The library samples uniform spanning trees with Wilson's loop-erased walk
 * (Sec. 2.2; Algorithm 1 "wilson(G, r)"), traverses each tree (subtree sizes,
 * volumes, depths, DFN: Algorithm 1 and Sec. 3.2), evaluates the per-tree
 * path-mapping value f(tau) of Theorem 3, and averages
 *     K_hat = sum_i w_i f(tau_i) / (2m sum_i w_i)
 * (Theorem 3: w_i = 1; Algorithm 3 uses per-tree weights after updates).
 * Sample maintenance after edge insertions and deletions follows Algorithm 2
 * (BSM) and Algorithm 3 (ISM).  Every step of the path runs in CUDA kernels on
 * one GPU; this header is plain C (no CUDA or torch types).
 *
 * Conventions for every call:
 *  - Every function returns a kc_status; nothing throws or aborts across the
 *    ABI.  On error the handle is left as it was before the call.
 *  - Array arguments are HOST pointers owned by the caller, unless the handle
 *    was created with kc_config.inputs_on_device = 1 (then the graph arrays of
 *    kc_graph_create are device pointers).  The library copies what it needs;
 *    the caller may free its arrays after the call returns.
 *  - Vertices are 0 .. n-1.  The graph must be simple, undirected (both
 *    directions present), connected, n >= 2 (Sec. 2.1), given in CSR with each
 *    row sorted strictly ascending (neighbour index k means the k-th smallest
 *    neighbour id; this fixes the random-walk stream).
 *  - One handle must not be used by two host threads at once.  Work runs on the
 *    handle's CUDA stream (kc_graph_set_stream); calls that return results to
 *    the host synchronise that stream.
 *
 * Random-number contract (the paper only asks for a uniform neighbour):
 * Philox4x32-10 (Salmon et al., SC'11) with key = (seed low 32, seed high 32)
 * and counter = (vertex u, departure index k of u, sample id, tag << 24 | retry);
 * the walk leaves u on its k-th departure along neighbour
 * Lemire-bounded(word, deg(u)), trying the block's four words in order and
 * bumping `retry` if all four are rejected.  Keying arrows by (u, k) makes a
 * tree and its step count independent of the order in which walks start
 * (Wilson's cycle-popping argument), so any launch shape gives the same trees.
 */
#ifndef KC_H
#define KC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KC_ABI_VERSION 1

typedef enum {
    KC_OK = 0,
    KC_ERR_INVALID_ARG = 1,    /* NULL handle/pointer, n < 2, bad sizes or options  */
    KC_ERR_NOT_SYMMETRIC = 2,  /* some (u,v) present without (v,u)                  */
    KC_ERR_SELF_LOOP = 3,      /* some (u,u)                                         */
    KC_ERR_MULTI_EDGE = 4,     /* a row not strictly ascending (repeat or unsorted) */
    KC_ERR_DISCONNECTED = 5,   /* the graph (or G' after a deletion) is disconnected */
    KC_ERR_OVERFLOW = 6,       /* 4 m^2 ecc(r) >= 2^62: int64 f(tau) could overflow  */
    KC_ERR_OUT_OF_MEMORY = 7,  /* device allocation failed                           */
    KC_ERR_CUDA = 8,           /* any other CUDA runtime error                       */
    KC_ERR_STEP_LIMIT = 9,     /* a Wilson walk exceeded kc_config.step_cap          */
    KC_ERR_EDGE_EXISTS = 10,   /* insert of an edge already present                  */
    KC_ERR_EDGE_MISSING = 11,  /* delete of an edge not present                      */
    KC_ERR_BRIDGE = 12,        /* delete of a bridge (G' would be disconnected)      */
    KC_ERR_NO_SAMPLES = 13,    /* estimate/update needs at least one sampled tree    */
    KC_ERR_NO_DEVICE = 14,     /* no CUDA device, or not an sm_103 device            */
    KC_ERR_NOT_RETAINED = 15,  /* trees were not kept (keep_trees = 0)               */
    KC_ERR_SCRATCH_LIMIT = 16  /* request larger than kc_wilson_noalloc's fixed scratch */
} kc_status;

/* TTF traversal variant (Theorem 8: O(n min(Delta, log n)) per tree). */
enum { KC_TTF_AUTO = 0,   /* SCAN when ecc(r) <= 2 log2 n, else BIT           */
       KC_TTF_SCAN = 1,   /* per-vertex walk up tau0 (O(n ecc)), all vertices in parallel */
       KC_TTF_BIT = 2 };  /* Algorithm 1's DFS with a BIT over the tau0 DFN     */

/* Stopping rule of kc_estimate. */
enum { KC_STOP_CLT = 0,        /* z_{1-delta/2} s / sqrt(w) <= eps K_hat (1 - eps), w >= 64 */
       KC_STOP_HOEFFDING = 1 }; /* Theorem 5 sample size (Delta read as ecc(r), kappa >= (n-1)^2/n) */

/* Sample maintenance (Sec. 4). */
enum { KC_UPDATE_BSM = 0,      /* Algorithm 2 */
       KC_UPDATE_ISM = 1 };    /* Algorithm 3 */

/* Wilson walkers per tree.  All give identical trees and step counts. */
enum { KC_WALK_AUTO = 0,       /* WARP; LANE under rejection by walk length on a graph
                                  whose TTF variant is BIT (long diameter)                */
       KC_WALK_LANE = 1,       /* one sequential walker per tree (one lane)              */
       KC_WALK_WARP = 2,       /* 32 concurrent walkers per tree popping cycles in any order */
       KC_WALK_HYBRID = 3 };   /* LANE for a prefix of the start order, then WARP for the
                                  rest; LANE trees still running when a share of the
                                  wave has finished are also handed to WARP          */

/* Path tree tau0 (Algorithm 1 uses BFS; Exp-II compares DFS and Wilson trees).
   Theorem 4 holds for any fixed spanning tree; shorter paths give lower variance. */
enum { KC_TAU0_BFS = 0,        /* BFS tree, parent = smallest-id neighbour one level up  */
       KC_TAU0_DFS = 1,        /* depth-first tree, rows scanned in ascending id          */
       KC_TAU0_WILSON = 2 };   /* uniform tree of sample id 0 under tau0_seed             */

/* Effective resistance source for insertions (Algorithm 2/3 "Compute R(u,v)"). */
enum { KC_R_CG = 0,            /* FP64 conjugate gradients on the Laplacian, on the device */
       KC_R_GIVEN = 1 };       /* kc_edge_op.r supplies R(u,v) in G + (u,v)               */

typedef struct {
    uint32_t struct_size;       /* sizeof(kc_config), for ABI growth              */
    int32_t root;               /* >= 0: this vertex.  -1: highest degree (Exp-III), ties
                                   broken towards the centre: among the highest-degree
                                   vertices the one minimising max(d(a,.), d(b,.),
                                   d(c,.)) for a = farthest from the smallest-id
                                   candidate, b = farthest from a, c = maximiser of
                                   min(d(a,.), d(b,.)); smallest id among equals.
                                   -2: highest degree, smallest id among ties.      */
    int32_t ttf_variant;        /* KC_TTF_*                                         */
    int32_t keep_trees;         /* 1: retain parent arrays (needed by kc_update,
                                   kc_get_tree of updated trees); 0: static mode      */
    int32_t stop_rule;          /* KC_STOP_*                                         */
    int32_t refresh_after_update; /* 1: recompute f of every retained tree after each
                                   update (exactly unbiased); 0: keep stale f of
                                   untouched trees (the paper's Theorem on BSM)     */
    int32_t inputs_on_device;   /* 1: kc_graph_create arrays are device pointers      */
    int32_t r_source;           /* KC_R_*                                            */
    int32_t walker;             /* KC_WALK_*: walkers per tree                        */
    int32_t autotune;           /* 1: the first kc_sample call with at least 64 trees
                                   times two pilot waves -- 32 walkers per tree with
                                   the chunked traversal, then one walker per tree
                                   with the leaf-to-root traversal (SCAN graphs) --
                                   and keeps the faster walker and traversal; the
                                   pilots' trees join the pool (every variant gives
                                   the same trees).  Overrides `walker`.            */
    int64_t max_trees_in_flight; /* 0: chosen from free device memory               */
    int64_t batch_trees;        /* kc_estimate batch size (0: 1024)                 */
    int64_t max_trees;          /* kc_estimate cap on the pool size (0: 1 << 24)     */
    int64_t step_cap;           /* cap on Wilson departures (0: max(2^22, 1024 n)), per
                                   tree for the one-walker kernel and per walker for
                                   the 32-walker kernel (a tree may then take up to
                                   32 x step_cap); exceeding it is KC_ERR_STEP_LIMIT */
    double mem_fraction;        /* share of free device memory for workspaces (0: 0.8) */
    int64_t sample_id_base;     /* first sample id of the pool (0); ranks of a
                                   multi-GPU run use disjoint bases, ids < 2^32   */
    int32_t hybrid_prefix_permille; /* KC_WALK_HYBRID: starts of the lane phase, in
                                   thousandths of n (0: default 1000 = all; the
                                   tail hand-off alone then moves work to WARP)     */
    int32_t hybrid_tail_permille; /* KC_WALK_HYBRID: lane trees still running when
                                   this many thousandths of the wave's trees have
                                   finished continue as WARP trees (0: default 900;
                                   >= 1000: never)                                  */
    int32_t tau0_kind;          /* KC_TAU0_*: the path tree (kc_update needs BFS)    */
    int32_t reserved1;
    uint64_t tau0_seed;         /* seed of the KC_TAU0_WILSON path tree              */
    int64_t reject_steps;       /* > 0: rejection by walk length.  A tree whose
                                   Wilson step count exceeds this is abandoned and
                                   the next sample id drawn instead, so the pool holds
                                   the first accepted ids (not consecutive).  The
                                   tree is independent of its step count, so the
                                   accepted trees stay uniform.  At least n - 1 (each
                                   non-root vertex departs once); needs the LANE or
                                   WARP walker, keep_trees = 0 and no autotune; not
                                   for kc_sample_multi.  0: off (default)           */
    double reject_accept_hint;  /* expected share of trees within reject_steps (e.g. the
                                   quantile the cap was taken at), in (0, 1]: sizes a
                                   handle's first rejection wave so that it usually
                                   accepts enough trees in one go; later waves use the
                                   share seen so far.  0: 8/9                       */
    int32_t ttf_segments;       /* BIT evaluation of f (Algorithm 1) split into preorder
                                   segments, each replayed by its own warp from the
                                   DFS state rebuilt at its first position (same f,
                                   exactly).  0: automatic -- the chunks evaluated
                                   after their wave's walk has ended, up to 16
                                   segments a tree and about 32 segment warps an SM,
                                   in memory the wave no longer needs (sub-wave slots
                                   the chunk leaves free, the stack buffer, rejected
                                   trees' walk arrays); 1: never; k >= 2
                                   (at most 64): up to k segments for every BIT
                                   evaluation, with a handle buffer for what free
                                   memory does not hold                             */
    int32_t reserved2;
} kc_config;

/* Fill *cfg with the defaults listed above. */
void kc_config_default(kc_config *cfg);

typedef struct kc_graph kc_graph; /* opaque; owns device copies of everything */

/*
 * Build a handle from an undirected connected CSR graph (Sec. 2.1).
 *  n        number of vertices (>= 2)
 *  row_off  int64[n+1], row_off[0] = 0, row_off[n] = 2m
 *  col      int32[2m], each row sorted strictly ascending, symmetric
 *  cfg      NULL for defaults
 *  out      receives the handle (NULL on error)
 * Runs graph validation, root choice, the BFS tree tau0 (parent = smallest-id
 * neighbour one level closer to r), its DFN and ecc(r) on the device
 * (Algorithm 1, first three lines).
 * Errors: INVALID_ARG, NOT_SYMMETRIC, SELF_LOOP, MULTI_EDGE, DISCONNECTED,
 * OVERFLOW, OUT_OF_MEMORY, NO_DEVICE, CUDA.
 */
kc_status kc_graph_create(int64_t n, const int64_t *row_off, const int32_t *col,
                          const kc_config *cfg, kc_graph **out);

/* Release every device and host resource of the handle.  NULL is accepted. */
kc_status kc_graph_destroy(kc_graph *g);

/* Use `cuda_stream` (a cudaStream_t, NULL = legacy default) for all later work. */
kc_status kc_graph_set_stream(kc_graph *g, void *cuda_stream);

/*
 * Serving helpers (no counterpart in the paper).
 * kc_graph_set_workspace_limit: later calls size their per-tree workspaces to
 *   at most `bytes` of device memory (0: a share of free memory, mem_fraction).
 * kc_graph_release_workspace: return the workspaces to the stream-ordered
 *   allocator (on the handle's stream, without synchronising the device).
 * kc_graph_reset: drop every sampled tree and fix `seed` and the next sample id
 *   (< 2^32), keeping the graph and tau0 resident; the next kc_sample or
 *   kc_estimate starts a fresh pool.
 * Errors: INVALID_ARG (negative bytes, id out of range), CUDA.
 */
kc_status kc_graph_set_workspace_limit(kc_graph *g, int64_t bytes);
kc_status kc_graph_release_workspace(kc_graph *g);
kc_status kc_graph_reset(kc_graph *g, uint64_t seed, int64_t sample_id_base);

/*
 * Draw n_trees uniform spanning trees rooted at r with sample ids
 * [pool, pool + n_trees) under `seed` (Algorithm 1 loop: wilson, subtree
 * volumes, DFS).  Appends each tree's f(tau) (int64, exact), step count and
 * unit weight to the pool; with keep_trees the parent array is kept too.  The
 * first call fixes the handle's seed; later calls must pass the same seed
 * (KC_ERR_INVALID_ARG otherwise) so sample ids are never reused.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, STEP_LIMIT, CUDA.
 */
kc_status kc_sample(kc_graph *g, uint64_t seed, int64_t n_trees);

/*
 * Reserve device memory ahead of sampling (no counterpart in the paper): pool
 * capacity for n_trees more trees and the workspace of a wave of n_trees, so
 * that later kc_sample calls allocate nothing.  Errors: INVALID_ARG,
 * OUT_OF_MEMORY, CUDA.
 */
kc_status kc_reserve(kc_graph *g, int64_t n_trees);

/*
 * Batched multi-graph sampling (no counterpart in the paper): the same result
 * as kc_sample(graphs[i], seeds[i], n_trees[i]) for every i, but the walks of
 * all graphs run in one 32-walker launch per round (one warp per tree, graphs
 * of uneven size mixed), which fills the GPU when each graph alone has too few
 * trees.  All work runs on graphs[0]'s stream.  The handles must be distinct
 * and on one device.  Errors: as kc_sample; on error no pool changes.
 */
kc_status kc_sample_multi(kc_graph *const *graphs, const uint64_t *seeds, const int64_t *n_trees,
                          int32_t count);

/*
 * Kemeny constant estimate K_hat = sum w f / (2m sum w) over the pool,
 * sampling more trees first (with the handle's seed, or 0 if none was set)
 * until the stopping rule for relative error eps at failure probability delta
 * holds (Theorem 5; KC_STOP_CLT by default).  eps <= 0 returns the estimate of
 * the current pool without sampling.  K_out receives K_hat.
 * Errors: INVALID_ARG, NO_SAMPLES (empty pool), OUT_OF_MEMORY, STEP_LIMIT, CUDA.
 * Batches sampled before a failing batch stay in the pool; a call that added
 * no tree leaves the handle's seed state as it was.
 */
kc_status kc_estimate(kc_graph *g, double eps, double delta, double *K_out);

/* One edge update (Sec. 4): op 0 = insert (u,v) (Ins), op 1 = delete (Del). */
typedef struct {
    int32_t u, v;
    int32_t op;       /* 0 insert, 1 delete */
    int32_t pad;
    double r;         /* R(u,v) in the graph containing (u,v); used when r_source = KC_R_GIVEN */
} kc_edge_op;

/*
 * Apply ops in array order, each as one paper update (Algorithm 2 when
 * mode = KC_UPDATE_BSM, Algorithm 3 when mode = KC_UPDATE_ISM), maintaining
 * the retained trees, their f and weights.  The whole batch is validated
 * against the evolving graph first; on any invalid op nothing is applied.
 * Requires keep_trees.  Errors: INVALID_ARG, EDGE_EXISTS, EDGE_MISSING,
 * BRIDGE, NO_SAMPLES, NOT_RETAINED, OVERFLOW, OUT_OF_MEMORY, STEP_LIMIT, CUDA.
 * OVERFLOW: 4 m^2 ecc(r) would reach 2^62 (the int64 margin of f); insertions
 * are checked before anything is applied, a deletion that rebuilds tau0 once
 * the new ecc(r) is known.  OVERFLOW from a rebuild and the last three arise
 * while ops are applied: the ops before the failing one stay applied
 * (kc_stats().updates_applied counts them) and the failing one may be partly
 * applied, so the handle should then be destroyed.
 */
kc_status kc_update(kc_graph *g, const kc_edge_op *ops, int64_t n_ops, int32_t mode);

/*
 * Test hook: everything computed for one sample (pool index `sample`).
 * Any output pointer may be NULL.  Arrays have n entries (host memory):
 * parent (parent[r] = -1), depth, DFN in/out (preorder from 0, children in
 * ascending id, out = in + size - 1), vol (subtree volume, int64).  Scalars:
 * f (int64, as stored in the pool), steps (Wilson departures).  With
 * keep_trees the arrays come from the retained parent array, traversed on the
 * current graph; without it they are recomputed on the device from (seed,
 * sample id).  Errors: INVALID_ARG, NOT_RETAINED, OUT_OF_MEMORY, CUDA.
 */
kc_status kc_get_tree(kc_graph *g, int64_t sample, int32_t *parent, int32_t *depth,
                      int32_t *dfn_in, int32_t *dfn_out, int64_t *vol, int64_t *f,
                      int64_t *steps);

/*
 * Copy the pool's per-tree values to host arrays of length count starting at
 * pool index first (any pointer may be NULL): f (int64), weight (fp64),
 * steps (int64), sample id (int64).  Errors: INVALID_ARG, CUDA.
 */
kc_status kc_get_samples(kc_graph *g, int64_t first, int64_t count, int64_t *f, double *weight,
                         int64_t *steps, int64_t *sample_id);

/*
 * The fixed tree tau0 (host arrays of n entries, any may be NULL): parent p0
 * (p0[r] = -1), BFS level, DFN in0/out0; scalars root and ecc(r).
 */
kc_status kc_get_tau0(kc_graph *g, int32_t *p0, int32_t *level, int32_t *in0, int32_t *out0,
                      int32_t *root, int32_t *ecc);

typedef struct {
    int64_t n, m;
    int32_t root, ecc;
    int32_t ttf_variant;         /* resolved KC_TTF_SCAN or KC_TTF_BIT */
    int32_t walker;              /* resolved KC_WALK_LANE or KC_WALK_WARP */
    int64_t pool_trees;          /* trees in the pool                        */
    int64_t next_sample_id;      /* never-reused sample id counter           */
    int64_t total_steps;         /* sum of Wilson departures over all samples */
    int64_t trees_in_flight;     /* wave size used by the last kc_sample      */
    int64_t pool_bytes;          /* device bytes held by the pool            */
    int64_t workspace_bytes;     /* device bytes held by wave workspaces     */
    int64_t updates_applied;
    int64_t trees_resampled;     /* trees replaced or transformed by updates  */
    /* device time (ms, CUDA events on the handle's stream) and launches, per phase */
    double ms_wilson, ms_traverse, ms_ttf, ms_reduce, ms_update, ms_setup, ms_wave_init;
    int64_t launches_wilson, launches_traverse, launches_ttf, launches_reduce,
            launches_update, launches_setup, launches_wave_init;
    /* sums over the pool: exact sum of w=1 f as two int64 limbs, and FP64 moments */
    int64_t f_sum_hi;            /* high limb (signed) of the int128 sum of f */
    uint64_t f_sum_lo;           /* low limb of the int128 sum of f           */
    double wf_sum, w_sum, x2_sum; /* sum w f/(2m), sum w, sum (f/2m)^2 over the pool */
    double last_resistance;      /* R(u,v) used by the last insertion            */
    int64_t last_cg_iters;       /* CG iterations of the last computed R          */
    int32_t traversal;           /* traversal for f: 1 chunked, 2 leaf-to-root      */
    int32_t tuned;               /* 1 once the autotuner has chosen                 */
    double tune_ms[4];           /* autotuner pilots: walk ms per tree (32 walkers,
                                   1 walker), traversal ms per tree (chunked,
                                   leaf-to-root); 0 when not measured              */
    int64_t trees_rejected;      /* trees abandoned by rejection by walk length  */
    int64_t resident_trees;      /* trees the 32-walker kernel runs at once on this
                                   GPU (SMs x resident one-warp blocks).  A wave of
                                   up to this many trees lasts about as long as its
                                   slowest tree, so it is the natural kc_estimate
                                   batch where single trees are slow            */
    /* kc_update wall time by part (ms; each part ends in a stream synchronisation):
       the device graph edit, R(u,v), the tree selection and transformation
       (link-cut / cut-link) or resampling, and the recomputation of f           */
    double ms_update_graph, ms_update_resistance, ms_update_trees, ms_update_refresh;
} kc_stats_t;

kc_status kc_stats(kc_graph *g, kc_stats_t *out);

/* Zero the per-phase timers and launch counters of kc_stats. */
kc_status kc_reset_timers(kc_graph *g);

/*
 * Pool sums of one handle or of several sample-id shards (the exchange step of
 * a sample-sharded multi-GPU run; no counterpart in the paper, which samples
 * on one machine).  f_sum is the exact int128 sum of the unit-weight f(tau) as
 * (signed high, unsigned low) 64-bit limbs, as in kc_stats_t.
 */
typedef struct {
    int64_t f_sum_hi;
    uint64_t f_sum_lo;
    double wf_sum;      /* sum w f / 2m  */
    double w_sum;       /* sum w         */
    double x2_sum;      /* sum (f / 2m)^2 */
    int64_t count;      /* trees         */
} kc_pool_sums;

/*
 * The pool's sums (one reduction on the device, read back on the handle's
 * stream): exact int128 sum of the unit-weight f, FP64 moments, tree count.
 * Errors: INVALID_ARG, CUDA.  An empty pool gives all zeros.
 */
kc_status kc_get_pool_sums(kc_graph *g, kc_pool_sums *out);

/*
 * Combine per-shard sums (host only, no device work): the int128 f sums are
 * added exactly; the FP64 sums are added in array order, so every rank that
 * combines the same gathered array gets the same bits.  Errors: INVALID_ARG
 * (NULL pointers, count < 1, or an int128 overflow of f_sum).
 */
kc_status kc_combine_sums(const kc_pool_sums *parts, int32_t count, kc_pool_sums *out);

/*
 * K_hat from (combined) pool sums (host only): with unit_weights the exact
 * numerator over 2m omega, K_hat = f_sum / (2m count) (Theorem 3, Algorithm 1's
 * last line: one FP64 division of the int128 sum, as kc_estimate does);
 * otherwise the weighted mean sum w f / (2m sum w) (Algorithm 3).
 * Errors: INVALID_ARG (NULL, twom < 2, count < 1, or w_sum <= 0 when weighted).
 */
kc_status kc_estimate_from_sums(const kc_pool_sums *sums, int64_t twom, int32_t unit_weights,
                                double *K_out);

/*
 * Wilson sampling without any device allocation.  (The paper has no
 * counterpart: this is an interface for callers that cannot allocate.)
 *
 * Some callers must not call cudaMalloc when they need trees: code running
 * inside an allocator or memory-pool callback, plugins handed a fixed device
 * budget by their host application, and latency-critical paths that cannot
 * afford the driver allocator's unbounded latency and implicit
 * synchronisation.  This call allocates nothing.  Its only working memory is a
 * fixed array of 8 Mi walker words (64 MiB) compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *
 * It draws n_trees uniform spanning trees rooted at `root` with sample ids
 * first_sample_id .. first_sample_id + n_trees - 1 under `seed`, using the
 * same random-number contract as kc_sample, so the trees and step counts are
 * identical to the ones kc_sample / kc_get_tree produce for those ids.
 *  d_row_off, d_col  device CSR as for kc_graph_create (caller-owned, not checked)
 *  step_cap          per-tree cap on departures (0: max(2^22, 1024 n))
 *  d_parent          device int32[n_trees][n] out: parent of each vertex (-1 at root)
 *  d_steps           device int64[n_trees] out: Wilson departures per tree
 *  d_status          device uint32[1] out: 0, or 1 if a tree hit step_cap or one
 *                    vertex departed 2^25 times (the other samplers' limit)
 *  stream            cudaStream_t to run on (NULL: legacy default stream)
 * Work is enqueued on `stream`; the call returns without synchronising.
 * Requires n * n_trees <= 8 Mi, else KC_ERR_SCRATCH_LIMIT.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call reuses the same array and clears the part it needs; calls that
 * overlap on the GPU (several streams or host threads) race on it and must be
 * serialised by the caller.
 * Errors: INVALID_ARG, SCRATCH_LIMIT, NO_DEVICE, CUDA.
 */
kc_status kc_wilson_noalloc(int64_t n, const int64_t *d_row_off, const int32_t *d_col,
                            int32_t root, uint64_t seed, int64_t first_sample_id,
                            int64_t n_trees, int64_t step_cap, int32_t *d_parent,
                            int64_t *d_steps, uint32_t *d_status, void *stream);

/* Static description of a status code (never NULL). */
const char *kc_status_string(kc_status s);

/* Last CUDA error text seen by this handle (empty if none). */
const char *kc_last_error(kc_graph *g);

#ifdef __cplusplus
}
#endif
#endif /* KC_H */
