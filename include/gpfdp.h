/*
 * gpfdp -- GB300 (sm_103a) fitness evaluation of populations of huge
 * prefix-encoded genetic-programming trees, full and incremental.
 *
 * The method is W. B. Langdon, "A Trillion Genetic Programming
 * Instructions per Second" (arXiv 2205.03251):
 *   - trees are flattened to one byte per node in depth-first prefix order
 *     and kept in fixed-size preallocated buffers (Sec. 3.1, Sec. 5);
 *   - every opcode is interpreted on every test case in one pass over the
 *     tree (Sec. 4.2);
 *   - children are made by subtree crossover, by copying or in place by
 *     shifting the mother's tail (Fig. 1, Fig. 2, Sec. 5), with donated
 *     subtrees copied out before any buffer is overwritten (Sec. 5,
 *     "fatherless" crossover);
 *   - a child is evaluated bottom up from the crossover point, carrying the
 *     mother's evaluation beside it, and evaluation stops at the first node
 *     where both agree on every test case (failed disruption propagation,
 *     Sec. 6.2, Fig. 3).
 *
 * Conventions for every entry point:
 *   - Return GP_OK (0) or a negative GP_E* code; gp_last_error() then holds
 *     a one-line message.  No entry point aborts the process.
 *   - Host pointers (const T* args) are read during the call only; the
 *     library never keeps a caller pointer.  All device memory is owned by
 *     the gp_pop object and released by gp_pop_destroy().
 *   - Work is queued on the stream given to gp_pop_create(); calls return
 *     before the GPU finishes except those documented as synchronising.
 *   - Device-side failures (capacity, budget, bounded waits) are recorded
 *     in a device status word and reported by the next synchronising call.
 *
 * Opcodes (one byte per node):
 *   GP_FP32_ARITH: 0 '+', 1 '-', 2 '*', 3 protected '/', 4 x,
 *                  5..255 constant consts[op-5]; protected '/' gives 1.0
 *                  when the divisor equals zero (+0 or -0), else the IEEE
 *                  single-precision quotient.  Left operand = first child.
 *   GP_BOOL_MUX6:  0 AND, 1 OR, 2 NAND, 3 NOR, 4..9 inputs a0 a1 d0 d1 d2 d3;
 *                  all 64 cases of the 6-multiplexer in one 64-bit word,
 *                  case i having a0 = bit 0 ... d3 = bit 5 of i (Sec. 4.2).
 *   GP_BOOL_MUX11: the same functions, 4..14 inputs a0 a1 a2 d0 .. d7 of the
 *                  11-multiplexer; 2,048 cases bit-packed in 32 words of 64
 *                  bits (Sec. 4.2, widened), case i having input j = bit j
 *                  of i; the target is d[a0 + 2 a1 + 4 a2].
 *   GP_INT32_ARITH: the GP_FP32_ARITH opcodes over 32-bit signed integers:
 *                  + - * wrap around modulo 2^32; protected '/' gives 1 for
 *                  a zero divisor, INT32_MIN for INT32_MIN / -1, else the
 *                  quotient truncated toward zero; consts, x and targets
 *                  hold int32 values (passed through the float pointers).
 * Arithmetic is IEEE binary32 with no contraction into fused multiply-add
 * and no flushing of subnormals.  Fitness is sum_c |root(c) - target(c)|
 * accumulated in case order in binary32 (Boolean: number of wrong cases;
 * integer: the sum exact in 64-bit integers, rounded once to binary32).
 */
#ifndef GPFDP_H
#define GPFDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GP_OK = 0,
    GP_EINVAL = -1,     /* bad argument, malformed tree, bad opcode */
    GP_ENOMEM = -2,     /* device allocation failed or cache budget exceeded */
    GP_ECAPACITY = -3,  /* a tree does not fit its buffer (max_nodes) */
    GP_ECUDA = -4,      /* a CUDA runtime call failed */
    GP_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    GP_ESTATE = -6      /* call out of order (e.g. incremental without crossover) */
};

enum { GP_FP32_ARITH = 0, GP_BOOL_MUX6 = 1, GP_BOOL_MUX11 = 2, GP_INT32_ARITH = 3 };
enum { GP_PACK_NONE = 0, GP_PACK_STATIC = 1, GP_PACK_MLP = 2 };

typedef struct gp_pop gp_pop;

/* Population configuration (all fields by value). */
typedef struct {
    uint32_t pop_size;          /* P individuals (one child per crossover, P children per generation) */
    uint32_t n_cases;           /* C test cases (FP32 and integer sets); ignored for the Boolean sets */
    uint32_t max_nodes;         /* per-tree buffer capacity in nodes (Sec. 4.2: user-set maximum size) */
    uint32_t funcset;           /* GP_FP32_ARITH, GP_BOOL_MUX6, GP_BOOL_MUX11 or GP_INT32_ARITH */
    uint32_t cache_threshold;   /* subtree size from which node values are cached, 2..1024 (default 1024) */
    uint32_t tournament;        /* tournament size (default 7) */
    uint32_t packing;           /* GP_PACK_* order of incremental work */
    uint32_t cases_per_lane;    /* 0 = auto; else 1, 2 or 4 test cases per GPU lane (words for the
                                   Boolean sets; 4 only for GP_FP32_ARITH; GP_BOOL_MUX6 uses 1) */
    uint64_t cache_budget_bytes;/* device bytes for cached value vectors (0 = 40 GiB) */
    uint64_t seed;              /* master seed of every stochastic choice */
    uint32_t walk_warps;        /* 0 = as many as fit; else at most this many warps run the walk */
    uint32_t mlp_lr_micro;      /* Adam learning rate of the packing MLP in 1e-6 units (0 = 1000) */
    uint32_t walk_team;         /* warps per child in the incremental walk: 1, 2, 4, 8, or 0 = auto (4) */
    uint32_t lazy_children;     /* 1 = fitness-first order (Sec. 6.3): the walk reads each child
                                   through its parents, the next generation's plan is drawn
                                   right after it, and only the children selected as parents
                                   get a tree buffer and a cache (in place with lazy_inplace);
                                   results are identical.  0 = build every child at crossover */
    uint32_t arena_buffers;     /* tree buffers of max_nodes bytes: 0 = 2 x pop_size.  Fitness-first
                                   order only, from pop_size + 1 up: a generation holds the buffers
                                   of its parents plus those of the children it selects as the next
                                   parents; one that finds too few free stops (later kernels return
                                   at once) and the next synchronising call reports GP_ECAPACITY,
                                   after which the population must be reloaded (gp_load_trees) */
    uint32_t long_walks;        /* the first long_walks children of the work order (the longest predicted
                                   walks, Sec. 3 and Sec. 4.1: the longest tasks first) are walked by teams
                                   of 16 warps (8 when 16 do not fit shared memory), beside the teams of
                                   walk_team warps that walk the others: 0 (or 0xFFFFFFFF) = none */
    uint32_t onepass_nodes;     /* children of at most this many nodes are interpreted in one pass
                                   instead of walked level by level (same values, bit for bit; the
                                   walk pays per level, a small child with a deep crossover point has
                                   many levels): 0 = 4,096 (the most allowed), 0xFFFFFFFF = none */
    uint32_t stack_window;      /* interpreter stack entries per warp kept in shared memory (deeper ones
                                   go to a slower per-warp global area): 0 = 16, or 16, 32, 64.  Deep
                                   trees (uniform random binary trees of n nodes need about 2 sqrt(n)
                                   entries) want more; each entry costs 128 x cases_per_lane bytes per
                                   warp of shared memory.  GP_EINVAL when the kernels' shared memory
                                   does not fit */
    uint32_t lazy_inplace;      /* fitness-first order only: 1 = memory-lean (Sec. 5, Fig. 2): the last
                                   child that the next tournaments select of each mother takes her
                                   buffer and is built there in place, whatever its size change, at the
                                   start of the next gp_crossover (until then it is read through its
                                   parents, as the children that are not built are); the other selected
                                   children are copied.  A generation then needs about P + (selected
                                   children - their distinct mothers) buffers.  0 = copy every selected
                                   child (beside the cache update, off the critical path) */
} gp_config;

/* Per-call statistics of the last evaluation (host copy). */
typedef struct {
    uint64_t equivalent_ops;    /* sum of tree sizes x cases: every opcode on every case (Sec. 1) */
    uint64_t actual_ops;        /* opcodes actually interpreted x cases */
    uint64_t interp_ops;        /* of which by the subtree interpreter kernel */
    uint64_t crossover_bytes;   /* algorithmic bytes moved by the last crossover */
    uint64_t cache_entries;     /* cached nodes (subtree >= threshold) after the call */
    uint64_t path_levels;       /* sum over children of levels walked above the crossover point */
    uint32_t stopped;           /* children whose walk stopped below the root (fitness inherited) */
    uint32_t children;          /* children evaluated */
    uint32_t launches;          /* kernels launched by the call */
    uint32_t cum_calls;         /* evaluations since profiling was (re)enabled */
    uint64_t cum_equivalent_ops;/* sums of the three counters above over those calls */
    uint64_t cum_actual_ops;
    uint64_t cum_crossover_bytes;
    float    ms[10];            /* per-phase device milliseconds when profiling is on, mean over
                                   the calls since profiling was (re)enabled (last 128 kept):
                                   structure, items, skeleton, fitness, crossover, walk, cache, pack,
                                   materialise (fitness-first order: copies of the children selected
                                   as parents), plan (fitness-first order: the next generation's
                                   selection and crossover points, buffers for the selected) */
} gp_stats;

/*
 * Create a population from host data.  x and targets hold n_cases floats
 * (int32 values for GP_INT32_ARITH; ignored for the Boolean sets); consts
 * holds 251 floats (int32 values for GP_INT32_ARITH); tree i is
 * ops[offsets[i] .. offsets[i+1]) (offsets has pop_size+1 entries).  Each
 * tree must be a complete prefix expression with valid opcodes and at most
 * max_nodes nodes.  `stream` is a cudaStream_t (NULL = legacy default);
 * the caller keeps it alive until gp_pop_destroy().  Synchronising.
 */
int gp_pop_create(const gp_config* cfg, const float* x, const float* targets, const float* consts,
                  const uint8_t* ops, const uint64_t* offsets, void* stream, gp_pop** out);

void gp_pop_destroy(gp_pop* pop);

/*
 * Replace the trees of an existing population with pop_size new ones from
 * host memory (same layout and rules as gp_pop_create; pinned host memory
 * makes the copy asynchronous).  Cached values become stale until the next
 * gp_eval_full().  The host buffers must stay valid until the stream
 * reaches this point (synchronise, or call gp_fitness).
 */
int gp_load_trees(gp_pop* pop, const uint8_t* ops, const uint64_t* offsets);

/* Message for the last failed call on pop (or on creation when pop is NULL). */
const char* gp_last_error(const gp_pop* pop);

/*
 * Full interpretation (Sec. 4.2): every tree on every test case.  Builds
 * the tree structure pass, evaluates all subtrees below the cache
 * threshold, then the cached nodes bottom up, writes the value vector of
 * every node whose subtree has >= cache_threshold nodes (and of each root)
 * to the cache, and the fitness of every tree.  Asynchronous.
 */
int gp_eval_full(gp_pop* pop);

/*
 * Breed the next generation (Sec. 5, Sec. 6.3): tournament selection of a
 * mother and a father per child, crossover points uniform over all nodes,
 * donated subtrees copied out first, then each child is materialised --
 * by copying into a free buffer (Fig. 1) or, for the last child of a
 * mother, in place by moving the mother's tail (Fig. 2).  All draws are a
 * function of (seed, generation, child, k).  The parents' cached values
 * are retained for gp_eval_incremental().  Asynchronous.
 */
int gp_crossover(gp_pop* pop, uint32_t generation);

/*
 * Incremental evaluation of the children of the last gp_crossover()
 * (Sec. 6.2, Fig. 3): from the crossover point towards the root, carrying
 * the mother's values beside the child's, stopping where both agree on all
 * cases bit for bit.  Leaves the children's fitness and cache in place of
 * the parents'.  `stats` may be NULL; when given the call synchronises.
 */
int gp_eval_incremental(gp_pop* pop, gp_stats* stats);

/* Copy P fitness values to host (FP32; Boolean: error counts as float).
 * Synchronising. */
int gp_fitness(const gp_pop* pop, float* host_out, uint32_t n);

/* Copy the root value vectors to host: P x n_cases 32-bit values (binary32
 * or int32), or for the Boolean sets P x (cases / 64) uint64 words.  A
 * child that keeps no cache (fitness-first order, not selected as a
 * parent) reads as NaN (binary32), 0x7FC00000 (int32) or 0 (Boolean).
 * `bytes` is the size of host_out.  Synchronising. */
int gp_root_values(const gp_pop* pop, void* host_out, size_t bytes);

/* Copy tree i (its size into *size) to host_out of capacity cap bytes;
 * host_out may be NULL to ask for the size only.  A child of the
 * fitness-first order that is not built (or built in its mother's buffer
 * only at the next crossover) is assembled from its parents (Fig. 1) by a
 * kernel on the population's stream.  GP_EINVAL if cap is smaller than the
 * tree, GP_ESTATE if its parents' buffers were given to other trees.
 * Synchronising. */
int gp_get_tree(const gp_pop* pop, uint32_t i, uint8_t* host_out, uint64_t cap, uint64_t* size);

/* Cached nodes of tree i: up to nmax entries of (position, subtree end,
 * parent entry index or -1), sorted by position; *n = count.  Any output
 * pointer may be NULL.  Synchronising. */
int gp_cache_entries(const gp_pop* pop, uint32_t i, uint32_t* pos, uint32_t* end, int32_t* parent,
                     uint32_t nmax, uint32_t* n);

/* Value vector of cache entry j of tree i (n_cases 32-bit values, or
 * cases / 64 uint64 words for the Boolean sets) to host.  Synchronising. */
int gp_cache_value(const gp_pop* pop, uint32_t i, uint32_t j, void* host_out, size_t bytes);

/* Per child of the last gp_eval_incremental: the level at which the walk
 * stopped (0 = at the crossover point; -1 = the root differed, fitness
 * recomputed; -2 = a child of at most onepass_nodes nodes, evaluated in one
 * pass instead of walked -- same fitness bits) and the number of levels
 * evaluated above the crossover point.  Either pointer may be NULL; n <=
 * pop_size.  Synchronising. */
int gp_walk_info(const gp_pop* pop, int32_t* stop_level, uint32_t* levels, uint32_t n);

/*
 * Disruption diagnostics (Fig. 4 and the walk of Sec. 6.2): how far a
 * crossover's change of the test-case values travels up the chain of
 * ancestors of the crossover point before it dies out.
 *
 * One record per child and walk level, level 0 being the crossover point
 * and level j its j-th ancestor, for the levels the walk compares (up to and
 * including the stop level, or up to the root):
 *   disrupted  cases whose child value differs from the mother's value at
 *              that node (bit patterns; Boolean: differing bits of the
 *              64-case word);
 *   finite     those of them where both values are finite (Boolean: all);
 *   sum_sq     sum over the finite ones of (child - mother)^2, each
 *              difference and square in binary64 (Boolean: 1 per case), so
 *              the RMS difference of the disrupted cases is
 *              sqrt(sum_sq / finite).  The summation order is not fixed:
 *              two runs agree bit for bit, the CPU definition to within
 *              2 (C - 1) binary64 roundings (every term is >= 0).
 * The record at the stop level has disrupted == 0.  A clone of its mother
 * has one record (level 0, zeros).
 */
typedef struct {
    uint32_t disrupted;
    uint32_t finite;
    double sum_sq;
} gp_disruption_level;

/* Record up to max_levels levels per child in the following incremental
 * evaluations (0 turns recording off and frees the records).  Allocates
 * pop_size * max_levels records of 16 bytes.  While recording, children
 * smaller than the cache threshold are walked level by level instead of
 * being evaluated in one pass (same fitness, trees and cache).  Drops a
 * captured graph (capture again afterwards).  Synchronising.  GP_EINVAL for
 * max_levels > 65,536, GP_ENOMEM when the records do not fit. */
int gp_set_disruption(gp_pop* pop, uint32_t max_levels);

/* Records of the last gp_eval_incremental (or graph replay) that ran with
 * recording on: records[i * max_levels + j] for child i and level j <
 * n_levels[i] (min(levels walked + 1, max_levels); 0 when the child's walk
 * failed).  `n` = pop_size * max_levels records must fit in records;
 * n_levels holds pop_size entries; either pointer may be NULL.  GP_ESTATE
 * when no such evaluation has run since recording was last set.
 * Synchronising. */
int gp_disruption(const gp_pop* pop, gp_disruption_level* records, size_t n, uint32_t* n_levels);

/*
 * Work packing of the last gp_eval_incremental (Sec. 3 and Sec. 4.1 of
 * the paper: run the longest tasks first; one slow evaluation holds up the
 * population).  Per child: the packing MLP's prediction of
 * log2(1 + levels walked) made before the walk, the measured value, the
 * static packing key log2(1 + mother size), and the walk queue (order[k] =
 * child walked k-th); *loss = mean squared error of the training step that
 * followed the walk.  Any pointer may be NULL; n <= pop_size.
 * Synchronising.
 */
int gp_pack_info(const gp_pop* pop, float* predicted, float* measured, float* size_key, uint32_t* order,
                 uint32_t n, float* loss);

/*
 * Loss and gradient of the packing MLP (16 -> 64 -> 64 -> 1, ReLU) on the
 * GPU for given host weights w (5,313 floats: W1[64][16], b1[64],
 * W2[64][64], b2[64], w3[64], b3), features x (n x 16) and targets y (n):
 * loss = mean (f(x) - y)^2, grad = d loss / d w.  Uses the same kernels as
 * the online training; allocates and frees its own device buffers.
 * Synchronising.
 */
int gp_mlp_eval_grad(const float* w, const float* x, const float* y, uint32_t n, float* loss, float* grad);

/* Statistics of the last gp_eval_full / gp_eval_incremental.  Synchronising. */
int gp_get_stats(const gp_pop* pop, gp_stats* out);

/*
 * Graph mode (on = 1): size both cache sets for reserve_entries cached
 * nodes (exactly that many when nonzero; 0 = at least twice the current
 * count plus 64 per tree) and stop the host-side regrowing, so that
 * gp_crossover, gp_eval_incremental (with stats NULL) and gp_eval_full
 * issue no synchronising call and can be captured into a CUDA graph on the
 * population's stream (gp_graph_capture).  A cache that outgrows the
 * reservation stops every later kernel and is reported as GP_ENOMEM by the
 * next synchronising call; the population must then be reloaded.  If the
 * current population's cache set was resized it must be evaluated again
 * (gp_eval_full) before the next gp_crossover.  on = 0 restores regrowing
 * and drops a captured graph.  Synchronising.
 */
int gp_set_graph_mode(gp_pop* pop, int on, uint64_t reserve_entries);

/*
 * Capture n_generations (even, >= 2) generations -- gp_crossover then
 * gp_eval_incremental each -- into one CUDA graph on the population's
 * stream.  Nothing runs during the capture.  Each gp_graph_launch replays
 * them: the r-th replay (r = 0, 1, ...) breeds generations
 * first_generation + r * n_generations + k, k = 0 .. n_generations - 1, so
 * replays give the same populations, bit for bit, as the eager calls with
 * those generation numbers.  Needs graph mode and an evaluated population;
 * a later cache regrow or gp_set_graph_mode(pop, 0, 0) drops the graph.
 * gp_graph_launch is asynchronous; errors raised by the replayed kernels
 * (e.g. GP_ENOMEM when the reservation is exceeded, after which the
 * population must be reloaded) surface at the next synchronising call.
 */
int gp_graph_capture(gp_pop* pop, uint32_t first_generation, uint32_t n_generations);
int gp_graph_launch(gp_pop* pop);

/* One autotuner candidate and what it measured. */
typedef struct {
    uint32_t cases_per_lane;    /* K: test cases per lane, i.e. 32 x K cases per warp task */
    uint32_t cache_threshold;   /* T: subtree size from which values are cached (the subtree split) */
    uint32_t walk_team;         /* warps per child in the incremental walk */
    uint32_t stack_window;      /* interpreter stack entries kept in shared memory */
    int32_t  status;            /* GP_OK, or the error that ruled the candidate out */
    uint32_t identical;         /* 1 when its fitness equals the first valid candidate's, bit for bit */
    float    ms_full;           /* one gp_eval_full, device milliseconds */
    float    ms_generation;     /* one generation (crossover + incremental), mean over a graph replay */
} gp_tune_result;

/*
 * Autotune the work splits for a population: for every combination of
 * ks[0..n_k) x ts[0..n_t) x teams[0..n_team) x ws[0..n_w) (cases_per_lane
 * x cache_threshold x walk_team x stack_window; ws may be NULL with n_w = 0:
 * base's stack window only) build the population described by base and
 * the host data (same rules as gp_pop_create), time one gp_eval_full and,
 * when generations > 0 (even), one replay of a captured graph of that many
 * generations (after four warm-up replays), and check that its fitness
 * matches the first candidate's bit for bit.
 * results[((a * n_t + b) * n_team + w) * max(n_w, 1) + v] receives candidate
 * (ks[a], ts[b], teams[w], ws[v]); *best = base with the fastest valid
 * candidate's four fields (fastest per generation when generations > 0,
 * else fastest full evaluation).  One candidate's population exists at a
 * time.  Synchronising.  Returns GP_ENOMEM when no candidate could run.
 * The paper has no counterpart: its CPU interpreter has one fixed layout.
 */
int gp_autotune(const gp_config* base, const float* x, const float* targets, const float* consts,
                const uint8_t* ops, const uint64_t* offsets, const uint32_t* ks, uint32_t n_k,
                const uint32_t* ts, uint32_t n_t, const uint32_t* teams, uint32_t n_team,
                const uint32_t* ws, uint32_t n_w, uint32_t generations, void* stream,
                gp_tune_result* results, gp_config* best);

/* The autotuner's choice rule on its own: index of the fastest candidate
 * with status GP_OK and identical = 1 (ties: the earlier), or -1. */
int gp_autotune_pick(const gp_tune_result* results, uint32_t n, uint32_t generations);

/*
 * Bound the polls of every wait inside an incremental-walk team (the
 * combining warp waiting for a sibling's values, an evaluator waiting for the
 * next level's descriptor; Sec. 6.2 walk, evaluated by a team of warps).
 * polls = 0 restores the default of 2^22 polls of about 64 ns each.  A wait
 * that runs out ends the team's walk of that child, the team goes on, and
 * the next synchronising call reports GP_ETIMEOUT; the population must then
 * be reloaded (gp_load_trees, gp_eval_full).  Meant for testing that every
 * device wait returns.  Drops a captured graph.  Synchronising.
 */
int gp_set_wait_limit(gp_pop* pop, uint32_t polls);

/*
 * Measured issue rate of the plain ALU operations the interpreters are made
 * of, on the current device: kind 0 binary32 add, 1 32-bit three-input
 * logic (the Boolean sets' AND/OR/NAND/NOR words); GP_EINVAL for others.
 * *lane_ops_per_s receives lane operations per second over all SMs (the
 * roofline of an interpreter that spends one lane operation per opcode and
 * test case, Sec. 4.2).  The paper has no counterpart.  Allocates 16 bytes
 * of device memory for the duration of the call.  Synchronising.
 */
int gp_alu_peak(int kind, double* lane_ops_per_s);

/* Turn per-phase CUDA-event timing on (1) or off (0); either resets the
 * recorded phase times. */
int gp_set_profiling(gp_pop* pop, int on);

/*
 * Full evaluation of a batch of small trees without any device allocation.
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc -- a plug-in whose host process has handed the device
 * memory to its own pool allocator, a real-time loop that must not take the
 * device synchronisation an allocation can bring, or an embedding whose
 * memory is fixed at start-up.
 * All pointers but status_out are device pointers owned by the caller:
 *   d_ops      16-byte aligned opcodes; tree i is d_ops[d_off[i] .. d_off[i+1]);
 *              ops_bytes (a multiple of 16) must cover every tree
 *   d_off      n_trees + 1 uint64 offsets; each tree 1..1023 nodes
 *   d_x, d_t   n_cases inputs and targets (1 <= n_cases <= 4096); d_consts 251 floats
 *   d_values   out: n_trees x n_cases root values (row per tree)
 *   d_fitness  out: n_trees fitness values (sum of |value - target| in case order)
 * Same arithmetic as gp_eval_full.  Scratch (the interpreter's deep-stack
 * overflow for 64 warps, a work counter, a status word) lives in one
 * file-scope device array of about 8.5 MB that every GPU loading the library
 * holds until exit.  The first call on a device (and the first after that
 * device's context was re-created) looks up the array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  Every call shares the array: calls whose GPU
 * work overlaps (other streams, or not yet finished) race and must be
 * serialised.  Each call clears its counter and status word first, and
 * synchronises its stream before returning.  Returns GP_EINVAL for bad
 * arguments or a malformed tree, GP_ECAPACITY when a tree is empty, larger
 * than 1023 nodes or outside ops_bytes; *status_out (host, may be NULL) gets
 * the raw flags (1: size or bounds, 2: malformed tree).
 */
int gp_eval_small_noalloc(const uint8_t* d_ops, size_t ops_bytes, const uint64_t* d_off, uint32_t n_trees,
                          const float* d_x, const float* d_t, const float* d_consts, uint32_t n_cases,
                          float* d_values, float* d_fitness, void* stream, uint32_t* status_out);

#ifdef __cplusplus
}
#endif
#endif /* GPFDP_H */
