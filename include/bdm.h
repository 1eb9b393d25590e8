/*
 * bdm.h -- C ABI of the GB300 (sm_103a) mechanical-interaction iteration for
 * spherical agents, after BioDynaMo (Breitwieser et al., PPoPP'23,
 * arXiv 2301.06984).
 *
 * One iteration (Algorithm 1 of the paper, specialised to the mechanics
 * operation) is, in this order:
 *   1. on sort steps, a stable reorder of the agents by the Morton code of
 *      their uniform-grid box (Sec. 4.2, agent sorting);
 *   2. the uniform-grid build on the current positions (Sec. 3.1): box edge
 *      L >= R, per-axis box floor((p - lo) / L), a one-box margin so that every
 *      3x3x3 stencil stays inside, agents of a box in ascending storage index;
 *   3. static-agent detection (Sec. 5, conditions i-iv, made box-granular);
 *   4. for every non-static agent, the sum over the 27 surrounding boxes of the
 *      overlap force F = k*delta - gamma*sqrt(rbar*delta) along the centre line
 *      (delta = r_i + r_j - d > 0, rbar = r_i r_j / (r_i + r_j); the paper
 *      defers to the Cortex3D force without a formula, Sec. 5), for neighbours
 *      with d^2 < R^2, j != i; displacement dt * sum F unless |sum F| <=
 *      adherence, clamped to max_displacement; every force reads the
 *      positions at the start of the iteration;
 *   5. behaviours: random walk (added after the clamp), growth, and division
 *      into two daughters;
 *   6. the parallel merge of the daughters (Sec. 3.2, additions committed at
 *      the end of the iteration): daughter slot = n + (number of dividing
 *      agents with a smaller storage index), uid = next_uid + that rank.
 *
 * Memory: the simulation owns all device memory it uses (sized at
 * bdm_create / bdm_set_agents from `capacity`); it never keeps a pointer the
 * caller passed.  Pointers tagged BDM_DEVICE must be device memory valid on
 * the simulation's stream; pointers tagged BDM_HOST are host memory (pinned
 * memory makes the copies asynchronous).  Agent arrays are structure-of-arrays
 * in storage order.
 *
 * Errors: every int-returning call returns BDM_OK (0) or a negative BDM_E*
 * code, and bdm_last_error() gives a message.  A failed bdm_step leaves the
 * state of the last completed iteration.  Calls on one simulation are not
 * thread-safe; different simulations are independent.
 */
#ifndef BDM_H
#define BDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BDM_OK 0
#define BDM_EINVAL (-1)    /* bad argument (NULL, negative size, non-finite input, L < R) */
#define BDM_ENOMEM (-2)    /* device or host allocation failed                             */
#define BDM_ECUDA (-3)     /* a CUDA call failed (message holds the CUDA error string)     */
#define BDM_ECAPACITY (-4) /* agents (with daughters) would exceed `capacity`              */
#define BDM_ETIMEOUT (-5)  /* reserved: no kernel of this library waits, so none returns it  */
#define BDM_ESTATE (-6)    /* call out of order (e.g. bdm_step before bdm_set_agents)       */

/* precision forms */
#define BDM_FP64 0       /* all pair arithmetic in FP64; bit-identical to the FP64 oracle */
#define BDM_FP32_FORCE 1 /* FP32 pair arithmetic and accumulation; FP64 cutoff predicate,
                            FP64 contact decision and FP64 positions; diameters in FP32  */

/* space-filling curves of the agent order */
#define BDM_CURVE_MORTON 0
#define BDM_CURVE_HILBERT 1

/* memory tags */
#define BDM_HOST 0
#define BDM_DEVICE 1

/* per-agent behaviour bits */
#define BDM_BEH_GROW 1u /* volume += growth_per_step; divide at divide_volume     */
#define BDM_BEH_WALK 2u /* random walk of walk_step um after the clamp            */
#define BDM_BEH_DIE 4u  /* removed with probability death_prob per iteration     */
#define BDM_TYPE_SHIFT 4 /* bits 4-5 of the behaviour byte: the agent's type (0-3) */

typedef struct bdm_sim bdm_sim;

typedef struct {
  double interaction_radius; /* R (um); neighbour iff d^2 < R^2 (strict), j != i      */
  double box_edge;           /* L (um) >= R; 0 selects L = R                          */
  double dt;                 /* time step (used when dt_per_sim is NULL)              */
  double max_displacement;   /* clamp of |dt * sum F| (um)                            */
  double k, gamma;           /* force constants (2, 1)                                */
  double adherence;          /* no displacement while |sum F| <= adherence (0)        */
  int32_t precision;         /* BDM_FP64 or BDM_FP32_FORCE                            */
  int32_t detect_static;     /* skip agents proven static (Sec. 5)                    */
  int32_t sort_every;        /* Morton reorder when step % sort_every == 0; 0 = never */
  int32_t n_sims;            /* >= 1: independent simulations advanced together       */
  const double *dt_per_sim;  /* host array of n_sims time steps, or NULL              */
  uint64_t seed;             /* Philox4x64-10 key of all in-iteration random draws     */
  double growth_per_step;    /* um^3 added per iteration to BDM_BEH_GROW agents       */
  double divide_volume;      /* divide when the grown volume >= this (um^3)           */
  double ratio_lo, ratio_hi; /* daughter volume ratio uniform in [lo, hi)             */
  double walk_step;          /* um per iteration for BDM_BEH_WALK agents              */
  int64_t capacity;          /* maximum number of agents, daughters included          */
  int32_t keep_forces;       /* 1: keep each iteration's summed forces (debug output) */
  int32_t reserved;
  double death_prob;         /* probability that a BDM_BEH_DIE agent is removed in an
                                iteration (0 = no removal)                           */
  int32_t n_types;           /* 0 or 1: k and gamma for every pair; 2..4: the pair of
                                agent types (a, b) uses type_k[4 a + b] and
                                type_gamma[4 a + b] (Sec. 6.5 cell sorting:
                                differential adhesion); the type is bits 4-5 of
                                the agent's behaviour byte (BDM_TYPE_SHIFT)          */
  int32_t curve;             /* order of the grid and of sort steps (Sec. 4.2):
                                BDM_CURVE_MORTON (0) or BDM_CURVE_HILBERT (1): the
                                4x4x4-box bricks along a Hilbert curve, the boxes
                                inside a brick in Morton order                      */
  double type_k[16];         /* symmetric, finite, >= 0 over the first n_types rows;
                                entries of types >= n_types are used as given       */
  double type_gamma[16];
} bdm_params;

typedef struct {
  int64_t n_agents;           /* current number of agents                          */
  int64_t step;               /* iterations completed                              */
  uint64_t next_uid;          /* uid the next daughter receives                    */
  int64_t n_static;           /* agents skipped as static in the last iteration     */
  int64_t n_moved;            /* agents whose position changed                     */
  int64_t n_divided;          /* divisions in the last iteration                   */
  int64_t n_candidates;       /* pairs examined in the 27-box stencils             */
  int64_t n_neighbors;        /* pairs with d^2 < R^2                              */
  int64_t n_contacts;         /* neighbour pairs with delta > 0                    */
  int64_t n_exact_fallback;   /* FP32 form: pairs decided by the FP64 path          */
  int64_t n_boxes;            /* boxes of the grid (all simulations)               */
  int64_t n_bricks;           /* 4x4x4-box bricks of the grid                      */
  int64_t n_occupied_bricks;  /* bricks holding at least one agent                 */
  int64_t max_brick_agents;   /* most agents in one brick                          */
  int64_t kernels_launched;   /* CUDA kernels this simulation has launched so far   */
  int32_t history_valid;      /* static detection has the previous iteration       */
  int32_t error;              /* sticky device error word (0 = none)               */
  int64_t n_removed;          /* agents removed in the last iteration              */
  int64_t n_fp64_fixup;       /* FP32 form: agents the FP64 fix-up pass evaluated  */
} bdm_counters;

/* Create a simulation: the parameters of the paper's problem statement
 * (Sec. 3.1: interaction radius R and box edge L >= R of the uniform grid;
 * Sec. 5: the mechanical force, the time step, the static-agent switch
 * detect_static and the force threshold "adherence"; Sec. 4.2: the agent
 * sorting frequency sort_every; Sec. 3.2: the capacity that additions by
 * division may fill).  `stream` is a cudaStream_t (NULL = legacy default
 * stream); all work of this simulation is ordered on it.  On success *out
 * owns device memory for params->capacity agents.
 * Errors: BDM_EINVAL (R <= 0, L < R, n_sims < 1, capacity < 1, precision
 * unknown, growth with n_sims > 1 or with BDM_FP32_FORCE), BDM_ENOMEM,
 * BDM_ECUDA. */
int bdm_create(const bdm_params *params, void *stream, bdm_sim **out);

/* Replace the agent population (the paper's model initialisation, Algorithm
 * 1).  xyz: 3 x n doubles (x[0..n), y[0..n), z[0..n)); diam: n doubles (um;
 * rounded to float in BDM_FP32_FORCE); vol: n doubles or NULL (= pi/6 d^3);
 * uid: n or NULL (= 0..n-1); behavior: n bytes of BDM_BEH_* bits or NULL
 * (= BDM_BEH_GROW if growth_per_step > 0, plus BDM_BEH_WALK if walk_step >
 * 0); sim_offsets: n_sims + 1 increasing offsets starting at 0 and ending at
 * n, or NULL when n_sims == 1; step and next_uid restore the iteration counter
 * and the uid counter (checkpoint/resume).  The history of static detection
 * starts empty, so no agent is static in the first iteration after this call.
 * The call returns when the population is set (or refused).
 * Errors: BDM_EINVAL (n < 0, NULL xyz/diam with n > 0, a coordinate that is
 * not finite or not within +-1e9 um, a diameter that is not finite or not in
 * (0, 1e6) um, bad offsets; no agents are set then), BDM_ECAPACITY
 * (n > capacity), BDM_ECUDA. */
int bdm_set_agents(bdm_sim *sim, int64_t n, const double *xyz, const double *diam, const double *vol,
                   const uint64_t *uid, const uint8_t *behavior, const int64_t *sim_offsets, int64_t step,
                   uint64_t next_uid, int mem);

/* Advance n_steps iterations of the simulation loop (Algorithm 1 with the
 * mechanical operation as its only agent operation: the six steps listed at
 * the top of this header, i.e. Sec. 4.2 sorting when due, the Sec. 3.1 grid
 * build, Sec. 5 static detection, force and displacement, behaviours, and
 * the Sec. 3.2 commit of additions at the end of the iteration).  The
 * per-iteration work is one captured CUDA graph replayed on the simulation's
 * stream.  Blocks until the iterations
 * are done and the device counters are read back.  Errors: BDM_ESTATE (no
 * agents set), BDM_EINVAL (n_steps < 0), BDM_ECAPACITY (daughters would
 * exceed capacity; the state is that of the last completed iteration),
 * BDM_ECUDA. */
int bdm_step(bdm_sim *sim, int n_steps);

/* Reorder the agents now by the Morton code of their box in the grid of the
 * current positions (stable: equal codes keep storage order), as a sort step
 * does.  Errors: BDM_ESTATE, BDM_ECUDA. */
int bdm_sort(bdm_sim *sim);

/* Copy the state out (storage order): the agent attributes the resource
 * manager holds (Sec. 3.2; after sort steps, storage is in the Morton order
 * of Sec. 4.2), with the iteration and uid counters needed to resume (the
 * paper has no checkpoint call; this is its model state).  Any output
 * pointer may be NULL.  cap
 * is the number of agents the arrays hold (xyz holds 3 x cap, x at 0, y at
 * cap, z at 2 cap); sim_offsets holds n_sims + 1.  *n_out gets the number of
 * agents.  Errors: BDM_ECAPACITY (cap < n; nothing written but *n_out),
 * BDM_EINVAL, BDM_ECUDA. */
int bdm_get_agents(bdm_sim *sim, int64_t cap, double *xyz, double *diam, double *vol, uint64_t *uid,
                   uint8_t *behavior, int64_t *sim_offsets, int64_t *n_out, int64_t *step, uint64_t *next_uid,
                   int mem);

/* Counters of the last iteration (host struct).  Errors: BDM_EINVAL, BDM_ECUDA. */
int bdm_get_counters(bdm_sim *sim, bdm_counters *out);

/* Diagnostic outputs: the intermediate results of one iteration that the
 * paper defines -- the summed force and contact count of the mechanical
 * operation (Sec. 5), the static flags (Sec. 5, conditions i-iv), the uniform
 * grid's boxes, geometry and agent order (Sec. 3.1), the Morton ranks of the
 * gap/offset mapping (Sec. 4.2) and the neighbour sets of the 27-box search
 * (Sec. 3.1).  `out` is always host memory.  `what`:
 *   BDM_DBG_FORCES       double 3 x n: summed force of the last iteration
 *                        (needs keep_forces; 0 for static agents)
 *   BDM_DBG_NZ           int32 n: contacts (delta > 0) of the last iteration,
 *                        saturated at 65535
 *   BDM_DBG_STATIC       uint8 n: 1 if the agent was skipped as static
 *   BDM_DBG_GRID_BOX     int32 3 x n: box coordinates of each agent in the grid
 *                        the next iteration builds
 *   BDM_DBG_GRID_ORDER   int64 n: storage indices in grid order (Morton order
 *                        of the boxes, ascending storage index inside a box)
 *   BDM_DBG_GRID_GEOMETRY double 6 x n_sims: lo[3] then box counts[3]
 *   BDM_DBG_BRICK_RANK   int64 n: Morton rank of each agent's 4x4x4 brick
 *                        among the bricks of its simulation's grid
 *   BDM_DBG_NEIGHBORS    int64: n + 1 CSR offsets then the neighbour storage
 *                        indices of every agent in the canonical stencil order
 *   BDM_DBG_FORCES_NOW   double 3 x n then int32 n (contacts) then int32 n
 *                        (neighbours): forces on the current state without
 *                        moving anything and without the static skip; cap and
 *                        *n_out count 8-byte words (4 n)
 * cap is the capacity of `out` in elements of its type; *n_out gets the number
 * of elements needed.  Errors: BDM_ECAPACITY (cap too small; nothing written),
 * BDM_EINVAL, BDM_ESTATE, BDM_ECUDA. */
#define BDM_DBG_FORCES 1
#define BDM_DBG_NZ 2
#define BDM_DBG_STATIC 3
#define BDM_DBG_GRID_BOX 4
#define BDM_DBG_GRID_ORDER 5
#define BDM_DBG_GRID_GEOMETRY 6
#define BDM_DBG_BRICK_RANK 7
#define BDM_DBG_NEIGHBORS 8
#define BDM_DBG_FORCES_NOW 9
int bdm_get_debug(bdm_sim *sim, int what, void *out, int64_t cap, int64_t *n_out);

/* Autotuner.  Times `trial_steps` iterations of the production path (after
 * one warm-up iteration) for each candidate setting, restoring the state
 * before every trial, and keeps the fastest: the box edge L in {R, 1.125 R,
 * 1.25 R, 1.5 R} (BDM_TUNE_BOX_EDGE), the FP32-force kernel in {the hybrid
 * launch, 4 lanes per agent, the sparse kernel, the tiled kernel}
 * (BDM_TUNE_LANES; the values -4, 4, -3, 0 of bdm_set_force_kernel), and the sort
 * cadence in {current, 0, 5, 10, 20} (BDM_TUNE_SORT), one dimension after the
 * other.  The state (agents, step, uid counter) is the same afterwards; the
 * static-detection history starts empty.  Changing L keeps neighbour sets
 * exact (any L >= R does) but changes the FP64 form's canonical summation
 * order.  Errors: BDM_ESTATE (no agents), BDM_EINVAL, BDM_ENOMEM, BDM_ECUDA. */
#define BDM_TUNE_BOX_EDGE 1
#define BDM_TUNE_LANES 2
#define BDM_TUNE_SORT 4
typedef struct {
  double box_edge;     /* chosen L (um)                                     */
  double ms_per_step;  /* measured time per iteration of the chosen setting */
  int32_t lanes;       /* FP32 kernel choice, as in bdm_set_force_kernel    */
  int32_t sort_every;  /* chosen sort cadence                               */
  int32_t n_trials;    /* settings timed                                    */
  int32_t reserved;
} bdm_tuning;
int bdm_autotune(bdm_sim *sim, int trial_steps, int what, bdm_tuning *out);

/* FP32-force kernel choice (no counterpart in the paper, whose force loop is
 * one thread per agent).  lanes = 1, 2, 4, 8, 16 or 32 selects the
 * lane-per-agent kernel: a warp takes a box's agents, that many lanes split
 * each agent's candidates, and each lane queues its prefiltered pairs before
 * evaluating them (with 4, the lanes follow the agents still to do in the
 * box: 2 while 11 or more are left, 8 to 32 for a last pass of 4 or
 * fewer);
 * agents whose FP32 error bound is not small against their
 * tolerance are finished by a fix-up pass.  lanes = -1 selects the same kernel
 * with the lanes chosen per box by a cost model.  lanes = 0 selects the tiled
 * kernel: a warp tests all of a box's agents against each staged chunk of the
 * 27-box stencil (one lane per candidate), collects the pairs that pass in a
 * shared list and evaluates the list 32 pairs per warp instruction.  lanes =
 * -3 selects the sparse kernel: one warp per brick, one lane per agent walking
 * its own 27-box stencil (for tissue of one to a few agents per box).  The
 * tiled and sparse kernels evaluate every contact the FP32 error analysis does
 * not cover in double-float arithmetic in place, so they need no fix-up pass.
 * lanes = -4 (the default) selects the hybrid launch: the sparse kernel for the
 * bricks of fewer than 192 agents, the lane-per-agent kernel with 4 lanes for
 * the others.  All give the same neighbour and contact decisions (FP64-exact)
 * and forces within the FP32-form tolerance; the choice takes effect at the
 * next iteration.  No effect on the FP64 form.  Errors: BDM_EINVAL (other lanes
 * values). */
int bdm_set_force_kernel(bdm_sim *sim, int lanes);

/* Phase profiling.  After bdm_profile_begin, bdm_step launches each
 * iteration kernel by kernel (no graph) with a CUDA event before every phase
 * on the simulation's stream; bdm_profile_end waits for the work, writes per
 * phase the summed device milliseconds and the kernel launches (arrays of at
 * least `cap` entries, phase order of bdm_phase_name), sets *n_phases to the
 * number of phases and stops profiling.  Errors: BDM_EINVAL, BDM_ECUDA. */
int bdm_profile_begin(bdm_sim *sim);
int bdm_profile_end(bdm_sim *sim, double *ms, int64_t *launches, int cap, int *n_phases);

/* Name of phase `phase` (0-based) of an iteration: "geometry", "brick_rank",
 * "keys", "brick_scan", "scatter", "brick_sort", "gather", "force",
 * "force_fix" (the FP32 form's fix-up pass; empty with the tiled and sparse
 * kernels), "divide" (division merge
 * and removal), "finish"; "" outside the range. */
const char *bdm_phase_name(int phase);

/* Change the stream all later work of this simulation is ordered on. */
int bdm_set_stream(bdm_sim *sim, void *stream);

/* Summed force on every agent of one simulation without allocating any
 * memory.  The paper has no counterpart: this entry point serves callers that
 * cannot call cudaMalloc -- host applications whose own allocator owns all
 * device memory (an allocation behind its back would break its accounting or
 * fail against its pool), and plug-ins or embedded solvers that their host
 * forbids to allocate.  It runs the same grid build and
 * force kernels as BDM_DBG_FORCES_NOW in the FP64 form (no displacement, no
 * static skip) on the caller's device buffers: xyz 3 x n doubles (x, y, z
 * blocks), diam n doubles; outputs forces 3 x n doubles (same layout) and
 * counts 2 x n int32 (contacts, then neighbours).  Every intermediate lives
 * in one fixed device array of about 23 MB, which each GPU that loads this
 * library holds until the process exits; it bounds the problem to at most
 * 131072 agents, 262144 4x4x4-box bricks and 16384 occupied bricks
 * (BDM_ECAPACITY beyond them, with nothing written).  All calls share that
 * array and it keeps the last call's contents, so calls that may overlap on
 * the GPU (other streams, other host threads, same device) race: serialise
 * them.  The first call on a device looks up the array's device address
 * (once per device, with that device current) and keeps it for the life of
 * the process; make that first call before any stream capture.  A
 * cudaDeviceReset unloads the array from the device, so do not call this
 * entry point on a device after resetting it.  Work is ordered on `stream` (a
 * cudaStream_t, NULL = legacy default) and the call waits for it to finish.  Errors: BDM_EINVAL,
 * BDM_ECAPACITY, BDM_ECUDA; bdm_noalloc_last_error() gives the message. */
int bdm_forces_noalloc(int64_t n, const double *xyz, const double *diam, double interaction_radius,
                       double box_edge, double k, double gamma, double *forces, int32_t *counts, void *stream);
const char *bdm_noalloc_last_error(void);

/* Release everything the simulation owns.  NULL-safe. */
void bdm_destroy(bdm_sim *sim);

/* Message of the last failed call on `sim` (or of the last failed
 * bdm_create when sim is NULL).  Never NULL; valid until the next call. */
const char *bdm_last_error(const bdm_sim *sim);

/* ABI version of this header (major * 100 + minor). */
int bdm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BDM_H */
