/*
 * fastgb.h -- C ABI of libfastgb: the time step of the F.A.S.T. pedestrian
 * model (T. Kretz, "Computation Speed of the F.A.S.T. Model", arXiv:0911.2900)
 * on one NVIDIA GB300 GPU.
 *
 * A time step is a planning phase in which every agent chooses a desired cell
 * from data common to all agents, which it only reads, followed by a movement
 * phase that is sequential, agent after agent, so that no two agents ever
 * share a cell (Sec. 1).  The model parameters are k_S = 1.2, k_other = 0 and
 * one maximum speed v_m for all agents of a simulation; one step is one
 * simulated second (Sec. 2).  The paper does not restate the model's rules;
 * this library fixes them as follows (the same rules as the FP64 reference
 * the tests compare against):
 *   - floor field S: shortest 8-neighbour path to any exit cell through
 *     non-wall cells, costs 1 and sqrt(2), kept exactly as a + b*sqrt(2);
 *   - candidates of an agent on cell c0: offsets (dx,dy) of the reach set
 *     (dx^2+dy^2 <= v_m^2 by default), in row order, inside the grid, whose
 *     straight path has no wall, whose target is free or is c0 itself;
 *   - weight exp(-k_S (S(c) - S(c0))), summed in that order in FP64; the
 *     choice is the smallest k with u*W < C_k, u a 53-bit uniform from
 *     Philox4x32-10 (key = seed, counter = (id, step, 0, 0));
 *   - movement in ascending order of a keyed permutation of the 24-bit ids
 *     (four Feistel rounds on 12-bit halves, round function
 *     fmix32(R ^ k_i) & 0xFFF, keys = Philox4x32-10(seed; (0, step, 2, 0)));
 *     each agent walks its straight path, stops before a blocked cell, leaves
 *     on entering an exit cell.
 *
 * Conventions for every call:
 *   - cells are row-major indices y*width + x; cell types are 0 free, 1 wall,
 *     2 exit;
 *   - host pointers are borrowed for the duration of the call and copied;
 *   - device memory is owned by the context; it comes from the allocator
 *     callbacks given to fast_create (or cudaMalloc when they are NULL);
 *   - work is queued on the CUDA stream given to fast_create; calls that
 *     return data to the host synchronise that stream;
 *   - the return value is FAST_OK (0) or a negative FAST_E* code, with a
 *     message in fast_last_error(); after FAST_ECUDA or FAST_ETIMEOUT the
 *     context is poisoned and only fast_last_error / fast_destroy are valid.
 */
#ifndef FASTGB_H
#define FASTGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FAST_OK 0
#define FAST_EINVAL (-1)   /* bad argument: shape, cell, id, v_m, ...        */
#define FAST_ESTATE (-2)   /* call out of order (e.g. step before placement) */
#define FAST_ENOMEM (-3)   /* device allocation failed                      */
#define FAST_ECUDA (-4)    /* CUDA runtime error                            */
#define FAST_ETIMEOUT (-5) /* a bounded device-side wait gave up            */

/* precision of the planning phase */
#define FAST_FP64 0           /* every agent with the FP64 rule               */
#define FAST_FP32_RECHECK 1   /* FP32 weights; draws near a boundary in FP64   */
#define FAST_FP32_NORECHECK 2 /* FP32 only (diagnostic: may differ from FP64)  */

/* reach set of one step */
#define FAST_REACH_L2 0   /* dx^2 + dy^2 <= v^2        (K = 5,13,29,49,81)   */
#define FAST_REACH_L2P 1  /* dx^2 + dy^2 <= v^2 + v    (K = 9,21,37,69,97)   */
#define FAST_REACH_LINF 2 /* max(|dx|,|dy|) <= v       (K = 9,25,49,81,121)  */

#define FAST_CELL_FREE 0
#define FAST_CELL_WALL 1
#define FAST_CELL_EXIT 2

/* options for fast_set_option */
#define FAST_OPT_RESORT_PERIOD 1  /* re-sort agents in spatial order every n steps (default 8; 0 never) */
#define FAST_OPT_DIGESTS 2        /* 1: record per-step digests (fast_get_digests)  */
#define FAST_OPT_LANES_V1 3       /* FP32 planning kernel for v_m=1 (..._V1 + v_m - 1 */
                                  /* for v_m = 1..5): 0 one thread per agent with   */
                                  /* per-warp record tiles; 1 one thread per agent  */
                                  /* reading records through L1 (default); 2, 4, 8  */
                                  /* lanes per agent with shuffle prefix sums       */
#define FAST_OPT_BARRIER_NS 10    /* time limit of one device-side wait, ns         */
#define FAST_OPT_USE_GRAPH 11     /* 1 (default): steps replay a captured CUDA graph */
#define FAST_OPT_MOVE_BLOCKS 12   /* blocks of the cooperative movement kernel (0: auto) */
#define FAST_OPT_TILE_SHIFT 13    /* re-sort bucket side = 2^shift cells, buckets in */
                                  /* Hilbert-curve order (default 4)                 */
#define FAST_OPT_GRAPH_STEPS 14   /* fast_step(n) with 2 <= n <= this (default 512)  */
                                  /* runs the whole n-step loop as one captured     */
                                  /* CUDA graph, kept for later calls at the same   */
                                  /* step phase; 0 or 1: one graph per step         */
#define FAST_OPT_CLAIM_RESERVE 15 /* movement claim tags (255 per clean-up of the   */
                                  /* claim arrays) a step must have left, else the  */
                                  /* arrays are cleared first (default 96; a step   */
                                  /* that runs out clears them itself)              */
#define FAST_OPT_CLAIM_TAG 16     /* clears the claims and sets the next step's     */
                                  /* first claim tag, 0..254: a test hook for the   */
                                  /* clean-ups; results do not depend on it         */

typedef struct fast_ctx fast_ctx;

/* Device allocator callbacks: alloc returns a device pointer of >= bytes
 * (256-byte aligned) or NULL; free releases it.  `user` is passed through. */
typedef void* (*fast_alloc_fn)(size_t bytes, void* user);
typedef void (*fast_free_fn)(void* ptr, void* user);

/* One replicate's grid. */
typedef struct {
  int32_t width, height;    /* cells, each <= 65535; width*height < 2^31     */
  const uint8_t* cell_type; /* host [width*height], borrowed for the call    */
  double k_S;               /* coupling to the static floor field (>= 0)     */
  int32_t v_m;              /* maximum speed, 1..5 cells per step            */
  uint64_t seed;            /* Philox key of this replicate                  */
  const double* static_field; /* host [width*height] or NULL, borrowed: the    */
                            /* caller's static floor field S per cell instead */
                            /* of the library's 8-neighbour distance to the   */
                            /* exits.  The library keeps S exactly as step    */
                            /* counts (a, b), S = a + b*sqrt(2), so every     */
                            /* value must be of that form as the FP64 rule    */
                            /* rounds it, fl(a + fl(b*sqrt2)), integers       */
                            /* 0 <= a, b <= 32766 (any field made of          */
                            /* orthogonal and diagonal steps is); exit cells  */
                            /* need 0 and no other cell may be 0; +inf marks  */
                            /* a free cell treated as a wall (no exit         */
                            /* reachable); values of wall cells are ignored.  */
                            /* Another field is refused with FAST_EINVAL.     */
} fast_grid_desc;

typedef struct {
  int64_t step;            /* index of the next step                            */
  int64_t steps_run;       /* steps run since the last placement                */
  int32_t alive;           /* agents of this replicate still in the simulation  */
  int32_t exited;          /* agents of this replicate that left through an exit */
  int64_t agent_steps;     /* all replicates: sum over steps of agents planned  */
  int64_t rechecked;       /* all replicates: draws re-evaluated in FP64        */
  int64_t move_rounds;     /* all replicates: movement rounds, total            */
  int32_t max_rounds;      /* largest number of movement rounds in one step     */
  int32_t last_rounds;     /* movement rounds of the last step                  */
  int64_t kernel_launches; /* CUDA kernels this context has queued, in total    */
  int64_t tile_fallbacks;  /* planning warps that read from global memory because */
                           /* their agents did not fit one shared-memory tile  */
  int64_t movers;          /* agents handed to the movement rounds, all steps  */
  int64_t footprint_cells; /* their footprint cells, all steps                 */
  int64_t diag_flips;      /* the last fast_precision_report_run: FP32-only     */
                           /* choices that differ from the FP64 rule (0: none) */
  double diag_max_abs_dp;  /* its largest |p32 - p64| over the candidates       */
} fast_stats;

typedef struct {
  int64_t agents;          /* agents evaluated                                  */
  int64_t flagged;         /* FP32 draws inside the margin (re-checked in FP64) */
  int64_t flips;           /* FP32 choice != FP64 choice                        */
  int64_t flips_unflagged; /* of those, outside the margin (must be 0)          */
  double max_abs_dp;       /* max |P32(k) - P64(k)| over cumulative probabilities */
  double margin;           /* relative margin M of the FP32 decision           */
  int64_t flips_after_recheck; /* choices of the FP32 pass with the FP64 re-check */
                           /* != FP64 rule (must be 0)                          */
} fast_precision_report;

typedef struct {
  int32_t tile_shift;      /* chosen re-sort bucket side, log2 of cells          */
  int32_t lanes[5];        /* chosen planning variant per v_m (FAST_OPT_LANES_V1 */
                           /* values: 0 tiled, 1/2/4/8 lanes per agent); -1 for  */
                           /* a v_m no replicate uses                           */
  float shift_us[4];       /* planning (tiled) + re-sort / period, us per step,  */
                           /* for bucket shifts 3, 4, 5, 6                       */
  float lanes_us[5][5];    /* [v_m - 1][variant]: planning time of that v_m's    */
                           /* agents, us, variants 0, 1, 2, 4, 8; 0: not tried  */
} fast_tune_report;

/* Creates a context for n_replicates independent replicates (1..256).
 * precision: FAST_FP64 / FAST_FP32_RECHECK / FAST_FP32_NORECHECK;
 * reach: FAST_REACH_*; cuda_stream: a cudaStream_t (NULL: legacy default).
 * Errors: FAST_EINVAL, FAST_ECUDA (no device). */
int fast_create(fast_ctx** out, int32_t n_replicates, int32_t precision, int32_t reach,
                void* cuda_stream, fast_alloc_fn dev_alloc, fast_free_fn dev_free,
                void* alloc_user);

/* Sets the grid of one replicate: validates the cell types, computes the
 * exact floor field on the host, uploads cell records and line-of-sight
 * masks.  Every free cell that no exit can be reached from is treated as a
 * wall.  With grid->static_field the caller's field replaces the computed
 * one (its +inf cells are the walls so added).  Errors: FAST_EINVAL (types,
 * size, v_m, k_S, no exit, distance too long for the 15-bit record fields, a
 * static_field value that is not of the form above), FAST_ENOMEM (the
 * replicate is then left without a grid and without agents; a later call on
 * it is refused with FAST_ESTATE until a fast_init_grid succeeds),
 * FAST_ECUDA. */
int fast_init_grid(fast_ctx* ctx, int32_t replicate, const fast_grid_desc* grid);

/* Gives the agents of one replicate maximum speeds of their own (Sec. 2 runs
 * its benchmark with one speed for all agents; the model allows one per
 * agent): speed_by_id: host [n_ids], the speed in 1..5 of every id below
 * n_ids, copied.  Each agent then plans over the reach set of its own speed;
 * the movement does not depend on the speed.  Call it after fast_init_grid
 * and before the replicate's first placement; the speeds hold for every later
 * placement (an agent whose id has no speed is rejected there) until the next
 * fast_init_grid.  n_ids = 0 returns to the grid's v_m for every agent.  The
 * line-of-sight masks of every speed present are built here (one mask array
 * per speed).  fast_plan_noalloc does not take such replicates.  Errors:
 * FAST_EINVAL (n_ids outside [0, 2^24], a speed outside 1..5, k_S too large
 * for the largest speed), FAST_ESTATE (grid not set, or agents already
 * placed), FAST_ENOMEM, FAST_ECUDA. */
int fast_set_speeds(fast_ctx* ctx, int32_t replicate, int32_t n_ids, const uint8_t* speed_by_id);

/* Places n agents of one replicate (replacing any previous ones).
 * cells: host [n] distinct free, reachable, non-exit cells; NULL: a seeded
 * uniform placement -- ids 0..n-1 on n distinct cells drawn uniformly from
 * the free, reachable, non-exit cells with a generator started from the
 * grid's seed, so the same grid, seed and n always give the same cells (ids
 * must then be NULL, and n at most the number of such cells);
 * ids: host [n] distinct ids in [0, 2^24); NULL: agent i has id i, and
 * cells[i] == -1 means there is no agent with id i (so the cells-by-id array
 * that fast_readback writes can be placed again as it is);
 * start_step: index of the next step (all replicates share one step index;
 * resuming a run = placing its read-back state with its step index).
 * The cells and ids are checked on the device.  Placing implicit ids again
 * with the same n keeps every agent in the storage slot its id holds (ids
 * without one are added after the others), so the spatial order of the
 * agents in memory stays and the next step does not sort them first; any
 * other placement stores agent i in slot i and sorts before the next step.
 * The storage order never changes a result.  Errors: FAST_EINVAL (a cell
 * outside the grid, on a wall, unreachable, an exit or taken twice, an id
 * out of range or repeated, or an id without a speed after fast_set_speeds;
 * the replicate is then left without agents),
 * FAST_ESTATE (grid not set), FAST_ENOMEM, FAST_ECUDA. */
int fast_place_agents(fast_ctx* ctx, int32_t replicate, int32_t n, const int32_t* cells,
                      const int32_t* ids, int32_t start_step);

/* All replicates in one call (for the batched form: one upload and one wait
 * instead of one per replicate).  counts[r] (host, [n_replicates]): number of
 * ids of replicate r, -1 to leave it as it is; cells_by_id (host): for each
 * replicate in order, counts[r] cells by id (-1: no agent with that id), all
 * concatenated.  Checks as fast_place_agents; on FAST_EINVAL every replicate
 * that failed is left without agents (the message names the first). */
int fast_place_all(fast_ctx* ctx, const int32_t* counts, const int32_t* cells_by_id,
                   int32_t start_step);

/* Queues n_steps full steps (planning + movement) of every replicate on the
 * context's stream; returns without waiting.  Errors: FAST_ESTATE, FAST_ECUDA. */
int fast_step(fast_ctx* ctx, int32_t n_steps);

/* Queues n planning passes only (no movement, the step index does not move):
 * used to time the planning phase alone. */
int fast_plan_only(fast_ctx* ctx, int32_t n);

/* Queues, after the work on the stream, the copies of the cell of each agent
 * of the replicate for ids 0..id_bound-1 (-1: left or not present) and of its
 * desired cell of the last planning pass (-1 likewise), then waits for them;
 * either pointer may be NULL.  stats may be NULL.  Errors: FAST_EINVAL,
 * FAST_ETIMEOUT / FAST_ECUDA (device error; the arrays' contents are then
 * unspecified). */
int fast_readback(fast_ctx* ctx, int32_t replicate, int32_t id_bound, int32_t* cells_by_id,
                  int32_t* desired_by_id, fast_stats* stats);

/* Reads every replicate back in one call (waits for the stream): for each
 * replicate in order, counts[r] (>= 0) ids, concatenated, into cells_by_id
 * and desired_by_id (either may be NULL; -1: not present), and alive[r] the
 * agents of replicate r still in the simulation (may be NULL).  Errors:
 * FAST_EINVAL, FAST_ETIMEOUT / FAST_ECUDA (device error). */
int fast_readback_all(fast_ctx* ctx, const int32_t* counts, int32_t* cells_by_id,
                      int32_t* desired_by_id, int32_t* alive);

/* Per-step digests recorded since the last placement while FAST_OPT_DIGESTS
 * is on: sum over agents still present of splitmix64(id << 32 | cell) after
 * the step's movement, and of splitmix64(id << 32 | desired) after its
 * planning.  Writes min(max_steps, recorded) values; returns that count or a
 * negative error. */
int fast_get_digests(fast_ctx* ctx, int32_t replicate, int32_t max_steps, uint64_t* cell_digest,
                     uint64_t* desired_digest);

/* Device times (ms) of the parts of the last step queued by fast_step, from
 * CUDA events recorded on the context's stream (waits for them):
 * ms5[0] planning kernels, ms5[1] FP64 re-check, ms5[2] movement order and
 * footprints, ms5[3] movement rounds, ms5[4] bookkeeping (digests, re-sort,
 * step counter).  Errors: FAST_ESTATE if no step has run. */
int fast_phase_times(fast_ctx* ctx, float* ms5);

/* Movement rounds of the last step (waits for the stream): n_wait[r] = agents
 * still waiting after round r, t_ns[r] = device global timer at the start of
 * round r (t_ns has one entry more).  Writes min(max_rounds, 64) rounds;
 * returns the number of rounds of the step or a negative error.  With
 * max_rounds >= 73, t_ns[65..72] also receive maxima over the blocks: the
 * first round's work (ns), the same plus its grid barrier (ns), the second
 * round's work (ns), the first round's claims (ns), movers per block, movers
 * per block still waiting after the first round, the round from which one
 * block finished alone (0: none), 0.  With max_rounds >= 137, t_ns[73 + r]
 * also receives the most movers still waiting in one block after round r,
 * for the rounds written. */
int fast_move_profile(fast_ctx* ctx, int32_t max_rounds, uint32_t* n_wait, uint64_t* t_ns);

/* Runs, on the current state, the planning pass (FP32 weights with the FP64
 * re-check), the FP32 planning without re-check and the FP64 rule, and
 * compares them.  Agents' cells and the step index do not change; the
 * desired cells read back afterwards are this pass's.  Errors:
 * FAST_ESTATE (precision is FAST_FP64 or no agents), FAST_ENOMEM, FAST_ECUDA. */
int fast_precision_report_run(fast_ctx* ctx, fast_precision_report* out);

/* Number of distinct cells whose record one planning pass of the replicate
 * reads (own cells and line-of-sight reach offsets), for byte accounting. */
int fast_reach_union(fast_ctx* ctx, int32_t replicate, int64_t* cells);

/* Planning pass that allocates no device memory (no counterpart in the
 * paper: it exists for callers that cannot allocate when they plan, such as
 * code capturing a CUDA graph on its stream, or a process whose device memory
 * is all held by another allocator).  It writes, for each agent of the
 * replicate present in the context with id < id_bound, the desired cell of
 * step `step` into desired_by_id_dev[id] (a device buffer the caller owns;
 * other entries are left as they are).  It always plans with FP32 weights
 * and the FP64 re-check inside the margin, whatever precision the context
 * has, so its output is the FP64 rule's choice (equal to a planning pass of a
 * FAST_FP64 or FAST_FP32_RECHECK context; a FAST_FP32_NORECHECK context's own
 * planning may differ near a boundary).  The
 * context's state is read, never changed, and the call only queues work on
 * the context's stream.  Its scratch is one fixed array of 4 MiB + 256 bytes
 * inside the library, held on every device that loads the library until the
 * process exits: hence at most 2^20 agent slots per replicate (FAST_EINVAL
 * beyond).  Every call on a device shares that array, so calls that can
 * overlap on the GPU race; order them on one stream.  The first call on a
 * device looks up the array's device address (make it before any stream
 * capture).  FAST_ESTATE if the replicate has no agents, or if an option
 * that changes the context's work lists (the bucket side) was set since the
 * last placement, fast_step or fast_plan_only. */
int fast_plan_noalloc(fast_ctx* ctx, int32_t replicate, int32_t step, int32_t id_bound,
                      int32_t* desired_by_id_dev);

/* Autotuner (the paper has no counterpart: it chooses how the GPU runs the
 * planning phase, never what it computes).  On the agents placed now, times
 * `trials` planning passes (after one untimed pass) of each candidate:
 * first the re-sort bucket side 2^3..2^6 cells with the tiled kernel (plus
 * the re-sort's own time divided by its period), then, at the chosen side,
 * each planning variant for every v_m present.  The fastest choices become
 * the context's options (FAST_OPT_TILE_SHIFT, FAST_OPT_LANES_V*); agents are
 * re-sorted, which permutes storage only.  The step index and every agent's
 * cell are unchanged; the desired cells of the last step are overwritten (a
 * step re-plans them anyway).  `out` (may be NULL) receives the choices and
 * the times.  With precision FAST_FP64 nothing is tuned.  Errors:
 * FAST_EINVAL (trials not in 1..1000), FAST_ESTATE (no agents), FAST_ECUDA. */
int fast_autotune(fast_ctx* ctx, int32_t trials, fast_tune_report* out);

/* Host only (no GPU, no context): the static floor field fast_init_grid
 * would use for this grid.  With static_field NULL, the library's field (the
 * exact 8-neighbour distance to the exits, costs 1 and sqrt(2)); else the
 * caller's field checked and decomposed as fast_grid_desc describes.  Writes
 * (each pointer may be NULL; host arrays [width*height]) S_out: S per cell as
 * the FP64 rule rounds it, fl(a + fl(b*sqrt2)), +inf for walls and cells no
 * exit is reached from; a_out, b_out: the step counts (-1 there).  For
 * editing a field before passing it back through fast_grid_desc.  Errors:
 * FAST_EINVAL (size, a cell type > 2, a static_field value of the wrong
 * form), with *bad_cell (may be NULL) the first offending cell, else -1. */
int fast_floor_field(int32_t width, int32_t height, const uint8_t* cell_type,
                     const double* static_field, double* S_out, int32_t* a_out, int32_t* b_out,
                     int64_t* bad_cell);

int fast_set_option(fast_ctx* ctx, int32_t option, int64_t value);
const char* fast_last_error(const fast_ctx* ctx);
void fast_destroy(fast_ctx* ctx);

/* ---- self tests of the device arithmetic (need a GPU; no context) -------- */
/* y[i] = the library's FP64 exponential of x[i] on the GPU; host arrays [n]. */
int fast_selftest_exp64(const double* x, double* y, int64_t n);
/* Philox4x32-10 on the GPU: ctr [4n], key [2n], out [4n], host arrays. */
int fast_selftest_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n);
/* Largest relative error of the SFU 2^y over every float y in [lo, hi]. */
int fast_selftest_ex2(float lo, float hi, double* max_rel_err);
/* 1 when this library is the debug build (FASTGB_CHECKED): its kernels check
 * the indices they derive from data (agent and desired cells, candidate and
 * path cells, mover and re-check queue entries) and turn one out of range
 * into FAST_ECUDA at the next call that reads device errors, with the index
 * in fast_last_error, instead of a memory access; 0 for the release build,
 * which compiles the checks away. */
int fast_build_checked(void);

/* One index check of the debug build on the GPU (the index is used for no
 * access): FAST_ECUDA with *recorded = index when it is outside [0, n), else
 * FAST_OK with *recorded = -1; the release build always gives FAST_OK, -1. */
int fast_selftest_bounds(int64_t index, int64_t n, int64_t* recorded);

/* L2 read bandwidth (GB/s): `iters` passes of every SM reading a buffer of
 * `bytes` (16-byte multiple, 4 KiB..1 GiB; small enough to stay in L2) at L2
 * level, after two untimed passes; CUDA-event timed.  For the roofline of
 * planning passes whose cell records stay in L2. */
int fast_selftest_l2_read(int64_t bytes, int32_t iters, double* gb_per_s);
/* Average time of the library's grid barrier: a cooperative kernel of
 * `blocks` x `threads` (all resident) runs `iters` barriers in a row.
 * Returns FAST_EINVAL if the grid cannot be co-resident. */
int fast_selftest_barrier_cost(int32_t blocks, int32_t threads, int32_t iters,
                               double* ns_per_barrier);
/* Check of the grid barrier's count sums (the movement rounds learn how many
 * agents still wait from them): a cooperative kernel of `blocks` x `threads`
 * (all resident) runs `iters` barriers in a row, at barrier i every block
 * bringing the count (block % 5) + (i % 4); *wrong receives the number of
 * (block, barrier) pairs whose total differed from the exact sum (0 when the
 * barrier is right).  Errors as fast_selftest_barrier_cost. */
int fast_selftest_barrier_sum(int32_t blocks, int32_t threads, int32_t iters, int64_t* wrong);
/* Runs a cooperative kernel whose grid barrier can never complete, with a
 * wait limit of limit_ns; returns FAST_ETIMEOUT when the wait gave up (the
 * expected outcome) and leaves the CUDA context usable. */
int fast_selftest_barrier_timeout(int64_t limit_ns);

#ifdef __cplusplus
}
#endif
#endif
