/*
 * oracle.h -- plain, slow, FP64 CPU oracle of one F.A.S.T. time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline / reference arm use it.  It shares no source with the CUDA library
 * (paper_0911_2900_gb300/csrc) and includes none of its headers.
 *
 * What it computes (Kretz, "Computation Speed of the F.A.S.T. Model"):
 *   Sec. 1: every time step is a planning phase in which each agent chooses a
 *           desired cell from data common to all agents (only read), followed
 *           by a movement phase that is carried out sequentially, agent after
 *           agent, so that no two agents ever share a cell;
 *   Sec. 2: k_S = 1.2, k_other = 0, one maximum speed v_m for all agents,
 *           one step = one simulated second; the planning loop is the only
 *           parallel region, its agents dealt to the cores in chunks taken
 *           on demand.
 * The paper does not restate the model's rules; each reading this oracle
 * implements (reach set, line of sight, weight, sampling rule, random numbers,
 * path rasterisation, movement order, exits) is stated in the comment of the
 * function of oracle.c that implements it.
 */
#ifndef FAST_ORACLE_H
#define FAST_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FREE = 0, ORC_WALL = 1, ORC_EXIT = 2 };
enum { ORC_REACH_L2 = 0, ORC_REACH_L2P = 1, ORC_REACH_LINF = 2 };
#define ORC_MAXK 121

typedef struct {
  int32_t W, H;        /* grid size in cells, row-major, cell = y*W + x      */
  int32_t v;           /* maximum speed v_m in cells per step, 1..5         */
  int32_t reach;       /* ORC_REACH_*                                      */
  double kS;           /* coupling to the static floor field               */
  uint64_t seed;       /* Philox key                                       */
  const uint8_t* type; /* [W*H] ORC_FREE / ORC_WALL / ORC_EXIT               */
  const double* S;     /* [W*H] static floor field (orc_floor_field)        */
  const uint8_t* speed; /* [ids] maximum speed of each agent id, 1..5, or   */
                        /* NULL: v for every agent (Sec. 2's benchmark)    */
} orc_world;

/* Philox4x32-10 (Salmon et al., SC'11), one 128-bit block. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* FP64 exponential, Cody-Waite reduction + degree-13 Taylor in Horner form. */
double orc_exp64(double x);

/* Candidate offsets in canonical order (dy ascending, then dx ascending). */
int32_t orc_offsets(int32_t v, int32_t reach, int32_t* dx, int32_t* dy);

/* Straight path to offset (dx,dy): writes steps s=1..L as offsets; returns L. */
int32_t orc_path(int32_t dx, int32_t dy, int32_t* px, int32_t* py);

/* Exact 8-neighbour Dijkstra from every exit cell: S = a + b*sqrt(2) with a
 * orthogonal and b diagonal steps; unreachable / wall cells: a=b=-1, S=+inf.
 * Returns the number of reachable cells, or -1 on allocation failure. */
int64_t orc_floor_field(int32_t W, int32_t H, const uint8_t* type,
                        int32_t* a, int32_t* b, double* S);

/* occ[c] = agent index, -1 free, -2 wall.  Returns 0, or -1 if an agent is on
 * a wall / exit / outside the grid / shares a cell. */
int32_t orc_build_occ(const orc_world* w, int32_t n, const int32_t* cell, int32_t* occ);

/* Planning of one agent at step t.  w_out[K] (optional) gets the weights in
 * canonical order, u_out (optional) the uniform draw.  Returns desired cell. */
int32_t orc_plan_agent(const orc_world* w, const int32_t* occ, int32_t cell,
                       int32_t id, int32_t t, double* w_out, double* u_out);

/* Planning of all agents (exited agents, cell < 0, get desired = -1).
 * threads <= 1: serial loop; threads > 1: the paper's OpenMP partition. */
void orc_plan_all(const orc_world* w, const int32_t* occ, int32_t n,
                  const int32_t* id, const int32_t* cell, int32_t t,
                  int32_t* desired, int32_t threads);

/* Movement priority of agent id at step t (smaller moves earlier; a
 * permutation of the 24-bit ids for each step). */
uint32_t orc_move_priority(uint64_t seed, int32_t id, int32_t t);

/* Sequential movement of all agents in priority order.  Updates cell (-1 when
 * an agent leaves through an exit) and occ.  Returns the number that left. */
int32_t orc_move(const orc_world* w, int32_t* occ, int32_t n, const int32_t* id,
                 int32_t* cell, const int32_t* desired, int32_t t);

/* Order-independent 64-bit digest of the (id, value) pairs with value >= 0
 * (splitmix64 output function of (id << 32 | value), summed mod 2^64). */
uint64_t orc_digest(int32_t n, const int32_t* id, const int32_t* val);

/* n_steps full steps from step t0.  Optional outputs (NULL to skip):
 * desired_last[n], dig_cell/dig_des/alive[n_steps], plan_s/move_s = seconds. */
int32_t orc_run(const orc_world* w, int32_t* occ, int32_t n, const int32_t* id,
                int32_t* cell, int32_t t0, int32_t n_steps, int32_t threads,
                int32_t* desired_last, uint64_t* dig_cell, uint64_t* dig_des,
                int32_t* alive, double* plan_s, double* move_s);

#ifdef __cplusplus
}
#endif
#endif
