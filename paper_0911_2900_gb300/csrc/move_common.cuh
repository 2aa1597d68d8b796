// move_common.cuh -- device pieces shared by the two schedules of the
// movement phase (move.cu: rounds of claims with a grid barrier each;
// move_flow.cu: a dataflow over the conflict graph): the mover entry's info
// word, straight-path tables, footprints, the two ways of committing a move,
// and the bounded grid barrier of a cooperative launch.
#pragma once
#include "fast_device.cuh"

namespace fastgb {

// info word of a work-list entry
constexpr uint32_t MV_LEN = 0x7u;      // footprint path length (0..5)
constexpr uint32_t MV_EXIT = 0x8u;     // the path reaches an exit cell after the footprint
constexpr int MV_DX = 4;               // dx + 8, 4 bits
constexpr int MV_DY = 8;               // dy + 8, 4 bits
constexpr int MV_FIN = 13;             // first-round outcome: last path step entered (3 bits)
constexpr uint32_t MV_GONE = 1u << 16; // first-round outcome: leaves through an exit
constexpr int MV_NEED = 17;            // footprint cells (bit s: cell s) whose claim the
                                       // agent has not held yet (6 bits)
constexpr int MV_CLM = 23;             // footprint cells the agent must keep claiming in
                                       // later rounds: those another agent also claims
                                       // (6 bits)

// Place of cell (x, y) in the tile-major claim arrays (16x16-cell tiles).
__device__ __forceinline__ int claim_index(const RepDev& R, int x, int y) {
  return ((((y >> 4) * R.claim_tx) + (x >> 4)) << 8) | ((y & 15) << 4) | (x & 15);
}

// Straight-path table for every offset (dx, dy) in [-5, 5]^2 and step
// s = 1..5: (dx_s, dy_s) = (q(s*dx, L), q(s*dy, L)), L = max(|dx|, |dy|),
// q = division rounded half away from zero.
struct PathTab {
  int8_t d[11 * 11 * 5][2];
};

__device__ __forceinline__ void build_path_tab(PathTab* t) {
  for (int i = threadIdx.x; i < 121; i += blockDim.x) {
    const int dx = i % 11 - 5, dy = i / 11 - 5;
    const int L = max(abs(dx), abs(dy));
    for (int s = 1; s <= 5; ++s) {
      const bool ok = L > 0 && s <= L;
      t->d[i * 5 + s - 1][0] = ok ? (int8_t)div_half_away(s * dx, L) : 0;
      t->d[i * 5 + s - 1][1] = ok ? (int8_t)div_half_away(s * dy, L) : 0;
    }
  }
}

__device__ __forceinline__ int path_cell_tab(const PathTab* t, int c0, int W, uint32_t info, int s) {
  if (s == 0) return c0;
  const int dx = (int)((info >> MV_DX) & 0xF) - 8, dy = (int)((info >> MV_DY) & 0xF) - 8;
  const int i = ((dy + 5) * 11 + (dx + 5)) * 5 + s - 1;
  return c0 + (int)t->d[i][1] * W + (int)t->d[i][0];
}

// ---------------------------------------------------------------------------
// Grid-wide barrier for a cooperative launch, with a time limit, that also
// adds up one count over the blocks.  Barriers n = 1, 2, 3, ... of a launch
// use the words w = ctl->bar_acc[n & 1][0] in turn, zero when the launch
// starts: every block adds 1 (its arrival) and its count << 32 to w, and
// the barrier is complete once the low half reaches k * gridDim.x, k the
// number of barriers so far that used w.  No block can add to w again before
// every block has passed the barrier in between, so the high half then holds
// the running sum (mod 2^32) of the counts of w's barriers.  `passed` counts
// the barriers this block has completed, sum0 and sum1 are the running sums
// of the two words it saw last; *total receives the sum of this barrier's
// counts.  The block whose arrival completes the barrier learns it from the
// atomic itself and does not poll.  A block that waits longer than
// ctl->barrier_ns_limit records the timeout in ctl->err, and every block then
// leaves the kernel at its next barrier (the function returns false).
static __device__ bool grid_barrier_sum(Ctl* ctl, uint32_t& passed, uint32_t& sum0, uint32_t& sum1,
                                 uint32_t count, uint32_t* total) {
  __shared__ int s_ok;
  __shared__ uint32_t s_total;
  __syncthreads();
  ++passed;
  if (threadIdx.x == 0) {
    const uint32_t p = passed & 1u;
    unsigned long long* w = &ctl->bar_acc[p][0];
    volatile int* verr = &ctl->err;
    int ok = 1;
    unsigned long long seen = 0ull;
    if (passed >= 0x7FFFFFFFu / gridDim.x) {
      // the arrivals would outgrow their half of the word
      atomicCAS(&ctl->err, 0, kDevErrRounds);
      ok = 0;
    } else {
      const uint32_t target = ((passed + p) >> 1) * gridDim.x;
      const unsigned long long add = ((unsigned long long)count << 32) | 1ull;
      const size_t gw = __cvta_generic_to_global(w);
      // the arrival releases this block's writes (ordered before it by the
      // block barrier above) and acquires those of the blocks that arrived
      // earlier; the polls acquire those of the rest
      asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                   : "=l"(seen)
                   : "l"(gw), "l"(add)
                   : "memory");
      seen += add;
      const unsigned long long t0 = global_ns();
      const unsigned long long lim = ctl->barrier_ns_limit;
      while ((uint32_t)seen != target) {
        if (*verr != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > lim) {
          atomicCAS(&ctl->err, 0, kDevErrTimeout);
          ok = 0;
          break;
        }
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(gw) : "memory");
      }
      if (*verr != 0) ok = 0;
    }
    const uint32_t run = (uint32_t)(seen >> 32);
    s_total = run - (p ? sum1 : sum0);
    if (p)
      sum1 = run;
    else
      sum0 = run;
    s_ok = ok;
  }
  __syncthreads();
  if (total) *total = s_total;
  return s_ok != 0;
}

// The barrier without a count (the running sum stays as it is).
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, uint32_t& passed) {
  uint32_t unused0 = 0u, unused1 = 0u;
  return grid_barrier_sum(ctl, passed, unused0, unused1, 0u, nullptr);
}

// Footprint of a mover at (x0, y0): row-major cells c[s] (records) and the
// cells' places q[s] in the tile-major claim arrays, s = 0..5 (start, path).
__device__ __forceinline__ void foot_cells(const PathTab* tab, uint32_t xy, const RepDev& R,
                                           uint32_t info, int* c, int* q) {
  const int x0 = (int)(xy & 0xFFFFu), y0 = (int)(xy >> 16);
  const int dx = (int)((info >> MV_DX) & 0xF) - 8, dy = (int)((info >> MV_DY) & 0xF) - 8;
  const int i0 = ((dy + 5) * 11 + (dx + 5)) * 5;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int x = x0 + (s == 0 ? 0 : (int)tab->d[i0 + s - 1][0]);
    const int y = y0 + (s == 0 ? 0 : (int)tab->d[i0 + s - 1][1]);
    c[s] = y * R.W + x;
    q[s] = claim_index(R, x, y);
  }
}

// Path records an agent may walk: path cells 1..min(L, n + 1), where past
// the footprint only one more cell can be reached, and it is constant (a
// stayer, which blocks, or the exit the agent leaves by).
__device__ __forceinline__ int walk_len(uint32_t info) {
  const int n = (int)(info & MV_LEN);
  const int dx = (int)((info >> MV_DX) & 0xF) - 8, dy = (int)((info >> MV_DY) & 0xF) - 8;
  return min(max(abs(dx), abs(dy)), n + 1);
}

// Moves one agent that owns its footprint, given the records of its start
// cell (pr[0]) and path cells (pr[s] for cell s; blocked past the walk
// length), all read after the last barrier.  The agent owns every cell it
// writes, so the records it read are still current.
__device__ __forceinline__ void commit_move(const StepArgs& a, const RepDev& R, int rep, int slot,
                                            const int* c, const uint32_t* pr) {
  int cfin = c[0];
  uint32_t rfin = pr[0];
  bool gone = false, stop = false;
#pragma unroll
  for (int s = 1; s <= 5; ++s) {
    const uint32_t rr = pr[s];
    stop = stop || (rr & REC_OCC);
    if (!stop) {
      cfin = c[s];
      rfin = rr;
      if (rec_exit(rr)) {
        gone = true;
        stop = true;
      }
    }
  }
  if (cfin == c[0]) return;
  __stcg(&R.rec[c[0]], pr[0] & ~(REC_OCC | REC_STA));
  if (!gone) {
    __stcg(&R.rec[cfin], rfin | REC_OCC);
    R.cell[slot] = cfin;
  } else {
    R.cell[slot] = -1;
    red_add_s32(&a.exited[rep], 1);
  }
}

// First-round move of an agent that owns its footprint: nobody has touched
// the footprint this step, so the outcome the movement-order pass recorded
// holds, and only occupancy bits change.
__device__ __forceinline__ void commit_first(const StepArgs& a, const RepDev& R, int rep, int slot,
                                             const int* c, uint32_t info) {
  const int fin = (int)((info >> MV_FIN) & 7u);
  const bool gone = (info & MV_GONE) != 0u;
  if (fin == 0) return;
  int cf = c[0];
#pragma unroll
  for (int s = 1; s <= 5; ++s)
    if (s == fin) cf = c[s];
  red_and_b32(&R.rec[c[0]], ~(REC_OCC | REC_STA));
  if (gone) {
    R.cell[slot] = -1;
    red_add_s32(&a.exited[rep], 1);
  } else {
    red_or_b32(&R.rec[cf], REC_OCC);
    R.cell[slot] = cf;
  }
}

}  // namespace fastgb
