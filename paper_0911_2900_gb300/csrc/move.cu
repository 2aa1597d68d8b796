// move.cu -- movement phase of the F.A.S.T. step on the GPU, equal bit for bit
// to moving the agents one after another (Kretz, Sec. 1: the movement is done
// sequentially, which rules out conflicts; it only uses simple operations).
//
// Sequential semantics: agents in ascending movement priority each walk the
// straight path to their desired cell, stop before a blocked cell, leave the
// simulation on entering an exit cell.
//
// Parallel schedule (deterministic reservations in rounds):
//   footprint F_i = start cell + path cells up to (not including) the first
//   cell held by an agent that stays this step, or the first exit cell.
//   Agent i reads only cells of F_i (plus constant cells: stayers and exits)
//   and writes only cells of F_i.  Two agents with disjoint footprints
//   commute; so committing, in each round, every agent whose footprint
//   touches no footprint of a lower-priority agent still waiting keeps every
//   conflicting pair in priority order, which is equivalent to the serial
//   loop.  Each round: P1 claims (64-bit atomicMin of the priority on every
//   footprint cell), grid barrier, P2 check-and-commit, grid barrier.  The
//   lowest-priority waiting agent always commits, so the loop ends after at
//   most (number of movers) rounds; in practice the longest local priority
//   chain.  Claims are cleared in the round after they were made (two claim
//   arrays), so no extra barrier is needed.
#include "fast_device.cuh"

namespace fastgb {

constexpr uint32_t MV_LEN = 0x7u;        // footprint path length (0..5)
constexpr uint32_t MV_EXIT = 0x8u;       // path ends on an exit cell
constexpr uint32_t MV_DONE = 0x10u;      // committed
constexpr uint32_t MV_GONE = 0x20u;      // left through an exit
constexpr int MV_SFIN_SHIFT = 8;         // final step index along the path

__device__ __forceinline__ int path_cell(int x0, int y0, int dx, int dy, int L, int s, int W) {
  return (y0 + div_half_away(s * dy, L)) * W + (x0 + div_half_away(s * dx, L));
}

// ---------------------------------------------------------------------------
// Footprints of all movers; agents that stay, or are blocked at their first
// path cell by an agent that stays, need no work at all.
__global__ void __launch_bounds__(256) k_move_prep(StepArgs a, Chunks ch) {
  const int t = a.ctl->t;
  unsigned alive_local = 0;
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const RepDev& R = a.reps[rep];
    const int end = min(ch.begin[c] + kChunk, a.n_slots[rep]);
    const int slot = ch.begin[c] + threadIdx.x;
    if (slot >= end) continue;
    const int cell = R.cell[slot];
    if (cell < 0) continue;
    ++alive_local;
    const int des = R.desired[slot];
    if (des == cell) continue;
    const int W = R.W;
    const int x0 = cell % W, y0 = cell / W;
    const int dx = des % W - x0, dy = des / W - y0;
    const int L = max(abs(dx), abs(dy));
    int fp = 0;
    uint32_t ex = 0;
    for (int s = 1; s <= L; ++s) {
      const uint32_t r = R.rec[path_cell(x0, y0, dx, dy, L, s, W)];
      if (r & REC_STA) break;
      if (rec_exit(r)) {
        ex = MV_EXIT;
        break;
      }
      fp = s;
    }
    if (fp == 0 && !ex) continue;
    R.prio[slot] = move_priority((uint32_t)R.id[slot], (uint32_t)t, R.seed_lo, R.seed_hi);
    R.mvinfo[slot] = (uint32_t)fp | ex;
    const uint32_t i = atomicAdd(&a.ctl->act_count[2], 1u);
    if (i < a.act_cap) a.act[2][i] = ((uint32_t)rep << 24) | (uint32_t)slot;
  }
  // agents alive at the start of the step
  for (int o = 16; o > 0; o >>= 1) alive_local += __shfl_xor_sync(0xffffffffu, alive_local, o);
  if ((threadIdx.x & 31) == 0 && alive_local)
    atomicAdd(&a.ctl->agent_steps, (unsigned long long)alive_local);
}

// ---------------------------------------------------------------------------
// Grid-wide barrier for a cooperative launch, with a time limit: a block that
// waits longer than ctl->barrier_ns_limit records FAST timeout in ctl->err and
// every block then leaves the kernel at its next barrier.
__device__ bool grid_barrier(Ctl* ctl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* vgen = &ctl->bar_gen;
    volatile int* verr = &ctl->err;
    const uint32_t g = *vgen;
    __threadfence();
    const uint32_t arrived = atomicAdd(&ctl->bar_count, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      const unsigned long long lim = ctl->barrier_ns_limit;
      while (*vgen == g) {
        if (*verr != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > lim) {
          atomicCAS(&ctl->err, 0, kDevErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*verr != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct Foot {
  int x0, y0, dx, dy, L, n, W;
  int c0;
};

__device__ __forceinline__ Foot footprint(const RepDev& R, int slot, uint32_t info) {
  Foot f;
  f.W = R.W;
  f.c0 = R.cell[slot];
  const int des = R.desired[slot];
  f.x0 = f.c0 % f.W;
  f.y0 = f.c0 / f.W;
  f.dx = des % f.W - f.x0;
  f.dy = des / f.W - f.y0;
  f.L = max(abs(f.dx), abs(f.dy));
  f.n = (int)(info & MV_LEN);
  return f;
}

__device__ __forceinline__ int foot_cell(const Foot& f, int s) {
  return s == 0 ? f.c0 : path_cell(f.x0, f.y0, f.dx, f.dy, f.L, s, f.W);
}

__global__ void __launch_bounds__(256) k_move_rounds(StepArgs a) {
  Ctl* ctl = a.ctl;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t gsz = gridDim.x * blockDim.x;
  const uint32_t n0 = min(__ldcg(&ctl->act_count[2]), a.act_cap);
  const uint32_t* in = a.act[2];
  uint32_t n_in = n0;
  int r = 0;
  bool ok = true;
  for (;;) {
    uint32_t* out = a.act[r & 1];
    uint32_t* out_cnt = &ctl->act_count[r & 1];
    // P1: clear last round's claims, claim this round's footprints
    for (uint32_t i = gtid; i < n_in; i += gsz) {
      const uint32_t e = in[i];
      const int rep = (int)(e >> 24), slot = (int)(e & 0xFFFFFFu);
      const RepDev& R = a.reps[rep];
      const uint32_t info = __ldcg(&R.mvinfo[slot]);
      const Foot f = footprint(R, slot, info);
      if (r > 0) {
        unsigned long long* old = R.claim[(r - 1) & 1];
        for (int s = 0; s <= f.n; ++s) __stcg(&old[foot_cell(f, s)], ~0ull);
      }
      if (!(info & MV_DONE)) {
        unsigned long long* now = R.claim[r & 1];
        const unsigned long long p = R.prio[slot];
        for (int s = 0; s <= f.n; ++s) atomicMin(&now[foot_cell(f, s)], p);
        const uint32_t j = atomicAdd(out_cnt, 1u);
        out[j] = e;
      }
    }
    if (!(ok = grid_barrier(ctl))) break;
    const uint32_t n_out = __ldcg(out_cnt);
    if (n_out == 0) break;
    if (r + 1 > (int)n0 + 1) {
      if (gtid == 0) atomicCAS(&ctl->err, 0, kDevErrRounds);
      ok = false;
      break;
    }
    if (gtid == 0) ctl->act_count[(r + 1) & 1] = 0u;  // next round's output counter
    // P2: commit the agents that own all their footprint cells
    for (uint32_t i = gtid; i < n_out; i += gsz) {
      const uint32_t e = out[i];
      const int rep = (int)(e >> 24), slot = (int)(e & 0xFFFFFFu);
      const RepDev& R = a.reps[rep];
      const uint32_t info = __ldcg(&R.mvinfo[slot]);
      const Foot f = footprint(R, slot, info);
      const unsigned long long p = R.prio[slot];
      const unsigned long long* now = R.claim[r & 1];
      bool mine = true;
      for (int s = 0; s <= f.n; ++s) mine = mine && (__ldcg(&now[foot_cell(f, s)]) == p);
      if (!mine) continue;
      // walk the path against the current occupancy
      int sfin = 0;
      bool gone = false;
      for (int s = 1; s <= f.L; ++s) {
        const int nc = foot_cell(f, s);
        const uint32_t rr = __ldcg(&R.rec[nc]);
        if (rr & REC_OCC) break;
        sfin = s;
        if (rec_exit(rr)) {
          gone = true;
          break;
        }
      }
      if (sfin > 0) {
        const uint32_t r0 = __ldcg(&R.rec[f.c0]);
        __stcg(&R.rec[f.c0], r0 & ~(REC_OCC | REC_STA));
        if (!gone) {
          const int fc = foot_cell(f, sfin);
          const uint32_t r1 = __ldcg(&R.rec[fc]);
          __stcg(&R.rec[fc], r1 | REC_OCC);
        }
      }
      __stcg(&R.mvinfo[slot],
             info | MV_DONE | (gone ? MV_GONE : 0u) | ((uint32_t)sfin << MV_SFIN_SHIFT));
    }
    if (!(ok = grid_barrier(ctl))) break;
    in = out;
    n_in = n_out;
    ++r;
  }
  if (!ok) return;
  // final positions
  for (uint32_t i = gtid; i < n0; i += gsz) {
    const uint32_t e = a.act[2][i];
    const int rep = (int)(e >> 24), slot = (int)(e & 0xFFFFFFu);
    const RepDev& R = a.reps[rep];
    const uint32_t info = __ldcg(&R.mvinfo[slot]);
    const int sfin = (int)(info >> MV_SFIN_SHIFT) & 0xF;
    if (info & MV_GONE) {
      R.cell[slot] = -1;
      atomicAdd(&a.exited[rep], 1);
    } else if (sfin > 0) {
      const Foot f = footprint(R, slot, info);
      R.cell[slot] = foot_cell(f, sfin);
    }
  }
  if (gtid == 0) {
    ctl->rounds_last = r;
    ctl->rounds_total += (unsigned long long)r;
    if (r > ctl->rounds_max) ctl->rounds_max = r;
  }
}

// ---------------------------------------------------------------------------
__global__ void k_step_begin(StepArgs a) {
  if (threadIdx.x == 0) {
    a.ctl->q_count = 0u;
    a.ctl->act_count[0] = 0u;
    a.ctl->act_count[1] = 0u;
    a.ctl->act_count[2] = 0u;
  }
}

__global__ void k_step_end(StepArgs a) {
  if (threadIdx.x == 0) {
    a.ctl->t += 1;
    a.ctl->q_count = 0u;
    a.ctl->act_count[0] = 0u;
    a.ctl->act_count[1] = 0u;
    a.ctl->act_count[2] = 0u;
  }
}

int move_prep_launch(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s) {
  if (ch.n <= 0) return 0;
  k_move_prep<<<grid, 256, 0, s>>>(a, ch);
  return 0;
}

int move_rounds_max_grid(int block, int* grid_out) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_move_rounds, block, 0) != cudaSuccess)
    return -1;
  *grid_out = sms * (per > 0 ? per : 1);
  return 0;
}

int move_rounds_launch(const StepArgs& a, int grid, int block, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_move_rounds, a) == cudaSuccess ? 0 : -1;
}

int step_begin_launch(const StepArgs& a, cudaStream_t s) {
  k_step_begin<<<1, 32, 0, s>>>(a);
  return 0;
}

int step_end_launch(const StepArgs& a, cudaStream_t s) {
  k_step_end<<<1, 32, 0, s>>>(a);
  return 0;
}

// A test of the bounded wait: block 0 leaves without arriving, so the other
// blocks' barrier can never complete; they must give up after the limit and
// report the timeout in ctl->err.
__global__ void k_test_barrier_timeout(Ctl* ctl) {
  if (blockIdx.x == 0) return;
  grid_barrier(ctl);
}

int test_barrier_timeout_launch(Ctl* ctl, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(64);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_test_barrier_timeout, ctl) == cudaSuccess ? 0 : -1;
}

}  // namespace fastgb
