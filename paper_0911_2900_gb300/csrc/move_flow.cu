// move_flow.cu -- the movement phase as a dataflow over its conflict graph,
// equal bit for bit to moving the agents one after another in priority order
// (Kretz, Sec. 1: the movement is sequential, which rules out conflicts).
//
// Footprints are those of move.cu: start cell + path cells up to (not
// including) the first cell held by an agent that stays this step, or the
// first exit cell.  A mover reads and writes only cells of its footprint
// (plus constant cells), so two movers conflict only when their footprints
// share a cell, and moving each mover once every conflicting mover that comes
// before it has moved gives the serial result (any topological order of the
// conflict graph does).  On each footprint cell it is enough to wait for the
// mover just before it on that cell: the movers of one cell form a chain.
//
//   pass 1   every mover pushes one node per footprint cell onto that cell's
//            list (an atomic exchange of the list head; heads carry the
//            pass's tag, so the heads of earlier passes read as empty lists);
//   barrier  the only grid barrier of a step without overflow (below);
//   pass 2   every mover walks the lists of its cells: on each cell, whether
//            some mover there comes before it (d counts such cells) and which
//            mover comes right after it (its successor there); it stores its
//            successors and adds d to its counter (zeroed in pass 1);
//   release  a mover that has moved takes one off the counter of its
//            successor on each cell; whoever's operation leaves a counter at
//            zero (the mover's own addition of d, or a predecessor's
//            subtraction) owns that mover: the thread moves one such mover
//            next itself and puts the others on its block's list;
//   rounds   a block moves its list in rounds separated by block barriers,
//            until the list stays empty -- no block waits for another;
//   waves    a full list spills into a global overflow list; after a grid
//            barrier the blocks share its new entries out and run rounds
//            again, until a barrier finds no new entries.
// A counter receives +d once and -1 once from each of its d cells'
// predecessors, in any order, so exactly one of those operations leaves it
// at zero: each mover moves exactly once, after all its predecessors.
// All counter updates are relaxed atomics: a fence before a mover's addition
// publishes its successor list, a fence before a moved mover's subtractions
// releases its writes, and the thread that moves a mover first reads its
// counter with an acquire load.  A mover with d = 0 finds its footprint as
// the movement-order pass read it and applies the outcome that pass
// recorded (occupancy bits only).  Every wait is bounded: the grid
// barrier has a time limit, list walks and rounds have length limits.
#include "move_common.cuh"

namespace fastgb {

constexpr uint32_t kEnd = 0xFFFFFFFFu;  // end of a list / no successor
constexpr int kMaxWalk = 1024;          // nodes of one list (at most (2*5+1)^2 movers reach a cell)
constexpr uint32_t kDeal = 32;          // movers dealt to the blocks at a time
constexpr int kDevErrFlow = 7;          // device error: a list or the overflow list is corrupt

// Tag of this pass's list heads: one more than the last pass's, restarting
// at 1 once the movement-order pass has cleared the heads (it does so when
// the tags reach kFlowEpochWrap).
__device__ __forceinline__ uint32_t flow_epoch(const Ctl* ctl) {
  const uint32_t e = __ldcg(&ctl->move_epoch);
  return e >= kFlowEpochWrap ? 1u : e + 1u;
}

struct FlowBlock {
  uint32_t* list[2];  // shared memory, kFlowQ entries each
  uint32_t* cnt;      // shared: entries pushed onto each list (may exceed the capacity)
  uint32_t* ovf;      // shared: entries this block spilled since the last grid barrier
  uint32_t* rel;      // shared: movers released to this block in the step
  uint32_t qcap;      // list capacity in use
};

// Hands mover j to this block: onto list `out`, or the overflow list.
__device__ __forceinline__ void flow_enqueue(const StepArgs& a, const FlowBlock& fb, int out,
                                             uint32_t j) {
  const uint32_t pos = atomicAdd(&fb.cnt[out], 1u);
  if (pos < fb.qcap) {
    fb.list[out][pos] = j;
    return;
  }
  atomicAdd(fb.ovf, 1u);
  const uint32_t o = atomicAdd(&a.ctl->ovf_count, 1u);
  if (o < a.act_cap)
    a.flow_ovf[o] = j;
  else
    atomicCAS(&a.ctl->err, 0, kDevErrFlow);  // cannot happen: each mover is enqueued once
}

// After a mover has moved and a fence has made its writes visible: one off
// the counter of its successor on each of its cells (relaxed atomics; the
// fence before them releases the mover's writes).  Returns one successor
// this leaves at zero (kEnd: none), for the calling thread to move next; the
// others go to the block.
__device__ __forceinline__ uint32_t flow_release(const StepArgs& a, const FlowBlock& fb, int out,
                                                 const uint32_t* sc) {
  int old[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) old[s] = sc[s] != kEnd ? atomicSub(&a.flow_cnt[sc[s]], 1) : 0;
  uint32_t next = kEnd;
#pragma unroll
  for (int s = 0; s < 6; ++s)
    if (sc[s] != kEnd && old[s] == 1) {
      atomicAdd(fb.rel, 1u);
      if (next == kEnd)
        next = sc[s];
      else
        flow_enqueue(a, fb, out, sc[s]);
    }
  return next;
}

// A release-acquire fence at GPU scope: orders this thread's earlier memory
// operations before its later ones as the release and acquire patterns of
// the counters need (lighter than __threadfence, a sequentially consistent
// fence).
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ int ld_acquire_s32(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];"
               : "=r"(v)
               : "l"(__cvta_generic_to_global(p))
               : "memory");
  return v;
}

// Moves mover m, whose counter is at zero and which this thread owns, then
// one after the other the successors each move leaves at zero (one per move;
// the others go to the block).  Per move: an acquire load of the counter
// orders the reads of the walk's records after every predecessor's writes
// (a mover without predecessors applies the outcome the movement-order pass
// recorded, reading nothing); a fence after the commit releases its writes
// to the successors.
__device__ __forceinline__ void flow_move_chain(const StepArgs& a, const PathTab* tab,
                                                const FlowBlock& fb, int out, uint32_t m,
                                                uint32_t limit) {
  for (uint32_t hop = 0; m != kEnd; ++hop) {
    if (hop > limit) {  // cannot happen: each mover moves once
      atomicCAS(&a.ctl->err, 0, kDevErrRounds);
      return;
    }
    const MoveEntry e = a.act[2][m];
    const uint4 s03 = __ldcg(reinterpret_cast<const uint4*>(a.flow_succ) + 2 * (size_t)m);
    const uint4 s47 = __ldcg(reinterpret_cast<const uint4*>(a.flow_succ) + 2 * (size_t)m + 1);
    if (ld_acquire_s32(&a.flow_cnt[m]) != 0) atomicCAS(&a.ctl->err, 0, kDevErrFlow);
    const int rep = (int)(e.ref >> 24), slot = (int)(e.ref & 0xFFFFFFu);
    const RepDev& R = a.reps[rep];
    int c[6], q[6];
    foot_cells(tab, e.c0, R, e.info, c, q);
    if (s47.z == 0u) {
      commit_first(a, R, rep, slot, c, e.info);
    } else {
      const int wl = walk_len(e.info);
      uint32_t pr[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) pr[s] = (s <= wl) ? __ldcg(&R.rec[c[s]]) : REC_OCC;
      commit_move(a, R, rep, slot, c, pr);
    }
    fence_acq_rel();
    const uint32_t sc[6] = {s03.x, s03.y, s03.z, s03.w, s47.x, s47.y};
    m = flow_release(a, fb, out, sc);
  }
}

// Moves every entry of list `in` (shared memory, n entries) and then the
// lists they release, round after round, until none is left.  Returns the
// number of rounds; the lists are empty on return.
__device__ __forceinline__ uint32_t flow_rounds(const StepArgs& a, const PathTab* tab,
                                                const FlowBlock& fb, int in, uint32_t limit) {
  uint32_t r = 0;
  for (;;) {
    __syncthreads();  // pushes onto `in` are complete, the other list's count is reset
    const uint32_t n = min(fb.cnt[in], fb.qcap);
    if (n == 0u) break;
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x)
      flow_move_chain(a, tab, fb, in ^ 1, fb.list[in][k], limit);
    __syncthreads();  // every read of list `in` is done
    if (threadIdx.x == 0) fb.cnt[in] = 0u;
    in ^= 1;
    if (++r > limit) {  // cannot happen: a round moves at least one mover
      if (threadIdx.x == 0) atomicCAS(&a.ctl->err, 0, kDevErrRounds);
      break;
    }
  }
  return r;
}

__global__ void __launch_bounds__(kMoveThreads, 2) k_move_flow(StepArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ PathTab tab;
  __shared__ uint32_t s_cnt[2], s_ovf, s_rel;
  build_path_tab(&tab);
  Ctl* ctl = a.ctl;
  const uint32_t E = flow_epoch(ctl);
  const uint32_t n0 = min(__ldcg(&ctl->act_count[2]), a.act_cap);
  const uint32_t G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  FlowBlock fb;
  fb.list[0] = reinterpret_cast<uint32_t*>(dsm);
  fb.list[1] = fb.list[0] + kFlowQ;
  fb.cnt = s_cnt;
  fb.ovf = &s_ovf;
  fb.rel = &s_rel;
  const uint32_t qc = __ldcg(&ctl->flow_qcap);
  fb.qcap = (qc == 0u || qc > (uint32_t)kFlowQ) ? (uint32_t)kFlowQ : qc;
  // the step's movers go to the blocks in turn, kDeal at a time: the block's
  // k-th mover is entry mover_at(k), k < nb
  const uint32_t nch = (n0 + kDeal - 1) / kDeal;
  uint32_t nb = (b < nch ? (nch - 1 - b) / G + 1 : 0u) * kDeal;
  if (n0 % kDeal && nch && (nch - 1) % G == b) nb -= kDeal - n0 % kDeal;
  auto mover_at = [&](uint32_t k) { return ((k / kDeal) * G + b) * kDeal + k % kDeal; };
  if (tid < 2) s_cnt[tid] = 0u;
  if (tid == 0) s_ovf = s_rel = 0u;
  const unsigned long long t_start = global_ns();
  if (b == 0 && tid == 0) ctl->round_ns[0] = t_start;
  __syncthreads();

  // ---- pass 1: one node per footprint cell, pushed onto the cell's list
  for (uint32_t k = tid; k < nb; k += blockDim.x) {
    const uint32_t m = mover_at(k);
    const MoveEntry e = a.act[2][m];
    const RepDev& R = a.reps[e.ref >> 24];
    int c[6], q[6];
    foot_cells(&tab, e.c0, R, e.info, c, q);
    const int n = (int)(e.info & MV_LEN);
    unsigned long long old[6];
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (s <= n) old[s] = atomicExch(&R.head[q[s]], ((unsigned long long)E << 32) | (6u * m + s));
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (s <= n) {
        const uint32_t nxt = (uint32_t)(old[s] >> 32) == E ? (uint32_t)old[s] : kEnd;
        a.flow_node[6 * (size_t)m + s] = ((unsigned long long)e.prio << 32) | nxt;
      }
    a.flow_cnt[m] = 0;
  }
  if (tid == 0) atomicMax(&ctl->phase_ns[0], global_ns() - t_start);
  uint32_t nbar = 0, bsum0 = 0u, bsum1 = 0u;
  if (!grid_barrier(ctl, nbar)) return;
  if (tid == 0) atomicMax(&ctl->phase_ns[1], global_ns() - t_start);

  // ---- pass 2: predecessors and successors on every footprint cell; the
  // lists of a mover's cells are walked side by side
  uint32_t n_first = 0, walk_max = 0;
  unsigned long long walk_sum = 0ull;
  for (uint32_t k = tid; k < nb; k += blockDim.x) {
    const uint32_t m = mover_at(k);
    const MoveEntry e = a.act[2][m];
    const RepDev& R = a.reps[e.ref >> 24];
    int c[6], q[6];
    foot_cells(&tab, e.c0, R, e.info, c, q);
    const int n = (int)(e.info & MV_LEN);
    uint32_t cur[6], sn[6], sp[6];
    uint32_t pred = 0u;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      cur[s] = (s <= n) ? (uint32_t)__ldcg(&R.head[q[s]]) : kEnd;
      sn[s] = kEnd;
      sp[s] = 0xFFFFFFFFu;
    }
    const uint32_t n_nodes = 6u * n0;
    for (int it = 0;; ++it) {
      bool any = false;
      unsigned long long nv[6];
#pragma unroll
      for (int s = 0; s < 6; ++s)
        if (cur[s] != kEnd && cur[s] >= n_nodes) {  // cannot happen: a corrupt list
          atomicCAS(&ctl->err, 0, kDevErrFlow);
          cur[s] = kEnd;
        }
#pragma unroll
      for (int s = 0; s < 6; ++s)
        if (cur[s] != kEnd) nv[s] = __ldcg(&a.flow_node[cur[s]]);
#pragma unroll
      for (int s = 0; s < 6; ++s)
        if (cur[s] != kEnd) {
          const uint32_t p = (uint32_t)(nv[s] >> 32);
          if (p < e.prio) pred |= 1u << s;
          if (p > e.prio && p < sp[s]) {
            sp[s] = p;
            sn[s] = cur[s];
          }
          cur[s] = (uint32_t)nv[s];
          any = any || cur[s] != kEnd;
          ++walk_sum;
        }
      walk_max = max(walk_max, (uint32_t)it + 1u);
      if (!any) break;
      if (it >= kMaxWalk) {
        atomicCAS(&ctl->err, 0, kDevErrFlow);
        break;
      }
    }
    uint32_t sc[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) sc[s] = sn[s] != kEnd ? sn[s] / 6u : kEnd;
    const int d = __popc(pred);
    // successors and d (word 6), published by the fence before the counter
    // can reach zero
    uint4* sd = reinterpret_cast<uint4*>(a.flow_succ) + 2 * (size_t)m;
    __stcg(sd, make_uint4(sc[0], sc[1], sc[2], sc[3]));
    __stcg(sd + 1, make_uint4(sc[4], sc[5], (uint32_t)d, kEnd));
    fence_acq_rel();
    const int old = atomicAdd(&a.flow_cnt[m], d);
    if (old + d == 0) flow_enqueue(a, fb, 0, m);  // no predecessors, or all have moved
    n_first += d == 0;
  }
  if (tid == 0) atomicMax(&ctl->phase_ns[2], global_ns() - t_start);

  // ---- rounds of the block's own list, then waves over the overflow list
  uint32_t rounds = flow_rounds(a, &tab, fb, 0, n0 + 1u);
  uint32_t waves = 0, ovf_done = 0;
  if (tid == 0) atomicMax(&ctl->phase_ns[3], global_ns() - t_start);
  for (;;) {
    __syncthreads();
    const uint32_t spilled = s_ovf;
    uint32_t fresh = 0u;
    if (!grid_barrier_sum(ctl, nbar, bsum0, bsum1, spilled, &fresh)) return;
    if (tid == 0) s_ovf = 0u;
    if (fresh == 0u) break;
    // this block's share of the overflow entries [ovf_done, ovf_done + fresh)
    const uint32_t lo = ovf_done + (uint32_t)(((unsigned long long)fresh * b) / G);
    const uint32_t hi = ovf_done + (uint32_t)(((unsigned long long)fresh * (b + 1)) / G);
    ovf_done += fresh;
    if (ovf_done > a.act_cap) {
      if (tid == 0) atomicCAS(&ctl->err, 0, kDevErrFlow);
      return;  // every block sees the same sums, so all leave here
    }
    __syncthreads();
    for (uint32_t i = lo + tid; i < hi; i += blockDim.x)
      flow_move_chain(a, &tab, fb, 0, __ldcg(&a.flow_ovf[i]), n0 + 1u);
    rounds += flow_rounds(a, &tab, fb, 0, n0 + 1u);
    ++waves;
    if (waves > n0 + 1u) {
      if (tid == 0) atomicCAS(&ctl->err, 0, kDevErrRounds);
      return;
    }
  }
  // statistics of the step (sums and maxima over the threads and blocks)
  for (int o = 16; o > 0; o >>= 1) {
    walk_max = max(walk_max, __shfl_xor_sync(0xffffffffu, walk_max, o));
    walk_sum += __shfl_xor_sync(0xffffffffu, walk_sum, o);
    n_first += __shfl_xor_sync(0xffffffffu, n_first, o);
  }
  if ((tid & 31) == 0) {
    atomicMax(&ctl->flow_stat[0], (unsigned long long)walk_max);
    atomicAdd(&ctl->flow_stat[1], walk_sum);
    atomicAdd(&ctl->flow_stat[2], (unsigned long long)n_first);
  }
  if (tid == 0) {
    atomicAdd(&ctl->flow_stat[3], (unsigned long long)s_rel);
    atomicMax(&ctl->flow_stat[4], (unsigned long long)nb);
    atomicMax(&ctl->flow_stat[5], (unsigned long long)s_rel);
    atomicMax(&ctl->phase_ns[7], (unsigned long long)rounds);
    atomicMax((unsigned int*)&ctl->rounds_last, rounds + waves + 2u);
  }
  if (b == 0 && tid == 0) {
    // every block has read the pass's tag (the last barrier is behind them)
    ctl->move_epoch = E;
    ctl->flow_waves = waves;
    ctl->phase_ns[6] = (unsigned long long)waves;
    ctl->movers_total += (unsigned long long)n0;
    ctl->round_ns[1] = global_ns();
  }
}

// Sums of the last step's movement statistics, kept by one thread after the
// movement kernel: rounds of the step (the most any block ran, plus the
// waves and pass 2), their total and maximum.
__global__ void k_move_flow_stats(Ctl* ctl) {
  if (threadIdx.x != 0) return;
  const int r = ctl->rounds_last;
  ctl->rounds_total += (unsigned long long)r;
  if (r > ctl->rounds_max) ctl->rounds_max = r;
}

size_t move_flow_smem() { return (size_t)2 * kFlowQ * sizeof(uint32_t); }

int move_flow_max_grid(int block, int* grid_out) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaFuncSetAttribute(k_move_flow, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)move_flow_smem()) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_move_flow, block, move_flow_smem()) !=
      cudaSuccess)
    return -1;
  *grid_out = sms * (per > 0 ? per : 1);
  return 0;
}

int move_flow_launch(const StepArgs& a, int grid, int block, cudaStream_t s) {
  // the step's largest round count is gathered by atomicMax from zero
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = move_flow_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_move_flow, a) != cudaSuccess) return -1;
  k_move_flow_stats<<<1, 32, 0, s>>>(a.ctl);
  return 0;
}

}  // namespace fastgb
