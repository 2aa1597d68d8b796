// plan.cu -- FP64 re-check kernel and the dispatch of the planning kernels
// (instantiated per v_m in plan_v1.cu .. plan_v5.cu, templates in
// plan_kernels.cuh).
#include "plan_kernels.cuh"

namespace fastgb {

int plan_launch_v1(const StepArgs&, int, int, int, const Chunks&, int, cudaStream_t, bool);
int plan_launch_v2(const StepArgs&, int, int, int, const Chunks&, int, cudaStream_t, bool);
int plan_launch_v3(const StepArgs&, int, int, int, const Chunks&, int, cudaStream_t, bool);
int plan_launch_v4(const StepArgs&, int, int, int, const Chunks&, int, cudaStream_t, bool);
int plan_launch_v5(const StepArgs&, int, int, int, const Chunks&, int, cudaStream_t, bool);
int diag_launch_v1(const StepArgs&, int, const Chunks&, int, cudaStream_t);
int diag_launch_v2(const StepArgs&, int, const Chunks&, int, cudaStream_t);
int diag_launch_v3(const StepArgs&, int, const Chunks&, int, cudaStream_t);
int diag_launch_v4(const StepArgs&, int, const Chunks&, int, cudaStream_t);
int diag_launch_v5(const StepArgs&, int, const Chunks&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 re-check of the queued agents, A agents per block of 256 threads:
// A = kRcAgents (8) when the queue is long, fewer when it is short, so that
// the few agents of a short queue spread over more SMs (the queue's length is
// known on the device only; the grid is sized for a long one).  The threads
// share out all FP64 weights of the block's agents (the
// flattened list of (agent, candidate) pairs, about one exp64 per thread, so
// their long FP64 latencies overlap and every FP64 instruction is full), then
// thread i forms agent i's cumulative sums C_k sequentially in canonical
// order, exactly as the FP64 rule does (W is the last of them: the same
// additions in the same order), and finds the first k with fl(u*W) < C_k by
// comparing bit patterns (order-preserving for non-negative doubles).
constexpr int kRcThreads = 256;
constexpr int kRcAgents = 8;

struct RcAgent {
  unsigned long long m0, m1;
  double S0, nks;
  const uint32_t* rec;
  int cell, W, v, H;
};

__global__ void __launch_bounds__(kRcThreads) k_recheck(StepArgs a) {
  __shared__ int8_t s_tab[5][kMaxK][2];
  __shared__ int s_K[5];
  __shared__ int s_first[kRcAgents + 1];  // prefix of the agents' candidate counts
  __shared__ RcAgent s_ag[kRcAgents];
  __shared__ double s_c[kRcAgents][kMaxK];  // weights, then C_k
  const uint32_t n = min(a.ctl->q_count, a.q_cap);
  const uint32_t A = n <= gridDim.x / 8u ? 2u : (n <= gridDim.x / 2u ? 4u : (uint32_t)kRcAgents);
  if ((uint32_t)blockIdx.x * A >= n) return;
  const int reach = a.reps[0].reach;  // one reach set per context
  if (threadIdx.x < 5) {
    const int v = threadIdx.x + 1;
    int k = 0;
    for (int dy = -v; dy <= v; ++dy)
      for (int dx = -v; dx <= v; ++dx)
        if (reach_in(dx, dy, v, reach)) {
          s_tab[v - 1][k][0] = (int8_t)dx;
          s_tab[v - 1][k][1] = (int8_t)dy;
          ++k;
        }
    s_K[v - 1] = k;
  }
  __syncthreads();
  const int tid = threadIdx.x;
  const int t = a.ctl->t;
  for (uint32_t q0 = blockIdx.x * A; q0 < n; q0 += gridDim.x * A) {
    // thread i < A: agent q0 + i (threads A..kRcAgents-1 have no agent and
    // no candidates)
    bool mine = (uint32_t)tid < A && q0 + tid < n;
    int rep = 0, slot = 0, K = 0;
    uint32_t rec0 = 0;
    if (mine) {
      const uint32_t e = a.queue[q0 + tid];
      rep = (int)(e >> 24);
      slot = (int)(e & 0xFFFFFFu);
      // debug build: the queue entry, the agent's cell and speed checked
      if (kChecked)
        mine = fg_in(a.ctl, rep, a.n_rep) && fg_in(a.ctl, slot, a.reps[rep].cap) &&
               fg_in(a.ctl, a.reps[rep].cell[slot], (long long)a.reps[rep].W * a.reps[rep].H) &&
               (!a.reps[rep].speed || fg_in(a.ctl, (long long)a.reps[rep].speed[slot] - 1, 5));
    }
    if (mine) {
      const RepDev& R = a.reps[rep];
      RcAgent x;
      x.cell = R.cell[slot];
      x.W = R.W;
      x.H = R.H;
      x.v = R.speed ? (int)R.speed[slot] : R.v;  // the agent's own maximum speed
      x.rec = R.rec;
      rec0 = R.rec[x.cell];
      x.S0 = s64_of(rec0);
      x.nks = -R.kS;
      const unsigned long long* mk = R.mask_v[x.v - 1];
      const int mw = s_K[x.v - 1] > 64 ? 2 : 1;
      x.m0 = mk[(size_t)x.cell * mw];
      x.m1 = (mw > 1) ? mk[(size_t)x.cell * mw + 1] : 0ull;
      s_ag[tid] = x;
      K = s_K[x.v - 1];
    }
    if (tid < 32) {
      int incl = K;  // lanes >= kRcAgents hold 0
#pragma unroll
      for (int o = 1; o < kRcAgents; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += y;
      }
      if (tid < kRcAgents) s_first[tid + 1] = incl;
      if (tid == 0) s_first[0] = 0;
    }
    __syncthreads();
    const int total = s_first[kRcAgents];
    // every FP64 weight of the block's agents
    for (int idx = tid; idx < total; idx += kRcThreads) {
      int i = 0;
#pragma unroll
      for (int step = kRcAgents / 2; step > 0; step >>= 1)
        if (s_first[i + step] <= idx) i += step;
      const int k = idx - s_first[i];
      const RcAgent& x = s_ag[i];
      double wk = 0.0;
      if (mask_bit(x.m0, x.m1, k)) {
        const int dx = s_tab[x.v - 1][k][0], dy = s_tab[x.v - 1][k][1];
        const bool center = (dx == 0 && dy == 0);
        const bool in = !kChecked || fg_in(a.ctl, (long long)x.cell + dy * x.W + dx,
                                            (long long)x.W * x.H);
        const uint32_t r = in ? x.rec[x.cell + dy * x.W + dx] : REC_OCC;
        if (center || !(r & REC_OCC)) wk = exp64(__dmul_rn(x.nks, __dsub_rn(s64_of(r), x.S0)));
      }
      s_c[i][k] = wk;
    }
    __syncthreads();
    if (mine) {
      // C_k in canonical order over the positive weights (a zero weight is
      // marked -1 and never chosen); W = the last C
      double* ci = s_c[tid];
      double acc = 0.0;
      for (int k = 0; k < K; ++k) {
        const double wk = ci[k];
        const bool pos = __double_as_longlong(wk) != 0ll;
        if (pos) acc = __dadd_rn(acc, wk);
        ci[k] = pos ? acc : -1.0;
      }
      const RepDev& R = a.reps[rep];
      const double u = plan_uniform((uint32_t)R.id[slot], (uint32_t)t, R.seed_lo, R.seed_hi);
      const long long rb = __double_as_longlong(__dmul_rn(u, acc));
      int chosen = -1, last = -1;
      for (int k = 0; k < K; ++k) {
        const long long cb = __double_as_longlong(ci[k]);
        if (cb >= 0) {
          if (chosen < 0 && rb < cb) chosen = k;
          last = k;
        }
      }
      const RcAgent& x = s_ag[tid];
      const int kk = chosen >= 0 ? chosen : last;
      const int target = x.cell + s_tab[x.v - 1][kk][1] * x.W + s_tab[x.v - 1][kk][0];
      R.desired[slot] = target;
      set_static(R.rec, x.cell, rec0, target == x.cell);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.ctl->rechecked_total, (unsigned long long)n);
}

int plan_groups_launch(const StepArgs& a, int v, int reach, int lanes, int precision,
                       const Chunks& ch, int grid, cudaStream_t s, bool diag) {
  if (ch.n <= 0) return 0;
  switch (v) {
    case 1: return plan_launch_v1(a, reach, lanes, precision, ch, grid, s, diag);
    case 2: return plan_launch_v2(a, reach, lanes, precision, ch, grid, s, diag);
    case 3: return plan_launch_v3(a, reach, lanes, precision, ch, grid, s, diag);
    case 4: return plan_launch_v4(a, reach, lanes, precision, ch, grid, s, diag);
    case 5: return plan_launch_v5(a, reach, lanes, precision, ch, grid, s, diag);
  }
  return -1;
}

int plan_recheck_launch(const StepArgs& a, int grid, cudaStream_t s) {
  k_recheck<<<grid, kRcThreads, 0, s>>>(a);
  return 0;
}

int plan_diag_compare_launch(const StepArgs& a, int v, int reach, const Chunks& ch, int grid,
                             cudaStream_t s) {
  if (ch.n <= 0) return 0;
  switch (v) {
    case 1: return diag_launch_v1(a, reach, ch, grid, s);
    case 2: return diag_launch_v2(a, reach, ch, grid, s);
    case 3: return diag_launch_v3(a, reach, ch, grid, s);
    case 4: return diag_launch_v4(a, reach, ch, grid, s);
    case 5: return diag_launch_v5(a, reach, ch, grid, s);
  }
  return -1;
}

}  // namespace fastgb
