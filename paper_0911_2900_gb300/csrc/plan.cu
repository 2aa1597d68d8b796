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
// FP64 re-check of the queued agents: 8 lanes per agent compute the FP64
// weights of candidates k = l, l+8, ... (independent, so their latency
// overlaps), then lane 0 of the group forms W and the cumulative sums
// sequentially in canonical order, exactly as the FP64 rule does.
constexpr int kRcLanes = 8;
constexpr int kRcPerBlock = 128 / kRcLanes;

__global__ void __launch_bounds__(128) k_recheck(StepArgs a) {
  __shared__ int8_t s_tab[5][kMaxK][2];
  __shared__ int s_K[5];
  __shared__ double s_w[kRcPerBlock][kMaxK];
  const uint32_t n = min(a.ctl->q_count, a.q_cap);
  if ((uint32_t)blockIdx.x * kRcPerBlock >= n) return;
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
  const int g = threadIdx.x / kRcLanes, l = threadIdx.x % kRcLanes;
  const int t = a.ctl->t;
  for (uint32_t base = blockIdx.x * kRcPerBlock; base < n; base += gridDim.x * kRcPerBlock) {
    const uint32_t q = base + g;
    const bool valid = q < n;
    int rep = 0, slot = 0, cell = 0, K = 0, v = 1, W = 0;
    uint32_t rec0 = 0;
    double* w = s_w[g];
    if (valid) {
      const uint32_t e = a.queue[q];
      rep = (int)(e >> 24);
      slot = (int)(e & 0xFFFFFFu);
      const RepDev& R = a.reps[rep];
      cell = R.cell[slot];
      v = R.v;
      W = R.W;
      K = s_K[v - 1];
      rec0 = R.rec[cell];
      const double S0 = s64_of(rec0);
      const unsigned long long m0 = R.mask[(size_t)cell * R.mw];
      const unsigned long long m1 = (R.mw > 1) ? R.mask[(size_t)cell * R.mw + 1] : 0ull;
      const double nks = -R.kS;
      for (int k = l; k < K; k += kRcLanes) {
        double wk = 0.0;
        if (mask_bit(m0, m1, k)) {
          const int dx = s_tab[v - 1][k][0], dy = s_tab[v - 1][k][1];
          const bool center = (dx == 0 && dy == 0);
          const uint32_t r = center ? rec0 : R.rec[cell + dy * W + dx];
          if (center || !(r & REC_OCC)) wk = exp64(__dmul_rn(nks, __dsub_rn(s64_of(r), S0)));
        }
        w[k] = wk;
      }
    }
    __syncwarp();
    if (valid && l == 0) {
      const RepDev& R = a.reps[rep];
      double Wsum = 0.0;
      for (int k = 0; k < K; ++k)
        if (w[k] > 0.0) Wsum = __dadd_rn(Wsum, w[k]);
      const double u = plan_uniform((uint32_t)R.id[slot], (uint32_t)t, R.seed_lo, R.seed_hi);
      const double r = __dmul_rn(u, Wsum);
      double c = 0.0;
      int chosen = -1, last = -1;
      for (int k = 0; k < K; ++k) {
        if (w[k] > 0.0) {
          c = __dadd_rn(c, w[k]);
          if (chosen < 0 && r < c) chosen = k;
          last = k;
        }
      }
      const int kk = chosen >= 0 ? chosen : last;
      const int target = cell + s_tab[v - 1][kk][1] * W + s_tab[v - 1][kk][0];
      R.desired[slot] = target;
      set_static(R.rec, cell, rec0, target == cell);
    }
    __syncwarp();
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
  k_recheck<<<grid, 128, 0, s>>>(a);
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
