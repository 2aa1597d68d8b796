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
// FP64 re-check, one warp per queued agent.  Lane l evaluates candidates
// l, l+32, l+64, l+96 in parallel; the sums are then formed in canonical
// order by broadcasting the weights one by one, exactly as the FP64 rule.
__global__ void __launch_bounds__(256) k_recheck(StepArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t n = min(a.ctl->q_count, a.q_cap);
  const int t = a.ctl->t;
  for (uint32_t q = warp; q < n; q += nwarps) {
    const uint32_t e = a.queue[q];
    const int rep = (int)(e >> 24), slot = (int)(e & 0xFFFFFFu);
    const RepDev& R = a.reps[rep];
    const int cell = R.cell[slot];
    const int id = R.id[slot];
    const uint32_t rec0 = R.rec[cell];
    const double S0 = s64_of(rec0);
    const unsigned long long m0 = R.mask[(size_t)cell * R.mw];
    const unsigned long long m1 = (R.K > 64) ? R.mask[(size_t)cell * R.mw + 1] : 0ull;
    const double nks = -R.kS;
    double w[4];
    int off[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = lane + 32 * j;
      w[j] = 0.0;
      off[j] = 0;
      if (k < R.K) {
        int dx, dy;
        kth_offset(R.v, R.reach, k, &dx, &dy);
        off[j] = dy * R.W + dx;
        const bool center = (dx == 0 && dy == 0);
        if (mask_bit(m0, m1, k)) {
          const uint32_t r = center ? rec0 : R.rec[cell + off[j]];
          if (center || !(r & REC_OCC))
            w[j] = exp64(__dmul_rn(nks, __dsub_rn(s64_of(r), S0)));
        }
      }
    }
    double W = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      for (int l = 0; l < 32; ++l) {
        const double wk = __shfl_sync(0xffffffffu, w[j], l);
        if (32 * j + l < R.K && wk > 0.0) W = __dadd_rn(W, wk);
      }
    const double u = plan_uniform((uint32_t)id, (uint32_t)t, R.seed_lo, R.seed_hi);
    const double r = __dmul_rn(u, W);
    double c = 0.0;
    int chosen = -1, last = -1;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      for (int l = 0; l < 32; ++l) {
        const int k = 32 * j + l;
        const double wk = __shfl_sync(0xffffffffu, w[j], l);
        if (k < R.K && wk > 0.0) {
          c = __dadd_rn(c, wk);
          if (chosen < 0 && r < c) chosen = k;
          last = k;
        }
      }
    if (chosen < 0) chosen = last;
    const int src = chosen & 31, jj = chosen >> 5;
    int o = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int oj = __shfl_sync(0xffffffffu, off[j], src);
      if (j == jj) o = oj;
    }
    if (lane == 0) {
      const int target = cell + o;
      R.desired[slot] = target;
      set_static(R.rec, cell, rec0, target == cell);
    }
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
  k_recheck<<<grid, 256, 0, s>>>(a);
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
