// plan_v3.cu -- planning kernels instantiated for v_m = 3 (all reach sets,
// lanes per agent and precisions); one translation unit per v_m so that the
// library compiles in parallel.
#include "plan_kernels.cuh"

namespace fastgb {

int plan_launch_v3(const StepArgs& a, int reach, int lanes, int precision, const Chunks& ch,
                    int grid, cudaStream_t s, bool diag) {
  return launch_one_v<3>(a, reach, lanes, precision, ch, grid, s, diag);
}

int diag_launch_v3(const StepArgs& a, int reach, const Chunks& ch, int grid, cudaStream_t s) {
  return diag_one_v<3>(a, reach, ch, grid, s);
}

}  // namespace fastgb
