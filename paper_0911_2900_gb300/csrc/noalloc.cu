// noalloc.cu -- a planning pass that allocates no device memory.
//
// Who needs it: code that must not call cudaMalloc (or any allocator) at the
// moment it plans -- for instance a caller that is in the middle of capturing
// a CUDA graph on its stream (allocation calls are not allowed there), a host
// whose device memory is entirely owned by another allocator, or a real-time
// loop that cannot afford an allocation's latency or its failure.  Such a
// caller gives the input state (a context set up earlier) and an output
// buffer it already owns; the only scratch this pass needs, the queue of
// draws to re-evaluate in FP64, lives in a fixed array that the library
// carries in the device's global memory for as long as it is loaded.
//
// What it computes: the desired cell of every agent of one replicate for a
// given step -- FP32 weights, margin test (the same draw and margin code as
// the context's planning kernels), FP64 re-check of the draws inside the
// margin -- written by agent id into the caller's buffer.  It always plans
// this way, whatever precision the context was created with, so its output
// is the FP64 rule's choice: equal to a planning pass of an FP64 or an
// FP32-with-re-check context (an FP32-without-re-check context, a
// diagnostic mode, may choose differently near a boundary).  The context's
// own state is not touched.
//
// Limits: at most kNoAllocMaxAgents agent slots per replicate (the queue must
// hold every agent in the worst case).  Every call on a device shares the one
// array, so calls that overlap on the GPU (on different streams, or from
// different host threads without ordering) race on it.
#include <algorithm>
#include <mutex>

#include "plan_kernels.cuh"

namespace fastgb {

constexpr int kNoAllocMaxAgents = 1 << 20;

// Word 0: number of queued agents of the current call; words 1..: their slots.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocMaxAgents + 64];

// FP32 planning, one thread per agent; a draw far from every cumulative
// boundary is written out, the others are queued for the FP64 rule.
template <int V, int REACH>
__global__ void __launch_bounds__(128) k_noalloc_plan(RepDev R, int32_t cap, int32_t t,
                                                      int32_t* out, int32_t bound,
                                                      uint32_t* scratch) {
  constexpr int K = reach_count(V, REACH);
  constexpr int CENTER = reach_center<V, REACH>();
  __shared__ int s_off[K];
  fill_offsets(s_off, V, REACH, R.W);
  __syncthreads();
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < cap;
       slot += gridDim.x * blockDim.x) {
    const int cell = R.cell[slot];
    if (cell < 0) continue;
    const int id = R.id[slot];
    const uint32_t rec0 = R.rec[cell];
    const unsigned long long m0 = R.mask[(size_t)cell * R.mw];
    const unsigned long long m1 = (K > 64) ? R.mask[(size_t)cell * R.mw + 1] : 0ull;
    const int a0 = rec_a(rec0), b0 = rec_b(rec0);
    float cw[K];  // cumulative weights C_k
    float Wt = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float wk = 0.f;
      if (k == CENTER) {
        wk = 1.0f;
      } else if (mask_bit(m0, m1, k)) {
        const uint32_t r = R.rec[cell + s_off[k]];
        if (!(r & REC_OCC)) wk = ex2_approx(ds32(rec_a(r) - a0, rec_b(r) - b0) * R.c32);
      }
      Wt += wk;
      cw[k] = Wt;
    }
    const float u = plan_uniform24((uint32_t)id, (uint32_t)t, R.seed_lo, R.seed_hi);
    bool certain = false;
    const int found = fp32_pick<K>(Wt, u, R.margin, [&](int k) { return cw[k]; }, certain);
    if (certain) {
      if (id < bound) out[id] = cell + s_off[found];
    } else {
      const uint32_t q = atomicAdd(&scratch[0], 1u);
      scratch[1 + q] = (uint32_t)slot;  // q < cap <= kNoAllocMaxAgents
    }
  }
}

// FP64 rule for the queued agents, one thread each (canonical order,
// sequential sums), as the context's re-check does.
__global__ void __launch_bounds__(64) k_noalloc_recheck(RepDev R, int32_t t, int32_t* out,
                                                        int32_t bound, const uint32_t* scratch) {
  const uint32_t n = scratch[0];
  const int v = R.v, reach = R.reach, W = R.W;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int slot = (int)scratch[1 + q];
    const int cell = R.cell[slot];
    const int id = R.id[slot];
    const uint32_t rec0 = R.rec[cell];
    const double S0 = s64_of(rec0);
    const unsigned long long m0 = R.mask[(size_t)cell * R.mw];
    const unsigned long long m1 = (R.mw > 1) ? R.mask[(size_t)cell * R.mw + 1] : 0ull;
    const double nks = -R.kS;
    double wk[kMaxK];
    double Wsum = 0.0;
    int k = 0;
    for (int dy = -v; dy <= v; ++dy)
      for (int dx = -v; dx <= v; ++dx) {
        if (!reach_in(dx, dy, v, reach)) continue;
        double w = 0.0;
        if (mask_bit(m0, m1, k)) {
          const bool center = (dx == 0 && dy == 0);
          const uint32_t r = center ? rec0 : R.rec[cell + dy * W + dx];
          if (center || !(r & REC_OCC)) {
            w = exp64(__dmul_rn(nks, __dsub_rn(s64_of(r), S0)));
            Wsum = __dadd_rn(Wsum, w);
          }
        }
        wk[k++] = w;
      }
    const double r = __dmul_rn(plan_uniform((uint32_t)id, (uint32_t)t, R.seed_lo, R.seed_hi), Wsum);
    double c = 0.0;
    int off_chosen = 0, off_last = 0;
    bool found = false;
    k = 0;
    for (int dy = -v; dy <= v; ++dy)
      for (int dx = -v; dx <= v; ++dx) {
        if (!reach_in(dx, dy, v, reach)) continue;
        if (wk[k] > 0.0) {
          c = __dadd_rn(c, wk[k]);
          if (!found && r < c) {
            found = true;
            off_chosen = dy * W + dx;
          }
          off_last = dy * W + dx;
        }
        ++k;
      }
    if (id < bound) out[id] = cell + (found ? off_chosen : off_last);
  }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.
static int noalloc_scratch(uint32_t** out) {
  static std::mutex mu;
  static uint32_t* ptr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return -1;
    ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = ptr[dev];
  return 0;
}

// Launches the FP32 pass for the replicate's speed; false for a speed
// outside 1..5 (nothing launched).
template <int REACH>
static bool launch_noalloc_v(const RepDev& R, int32_t cap, int32_t t, int32_t* out, int32_t bound,
                             uint32_t* sc, int grid, cudaStream_t s) {
  switch (R.v) {
    case 1: k_noalloc_plan<1, REACH><<<grid, 128, 0, s>>>(R, cap, t, out, bound, sc); return true;
    case 2: k_noalloc_plan<2, REACH><<<grid, 128, 0, s>>>(R, cap, t, out, bound, sc); return true;
    case 3: k_noalloc_plan<3, REACH><<<grid, 128, 0, s>>>(R, cap, t, out, bound, sc); return true;
    case 4: k_noalloc_plan<4, REACH><<<grid, 128, 0, s>>>(R, cap, t, out, bound, sc); return true;
    case 5: k_noalloc_plan<5, REACH><<<grid, 128, 0, s>>>(R, cap, t, out, bound, sc); return true;
  }
  return false;
}

// Returns 0, -1 (scratch address unavailable), -2 (too many agent slots) or
// -3 (an error was already pending on this thread, a launch failed, or the
// replicate's speed or reach set is unknown, so that nothing was launched).
// Launch errors are read with cudaPeekAtLastError, so that an error another
// caller left pending is not taken (and cleared) as this pass's own; an
// error of this pass's own launches is cleared after it is reported.
int noalloc_plan_launch(const RepDev& R, int32_t cap, int32_t t, int32_t* out, int32_t bound,
                        int sms, cudaStream_t s) {
  if (cap > kNoAllocMaxAgents) return -2;
  if (cudaPeekAtLastError() != cudaSuccess) return -3;
  uint32_t* sc = nullptr;
  if (noalloc_scratch(&sc) != 0) return -1;
  if (cudaMemsetAsync(sc, 0, sizeof(uint32_t), s) != cudaSuccess) return -3;
  const int grid = std::max(1, std::min((cap + 127) / 128, sms * 8));
  bool launched = false;
  if (R.reach == REACH_L2) launched = launch_noalloc_v<REACH_L2>(R, cap, t, out, bound, sc, grid, s);
  if (R.reach == REACH_L2P) launched = launch_noalloc_v<REACH_L2P>(R, cap, t, out, bound, sc, grid, s);
  if (R.reach == REACH_LINF) launched = launch_noalloc_v<REACH_LINF>(R, cap, t, out, bound, sc, grid, s);
  if (!launched) return -3;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return -3;
  }
  k_noalloc_recheck<<<std::max(1, sms * 4), 64, 0, s>>>(R, t, out, bound, sc);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return -3;
  }
  return 0;
}

int noalloc_max_agents() { return kNoAllocMaxAgents; }

}  // namespace fastgb
