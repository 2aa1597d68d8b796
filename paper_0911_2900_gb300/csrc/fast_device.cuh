// fast_device.cuh -- device-side building blocks of the F.A.S.T. step on sm_103a.
//
// Cell record (one uint32 per cell, row-major, the only per-cell state the
// planning and movement kernels touch):
//   bits  0..14  a  : orthogonal steps of the shortest path to an exit
//   bits 15..29  b  : diagonal steps     (floor field S = a + b*sqrt(2))
//   bit  30      OCC: cell blocked (agent on it, wall, or unreachable cell)
//   bit  31      STA: the agent on it does not move this step
// a = b = 0x7FFF marks walls and cells no exit can be reached from.  Exit
// cells are the only cells with a = b = 0 and are never occupied.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "fast_internal.h"

namespace fastgb {

constexpr uint32_t REC_AB = 0x3FFFFFFFu;
constexpr uint32_t REC_OCC = 0x40000000u;
constexpr uint32_t REC_STA = 0x80000000u;
constexpr uint32_t REC_SENT = 0x7FFFu;

__device__ __forceinline__ int rec_a(uint32_t r) { return (int)(r & 0x7FFFu); }
__device__ __forceinline__ int rec_b(uint32_t r) { return (int)((r >> 15) & 0x7FFFu); }
__device__ __forceinline__ bool rec_exit(uint32_t r) { return (r & REC_AB) == 0u; }
__device__ __forceinline__ bool rec_sentinel(uint32_t r) {
  return (r & 0x7FFFu) == REC_SENT;
}

// --------------------------------------------------------------------------
// Debug build (compiled with FASTGB_CHECKED): the indices the step kernels
// derive from data -- an agent's cell and desired cell, candidate and path
// cells, mover and re-check queue entries -- are checked against the array
// they index before use.  One out of range records kDevErrBounds and the
// index in the control block, and the access is skipped (the agent is left
// where it is); nothing traps.  The release build compiles the checks away.
#ifdef FASTGB_CHECKED
constexpr bool kChecked = true;
static __device__ __noinline__ bool fg_bad_index(Ctl* ctl, long long i) {
  if (atomicCAS(&ctl->err, 0, kDevErrBounds) == 0) ctl->bad_index = i;
  return false;
}
__device__ __forceinline__ bool fg_in(Ctl* ctl, long long i, long long n) {
  return (i >= 0 && i < n) ? true : fg_bad_index(ctl, i);
}
#else
constexpr bool kChecked = false;
__device__ __forceinline__ bool fg_in(Ctl*, long long, long long) { return true; }
#endif

// --------------------------------------------------------------------------
// Reach sets (movement reach of one step): offsets (dx,dy) with
// dx^2+dy^2 <= v^2 (L2), <= v^2+v (L2P) or max(|dx|,|dy|) <= v (LINF), listed
// row by row (dy ascending, then dx ascending).
__host__ __device__ constexpr bool reach_in(int dx, int dy, int v, int reach) {
  return reach == REACH_L2    ? (dx * dx + dy * dy <= v * v)
         : reach == REACH_L2P ? (dx * dx + dy * dy <= v * v + v)
                              : ((dx < 0 ? -dx : dx) <= v && (dy < 0 ? -dy : dy) <= v);
}

__host__ __device__ constexpr int reach_count(int v, int reach) {
  int k = 0;
  for (int y = -v; y <= v; ++y)
    for (int x = -v; x <= v; ++x) k += reach_in(x, y, v, reach) ? 1 : 0;
  return k;
}

template <int V, int REACH>
struct ReachTable {
  static constexpr int K = reach_count(V, REACH);
  int8_t dx[K > 0 ? K : 1];
  int8_t dy[K > 0 ? K : 1];
  int center;
  __host__ __device__ constexpr ReachTable() : dx(), dy(), center(0) {
    int k = 0;
    for (int y = -V; y <= V; ++y)
      for (int x = -V; x <= V; ++x)
        if (reach_in(x, y, V, REACH)) {
          if (x == 0 && y == 0) center = k;
          dx[k] = (int8_t)x;
          dy[k] = (int8_t)y;
          ++k;
        }
  }
};

// Straight path: L = max(|dx|,|dy|) Moore moves, step s at
// (q(s*dx, L), q(s*dy, L)) with q = division rounded half away from zero.
__host__ __device__ __forceinline__ int div_half_away(int num, int L) {
  return num >= 0 ? (2 * num + L) / (2 * L) : -((-2 * num + L) / (2 * L));
}

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// 53-bit uniform in [0,1) from the first two words of the planning stream
// (counter (id, t, 0, 0)).
__device__ __forceinline__ double plan_uniform(uint32_t id, uint32_t t, uint32_t k0, uint32_t k1) {
  const U4 r = philox10(id, t, 0u, 0u, k0, k1);
  const double hi = (double)(r.x >> 5), lo = (double)(r.y >> 6);
  return __dmul_rn(__dadd_rn(__dmul_rn(hi, 67108864.0), lo), 0x1p-53);
}

// The same draw truncated to its top 24 bits, as a float (exact), for the
// FP32 kernels: 0 <= u - u24 < 2^-24, which the FP32 margin covers; no FP64
// instruction is involved.
__device__ __forceinline__ float plan_uniform24(uint32_t id, uint32_t t, uint32_t k0, uint32_t k1) {
  const U4 r = philox10(id, t, 0u, 0u, k0, k1);
  return __uint2float_rz(r.x >> 8) * 0x1p-24f;
}

// Movement order of step t: a keyed permutation of the 24-bit agent ids.
// The step keys are the four words of Philox(seed; (0, t, 2, 0)); the id's
// 12-bit halves (L, R) pass through four Feistel rounds
// (L, R) <- (R, L ^ (fmix32(R ^ k_i) & 0xFFF)), fmix32 being MurmurHash3's
// finalizer.  Each round is invertible, so no two agents of a replicate share
// a priority.  Smaller priorities move earlier.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ U4 move_step_keys(uint32_t t, uint32_t s0, uint32_t s1) {
  return philox10(0u, t, 2u, 0u, s0, s1);
}

__device__ __forceinline__ uint32_t move_priority(uint32_t id, const U4& k) {
  uint32_t L = (id >> 12) & 0xFFFu, R = id & 0xFFFu;
  const uint32_t ks[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t nr = L ^ (fmix32(R ^ ks[i]) & 0xFFFu);
    L = R;
    R = nr;
  }
  return (L << 12) | R;
}

// --------------------------------------------------------------------------
// FP64 exponential (Cody-Waite reduction by ln 2 split in two parts, then a
// degree-13 Taylor polynomial in Horner form with one fused multiply-add per
// step, then scaling by 2^n through the exponent field).  Every operation is
// an explicitly rounded intrinsic, so the result is fixed bit for bit.
//   n  = rint(x * log2e)
//   r  = fma(-n, LN2_HI, x);  r = fma(-n, LN2_LO, r)
//   p  = 1 + r(1 + r(1/2 + r(1/6 + ... + r/13!)))
// LN2_HI = ln 2 cut to 32 significant bits (2977044471 / 2^32), LN2_LO the
// double nearest ln 2 - LN2_HI; coefficients are the doubles nearest 1/k!.
__device__ __forceinline__ double exp64(double x) {
  const double n = rint(__dmul_rn(x, 0x1.71547652b82fep+0));
  double r = __fma_rn(-n, 0x1.62e42feep-1, x);
  r = __fma_rn(-n, 0x1.a39ef35793c76p-33, r);
  double p = 1.0 / 6227020800.0;
  p = __fma_rn(p, r, 1.0 / 479001600.0);
  p = __fma_rn(p, r, 1.0 / 39916800.0);
  p = __fma_rn(p, r, 1.0 / 3628800.0);
  p = __fma_rn(p, r, 1.0 / 362880.0);
  p = __fma_rn(p, r, 1.0 / 40320.0);
  p = __fma_rn(p, r, 1.0 / 5040.0);
  p = __fma_rn(p, r, 1.0 / 720.0);
  p = __fma_rn(p, r, 1.0 / 120.0);
  p = __fma_rn(p, r, 1.0 / 24.0);
  p = __fma_rn(p, r, 1.0 / 6.0);
  p = __fma_rn(p, r, 0.5);
  p = __fma_rn(p, r, 1.0);
  p = __fma_rn(p, r, 1.0);
  const long long e = (long long)n + 1023;
  return __dmul_rn(p, __longlong_as_double(e << 52));
}

// S as the oracle rounds it: fl(a + fl(b * sqrt2)).
__device__ __forceinline__ double s64_of(uint32_t r) {
  return __dadd_rn((double)rec_a(r), __dmul_rn((double)rec_b(r), 0x1.6a09e667f3bcdp+0));
}

// 2^y on the SFU (MUFU.EX2).
__device__ __forceinline__ float ex2_approx(float y) {
  float o;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(o) : "f"(y));
  return o;
}

// S(c) - S(c0) in FP32 from the exact integer differences:
// da + db*sqrt2 with sqrt2 split in two floats, two roundings.
__device__ __forceinline__ float ds32(int da, int db) {
  const float fb = (float)db;
  const float t1 = __fmaf_rn(fb, 0x1.6a09e6p+0f, (float)da);
  return __fmaf_rn(fb, 0x1.9fcef4p-26f, t1);
}


// The same from a raw record: the 15-bit fields become exact floats through
// the 2^23 exponent (0x4B000000 | v is the float 2^23 + v), so that the
// differences a - a0 and b - b0 are float subtractions of exact integers;
// a0m = 2^23 + a0 and b0m = 2^23 + b0 are the agent's own fields likewise.
// Identical values to ds32(a - a0, b - b0).
__device__ __forceinline__ float ds32_rec(uint32_t r, float a0m, float b0m) {
  const float fa = __fsub_rn(__uint_as_float((r & 0x7FFFu) | 0x4B000000u), a0m);
  const float fb = __fsub_rn(__uint_as_float(((r >> 15) & 0x7FFFu) | 0x4B000000u), b0m);
  const float t1 = __fmaf_rn(fb, 0x1.6a09e6p+0f, fa);
  return __fmaf_rn(fb, 0x1.9fcef4p-26f, t1);
}

// 2^23 + v as a float (exact for 0 <= v < 2^23).
__device__ __forceinline__ float field_m(int v) {
  return __uint_as_float(0x4B000000u | (uint32_t)v);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
  return __ldcg(p);
}

// Fire-and-forget reductions on global memory (relaxed, device scope, no
// value returned), for pointers that point into device global memory.  A
// plain atomicMin/And/Or/Add through a generic pointer returns the old value
// to the thread whether or not it is used.
__device__ __forceinline__ void red_min_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v)
               : "memory");
}
__device__ __forceinline__ void red_and_b32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.and.b32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v)
               : "memory");
}
__device__ __forceinline__ void red_or_b32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v)
               : "memory");
}
__device__ __forceinline__ void red_add_s32(int32_t* p, int32_t v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(v)
               : "memory");
}

// Appends to a global list with one atomic per group of converged lanes:
// returns this lane's slot (called only by the lanes that append).
__device__ __forceinline__ uint32_t append_slot(uint32_t* counter) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  uint32_t base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, (uint32_t)g.size());
  return g.shfl(base, 0) + (uint32_t)g.thread_rank();
}

}  // namespace fastgb
