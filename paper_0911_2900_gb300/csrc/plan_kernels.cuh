// plan_kernels.cuh -- planning phase of the F.A.S.T. step: every agent draws its desired
// cell from the static floor field and the occupancy at the start of the step
// (Kretz, Sec. 1: the planning phase only reads data common to all agents;
// Sec. 2: k_S = 1.2, k_other = 0).
//
//   k_plan_tile<V,REACH>    one thread per agent, per-warp record tiles
//   k_plan_direct<V,REACH>  one thread per agent, records through L1
//   k_plan_fp32<V,REACH,G>  G = 2, 4, 8 lanes per agent; FP32 weights exp(-k_S dS) on
//                           the SFU, shuffle prefix sums over the G lanes,
//                           Philox draw, margin test; draws that fall within
//                           the margin of a cumulative boundary go to a queue
//   k_recheck               one warp per queued agent, FP64 weights and the
//                           sequential canonical-order sums of the FP64 rule
//   k_plan_fp64<V,REACH>    one thread per agent, the FP64 rule for everyone
//   k_diag_compare<V,REACH> FP64 rule vs the FP32 kernel's recorded choice,
//                           flags and cumulative probabilities (diagnostics)
#pragma once
#include "fast_device.cuh"

namespace fastgb {

template <int V, int REACH>
__host__ __device__ constexpr int reach_center() {
  int k = 0;
  for (int y = -V; y <= V; ++y)
    for (int x = -V; x <= V; ++x) {
      if (x == 0 && y == 0) return k;
      k += reach_in(x, y, V, REACH) ? 1 : 0;
    }
  return -1;
}

// With speeds per agent, each speed's launch plans only its own agents.
template <int V>
__device__ __forceinline__ bool other_speed(const RepDev& R, int slot) {
  return R.speed != nullptr && R.speed[slot] != V;
}

// Line-of-sight mask words of a cell for speed V (K > 64: two words).
template <int V, int K>
__device__ __forceinline__ void mask_words(const RepDev& R, int cell, unsigned long long& m0,
                                           unsigned long long& m1) {
  constexpr int MW = K > 64 ? 2 : 1;
  const unsigned long long* mk = R.mask_v[V - 1];
  m0 = mk[(size_t)cell * MW];
  m1 = (K > 64) ? mk[(size_t)cell * MW + 1] : 0ull;
}

// Canonical offsets of one reach set, as cell-index deltas for row length W.
__device__ __forceinline__ void fill_offsets(int* s_off, int v, int reach, int W) {
  if (threadIdx.x == 0) {
    int k = 0;
    for (int y = -v; y <= v; ++y)
      for (int x = -v; x <= v; ++x)
        if (reach_in(x, y, v, reach)) s_off[k++] = y * W + x;
  }
}

// k-th canonical offset of a reach set (runtime v), as (dx, dy).
__device__ __forceinline__ void kth_offset(int v, int reach, int k, int* dx, int* dy) {
  for (int y = -v; y <= v; ++y) {
    int row = 0;
    for (int x = -v; x <= v; ++x) row += reach_in(x, y, v, reach) ? 1 : 0;
    if (k < row) {
      for (int x = -v; x <= v; ++x)
        if (reach_in(x, y, v, reach)) {
          if (k == 0) {
            *dx = x;
            *dy = y;
            return;
          }
          --k;
        }
    }
    k -= row;
  }
  *dx = 0;
  *dy = 0;
}

__device__ __forceinline__ bool mask_bit(unsigned long long m0, unsigned long long m1, int k) {
  return k < 64 ? ((m0 >> k) & 1ull) : ((m1 >> (k - 64)) & 1ull);
}

__device__ __forceinline__ void set_static(uint32_t* rec, int cell, uint32_t rec0, bool stays) {
  rec[cell] = stays ? (rec0 | REC_STA) : (rec0 & ~REC_STA);
}

// The same as an atomic bit update (no dependence on an earlier read).
__device__ __forceinline__ void set_static_red(uint32_t* rec, int cell, bool stays) {
  if (stays)
    atomicOr(&rec[cell], REC_STA);
  else
    atomicAnd(&rec[cell], ~REC_STA);
}

// Offsets of a reach set packed as (dx + 16) | (dy + 16) << 8, canonical order.
template <int V, int REACH>
__device__ __forceinline__ void fill_dxdy(int* s_dxdy) {
  constexpr ReachTable<V, REACH> T{};
  constexpr int K = reach_count(V, REACH);
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    s_dxdy[k] = (T.dx[k] + 16) | ((T.dy[k] + 16) << 8);
}

// FP32 weight of a candidate record seen from (a0, b0): 0 if blocked.
__device__ __forceinline__ float rec_weight(uint32_t r, float a0m, float b0m, float c32) {
  return (r & REC_OCC) ? 0.f : ex2_approx(ds32_rec(r, a0m, b0m) * c32);
}

// The FP32 draw of one agent: r = u*W against the cumulative weights
// C_k = w(0) + ... + w(k), summed in canonical order (C(k) returns them; W is
// the last).  The choice is the first k with r < C_k.  C never decreases (a
// zero weight leaves it unchanged and so is never first), so that k is the
// number of C_k <= r; K of them means none, only through rounding, which the
// FP64 rule then settles.  Returns k (-1: none) and sets `certain` when r
// lies farther than margin*W from both boundaries C_{k-1} (0 for k = 0) and
// C_k of that k: only then is the FP32 choice sure to be the FP64 rule's (the
// margin bounds the FP32 weights' and sums' error).
template <int K, typename CF>
__device__ __forceinline__ int fp32_pick(float Wt, float u, float margin, CF C, bool& certain) {
  const float r = __fmul_rn(u, Wt);
  int below = 0;
  float lo = 0.f, hi = __int_as_float(0x7F800000);  // the boundaries around r
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float ck = C(k);
    const bool le = ck <= r;
    below += le ? 1 : 0;
    lo = le ? ck : lo;
    hi = le ? hi : fminf(hi, ck);
  }
  const int found = below < K ? below : -1;
  const float mw = margin * Wt;
  certain = (found >= 0) && (r > lo + mw) && (r < hi - mw);
  return found;
}

// Shared end of the one-thread kernels: the draw and margin test
// (fp32_pick), and the outputs.
template <int K, int CENTER, bool DIAG, typename CF>
__device__ __forceinline__ void finish_g1(const StepArgs& a, const RepDev& R, int rep, int slot,
                                          int cell, float Wt, float u, float margin,
                                          int norecheck, const int* s_dxdy, CF C) {
  bool ok = false;
  const int found = fp32_pick<K>(Wt, u, margin, C, ok);
  if (DIAG) {
    float* dp = a.diag_p32 + (a.diag_base[rep] + slot) * (int64_t)kMaxK;
#pragma unroll
    for (int k = 0; k < K; ++k) dp[k] = C(k) / Wt;
  }
  const int dd = s_dxdy[found >= 0 ? found : CENTER];
  const int target = cell + ((dd >> 8) - 16) * R.W + ((dd & 0xFF) - 16);
  if (DIAG) {
    const int64_t di = a.diag_base[rep] + slot;
    a.diag_choice32[di] = target;
    a.diag_flag[di] = ok ? 0 : 1;
  }
  if (ok || norecheck) {
    R.desired[slot] = target;
    set_static_red(R.rec, cell, target == cell);
  } else {
    const uint32_t qi = append_slot(&a.ctl->q_count);
    if (qi < a.q_cap) a.queue[qi] = ((uint32_t)rep << 24) | (uint32_t)slot;
  }
}

// ---------------------------------------------------------------------------
// FP32 planning, G lanes per agent.  Lane `sub` of a group owns the
// candidates [sub*Q, sub*Q + Q) of the canonical order.  Every cumulative
// value the decision uses is a sum of at most K positive FP32 weights, so its
// relative error is bounded by gamma = (1+delta)(1+2^-24)^K - 1 (delta: one
// weight's error); the host folds this into the margin M.  A draw r = u*W
// is accepted only if C_prev + M*W < r < C_k - M*W; otherwise the agent is
// re-evaluated with the FP64 rule.
template <int V, int REACH, int G, bool DIAG>
__global__ void __launch_bounds__(256) k_plan_fp32(StepArgs a, Chunks ch, int norecheck) {
  constexpr int K = reach_count(V, REACH);
  constexpr int Q = (K + G - 1) / G;
  constexpr int CENTER = reach_center<V, REACH>();
  constexpr int PER_PASS = 256 / G;
  __shared__ int s_off[K];

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int sub = lane & (G - 1);
  const int grp = tid / G;
  const unsigned gmask =
      (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int t = a.ctl->t;
  int cur_rep = -1;

  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const int begin = ch.begin[c];
    if (rep != cur_rep) {
      __syncthreads();
      fill_offsets(s_off, V, REACH, a.reps[rep].W);
      __syncthreads();
      cur_rep = rep;
    }
    const RepDev& R = a.reps[rep];
    uint32_t* rec = R.rec;
    const int end = min(begin + kChunk, a.n_slots[rep]);
    const float c32 = R.c32;
    for (int pass = 0; pass < G; ++pass) {
      const int slot = begin + pass * PER_PASS + grp;
      if (slot >= end) continue;
      const int cell = R.cell[slot];
      if (cell < 0 || other_speed<V>(R, slot)) continue;
      const long long C = (long long)R.W * R.H;
      if (!fg_in(a.ctl, cell, C)) continue;
      const int id = R.id[slot];
      const uint32_t rec0 = rec[cell];
      unsigned long long m0, m1;
      mask_words<V, K>(R, cell, m0, m1);
      // all candidate records first (independent loads in flight together),
      // then the weights; an inadmissible candidate reads as blocked
      uint32_t rr[Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int k = sub * Q + j;
        const bool adm = (k < K) && (k != CENTER) && mask_bit(m0, m1, k) &&
                         (!kChecked || fg_in(a.ctl, (long long)cell + s_off[k], C));
        rr[j] = adm ? rec[cell + s_off[k]] : REC_OCC;
      }
      const float a0m = field_m(rec_a(rec0)), b0m = field_m(rec_b(rec0));
      float w[Q];
      float lsum = 0.f;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int k = sub * Q + j;
        float wk = 0.f;
        if (k == CENTER) {
          wk = 1.0f;
        } else if (!(rr[j] & REC_OCC)) {
          wk = ex2_approx(ds32_rec(rr[j], a0m, b0m) * c32);
        }
        w[j] = wk;
        lsum += wk;
      }
      // inclusive / exclusive scan of the lane sums inside the group
      float incl = lsum;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const float tv = __shfl_up_sync(gmask, incl, o, G);
        if (sub >= o) incl += tv;
      }
      float excl = __shfl_up_sync(gmask, incl, 1, G);
      if (sub == 0) excl = 0.f;
      const float Wt = __shfl_sync(gmask, incl, G - 1, G);
      float uf = 0.f;
      if (sub == 0) uf = plan_uniform24((uint32_t)id, (uint32_t)t, R.seed_lo, R.seed_hi);
      uf = __shfl_sync(gmask, uf, 0, G);
      const float r = __fmul_rn(uf, Wt);

      // walk the lane's candidates: first k with r < C_k
      float cacc = excl, cprev = 0.f, ck = 0.f, clast_prev = excl;
      int found = -1, lastnz = -1;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        if (w[j] > 0.f) {
          const float cn = cacc + w[j];
          if (found < 0 && r < cn) {
            found = sub * Q + j;
            cprev = cacc;
            ck = cn;
          }
          clast_prev = cacc;
          lastnz = sub * Q + j;
          cacc = cn;
        }
      }
      if (DIAG) {
        float* dp = a.diag_p32 + (a.diag_base[rep] + slot) * (int64_t)kMaxK;
        float cc = excl;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const int k = sub * Q + j;
          cc = (w[j] > 0.f) ? cc + w[j] : cc;
          if (k < K) dp[k] = cc / Wt;
        }
      }
      const unsigned fb = __ballot_sync(gmask, found >= 0) & gmask;
      int owner;
      bool any = fb != 0u;
      if (any) {
        owner = __ffs(fb) - 1;
      } else {
        const unsigned nb = __ballot_sync(gmask, lastnz >= 0) & gmask;
        owner = 31 - __clz(nb);
      }
      if (lane == owner) {
        int kk;
        bool ok;
        if (any) {
          kk = found;
          const float mw = R.margin_v[V - 1] * Wt;
          ok = (r > cprev + mw) && (r < ck - mw);
        } else {
          kk = lastnz;
          ok = false;
          (void)clast_prev;
        }
        const int target = cell + s_off[kk];
        if (DIAG) {
          const int64_t di = a.diag_base[rep] + slot;
          a.diag_choice32[di] = target;
          a.diag_flag[di] = ok ? 0 : 1;
        }
        if (ok || norecheck) {
          R.desired[slot] = target;
          set_static(rec, cell, rec0, target == cell);
        } else {
          const uint32_t qi = append_slot(&a.ctl->q_count);
          if (qi < a.q_cap) a.queue[qi] = ((uint32_t)rep << 24) | (uint32_t)slot;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 planning, one thread per agent, records from a per-warp tile.
// Each warp copies into shared memory the box of cell records that covers
// the reach sets of its 32 agents (coalesced row loads), then every thread
// evaluates its agent's candidates at compile-time offsets into the tile.  A
// warp whose agents are spread wider than the tile reads the records from
// global memory instead.  Same weights, margin and outputs as k_plan_fp32.
constexpr int kTileW = 48, kTileH = 48, kTileP = 49;   // per-warp record tile
constexpr int kTileWarps = 8;
constexpr size_t kTileSmem = (size_t)kTileWarps * kTileH * kTileP * 4;

template <int V, int REACH, bool DIAG, bool TILE>
__device__ __forceinline__ void plan_one_g1(const StepArgs& a, const RepDev& R, int rep, int slot,
                                            int cell, const uint32_t* p0, int pitch, int t,
                                            int norecheck, const int* s_dxdy) {
  constexpr int K = reach_count(V, REACH);
  constexpr int CENTER = reach_center<V, REACH>();
  constexpr ReachTable<V, REACH> T{};
  const int id = R.id[slot];
  const uint32_t rec0 = p0[0];
  unsigned long long m0, m1;
  mask_words<V, K>(R, cell, m0, m1);
  uint32_t rr[K];
  // a warp whose agents see every candidate (no wall in sight, inside the
  // grid) skips the per-candidate mask tests
  constexpr unsigned long long kFull0 = K >= 64 ? ~0ull : ((1ull << K) - 1ull);
  constexpr unsigned long long kFull1 = K > 64 ? ((1ull << (K - 64)) - 1ull) : 0ull;
  // (debug build: every candidate's cell index checked against the grid)
  const long long C = (long long)R.W * R.H;
  if (__all_sync(__activemask(), m0 == kFull0 && m1 == kFull1)) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int off = TILE ? (T.dy[k] * kTileP + T.dx[k]) : (T.dy[k] * pitch + T.dx[k]);
      const bool adm = (k != CENTER) &&
                       (!kChecked || fg_in(a.ctl, (long long)cell + T.dy[k] * R.W + T.dx[k], C));
      rr[k] = adm ? p0[off] : REC_OCC;
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int off = TILE ? (T.dy[k] * kTileP + T.dx[k]) : (T.dy[k] * pitch + T.dx[k]);
      const bool adm = (k != CENTER) && mask_bit(m0, m1, k) &&
                       (!kChecked || fg_in(a.ctl, (long long)cell + T.dy[k] * R.W + T.dx[k], C));
      rr[k] = adm ? p0[off] : REC_OCC;
    }
  }
  const float a0m = field_m(rec_a(rec0)), b0m = field_m(rec_b(rec0));
  const float c32 = R.c32;
  float cw[K];  // cumulative weights C_k
  float Wt = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float wk = (k == CENTER) ? 1.0f : rec_weight(rr[k], a0m, b0m, c32);
    Wt += wk;
    cw[k] = Wt;
  }
  const float u = plan_uniform24((uint32_t)id, (uint32_t)t, R.seed_lo, R.seed_hi);
  finish_g1<K, CENTER, DIAG>(a, R, rep, slot, cell, Wt, u, R.margin_v[V - 1], norecheck, s_dxdy,
                             [&](int k) { return cw[k]; });
}

// ---------------------------------------------------------------------------
// FP32 planning, one thread per agent (the 1-lane variant), candidate records
// read through L1 at compile-time offsets from row pointers; same weights,
// margin and outputs as the other variants.
template <int V, int REACH, bool DIAG>
__global__ void __launch_bounds__(256) k_plan_direct(StepArgs a, Chunks ch, int norecheck) {
  __shared__ int s_dxdy[reach_count(V, REACH)];
  fill_dxdy<V, REACH>(s_dxdy);
  __syncthreads();
  const int t = a.ctl->t;
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const RepDev& R = a.reps[rep];
    const int end = min(ch.begin[c] + kChunk, a.n_slots[rep]);
    const int slot = ch.begin[c] + threadIdx.x;
    if (slot >= end) continue;
    const int cell = R.cell[slot];
    if (cell < 0 || other_speed<V>(R, slot)) continue;
    if (!fg_in(a.ctl, cell, (long long)R.W * R.H)) continue;
    plan_one_g1<V, REACH, DIAG, false>(a, R, rep, slot, cell, R.rec + cell, R.W, t, norecheck,
                                       s_dxdy);
  }
}

template <int V, int REACH, bool DIAG>
__global__ void __launch_bounds__(256, 2) k_plan_tile(StepArgs a, Chunks ch, int norecheck) {
  extern __shared__ __align__(16) uint32_t s_tiles[];
  __shared__ int s_dxdy[reach_count(V, REACH)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* tile = s_tiles + warp * (kTileH * kTileP);
  const int t = a.ctl->t;
  fill_dxdy<V, REACH>(s_dxdy);
  __syncthreads();
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const RepDev& R = a.reps[rep];
    const int end = min(ch.begin[c] + kChunk, a.n_slots[rep]);
    const int slot = ch.begin[c] + threadIdx.x;
    int cell = (slot < end && !other_speed<V>(R, slot)) ? R.cell[slot] : -1;
    if (cell >= 0 && !fg_in(a.ctl, cell, (long long)R.W * R.H)) cell = -1;
    const bool live = cell >= 0;
    const int W = R.W;
    int x = 0, y = 0;
    if (live) {
      y = cell / W;
      x = cell - y * W;
    }
    const unsigned any = __ballot_sync(0xffffffffu, live);
    if (!any) continue;
    const int xmin = (int)__reduce_min_sync(0xffffffffu, live ? (unsigned)x : 0xFFFFFFFFu);
    const int ymin = (int)__reduce_min_sync(0xffffffffu, live ? (unsigned)y : 0xFFFFFFFFu);
    const int xmax = (int)__reduce_max_sync(0xffffffffu, live ? (unsigned)x : 0u);
    const int ymax = (int)__reduce_max_sync(0xffffffffu, live ? (unsigned)y : 0u);
    const int bx0 = max(xmin - V, 0), by0 = max(ymin - V, 0);
    const int bx1 = min(xmax + V, W - 1), by1 = min(ymax + V, R.H - 1);
    const int bw = bx1 - bx0 + 1, bh = by1 - by0 + 1;
    const bool use_tile = bw <= kTileW && bh <= kTileH;
    if (use_tile) {
      // rows in batches of 8: all loads of a batch in flight before the stores
      const bool c1 = lane + 32 < bw;
      for (int row0 = 0; row0 < bh; row0 += 8) {
        uint32_t v0[8], v1[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int row = row0 + j;
          const uint32_t* src = R.rec + (size_t)(by0 + min(row, bh - 1)) * W + bx0;
          v0[j] = (row < bh && lane < bw) ? src[lane] : 0u;
          v1[j] = (row < bh && c1) ? src[lane + 32] : 0u;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int row = row0 + j;
          if (row < bh) {
            if (lane < bw) tile[row * kTileP + lane] = v0[j];
            if (c1) tile[row * kTileP + lane + 32] = v1[j];
          }
        }
      }
      __syncwarp();
      if (live)
        plan_one_g1<V, REACH, DIAG, true>(a, R, rep, slot, cell,
                                          tile + (y - by0) * kTileP + (x - bx0), kTileP, t,
                                          norecheck, s_dxdy);
    } else {
      if (lane == 0) atomicAdd(&a.ctl->tile_fallbacks, 1ull);
      if (live)
        plan_one_g1<V, REACH, DIAG, false>(a, R, rep, slot, cell, R.rec + cell, W, t, norecheck,
                                           s_dxdy);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// FP64 rule for one agent (thread-serial): weights in canonical order,
// W and C_k summed sequentially, smallest k with fl(u*W) < C_k.
template <int V, int REACH>
__device__ __forceinline__ int plan_fp64_one(const RepDev& R, const int* s_off, int cell, int id,
                                             int t, double* cum_out) {
  constexpr int K = reach_count(V, REACH);
  constexpr int CENTER = reach_center<V, REACH>();
  const uint32_t* rec = R.rec;
  const uint32_t rec0 = rec[cell];
  const double S0 = s64_of(rec0);
  unsigned long long m0, m1;
  mask_words<V, K>(R, cell, m0, m1);
  const double nks = -R.kS;
  double wk[K];
  double W = 0.0;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    double w = 0.0;
    if (mask_bit(m0, m1, k)) {
      const uint32_t r = (k == CENTER) ? rec0 : rec[cell + s_off[k]];
      if (k == CENTER || !(r & REC_OCC)) {
        const double d = __dsub_rn(s64_of(r), S0);
        w = exp64(__dmul_rn(nks, d));
        W = __dadd_rn(W, w);
      }
    }
    wk[k] = w;
  }
  const double u = plan_uniform((uint32_t)id, (uint32_t)t, R.seed_lo, R.seed_hi);
  const double r = __dmul_rn(u, W);
  double c = 0.0;
  int chosen = -1, last = -1;
  for (int k = 0; k < K; ++k) {
    if (wk[k] > 0.0) {
      c = __dadd_rn(c, wk[k]);
      if (chosen < 0 && r < c) chosen = k;
      last = k;
    }
    if (cum_out) cum_out[k] = c / W;
  }
  if (chosen < 0) chosen = last;
  return cell + s_off[chosen];
}

template <int V, int REACH>
__global__ void __launch_bounds__(128) k_plan_fp64(StepArgs a, Chunks ch) {
  constexpr int K = reach_count(V, REACH);
  __shared__ int s_off[K];
  const int t = a.ctl->t;
  int cur_rep = -1;
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const int begin = ch.begin[c];
    if (rep != cur_rep) {
      __syncthreads();
      fill_offsets(s_off, V, REACH, a.reps[rep].W);
      __syncthreads();
      cur_rep = rep;
    }
    const RepDev& R = a.reps[rep];
    const int end = min(begin + kChunk, a.n_slots[rep]);
    for (int slot = begin + threadIdx.x; slot < end; slot += blockDim.x) {
      const int cell = R.cell[slot];
      if (cell < 0 || other_speed<V>(R, slot)) continue;
      if (!fg_in(a.ctl, cell, (long long)R.W * R.H)) continue;
      const uint32_t rec0 = R.rec[cell];
      const int target = plan_fp64_one<V, REACH>(R, s_off, cell, R.id[slot], t, nullptr);
      R.desired[slot] = target;
      set_static(R.rec, cell, rec0, target == cell);
    }
  }
}

// ---------------------------------------------------------------------------
// Diagnostics: FP64 rule for every agent against the FP32 kernel's recorded
// choice (no re-check), flag and cumulative probabilities.
template <int V, int REACH>
__global__ void __launch_bounds__(128) k_diag_compare(StepArgs a, Chunks ch) {
  constexpr int K = reach_count(V, REACH);
  __shared__ int s_off[K];
  const int t = a.ctl->t;
  int cur_rep = -1;
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const int begin = ch.begin[c];
    if (rep != cur_rep) {
      __syncthreads();
      fill_offsets(s_off, V, REACH, a.reps[rep].W);
      __syncthreads();
      cur_rep = rep;
    }
    const RepDev& R = a.reps[rep];
    const int end = min(begin + kChunk, a.n_slots[rep]);
    for (int slot = begin + threadIdx.x; slot < end; slot += blockDim.x) {
      const int cell = R.cell[slot];
      if (cell < 0 || other_speed<V>(R, slot)) continue;
      if (!fg_in(a.ctl, cell, (long long)R.W * R.H)) continue;
      double cum[K];
      const int target = plan_fp64_one<V, REACH>(R, s_off, cell, R.id[slot], t, cum);
      const int64_t di = a.diag_base[rep] + slot;
      const int t32 = a.diag_choice32[di];
      const bool flagged = a.diag_flag[di] != 0;
      if (flagged) atomicAdd(&a.ctl->flagged, 1ull);
      if (t32 != target) {
        atomicAdd(&a.ctl->flips, 1ull);
        if (!flagged) atomicAdd(&a.ctl->flips_unflagged, 1ull);
      }
      // the real planning pass (FP32 weights, FP64 re-check inside the
      // margin) that ran before the diagnostic one left its choice here
      if (R.desired[slot] != target) atomicAdd(&a.ctl->flips_after, 1u);
      const float* dp = a.diag_p32 + di * (int64_t)kMaxK;
      float mx = 0.f;
      for (int k = 0; k < K; ++k) mx = fmaxf(mx, (float)fabs((double)dp[k] - cum[k]));
      atomicMax(&a.ctl->max_dp_bits, __float_as_uint(mx));
    }
  }
}

// ---------------------------------------------------------------------------
template <int V, int REACH, bool DIAG>
static int launch_tile(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s,
                       int norecheck) {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_plan_tile<V, REACH, DIAG>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTileSmem) != cudaSuccess)
      return -1;
    attr_set = true;
  }
  k_plan_tile<V, REACH, DIAG><<<grid, 256, kTileSmem, s>>>(a, ch, norecheck);
  return 0;
}

template <int V, int REACH>
static int launch_fp32(const StepArgs& a, int lanes, const Chunks& ch, int grid, cudaStream_t s,
                       bool diag, int norecheck) {
  if (lanes == 0)
    return diag ? launch_tile<V, REACH, true>(a, ch, grid, s, norecheck)
                : launch_tile<V, REACH, false>(a, ch, grid, s, norecheck);
#define FAST_L(G)                                                                  \
  if (lanes == G) {                                                                \
    if (diag)                                                                      \
      k_plan_fp32<V, REACH, G, true><<<grid, 256, 0, s>>>(a, ch, norecheck);       \
    else                                                                           \
      k_plan_fp32<V, REACH, G, false><<<grid, 256, 0, s>>>(a, ch, norecheck);      \
    return 0;                                                                      \
  }
  if (lanes == 1) {
    if (diag)
      k_plan_direct<V, REACH, true><<<grid, 256, 0, s>>>(a, ch, norecheck);
    else
      k_plan_direct<V, REACH, false><<<grid, 256, 0, s>>>(a, ch, norecheck);
    return 0;
  }
  FAST_L(2)
  FAST_L(4)
  FAST_L(8)
#undef FAST_L
  return -1;
}

template <int V, int REACH>
static int launch_v(const StepArgs& a, int lanes, int precision, const Chunks& ch, int grid,
                    cudaStream_t s, bool diag) {
  if (precision == PREC_FP64) {
    k_plan_fp64<V, REACH><<<grid, 128, 0, s>>>(a, ch);
    return 0;
  }
  return launch_fp32<V, REACH>(a, lanes, ch, grid, s, diag,
                               (precision == PREC_FP32_NORECHECK || diag) ? 1 : 0);
}

// All reach variants of one v_m (one translation unit per v_m).
template <int V>
static int launch_one_v(const StepArgs& a, int reach, int lanes, int precision, const Chunks& ch,
                        int grid, cudaStream_t s, bool diag) {
  if (reach == REACH_L2) return launch_v<V, REACH_L2>(a, lanes, precision, ch, grid, s, diag);
  if (reach == REACH_L2P) return launch_v<V, REACH_L2P>(a, lanes, precision, ch, grid, s, diag);
  if (reach == REACH_LINF) return launch_v<V, REACH_LINF>(a, lanes, precision, ch, grid, s, diag);
  return -1;
}

template <int V>
static int diag_one_v(const StepArgs& a, int reach, const Chunks& ch, int grid, cudaStream_t s) {
  if (reach == REACH_L2) {
    k_diag_compare<V, REACH_L2><<<grid, 128, 0, s>>>(a, ch);
    return 0;
  }
  if (reach == REACH_L2P) {
    k_diag_compare<V, REACH_L2P><<<grid, 128, 0, s>>>(a, ch);
    return 0;
  }
  if (reach == REACH_LINF) {
    k_diag_compare<V, REACH_LINF><<<grid, 128, 0, s>>>(a, ch);
    return 0;
  }
  return -1;
}

}  // namespace fastgb
