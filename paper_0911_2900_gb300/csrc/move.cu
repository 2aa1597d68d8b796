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
//   commute; so moving, in each round, every waiting agent whose footprint
//   holds no claim of a lower-priority waiting agent keeps every conflicting
//   pair in priority order, which is equivalent to the serial loop.
//   Claims are 32-bit atomicMin of (8-bit round tag, 24-bit priority) on
//   every footprint cell, in two arrays used in turn.  The tag falls with a
//   round counter that runs on across steps, so a fresh claim beats every
//   stale one; the arrays are cleared only when the tags run out (every few
//   steps).  In a round with tag g every waiting agent checks its claims in
//   array g&1 and either moves or claims again, with tag g+1, in the other
//   array.  One grid barrier per round.  The lowest-priority
//   waiting agent always moves, so the loop ends after at most (number of
//   movers) rounds; in practice after the longest local priority chain.
//   An agent that moves in the first round moves exactly as the records read
//   by the movement-order pass say (nobody touched its footprint before it),
//   so it only flips occupancy bits.  Waiting agents are kept per block in
//   shared memory when they fit; once few are left, one block takes them all
//   and finishes the step with block-level barriers.
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

constexpr int kTail = 256;             // waiting movers one block finishes alone

// Debug build: a mover entry names a replicate, a slot, a start cell inside
// the grid and offsets within the path table (the movement-order pass only
// writes such entries; this guards the rounds against anything else).
__device__ __forceinline__ bool entry_ok(const StepArgs& a, const MoveEntry& e) {
  if (!kChecked) return true;
  const int rep = (int)(e.ref >> 24);
  if (!fg_in(a.ctl, rep, a.n_rep)) return false;
  const RepDev& R = a.reps[rep];
  return fg_in(a.ctl, e.ref & 0xFFFFFFu, R.cap) && fg_in(a.ctl, e.c0 & 0xFFFFu, R.W) &&
         fg_in(a.ctl, e.c0 >> 16, R.H) && fg_in(a.ctl, (long long)((e.info >> MV_DX) & 15u) - 3, 11) &&
         fg_in(a.ctl, (long long)((e.info >> MV_DY) & 15u) - 3, 11);
}

// Claim value: an 8-bit round tag g (0..kTags-1; the value falls as g grows)
// above the 24-bit priority, so a claim of a later round always wins
// atomicMin over an older one.  Tags run on from step to step; the claim
// arrays are cleared, and g restarts at 0, before a step that would start
// with fewer than ctl->tag_reserve tags left, and within a step that runs out.
constexpr uint32_t kTags = 255;
__device__ __forceinline__ uint32_t claim_of(uint32_t g, uint32_t prio) {
  return ((254u - g) << 24) | prio;
}

// Sets every claim of every replicate to "none" (and, with marks, every
// contested-cell mark to "never"): grid-stride, or by the calling block alone.
__device__ __forceinline__ void clear_all_claims(const StepArgs& a, bool block_only = false,
                                                 bool marks = false) {
  const uint32_t stride = block_only ? blockDim.x : gridDim.x * blockDim.x;
  const uint32_t first = block_only ? threadIdx.x : blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < a.n_rep; ++r) {
    const RepDev& R = a.reps[r];
    if (!R.claim[0]) continue;
    const uint32_t n = (uint32_t)R.claim_tx * (uint32_t)((R.H + 15) >> 4) * 256u;
    for (uint32_t i = first; i < n; i += stride) {
      __stcg(&R.claim[0][i], 0xFFFFFFFFu);
      __stcg(&R.claim[1][i], 0xFFFFFFFFu);
    }
    if (marks)
      for (uint32_t i = first; i < n / 4; i += stride)
        __stcg(reinterpret_cast<uint32_t*>(R.cmark) + i, 0u);
  }
}

// A step starts a new claim epoch (all claims and marks cleared, tags and
// mark stamps from the start) if it could run out of tags or stamps.
__device__ __forceinline__ bool epoch_ends(const Ctl* ctl) {
  return ctl->claim_tag + ctl->tag_reserve > kTags || ctl->mark_stamp >= 254u;
}

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
// Footprints, priorities and first-round outcomes of all movers; agents that
// stay, or are blocked at their first path cell by an agent that stays, need
// no work at all.  Also clears the claims at the end of a claim epoch.
// s * d / L rounded half away from zero (the path cells of Sec. 2), for
// |d| <= L <= 5 and 1 <= s <= L, given invL = 1/L rounded to nearest.  The
// quotient is exact in binary for L = 1, 2, 4 and at least 1/10 away from a
// half for L = 3, 5, so |s * d| * invL + 1/2, rounded once, truncates to the
// same integer as the exact quotient (checked for every case on the host).
__device__ __forceinline__ int path_offset(int num, float invL) {
  const int r = (int)fmaf(fabsf((float)num), invL, 0.5f);
  return num < 0 ? -r : r;
}

__global__ void __launch_bounds__(256, 8) k_move_prep(StepArgs a, Chunks ch) {
  // a new claim epoch starts with clean claim and mark arrays (the rounds
  // kernel then starts its tags and stamps from the beginning)
  if (epoch_ends(a.ctl)) clear_all_claims(a, false, true);
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_base;
  const int t = a.ctl->t;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned alive_local = 0, foot_local = 0;
  int krep = -1;
  U4 k;
  int nrep = blockIdx.x < ch.n ? ch.rep[blockIdx.x] : 0;
  int nbeg = blockIdx.x < ch.n ? ch.begin[blockIdx.x] : 0;
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {  // the same chunks for the whole block
    const int rep = nrep;
    const RepDev& R = a.reps[rep];
    const int end = min(nbeg + kChunk, a.n_slots[rep]);
    const int slot = nbeg + threadIdx.x;
    // the agent's cell, desired cell and id together; the next chunk's place
    const int cell = slot < end ? R.cell[slot] : -1;
    const int des_ld = slot < end ? R.desired[slot] : -1;
    const uint32_t id_ld = slot < end ? (uint32_t)R.id[slot] : 0u;
    if (c + (int)gridDim.x < ch.n) {
      nrep = ch.rep[c + gridDim.x];
      nbeg = ch.begin[c + gridDim.x];
    }
    // the replicate's movement-order keys for this step (one Philox block
    // per warp, shared; kept while the block's chunks stay in one replicate)
    if (rep != krep) {
      if (lane == 0) k = move_step_keys((uint32_t)t, R.seed_lo, R.seed_hi);
      k.x = __shfl_sync(0xffffffffu, k.x, 0);
      k.y = __shfl_sync(0xffffffffu, k.y, 0);
      k.z = __shfl_sync(0xffffffffu, k.z, 0);
      k.w = __shfl_sync(0xffffffffu, k.w, 0);
      krep = rep;
    }
    bool mover = false;
    MoveEntry e;
    if (cell >= 0) ++alive_local;
    // debug build: the agent's cell and desired cell inside the grid, the
    // desired cell within the path table's reach (|dx|, |dy| <= 5)
    const long long C = (long long)R.W * R.H;
    const int des0 = cell >= 0 ? des_ld : -1;
    const bool sane = !kChecked || cell < 0 ||
                      (fg_in(a.ctl, cell, C) && fg_in(a.ctl, des0, C) &&
                       fg_in(a.ctl, des0 % R.W - cell % R.W + 5, 11) &&
                       fg_in(a.ctl, des0 / R.W - cell / R.W + 5, 11));
    if (cell >= 0 && sane) {
      const int des = des0;
      const int W = R.W;
      const int x0 = cell % W, y0 = cell / W;
      const int dx = des % W - x0, dy = des / W - y0;
      const int L = max(abs(dx), abs(dy));
      const float invL = __frcp_rn((float)max(L, 1));
      // all path records first (independent loads), then the scan
      uint32_t pr[6];
#pragma unroll
      for (int s = 1; s <= 5; ++s)
        pr[s] = (s <= L) ? R.rec[(y0 + path_offset(s * dy, invL)) * W +
                                 (x0 + path_offset(s * dx, invL))]
                         : REC_STA;
      int fp = 0;
      uint32_t ex = 0;
#pragma unroll
      for (int s = 1; s <= 5; ++s) {
        const uint32_t r = pr[s];
        if (s > L || (r & REC_STA)) break;
        if (rec_exit(r)) {
          ex = MV_EXIT;
          break;
        }
        fp = s;
      }
      if (fp > 0 || ex) {
        // the walk if nobody touches the footprint first: up to the first
        // occupied cell, or into an exit
        int fin = 0;
        bool gone = false, stop = false;
#pragma unroll
        for (int s = 1; s <= 5; ++s) {
          const uint32_t r = pr[s];
          stop = stop || s > L || (r & REC_OCC);
          if (!stop) {
            fin = s;
            if (rec_exit(r)) {
              gone = true;
              stop = true;
            }
          }
        }
        foot_local += (unsigned)fp + 1u;
        e.c0 = ((uint32_t)y0 << 16) | (uint32_t)x0;
        e.ref = ((uint32_t)rep << 24) | (uint32_t)slot;
        e.prio = move_priority(id_ld, k);
        e.info = (uint32_t)fp | ex | ((uint32_t)(dx + 8) << MV_DX) |
                 ((uint32_t)(dy + 8) << MV_DY) | ((uint32_t)fin << MV_FIN) |
                 (gone ? MV_GONE : 0u);
        mover = true;
      }
    }
    // the chunk's movers in one block-wide reservation of the mover list
    const unsigned bal = __ballot_sync(0xffffffffu, mover);
    if (lane == 0) s_warp[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t sum = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const uint32_t x = s_warp[w];
        s_warp[w] = sum;
        sum += x;
      }
      s_base = sum ? atomicAdd(&a.ctl->act_count[2], sum) : 0u;
    }
    __syncthreads();
    if (mover) {
      const uint32_t i = s_base + s_warp[wid] + __popc(bal & ((1u << lane) - 1u));
      if (i < a.act_cap) a.act[2][i] = e;
    }
    __syncthreads();
  }
  // agents alive at the start of the step, footprint cells of the movers
  for (int o = 16; o > 0; o >>= 1) {
    alive_local += __shfl_xor_sync(0xffffffffu, alive_local, o);
    foot_local += __shfl_xor_sync(0xffffffffu, foot_local, o);
  }
  if (lane == 0) {
    s_warp[wid] = alive_local;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long al = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) al += s_warp[w];
    if (al) atomicAdd(&a.ctl->agent_steps, al);
  }
  __syncthreads();
  if (lane == 0) s_warp[wid] = foot_local;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long fo = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) fo += s_warp[w];
    if (fo) atomicAdd(&a.ctl->foot_total, fo);
  }
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
__device__ bool grid_barrier_sum(Ctl* ctl, uint32_t& passed, uint32_t& sum0, uint32_t& sum1,
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
      // earlier; the poll acquires those of the rest
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

__device__ __forceinline__ bool round_barrier(Ctl* ctl, bool single, uint32_t& passed) {
  if (single) {
    __threadfence_block();
    __syncthreads();
    return true;
  }
  return grid_barrier(ctl, passed);
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

// A block's waiting movers: fields by mover, and the two index lists used in
// turn by the rounds (in shared memory or in the block's global slice).
struct MoverLists {
  uint32_t *P, *C0, *RF, *IN, *L0, *L1;
  __device__ __forceinline__ uint32_t* list(int i) const { return i ? L1 : L0; }
};

__device__ __forceinline__ MoverLists smem_lists(unsigned char* dsm) {
  MoverLists m;
  m.P = reinterpret_cast<uint32_t*>(dsm);
  m.C0 = m.P + kMoveSmemCap;
  m.RF = m.C0 + kMoveSmemCap;
  m.IN = m.RF + kMoveSmemCap;
  m.L0 = m.IN + kMoveSmemCap;
  m.L1 = m.L0 + kMoveSmemCap;
  return m;
}

// Claims of round tag g for the movers of a list (waiting movers that lost
// theirs when the claim arrays were cleared).
__device__ __forceinline__ void claim_list(const StepArgs& a, const PathTab* tab,
                                           const MoverLists& ml, const uint32_t* list,
                                           uint32_t n, uint32_t g) {
  for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
    const uint32_t idx = list[k];
    const uint32_t info = ml.IN[idx];
    const RepDev& R = a.reps[ml.RF[idx] >> 24];
    int c[6], q[6];
    foot_cells(tab, ml.C0[idx], R, info, c, q);
    const int n_fp = (int)(info & MV_LEN);
    const uint32_t v = claim_of(g, ml.P[idx]);
    uint32_t* cl = R.claim[g & 1u];
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (s <= n_fp) red_min_u32(&cl[q[s]], v);
  }
}

// Movers dealt to the blocks of the rounds kernel at a time (one warp's
// worth of consecutive list entries, so that the entry loads coalesce).
constexpr uint32_t kSpread = 32;

__global__ void __launch_bounds__(kMoveThreads, 2) k_move_rounds(StepArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ PathTab tab;
  __shared__ uint32_t s_cnt[2];
  __shared__ uint32_t s_base;
  build_path_tab(&tab);
  Ctl* ctl = a.ctl;
  uint32_t nbar = 0;                     // grid barriers passed
  // a new epoch (claims and marks cleared by the movement-order pass) starts
  // with tag 0 and stamp 1; every block decides alike, since nothing below
  // changes the two counters before the last barrier
  const bool fresh = epoch_ends(ctl);
  uint32_t g = fresh ? 0u : __ldcg(&ctl->claim_tag);  // tag of the current round
  const uint32_t stamp32 = fresh ? 1u : __ldcg(&ctl->mark_stamp) + 1u;
  const uint8_t stamp = (uint8_t)stamp32;
  const uint32_t n0 = min(__ldcg(&ctl->act_count[2]), a.act_cap);
  const uint32_t G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  // the step's movers go to the blocks in turn, kSpread at a time, so that
  // each block takes movers from all over the list; the block's k-th mover
  // is entry mover_at(k), and its slice of the global lists is [start, start + nb)
  const uint32_t nch = (n0 + kSpread - 1) / kSpread;
  const uint32_t rem = n0 % kSpread, last_owner = nch ? (nch - 1) % G : 0u;
  uint32_t start = (b * (nch / G) + min(b, nch % G)) * kSpread;
  uint32_t nb = (b < nch ? (nch - 1 - b) / G + 1 : 0u) * kSpread;
  if (rem) {
    if (last_owner < b) start -= kSpread - rem;
    else if (last_owner == b) nb -= kSpread - rem;
  }
  auto mover_at = [&](uint32_t k) { return ((k / kSpread) * G + b) * kSpread + k % kSpread; };
  const MoverLists sm = smem_lists(dsm);  // the block's shared-memory lists
  MoverLists gl;  // the block's slice of global memory
  gl.P = a.mv_prio + start;
  gl.C0 = a.mv_c0 + start;
  gl.RF = a.mv_ref + start;
  gl.IN = a.mv_info + start;
  gl.L0 = a.mv_list[0] + start;
  gl.L1 = a.mv_list[1] + start;
  if (tid < 2) s_cnt[tid] = 0u;
  const unsigned long long t_start = global_ns();
  if (b == 0 && tid == 0) {
    ctl->round_ns[0] = t_start;
    for (int i = 0; i < 8; ++i) ctl->phase_ns[i] = 0ull;
  }
  // the per-block maxima are first written after the first grid barrier
  if (b == 0)
    for (int i = tid; i < kRoundLog; i += blockDim.x) ctl->round_bmax[i] = 0u;
  __syncthreads();
  bool reclaim = g + 1u < kTags;  // tags left for the next round's claims

  // ---- claims of round 0, straight from the step's list
  for (uint32_t k = tid; k < nb; k += blockDim.x) {
    const MoveEntry e = a.act[2][mover_at(k)];
    if (!entry_ok(a, e)) continue;
    const RepDev& R = a.reps[e.ref >> 24];
    int c[6], q[6];
    foot_cells(&tab, e.c0, R, e.info, c, q);
    const int n = (int)(e.info & MV_LEN);
    uint32_t* cl = R.claim[g & 1u];
    const uint32_t v = claim_of(g, e.prio);
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (s <= n) red_min_u32(&cl[q[s]], v);
  }
  if (tid == 0) atomicMax(&ctl->phase_ns[3], global_ns() - t_start);
  if (!grid_barrier(ctl, nbar)) return;

  // ---- round 0: the ones that must wait claim for round 1 and go to the
  // block's lists (shared memory first, global memory beyond its capacity).
  // Two movers per pass: both movers' claim words are in flight together.
  auto r0_load = [&](const MoveEntry& e, uint32_t* cl) {
    const RepDev& R = a.reps[e.ref >> 24];
    int c[6], q[6];
    foot_cells(&tab, e.c0, R, e.info, c, q);
    const int n = (int)(e.info & MV_LEN);
    const uint32_t* now = R.claim[g & 1u];
    const uint32_t mine_v = claim_of(g, e.prio);
#pragma unroll
    for (int s = 0; s < 6; ++s) cl[s] = (s <= n) ? __ldcg(&now[q[s]]) : mine_v;
  };
  auto r0_decide = [&](const MoveEntry& e, const uint32_t* cl) {
    const int rep = (int)(e.ref >> 24), slot = (int)(e.ref & 0xFFFFFFu);
    const RepDev& R = a.reps[rep];
    int c[6], q[6];
    foot_cells(&tab, e.c0, R, e.info, c, q);
    const uint32_t mine_v = claim_of(g, e.prio);
    uint32_t need = 0u;
#pragma unroll
    for (int s = 0; s < 6; ++s) need |= (cl[s] != mine_v) ? (1u << s) : 0u;
    if (need == 0u) {
      commit_first(a, R, rep, slot, c, e.info);
    } else {
      // the cells this agent lost are contested: mark them for this step
#pragma unroll
      for (int s = 0; s < 6; ++s)
        if ((need >> s) & 1u) R.cmark[q[s]] = stamp;
      const uint32_t j = append_slot(&s_cnt[1]);
      const MoverLists& dst = j < (uint32_t)kMoveSmemCap ? sm : gl;
      dst.P[j] = e.prio;
      dst.C0[j] = e.c0;
      dst.RF[j] = e.ref;
      dst.IN[j] = (e.info & ~(0x3Fu << MV_NEED)) | (need << MV_NEED);
    }
  };
  for (uint32_t k = tid; k < nb; k += 2u * blockDim.x) {
    bool two = k + blockDim.x < nb;
    const MoveEntry e1 = a.act[2][mover_at(k)];
    MoveEntry e2 = e1;
    if (two) e2 = a.act[2][mover_at(k + blockDim.x)];
    const bool one = entry_ok(a, e1);
    two = two && entry_ok(a, e2);
    uint32_t cl1[6], cl2[6];
    if (one) r0_load(e1, cl1);
    if (two) r0_load(e2, cl2);
    if (one) r0_decide(e1, cl1);
    if (two) r0_decide(e2, cl2);
  }
  __syncthreads();
  const uint32_t w0 = s_cnt[1];
  // the waiting movers stay in shared memory when they all fit there (a
  // block's choice); else the first kMoveSmemCap join the rest in global
  const bool in_smem = w0 <= (uint32_t)kMoveSmemCap;
  if (!in_smem)
    for (uint32_t k = tid; k < (uint32_t)kMoveSmemCap; k += blockDim.x) {
      gl.P[k] = sm.P[k];
      gl.C0[k] = sm.C0[k];
      gl.RF[k] = sm.RF[k];
      gl.IN[k] = sm.IN[k];
    }
  MoverLists ml = in_smem ? sm : gl;
  for (uint32_t k = tid; k < w0; k += blockDim.x) ml.L1[k] = k;
  if (tid == 0) {
    atomicMax(&ctl->phase_ns[0], global_ns() - t_start);
    atomicMax(&ctl->phase_ns[4], (unsigned long long)nb);
    atomicMax(&ctl->phase_ns[5], (unsigned long long)w0);
    if (w0) atomicMax(&ctl->round_bmax[0], w0);
  }
  uint32_t bsum0 = 0u, bsum1 = 0u, waiting = 0u;  // running sums of the barrier words
  if (!grid_barrier_sum(ctl, nbar, bsum0, bsum1, w0, &waiting)) return;
  if (tid == 0) atomicMax(&ctl->phase_ns[1], global_ns() - t_start);
  // the cells each waiting agent must keep claiming: the ones it has not
  // held, and the ones it held that another agent lost (claimed too); a
  // cell only it claims is nobody else's concern for the rest of the step.
  // Round 1's claims are made here, on those cells only.
  for (uint32_t k = tid; k < w0; k += blockDim.x) {
    const uint32_t info = ml.IN[k];
    const RepDev& R = a.reps[ml.RF[k] >> 24];
    int c[6], q[6];
    foot_cells(&tab, ml.C0[k], R, info, c, q);
    const int n = (int)(info & MV_LEN);
    const uint32_t need = (info >> MV_NEED) & 0x3Fu;
    uint32_t clm = need;
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (s <= n && !((need >> s) & 1u) && __ldcg(&R.cmark[q[s]]) == stamp) clm |= 1u << s;
    ml.IN[k] = (info & ~(0x3Fu << MV_CLM)) | (clm << MV_CLM);
    if (reclaim) {
      uint32_t* nxt = R.claim[(g + 1u) & 1u];
      const uint32_t v = claim_of(g + 1u, ml.P[k]);
#pragma unroll
      for (int s = 0; s < 6; ++s)
        if ((clm >> s) & 1u) red_min_u32(&nxt[q[s]], v);
    }
  }
  if (!grid_barrier(ctl, nbar)) return;
  if (b == 0 && tid == 0) {
    ctl->round_n[0] = waiting;
    ctl->round_ns[1] = global_ns();
  }
  int r = 1;
  bool single = (G == 1);
  while (waiting > 0) {
    const int in_l = r & 1, out_l = (r + 1) & 1;
    if (!reclaim) {
      // out of tags: clear every claim, then the waiting movers claim again
      // with the first tag
      __syncthreads();
      clear_all_claims(a, single);
      if (!round_barrier(ctl, single, nbar)) return;
      g = 0u;
      claim_list(a, &tab, ml, ml.list(in_l), s_cnt[in_l], 0u);
      if (!round_barrier(ctl, single, nbar)) return;
    } else {
      ++g;
    }
    if (!single && waiting <= (uint32_t)kTail) {
      // hand every waiting mover to block 0, which finishes alone
      const uint32_t n_it = s_cnt[in_l];
      if (tid == 0) s_base = n_it ? atomicAdd(&ctl->tail_count, n_it) : 0u;
      __syncthreads();
      const uint32_t* lin = ml.list(in_l);
      for (uint32_t k = tid; k < n_it; k += blockDim.x) {
        const uint32_t idx = lin[k];
        MoveEntry e;
        e.c0 = ml.C0[idx];
        e.ref = ml.RF[idx];
        e.prio = ml.P[idx];
        e.info = ml.IN[idx];
        a.act[0][s_base + k] = e;
      }
      if (!grid_barrier(ctl, nbar)) return;
      if (b != 0) return;
      const uint32_t nt = __ldcg(&ctl->tail_count);
      ml = smem_lists(dsm);
      uint32_t* lt = ml.list(in_l);
      for (uint32_t k = tid; k < nt; k += blockDim.x) {
        const MoveEntry e = a.act[0][k];
        ml.P[k] = e.prio;
        ml.C0[k] = e.c0;
        ml.RF[k] = e.ref;
        ml.IN[k] = e.info;
        lt[k] = k;
      }
      if (tid == 0) {
        s_cnt[in_l] = nt;
        ctl->phase_ns[6] = (unsigned long long)r;
      }
      single = true;
      __syncthreads();
    }
    // every agent still waiting checks its claims of tag g, moves if it
    // holds all its cells, else claims with tag g+1
    reclaim = g + 1u < kTags;
    const uint32_t n_it = s_cnt[in_l];
    __syncthreads();
    if (tid == 0) s_cnt[out_l] = 0u;
    __syncthreads();
    const unsigned long long t_round = global_ns();
    const uint32_t* lin = ml.list(in_l);
    uint32_t* lout = ml.list(out_l);
    for (uint32_t k = tid; k < n_it; k += blockDim.x) {
      const uint32_t idx = lin[k];
      const uint32_t info = ml.IN[idx];
      const uint32_t ref = ml.RF[idx];
      const uint32_t p = ml.P[idx];
      const int rep = (int)(ref >> 24), slot = (int)(ref & 0xFFFFFFu);
      const RepDev& R = a.reps[rep];
      int c[6], q[6];
      foot_cells(&tab, ml.C0[idx], R, info, c, q);
      const int n = (int)(info & MV_LEN);
      const uint32_t* now = R.claim[g & 1u];
      const uint32_t mine_v = claim_of(g, p);
      // only the cells not held yet need a look: a cell once held stays
      // held, since its claimants can only leave
      const uint32_t need0 = (info >> MV_NEED) & 0x3Fu;
      uint32_t cl[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) cl[s] = ((need0 >> s) & 1u) ? __ldcg(&now[q[s]]) : mine_v;
      uint32_t need = 0u;
#pragma unroll
      for (int s = 0; s < 6; ++s) need |= (cl[s] != mine_v) ? (1u << s) : 0u;
      const bool mine = need == 0u;
      if (mine) {
        const int wl = walk_len(info);
        uint32_t pr[6];
#pragma unroll
        for (int s = 0; s < 6; ++s) pr[s] = (s <= wl) ? __ldcg(&R.rec[c[s]]) : REC_OCC;
        commit_move(a, R, rep, slot, c, pr);
      } else {
        if (reclaim) {
          uint32_t* nxt = R.claim[(g + 1u) & 1u];
          const uint32_t v = claim_of(g + 1u, p);
          const uint32_t clm = (info >> MV_CLM) & 0x3Fu;
#pragma unroll
          for (int s = 0; s < 6; ++s)
            if ((clm >> s) & 1u) red_min_u32(&nxt[q[s]], v);
        }
        if (need != need0) ml.IN[idx] = (info & ~(0x3Fu << MV_NEED)) | (need << MV_NEED);
        lout[append_slot(&s_cnt[out_l])] = idx;
      }
    }
    __syncthreads();
    if (tid == 0 && r == 1) atomicMax(&ctl->phase_ns[2], global_ns() - t_round);
    if (tid == 0 && r < kRoundLog && s_cnt[out_l]) atomicMax(&ctl->round_bmax[r], s_cnt[out_l]);
    if (single) {
      __threadfence_block();
      waiting = s_cnt[out_l];
    } else {
      if (!grid_barrier_sum(ctl, nbar, bsum0, bsum1, s_cnt[out_l], &waiting)) return;
    }
    if (b == 0 && tid == 0 && r < kRoundLog) {
      ctl->round_n[r] = waiting;
      ctl->round_ns[r + 1] = global_ns();
    }
    ++r;
    if (r > (int)n0 + 1) {
      if (b == 0 && tid == 0) atomicCAS(&ctl->err, 0, kDevErrRounds);
      return;
    }
  }
  if (b == 0 && tid == 0) {
    // the next step's first claims use a tag below every one used so far
    ctl->claim_tag = min(g + 1u, kTags);
    ctl->mark_stamp = stamp32;
    ctl->movers_total += (unsigned long long)n0;
    ctl->rounds_last = r;
    ctl->rounds_total += (unsigned long long)r;
    if (r > ctl->rounds_max) ctl->rounds_max = r;
  }
}

// Cost of the grid barrier: `iters` barriers in a row, block 0 thread 0
// records the elapsed global time in ctl->round_ns[0].
__global__ void __launch_bounds__(1024, 1) k_barrier_cost(Ctl* ctl, int iters) {
  uint32_t nbar = 0;
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < iters; ++i)
    if (!grid_barrier(ctl, nbar)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->round_ns[0] = global_ns() - t0;
}

// Check of the counting barrier: at barrier i every block brings the count
// (block % 5) + (i % 4); every block compares each total with the exact sum
// and counts the differences in ctl->flips.
__global__ void __launch_bounds__(1024, 1) k_barrier_sum(Ctl* ctl, int iters) {
  uint32_t nbar = 0, sum0 = 0u, sum1 = 0u;
  const uint32_t G = gridDim.x;
  const uint32_t base = (G / 5u) * 10u + (G % 5u) * (G % 5u - 1u) / 2u;  // sum of b % 5
  for (int i = 0; i < iters; ++i) {
    uint32_t total = 0u;
    const uint32_t count = blockIdx.x % 5u + (uint32_t)(i & 3);
    if (!grid_barrier_sum(ctl, nbar, sum0, sum1, count, &total)) return;
    if (threadIdx.x == 0 && total != base + G * (uint32_t)(i & 3)) atomicAdd(&ctl->flips, 1ull);
  }
}

int test_barrier_sum_launch(Ctl* ctl, int grid, int block, int iters, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_barrier_sum, ctl, iters) == cudaSuccess ? 0 : -1;
}

int test_barrier_cost_launch(Ctl* ctl, int grid, int block, int iters, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_barrier_cost, ctl, iters) == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ void reset_step_counters(Ctl* c) {
  c->q_count = 0u;
  for (int i = 0; i < 3; ++i) c->act_count[i] = 0u;
  c->tail_count = 0u;
  c->bar_acc[0][0] = 0ull;
  c->bar_acc[1][0] = 0ull;
}

__global__ void k_step_begin(StepArgs a) {
  if (threadIdx.x == 0) reset_step_counters(a.ctl);
}

__global__ void k_step_end(StepArgs a) {
  if (threadIdx.x == 0) {
    a.ctl->t += 1;
    reset_step_counters(a.ctl);
  }
}

// Launched every step, even without agents: the claim clean-up must not be
// skipped when the rounds kernel starts a new epoch.
int move_prep_launch(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s) {
  k_move_prep<<<grid > 0 ? grid : 1, 256, 0, s>>>(a, ch);
  return 0;
}

size_t move_rounds_smem() { return (size_t)kMoveSmemCap * 24; }

int move_rounds_max_grid(int block, int* grid_out) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaFuncSetAttribute(k_move_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)move_rounds_smem()) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_move_rounds, block,
                                                    move_rounds_smem()) != cudaSuccess)
    return -1;
  *grid_out = sms * (per > 0 ? per : 1);
  return 0;
}

int move_rounds_launch(const StepArgs& a, int grid, int block, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = move_rounds_smem();
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
  uint32_t nbar = 0;
  grid_barrier(ctl, nbar);
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
