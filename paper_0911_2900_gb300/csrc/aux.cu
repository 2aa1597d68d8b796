// aux.cu -- set-up and bookkeeping kernels: line-of-sight masks, agent
// placement, spatial (Hilbert-order) re-sort with compaction of agents that left, digests,
// read-back gathers, the reach-union counter used for byte accounting, and
// the kernels behind the library's self-test entry points.
#include <algorithm>

#include "fast_device.cuh"

namespace fastgb {

// ---------------------------------------------------------------------------
// Line-of-sight mask of every cell: bit k set when the k-th reach offset lands
// inside the grid and its straight path crosses no wall (nor any cell that no
// exit can be reached from).  Static for the lifetime of the grid.
__global__ void k_masks(const RepDev* rp, int64_t cells, int v, int mw, unsigned long long* out) {
  const RepDev R = *rp;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long m[2] = {0ull, 0ull};
    if (!rec_sentinel(R.rec[c])) {
      const int x0 = (int)(c % R.W), y0 = (int)(c / R.W);
      int k = 0;
      for (int dy = -v; dy <= v; ++dy)
        for (int dx = -v; dx <= v; ++dx) {
          if (!reach_in(dx, dy, v, R.reach)) continue;
          const int tx = x0 + dx, ty = y0 + dy;
          bool ok = tx >= 0 && tx < R.W && ty >= 0 && ty < R.H;
          const int L = max(abs(dx), abs(dy));
          for (int s = 1; ok && s <= L; ++s) {
            const int px = x0 + div_half_away(s * dx, L), py = y0 + div_half_away(s * dy, L);
            ok = !rec_sentinel(R.rec[(int64_t)py * R.W + px]);
          }
          if (ok) m[k >> 6] |= 1ull << (k & 63);
          ++k;
        }
    }
    out[c * mw] = m[0];
    if (mw > 1) out[c * mw + 1] = m[1];
  }
}

int masks_launch(const RepDev& h, RepDev* d, int64_t cells, cudaStream_t s) {
  return masks_speed_launch(d, cells, h.v, h.mw, h.mask, s);
}

int masks_speed_launch(RepDev* d, int64_t cells, int v, int mw, unsigned long long* out,
                       cudaStream_t s) {
  const int64_t blocks = (cells + 255) / 256;
  k_masks<<<(int)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(d, cells, v, mw, out);
  return 0;
}

// ---------------------------------------------------------------------------
// Placement: clear the previous agents' marks, then write the new agents.
// With slot_of_id, also records the slot each id below n_ids holds (the
// caller sets the array to -1 first), so that a new placement can keep the
// storage order.
__global__ void k_clear_occ(RepDev* rp, const int32_t* n_slots, int rep, int cap,
                            int32_t* slot_of_id, int n_ids) {
  const RepDev& R = *rp;
  const int n = min(n_slots[rep], cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = R.cell[i];
    if (c >= 0) R.rec[c] &= ~(REC_OCC | REC_STA);
    R.cell[i] = -1;
    if (slot_of_id) {
      const int id = R.id[i];
      if (id >= 0 && id < n_ids) slot_of_id[id] = i;
    }
  }
}

int clear_occ_launch(RepDev* d, const int32_t* n_slots, int rep, int cap, int32_t* slot_of_id,
                     int n_ids, cudaStream_t s) {
  k_clear_occ<<<(cap + 255) / 256 > 0 ? (cap + 255) / 256 : 1, 256, 0, s>>>(d, n_slots, rep, cap,
                                                                           slot_of_id, n_ids);
  return 0;
}

// Places agents i < n in slots i, checking on the device what the host used
// to check: the cell is inside the grid, free, reachable and not an exit, no
// two agents share a cell, and (with explicit ids) every id is in [0, 2^24)
// and unique.  The occupancy bit is taken with an atomic, so a taken cell is
// found by whichever agent comes second.  Without explicit ids, id i is
// absent when cells[i] == -1.  err[0] receives the smallest failing index,
// err[1] the number of agents placed; placed[i] marks the cells this call
// took, for a roll-back.  With slot_of_id (implicit ids only), agent i goes
// to the slot its id held before instead (the storage order stays as the
// last spatial sort left it), or, if it held none, to slot
// *n_slots_old + err[2]++; an absent agent then takes no slot.
// One agent of a placement (see k_place_checked); returns whether it counts
// as present (placed, or refused: err[0] then names it).
__device__ __forceinline__ bool place_one(const RepDev& R, int i, int c, int id, bool explicit_ids,
                                          long long n_cells, uint32_t* id_bits, uint8_t* placed,
                                          const uint8_t* speed_by_id, int n_speed_ids,
                                          const int32_t* slot_of_id, const int32_t* n_slots_old,
                                          int32_t* err) {
  placed[i] = 0;
  if (slot_of_id && c == -1) return false;
  int slot = i;
  if (slot_of_id) {
    slot = slot_of_id[i];
    if (slot < 0) slot = *n_slots_old + atomicAdd(&err[2], 1);
    if (slot >= R.cap) {  // cannot happen with the host's conditions; refused all the same
      atomicMin(&err[0], i);
      return false;
    }
  }
  if (speed_by_id) R.speed[slot] = (id >= 0 && id < n_speed_ids) ? speed_by_id[id] : (uint8_t)1;
  if (!explicit_ids && c == -1) {
    R.cell[slot] = -1;
    R.id[slot] = i;
    R.desired[slot] = -1;
    return false;
  }
  bool ok = c >= 0 && (long long)c < n_cells;
  // with speeds per agent, every placed id needs one
  ok = ok && (!speed_by_id || (id >= 0 && id < n_speed_ids));
  if (ok) {
    const uint32_t old = atomicOr(&R.rec[c], REC_OCC);
    if (!(old & REC_OCC)) placed[i] = 1;
    ok = !(old & REC_OCC) && !rec_exit(old);
  }
  if (ok && explicit_ids) {
    ok = id >= 0 && id < (1 << kMaxIdBits);
    if (ok) {
      const uint32_t bit = 1u << (id & 31);
      ok = !(atomicOr(&id_bits[id >> 5], bit) & bit);
    }
  }
  if (!ok) atomicMin(&err[0], i);
  R.cell[slot] = ok ? c : -1;
  R.id[slot] = id;
  R.desired[slot] = ok ? c : -1;
  return true;
}

__global__ void k_place_checked(RepDev* rp, const int32_t* cells, const int32_t* ids, int n,
                                long long n_cells, uint32_t* id_bits, uint8_t* placed,
                                const uint8_t* speed_by_id, int n_speed_ids,
                                const int32_t* slot_of_id, const int32_t* n_slots_old,
                                int32_t* err) {
  const RepDev& R = *rp;
  int present = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    present += place_one(R, i, cells[i], ids ? ids[i] : i, ids != nullptr, n_cells, id_bits,
                         placed, speed_by_id, n_speed_ids, slot_of_id, n_slots_old, err)
                   ? 1
                   : 0;
  // the block's count first, then one atomic per block (one per warp on a
  // single word was most of the kernel's time)
  __shared__ int s_present[32];
  for (int o = 16; o > 0; o >>= 1) present += __shfl_xor_sync(0xffffffffu, present, o);
  if ((threadIdx.x & 31) == 0) s_present[threadIdx.x >> 5] = present;
  __syncthreads();
  if (threadIdx.x == 0) {
    int sum = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_present[w];
    if (sum) atomicAdd(&err[1], sum);
  }
}

// Undoes the occupancy bits a failed placement took.
__global__ void k_place_rollback(RepDev* rp, const int32_t* cells, int n, const uint8_t* placed) {
  const RepDev& R = *rp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (placed[i]) atomicAnd(&R.rec[cells[i]], ~(REC_OCC | REC_STA));
    R.cell[i] = -1;
  }
}

int place_checked_launch(RepDev* d, const int32_t* cells, const int32_t* ids, int n,
                         long long n_cells, uint32_t* id_bits, uint8_t* placed,
                         const uint8_t* speed_by_id, int n_speed_ids, const int32_t* slot_of_id,
                         const int32_t* n_slots_old, int32_t* err, cudaStream_t s) {
  if (n <= 0) return 0;
  const int grid = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  k_place_checked<<<grid, 256, 0, s>>>(d, cells, ids, n, n_cells, id_bits, placed, speed_by_id,
                                       n_speed_ids, slot_of_id, n_slots_old, err);
  return 0;
}

int place_rollback_launch(RepDev* d, const int32_t* cells, int n, const uint8_t* placed,
                          cudaStream_t s) {
  if (n <= 0) return 0;
  const int grid = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  k_place_rollback<<<grid, 256, 0, s>>>(d, cells, n, placed);
  return 0;
}

// ---------------------------------------------------------------------------
// Batched placement and read-back: every replicate of a context in one launch
// per stage (a launch per replicate and stage cost more than the work of a
// small replicate).  bp[r] describes replicate r for the call; the chunk
// kernels walk the work list of all placed replicates' slots.

// Slot-of-id maps (in id2) set to "none" for the replicates that keep their
// storage order.
__global__ void k_batch_prepare(RepDev* reps, Chunks ch, const BatchRep* bp) {
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const BatchRep& b = bp[rep];
    const int s = ch.begin[c] + threadIdx.x;
    if (b.keep && s < b.n) reps[rep].id2[s] = -1;
  }
}

// The previous agents' marks cleared and every slot emptied, as k_clear_occ,
// for the replicates this call places; the slot-of-id maps filled.
__global__ void k_batch_clear(RepDev* reps, const int32_t* n_slots, Chunks ch, const BatchRep* bp) {
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const BatchRep& b = bp[rep];
    if (!b.clear) continue;
    const RepDev& R = reps[rep];
    const int s = ch.begin[c] + threadIdx.x;
    if (s >= R.cap) continue;
    if (s < min(n_slots[rep], R.cap)) {
      const int cell = R.cell[s];
      if (cell >= 0) R.rec[cell] &= ~(REC_OCC | REC_STA);
      if (b.keep) {
        const int id = R.id[s];
        if (id >= 0 && id < b.n) R.id2[id] = s;
      }
    }
    R.cell[s] = -1;
  }
}

// The staged agents of all replicates (implicit ids), checked and placed as
// k_place_checked does; errs[3r..3r+2] as its err for replicate r.
__global__ void k_batch_place(RepDev* reps, const int32_t* staged, long long total,
                              const BatchRep* bp, int n_rep, const int32_t* n_slots,
                              int32_t* errs) {
  const int lane = threadIdx.x & 31;
  for (long long g0 = (long long)blockIdx.x * blockDim.x; g0 < total;
       g0 += (long long)gridDim.x * blockDim.x) {  // the same g0 for the whole block
    const long long g = g0 + threadIdx.x;
    bool present = false;
    int rep = 0;
    if (g < total) {
      // the replicate whose range holds g: the last with bp[r].off <= g
      int lo = 0, hi = n_rep - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bp[mid].off <= g) lo = mid;
        else hi = mid - 1;
      }
      rep = lo;
      const BatchRep& b = bp[rep];
      const RepDev& R = reps[rep];
      const int i = (int)(g - b.off);
      present = place_one(R, i, staged[g], i, false, (long long)R.W * R.H, nullptr,
                          reinterpret_cast<uint8_t*>(R.mvinfo), b.speed_by_id, b.n_speed_ids,
                          b.keep ? R.id2 : nullptr, n_slots + rep, errs + 3 * rep);
    }
    // the lanes that place agents of one replicate count them with one atomic
    const unsigned same = __match_any_sync(0xffffffffu, present ? rep : -1 - lane);
    if (present && __ffs(same) - 1 == lane) atomicAdd(&errs[3 * rep + 1], __popc(same));
  }
}

// Read-back of all replicates: cell and desired cell by id, at bp[r].off + id.
__global__ void k_batch_gather(const RepDev* reps, const int32_t* n_slots, Chunks ch,
                               const BatchRep* bp, int32_t* out_cell, int32_t* out_des) {
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const BatchRep& b = bp[rep];
    const RepDev& R = reps[rep];
    const int s = ch.begin[c] + threadIdx.x;
    if (s >= min(n_slots[rep], R.cap)) continue;
    const int cell = R.cell[s];
    if (cell < 0) continue;
    const int id = R.id[s];
    if (id < 0 || id >= b.n) continue;
    out_cell[b.off + id] = cell;
    out_des[b.off + id] = R.desired[s];
  }
}

int batch_prepare_launch(RepDev* reps, const Chunks& ch, const BatchRep* bp, int grid,
                         cudaStream_t s) {
  if (ch.n > 0) k_batch_prepare<<<grid, kChunk, 0, s>>>(reps, ch, bp);
  return 0;
}

int batch_clear_launch(RepDev* reps, const int32_t* n_slots, const Chunks& ch, const BatchRep* bp,
                       int grid, cudaStream_t s) {
  if (ch.n > 0) k_batch_clear<<<grid, kChunk, 0, s>>>(reps, n_slots, ch, bp);
  return 0;
}

int batch_place_launch(RepDev* reps, const int32_t* staged, long long total, const BatchRep* bp,
                       int n_rep, const int32_t* n_slots, int32_t* errs, int grid,
                       cudaStream_t s) {
  if (total > 0) k_batch_place<<<grid, 256, 0, s>>>(reps, staged, total, bp, n_rep, n_slots, errs);
  return 0;
}

int batch_gather_launch(const RepDev* reps, const int32_t* n_slots, const Chunks& ch,
                        const BatchRep* bp, int32_t* out_cell, int32_t* out_des, int grid,
                        cudaStream_t s) {
  if (ch.n > 0) k_batch_gather<<<grid, kChunk, 0, s>>>(reps, n_slots, ch, bp, out_cell, out_des);
  return 0;
}

// ---------------------------------------------------------------------------
// Spatial re-sort.  Buckets are 2^tile_shift square tiles numbered along a
// Hilbert curve inside each replicate (consecutive buckets are always
// neighbouring tiles, so a run of consecutive agents stays compact); a
// counting sort by bucket keeps agents that are close on the grid close in
// memory and drops agents that left.
//
// Hilbert index of tile (x, y) in a side x side square (side a power of two):
// at each scale s the quadrant (rx, ry) contributes s*s*((3*rx) ^ ry), then
// the coordinates are reflected / swapped into the quadrant's own frame.
__device__ __forceinline__ uint32_t hilbert_index(uint32_t side, uint32_t x, uint32_t y) {
  uint32_t d = 0;
  for (uint32_t s = side >> 1; s > 0; s >>= 1) {
    const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
    d += s * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = side - 1 - x;
        y = side - 1 - y;
      }
      const uint32_t tmp = x;
      x = y;
      y = tmp;
    }
  }
  return d;
}

// With speeds per agent the buckets come in five speed classes, one after the
// other, so that the agents of one speed are contiguous (each speed's
// planning launch then finds its agents together in a warp).
__device__ __forceinline__ int bucket_classes(const RepDev& R) { return R.speed ? 5 : 1; }

__device__ __forceinline__ int bucket_of(const RepDev& R, int cell, int slot) {
  const int x = cell % R.W, y = cell / R.W;
  uint32_t side = 1;
  while (side * side < (uint32_t)R.bucket_span) side <<= 1;
  const int cls = R.speed ? (int)R.speed[slot] - 1 : 0;
  return R.bucket_base + cls * R.bucket_span +
         (int)hilbert_index(side, (uint32_t)(x >> R.tile_shift), (uint32_t)(y >> R.tile_shift));
}

__global__ void k_bucket_zero(StepArgs a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= a.n_buckets;
       i += gridDim.x * blockDim.x)
    a.bucket_count[i] = 0u;
}

// The agents of a warp are mostly in one or two buckets (they were sorted by
// bucket the last time): lanes with the same bucket make one atomic together.
// Returns, for lane `lane`, its bucket (-1: none), the lanes that share it and
// whether it leads them (the lowest of them).
struct BucketGroup {
  int bucket;
  unsigned lanes;
  bool leader;
};

__device__ __forceinline__ BucketGroup bucket_group(const RepDev& R, int cell, int slot, bool valid) {
  const int lane = threadIdx.x & 31;
  BucketGroup g;
  g.bucket = valid ? bucket_of(R, cell, slot) : -1;
  // lanes without an agent get keys of their own
  g.lanes = __match_any_sync(0xffffffffu, valid ? g.bucket : -1 - lane);
  g.leader = valid && (__ffs(g.lanes) - 1 == lane);
  return g;
}

__global__ void k_bucket_count(StepArgs a, Chunks ch) {
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {  // the same chunks for the whole block
    const int rep = ch.rep[c];
    const RepDev& R = a.reps[rep];
    const int slot = ch.begin[c] + threadIdx.x;
    const bool in = slot < min(ch.begin[c] + kChunk, a.n_slots[rep]);
    const int cell = in ? R.cell[slot] : -1;
    const BucketGroup g = bucket_group(R, cell, slot, cell >= 0);
    if (g.leader) atomicAdd(&a.bucket_count[g.bucket], (uint32_t)__popc(g.lanes));
  }
}

// Exclusive scan of the bucket counts in place, in three launches: every
// block sums its range of buckets (coalesced), then every block scans its
// range in tiles of 1024 starting from the sum of the blocks before it, then
// one block derives each replicate's first offset and new agent count.  The
// block sums live after the per-replicate words of the bucket array.
constexpr int kScanThreads = 1024;
constexpr int kScanMaxBlocks = 1024;

__device__ __forceinline__ uint32_t* scan_parts(const StepArgs& a) {
  return a.bucket_count + a.n_buckets + 1 + 2 * a.n_rep;
}

__device__ __forceinline__ void scan_range(int n, int b, int nb, int* lo, int* hi) {
  const int per = ((n + nb - 1) / nb + kScanThreads - 1) / kScanThreads * kScanThreads;
  *lo = min(n, b * per);
  *hi = min(n, *lo + per);
}

// Block-wide inclusive scan of one value per thread (kScanThreads threads).
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) s_warp[wid] = v;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t add = wid > 0 ? s_warp[wid - 1] : 0u;
  __syncthreads();
  return v + add;
}

__global__ void __launch_bounds__(kScanThreads) k_bucket_scan_parts(StepArgs a) {
  __shared__ uint32_t s_warp[32];
  int lo, hi;
  scan_range(a.n_buckets, blockIdx.x, gridDim.x, &lo, &hi);
  uint32_t sum = 0;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) sum += a.bucket_count[i];
  const uint32_t tot = block_incl_scan(sum, s_warp);
  if (threadIdx.x == blockDim.x - 1) scan_parts(a)[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_bucket_scan_apply(StepArgs a) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_run;
  const uint32_t* parts = scan_parts(a);
  // the sum of the blocks before this one
  const uint32_t before = threadIdx.x < blockIdx.x ? parts[threadIdx.x] : 0u;
  const uint32_t off = block_incl_scan(before, s_warp);
  if (threadIdx.x == blockDim.x - 1) s_run = off;
  __syncthreads();
  int lo, hi;
  scan_range(a.n_buckets, blockIdx.x, gridDim.x, &lo, &hi);
  for (int base = lo; base < hi; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < hi ? a.bucket_count[i] : 0u;
    const uint32_t incl = block_incl_scan(v, s_warp);
    const uint32_t run = s_run;
    if (i < hi) a.bucket_count[i] = run + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_run = run + incl;
    __syncthreads();
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) a.bucket_count[a.n_buckets] = s_run;
}

// Per replicate: its first offset (the scatter subtracts it) and its new
// agent count (the copy and the commit use it).
__global__ void k_bucket_scan_reps(StepArgs a) {
  for (int r = threadIdx.x; r < a.n_rep; r += blockDim.x) {
    const RepDev& R = a.reps[r];
    const uint32_t b0 = a.bucket_count[R.bucket_base];
    const uint32_t b1 = a.bucket_count[R.bucket_base + R.bucket_span * bucket_classes(R)];
    a.bucket_count[a.n_buckets + 1 + 2 * r] = b0;
    a.bucket_count[a.n_buckets + 2 + 2 * r] = b1 - b0;
  }
}

__global__ void k_bucket_scatter(StepArgs a, Chunks ch) {
  const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {  // the same chunks for the whole block
    const int rep = ch.rep[c];
    const RepDev& R = a.reps[rep];
    const int slot = ch.begin[c] + threadIdx.x;
    const bool in = slot < min(ch.begin[c] + kChunk, a.n_slots[rep]);
    const int cell = in ? R.cell[slot] : -1;
    const BucketGroup g = bucket_group(R, cell, slot, cell >= 0);
    // the group's leader takes its places in the bucket, every lane its own
    // one in lane order
    uint32_t base = 0u;
    if (g.leader) base = atomicAdd(&a.bucket_count[g.bucket], (uint32_t)__popc(g.lanes));
    base = __shfl_sync(0xffffffffu, base, g.bucket >= 0 ? __ffs(g.lanes) - 1 : 0);
    if (cell < 0) continue;
    const uint32_t pos = base + (uint32_t)__popc(g.lanes & below) -
                         a.bucket_count[a.n_buckets + 1 + 2 * rep];
    R.id2[pos] = R.id[slot];
    R.cell2[pos] = cell;
    if (R.speed) R.speed2[pos] = R.speed[slot];
    R.mvinfo[pos] = (uint32_t)R.desired[slot];  // movement scratch, free until the next step
  }
}

__global__ void k_bucket_copy(StepArgs a, Chunks ch) {
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const RepDev& R = a.reps[rep];
    const int n_new = (int)a.bucket_count[a.n_buckets + 2 + 2 * rep];
    const int slot = ch.begin[c] + threadIdx.x;
    if (slot >= min(ch.begin[c] + kChunk, a.n_slots[rep])) continue;
    if (slot < n_new) {
      R.id[slot] = R.id2[slot];
      R.cell[slot] = R.cell2[slot];
      if (R.speed) R.speed[slot] = R.speed2[slot];
      R.desired[slot] = (int32_t)R.mvinfo[slot];
    } else {
      R.cell[slot] = -1;
    }
  }
}

__global__ void k_bucket_commit(StepArgs a) {
  for (int r = threadIdx.x; r < a.n_rep; r += blockDim.x)
    a.n_slots[r] = (int)a.bucket_count[a.n_buckets + 2 + 2 * r];
}

int resort_launch(const StepArgs& a, const Chunks& ch, int grid, bool force, cudaStream_t s) {
  (void)force;
  if (ch.n <= 0) return 0;
  k_bucket_zero<<<256, 256, 0, s>>>(a);
  k_bucket_count<<<grid, kChunk, 0, s>>>(a, ch);
  const int nb = std::min(kScanMaxBlocks, std::max(1, (a.n_buckets + 4095) / 4096));
  k_bucket_scan_parts<<<nb, kScanThreads, 0, s>>>(a);
  k_bucket_scan_apply<<<nb, kScanThreads, 0, s>>>(a);
  k_bucket_scan_reps<<<1, 256, 0, s>>>(a);
  k_bucket_scatter<<<grid, kChunk, 0, s>>>(a, ch);
  k_bucket_copy<<<grid, kChunk, 0, s>>>(a, ch);
  k_bucket_commit<<<1, 256, 0, s>>>(a);
  return 0;
}

// ---------------------------------------------------------------------------
// Digests (splitmix64 output function of (id << 32 | value), summed).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_digest(StepArgs a, Chunks ch, int which) {
  const int idx = a.ctl->dig_count;
  if (idx >= a.dig_cap) return;
  unsigned long long* out = (which == 0 ? a.dig_cell : a.dig_des) + (int64_t)idx * a.n_rep;
  for (int c = blockIdx.x; c < ch.n; c += gridDim.x) {
    const int rep = ch.rep[c];
    const RepDev& R = a.reps[rep];
    const int slot = ch.begin[c] + threadIdx.x;
    if (slot >= min(ch.begin[c] + kChunk, a.n_slots[rep])) continue;
    const int cell = R.cell[slot];
    if (cell < 0) continue;
    const int v = which == 0 ? cell : R.desired[slot];
    atomicAdd(&out[rep], mix64(((unsigned long long)(uint32_t)R.id[slot] << 32) | (uint32_t)v));
  }
}

__global__ void k_digest_advance(StepArgs a) {
  if (threadIdx.x == 0) a.ctl->dig_count += 1;
}

int digest_des_launch(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s) {
  if (ch.n <= 0) return 0;
  k_digest<<<grid, kChunk, 0, s>>>(a, ch, 1);
  return 0;
}

int digest_cell_launch(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s) {
  if (ch.n > 0) k_digest<<<grid, kChunk, 0, s>>>(a, ch, 0);
  k_digest_advance<<<1, 32, 0, s>>>(a);
  return 0;
}

// ---------------------------------------------------------------------------
__global__ void k_gather_by_id(const RepDev* rp, const int32_t* n_slots, int rep, int cap,
                               int32_t* out_cell, int32_t* out_desired, int32_t bound) {
  const RepDev& R = *rp;
  const int n = min(n_slots[rep], cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = R.cell[i];
    if (c < 0) continue;
    const int id = R.id[i];
    if (id < 0 || id >= bound) continue;
    if (out_cell) out_cell[id] = c;
    if (out_desired) out_desired[id] = R.desired[i];
  }
}

int gather_by_id_launch(const RepDev* d, const int32_t* n_slots, int rep, int cap,
                        int32_t* out_cell, int32_t* out_desired, int32_t bound, cudaStream_t s) {
  const int blocks = cap > 0 ? (cap + 255) / 256 : 1;
  k_gather_by_id<<<blocks, 256, 0, s>>>(d, n_slots, rep, cap, out_cell, out_desired, bound);
  return 0;
}

// Number of distinct cells whose record one planning pass reads: the own cell
// of every agent and every in-grid, line-of-sight offset of its reach set.
__global__ void k_union_mark(const RepDev* rp, const int32_t* n_slots, int rep, int cap,
                             uint32_t* bitmap) {
  const RepDev& R = *rp;
  const int n = min(n_slots[rep], cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = R.cell[i];
    if (c < 0) continue;
    const int v = R.speed ? (int)R.speed[i] : R.v;
    int K = 0;
    for (int dy = -v; dy <= v; ++dy)
      for (int dx = -v; dx <= v; ++dx) K += reach_in(dx, dy, v, R.reach) ? 1 : 0;
    const int mw = K > 64 ? 2 : 1;
    const unsigned long long* mk = R.mask_v[v - 1];
    const unsigned long long m0 = mk[(size_t)c * mw];
    const unsigned long long m1 = mw > 1 ? mk[(size_t)c * mw + 1] : 0ull;
    int k = 0;
    for (int dy = -v; dy <= v; ++dy)
      for (int dx = -v; dx <= v; ++dx) {
        if (!reach_in(dx, dy, v, R.reach)) continue;
        const bool bit = k < 64 ? ((m0 >> k) & 1ull) : ((m1 >> (k - 64)) & 1ull);
        if (bit) {
          const int64_t cc = (int64_t)c + (int64_t)dy * R.W + dx;
          atomicOr(&bitmap[cc >> 5], 1u << (cc & 31));
        }
        ++k;
      }
  }
}

__global__ void k_union_pop(const uint32_t* bitmap, int64_t words, unsigned long long* out) {
  unsigned long long s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words;
       i += (int64_t)gridDim.x * blockDim.x)
    s += __popc(bitmap[i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

int union_count_launch(const RepDev* d, const int32_t* n_slots, int rep, int cap, int v,
                       int reach, int W, int H, uint32_t* bitmap, unsigned long long* out,
                       cudaStream_t s) {
  (void)v;
  (void)reach;
  const int64_t words = ((int64_t)W * H + 31) / 32;
  cudaMemsetAsync(bitmap, 0, (size_t)words * 4, s);
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  k_union_mark<<<cap > 0 ? (cap + 255) / 256 : 1, 256, 0, s>>>(d, n_slots, rep, cap, bitmap);
  k_union_pop<<<1024, 256, 0, s>>>(bitmap, words, out);
  return 0;
}

// ---------------------------------------------------------------------------
// Self-test kernels.
__global__ void k_test_exp64(const double* x, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = exp64(x[i]);
}

int test_exp64_launch(const double* x, double* y, int64_t n, cudaStream_t s) {
  k_test_exp64<<<1024, 256, 0, s>>>(x, y, n);
  return 0;
}

__global__ void k_test_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const U4 r = philox10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], key[2 * i],
                          key[2 * i + 1]);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
  }
}

int test_philox_launch(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                       cudaStream_t s) {
  k_test_philox<<<256, 256, 0, s>>>(ctr, key, out, n);
  return 0;
}

// Largest relative error of ex2.approx.ftz.f32 over every float in [lo, hi],
// against the FP64 exponential of this file (exp64(y * ln 2)), as float bits.
__global__ void k_test_ex2(float lo, float hi, unsigned long long* out) {
  const int32_t blo = __float_as_int(lo), bhi = __float_as_int(hi);
  double worst = 0.0;
  // walk the float bit patterns between lo and hi (both of one sign handled
  // by the host splitting the range at zero)
  const int64_t n = (int64_t)bhi - blo + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float y = __int_as_float((int32_t)(blo + i));
    const float e = ex2_approx(y);
    const double ref = exp64(__dmul_rn((double)y, 0x1.62e42fefa39efp-1));
    const double rel = fabs(((double)e - ref) / ref);
    worst = fmax(worst, rel);
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(worst));
}

int test_ex2_launch(float lo, float hi, unsigned long long* out, cudaStream_t s) {
  k_test_ex2<<<1024, 256, 0, s>>>(lo, hi, out);
  return 0;
}

// One index check of the debug build (the index is not used for any access).
__global__ void k_test_bounds(Ctl* ctl, long long index, long long n) {
  if (blockIdx.x == 0 && threadIdx.x == 0) (void)fg_in(ctl, index, n);
}

int test_bounds_launch(Ctl* ctl, long long index, long long n, cudaStream_t s) {
  k_test_bounds<<<1, 32, 0, s>>>(ctl, index, n);
  return 0;
}

int build_checked() { return kChecked ? 1 : 0; }

// L2 read bandwidth: every thread reads 16-byte words of a buffer that fits
// in L2 at global (L2) level, `iters` passes; the xor of what it read keeps
// the loads from being dropped.
__global__ void k_test_l2_read(const uint4* buf, size_t n16, int iters, unsigned int* sink) {
  uint32_t acc = 0u;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int it = 0; it < iters; ++it)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += stride) {
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);
}

int test_l2_read_launch(const void* buf, size_t bytes, int iters, unsigned int* sink, int grid,
                        cudaStream_t s) {
  k_test_l2_read<<<grid, 512, 0, s>>>(static_cast<const uint4*>(buf), bytes / 16, iters, sink);
  return 0;
}

}  // namespace fastgb
