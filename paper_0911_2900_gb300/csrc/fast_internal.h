// fast_internal.h -- declarations shared by the host API (api.cpp) and the
// CUDA translation units of libfastgb.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace fastgb {

enum { REACH_L2 = 0, REACH_L2P = 1, REACH_LINF = 2 };
enum { PREC_FP64 = 0, PREC_FP32_RECHECK = 1, PREC_FP32_NORECHECK = 2 };

constexpr int kMaxRep = 256;        // replicates per context (8-bit field in work refs)
constexpr int kMaxIdBits = 24;      // agent ids < 2^24 (movement priority layout)
constexpr int kChunk = 256;         // agents per work chunk
constexpr int kMaxK = 121;          // largest reach set (L-infinity, v_m = 5)
constexpr int kDevErrTimeout = 5;   // device error: a bounded wait gave up
constexpr int kDevErrRounds = 6;    // device error: movement rounds exceeded the bound
constexpr int kDevErrBounds = 9;    // device error (debug build): an index out of range
constexpr int kRoundLog = 64;       // movement rounds recorded per step
constexpr int kMoveThreads = 512;   // threads per block of the movement rounds (2 per SM)
constexpr int kMoveSmemCap = 4500;  // movers per block kept in shared memory (24 B each)

// One mover of the current step (16 bytes): start cell, (replicate << 24 |
// slot), movement priority, footprint info.
struct alignas(16) MoveEntry {
  uint32_t c0;
  uint32_t ref;
  uint32_t prio;
  uint32_t info;
};

// Per-replicate descriptor, resident in device memory.
struct RepDev {
  int32_t W, H, v, reach, K, mw;    // mw: 64-bit mask words per cell (1 or 2)
  int32_t cap;                      // agent slots allocated
  int32_t tile_shift;               // re-sort buckets are 2^tile_shift square tiles
  int32_t tiles_x, tiles_y;         // tiles per row / column
  int32_t bucket_base, bucket_span; // this replicate's range in the bucket arrays
  int32_t claim_tx;                 // 16x16 tiles per row of the claim arrays
  float c32;                        // fl32(-k_S * log2(e))
  float margin;                     // relative margin M of the FP32 decision
  double kS;
  uint32_t seed_lo, seed_hi;
  uint32_t* rec;                    // [W*H] cell records
  unsigned long long* mask;         // [W*H*mw] line-of-sight masks
  uint32_t* claim[2];               // movement claims: round tag << 24 | priority,
                                    // tile-major (16x16-cell tiles of 1 KB)
  uint8_t* cmark;                   // same layout: stamp of the last step in which an
                                    // agent lost the cell's first-round claim
  int32_t* id;                      // [cap]
  int32_t* cell;                    // [cap]  -1: slot empty / agent left
  int32_t* desired;                 // [cap]
  int32_t* id2;                     // [cap]  re-sort buffers
  int32_t* cell2;                   // [cap]
  uint32_t* mvinfo;                 // [cap]  scratch of the re-sort (desired cells)
  // maximum speed per agent (Sec. 2's benchmark gives every agent the same
  // one; the model allows one per agent): speed[slot] in 1..5, or nullptr
  // when every agent has speed v.  Speed classes are re-sorted apart.
  uint8_t* speed;                   // [cap]
  uint8_t* speed2;                  // [cap]  re-sort buffer
  unsigned long long* mask_v[5];    // line-of-sight masks per speed (mask_v[v-1] == mask),
                                    // K(s) > 64 ? 2 : 1 words per cell; nullptr if unused
  float margin_v[5];                // margin M of the FP32 decision per speed
};

// Step-wide control block, resident in device memory.
struct Ctl {
  int32_t t;                  // step index of the next step
  int32_t err;                // first device error (0 = none)
  uint32_t q_count;           // FP64 re-check queue length, this step
  uint32_t act_count[3];      // [2]: movers this step
  int32_t rounds_last;        // movement rounds of the last step
  int32_t rounds_max;
  int32_t resort_period;      // re-sort agents every this many steps (0: never)
  int32_t digests_on;
  int32_t dig_count;          // digests written
  uint32_t tail_count;        // waiting movers handed to one block, this step
  uint32_t claim_tag;         // tag of the next step's first movement claims
  uint32_t tag_reserve;       // clear the claims before a step with fewer tags left
  uint32_t mark_stamp;        // this step's stamp for contested-cell marks (1..254)
  uint32_t pad3;
  unsigned long long rounds_total;
  unsigned long long rechecked_total;
  unsigned long long agent_steps;
  unsigned long long barrier_ns_limit;
  unsigned long long flips;          // diagnostics
  unsigned long long flips_unflagged;
  unsigned long long flagged;
  unsigned int max_dp_bits;          // float bits of max |p32 - p64|
  unsigned int flips_after;          // choices of the FP32 + FP64 re-check pass != FP64 rule
  unsigned long long tile_fallbacks; // planning warps whose agents did not fit a tile
  long long bad_index;               // debug build: the first index found out of range
  unsigned long long movers_total;   // movers handed to the movement rounds, all steps
  unsigned long long foot_total;     // their footprint cells, all steps
  // movement instrumentation of the last step: agents still waiting after
  // each round's claims, and the global timer at the start of each round
  uint32_t round_n[kRoundLog];
  unsigned long long round_ns[kRoundLog + 1];
  // per-phase timings of the last step's movement rounds (max over blocks, ns)
  unsigned long long phase_ns[8];
  // most movers still waiting in one block after each round, last step
  uint32_t round_bmax[kRoundLog];
  // grid barrier words of odd and even barriers, each on a line of its own:
  // arrivals during the running launch (low half), running sum of the
  // counts the blocks bring (high half)
  alignas(128) unsigned long long bar_acc[2][16];
};

struct Chunks {
  const int32_t* rep;    // [n]
  const int32_t* begin;  // [n]
  int32_t n;
};

struct StepArgs {
  RepDev* reps;          // [n_rep] device
  int32_t n_rep;
  Ctl* ctl;              // device
  int32_t* n_slots;      // [n_rep] slots in use (agents, alive or not yet compacted)
  int32_t* exited;       // [n_rep] agents that left through an exit, total
  uint32_t* queue;       // [q_cap] FP64 re-check queue (rep << 24 | slot)
  uint32_t q_cap;
  MoveEntry* act[3];     // [2]: movers of the step; [0]: movers one block finishes
  uint32_t act_cap;
  // movement state when a block's movers do not fit its shared memory
  uint32_t *mv_prio, *mv_c0, *mv_ref, *mv_info, *mv_list[3];
  unsigned long long* dig_cell;  // [dig_cap * n_rep] per-step digests (optional)
  unsigned long long* dig_des;
  int32_t dig_cap;
  // re-sort scratch: [n_buckets + 1] offsets, 2 words per replicate, then the
  // scan's block sums (up to 1024)
  uint32_t* bucket_count;
  int32_t n_buckets;
  // diagnostics
  float* diag_p32;         // [total slots * kMaxK] FP32 cumulative probabilities
  int32_t* diag_choice32;  // [total slots]
  uint8_t* diag_flag;      // [total slots]
  int64_t* diag_base;      // [n_rep] offset of each replicate's slots in the diag arrays
};

// ---- launch wrappers (defined in the .cu files) ---------------------------
int plan_groups_launch(const StepArgs& a, int v, int reach, int lanes, int precision,
                       const Chunks& ch, int grid, cudaStream_t s, bool diag);
int plan_recheck_launch(const StepArgs& a, int grid, cudaStream_t s);
int plan_diag_compare_launch(const StepArgs& a, int v, int reach, const Chunks& ch, int grid,
                             cudaStream_t s);
int move_prep_launch(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s);
int move_rounds_launch(const StepArgs& a, int grid, int block, cudaStream_t s);
int move_rounds_max_grid(int block, int* grid_out);
int step_end_launch(const StepArgs& a, cudaStream_t s);
int step_begin_launch(const StepArgs& a, cudaStream_t s);
int digest_des_launch(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s);
int digest_cell_launch(const StepArgs& a, const Chunks& ch, int grid, cudaStream_t s);
int resort_launch(const StepArgs& a, const Chunks& ch, int grid, bool force, cudaStream_t s);
int masks_launch(const RepDev& host_rep, RepDev* dev_rep, int64_t cells, cudaStream_t s);
int masks_speed_launch(RepDev* dev_rep, int64_t cells, int v, int mw, unsigned long long* out,
                       cudaStream_t s);
int clear_occ_launch(RepDev* dev_rep, const int32_t* n_slots_dev, int rep, int cap,
                     int32_t* slot_of_id, int n_ids, cudaStream_t s);
int place_checked_launch(RepDev* dev_rep, const int32_t* cells, const int32_t* ids, int n,
                         long long n_cells, uint32_t* id_bits, uint8_t* placed,
                         const uint8_t* speed_by_id, int n_speed_ids, const int32_t* slot_of_id,
                         const int32_t* n_slots_old, int32_t* err, cudaStream_t s);
int place_rollback_launch(RepDev* dev_rep, const int32_t* cells, int n, const uint8_t* placed,
                          cudaStream_t s);
// Batched placement and read-back, one entry per replicate (uploaded by the
// host for one call).
struct BatchRep {
  long long off;               // its first agent in the staged or gathered arrays
  int32_t n;                   // its ids 0..n-1; -1: not placed by this call
  int32_t keep;                // 1: agents go back to the slots their ids hold
  int32_t clear;               // 1: its previous agents are cleared first
  int32_t n_speed_ids;
  const uint8_t* speed_by_id;  // nullptr: no speeds per agent
};
int batch_prepare_launch(RepDev* reps, const Chunks& ch, const BatchRep* bp, int grid,
                         cudaStream_t s);
int batch_clear_launch(RepDev* reps, const int32_t* n_slots, const Chunks& ch, const BatchRep* bp,
                       int grid, cudaStream_t s);
int batch_place_launch(RepDev* reps, const int32_t* staged, long long total, const BatchRep* bp,
                       int n_rep, const int32_t* n_slots, int32_t* errs, int grid,
                       cudaStream_t s);
int batch_gather_launch(const RepDev* reps, const int32_t* n_slots, const Chunks& ch,
                        const BatchRep* bp, int32_t* out_cell, int32_t* out_des, int grid,
                        cudaStream_t s);
int gather_by_id_launch(const RepDev* dev_rep, const int32_t* n_slots_dev, int rep, int cap,
                        int32_t* out_cell, int32_t* out_desired, int32_t bound,
                        cudaStream_t s);
int union_count_launch(const RepDev* dev_rep, const int32_t* n_slots_dev, int rep, int cap,
                       int v, int reach, int W, int H, uint32_t* bitmap,
                       unsigned long long* out, cudaStream_t s);
int test_exp64_launch(const double* x, double* y, int64_t n, cudaStream_t s);
int test_philox_launch(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                       cudaStream_t s);
int test_ex2_launch(float lo, float hi, unsigned long long* out_max_rel_bits, cudaStream_t s);
int test_bounds_launch(Ctl* ctl, long long index, long long n, cudaStream_t s);
int build_checked();
int test_l2_read_launch(const void* buf, size_t bytes, int iters, unsigned int* sink, int grid,
                        cudaStream_t s);
int test_barrier_timeout_launch(Ctl* ctl, int grid, cudaStream_t s);
int test_barrier_cost_launch(Ctl* ctl, int grid, int block, int iters, cudaStream_t s);
int test_barrier_sum_launch(Ctl* ctl, int grid, int block, int iters, cudaStream_t s);
int noalloc_plan_launch(const RepDev& R, int32_t cap, int32_t t, int32_t* out, int32_t bound,
                        int sms, cudaStream_t s);
int noalloc_max_agents();

}  // namespace fastgb
