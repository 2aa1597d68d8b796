// api.cpp -- host side of libfastgb: the C ABI declared in include/fastgb.h.
//
// Owns the context (replicates, device buffers, work chunks, the captured
// CUDA graph of one step) and validates every input before anything reaches
// the GPU.  All arithmetic of the step runs in the kernels of plan.cu,
// move.cu and aux.cu; the host only computes the exact floor field at grid
// set-up (floor_field.cpp) and checks placements.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "fast_internal.h"
#include "fastgb.h"

namespace fastgb {
int64_t exact_floor_field(int32_t W, int32_t H, const uint8_t* type, int32_t* a, int32_t* b);
int64_t decompose_field(int32_t W, int32_t H, const uint8_t* type, const double* S, int32_t max_ab,
                        int32_t* a, int32_t* b);
}

using namespace fastgb;

namespace {

// Largest relative error of one SFU 2^y used in the FP32 margin (covers the
// measured maximum of ex2.approx.ftz.f32 over the argument range with a
// factor of two to spare; see the self test fast_selftest_ex2).
constexpr double kEx2RelErr = 0x1p-21;
constexpr int kDefaultLanes[5] = {1, 1, 1, 1, 1};  // 1: one thread per agent, records via L1
constexpr double kSqrt2 = 1.4142135623730951;
constexpr double kLn2 = 0.6931471805599453;
constexpr double kLog2e = 1.4426950408889634;

struct RepHost {
  bool grid_set = false;
  bool placed = false;
  int32_t W = 0, H = 0, v = 0, K = 0, mw = 1;
  double kS = 0.0;
  uint64_t seed = 0;
  int32_t cap = 0;                 // agent slots allocated
  int32_t n = 0;                   // agents placed
  int32_t n_ids = -1;              // ids of the last placement if they were implicit (0..n-1)
  std::vector<uint64_t> eligible;  // bit i: cell i may hold an agent (free, reachable)
  int64_t n_eligible = 0;
  uint32_t speed_set = 0;          // speeds given per agent (bit s-1: speed s), 0: all v
  uint8_t* d_speed_by_id = nullptr;  // device copy of the speeds by id
  int32_t n_speed_ids = 0;
  RepDev d{};                      // device pointers and parameters
};

// Pinned staging of the batched calls: BatchRep per replicate, then error
// words (3), slot counts and exit counts per replicate, then 16 spare words.
constexpr size_t kBatchHostBytes = sizeof(BatchRep) * kMaxRep + 4 * 5 * kMaxRep + 64;

// Speeds whose planning launch covers this replicate.
uint32_t speeds_of(const RepHost& R) { return R.speed_set ? R.speed_set : 1u << (R.v - 1); }

}  // namespace

struct fast_ctx {
  int32_t n_rep = 0, precision = 0, reach = 0;
  cudaStream_t stream = nullptr;      // the caller's stream: all work runs here
  cudaStream_t cap_stream = nullptr;  // private stream the step graph is captured on
  cudaStream_t cur = nullptr;         // where enqueue_* put their work
  fast_alloc_fn alloc = nullptr;
  fast_free_fn release = nullptr;
  void* user = nullptr;
  std::string err;
  bool poisoned = false;
  int sms = 0;
  std::vector<RepHost> reps;
  std::unordered_map<void*, size_t> live;  // allocations

  // device-resident shared state
  RepDev* d_reps = nullptr;
  Ctl* d_ctl = nullptr;
  int32_t* d_nslots = nullptr;
  int32_t* d_exited = nullptr;
  uint32_t* d_queue = nullptr;
  MoveEntry* d_act[3] = {nullptr, nullptr, nullptr};
  uint32_t* d_mv_prio = nullptr;
  Ctl* h_ctl = nullptr;      // pinned: a copy of the control block, then 16 words (an exit
                             // count read back with the data; placement's small copies)
  uint32_t* d_mv[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

  uint32_t list_cap = 0;
  uint32_t* d_bucket = nullptr;
  int32_t n_buckets = 0;
  size_t bucket_words = 0;
  unsigned long long* d_dig_cell = nullptr;
  unsigned long long* d_dig_des = nullptr;
  int32_t dig_cap = 0;
  int32_t* d_gather = nullptr;
  int32_t gather_cap = 0;
  uint32_t* d_id_bits = nullptr;  // 2^24-bit set of the ids a placement has seen
  int32_t* d_place_err = nullptr;  // placement check: first bad index, agents placed
  int32_t* d_stage = nullptr;      // fast_place_all: the uploaded cells of all replicates
  int64_t stage_cap = 0;

  struct Group {
    int v = 0;
    int n = 0;
    int32_t* d_rep = nullptr;
    int32_t* d_begin = nullptr;
  };
  std::vector<Group> groups;
  int32_t* d_all_rep = nullptr;
  int32_t* d_all_begin = nullptr;
  int all_n = 0;
  bool layout_dirty = true;

  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_state[2] = {0, 0};  // 0 not built, 1 built, 2 capture failed
  // step loops captured whole, keyed by (step index mod re-sort period, steps);
  // a null executable records a capture that failed
  struct Multi {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
  };
  std::map<std::pair<int, int>, Multi> multi;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_upload = nullptr;  // placement: the cells' upload on the private stream is done
  BatchRep* d_bp = nullptr;        // batched placement / read-back: per replicate
  int32_t* d_berr = nullptr;       // its per-replicate error words (3 each)
  char* h_batch = nullptr;         // pinned: BatchRep[kMaxRep], then 3+1+1 words per
                                   // replicate (errors, slots, exits), then 16 words
  bool ran_step = false;
  int64_t launches = 0;          // kernels queued by this context
  int launches_per_graph[2] = {0, 0};

  // options
  int resort_period = 8;
  bool digests = false;
  int lanes[5] = {1, 1, 1, 1, 1};
  long long barrier_ns = 2000000000ll;
  bool use_graph = true;
  int move_blocks = 0;
  int tile_shift = 4;
  int graph_steps = 512;  // longest step loop captured as one graph
  bool resort_pending = false;  // agents placed since the last spatial sort

  int64_t t_host = 0;
  int64_t steps_since_place = 0;
};

// ---------------------------------------------------------------------------
namespace {

int fail(fast_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (code == FAST_ECUDA || code == FAST_ETIMEOUT) c->poisoned = true;
  }
  return code;
}

#define CUDA_TRY(ctx, call)                                                               \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, FAST_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                              \
  } while (0)

#define LAUNCH_TRY(ctx, call)                                                        \
  do {                                                                               \
    (ctx)->launches += 1;                                                            \
    int r_ = (call);                                                                 \
    cudaError_t e_ = cudaGetLastError();                                             \
    if (r_ != 0 || e_ != cudaSuccess)                                                \
      return fail(ctx, FAST_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

void* dalloc(fast_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, c->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->live[p] = bytes;
  return p;
}

void dfree(fast_ctx* c, void* p) {
  if (!p) return;
  auto it = c->live.find(p);
  if (it == c->live.end()) return;
  c->live.erase(it);
  if (c->release)
    c->release(p, c->user);
  else
    cudaFree(p);
}

template <typename T>
int alloc_into(fast_ctx* c, T** out, size_t count) {
  *out = (T*)dalloc(c, count * sizeof(T));
  if (!*out) return fail(c, FAST_ENOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
  return FAST_OK;
}

int reach_count_host(int v, int reach) {
  int k = 0;
  for (int y = -v; y <= v; ++y)
    for (int x = -v; x <= v; ++x) {
      const int r2 = x * x + y * y;
      const bool in = reach == FAST_REACH_L2    ? r2 <= v * v
                      : reach == FAST_REACH_L2P ? r2 <= v * v + v
                                                : (std::abs(x) <= v && std::abs(y) <= v);
      k += in ? 1 : 0;
    }
  return k;
}

// Relative margin M of the FP32 decision (see the comment of k_plan_fp32).
// One weight 2^y, y = fl(fl(dS) * fl(-k_S log2 e)):
//   |dS32 - dS| <= 2^-23 (v sqrt2 + 0.002)       (exact integers a, b; sqrt2
//                                                  split in two floats)
//   |y32 - y|   <= |c| |dS32 - dS| + |y|max 2^-22  (constant and product rounding)
//   delta       = 2^{|y32 - y|} - 1 + e_ex2 + 2^-24
// A cumulative value is a sum of at most K such weights in some order:
//   gamma = (1 + delta)(1 + 2^-24)^K - 1.
// |C32/W32 - C*/W*| <= 2 gamma / (1 - gamma) for the FP32 side and 2A for the
// FP64 side (A = 1e-10 bounds the FP64 rule's own error against exact
// arithmetic); the test itself and the 24-bit float draw (|u - u24| < 2^-24)
// add 2^-21.  M doubles the sum.
float margin_of(int v, int K, double kS) {
  const double u24 = std::ldexp(1.0, -24);
  const double ds_err = std::ldexp(1.0, -23) * (v * kSqrt2 + 0.002);
  const double c = kS * kLog2e;
  const double ymax = c * v * kSqrt2;
  const double y_err = c * ds_err + ymax * std::ldexp(1.0, -22);
  const double delta = std::expm1(kLn2 * y_err) + kEx2RelErr + u24;
  const double gamma = (1.0 + delta) * std::pow(1.0 + u24, K) - 1.0;
  const double A = 1e-10;
  const double M = 2.0 * (4.0 * gamma / (1.0 - gamma) + std::ldexp(1.0, -21) + 2.0 * A);
  return (float)M;
}

bool rep_ok(fast_ctx* c, int32_t r) { return c && r >= 0 && r < c->n_rep; }

int upload_reps(fast_ctx* c) {
  std::vector<RepDev> h(c->n_rep);
  for (int r = 0; r < c->n_rep; ++r) h[r] = c->reps[r].d;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_reps, h.data(), sizeof(RepDev) * c->n_rep,
                              cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FAST_OK;
}

void drop_graphs(fast_ctx* c) {
  for (int i = 0; i < 2; ++i) {
    if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
    c->graph[i] = nullptr;
    c->graph_state[i] = 0;
  }
  for (auto& kv : c->multi)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  c->multi.clear();
}

// (Re)allocates a replicate's per-slot arrays for cap >= n slots.
int realloc_slots(fast_ctx* c, RepHost& R, int32_t n) {
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int32_t cap = std::max(n, std::max(R.cap, 1));
  int32_t* arrs[] = {R.d.id, R.d.cell, R.d.desired, R.d.id2, R.d.cell2};
  for (auto p : arrs) dfree(c, p);
  dfree(c, R.d.mvinfo);
  dfree(c, R.d.speed);
  dfree(c, R.d.speed2);
  R.d.id = R.d.cell = R.d.desired = R.d.id2 = R.d.cell2 = nullptr;
  R.d.mvinfo = nullptr;
  R.d.speed = R.d.speed2 = nullptr;
  // no agents until the new arrays are in place (an allocation that fails
  // below leaves the replicate empty and out of the work lists)
  R.placed = false;
  R.n = 0;
  R.n_ids = -1;
  R.cap = 0;
  R.d.cap = 0;
  c->layout_dirty = true;
  if (int e = alloc_into(c, &R.d.id, cap)) return e;
  if (int e = alloc_into(c, &R.d.cell, cap)) return e;
  if (int e = alloc_into(c, &R.d.desired, cap)) return e;
  if (int e = alloc_into(c, &R.d.id2, cap)) return e;
  if (int e = alloc_into(c, &R.d.cell2, cap)) return e;
  if (int e = alloc_into(c, &R.d.mvinfo, cap)) return e;
  if (R.speed_set) {
    if (int e = alloc_into(c, &R.d.speed, cap)) return e;
    if (int e = alloc_into(c, &R.d.speed2, cap)) return e;
  }
  R.cap = cap;
  R.d.cap = cap;
  c->layout_dirty = true;
  return FAST_OK;
}

// Work chunks (replicate, first slot) per v_m group and over all replicates;
// re-sort bucket ranges; shared lists sized for all agent slots.
int rebuild_layout(fast_ctx* c) {
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  for (auto& g : c->groups) {
    dfree(c, g.d_rep);
    dfree(c, g.d_begin);
  }
  c->groups.clear();
  dfree(c, c->d_all_rep);
  dfree(c, c->d_all_begin);
  c->d_all_rep = c->d_all_begin = nullptr;

  std::vector<int32_t> all_r, all_b;
  uint64_t total_cap = 0;
  int64_t bucket_base = 0;
  for (int r = 0; r < c->n_rep; ++r) {
    RepHost& R = c->reps[r];
    if (!R.grid_set) continue;
    const int ts = c->tile_shift;
    const int tx = (R.W + (1 << ts) - 1) >> ts, ty = (R.H + (1 << ts) - 1) >> ts;
    int side = 1;
    while (side < std::max(tx, ty)) side <<= 1;
    R.d.tile_shift = ts;
    R.d.tiles_x = tx;
    R.d.tiles_y = ty;
    R.d.bucket_base = (int32_t)bucket_base;
    R.d.bucket_span = side * side;
    bucket_base += (int64_t)side * side * (R.d.speed ? 5 : 1);  // speed classes
    if (!R.placed) continue;
    total_cap += (uint64_t)R.cap;
    for (int b = 0; b < R.cap; b += kChunk) {
      all_r.push_back(r);
      all_b.push_back(b);
    }
  }
  if (bucket_base > (int64_t)1 << 30)
    return fail(c, FAST_EINVAL, "too many re-sort buckets (%lld); raise the tile shift",
                (long long)bucket_base);
  for (int v = 1; v <= 5; ++v) {
    std::vector<int32_t> gr, gb;
    for (int r = 0; r < c->n_rep; ++r) {
      RepHost& R = c->reps[r];
      if (!R.grid_set || !R.placed || !((speeds_of(R) >> (v - 1)) & 1u)) continue;
      for (int b = 0; b < R.cap; b += kChunk) {
        gr.push_back(r);
        gb.push_back(b);
      }
    }
    if (gr.empty()) continue;
    fast_ctx::Group g;
    g.v = v;
    g.n = (int)gr.size();
    if (int e = alloc_into(c, &g.d_rep, gr.size())) return e;
    if (int e = alloc_into(c, &g.d_begin, gb.size())) return e;
    CUDA_TRY(c, cudaMemcpy(g.d_rep, gr.data(), gr.size() * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(g.d_begin, gb.data(), gb.size() * 4, cudaMemcpyHostToDevice));
    c->groups.push_back(g);
  }
  c->all_n = (int)all_r.size();
  if (c->all_n > 0) {
    if (int e = alloc_into(c, &c->d_all_rep, all_r.size())) return e;
    if (int e = alloc_into(c, &c->d_all_begin, all_b.size())) return e;
    CUDA_TRY(c, cudaMemcpy(c->d_all_rep, all_r.data(), all_r.size() * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_all_begin, all_b.data(), all_b.size() * 4,
                           cudaMemcpyHostToDevice));
  }
  if (total_cap > c->list_cap) {
    dfree(c, c->d_queue);
    dfree(c, c->d_act[2]);
    dfree(c, c->d_act[0]);
    dfree(c, c->d_mv_prio);
    for (auto& p : c->d_mv) dfree(c, p);
    const size_t n = (size_t)total_cap;
    if (int e = alloc_into(c, &c->d_queue, n)) return e;
    if (int e = alloc_into(c, &c->d_act[2], n)) return e;
    if (int e = alloc_into(c, &c->d_act[0], n)) return e;
    if (int e = alloc_into(c, &c->d_mv_prio, n)) return e;
    for (auto& p : c->d_mv)
      if (int e = alloc_into(c, &p, n)) return e;
    c->list_cap = (uint32_t)total_cap;
  }
  // bucket offsets, 2 words per replicate, the scan's block sums (<= 1024)
  const size_t words = (size_t)bucket_base + 1 + 2 * (size_t)c->n_rep + 1024;
  if (words > c->bucket_words) {
    dfree(c, c->d_bucket);
    c->d_bucket = nullptr;
    if (int e = alloc_into(c, &c->d_bucket, words)) return e;
    c->bucket_words = words;
  }
  c->n_buckets = (int32_t)bucket_base;
  if (int e = upload_reps(c)) return e;
  c->layout_dirty = false;
  return FAST_OK;
}

StepArgs args_of(fast_ctx* c) {
  StepArgs a{};
  a.reps = c->d_reps;
  a.n_rep = c->n_rep;
  a.ctl = c->d_ctl;
  a.n_slots = c->d_nslots;
  a.exited = c->d_exited;
  a.queue = c->d_queue;
  a.q_cap = c->list_cap;
  for (int i = 0; i < 3; ++i) {
    a.act[i] = c->d_act[i];
    a.mv_list[i] = c->d_mv[3 + i];
  }
  a.mv_prio = c->d_mv_prio;
  a.mv_c0 = c->d_mv[0];
  a.mv_ref = c->d_mv[1];
  a.mv_info = c->d_mv[2];
  a.act_cap = c->list_cap;
  a.dig_cell = c->d_dig_cell;
  a.dig_des = c->d_dig_des;
  a.dig_cap = c->dig_cap;
  a.bucket_count = c->d_bucket;
  a.n_buckets = c->n_buckets;
  return a;
}

Chunks all_chunks(fast_ctx* c) { return Chunks{c->d_all_rep, c->d_all_begin, c->all_n}; }

int plan_grid(fast_ctx* c, int n_chunks) { return std::max(1, std::min(n_chunks, c->sms * 8)); }

// Cooperative grid of the movement rounds: every block that can be resident
// (the rounds are latency-bound), capped by the work and by the option.
int move_grid(fast_ctx* c) {
  int g = 0;
  if (move_rounds_max_grid(kMoveThreads, &g) != 0 || g <= 0) g = c->sms;
  if (c->move_blocks > 0) g = std::min(g, c->move_blocks);
  return std::max(g, 1);
}

int link_grid(fast_ctx* c) {
  return std::max(1, std::min((int)((c->list_cap + 255) / 256), c->sms * 8));
}

// Inside a capture the record must be an external event-record node, so that
// the event is really recorded each time the graph is replayed.
cudaError_t record_event(fast_ctx* c, int i) {
  return cudaEventRecordWithFlags(c->ev[i], c->cur,
                                  c->cur == c->cap_stream ? cudaEventRecordExternal : 0);
}

int enqueue_plan(fast_ctx* c, const StepArgs& a, bool diag, bool events) {
  for (auto& g : c->groups) {
    Chunks ch{g.d_rep, g.d_begin, g.n};
    LAUNCH_TRY(c, plan_groups_launch(a, g.v, c->reach, c->lanes[g.v - 1], c->precision, ch,
                                     plan_grid(c, g.n), c->cur, diag));
  }
  if (events) CUDA_TRY(c, record_event(c, 1));
  if (c->precision == FAST_FP32_RECHECK && !diag)
    LAUNCH_TRY(c, plan_recheck_launch(a, std::max(1, c->sms * 16), c->cur));
  return FAST_OK;
}

// One step: planning kernels | FP64 re-check | movement footprints |
// movement rounds | bookkeeping; events ev[0..5] bracket the five parts.
int enqueue_step(fast_ctx* c, bool resort) {
  const StepArgs a = args_of(c);
  const Chunks all = all_chunks(c);
  CUDA_TRY(c, record_event(c, 0));
  if (int e = enqueue_plan(c, a, false, true)) return e;
  CUDA_TRY(c, record_event(c, 2));
  if (c->digests) LAUNCH_TRY(c, digest_des_launch(a, all, plan_grid(c, all.n), c->cur));
  LAUNCH_TRY(c, move_prep_launch(a, all, plan_grid(c, all.n), c->cur));
  CUDA_TRY(c, record_event(c, 3));
  LAUNCH_TRY(c, move_rounds_launch(a, move_grid(c), kMoveThreads, c->cur));
  CUDA_TRY(c, record_event(c, 4));
  if (c->digests) {
    LAUNCH_TRY(c, digest_cell_launch(a, all, plan_grid(c, all.n), c->cur));
    c->launches += 1;  // digest_cell_launch queues two kernels
  }
  if (resort) {
    LAUNCH_TRY(c, resort_launch(a, all, plan_grid(c, all.n), false, c->cur));
    c->launches += 7;  // resort_launch queues eight kernels
  }
  LAUNCH_TRY(c, step_end_launch(a, c->cur));
  CUDA_TRY(c, record_event(c, 5));
  return FAST_OK;
}

// Captures one step on the private stream; the graph is then replayed on the
// caller's stream.  If capture is not possible, steps are queued directly.
int build_graph(fast_ctx* c, int which) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    c->graph_state[which] = 2;
    return FAST_OK;
  }
  c->cur = c->cap_stream;
  const int64_t before = c->launches;
  const std::string err_before = c->err;
  const int e = enqueue_step(c, which == 1);
  c->cur = c->stream;
  c->launches_per_graph[which] = (int)(c->launches - before);
  c->launches = before;
  cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != FAST_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    c->poisoned = false;  // capture failure: fall back to direct launches
    c->err = err_before;
    c->graph_state[which] = 2;
    return FAST_OK;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    c->graph_state[which] = 2;
    return FAST_OK;
  }
  cudaGraphDestroy(g);
  c->graph[which] = ex;
  c->graph_state[which] = 1;
  return FAST_OK;
}

// Captures the next n steps (re-sorts where the step index calls for one) as
// one graph; on any capture failure the entry stays null and steps are
// queued one graph at a time instead.
int build_multi(fast_ctx* c, int n, fast_ctx::Multi* out) {
  out->exec = nullptr;
  out->launches = 0;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return FAST_OK;
  }
  c->cur = c->cap_stream;
  const int64_t before = c->launches;
  const std::string err_before = c->err;
  int e = FAST_OK;
  for (int i = 0; i < n && e == FAST_OK; ++i) {
    const int64_t t = c->t_host + i;
    e = enqueue_step(c, c->resort_period > 0 && ((t + 1) % c->resort_period == 0));
  }
  c->cur = c->stream;
  out->launches = (int)(c->launches - before);
  c->launches = before;
  cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != FAST_OK || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    c->poisoned = false;
    c->err = err_before;
    return FAST_OK;
  }
  if (cudaGraphInstantiate(&out->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    out->exec = nullptr;
  }
  cudaGraphDestroy(g);
  return FAST_OK;
}

int write_ctl_int(fast_ctx* c, size_t offset, int32_t v) {
  CUDA_TRY(c, cudaMemcpyAsync((char*)c->d_ctl + offset, &v, 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FAST_OK;
}

// The error a copy of the control block records, as the call's result.
int device_error_of(fast_ctx* c, const Ctl& h) {
  if (h.err == kDevErrTimeout)
    return fail(c, FAST_ETIMEOUT, "a device-side wait exceeded its limit (%lld ns)",
                (long long)c->barrier_ns);
  if (h.err == kDevErrBounds)
    return fail(c, FAST_ECUDA, "a kernel found index %lld out of range (debug build)",
                (long long)h.bad_index);
  if (h.err != 0) return fail(c, FAST_ECUDA, "device error code %d", h.err);
  return FAST_OK;
}

int check_device_error(fast_ctx* c) {
  Ctl h{};
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  CUDA_TRY(c, cudaMemcpy(&h, c->d_ctl, sizeof h, cudaMemcpyDeviceToHost));
  return device_error_of(c, h);
}

}  // namespace

namespace {
// Views of the pinned staging of the batched calls.
struct BatchHost {  // views of the pinned staging of the batched calls
  BatchRep* bp;
  int32_t *err, *slots, *exited, *misc;
};
BatchHost batch_host(fast_ctx* c) {
  BatchHost h;
  h.bp = reinterpret_cast<BatchRep*>(c->h_batch);
  h.err = reinterpret_cast<int32_t*>(c->h_batch + sizeof(BatchRep) * kMaxRep);
  h.slots = h.err + 3 * kMaxRep;
  h.exited = h.slots + kMaxRep;
  h.misc = h.exited + kMaxRep;
  return h;
}
int batch_buffers(fast_ctx* c) {
  if (c->d_bp) return FAST_OK;
  if (int e = alloc_into(c, &c->d_bp, kMaxRep)) return e;
  return alloc_into(c, &c->d_berr, 3 * kMaxRep);
}
}  // namespace

namespace {
// Seeded uniform placement: n distinct cells drawn uniformly from the
// replicate's eligible cells (free, reachable, not an exit) in one pass of
// selection sampling (Knuth's Algorithm S: keep a cell with probability
// needed / left), then handed to ids 0..n-1 in a random order (Fisher-Yates
// shuffle).  Both draw from one splitmix64 stream (Steele, Lea and Flood's
// generator) started from the grid's seed, so one (grid, seed, n) always
// gives one placement.  Requires n <= R.n_eligible.
void uniform_cells(const RepHost& R, int32_t n, std::vector<int32_t>& out) {
  uint64_t state = R.seed;
  auto next = [&state]() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  out.clear();
  out.reserve((size_t)n);
  int64_t left = R.n_eligible, need = n;
  for (size_t w = 0; w < R.eligible.size() && need > 0; ++w) {
    uint64_t bits = R.eligible[w];
    while (bits && need > 0) {
      const int64_t i = (int64_t)(w << 6) + __builtin_ctzll(bits);
      bits &= bits - 1;
      const double u = (double)(next() >> 11) * 0x1.0p-53;  // uniform in [0, 1)
      if (u * (double)left < (double)need) {
        out.push_back((int32_t)i);
        --need;
      }
      --left;
    }
  }
  for (int64_t k = (int64_t)out.size() - 1; k > 0; --k)
    std::swap(out[(size_t)k], out[(size_t)(next() % (uint64_t)(k + 1))]);
}
}  // namespace

// ===========================================================================
extern "C" {

// Queues the spatial sort that placements leave pending (one for any number
// of fast_place_agents calls in a row).
int sort_if_pending(fast_ctx* c) {
  if (!c->resort_pending) return FAST_OK;
  const StepArgs a = args_of(c);
  const Chunks all = all_chunks(c);
  LAUNCH_TRY(c, resort_launch(a, all, plan_grid(c, all.n), true, c->stream));
  c->launches += 7;
  c->resort_pending = false;
  return FAST_OK;
}

static int create_impl(fast_ctx* c, int32_t n_replicates);

int fast_create(fast_ctx** out, int32_t n_replicates, int32_t precision, int32_t reach,
                void* cuda_stream, fast_alloc_fn dev_alloc, fast_free_fn dev_free,
                void* alloc_user) {
  if (!out) return FAST_EINVAL;
  *out = nullptr;
  if (n_replicates < 1 || n_replicates > kMaxRep) return FAST_EINVAL;
  if (precision < FAST_FP64 || precision > FAST_FP32_NORECHECK) return FAST_EINVAL;
  if (reach < FAST_REACH_L2 || reach > FAST_REACH_LINF) return FAST_EINVAL;
  if ((dev_alloc == nullptr) != (dev_free == nullptr)) return FAST_EINVAL;
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return FAST_ECUDA;
  }
  fast_ctx* c = new fast_ctx();
  c->n_rep = n_replicates;
  c->precision = precision;
  c->reach = reach;
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = dev_alloc;
  c->release = dev_free;
  c->user = alloc_user;
  c->reps.resize(n_replicates);
  for (int i = 0; i < 5; ++i) c->lanes[i] = kDefaultLanes[i];
  const int rc = create_impl(c, n_replicates);
  if (rc != FAST_OK) {
    fast_destroy(c);
    return rc;
  }
  *out = c;
  (void)dev;
  return FAST_OK;
}

static int create_impl(fast_ctx* c, int32_t n_replicates) {
  int dev = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  CUDA_TRY(c, cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
  if (int e = alloc_into(c, &c->d_reps, n_replicates)) return e;
  if (int e = alloc_into(c, &c->d_ctl, 1)) return e;
  if (int e = alloc_into(c, &c->d_nslots, n_replicates)) return e;
  if (int e = alloc_into(c, &c->d_exited, n_replicates)) return e;
  for (auto& ev : c->ev) CUDA_TRY(c, cudaEventCreate(&ev));
  CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  CUDA_TRY(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_ctl), sizeof(Ctl) + 64));
  CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_upload, cudaEventDisableTiming));
  CUDA_TRY(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_batch), kBatchHostBytes));
  c->cur = c->stream;
  Ctl h{};
  h.resort_period = c->resort_period;
  h.barrier_ns_limit = (unsigned long long)c->barrier_ns;
  h.tag_reserve = 96;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_ctl, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_nslots, 0, 4 * n_replicates, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_exited, 0, 4 * n_replicates, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FAST_OK;
}

int fast_init_grid(fast_ctx* c, int32_t r, const fast_grid_desc* g) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!rep_ok(c, r) || !g) return fail(c, FAST_EINVAL, "bad replicate index or NULL grid");
  if (g->width < 1 || g->height < 1 || g->width > 65535 || g->height > 65535 ||
      (int64_t)g->width * g->height >= ((int64_t)1 << 31))
    return fail(c, FAST_EINVAL, "grid %d x %d out of range", g->width, g->height);
  if (!g->cell_type) return fail(c, FAST_EINVAL, "cell_type is NULL");
  if (g->v_m < 1 || g->v_m > 5) return fail(c, FAST_EINVAL, "v_m = %d not in 1..5", g->v_m);
  if (!(g->k_S >= 0.0) || !std::isfinite(g->k_S))
    return fail(c, FAST_EINVAL, "k_S must be finite and >= 0");
  const double span = g->k_S * g->v_m * kSqrt2;
  if (c->precision != FAST_FP64 && span * kLog2e > 120.0)
    return fail(c, FAST_EINVAL, "k_S * v_m * sqrt2 too large for FP32 weights");
  if (span > 700.0) return fail(c, FAST_EINVAL, "k_S * v_m * sqrt2 too large");
  const int64_t C = (int64_t)g->width * g->height;
  int64_t exits = 0;
  for (int64_t i = 0; i < C; ++i) {
    if (g->cell_type[i] > 2) return fail(c, FAST_EINVAL, "cell type %d at %lld", g->cell_type[i], (long long)i);
    exits += g->cell_type[i] == FAST_CELL_EXIT;
  }
  if (exits == 0) return fail(c, FAST_EINVAL, "grid has no exit cell");

  std::vector<int32_t> a(C), b(C);
  if (g->static_field) {
    const int64_t bad = decompose_field(g->width, g->height, g->cell_type, g->static_field, 0x7FFE,
                                        a.data(), b.data());
    if (bad >= 0)
      return fail(c, FAST_EINVAL,
                  "static_field at cell %lld (%.17g): an exit needs 0, a free cell +inf "
                  "(no exit reachable) or a + b*sqrt(2) rounded as fl(a + fl(b*sqrt2)), "
                  "integers 0 <= a, b <= 32766, not both 0",
                  (long long)bad, g->static_field[bad]);
  } else {
    exact_floor_field(g->width, g->height, g->cell_type, a.data(), b.data());
  }
  std::vector<uint32_t> rec(C);
  RepHost& R = c->reps[r];
  for (int64_t i = 0; i < C; ++i) {
    if (a[i] < 0) {
      rec[i] = 0x7FFFu | (0x7FFFu << 15) | 0x40000000u;
      continue;
    }
    if (a[i] > 0x7FFE || b[i] > 0x7FFE)
      return fail(c, FAST_EINVAL, "distance to the nearest exit too long at cell %lld", (long long)i);
    rec[i] = (uint32_t)a[i] | ((uint32_t)b[i] << 15);
  }
  // the cells a seeded uniform placement draws from
  R.eligible.assign((size_t)((C + 63) / 64), 0ull);
  R.n_eligible = 0;
  for (int64_t i = 0; i < C; ++i)
    if (g->cell_type[i] == FAST_CELL_FREE && a[i] >= 0) {
      R.eligible[(size_t)(i >> 6)] |= 1ull << (i & 63);
      ++R.n_eligible;
    }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  // (re)allocate the per-cell arrays
  dfree(c, R.d.rec);
  for (int s = 0; s < 5; ++s)
    if (R.d.mask_v[s] != R.d.mask) dfree(c, R.d.mask_v[s]);
  dfree(c, R.d.mask);
  for (int s = 0; s < 5; ++s) R.d.mask_v[s] = nullptr;
  dfree(c, R.d_speed_by_id);
  R.d_speed_by_id = nullptr;
  R.n_speed_ids = 0;
  R.speed_set = 0;
  for (auto& p : R.d.claim) dfree(c, p);
  dfree(c, R.d.cmark);
  R.d.cmark = nullptr;
  R.d.rec = nullptr;
  R.d.mask = nullptr;
  R.d.claim[0] = R.d.claim[1] = nullptr;
  // until the new arrays are in place the replicate has no grid and no
  // agents, and the work lists are rebuilt without it (so an allocation that
  // fails below leaves a state that later calls refuse, not freed memory)
  R.grid_set = false;
  R.placed = false;
  R.n_ids = -1;
  c->layout_dirty = true;
  R.W = g->width;
  R.H = g->height;
  R.v = g->v_m;
  R.kS = g->k_S;
  R.seed = g->seed;
  R.K = reach_count_host(R.v, c->reach);
  R.mw = R.K > 64 ? 2 : 1;
  if (int e = alloc_into(c, &R.d.rec, C)) return e;
  if (int e = alloc_into(c, &R.d.mask, C * R.mw)) return e;
  const int64_t claim_cells = (int64_t)((R.W + 15) / 16) * ((R.H + 15) / 16) * 256;
  for (auto& p : R.d.claim)
    if (int e = alloc_into(c, &p, claim_cells)) return e;
  if (int e = alloc_into(c, &R.d.cmark, claim_cells)) return e;
  RepDev& d = R.d;
  d.W = R.W;
  d.H = R.H;
  d.v = R.v;
  d.reach = c->reach;
  d.K = R.K;
  d.mw = R.mw;
  d.kS = R.kS;
  d.c32 = (float)(-R.kS * kLog2e);
  d.margin = margin_of(R.v, R.K, R.kS);
  for (int s = 1; s <= 5; ++s) d.margin_v[s - 1] = margin_of(s, reach_count_host(s, c->reach), R.kS);
  d.mask_v[R.v - 1] = d.mask;
  d.seed_lo = (uint32_t)R.seed;
  d.seed_hi = (uint32_t)(R.seed >> 32);
  CUDA_TRY(c, cudaMemcpyAsync(d.rec, rec.data(), C * 4, cudaMemcpyHostToDevice, c->stream));
  d.claim_tx = (R.W + 15) / 16;
  for (auto p : d.claim) CUDA_TRY(c, cudaMemsetAsync(p, 0xFF, claim_cells * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(d.cmark, 0, claim_cells, c->stream));
  R.grid_set = true;
  R.placed = false;
  R.n_ids = -1;
  R.n = 0;
  const int32_t zero = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_nslots + r, &zero, 4, cudaMemcpyHostToDevice, c->stream));
  if (int e = upload_reps(c)) return e;
  LAUNCH_TRY(c, masks_launch(d, c->d_reps + r, C, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->layout_dirty = true;
  return FAST_OK;
}

int fast_set_speeds(fast_ctx* c, int32_t r, int32_t n_ids, const uint8_t* speed_by_id) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!rep_ok(c, r)) return fail(c, FAST_EINVAL, "bad replicate index %d", r);
  RepHost& R = c->reps[r];
  if (!R.grid_set) return fail(c, FAST_ESTATE, "grid of replicate %d not set", r);
  if (R.placed)
    return fail(c, FAST_ESTATE, "replicate %d already has agents: set speeds before placing", r);
  if (n_ids < 0 || n_ids > (1 << kMaxIdBits))
    return fail(c, FAST_EINVAL, "id count %d out of range", n_ids);
  if (n_ids > 0 && !speed_by_id) return fail(c, FAST_EINVAL, "speed_by_id is NULL");
  uint32_t set = 0;
  int smax = 0;
  for (int32_t i = 0; i < n_ids; ++i) {
    const int v = speed_by_id[i];
    if (v < 1 || v > 5) return fail(c, FAST_EINVAL, "speed %d of id %d not in 1..5", v, i);
    set |= 1u << (v - 1);
    smax = std::max(smax, v);
  }
  const double span = R.kS * smax * kSqrt2;
  if (c->precision != FAST_FP64 && span * kLog2e > 120.0)
    return fail(c, FAST_EINVAL, "k_S * speed * sqrt2 too large for FP32 weights");
  if (span > 700.0) return fail(c, FAST_EINVAL, "k_S * speed * sqrt2 too large");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  dfree(c, R.d_speed_by_id);
  R.d_speed_by_id = nullptr;
  R.n_speed_ids = 0;
  const int64_t C = (int64_t)R.W * R.H;
  for (int v = 1; v <= 5; ++v) {
    unsigned long long*& mk = R.d.mask_v[v - 1];
    const bool want = v == R.v || ((set >> (v - 1)) & 1u);
    if (!want && mk && mk != R.d.mask) {
      dfree(c, mk);
      mk = nullptr;
    }
    if (want && !mk) {
      const int mw = reach_count_host(v, c->reach) > 64 ? 2 : 1;
      if (int e = alloc_into(c, &mk, (size_t)C * mw)) return e;
      LAUNCH_TRY(c, masks_speed_launch(c->d_reps + r, C, v, mw, mk, c->stream));
    }
  }
  if (n_ids > 0) {
    if (int e = alloc_into(c, &R.d_speed_by_id, (size_t)n_ids)) return e;
    CUDA_TRY(c, cudaMemcpyAsync(R.d_speed_by_id, speed_by_id, (size_t)n_ids,
                                cudaMemcpyHostToDevice, c->stream));
    R.n_speed_ids = n_ids;
  }
  R.speed_set = set;
  if (int e = upload_reps(c)) return e;
  c->layout_dirty = true;
  return FAST_OK;
}

int fast_place_agents(fast_ctx* c, int32_t r, int32_t n, const int32_t* cells, const int32_t* ids,
                      int32_t start_step) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!rep_ok(c, r)) return fail(c, FAST_EINVAL, "bad replicate index %d", r);
  RepHost& R = c->reps[r];
  if (!R.grid_set) return fail(c, FAST_ESTATE, "grid of replicate %d not set", r);
  if (n < 0 || n > (1 << kMaxIdBits)) return fail(c, FAST_EINVAL, "agent count %d out of range", n);
  if (start_step < 0) return fail(c, FAST_EINVAL, "start_step < 0");
  // no cells: a seeded uniform placement of ids 0..n-1
  const bool uniform = n > 0 && !cells;
  std::vector<int32_t> drawn;
  if (uniform) {
    if (ids) return fail(c, FAST_EINVAL, "a uniform placement (cells NULL) takes no ids");
    if (n > R.n_eligible)
      return fail(c, FAST_EINVAL, "%d agents but only %lld free reachable cells", n,
                  (long long)R.n_eligible);
    uniform_cells(R, n, drawn);
    cells = drawn.data();
  }
  const int64_t C = (int64_t)R.W * R.H;

  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  // The same implicit ids again (a caller that places what it read back):
  // every agent goes back to the slot its id holds, so the storage order the
  // last spatial sort made stays, and no sort is needed before the next step
  // (agents move at most a few cells per step).
  const bool keep_order = R.placed && !ids && !uniform && n > 0 && n == R.n_ids && n <= R.cap;
  int32_t* slot_of_id = keep_order ? R.d.id2 : nullptr;  // free scratch of cap slots here
  if (keep_order) CUDA_TRY(c, cudaMemsetAsync(slot_of_id, 0xFF, (size_t)n * 4, c->stream));
  // clear the previous agents' occupancy marks
  if (R.placed && R.cap > 0)
    LAUNCH_TRY(c, clear_occ_launch(c->d_reps + r, c->d_nslots, r, R.cap, slot_of_id, n, c->stream));
  if (n > R.cap || !R.placed)
    if (int e = realloc_slots(c, R, n)) return e;
  // the upload runs on the private stream beside the clean-up below (the
  // staging arrays are free: the stream was idle when this call began)
  if (n > 0) {
    CUDA_TRY(c, cudaMemcpyAsync(R.d.cell2, cells, (size_t)n * 4, cudaMemcpyHostToDevice,
                                c->cap_stream));
    if (ids)
      CUDA_TRY(c, cudaMemcpyAsync(R.d.id2, ids, (size_t)n * 4, cudaMemcpyHostToDevice,
                                  c->cap_stream));
  }
  CUDA_TRY(c, cudaEventRecord(c->ev_upload, c->cap_stream));
  if (ids && !c->d_id_bits) {
    if (int e = alloc_into(c, &c->d_id_bits, (size_t)1 << (kMaxIdBits - 5))) return e;
    CUDA_TRY(c, cudaMemsetAsync(c->d_id_bits, 0, (size_t)4 << (kMaxIdBits - 5), c->stream));
  }
  if (!c->d_place_err)
    if (int e = alloc_into(c, &c->d_place_err, 4)) return e;
  R.placed = true;
  R.n = 0;
  R.n_ids = -1;
  CUDA_TRY(c, cudaMemsetAsync(R.d.cell, 0xFF, (size_t)R.cap * 4, c->stream));
  // first failing index, agents placed, slots appended, and the slot count
  // before this call
  int32_t* words = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(c->h_ctl) + sizeof(Ctl));
  words[0] = INT32_MAX;
  words[1] = 0;
  words[2] = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_place_err, words, 12, cudaMemcpyHostToDevice, c->stream));
  if (c->layout_dirty) {
    if (int e = rebuild_layout(c)) return e;
  }
  CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_upload, 0));
  // the check and the placement in one pass on the device
  uint8_t* placed = reinterpret_cast<uint8_t*>(R.d.mvinfo);
  LAUNCH_TRY(c, place_checked_launch(c->d_reps + r, R.d.cell2, ids ? R.d.id2 : nullptr, n, C,
                                     c->d_id_bits, placed, R.d_speed_by_id, R.n_speed_ids,
                                     slot_of_id, c->d_nslots + r, c->d_place_err, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(words + 4, c->d_place_err, 12, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(words + 7, c->d_nslots + r, 4, cudaMemcpyDeviceToHost, c->stream));
  if (ids)
    CUDA_TRY(c, cudaMemsetAsync(c->d_id_bits, 0, (size_t)4 << (kMaxIdBits - 5), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int32_t res0 = words[4], res1 = words[5], appended = words[6], slots_old = words[7];
  const int32_t zero = 0;
  if (res0 != INT32_MAX) {
    // undo: the replicate is left without agents (every slot this call wrote
    // is below n)
    LAUNCH_TRY(c, place_rollback_launch(c->d_reps + r, R.d.cell2, n, placed, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_nslots + r, &zero, 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_exited + r, &zero, 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int32_t bad_cell = -1, bad_id = res0;
    if (cells) bad_cell = cells[res0];
    if (ids) bad_id = ids[res0];
    return fail(c, FAST_EINVAL,
                "agent %d (id %d): cell %d is outside, not free, unreachable, an exit or taken, "
                "or the id is outside [0, 2^24), repeated or without a speed; the replicate "
                "now has no agents",
                res0, bad_id, bad_cell);
  }
  R.n = res1;
  R.n_ids = ids ? -1 : n;
  const int32_t slots = keep_order ? slots_old + appended : n;
  words[8] = slots;
  words[9] = start_step;
  words[10] = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_nslots + r, words + 8, 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_exited + r, words + 10, 4, cudaMemcpyHostToDevice, c->stream));
  // step index and per-step counters
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->t, words + 9, 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->dig_count, words + 10, 4, cudaMemcpyHostToDevice,
                              c->stream));
  const StepArgs a = args_of(c);
  LAUNCH_TRY(c, step_begin_launch(a, c->stream));
  // the spatial order of new agents is made once, before the next step
  if (!keep_order) c->resort_pending = true;
  // no wait here: what is still queued reads the pinned staging words 8..10,
  // which only the next placement rewrites, after its own wait
  c->t_host = start_step;
  c->steps_since_place = 0;
  return FAST_OK;
}

// Every replicate in one call: one upload, one launch per stage for all
// replicates, one wait.

int fast_place_all(fast_ctx* c, const int32_t* counts, const int32_t* cells_by_id,
                   int32_t start_step) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!counts) return fail(c, FAST_EINVAL, "counts is NULL");
  if (start_step < 0) return fail(c, FAST_EINVAL, "start_step < 0");
  std::vector<int64_t> off(c->n_rep + 1, 0);
  for (int r = 0; r < c->n_rep; ++r) {
    const int32_t n = counts[r];
    if (n < -1 || n > (1 << kMaxIdBits)) return fail(c, FAST_EINVAL, "replicate %d: count %d", r, n);
    if (n >= 0 && !c->reps[r].grid_set) return fail(c, FAST_ESTATE, "grid of replicate %d not set", r);
    off[r + 1] = off[r] + std::max(n, 0);
  }
  const int64_t total = off[c->n_rep];
  if (total > 0 && !cells_by_id) return fail(c, FAST_EINVAL, "cells_by_id is NULL");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  // the work list below must cover every placed replicate's slots
  if (c->layout_dirty)
    if (int e = rebuild_layout(c)) return e;
  if (int e = batch_buffers(c)) return e;
  const BatchHost h = batch_host(c);
  bool any_keep = false, any_clear = false;
  for (int r = 0; r < c->n_rep; ++r) {
    const RepHost& R = c->reps[r];
    const int32_t n = counts[r];
    BatchRep& b = h.bp[r];
    b.off = off[r];
    b.n = n;
    // the same implicit ids again: agents go back to the slots their ids
    // hold (as fast_place_agents does)
    b.keep = (R.placed && n > 0 && n == R.n_ids && n <= R.cap) ? 1 : 0;
    b.clear = (R.placed && n >= 0) ? 1 : 0;
    b.n_speed_ids = R.n_speed_ids;
    b.speed_by_id = R.d_speed_by_id;
    h.err[3 * r] = INT32_MAX;
    h.err[3 * r + 1] = 0;
    h.err[3 * r + 2] = 0;
    any_keep = any_keep || b.keep;
    any_clear = any_clear || b.clear;
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_bp, h.bp, sizeof(BatchRep) * c->n_rep, cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_berr, h.err, 12 * (size_t)c->n_rep, cudaMemcpyHostToDevice,
                              c->stream));
  {
    const Chunks all = all_chunks(c);
    const int grid = plan_grid(c, all.n);
    if (any_keep) LAUNCH_TRY(c, batch_prepare_launch(c->d_reps, all, c->d_bp, grid, c->stream));
    if (any_clear)
      LAUNCH_TRY(c, batch_clear_launch(c->d_reps, c->d_nslots, all, c->d_bp, grid, c->stream));
  }
  // capacities (a reallocation changes the device descriptors; freeing the
  // old arrays waits for the clean-up above)
  for (int r = 0; r < c->n_rep; ++r) {
    RepHost& R = c->reps[r];
    const int32_t n = counts[r];
    if (n < 0) continue;
    if (n > R.cap || !R.placed) {
      if (int e = realloc_slots(c, R, n)) return e;
      CUDA_TRY(c, cudaMemsetAsync(R.d.cell, 0xFF, (size_t)R.cap * 4, c->stream));
    }
    R.placed = true;
    R.n_ids = -1;
  }
  if (c->layout_dirty)
    if (int e = rebuild_layout(c)) return e;
  if (total > c->stage_cap) {
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(c, c->d_stage);
    c->d_stage = nullptr;
    if (int e = alloc_into(c, &c->d_stage, (size_t)total)) return e;
    c->stage_cap = total;
  }
  if (total > 0) {
    CUDA_TRY(c, cudaMemcpyAsync(c->d_stage, cells_by_id, (size_t)total * 4,
                                cudaMemcpyHostToDevice, c->stream));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, c->sms * 8));
    LAUNCH_TRY(c, batch_place_launch(c->d_reps, c->d_stage, total, c->d_bp, c->n_rep,
                                     c->d_nslots, c->d_berr, grid, c->stream));
  }
  CUDA_TRY(c, cudaMemcpyAsync(h.err, c->d_berr, 12 * (size_t)c->n_rep, cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(h.slots, c->d_nslots, 4 * (size_t)c->n_rep, cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(h.exited, c->d_exited, 4 * (size_t)c->n_rep, cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  int first_bad = -1;
  bool resort = false;
  for (int r = 0; r < c->n_rep; ++r) {
    const int32_t n = counts[r];
    if (n < 0) continue;
    RepHost& R = c->reps[r];
    h.exited[r] = 0;
    if (h.err[3 * r] != INT32_MAX) {
      // undo: the replicate is left without agents (every slot written is below n)
      LAUNCH_TRY(c, place_rollback_launch(c->d_reps + r, c->d_stage + off[r], n,
                                          reinterpret_cast<uint8_t*>(R.d.mvinfo), c->stream));
      h.slots[r] = 0;
      R.n = 0;
      if (first_bad < 0) first_bad = r;
    } else {
      h.slots[r] = h.bp[r].keep ? h.slots[r] + h.err[3 * r + 2] : n;
      R.n = h.err[3 * r + 1];
      R.n_ids = n;
      resort = resort || !h.bp[r].keep;
    }
  }
  h.misc[0] = start_step;
  h.misc[1] = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_nslots, h.slots, 4 * (size_t)c->n_rep, cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_exited, h.exited, 4 * (size_t)c->n_rep, cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->t, h.misc, 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->dig_count, h.misc + 1, 4, cudaMemcpyHostToDevice,
                              c->stream));
  const StepArgs a = args_of(c);
  LAUNCH_TRY(c, step_begin_launch(a, c->stream));
  // new agents are put in spatial order once, before the next step
  if (resort) c->resort_pending = true;
  // no wait here: what is still queued reads the pinned slot, exit and step
  // words, which only the next batched call rewrites, after its own wait
  c->t_host = start_step;
  c->steps_since_place = 0;
  if (first_bad >= 0) {
    const int32_t i = h.err[3 * first_bad];
    return fail(c, FAST_EINVAL,
                "replicate %d, agent %d: cell %d is outside, not free, unreachable, an exit or "
                "taken; the replicates that failed now have no agents",
                first_bad, i, cells_by_id[off[first_bad] + i]);
  }
  return FAST_OK;
}

int fast_readback_all(fast_ctx* c, const int32_t* counts, int32_t* cells_by_id,
                      int32_t* desired_by_id, int32_t* alive) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!counts) return fail(c, FAST_EINVAL, "counts is NULL");
  std::vector<int64_t> off(c->n_rep + 1, 0);
  for (int r = 0; r < c->n_rep; ++r) {
    if (counts[r] < 0) return fail(c, FAST_EINVAL, "replicate %d: count %d", r, counts[r]);
    off[r + 1] = off[r] + counts[r];
  }
  const int64_t total = off[c->n_rep];
  if (int e = batch_buffers(c)) return e;
  const BatchHost h = batch_host(c);
  if (total > 0 && (cells_by_id || desired_by_id)) {
    if (total * 2 > c->gather_cap) {
      dfree(c, c->d_gather);
      c->d_gather = nullptr;
      if (int e = alloc_into(c, &c->d_gather, (size_t)total * 2)) return e;
      c->gather_cap = total * 2;
    }
    if (c->layout_dirty)
      if (int e = rebuild_layout(c)) return e;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the staging's last use is done
    for (int r = 0; r < c->n_rep; ++r) {
      BatchRep& b = h.bp[r];
      b.off = off[r];
      b.n = c->reps[r].placed ? counts[r] : 0;
      b.keep = b.clear = 0;
      b.n_speed_ids = 0;
      b.speed_by_id = nullptr;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_bp, h.bp, sizeof(BatchRep) * c->n_rep,
                                cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_gather, 0xFF, (size_t)total * 8, c->stream));
    const Chunks all = all_chunks(c);
    LAUNCH_TRY(c, batch_gather_launch(c->d_reps, c->d_nslots, all, c->d_bp, c->d_gather,
                                      c->d_gather + total, plan_grid(c, all.n), c->stream));
    if (cells_by_id)
      CUDA_TRY(c, cudaMemcpyAsync(cells_by_id, c->d_gather, (size_t)total * 4,
                                  cudaMemcpyDeviceToHost, c->stream));
    if (desired_by_id)
      CUDA_TRY(c, cudaMemcpyAsync(desired_by_id, c->d_gather + total, (size_t)total * 4,
                                  cudaMemcpyDeviceToHost, c->stream));
  }
  // the control block (device error) and the exit counts come back with the
  // data: one wait for all of it
  CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(h.exited, c->d_exited, 4 * (size_t)c->n_rep, cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (int e = device_error_of(c, *c->h_ctl)) return e;
  if (alive)
    for (int r = 0; r < c->n_rep; ++r)
      alive[r] = c->reps[r].placed ? c->reps[r].n - h.exited[r] : 0;
  return FAST_OK;
}

int fast_step(fast_ctx* c, int32_t n_steps) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (n_steps < 0) return fail(c, FAST_EINVAL, "n_steps < 0");
  bool any = false;
  for (auto& R : c->reps) any = any || R.placed;
  if (!any) return fail(c, FAST_ESTATE, "no agents placed");
  if (c->layout_dirty)
    if (int e = rebuild_layout(c)) return e;
  if (int e = sort_if_pending(c)) return e;
  if (c->digests && c->steps_since_place + n_steps > c->dig_cap) {
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int32_t want = (int32_t)std::max<int64_t>(1024, 2 * (c->steps_since_place + n_steps));
    unsigned long long *dc = nullptr, *dd = nullptr;
    if (int e = alloc_into(c, &dc, (size_t)want * c->n_rep)) return e;
    if (int e = alloc_into(c, &dd, (size_t)want * c->n_rep)) return e;
    CUDA_TRY(c, cudaMemsetAsync(dc, 0, (size_t)want * c->n_rep * 8, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(dd, 0, (size_t)want * c->n_rep * 8, c->stream));
    if (c->d_dig_cell) {
      CUDA_TRY(c, cudaMemcpyAsync(dc, c->d_dig_cell, (size_t)c->dig_cap * c->n_rep * 8,
                                  cudaMemcpyDeviceToDevice, c->stream));
      CUDA_TRY(c, cudaMemcpyAsync(dd, c->d_dig_des, (size_t)c->dig_cap * c->n_rep * 8,
                                  cudaMemcpyDeviceToDevice, c->stream));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(c, c->d_dig_cell);
    dfree(c, c->d_dig_des);
    c->d_dig_cell = dc;
    c->d_dig_des = dd;
    c->dig_cap = want;
    drop_graphs(c);
  }
  if (c->use_graph && n_steps >= 2 && n_steps <= c->graph_steps) {
    const int phase = c->resort_period > 0 ? (int)(c->t_host % c->resort_period) : 0;
    const auto key = std::make_pair(phase, (int)n_steps);
    auto it = c->multi.find(key);
    if (it == c->multi.end()) {
      if (c->multi.size() >= 8) {
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (auto& kv : c->multi)
          if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        c->multi.clear();
      }
      fast_ctx::Multi m;
      if (int e = build_multi(c, n_steps, &m)) return e;
      it = c->multi.emplace(key, m).first;
    }
    if (it->second.exec) {
      CUDA_TRY(c, cudaGraphLaunch(it->second.exec, c->stream));
      c->launches += it->second.launches;
      c->t_host += n_steps;
      c->steps_since_place += n_steps;
      c->ran_step = true;
      return FAST_OK;
    }
  }
  for (int32_t i = 0; i < n_steps; ++i) {
    const bool resort = c->resort_period > 0 && ((c->t_host + 1) % c->resort_period == 0);
    const int which = resort ? 1 : 0;
    if (c->use_graph && c->graph_state[which] == 0) {
      if (int e = build_graph(c, which)) return e;
    }
    if (c->use_graph && c->graph_state[which] == 1) {
      CUDA_TRY(c, cudaGraphLaunch(c->graph[which], c->stream));
      c->launches += c->launches_per_graph[which];
    } else {
      if (int e = enqueue_step(c, resort)) return e;
    }
    c->t_host += 1;
    c->steps_since_place += 1;
  }
  c->ran_step = c->ran_step || n_steps > 0;
  return FAST_OK;
}

int fast_plan_only(fast_ctx* c, int32_t n) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  bool any = false;
  for (auto& R : c->reps) any = any || R.placed;
  if (!any) return fail(c, FAST_ESTATE, "no agents placed");
  if (c->layout_dirty)
    if (int e = rebuild_layout(c)) return e;
  if (int e = sort_if_pending(c)) return e;
  const StepArgs a = args_of(c);
  for (int32_t i = 0; i < n; ++i) {
    LAUNCH_TRY(c, step_begin_launch(a, c->stream));
    if (int e = enqueue_plan(c, a, false, false)) return e;
  }
  return FAST_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times the planning kernels on the context's own agents and keeps
// the fastest re-sort bucket size and, per v_m group, the fastest planning
// variant.  Choices change speed only: every variant computes the same
// desired cells.
namespace {

constexpr int kTuneShifts[4] = {3, 4, 5, 6};
constexpr int kTuneLanes[5] = {0, 1, 2, 4, 8};

// Mean time (us) of `trials` planning passes of group gi (-1: every group)
// with the context's current variants; one untimed pass first.
int time_planning(fast_ctx* c, int gi, int trials, cudaEvent_t e0, cudaEvent_t e1, float* us) {
  const StepArgs a = args_of(c);
  for (int i = 0; i <= trials; ++i) {
    if (i == 1) CUDA_TRY(c, cudaEventRecord(e0, c->stream));
    LAUNCH_TRY(c, step_begin_launch(a, c->stream));
    for (int g = 0; g < (int)c->groups.size(); ++g) {
      if (gi >= 0 && g != gi) continue;
      const auto& G = c->groups[g];
      Chunks ch{G.d_rep, G.d_begin, G.n};
      LAUNCH_TRY(c, plan_groups_launch(a, G.v, c->reach, c->lanes[G.v - 1], c->precision, ch,
                                       plan_grid(c, G.n), c->stream, false));
    }
  }
  CUDA_TRY(c, cudaEventRecord(e1, c->stream));
  CUDA_TRY(c, cudaEventSynchronize(e1));
  float ms = 0.f;
  CUDA_TRY(c, cudaEventElapsedTime(&ms, e0, e1));
  *us = 1e3f * ms / (float)trials;
  return FAST_OK;
}

int time_resort(fast_ctx* c, int trials, cudaEvent_t e0, cudaEvent_t e1, float* us) {
  const StepArgs a = args_of(c);
  const Chunks all = all_chunks(c);
  for (int i = 0; i <= trials; ++i) {
    if (i == 1) CUDA_TRY(c, cudaEventRecord(e0, c->stream));
    LAUNCH_TRY(c, resort_launch(a, all, plan_grid(c, all.n), true, c->stream));
  }
  CUDA_TRY(c, cudaEventRecord(e1, c->stream));
  CUDA_TRY(c, cudaEventSynchronize(e1));
  float ms = 0.f;
  CUDA_TRY(c, cudaEventElapsedTime(&ms, e0, e1));
  *us = 1e3f * ms / (float)trials;
  return FAST_OK;
}

int apply_shift(fast_ctx* c, int shift) {
  c->tile_shift = shift;
  c->layout_dirty = true;
  if (int e = rebuild_layout(c)) return e;
  const StepArgs a = args_of(c);
  const Chunks all = all_chunks(c);
  LAUNCH_TRY(c, resort_launch(a, all, plan_grid(c, all.n), true, c->stream));
  c->launches += 7;
  c->resort_pending = false;
  return FAST_OK;
}

int autotune_impl(fast_ctx* c, int trials, fast_tune_report* rep, cudaEvent_t e0,
                  cudaEvent_t e1) {
  // 1. bucket size: planning with the tiled kernel everywhere, plus the
  //    re-sort amortised over its period
  int saved[5];
  std::memcpy(saved, c->lanes, sizeof saved);
  for (int v = 0; v < 5; ++v) c->lanes[v] = 0;
  int best_shift = c->tile_shift;
  float best = 1e30f;
  for (int i = 0; i < 4; ++i) {
    if (int e = apply_shift(c, kTuneShifts[i])) return e;
    float plan_us = 0.f, sort_us = 0.f;
    if (int e = time_planning(c, -1, trials, e0, e1, &plan_us)) return e;
    if (int e = time_resort(c, 1, e0, e1, &sort_us)) return e;
    const float per_step = plan_us + (c->resort_period > 0 ? sort_us / c->resort_period : 0.f);
    rep->shift_us[i] = per_step;
    if (per_step < best) {
      best = per_step;
      best_shift = kTuneShifts[i];
    }
  }
  if (int e = apply_shift(c, best_shift)) return e;
  rep->tile_shift = best_shift;
  // 2. planning variant per v_m group
  for (int v = 0; v < 5; ++v) rep->lanes[v] = -1;
  for (int g = 0; g < (int)c->groups.size(); ++g) {
    const int v = c->groups[g].v;
    int best_l = 0;
    float best_t = 1e30f;
    for (int j = 0; j < 5; ++j) {
      c->lanes[v - 1] = kTuneLanes[j];
      float us = 0.f;
      if (int e = time_planning(c, g, trials, e0, e1, &us)) return e;
      rep->lanes_us[v - 1][j] = us;
      if (us < best_t) {
        best_t = us;
        best_l = kTuneLanes[j];
      }
    }
    c->lanes[v - 1] = best_l;
    rep->lanes[v - 1] = best_l;
  }
  for (int v = 0; v < 5; ++v)
    if (rep->lanes[v] < 0) c->lanes[v] = saved[v];
  return FAST_OK;
}

}  // namespace

int fast_autotune(fast_ctx* c, int32_t trials, fast_tune_report* out) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (trials < 1 || trials > 1000) return fail(c, FAST_EINVAL, "trials not in 1..1000");
  bool any = false;
  for (auto& R : c->reps) any = any || R.placed;
  if (!any) return fail(c, FAST_ESTATE, "no agents placed");
  fast_tune_report rep{};
  rep.tile_shift = c->tile_shift;
  for (int v = 0; v < 5; ++v) rep.lanes[v] = -1;
  if (c->precision != FAST_FP64) {
    if (c->layout_dirty)
      if (int e = rebuild_layout(c)) return e;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      return fail(c, FAST_ECUDA, "cudaEventCreate failed");
    }
    const int e = autotune_impl(c, trials, &rep, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) return e;
    if (int e2 = check_device_error(c)) return e2;
    drop_graphs(c);
  }
  if (out) *out = rep;
  return FAST_OK;
}

int fast_readback(fast_ctx* c, int32_t r, int32_t id_bound, int32_t* cells_by_id,
                  int32_t* desired_by_id, fast_stats* stats) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!rep_ok(c, r) || id_bound < 0) return fail(c, FAST_EINVAL, "bad replicate or id_bound");
  RepHost& R = c->reps[r];
  if (id_bound > 0 && (cells_by_id || desired_by_id)) {
    if (id_bound * 2 > c->gather_cap) {
      dfree(c, c->d_gather);
      c->d_gather = nullptr;
      if (int e = alloc_into(c, &c->d_gather, (size_t)id_bound * 2)) return e;
      c->gather_cap = id_bound * 2;
    }
    CUDA_TRY(c, cudaMemsetAsync(c->d_gather, 0xFF, (size_t)id_bound * 8, c->stream));
    if (R.placed)
      LAUNCH_TRY(c, gather_by_id_launch(c->d_reps + r, c->d_nslots, r, R.cap, c->d_gather,
                                        c->d_gather + id_bound, id_bound, c->stream));
    if (cells_by_id)
      CUDA_TRY(c, cudaMemcpyAsync(cells_by_id, c->d_gather, (size_t)id_bound * 4,
                                  cudaMemcpyDeviceToHost, c->stream));
    if (desired_by_id)
      CUDA_TRY(c, cudaMemcpyAsync(desired_by_id, c->d_gather + id_bound, (size_t)id_bound * 4,
                                  cudaMemcpyDeviceToHost, c->stream));
  }
  // the control block (device error, counters) and the replicate's exit count
  // come back with the data: one wait for all of it
  int32_t* h_exited = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(c->h_ctl) + sizeof(Ctl));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(h_exited, c->d_exited + r, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const Ctl& h = *c->h_ctl;
  if (int e = device_error_of(c, h)) return e;
  if (stats) {
    const int32_t ex = *h_exited;
    stats->step = h.t;
    stats->steps_run = c->steps_since_place;
    stats->exited = ex;
    stats->alive = R.n - ex;
    stats->agent_steps = (int64_t)h.agent_steps;
    stats->rechecked = (int64_t)h.rechecked_total;
    stats->move_rounds = (int64_t)h.rounds_total;
    stats->max_rounds = h.rounds_max;
    stats->last_rounds = h.rounds_last;
    stats->kernel_launches = c->launches;
    stats->tile_fallbacks = (int64_t)h.tile_fallbacks;
    stats->movers = (int64_t)h.movers_total;
    stats->footprint_cells = (int64_t)h.foot_total;
    stats->diag_flips = (int64_t)h.flips;
    float mdp;
    std::memcpy(&mdp, &h.max_dp_bits, 4);
    stats->diag_max_abs_dp = mdp;
  }
  return FAST_OK;
}

int fast_get_digests(fast_ctx* c, int32_t r, int32_t max_steps, uint64_t* cell_digest,
                     uint64_t* desired_digest) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!rep_ok(c, r) || max_steps < 0) return fail(c, FAST_EINVAL, "bad arguments");
  if (int e = check_device_error(c)) return e;
  int32_t cnt = 0;
  CUDA_TRY(c, cudaMemcpy(&cnt, &c->d_ctl->dig_count, 4, cudaMemcpyDeviceToHost));
  cnt = std::min(cnt, std::min(max_steps, c->dig_cap));
  if (cnt <= 0 || !c->d_dig_cell) return 0;
  std::vector<unsigned long long> a((size_t)cnt * c->n_rep), b((size_t)cnt * c->n_rep);
  CUDA_TRY(c, cudaMemcpy(a.data(), c->d_dig_cell, a.size() * 8, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(b.data(), c->d_dig_des, b.size() * 8, cudaMemcpyDeviceToHost));
  for (int32_t i = 0; i < cnt; ++i) {
    if (cell_digest) cell_digest[i] = a[(size_t)i * c->n_rep + r];
    if (desired_digest) desired_digest[i] = b[(size_t)i * c->n_rep + r];
  }
  return cnt;
}

int fast_phase_times(fast_ctx* c, float* ms5) {
  if (!c || !ms5) return FAST_EINVAL;
  if (!c->ran_step) return fail(c, FAST_ESTATE, "no step has run");
  CUDA_TRY(c, cudaEventSynchronize(c->ev[5]));
  for (int i = 0; i < 5; ++i) CUDA_TRY(c, cudaEventElapsedTime(&ms5[i], c->ev[i], c->ev[i + 1]));
  return FAST_OK;
}

int fast_move_profile(fast_ctx* c, int32_t max_rounds, uint32_t* n_wait, uint64_t* t_ns) {
  if (!c || max_rounds < 0) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (int e = check_device_error(c)) return e;
  Ctl h{};
  CUDA_TRY(c, cudaMemcpy(&h, c->d_ctl, sizeof h, cudaMemcpyDeviceToHost));
  const int n = std::min(std::min(max_rounds, kRoundLog), h.rounds_last);
  for (int i = 0; i < n; ++i) {
    if (n_wait) n_wait[i] = h.round_n[i];
    if (t_ns) t_ns[i] = h.round_ns[i];
  }
  if (t_ns && n > 0) t_ns[n] = h.round_ns[n];
  if (t_ns && max_rounds >= 64 + 1 + 8)
    for (int i = 0; i < 8; ++i) t_ns[65 + i] = h.phase_ns[i];
  if (t_ns && max_rounds >= 64 + 1 + 8 + 64)
    for (int i = 0; i < n; ++i) t_ns[73 + i] = h.round_bmax[i];
  return h.rounds_last;
}

int fast_precision_report_run(fast_ctx* c, fast_precision_report* out) {
  if (!c || !out) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (c->precision == FAST_FP64) return fail(c, FAST_ESTATE, "context plans in FP64");
  bool any = false;
  for (auto& R : c->reps) any = any || R.placed;
  if (!any) return fail(c, FAST_ESTATE, "no agents placed");
  if (c->layout_dirty)
    if (int e = rebuild_layout(c)) return e;
  if (int e = sort_if_pending(c)) return e;
  std::vector<int64_t> base(c->n_rep, 0);
  int64_t total = 0;
  double margin = 0.0;
  for (int r = 0; r < c->n_rep; ++r) {
    base[r] = total;
    if (c->reps[r].placed) {
      total += c->reps[r].cap;
      margin = std::max(margin, (double)c->reps[r].d.margin);
    }
  }
  float* p32 = nullptr;
  int32_t* ch32 = nullptr;
  uint8_t* fl = nullptr;
  int64_t* db = nullptr;
  if (int e = alloc_into(c, &p32, (size_t)total * kMaxK)) return e;
  if (int e = alloc_into(c, &ch32, (size_t)total)) return e;
  if (int e = alloc_into(c, &fl, (size_t)total)) return e;
  if (int e = alloc_into(c, &db, (size_t)c->n_rep)) return e;
  CUDA_TRY(c, cudaMemcpyAsync(db, base.data(), 8 * c->n_rep, cudaMemcpyHostToDevice, c->stream));
  const unsigned long long z[3] = {0, 0, 0};
  const unsigned int zi = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->flips, z, 24, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->max_dp_bits, &zi, 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->flips_after, &zi, 4, cudaMemcpyHostToDevice, c->stream));
  StepArgs a = args_of(c);
  // the FP32 pass without re-check that records its choices, flags and
  // cumulative probabilities (it writes its own choice into every desired
  // cell), then the real planning pass (FP32 weights, FP64 re-check inside
  // the margin), whose choices the comparison reads from the desired cells
  LAUNCH_TRY(c, step_begin_launch(a, c->stream));
  StepArgs ad = a;
  ad.diag_p32 = p32;
  ad.diag_choice32 = ch32;
  ad.diag_flag = fl;
  ad.diag_base = db;
  if (int e = enqueue_plan(c, ad, true, false)) return e;
  LAUNCH_TRY(c, step_begin_launch(a, c->stream));
  if (int e = enqueue_plan(c, a, false, false)) return e;
  a = ad;
  for (auto& g : c->groups) {
    Chunks ch{g.d_rep, g.d_begin, g.n};
    LAUNCH_TRY(c, plan_diag_compare_launch(a, g.v, c->reach, ch, plan_grid(c, g.n), c->stream));
  }
  Ctl h{};
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  CUDA_TRY(c, cudaMemcpy(&h, c->d_ctl, sizeof h, cudaMemcpyDeviceToHost));
  int64_t agents = 0;
  for (int r = 0; r < c->n_rep; ++r) {
    if (!c->reps[r].placed) continue;
    int32_t ns = 0, ex = 0;
    CUDA_TRY(c, cudaMemcpy(&ns, c->d_nslots + r, 4, cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(&ex, c->d_exited + r, 4, cudaMemcpyDeviceToHost));
    agents += c->reps[r].n - ex;
  }
  dfree(c, p32);
  dfree(c, ch32);
  dfree(c, fl);
  dfree(c, db);
  out->agents = agents;
  out->flagged = (int64_t)h.flagged;
  out->flips = (int64_t)h.flips;
  out->flips_unflagged = (int64_t)h.flips_unflagged;
  out->flips_after_recheck = (int64_t)h.flips_after;
  float mdp;
  std::memcpy(&mdp, &h.max_dp_bits, 4);
  out->max_abs_dp = mdp;
  out->margin = margin;
  return FAST_OK;
}

int fast_reach_union(fast_ctx* c, int32_t r, int64_t* cells) {
  if (!c || !cells) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!rep_ok(c, r) || !c->reps[r].placed) return fail(c, FAST_ESTATE, "replicate not placed");
  if (c->layout_dirty)
    if (int e = rebuild_layout(c)) return e;
  RepHost& R = c->reps[r];
  const int64_t words = ((int64_t)R.W * R.H + 31) / 32;
  uint32_t* bm = nullptr;
  unsigned long long* cnt = nullptr;
  if (int e = alloc_into(c, &bm, (size_t)words)) return e;
  if (int e = alloc_into(c, &cnt, 1)) return e;
  LAUNCH_TRY(c, union_count_launch(c->d_reps + r, c->d_nslots, r, R.cap, R.v, c->reach, R.W, R.H,
                                   bm, cnt, c->stream));
  unsigned long long h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  dfree(c, bm);
  dfree(c, cnt);
  *cells = (int64_t)h;
  return FAST_OK;
}

// Planning pass into a caller buffer without any device allocation: see
// noalloc.cu.  Reads the context's state, never changes it, never
// synchronises; the only scratch is the library's fixed re-check queue.
int fast_plan_noalloc(fast_ctx* c, int32_t r, int32_t step, int32_t id_bound,
                      int32_t* desired_by_id_dev) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  if (!rep_ok(c, r) || step < 0 || id_bound < 0 || (id_bound > 0 && !desired_by_id_dev))
    return fail(c, FAST_EINVAL, "bad replicate, step, id_bound or output pointer");
  RepHost& R = c->reps[r];
  if (!R.placed) return fail(c, FAST_ESTATE, "replicate %d has no agents", r);
  if (R.speed_set) return fail(c, FAST_EINVAL, "replicate %d has speeds per agent", r);
  if (c->layout_dirty)
    return fail(c, FAST_ESTATE, "layout not built yet: run fast_step or fast_plan_only once first");
  if (R.cap > noalloc_max_agents())
    return fail(c, FAST_EINVAL, "replicate %d has %d agent slots; this pass holds at most %d", r,
                R.cap, noalloc_max_agents());
  const int rc = noalloc_plan_launch(R.d, R.cap, step, desired_by_id_dev, id_bound, c->sms,
                                     c->stream);
  if (rc == -1) return fail(c, FAST_ECUDA, "address of the fixed re-check queue unavailable");
  if (rc == -2) return fail(c, FAST_EINVAL, "replicate %d has too many agent slots", r);
  if (rc != 0)
    return fail(c, FAST_ECUDA,
                "allocation-free planning pass not queued: a CUDA error was pending, a launch "
                "failed, or the replicate's speed or reach set is unknown");
  return FAST_OK;
}

int fast_set_option(fast_ctx* c, int32_t option, int64_t value) {
  if (!c) return FAST_EINVAL;
  if (c->poisoned) return FAST_ESTATE;
  switch (option) {
    case FAST_OPT_RESORT_PERIOD:
      if (value < 0) return fail(c, FAST_EINVAL, "resort period < 0");
      c->resort_period = (int)value;
      break;
    case FAST_OPT_DIGESTS:
      c->digests = value != 0;
      break;
    case FAST_OPT_BARRIER_NS: {
      if (value < 1000) return fail(c, FAST_EINVAL, "barrier limit below 1 us");
      c->barrier_ns = value;
      const unsigned long long v = (unsigned long long)value;
      CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->barrier_ns_limit, &v, 8, cudaMemcpyHostToDevice,
                                  c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      break;
    }
    case FAST_OPT_USE_GRAPH:
      c->use_graph = value != 0;
      break;
    case FAST_OPT_MOVE_BLOCKS:
      if (value < 0) return fail(c, FAST_EINVAL, "move blocks < 0");
      c->move_blocks = (int)value;
      break;
    case FAST_OPT_TILE_SHIFT:
      if (value < 0 || value > 10) return fail(c, FAST_EINVAL, "tile shift not in 0..10");
      c->tile_shift = (int)value;
      c->layout_dirty = true;
      break;
    case FAST_OPT_CLAIM_RESERVE:
      if (value < 0 || value > 254) return fail(c, FAST_EINVAL, "claim reserve not in 0..254");
      if (int e = write_ctl_int(c, offsetof(Ctl, tag_reserve), (int32_t)value)) return e;
      break;
    case FAST_OPT_CLAIM_TAG:
      // any tag is safe once no claim is left
      if (value < 0 || value > 254) return fail(c, FAST_EINVAL, "claim tag not in 0..254");
      for (auto& R : c->reps) {
        if (!R.grid_set) continue;
        const size_t n = (size_t)((R.W + 15) / 16) * ((R.H + 15) / 16) * 256;
        for (auto p : R.d.claim) CUDA_TRY(c, cudaMemsetAsync(p, 0xFF, n * 4, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(R.d.cmark, 0, n, c->stream));
      }
      if (int e = write_ctl_int(c, offsetof(Ctl, claim_tag), (int32_t)value)) return e;
      break;
    case FAST_OPT_GRAPH_STEPS:
      if (value < 0 || value > 4096) return fail(c, FAST_EINVAL, "graph steps not in 0..4096");
      c->graph_steps = (int)value;
      break;
    default:
      if (option >= FAST_OPT_LANES_V1 && option < FAST_OPT_LANES_V1 + 5) {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
          return fail(c, FAST_EINVAL, "lanes must be 0 (tiled), 1, 2, 4 or 8");
        c->lanes[option - FAST_OPT_LANES_V1] = (int)value;
        break;
      }
      return fail(c, FAST_EINVAL, "unknown option %d", option);
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  return FAST_OK;
}

const char* fast_last_error(const fast_ctx* c) { return c ? c->err.c_str() : "no context"; }

void fast_destroy(fast_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaGetLastError();
  drop_graphs(c);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->ev_upload) cudaEventDestroy(c->ev_upload);
  if (c->h_batch) cudaFreeHost(c->h_batch);
  std::vector<void*> ptrs;
  for (auto& kv : c->live) ptrs.push_back(kv.first);
  for (void* p : ptrs) dfree(c, p);
  delete c;
}

int fast_floor_field(int32_t width, int32_t height, const uint8_t* cell_type,
                     const double* static_field, double* S_out, int32_t* a_out, int32_t* b_out,
                     int64_t* bad_cell) {
  if (bad_cell) *bad_cell = -1;
  if (width < 1 || height < 1 || width > 65535 || height > 65535 ||
      (int64_t)width * height >= ((int64_t)1 << 31) || !cell_type)
    return FAST_EINVAL;
  const int64_t C = (int64_t)width * height;
  for (int64_t i = 0; i < C; ++i)
    if (cell_type[i] > 2) {
      if (bad_cell) *bad_cell = i;
      return FAST_EINVAL;
    }
  std::vector<int32_t> a(C), b(C);
  if (static_field) {
    const int64_t bad = decompose_field(width, height, cell_type, static_field, 0x7FFE, a.data(),
                                        b.data());
    if (bad >= 0) {
      if (bad_cell) *bad_cell = bad;
      return FAST_EINVAL;
    }
  } else {
    exact_floor_field(width, height, cell_type, a.data(), b.data());
  }
  for (int64_t i = 0; i < C; ++i) {
    if (S_out)
      S_out[i] = a[i] < 0 ? HUGE_VAL : (double)a[i] + (double)b[i] * kSqrt2;
    if (a_out) a_out[i] = a[i];
    if (b_out) b_out[i] = b[i];
  }
  return FAST_OK;
}

// ---- self tests ------------------------------------------------------------
int fast_selftest_exp64(const double* x, double* y, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !y))) return FAST_EINVAL;
  if (n == 0) return FAST_OK;
  double *dx = nullptr, *dy = nullptr;
  if (cudaMalloc(&dx, n * 8) != cudaSuccess) return FAST_ENOMEM;
  if (cudaMalloc(&dy, n * 8) != cudaSuccess) {
    cudaFree(dx);
    return FAST_ENOMEM;
  }
  int rc = FAST_OK;
  if (cudaMemcpy(dx, x, n * 8, cudaMemcpyHostToDevice) != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK) {
    test_exp64_launch(dx, dy, n, 0);
    if (cudaGetLastError() != cudaSuccess) rc = FAST_ECUDA;
  }
  if (rc == FAST_OK && cudaMemcpy(y, dy, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = FAST_ECUDA;
  cudaFree(dx);
  cudaFree(dy);
  return rc;
}

int fast_selftest_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return FAST_EINVAL;
  if (n == 0) return FAST_OK;
  uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
  if (cudaMalloc(&dc, n * 16) != cudaSuccess) return FAST_ENOMEM;
  if (cudaMalloc(&dk, n * 8) != cudaSuccess || cudaMalloc(&dout, n * 16) != cudaSuccess) {
    cudaFree(dc);
    cudaFree(dk);
    return FAST_ENOMEM;
  }
  int rc = FAST_OK;
  if (cudaMemcpy(dc, ctr, n * 16, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = FAST_ECUDA;
  if (rc == FAST_OK) {
    test_philox_launch(dc, dk, dout, n, 0);
    if (cudaGetLastError() != cudaSuccess) rc = FAST_ECUDA;
  }
  if (rc == FAST_OK && cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FAST_ECUDA;
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return rc;
}

int fast_selftest_ex2(float lo, float hi, double* max_rel_err) {
  if (!max_rel_err || !(lo <= hi)) return FAST_EINVAL;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 8) != cudaSuccess) return FAST_ENOMEM;
  int rc = FAST_OK;
  if (cudaMemset(d, 0, 8) != cudaSuccess) rc = FAST_ECUDA;
  // walk non-negative and negative floats separately (bit order = value order
  // for non-negative floats, reversed for negative ones)
  if (rc == FAST_OK && hi >= 0.f) test_ex2_launch(lo > 0.f ? lo : 0.f, hi, d, 0);
  if (rc == FAST_OK && lo < 0.f) test_ex2_launch(-0.0f, lo, d, 0);
  if (rc == FAST_OK && cudaGetLastError() != cudaSuccess) rc = FAST_ECUDA;
  unsigned long long h = 0;
  if (rc == FAST_OK && cudaMemcpy(&h, d, 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = FAST_ECUDA;
  cudaFree(d);
  double v;
  std::memcpy(&v, &h, 8);
  *max_rel_err = v;
  return rc;
}

int fast_build_checked(void) { return build_checked(); }

int fast_selftest_bounds(int64_t index, int64_t n, int64_t* recorded) {
  if (!recorded || n < 0) return FAST_EINVAL;
  *recorded = -1;
  Ctl* d = nullptr;
  if (cudaMalloc(&d, sizeof(Ctl)) != cudaSuccess) return FAST_ENOMEM;
  Ctl h{};
  int rc = FAST_OK;
  if (cudaMemcpy(d, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK) test_bounds_launch(d, (long long)index, (long long)n, 0);
  if (rc == FAST_OK && (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess))
    rc = FAST_ECUDA;
  if (rc == FAST_OK && cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FAST_ECUDA;
  cudaFree(d);
  if (rc != FAST_OK) return rc;
  if (h.err == kDevErrBounds) {
    *recorded = h.bad_index;
    return FAST_ECUDA;
  }
  return FAST_OK;
}

int fast_selftest_l2_read(int64_t bytes, int32_t iters, double* gb_per_s) {
  if (bytes < 4096 || bytes > ((int64_t)1 << 30) || (bytes & 15) || iters < 1 || iters > 10000 ||
      !gb_per_s)
    return FAST_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FAST_ECUDA;
  void* buf = nullptr;
  unsigned int* sink = nullptr;
  if (cudaMalloc(&buf, (size_t)bytes) != cudaSuccess) return FAST_ENOMEM;
  if (cudaMalloc(&sink, 4) != cudaSuccess) {
    cudaFree(buf);
    return FAST_ENOMEM;
  }
  int rc = FAST_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMemset(buf, 1, (size_t)bytes) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = FAST_ECUDA;
  float ms = 0.f;
  if (rc == FAST_OK) {
    test_l2_read_launch(buf, (size_t)bytes, 2, sink, sms * 4, 0);  // warm the L2
    cudaEventRecord(e0, 0);
    test_l2_read_launch(buf, (size_t)bytes, iters, sink, sms * 4, 0);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
      rc = FAST_ECUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(sink);
  if (rc != FAST_OK) return rc;
  *gb_per_s = (double)bytes * iters / (ms * 1e-3) / 1e9;
  return FAST_OK;
}

int fast_selftest_barrier_cost(int32_t blocks, int32_t threads, int32_t iters, double* ns_per_barrier) {
  if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !ns_per_barrier) return FAST_EINVAL;
  Ctl* d = nullptr;
  if (cudaMalloc(&d, sizeof(Ctl)) != cudaSuccess) return FAST_ENOMEM;
  Ctl h{};
  h.barrier_ns_limit = 2000000000ull;
  int rc = FAST_OK;
  if (cudaMemcpy(d, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK && test_barrier_cost_launch(d, blocks, threads, iters, 0) != 0) rc = FAST_EINVAL;
  if (rc == FAST_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK && cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FAST_ECUDA;
  cudaGetLastError();
  cudaFree(d);
  if (rc != FAST_OK) return rc;
  if (h.err != 0) return FAST_ETIMEOUT;
  *ns_per_barrier = (double)h.round_ns[0] / iters;
  return FAST_OK;
}

int fast_selftest_barrier_sum(int32_t blocks, int32_t threads, int32_t iters, int64_t* wrong) {
  if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !wrong) return FAST_EINVAL;
  Ctl* d = nullptr;
  if (cudaMalloc(&d, sizeof(Ctl)) != cudaSuccess) return FAST_ENOMEM;
  Ctl h{};
  h.barrier_ns_limit = 2000000000ull;
  int rc = FAST_OK;
  if (cudaMemcpy(d, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK && test_barrier_sum_launch(d, blocks, threads, iters, 0) != 0) rc = FAST_EINVAL;
  if (rc == FAST_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK && cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FAST_ECUDA;
  cudaGetLastError();
  cudaFree(d);
  if (rc != FAST_OK) return rc;
  if (h.err != 0) return FAST_ETIMEOUT;
  *wrong = (int64_t)h.flips;
  return FAST_OK;
}

int fast_selftest_barrier_timeout(int64_t limit_ns) {
  if (limit_ns < 1000 || limit_ns > 10000000000ll) return FAST_EINVAL;
  Ctl* d = nullptr;
  if (cudaMalloc(&d, sizeof(Ctl)) != cudaSuccess) return FAST_ENOMEM;
  Ctl h{};
  h.barrier_ns_limit = (unsigned long long)limit_ns;
  int rc = FAST_OK;
  if (cudaMemcpy(d, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK && test_barrier_timeout_launch(d, 2, 0) != 0) rc = FAST_ECUDA;
  if (rc == FAST_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FAST_ECUDA;
  if (rc == FAST_OK && cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FAST_ECUDA;
  cudaFree(d);
  if (rc != FAST_OK) return rc;
  return h.err == kDevErrTimeout ? FAST_ETIMEOUT : FAST_OK;
}

}  // extern "C"
