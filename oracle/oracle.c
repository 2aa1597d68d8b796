/*
 * oracle.c -- plain FP64 CPU oracle of one F.A.S.T. time step (planning +
 * sequential movement).  TEST INFRASTRUCTURE ONLY; see oracle.h.
 *
 * Built with -O2 -ffp-contract=off -fno-fast-math so that every FP64
 * expression below is evaluated exactly as written (one rounding per
 * operation, fma only where fma() is called).  No blocking, fusion or
 * reordering: each function follows the rule it cites, step by step.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11.  One round maps the
 * counter (c0,c1,c2,c3) with key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
 * the key is advanced by the Weyl constants (W0,W1) between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* exp64: the FP64 exponential used for the weights (reading R4).
 *   n = rint(x * log2e)                       (round half to even)
 *   r = fma(-n, LN2_HI, x); r = fma(-n, LN2_LO, r)   (Cody-Waite reduction)
 *   p = sum_{k=0..13} r^k / k!  in Horner form, each step one fma
 *   exp(x) = p * 2^n   (2^n assembled from its exponent bits)
 * LN2_HI is ln 2 truncated to 32 significant bits, so n*LN2_HI is exact for
 * |n| < 2^20; LN2_LO is the double nearest to ln 2 - LN2_HI; the Taylor
 * coefficients are the doubles nearest to 1/k! (one correctly rounded
 * division each).  Valid for |x| <= 700; the weights use |x| <= 12. */
static const double ORC_LOG2E = 0x1.71547652b82fep+0;   /* nearest to log2(e) */
static const double ORC_LN2_HI = 0x1.62e42feep-1;       /* 2977044471 / 2^32  */
static const double ORC_LN2_LO = 0x1.a39ef35793c76p-33; /* ln2 - LN2_HI      */

double orc_exp64(double x) {
  double n = nearbyint(x * ORC_LOG2E);
  double r = fma(-n, ORC_LN2_HI, x);
  r = fma(-n, ORC_LN2_LO, r);
  /* 1/k!, k = 13 .. 0 */
  double p = 1.0 / 6227020800.0;
  p = fma(p, r, 1.0 / 479001600.0);
  p = fma(p, r, 1.0 / 39916800.0);
  p = fma(p, r, 1.0 / 3628800.0);
  p = fma(p, r, 1.0 / 362880.0);
  p = fma(p, r, 1.0 / 40320.0);
  p = fma(p, r, 1.0 / 5040.0);
  p = fma(p, r, 1.0 / 720.0);
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 1.0 / 2.0);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  int64_t e = (int64_t)n + 1023;
  uint64_t bits = (uint64_t)e << 52;
  double scale;
  memcpy(&scale, &bits, sizeof scale);
  return p * scale;
}

/* ------------------------------------------------------------------------- */
/* Reach set (reading R3): offsets (dx,dy) with dx^2+dy^2 <= v^2 (default),
 * <= v^2+v, or max(|dx|,|dy|) <= v; canonical order dy ascending, then dx. */
static int in_reach(int dx, int dy, int v, int reach) {
  int r2 = dx * dx + dy * dy;
  if (reach == ORC_REACH_L2) return r2 <= v * v;
  if (reach == ORC_REACH_L2P) return r2 <= v * v + v;
  return abs(dx) <= v && abs(dy) <= v;
}

int32_t orc_offsets(int32_t v, int32_t reach, int32_t* dx, int32_t* dy) {
  int k = 0;
  for (int y = -v; y <= v; ++y)
    for (int x = -v; x <= v; ++x)
      if (in_reach(x, y, v, reach)) {
        dx[k] = x;
        dy[k] = y;
        ++k;
      }
  return k;
}

/* Path rasterisation (reading R6): L = max(|dx|,|dy|) Moore moves; step s
 * visits (rdiv(s*dx, L), rdiv(s*dy, L)) with rdiv rounding half away from 0. */
static int rdiv(int num, int L) {
  if (num >= 0) return (2 * num + L) / (2 * L);
  return -((-2 * num + L) / (2 * L));
}

int32_t orc_path(int32_t dx, int32_t dy, int32_t* px, int32_t* py) {
  int L = abs(dx) > abs(dy) ? abs(dx) : abs(dy);
  for (int s = 1; s <= L; ++s) {
    px[s - 1] = rdiv(s * dx, L);
    py[s - 1] = rdiv(s * dy, L);
  }
  return L;
}

/* ------------------------------------------------------------------------- */
/* Static floor field (reading R2): shortest 8-neighbour path from any exit
 * cell through non-wall cells, orthogonal step cost 1, diagonal step cost
 * sqrt(2), no corner-cutting rule.  Distances are kept exactly as integer
 * pairs (a, b) meaning a + b*sqrt(2) and compared exactly: the sign of
 * da + db*sqrt(2) is the sign of da when da, db agree in sign, otherwise the
 * comparison of da^2 with 2*db^2 (never equal, sqrt(2) being irrational).
 * S = fl(a + fl(b * sqrt2)). */
static int cmp_ab(int64_t a1, int64_t b1, int64_t a2, int64_t b2) {
  int64_t da = a1 - a2, db = b1 - b2;
  if (da == 0 && db == 0) return 0;
  if (da >= 0 && db >= 0) return 1;
  if (da <= 0 && db <= 0) return -1;
  if (da > 0) return (da * da > 2 * db * db) ? 1 : -1; /* db < 0 */
  return (2 * db * db > da * da) ? 1 : -1;             /* da < 0 < db */
}

typedef struct {
  int32_t a, b, c;
} orc_hitem;

typedef struct {
  orc_hitem* v;
  int64_t n, cap;
} orc_heap;

static int h_less(const orc_hitem* x, const orc_hitem* y) {
  return cmp_ab(x->a, x->b, y->a, y->b) < 0;
}

static int h_push(orc_heap* h, orc_hitem it) {
  if (h->n == h->cap) {
    int64_t nc = h->cap ? h->cap * 2 : 1024;
    orc_hitem* nv = (orc_hitem*)realloc(h->v, (size_t)nc * sizeof(orc_hitem));
    if (!nv) return -1;
    h->v = nv;
    h->cap = nc;
  }
  int64_t i = h->n++;
  h->v[i] = it;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!h_less(&h->v[i], &h->v[p])) break;
    orc_hitem t = h->v[i];
    h->v[i] = h->v[p];
    h->v[p] = t;
    i = p;
  }
  return 0;
}

static orc_hitem h_pop(orc_heap* h) {
  orc_hitem top = h->v[0];
  h->v[0] = h->v[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->n && h_less(&h->v[l], &h->v[m])) m = l;
    if (r < h->n && h_less(&h->v[r], &h->v[m])) m = r;
    if (m == i) break;
    orc_hitem t = h->v[i];
    h->v[i] = h->v[m];
    h->v[m] = t;
    i = m;
  }
  return top;
}

int64_t orc_floor_field(int32_t W, int32_t H, const uint8_t* type, int32_t* a, int32_t* b,
                        double* S) {
  const int64_t C = (int64_t)W * H;
  orc_heap h = {0, 0, 0};
  for (int64_t c = 0; c < C; ++c) {
    a[c] = -1;
    b[c] = -1;
  }
  for (int64_t c = 0; c < C; ++c)
    if (type[c] == ORC_EXIT) {
      a[c] = 0;
      b[c] = 0;
      orc_hitem it = {0, 0, (int32_t)c};
      if (h_push(&h, it)) { free(h.v); return -1; }
    }
  char* done = (char*)calloc((size_t)C, 1);
  if (!done) { free(h.v); return -1; }
  int64_t reached = 0;
  while (h.n > 0) {
    orc_hitem it = h_pop(&h);
    if (done[it.c]) continue;
    if (it.a != a[it.c] || it.b != b[it.c]) continue; /* stale entry */
    done[it.c] = 1;
    ++reached;
    int x = it.c % W, y = it.c / W;
    for (int ny = y - 1; ny <= y + 1; ++ny)
      for (int nx = x - 1; nx <= x + 1; ++nx) {
        if (nx == x && ny == y) continue;
        if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
        int64_t nc = (int64_t)ny * W + nx;
        if (type[nc] == ORC_WALL || done[nc]) continue;
        int diag = (nx != x) && (ny != y);
        int32_t na = it.a + (diag ? 0 : 1);
        int32_t nb = it.b + (diag ? 1 : 0);
        if (a[nc] < 0 || cmp_ab(na, nb, a[nc], b[nc]) < 0) {
          a[nc] = na;
          b[nc] = nb;
          orc_hitem ni = {na, nb, (int32_t)nc};
          if (h_push(&h, ni)) { free(h.v); free(done); return -1; }
        }
      }
  }
  for (int64_t c = 0; c < C; ++c) {
    if (a[c] < 0)
      S[c] = INFINITY;
    else
      S[c] = (double)a[c] + (double)b[c] * M_SQRT2;
  }
  free(h.v);
  free(done);
  return reached;
}

int32_t orc_build_occ(const orc_world* w, int32_t n, const int32_t* cell, int32_t* occ) {
  const int64_t C = (int64_t)w->W * w->H;
  for (int64_t c = 0; c < C; ++c) occ[c] = (w->type[c] == ORC_WALL) ? -2 : -1;
  for (int32_t i = 0; i < n; ++i) {
    int32_t c = cell[i];
    if (c < 0) continue; /* already left */
    if (c >= C) return -1;
    if (w->type[c] != ORC_FREE || occ[c] != -1) return -1;
    occ[c] = i;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Line of sight (reading R3): the straight path (R6) from (x0,y0) to the
 * target, target included, crosses no wall cell. */
static int path_clear(const orc_world* w, int x0, int y0, int dx, int dy) {
  int32_t px[8], py[8];
  int L = orc_path(dx, dy, px, py);
  for (int s = 0; s < L; ++s) {
    int64_t c = (int64_t)(y0 + py[s]) * w->W + (x0 + px[s]);
    if (w->type[c] == ORC_WALL) return 0;
  }
  return 1;
}

/* Planning of one agent (Sec. 1: reads only common data; readings R3-R5):
 * candidates are the offsets of the reach set of the agent's maximum speed
 * (w->v, or w->speed[id] when the agents' speeds differ: Sec. 2 notes that
 * its benchmark gave all agents the same one), in canonical order, whose
 * target is inside the grid, whose path has no wall and whose target is free
 * or is the agent's own cell.  Candidate k gets
 *   d = S[c_k] - S[c0];  x = (-kS) * d;  w_k = exp64(x)
 * (k_other = 0, Sec. 2), the others w_k = 0.  W and the cumulative sums C_k
 * are summed sequentially in canonical order; u is a 53-bit uniform from
 * Philox(key = seed, ctr = (id, t, 0, 0)); the choice is the smallest k with
 * fl(u * W) < C_k, else (rounding) the last k with w_k > 0. */
int32_t orc_plan_agent(const orc_world* w, const int32_t* occ, int32_t cell, int32_t id,
                       int32_t t, double* w_out, double* u_out) {
  int32_t dx[ORC_MAXK], dy[ORC_MAXK];
  double wk[ORC_MAXK], Ck[ORC_MAXK];
  const int32_t v = w->speed ? (int32_t)w->speed[id] : w->v;
  int32_t K = orc_offsets(v, w->reach, dx, dy);
  const int x0 = cell % w->W, y0 = cell / w->W;

  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)t, 0u, 0u};
  uint32_t key[2] = {(uint32_t)w->seed, (uint32_t)(w->seed >> 32)};
  uint32_t rnd[4];
  orc_philox4x32_10(ctr, key, rnd);
  const double u = ((double)(rnd[0] >> 5) * 67108864.0 + (double)(rnd[1] >> 6)) *
                   (1.0 / 9007199254740992.0);

  const double S0 = w->S[cell];
  double Wsum = 0.0;
  for (int k = 0; k < K; ++k) {
    wk[k] = 0.0;
    Ck[k] = Wsum;
    int x = x0 + dx[k], y = y0 + dy[k];
    if (x < 0 || x >= w->W || y < 0 || y >= w->H) continue;
    int64_t c = (int64_t)y * w->W + x;
    if (dx[k] != 0 || dy[k] != 0) {
      if (occ[c] != -1) continue;
      if (!path_clear(w, x0, y0, dx[k], dy[k])) continue;
    }
    double d = w->S[c] - S0;
    double xarg = (-w->kS) * d;
    wk[k] = orc_exp64(xarg);
    Wsum = Wsum + wk[k];
    Ck[k] = Wsum;
  }
  if (w_out)
    for (int k = 0; k < K; ++k) w_out[k] = wk[k];
  if (u_out) *u_out = u;

  const double r = u * Wsum;
  int chosen = -1;
  for (int k = 0; k < K; ++k)
    if (wk[k] > 0.0 && r < Ck[k]) {
      chosen = k;
      break;
    }
  if (chosen < 0)
    for (int k = K - 1; k >= 0; --k)
      if (wk[k] > 0.0) {
        chosen = k;
        break;
      }
  return (y0 + dy[chosen]) * w->W + (x0 + dx[chosen]);
}

/* Agents per chunk of the timed planning loop (Sec. 2 gives the rule): about
 * an equal share per thread, capped at 32767 agents, at least one. */
static int32_t orc_chunk_agents(int32_t n, int32_t threads) {
  const int32_t share = n / threads;
  return share < 1 ? 1 : (share > 32767 ? 32767 : share);
}

/* All agents.  With threads > 1 (the timed CPU baseline) the threads take
 * chunks of consecutive agents on demand, each from a shared counter, until
 * none is left; the result does not depend on who plans which agent (every
 * draw is keyed by the agent's id and the step). */
void orc_plan_all(const orc_world* w, const int32_t* occ, int32_t n, const int32_t* id,
                  const int32_t* cell, int32_t t, int32_t* desired, int32_t threads) {
  int32_t next = 0;
  const int32_t chunk = threads > 1 ? orc_chunk_agents(n, threads) : (n > 0 ? n : 1);
#ifdef _OPENMP
#pragma omp parallel num_threads(threads > 1 ? threads : 1)
#endif
  for (;;) {
    int32_t begin;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
    {
      begin = next;
      next += chunk;
    }
    if (begin >= n) break;
    const int32_t end = n - begin < chunk ? n : begin + chunk;
    for (int32_t i = begin; i < end; ++i)
      desired[i] = cell[i] < 0 ? -1 : orc_plan_agent(w, occ, cell[i], id[i], t, 0, 0);
  }
}

/* ------------------------------------------------------------------------- */
/* Movement order (reading R7): a fresh pseudo-random permutation of the
 * agents every step, as a keyed permutation of the 24-bit agent ids.  The
 * step keys k0..k3 are the four words of Philox(key = seed, ctr =
 * (0, t, 2, 0)); the id is split into 12-bit halves (L, R) and passed through
 * a four-round Feistel network (Luby and Rackoff, 1988)
 *   (L, R) <- (R, L ^ (fmix32(R ^ k_i) & 0xFFF)),  i = 0..3,
 * fmix32 being the finalizer of MurmurHash3 (A. Appleby).  Every Feistel
 * round is invertible, so pi_t is a permutation of [0, 2^24) and no two agents
 * share a priority.  Agents move in ascending pi_t(id). */
static uint32_t orc_fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

static void orc_step_keys(uint64_t seed, int32_t t, uint32_t k[4]) {
  uint32_t ctr[4] = {0u, (uint32_t)t, 2u, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, k);
}

static uint32_t orc_feistel24(uint32_t id, const uint32_t k[4]) {
  uint32_t L = (id >> 12) & 0xFFFu, R = id & 0xFFFu;
  for (int i = 0; i < 4; ++i) {
    uint32_t nl = R;
    uint32_t nr = L ^ (orc_fmix32(R ^ k[i]) & 0xFFFu);
    L = nl;
    R = nr;
  }
  return (L << 12) | R;
}

uint32_t orc_move_priority(uint64_t seed, int32_t id, int32_t t) {
  uint32_t k[4];
  orc_step_keys(seed, t, k);
  return orc_feistel24((uint32_t)id, k);
}

typedef struct {
  uint32_t p;
  int32_t i;
} orc_pi;

static int cmp_pi(const void* x, const void* y) {
  uint32_t a = ((const orc_pi*)x)->p, b = ((const orc_pi*)y)->p;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* Sequential movement (Sec. 1; reading R7).  One agent after the other, in
 * priority order, walks the path (R6) to its desired cell; it stops before a
 * cell that is a wall or occupied at that moment, leaves the simulation as
 * soon as it enters an exit cell (which stays free), and otherwise ends on
 * the last cell it reached.  occ is updated at once for the next agent. */
int32_t orc_move(const orc_world* w, int32_t* occ, int32_t n, const int32_t* id, int32_t* cell,
                 const int32_t* desired, int32_t t) {
  orc_pi* order = (orc_pi*)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_pi));
  int32_t m = 0;
  uint32_t k[4];
  orc_step_keys(w->seed, t, k);
  for (int32_t i = 0; i < n; ++i)
    if (cell[i] >= 0) {
      order[m].p = orc_feistel24((uint32_t)id[i], k);
      order[m].i = i;
      ++m;
    }
  qsort(order, (size_t)m, sizeof(orc_pi), cmp_pi);
  int32_t left = 0;
  for (int32_t j = 0; j < m; ++j) {
    const int32_t i = order[j].i;
    const int32_t c0 = cell[i], tgt = desired[i];
    if (tgt == c0) continue;
    const int x0 = c0 % w->W, y0 = c0 / w->W;
    const int dx = tgt % w->W - x0, dy = tgt / w->W - y0;
    int32_t px[8], py[8];
    int L = orc_path(dx, dy, px, py);
    int32_t cur = c0;
    int gone = 0;
    for (int s = 0; s < L; ++s) {
      int32_t nxt = (y0 + py[s]) * w->W + (x0 + px[s]);
      if (w->type[nxt] == ORC_WALL || occ[nxt] != -1) break;
      cur = nxt;
      if (w->type[cur] == ORC_EXIT) {
        gone = 1;
        break;
      }
    }
    occ[c0] = -1;
    if (gone) {
      cell[i] = -1;
      ++left;
    } else {
      occ[cur] = i;
      cell[i] = cur;
    }
  }
  free(order);
  return left;
}

/* ------------------------------------------------------------------------- */
/* splitmix64 output function (S. Vigna), used only to digest states. */
static uint64_t orc_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Sum over the entries with val >= 0 (agents still in the simulation). */
uint64_t orc_digest(int32_t n, const int32_t* id, const int32_t* val) {
  uint64_t s = 0;
  for (int32_t i = 0; i < n; ++i)
    if (val[i] >= 0) s += orc_mix(((uint64_t)(uint32_t)id[i] << 32) | (uint64_t)(uint32_t)val[i]);
  return s;
}

static double orc_now(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int32_t orc_run(const orc_world* w, int32_t* occ, int32_t n, const int32_t* id, int32_t* cell,
                int32_t t0, int32_t n_steps, int32_t threads, int32_t* desired_last,
                uint64_t* dig_cell, uint64_t* dig_des, int32_t* alive, double* plan_s,
                double* move_s) {
  int32_t* desired = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t left = 0;
  double tp = 0.0, tm = 0.0;
  for (int32_t s = 0; s < n_steps; ++s) {
    const int32_t t = t0 + s;
    double a0 = orc_now();
    orc_plan_all(w, occ, n, id, cell, t, desired, threads);
    double a1 = orc_now();
    if (dig_des) dig_des[s] = orc_digest(n, id, desired);
    left += orc_move(w, occ, n, id, cell, desired, t);
    double a2 = orc_now();
    tp += a1 - a0;
    tm += a2 - a1;
    if (dig_cell) dig_cell[s] = orc_digest(n, id, cell);
    if (alive) {
      int32_t m = 0;
      for (int32_t i = 0; i < n; ++i) m += cell[i] >= 0;
      alive[s] = m;
    }
  }
  if (desired_last) memcpy(desired_last, desired, (size_t)n * sizeof(int32_t));
  if (plan_s) *plan_s = tp;
  if (move_s) *move_s = tm;
  free(desired);
  return left;
}
