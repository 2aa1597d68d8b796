// floor_field.cpp -- exact static floor field of a grid, on the host.
//
// S(c) = length of the shortest 8-neighbour path from c to any exit cell
// through non-wall cells, orthogonal steps costing 1 and diagonal steps
// sqrt(2).  Lengths are kept as integer pairs (a, b) = (orthogonal steps,
// diagonal steps), S = a + b*sqrt(2), and compared exactly.
//
// Algorithm: Dial's bucket queue with unit-wide buckets on floor(S), where
// floor(a + b*sqrt(2)) = a + isqrt(2 b^2) exactly.  Every edge costs at least
// 1, so no cell of bucket k can lower another cell of bucket k: when bucket k
// is reached all its cells are final, and each relaxation lands in bucket
// k+1 or k+2 (edge costs < 2), so three buckets in a ring suffice.  Inside a
// bucket the exact (a, b) minimum of every cell is kept by exact comparison.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

namespace fastgb {

namespace {

// sign of (a1 + b1*sqrt2) - (a2 + b2*sqrt2)
inline int compare_exact(int64_t a1, int64_t b1, int64_t a2, int64_t b2) {
  const int64_t da = a1 - a2, db = b1 - b2;
  if (da == 0 && db == 0) return 0;
  if (da >= 0 && db >= 0) return 1;
  if (da <= 0 && db <= 0) return -1;
  const int64_t l = da * da, r = 2 * db * db;  // |da| vs |db|*sqrt2
  if (da > 0) return l > r ? 1 : -1;
  return r > l ? 1 : -1;
}

inline int64_t isqrt64(int64_t v) {
  int64_t x = (int64_t)std::sqrt((double)v);
  while (x * x > v) --x;
  while ((x + 1) * (x + 1) <= v) ++x;
  return x;
}

inline int64_t floor_len(int64_t a, int64_t b) { return a + isqrt64(2 * b * b); }

}  // namespace

// type: [W*H] 0 free / 1 wall / 2 exit.  Outputs a, b: [W*H], -1 for walls and
// cells no exit can be reached from.  Returns the number of reachable cells.
int64_t exact_floor_field(int32_t W, int32_t H, const uint8_t* type, int32_t* a, int32_t* b) {
  const int64_t C = (int64_t)W * H;
  std::vector<uint8_t> final_(C, 0);
  for (int64_t c = 0; c < C; ++c) a[c] = b[c] = -1;
  std::vector<int32_t> ring[3];
  for (int64_t c = 0; c < C; ++c)
    if (type[c] == 2) {
      a[c] = b[c] = 0;
      ring[0].push_back((int32_t)c);
    }
  int64_t reached = 0;
  int64_t k = 0;
  int64_t pending = (int64_t)ring[0].size();
  static const int ddx[8] = {1, -1, 0, 0, 1, 1, -1, -1};
  static const int ddy[8] = {0, 0, 1, -1, 1, -1, 1, -1};
  while (pending > 0) {
    std::vector<int32_t>& cur = ring[k % 3];
    for (size_t i = 0; i < cur.size(); ++i) {
      const int32_t c = cur[i];
      --pending;
      if (final_[c]) continue;
      if (floor_len(a[c], b[c]) != k) continue;  // superseded entry
      final_[c] = 1;
      ++reached;
      const int x = c % W, y = c / W;
      for (int d = 0; d < 8; ++d) {
        const int nx = x + ddx[d], ny = y + ddy[d];
        if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
        const int64_t n = (int64_t)ny * W + nx;
        if (type[n] == 1 || final_[n]) continue;
        const int32_t na = a[c] + (d < 4 ? 1 : 0), nb = b[c] + (d < 4 ? 0 : 1);
        if (a[n] < 0 || compare_exact(na, nb, a[n], b[n]) < 0) {
          a[n] = na;
          b[n] = nb;
          const int64_t kk = floor_len(na, nb);
          ring[kk % 3].push_back((int32_t)n);
          ++pending;
        }
      }
    }
    cur.clear();
    ++k;
  }
  return reached;
}

// A caller's floor field S (doubles, row-major) as exact step counts: for
// every reachable cell the integers 0 <= a, b <= max_ab with
// S == fl(a + fl(b * sqrt2)), the rounding the FP64 rule applies to (a, b).
// sqrt2 being irrational, two pairs with b <= 2^15 differ by more than about
// 1e-5, far above the rounding of S, so the pair is unique when it exists.
// Walls: a = b = -1 whatever S says.  Exit cells must have S == 0 (a = b = 0);
// a free cell with S == +inf is one no exit can be reached from (a = b = -1);
// any other free cell must have a positive S of that form.  Returns the index
// of the first cell that breaks these rules, or -1.
int64_t decompose_field(int32_t W, int32_t H, const uint8_t* type, const double* S, int32_t max_ab,
                        int32_t* a, int32_t* b) {
  const double kR2 = 1.4142135623730951;  // the double nearest sqrt2
  std::vector<double> tb((size_t)max_ab + 1);
  std::vector<std::pair<double, int32_t>> fr((size_t)max_ab + 1);
  for (int32_t j = 0; j <= max_ab; ++j) {
    tb[j] = (double)j * kR2;
    fr[j] = {tb[j] - std::floor(tb[j]), j};
  }
  std::sort(fr.begin(), fr.end());
  // does b = j give an integer a in range with fl(a + tb[j]) == s?
  auto fits = [&](double s, int32_t j, int32_t* ao) {
    if (j < 0 || j > max_ab || tb[j] > s + 0.5) return false;
    const double af = std::nearbyint(s - tb[j]);
    if (af < 0.0 || af > (double)max_ab) return false;
    if ((double)(int32_t)af + tb[j] != s) return false;
    *ao = (int32_t)af;
    return true;
  };
  const int64_t C = (int64_t)W * H;
  int32_t hint = 0;
  for (int64_t c = 0; c < C; ++c) {
    a[c] = b[c] = -1;
    const double s = S[c];
    if (type[c] == 1) continue;
    if (type[c] == 2) {
      if (s != 0.0) return c;
      a[c] = b[c] = 0;
      continue;
    }
    if (std::isinf(s) && s > 0.0) continue;  // no exit reachable: a wall
    if (!(s > 0.0) || !std::isfinite(s)) return c;
    int32_t ao = -1, bo = -1;
    // neighbouring cells mostly differ by a step or two in b
    for (int32_t d = 0; d <= 4 && bo < 0; ++d) {
      if (fits(s, hint + d, &ao)) bo = hint + d;
      else if (d > 0 && fits(s, hint - d, &ao)) bo = hint - d;
    }
    if (bo < 0) {
      // every b whose fractional part of fl(b sqrt2) is within 1e-6 of S's
      const double f = s - std::floor(s);
      for (double g : {f, f - 1.0, f + 1.0}) {
        auto it = std::lower_bound(fr.begin(), fr.end(), std::make_pair(g - 1e-6, (int32_t)-1));
        for (; it != fr.end() && it->first <= g + 1e-6 && bo < 0; ++it)
          if (fits(s, it->second, &ao)) bo = it->second;
      }
    }
    if (bo < 0) return c;
    a[c] = ao;
    b[c] = bo;
    hint = bo;
  }
  return -1;
}

}  // namespace fastgb
