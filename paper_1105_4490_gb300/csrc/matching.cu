// Strengthened diagonal for the matched ordering: a perfect matching of the
// bipartite model of a square pattern, as the paper obtains it for its LU
// experiments (Sec. 5: a heavy-edge matching of the bipartite representation
// augmented to a perfect matching by the Hopcroft-Karp algorithm).  This is
// host preprocessing of the input, outside the ordering's GPU path: the
// ordering (vmo_order_matched) takes the matching as given.
#include <algorithm>
#include <cmath>
#include <vector>

#include "vmo_internal.cuh"

namespace vmo {
namespace {

// Hopcroft-Karp: phases of a breadth-first layering from the free rows, then
// vertex-disjoint shortest augmenting paths found by iterative depth-first
// search along the layers, until no augmenting path is left.
int32_t hopcroft_karp(int32_t m, const int32_t* rowptr, const int32_t* colidx, std::vector<int32_t>& row_mate,
                      std::vector<int32_t>& col_mate) {
  const int32_t kInf = INT32_MAX;
  std::vector<int32_t> dist(m), queue(m), it(m), stack;
  int32_t matched = 0;
  for (int32_t i = 0; i < m; ++i) matched += row_mate[i] >= 0;
  for (;;) {
    // layers: dist of free rows 0; a row reached through its mate's column
    // gets the distance of the row that reached the column + 1
    int32_t qh = 0, qt = 0;
    for (int32_t i = 0; i < m; ++i) {
      if (row_mate[i] < 0) {
        dist[i] = 0;
        queue[qt++] = i;
      } else {
        dist[i] = kInf;
      }
    }
    int32_t free_dist = kInf;  // length (in rows) of the shortest augmenting paths
    while (qh < qt) {
      const int32_t i = queue[qh++];
      if (dist[i] >= free_dist) continue;
      for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
        const int32_t r = col_mate[colidx[t]];
        if (r < 0) {
          free_dist = std::min(free_dist, dist[i] + 1);
        } else if (dist[r] == kInf) {
          dist[r] = dist[i] + 1;
          queue[qt++] = r;
        }
      }
    }
    if (free_dist == kInf) break;
    // augment along disjoint shortest paths
    for (int32_t i = 0; i < m; ++i) it[i] = rowptr[i];
    int32_t found = 0;
    for (int32_t s = 0; s < m; ++s) {
      if (row_mate[s] >= 0 || dist[s] != 0) continue;
      stack.assign(1, s);
      while (!stack.empty()) {
        const int32_t i = stack.back();
        bool advanced = false;
        while (it[i] < rowptr[i + 1]) {
          const int32_t c = colidx[it[i]];
          const int32_t r = col_mate[c];
          if (r < 0 ? dist[i] + 1 == free_dist : dist[r] == dist[i] + 1) {
            if (r < 0) {  // a free column: flip the path on the stack
              for (size_t k = stack.size(); k-- > 0;) {
                const int32_t row = stack[k];
                const int32_t col = colidx[it[row]];
                row_mate[row] = col;
                col_mate[col] = row;
              }
              ++found;
              stack.clear();
              advanced = true;
              break;
            }
            stack.push_back(r);
            advanced = true;
            break;
          }
          ++it[i];
        }
        if (stack.empty()) break;
        if (!advanced) {  // dead end: drop the row from this phase
          dist[i] = kInf;
          stack.pop_back();
          if (!stack.empty()) ++it[stack.back()];
        }
      }
    }
    if (found == 0) break;
    matched += found;
  }
  return matched;
}

}  // namespace
}  // namespace vmo

using namespace vmo;

extern "C" vmo_status vmo_perfect_matching_host(int32_t m, const int32_t* rowptr, const int32_t* colidx,
                                                const float* values, int32_t* match, int32_t* matched) {
  if (m < 0) return invalid("m must be >= 0");
  if (!rowptr || !match || (m > 0 && rowptr[m] > 0 && !colidx)) return invalid("null pointer");
  if (rowptr[0] != 0) return invalid("rowptr[0] must be 0");
  for (int32_t i = 0; i < m; ++i)
    if (rowptr[i + 1] < rowptr[i]) return invalid("rowptr must be nondecreasing");
  const int64_t nnz = rowptr[m];
  for (int64_t t = 0; t < nnz; ++t)
    if (colidx[t] < 0 || colidx[t] >= m) return invalid("column index outside [0, m)");
  if (values)
    for (int64_t t = 0; t < nnz; ++t)
      if (std::isnan(values[t])) return invalid("values must not be NaN");
  std::vector<int32_t> row_mate(m, -1), col_mate(m, -1);
  // heavy-edge start: entries by decreasing |value| (ties: row, then column);
  // without values, rows in order take their first free column
  if (values) {
    std::vector<int64_t> order(nnz);
    std::vector<int32_t> row_of(nnz);
    for (int32_t i = 0; i < m; ++i)
      for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) row_of[t] = i;
    for (int64_t t = 0; t < nnz; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      const float va = std::fabs(values[a]), vb = std::fabs(values[b]);
      if (va != vb) return va > vb;
      if (row_of[a] != row_of[b]) return row_of[a] < row_of[b];
      return colidx[a] < colidx[b];
    });
    for (int64_t t : order) {
      const int32_t i = row_of[t], c = colidx[t];
      if (row_mate[i] < 0 && col_mate[c] < 0) {
        row_mate[i] = c;
        col_mate[c] = i;
      }
    }
  } else {
    for (int32_t i = 0; i < m; ++i)
      for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t)
        if (col_mate[colidx[t]] < 0) {
          row_mate[i] = colidx[t];
          col_mate[colidx[t]] = i;
          break;
        }
  }
  const int32_t size = hopcroft_karp(m, rowptr, colidx, row_mate, col_mate);
  for (int32_t i = 0; i < m; ++i) match[i] = row_mate[i];
  if (matched) *matched = size;
  if (size < m) return unsupported("the pattern is structurally singular: no perfect matching");
  return VMO_OK;
}
