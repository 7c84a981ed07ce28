// Seeded synthetic sparse-matrix generators (R-MAT, Erdos-Renyi) and the CSR
// assembly they need.  This file produces INPUTS only: it holds none of the
// SpMV / PageRank arithmetic, and both the CUDA library and the CPU oracle
// consume what it writes.
//
// Randomness: every draw is a pure function of (seed, stream, index) through
// the splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014), so results do not depend on the thread
// count or on the machine.
//
// Build: g++ -O3 -fopenmp -shared -fPIC gen.cpp -o libmerbit_gen.so
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <omp.h>

namespace {

inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One 64-bit draw for (seed, stream, index).
inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t index) {
  return mix64(mix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + index);
}

// Stable LSD radix sort of 64-bit keys on their low `bits` bits.
void radix_sort(uint64_t* a, uint64_t* tmp, int64_t n, int bits) {
  const int RB = 12, R = 1 << RB;
  const int passes = (bits + RB - 1) / RB;
  const int nt = std::max(1, omp_get_max_threads());
  std::vector<int64_t> hist((size_t)nt * R);
  uint64_t* src = a;
  uint64_t* dst = tmp;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * RB;
#pragma omp parallel num_threads(nt)
    {
      const int t = omp_get_thread_num();
      const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
      int64_t* h = &hist[(size_t)t * R];
      std::fill(h, h + R, 0);
      for (int64_t i = lo; i < hi; ++i) h[(src[i] >> shift) & (R - 1)]++;
#pragma omp barrier
#pragma omp single
      {
        int64_t s = 0;
        for (int d = 0; d < R; ++d)
          for (int u = 0; u < nt; ++u) {
            int64_t c = hist[(size_t)u * R + d];
            hist[(size_t)u * R + d] = s;
            s += c;
          }
      }
      for (int64_t i = lo; i < hi; ++i) {
        uint64_t v = src[i];
        dst[h[(v >> shift) & (R - 1)]++] = v;
      }
    }
    std::swap(src, dst);
  }
  if (src != a) std::memcpy(a, src, (size_t)n * sizeof(uint64_t));
}

}  // namespace

extern "C" {

// R-MAT edge list (Chakrabarti, Zhan, Faloutsos, SDM 2004): each edge descends
// `scale` levels of the 2x2 quadrant recursion with probabilities a, b, c,
// d = 1-a-b-c.  The quadrant's first bit goes to the source, the second to the
// destination.  Three levels share one 64-bit draw (21 bits each).
// Output key = (dst << scale) | src, i.e. (row, col) of the transposed
// adjacency matrix A^T, so rows are destinations.
void gen_rmat_keys(int scale, int64_t n_edges, double a, double b, double c,
                   uint64_t seed, uint64_t* keys) {
  const uint64_t ONE = 1ull << 21;
  const uint64_t ta = (uint64_t)(a * (double)ONE);
  const uint64_t tab = (uint64_t)((a + b) * (double)ONE);
  const uint64_t tabc = (uint64_t)((a + b + c) * (double)ONE);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n_edges; ++e) {
    uint64_t src = 0, dst = 0, r = 0;
    for (int l = 0; l < scale; ++l) {
      if (l % 3 == 0) r = draw(seed, 1 + (uint64_t)(l / 3), (uint64_t)e);
      const uint64_t u = (r >> (21 * (l % 3))) & (ONE - 1);
      uint64_t sb, db;
      if (u < ta) { sb = 0; db = 0; }
      else if (u < tab) { sb = 0; db = 1; }
      else if (u < tabc) { sb = 1; db = 0; }
      else { sb = 1; db = 1; }
      src = (src << 1) | sb;
      dst = (dst << 1) | db;
    }
    keys[e] = (dst << scale) | src;
  }
}

// Uniform (row, col) draws on an n_rows x n_cols grid; key = row << col_bits | col.
void gen_uniform_keys(int64_t n_rows, int64_t n_cols, int col_bits, int64_t n_draws,
                      uint64_t seed, uint64_t* keys) {
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n_draws; ++e) {
    const uint64_t r = draw(seed, 11, (uint64_t)e) % (uint64_t)n_rows;
    const uint64_t c = draw(seed, 12, (uint64_t)e) % (uint64_t)n_cols;
    keys[e] = (r << col_bits) | c;
  }
}

// Sort keys, drop duplicates and (optionally) keys whose row equals its col.
// Returns the number of keys kept (compacted to the front of `keys`).
int64_t keys_sort_unique(uint64_t* keys, uint64_t* tmp, int64_t n, int col_bits,
                         int row_bits, int drop_diag) {
  if (n == 0) return 0;
  radix_sort(keys, tmp, n, col_bits + row_bits);
  const uint64_t cmask = (1ull << col_bits) - 1;
  int64_t w = 0;
  uint64_t prev = ~0ull;
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t k = keys[i];
    if (k == prev) continue;
    prev = k;
    if (drop_diag && (k >> col_bits) == (k & cmask)) continue;
    keys[w++] = k;
  }
  return w;
}

// Sorted unique keys -> CSR (row_ptr has n_rows + 1 entries).
void keys_to_csr(const uint64_t* keys, int64_t nnz, int col_bits, int64_t n_rows,
                 int32_t* row_ptr, int32_t* col) {
  const uint64_t cmask = (1ull << col_bits) - 1;
  std::fill(row_ptr, row_ptr + n_rows + 1, 0);
  for (int64_t i = 0; i < nnz; ++i) row_ptr[(keys[i] >> col_bits) + 1]++;
  for (int64_t r = 0; r < n_rows; ++r) row_ptr[r + 1] += row_ptr[r];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nnz; ++i) col[i] = (int32_t)(keys[i] & cmask);
}

// Values of the transposed column-stochastic transition matrix P^T: an entry
// in column j (source vertex j) gets 1 / outdeg(j), where outdeg(j) is the
// number of stored entries in column j.
void vals_transition(const int32_t* col, int64_t nnz, int64_t n_cols, double* val) {
  std::vector<int64_t> cnt((size_t)n_cols, 0);
  for (int64_t i = 0; i < nnz; ++i) cnt[(size_t)col[i]]++;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nnz; ++i) val[i] = 1.0 / (double)cnt[(size_t)col[i]];
}

// U(0,1]: (k + 1) / 2^53 with k the top 53 bits of a draw.
void fill_uniform_open0(int64_t n, uint64_t seed, uint64_t stream, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    out[i] = (double)((draw(seed, stream, (uint64_t)i) >> 11) + 1) * 0x1.0p-53;
}

// U[0,1): k / 2^53.
void fill_uniform_open1(int64_t n, uint64_t seed, uint64_t stream, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    out[i] = (double)(draw(seed, stream, (uint64_t)i) >> 11) * 0x1.0p-53;
}

// Raw 64-bit draws (for row selections and lengths done on the Python side).
void fill_draws(int64_t n, uint64_t seed, uint64_t stream, uint64_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = draw(seed, stream, (uint64_t)i);
}

int gen_num_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
