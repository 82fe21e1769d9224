// Integer helpers of the tiled kernels: division of row indices by lattice
// sides with one multiply-high, and rounding of byte counts.
#pragma once

#include <stddef.h>

namespace kpm {

// Division of 31-bit numerators by a fixed divisor d >= 1 with one
// multiply-high (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994, Thm. 4.2): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(n, m) + n) >> l.  The sum
// stays below 2^32 for n < 2^31.
struct FastDiv {
  unsigned m;
  int l;
};
__host__ __device__ inline FastDiv fast_div(unsigned d) {
  int l = 0;
  while (l < 31 && (1u << l) < d) ++l;
  const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return {(unsigned)m, l};
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
  return (__umulhi(n, f.m) + n) >> f.l;
}

__host__ __device__ inline size_t stg_round(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace kpm
