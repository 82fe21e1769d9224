// Counter-based random start vectors (the stochastic trace of Sec. II-A-3):
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) applied to
// (seed ^ (0x9E3779B97F4A7C15 * (1 + stream))) + counter.  Entry (s, r, i) of
// an N x R block uses stream 0 and counter (s R + r) N + i: Rademacher +-1
// from the top bit (real field) or exp(2 pi i u), u = (u64 >> 11) 2^-53
// (complex field).
#pragma once

#include <stdint.h>

namespace kpm {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long draw(unsigned long long seed, int stream,
                                                   unsigned long long counter) {
  const unsigned long long key = seed ^ (0x9E3779B97F4A7C15ULL * (unsigned long long)(1 + stream));
  return splitmix64(key + counter);
}

// Scalar offsets of the real and imaginary parts of entry (i, r) of an N x Rp
// complex block.  FP64 blocks interleave (re, im); FP32 blocks store 32-byte
// chunks of 4 columns split as (re0..re3, im0..im3).
template <typename T>
__device__ __forceinline__ void cplx_offsets(int64_t i, int r, int Rp, int64_t& re, int64_t& im) {
  if (sizeof(T) == 8) {
    re = 2 * (i * Rp + r);
    im = re + 1;
  } else {
    re = i * 2 * Rp + (r / 4) * 8 + (r % 4);
    im = re + 4;
  }
}

// Entry (i, r) of realisation s of the start block, r < R: Rademacher +-1
// (real field) or a unit phase (complex field; im is left untouched for the
// real field).
template <typename T, bool CPLX>
__device__ __forceinline__ void random_value(int64_t n, int R, unsigned long long seed,
                                             unsigned long long s, int64_t i, int r, T& re,
                                             T& im) {
  const unsigned long long ctr = (s * (unsigned long long)R + (unsigned long long)r) *
                                     (unsigned long long)n + (unsigned long long)i;
  const unsigned long long z = draw(seed, 0, ctr);
  if (CPLX) {
    const double u = (double)(z >> 11) * 0x1.0p-53;
    if (sizeof(T) == 8) {
      double sv, cv;
      sincospi(2.0 * u, &sv, &cv);
      re = (T)cv;
      im = (T)sv;
    } else {
      float sv, cv;
      sincospif(2.0f * (float)u, &sv, &cv);
      re = (T)cv;
      im = (T)sv;
    }
  } else {
    re = (z >> 63) ? T(-1) : T(1);
  }
}

// Writes element e = i * Rp + r of the start block (zero for padded columns r >= R).
template <typename T, bool CPLX>
__device__ __forceinline__ void random_entry(T* v0, int64_t n, int Rp, int R,
                                             unsigned long long seed, unsigned long long s,
                                             int64_t e) {
  const int64_t i = e / Rp;
  const int r = (int)(e % Rp);
  int64_t ore = e, oim = e;
  if (CPLX) cplx_offsets<T>(i, r, Rp, ore, oim);
  if (r >= R) {
    if (CPLX) { v0[ore] = T(0); v0[oim] = T(0); }
    else v0[e] = T(0);
    return;
  }
  T re, im = T(0);
  random_value<T, CPLX>(n, R, seed, s, i, r, re, im);
  v0[ore] = re;
  if (CPLX) v0[oim] = im;
}

}  // namespace kpm
