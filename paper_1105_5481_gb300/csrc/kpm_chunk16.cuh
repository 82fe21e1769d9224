// 16-byte FP32 chunk policy (real field): 4 vector columns per thread held
// as 2 packed pairs, twice the threads per row of the 32-byte chunk
// (ChunkF32).  The row layout of a real FP32 block does not depend on the
// chunk width (Rp floats, columns contiguous), so the batched kernel can run
// the same vector blocks with either: the autotuner's threads-per-row choice.
#pragma once

#include "kpm_step.cuh"

namespace kpm {

template <bool NC_ = true>
struct ChunkF32h {
  using T = float;
  static constexpr bool CPLX = false;
  static constexpr bool NC = NC_;
  static constexpr int SC = 4;   // scalars per chunk
  static constexpr int VEC = 4;  // vector columns per chunk
  float2 p[2];

  __device__ __forceinline__ void ld_nc(const float* a) {
    asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(p[0].x), "=f"(p[0].y), "=f"(p[1].x), "=f"(p[1].y)
                 : "l"(a));
  }
  __device__ __forceinline__ void ld_cs(const float* a) {
    asm volatile("ld.global.cs.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(p[0].x), "=f"(p[0].y), "=f"(p[1].x), "=f"(p[1].y)
                 : "l"(a));
  }
  __device__ __forceinline__ void ld_x(const float* a) {
    if constexpr (NC) {
      ld_nc(a);
    } else {
      asm volatile("ld.global.v4.f32 {%0,%1,%2,%3}, [%4];"
                   : "=f"(p[0].x), "=f"(p[0].y), "=f"(p[1].x), "=f"(p[1].y)
                   : "l"(a)
                   : "memory");
    }
  }
  __device__ __forceinline__ void st(float* a) const {
    asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(a), "f"(p[0].x), "f"(p[0].y),
                 "f"(p[1].x), "f"(p[1].y)
                 : "memory");
  }
  __device__ __forceinline__ void zero() { p[0] = p[1] = f2(0.0f); }
  __device__ __forceinline__ void set_neg(const ChunkF32h& w) {
#pragma unroll
    for (int j = 0; j < 2; ++j) p[j] = make_float2(-w.p[j].x, -w.p[j].y);
  }
  __device__ __forceinline__ void half() {
#pragma unroll
    for (int j = 0; j < 2; ++j) p[j] = __fmul2_rn(p[j], f2(0.5f));
  }
  __device__ __forceinline__ void axpy(float d, const ChunkF32h& x) {
    const float2 D = f2(d);
#pragma unroll
    for (int j = 0; j < 2; ++j) p[j] = __ffma2_rn(D, x.p[j], p[j]);
  }
  // real field: the imaginary part of the coefficient is zero
  __device__ __forceinline__ void cmac(float hr, float, const ChunkF32h& x) { axpy(hr, x); }
  struct Acc {
    float2 a[2], ca[2], b[2], cb[2];
  };
  static __device__ __forceinline__ void acc_zero(Acc& s) {
#pragma unroll
    for (int j = 0; j < 2; ++j) s.a[j] = s.ca[j] = s.b[j] = s.cb[j] = f2(0.0f);
  }
  // s.a += x^2, s.b += y x per column, Kahan-compensated
  static __device__ __forceinline__ void acc_add(Acc& s, const ChunkF32h& x, const ChunkF32h& y) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      kahan2(s.a[j], s.ca[j], __fmul2_rn(x.p[j], x.p[j]));
      kahan2(s.b[j], s.cb[j], __fmul2_rn(y.p[j], x.p[j]));
    }
  }
  // sum over the lanes of a warp that hold the same columns, in compensated pairs
  static __device__ __forceinline__ void warp_reduce(Acc& s, int Gt) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll 1
      for (int off = Gt; off < 32; off <<= 1) {
        pair_add2(s.a[j], s.ca[j], shfl2(s.a[j], off), shfl2(s.ca[j], off));
        pair_add2(s.b[j], s.cb[j], shfl2(s.b[j], off), shfl2(s.cb[j], off));
      }
    }
  }
  static __device__ __forceinline__ void acc_out(const Acc& s, double (&A)[VEC], double (&B)[VEC]) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      A[2 * j] = (double)s.a[j].x - (double)s.ca[j].x;
      A[2 * j + 1] = (double)s.a[j].y - (double)s.ca[j].y;
      B[2 * j] = (double)s.b[j].x - (double)s.cb[j].x;
      B[2 * j + 1] = (double)s.b[j].y - (double)s.cb[j].y;
    }
  }
};

}  // namespace kpm
