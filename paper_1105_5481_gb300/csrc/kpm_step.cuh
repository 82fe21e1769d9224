// Fused Chebyshev step: v_{n+1} = 2 H~ v_n - v_{n-1} (Eq. (rn)) with the two
// moment dot products of the doubling identities, one pass over the vectors.
//
// Vector blocks are N x Rp, row-major with the Rp vectors of a site
// contiguous.  A row is split into G chunks; a group of Gt consecutive threads
// owns one row (Gt = G, or a slice of a wider row selected by blockIdx.y),
// each thread one chunk, so every access to a vector is one coalesced vector
// load or store per thread:
//   FP64 path (ChunkF64): 16-byte chunks, 2 real columns or 1 complex column
//     stored (re, im).
//   FP32 path (ChunkF32): 32-byte chunks moved with 256-bit loads/stores, 8
//     real columns or 4 complex columns stored split as (re0..re3, im0..im3),
//     so that the complex arithmetic runs on packed f32x2 FMAs.
// v_n is read through the read-only path, v_{n-1} is streamed and v_{n+1} is
// written over it in place.  The traversal (StepArgs) makes every neighbour
// row of v_n come from L1/L2 within about one pass of its first use.
//
// Moments: per vector column, A = <v_n|v_n> and B = Re<v_{n+1}|v_n> are
// accumulated per thread (FP64 on the FP64 path; Kahan-compensated f32x2 sums
// promoted to FP64 once per thread on the FP32 path), reduced over the lanes
// that share a column with warp shuffles, over the warps in shared memory in a
// fixed order, and written as one [2][Rp] FP64 partial per CTA.  The cross-CTA
// sum is done later by a separate fixed-order kernel, so results are bitwise
// reproducible for a given launch shape.
#pragma once

#include <atomic>
#include <type_traits>

#include "kpm_internal.h"

// Sliding register window along x in the line traversal (1: on).
#ifndef KPM_STEP_XWINDOW
#define KPM_STEP_XWINDOW 1
#endif

// Minimum resident CTAs per SM requested from the register allocator
// (stencil steps; CSR/ELL steps).
#ifndef KPM_STEP_MIN_BLOCKS
#define KPM_STEP_MIN_BLOCKS 2
#endif
#ifndef KPM_SPARSE_MIN_BLOCKS
#define KPM_SPARSE_MIN_BLOCKS 3
#endif

namespace kpm {

// ================================================================ chunk policies
// Vector rows of v_n are read with ld_x: through the read-only path (NC) when
// no thread writes them during the kernel (one fused step per launch), or with
// plain coherent loads when the same launch writes them in an earlier step
// (the batched persistent kernel).
//
// FP64: 16 bytes = 2 doubles.
template <bool CPLX_, bool NC_ = true>
struct ChunkF64 {
  using T = double;
  static constexpr bool CPLX = CPLX_;
  static constexpr bool NC = NC_;
  static constexpr int SC = 2;                // scalars per chunk
  static constexpr int VEC = CPLX ? 1 : 2;    // vector columns per chunk
  double v[2];

  __device__ __forceinline__ void ld_nc(const double* p) {
    const double2 q = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = q.x; v[1] = q.y;
  }
  __device__ __forceinline__ void ld_cs(const double* p) {
    const double2 q = __ldcs(reinterpret_cast<const double2*>(p));
    v[0] = q.x; v[1] = q.y;
  }
  __device__ __forceinline__ void ld_x(const double* p) {
    if constexpr (NC) {
      ld_nc(p);
    } else {
      const double2 q = *reinterpret_cast<const double2*>(p);
      v[0] = q.x; v[1] = q.y;
    }
  }
  __device__ __forceinline__ void st(double* p) const {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
  // from shared memory (16-byte aligned)
  __device__ __forceinline__ void ld_shared(const double* p) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
  __device__ __forceinline__ void zero() { v[0] = v[1] = 0.0; }
  __device__ __forceinline__ void set_neg(const ChunkF64& w) { v[0] = -w.v[0]; v[1] = -w.v[1]; }
  __device__ __forceinline__ void half() { v[0] *= 0.5; v[1] *= 0.5; }
  // this += d x (real d)
  __device__ __forceinline__ void axpy(double d, const ChunkF64& x) {
    v[0] = fma(d, x.v[0], v[0]);
    v[1] = fma(d, x.v[1], v[1]);
  }
  // this += h x (h = hr + i hi; the real field ignores hi)
  __device__ __forceinline__ void cmac(double hr, double hi, const ChunkF64& x) {
    if constexpr (CPLX) {
      v[0] = fma(hr, x.v[0], v[0]);
      v[0] = fma(-hi, x.v[1], v[0]);
      v[1] = fma(hr, x.v[1], v[1]);
      v[1] = fma(hi, x.v[0], v[1]);
    } else {
      axpy(hr, x);
    }
  }
  struct Acc {
    double a[VEC], b[VEC];
  };
  static __device__ __forceinline__ void acc_zero(Acc& s) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) s.a[k] = s.b[k] = 0.0;
  }
  // s.a_k += |x_k|^2,  s.b_k += Re(conj(y_k) x_k), accumulated by FMAs only
  // (the FP64 pipe is the step's limit: one instruction per product term)
  static __device__ __forceinline__ void acc_add(Acc& s, const ChunkF64& x, const ChunkF64& y) {
    if constexpr (CPLX) {
      s.a[0] = fma(x.v[1], x.v[1], fma(x.v[0], x.v[0], s.a[0]));
      s.b[0] = fma(y.v[1], x.v[1], fma(y.v[0], x.v[0], s.b[0]));
    } else {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        s.a[k] = fma(x.v[k], x.v[k], s.a[k]);
        s.b[k] = fma(y.v[k], x.v[k], s.b[k]);
      }
    }
  }
  static __device__ __forceinline__ void acc_out(const Acc& s, double (&A)[VEC], double (&B)[VEC]) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) { A[k] = s.a[k]; B[k] = s.b[k]; }
  }
  // sum over the lanes of a warp that hold the same columns (xor offsets Gt .. 16)
  static __device__ __forceinline__ void warp_reduce(Acc& s, int Gt) {
    for (int off = Gt; off < 32; off <<= 1) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        s.a[k] += __shfl_xor_sync(0xffffffffu, s.a[k], off);
        s.b[k] += __shfl_xor_sync(0xffffffffu, s.b[k], off);
      }
    }
  }
};

// FP32: 32 bytes = 8 floats held as 4 packed pairs.  Complex: p[0] = (re0,
// re1), p[1] = (re2, re3), p[2] = (im0, im1), p[3] = (im2, im3); real: p[j] =
// columns (2j, 2j+1).
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {  // a - b
  return __ffma2_rn(b, f2(-1.0f), a);
}
// (s1, c1) += (s2, c2) for compensated pairs whose value is s - c: the sum of
// the leading parts with its exact rounding error (TwoSum, Knuth), the error
// folded into the compensation.
__device__ __forceinline__ void pair_add2(float2& s1, float2& c1, float2 s2, float2 c2) {
  const float2 t = __fadd2_rn(s1, s2);
  const float2 bb = sub2(t, s1);
  const float2 err = __fadd2_rn(sub2(s1, sub2(t, bb)), sub2(s2, bb));  // s1 + s2 = t + err
  c1 = sub2(__fadd2_rn(c1, c2), err);
  s1 = t;
}

// scalar form of pair_add2: (s1, c1) += (s2, c2), s - c being the value
__device__ __forceinline__ void pair_add(float& s1, float& c1, float s2, float c2) {
  const float t = __fadd_rn(s1, s2);
  const float bb = __fsub_rn(t, s1);
  const float err = __fadd_rn(__fsub_rn(s1, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
  c1 = __fsub_rn(__fadd_rn(c1, c2), err);
  s1 = t;
}

__device__ __forceinline__ float2 shfl2(float2 v, int off) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, off), __shfl_xor_sync(0xffffffffu, v.y, off));
}

// Kahan step: s += v with compensation c
__device__ __forceinline__ void kahan2(float2& s, float2& c, float2 v) {
  const float2 y = sub2(v, c);
  const float2 t = __fadd2_rn(s, y);
  c = sub2(sub2(t, s), y);
  s = t;
}

template <bool CPLX_, bool NC_ = true>
struct ChunkF32 {
  using T = float;
  static constexpr bool CPLX = CPLX_;
  static constexpr bool NC = NC_;
  static constexpr int SC = 8;
  static constexpr int VEC = CPLX ? 4 : 8;
  float2 p[4];

  __device__ __forceinline__ void ld_nc(const float* a) {
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(p[0].x), "=f"(p[0].y), "=f"(p[1].x), "=f"(p[1].y), "=f"(p[2].x),
                   "=f"(p[2].y), "=f"(p[3].x), "=f"(p[3].y)
                 : "l"(a));
  }
  __device__ __forceinline__ void ld_cs(const float* a) {
    asm volatile("ld.global.cs.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(p[0].x), "=f"(p[0].y), "=f"(p[1].x), "=f"(p[1].y), "=f"(p[2].x),
                   "=f"(p[2].y), "=f"(p[3].x), "=f"(p[3].y)
                 : "l"(a));
  }
  __device__ __forceinline__ void ld_x(const float* a) {
    if constexpr (NC) {
      ld_nc(a);
    } else {
      asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=f"(p[0].x), "=f"(p[0].y), "=f"(p[1].x), "=f"(p[1].y), "=f"(p[2].x),
                     "=f"(p[2].y), "=f"(p[3].x), "=f"(p[3].y)
                   : "l"(a)
                   : "memory");
    }
  }
  // from shared memory (16-byte aligned)
  __device__ __forceinline__ void ld_shared(const float* a) {
    const float4 u = *reinterpret_cast<const float4*>(a);
    const float4 w = *reinterpret_cast<const float4*>(a + 4);
    p[0] = make_float2(u.x, u.y); p[1] = make_float2(u.z, u.w);
    p[2] = make_float2(w.x, w.y); p[3] = make_float2(w.z, w.w);
  }
  __device__ __forceinline__ void st(float* a) const {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(a), "f"(p[0].x),
                 "f"(p[0].y), "f"(p[1].x), "f"(p[1].y), "f"(p[2].x), "f"(p[2].y), "f"(p[3].x),
                 "f"(p[3].y)
                 : "memory");
  }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = f2(0.0f);
  }
  __device__ __forceinline__ void set_neg(const ChunkF32& w) {
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = make_float2(-w.p[j].x, -w.p[j].y);
  }
  __device__ __forceinline__ void half() {
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = __fmul2_rn(p[j], f2(0.5f));
  }
  __device__ __forceinline__ void axpy(float d, const ChunkF32& x) {
    const float2 D = f2(d);
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = __ffma2_rn(D, x.p[j], p[j]);
  }
  __device__ __forceinline__ void cmac(float hr, float hi, const ChunkF32& x) {
    if constexpr (CPLX) {
      const float2 H = f2(hr), Hp = f2(hi), Hn = f2(-hi);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        p[j] = __ffma2_rn(H, x.p[j], p[j]);              // re += hr re_x
        p[j] = __ffma2_rn(Hn, x.p[j + 2], p[j]);         // re -= hi im_x
        p[j + 2] = __ffma2_rn(H, x.p[j + 2], p[j + 2]);  // im += hr im_x
        p[j + 2] = __ffma2_rn(Hp, x.p[j], p[j + 2]);     // im += hi re_x
      }
    } else {
      axpy(hr, x);
    }
  }
  struct Acc {
    float2 a[VEC / 2], ca[VEC / 2], b[VEC / 2], cb[VEC / 2];
  };
  static __device__ __forceinline__ void acc_zero(Acc& s) {
#pragma unroll
    for (int j = 0; j < VEC / 2; ++j) s.a[j] = s.ca[j] = s.b[j] = s.cb[j] = f2(0.0f);
  }
  static __device__ __forceinline__ void acc_add(Acc& s, const ChunkF32& x, const ChunkF32& y) {
    if constexpr (CPLX) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float2 a2 = __ffma2_rn(x.p[j + 2], x.p[j + 2], __fmul2_rn(x.p[j], x.p[j]));
        const float2 b2 = __ffma2_rn(y.p[j + 2], x.p[j + 2], __fmul2_rn(y.p[j], x.p[j]));
        kahan2(s.a[j], s.ca[j], a2);
        kahan2(s.b[j], s.cb[j], b2);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        kahan2(s.a[j], s.ca[j], __fmul2_rn(x.p[j], x.p[j]));
        kahan2(s.b[j], s.cb[j], __fmul2_rn(y.p[j], x.p[j]));
      }
    }
  }
  // sum over the lanes of a warp that hold the same columns, in compensated
  // FP32 pairs (FP32 pipes; accuracy of about 2^-44 relative)
  static __device__ __forceinline__ void warp_reduce(Acc& s, int Gt) {
#pragma unroll
    for (int j = 0; j < VEC / 2; ++j) {
#pragma unroll 1
      for (int off = Gt; off < 32; off <<= 1) {
        pair_add2(s.a[j], s.ca[j], shfl2(s.a[j], off), shfl2(s.ca[j], off));
        pair_add2(s.b[j], s.cb[j], shfl2(s.b[j], off), shfl2(s.cb[j], off));
      }
    }
  }
  static __device__ __forceinline__ void acc_out(const Acc& s, double (&A)[VEC], double (&B)[VEC]) {
#pragma unroll
    for (int j = 0; j < VEC / 2; ++j) {
      A[2 * j] = (double)s.a[j].x - (double)s.ca[j].x;
      A[2 * j + 1] = (double)s.a[j].y - (double)s.ca[j].y;
      B[2 * j] = (double)s.b[j].x - (double)s.cb[j].x;
      B[2 * j + 1] = (double)s.b[j].y - (double)s.cb[j].y;
    }
  }
};

template <typename T>
__device__ __forceinline__ void scal_from_block(const ScalarBlock* sc, T& hr, T& hi, T& du);
template <>
__device__ __forceinline__ void scal_from_block<float>(const ScalarBlock* sc, float& hr, float& hi,
                                                       float& du) {
  hr = sc->hu_re_f; hi = sc->hu_im_f; du = sc->du_f;
}
template <>
__device__ __forceinline__ void scal_from_block<double>(const ScalarBlock* sc, double& hr,
                                                        double& hi, double& du) {
  hr = sc->hu_re; hi = sc->hu_im; du = sc->du;
}

// ================================================================ operators
// Matrix-free hypercubic stencil: forward bond (i, i+e_d) carries the scaled
// hopping h_{i,d}; the backward bond (i, i-e_d) carries conj(h_{i-e_d,d}).
template <class CH, int DIMS, bool HAS_HOP, bool HAS_DS>
struct StencilOp {
  using T = typename CH::T;
  static constexpr bool CPLX = CH::CPLX;
  static constexpr bool kLines = DIMS >= 2;
  static constexpr int kDims = DIMS;
  static constexpr int kMinBlocks = KPM_STEP_MIN_BLOCKS;
  static constexpr bool kPairReduce = true;

  // Neighbour offsets along d >= 1 depend only on the lattice line (y, z):
  // computed once per chunk of passes.
  struct LineCtx {
    int row0;                // row of x = 0 on this line
    int df[DIMS], db[DIMS];  // row deltas of the forward / backward neighbour
    bool hf[DIMS], hb[DIMS];
    bool valid;
  };

  __device__ __forceinline__ LineCtx line_ctx(const StepArgs& a, int line) const {
    LineCtx k{};
    k.valid = line < a.lines;
    k.row0 = line * a.line_len;
    int co[3] = {0, 0, 0};
    if constexpr (DIMS == 2) co[1] = line;
    if constexpr (DIMS == 3) {
      co[1] = line % a.line_L1;
      co[2] = line / a.line_L1;
    }
#pragma unroll
    for (int d2 = 1; d2 < DIMS; ++d2) {
      const int L = a.geom.L[d2], s = a.geom.stride[d2], x = co[d2];
      const bool per = a.geom.periodic[d2] != 0;
      k.hf[d2] = (x + 1 < L) || per;
      k.df[d2] = (x + 1 < L) ? s : (per ? -(L - 1) * s : 0);
      k.hb[d2] = (x > 0) || per;
      k.db[d2] = (x > 0) ? -s : (per ? (L - 1) * s : 0);
    }
    return k;
  }

  // The shared core: diagonal, hoppings and the 2*DIMS neighbour rows.  With
  // WIN the x-neighbour rows (d = 0) are supplied by the caller (xm: x-1,
  // xp: x+1) from its sliding register window instead of being loaded.
  template <bool WIN = false>
  __device__ __forceinline__ void core(const StepArgs& a, int i, const int (&jf)[DIMS],
                                       const int (&jb)[DIMS], const bool (&hf)[DIMS],
                                       const bool (&hb)[DIMS], const T* __restrict__ Xc,
                                       const CH& xi, CH& acc, T hu_r, T hu_i, T du,
                                       const CH* xm = nullptr, const CH* xp = nullptr) const {
    const T d = HAS_DS ? __ldg(reinterpret_cast<const T*>(a.ds) + i) : du;
    acc.axpy(d, xi);
    T fr[DIMS], fi[DIMS], br[DIMS], bi[DIMS];
#pragma unroll
    for (int d2 = 0; d2 < DIMS; ++d2) {
      if constexpr (HAS_HOP) {
        const T* hs = reinterpret_cast<const T*>(a.hs);
        if constexpr (CPLX) {
          using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
          const T2 f = __ldg(reinterpret_cast<const T2*>(hs) + ((size_t)i * DIMS + d2));
          const T2 bk = __ldg(reinterpret_cast<const T2*>(hs) + ((size_t)jb[d2] * DIMS + d2));
          fr[d2] = f.x;
          fi[d2] = f.y;
          br[d2] = bk.x;
          bi[d2] = -bk.y;
        } else {
          fr[d2] = __ldg(hs + (size_t)i * DIMS + d2);
          br[d2] = __ldg(hs + (size_t)jb[d2] * DIMS + d2);
          fi[d2] = bi[d2] = T(0);
        }
      } else {
        fr[d2] = hu_r; fi[d2] = hu_i; br[d2] = hu_r; bi[d2] = -hu_i;
      }
      if (!hf[d2]) { fr[d2] = T(0); fi[d2] = T(0); }
      if (!hb[d2]) { br[d2] = T(0); bi[d2] = T(0); }
    }
    const size_t rowS = (size_t)a.G * CH::SC;
    CH xf[DIMS], xb[DIMS];
#pragma unroll
    for (int d2 = WIN ? 1 : 0; d2 < DIMS; ++d2) {
      xf[d2].ld_x(Xc + (size_t)jf[d2] * rowS);
      xb[d2].ld_x(Xc + (size_t)jb[d2] * rowS);
    }
    if constexpr (WIN) {
      acc.cmac(fr[0], fi[0], *xp);
      acc.cmac(br[0], bi[0], *xm);
    }
#pragma unroll
    for (int d2 = WIN ? 1 : 0; d2 < DIMS; ++d2) {
      acc.cmac(fr[d2], fi[d2], xf[d2]);
      acc.cmac(br[d2], bi[d2], xb[d2]);
    }
  }

  // Row indices of the x-neighbours of position cx (periodic wrap, or the
  // row itself with a zero hopping at an open edge).
  __device__ __forceinline__ void x_neighbours(const StepArgs& a, int i, int cx, int& jf0,
                                               int& jb0) const {
    const int L0 = a.line_len;
    const bool per0 = a.geom.periodic[0] != 0;
    jf0 = (cx + 1 < L0) ? i + 1 : (per0 ? i - (L0 - 1) : i);
    jb0 = (cx > 0) ? i - 1 : (per0 ? i + (L0 - 1) : i);
  }

  // Line traversal with the x-neighbours taken from the caller's window.
  __device__ __forceinline__ void apply_line_win(const StepArgs& a, int i, int cx,
                                                 const LineCtx& k, const T* __restrict__ Xc,
                                                 const CH& xi, const CH& xm, const CH& xp,
                                                 CH& acc, T hu_r, T hu_i, T du) const {
    int jf[DIMS], jb[DIMS];
    bool hf[DIMS], hb[DIMS];
    const int L0 = a.line_len;
    const bool per0 = a.geom.periodic[0] != 0;
    hf[0] = (cx + 1 < L0) || per0;
    hb[0] = (cx > 0) || per0;
    x_neighbours(a, i, cx, jf[0], jb[0]);
#pragma unroll
    for (int d2 = 1; d2 < DIMS; ++d2) {
      jf[d2] = i + k.df[d2];
      jb[d2] = i + k.db[d2];
      hf[d2] = k.hf[d2];
      hb[d2] = k.hb[d2];
    }
    core<true>(a, i, jf, jb, hf, hb, Xc, xi, acc, hu_r, hu_i, du, &xm, &xp);
  }

  // Row i at position cx on a line described by k (line traversal).
  __device__ __forceinline__ void apply_line(const StepArgs& a, int i, int cx, const LineCtx& k,
                                             const T* __restrict__ Xc, const CH& xi, CH& acc,
                                             T hu_r, T hu_i, T du) const {
    int jf[DIMS], jb[DIMS];
    bool hf[DIMS], hb[DIMS];
    const int L0 = a.line_len;
    const bool per0 = a.geom.periodic[0] != 0;
    hf[0] = (cx + 1 < L0) || per0;
    jf[0] = (cx + 1 < L0) ? i + 1 : (per0 ? i - (L0 - 1) : i);
    hb[0] = (cx > 0) || per0;
    jb[0] = (cx > 0) ? i - 1 : (per0 ? i + (L0 - 1) : i);
#pragma unroll
    for (int d2 = 1; d2 < DIMS; ++d2) {
      jf[d2] = i + k.df[d2];
      jb[d2] = i + k.db[d2];
      hf[d2] = k.hf[d2];
      hb[d2] = k.hb[d2];
    }
    core(a, i, jf, jb, hf, hb, Xc, xi, acc, hu_r, hu_i, du);
  }

  // Row i in natural order: coordinates decoded from the index.
  __device__ __forceinline__ void apply(const StepArgs& a, int64_t i64, const T* __restrict__ Xc,
                                        const CH& xi, CH& acc, T hu_r, T hu_i, T du) const {
    const int i = (int)i64;
    int jf[DIMS], jb[DIMS];
    bool hf[DIMS], hb[DIMS];
    int rem = i;
#pragma unroll
    for (int d2 = 0; d2 < DIMS; ++d2) {
      const int L = a.geom.L[d2], s = a.geom.stride[d2];
      const int x = rem % L;
      rem /= L;
      const bool per = a.geom.periodic[d2] != 0;
      hf[d2] = (x + 1 < L) || per;
      jf[d2] = (x + 1 < L) ? i + s : (per ? i - (L - 1) * s : i);
      hb[d2] = (x > 0) || per;
      jb[d2] = (x > 0) ? i - s : (per ? i + (L - 1) * s : i);
    }
    core(a, i, jf, jb, hf, hb, Xc, xi, acc, hu_r, hu_i, du);
  }
};

// CSR rows: y_i = du x_i + sum_k vals[k] x_{col[k]}
template <class CH>
struct CsrOp {
  using T = typename CH::T;
  static constexpr bool CPLX = CH::CPLX;
  static constexpr bool kLines = false;
  static constexpr int kMinBlocks = KPM_SPARSE_MIN_BLOCKS;
  static constexpr bool kPairReduce = false;
  struct LineCtx {};
  __device__ __forceinline__ void hop(const T* V, int64_t k, T& hr, T& hi) const {
    if constexpr (CPLX) {
      using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
      const T2 h = __ldg(reinterpret_cast<const T2*>(V) + k);
      hr = h.x;
      hi = h.y;
    } else {
      hr = __ldg(V + k);
      hi = T(0);
    }
  }
  __device__ __forceinline__ void apply(const StepArgs& a, int64_t i, const T* __restrict__ Xc,
                                        const CH& xi, CH& acc, T, T, T du) const {
    acc.axpy(du, xi);
    const int64_t k0 = __ldg(a.rowptr + i), k1 = __ldg(a.rowptr + i + 1);
    const T* V = reinterpret_cast<const T*>(a.vals);
    const size_t rowS = (size_t)a.G * CH::SC;
    int64_t k = k0;
    for (; k + 4 <= k1; k += 4) {
      int j[4];
      T hr[4], hi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        j[u] = __ldg(a.col + k + u);
        hop(V, k + u, hr[u], hi[u]);
      }
      CH xj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xj[u].ld_x(Xc + (size_t)j[u] * rowS);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc.cmac(hr[u], hi[u], xj[u]);
    }
    for (; k < k1; ++k) {
      const int j = __ldg(a.col + k);
      T hr, hi;
      hop(V, k, hr, hi);
      CH xj;
      xj.ld_x(Xc + (size_t)j * rowS);
      acc.cmac(hr, hi, xj);
    }
  }
};

// Padded ELL rows (built by the library from a CSR with short rows): row i
// holds exactly W (even) entries col[i*W + k], vals[i*W + k]; padding entries
// point at row i with value 0.  No row pointer, fixed trip count, and every
// neighbour load of the row is issued in one batch.
template <class CH, int W>
struct EllOp {
  using T = typename CH::T;
  static constexpr bool CPLX = CH::CPLX;
  static constexpr bool kLines = false;
  static constexpr int kMinBlocks = KPM_SPARSE_MIN_BLOCKS;
  static constexpr bool kPairReduce = false;
  struct LineCtx {};
  __device__ __forceinline__ void apply(const StepArgs& a, int64_t i, const T* __restrict__ Xc,
                                        const CH& xi, CH& acc, T, T, T du) const {
    acc.axpy(du, xi);
    const int2* cp = reinterpret_cast<const int2*>(a.col + (size_t)i * W);
    int j[W];
    T hr[W], hi[W];
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
      const int2 c2 = __ldg(cp + k);
      j[2 * k] = c2.x;
      j[2 * k + 1] = c2.y;
    }
    if constexpr (CPLX) {
      using T4 = typename std::conditional<sizeof(T) == 4, float4, double4>::type;
      if constexpr (sizeof(T) == 4) {
        const float4* vp = reinterpret_cast<const float4*>(a.vals) + (size_t)i * (W / 2);
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
          const float4 v = __ldg(vp + k);
          hr[2 * k] = v.x; hi[2 * k] = v.y; hr[2 * k + 1] = v.z; hi[2 * k + 1] = v.w;
        }
      } else {
        const double2* vp = reinterpret_cast<const double2*>(a.vals) + (size_t)i * W;
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const double2 v = __ldg(vp + k);
          hr[k] = v.x; hi[k] = v.y;
        }
      }
      (void)sizeof(T4);
    } else {
      const T* vp = reinterpret_cast<const T*>(a.vals) + (size_t)i * W;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        hr[k] = __ldg(vp + k);
        hi[k] = T(0);
      }
    }
    const size_t rowS = (size_t)a.G * CH::SC;
    CH xj[W];
#pragma unroll
    for (int k = 0; k < W; ++k) xj[k].ld_x(Xc + (size_t)j[k] * rowS);
#pragma unroll
    for (int k = 0; k < W; ++k) acc.cmac(hr[k], hi[k], xj[k]);
  }
};

// ================================================================ the fused step
// Rows of one step handled by CTA `cta` of `ncta` CTAs working on the same
// vectors: chunks of a.chunk passes taken in a stride-ncta loop (see
// StepArgs).  Accumulates this thread's moment dots into s.
// SWEEP = false: always the forward chunk order (a.reverse ignored).
// UNROLL4: four-pass chunks that stay on one lattice line are fully unrolled,
// the x-window rotating through registers instead of being moved (measured:
// 5 % faster in the batched persistent kernel, 5 % slower in the single-solve
// step, where the compiler's hoisting across passes costs more than it saves).
template <class CH, int MODE, class OP, bool SWEEP = true, bool UNROLL4 = false>
__device__ __forceinline__ void step_rows(const StepArgs& a, const OP& op, int cta, int ncta,
                                          int ycol, typename CH::Acc& s, bool first = false) {
  using T = typename CH::T;
  constexpr int SC = CH::SC;
  const int Gt = a.Gt;
  const int t = threadIdx.x;
  const int c = ycol * Gt + t % Gt;       // chunk within the row
  const int q = t / Gt;
  const int spi = blockDim.x / Gt;
  const size_t rowS = (size_t)a.G * SC;
  const T* __restrict__ Xc = reinterpret_cast<const T*>(a.x) + (size_t)c * SC;
  const T* Wc = reinterpret_cast<const T*>(a.w) + (size_t)c * SC;
  T* Yc = reinterpret_cast<T*>(a.y) + (size_t)c * SC;
  T hu_r, hu_i, du;
  scal_from_block<T>(a.sc, hu_r, hu_i, du);

  const int Lx = a.line_len;
  const int u = a.chunk;
  const int64_t nchunks = (a.passes + u - 1) / u;
  for (int64_t kc = cta; kc < nchunks; kc += ncta) {
    const int64_t ch = (SWEEP && a.reverse) ? nchunks - 1 - kc : kc;
    const int64_t p_beg = ch * (int64_t)u;
    const int np = (int)min((int64_t)u, a.passes - p_beg);
    // line traversal: x and the line context advance incrementally
    int cx = 0, blk = 0;
    typename OP::LineCtx lctx{};
    if constexpr (OP::kLines) {
      if (Lx > 0) {
        const int pb = (int)p_beg;  // passes < 2^31
        blk = pb / Lx;
        cx = pb - blk * Lx;
        lctx = op.line_ctx(a, blk * spi + q);
      }
    }
#if KPM_STEP_XWINDOW
    if constexpr (OP::kLines) {
      if (Lx > 0) {
        // line traversal with a sliding window (x-1, x, x+1) of v_n rows in
        // registers: one new x-neighbour row per pass instead of three rows
        const size_t rowS2 = rowS;
        auto pass = [&](int i, int cxp, const CH& xm, const CH& x0, const CH& xp) {
          const size_t base = (size_t)i * rowS2;
          CH acc;
          if (MODE == MODE_STEP || (MODE == MODE_DYN && !first)) {
            CH wv;
            wv.ld_cs(Wc + base);
            acc.set_neg(wv);
          } else {
            acc.zero();
          }
          op.apply_line_win(a, i, cxp, lctx, Xc, x0, xm, xp, acc, hu_r, hu_i, du);
          if (MODE == MODE_FIRST || (MODE == MODE_DYN && first)) acc.half();
          acc.st(Yc + base);
          if constexpr (MODE != MODE_SPMV) CH::acc_add(s, x0, acc);
        };
        if (UNROLL4 && np == 4 && cx + 4 <= Lx && lctx.valid) {
          // four positions on one line: the window rotates through unrolled
          // registers instead of being moved
          CH r[6];
          int jf0, jb0;
          op.x_neighbours(a, lctx.row0 + cx, cx, jf0, jb0);
          r[0].ld_x(Xc + (size_t)jb0 * rowS2);
          r[1].ld_x(Xc + (size_t)(lctx.row0 + cx) * rowS2);
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) {
            const int c2 = cx + jp, i = lctx.row0 + c2;
            op.x_neighbours(a, i, c2, jf0, jb0);
            r[jp + 2].ld_x(Xc + (size_t)jf0 * rowS2);
            pass(i, c2, r[jp], r[jp + 1], r[jp + 2]);
          }
          continue;
        }
        bool have = false;
        CH xm, x0, xp;
        for (int jp = 0; jp < np; ++jp) {
          if (jp > 0 && ++cx == Lx) {
            cx = 0;
            ++blk;
            lctx = op.line_ctx(a, blk * spi + q);
            have = false;
          }
          if (!lctx.valid) continue;
          const int i = lctx.row0 + cx;
          int jf0, jb0;
          op.x_neighbours(a, i, cx, jf0, jb0);
          if (!have) {
            xm.ld_x(Xc + (size_t)jb0 * rowS2);
            x0.ld_x(Xc + (size_t)i * rowS2);
            have = true;
          } else {
            xm = x0;
            x0 = xp;
          }
          xp.ld_x(Xc + (size_t)jf0 * rowS2);
          pass(i, cx, xm, x0, xp);
        }
        continue;
      }
    }
#endif
    for (int jp = 0; jp < np; ++jp) {
      int64_t i;
      bool line_mode = false;
      if constexpr (OP::kLines) {
        if (Lx > 0) {
          line_mode = true;
          if (jp > 0 && ++cx == Lx) {
            cx = 0;
            ++blk;
            lctx = op.line_ctx(a, blk * spi + q);
          }
          if (!lctx.valid) continue;
          i = lctx.row0 + cx;
        }
      }
      if (!line_mode) {
        i = (p_beg + jp) * spi + q;
        if (i >= a.n) continue;
      }
      const size_t base = (size_t)i * rowS;
      CH xi, acc;
      xi.ld_x(Xc + base);
      if (MODE == MODE_STEP || (MODE == MODE_DYN && !first)) {
        CH wv;
        wv.ld_cs(Wc + base);
        acc.set_neg(wv);
      } else {
        acc.zero();
      }
      if constexpr (OP::kLines) {
        if (line_mode) op.apply_line(a, (int)i, cx, lctx, Xc, xi, acc, hu_r, hu_i, du);
        else op.apply(a, i, Xc, xi, acc, hu_r, hu_i, du);
      } else {
        op.apply(a, i, Xc, xi, acc, hu_r, hu_i, du);
      }
      if (MODE == MODE_FIRST || (MODE == MODE_DYN && first)) acc.half();
      acc.st(Yc + base);
      if constexpr (MODE != MODE_SPMV) CH::acc_add(s, xi, acc);
    }
  }
}

// CTA-wide sum of the threads' moment dots: lanes sharing a column are
// combined with warp shuffles in the chunk's own precision (compensated FP32
// pairs on the FP32 path), then summed over the warps in shared memory `red`
// in warp order (FP64 path: in FP64; FP32 path: still in compensated pairs,
// and only the 2 Rp column totals are converted to FP64, because GB300's FP64
// pipe, at 1/64 of the FP32 rate, made per-thread conversions a visible tail
// of every step).
// PAIRS = false keeps the FP64 cross-warp stage on the FP32 path (the sparse
// operators, whose 80-register budget fares better with it).
// Writes dst[which * Rp + ycol * Rt + col] for which in {A, B} and the Rt
// columns of this column slice.  All threads of the CTA must call it.
template <class CH, bool PAIRS = true>
__device__ __forceinline__ void cta_reduce(const StepArgs& a, typename CH::Acc s, int ycol,
                                           double* red, double* dst) {
  constexpr int VEC = CH::VEC;
  const int Gt = a.Gt;
  const int t = threadIdx.x;
  const int cl = t % Gt, q = t / Gt, spi = blockDim.x / Gt;
  if (Gt < 32) CH::warp_reduce(s, Gt);
  if constexpr (PAIRS && sizeof(typename CH::T) == 4) {
    const int lane = t & 31, warp = t >> 5;
    bool rep;
    int qrep, nq;
    if (Gt < 32) {
      rep = lane < Gt;
      qrep = warp;
      nq = blockDim.x >> 5;
    } else {
      rep = true;
      qrep = q;
      nq = spi;
    }
    const int Rp = a.Rp, Rt = Gt * VEC;
    // per (qrep, cl): for each float2 j of the chunk, the pairs (a, ca, b, cb)
    float2* r2 = reinterpret_cast<float2*>(red);
    if (rep) {
      float2* o = r2 + (size_t)(qrep * Gt + cl) * 2 * VEC;
#pragma unroll
      for (int j = 0; j < VEC / 2; ++j) {
        o[4 * j + 0] = s.a[j];
        o[4 * j + 1] = s.ca[j];
        o[4 * j + 2] = s.b[j];
        o[4 * j + 3] = s.cb[j];
      }
    }
    __syncthreads();
    const float* rf = reinterpret_cast<const float*>(red);
    for (int o = t; o < 2 * Rt; o += blockDim.x) {
      const int which = o / Rt, col = o % Rt, cc = col / VEC, k = col % VEC;
      const int j = k / 2, h = k % 2;
      float sum = 0.0f, comp = 0.0f;
      for (int qq = 0; qq < nq; ++qq) {
        const float* e = rf + ((size_t)(qq * Gt + cc) * 2 * VEC + 4 * j + 2 * which) * 2;
        pair_add(sum, comp, e[h], e[2 + h]);
      }
      dst[which * Rp + ycol * Rt + col] = (double)sum - (double)comp;
    }
  } else {
    double dA[VEC], dB[VEC];
    CH::acc_out(s, dA, dB);
    const int lane = t & 31, warp = t >> 5;
    bool rep;
    int qrep, nq;
    if (Gt < 32) {
      rep = lane < Gt;
      qrep = warp;
      nq = blockDim.x >> 5;
    } else {
      rep = true;
      qrep = q;
      nq = spi;
    }
    if (rep) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        red[((qrep * Gt + cl) * 2 + 0) * VEC + k] = dA[k];
        red[((qrep * Gt + cl) * 2 + 1) * VEC + k] = dB[k];
      }
    }
    __syncthreads();
    const int Rp = a.Rp, Rt = Gt * VEC;
    for (int o = t; o < 2 * Rt; o += blockDim.x) {
      const int which = o / Rt, col = o % Rt, cc = col / VEC, k = col % VEC;
      double sum = 0.0;
      for (int qq = 0; qq < nq; ++qq) sum += red[((qq * Gt + cc) * 2 + which) * VEC + k];
      dst[which * Rp + ycol * Rt + col] = sum;
    }
  }
}

// Programmatic dependent launch: consecutive short steps of a chain are
// launched with programmatic stream serialisation, so the next step's CTAs
// are set up while this step finishes; each step waits for its
// predecessor's completion (and memory) before touching any data.  Without
// the launch attribute both instructions are no-ops.  Measured on the 2D
// L = 32 FP64 solve (64 KB vector blocks): 4.37 -> 3.98 us per step; on the
// 134 MB blocks of the 3D L = 64 FP32 solve no gain (75.45 -> 75.57 us), so
// only steps on vector blocks up to KPM_PDL_MAX_BYTES use it.
#ifndef KPM_PDL
#define KPM_PDL 1
#endif
#ifndef KPM_PDL_MAX_BYTES
#define KPM_PDL_MAX_BYTES (16u << 20)
#endif

template <class CH, int MODE, class OP>
__global__ void __launch_bounds__(256, OP::kMinBlocks) cheb_step_kernel(const StepArgs a) {
#if KPM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
  const OP op;
  typename CH::Acc s;
  CH::acc_zero(s);
  step_rows<CH, MODE, OP>(a, op, blockIdx.x, gridDim.x, blockIdx.y, s);
  if constexpr (MODE != MODE_SPMV) {
    extern __shared__ double red[];
    cta_reduce<CH, OP::kPairReduce>(a, s, blockIdx.y, red,
                                    a.partial + (size_t)blockIdx.x * 2 * a.Rp);
  }
}

__host__ __device__ inline size_t step_smem_bytes(int Gt, int block, int vec) {
  const int nq = Gt < 32 ? block / 32 : block / Gt;
  return (size_t)nq * Gt * 2 * vec * sizeof(double);
}

// Raises a kernel's dynamic shared-memory limit above the default 48 KB, once
// per kernel (Tag: the kernel's own template instance) and device (ordinals
// below 64), so that no attribute is set while a stream is being captured.
template <class Tag, class K>
cudaError_t allow_smem(K kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <class CH, int MODE, class OP>
cudaError_t launch_one(const StepArgs& a, const LaunchCfg& cfg, cudaStream_t st) {
  const size_t smem = MODE == MODE_SPMV ? 0 : step_smem_bytes(a.Gt, cfg.block, CH::VEC);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const size_t block_bytes =
      (size_t)a.n * a.Rp * sizeof(typename CH::T) * (CH::CPLX ? 2 : 1);
  if (KPM_PDL && MODE == MODE_STEP && block_bytes <= KPM_PDL_MAX_BYTES) {
    // a regular step follows the first step or another step of the same chain
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(cfg.grid, a.G / a.Gt);
    lc.blockDim = dim3(cfg.block);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, cheb_step_kernel<CH, MODE, OP>, a);
  }
  cheb_step_kernel<CH, MODE, OP><<<dim3(cfg.grid, a.G / a.Gt), cfg.block, smem, st>>>(a);
  return cudaGetLastError();
}

template <class CH, int MODE, class OP>
int occupancy_one(int block, int Gt) {
  int nb = 0;
  const size_t smem = MODE == MODE_SPMV ? 0 : step_smem_bytes(Gt, block, CH::VEC);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cheb_step_kernel<CH, MODE, OP>, block, smem);
  return nb;
}

}  // namespace kpm
