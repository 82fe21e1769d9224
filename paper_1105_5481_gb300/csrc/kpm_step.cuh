// Fused Chebyshev step: v_{n+1} = 2 H~ v_n - v_{n-1} (Eq. (rn)) with the two
// moment dot products of the doubling identities, one pass over the vectors.
//
// Vector blocks are N x Rp, row-major with the Rp vectors of a site contiguous
// (complex entries interleaved re, im).  A row is split into G 16-byte chunks;
// a group of Gt consecutive threads owns one row (Gt = G, or a slice of a
// wider row selected by blockIdx.y), each thread one chunk, so every load and
// store of a vector is a coalesced 128-bit access.  Each CTA
// walks a contiguous range of rows, so the lattice neighbours at +-1 and
// +-L_x rows are re-read from L1 while the far neighbours (+-L_x L_y rows)
// come from L2; v_n is read through the read-only path, v_{n-1} is streamed
// and v_{n+1} is written over it in place.
//
// Moments: per vector column, A = <v_n|v_n> and B = Re<v_{n+1}|v_n> are
// accumulated per thread (FP64 on the FP64 path; FP32 partial sums over
// PROMOTE rows promoted into FP64 on the FP32 path), reduced over the lanes
// that share a column with warp shuffles, over the warps in shared memory in a
// fixed order, and written as one [2][Rp] FP64 partial per CTA.  The cross-CTA
// sum is done later by a separate fixed-order kernel, so results are bitwise
// reproducible for a given launch shape.
#pragma once

#include "kpm_internal.h"

namespace kpm {

constexpr int PROMOTE = 8;  // FP32 rows summed before promotion to FP64

__device__ __forceinline__ void ld16_nc(const float* p, float (&r)[4]) {
  float4 q = __ldg(reinterpret_cast<const float4*>(p));
  r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
}
__device__ __forceinline__ void ld16_nc(const double* p, double (&r)[2]) {
  double2 q = __ldg(reinterpret_cast<const double2*>(p));
  r[0] = q.x; r[1] = q.y;
}
__device__ __forceinline__ void ld16_cs(const float* p, float (&r)[4]) {
  float4 q = __ldcs(reinterpret_cast<const float4*>(p));
  r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
}
__device__ __forceinline__ void ld16_cs(const double* p, double (&r)[2]) {
  double2 q = __ldcs(reinterpret_cast<const double2*>(p));
  r[0] = q.x; r[1] = q.y;
}
__device__ __forceinline__ void st16(float* p, const float (&r)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void st16(double* p, const double (&r)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
}

template <typename T>
struct Traits {
  static constexpr int SC = 16 / sizeof(T);  // scalars per chunk
};

// acc += h * x for one chunk (h complex when CPLX; conj handled by caller via hi sign)
template <typename T, bool CPLX>
__device__ __forceinline__ void mac(T (&acc)[Traits<T>::SC], T hr, T hi, const T (&x)[Traits<T>::SC]) {
  constexpr int SC = Traits<T>::SC;
  if constexpr (CPLX) {
#pragma unroll
    for (int k = 0; k < SC / 2; ++k) {
      const T xr = x[2 * k], xi = x[2 * k + 1];
      acc[2 * k] = fma(hr, xr, acc[2 * k]);
      acc[2 * k] = fma(-hi, xi, acc[2 * k]);
      acc[2 * k + 1] = fma(hr, xi, acc[2 * k + 1]);
      acc[2 * k + 1] = fma(hi, xr, acc[2 * k + 1]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < SC; ++k) acc[k] = fma(hr, x[k], acc[k]);
  }
}

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

// ---------------------------------------------------------------- operators
// Matrix-free hypercubic stencil: forward bond (i, i+e_d) carries the scaled
// hopping h_{i,d}; the backward bond (i, i-e_d) carries conj(h_{i-e_d,d}).
template <typename T, bool CPLX, int DIMS, bool HAS_HOP, bool HAS_DS>
struct StencilOp {
  static constexpr int SC = Traits<T>::SC;
  __device__ __forceinline__ void apply(const StepArgs& a, int64_t i64, int c, const T* __restrict__ X,
                                        const T (&xi)[SC], T (&acc)[SC], T hu_r, T hu_i,
                                        T du) const {
    const int i = (int)i64;
    const T d = HAS_DS ? __ldg(reinterpret_cast<const T*>(a.ds) + i) : du;
#pragma unroll
    for (int k = 0; k < SC; ++k) acc[k] = fma(d, xi[k], acc[k]);
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
    // hoppings
    T fr[DIMS], fi[DIMS], br[DIMS], bi[DIMS];
#pragma unroll
    for (int d2 = 0; d2 < DIMS; ++d2) {
      if constexpr (HAS_HOP) {
        const T* hs = reinterpret_cast<const T*>(a.hs);
        if constexpr (CPLX) {
          fr[d2] = __ldg(hs + 2 * ((size_t)i * DIMS + d2));
          fi[d2] = __ldg(hs + 2 * ((size_t)i * DIMS + d2) + 1);
          br[d2] = __ldg(hs + 2 * ((size_t)jb[d2] * DIMS + d2));
          bi[d2] = -__ldg(hs + 2 * ((size_t)jb[d2] * DIMS + d2) + 1);
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
    const int G = a.G;
    T xf[DIMS][SC], xb[DIMS][SC];
#pragma unroll
    for (int d2 = 0; d2 < DIMS; ++d2) {
      ld16_nc(X + ((size_t)jf[d2] * G + c) * SC, xf[d2]);
      ld16_nc(X + ((size_t)jb[d2] * G + c) * SC, xb[d2]);
    }
#pragma unroll
    for (int d2 = 0; d2 < DIMS; ++d2) {
      mac<T, CPLX>(acc, fr[d2], fi[d2], xf[d2]);
      mac<T, CPLX>(acc, br[d2], bi[d2], xb[d2]);
    }
  }
};

// CSR rows: y_i = du x_i + sum_k vals[k] x_{col[k]}
template <typename T, bool CPLX>
struct CsrOp {
  static constexpr int SC = Traits<T>::SC;
  __device__ __forceinline__ void apply(const StepArgs& a, int64_t i, int c, const T* __restrict__ X,
                                        const T (&xi)[SC], T (&acc)[SC], T, T, T du) const {
#pragma unroll
    for (int k = 0; k < SC; ++k) acc[k] = fma(du, xi[k], acc[k]);
    const int64_t k0 = __ldg(a.rowptr + i), k1 = __ldg(a.rowptr + i + 1);
    const T* V = reinterpret_cast<const T*>(a.vals);
    const int G = a.G;
    int64_t k = k0;
    for (; k + 4 <= k1; k += 4) {
      int j[4];
      T hr[4], hi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        j[u] = __ldg(a.col + k + u);
        if constexpr (CPLX) {
          hr[u] = __ldg(V + 2 * (k + u));
          hi[u] = __ldg(V + 2 * (k + u) + 1);
        } else {
          hr[u] = __ldg(V + k + u);
          hi[u] = T(0);
        }
      }
      T xj[4][SC];
#pragma unroll
      for (int u = 0; u < 4; ++u) ld16_nc(X + ((size_t)j[u] * G + c) * SC, xj[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) mac<T, CPLX>(acc, hr[u], hi[u], xj[u]);
    }
    for (; k < k1; ++k) {
      const int j = __ldg(a.col + k);
      T hr, hi;
      if constexpr (CPLX) {
        hr = __ldg(V + 2 * k);
        hi = __ldg(V + 2 * k + 1);
      } else {
        hr = __ldg(V + k);
        hi = T(0);
      }
      T xj[SC];
      ld16_nc(X + ((size_t)j * G + c) * SC, xj);
      mac<T, CPLX>(acc, hr, hi, xj);
    }
  }
};

// ---------------------------------------------------------------- the fused step
template <typename T, bool CPLX, int MODE, class OP>
__global__ void __launch_bounds__(256) cheb_step_kernel(const StepArgs a) {
  constexpr int SC = Traits<T>::SC;
  constexpr int VEC = CPLX ? SC / 2 : SC;
  constexpr bool F32 = sizeof(T) == 4;
  const OP op;
  const int Gt = a.Gt;
  const int t = threadIdx.x;
  const int cl = t % Gt;                  // chunk within this CTA's column slice
  const int c = blockIdx.y * Gt + cl;     // chunk within the row
  const int q = t / Gt;
  const int spi = blockDim.x / Gt;
  const int G = a.G;
  const int64_t s0 = (int64_t)blockIdx.x * a.sites_per_cta;
  const int64_t s1 = min(s0 + (int64_t)a.sites_per_cta, a.n);
  const T* __restrict__ X = reinterpret_cast<const T*>(a.x);
  const T* W = reinterpret_cast<const T*>(a.w);
  T* Y = reinterpret_cast<T*>(a.y);
  T hu_r, hu_i, du;
  scal_from_block<T>(a.sc, hu_r, hu_i, du);

  double dA[VEC], dB[VEC];
  T fA[VEC], fB[VEC];
#pragma unroll
  for (int k = 0; k < VEC; ++k) { dA[k] = 0.0; dB[k] = 0.0; fA[k] = T(0); fB[k] = T(0); }
  int cnt = 0;

  for (int64_t i = s0 + q; i < s1; i += spi) {
    const size_t base = ((size_t)i * G + c) * SC;
    T xi[SC], acc[SC];
    ld16_nc(X + base, xi);
    if constexpr (MODE == MODE_STEP) {
      T wv[SC];
      ld16_cs(W + base, wv);
#pragma unroll
      for (int k = 0; k < SC; ++k) acc[k] = -wv[k];
    } else {
#pragma unroll
      for (int k = 0; k < SC; ++k) acc[k] = T(0);
    }
    op.apply(a, i, c, X, xi, acc, hu_r, hu_i, du);
    if constexpr (MODE == MODE_FIRST) {
#pragma unroll
      for (int k = 0; k < SC; ++k) acc[k] *= T(0.5);
    }
    st16(Y + base, acc);
    if constexpr (MODE != MODE_SPMV) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        T a2, b2;
        if constexpr (CPLX) {
          a2 = fma(xi[2 * k], xi[2 * k], xi[2 * k + 1] * xi[2 * k + 1]);
          b2 = fma(acc[2 * k], xi[2 * k], acc[2 * k + 1] * xi[2 * k + 1]);
        } else {
          a2 = xi[k] * xi[k];
          b2 = acc[k] * xi[k];
        }
        if constexpr (F32) {
          fA[k] += a2;
          fB[k] += b2;
        } else {
          dA[k] += a2;
          dB[k] += b2;
        }
      }
      if constexpr (F32) {
        if (++cnt == PROMOTE) {
#pragma unroll
          for (int k = 0; k < VEC; ++k) {
            dA[k] += (double)fA[k]; dB[k] += (double)fB[k];
            fA[k] = T(0); fB[k] = T(0);
          }
          cnt = 0;
        }
      }
    }
  }
  if constexpr (MODE == MODE_SPMV) return;
  else {
    if constexpr (F32) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) { dA[k] += (double)fA[k]; dB[k] += (double)fB[k]; }
    }
    extern __shared__ double red[];
    const int lane = t & 31, warp = t >> 5;
    bool rep;
    int qrep, nq;
    if (Gt < 32) {
      for (int off = Gt; off < 32; off <<= 1) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          dA[k] += __shfl_xor_sync(0xffffffffu, dA[k], off);
          dB[k] += __shfl_xor_sync(0xffffffffu, dB[k], off);
        }
      }
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
      double s = 0.0;
      for (int qq = 0; qq < nq; ++qq) s += red[((qq * Gt + cc) * 2 + which) * VEC + k];
      a.partial[(size_t)blockIdx.x * 2 * Rp + which * Rp + blockIdx.y * Rt + col] = s;
    }
  }
}

inline size_t step_smem_bytes(int G, int block, int vec) {
  const int nq = G < 32 ? block / 32 : block / G;
  return (size_t)nq * G * 2 * vec * sizeof(double);
}

template <typename T, bool CPLX, int MODE, class OP>
cudaError_t launch_one(const StepArgs& a, const LaunchCfg& cfg, cudaStream_t st) {
  constexpr int SC = Traits<T>::SC;
  constexpr int VEC = CPLX ? SC / 2 : SC;
  const size_t smem = MODE == MODE_SPMV ? 0 : step_smem_bytes(a.Gt, cfg.block, VEC);
  cheb_step_kernel<T, CPLX, MODE, OP><<<dim3(cfg.grid, a.G / a.Gt), cfg.block, smem, st>>>(a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T, bool CPLX, int MODE, class OP>
int occupancy_one(int block, int G) {
  constexpr int SC = Traits<T>::SC;
  constexpr int VEC = CPLX ? SC / 2 : SC;
  int nb = 0;
  const size_t smem = MODE == MODE_SPMV ? 0 : step_smem_bytes(G, block, VEC);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cheb_step_kernel<T, CPLX, MODE, OP>, block,
                                                smem);
  return nb;
}

}  // namespace kpm
