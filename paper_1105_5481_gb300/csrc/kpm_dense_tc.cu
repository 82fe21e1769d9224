// Dense FP64 products on the bf16 tensor cores: the paper's dense
// formulation (Sec. II-A-4 without CRS, Sec. III), whose product Y = S X is
// a dense contraction, computed by the splitting scheme of Ozaki, Ogita and
// Oishi (Numer. Algorithms 59, 2012; "error-free transformation of matrix
// multiplication"), in FP64 accuracy from low-precision products.
//
// Every row i of S (= 2 H~, FP64) is scaled by 2^-e_i (e_i the exponent of
// its largest magnitude) and cut into k slices of beta bits,
//     S_ij = 2^e_i sum_{s=1..k} 2^{-beta s} A_s[i][j]  + O(2^{e_i - beta k}),
// each A_s an integer matrix with |A_1| <= 2^beta, |A_s| <= 2^{beta-1} (s > 1),
// stored exactly in bf16.  Every column j of X (= v_n) is cut the same way
// with its own exponent f_j into slices B_t.  Then
//     (S X)_ij = 2^{e_i + f_j} sum_{s + t <= k + 1} 2^{-beta (s+t)} (A_s B_t)_ij
// up to 2^{-beta k} relative to max|S_i.| max|X_.j| times n, and every
// product A_s B_t is an integer matrix that the tensor cores' FP32
// accumulation holds exactly, because beta is chosen so that n 2^{2 beta} <=
// 2^24.  The products are plain bf16 GEMMs with FP32 results (cuBLAS): for
// each t one GEMM of X's slice t with the stacked slices A_1 .. A_{k+1-t}.
// This file's kernels do the rest: the row and column slicing (integer
// arithmetic on the FP64 significands), and one epilogue that adds the exact
// partial products of each level in int32, combines the levels in FP64,
// applies the exponents, and fuses the Chebyshev recursion (diagonal shift,
// subtraction of v_{n-1}, in-place store) with the two moment dots of each
// column, written as per-CTA partials in the layout of the FP64 dense step.
//
// With n = 4096: beta = 6, k = 9, 45 slice products per step.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <math.h>

#include "kpm_internal.h"

namespace kpm {

namespace {

// The balanced beta-bit digits of v 2^-f (|v| 2^-f < 1) in integer
// arithmetic: F = round(v 2^(beta k - f)) exactly in int64 from the FP64
// significand (|F| < 2^(beta k) <= 2^56), then a_s = round(F / 2^(beta (k-s)))
// and F -= a_s 2^(beta (k-s)) for s = 1 .. k, so |a_1| <= 2^beta and |a_s| <=
// 2^(beta-1) after it; every digit is an exact bf16 integer.
__device__ __forceinline__ void split_digits(double v, int f, int beta, int k,
                                             __nv_bfloat16* out, size_t stride) {
  const long long bits = __double_as_longlong(v);
  const int bexp = (int)((bits >> 52) & 0x7ff);
  long long M = bits & 0xFFFFFFFFFFFFFLL;
  int E;
  if (bexp == 0) {
    E = 1 - 1075;
  } else {
    M |= (1LL << 52);
    E = bexp - 1075;
  }
  const int sh = E + beta * k - f;
  long long F = 0;
  if (M != 0) {
    if (sh >= 0) F = M << sh;
    else if (sh > -62) F = (M + (1LL << (-sh - 1))) >> (-sh);
  }
  if (bits < 0) F = -F;
  for (int s = 1; s <= k; ++s) {
    const int D = beta * (k - s);
    const long long a = D > 0 ? ((F + (1LL << (D - 1))) >> D) : F;
    F -= a << D;
    out[(size_t)(s - 1) * stride] = __int2bfloat16_rn((int)a);
  }
}

// Exponent f with m = g 2^f, g in [0.5, 1) (0 for m = 0): |x| <= m < 2^f.
__device__ __forceinline__ int exponent_of(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// Row slicing of S: one CTA per row (max over the row, then the digits).
// row_scale[i] = 2^(e_i - beta (k + 1)).
__global__ void slice_rows_kernel(int64_t n, const double* __restrict__ S, int beta, int k,
                                  __nv_bfloat16* __restrict__ A, double* __restrict__ row_scale) {
  const int64_t i = blockIdx.x;
  const double* row = S + i * n;
  double m = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) m = fmax(m, fabs(row[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wm[w]);
  const int e = exponent_of(m);
  if (threadIdx.x == 0) row_scale[i] = ldexp(1.0, e - beta * (k + 1));
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
    split_digits(row[j], e, beta, k, A + i * n + j, (size_t)n * n);
}

// Column maxima of X (n x Rp row-major) as ordered bit patterns of |x|.
__global__ void col_max_kernel(int64_t n, int Rp, const double* __restrict__ X,
                               unsigned long long* __restrict__ cmax) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Rp) return;
  const int64_t r0 = (int64_t)blockIdx.y * 64, r1 = min(n, r0 + 64);
  double m = 0.0;
  for (int64_t i = r0; i < r1; ++i) m = fmax(m, fabs(X[i * Rp + j]));
  if (m > 0.0) atomicMax(cmax + j, (unsigned long long)__double_as_longlong(m));
}

// Column slicing of X into B[t][i][j]; col_scale[j] = 2^(f_j).
__global__ void slice_cols_kernel(int64_t n, int Rp, const double* __restrict__ X,
                                  const unsigned long long* __restrict__ cmax, int beta, int k,
                                  __nv_bfloat16* __restrict__ B, double* __restrict__ col_scale) {
  const int64_t total = n * Rp;
  for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e0 < total;
       e0 += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e0 % Rp);
    const int f = exponent_of(__longlong_as_double((long long)cmax[j]));
    if (e0 < Rp) col_scale[j] = ldexp(1.0, f);
    split_digits(X[e0], f, beta, k, B + e0, (size_t)total);
  }
}

// Epilogue: P_ij from the exact slice products.  The products of one level
// l = s + t (at most k of them, each an integer below 2^24 in magnitude) are
// added exactly in int32; the levels are combined in FP64 from the smallest
// (l = k + 1) up, weighted 2^(beta (k + 1 - l)), and scaled by the row and
// column exponents.  Then the recursion and the moment dots.  Block: 64
// columns x 4 row lanes; grid (row tiles of bm rows, column tiles of 64),
// partials of this CTA's columns in the layout of the FP64 dense step.
// K (the slice count) is a template parameter, so that the k(k+1)/2 loads of
// an element unroll at constant offsets and issue back to back.  The kernel
// then holds them all in registers (254 at k = 9, one CTA per SM), which
// measured faster than the run-time loops (557 -> about 520 us per step at
// n = 4096, 1792 vectors) and than capping it at 128 registers for two CTAs
// per SM (slower by a fifth).
template <int MODE, int K>
__global__ void __launch_bounds__(256) tc_epilogue_kernel(const StepArgs a, const float* __restrict__ C,
                                                          int beta, int bm,
                                                          const double* __restrict__ row_scale,
                                                          const double* __restrict__ col_scale) {
  const int64_t n = a.n;
  const int Rp = a.Rp;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int j = blockIdx.y * 64 + tx;
  const int64_t row0 = (int64_t)blockIdx.x * bm;
  const size_t blk = (size_t)n * Rp;
  const double* __restrict__ X = reinterpret_cast<const double*>(a.x);
  const double* __restrict__ W = reinterpret_cast<const double*>(a.w);
  double* Y = reinterpret_cast<double*>(a.y);
  const double du = a.sc->du;
  double da = 0.0, db = 0.0;
  if (j < Rp) {
    const double cs = col_scale[j];
    for (int64_t i = row0 + ty; i < min(n, row0 + bm); i += 4) {
      const size_t o = (size_t)i * Rp + j;
      // blocks in memory order: C_t (t = 1..K) holds A_s B_t for s = 1..K+1-t
      int lv[K];
#pragma unroll
      for (int q = 0; q < K; ++q) lv[q] = 0;
      const float* Cp = C + o;
#pragma unroll
      for (int t = 1; t <= K; ++t) {
#pragma unroll
        for (int s2 = 1; s2 <= K + 1 - t; ++s2) {
          lv[s2 + t - 2] += __float2int_rn(__ldcs(Cp));  // level l = s + t
          Cp += blk;
        }
      }
      // levels from the smallest (l = K + 1) up, weighted 2^(beta (K + 1 - l))
      double total = 0.0;
#pragma unroll
      for (int l = K + 1; l >= 2; --l)
        total = fma((double)lv[l - 2],
                    __longlong_as_double((long long)(1023 + beta * (K + 1 - l)) << 52), total);
      const double p = total * row_scale[i] * cs;
      const double x = X[o];
      double y = fma(du, x, p);
      if (MODE == MODE_FIRST) y *= 0.5;
      if (MODE == MODE_STEP) y -= W[o];
      Y[o] = y;
      da = fma(x, x, da);
      db = fma(y, x, db);
    }
  }
  __shared__ double red[2][4][64];
  red[0][ty][tx] = da;
  red[1][ty][tx] = db;
  __syncthreads();
  if (threadIdx.x < 128) {
    const int which = threadIdx.x >> 6, c = threadIdx.x & 63;
    if (blockIdx.y * 64 + c < Rp) {
      double s = 0.0;
      for (int q = 0; q < 4; ++q) s += red[which][q][c];  // fixed order
      a.partial[(size_t)blockIdx.x * 2 * Rp + (size_t)which * Rp + blockIdx.y * 64 + c] = s;
    }
  }
}

}  // namespace

// Bits per slice and number of slices for an n x n contraction.
void dense_tc_split(int64_t n, int* beta, int* k) {
  int lg = 0;
  while (((int64_t)1 << lg) < n) ++lg;
  int b = (24 - lg) / 2;
  if (b > 7) b = 7;   // |slice| <= 2^beta must stay an exact bf16 integer
  if (b < 1) b = 1;
  *beta = b;
  *k = (54 + b - 1) / b;
}

size_t dense_tc_c_floats(int64_t n, int Rp, int k) {
  return (size_t)k * (k + 1) / 2 * (size_t)n * Rp;
}

cudaError_t launch_dense_tc_slice_rows(const DenseTC& d, const double* S, cudaStream_t st) {
  slice_rows_kernel<<<(unsigned)d.n, 256, 0, st>>>(d.n, S, d.beta, d.k,
                                                   reinterpret_cast<__nv_bfloat16*>(d.A), d.row_scale);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_dense_tc_step(const DenseTC& d, StepMode mode, const StepArgs& a,
                                 const LaunchCfg& cfg, cudaStream_t st) {
  if (mode != MODE_FIRST && mode != MODE_STEP) return cudaErrorInvalidValue;
  const int64_t n = a.n;
  const int Rp = a.Rp;
  cudaError_t e = cudaMemsetAsync(d.cmax, 0, (size_t)Rp * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  col_max_kernel<<<dim3((Rp + 255) / 256, (unsigned)((n + 63) / 64)), 256, 0, st>>>(
      n, Rp, reinterpret_cast<const double*>(a.x), d.cmax);
  slice_cols_kernel<<<(unsigned)std::min<int64_t>((n * Rp + 255) / 256, 65535LL * 8), 256, 0, st>>>(
      n, Rp, reinterpret_cast<const double*>(a.x), d.cmax, d.beta, d.k,
      reinterpret_cast<__nv_bfloat16*>(d.B), d.col_scale);
  g_launches.fetch_add(2, std::memory_order_relaxed);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cublasHandle_t h = reinterpret_cast<cublasHandle_t>(d.blas);
  if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  const float one = 1.0f, zero = 0.0f;
  size_t off = 0;
  for (int t = 1; t <= d.k; ++t) {
    const int ns = d.k + 1 - t;  // slices A_1 .. A_{k+1-t}
    // column-major: C_t^T (Rp x ns n) = X_t^T (Rp x n) * [A_1^T .. A_ns^T] (n x ns n)
    const cublasStatus_t bs = cublasGemmEx(
        h, CUBLAS_OP_N, CUBLAS_OP_N, Rp, (int)(ns * n), (int)n, &one, d.B + (size_t)(t - 1) * n * Rp,
        CUDA_R_16BF, Rp, d.A, CUDA_R_16BF, (int)n, &zero, d.C + off, CUDA_R_32F, Rp,
        CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    if (bs != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    off += (size_t)ns * n * Rp;
  }
  const int bm = (int)((n + cfg.grid - 1) / cfg.grid);
  const dim3 g((unsigned)cfg.grid, (unsigned)((Rp + 63) / 64));
#define KPM_TC_EPI(KK)                                                                            \
  if (d.k == KK) {                                                                                \
    if (mode == MODE_FIRST)                                                                       \
      tc_epilogue_kernel<MODE_FIRST, KK><<<g, 256, 0, st>>>(a, d.C, d.beta, bm, d.row_scale,        \
                                                            d.col_scale);                         \
    else                                                                                          \
      tc_epilogue_kernel<MODE_STEP, KK><<<g, 256, 0, st>>>(a, d.C, d.beta, bm, d.row_scale,         \
                                                           d.col_scale);                          \
    g_launches.fetch_add(1, std::memory_order_relaxed);                                           \
    return cudaGetLastError();                                                                    \
  }
  KPM_TC_EPI(8) KPM_TC_EPI(9) KPM_TC_EPI(11) KPM_TC_EPI(14)
#undef KPM_TC_EPI
  return cudaErrorInvalidValue;  // dense_tc_split gives k in {8, 9, 11, 14} for n <= 65536
}

cudaError_t dense_tc_create_blas(DenseTC& d) {
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  if (cublasSetWorkspace(h, d.workspace, d.ws_bytes) != CUBLAS_STATUS_SUCCESS) {
    cublasDestroy(h);
    return cudaErrorUnknown;
  }
  d.blas = h;
  return cudaSuccess;
}

void dense_tc_destroy_blas(DenseTC& d) {
  if (d.blas) cublasDestroy(reinterpret_cast<cublasHandle_t>(d.blas));
  d.blas = nullptr;
}

}  // namespace kpm
