// Dense Hamiltonians: the paper's own formulation (Sec. II-A-4 and Sec. III:
// every element of H~ takes part in every product, no CRS), in FP64 as the
// paper computes it.
//
// The step  Y = S X - W  (S = 2 H~, scaled once per call by the CSR prescale
// kernel over the n*n values, its diagonal shift -2b/a applied here as
// du * x) is a dense contraction of the n x n matrix with the n x Rp vector
// block, fused with the subtraction of v_{n-1} and the two moment dots of
// each column.  GB300's FP64 tensor rate is no higher than its FP64 pipe and
// tcgen05 has no FP64 kind, so the contraction runs on the FP64 pipe: tiles of
// BM x BN outputs per 256-thread CTA, BK = 16 wide slices of S (transposed)
// and X staged in shared memory, RM x CN outputs per thread in registers.
// With 2 FP64 FMAs per SM and clock the kernel is FP64-bound by a wide
// margin (8 shared loads per 16 FMAs, 16 KB of global loads per 64K FMAs).
#include "kpm_internal.h"

namespace kpm {

namespace {

template <bool CPLX>
struct DenseElem;
template <>
struct DenseElem<false> {
  using E = double;
  static __device__ __forceinline__ E zero() { return 0.0; }
  static __device__ __forceinline__ void mac(E& acc, E a, E b) { acc = fma(a, b, acc); }
  static __device__ __forceinline__ double norm2(E x) { return x * x; }
  static __device__ __forceinline__ double re_dot(E y, E x) { return y * x; }  // Re(conj(y) x)
  static __device__ __forceinline__ E axpy(double s, E x, E y) { return fma(s, x, y); }
  static __device__ __forceinline__ E scale(double s, E x) { return s * x; }
  static __device__ __forceinline__ E sub(E a, E b) { return a - b; }
};
template <>
struct DenseElem<true> {
  using E = double2;  // (re, im)
  static __device__ __forceinline__ E zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ void mac(E& acc, E a, E b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
  }
  static __device__ __forceinline__ double norm2(E x) { return x.x * x.x + x.y * x.y; }
  static __device__ __forceinline__ double re_dot(E y, E x) { return y.x * x.x + y.y * x.y; }
  static __device__ __forceinline__ E axpy(double s, E x, E y) {
    return make_double2(fma(s, x.x, y.x), fma(s, x.y, y.y));
  }
  static __device__ __forceinline__ E scale(double s, E x) { return make_double2(s * x.x, s * x.y); }
  static __device__ __forceinline__ E sub(E a, E b) { return make_double2(a.x - b.x, a.y - b.y); }
};

constexpr int DBK = 16;  // k-slice width

// MODE_FIRST: y = (S x) / 2 = H~ x;  MODE_STEP: y = S x - w (y may alias w).
// Moment partials of the CTA's rows, per column r: [0][r] = <x|x>, [1][r] =
// Re<y|x>, written to a.partial[blockIdx.x][2][Rp] (columns of this CTA only).
template <bool CPLX, int MODE, int RM>
__global__ void __launch_bounds__(256) dense_step_kernel(const StepArgs a) {
  using D = DenseElem<CPLX>;
  using E = typename D::E;
  constexpr int CN = CPLX ? 2 : 4;  // columns per thread
  constexpr int BM = 16 * RM, BN = 16 * CN;
  __shared__ E As[DBK][BM + 1];  // As[k][m] = S[row0 + m][k0 + k]
  __shared__ E Bs[DBK][BN];      // Bs[k][c] = X[k0 + k][col0 + c]
  __shared__ double red[8][2][BN];
  const int64_t n = a.n;
  const int Rp = a.Rp;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const E* __restrict__ S = reinterpret_cast<const E*>(a.vals);
  const E* __restrict__ X = reinterpret_cast<const E*>(a.x);
  E acc[RM][CN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < CN; ++j) acc[i][j] = D::zero();

  for (int64_t k0 = 0; k0 < n; k0 += DBK) {
    for (int idx = t; idx < BM * DBK; idx += 256) {
      const int m = idx / DBK, kk = idx % DBK;
      const int64_t r = row0 + m, k = k0 + kk;
      As[kk][m] = (r < n && k < n) ? S[r * n + k] : D::zero();
    }
    for (int idx = t; idx < DBK * BN; idx += 256) {
      const int kk = idx / BN, c = idx % BN;
      const int64_t k = k0 + kk;
      const int col = col0 + c;
      Bs[kk][c] = (k < n && col < Rp) ? X[k * Rp + col] : D::zero();
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DBK; ++kk) {
      E av[RM], bv[CN];
#pragma unroll
      for (int i = 0; i < RM; ++i) av[i] = As[kk][ty * RM + i];
#pragma unroll
      for (int j = 0; j < CN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) D::mac(acc[i][j], av[i], bv[j]);
    }
    __syncthreads();
  }

  // epilogue: diagonal shift, recursion, store, moment dots
  const double du = a.sc->du;
  const E* __restrict__ W = reinterpret_cast<const E*>(a.w);
  E* Y = reinterpret_cast<E*>(a.y);
  double da[CN], db[CN];
#pragma unroll
  for (int j = 0; j < CN; ++j) da[j] = db[j] = 0.0;
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int64_t r = row0 + ty * RM + i;
#pragma unroll
    for (int j = 0; j < CN; ++j) {
      const int col = col0 + tx + 16 * j;
      if (r < n && col < Rp) {
        const size_t o = (size_t)r * Rp + col;
        const E x = X[o];
        E y = D::axpy(du, x, acc[i][j]);
        if (MODE == MODE_FIRST) y = D::scale(0.5, y);
        if (MODE == MODE_STEP) y = D::sub(y, W[o]);
        Y[o] = y;
        da[j] += D::norm2(x);
        db[j] += D::re_dot(y, x);
      }
    }
  }
  if (MODE == MODE_SPMV) return;
  // rows ty = 2w and 2w + 1 of warp w share columns: lanes tx and tx + 16
#pragma unroll
  for (int j = 0; j < CN; ++j) {
    da[j] += __shfl_down_sync(0xffffffffu, da[j], 16);
    db[j] += __shfl_down_sync(0xffffffffu, db[j], 16);
  }
  const int warp = t >> 5, lane = t & 31;
  if (lane < 16) {
#pragma unroll
    for (int j = 0; j < CN; ++j) {
      red[warp][0][lane + 16 * j] = da[j];
      red[warp][1][lane + 16 * j] = db[j];
    }
  }
  __syncthreads();
  for (int o = t; o < 2 * BN; o += 256) {
    const int which = o / BN, c = o % BN;
    if (col0 + c >= Rp) continue;
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][which][c];  // fixed order
    a.partial[(size_t)blockIdx.x * 2 * Rp + (size_t)which * Rp + col0 + c] = s;
  }
}

// y = S x for a narrow block (the Lanczos product, Rp <= 2): one warp per
// row, lanes striding over the row, shuffle reduction.
template <bool CPLX>
__global__ void __launch_bounds__(256) dense_spmv_kernel(const StepArgs a) {
  using D = DenseElem<CPLX>;
  using E = typename D::E;
  const int64_t n = a.n;
  const int Rp = a.Rp;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const E* __restrict__ S = reinterpret_cast<const E*>(a.vals);
  const E* __restrict__ X = reinterpret_cast<const E*>(a.x);
  E* Y = reinterpret_cast<E*>(a.y);
  const double du = a.sc->du;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n;
       r += warps) {
    for (int c = 0; c < Rp; ++c) {
      E s = D::zero();
      for (int64_t k = lane; k < n; k += 32) D::mac(s, S[r * n + k], X[k * Rp + c]);
      double sx, sy = 0.0;
      if constexpr (CPLX) {
        sx = s.x;
        sy = s.y;
      } else {
        sx = s;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0) {
        E v;
        if constexpr (CPLX) {
          v = make_double2(sx, sy);
        } else {
          v = sx;
        }
        Y[r * Rp + c] = D::axpy(du, X[r * Rp + c], v);
      }
    }
  }
}

// Gershgorin enclosure of a dense matrix: per row, centre Re H_ii and radius
// sum_{j != i} |H_ij|; one warp per row, block min / max.
__global__ void gershgorin_dense_kernel(bool cplx, int64_t n, const double* __restrict__ H,
                                        double* pmin, double* pmax) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; i < n; i += warps) {
    double rad = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
      if (j == i) continue;
      const double re = cplx ? H[2 * (i * n + j)] : H[i * n + j];
      const double im = cplx ? H[2 * (i * n + j) + 1] : 0.0;
      rad += hypot(re, im);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rad += __shfl_xor_sync(0xffffffffu, rad, o);
    const double centre = cplx ? H[2 * (i * n + i)] : H[i * n + i];
    lo = fmin(lo, centre - rad);
    hi = fmax(hi, centre + rad);
  }
  __shared__ double smin[8], smax[8];
  if (lane == 0) {
    smin[warp] = lo;
    smax[warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = fmin(lo, smin[w]);
      hi = fmax(hi, smax[w]);
    }
    pmin[blockIdx.x] = lo;
    pmax[blockIdx.x] = hi;
  }
}

template <bool CPLX, int MODE>
cudaError_t launch_tiles(const StepArgs& a, int grid, cudaStream_t st) {
  constexpr int BN = 16 * (CPLX ? 2 : 4);
  const int64_t nb64 = (a.n + 63) / 64;
  const dim3 g((unsigned)grid, (unsigned)((a.Rp + BN - 1) / BN));
  if (grid == nb64)
    dense_step_kernel<CPLX, MODE, 4><<<g, 256, 0, st>>>(a);
  else
    dense_step_kernel<CPLX, MODE, 1><<<g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int dense_row_tile(int64_t n, int Rp, bool cplx, int num_sms) {
  const int BN = 16 * (cplx ? 2 : 4);
  const int64_t cols = (Rp + BN - 1) / BN;
  return ((n + 63) / 64) * cols >= 2 * (int64_t)num_sms ? 64 : 16;
}

cudaError_t launch_dense_step(bool cplx, StepMode mode, const StepArgs& a, const LaunchCfg& cfg,
                              cudaStream_t st) {
  cudaError_t e;
  if (mode == MODE_SPMV) {
    const int64_t blocks = std::min<int64_t>((a.n + 7) / 8, 4096);
    if (cplx)
      dense_spmv_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(a);
    else
      dense_spmv_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(a);
    e = cudaGetLastError();
  } else if (mode == MODE_FIRST) {
    e = cplx ? launch_tiles<true, MODE_FIRST>(a, cfg.grid, st)
             : launch_tiles<false, MODE_FIRST>(a, cfg.grid, st);
  } else if (mode == MODE_STEP) {
    e = cplx ? launch_tiles<true, MODE_STEP>(a, cfg.grid, st)
             : launch_tiles<false, MODE_STEP>(a, cfg.grid, st);
  } else {
    return cudaErrorInvalidValue;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

cudaError_t launch_gershgorin_dense(bool cplx, int64_t n, const double* H, double* part_min,
                                    double* part_max, int nblk, cudaStream_t st) {
  gershgorin_dense_kernel<<<nblk, 256, 0, st>>>(cplx, n, H, part_min, part_max);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace kpm
