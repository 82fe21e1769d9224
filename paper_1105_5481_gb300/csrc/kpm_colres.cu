// Column-resident solve: a whole realisation of a small stencil operator in
// one launch, one thread-block cluster per group of vector columns.
//
// The columns of the random block are independent recursions (Eq. (rn) acts
// on each |r> separately; only the moment sums of Eq. (munr) mix them), so a
// small lattice need not run its products as a chain of dependent launches
// over the whole GPU.  Cluster g of C CTAs owns the columns
// [g cpc, g cpc + cpc) and keeps both of their vector blocks in its CTAs'
// shared memory for every product: CTA q holds the rows [q P, q P + P),
// P = ceil(N / C), one (row, column) element per thread.  A neighbour row
// owned by another CTA of the cluster is read through distributed shared
// memory (`ld.shared::cluster` at the address `mapa` gives for that CTA); the
// thread's neighbour addresses, hoppings and on-site term are computed once
// and kept in registers.  Each product writes v_{n+1} over the thread's own
// element of v_{n-1}; no element is written while another CTA may read it, so
// one cluster barrier (release/acquire) per product is the only
// synchronisation, and the clusters never wait on one another.
//
// Moments: every thread adds |x|^2 and Re(conj(y) x) of its element in FP64,
// lanes of one column are combined by an XOR butterfly, the warp results of a
// product are summed in warp order after the product's barrier and stored as
// the CTA's partial in global scratch; after the last product the partials
// are summed in rank order into the per-step sums that the finalisation
// kernels read.  The order of every sum is fixed by (C, cpc, block), so a
// repeated call, a replayed graph and a continued solve give the same bits.
//
// The operator arithmetic is that of the fused stencil step (diagonal term,
// then the forward and backward bond of each dimension, FMAs in that order,
// Sec. II-A-2 / Eq. (rn)); the dots are accumulated in FP64 on both the FP64
// and the FP32-vector path.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "kpm_colres.h"
#include "kpm_rng.cuh"

namespace cg = cooperative_groups;

namespace kpm {

namespace {

template <typename T>
struct Cx {
  T re, im;
};

// 32-bit shared::cluster address of `p` (this CTA's shared memory) in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

template <typename T, bool CPLX>
__device__ __forceinline__ Cx<T> ld_cluster(uint32_t addr) {
  Cx<T> v;
  v.im = T(0);
  if constexpr (sizeof(T) == 8) {
    if constexpr (CPLX)
      asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];"
                   : "=d"(v.re), "=d"(v.im) : "r"(addr) : "memory");
    else
      asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v.re) : "r"(addr) : "memory");
  } else {
    if constexpr (CPLX)
      asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];"
                   : "=f"(v.re), "=f"(v.im) : "r"(addr) : "memory");
    else
      asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v.re) : "r"(addr) : "memory");
  }
  return v;
}

// Element (i, r) of an N x Rp block in the library's layout (real: i Rp + r;
// complex FP64: interleaved pairs; complex FP32: 32-byte chunks of four
// columns split as re0..re3, im0..im3).
template <typename T, bool CPLX>
__device__ __forceinline__ void g_offsets(int64_t i, int r, int Rp, int64_t& ore, int64_t& oim) {
  if constexpr (CPLX) {
    cplx_offsets<T>(i, r, Rp, ore, oim);
  } else {
    ore = i * Rp + r;
    oim = ore;
  }
}

template <typename T, bool CPLX>
__device__ __forceinline__ Cx<T> g_load(const void* v, int64_t i, int r, int Rp) {
  int64_t ore, oim;
  g_offsets<T, CPLX>(i, r, Rp, ore, oim);
  const T* p = reinterpret_cast<const T*>(v);
  Cx<T> x;
  x.re = p[ore];
  x.im = CPLX ? p[oim] : T(0);
  return x;
}

template <typename T, bool CPLX>
__device__ __forceinline__ void g_store(void* v, int64_t i, int r, int Rp, const Cx<T>& x) {
  int64_t ore, oim;
  g_offsets<T, CPLX>(i, r, Rp, ore, oim);
  T* p = reinterpret_cast<T*>(v);
  p[ore] = x.re;
  if (CPLX) p[oim] = x.im;
}

template <typename T>
__device__ __forceinline__ void scalars(const ScalarBlock* sc, T& hr, T& hi, T& du) {
  if constexpr (sizeof(T) == 8) {
    hr = sc->hu_re;
    hi = sc->hu_im;
    du = sc->du;
  } else {
    hr = sc->hu_re_f;
    hi = sc->hu_im_f;
    du = sc->du_f;
  }
}

// acc += h x for h = hr + i hi (the real field ignores the imaginary parts)
template <typename T, bool CPLX>
__device__ __forceinline__ void cmac(Cx<T>& acc, T hr, T hi, const Cx<T>& x) {
  if constexpr (CPLX) {
    acc.re = fma(hr, x.re, acc.re);
    acc.re = fma(-hi, x.im, acc.re);
    acc.im = fma(hr, x.im, acc.im);
    acc.im = fma(hi, x.re, acc.im);
  } else {
    acc.re = fma(hr, x.re, acc.re);
  }
}

template <typename T, bool CPLX>
using Elem = typename std::conditional<CPLX, Cx<T>, T>::type;

}  // namespace

template <typename T, bool CPLX, int DIMS>
__global__ void __launch_bounds__(1024, 1) colres_kernel(const ColresArgs p) {
  using E = Elem<T, CPLX>;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int g = (int)(blockIdx.x / C);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  const int cpc = p.cpc;
  const int c = t % cpc, li = t / cpc;
  const int64_t r0 = (int64_t)q * p.P;
  const int own = (int)max((int64_t)0, min(p.n - r0, (int64_t)p.P));
  const bool valid = li < own;
  const int col = g * cpc + c;
  const int64_t i = r0 + li;
  const int e = li * cpc + c;  // the thread's element in a block of P x cpc
  extern __shared__ __align__(16) unsigned char sm[];
  E* buf0 = reinterpret_cast<E*>(sm);
  E* buf1 = buf0 + (size_t)p.P * cpc;
  const uint32_t buf_bytes = (uint32_t)((size_t)p.P * cpc * sizeof(E));
  double* wp = reinterpret_cast<double*>(sm + colres_head_bytes(2 * (size_t)buf_bytes));  // [2][nw][2][cpc]
  const int nprod = p.n1 - p.n0;

  // the thread's operator row: neighbour addresses, bond coefficients, diagonal
  uint32_t af[DIMS], ab[DIMS];
  T fr[DIMS], fi[DIMS], br[DIMS], bi[DIMS];
  T hu_r, hu_i, du;
  scalars<T>(p.sc, hu_r, hu_i, du);
  T dg = du;
  if (valid) {
    if (p.ds) dg = reinterpret_cast<const T*>(p.ds)[i];
    int64_t rem = i;
#pragma unroll
    for (int d = 0; d < DIMS; ++d) {
      const int L = p.geom.L[d], s = p.geom.stride[d];
      const int x = (int)(rem % L);
      rem /= L;
      const bool per = p.geom.periodic[d] != 0;
      const bool hf = (x + 1 < L) || per, hb = (x > 0) || per;
      const int64_t jf = (x + 1 < L) ? i + s : (per ? i - (int64_t)(L - 1) * s : i);
      const int64_t jb = (x > 0) ? i - s : (per ? i + (int64_t)(L - 1) * s : i);
      if (p.hs) {
        if constexpr (CPLX) {
          const Cx<T>* hs = reinterpret_cast<const Cx<T>*>(p.hs);
          const Cx<T> f = hs[i * DIMS + d], bk = hs[jb * DIMS + d];
          fr[d] = f.re;
          fi[d] = f.im;
          br[d] = bk.re;
          bi[d] = -bk.im;
        } else {
          const T* hs = reinterpret_cast<const T*>(p.hs);
          fr[d] = hs[i * DIMS + d];
          br[d] = hs[jb * DIMS + d];
          fi[d] = bi[d] = T(0);
        }
      } else {
        fr[d] = hu_r;
        fi[d] = hu_i;
        br[d] = hu_r;
        bi[d] = -hu_i;
      }
      if (!hf) fr[d] = fi[d] = T(0);
      if (!hb) br[d] = bi[d] = T(0);
      const int qf = (int)(jf / p.P), qb = (int)(jb / p.P);
      af[d] = cluster_addr(buf0 + ((jf - (int64_t)qf * p.P) * cpc + c), (uint32_t)qf);
      ab[d] = cluster_addr(buf0 + ((jb - (int64_t)qb * p.P) * cpc + c), (uint32_t)qb);
    }
  }

  // start: v_0 drawn here or loaded, or v_{n0-1} and v_{n0} of a continued solve
  if (valid) {
    const bool in_cols = col < p.R;
    auto put = [&](E* b, const Cx<T>& v) {
      if constexpr (CPLX) b[e] = v;
      else b[e] = v.re;
    };
    Cx<T> z{T(0), T(0)};
    if (p.n0 == 0) {
      Cx<T> v = z;
      if (in_cols) {
        if (p.gen)
          random_value<T, CPLX>(p.n, p.R, p.prm->seed,
                                (unsigned long long)(p.prm->s + p.prm->s0), i, col, v.re, v.im);
        else
          v = g_load<T, CPLX>(p.vg[0], i, col, p.Rp);
      }
      put(buf0, v);
    } else {
      const int a = p.n0 & 1;
      put(a ? buf1 : buf0, in_cols ? g_load<T, CPLX>(p.vg[a], i, col, p.Rp) : z);
      put(a ? buf0 : buf1, in_cols ? g_load<T, CPLX>(p.vg[a ^ 1], i, col, p.Rp) : z);
    }
  }
  cl.sync();

  for (int n = p.n0; n < p.n1; ++n) {
    const int par = n & 1;
    E* X = par ? buf1 : buf0;
    E* Y = par ? buf0 : buf1;
    const uint32_t off = par ? buf_bytes : 0u;
    double sa = 0.0, sb = 0.0;
    if (valid) {
      Cx<T> x, acc;
      if constexpr (CPLX) x = X[e];
      else x = Cx<T>{X[e], T(0)};
      if (n == 0) {
        acc.re = acc.im = T(0);
      } else {
        if constexpr (CPLX) {
          const Cx<T> wv = Y[e];
          acc.re = -wv.re;
          acc.im = -wv.im;
        } else {
          acc.re = -Y[e];
          acc.im = T(0);
        }
      }
      acc.re = fma(dg, x.re, acc.re);
      if (CPLX) acc.im = fma(dg, x.im, acc.im);
      Cx<T> xf[DIMS], xb[DIMS];
#pragma unroll
      for (int d = 0; d < DIMS; ++d) {
        xf[d] = ld_cluster<T, CPLX>(af[d] + off);
        xb[d] = ld_cluster<T, CPLX>(ab[d] + off);
      }
#pragma unroll
      for (int d = 0; d < DIMS; ++d) {
        cmac<T, CPLX>(acc, fr[d], fi[d], xf[d]);
        cmac<T, CPLX>(acc, br[d], bi[d], xb[d]);
      }
      if (n == 0) {
        acc.re *= T(0.5);
        acc.im *= T(0.5);
      }
      if constexpr (CPLX) Y[e] = acc;
      else Y[e] = acc.re;
      const double xr = (double)x.re, xi = (double)x.im;
      const double yr = (double)acc.re, yi = (double)acc.im;
      sa = fma(xr, xr, xi * xi);
      sb = fma(yr, xr, yi * xi);
    }
    // lanes of one column: lane, lane ^ cpc, lane ^ 2 cpc, ...
    for (int o = cpc; o < 32; o <<= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (lane < cpc) {
      double* w = wp + ((size_t)(par * nw + warp) * 2) * cpc;
      w[lane] = sa;
      w[cpc + lane] = sb;
    }
    // v_{n+1} of every CTA and this product's warp partials are complete
    cl.sync();
    if (t < 2 * cpc) {
      double s = 0.0;
      for (int k = 0; k < nw; ++k) s += wp[(size_t)(par * nw + k) * 2 * cpc + t];
      p.gp[(((size_t)g * C + q) * nprod + (n - p.n0)) * 2 * cpc + t] = s;
    }
  }

  // v_{n1} and v_{n1-1} to the global blocks (where a continued solve reads them)
  if (valid && col < p.Rp) {
    const int a = p.n1 & 1;
    const E* Xa = a ? buf1 : buf0;
    const E* Xb = a ? buf0 : buf1;
    Cx<T> va, vb;
    if constexpr (CPLX) {
      va = Xa[e];
      vb = Xb[e];
    } else {
      va = Cx<T>{Xa[e], T(0)};
      vb = Cx<T>{Xb[e], T(0)};
    }
    g_store<T, CPLX>(p.vg[a], i, col, p.Rp, va);
    g_store<T, CPLX>(p.vg[a ^ 1], i, col, p.Rp, vb);
  }
  // every CTA's partials are stored; no shared memory is read past this point
  cl.sync();
  const int total = nprod * 2 * cpc;
  const unsigned long long s_idx = (unsigned long long)p.prm->s;
  for (int idx = q * blockDim.x + t; idx < total; idx += C * blockDim.x) {
    const int step = idx / (2 * cpc), kc = idx % (2 * cpc);
    const int k = kc / cpc, cc = kc % cpc;
    const int cl_col = g * cpc + cc;
    if (cl_col >= p.R) continue;
    double s = 0.0;
    for (int r = 0; r < C; ++r) s += p.gp[(((size_t)g * C + r) * nprod + step) * 2 * cpc + kc];
    p.sums[((size_t)s_idx * p.steps + p.n0 + step) * 2 * p.Rp + (size_t)k * p.Rp + cl_col] = s;
  }
}

namespace {

template <typename T, bool CPLX, int DIMS>
const void* colres_fn() {
  return reinterpret_cast<const void*>(colres_kernel<T, CPLX, DIMS>);
}

const void* pick(bool fp32, bool cplx, int dims) {
  if (fp32) {
    if (cplx) return dims == 1 ? colres_fn<float, true, 1>() : dims == 2 ? colres_fn<float, true, 2>()
                                                                        : colres_fn<float, true, 3>();
    return dims == 1 ? colres_fn<float, false, 1>() : dims == 2 ? colres_fn<float, false, 2>()
                                                                 : colres_fn<float, false, 3>();
  }
  if (cplx) return dims == 1 ? colres_fn<double, true, 1>() : dims == 2 ? colres_fn<double, true, 2>()
                                                                       : colres_fn<double, true, 3>();
  return dims == 1 ? colres_fn<double, false, 1>() : dims == 2 ? colres_fn<double, false, 2>()
                                                                : colres_fn<double, false, 3>();
}

// Once per kernel and device: 16-CTA clusters (a non-portable size) and
// dynamic shared memory up to COLRES_MAX_SMEM.
bool configure(bool fp32, bool cplx, int dims) {
  static std::atomic<unsigned long long> done[12];
  const int slot = (fp32 ? 6 : 0) + (cplx ? 3 : 0) + dims - 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const unsigned long long bit = 1ull << (dev & 63);
  if (done[slot].load(std::memory_order_acquire) & bit) return true;
  const void* fn = pick(fp32, cplx, dims);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)COLRES_MAX_SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  done[slot].fetch_or(bit, std::memory_order_acq_rel);
  return true;
}

size_t elem_size(bool fp32, bool cplx) { return (fp32 ? 4 : 8) * (cplx ? 2 : 1); }

size_t smem_bytes(bool fp32, bool cplx, int64_t P, int cpc, int block) {
  return colres_head_bytes(2 * (size_t)P * cpc * elem_size(fp32, cplx)) +
         (size_t)2 * (block / 32) * 2 * cpc * 8;
}

int max_clusters(bool fp32, bool cplx, int dims, int C, int block, size_t smem) {
  const void* fn = pick(fp32, cplx, dims);
  if (!configure(fp32, cplx, dims)) return 0;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

bool colres_plan(int64_t n, int dims, bool cplx, bool fp32, int R, ColresPlan* out) {
  *out = ColresPlan{};
  if (n < 1 || dims < 1 || dims > 3 || R < 1) return false;
  int forceC = 0, forceCpc = 0;
  if (const char* env = getenv("KPM_COLRES")) {
    int c_ = -1, k_ = 0;
    const int got = sscanf(env, "%d,%d", &c_, &k_);
    if (got >= 1 && c_ == 0) return false;
    if (got == 2 && c_ > 0 && k_ > 0) {
      forceC = c_;
      forceCpc = k_;
    }
  }
  ColresPlan best{};
  int64_t best_cost = INT64_MAX;
  for (int C : {1, 2, 4, 8, 16}) {
    if (forceC && C != forceC) continue;
    const int64_t P = (n + C - 1) / C;
    for (int cpc = 1; cpc <= 32; cpc *= 2) {
      if (forceCpc && cpc != forceCpc) continue;
      const int64_t elems = P * cpc;
      if (elems > COLRES_MAX_ELEMS) break;
      const int block = (int)std::max<int64_t>(32, (elems + 31) / 32 * 32);
      const int groups = (R + cpc - 1) / cpc;
      const size_t smem = smem_bytes(fp32, cplx, P, cpc, block);
      if (smem > COLRES_MAX_SMEM) continue;
      const int fit = max_clusters(fp32, cplx, dims, C, block, smem);
      if (fit < 1) continue;
      // every cluster resident at once: the solve is one wave; forced shapes may take more
      if (groups > fit && !forceC) continue;
      const int64_t cost = elems;
      if (cost < best_cost) {  // ties keep the smaller cluster (cheaper barrier)
        best_cost = cost;
        best.C = C;
        best.cpc = cpc;
        best.groups = groups;
        best.block = block;
        best.P = P;
        best.smem = smem;
      }
    }
  }
  if (best.C == 0) return false;
  *out = best;
  return true;
}

size_t colres_partial_doubles(const ColresPlan& pl, int nprod) {
  return (size_t)pl.groups * pl.C * nprod * 2 * pl.cpc;
}

cudaError_t launch_colres(bool fp32, bool cplx, int dims, const ColresPlan& pl,
                          const ColresArgs& a, cudaStream_t st) {
  const void* fn = pick(fp32, cplx, dims);
  if (!configure(fp32, cplx, dims) || pl.smem > COLRES_MAX_SMEM) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(pl.groups * pl.C);
  cfg.blockDim = dim3(pl.block);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[1] = {const_cast<ColresArgs*>(&a)};
  const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

}  // namespace kpm
