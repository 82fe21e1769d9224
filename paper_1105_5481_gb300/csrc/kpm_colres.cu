// Column-resident solve: a whole realisation of a small stencil or padded-ELL
// (CSR rows of at most 8 entries) operator in one launch, one thread-block
// cluster per group of vector columns.
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
// thread's neighbour addresses (and, for a stencil, its hoppings and on-site
// term) are computed once and kept in registers; the ELL values of a CTA's
// rows are copied into its shared memory once.  Each product writes v_{n+1}
// over the thread's own
// element of v_{n-1}; no element is written while another CTA may read it, so
// one cluster barrier (release/acquire) per product is the only
// synchronisation, and the clusters never wait on one another.
//
// Moments: every thread adds |x|^2 and Re(conj(y) x) of its element in FP64.
// The cluster barrier of a product is split: the arrive follows the write of
// v_{n+1}, the wait comes after the thread has handed its dot terms on, so the
// summing overlaps the barrier.  Two ways to sum them:
//  - bulk (CTAs whose batch buffer fits COLRES_BULK_BYTES): the terms are
//    parked in shared memory, and every K products a few lanes per
//    (product, dot, column) add the batch up in thread order, about two FP64
//    adds per thread and product;
//  - tree (larger CTAs): an XOR butterfly over the lanes of a column, the
//    warp results summed in warp order one product later, kept in a
//    shared-memory ring.
// Either way the CTA partials go to global scratch (never once per product:
// a global store would make the next barrier's release wait for L2), and
// after the last product they are summed in rank order into the per-step
// sums that the finalisation kernels read.  The order of every sum is fixed
// by (C, cpc, block), so a repeated call, a replayed graph and a continued
// solve give the same bits.
//
// The operator arithmetic is that of the fused step (diagonal term, then the
// forward and backward bond of each stencil dimension, or the ELL entries in
// order; FMAs in that order, Sec. II-A-2 / Eq. (rn)); the dots are
// accumulated in FP64 on both the FP64 and the FP32-vector path.
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

// The two halves of the cluster barrier: the arrive publishes this thread's
// earlier writes to the cluster, the wait returns once every thread of the
// cluster has arrived and makes their writes visible.
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

}  // namespace

// W = 0: the stencil operator of DIMS dimensions; W > 0: a padded-ELL
// operator of W entries per row (DIMS unused).
template <typename T, bool CPLX, int DIMS, int W>
__global__ void __launch_bounds__(1024, 1) colres_kernel(const ColresArgs p) {
  using E = Elem<T, CPLX>;
  constexpr int NB = W > 0 ? W : 2 * DIMS;  // neighbour slots of a row
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
  double* wp = reinterpret_cast<double*>(sm + colres_head_bytes(2 * (size_t)buf_bytes));  // [3][nw][2][cpc]
  const int nprod = p.n1 - p.n0;

  // The thread's operator row: the shared::cluster addresses of its neighbour
  // elements (slot 2d the forward and 2d+1 the backward bond of dimension d
  // of the stencil, or the W entries of the ELL row), the stencil's bond
  // coefficients and the diagonal.  ELL values are read from shared memory.
  uint32_t an[NB];
  T cr[W > 0 ? 1 : NB], ci[W > 0 ? 1 : NB];
  T hu_r, hu_i, du;
  scalars<T>(p.sc, hu_r, hu_i, du);
  T dg = du;
  auto addr_of = [&](int64_t j) {
    const int qj = (int)(j / p.P);
    return cluster_addr(buf0 + ((j - (int64_t)qj * p.P) * cpc + c), (uint32_t)qj);
  };
  if (valid) {
    if constexpr (W > 0) {
#pragma unroll
      for (int k = 0; k < W; ++k) an[k] = addr_of(p.ecol[i * W + k]);
    } else {
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
        T fr, fi, br, bi;
        if (p.hs) {
          if constexpr (CPLX) {
            const Cx<T>* hs = reinterpret_cast<const Cx<T>*>(p.hs);
            const Cx<T> f = hs[i * DIMS + d], bk = hs[jb * DIMS + d];
            fr = f.re;
            fi = f.im;
            br = bk.re;
            bi = -bk.im;
          } else {
            const T* hs = reinterpret_cast<const T*>(p.hs);
            fr = hs[i * DIMS + d];
            br = hs[jb * DIMS + d];
            fi = bi = T(0);
          }
        } else {
          fr = hu_r;
          fi = hu_i;
          br = hu_r;
          bi = -hu_i;
        }
        if (!hf) fr = fi = T(0);
        if (!hb) br = bi = T(0);
        cr[2 * d] = fr;
        ci[2 * d] = fi;
        cr[2 * d + 1] = br;
        ci[2 * d + 1] = bi;
        an[2 * d] = addr_of(jf);
        an[2 * d + 1] = addr_of(jb);
      }
    }
  }

  // CTA partial of product k (k = n - n0) by thread t < 2 cpc: the warp sums
  // in warp order, kept in a shared-memory ring of `kr` products that goes to
  // the global scratch only when it is full and after the last product (a
  // global store inside the product loop would make the release half of the
  // next cluster barrier wait for its round trip to L2)
  double* ring = wp + (size_t)3 * nw * 2 * cpc;  // [kr][2 cpc]
  const int kr = p.kr;
  auto cta_partial = [&](int k) {
    const int ps = k % 3;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += wp[(size_t)(ps * nw + w) * 2 * cpc + t];
    ring[(size_t)(k % kr) * 2 * cpc + t] = s;
    if (k % kr == kr - 1 || k == nprod - 1) {
      const int k0 = k - k % kr;
      double* dst = p.gp + (((size_t)g * C + q) * nprod) * 2 * cpc + t;
      for (int j = k0; j <= k; ++j) dst[(size_t)j * 2 * cpc] = ring[(size_t)(j - k0) * 2 * cpc + t];
    }
  };

  // Bulk form of the dot sums (p.bulk_k = K > 0): every thread parks its two
  // dot terms of each product in bb[batch & 1][k % K][t][2], no shuffle tree;
  // once a batch of K products is complete, each (product, dot, column) sum
  // of the batch is taken by tps adjacent lanes: lane `sub` adds the column's
  // terms of threads u = cc + cpc (sub + tps m) in increasing u, then an XOR
  // butterfly over the tps lanes (K = B / (2 cpc tps): the B threads cover
  // the batch exactly).  About 2 FP64 adds per thread and product instead of
  // the 2 log2(32 / cpc) of the per-product shuffle tree.
  const int K = p.bulk_k, tps = p.bulk_tps;
  double* bb = ring + (size_t)kr * 2 * cpc;  // [2][K][B][2]
  // ELL: the scaled values of this CTA's rows, [own][W] (x2 complex), copied
  // once per solve so that no product reads them from global memory
  T* evs = reinterpret_cast<T*>(bb + (size_t)2 * K * blockDim.x * 2);
  if constexpr (W > 0) {
    constexpr int VC = CPLX ? 2 : 1;
    const T* src = reinterpret_cast<const T*>(p.evals) + (size_t)r0 * W * VC;
    for (int x = t; x < own * W * VC; x += blockDim.x) evs[x] = src[x];
  }
  auto bulk_reduce = [&](int b, int cnt) {
    const int B = (int)blockDim.x;
    const int sidx = t / tps, sub = t % tps;
    const bool act = sidx < cnt * 2 * cpc;
    const int pi = sidx / (2 * cpc), r = sidx % (2 * cpc);
    double s = 0.0;
    if (act) {
      const int v = r / cpc, cc = r % cpc;
      const double* base = bb + ((size_t)(b & 1) * K + pi) * B * 2;
      for (int u = cc + cpc * sub; u < B; u += cpc * tps) s += base[2 * u + v];
    }
    for (int o = 1; o < tps; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (act && sub == 0)
      p.gp[(((size_t)g * C + q) * nprod + (size_t)b * K + pi) * 2 * cpc + r] = s;
  };

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
      Cx<T> xn[NB];
#pragma unroll
      for (int k = 0; k < NB; ++k) xn[k] = ld_cluster<T, CPLX>(an[k] + off);
      if constexpr (W > 0) {
        // the ELL row's scaled values, in entry order (as the fused ELL step)
#pragma unroll
        for (int k = 0; k < W; ++k) {
          T vr, vi = T(0);
          if constexpr (CPLX) {
            vr = evs[2 * (li * W + k)];
            vi = evs[2 * (li * W + k) + 1];
          } else {
            vr = evs[li * W + k];
          }
          cmac<T, CPLX>(acc, vr, vi, xn[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < NB; ++k) cmac<T, CPLX>(acc, cr[k], ci[k], xn[k]);
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
    if (K > 0) {
      const int k = n - p.n0;
      double* slotp = bb + ((size_t)((k / K) & 1) * K + (k % K)) * blockDim.x * 2;
      slotp[2 * t] = sa;
      slotp[2 * t + 1] = sb;
      cluster_arrive_release();
      // the previous batch (complete since the last wait; its half of bb is
      // next written K products later, after this thread's next arrive)
      if (k % K == 0 && k > 0) bulk_reduce(k / K - 1, K);
      cluster_wait_acquire();
      continue;
    }
    // this CTA's rows of v_{n+1} are published; the warp sums of the dots run
    // while the slower CTAs of the cluster finish theirs
    cluster_arrive_release();
    // lanes of one column: lane, lane ^ cpc, lane ^ 2 cpc, ...
    for (int o = cpc; o < 32; o <<= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    const int slot = (n - p.n0) % 3;
    if (lane < cpc) {
      double* w = wp + ((size_t)(slot * nw + warp) * 2) * cpc;
      w[lane] = sa;
      w[cpc + lane] = sb;
    }
    // v_{n+1} of every CTA is complete
    cluster_wait_acquire();
    // the previous product's warp sums (written before every thread's arrive
    // of this product; their slot is next written three products later, after
    // this thread's next arrive)
    if (t < 2 * cpc && n > p.n0) cta_partial(n - 1 - p.n0);
  }
  // the last product's warp sums, or the last batch of the bulk form
  __syncthreads();
  if (K > 0) {
    const int bl = (nprod - 1) / K;
    bulk_reduce(bl, nprod - bl * K);
  } else if (t < 2 * cpc) {
    cta_partial(nprod - 1);
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

template <typename T, bool CPLX, int DIMS, int W>
const void* colres_fn() {
  return reinterpret_cast<const void*>(colres_kernel<T, CPLX, DIMS, W>);
}

template <typename T, bool CPLX>
const void* pick_t(int dims, int W) {
  switch (W) {
    case 2: return colres_fn<T, CPLX, 0, 2>();
    case 4: return colres_fn<T, CPLX, 0, 4>();
    case 6: return colres_fn<T, CPLX, 0, 6>();
    case 8: return colres_fn<T, CPLX, 0, 8>();
    default: break;
  }
  return dims == 1 ? colres_fn<T, CPLX, 1, 0>() : dims == 2 ? colres_fn<T, CPLX, 2, 0>()
                                                              : colres_fn<T, CPLX, 3, 0>();
}

// The kernel of a stencil operator of `dims` dimensions (W = 0) or of a
// padded-ELL operator of width W (2, 4, 6 or 8).
const void* pick(bool fp32, bool cplx, int dims, int W) {
  if (fp32) return cplx ? pick_t<float, true>(dims, W) : pick_t<float, false>(dims, W);
  return cplx ? pick_t<double, true>(dims, W) : pick_t<double, false>(dims, W);
}

// Once per kernel and device: 16-CTA clusters (a non-portable size) and
// dynamic shared memory up to COLRES_MAX_SMEM.
bool configure(bool fp32, bool cplx, int dims, int W) {
  static std::atomic<unsigned long long> done[28];
  const int slot = W > 0 ? 12 + (fp32 ? 8 : 0) + (cplx ? 4 : 0) + W / 2 - 1
                         : (fp32 ? 6 : 0) + (cplx ? 3 : 0) + dims - 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const unsigned long long bit = 1ull << (dev & 63);
  if (done[slot].load(std::memory_order_acquire) & bit) return true;
  const void* fn = pick(fp32, cplx, dims, W);
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

// Products held by the shared-memory ring of CTA partials (at most 16 KB).
int ring_products(int cpc) { return (int)(COLRES_RING_BYTES / (2 * (size_t)cpc * 8)); }

// Shape of the bulk dot sums.  Small CTAs: the fewest lanes per sum (tps, a
// power of two <= 32) whose batch of K = block / (2 cpc tps) products covers
// the block exactly within COLRES_BULK_SMALL.  Larger CTAs: 32 lanes per sum
// and as many products per batch as COLRES_BULK_BYTES holds (the threads
// past K 2 cpc 32 sit the sums out).  K = 0: the per-product shuffle tree.
void bulk_shape(int cpc, int block, int* K, int* tps) {
  *K = 0;
  *tps = 1;
  for (int l = 1; l <= 32; l *= 2) {
    if (block % (2 * cpc * l) != 0) break;
    const int k = block / (2 * cpc * l);
    if ((size_t)2 * k * block * 2 * 8 <= COLRES_BULK_SMALL) {
      *K = k;
      *tps = l;
      return;
    }
  }
  const int k = (int)std::min<size_t>((size_t)block / (2 * cpc * 32),
                                      COLRES_BULK_BYTES / ((size_t)2 * block * 2 * 8));
  if (k >= 1) {
    *K = k;
    *tps = 32;
  }
}

int bulk_batch(int cpc, int block) {
  int k, l;
  bulk_shape(cpc, block, &k, &l);
  return k;
}

// Estimated microseconds per product (GB300, fitted to measurements of both
// forms on 2D/3D lattices of 512-9216 sites, R = 8-32).  Work is counted in
// real FP64 elements per SM: the elements of a CTA times the CTAs an SM holds,
// x3.9 for complex FP64 (four FMAs per bond; the FP64 pipe bounds it), x1.2
// for complex FP32, x0.8 for FP32 vectors (only the dots are FP64).
//   column-resident: 0.64 + 0.0040 w + 5e-6 e^2 (bulk dot sums; e the
//     elements of a CTA: large CTAs crowd their SMs) or 0.64 + 0.0105 w
//     (shuffle tree).  Measured: real FP64 2D L=32/48/64/80/96, R=8, bulk:
//     0.90/1.28/1.84/3.01/4.55; tree at L=80/96: 4.93/8.32; complex FP64 3D
//     L=8/12/16, R=16: 1.94/3.93/7.83; FP32 2D L=32/64, R=16: 0.74/1.81.
//   step chain: 2.9 + 1.49e-5 N R (x3.9 complex FP64; FP32 vectors x0.15, x1.2
//     more when complex), the launch
//     latency of a dependent step plus its work.  Measured: 2D L=32/64/80/96,
//     R=8: 2.91/3.09/3.87/3.91; L=64, R=32: 4.85; complex 3D L=12/16, R=16:
//     4.51/7.27; FP32 2D L=64/96, R=16: 3.14/3.30; complex 3D L=16, R=32: 3.25.
double work_factor(bool cplx, bool fp32) {
  return (cplx ? (fp32 ? 1.2 : 3.9) : 1.0) * (fp32 ? 0.8 : 1.0);
}

double colres_us(int64_t elems, double per_sm, bool cplx, bool fp32, bool bulk) {
  const double w = (double)elems * per_sm * work_factor(cplx, fp32);
  return bulk ? 0.64 + 0.0040 * w + 5e-6 * (double)elems * (double)elems : 0.64 + 0.0105 * w;
}

// Padded-ELL operators (CSR rows of at most 8 entries).  A row costs a
// little more than a stencil row (W values from shared memory and arbitrary
// neighbours): x1.15 real, x1.0 complex.  Their step chain is slower: x1.1
// (FP64 vectors), x1.65 (FP32).  Measured in us per product, column-resident
// against step chain: real FP64 2D L=32/48/64, R=8: 1.00/1.41/2.40 against
// 3.15/3.23/3.28; complex FP64 3D L=8/12, R=16: 1.73/3.78 against 3.23/4.27;
// FP32 2D L=32/64, R=16: 0.77/1.83 against 4.93/5.23.
double ell_factor(bool cplx) { return cplx ? 1.0 : 1.15; }

double chain_us(int64_t n, int R, bool cplx, bool fp32, bool ell) {
  const double t =
      2.9 + 1.49e-5 * (double)n * R * (cplx ? (fp32 ? 1.2 : 3.9) : 1.0) * (fp32 ? 0.15 : 1.0);
  return ell ? t * (fp32 ? 1.65 : 1.1) : t;
}

size_t smem_bytes(bool fp32, bool cplx, int64_t P, int cpc, int block, int ell_w) {
  return colres_head_bytes(2 * (size_t)P * cpc * elem_size(fp32, cplx)) +
         (size_t)3 * (block / 32) * 2 * cpc * 8 + COLRES_RING_BYTES +
         (size_t)2 * bulk_batch(cpc, block) * block * 2 * 8 +
         (size_t)P * ell_w * elem_size(fp32, cplx);
}

int max_clusters(bool fp32, bool cplx, int dims, int W, int C, int block, size_t smem) {
  const void* fn = pick(fp32, cplx, dims, W);
  if (!configure(fp32, cplx, dims, W)) return 0;
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

bool colres_plan(int64_t n, int dims, int ell_w, bool cplx, bool fp32, int R, ColresPlan* out) {
  *out = ColresPlan{};
  if (n < 1 || R < 1) return false;
  if (ell_w > 0 ? (ell_w > 8 || ell_w % 2 != 0) : (dims < 1 || dims > 3)) return false;
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
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ColresPlan best{};
  double best_cost = 1e300;
  for (int C : {1, 2, 4, 8, 16}) {
    if (forceC && C != forceC) continue;
    const int64_t P = (n + C - 1) / C;
    for (int cpc = 1; cpc <= 32; cpc *= 2) {
      if (forceCpc && cpc != forceCpc) continue;
      const int64_t elems = P * cpc;
      if (elems > COLRES_MAX_ELEMS) break;
      const int block = (int)std::max<int64_t>(32, (elems + 31) / 32 * 32);
      const int groups = (R + cpc - 1) / cpc;
      const size_t smem = smem_bytes(fp32, cplx, P, cpc, block, ell_w);
      if (smem > COLRES_MAX_SMEM) continue;
      const int fit = max_clusters(fp32, cplx, dims, ell_w, C, block, smem);
      if (fit < 1) continue;
      // every cluster resident at once: the solve is one wave; forced shapes may take more
      if (groups > fit && !forceC) continue;
      const double per_sm = std::max(1.0, (double)groups * C / sms);
      const double cost = colres_us(elems, per_sm, cplx, fp32, bulk_batch(cpc, block) > 0) *
                          (ell_w > 0 ? ell_factor(cplx) : 1.0);
      if (cost < best_cost) {  // ties keep the smaller cluster (cheaper barrier)
        best_cost = cost;
        best.C = C;
        best.cpc = cpc;
        best.groups = groups;
        best.block = block;
        best.P = P;
        best.smem = smem;
        best.ell_w = ell_w;
      }
    }
  }
  if (best.C == 0) return false;
  if (!forceC && best_cost >= chain_us(n, R, cplx, fp32, ell_w > 0)) return false;
  *out = best;
  return true;
}

size_t colres_partial_doubles(const ColresPlan& pl, int nprod) {
  return (size_t)pl.groups * pl.C * nprod * 2 * pl.cpc;
}

cudaError_t launch_colres(bool fp32, bool cplx, int dims, const ColresPlan& pl,
                          const ColresArgs& a, cudaStream_t st) {
  const void* fn = pick(fp32, cplx, dims, pl.ell_w);
  if (!configure(fp32, cplx, dims, pl.ell_w) || pl.smem > COLRES_MAX_SMEM)
    return cudaErrorInvalidConfiguration;
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
  ColresArgs ca = a;
  ca.kr = ring_products(pl.cpc);
  bulk_shape(pl.cpc, pl.block, &ca.bulk_k, &ca.bulk_tps);
  if (getenv("KPM_COLRES_TREE")) ca.bulk_k = 0;
  void* args[1] = {&ca};
  const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

}  // namespace kpm
