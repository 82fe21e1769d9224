// Cluster-resident batched kernel: the batched persistent launch with every
// instance's two vector blocks held in the shared memory of its cluster.
//
// A small instance's product is bound by latency, not bandwidth: in the
// global-memory form each product waits on a chain of L2 round trips (the
// rows the cluster wrote in the previous product) before its reduction and
// cluster barrier.  Here CTA `rank` of a C-CTA cluster owns the contiguous
// rows [rank * P, rank * P + P) of the instance (P = ceil(N / C)) and keeps
// them, for both vector blocks, in its shared memory for the whole solve.  A
// neighbour row owned by another CTA of the cluster is read through
// distributed shared memory (a generic load from the address that
// `map_shared_rank` gives); no vector row ever goes to global memory.
//
// One product (Eq. (rn)): every CTA reads v_n (its own rows and the remote
// neighbour rows) and overwrites its own rows of v_{n-1} with v_{n+1}; no CTA
// writes a row that another CTA reads during the same product, so the one
// cluster barrier after each product (release/acquire at cluster scope) is
// the only synchronisation the vectors need.  The moment partials, the rank-0
// sums in rank order and the finalisation are those of the global-memory
// batched kernel, so an instance's moments depend only on C and the
// instance.  Tasks must be untiled and cover all of the instance's products
// (the vectors do not outlive the launch).  Stencil operators only.
#pragma once

#include "kpm_batch.cuh"

namespace kpm {

// A chunk moved through a generic address (this CTA's shared memory or
// another CTA's through the cluster window).
template <class CH>
__device__ __forceinline__ void res_ld(CH& x, const typename CH::T* p) {
  if constexpr (sizeof(typename CH::T) == 8) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    x.v[0] = q.x;
    x.v[1] = q.y;
  } else {
    const float4 q0 = reinterpret_cast<const float4*>(p)[0];
    const float4 q1 = reinterpret_cast<const float4*>(p)[1];
    x.p[0] = make_float2(q0.x, q0.y);
    x.p[1] = make_float2(q0.z, q0.w);
    x.p[2] = make_float2(q1.x, q1.y);
    x.p[3] = make_float2(q1.z, q1.w);
  }
}

template <class CH>
__device__ __forceinline__ void res_st(const CH& x, typename CH::T* p) {
  if constexpr (sizeof(typename CH::T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(x.v[0], x.v[1]);
  } else {
    reinterpret_cast<float4*>(p)[0] = make_float4(x.p[0].x, x.p[0].y, x.p[1].x, x.p[1].y);
    reinterpret_cast<float4*>(p)[1] = make_float4(x.p[2].x, x.p[2].y, x.p[3].x, x.p[3].y);
  }
}

template <class OP>
struct ResStencil : std::false_type {};
template <class CH, int D, bool H, bool S>
struct ResStencil<StencilOp<CH, D, H, S>> : std::true_type {
  static constexpr int DIMS = D;
  static constexpr bool HAS_HOP = H;
  static constexpr bool HAS_DS = S;
};

// acc += (S x)_i for the stencil operator of `a`: the diagonal term with x_i,
// then the 2*DIMS bonds (forward bond h_{i,d}, backward bond conj(h_{i-e_d,d}),
// zero across an open edge).  rowp(j) is the address of chunk c of row j of
// v_n wherever that row lives in the cluster.
template <class CH, class OP, class RowP>
__device__ __forceinline__ void res_stencil(const StepArgs& a, int i, const CH& xi, CH& acc,
                                            typename CH::T hu_r, typename CH::T hu_i,
                                            typename CH::T du, RowP&& rowp) {
  using T = typename CH::T;
  using RS = ResStencil<OP>;
  constexpr int DIMS = RS::DIMS;
  const T d = RS::HAS_DS ? __ldg(reinterpret_cast<const T*>(a.ds) + i) : du;
  acc.axpy(d, xi);
  int rem = i;
#pragma unroll
  for (int d2 = 0; d2 < DIMS; ++d2) {
    const int L = a.geom.L[d2], s = a.geom.stride[d2];
    const int x = rem % L;
    rem /= L;
    const bool per = a.geom.periodic[d2] != 0;
    const bool hf = (x + 1 < L) || per, hb = (x > 0) || per;
    const int jf = (x + 1 < L) ? i + s : (per ? i - (L - 1) * s : i);
    const int jb = (x > 0) ? i - s : (per ? i + (L - 1) * s : i);
    T fr, fi, br, bi;
    if constexpr (RS::HAS_HOP) {
      const T* hs = reinterpret_cast<const T*>(a.hs);
      if constexpr (CH::CPLX) {
        using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        const T2 f = __ldg(reinterpret_cast<const T2*>(hs) + ((size_t)i * DIMS + d2));
        const T2 bk = __ldg(reinterpret_cast<const T2*>(hs) + ((size_t)jb * DIMS + d2));
        fr = f.x;
        fi = f.y;
        br = bk.x;
        bi = -bk.y;
      } else {
        fr = __ldg(hs + (size_t)i * DIMS + d2);
        br = __ldg(hs + (size_t)jb * DIMS + d2);
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
    CH xf, xb;
    res_ld(xf, rowp(jf));
    res_ld(xb, rowp(jb));
    acc.cmac(fr, fi, xf);
    acc.cmac(br, bi, xb);
  }
}

// Bytes of the dynamic shared memory before the vector rows: reduction
// scratch, then the partials [2 parities][C][2 Rp] (rank 0), rounded to 256.
__host__ __device__ inline size_t res_head_bytes(int G, int block, int vec, int C, int Rp) {
  const size_t b = step_smem_bytes(G, block, vec) + (size_t)2 * C * 2 * Rp * sizeof(double);
  return (b + 255) / 256 * 256;
}

// Bytes of one block of `rows` vector rows of G chunks (rounded to 256).
__host__ __device__ inline size_t res_rows_bytes(int64_t rows, int G, int chunk_bytes) {
  return ((size_t)rows * G * chunk_bytes + 255) / 256 * 256;
}

template <class CH, class OP>
__global__ void __launch_bounds__(256, KPM_BATCH_MIN_BLOCKS)
    batch_res_kernel(BatchTask* tasks, int ntasks, int* queue, int rows_cap) {
  using T = typename CH::T;
  constexpr int SC = CH::SC;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const int t = threadIdx.x;
  extern __shared__ __align__(16) double rsm[];
  __shared__ int s_task;
  __shared__ StepArgs s_a;  // the task's operator and geometry, read where used
  for (;;) {
    if (rank == 0 && t == 0) s_task = atomicAdd(queue, 1);
    cluster.sync();
    const int task = *cluster.map_shared_rank(&s_task, 0);
    // every CTA has read rank 0's s_task before rank 0 may overwrite it or exit
    cluster.sync();
    if (task >= ntasks) break;
    BatchTask& bt = tasks[task];
    if (t == 0) s_a = bt.a;
    __syncthreads();
    const int n = (int)s_a.n, G = s_a.G, Rp = s_a.Rp;
    const int rowS = G * SC;  // scalars per row
    const int P = (n + C - 1) / C;
    const int r0 = rank * P;
    const int own = max(0, min(n - r0, P));
    double* red = rsm;
    double* part = rsm + step_smem_bytes(G, blockDim.x, CH::VEC) / sizeof(double);
    double* part0 = cluster.map_shared_rank(part, 0);
    char* vbase = reinterpret_cast<char*>(rsm) + res_head_bytes(G, blockDim.x, CH::VEC, C, Rp);
    T* B0 = reinterpret_cast<T*>(vbase);
    T* B1 = reinterpret_cast<T*>(vbase + res_rows_bytes(rows_cap, G, SC * (int)sizeof(T)));
    const int nsteps = bt.M / 2;

    // random start block, own rows (entry (i, r) of the instance's N x Rp block)
    {
      T* v0 = B0 - (ptrdiff_t)r0 * rowS;  // indexed by the global row
      const int64_t total = (int64_t)own * Rp;
      for (int64_t e = t; e < total; e += blockDim.x)
        random_entry<T, CH::CPLX>(v0, n, Rp, bt.R, bt.seed, (unsigned long long)bt.realisation,
                                  (int64_t)r0 * Rp + e);
    }
    cluster.sync();

    T hu_r, hu_i, du;
    scal_from_block<T>(s_a.sc, hu_r, hu_i, du);
    const int c = t % G;  // G divides the block: a thread keeps its chunk column
    const int rstep = blockDim.x / G;
    for (int step = 0; step < nsteps; ++step) {
      const bool first = step == 0;
      const T* X = (step & 1) ? B1 : B0;
      T* Y = (step & 1) ? B0 : B1;
      auto rowp = [&](int j) -> const T* {
        const unsigned lj = (unsigned)(j - r0);
        if (lj < (unsigned)own) return X + (size_t)lj * rowS + c * SC;
        const unsigned q = (unsigned)j / (unsigned)P;
        const T* rx = cluster.map_shared_rank(X, q);
        return rx + (size_t)((unsigned)j - q * (unsigned)P) * rowS + c * SC;
      };
      typename CH::Acc s;
      CH::acc_zero(s);
      for (int li = t / G; li < own; li += rstep) {
        const size_t off = (size_t)li * rowS + c * SC;
        CH xi, acc;
        res_ld(xi, X + off);
        if (first) {
          acc.zero();
        } else {
          CH wv;
          res_ld(wv, Y + off);
          acc.set_neg(wv);
        }
        res_stencil<CH, OP>(s_a, r0 + li, xi, acc, hu_r, hu_i, du, rowp);
        if (first) acc.half();
        res_st(acc, Y + off);
        CH::acc_add(s, xi, acc);
      }
      cta_reduce<CH>(s_a, s, 0, red, part0 + ((size_t)(step & 1) * C + rank) * 2 * Rp);
      // v_{n+1} of every CTA and the partials at rank 0 are complete
      cluster.sync();
      if (rank == 0) {
        const double* pp = part + (size_t)(step & 1) * C * 2 * Rp;
        for (int q = t; q < 2 * Rp; q += blockDim.x) {
          double sum = 0.0;
          for (int r = 0; r < C; ++r) sum += pp[(size_t)r * 2 * Rp + q];
          bt.sums[(size_t)step * 2 * Rp + q] = sum;
        }
      }
    }
    if (rank == 0) {
      __syncthreads();  // rank 0's own sums writes above
      const int R = bt.R, M = bt.M;
      const double inv_n = 1.0 / (double)n;
      for (int e = t; e < R * nsteps; e += blockDim.x) {
        const int r = e / nsteps, step = e % nsteps;
        const double mu0 = bt.sums[r] * inv_n, mu1 = bt.sums[Rp + r] * inv_n;
        double me = mu0, mo = mu1;
        if (step > 0) {
          me = 2.0 * bt.sums[(size_t)step * 2 * Rp + r] * inv_n - mu0;
          mo = 2.0 * bt.sums[(size_t)step * 2 * Rp + Rp + r] * inv_n - mu1;
        }
        bt.per_vec[(size_t)r * M + 2 * step] = me;
        bt.per_vec[(size_t)r * M + 2 * step + 1] = mo;
        if (!(fabs(me) <= 1.0 + 1e-6) || !(fabs(mo) <= 1.0 + 1e-6)) atomicOr(&bt.flags, 1);
      }
      __syncthreads();
      for (int m = t; m < M; m += blockDim.x) {
        double acc = 0.0;
        for (int r = 0; r < R; ++r) acc += bt.per_vec[(size_t)r * M + m];
        bt.mu[m] = acc / (double)R;
      }
    }
    // the instance is complete on every CTA: no remote read of this task's
    // rows or partials can follow, and s_a may be overwritten
    cluster.sync();
  }
}

template <class CH, class OP>
struct BatchResTag {};

// Dynamic shared memory of the resident kernel for at most rows_cap rows per CTA.
template <class CH>
inline size_t batch_res_smem_bytes(int G, int C, int Rp, int64_t rows_cap) {
  return res_head_bytes(G, 256, CH::VEC, C, Rp) +
         2 * res_rows_bytes(rows_cap, G, CH::SC * (int)sizeof(typename CH::T));
}

// Largest dynamic shared memory the resident kernel may request (the opt-in
// limit of a block minus the kernel's static shared memory), raising the
// kernel's limit to it once per device.
template <class CH, class OP>
size_t batch_res_smem_limit() {
  auto kern = batch_res_kernel<CH, OP>;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  static std::atomic<unsigned long long> done{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_acquire) & bit)) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    done.fetch_or(bit, std::memory_order_acq_rel);
  }
  return lim;
}

template <class CH, class OP>
cudaError_t launch_batch_res_one(BatchTask* tasks, int ntasks, int* queue, int grid, int C, int G,
                                 int Rp, int64_t rows_cap, cudaStream_t st) {
  if constexpr (!ResStencil<OP>::value) {
    return cudaErrorNotSupported;
  } else {
    const size_t smem = batch_res_smem_bytes<CH>(G, C, Rp, rows_cap);
    if (smem > batch_res_smem_limit<CH, OP>()) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        cudaLaunchKernelEx(&cfg, batch_res_kernel<CH, OP>, tasks, ntasks, queue, (int)rows_cap);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
  }
}

// Co-resident clusters of the resident kernel (0: not launchable).
template <class CH, class OP>
int batch_res_max_clusters(int C, int G, int Rp, int64_t rows_cap) {
  if constexpr (!ResStencil<OP>::value) {
    return 0;
  } else {
    const size_t smem = batch_res_smem_bytes<CH>(G, C, Rp, rows_cap);
    if (smem > batch_res_smem_limit<CH, OP>()) return 0;
    auto kern = batch_res_kernel<CH, OP>;
    int n = 0;
    if (C == 1) {
      int dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return n * sms;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  }
}

}  // namespace kpm
