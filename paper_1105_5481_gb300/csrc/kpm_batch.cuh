// Batched persistent launch: many independent KPM instances (different
// lattices, sizes and moment counts) advanced by one kernel launch.
//
// The grid is made of thread-block clusters of C CTAs.  Each cluster takes the
// next instance from an atomic queue (instances are ordered by decreasing
// work, so the longest start first), splits the instance's rows among its C
// CTAs with the same traversal as the single-instance fused step, and runs the
// instance's steps [step_begin, step_end) back to back, separated by the
// hardware cluster barrier (release/acquire at cluster scope, which orders the
// vector rows written by one CTA before the next step's reads by the others).
// Each CTA's moment partial goes to CTA rank 0 through distributed shared
// memory (reduced while the cluster barrier is pending); rank 0 adds the C
// partials in rank order, one product later.  Every access to another
// CTA's shared memory is followed by a cluster barrier before any CTA can
// leave the kernel.  An instance's result thus
// depends only on C and the instance, never on the other instances in the
// batch or on which cluster ran it.
//
// Vectors of v_n are written by the same launch in the previous step, so
// they are read with coherent loads (chunk policy NC = false).
#pragma once

#include <cooperative_groups.h>

#include "kpm_rng.cuh"
#include "kpm_step.cuh"

// Minimum resident CTAs per SM requested from the register allocator.
#ifndef KPM_BATCH_MIN_BLOCKS
#define KPM_BATCH_MIN_BLOCKS 2
#endif

namespace kpm {

namespace cg = cooperative_groups;

// The two halves of a cluster barrier (all threads of every CTA of the
// cluster execute both, in this order): arrive with release semantics at
// cluster scope, then wait with acquire semantics.
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

constexpr int BATCH_FLAG_TIMEOUT = 2;

struct BatchTask {
  StepArgs a;         // operator, geometry, traversal (x, y, w, partial set per step)
  void* v[2];         // the two vector blocks; step s reads v[s & 1], writes v[(s + 1) & 1]
  double* sums;       // [M/2][2 Rp] per-step moment sums (A, B per column)
  double* per_vec;    // [R][M]
  double* mu;         // [M]
  int step_begin;     // steps advanced by this launch: [step_begin, step_end);
  int step_end;       //   step 0 = random start block + first product
  int M, R;
  unsigned long long seed;
  int realisation;
  int flags;          // set by the kernel: bit0 = a moment left [-1, 1],
                      //   bit1 = a bounded wait ran out (BATCH_FLAG_TIMEOUT)
  // R-tiling: an instance's vector columns split into `ntiles` independent
  // tasks (tile `ycol` holds columns ycol*Rt .. ycol*Rt + Rt - 1, Rt = Gt*VEC);
  // the last tile to finish averages the per-vector moments.  ntiles 0 or 1:
  // one task holds all columns.
  int ycol;
  int ntiles;
  int* tiles_done;    // per-instance count of finished tiles (zeroed per launch)
};

// Resident CTAs per SM requested from the register allocator, per chunk
// policy (the 16-byte chunk's smaller vector registers allow three).
template <class CH>
struct BatchMinBlocks {
  static constexpr int value = KPM_BATCH_MIN_BLOCKS;
};
template <bool NC>
struct ChunkF32h;
template <bool NC>
struct BatchMinBlocks<ChunkF32h<NC>> {
  static constexpr int value = 3;
};

template <class CH, class OP>
__global__ void __launch_bounds__(256, BatchMinBlocks<CH>::value)
    batch_kernel(BatchTask* tasks, int ntasks, int* queue) {
  using T = typename CH::T;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const int t = threadIdx.x;
  extern __shared__ double smem[];
  __shared__ int s_task;
  __shared__ int s_last;
  // the task's column tile (first column, columns): read where used, after a
  // barrier, so that the values are not held in registers across the steps
  __shared__ int s_tile[2];
  // The task's step arguments for even and odd steps (x and y swapped), kept
  // in shared memory: read where used instead of held in registers across
  // the step loop.
  __shared__ StepArgs s_args[2];
  const OP op;
  for (;;) {
    if (rank == 0 && t == 0) s_task = atomicAdd(queue, 1);
    cluster.sync();
    const int task = *cluster.map_shared_rank(&s_task, 0);
    // Every CTA has read rank 0's s_task before any CTA goes on: rank 0 may
    // then overwrite it, or exit (a CTA's shared memory must not be accessed
    // by the rest of its cluster after it has exited).
    cluster.sync();
    if (task >= ntasks) break;
    BatchTask& bt = tasks[task];
    if (t < 2) {
      // a column tile is addressed as a block whose rows start at the tile's
      // first chunk (the row stride stays G chunks)
      const size_t coff = (size_t)bt.ycol * bt.a.Gt * CH::SC * sizeof(T);
      StepArgs a = bt.a;
      a.x = reinterpret_cast<const char*>(bt.v[t]) + coff;
      a.y = reinterpret_cast<char*>(bt.v[t ^ 1]) + coff;
      a.w = a.y;
      s_args[t] = a;
      if (t == 0) {
        s_tile[0] = bt.ycol * bt.a.Gt * CH::VEC;
        s_tile[1] = bt.a.Gt * CH::VEC;
      }
    }
    __syncthreads();
    const int Rp = s_args[0].Rp;
    const int nsteps = bt.M / 2;
    // shared memory: CTA reduction scratch, then partials [3 slots][C][2 Rp] (rank 0)
    double* red = smem;
    double* part = smem + step_smem_bytes(s_args[0].Gt, blockDim.x, CH::VEC) / sizeof(double);
    double* part0 = cluster.map_shared_rank(part, 0);
    // rank 0: the C partials of product `st`, added in rank order
    auto sum_partials = [&](int st) {
      const double* pp = part + (size_t)(st % 3) * C * 2 * Rp;
      const int c0 = s_tile[0], Rt = s_tile[1];
      for (int o = t; o < 2 * Rt; o += blockDim.x) {
        const int q = (o / Rt) * Rp + c0 + o % Rt;  // (A or B, column)
        double sum = 0.0;
        for (int r = 0; r < C; ++r) sum += pp[(size_t)r * 2 * Rp + q];
        bt.sums[(size_t)st * 2 * Rp + q] = sum;
      }
    };

    for (int step = bt.step_begin; step < bt.step_end; ++step) {
      const StepArgs& a = s_args[step & 1];
      if (step == 0) {
        T* v0 = reinterpret_cast<T*>(bt.v[0]);
        const int c0 = s_tile[0], Rt = s_tile[1];
        const int64_t total = a.n * Rt;
        for (int64_t e = (int64_t)rank * blockDim.x + t; e < total; e += (int64_t)C * blockDim.x)
          random_entry<T, CH::CPLX>(v0, a.n, Rp, bt.R, bt.seed, (unsigned long long)bt.realisation,
                                    (e / Rt) * Rp + c0 + e % Rt);
        cluster.sync();
      }
      typename CH::Acc s;
      CH::acc_zero(s);
      step_rows<CH, MODE_DYN, OP, false, true>(a, op, rank, C, 0, s, step == 0);
      // Split cluster barrier: the arrive publishes this CTA's rows of v_{n+1};
      // the CTA reduction of its moment partial runs while the other CTAs
      // finish, and its result (slot step % 3 at rank 0) is published by the
      // next product's arrive.  Rank 0 sums a product's partials one product
      // later; three slots keep a slot from being rewritten before it is read.
      cluster_arrive_release();
      cta_reduce<CH>(a, s, 0, red, part0 + ((size_t)(step % 3) * C + rank) * 2 * Rp + s_tile[0]);
      cluster_wait_acquire();
      if (rank == 0 && step > bt.step_begin) sum_partials(step - 1);
    }
    if (bt.step_begin < bt.step_end) {
      cluster.sync();  // the partials of the last product of this launch
      if (rank == 0) sum_partials(bt.step_end - 1);
    }
    if (bt.step_end == nsteps && bt.step_begin < bt.step_end && rank == 0) {
      __syncthreads();  // rank 0's own sums writes above
      const int R = bt.R, M = bt.M;
      const double inv_n = 1.0 / (double)s_args[0].n;
      const int r0 = s_tile[0], nr = max(0, min(R, r0 + s_tile[1]) - r0);  // this task's vectors
      for (int e = t; e < nr * nsteps; e += blockDim.x) {
        const int r = r0 + e / nsteps, step = e % nsteps;
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
      bool last = true;
      if (bt.ntiles > 1) {
        // the other tiles' per-vector moments: written by other clusters,
        // published by their fence before their count, read through L2
        __threadfence();
        if (t == 0) s_last = atomicAdd(bt.tiles_done, 1) == bt.ntiles - 1;
        __syncthreads();
        last = s_last != 0;
        if (last) __threadfence();
      }
      if (last)
        for (int m = t; m < M; m += blockDim.x) {
          double acc = 0.0;
          for (int r = 0; r < R; ++r) acc += __ldcg(bt.per_vec + (size_t)r * M + m);
          bt.mu[m] = acc / (double)R;
        }
    }
    cluster.sync();  // the instance is complete on every CTA of the cluster (and s_args free)
  }
}

// reduction scratch, then partials [3 slots][C][2 Rp]
template <class CH, class OP>
inline size_t batch_smem_bytes(int Gt, int block, int C, int Rp) {
  return step_smem_bytes(Gt, block, CH::VEC) + (size_t)3 * C * 2 * Rp * sizeof(double);
}

template <class CH, class OP>
struct BatchTag {};

template <class CH, class OP>
cudaError_t launch_batch_one(BatchTask* tasks, int ntasks, int* queue, int grid, int C, int Gt,
                             int Rp, cudaStream_t st) {
  const int block = 256;
  const size_t smem = batch_smem_bytes<CH, OP>(Gt, block, C, Rp);
  auto kern = batch_kernel<CH, OP>;
  cudaError_t e = allow_smem<BatchTag<CH, OP>>(kern, smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, tasks, ntasks, queue);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

template <class CH, class OP>
int batch_max_clusters(int C, int Gt, int Rp) {
  const int block = 256;
  const size_t smem = batch_smem_bytes<CH, OP>(Gt, block, C, Rp);
  auto kern = batch_kernel<CH, OP>;
  if (allow_smem<BatchTag<CH, OP>>(kern, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (C > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
  if (C == 1) {
    // one-CTA clusters: the block occupancy (the cluster query reports one per SM)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n * sms;
  }
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace kpm
