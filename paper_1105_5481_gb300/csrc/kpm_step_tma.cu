// Fused Chebyshev step (Eq. (rn) with the two moment dots of the doubling
// identities) for padded-ELL operators with FP32 vectors, fed by the tensor
// memory accelerator through a shared-memory pipeline.
//
// The plain ELL step (EllOp in kpm_step.cuh) is bound by the latency of each
// row's chain of accesses: the column indices must arrive before the
// neighbour rows can be requested, and the streamed rows (v_{n-1}, the row's
// own v_n) occupy registers while in flight.  Here the contiguous part of a
// tile of rows - v_n and v_{n-1} rows, ELL column indices and scaled values -
// is copied into a ring of shared-memory stages by one producer warp with
// bulk asynchronous copies (cp.async.bulk, completion counted in bytes on an
// mbarrier per stage), several tiles ahead.  Eight consumer warps wait for a
// stage, read the indices, values and streamed rows from shared memory,
// gather the neighbour rows of v_n from global memory (L2), compute
// v_{n+1} = 2 H~ v_n - v_{n-1} and the dots A = <v_n|v_n>, B = Re<v_{n+1}|v_n>,
// store v_{n+1} in place over v_{n-1}, and release the stage to the producer
// through a second mbarrier.  The arithmetic and its order per row are those
// of EllOp (explicitly rounded intrinsics); rows go to threads differently,
// so the compensated FP32 moment dots are summed in another order and the
// moments differ from the plain step's within that summation's bound.
//
// Every wait is bounded (about a second of clock64 cycles).  A wait that runs
// out sets bit 2 of *a.err, stops the warp's work, and the producer waits
// (again bounded) for every copy it issued before the CTA leaves, so no copy
// can land in the shared memory of a CTA that has exited.
#include "kpm_step.cuh"

namespace kpm {
namespace {

constexpr int TMA_CONSUMER_WARPS = 8;
constexpr int TMA_CONSUMERS = 32 * TMA_CONSUMER_WARPS;
constexpr int TMA_THREADS = TMA_CONSUMERS + 32;
constexpr int TMA_MAX_STAGES = 8;
constexpr long long TMA_WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz
constexpr int TMA_ERR_TIMEOUT = 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `parity` to complete; false once the limit has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > TMA_WAIT_CYCLES) return false;
  return true;
}
// global -> this CTA's shared memory, `bytes` (a multiple of 16, both
// addresses 16-byte aligned) counted on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__host__ __device__ inline size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

// Byte layout of one stage of `rows` rows.
struct TmaStage {
  uint32_t off_x, off_w, off_c, off_v, bytes;
  __host__ __device__ TmaStage(int rows, int rowB, int W, int valB) {
    off_x = 0;
    off_w = (uint32_t)round_up((size_t)rows * rowB, 128);
    off_c = off_w + (uint32_t)round_up((size_t)rows * rowB, 128);
    off_v = off_c + (uint32_t)round_up((size_t)rows * W * 4, 128);
    bytes = off_v + (uint32_t)round_up((size_t)rows * W * valB, 128);
  }
};

// Dynamic shared memory: stage barriers, the CTA reduction's scratch, stages.
__host__ __device__ inline size_t tma_red_bytes(int G, int vec) {
  return step_smem_bytes(G, TMA_THREADS, vec);
}
__host__ __device__ inline size_t tma_smem_bytes(int stages, int rows, int rowB, int W, int valB,
                                                 int G, int vec) {
  return 128 + round_up(tma_red_bytes(G, vec), 128) +
         (size_t)stages * TmaStage(rows, rowB, W, valB).bytes;
}

template <class CH, int W, int MINB>
__global__ void __launch_bounds__(TMA_THREADS, MINB)
    ell_tma_step_kernel(const StepArgs a, int stages, int tile_passes) {
  using T = typename CH::T;
  constexpr int SC = CH::SC;
  constexpr bool CPLX = CH::CPLX;
  constexpr int VALB = (int)sizeof(T) * (CPLX ? 2 : 1);
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + TMA_MAX_STAGES;
  double* red = reinterpret_cast<double*>(smem + 128);
  const int G = a.G;
  const int rowB = G * SC * (int)sizeof(T);
  const int spi = TMA_CONSUMERS / G;  // rows per pass
  const int rows = spi * tile_passes; // rows per tile
  const TmaStage L(rows, rowB, W, VALB);
  unsigned char* stage0 = smem + 128 + round_up(tma_red_bytes(G, CH::VEC), 128);
  const int64_t ntiles = (a.n + rows - 1) / rows;
  const int ncta = gridDim.x, cta = blockIdx.x;
  const int64_t my_tiles = ntiles > cta ? (ntiles - 1 - cta) / ncta + 1 : 0;
  auto tile_of = [&](int64_t k) {
    const int64_t t = cta + k * ncta;
    return a.reverse ? ntiles - 1 - t : t;
  };
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TMA_CONSUMER_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  typename CH::Acc s;
  CH::acc_zero(s);
  bool timed_out = false;
  if (warp == TMA_CONSUMER_WARPS) {
    // producer warp: lane 0 issues the copies of tile k into stage k % stages,
    // the whole warp running the loop together.  With a.tma_prefetch >= 0
    // every lane also asks L2 for the off-tile neighbour rows of the tile that
    // many tiles ahead (rows ahead of the sweep are first touched there, from
    // DRAM).  That prefetch measured slower at every distance (0..3 tiles) and
    // is off by default; the kernel with it compiled in but off measured 5 %
    // faster than the same kernel without the branch (589 vs 618 us per step
    // on the L = 160 CSR workload, alternating runs on one GPU), so it stays.
    int64_t issued = 0;
    // a.tma_stall (a testing aid): issue nothing, so that the consumers'
    // bounded waits run out and report a timeout
    const int64_t to_issue = a.tma_stall ? 0 : my_tiles;
    for (int64_t k = 0; k < to_issue; ++k) {
      const int st = (int)(k % stages);
      bool ok = k < stages || mbar_wait(&empty[st], (uint32_t)((k / stages - 1) & 1));
      if (!__all_sync(0xffffffffu, ok)) {
        timed_out = true;
        break;
      }
      const int64_t r0 = tile_of(k) * rows;
      const int nr = (int)min((int64_t)rows, a.n - r0);
      if (lane == 0) {
        unsigned char* sp = stage0 + (size_t)st * L.bytes;
        const uint32_t bx = (uint32_t)nr * rowB;
        const uint32_t bc = (uint32_t)round_up((size_t)nr * W * 4, 16);
        const uint32_t bv = (uint32_t)round_up((size_t)nr * W * VALB, 16);
        mbar_expect_tx(&full[st], 2 * bx + bc + bv);
        bulk_g2s(sp + L.off_x, reinterpret_cast<const unsigned char*>(a.x) + r0 * rowB, bx, &full[st]);
        bulk_g2s(sp + L.off_w, reinterpret_cast<const unsigned char*>(a.w) + r0 * rowB, bx, &full[st]);
        bulk_g2s(sp + L.off_c, a.col + r0 * W, bc, &full[st]);
        bulk_g2s(sp + L.off_v, reinterpret_cast<const unsigned char*>(a.vals) + r0 * W * VALB, bv,
                 &full[st]);
      }
      issued = k + 1;
      if (a.tma_prefetch >= 0 && k + a.tma_prefetch < my_tiles) {
        const char* xb = reinterpret_cast<const char*>(a.x);
        const int64_t p0 = tile_of(k + a.tma_prefetch) * rows;
        const int np = (int)min((int64_t)rows, a.n - p0);
        for (int lr = lane; lr < np; lr += 32) {
          const int2* cp = reinterpret_cast<const int2*>(a.col + (p0 + lr) * W);
#pragma unroll
          for (int kk = 0; kk < W / 2; ++kk) {
            const int2 c2 = __ldg(cp + kk);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int64_t j = h ? c2.y : c2.x;
              if (j >= p0 && j < p0 + np) continue;
              for (int off = 0; off < rowB; off += 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(xb + j * rowB + off));
            }
          }
        }
      }
    }
    __syncwarp();
    // every copy this CTA issued must have landed before the CTA may exit
    if (lane == 0)
      for (int64_t k = issued > stages ? issued - stages : 0; k < issued; ++k)
        if (!mbar_wait(&full[k % stages], (uint32_t)((k / stages) & 1))) timed_out = true;
    __syncwarp();
  } else {
    // consumers
    const int c = t % G;
    const int q = t / G;
    T hu_r, hu_i, du;
    scal_from_block<T>(a.sc, hu_r, hu_i, du);
    const size_t rowS = (size_t)G * SC;
    const T* __restrict__ Xc = reinterpret_cast<const T*>(a.x) + (size_t)c * SC;
    T* Yc = reinterpret_cast<T*>(a.y) + (size_t)c * SC;
    for (int64_t k = 0; k < my_tiles; ++k) {
      const int st = (int)(k % stages);
      if (!mbar_wait(&full[st], (uint32_t)((k / stages) & 1))) {
        timed_out = true;
        break;
      }
      const int64_t r0 = tile_of(k) * rows;
      const unsigned char* sp = stage0 + (size_t)st * L.bytes;
      for (int p = 0; p < tile_passes; ++p) {
        const int lr = p * spi + q;
        const int64_t i = r0 + lr;
        if (i >= a.n) continue;
        const T* sx = reinterpret_cast<const T*>(sp + L.off_x) + (size_t)lr * rowS + (size_t)c * SC;
        const T* sw = reinterpret_cast<const T*>(sp + L.off_w) + (size_t)lr * rowS + (size_t)c * SC;
        CH xi, wv, acc;
        xi.ld_shared(sx);
        wv.ld_shared(sw);
        acc.set_neg(wv);
        acc.axpy(du, xi);
        const int2* cp = reinterpret_cast<const int2*>(sp + L.off_c) + (size_t)lr * (W / 2);
        int j[W];
        T hr[W], hi[W];
#pragma unroll
        for (int kk = 0; kk < W / 2; ++kk) {
          const int2 c2 = cp[kk];
          j[2 * kk] = c2.x;
          j[2 * kk + 1] = c2.y;
        }
        if constexpr (CPLX) {
          const T* vp = reinterpret_cast<const T*>(sp + L.off_v) + (size_t)lr * W * 2;
#pragma unroll
          for (int kk = 0; kk < W; ++kk) {
            hr[kk] = vp[2 * kk];
            hi[kk] = vp[2 * kk + 1];
          }
        } else {
          const T* vp = reinterpret_cast<const T*>(sp + L.off_v) + (size_t)lr * W;
#pragma unroll
          for (int kk = 0; kk < W; ++kk) {
            hr[kk] = vp[kk];
            hi[kk] = T(0);
          }
        }
        // (reading the neighbours that fall inside the tile from its copy of
        // v_n measured slower: the gathers are latency-, not L2-bound)
        CH xj[W];
#pragma unroll
        for (int kk = 0; kk < W; ++kk) xj[kk].ld_x(Xc + (size_t)j[kk] * rowS);
#pragma unroll
        for (int kk = 0; kk < W; ++kk) acc.cmac(hr[kk], hi[kk], xj[kk]);
        acc.st(Yc + (size_t)i * rowS);
        CH::acc_add(s, xi, acc);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  if (timed_out && a.err) atomicOr(a.err, TMA_ERR_TIMEOUT);
  cta_reduce<CH, false>(a, s, 0, red, a.partial + (size_t)blockIdx.x * 2 * a.Rp);
}

template <class CH, int W, int MINB>
struct TmaTag {};

template <class CH, int W, int MINB>
cudaError_t launch_tma(const StepArgs& a, const LaunchCfg& cfg, int stages, int tile_passes,
                       cudaStream_t st) {
  const int rowB = a.G * CH::SC * (int)sizeof(typename CH::T);
  const int valB = (int)sizeof(typename CH::T) * (CH::CPLX ? 2 : 1);
  const int rows = TMA_CONSUMERS / a.G * tile_passes;
  const size_t smem = tma_smem_bytes(stages, rows, rowB, W, valB, a.G, CH::VEC);
  auto kern = ell_tma_step_kernel<CH, W, MINB>;
  cudaError_t e = allow_smem<TmaTag<CH, W, MINB>>(kern, smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  kern<<<cfg.grid, TMA_THREADS, smem, st>>>(a, stages, tile_passes);
  return cudaGetLastError();
}

template <class CH, int W, int MINB>
int occupancy_tma(const StepArgs& a, int stages, int tile_passes) {
  const int rowB = a.G * CH::SC * (int)sizeof(typename CH::T);
  const int valB = (int)sizeof(typename CH::T) * (CH::CPLX ? 2 : 1);
  const int rows = TMA_CONSUMERS / a.G * tile_passes;
  const size_t smem = tma_smem_bytes(stages, rows, rowB, W, valB, a.G, CH::VEC);
  auto kern = ell_tma_step_kernel<CH, W, MINB>;
  if (allow_smem<TmaTag<CH, W, MINB>>(kern, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TMA_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <class CH, class F>
auto visit_tma(int W, int minb, F&& f) {
#define KPM_TMA_W(WW)                                                        \
  if (W == WW) {                                                             \
    if (minb >= 3) return f.template operator()<CH, WW, 3>();                \
    return f.template operator()<CH, WW, 2>();                               \
  }
  KPM_TMA_W(2) KPM_TMA_W(4) KPM_TMA_W(6)
#undef KPM_TMA_W
  return f.template operator()<CH, 8, 2>();
}

}  // namespace

bool ell_tma_supported(const StepArgs& a, bool fp32) {
  // FP32 vectors, padded ELL of width <= 8, whole rows per warp (G <= 32 chunks
  // handled by one CTA), and 16-byte aligned tiles of any row count
  return fp32 && a.ell_w >= 2 && a.ell_w <= 8 && (a.ell_w % 2) == 0 && a.G == a.Gt && a.G <= 32 &&
         a.n >= 1;
}

cudaError_t launch_ell_tma_f32(bool cplx, const StepArgs& a, const LaunchCfg& cfg, cudaStream_t st) {
  if (a.tma_stages < 1 || a.tma_stages > TMA_MAX_STAGES || a.tma_passes < 1)
    return cudaErrorInvalidValue;
  if (cplx)
    return visit_tma<ChunkF32<true>>(a.ell_w, a.tma_minb, [&]<class CH, int W, int MB>() {
      return launch_tma<CH, W, MB>(a, cfg, a.tma_stages, a.tma_passes, st);
    });
  return visit_tma<ChunkF32<false>>(a.ell_w, a.tma_minb, [&]<class CH, int W, int MB>() {
    return launch_tma<CH, W, MB>(a, cfg, a.tma_stages, a.tma_passes, st);
  });
}

int occ_ell_tma_f32(bool cplx, const StepArgs& a) {
  if (a.tma_stages < 1 || a.tma_stages > TMA_MAX_STAGES || a.tma_passes < 1) return 0;
  if (cplx)
    return visit_tma<ChunkF32<true>>(a.ell_w, a.tma_minb, [&]<class CH, int W, int MB>() {
      return occupancy_tma<CH, W, MB>(a, a.tma_stages, a.tma_passes);
    });
  return visit_tma<ChunkF32<false>>(a.ell_w, a.tma_minb, [&]<class CH, int W, int MB>() {
    return occupancy_tma<CH, W, MB>(a, a.tma_stages, a.tma_passes);
  });
}

}  // namespace kpm
