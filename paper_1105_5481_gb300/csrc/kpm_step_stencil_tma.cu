// Fused Chebyshev step (Eq. (rn) with the two moment dots of the doubling
// identities) for matrix-free stencil operators with FP32 vectors, fed by
// bulk asynchronous copies through a shared-memory pipeline.
//
// The plain stencil step (StencilOp in kpm_step.cuh) keeps, per thread, the
// streamed row of v_{n-1}, the row's own v_n and its neighbour rows in
// registers while they are in flight, and is bound by the latency of those
// loads (about 62 % of the DRAM cycles busy on the 3D L = 64 spin lattice).
// Here the contiguous part of a tile of T consecutive rows - the rows of v_n
// and v_{n-1}, the forward hoppings and the on-site terms - is copied into a
// ring of shared-memory stages by one producer warp (cp.async.bulk,
// completion counted in bytes on an mbarrier per stage), several tiles
// ahead.  Eight consumer warps wait for a stage, take the row's own v_n,
// v_{n-1}, forward hoppings and on-site term from it, read the x-neighbours
// inside the tile from it as well, gather the other neighbour rows of v_n
// (y and z, and x across the tile's edge) and the backward hoppings from
// global memory (L2: the tiles are handed to the CTAs in row order, so the
// rows one line or plane away were read by another CTA shortly before),
// compute v_{n+1} = 2 H~ v_n - v_{n-1} and the dots A = <v_n|v_n>,
// B = Re<v_{n+1}|v_n>, store v_{n+1} in place over v_{n-1} and release the
// stage.  The per-row arithmetic and its order are those of StencilOp (the
// diagonal term, then the forward and backward bond of each dimension);
// rows go to threads differently, so the compensated FP32 moment dots are
// summed in another order and the moments differ from the plain step's
// within that summation's bound.
//
// Every wait is bounded (about a second).  A wait that runs out sets bit 2
// of *a.err, stops the warp's work, and the producer waits (again bounded)
// for every copy it issued before the CTA leaves.
//
// The planner takes this form only when asked (KPM_STENCIL_TMA): on the 3D
// L = 64 spin lattice (R = 64 complex) it measured 77.8 us per step against
// 75.9 us for the plain step.  Unlike the padded-ELL step, whose neighbour
// loads wait for their column indices, the stencil's neighbour addresses are
// arithmetic, so the plain step already issues all its loads at once; what
// remains is the latency of the four neighbour rows a line or plane away,
// which this form still gathers through L2.
#include "kpm_batch_res.cuh"
#include "kpm_fastdiv.cuh"
#include "kpm_mbar.cuh"

namespace kpm {
namespace {

constexpr int ST_CONSUMER_WARPS = 8;
constexpr int ST_CONSUMERS = 32 * ST_CONSUMER_WARPS;
constexpr int ST_THREADS = ST_CONSUMERS + 32;
constexpr int ST_MAX_STAGES = 8;
constexpr int ST_ERR_TIMEOUT = 4;

// Byte layout of one stage of T rows: v_n rows, v_{n-1} rows, forward
// hoppings [T][DIMS], on-site terms [T] (each part 128-byte aligned).
struct StStage {
  uint32_t off_x, off_w, off_h, off_d, bytes;
  __host__ __device__ StStage(int rows, int rowB, int hopB, int dsB) {
    off_x = 0;
    off_w = (uint32_t)stg_round((size_t)rows * rowB, 128);
    off_h = off_w + (uint32_t)stg_round((size_t)rows * rowB, 128);
    off_d = off_h + (uint32_t)stg_round((size_t)rows * hopB, 128);
    bytes = off_d + (uint32_t)stg_round((size_t)rows * dsB, 128);
  }
};

__host__ __device__ inline size_t st_red_bytes(int G, int vec) {
  return step_smem_bytes(G, ST_THREADS, vec);
}
__host__ __device__ inline size_t st_smem_bytes(int stages, int rows, int rowB, int hopB, int dsB,
                                                int G, int vec) {
  return 256 + stg_round(st_red_bytes(G, vec), 128) +
         (size_t)stages * StStage(rows, rowB, hopB, dsB).bytes;
}

template <class CH, class OP, int MINB>
__global__ void __launch_bounds__(ST_THREADS, MINB)
    stencil_tma_step_kernel(const StepArgs a, int stages, int tile_passes) {
  using T = typename CH::T;
  using RS = ResStencil<OP>;
  constexpr int DIMS = RS::DIMS;
  constexpr int SC = CH::SC;
  constexpr bool CPLX = CH::CPLX;
  constexpr int HOPB = RS::HAS_HOP ? DIMS * (int)sizeof(T) * (CPLX ? 2 : 1) : 0;
  constexpr int DSB = RS::HAS_DS ? (int)sizeof(T) : 0;
  extern __shared__ __align__(128) double st_smem_d[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(st_smem_d);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + ST_MAX_STAGES;
  double* red = reinterpret_cast<double*>(smem + 256);
  const int G = a.G;
  const int rowB = G * SC * (int)sizeof(T);
  const int spi = ST_CONSUMERS / G;  // rows per pass
  const int rows = spi * tile_passes;
  const StStage L(rows, rowB, HOPB, DSB);
  unsigned char* stage0 = smem + 256 + stg_round(st_red_bytes(G, CH::VEC), 128);
  const int n = (int)a.n;
  const int ntiles = (n + rows - 1) / rows;
  const int ncta = gridDim.x, cta = blockIdx.x;
  const int my_tiles = ntiles > cta ? (ntiles - 1 - cta) / ncta + 1 : 0;
  auto tile_of = [&](int k) {
    const int t_ = cta + k * ncta;
    return a.reverse ? ntiles - 1 - t_ : t_;
  };
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar::init(&full[s], 1);
      mbar::init(&empty[s], ST_CONSUMER_WARPS);
    }
    mbar::init_fence();
  }
  __syncthreads();
  typename CH::Acc s;
  CH::acc_zero(s);
  bool timed_out = false;
  if (warp == ST_CONSUMER_WARPS) {
    // producer warp: lane 0 issues the copies of tile k into stage k % stages,
    // the whole warp running the loop together
    int issued = 0;
    const int to_issue = a.tma_stall ? 0 : my_tiles;  // testing aid: no copies
    for (int k = 0; k < to_issue; ++k) {
      const int st = k % stages;
      const bool ok = k < stages || mbar::wait(&empty[st], (uint32_t)((k / stages - 1) & 1));
      if (!__all_sync(0xffffffffu, ok)) {
        timed_out = true;
        break;
      }
      const int r0 = tile_of(k) * rows;
      const int nr = min(rows, n - r0);
      if (lane == 0) {
        unsigned char* sp = stage0 + (size_t)st * L.bytes;
        const uint32_t bx = (uint32_t)nr * rowB;
        const uint32_t bh = (uint32_t)stg_round((size_t)nr * HOPB, 16);
        const uint32_t bd = (uint32_t)stg_round((size_t)nr * DSB, 16);
        mbar::expect_tx(&full[st], 2 * bx + bh + bd);
        mbar::bulk_g2s(sp + L.off_x, reinterpret_cast<const unsigned char*>(a.x) + (size_t)r0 * rowB,
                       bx, &full[st]);
        mbar::bulk_g2s(sp + L.off_w, reinterpret_cast<const unsigned char*>(a.w) + (size_t)r0 * rowB,
                       bx, &full[st]);
        if (bh)
          mbar::bulk_g2s(sp + L.off_h,
                         reinterpret_cast<const unsigned char*>(a.hs) + (size_t)r0 * HOPB, bh,
                         &full[st]);
        if (bd)
          mbar::bulk_g2s(sp + L.off_d,
                         reinterpret_cast<const unsigned char*>(a.ds) + (size_t)r0 * DSB, bd,
                         &full[st]);
      }
      issued = k + 1;
    }
    __syncwarp();
    // every copy this CTA issued must have landed before the CTA may exit
    if (lane == 0)
      for (int k = issued > stages ? issued - stages : 0; k < issued; ++k)
        if (!mbar::wait(&full[k % stages], (uint32_t)((k / stages) & 1))) timed_out = true;
    __syncwarp();
  } else {
    // consumers
    const int c = t % G, q = t / G;
    T hu_r, hu_i, du;
    scal_from_block<T>(a.sc, hu_r, hu_i, du);
    const size_t rowS = (size_t)G * SC;
    const T* __restrict__ Xc = reinterpret_cast<const T*>(a.x) + (size_t)c * SC;
    T* Yc = reinterpret_cast<T*>(a.y) + (size_t)c * SC;
    int Ld[DIMS], Sd[DIMS];
    bool Pd[DIMS];
#pragma unroll
    for (int d2 = 0; d2 < DIMS; ++d2) {
      Ld[d2] = a.geom.L[d2];
      Sd[d2] = a.geom.stride[d2];
      Pd[d2] = a.geom.periodic[d2] != 0;
    }
    const FastDiv f0 = fast_div((unsigned)Ld[0]);
    const FastDiv f1 = fast_div(DIMS == 3 ? (unsigned)Ld[1] : 1u);
    for (int k = 0; k < my_tiles; ++k) {
      const int st = k % stages;
      if (!__all_sync(0xffffffffu, mbar::wait(&full[st], (uint32_t)((k / stages) & 1)))) {
        timed_out = true;
        break;
      }
      const int r0 = tile_of(k) * rows;
      const unsigned char* sp = stage0 + (size_t)st * L.bytes;
      for (int p = 0; p < tile_passes; ++p) {
        const int lr = p * spi + q;
        const int i = r0 + lr;
        if (i >= n) break;
        const T* sx = reinterpret_cast<const T*>(sp + L.off_x + (size_t)lr * rowB) + c * SC;
        const T* sw = reinterpret_cast<const T*>(sp + L.off_w + (size_t)lr * rowB) + c * SC;
        CH xi, wv, acc;
        xi.ld_shared(sx);
        wv.ld_shared(sw);
        acc.set_neg(wv);
        int xc[DIMS];
        {
          const unsigned r1 = fdiv((unsigned)i, f0);
          xc[0] = i - (int)r1 * Ld[0];
          if constexpr (DIMS == 2) xc[1] = (int)r1;
          if constexpr (DIMS == 3) {
            const unsigned r2 = fdiv(r1, f1);
            xc[1] = (int)r1 - (int)r2 * Ld[1];
            xc[2] = (int)r2;
          }
        }
        const T d = RS::HAS_DS ? reinterpret_cast<const T*>(sp + L.off_d)[lr] : du;
        acc.axpy(d, xi);
        T fr[DIMS], fi[DIMS], br[DIMS], bi[DIMS];
        int jf[DIMS], jb[DIMS];
#pragma unroll
        for (int d2 = 0; d2 < DIMS; ++d2) {
          const int Lx = Ld[d2], sd = Sd[d2], x = xc[d2];
          const bool per = Pd[d2];
          const bool hf = (x + 1 < Lx) || per, hb = (x > 0) || per;
          jf[d2] = (x + 1 < Lx) ? i + sd : (per ? i - (Lx - 1) * sd : i);
          jb[d2] = (x > 0) ? i - sd : (per ? i + (Lx - 1) * sd : i);
          if constexpr (RS::HAS_HOP) {
            const T* hrow = reinterpret_cast<const T*>(sp + L.off_h + (size_t)lr * HOPB);
            const T* hs = reinterpret_cast<const T*>(a.hs);
            if constexpr (CPLX) {
              using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
              const T2 bk = __ldg(reinterpret_cast<const T2*>(hs) + ((size_t)jb[d2] * DIMS + d2));
              fr[d2] = hrow[2 * d2];
              fi[d2] = hrow[2 * d2 + 1];
              br[d2] = bk.x;
              bi[d2] = -bk.y;
            } else {
              fr[d2] = hrow[d2];
              br[d2] = __ldg(hs + (size_t)jb[d2] * DIMS + d2);
              fi[d2] = bi[d2] = T(0);
            }
          } else {
            fr[d2] = hu_r;
            fi[d2] = hu_i;
            br[d2] = hu_r;
            bi[d2] = -hu_i;
          }
          if (!hf) fr[d2] = fi[d2] = T(0);
          if (!hb) br[d2] = bi[d2] = T(0);
        }
        // neighbour rows: inside the tile from its copy, else through L2
        CH xf[DIMS], xb[DIMS];
#pragma unroll
        for (int d2 = 0; d2 < DIMS; ++d2) {
          const int lf = jf[d2] - r0, lb = jb[d2] - r0;
          if (d2 == 0 && (unsigned)lf < (unsigned)rows && jf[d2] < n)
            xf[d2].ld_shared(reinterpret_cast<const T*>(sp + L.off_x + (size_t)lf * rowB) + c * SC);
          else
            xf[d2].ld_nc(Xc + (size_t)jf[d2] * rowS);
          if (d2 == 0 && (unsigned)lb < (unsigned)rows && jb[d2] < n)
            xb[d2].ld_shared(reinterpret_cast<const T*>(sp + L.off_x + (size_t)lb * rowB) + c * SC);
          else
            xb[d2].ld_nc(Xc + (size_t)jb[d2] * rowS);
        }
#pragma unroll
        for (int d2 = 0; d2 < DIMS; ++d2) {
          acc.cmac(fr[d2], fi[d2], xf[d2]);
          acc.cmac(br[d2], bi[d2], xb[d2]);
        }
        acc.st(Yc + (size_t)i * rowS);
        CH::acc_add(s, xi, acc);
      }
      __syncwarp();
      if (lane == 0) mbar::arrive(&empty[st]);
    }
  }
  if (timed_out && a.err) atomicOr(a.err, ST_ERR_TIMEOUT);
  cta_reduce<CH, OP::kPairReduce>(a, s, 0, red, a.partial + (size_t)blockIdx.x * 2 * a.Rp);
}

template <class CH, class OP, int MINB>
struct StTag {};

template <class CH, class OP, int MINB>
size_t st_smem(const StepArgs& a, int stages, int tile_passes) {
  using RS = ResStencil<OP>;
  constexpr int HOPB =
      RS::HAS_HOP ? RS::DIMS * (int)sizeof(typename CH::T) * (CH::CPLX ? 2 : 1) : 0;
  constexpr int DSB = RS::HAS_DS ? (int)sizeof(typename CH::T) : 0;
  const int rowB = a.G * CH::SC * (int)sizeof(typename CH::T);
  const int rows = ST_CONSUMERS / a.G * tile_passes;
  return st_smem_bytes(stages, rows, rowB, HOPB, DSB, a.G, CH::VEC);
}

template <class CH, class OP, int MINB>
cudaError_t launch_st(const StepArgs& a, const LaunchCfg& cfg, cudaStream_t st) {
  const size_t smem = st_smem<CH, OP, MINB>(a, a.tma_stages, a.tma_passes);
  auto kern = stencil_tma_step_kernel<CH, OP, MINB>;
  cudaError_t e = allow_smem<StTag<CH, OP, MINB>>(kern, smem);
  if (e != cudaSuccess) return e;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  kern<<<cfg.grid, ST_THREADS, smem, st>>>(a, a.tma_stages, a.tma_passes);
  return cudaGetLastError();
}

template <class CH, class OP, int MINB>
int occupancy_st(const StepArgs& a) {
  const size_t smem = st_smem<CH, OP, MINB>(a, a.tma_stages, a.tma_passes);
  auto kern = stencil_tma_step_kernel<CH, OP, MINB>;
  if (allow_smem<StTag<CH, OP, MINB>>(kern, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, ST_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

// Stencil operators of two or three dimensions (a one-dimensional chain has
// no rows that are far apart to overlap).
template <class CH, class F>
auto visit_st(const StepArgs& a, F&& f) {
  const bool hh = a.hs != nullptr, hd = a.ds != nullptr;
  const bool m3 = a.tma_minb >= 3;
#define KPM_ST_CASE(D, H, S)                                                        \
  if (a.geom.dims == D && hh == H && hd == S)                                       \
    return m3 ? f.template operator()<CH, StencilOp<CH, D, H, S>, 3>()              \
              : f.template operator()<CH, StencilOp<CH, D, H, S>, 2>();
  KPM_ST_CASE(3, true, false) KPM_ST_CASE(3, true, true) KPM_ST_CASE(3, false, false)
  KPM_ST_CASE(3, false, true) KPM_ST_CASE(2, true, false) KPM_ST_CASE(2, true, true)
  KPM_ST_CASE(2, false, false)
#undef KPM_ST_CASE
  return m3 ? f.template operator()<CH, StencilOp<CH, 2, false, true>, 3>()
            : f.template operator()<CH, StencilOp<CH, 2, false, true>, 2>();
}

}  // namespace

bool stencil_tma_supported(const StepArgs& a, bool fp32) {
  // FP32 vectors, 2D or 3D stencils, whole rows per CTA of at most 32 chunks
  return fp32 && (a.geom.dims == 2 || a.geom.dims == 3) && a.G == a.Gt && a.G <= 32 && a.n >= 1 &&
         a.n < (int64_t)1 << 31;
}

cudaError_t launch_stencil_tma_f32(bool cplx, const StepArgs& a, const LaunchCfg& cfg,
                                   cudaStream_t st) {
  if (a.tma_stages < 1 || a.tma_stages > ST_MAX_STAGES || a.tma_passes < 1)
    return cudaErrorInvalidValue;
  auto go = [&]<class CH, class OP, int MB>() { return launch_st<CH, OP, MB>(a, cfg, st); };
  return cplx ? visit_st<ChunkF32<true>>(a, go) : visit_st<ChunkF32<false>>(a, go);
}

int occ_stencil_tma_f32(bool cplx, const StepArgs& a) {
  if (a.tma_stages < 1 || a.tma_stages > ST_MAX_STAGES || a.tma_passes < 1) return 0;
  auto go = [&]<class CH, class OP, int MB>() { return occupancy_st<CH, OP, MB>(a); };
  return cplx ? visit_st<ChunkF32<true>>(a, go) : visit_st<ChunkF32<false>>(a, go);
}

}  // namespace kpm
