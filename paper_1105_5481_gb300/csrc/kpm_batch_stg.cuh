// Staged batched kernel: the batched persistent launch of kpm_batch.cuh for
// stencil operators, with the vector rows brought into shared memory by bulk
// asynchronous copies instead of being loaded by the computing threads.
//
// In the global-memory form every thread requests its rows of v_n, their
// neighbour rows and its rows of v_{n-1} itself, so each pass waits on a
// chain of L2 round trips with a few hundred bytes per warp in flight, and
// decodes the lattice coordinates of each row by integer division.  Here a
// cluster's instance is cut into tiles of T consecutive rows (T a power of
// two); CTA `rank` owns a contiguous band of tiles.  Thread 0 copies the
// tiles of v_n that the band reads (its own tiles and `hs` halo tiles on
// either side, enough to hold the neighbours one lattice line or plane away
// when they fit) into a ring of S shared-memory stages, and the band's tiles
// of v_{n-1} (with the scaled on-site terms) into a second ring of SW stages,
// several tiles ahead of use (cp.async.bulk, completion counted in bytes on
// one mbarrier per stage); it issues them at the start of each tile.  The
// eight warps take the band's tiles in order: every row's own row, its
// neighbour rows inside the halo and its row of v_{n-1} come from shared
// memory; only neighbours across a periodic wrap farther than the halo are
// read from global memory.  A warp releases a stage through a second mbarrier
// once no later tile of the band reads it.  (A dedicated producer warp made
// the block 288 threads, which at two CTAs per SM left 96 registers a thread
// and spilled.)  The per-row arithmetic and its order are those of the
// stencil operator of the fused step (diagonal term, then the forward and
// backward bond of each dimension); the lattice coordinates come from
// multiply-high division by the lattice sides.  v_{n+1} is stored to global
// memory in place over v_{n-1}.  Rows go to threads differently from the
// other forms, so the compensated FP32 moment dots are summed in another
// order: an instance's moments depend only on C, the tile shape and the
// instance (bitwise alone and in any mix), and agree with the other forms to
// rounding.
//
// Between products the cluster barrier orders every CTA's stores of v_{n+1}
// before the next product's copies; the stores are generic-proxy writes and
// the copies asynchronous-proxy reads, so the storing threads and the
// issuing thread each issue a proxy fence on their side of the barrier.  The
// moment partials, the rank-0 sums in rank order, the split cluster barrier
// and the finalisation are those of the global-memory batched kernel.
// Untiled instances only (one task per instance); any step range.
//
// Every wait is bounded (about a second).  A wait that runs out marks the
// CTA: it skips all further copies and waits (still meeting every cluster
// barrier), sets bit 1 of the task's flags for every task it takes part in,
// and the issuing thread waits (again bounded) for every copy it issued before the
// CTA leaves, so no copy can land in the shared memory of an exited CTA.
// The issuing thread waits for a free stage only for a tile two tiles
// behind the one it starts, so no wait depends on a copy not yet issued.
#pragma once

#include "kpm_batch_res.cuh"
#include "kpm_fastdiv.cuh"
#include "kpm_mbar.cuh"

namespace kpm {

constexpr int STG_WARPS = 8;
constexpr int STG_THREADS = 32 * STG_WARPS;
constexpr int STG_MAX_STAGES = 16;     // per ring (the four barrier arrays fill 512 bytes)
#ifndef KPM_STG_MIN_BLOCKS
#define KPM_STG_MIN_BLOCKS 2
#endif

// Global memory access of a chunk without a compiler memory barrier: the
// loads read v_n (not written during a product), the stores write this
// thread's own row of v_{n+1}; ordering across products comes from the
// cluster barrier.
template <class CH>
__device__ __forceinline__ void stg_ld_global(CH& x, const typename CH::T* p) {
  if constexpr (sizeof(typename CH::T) == 8) {
    asm volatile("ld.global.v2.f64 {%0,%1}, [%2];" : "=d"(x.v[0]), "=d"(x.v[1]) : "l"(p));
  } else {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(x.p[0].x), "=f"(x.p[0].y), "=f"(x.p[1].x), "=f"(x.p[1].y), "=f"(x.p[2].x),
                   "=f"(x.p[2].y), "=f"(x.p[3].x), "=f"(x.p[3].y)
                 : "l"(p));
  }
}
template <class CH>
__device__ __forceinline__ void stg_st_global(const CH& x, typename CH::T* p) {
  if constexpr (sizeof(typename CH::T) == 8) {
    asm volatile("st.global.v2.f64 [%0], {%1,%2};" ::"l"(p), "d"(x.v[0]), "d"(x.v[1]));
  } else {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(x.p[0].x),
                 "f"(x.p[0].y), "f"(x.p[1].x), "f"(x.p[1].y), "f"(x.p[2].x), "f"(x.p[2].y),
                 "f"(x.p[3].x), "f"(x.p[3].y));
  }
}

// Shared-memory layout: barriers, CTA reduction scratch, rank-0 partials
// [3 slots][C][2 Rp], then the rings.  A stream stage holds T rows of
// v_{n-1} followed by T scaled on-site terms.
struct StgLayout {
  uint32_t off_red, off_part, off_x, off_w, x_stage, w_stage, w_ds, bytes;
  __host__ __device__ StgLayout(int G, int vec, int chunkB, int scalarB, int C, int Rp, int T,
                                int S, int SW) {
    const size_t rowB = (size_t)G * chunkB;
    off_red = 512;
    off_part = (uint32_t)stg_round(off_red + step_smem_bytes(G, STG_THREADS, vec), 16);
    off_x = (uint32_t)stg_round(off_part + (size_t)3 * C * 2 * Rp * sizeof(double), 128);
    x_stage = (uint32_t)stg_round((size_t)T * rowB, 128);
    w_ds = (uint32_t)stg_round((size_t)T * rowB, 128);
    w_stage = w_ds + (uint32_t)stg_round((size_t)T * scalarB, 128);
    off_w = off_x + (uint32_t)S * x_stage;
    bytes = off_w + (uint32_t)SW * w_stage;
  }
};

template <class CH, class OP>
__global__ void __launch_bounds__(STG_THREADS, KPM_STG_MIN_BLOCKS)
    batch_stg_kernel(BatchTask* tasks, int ntasks, int* queue, int G, int Rp, int Tl, int Sl,
                     int SWl) {
  using T = typename CH::T;
  using RS = ResStencil<OP>;
  constexpr int DIMS = RS::DIMS;
  constexpr int SC = CH::SC;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int TR = 1 << Tl, S = 1 << Sl, SW = 1 << SWl;
  extern __shared__ __align__(128) double stg_smem_d[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(stg_smem_d);
  const StgLayout lay(G, CH::VEC, SC * (int)sizeof(T), (int)sizeof(T), C, Rp, TR, S, SW);
  uint64_t* full_x = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty_x = full_x + STG_MAX_STAGES;
  uint64_t* full_w = full_x + 2 * STG_MAX_STAGES;
  uint64_t* empty_w = full_x + 3 * STG_MAX_STAGES;
  double* red = reinterpret_cast<double*>(smem + lay.off_red);
  double* part = reinterpret_cast<double*>(smem + lay.off_part);
  double* part0 = cluster.map_shared_rank(part, 0);
  unsigned char* ring_x = smem + lay.off_x;
  unsigned char* ring_w = smem + lay.off_w;
  __shared__ int s_task;
  __shared__ int s_bad;
  __shared__ StepArgs s_a;
  __shared__ const void* s_v[2];
  if (t == 0) {
    for (int k = 0; k < S; ++k) {
      mbar::init(&full_x[k], 1);
      mbar::init(&empty_x[k], STG_WARPS);
    }
    for (int k = 0; k < SW; ++k) {
      mbar::init(&full_w[k], 1);
      mbar::init(&empty_w[k], STG_WARPS);
    }
    mbar::init_fence();
    s_bad = 0;
  }
  __syncthreads();
  const int rowB = G * SC * (int)sizeof(T);
  const int rowS = G * SC;
  // running counts of the tiles this CTA has put into each ring (the same in
  // every thread): the k-th goes to stage k mod S, its phase is (k / S) & 1
  int sx = 0, sw = 0;
  // copies issued in total (thread 0; for the final wait after a failure)
  int px = 0, pw = 0;
  bool dead = false;

  for (;;) {
    if (rank == 0 && t == 0) s_task = atomicAdd(queue, 1);
    cluster.sync();
    const int task = *cluster.map_shared_rank(&s_task, 0);
    cluster.sync();
    if (task >= ntasks) break;
    BatchTask& bt = tasks[task];
    if (t == 0) {
      s_a = bt.a;
      s_v[0] = bt.v[0];
      s_v[1] = bt.v[1];
    }
    __syncthreads();
    const int n = (int)s_a.n;
    const int ntiles = (n + TR - 1) >> Tl;
    const int tpc = (ntiles + C - 1) / C;
    const int kf = rank * tpc, kl = min(ntiles, kf + tpc) - 1;  // own tiles (none if kf > kl)
    const int H = DIMS == 1 ? 1 : s_a.geom.stride[DIMS - 1];
    const int hs = min((H + TR - 1) >> Tl, (S - 2) >> 1);      // halo tiles held on each side
    const int tlo = max(0, kf - hs), thi = min(ntiles - 1, kl + hs);
    const int nx = kf <= kl ? thi - tlo + 1 : 0;                // v_n tiles copied per product
    const int nown = kf <= kl ? kl - kf + 1 : 0;
    // copy look-ahead in tiles: a stage is refilled once every warp has
    // finished the tile two before the one being started
    const int ahead_x = S - 2 * hs - 2, ahead_w = SW - 2;
    const int nsteps = bt.M / 2;
    auto sum_partials = [&](int st) {
      const double* pp = part + (size_t)(st % 3) * C * 2 * Rp;
      for (int o = t; o < 2 * Rp; o += blockDim.x) {
        double sum = 0.0;
        for (int r = 0; r < C; ++r) sum += pp[(size_t)r * 2 * Rp + o];
        bt.sums[(size_t)st * 2 * Rp + o] = sum;
      }
    };

    for (int step = bt.step_begin; step < bt.step_end; ++step) {
      const bool first = step == 0;
      const unsigned char* X = reinterpret_cast<const unsigned char*>(s_v[step & 1]);
      unsigned char* Y = reinterpret_cast<unsigned char*>(const_cast<void*>(s_v[(step + 1) & 1]));
      // the stream ring carries v_{n-1} (after the first step) and the on-site terms
      const bool use_w = !first || RS::HAS_DS;
      if (first) {
        T* v0 = reinterpret_cast<T*>(const_cast<void*>(s_v[0]));
        const int64_t total = (int64_t)n * Rp;
        for (int64_t e = (int64_t)rank * blockDim.x + t; e < total; e += (int64_t)C * blockDim.x)
          random_entry<T, CH::CPLX>(v0, n, Rp, bt.R, bt.seed, (unsigned long long)bt.realisation, e);
        mbar::fence_proxy_async_global();
        cluster.sync();
      }
      dead = dead || s_bad != 0;
      typename CH::Acc s;
      CH::acc_zero(s);
      if (!dead && nown > 0) {
        // Copies are issued by thread 0 at the start of each tile, up to the
        // look-ahead; a stage's previous tile was released by every warp one
        // tile earlier, so its wait rarely blocks.  The stores of the last
        // product (every CTA's, ordered by the cluster barrier) precede
        // these asynchronous-proxy reads.
        int ix = tlo, iw = kf;
        auto issue = [&](int k) {
          if (t != 0) return;
          const int xt = min(thi, k + hs + ahead_x);
          for (; ix <= xt && !dead; ++ix) {
            const int q = sx + (ix - tlo), st = q & (S - 1);
            if (q >= S && !mbar::wait(&empty_x[st], (uint32_t)(((q >> Sl) - 1) & 1))) {
              dead = true;
              break;
            }
            const uint32_t bytes = (uint32_t)min(TR, n - (ix << Tl)) * rowB;
            mbar::expect_tx(&full_x[st], bytes);
            mbar::bulk_g2s(ring_x + (size_t)st * lay.x_stage, X + (size_t)(ix << Tl) * rowB, bytes,
                           &full_x[st]);
            ++px;
          }
          if (!use_w) return;
          const int wt = min(kl, k + ahead_w);
          for (; iw <= wt && !dead; ++iw) {
            const int q = sw + (iw - kf), st = q & (SW - 1);
            if (q >= SW && !mbar::wait(&empty_w[st], (uint32_t)(((q >> SWl) - 1) & 1))) {
              dead = true;
              break;
            }
            const int nr = min(TR, n - (iw << Tl));
            const uint32_t bw = first ? 0u : (uint32_t)nr * rowB;
            const uint32_t bd = RS::HAS_DS ? (uint32_t)stg_round((size_t)nr * sizeof(T), 16) : 0u;
            mbar::expect_tx(&full_w[st], bw + bd);
            unsigned char* dst = ring_w + (size_t)st * lay.w_stage;
            if (bw) mbar::bulk_g2s(dst, Y + (size_t)(iw << Tl) * rowB, bw, &full_w[st]);
            if (bd)
              mbar::bulk_g2s(dst + lay.w_ds, reinterpret_cast<const T*>(s_a.ds) + ((size_t)iw << Tl),
                             bd, &full_w[st]);
            ++pw;
          }
        };
        if (t == 0) mbar::fence_proxy_async_global();
        T hu_r, hu_i, du;
        scal_from_block<T>(s_a.sc, hu_r, hu_i, du);
        const int c = t % G, q = t / G, spi = STG_THREADS / G;
        const int tp = TR / spi;
        int Ld[DIMS], Sd[DIMS];
        bool Pd[DIMS];
#pragma unroll
        for (int d2 = 0; d2 < DIMS; ++d2) {
          Ld[d2] = s_a.geom.L[d2];
          Sd[d2] = s_a.geom.stride[d2];
          Pd[d2] = s_a.geom.periodic[d2] != 0;
        }
        const FastDiv f0 = fast_div((unsigned)Ld[0]);
        const FastDiv f1 = fast_div(DIMS == 3 ? (unsigned)Ld[1] : 1u);
        const T* Xg = reinterpret_cast<const T*>(X) + c * SC;
        T* Yg = reinterpret_cast<T*>(Y) + c * SC;
        int wx = tlo - 1;  // last v_n tile waited for
        for (int k = kf; k <= kl; ++k) {
          issue(k);
          // a failed wait ends the warp's work (decided for the whole warp)
          if (warp == 0) dead = __any_sync(0xffffffffu, dead);
          if (dead) break;
          const int need = min(k + hs, thi);
          bool ok = true;
          while (wx < need && ok) {
            ++wx;
            const int qq = sx + (wx - tlo);
            ok = mbar::wait(&full_x[qq & (S - 1)], (uint32_t)((qq >> Sl) & 1));
          }
          const int qw = sw + (k - kf);
          if (ok && use_w) ok = mbar::wait(&full_w[qw & (SW - 1)], (uint32_t)((qw >> SWl) & 1));
          if (!__all_sync(0xffffffffu, ok)) {
            dead = true;
            break;
          }
          const unsigned char* tx = ring_x + (size_t)((sx + (k - tlo)) & (S - 1)) * lay.x_stage;
          const unsigned char* tw = ring_w + (size_t)(qw & (SW - 1)) * lay.w_stage;
          // chunk c of v_n row j: from shared memory inside the halo, from
          // global memory across a farther periodic wrap
          auto load_x = [&](CH& out, int j) {
            const int tj = j >> Tl;
            if ((unsigned)(tj - tlo) <= (unsigned)(thi - tlo) &&
                (unsigned)(tj - k + hs) <= (unsigned)(2 * hs)) {
              const unsigned char* sp =
                  ring_x + ((size_t)((sx + (tj - tlo)) & (S - 1)) * lay.x_stage +
                            (size_t)(j & (TR - 1)) * rowB);
              out.ld_shared(reinterpret_cast<const T*>(sp) + c * SC);
            } else {
              stg_ld_global(out, Xg + (size_t)j * rowS);
            }
          };
          for (int p = 0; p < tp; ++p) {
            const int lr = p * spi + q;
            const int i = (k << Tl) + lr;
            if (i >= n) break;
            CH xi, acc;
            xi.ld_shared(reinterpret_cast<const T*>(tx + (size_t)lr * rowB) + c * SC);
            if (first) {
              acc.zero();
            } else {
              CH wv;
              wv.ld_shared(reinterpret_cast<const T*>(tw + (size_t)lr * rowB) + c * SC);
              acc.set_neg(wv);
            }
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
            const T d = RS::HAS_DS ? reinterpret_cast<const T*>(tw + lay.w_ds)[lr] : du;
            acc.axpy(d, xi);
#pragma unroll
            for (int d2 = 0; d2 < DIMS; ++d2) {
              const int L = Ld[d2], sd = Sd[d2], x = xc[d2];
              const bool per = Pd[d2];
              const bool hf = (x + 1 < L) || per, hb = (x > 0) || per;
              const int jf = (x + 1 < L) ? i + sd : (per ? i - (L - 1) * sd : i);
              const int jb = (x > 0) ? i - sd : (per ? i + (L - 1) * sd : i);
              T fr, fi, br, bi;
              if constexpr (RS::HAS_HOP) {
                const T* hsp = reinterpret_cast<const T*>(s_a.hs);
                if constexpr (CH::CPLX) {
                  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
                  const T2 f = __ldg(reinterpret_cast<const T2*>(hsp) + ((size_t)i * DIMS + d2));
                  const T2 bk = __ldg(reinterpret_cast<const T2*>(hsp) + ((size_t)jb * DIMS + d2));
                  fr = f.x;
                  fi = f.y;
                  br = bk.x;
                  bi = -bk.y;
                } else {
                  fr = __ldg(hsp + (size_t)i * DIMS + d2);
                  br = __ldg(hsp + (size_t)jb * DIMS + d2);
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
              load_x(xf, jf);
              load_x(xb, jb);
              acc.cmac(fr, fi, xf);
              acc.cmac(br, bi, xb);
            }
            if (first) acc.half();
            stg_st_global(acc, Yg + (size_t)i * rowS);
            CH::acc_add(s, xi, acc);
          }
          __syncwarp();
          if (lane == 0) {
            if (use_w) mbar::arrive(&empty_w[qw & (SW - 1)]);
            if (k - hs >= tlo) mbar::arrive(&empty_x[(sx + (k - hs - tlo)) & (S - 1)]);
          }
        }
        // the halo tiles above the band are no longer needed either
        if (!dead && lane == 0)
          for (int t2 = max(tlo, kl - hs + 1); t2 <= thi; ++t2)
            mbar::arrive(&empty_x[(sx + (t2 - tlo)) & (S - 1)]);
        if (dead) s_bad = 1;
        __syncwarp();
        mbar::fence_proxy_async_global();  // this product's stores before the next copies
      }
      sx += nx;
      if (use_w) sw += nown;
      cluster_arrive_release();
      cta_reduce<CH>(s_a, s, 0, red, part0 + ((size_t)(step % 3) * C + rank) * 2 * Rp);
      cluster_wait_acquire();
      if (rank == 0 && step > bt.step_begin) sum_partials(step - 1);
    }
    if (bt.step_begin < bt.step_end) {
      cluster.sync();  // the partials of the last product of this launch
      if (rank == 0) sum_partials(bt.step_end - 1);
    }
    if (s_bad && t == 0) atomicOr(&bt.flags, BATCH_FLAG_TIMEOUT);
    if (bt.step_end == nsteps && bt.step_begin < bt.step_end && rank == 0) {
      __syncthreads();  // rank 0's own sums writes above
      const int R = bt.R, M = bt.M;
      const double inv_n = 1.0 / (double)n;
      for (int e = t; e < R * nsteps; e += blockDim.x) {
        const int r = e / nsteps, st = e % nsteps;
        const double mu0 = bt.sums[r] * inv_n, mu1 = bt.sums[Rp + r] * inv_n;
        double me = mu0, mo = mu1;
        if (st > 0) {
          me = 2.0 * bt.sums[(size_t)st * 2 * Rp + r] * inv_n - mu0;
          mo = 2.0 * bt.sums[(size_t)st * 2 * Rp + Rp + r] * inv_n - mu1;
        }
        bt.per_vec[(size_t)r * M + 2 * st] = me;
        bt.per_vec[(size_t)r * M + 2 * st + 1] = mo;
        if (!(fabs(me) <= 1.0 + 1e-6) || !(fabs(mo) <= 1.0 + 1e-6)) atomicOr(&bt.flags, 1);
      }
      __syncthreads();
      for (int m = t; m < M; m += blockDim.x) {
        double acc = 0.0;
        for (int r = 0; r < R; ++r) acc += bt.per_vec[(size_t)r * M + m];
        bt.mu[m] = acc / (double)R;
      }
    }
    cluster.sync();  // the instance is complete on every CTA of the cluster (and s_a free)
  }
  // after a wait that ran out, copies may still be in flight: wait for them
  // (bounded) before the CTA's shared memory is released
  if (t == 0 && (dead || s_bad)) {
    for (int k = max(0, px - S); k < px; ++k)
      mbar::wait(&full_x[k & (S - 1)], (uint32_t)((k >> Sl) & 1));
    for (int k = max(0, pw - SW); k < pw; ++k)
      mbar::wait(&full_w[k & (SW - 1)], (uint32_t)((k >> SWl) & 1));
  }
}

template <class CH>
inline StgLayout stg_layout(int G, int C, int Rp, int Tl, int Sl, int SWl) {
  return StgLayout(G, CH::VEC, CH::SC * (int)sizeof(typename CH::T), (int)sizeof(typename CH::T),
                   C, Rp, 1 << Tl, 1 << Sl, 1 << SWl);
}

// Raises the staged kernel's dynamic shared-memory limit to the opt-in
// limit of a block minus its static shared memory, and allows clusters of
// 16, once per device; returns the limit (0 on failure).
template <class CH, class OP>
size_t stg_smem_limit() {
  auto kern = batch_stg_kernel<CH, OP>;
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
cudaError_t launch_batch_stg_one(BatchTask* tasks, int ntasks, int* queue, int grid, int C, int G,
                                 int Rp, int Tl, int Sl, int SWl, cudaStream_t st) {
  if constexpr (!ResStencil<OP>::value) {
    return cudaErrorNotSupported;
  } else {
    const size_t smem = stg_layout<CH>(G, C, Rp, Tl, Sl, SWl).bytes;
    if (smem > stg_smem_limit<CH, OP>()) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STG_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, batch_stg_kernel<CH, OP>, tasks, ntasks, queue,
                                             G, Rp, Tl, Sl, SWl);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
  }
}

// Co-resident clusters of the staged kernel (0: not launchable).
template <class CH, class OP>
int batch_stg_max_clusters(int C, int G, int Rp, int Tl, int Sl, int SWl) {
  if constexpr (!ResStencil<OP>::value) {
    return 0;
  } else {
    const size_t smem = stg_layout<CH>(G, C, Rp, Tl, Sl, SWl).bytes;
    if (smem > stg_smem_limit<CH, OP>()) return 0;
    auto kern = batch_stg_kernel<CH, OP>;
    int n = 0;
    if (C == 1) {
      int dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, STG_THREADS, smem) !=
              cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return n * sms;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(STG_THREADS);
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
