// C ABI of the KPM library: handle creation (lattice stencil or CSR), spectral
// bounds, Chebyshev moments and the DOS.  The host code here validates
// arguments, owns device memory, captures the per-realisation kernel sequence
// into a CUDA graph and replays it; every arithmetic step runs in the kernels
// of kpm_step_*.cu and kpm_aux.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kpm_colres.h"
#include "kpm_internal.h"

namespace kpm {

// vector columns per chunk (FP32: 32-byte chunks; FP64: 16-byte chunks)
int vec_per_chunk(bool fp32, bool cplx) { return fp32 ? (cplx ? 4 : 8) : (cplx ? 1 : 2); }

void padded_width(int R, bool fp32, bool cplx, int* Rp, int* G) {
  const int vec = vec_per_chunk(fp32, cplx);
  int g = (R + vec - 1) / vec;
  int p2 = 1;
  while (p2 < g) p2 <<= 1;
  *G = p2;
  *Rp = p2 * vec;
}

size_t elem_bytes(bool fp32, bool cplx) { return (fp32 ? 4 : 8) * (cplx ? 2 : 1); }

static thread_local std::string t_err;
std::atomic<uint64_t> g_launches{0};

void set_error(const std::string& msg) { t_err = msg; }
kpm_status fail(kpm_status st, const std::string& msg) {
  t_err = msg;
  return st;
}
kpm_status cuda_fail(cudaError_t e, const char* what) {
  t_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? KPM_ENOMEM : KPM_ECUDA;
}

namespace {

constexpr int RING = 64;          // step slots between two cross-CTA reductions
constexpr int BLOCK = 256;

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device memory comes from a library-owned, stream-ordered pool per device
// that keeps freed memory (release threshold = unlimited): creating, solving
// and destroying handles repeatedly reuses it without cudaMalloc/cudaFree.
constexpr int MAX_DEVICES = 64;
cudaMemPool_t g_pools[MAX_DEVICES] = {};
std::mutex g_pool_mu;

cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = p;
  }
  return g_pools[dev];
}

// Allocation ordered on `st` (memory usable by work enqueued on `st` after it).
cudaError_t palloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = device_pool();
  if (!pool) return cudaMalloc(p, bytes);
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void pfree(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// Synchronous-use allocation: ordered on the legacy stream and completed
// before return, so any stream may use the memory afterwards.
// Host-side fault injection for tests (kpm_testing_fail_allocations): the
// number of dalloc calls that still succeed before one fails; -1 = off.
std::atomic<long long> g_fail_alloc_after{-1};
// Testing aid (kpm_testing_stall_step_pipeline): plans made while it is set
// give the TMA-fed step a producer that issues nothing.
std::atomic<int> g_test_stall{0};

bool injected_alloc_failure() {
  long long k = g_fail_alloc_after.load();
  while (k >= 0) {
    if (g_fail_alloc_after.compare_exchange_weak(k, k - 1)) return k == 0;
  }
  return false;
}

template <typename T>
kpm_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return KPM_OK;
  if (injected_alloc_failure())
    return fail(KPM_ENOMEM, "device allocation (failure injected by kpm_testing_fail_allocations)");
  cudaError_t e = palloc((void**)p, count * sizeof(T), 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "device allocation");
  }
  return KPM_OK;
}

void dfree(void* p) { pfree(p, 0); }

kpm_status check_device(int* dev) {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(KPM_ECUDA, "no usable CUDA device");
  }
  KPM_CUDA(cudaGetDevice(dev));
  return KPM_OK;
}

void free_dense_tc(kpm_handle_s::Work& w) {
  if (!w.dtc) return;
  DenseTC& d = *w.dtc;
  dense_tc_destroy_blas(d);
  dfree(d.workspace);
  dfree(d.A);
  dfree(d.B);
  dfree(d.C);
  dfree(d.row_scale);
  dfree(d.col_scale);
  dfree(d.cmax);
  delete w.dtc;
  w.dtc = nullptr;
}

// The dense product of a real FP64 dense handle runs on the tensor cores
// (kpm_dense_tc.cu) unless KPM_DENSE_TENSOR=0; by default from n = 512 on
// (below that the FP64 kernel is as fast), always with KPM_DENSE_TENSOR=1.
bool dense_tc_wanted(const kpm_handle_s* h, bool fp32) {
  if (!h->dense || h->cplx || fp32) return false;
  const char* env = getenv("KPM_DENSE_TENSOR");
  if (env && env[0] == '0') return false;
  if (env && env[0] == '1') return true;
  return h->n >= 512;
}

// Buffers of the tensor-core form; false (and nothing kept) if they do not fit.
bool setup_dense_tc(kpm_handle_s* h, int Rp) {
  auto& w = h->work;
  free_dense_tc(w);
  auto* d = new DenseTC;
  d->n = h->n;
  d->Rp = Rp;
  dense_tc_split(h->n, &d->beta, &d->k);
  const size_t n = (size_t)h->n, k = (size_t)d->k;
  const size_t cbytes = dense_tc_c_floats(h->n, Rp, d->k) * sizeof(float);
  d->ws_bytes = 32u << 20;
  bool ok = cbytes <= ((size_t)64 << 30) && dalloc((char**)&d->workspace, d->ws_bytes) == KPM_OK &&
            dalloc(&d->A, k * n * n) == KPM_OK && dalloc(&d->B, k * n * Rp) == KPM_OK &&
            dalloc((char**)&d->C, cbytes) == KPM_OK && dalloc(&d->row_scale, n) == KPM_OK &&
            dalloc(&d->col_scale, (size_t)Rp) == KPM_OK && dalloc(&d->cmax, (size_t)Rp) == KPM_OK;
  w.dtc = d;
  if (ok) ok = dense_tc_create_blas(*d) == cudaSuccess;
  if (!ok) {
    free_dense_tc(w);
    t_err.clear();
  }
  return ok;
}

void free_work(kpm_handle_s* h) {
  auto& w = h->work;
  if (w.exec) cudaGraphExecDestroy(w.exec);
  free_dense_tc(w);
  dfree(w.v[0]);
  dfree(w.v[1]);
  dfree(w.ring);
  dfree(w.sums);
  dfree(w.per_vec);  // w.mu points into per_vec
  dfree(w.v0stage);
  dfree(w.sb_dev);
  dfree(w.cr_gp);
  if (w.ev[0]) cudaEventDestroy(w.ev[0]);
  if (w.ev[1]) cudaEventDestroy(w.ev[1]);
  w = kpm_handle_s::Work{};
}

// Step arguments common to every step of a call.
StepArgs base_args(const kpm_handle_s* h, int slot, int Rp, int G) {
  StepArgs a{};
  a.n = h->n;
  a.Rp = Rp;
  a.G = G;
  a.Gt = std::min(G, BLOCK);
  a.sc = h->d_sc + slot;
  a.geom = h->geom;
  a.err = &h->d_prm->flags;
  if (h->stencil) {
    a.hs = h->has_hop ? h->d_hs[slot] : nullptr;
    a.ds = h->has_onsite ? h->d_ds[slot] : nullptr;
  } else if (h->ell_w > 0) {
    a.rowptr = nullptr;
    a.col = h->d_ell_col;
    a.vals = h->d_vals[slot];
    a.ell_w = h->ell_w;
  } else {
    a.rowptr = h->d_rowptr;
    a.col = h->d_col;
    a.vals = h->d_vals[slot];
  }
  return a;
}

cudaError_t launch_step(bool stencil, bool fp32, bool cplx, StepMode mode, const StepArgs& a,
                        const LaunchCfg& cfg, cudaStream_t st) {
  if (fp32 && stencil && mode == MODE_STEP && a.tma_stages > 0)
    return launch_stencil_tma_f32(cplx, a, cfg, st);
  return fp32 ? launch_step_f32(stencil, cplx, mode, a, cfg, st)
              : launch_step_f64(stencil, cplx, mode, a, cfg, st);
}

// One product of the handle's operator (stencil, CSR / ELL, or dense FP64).
cudaError_t launch_op(const kpm_handle_s* h, bool fp32, StepMode mode, const StepArgs& a,
                      const LaunchCfg& cfg, cudaStream_t st) {
  if (h->dense) {
    if (fp32) return cudaErrorInvalidValue;
    if (h->work.dtc && mode != MODE_SPMV) return launch_dense_tc_step(*h->work.dtc, mode, a, cfg, st);
    return launch_dense_step(h->cplx, mode, a, cfg, st);
  }
  return launch_step(h->stencil, fp32, h->cplx, mode, a, cfg, st);
}

// Traversal and grid of the fused step (see StepArgs).  Stencils with enough
// lattice lines are walked in line blocks so that the rows of one pass are
// each other's y-neighbours; CSR matrices and small or 1D lattices use the
// natural row order.  CTAs: at most (CTAs per SM x SMs), each taking chunks
// of STEP_CHUNK passes in a grid-stride loop.
#ifndef KPM_STEP_CHUNK
#define KPM_STEP_CHUNK 4   // passes per chunk; 0 = one whole lattice line
#endif

// Default of the TMA-fed ELL step: shared-memory stages, passes per tile,
// CTAs per SM (0 stages: the plain ELL step).
#ifndef ELL_TMA_STAGES
#define ELL_TMA_STAGES 2
#endif
#ifndef ELL_TMA_PASSES
#define ELL_TMA_PASSES 2
#endif
#ifndef ELL_TMA_MINB
#define ELL_TMA_MINB 2
#endif
// Default of the TMA-fed stencil step (FP32 vector blocks of at least
// STENCIL_TMA_MIN_MB megabytes; 0 stages: the plain stencil step).  Off by
// default: on the 3D L = 64 spin lattice it measured 77.8 us per step (2
// stages x 2 passes, 2 CTAs per SM) against 75.9 us for the plain step, and
// slower in every other shape tried.
#ifndef STENCIL_TMA_STAGES
#define STENCIL_TMA_STAGES 0
#endif
#ifndef STENCIL_TMA_PASSES
#define STENCIL_TMA_PASSES 2
#endif
#ifndef STENCIL_TMA_MINB
#define STENCIL_TMA_MINB 2
#endif
#ifndef STENCIL_TMA_MIN_MB
#define STENCIL_TMA_MIN_MB 16
#endif

void plan_grid(const kpm_handle_s* h, bool fp32, StepArgs& a, int* block, int* grid) {
  if (h->dense) {
    // one CTA per tile of rows (and of columns, in the launch's y dimension)
    const int bm = dense_row_tile(h->n, a.Rp, h->cplx, h->num_sms);
    a.line_len = 0;
    a.lines = 0;
    a.passes = (h->n + bm - 1) / bm;
    a.chunk = 1;
    *block = BLOCK;
    *grid = (int)a.passes;
    return;
  }
  const int G = a.Gt;            // chunks per row handled by one CTA (<= BLOCK)
  // Lattices too small to give every SM a one-pass CTA of BLOCK threads take
  // smaller CTAs (down to one warp, at least one row per pass), so that the
  // step's arithmetic spreads over more SMs: GB300's FP64 pipe (2 FMA per SM
  // and clock) otherwise makes the few busy SMs the limit of each step.
  int blk = BLOCK;
  while (blk / 2 >= std::max(32, G) && (h->n * G + blk - 1) / blk < h->num_sms) blk /= 2;
  const int spi = blk / G;
  int occ = fp32 ? occ_step_f32(h->stencil, h->cplx, a, blk)
                 : occ_step_f64(h->stencil, h->cplx, a, blk);
  occ = std::max(1, std::min(occ, 8));
  a.line_len = 0;
  a.lines = 0;
  a.line_L1 = h->geom.L[1];
  a.passes = (h->n + spi - 1) / spi;
  if (h->stencil && h->geom.dims >= 2 && h->geom.L[0] >= 4) {
    const int64_t lines = h->n / h->geom.L[0];
    const int64_t padded = (lines + spi - 1) / spi * spi;
    if (lines >= spi && 8 * (padded - lines) <= lines) {
      a.line_len = h->geom.L[0];
      a.lines = (int)lines;
      a.passes = padded / spi * (int64_t)h->geom.L[0];
    }
  }
  a.chunk = KPM_STEP_CHUNK > 0 ? KPM_STEP_CHUNK : (a.line_len > 0 ? a.line_len : 4);
  // small lattices: shorter chunks until every resident CTA has one (each
  // CTA then walks fewer dependent passes per step)
  const int64_t slots = (int64_t)h->num_sms * occ;
  while (a.chunk > 1 && (a.passes + a.chunk - 1) / a.chunk < slots) a.chunk /= 2;
  const int64_t nchunks = (a.passes + a.chunk - 1) / a.chunk;
  int64_t g = std::min<int64_t>(slots, nchunks);
  *block = blk;
  *grid = (int)std::max<int64_t>(g, 1);
  a.tma_stages = a.tma_passes = a.tma_minb = 0;
  a.tma_prefetch = -1;
  a.tma_stall = 0;
  if (!h->stencil && blk == BLOCK && ell_tma_supported(a, fp32)) {
    // the TMA-fed step (kpm_step_tma.cu): stages, passes per tile and CTAs per
    // SM and L2 prefetch distance in tiles (negative: none) from
    // KPM_ELL_TMA="stages,passes,ctas[,prefetch]" ("0" turns the form off)
    int S = ELL_TMA_STAGES, P = ELL_TMA_PASSES, B = ELL_TMA_MINB, D = -1;
    if (const char* env = getenv("KPM_ELL_TMA")) {
      int s_ = 0, p_ = P, b_ = B, d_ = -1;
      if (sscanf(env, "%d,%d,%d,%d", &s_, &p_, &b_, &d_) >= 1) {
        S = s_;
        P = p_;
        B = b_;
        D = d_;
      }
    }
    if (S > 0 && P > 0) {
      a.tma_stages = S;
      a.tma_passes = P;
      a.tma_minb = B;
      a.tma_prefetch = D;
      a.tma_stall = g_test_stall.load();
      const int occ_t = std::max(0, std::min(occ_ell_tma_f32(h->cplx, a), 8));
      const int64_t tiles = (h->n + (int64_t)(BLOCK / a.G) * P - 1) / ((int64_t)(BLOCK / a.G) * P);
      if (occ_t > 0) {
        *grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->num_sms * occ_t, tiles));
      } else {
        a.tma_stages = a.tma_passes = a.tma_minb = 0;  // does not fit: the plain step
      }
    }
  }
  // the TMA-fed stencil step (kpm_step_stencil_tma.cu) for vector blocks of
  // at least MB megabytes: stages, passes per tile, CTAs per SM and MB from
  // KPM_STENCIL_TMA="stages,passes,ctas[,MB]" ("0", the default, keeps the
  // plain step)
  int S = STENCIL_TMA_STAGES, P = STENCIL_TMA_PASSES, B = STENCIL_TMA_MINB;
  int min_mb = STENCIL_TMA_MIN_MB;
  if (const char* env = getenv("KPM_STENCIL_TMA")) {
    int s_ = 0, p_ = P, b_ = B, m_ = min_mb;
    if (sscanf(env, "%d,%d,%d,%d", &s_, &p_, &b_, &m_) >= 1) {
      S = s_;
      P = p_;
      B = b_;
      min_mb = std::max(0, m_);
    }
  }
  const size_t block_bytes = (size_t)h->n * a.G * (fp32 ? 32 : 16);
  if (h->stencil && fp32 && blk == BLOCK && block_bytes >= ((size_t)min_mb << 20) &&
      stencil_tma_supported(a, fp32)) {
    if (S > 0 && P > 0) {
      a.tma_stages = S;
      a.tma_passes = P;
      a.tma_minb = B;
      a.tma_stall = g_test_stall.load();
      const int occ_t = std::max(0, std::min(occ_stencil_tma_f32(h->cplx, a), 8));
      const int64_t rows = (int64_t)(BLOCK / a.G) * P;
      const int64_t tiles = (h->n + rows - 1) / rows;
      if (occ_t > 0) {
        *grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->num_sms * occ_t, tiles));
      } else {
        a.tma_stages = a.tma_passes = a.tma_minb = 0;
      }
    }
  }
}

kpm_status ensure_scaled(kpm_handle_s* h, int slot, bool fp32) {
  const size_t s = fp32 ? 4 : 8;
  const size_t c = h->cplx ? 2 : 1;
  if (h->stencil) {
    // + 16 bytes: the TMA-fed stencil step copies the last tile's hoppings and
    // on-site terms in whole 16-byte units
    if (h->has_hop && !h->d_hs[slot]) {
      char* p = nullptr;
      kpm_status st = dalloc(&p, (size_t)h->n * h->geom.dims * c * s + 16);
      if (st != KPM_OK) return st;
      h->d_hs[slot] = p;
    }
    if (h->has_onsite && !h->d_ds[slot]) {
      char* p = nullptr;
      kpm_status st = dalloc(&p, (size_t)h->n * s + 16);
      if (st != KPM_OK) return st;
      h->d_ds[slot] = p;
    }
  } else if (!h->d_vals[slot] && h->nnz > 0) {
    char* p = nullptr;
    const size_t entries = h->ell_w > 0 ? (size_t)h->n * h->ell_w : (size_t)h->nnz;
    // + 16 bytes: the TMA-fed ELL step copies the last tile in whole 16-byte units
    kpm_status st = dalloc(&p, entries * c * s + 16);
    if (st != KPM_OK) return st;
    h->d_vals[slot] = p;
  }
  return KPM_OK;
}

cudaError_t prescale(kpm_handle_s* h, int slot, bool fp32, bool lanczos, cudaStream_t st) {
  if (h->stencil)
    return launch_prescale_stencil(fp32, h->cplx, h->n, h->geom.dims, h->d_onsite, h->d_hop,
                                   h->t_re, h->t_im, h->d_prm, lanczos, h->d_hs[slot],
                                   h->d_ds[slot], h->d_sc + slot, st);
  if (h->ell_w > 0)
    return launch_prescale_csr(fp32, h->cplx, h->n * h->ell_w, h->d_ell_val, h->d_prm, lanczos,
                               h->d_vals[slot], h->d_sc + slot, st);
  return launch_prescale_csr(fp32, h->cplx, h->nnz, h->d_val, h->d_prm, lanczos,
                             h->d_vals[slot], h->d_sc + slot, st);
}

kpm_status common_init(kpm_handle_s* h) {
  int dev = 0;
  kpm_status st = check_device(&dev);
  if (st != KPM_OK) return st;
  h->device = dev;
  KPM_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
  kpm_status st0 = dalloc(&h->d_sc, 3);
  if (st0 == KPM_OK) st0 = dalloc(&h->d_prm, 1);
  if (st0 != KPM_OK) return st0;
  KPM_CUDA(cudaMemset(h->d_prm, 0, sizeof(RunParams)));
  KPM_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  return KPM_OK;
}

void destroy_handle(kpm_handle_s* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  free_work(h);
  dfree(h->d_onsite);
  dfree(h->d_hop);
  dfree(h->d_rowptr);
  dfree(h->d_col);
  dfree(h->d_val);
  dfree(h->d_ell_col);
  dfree(h->d_ell_val);
  for (int i = 0; i < 3; ++i) {
    dfree(h->d_hs[i]);
    dfree(h->d_ds[i]);
    dfree(h->d_vals[i]);
  }
  dfree(h->d_sc);
  dfree(h->d_prm);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  cudaStreamSynchronize(0);
  delete h;
}

// Stencil validation shared by the handle builder and the CSR converter.
kpm_status check_stencil(const kpm_stencil_desc* d, kpm_field field, int64_t* n_out) {
  if (!d) return fail(KPM_EINVAL, "desc is NULL");
  if (d->dims < 1 || d->dims > 3) return fail(KPM_EINVAL, "dims must be 1, 2 or 3");
  if (field != KPM_REAL && field != KPM_COMPLEX) return fail(KPM_EINVAL, "bad field");
  int64_t n = 1;
  for (int k = 0; k < d->dims; ++k) {
    if (d->L[k] < 1) return fail(KPM_EINVAL, "L[d] must be >= 1");
    n *= d->L[k];
    if (n >= (int64_t)1 << 31) return fail(KPM_EINVAL, "lattice too large (N must be < 2^31)");
  }
  if (field == KPM_REAL && !d->hop && d->t_im != 0.0)
    return fail(KPM_EINVAL, "complex uniform hopping with the real field");
  *n_out = n;
  return KPM_OK;
}

// Row i of the stencil matrix as (column, value) pairs, merged by column and
// sorted: H_ii = onsite_i; for each direction d the forward neighbour j gets
// -t_{i,d} and the backward neighbour j' (whose forward bond ends at i) gets
// -conj(t_{j',d}); absent bonds (open edge, mask 0) are skipped.
struct RowEnt {
  int64_t j;
  double re, im;
};
int stencil_row(const kpm_stencil_desc* d, int c, int64_t i, RowEnt* out) {
  int cnt = 0;
  auto add = [&](int64_t j, double re, double im) {
    for (int k = 0; k < cnt; ++k)
      if (out[k].j == j) { out[k].re += re; out[k].im += im; return; }
    out[cnt++] = RowEnt{j, re, im};
  };
  if (d->onsite) add(i, d->onsite[i], 0.0);
  int64_t stride = 1;
  for (int k = 0; k < d->dims; ++k) {
    const int64_t L = d->L[k];
    const int64_t x = (i / stride) % L;
    const bool per = d->periodic[k] != 0;
    const int64_t jf = x + 1 < L ? i + stride : (per ? i - (L - 1) * stride : -1);
    const int64_t jb = x > 0 ? i - stride : (per ? i + (L - 1) * stride : -1);
    auto hop = [&](int64_t site, double& re, double& im) {
      const size_t o = (size_t)site * d->dims + k;
      re = d->hop ? d->hop[o * c] : d->t_re;
      im = c == 2 ? (d->hop ? d->hop[o * c + 1] : d->t_im) : 0.0;
      return !d->bond_mask || d->bond_mask[o] != 0;
    };
    double re, im;
    if (jf >= 0 && hop(i, re, im)) add(jf, -re, -im);
    if (jb >= 0 && hop(jb, re, im)) add(jb, -re, im);
    stride *= L;
  }
  std::sort(out, out + cnt, [](const RowEnt& a, const RowEnt& b) { return a.j < b.j; });
  return cnt;
}

int64_t stencil_nnz(const kpm_stencil_desc* d, int c, int64_t n) {
  RowEnt buf[8];
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) nnz += stencil_row(d, c, i, buf);
  return nnz;
}

}  // namespace

void plan_step_grid(const kpm_handle_s* h, bool fp32, StepArgs& a, int* block, int* grid) {
  plan_grid(h, fp32, a, block, grid);
}

void operator_args(StepArgs& a, const kpm_handle_s* h, void* hs, void* ds, const ScalarBlock* sc,
                   int Rp, int G) {
  a.n = h->n;
  a.Rp = Rp;
  a.G = G;
  a.Gt = std::min(G, BLOCK);
  a.sc = sc;
  a.geom = h->geom;
  a.hs = a.ds = nullptr;
  a.rowptr = nullptr;
  a.col = nullptr;
  a.vals = nullptr;
  a.ell_w = 0;
  if (h->stencil) {
    a.hs = h->has_hop ? hs : nullptr;
    a.ds = h->has_onsite ? ds : nullptr;
  } else if (h->ell_w > 0) {
    a.col = h->d_ell_col;
    a.vals = hs;
    a.ell_w = h->ell_w;
  } else {
    a.rowptr = h->d_rowptr;
    a.col = h->d_col;
    a.vals = hs;
  }
}

void scaled_operator_bytes(const kpm_handle_s* h, bool fp32, size_t* hs_bytes, size_t* ds_bytes) {
  const size_t ssz = fp32 ? 4 : 8, c = h->cplx ? 2 : 1;
  *hs_bytes = *ds_bytes = 0;
  if (h->stencil) {
    if (h->has_hop) *hs_bytes = (size_t)h->n * h->geom.dims * c * ssz;
    if (h->has_onsite) *ds_bytes = (size_t)h->n * ssz;
  } else {
    *hs_bytes = (h->ell_w > 0 ? (size_t)h->n * h->ell_w : (size_t)h->nnz) * c * ssz;
  }
}

cudaError_t prescale_into(const kpm_handle_s* h, bool fp32, const RunParams* prm, void* hs,
                          void* ds, ScalarBlock* sc, cudaStream_t st) {
  if (h->stencil)
    return launch_prescale_stencil(fp32, h->cplx, h->n, h->geom.dims, h->d_onsite, h->d_hop,
                                   h->t_re, h->t_im, prm, false, h->has_hop ? hs : nullptr,
                                   h->has_onsite ? ds : nullptr, sc, st);
  if (h->ell_w > 0)
    return launch_prescale_csr(fp32, h->cplx, h->n * h->ell_w, h->d_ell_val, prm, false, hs, sc, st);
  return launch_prescale_csr(fp32, h->cplx, h->nnz, h->d_val, prm, false, hs, sc, st);
}

// Every col[k] in [0, n): the scan of a large matrix's column indices (22 M
// on the 3D L = 160 lattice, about 13 ms on one Grace core) split over up to
// 16 host threads.
bool columns_in_range(const int32_t* col, int64_t nnz, int64_t n) {
  auto scan = [col, n](int64_t b, int64_t e) {
    bool ok = true;
    for (int64_t k = b; k < e; ++k) ok &= (col[k] >= 0) & (col[k] < n);
    return ok;
  };
  const int64_t per = int64_t(1) << 21;
  const int nt = (int)std::min<int64_t>(
      std::max(1u, std::min(16u, std::thread::hardware_concurrency())), (nnz + per - 1) / per);
  if (nt <= 1) return scan(0, nnz);
  std::vector<char> ok(nt, 1);
  std::vector<std::thread> th;
  const int64_t chunk = (nnz + nt - 1) / nt;
  int started = 1;
  try {
    for (int t = 1; t < nt; ++t, ++started)
      th.emplace_back([&, t] {
        ok[t] = scan(t * chunk, std::min(nnz, (t + 1) * chunk)) ? 1 : 0;
      });
  } catch (...) {
    // no more threads: this thread scans what none was started for
  }
  ok[0] = scan(0, std::min(nnz, chunk)) ? 1 : 0;
  if (started < nt && !scan(started * chunk, nnz)) ok[0] = 0;
  for (auto& x : th) x.join();
  return std::all_of(ok.begin(), ok.end(), [](char c) { return c != 0; });
}
}  // namespace kpm

using namespace kpm;

extern "C" {

const char* kpm_last_error(void) { return t_err.c_str(); }

uint64_t kpm_kernel_launches(void) { return g_launches.load(); }

kpm_status kpm_testing_last_step_form(kpm_handle h, int* form) {
  if (!h || !form) return fail(KPM_EINVAL, "NULL argument");
  const auto& w = h->work;
  if (w.M == 0) return fail(KPM_ENOTREADY, "no kpm_moments call has planned its launches yet");
  if (h->dense) *form = w.dtc ? 3 : 2;
  else if (w.cr.C > 0) *form = 5;
  else *form = w.proto.tma_stages > 0 ? (h->stencil ? 4 : 1) : 0;
  return KPM_OK;
}

kpm_status kpm_testing_stall_step_pipeline(int on) {
  g_test_stall.store(on ? 1 : 0);
  return KPM_OK;
}

kpm_status kpm_testing_fail_allocations(int64_t after) {
  if (after < -1) return fail(KPM_EINVAL, "after must be >= -1");
  g_fail_alloc_after.store((long long)after);
  return KPM_OK;
}

kpm_status kpm_create_stencil(const kpm_stencil_desc* d, kpm_field field, kpm_handle* out) {
  if (!out) return fail(KPM_EINVAL, "out is NULL");
  *out = nullptr;
  int64_t n = 0;
  kpm_status st = check_stencil(d, field, &n);
  if (st != KPM_OK) return st;
  auto* h = new kpm_handle_s();
  h->stencil = true;
  h->cplx = field == KPM_COMPLEX;
  h->n = n;
  h->geom.dims = d->dims;
  int64_t stride = 1;
  for (int k = 0; k < 3; ++k) {
    h->geom.L[k] = k < d->dims ? (int)d->L[k] : 1;
    h->geom.stride[k] = (int)stride;
    h->geom.periodic[k] = k < d->dims ? (d->periodic[k] != 0) : 0;
    stride *= h->geom.L[k];
  }
  h->t_re = d->t_re;
  h->t_im = h->cplx ? d->t_im : 0.0;
  // stored entries: closed form for unmasked lattices, one host pass otherwise
  if (d->bond_mask) {
    h->nnz = stencil_nnz(d, field == KPM_COMPLEX ? 2 : 1, n);
  } else {
    int64_t nnz = 0;
    bool diag = d->onsite != nullptr;
    for (int k = 0; k < d->dims; ++k) {
      const int64_t Lk = d->L[k], lines_k = n / Lk;
      if (d->periodic[k]) {
        if (Lk == 1) diag = true;                 // self bond: on the diagonal
        else nnz += lines_k * (Lk == 2 ? 2 : 2 * Lk);
      } else {
        nnz += lines_k * 2 * (Lk - 1);
      }
    }
    h->nnz = nnz + (diag ? n : 0);
  }
  if ((st = common_init(h)) != KPM_OK) {
    destroy_handle(h);
    return st;
  }
  const int c = h->cplx ? 2 : 1;
  if (d->onsite) {
    h->has_onsite = true;
    if ((st = dalloc(&h->d_onsite, n)) != KPM_OK) { destroy_handle(h); return st; }
    cudaError_t e = cudaMemcpy(h->d_onsite, d->onsite, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { destroy_handle(h); return cuda_fail(e, "copy onsite"); }
  }
  if (d->hop && !d->bond_mask) {
    h->has_hop = true;
    const size_t cnt = (size_t)n * d->dims * c;
    if ((st = dalloc(&h->d_hop, cnt)) != KPM_OK) { destroy_handle(h); return st; }
    cudaError_t e = cudaMemcpy(h->d_hop, d->hop, cnt * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { destroy_handle(h); return cuda_fail(e, "copy hop"); }
  } else if (d->bond_mask) {
    h->has_hop = true;
    std::vector<double> hop((size_t)n * d->dims * c);
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < d->dims; ++k) {
        const size_t o = (size_t)i * d->dims + k;
        const bool keep = !d->bond_mask || d->bond_mask[o] != 0;
        for (int q = 0; q < c; ++q) {
          const double v = d->hop ? d->hop[o * c + q] : (q == 0 ? d->t_re : d->t_im);
          hop[o * c + q] = keep ? v : 0.0;
        }
      }
    if ((st = dalloc(&h->d_hop, hop.size())) != KPM_OK) { destroy_handle(h); return st; }
    cudaError_t e = cudaMemcpy(h->d_hop, hop.data(), hop.size() * sizeof(double),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { destroy_handle(h); return cuda_fail(e, "copy hop"); }
  }
  *out = h;
  return KPM_OK;
}

kpm_status kpm_create_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                          kpm_field field, kpm_handle* out) {
  if (!out) return fail(KPM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n >= ((int64_t)1 << 31)) return fail(KPM_EINVAL, "n must be in [1, 2^31)");
  if (!rowptr) return fail(KPM_EINVAL, "rowptr is NULL");
  if (field != KPM_REAL && field != KPM_COMPLEX) return fail(KPM_EINVAL, "bad field");
  if (rowptr[0] != 0) return fail(KPM_EINVAL, "rowptr[0] must be 0");
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return fail(KPM_EINVAL, "rowptr must be non-decreasing");
  const int64_t nnz = rowptr[n];
  if (nnz > 0 && (!col || !val)) return fail(KPM_EINVAL, "col/val NULL with nnz > 0");
  if (!columns_in_range(col, nnz, n)) return fail(KPM_EINVAL, "column index out of range");
  auto* h = new kpm_handle_s();
  h->stencil = false;
  h->cplx = field == KPM_COMPLEX;
  h->n = n;
  h->nnz = nnz;
  kpm_status st = common_init(h);
  if (st != KPM_OK) { destroy_handle(h); return st; }
  const int c = h->cplx ? 2 : 1;
  if ((st = dalloc(&h->d_rowptr, n + 1)) != KPM_OK ||
      (st = dalloc(&h->d_col, std::max<int64_t>(nnz, 1))) != KPM_OK ||
      (st = dalloc(&h->d_val, std::max<int64_t>(nnz * c, 1))) != KPM_OK) {
    destroy_handle(h);
    return st;
  }
  cudaError_t e = cudaMemcpy(h->d_rowptr, rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nnz)
    e = cudaMemcpy(h->d_col, col, nnz * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nnz)
    e = cudaMemcpy(h->d_val, val, nnz * c * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { destroy_handle(h); return cuda_fail(e, "copy CSR"); }
  // Short rows: keep a padded ELL copy for the fused step (fixed trip count, no
  // row-pointer indirection).  Width = longest row rounded up to even, used when
  // it is at most 8 and the padding at most doubles the stored entries.
  int64_t wmax = 0;
  for (int64_t i = 0; i < n; ++i) wmax = std::max(wmax, rowptr[i + 1] - rowptr[i]);
  const int64_t W = std::max<int64_t>(2, (wmax + 1) / 2 * 2);
  if (wmax <= 8 && n * W <= 2 * std::max<int64_t>(nnz, 1)) {
    // built on the device from the CSR arrays just copied (padding slots point
    // at the row itself with value 0); + 4 entries: the TMA-fed ELL step copies
    // the last tile in whole 16-byte units
    if ((st = dalloc(&h->d_ell_col, (size_t)n * W + 4)) != KPM_OK ||
        (st = dalloc(&h->d_ell_val, (size_t)n * W * c)) != KPM_OK) {
      destroy_handle(h);
      return st;
    }
    e = launch_ell_build(n, (int)W, h->cplx, h->d_rowptr, h->d_col, h->d_val, h->d_ell_col,
                         h->d_ell_val, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { destroy_handle(h); return cuda_fail(e, "padded-ELL build"); }
    h->ell_w = (int)W;
  }
  *out = h;
  return KPM_OK;
}

kpm_status kpm_create_dense(int64_t n, const double* H, kpm_field field, kpm_handle* out) {
  if (!out) return fail(KPM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 65536) return fail(KPM_EINVAL, "n must be in [1, 65536]");
  if (!H) return fail(KPM_EINVAL, "H is NULL");
  if (field != KPM_REAL && field != KPM_COMPLEX) return fail(KPM_EINVAL, "bad field");
  const int c = field == KPM_COMPLEX ? 2 : 1;
  // Hermitian to rounding: |H_ij - conj(H_ji)| <= 1e-12 max|H|
  double hmax = 0.0;
  for (int64_t q = 0; q < n * n * c; ++q) {
    if (!isfinite(H[q])) return fail(KPM_EINVAL, "H has a non-finite entry");
    hmax = std::max(hmax, fabs(H[q]));
  }
  const double tol = 1e-12 * hmax;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i; j < n; ++j) {
      const double* u = H + (i * n + j) * c;
      const double* v = H + (j * n + i) * c;
      const double dre = u[0] - v[0], dim = c == 2 ? u[1] + v[1] : 0.0;
      if (fabs(dre) > tol || fabs(dim) > tol)
        return fail(KPM_EINVAL, "H is not Hermitian");
    }
  auto* h = new kpm_handle_s();
  h->stencil = false;
  h->dense = true;
  h->cplx = field == KPM_COMPLEX;
  h->n = n;
  h->nnz = n * n;
  kpm_status st = common_init(h);
  if (st != KPM_OK) { destroy_handle(h); return st; }
  if ((st = dalloc(&h->d_val, (size_t)n * n * c)) != KPM_OK) {
    destroy_handle(h);
    return st;
  }
  cudaError_t e = cudaMemcpy(h->d_val, H, (size_t)n * n * c * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { destroy_handle(h); return cuda_fail(e, "copy dense H"); }
  *out = h;
  return KPM_OK;
}

kpm_status kpm_stencil_to_csr(const kpm_stencil_desc* d, kpm_field field, int64_t* nnz_out,
                              int64_t* rowptr, int32_t* col, double* val) {
  int64_t n = 0;
  kpm_status st = check_stencil(d, field, &n);
  if (st != KPM_OK) return st;
  if (!nnz_out) return fail(KPM_EINVAL, "nnz is NULL");
  const int c = field == KPM_COMPLEX ? 2 : 1;
  if (!rowptr && !col && !val) {
    *nnz_out = stencil_nnz(d, c, n);
    return KPM_OK;
  }
  if (!rowptr || !col || !val) return fail(KPM_EINVAL, "rowptr/col/val must all be given");
  RowEnt buf[8];
  int64_t k = 0;
  rowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int cnt = stencil_row(d, c, i, buf);
    for (int e = 0; e < cnt; ++e, ++k) {
      col[k] = (int32_t)buf[e].j;
      val[k * c] = buf[e].re;
      if (c == 2) val[k * c + 1] = buf[e].im;
    }
    rowptr[i + 1] = k;
  }
  *nnz_out = k;
  return KPM_OK;
}

kpm_status kpm_step_timing(kpm_handle h, double* ms, int* step_launches) {
  if (!h) return fail(KPM_EINVAL, "handle is NULL");
  if (!h->work.timed || !h->work.ev[0]) return fail(KPM_ENOTREADY, "no kpm_moments call yet");
  KPM_CUDA(cudaSetDevice(h->device));
  float t = 0.f;
  KPM_CUDA(cudaEventElapsedTime(&t, h->work.ev[0], h->work.ev[1]));
  if (ms) *ms = t;
  if (step_launches) *step_launches = h->work.M / 2;
  return KPM_OK;
}

kpm_status kpm_info(kpm_handle h, int64_t* n, int64_t* nnz, int* field, int* is_stencil) {
  if (!h) return fail(KPM_EINVAL, "handle is NULL");
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (field) *field = h->cplx ? KPM_COMPLEX : KPM_REAL;
  if (is_stencil) *is_stencil = h->stencil ? 1 : 0;
  return KPM_OK;
}

void kpm_destroy(kpm_handle h) { destroy_handle(h); }

kpm_status kpm_bounds(kpm_handle h, int lanczos_steps, double pad_eps, uint64_t seed,
                      double* emin, double* emax, double* a_out, double* b_out, void* stream) {
  if (!h) return fail(KPM_EINVAL, "handle is NULL");
  if (lanczos_steps < 0 || lanczos_steps > 256)
    return fail(KPM_EINVAL, "lanczos_steps must be in [0, 256]");
  if (!(pad_eps >= 0.0 && pad_eps < 1.0)) return fail(KPM_EINVAL, "pad_eps must be in [0, 1)");
  KPM_CUDA(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int nblk = (int)std::min<int64_t>((h->n + 255) / 256, 2 * (int64_t)h->num_sms);
  const int k = (int)std::min<int64_t>(lanczos_steps, h->n);
  const int64_t len = 2 * h->n;  // flat FP64 scalars of one Lanczos vector
  double *pmin = nullptr, *pmax = nullptr, *gersh = nullptr, *out = nullptr;
  double *Q = nullptr, *y = nullptr, *part = nullptr, *part_loc = nullptr, *coef = nullptr,
         *alpha = nullptr, *beta = nullptr;
  kpm_status st_ = KPM_OK;
  auto cleanup = [&]() {
    dfree(pmin); dfree(pmax); dfree(gersh); dfree(out); dfree(Q); dfree(y); dfree(part);
    dfree(part_loc); dfree(coef); dfree(alpha); dfree(beta);
  };
#define KPM_TRY(call)                                \
  do {                                               \
    cudaError_t e__ = (call);                        \
    if (e__ != cudaSuccess) {                        \
      cudaStreamSynchronize(st);                     \
      cleanup();                                     \
      return cuda_fail(e__, #call);                  \
    }                                                \
  } while (0)
  if ((st_ = dalloc(&pmin, nblk)) || (st_ = dalloc(&pmax, nblk)) || (st_ = dalloc(&gersh, 2)) ||
      (st_ = dalloc(&out, 8)) || (st_ = dalloc(&alpha, std::max(k, 1))) ||
      (st_ = dalloc(&beta, std::max(k, 1)))) {
    cleanup();
    return st_;
  }
  if (h->stencil)
    KPM_TRY(launch_gershgorin_stencil(h->cplx, h->n, h->geom, h->d_onsite, h->d_hop, h->t_re,
                                      h->t_im, pmin, pmax, nblk, st));
  else if (h->dense)
    KPM_TRY(launch_gershgorin_dense(h->cplx, h->n, h->d_val, pmin, pmax, nblk, st));
  else
    KPM_TRY(launch_gershgorin_csr(h->cplx, h->n, h->d_rowptr, h->d_col, h->d_val, pmin, pmax,
                                  nblk, st));
  KPM_TRY(launch_minmax_final(pmin, pmax, nblk, gersh, st));
  if (k > 0) {
    if ((st_ = dalloc(&Q, (size_t)(k + 1) * len)) || (st_ = dalloc(&y, len)) ||
        (st_ = dalloc(&part, (size_t)nblk * 2 * (k + 1))) || (st_ = dalloc(&part_loc, (size_t)nblk * 4)) ||
        (st_ = dalloc(&coef, 2 * (k + 1)))) {
      cudaStreamSynchronize(st);
      cleanup();
      return st_;
    }
    if ((st_ = ensure_scaled(h, 2, false)) != KPM_OK) {
      cudaStreamSynchronize(st);
      cleanup();
      return st_;
    }
    KPM_TRY(prescale(h, 2, false, true, st));
    int Rp, G;
    padded_width(1, false, h->cplx, &Rp, &G);
    StepArgs sa = base_args(h, 2, Rp, G);
    int block, grid;
    plan_grid(h, false, sa, &block, &grid);
    KPM_TRY(launch_lanczos_start(h->cplx, h->n, (unsigned long long)seed, Q, st));
    for (int j = 0; j < k; ++j) {
      sa.x = Q + (size_t)j * len;
      sa.y = y;
      sa.w = nullptr;
      sa.partial = nullptr;
      KPM_TRY(launch_op(h, false, MODE_SPMV, sa, LaunchCfg{block, grid}, st));
      // three-term step against q_j, q_{j-1}, then one full Gram-Schmidt pass
      KPM_TRY(launch_lz_local_dots(h->cplx, h->n, Q, len, j, y, part_loc, nblk, st));
      KPM_TRY(launch_lz_reorth_dots(h->cplx, h->n, Q, len, j, part_loc, y, part, alpha, nblk, st));
      KPM_TRY(launch_dots_final(part, nblk, j, coef, st));
      KPM_TRY(launch_lz_update_norm(h->cplx, h->n, Q, len, j, coef, y, part, nblk, st));
      KPM_TRY(launch_lanczos_next(h->n, y, part, nblk, beta, j, Q + (size_t)(j + 1) * len, st));
    }
  }
  KPM_TRY(launch_tridiag_bounds(alpha, beta, k, gersh, pad_eps, out, st));
  double host[8];
  KPM_TRY(cudaMemcpyAsync(host, out, sizeof(host), cudaMemcpyDeviceToHost, st));
  KPM_TRY(cudaStreamSynchronize(st));
#undef KPM_TRY
  cleanup();
  if (emin) *emin = host[0];
  if (emax) *emax = host[1];
  if (a_out) *a_out = host[2];
  if (b_out) *b_out = host[3];
  return KPM_OK;
}

}  // extern "C"

namespace kpm {
// The moment computation behind kpm_moments, kpm_ldos_moments and
// kpm_spectral_moments.  sb.kind != START_RANDOM replaces the random block by
// a start block built on the device (see StartBlock); with internal = true
// both outputs may be NULL (the caller reads w.per_vec itself).
// Arguments of a column-resident launch over products [n0, n1) of a
// realisation of `steps` products (vector blocks and operator of the plan).
ColresArgs colres_args(const kpm_handle_s* h, int R, int n0, int n1, int steps, bool gen) {
  const auto& w = h->work;
  ColresArgs c{};
  c.vg[0] = w.v[0];
  c.vg[1] = w.v[1];
  c.sc = w.proto.sc;
  c.hs = w.proto.hs;
  c.ds = w.proto.ds;
  c.ecol = w.proto.ell_w > 0 ? w.proto.col : nullptr;
  c.evals = w.proto.ell_w > 0 ? w.proto.vals : nullptr;
  c.geom = w.proto.geom;
  c.prm = h->d_prm;
  c.sums = w.sums;
  c.gp = w.cr_gp;
  c.n = h->n;
  c.Rp = w.Rp;
  c.R = R;
  c.P = w.cr.P;
  c.cpc = w.cr.cpc;
  c.n0 = n0;
  c.n1 = n1;
  c.steps = steps;
  c.gen = gen ? 1 : 0;
  return c;
}

// Partial scratch of the column-resident form for launches of up to nprod products.
kpm_status colres_scratch(kpm_handle_s* h, int nprod) {
  auto& w = h->work;
  const size_t need = colres_partial_doubles(w.cr, nprod);
  if (w.cr_gp_doubles >= need) return KPM_OK;
  // a launch of an earlier call may still be using the old scratch
  KPM_CUDA(cudaDeviceSynchronize());
  dfree(w.cr_gp);
  w.cr_gp = nullptr;
  w.cr_gp_doubles = 0;
  kpm_status sa = dalloc(&w.cr_gp, need);
  if (sa != KPM_OK) return sa;
  w.cr_gp_doubles = need;
  return KPM_OK;
}

kpm_status moments_impl(kpm_handle h, const kpm_params* p, double* mu, double* mu_per_vec,
                        void* stream, const StartBlock& sb, bool internal) {
  if (!h) return fail(KPM_EINVAL, "handle is NULL");
  if (!p) return fail(KPM_EINVAL, "params is NULL");
  const int M = p->M, R = p->R, S = p->S > 0 ? p->S : 1;
  if (M < 2 || (M & 1)) return fail(KPM_EINVAL, "M must be even and >= 2");
  if (R < 1) return fail(KPM_EINVAL, "R must be >= 1");
  if (!(p->a > 0.0) || !isfinite(p->a) || !isfinite(p->b))
    return fail(KPM_EINVAL, "a must be > 0 and finite, b finite");
  if (p->precision != KPM_FP64 && p->precision != KPM_FP32_VEC_FP64_MOM)
    return fail(KPM_EINVAL, "bad precision");
  if (p->user_v0 && S != 1) return fail(KPM_EINVAL, "user_v0 requires S == 1");
  if (p->s0 < 0 || (int64_t)p->s0 + S > ((int64_t)1 << 30))
    return fail(KPM_EINVAL, "s0 must be >= 0 with s0 + S <= 2^30");
  if (h->dense && p->precision != KPM_FP64)
    return fail(KPM_EINVAL, "dense handles compute in FP64 (the paper's formulation)");
  if (!mu && !mu_per_vec && !internal) return fail(KPM_EINVAL, "no output requested");
  if ((int64_t)S * R * (int64_t)M > ((int64_t)1 << 40)) return fail(KPM_EINVAL, "S*R*M too large");
  if (sb.kind != START_RANDOM && (S != 1 || p->user_v0))
    return fail(KPM_EINVAL, "a device-built start block takes S = 1 and no user_v0");
  const bool fp32 = p->precision == KPM_FP32_VEC_FP64_MOM;
  int Rp, G;
  padded_width(R, fp32, h->cplx, &Rp, &G);
  if (h->dense) {
    // the dense step tiles columns itself: pad only to whole 16-byte chunks
    const int vec = vec_per_chunk(fp32, h->cplx);
    G = (R + vec - 1) / vec;
    Rp = G * vec;
  } else if (G > 1024) {
    return fail(KPM_EINVAL, "R too large for one block of vectors");
  }
  // the arguments are valid: this call replaces any resumable state (set
  // again below once its products are enqueued)
  h->work.resumable = false;
  KPM_CUDA(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int slot = fp32 ? 1 : 0;
  const bool user_v0 = p->user_v0 != nullptr || sb.kind != START_RANDOM;
  const int steps = M / 2;
  auto& w = h->work;
  kpm_status s_ = ensure_scaled(h, slot, fp32);
  if (s_ != KPM_OK) return s_;

  const size_t sums_bytes = (size_t)S * steps * 2 * Rp * sizeof(double);
  const size_t out_bytes = ((size_t)S * R * M + M) * sizeof(double);
  const bool rebuild = w.Rp != Rp || w.prec != p->precision || w.M != M ||
                       w.user_v0 != user_v0 || !w.ready || w.sums_bytes < sums_bytes ||
                       (w.cr.C > 0 && w.cr_R != R);
  // The kernel sequence of one realisation.  The first call of a shape
  // launches it directly on the caller's stream (the solve is GPU-bound, so
  // the launches hide behind it); a second call of the same shape captures it
  // once into a CUDA graph (events recorded as external graph nodes) that
  // every later call replays.  Both forms run the same kernels in the same
  // order, so the results are identical.
  auto enqueue = [&](cudaStream_t cs, bool capture) -> cudaError_t {
    const int grid = w.nCTA;
    const LaunchCfg cfg{w.block, grid};
    auto rec = [&](cudaEvent_t ev) {
      return capture ? cudaEventRecordWithFlags(ev, cs, cudaEventRecordExternal)
                     : cudaEventRecord(ev, cs);
    };
    cudaError_t e = cudaSuccess;
    if (w.cr.C > 0) {
      // the whole realisation in one cluster launch (it draws v_0 itself)
      e = rec(w.ev[0]);
      if (e == cudaSuccess)
        e = launch_colres(fp32, h->cplx, h->geom.dims, w.cr,
                          colres_args(h, R, 0, steps, steps, !user_v0), cs);
      if (e == cudaSuccess) e = rec(w.ev[1]);
      if (e == cudaSuccess) e = launch_advance_realisation(h->d_prm, cs);
      return e;
    }
    if (!user_v0) e = launch_rng_init(fp32, h->cplx, h->n, Rp, h->d_prm, w.v[0], cs);
    StepArgs a = w.proto;
    if (e == cudaSuccess) e = rec(w.ev[0]);
    if (e == cudaSuccess) {
      a.x = w.v[0];
      a.y = w.v[1];
      a.w = nullptr;
      a.partial = w.ring;
      a.reverse = 1;  // step n sweeps backwards for even n (see StepArgs)
      e = launch_op(h, fp32, MODE_FIRST, a, cfg, cs);
    }
    if (e == cudaSuccess && steps == 1)
      e = launch_reduce_ring(w.ring, RING, 0, 1, grid, Rp, h->d_prm, steps, w.sums, cs);
    for (int n = 1; n < steps && e == cudaSuccess; ++n) {
      a.x = w.v[n & 1];
      a.y = w.v[(n + 1) & 1];
      a.w = w.v[(n + 1) & 1];
      a.partial = w.ring + (size_t)(n % RING) * grid * 2 * Rp;
      a.reverse = (n & 1) ^ 1;
      e = launch_op(h, fp32, MODE_STEP, a, cfg, cs);
      if (e != cudaSuccess) break;
      if ((n + 1) % RING == 0)
        e = launch_reduce_ring(w.ring, RING, n + 1 - RING, RING, grid, Rp, h->d_prm, steps,
                               w.sums, cs);
      else if (n == steps - 1)
        e = launch_reduce_ring(w.ring, RING, steps - steps % RING, steps % RING, grid, Rp,
                               h->d_prm, steps, w.sums, cs);
    }
    if (e == cudaSuccess) e = rec(w.ev[1]);
    if (e == cudaSuccess) e = launch_advance_realisation(h->d_prm, cs);
    return e;
  };
  if (rebuild) {
    KPM_CUDA(cudaDeviceSynchronize());
    if (w.exec) {
      cudaGraphExecDestroy(w.exec);
      w.exec = nullptr;
    }
    // buffers are about to be replaced: until the plan below is complete no
    // later call may take the old one (an allocation failing half way leaves
    // the handle to rebuild on its next call)
    w.ready = false;
    const size_t vbytes = (size_t)h->n * Rp * elem_bytes(fp32, h->cplx);
    if (w.vbytes < vbytes) {
      dfree(w.v[0]);
      dfree(w.v[1]);
      w.v[0] = w.v[1] = nullptr;
      w.vbytes = 0;
      char *v0 = nullptr, *v1 = nullptr;
      kpm_status sa = dalloc(&v0, vbytes);
      if (sa == KPM_OK) sa = dalloc(&v1, vbytes);
      if (sa != KPM_OK) {
        dfree(v0);
        return sa;
      }
      w.v[0] = v0;
      w.v[1] = v1;
      w.vbytes = vbytes;
    }
    if (w.sums_bytes < sums_bytes) {
      dfree(w.sums);
      w.sums = nullptr;
      w.sums_bytes = 0;
      kpm_status sa = dalloc((char**)&w.sums, sums_bytes);
      if (sa != KPM_OK) return sa;
      w.sums_bytes = sums_bytes;
    }
    StepArgs proto = base_args(h, slot, Rp, G);
    int block, grid;
    plan_grid(h, fp32, proto, &block, &grid);
    w.proto = proto;
    // small stencil and padded-ELL operators: the column-resident solve
    // replaces the chain of step launches (unless a TMA-fed step was planned)
    w.cr = ColresPlan{};
    w.cr_R = R;
    if (!h->dense && (h->stencil || (h->ell_w > 0 && h->nnz > 0)) && proto.tma_stages == 0 &&
        colres_plan(h->n, h->stencil ? h->geom.dims : 0, h->stencil ? 0 : h->ell_w, h->cplx, fp32,
                    R, &w.cr)) {
      kpm_status sa = colres_scratch(h, steps);
      if (sa != KPM_OK) {
        w.cr = ColresPlan{};
        return sa;
      }
    }
    if (dense_tc_wanted(h, fp32)) setup_dense_tc(h, Rp);
    else free_dense_tc(w);
    dfree(w.ring);
    w.ring = nullptr;
    {
      kpm_status sa = dalloc(&w.ring, (size_t)RING * grid * 2 * Rp);
      if (sa != KPM_OK) return sa;
    }
    w.Rp = Rp;
    w.prec = p->precision;
    w.M = M;
    w.user_v0 = user_v0;
    w.nCTA = grid;
    w.block = block;
    if (!w.ev[0]) KPM_CUDA(cudaEventCreate(&w.ev[0]));
    if (!w.ev[1]) KPM_CUDA(cudaEventCreate(&w.ev[1]));
    w.timed = false;
    w.ready = true;
    w.direct_done = false;
  }
  if (w.out_bytes < out_bytes) {
    KPM_CUDA(cudaStreamSynchronize(st));
    dfree(w.per_vec);
    w.per_vec = nullptr;
    w.mu = nullptr;
    w.out_bytes = 0;
    {
      kpm_status sa = dalloc((char**)&w.per_vec, out_bytes);
      if (sa != KPM_OK) return sa;
    }
    w.mu = w.per_vec + (size_t)S * R * M;
    w.out_bytes = out_bytes;
  }
  w.mu = w.per_vec + (size_t)S * R * M;

  // per-call parameters (pageable source: staged before the call returns)
  RunParams prm{};
  prm.a = p->a;
  prm.b = p->b;
  prm.seed = (unsigned long long)p->seed;
  prm.s = 0;
  prm.s0 = p->s0;
  prm.R = R;
  prm.S = S;
  prm.M = M;
  prm.flags = 0;
  KPM_CUDA(cudaMemcpyAsync(h->d_prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, st));
  // the operator scaled with this call's (a, b): kept from the previous call
  // on the same stream when that used the same (a, b)
  if (!(h->scaled_ok[slot] && h->scaled_a[slot] == p->a && h->scaled_b[slot] == p->b &&
        h->scaled_st[slot] == stream)) {
    h->scaled_ok[slot] = false;
    KPM_CUDA(prescale(h, slot, fp32, false, st));
    h->scaled_ok[slot] = true;
    h->scaled_a[slot] = p->a;
    h->scaled_b[slot] = p->b;
    h->scaled_st[slot] = stream;
  }
  if (w.dtc) KPM_CUDA(launch_dense_tc_slice_rows(*w.dtc, (const double*)h->d_vals[slot], st));
  if (sb.kind != START_RANDOM) {
    // the start block's parameters (site indices or wave vectors) go to the
    // device; the block itself is written there by one kernel
    const size_t pb = (size_t)sb.count * (sb.kind == START_PLANE_WAVES ? 3 : 1) * 8;
    if (w.sb_bytes < pb) {
      KPM_CUDA(cudaStreamSynchronize(st));
      dfree(w.sb_dev);
      w.sb_dev = nullptr;
      w.sb_bytes = 0;
      {
        kpm_status sa = dalloc((char**)&w.sb_dev, pb);
        if (sa != KPM_OK) return sa;
      }
      w.sb_bytes = pb;
    }
    KPM_CUDA(cudaMemcpyAsync(w.sb_dev, sb.kind == START_PLANE_WAVES ? (const void*)sb.k
                                                                    : (const void*)sb.sites,
                             pb, cudaMemcpyHostToDevice, st));
    KPM_CUDA(launch_start_block(fp32, h->cplx, sb.kind, h->n, R, Rp, w.sb_dev, h->geom,
                                w.v[0], st));
  } else if (user_v0) {
    const size_t vb = (size_t)h->n * R * (h->cplx ? 2 : 1) * sizeof(double);
    const double* src = (const double*)p->user_v0;
    if (!is_device_ptr(p->user_v0)) {
      if (w.v0stage_bytes < vb) {
        KPM_CUDA(cudaStreamSynchronize(st));
        dfree(w.v0stage);
        w.v0stage = nullptr;
        w.v0stage_bytes = 0;
        {
          kpm_status sa = dalloc((char**)&w.v0stage, vb);
          if (sa != KPM_OK) return sa;
        }
        w.v0stage_bytes = vb;
      }
      KPM_CUDA(cudaMemcpyAsync(w.v0stage, p->user_v0, vb, cudaMemcpyHostToDevice, st));
      src = w.v0stage;
    }
    KPM_CUDA(launch_load_v0(fp32, h->cplx, h->n, R, Rp, src, w.v[0], st));
  }
  if (!w.exec && w.direct_done) {
    // second call of this shape: capture the sequence once
    const uint64_t before = g_launches.load();
    KPM_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue(h->cap_stream, true);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&w.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    w.kernels_per_replay = g_launches.load() - before;
    g_launches.fetch_sub(w.kernels_per_replay);  // captured, not yet run
    if (e != cudaSuccess) {
      w.exec = nullptr;
      cudaGetLastError();
      return cuda_fail(e, "capture of the moment graph");
    }
  }
  for (int s = 0; s < S; ++s) {
    if (w.exec) {
      KPM_CUDA(cudaGraphLaunch(w.exec, st));
      g_launches.fetch_add(w.kernels_per_replay);
    } else {
      KPM_CUDA(enqueue(st, false));
    }
  }
  w.direct_done = true;
  w.timed = true;
  if (S == 1) {
    // v_{M/2-1} and v_{M/2} stay in v[] with the per-step sums: kpm_moments_extend
    // can continue this realisation
    w.resumable = true;
    w.res_steps = steps;
    w.res_R = R;
    w.res_a = p->a;
    w.res_b = p->b;
    w.res_seed = (unsigned long long)p->seed;
    w.res_s0 = p->s0;
  }
  // a device output receives the mean directly; a host output is copied
  const bool mu_dev = mu && is_device_ptr(mu);
  KPM_CUDA(launch_finalize(w.sums, S, steps, R, Rp, h->n, M, w.per_vec, mu_dev ? mu : w.mu,
                           h->d_prm, st));
  bool host_out = false;
  if (mu && !mu_dev) {
    host_out = true;
    KPM_CUDA(cudaMemcpyAsync(mu, w.mu, M * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (mu_per_vec) {
    const bool dev = is_device_ptr(mu_per_vec);
    host_out |= !dev;
    KPM_CUDA(cudaMemcpyAsync(mu_per_vec, w.per_vec, (size_t)S * R * M * sizeof(double),
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (host_out) {
    int flags = 0;
    KPM_CUDA(cudaMemcpyAsync(&flags, &h->d_prm->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    if (flags & 4)
      return fail(KPM_ETIMEOUT, "a bounded wait inside the fused step gave up (results invalid)");
    if (flags & 1)
      return fail(KPM_EDIVERGE,
                  "a moment left [-1, 1]: the bounds (a, b) do not enclose the spectrum");
  }
  return KPM_OK;
}
}  // namespace kpm

extern "C" {

kpm_status kpm_moments(kpm_handle h, const kpm_params* p, double* mu, double* mu_per_vec,
                       void* stream) {
  return moments_impl(h, p, mu, mu_per_vec, stream, StartBlock{}, false);
}

kpm_status kpm_ldos_moments(kpm_handle h, const int64_t* sites, int nsites, int M, double a,
                            double b, int precision, double* mu_loc, void* stream) {
  if (!h) return fail(KPM_EINVAL, "handle is NULL");
  if (!sites || nsites < 1) return fail(KPM_EINVAL, "need nsites >= 1 site indices");
  if (!mu_loc) return fail(KPM_EINVAL, "mu_loc is NULL");
  if (is_device_ptr(sites)) return fail(KPM_EINVAL, "sites must be a host array");
  for (int j = 0; j < nsites; ++j)
    if (sites[j] < 0 || sites[j] >= h->n) return fail(KPM_EINVAL, "site index outside [0, N)");
  kpm_params p{};
  p.M = M;
  p.R = nsites;
  p.S = 1;
  p.precision = precision;
  p.a = a;
  p.b = b;
  StartBlock sb;
  sb.kind = START_UNIT_SITES;
  sb.sites = sites;
  sb.count = nsites;
  return moments_impl(h, &p, nullptr, mu_loc, stream, sb, false);
}

kpm_status kpm_spectral_moments(kpm_handle h, const double* k, int nk, int M, double a, double b,
                                int precision, double* mu_k, void* stream) {
  if (!h) return fail(KPM_EINVAL, "handle is NULL");
  if (!h->stencil) return fail(KPM_EINVAL, "plane waves need a lattice: a stencil handle");
  if (!k || nk < 1) return fail(KPM_EINVAL, "need nk >= 1 wave vectors");
  if (!mu_k) return fail(KPM_EINVAL, "mu_k is NULL");
  if (is_device_ptr(k)) return fail(KPM_EINVAL, "k must be a host array");
  for (int j = 0; j < 3 * nk; ++j)
    if (!isfinite(k[j])) return fail(KPM_EINVAL, "non-finite wave vector component");
  // complex field: one column e^{i k.x} per wave vector; real field: the
  // columns cos(k.x) and sin(k.x), whose moments add up to those of the plane
  // wave because H~ is real symmetric
  const int per = h->cplx ? 1 : 2;
  if ((int64_t)nk * per > (1 << 20)) return fail(KPM_EINVAL, "too many wave vectors");
  kpm_params p{};
  p.M = M;
  p.R = nk * per;
  p.S = 1;
  p.precision = precision;
  p.a = a;
  p.b = b;
  StartBlock sb;
  sb.kind = START_PLANE_WAVES;
  sb.k = k;
  sb.count = nk;
  cudaStream_t st = (cudaStream_t)stream;
  if (per == 1) return moments_impl(h, &p, nullptr, mu_k, stream, sb, false);
  kpm_status r = moments_impl(h, &p, nullptr, nullptr, stream, sb, true);
  if (r != KPM_OK) return r;
  auto& w = h->work;
  const bool dev = is_device_ptr(mu_k);
  double* out = mu_k;
  if (!dev) {
    // host output: the pair sums are staged in the handle's staging buffer
    const size_t ob = (size_t)nk * M * sizeof(double);
    if (w.v0stage_bytes < ob) {
      KPM_CUDA(cudaStreamSynchronize(st));
      dfree(w.v0stage);
      w.v0stage = nullptr;
      w.v0stage_bytes = 0;
      kpm_status sa = dalloc((char**)&w.v0stage, ob);
      if (sa != KPM_OK) return sa;
      w.v0stage_bytes = ob;
    }
    out = w.v0stage;
  }
  KPM_CUDA(launch_pair_sum(w.per_vec, nk, M, out, st));
  if (!dev) {
    int flags = 0;
    KPM_CUDA(cudaMemcpyAsync(mu_k, out, (size_t)nk * M * sizeof(double), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaMemcpyAsync(&flags, &h->d_prm->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    if (flags & 4)
      return fail(KPM_ETIMEOUT, "a bounded wait inside the fused step gave up (results invalid)");
    if (flags & 1)
      return fail(KPM_EDIVERGE, "a moment left [-1, 1]: the bounds (a, b) do not enclose the spectrum");
  }
  return KPM_OK;
}

kpm_status kpm_moments_extend(kpm_handle h, int M, double* mu, double* mu_per_vec, void* stream) {
  if (!h) return fail(KPM_EINVAL, "handle is NULL");
  auto& w = h->work;
  if (!w.resumable)
    return fail(KPM_ENOTREADY,
                "no resumable state: extend follows a kpm_moments call with S = 1 on this handle");
  const int old_steps = w.res_steps;
  if (M < 2 || (M & 1)) return fail(KPM_EINVAL, "M must be even and >= 2");
  if (M / 2 <= old_steps) return fail(KPM_EINVAL, "M must exceed the moments already computed");
  if (!mu && !mu_per_vec) return fail(KPM_EINVAL, "no output requested");
  // From here on buffers change: the captured graph and launch plan of the
  // resumed call no longer match (the next kpm_moments rebuilds), and the
  // state is resumable again only once every product below is enqueued, so a
  // failure part way (an allocation, a launch) leaves nothing to resume from.
  w.ready = false;
  w.resumable = false;
  KPM_CUDA(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int steps = M / 2, Rp = w.Rp, R = w.res_R, grid = w.nCTA;
  const bool fp32 = w.prec == KPM_FP32_VEC_FP64_MOM;
  // per-step sums for the longer chain, keeping those of the steps already done
  const size_t sums_bytes = (size_t)steps * 2 * Rp * sizeof(double);
  if (w.sums_bytes < sums_bytes) {
    double* ns = nullptr;
    kpm_status sa = dalloc((char**)&ns, sums_bytes);
    if (sa != KPM_OK) return sa;
    KPM_CUDA(cudaMemcpyAsync(ns, w.sums, (size_t)old_steps * 2 * Rp * sizeof(double),
                             cudaMemcpyDeviceToDevice, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    dfree(w.sums);
    w.sums = ns;
    w.sums_bytes = sums_bytes;
  }
  const size_t out_bytes = ((size_t)R * M + M) * sizeof(double);
  if (w.out_bytes < out_bytes) {
    KPM_CUDA(cudaStreamSynchronize(st));
    dfree(w.per_vec);
    w.per_vec = nullptr;
    w.mu = nullptr;
    w.out_bytes = 0;
    kpm_status sa = dalloc((char**)&w.per_vec, out_bytes);
    if (sa != KPM_OK) return sa;
    w.out_bytes = out_bytes;
  }
  w.mu = w.per_vec + (size_t)R * M;
  // the call's parameters for realisation 0 at the new M (the scaled operator
  // of the resumed call is still in place)
  RunParams prm{};
  prm.a = w.res_a;
  prm.b = w.res_b;
  prm.seed = w.res_seed;
  prm.s = 0;
  prm.s0 = w.res_s0;
  prm.R = R;
  prm.S = 1;
  prm.M = M;
  prm.flags = 0;
  KPM_CUDA(cudaMemcpyAsync(h->d_prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, st));
  // the same step launches as the uninterrupted chain: product n reads v_n
  // from v[n & 1] and writes v_{n+1} over v_{n-1}; the ring is reduced at the
  // same step boundaries, so the sums equal those of a single call with this M
  if (w.cr.C > 0) {
    // the column-resident form continues from v_{n-1}, v_n in v[] with the
    // same per-product arithmetic and sum order
    kpm_status sa = colres_scratch(h, steps - old_steps);
    if (sa != KPM_OK) return sa;
    KPM_CUDA(launch_colres(fp32, h->cplx, h->geom.dims, w.cr,
                           colres_args(h, R, old_steps, steps, steps, false), st));
  }
  StepArgs a = w.proto;
  const LaunchCfg cfg{w.block, grid};
  for (int n = w.cr.C > 0 ? steps : old_steps; n < steps; ++n) {
    a.x = w.v[n & 1];
    a.y = w.v[(n + 1) & 1];
    a.w = w.v[(n + 1) & 1];
    a.partial = w.ring + (size_t)(n % RING) * grid * 2 * Rp;
    a.reverse = (n & 1) ^ 1;
    KPM_CUDA(launch_op(h, fp32, MODE_STEP, a, cfg, st));
    if ((n + 1) % RING == 0 || n == steps - 1) {
      const int first = std::max(old_steps, n / RING * RING);
      KPM_CUDA(launch_reduce_ring(w.ring, RING, first, n + 1 - first, grid, Rp, h->d_prm, steps,
                                  w.sums, st));
    }
  }
  KPM_CUDA(launch_finalize(w.sums, 1, steps, R, Rp, h->n, M, w.per_vec, w.mu, h->d_prm, st));
  w.res_steps = steps;
  w.resumable = true;
  bool host_out = false;
  if (mu) {
    const bool dev = is_device_ptr(mu);
    host_out |= !dev;
    KPM_CUDA(cudaMemcpyAsync(mu, w.mu, M * sizeof(double),
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (mu_per_vec) {
    const bool dev = is_device_ptr(mu_per_vec);
    host_out |= !dev;
    KPM_CUDA(cudaMemcpyAsync(mu_per_vec, w.per_vec, (size_t)R * M * sizeof(double),
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (host_out) {
    int flags = 0;
    KPM_CUDA(cudaMemcpyAsync(&flags, &h->d_prm->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    if (flags & 4)
      return fail(KPM_ETIMEOUT, "a bounded wait inside the fused step gave up (results invalid)");
    if (flags & 1)
      return fail(KPM_EDIVERGE,
                  "a moment left [-1, 1]: the bounds (a, b) do not enclose the spectrum");
  }
  return KPM_OK;
}

kpm_status kpm_dos(const double* mu, int M, double a, double b, int K, int kernel, double* E,
                   double* rho, void* stream) {
  if (kernel == KPM_KERNEL_LORENTZ) return fail(KPM_EINVAL, "the Lorentz kernel needs kpm_dos_kernel");
  return kpm_dos_kernel(mu, M, a, b, K, kernel, 0.0, E, rho, stream);
}

static kpm_status check_series(int M, double a, double b, int K, int kernel, double lambda) {
  if (M < 1 || M > (1 << 20) || K < 1 || K > (1 << 20)) return fail(KPM_EINVAL, "bad M or K");
  if (!(a > 0.0) || !isfinite(a) || !isfinite(b)) return fail(KPM_EINVAL, "bad a or b");
  if (kernel != KPM_KERNEL_JACKSON && kernel != KPM_KERNEL_NONE && kernel != KPM_KERNEL_LORENTZ)
    return fail(KPM_EINVAL, "bad kernel");
  if (kernel == KPM_KERNEL_LORENTZ && !(lambda > 0.0 && lambda < 700.0))
    return fail(KPM_EINVAL, "the Lorentz kernel needs 0 < lambda < 700");
  return KPM_OK;
}

kpm_status kpm_dos_kernel(const double* mu, int M, double a, double b, int K, int kernel,
                          double lambda, double* E, double* rho, void* stream) {
  if (!mu || !E || !rho) return fail(KPM_EINVAL, "NULL pointer");
  kpm_status s_ = check_series(M, a, b, K, kernel, lambda);
  if (s_ != KPM_OK) return s_;
  int dev = 0;
  s_ = check_device(&dev);
  if (s_ != KPM_OK) return s_;
  cudaStream_t st = (cudaStream_t)stream;
  const bool dmu = is_device_ptr(mu), dE = is_device_ptr(E), drho = is_device_ptr(rho);
  // work: coef[M] table[4K] (+ mu[M] E[K] rho[K] staging)
  const size_t nwork = (size_t)M + 4 * (size_t)K + (dmu ? 0 : M) + (dE ? 0 : K) + (drho ? 0 : K);
  double* work = nullptr;
  KPM_CUDA(cudaMallocAsync((void**)&work, nwork * sizeof(double), st));
  double* cur = work + M + 4 * (size_t)K;
  const double* mu_d = mu;
  if (!dmu) {
    KPM_CUDA(cudaMemcpyAsync(cur, mu, M * sizeof(double), cudaMemcpyHostToDevice, st));
    mu_d = cur;
    cur += M;
  }
  double* E_d = E;
  if (!dE) { E_d = cur; cur += K; }
  double* rho_d = rho;
  if (!drho) { rho_d = cur; cur += K; }
  cudaError_t e = launch_dos(mu_d, M, a, b, K, kernel, lambda, E_d, rho_d, work, st);
  if (e == cudaSuccess && !dE)
    e = cudaMemcpyAsync(E, E_d, K * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !drho)
    e = cudaMemcpyAsync(rho, rho_d, K * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(work, st);
  if (e != cudaSuccess) return cuda_fail(e, "kpm_dos_kernel");
  if (!dE || !drho) KPM_CUDA(cudaStreamSynchronize(st));
  return KPM_OK;
}

kpm_status kpm_green(const double* mu, int M, double a, double b, int K, int kernel,
                     double lambda, double* E, double* g_re, double* g_im, void* stream) {
  if (!mu || !g_re || !g_im) return fail(KPM_EINVAL, "NULL pointer");
  kpm_status s_ = check_series(M, a, b, K, kernel, lambda);
  if (s_ != KPM_OK) return s_;
  int dev = 0;
  s_ = check_device(&dev);
  if (s_ != KPM_OK) return s_;
  cudaStream_t st = (cudaStream_t)stream;
  double* outs[3] = {E, g_re, g_im};
  bool host[3];
  size_t stage = 0;
  for (int i = 0; i < 3; ++i) {
    host[i] = outs[i] && !is_device_ptr(outs[i]);
    if (host[i]) stage += K;
  }
  const bool dmu = is_device_ptr(mu);
  const size_t nwork = (size_t)M + 4 * (size_t)K + (dmu ? 0 : M) + stage;
  double* work = nullptr;
  KPM_CUDA(cudaMallocAsync((void**)&work, nwork * sizeof(double), st));
  double* cur = work + M + 4 * (size_t)K;
  const double* mu_d = mu;
  cudaError_t e = cudaSuccess;
  if (!dmu) {
    e = cudaMemcpyAsync(cur, mu, M * sizeof(double), cudaMemcpyHostToDevice, st);
    mu_d = cur;
    cur += M;
  }
  double* dst[3];
  for (int i = 0; i < 3; ++i) {
    dst[i] = outs[i];
    if (host[i]) { dst[i] = cur; cur += K; }
  }
  if (e == cudaSuccess)
    e = launch_green(mu_d, M, a, b, K, kernel, lambda, dst[0], dst[1], dst[2], work, st);
  bool any_host = false;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    if (host[i]) {
      any_host = true;
      e = cudaMemcpyAsync(outs[i], dst[i], K * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
  cudaFreeAsync(work, st);
  if (e != cudaSuccess) return cuda_fail(e, "kpm_green");
  if (any_host) KPM_CUDA(cudaStreamSynchronize(st));
  return KPM_OK;
}

kpm_status kpm_thermo(const double* mu, int M, double a, double b, int K, int kernel,
                      double lambda, const double* beta, int nT, double mu_c, double* out,
                      void* stream) {
  if (!mu || !beta || !out) return fail(KPM_EINVAL, "NULL pointer");
  if (nT < 1 || nT > 65535) return fail(KPM_EINVAL, "nT must be in 1..65535");
  if (!isfinite(mu_c)) return fail(KPM_EINVAL, "mu_c must be finite");
  kpm_status s_ = check_series(M, a, b, K, kernel, lambda);
  if (s_ != KPM_OK) return s_;
  const bool dbeta = is_device_ptr(beta);
  if (!dbeta)
    for (int t = 0; t < nT; ++t)
      if (!(beta[t] >= 0.0)) return fail(KPM_EINVAL, "beta must be >= 0 (or +inf)");
  int dev = 0;
  s_ = check_device(&dev);
  if (s_ != KPM_OK) return s_;
  cudaStream_t st = (cudaStream_t)stream;
  const bool dmu = is_device_ptr(mu), dout = is_device_ptr(out);
  // work: coef[M] table[4K] E[K] rho[K] (+ mu[M] beta[nT] out[4 nT] staging)
  const size_t nwork = (size_t)M + 6 * (size_t)K + (dmu ? 0 : M) + (dbeta ? 0 : nT) +
                       (dout ? 0 : 4 * (size_t)nT);
  double* work = nullptr;
  KPM_CUDA(cudaMallocAsync((void**)&work, nwork * sizeof(double), st));
  double* E_d = work + M + 4 * (size_t)K;
  double* rho_d = E_d + K;
  double* cur = rho_d + K;
  const double* mu_d = mu;
  const double* beta_d = beta;
  double* out_d = out;
  cudaError_t e = cudaSuccess;
  if (!dmu) {
    e = cudaMemcpyAsync(cur, mu, M * sizeof(double), cudaMemcpyHostToDevice, st);
    mu_d = cur;
    cur += M;
  }
  if (e == cudaSuccess && !dbeta) {
    e = cudaMemcpyAsync(cur, beta, nT * sizeof(double), cudaMemcpyHostToDevice, st);
    beta_d = cur;
    cur += nT;
  }
  if (!dout) { out_d = cur; cur += 4 * (size_t)nT; }
  if (e == cudaSuccess) e = launch_dos(mu_d, M, a, b, K, kernel, lambda, E_d, rho_d, work, st);
  if (e == cudaSuccess) e = launch_thermo(E_d, rho_d, K, a, beta_d, nT, mu_c, out_d, st);
  if (e == cudaSuccess && !dout)
    e = cudaMemcpyAsync(out, out_d, 4 * (size_t)nT * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(work, st);
  if (e != cudaSuccess) return cuda_fail(e, "kpm_thermo");
  if (!dout || !dmu || !dbeta) KPM_CUDA(cudaStreamSynchronize(st));
  return KPM_OK;
}

// Device-side statistics into device or host outputs (NULL: skipped); pv_d on
// the device.  Synchronises the stream when a host output was requested.
static kpm_status stats_to(const double* pv_d, int nvec, int M, double a, double b, int K,
                           int kernel, double lambda, double* mu_mean, double* mu_err, double* E,
                           double* rho_mean, double* rho_err, cudaStream_t st) {
  double* outs[5] = {mu_mean, mu_err, E, rho_mean, rho_err};
  const size_t len[5] = {(size_t)M, (size_t)M, (size_t)K, (size_t)K, (size_t)K};
  bool host[5];
  size_t stage = 0;
  for (int i = 0; i < 5; ++i) {
    host[i] = outs[i] && !is_device_ptr(outs[i]);
    if (host[i]) stage += len[i];
  }
  const size_t nwork = (size_t)M + 4 * (size_t)K + (size_t)K * nvec + stage;
  double* work = nullptr;
  KPM_CUDA(cudaMallocAsync((void**)&work, nwork * sizeof(double), st));
  double* cur = work + M + 4 * (size_t)K + (size_t)K * nvec;
  double* dst[5];
  for (int i = 0; i < 5; ++i) {
    dst[i] = outs[i];
    if (host[i]) { dst[i] = cur; cur += len[i]; }
  }
  cudaError_t e = launch_stats(pv_d, nvec, M, a, b, K, kernel, lambda, dst[0], dst[1], dst[2],
                               dst[3], dst[4], work, st);
  bool any_host = false;
  for (int i = 0; i < 5 && e == cudaSuccess; ++i)
    if (host[i]) {
      any_host = true;
      e = cudaMemcpyAsync(outs[i], dst[i], len[i] * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
  cudaFreeAsync(work, st);
  if (e != cudaSuccess) return cuda_fail(e, "kpm_stats");
  if (any_host) KPM_CUDA(cudaStreamSynchronize(st));
  return KPM_OK;
}

kpm_status kpm_stats(const double* pv, int nvec, int M, double a, double b, int K, int kernel,
                     double lambda, double* mu_mean, double* mu_err, double* E,
                     double* rho_mean, double* rho_err, void* stream) {
  if (!pv) return fail(KPM_EINVAL, "NULL pointer");
  if (nvec < 1) return fail(KPM_EINVAL, "nvec must be >= 1");
  kpm_status s_ = check_series(M, a, b, K, kernel, lambda);
  if (s_ != KPM_OK) return s_;
  if ((int64_t)nvec * K > (1LL << 28)) return fail(KPM_EINVAL, "nvec * K too large");
  int dev = 0;
  s_ = check_device(&dev);
  if (s_ != KPM_OK) return s_;
  cudaStream_t st = (cudaStream_t)stream;
  const double* pv_d = pv;
  double* pv_tmp = nullptr;
  if (!is_device_ptr(pv)) {
    KPM_CUDA(cudaMallocAsync((void**)&pv_tmp, (size_t)nvec * M * sizeof(double), st));
    KPM_CUDA(cudaMemcpyAsync(pv_tmp, pv, (size_t)nvec * M * sizeof(double),
                             cudaMemcpyHostToDevice, st));
    pv_d = pv_tmp;
  }
  s_ = stats_to(pv_d, nvec, M, a, b, K, kernel, lambda, mu_mean, mu_err, E, rho_mean, rho_err, st);
  if (pv_tmp) cudaFreeAsync(pv_tmp, st);
  return s_;
}

kpm_status kpm_moments_adaptive(kpm_handle h, const kpm_params* p, int K, int kernel,
                                double lambda, double target, int max_rounds, double* mu,
                                double* mu_err, double* E, double* rho, double* rho_err,
                                int* rounds, double* achieved, void* stream) {
  if (!h || !p) return fail(KPM_EINVAL, "NULL handle or params");
  if (p->user_v0) return fail(KPM_EINVAL, "adaptive rounds draw their own vectors (user_v0 must be NULL)");
  if (max_rounds < 1 || !(target >= 0.0)) return fail(KPM_EINVAL, "bad max_rounds or target");
  const int S = p->S > 0 ? p->S : 1, R = p->R, M = p->M;
  if (R < 1 || M < 2 || (M & 1)) return fail(KPM_EINVAL, "M must be even and >= 2, R >= 1");
  kpm_status s_ = check_series(M, p->a, p->b, K, kernel, lambda);
  if (s_ != KPM_OK) return s_;
  const int64_t per_round = (int64_t)S * R;
  if (per_round * max_rounds > (1LL << 28) / K) return fail(KPM_EINVAL, "too many vectors for K");
  KPM_CUDA(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  double* pv = nullptr;
  double* rerr_d = nullptr;
  if ((s_ = dalloc(&pv, (size_t)per_round * max_rounds * M)) != KPM_OK) return s_;
  if ((s_ = dalloc(&rerr_d, (size_t)K)) != KPM_OK) {
    dfree(pv);
    return s_;
  }
  std::vector<double> rerr((size_t)K);
  double err = INFINITY;
  int done = 0;
  for (int round = 0; round < max_rounds; ++round) {
    kpm_params q = *p;
    q.seed = p->seed + (uint64_t)round;
    s_ = kpm_moments(h, &q, nullptr, pv + (size_t)round * per_round * M, st);
    if (s_ != KPM_OK) break;
    done = round + 1;
    s_ = stats_to(pv, (int)(per_round * done), M, p->a, p->b, K, kernel, lambda, nullptr, nullptr,
                  nullptr, nullptr, rerr_d, st);
    if (s_ != KPM_OK) break;
    cudaError_t e = cudaMemcpyAsync(rerr.data(), rerr_d, K * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      s_ = cuda_fail(e, "kpm_moments_adaptive");
      break;
    }
    err = 0.0;
    for (int k = 0; k < K; ++k) err += rerr[k] * p->a * M_PI * sin(M_PI * (k + 0.5) / K) / K;
    if (err <= target) break;
  }
  if (s_ == KPM_OK)
    s_ = stats_to(pv, (int)(per_round * done), M, p->a, p->b, K, kernel, lambda, mu, mu_err, E,
                  rho, rho_err, st);
  cudaStreamSynchronize(st);
  dfree(pv);
  dfree(rerr_d);
  if (rounds) *rounds = done;
  if (achieved) *achieved = err;
  if (s_ == KPM_OK && mu && !is_device_ptr(mu)) {
    for (int n = 0; n < M; ++n)
      if (!(fabs(mu[n]) <= 1.0 + 1e-6)) return fail(KPM_EDIVERGE, "a moment left [-1, 1]");
  }
  return s_;
}

}  // extern "C"
