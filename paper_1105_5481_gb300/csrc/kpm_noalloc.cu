// kpm_moments_csr_noalloc: the FP64 moment computation of kpm_moments for a
// CSR matrix that already lives in device memory, with every piece of scratch
// (vector blocks, scaled matrix values, per-CTA partial sums, moment sums,
// per-vector moments, run parameters) carved out of one fixed, file-scope
// device array instead of allocated memory.
//
// It exists for callers that must not allocate device memory during the call:
// code that runs while a memory pool is frozen or nearly exhausted, processes
// that budget all of their device memory at start-up, and hosts (plugins,
// real-time loops) where a cudaMalloc/cudaFree would synchronise the device or
// take a lock they cannot afford.  It runs the library's generic CSR form of
// the fused step (rows walked through the row pointers), not the padded-ELL
// form that kpm_moments picks for short rows, so its moments agree with
// kpm_moments to rounding (1e-10), not bit for bit.
//
// The caller's structure arrays are device memory the library cannot inspect
// from the host, so a check kernel reads them first: it copies the row
// pointers clamped to [0, nnz] and the column indices (out-of-range ones
// replaced by 0) into the scratch, and flags any violation of the CSR rules.
// The steps read only those copies, so a malformed structure cannot send a
// load outside the caller's arrays or the vector blocks.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "kpm_internal.h"

namespace kpm {
namespace {

constexpr size_t NOALLOC_BYTES = (size_t)KPM_NOALLOC_SCRATCH_BYTES;
constexpr int NA_RING = 8;    // step slots between two cross-CTA reductions
constexpr int NA_BLOCK = 256;
constexpr int MAX_DEVICES = 64;

// The scratch.  Every device that loads this library holds it until the
// process exits.  All calls share it: a call overwrites what the previous one
// left, and two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_setup_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch on the current device (looked up once per device).
kpm_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return fail(KPM_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_ptr[dev];
  return KPM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// RunParams::flags bit set when the caller's CSR structure breaks a rule
constexpr int BAD_CSR = 2;

// Copies the structure into the scratch with every index made safe, and
// flags: rowptr[0] != 0, rowptr[n] != nnz, a decreasing or out-of-range row
// pointer, a column index outside [0, n).
__global__ void noalloc_csr_check_kernel(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                                         const int32_t* __restrict__ col, int64_t* __restrict__ rp_out,
                                         int32_t* __restrict__ col_out, RunParams* prm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  for (int64_t i = t0; i <= n; i += stride) {
    const int64_t r = rowptr[i];
    bad |= (i == 0 && r != 0) || (i == n && r != nnz) || r < 0 || r > nnz;
    if (i > 0) bad |= rowptr[i - 1] > r;
    rp_out[i] = r < 0 ? 0 : (r > nnz ? nnz : r);
  }
  for (int64_t k = t0; k < nnz; k += stride) {
    const int32_t c = col[k];
    const bool ok = c >= 0 && (int64_t)c < n;
    bad |= !ok;
    col_out[k] = ok ? c : 0;
  }
  if (bad) atomicOr(&prm->flags, BAD_CSR);
}

// Device outputs of a call whose structure was flagged become NaN.
__global__ void noalloc_poison_kernel(const RunParams* prm, double* mu, int M) {
  if (!(prm->flags & BAD_CSR)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x)
    mu[i] = __longlong_as_double(0x7ff8000000000000LL);
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace kpm

using namespace kpm;

extern "C" kpm_status kpm_moments_csr_noalloc(int64_t n, int64_t nnz, const int64_t* d_rowptr,
                                              const int32_t* d_col, const double* d_val,
                                              kpm_field field, int M, int R, uint64_t seed,
                                              double a, double b, double* mu, void* stream) {
  if (n < 1 || n >= ((int64_t)1 << 31) || nnz < 0) return fail(KPM_EINVAL, "bad n or nnz");
  if (!d_rowptr || (nnz > 0 && (!d_col || !d_val)) || !mu)
    return fail(KPM_EINVAL, "NULL pointer");
  if (field != KPM_REAL && field != KPM_COMPLEX) return fail(KPM_EINVAL, "bad field");
  if (M < 2 || (M & 1)) return fail(KPM_EINVAL, "M must be even and >= 2");
  if (R < 1) return fail(KPM_EINVAL, "R must be >= 1");
  if (!(a > 0.0) || !isfinite(a) || !isfinite(b)) return fail(KPM_EINVAL, "bad a or b");
  const bool cplx = field == KPM_COMPLEX;
  const int c = cplx ? 2 : 1;
  // FP64 vectors: 2 (real) or 1 (complex) columns per 16-byte chunk, chunks per row a power of two
  const int vec = cplx ? 1 : 2;
  int G = 1;
  while (G * vec < R) G <<= 1;
  if (G > NA_BLOCK) return fail(KPM_EINVAL, "R too large for kpm_moments_csr_noalloc");
  const int Rp = G * vec;
  const int steps = M / 2;

  int dev = 0;
  KPM_CUDA(cudaGetDevice(&dev));
  int sms = 0;
  KPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  // launch shape of the fused step (same rule as kpm_moments)
  StepArgs a0{};
  a0.n = n;
  a0.Rp = Rp;
  a0.G = G;
  a0.Gt = G;
  const int spi = NA_BLOCK / G;
  a0.passes = (n + spi - 1) / spi;  // natural row order (CSR)
  a0.chunk = 4;
  int occ = std::max(1, std::min(occ_step_f64(false, cplx, a0, NA_BLOCK), 8));
  const int64_t nchunks = (a0.passes + a0.chunk - 1) / a0.chunk;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * occ, nchunks));

  // scratch layout, checked against the fixed size before anything is launched
  size_t off = 0;
  const size_t o_prm = off; off = align256(off + sizeof(RunParams));
  const size_t o_sc = off; off = align256(off + sizeof(ScalarBlock));
  const size_t o_vals = off; off = align256(off + (size_t)std::max<int64_t>(nnz, 1) * c * 8);
  const size_t o_rp = off; off = align256(off + (size_t)(n + 1) * 8);
  const size_t o_col = off; off = align256(off + (size_t)std::max<int64_t>(nnz, 1) * 4);
  const size_t o_v0 = off; off = align256(off + (size_t)n * Rp * c * 8);
  const size_t o_v1 = off; off = align256(off + (size_t)n * Rp * c * 8);
  const size_t o_ring = off; off = align256(off + (size_t)NA_RING * grid * 2 * Rp * 8);
  const size_t o_sums = off; off = align256(off + (size_t)steps * 2 * Rp * 8);
  const size_t o_pv = off; off = align256(off + (size_t)R * M * 8);
  const size_t o_mu = off; off = align256(off + (size_t)M * 8);
  if (off > NOALLOC_BYTES)
    return fail(KPM_EINVAL, "problem needs " + std::to_string(off) + " bytes of scratch; "
                "kpm_moments_csr_noalloc is limited to KPM_NOALLOC_SCRATCH_BYTES = " +
                std::to_string(NOALLOC_BYTES));

  unsigned char* base = nullptr;
  kpm_status st_ = scratch_address(dev, &base);
  if (st_ != KPM_OK) return st_;
  cudaStream_t st = (cudaStream_t)stream;
  auto* prm = (RunParams*)(base + o_prm);
  auto* sc = (ScalarBlock*)(base + o_sc);
  auto* vals = (double*)(base + o_vals);
  auto* rp_safe = (int64_t*)(base + o_rp);
  auto* col_safe = (int32_t*)(base + o_col);
  auto* v0 = (double*)(base + o_v0);
  auto* v1 = (double*)(base + o_v1);
  auto* ring = (double*)(base + o_ring);
  auto* sums = (double*)(base + o_sums);
  auto* per_vec = (double*)(base + o_pv);
  const bool dev_out = on_device(mu);
  double* mu_dev = dev_out ? mu : (double*)(base + o_mu);

  // The parameters (realisation counter and divergence flag included) are
  // rewritten by every call; every other region is fully written by a kernel
  // before it is read, so nothing else needs clearing.
  RunParams hp{};
  hp.a = a;
  hp.b = b;
  hp.seed = (unsigned long long)seed;
  hp.R = R;
  hp.S = 1;
  hp.M = M;
  KPM_CUDA(cudaMemcpyAsync(prm, &hp, sizeof(hp), cudaMemcpyHostToDevice, st));
  {
    const int64_t work = std::max<int64_t>(n + 1, nnz);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4 * (int64_t)sms));
    noalloc_csr_check_kernel<<<blocks, 256, 0, st>>>(n, nnz, d_rowptr, d_col, rp_safe, col_safe, prm);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    KPM_CUDA(cudaGetLastError());
  }
  if (!dev_out) {
    // host output: the call synchronises anyway, so a malformed structure is
    // reported before any product is launched
    int flags = 0;
    KPM_CUDA(cudaMemcpyAsync(&flags, &prm->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    if (flags & BAD_CSR)
      return fail(KPM_EINVAL, "malformed CSR structure: rowptr[0] must be 0, rowptr non-decreasing "
                  "with rowptr[n] = nnz, and every column index in [0, n)");
  }
  KPM_CUDA(launch_prescale_csr(false, cplx, nnz, d_val, prm, false, vals, sc, st));
  KPM_CUDA(launch_rng_init(false, cplx, n, Rp, prm, v0, st));
  StepArgs sa = a0;
  sa.sc = sc;
  sa.rowptr = rp_safe;
  sa.col = col_safe;
  sa.vals = vals;
  const LaunchCfg cfg{NA_BLOCK, (int)grid};
  void* v[2] = {v0, v1};
  sa.x = v0;
  sa.y = v1;
  sa.w = nullptr;
  sa.partial = ring;
  KPM_CUDA(launch_step_f64(false, cplx, MODE_FIRST, sa, cfg, st));
  if (steps == 1) KPM_CUDA(launch_reduce_ring(ring, NA_RING, 0, 1, (int)grid, Rp, prm, steps, sums, st));
  for (int k = 1; k < steps; ++k) {
    sa.x = v[k & 1];
    sa.y = v[(k + 1) & 1];
    sa.w = v[(k + 1) & 1];
    sa.partial = ring + (size_t)(k % NA_RING) * grid * 2 * Rp;
    KPM_CUDA(launch_step_f64(false, cplx, MODE_STEP, sa, cfg, st));
    if ((k + 1) % NA_RING == 0)
      KPM_CUDA(launch_reduce_ring(ring, NA_RING, k + 1 - NA_RING, NA_RING, (int)grid, Rp, prm, steps,
                                  sums, st));
    else if (k == steps - 1)
      KPM_CUDA(launch_reduce_ring(ring, NA_RING, steps - steps % NA_RING, steps % NA_RING, (int)grid,
                                  Rp, prm, steps, sums, st));
  }
  KPM_CUDA(launch_finalize(sums, 1, steps, R, Rp, n, M, per_vec, mu_dev, prm, st));
  if (dev_out) {
    noalloc_poison_kernel<<<1, 256, 0, st>>>(prm, mu_dev, M);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    KPM_CUDA(cudaGetLastError());
  } else {
    int flags = 0;
    KPM_CUDA(cudaMemcpyAsync(mu, mu_dev, (size_t)M * 8, cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaMemcpyAsync(&flags, &prm->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    if (flags & 1)
      return fail(KPM_EDIVERGE, "a moment left [-1, 1]: the bounds (a, b) do not enclose the spectrum");
  }
  return KPM_OK;
}
