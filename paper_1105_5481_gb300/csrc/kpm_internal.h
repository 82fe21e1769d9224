// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "kpm.h"
#include "kpm_args.h"

namespace kpm {

// ----------------------------------------------------------------- errors
void set_error(const std::string& msg);
kpm_status fail(kpm_status st, const std::string& msg);
kpm_status cuda_fail(cudaError_t e, const char* what);
extern std::atomic<uint64_t> g_launches;

#define KPM_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return ::kpm::cuda_fail(e__, #call); \
  } while (0)

// is_stencil, fp32, complex -> launches one fused step.
cudaError_t launch_step_f32(bool stencil, bool cplx, StepMode mode, const StepArgs& a,
                            const LaunchCfg& cfg, cudaStream_t st);
cudaError_t launch_step_f64(bool stencil, bool cplx, StepMode mode, const StepArgs& a,
                            const LaunchCfg& cfg, cudaStream_t st);
// TMA-fed padded-ELL step (kpm_step_tma.cu): whether `a` admits it, its
// launch (cfg.grid CTAs of its own size) and its CTAs per SM
bool ell_tma_supported(const StepArgs& a, bool fp32);
cudaError_t launch_ell_tma_f32(bool cplx, const StepArgs& a, const LaunchCfg& cfg, cudaStream_t st);
int occ_ell_tma_f32(bool cplx, const StepArgs& a);
// TMA-fed stencil step (FP32 vectors, 2D/3D stencils; kpm_step_stencil_tma.cu):
// tma_stages, tma_passes, tma_minb and tma_stall of StepArgs as for the ELL form
bool stencil_tma_supported(const StepArgs& a, bool fp32);
cudaError_t launch_stencil_tma_f32(bool cplx, const StepArgs& a, const LaunchCfg& cfg,
                                   cudaStream_t st);
int occ_stencil_tma_f32(bool cplx, const StepArgs& a);
// occupancy-derived CTAs per SM of the step variant selected by `a`
int occ_step_f32(bool stencil, bool cplx, const StepArgs& a, int block);
int occ_step_f64(bool stencil, bool cplx, const StepArgs& a, int block);

// Launch shape of the column-resident solve (kpm_colres.h): C = 0 when the
// form does not apply.
struct ColresPlan {
  int C = 0;        // CTAs per cluster
  int cpc = 0;      // vector columns per cluster (a power of two <= 32)
  int groups = 0;   // clusters: ceil(R / cpc)
  int block = 0;    // threads per CTA
  int64_t P = 0;    // rows per CTA: ceil(N / C)
  size_t smem = 0;  // dynamic shared memory per CTA
  int ell_w = 0;    // 0: stencil operator; > 0: padded-ELL operator of this width
};

// Dense products on the bf16 tensor cores by the Ozaki splitting scheme
// (kpm_dense_tc.cu), real FP64 dense handles: slices of S (per call) and of
// the current vector block (per step), the exact slice products, exponents.
struct DenseTC {
  int64_t n = 0;
  int Rp = 0, beta = 0, k = 0;
  void* blas = nullptr;             // cublasHandle_t
  void* workspace = nullptr;        // the cuBLAS workspace (no allocation during capture)
  size_t ws_bytes = 0;
  uint16_t* A = nullptr;            // bf16 [k][n][n]
  uint16_t* B = nullptr;            // bf16 [k][n][Rp]
  float* C = nullptr;               // k(k+1)/2 blocks of n x Rp
  double* row_scale = nullptr;      // [n]: 2^(e_i - beta (k + 1))
  double* col_scale = nullptr;      // [Rp]: 2^(f_j)
  unsigned long long* cmax = nullptr;  // [Rp]
};
void dense_tc_split(int64_t n, int* beta, int* k);
size_t dense_tc_c_floats(int64_t n, int Rp, int k);
cudaError_t launch_dense_tc_slice_rows(const DenseTC& d, const double* S, cudaStream_t st);
cudaError_t launch_dense_tc_step(const DenseTC& d, StepMode mode, const StepArgs& a,
                                 const LaunchCfg& cfg, cudaStream_t st);
cudaError_t dense_tc_create_blas(DenseTC& d);
void dense_tc_destroy_blas(DenseTC& d);
// dense operators (kpm_dense.cu): FP64 only
cudaError_t launch_dense_step(bool cplx, StepMode mode, const StepArgs& a, const LaunchCfg& cfg,
                              cudaStream_t st);
cudaError_t launch_gershgorin_dense(bool cplx, int64_t n, const double* H, double* part_min,
                                    double* part_max, int nblk, cudaStream_t st);
// rows per CTA of the dense step (64, or 16 when 64-row tiles would leave SMs idle)
int dense_row_tile(int64_t n, int Rp, bool cplx, int num_sms);

// auxiliary kernels (kpm_aux.cu)
cudaError_t launch_prescale_stencil(bool fp32, bool cplx, int64_t n, int dims, const double* onsite,
                                    const double* hop, double t_re, double t_im,
                                    const RunParams* prm, bool lanczos, void* hs, void* ds,
                                    ScalarBlock* sc, cudaStream_t st);
// Padded-ELL copy (width W) of a device CSR matrix (kpm_aux.cu).
cudaError_t launch_ell_build(int64_t n, int W, bool cplx, const int64_t* rowptr, const int32_t* col,
                             const double* val, int32_t* ecol, double* eval, cudaStream_t st);
cudaError_t launch_prescale_csr(bool fp32, bool cplx, int64_t nnz, const double* val,
                                const RunParams* prm, bool lanczos, void* vals, ScalarBlock* sc,
                                cudaStream_t st);
cudaError_t launch_rng_init(bool fp32, bool cplx, int64_t n, int Rp, const RunParams* prm, void* v0,
                            cudaStream_t st);
cudaError_t launch_load_v0(bool fp32, bool cplx, int64_t n, int R, int Rp, const double* src,
                           void* v0, cudaStream_t st);
// Start blocks built on the device (local and momentum-resolved moments).
enum StartKind { START_RANDOM = 0, START_UNIT_SITES = 1, START_PLANE_WAVES = 2 };
struct StartBlock {
  int kind = START_RANDOM;
  const int64_t* sites = nullptr;  // host, START_UNIT_SITES: column j = sqrt(N) e_{sites[j]}
  const double* k = nullptr;       // host, START_PLANE_WAVES: k[3j..3j+2], column(s) of e^{i k.x}
  int count = 0;
};
// params: int64 site indices (unit sites) or FP64 [count][3] wave vectors
cudaError_t launch_start_block(bool fp32, bool cplx, int kind, int64_t n, int R, int Rp,
                               const void* params, const StencilGeom& g, void* v0, cudaStream_t st);
// out[j*M + n] = pv[(2j)*M + n] + pv[(2j+1)*M + n], j < npairs
cudaError_t launch_pair_sum(const double* pv, int npairs, int M, double* out, cudaStream_t st);
cudaError_t launch_reduce_ring(const double* ring, int ring_slots, int first_step, int count,
                               int nCTA, int Rp, const RunParams* prm, int steps_per_real,
                               double* sums, cudaStream_t st);
cudaError_t launch_advance_realisation(RunParams* prm, cudaStream_t st);
cudaError_t launch_finalize(const double* sums, int S, int steps, int R, int Rp, int64_t n, int M,
                            double* per_vec, double* mu, RunParams* prm, cudaStream_t st);
cudaError_t launch_gershgorin_stencil(bool cplx, int64_t n, const StencilGeom& g,
                                      const double* onsite, const double* hop, double t_re,
                                      double t_im, double* part_min, double* part_max, int nblk,
                                      cudaStream_t st);
cudaError_t launch_gershgorin_csr(bool cplx, int64_t n, const int64_t* rowptr, const int32_t* col,
                                  const double* val, double* part_min, double* part_max, int nblk,
                                  cudaStream_t st);
cudaError_t launch_minmax_final(const double* part_min, const double* part_max, int nblk,
                                double* out2, cudaStream_t st);
// Lanczos helpers (FP64; vectors are flat arrays of 2N doubles: real values
// with a zero pad column, or interleaved complex pairs)
cudaError_t launch_lanczos_start(bool cplx, int64_t n, unsigned long long seed, double* q,
                                 cudaStream_t st);
cudaError_t launch_lz_local_dots(bool cplx, int64_t n, const double* Q, int64_t ldq, int j,
                                const double* y, double* part_loc, int nblk, cudaStream_t st);
cudaError_t launch_lz_reorth_dots(bool cplx, int64_t n, const double* Q, int64_t ldq, int j,
                                  const double* part_loc, double* y, double* part, double* alpha,
                                  int nblk, cudaStream_t st);
cudaError_t launch_dots_final(const double* part, int nblk, int j, double* out, cudaStream_t st);
cudaError_t launch_lz_update_norm(bool cplx, int64_t n, const double* Q, int64_t ldq, int j,
                                  const double* coef, double* y, double* part, int nblk,
                                  cudaStream_t st);
cudaError_t launch_lanczos_next(int64_t n, const double* y, const double* part, int nblk,
                                double* beta, int j, double* qnext, cudaStream_t st);
cudaError_t launch_tridiag_bounds(const double* alpha, const double* beta, int m,
                                  const double* gersh, double pad_eps, double* out,
                                  cudaStream_t st);
cudaError_t launch_dos(const double* mu, int M, double a, double b, int K, int kernel,
                       double lambda, double* E, double* rho, double* work, cudaStream_t st);
// Fermi-occupation integrals (n, u, s, c per site) of a DOS on the K nodes
cudaError_t launch_thermo(const double* E, const double* rho, int K, double a,
                          const double* beta, int nT, double mu_c, double* out, cudaStream_t st);
// local Green's function on the K nodes (work holds M + 4K doubles)
cudaError_t launch_green(const double* mu, int M, double a, double b, int K, int kernel,
                         double lambda, double* E, double* g_re, double* g_im, double* work,
                         cudaStream_t st);
// mean and standard error over nvec vectors (pv[r*M + n]) of the moments and
// of the per-vector DOS; any output may be NULL; work holds M + 4K + K*nvec doubles
cudaError_t launch_stats(const double* pv, int nvec, int M, double a, double b, int K, int kernel,
                         double lambda, double* mu_mean, double* mu_err, double* E, double* rmean,
                         double* rerr, double* work, cudaStream_t st);

// Vector columns per chunk and chunk rounding of R (shared by all entry points).
int vec_per_chunk(bool fp32, bool cplx);
void padded_width(int R, bool fp32, bool cplx, int* Rp, int* G);
size_t elem_bytes(bool fp32, bool cplx);

}  // namespace kpm

struct kpm_handle_s;
namespace kpm {
kpm_status moments_impl(kpm_handle_s* h, const kpm_params* p, double* mu, double* mu_per_vec,
                        void* stream, const StartBlock& sb, bool internal);
// Fills the operator part of a step's arguments from a handle and scaled
// operator arrays (stencil: hs, ds; CSR/ELL: vals in hs).
void operator_args(StepArgs& a, const kpm_handle_s* h, void* hs, void* ds, const ScalarBlock* sc,
                   int Rp, int G);
// Traversal and grid of the single-instance fused step (fills a.line_len,
// a.lines, a.line_L1, a.passes, a.chunk).
void plan_step_grid(const kpm_handle_s* h, bool fp32, StepArgs& a, int* block, int* grid);
// Bytes of the scaled operator arrays of a handle at one precision.
void scaled_operator_bytes(const kpm_handle_s* h, bool fp32, size_t* hs_bytes, size_t* ds_bytes);
cudaError_t prescale_into(const kpm_handle_s* h, bool fp32, const RunParams* prm, void* hs,
                          void* ds, ScalarBlock* sc, cudaStream_t st);
// Batched persistent kernel (kpm_batch_f32.cu / kpm_batch_f64.cu)
struct BatchTask;
cudaError_t launch_batch_f32(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                             int* queue, int grid, int C, cudaStream_t st);
cudaError_t launch_batch_f64(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                             int* queue, int grid, int C, cudaStream_t st);
int max_clusters_batch_f32(bool cplx, const StepArgs& proto, int C);
int max_clusters_batch_f64(bool cplx, const StepArgs& proto, int C);
// 16-byte chunks of a real FP32 block (twice the threads per row; stencil operators)
cudaError_t launch_batch_f32h(const StepArgs& proto, BatchTask* tasks, int ntasks, int* queue,
                              int grid, int C, cudaStream_t st);
int max_clusters_batch_f32h(const StepArgs& proto, int C);
// Cluster-resident form (vector rows in the clusters' shared memory, at most
// rows_cap rows per CTA; stencil operators only)
cudaError_t launch_batch_res_f32(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                                 int* queue, int grid, int C, int64_t rows_cap, cudaStream_t st);
cudaError_t launch_batch_res_f64(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                                 int* queue, int grid, int C, int64_t rows_cap, cudaStream_t st);
int max_clusters_batch_res_f32(bool cplx, const StepArgs& proto, int C, int64_t rows_cap);
int max_clusters_batch_res_f64(bool cplx, const StepArgs& proto, int C, int64_t rows_cap);
// Staged form (vector tiles copied into shared-memory rings by a producer
// warp: tiles of 2^Tl rows, 2^Sl stages of v_n, 2^SWl of v_{n-1}; stencil
// operators, untiled tasks)
cudaError_t launch_batch_stg_f32(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                                 int* queue, int grid, int C, int Tl, int Sl, int SWl,
                                 cudaStream_t st);
cudaError_t launch_batch_stg_f64(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                                 int* queue, int grid, int C, int Tl, int Sl, int SWl,
                                 cudaStream_t st);
int max_clusters_batch_stg_f32(bool cplx, const StepArgs& proto, int C, int Tl, int Sl, int SWl);
int max_clusters_batch_stg_f64(bool cplx, const StepArgs& proto, int C, int Tl, int Sl, int SWl);
}  // namespace kpm

// The handle (opaque to callers).
struct kpm_handle_s {
  int device = 0;
  bool cplx = false;
  bool stencil = false;
  bool dense = false;  // dense n x n matrix in d_val (nnz = n*n), no rowptr / col
  int64_t n = 0;
  int64_t nnz = 0;
  // stencil
  kpm::StencilGeom geom{};
  bool has_onsite = false, has_hop = false;
  double t_re = 1.0, t_im = 0.0;
  double* d_onsite = nullptr;   // FP64 raw
  double* d_hop = nullptr;      // FP64 raw (masked bonds zeroed)
  // CSR
  int64_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_val = nullptr;      // FP64 raw
  // padded ELL copy used by the fused step when rows are short (ell_w > 0)
  int ell_w = 0;
  int32_t* d_ell_col = nullptr;
  double* d_ell_val = nullptr;  // FP64 raw, [n][ell_w] (x2 complex)
  // scaled operator copies: [0] = KPM FP64, [1] = KPM FP32, [2] = Lanczos FP64
  void* d_hs[3] = {nullptr, nullptr, nullptr};
  void* d_ds[3] = {nullptr, nullptr, nullptr};
  void* d_vals[3] = {nullptr, nullptr, nullptr};
  kpm::ScalarBlock* d_sc = nullptr;  // [3]
  // the (a, b) and stream that slots 0 and 1 were last scaled with on the
  // device (kpm_moments skips the rescale while a call repeats them)
  bool scaled_ok[2] = {false, false};
  double scaled_a[2] = {0.0, 0.0}, scaled_b[2] = {0.0, 0.0};
  void* scaled_st[2] = {nullptr, nullptr};
  kpm::RunParams* d_prm = nullptr;
  // moments workspace
  struct Work {
    int Rp = 0, prec = -1, M = 0, nCTA = 0, block = 0;
    bool user_v0 = false;
    void* v[2] = {nullptr, nullptr};
    size_t vbytes = 0;
    double* ring = nullptr;
    double* sums = nullptr;
    size_t sums_bytes = 0;
    double* per_vec = nullptr;
    double* mu = nullptr;
    size_t out_bytes = 0;
    double* v0stage = nullptr;
    size_t v0stage_bytes = 0;
    void* sb_dev = nullptr;   // parameters of a device-built start block
    size_t sb_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels_per_replay = 0;
    bool ready = false;        // buffers and launch plan match the current shape
    bool direct_done = false;  // one call of this shape ran without a graph
    kpm::StepArgs proto{};                    // launch arguments common to all steps
    // the dense product on the tensor cores (real FP64 dense handles)
    kpm::DenseTC* dtc = nullptr;
    // resumable state of the last kpm_moments call (S == 1): v_{n-1}, v_n in
    // v[], the per-step sums of its steps, and its parameters
    bool resumable = false;
    int res_steps = 0, res_R = 0, res_s0 = 0;
    double res_a = 0.0, res_b = 0.0;
    unsigned long long res_seed = 0;
    // column-resident solve (kpm_colres.cu) in place of the step chain when
    // cr.C > 0: its plan, the column count it was made for, and the scratch
    // of its CTA partials
    kpm::ColresPlan cr{};
    int cr_R = 0;
    double* cr_gp = nullptr;
    size_t cr_gp_doubles = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};  // recorded around the step chain in the graph
    bool timed = false;
  } work;
  cudaStream_t cap_stream = nullptr;
  int num_sms = 0;
};
