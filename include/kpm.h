/*
 * kpm.h - C ABI of the GB300-native kernel polynomial method (KPM) library.
 *
 * The library computes the density of states (DOS) of a sparse Hermitian
 * lattice Hamiltonian H with the kernel polynomial method of Zhang, Yamagiwa,
 * Okumura and Yunoki, "Performance Acceleration of Kernel Polynomial Method
 * Applying Graphics Processing Units" (arXiv:1105.5481), Sec. II-A:
 *
 *   H~ = (H - b) / a                                   Eq. (tilde)
 *   v_0 = r,  v_1 = H~ v_0,  v_{n+1} = 2 H~ v_n - v_{n-1}   Eq. (rn)
 *   mu_n ~ << (1/(N R)) sum_r <r|T_n(H~)|r> >>          Eq. (munr), stochastic trace
 *   f(x) = [g_0 mu_0 + 2 sum_{n=1}^{M-1} g_n mu_n T_n(x)] / (pi sqrt(1-x^2))   Eq. (fKPM)
 *
 * with the moments gathered two per matrix product by the doubling identities
 * mu_{2n} = 2<v_n|v_n> - mu_0 and mu_{2n+1} = 2<v_{n+1}|v_n> - mu_1 and the
 * Jackson kernel g_n (the paper names both through its KPM reference).
 *
 * Notation: N = matrix dimension (the paper's D or H_SIZE), M = number of
 * moments (the paper's N), R = random vectors per realisation, S = number of
 * realisations (Sec. II-A-4).
 *
 * Conventions for every entry point:
 *  - Every call returns a kpm_status; nothing aborts.  On failure the calling
 *    thread's message is available from kpm_last_error().
 *  - Host input arrays are copied; the caller keeps ownership.  Output arrays
 *    are caller-owned and may be host or device pointers (the library tells
 *    them apart with cudaPointerGetAttributes).
 *  - Device memory for the Hamiltonian and the vector blocks is owned by the
 *    handle and released by kpm_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls that write host outputs synchronise that stream before returning;
 *    calls whose outputs are all device pointers are asynchronous.
 *  - All compute runs in the library's CUDA kernels on the device that was
 *    current when the handle was created; there is no CPU fallback.  A call on
 *    a machine without a usable CUDA device returns KPM_ECUDA.
 */
#ifndef KPM_H
#define KPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kpm_handle_s* kpm_handle;

typedef enum {
  KPM_OK = 0,
  KPM_EINVAL = 1,    /* invalid argument (sizes, pointers, CSR structure, M odd ...) */
  KPM_ENOMEM = 2,    /* device allocation failed or budget exceeded */
  KPM_ECUDA = 3,     /* CUDA runtime error (message in kpm_last_error) */
  KPM_ETIMEOUT = 4,  /* a bounded device wait gave up */
  KPM_EDIVERGE = 5,  /* some |mu_n^r| > 1 + 1e-6 or non-finite: bounds do not
                        enclose the spectrum.  Outputs are still written. */
  KPM_EBUSY = 6,
  KPM_ENOTREADY = 7
} kpm_status;

typedef enum { KPM_REAL = 0, KPM_COMPLEX = 1 } kpm_field;

typedef enum {
  KPM_FP64 = 0,               /* vectors, products and moment sums in FP64 */
  KPM_FP32_VEC_FP64_MOM = 1   /* vectors stored/streamed and products in FP32;
                                 moment dot products summed in FP64 from short
                                 FP32 partial sums; bounds and DOS in FP64 */
} kpm_precision;

typedef enum { KPM_KERNEL_JACKSON = 0, KPM_KERNEL_NONE = 1, KPM_KERNEL_LORENTZ = 2 } kpm_kernel;

/*
 * Lattice stencil description (matrix-free Hamiltonian; the paper's
 * evaluation lattice, Sec. IV-A, is dims=3, L={10,10,10}, periodic, t=1).
 *
 * Sites are numbered i = x0 + L[0]*(x1 + L[1]*x2).  Direction d joins site i
 * to its forward neighbour x_d+1 (wrapping when periodic[d] != 0, no bond at
 * the open edge otherwise).  The matrix is
 *     H_ii = onsite[i],   H_{i,i+e_d} += -t_{i,d},   H_{i+e_d,i} += -conj(t_{i,d}),
 * repeated pairs adding up (L[d] = 1 or 2 with wrap).
 *   onsite     [N] FP64, NULL => 0.
 *   hop        forward-bond hoppings t_{i,d}, layout [N][dims] (real field) or
 *              [N][dims][2] (re, im) (complex field); NULL => uniform t.
 *   t_re, t_im uniform hopping used when hop == NULL (t_im must be 0 for the
 *              real field).
 *   bond_mask  [N][dims] bytes, NULL => all bonds kept; 0 removes the bond.
 */
typedef struct {
  int dims;            /* 1, 2 or 3 */
  int64_t L[3];        /* extents, L[d] >= 1; entries beyond dims are ignored */
  int periodic[3];     /* per-dimension wrap flag */
  const double* onsite;
  const double* hop;
  double t_re, t_im;
  const uint8_t* bond_mask;
} kpm_stencil_desc;

/* Builds a matrix-free stencil Hamiltonian (Sec. IV-A lattice model) on the
 * current device.  Host arrays are copied.  N = prod L[d] must be < 2^31.
 * Returns KPM_EINVAL for dims outside 1..3, L[d] < 1, a complex t with the
 * real field, or N too large. */
kpm_status kpm_create_stencil(const kpm_stencil_desc* desc, kpm_field field, kpm_handle* out);

/* Builds a CSR Hamiltonian (the paper's CRS format, Sec. II-A-4) from host
 * arrays: rowptr[n+1] (rowptr[0] = 0, non-decreasing, rowptr[n] = nnz),
 * col[nnz] in [0, n), val[nnz] FP64 (real field) or [nnz][2] (re, im)
 * (complex field).  H must be Hermitian (not checked); duplicate entries add.
 * Returns KPM_EINVAL on a malformed structure. */
kpm_status kpm_create_csr(int64_t n, const int64_t* rowptr, const int32_t* col,
                          const double* val, kpm_field field, kpm_handle* out);

/* Builds a dense Hamiltonian: the paper's own formulation (Sec. II-A-4 with
 * CRS not applied, Sec. III), in which every element of H~ takes part in
 * every product.  H is a host array of n*n FP64 values, row-major (real
 * field) or n*n (re, im) pairs (complex field), copied to the device; it must
 * be Hermitian to rounding (|H_ij - conj(H_ji)| <= 1e-12 max|H|).  Dense
 * handles compute in FP64 (kpm_moments with KPM_FP64; KPM_FP32_VEC_FP64_MOM
 * returns KPM_EINVAL) and work with kpm_bounds, kpm_moments and the calls
 * built on them, not with the batch or the server.  For real dense handles
 * with n >= 512 the product runs on the bf16 tensor cores by the Ozaki
 * splitting scheme (beta-bit integer slices of H~ and of the vector block,
 * exact FP32 slice products, recombination in FP64; FP64-accurate results);
 * complex and smaller handles use the FP64 pipe.  The environment variable
 * KPM_DENSE_TENSOR=0 or =1, read when a call plans its launches, forces
 * either form.  kpm_info reports nnz = n*n and is_stencil = 0.  Returns
 * KPM_EINVAL for n outside [1, 65536], a NULL H, a non-finite entry or a
 * non-Hermitian H. */
kpm_status kpm_create_dense(int64_t n, const double* H, kpm_field field, kpm_handle* out);

/* Converts a stencil description into CSR arrays on the host (library-side
 * builder; rows sorted by column, duplicates summed, zero-valued bonds from the
 * mask dropped, diagonal stored only where onsite != NULL).  Call once with
 * rowptr/col/val NULL to obtain *nnz, then again with rowptr[N+1], col[nnz],
 * val[nnz] (or [nnz][2] complex) allocated by the caller. */
kpm_status kpm_stencil_to_csr(const kpm_stencil_desc* desc, kpm_field field, int64_t* nnz,
                              int64_t* rowptr, int32_t* col, double* val);

/* Spectral bounds (Eq. (tilde) and the text below it): the Gershgorin
 * enclosure [min_i(H_ii - sum_j|H_ij|), max_i(H_ii + sum_j|H_ij|)], tightened
 * by a lanczos_steps-step FP64 Lanczos run with full reorthogonalisation from
 * a Rademacher start vector drawn from (seed, stream 6): the extreme Ritz
 * values widened by their residuals beta_k |s_k|, clamped to the Gershgorin
 * enclosure (lanczos_steps = 0 gives Gershgorin alone).  Outputs (host
 * pointers, any may be NULL): emin, emax, and the rescaling
 *     a = (emax - emin) / (2 - pad_eps),  b = (emax + emin) / 2,
 * pad_eps in [0, 1) (0 reproduces the paper's unpadded scaling).  Runs on
 * `stream` and synchronises it. */
kpm_status kpm_bounds(kpm_handle h, int lanczos_steps, double pad_eps, uint64_t seed,
                      double* emin, double* emax, double* a, double* b, void* stream);

typedef struct {
  int M;                  /* number of moments, even, >= 2 */
  int R;                  /* random vectors per realisation, >= 1 */
  int S;                  /* realisations, >= 1 (0 is read as 1) */
  uint64_t seed;          /* random vectors: entry (s, r, i) from (seed, stream 0,
                             counter ((s0 + s)*R + r)*N + i): Rademacher +-1 (real
                             field) or exp(2 pi i u) (complex field) */
  int precision;          /* kpm_precision */
  double a, b;            /* H~ = (H - b)/a, a > 0; never chosen implicitly */
  const void* user_v0;    /* NULL, or an N x R start block (row-major, R
                             contiguous; FP64 or interleaved complex FP64), host
                             or device; requires S == 1.  The estimator uses the
                             paper's 1/(N R) normalisation, so the full basis is
                             sqrt(N) times the identity. */
  int s0;                 /* first realisation: realisation s of this call draws
                             its vectors as realisation s0 + s of the seed's
                             sequence (counter ((s0 + s)*R + r)*N + i), so
                             processes that run s0 = 0, 1, ... of one seed split
                             one run of S realisations (Sec. II-A-4) between
                             them.  >= 0, s0 + S <= 2^30; 0 for one process.
                             Batches and the server take s0 = 0. */
} kpm_params;

/* Chebyshev moments mu[0..M) (Eqs. (rn), (munr), doubling form), averaged over
 * the S*R vectors, and optionally the per-vector moments
 * mu_per_vec[(s*R + r)*M + n] (NULL to skip).  One fused CUDA kernel per
 * matrix product (v_{n+1} = 2 H~ v_n - v_{n-1} plus the two moment dots),
 * replayed from a captured CUDA graph.  A stencil operator, or a CSR operator
 * with a padded-ELL copy (rows of at most 8 entries), small enough that one
 * cluster of at most 16 CTAs holds one column's two vectors in shared memory
 * with one element per thread (and every column group fits the GPU at once)
 * instead runs all M/2 products of a realisation in one launch of
 * independent clusters, one per group of columns, when the planner's
 * estimate says that is faster (the column-resident solve; KPM_COLRES=0 in
 * the environment keeps the chain).  Returns KPM_EDIVERGE (after writing
 * the outputs) when host outputs show |mu_n^r| > 1 + 1e-6 or a non-finite
 * value, and KPM_EINVAL when R exceeds one block of vectors (more than 1024
 * chunks of 16 bytes (FP64) or 32 bytes (FP32) per row, after rounding the
 * chunk count up to a power of two; dense handles have no such limit). */
kpm_status kpm_moments(kpm_handle h, const kpm_params* p, double* mu, double* mu_per_vec,
                       void* stream);

/* Local moments (the local density of states; the paper lists local
 * quantities among the KPM's uses, Sec. I, and the cited KPM review defines
 * them): mu_loc[j*M + n] = <i_j| T_n(H~) |i_j> for the nsites sites
 * i_j = sites[j], from the recursion of Eq. (rn) started on the unit vectors
 * sqrt(N) e_{i_j} (one vector column per site, so that the estimator's 1/N
 * normalisation of Eq. (munr) gives the local moment).  The start block is
 * written on the device from the site indices; nothing N-sized crosses the
 * bus.  sites is a host array of nsites indices in [0, N) (repeats allowed);
 * M, a, b and precision as kpm_params; mu_loc host or device (host output
 * synchronises and reports KPM_EDIVERGE like kpm_moments).  The sum over all
 * N sites of the local moments is N times the moments of kpm_moments' exact
 * trace.  The call replaces the handle's resumable state like kpm_moments.
 * Returns KPM_EINVAL for an index outside [0, N), nsites < 1, a device
 * pointer for sites, or what kpm_moments rejects with R = nsites. */
kpm_status kpm_ldos_moments(kpm_handle h, const int64_t* sites, int nsites, int M, double a,
                            double b, int precision, double* mu_loc, void* stream);

/* Momentum-resolved moments (the spectral function A(k, E); the paper names
 * spectral functions among the KPM's uses, Sec. I):
 *   mu_k[j*M + n] = <k_j| T_n(H~) |k_j>,  |k> = N^{-1/2} sum_x e^{i k.x} |x>,
 * for nk wave vectors k_j = (k[3j], k[3j+1], k[3j+2]) in radians per lattice
 * spacing (components beyond the lattice's dims are ignored; x are the
 * integer site coordinates of kpm_stencil_desc).  The Jackson-damped series
 * of these moments (kpm_dos) is A(k_j, E); on a clean periodic lattice with
 * k on the reciprocal grid (k_d = 2 pi m_d / L_d) the plane wave is an
 * eigenvector and mu_n = T_n(E~(k)) exactly.  The plane waves are written on
 * the device.  Complex field: one vector column per wave vector.  Real
 * field: the columns cos(k.x) and sin(k.x), whose moments add up to those of
 * the plane wave because H~ is real symmetric (a device kernel adds the
 * pairs).  Stencil handles only (CSR and dense handles carry no lattice
 * coordinates: KPM_EINVAL); k a host array; mu_k host or device; M, a, b,
 * precision and errors as kpm_moments; replaces the resumable state. */
kpm_status kpm_spectral_moments(kpm_handle h, const double* k, int nk, int M, double a, double b,
                                int precision, double* mu_k, void* stream);

/* Checkpoint and resume (the paper has no counterpart; a library service):
 * continues the realisation of the most recent kpm_moments call on `h` to M
 * moments (M even, larger than that call's M).  A call with S == 1 leaves
 * v_{n-1}, v_n and the per-step moment sums of its realisation in the
 * handle; this entry point runs products n = M_old/2 .. M/2 - 1 from there
 * with the same launches as one uninterrupted call, so mu[0..M) (and
 * mu_per_vec[r*M + n], the R vectors of that call) equal those of a single
 * kpm_moments call with this M and the same parameters bit for bit.  It may
 * be repeated (256 -> 512 -> 1024).  Outputs as kpm_moments (host or device;
 * host outputs synchronise and report KPM_EDIVERGE).  A kpm_moments call
 * rejected by its argument checks touches nothing and leaves the state as it
 * was; any other kpm_moments call replaces it.  KPM_ENOTREADY if there is no
 * such state: no previous call, the last call had S > 1, or the last
 * kpm_moments or kpm_moments_extend call that passed its argument checks
 * failed part way (an allocation or a launch), which drops the state;
 * KPM_EINVAL if M is odd or not larger (the state is then kept). */
kpm_status kpm_moments_extend(kpm_handle h, int M, double* mu, double* mu_per_vec, void* stream);

/* Kernel-damped Chebyshev series on K Chebyshev nodes (Eq. (fKPM)):
 *   x_k = cos(pi (k + 1/2) / K),  E[k] = a x_k + b,
 *   rho[k] = [g_0 mu_0 + 2 sum_{n=1}^{M-1} g_n mu_n cos(pi n (k+1/2)/K)] / (pi a sqrt(1 - x_k^2))
 * for k = 0 .. K-1 (E descending), g_n the Jackson kernel
 *   g_n = [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))] / (M+1)
 * or 1 (KPM_KERNEL_NONE).  mu, E, rho host or device; computed in FP64 on the
 * device.  1 <= M <= 1<<20, 1 <= K <= 1<<20. */
kpm_status kpm_dos(const double* mu, int M, double a, double b, int K, int kernel,
                   double* E, double* rho, void* stream);

/* kpm_dos with any damping kernel, including the Lorentz kernel
 *   g_n = sinh(lambda (1 - n/M)) / sinh(lambda),  lambda > 0
 * of the KPM review the paper cites (Eq. 74 there; the paper itself names only
 * the Jackson kernel, Sec. I).  lambda is read only for KPM_KERNEL_LORENTZ.
 * Arguments, ranges and errors as kpm_dos. */
kpm_status kpm_dos_kernel(const double* mu, int M, double a, double b, int K, int kernel,
                          double lambda, double* E, double* rho, void* stream);

/* Local Green's function from moments mu (e.g. the local moments of a unit
 * start vector) by the KPM review's expansion (Eq. 86 there; the paper names
 * Green's functions among the KPM quantities, Sec. I):
 *   G(x + i0) = -i / sqrt(1 - x^2) [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n exp(-i n arccos x)]
 * on the K Chebyshev nodes of kpm_dos (E[k] = a x_k + b), in energy units
 * (divided by a): g_re[k] = Re G, g_im[k] = Im G = -pi rho[k].  Damping as
 * kpm_dos_kernel (the review recommends the Lorentz kernel for G).  mu, E,
 * g_re, g_im host or device (E may be NULL); FP64 on the device; ranges and
 * errors as kpm_dos_kernel. */
kpm_status kpm_green(const double* mu, int M, double a, double b, int K, int kernel,
                     double lambda, double* E, double* g_re, double* g_im, void* stream);

/* Finite-temperature integrals of the DOS (the thermodynamic quantities the
 * KPM review obtains from the moments, Sec. IV there; the paper lists them
 * among the KPM's uses, Sec. I).  For each inverse temperature beta[t]
 * (+INFINITY: the ground state) and chemical potential mu_c, with Fermi
 * occupation f(E) = 1/(1 + exp(beta (E - mu_c))), per site:
 *   out[4t+0] = n = int rho f dE,   out[4t+1] = u = int E rho f dE,
 *   out[4t+2] = s = -int rho [f ln f + (1-f) ln(1-f)] dE   (k_B = 1),
 *   out[4t+3] = c = beta^2 int rho (E - mu_c)^2 f (1-f) dE = d(u - mu_c n)/dT,
 * by the Gauss-Chebyshev rule on the K nodes of the damped DOS
 * (kpm_dos_kernel): int g rho dE = sum_k g(E_k) rho_k a pi sqrt(1 - x_k^2) / K.
 * mu, beta, out host or device; 1 <= nT <= 65535, beta >= 0; FP64 on the
 * device; other ranges and errors as kpm_dos_kernel. */
kpm_status kpm_thermo(const double* mu, int M, double a, double b, int K, int kernel,
                      double lambda, const double* beta, int nT, double mu_c, double* out,
                      void* stream);

/* Stochastic error bars (the paper's estimator Eq. (munr) averages over
 * independent random vectors, Sec. II-A-3; this reports their spread).  From
 * the per-vector moments pv[r*M + n] of nvec independent vectors (the
 * mu_per_vec output of kpm_moments): mu_mean[n] and mu_err[n], the mean and
 * its standard error sqrt(sum_r (mu_n^r - mean)^2 / ((nvec-1) nvec)) (0 when
 * nvec = 1); and the DOS of every vector on the K nodes of kpm_dos_kernel,
 * with rho_mean[k] (equal to the DOS of mu_mean) and its standard error
 * rho_err[k].  Any output may be NULL; inputs and outputs host or device;
 * FP64 on the device.  nvec >= 1, M and K as kpm_dos, nvec * K <= 1<<28. */
kpm_status kpm_stats(const double* pv, int nvec, int M, double a, double b, int K, int kernel,
                     double lambda, double* mu_mean, double* mu_err, double* E,
                     double* rho_mean, double* rho_err, void* stream);

/* Adaptive number of random vectors: repeats kpm_moments with the parameters
 * p (seed p->seed + round for round = 0, 1, ...) until the integrated
 * standard error of the DOS, sum_k rho_err[k] * a pi sqrt(1 - x_k^2) / K
 * (the Gauss-Chebyshev quadrature of int |sigma_rho(E)| dE), is at most
 * target or max_rounds rounds have run.  Outputs are over all rounds' vectors
 * as kpm_stats (mu, E, rho, rho_err host or device; mu_err may be NULL);
 * *rounds and *achieved (host) receive the rounds run and the final error.
 * Requires p->user_v0 == NULL.  Returns what kpm_moments returns on error. */
kpm_status kpm_moments_adaptive(kpm_handle h, const kpm_params* p, int K, int kernel,
                                double lambda, double target, int max_rounds, double* mu,
                                double* mu_err, double* E, double* rho, double* rho_err,
                                int* rounds, double* achieved, void* stream);

/* Device time of the fused-step chain of the most recent kpm_moments call on
 * this handle: from the first fused step to the end of the last cross-CTA
 * moment reduction of its last realisation, measured with two CUDA events
 * recorded inside the replayed graph on the call's stream.  *step_launches
 * receives the number of fused-step kernels in that chain (M/2), so ms /
 * step_launches is the average duration of one fused step launch (for the
 * column-resident solve: the one launch that runs all M/2 products, and ms /
 * step_launches the average product inside it).  Call after
 * the kpm_moments stream has completed; KPM_ENOTREADY if no call was made. */
kpm_status kpm_step_timing(kpm_handle h, double* ms, int* step_launches);

/* ---------------------------------------------------------------- batches
 * Many independent solves of uneven size (different lattices, N and M) run
 * by ONE persistent kernel launch, captured once into a CUDA graph and
 * replayed.  The launch is made of thread-block clusters of C CTAs; each
 * cluster takes the next instance from a device queue (longest first), splits
 * its rows among its C CTAs and runs all of its M/2 products back to back,
 * the CTAs meeting at the hardware cluster barrier between products and
 * adding their moment partials through distributed shared memory in rank
 * order.  An instance's moments therefore depend only on C and the instance,
 * not on the rest of the batch.  This is the batched form of kpm_moments for
 * the paper's many-realisation workload (Sec. II-A-4: S realisations, each a
 * different Hamiltonian for disorder averages). */
typedef struct kpm_batch_s* kpm_batch;

/* Builds a batch of `count` instances: handles[i] with params[i] (M even,
 * a, b, seed; S must be 1 and user_v0 NULL).  All handles must be on the same
 * device and of the same kind (field; stencil dims, presence of per-bond
 * hoppings and on-site terms; or CSR with the same padded-ELL width), and all
 * params must share precision and R.  The batch owns its vector blocks and
 * its own scaled copies of the operators (later calls on the handles do not
 * affect it); the handles must outlive the batch.  If an autotuned
 * configuration for this device and batch shape is in the tuning cache
 * (file $KPM_TUNE_CACHE, default ~/.cache/kpm_gb300_autotune.txt) it is used. */
kpm_status kpm_batch_create(int count, const kpm_handle* handles, const kpm_params* params,
                            kpm_batch* out);

/* Runs the whole batch (every instance from its first to its last product)
 * on `stream` by replaying the captured graph, and writes the moments of
 * instance i to mu[off_i .. off_i + M_i) with off_i = M_0 + ... + M_{i-1}
 * (host or device; NULL skips the copy).  Host outputs synchronise and
 * report KPM_EDIVERGE like kpm_moments. */
kpm_status kpm_batch_run(kpm_batch b, double* mu, void* stream);

/* Autotuner: times `reps` replays of every launchable untiled configuration
 * (cluster size C in {1, 2, 4, 8, 16}, traversal chunk in {2, 4, 16} passes,
 * 100 % or 50 % of the co-resident clusters), then twice the threads per row
 * (kpm_batch_set_chunk_bytes 16, real FP32 stencils) at every cluster size
 * and traversal chunk, then the resident form
 * (kpm_batch_set_resident) at every cluster size where it fits, and, if the
 * global-memory form is still the fastest, R-tiling (2 or 4 tiles dividing
 * the chunks per row) of all, half, an eighth or a thirty-second of the
 * instances, largest work first, at the best configuration and at half its
 * cluster size; keeps the fastest for this batch and appends it to the
 * tuning cache. */
kpm_status kpm_batch_tune(kpm_batch b, int reps, void* stream);

/* Fixes the configuration (cluster size a power of two <= 16, chunk >= 1,
 * percent of co-resident clusters in 1..100) without tuning. */
kpm_status kpm_batch_set_config(kpm_batch b, int cluster, int chunk, int percent);

/* Current configuration, clusters launched, and the device time (ms) of the
 * most recent replay (CUDA events recorded inside the graph). */
kpm_status kpm_batch_info(kpm_batch b, int* cluster, int* chunk, int* clusters_launched,
                          double* last_ms);

/* R-tiling: the padded vector block (Rp columns in G chunks per row) of each
 * of the `top` instances of largest work (N*M; top <= 0 or >= count: all) is
 * split into `rtiles` column tiles run as independent tasks, possibly on
 * different clusters at the same time (each tile a self-contained KPM
 * recursion on its vectors, Eq. (rn)); the last tile to finish averages the
 * per-vector moments.  rtiles in {1, 2, 4} and dividing G (KPM_EINVAL
 * otherwise); 1 = no tiling.  An instance's moments depend only on C, its
 * tile count and the instance. */
kpm_status kpm_batch_set_rtiles(kpm_batch b, int rtiles, int top);

/* Threads per row: each thread moves one chunk of `bytes` bytes of a row per
 * product, so a row of Rp columns takes Rp*4/bytes threads (real FP32).
 * bytes = 32 (the default: 8 real or 4 complex FP32 columns per thread) or
 * 16 (4 real columns: twice the threads per row, half the registers of
 * vector data per thread); 16 needs a real FP32 batch of stencil operators
 * in the global-memory form (KPM_EINVAL otherwise).  FP64 batches always
 * move 16-byte chunks (2 real or 1 complex column).  The row layout is the
 * same for both widths. */
kpm_status kpm_batch_set_chunk_bytes(kpm_batch b, int bytes);

/* Current chunk width in bytes and threads per row (chunks per row). */
kpm_status kpm_batch_get_chunk_bytes(kpm_batch b, int* bytes, int* threads_per_row);

/* Resident form (resident = 1): each cluster keeps the two vector blocks of
 * the instance it runs in its CTAs' shared memory for the whole solve, CTA
 * rank k holding the rows [k P, k P + P) with P = ceil(N / C), and reads the
 * neighbour rows held by the other CTAs through distributed shared memory;
 * the products (Eq. (rn)) and the moment identities are unchanged and no
 * vector row goes to global memory.  For stencil operators whose largest
 * instance fits (KPM_EINVAL otherwise); untiled (setting resident clears the
 * R-tiling, and R-tiling is refused while it is set).  The cluster size and
 * the share of co-resident clusters still come from kpm_batch_set_config;
 * the traversal chunk does not apply.  An instance's moments depend only on
 * C and the instance, as in the global-memory form. */
kpm_status kpm_batch_set_resident(kpm_batch b, int resident);

/* Whether the resident form is set, and the smallest cluster size at which
 * the batch's largest instance fits in shared memory (0: none does, or the
 * operator is not a stencil). */
kpm_status kpm_batch_get_resident(kpm_batch b, int* resident, int* min_cluster);

/* Staged form (staged = 1): the products of Eq. (rn) with the vector rows
 * brought into shared memory by bulk asynchronous copies (cp.async.bulk)
 * instead of per-thread loads.  Each instance's rows are cut into tiles of
 * T consecutive rows (a power of two, about 4 KB x the traversal chunk of
 * kpm_batch_set_config, 1..4); CTA k of a cluster owns a contiguous band of
 * tiles, and one thread per CTA copies, several tiles ahead of use, the
 * band's tiles of v_n with the halo tiles that hold neighbours one lattice
 * line (or plane) away into a ring of shared-memory stages, and the band's
 * tiles of v_{n-1} and of the scaled on-site terms into a second ring.  The
 * rows are computed from shared memory; neighbours across a periodic wrap
 * beyond the halo are read from global memory; v_{n+1} is stored in place
 * over v_{n-1}.  The moment identities, partial sums and finalisation are
 * unchanged.  Stencil operators with rows of at most 32 chunks (R <= 256
 * real or 128 complex FP32, R <= 64 real or 32 complex FP64; KPM_EINVAL
 * otherwise); untiled (setting it clears the R-tiling); 32-byte chunks.  An
 * instance's moments depend only on C, the tile size and the instance, and
 * agree with the other forms to rounding (the moment dots are summed in
 * another order).  Every wait inside the kernel is bounded: one that runs
 * out makes kpm_batch_run with host output return KPM_ETIMEOUT.  staged = 0
 * returns to the global-memory form. */
kpm_status kpm_batch_set_staged(kpm_batch b, int staged);

/* Whether the staged form is set, and its tile rows T and v_n ring stages at
 * the current traversal chunk (any output may be NULL). */
kpm_status kpm_batch_get_staged(kpm_batch b, int* staged, int* tile_rows, int* stages);

/* Current R-tiles, the number of instances tiled, and the largest R-tiles
 * this batch admits (min(4, G)). */
kpm_status kpm_batch_get_rtiles(kpm_batch b, int* rtiles, int* top, int* max_rtiles);

void kpm_batch_destroy(kpm_batch b);

/* ---------------------------------------------------------------- serving
 * A request loop with continuous batching.  Requests (a handle, its
 * parameters and a DOS node count) may be submitted from any thread while
 * others run.  A scheduler thread owns a device arena of `hbm_budget_bytes`
 * and runs ticks: pending requests are admitted first come first served as
 * soon as their device memory fits in the budget (two N x R vector blocks,
 * a scaled copy of the operator, moment sums and outputs, DOS buffers);
 * every resident request then advances up to `steps_per_tick` products -
 * small ones (a product moving < 8 MB) together in one batched persistent
 * cluster launch per operator kind and vector width, large ones as full-GPU
 * fused steps on a pool of streams - so requests that arrive while others are
 * on the GPU join the next tick and their work overlaps; finished requests
 * get the Jackson DOS on the device, their results are copied to the host and
 * their memory is released.  A request's moments are the same alone and in
 * any mix.  Handles must outlive their requests. */
typedef struct kpm_server_s* kpm_server;

typedef struct {
  uint64_t submitted, completed, failed, cancelled, ticks;
  double p50_s, p99_s, mean_s, max_s;  /* submit -> results-on-host latency of completed requests */
  double solves_per_s;                 /* completed / (last completion - first submission) */
  int peak_resident;
  size_t peak_bytes, budget_bytes;
} kpm_server_stats_t;

/* cluster: CTAs per cluster of the batched launches (power of two <= 16);
 * steps_per_tick in 1..64. */
kpm_status kpm_server_create(size_t hbm_budget_bytes, int steps_per_tick, int cluster,
                             kpm_server* out);

/* Queues a request: params as for kpm_moments (S = 1, no user_v0; a and b
 * given), K Jackson-DOS nodes (0: moments only).  KPM_ENOMEM if the request
 * alone exceeds the budget. */
kpm_status kpm_server_submit(kpm_server s, kpm_handle h, const kpm_params* p, int K,
                             uint64_t* req_id);

/* Blocks until the request has finished, failed or been cancelled
 * (timeout_s < 0: no limit; KPM_ETIMEOUT otherwise). */
kpm_status kpm_server_wait(kpm_server s, uint64_t req_id, double timeout_s);

/* Copies a finished request's results (mu[M], E[K], rho[K] host buffers, any
 * may be NULL) and its latency, then forgets the request.  KPM_ENOTREADY while
 * it is pending or running; the request's own status (e.g. KPM_EDIVERGE)
 * otherwise. */
kpm_status kpm_server_poll(kpm_server s, uint64_t req_id, double* mu, double* E, double* rho,
                           double* latency_s);

/* Cancels a pending or running request at the next tick boundary; the other
 * requests are unaffected.  Its poll then reports KPM_EINVAL. */
kpm_status kpm_server_cancel(kpm_server s, uint64_t req_id);

kpm_status kpm_server_stats(kpm_server s, kpm_server_stats_t* out);

/* Stops the scheduler (requests still queued or running are dropped) and
 * releases the arena. */
void kpm_server_destroy(kpm_server s);

/* Size of the fixed device scratch array behind kpm_moments_csr_noalloc. */
#define KPM_NOALLOC_SCRATCH_BYTES (32u << 20)

/* kpm_moments without any device allocation (the paper has no counterpart;
 * this is a library service).  Some callers cannot allocate device memory
 * during a call: they run with a frozen or exhausted memory pool, budget all
 * device memory at start-up, or cannot afford the device synchronisation and
 * locking that cudaMalloc/cudaFree may cause.  This entry point computes the
 * FP64 Chebyshev moments mu[0..M) of a CSR matrix that is already in device
 * memory (d_rowptr[n+1] int64, d_col[nnz] int32, d_val[nnz] FP64 or [nnz][2]
 * complex FP64, same layout and meaning as kpm_create_csr) with the same
 * random vectors and the same doubling identities as kpm_moments with S = 1
 * and precision KPM_FP64, and allocates nothing: all of its scratch (a
 * checked copy of the structure, two N x R vector blocks, the scaled matrix
 * values, partial and moment sums, the per-vector moments the mean is
 * taken from) lives in one file-scope device array of
 * KPM_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds
 * until the process exits.  Its fused step is the library's generic CSR
 * kernel (rows walked through the row pointers); kpm_moments takes a padded
 * ELL copy for short rows, so the two agree to rounding (1e-10), not bit for
 * bit.
 *   Preconditions: the three arrays hold at least n+1, nnz and nnz (x2
 *       complex) elements, and H is Hermitian.  The structure is checked on
 *       the device before use: rowptr[0] == 0, rowptr non-decreasing,
 *       rowptr[n] == nnz, every col in [0, n).  The products read only a copy
 *       of it whose indices are made safe, so a broken rule never sends a
 *       load out of bounds; it makes a host-output call return KPM_EINVAL
 *       before any product is launched, and a device-output call write NaN
 *       to every mu[n].
 *   mu: M doubles, device (asynchronous on `stream`) or host (synchronises and
 *       reports KPM_EDIVERGE like kpm_moments).
 * Returns KPM_EINVAL, naming the bytes it would need, when the problem does
 * not fit in the scratch: about 16 N Rp + 8 N + 12 nnz + 8 M (Rp + R) bytes
 * for the real field, plus 128 Rp bytes per CTA of the step for the moment
 * partials (Rp = R rounded up to a power of two, at least 2; complex: twice
 * the vector and value terms, Rp = R rounded up to a power of two), R at
 * most 512 real or 256 complex.  The
 * first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * call the entry point after a cudaDeviceReset of that device (the kept
 * address would be stale).  All calls share the scratch and each leaves its
 * contents behind: calls whose work can overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller. */
kpm_status kpm_moments_csr_noalloc(int64_t n, int64_t nnz, const int64_t* d_rowptr,
                                   const int32_t* d_col, const double* d_val, kpm_field field,
                                   int M, int R, uint64_t seed, double a, double b, double* mu,
                                   void* stream);

/* Handle properties (any output may be NULL): dimension, stored nonzeros of H
 * (bonds in both directions plus stored diagonal entries), field, and
 * stencil (1) or CSR (0). */
kpm_status kpm_info(kpm_handle h, int64_t* n, int64_t* nnz, int* field, int* is_stencil);

/* Releases the handle and its device memory (NULL is a no-op). */
void kpm_destroy(kpm_handle h);

/* Message of the calling thread's last failure ("" if none). */
const char* kpm_last_error(void);

/* Number of CUDA kernels the library has enqueued in this process (kernels in
 * a replayed graph count once per replay). */
uint64_t kpm_kernel_launches(void);

/* Testing aid (the paper has no counterpart): host-side fault injection for
 * the library's own device allocations.  The next `after` allocations of the
 * library's handles and calls succeed and the one after them fails with
 * KPM_ENOMEM, as a real out-of-memory would; the injector then disarms.
 * after = -1 disarms it at once.  Process-wide; no device work is involved.
 * Returns KPM_EINVAL for after < -1. */
kpm_status kpm_testing_fail_allocations(int64_t after);

/* Testing aid (the paper has no counterpart): with on != 0, kpm_moments calls
 * that plan their launches from now on (a new handle, or a new shape) give
 * the TMA-fed padded-ELL step (FP32 vectors on a CSR handle with short rows)
 * and the TMA-fed stencil step (FP32 vectors on a 2D or 3D stencil handle,
 * where the environment variable KPM_STENCIL_TMA selects it) a producer that
 * issues no copy, so
 * the consumers' bounded waits run out
 * (after about a second per step) and the call returns KPM_ETIMEOUT with its
 * outputs invalid; the context stays usable.  on = 0 stops it for plans made
 * afterwards.  Process-wide.  Always returns KPM_OK. */
kpm_status kpm_testing_stall_step_pipeline(int on);

/* Testing aid (the paper has no counterpart): the form of the product that
 * the most recent plan of kpm_moments on h chose (host output *form):
 * 0 the fused step (stencil, CSR or padded ELL), 1 the TMA-fed padded-ELL
 * step, 2 the dense product on the FP64 pipe, 3 the dense product on the
 * tensor cores, 4 the TMA-fed stencil step, 5 the column-resident solve
 * (all products of a realisation of a small stencil or padded-ELL operator in
 * one cluster launch).  KPM_ENOTREADY before the first kpm_moments call. */
kpm_status kpm_testing_last_step_form(kpm_handle h, int* form);

#ifdef __cplusplus
}
#endif

#endif /* KPM_H */
