// Auxiliary kernels of the KPM path: operator rescaling (Eq. (tilde)),
// random start vectors (stochastic trace, Sec. II-A-3), the deterministic
// moment reduction and doubling (Eq. (munr)), Gershgorin and Lanczos spectral
// bounds, and the Jackson-damped Chebyshev series of Eq. (fKPM).
#include <math.h>

#include "kpm_internal.h"
#include "kpm_rng.cuh"

namespace kpm {

namespace {

inline unsigned blocks_for(int64_t n, int block) {
  int64_t b = (n + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 65535LL * 32) b = 65535LL * 32;
  return (unsigned)b;
}

inline cudaError_t counted(cudaError_t e) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

// ------------------------------------------------------------------ prescale
// S = scale (H - shift): scaled hoppings -scale*t, scaled diagonal scale*(eps - shift).
template <typename T, bool CPLX>
__global__ void prescale_stencil_kernel(int64_t n, int dims, const double* __restrict__ onsite,
                                        const double* __restrict__ hop, double t_re, double t_im,
                                        const RunParams* prm, bool lanczos, T* hs, T* ds,
                                        ScalarBlock* sc) {
  __shared__ double s_scale, s_shift;
  if (threadIdx.x == 0) {
    s_scale = lanczos ? 1.0 : 2.0 / prm->a;
    s_shift = lanczos ? 0.0 : prm->b;
  }
  __syncthreads();
  const double scale = s_scale, shift = s_shift;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    sc->hu_re = -scale * t_re;
    sc->hu_im = -scale * t_im;
    sc->du = -scale * shift;
    sc->hu_re_f = (float)sc->hu_re;
    sc->hu_im_f = (float)sc->hu_im;
    sc->du_f = (float)sc->du;
  }
  for (int64_t s = i; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (ds) ds[s] = (T)(scale * (onsite[s] - shift));
    if (hs) {
      for (int d = 0; d < dims; ++d) {
        if (CPLX) {
          hs[2 * (s * dims + d)] = (T)(-scale * hop[2 * (s * dims + d)]);
          hs[2 * (s * dims + d) + 1] = (T)(-scale * hop[2 * (s * dims + d) + 1]);
        } else {
          hs[s * dims + d] = (T)(-scale * hop[s * dims + d]);
        }
      }
    }
  }
}

template <typename T, bool CPLX>
__global__ void prescale_csr_kernel(int64_t nnz, const double* __restrict__ val,
                                    const RunParams* prm, bool lanczos, T* vals, ScalarBlock* sc) {
  __shared__ double s_scale, s_shift;
  if (threadIdx.x == 0) {
    s_scale = lanczos ? 1.0 : 2.0 / prm->a;
    s_shift = lanczos ? 0.0 : prm->b;
  }
  __syncthreads();
  const double scale = s_scale, shift = s_shift;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    sc->hu_re = 0.0;
    sc->hu_im = 0.0;
    sc->du = -scale * shift;
    sc->hu_re_f = 0.f;
    sc->hu_im_f = 0.f;
    sc->du_f = (float)sc->du;
  }
  const int64_t m = CPLX ? 2 * nnz : nnz;
  for (int64_t s = i; s < m; s += (int64_t)gridDim.x * blockDim.x) vals[s] = (T)(scale * val[s]);
}

// ------------------------------------------------------------------ random vectors
template <typename T, bool CPLX>
__global__ void rng_init_kernel(int64_t n, int Rp, const RunParams* __restrict__ prm, T* v0) {
  const int R = prm->R;
  const unsigned long long seed = prm->seed;
  const unsigned long long s = (unsigned long long)(prm->s + prm->s0);
  const int64_t total = n * Rp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    random_entry<T, CPLX>(v0, n, Rp, R, seed, s, e);
}

template <typename T, bool CPLX>
__global__ void load_v0_kernel(int64_t n, int R, int Rp, const double* __restrict__ src, T* v0) {
  const int64_t total = n * Rp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Rp;
    const int r = (int)(e % Rp);
    if (CPLX) {
      int64_t ore, oim;
      cplx_offsets<T>(i, r, Rp, ore, oim);
      v0[ore] = r < R ? (T)src[2 * (i * R + r)] : T(0);
      v0[oim] = r < R ? (T)src[2 * (i * R + r) + 1] : T(0);
    } else {
      v0[e] = r < R ? (T)src[i * R + r] : T(0);
    }
  }
}

// Start blocks built on the device.  Unit sites (local moments): column r is
// sqrt(N) e_{sites[r]}, so that the estimator's 1/N normalisation of
// Eq. (munr) gives <i|T_n(H~)|i>.  Plane waves (momentum-resolved moments):
// column r (complex field) is e^{i k_r . x}, x the lattice coordinates of the
// site; on the real field columns 2j and 2j+1 are cos(k_j . x) and
// sin(k_j . x).  Either way |column|^2 = N (a pair's two columns together).
template <typename T, bool CPLX>
__global__ void start_block_kernel(int kind, int64_t n, int R, int Rp, const void* __restrict__ params,
                                   StencilGeom g, T* v0) {
  const int64_t total = n * Rp;
  const double root_n = sqrt((double)n);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Rp;
    const int r = (int)(e % Rp);
    double re = 0.0, im = 0.0;
    if (r < R) {
      if (kind == 1) {
        if (reinterpret_cast<const int64_t*>(params)[r] == i) re = root_n;
      } else {
        const int j = CPLX ? r : r / 2;
        const double* k = reinterpret_cast<const double*>(params) + 3 * (size_t)j;
        double phase = 0.0;
        for (int d = 0; d < g.dims; ++d) phase += k[d] * (double)((i / g.stride[d]) % g.L[d]);
        double sv, cv;
        sincos(phase, &sv, &cv);
        if (CPLX) {
          re = cv;
          im = sv;
        } else {
          re = (r & 1) ? sv : cv;
        }
      }
    }
    if (CPLX) {
      int64_t ore, oim;
      cplx_offsets<T>(i, r, Rp, ore, oim);
      v0[ore] = (T)re;
      v0[oim] = (T)im;
    } else {
      v0[e] = (T)re;
    }
  }
}

__global__ void pair_sum_kernel(const double* __restrict__ pv, int npairs, int M,
                                double* __restrict__ out) {
  const int64_t total = (int64_t)npairs * M;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / M, m = e % M;
    out[e] = pv[(2 * j) * M + m] + pv[(2 * j + 1) * M + m];
  }
}

// ------------------------------------------------------------------ moment reduction
// ring[slot][cta][2*Rp] -> sums[s][step][2*Rp].  Block (k, g) sums 32 output
// columns of step first+k: warp w adds CTAs w, w+8, w+16, ... in order, then
// the 8 warp sums are added in warp order (a fixed order for a given grid).
__global__ void reduce_ring_kernel(const double* __restrict__ ring, int ring_slots, int first_step,
                                   int nCTA, int Rp, const RunParams* __restrict__ prm,
                                   int steps_per_real, double* sums) {
  __shared__ double part[8][33];
  const int w = 2 * Rp;
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int o = blockIdx.y * 32 + lane;
  const int step = first_step + blockIdx.x;
  double acc = 0.0;
  if (o < w) {
    const double* src = ring + (size_t)(step % ring_slots) * nCTA * w + o;
#pragma unroll 4
    for (int c = slice; c < nCTA; c += 8) acc += src[(size_t)c * w];
  }
  part[slice][lane] = acc;
  __syncthreads();
  if (slice == 0 && o < w) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += part[k][lane];
    sums[((size_t)prm->s * steps_per_real + step) * w + o] = t;
  }
}

__global__ void advance_realisation_kernel(RunParams* prm) { prm->s += 1; }

// Doubling identities per vector, then the average over all S*R vectors.
__global__ void finalize_pervec_kernel(const double* __restrict__ sums, int S, int steps, int R,
                                       int Rp, int64_t n, int M, double* per_vec, RunParams* prm) {
  const int64_t total = (int64_t)S * R * steps;
  const int w = 2 * Rp;
  const double inv_n = 1.0 / (double)n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int step = (int)(e % steps);
    const int64_t sr = e / steps;
    const int r = (int)(sr % R), s = (int)(sr / R);
    const double* base = sums + (size_t)s * steps * w;
    const double mu0 = base[r] * inv_n, mu1 = base[Rp + r] * inv_n;
    double me, mo;
    if (step == 0) {
      me = mu0;
      mo = mu1;
    } else {
      me = 2.0 * base[(size_t)step * w + r] * inv_n - mu0;
      mo = 2.0 * base[(size_t)step * w + Rp + r] * inv_n - mu1;
    }
    per_vec[(size_t)sr * M + 2 * step] = me;
    per_vec[(size_t)sr * M + 2 * step + 1] = mo;
    const double lim = 1.0 + 1e-6;
    if (!(fabs(me) <= lim) || !(fabs(mo) <= lim)) atomicOr(&prm->flags, 1);
  }
}

__global__ void finalize_mean_kernel(const double* __restrict__ per_vec, int cols, int M,
                                     double* mu) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < cols; ++c) acc += per_vec[(size_t)c * M + m];
    mu[m] = acc / (double)cols;
  }
}

// ------------------------------------------------------------------ Gershgorin
__device__ __forceinline__ double cabs2(double re, double im) { return hypot(re, im); }

__global__ void gershgorin_stencil_kernel(bool cplx, int64_t n, StencilGeom g,
                                          const double* __restrict__ onsite,
                                          const double* __restrict__ hop, double t_re,
                                          double t_im, double* pmin, double* pmax) {
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i64 < n;
       i64 += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)i64;
    double center = onsite ? onsite[i] : 0.0, rad = 0.0;
    int rem = i;
    for (int d = 0; d < g.dims; ++d) {
      const int L = g.L[d], s = g.stride[d];
      const int x = rem % L;
      rem /= L;
      const bool per = g.periodic[d] != 0;
      auto hopv = [&](int site, double& re, double& im) {
        if (hop) {
          re = cplx ? hop[2 * ((size_t)site * g.dims + d)] : hop[(size_t)site * g.dims + d];
          im = cplx ? hop[2 * ((size_t)site * g.dims + d) + 1] : 0.0;
        } else {
          re = t_re;
          im = t_im;
        }
      };
      double fr, fi, br, bi;
      if (L == 1) {
        if (per) {  // the bond joins the site to itself: H_ii += -t - conj(t)
          hopv(i, fr, fi);
          center += -2.0 * fr;
        }
        continue;
      }
      const bool hasf = (x + 1 < L) || per, hasb = (x > 0) || per;
      const int jf = (x + 1 < L) ? i + s : i - (L - 1) * s;
      const int jb = (x > 0) ? i - s : i + (L - 1) * s;
      if (L == 2 && per) {  // both bonds join the same pair: |H_ij| = |t_f + conj(t_b)|
        hopv(i, fr, fi);
        hopv(jb, br, bi);
        rad += cabs2(fr + br, fi - bi);
        continue;
      }
      if (hasf) { hopv(i, fr, fi); rad += cabs2(fr, fi); }
      if (hasb) { hopv(jb, br, bi); rad += cabs2(br, bi); }
      (void)jf;
    }
    lo = fmin(lo, center - rad);
    hi = fmax(hi, center + rad);
  }
  __shared__ double smin[256], smax[256];
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pmin[blockIdx.x] = smin[0];
    pmax[blockIdx.x] = smax[0];
  }
}

__global__ void gershgorin_csr_kernel(bool cplx, int64_t n, const int64_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ col,
                                      const double* __restrict__ val, double* pmin, double* pmax) {
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double center = 0.0, rad = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double re = cplx ? val[2 * k] : val[k];
      const double im = cplx ? val[2 * k + 1] : 0.0;
      if (col[k] == i) center += re;
      else rad += cabs2(re, im);
    }
    lo = fmin(lo, center - rad);
    hi = fmax(hi, center + rad);
  }
  __shared__ double smin[256], smax[256];
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pmin[blockIdx.x] = smin[0];
    pmax[blockIdx.x] = smax[0];
  }
}

__global__ void minmax_final_kernel(const double* pmin, const double* pmax, int nblk, double* out) {
  double lo = INFINITY, hi = -INFINITY;
  for (int b = threadIdx.x; b < nblk; b += 32) {
    lo = fmin(lo, pmin[b]);
    hi = fmax(hi, pmax[b]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (threadIdx.x == 0) {
    out[0] = lo;
    out[1] = hi;
  }
}

// ------------------------------------------------------------------ Lanczos pieces
// Vectors are flat FP64 arrays of `len` scalars (complex: interleaved pairs).
__global__ void lanczos_start_kernel(bool cplx, int64_t n, int stride_scal,
                                     unsigned long long seed, double* q) {
  const double inv = rsqrt((double)n);
  const int64_t total = n * stride_scal;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / stride_scal;
    const int o = (int)(e % stride_scal);
    double v = 0.0;
    if (o == 0) v = (draw(seed, 6, (unsigned long long)i) >> 63) ? -inv : inv;
    q[e] = v;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reorthogonalisation.  The vectors are n pairs (double2): complex entries,
// or a real value beside a zero pad.  One Lanczos step j, after y = H q_j:
//   lz_local_dots:   c = (<q_j|y>, <q_{j-1}|y>) per block
//   lz_reorth_dots:  y' = y - c_j q_j - c_{j-1} q_{j-1} (the three-term step),
//                    then <q_l|y'> for l = 0..j per block (one full classical
//                    Gram-Schmidt pass), alpha_j = Re <q_j|y>
//   dots_final:      the coefficients d_l summed over the blocks
//   lz_update_norm:  y'' = y' - sum_l d_l q_l, per-block |y''|^2
//   lanczos_next:    beta_j = |y''|, q_{j+1} = y'' / beta_j
// GB300 runs FP64 at 1/64 of its FP32 rate, so these kernels are bound by
// FP64 instruction issue; the per-block sums of many values use a
// recursive-halving warp reduction (about one add per value per lane instead
// of five) so that the reductions stay small beside the dot products.

// Sums each of V values over the 32 lanes of a warp.  At each of the log2 V
// exchange steps a lane keeps one half of its values and adds the partner
// lane's copy of that half; the single value left is then summed over the
// remaining lane bits.  The result is the total of value index
// lane >> (5 - log2 V), the same in every lane that holds that index.
template <int V>
__device__ __forceinline__ double warp_multi_sum(double (&v)[V]) {
  static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V: a power of two up to 32");
  const int lane = threadIdx.x & 31;
  int o = 16;
#pragma unroll
  for (int h = V / 2; h >= 1; h /= 2, o /= 2) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double send = up ? v[i] : v[i + h];
      const double keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double s = v[0];
#pragma unroll
  for (; o >= 1; o /= 2) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

constexpr int LZ_BLOCK = 256;
constexpr int LZ_WARPS = LZ_BLOCK / 32;
constexpr int LZ_TILE = 8;  // Gram-Schmidt columns per reduction tile

// CTA sum of V values per thread (warp_multi_sum, then the warps in order);
// threads t < V return the total of value t.  `red` holds LZ_WARPS * V doubles.
template <int V>
__device__ __forceinline__ double block_multi_sum(double (&v)[V], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int SH = (V == 1) ? 5 : (V == 2) ? 4 : (V == 4) ? 3 : (V == 8) ? 2 : (V == 16) ? 1 : 0;
  const double s = warp_multi_sum<V>(v);
  if ((lane & ((1 << SH) - 1)) == 0) red[warp * V + (lane >> SH)] = s;
  __syncthreads();
  double tot = 0.0;
  if ((int)threadIdx.x < V)
    for (int w = 0; w < LZ_WARPS; ++w) tot += red[w * V + threadIdx.x];
  return tot;
}

// acc += conj(q) * y  (real: the value only)
template <bool CPLX>
__device__ __forceinline__ void cdot_acc(double& re, double& im, double2 q, double2 y) {
  if constexpr (CPLX) {
    re = fma(q.x, y.x, fma(q.y, y.y, re));
    im = fma(q.x, y.y, fma(-q.y, y.x, im));
  } else {
    re = fma(q.x, y.x, re);
  }
}

// y -= c * q
template <bool CPLX>
__device__ __forceinline__ void caxpy_sub(double2& y, double cr, double ci, double2 q) {
  if constexpr (CPLX) {
    y.x = fma(-cr, q.x, fma(ci, q.y, y.x));
    y.y = fma(-cr, q.y, fma(-ci, q.x, y.y));
  } else {
    y.x = fma(-cr, q.x, y.x);
  }
}

// part[blk][4] = (<q_j|y>, <q_{j-1}|y>) as (re, im, re, im); qm = NULL at j = 0
template <bool CPLX>
__global__ void __launch_bounds__(LZ_BLOCK) lz_local_dots_kernel(int64_t n,
                                                                 const double2* __restrict__ qj,
                                                                 const double2* __restrict__ qm,
                                                                 const double2* __restrict__ y,
                                                                 double* part) {
  __shared__ double red[LZ_WARPS * 4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t e = (int64_t)blockIdx.x * LZ_BLOCK + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * LZ_BLOCK) {
    const double2 yv = y[e];
    cdot_acc<CPLX>(acc[0], acc[1], qj[e], yv);
    if (qm) cdot_acc<CPLX>(acc[2], acc[3], qm[e], yv);
  }
  const double tot = block_multi_sum<4>(acc, red);
  if (threadIdx.x < 4) part[(size_t)blockIdx.x * 4 + threadIdx.x] = tot;
}

// The three-term step and the dot products of one classical Gram-Schmidt
// pass (see above).  part[l][blk][2] for l = 0..j; alpha[j] = Re <q_j|y>.
// Every block sums the local partials in the same order.
template <bool CPLX>
__global__ void __launch_bounds__(LZ_BLOCK) lz_reorth_dots_kernel(
    int64_t n, const double2* __restrict__ Q, int64_t ldq, int j,
    const double* __restrict__ part_loc, int nblk_loc, double2* y, double* part, double* alpha) {
  __shared__ double s_c[4];
  __shared__ double red[LZ_WARPS * 2 * LZ_TILE];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < 4) {
    double s = 0.0;
    for (int b = lane; b < nblk_loc; b += 32) s += part_loc[(size_t)b * 4 + warp];
    s = warp_sum(s);
    if (lane == 0) s_c[warp] = s;
  }
  __syncthreads();
  const double c0r = s_c[0], c0i = CPLX ? s_c[1] : 0.0, c1r = s_c[2], c1i = CPLX ? s_c[3] : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) alpha[j] = c0r;
  const double2* qj = Q + (size_t)j * ldq;
  const double2* qm = j > 0 ? Q + (size_t)(j - 1) * ldq : nullptr;
  const int64_t e0 = (int64_t)blockIdx.x * LZ_BLOCK + threadIdx.x, es = (int64_t)gridDim.x * LZ_BLOCK;
  for (int64_t e = e0; e < n; e += es) {
    double2 yv = y[e];
    caxpy_sub<CPLX>(yv, c0r, c0i, qj[e]);
    if (qm) caxpy_sub<CPLX>(yv, c1r, c1i, qm[e]);
    y[e] = yv;  // read back below by this same thread
  }
  constexpr int V = CPLX ? 2 * LZ_TILE : LZ_TILE;
  for (int l0 = 0; l0 <= j; l0 += LZ_TILE) {
    double acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.0;
    const int nt = min(LZ_TILE, j + 1 - l0);
    for (int64_t e = e0; e < n; e += es) {
      const double2 yv = y[e];
#pragma unroll
      for (int l = 0; l < LZ_TILE; ++l) {
        if (l < nt) {
          const double2 q = Q[(size_t)(l0 + l) * ldq + e];
          if constexpr (CPLX) cdot_acc<true>(acc[2 * l], acc[2 * l + 1], q, yv);
          else cdot_acc<false>(acc[l], acc[l], q, yv);
        }
      }
    }
    const double tot = block_multi_sum<V>(acc, red);
    if ((int)threadIdx.x < V) {
      const int l = CPLX ? (int)threadIdx.x / 2 : (int)threadIdx.x;
      const int c = CPLX ? (int)threadIdx.x % 2 : 0;
      if (l < nt) {
        part[((size_t)(l0 + l) * gridDim.x + blockIdx.x) * 2 + c] = tot;
        if (!CPLX) part[((size_t)(l0 + l) * gridDim.x + blockIdx.x) * 2 + 1] = 0.0;
      }
    }
    __syncthreads();  // red is reused by the next tile
  }
}

// y -= sum_{l <= j} coef_l q_l; part[blk] = partial |y|^2
template <bool CPLX>
__global__ void __launch_bounds__(LZ_BLOCK) lz_update_norm_kernel(int64_t n,
                                                                  const double2* __restrict__ Q,
                                                                  int64_t ldq, int j,
                                                                  const double* __restrict__ coef,
                                                                  double2* y, double* part) {
  __shared__ double red[LZ_WARPS];
  double acc[1] = {0.0};
  for (int64_t e = (int64_t)blockIdx.x * LZ_BLOCK + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * LZ_BLOCK) {
    double2 yv = y[e];
    for (int l = 0; l <= j; ++l)
      caxpy_sub<CPLX>(yv, __ldg(coef + 2 * l), CPLX ? __ldg(coef + 2 * l + 1) : 0.0,
                      Q[(size_t)l * ldq + e]);
    y[e] = yv;
    acc[0] = fma(yv.x, yv.x, acc[0]);
    if constexpr (CPLX) acc[0] = fma(yv.y, yv.y, acc[0]);
  }
  const double tot = block_multi_sum<1>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// out[2l + c] = sum over blocks of part[l][blk][c]: one warp per output, lanes
// striding over the blocks, then a shuffle sum (fixed order).
__global__ void dots_final_kernel(const double* part, int nblk, int j, double* out) {
  const int nl = j + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = warp; o < 2 * nl; o += nw) {
    const int l = o / 2, c = o % 2;
    double acc = 0.0;
    for (int b = lane; b < nblk; b += 32) acc += part[((size_t)l * nblk + b) * 2 + c];
    acc = warp_sum(acc);
    if (lane == 0) out[o] = acc;
  }
}

// beta_j = ||y|| from the norm partials (each block sums them in the same
// order; block 0 stores beta_j), then q_{j+1} = y / beta_j.
__global__ void lanczos_next_kernel(int64_t len, const double* __restrict__ y,
                                    const double* __restrict__ part, int nblk, double* beta, int j,
                                    double* qnext) {
  __shared__ double s_inv;
  if (threadIdx.x < 32) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 32) acc += part[k];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) {
      const double b = sqrt(acc);
      if (blockIdx.x == 0) beta[j] = b;
      s_inv = b > 0.0 ? 1.0 / b : 0.0;
    }
  }
  __syncthreads();
  const double inv = s_inv;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x)
    qnext[e] = y[e] * inv;
}

// ------------------------------------------------------------------ tridiagonal bounds
// Number of eigenvalues of the m x m symmetric tridiagonal T below x (Sturm count
// from the signs of the LDL^T pivots of T - x I).
__device__ int sturm_count(const double* al, const double* be, int m, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int j = 0; j < m; ++j) {
    const double b2 = j > 0 ? be[j - 1] * be[j - 1] : 0.0;
    d = (al[j] - x) - (j > 0 ? b2 / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// k-th smallest eigenvalue (0-based), by multisection with one warp: every
// lane evaluates the Sturm count at one of 32 interior points of the current
// bracket, which shrinks 33-fold per round, down to adjacent doubles.  All 32
// lanes of the calling warp must call it with the same arguments.
__device__ double multisect_eig(const double* al, const double* be, int m, int k, double lo,
                                double hi) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 64; ++it) {
    const double w = (hi - lo) / 33.0;
    const double x = lo + w * (double)(lane + 1);
    const bool above = sturm_count(al, be, m, x) > k;  // eigenvalue k lies below x
    const unsigned ball = __ballot_sync(0xffffffffu, above);
    const int first = ball ? __ffs(ball) - 1 : 32;      // first point above eigenvalue k
    const double nlo = first == 0 ? lo : lo + w * (double)first;
    const double nhi = first == 32 ? hi : lo + w * (double)(first + 1);
    if (!(nlo > lo || nhi < hi) || nhi - nlo <= 0.0) break;
    lo = nlo;
    hi = nhi;
    if (hi - lo <= 4.0 * fmax(fabs(lo), fabs(hi)) * 1.1102230246251565e-16) break;
  }
  return 0.5 * (lo + hi);
}

// |last component| of the normalised eigenvector of T for eigenvalue theta, by
// two steps of inverse iteration with a tridiagonal LU with partial pivoting.
__device__ double last_component(const double* al, const double* be, int m, double theta,
                                 double scale) {
  constexpr int MAXM = 256;
  double dl[MAXM], d[MAXM], du[MAXM], du2[MAXM], x[MAXM];
  int piv[MAXM];
  const double sh = theta + 1e-13 * scale;  // keep T - sh I nonsingular
  for (int j = 0; j < m; ++j) {
    d[j] = al[j] - sh;
    du[j] = j + 1 < m ? be[j] : 0.0;
    dl[j] = j + 1 < m ? be[j] : 0.0;
    du2[j] = 0.0;
    x[j] = 1.0;
  }
  // factorisation (row interchanges between j and j+1)
  for (int j = 0; j < m - 1; ++j) {
    if (fabs(d[j]) >= fabs(dl[j])) {
      piv[j] = 0;
      const double f = d[j] != 0.0 ? dl[j] / d[j] : 0.0;
      dl[j] = f;
      d[j + 1] -= f * du[j];
      du2[j] = 0.0;
    } else {
      piv[j] = 1;
      const double f = d[j] / dl[j];
      d[j] = dl[j];
      dl[j] = f;
      const double tmp = du[j];
      du[j] = d[j + 1];
      d[j + 1] = tmp - f * d[j + 1];
      if (j + 1 < m - 1) {
        du2[j] = du[j + 1];
        du[j + 1] = -f * du[j + 1];
      }
    }
  }
  if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
  for (int iter = 0; iter < 3; ++iter) {
    // forward: apply L^-1 P
    for (int j = 0; j < m - 1; ++j) {
      if (piv[j] == 0) {
        x[j + 1] -= dl[j] * x[j];
      } else {
        const double tmp = x[j];
        x[j] = x[j + 1];
        x[j + 1] = tmp - dl[j] * x[j];
      }
    }
    // back substitution with U (diagonal d, super du, super-super du2)
    for (int j = m - 1; j >= 0; --j) {
      double v = x[j];
      if (j + 1 < m) v -= du[j] * x[j + 1];
      if (j + 2 < m) v -= du2[j] * x[j + 2];
      x[j] = v / (d[j] != 0.0 ? d[j] : 1e-300);
    }
    double nrm = 0.0;
    for (int j = 0; j < m; ++j) nrm = fmax(nrm, fabs(x[j]));
    for (int j = 0; j < m; ++j) x[j] /= nrm;
  }
  double n2 = 0.0;
  for (int j = 0; j < m; ++j) n2 += x[j] * x[j];
  return fabs(x[m - 1]) / sqrt(n2);
}

// out = [emin, emax, a, b, theta_min, theta_max, beta_k, m].  Two warps:
// warp 0 finds theta_min, warp 1 theta_max (multisection), lane 0 of each
// its eigenvector's last component; thread 0 then combines.
__global__ void tridiag_bounds_kernel(const double* alpha, const double* beta, int kmax,
                                      const double* gersh, double pad_eps, double* out) {
  __shared__ double s_theta[2], s_last[2];
  __shared__ int s_m;
  __shared__ double s_bk, s_lo, s_hi;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double gmin = gersh[0], gmax = gersh[1];
  if (threadIdx.x == 0) {
    int m = kmax;
    for (int j = 0; j < kmax; ++j) {
      if (beta[j] <= 1e-12 * fmax(1.0, fabs(alpha[j]))) {
        m = j + 1;
        break;
      }
    }
    s_m = m;
    s_bk = m > 0 ? beta[m - 1] : 0.0;
    double lo = INFINITY, hi = -INFINITY;
    for (int j = 0; j < m; ++j) {
      const double r = (j > 0 ? fabs(beta[j - 1]) : 0.0) + (j + 1 < m ? fabs(beta[j]) : 0.0);
      lo = fmin(lo, alpha[j] - r);
      hi = fmax(hi, alpha[j] + r);
    }
    const double span = fmax(hi - lo, 1e-300);
    s_lo = lo - 1e-3 * span;
    s_hi = hi + 1e-3 * span;
  }
  __syncthreads();
  const int m = s_m;
  if (m > 0 && warp < 2) {
    const double th = multisect_eig(alpha, beta, m, warp == 0 ? 0 : m - 1, s_lo, s_hi);
    if (lane == 0) {
      s_theta[warp] = th;
      s_last[warp] = m > 1 ? last_component(alpha, beta, m, th, s_hi - s_lo) : 1.0;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double emin = gmin, emax = gmax, tmin = gmin, tmax = gmax;
  const double bk = s_bk;
  if (m > 0) {
    tmin = s_theta[0];
    tmax = s_theta[1];
    emin = fmax(gmin, tmin - bk * s_last[0]);
    emax = fmin(gmax, tmax + bk * s_last[1]);
  }
  out[0] = emin;
  out[1] = emax;
  out[2] = (emax - emin) / (2.0 - pad_eps);
  out[3] = 0.5 * (emax + emin);
  out[4] = tmin;
  out[5] = tmax;
  out[6] = bk;
  out[7] = (double)m;
}

// ------------------------------------------------------------------ DOS (Eq. (fKPM))
// coef[n] = c_n g_n mu_n with c_0 = 1, c_n = 2; Jackson g_n from the closed form.
// Damping factor g_n of the kernel: Jackson (review Eq. 71), Lorentz
// g_n = sinh(lambda (1 - n/M)) / sinh(lambda) (review Eq. 74), or 1.
__device__ __forceinline__ double damping(int n, int M, int kernel, double lambda, double cotq) {
  if (kernel == KPM_KERNEL_JACKSON) {
    double sn, cn;
    sincospi((double)n / (double)(M + 1), &sn, &cn);
    return ((double)(M - n + 1) * cn + sn * cotq) / (double)(M + 1);
  }
  if (kernel == KPM_KERNEL_LORENTZ) return sinh(lambda * (1.0 - (double)n / M)) / sinh(lambda);
  return 1.0;
}

// Block size of the kernels that evaluate an FP64 transcendental per element
// (damping coefficients, cosine table): one warp per block spreads them over
// as many SMs as there are warps of work (GB300 issues 2 FP64 FMA per SM per
// clock; a 256-thread block of cos/sin on one SM took about 12 us for M = 256).
constexpr int FP64_SPREAD = 32;

__global__ void dos_coef_kernel(const double* __restrict__ mu, int M, int kernel, double lambda,
                                double* coef) {
  const double q = M_PI / (double)(M + 1);
  const double cotq = cos(q) / sin(q);
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < M; n += gridDim.x * blockDim.x)
    coef[n] = (n == 0 ? 1.0 : 2.0) * damping(n, M, kernel, lambda, cotq) * (mu ? mu[n] : 1.0);
}

// table[j] = cos(pi j / (2K)), j = 0 .. 4K-1 (exact argument reduction for the DCT)
__global__ void cos_table_kernel(int K, double* table) {
  const int64_t n4 = 4LL * K;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n4;
       j += (int64_t)gridDim.x * blockDim.x)
    table[j] = cospi((double)j / (2.0 * (double)K));
}

// T lanes per node k (T a power of two <= 32): lane `sub` adds the terms
// n = sub, sub + T, ... with cos(pi n (2k+1)/(2K)) = table[n(2k+1) mod 4K]
// (the index advanced by T (2k+1) mod 4K), then an XOR butterfly over the T
// lanes.  The node's x_k = cos(pi (2k+1)/(2K)) = table[2k+1] and
// sin(pi (2k+1)/(2K)) = table[(2k+1+3K) mod 4K] come from the same table, so
// no FP64 transcendental is evaluated per node (GB300's FP64 pipe makes those
// the larger part of the kernel otherwise).
__global__ void dct_kernel(const double* __restrict__ coef, int M, double a, double b, int K,
                           const double* __restrict__ table, double* E, double* rho, int T) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t node = gt / T;
  const int sub = (int)(gt % T);
  const bool act = node < K;
  const int64_t n4 = 4LL * K;
  double acc = 0.0;
  if (act) {
    const int64_t step = 2 * node + 1;
    const int64_t dj = ((int64_t)T * step) % n4;
    int64_t j = ((int64_t)sub * step) % n4;
    for (int n = sub; n < M; n += T) {
      acc = fma(coef[n], table[j], acc);
      j += dj;
      if (j >= n4) j -= n4;
    }
  }
  for (int o = 1; o < T; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (act && sub == 0) {
    const int64_t jc = 2 * node + 1;
    const double cx = table[jc], sx = table[(jc + 3LL * K) % n4];
    E[node] = a * cx + b;
    rho[node] = acc / (M_PI * sx * a);
  }
}

// Local Green's function on the nodes (one warp per node k): with c_n the
// damped coefficients (factor 2 for n >= 1 included),
//   C_k = sum_n c_n cos(n theta_k),  S_k = sum_n c_n sin(n theta_k),
//   G(E_k + i0) = (-S_k - i C_k) / (a sin theta_k)   (Im G = -pi rho);
// sin(pi j / (2K)) = cos(pi (j - K) / (2K)) = table[(j + 3K) mod 4K].
__global__ void green_kernel(const double* __restrict__ coef, int M, double a, double b, int K,
                             const double* __restrict__ table, double* E, double* g_re,
                             double* g_im) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= K) return;
  const int64_t step = 2LL * warp + 1, n4 = 4LL * K, k3 = 3LL * K;
  double c = 0.0, sn = 0.0;
  for (int n = lane; n < M; n += 32) {
    const int64_t j = ((int64_t)n * step) % n4;
    c = fma(coef[n], table[j], c);
    sn = fma(coef[n], table[(j + k3) % n4], sn);
  }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    sn += __shfl_xor_sync(0xffffffffu, sn, o);
  }
  if (lane == 0) {
    double sx, cx;
    sincospi(((double)warp + 0.5) / (double)K, &sx, &cx);
    if (E) E[warp] = a * cx + b;
    g_re[warp] = -sn / (a * sx);
    g_im[warp] = -c / (a * sx);
  }
}

// Fermi-occupation integrals of the DOS on the K nodes, one CTA per inverse
// temperature beta[t] (Gauss-Chebyshev weights w_k = a pi sin(theta_k) / K):
// out[t] = (n, u, s, c) per site with f = 1/(1 + e^x), x = beta (E - mu_c):
//   n = sum w rho f,  u = sum w rho E f,
//   s = sum w rho [min(f, 1-f) |x| + log1p(e^-|x|)],  c = sum w rho x^2 f (1-f);
// beta = +inf is the ground state (f = step, s = c = 0).
__global__ void __launch_bounds__(LZ_BLOCK) thermo_kernel(const double* __restrict__ E,
                                                          const double* __restrict__ rho, int K,
                                                          double a, const double* __restrict__ beta,
                                                          double mu_c, double* out) {
  __shared__ double red[LZ_WARPS * 4];
  const double bt = beta[blockIdx.x];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < K; k += LZ_BLOCK) {
    double sx, cx;
    sincospi(((double)k + 0.5) / (double)K, &sx, &cx);
    const double wr = a * M_PI * sx / (double)K * rho[k];
    const double e = E[k], d = e - mu_c;
    double f, ent = 0.0, cv = 0.0;
    if (isinf(bt)) {
      f = d < 0.0 ? 1.0 : (d > 0.0 ? 0.0 : 0.5);
    } else {
      const double x = bt * d, ax = fabs(x), q = exp(-ax);  // q in (0, 1]
      f = x >= 0.0 ? q / (1.0 + q) : 1.0 / (1.0 + q);
      const double g = fmin(f, 1.0 - f);
      ent = g * ax + log1p(q);
      cv = x * x * f * (1.0 - f);
    }
    acc[0] = fma(wr, f, acc[0]);
    acc[1] = fma(wr * e, f, acc[1]);
    acc[2] = fma(wr, ent, acc[2]);
    acc[3] = fma(wr, cv, acc[3]);
  }
  const double tot = block_multi_sum<4>(acc, red);
  if (threadIdx.x < 4) out[(size_t)blockIdx.x * 4 + threadIdx.x] = tot;
}

// Mean and standard error over nvec vectors of each moment: pv[r * M + n].
__global__ void moment_stats_kernel(const double* __restrict__ pv, int nvec, int M, double* mean,
                                    double* err) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < M; n += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < nvec; ++r) s += pv[(size_t)r * M + n];
    const double m = s / nvec;
    double v = 0.0;
    for (int r = 0; r < nvec; ++r) {
      const double d = pv[(size_t)r * M + n] - m;
      v = fma(d, d, v);
    }
    if (mean) mean[n] = m;
    if (err) err[n] = nvec > 1 ? sqrt(v / ((double)(nvec - 1) * nvec)) : 0.0;
  }
}

// One CTA (LZ_BLOCK threads) per node k: the DOS of every vector's moments
// (Eq. (fKPM) with the damping in g, which carries the factor 2 of n >= 1),
// eight vectors at a time, kept in scratch[k * nvec + r]; then their mean and
// standard error (two passes).
__global__ void __launch_bounds__(LZ_BLOCK) dos_stats_kernel(
    const double* __restrict__ pv, const double* __restrict__ g, int nvec, int M, double a,
    double b, int K, const double* __restrict__ table, double* scratch, double* E, double* rmean,
    double* rerr) {
  __shared__ double red[LZ_WARPS * 8];
  __shared__ double s_mean;
  const int k = blockIdx.x;
  const int64_t step = 2LL * k + 1, n4 = 4LL * K;
  double sx, cx;
  sincospi(((double)k + 0.5) / (double)K, &sx, &cx);
  const double scale = 1.0 / (M_PI * sx) / a;
  double* rk = scratch + (size_t)k * nvec;
  for (int r0 = 0; r0 < nvec; r0 += 8) {
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    for (int n = threadIdx.x; n < M; n += LZ_BLOCK) {
      const double t = g[n] * table[((int64_t)n * step) % n4];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (r0 + i < nvec) acc[i] = fma(pv[(size_t)(r0 + i) * M + n], t, acc[i]);
    }
    const double tot = block_multi_sum<8>(acc, red);
    if ((int)threadIdx.x < 8 && r0 + (int)threadIdx.x < nvec) rk[r0 + threadIdx.x] = tot * scale;
    __syncthreads();
  }
  double v[1] = {0.0};
  for (int r = threadIdx.x; r < nvec; r += LZ_BLOCK) v[0] += rk[r];
  double tot = block_multi_sum<1>(v, red);
  if (threadIdx.x == 0) s_mean = tot / nvec;
  __syncthreads();
  const double m = s_mean;
  v[0] = 0.0;
  for (int r = threadIdx.x; r < nvec; r += LZ_BLOCK) {
    const double d = rk[r] - m;
    v[0] = fma(d, d, v[0]);
  }
  __syncthreads();
  tot = block_multi_sum<1>(v, red);
  if (threadIdx.x == 0) {
    if (E) E[k] = a * cx + b;
    if (rmean) rmean[k] = m;
    if (rerr) rerr[k] = nvec > 1 ? sqrt(tot / ((double)(nvec - 1) * nvec)) : 0.0;
  }
}

}  // namespace

// ================================================================== launchers
cudaError_t launch_prescale_stencil(bool fp32, bool cplx, int64_t n, int dims, const double* onsite,
                                    const double* hop, double t_re, double t_im,
                                    const RunParams* prm, bool lanczos, void* hs, void* ds,
                                    ScalarBlock* sc, cudaStream_t st) {
  const unsigned g = blocks_for(n, 256);
#define KPM_PS(T, C) \
  prescale_stencil_kernel<T, C><<<g, 256, 0, st>>>(n, dims, onsite, hop, t_re, t_im, prm, lanczos, \
                                                   (T*)hs, (T*)ds, sc)
  if (fp32) { if (cplx) KPM_PS(float, true); else KPM_PS(float, false); }
  else { if (cplx) KPM_PS(double, true); else KPM_PS(double, false); }
#undef KPM_PS
  return counted(cudaGetLastError());
}

// Padded-ELL copy of a CSR matrix already on the device: row i's entries in
// its W slots in CSR order, the remaining slots pointing at row i with value 0.
__global__ void ell_build_kernel(int64_t n, int W, int c, const int64_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col, const double* __restrict__ val,
                                 int32_t* __restrict__ ecol, double* __restrict__ eval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q0 = rowptr[i], q1 = rowptr[i + 1];
    for (int k = 0; k < W; ++k) {
      const int64_t q = q0 + k;
      const size_t o = (size_t)i * W + k;
      const bool in = q < q1;
      ecol[o] = in ? col[q] : (int32_t)i;
      for (int z = 0; z < c; ++z) eval[o * c + z] = in ? val[q * c + z] : 0.0;
    }
  }
}

cudaError_t launch_ell_build(int64_t n, int W, bool cplx, const int64_t* rowptr, const int32_t* col,
                             const double* val, int32_t* ecol, double* eval, cudaStream_t st) {
  const unsigned g = blocks_for(n, 256);
  ell_build_kernel<<<g, 256, 0, st>>>(n, W, cplx ? 2 : 1, rowptr, col, val, ecol, eval);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_prescale_csr(bool fp32, bool cplx, int64_t nnz, const double* val,
                                const RunParams* prm, bool lanczos, void* vals, ScalarBlock* sc,
                                cudaStream_t st) {
  const unsigned g = blocks_for((cplx ? 2 : 1) * nnz, 256);
#define KPM_PC(T, C) \
  prescale_csr_kernel<T, C><<<g, 256, 0, st>>>(nnz, val, prm, lanczos, (T*)vals, sc)
  if (fp32) { if (cplx) KPM_PC(float, true); else KPM_PC(float, false); }
  else { if (cplx) KPM_PC(double, true); else KPM_PC(double, false); }
#undef KPM_PC
  return counted(cudaGetLastError());
}

cudaError_t launch_rng_init(bool fp32, bool cplx, int64_t n, int Rp, const RunParams* prm, void* v0,
                            cudaStream_t st) {
  const unsigned g = blocks_for(n * Rp, 256);
  if (fp32) {
    if (cplx) rng_init_kernel<float, true><<<g, 256, 0, st>>>(n, Rp, prm, (float*)v0);
    else rng_init_kernel<float, false><<<g, 256, 0, st>>>(n, Rp, prm, (float*)v0);
  } else {
    if (cplx) rng_init_kernel<double, true><<<g, 256, 0, st>>>(n, Rp, prm, (double*)v0);
    else rng_init_kernel<double, false><<<g, 256, 0, st>>>(n, Rp, prm, (double*)v0);
  }
  return counted(cudaGetLastError());
}

cudaError_t launch_load_v0(bool fp32, bool cplx, int64_t n, int R, int Rp, const double* src,
                           void* v0, cudaStream_t st) {
  const unsigned g = blocks_for(n * Rp, 256);
  if (fp32) {
    if (cplx) load_v0_kernel<float, true><<<g, 256, 0, st>>>(n, R, Rp, src, (float*)v0);
    else load_v0_kernel<float, false><<<g, 256, 0, st>>>(n, R, Rp, src, (float*)v0);
  } else {
    if (cplx) load_v0_kernel<double, true><<<g, 256, 0, st>>>(n, R, Rp, src, (double*)v0);
    else load_v0_kernel<double, false><<<g, 256, 0, st>>>(n, R, Rp, src, (double*)v0);
  }
  return counted(cudaGetLastError());
}

cudaError_t launch_start_block(bool fp32, bool cplx, int kind, int64_t n, int R, int Rp,
                               const void* params, const StencilGeom& g, void* v0, cudaStream_t st) {
  const unsigned gr = blocks_for(n * Rp, 256);
  if (fp32) {
    if (cplx) start_block_kernel<float, true><<<gr, 256, 0, st>>>(kind, n, R, Rp, params, g, (float*)v0);
    else start_block_kernel<float, false><<<gr, 256, 0, st>>>(kind, n, R, Rp, params, g, (float*)v0);
  } else {
    if (cplx) start_block_kernel<double, true><<<gr, 256, 0, st>>>(kind, n, R, Rp, params, g, (double*)v0);
    else start_block_kernel<double, false><<<gr, 256, 0, st>>>(kind, n, R, Rp, params, g, (double*)v0);
  }
  return counted(cudaGetLastError());
}

cudaError_t launch_pair_sum(const double* pv, int npairs, int M, double* out, cudaStream_t st) {
  pair_sum_kernel<<<blocks_for((int64_t)npairs * M, 256), 256, 0, st>>>(pv, npairs, M, out);
  return counted(cudaGetLastError());
}

cudaError_t launch_reduce_ring(const double* ring, int ring_slots, int first_step, int count,
                               int nCTA, int Rp, const RunParams* prm, int steps_per_real,
                               double* sums, cudaStream_t st) {
  const dim3 grid((unsigned)count, (unsigned)((2 * Rp + 31) / 32));
  reduce_ring_kernel<<<grid, 256, 0, st>>>(ring, ring_slots, first_step, nCTA, Rp, prm,
                                           steps_per_real, sums);
  return counted(cudaGetLastError());
}

cudaError_t launch_advance_realisation(RunParams* prm, cudaStream_t st) {
  advance_realisation_kernel<<<1, 1, 0, st>>>(prm);
  return counted(cudaGetLastError());
}

cudaError_t launch_finalize(const double* sums, int S, int steps, int R, int Rp, int64_t n, int M,
                            double* per_vec, double* mu, RunParams* prm, cudaStream_t st) {
  const unsigned g = blocks_for((int64_t)S * R * steps, 256);
  finalize_pervec_kernel<<<g, 256, 0, st>>>(sums, S, steps, R, Rp, n, M, per_vec, prm);
  counted(cudaSuccess);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_mean_kernel<<<blocks_for(M, 128), 128, 0, st>>>(per_vec, S * R, M, mu);
  return counted(cudaGetLastError());
}

cudaError_t launch_gershgorin_stencil(bool cplx, int64_t n, const StencilGeom& g,
                                      const double* onsite, const double* hop, double t_re,
                                      double t_im, double* part_min, double* part_max, int nblk,
                                      cudaStream_t st) {
  gershgorin_stencil_kernel<<<nblk, 256, 0, st>>>(cplx, n, g, onsite, hop, t_re, t_im, part_min,
                                                  part_max);
  return counted(cudaGetLastError());
}

cudaError_t launch_gershgorin_csr(bool cplx, int64_t n, const int64_t* rowptr, const int32_t* col,
                                  const double* val, double* part_min, double* part_max, int nblk,
                                  cudaStream_t st) {
  gershgorin_csr_kernel<<<nblk, 256, 0, st>>>(cplx, n, rowptr, col, val, part_min, part_max);
  return counted(cudaGetLastError());
}

cudaError_t launch_minmax_final(const double* part_min, const double* part_max, int nblk,
                                double* out2, cudaStream_t st) {
  minmax_final_kernel<<<1, 32, 0, st>>>(part_min, part_max, nblk, out2);
  return counted(cudaGetLastError());
}

cudaError_t launch_lanczos_start(bool cplx, int64_t n, unsigned long long seed, double* q,
                                 cudaStream_t st) {
  // real: a zero pad column beside each value; complex: (re, 0)
  lanczos_start_kernel<<<blocks_for(2 * n, 256), 256, 0, st>>>(cplx, n, 2, seed, q);
  return counted(cudaGetLastError());
}

cudaError_t launch_lz_local_dots(bool cplx, int64_t n, const double* Q, int64_t ldq, int j,
                                const double* y, double* part_loc, int nblk, cudaStream_t st) {
  const double2* q = reinterpret_cast<const double2*>(Q);
  const double2* qj = q + (size_t)j * (ldq / 2);
  const double2* qm = j > 0 ? q + (size_t)(j - 1) * (ldq / 2) : nullptr;
  const double2* y2 = reinterpret_cast<const double2*>(y);
  if (cplx) lz_local_dots_kernel<true><<<nblk, LZ_BLOCK, 0, st>>>(n, qj, qm, y2, part_loc);
  else lz_local_dots_kernel<false><<<nblk, LZ_BLOCK, 0, st>>>(n, qj, qm, y2, part_loc);
  return counted(cudaGetLastError());
}

cudaError_t launch_lz_reorth_dots(bool cplx, int64_t n, const double* Q, int64_t ldq, int j,
                                  const double* part_loc, double* y, double* part, double* alpha,
                                  int nblk, cudaStream_t st) {
  const double2* q = reinterpret_cast<const double2*>(Q);
  double2* y2 = reinterpret_cast<double2*>(y);
  if (cplx)
    lz_reorth_dots_kernel<true><<<nblk, LZ_BLOCK, 0, st>>>(n, q, ldq / 2, j, part_loc, nblk, y2,
                                                            part, alpha);
  else
    lz_reorth_dots_kernel<false><<<nblk, LZ_BLOCK, 0, st>>>(n, q, ldq / 2, j, part_loc, nblk, y2,
                                                             part, alpha);
  return counted(cudaGetLastError());
}

cudaError_t launch_dots_final(const double* part, int nblk, int j, double* out, cudaStream_t st) {
  dots_final_kernel<<<1, 1024, 0, st>>>(part, nblk, j, out);
  return counted(cudaGetLastError());
}

cudaError_t launch_lz_update_norm(bool cplx, int64_t n, const double* Q, int64_t ldq, int j,
                                  const double* coef, double* y, double* part, int nblk,
                                  cudaStream_t st) {
  const double2* q = reinterpret_cast<const double2*>(Q);
  double2* y2 = reinterpret_cast<double2*>(y);
  if (cplx)
    lz_update_norm_kernel<true><<<nblk, LZ_BLOCK, 0, st>>>(n, q, ldq / 2, j, coef, y2, part);
  else
    lz_update_norm_kernel<false><<<nblk, LZ_BLOCK, 0, st>>>(n, q, ldq / 2, j, coef, y2, part);
  return counted(cudaGetLastError());
}

cudaError_t launch_lanczos_next(int64_t n, const double* y, const double* part, int nblk,
                                double* beta, int j, double* qnext, cudaStream_t st) {
  lanczos_next_kernel<<<blocks_for(2 * n, 256), 256, 0, st>>>(2 * n, y, part, nblk, beta, j, qnext);
  return counted(cudaGetLastError());
}

cudaError_t launch_tridiag_bounds(const double* alpha, const double* beta, int m,
                                  const double* gersh, double pad_eps, double* out,
                                  cudaStream_t st) {
  tridiag_bounds_kernel<<<1, 64, 0, st>>>(alpha, beta, m, gersh, pad_eps, out);
  return counted(cudaGetLastError());
}

cudaError_t launch_stats(const double* pv, int nvec, int M, double a, double b, int K, int kernel,
                         double lambda, double* mu_mean, double* mu_err, double* E, double* rmean,
                         double* rerr, double* work, cudaStream_t st) {
  // work: g[M], table[4K], scratch[K * nvec]
  double* g = work;
  double* table = work + M;
  double* scratch = table + 4 * (size_t)K;
  if (mu_mean || mu_err) {
    moment_stats_kernel<<<blocks_for(M, 256), 256, 0, st>>>(pv, nvec, M, mu_mean, mu_err);
    counted(cudaSuccess);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!E && !rmean && !rerr) return cudaSuccess;
  dos_coef_kernel<<<blocks_for(M, FP64_SPREAD), FP64_SPREAD, 0, st>>>(nullptr, M, kernel, lambda, g);
  counted(cudaSuccess);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cos_table_kernel<<<blocks_for(4LL * K, FP64_SPREAD), FP64_SPREAD, 0, st>>>(K, table);
  counted(cudaSuccess);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dos_stats_kernel<<<K, LZ_BLOCK, 0, st>>>(pv, g, nvec, M, a, b, K, table, scratch, E, rmean,
                                           rerr);
  return counted(cudaGetLastError());
}

cudaError_t launch_green(const double* mu, int M, double a, double b, int K, int kernel,
                         double lambda, double* E, double* g_re, double* g_im, double* work,
                         cudaStream_t st) {
  double* coef = work;
  double* table = work + M;
  dos_coef_kernel<<<blocks_for(M, FP64_SPREAD), FP64_SPREAD, 0, st>>>(mu, M, kernel, lambda, coef);
  counted(cudaSuccess);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cos_table_kernel<<<blocks_for(4LL * K, FP64_SPREAD), FP64_SPREAD, 0, st>>>(K, table);
  counted(cudaSuccess);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  green_kernel<<<blocks_for(32LL * K, 256), 256, 0, st>>>(coef, M, a, b, K, table, E, g_re, g_im);
  return counted(cudaGetLastError());
}

cudaError_t launch_thermo(const double* E, const double* rho, int K, double a,
                          const double* beta, int nT, double mu_c, double* out, cudaStream_t st) {
  thermo_kernel<<<nT, LZ_BLOCK, 0, st>>>(E, rho, K, a, beta, mu_c, out);
  return counted(cudaGetLastError());
}

cudaError_t launch_dos(const double* mu, int M, double a, double b, int K, int kernel,
                       double lambda, double* E, double* rho, double* work, cudaStream_t st) {
  double* coef = work;
  double* table = work + M;
  dos_coef_kernel<<<blocks_for(M, FP64_SPREAD), FP64_SPREAD, 0, st>>>(mu, M, kernel, lambda, coef);
  counted(cudaSuccess);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cos_table_kernel<<<blocks_for(4LL * K, FP64_SPREAD), FP64_SPREAD, 0, st>>>(K, table);
  counted(cudaSuccess);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // lanes per node: enough threads for about 4 warps per SM, at most a warp
  int T = 1;
  while (T < 32 && (int64_t)K * T < 19456) T *= 2;
  dct_kernel<<<blocks_for((int64_t)K * T, 256), 256, 0, st>>>(coef, M, a, b, K, table, E, rho, T);
  return counted(cudaGetLastError());
}

}  // namespace kpm
