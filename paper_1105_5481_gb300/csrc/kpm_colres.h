// Column-resident solve (kpm_colres.cu): every product of one realisation of
// a small stencil operator in a single cluster launch, the vector columns
// split among independent clusters and held in their shared memory.
#pragma once

#include "kpm_internal.h"

namespace kpm {

// Largest (row, column) element count per CTA: one element per thread of a
// CTA of at most 1024 threads.
constexpr int64_t COLRES_MAX_ELEMS = 1024;
// Shared-memory buffer of the bulk dot sums (two batches of per-thread
// terms): the exact-cover shape of small CTAs fits the first, larger CTAs
// take batches of up to the second.
constexpr size_t COLRES_BULK_SMALL = 32 * 1024;
constexpr size_t COLRES_BULK_BYTES = 160 * 1024;
// Shared-memory ring of per-product CTA partials (flushed to the global
// scratch when full).
constexpr size_t COLRES_RING_BYTES = 16 * 1024;
// Dynamic shared memory a CTA may take (the two vector blocks, the warp
// partials, the ring and the bulk buffer), within the 227 KB of an SM.
constexpr size_t COLRES_MAX_SMEM = 220 * 1024;

struct ColresArgs {
  void* vg[2];               // the N x Rp vector blocks in global memory (library layout)
  const ScalarBlock* sc;     // scaled uniform hopping and diagonal
  const void* hs;            // scaled per-bond hoppings [N][dims], or NULL (uniform)
  const void* ds;            // scaled diagonal [N], or NULL (uniform)
  StencilGeom geom;
  const int32_t* ecol;       // padded ELL [N][W] column indices (W > 0)
  const void* evals;         // padded ELL [N][W] scaled values (T or complex T)
  const RunParams* prm;      // seed, realisation s, s0, R
  double* sums;              // [S][steps][2][Rp]: the per-step sums over rows
  double* gp;                // scratch: [groups][C][n1 - n0][2][cpc] CTA partials
  int64_t n;
  int Rp, R;
  int64_t P;
  int cpc;
  int n0, n1;                // products n0 .. n1-1 (product n reads v_n, writes v_{n+1})
  int steps;                 // products per realisation (row stride of sums)
  int gen;                   // n0 == 0: 1 draws v_0 in the kernel, 0 loads it from vg[0];
                             // n0 > 0 loads v_{n0} from vg[n0 & 1], v_{n0-1} from the other
  int kr;                    // products in the shared-memory ring of CTA partials
  int bulk_k;                // > 0: products per batch of the bulk dot sums; 0: shuffle tree
  int bulk_tps;              // lanes per sum of the bulk dot sums
};

// Bytes of the two vector blocks, rounded up to 16 (the warp partials follow).
__host__ __device__ inline size_t colres_head_bytes(size_t vec_bytes) {
  return (vec_bytes + 15) / 16 * 16;
}

// The plan for an N-row operator (a stencil of `dims` dimensions, ell_w = 0,
// or a padded ELL of width ell_w in {2, 4, 6, 8}) and R columns:
// the cluster shape (every column group resident at once, at most
// COLRES_MAX_ELEMS elements per CTA) of least estimated time per product, or
// false if none is estimated faster than the chain of step launches.
// KPM_COLRES="0" turns the form off; KPM_COLRES="C,cpc" forces a shape (which
// may then take several waves); KPM_COLRES_TREE set forces the shuffle tree.
bool colres_plan(int64_t n, int dims, int ell_w, bool cplx, bool fp32, int R, ColresPlan* out);
// Doubles of the partial scratch for a launch of nprod products.
size_t colres_partial_doubles(const ColresPlan& pl, int nprod);
// dims is that of the stencil (unused for a padded-ELL plan, pl.ell_w > 0)
cudaError_t launch_colres(bool fp32, bool cplx, int dims, const ColresPlan& pl,
                          const ColresArgs& a, cudaStream_t st);

}  // namespace kpm
