// FP32-vector instantiations of the fused Chebyshev step (stencil and CSR):
// 32-byte chunks, packed f32x2 arithmetic, FP64 moment sums.
#include "kpm_internal.h"
#include "kpm_step_dispatch.cuh"

namespace kpm {

cudaError_t launch_step_f32(bool stencil, bool cplx, StepMode mode, const StepArgs& a,
                            const LaunchCfg& cfg, cudaStream_t st) {
  if (mode == MODE_SPMV) return cudaErrorInvalidValue;  // the Lanczos product is FP64 only
  if (mode == MODE_STEP && !stencil && a.tma_stages > 0) return launch_ell_tma_f32(cplx, a, cfg, st);
  if (cplx)
    return mode == MODE_FIRST ? run_mode<ChunkF32<true>, MODE_FIRST>(stencil, a, cfg, st)
                              : run_mode<ChunkF32<true>, MODE_STEP>(stencil, a, cfg, st);
  return mode == MODE_FIRST ? run_mode<ChunkF32<false>, MODE_FIRST>(stencil, a, cfg, st)
                            : run_mode<ChunkF32<false>, MODE_STEP>(stencil, a, cfg, st);
}

int occ_step_f32(bool stencil, bool cplx, const StepArgs& a, int block) {
  return cplx ? occ_mode<ChunkF32<true>, MODE_STEP>(stencil, a, block)
              : occ_mode<ChunkF32<false>, MODE_STEP>(stencil, a, block);
}

}  // namespace kpm
