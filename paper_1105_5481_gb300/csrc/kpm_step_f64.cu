// FP64 instantiations of the fused Chebyshev step (stencil and CSR) and of
// the plain FP64 product used by the Lanczos bound estimate.
#include "kpm_step_dispatch.cuh"

namespace kpm {

cudaError_t launch_step_f64(bool stencil, bool cplx, StepMode mode, const StepArgs& a,
                            const LaunchCfg& cfg, cudaStream_t st) {
  if (cplx) {
    switch (mode) {
      case MODE_FIRST: return run_mode<ChunkF64<true>, MODE_FIRST>(stencil, a, cfg, st);
      case MODE_STEP: return run_mode<ChunkF64<true>, MODE_STEP>(stencil, a, cfg, st);
      default: return run_mode<ChunkF64<true>, MODE_SPMV>(stencil, a, cfg, st);
    }
  }
  switch (mode) {
    case MODE_FIRST: return run_mode<ChunkF64<false>, MODE_FIRST>(stencil, a, cfg, st);
    case MODE_STEP: return run_mode<ChunkF64<false>, MODE_STEP>(stencil, a, cfg, st);
    default: return run_mode<ChunkF64<false>, MODE_SPMV>(stencil, a, cfg, st);
  }
}

int occ_step_f64(bool stencil, bool cplx, const StepArgs& a, int block) {
  return cplx ? occ_mode<ChunkF64<true>, MODE_STEP>(stencil, a, block)
              : occ_mode<ChunkF64<false>, MODE_STEP>(stencil, a, block);
}

}  // namespace kpm
