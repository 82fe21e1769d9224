// Selects the operator specialisation of the fused step for one chunk policy.
#pragma once

#include "kpm_step.cuh"

namespace kpm {

template <class CH, class F>
auto visit_op(bool stencil, const StepArgs& a, F&& f) {
  if (!stencil) {
    switch (a.ell_w) {
      case 2: return f.template operator()<EllOp<CH, 2>>();
      case 4: return f.template operator()<EllOp<CH, 4>>();
      case 6: return f.template operator()<EllOp<CH, 6>>();
      case 8: return f.template operator()<EllOp<CH, 8>>();
      default: return f.template operator()<CsrOp<CH>>();
    }
  }
  const bool hh = a.hs != nullptr, hd = a.ds != nullptr;
#define KPM_CASE(D, H, S) \
  if (a.geom.dims == D && hh == H && hd == S) return f.template operator()<StencilOp<CH, D, H, S>>();
  KPM_CASE(3, true, false) KPM_CASE(3, true, true) KPM_CASE(3, false, false) KPM_CASE(3, false, true)
  KPM_CASE(2, true, false) KPM_CASE(2, true, true) KPM_CASE(2, false, false) KPM_CASE(2, false, true)
  KPM_CASE(1, true, false) KPM_CASE(1, true, true) KPM_CASE(1, false, false)
#undef KPM_CASE
  return f.template operator()<StencilOp<CH, 1, false, true>>();
}

template <class CH, int MODE>
cudaError_t run_mode(bool stencil, const StepArgs& a, const LaunchCfg& cfg, cudaStream_t st) {
  return visit_op<CH>(stencil, a, [&]<class OP>() { return launch_one<CH, MODE, OP>(a, cfg, st); });
}

template <class CH, int MODE>
int occ_mode(bool stencil, const StepArgs& a, int block) {
  return visit_op<CH>(stencil, a, [&]<class OP>() { return occupancy_one<CH, MODE, OP>(block, a.Gt); });
}

}  // namespace kpm
