// Operator selection for the batched persistent kernel (coherent vector loads).
#pragma once

#include "kpm_batch.cuh"
#include "kpm_step_dispatch.cuh"

namespace kpm {

template <class CH>
cudaError_t run_batch(const StepArgs& proto, BatchTask* tasks, int ntasks, int* queue, int grid,
                      int C, cudaStream_t st) {
  // stencil operators carry neither a row pointer nor column indices
  return visit_op<CH>(proto.rowptr == nullptr && proto.col == nullptr, proto, [&]<class OP>() {
    return launch_batch_one<CH, OP>(tasks, ntasks, queue, grid, C, proto.Gt, proto.Rp, st);
  });
}

template <class CH>
int clusters_batch(const StepArgs& proto, int C) {
  return visit_op<CH>(proto.rowptr == nullptr && proto.col == nullptr, proto, [&]<class OP>() {
    return batch_max_clusters<CH, OP>(C, proto.Gt, proto.Rp);
  });
}

}  // namespace kpm
