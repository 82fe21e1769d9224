// Operator selection for the batched persistent kernel (coherent vector loads).
#pragma once

#include "kpm_batch.cuh"
#include "kpm_batch_res.cuh"
#include "kpm_chunk16.cuh"
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

// Stencil operators only (the 16-byte chunk's threads-per-row choice).
template <class CH>
cudaError_t run_batch_stencil(const StepArgs& proto, BatchTask* tasks, int ntasks, int* queue,
                              int grid, int C, cudaStream_t st) {
  if (proto.rowptr != nullptr || proto.col != nullptr) return cudaErrorNotSupported;
  return visit_op<CH>(true, proto, [&]<class OP>() -> cudaError_t {
    if constexpr (ResStencil<OP>::value)
      return launch_batch_one<CH, OP>(tasks, ntasks, queue, grid, C, proto.Gt, proto.Rp, st);
    else
      return cudaErrorNotSupported;
  });
}

template <class CH>
int clusters_batch_stencil(const StepArgs& proto, int C) {
  if (proto.rowptr != nullptr || proto.col != nullptr) return 0;
  return visit_op<CH>(true, proto, [&]<class OP>() -> int {
    if constexpr (ResStencil<OP>::value)
      return batch_max_clusters<CH, OP>(C, proto.Gt, proto.Rp);
    else
      return 0;
  });
}

// The cluster-resident form: stencil operators only.
template <class CH>
cudaError_t run_batch_res(const StepArgs& proto, BatchTask* tasks, int ntasks, int* queue, int grid,
                          int C, int64_t rows_cap, cudaStream_t st) {
  if (proto.rowptr != nullptr || proto.col != nullptr) return cudaErrorNotSupported;
  return visit_op<CH>(true, proto, [&]<class OP>() {
    return launch_batch_res_one<CH, OP>(tasks, ntasks, queue, grid, C, proto.G, proto.Rp,
                                        rows_cap, st);
  });
}

template <class CH>
int clusters_batch_res(const StepArgs& proto, int C, int64_t rows_cap) {
  if (proto.rowptr != nullptr || proto.col != nullptr) return 0;
  return visit_op<CH>(true, proto, [&]<class OP>() {
    return batch_res_max_clusters<CH, OP>(C, proto.G, proto.Rp, rows_cap);
  });
}

}  // namespace kpm
