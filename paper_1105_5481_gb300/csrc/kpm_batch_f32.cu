// FP32-vector instantiations of the batched persistent kernel.
#include "kpm_batch_dispatch.cuh"

namespace kpm {

cudaError_t launch_batch_f32(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                             int* queue, int grid, int C, cudaStream_t st) {
  return cplx ? run_batch<ChunkF32<true, false>>(proto, tasks, ntasks, queue, grid, C, st)
              : run_batch<ChunkF32<false, false>>(proto, tasks, ntasks, queue, grid, C, st);
}

int max_clusters_batch_f32(bool cplx, const StepArgs& proto, int C) {
  return cplx ? clusters_batch<ChunkF32<true, false>>(proto, C)
              : clusters_batch<ChunkF32<false, false>>(proto, C);
}

// 16-byte chunks (real field, stencil operators): twice the threads per row
cudaError_t launch_batch_f32h(const StepArgs& proto, BatchTask* tasks, int ntasks, int* queue,
                              int grid, int C, cudaStream_t st) {
  return run_batch_stencil<ChunkF32h<false>>(proto, tasks, ntasks, queue, grid, C, st);
}

int max_clusters_batch_f32h(const StepArgs& proto, int C) {
  return clusters_batch_stencil<ChunkF32h<false>>(proto, C);
}

cudaError_t launch_batch_res_f32(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                                 int* queue, int grid, int C, int64_t rows_cap, cudaStream_t st) {
  return cplx ? run_batch_res<ChunkF32<true, false>>(proto, tasks, ntasks, queue, grid, C, rows_cap, st)
              : run_batch_res<ChunkF32<false, false>>(proto, tasks, ntasks, queue, grid, C, rows_cap, st);
}

int max_clusters_batch_res_f32(bool cplx, const StepArgs& proto, int C, int64_t rows_cap) {
  return cplx ? clusters_batch_res<ChunkF32<true, false>>(proto, C, rows_cap)
              : clusters_batch_res<ChunkF32<false, false>>(proto, C, rows_cap);
}

}  // namespace kpm
