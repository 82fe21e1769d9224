// FP64 instantiations of the staged batched kernel (stencil operators).
#include "kpm_batch_stg.cuh"
#include "kpm_step_dispatch.cuh"

namespace kpm {
namespace {

template <class CH>
cudaError_t run_stg(const StepArgs& proto, BatchTask* tasks, int ntasks, int* queue, int grid,
                    int C, int Tl, int Sl, int SWl, cudaStream_t st) {
  if (proto.rowptr != nullptr || proto.col != nullptr) return cudaErrorNotSupported;
  return visit_op<CH>(true, proto, [&]<class OP>() {
    return launch_batch_stg_one<CH, OP>(tasks, ntasks, queue, grid, C, proto.G, proto.Rp, Tl, Sl,
                                        SWl, st);
  });
}

template <class CH>
int clusters_stg(const StepArgs& proto, int C, int Tl, int Sl, int SWl) {
  if (proto.rowptr != nullptr || proto.col != nullptr) return 0;
  return visit_op<CH>(true, proto, [&]<class OP>() {
    return batch_stg_max_clusters<CH, OP>(C, proto.G, proto.Rp, Tl, Sl, SWl);
  });
}

}  // namespace

cudaError_t launch_batch_stg_f64(bool cplx, const StepArgs& proto, BatchTask* tasks, int ntasks,
                                 int* queue, int grid, int C, int Tl, int Sl, int SWl,
                                 cudaStream_t st) {
  return cplx ? run_stg<ChunkF64<true, false>>(proto, tasks, ntasks, queue, grid, C, Tl, Sl, SWl, st)
              : run_stg<ChunkF64<false, false>>(proto, tasks, ntasks, queue, grid, C, Tl, Sl, SWl, st);
}

int max_clusters_batch_stg_f64(bool cplx, const StepArgs& proto, int C, int Tl, int Sl, int SWl) {
  return cplx ? clusters_stg<ChunkF64<true, false>>(proto, C, Tl, Sl, SWl)
              : clusters_stg<ChunkF64<false, false>>(proto, C, Tl, Sl, SWl);
}

}  // namespace kpm
