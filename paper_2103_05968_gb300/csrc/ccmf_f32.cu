// Explicit instantiation of the solver launch sequences for float fields.
#include "ccmf_launch.cuh"

namespace ccmf {
template cudaError_t configure_kernels<float>(const LaunchShape&);
template int pipe_blocks_per_sm<float>(int, size_t);
template int plane_cluster_capacity<float>(int, size_t);
template int lines_blocks_per_sm<float>(int, int, size_t);
template int wlines_blocks_per_sm<float>(int, int, size_t);
template int update_vec_blocks_per_sm<float>();
template int update_vec_half_blocks_per_sm<float>(int);
template int ab_blocks_per_sm<float>(int, size_t);
template void launch_init<float>(const Ctx<float>&, cudaStream_t);
template void launch_iteration<float>(const Ctx<float>&, cudaStream_t);
template void launch_iteration_range<float>(const Ctx<float>&, int, int, cudaStream_t);
template void launch_iteration_timed<float>(const Ctx<float>&, cudaStream_t, cudaEvent_t*);
template void launch_final<float>(const Ctx<float>&, cudaStream_t, float*, float*);
template void launch_adj_restore<float>(const Ctx<float>&, int, const double*, int, cudaStream_t);
template void launch_adj_seed<float>(const Ctx<float>&, float*, float*, SolveScalars*, cudaStream_t);
template void launch_adj_step<float>(const Ctx<float>&, const float*, float*, float*, float*, float*, float*, const float*, SolveScalars*, float*,
                                   const double*, int, int, cudaStream_t, const unsigned*);
template int batch_persist_blocks_per_sm<float>(int, size_t);
template void launch_batch_persist<float>(const PersistArgs<float>&, int, int, size_t, cudaStream_t);
template int wx_tma_blocks_per_sm<float>();
}  // namespace ccmf
