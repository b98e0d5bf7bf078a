// Explicit instantiation of the solver launch sequences for double fields.
#include "ccmf_launch.cuh"

namespace ccmf {
template cudaError_t configure_kernels<double>(const LaunchShape&);
template int pipe_blocks_per_sm<double>(int, size_t);
template int plane_cluster_capacity<double>(int, size_t);
template int lines_blocks_per_sm<double>(int, int, size_t);
template int wlines_blocks_per_sm<double>(int, int, size_t);
template int update_vec_blocks_per_sm<double>();
template int update_vec_half_blocks_per_sm<double>(int);
template int ab_blocks_per_sm<double>(int, size_t);
template void launch_init<double>(const Ctx<double>&, cudaStream_t);
template void launch_iteration<double>(const Ctx<double>&, cudaStream_t);
template void launch_iteration_range<double>(const Ctx<double>&, int, int, cudaStream_t);
template void launch_iteration_timed<double>(const Ctx<double>&, cudaStream_t, cudaEvent_t*);
template void launch_final<double>(const Ctx<double>&, cudaStream_t, double*, double*);
template void launch_adj_restore<double>(const Ctx<double>&, int, const double*, int, cudaStream_t);
template void launch_adj_seed<double>(const Ctx<double>&, double*, double*, SolveScalars*, cudaStream_t);
template void launch_adj_step<double>(const Ctx<double>&, const double*, double*, double*, double*, double*, double*, const double*, SolveScalars*, double*,
                                   const double*, int, int, cudaStream_t, const unsigned*);
template int batch_persist_blocks_per_sm<double>(int, size_t);
template void launch_batch_persist<double>(const PersistArgs<double>&, int, int, size_t, cudaStream_t);
}  // namespace ccmf
