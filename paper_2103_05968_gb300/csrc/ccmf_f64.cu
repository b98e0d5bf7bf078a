// Explicit instantiation of the solver launch sequences for double fields.
#include "ccmf_launch.cuh"

namespace ccmf {
template cudaError_t configure_kernels<double>(const LaunchShape&);
template int pipe_blocks_per_sm<double>(int, size_t);
template void launch_init<double>(const Ctx<double>&, cudaStream_t);
template void launch_iteration<double>(const Ctx<double>&, cudaStream_t);
template void launch_iteration_range<double>(const Ctx<double>&, int, int, cudaStream_t);
template void launch_iteration_timed<double>(const Ctx<double>&, cudaStream_t, cudaEvent_t*);
template void launch_final<double>(const Ctx<double>&, cudaStream_t, double*, double*);
}  // namespace ccmf
