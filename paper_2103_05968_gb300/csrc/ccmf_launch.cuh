// Host-side launch sequences of the solver passes (one instantiation per precision).
#pragma once

#include "ccmf_kernels.cuh"

namespace ccmf {

template <typename T>
struct Ctx {
    Geom g;
    Ptrs<T> p;
    LoopConfig cfg;
    AxisPlan ax[3];
    const cx<T>* tw[3];   // twiddle tables W_n^t, t < n, per axis
    const T* sym[3];      // 4 sin^2(pi k / N_a) per axis
    const double* xi_stage;  // [batch][3] unit normals (device)
    LaunchShape sh;
};

// Kernel classes of one loop iteration, in launch order.
enum KernelClass { kKDivRfftZ = 0, kKFftYFwd, kKFftXSolve, kKFftYInv, kKIrfftZ, kKUpdate, kNumKernelClasses };

inline const char* kernel_class_name(int c) {
    static const char* names[kNumKernelClasses] = {"k_div_rfft_z", "k_fft_y_fwd", "k_fft_x_solve",
                                                   "k_fft_y_inv", "k_irfft_z", "k_update"};
    return (c >= 0 && c < kNumKernelClasses) ? names[c] : "?";
}

template <typename T>
__global__ void k_setup(SolveScalars* sc, const double* __restrict__ xi, int batch) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    sc[s].xi[0] = xi[3 * s + 0];
    sc[s].xi[1] = xi[3 * s + 1];
    sc[s].xi[2] = xi[3 * s + 2];
    sc[s].counter = 0;
    sc[s].active = 0;
}

template <typename T>
cudaError_t configure_kernels(const LaunchShape& sh) {
    cudaError_t err = cudaSuccess;
    auto set = [&](const void* f, size_t bytes) {
        if (err == cudaSuccess && bytes > 48 * 1024)
            err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void*)k_div_rfft_z<T>, sh.smem_z);
    set((const void*)k_irfft_z<T>, sh.smem_z);
    set((const void*)k_fft_strided<T, 0>, sh.smem_y);
    set((const void*)k_fft_strided<T, 2>, sh.smem_y);
    set((const void*)k_fft_strided<T, 1>, sh.smem_x);
    return err;
}

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

template <typename T>
void launch_init(const Ctx<T>& c, cudaStream_t st) {
    k_setup<T><<<(unsigned)ceil_div(c.g.batch, 128), 128, 0, st>>>(c.p.sc, c.xi_stage, c.g.batch);
    dim3 grid((unsigned)c.sh.grid_update, (unsigned)c.g.batch);
    k_init_stats<T><<<grid, kThreads, 0, st>>>(c.g, c.p, c.cfg);
    if (!c.cfg.resume) k_init_state<T><<<grid, kThreads, 0, st>>>(c.g, c.p);
}

// Enqueue one ADMM iteration (or, with p.run_all and OUT, the final evaluation).
// `between` is called after every kernel with its class (used to record events).
template <typename T, bool OUT, typename F>
void launch_passes(const Ctx<T>& c, const Ptrs<T>& p, cudaStream_t st, F&& between) {
    const Geom& g = c.g;
    const LaunchShape& sh = c.sh;
    const long long pairs = ceil_div((long long)g.n1 * g.n2, 2);
    dim3 gz((unsigned)ceil_div(pairs, sh.pairs_per_block), (unsigned)g.batch);
    dim3 gy((unsigned)ceil_div((long long)g.n1 * g.n3h, sh.lpb_y), (unsigned)g.batch);
    dim3 gx((unsigned)ceil_div((long long)g.n2 * g.n3h, sh.lpb_x), (unsigned)g.batch);
    dim3 gu((unsigned)sh.grid_update, (unsigned)g.batch);
    const T inv_n = (T)(1.0 / (double)g.N);
    k_div_rfft_z<T><<<gz, kThreads, sh.smem_z, st>>>(g, p, c.ax[2], c.tw[2], sh.pairs_per_block);
    between(kKDivRfftZ);
    k_fft_strided<T, 0><<<gy, kThreads, sh.smem_y, st>>>(g, p, c.ax[1], c.tw[1], sh.lpb_y, c.sym[0], c.sym[1],
                                                         c.sym[2], inv_n);
    between(kKFftYFwd);
    k_fft_strided<T, 1><<<gx, kThreads, sh.smem_x, st>>>(g, p, c.ax[0], c.tw[0], sh.lpb_x, c.sym[0], c.sym[1],
                                                         c.sym[2], inv_n);
    between(kKFftXSolve);
    k_fft_strided<T, 2><<<gy, kThreads, sh.smem_y, st>>>(g, p, c.ax[1], c.tw[1], sh.lpb_y, c.sym[0], c.sym[1],
                                                         c.sym[2], inv_n);
    between(kKFftYInv);
    k_irfft_z<T><<<gz, kThreads, sh.smem_z, st>>>(g, p, c.ax[2], c.tw[2], sh.pairs_per_block);
    between(kKIrfftZ);
    k_update<T, OUT><<<gu, kThreads, 0, st>>>(g, p, c.cfg);
    between(kKUpdate);
}

struct NoHook {
    void operator()(int) const {}
};

template <typename T>
void launch_iteration(const Ctx<T>& c, cudaStream_t st) {
    launch_passes<T, false>(c, c.p, st, NoHook());
}

template <typename T>
void launch_iteration_timed(const Ctx<T>& c, cudaStream_t st, cudaEvent_t* ev) {
    int idx = 0;
    launch_passes<T, false>(c, c.p, st, [&](int) {
        cudaEventRecordWithFlags(ev[++idx], st, cudaEventRecordExternal);
    });
}

template <typename T>
void launch_final(const Ctx<T>& c, cudaStream_t st, T* cut, T* flow) {
    Ptrs<T> p = c.p;
    p.run_all = 1;
    p.cut = cut;
    p.flow = flow;
    launch_passes<T, true>(c, p, st, NoHook());
}

}  // namespace ccmf
