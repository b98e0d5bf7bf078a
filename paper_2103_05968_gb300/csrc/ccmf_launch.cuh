// Host-side launch sequences of the solver passes (one instantiation per precision).
#pragma once

#include "ccmf_kernels.cuh"
#include "ccmf_persist.cuh"
#include "ccmf_tma_x.cuh"

namespace ccmf {

// Raise a kernel's dynamic shared memory limit to at least `bytes`. The limit is a
// property of the kernel, shared by every plan in the process, so it is only ever
// raised: a plan with smaller tiles must not lower what another plan's launches need.
inline cudaError_t raise_smem_limit(const void* f, size_t bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, f);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
struct Ctx {
    Geom g;
    Ptrs<T> p;
    LoopConfig cfg;
    AxisPlan ax[3];
    const cx<T>* tw[3];   // twiddle tables W_n^t, t < n, per axis
    const T* sym[3];      // 4 sin^2(pi k / N_a) per axis
    const T* rsym[2];     // the x and y tables in digit-reversed order (fused plane pass)
    const double* xi_stage;  // [batch][3] unit normals (device)
    LaunchShape sh;
    bool vec_div;         // 16-byte path of the divergence pass (N3 % W == 0)
    bool vec_update;      // 16-byte path of the update pass (also needs gamma 16-byte aligned)
    bool use_ab;          // stored-divergence schedule: update variants 8 .. 10 write a, b; the first pass reads them
};

// Kernel classes of one loop iteration.
enum KernelClass {
    kKDivRfftZ = 0, kKFftYFwd, kKFftXSolve, kKFftYInv, kKFftPlane, kKIrfftZ, kKUpdate, kNumKernelClasses
};

inline const char* kernel_class_name(int c) {
    static const char* names[kNumKernelClasses] = {"k_div_rfft_z", "k_fft_y_fwd", "k_fft_x_solve", "k_fft_y_inv",
                                                   "k_fft_plane", "k_irfft_z", "k_update"};
    return (c >= 0 && c < kNumKernelClasses) ? names[c] : "?";
}

// The kernel classes one iteration launches, in order; returns their number.
inline int iteration_classes(const LaunchShape& sh, int* cls) {
    int n = 0;
    cls[n++] = kKDivRfftZ;
    if (sh.plane_fused) {
        cls[n++] = kKFftPlane;
    } else {
        cls[n++] = kKFftYFwd;
        cls[n++] = kKFftXSolve;
        cls[n++] = kKFftYInv;
    }
    cls[n++] = kKIrfftZ;
    cls[n++] = kKUpdate;
    return n;
}

template <typename T>
__global__ void k_setup(SolveScalars* sc, const double* __restrict__ xi, int batch) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    sc[s].xi[0] = xi[3 * s + 0];
    sc[s].xi[1] = xi[3 * s + 1];
    sc[s].xi[2] = xi[3 * s + 2];
    sc[s].counter = 0;
    sc[s].chunk = 0;
    sc[s].active = 0;
}

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// Runs the statement list with the compile-time constant LN equal to the runtime
// line count L (a power of two <= 16).
#define CCMF_DISPATCH_LINES(L, ...)                              \
    switch (L) {                                                 \
        case 16: { constexpr int LN = 16; __VA_ARGS__; } break; \
        case 8: { constexpr int LN = 8; __VA_ARGS__; } break;   \
        case 4: { constexpr int LN = 4; __VA_ARGS__; } break;   \
        case 2: { constexpr int LN = 2; __VA_ARGS__; } break;   \
        default: { constexpr int LN = 1; __VA_ARGS__; } break;  \
    }

// Runs the statement list with the compile-time line length NN equal to the runtime
// power of two n (128 ... 1024, the warp-per-line passes).
#define CCMF_DISPATCH_N(n, ...)                                   \
    switch (n) {                                                  \
        case 128: { constexpr int NN = 128; __VA_ARGS__; } break;  \
        case 256: { constexpr int NN = 256; __VA_ARGS__; } break;  \
        case 512: { constexpr int NN = 512; __VA_ARGS__; } break;  \
        default: { constexpr int NN = 1024; __VA_ARGS__; } break;  \
    }

// Runs the statement list with the compile-time stored-divergence variant AV (8, 9, 10).
#define CCMF_DISPATCH_AB(VAR, ...)                                 \
    switch (VAR) {                                                 \
        case 8: { constexpr int AV = 8; __VA_ARGS__; } break;      \
        case 9: { constexpr int AV = 9; __VA_ARGS__; } break;      \
        default: { constexpr int AV = 10; __VA_ARGS__; } break;    \
    }

// Runs the statement list with compile-time ST (stages) and NTH (threads) of a
// pipelined update variant 2..7.
#define CCMF_DISPATCH_PIPE(VAR, ...)                                                 \
    switch (VAR) {                                                                   \
        case 2: { constexpr int NTH = 256, ST = 2; __VA_ARGS__; } break;            \
        case 3: { constexpr int NTH = 128, ST = 3; __VA_ARGS__; } break;            \
        case 4: { constexpr int NTH = 128, ST = 4; __VA_ARGS__; } break;            \
        case 5: { constexpr int NTH = 256, ST = 3; __VA_ARGS__; } break;            \
        case 6: { constexpr int NTH = 128, ST = 2; __VA_ARGS__; } break;            \
        default: { constexpr int NTH = 64, ST = 3; __VA_ARGS__; } break;            \
    }

// Blocks per SM of a pipelined update variant (occupancy API), 0 on error.
template <typename T>
int pipe_blocks_per_sm(int variant, size_t smem) {
    int nb = 0;
    cudaError_t err = cudaSuccess;
    CCMF_DISPATCH_PIPE(variant, {
        err = raise_smem_limit((const void*)k_update_pipe<T, 0, ST, NTH>, smem);
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_update_pipe<T, 0, ST, NTH>, NTH, smem);
    });
    return err == cudaSuccess ? nb : 0;
}

// Cluster plane pass: launch with a cluster of CL blocks per plane (CL = 2, 4, 8, 16).
template <typename T, int CL>
cudaError_t launch_plane_cluster_t(const Geom& g, const Ptrs<T>& p, const Ctx<T>& c, T inv_n, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g.n3h * CL), (unsigned)g.batch);
    cfg.blockDim = dim3(kPlaneClusterThreads);
    cfg.dynamicSmemBytes = c.sh.smem_plane;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fft_plane_cluster<T, CL>, g, p, c.ax[0], c.ax[1], c.tw[0], c.tw[1],
                              c.rsym[0], c.rsym[1], c.sym[2], inv_n, c.sh.div_r1, c.sh.div_r2);
}

template <typename T>
cudaError_t launch_plane_cluster(const Geom& g, const Ptrs<T>& p, const Ctx<T>& c, T inv_n, cudaStream_t st) {
    switch (c.sh.plane_cluster) {
        case 2: return launch_plane_cluster_t<T, 2>(g, p, c, inv_n, st);
        case 4: return launch_plane_cluster_t<T, 4>(g, p, c, inv_n, st);
        case 8: return launch_plane_cluster_t<T, 8>(g, p, c, inv_n, st);
        default: return launch_plane_cluster_t<T, 16>(g, p, c, inv_n, st);
    }
}

// Blocks per SM of a y / x line pass with L lines per tile (occupancy API), 0 on error.
template <typename T>
int lines_blocks_per_sm(int mode, int lines, size_t smem) {
    int nb = 0;
    cudaError_t err = cudaSuccess;
    CCMF_DISPATCH_LINES(lines, {
        const void* f = mode == 0 ? (const void*)k_fft_lines<T, 0, LN>
                                  : mode == 1 ? (const void*)k_fft_lines<T, 1, LN> : (const void*)k_fft_lines<T, 2, LN>;
        err = raise_smem_limit(f, smem);
        if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, smem);
    });
    if (err != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// Resident blocks per SM of the vector update pass (the smaller of the advancing and
// the final-evaluation kernels), at least 1.
template <typename T>
int update_vec_blocks_per_sm() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_update_vec<T, false>, kThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update_vec<T, true>, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const int m = a < b ? a : b;
    return m < 1 ? 1 : m;
}

// Update variant 11: the vector update pass with half the voxels per thread, two blocks per SM.
template <typename T>
constexpr int kVecHalfW = Vec16<T>::W / 2;

#define CCMF_DISPATCH_ABW(var, ...)                                                      \
    do {                                                                                 \
        if ((var) == 13) {                                                               \
            using AW = AbwVariant<T, 13>;                                                \
            __VA_ARGS__;                                                                 \
        } else if ((var) == 14) {                                                        \
            using AW = AbwVariant<T, 14>;                                                \
            __VA_ARGS__;                                                                 \
        } else {                                                                         \
            using AW = AbwVariant<T, 15>;                                                \
            __VA_ARGS__;                                                                 \
        }                                                                                \
    } while (0)

// Resident blocks per SM of update variant 11 (12: the same vectors, three blocks per SM), at
// least 1.
template <typename T>
int update_vec_half_blocks_per_sm(int variant) {
    int a = 0;
    const cudaError_t e =
        variant == 12
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_update_vec<T, false, kVecHalfW<T>, 3>, kThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_update_vec<T, false, kVecHalfW<T>, 2>, kThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return a < 1 ? 1 : a;
}

// Blocks per SM of a warp-per-line pass of length n (power of two 128 ... 1024), 0 on error.
template <typename T>
int wlines_blocks_per_sm(int mode, int n, size_t smem) {
    int nb = 0;
    cudaError_t err = cudaSuccess;
    CCMF_DISPATCH_N(n, {
        const void* f = mode == 0 ? (const void*)k_fft_wlines<T, 0, NN>
                                  : mode == 1 ? (const void*)k_fft_wlines<T, 1, NN> : (const void*)k_fft_wlines<T, 2, NN>;
        err = raise_smem_limit(f, smem);
        if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, smem);
    });
    if (err != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// Blocks per SM of the TMA-staged x pass (FP32 only), 0 on error.
template <typename T>
int wx_tma_blocks_per_sm() {
    if constexpr (sizeof(T) != 4) {
        return 0;
    } else {
        int nb = 0;
        cudaError_t err = raise_smem_limit((const void*)k_fft_wx_tma<kTmaXN>, kTmaXSmem);
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fft_wx_tma<kTmaXN>, kThreads, kTmaXSmem);
        if (err != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nb;
    }
}

// Sets the launch attributes of the cluster plane pass and returns how many of its
// clusters can be resident at once (0: this cluster size cannot be launched).
template <typename T, int CL>
int plane_cluster_capacity_t(size_t smem) {
    const void* f = (const void*)k_fft_plane_cluster<T, CL>;
    if (raise_smem_limit(f, smem) != cudaSuccess ||
        (CL > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL * 16);
    cfg.blockDim = dim3(kPlaneClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <typename T>
int plane_cluster_capacity(int cl, size_t smem) {
    switch (cl) {
        case 2: return plane_cluster_capacity_t<T, 2>(smem);
        case 4: return plane_cluster_capacity_t<T, 4>(smem);
        case 8: return plane_cluster_capacity_t<T, 8>(smem);
        case 16: return plane_cluster_capacity_t<T, 16>(smem);
        default: return 0;
    }
}

template <typename T>
cudaError_t configure_kernels(const LaunchShape& sh) {
    cudaError_t err = cudaSuccess;
    auto set = [&](const void* f, size_t bytes) {
        if (err == cudaSuccess && bytes > 48 * 1024)
            err = raise_smem_limit(f, bytes);
    };
    CCMF_DISPATCH_LINES(sh.pairs_per_block, {
        set((const void*)k_div_rfft_z<T, LN, true, false>, sh.smem_z);
        set((const void*)k_div_rfft_z<T, LN, false, false>, sh.smem_z);
        set((const void*)k_div_rfft_z<T, LN, true, true>, sh.smem_z);
    });
    CCMF_DISPATCH_LINES(sh.pairs_inv, { set((const void*)k_irfft_z<T, LN>, sh.smem_zi); });
    if (sh.wz) { CCMF_DISPATCH_N(sh.wz, { set((const void*)k_irfft_wz<T, NN>, sh.smem_wzi); }); }
    if (sh.wzd) {
        CCMF_DISPATCH_N(sh.wzd, {
            set((const void*)k_div_rfft_wz<T, NN, false>, sh.smem_wzd);
            set((const void*)k_div_rfft_wz<T, NN, true>, sh.smem_wzd);
        });
    }
    CCMF_DISPATCH_LINES(sh.lpb_y, {
        set((const void*)k_fft_lines<T, 0, LN>, sh.smem_y);
        set((const void*)k_fft_lines<T, 2, LN>, sh.smem_y);
    });
    CCMF_DISPATCH_LINES(sh.lpb_x, { set((const void*)k_fft_lines<T, 1, LN>, sh.smem_x); });
    if (sh.wl_y) {
        CCMF_DISPATCH_N(sh.wl_y, {
            set((const void*)k_fft_wlines<T, 0, NN>, sh.smem_wy);
            set((const void*)k_fft_wlines<T, 2, NN>, sh.smem_wy);
        });
    }
    if (sh.wl_x) { CCMF_DISPATCH_N(sh.wl_x, { set((const void*)k_fft_wlines<T, 1, NN>, sh.smem_wx); }); }
    if constexpr (sizeof(T) == 4) {
        if (sh.x_tma) set((const void*)k_fft_wx_tma<kTmaXN>, kTmaXSmem);
    }
    if (sh.plane_fused && sh.plane_cluster <= 1) set((const void*)k_fft_plane<T>, sh.smem_plane);
    if (sh.plane_fused && sh.plane_cluster > 1 && err == cudaSuccess &&
        plane_cluster_capacity<T>(sh.plane_cluster, sh.smem_plane) < 1)
        err = cudaErrorInvalidConfiguration;
    if (sh.tma_rows > 0) {
        set((const void*)k_update_tma<T, 0>, sh.smem_tma);
        set((const void*)k_update_tma<T, 1>, sh.smem_tma);
        set((const void*)k_update_tma<T, 2>, sh.smem_tma);
    }
    if (is_abw_variant(sh.upd_variant)) {
        CCMF_DISPATCH_ABW(sh.upd_variant, { set((const void*)k_update_abw<T, AW::VW, AW::MINB>, sh.smem_ab); });
    } else if (is_ab_variant(sh.upd_variant)) {
        CCMF_DISPATCH_AB(sh.upd_variant, { set((const void*)k_update_ab<T, AV>, sh.smem_ab); });
    }
    if (sh.upd_variant >= 2 && sh.upd_variant <= 7) {
        CCMF_DISPATCH_PIPE(sh.upd_variant, {
            set((const void*)k_update_pipe<T, 0, ST, NTH>, sh.smem_pipe);
            set((const void*)k_update_pipe<T, 1, ST, NTH>, sh.smem_pipe);
            set((const void*)k_update_pipe<T, 2, ST, NTH>, sh.smem_pipe);
        });
    }
    return err;
}

template <typename T>
void launch_init(const Ctx<T>& c, cudaStream_t st) {
    k_setup<T><<<(unsigned)ceil_div(c.g.batch, 128), 128, 0, st>>>(c.p.sc, c.xi_stage, c.g.batch);
    dim3 grid((unsigned)c.sh.grid_update, (unsigned)c.g.batch);
    k_init_stats<T><<<grid, kThreads, 0, st>>>(c.g, c.p, c.cfg);
    if (!c.cfg.resume) k_init_state<T><<<grid, kThreads, 0, st>>>(c.g, c.p);
    if (c.use_ab) k_ab_init<T><<<grid, kThreads, 0, st>>>(c.g, c.p);
}

// Blocks per SM of the stored-divergence update variants 8 .. 10 and 13 .. 15 (occupancy API), 0 on error.
template <typename T>
int ab_blocks_per_sm(int variant, size_t smem) {
    const void* f = nullptr;
    int nt = 0;
    if (is_abw_variant(variant)) {
        CCMF_DISPATCH_ABW(variant, { f = (const void*)k_update_abw<T, AW::VW, AW::MINB>; });
        nt = 32 * kAbwWarps;
    } else {
        CCMF_DISPATCH_AB(variant, {
            f = (const void*)k_update_ab<T, AV>;
            nt = 32 * AbVariant<T, AV>::NW;
        });
    }
    int nb = 0;
    if (raise_smem_limit(f, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, nt, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// The 16-byte final evaluation pass needs 16-byte aligned cut and flow outputs.
template <typename T>
bool vec_out_ok(const Ptrs<T>& p) {
    return ((uintptr_t)p.cut % 16) == 0 && ((uintptr_t)p.flow % 16) == 0;
}

// Enqueue one ADMM iteration (or, with OUT, the final evaluation).
// `between` is called after every kernel with its class (used to record events).
template <typename T, bool OUT, typename F>
void launch_passes(const Ctx<T>& c, const Ptrs<T>& p, cudaStream_t st, F&& between) {
    const Geom& g = c.g;   // g.batch = number of solves of this launch, starting at p.s0
    const LaunchShape& sh = c.sh;
    const long long pairs = ceil_div((long long)g.n1 * g.n2, 2);
    dim3 gz((unsigned)ceil_div(pairs, sh.pairs_per_block), (unsigned)g.batch);
    long long ty = ceil_div((long long)g.n1 * g.n3h, sh.lpb_y), tx = ceil_div((long long)g.n2 * g.n3h, sh.lpb_x);
    if (sh.grid_y > 0 && sh.grid_y < ty) ty = sh.grid_y;
    if (sh.grid_x > 0 && sh.grid_x < tx) tx = sh.grid_x;
    dim3 gy((unsigned)ty, (unsigned)g.batch);
    dim3 gx((unsigned)tx, (unsigned)g.batch);
    constexpr int kWarpLines = kThreads / 32;   // lines per block round of the warp-per-line passes
    long long twy = ceil_div((long long)g.n1 * g.n3h, kWarpLines), twx = ceil_div((long long)g.n2 * g.n3h, kWarpLines);
    if (sh.grid_y > 0 && sh.grid_y < twy) twy = sh.grid_y;
    if (sh.grid_x > 0 && sh.grid_x < twx) twx = sh.grid_x;
    dim3 gwy((unsigned)twy, (unsigned)g.batch);
    dim3 gwx((unsigned)twx, (unsigned)g.batch);
    dim3 gu((unsigned)sh.grid_update, (unsigned)g.batch);
    // the vector update pass takes its chunks from a ticket counter: the resident blocks, shared
    // by the solves of this launch, so that every solve's chunks run at once on all SMs
    const int vpb = sh.vec_resident > 0 ? sh.vec_resident / g.batch : sh.grid_update;
    const dim3 gv((unsigned)(vpb < 1 ? 1 : vpb), (unsigned)g.batch);
    const T inv_n = (T)(1.0 / (double)g.N);
    const dim3 gwz((unsigned)ceil_div((long long)g.n1 * g.n2, 2 * (kThreads / 32)), (unsigned)g.batch);
    const bool ab = !OUT && c.use_ab;   // the first pass reads the stored divergences a, b
    if (sh.wzd && c.vec_div) {
        CCMF_DISPATCH_N(sh.wzd, {
            if (ab)
                k_div_rfft_wz<T, NN, true><<<gwz, kThreads, sh.smem_wzd, st>>>(g, p, c.tw[2]);
            else
                k_div_rfft_wz<T, NN, false><<<gwz, kThreads, sh.smem_wzd, st>>>(g, p, c.tw[2]);
        });
    } else {
        CCMF_DISPATCH_LINES(sh.pairs_per_block, {
            if (c.vec_div && ab)
                k_div_rfft_z<T, LN, true, true><<<gz, kThreads, sh.smem_z, st>>>(g, p, c.ax[2], c.tw[2]);
            else if (c.vec_div)
                k_div_rfft_z<T, LN, true, false><<<gz, kThreads, sh.smem_z, st>>>(g, p, c.ax[2], c.tw[2]);
            else
                k_div_rfft_z<T, LN, false, false><<<gz, kThreads, sh.smem_z, st>>>(g, p, c.ax[2], c.tw[2]);
        });
    }
    between(kKDivRfftZ);
    if (sh.plane_fused && sh.plane_cluster > 1) {
        launch_plane_cluster<T>(g, p, c, inv_n, st);
        between(kKFftPlane);
    } else if (sh.plane_fused) {
        k_fft_plane<T><<<dim3((unsigned)g.n3h, (unsigned)g.batch), plane_threads<T>(), sh.smem_plane, st>>>(
            g, p, c.ax[0], c.ax[1], c.tw[0], c.tw[1], c.rsym[0], c.rsym[1], c.sym[2], inv_n);
        between(kKFftPlane);
    } else {
        const FastDiv dly = make_fastdiv((unsigned)sh.lpb_y), dlx = make_fastdiv((unsigned)sh.lpb_x);
        // the y symbol in the order the y pass leaves: natural (warp lines) or digit-reversed
        const T* ysym = sh.wl_y ? c.sym[1] : c.rsym[1];
        if (sh.wl_y) {
            CCMF_DISPATCH_N(sh.wl_y, {
                k_fft_wlines<T, 0, NN><<<gwy, kThreads, sh.smem_wy, st>>>(g, p, c.tw[1], c.sym[0], ysym, c.sym[2],
                                                                          inv_n);
            });
        } else {
            CCMF_DISPATCH_LINES(sh.lpb_y, {
                k_fft_lines<T, 0, LN><<<gy, kThreads, sh.smem_y, st>>>(g, p, c.ax[1], c.tw[1], c.rsym[0], ysym,
                                                                        c.sym[2], inv_n, dly);
            });
        }
        between(kKFftYFwd);
        bool x_done = false;
        if constexpr (sizeof(T) == 4) {
            if (sh.x_tma) {
                // the tensor map covers the planes of the solves this launch touches; the plan's
                // launch rules checked the shape, so a failed encoding leaves no valid launch
                alignas(64) CUtensorMap xmap;
                if (encode_x_tensor_map(&xmap, p.spec, g.n1, g.n2, (long long)g.n3h * (p.s0 + g.batch)))
                    k_fft_wx_tma<kTmaXN><<<gwx, kThreads, kTmaXSmem, st>>>(xmap, g, p, c.tw[0], c.sym[0], ysym,
                                                                          c.sym[2], inv_n, c.cfg.spin_limit);
                else
                    k_launch_failed<0><<<1, 32, 0, st>>>(p.sc, p.s0, g.batch);
                x_done = true;
            }
        }
        if (x_done) {
        } else if (sh.wl_x) {
            CCMF_DISPATCH_N(sh.wl_x, {
                k_fft_wlines<T, 1, NN><<<gwx, kThreads, sh.smem_wx, st>>>(g, p, c.tw[0], c.sym[0], ysym, c.sym[2],
                                                                          inv_n);
            });
        } else {
            CCMF_DISPATCH_LINES(sh.lpb_x, {
                k_fft_lines<T, 1, LN><<<gx, kThreads, sh.smem_x, st>>>(g, p, c.ax[0], c.tw[0], c.rsym[0], ysym,
                                                                        c.sym[2], inv_n, dlx);
            });
        }
        between(kKFftXSolve);
        if (sh.wl_y) {
            CCMF_DISPATCH_N(sh.wl_y, {
                k_fft_wlines<T, 2, NN><<<gwy, kThreads, sh.smem_wy, st>>>(g, p, c.tw[1], c.sym[0], ysym, c.sym[2],
                                                                          inv_n);
            });
        } else {
            CCMF_DISPATCH_LINES(sh.lpb_y, {
                k_fft_lines<T, 2, LN><<<gy, kThreads, sh.smem_y, st>>>(g, p, c.ax[1], c.tw[1], c.rsym[0], ysym,
                                                                        c.sym[2], inv_n, dly);
            });
        }
        between(kKFftYInv);
    }
    const dim3 gzi((unsigned)ceil_div(pairs, sh.pairs_inv), (unsigned)g.batch);
    if (sh.wz) {
        CCMF_DISPATCH_N(sh.wz, { k_irfft_wz<T, NN><<<gwz, kThreads, sh.smem_wzi, st>>>(g, p, c.tw[2]); });
    } else {
        CCMF_DISPATCH_LINES(sh.pairs_inv,
                            { k_irfft_z<T, LN><<<gzi, kThreads, sh.smem_zi, st>>>(g, p, c.ax[2], c.tw[2]); });
    }
    between(kKIrfftZ);
    if (OUT && c.vec_update && vec_out_ok(p))
        k_update_vec<T, true><<<gv, kThreads, 0, st>>>(g, p, c.cfg);
    else if (OUT)
        k_update<T, true><<<gu, kThreads, 0, st>>>(g, p, c.cfg);
    else if (ab && is_abw_variant(sh.upd_variant)) {
        const long long items = (long long)sh.ab.nq * sh.ab.nr * sh.ab.npass;
        const dim3 ga((unsigned)ceil_div(items, kAbwWarps), (unsigned)g.batch);
        CCMF_DISPATCH_ABW(sh.upd_variant, {
            k_update_abw<T, AW::VW, AW::MINB><<<ga, kAbwWarps * 32, sh.smem_ab, st>>>(g, p, c.cfg, sh.ab);
        });
    } else if (ab) {
        const dim3 ga((unsigned)(sh.ab.nq * sh.ab.nr), (unsigned)g.batch);
        CCMF_DISPATCH_AB(sh.upd_variant, {
            k_update_ab<T, AV><<<ga, AbVariant<T, AV>::NW * 32, sh.smem_ab, st>>>(g, p, c.cfg, sh.ab);
        });
    } else if (c.vec_update && sh.upd_variant >= 2 && sh.upd_variant <= 7) {
        const dim3 gp((unsigned)sh.grid_pipe, (unsigned)g.batch);
        CCMF_DISPATCH_PIPE(sh.upd_variant, {
            if (c.cfg.rho_rule == 0 || c.cfg.rho_rule == 3)   // BB and residual balancing need |de|^2
                k_update_pipe<T, 0, ST, NTH><<<gp, NTH, sh.smem_pipe, st>>>(g, p, c.cfg);
            else if (c.cfg.rho_rule == 2)
                k_update_pipe<T, 2, ST, NTH><<<gp, NTH, sh.smem_pipe, st>>>(g, p, c.cfg);
            else
                k_update_pipe<T, 1, ST, NTH><<<gp, NTH, sh.smem_pipe, st>>>(g, p, c.cfg);
        });
    } else if (c.vec_update && sh.upd_variant == 1 && sh.tma_rows > 0) {
        const dim3 gt((unsigned)sh.grid_tma, (unsigned)g.batch);
        if (c.cfg.rho_rule == 0 || c.cfg.rho_rule == 3)   // BB and residual balancing need |de|^2
            k_update_tma<T, 0><<<gt, kThreads, sh.smem_tma, st>>>(g, p, c.cfg, sh.tma_rows);
        else if (c.cfg.rho_rule == 2)
            k_update_tma<T, 2><<<gt, kThreads, sh.smem_tma, st>>>(g, p, c.cfg, sh.tma_rows);
        else
            k_update_tma<T, 1><<<gt, kThreads, sh.smem_tma, st>>>(g, p, c.cfg, sh.tma_rows);
    }
    else if (c.vec_update && (sh.upd_variant == 11 || sh.upd_variant == 12)) {
        const int vpb2 = sh.vec_resident_half > 0 ? sh.vec_resident_half / g.batch : sh.grid_update;
        const dim3 gv2((unsigned)(vpb2 < 1 ? 1 : vpb2), (unsigned)g.batch);
        if (sh.upd_variant == 12)
            k_update_vec<T, false, kVecHalfW<T>, 3><<<gv2, kThreads, 0, st>>>(g, p, c.cfg);
        else
            k_update_vec<T, false, kVecHalfW<T>, 2><<<gv2, kThreads, 0, st>>>(g, p, c.cfg);
    } else if (c.vec_update)
        k_update_vec<T, false><<<gv, kThreads, 0, st>>>(g, p, c.cfg);
    else
        k_update<T, false><<<gu, kThreads, 0, st>>>(g, p, c.cfg);
    between(kKUpdate);
}

struct NoHook {
    void operator()(int) const {}
};

template <typename T>
void launch_iteration(const Ctx<T>& c, cudaStream_t st) {
    launch_passes<T, false>(c, c.p, st, NoHook());
}

// One iteration for the solves [s0, s0 + ns) only (a branch of the captured graph).
template <typename T>
void launch_iteration_range(const Ctx<T>& c, int s0, int ns, cudaStream_t st) {
    Ctx<T> cr = c;
    cr.g.batch = ns;
    cr.p.s0 = s0;
    launch_passes<T, false>(cr, cr.p, st, NoHook());
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

// ---- reverse mode (adjoint) helpers ------------------------------------------
template <typename T>
__global__ void k_adj_restore(SolveScalars* sc, int batch, int k0, const double* __restrict__ sched, int sched_len) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    sc[s].iters = k0;
    sc[s].call_start = 0;
    sc[s].rho = sched[(size_t)s * sched_len + k0];
    sc[s].active = 1;
    sc[s].counter = 0;
    sc[s].chunk = 0;
}

template <typename T>
__global__ void k_adj_dummy(SolveScalars* sc, int batch) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    SolveScalars z = {};
    z.rho = 1.0;   // w = e - v / rho with e = y, v = 0: the passes apply M to y
    sc[s] = z;
}

template <typename T>
void launch_adj_restore(const Ctx<T>& c, int k0, const double* sched, int sched_len, cudaStream_t st) {
    k_adj_restore<T><<<(unsigned)ceil_div(c.g.batch, 128), 128, 0, st>>>(c.p.sc, c.g.batch, k0, sched, sched_len);
}

template <typename T>
void launch_adj_seed(const Ctx<T>& c, T* ebar, T* vbar, SolveScalars* dummy, cudaStream_t st) {
    dim3 grid((unsigned)c.sh.grid_update, (unsigned)c.g.batch);
    k_adj_seed<T><<<grid, kThreads, 0, st>>>(c.g, c.p.sc, ebar, vbar);
    k_adj_dummy<T><<<(unsigned)ceil_div(c.g.batch, 128), 128, 0, st>>>(dummy, c.g.batch);
}

// One reverse step k: zbar, y from (ebar, vbar, z^k); M y by the forward passes
// (final-evaluation mode, xi_bar = 0, e = y, v = 0); then ebar, vbar.
// clip_bits: optional [solve][ceil(N / 32)] branches of P_C recorded by an FP64 forward pass.
template <typename T>
void launch_adj_step(const Ctx<T>& c, const T* zk, T* ebar, T* vbar, T* zbar, T* y, T* my, const T* zero,
                     SolveScalars* dummy, T* grad, const double* sched, int sched_len, int k, cudaStream_t st,
                     const unsigned* clip_bits) {
    const double a = 2.0 * (1.0 - c.cfg.delta), b = 1.0 - 2.0 * c.cfg.delta;
    dim3 grid((unsigned)c.sh.grid_update, (unsigned)c.g.batch);
    const T* gam = c.p.gptrs ? nullptr : c.p.gamma;
    k_adj_pre<T><<<grid, kThreads, 0, st>>>(c.g, zk, gam, c.p.gstride, ebar, vbar, sched, sched_len, k, a, zbar, y,
                                             grad, clip_bits);
    Ctx<T> cm = c;
    cm.p.e = y;
    cm.p.v = const_cast<T*>(zero);
    cm.p.sstride = 0;
    cm.p.sc = dummy;
    cm.p.zout = nullptr;
    launch_final<T>(cm, st, my, nullptr);
    k_adj_post<T><<<grid, kThreads, 0, st>>>(c.g, zbar, my, sched, sched_len, k, b, ebar, vbar);
}

// Tile shapes of the batched persistent kernel: {z line pairs, y / x lines} per tile.
// Variant 0 unless its tiles do not fit 110 KB of shared memory (axes beyond about 400 in FP32,
// 200 in FP64), variant 1 then. On the 192-solve workload 16 line pairs per z tile ran 13.57 ms
// per iteration against 14.57 ms with 8, and 32 lines per y / x tile 13.13 ms against 13.57 ms
// with 16: the line passes are bound by their stage barriers, and wider tiles give each barrier
// more butterflies (build-time knobs).
#ifndef CCMF_PERSIST_ZPAIRS
#define CCMF_PERSIST_ZPAIRS 16
#endif
#ifndef CCMF_PERSIST_LINES
#define CCMF_PERSIST_LINES 32
#endif
constexpr int kPersistZPairs = CCMF_PERSIST_ZPAIRS;
constexpr int kPersistLines = CCMF_PERSIST_LINES;
constexpr int kPersistTiles[2][2] = {{kPersistZPairs, kPersistLines}, {4, 8}};

// Resident blocks per SM of k_batch_persist variant `variant` with `smem` bytes of dynamic
// shared memory (raises the kernel's limit first), 0 on error.
template <typename T>
int batch_persist_blocks_per_sm(int variant, size_t smem) {
    int nb = 0;
    const void* f = variant == 0 ? (const void*)k_batch_persist<T, kPersistZPairs, kPersistLines>
                                 : (const void*)k_batch_persist<T, 4, 8>;
    cudaError_t err = raise_smem_limit(f, smem);
    if (err == cudaSuccess)
        err = variant == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_persist<T, kPersistZPairs, kPersistLines>,
                                                                           kThreads, smem)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_persist<T, 4, 8>, kThreads, smem);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// One persistent launch: every pass of one iteration of every solve of the batch.
template <typename T>
void launch_batch_persist(const PersistArgs<T>& a, int variant, int grid, size_t smem, cudaStream_t st) {
    if (variant == 0)
        k_batch_persist<T, kPersistZPairs, kPersistLines><<<grid, kThreads, smem, st>>>(a);
    else
        k_batch_persist<T, 4, 8><<<grid, kThreads, smem, st>>>(a);
}

}  // namespace ccmf
