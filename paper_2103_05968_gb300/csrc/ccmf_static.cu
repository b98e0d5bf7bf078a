// ccmf_solve_static: a solve that allocates no memory at all.
//
// Every other entry point of this library takes a workspace that the caller
// allocated, and ccmf_plan_create allocates small tables. Some callers cannot
// allocate device memory at the point where they need a solve: plug-ins whose
// host application owns the whole device memory through its own pool (a
// cudaMalloc of theirs would fail or fragment that pool), and latency-critical
// paths that must not take the implicit device synchronisation of cudaMalloc /
// cudaFree. For them this file keeps a fixed scratch area in a file-scope
// __device__ array and runs one single-normal solve on it; the caller still
// passes gamma and the outputs.
//
// The call copies the unit normal from host memory with cudaMemcpyAsync, and it
// synchronises the stream when it stops on a tolerance (it reads an active
// counter every check_every updates) or returns a result.
//
// The scratch array is part of the library image: every GPU that loads the
// library holds kStaticScratchBytes of device memory for it until the process
// exits. All calls on a device share it, so calls whose GPU work overlaps (two
// streams, two host threads) race with each other; each call leaves its state
// behind and the next call overwrites it.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/ccmf.h"
#include "ccmf_launch.cuh"

using namespace ccmf;

namespace ccmf {
template <typename T> cudaError_t configure_kernels(const LaunchShape&);
template <typename T> void launch_init(const Ctx<T>&, cudaStream_t);
template <typename T> void launch_iteration(const Ctx<T>&, cudaStream_t);
template <typename T> void launch_final(const Ctx<T>&, cudaStream_t, T*, T*);
}  // namespace ccmf

namespace {

constexpr size_t kStaticScratchBytes = (size_t)CCMF_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kStaticGridUpdate = 608;

}  // namespace

// The scratch area (see the file comment). Host code must not use its name as a
// device address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_ccmf_scratch[CCMF_STATIC_SCRATCH_BYTES];

namespace {

unsigned char* g_scratch_ptr[kMaxDevices];   // device address of g_ccmf_scratch per device
std::mutex g_scratch_mutex;                   // first calls from several host threads look it up once

// Frequency held by slot p after the in-place decimation-in-frequency stages of
// the radix schedule ap: k(p) = sum_s q_s prod_{t<s} R_t, q_s = (p / m_s) mod R_s.
__device__ int slot_frequency(const AxisPlan& ap, int p) {
    int k = 0, w = 1;
    for (int t = 0; t < ap.nst; ++t) {
        const int m = ap.span[t] / ap.rad[t];
        k += ((p / m) % ap.rad[t]) * w;
        w *= ap.rad[t];
    }
    return k;
}

// Twiddle W_n^t = exp(-2 pi i t / n) and symbol 4 sin^2(pi t / n) tables of the
// three axes, and the x and y symbols in digit-reversed slot order, written into
// the scratch area (double arithmetic, stored as T).
template <typename T>
__global__ void k_static_tables(cx<T>* tw0, cx<T>* tw1, cx<T>* tw2, T* sy0, T* sy1, T* sy2, T* rs0, T* rs1,
                                AxisPlan ax0, AxisPlan ax1, int n1, int n2, int n3) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n[3] = {n1, n2, n3};
    cx<T>* tw[3] = {tw0, tw1, tw2};
    T* sy[3] = {sy0, sy1, sy2};
    for (int a = 0; a < 3; ++a) {
        if (t >= n[a]) continue;
        double s, c;
        sincospi(-2.0 * (double)t / (double)n[a], &s, &c);
        tw[a][t] = cmake<cx<T>>((T)c, (T)s);
        const double h = sinpi((double)t / (double)n[a]);
        sy[a][t] = (T)(4.0 * h * h);
    }
    if (t < n1) {
        const double h = sinpi((double)slot_frequency(ax0, t) / (double)n1);
        rs0[t] = (T)(4.0 * h * h);
    }
    if (t < n2) {
        const double h = sinpi((double)slot_frequency(ax1, t) / (double)n2);
        rs1[t] = (T)(4.0 * h * h);
    }
}

bool radix_plan(int n, AxisPlan* ap) {
    memset(ap, 0, sizeof(*ap));
    ap->n = n;
    int m = n, st = 0;
    const int order[5] = {8, 4, 2, 3, 5};
    for (int r : order)
        while (m % r == 0) {
            if (st >= kMaxStages) return false;
            ap->rad[st++] = r;
            m /= r;
        }
    ap->nst = st;
    unsigned ns = 1;
    int span = n;
    for (int t = 0; t < st; ++t) {
        ap->ns[t] = make_fastdiv(ns);
        ns *= (unsigned)ap->rad[t];
        ap->span[t] = span;
        ap->sub[t] = make_fastdiv((unsigned)(span / ap->rad[t]));
        span /= ap->rad[t];
    }
    return m == 1;
}

int lines_for(int n, size_t cs) {
    const long long L = ((long long)((96 * 1024) / cs) - n) / (2LL * n) - 1;
    int r = 1;
    while (r * 2 <= 16 && r * 2 <= L) r *= 2;
    return r;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// One-time set-up per device, with that device current: the device address of
// the scratch array (host code cannot use the array's name as an address). It runs
// in the first call on the device, which should come before any stream capture
// begins. The address belongs to the device's primary context; a cudaDeviceReset
// ends that context, and ccmf_solve_static must not be called on the device afterwards.
int static_setup(int dev, unsigned char** base) {
    if (dev < 0 || dev >= kMaxDevices) return CCMF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_ccmf_scratch) != cudaSuccess || !ptr) return CCMF_ERR_CUDA;
        g_scratch_ptr[dev] = reinterpret_cast<unsigned char*>(ptr);
    }
    *base = g_scratch_ptr[dev];
    return CCMF_OK;
}

template <typename T>
int static_solve(int n1, int n2, int n3, const T* gamma, const double* xi_bar, const ccmf_params& prm, T* flow,
                 T* cut, ccmf_result* result, cudaStream_t st, int dev) {
    Ctx<T> c;
    memset(&c, 0, sizeof(c));
    Geom& g = c.g;
    g.n1 = n1;
    g.n2 = n2;
    g.n3 = n3;
    g.n3h = n3 / 2 + 1;
    g.batch = 1;
    g.N = (long long)n1 * n2 * n3;
    g.Nh = (long long)n1 * n2 * g.n3h;
    g.div_n3 = make_fastdiv((unsigned)n3);
    g.div_n2 = make_fastdiv((unsigned)n2);
    g.div_n3h = make_fastdiv((unsigned)g.n3h);
    const int nn[3] = {n1, n2, n3};
    for (int a = 0; a < 3; ++a)
        if (!radix_plan(nn[a], &c.ax[a])) return CCMF_ERR_UNSUPPORTED_SIZE;
    const size_t cs = 2 * sizeof(T);
    LaunchShape& sh = c.sh;
    sh.pairs_per_block = lines_for(n3, cs);
    sh.lpb_y = lines_for(n2, cs);
    sh.lpb_x = lines_for(n1, cs);
    sh.smem_z = ((size_t)n3 + 2 * (size_t)n3 * (sh.pairs_per_block + 1)) * cs;
    sh.pairs_inv = sh.pairs_per_block;
    sh.smem_zi = sh.smem_z;
    sh.smem_y = ((size_t)n2 + 2 * (size_t)n2 * (sh.lpb_y + 1)) * cs;
    sh.smem_x = ((size_t)n1 + 2 * (size_t)n1 * (sh.lpb_x + 1)) * cs;
    long long gu = (g.N + kThreads - 1) / kThreads;
    sh.grid_update = (int)(gu < kStaticGridUpdate ? gu : kStaticGridUpdate);
    sh.vec_resident = 0;   // the vector update pass runs grid_update blocks per solve

    // scratch layout: scalars, counter, normal, partials, history, state (two copies),
    // spectrum, phi, tables
    const size_t N = (size_t)g.N;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + bytes);
        return o;
    };
    const size_t o_sc = take(256), o_nact = take(256), o_xi = take(3 * sizeof(double));
    // partial sums: one slot per update block, or per chunk of the vector update pass
    const long long nparts = std::max<long long>(sh.grid_update, vec_update_chunks(g.N, 16 / (int)sizeof(T)));
    const size_t o_part = take(sizeof(double) * kNSum * (size_t)nparts);
    const size_t o_hist = take(sizeof(double) * kHistFields * (size_t)kHistCap);
    const size_t o_e = take(sizeof(T) * 6 * N * 2), o_v = take(sizeof(T) * 6 * N * 2);
    const size_t o_spec = take(cs * (size_t)g.Nh), o_phi = take(sizeof(T) * N);
    size_t o_tw[3], o_sy[3];
    for (int a = 0; a < 3; ++a) o_tw[a] = take(cs * (size_t)nn[a]);
    for (int a = 0; a < 3; ++a) o_sy[a] = take(sizeof(T) * (size_t)nn[a]);
    size_t o_rs[2];
    for (int a = 0; a < 2; ++a) o_rs[a] = take(sizeof(T) * (size_t)nn[a]);
    if (off > kStaticScratchBytes) return CCMF_ERR_UNSUPPORTED_SIZE;

    unsigned char* ws = nullptr;
    int rc = static_setup(dev, &ws);
    if (rc != CCMF_OK) return rc;
    // shared-memory limits depend on the grid, so they are set on every call (no allocation)
    if (configure_kernels<T>(sh) != cudaSuccess) return CCMF_ERR_CUDA;

    LoopConfig& cfg = c.cfg;
    cfg.tol = prm.tol;
    cfg.delta = prm.delta;
    cfg.rho0 = prm.rho0;
    cfg.bb_corr_min = prm.bb_corr_min;
    cfg.rho_step_max = prm.rho_step_max;
    cfg.max_iter = prm.max_iter;
    cfg.fixed_iters = prm.fixed_iters;
    cfg.rho_rule = prm.rho_rule;
    cfg.hist_len = prm.history_len;
    cfg.resume = 0;

    for (int a = 0; a < 3; ++a) {
        c.tw[a] = reinterpret_cast<const cx<T>*>(ws + o_tw[a]);
        c.sym[a] = reinterpret_cast<const T*>(ws + o_sy[a]);
    }
    for (int a = 0; a < 2; ++a) c.rsym[a] = reinterpret_cast<const T*>(ws + o_rs[a]);
    c.xi_stage = reinterpret_cast<const double*>(ws + o_xi);
    c.p.sc = reinterpret_cast<SolveScalars*>(ws + o_sc);
    c.p.n_active = reinterpret_cast<int*>(ws + o_nact);
    c.p.partial = reinterpret_cast<double*>(ws + o_part);
    c.p.hist = reinterpret_cast<double*>(ws + o_hist);
    c.p.e = reinterpret_cast<T*>(ws + o_e);
    c.p.v = reinterpret_cast<T*>(ws + o_v);
    c.p.sstride = 6 * g.N;
    c.p.spec = reinterpret_cast<cx<T>*>(ws + o_spec);
    c.p.phi = reinterpret_cast<T*>(ws + o_phi);
    c.p.gamma = gamma;
    c.p.gstride = 0;
    const int W = 16 / (int)sizeof(T);
    c.vec_div = (n3 % W) == 0;
    c.vec_update = c.vec_div && ((uintptr_t)gamma % 16) == 0;

    // clear what must start from a known value: the active counter, the history ring
    const double nn2 = xi_bar[0] * xi_bar[0] + xi_bar[1] * xi_bar[1] + xi_bar[2] * xi_bar[2];
    const double inv = 1.0 / sqrt(nn2);
    const double xi[3] = {xi_bar[0] * inv, xi_bar[1] * inv, xi_bar[2] * inv};
    if (cudaMemcpyAsync(ws + o_xi, xi, sizeof(xi), cudaMemcpyHostToDevice, st) != cudaSuccess) return CCMF_ERR_CUDA;
    if (cudaMemsetAsync(ws + o_nact, 0, sizeof(int), st) != cudaSuccess) return CCMF_ERR_CUDA;
    if (cudaMemsetAsync(ws + o_hist, 0xFF, sizeof(double) * kHistFields * (size_t)kHistCap, st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    const int nmax = n1 > n2 ? (n1 > n3 ? n1 : n3) : (n2 > n3 ? n2 : n3);
    k_static_tables<T><<<(nmax + 127) / 128, 128, 0, st>>>(
        reinterpret_cast<cx<T>*>(ws + o_tw[0]), reinterpret_cast<cx<T>*>(ws + o_tw[1]),
        reinterpret_cast<cx<T>*>(ws + o_tw[2]), reinterpret_cast<T*>(ws + o_sy[0]), reinterpret_cast<T*>(ws + o_sy[1]),
        reinterpret_cast<T*>(ws + o_sy[2]), reinterpret_cast<T*>(ws + o_rs[0]), reinterpret_cast<T*>(ws + o_rs[1]),
        c.ax[0], c.ax[1], n1, n2, n3);
    launch_init<T>(c, st);
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;

    // the loop: kernels launched directly on the caller's stream; with a tolerance
    // the host reads the active counter after every check_every updates
    const bool fixed = prm.fixed_iters > 0;
    const int total = fixed ? prm.fixed_iters : prm.max_iter;
    int done = 0;
    while (done < total) {
        const int chunk = fixed ? total : (prm.check_every < total - done ? prm.check_every : total - done);
        for (int it = 0; it < chunk; ++it) launch_iteration<T>(c, st);
        if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
        done += chunk;
        if (!fixed) {
            int active = 0;
            if (cudaMemcpyAsync(&active, ws + o_nact, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return CCMF_ERR_CUDA;
            if (active <= 0) break;
        }
    }
    launch_final<T>(c, st, cut, flow);
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
    if (result) {
        SolveScalars sc;
        if (cudaMemcpyAsync(&sc, ws + o_sc, sizeof(sc), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        result->gamma_eff = sc.dual;
        result->gamma_primal = sc.primal;
        result->gamma_dual = sc.dual;
        result->residual = sc.residual;
        result->mean_v_norm = sc.mean_v;
        result->rho = sc.rho;
        result->iters = sc.iters;
        result->converged = sc.converged;
        result->status = sc.status;
        result->reserved = 0;
    }
    return CCMF_OK;
}

bool device_pointer(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int ccmf_solve_static(int n1, int n2, int n3, int precision, const void* gamma, const double* xi_bar,
                                 const ccmf_params* params, void* flow, void* cut, ccmf_result* result,
                                 void* stream) {
    if (n1 < 1 || n2 < 1 || n3 < 1 || !gamma || !xi_bar) return CCMF_ERR_INVALID_ARG;
    if (precision != CCMF_FP64 && precision != CCMF_FP32_MIXED) return CCMF_ERR_INVALID_ARG;
    if (n1 > 1024 || n2 > 1024 || n3 > 1024) return CCMF_ERR_UNSUPPORTED_SIZE;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(xi_bar[a])) return CCMF_ERR_INVALID_ARG;
    const double nn = xi_bar[0] * xi_bar[0] + xi_bar[1] * xi_bar[1] + xi_bar[2] * xi_bar[2];
    if (!(nn > 0.0) || !isfinite(nn)) return CCMF_ERR_INVALID_ARG;
    ccmf_params prm;
    if (params) {
        prm = *params;
    } else {
        ccmf_params_default(&prm);
    }
    if (prm.fixed_iters < 0 || prm.max_iter < 1 || prm.check_every < 1) return CCMF_ERR_INVALID_ARG;
    if (prm.fixed_iters == 0 && !(prm.tol > 0.0)) return CCMF_ERR_INVALID_ARG;
    if (!(prm.delta > 0.0 && prm.delta < 1.0)) return CCMF_ERR_INVALID_ARG;
    if (prm.rho_rule < CCMF_RHO_BB || prm.rho_rule > CCMF_RHO_RB) return CCMF_ERR_INVALID_ARG;
    if (!(prm.rho_step_max >= 1.0) || !isfinite(prm.rho0) || !isfinite(prm.bb_corr_min)) return CCMF_ERR_INVALID_ARG;
    if (prm.history_len < 0 || prm.history_len > kHistCap) return CCMF_ERR_INVALID_ARG;
    if (prm.resume != 0) return CCMF_ERR_INVALID_ARG;   // the scratch keeps no state between calls
    if (!device_pointer(gamma) || (flow && !device_pointer(flow)) || (cut && !device_pointer(cut)))
        return CCMF_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (precision == CCMF_FP64)
        return static_solve<double>(n1, n2, n3, reinterpret_cast<const double*>(gamma), xi_bar, prm,
                                    reinterpret_cast<double*>(flow), reinterpret_cast<double*>(cut), result, st, dev);
    return static_solve<float>(n1, n2, n3, reinterpret_cast<const float*>(gamma), xi_bar, prm,
                               reinterpret_cast<float*>(flow), reinterpret_cast<float*>(cut), result, st, dev);
}
