// CUDA kernels of one damped-ADMM iteration (Eq. 30 of the paper) on the CCMF
// discretisation, templated on the field type T (float: FP32-mixed, double: FP64).
//
// One iteration from (e^k, v^k, rho^k) is five passes:
//   1. k_div_rfft_z     w = e - v/rho, d = div^- A* w (Sec. 2.2, Eq. 17) fused
//                       with the real-to-complex FFT along z (two real lines per
//                       complex transform);
//   2. k_fft_lines<0>   forward FFT along y (k_fft_wlines<0> for power-of-two n2);
//   3. k_fft_lines<1>   forward FFT along x, Poisson solve
//                       phi^ = d^ / (-sum_a 4 sin^2(pi k_a / N_a)), phi^(0) = 0
//                       (the (div^- grad^+)^+ of Eq. 28), inverse FFT along x;
//   4. k_fft_lines<2>   inverse FFT along y;
//   5. k_irfft_z        complex-to-real inverse FFT along z -> phi;
//   6. k_update<false>  xi^{k+1/2} = w - A(A* w - grad^+ phi - xi_bar) (= P_K(w),
//                       Eq. 28), over-relaxation, z = v + rho xi, node-wise
//                       projection onto C_gamma (Eq. 19), e^{k+1}, v^{k+1}
//                       (Eq. 30), block partial sums; the last block reduces
//                       them in double and updates rho, the history and the stop
//                       flag on the device (Eq. 31, BB / LTD scaling).
// k_update<true> is the final evaluation: it writes the cut xi^{K+1/2} and the
// flow A* v^K instead of advancing the state.
#pragma once

#include <math.h>

#include <cooperative_groups.h>

#include "ccmf_types.cuh"

namespace ccmf {

template <typename T> struct Real;
template <> struct Real<float> {
    __device__ __forceinline__ static float sqrt_(float x) { return sqrtf(x); }
};
template <> struct Real<double> {
    __device__ __forceinline__ static double sqrt_(double x) { return sqrt(x); }
};

// Asynchronous global -> shared copy of one complex element (cp.async: the thread
// issues all its copies before waiting, instead of one load latency per element).
template <typename C>
__device__ __forceinline__ void cp_async_cx(C* smem_dst, const C* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// gamma field of solve s: a per-solve pointer table when given, else base + s * stride.
template <typename T>
__device__ __forceinline__ const T* gamma_of(const Ptrs<T>& p, int s) {
    return p.gptrs ? p.gptrs[s] : p.gamma + (size_t)s * p.gstride;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// Block reduction of NQ per-thread values (T) into one double each, written to
// partial[b * NQ + q] (fixed order: warp shuffles, then the warps in turn).
template <typename T, int NQ, int NT = kThreads>
__device__ void block_store_partial(const T (&acc)[NQ], double* __restrict__ partial, long long b) {
    __shared__ double red[NT / 32][NQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        T s = warp_sum(acc[q]);
        if (lane == 0) red[wid][q] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
        partial[b * NQ + threadIdx.x] = s;
    }
}

// Ticket of a block that has stored its partials: true in every thread of the block
// that finishes last of nblocks (every partial is then visible to it).
template <int NT = kThreads>
__device__ bool block_ticket(unsigned int* counter, int nblocks) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(counter, 1u);
        last = (t == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    return last != 0;
}

// Both: the block's partials, then its ticket.
template <typename T, int NQ, int NT = kThreads>
__device__ bool block_partials(T (&acc)[NQ], double* __restrict__ partial, unsigned int* counter,
                               int nblocks, int b) {
    block_store_partial<T, NQ, NT>(acc, partial, b);
    return block_ticket<NT>(counter, nblocks);
}

// Deterministic double reduction of nblocks x NQ partials by one block.
template <int NQ, int NT = kThreads>
__device__ void reduce_partials(const double* __restrict__ partial, int nblocks, double (&out)[NQ]) {
    __shared__ double red[NT / 32][NQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += NT) s += __ldcg(partial + (size_t)b * NQ + q);
        s = warp_sum(s);
        if (lane == 0) red[wid][q] = s;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w][q];
        out[q] = s;
    }
}

// ---------------------------------------------------------------------------
// Initialisation: statistics of gamma, rho^0 (reading R2 of the design notes)
// and the initial state e^0 = A xi_bar, v^0 = 0.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_init_stats(Geom g, Ptrs<T> p, LoopConfig cfg) {
    const int s = blockIdx.y + p.s0;
    const T* gam = gamma_of(p, s);
    // element type per element (min / max are exact in T); the sum goes to double every
    // 32 elements, so FP32 plans do not pay the FP64 rate per element
    T tmin = T(INFINITY), tmax = T(-INFINITY), csum = T(0);
    double acc_sum = 0.0, acc_bad = 0.0;
    int cnt = 0;
    auto take = [&](T x) {
        if (!(x >= T(0)) || !isfinite(x)) {
            acc_bad += 1.0;
        } else {
            tmin = fmin(tmin, x);
            tmax = fmax(tmax, x);
            csum += x;
            if (++cnt == 32) {
                acc_sum += (double)csum;
                csum = T(0);
                cnt = 0;
            }
        }
    };
    const long long stride = (long long)gridDim.x * kThreads;
    const long long t0 = (long long)blockIdx.x * kThreads + threadIdx.x;
    // 16-byte loads when gamma is 16-byte aligned and N a multiple of the vector width (every
    // thread of the launch takes the same branch)
    constexpr int W = 16 / (int)sizeof(T);
    if (((uintptr_t)gam % 16) == 0 && g.N % W == 0) {
        const long long nv = g.N / W;
        for (long long q = t0; q < nv; q += stride) {
            if constexpr (sizeof(T) == 4) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(gam) + q);
                take(x.x);
                take(x.y);
                take(x.z);
                take(x.w);
            } else {
                const double2 x = __ldg(reinterpret_cast<const double2*>(gam) + q);
                take(x.x);
                take(x.y);
            }
        }
    } else {
        for (long long lin = t0; lin < g.N; lin += stride) take(gam[lin]);
    }
    acc_sum += (double)csum;
    double acc_min = (double)tmin, acc_max = (double)tmax;
    // min / max via shuffles, sums via the generic partial path
    for (int off = 16; off > 0; off >>= 1) {
        acc_min = fmin(acc_min, __shfl_xor_sync(0xffffffffu, acc_min, off));
        acc_max = fmax(acc_max, __shfl_xor_sync(0xffffffffu, acc_max, off));
    }
    __shared__ double mm[kThreads / 32][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        mm[wid][0] = acc_min;
        mm[wid][1] = acc_max;
    }
    __syncthreads();
    double bmin = INFINITY, bmax = -INFINITY;
    for (int w = 0; w < kThreads / 32; ++w) {
        bmin = fmin(bmin, mm[w][0]);
        bmax = fmax(bmax, mm[w][1]);
    }
    double* part = p.partial + (size_t)s * gridDim.x * 4;
    double acc2[2] = {acc_sum, acc_bad};
    __shared__ double red[kThreads / 32][2];
    for (int q = 0; q < 2; ++q) {
        double v = warp_sum(acc2[q]);
        if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            s0 += red[w][0];
            s1 += red[w][1];
        }
        part[blockIdx.x * 4 + 0] = bmin;
        part[blockIdx.x * 4 + 1] = bmax;
        part[blockIdx.x * 4 + 2] = s0;
        part[blockIdx.x * 4 + 3] = s1;
    }
    __threadfence();
    __syncthreads();
    __shared__ int last;
    SolveScalars& S = p.sc[s];
    if (threadIdx.x == 0) last = (atomicAdd(&S.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    // the last block reduces the block partials: thread t takes blocks t, t + 256, ... in
    // order, then a fixed shuffle tree and the warps in order (deterministic sums; one
    // thread walking every partial took about 0.2 ms for 608 blocks x 3 solves)
    double gmin = INFINITY, gmax = -INFINITY, gsum = 0.0, bad = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
        gmin = fmin(gmin, __ldcg(part + b * 4 + 0));
        gmax = fmax(gmax, __ldcg(part + b * 4 + 1));
        gsum += __ldcg(part + b * 4 + 2);
        bad += __ldcg(part + b * 4 + 3);
    }
    for (int off = 16; off > 0; off >>= 1) {
        gmin = fmin(gmin, __shfl_xor_sync(0xffffffffu, gmin, off));
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, off));
    }
    gsum = warp_sum(gsum);
    bad = warp_sum(bad);
    __shared__ double fin[kThreads / 32][4];
    if (lane == 0) {
        fin[wid][0] = gmin;
        fin[wid][1] = gmax;
        fin[wid][2] = gsum;
        fin[wid][3] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        gmin = INFINITY;
        gmax = -INFINITY;
        gsum = 0.0;
        bad = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            gmin = fmin(gmin, fin[w][0]);
            gmax = fmax(gmax, fin[w][1]);
            gsum += fin[w][2];
            bad += fin[w][3];
        }
        S.counter = 0;
        S.gmin = gmin;
        S.gmax = gmax;
        S.gsum = gsum;
        S.bad = (int)bad;
        int status = 0;
        double rho0 = cfg.rho0 > 0.0 ? cfg.rho0 : (gmin > 0.0 ? gmin : gsum / (double)g.N);
        if (bad > 0.0) status = 5;                        // CCMF_ERR_NUMERICAL
        else if (!(rho0 > 0.0) || !isfinite(rho0)) status = 1;  // gamma identically zero
        if (!cfg.resume) {
            S.rho = cfg.rho_sched ? cfg.rho_sched[(size_t)s * cfg.sched_len] : rho0;
            S.iters = 0;
            S.ab_iter = -1;
        }
        S.status = status;
        S.converged = 0;
        S.call_start = S.iters;
        S.active = (status == 0) ? 1 : 0;
        if (status == 0) atomicAdd(p.n_active, 1);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_init_state(Geom g, Ptrs<T> p) {
    const int s = blockIdx.y + p.s0;
    const double h = 0.70710678118654752440084436210485;
    const SolveScalars& S = p.sc[s];
    const T a0 = (T)(S.xi[0] * h), a1 = (T)(S.xi[1] * h), a2 = (T)(S.xi[2] * h);
    const long long cur = (long long)(S.iters & 1) * p.sstride + (long long)s * 6 * g.N;
    T* e = p.e + cur;
    T* v = p.v + cur;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < g.N; lin += stride) {
        e[0 * g.N + lin] = a0;
        e[1 * g.N + lin] = a1;
        e[2 * g.N + lin] = a2;
        e[3 * g.N + lin] = a0;
        e[4 * g.N + lin] = a1;
        e[5 * g.N + lin] = a2;
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c * g.N + lin] = T(0);
    }
}

// ---------------------------------------------------------------------------
// 16-byte vectors of the field type (4 floats or 2 doubles).
// ---------------------------------------------------------------------------
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int W = 4;
    __device__ __forceinline__ static void ld(const float* __restrict__ p, float (&o)[4]) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
    __device__ __forceinline__ static void st(float* p, const float (&o)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int W = 2;
    __device__ __forceinline__ static void ld(const double* __restrict__ p, double (&o)[2]) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = t.x; o[1] = t.y;
    }
    __device__ __forceinline__ static void st(double* p, const double (&o)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
};

// Neighbour offsets of the row (i, j) of a solve: rows (i+1, j), (i-1, j), (i, j+1), (i, j-1).
struct RowNb {
    long long row, ip, im, jp, jm;  // element offsets of k = 0 of each row
};

__device__ __forceinline__ RowNb row_neighbours(const Geom& g, unsigned row) {
    const unsigned i = fdiv(row, g.div_n2);
    const int j = (int)(row - i * (unsigned)g.n2);
    const int ip = ((int)i + 1 == g.n1) ? 0 : (int)i + 1, im = (i == 0) ? g.n1 - 1 : (int)i - 1;
    const int jp = (j + 1 == g.n2) ? 0 : j + 1, jm = (j == 0) ? g.n2 - 1 : j - 1;
    RowNb r;
    const long long n3 = g.n3;
    r.row = (long long)row * n3;
    r.ip = ((long long)ip * g.n2 + j) * n3;
    r.im = ((long long)im * g.n2 + j) * n3;
    r.jp = ((long long)i * g.n2 + jp) * n3;
    r.jm = ((long long)i * g.n2 + jm) * n3;
    return r;
}

// ---------------------------------------------------------------------------
// Pass 1: divergence of A*(e - v/rho) fused with the real-to-complex z FFT.
// Line l = i * n2 + j of a solve; block b packs line pairs (2q, 2q+1) for
// q in [b P, b P + P) as real and imaginary parts of one complex line.
// d(p) = (1/sqrt2) sum_a [w1_a(p) - w1_a(p - e_a) + w2_a(p + e_a) - w2_a(p)].
// VEC: each thread reads W consecutive voxels of a line with 16-byte loads.
// ---------------------------------------------------------------------------
template <typename T, int P, bool VEC, bool AB = false>
__global__ void __launch_bounds__(kThreads) k_div_rfft_z(Geom g, Ptrs<T> p, AxisPlan az,
                                                         const cx<T>* __restrict__ tw) {
    using C = cx<T>;
    constexpr int stride = P + 1;
    constexpr int W = VEC ? Vec16<T>::W : 1;
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twl = reinterpret_cast<C*>(smem_raw);
    C* A = twl + g.n3;
    C* B = A + (size_t)g.n3 * stride;
    for (int t = threadIdx.x; t < g.n3; t += kThreads) twl[t] = tw[t];
    const T irho = T(1) / (T)p.sc[s].rho;
    const T h = T(0.70710678118654752440084436210485);
    const long long N = g.N;
    const long long cur = (long long)(p.sc[s].iters & 1) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ e = p.e + cur;
    const T* __restrict__ v = p.v + cur;
    const long long L = (long long)g.n1 * g.n2;
    const long long l0 = (long long)blockIdx.x * 2 * P;
    const int n3w = g.n3 / W;
    const int cnt = 2 * P * n3w;
    T* Ar = reinterpret_cast<T*>(A);
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int ll = idx / n3w;
        const int k0 = (idx - ll * n3w) * W;
        const long long l = l0 + ll;
        T d[W];
#pragma unroll
        for (int u = 0; u < W; ++u) d[u] = T(0);
        if (AB && l < L) {
            // stored divergences of the state: d = a - b / rho
            const T* a = p.ab + (size_t)s * 2 * N + l * g.n3 + k0;
            if constexpr (VEC) {
                T ta[W], tb[W];
                Vec16<T>::ld(a, ta);
                Vec16<T>::ld(a + N, tb);
#pragma unroll
                for (int u = 0; u < W; ++u) d[u] = ta[u] - tb[u] * irho;
            } else {
                d[0] = a[0] - a[N] * irho;
            }
        } else if (l < L) {
            const RowNb rn = row_neighbours(g, (unsigned)l);
            const int kp = (k0 + W == g.n3) ? 0 : k0 + W;      // first voxel after the group
            const int km = (k0 == 0) ? g.n3 - 1 : k0 - 1;        // last voxel before the group
            if constexpr (VEC) {
                T w[6][W], tmp_e[W], tmp_v[W];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    Vec16<T>::ld(e + c * N + rn.row + k0, tmp_e);
                    Vec16<T>::ld(v + c * N + rn.row + k0, tmp_v);
#pragma unroll
                    for (int u = 0; u < W; ++u) w[c][u] = tmp_e[u] - tmp_v[u] * irho;
                }
                T xp[W], xm[W], yp[W], ym[W];
                Vec16<T>::ld(e + 3 * N + rn.ip + k0, tmp_e);
                Vec16<T>::ld(v + 3 * N + rn.ip + k0, tmp_v);
#pragma unroll
                for (int u = 0; u < W; ++u) xp[u] = tmp_e[u] - tmp_v[u] * irho;
                Vec16<T>::ld(e + 0 * N + rn.im + k0, tmp_e);
                Vec16<T>::ld(v + 0 * N + rn.im + k0, tmp_v);
#pragma unroll
                for (int u = 0; u < W; ++u) xm[u] = tmp_e[u] - tmp_v[u] * irho;
                Vec16<T>::ld(e + 4 * N + rn.jp + k0, tmp_e);
                Vec16<T>::ld(v + 4 * N + rn.jp + k0, tmp_v);
#pragma unroll
                for (int u = 0; u < W; ++u) yp[u] = tmp_e[u] - tmp_v[u] * irho;
                Vec16<T>::ld(e + 1 * N + rn.jm + k0, tmp_e);
                Vec16<T>::ld(v + 1 * N + rn.jm + k0, tmp_v);
#pragma unroll
                for (int u = 0; u < W; ++u) ym[u] = tmp_e[u] - tmp_v[u] * irho;
                const T zp = __ldg(e + 5 * N + rn.row + kp) - __ldg(v + 5 * N + rn.row + kp) * irho;
                const T zm = __ldg(e + 2 * N + rn.row + km) - __ldg(v + 2 * N + rn.row + km) * irho;
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const T w2zp = (u + 1 < W) ? w[5][(u + 1) % W] : zp;
                    const T w1zm = (u > 0) ? w[2][(u + W - 1) % W] : zm;
                    const T sx = w[0][u] - xm[u] + xp[u] - w[3][u];
                    const T sy = w[1][u] - ym[u] + yp[u] - w[4][u];
                    const T sz = w[2][u] - w1zm + w2zp - w[5][u];
                    d[u] = h * (sx + sy + sz);
                }
            } else {
                const long long p0 = rn.row + k0;
                auto wc = [&](int c, long long off) { return e[c * N + off] - v[c * N + off] * irho; };
                const T sx = wc(0, p0) - wc(0, rn.im + k0) + wc(3, rn.ip + k0) - wc(3, p0);
                const T sy = wc(1, p0) - wc(1, rn.jm + k0) + wc(4, rn.jp + k0) - wc(4, p0);
                const T sz = wc(2, p0) - wc(2, rn.row + km) + wc(5, rn.row + kp) - wc(5, p0);
                d[0] = h * (sx + sy + sz);
            }
        }
#pragma unroll
        for (int u = 0; u < W; ++u) Ar[2 * ((k0 + u) * stride + (ll >> 1)) + (ll & 1)] = d[u];
    }
    __syncthreads();
    C* R = block_fft<C, P>(A, B, az, twl);
    // half spectrum, k_z-major: spec[kz][i][j]; consecutive threads take consecutive line pairs
    const int cnt2 = P * g.n3h;
    C* spec = p.spec + (size_t)s * g.Nh;
    for (int idx = threadIdx.x; idx < cnt2; idx += kThreads) {
        const int kz = idx / P;
        const int c = idx - kz * P;
        const C Z = R[kz * stride + c];
        const int kmr = (kz == 0) ? 0 : g.n3 - kz;
        const C Zm = cconj(R[kmr * stride + c]);
        const C Sm = cadd(Z, Zm), D = csub(Z, Zm);
        const long long la = l0 + 2 * c, lb = la + 1;
        C* dst = spec + (long long)kz * L + la;
        if (la < L) dst[0] = cmake<C>(T(0.5) * Sm.x, T(0.5) * Sm.y);
        if (lb < L) dst[1] = cmake<C>(T(0.5) * D.y, T(-0.5) * D.x);
    }
}

// ---------------------------------------------------------------------------
// Passes 2-4 for planes too large for one block: FFTs along y and x of the half
// spectrum, stored k_z-major as [n3h][n1][n2], run in place on tiles of L lines.
// MODE 0: forward along y as decimation in frequency; the spectrum is left in
//         digit-reversed y order.
// MODE 1: forward along x (DIF), multiply by 1 / (N lambda(k)) with
//         lambda(k) = -sum_a 4 sin^2(pi k_a / N_a) and 0 at k = 0, read from
//         digit-reversed x and y tables, then the inverse along x as
//         conj(DIT(conj(.))); the result is stored conjugated.
// MODE 2: inverse along y: DIT of the conjugated data, conjugated on store,
//         which returns natural order.
// y-lines (kz, i) are contiguous runs of n2 elements; x-lines (kz, j) have
// stride n2 and consecutive lines are adjacent. Blocks are persistent: each
// loops over tiles and copies the next tile into its second buffer (cp.async
// groups) while it transforms the current one.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T, int MODE, int L>
__global__ void __launch_bounds__(kThreads) k_fft_lines(Geom g, Ptrs<T> p, AxisPlan ap, const cx<T>* __restrict__ tw,
                                                        const T* __restrict__ rsym1, const T* __restrict__ rsym2,
                                                        const T* __restrict__ sym3, T inv_n, FastDiv dl) {
    using C = cx<T>;
    constexpr int stride = L + 1;
    constexpr int lsh = (L >= 16) ? 4 : (L >= 8) ? 3 : (L >= 4) ? 2 : (L >= 2) ? 1 : 0;
    static_assert((1 << lsh) == L, "L must be a power of two <= 16");
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = ap.n;
    C* twl = reinterpret_cast<C*>(smem_raw);
    C* buf[2];
    buf[0] = twl + n;
    buf[1] = buf[0] + (size_t)n * stride;
    for (int t = threadIdx.x; t < n; t += kThreads) twl[t] = tw[t];
    const long long plane = (long long)g.n1 * g.n2;
    const long long nlines = (MODE == 1) ? (long long)g.n3h * g.n2 : (long long)g.n3h * g.n1;
    const long long ntiles = (nlines + L - 1) / L;
    C* spec = p.spec + (size_t)s * g.Nh;
    const int cnt = L * n;
    // MODE 1: each thread keeps one line c of every tile and walks its elements
    const int cl = threadIdx.x & (L - 1);
    const int m0 = threadIdx.x >> lsh;
    constexpr int mstep = kThreads / L;
    auto issue = [&](long long t, C* b) {
        const long long l0 = t * L;
        if (MODE == 1) {
            const long long l = l0 + cl;
            if (l < nlines) {
                const int kz = (int)fdiv((unsigned)l, g.div_n2);
                const int k2 = (int)(l - (long long)kz * g.n2);
                const C* src = spec + (long long)kz * plane + k2;
                for (int m = m0; m < n; m += mstep) cp_async_cx(&b[m * stride + cl], src + (long long)m * g.n2);
            } else {
                for (int m = m0; m < n; m += mstep) b[m * stride + cl] = cmake<C>(T(0), T(0));
            }
        } else {
            for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
                const int c = (int)fdiv((unsigned)idx, g.div_n2);
                const int m = idx - c * n;
                const long long l = l0 + c;
                if (l < nlines)
                    cp_async_cx(&b[m * stride + c], spec + l * n + m);
                else
                    b[m * stride + c] = cmake<C>(T(0), T(0));
            }
        }
        cp_async_commit();
    };
    long long t = blockIdx.x;
    int cur = 0;
    if (t < ntiles) issue(t, buf[0]);
    for (; t < ntiles; t += gridDim.x) {
        const long long tn = t + gridDim.x;
        if (tn < ntiles)
            issue(tn, buf[cur ^ 1]);
        else
            cp_async_commit();   // an empty group keeps the count of pending groups at one
        cp_async_wait_one();
        __syncthreads();
        C* b = buf[cur];
        const long long l0 = t * L;
        if (MODE == 0) {
            inplace_fft<C, true, kThreads>(b, ap, L, stride, 1, dl, twl);
        } else if (MODE == 2) {
            inplace_fft<C, false, kThreads>(b, ap, L, stride, 1, dl, twl);
        } else {
            inplace_fft<C, true, kThreads>(b, ap, L, stride, 1, dl, twl);
            const long long l = l0 + cl;
            const bool valid = l < nlines;
            int kz = 0, k2 = 0;
            if (valid) {
                kz = (int)fdiv((unsigned)l, g.div_n2);
                k2 = (int)(l - (long long)kz * g.n2);
            }
            const T lam23 = valid ? rsym2[k2] + sym3[kz] : T(0);
            for (int m = m0; m < n; m += mstep) {
                const T lam = rsym1[m] + lam23;
                const T gk = (valid && lam > T(0)) ? -inv_n / lam : T(0);
                const C z = b[m * stride + cl];
                b[m * stride + cl] = cmake<C>(z.x * gk, -z.y * gk);
            }
            __syncthreads();
            inplace_fft<C, false, kThreads>(b, ap, L, stride, 1, dl, twl);
        }
        if (MODE == 1) {
            const long long l = l0 + cl;
            if (l < nlines) {
                const int kz = (int)fdiv((unsigned)l, g.div_n2);
                const int k2 = (int)(l - (long long)kz * g.n2);
                C* dst = spec + (long long)kz * plane + k2;
                for (int m = m0; m < n; m += mstep) dst[(long long)m * g.n2] = b[m * stride + cl];
            }
        } else {
            for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
                const int c = (int)fdiv((unsigned)idx, g.div_n2);
                const int m = idx - c * n;
                const long long l = l0 + c;
                if (l < nlines) {
                    const C v = b[m * stride + c];
                    spec[l * n + m] = (MODE == 2) ? cconj(v) : v;
                }
            }
        }
        __syncthreads();   // the buffer is refilled two tiles later
        cur ^= 1;
    }
}

// ---------------------------------------------------------------------------
// The same three line passes for power-of-two line lengths N (128 ... 1024), with
// one warp per line and the warp-local Stockham FFT (natural order in and out, no
// block barrier between radix passes).
// MODE 0 / 2 (y lines, contiguous): every warp takes lines on its own; the first
// radix pass reads the line from global memory and the last one writes it back
// (MODE 2 conjugated), so the line crosses shared memory only between passes.
// Latency is hidden by the resident warps (the line's loads of all lanes are in
// flight together).
// MODE 1 (x lines, stride n2): tiles of 8 lines are copied through shared memory
// cooperatively (8 adjacent lines give 64-byte row segments; cp.async into the
// second buffer while the first is transformed); the line stride is 2 mod 4
// elements so the tile copies do not conflict. MODE 1 reads the x symbol in
// natural order and the y symbol in the order the y pass left (ysym: natural
// after this kernel's MODE 0, digit-reversed after k_fft_lines).
// ---------------------------------------------------------------------------
// Blocks per SM the register budget is sized for. FP32 y passes at N <= 512 fit
// 3 blocks without spills. The x pass at N = 512 holds the whole transformed
// line in registers between its two FFTs: capped for 3 blocks it spills, and on
// GB300 2 blocks without spills are 13 % faster. FP64 and N = 1024 leave room for
// fewer blocks.
template <typename T, int MODE, int N>
constexpr int wlines_min_blocks() {
    return (sizeof(T) == 4 && N <= 512) ? ((MODE == 1 && N == 512) ? 2 : 3) : 1;
}

template <int MODE, int N>
__host__ __device__ constexpr int wlines_stride() { return N + N / 16 + (MODE == 1 ? 2 : 0); }

// -inv_n / lambda of the Poisson solve: the fast division in FP32 (relative error
// 2 ulp, far below the FP32 field noise), IEEE division in FP64.
__device__ __forceinline__ float poisson_gain(float inv_n, float lam) { return __fdividef(-inv_n, lam); }
__device__ __forceinline__ double poisson_gain(double inv_n, double lam) { return -inv_n / lam; }

template <typename T, int MODE, int N>
__global__ void __launch_bounds__(kThreads, wlines_min_blocks<T, MODE, N>())
    k_fft_wlines(Geom g, Ptrs<T> p, const cx<T>* __restrict__ tw, const T* __restrict__ xsym,
                 const T* __restrict__ ysym, const T* __restrict__ sym3, T inv_n) {
    using C = cx<T>;
    constexpr int L = kThreads / 32;              // warps per block
    constexpr int LS = wlines_stride<MODE, N>();  // padded line (wpad)
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twl = reinterpret_cast<C*>(smem_raw);
    warp_tw_fill<C, N>(twl, tw);
    C* spec = p.spec + (size_t)s * g.Nh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (MODE != 1) {
        __syncthreads();
        C* x = twl + N + warp * LS;
        const long long nlines = (long long)g.n3h * g.n1;
        const long long wstep = (long long)gridDim.x * L;
        for (long long l = (long long)blockIdx.x * L + warp; l < nlines; l += wstep) {
            C* line = spec + l * N;
            warp_fft_global<C, N, MODE == 2>(line, line, x, twl, lane);
        }
    } else {
        C* const buf0 = twl + N;
        C* const buf1 = buf0 + (size_t)L * LS;
        const long long plane = (long long)g.n1 * g.n2;
        // FP32 at N = 512: per-lane twiddles W_512^{lane k'} and the x symbol in the permuted order of
        // fft512_to_perm, loaded once for all tiles
        constexpr bool kReg512 = sizeof(T) == 4 && N == 512;
        C tw512[16];
        T xs512[16];
        if constexpr (kReg512) {
#pragma unroll
            for (int kp = 0; kp < 16; ++kp) tw512[kp] = tw[(lane * kp) & (N - 1)];
#pragma unroll
            for (int q = 0; q < 16; ++q) xs512[q] = xsym[(lane >> 1) + 16 * q + 256 * (lane & 1)];
        }
        const long long nlines = (long long)g.n3h * g.n2;
        const long long ntiles = (nlines + L - 1) / L;
        // thread (cl, m0) moves elements m0 + 32 i of line cl of a tile (64-byte row
        // segments per 8 threads): a per-thread base plus compile-time offsets
        constexpr int MSTEP = kThreads / L;
        const int cl = threadIdx.x & (L - 1);
        const int m0 = threadIdx.x / L;
        const int sb = cl * LS + wpad(m0);
        auto issue = [&](long long t, C* b) {
            const long long l = t * L + cl;
            if (l < nlines) {
                const int kz = (int)fdiv((unsigned)l, g.div_n2);
                const int k2 = (int)(l - (long long)kz * g.n2);
                const C* src = spec + (long long)kz * plane + k2 + (long long)m0 * g.n2;
                const long long st = (long long)MSTEP * g.n2;
#pragma unroll
                for (int i = 0; i < N / MSTEP; ++i) cp_async_cx(&b[sb + cpad(MSTEP * i)], src + i * st);
            } else {
#pragma unroll
                for (int i = 0; i < N / MSTEP; ++i) b[sb + cpad(MSTEP * i)] = cmake<C>(T(0), T(0));
            }
            cp_async_commit();
        };
        long long t = blockIdx.x;
        bool cur = false;
        if (t < ntiles) issue(t, buf0);
        for (; t < ntiles; t += gridDim.x) {
            C* const b = cur ? buf1 : buf0;
            const long long tn = t + gridDim.x;
            if (tn < ntiles)
                issue(tn, cur ? buf0 : buf1);
            else
                cp_async_commit();
            cp_async_wait_one();
            __syncthreads();
            const long long l0 = t * L;
            C* x = b + warp * LS;
            const long long lw = l0 + warp;
            const bool valid = lw < nlines;
            int kz = 0, k2 = 0;
            if (valid) {
                kz = (int)fdiv((unsigned)lw, g.div_n2);
                k2 = (int)(lw - (long long)kz * g.n2);
            }
            const T lam23 = valid ? ysym[k2] + sym3[kz] : T(0);
            if constexpr (kReg512) {
                // the 512-point transforms in registers with one exchange each (fft512_to_perm /
                // fft512_from_perm); the gain in the permuted order, symbol values per lane preloaded
                C u[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) u[k] = x[wpad(lane) + cpad(32 * k)];
                fft512_to_perm(u, x, tw512, lane);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const T lam = xs512[q] + lam23;
                    const T gk = (valid && lam > T(0)) ? poisson_gain(inv_n, lam) : T(0);
                    u[q] = cmake<C>(u[q].x * gk, -u[q].y * gk);   // conj: the inverse runs as conj(FFT(conj(.)))
                }
                fft512_from_perm(u, x, tw512, lane);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 16; ++k) x[wpad(lane) + cpad(32 * k)] = u[k];
            } else {
                // forward x FFT into registers (u[k] = X[lane + 32 k]), the Poisson gain,
                // then the inverse from the same registers: the spectrum line does not
                // go through shared memory in between
                C u[N / 32];
                warp_fft_to_regs<C, N>(x, twl, lane, u);
#pragma unroll
                for (int k = 0; k < N / 32; ++k) {
                    const T lam = xsym[lane + 32 * k] + lam23;
                    const T gk = (valid && lam > T(0)) ? poisson_gain(inv_n, lam) : T(0);
                    u[k] = cmake<C>(u[k].x * gk, -u[k].y * gk);   // conj: the inverse runs as conj(FFT(conj(.)))
                }
                warp_fft_from_regs<C, N>(x, twl, lane, u);
            }
            __syncthreads();
            const long long l = l0 + cl;
            if (l < nlines) {
                const int kzs = (int)fdiv((unsigned)l, g.div_n2);
                const int k2s = (int)(l - (long long)kzs * g.n2);
                C* dst = spec + (long long)kzs * plane + k2s + (long long)m0 * g.n2;
                const long long st = (long long)MSTEP * g.n2;
#pragma unroll
                for (int i = 0; i < N / MSTEP; ++i) dst[i * st] = b[sb + cpad(MSTEP * i)];
            }
            __syncthreads();
            cur = !cur;
        }
    }
}

// ---------------------------------------------------------------------------
// Fused plane pass (planes up to kPlaneMax elements): one block per (k_z, solve)
// holds the whole (x, y) plane of the half spectrum in shared memory (rows of
// n2 + 1 elements). Forward transforms along y then x run in place as
// decimation in frequency, leaving both axes in digit-reversed order; the
// Poisson symbol is applied there (tables of 4 sin^2 in digit-reversed order);
// the inverse runs as conj(DIT(conj(.))) along x then y, which returns natural
// order. No permutation pass and no second buffer are needed.
// ---------------------------------------------------------------------------
// Threads of the one-block plane pass: 1024 in FP32 (64 registers, no spills; 0.066 against 0.070 ms per
// 128^3 x 3 launch with 512 on GB300), 512 in FP64 (at 1024 the FP64 kernel spills).
template <typename T>
__host__ __device__ constexpr int plane_threads() { return sizeof(T) == 4 ? 1024 : 512; }
constexpr int kPlaneMax = 16384;

template <typename T>
__global__ void __launch_bounds__(plane_threads<T>(), 1) k_fft_plane(Geom g, Ptrs<T> p, AxisPlan ax1, AxisPlan ax2,
                                                                const cx<T>* __restrict__ tw1,
                                                                const cx<T>* __restrict__ tw2,
                                                                const T* __restrict__ rsym1,
                                                                const T* __restrict__ rsym2,
                                                                const T* __restrict__ sym3, T inv_n) {
    using C = cx<T>;
    constexpr int kPlaneThreads = plane_threads<T>();
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    const int kz = blockIdx.x;
    const int n1 = g.n1, n2 = g.n2;
    const int P2 = n2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tx = reinterpret_cast<C*>(smem_raw);
    C* ty = tx + n1;
    C* tile = ty + n2;
    for (int t = threadIdx.x; t < n1; t += kPlaneThreads) tx[t] = tw1[t];
    for (int t = threadIdx.x; t < n2; t += kPlaneThreads) ty[t] = tw2[t];
    C* spec = p.spec + (size_t)s * g.Nh + (long long)kz * n1 * n2;
    const int cnt = n1 * n2;
    for (int idx = threadIdx.x; idx < cnt; idx += kPlaneThreads) {
        const int i = (int)fdiv((unsigned)idx, g.div_n2);
        cp_async_cx(&tile[i * P2 + (idx - i * n2)], &spec[idx]);
    }
    cp_async_wait_all();
    __syncthreads();
    const FastDiv dn1 = g.div_n1, dn2 = g.div_n2;
    inplace_fft<C, true, kPlaneThreads>(tile, ax2, n1, 1, P2, dn1, ty);    // y: n1 rows
    inplace_fft<C, true, kPlaneThreads>(tile, ax1, n2, P2, 1, dn2, tx);    // x: n2 columns
    const T l3 = sym3[kz];
    for (int idx = threadIdx.x; idx < cnt; idx += kPlaneThreads) {
        const int i = (int)fdiv((unsigned)idx, g.div_n2);
        const int j = idx - i * n2;
        const T lam = rsym1[i] + rsym2[j] + l3;
        const T gk = (lam > T(0)) ? -inv_n / lam : T(0);
        const C z = tile[i * P2 + j];
        tile[i * P2 + j] = cmake<C>(z.x * gk, -z.y * gk);   // conj: the inverse runs as conj(DIT(conj))
    }
    __syncthreads();
    inplace_fft<C, false, kPlaneThreads>(tile, ax1, n2, P2, 1, dn2, tx);
    inplace_fft<C, false, kPlaneThreads>(tile, ax2, n1, 1, P2, dn1, ty);
    for (int idx = threadIdx.x; idx < cnt; idx += kPlaneThreads) {
        const int i = (int)fdiv((unsigned)idx, g.div_n2);
        spec[idx] = cconj(tile[i * P2 + (idx - i * n2)]);
    }
}

// ---------------------------------------------------------------------------
// Cluster plane pass (planes too large for one block): a thread-block cluster of
// C blocks transforms one (x, y) plane of one k_z. Block r first holds rows
// [r R1, (r + 1) R1) (R1 = n1 / C) as Y[rr][j] (row stride n2 + 1) and runs the
// forward y transforms (DIF, in place). The blocks then exchange sub-blocks
// through distributed shared memory so that block r holds columns
// [r R2, (r + 1) R2) (R2 = n2 / C) as X[cc][i] (line stride n1 + 1): each thread
// reads its elements from the owning blocks into registers, the cluster
// synchronises, and each block writes its new layout over its own buffer. The
// x transforms, the Poisson symbol (digit-reversed tables on both axes) and the
// inverse x transforms run on X; the inverse exchange returns the rows, the
// inverse y transforms run on Y and the rows are stored. Reads from another
// block always walk consecutive addresses of that block's buffer.
// ---------------------------------------------------------------------------
template <typename T> struct PlaneRegs;
template <> struct PlaneRegs<float> { static constexpr int M = 32; };    // elements per thread in an exchange
template <> struct PlaneRegs<double> { static constexpr int M = 16; };
constexpr int kPlaneClusterThreads = 512;

template <typename T, int CL>
__global__ void __launch_bounds__(kPlaneClusterThreads, 1)
    k_fft_plane_cluster(Geom g, Ptrs<T> p, AxisPlan ax1, AxisPlan ax2, const cx<T>* __restrict__ tw1,
                        const cx<T>* __restrict__ tw2, const T* __restrict__ rsym1, const T* __restrict__ rsym2,
                        const T* __restrict__ sym3, T inv_n, FastDiv dr1, FastDiv dr2) {
    using C = cx<T>;
    namespace cg = cooperative_groups;
    constexpr int NT = kPlaneClusterThreads;
    constexpr int M = PlaneRegs<T>::M;
    cg::cluster_group cluster = cg::this_cluster();
    const int s = blockIdx.y + p.s0;
    // uniform over the cluster (same solve): either every block returns here or none does
    if (!p.run_all && !p.sc[s].active) return;
    const int r = (int)cluster.block_rank();
    const int kz = blockIdx.x / CL;
    const int n1 = g.n1, n2 = g.n2;
    const int R1 = (int)dr1.d, R2 = (int)dr2.d;
    const int P2 = n2 + 1, Q = n1 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tx = reinterpret_cast<C*>(smem_raw);
    C* ty = tx + n1;
    C* buf = ty + n2;
    for (int t = threadIdx.x; t < n1; t += NT) tx[t] = tw1[t];
    for (int t = threadIdx.x; t < n2; t += NT) ty[t] = tw2[t];
    C* spec = p.spec + (size_t)s * g.Nh + (long long)kz * n1 * n2 + (long long)r * R1 * n2;
    const int E = R1 * n2;   // elements per block (= n1 * R2)
    for (int idx = threadIdx.x; idx < E; idx += NT) {
        const int rr = (int)fdiv((unsigned)idx, g.div_n2);
        cp_async_cx(&buf[rr * P2 + (idx - rr * n2)], &spec[idx]);
    }
    cp_async_wait_all();
    __syncthreads();
    inplace_fft<C, true, NT>(buf, ax2, R1, 1, P2, dr1, ty);   // y, rows of this block
    cluster.sync();
    C v[M];
    // rows -> columns: element (i, cc) of column block r sits in block q = i / R1, row i - q R1
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int e = threadIdx.x + u * NT;
        if (e < E) {
            const int i = (int)fdiv((unsigned)e, dr2);
            const int cc = e - i * R2;
            const int q = (int)fdiv((unsigned)i, dr1);
            const C* src = cluster.map_shared_rank(buf, q);
            v[u] = src[(i - q * R1) * P2 + r * R2 + cc];
        }
    }
    cluster.sync();
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int e = threadIdx.x + u * NT;
        if (e < E) {
            const int i = (int)fdiv((unsigned)e, dr2);
            buf[(e - i * R2) * Q + i] = v[u];
        }
    }
    __syncthreads();
    inplace_fft<C, true, NT>(buf, ax1, R2, 1, Q, dr2, tx);    // x, columns of this block
    const T l3 = sym3[kz];
    for (int e = threadIdx.x; e < E; e += NT) {
        const int cc = (int)fdiv((unsigned)e, g.div_n1);
        const int i = e - cc * n1;
        const T lam = rsym1[i] + rsym2[r * R2 + cc] + l3;
        const T gk = (lam > T(0)) ? -inv_n / lam : T(0);
        const C z = buf[cc * Q + i];
        buf[cc * Q + i] = cmake<C>(z.x * gk, -z.y * gk);   // conj: the inverse runs as conj(DIT(conj))
    }
    __syncthreads();
    inplace_fft<C, false, NT>(buf, ax1, R2, 1, Q, dr2, tx);
    cluster.sync();
    // columns -> rows: element (rr, j) of row block r sits in block q = j / R2, line j - q R2, slot r R1 + rr
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int e = threadIdx.x + u * NT;
        if (e < E) {
            const int j = (int)fdiv((unsigned)e, dr1);
            const int rr = e - j * R1;
            const int q = (int)fdiv((unsigned)j, dr2);
            const C* src = cluster.map_shared_rank(buf, q);
            v[u] = src[(j - q * R2) * Q + r * R1 + rr];
        }
    }
    cluster.sync();
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int e = threadIdx.x + u * NT;
        if (e < E) {
            const int j = (int)fdiv((unsigned)e, dr1);
            buf[(e - j * R1) * P2 + j] = v[u];
        }
    }
    __syncthreads();
    inplace_fft<C, false, NT>(buf, ax2, R1, 1, P2, dr1, ty);
    for (int idx = threadIdx.x; idx < E; idx += NT) {
        const int rr = (int)fdiv((unsigned)idx, g.div_n2);
        spec[idx] = cconj(buf[rr * P2 + (idx - rr * n2)]);
    }
}

// ---------------------------------------------------------------------------
// Passes 1 and 5 for power-of-two N3 (128 ... 1024): one warp per packed complex
// z line (two real lines), 8 warps = 16 real lines per block, with the
// warp-local Stockham FFT on padded lines (wpad). The spectrum is read and
// written by the whole block, 16 consecutive lines (128 contiguous bytes in FP32)
// per k_z row, instead of a few lines per block. The divergence pass needs
// N3 % 4 == 0 (FP32) / N3 % 2 == 0 (FP64) 16-byte groups, which power-of-two N3 >= 128 has.
// ---------------------------------------------------------------------------
// Blocks per SM the register budget of the divergence pass is sized for: four blocks of 256 threads
// (64 registers; the pass's shared memory allows them too) up to N3 = 512 in FP32 and 256 in FP64, two
// at 512 in FP64, one at 1024 (the register use of an unbounded build, so the bound only keeps it there).
template <typename T, int N>
constexpr int wz_min_blocks() {
    return N >= 1024 ? 1 : (sizeof(T) == 4 || N <= 256) ? 4 : 2;
}

template <typename T, int N, bool AB = false>
__global__ void __launch_bounds__(kThreads, wz_min_blocks<T, N>())
    k_div_rfft_wz(Geom g, Ptrs<T> p, const cx<T>* __restrict__ tw) {
    using C = cx<T>;
    constexpr int NW = kThreads / 32;     // packed lines per block
    constexpr int RL = 2 * NW;            // real lines per block
    constexpr int NH = N / 2 + 1;
    constexpr int LS = N + N / 16 + 1;    // padded line, odd stride between lines
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twl = reinterpret_cast<C*>(smem_raw);
    C* lines = twl + N;
    warp_tw_fill<C, N>(twl, tw);
    __syncthreads();   // the twiddle table is filled by all threads of the block, then read by every warp
    const T irho = T(1) / (T)p.sc[s].rho;
    const T h = T(0.70710678118654752440084436210485);
    const long long Nv = g.N;
    const long long cur = (long long)(p.sc[s].iters & 1) * p.sstride + (long long)s * 6 * Nv;
    const T* __restrict__ e = p.e + cur;
    const T* __restrict__ v = p.v + cur;
    const long long L = (long long)g.n1 * g.n2;
    const long long l0 = (long long)blockIdx.x * RL;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    C* x = lines + w * LS;
    // each lane takes groups of W consecutive z (16-byte loads), groups 32 W apart
    constexpr int W = Vec16<T>::W;
    constexpr int G = N / (32 * W);      // groups per lane
    static_assert(G >= 1, "line too short for the warp z pass");
    // Group by group, both lines of the pair: a line's y-neighbour rows are the other line of
    // the pair and the neighbouring warps' lines, so they are read again while still in cache.
    // (Line by line, at N3 = 512 the y-neighbour rows were evicted between the neighbour read and
    // the line's own read and came back from DRAM.)
    RowNb rnq[2];
    bool validq[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const long long l = l0 + 2 * w + q;
        validq[q] = l < L;
        rnq[q] = row_neighbours(g, (unsigned)(validq[q] ? l : 0));
    }
#pragma unroll 1
    for (int t = 0; t < G; ++t) {   // one group at a time keeps the registers low
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const bool valid = validq[q];
            const RowNb& rn = rnq[q];
            const int k0 = W * lane + 32 * W * t;
            T d[W];
#pragma unroll
            for (int u = 0; u < W; ++u) d[u] = T(0);
            if (AB && valid) {
                // stored divergences of the state: d = a - b / rho
                const T* a = p.ab + (size_t)s * 2 * Nv + rn.row + k0;
                T ta[W], tb[W];
                Vec16<T>::ld(a, ta);
                Vec16<T>::ld(a + Nv, tb);
#pragma unroll
                for (int u = 0; u < W; ++u) d[u] = ta[u] - tb[u] * irho;
            } else if (valid) {
                const int kp = (k0 + W == N) ? 0 : k0 + W;   // first voxel after the group
                const int km = (k0 == 0) ? N - 1 : k0 - 1;   // last voxel before the group
                T wv[6][W], te[W], tv[W];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    Vec16<T>::ld(e + c * Nv + rn.row + k0, te);
                    Vec16<T>::ld(v + c * Nv + rn.row + k0, tv);
#pragma unroll
                    for (int u = 0; u < W; ++u) wv[c][u] = te[u] - tv[u] * irho;
                }
                T xp[W], xm[W], yp[W], ym[W];
                Vec16<T>::ld(e + 3 * Nv + rn.ip + k0, te);
                Vec16<T>::ld(v + 3 * Nv + rn.ip + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) xp[u] = te[u] - tv[u] * irho;
                Vec16<T>::ld(e + 0 * Nv + rn.im + k0, te);
                Vec16<T>::ld(v + 0 * Nv + rn.im + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) xm[u] = te[u] - tv[u] * irho;
                Vec16<T>::ld(e + 4 * Nv + rn.jp + k0, te);
                Vec16<T>::ld(v + 4 * Nv + rn.jp + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) yp[u] = te[u] - tv[u] * irho;
                Vec16<T>::ld(e + 1 * Nv + rn.jm + k0, te);
                Vec16<T>::ld(v + 1 * Nv + rn.jm + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) ym[u] = te[u] - tv[u] * irho;
                const T zp = __ldg(e + 5 * Nv + rn.row + kp) - __ldg(v + 5 * Nv + rn.row + kp) * irho;
                const T zm = __ldg(e + 2 * Nv + rn.row + km) - __ldg(v + 2 * Nv + rn.row + km) * irho;
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const T w2zp = (u + 1 < W) ? wv[5][(u + 1) % W] : zp;
                    const T w1zm = (u > 0) ? wv[2][(u + W - 1) % W] : zm;
                    const T sx = wv[0][u] - xm[u] + xp[u] - wv[3][u];
                    const T sy = wv[1][u] - ym[u] + yp[u] - wv[4][u];
                    const T sz = wv[2][u] - w1zm + w2zp - wv[5][u];
                    d[u] = h * (sx + sy + sz);
                }
            }
            // line 2w + q is the real (q = 0) or imaginary (q = 1) part of packed line w
#pragma unroll
            for (int u = 0; u < W; ++u) {
                T* xr = reinterpret_cast<T*>(&x[wpad(k0 + u)]);
                xr[q] = d[u];
            }
        }
    }
    __syncwarp();
    warp_fft<C, N>(x, twl, lane);
    __syncthreads();
    // half spectrum, k_z-major: line pair (2c, 2c + 1) from Z(k) and conj Z(N - k) of packed line c
    C* spec = p.spec + (size_t)s * g.Nh;
    for (int idx = threadIdx.x; idx < NH * RL; idx += kThreads) {
        const int kz = idx / RL, t = idx % RL;
        const long long l = l0 + t;
        if (l >= L) continue;
        const C* xc = lines + (t >> 1) * LS;
        const C Z = xc[wpad(kz)];
        const C Zm = cconj(xc[wpad(kz == 0 ? 0 : N - kz)]);
        const C Sm = cadd(Z, Zm), D = csub(Z, Zm);
        spec[(long long)kz * L + l] = (t & 1) ? cmake<C>(T(0.5) * D.y, T(-0.5) * D.x)
                                              : cmake<C>(T(0.5) * Sm.x, T(0.5) * Sm.y);
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_irfft_wz(Geom g, Ptrs<T> p, const cx<T>* __restrict__ tw) {
    using C = cx<T>;
    constexpr int NW = kThreads / 32;
    constexpr int RL = 2 * NW;
    constexpr int RLP = RL + 1;           // padded slab row (consecutive k_z in distinct banks)
    constexpr int NH = N / 2 + 1;
    constexpr int LS = N + N / 16 + 1;
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twl = reinterpret_cast<C*>(smem_raw);
    // the slab [NH][RLP] of the block's spectrum rows; once the lanes hold their
    // elements in registers the same memory serves as the warps' scratch lines
    C* raw = twl + N;
    C* lines = raw;
    warp_tw_fill<C, N>(twl, tw);
    const long long L = (long long)g.n1 * g.n2;
    const long long l0 = (long long)blockIdx.x * RL;
    const C* spec = p.spec + (size_t)s * g.Nh;
    for (int idx = threadIdx.x; idx < NH * RL; idx += kThreads) {
        const int kz = idx / RL, t = idx % RL;
        const long long l = l0 + t;
        if (l < L)
            cp_async_cx(&raw[kz * RLP + t], spec + (long long)kz * L + l);
        else
            raw[kz * RLP + t] = cmake<C>(T(0), T(0));
    }
    cp_async_wait_all();
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    C* x = lines + w * LS;
    // element m = lane + 32 k of packed line w, straight into registers:
    // Z(m) = conj(a + i b) from slab row m for m <= N / 2 (a, b the spectra of the
    // line pair), conj(conj(a) + i conj(b)) from row N - m above
    C u[N / 32];
#pragma unroll
    for (int k = 0; k < N / 32; ++k) {
        const int m = lane + 32 * k;
        if (2 * m <= N) {
            const C a = raw[m * RLP + 2 * w], b = raw[m * RLP + 2 * w + 1];
            u[k] = (m == 0 || 2 * m == N) ? cmake<C>(a.x, -b.x)                   // Z = Re(a) + i Re(b), conjugated
                                          : cmake<C>(a.x - b.y, -(a.y + b.x));
        } else {
            const int mm = N - m;
            const C a = raw[mm * RLP + 2 * w], b = raw[mm * RLP + 2 * w + 1];
            u[k] = cmake<C>(a.x + b.y, a.y - b.x);
        }
    }
    __syncthreads();   // the slab is read out: its memory becomes the scratch lines
    warp_fft_regs<C, N>(x, twl, lane, u);
    // real line 2w is Re, line 2w + 1 is -Im of the result (the conjugated inverse)
    T* phi = p.phi + (size_t)s * g.N;
    const long long la = l0 + 2 * w;
#pragma unroll
    for (int k = 0; k < N / 32; ++k) {
        if (la < L) phi[la * N + lane + 32 * k] = u[k].x;
        if (la + 1 < L) phi[(la + 1) * N + lane + 32 * k] = -u[k].y;
    }
}

// ---------------------------------------------------------------------------
// Pass 5: complex-to-real inverse FFT along z, two real lines per transform.
// ---------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_irfft_z(Geom g, Ptrs<T> p, AxisPlan az,
                                                      const cx<T>* __restrict__ tw) {
    using C = cx<T>;
    constexpr int stride = P + 1;
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twl = reinterpret_cast<C*>(smem_raw);
    C* A = twl + g.n3;
    C* B = A + (size_t)g.n3 * stride;
    for (int t = threadIdx.x; t < g.n3; t += kThreads) twl[t] = tw[t];
    const long long L = (long long)g.n1 * g.n2;
    const long long l0 = (long long)blockIdx.x * 2 * P;
    const C* spec = p.spec + (size_t)s * g.Nh;
    const int cnt = P * g.n3h;
    // stage the raw slab spec[kz][l0 .. l0 + 2P) in the second buffer with asynchronous
    // copies when it fits there (2P <= n3), then build the packed lines from shared memory
    const bool staged = 2 * P <= g.n3;
    if (staged) {
        for (int idx = threadIdx.x; idx < 2 * cnt; idx += kThreads) {
            const int kz = idx / (2 * P);
            const int t = idx - kz * 2 * P;
            const long long l = l0 + t;
            if (l < L)
                cp_async_cx(&B[idx], spec + (long long)kz * L + l);
            else
                B[idx] = cmake<C>(T(0), T(0));
        }
        cp_async_wait_all();
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int kz = idx / P;
        const int c = idx - kz * P;
        const long long la = l0 + 2 * c, lb = la + 1;
        const C* src = spec + (long long)kz * L + la;
        C a, b;
        if (staged) {
            a = B[kz * 2 * P + 2 * c];
            b = B[kz * 2 * P + 2 * c + 1];
        } else {
            a = (la < L) ? src[0] : cmake<C>(T(0), T(0));
            b = (lb < L) ? src[1] : cmake<C>(T(0), T(0));
        }
        if (kz == 0 || 2 * kz == g.n3) {
            // Z = Re(a) + i Re(b); store conj(Z)
            A[kz * stride + c] = cmake<C>(a.x, -b.x);
        } else {
            // Z[kz] = a + i b ; Z[n3 - kz] = conj(a) + i conj(b); store conjugates
            A[kz * stride + c] = cmake<C>(a.x - b.y, -(a.y + b.x));
            A[(g.n3 - kz) * stride + c] = cmake<C>(a.x + b.y, a.y - b.x);
        }
    }
    __syncthreads();
    C* R = block_fft<C, P>(A, B, az, twl);
    const int cnt2 = 2 * P * g.n3;
    T* phi = p.phi + (size_t)s * g.N;
    for (int idx = threadIdx.x; idx < cnt2; idx += kThreads) {
        const int ll = (int)fdiv((unsigned)idx, g.div_n3);
        const int k = idx - ll * g.n3;
        const long long l = l0 + ll;
        if (l < L) {
            const C z = R[k * stride + (ll >> 1)];
            phi[l * g.n3 + k] = (ll & 1) ? -z.y : z.x;
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 6: projection completion, node-wise projection, multiplier update and
// reductions; the last block of each solve runs the penalty / stop logic.
// ---------------------------------------------------------------------------
template <typename T>
struct StepConsts {
    T rho, irho, h, alpha, beta;
    T xi[3];
};

// Projection helpers. FP64 uses correctly rounded sqrt and division, as the
// FP64 path is compared with the oracle at the 1e-10 level. FP32 uses the
// hardware reciprocal square root (relative error ~1e-7, below FP32 field noise):
// scale = gamma / |z| when |z| > gamma is gamma * rsqrt(|z|^2), compared in squares.
template <typename T> struct Proj;
template <> struct Proj<double> {
    __device__ __forceinline__ static double scale(double nz2, double gm) {
        const double nz = sqrt(nz2);
        return (nz > gm) ? gm / nz : 1.0;
    }
    __device__ __forceinline__ static double norm(double x2) { return sqrt(x2); }
};
template <> struct Proj<float> {
    __device__ __forceinline__ static float scale(float nz2, float gm) {
        return (nz2 > gm * gm) ? gm * rsqrtf(nz2) : 1.0f;
    }
    __device__ __forceinline__ static float norm(float x2) { return x2 > 0.0f ? x2 * rsqrtf(x2) : 0.0f; }
};

// Per-voxel work of the update pass. Inputs: the voxel's own state (ec, vc),
// gamma, phi at the voxel and at p +- e_a, and the neighbour state components
// the stencil needs: e/v of w2_a at p + e_a and of w1_a at p - e_a.
// RULE selects which penalty sums are accumulated (0 BB, 1 constant, 2 LTD,
// -1 all of them).
template <typename T, bool OUT, int RULE = -1>
__device__ __forceinline__ void voxel_step(const StepConsts<T>& K, const T (&ec)[6], const T (&vc)[6], T gm, T ph0,
                                           const T (&php)[3], const T (&phm)[3], const T (&e2p)[3],
                                           const T (&v2p)[3], const T (&e1m)[3], const T (&v1m)[3],
                                           T (&acc)[kNSum], T (&eo)[6], T (&vo)[6], T (&flow)[3],
                                           T* zo = nullptr, bool count = true) {
    T w[6], xh[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) w[c] = ec[c] - vc[c] * K.irho;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T w2p = e2p[a] - v2p[a] * K.irho;   // w2_a(p + e_a)
        const T w1m = e1m[a] - v1m[a] * K.irho;   // w1_a(p - e_a)
        const T ua = K.h * (w[a] + w2p);          // (A* w)_a(p)
        const T uam = K.h * (w1m + w[3 + a]);     // (A* w)_a(p - e_a)
        const T ya = ua - (php[a] - ph0) - K.xi[a];
        const T yam = uam - (ph0 - phm[a]) - K.xi[a];
        xh[a] = w[a] - K.h * ya;
        xh[3 + a] = w[3 + a] - K.h * yam;
    }
    T r2 = T(0), nx2 = T(0);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const T dd = ec[c] - xh[c];
        r2 += dd * dd;
        nx2 += xh[c] * xh[c];
        if (count) acc[kSumV + c] += vc[c];
    }
    if (count) {
        acc[kSumRes] += r2;
        acc[kSumPrimal] += gm * Proj<T>::norm(nx2);
    }
    if (OUT) {
#pragma unroll
        for (int c = 0; c < 6; ++c) eo[c] = xh[c];                   // the cut xi^{K+1/2}
#pragma unroll
        for (int a = 0; a < 3; ++a) flow[a] = K.h * (vc[a] + v2p[a]);  // A* v
    } else {
        T z[6];
        T nz2 = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            z[c] = vc[c] + K.rho * (K.alpha * xh[c] - K.beta * ec[c]);
            nz2 += z[c] * z[c];
        }
        if (zo) {
#pragma unroll
            for (int c = 0; c < 6; ++c) zo[c] = z[c];
        }
        const T scale = Proj<T>::scale(nz2, gm);
        T dvde = T(0), dede = T(0), dvdv = T(0), vv = T(0), ee = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const T vn = z[c] * scale;
            const T en = (z[c] - vn) * K.irho;
            if (RULE == 0 || RULE == -1) {
                const T dv = vn - vc[c], de = en - ec[c];
                dvde += dv * de;
                dede += de * de;
                dvdv += dv * dv;
            }
            if (RULE == 2 || RULE == -1) {
                vv += vn * vn;
                ee += en * en;
            }
            eo[c] = en;
            vo[c] = vn;
        }
        if (count) {
            acc[kSumDvDe] += dvde;
            acc[kSumDeDe] += dede;
            acc[kSumDvDv] += dvdv;
            acc[kSumVV] += vv;
            acc[kSumEE] += ee;
        }
    }
}

// Reduction epilogue of the update pass: block partials, then the last block of
// the solve reduces them in double and runs the penalty / history / stop logic.
template <typename T, bool OUT, int NT = kThreads, bool AB = false>
__device__ void update_finish(const Geom& g, const Ptrs<T>& p, const LoopConfig& cfg, SolveScalars& S, int s,
                              double rho_d, const double* part, int nparts);

template <typename T, bool OUT, int NT = kThreads>
__device__ void update_epilogue(const Geom& g, const Ptrs<T>& p, const LoopConfig& cfg, SolveScalars& S, int s,
                                double rho_d, T (&acc)[kNSum]) {
    const int nblocks = gridDim.x;
    double* part = p.partial + (size_t)s * nblocks * kNSum;
    const bool last = block_partials<T, kNSum, NT>(acc, part, &S.counter, nblocks, blockIdx.x);
    if (!last) return;
    update_finish<T, OUT, NT>(g, p, cfg, S, s, rho_d, part, nblocks);
}

// The last block of a solve's update pass: reduce the nparts partials in a fixed
// order, then the penalty rule, the history row and the stop decision.
template <typename T, bool OUT, int NT, bool AB>
__device__ void update_finish(const Geom& g, const Ptrs<T>& p, const LoopConfig& cfg, SolveScalars& S, int s,
                              double rho_d, const double* part, int nparts) {
    double sums[kNSum];
    reduce_partials<kNSum, NT>(part, nparts, sums);
    if (threadIdx.x != 0) return;
    S.counter = 0;
    S.chunk = 0;   // every block has left its work loop: the next launch starts from ticket 0
    const double Nd = (double)g.N;
    bool finite = true;
    for (int q = 0; q < kNSum; ++q) {
        S.sums[q] = sums[q];
        finite = finite && isfinite(sums[q]);
    }
    const double r = sqrt(fmax(sums[kSumRes], 0.0) / Nd);
    double mv2 = 0.0;
    for (int c = 0; c < 6; ++c) mv2 += (sums[kSumV + c] / Nd) * (sums[kSumV + c] / Nd);
    const double mv = sqrt(mv2);
    const double prim = sums[kSumPrimal] / Nd;
    S.residual = r;
    S.mean_v = mv;
    S.primal = prim;
    if (OUT) {
        const double hd = 0.70710678118654752440084436210485;
        double dual = 0.0;
        for (int a = 0; a < 3; ++a) dual += S.xi[a] * hd * (sums[kSumV + a] + sums[kSumV + 3 + a]) / Nd;
        S.dual = dual;
        if (!finite && S.status == 0) S.status = 5;
        return;
    }
    const int kk = S.iters;
    if (cfg.hist_len > 0) {
        double* hrow = p.hist + ((size_t)s * kHistCap + (kk % cfg.hist_len)) * kHistFields;
        hrow[0] = (double)kk;
        hrow[1] = rho_d;
        hrow[2] = r;
        hrow[3] = mv;
        hrow[4] = prim;
        const double hd = 0.70710678118654752440084436210485;
        double dual = 0.0;   // <xi_bar, mean A* v^k>, the max-flow value of Eq. 12 at iteration k
        for (int a = 0; a < 3; ++a) dual += S.xi[a] * hd * (sums[kSumV + a] + sums[kSumV + 3 + a]) / Nd;
        hrow[5] = dual;
    }
    double rho_new = rho_d;
    const double lo = rho_d / cfg.rho_step_max, hi = rho_d * cfg.rho_step_max;
    if (cfg.rho_sched) {
        if (kk + 1 < cfg.sched_len) rho_new = cfg.rho_sched[(size_t)s * cfg.sched_len + kk + 1];
    } else if (cfg.rho_rule == 0) {
        const double sve = sums[kSumDvDe], see = sums[kSumDeDe], svv = sums[kSumDvDv];
        if (sve > 0.0 && see > 0.0 && svv > 0.0 && sve / sqrt(svv * see) > cfg.bb_corr_min)
            rho_new = fmin(fmax(sve / see, lo), hi);
    } else if (cfg.rho_rule == 2) {
        const double nv = sqrt(sums[kSumVV]), ne = sqrt(sums[kSumEE]);
        if (nv > 0.0 && ne > 0.0) rho_new = fmin(fmax(nv / ne, lo), hi);
    } else if (cfg.rho_rule == 3) {
        // residual balancing: primal residual r (Eq. 31) against rho |e^{k+1} - e^k|
        const double sd = rho_d * sqrt(fmax(sums[kSumDeDe], 0.0) / Nd);
        if (r > 10.0 * sd)
            rho_new = hi;
        else if (sd > 10.0 * r)
            rho_new = lo;
    }
    const int done = kk + 1 - S.call_start;
    S.iters = kk + 1;
    S.ab_iter = AB ? kk + 1 : -1;   // whether the pass also wrote the divergences of the new state
    bool stop = false;
    if (S.status != 0) {
        stop = true;   // a failure recorded during the pass (e.g. a bounded wait that gave up)
    } else if (!finite || !isfinite(rho_new) || !(rho_new > 0.0)) {
        S.status = 5;  // CCMF_ERR_NUMERICAL: rho and the state are left as they are
        stop = true;
    } else {
        S.rho = rho_new;
        if (cfg.fixed_iters > 0) {
            stop = done >= cfg.fixed_iters;
        } else if (kk >= 1 && r <= cfg.tol * mv) {
            S.converged = 1;
            stop = true;
        } else if (done >= cfg.max_iter) {
            stop = true;
        }
    }
    if (stop) {
        S.active = 0;
        atomicSub(p.n_active, 1);
    }
}

template <typename T>
__device__ __forceinline__ StepConsts<T> step_consts(const SolveScalars& S, const LoopConfig& cfg) {
    StepConsts<T> K;
    K.rho = (T)S.rho;
    K.irho = T(1) / K.rho;
    K.h = T(0.70710678118654752440084436210485);
    K.alpha = (T)(2.0 * (1.0 - cfg.delta));
    K.beta = (T)(1.0 - 2.0 * cfg.delta);
    K.xi[0] = (T)S.xi[0];
    K.xi[1] = (T)S.xi[1];
    K.xi[2] = (T)S.xi[2];
    return K;
}

// Scalar version (any N3, unaligned inputs, and the final evaluation pass).
template <typename T, bool OUT>
__global__ void __launch_bounds__(kThreads) k_update(Geom g, Ptrs<T> p, LoopConfig cfg) {
    const int s = blockIdx.y + p.s0;
    SolveScalars& S = p.sc[s];
    if (!OUT && !S.active) return;
    const long long N = g.N;
    const double rho_d = S.rho;
    const StepConsts<T> K = step_consts<T>(S, cfg);
    // read the current copy of the state, write the other one (the stencil reads
    // neighbours, so an in-place update would race)
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ phi = p.phi + (size_t)s * N;
    const T* __restrict__ gam = gamma_of(p, s);
    T acc[kNSum];
#pragma unroll
    for (int q = 0; q < kNSum; ++q) acc[q] = T(0);
    const long long gstride = (long long)gridDim.x * kThreads;
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < N; lin += gstride) {
        const unsigned row = fdiv((unsigned)lin, g.div_n3);
        const int k = (int)(lin - (long long)row * g.n3);
        const RowNb rn = row_neighbours(g, row);
        const int kp = (k + 1 == g.n3) ? 0 : k + 1, km = (k == 0) ? g.n3 - 1 : k - 1;
        const long long nb_p[3] = {rn.ip + k, rn.jp + k, rn.row + kp};
        const long long nb_m[3] = {rn.im + k, rn.jm + k, rn.row + km};
        T ec[6], vc[6], php[3], phm[3], e2p[3], v2p[3], e1m[3], v1m[3];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            ec[c] = e[c * N + lin];
            vc[c] = v[c * N + lin];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            php[a] = phi[nb_p[a]];
            phm[a] = phi[nb_m[a]];
            e2p[a] = e[(3 + a) * N + nb_p[a]];
            v2p[a] = v[(3 + a) * N + nb_p[a]];
            e1m[a] = e[a * N + nb_m[a]];
            v1m[a] = v[a * N + nb_m[a]];
        }
        T eo[6], vo[6], fl[3], zz[6];
        voxel_step<T, OUT>(K, ec, vc, gam[lin], phi[lin], php, phm, e2p, v2p, e1m, v1m, acc, eo, vo, fl,
                           (!OUT && p.zout) ? zz : nullptr);
        if (!OUT && p.zout) {
            // the pre-projection point z = v + rho xi of this update, kept for the reverse pass
            T* zo = p.zout + (size_t)s * 6 * N;
#pragma unroll
            for (int c = 0; c < 6; ++c) zo[c * N + lin] = zz[c];
        }
        if (OUT) {
            if (p.cut) {
                T* cut = p.cut + (size_t)s * 6 * N;
#pragma unroll
                for (int c = 0; c < 6; ++c) cut[c * N + lin] = eo[c];
            }
            if (p.flow) {
                T* flow = p.flow + (size_t)s * 3 * N;
#pragma unroll
                for (int a = 0; a < 3; ++a) flow[a * N + lin] = fl[a];
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                e_out[c * N + lin] = eo[c];
                v_out[c * N + lin] = vo[c];
            }
        }
    }
    update_epilogue<T, OUT>(g, p, cfg, S, s, rho_d, acc);
}

// VW consecutive elements of the field type with one aligned load / store.
template <typename T, int VW> struct VecN;
template <> struct VecN<float, 4> {
    __device__ __forceinline__ static void ld(const float* __restrict__ p, float (&o)[4]) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
    __device__ __forceinline__ static void st(float* p, const float (&o)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct VecN<float, 2> {
    __device__ __forceinline__ static void ld(const float* __restrict__ p, float (&o)[2]) {
        const float2 t = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = t.x; o[1] = t.y;
    }
    __device__ __forceinline__ static void st(float* p, const float (&o)[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    }
};
template <> struct VecN<float, 1> {
    __device__ __forceinline__ static void ld(const float* __restrict__ p, float (&o)[1]) { o[0] = __ldg(p); }
    __device__ __forceinline__ static void st(float* p, const float (&o)[1]) { p[0] = o[0]; }
};
template <> struct VecN<double, 2> {
    __device__ __forceinline__ static void ld(const double* __restrict__ p, double (&o)[2]) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = t.x; o[1] = t.y;
    }
    __device__ __forceinline__ static void st(double* p, const double (&o)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
};
template <> struct VecN<double, 1> {
    __device__ __forceinline__ static void ld(const double* __restrict__ p, double (&o)[1]) { o[0] = __ldg(p); }
    __device__ __forceinline__ static void st(double* p, const double (&o)[1]) { p[0] = o[0]; }
};

// Vector version of the advancing update: W consecutive voxels of a z line per
// thread, 16-byte loads and stores (N3 % W == 0, 16-byte aligned gamma). The
// instantiation with half the voxels per thread (8-byte vectors in FP32) needs about
// half the registers and runs two blocks per SM (update variant 11).
template <typename T, bool OUT, int W = Vec16<T>::W, int MINB = 1>
__global__ void __launch_bounds__(kThreads, MINB) k_update_vec(Geom g, Ptrs<T> p, LoopConfig cfg) {
    using V = VecN<T, W>;
    const int s = blockIdx.y + p.s0;
    SolveScalars& S = p.sc[s];
    if (!OUT && !S.active) return;
    const long long N = g.N;
    const double rho_d = S.rho;
    const StepConsts<T> K = step_consts<T>(S, cfg);
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ phi = p.phi + (size_t)s * N;
    const T* __restrict__ gam = gamma_of(p, s);
    const long long ngroups = N / W;
    // Dynamic schedule: blocks take chunks of kVecChunkGroups x kThreads groups (32 rows at
    // N3 = 512) in order from a per-solve ticket counter, the next ticket fetched while the
    // current chunk runs. The chunks in flight then form one narrow front through the grid, and
    // the x- and y-neighbour rows a chunk reads were read as other chunks' own rows moments
    // before, so they come from L2. (With a grid-stride loop the blocks drift apart over a long
    // pass; at 512^3, 42 % more than the algorithmic reads came from DRAM.) Each chunk stores its
    // own partial sums and the last block reduces them in chunk order, so the result does not
    // depend on which block took which chunk.
    const long long nchunks = vec_update_chunks(N, W);
    double* part = p.partial + (size_t)s * nchunks * kNSum;
    __shared__ unsigned ticket[2];
    if (threadIdx.x == 0) ticket[0] = atomicAdd(&S.chunk, 1u);
    __syncthreads();
    for (int it = 0;; ++it) {
        const unsigned ck = ticket[it & 1];
        if (ck >= nchunks) break;   // the same value for the whole block
        if (threadIdx.x == 0) ticket[(it + 1) & 1] = atomicAdd(&S.chunk, 1u);
        T acc[kNSum];
#pragma unroll
        for (int q = 0; q < kNSum; ++q) acc[q] = T(0);
#pragma unroll 1
        for (int gi = 0; gi < kVecChunkGroups; ++gi) {
            const long long q = ((long long)ck * kVecChunkGroups + gi) * kThreads + threadIdx.x;
            if (q < ngroups) {
                const long long lin0 = q * W;
                const unsigned row = fdiv((unsigned)lin0, g.div_n3);
                const int k0 = (int)(lin0 - (long long)row * g.n3);
                const RowNb rn = row_neighbours(g, row);
                const int kp = (k0 + W == g.n3) ? 0 : k0 + W;
                const int km = (k0 == 0) ? g.n3 - 1 : k0 - 1;
                T ec[6][W], vc[6][W];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    V::ld(e + c * N + lin0, ec[c]);
                    V::ld(v + c * N + lin0, vc[c]);
                }
                T gm[W], ph[W];
                V::ld(gam + lin0, gm);
                V::ld(phi + lin0, ph);
                // x and y neighbours (whole groups), z neighbours inside the group or one scalar each side
                T e2x[W], v2x[W], e1x[W], v1x[W], e2y[W], v2y[W], e1y[W], v1y[W];
                T phxp[W], phxm[W], phyp[W], phym[W];
                V::ld(e + 3 * N + rn.ip + k0, e2x);
                V::ld(v + 3 * N + rn.ip + k0, v2x);
                V::ld(e + 0 * N + rn.im + k0, e1x);
                V::ld(v + 0 * N + rn.im + k0, v1x);
                V::ld(e + 4 * N + rn.jp + k0, e2y);
                V::ld(v + 4 * N + rn.jp + k0, v2y);
                V::ld(e + 1 * N + rn.jm + k0, e1y);
                V::ld(v + 1 * N + rn.jm + k0, v1y);
                V::ld(phi + rn.ip + k0, phxp);
                V::ld(phi + rn.im + k0, phxm);
                V::ld(phi + rn.jp + k0, phyp);
                V::ld(phi + rn.jm + k0, phym);
                const T e2z_after = __ldg(e + 5 * N + rn.row + kp), v2z_after = __ldg(v + 5 * N + rn.row + kp);
                const T e1z_before = __ldg(e + 2 * N + rn.row + km), v1z_before = __ldg(v + 2 * N + rn.row + km);
                const T ph_after = __ldg(phi + rn.row + kp), ph_before = __ldg(phi + rn.row + km);
                T eo[6][W], vo[6][W], fo[3][W];
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    T ecu[6], vcu[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        ecu[c] = ec[c][u];
                        vcu[c] = vc[c][u];
                    }
                    const bool last = (u + 1 == W), first = (u == 0);
                    const T php[3] = {phxp[u], phyp[u], last ? ph_after : ph[(u + 1) % W]};
                    const T phm[3] = {phxm[u], phym[u], first ? ph_before : ph[(u + W - 1) % W]};
                    const T e2p[3] = {e2x[u], e2y[u], last ? e2z_after : ec[5][(u + 1) % W]};
                    const T v2p[3] = {v2x[u], v2y[u], last ? v2z_after : vc[5][(u + 1) % W]};
                    const T e1m[3] = {e1x[u], e1y[u], first ? e1z_before : ec[2][(u + W - 1) % W]};
                    const T v1m[3] = {v1x[u], v1y[u], first ? v1z_before : vc[2][(u + W - 1) % W]};
                    T eou[6], vou[6], fl[3];
                    voxel_step<T, OUT>(K, ecu, vcu, gm[u], ph[u], php, phm, e2p, v2p, e1m, v1m, acc, eou, vou, fl);
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        eo[c][u] = eou[c];
                        vo[c][u] = vou[c];
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a) fo[a][u] = fl[a];
                }
                if (OUT) {
                    // final evaluation: the cut xi^{K+1/2} and the flow A* v^K
                    if (p.cut) {
                        T* cut = p.cut + (size_t)s * 6 * N;
#pragma unroll
                        for (int c = 0; c < 6; ++c) V::st(cut + c * N + lin0, eo[c]);
                    }
                    if (p.flow) {
                        T* flow = p.flow + (size_t)s * 3 * N;
#pragma unroll
                        for (int a = 0; a < 3; ++a) V::st(flow + a * N + lin0, fo[a]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        V::st(e_out + c * N + lin0, eo[c]);
                        V::st(v_out + c * N + lin0, vo[c]);
                    }
                }
            }
        }
        block_store_partial<T, kNSum>(acc, part, ck);
        __syncthreads();   // the next ticket is visible, this one is read by everyone, red[] is free
    }
    if (block_ticket(&S.counter, gridDim.x)) update_finish<T, OUT>(g, p, cfg, S, s, rho_d, part, (int)nchunks);
}


// ---------------------------------------------------------------------------
// Stored-divergence schedule (update variants 8 and 9). By Eq. 28 and Eq. 30 the
// divergence the first pass needs is linear in the state: d = div^- A* (e - v / rho)
// = a - b / rho with a = div^- A* e and b = div^- A* v. This update pass writes a and
// b of the state it produces, so the first pass of the next iteration reads two
// scalars per voxel instead of the twelve state components.
//
// div^- A* of the new state at voxel p takes, besides p itself, component 1a of the
// voxel p - e_a and component 2a of p + e_a (the backward divergence of Sec. 2.2 applied
// to A* of Eq. 17), i.e. updates of the six neighbours. A block owns tj consecutive y
// rows of whole z rows (warps 1 .. tj; warps 0 and tj + 1 recompute the updates of the
// rows just outside) and sweeps x over a segment of slabs, recomputing the slab before
// and after the segment. The x terms wait one slab in shared memory (pending sums and
// the component 1x of the previous slab), the y terms go through shared memory between
// warps, the z terms between lanes (across the passes of a row, the first and last
// voxels of a pass are completed by a fix-up in the next pass / at the end of the row).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t ab_smem_elems(int tj, int n3, int nw, int vw) {
    return 4 * (size_t)tj * n3 + 2 * (size_t)nw * 4 * 32 * vw;
}

template <typename T, int VAR>
__global__ void __launch_bounds__(AbVariant<T, VAR>::NW * 32, AbVariant<T, VAR>::MINB)
    k_update_ab(Geom g, Ptrs<T> p, LoopConfig cfg, AbShape ab) {
    constexpr int NW = AbVariant<T, VAR>::NW, VW = AbVariant<T, VAR>::VW;
    constexpr int NT = NW * 32, KZ = 32 * VW;
    using V = VecN<T, VW>;
    const int s = blockIdx.y + p.s0;
    SolveScalars& S = p.sc[s];
    if (!S.active) return;
    const long long N = g.N;
    const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
    const double rho_d = S.rho;
    const StepConsts<T> K = step_consts<T>(S, cfg);
    const T h = K.h;
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ phi = p.phi + (size_t)s * N;
    const T* __restrict__ gam = gamma_of(p, s);
    T* __restrict__ a_out = p.ab + (size_t)s * 2 * N;
    T* __restrict__ b_out = a_out + N;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tj = ab.tj;
    const int q = (int)(blockIdx.x % (unsigned)ab.nq), r = (int)(blockIdx.x / (unsigned)ab.nq);
    const int j0 = q * tj;
    const int nint = min(tj, n2 - j0);
    const bool active_w = w <= nint + 1;              // warp-uniform
    const bool interior_row = w >= 1 && w <= nint;    // warp-uniform (the recomputed rows 0, nint + 1
                                                      // are needed for interior slabs only)
    int j = j0 - 1 + w;
    if (j < 0) j += n2;
    if (j >= n2) j -= n2;
    if (j >= n2) j -= n2;
    const int jp = (j + 1 == n2) ? 0 : j + 1, jm = (j == 0) ? n2 - 1 : j - 1;
    const int i0 = r * ab.xs, i1 = min(i0 + ab.xs, n1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* pe = reinterpret_cast<T*>(smem_raw);     // pending a of the current slab, [tj][n3] (slot order)
    T* pv = pe + (size_t)tj * n3;               // pending b
    T* ex = pv + (size_t)tj * n3;               // component 1x of e' of the previous slab
    T* vx = ex + (size_t)tj * n3;               // component 1x of v'
    // [2][NW][4][KZ]: e'1y, e'2y, v'1y, v'2y of a pass, two buffers alternating by pass, so
    // that one barrier per pass separates a buffer's writes from its reads and its reads
    // (pass q) from its next writes (pass q + 2)
    T* yb2 = vx + (size_t)tj * n3;
    const size_t rbase = (size_t)(w - 1) * n3;  // this warp's row of the pending arrays
    T acc[kNSum];
#pragma unroll
    for (int qq = 0; qq < kNSum; ++qq) acc[qq] = T(0);
    T carry_e = T(0), carry_v = T(0);   // e'1z, v'1z of the last voxel of the previous pass
    T z0_e = T(0), z0_v = T(0);         // e'2z, v'2z of voxel k = 0 (lane 0), for the row's wrap
    const int npass = ab.npass;
    for (int i = i0 - 1; i <= i1; ++i) {
        const bool ring_lo = (i == i0 - 1), ring_hi = (i == i1), inner = !ring_lo && !ring_hi;
        const int ii = (i < 0) ? i + n1 : (i >= n1 ? i - n1 : i);
        const int ip = (ii + 1 == n1) ? 0 : ii + 1, im = (ii == 0) ? n1 - 1 : ii - 1;
        const long long row = ((long long)ii * n2 + j) * n3;
        const long long rxp = ((long long)ip * n2 + j) * n3, rxm = ((long long)im * n2 + j) * n3;
        const long long ryp = ((long long)ii * n2 + jp) * n3, rym = ((long long)ii * n2 + jm) * n3;
        const long long rprev = ((long long)im * n2 + j) * n3;   // slab i - 1, finalised in this step
        const bool count = inner && interior_row;
        for (int pz = 0; pz < npass; ++pz) {
            const int k0 = pz * KZ + lane * VW;
            T* yb = yb2 + (size_t)(((i - i0 + 1) * npass + pz) & 1) * NW * 4 * KZ;
            T eo[6][VW], vo[6][VW];
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
                for (int u = 0; u < VW; ++u) eo[c][u] = vo[c][u] = T(0);
            if (interior_row || (active_w && inner)) {
                const int kp = (k0 + VW == n3) ? 0 : k0 + VW;
                const int km = (k0 == 0) ? n3 - 1 : k0 - 1;
                T ec[6][VW], vc[6][VW];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    V::ld(e + c * N + row + k0, ec[c]);
                    V::ld(v + c * N + row + k0, vc[c]);
                }
                T gm[VW], ph[VW];
                V::ld(gam + row + k0, gm);
                V::ld(phi + row + k0, ph);
                T e2x[VW], v2x[VW], e1x[VW], v1x[VW], e2y[VW], v2y[VW], e1y[VW], v1y[VW];
                T phxp[VW], phxm[VW], phyp[VW], phym[VW];
                V::ld(e + 3 * N + rxp + k0, e2x);
                V::ld(v + 3 * N + rxp + k0, v2x);
                V::ld(e + 0 * N + rxm + k0, e1x);
                V::ld(v + 0 * N + rxm + k0, v1x);
                V::ld(e + 4 * N + ryp + k0, e2y);
                V::ld(v + 4 * N + ryp + k0, v2y);
                V::ld(e + 1 * N + rym + k0, e1y);
                V::ld(v + 1 * N + rym + k0, v1y);
                V::ld(phi + rxp + k0, phxp);
                V::ld(phi + rxm + k0, phxm);
                V::ld(phi + ryp + k0, phyp);
                V::ld(phi + rym + k0, phym);
                const T e2z_after = __ldg(e + 5 * N + row + kp), v2z_after = __ldg(v + 5 * N + row + kp);
                const T e1z_before = __ldg(e + 2 * N + row + km), v1z_before = __ldg(v + 2 * N + row + km);
                const T ph_after = __ldg(phi + row + kp), ph_before = __ldg(phi + row + km);
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    T ecu[6], vcu[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        ecu[c] = ec[c][u];
                        vcu[c] = vc[c][u];
                    }
                    const bool last = (u + 1 == VW), first = (u == 0);
                    const T php[3] = {phxp[u], phyp[u], last ? ph_after : ph[(u + 1) % VW]};
                    const T phm[3] = {phxm[u], phym[u], first ? ph_before : ph[(u + VW - 1) % VW]};
                    const T e2p[3] = {e2x[u], e2y[u], last ? e2z_after : ec[5][(u + 1) % VW]};
                    const T v2p[3] = {v2x[u], v2y[u], last ? v2z_after : vc[5][(u + 1) % VW]};
                    const T e1m[3] = {e1x[u], e1y[u], first ? e1z_before : ec[2][(u + VW - 1) % VW]};
                    const T v1m[3] = {v1x[u], v1y[u], first ? v1z_before : vc[2][(u + VW - 1) % VW]};
                    T eou[6], vou[6], fl[3];
                    voxel_step<T, false>(K, ecu, vcu, gm[u], ph[u], php, phm, e2p, v2p, e1m, v1m, acc, eou, vou, fl,
                                         nullptr, count);
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        eo[c][u] = eou[c];
                        vo[c][u] = vou[c];
                    }
                }
                if (count) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        V::st(e_out + c * N + row + k0, eo[c]);
                        V::st(v_out + c * N + row + k0, vo[c]);
                    }
                }
                if (inner) {   // the y terms of the pending sums of interior slabs
                    T* yw = yb + (size_t)w * 4 * KZ;
#pragma unroll
                    for (int u = 0; u < VW; ++u) {
                        yw[0 * KZ + u * 32 + lane] = eo[1][u];
                        yw[1 * KZ + u * 32 + lane] = eo[4][u];
                        yw[2 * KZ + u * 32 + lane] = vo[1][u];
                        yw[3 * KZ + u * 32 + lane] = vo[4][u];
                    }
                }
            }
            __syncthreads();
            if (interior_row) {
                // z neighbours from the neighbouring lanes (a row of one pass wraps within the warp)
                const T e1z_l = __shfl_sync(0xffffffffu, eo[2][VW - 1], (lane + 31) & 31);
                const T v1z_l = __shfl_sync(0xffffffffu, vo[2][VW - 1], (lane + 31) & 31);
                const T e2z_r = __shfl_sync(0xffffffffu, eo[5][0], (lane + 1) & 31);
                const T v2z_r = __shfl_sync(0xffffffffu, vo[5][0], (lane + 1) & 31);
                T fa[VW], fb[VW];
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    const size_t slot = rbase + (size_t)pz * KZ + u * 32 + lane;
                    if (!ring_lo && i > i0) {   // a', b' of slab i - 1: its x+ terms are this slab's 2x
                        fa[u] = pe[slot] + h * eo[3][u];
                        fb[u] = pv[slot] + h * vo[3][u];
                    }
                    if (inner) {
                        T tm_e, tm_v, tp_e, tp_v;
                        if (u > 0) {
                            tm_e = eo[2][u - 1];
                            tm_v = vo[2][u - 1];
                        } else if (lane > 0 || npass == 1) {
                            tm_e = e1z_l;
                            tm_v = v1z_l;
                        } else {   // lane 0: the previous pass's last voxel (pass 0: fixed up at the row's end)
                            tm_e = pz > 0 ? carry_e : T(0);
                            tm_v = pz > 0 ? carry_v : T(0);
                        }
                        if (u + 1 < VW) {
                            tp_e = eo[5][u + 1];
                            tp_v = vo[5][u + 1];
                        } else if (lane < 31 || npass == 1) {
                            tp_e = e2z_r;
                            tp_v = v2z_r;
                        } else {   // lane 31: the next pass's first voxel (fixed up in the next pass)
                            tp_e = T(0);
                            tp_v = T(0);
                        }
                        const T* ym = yb + (size_t)(w - 1) * 4 * KZ;
                        const T* yp = yb + (size_t)(w + 1) * 4 * KZ;
                        const int ys = u * 32 + lane;
                        const T la = h * ((eo[0][u] + eo[1][u] + eo[2][u]) - (eo[3][u] + eo[4][u] + eo[5][u]));
                        const T lb = h * ((vo[0][u] + vo[1][u] + vo[2][u]) - (vo[3][u] + vo[4][u] + vo[5][u]));
                        pe[slot] = la + h * ((tp_e - tm_e) + (yp[1 * KZ + ys] - ym[0 * KZ + ys]) - ex[slot]);
                        pv[slot] = lb + h * ((tp_v - tm_v) + (yp[3 * KZ + ys] - ym[2 * KZ + ys]) - vx[slot]);
                    }
                    if (!ring_hi) {
                        ex[slot] = eo[0][u];
                        vx[slot] = vo[0][u];
                    }
                }
                if (!ring_lo && i > i0) {
                    V::st(a_out + rprev + k0, fa);
                    V::st(b_out + rprev + k0, fb);
                }
                if (inner && npass > 1) {
                    // z terms across passes of the row
                    if (lane == 0 && pz > 0) {   // the previous pass's last voxel gets this voxel's 2z
                        const size_t sl = rbase + (size_t)(pz - 1) * KZ + (VW - 1) * 32 + 31;
                        pe[sl] += h * eo[5][0];
                        pv[sl] += h * vo[5][0];
                    }
                    if (lane == 0 && pz == 0) {
                        z0_e = eo[5][0];
                        z0_v = vo[5][0];
                    }
                    if (pz == npass - 1) {
                        __syncwarp();
                        if (lane == 31) {   // voxel 0 gets the 1z of voxel n3 - 1
                            pe[rbase] -= h * eo[2][VW - 1];
                            pv[rbase] -= h * vo[2][VW - 1];
                        }
                        if (lane == 0) {   // voxel n3 - 1 gets the 2z of voxel 0
                            const size_t sl = rbase + (size_t)(npass - 1) * KZ + (VW - 1) * 32 + 31;
                            pe[sl] += h * z0_e;
                            pv[sl] += h * z0_v;
                        }
                    }
                }
                carry_e = __shfl_sync(0xffffffffu, eo[2][VW - 1], 31);
                carry_v = __shfl_sync(0xffffffffu, vo[2][VW - 1], 31);
                __syncwarp();   // the fix-ups above before this warp's next writes of its slots
            }
        }
    }
    const int nblocks = gridDim.x;
    double* part = p.partial + (size_t)s * nblocks * kNSum;
    if (block_partials<T, kNSum, NT>(acc, part, &S.counter, nblocks, blockIdx.x))
        update_finish<T, false, NT, true>(g, p, cfg, S, s, rho_d, part, nblocks);
}

// Warp-independent stored-divergence update (update variants 13 .. 15). Each warp owns one item: tj
// consecutive y rows of one z segment of KZ = 32 VW voxels, over an x segment of slabs. It
// walks the slabs and, within a slab, the rows (the row before and after the tile are
// recomputed), so the y terms of the new state's divergence wait one row (in registers) and the
// x terms one slab (in the warp's own shared-memory slots); no warp waits for another. A z
// segment shorter than the row recomputes the update of the voxel just before and just after it
// (lanes 0 and 31) for the z terms at its ends.
constexpr int kAbwWarps = 4;   // warps (items) per block

template <typename T, int VW>
__device__ __forceinline__ void abw_halo_voxel(const StepConsts<T>& K, const T* __restrict__ e,
                                               const T* __restrict__ v, const T* __restrict__ phi,
                                               const T* __restrict__ gam, long long N, long long row, long long rxp,
                                               long long rxm, long long ryp, long long rym, int kh, int n3,
                                               T (&eo)[6], T (&vo)[6]) {
    const int kp = (kh + 1 == n3) ? 0 : kh + 1, km = (kh == 0) ? n3 - 1 : kh - 1;
    T ec[6], vc[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        ec[c] = __ldg(e + c * N + row + kh);
        vc[c] = __ldg(v + c * N + row + kh);
    }
    const T php[3] = {__ldg(phi + rxp + kh), __ldg(phi + ryp + kh), __ldg(phi + row + kp)};
    const T phm[3] = {__ldg(phi + rxm + kh), __ldg(phi + rym + kh), __ldg(phi + row + km)};
    const T e2p[3] = {__ldg(e + 3 * N + rxp + kh), __ldg(e + 4 * N + ryp + kh), __ldg(e + 5 * N + row + kp)};
    const T v2p[3] = {__ldg(v + 3 * N + rxp + kh), __ldg(v + 4 * N + ryp + kh), __ldg(v + 5 * N + row + kp)};
    const T e1m[3] = {__ldg(e + 0 * N + rxm + kh), __ldg(e + 1 * N + rym + kh), __ldg(e + 2 * N + row + km)};
    const T v1m[3] = {__ldg(v + 0 * N + rxm + kh), __ldg(v + 1 * N + rym + kh), __ldg(v + 2 * N + row + km)};
    T acc[kNSum], fl[3];
    voxel_step<T, false>(K, ec, vc, __ldg(gam + row + kh), __ldg(phi + row + kh), php, phm, e2p, v2p, e1m, v1m,
                         acc, eo, vo, fl, nullptr, false);
}

template <typename T, int VW, int MINB>
__global__ void __launch_bounds__(kAbwWarps * 32, MINB) k_update_abw(Geom g, Ptrs<T> p, LoopConfig cfg, AbShape ab) {
    constexpr int NT = kAbwWarps * 32, KZ = 32 * VW;
    using V = VecN<T, VW>;
    const int s = blockIdx.y + p.s0;
    SolveScalars& S = p.sc[s];
    if (!S.active) return;
    const long long N = g.N;
    const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
    const double rho_d = S.rho;
    const StepConsts<T> K = step_consts<T>(S, cfg);
    const T h = K.h;
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ phi = p.phi + (size_t)s * N;
    const T* __restrict__ gam = gamma_of(p, s);
    T* __restrict__ a_out = p.ab + (size_t)s * 2 * N;
    T* __restrict__ b_out = a_out + N;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tj = ab.tj, npass = ab.npass;
    // item = (x segment r, y tile q, z segment zs), z segments fastest, then y tiles
    const long long item = (long long)blockIdx.x * kAbwWarps + w;
    const int zs = (int)(item % npass);
    const long long rest = item / npass;
    const int q = (int)(rest % ab.nq), r = (int)(rest / ab.nq);
    const bool have = r < ab.nr;   // warp-uniform
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // this warp's slots, [row][u][lane]: pending a and b of the current slab, the component 1x of
    // e' and v' of the previous slab
    T* pe = reinterpret_cast<T*>(smem_raw) + (size_t)w * 4 * tj * KZ;
    T* pv = pe + (size_t)tj * KZ;
    T* ex = pv + (size_t)tj * KZ;
    T* vx = ex + (size_t)tj * KZ;
    T acc[kNSum];
#pragma unroll
    for (int qq = 0; qq < kNSum; ++qq) acc[qq] = T(0);
    if (have) {
        const int j0 = q * tj, nint = min(tj, n2 - j0);
        const int i0 = r * ab.xs, i1 = min(i0 + ab.xs, n1);
        const int seg0 = zs * KZ, k0 = seg0 + lane * VW;
        const int kp = (k0 + VW == n3) ? 0 : k0 + VW, km = (k0 == 0) ? n3 - 1 : k0 - 1;
        const int khb = (seg0 == 0) ? n3 - 1 : seg0 - 1;            // halo voxel before the segment (lane 0)
        const int kha = (seg0 + KZ == n3) ? 0 : seg0 + KZ;          // halo voxel after it (lane 31)
        for (int i = i0 - 1; i <= i1; ++i) {
            const bool ring_lo = (i == i0 - 1), ring_hi = (i == i1), inner = !ring_lo && !ring_hi;
            const int ii = (i < 0) ? i + n1 : (i >= n1 ? i - n1 : i);
            const int ip = (ii + 1 == n1) ? 0 : ii + 1, im = (ii == 0) ? n1 - 1 : ii - 1;
            T y1e[VW], y1v[VW];   // e'1y, v'1y of the previous row
#pragma unroll
            for (int u = 0; u < VW; ++u) y1e[u] = y1v[u] = T(0);
            const int jr_lo = inner ? -1 : 0, jr_hi = inner ? nint : nint - 1;
            for (int jr = jr_lo; jr <= jr_hi; ++jr) {
                int j = j0 + jr;
                if (j < 0) j += n2;
                if (j >= n2) j -= n2;
                const int jp = (j + 1 == n2) ? 0 : j + 1, jm = (j == 0) ? n2 - 1 : j - 1;
                const bool interior_row = jr >= 0 && jr < nint;
                const bool count = inner && interior_row;
                const long long row = ((long long)ii * n2 + j) * n3;
                const long long rxp = ((long long)ip * n2 + j) * n3, rxm = ((long long)im * n2 + j) * n3;
                const long long ryp = ((long long)ii * n2 + jp) * n3, rym = ((long long)ii * n2 + jm) * n3;
                T eo[6][VW], vo[6][VW];
                {
                    T ec[6][VW], vc[6][VW];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        V::ld(e + c * N + row + k0, ec[c]);
                        V::ld(v + c * N + row + k0, vc[c]);
                    }
                    T gm[VW], ph[VW];
                    V::ld(gam + row + k0, gm);
                    V::ld(phi + row + k0, ph);
                    T e2x[VW], v2x[VW], e1x[VW], v1x[VW], e2y[VW], v2y[VW], e1y[VW], v1y[VW];
                    T phxp[VW], phxm[VW], phyp[VW], phym[VW];
                    V::ld(e + 3 * N + rxp + k0, e2x);
                    V::ld(v + 3 * N + rxp + k0, v2x);
                    V::ld(e + 0 * N + rxm + k0, e1x);
                    V::ld(v + 0 * N + rxm + k0, v1x);
                    V::ld(e + 4 * N + ryp + k0, e2y);
                    V::ld(v + 4 * N + ryp + k0, v2y);
                    V::ld(e + 1 * N + rym + k0, e1y);
                    V::ld(v + 1 * N + rym + k0, v1y);
                    V::ld(phi + rxp + k0, phxp);
                    V::ld(phi + rxm + k0, phxm);
                    V::ld(phi + ryp + k0, phyp);
                    V::ld(phi + rym + k0, phym);
                    const T e2z_after = __ldg(e + 5 * N + row + kp), v2z_after = __ldg(v + 5 * N + row + kp);
                    const T e1z_before = __ldg(e + 2 * N + row + km), v1z_before = __ldg(v + 2 * N + row + km);
                    const T ph_after = __ldg(phi + row + kp), ph_before = __ldg(phi + row + km);
#pragma unroll
                    for (int u = 0; u < VW; ++u) {
                        T ecu[6], vcu[6];
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                            ecu[c] = ec[c][u];
                            vcu[c] = vc[c][u];
                        }
                        const bool last = (u + 1 == VW), first = (u == 0);
                        const T php[3] = {phxp[u], phyp[u], last ? ph_after : ph[(u + 1) % VW]};
                        const T phm[3] = {phxm[u], phym[u], first ? ph_before : ph[(u + VW - 1) % VW]};
                        const T e2p[3] = {e2x[u], e2y[u], last ? e2z_after : ec[5][(u + 1) % VW]};
                        const T v2p[3] = {v2x[u], v2y[u], last ? v2z_after : vc[5][(u + 1) % VW]};
                        const T e1m[3] = {e1x[u], e1y[u], first ? e1z_before : ec[2][(u + VW - 1) % VW]};
                        const T v1m[3] = {v1x[u], v1y[u], first ? v1z_before : vc[2][(u + VW - 1) % VW]};
                        T eou[6], vou[6], fl[3];
                        voxel_step<T, false>(K, ecu, vcu, gm[u], ph[u], php, phm, e2p, v2p, e1m, v1m, acc, eou, vou,
                                             fl, nullptr, count);
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                            eo[c][u] = eou[c];
                            vo[c][u] = vou[c];
                        }
                    }
                }
                if (count) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        V::st(e_out + c * N + row + k0, eo[c]);
                        V::st(v_out + c * N + row + k0, vo[c]);
                    }
                }
                // z neighbours of the voxels at the ends of the lane group: the neighbouring lanes, or at
                // the ends of the segment the recomputed halo voxels (a whole row wraps within the warp)
                T tme = __shfl_sync(0xffffffffu, eo[2][VW - 1], (lane + 31) & 31);
                T tmv = __shfl_sync(0xffffffffu, vo[2][VW - 1], (lane + 31) & 31);
                T tpe = __shfl_sync(0xffffffffu, eo[5][0], (lane + 1) & 31);
                T tpv = __shfl_sync(0xffffffffu, vo[5][0], (lane + 1) & 31);
                if (npass > 1 && count && (lane == 0 || lane == 31)) {
                    T he[6], hv[6];
                    abw_halo_voxel<T, VW>(K, e, v, phi, gam, N, row, rxp, rxm, ryp, rym, lane == 0 ? khb : kha, n3,
                                          he, hv);
                    if (lane == 0) {
                        tme = he[2];
                        tmv = hv[2];
                    } else {
                        tpe = he[5];
                        tpv = hv[5];
                    }
                }
                if (interior_row) {
                    T fa[VW], fb[VW];
#pragma unroll
                    for (int u = 0; u < VW; ++u) {
                        const size_t slot = (size_t)jr * KZ + u * 32 + lane;
                        if (!ring_lo && i > i0) {   // a', b' of slab i - 1: its x+ terms are this slab's 2x
                            fa[u] = pe[slot] + h * eo[3][u];
                            fb[u] = pv[slot] + h * vo[3][u];
                        }
                        if (inner) {
                            const T tm_e = (u > 0) ? eo[2][u - 1] : tme, tm_v = (u > 0) ? vo[2][u - 1] : tmv;
                            const T tp_e = (u + 1 < VW) ? eo[5][u + 1] : tpe, tp_v = (u + 1 < VW) ? vo[5][u + 1] : tpv;
                            const T la = (eo[0][u] + eo[1][u] + eo[2][u]) - (eo[3][u] + eo[4][u] + eo[5][u]);
                            const T lb = (vo[0][u] + vo[1][u] + vo[2][u]) - (vo[3][u] + vo[4][u] + vo[5][u]);
                            // pending until the next row (+2y) and the next slab (+2x)
                            pe[slot] = h * (la + (tp_e - tm_e) - y1e[u] - ex[slot]);
                            pv[slot] = h * (lb + (tp_v - tm_v) - y1v[u] - vx[slot]);
                        }
                        if (!ring_hi) {
                            ex[slot] = eo[0][u];
                            vx[slot] = vo[0][u];
                        }
                    }
                    if (!ring_lo && i > i0) {
                        const long long rprev = ((long long)im * n2 + j) * n3;
                        V::st(a_out + rprev + k0, fa);
                        V::st(b_out + rprev + k0, fb);
                    }
                }
                if (inner && jr >= 1) {   // the previous (interior) row gets this row's 2y
#pragma unroll
                    for (int u = 0; u < VW; ++u) {
                        const size_t slot = (size_t)(jr - 1) * KZ + u * 32 + lane;
                        pe[slot] += h * eo[4][u];
                        pv[slot] += h * vo[4][u];
                    }
                }
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    y1e[u] = eo[1][u];
                    y1v[u] = vo[1][u];
                }
            }
        }
    }
    const int nblocks = gridDim.x;
    double* part = p.partial + (size_t)s * nblocks * kNSum;
    if (block_partials<T, kNSum, NT>(acc, part, &S.counter, nblocks, blockIdx.x))
        update_finish<T, false, NT, true>(g, p, cfg, S, s, rho_d, part, nblocks);
}

// The stored divergences a = div^- A* e, b = div^- A* v of the current state, for a
// state that the stored-divergence update did not write (a new solve, an imported
// state, a state advanced by another update pass). Skipped for solves whose stored
// divergences are current.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ab_init(Geom g, Ptrs<T> p) {
    const int s = blockIdx.y + p.s0;
    const SolveScalars& S = p.sc[s];
    if (S.ab_iter == S.iters) return;
    const long long N = g.N;
    const T h = T(0.70710678118654752440084436210485);
    const long long cur = (long long)(S.iters & 1) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ e = p.e + cur;
    const T* __restrict__ v = p.v + cur;
    T* a_out = p.ab + (size_t)s * 2 * N;
    T* b_out = a_out + N;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < N; lin += stride) {
        const unsigned row = fdiv((unsigned)lin, g.div_n3);
        const int k = (int)(lin - (long long)row * g.n3);
        const RowNb rn = row_neighbours(g, row);
        const int kp = (k + 1 == g.n3) ? 0 : k + 1, km = (k == 0) ? g.n3 - 1 : k - 1;
        auto dv = [&](const T* f) {
            const T sx = f[0 * N + lin] - f[0 * N + rn.im + k] + f[3 * N + rn.ip + k] - f[3 * N + lin];
            const T sy = f[1 * N + lin] - f[1 * N + rn.jm + k] + f[4 * N + rn.jp + k] - f[4 * N + lin];
            const T sz = f[2 * N + lin] - f[2 * N + rn.row + km] + f[5 * N + rn.row + kp] - f[5 * N + lin];
            return h * (sx + sy + sz);
        };
        a_out[lin] = dv(e);
        b_out[lin] = dv(v);
    }
}

// ---------------------------------------------------------------------------
// TMA-staged update pass. A tile is J consecutive z rows (i, j0 .. j0+J-1) of one
// solve, TV = J * N3 voxels. One elected thread copies everything the tile's
// stencil reads into shared memory with bulk asynchronous copies (cp.async.bulk,
// completion counted in bytes on an mbarrier): the 12 state fields, gamma and phi
// of the tile, the halo rows j0-1 / j0+J of the fields that reach across y, and
// the rows of the planes i-1 / i+1 that reach across x. Two stages alternate so
// that the copies of the next tiles overlap the arithmetic of the current one.
// Every wait is bounded: a wait that gives up records CCMF_ERR_TIMEOUT for the
// solve, waits (bounded) for its copies in flight and leaves the loop.
// ---------------------------------------------------------------------------
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
    return (unsigned)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned limit = kSpinLimit) {
    for (unsigned spin = 0; spin < limit; ++spin)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Elements of one stage: own[14][TV] (e0..e5, v0..v5, gamma, phi), yh[6][N3]
// (e1, v1 at row j0-1; e4, v4 at row j0+J; phi at j0-1, j0+J), xn[6][TV]
// (e0, v0 at plane i-1; e3, v3 at plane i+1; phi at i-1, i+1).
__host__ __device__ inline long long tma_stage_elems(int TV, int n3) { return 20LL * TV + 6LL * n3; }

// Vector of VW = 8 / sizeof(T) values (float2 for FP32, one double for FP64)
// read from shared memory in one access.
template <typename T> struct Vec8;
template <> struct Vec8<float> {
    static constexpr int W = 2;
    __device__ __forceinline__ static void ld(const float* p, float (&o)[2]) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        o[0] = t.x;
        o[1] = t.y;
    }
    __device__ __forceinline__ static void st(float* p, const float (&o)[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    }
};
template <> struct Vec8<double> {
    static constexpr int W = 1;
    __device__ __forceinline__ static void ld(const double* p, double (&o)[1]) { o[0] = *p; }
    __device__ __forceinline__ static void st(double* p, const double (&o)[1]) { *p = o[0]; }
};

template <typename T, int RULE>
__global__ void __launch_bounds__(kThreads, 2) k_update_tma(Geom g, Ptrs<T> p, LoopConfig cfg, int J) {
    using V = Vec8<T>;
    constexpr int W = V::W;
    const int s = blockIdx.y + p.s0;
    SolveScalars& S = p.sc[s];
    if (!S.active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n3 = g.n3;
    const int TV = J * n3;
    const long long selems = tma_stage_elems(TV, n3);
    T* stage0 = reinterpret_cast<T*>(smem_raw);
    T* stage1 = stage0 + selems;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(stage0 + 2 * selems);
    const unsigned stage_bytes = (unsigned)(selems * sizeof(T));
    const unsigned tv_bytes = (unsigned)(TV * sizeof(T)), row_bytes = (unsigned)(n3 * sizeof(T));

    const long long N = g.N;
    const double rho_d = S.rho;
    const StepConsts<T> K = step_consts<T>(S, cfg);
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ phi = p.phi + (size_t)s * N;
    const T* __restrict__ gam = gamma_of(p, s);
    const int tiles_j = g.n2 / J;
    const int ntiles = g.n1 * tiles_j;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // producer: all copies of one tile into one stage (thread 0 only)
    auto issue = [&](int tile, int st) {
        T* b = st ? stage1 : stage0;
        const int i = tile / tiles_j;
        const int j0 = (tile - i * tiles_j) * J;
        const int ip = (i + 1 == g.n1) ? 0 : i + 1, im = (i == 0) ? g.n1 - 1 : i - 1;
        const int jp = (j0 + J == g.n2) ? 0 : j0 + J, jm = (j0 == 0) ? g.n2 - 1 : j0 - 1;
        const long long base = ((long long)i * g.n2 + j0) * n3;
        const long long bip = ((long long)ip * g.n2 + j0) * n3, bim = ((long long)im * g.n2 + j0) * n3;
        const long long rjp = ((long long)i * g.n2 + jp) * n3, rjm = ((long long)i * g.n2 + jm) * n3;
        unsigned long long* bar = &bars[st];
        mbar_expect_tx(bar, stage_bytes);
        T* own = b;
        T* yh = b + 14LL * TV;
        T* xn = yh + 6LL * n3;
        for (int c = 0; c < 6; ++c) {
            bulk_g2s(own + (long long)c * TV, e + c * N + base, tv_bytes, bar);
            bulk_g2s(own + (long long)(6 + c) * TV, v + c * N + base, tv_bytes, bar);
        }
        bulk_g2s(own + 12LL * TV, gam + base, tv_bytes, bar);
        bulk_g2s(own + 13LL * TV, phi + base, tv_bytes, bar);
        bulk_g2s(yh + 0LL * n3, e + 1 * N + rjm, row_bytes, bar);
        bulk_g2s(yh + 1LL * n3, v + 1 * N + rjm, row_bytes, bar);
        bulk_g2s(yh + 2LL * n3, e + 4 * N + rjp, row_bytes, bar);
        bulk_g2s(yh + 3LL * n3, v + 4 * N + rjp, row_bytes, bar);
        bulk_g2s(yh + 4LL * n3, phi + rjm, row_bytes, bar);
        bulk_g2s(yh + 5LL * n3, phi + rjp, row_bytes, bar);
        bulk_g2s(xn + 0LL * TV, e + 0 * N + bim, tv_bytes, bar);
        bulk_g2s(xn + 1LL * TV, v + 0 * N + bim, tv_bytes, bar);
        bulk_g2s(xn + 2LL * TV, e + 3 * N + bip, tv_bytes, bar);
        bulk_g2s(xn + 3LL * TV, v + 3 * N + bip, tv_bytes, bar);
        bulk_g2s(xn + 4LL * TV, phi + bim, tv_bytes, bar);
        bulk_g2s(xn + 5LL * TV, phi + bip, tv_bytes, bar);
    };

    const int t0 = blockIdx.x;
    const int tstep = gridDim.x;
    if (threadIdx.x == 0) {
        if (t0 < ntiles) issue(t0, 0);
        if (t0 + tstep < ntiles) issue(t0 + tstep, 1);
    }
    T acc[kNSum];
#pragma unroll
    for (int q = 0; q < kNSum; ++q) acc[q] = T(0);
    unsigned phase0 = 0, phase1 = 0;
    int it = 0;
    bool failed = false;
    const int ngroups = TV / W;
    for (int tile = t0; tile < ntiles; tile += tstep, ++it) {
        const int st = it & 1;
        const unsigned ph = st ? phase1 : phase0;
        const bool ok = mbar_wait_bounded(&bars[st], ph, cfg.spin_limit ? cfg.spin_limit - 1 : kSpinLimit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (st) phase1 ^= 1u; else phase0 ^= 1u;
        const T* b = st ? stage1 : stage0;
        const T* own = b;
        const T* yh = b + 14LL * TV;
        const T* xn = yh + 6LL * n3;
        const int i = tile / tiles_j;
        const int j0 = (tile - i * tiles_j) * J;
        const long long base = ((long long)i * g.n2 + j0) * n3;
        for (int gi = threadIdx.x; gi < ngroups; gi += kThreads) {
            const int lv0 = gi * W;
            const int r = (int)fdiv((unsigned)lv0, g.div_n3);
            const int k0 = lv0 - r * n3;
            const int kp = (k0 + W == n3) ? 0 : k0 + W, km = (k0 == 0) ? n3 - 1 : k0 - 1;
            const bool top = (r + 1 == J), bot = (r == 0);
            // W-wide reads of every field this group needs
            T ec[6][W], vc[6][W], gm[W], ph[W];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                V::ld(own + c * TV + lv0, ec[c]);
                V::ld(own + (6 + c) * TV + lv0, vc[c]);
            }
            V::ld(own + 12 * TV + lv0, gm);
            V::ld(own + 13 * TV + lv0, ph);
            T e2x[W], v2x[W], e1x[W], v1x[W], phxp[W], phxm[W];
            V::ld(xn + 2 * TV + lv0, e2x);
            V::ld(xn + 3 * TV + lv0, v2x);
            V::ld(xn + 0 * TV + lv0, e1x);
            V::ld(xn + 1 * TV + lv0, v1x);
            V::ld(xn + 5 * TV + lv0, phxp);
            V::ld(xn + 4 * TV + lv0, phxm);
            T e2y[W], v2y[W], e1y[W], v1y[W], phyp[W], phym[W];
            V::ld(top ? yh + 2 * n3 + k0 : own + 4 * TV + lv0 + n3, e2y);
            V::ld(top ? yh + 3 * n3 + k0 : own + 10 * TV + lv0 + n3, v2y);
            V::ld(bot ? yh + 0 * n3 + k0 : own + 1 * TV + lv0 - n3, e1y);
            V::ld(bot ? yh + 1 * n3 + k0 : own + 7 * TV + lv0 - n3, v1y);
            V::ld(top ? yh + 5 * n3 + k0 : own + 13 * TV + lv0 + n3, phyp);
            V::ld(bot ? yh + 4 * n3 + k0 : own + 13 * TV + lv0 - n3, phym);
            const int rz = r * n3;
            const T e2z_after = own[5 * TV + rz + kp], v2z_after = own[11 * TV + rz + kp];
            const T e1z_before = own[2 * TV + rz + km], v1z_before = own[8 * TV + rz + km];
            const T ph_after = own[13 * TV + rz + kp], ph_before = own[13 * TV + rz + km];
            T eo[6][W], vo[6][W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                T ecu[6], vcu[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    ecu[c] = ec[c][u];
                    vcu[c] = vc[c][u];
                }
                const bool last = (u + 1 == W), first = (u == 0);
                const T php[3] = {phxp[u], phyp[u], last ? ph_after : ph[(u + 1) % W]};
                const T phm[3] = {phxm[u], phym[u], first ? ph_before : ph[(u + W - 1) % W]};
                const T e2p[3] = {e2x[u], e2y[u], last ? e2z_after : ec[5][(u + 1) % W]};
                const T v2p[3] = {v2x[u], v2y[u], last ? v2z_after : vc[5][(u + 1) % W]};
                const T e1m[3] = {e1x[u], e1y[u], first ? e1z_before : ec[2][(u + W - 1) % W]};
                const T v1m[3] = {v1x[u], v1y[u], first ? v1z_before : vc[2][(u + W - 1) % W]};
                T eou[6], vou[6], fl[3];
                voxel_step<T, false, RULE>(K, ecu, vcu, gm[u], ph[u], php, phm, e2p, v2p, e1m, v1m, acc, eou, vou,
                                           fl);
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    eo[c][u] = eou[c];
                    vo[c][u] = vou[c];
                }
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                V::st(e_out + c * N + base + lv0, eo[c]);
                V::st(v_out + c * N + base + lv0, vo[c]);
            }
        }
        __syncthreads();   // every thread is done with this stage
        if (threadIdx.x == 0 && tile + 2 * tstep < ntiles) {
            fence_proxy_async_smem();
            issue(tile + 2 * tstep, st);
        }
    }
    if (failed) {
        // the copies still in flight land in this block's shared memory: wait for them (bounded)
        if (threadIdx.x == 0) {
            for (int extra = 0; extra < 2; ++extra) {
                const int st = (it + extra) & 1;
                const int tile = t0 + (it + extra) * tstep;
                if (tile < ntiles) (void)mbar_wait_bounded(&bars[st], st ? phase1 : phase0);
            }
            atomicExch(&S.status, 6);   // CCMF_ERR_TIMEOUT
        }
        __syncthreads();
    }
    update_epilogue<T, false>(g, p, cfg, S, s, rho_d, acc);
}

// Pipelined variant: NT threads, each owning one W-wide group of every tile
// (TV = NT * W voxels), so that all per-thread index arithmetic is fixed for the
// whole kernel; STAGES tiles are in flight. A tile is either J = TV / N3 whole z
// rows (N3 <= TV, J dividing N2) or a segment of KT = TV voxels of one row
// (N3 > TV, TV dividing N3); segments add the 16-byte z-halo chunks holding the
// voxels just before and after them. Same copies, waits and arithmetic as
// k_update_tma.
__host__ __device__ inline long long pipe_stage_elems(int TV, int KT, bool seg, int cw) {
    return 20LL * TV + 6LL * KT + (seg ? 6LL * cw : 0LL);
}

template <typename T, int RULE, int STAGES, int NT>
__global__ void __launch_bounds__(NT) k_update_pipe(Geom g, Ptrs<T> p, LoopConfig cfg) {
    using V = Vec8<T>;
    constexpr int W = V::W;
    constexpr int TV = NT * W;
    constexpr int CW = 16 / (int)sizeof(T);   // elements of a 16-byte z-halo chunk
    const int s = blockIdx.y + p.s0;
    SolveScalars& S = p.sc[s];
    if (!S.active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n3 = g.n3;
    const bool seg = n3 > TV;
    const int KT = seg ? TV : n3;            // z extent of a tile
    const int J = TV / KT;                   // rows of a tile
    const int nseg = n3 / KT;                // tiles per row
    const long long selems = pipe_stage_elems(TV, KT, seg, CW);
    T* stages = reinterpret_cast<T*>(smem_raw);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(stages + STAGES * selems);
    const unsigned stage_bytes = (unsigned)(selems * sizeof(T));
    constexpr unsigned tv_bytes = (unsigned)(TV * sizeof(T));
    const unsigned kt_bytes = (unsigned)(KT * sizeof(T));
    constexpr unsigned cw_bytes = 16;

    const long long N = g.N;
    const double rho_d = S.rho;
    const StepConsts<T> K = step_consts<T>(S, cfg);
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ phi = p.phi + (size_t)s * N;
    const T* __restrict__ gam = gamma_of(p, s);
    const int tiles_j = g.n2 / J;
    const int ntiles = g.n1 * tiles_j * nseg;

    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < STAGES; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // tile -> (i, j0, k0)
    auto tile_origin = [&](int tile, int& i, int& j0, int& k0) {
        const int row_tile = tile / nseg;
        k0 = (tile - row_tile * nseg) * KT;
        i = row_tile / tiles_j;
        j0 = (row_tile - i * tiles_j) * J;
    };
    auto issue = [&](int tile, int st) {
        T* b = stages + st * selems;
        int i, j0, k0;
        tile_origin(tile, i, j0, k0);
        const int ip = (i + 1 == g.n1) ? 0 : i + 1, im = (i == 0) ? g.n1 - 1 : i - 1;
        const int jp = (j0 + J == g.n2) ? 0 : j0 + J, jm = (j0 == 0) ? g.n2 - 1 : j0 - 1;
        const long long base = ((long long)i * g.n2 + j0) * n3 + k0;
        const long long bip = ((long long)ip * g.n2 + j0) * n3 + k0, bim = ((long long)im * g.n2 + j0) * n3 + k0;
        const long long rjp = ((long long)i * g.n2 + jp) * n3 + k0, rjm = ((long long)i * g.n2 + jm) * n3 + k0;
        unsigned long long* bar = &bars[st];
        mbar_expect_tx(bar, stage_bytes);
        T* own = b;
        T* yh = b + 14 * TV;
        T* xn = yh + 6LL * KT;
        T* zh = xn + 6 * TV;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            bulk_g2s(own + c * TV, e + c * N + base, tv_bytes, bar);
            bulk_g2s(own + (6 + c) * TV, v + c * N + base, tv_bytes, bar);
        }
        bulk_g2s(own + 12 * TV, gam + base, tv_bytes, bar);
        bulk_g2s(own + 13 * TV, phi + base, tv_bytes, bar);
        bulk_g2s(yh + 0LL * KT, e + 1 * N + rjm, kt_bytes, bar);
        bulk_g2s(yh + 1LL * KT, v + 1 * N + rjm, kt_bytes, bar);
        bulk_g2s(yh + 2LL * KT, e + 4 * N + rjp, kt_bytes, bar);
        bulk_g2s(yh + 3LL * KT, v + 4 * N + rjp, kt_bytes, bar);
        bulk_g2s(yh + 4LL * KT, phi + rjm, kt_bytes, bar);
        bulk_g2s(yh + 5LL * KT, phi + rjp, kt_bytes, bar);
        bulk_g2s(xn + 0 * TV, e + 0 * N + bim, tv_bytes, bar);
        bulk_g2s(xn + 1 * TV, v + 0 * N + bim, tv_bytes, bar);
        bulk_g2s(xn + 2 * TV, e + 3 * N + bip, tv_bytes, bar);
        bulk_g2s(xn + 3 * TV, v + 3 * N + bip, tv_bytes, bar);
        bulk_g2s(xn + 4 * TV, phi + bim, tv_bytes, bar);
        bulk_g2s(xn + 5 * TV, phi + bip, tv_bytes, bar);
        if (seg) {
            // 16-byte chunks ending at k0 - 1 and starting at k0 + KT (periodic in z)
            const long long row = ((long long)i * g.n2 + j0) * n3;
            const long long cb = row + ((k0 == 0) ? n3 - CW : k0 - CW);
            const long long ca = row + ((k0 + KT == n3) ? 0 : k0 + KT);
            bulk_g2s(zh + 0 * CW, e + 2 * N + cb, cw_bytes, bar);
            bulk_g2s(zh + 1 * CW, v + 2 * N + cb, cw_bytes, bar);
            bulk_g2s(zh + 2 * CW, phi + cb, cw_bytes, bar);
            bulk_g2s(zh + 3 * CW, e + 5 * N + ca, cw_bytes, bar);
            bulk_g2s(zh + 4 * CW, v + 5 * N + ca, cw_bytes, bar);
            bulk_g2s(zh + 5 * CW, phi + ca, cw_bytes, bar);
        }
    };

    const int t0 = blockIdx.x;
    const int tstep = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < STAGES; ++q)
            if (t0 + q * tstep < ntiles) issue(t0 + q * tstep, q);
    }
    // this thread's group: fixed stage offsets for the whole kernel
    const int lv0 = threadIdx.x * W;
    const int r = lv0 / KT;
    const int kk = lv0 - r * KT;
    const int rz = r * KT;
    const bool top = (r + 1 == J), bot = (r == 0);
    const int o_e2y = top ? 14 * TV + 2 * KT + kk : 4 * TV + lv0 + KT;
    const int o_v2y = top ? 14 * TV + 3 * KT + kk : 10 * TV + lv0 + KT;
    const int o_e1y = bot ? 14 * TV + 0 * KT + kk : 1 * TV + lv0 - KT;
    const int o_v1y = bot ? 14 * TV + 1 * KT + kk : 7 * TV + lv0 - KT;
    const int o_pyp = top ? 14 * TV + 5 * KT + kk : 13 * TV + lv0 + KT;
    const int o_pym = bot ? 14 * TV + 4 * KT + kk : 13 * TV + lv0 - KT;
    const int xo = 14 * TV + 6 * KT + lv0;   // xn[0] at this group
    const int zo = 20 * TV + 6 * KT;         // zh[0]
    // z neighbours just outside the group: inside the tile, wrapped within a whole
    // row, or from the z-halo chunks of a segment
    const bool after_in = kk + W < KT, before_in = kk > 0;
    const int o_after = after_in ? rz + kk + W : (seg ? -1 : rz);
    const int o_before = before_in ? rz + kk - 1 : (seg ? -1 : rz + KT - 1);

    T acc[kNSum];
#pragma unroll
    for (int q = 0; q < kNSum; ++q) acc[q] = T(0);
    int it = 0;
    bool failed = false;
    for (int tile = t0; tile < ntiles; tile += tstep, ++it) {
        const int st = it % STAGES;
        const unsigned ph = (unsigned)(it / STAGES) & 1u;
        const bool ok = mbar_wait_bounded(&bars[st], ph, cfg.spin_limit ? cfg.spin_limit - 1 : kSpinLimit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const T* b = stages + st * selems;
        T ec[6][W], vc[6][W], gm[W], ph_[W];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            V::ld(b + c * TV + lv0, ec[c]);
            V::ld(b + (6 + c) * TV + lv0, vc[c]);
        }
        V::ld(b + 12 * TV + lv0, gm);
        V::ld(b + 13 * TV + lv0, ph_);
        T e2x[W], v2x[W], e1x[W], v1x[W], phxp[W], phxm[W];
        V::ld(b + xo + 2 * TV, e2x);
        V::ld(b + xo + 3 * TV, v2x);
        V::ld(b + xo + 0 * TV, e1x);
        V::ld(b + xo + 1 * TV, v1x);
        V::ld(b + xo + 5 * TV, phxp);
        V::ld(b + xo + 4 * TV, phxm);
        T e2y[W], v2y[W], e1y[W], v1y[W], phyp[W], phym[W];
        V::ld(b + o_e2y, e2y);
        V::ld(b + o_v2y, v2y);
        V::ld(b + o_e1y, e1y);
        V::ld(b + o_v1y, v1y);
        V::ld(b + o_pyp, phyp);
        V::ld(b + o_pym, phym);
        T e2z_after, v2z_after, ph_after, e1z_before, v1z_before, ph_before;
        if (o_after >= 0) {
            e2z_after = b[5 * TV + o_after];
            v2z_after = b[11 * TV + o_after];
            ph_after = b[13 * TV + o_after];
        } else {
            e2z_after = b[zo + 3 * CW];
            v2z_after = b[zo + 4 * CW];
            ph_after = b[zo + 5 * CW];
        }
        if (o_before >= 0) {
            e1z_before = b[2 * TV + o_before];
            v1z_before = b[8 * TV + o_before];
            ph_before = b[13 * TV + o_before];
        } else {
            e1z_before = b[zo + 0 * CW + CW - 1];
            v1z_before = b[zo + 1 * CW + CW - 1];
            ph_before = b[zo + 2 * CW + CW - 1];
        }
        __syncthreads();   // the stage has been read into registers: refill it
        if (threadIdx.x == 0 && tile + STAGES * tstep < ntiles) {
            fence_proxy_async_smem();
            issue(tile + STAGES * tstep, st);
        }
        int ti, tj0, tk0;
        tile_origin(tile, ti, tj0, tk0);
        const long long gbase = ((long long)ti * g.n2 + tj0) * n3 + tk0 + (long long)r * n3 + kk;
        T eo[6][W], vo[6][W];
#pragma unroll
        for (int u = 0; u < W; ++u) {
            T ecu[6], vcu[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                ecu[c] = ec[c][u];
                vcu[c] = vc[c][u];
            }
            const bool last = (u + 1 == W), first = (u == 0);
            const T php[3] = {phxp[u], phyp[u], last ? ph_after : ph_[(u + 1) % W]};
            const T phm[3] = {phxm[u], phym[u], first ? ph_before : ph_[(u + W - 1) % W]};
            const T e2p[3] = {e2x[u], e2y[u], last ? e2z_after : ec[5][(u + 1) % W]};
            const T v2p[3] = {v2x[u], v2y[u], last ? v2z_after : vc[5][(u + 1) % W]};
            const T e1m[3] = {e1x[u], e1y[u], first ? e1z_before : ec[2][(u + W - 1) % W]};
            const T v1m[3] = {v1x[u], v1y[u], first ? v1z_before : vc[2][(u + W - 1) % W]};
            T eou[6], vou[6], fl[3];
            voxel_step<T, false, RULE>(K, ecu, vcu, gm[u], ph_[u], php, phm, e2p, v2p, e1m, v1m, acc, eou, vou, fl);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                eo[c][u] = eou[c];
                vo[c][u] = vou[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            V::st(e_out + c * N + gbase, eo[c]);
            V::st(v_out + c * N + gbase, vo[c]);
        }
    }
    if (failed) {
        if (threadIdx.x == 0) {
            for (int extra = 0; extra < STAGES; ++extra) {
                const int n = it + extra;
                if (t0 + n * tstep < ntiles) (void)mbar_wait_bounded(&bars[n % STAGES], (unsigned)(n / STAGES) & 1u);
            }
            atomicExch(&S.status, 6);   // CCMF_ERR_TIMEOUT
        }
        __syncthreads();
    }
    update_epilogue<T, false, NT>(g, p, cfg, S, s, rho_d, acc);
}

// ---------------------------------------------------------------------------
// Reverse mode of one update with rho fixed (the derivation is in the oracle's
// gradient module and the design notes). Per voxel, with u = vbar' - ebar'/rho:
//   zbar = ebar'/rho + J_C(z) u,  gbar += [|z| > gamma] (z/|z|) . u,
//   y = a rho zbar  (then My = M y by the forward passes with xi_bar = 0),
//   ebar = My - b rho zbar,  vbar = zbar - My / rho.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_adj_pre(Geom g, const T* __restrict__ z, const T* __restrict__ gamma,
                                                      long long gstride, const T* __restrict__ ebar,
                                                      const T* __restrict__ vbar, const double* __restrict__ rho_k,
                                                      int sched_len, int k, double a, T* __restrict__ zbar,
                                                      T* __restrict__ y, T* __restrict__ gbar,
                                                      const unsigned* __restrict__ clip_bits) {
    const int s = blockIdx.y;
    const long long N = g.N;
    const T rho = (T)rho_k[(size_t)s * sched_len + k];
    const T irho = T(1) / rho;
    const T ar = (T)(a * (double)rho);
    const T* zs = z + (size_t)s * 6 * N;
    const T* es = ebar + (size_t)s * 6 * N;
    const T* vs = vbar + (size_t)s * 6 * N;
    const T* gs = gamma + (size_t)s * gstride;
    T* zb = zbar + (size_t)s * 6 * N;
    T* ys = y + (size_t)s * 6 * N;
    T* gb = gbar + (size_t)s * N;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < N; lin += stride) {
        T zc[6], u[6];
        T nz2 = T(0), zu = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            zc[c] = zs[c * N + lin];
            u[c] = vs[c * N + lin] - es[c * N + lin] * irho;
            nz2 += zc[c] * zc[c];
        }
        const T gm = gs[lin];
        const T nz = Real<T>::sqrt_(nz2);
        // the branch of P_C: taken here, or recorded by a forward pass in higher precision
        // (one bit per voxel, [solve][ceil(N / 32)] words)
        const bool clip = clip_bits ? ((clip_bits[(size_t)s * ((N + 31) / 32) + (lin >> 5)] >> (lin & 31)) & 1u) != 0
                                    : nz > gm;
        if (clip) {
#pragma unroll
            for (int c = 0; c < 6; ++c) zu += zc[c] * u[c];
            zu /= nz;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            T ju = u[c];
            if (clip) ju = (gm / nz) * (u[c] - zc[c] / nz * zu);
            const T zbc = es[c * N + lin] * irho + ju;
            zb[c * N + lin] = zbc;
            ys[c * N + lin] = ar * zbc;
        }
        if (clip) gb[lin] += zu;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_adj_post(Geom g, const T* __restrict__ zbar, const T* __restrict__ my,
                                                       const double* __restrict__ rho_k, int sched_len, int k,
                                                       double b, T* __restrict__ ebar, T* __restrict__ vbar) {
    const int s = blockIdx.y;
    const long long N6 = 6 * g.N;
    const T rho = (T)rho_k[(size_t)s * sched_len + k];
    const T irho = T(1) / rho;
    const T br = (T)(b * (double)rho);
    const T* zb = zbar + (size_t)s * N6;
    const T* m = my + (size_t)s * N6;
    T* eb = ebar + (size_t)s * N6;
    T* vb = vbar + (size_t)s * N6;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long q = (long long)blockIdx.x * kThreads + threadIdx.x; q < N6; q += stride) {
        const T zq = zb[q], mq = m[q];
        eb[q] = mq - br * zq;
        vb[q] = zq - mq * irho;
    }
}

// seed of the reverse pass: vbar = A xi_bar / N (gradient of <xi_bar, A* v>), ebar = 0
template <typename T>
__global__ void __launch_bounds__(kThreads) k_adj_seed(Geom g, const SolveScalars* __restrict__ sc, T* __restrict__ ebar,
                                                       T* __restrict__ vbar) {
    const int s = blockIdx.y;
    const long long N = g.N;
    const double h = 0.70710678118654752440084436210485 / (double)N;
    const T a0 = (T)(sc[s].xi[0] * h), a1 = (T)(sc[s].xi[1] * h), a2 = (T)(sc[s].xi[2] * h);
    T* eb = ebar + (size_t)s * 6 * N;
    T* vb = vbar + (size_t)s * 6 * N;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < N; lin += stride) {
        const T av[3] = {a0, a1, a2};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            eb[c * N + lin] = T(0);
            vb[c * N + lin] = av[c % 3];
        }
    }
}

}  // namespace ccmf
