// CUDA kernels of one damped-ADMM iteration (Eq. 30 of the paper) on the CCMF
// discretisation, templated on the field type T (float: FP32-mixed, double: FP64).
//
// One iteration from (e^k, v^k, rho^k) is five passes:
//   1. k_div_rfft_z     w = e - v/rho, d = div^- A* w (Sec. 2.2, Eq. 17) fused
//                       with the real-to-complex FFT along z (two real lines per
//                       complex transform);
//   2. k_fft_strided<0> forward FFT along y;
//   3. k_fft_strided<1> forward FFT along x, Poisson solve
//                       phi^ = d^ / (-sum_a 4 sin^2(pi k_a / N_a)), phi^(0) = 0
//                       (the (div^- grad^+)^+ of Eq. 28), inverse FFT along x;
//   4. k_fft_strided<2> inverse FFT along y;
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

#include "ccmf_types.cuh"

namespace ccmf {

template <typename T> struct Real;
template <> struct Real<float> {
    __device__ __forceinline__ static float sqrt_(float x) { return sqrtf(x); }
};
template <> struct Real<double> {
    __device__ __forceinline__ static double sqrt_(double x) { return sqrt(x); }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// Block reduction of kNSum per-thread values (T) into one double each, written
// to partial[b * kNSum + q]; returns true in every thread of the block that
// finishes last for this solve (its partials are then visible to it).
template <typename T, int NQ>
__device__ bool block_partials(T (&acc)[NQ], double* __restrict__ partial, unsigned int* counter,
                               int nblocks, int b) {
    __shared__ double red[kThreads / 32][NQ];
    __shared__ int last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        T s = warp_sum(acc[q]);
        if (lane == 0) red[wid][q] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
        partial[(size_t)b * NQ + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(counter, 1u);
        last = (t == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    return last != 0;
}

// Deterministic double reduction of nblocks x NQ partials by one block.
template <int NQ>
__device__ void reduce_partials(const double* __restrict__ partial, int nblocks, double (&out)[NQ]) {
    __shared__ double red[kThreads / 32][NQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kThreads) s += __ldcg(partial + (size_t)b * NQ + q);
        s = warp_sum(s);
        if (lane == 0) red[wid][q] = s;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][q];
        out[q] = s;
    }
}

// ---------------------------------------------------------------------------
// Initialisation: statistics of gamma, rho^0 (reading R2 of the design notes)
// and the initial state e^0 = A xi_bar, v^0 = 0.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_init_stats(Geom g, Ptrs<T> p, LoopConfig cfg) {
    const int s = blockIdx.y;
    const T* gam = p.gamma + (size_t)s * p.gstride;
    double acc_min = INFINITY, acc_max = -INFINITY, acc_sum = 0.0, acc_bad = 0.0;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < g.N; lin += stride) {
        double x = (double)gam[lin];
        if (!(x >= 0.0) || !isfinite(x)) {
            acc_bad += 1.0;
        } else {
            acc_min = fmin(acc_min, x);
            acc_max = fmax(acc_max, x);
            acc_sum += x;
        }
    }
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
    if (threadIdx.x == 0) {
        double gmin = INFINITY, gmax = -INFINITY, gsum = 0.0, bad = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            gmin = fmin(gmin, __ldcg(part + b * 4 + 0));
            gmax = fmax(gmax, __ldcg(part + b * 4 + 1));
            gsum += __ldcg(part + b * 4 + 2);
            bad += __ldcg(part + b * 4 + 3);
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
            S.rho = rho0;
            S.iters = 0;
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
    const int s = blockIdx.y;
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
// Pass 1: divergence of A*(e - v/rho) fused with the real-to-complex z FFT.
// Line l = i * n2 + j of a solve; block b packs line pairs (2q, 2q+1) for
// q in [b P, b P + P) as real and imaginary parts of one complex line.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T wcomp(const T* __restrict__ e, const T* __restrict__ v, long long off, T irho) {
    return e[off] - v[off] * irho;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_div_rfft_z(Geom g, Ptrs<T> p, AxisPlan az,
                                                         const cx<T>* __restrict__ tw, int P) {
    using C = cx<T>;
    const int s = blockIdx.y;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twl = reinterpret_cast<C*>(smem_raw);
    C* A = twl + g.n3;
    C* B = A + (size_t)g.n3 * (P + 1);
    const int stride = P + 1;
    for (int t = threadIdx.x; t < g.n3; t += kThreads) twl[t] = tw[t];
    const T irho = T(1) / (T)p.sc[s].rho;
    const T h = T(0.70710678118654752440084436210485);
    const long long N = g.N;
    const long long cur = (long long)(p.sc[s].iters & 1) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ e = p.e + cur;
    const T* __restrict__ v = p.v + cur;
    const long long L = (long long)g.n1 * g.n2;
    const long long l0 = (long long)blockIdx.x * 2 * P;
    const int cnt = 2 * P * g.n3;
    T* Ar = reinterpret_cast<T*>(A);
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int ll = (int)fdiv((unsigned)idx, g.div_n3);
        const int k = idx - ll * g.n3;
        const long long l = l0 + ll;
        T d = T(0);
        if (l < L) {
            const int i = (int)fdiv((unsigned)l, g.div_n2);
            const int j = (int)l - i * g.n2;
            const int ip = (i + 1 == g.n1) ? 0 : i + 1, im = (i == 0) ? g.n1 - 1 : i - 1;
            const int jp = (j + 1 == g.n2) ? 0 : j + 1, jm = (j == 0) ? g.n2 - 1 : j - 1;
            const int kp = (k + 1 == g.n3) ? 0 : k + 1, km = (k == 0) ? g.n3 - 1 : k - 1;
            const long long row = l * g.n3;
            const long long p0 = row + k;
            const long long pxp = ((long long)ip * g.n2 + j) * g.n3 + k;
            const long long pxm = ((long long)im * g.n2 + j) * g.n3 + k;
            const long long pyp = ((long long)i * g.n2 + jp) * g.n3 + k;
            const long long pym = ((long long)i * g.n2 + jm) * g.n3 + k;
            const long long pzp = row + kp, pzm = row + km;
            // d = (1/sqrt2) sum_a [w1_a(p) - w1_a(p - e_a) + w2_a(p + e_a) - w2_a(p)]
            T sx = wcomp(e, v, 0 * N + p0, irho) - wcomp(e, v, 0 * N + pxm, irho) +
                   wcomp(e, v, 3 * N + pxp, irho) - wcomp(e, v, 3 * N + p0, irho);
            T sy = wcomp(e, v, 1 * N + p0, irho) - wcomp(e, v, 1 * N + pym, irho) +
                   wcomp(e, v, 4 * N + pyp, irho) - wcomp(e, v, 4 * N + p0, irho);
            T sz = wcomp(e, v, 2 * N + p0, irho) - wcomp(e, v, 2 * N + pzm, irho) +
                   wcomp(e, v, 5 * N + pzp, irho) - wcomp(e, v, 5 * N + p0, irho);
            d = h * (sx + sy + sz);
        }
        Ar[2 * (k * stride + (ll >> 1)) + (ll & 1)] = d;
    }
    __syncthreads();
    C* R = block_fft<C>(A, B, stride, P, az, twl);
    const int cnt2 = P * g.n3h;
    C* spec = p.spec + (size_t)s * g.Nh;
    for (int idx = threadIdx.x; idx < cnt2; idx += kThreads) {
        const int c = (int)fdiv((unsigned)idx, g.div_n3h);
        const int kz = idx - c * g.n3h;
        const C Z = R[kz * stride + c];
        const int km = (kz == 0) ? 0 : g.n3 - kz;
        const C Zm = cconj(R[km * stride + c]);
        const C S = cadd(Z, Zm), D = csub(Z, Zm);
        const long long la = l0 + 2 * c, lb = la + 1;
        if (la < L) spec[la * g.n3h + kz] = cmake<C>(T(0.5) * S.x, T(0.5) * S.y);
        if (lb < L) spec[lb * g.n3h + kz] = cmake<C>(T(0.5) * D.y, T(-0.5) * D.x);
    }
}

// ---------------------------------------------------------------------------
// Passes 2-4: FFTs along the strided axes of the half spectrum [n1][n2][n3h].
// MODE 0: forward along y.  MODE 2: inverse along y.
// MODE 1: forward along x, multiply by 1 / (N lambda(k)) with
//         lambda(k) = -sum_a 4 sin^2(pi k_a / N_a) and 0 at k = 0, inverse along x.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_fft_strided(Geom g, Ptrs<T> p, AxisPlan ap,
                                                          const cx<T>* __restrict__ tw, int LPB,
                                                          const T* __restrict__ sym1, const T* __restrict__ sym2,
                                                          const T* __restrict__ sym3, T inv_n) {
    using C = cx<T>;
    const int s = blockIdx.y;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = ap.n;
    C* twl = reinterpret_cast<C*>(smem_raw);
    C* A = twl + n;
    C* B = A + (size_t)n * (LPB + 1);
    const int stride = LPB + 1;
    for (int t = threadIdx.x; t < n; t += kThreads) twl[t] = tw[t];
    const long long nlines = (MODE == 1) ? (long long)g.n2 * g.n3h : (long long)g.n1 * g.n3h;
    const long long es = (MODE == 1) ? (long long)g.n2 * g.n3h : (long long)g.n3h;
    const long long l0 = (long long)blockIdx.x * LPB;
    C* spec = p.spec + (size_t)s * g.Nh;
    const int cnt = LPB * n;
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int m = idx / LPB;
        const int c = idx - m * LPB;
        const long long l = l0 + c;
        C val = cmake<C>(T(0), T(0));
        if (l < nlines) {
            long long base;
            if (MODE == 1) {
                base = l;
            } else {
                const long long i = fdiv((unsigned)l, g.div_n3h);
                base = i * g.n2 * g.n3h + (l - i * g.n3h);
            }
            val = spec[base + m * es];
            if (MODE == 2) val = cconj(val);
        }
        A[m * stride + c] = val;
    }
    __syncthreads();
    C* R = block_fft<C>(A, B, stride, LPB, ap, twl);
    if (MODE == 1) {
        for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
            const int m = idx / LPB;
            const int c = idx - m * LPB;
            const long long l = l0 + c;
            T gk = T(0);
            if (l < nlines) {
                const int k2 = (int)fdiv((unsigned)l, g.div_n3h);
                const int kz = (int)l - k2 * g.n3h;
                const T lam = sym1[m] + sym2[k2] + sym3[kz];
                gk = (lam > T(0)) ? -inv_n / lam : T(0);
            }
            const C z = R[m * stride + c];
            R[m * stride + c] = cmake<C>(z.x * gk, -z.y * gk);   // conj for the inverse transform
        }
        __syncthreads();
        C* other = (R == A) ? B : A;
        R = block_fft<C>(R, other, stride, LPB, ap, twl);
    }
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int m = idx / LPB;
        const int c = idx - m * LPB;
        const long long l = l0 + c;
        if (l < nlines) {
            long long base;
            if (MODE == 1) {
                base = l;
            } else {
                const long long i = fdiv((unsigned)l, g.div_n3h);
                base = i * g.n2 * g.n3h + (l - i * g.n3h);
            }
            C val = R[m * stride + c];
            if (MODE != 0) val = cconj(val);
            spec[base + m * es] = val;
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 5: complex-to-real inverse FFT along z, two real lines per transform.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_irfft_z(Geom g, Ptrs<T> p, AxisPlan az,
                                                      const cx<T>* __restrict__ tw, int P) {
    using C = cx<T>;
    const int s = blockIdx.y;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twl = reinterpret_cast<C*>(smem_raw);
    C* A = twl + g.n3;
    C* B = A + (size_t)g.n3 * (P + 1);
    const int stride = P + 1;
    for (int t = threadIdx.x; t < g.n3; t += kThreads) twl[t] = tw[t];
    const long long L = (long long)g.n1 * g.n2;
    const long long l0 = (long long)blockIdx.x * 2 * P;
    const C* spec = p.spec + (size_t)s * g.Nh;
    const int cnt = P * g.n3h;
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int c = (int)fdiv((unsigned)idx, g.div_n3h);
        const int kz = idx - c * g.n3h;
        const long long la = l0 + 2 * c, lb = la + 1;
        const C a = (la < L) ? spec[la * g.n3h + kz] : cmake<C>(T(0), T(0));
        const C b = (lb < L) ? spec[lb * g.n3h + kz] : cmake<C>(T(0), T(0));
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
    C* R = block_fft<C>(A, B, stride, P, az, twl);
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
template <typename T, bool OUT>
__global__ void __launch_bounds__(kThreads) k_update(Geom g, Ptrs<T> p, LoopConfig cfg) {
    const int s = blockIdx.y;
    SolveScalars& S = p.sc[s];
    if (!OUT && !S.active) return;
    const long long N = g.N;
    const double rho_d = S.rho;
    const T rho = (T)rho_d;
    const T irho = T(1) / rho;
    const T h = T(0.70710678118654752440084436210485);
    const T xi0 = (T)S.xi[0], xi1 = (T)S.xi[1], xi2 = (T)S.xi[2];
    const T alpha = (T)(2.0 * (1.0 - cfg.delta)), beta = (T)(1.0 - 2.0 * cfg.delta);
    // read the current copy of the state, write the other one (the stencil reads
    // neighbours, so an in-place update would race)
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ phi = p.phi + (size_t)s * N;
    const T* __restrict__ gam = p.gamma + (size_t)s * p.gstride;
    T acc[kNSum];
#pragma unroll
    for (int q = 0; q < kNSum; ++q) acc[q] = T(0);
    const long long gstride = (long long)gridDim.x * kThreads;
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < N; lin += gstride) {
        const unsigned row = fdiv((unsigned)lin, g.div_n3);
        const int k = (int)(lin - (long long)row * g.n3);
        const unsigned i = fdiv(row, g.div_n2);
        const int j = (int)(row - i * g.n2);
        const long long base_i = (long long)i * g.n2 * g.n3;
        const long long base_j = (long long)j * g.n3;
        const int ip = ((int)i + 1 == g.n1) ? 0 : (int)i + 1, im = (i == 0) ? g.n1 - 1 : (int)i - 1;
        const int jp = (j + 1 == g.n2) ? 0 : j + 1, jm = (j == 0) ? g.n2 - 1 : j - 1;
        const int kp = (k + 1 == g.n3) ? 0 : k + 1, km = (k == 0) ? g.n3 - 1 : k - 1;
        const long long nb_p[3] = {(long long)ip * g.n2 * g.n3 + base_j + k, base_i + (long long)jp * g.n3 + k,
                                   base_i + base_j + kp};
        const long long nb_m[3] = {(long long)im * g.n2 * g.n3 + base_j + k, base_i + (long long)jm * g.n3 + k,
                                   base_i + base_j + km};
        T ec[6], vc[6], w[6], xh[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            ec[c] = e[c * N + lin];
            vc[c] = v[c * N + lin];
            w[c] = ec[c] - vc[c] * irho;
        }
        const T ph0 = phi[lin];
        const T xi[3] = {xi0, xi1, xi2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const long long qp = nb_p[a], qm = nb_m[a];
            const T w2p = e[(3 + a) * N + qp] - v[(3 + a) * N + qp] * irho;   // w2_a(p + e_a)
            const T w1m = e[a * N + qm] - v[a * N + qm] * irho;               // w1_a(p - e_a)
            const T ua = h * (w[a] + w2p);                                    // (A* w)_a(p)
            const T uam = h * (w1m + w[3 + a]);                               // (A* w)_a(p - e_a)
            const T ya = ua - (phi[qp] - ph0) - xi[a];
            const T yam = uam - (ph0 - phi[qm]) - xi[a];
            xh[a] = w[a] - h * ya;
            xh[3 + a] = w[3 + a] - h * yam;
        }
        const T gm = gam[lin];
        T r2 = T(0), nx2 = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const T dd = ec[c] - xh[c];
            r2 += dd * dd;
            nx2 += xh[c] * xh[c];
            acc[kSumV + c] += vc[c];
        }
        acc[kSumRes] += r2;
        acc[kSumPrimal] += gm * Real<T>::sqrt_(nx2);
        if (OUT) {
            if (p.cut) {
                T* cut = p.cut + (size_t)s * 6 * N;
#pragma unroll
                for (int c = 0; c < 6; ++c) cut[c * N + lin] = xh[c];
            }
            if (p.flow) {
                T* flow = p.flow + (size_t)s * 3 * N;
#pragma unroll
                for (int a = 0; a < 3; ++a) flow[a * N + lin] = h * (vc[a] + v[(3 + a) * N + nb_p[a]]);
            }
        } else {
            T z[6];
            T nz2 = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                z[c] = vc[c] + rho * (alpha * xh[c] - beta * ec[c]);
                nz2 += z[c] * z[c];
            }
            const T nz = Real<T>::sqrt_(nz2);
            const T scale = (nz > gm) ? gm / nz : T(1);
            T dvde = T(0), dede = T(0), dvdv = T(0), vv = T(0), ee = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const T vn = z[c] * scale;
                const T en = (z[c] - vn) * irho;
                const T dv = vn - vc[c], de = en - ec[c];
                dvde += dv * de;
                dede += de * de;
                dvdv += dv * dv;
                vv += vn * vn;
                ee += en * en;
                e_out[c * N + lin] = en;
                v_out[c * N + lin] = vn;
            }
            acc[kSumDvDe] += dvde;
            acc[kSumDeDe] += dede;
            acc[kSumDvDv] += dvdv;
            acc[kSumVV] += vv;
            acc[kSumEE] += ee;
        }
    }
    const int nblocks = gridDim.x;
    double* part = p.partial + (size_t)s * nblocks * kNSum;
    const bool last = block_partials<T, kNSum>(acc, part, &S.counter, nblocks, blockIdx.x);
    if (!last) return;
    double sums[kNSum];
    reduce_partials<kNSum>(part, nblocks, sums);
    if (threadIdx.x != 0) return;
    S.counter = 0;
    const double Nd = (double)N;
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
    }
    double rho_new = rho_d;
    const double lo = rho_d / cfg.rho_step_max, hi = rho_d * cfg.rho_step_max;
    if (cfg.rho_rule == 0) {
        const double sve = sums[kSumDvDe], see = sums[kSumDeDe], svv = sums[kSumDvDv];
        if (sve > 0.0 && see > 0.0 && svv > 0.0 && sve / sqrt(svv * see) > cfg.bb_corr_min)
            rho_new = fmin(fmax(sve / see, lo), hi);
    } else if (cfg.rho_rule == 2) {
        const double nv = sqrt(sums[kSumVV]), ne = sqrt(sums[kSumEE]);
        if (nv > 0.0 && ne > 0.0) rho_new = fmin(fmax(nv / ne, lo), hi);
    }
    const int done = kk + 1 - S.call_start;
    S.iters = kk + 1;
    bool stop = false;
    if (!finite || !isfinite(rho_new) || !(rho_new > 0.0)) {
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

}  // namespace ccmf
