// Batched persistent launch: one ADMM iteration (Eq. 28 and Eq. 30 of the paper) of
// every solve of a batch of grids of different shapes in ONE kernel launch.
//
// The launch runs six passes per solve as work items (pass, solve, tile):
//   pass 0  w = e - v / rho, d = div^- A* w (Sec. 2.2, Eq. 17) and the real-to-complex
//           FFT along z (two real lines per complex transform), tiles of 2P lines;
//   pass 1  forward FFT along y (decimation in frequency: digit-reversed y order),
//           tiles of L lines;
//   pass 2  forward FFT along x, the Poisson gain phi^ = d^ / (N lambda(k)) with
//           lambda(k) = -sum_a 4 sin^2(pi k_a / N_a), phi^(0) = 0 ((div^- grad^+)^+ of
//           Eq. 28), inverse FFT along x, tiles of L lines;
//   pass 3  inverse FFT along y, tiles of L lines;
//   pass 4  complex-to-real inverse FFT along z -> phi, tiles of 2P lines;
//   pass 5  xi^{k+1/2} = P_K(w), over-relaxation, z = v + rho xi, projection onto
//           C_gamma (Eq. 19), e^{k+1}, v^{k+1} (Eq. 30) and the partial sums of one
//           chunk of voxels; the chunk that completes the pass reduces the partials in
//           chunk order and runs the penalty rule, history and stop test of the solve.
// The items sit in one queue in pass-major order: every solve's pass-0 tiles, then every
// solve's pass-1 tiles, and so on. A grid of resident blocks takes items in queue order
// from one atomic ticket. An item of pass p > 0 starts only once every item of pass p - 1
// of its solve has completed (a per-(solve, pass) counter, polled with a bounded wait that
// records CCMF_ERR_TIMEOUT in the solve's status and gives up). Every item an item waits on
// sits earlier in the queue and was taken by a block that is running, so the earliest
// unfinished item never waits and the launch always progresses, whatever the number of
// blocks resident at a time.
// Data produced inside the launch (the half spectrum, phi, the partial sums) is read with
// L2-only loads (ld.global.cg): the incoherent L1 / read-only paths may hold lines of an
// earlier pass. The state e, v and gamma come from earlier launches and use the read-only
// path as in the other kernels.
#pragma once

#include "ccmf_kernels.cuh"

namespace ccmf {

constexpr int kPersistPasses = 6;
// Blocks per SM the persistent kernel's register budget is sized for (a build-time knob): three
// blocks (80 registers, a few spilled bytes in the update body) ran the 192-solve batch in
// 14.5 ms per iteration on GB300 against 16.6 ms with two (128 registers, no spills).
#ifndef CCMF_PERSIST_MIN_BLOCKS
#define CCMF_PERSIST_MIN_BLOCKS 3
#endif
constexpr int kPersistMinBlocks = CCMF_PERSIST_MIN_BLOCKS;

// One shape group of the batch (a sub-plan's grid, workspace slice and tables).
template <typename T>
struct PersistGroup {
    Geom g;
    Ptrs<T> p;                  // the group's workspace; p.partial = the persistent chunk slots
    AxisPlan ax[3];             // x, y, z radix schedules of the in-place and Stockham stages
    const cx<T>* tw[3];         // W_n^t, t < n, per axis
    const T* rsym_x;            // 4 sin^2(pi k / n1) in the digit-reversed order of the x DIF stages
    const T* rsym_y;            // the same for y (the order pass 1 leaves)
    const T* sym_z;             // 4 sin^2(pi k / n3), natural order
    FastDiv div_l;              // the tile's line count L (in-place stage indexing)
    T inv_n;                    // 1 / N
    int vec_div;                // pass 0 reads 16-byte vectors (n3 % (16 / sizeof(T)) == 0)
    int upd_w;                  // voxels per thread group of pass 5 (vector width)
    long long nchunks;          // pass-5 chunks per solve
    int tiles[kPersistPasses];  // tiles per solve of each pass (pass 5: chunks)
    int tpi[kPersistPasses];    // consecutive tiles per work item (1 for pass 5: one partial slot per chunk)
    int ntiles[kPersistPasses]; // items per solve of each pass: ceil(tiles / tpi)
};

template <typename T>
struct PersistArgs {
    const PersistGroup<T>* groups;
    const long long* pg_base;   // [kPersistPasses * ngroups + 1] first item of (pass, group), pass-major;
                                // inside (pass, group) the group's solves follow one another, ntiles each
    const int* gstart;          // [ngroups] index j of each group's first solve (solves numbered group by group)
    unsigned* done;             // [nsolve][kPersistPasses] completed items (zeroed before each launch)
    unsigned* head;             // next item of the queue (zeroed before each launch)
    int ngroups, nsolve;
    int tw_off, work_off;       // byte offsets of the twiddle table and the tile buffers in dynamic shared memory
    LoopConfig cfg;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ float2 ldcg_cx(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg_cx(const double2* p) { return __ldcg(p); }

// W consecutive elements through L2 only.
template <typename T, int W> struct VecCg;
template <> struct VecCg<float, 2> {
    __device__ __forceinline__ static void ld(const float* p, float (&o)[2]) {
        const float2 t = __ldcg(reinterpret_cast<const float2*>(p));
        o[0] = t.x; o[1] = t.y;
    }
};
template <> struct VecCg<float, 1> {
    __device__ __forceinline__ static void ld(const float* p, float (&o)[1]) { o[0] = __ldcg(p); }
};
template <> struct VecCg<double, 1> {
    __device__ __forceinline__ static void ld(const double* p, double (&o)[1]) { o[0] = __ldcg(p); }
};

// Dynamic shared memory of k_batch_persist, in three parts: the queue tables (first item of
// every (pass, group), each group's scalar slots, first solve and tiles per pass), the
// twiddle table of the current axis (kept while consecutive items use the same one) and
// the tile buffers.
__host__ __device__ inline size_t persist_off_sc(int ng) {
    return ((size_t)(kPersistPasses * ng + 1) * 8 + 15) / 16 * 16;
}
__host__ __device__ inline size_t persist_off_start(int ng) { return persist_off_sc(ng) + (size_t)ng * 8; }
__host__ __device__ inline size_t persist_table_bytes(int ng) {
    return (persist_off_start(ng) + (size_t)ng * 4 * (1 + kPersistPasses) + 15) / 16 * 16;
}
// Tile buffers (bytes) of a group of this shape.
template <typename T>
__host__ __device__ inline size_t persist_work_bytes(int n1, int n2, int n3, int P, int L) {
    const size_t z = 2 * (size_t)n3 * (P + 1);
    const size_t y = (size_t)n2 * (L + 1);
    const size_t x = (size_t)n1 * (L + 1);
    size_t m = z > y ? z : y;
    m = m > x ? m : x;
    return m * sizeof(cx<T>);
}

// Pass 0 on tile t: line pairs (2q, 2q + 1), q in [t P, t P + P), packed as the real and
// imaginary parts of one complex line (as k_div_rfft_z).
template <typename T, int P, bool VEC>
__device__ void persist_div_rfft_z(const PersistGroup<T>& G, int s, long long t, const cx<T>* twl,
                                   unsigned char* work) {
    using C = cx<T>;
    constexpr int stride = P + 1;
    constexpr int W = VEC ? Vec16<T>::W : 1;
    const Geom& g = G.g;
    const Ptrs<T>& p = G.p;
    C* A = reinterpret_cast<C*>(work);
    C* B = A + (size_t)g.n3 * stride;
    const T irho = T(1) / (T)p.sc[s].rho;
    const T h = T(0.70710678118654752440084436210485);
    const long long N = g.N;
    const long long cur = (long long)(p.sc[s].iters & 1) * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ e = p.e + cur;
    const T* __restrict__ v = p.v + cur;
    const long long Lp = (long long)g.n1 * g.n2;
    const long long l0 = t * 2 * P;
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
        if (l < Lp) {
            const RowNb rn = row_neighbours(g, (unsigned)l);
            const int kp = (k0 + W == g.n3) ? 0 : k0 + W;
            const int km = (k0 == 0) ? g.n3 - 1 : k0 - 1;
            if constexpr (VEC) {
                T w[6][W], te[W], tv[W];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    Vec16<T>::ld(e + c * N + rn.row + k0, te);
                    Vec16<T>::ld(v + c * N + rn.row + k0, tv);
#pragma unroll
                    for (int u = 0; u < W; ++u) w[c][u] = te[u] - tv[u] * irho;
                }
                T xp[W], xm[W], yp[W], ym[W];
                Vec16<T>::ld(e + 3 * N + rn.ip + k0, te);
                Vec16<T>::ld(v + 3 * N + rn.ip + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) xp[u] = te[u] - tv[u] * irho;
                Vec16<T>::ld(e + 0 * N + rn.im + k0, te);
                Vec16<T>::ld(v + 0 * N + rn.im + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) xm[u] = te[u] - tv[u] * irho;
                Vec16<T>::ld(e + 4 * N + rn.jp + k0, te);
                Vec16<T>::ld(v + 4 * N + rn.jp + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) yp[u] = te[u] - tv[u] * irho;
                Vec16<T>::ld(e + 1 * N + rn.jm + k0, te);
                Vec16<T>::ld(v + 1 * N + rn.jm + k0, tv);
#pragma unroll
                for (int u = 0; u < W; ++u) ym[u] = te[u] - tv[u] * irho;
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
    C* R = block_fft<C, P>(A, B, G.ax[2], twl);
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
        C* dst = spec + (long long)kz * Lp + la;
        if (la < Lp) dst[0] = cmake<C>(T(0.5) * Sm.x, T(0.5) * Sm.y);
        if (lb < Lp) dst[1] = cmake<C>(T(0.5) * D.y, T(-0.5) * D.x);
    }
}

// Passes 1 and 3 on tile t: L contiguous y lines (k_z, i) of the half spectrum, in place.
// MODE 0: forward (DIF, leaves digit-reversed y order). MODE 2: inverse of the
// conjugated data that pass 2 stores (DIT, natural order), conjugated on store.
template <typename T, int MODE, int L>
__device__ void persist_y_lines(const PersistGroup<T>& G, int s, long long t, const cx<T>* twl, unsigned char* work) {
    using C = cx<T>;
    constexpr int stride = L + 1;
    const Geom& g = G.g;
    const int n = g.n2;
    C* b = reinterpret_cast<C*>(work);
    const long long nlines = (long long)g.n3h * g.n1;
    C* spec = G.p.spec + (size_t)s * g.Nh;
    const long long l0 = t * L;
    const int cnt = L * n;
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int c = (int)fdiv((unsigned)idx, g.div_n2);
        const int m = idx - c * n;
        const long long l = l0 + c;
        b[m * stride + c] = (l < nlines) ? ldcg_cx(spec + l * n + m) : cmake<C>(T(0), T(0));
    }
    __syncthreads();
    inplace_fft<C, MODE == 0, kThreads>(b, G.ax[1], L, stride, 1, G.div_l, twl);
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int c = (int)fdiv((unsigned)idx, g.div_n2);
        const int m = idx - c * n;
        const long long l = l0 + c;
        if (l < nlines) {
            const C z = b[m * stride + c];
            spec[l * n + m] = (MODE == 2) ? cconj(z) : z;
        }
    }
}

// Pass 2 on tile t: L adjacent x lines (k_z, k_y) (stride n2): forward FFT (DIF), the
// Poisson gain from the digit-reversed x and y symbols, inverse as conj(DIT(conj(.)));
// the result is stored conjugated (pass 3 undoes it).
template <typename T, int L>
__device__ void persist_x_lines(const PersistGroup<T>& G, int s, long long t, const cx<T>* twl, unsigned char* work) {
    using C = cx<T>;
    constexpr int stride = L + 1;
    constexpr int lsh = (L >= 32) ? 5 : (L >= 16) ? 4 : (L >= 8) ? 3 : (L >= 4) ? 2 : (L >= 2) ? 1 : 0;
    static_assert((1 << lsh) == L, "L must be a power of two <= 32");
    constexpr int mstep = kThreads / L;
    const Geom& g = G.g;
    const int n = g.n1;
    C* b = reinterpret_cast<C*>(work);
    const long long plane = (long long)g.n1 * g.n2;
    const long long nlines = (long long)g.n3h * g.n2;
    C* spec = G.p.spec + (size_t)s * g.Nh;
    const int cl = threadIdx.x & (L - 1);
    const int m0 = threadIdx.x >> lsh;
    const long long l = t * L + cl;
    const bool valid = l < nlines;
    int kz = 0, k2 = 0;
    if (valid) {
        kz = (int)fdiv((unsigned)l, g.div_n2);
        k2 = (int)(l - (long long)kz * g.n2);
    }
    C* line = spec + (long long)kz * plane + k2;
    for (int m = m0; m < n; m += mstep)
        b[m * stride + cl] = valid ? ldcg_cx(line + (long long)m * g.n2) : cmake<C>(T(0), T(0));
    __syncthreads();
    inplace_fft<C, true, kThreads>(b, G.ax[0], L, stride, 1, G.div_l, twl);
    const T lam23 = valid ? G.rsym_y[k2] + G.sym_z[kz] : T(0);
    for (int m = m0; m < n; m += mstep) {
        const T lam = G.rsym_x[m] + lam23;
        const T gk = (valid && lam > T(0)) ? -G.inv_n / lam : T(0);
        const C z = b[m * stride + cl];
        b[m * stride + cl] = cmake<C>(z.x * gk, -z.y * gk);
    }
    __syncthreads();
    inplace_fft<C, false, kThreads>(b, G.ax[0], L, stride, 1, G.div_l, twl);
    if (valid)
        for (int m = m0; m < n; m += mstep) line[(long long)m * g.n2] = b[m * stride + cl];
}

// Pass 4 on tile t: the packed C2R along z of line pairs (2q, 2q + 1), q in [t P, t P + P)
// (as k_irfft_z), writing phi.
template <typename T, int P>
__device__ void persist_irfft_z(const PersistGroup<T>& G, int s, long long t, const cx<T>* twl, unsigned char* work) {
    using C = cx<T>;
    constexpr int stride = P + 1;
    const Geom& g = G.g;
    C* A = reinterpret_cast<C*>(work);
    C* B = A + (size_t)g.n3 * stride;
    const long long Lp = (long long)g.n1 * g.n2;
    const long long l0 = t * 2 * P;
    const C* spec = G.p.spec + (size_t)s * g.Nh;
    const int cnt = P * g.n3h;
    const bool staged = 2 * P <= g.n3;   // the raw slab fits the second buffer
    if (staged) {
        for (int idx = threadIdx.x; idx < 2 * cnt; idx += kThreads) {
            const int kz = idx / (2 * P);
            const int r = idx - kz * 2 * P;
            const long long l = l0 + r;
            B[idx] = (l < Lp) ? ldcg_cx(spec + (long long)kz * Lp + l) : cmake<C>(T(0), T(0));
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < cnt; idx += kThreads) {
        const int kz = idx / P;
        const int c = idx - kz * P;
        const long long la = l0 + 2 * c, lb = la + 1;
        const C* src = spec + (long long)kz * Lp + la;
        C a, b;
        if (staged) {
            a = B[kz * 2 * P + 2 * c];
            b = B[kz * 2 * P + 2 * c + 1];
        } else {
            a = (la < Lp) ? ldcg_cx(src) : cmake<C>(T(0), T(0));
            b = (lb < Lp) ? ldcg_cx(src + 1) : cmake<C>(T(0), T(0));
        }
        if (kz == 0 || 2 * kz == g.n3) {
            A[kz * stride + c] = cmake<C>(a.x, -b.x);
        } else {
            A[kz * stride + c] = cmake<C>(a.x - b.y, -(a.y + b.x));
            A[(g.n3 - kz) * stride + c] = cmake<C>(a.x + b.y, a.y - b.x);
        }
    }
    __syncthreads();
    C* R = block_fft<C, P>(A, B, G.ax[2], twl);
    const int cnt2 = 2 * P * g.n3;
    T* phi = G.p.phi + (size_t)s * g.N;
    for (int idx = threadIdx.x; idx < cnt2; idx += kThreads) {
        const int ll = (int)fdiv((unsigned)idx, g.div_n3);
        const int k = idx - ll * g.n3;
        const long long l = l0 + ll;
        if (l < Lp) {
            const C z = R[k * stride + (ll >> 1)];
            phi[l * g.n3 + k] = (ll & 1) ? -z.y : z.x;
        }
    }
}

// Pass 5 on chunk ck: kVecChunkGroups x kThreads groups of W consecutive voxels of a z line
// (as the chunks of k_update_vec); stores the chunk's partial sums in slot ck.
template <typename T, int W>
__device__ void persist_update(const PersistGroup<T>& G, int s, long long ck, const LoopConfig& cfg) {
    using V = VecN<T, W>;
    using VC = VecCg<T, W>;
    const Geom& g = G.g;
    const Ptrs<T>& p = G.p;
    const SolveScalars& S = p.sc[s];
    const long long N = g.N;
    const StepConsts<T> K = step_consts<T>(S, cfg);
    const int par = S.iters & 1;
    const T* __restrict__ e = p.e + (long long)par * p.sstride + (long long)s * 6 * N;
    const T* __restrict__ v = p.v + (long long)par * p.sstride + (long long)s * 6 * N;
    T* __restrict__ e_out = p.e + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    T* __restrict__ v_out = p.v + (long long)(1 - par) * p.sstride + (long long)s * 6 * N;
    const T* phi = p.phi + (size_t)s * N;   // written by pass 4 of this launch: L2-only loads
    const T* __restrict__ gam = gamma_of(p, s);
    const long long ngroups = N / W;
    T acc[kNSum];
#pragma unroll
    for (int q = 0; q < kNSum; ++q) acc[q] = T(0);
#pragma unroll 1
    for (int gi = 0; gi < kVecChunkGroups; ++gi) {
        const long long q = (ck * kVecChunkGroups + gi) * kThreads + threadIdx.x;
        if (q >= ngroups) break;
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
        VC::ld(phi + lin0, ph);
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
        VC::ld(phi + rn.ip + k0, phxp);
        VC::ld(phi + rn.im + k0, phxm);
        VC::ld(phi + rn.jp + k0, phyp);
        VC::ld(phi + rn.jm + k0, phym);
        const T e2z_after = __ldg(e + 5 * N + rn.row + kp), v2z_after = __ldg(v + 5 * N + rn.row + kp);
        const T e1z_before = __ldg(e + 2 * N + rn.row + km), v1z_before = __ldg(v + 2 * N + rn.row + km);
        const T ph_after = __ldcg(phi + rn.row + kp), ph_before = __ldcg(phi + rn.row + km);
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
            voxel_step<T, false>(K, ecu, vcu, gm[u], ph[u], php, phm, e2p, v2p, e1m, v1m, acc, eou, vou, fl);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                eo[c][u] = eou[c];
                vo[c][u] = vou[c];
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            V::st(e_out + c * N + lin0, eo[c]);
            V::st(v_out + c * N + lin0, vo[c]);
        }
    }
    block_store_partial<T, kNSum>(acc, p.partial + (size_t)s * G.nchunks * kNSum, ck);
}

// Bounded wait of thread 0 until *ctr >= need (acquire). Returns false when the budget
// (cfg.spin_limit - 1 polls when set, else kSpinLimit) runs out.
__device__ __forceinline__ bool persist_wait(const unsigned* ctr, unsigned need, unsigned budget) {
    for (unsigned it = 0; it < budget; ++it) {
        if (ld_acquire_gpu(ctr) >= need) return true;
        __nanosleep(it < 32 ? 32 : 256);
    }
    return false;
}

// The persistent kernel: P line pairs per z tile, L lines per y / x tile.
// Thread 0 of a block takes the tickets: it fetches the next one while the current item
// runs (a block holds at most one item that has not started, so the earliest unfinished
// item is always running or about to start), decodes an item from the (pass, group) table
// in shared memory, and remembers which (solve, pass) dependency it has already seen
// complete and the active flag of the last solve it decoded.
template <typename T, int P, int L>
__global__ void __launch_bounds__(kThreads, kPersistMinBlocks) k_batch_persist(PersistArgs<T> a) {
    using C = cx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) PersistGroup<T> sg;   // the current item's group, copied from global memory
    __shared__ long long s_tile;
    __shared__ int s_pass, s_j, s_group, s_local, s_run, s_last, s_loaded, s_twkey;
    static_assert(sizeof(PersistGroup<T>) % 4 == 0, "group copy by words");
    const int ng = a.ngroups;
    long long* t_base = reinterpret_cast<long long*>(smem_raw);
    SolveScalars** t_sc = reinterpret_cast<SolveScalars**>(smem_raw + persist_off_sc(ng));
    int* t_start = reinterpret_cast<int*>(smem_raw + persist_off_start(ng));
    int* t_tiles = t_start + ng;
    C* twl = reinterpret_cast<C*>(smem_raw + a.tw_off);
    unsigned char* work = smem_raw + a.work_off;
    for (int i = threadIdx.x; i <= kPersistPasses * ng; i += kThreads) t_base[i] = a.pg_base[i];
    for (int b = threadIdx.x; b < ng; b += kThreads) {
        t_sc[b] = a.groups[b].p.sc;
        t_start[b] = a.gstart[b];
    }
    for (int i = threadIdx.x; i < ng * kPersistPasses; i += kThreads)
        t_tiles[i] = a.groups[i / kPersistPasses].ntiles[i % kPersistPasses];
    const unsigned budget = a.cfg.spin_limit ? a.cfg.spin_limit - 1 : kSpinLimit;
    long long next = 0;
    int ok_j = -1, ok_p = -1, act_j = -1, act_v = 0;   // thread 0's caches
    if (threadIdx.x == 0) {
        s_loaded = -1;
        s_twkey = -1;
        next = (long long)atomicAdd(a.head, 1u);
    }
    for (;;) {
        __syncthreads();   // tables ready; every thread is done with the previous item's shared values
        if (threadIdx.x == 0) {
            const long long item = next;
            const long long total = t_base[kPersistPasses * ng];
            int pass = -1, j = 0, grp = 0, loc = 0, run = 0;
            long long tile = 0;
            if (item < total) {
                next = (long long)atomicAdd(a.head, 1u);   // the following ticket, while this item runs
                pass = 0;
                while (pass + 1 < kPersistPasses && item >= t_base[(pass + 1) * ng]) ++pass;
                while (grp + 1 < ng && item >= t_base[pass * ng + grp + 1]) ++grp;
                const long long off = item - t_base[pass * ng + grp];
                const long long nt = t_tiles[grp * kPersistPasses + pass];
                const long long q = off / nt;
                tile = off - q * nt;
                loc = (int)q;
                j = t_start[grp] + loc;
                // a solve's active flag changes only when its last pass-5 item completes, after
                // every other item of the solve in this launch
                if (j != act_j) {
                    act_j = j;
                    act_v = t_sc[grp][loc].active;
                }
                run = act_v ? 1 : 0;
                if (run && pass > 0 && !(j == ok_j && pass == ok_p)) {
                    const unsigned* ctr = a.done + (size_t)j * kPersistPasses + (pass - 1);
                    if (persist_wait(ctr, (unsigned)t_tiles[grp * kPersistPasses + pass - 1], budget)) {
                        ok_j = j;
                        ok_p = pass;
                    } else {
                        atomicCAS(&t_sc[grp][loc].status, 0, 6);   // CCMF_ERR_TIMEOUT; the solve retires
                        run = 2;                                    // at its pass-5 completion
                    }
                }
            }
            s_pass = pass;
            s_j = j;
            s_group = grp;
            s_local = loc;
            s_run = run;
            s_tile = tile;
        }
        __syncthreads();
        const int pass = s_pass;
        if (pass < 0) break;
        const int run = s_run;
        if (run == 0) continue;   // a retired solve: its items are skipped
        const int j = s_j, grp = s_group, s = s_local;
        const long long tile = s_tile;
        const int axis = (pass == 2) ? 0 : (pass == 1 || pass == 3) ? 1 : 2;
        const int twkey = grp * 3 + axis;
        // both decisions are taken before thread 0 updates s_loaded / s_twkey below
        const bool new_group = grp != s_loaded;
        const bool new_tw = run == 1 && pass < kPersistPasses - 1 && twkey != s_twkey;
        if (new_group) {
            const int* src = reinterpret_cast<const int*>(a.groups + grp);
            int* dst = reinterpret_cast<int*>(&sg);
            for (int w = threadIdx.x; w < (int)(sizeof(PersistGroup<T>) / 4); w += kThreads) dst[w] = src[w];
        }
        if (new_group || new_tw) __syncthreads();
        if (new_tw) {
            const int n = axis == 0 ? sg.g.n1 : axis == 1 ? sg.g.n2 : sg.g.n3;
            for (int i = threadIdx.x; i < n; i += kThreads) twl[i] = sg.tw[axis][i];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_loaded = grp;
            if (new_tw) s_twkey = twkey;
        }
        if (run == 1 && pass < kPersistPasses - 1) {
            // an item covers tpi consecutive tiles of its pass
            const long long t0 = tile * sg.tpi[pass];
            const long long t1 = min(t0 + sg.tpi[pass], (long long)sg.tiles[pass]);
            for (long long t = t0; t < t1; ++t) {
                if (t > t0) __syncthreads();   // the previous tile's buffers have been stored
                switch (pass) {
                    case 0:
                        if (sg.vec_div)
                            persist_div_rfft_z<T, P, true>(sg, s, t, twl, work);
                        else
                            persist_div_rfft_z<T, P, false>(sg, s, t, twl, work);
                        break;
                    case 1: persist_y_lines<T, 0, L>(sg, s, t, twl, work); break;
                    case 2: persist_x_lines<T, L>(sg, s, t, twl, work); break;
                    case 3: persist_y_lines<T, 2, L>(sg, s, t, twl, work); break;
                    default: persist_irfft_z<T, P>(sg, s, t, twl, work); break;
                }
            }
        } else if (run == 1) {
            switch (pass) {
                default:
                    if constexpr (sizeof(T) == 4) {
                        if (sg.upd_w == 2)
                            persist_update<T, 2>(sg, s, tile, a.cfg);
                        else
                            persist_update<T, 1>(sg, s, tile, a.cfg);
                    } else {
                        persist_update<T, 1>(sg, s, tile, a.cfg);
                    }
                    break;
            }
        }
        __syncthreads();   // every thread's writes of this item precede thread 0's release below
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned old = atomicAdd(a.done + (size_t)j * kPersistPasses + pass, 1u);
            s_last = (pass == kPersistPasses - 1) && (old + 1 == (unsigned)t_tiles[grp * kPersistPasses + pass]);
            if (s_last) __threadfence();
        }
        __syncthreads();
        if (s_last) {
            // every chunk of the solve has stored its partials: reduce them in chunk order, then
            // the penalty rule, history row and stop test (rho, iters, active change here)
            SolveScalars& S = sg.p.sc[s];
            const double* part = sg.p.partial + (size_t)s * sg.nchunks * kNSum;
            update_finish<T, false>(sg.g, sg.p, a.cfg, S, s, S.rho, part, (int)sg.nchunks);
        }
    }
}

}  // namespace ccmf
