// Mixed-radix (2, 3, 4, 5, 8) Stockham FFT of a tile of lines held in shared memory.
//
// The Poisson solve inside the projection onto K (Eq. 28 of the paper,
// Gamma = grad^+ (div^- grad^+)^+ div^-) is diagonal in Fourier space; these
// routines provide the forward transforms X[m] = sum_t x[t] exp(-2 pi i m t / n)
// that the solver kernels apply along each grid axis. The inverse transform is
// obtained by conjugating input and output.
//
// Tile layout: `lines` complex lines of length n, element m of line c at
// buf[m * stride + c] (stride >= lines; stride = lines + 1 avoids bank conflicts).
// Each stage of radix R reads from one buffer and writes to the other
// (autosort: the result is in natural order), so the caller provides two buffers
// and gets back the one that holds the result.
#pragma once

#include <cuda_runtime.h>

namespace ccmf {

constexpr int kMaxStages = 12;

// Unsigned division by a fixed divisor through a multiply-high and shift
// (Granlund & Montgomery, PLDI 1994): q = (umulhi(n, m) + n) >> s, exact for n < 2^32.
struct FastDiv {
    unsigned d, m, s;
};

inline FastDiv make_fastdiv(unsigned d) {
    FastDiv f;
    f.d = d;
    unsigned s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    f.m = (unsigned)((((1ull << 32) * ((1ull << s) - d)) / d) + 1ull);
    return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
    return (unsigned)(((unsigned long long)__umulhi(n, f.m) + n) >> f.s);
}

struct AxisPlan {
    int n;                     // line length
    int nst;                   // number of radix stages
    int rad[kMaxStages];       // radix of each stage, product = n
    FastDiv ns[kMaxStages];    // divisor Ns (product of the earlier radices) of each stage
    int span[kMaxStages];      // in-place stages: sub-transform length Ls = n / (rad[0] ... rad[st-1])
    FastDiv sub[kMaxStages];   // in-place stages: divisor m = Ls / rad[st]
};

template <typename T> struct CxOf;
template <> struct CxOf<float> { using type = float2; };
template <> struct CxOf<double> { using type = double2; };
template <typename T> using cx = typename CxOf<T>::type;

template <typename C> __device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
// multiply by -i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmake<C>(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmake<C>(a.x * s, a.y * s); }

// In-register forward DFTs of size R (omega = exp(-2 pi i / R)).
template <typename C, int R> struct Dft;

template <typename C> struct Dft<C, 2> {
    __device__ __forceinline__ static void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <typename C> struct Dft<C, 4> {
    __device__ __forceinline__ static void run(C* v) {
        C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        C s13 = cadd(v[1], v[3]), d13 = cmul_mi(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <typename C> struct Dft<C, 8> {
    __device__ __forceinline__ static void run(C* v) {
        using R = decltype(C::x);
        const R h = R(0.70710678118654752440084436210485);
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<C, 4>::run(e);
        Dft<C, 4>::run(o);
        // o[m] *= exp(-2 pi i m / 8)
        C o1 = cmake<C>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        C o2 = cmul_mi(o[2]);
        C o3 = cmake<C>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <typename C> struct Dft<C, 3> {
    __device__ __forceinline__ static void run(C* v) {
        using R = decltype(C::x);
        const R s = R(0.86602540378443864676372317075294);  // sin(2 pi / 3)
        C t = cadd(v[1], v[2]);
        C m = cmake<C>(v[0].x - R(0.5) * t.x, v[0].y - R(0.5) * t.y);
        C d = csub(v[1], v[2]);
        C j = cmake<C>(s * d.y, -s * d.x);  // -i s (b - c)
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, j);
        v[2] = csub(m, j);
    }
};

template <typename C> struct Dft<C, 5> {
    __device__ __forceinline__ static void run(C* v) {
        using R = decltype(C::x);
        const R c1 = R(0.30901699437494742410229341718282);   // cos(2 pi / 5)
        const R c2 = R(-0.80901699437494742410229341718282);  // cos(4 pi / 5)
        const R s1 = R(0.95105651629515357211643933337938);   // sin(2 pi / 5)
        const R s2 = R(0.58778525229247312916870595463907);   // sin(4 pi / 5)
        C a = v[0];
        C p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
        C p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
        C r1 = cmake<C>(a.x + c1 * p1.x + c2 * p2.x, a.y + c1 * p1.y + c2 * p2.y);
        C r2 = cmake<C>(a.x + c2 * p1.x + c1 * p2.x, a.y + c2 * p1.y + c1 * p2.y);
        // i1 = s1 m1 + s2 m2 ; i2 = s2 m1 - s1 m2 ; X1 = r1 - i i1, X4 = r1 + i i1 ; X2 = r2 - i i2, X3 = r2 + i i2
        C i1 = cmake<C>(s1 * m1.x + s2 * m2.x, s1 * m1.y + s2 * m2.y);
        C i2 = cmake<C>(s2 * m1.x - s1 * m2.x, s2 * m1.y - s1 * m2.y);
        v[0] = cadd(a, cadd(p1, p2));
        v[1] = cmake<C>(r1.x + i1.y, r1.y - i1.x);
        v[4] = cmake<C>(r1.x - i1.y, r1.y + i1.x);
        v[2] = cmake<C>(r2.x + i2.y, r2.y - i2.x);
        v[3] = cmake<C>(r2.x - i2.y, r2.y + i2.x);
    }
};

// One Stockham stage of radix R over LINES lines (LINES a power of two):
// butterfly j of line c reads elements j + r n/R, applies the twiddles
// W_{Ns R}^{(j mod Ns) r}, transforms, and writes to
// (j div Ns) Ns R + (j mod Ns) + r Ns.
template <typename C, int R, int LINES>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst, int n,
                                               const FastDiv& nsd, const C* __restrict__ tw) {
    constexpr int stride = LINES + 1;
    constexpr int lsh = (LINES >= 16) ? 4 : (LINES >= 8) ? 3 : (LINES >= 4) ? 2 : (LINES >= 2) ? 1 : 0;
    static_assert((1 << lsh) == LINES, "LINES must be a power of two <= 16");
    const int Ns = (int)nsd.d;
    const int nR = n / R;
    const int total = LINES * nR;
    const int twstep = n / (Ns * R);
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int c = q & (LINES - 1);
        const int j = q >> lsh;
        const int jm = j - (int)fdiv((unsigned)j, nsd) * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * nR) * stride + c];
        if (Ns > 1) {
            const int t = jm * twstep;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[t * r]);
        }
        Dft<C, R>::run(v);
        const int od = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(od + r * Ns) * stride + c] = v[r];
    }
}

// Forward FFT of LINES lines (layout above, stride LINES + 1). Must be called by
// all threads of the block; ends with a barrier. Returns the buffer that holds
// the result.
template <typename C, int LINES>
__device__ C* block_fft(C* a, C* b, const AxisPlan& ap, const C* __restrict__ tw) {
    for (int st = 0; st < ap.nst; ++st) {
        const int R = ap.rad[st];
        switch (R) {
            case 8: stockham_stage<C, 8, LINES>(a, b, ap.n, ap.ns[st], tw); break;
            case 4: stockham_stage<C, 4, LINES>(a, b, ap.n, ap.ns[st], tw); break;
            case 2: stockham_stage<C, 2, LINES>(a, b, ap.n, ap.ns[st], tw); break;
            case 3: stockham_stage<C, 3, LINES>(a, b, ap.n, ap.ns[st], tw); break;
            default: stockham_stage<C, 5, LINES>(a, b, ap.n, ap.ns[st], tw); break;
        }
        __syncthreads();
        C* t = a;
        a = b;
        b = t;
    }
    return a;
}

// In-place mixed-radix Cooley-Tukey stages on lines held in shared memory
// (element m of line c at buf[c * ls + m * es]). Stage st works on blocks of Ls
// elements; butterfly (block b, offset j < m = Ls / R) combines the elements
// b Ls + j + r m, r < R, and writes its outputs back to the same slots, so a stage
// needs no second buffer. Decimation in frequency (DIF: transform, then twiddle
// W_Ls^{j q}) maps natural order to digit-reversed order: slot p holds
// frequency k(p) = sum_s q_s prod_{t<s} R_t with q_s = (p / m_s) mod R_s.
// Decimation in time (DIT: twiddle, then transform, stages in reverse order)
// maps digit-reversed input to natural-order output. Both use the forward
// kernel exp(-2 pi i / n). Threads take consecutive lines first.
template <typename C, int R, bool DIF, int NT>
__device__ __forceinline__ void inplace_stage(C* buf, int n, int nlines, int es, int ls, int Ls,
                                              const FastDiv& msub, const FastDiv& nld,
                                              const C* __restrict__ tw) {
    const int m = (int)msub.d;
    const int total = nlines * (n / R);
    const int tws = n / Ls;
    for (int q = threadIdx.x; q < total; q += NT) {
        const int bj = (int)fdiv((unsigned)q, nld);
        const int c = q - bj * nlines;
        const int b = (int)fdiv((unsigned)bj, msub);
        const int j = bj - b * m;
        C* x = buf + c * ls + (b * Ls + j) * es;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[r * m * es];
        if (DIF) {
            Dft<C, R>::run(v);
            if (j > 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * tws]);
            }
        } else {
            if (j > 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * tws]);
            }
            Dft<C, R>::run(v);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) x[r * m * es] = v[r];
    }
    __syncthreads();
}

template <typename C, bool DIF, int NT>
__device__ void inplace_fft(C* buf, const AxisPlan& ap, int nlines, int es, int ls, const FastDiv& nld,
                            const C* __restrict__ tw) {
    for (int k = 0; k < ap.nst; ++k) {
        const int st = DIF ? k : ap.nst - 1 - k;
        switch (ap.rad[st]) {
            case 8: inplace_stage<C, 8, DIF, NT>(buf, ap.n, nlines, es, ls, ap.span[st], ap.sub[st], nld, tw); break;
            case 4: inplace_stage<C, 4, DIF, NT>(buf, ap.n, nlines, es, ls, ap.span[st], ap.sub[st], nld, tw); break;
            case 2: inplace_stage<C, 2, DIF, NT>(buf, ap.n, nlines, es, ls, ap.span[st], ap.sub[st], nld, tw); break;
            case 3: inplace_stage<C, 3, DIF, NT>(buf, ap.n, nlines, es, ls, ap.span[st], ap.sub[st], nld, tw); break;
            default: inplace_stage<C, 5, DIF, NT>(buf, ap.n, nlines, es, ls, ap.span[st], ap.sub[st], nld, tw); break;
        }
    }
}

// Padded position of element i of a warp-FFT line in shared memory: one pad slot
// every 16 elements, so that the stride-R stores of the early Stockham passes fall
// into distinct banks (2 wavefronts per warp access instead of up to 16).
__device__ __forceinline__ int wpad(int i) { return i + (i >> 4); }
// The same for a compile-time multiple of 16: wpad(a + k) = wpad(a) + cpad(k) for a >= 0.
__host__ __device__ constexpr int cpad(int k) { return k + k / 16; }

// Radix of the warp Stockham pass that starts at sub-transform length NS: the largest
// radix (8, 4, 2) that divides N / NS and still gives every lane a butterfly.
template <int N, int NS>
__host__ __device__ constexpr int warp_radix() {
    return ((N / NS) % 8 == 0 && N / 8 >= 32) ? 8 : ((N / NS) % 4 == 0 && N / 4 >= 32) ? 4 : 2;
}

// Twiddle table of the warp FFT, per pass: the pass at NS > 1 owns (R - 1) NS
// entries, entry (r - 1) NS + j = W_N^{j r N / (NS R)} for j < NS, 1 <= r < R, so
// that a lane reads its R - 1 twiddles at fixed offsets from one address and
// consecutive lanes read consecutive entries. At most N entries for N = 128 ... 1024.
template <int N, int NS = 1>
__host__ __device__ constexpr int warp_tw_count() {
    if constexpr (NS >= N) {
        return 0;
    } else {
        constexpr int R = warp_radix<N, NS>();
        return (NS > 1 ? (R - 1) * NS : 0) + warp_tw_count<N, NS * R>();
    }
}

// Fills the per-pass table from tw[t] = W_N^t (t < N); called by the whole block.
template <typename C, int N, int NS = 1, int OFF = 0>
__device__ __forceinline__ void warp_tw_fill(C* twl, const C* __restrict__ tw) {
    if constexpr (NS < N) {
        constexpr int R = warp_radix<N, NS>();
        if constexpr (NS > 1) {
            constexpr int TWS = N / (NS * R);
            for (int q = threadIdx.x; q < (R - 1) * NS; q += blockDim.x) {
                const int r = 1 + q / NS, j = q % NS;
                twl[OFF + q] = tw[j * r * TWS];
            }
            warp_tw_fill<C, N, NS * R, OFF + (R - 1) * NS>(twl, tw);
        } else {
            warp_tw_fill<C, N, NS * R, OFF>(twl, tw);
        }
    }
}

// Warp-local Stockham FFT of one line of compile-time length N (a power of two,
// 128 <= N <= 1024) held in shared memory at x[wpad(m)]: the 32 lanes of one warp
// run the radix-8 / 4 / 2 passes (Ns = 1, R, R R', ...) alone, with __syncwarp
// between the load and store halves of each pass, so no block barrier is needed.
// Each lane keeps its butterflies' inputs in registers for the store half, which
// makes the autosort pass safe in place. Forward kernel exp(-2 pi i / N);
// natural-order input and output; twl is the per-pass table of warp_tw_fill.
//
// Addressing: butterfly j = lane + 32 b of a pass reads elements j + r N/R and
// writes od + r NS, od = (j - j mod NS) R + j mod NS. For the lengths used every
// such padded position is a per-lane base plus a compile-time offset: the loads
// from wpad(lane); the stores from wpad(lane R) (NS = 1), wpad(od of b = 0)
// (1 < NS < 32, where j mod NS = lane mod NS and NS R >= 16 keeps the pad of
// od + r NS separable) or wpad(lane) (NS >= 32). So every shared-memory access
// of a pass is one instruction with an immediate offset.
//
// Where the first pass reads the line and the last pass writes it (IN, OUT):
// kIoSmem: x itself. kIoGlobal: gin / gout in global memory (natural order,
// unpadded; consecutive lanes take consecutive elements; gout conjugated if
// CONJ). kIoReg: the register array u of the lane, u[k] = element lane + 32 k
// (the last pass has NS >= 32, so its outputs are exactly those elements, and
// the first pass reads exactly those elements). kIoGlobal and kIoReg skip a
// shared-memory round trip of the whole line.
constexpr int kIoSmem = 0, kIoGlobal = 1, kIoReg = 2;

// True for the layout the pass at sub-length NS reads when the passes before it were NS = 1 and 8,
// both radix 8 (N >= 256): the NS = 8 pass stores that layout unpadded with an XOR swizzle (element p
// at p ^ 8 when bit 6 of p is set) instead of at wpad(p).
template <int N, int NS>
__host__ __device__ constexpr bool warp_swizzled() {
    return NS == 64 && N >= 256 && warp_radix<N, 1>() == 8 && warp_radix<N, 8>() == 8;
}

template <typename C, int N, int NS, int OFF, int IN = kIoSmem, int OUT = kIoSmem, bool CONJ = false>
__device__ __forceinline__ void warp_stockham(C* x, const C* __restrict__ twl, int lane, C (&u)[N / 32],
                                              const C* gin = nullptr, C* gout = nullptr) {
    if constexpr (NS < N) {
        constexpr int R = warp_radix<N, NS>();
        constexpr int NB = N / R;                 // butterflies of the pass
        constexpr int PER = NB / 32;              // butterflies per lane
        constexpr int SRC = NS == 1 ? IN : kIoSmem;
        constexpr int DST = NS * R == N ? OUT : kIoSmem;
        static_assert(NB % 32 == 0, "every lane takes whole butterflies");
        static_assert(NS == 1 || NS >= 16 || NS * R >= 16, "separable store offsets");
        static_assert(DST == kIoSmem || NS >= 32, "the last pass writes lane + const");
        C v[PER][R];
        if constexpr (SRC == kIoGlobal) {
            const C* gl = gin + lane;
#pragma unroll
            for (int b = 0; b < PER; ++b) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = gl[32 * b + r * NB];
            }
            __syncwarp();   // the warp's previous line has been read out of x
        } else if constexpr (SRC == kIoReg) {
#pragma unroll
            for (int b = 0; b < PER; ++b) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = u[(32 * b + r * NB) / 32];
            }
        } else if constexpr (warp_swizzled<N, NS>()) {
            // the line as the NS = 8 pass left it: unpadded, position q + lane at (q + lane) ^ 8 when
            // bit 6 of q is set (q = 32 b + r NB is a multiple of 32, so that bit is q's own)
            const C* xl0 = x + lane;
            const C* xl1 = x + (lane ^ 8);
#pragma unroll
            for (int b = 0; b < PER; ++b) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int q = 32 * b + r * NB;
                    v[b][r] = ((q >> 6) & 1) ? xl1[q] : xl0[q];
                }
            }
            __syncwarp();
        } else {
            const C* xl = x + wpad(lane);
#pragma unroll
            for (int b = 0; b < PER; ++b) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = xl[cpad(32 * b + r * NB)];
            }
            __syncwarp();
        }
        if constexpr (NS > 1) {
            // twiddles W_N^{jm r N/(NS R)} with jm = j mod NS
            const C* tl = twl + OFF + (NS <= 32 ? (lane & (NS - 1)) : lane);
#pragma unroll
            for (int b = 0; b < PER; ++b) {
                const int jb = (NS <= 32) ? 0 : ((32 * b) & (NS - 1));
#pragma unroll
                for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], tl[jb + (r - 1) * NS]);
            }
        }
#pragma unroll
        for (int b = 0; b < PER; ++b) Dft<C, R>::run(v[b]);
        if constexpr (DST == kIoGlobal || DST == kIoReg) {
            C* gl = gout + lane;
#pragma unroll
            for (int b = 0; b < PER; ++b) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int kb = ((32 * b) & ~(NS - 1)) * R + ((32 * b) & (NS - 1));
                    if constexpr (DST == kIoReg)
                        u[(kb + r * NS) / 32] = v[b][r];
                    else
                        gl[kb + r * NS] = CONJ ? cmake<C>(v[b][r].x, -v[b][r].y) : v[b][r];
                }
            }
        } else {
            if constexpr (NS == 1) {
                C* xs = x + wpad(lane * R);
#pragma unroll
                for (int b = 0; b < PER; ++b) {
#pragma unroll
                    for (int r = 0; r < R; ++r) xs[cpad(32 * b * R) + r] = v[b][r];
                }
            } else if constexpr (warp_swizzled<N, NS * R>()) {
                // NS = 8, R = 8, read next by the NS = 64 pass: unpadded, element p at p ^ 8 when bit 6 of p
                // is set. Here p = 64 (lane >> 3) + jm + 256 b + 8 r, so bit 6 is bit 3 of the lane: the
                // lanes with it set write r ^ 1 in place of r. The 8-lane groups of a half-warp then use
                // disjoint halves of the banks (the padded layout conflicts 2-way here).
                const int jm = lane & 7, sw = (lane >> 3) & 1;
                C* xe = x + (lane >> 3) * 64 + jm + 8 * sw;   // even r
                C* xo = x + (lane >> 3) * 64 + jm - 8 * sw;   // odd r
#pragma unroll
                for (int b = 0; b < PER; ++b) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (r & 1)
                            xo[256 * b + 8 * r] = v[b][r];
                        else
                            xe[256 * b + 8 * r] = v[b][r];
                    }
                }
            } else if constexpr (NS < 32) {
                const int jm = lane & (NS - 1);
                C* xs = x + wpad((lane - jm) * R + jm);
#pragma unroll
                for (int b = 0; b < PER; ++b) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if constexpr (NS < 16)
                            xs[cpad(32 * b * R) + r * NS + (r * NS) / 16] = v[b][r];
                        else
                            xs[cpad(32 * b * R) + cpad(r * NS)] = v[b][r];
                    }
                }
            } else {
                C* xs = x + wpad(lane);
#pragma unroll
                for (int b = 0; b < PER; ++b) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int kb = ((32 * b) & ~(NS - 1)) * R + ((32 * b) & (NS - 1));
                        xs[cpad(kb + r * NS)] = v[b][r];
                    }
                }
            }
            __syncwarp();
        }
        warp_stockham<C, N, NS * R, (NS > 1 ? OFF + (R - 1) * NS : OFF), IN, OUT, CONJ>(x, twl, lane, u, gin, gout);
    }
}

// ---------------------------------------------------------------------------
// Register-resident 512-point DFT of one warp's line (512 = 32 lanes x 16 registers), with one
// exchange through shared memory per transform instead of the two of the radix-8 Stockham passes.
// With x[m], m = l + 32 k, held as u[k] by lane l:
//   1. a 16-point DFT over k in each lane, then the twiddle W_512^{l k'};
//   2. an exchange: lane L receives, for k' = L >> 1, the values of the lanes l = (L & 1) + 2 j;
//   3. a 16-point DFT over j, then the radix-2 step between lanes L and L ^ 1 (twiddle W_32^q),
// which leaves X[f] with f = (L >> 1) + 16 q + 256 (L & 1) in register q of lane L. The DFT matrix
// is symmetric, so the transposed steps in reverse order take a line held in that order back to
// natural order (again a forward DFT). Exchange rows of 34 elements make both sides of the
// exchange conflict-free.
// ---------------------------------------------------------------------------

// cos(2 pi m / 32) and sin(2 pi m / 32) for 0 <= m < 32, from the first quadrant by symmetry
__host__ __device__ constexpr double cos32_q(int r) {
    return r == 0 ? 1.0
         : r == 1 ? 0.98078528040323044913
         : r == 2 ? 0.92387953251128675613
         : r == 3 ? 0.83146961230254523708
         : r == 4 ? 0.70710678118654752440
         : r == 5 ? 0.55557023301960222474
         : r == 6 ? 0.38268343236508977173
         : r == 7 ? 0.19509032201612826785
                  : 0.0;
}
__host__ __device__ constexpr double cos32(int m) {
    return m <= 8 ? cos32_q(m) : m <= 16 ? -cos32_q(16 - m) : m <= 24 ? -cos32_q(m - 16) : cos32_q(32 - m);
}
__host__ __device__ constexpr double sin32(int m) { return cos32((m + 24) % 32); }

// W_32^m = exp(-2 pi i m / 32) (m a compile-time value after unrolling)
template <typename C>
__device__ __forceinline__ C w32c(int m) {
    using R = decltype(C::x);
    return cmake<C>(R(cos32(m)), R(-sin32(m)));
}

// 16-point forward DFT in registers, natural order in and out: 4-point DFTs of the stride-4
// subsequences, twiddles W_16^{a b'}, 4-point DFTs across them.
template <typename C>
__device__ __forceinline__ void dft16(C (&v)[16]) {
    C t[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        C q[4] = {v[a], v[a + 4], v[a + 8], v[a + 12]};
        Dft<C, 4>::run(q);
#pragma unroll
        for (int bp = 0; bp < 4; ++bp) t[a][bp] = (a * bp == 0) ? q[bp] : cmul(q[bp], w32c<C>(2 * a * bp));
    }
#pragma unroll
    for (int bp = 0; bp < 4; ++bp) {
        C q[4] = {t[0][bp], t[1][bp], t[2][bp], t[3][bp]};
        Dft<C, 4>::run(q);
#pragma unroll
        for (int ap = 0; ap < 4; ++ap) v[bp + 4 * ap] = q[ap];
    }
}

template <typename C>
__device__ __forceinline__ C shfl_xor_cx(C a, int m) {
    return cmake<C>(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
}

constexpr int kReg512Row = 34;   // exchange row stride (16 rows: 544 elements of scratch per warp)

// Natural order in (u[k] = x[lane + 32 k]), permuted order out (u[q] = X[(lane >> 1) + 16 q +
// 256 (lane & 1)]). tw[k'] = W_512^{lane k'} (tw[0] unused). s: the warp's scratch; the caller has
// finished its own reads of s before the call.
template <typename C>
__device__ __forceinline__ void fft512_to_perm(C (&u)[16], C* s, const C (&tw)[16], int lane) {
    dft16(u);
#pragma unroll
    for (int kp = 1; kp < 16; ++kp) u[kp] = cmul(u[kp], tw[kp]);
    __syncwarp();
#pragma unroll
    for (int kp = 0; kp < 16; ++kp) s[kp * kReg512Row + lane] = u[kp];
    __syncwarp();
    const C* sr = s + (lane >> 1) * kReg512Row + (lane & 1);
#pragma unroll
    for (int j = 0; j < 16; ++j) u[j] = sr[2 * j];
    dft16(u);
    const bool odd = (lane & 1) != 0;
    using R = decltype(C::x);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        // odd lanes hold O[q]: scale by W_32^q; then E + W O (even lane) and E - W O (odd lane)
        const C w = odd ? w32c<C>(q) : cmake<C>(R(1), R(0));
        const C mine = cmul(u[q], w);
        const C other = shfl_xor_cx(mine, 1);
        u[q] = odd ? csub(other, mine) : cadd(mine, other);
    }
}

// Permuted order in (as fft512_to_perm leaves it), natural order out: the forward DFT of the
// line, u[k] = Y[lane + 32 k]. The caller reads s only after a __syncwarp.
template <typename C>
__device__ __forceinline__ void fft512_from_perm(C (&u)[16], C* s, const C (&tw)[16], int lane) {
    const bool odd = (lane & 1) != 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        // even lane (a = X[k' + 16 q]): a + b; odd lane (b = X[k' + 16 (q + 16)]): W_32^q (a - b)
        const C other = shfl_xor_cx(u[q], 1);
        u[q] = odd ? cmul(csub(other, u[q]), w32c<C>(q)) : cadd(u[q], other);
    }
    dft16(u);
    __syncwarp();
    C* sw = s + (lane >> 1) * kReg512Row + (lane & 1);
#pragma unroll
    for (int j = 0; j < 16; ++j) sw[2 * j] = u[j];
    __syncwarp();
#pragma unroll
    for (int kp = 0; kp < 16; ++kp) u[kp] = s[kp * kReg512Row + lane];
#pragma unroll
    for (int kp = 1; kp < 16; ++kp) u[kp] = cmul(u[kp], tw[kp]);
    dft16(u);
}

template <int N>
__host__ __device__ constexpr bool warp_fft_ok() {
    return N >= 128 && N <= 1024 && (N & (N - 1)) == 0 && warp_tw_count<N>() <= N;
}

// Shared-memory line x[wpad(m)] in and out.
template <typename C, int N>
__device__ __forceinline__ void warp_fft(C* x, const C* __restrict__ twl, int lane) {
    static_assert(warp_fft_ok<N>(), "warp FFT length");
    C u[N / 32];
    warp_stockham<C, N, 1, 0>(x, twl, lane, u);
}

// Global line gin to global line gout (conjugated if CONJ; gin == gout allowed:
// the whole line is in registers or x in between), x as the warp's scratch line.
template <typename C, int N, bool CONJ>
__device__ __forceinline__ void warp_fft_global(const C* gin, C* gout, C* x, const C* __restrict__ twl, int lane) {
    static_assert(warp_fft_ok<N>(), "warp FFT length");
    C u[N / 32];
    warp_stockham<C, N, 1, 0, kIoGlobal, kIoGlobal, CONJ>(x, twl, lane, u, gin, gout);
}

// Shared-memory line in, result in registers: u[k] = X[lane + 32 k].
template <typename C, int N>
__device__ __forceinline__ void warp_fft_to_regs(C* x, const C* __restrict__ twl, int lane, C (&u)[N / 32]) {
    static_assert(warp_fft_ok<N>(), "warp FFT length");
    warp_stockham<C, N, 1, 0, kIoSmem, kIoReg>(x, twl, lane, u);
}

// Registers in and out (u[k] = element lane + 32 k), x as scratch between passes.
template <typename C, int N>
__device__ __forceinline__ void warp_fft_regs(C* x, const C* __restrict__ twl, int lane, C (&u)[N / 32]) {
    static_assert(warp_fft_ok<N>(), "warp FFT length");
    warp_stockham<C, N, 1, 0, kIoReg, kIoReg>(x, twl, lane, u);
}

// Registers in (u[k] = x[lane + 32 k]), result in the shared-memory line x.
template <typename C, int N>
__device__ __forceinline__ void warp_fft_from_regs(C* x, const C* __restrict__ twl, int lane, C (&u)[N / 32]) {
    static_assert(warp_fft_ok<N>(), "warp FFT length");
    warp_stockham<C, N, 1, 0, kIoReg, kIoSmem>(x, twl, lane, u);
}

}  // namespace ccmf
