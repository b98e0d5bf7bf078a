// Shared types of the CCMF solver kernels and the host driver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ccmf_fft.cuh"

namespace ccmf {

// Global sums reduced by the update pass (all in double once past the warp level).
enum SumIndex {
    kSumRes = 0,      // sum |e^k - xi^{k+1/2}|^2            (Eq. 31, left side)
    kSumV = 1,        // 1..6: sum of v^k components           (Eq. 31, right side; dual objective)
    kSumPrimal = 7,   // sum gamma |xi^{k+1/2}|                (Eq. 21)
    kSumDvDe = 8,     // sum <v^{k+1}-v^k, e^{k+1}-e^k>        (BB scaling)
    kSumDeDe = 9,     // sum |e^{k+1}-e^k|^2
    kSumDvDv = 10,    // sum |v^{k+1}-v^k|^2                   (BB safeguard)
    kSumVV = 11,      // sum |v^{k+1}|^2                       (LTD scaling)
    kSumEE = 12,      // sum |e^{k+1}|^2
    kNSum = 13
};

constexpr int kHistFields = 6;
constexpr int kHistCap = 4096;   // history entries reserved per solve
constexpr int kThreads = 256;

// The vector update pass works in chunks of kVecChunkGroups groups of 16 bytes per
// thread (16 K voxels in FP32), taken in order from a ticket counter, with one
// partial-sum slot per chunk.
constexpr int kVecChunkGroups = 16;
__host__ __device__ inline long long vec_update_chunks(long long n_voxels, int voxels_per_group) {
    const long long per = (long long)kThreads * kVecChunkGroups;
    return (n_voxels / voxels_per_group + per - 1) / per;
}

// One per solve, in the workspace (256-byte slot).
struct SolveScalars {
    double rho;          // current penalty rho^k
    double xi[3];        // unit crack normal
    double gmin, gmax, gsum;
    double residual, mean_v, primal, dual;
    double sums[kNSum];
    int active;          // 1 while the solve iterates
    int status;          // CCMF_OK or an error code
    int iters;           // updates performed so far (k)
    int converged;
    int call_start;      // iters at the start of the current solve call
    unsigned int counter;  // last-block ticket of the reductions
    int bad;             // number of invalid gamma values seen at init
    unsigned int chunk;  // next work ticket of the vector update pass (dynamic schedule)
    int ab_iter;         // update count the stored divergences a, b belong to (-1: not current)
};
static_assert(sizeof(SolveScalars) <= 256, "scalar slot");

struct LoopConfig {
    double tol, delta, rho0, bb_corr_min, rho_step_max;
    int max_iter, fixed_iters, rho_rule, hist_len, resume;
    const double* rho_sched;  // replayed penalties rho^k = rho_sched[s * sched_len + k] (null: adaptive rule)
    int sched_len;
    unsigned spin_limit;      // 0: the default budget of a bounded device wait; n > 0: n - 1 polls, only to
                              // test the timeout path (CCMF_DEBUG_SPIN_LIMIT; each poll may itself block
                              // for a while, so 0 polls is the budget that reliably gives up)
};

struct Geom {
    int n1, n2, n3, n3h, batch;
    long long N;    // voxels per solve
    long long Nh;   // half-spectrum entries per solve (n1 n2 n3h)
    FastDiv div_n3, div_n2, div_n3h, div_n1;
};

template <typename T>
struct Ptrs {
    SolveScalars* sc;
    int* n_active;
    double* partial;      // [batch][grid_update][kNSum]
    double* hist;         // [batch][hist_len][kHistFields]
    T* e;                 // [2][batch][6][N]: two copies, the current one is (iters & 1)
    T* v;                 // [2][batch][6][N]
    long long sstride;    // elements between the two copies (batch * 6 * N)
    cx<T>* spec;          // [batch][Nh]
    T* phi;               // [batch][N]
    const T* gamma;       // solve s at gamma + s * gstride ...
    long long gstride;
    const T* const* gptrs;  // ... or, when not null, at gptrs[s] (device array of pointers)
    T* cut;               // [batch][6][N] (final pass, may be null)
    T* flow;              // [batch][3][N] (final pass, may be null)
    int run_all;          // 1: passes run for every solve (final evaluation), 0: active solves only
    int s0;               // first solve of this launch (blockIdx.y counts from it)
    T* zout;              // when not null the (scalar) update pass also writes z = v + rho xi, [batch][6][N]
    T* ab;                // stored divergences a = div^- A* e, b = div^- A* v of the state, [batch][2][N]
};

// Shape of the stored-divergence update (update variants 8, 9, 10): a block owns tj
// consecutive y rows (plus one recomputed row on each side) of whole z rows and sweeps
// x over a segment of xs slabs (plus one recomputed slab on each side).
struct AbShape {
    int tj;      // interior y rows per block (warps per block - 2)
    int nq;      // y tiles: ceil(n2 / tj)
    int xs;      // interior x slabs per block
    int nr;      // x segments: ceil(n1 / xs)
    int npass;   // z passes of 32 VW voxels per row (n3 / (32 VW))
};

struct LaunchShape {
    int pairs_per_block;      // divergence + forward z pass: line pairs per block
    int pairs_inv;            // inverse z pass: line pairs per block
    size_t smem_zi;           // its dynamic shared memory
    int lpb_y, lpb_x;         // strided passes: lines per block
    int grid_update;          // blocks per solve of the voxel passes
    int vec_resident;         // resident blocks of the vector update pass on the whole GPU
    int vec_resident_half;    // the same for update variants 11, 12 (fewer voxels per thread)
    size_t smem_z, smem_y, smem_x;
    int tma_rows;             // TMA-staged update: z rows per tile (0 = path not available)
    int grid_tma;             // blocks per solve of the TMA-staged update
    size_t smem_tma;          // its dynamic shared memory (two stages + barriers)
    int grid_partials;        // partial-sum slots per solve (max of the update grids)
    int upd_variant;          // update pass: 0 register vectors, 1 TMA (2 stages, any tile),
                              // 2..7 pipelined TMA (see kUpdatePipe)
    int grid_pipe;            // blocks per solve of the pipelined update
    size_t smem_pipe;         // its dynamic shared memory
    int plane_fused;          // 1: y / x / solve / x / y in one plane launch per iteration
    size_t smem_plane;        // its dynamic shared memory (per block)
    int plane_cluster;        // blocks sharing one plane: 1 = k_fft_plane, 2..16 = k_fft_plane_cluster
    int grid_y, grid_x;       // persistent blocks per solve of the y / x line passes (0: one tile per block)
    int wl_y, wl_x;           // > 0: the y / x line passes run one warp per line (k_fft_wlines); the line length
    int x_tma;                // 1: the x pass is k_fft_wx_tma (tiles moved by TMA; FP32, n1 = 512)
    size_t smem_wy, smem_wx;  // their dynamic shared memory
    int wz, wzd;              // > 0: the inverse / divergence z pass runs one warp per line pair; N3
    size_t smem_wzd, smem_wzi;
    FastDiv div_r1, div_r2;   // rows (n1 / C) and columns (n2 / C) of one cluster block
    AbShape ab;               // update variants 8, 9, 10: the stored-divergence update
    size_t smem_ab;           // its dynamic shared memory
};

// Pipelined update variants: {threads per block, stages}.
constexpr int kUpdatePipe[8][2] = {{0, 0}, {0, 0}, {256, 2}, {128, 3}, {128, 4}, {256, 3}, {128, 2}, {64, 3}};

// Stored-divergence update variants 8, 9, 10: warps per block, voxels per lane and z pass,
// blocks per SM the register budget is sized for.
template <typename T, int VAR> struct AbVariant;
template <> struct AbVariant<float, 8> { static constexpr int NW = 8, VW = 4, MINB = 1; };
template <> struct AbVariant<float, 9> { static constexpr int NW = 16, VW = 2, MINB = 1; };
template <> struct AbVariant<float, 10> { static constexpr int NW = 8, VW = 2, MINB = 2; };
template <> struct AbVariant<double, 8> { static constexpr int NW = 8, VW = 2, MINB = 1; };
template <> struct AbVariant<double, 9> { static constexpr int NW = 16, VW = 1, MINB = 1; };
template <> struct AbVariant<double, 10> { static constexpr int NW = 8, VW = 1, MINB = 2; };
// Warp-independent stored-divergence update variants 13, 14, 15: voxels per lane and z pass, blocks
// (of 4 warps) per SM the register budget is sized for, y rows per warp. Fewer rows per warp recompute
// more ring rows but stream fewer bytes per slab step across the resident warps, which decides
// whether the x-neighbour rows of one step are still in L2 at the next.
template <typename T, int VAR> struct AbwVariant;
template <> struct AbwVariant<float, 13> { static constexpr int VW = 4, MINB = 2, TJ = 8; };
template <> struct AbwVariant<float, 14> { static constexpr int VW = 4, MINB = 2, TJ = 4; };
template <> struct AbwVariant<float, 15> { static constexpr int VW = 4, MINB = 2, TJ = 6; };
template <> struct AbwVariant<double, 13> { static constexpr int VW = 2, MINB = 2, TJ = 8; };
template <> struct AbwVariant<double, 14> { static constexpr int VW = 2, MINB = 2, TJ = 4; };
template <> struct AbwVariant<double, 15> { static constexpr int VW = 2, MINB = 2, TJ = 6; };
constexpr int kNumUpdateVariants = 16;
__host__ __device__ constexpr bool is_abw_variant(int v) { return v >= 13 && v <= 15; }
// update variants that write the stored divergences: 8 .. 10 (block-cooperative), 13 .. 15 (warp-independent)
__host__ __device__ constexpr bool is_ab_variant(int v) { return (v >= 8 && v <= 10) || is_abw_variant(v); }

}  // namespace ccmf
