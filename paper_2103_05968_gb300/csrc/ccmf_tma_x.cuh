// x line pass of the Poisson solve (forward FFT along x, the gain 1 / (N lambda(k)) of
// (div^- grad^+)^+ in Eq. 28, inverse FFT along x) for n1 = 512 in FP32, with the tiles
// moved between the half spectrum and shared memory by the tensor memory accelerator.
//
// A tile is 8 adjacent x lines (k_y .. k_y + 7) of one k_z plane: in global memory a box of
// 8 complex elements (64 bytes) by 512 rows with row stride n2. One elected thread loads it
// with cp.async.bulk.tensor (two boxes of 256 rows, the box height limit) into a 64-byte
// swizzled buffer, completion counted in bytes on an mbarrier; the next tile's load runs
// while the current one is transformed. Each warp transforms one line through registers
// (the 512-point register transforms of the warp engine), writes it back into the tile
// buffer, and the elected thread stores the tile with cp.async.bulk.tensor. The transpose
// between the contiguous k_y axis in memory and the line-per-warp view is the swizzled
// shared-memory addressing: element (m, c) of the tile sits in row m (64 bytes) at 16-byte
// chunk (c / 2) XOR ((m / 2) mod 4), half (c mod 2).
#pragma once

#include <cuda.h>

#include "ccmf_kernels.cuh"

namespace ccmf {

constexpr int kTmaXN = 512;                                  // x line length of this pass
constexpr int kTmaXLines = kThreads / 32;                    // lines per tile, one per warp
constexpr int kTmaXBoxRows = 256;                            // rows per box (the box size limit)
constexpr unsigned kTmaXTileBytes = kTmaXN * kTmaXLines * 8; // 32 KB per tile
constexpr unsigned kTmaXScratch = 16 * kReg512Row * 8;       // exchange rows of one warp's transforms
// dynamic shared memory: alignment slack (the swizzle pattern follows the address bits, so the
// tiles start on a 1024-byte boundary), two tiles, the warps' exchange scratch, two mbarriers
constexpr size_t kTmaXSmem = 1024 + 2 * (size_t)kTmaXTileBytes + (size_t)kTmaXLines * kTmaXScratch + 16;

// Byte offset of element (m, c) in a tile: row m of 64 bytes, 16-byte chunk c / 2 XOR bits 1..2 of m.
__host__ __device__ inline unsigned tma_x_offset(unsigned m, unsigned c) {
    return m * 64u + (((c >> 1) ^ ((m >> 1) & 3u)) << 4) + ((c & 1u) << 3);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit_group() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the committed bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// tmap: the half spectrum as a 3-D tensor of 8-byte elements {n2, n1, n3h * solves}, box {8, 256, 1},
// 64-byte swizzle. Needs n1 = 512 and n2 % 8 == 0 (a tile never straddles two planes).
template <int N>
__global__ void __launch_bounds__(kThreads, 2)
    k_fft_wx_tma(const __grid_constant__ CUtensorMap tmap, Geom g, Ptrs<float> p, const float2* __restrict__ tw,
                 const float* __restrict__ xsym, const float* __restrict__ ysym, const float* __restrict__ sym3,
                 float inv_n, unsigned spin_limit) {
    static_assert(N == kTmaXN, "the register transforms are 512-point");
    using C = float2;
    constexpr int L = kTmaXLines;
    const int s = blockIdx.y + p.s0;
    if (!p.run_all && !p.sc[s].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* tile0 = base;
    unsigned char* tile1 = base + kTmaXTileBytes;
    C* scratch = reinterpret_cast<C*>(base + 2 * kTmaXTileBytes);
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(base + 2 * kTmaXTileBytes + (size_t)L * kTmaXScratch);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C* xs = scratch + (size_t)warp * (kTmaXScratch / sizeof(C));
    // per-lane twiddles W_512^{lane k'} and the x symbol in the permuted order of fft512_to_perm
    C tw512[16];
    float xs512[16];
#pragma unroll
    for (int kp = 0; kp < 16; ++kp) tw512[kp] = tw[(lane * kp) & (N - 1)];
#pragma unroll
    for (int q = 0; q < 16; ++q) xs512[q] = xsym[(lane >> 1) + 16 * q + 256 * (lane & 1)];
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long ntiles = (long long)g.n3h * g.n2 / L;
    const unsigned limit = spin_limit ? spin_limit - 1 : kSpinLimit;
    // first line l = t L of tile t: plane k_z = l / n2, first k_y = l mod n2 (a multiple of 8)
    auto tile_coords = [&](long long t, int& ky, int& kz) {
        const long long l = t * L;
        kz = (int)fdiv((unsigned)l, g.div_n2);
        ky = (int)(l - (long long)kz * g.n2);
    };
    auto issue = [&](long long t, unsigned char* dst, unsigned long long* bar) {
        int ky, kz;
        tile_coords(t, ky, kz);
        const int z = s * g.n3h + kz;
        mbar_expect_tx(bar, kTmaXTileBytes);
        tma_load_3d(dst, &tmap, ky, 0, z, bar);
        tma_load_3d(dst + kTmaXTileBytes / 2, &tmap, ky, kTmaXBoxRows, z, bar);
    };
    const long long t0 = blockIdx.x, step = gridDim.x;
    if (threadIdx.x == 0 && t0 < ntiles) issue(t0, tile0, &bars[0]);
    unsigned phase0 = 0, phase1 = 0;
    int it = 0;
    bool failed = false;
    // row lane, line warp; rows lane + 32 k lie 2048 k bytes further (bits 1..2 of the row unchanged)
    const unsigned off = tma_x_offset((unsigned)lane, (unsigned)warp);
    for (long long t = t0; t < ntiles; t += step, ++it) {
        const int st = it & 1;
        unsigned char* tb = st ? tile1 : tile0;
        if (threadIdx.x == 0 && t + step < ntiles) {
            bulk_wait_read_all();   // the other buffer's last store has read it
            issue(t + step, st ? tile0 : tile1, &bars[st ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bars[st], st ? phase1 : phase0, limit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (st)
            phase1 ^= 1u;
        else
            phase0 ^= 1u;
        int ky, kz;
        tile_coords(t, ky, kz);
        const float lam23 = ysym[ky + warp] + sym3[kz];
        C u[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) u[k] = *reinterpret_cast<const C*>(tb + off + 2048u * k);
        fft512_to_perm(u, xs, tw512, lane);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float lam = xs512[q] + lam23;
            const float gk = (lam > 0.0f) ? poisson_gain(inv_n, lam) : 0.0f;
            u[q] = make_float2(u[q].x * gk, -u[q].y * gk);   // conj: the inverse runs as conj(FFT(conj(.)))
        }
        fft512_from_perm(u, xs, tw512, lane);
#pragma unroll
        for (int k = 0; k < 16; ++k) *reinterpret_cast<C*>(tb + off + 2048u * k) = u[k];
        fence_proxy_async_smem();   // the generic-proxy writes before the bulk store reads them
        __syncthreads();
        if (threadIdx.x == 0) {
            const int z = s * g.n3h + kz;
            tma_store_3d(&tmap, ky, 0, z, tb);
            tma_store_3d(&tmap, ky, kTmaXBoxRows, z, tb + kTmaXTileBytes / 2);
            bulk_commit_group();
        }
    }
    if (threadIdx.x == 0) {
        if (failed) {
            // loads still in flight land in this block's shared memory: wait for them (bounded)
            const long long t = t0 + (long long)it * step;
            const int st = it & 1;
            if (t < ntiles) (void)mbar_wait_bounded(&bars[st], st ? phase1 : phase0);
            if (t + step < ntiles) (void)mbar_wait_bounded(&bars[st ^ 1], st ? phase0 : phase1);
            atomicExch(&p.sc[s].status, 6);   // CCMF_ERR_TIMEOUT
        }
        bulk_wait_all();   // the stores have completed before the block's shared memory is released
    }
}

// Marks the solves [s0, s0 + n) failed (CCMF_ERR_CUDA) when their x pass could not be launched.
template <int Unused>
__global__ void k_launch_failed(SolveScalars* sc, int s0, int n) {
    for (int s = threadIdx.x; s < n; s += blockDim.x) atomicExch(&sc[s0 + s].status, 4);
}

// cuTensorMapEncodeTiled, taken from the driver through the runtime (the library links the
// runtime only); null when the driver does not provide it.
typedef CUresult (*TensorMapEncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                           const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                           CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                           CUtensorMapFloatOOBfill);
inline TensorMapEncodeTiledFn tensor_map_encoder() {
    static const TensorMapEncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<TensorMapEncodeTiledFn>(f);
    }();
    return fn;
}

// The tensor map of the x pass: the half spectrum at `spec` as {n2, n1, planes} elements of 8 bytes
// (one FP32 complex), box {8, 256, 1}, 64-byte swizzle. False if the encoder is missing or
// rejects the shape (spec must be 16-byte aligned, n2 a multiple of 2).
inline bool encode_x_tensor_map(CUtensorMap* map, const void* spec, int n1, int n2, long long planes) {
    const TensorMapEncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)n2, (cuuint64_t)n1, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)n2 * 8u, (cuuint64_t)n1 * (cuuint64_t)n2 * 8u};
    const cuuint32_t box[3] = {(cuuint32_t)kTmaXLines, (cuuint32_t)kTmaXBoxRows, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(spec), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Whether a plan of this shape can run the TMA-staged x pass.
inline bool x_tma_shape_ok(int n1, int n2, int n3h, int batch) {
    if (n1 != kTmaXN || n2 % kTmaXLines != 0) return false;
    alignas(64) CUtensorMap map;
    return encode_x_tensor_map(&map, reinterpret_cast<const void*>(256), n1, n2, (long long)n3h * batch);
}

}  // namespace ccmf
