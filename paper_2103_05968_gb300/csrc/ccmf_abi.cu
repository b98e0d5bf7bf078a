// C ABI of the CCMF FFT-ADMM solver: plans, workspace layout, the device-side
// iteration loop (captured CUDA graphs) and state / history / timing access.
// See include/ccmf.h for the contract of every entry point.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ccmf.h"
#include "ccmf_launch.cuh"

using namespace ccmf;

namespace ccmf {
template <typename T> cudaError_t configure_kernels(const LaunchShape&);
template <typename T> int pipe_blocks_per_sm(int, size_t);
template <typename T> int plane_cluster_capacity(int, size_t);

// Voxels per lane and rows per warp of the warp-independent stored-divergence update variant v.
template <typename T>
void abw_params(int v, int& vw, int& tj) {
    if (v == 13) {
        vw = AbwVariant<T, 13>::VW;
        tj = AbwVariant<T, 13>::TJ;
    } else if (v == 14) {
        vw = AbwVariant<T, 14>::VW;
        tj = AbwVariant<T, 14>::TJ;
    } else {
        vw = AbwVariant<T, 15>::VW;
        tj = AbwVariant<T, 15>::TJ;
    }
}
template <typename T> int lines_blocks_per_sm(int, int, size_t);
template <typename T> int wlines_blocks_per_sm(int, int, size_t);
template <typename T> int update_vec_blocks_per_sm();
template <typename T> int update_vec_half_blocks_per_sm(int);
template <typename T> int ab_blocks_per_sm(int, size_t);
template <typename T> void launch_init(const Ctx<T>&, cudaStream_t);
template <typename T> void launch_iteration(const Ctx<T>&, cudaStream_t);
template <typename T> void launch_iteration_range(const Ctx<T>&, int, int, cudaStream_t);
template <typename T> void launch_iteration_timed(const Ctx<T>&, cudaStream_t, cudaEvent_t*);
template <typename T> void launch_final(const Ctx<T>&, cudaStream_t, T*, T*);
template <typename T> void launch_adj_restore(const Ctx<T>&, int, const double*, int, cudaStream_t);
template <typename T> void launch_adj_seed(const Ctx<T>&, T*, T*, SolveScalars*, cudaStream_t);
template <typename T>
void launch_adj_step(const Ctx<T>&, const T*, T*, T*, T*, T*, T*, const T*, SolveScalars*, T*, const double*, int, int,
                     cudaStream_t, const unsigned*);
// the persistent batch kernel is instantiated in ccmf_f32.cu / ccmf_f64.cu only
template <typename T> int wx_tma_blocks_per_sm();
extern template int wx_tma_blocks_per_sm<float>();
extern template int batch_persist_blocks_per_sm<float>(int, size_t);
extern template int batch_persist_blocks_per_sm<double>(int, size_t);
extern template void launch_batch_persist<float>(const PersistArgs<float>&, int, int, size_t, cudaStream_t);
extern template void launch_batch_persist<double>(const PersistArgs<double>&, int, int, size_t, cudaStream_t);
}  // namespace ccmf

namespace {

constexpr int kMaxN = 1024;
constexpr size_t kSmemBudget = 96 * 1024;
constexpr size_t kSmemMax = 200 * 1024;   // dynamic shared memory of one block, at most
constexpr int kMaxTimedIters = 2048;
// update-pass variant per precision, from measurements on GB300: register vectors in
// ticket-ordered chunks. FP32 is bandwidth-bound: with half the voxels per thread and two
// blocks per SM (variant 11) a 512^3 pass takes 2.37 ms against 2.41 ms (variant 0) and
// 4.1 TB/s for the pipelines; at 128^3 x 3, 0.1525 against 0.1538 ms. FP64 is ALU-bound.
constexpr int kDefaultUpdateVariantF32 = 11;
constexpr int kDefaultUpdateVariantF64 = 0;
// the captured loop runs the solves of a batch as up to this many independent graph
// branches, so that one branch's FFT pass (on-chip work) overlaps another branch's
// streaming passes (HBM work)
constexpr int kMaxBranches = 4;
constexpr double kPi = 3.14159265358979323846264338327950288;

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Radix schedule for a line of length n (prime factors 2, 3, 5). mode 0: 8s first,
// then 4 / 2, then 3s and 5s; mode 1: as 0, but a power-of-two part of the form
// 8^a * 2 becomes 8^(a-1) * 4 * 4; mode 2: radix 4 at most. Returns false for
// unsupported n.
bool make_axis_plan(int n, AxisPlan* ap, int mode = 0) {
    memset(ap, 0, sizeof(*ap));
    ap->n = n;
    int m = n, st = 0;
    auto push = [&](int r) {
        if (st >= kMaxStages) return false;
        ap->rad[st++] = r;
        m /= r;
        return true;
    };
    int p2 = 1;
    while ((m / p2) % 2 == 0) p2 *= 2;
    int n8 = 0, t = p2;
    while (mode != 2 && t % 8 == 0) {
        ++n8;
        t /= 8;
    }
    if (mode == 1 && t == 2 && n8 >= 1) --n8;   // 8^a * 2 -> 8^(a-1) * 16 = 8^(a-1) * 4 * 4
    for (int k = 0; k < n8; ++k)
        if (!push(8)) return false;
    while (m % 4 == 0)
        if (!push(4)) return false;
    while (m % 2 == 0)
        if (!push(2)) return false;
    while (m % 3 == 0)
        if (!push(3)) return false;
    while (m % 5 == 0)
        if (!push(5)) return false;
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

// Frequency held by slot p after the in-place decimation-in-frequency stages:
// k(p) = sum_s q_s prod_{t<s} R_t with q_s = (p / m_s) mod R_s.
int digit_reversed_frequency(const AxisPlan& ap, int p) {
    int k = 0, w = 1;
    for (int t = 0; t < ap.nst; ++t) {
        const int m = ap.span[t] / ap.rad[t];
        const int q = (p / m) % ap.rad[t];
        k += q * w;
        w *= ap.rad[t];
    }
    return k;
}

// Largest power of two <= min(cap, x), at least 1.
int pow2_floor(long long x, int cap) {
    int r = 1;
    while (r * 2 <= cap && r * 2 <= x) r *= 2;
    return r;
}

struct GraphKey {
    int chunk, timed;
    const void* ws;
    const void* gamma;
    long long gstride;
    LoopConfig cfg;
};

}  // namespace

struct ccmf_plan {
    int n1, n2, n3, n3h, batch, prec, device;
    size_t esize;  // bytes per real element
    Geom g;
    AxisPlan ax[3];
    LaunchShape sh;
    void* tw[3];
    void* sym[3];
    void* rsym[2];   // x, y symbol tables in digit-reversed order
    // workspace layout
    size_t off_sc, off_nact, off_xi, off_part, off_hist, off_e, off_v, off_spec, off_phi, off_gam, off_cut,
        off_flow, off_ab, total;
    cudaStream_t cap_stream;
    cudaStream_t branch_stream[kMaxBranches];
    cudaEvent_t fork_event, join_event[kMaxBranches];
    int branches;    // graph branches of the loop (1 = one chain for the whole batch)
    int sms;         // SM count of the device
    int part_cap;    // partial-sum slots per solve reserved in the workspace
    ccmf_tuning tune;  // knob values of the current launch shape
    int* h_nactive;  // pinned
    // captured loop graph
    cudaGraphExec_t gexec;
    GraphKey gkey;
    bool have_graph;
    // timing
    int timing;
    std::vector<cudaEvent_t> events;
    int timed_iters;
    double kms[kNumKernelClasses];
    long long klaunch[kNumKernelClasses];
    long long launches_last;
    // reverse mode of an FP32 plan with an FP64 forward (ccmf_set_adjoint_forward)
    int adj_forward;         // precision of the adjoint's forward and recompute passes
    ccmf_plan* shadow64;     // FP64 plan of the same grid and batch for those passes
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? CCMF_OK : CCMF_ERR_CUDA; }

// NVTX range over a scope (host-side enqueue of a call or phase; visible in nsys / ncu
// --nvtx; header-only, no cost without a profiler attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

int device_sms() {
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 152;
    }
    return sms;
}

void tuning_auto(ccmf_tuning* t) {
    t->update_variant = -1;
    t->plane_blocks = -1;
    t->z_pairs_per_block = -1;
    t->y_lines_per_block = -1;
    t->x_lines_per_block = -1;
    t->branches = -1;
    t->radix_mode = 0;
    t->zinv_pairs_per_block = -1;
    t->line_engine = -1;
    t->z_engine = -1;
}

bool pow2_in(int x, int lo, int hi) { return x >= lo && x <= hi && (x & (x - 1)) == 0; }

// Knob values -> launch shape of the plan's grid. A negative knob takes the built-in
// rule (the environment overrides CCMF_UPDATE_VARIANT, CCMF_PLANE_FUSED,
// CCMF_PLANE_CLUSTER and CCMF_BRANCHES apply to those only). Returns
// CCMF_ERR_UNSUPPORTED_SIZE when an explicit knob cannot run here; `res` receives
// every knob resolved.
int shape_for(const ccmf_plan* pl, const ccmf_tuning& t, LaunchShape* out, ccmf_tuning* res) {
    const int n1 = pl->n1, n2 = pl->n2, n3 = pl->n3, batch = pl->batch;
    const bool f64 = pl->prec == CCMF_FP64;
    const size_t cs = 2 * pl->esize;
    const int sms = pl->sms;
    LaunchShape sh;
    memset(&sh, 0, sizeof(sh));
    ccmf_tuning r = t;
    if (r.radix_mode < 0) r.radix_mode = 0;
    if (r.radix_mode > 2) return CCMF_ERR_UNSUPPORTED_SIZE;
    // FFT passes: lines per block (powers of two), shared memory = twiddles + 2 tiles
    auto smem_lines = [&](int n, int L) { return ((size_t)n + 2 * (size_t)n * (L + 1)) * cs; };
    auto lines_for = [&](int n) {
        long long L = ((long long)(kSmemBudget / cs) - n) / (2LL * n) - 1;
        return pow2_floor(L, 16);
    };
    auto pick = [&](int want, int n, int* L) {
        if (want < 0) {
            *L = lines_for(n);
            return true;
        }
        if (!pow2_in(want, 1, 16) || smem_lines(n, want) > kSmemMax) return false;
        *L = want;
        return true;
    };
    if (!pick(r.z_pairs_per_block, n3, &sh.pairs_per_block) || !pick(r.y_lines_per_block, n2, &sh.lpb_y) ||
        !pick(r.x_lines_per_block, n1, &sh.lpb_x) || !pick(r.zinv_pairs_per_block, n3, &sh.pairs_inv))
        return CCMF_ERR_UNSUPPORTED_SIZE;
    sh.smem_z = smem_lines(n3, sh.pairs_per_block);
    sh.smem_zi = smem_lines(n3, sh.pairs_inv);
    r.zinv_pairs_per_block = sh.pairs_inv;
    sh.smem_y = smem_lines(n2, sh.lpb_y);
    sh.smem_x = smem_lines(n1, sh.lpb_x);
    r.z_pairs_per_block = sh.pairs_per_block;
    r.y_lines_per_block = sh.lpb_y;
    r.x_lines_per_block = sh.lpb_x;
    long long gu = (pl->g.N + kThreads - 1) / kThreads;
    if (gu > 608) gu = 608;
    sh.grid_update = (int)gu;
    sh.vec_resident = (f64 ? update_vec_blocks_per_sm<double>() : update_vec_blocks_per_sm<float>()) * sms;
    sh.vec_resident_half = 0;
    // TMA-staged update: tiles of J z rows with J * N3 <= 512 (FP32) / 256 (FP64) voxels,
    // J a power of two dividing N2; two stages must fit the shared memory of a block
    const int tv_max = f64 ? 256 : 512;
    const int W = f64 ? 2 : 4;
    int J = 1;
    while (2 * J * n3 <= tv_max && n2 % (2 * J) == 0) J *= 2;
    const size_t smem_tma = 2 * (size_t)tma_stage_elems(J * n3, n3) * pl->esize + 16;
    sh.tma_rows = (n3 % W == 0 && smem_tma <= kSmemMax) ? J : 0;
    sh.smem_tma = smem_tma;
    long long ntiles = (long long)n1 * (n2 / J);
    long long gt = (2LL * sms + batch - 1) / batch;
    if (gt > ntiles) gt = ntiles;
    if (gt < 1) gt = 1;
    sh.grid_tma = (int)gt;
    // update variant: a pipelined update tile is one W-group per thread, TV = threads * W
    // voxels = whole z rows (or z segments)
    int variant = r.update_variant;
    const bool explicit_variant = variant >= 0;
    if (!explicit_variant) {
        const char* env = getenv("CCMF_UPDATE_VARIANT");
        const int vdef = f64 ? kDefaultUpdateVariantF64 : kDefaultUpdateVariantF32;
        variant = env ? atoi(env) : vdef;
        if (variant < 0 || variant > 7) variant = vdef;
    }
    if (variant >= kNumUpdateVariants) return CCMF_ERR_UNSUPPORTED_SIZE;
    sh.upd_variant = 0;
    if ((variant == 11 || variant == 12) && n3 % W == 0) {
        // the vector update with half the voxels per thread (8-byte vectors in FP32), two blocks per
        // SM (11) or three (12)
        sh.upd_variant = variant;
        sh.vec_resident_half = (f64 ? update_vec_half_blocks_per_sm<double>(variant)
                                    : update_vec_half_blocks_per_sm<float>(variant)) * sms;
    }
    if (is_abw_variant(variant)) {
        // warp-independent stored-divergence update: an item is tj rows of one z segment of 32 VW
        // voxels over an x segment; x segments sized like those of variants 8 .. 10
        int vw = 0, tj = 0;
        if (f64)
            abw_params<double>(variant, vw, tj);
        else
            abw_params<float>(variant, vw, tj);
        const int kz = 32 * vw;
        const size_t smem = (size_t)kAbwWarps * 4 * tj * kz * pl->esize;
        if (n3 % kz == 0 && smem <= kSmemMax) {
            const int nb = f64 ? ab_blocks_per_sm<double>(variant, smem) : ab_blocks_per_sm<float>(variant, smem);
            if (nb > 0) {
                AbShape& a = sh.ab;
                a.tj = tj;
                a.nq = (n2 + tj - 1) / tj;
                a.npass = n3 / kz;
                const long long slots = (long long)nb * kAbwWarps * sms;
                double best = -1.0;
                for (int nr = 1; nr <= n1; ++nr) {
                    const int xs = (n1 + nr - 1) / nr;
                    if ((long long)(nr - 1) * xs >= n1) continue;
                    const long long items = (long long)a.nq * nr * a.npass * batch;
                    const long long waves = (items + slots - 1) / slots;
                    const double eff = (double)n1 / ((double)nr * (xs + 2)) * (double)items / (double)(waves * slots);
                    if (eff > best + 1e-9) {
                        best = eff;
                        a.nr = nr;
                        a.xs = xs;
                    }
                }
                sh.upd_variant = variant;
                sh.smem_ab = smem;
            }
        }
    }
    if (variant >= 8 && variant <= 10) {
        // stored-divergence update: whole z rows in passes of 32 VW voxels, a block of NW warps
        // (NW - 2 interior rows); x segments sized so that the blocks of a launch fill the
        // resident slots of the GPU in whole waves as far as possible
        int nw = 0, vw = 0;
        if (f64) {
            CCMF_DISPATCH_AB(variant, {
                nw = AbVariant<double, AV>::NW;
                vw = AbVariant<double, AV>::VW;
            });
        } else {
            CCMF_DISPATCH_AB(variant, {
                nw = AbVariant<float, AV>::NW;
                vw = AbVariant<float, AV>::VW;
            });
        }
        const int kz = 32 * vw, tj = nw - 2;
        const size_t smem = ab_smem_elems(tj, n3, nw, vw) * pl->esize;
        if (n3 % kz == 0 && smem <= kSmemMax) {
            const int nb = f64 ? ab_blocks_per_sm<double>(variant, smem) : ab_blocks_per_sm<float>(variant, smem);
            if (nb > 0) {
                AbShape& a = sh.ab;
                a.tj = tj;
                a.nq = (n2 + tj - 1) / tj;
                a.npass = n3 / kz;
                const long long slots = (long long)nb * sms;
                double best = -1.0;
                for (int nr = 1; nr <= n1; ++nr) {
                    const int xs = (n1 + nr - 1) / nr;
                    if ((long long)(nr - 1) * xs >= n1) continue;   // the same xs with fewer segments
                    const long long items = (long long)a.nq * nr * batch;
                    const long long waves = (items + slots - 1) / slots;
                    // useful slab updates over slab updates done, times the share of busy slots
                    const double eff = (double)n1 / ((double)nr * (xs + 2)) * (double)items / (double)(waves * slots);
                    if (eff > best + 1e-9) {
                        best = eff;
                        a.nr = nr;
                        a.xs = xs;
                    }
                }
                sh.upd_variant = variant;
                sh.smem_ab = smem;
            }
        }
    }
    if (variant >= 2 && variant <= 7) {
        const int vw = f64 ? 1 : 2;
        const int tv = kUpdatePipe[variant][0] * vw;
        const int stages = kUpdatePipe[variant][1];
        const bool rows_ok = n3 <= tv && tv % n3 == 0 && n2 % (tv / n3) == 0;
        const bool seg_ok = n3 > tv && n3 % tv == 0;
        if (n3 % W == 0 && (rows_ok || seg_ok)) {
            const int kt = seg_ok ? tv : n3;
            const size_t smem =
                (size_t)stages * (size_t)pipe_stage_elems(tv, kt, seg_ok, 16 / (int)pl->esize) * pl->esize +
                8 * stages;
            const int nb = f64 ? pipe_blocks_per_sm<double>(variant, smem) : pipe_blocks_per_sm<float>(variant, smem);
            if (nb > 0) {
                sh.upd_variant = variant;
                sh.smem_pipe = smem;
                long long nt = (long long)n1 * (n2 / (tv / kt)) * (n3 / kt);
                long long gp = ((long long)nb * sms + batch - 1) / batch;
                if (gp > nt) gp = nt;
                sh.grid_pipe = (int)(gp < 1 ? 1 : gp);
            }
        }
    }
    if (sh.upd_variant == 0 && variant >= 1 && sh.tma_rows > 0) sh.upd_variant = 1;
    if (explicit_variant && sh.upd_variant != variant) return CCMF_ERR_UNSUPPORTED_SIZE;
    r.update_variant = sh.upd_variant;
    sh.grid_partials = std::max(sh.grid_update, sh.grid_tma);
    if (sh.upd_variant >= 2 && sh.upd_variant <= 7) sh.grid_partials = std::max(sh.grid_partials, sh.grid_pipe);
    if (is_abw_variant(sh.upd_variant))
        sh.grid_partials = std::max<int>(sh.grid_partials,
                                         (int)ceil_div((long long)sh.ab.nq * sh.ab.nr * sh.ab.npass, kAbwWarps));
    else if (is_ab_variant(sh.upd_variant))
        sh.grid_partials = std::max(sh.grid_partials, sh.ab.nq * sh.ab.nr);
    // the vector update pass (variant 0 and every final evaluation) keeps one slot per chunk
    sh.grid_partials = (int)std::max<long long>(sh.grid_partials, vec_update_chunks(pl->g.N, f64 ? 2 : 4));
    if (sh.upd_variant == 11 || sh.upd_variant == 12)
        sh.grid_partials = (int)std::max<long long>(sh.grid_partials,
                                                    vec_update_chunks(pl->g.N, f64 ? 1 : 2));
    // y / x passes: one block per k_z plane when the plane fits its shared memory, a
    // cluster of C blocks (C divides n1 and n2) sharing the plane through distributed
    // shared memory, or the three strided passes
    sh.plane_fused = 0;
    sh.plane_cluster = 1;
    sh.smem_plane = 0;
    const size_t smem1 = ((size_t)n1 + n2 + (size_t)n1 * (n2 + 1)) * cs;
    const bool one_fits = (long long)n1 * n2 <= kPlaneMax && smem1 <= kSmemMax;
    int pb = r.plane_blocks;
    if (pb < 0) {
        const char* envp = getenv("CCMF_PLANE_FUSED");
        const char* envc = getenv("CCMF_PLANE_CLUSTER");
        if (envp && atoi(envp) == 0)
            pb = 0;
        else if (envc && atoi(envc) > 0)
            pb = atoi(envc);
        else
            pb = one_fits ? 1 : 0;
    }
    if (pb == 1) {
        if (!one_fits) return CCMF_ERR_UNSUPPORTED_SIZE;
        sh.plane_fused = 1;
        sh.smem_plane = smem1;
    } else if (pb >= 2) {
        if (!pow2_in(pb, 2, 16) || n1 % pb != 0 || n2 % pb != 0) return CCMF_ERR_UNSUPPORTED_SIZE;
        const long long emax = (long long)(f64 ? PlaneRegs<double>::M : PlaneRegs<float>::M) * kPlaneClusterThreads;
        if ((long long)n1 * n2 / pb > emax) return CCMF_ERR_UNSUPPORTED_SIZE;
        const long long r1 = n1 / pb, r2 = n2 / pb;
        const long long tile = std::max(r1 * (n2 + 1), r2 * (n1 + 1));
        const size_t smem = ((size_t)n1 + n2 + (size_t)tile) * cs;
        if (smem > kSmemMax) return CCMF_ERR_UNSUPPORTED_SIZE;
        const int cap = f64 ? plane_cluster_capacity<double>(pb, smem) : plane_cluster_capacity<float>(pb, smem);
        if (cap < 1) return CCMF_ERR_UNSUPPORTED_SIZE;
        sh.plane_fused = 1;
        sh.plane_cluster = pb;
        sh.smem_plane = smem;
        sh.div_r1 = make_fastdiv((unsigned)r1);
        sh.div_r2 = make_fastdiv((unsigned)r2);
    } else if (pb != 0) {
        return CCMF_ERR_UNSUPPORTED_SIZE;
    }
    r.plane_blocks = sh.plane_fused ? sh.plane_cluster : 0;
    // strided line passes: one warp per line for power-of-two lengths 128 ... 1024
    // (line_engine 1), else in-place radix stages over tiles of lines
    int le = r.line_engine;
    const bool le_auto = le < 0 && !getenv("CCMF_LINE_ENGINE");
    if (le < 0) {
        // warp per line by default (GB300, 512^2 planes: y passes 0.29 ms against 0.37 ms
        // for the block stages, x pass 0.62 against 0.64 ms); the autotuner tries both
        const char* env = getenv("CCMF_LINE_ENGINE");
        le = env ? atoi(env) : 1;
        if (le < 0 || le > 1) le = 1;
    }
    if (le > 2) return CCMF_ERR_UNSUPPORTED_SIZE;
    r.line_engine = le;
    auto warp_len_ok = [](int n) { return n >= 128 && n <= 1024 && (n & (n - 1)) == 0; };
    sh.wl_y = sh.wl_x = 0;
    sh.x_tma = 0;
    if (!sh.plane_fused && le >= 1) {
        // y: twiddles + one padded line per warp; x: twiddles + two tiles of 8 lines
        const size_t swy = ((size_t)n2 + 8 * (size_t)(n2 + n2 / 16)) * cs;
        const size_t swx = ((size_t)n1 + 2 * 8 * (size_t)(n1 + n1 / 16 + 2)) * cs;
        if (warp_len_ok(n2) && swy <= kSmemMax) {
            sh.wl_y = n2;
            sh.smem_wy = swy;
        }
        if (warp_len_ok(n1) && swx <= kSmemMax) {
            sh.wl_x = n1;
            sh.smem_wx = swx;
        }
        // line engine 2: the x pass with its tiles moved by TMA (FP32, n1 = 512, n2 % 8 == 0); the
        // built-in choice where it applies (GB300, 512^3: 0.218 against 0.339 ms per x pass)
        if (le_auto && le == 1 && !f64 && sh.wl_x == kTmaXN && x_tma_shape_ok(n1, n2, pl->n3h, batch)) {
            le = 2;
            r.line_engine = 2;
        }
        if (le == 2) {
            if (f64 || sh.wl_x != kTmaXN || !x_tma_shape_ok(n1, n2, pl->n3h, batch))
                return CCMF_ERR_UNSUPPORTED_SIZE;
            sh.x_tma = 1;
        }
    } else if (le == 2) {
        return CCMF_ERR_UNSUPPORTED_SIZE;
    }
    // z passes: one warp per line pair for power-of-two N3 128 ... 1024: z_engine 1 the
    // inverse pass only, 2 both passes (the divergence pass's stencil loads favour the
    // block tiles on GB300)
    int ze = r.z_engine;
    if (ze < 0) {
        // measured on GB300: the warp divergence pass wins at N3 = 512 (1.30 against 1.41 ms
        // per 512^3 pass) and loses at 128; the warp inverse pass wins at both
        const char* env = getenv("CCMF_Z_ENGINE");
        const int zdef = n3 >= 512 ? 2 : 1;
        ze = env ? atoi(env) : zdef;
        if (ze < 0 || ze > 2) ze = zdef;
    }
    if (ze > 2) return CCMF_ERR_UNSUPPORTED_SIZE;
    r.z_engine = ze;
    sh.wz = sh.wzd = 0;
    if (ze >= 1 && warp_len_ok(n3)) {
        const size_t lsz = (size_t)n3 + n3 / 16 + 1;
        const size_t sd = ((size_t)n3 + 8 * lsz) * cs;
        // inverse: twiddles + the larger of the slab of 16 spectrum rows and the 8 scratch lines
        const size_t si = ((size_t)n3 + std::max(8 * lsz, (size_t)(n3 / 2 + 1) * 17)) * cs;
        if (si <= kSmemMax) {
            sh.wz = n3;
            sh.smem_wzi = si;
        }
        if (ze == 2 && sd <= kSmemMax) {
            sh.wzd = n3;
            sh.smem_wzd = sd;
        }
    }
    if (!sh.plane_fused) {
        // persistent line passes: resident blocks x SMs, shared by the solves of the batch
        const int by = sh.wl_y ? (f64 ? wlines_blocks_per_sm<double>(0, n2, sh.smem_wy)
                                      : wlines_blocks_per_sm<float>(0, n2, sh.smem_wy))
                               : (f64 ? lines_blocks_per_sm<double>(0, sh.lpb_y, sh.smem_y)
                                      : lines_blocks_per_sm<float>(0, sh.lpb_y, sh.smem_y));
        const int bx = sh.x_tma  ? wx_tma_blocks_per_sm<float>()
                       : sh.wl_x ? (f64 ? wlines_blocks_per_sm<double>(1, n1, sh.smem_wx)
                                        : wlines_blocks_per_sm<float>(1, n1, sh.smem_wx))
                                 : (f64 ? lines_blocks_per_sm<double>(1, sh.lpb_x, sh.smem_x)
                                        : lines_blocks_per_sm<float>(1, sh.lpb_x, sh.smem_x));
        if (by < 1 || bx < 1) return CCMF_ERR_UNSUPPORTED_SIZE;
        sh.grid_y = (int)std::max(1LL, ((long long)by * sms + batch - 1) / batch);
        sh.grid_x = (int)std::max(1LL, ((long long)bx * sms + batch - 1) / batch);
    }
    // graph branches of a batch (never more than the solves)
    int nb = r.branches;
    if (nb < 0) {
        const char* envb = getenv("CCMF_BRANCHES");
        nb = envb ? atoi(envb) : kMaxBranches;
        if (nb < 1) nb = 1;
        if (nb > kMaxBranches) nb = kMaxBranches;
    }
    if (nb < 1 || nb > kMaxBranches) return CCMF_ERR_UNSUPPORTED_SIZE;
    r.branches = std::min(nb, batch);
    *out = sh;
    if (res) *res = r;
    return CCMF_OK;
}

// Partial-sum slots per solve the workspace reserves: the largest grid of any update
// variant, so that every tuning fits the same workspace.
int partials_capacity(const ccmf_plan* pl) {
    int cap = std::max(608, pl->sh.grid_partials);
    for (int v = 0; v < kNumUpdateVariants; ++v) {
        ccmf_tuning t;
        tuning_auto(&t);
        t.update_variant = v;
        LaunchShape sh;
        if (shape_for(pl, t, &sh, nullptr) == CCMF_OK) cap = std::max(cap, sh.grid_partials);
    }
    return cap;
}

// ---- the tuning table: (N1, N2, N3, batch, precision, SM count) -> knob values ----
struct TuneKey {
    int n1, n2, n3, batch, prec, sms;
    bool operator<(const TuneKey& o) const {
        const int a[6] = {n1, n2, n3, batch, prec, sms}, b[6] = {o.n1, o.n2, o.n3, o.batch, o.prec, o.sms};
        return std::lexicographical_compare(a, a + 6, b, b + 6);
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, ccmf_tuning> g_tune_table;

TuneKey tune_key(const ccmf_plan* pl) { return TuneKey{pl->n1, pl->n2, pl->n3, pl->batch, pl->prec, pl->sms}; }

bool tuning_lookup(const ccmf_plan* pl, ccmf_tuning* t) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_table.find(tune_key(pl));
    if (it == g_tune_table.end()) return false;
    *t = it->second;
    return true;
}

void tuning_store(const ccmf_plan* pl, const ccmf_tuning& t) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_table[tune_key(pl)] = t;
}



bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
Ctx<T> make_ctx(const ccmf_plan* pl, unsigned char* ws, const T* gamma, long long gstride, const LoopConfig& cfg) {
    Ctx<T> c;
    memset(&c, 0, sizeof(c));
    c.g = pl->g;
    c.cfg = cfg;
    for (int a = 0; a < 3; ++a) {
        c.ax[a] = pl->ax[a];
        c.tw[a] = reinterpret_cast<const cx<T>*>(pl->tw[a]);
        c.sym[a] = reinterpret_cast<const T*>(pl->sym[a]);
    }
    c.rsym[0] = reinterpret_cast<const T*>(pl->rsym[0]);
    c.rsym[1] = reinterpret_cast<const T*>(pl->rsym[1]);
    c.sh = pl->sh;
    c.xi_stage = reinterpret_cast<const double*>(ws + pl->off_xi);
    c.p.sc = reinterpret_cast<SolveScalars*>(ws + pl->off_sc);
    c.p.n_active = reinterpret_cast<int*>(ws + pl->off_nact);
    c.p.partial = reinterpret_cast<double*>(ws + pl->off_part);
    c.p.hist = reinterpret_cast<double*>(ws + pl->off_hist);
    c.p.e = reinterpret_cast<T*>(ws + pl->off_e);
    c.p.v = reinterpret_cast<T*>(ws + pl->off_v);
    c.p.sstride = 6 * pl->g.N * (long long)pl->batch;
    c.p.spec = reinterpret_cast<cx<T>*>(ws + pl->off_spec);
    c.p.phi = reinterpret_cast<T*>(ws + pl->off_phi);
    c.p.gamma = gamma;
    c.p.gstride = gstride;
    c.p.cut = nullptr;
    c.p.flow = nullptr;
    c.p.run_all = 0;
    const int W = 16 / (int)sizeof(T);
    c.vec_div = (pl->n3 % W) == 0;
    c.vec_update = c.vec_div && ((uintptr_t)gamma % 16) == 0;
    c.p.ab = reinterpret_cast<T*>(ws + pl->off_ab);
    // the stored-divergence schedule needs the vector loads of gamma (a per-solve pointer
    // table is aligned by the batch API's allocations of whole fields)
    c.use_ab = is_ab_variant(pl->sh.upd_variant) && c.vec_update;
    return c;
}

void destroy_graph(ccmf_plan* pl) {
    if (pl->have_graph) cudaGraphExecDestroy(pl->gexec);
    pl->have_graph = false;
}

template <typename T>
int capture_loop(ccmf_plan* pl, const Ctx<T>& c, const GraphKey& key) {
    if (pl->have_graph && memcmp(&pl->gkey, &key, sizeof(key)) == 0) return CCMF_OK;
    destroy_graph(pl);
    int cls[kNumKernelClasses];
    const int nk = iteration_classes(pl->sh, cls);
    if (key.timed) {
        size_t need = (size_t)key.chunk * nk + 1;
        while (pl->events.size() < need) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return CCMF_ERR_CUDA;
            pl->events.push_back(ev);
        }
    }
    cudaGraph_t graph;
    cudaError_t err = cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return CCMF_ERR_CUDA;
    if (key.timed) cudaEventRecordWithFlags(pl->events[0], pl->cap_stream, cudaEventRecordExternal);
    if (key.timed || pl->branches <= 1) {
        for (int it = 0; it < key.chunk; ++it) {
            if (key.timed)
                launch_iteration_timed<T>(c, pl->cap_stream, pl->events.data() + (size_t)it * nk);
            else
                launch_iteration<T>(c, pl->cap_stream);
        }
    } else {
        // fork: each branch runs its solves' chain of iterations; join at the end of the chunk
        const int nb = pl->branches;
        cudaEventRecord(pl->fork_event, pl->cap_stream);
        for (int b = 0; b < nb; ++b) {
            const int s0 = (int)((long long)pl->batch * b / nb), s1 = (int)((long long)pl->batch * (b + 1) / nb);
            cudaStreamWaitEvent(pl->branch_stream[b], pl->fork_event, 0);
            for (int it = 0; it < key.chunk; ++it) launch_iteration_range<T>(c, s0, s1 - s0, pl->branch_stream[b]);
            cudaEventRecord(pl->join_event[b], pl->branch_stream[b]);
            cudaStreamWaitEvent(pl->cap_stream, pl->join_event[b], 0);
        }
    }
    err = cudaStreamEndCapture(pl->cap_stream, &graph);
    if (err != cudaSuccess) return CCMF_ERR_CUDA;
    err = cudaGraphInstantiate(&pl->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) return CCMF_ERR_CUDA;
    pl->gkey = key;
    pl->have_graph = true;
    return CCMF_OK;
}

template <typename T>
int solve_impl(ccmf_plan* pl, const void* gamma_in, long long gstride_in, const double* xi_host,
               const ccmf_params* prm, unsigned char* ws, void* flow, void* cut, ccmf_result* results,
               cudaStream_t st) {
    const Geom& g = pl->g;
    const size_t N = (size_t)g.N;
    // gamma: device pointer or host memory staged into the workspace
    const T* gamma = reinterpret_cast<const T*>(gamma_in);
    long long gstride = gstride_in;
    if (!is_device_ptr(gamma_in)) {
        T* stage = reinterpret_cast<T*>(ws + pl->off_gam);
        size_t fields = gstride_in == 0 ? 1 : (size_t)g.batch;
        for (size_t s = 0; s < fields; ++s) {
            if (cudaMemcpyAsync(stage + s * N, reinterpret_cast<const T*>(gamma_in) + s * (size_t)gstride_in,
                                N * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
                return CCMF_ERR_CUDA;
        }
        gamma = stage;
        gstride = gstride_in == 0 ? 0 : (long long)N;
    }
    // unit normals
    std::vector<double> xi(3 * (size_t)g.batch);
    for (int s = 0; s < g.batch; ++s) {
        const double* x = xi_host + 3 * s;
        double nn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int a = 0; a < 3; ++a) xi[3 * s + a] = x[a] / nn;
    }
    if (cudaMemcpyAsync(ws + pl->off_xi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return CCMF_ERR_CUDA;
    if (cudaMemsetAsync(ws + pl->off_nact, 0, sizeof(int), st) != cudaSuccess) return CCMF_ERR_CUDA;
    if (!prm->resume &&
        cudaMemsetAsync(ws + pl->off_hist, 0xFF, sizeof(double) * kHistFields * (size_t)kHistCap * g.batch, st) !=
            cudaSuccess)
        return CCMF_ERR_CUDA;

    LoopConfig cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.tol = prm->tol;
    cfg.delta = prm->delta;
    cfg.rho0 = prm->rho0;
    cfg.bb_corr_min = prm->bb_corr_min;
    cfg.rho_step_max = prm->rho_step_max;
    cfg.max_iter = prm->max_iter;
    cfg.fixed_iters = prm->fixed_iters;
    cfg.rho_rule = prm->rho_rule;
    cfg.hist_len = prm->history_len;
    cfg.resume = prm->resume;
    {
        // debug only: a tiny budget for the bounded device waits makes them give up, to test
        // the CCMF_ERR_TIMEOUT path; the waits for copies still in flight keep the full budget
        const char* env = getenv("CCMF_DEBUG_SPIN_LIMIT");
        cfg.spin_limit = env ? (unsigned)strtoul(env, nullptr, 10) + 1u : 0u;
    }
    Ctx<T> c = make_ctx<T>(pl, ws, gamma, gstride, cfg);

    {
        NvtxRange r("ccmf init");
        launch_init<T>(c, st);
    }
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;

    const bool fixed = prm->fixed_iters > 0;
    const int total = fixed ? prm->fixed_iters : prm->max_iter;
    const bool timed = pl->timing && fixed;
    int chunk = timed ? total : (prm->check_every < total ? prm->check_every : total);
    if (timed && total > kMaxTimedIters) return CCMF_ERR_INVALID_ARG;
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.chunk = chunk;
    key.timed = timed ? 1 : 0;
    key.ws = ws;
    key.gamma = gamma;
    key.gstride = gstride;
    key.cfg = cfg;
    int rc = capture_loop<T>(pl, c, key);
    if (rc != CCMF_OK) return rc;
    const long long nchunks_max = ((long long)total + chunk - 1) / chunk;
    pl->launches_last = 0;
    NvtxRange r_loop("ccmf loop");
    for (long long ch = 0; ch < nchunks_max; ++ch) {
        if (cudaGraphLaunch(pl->gexec, st) != cudaSuccess) return CCMF_ERR_CUDA;
        int cls_tmp[kNumKernelClasses];
        pl->launches_last += (long long)chunk * iteration_classes(pl->sh, cls_tmp);
        if (!fixed) {
            if (cudaMemcpyAsync(pl->h_nactive, ws + pl->off_nact, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess)
                return CCMF_ERR_CUDA;
            if (cudaStreamSynchronize(st) != cudaSuccess) return CCMF_ERR_CUDA;
            if (*pl->h_nactive <= 0) break;
        }
    }
    // final evaluation of the state (cut, flow, primal and dual objectives)
    NvtxRange r_final("ccmf final evaluation");
    const bool cut_host = cut && !is_device_ptr(cut);
    const bool flow_host = flow && !is_device_ptr(flow);
    T* cut_d = cut_host ? reinterpret_cast<T*>(ws + pl->off_cut) : reinterpret_cast<T*>(cut);
    T* flow_d = flow_host ? reinterpret_cast<T*>(ws + pl->off_flow) : reinterpret_cast<T*>(flow);
    launch_final<T>(c, st, cut_d, flow_d);
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
    if (cut_host && cudaMemcpyAsync(cut, cut_d, (size_t)g.batch * 6 * N * sizeof(T), cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess)
        return CCMF_ERR_CUDA;
    if (flow_host &&
        cudaMemcpyAsync(flow, flow_d, (size_t)g.batch * 3 * N * sizeof(T), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    if (results || cut_host || flow_host || timed) {
        std::vector<SolveScalars> sc(g.batch);
        if (cudaMemcpyAsync(sc.data(), ws + pl->off_sc, sizeof(SolveScalars) * g.batch, cudaMemcpyDeviceToHost,
                            st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return CCMF_ERR_CUDA;
        if (results) {
            for (int s = 0; s < g.batch; ++s) {
                ccmf_result& r = results[s];
                r.gamma_primal = sc[s].primal;
                r.gamma_eff = sc[s].dual;
                r.gamma_dual = sc[s].dual;
                r.residual = sc[s].residual;
                r.mean_v_norm = sc[s].mean_v;
                r.rho = sc[s].rho;
                r.iters = sc[s].iters;
                r.converged = sc[s].converged;
                r.status = sc[s].status;
                r.reserved = 0;
            }
        }
    }
    if (timed) {
        for (int k = 0; k < kNumKernelClasses; ++k) {
            pl->kms[k] = 0.0;
            pl->klaunch[k] = 0;
        }
        int cls[kNumKernelClasses];
        const int nk = iteration_classes(pl->sh, cls);
        for (int it = 0; it < chunk; ++it)
            for (int k = 0; k < nk; ++k) {
                float ms = 0.f;
                size_t a = (size_t)it * nk + k;
                if (cudaEventElapsedTime(&ms, pl->events[a], pl->events[a + 1]) == cudaSuccess) {
                    pl->kms[cls[k]] += ms;
                    pl->klaunch[cls[k]] += 1;
                }
            }
        pl->timed_iters = chunk;
    }
    return CCMF_OK;
}

}  // namespace


// Symbol tables of the x and y axes in the digit-reversed order of the plan's radix
// schedule, copied into the plan's existing device buffers.
int upload_rsym(ccmf_plan* pl) {
    const int nn[2] = {pl->n1, pl->n2};
    for (int a = 0; a < 2; ++a) {
        const int n = nn[a];
        std::vector<double> rs((size_t)n);
        for (int t = 0; t < n; ++t) {
            const double sn = sin(kPi * (double)digit_reversed_frequency(pl->ax[a], t) / (double)n);
            rs[t] = 4.0 * sn * sn;
        }
        cudaError_t e;
        if (pl->prec == CCMF_FP64) {
            e = cudaMemcpy(pl->rsym[a], rs.data(), rs.size() * 8, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> rf(rs.begin(), rs.end());
            e = cudaMemcpy(pl->rsym[a], rf.data(), rf.size() * 4, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return CCMF_ERR_CUDA;
    }
    return CCMF_OK;
}

// Switch the plan to the knob values t (resolved against the built-in rules).
int apply_tuning(ccmf_plan* pl, const ccmf_tuning& t) {
    LaunchShape sh;
    ccmf_tuning res;
    int rc = shape_for(pl, t, &sh, &res);
    if (rc != CCMF_OK) return rc;
    if (sh.grid_partials > pl->part_cap) return CCMF_ERR_UNSUPPORTED_SIZE;
    if (cudaSetDevice(pl->device) != cudaSuccess) return CCMF_ERR_CUDA;
    const cudaError_t e = pl->prec == CCMF_FP64 ? configure_kernels<double>(sh) : configure_kernels<float>(sh);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CCMF_ERR_UNSUPPORTED_SIZE;
    }
    if (res.radix_mode != pl->tune.radix_mode) {
        const int nn[3] = {pl->n1, pl->n2, pl->n3};
        AxisPlan ax[3];
        for (int a = 0; a < 3; ++a)
            if (!make_axis_plan(nn[a], &ax[a], res.radix_mode)) return CCMF_ERR_UNSUPPORTED_SIZE;
        for (int a = 0; a < 3; ++a) pl->ax[a] = ax[a];
        rc = upload_rsym(pl);
        if (rc != CCMF_OK) return rc;
    }
    destroy_graph(pl);
    pl->sh = sh;
    pl->tune = res;
    pl->branches = res.branches;
    return CCMF_OK;
}


// Coordinate descent over the tuning knobs of a plan in the order of ccmf_tuning,
// from its current tuning; measure(&ms) times the plan as it is. A candidate must
// win by 1 % to be kept. Leaves the plan in the best tuning found.
int tune_descent(ccmf_plan* plan, const std::function<int(double*)>& measure, double* best_ms) {
    ccmf_tuning cur = plan->tune;
    double cur_ms = 0.0;
    int rc = measure(&cur_ms);
    // coordinate descent over the knobs; a candidate must win by 1 % to be kept
    struct Knob {
        int ccmf_tuning::*field;
        std::vector<int> values;
    };
    std::vector<int> brs;
    for (int b = 1; b <= std::min(kMaxBranches, plan->batch); ++b) brs.push_back(b);
    const Knob knobs[] = {
        {&ccmf_tuning::update_variant, {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15}},
        {&ccmf_tuning::plane_blocks, {0, 1, 2, 4, 8, 16}},
        {&ccmf_tuning::z_pairs_per_block, {1, 2, 4, 8, 16}},
        {&ccmf_tuning::y_lines_per_block, {1, 2, 4, 8, 16}},
        {&ccmf_tuning::x_lines_per_block, {1, 2, 4, 8, 16}},
        {&ccmf_tuning::branches, brs},
        {&ccmf_tuning::radix_mode, {0, 1, 2}},
        {&ccmf_tuning::zinv_pairs_per_block, {1, 2, 4, 8, 16}},
        {&ccmf_tuning::line_engine, {0, 1, 2}},
        {&ccmf_tuning::z_engine, {0, 1, 2}},
    };
    for (const Knob& k : knobs) {
        if (rc != CCMF_OK) break;
        const bool strided_only = k.field == &ccmf_tuning::y_lines_per_block ||
                                  k.field == &ccmf_tuning::x_lines_per_block || k.field == &ccmf_tuning::line_engine;
        if (strided_only && cur.plane_blocks != 0) continue;
        for (int v : k.values) {
            if (v == cur.*(k.field)) continue;
            ccmf_tuning cand = cur;
            cand.*(k.field) = v;
            if (apply_tuning(plan, cand) != CCMF_OK) continue;
            double ms = 0.0;
            rc = measure(&ms);
            if (rc != CCMF_OK) break;
            if (ms < 0.99 * cur_ms) {
                cur = plan->tune;
                cur_ms = ms;
            }
        }
        if (rc == CCMF_OK) rc = apply_tuning(plan, cur);
    }
    *best_ms = cur_ms;
    return rc;
}

extern "C" {

void ccmf_params_default(ccmf_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->tol = 1e-4;
    p->delta = 0.25;
    p->rho0 = 0.0;
    p->bb_corr_min = 0.2;
    p->rho_step_max = 2.0;
    p->max_iter = 20000;
    p->rho_rule = CCMF_RHO_BB;
    p->fixed_iters = 0;
    p->check_every = 32;
    p->resume = 0;
    p->history_len = 1024;
}

const char* ccmf_status_string(int status) {
    switch (status) {
        case CCMF_OK: return "ok";
        case CCMF_ERR_INVALID_ARG: return "invalid argument";
        case CCMF_ERR_UNSUPPORTED_SIZE: return "unsupported grid size (N_i must be 1..1024 with prime factors 2, 3, 5)";
        case CCMF_ERR_WORKSPACE: return "workspace missing or too small";
        case CCMF_ERR_CUDA: return "CUDA runtime error";
        case CCMF_ERR_NUMERICAL: return "numerical failure (invalid gamma or non-finite reduction)";
        case CCMF_ERR_TIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

int ccmf_plan_create(int n1, int n2, int n3, int batch, int precision, ccmf_plan** out) {
    if (!out) return CCMF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n1 < 1 || n2 < 1 || n3 < 1 || batch < 1 || batch > 65535) return CCMF_ERR_INVALID_ARG;
    if (precision != CCMF_FP64 && precision != CCMF_FP32_MIXED) return CCMF_ERR_INVALID_ARG;
    if (n1 > kMaxN || n2 > kMaxN || n3 > kMaxN) return CCMF_ERR_UNSUPPORTED_SIZE;
    AxisPlan ax[3];
    const int nn[3] = {n1, n2, n3};
    for (int a = 0; a < 3; ++a)
        if (!make_axis_plan(nn[a], &ax[a])) return CCMF_ERR_UNSUPPORTED_SIZE;

    ccmf_plan* pl = new (std::nothrow) ccmf_plan();
    if (!pl) return CCMF_ERR_INVALID_ARG;
    pl->n1 = n1;
    pl->n2 = n2;
    pl->n3 = n3;
    pl->n3h = n3 / 2 + 1;
    pl->batch = batch;
    pl->prec = precision;
    pl->adj_forward = precision;
    pl->esize = precision == CCMF_FP64 ? 8 : 4;
    for (int a = 0; a < 3; ++a) pl->ax[a] = ax[a];
    Geom& g = pl->g;
    g.n1 = n1;
    g.n2 = n2;
    g.n3 = n3;
    g.n3h = pl->n3h;
    g.batch = batch;
    g.N = (long long)n1 * n2 * n3;
    g.Nh = (long long)n1 * n2 * pl->n3h;
    g.div_n3 = make_fastdiv((unsigned)n3);
    g.div_n2 = make_fastdiv((unsigned)n2);
    g.div_n3h = make_fastdiv((unsigned)pl->n3h);
    g.div_n1 = make_fastdiv((unsigned)n1);

    // launch shape: the tuning table's entry for this key, else the built-in rules
    pl->sms = device_sms();
    ccmf_tuning auto_t;
    tuning_auto(&auto_t);
    ccmf_tuning want_t = auto_t;
    const bool cached = tuning_lookup(pl, &want_t);
    int src = shape_for(pl, want_t, &pl->sh, &pl->tune);
    if (src != CCMF_OK && cached) src = shape_for(pl, auto_t, &pl->sh, &pl->tune);
    if (src != CCMF_OK) {
        delete pl;
        return src;
    }
    if (pl->tune.radix_mode != 0)
        for (int a = 0; a < 3; ++a) make_axis_plan(nn[a], &pl->ax[a], pl->tune.radix_mode);
    pl->part_cap = partials_capacity(pl);
    const size_t cs = 2 * pl->esize;  // complex element
    LaunchShape& sh = pl->sh;

    // workspace layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t N = (size_t)g.N;
    pl->off_sc = take(256 * (size_t)batch);
    pl->off_nact = take(256);
    pl->off_xi = take(3 * sizeof(double) * batch);
    pl->off_part = take(sizeof(double) * kNSum * (size_t)pl->part_cap * batch);
    pl->off_hist = take(sizeof(double) * kHistFields * (size_t)kHistCap * batch);
    pl->off_e = take(pl->esize * 6 * N * batch * 2);
    pl->off_v = take(pl->esize * 6 * N * batch * 2);
    pl->off_spec = take(cs * (size_t)g.Nh * batch);
    pl->off_phi = take(pl->esize * N * batch);
    pl->off_ab = take(pl->esize * 2 * N * batch);
    pl->off_gam = take(pl->esize * N * batch);
    pl->off_cut = take(pl->esize * 6 * N * batch);
    pl->off_flow = take(pl->esize * 3 * N * batch);
    pl->total = off;

    int rc = CCMF_OK;
    if (cudaGetDevice(&pl->device) != cudaSuccess) rc = CCMF_ERR_CUDA;
    // twiddle and symbol tables
    for (int a = 0; a < 3 && rc == CCMF_OK; ++a) {
        const int n = nn[a];
        std::vector<double> tw(2 * (size_t)n), sy((size_t)n), rs((size_t)n);
        for (int t = 0; t < n; ++t) {
            const double ang = -2.0 * kPi * (double)t / (double)n;
            tw[2 * t] = cos(ang);
            tw[2 * t + 1] = sin(ang);
            const double sn = sin(kPi * (double)t / (double)n);
            sy[t] = 4.0 * sn * sn;
        }
        for (int t = 0; t < n; ++t) rs[t] = sy[digit_reversed_frequency(pl->ax[a], t)];
        if (precision == CCMF_FP64) {
            if (cudaMalloc(&pl->tw[a], tw.size() * 8) != cudaSuccess ||
                cudaMemcpy(pl->tw[a], tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMalloc(&pl->sym[a], sy.size() * 8) != cudaSuccess ||
                cudaMemcpy(pl->sym[a], sy.data(), sy.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
                rc = CCMF_ERR_CUDA;
            if (rc == CCMF_OK && a < 2 &&
                (cudaMalloc(&pl->rsym[a], rs.size() * 8) != cudaSuccess ||
                 cudaMemcpy(pl->rsym[a], rs.data(), rs.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess))
                rc = CCMF_ERR_CUDA;
        } else {
            std::vector<float> twf(tw.begin(), tw.end()), syf(sy.begin(), sy.end()), rsf(rs.begin(), rs.end());
            if (cudaMalloc(&pl->tw[a], twf.size() * 4) != cudaSuccess ||
                cudaMemcpy(pl->tw[a], twf.data(), twf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMalloc(&pl->sym[a], syf.size() * 4) != cudaSuccess ||
                cudaMemcpy(pl->sym[a], syf.data(), syf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                rc = CCMF_ERR_CUDA;
            if (rc == CCMF_OK && a < 2 &&
                (cudaMalloc(&pl->rsym[a], rsf.size() * 4) != cudaSuccess ||
                 cudaMemcpy(pl->rsym[a], rsf.data(), rsf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess))
                rc = CCMF_ERR_CUDA;
        }
    }
    if (rc == CCMF_OK) {
        cudaError_t e = precision == CCMF_FP64 ? configure_kernels<double>(sh) : configure_kernels<float>(sh);
        if (e != cudaSuccess) rc = CCMF_ERR_CUDA;
    }
    if (rc == CCMF_OK && cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = CCMF_ERR_CUDA;
    {
        // streams for every branch count a tuning may choose
        pl->branches = pl->tune.branches;
        if (rc == CCMF_OK && cudaEventCreateWithFlags(&pl->fork_event, cudaEventDisableTiming) != cudaSuccess)
            rc = CCMF_ERR_CUDA;
        for (int b = 0; b < std::min(kMaxBranches, batch) && rc == CCMF_OK; ++b) {
            if (cudaStreamCreateWithFlags(&pl->branch_stream[b], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&pl->join_event[b], cudaEventDisableTiming) != cudaSuccess)
                rc = CCMF_ERR_CUDA;
        }
    }
    if (rc == CCMF_OK && cudaMallocHost((void**)&pl->h_nactive, sizeof(int)) != cudaSuccess) rc = CCMF_ERR_CUDA;
    if (rc != CCMF_OK) {
        ccmf_plan_destroy(pl);
        return rc;
    }
    *out = pl;
    return CCMF_OK;
}

int ccmf_plan_destroy(ccmf_plan* pl) {
    if (!pl) return CCMF_OK;
    if (pl->shadow64) ccmf_plan_destroy(pl->shadow64);
    destroy_graph(pl);
    for (cudaEvent_t ev : pl->events) cudaEventDestroy(ev);
    for (int a = 0; a < 3; ++a) {
        if (pl->tw[a]) cudaFree(pl->tw[a]);
        if (pl->sym[a]) cudaFree(pl->sym[a]);
    }
    for (int a = 0; a < 2; ++a)
        if (pl->rsym[a]) cudaFree(pl->rsym[a]);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    for (int b = 0; b < kMaxBranches; ++b) {
        if (pl->branch_stream[b]) cudaStreamDestroy(pl->branch_stream[b]);
        if (pl->join_event[b]) cudaEventDestroy(pl->join_event[b]);
    }
    if (pl->fork_event) cudaEventDestroy(pl->fork_event);
    if (pl->h_nactive) cudaFreeHost(pl->h_nactive);
    delete pl;
    return CCMF_OK;
}

int ccmf_plan_workspace_bytes(const ccmf_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return CCMF_ERR_INVALID_ARG;
    *bytes = plan->total;
    return CCMF_OK;
}

int ccmf_solve(ccmf_plan* plan, const void* gamma, long long gamma_stride, const double* xi_bar,
               const ccmf_params* params, void* workspace, size_t workspace_bytes, void* flow, void* cut,
               ccmf_result* results, void* stream) {
    NvtxRange nvtx_call("ccmf_solve");
    if (!plan || !gamma || !xi_bar || gamma_stride < 0) return CCMF_ERR_INVALID_ARG;
    ccmf_params prm;
    if (params)
        prm = *params;
    else
        ccmf_params_default(&prm);
    for (int s = 0; s < plan->batch; ++s) {
        const double* x = xi_bar + 3 * s;
        const double nn = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]) || !(nn > 0.0) || !isfinite(nn))
            return CCMF_ERR_INVALID_ARG;
    }
    if (prm.fixed_iters < 0 || prm.max_iter < 1 || prm.check_every < 1) return CCMF_ERR_INVALID_ARG;
    if (prm.fixed_iters == 0 && !(prm.tol > 0.0)) return CCMF_ERR_INVALID_ARG;
    if (!(prm.delta > 0.0 && prm.delta < 1.0)) return CCMF_ERR_INVALID_ARG;
    if (prm.rho_rule < CCMF_RHO_BB || prm.rho_rule > CCMF_RHO_RB) return CCMF_ERR_INVALID_ARG;
    if (!(prm.rho_step_max >= 1.0) || !isfinite(prm.rho0) || !isfinite(prm.bb_corr_min)) return CCMF_ERR_INVALID_ARG;
    if (prm.history_len < 0 || prm.history_len > kHistCap) return CCMF_ERR_INVALID_ARG;
    if (prm.resume != 0 && prm.resume != 1) return CCMF_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < plan->total) return CCMF_ERR_WORKSPACE;
    if (((uintptr_t)workspace & 255u) != 0) return CCMF_ERR_WORKSPACE;
    if (cudaSetDevice(plan->device) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = reinterpret_cast<unsigned char*>(workspace);
    if (plan->prec == CCMF_FP64)
        return solve_impl<double>(plan, gamma, gamma_stride, xi_bar, &prm, ws, flow, cut, results, st);
    return solve_impl<float>(plan, gamma, gamma_stride, xi_bar, &prm, ws, flow, cut, results, st);
}

int ccmf_state_export(const ccmf_plan* plan, const void* workspace, void* e, void* v, double* rho, int* iters,
                      void* stream) {
    if (!plan || !workspace) return CCMF_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const unsigned char* ws = reinterpret_cast<const unsigned char*>(workspace);
    std::vector<SolveScalars> sc(plan->batch);
    if (cudaMemcpyAsync(sc.data(), ws + plan->off_sc, sizeof(SolveScalars) * plan->batch, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CCMF_ERR_CUDA;
    // the current copy of solve s is (iters & 1)
    const size_t one = plan->esize * 6 * (size_t)plan->g.N;
    const size_t copy = one * plan->batch;
    for (int s = 0; s < plan->batch; ++s) {
        const size_t src = (size_t)(sc[s].iters & 1) * copy + (size_t)s * one;
        if (e && cudaMemcpyAsync((unsigned char*)e + (size_t)s * one, ws + plan->off_e + src, one, cudaMemcpyDefault,
                                 st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        if (v && cudaMemcpyAsync((unsigned char*)v + (size_t)s * one, ws + plan->off_v + src, one, cudaMemcpyDefault,
                                 st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        if (rho) rho[s] = sc[s].rho;
        if (iters) iters[s] = sc[s].iters;
    }
    return cuda_status(cudaStreamSynchronize(st));
}

int ccmf_state_import(const ccmf_plan* plan, void* workspace, const void* e, const void* v, const double* rho,
                      const int* iters, void* stream) {
    if (!plan || !workspace || !e || !v || !rho || !iters) return CCMF_ERR_INVALID_ARG;
    for (int s = 0; s < plan->batch; ++s)
        if (!(rho[s] > 0.0) || !isfinite(rho[s]) || iters[s] < 0) return CCMF_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = reinterpret_cast<unsigned char*>(workspace);
    std::vector<SolveScalars> sc(plan->batch);
    if (cudaMemcpyAsync(sc.data(), ws + plan->off_sc, sizeof(SolveScalars) * plan->batch, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CCMF_ERR_CUDA;
    const size_t one = plan->esize * 6 * (size_t)plan->g.N;
    const size_t copy = one * plan->batch;
    for (int s = 0; s < plan->batch; ++s) {
        const size_t dst = (size_t)(iters[s] & 1) * copy + (size_t)s * one;
        if (cudaMemcpyAsync(ws + plan->off_e + dst, (const unsigned char*)e + (size_t)s * one, one, cudaMemcpyDefault,
                            st) != cudaSuccess ||
            cudaMemcpyAsync(ws + plan->off_v + dst, (const unsigned char*)v + (size_t)s * one, one, cudaMemcpyDefault,
                            st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        sc[s].rho = rho[s];
        sc[s].iters = iters[s];
        sc[s].ab_iter = -1;   // stored divergences are recomputed from the imported state
    }
    if (cudaMemcpyAsync(ws + plan->off_sc, sc.data(), sizeof(SolveScalars) * plan->batch, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(st));
}

int ccmf_history_export(const ccmf_plan* plan, const void* workspace, double* out, int max_entries, int* count,
                        void* stream) {
    if (!plan || !workspace || !out || max_entries < 1 || !count) return CCMF_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const unsigned char* ws = reinterpret_cast<const unsigned char*>(workspace);
    std::vector<SolveScalars> sc(plan->batch);
    std::vector<double> hist((size_t)plan->batch * kHistCap * kHistFields);
    if (cudaMemcpyAsync(sc.data(), ws + plan->off_sc, sizeof(SolveScalars) * plan->batch, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(hist.data(), ws + plan->off_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CCMF_ERR_CUDA;
    // history_len of the last solve is not stored; entries carry their own k.
    int written = 0;
    for (int s = 0; s < plan->batch; ++s) {
        const double* hs = hist.data() + (size_t)s * kHistCap * kHistFields;
        const int iters = sc[s].iters;
        // collect entries with k in [iters - max_entries, iters), oldest first
        std::vector<const double*> rows;
        for (int t = 0; t < kHistCap; ++t) {
            const double* r = hs + (size_t)t * kHistFields;
            const double k = r[0];
            if (k >= 0.0 && k < iters && k >= (double)(iters - max_entries) && k == floor(k)) rows.push_back(r);
        }
        std::sort(rows.begin(), rows.end(), [](const double* a, const double* b) { return a[0] < b[0]; });
        int n = 0;
        double* dst = out + (size_t)s * max_entries * kHistFields;
        for (size_t a = 0; a < rows.size() && n < max_entries; ++a) {
            if (n > 0 && dst[(size_t)(n - 1) * kHistFields] == rows[a][0]) continue;
            memcpy(dst + (size_t)n * kHistFields, rows[a], kHistFields * sizeof(double));
            ++n;
        }
        written = n > written ? n : written;
    }
    *count = written;
    return CCMF_OK;
}

int ccmf_plan_get_tuning(const ccmf_plan* plan, ccmf_tuning* out) {
    if (!plan || !out) return CCMF_ERR_INVALID_ARG;
    *out = plan->tune;
    return CCMF_OK;
}

int ccmf_plan_set_tuning(ccmf_plan* plan, const ccmf_tuning* tuning) {
    if (!plan || !tuning) return CCMF_ERR_INVALID_ARG;
    const ccmf_tuning keep = plan->tune;
    const int rc = apply_tuning(plan, *tuning);
    if (rc != CCMF_OK && apply_tuning(plan, keep) != CCMF_OK) return CCMF_ERR_CUDA;
    return rc;
}

int ccmf_plan_autotune(ccmf_plan* plan, const void* gamma, long long gamma_stride, const double* xi_bar,
                       void* workspace, size_t workspace_bytes, int iters, ccmf_tuning* best, double* best_ms,
                       void* stream) {
    NvtxRange nvtx_call("ccmf_plan_autotune");
    if (!plan || !gamma || !xi_bar || gamma_stride < 0 || iters < 1 || iters > 1000) return CCMF_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < plan->total) return CCMF_ERR_WORKSPACE;
    if (cudaSetDevice(plan->device) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ccmf_params prm;
    ccmf_params_default(&prm);
    prm.fixed_iters = iters;
    prm.check_every = iters;
    prm.resume = 1;
    prm.history_len = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return CCMF_ERR_CUDA;
    }
    // one untimed run (it also captures the graph of this tuning), then the faster of two timed runs
    auto measure = [&](double* ms) {
        int rc = ccmf_solve(plan, gamma, gamma_stride, xi_bar, &prm, workspace, workspace_bytes, nullptr, nullptr,
                            nullptr, stream);
        if (rc != CCMF_OK) return rc;
        double best_run = 0.0;
        for (int rep = 0; rep < 2; ++rep) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return CCMF_ERR_CUDA;
            rc = ccmf_solve(plan, gamma, gamma_stride, xi_bar, &prm, workspace, workspace_bytes, nullptr, nullptr,
                            nullptr, stream);
            if (rc != CCMF_OK) return rc;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return CCMF_ERR_CUDA;
            float f = 0.f;
            if (cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) return CCMF_ERR_CUDA;
            const double t = (double)f / iters;
            if (rep == 0 || t < best_run) best_run = t;
        }
        *ms = best_run;
        return CCMF_OK;
    };
    double cur_ms = 0.0;
    const int rc = tune_descent(plan, measure, &cur_ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CCMF_OK) return rc;
    tuning_store(plan, plan->tune);
    if (best) *best = plan->tune;
    if (best_ms) *best_ms = cur_ms;
    return CCMF_OK;
}

int ccmf_tuning_export(char* text, size_t capacity, size_t* length) {
    if (!length || (capacity > 0 && !text)) return CCMF_ERR_INVALID_ARG;
    std::string out;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        char line[256];
        for (const auto& kv : g_tune_table) {
            const TuneKey& k = kv.first;
            const ccmf_tuning& t = kv.second;
            snprintf(line, sizeof(line), "ccmf-tuning %d %d %d %d %d %d : %d %d %d %d %d %d %d %d %d %d\n", k.n1,
                     k.n2, k.n3, k.batch, k.prec, k.sms, t.update_variant, t.plane_blocks, t.z_pairs_per_block,
                     t.y_lines_per_block, t.x_lines_per_block, t.branches, t.radix_mode, t.zinv_pairs_per_block,
                     t.line_engine, t.z_engine);
            out += line;
        }
    }
    *length = out.size();
    if (capacity > 0) {
        const size_t n = std::min(capacity - 1, out.size());
        memcpy(text, out.data(), n);
        text[n] = '\0';
    }
    return CCMF_OK;
}

int ccmf_tuning_import(const char* text) {
    if (!text) return CCMF_ERR_INVALID_ARG;
    const char* p = text;
    std::vector<std::pair<TuneKey, ccmf_tuning>> rows;
    while (*p) {
        const char* eol = strchr(p, '\n');
        const size_t len = eol ? (size_t)(eol - p) : strlen(p);
        std::string line(p, len);
        p += len + (eol ? 1 : 0);
        if (line.empty()) continue;
        TuneKey k;
        ccmf_tuning t;
        memset(&t, 0, sizeof(t));
        if (sscanf(line.c_str(), "ccmf-tuning %d %d %d %d %d %d : %d %d %d %d %d %d %d %d %d %d", &k.n1, &k.n2,
                   &k.n3, &k.batch, &k.prec, &k.sms, &t.update_variant, &t.plane_blocks, &t.z_pairs_per_block,
                   &t.y_lines_per_block, &t.x_lines_per_block, &t.branches, &t.radix_mode,
                   &t.zinv_pairs_per_block, &t.line_engine, &t.z_engine) != 16)
            return CCMF_ERR_INVALID_ARG;
        rows.emplace_back(k, t);
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& r : rows) g_tune_table[r.first] = r.second;
    return CCMF_OK;
}

int ccmf_plan_launch_info(const ccmf_plan* plan, int* out, int capacity, int* count) {
    if (!plan || !count || (capacity > 0 && !out)) return CCMF_ERR_INVALID_ARG;
    const LaunchShape& sh = plan->sh;
    const int grid_upd = is_abw_variant(sh.upd_variant) ? (int)ceil_div((long long)sh.ab.nq * sh.ab.nr * sh.ab.npass, kAbwWarps)
                         : is_ab_variant(sh.upd_variant) ? sh.ab.nq * sh.ab.nr
                         : (sh.upd_variant == 11 || sh.upd_variant == 12) ? sh.vec_resident_half / std::max(1, plan->batch)
                         : sh.upd_variant >= 2 ? sh.grid_pipe
                         : sh.upd_variant == 1 ? sh.grid_tma
                                               : sh.grid_update;
    const int v[8] = {sh.upd_variant, sh.plane_fused, sh.plane_fused ? sh.plane_cluster : 0, sh.pairs_per_block,
                      sh.lpb_y, sh.lpb_x, grid_upd, plan->branches};
    for (int i = 0; i < 8 && i < capacity; ++i) out[i] = v[i];
    *count = 8;
    return CCMF_OK;
}

int ccmf_kernel_times(const ccmf_plan* plan, double* ms, long long* launches, const char** names, int capacity,
                      int* count) {
    if (!plan || !count) return CCMF_ERR_INVALID_ARG;
    *count = kNumKernelClasses;
    for (int k = 0; k < kNumKernelClasses && k < capacity; ++k) {
        if (ms) ms[k] = plan->kms[k];
        if (launches) launches[k] = plan->klaunch[k];
        if (names) names[k] = kernel_class_name(k);
    }
    return CCMF_OK;
}

int ccmf_set_kernel_timing(ccmf_plan* plan, int enable) {
    if (!plan || (enable != 0 && enable != 1)) return CCMF_ERR_INVALID_ARG;
    plan->timing = enable;
    return CCMF_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of solves on grids of different shapes. Solves are grouped by shape
// into sub-plans (buckets); every bucket keeps its state in its own slice of the
// workspace, and one captured CUDA graph runs the iteration chains of all
// buckets (and of the solve branches inside each bucket) as independent
// branches, so that short and long passes of different grids fill the GPU
// together. The graph's executor plays the role of the work queue: no kernel
// waits on another.
// ---------------------------------------------------------------------------
struct ccmf_batch {
    int count, prec;
    std::vector<ccmf_plan*> plans;           // one per distinct shape
    std::vector<std::vector<int>> members;   // original solve indices of each bucket
    std::vector<size_t> ws_off;              // offset of each bucket's workspace slice
    std::vector<size_t> gp_off;              // offset of each bucket's gamma pointer table
    size_t total;
    cudaStream_t cap_stream;
    cudaEvent_t fork_event;
    std::vector<cudaEvent_t> join_events;
    cudaGraphExec_t gexec;
    bool have_graph;
    GraphKey gkey;
    int* h_active;                           // pinned, one counter per bucket
    // the persistent launch (ccmf_batch_set_persistent): its tables in the workspace
    int persistent;                          // 1: one k_batch_persist launch per iteration
    size_t pers_groups_off, pers_map_off, pers_base_off, pers_done_off, pers_part_off;
    std::vector<size_t> pers_part_b;         // each bucket's chunk partial slots (from pers_part_off)
};

namespace {

void batch_free(ccmf_batch* b) {
    if (!b) return;
    if (b->have_graph) cudaGraphExecDestroy(b->gexec);
    for (ccmf_plan* pl : b->plans) ccmf_plan_destroy(pl);
    for (cudaEvent_t ev : b->join_events) cudaEventDestroy(ev);
    if (b->fork_event) cudaEventDestroy(b->fork_event);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->h_active) cudaFreeHost(b->h_active);
    delete b;
}

// The persistent launch of a batch: uploads the work-queue tables (group descriptors,
// solve map, first item of every (pass, solve)) into the workspace and, when the key
// changed, captures the loop graph: per iteration one memset of the queue counters and one
// k_batch_persist launch over every solve of every shape group.
template <typename T>
int batch_persist_capture(ccmf_batch* bt, const std::vector<Ctx<T>>& ctx, unsigned char* ws, bool aligned,
                          const GraphKey& key, const LoopConfig& cfg, cudaStream_t st) {
    const int nb = (int)bt->plans.size();
    const int ns = bt->count;
    // tile shapes: the wider tiles unless some group's axis is too long for them. Dynamic shared
    // memory: the queue tables, the twiddle table of the longest axis, the largest tile buffers.
    int maxn = 1;
    for (ccmf_plan* pl : bt->plans) maxn = std::max(maxn, std::max(pl->n1, std::max(pl->n2, pl->n3)));
    const size_t tw_off = persist_table_bytes(nb);
    const size_t work_off = tw_off + align_up(sizeof(cx<T>) * (size_t)maxn, 16);
    size_t smem = 0;
    int variant = 0;
    for (int pass = 0; pass < 2; ++pass) {
        variant = pass;
        size_t wmax = 0;
        for (ccmf_plan* pl : bt->plans)
            wmax = std::max(wmax, persist_work_bytes<T>(pl->n1, pl->n2, pl->n3, kPersistTiles[variant][0],
                                                        kPersistTiles[variant][1]));
        smem = work_off + wmax;
        if (smem <= 110 * 1024) break;
    }
    if (smem > 220 * 1024) return CCMF_ERR_UNSUPPORTED_SIZE;
    const int P = kPersistTiles[variant][0], L = kPersistTiles[variant][1];
    std::vector<PersistGroup<T>> groups(nb);
    std::vector<int> gstart(nb);
    int first = 0;
    for (int b = 0; b < nb; ++b) {
        ccmf_plan* pl = bt->plans[b];
        const Ctx<T>& c = ctx[b];
        PersistGroup<T>& G = groups[b];
        memset(&G, 0, sizeof(G));
        G.g = c.g;
        G.p = c.p;
        G.p.s0 = 0;
        G.p.run_all = 0;
        G.p.partial = reinterpret_cast<double*>(ws + bt->pers_part_off + bt->pers_part_b[b]);
        for (int a = 0; a < 3; ++a) {
            G.ax[a] = c.ax[a];
            G.tw[a] = c.tw[a];
        }
        G.rsym_x = c.rsym[0];
        G.rsym_y = c.rsym[1];
        G.sym_z = c.sym[2];
        G.div_l = make_fastdiv((unsigned)L);
        G.inv_n = (T)(1.0 / (double)c.g.N);
        G.vec_div = c.vec_div ? 1 : 0;
        G.upd_w = (sizeof(T) == 4 && aligned && pl->n3 % 2 == 0) ? 2 : 1;
        G.nchunks = vec_update_chunks(c.g.N, G.upd_w);
        const long long pairs = ceil_div((long long)pl->n1 * pl->n2, 2);
        G.tiles[0] = (int)ceil_div(pairs, P);
        G.tiles[1] = (int)ceil_div((long long)pl->n3h * pl->n1, L);
        G.tiles[2] = (int)ceil_div((long long)pl->n3h * pl->n2, L);
        G.tiles[3] = G.tiles[1];
        G.tiles[4] = G.tiles[0];
        G.tiles[5] = (int)G.nchunks;
        // bytes one tile of each pass moves (FP32 fields; FP64 doubles them): items of about
        // 256 KB keep the per-item cost (ticket, barriers, release) small against the tile work
        const double es = (double)sizeof(T) / 4.0;
        const double tile_bytes[kPersistPasses] = {2.0 * P * pl->n3 * 52.0 * es, (double)L * pl->n2 * 16.0 * es,
                                                   (double)L * pl->n1 * 16.0 * es, (double)L * pl->n2 * 16.0 * es,
                                                   2.0 * P * pl->n3 * 8.0 * es, 1.0};
        for (int q = 0; q < kPersistPasses; ++q)
            G.tpi[q] = q == kPersistPasses - 1 ? 1 : std::max(1, (int)(256.0 * 1024.0 / tile_bytes[q]));
        gstart[b] = first;   // solves are numbered group by group (the done counters' index j)
        first += pl->batch;
    }
    const int per_sm = batch_persist_blocks_per_sm<T>(variant, smem);
    if (per_sm < 1) return CCMF_ERR_UNSUPPORTED_SIZE;
    const int grid = per_sm * bt->plans[0]->sms;
    for (int q = 0; q < kPersistPasses; ++q) {
        long long tiles = 0;
        for (int b = 0; b < nb; ++b) tiles += (long long)groups[b].tiles[q] * bt->plans[b]->batch;
        const int cap = (int)std::max<long long>(1, tiles / (4ll * grid));
        for (int b = 0; b < nb; ++b) {
            PersistGroup<T>& G = groups[b];
            G.tpi[q] = std::min(G.tpi[q], cap);
            G.ntiles[q] = (int)ceil_div(G.tiles[q], G.tpi[q]);
        }
    }
    // first queue item of every (pass, group), pass-major; inside (pass, group) the group's
    // solves follow one another with ntiles items each
    std::vector<long long> pg_base((size_t)kPersistPasses * nb + 1);
    long long acc = 0;
    for (int pass = 0; pass < kPersistPasses; ++pass)
        for (int b = 0; b < nb; ++b) {
            pg_base[(size_t)pass * nb + b] = acc;
            acc += (long long)groups[b].ntiles[pass] * bt->plans[b]->batch;
        }
    pg_base[(size_t)kPersistPasses * nb] = acc;
    if (acc >= (1ll << 32) - (1ll << 24)) return CCMF_ERR_UNSUPPORTED_SIZE;   // the 32-bit ticket
    if (cudaMemcpyAsync(ws + bt->pers_groups_off, groups.data(), sizeof(PersistGroup<T>) * nb, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(ws + bt->pers_map_off, gstart.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(ws + bt->pers_base_off, pg_base.data(), sizeof(long long) * pg_base.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    if (bt->have_graph && memcmp(&bt->gkey, &key, sizeof(key)) == 0) return CCMF_OK;
    if (bt->have_graph) cudaGraphExecDestroy(bt->gexec);
    bt->have_graph = false;
    PersistArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.groups = reinterpret_cast<const PersistGroup<T>*>(ws + bt->pers_groups_off);
    a.pg_base = reinterpret_cast<const long long*>(ws + bt->pers_base_off);
    a.gstart = reinterpret_cast<const int*>(ws + bt->pers_map_off);
    a.done = reinterpret_cast<unsigned*>(ws + bt->pers_done_off);
    a.head = a.done + (size_t)ns * kPersistPasses;
    a.ngroups = nb;
    a.nsolve = ns;
    a.tw_off = (int)tw_off;
    a.work_off = (int)work_off;
    a.cfg = cfg;
    const size_t counters = sizeof(unsigned) * ((size_t)ns * kPersistPasses + 1);
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CCMF_ERR_CUDA;
    for (int it = 0; it < key.chunk; ++it) {
        cudaMemsetAsync(a.done, 0, counters, bt->cap_stream);
        launch_batch_persist<T>(a, variant, grid, smem, bt->cap_stream);
    }
    cudaError_t err = cudaStreamEndCapture(bt->cap_stream, &graph);
    if (err != cudaSuccess) return CCMF_ERR_CUDA;
    err = cudaGraphInstantiate(&bt->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) return CCMF_ERR_CUDA;
    bt->gkey = key;
    bt->have_graph = true;
    return CCMF_OK;
}

template <typename T>
int batch_solve_impl(ccmf_batch* bt, const void* const* gammas, const double* xi_host, const ccmf_params* prm,
                     unsigned char* ws, ccmf_result* results, cudaStream_t st) {
    const int nb = (int)bt->plans.size();
    LoopConfig cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.tol = prm->tol;
    cfg.delta = prm->delta;
    cfg.rho0 = prm->rho0;
    cfg.bb_corr_min = prm->bb_corr_min;
    cfg.rho_step_max = prm->rho_step_max;
    cfg.max_iter = prm->max_iter;
    cfg.fixed_iters = prm->fixed_iters;
    cfg.rho_rule = prm->rho_rule;
    cfg.hist_len = prm->history_len;
    cfg.resume = 0;
    {
        const char* env = getenv("CCMF_DEBUG_SPIN_LIMIT");
        cfg.spin_limit = env ? (unsigned)strtoul(env, nullptr, 10) + 1u : 0u;
    }
    std::vector<Ctx<T>> ctx(nb);
    bool aligned = true;
    for (int b = 0; b < nb; ++b) {
        ccmf_plan* pl = bt->plans[b];
        unsigned char* wsb = ws + bt->ws_off[b];
        const std::vector<int>& mem = bt->members[b];
        std::vector<double> xi(3 * mem.size());
        std::vector<const void*> gp(mem.size());
        for (size_t q = 0; q < mem.size(); ++q) {
            const double* x = xi_host + 3 * mem[q];
            const double nn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            for (int a = 0; a < 3; ++a) xi[3 * q + a] = x[a] / nn;
            gp[q] = gammas[mem[q]];
            aligned = aligned && ((uintptr_t)gp[q] % 16) == 0;
        }
        if (cudaMemcpyAsync(wsb + pl->off_xi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(ws + bt->gp_off[b], gp.data(), gp.size() * sizeof(void*), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemsetAsync(wsb + pl->off_nact, 0, sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(wsb + pl->off_hist, 0xFF,
                            sizeof(double) * kHistFields * (size_t)kHistCap * pl->batch, st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        ctx[b] = make_ctx<T>(pl, wsb, nullptr, 0, cfg);
        ctx[b].p.gptrs = reinterpret_cast<const T* const*>(ws + bt->gp_off[b]);
    }
    for (int b = 0; b < nb; ++b) {
        ctx[b].vec_update = ctx[b].vec_div && aligned;
        launch_init<T>(ctx[b], st);
    }
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;

    const bool fixed = prm->fixed_iters > 0;
    const int total = fixed ? prm->fixed_iters : prm->max_iter;
    const int chunk = prm->check_every < total ? prm->check_every : total;
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.chunk = chunk;
    key.timed = (bt->persistent ? 4 : 2) + (aligned ? 0 : 1);   // launch mode and the alignment assumed
    key.ws = ws;
    key.cfg = cfg;
    if (bt->persistent) {
        const int rc = batch_persist_capture<T>(bt, ctx, ws, aligned, key, cfg, st);
        if (rc != CCMF_OK) return rc;
    } else if (!(bt->have_graph && memcmp(&bt->gkey, &key, sizeof(key)) == 0)) {
        if (bt->have_graph) cudaGraphExecDestroy(bt->gexec);
        bt->have_graph = false;
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return CCMF_ERR_CUDA;
        cudaEventRecord(bt->fork_event, bt->cap_stream);
        int ev = 0;
        for (int b = 0; b < nb; ++b) {
            ccmf_plan* pl = bt->plans[b];
            const int nbr = pl->branches;
            for (int r = 0; r < nbr; ++r) {
                const int s0 = (int)((long long)pl->batch * r / nbr), s1 = (int)((long long)pl->batch * (r + 1) / nbr);
                cudaStreamWaitEvent(pl->branch_stream[r], bt->fork_event, 0);
                for (int it = 0; it < chunk; ++it) launch_iteration_range<T>(ctx[b], s0, s1 - s0, pl->branch_stream[r]);
                cudaEventRecord(bt->join_events[ev], pl->branch_stream[r]);
                cudaStreamWaitEvent(bt->cap_stream, bt->join_events[ev], 0);
                ++ev;
            }
        }
        cudaError_t err = cudaStreamEndCapture(bt->cap_stream, &graph);
        if (err != cudaSuccess) return CCMF_ERR_CUDA;
        err = cudaGraphInstantiate(&bt->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess) return CCMF_ERR_CUDA;
        bt->gkey = key;
        bt->have_graph = true;
    }
    const long long nchunks = ((long long)total + chunk - 1) / chunk;
    for (long long ch = 0; ch < nchunks; ++ch) {
        if (cudaGraphLaunch(bt->gexec, st) != cudaSuccess) return CCMF_ERR_CUDA;
        if (!fixed) {
            for (int b = 0; b < nb; ++b)
                if (cudaMemcpyAsync(bt->h_active + b, ws + bt->ws_off[b] + bt->plans[b]->off_nact, sizeof(int),
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    return CCMF_ERR_CUDA;
            if (cudaStreamSynchronize(st) != cudaSuccess) return CCMF_ERR_CUDA;
            int act = 0;
            for (int b = 0; b < nb; ++b) act += bt->h_active[b];
            if (act <= 0) break;
        }
    }
    for (int b = 0; b < nb; ++b) launch_final<T>(ctx[b], st, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
    if (results) {
        for (int b = 0; b < nb; ++b) {
            ccmf_plan* pl = bt->plans[b];
            std::vector<SolveScalars> sc(pl->batch);
            if (cudaMemcpyAsync(sc.data(), ws + bt->ws_off[b] + pl->off_sc, sizeof(SolveScalars) * pl->batch,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return CCMF_ERR_CUDA;
            for (int q = 0; q < pl->batch; ++q) {
                ccmf_result& r = results[bt->members[b][q]];
                r.gamma_eff = sc[q].dual;
                r.gamma_primal = sc[q].primal;
                r.gamma_dual = sc[q].dual;
                r.residual = sc[q].residual;
                r.mean_v_norm = sc[q].mean_v;
                r.rho = sc[q].rho;
                r.iters = sc[q].iters;
                r.converged = sc[q].converged;
                r.status = sc[q].status;
                r.reserved = 0;
            }
        }
    }
    return CCMF_OK;
}


// Times `iters` iterations of bucket b's solves alone (a captured graph of its
// branches, on the solves' current state), the faster of two runs.
template <typename T>
int batch_time_bucket(ccmf_batch* bt, int b, unsigned char* ws, bool aligned, int iters, cudaStream_t st,
                      cudaEvent_t e0, cudaEvent_t e1, double* ms) {
    ccmf_plan* pl = bt->plans[b];
    unsigned char* wsb = ws + bt->ws_off[b];
    LoopConfig cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.tol = 1e-4;
    cfg.delta = 0.25;
    cfg.bb_corr_min = 0.2;
    cfg.rho_step_max = 2.0;
    cfg.max_iter = 1 << 30;
    cfg.fixed_iters = 1 << 30;   // the solves stay active for the timing
    cfg.resume = 1;
    Ctx<T> c = make_ctx<T>(pl, wsb, nullptr, 0, cfg);
    c.p.gptrs = reinterpret_cast<const T* const*>(ws + bt->gp_off[b]);
    c.vec_update = c.vec_div && aligned;
    if (cudaMemsetAsync(wsb + pl->off_nact, 0, sizeof(int), st) != cudaSuccess) return CCMF_ERR_CUDA;
    launch_init<T>(c, st);   // resume: re-activates the solves without touching their state
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaEventRecord(bt->fork_event, bt->cap_stream);
    const int nbr = pl->branches;
    for (int r = 0; r < nbr; ++r) {
        const int s0 = (int)((long long)pl->batch * r / nbr), s1 = (int)((long long)pl->batch * (r + 1) / nbr);
        cudaStreamWaitEvent(pl->branch_stream[r], bt->fork_event, 0);
        for (int it = 0; it < iters; ++it) launch_iteration_range<T>(c, s0, s1 - s0, pl->branch_stream[r]);
        cudaEventRecord(bt->join_events[r], pl->branch_stream[r]);
        cudaStreamWaitEvent(bt->cap_stream, bt->join_events[r], 0);
    }
    if (cudaStreamEndCapture(bt->cap_stream, &graph) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaGraphExec_t gx;
    const cudaError_t ie = cudaGraphInstantiate(&gx, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return CCMF_ERR_CUDA;
    int rc = CCMF_OK;
    double best = 0.0;
    for (int rep = 0; rep < 3 && rc == CCMF_OK; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess || cudaGraphLaunch(gx, st) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = CCMF_ERR_CUDA;
            break;
        }
        float f = 0.f;
        if (cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) rc = CCMF_ERR_CUDA;
        const double t = (double)f / iters;
        if (rep == 1 || (rep == 2 && t < best)) best = t;   // the first run warms up
    }
    cudaGraphExecDestroy(gx);
    *ms = best;
    return rc;
}

template <typename T>
int batch_autotune_impl(ccmf_batch* bt, const void* const* gammas, const double* xi_host, unsigned char* ws,
                        int iters, double* ms_out, cudaStream_t st) {
    // the solves' state: a short fixed-iteration run of the whole batch
    ccmf_params prm;
    ccmf_params_default(&prm);
    prm.fixed_iters = 2;
    prm.check_every = 2;
    prm.history_len = 0;
    int rc = batch_solve_impl<T>(bt, gammas, xi_host, &prm, ws, nullptr, st);
    if (rc != CCMF_OK) return rc;
    bool aligned = true;
    for (int s = 0; s < bt->count; ++s) aligned = aligned && ((uintptr_t)gammas[s] % 16) == 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return CCMF_ERR_CUDA;
    }
    for (int b = 0; b < (int)bt->plans.size() && rc == CCMF_OK; ++b) {
        ccmf_plan* pl = bt->plans[b];
        auto measure = [&](double* ms) { return batch_time_bucket<T>(bt, b, ws, aligned, iters, st, e0, e1, ms); };
        double ms = 0.0;
        rc = tune_descent(pl, measure, &ms);
        if (rc == CCMF_OK) {
            tuning_store(pl, pl->tune);
            if (ms_out) ms_out[b] = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bt->have_graph) cudaGraphExecDestroy(bt->gexec);   // the batch graph is captured again
    bt->have_graph = false;
    return rc;
}

}  // namespace

extern "C" {

int ccmf_batch_create(int count, const int* shapes, int precision, ccmf_batch** out) {
    if (!out) return CCMF_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || !shapes || (precision != CCMF_FP64 && precision != CCMF_FP32_MIXED)) return CCMF_ERR_INVALID_ARG;
    for (int s = 0; s < count; ++s) {
        const int* sh = shapes + 3 * s;
        if (sh[0] < 1 || sh[1] < 1 || sh[2] < 1) return CCMF_ERR_INVALID_ARG;
        AxisPlan ap;
        for (int a = 0; a < 3; ++a)
            if (sh[a] > kMaxN || !make_axis_plan(sh[a], &ap)) return CCMF_ERR_UNSUPPORTED_SIZE;
    }
    ccmf_batch* bt = new (std::nothrow) ccmf_batch();
    if (!bt) return CCMF_ERR_INVALID_ARG;
    bt->count = count;
    bt->prec = precision;
    // buckets of equal shape, in order of first appearance
    std::vector<std::vector<int>> keys;
    for (int s = 0; s < count; ++s) {
        const int* sh = shapes + 3 * s;
        size_t b = 0;
        for (; b < keys.size(); ++b)
            if (keys[b][0] == sh[0] && keys[b][1] == sh[1] && keys[b][2] == sh[2]) break;
        if (b == keys.size()) {
            keys.push_back({sh[0], sh[1], sh[2]});
            bt->members.push_back({});
        }
        bt->members[b].push_back(s);
    }
    int rc = CCMF_OK;
    size_t off = 0;
    for (size_t b = 0; b < keys.size() && rc == CCMF_OK; ++b) {
        ccmf_plan* pl = nullptr;
        rc = ccmf_plan_create(keys[b][0], keys[b][1], keys[b][2], (int)bt->members[b].size(), precision, &pl);
        if (rc != CCMF_OK) break;
        bt->plans.push_back(pl);
        bt->ws_off.push_back(off);
        off = align_up(off + pl->total);
        bt->gp_off.push_back(off);
        off = align_up(off + sizeof(void*) * bt->members[b].size());
    }
    // tables of the persistent launch (sized for either precision) and its chunk partial slots
    // (one per chunk of kVecChunkGroups x kThreads voxels, the narrowest update vectors)
    bt->pers_groups_off = off;
    off = align_up(off + sizeof(PersistGroup<double>) * keys.size());
    bt->pers_map_off = off;
    off = align_up(off + 2 * sizeof(int) * (size_t)count);
    bt->pers_base_off = off;
    off = align_up(off + sizeof(long long) * ((size_t)kPersistPasses * count + 1));
    bt->pers_done_off = off;
    off = align_up(off + sizeof(unsigned) * ((size_t)kPersistPasses * count + 1));
    bt->pers_part_off = off;
    {
        size_t po = 0;
        for (ccmf_plan* pl : bt->plans) {
            bt->pers_part_b.push_back(po);
            po = align_up(po + sizeof(double) * kNSum * (size_t)pl->batch * (size_t)vec_update_chunks(pl->g.N, 1));
        }
        off = align_up(off + po);
    }
    bt->total = off;
    int nev = 0;
    // join events for the largest branch count any tuning of the buckets may choose
    for (ccmf_plan* pl : bt->plans) nev += std::min(kMaxBranches, pl->batch);
    if (rc == CCMF_OK && cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = CCMF_ERR_CUDA;
    if (rc == CCMF_OK && cudaEventCreateWithFlags(&bt->fork_event, cudaEventDisableTiming) != cudaSuccess)
        rc = CCMF_ERR_CUDA;
    for (int e = 0; e < nev && rc == CCMF_OK; ++e) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = CCMF_ERR_CUDA;
        else bt->join_events.push_back(ev);
    }
    if (rc == CCMF_OK && cudaMallocHost((void**)&bt->h_active, sizeof(int) * bt->plans.size()) != cudaSuccess)
        rc = CCMF_ERR_CUDA;
    if (rc != CCMF_OK) {
        batch_free(bt);
        return rc;
    }
    *out = bt;
    return CCMF_OK;
}

int ccmf_batch_destroy(ccmf_batch* batch) {
    batch_free(batch);
    return CCMF_OK;
}

int ccmf_batch_workspace_bytes(const ccmf_batch* batch, size_t* bytes) {
    if (!batch || !bytes) return CCMF_ERR_INVALID_ARG;
    *bytes = batch->total;
    return CCMF_OK;
}

int ccmf_batch_solve(ccmf_batch* batch, const void* const* gammas, const double* xi_bar, const ccmf_params* params,
                     void* workspace, size_t workspace_bytes, ccmf_result* results, void* stream) {
    NvtxRange nvtx_call("ccmf_batch_solve");
    if (!batch || !gammas || !xi_bar) return CCMF_ERR_INVALID_ARG;
    ccmf_params prm;
    if (params)
        prm = *params;
    else
        ccmf_params_default(&prm);
    for (int s = 0; s < batch->count; ++s) {
        const double* x = xi_bar + 3 * s;
        const double nn = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]) || !(nn > 0.0) || !isfinite(nn))
            return CCMF_ERR_INVALID_ARG;
        if (!gammas[s] || !is_device_ptr(gammas[s])) return CCMF_ERR_INVALID_ARG;
    }
    if (prm.fixed_iters < 0 || prm.max_iter < 1 || prm.check_every < 1) return CCMF_ERR_INVALID_ARG;
    if (prm.fixed_iters == 0 && !(prm.tol > 0.0)) return CCMF_ERR_INVALID_ARG;
    if (!(prm.delta > 0.0 && prm.delta < 1.0)) return CCMF_ERR_INVALID_ARG;
    if (prm.rho_rule < CCMF_RHO_BB || prm.rho_rule > CCMF_RHO_RB) return CCMF_ERR_INVALID_ARG;
    if (!(prm.rho_step_max >= 1.0) || !isfinite(prm.rho0) || !isfinite(prm.bb_corr_min)) return CCMF_ERR_INVALID_ARG;
    if (prm.history_len < 0 || prm.history_len > kHistCap) return CCMF_ERR_INVALID_ARG;
    if (prm.resume != 0) return CCMF_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < batch->total || ((uintptr_t)workspace & 255u) != 0)
        return CCMF_ERR_WORKSPACE;
    if (cudaSetDevice(batch->plans[0]->device) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = reinterpret_cast<unsigned char*>(workspace);
    if (batch->prec == CCMF_FP64) return batch_solve_impl<double>(batch, gammas, xi_bar, &prm, ws, results, st);
    return batch_solve_impl<float>(batch, gammas, xi_bar, &prm, ws, results, st);
}

int ccmf_batch_autotune(ccmf_batch* batch, const void* const* gammas, const double* xi_bar, void* workspace,
                        size_t workspace_bytes, int iters, double* ms, void* stream) {
    NvtxRange nvtx_call("ccmf_batch_autotune");
    if (!batch || !gammas || !xi_bar || iters < 1 || iters > 1000) return CCMF_ERR_INVALID_ARG;
    for (int s = 0; s < batch->count; ++s) {
        const double* x = xi_bar + 3 * s;
        const double nn = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (!isfinite(nn) || !(nn > 0.0)) return CCMF_ERR_INVALID_ARG;
        if (!gammas[s] || !is_device_ptr(gammas[s])) return CCMF_ERR_INVALID_ARG;
    }
    if (!workspace || workspace_bytes < batch->total || ((uintptr_t)workspace & 255u) != 0)
        return CCMF_ERR_WORKSPACE;
    if (cudaSetDevice(batch->plans[0]->device) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = reinterpret_cast<unsigned char*>(workspace);
    if (batch->prec == CCMF_FP64) return batch_autotune_impl<double>(batch, gammas, xi_bar, ws, iters, ms, st);
    return batch_autotune_impl<float>(batch, gammas, xi_bar, ws, iters, ms, st);
}

int ccmf_batch_set_persistent(ccmf_batch* batch, int enable) {
    if (!batch || (enable != 0 && enable != 1)) return CCMF_ERR_INVALID_ARG;
    if (batch->persistent != enable) {
        if (batch->have_graph) cudaGraphExecDestroy(batch->gexec);
        batch->have_graph = false;
        batch->persistent = enable;
    }
    return CCMF_OK;
}

int ccmf_batch_buckets(const ccmf_batch* batch, int* buckets) {
    if (!batch || !buckets) return CCMF_ERR_INVALID_ARG;
    *buckets = (int)batch->plans.size();
    return CCMF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Reverse mode: d gamma_eff / d gamma through K replayed updates (see the
// header). The forward replay keeps (e, v) every ckpt_every updates; the
// reverse sweep recomputes each segment from its checkpoint, keeping the
// pre-projection points z^k, and runs the adjoint steps backwards.
// ---------------------------------------------------------------------------
namespace {

struct AdjLayout {
    size_t sched, dummy, ckpt, z, ebar, vbar, zbar, y, my, zero, total;
};

AdjLayout adj_layout(const ccmf_plan* pl, int K, int m) {
    AdjLayout L;
    const size_t f6 = pl->esize * 6 * (size_t)pl->g.N * pl->batch;   // one 6-component field, all solves
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.sched = take(sizeof(double) * (size_t)K * pl->batch);
    L.dummy = take(256 * (size_t)pl->batch);
    L.ckpt = take(2 * f6 * (size_t)((K + m - 1) / m));
    L.z = take(f6 * (size_t)m);
    L.ebar = take(f6);
    L.vbar = take(f6);
    L.zbar = take(f6);
    L.y = take(f6);
    L.my = take(f6);
    L.zero = take(f6);
    L.total = off;
    return L;
}

template <typename T>
int adjoint_impl(ccmf_plan* pl, const T* gamma, long long gstride, const double* xi_host, const ccmf_params* prm,
                 int K, int m, const double* sched_host, unsigned char* ws, unsigned char* aws, T* grad,
                 double* rho_out, ccmf_result* results, cudaStream_t st) {
    const Geom& g = pl->g;
    const int B = pl->batch;
    const AdjLayout L = adj_layout(pl, K, m);
    std::vector<double> sched((size_t)K * B);
    if (sched_host) {
        memcpy(sched.data(), sched_host, sched.size() * sizeof(double));
    } else {
        // record the penalties of an adaptive run of K updates
        ccmf_params rec = *prm;
        rec.fixed_iters = K;
        rec.check_every = K;
        rec.resume = 0;
        rec.history_len = K;
        int rc = solve_impl<T>(pl, gamma, gstride, xi_host, &rec, ws, nullptr, nullptr, nullptr, st);
        if (rc != CCMF_OK) return rc;
        std::vector<double> hist((size_t)B * K * kHistFields);
        int cnt = 0;
        rc = ccmf_history_export(pl, ws, hist.data(), K, &cnt, st);
        if (rc != CCMF_OK) return rc;
        if (cnt != K) return CCMF_ERR_NUMERICAL;
        for (int s = 0; s < B; ++s)
            for (int k = 0; k < K; ++k) sched[(size_t)s * K + k] = hist[((size_t)s * K + k) * kHistFields + 1];
    }
    if (rho_out) memcpy(rho_out, sched.data(), sched.size() * sizeof(double));
    double* dsched = reinterpret_cast<double*>(aws + L.sched);
    if (cudaMemcpyAsync(dsched, sched.data(), sched.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return CCMF_ERR_CUDA;

    // forward replay from e^0, v^0 with checkpoints
    std::vector<double> xi(3 * (size_t)B);
    for (int s = 0; s < B; ++s) {
        const double* x = xi_host + 3 * s;
        const double nn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int a = 0; a < 3; ++a) xi[3 * s + a] = x[a] / nn;
    }
    if (cudaMemcpyAsync(ws + pl->off_xi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(ws + pl->off_nact, 0, sizeof(int), st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    LoopConfig cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.tol = 1.0;
    cfg.delta = prm->delta;
    cfg.rho0 = prm->rho0;
    cfg.bb_corr_min = prm->bb_corr_min;
    cfg.rho_step_max = prm->rho_step_max;
    cfg.max_iter = K;
    cfg.fixed_iters = K;
    cfg.rho_rule = CCMF_RHO_CONST;
    cfg.hist_len = 0;
    cfg.resume = 0;
    cfg.rho_sched = dsched;
    cfg.sched_len = K;
    Ctx<T> c = make_ctx<T>(pl, ws, gamma, gstride, cfg);
    c.vec_update = false;   // the scalar update pass can also emit z
    c.use_ab = false;
    const size_t f6 = (size_t)6 * g.N * B;
    T* ckpt = reinterpret_cast<T*>(aws + L.ckpt);
    T* e_state = reinterpret_cast<T*>(ws + pl->off_e);
    T* v_state = reinterpret_cast<T*>(ws + pl->off_v);
    launch_init<T>(c, st);
    for (int k = 0; k < K; ++k) {
        if (k % m == 0) {
            const size_t cur = (size_t)(k & 1) * f6;
            T* slot = ckpt + (size_t)(k / m) * 2 * f6;
            if (cudaMemcpyAsync(slot, e_state + cur, f6 * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(slot + f6, v_state + cur, f6 * sizeof(T), cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess)
                return CCMF_ERR_CUDA;
        }
        launch_iteration<T>(c, st);
    }
    launch_final<T>(c, st, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
    if (results) {
        std::vector<SolveScalars> sc(B);
        if (cudaMemcpyAsync(sc.data(), ws + pl->off_sc, sizeof(SolveScalars) * B, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        for (int s = 0; s < B; ++s) {
            ccmf_result& r = results[s];
            r.gamma_eff = sc[s].dual;
            r.gamma_primal = sc[s].primal;
            r.gamma_dual = sc[s].dual;
            r.residual = sc[s].residual;
            r.mean_v_norm = sc[s].mean_v;
            r.rho = sc[s].rho;
            r.iters = sc[s].iters;
            r.converged = 0;
            r.status = sc[s].status;
            r.reserved = 0;
        }
    }

    // reverse sweep
    T* zbuf = reinterpret_cast<T*>(aws + L.z);
    T* ebar = reinterpret_cast<T*>(aws + L.ebar);
    T* vbar = reinterpret_cast<T*>(aws + L.vbar);
    T* zbar = reinterpret_cast<T*>(aws + L.zbar);
    T* y = reinterpret_cast<T*>(aws + L.y);
    T* my = reinterpret_cast<T*>(aws + L.my);
    T* zero = reinterpret_cast<T*>(aws + L.zero);
    SolveScalars* dummy = reinterpret_cast<SolveScalars*>(aws + L.dummy);
    if (cudaMemsetAsync(zero, 0, f6 * sizeof(T), st) != cudaSuccess ||
        cudaMemsetAsync(grad, 0, sizeof(T) * (size_t)g.N * B, st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    launch_adj_seed<T>(c, ebar, vbar, dummy, st);
    const int nseg = (K + m - 1) / m;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int k0 = sg * m, k1 = (k0 + m < K) ? k0 + m : K;
        const size_t cur = (size_t)(k0 & 1) * f6;
        T* slot = ckpt + (size_t)sg * 2 * f6;
        if (cudaMemcpyAsync(e_state + cur, slot, f6 * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(v_state + cur, slot + f6, f6 * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        launch_adj_restore<T>(c, k0, dsched, K, st);
        for (int k = k0; k < k1; ++k) {
            Ctx<T> ck = c;
            ck.p.zout = zbuf + (size_t)(k - k0) * f6;
            launch_iteration<T>(ck, st);
        }
        for (int k = k1 - 1; k >= k0; --k)
            launch_adj_step<T>(c, zbuf + (size_t)(k - k0) * f6, ebar, vbar, zbar, y, my, zero, dummy, grad, dsched, K,
                               k, st, nullptr);
        if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
    }
    return CCMF_OK;
}

// Reverse mode of an FP32 plan with the forward and the segment recomputation in FP64
// (the FP64 shadow plan) and the reverse sweep in FP32: the FP32 trajectory takes the
// other branch of P_C at near-tied voxels (|z| close to gamma), so an FP32 forward
// differentiates another piece of the piecewise-smooth map. Here the FP64 forward keeps
// its checkpoints in double; each segment is recomputed in double and every update's
// pre-projection point z^k is rounded to float together with one bit per voxel, the
// branch the FP64 projection took; the FP32 reverse steps take the branches from the bits.
// FP64 forward, FP32 reverse: the pre-projection point z^k of an FP64 update, rounded to
// float, and the branch the FP64 projection took, [|z^k| > gamma] (Eq. 19), one bit per
// voxel. Threads of a warp take 32 consecutive voxels and the warp writes one word.
__global__ void __launch_bounds__(kThreads) k_adj_pack(Geom g, const double* __restrict__ z,
                                                       const double* __restrict__ gamma, long long gstride,
                                                       float* __restrict__ z32, unsigned* __restrict__ bits) {
    const int s = blockIdx.y;
    const long long N = g.N;
    const long long words = (N + 31) / 32;
    const double* zs = z + (size_t)s * 6 * N;
    const double* gs = gamma + (size_t)s * gstride;
    float* zo = z32 + (size_t)s * 6 * N;
    unsigned* bo = bits + (size_t)s * words;
    const long long stride = (long long)gridDim.x * kThreads;   // a multiple of 32
    for (long long lin = (long long)blockIdx.x * kThreads + threadIdx.x; lin < words * 32; lin += stride) {
        bool clip = false;
        if (lin < N) {
            double nz2 = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const double zc = zs[c * N + lin];
                nz2 += zc * zc;
                zo[c * N + lin] = (float)zc;
            }
            clip = sqrt(nz2) > gs[lin];
        }
        const unsigned word = __ballot_sync(0xffffffffu, clip);
        if ((threadIdx.x & 31) == 0) bo[lin >> 5] = word;
    }
}

// A float field widened to double (gamma for the FP64 forward of an FP32 plan).
__global__ void __launch_bounds__(kThreads) k_widen(const float* __restrict__ src, double* __restrict__ dst,
                                                    long long n) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long q = (long long)blockIdx.x * kThreads + threadIdx.x; q < n; q += stride) dst[q] = (double)src[q];
}

// Pack the FP64 pre-projection points of one update into float plus clip bits.
void launch_adj_pack(const Ctx<double>& c, const double* zk, const double* gamma64, long long gstride,
                            float* z32, unsigned* bits, cudaStream_t st) {
    dim3 grid((unsigned)c.sh.grid_update, (unsigned)c.g.batch);
    k_adj_pack<<<grid, kThreads, 0, st>>>(c.g, zk, gamma64, gstride, z32, bits);
}

void launch_widen(const float* src, double* dst, long long n, cudaStream_t st) {
    long long blocks = ceil_div(n, kThreads);
    if (blocks > 4096) blocks = 4096;
    k_widen<<<(unsigned)(blocks < 1 ? 1 : blocks), kThreads, 0, st>>>(src, dst, n);
}

struct AdjLayoutMixed {
    size_t sched, dummy, ws64, gamma64, ckpt, ztmp, z, bits, ebar, vbar, zbar, y, my, zero, total;
};

AdjLayoutMixed adj_layout_mixed(const ccmf_plan* pl, int K, int m) {
    AdjLayoutMixed L;
    const ccmf_plan* p64 = pl->shadow64;
    const size_t N = (size_t)pl->g.N, B = (size_t)pl->batch;
    const size_t f6_32 = 4 * 6 * N * B, f6_64 = 8 * 6 * N * B;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.sched = take(sizeof(double) * (size_t)K * B);
    L.dummy = take(256 * B);
    L.ws64 = take(p64 ? p64->total : 0);
    L.gamma64 = take(8 * N * B);
    L.ckpt = take(2 * f6_64 * (size_t)((K + m - 1) / m));
    L.ztmp = take(f6_64);
    L.z = take(f6_32 * (size_t)m);
    L.bits = take(sizeof(unsigned) * ((N + 31) / 32) * B * (size_t)m);
    L.ebar = take(f6_32);
    L.vbar = take(f6_32);
    L.zbar = take(f6_32);
    L.y = take(f6_32);
    L.my = take(f6_32);
    L.zero = take(f6_32);
    L.total = off;
    return L;
}

int adjoint_mixed_impl(ccmf_plan* pl, const float* gamma, long long gstride, const double* xi_host,
                       const ccmf_params* prm, int K, int m, const double* sched_host, unsigned char* ws,
                       unsigned char* aws, float* grad, double* rho_out, ccmf_result* results, cudaStream_t st) {
    ccmf_plan* p64 = pl->shadow64;
    const Geom& g = pl->g;
    const int B = pl->batch;
    const size_t N = (size_t)g.N;
    const AdjLayoutMixed L = adj_layout_mixed(pl, K, m);
    unsigned char* ws64 = aws + L.ws64;
    double* gam64 = reinterpret_cast<double*>(aws + L.gamma64);
    const size_t gfields = gstride == 0 ? 1 : (size_t)B;
    for (size_t s = 0; s < gfields; ++s) launch_widen(gamma + s * (size_t)gstride, gam64 + s * N, (long long)N, st);
    const long long gstride64 = gstride == 0 ? 0 : (long long)N;

    std::vector<double> sched((size_t)K * B);
    if (sched_host) {
        memcpy(sched.data(), sched_host, sched.size() * sizeof(double));
    } else {
        // the penalties of an adaptive FP64 run of K updates
        ccmf_params rec = *prm;
        rec.fixed_iters = K;
        rec.check_every = K;
        rec.resume = 0;
        rec.history_len = K;
        int rc = solve_impl<double>(p64, gam64, gstride64, xi_host, &rec, ws64, nullptr, nullptr, nullptr, st);
        if (rc != CCMF_OK) return rc;
        std::vector<double> hist((size_t)B * K * kHistFields);
        int cnt = 0;
        rc = ccmf_history_export(p64, ws64, hist.data(), K, &cnt, st);
        if (rc != CCMF_OK) return rc;
        if (cnt != K) return CCMF_ERR_NUMERICAL;
        for (int s = 0; s < B; ++s)
            for (int k = 0; k < K; ++k) sched[(size_t)s * K + k] = hist[((size_t)s * K + k) * kHistFields + 1];
    }
    if (rho_out) memcpy(rho_out, sched.data(), sched.size() * sizeof(double));
    double* dsched = reinterpret_cast<double*>(aws + L.sched);
    if (cudaMemcpyAsync(dsched, sched.data(), sched.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return CCMF_ERR_CUDA;

    std::vector<double> xi(3 * (size_t)B);
    for (int s = 0; s < B; ++s) {
        const double* x = xi_host + 3 * s;
        const double nn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int a = 0; a < 3; ++a) xi[3 * s + a] = x[a] / nn;
    }
    if (cudaMemcpyAsync(ws64 + p64->off_xi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(ws + pl->off_xi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(ws64 + p64->off_nact, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(ws + pl->off_nact, 0, sizeof(int), st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    LoopConfig cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.tol = 1.0;
    cfg.delta = prm->delta;
    cfg.rho0 = prm->rho0;
    cfg.bb_corr_min = prm->bb_corr_min;
    cfg.rho_step_max = prm->rho_step_max;
    cfg.max_iter = K;
    cfg.fixed_iters = K;
    cfg.rho_rule = CCMF_RHO_CONST;
    cfg.hist_len = 0;
    cfg.resume = 0;
    cfg.rho_sched = dsched;
    cfg.sched_len = K;

    // FP64 forward replay with FP64 checkpoints of (e, v)
    Ctx<double> c64 = make_ctx<double>(p64, ws64, gam64, gstride64, cfg);
    c64.vec_update = false;   // the scalar update pass can also emit z
    c64.use_ab = false;
    const size_t f6 = (size_t)6 * N * B;
    double* ckpt = reinterpret_cast<double*>(aws + L.ckpt);
    double* e_state = reinterpret_cast<double*>(ws64 + p64->off_e);
    double* v_state = reinterpret_cast<double*>(ws64 + p64->off_v);
    launch_init<double>(c64, st);
    for (int k = 0; k < K; ++k) {
        if (k % m == 0) {
            const size_t cur = (size_t)(k & 1) * f6;
            double* slot = ckpt + (size_t)(k / m) * 2 * f6;
            if (cudaMemcpyAsync(slot, e_state + cur, f6 * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(slot + f6, v_state + cur, f6 * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess)
                return CCMF_ERR_CUDA;
        }
        launch_iteration<double>(c64, st);
    }
    launch_final<double>(c64, st, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
    if (results) {
        std::vector<SolveScalars> sc(B);
        if (cudaMemcpyAsync(sc.data(), ws64 + p64->off_sc, sizeof(SolveScalars) * B, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CCMF_ERR_CUDA;
        for (int s = 0; s < B; ++s) {
            ccmf_result& r = results[s];
            r.gamma_eff = sc[s].dual;
            r.gamma_primal = sc[s].primal;
            r.gamma_dual = sc[s].dual;
            r.residual = sc[s].residual;
            r.mean_v_norm = sc[s].mean_v;
            r.rho = sc[s].rho;
            r.iters = sc[s].iters;
            r.converged = 0;
            r.status = sc[s].status;
            r.reserved = 0;
        }
    }

    // FP32 reverse sweep; the FP32 context supplies the M applications and the seed
    Ctx<float> c32 = make_ctx<float>(pl, ws, gamma, gstride, cfg);
    c32.use_ab = false;
    launch_init<float>(c32, st);   // unit normals and gamma statistics of the FP32 workspace
    float* zbuf = reinterpret_cast<float*>(aws + L.z);
    unsigned* bits = reinterpret_cast<unsigned*>(aws + L.bits);
    const size_t words = ((N + 31) / 32) * (size_t)B;
    double* ztmp = reinterpret_cast<double*>(aws + L.ztmp);
    float* ebar = reinterpret_cast<float*>(aws + L.ebar);
    float* vbar = reinterpret_cast<float*>(aws + L.vbar);
    float* zbar = reinterpret_cast<float*>(aws + L.zbar);
    float* y = reinterpret_cast<float*>(aws + L.y);
    float* my = reinterpret_cast<float*>(aws + L.my);
    float* zero = reinterpret_cast<float*>(aws + L.zero);
    SolveScalars* dummy = reinterpret_cast<SolveScalars*>(aws + L.dummy);
    if (cudaMemsetAsync(zero, 0, f6 * sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(grad, 0, sizeof(float) * N * B, st) != cudaSuccess)
        return CCMF_ERR_CUDA;
    launch_adj_seed<float>(c32, ebar, vbar, dummy, st);
    const int nseg = (K + m - 1) / m;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int k0 = sg * m, k1 = (k0 + m < K) ? k0 + m : K;
        const size_t cur = (size_t)(k0 & 1) * f6;
        double* slot = ckpt + (size_t)sg * 2 * f6;
        if (cudaMemcpyAsync(e_state + cur, slot, f6 * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(v_state + cur, slot + f6, f6 * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
            return CCMF_ERR_CUDA;
        launch_adj_restore<double>(c64, k0, dsched, K, st);
        for (int k = k0; k < k1; ++k) {
            Ctx<double> ck = c64;
            ck.p.zout = ztmp;
            launch_iteration<double>(ck, st);
            launch_adj_pack(c64, ztmp, gam64, gstride64, zbuf + (size_t)(k - k0) * f6, bits + (size_t)(k - k0) * words,
                            st);
        }
        for (int k = k1 - 1; k >= k0; --k)
            launch_adj_step<float>(c32, zbuf + (size_t)(k - k0) * f6, ebar, vbar, zbar, y, my, zero, dummy, grad,
                                   dsched, K, k, st, bits + (size_t)(k - k0) * words);
        if (cudaGetLastError() != cudaSuccess) return CCMF_ERR_CUDA;
    }
    return CCMF_OK;
}

}  // namespace

extern "C" {

int ccmf_set_adjoint_forward(ccmf_plan* plan, int precision) {
    if (!plan || (precision != CCMF_FP64 && precision != CCMF_FP32_MIXED)) return CCMF_ERR_INVALID_ARG;
    if (plan->prec == CCMF_FP64 && precision != CCMF_FP64) return CCMF_ERR_INVALID_ARG;
    if (plan->prec == CCMF_FP32_MIXED && precision == CCMF_FP64 && !plan->shadow64) {
        if (cudaSetDevice(plan->device) != cudaSuccess) return CCMF_ERR_CUDA;
        ccmf_plan* p64 = nullptr;
        const int rc = ccmf_plan_create(plan->n1, plan->n2, plan->n3, plan->batch, CCMF_FP64, &p64);
        if (rc != CCMF_OK) return rc;
        plan->shadow64 = p64;
    }
    plan->adj_forward = precision;
    return CCMF_OK;
}

int ccmf_adjoint_workspace_bytes(const ccmf_plan* plan, int K, int ckpt_every, size_t* bytes) {
    if (!plan || !bytes || K < 1 || ckpt_every < 1) return CCMF_ERR_INVALID_ARG;
    const bool mixed = plan->prec == CCMF_FP32_MIXED && plan->adj_forward == CCMF_FP64 && plan->shadow64;
    *bytes = mixed ? adj_layout_mixed(plan, K, ckpt_every).total : adj_layout(plan, K, ckpt_every).total;
    return CCMF_OK;
}

int ccmf_adjoint(ccmf_plan* plan, const void* gamma, long long gamma_stride, const double* xi_bar,
                 const ccmf_params* params, int K, int ckpt_every, const double* rho_schedule, void* workspace,
                 size_t workspace_bytes, void* adj_workspace, size_t adj_workspace_bytes, void* grad_gamma,
                 double* rho_out, ccmf_result* results, void* stream) {
    NvtxRange nvtx_call("ccmf_adjoint");
    if (!plan || !gamma || !xi_bar || !grad_gamma || gamma_stride < 0 || K < 1 || ckpt_every < 1)
        return CCMF_ERR_INVALID_ARG;
    if (!rho_schedule && K > kHistCap) return CCMF_ERR_INVALID_ARG;
    ccmf_params prm;
    if (params)
        prm = *params;
    else
        ccmf_params_default(&prm);
    if (!(prm.delta > 0.0 && prm.delta < 1.0) || prm.rho_rule < CCMF_RHO_BB || prm.rho_rule > CCMF_RHO_RB ||
        !(prm.rho_step_max >= 1.0))
        return CCMF_ERR_INVALID_ARG;
    for (int s = 0; s < plan->batch; ++s) {
        const double* x = xi_bar + 3 * s;
        const double nn = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]) || !(nn > 0.0) || !isfinite(nn))
            return CCMF_ERR_INVALID_ARG;
    }
    if (rho_schedule)
        for (size_t q = 0; q < (size_t)K * plan->batch; ++q)
            if (!(rho_schedule[q] > 0.0) || !isfinite(rho_schedule[q])) return CCMF_ERR_INVALID_ARG;
    if (!is_device_ptr(gamma) || !is_device_ptr(grad_gamma)) return CCMF_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < plan->total || ((uintptr_t)workspace & 255u) != 0) return CCMF_ERR_WORKSPACE;
    const bool mixed = plan->prec == CCMF_FP32_MIXED && plan->adj_forward == CCMF_FP64 && plan->shadow64;
    const size_t need = mixed ? adj_layout_mixed(plan, K, ckpt_every).total : adj_layout(plan, K, ckpt_every).total;
    if (!adj_workspace || adj_workspace_bytes < need || ((uintptr_t)adj_workspace & 255u) != 0)
        return CCMF_ERR_WORKSPACE;
    if (cudaSetDevice(plan->device) != cudaSuccess) return CCMF_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = reinterpret_cast<unsigned char*>(workspace);
    unsigned char* aws = reinterpret_cast<unsigned char*>(adj_workspace);
    if (mixed)
        return adjoint_mixed_impl(plan, reinterpret_cast<const float*>(gamma), gamma_stride, xi_bar, &prm, K,
                                  ckpt_every, rho_schedule, ws, aws, reinterpret_cast<float*>(grad_gamma), rho_out,
                                  results, st);
    if (plan->prec == CCMF_FP64)
        return adjoint_impl<double>(plan, reinterpret_cast<const double*>(gamma), gamma_stride, xi_bar, &prm, K,
                                    ckpt_every, rho_schedule, ws, aws, reinterpret_cast<double*>(grad_gamma), rho_out,
                                    results, st);
    return adjoint_impl<float>(plan, reinterpret_cast<const float*>(gamma), gamma_stride, xi_bar, &prm, K, ckpt_every,
                               rho_schedule, ws, aws, reinterpret_cast<float*>(grad_gamma), rho_out, results, st);
}

}  // extern "C"
