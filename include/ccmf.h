/*
 * ccmf.h - C ABI of the GB300 solver for the effective crack energy on a
 * combinatorially consistent grid (CCMF discretisation, FFT-based damped ADMM).
 *
 * Paper: Ernesti & Schneider, "An FFT-based method for computing the effective
 * crack energy of a heterogeneous material on a combinatorially consistent
 * grid", arXiv:2103.05968. Equations are numbered as in the paper.
 *
 * Problem (Sec. 2.2, Sec. 3.1): given crack resistances gamma >= 0 sampled at
 * the voxel centres of a periodic N1 x N2 x N3 grid and a crack normal xi_bar,
 * compute the effective crack energy gamma_eff(xi_bar) as the common value of
 * the CCMF maximum flow (Eq. 12) and the min-cut problem (Eq. 21), by the
 * damped ADMM of Eq. 30 with the convergence criterion of Eq. 31.
 *
 * Memory layout (all arrays C-ordered, z fastest):
 *   gamma : [batch][N1][N2][N3] (or one shared field, batch stride 0)
 *   cut   : [batch][6][N1][N2][N3]  xi^{K+1/2}, the min-cut normal field (Eq. 21)
 *   flow  : [batch][3][N1][N2][N3]  A* v^K, the face flows of Eq. 12
 *           (component a of voxel p is the flow on face p + e_a / 2, Sec. 2.2)
 *   state : e and v, each [batch][6][N1][N2][N3] (the split variable and the
 *           multiplier of Eq. 24 / Eq. 30)
 * Element type: double for CCMF_FP64 plans, float for CCMF_FP32_MIXED plans
 * (the latter keep all global reductions and the penalty logic in double).
 *
 * Ownership: the caller owns every buffer. The library allocates only small
 * constant tables inside the plan (plan_create) and never frees caller memory.
 * Device pointers must come from the CUDA device that was current at
 * plan_create. Where noted, a pointer may also be ordinary host memory; the
 * library then stages it through the workspace and the call synchronises the
 * stream before returning.
 *
 * Errors: every call returns a status code (CCMF_OK = 0); nothing throws.
 * Non-convergence within max_iter is not an error (result.converged = 0).
 * Per-solve device-side failures (invalid gamma, non-finite reductions) are
 * reported in ccmf_result.status.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream). Calls enqueue work on it; the calls that return host results
 * synchronise it.
 */
#ifndef CCMF_H
#define CCMF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CCMF_OK 0
#define CCMF_ERR_INVALID_ARG 1      /* bad pointer, size, normal, tolerance, damping, rule */
#define CCMF_ERR_UNSUPPORTED_SIZE 2 /* an N_i with a prime factor other than 2, 3, 5, or N_i > 1024 */
#define CCMF_ERR_WORKSPACE 3        /* workspace missing or smaller than ccmf_plan_workspace_bytes */
#define CCMF_ERR_CUDA 4             /* a CUDA runtime call failed */
#define CCMF_ERR_NUMERICAL 5        /* gamma < 0 or non-finite, or a non-finite reduction */
#define CCMF_ERR_TIMEOUT 6          /* a bounded device-side wait gave up */

/* Precision of a plan. */
#define CCMF_FP64 0        /* every field, FFT and reduction in double */
#define CCMF_FP32_MIXED 1  /* fields and FFTs in float, reductions and penalty logic in double */

/* Penalty rules (text after Eq. 30). */
#define CCMF_RHO_BB 0     /* Barzilai-Borwein scaling with safeguard (default, Sec. 4.1) */
#define CCMF_RHO_CONST 1  /* constant rho (Sec. 4.2, Sec. 4.3: the lower bound min gamma) */
#define CCMF_RHO_LTD 2    /* Lorenz-Tran-Dinh scaling |v| / |e| */
#define CCMF_RHO_RB 3     /* residual balancing (compared in Sec. 4.3): rho * s if the primal residual
                             |e^k - xi^{k+1/2}| exceeds 10 x the dual residual rho |e^{k+1} - e^k|,
                             rho / s in the opposite case, s = rho_step_max */

typedef struct ccmf_plan ccmf_plan;

/* ADMM parameters (Eq. 30, Eq. 31, Sec. 4.1). */
typedef struct {
    double tol;          /* Eq. 31: stop once |e^k - xi^{k+1/2}|_L2 <= tol |<v^k>| (k >= 1); default 1e-4 */
    double delta;        /* damping of Eq. 30, in (0, 1); default 0.25 */
    double rho0;         /* initial penalty; <= 0 selects min(gamma) if positive, else mean(gamma) */
    double bb_corr_min;  /* BB safeguard: minimum correlation <dv,de>/(|dv||de|); default 0.2 */
    double rho_step_max; /* BB/LTD safeguard: rho changes by at most this factor per iteration; default 2 */
    int max_iter;        /* upper bound on ADMM updates; default 20000 */
    int rho_rule;        /* CCMF_RHO_BB (default), CCMF_RHO_CONST, CCMF_RHO_LTD or CCMF_RHO_RB */
    int fixed_iters;     /* > 0: run exactly this many updates and ignore tol; default 0 */
    int check_every;     /* updates per device-side loop chunk between host checks; default 32 */
    int resume;          /* 1: start from the state already in the workspace instead of e^0, v^0 */
    int history_len;     /* entries of the per-solve history ring kept in the workspace (<= 4096); default 1024 */
} ccmf_params;

/* Per-solve result (Eq. 21, Eq. 12, Eq. 31), evaluated on the final state. */
typedef struct {
    double gamma_eff;     /* reported effective crack energy = gamma_dual, the objective of the CCMF
                             maximum-flow problem (Eq. 8 / Eq. 12) that defines the discretisation */
    double gamma_primal;  /* mean(gamma |xi^{K+1/2}|), the min-cut objective of Eq. 21 */
    double gamma_dual;    /* <xi_bar, A* v^K>, the max-flow objective of Eq. 12 */
    double residual;      /* |e^K - xi^{K+1/2}|_L2 */
    double mean_v_norm;   /* |<v^K>| (right-hand side of Eq. 31 without tol) */
    double rho;           /* final penalty rho^K */
    int iters;            /* ADMM updates performed (K) */
    int converged;        /* 1 if Eq. 31 held */
    int status;           /* CCMF_OK or CCMF_ERR_NUMERICAL / CCMF_ERR_INVALID_ARG for this solve */
    int reserved;
} ccmf_result;

/* Fill *p with the defaults listed above. */
void ccmf_params_default(ccmf_params* p);

/* Human-readable text of a status code (static storage). */
const char* ccmf_status_string(int status);

/*
 * Create a plan for `batch` independent solves on one n1 x n2 x n3 grid
 * (Sec. 2.2: periodic grid, z fastest) in the given precision. Each N_i must be
 * 1..1024 with prime factors 2, 3, 5 only (CCMF_ERR_UNSUPPORTED_SIZE otherwise);
 * batch >= 1. Builds the FFT schedules and uploads twiddle and Laplacian-symbol
 * tables (Eq. 28: div^- grad^+ has the symbol -sum_a 4 sin^2(pi k_a / N_a)) to
 * the current device. *out receives the plan; free it with ccmf_plan_destroy.
 */
int ccmf_plan_create(int n1, int n2, int n3, int batch, int precision, ccmf_plan** out);

/* Release a plan and its tables (NULL is accepted). */
int ccmf_plan_destroy(ccmf_plan* plan);

/* Bytes of device workspace a solve with this plan needs (state, spectra,
 * reduction partials, history, host-I/O staging). */
int ccmf_plan_workspace_bytes(const ccmf_plan* plan, size_t* bytes);

/*
 * Run the damped ADMM of Eq. 30 for every solve of the plan.
 *   gamma        : crack resistances, device or host memory (element type of the plan)
 *   gamma_stride : elements between consecutive solves' gamma fields (0 = all share one field)
 *   xi_bar       : host array [batch][3], crack normals; normalised internally
 *                  (gamma_eff is 1-homogeneous in xi_bar, Eq. 3); zero or non-finite -> INVALID_ARG
 *   params       : ADMM parameters (NULL = defaults)
 *   workspace    : device memory of at least ccmf_plan_workspace_bytes bytes, 256-byte aligned
 *   flow, cut    : optional outputs (NULL to skip), device or host memory
 *   results      : optional host array [batch]; when given, the call synchronises the stream
 * The loop runs on the device; the host only relaunches a captured CUDA graph
 * of params->check_every updates and reads one counter between chunks (no
 * host round trip in fixed_iters mode).
 * Every reduction sums in a fixed order (per block or per work chunk, then by the
 * last block in index order), so repeated solves with the same plan, tuning and
 * inputs give bit-identical results, whatever the order the blocks ran in.
 */
int ccmf_solve(ccmf_plan* plan, const void* gamma, long long gamma_stride, const double* xi_bar,
               const ccmf_params* params, void* workspace, size_t workspace_bytes,
               void* flow, void* cut, ccmf_result* results, void* stream);

/*
 * Copy the ADMM state of the workspace out (checkpoint): e and v ([batch][6][N]
 * each, device or host memory, may be NULL), and per solve the penalty rho and
 * the number of updates performed (host arrays [batch], may be NULL).
 * Synchronises the stream.
 */
int ccmf_state_export(const ccmf_plan* plan, const void* workspace, void* e, void* v,
                      double* rho, int* iters, void* stream);

/*
 * Load an ADMM state into the workspace (resume): e, v as in ccmf_state_export,
 * rho and iters host arrays [batch]. A following ccmf_solve with params->resume = 1
 * continues from it bit for bit. Synchronises the stream.
 */
int ccmf_state_import(const ccmf_plan* plan, void* workspace, const void* e, const void* v,
                      const double* rho, const int* iters, void* stream);

/*
 * Copy the per-solve history ring to host memory: out[batch][max_entries][6]
 * with (k, rho^k, |e^k - xi^{k+1/2}|_L2, |<v^k>|, mean(gamma |xi^{k+1/2}|),
 * <xi_bar, mean A* v^k>) -- the last two are the min-cut (Eq. 21) and max-flow
 * (Eq. 12) values at iteration k -- for
 * the most recent min(max_entries, history_len, iterations) updates, oldest
 * first; *count receives the number of entries written per solve.
 * Synchronises the stream.
 */
int ccmf_history_export(const ccmf_plan* plan, const void* workspace, double* out, int max_entries,
                        int* count, void* stream);

/*
 * Per-kernel device time of the most recent ccmf_solve that ran with
 * ccmf_set_kernel_timing(plan, 1): ms[i] = total milliseconds spent in kernel
 * class i over the ADMM loop, launches[i] = number of launches; names[i]
 * points to a static string. Returns the number of kernel classes in *count.
 */
int ccmf_kernel_times(const ccmf_plan* plan, double* ms, long long* launches, const char** names,
                      int capacity, int* count);

/*
 * Launch shape the plan chose, for tests and reports: out[0..7] = {update-pass
 * variant (0 registers, 1 TMA rows, 2..7 pipelined TMA, 8..10 and 13..15 stored divergences, 11, 12
 * narrower registers),
 * plane pass fused (0 / 1),
 * blocks sharing one (x, y) plane (1 = one block, 2..16 = a thread-block cluster),
 * z-pass line pairs per block, y-pass lines per block, x-pass lines per block,
 * update-pass blocks per solve, graph branches}. Writes min(capacity, 8) entries and
 * returns 8 in *count.
 */
int ccmf_plan_launch_info(const ccmf_plan* plan, int* out, int capacity, int* count);

/*
 * Tuning knobs of a plan: the launch shape of the passes of one iteration (Eq. 30
 * step) and the radix schedule of its FFTs. None of them changes what is computed;
 * a different radix schedule or reduction grid changes the rounding only.
 * In ccmf_plan_set_tuning a negative entry selects the built-in rule.
 */
typedef struct {
    int update_variant;     /* update pass: 0 register vectors in ticket-ordered chunks, 1 TMA rows,
                               2..7 pipelined TMA; 8, 9 the stored-divergence schedule: the update
                               pass also writes a = div^- A* e and b = div^- A* v of the new state
                               (Eq. 28, Eq. 30: the divergence of e - v / rho is a - b / rho), so the
                               first pass of the next iteration reads 2 scalars per voxel instead of
                               the 12 state components; 8: 8 warps per block, 9: 16 warps with half
                               the voxels per lane, 10: 8 warps with half the voxels per lane and two
                               blocks per SM; needs N3 a multiple of 128 / 64 / 64 (variant 8 / 9 / 10,
                               FP32) or 64 / 32 / 32 (FP64); 11 register vectors as 0 with half the
                               voxels per thread, two blocks per SM; 12 the same with three blocks
                               per SM; 13 .. 15 the stored-divergence schedule with independent warps
                               (each walks tj = 8, 4, 6 rows of one z segment of 32 VW voxels, VW = 4
                               (FP32) / 2 (FP64), two blocks of 4 warps per SM; needs N3 a multiple of
                               32 VW) */
    int plane_blocks;       /* y / x passes: 0 three strided passes, 1 one block per (x, y) plane,
                               2, 4, 8, 16 a thread-block cluster per plane */
    int z_pairs_per_block;  /* divergence + forward z pass: line pairs per block, power of two 1..16 */
    int y_lines_per_block;  /* strided y passes, line engine 0: lines per block, power of two 1..16 */
    int x_lines_per_block;  /* strided x pass, line engine 0: lines per block, power of two 1..16 */
    int branches;           /* independent graph branches of a batch, 1..4 */
    int radix_mode;         /* radix schedule of every axis: 0 radix 8 first, then 4, 2, 3, 5;
                               1 as 0 but radix 4s in place of a radix 8 + 2 tail; 2 radix 4 at most */
    int zinv_pairs_per_block; /* inverse z pass: line pairs per block, power of two 1..16 */
    int line_engine;        /* strided y / x passes: 0 in-place radix stages per block (any length),
                               1 one warp per line for power-of-two lengths 128..1024, 2 as 1 with
                               the x pass's tiles of 8 lines moved between the half spectrum and
                               shared memory by TMA (cp.async.bulk.tensor loads and stores;
                               FP32, N1 = 512, N2 a multiple of 8) */
    int z_engine;           /* z passes: 0 Stockham stages over tiles of line pairs (any N3);
                               one warp per line pair for power-of-two N3 128..1024 in the
                               inverse pass (1) or in both passes (2) */
} ccmf_tuning;

/* The plan's current knob values (every entry resolved, none negative). */
int ccmf_plan_get_tuning(const ccmf_plan* plan, ccmf_tuning* out);

/* Apply knob values. Returns CCMF_ERR_UNSUPPORTED_SIZE (and keeps the current
 * tuning) when a requested value cannot run on this grid and device, e.g. a
 * cluster size that does not divide N1 and N2 or whose blocks do not fit. */
int ccmf_plan_set_tuning(ccmf_plan* plan, const ccmf_tuning* tuning);

/*
 * Autotuner: times `iters` iterations of the loop (CUDA events on `stream`, after
 * one untimed run that also captures the graph) for candidate tunings and keeps the
 * fastest. The search is coordinate descent over the knobs in the order of
 * ccmf_tuning, starting from the current tuning. It advances the plan's ADMM state
 * (the workspace must hold a solve of these inputs, as ccmf_solve leaves it), runs
 * every candidate for `iters` iterations three times (the fastest of the last two
 * counts; a candidate must win by 1 %), and records the winner in the
 * library's tuning table under (N1, N2, N3, batch, precision, SM count): plans
 * created later with that key start from it.
 *   gamma, gamma_stride, xi_bar, workspace : as for ccmf_solve
 *   best    : optional host output, the kept tuning
 *   best_ms : optional host output, its time per iteration in milliseconds
 * Synchronises the stream.
 */
int ccmf_plan_autotune(ccmf_plan* plan, const void* gamma, long long gamma_stride, const double* xi_bar,
                       void* workspace, size_t workspace_bytes, int iters, ccmf_tuning* best, double* best_ms,
                       void* stream);

/*
 * The tuning table as text, one line per key
 * ("ccmf-tuning N1 N2 N3 batch precision sms : 10 knob values"). Writes at most
 * capacity bytes (NUL-terminated) and the full length in *length.
 */
int ccmf_tuning_export(char* text, size_t capacity, size_t* length);

/* Add the lines of a text written by ccmf_tuning_export to the table (later lines win). */
int ccmf_tuning_import(const char* text);

/* Enable (1) or disable (0) CUDA-event timing of every loop kernel for later
 * ccmf_solve calls on this plan (events are recorded on the solve's stream
 * inside the captured graph; fixed_iters mode only). */
int ccmf_set_kernel_timing(ccmf_plan* plan, int enable);

/*
 * Gradient of the effective crack energy with respect to the crack resistances,
 * d gamma_eff / d gamma(x), through K unrolled updates of Eq. 30 (reverse mode).
 * The differentiated function is the reported gamma_eff (the max-flow value
 * <xi_bar, A* v^K> of Eq. 12) after K updates with the penalty sequence rho^0 ...
 * rho^{K-1} held fixed: either the given schedule, or the one an adaptive run of
 * K updates with `params` chooses (recorded first). At convergence the gradient
 * tends to |xi*(x)| / N, the envelope derivative of the min-cut value (Eq. 21).
 * Checkpoints of (e, v) are kept every ckpt_every updates; each segment is
 * recomputed once during the reverse sweep (memory: ~K / ckpt_every + ckpt_every
 * state copies).
 *   gamma, gamma_stride : device gamma as for ccmf_solve
 *   xi_bar              : host [batch][3]
 *   params              : delta, rho rule and safeguard of the recording run (NULL = defaults)
 *   K, ckpt_every       : unrolled updates (K <= 4096 when the schedule is recorded), checkpoint interval
 *   rho_schedule        : optional host [batch][K] penalties to replay
 *   workspace           : the plan's workspace (ccmf_plan_workspace_bytes)
 *   adj_workspace       : device memory of ccmf_adjoint_workspace_bytes bytes, 256-byte aligned
 *   grad_gamma          : device output [batch][N] (element type of the plan)
 *   rho_out             : optional host output [batch][K], the schedule used
 *   results             : optional host [batch]: gamma_eff of the replayed run; synchronises the stream
 */
int ccmf_adjoint_workspace_bytes(const ccmf_plan* plan, int K, int ckpt_every, size_t* bytes);

/*
 * Precision of the forward and recompute passes of ccmf_adjoint (the benchmark spec's precision
 * pattern applied to reverse mode; the update differentiated is still Eq. 30 with the
 * penalties replayed). For a CCMF_FP32_MIXED plan, CCMF_FP64 runs the recorded schedule,
 * the forward replay with its checkpoints and every segment recomputation in double,
 * rounds each update's pre-projection point z^k to float and records the branch of the
 * radial projection (Eq. 19, [|z^k| > gamma] in double) as one bit per voxel and update;
 * the reverse sweep then runs in float and takes the branches from those bits. The FP32
 * forward takes the other branch at near-tied voxels and so differentiates another piece
 * of the piecewise-smooth map; with the FP64 forward the FP32 gradient agrees with central
 * differences of the FP64 replayed map. gamma_eff in the results is the FP64 forward's.
 * The first call with CCMF_FP64 creates an FP64 plan of the same grid (its small tables);
 * ccmf_adjoint_workspace_bytes then also counts the FP64 workspace, the FP64 checkpoints
 * and the bits. CCMF_FP32_MIXED (the default of an FP32 plan) keeps everything in float.
 * An FP64 plan accepts only CCMF_FP64.
 */
int ccmf_set_adjoint_forward(ccmf_plan* plan, int precision);
int ccmf_adjoint(ccmf_plan* plan, const void* gamma, long long gamma_stride, const double* xi_bar,
                 const ccmf_params* params, int K, int ckpt_every, const double* rho_schedule,
                 void* workspace, size_t workspace_bytes, void* adj_workspace, size_t adj_workspace_bytes,
                 void* grad_gamma, double* rho_out, ccmf_result* results, void* stream);

/*
 * Batches of independent solves on grids of different shapes (for example many
 * microstructure realisations and crack normals, Sec. 4.5 / Sec. 4.6 style studies).
 * The solves are grouped by shape into sub-plans; one captured CUDA graph runs all
 * groups as independent branches and each solve iterates until its own Eq. 31
 * test holds (or for fixed_iters updates).
 */
typedef struct ccmf_batch ccmf_batch;

/* count solves; shapes = host array [count][3] of (N1, N2, N3), each as for
 * ccmf_plan_create. Allocates the sub-plans' tables. */
int ccmf_batch_create(int count, const int* shapes, int precision, ccmf_batch** out);

/* Release a batch (NULL is accepted). */
int ccmf_batch_destroy(ccmf_batch* batch);

/* Bytes of device workspace ccmf_batch_solve needs. */
int ccmf_batch_workspace_bytes(const ccmf_batch* batch, size_t* bytes);

/*
 * Autotuner of a batch: for every shape group in turn, times `iters` iterations of
 * that group's solves alone (a captured graph of its branches, on their current
 * state) for candidate tunings of its sub-plan and keeps the fastest, by the
 * coordinate descent of ccmf_plan_autotune. The winners go into the tuning table,
 * so later batches and plans with the same group shapes and sizes start from them.
 * It first runs a 2-iteration solve of the whole batch to set up the state, and the
 * next ccmf_batch_solve captures its graph again.
 *   gammas, xi_bar, workspace : as for ccmf_batch_solve
 *   ms                        : optional host [buckets], each group's time per iteration
 * Synchronises the stream.
 */
int ccmf_batch_autotune(ccmf_batch* batch, const void* const* gammas, const double* xi_bar, void* workspace,
                        size_t workspace_bytes, int iters, double* ms, void* stream);

/*
 * Launch mode of ccmf_batch_solve (spec batching pattern; the paper has no batched
 * solver: each solve is the iteration of Eq. 30 with the stopping test of Eq. 31).
 *   enable = 0 (default): one captured graph with one branch of per-shape sub-plan
 *            passes per shape group (the launch shapes ccmf_batch_autotune picks);
 *   enable = 1: one persistent kernel launch per iteration for the whole batch. Its
 *            work items (pass, solve, tile) of the six passes of Eq. 28 / Eq. 30 (z
 *            forward FFT with the divergence, y, x with the Poisson gain, y inverse, z
 *            inverse, the update) sit in one device queue in pass-major order; resident
 *            blocks take them in order, and an item waits (bounded) until the previous
 *            pass of its solve has completed. A wait that runs out sets that solve's
 *            status to CCMF_ERR_TIMEOUT and retires it. The FFT stages are the in-place /
 *            Stockham block stages for every axis length, so results differ from the
 *            graph mode by rounding only. Axes longer than about 400 (FP32) / 200 (FP64)
 *            use narrower tiles; a batch whose tiles do not fit shared memory returns
 *            CCMF_ERR_UNSUPPORTED_SIZE from ccmf_batch_solve.
 * The next ccmf_batch_solve captures its graph again. Returns CCMF_ERR_INVALID_ARG for
 * a NULL batch or enable not in {0, 1}.
 */
int ccmf_batch_set_persistent(ccmf_batch* batch, int enable);

/* Number of shape groups (sub-plans) of the batch. */
int ccmf_batch_buckets(const ccmf_batch* batch, int* buckets);

/*
 * Solve every problem of the batch (Eq. 30, Eq. 31).
 *   gammas    : host array [count] of DEVICE pointers to each solve's gamma field
 *               (element type of the precision; solves may share a pointer)
 *   xi_bar    : host array [count][3] of crack normals
 *   params    : as for ccmf_solve (NULL = defaults); resume must be 0
 *   workspace : device memory of ccmf_batch_workspace_bytes bytes, 256-byte aligned
 *   results   : optional host array [count]; when given, the call synchronises the stream
 */
int ccmf_batch_solve(ccmf_batch* batch, const void* const* gammas, const double* xi_bar,
                     const ccmf_params* params, void* workspace, size_t workspace_bytes,
                     ccmf_result* results, void* stream);

/*
 * Size of the fixed device scratch area used by ccmf_solve_static (64 MiB). The
 * area is a file-scope __device__ array of the library: every GPU that loads the
 * library holds it until the process exits.
 */
#define CCMF_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

/*
 * ccmf_solve_static - one solve (batch 1) that allocates no memory.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory where they need a solve, for example plug-ins whose host
 * application owns all device memory through its own pool (an allocation of theirs
 * would fail or fragment that pool), or latency-critical paths that must avoid the
 * implicit device synchronisation of cudaMalloc and cudaFree. It needs no plan and no workspace:
 * its state, spectra, reduction partials, history and FFT tables live in the
 * library's fixed scratch area of CCMF_STATIC_SCRATCH_BYTES bytes, and it calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 *   n1, n2, n3 : grid as for ccmf_plan_create; a grid whose state does not fit the
 *                scratch area is rejected with CCMF_ERR_UNSUPPORTED_SIZE (about
 *                500k voxels in CCMF_FP32_MIXED, 260k in CCMF_FP64, e.g. 80^3 / 64^3)
 *   precision  : CCMF_FP64 or CCMF_FP32_MIXED (element type of gamma, flow, cut)
 *   gamma      : device array [N1][N2][N3]
 *   xi_bar     : host array [3], the crack normal (normalised internally)
 *   params     : as for ccmf_solve (NULL = defaults); resume must be 0
 *   flow, cut  : optional device outputs [3][N] and [6][N] (NULL to skip)
 *   result     : optional host result; when given, the call synchronises the stream
 * Returns CCMF_OK or an error code; per-solve failures are in result->status.
 *
 * The first call on a device looks up the device address of the scratch area
 * (cudaGetSymbolAddress) with that device current, once per device (thread-safe);
 * make that first call before any stream capture begins. The address belongs to the
 * device's primary context, so the entry point must not be used on a device after a
 * cudaDeviceReset of it. Kernels are launched directly
 * on `stream` (no graph). The call copies the unit normal from host memory with
 * cudaMemcpyAsync; with a tolerance (fixed_iters = 0) the host reads a counter from
 * the device every check_every updates, and with a non-NULL result it synchronises
 * the stream before returning. Every call on a device shares the one scratch area and
 * overwrites what the previous call left there: calls whose GPU work overlaps in
 * time (other streams, other host threads) race with each other and must be
 * serialised by the caller.
 */
int ccmf_solve_static(int n1, int n2, int n3, int precision, const void* gamma, const double* xi_bar,
                      const ccmf_params* params, void* flow, void* cut, ccmf_result* result, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CCMF_H */
