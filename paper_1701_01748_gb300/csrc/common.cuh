// Internal declarations of libppd (not part of the public ABI).
//
// Layout of the solver state in HBM (one context, one GPU):
//   image side   x, xt, g (= Phi^dagger v), ut (= Psi u): n0*n1 reals each
//                u: the 9 SARA dual images, basis-major, 9*n0*n1 reals
//                grid_a (forward FFT output, row-major: the degridding reads
//                its rows by TMA) and grid_v (gridding output, column-major:
//                the inverse column pass reads whole columns): K0*K1 complex
//                each, zero frequency at the centre (plain grid index k
//                stored at (k + K/2) mod K); the FFT temporaries: the forward
//                row pass output column-major (L0 per column), the inverse
//                column pass output row-major (K1 per row)
//   visibility   sorted by (tile, block, centred base row, centred base col,
//   side         caller index); per visibility a 16 B (float) / 32 B (double)
//                record {packed centred base cell, frac0, frac1, U} and the
//                complex arrays y (whitened), v (dual), z, w (Algorithm 2
//                work) and p (prox output, warm start)
//   work items   "chunks": runs of <= chunk visibilities sharing one tile and
//                one block; every gridding/degridding CTA owns one chunk
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/ppd.h"

namespace ppd {

// ---------------------------------------------------------------- types
template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };
template <typename R> using cplx_t = typename Cplx<R>::T;

template <typename R> struct VisRec;
template <> struct __align__(16) VisRec<float> { int packed; float f0, f1, U; };
template <> struct __align__(16) VisRec<double> { int packed; int pad; double f0, f1, U; };

constexpr int KB_J = 8;          // interpolation taps per axis
constexpr int KB_DEG = 7;        // degree of the per-tap FP32 weight polynomial (fit error 4e-8)
constexpr int HALO = 8;          // extended tile = (T + HALO)^2 cells
constexpr int N_BASES = 9;       // Dirac + db1..db8
constexpr int N_WAVELETS = 8;
constexpr int MAX_TAPS = 16;     // db8
// per-chunk norm partials: ||w-y||^2, ||Theta q - y||^2 and, for the
// Algorithm 2 stopping test, ||zbar^t - zbar^(t-1)||^2, ||zbar^t||^2
constexpr int NPART = 4;
constexpr int UNIT = 1 << 30;    // visibilities per work unit of the degridding / sub-iterations (no split: a unit is a chunk)
constexpr double INV_TWO_PI = 0.15915494309189535;

// device error word bits
constexpr int ERR_TMA_TIMEOUT = 1;
constexpr int ERR_NONFINITE = 2;
constexpr int ERR_BOUNDS = 4;

// bounded spin for mbarrier waits (iterations of try_wait)
constexpr long long SPIN_LIMIT = 1ll << 21;

// ---------------------------------------------------------------- overlapped launches
// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later).  A
// kernel started by launch() below may be scheduled while the kernel before
// it in the stream is still draining: its CTAs do their setup (shared
// memory, static tables), then pdl_wait() returns once that kernel has
// completed and its writes are visible.  Every CTA of such a kernel calls
// pdl_wait() before it touches global data that another kernel writes or
// reads, and before it exits, so a kernel's completion still implies the
// completion of everything before it in the stream.  pdl_trigger(), issued
// right after the wait, lets the next kernel's CTAs be scheduled; it takes
// effect once every CTA has issued it or exited, so at most one kernel
// waits ahead.  Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

// ---------------------------------------------------------------- status
struct Error {
    int code;
    std::string msg;
};
void set_last_error(const std::string &msg);
int fail(int code, const std::string &msg);

#define PPD_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::ppd::fail(e_ == cudaErrorMemoryAllocation ? PPD_ERR_OOM : PPD_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

// Makes a context's device current for the duration of an entry point and
// gives the caller's current device back on return.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess || prev == dev || cudaSetDevice(dev) != cudaSuccess) prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Lets kernel `fn` launch with `bytes` of dynamic shared memory on the
// current device (the attribute is one value per device and kernel, raised
// to the largest size any context has asked for).
int smem_attr(const void *fn, int bytes);

#define PPD_CHECK(call)                 \
    do {                                \
        int s_ = (call);                \
        if (s_ != PPD_OK) return s_;    \
    } while (0)

// ---------------------------------------------------------------- context
struct TimingSite {
    const char *name;
    cudaEvent_t start, stop;
};

// Stages of a mixed-radix FFT of length K (radices 2, 3, 4, 5; ns = 0 when
// K has another prime factor).
struct FftPlan {
    static constexpr int MAX_STAGES = 16;
    int K = 0, ns = 0;
    int rad[MAX_STAGES] = {};
};
FftPlan make_fft_plan(int K);
// lengths the FFT passes handle: 32 <= K <= 8192 with prime factors 2, 3, 5
// (lengths that are not powers of two up to 4096 in FP64)
bool fft_length_supported(int K, bool fp64);

struct Chunks {
    int64_t n = 0;
    int32_t *start = nullptr, *count = nullptr, *tile = nullptr, *block = nullptr;   // device
    int32_t *tile_first = nullptr, *tile_n = nullptr;                                // device, n_tiles
    // work units of the degridding and sub-iterations: runs of at most UNIT
    // visibilities of one chunk (device arrays of nu entries); unit u writes
    // its norm partials to slot u_pos[u], block b owns slots blk_ptr[b] ..
    // blk_ptr[b+1] - 1; u_order lists the units by decreasing size (the
    // degridding's visiting order)
    int64_t nu = 0;
    int32_t *u_start = nullptr, *u_count = nullptr, *u_chunk = nullptr, *u_pos = nullptr, *u_order = nullptr;
    int32_t *blk_ptr = nullptr;
    int32_t *order = nullptr;    // chunks by decreasing size (the gridding's CTA order)
    int32_t *active = nullptr;   // tiles the combine pass writes (device)
    int64_t n_active = 0;
};

}  // namespace ppd

struct ppd_ctx {
    ppd_config cfg;
    int is_f32 = 1;
    size_t rsz = 4;            // sizeof(real)
    int L0 = 0, L1 = 0, K0 = 0, K1 = 0, T = 32, C = 1024, levels = 4, d = 1;
    int grid_nw = 8;           // warps per gridding CTA (FP32: 4 or 8; FP64: 4)
    int degrid_nt = 256;       // threads per degridding CTA (FP32: 128 or 256; FP64: 256)
    bool shape_tuned = false;  // the autotuner fixed grid_nw and degrid_nt
    int64_t N = 0;
    double beta = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;

    // image side
    void *x = nullptr, *xt = nullptr, *g = nullptr, *ut = nullptr, *xtrue = nullptr;
    void *u = nullptr, *wtmp = nullptr, *wtmp2 = nullptr;
    void *grid_a = nullptr, *grid_v = nullptr, *fft_tmp = nullptr, *fft_tmp_inv = nullptr;
    // FFT pruning (set by ppd_set_visibilities): column strips the forward /
    // inverse column passes process, grid rows the degridding reads, grid
    // rows the gridding can write, tmp columns the forward column pass reads
    int32_t *fwd_strips = nullptr, *inv_strips = nullptr;
    int n_fwd_strips = 0, n_inv_strips = 0;
    uint8_t *row_fwd = nullptr, *row_inv = nullptr, *col_fwd = nullptr;
    void *tw0 = nullptr, *tw1 = nullptr, *deap0 = nullptr, *deap1 = nullptr;   // twiddles of K0 / K1, Z's scalings
    ppd::FftPlan plan0, plan1;                                               // FFT plans of K0 (columns), K1 (rows)
    void *twst0 = nullptr, *twst1 = nullptr;   // twiddles of the power-of-two core, stage by stage
    void *filt = nullptr;       // 8 x 16 reals (low-pass, zero padded)
    void *kbpoly = nullptr;     // (KB_DEG+1) x 8 floats
    std::vector<float> kbpoly_h;   // host copy (kernel argument of the visibility kernels)
    double *prim_part = nullptr;
    int n_prim_blocks = 0;
    int n_stat_parts = 0;        // primal statistics partials the last primal launch wrote
    bool xt_rows_valid = false;  // fft_tmp holds the forward row pass of xt
    double *stat_out = nullptr; // 3 doubles

    // visibility side
    int64_t M = 0;
    void *rec = nullptr, *theta_v = nullptr, *y = nullptr, *v = nullptr, *z = nullptr,
         *w = nullptr, *p = nullptr, *y_raw = nullptr;
    double theta_scalar = 1.0;
    int64_t *perm = nullptr;
    std::vector<int64_t> perm_h;
    std::vector<int32_t> base0_h, base1_h, count_h, block_h, packed_h;
    std::vector<double> frac_h, eps_h, mu_h;
    // host copies of the last inputs (the autotuner rebuilds the ordering)
    std::vector<double> in_uv, in_y, in_theta, in_U, in_eps;
    std::vector<int32_t> in_block;
    bool has_theta = false, has_U = false, has_eps = false;
    std::vector<int64_t> block_count_h;
    int32_t *count_cell = nullptr;   // per visibility (sorted order), device
    ppd::Chunks ch;
    double *partials = nullptr, *scale = nullptr, *resid2 = nullptr, *eps_d = nullptr,
           *mu_d = nullptr;
    double *part_in = nullptr, *part_out = nullptr;   // chunk-partial banks for the next launch
    // Algorithm 2 stopping test (cfg.inner_tol > 0): per block the step at
    // which the test held in the current iteration (0 = still running) and
    // the steps taken in the last iteration; the arguments of the next
    // sub-iteration / gridding launch: its step number and whether its input
    // bank holds the test partials of the previous step
    int *inner_state = nullptr, *inner_steps = nullptr;
    int next_step = 0, next_test_in = 0;
    int *stop_flag = nullptr;                          // global stopping rule (device, 1 int)
    int *dg_claim = nullptr;                           // degridding work counters (device, 2 ints, zero between launches)
    cudaStream_t stream2 = nullptr;                   // prior (SARA) branch of the iteration
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    void *gpart = nullptr;           // n_chunks x (T+HALO)^2 complex
    int *err = nullptr;              // device error word
    long long wait_first = ppd::SPIN_LIMIT;   // polls of the degridding's first TMA wait (ppd_set_wait_limit)
    CUtensorMap tmap_a;              // TMA descriptor of grid_a
    bool tma_ok = false;

    // prior weights of the re-weighted l1 scheme (Algorithm 1): W (9N reals,
    // basis-major like u) or null for W = I; ||Psi W||_S^2 sets the clip
    // level kappa ||Psi W||^2 and the primal step zeta / ||Psi W||^2
    void *wgt = nullptr, *wcoef = nullptr;
    double psiw2 = 1.0;
    int psiw_iters = 0;
    uint64_t gen = 0;   // bumped whenever captured graphs of this context go stale

    // randomised active sets of Algorithm 3 (ppd_set_active_sets): masks for
    // the next rand_n iterations, rand_n x (d + 9) bytes (d block flags, then
    // 9 basis flags, Dirac first); the current iteration's row; per block
    // whether it has a prox output (Algorithm 2 warm start); and a device
    // flag that makes the gridding recompute the partial tiles of inactive
    // blocks (set while gpart may hold other data than their last tiles)
    bool rand_on = false;
    uint8_t *mask_all = nullptr, *mask_cur = nullptr, *blk_seen = nullptr;
    int32_t rand_n = 0, rand_next = 0;
    int *regrid_d = nullptr;
    bool gpart_stale = true;

    // parameters
    double eta = 0, zeta = 1, tau = 0.49, kappa = 1e-4, op_norm_sq = 0;
    int power_done = 0;
    bool have_vis = false, have_weights = false, p_valid = false;
    int32_t iters = 0;
    bool xtrue_set = false;
    double xtrue_norm2 = 0;

    // graph
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    int64_t graph_kernels = 0;

    // timing
    bool timing = false;
    bool capturing = false;
    // kernels of a stream overlap the drain of their predecessor
    // (programmatic dependent launch; off with per-kernel timing)
    bool overlap = false;
    std::vector<ppd::TimingSite> sites_graph;   // fixed sites inside the captured graph
    std::vector<ppd::TimingSite> sites_eager;   // sites since last collect (eager launches)
    std::vector<cudaEvent_t> event_pool;
    std::vector<std::pair<const char *, std::pair<double, int64_t>>> tsum;
    bool graph_ran_since_collect = false;
    int64_t launches = 0;
};

namespace ppd {

// launch bookkeeping: every kernel launch goes through these so that the
// launch count and optional per-kernel events are recorded.
int launch_begin(ppd_ctx *c, const char *name, cudaStream_t s, int *site);
int launch_end(ppd_ctx *c, int site, cudaStream_t s);

// Launches kernel k, which follows the pdl_wait() rule above, with
// programmatic stream serialisation when the context allows it and `chain`
// is set (the caller clears it after a cross-stream join, so that such a
// kernel waits for all of its inputs in the ordinary way).  Errors are left
// for launch_end to report.
template <typename... P, typename... A>
void launch(ppd_ctx *c, bool chain, void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
            A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (chain && c->overlap && !c->timing) ? 1 : 0;
    (void)cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// ---------------------------------------------------------------- launchers
// FFT (fft.cu)
template <typename R> int fft_forward(ppd_ctx *c, const R *x, cplx_t<R> *grid, cudaStream_t s);
template <typename R> int fft_inverse(ppd_ctx *c, const cplx_t<R> *grid, R *img, cudaStream_t s);
int make_twiddles(ppd_ctx *c);
int fft_plan_pruning(ppd_ctx *c, const std::vector<char> &rows_fwd, const std::vector<char> &cols_fwd,
                     const std::vector<char> &rows_inv, const std::vector<char> &cols_inv);
int make_deapodisation(ppd_ctx *c);

// visibilities (vis.cu)
int bin_all(ppd_ctx *c, const double *uv_d, const int32_t *blk_d, int64_t M, uint64_t *key_d, int32_t *base_d,
            double *frac_d, int32_t *count_d, int *bad_d);
int make_kb_poly(ppd_ctx *c);

enum DegridMode { DG_OP = 0, DG_DUAL = 1, DG_FIRST = 2 };
enum GridMode { GR_OP = 0, GR_OP_U = 1, GR_DUAL = 2 };

template <typename R>
int degrid(ppd_ctx *c, int mode, const cplx_t<R> *grid, cplx_t<R> *out, const int64_t *perm_out,
           cudaStream_t s);
template <typename R>
int subiter(ppd_ctx *c, cudaStream_t s, int only_first = 0, double beta = 0.0, int write_p = 0);
int block_norms(ppd_ctx *c, int which, cudaStream_t s);
template <typename R>
int grid_vis(ppd_ctx *c, int mode, const cplx_t<R> *in, const int64_t *perm_in, cplx_t<R> *grid,
             cudaStream_t s, bool combine = true);

template <typename R>
int grid_vis_into(ppd_ctx *c, int mode, const cplx_t<R> *in, const int64_t *perm, cplx_t<R> *grid, void *gpart,
                  cudaStream_t s);

// SARA (sara.cu)
int make_filters(ppd_ctx *c);
template <typename R> int psi_analysis(ppd_ctx *c, const R *x, R *coef, cudaStream_t s);
template <typename R> int psi_synthesis(ppd_ctx *c, const R *coef, R *x, cudaStream_t s);
template <typename R> int sara_prior_branch(ppd_ctx *c, const R **ll0, cudaStream_t s);
template <typename R> int sara_level0(ppd_ctx *c, const R *ll0, cudaStream_t s);

// image side (image.cu)
// Deterministic CTA sum of three doubles per thread (fixed shuffle tree, then
// warps in order); thread 0 writes out3[0..2].
template <int NTH> __device__ __forceinline__ void cta_sum3(double a, double b, double c, double *out3) {
    __shared__ double red[3][NTH / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][wid] = a;
        red[1][wid] = b;
        red[2][wid] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int i = 0; i < NTH / 32; ++i) {
            s0 += red[0][i];
            s1 += red[1][i];
            s2 += red[2][i];
        }
        out3[0] = s0;
        out3[1] = s1;
        out3[2] = s2;
    }
}

// Primal step of Algorithm 3 on one pixel, with the Dirac basis of the
// prior step (prior weight w0 of Algorithm 1, 1 when w0 is null; kappa is
// the clip level alpha = kappa ||Psi W||^2, zeta the effective zeta /
// ||Psi W||^2; a Dirac basis outside the active set P keeps u0):
//   u0 <- clip(u0 + w0 xt/3, kappa); ut_all = (w0 u0 + ut)/3;
//   xbar = P_C(x - tau (eta g + zeta ut_all)); xt = 2 xbar - x; x = xbar.
// Kahan-compensated per-thread sums of ||xbar - x||^2, ||xbar||^2 and
// ||xbar - x_true||^2 in the working precision.  Returns the new xt.
template <typename R> struct PrimalArgs {
    R *x, *xt, *u0;
    const R *ut, *w0, *xtrue;
    R tau, eta, zeta, kappa;
    const uint8_t *pmask;
};

template <typename R> struct PrimalSums {
    R sd = 0, cd = 0, sx = 0, cx = 0, se = 0, ce = 0;
    __device__ __forceinline__ static void kadd(R &s, R &c, R v) {
        const R y = v - c, t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ void write(double *part3) const {
        cta_sum3<256>((double)sd - (double)cd, (double)sx - (double)cx, (double)se - (double)ce, part3);
    }
};

// The pixel's inputs of the primal step, loadable before g is known.
template <typename R> struct PrimalIn {
    R xo, xte, wd, un, ut, xtr;
};
template <typename R> __device__ __forceinline__ PrimalIn<R> primal_load(const PrimalArgs<R> &P, int64_t e) {
    PrimalIn<R> in;
    in.xo = P.x[e];
    in.xte = P.xt[e];
    in.wd = P.w0 ? P.w0[e] : R(1);
    in.un = P.u0[e];
    in.ut = P.ut[e];
    in.xtr = P.xtrue ? P.xtrue[e] : R(0);
    return in;
}

template <typename R>
__device__ __forceinline__ R primal_pixel(const PrimalArgs<R> &P, int64_t e, R g, const PrimalIn<R> &in,
                                          PrimalSums<R> &acc) {
    const R third = R(1.0 / 3.0);
    const R xo = in.xo, xte = in.xte, wd = in.wd;
    R un = in.un;
    if (!P.pmask || P.pmask[0]) {
        un = fmin(fmax(un + wd * (xte * third), -P.kappa), P.kappa);
        P.u0[e] = un;
    }
    const R utot = (wd * un + in.ut) * third;
    const R xb = fmax(R(0), xo - P.tau * (P.eta * g + P.zeta * utot));
    const R xtn = R(2) * xb - xo;
    P.xt[e] = xtn;
    P.x[e] = xb;
    const R dd = xb - xo;
    PrimalSums<R>::kadd(acc.sd, acc.cd, dd * dd);
    PrimalSums<R>::kadd(acc.sx, acc.cx, xb * xb);
    if (P.xtrue) {
        const R de = xb - in.xtr;
        PrimalSums<R>::kadd(acc.se, acc.ce, de * de);
    }
    return xtn;
}
template <typename R>
__device__ __forceinline__ R primal_pixel(const PrimalArgs<R> &P, int64_t e, R g, PrimalSums<R> &acc) {
    return primal_pixel(P, e, g, primal_load(P, e), acc);
}

template <typename R> PrimalArgs<R> primal_args(ppd_ctx *c);
template <typename R> int primal_step(ppd_ctx *c, cudaStream_t s);   // from g = Phi^dagger v in memory
template <typename R> int fft_inverse_rows(ppd_ctx *c, R *img, cudaStream_t s);
// Grids up to K = 2048 end the iteration with the fused row kernel; larger
// grids with the plain inverse row pass and the primal kernel (an 8192-point
// row pair per CTA costs more registers than the two launches it saves).
inline bool fused_rows(const ppd_ctx *c) { return c->K1 <= 2048; }
// inverse row pass + primal step + the next iteration's forward row pass (fft.cu)
template <typename R> int rows_primal(ppd_ctx *c, cudaStream_t s);
template <typename R> int fft_forward_rows(ppd_ctx *c, const R *x, cudaStream_t s);
template <typename R> int fft_forward_cols(ppd_ctx *c, cplx_t<R> *grid, cudaStream_t s);
template <typename R> int fft_inverse_cols(ppd_ctx *c, const cplx_t<R> *grid, cudaStream_t s);
int reduce_primal_stats(ppd_ctx *c, cudaStream_t s);
// stop_flag = (sqrt(stat_out[0] / stat_out[1]) < tol && every sqrt(resid2_j) <= fac eps_j)
int stop_flag(ppd_ctx *c, double tol, double fac, cudaStream_t s);
template <typename R> int scale_copy(ppd_ctx *c, const R *in, R *out, int64_t n, double a, cudaStream_t s);
// Lanczos steps (image.cu): w -= beta vp, out_dev[0] = <w, v>; w -= alpha v, out_dev[0] = ||w||^2
template <typename R>
int lanczos_dot(ppd_ctx *c, R *w, const R *vp, const R *v, double beta, double *out_dev, cudaStream_t s);
template <typename R> int lanczos_orth(ppd_ctx *c, R *w, const R *v, double alpha, double *out_dev, cudaStream_t s);
template <typename R> int reweight_from(ppd_ctx *c, R *coef_to_w, int64_t n, double omega, cudaStream_t s);
template <typename R> int mul_sq(ppd_ctx *c, R *inout, const R *w, int64_t n, cudaStream_t s);
template <typename R> int sumsq(ppd_ctx *c, const R *in, int64_t n, double *out_dev, cudaStream_t s);

// host-side helpers
std::vector<double> daubechies(int p);   // db_p low-pass filter (2p taps)

}  // namespace ppd
