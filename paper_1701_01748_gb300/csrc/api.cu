// C ABI of libppd (declared in include/ppd.h): context management, set-up of
// the visibilities and weights, the PPD iteration driver (Algorithm 3) and
// the operator entry points.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace ppd {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int smem_attr(const void *fn, int bytes) {
    // the attribute is one value per device and kernel: it only ever grows,
    // so that contexts of different sizes sharing a kernel (the mixed-radix
    // FFT passes) never lower the limit another context's launches rely on
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> limit;
    int dev = 0;
    PPD_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = limit.find(std::make_pair(dev, fn));
    if (it != limit.end() && it->second >= bytes) return PPD_OK;
    PPD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    limit[std::make_pair(dev, fn)] = bytes;
    return PPD_OK;
}

// ----------------------------------------------------------------- launches and timing
static int take_event(ppd_ctx *c, cudaEvent_t *ev) {
    if (!c->event_pool.empty()) {
        *ev = c->event_pool.back();
        c->event_pool.pop_back();
        return PPD_OK;
    }
    PPD_CUDA(cudaEventCreate(ev));
    return PPD_OK;
}

static int record(ppd_ctx *c, cudaEvent_t ev, cudaStream_t s) {
    if (c->capturing) {
        PPD_CUDA(cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal));
    } else {
        PPD_CUDA(cudaEventRecord(ev, s));
    }
    return PPD_OK;
}

int launch_begin(ppd_ctx *c, const char *name, cudaStream_t s, int *site) {
    c->launches++;
    *site = -1;
    if (!c->timing) return PPD_OK;
    TimingSite t{name, nullptr, nullptr};
    PPD_CHECK(take_event(c, &t.start));
    PPD_CHECK(take_event(c, &t.stop));
    PPD_CHECK(record(c, t.start, s));
    auto &v = c->capturing ? c->sites_graph : c->sites_eager;
    v.push_back(t);
    *site = (int)v.size() - 1;
    return PPD_OK;
}

int launch_end(ppd_ctx *c, int site, cudaStream_t s) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PPD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (site < 0) return PPD_OK;
    auto &v = c->capturing ? c->sites_graph : c->sites_eager;
    return record(c, v[site].stop, s);
}

static void tsum_add(ppd_ctx *c, const char *name, double ms) {
    for (auto &p : c->tsum)
        if (std::strcmp(p.first, name) == 0) {
            p.second.first += ms;
            p.second.second += 1;
            return;
        }
    c->tsum.push_back({name, {ms, 1}});
}

}  // namespace ppd

using namespace ppd;

// ----------------------------------------------------------------- helpers
namespace {

template <typename T> int dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? PPD_ERR_OOM : PPD_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return PPD_OK;
}

int dalloc_bytes(void **p, size_t bytes) { return dalloc(reinterpret_cast<unsigned char **>(p), bytes); }

void dfree(void *p) {
    if (p) cudaFree(p);
}

void free_vis(ppd_ctx *c) {
    for (void *p : {c->rec, c->theta_v, c->y, c->v, c->z, c->w, c->p, c->y_raw, (void *)c->perm,
                    (void *)c->count_cell, (void *)c->ch.start, (void *)c->ch.count, (void *)c->ch.tile,
                    (void *)c->ch.block, (void *)c->ch.tile_first, (void *)c->ch.tile_n, (void *)c->ch.blk_ptr,
                    (void *)c->ch.u_start, (void *)c->ch.u_count, (void *)c->ch.u_chunk, (void *)c->ch.u_pos, (void *)c->ch.u_order, (void *)c->ch.order, (void *)c->ch.active, (void *)c->partials, (void *)c->scale, (void *)c->resid2,
                    (void *)c->eps_d, (void *)c->mu_d, c->gpart})
        dfree(p);
    c->rec = c->theta_v = c->y = c->v = c->z = c->w = c->p = c->y_raw = c->gpart = nullptr;
    c->perm = nullptr;
    c->count_cell = nullptr;
    c->ch = Chunks{};
    c->partials = c->scale = c->resid2 = c->eps_d = c->mu_d = nullptr;
    c->have_vis = c->have_weights = false;
    c->gpart_stale = true;
}

void drop_graph(ppd_ctx *c) {
    ++c->gen;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    for (auto &t : c->sites_graph) {
        c->event_pool.push_back(t.start);
        c->event_pool.push_back(t.stop);
    }
    c->sites_graph.clear();
}

cudaStream_t pick(ppd_ctx *c, void *s) { return s ? static_cast<cudaStream_t>(s) : c->stream; }

// Stable LSD radix sort of indices by 64-bit key (16-bit digits).
void radix_sort(const std::vector<uint64_t> &key, std::vector<int64_t> &perm) {
    const int64_t M = (int64_t)key.size();
    perm.resize(M);
    for (int64_t i = 0; i < M; ++i) perm[i] = i;
    uint64_t maxk = 0;
    for (uint64_t k : key) maxk = std::max(maxk, k);
    std::vector<int64_t> tmp(M);
    std::vector<int64_t> cnt(65537);
    for (int shift = 0; shift < 64 && (maxk >> shift) != 0; shift += 16) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int64_t i = 0; i < M; ++i) cnt[((key[perm[i]] >> shift) & 0xffff) + 1]++;
        for (int d = 0; d < 65536; ++d) cnt[d + 1] += cnt[d];
        for (int64_t i = 0; i < M; ++i) tmp[cnt[(key[perm[i]] >> shift) & 0xffff]++] = perm[i];
        perm.swap(tmp);
    }
}

// TMA descriptor of grid_a as a 2-D array of reals (re, im interleaved):
// dims {2*K1, K0}; box {2*(T+8), T+8}; no swizzle, zero fill out of bounds.
int make_tmap(ppd_ctx *c) {
    c->tma_ok = false;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return PPD_OK;   // plain-load path
    }
    const int E = c->T + HALO;
    if (c->K0 < E || c->K1 < E) return PPD_OK;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    cuuint64_t dims[2] = {(cuuint64_t)2 * c->K1, (cuuint64_t)c->K0};
    cuuint64_t strides[1] = {(cuuint64_t)2 * c->K1 * c->rsz};
    cuuint32_t box[2] = {(cuuint32_t)2 * E, (cuuint32_t)E};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&c->tmap_a, c->is_f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                        c->grid_a, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    c->tma_ok = (r == CUDA_SUCCESS);
    return PPD_OK;
}

// Reads the device error word and clears it, so that a failure is reported
// once, by the call that observes it, and the context stays usable.
int check_err_word(ppd_ctx *c) {
    int h = 0;
    PPD_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    if (h) PPD_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (h & ERR_TMA_TIMEOUT) return fail(PPD_ERR_TIMEOUT, "a bounded TMA wait in the degridding kernel gave up");
    if (h & ERR_NONFINITE) return fail(PPD_ERR_NONFINITE, "non-finite block norm");
    return PPD_OK;
}

// Global stopping rule of Algorithm 3 on the last iteration: relative
// variation of x below tol and every block residual within fac eps_j,
// evaluated in FP64 on the device; *flag = 1 when it holds (synchronises).
int stop_rule(ppd_ctx *c, double tol, double fac, int *flag) {
    c->part_out = c->partials;   // bank 0: the data step's residual partials
    PPD_CHECK(block_norms(c, 1, c->stream));
    PPD_CHECK(reduce_primal_stats(c, c->stream));
    PPD_CHECK(stop_flag(c, tol, fac, c->stream));
    PPD_CUDA(cudaMemcpyAsync(flag, c->stop_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    return check_err_word(c);
}

// One PPD iteration (Algorithm 3, lambda = 1, all blocks and bases).  The
// prior branch (SARA analysis, clip, synthesis down to level 1) needs only
// xt and u, so in the FP32 path it runs on a second stream beside the data
// branch (FFT, degridding with the data step, gridding, inverse FFT); both
// join before the primal step.  The per-block P_B
// scales are computed in the prologue of the kernel that uses them, from the
// previous launch's chunk partials (two banks).
template <typename R> int iteration_body(ppd_ctx *c, cudaStream_t s, bool first) {
    using C = cplx_t<R>;
    C *ga = static_cast<C *>(c->grid_a), *gv = static_cast<C *>(c->grid_v);
    // with per-kernel timing on, the branches run serialized so that every
    // event pair brackets exactly one kernel
    const bool fork = c->is_f32 && c->stream2 && !c->timing;
    cudaStream_t s2 = fork ? c->stream2 : s;
    if (fork) {
        PPD_CUDA(cudaEventRecord(c->ev_fork, s));
        PPD_CUDA(cudaStreamWaitEvent(s2, c->ev_fork, 0));
    }
    const R *ll0 = nullptr;
    PPD_CHECK(sara_prior_branch<R>(c, &ll0, s2));
    PPD_CHECK(sara_level0<R>(c, ll0, s2));
    if (fork) PPD_CUDA(cudaEventRecord(c->ev_join, s2));

    double *bank[2] = {c->partials, c->partials + NPART * c->ch.nu};
    int cur = 0;
    // with the fused row kernel the forward row pass of xt was done by the
    // previous iteration's last kernel (or by run_iterations before the first)
    if (!fused_rows(c)) PPD_CHECK(fft_forward_rows<R>(c, static_cast<const R *>(c->xt), s));
    PPD_CHECK(fft_forward_cols<R>(c, ga, s));
    const bool current = c->cfg.inner_init == PPD_INNER_CURRENT;
    // with randomised active sets the warm start is decided per block on
    // the device (blocks without a prox output start from z, then one extra
    // step gives P_B(z)), so the captured iteration is the same every time
    const bool rnd = c->rand_on;
    c->part_out = bank[0];
    c->part_in = bank[1];
    PPD_CHECK(degrid<R>(c, (current || (first && !rnd)) ? DG_FIRST : DG_DUAL, ga, nullptr, nullptr, s));
    // warm start at t = 1: zbar^(0) = P_B(z) (an extra step from z), then
    // the n_itr - 1 steps between the degridding and the gridding; the
    // accelerated solver extrapolates with beta_k = (t_k - 1) / t_{k+1},
    // t_1 = 1, from the second of them on
    const bool extra = !current && (rnd || first);
    if (extra) {
        c->part_in = bank[cur];
        c->part_out = bank[cur ^ 1];
        c->next_step = 0;
        c->next_test_in = 0;
        PPD_CHECK(subiter<R>(c, s, /*only_first=*/rnd ? 1 : 0));
        cur ^= 1;
    }
    const bool fista = c->cfg.inner_solver == PPD_INNER_FISTA;
    double t_k = 1.0;
    for (int k = 1; k < c->cfg.n_itr; ++k) {
        const double t_next = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t_k * t_k));
        const double beta = fista ? (t_k - 1.0) / t_next : 0.0;
        t_k = t_next;
        c->part_in = bank[cur];
        c->part_out = bank[cur ^ 1];
        c->next_step = k;
        c->next_test_in = k >= 2;   // step k - 1 >= 1 left the test partials
        PPD_CHECK(subiter<R>(c, s, 0, beta, fista ? 1 : 0));
        cur ^= 1;
    }
    c->part_in = bank[cur];
    c->part_out = bank[0];
    c->next_step = c->cfg.n_itr;
    c->next_test_in = c->cfg.n_itr >= 2;
    // the combine pass sums the partial tiles into the column-major grid,
    // which the inverse column pass reads in whole columns
    PPD_CHECK(grid_vis<R>(c, GR_DUAL, nullptr, nullptr, gv, s));
    PPD_CHECK(fft_inverse_cols<R>(c, gv, s));
    if (fused_rows(c)) {
        if (fork) PPD_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
        // inverse row pass, primal step and the next iteration's forward row pass
        PPD_CHECK(rows_primal<R>(c, s));
    } else {
        PPD_CHECK(fft_inverse_rows<R>(c, static_cast<R *>(c->g), s));
        if (fork) PPD_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
        PPD_CHECK(primal_step<R>(c, s));
    }
    return PPD_OK;
}

// Before an iteration with randomised active sets: the iteration's masks
// (the next queued row, or all ones once the queue is used up) and, when the
// partial tiles may hold other data, the flag that regrids inactive blocks.
int rand_prepare(ppd_ctx *c, cudaStream_t s) {
    if (!c->rand_on) return PPD_OK;
    const size_t row = (size_t)c->d + N_BASES;
    if (c->rand_next < c->rand_n) {
        PPD_CUDA(cudaMemcpyAsync(c->mask_cur, c->mask_all + (size_t)c->rand_next * row, row, cudaMemcpyDeviceToDevice, s));
        c->rand_next++;
    } else {
        PPD_CUDA(cudaMemsetAsync(c->mask_cur, 1, row, s));
    }
    if (c->gpart_stale) PPD_CUDA(cudaMemsetAsync(c->regrid_d, 1, sizeof(int), s));
    return PPD_OK;
}

int rand_finish(ppd_ctx *c, cudaStream_t s) {
    if (!c->rand_on || !c->gpart_stale) return PPD_OK;
    PPD_CUDA(cudaMemsetAsync(c->regrid_d, 0, sizeof(int), s));
    c->gpart_stale = false;
    return PPD_OK;
}

// The iteration starts at the forward column pass: its row pass of xt is
// the last step of the previous iteration.  When the FFT temporary holds
// anything else (a reset, a restored state, an operator call, the power
// iteration) the row pass runs on its own first.
template <typename R> int xt_rows_ready(ppd_ctx *c, cudaStream_t s) {
    if (c->xt_rows_valid || !fused_rows(c)) return PPD_OK;
    PPD_CHECK(fft_forward_rows<R>(c, static_cast<const R *>(c->xt), s));
    c->xt_rows_valid = true;
    return PPD_OK;
}

template <typename R> int run_iterations(ppd_ctx *c, int n) {
    cudaStream_t s = c->stream;
    for (int it = 0; it < n; ++it) {
        const bool first = !c->p_valid;
        PPD_CHECK(rand_prepare(c, s));
        PPD_CHECK(xt_rows_ready<R>(c, s));
        if (first || !c->cfg.use_graph || !c->is_f32) {
            PPD_CHECK(iteration_body<R>(c, s, first));
        } else {
            if (!c->gexec) {
                c->capturing = true;
                const int64_t before = c->launches;
                cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) {
                    c->capturing = false;
                    return fail(PPD_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
                }
                int st = iteration_body<R>(c, s, false);
                cudaGraph_t g = nullptr;
                e = cudaStreamEndCapture(s, &g);
                c->capturing = false;
                c->launches = before;
                if (st != PPD_OK) {
                    if (g) cudaGraphDestroy(g);
                    return st;
                }
                if (e != cudaSuccess) return fail(PPD_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
                c->graph = g;
                e = cudaGraphInstantiate(&c->gexec, g, 0);
                if (e != cudaSuccess) return fail(PPD_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
                size_t nn = 0;
                cudaGraphGetNodes(g, nullptr, &nn);
                std::vector<cudaGraphNode_t> nodes(nn);
                cudaGraphGetNodes(g, nodes.data(), &nn);
                int64_t kernels = 0;
                for (auto nd : nodes) {
                    cudaGraphNodeType t;
                    cudaGraphNodeGetType(nd, &t);
                    if (t == cudaGraphNodeTypeKernel) kernels++;
                }
                c->graph_kernels = kernels;
            }
            PPD_CUDA(cudaGraphLaunch(c->gexec, s));
            c->launches += c->graph_kernels;
            c->graph_ran_since_collect = true;
        }
        PPD_CHECK(rand_finish(c, s));
        c->xt_rows_valid = fused_rows(c);
        c->p_valid = true;
        c->iters++;
    }
    return PPD_OK;
}

// Start vector of the power iteration, normalised: all ones for seed 0,
// else x_i = 0.5 + 2^-53 (s_i >> 11) with s_i = SplitMix64(seed + (i+1) g),
// g = 0x9E3779B97F4A7C15 (Steele, Lea & Flood 2014, the generator's
// published finaliser), i the row-major pixel index.
std::vector<double> power_start(int n0, int n1, uint64_t seed) {
    const size_t n = (size_t)n0 * n1;
    std::vector<double> x(n, 1.0);
    if (seed != 0) {
        for (size_t i = 0; i < n; ++i) {
            uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            x[i] = 0.5 + (double)(z >> 11) * 0x1.0p-53;
        }
    }
    double s2 = 0;
    for (double v : x) s2 += v * v;
    const double inv = 1.0 / std::sqrt(s2);
    for (double &v : x) v *= inv;
    return x;
}

template <typename R> int power_iteration(ppd_ctx *c) {
    using C = cplx_t<R>;
    cudaStream_t s = c->stream;
    const int64_t N = c->N;
    std::vector<double> x0 = power_start(c->L0, c->L1, c->cfg.seed);
    std::vector<R> start(x0.begin(), x0.end());
    PPD_CUDA(cudaMemcpy(c->x, start.data(), N * sizeof(R), cudaMemcpyHostToDevice));
    double *nrm = c->stat_out;
    double prev = 0, val = 0;
    const int maxit = c->cfg.power_iters > 0 ? c->cfg.power_iters : 1000;
    const double tol = c->cfg.power_tol > 0 ? c->cfg.power_tol : 1e-10;
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
        PPD_CHECK(fft_forward<R>(c, static_cast<const R *>(c->x), static_cast<C *>(c->grid_a), s));
        PPD_CHECK(degrid<R>(c, DG_OP, static_cast<C *>(c->grid_a), static_cast<C *>(c->z), nullptr, s));
        PPD_CHECK(grid_vis<R>(c, GR_OP_U, static_cast<const C *>(c->z), nullptr, static_cast<C *>(c->grid_v), s));
        PPD_CHECK(fft_inverse<R>(c, static_cast<const C *>(c->grid_v), static_cast<R *>(c->g), s));
        PPD_CHECK(sumsq<R>(c, static_cast<const R *>(c->g), N, nrm, s));
        double h[3];
        PPD_CUDA(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, s));
        PPD_CUDA(cudaStreamSynchronize(s));
        val = std::sqrt(h[0]);
        if (!std::isfinite(val) || val <= 0) return fail(PPD_ERR_NONFINITE, "power iteration: non-finite or zero norm");
        PPD_CHECK(scale_copy<R>(c, static_cast<const R *>(c->g), static_cast<R *>(c->x), N, 1.0 / val, s));
        if (std::abs(val - prev) <= tol * val) break;
        prev = val;
    }
    c->op_norm_sq = val;
    c->power_done = std::min(it, maxit);
    c->gpart_stale = true;
    return PPD_OK;
}

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a and
// off-diagonal b (|b| = |a| - 1) by bisection on the Sturm sequence, FP64.
double tridiag_max_eig(const std::vector<double> &a, const std::vector<double> &b) {
    const int m = (int)a.size();
    double lo = std::numeric_limits<double>::infinity(), hi = -lo;
    for (int i = 0; i < m; ++i) {   // Gershgorin interval
        const double r = (i > 0 ? std::abs(b[i - 1]) : 0.0) + (i + 1 < m ? std::abs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto below = [&](double x) {   // eigenvalues < x
        int cnt = 0;
        double d = 1.0;
        for (int i = 0; i < m; ++i) {
            d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 400 && hi - lo > 1e-16 * std::max(std::abs(lo), std::abs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) >= m) hi = mid;
        else lo = mid;
    }
    return hi;
}

// ||U^{1/2} Phi||_S^2 as the largest eigenvalue of Phi^dagger U Phi by the
// Lanczos process (Lanczos 1950) from the same start as the power iteration:
// w = A v_j - beta_{j-1} v_{j-1}, alpha_j = <w, v_j>, w -= alpha_j v_j,
// beta_j = ||w||, v_{j+1} = w / beta_j, with the inner products in FP64; the
// estimate is the largest eigenvalue of the tridiagonal (alpha, beta) after
// each step, stopped when it has changed by at most tol (relative; at least
// 2e-6 in FP32, where the operator itself is accurate to ~1e-7) in three
// consecutive steps, or after maxit steps.  On strongly non-uniform coverages the two largest eigenvalues are
// close and the power iteration needs thousands of steps; Lanczos converges
// in tens.  Vectors: v_{j-1} in xt, v_j in x, w in g.
template <typename R> int lanczos(ppd_ctx *c) {
    using C = cplx_t<R>;
    cudaStream_t s = c->stream;
    const int64_t N = c->N;
    R *v = static_cast<R *>(c->x), *vp = static_cast<R *>(c->xt), *w = static_cast<R *>(c->g);
    std::vector<double> x0 = power_start(c->L0, c->L1, c->cfg.seed);
    std::vector<R> start(x0.begin(), x0.end());
    PPD_CUDA(cudaMemcpy(v, start.data(), N * sizeof(R), cudaMemcpyHostToDevice));
    PPD_CUDA(cudaMemsetAsync(vp, 0, N * sizeof(R), s));
    const int maxit = c->cfg.power_iters > 0 ? c->cfg.power_iters : 1000;
    double tol = c->cfg.power_tol > 0 ? c->cfg.power_tol : 1e-10;
    if (sizeof(R) == 4) tol = std::max(tol, 2e-6);
    std::vector<double> al, be;
    double theta = 0, beta = 0;
    int it = 0, calm = 0;
    for (it = 1; it <= maxit; ++it) {
        PPD_CHECK(fft_forward<R>(c, v, static_cast<C *>(c->grid_a), s));
        PPD_CHECK(degrid<R>(c, DG_OP, static_cast<C *>(c->grid_a), static_cast<C *>(c->z), nullptr, s));
        PPD_CHECK(grid_vis<R>(c, GR_OP_U, static_cast<const C *>(c->z), nullptr, static_cast<C *>(c->grid_v), s));
        PPD_CHECK(fft_inverse<R>(c, static_cast<const C *>(c->grid_v), w, s));
        double h[3];
        PPD_CHECK(lanczos_dot(c, w, vp, v, beta, c->stat_out, s));   // w -= beta v_{j-1}; <w, v_j>
        PPD_CUDA(cudaMemcpyAsync(h, c->stat_out, sizeof(h), cudaMemcpyDeviceToHost, s));
        PPD_CUDA(cudaStreamSynchronize(s));
        const double alpha = h[0];
        PPD_CHECK(lanczos_orth(c, w, v, alpha, c->stat_out, s));     // w -= alpha v_j; ||w||^2
        PPD_CUDA(cudaMemcpyAsync(h, c->stat_out, sizeof(h), cudaMemcpyDeviceToHost, s));
        PPD_CUDA(cudaStreamSynchronize(s));
        if (!std::isfinite(alpha) || !std::isfinite(h[0]))
            return fail(PPD_ERR_NONFINITE, "Lanczos: non-finite inner product");
        al.push_back(alpha);
        const double prev = theta;
        theta = tridiag_max_eig(al, be);
        // stop after three consecutive steps within the tolerance
        calm = (it > 1 && std::abs(theta - prev) <= tol * theta) ? calm + 1 : 0;
        if (calm >= 3) break;
        beta = std::sqrt(std::max(h[0], 0.0));
        if (beta <= 1e-300) break;   // invariant subspace: theta is exact
        be.push_back(beta);
        PPD_CHECK(scale_copy<R>(c, v, vp, N, 1.0, s));          // v_{j-1} <- v_j
        PPD_CHECK(scale_copy<R>(c, w, v, N, 1.0 / beta, s));    // v_j <- w / beta_j
    }
    if (!(theta > 0) || !std::isfinite(theta)) return fail(PPD_ERR_NONFINITE, "Lanczos: non-positive norm");
    c->op_norm_sq = theta;
    c->power_done = std::min(it, maxit);
    c->gpart_stale = true;
    return PPD_OK;
}

int reset_state(ppd_ctx *c) {
    const size_t rb = c->rsz;
    PPD_CUDA(cudaMemsetAsync(c->x, 0, c->N * rb, c->stream));
    PPD_CUDA(cudaMemsetAsync(c->xt, 0, c->N * rb, c->stream));
    PPD_CUDA(cudaMemsetAsync(c->u, 0, N_BASES * c->N * rb, c->stream));
    if (c->M > 0) {
        PPD_CUDA(cudaMemsetAsync(c->v, 0, 2 * c->M * rb, c->stream));
        PPD_CUDA(cudaMemsetAsync(c->p, 0, 2 * c->M * rb, c->stream));
    }
    PPD_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (c->blk_seen) PPD_CUDA(cudaMemsetAsync(c->blk_seen, 0, c->d, c->stream));
    if (c->inner_state) PPD_CUDA(cudaMemsetAsync(c->inner_state, 0, c->d * sizeof(int), c->stream));
    if (c->inner_steps) PPD_CUDA(cudaMemsetAsync(c->inner_steps, 0, c->d * sizeof(int), c->stream));
    c->p_valid = false;
    c->iters = 0;
    c->gpart_stale = true;
    c->xt_rows_valid = false;
    drop_graph(c);
    return PPD_OK;
}

template <typename R> int upload_real(void *dst, const std::vector<double> &src) {
    std::vector<R> t(src.begin(), src.end());
    PPD_CUDA(cudaMemcpy(dst, t.data(), t.size() * sizeof(R), cudaMemcpyHostToDevice));
    return PPD_OK;
}

// ||Psi W||_S^2 by power iteration on Psi W^2 Psi^dagger from the all-ones
// image (same start and stop rule as the one for Phi).  The iterate lives in
// g and ut, which every PPD iteration recomputes before use.
template <typename R> int psiw_power_iteration(ppd_ctx *c) {
    cudaStream_t s = c->stream;
    const int64_t N = c->N;
    R *v = static_cast<R *>(c->g), *y = static_cast<R *>(c->ut), *cw = static_cast<R *>(c->wcoef);
    const R *w = static_cast<const R *>(c->wgt);
    std::vector<R> ones(N, R(1.0 / std::sqrt((double)N)));
    PPD_CUDA(cudaMemcpyAsync(v, ones.data(), N * sizeof(R), cudaMemcpyHostToDevice, s));
    double prev = 0, val = 0;
    const int maxit = c->cfg.power_iters > 0 ? c->cfg.power_iters : 1000;
    const double tol = c->cfg.power_tol > 0 ? c->cfg.power_tol : 1e-10;
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
        PPD_CHECK(psi_analysis<R>(c, v, cw, s));
        PPD_CHECK(mul_sq<R>(c, cw, w, N_BASES * N, s));
        PPD_CHECK(psi_synthesis<R>(c, cw, y, s));
        PPD_CHECK(sumsq<R>(c, y, N, c->stat_out, s));
        double h[3];
        PPD_CUDA(cudaMemcpyAsync(h, c->stat_out, sizeof(h), cudaMemcpyDeviceToHost, s));
        PPD_CUDA(cudaStreamSynchronize(s));
        val = std::sqrt(h[0]);
        if (!std::isfinite(val) || val <= 0)
            return fail(PPD_ERR_NONFINITE, "prior weights: ||Psi W|| is zero or not finite");
        PPD_CHECK(scale_copy<R>(c, y, v, N, 1.0 / val, s));
        if (std::abs(val - prev) <= tol * val) break;
        prev = val;
    }
    c->psiw2 = val;
    c->psiw_iters = std::min(it, maxit);
    return PPD_OK;
}

int ensure_weight_buffers(ppd_ctx *c) {
    const size_t bytes = (size_t)N_BASES * c->N * c->rsz;
    if (!c->wgt) PPD_CHECK(dalloc_bytes(&c->wgt, bytes));
    if (!c->wcoef) PPD_CHECK(dalloc_bytes(&c->wcoef, bytes));
    return PPD_OK;
}

int finish_weights(ppd_ctx *c) {
    drop_graph(c);
    const int st = c->is_f32 ? psiw_power_iteration<float>(c) : psiw_power_iteration<double>(c);
    if (st != PPD_OK) {   // leave the context unweighted rather than half-set
        dfree(c->wgt);
        c->wgt = nullptr;
        c->psiw2 = 1.0;
    }
    return st;
}

}  // namespace

// ======================================================================= ABI
extern "C" {

void ppd_config_default(ppd_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->oversample = 2;
    cfg->kernel_width = 8;
    cfg->kb_beta = 0.0;
    cfg->n_blocks = 1;
    cfg->wavelet_levels = 4;
    cfg->n_itr = 1;
    cfg->tau = 0.49;
    cfg->lambda = 1.0;
    cfg->kappa = 1e-4;
    cfg->eta = 0.0;
    cfg->zeta = 0.0;
    cfg->precision = PPD_FP32_FP64NORMS;
    cfg->precond = 1;
    cfg->inner_init = PPD_INNER_WARM;
    cfg->use_graph = 1;
    cfg->tile = 0;
    cfg->chunk = 0;
    cfg->power_iters = 0;
    cfg->power_tol = 0.0;
    cfg->stream = nullptr;
    cfg->inner_solver = PPD_INNER_FB;
    cfg->inner_tol = 0.0;
    cfg->stop_tol = 0.0;
    cfg->stop_eps_factor = 1.005;
    cfg->stop_every = 1;
    cfg->seed = 0;
    cfg->norm_method = PPD_NORM_LANCZOS;
}

const char *ppd_status_string(int status) {
    switch (status) {
        case PPD_OK: return "ok";
        case PPD_ERR_INVALID_ARG: return "invalid argument";
        case PPD_ERR_OOM: return "out of device memory";
        case PPD_ERR_CUDA: return "CUDA error";
        case PPD_ERR_NONFINITE: return "non-finite value";
        case PPD_ERR_TIMEOUT: return "bounded device wait timed out";
        case PPD_ERR_NOT_READY: return "call out of order";
        case PPD_ERR_UNSUPPORTED: return "unsupported size or option";
        default: return "unknown status";
    }
}

const char *ppd_last_error(void) { return g_last_error.c_str(); }

int ppd_create(ppd_ctx **out, const ppd_config *cfg) {
    if (!out || !cfg) return fail(PPD_ERR_INVALID_ARG, "ppd_create: NULL argument");
    *out = nullptr;
    const ppd_config &k = *cfg;
    if (k.n0 < 16 || k.n1 < 16 || k.n0 > 4096 || k.n1 > 4096 || k.n0 % 16 || k.n1 % 16)
        return fail(PPD_ERR_UNSUPPORTED, "ppd_create: image sides must be multiples of 16 in [16, 4096]");
    const bool fp64 = k.precision == PPD_FP64_PLAIN;
    if (!fft_length_supported(2 * k.n0, fp64) || !fft_length_supported(2 * k.n1, fp64))
        return fail(PPD_ERR_UNSUPPORTED,
                    "ppd_create: the oversampled grid sides 2 n0, 2 n1 must have no prime factor above 5 "
                    "(and be powers of two above 4096 in FP64)");
    if (k.oversample != 2 || k.kernel_width != 8 || k.wavelet_levels != 4)
        return fail(PPD_ERR_UNSUPPORTED, "ppd_create: oversample 2, kernel width 8 and 4 levels are required");
    if (k.n_blocks < 1 || k.n_itr < 1 || !(k.tau > 0) || k.lambda != 1.0 || !(k.kappa > 0) || k.eta < 0 ||
        k.zeta < 0 || k.kb_beta < 0)
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: invalid solver parameter");
    if (k.precision != PPD_FP64_PLAIN && k.precision != PPD_FP32_FP64NORMS)
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: unknown precision");
    if (k.inner_init != PPD_INNER_WARM && k.inner_init != PPD_INNER_CURRENT)
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: unknown inner_init");
    if (k.inner_solver != PPD_INNER_FB && k.inner_solver != PPD_INNER_FISTA)
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: unknown inner_solver");
    if (k.norm_method != PPD_NORM_LANCZOS && k.norm_method != PPD_NORM_POWER)
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: unknown norm_method");
    if (k.tile != 0 && k.tile != 16 && k.tile != 32) return fail(PPD_ERR_INVALID_ARG, "ppd_create: tile must be 16 or 32");
    if (k.chunk < 0) return fail(PPD_ERR_INVALID_ARG, "ppd_create: chunk must be >= 0");
    if (!(k.grid_warps == 0 || k.grid_warps == 4 || (k.grid_warps == 8 && k.precision == PPD_FP32_FP64NORMS)))
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: grid_warps must be 0, 4 or (FP32) 8");
    if (!(k.degrid_threads == 0 || k.degrid_threads == 256 ||
          (k.degrid_threads == 128 && k.precision == PPD_FP32_FP64NORMS)))
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: degrid_threads must be 0, 256 or (FP32) 128");
    if (k.launch_overlap != 0 && k.launch_overlap != 1)
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: launch_overlap must be 0 or 1");
    if (!(k.inner_tol >= 0) || !(k.stop_tol >= 0) || !(k.stop_eps_factor >= 0) || k.stop_every < 0 ||
        !std::isfinite(k.inner_tol) || !std::isfinite(k.stop_tol) || !std::isfinite(k.stop_eps_factor))
        return fail(PPD_ERR_INVALID_ARG, "ppd_create: invalid stopping-test parameter");

    ppd_ctx *c = new (std::nothrow) ppd_ctx();
    if (!c) return fail(PPD_ERR_OOM, "ppd_create: host allocation");
    c->cfg = k;
    c->is_f32 = k.precision == PPD_FP32_FP64NORMS;
    c->rsz = c->is_f32 ? 4 : 8;
    c->L0 = k.n0;
    c->L1 = k.n1;
    c->K0 = 2 * k.n0;
    c->K1 = 2 * k.n1;
    c->N = (int64_t)k.n0 * k.n1;
    c->d = k.n_blocks;
    c->levels = k.wavelet_levels;
    c->T = k.tile ? k.tile : 16;
    if (c->K0 % c->T || c->K1 % c->T) c->T = 16;
    c->C = k.chunk ? k.chunk : 1024;
    c->grid_nw = k.grid_warps ? k.grid_warps : (c->is_f32 ? 8 : 4);
    c->degrid_nt = k.degrid_threads ? k.degrid_threads : 256;
    c->beta = k.kb_beta > 0 ? k.kb_beta : 2.34 * KB_J;
    c->tau = k.tau;
    c->kappa = k.kappa;
    c->zeta = k.zeta > 0 ? k.zeta : 1.0;
    cudaGetDevice(&c->device);
    {
        int major = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
        c->overlap = k.launch_overlap == 1 && major >= 9;
    }
    auto bail = [&](int st) {
        ppd_destroy(c);
        return st;
    };
    if (k.stream) {
        c->stream = static_cast<cudaStream_t>(k.stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(PPD_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(PPD_ERR_CUDA, "ppd_create: stream/event creation"));
    const size_t rb = c->rsz, cb = 2 * c->rsz;
    const int64_t N = c->N, G = (int64_t)c->K0 * c->K1;
    int st = PPD_OK;
    if ((st = dalloc_bytes(&c->x, N * rb)) || (st = dalloc_bytes(&c->xt, N * rb)) ||
        (st = dalloc_bytes(&c->g, N * rb)) || (st = dalloc_bytes(&c->ut, N * rb)) ||
        (st = dalloc_bytes(&c->u, N_BASES * N * rb)) || (st = dalloc_bytes(&c->wtmp, N_WAVELETS * N * rb)) ||
        (st = dalloc_bytes(&c->wtmp2, 4 * N * rb)) || (st = dalloc_bytes(&c->grid_a, G * cb)) ||
        (st = dalloc_bytes(&c->grid_v, G * cb)) || (st = dalloc_bytes(&c->fft_tmp, (int64_t)c->L0 * c->K1 * cb)) ||
        (st = dalloc_bytes(&c->fft_tmp_inv, (int64_t)c->L0 * c->K1 * cb)) ||
        (st = dalloc(&c->fwd_strips, c->K1)) || (st = dalloc(&c->inv_strips, c->K1)) ||
        (st = dalloc(&c->row_fwd, c->K0)) || (st = dalloc(&c->row_inv, c->K0)) || (st = dalloc(&c->col_fwd, c->K1)) ||
        (st = dalloc_bytes(&c->tw0, c->K0 * cb)) || (st = dalloc_bytes(&c->tw1, c->K1 * cb)) ||
        (st = dalloc_bytes(&c->twst0, c->K0 * cb)) || (st = dalloc_bytes(&c->twst1, c->K1 * cb)) ||
        (st = dalloc_bytes(&c->deap0, c->L0 * rb)) ||
        (st = dalloc_bytes(&c->deap1, c->L1 * rb)) ||
        (st = dalloc_bytes(&c->kbpoly, (KB_DEG + 1) * KB_J * sizeof(float))) || (st = dalloc(&c->err, 1)) ||
        (st = dalloc(&c->stat_out, 3)))
        return bail(st);
    c->n_prim_blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 4);
    if ((st = dalloc(&c->prim_part, 3 * (size_t)std::max(c->n_prim_blocks, c->L0)))) return bail(st);
    if ((st = dalloc(&c->mask_cur, (size_t)c->d + N_BASES)) || (st = dalloc(&c->blk_seen, (size_t)c->d)) ||
        (st = dalloc(&c->regrid_d, 1)) || (st = dalloc(&c->inner_state, (size_t)c->d)) ||
        (st = dalloc(&c->inner_steps, (size_t)c->d)) || (st = dalloc(&c->stop_flag, 1)) ||
        (st = dalloc(&c->dg_claim, 2)))
        return bail(st);
    if (cudaMemsetAsync(c->mask_cur, 1, (size_t)c->d + N_BASES, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->dg_claim, 0, 2 * sizeof(int), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->blk_seen, 0, (size_t)c->d, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->regrid_d, 0, sizeof(int), c->stream) != cudaSuccess)
        return bail(fail(PPD_ERR_CUDA, "ppd_create: initialisation"));
    if ((st = make_twiddles(c)) || (st = make_deapodisation(c)) || (st = make_filters(c)) || (st = make_kb_poly(c)))
        return bail(st);
    if (cudaMemsetAsync(c->grid_a, 0, G * cb, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->grid_v, 0, G * cb, c->stream) != cudaSuccess || reset_state(c) != PPD_OK)
        return bail(fail(PPD_ERR_CUDA, "ppd_create: initialisation"));
    if ((st = make_tmap(c))) return bail(st);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(fail(PPD_ERR_CUDA, "ppd_create: sync"));
    *out = c;
    return PPD_OK;
}

void ppd_destroy(ppd_ctx *c) {
    if (!c) return;
    DeviceGuard dg_(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    for (auto &t : c->sites_eager) {
        c->event_pool.push_back(t.start);
        c->event_pool.push_back(t.stop);
    }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    free_vis(c);
    for (void *p : {(void *)c->fwd_strips, (void *)c->inv_strips, (void *)c->row_fwd, (void *)c->row_inv,
                    (void *)c->col_fwd, c->fft_tmp_inv})
        dfree(p);
    for (void *p : {c->wgt, c->wcoef, (void *)c->mask_all, (void *)c->mask_cur, (void *)c->blk_seen,
                    (void *)c->regrid_d, (void *)c->inner_state, (void *)c->inner_steps, (void *)c->stop_flag,
                    (void *)c->dg_claim})
        dfree(p);
    for (void *p : {c->x, c->xt, c->g, c->ut, c->xtrue, c->u, c->wtmp, c->wtmp2, c->grid_a, c->grid_v, c->fft_tmp,
                    c->tw0, c->tw1, c->twst0, c->twst1, c->deap0, c->deap1, c->kbpoly, (void *)c->prim_part, (void *)c->stat_out,
                    (void *)c->err})
        dfree(p);
    if (c->stream2) {
        cudaStreamSynchronize(c->stream2);
        cudaStreamDestroy(c->stream2);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int ppd_set_visibilities(ppd_ctx *c, int64_t M, const double *uv, const double *y, const int32_t *block_id) {
    if (!c || !uv || !y || !block_id) return fail(PPD_ERR_INVALID_ARG, "ppd_set_visibilities: NULL argument");
    DeviceGuard dg_(c->device);
    if (M < 1 || M >= (int64_t)1 << 31) return fail(PPD_ERR_INVALID_ARG, "ppd_set_visibilities: M out of range");
    for (int64_t i = 0; i < 2 * M; ++i)
        if (!std::isfinite(y[i])) return fail(PPD_ERR_INVALID_ARG, "ppd_set_visibilities: non-finite visibility");
    for (int64_t i = 0; i < M; ++i)
        if (!(uv[2 * i] >= -M_PI && uv[2 * i] <= M_PI && uv[2 * i + 1] >= -M_PI && uv[2 * i + 1] <= M_PI) ||
            block_id[i] < 0 || block_id[i] >= c->d)
            return fail(PPD_ERR_INVALID_ARG,
                        "ppd_set_visibilities: omega outside [-pi, pi] or block id out of range");
    free_vis(c);
    drop_graph(c);
    c->M = M;
    const int64_t G = (int64_t)c->K0 * c->K1;
    (void)G;
    double *uv_d = nullptr, *frac_d = nullptr;
    int32_t *blk_d = nullptr, *base_d = nullptr, *cnt_d = nullptr;
    uint64_t *key_d = nullptr;
    int *bad_d = nullptr;
    int st = PPD_OK;
    auto cleanup = [&]() {
        dfree(uv_d);
        dfree(frac_d);
        dfree(blk_d);
        dfree(base_d);
        dfree(cnt_d);
        dfree(key_d);
        dfree(bad_d);
    };
    if ((st = dalloc(&uv_d, 2 * M)) || (st = dalloc(&frac_d, 2 * M)) || (st = dalloc(&blk_d, M)) ||
        (st = dalloc(&base_d, 2 * M)) || (st = dalloc(&cnt_d, M)) || (st = dalloc(&key_d, M)) ||
        (st = dalloc(&bad_d, 1))) {
        cleanup();
        return st;
    }
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        cleanup();
        return fail(e == cudaErrorMemoryAllocation ? PPD_ERR_OOM : PPD_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMemcpy(uv_d, uv, 2 * M * sizeof(double), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(blk_d, block_id, M * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(bad_d, 0, sizeof(int))))
        return cuda_fail(e, "ppd_set_visibilities: upload");
    if ((st = bin_all(c, uv_d, blk_d, M, key_d, base_d, frac_d, cnt_d, bad_d))) {
        cleanup();
        return st;
    }
    int bad = 0;
    std::vector<uint64_t> key(M);
    std::vector<int32_t> base(2 * M), cnt(M);
    std::vector<double> frac(2 * M);
    if ((e = cudaMemcpy(&bad, bad_d, sizeof(int), cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(key.data(), key_d, M * 8, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(base.data(), base_d, 2 * M * 4, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(frac.data(), frac_d, 2 * M * 8, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(cnt.data(), cnt_d, M * 4, cudaMemcpyDeviceToHost)))
        return cuda_fail(e, "ppd_set_visibilities: download");
    cleanup();
    if (bad) return fail(PPD_ERR_INVALID_ARG, "ppd_set_visibilities: omega outside [-pi, pi] or block id out of range");

    // processing order and work items
    radix_sort(key, c->perm_h);
    c->base0_h.resize(M);
    c->base1_h.resize(M);
    c->count_h = cnt;
    c->block_h.assign(block_id, block_id + M);
    for (int64_t i = 0; i < M; ++i) {
        c->base0_h[i] = base[2 * i];
        c->base1_h[i] = base[2 * i + 1];
    }
    const uint64_t KK = (uint64_t)c->K0 * c->K1;
    const int ntiles = (c->K0 / c->T) * (c->K1 / c->T);
    std::vector<int32_t> cs, cn, ct, cbk, tfirst(ntiles, 0), tn(ntiles, 0);
    for (int64_t i = 0; i < M;) {
        const uint64_t k0 = key[c->perm_h[i]];
        const uint64_t tb = k0 / KK;   // tile * d + block
        int64_t j = i;
        while (j < M && key[c->perm_h[j]] / KK == tb) ++j;
        for (int64_t s = i; s < j; s += c->C) {
            const int tile = (int)(tb / (uint64_t)c->d), blk = (int)(tb % (uint64_t)c->d);
            if (tn[tile] == 0) tfirst[tile] = (int32_t)cs.size();
            tn[tile]++;
            cs.push_back((int32_t)s);
            cn.push_back((int32_t)std::min<int64_t>(c->C, j - s));
            ct.push_back(tile);
            cbk.push_back(blk);
        }
        i = j;
    }
    const int64_t nch = (int64_t)cs.size();
    // tiles the gridding can reach: a tile with chunks and the tiles below,
    // right and below-right of it (the extended footprint's halo)
    std::vector<int32_t> active;
    {
        const int nt0 = c->K0 / c->T, nt1 = c->K1 / c->T;
        std::vector<char> mark(ntiles, 0);
        for (int t = 0; t < ntiles; ++t)
            if (tn[t]) {
                const int a0 = t / nt1, a1 = t % nt1;
                for (int d0 = 0; d0 < 2; ++d0)
                    for (int d1 = 0; d1 < 2; ++d1) mark[((a0 + d0) % nt0) * nt1 + (a1 + d1) % nt1] = 1;
            }
        for (int t = 0; t < ntiles; ++t)
            if (mark[t]) active.push_back(t);
    }
    // FFT pruning: rows/columns the degridding reads (tiles with chunks plus
    // their halo) and rows/columns the gridding can write (active tiles)
    std::vector<char> rf(c->K0, 0), cf(c->K1, 0), ri(c->K0, 0), ci(c->K1, 0);
    {
        const int nt1 = c->K1 / c->T;
        for (int t = 0; t < ntiles; ++t) {
            if (!tn[t]) continue;
            const int r0 = (t / nt1) * c->T, c0 = (t % nt1) * c->T;
            for (int k = 0; k < c->T + HALO; ++k) {
                rf[(r0 + k) % c->K0] = 1;
                cf[(c0 + k) % c->K1] = 1;
            }
        }
        for (int t : active) {
            const int r0 = (t / nt1) * c->T, c0 = (t % nt1) * c->T;
            for (int k = 0; k < c->T; ++k) {
                ri[r0 + k] = 1;
                ci[c0 + k] = 1;
            }
        }
    }
    // work units of the degridding and sub-iterations (runs of at most UNIT
    // visibilities of one chunk) and their block-major partial slots: block
    // b owns slots bptr[b] .. bptr[b+1] - 1, unit u writes slot upos[u]
    std::vector<int32_t> us, un, uc;
    for (int64_t k = 0; k < nch; ++k)
        for (int32_t o = 0; o < cn[k]; o += UNIT) {
            us.push_back(cs[k] + o);
            un.push_back(std::min<int32_t>(UNIT, cn[k] - o));
            uc.push_back((int32_t)k);
        }
    const int64_t nu = (int64_t)us.size();
    std::vector<int32_t> uord(nu);
    for (int64_t u = 0; u < nu; ++u) uord[u] = (int32_t)u;
    std::stable_sort(uord.begin(), uord.end(), [&](int32_t a, int32_t b) { return un[a] > un[b]; });
    // the gridding's CTA order: chunks by decreasing size
    std::vector<int32_t> cord(nch);
    for (int64_t k = 0; k < nch; ++k) cord[k] = (int32_t)k;
    std::stable_sort(cord.begin(), cord.end(), [&](int32_t a, int32_t b) { return cn[a] > cn[b]; });
    std::vector<int32_t> bptr(c->d + 1, 0), upos(nu);
    for (int64_t u = 0; u < nu; ++u) bptr[cbk[uc[u]] + 1]++;
    for (int j = 0; j < c->d; ++j) bptr[j + 1] += bptr[j];
    {
        std::vector<int32_t> fill(bptr.begin(), bptr.end() - 1);
        for (int64_t u = 0; u < nu; ++u) upos[u] = fill[cbk[uc[u]]]++;
    }
    c->ch.n = nch;
    c->ch.nu = nu;
    // default gridding CTA shape (unless configured or autotuned): eight
    // warps while the chunks make few waves, four (more CTAs per SM) beyond
    // twelve chunks per SM
    if (c->cfg.grid_warps == 0 && !c->shape_tuned && c->is_f32) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        c->grid_nw = nch > 12LL * std::max(sms, 1) ? 4 : 8;
    }
    c->ch.n_active = (int64_t)active.size();
    const size_t cbsz = 2 * c->rsz;
    const int E = c->T + HALO;
    if ((st = dalloc(&c->ch.start, nch)) || (st = dalloc(&c->ch.count, nch)) || (st = dalloc(&c->ch.tile, nch)) ||
        (st = dalloc(&c->ch.block, nch)) || (st = dalloc(&c->ch.tile_first, ntiles)) ||
        (st = dalloc(&c->ch.tile_n, ntiles)) || (st = dalloc(&c->ch.blk_ptr, c->d + 1)) ||
        (st = dalloc(&c->ch.u_start, nu)) ||
        (st = dalloc(&c->ch.u_count, nu)) || (st = dalloc(&c->ch.u_chunk, nu)) || (st = dalloc(&c->ch.u_pos, nu)) || (st = dalloc(&c->ch.u_order, nu)) || (st = dalloc(&c->ch.order, nch)) ||
        (st = dalloc(&c->ch.active, active.size())) ||
        (st = dalloc(&c->partials, 2 * NPART * (size_t)nu)) ||
        (st = dalloc(&c->scale, c->d)) || (st = dalloc(&c->resid2, c->d)) || (st = dalloc(&c->eps_d, c->d)) ||
        (st = dalloc(&c->mu_d, c->d)) || (st = dalloc_bytes(&c->gpart, (size_t)nch * E * E * cbsz)) ||
        (st = dalloc(&c->perm, M)) || (st = dalloc_bytes(&c->rec, M * (c->is_f32 ? 16 : 32))) ||
        (st = dalloc_bytes(&c->y, M * cbsz)) || (st = dalloc_bytes(&c->v, M * cbsz)) ||
        (st = dalloc_bytes(&c->z, M * cbsz)) || (st = dalloc_bytes(&c->w, M * cbsz)) ||
        (st = dalloc_bytes(&c->p, M * cbsz)) || (st = dalloc_bytes(&c->y_raw, M * 2 * sizeof(double)))) {
        free_vis(c);
        return st;
    }
    std::vector<double> yraw_sorted(2 * M);
    for (int64_t i = 0; i < M; ++i) {
        yraw_sorted[2 * i] = y[2 * c->perm_h[i]];
        yraw_sorted[2 * i + 1] = y[2 * c->perm_h[i] + 1];
    }
    // frac, packed centred base are rebuilt into records by ppd_set_weights;
    // keep the sorted fractions in the host copy until then.
    c->frac_h.resize(2 * M);
    c->packed_h.resize(M);
    for (int64_t i = 0; i < M; ++i) {
        const int64_t o = c->perm_h[i];
        c->frac_h[2 * i] = frac[2 * o];
        c->frac_h[2 * i + 1] = frac[2 * o + 1];
        const int cb0 = (base[2 * o] + c->K0 / 2) % c->K0, cb1 = (base[2 * o + 1] + c->K1 / 2) % c->K1;
        c->packed_h[i] = cb0 | (cb1 << 16);
    }
    if ((e = cudaMemcpy(c->ch.start, cs.data(), nch * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.count, cn.data(), nch * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.tile, ct.data(), nch * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.block, cbk.data(), nch * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.tile_first, tfirst.data(), ntiles * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.tile_n, tn.data(), ntiles * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.blk_ptr, bptr.data(), (c->d + 1) * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.u_start, us.data(), nu * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.u_count, un.data(), nu * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.u_chunk, uc.data(), nu * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.u_pos, upos.data(), nu * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.u_order, uord.data(), nu * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.order, cord.data(), nch * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->ch.active, active.data(), active.size() * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->perm, c->perm_h.data(), M * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->y_raw, yraw_sorted.data(), 2 * M * 8, cudaMemcpyHostToDevice))) {
        free_vis(c);
        return fail(PPD_ERR_CUDA, std::string("ppd_set_visibilities: upload: ") + cudaGetErrorString(e));
    }
    // the combine pass only writes tiles this coverage reaches: clear the rest
    if ((e = cudaMemset(c->grid_v, 0, (size_t)c->K0 * c->K1 * 2 * c->rsz))) {
        free_vis(c);
        return fail(PPD_ERR_CUDA, std::string("ppd_set_visibilities: clear: ") + cudaGetErrorString(e));
    }
    if ((st = fft_plan_pruning(c, rf, cf, ri, ci))) {
        free_vis(c);
        return st;
    }
    c->block_count_h.assign(c->d, 0);
    for (int64_t i = 0; i < M; ++i) c->block_count_h[block_id[i]]++;
    if (c->in_uv.data() != uv) {   // (the autotuner passes the stored copies back in)
        c->in_uv.assign(uv, uv + 2 * M);
        c->in_y.assign(y, y + 2 * M);
        c->in_block.assign(block_id, block_id + M);
    }
    if ((st = make_tmap(c))) {   // the TMA box depends on the tile side
        free_vis(c);
        return st;
    }
    c->have_vis = true;
    c->have_weights = false;
    return PPD_OK;
}

int ppd_set_weights(ppd_ctx *c, const double *theta, const double *U, const double *eps) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_set_weights: NULL context");
    DeviceGuard dg_(c->device);
    if (!c->have_vis) return fail(PPD_ERR_NOT_READY, "ppd_set_weights: call ppd_set_visibilities first");
    const int64_t M = c->M;
    if (c->in_theta.data() != theta || !theta) {
        c->has_theta = theta != nullptr;
        if (theta) c->in_theta.assign(theta, theta + M);
    }
    if (c->in_U.data() != U || !U) {
        c->has_U = U != nullptr;
        if (U) c->in_U.assign(U, U + M);
    }
    if (c->in_eps.data() != eps || !eps) {
        c->has_eps = eps != nullptr;
        if (eps) c->in_eps.assign(eps, eps + c->d);
    }
    std::vector<double> th(M), uu(M);
    bool uniform = true;
    for (int64_t i = 0; i < M; ++i) {
        const int64_t o = c->perm_h[i];
        th[i] = theta ? theta[o] : 1.0;
        if (U) uu[i] = U[o];
        else uu[i] = c->cfg.precond ? 1.0 / (double)c->count_h[o] : 1.0;
        if (!(th[i] > 0) || !std::isfinite(th[i]) || !(uu[i] > 0) || !std::isfinite(uu[i]))
            return fail(PPD_ERR_INVALID_ARG, "ppd_set_weights: theta and U must be finite and > 0");
        if (th[i] != th[0]) uniform = false;
    }
    std::vector<double> ep(c->d), mu(c->d, 1.0), umax(c->d, 0.0);
    for (int j = 0; j < c->d; ++j) {
        const double Mj = (double)c->block_count_h[j];
        ep[j] = eps ? eps[j] : std::sqrt(Mj + 2.0 * std::sqrt(Mj));
        if (Mj == 0) {   // an empty block has no constraint; its bound is never used
            ep[j] = 1.0;
            continue;
        }
        if (!(ep[j] > 0) || !std::isfinite(ep[j]))
            return fail(PPD_ERR_INVALID_ARG, "ppd_set_weights: eps must be finite and > 0");
    }
    for (int64_t i = 0; i < M; ++i) {
        const int b = c->block_h[c->perm_h[i]];
        umax[b] = std::max(umax[b], uu[i]);
    }
    for (int j = 0; j < c->d; ++j)
        if (umax[j] > 0) mu[j] = 1.0 / (umax[j] * umax[j]);
    c->eps_h = ep;
    c->mu_h = mu;
    // records, whitened data, weights
    cudaError_t e;
    std::vector<double> yw(2 * M);
    {
        std::vector<double> yr(2 * M);
        if ((e = cudaMemcpy(yr.data(), c->y_raw, 2 * M * 8, cudaMemcpyDeviceToHost)))
            return fail(PPD_ERR_CUDA, std::string("ppd_set_weights: ") + cudaGetErrorString(e));
        for (int64_t i = 0; i < M; ++i) {
            yw[2 * i] = th[i] * yr[2 * i];
            yw[2 * i + 1] = th[i] * yr[2 * i + 1];
        }
    }
    if (c->is_f32) {
        std::vector<VisRec<float>> rec(M);
        for (int64_t i = 0; i < M; ++i)
            rec[i] = VisRec<float>{c->packed_h[i], (float)c->frac_h[2 * i], (float)c->frac_h[2 * i + 1], (float)uu[i]};
        if ((e = cudaMemcpy(c->rec, rec.data(), M * sizeof(rec[0]), cudaMemcpyHostToDevice)))
            return fail(PPD_ERR_CUDA, std::string("ppd_set_weights: ") + cudaGetErrorString(e));
    } else {
        std::vector<VisRec<double>> rec(M);
        for (int64_t i = 0; i < M; ++i)
            rec[i] = VisRec<double>{c->packed_h[i], 0, c->frac_h[2 * i], c->frac_h[2 * i + 1], uu[i]};
        if ((e = cudaMemcpy(c->rec, rec.data(), M * sizeof(rec[0]), cudaMemcpyHostToDevice)))
            return fail(PPD_ERR_CUDA, std::string("ppd_set_weights: ") + cudaGetErrorString(e));
    }
    int st;
    if ((st = c->is_f32 ? upload_real<float>(c->y, yw) : upload_real<double>(c->y, yw))) return st;
    dfree(c->theta_v);
    c->theta_v = nullptr;
    c->theta_scalar = th[0];
    if (!uniform) {
        if ((st = dalloc_bytes(&c->theta_v, M * c->rsz))) return st;
        if ((st = c->is_f32 ? upload_real<float>(c->theta_v, th) : upload_real<double>(c->theta_v, th))) return st;
    }
    if ((e = cudaMemcpy(c->eps_d, ep.data(), c->d * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->mu_d, mu.data(), c->d * 8, cudaMemcpyHostToDevice)))
        return fail(PPD_ERR_CUDA, std::string("ppd_set_weights: ") + cudaGetErrorString(e));
    c->have_weights = true;
    drop_graph(c);
    if ((st = reset_state(c))) return st;
    // eta = 1 / ||U^{1/2} Phi||^2 (Section 5.1)
    if (c->cfg.eta > 0) {
        c->eta = c->cfg.eta;
        c->op_norm_sq = 0;
        c->power_done = 0;
    } else {
        if (c->cfg.norm_method == PPD_NORM_POWER)
            st = c->is_f32 ? power_iteration<float>(c) : power_iteration<double>(c);
        else
            st = c->is_f32 ? lanczos<float>(c) : lanczos<double>(c);
        if (st) return st;
        c->eta = 1.0 / c->op_norm_sq;
    }
    if ((st = reset_state(c))) return st;
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    return check_err_word(c);
}

int ppd_set_ground_truth(ppd_ctx *c, const double *x_true, int64_t len) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_set_ground_truth: NULL context");
    DeviceGuard dg_(c->device);
    if (!x_true) {
        dfree(c->xtrue);
        c->xtrue = nullptr;
        c->xtrue_set = false;
        drop_graph(c);
        return PPD_OK;
    }
    if (len != c->N) return fail(PPD_ERR_INVALID_ARG, "ppd_set_ground_truth: len must be n0*n1");
    if (!c->xtrue) PPD_CHECK(dalloc_bytes(&c->xtrue, c->N * c->rsz));
    std::vector<double> v(x_true, x_true + len);
    double n2 = 0;
    for (double a : v) n2 += a * a;
    c->xtrue_norm2 = n2;
    PPD_CHECK(c->is_f32 ? upload_real<float>(c->xtrue, v) : upload_real<double>(c->xtrue, v));
    c->xtrue_set = true;
    drop_graph(c);
    return PPD_OK;
}

int ppd_iterate(ppd_ctx *c, int32_t n_iters, ppd_stats *stats) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_iterate: NULL context");
    DeviceGuard dg_(c->device);
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_iterate: call ppd_set_weights first");
    if (n_iters < 0) return fail(PPD_ERR_INVALID_ARG, "ppd_iterate: n_iters < 0");
    int st = PPD_OK, ran = 0, stopped = 0;
    if (c->cfg.stop_tol > 0 && n_iters > 0) {
        // Algorithm 3 until its stopping rule holds: the rule is evaluated on
        // the device in FP64 after every `every`-th iteration of this call
        const int every = c->cfg.stop_every > 0 ? c->cfg.stop_every : 1;
        const double fac = c->cfg.stop_eps_factor > 0 ? c->cfg.stop_eps_factor : 1.005;
        while (ran < n_iters && st == PPD_OK) {
            const int n = std::min(every, n_iters - ran);
            st = c->is_f32 ? run_iterations<float>(c, n) : run_iterations<double>(c, n);
            if (st != PPD_OK) break;
            ran += n;
            if (ran % every == 0) {
                int flag = 0;
                st = stop_rule(c, c->cfg.stop_tol, fac, &flag);
                if (st == PPD_OK && flag) {
                    stopped = 1;
                    break;
                }
            }
        }
    } else {
        st = c->is_f32 ? run_iterations<float>(c, n_iters) : run_iterations<double>(c, n_iters);
        ran = n_iters;
    }
    if (st != PPD_OK) {
        if (stats) stats->status = st;
        return st;
    }
    if (stats) {
        c->part_out = c->partials;   // bank 0 holds the last data step's residual partials
        PPD_CHECK(block_norms(c, 1, c->stream));
        PPD_CHECK(reduce_primal_stats(c, c->stream));
        double h[3];
        std::vector<double> r2(c->d);
        std::vector<int32_t> steps(c->d);
        PPD_CUDA(cudaMemcpyAsync(h, c->stat_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        PPD_CUDA(cudaMemcpyAsync(r2.data(), c->resid2, c->d * 8, cudaMemcpyDeviceToHost, c->stream));
        if (stats->inner_steps)
            PPD_CUDA(cudaMemcpyAsync(steps.data(), c->inner_steps, c->d * 4, cudaMemcpyDeviceToHost, c->stream));
        PPD_CUDA(cudaStreamSynchronize(c->stream));
        st = check_err_word(c);
        stats->iters_done = c->iters;
        stats->iters_run = ran;
        stats->stopped = stopped;
        stats->status = st;
        stats->rel_var = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::numeric_limits<double>::infinity();
        stats->snr_db = c->xtrue_set && h[2] > 0 ? 20.0 * std::log10(std::sqrt(c->xtrue_norm2 / h[2]))
                                                 : std::numeric_limits<double>::quiet_NaN();
        double mx = 0;
        for (int j = 0; j < c->d; ++j) {
            const double rj = std::sqrt(r2[j]);
            if (stats->block_residual) stats->block_residual[j] = rj;
            if (stats->inner_steps) stats->inner_steps[j] = steps[j];
            mx = std::max(mx, rj / c->eps_h[j]);
        }
        stats->max_res_over_eps = mx;
        if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return fail(PPD_ERR_NONFINITE, "ppd_iterate: non-finite image");
        return st;
    }
    return PPD_OK;
}

int ppd_get_image(ppd_ctx *c, double *x_out, int64_t len) {
    if (!c || !x_out) return fail(PPD_ERR_INVALID_ARG, "ppd_get_image: NULL argument");
    DeviceGuard dg_(c->device);
    if (len != c->N) return fail(PPD_ERR_INVALID_ARG, "ppd_get_image: len must be n0*n1");
    if (c->is_f32) {
        std::vector<float> t(c->N);
        PPD_CUDA(cudaMemcpyAsync(t.data(), c->x, c->N * 4, cudaMemcpyDeviceToHost, c->stream));
        PPD_CUDA(cudaStreamSynchronize(c->stream));
        for (int64_t i = 0; i < c->N; ++i) x_out[i] = t[i];
    } else {
        PPD_CUDA(cudaMemcpyAsync(x_out, c->x, c->N * 8, cudaMemcpyDeviceToHost, c->stream));
        PPD_CUDA(cudaStreamSynchronize(c->stream));
    }
    return PPD_OK;
}

int ppd_get_params(ppd_ctx *c, ppd_params *o) {
    if (!c || !o) return fail(PPD_ERR_INVALID_ARG, "ppd_get_params: NULL argument");
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_get_params: call ppd_set_weights first");
    o->eta = c->eta;
    o->zeta = c->zeta / c->psiw2;
    o->tau = c->tau;
    o->kappa = c->kappa;
    o->op_norm_sq = c->op_norm_sq;
    o->power_iters_done = c->power_done;
    o->K0 = c->K0;
    o->K1 = c->K1;
    o->tile = c->T;
    o->chunk = c->C;
    o->grid_warps = c->grid_nw;
    o->degrid_threads = c->degrid_nt;
    o->n_chunks = c->ch.n;
    o->M = c->M;
    o->psiw_norm_sq = c->psiw2;
    o->alpha = c->kappa * c->psiw2;
    const double phi2 = c->op_norm_sq > 0 ? c->op_norm_sq : 1.0 / c->eta;
    o->convergence_lhs = c->tau * (c->zeta / c->psiw2) * c->psiw2 + c->tau * c->eta * phi2;
    return PPD_OK;
}

int ppd_get_bins(ppd_ctx *c, int64_t *perm, int32_t *base0, int32_t *base1, int32_t *count) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_get_bins: NULL context");
    if (!c->have_vis) return fail(PPD_ERR_NOT_READY, "ppd_get_bins: call ppd_set_visibilities first");
    const int64_t M = c->M;
    if (perm) std::copy(c->perm_h.begin(), c->perm_h.end(), perm);
    if (base0) std::copy(c->base0_h.begin(), c->base0_h.end(), base0);
    if (base1) std::copy(c->base1_h.begin(), c->base1_h.end(), base1);
    if (count) std::copy(c->count_h.begin(), c->count_h.end(), count);
    (void)M;
    return PPD_OK;
}

int ppd_op_forward(ppd_ctx *c, const void *x_dev, void *y_dev, void *stream) {
    if (!c || !x_dev || !y_dev) return fail(PPD_ERR_INVALID_ARG, "ppd_op_forward: NULL argument");
    DeviceGuard dg_(c->device);
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_op_forward: call ppd_set_weights first");
    cudaStream_t s = pick(c, stream);
    if (c->is_f32) {
        PPD_CHECK(fft_forward<float>(c, static_cast<const float *>(x_dev), static_cast<float2 *>(c->grid_a), s));
        return degrid<float>(c, DG_OP, static_cast<float2 *>(c->grid_a), static_cast<float2 *>(y_dev), c->perm, s);
    }
    PPD_CHECK(fft_forward<double>(c, static_cast<const double *>(x_dev), static_cast<double2 *>(c->grid_a), s));
    return degrid<double>(c, DG_OP, static_cast<double2 *>(c->grid_a), static_cast<double2 *>(y_dev), c->perm, s);
}

int ppd_op_adjoint(ppd_ctx *c, const void *y_dev, void *x_dev, void *stream) {
    if (!c || !x_dev || !y_dev) return fail(PPD_ERR_INVALID_ARG, "ppd_op_adjoint: NULL argument");
    DeviceGuard dg_(c->device);
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_op_adjoint: call ppd_set_weights first");
    cudaStream_t s = pick(c, stream);
    c->gpart_stale = true;   // the partial tiles now hold this call's data
    if (c->is_f32) {
        PPD_CHECK(grid_vis<float>(c, GR_OP, static_cast<const float2 *>(y_dev), c->perm,
                                  static_cast<float2 *>(c->grid_v), s));
        return fft_inverse<float>(c, static_cast<const float2 *>(c->grid_v), static_cast<float *>(x_dev), s);
    }
    PPD_CHECK(grid_vis<double>(c, GR_OP, static_cast<const double2 *>(y_dev), c->perm,
                               static_cast<double2 *>(c->grid_v), s));
    return fft_inverse<double>(c, static_cast<const double2 *>(c->grid_v), static_cast<double *>(x_dev), s);
}

int ppd_psi_analysis(ppd_ctx *c, const void *x_dev, void *c_dev, void *stream) {
    if (!c || !x_dev || !c_dev) return fail(PPD_ERR_INVALID_ARG, "ppd_psi_analysis: NULL argument");
    DeviceGuard dg_(c->device);
    cudaStream_t s = pick(c, stream);
    if (c->is_f32) return psi_analysis<float>(c, static_cast<const float *>(x_dev), static_cast<float *>(c_dev), s);
    return psi_analysis<double>(c, static_cast<const double *>(x_dev), static_cast<double *>(c_dev), s);
}

int ppd_psi_synthesis(ppd_ctx *c, const void *c_dev, void *x_dev, void *stream) {
    if (!c || !x_dev || !c_dev) return fail(PPD_ERR_INVALID_ARG, "ppd_psi_synthesis: NULL argument");
    DeviceGuard dg_(c->device);
    cudaStream_t s = pick(c, stream);
    if (c->is_f32) return psi_synthesis<float>(c, static_cast<const float *>(c_dev), static_cast<float *>(x_dev), s);
    return psi_synthesis<double>(c, static_cast<const double *>(c_dev), static_cast<double *>(x_dev), s);
}

int ppd_set_prior_weights(ppd_ctx *c, const double *w, int64_t len) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_set_prior_weights: NULL context");
    DeviceGuard dg_(c->device);
    if (!w) {
        PPD_CUDA(cudaStreamSynchronize(c->stream));
        dfree(c->wgt);
        c->wgt = nullptr;
        c->psiw2 = 1.0;
        c->psiw_iters = 0;
        drop_graph(c);
        return PPD_OK;
    }
    if (len != (int64_t)N_BASES * c->N) return fail(PPD_ERR_INVALID_ARG, "ppd_set_prior_weights: len != 9 n0 n1");
    for (int64_t i = 0; i < len; ++i)
        if (!(w[i] >= 0.0) || !std::isfinite(w[i]))
            return fail(PPD_ERR_INVALID_ARG, "ppd_set_prior_weights: weights must be finite and >= 0");
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    PPD_CHECK(ensure_weight_buffers(c));
    if (c->is_f32) {
        PPD_CHECK(upload_real<float>(c->wgt, std::vector<double>(w, w + len)));
    } else {
        PPD_CHECK(upload_real<double>(c->wgt, std::vector<double>(w, w + len)));
    }
    return finish_weights(c);
}

int ppd_reweight(ppd_ctx *c, double omega) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_reweight: NULL context");
    DeviceGuard dg_(c->device);
    if (!(omega > 0) || !std::isfinite(omega)) return fail(PPD_ERR_INVALID_ARG, "ppd_reweight: omega must be > 0");
    PPD_CHECK(ensure_weight_buffers(c));
    cudaStream_t s = c->stream;
    if (c->is_f32) {
        PPD_CHECK(psi_analysis<float>(c, static_cast<const float *>(c->x), static_cast<float *>(c->wgt), s));
        PPD_CHECK(reweight_from<float>(c, static_cast<float *>(c->wgt), N_BASES * c->N, omega, s));
    } else {
        PPD_CHECK(psi_analysis<double>(c, static_cast<const double *>(c->x), static_cast<double *>(c->wgt), s));
        PPD_CHECK(reweight_from<double>(c, static_cast<double *>(c->wgt), N_BASES * c->N, omega, s));
    }
    return finish_weights(c);
}

int ppd_set_active_sets(ppd_ctx *c, int32_t n_iters, const uint8_t *blocks, const uint8_t *bases) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_set_active_sets: NULL context");
    DeviceGuard dg_(c->device);
    if (n_iters < 0) return fail(PPD_ERR_INVALID_ARG, "ppd_set_active_sets: n_iters < 0");
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    dfree(c->mask_all);
    c->mask_all = nullptr;
    c->rand_n = c->rand_next = 0;
    if (n_iters == 0) {
        if (c->rand_on) {
            c->rand_on = false;
            drop_graph(c);
        }
        return PPD_OK;
    }
    const size_t row = (size_t)c->d + N_BASES;
    std::vector<uint8_t> h((size_t)n_iters * row);
    for (int32_t t = 0; t < n_iters; ++t) {
        for (int j = 0; j < c->d; ++j) h[t * row + j] = blocks ? (blocks[(size_t)t * c->d + j] != 0) : 1;
        for (int i = 0; i < N_BASES; ++i) h[t * row + c->d + i] = bases ? (bases[(size_t)t * N_BASES + i] != 0) : 1;
    }
    PPD_CHECK(dalloc(&c->mask_all, h.size()));
    PPD_CUDA(cudaMemcpy(c->mask_all, h.data(), h.size(), cudaMemcpyHostToDevice));
    if (!c->rand_on) {
        // after plain iterations every block holds a prox output
        PPD_CUDA(cudaMemset(c->blk_seen, c->p_valid ? 1 : 0, c->d));
        c->rand_on = true;
        c->gpart_stale = true;
        drop_graph(c);
    }
    c->rand_n = n_iters;
    return PPD_OK;
}

int ppd_get_prior_weights(ppd_ctx *c, double *w, int64_t len) {
    if (!c || !w) return fail(PPD_ERR_INVALID_ARG, "ppd_get_prior_weights: NULL argument");
    DeviceGuard dg_(c->device);
    if (len != (int64_t)N_BASES * c->N) return fail(PPD_ERR_INVALID_ARG, "ppd_get_prior_weights: len != 9 n0 n1");
    if (!c->wgt) {
        std::fill(w, w + len, 1.0);
        return PPD_OK;
    }
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    if (c->is_f32) {
        std::vector<float> t(len);
        PPD_CUDA(cudaMemcpy(t.data(), c->wgt, len * sizeof(float), cudaMemcpyDeviceToHost));
        std::copy(t.begin(), t.end(), w);
    } else {
        PPD_CUDA(cudaMemcpy(w, c->wgt, len * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return PPD_OK;
}

int ppd_autotune(ppd_ctx *c, int32_t iters, int32_t *tile_out, int32_t *chunk_out) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_autotune: NULL context");
    DeviceGuard dg_(c->device);
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_autotune: call ppd_set_weights first");
    if (iters < 1) return fail(PPD_ERR_INVALID_ARG, "ppd_autotune: iters < 1");
    const double eta_cfg = c->cfg.eta;
    c->cfg.eta = c->eta;   // keep the resolved eta: no power iteration per candidate
    const std::vector<double> uv = c->in_uv, y = c->in_y, th = c->in_theta, U = c->in_U, ep = c->in_eps;
    const std::vector<int32_t> blk = c->in_block;
    const bool hth = c->has_theta, hU = c->has_U, hep = c->has_eps;
    const bool timing = c->timing;
    c->timing = false;
    auto rebuild = [&](int T, int C) {
        c->T = T;
        c->C = C;
        int st = ppd_set_visibilities(c, c->M, uv.data(), y.data(), blk.data());
        if (st == PPD_OK) st = ppd_set_weights(c, hth ? th.data() : nullptr, hU ? U.data() : nullptr,
                                               hep ? ep.data() : nullptr);
        return st;
    };
    cudaEvent_t e0, e1;
    PPD_CUDA(cudaEventCreate(&e0));
    PPD_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bt = c->T, bc = c->C, bw = c->grid_nw, bd = c->degrid_nt, st = PPD_OK;
    const std::vector<int> warps = c->is_f32 ? std::vector<int>{8, 4} : std::vector<int>{4};
    const std::vector<int> dthreads = c->is_f32 ? std::vector<int>{256, 128} : std::vector<int>{256};
    for (int T : {16, 32}) {
        if (c->K0 % T || c->K1 % T || c->K0 < 2 * T || c->K1 < 2 * T) continue;
        for (int C : {512, 1024, 2048}) {
            // the CTA shapes need no new visibility order, only a new graph;
            // each shape is timed twice, the passes interleaved, and keeps
            // its faster time
            if ((st = rebuild(T, C))) break;
            for (int pass = 0; pass < 2 && !st; ++pass) {
                for (int NW : warps) {
                    for (int ND : dthreads) {
                        c->grid_nw = NW;
                        c->degrid_nt = ND;
                        drop_graph(c);
                        if ((st = ppd_iterate(c, 3, nullptr))) break;
                        cudaEventRecord(e0, c->stream);
                        if ((st = ppd_iterate(c, iters, nullptr))) break;
                        cudaEventRecord(e1, c->stream);
                        cudaEventSynchronize(e1);
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (ms < best) {
                            best = ms;
                            bt = T;
                            bc = C;
                            bw = NW;
                            bd = ND;
                        }
                    }
                    if (st) break;
                }
            }
            if (st) break;
        }
        if (st) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->grid_nw = bw;
    c->degrid_nt = bd;
    c->shape_tuned = true;
    if (st == PPD_OK) st = rebuild(bt, bc);
    c->cfg.eta = eta_cfg;
    c->timing = timing;
    if (st) return st;
    if (tile_out) *tile_out = bt;
    if (chunk_out) *chunk_out = bc;
    return PPD_OK;
}

struct ppd_group {
    std::vector<ppd_ctx *> ctxs;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> kernels;   // kernels each context contributes to one replay
    std::vector<uint64_t> gens;     // the contexts' graph generations at capture
};

void ppd_group_destroy(ppd_group *g) {
    if (!g) return;
    DeviceGuard dg_(g->ctxs.empty() ? 0 : g->ctxs[0]->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (cudaEvent_t e : g->joins) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

int ppd_group_create(ppd_group **out, ppd_ctx *const *ctxs, int32_t n) {
    if (!out || !ctxs || n < 1) return fail(PPD_ERR_INVALID_ARG, "ppd_group_create: invalid argument");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(PPD_ERR_INVALID_ARG, "ppd_group_create: NULL context");
        if (!ctxs[i]->is_f32) return fail(PPD_ERR_INVALID_ARG, "ppd_group_create: groups hold FP32 contexts");
        if (ctxs[i]->timing) return fail(PPD_ERR_INVALID_ARG, "ppd_group_create: per-kernel timing must be off");
        if (!ctxs[i]->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_group_create: context without weights");
        if (ctxs[i]->device != ctxs[0]->device)
            return fail(PPD_ERR_INVALID_ARG, "ppd_group_create: contexts on different devices");
    }
    DeviceGuard dg_(ctxs[0]->device);
    ppd_group *g = new (std::nothrow) ppd_group();
    if (!g) return fail(PPD_ERR_OOM, "ppd_group_create: host allocation");
    g->ctxs.assign(ctxs, ctxs + n);
    g->joins.resize(n, nullptr);
    bool ok = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i)
        ok = cudaEventCreateWithFlags(&g->joins[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        ppd_group_destroy(g);
        return fail(PPD_ERR_CUDA, "ppd_group_create: stream/event creation");
    }
    *out = g;
    return PPD_OK;
}

int ppd_group_iterate(ppd_group *g, int32_t n_iters) {
    if (!g) return fail(PPD_ERR_INVALID_ARG, "ppd_group_iterate: NULL group");
    if (n_iters < 0) return fail(PPD_ERR_INVALID_ARG, "ppd_group_iterate: n_iters < 0");
    DeviceGuard dg_(g->ctxs[0]->device);
    if (n_iters == 0) return PPD_OK;
    // a context's first iteration (Algorithm 2 starts from P_B(z)) differs
    // from the captured one: if any context needs it, every context runs one
    // iteration eagerly and the graph covers the remaining n_iters - 1
    bool any_first = false;
    for (ppd_ctx *c : g->ctxs) any_first = any_first || !c->p_valid;
    if (any_first) {
        for (ppd_ctx *c : g->ctxs) {
            PPD_CHECK(rand_prepare(c, c->stream));
            PPD_CHECK(xt_rows_ready<float>(c, c->stream));
            PPD_CHECK(iteration_body<float>(c, c->stream, !c->p_valid));
            PPD_CHECK(rand_finish(c, c->stream));
            c->xt_rows_valid = fused_rows(c);
            c->p_valid = true;
            c->iters++;
        }
        if (--n_iters == 0) return PPD_OK;
    }
    bool stale = g->gens.size() != g->ctxs.size();
    for (size_t i = 0; !stale && i < g->ctxs.size(); ++i) stale = g->gens[i] != g->ctxs[i]->gen;
    if (stale && g->exec) {   // a context's parameters, weights or buffers changed since the capture
        PPD_CUDA(cudaStreamSynchronize(g->stream));
        cudaGraphExecDestroy(g->exec);
        cudaGraphDestroy(g->graph);
        g->exec = nullptr;
        g->graph = nullptr;
    }
    if (!g->exec) {
        g->gens.clear();
        for (ppd_ctx *c : g->ctxs) g->gens.push_back(c->gen);
        std::vector<int64_t> before;
        for (ppd_ctx *c : g->ctxs) before.push_back(c->launches);
        PPD_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        int st = PPD_OK;
        cudaError_t e = cudaEventRecord(g->fork, g->stream);
        for (size_t i = 0; st == PPD_OK && e == cudaSuccess && i < g->ctxs.size(); ++i) {
            ppd_ctx *c = g->ctxs[i];
            e = cudaStreamWaitEvent(c->stream, g->fork, 0);
            if (e == cudaSuccess) st = iteration_body<float>(c, c->stream, false);
            if (st == PPD_OK && e == cudaSuccess) e = cudaEventRecord(g->joins[i], c->stream);
            if (st == PPD_OK && e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->joins[i], 0);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(g->stream, &graph);
        g->kernels.clear();
        for (size_t i = 0; i < g->ctxs.size(); ++i) {   // captured, not yet run
            g->kernels.push_back(g->ctxs[i]->launches - before[i]);
            g->ctxs[i]->launches = before[i];
        }
        if (st != PPD_OK || e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (st != PPD_OK) return st;
            return fail(PPD_ERR_CUDA, std::string("ppd_group_iterate: capture: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        g->graph = graph;
        PPD_CUDA(cudaGraphInstantiate(&g->exec, graph, 0));
    }
    // order the group's stream after everything already queued on the contexts' streams
    for (size_t i = 0; i < g->ctxs.size(); ++i) {
        PPD_CUDA(cudaEventRecord(g->joins[i], g->ctxs[i]->stream));
        PPD_CUDA(cudaStreamWaitEvent(g->stream, g->joins[i], 0));
    }
    for (int it = 0; it < n_iters; ++it) {
        for (ppd_ctx *c : g->ctxs) {
            PPD_CHECK(rand_prepare(c, g->stream));
            PPD_CHECK(xt_rows_ready<float>(c, g->stream));
        }
        PPD_CUDA(cudaGraphLaunch(g->exec, g->stream));
        for (ppd_ctx *c : g->ctxs) {
            PPD_CHECK(rand_finish(c, g->stream));
            c->xt_rows_valid = fused_rows(c);
        }
        for (size_t i = 0; i < g->ctxs.size(); ++i) {
            g->ctxs[i]->iters++;
            g->ctxs[i]->launches += g->kernels[i];
        }
    }
    // keep each context's own stream ordered after the group's work
    PPD_CUDA(cudaEventRecord(g->fork, g->stream));
    for (ppd_ctx *c : g->ctxs) PPD_CUDA(cudaStreamWaitEvent(c->stream, g->fork, 0));
    return PPD_OK;
}

namespace {
struct StateHeader {
    char magic[8];
    int32_t version, precision, n0, n1;
    int64_t M;
    int32_t d, iters, p_valid, pad;
    uint64_t order_hash;
};

uint64_t order_fingerprint(const ppd_ctx *c) {   // FNV-1a over the processing order
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : c->perm_h) {
        for (int k = 0; k < 8; ++k) {
            h ^= (uint64_t)((v >> (8 * k)) & 0xff);
            h *= 1099511628211ull;
        }
    }
    return h;
}

int64_t state_bytes(const ppd_ctx *c) {
    return (int64_t)sizeof(StateHeader) + (int64_t)c->rsz * (11 * c->N + 4 * c->M) + c->d;
}
}  // namespace

int ppd_get_state(ppd_ctx *c, void *blob, int64_t *bytes) {
    if (!c || !bytes) return fail(PPD_ERR_INVALID_ARG, "ppd_get_state: NULL argument");
    DeviceGuard dg_(c->device);
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_get_state: call ppd_set_weights first");
    const int64_t need = state_bytes(c);
    if (!blob) {
        *bytes = need;
        return PPD_OK;
    }
    if (*bytes < need) return fail(PPD_ERR_INVALID_ARG, "ppd_get_state: buffer too small");
    StateHeader h{};
    std::memcpy(h.magic, "PPDSTATE", 8);
    h.version = 2;
    h.precision = c->cfg.precision;
    h.n0 = c->L0;
    h.n1 = c->L1;
    h.M = c->M;
    h.d = c->d;
    h.iters = c->iters;
    h.p_valid = c->p_valid ? 1 : 0;
    h.order_hash = order_fingerprint(c);
    unsigned char *o = static_cast<unsigned char *>(blob);
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const size_t rb = c->rsz;
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    if (c->stream2) PPD_CUDA(cudaStreamSynchronize(c->stream2));
    PPD_CUDA(cudaMemcpy(o, c->x, c->N * rb, cudaMemcpyDeviceToHost));
    o += c->N * rb;
    PPD_CUDA(cudaMemcpy(o, c->xt, c->N * rb, cudaMemcpyDeviceToHost));
    o += c->N * rb;
    PPD_CUDA(cudaMemcpy(o, c->u, N_BASES * c->N * rb, cudaMemcpyDeviceToHost));
    o += N_BASES * c->N * rb;
    PPD_CUDA(cudaMemcpy(o, c->v, 2 * c->M * rb, cudaMemcpyDeviceToHost));
    o += 2 * c->M * rb;
    PPD_CUDA(cudaMemcpy(o, c->p, 2 * c->M * rb, cudaMemcpyDeviceToHost));
    o += 2 * c->M * rb;
    PPD_CUDA(cudaMemcpy(o, c->blk_seen, c->d, cudaMemcpyDeviceToHost));
    *bytes = need;
    return PPD_OK;
}

int ppd_set_state(ppd_ctx *c, const void *blob, int64_t bytes) {
    if (!c || !blob) return fail(PPD_ERR_INVALID_ARG, "ppd_set_state: NULL argument");
    DeviceGuard dg_(c->device);
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_set_state: call ppd_set_weights first");
    if (bytes != state_bytes(c)) return fail(PPD_ERR_INVALID_ARG, "ppd_set_state: size mismatch");
    StateHeader h;
    std::memcpy(&h, blob, sizeof(h));
    if (std::memcmp(h.magic, "PPDSTATE", 8) != 0 || h.version != 2 || h.precision != c->cfg.precision ||
        h.n0 != c->L0 || h.n1 != c->L1 || h.M != c->M || h.d != c->d)
        return fail(PPD_ERR_INVALID_ARG, "ppd_set_state: blob made for another configuration");
    if (h.order_hash != order_fingerprint(c))
        return fail(PPD_ERR_INVALID_ARG, "ppd_set_state: blob made for another visibility order");
    const unsigned char *o = static_cast<const unsigned char *>(blob) + sizeof(h);
    const size_t rb = c->rsz;
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    if (c->stream2) PPD_CUDA(cudaStreamSynchronize(c->stream2));
    PPD_CUDA(cudaMemcpy(c->x, o, c->N * rb, cudaMemcpyHostToDevice));
    o += c->N * rb;
    PPD_CUDA(cudaMemcpy(c->xt, o, c->N * rb, cudaMemcpyHostToDevice));
    o += c->N * rb;
    PPD_CUDA(cudaMemcpy(c->u, o, N_BASES * c->N * rb, cudaMemcpyHostToDevice));
    o += N_BASES * c->N * rb;
    PPD_CUDA(cudaMemcpy(c->v, o, 2 * c->M * rb, cudaMemcpyHostToDevice));
    o += 2 * c->M * rb;
    PPD_CUDA(cudaMemcpy(c->p, o, 2 * c->M * rb, cudaMemcpyHostToDevice));
    o += 2 * c->M * rb;
    PPD_CUDA(cudaMemcpy(c->blk_seen, o, c->d, cudaMemcpyHostToDevice));
    c->iters = h.iters;
    c->p_valid = h.p_valid != 0;
    c->gpart_stale = true;   // the partial tiles belong to the replaced dual
    c->xt_rows_valid = false;
    return PPD_OK;
}

int ppd_timing_enable(ppd_ctx *c, int32_t enable) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_timing_enable: NULL context");
    if ((bool)enable != c->timing) {
        c->timing = enable != 0;
        drop_graph(c);
    }
    c->tsum.clear();
    return PPD_OK;
}

int ppd_timing_collect(ppd_ctx *c) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_timing_collect: NULL context");
    DeviceGuard dg_(c->device);
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    for (auto &t : c->sites_eager) {
        float ms = 0;
        PPD_CUDA(cudaEventElapsedTime(&ms, t.start, t.stop));
        tsum_add(c, t.name, ms);
        c->event_pool.push_back(t.start);
        c->event_pool.push_back(t.stop);
    }
    c->sites_eager.clear();
    if (c->graph_ran_since_collect) {
        for (auto &t : c->sites_graph) {
            float ms = 0;
            PPD_CUDA(cudaEventElapsedTime(&ms, t.start, t.stop));
            tsum_add(c, t.name, ms);
        }
        c->graph_ran_since_collect = false;
    }
    return PPD_OK;
}

int ppd_timing_read(ppd_ctx *c, int32_t n, const char **names, double *ms, int64_t *launches, int32_t *n_out) {
    if (!c || !n_out) return fail(PPD_ERR_INVALID_ARG, "ppd_timing_read: NULL argument");
    const int m = (int)std::min<size_t>((size_t)std::max(n, 0), c->tsum.size());
    for (int i = 0; i < m; ++i) {
        if (names) names[i] = c->tsum[i].first;
        if (ms) ms[i] = c->tsum[i].second.first;
        if (launches) launches[i] = c->tsum[i].second.second;
    }
    *n_out = (int32_t)c->tsum.size();
    return PPD_OK;
}

int64_t ppd_launch_count(ppd_ctx *c) { return c ? c->launches : 0; }

int ppd_set_wait_limit(ppd_ctx *c, int64_t polls) {
    if (!c) return fail(PPD_ERR_INVALID_ARG, "ppd_set_wait_limit: NULL context");
    if (polls < 0) return fail(PPD_ERR_INVALID_ARG, "ppd_set_wait_limit: polls < 0");
    DeviceGuard dg_(c->device);
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    c->wait_first = polls;
    drop_graph(c);   // the limit is a kernel argument of the captured iteration
    return PPD_OK;
}

}  // extern "C"
