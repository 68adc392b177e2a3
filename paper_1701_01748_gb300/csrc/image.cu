// Image-side kernels: deterministic FP64 reductions for the statistics and
// the power iteration, a scaled copy, the re-weighting kernels, and the
// arguments of the primal step of Algorithm 3 (projection onto the positive
// orthant, Section 3.3 Eq. "proj-plus"), whose kernel is fused with the row
// FFT passes in fft.cu.
#include "common.cuh"

namespace ppd {

namespace {

constexpr int NT = 256;

// Primal step of Algorithm 3 (primal_pixel) over all pixels, grid-stride,
// from g = Phi^dagger v in memory, with FP64 partials per CTA.
template <typename R>
__global__ void __launch_bounds__(NT) k_primal(PrimalArgs<R> P, const R *__restrict__ g, int64_t N,
                                               double *__restrict__ part) {
    PrimalSums<R> acc;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < N; e += (int64_t)gridDim.x * NT)
        primal_pixel(P, e, g[e], acc);
    acc.write(part + 3 * (int64_t)blockIdx.x);
}

__global__ void k_reduce3(const double *__restrict__ part, int n, double *__restrict__ out) {
    double a = 0, b = 0, c = 0;
    for (int i = threadIdx.x; i < n; i += NT) {
        a += part[3 * i];
        b += part[3 * i + 1];
        c += part[3 * i + 2];
    }
    cta_sum3<NT>(a, b, c, out);
}

// Global stopping rule of Algorithm 3 in FP64: relative variation
// sqrt(||x - x_prev||^2 / ||x||^2) below tol and every block residual
// sqrt(resid2_j) within fac eps_j.  One warp.
__global__ void k_stop_flag(const double *__restrict__ stat, const double *__restrict__ resid2,
                            const double *__restrict__ eps, int d, double tol, double fac, int *__restrict__ flag) {
    bool ok = true;
    for (int j = threadIdx.x; j < d; j += 32) ok = ok && sqrt(resid2[j]) <= fac * eps[j];
    ok = __all_sync(0xffffffffu, ok);
    if (threadIdx.x == 0) {
        const bool rv = stat[1] > 0 && sqrt(stat[0] / stat[1]) < tol;
        *flag = (ok && rv) ? 1 : 0;
    }
}

template <typename R>
__global__ void __launch_bounds__(NT) k_sumsq(const R *__restrict__ in, int64_t n, double *__restrict__ part) {
    double s = 0;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) {
        const double v = (double)in[e];
        s += v * v;
    }
    cta_sum3<NT>(s, 0.0, 0.0, part + 3 * (int64_t)blockIdx.x);
}

// Lanczos steps: w -= beta vp with the partials of <w, v>; w -= alpha v
// with the partials of ||w||^2 (FP64 per-CTA sums, fixed order).
template <typename R>
__global__ void __launch_bounds__(NT) k_lz_dot(R *__restrict__ w, const R *__restrict__ vp, const R *__restrict__ v,
                                               int64_t n, R beta, double *__restrict__ part) {
    double s = 0;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) {
        const R we = w[e] - beta * vp[e];
        w[e] = we;
        s += (double)we * (double)v[e];
    }
    cta_sum3<NT>(s, 0.0, 0.0, part + 3 * (int64_t)blockIdx.x);
}

template <typename R>
__global__ void __launch_bounds__(NT) k_lz_orth(R *__restrict__ w, const R *__restrict__ v, int64_t n, R alpha,
                                                double *__restrict__ part) {
    double s = 0;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) {
        const R we = w[e] - alpha * v[e];
        w[e] = we;
        s += (double)we * (double)we;
    }
    cta_sum3<NT>(s, 0.0, 0.0, part + 3 * (int64_t)blockIdx.x);
}

template <typename R> __global__ void k_scale(const R *__restrict__ in, R *__restrict__ out, int64_t n, R a) {
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) out[e] = a * in[e];
}

// Weights of the re-weighted scheme (Eq. "reweighting"), in place over the
// analysis coefficients: w = omega / (omega + |c|).
template <typename R> __global__ void k_reweight(R *__restrict__ cw, int64_t n, R omega) {
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT)
        cw[e] = omega / (omega + fabs(cw[e]));
}

// c <- w^2 c (one application of W^2 inside the power iteration on Psi W^2 Psi^dagger)
template <typename R> __global__ void k_mul_sq(R *__restrict__ c, const R *__restrict__ w, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) {
        const R wv = w[e];
        c[e] = (wv * wv) * c[e];
    }
}

}  // namespace

template <typename R> PrimalArgs<R> primal_args(ppd_ctx *c) {
    PrimalArgs<R> P;
    P.x = static_cast<R *>(c->x);
    P.xt = static_cast<R *>(c->xt);
    P.u0 = static_cast<R *>(c->u);
    P.ut = static_cast<const R *>(c->ut);
    P.w0 = static_cast<const R *>(c->wgt);
    P.xtrue = static_cast<const R *>(c->xtrue);
    P.tau = (R)c->tau;
    P.eta = (R)c->eta;
    P.zeta = (R)(c->zeta / c->psiw2);
    P.kappa = (R)(c->kappa * c->psiw2);
    P.pmask = c->rand_on ? c->mask_cur + c->d : nullptr;
    return P;
}

template <typename R> int primal_step(ppd_ctx *c, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "primal", s, &site));
    k_primal<R><<<c->n_prim_blocks, NT, 0, s>>>(primal_args<R>(c), static_cast<const R *>(c->g), c->N, c->prim_part);
    c->n_stat_parts = c->n_prim_blocks;
    return launch_end(c, site, s);
}

int reduce_primal_stats(ppd_ctx *c, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "stats", s, &site));
    k_reduce3<<<1, NT, 0, s>>>(c->prim_part, c->n_stat_parts, c->stat_out);
    return launch_end(c, site, s);
}

int stop_flag(ppd_ctx *c, double tol, double fac, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "stop_rule", s, &site));
    k_stop_flag<<<1, 32, 0, s>>>(c->stat_out, c->resid2, c->eps_d, c->d, tol, fac, c->stop_flag);
    return launch_end(c, site, s);
}

template <typename R> int sumsq(ppd_ctx *c, const R *in, int64_t n, double *out_dev, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "sumsq", s, &site));
    k_sumsq<R><<<c->n_prim_blocks, NT, 0, s>>>(in, n, c->prim_part);
    PPD_CHECK(launch_end(c, site, s));
    PPD_CHECK(launch_begin(c, "stats", s, &site));
    k_reduce3<<<1, NT, 0, s>>>(c->prim_part, c->n_prim_blocks, out_dev);
    return launch_end(c, site, s);
}

template <typename R> int lanczos_dot(ppd_ctx *c, R *w, const R *vp, const R *v, double beta, double *out_dev,
                                      cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "lanczos", s, &site));
    k_lz_dot<R><<<c->n_prim_blocks, NT, 0, s>>>(w, vp, v, c->N, (R)beta, c->prim_part);
    PPD_CHECK(launch_end(c, site, s));
    PPD_CHECK(launch_begin(c, "stats", s, &site));
    k_reduce3<<<1, NT, 0, s>>>(c->prim_part, c->n_prim_blocks, out_dev);
    return launch_end(c, site, s);
}

template <typename R> int lanczos_orth(ppd_ctx *c, R *w, const R *v, double alpha, double *out_dev, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "lanczos", s, &site));
    k_lz_orth<R><<<c->n_prim_blocks, NT, 0, s>>>(w, v, c->N, (R)alpha, c->prim_part);
    PPD_CHECK(launch_end(c, site, s));
    PPD_CHECK(launch_begin(c, "stats", s, &site));
    k_reduce3<<<1, NT, 0, s>>>(c->prim_part, c->n_prim_blocks, out_dev);
    return launch_end(c, site, s);
}

template int lanczos_dot<float>(ppd_ctx *, float *, const float *, const float *, double, double *, cudaStream_t);
template int lanczos_dot<double>(ppd_ctx *, double *, const double *, const double *, double, double *, cudaStream_t);
template int lanczos_orth<float>(ppd_ctx *, float *, const float *, double, double *, cudaStream_t);
template int lanczos_orth<double>(ppd_ctx *, double *, const double *, double, double *, cudaStream_t);

template <typename R> int scale_copy(ppd_ctx *c, const R *in, R *out, int64_t n, double a, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "scale", s, &site));
    k_scale<R><<<c->n_prim_blocks, NT, 0, s>>>(in, out, n, (R)a);
    return launch_end(c, site, s);
}

template <typename R> int reweight_from(ppd_ctx *c, R *cw, int64_t n, double omega, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "reweight", s, &site));
    k_reweight<R><<<c->n_prim_blocks, NT, 0, s>>>(cw, n, (R)omega);
    return launch_end(c, site, s);
}

template <typename R> int mul_sq(ppd_ctx *c, R *inout, const R *w, int64_t n, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "reweight", s, &site));
    k_mul_sq<R><<<c->n_prim_blocks, NT, 0, s>>>(inout, w, n);
    return launch_end(c, site, s);
}

template int reweight_from<float>(ppd_ctx *, float *, int64_t, double, cudaStream_t);
template int reweight_from<double>(ppd_ctx *, double *, int64_t, double, cudaStream_t);
template int mul_sq<float>(ppd_ctx *, float *, const float *, int64_t, cudaStream_t);
template int mul_sq<double>(ppd_ctx *, double *, const double *, int64_t, cudaStream_t);
template PrimalArgs<float> primal_args<float>(ppd_ctx *);
template PrimalArgs<double> primal_args<double>(ppd_ctx *);
template int primal_step<float>(ppd_ctx *, cudaStream_t);
template int primal_step<double>(ppd_ctx *, cudaStream_t);
template int sumsq<float>(ppd_ctx *, const float *, int64_t, double *, cudaStream_t);
template int sumsq<double>(ppd_ctx *, const double *, int64_t, double *, cudaStream_t);
template int scale_copy<float>(ppd_ctx *, const float *, float *, int64_t, double, cudaStream_t);
template int scale_copy<double>(ppd_ctx *, const double *, double *, int64_t, double, cudaStream_t);

}  // namespace ppd
