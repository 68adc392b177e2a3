// Image-side kernels: the primal step of Algorithm 3 (projection onto the
// positive orthant, Section 3.3 Eq. "proj-plus") with the Dirac basis of the
// prior step fused in, deterministic FP64 reductions for the statistics and
// the power iteration, and a scaled copy.
#include "common.cuh"

namespace ppd {

namespace {

constexpr int NT = 256;

template <int NTH> __device__ void cta_sum3(double a, double b, double c, double *out3) {
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

// Primal step of Algorithm 3 with the Dirac basis of the prior step
// (prior weights w0 of Algorithm 1, 1 when w0 is null; kappa here is the
// clip level alpha = kappa ||Psi W||^2 and zeta the effective zeta / ||Psi W||^2):
// u0 <- clip(u0 + w0 xt/3, kappa); ut_all = (w0 u0 + ut)/3;
// xbar = P_C(x - tau (eta g + zeta ut_all)); xt = 2 xbar - x; x = xbar;
// FP64 partials (||xbar - x||^2, ||xbar||^2, ||xbar - x0||^2) per CTA.
// pmask: active set P of Algorithm 3 (Dirac flag first) or null; a Dirac
// basis outside P keeps u0.
template <typename R>
__global__ void __launch_bounds__(NT) k_primal(R *__restrict__ x, R *__restrict__ xt, const R *__restrict__ g,
                                               const R *__restrict__ ut, R *__restrict__ u0,
                                               const R *__restrict__ w0, const R *__restrict__ xtrue, int64_t N,
                                               R tau, R eta, R zeta, R kappa, double *__restrict__ part,
                                               const uint8_t *__restrict__ pmask) {
    // per-thread sums in the working precision, Kahan-compensated, then a
    // fixed-order FP64 reduction across the CTA
    R sd = 0, sx = 0, se = 0, cd = 0, cx = 0, ce = 0;
    auto kadd = [](R &s, R &c, R v) {
        const R y = v - c, t = s + y;
        c = (t - s) - y;
        s = t;
    };
    const R third = R(1.0 / 3.0);
    const bool dirac_on = !pmask || pmask[0];
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < N; e += (int64_t)gridDim.x * NT) {
        const R xo = x[e], xte = xt[e];
        const R wd = w0 ? w0[e] : R(1);
        R un = u0[e];
        if (dirac_on) {
            un = fmin(fmax(un + wd * (xte * third), -kappa), kappa);
            u0[e] = un;
        }
        const R utot = (wd * un + ut[e]) * third;
        const R xb = fmax(R(0), xo - tau * (eta * g[e] + zeta * utot));
        xt[e] = R(2) * xb - xo;
        x[e] = xb;
        const R dd = xb - xo;
        kadd(sd, cd, dd * dd);
        kadd(sx, cx, xb * xb);
        if (xtrue) {
            const R de = xb - xtrue[e];
            kadd(se, ce, de * de);
        }
    }
    cta_sum3<NT>((double)sd - (double)cd, (double)sx - (double)cx, (double)se - (double)ce,
                 part + 3 * (int64_t)blockIdx.x);
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

template <typename R>
__global__ void __launch_bounds__(NT) k_sumsq(const R *__restrict__ in, int64_t n, double *__restrict__ part) {
    double s = 0;
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) {
        const double v = (double)in[e];
        s += v * v;
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

template <typename R> int primal_step(ppd_ctx *c, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "primal", s, &site));
    k_primal<R><<<c->n_prim_blocks, NT, 0, s>>>(static_cast<R *>(c->x), static_cast<R *>(c->xt),
                                                static_cast<const R *>(c->g), static_cast<const R *>(c->ut),
                                                static_cast<R *>(c->u), static_cast<const R *>(c->wgt),
                                                static_cast<const R *>(c->xtrue), c->N, (R)c->tau, (R)c->eta,
                                                (R)(c->zeta / c->psiw2), (R)(c->kappa * c->psiw2), c->prim_part,
                                                c->rand_on ? c->mask_cur + c->d : nullptr);
    return launch_end(c, site, s);
}

int reduce_primal_stats(ppd_ctx *c, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "stats", s, &site));
    k_reduce3<<<1, NT, 0, s>>>(c->prim_part, c->n_prim_blocks, c->stat_out);
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
template int primal_step<float>(ppd_ctx *, cudaStream_t);
template int primal_step<double>(ppd_ctx *, cudaStream_t);
template int sumsq<float>(ppd_ctx *, const float *, int64_t, double *, cudaStream_t);
template int sumsq<double>(ppd_ctx *, const double *, int64_t, double *, cudaStream_t);
template int scale_copy<float>(ppd_ctx *, const float *, float *, int64_t, double, cudaStream_t);
template int scale_copy<double>(ppd_ctx *, const double *, double *, int64_t, double, cudaStream_t);

}  // namespace ppd
