// SARA dictionary Psi = (1/3) [Dirac, db1, ..., db8] (Section 2.2, Section
// 5.1): separable periodic 2-D DWT, 4 levels, rows then columns per level,
// Mallat quadrant layout per basis; and the prior dual step of Algorithm 3,
// u_i <- (I - S_kappa)(u_i + Psi_i^dagger xt) = clip(u_i + Psi_i^dagger xt, +-kappa),
// fused into the analysis output.
//
// The eight wavelet bases run together (grid.z = basis); every pass maps one
// thread to one output sample and reads its filter taps through the L1/L2.
// Filters are derived on the host by minimum-phase spectral factorisation
// (Daubechies 1988) with a Durand-Kerner root finder.
#include <cmath>
#include <algorithm>
#include <complex>

#include "common.cuh"

namespace ppd {

__constant__ float c_filt_f[N_WAVELETS][MAX_TAPS];
__constant__ double c_filt_d[N_WAVELETS][MAX_TAPS];

namespace {

template <typename R> __device__ __forceinline__ R filt(int b, int k);
template <> __device__ __forceinline__ float filt<float>(int b, int k) { return c_filt_f[b][k]; }
template <> __device__ __forceinline__ double filt<double>(int b, int k) { return c_filt_d[b][k]; }

// high-pass g[k] = (-1)^k h[F-1-k]
template <typename R> __device__ __forceinline__ R hfilt(int b, int F, int k) {
    const R v = filt<R>(b, F - 1 - k);
    return (k & 1) ? -v : v;
}

constexpr int NT = 256;

// analysis along rows of an n x n block: out[r][m] = [a | d]
template <typename R>
__global__ void k_ana_rows(const R *__restrict__ x, int x_pitch, int x_stride_basis, R *__restrict__ out, int n,
                           int64_t out_stride_basis) {
    const int b = blockIdx.z, F = 2 * (b + 1);
    const R *in = x + (int64_t)b * x_stride_basis;
    R *o = out + (int64_t)b * out_stride_basis;
    const int h = n / 2;
    for (int e = blockIdx.x * NT + threadIdx.x; e < n * n; e += gridDim.x * NT) {
        const int r = e / n, m = e % n;
        const int mm = m < h ? m : m - h;
        const R *row = in + (int64_t)r * x_pitch;
        R s = 0;
        if (m < h) {
            for (int k = 0; k < F; ++k) s += filt<R>(b, k) * row[(2 * mm + k) % n];
        } else {
            for (int k = 0; k < F; ++k) s += hfilt<R>(b, F, k) * row[(2 * mm + k) % n];
        }
        o[e] = s;
    }
}

// analysis along columns; LL quadrant to ll (compact, pitch n/2) unless last
// level, every other coefficient (times 1/3) to coef[b+1] (pitch L):
// mode 0 writes it, mode 1 applies u = clip(u + c, -kappa, kappa).
template <typename R>
__global__ void k_ana_cols(const R *__restrict__ t, int64_t t_stride_basis, int n, R *__restrict__ ll,
                           int64_t ll_stride_basis, int last, R *__restrict__ coef, int L, int64_t N, int mode,
                           R kappa) {
    const int b = blockIdx.z, F = 2 * (b + 1);
    const R *in = t + (int64_t)b * t_stride_basis;
    const int h = n / 2;
    R *cb = coef + (int64_t)(b + 1) * N;
    for (int e = blockIdx.x * NT + threadIdx.x; e < n * n; e += gridDim.x * NT) {
        const int r = e / n, c = e % n;
        const int rr = r < h ? r : r - h;
        R s = 0;
        if (r < h) {
            for (int k = 0; k < F; ++k) s += filt<R>(b, k) * in[(int64_t)((2 * rr + k) % n) * n + c];
        } else {
            for (int k = 0; k < F; ++k) s += hfilt<R>(b, F, k) * in[(int64_t)((2 * rr + k) % n) * n + c];
        }
        if (r < h && c < h && !last) {
            ll[(int64_t)b * ll_stride_basis + r * h + c] = s;
        } else {
            const R cv = s * R(1.0 / 3.0);
            R *dst = cb + (int64_t)r * L + c;
            if (mode == 0) {
                *dst = cv;
            } else {
                const R u = *dst + cv;
                *dst = fmin(fmax(u, -kappa), kappa);
            }
        }
    }
}

// synthesis along columns: out[r][c] (compact pitch n) from the A rows
// (top h rows: the LL' block for c < h, coefficients otherwise) and D rows.
template <typename R>
__global__ void k_syn_cols(const R *__restrict__ coef, int L, int64_t N, const R *__restrict__ sll, int sll_from_coef,
                           int64_t sll_stride_basis, int n, R *__restrict__ out, int64_t out_stride_basis) {
    const int b = blockIdx.z, F = 2 * (b + 1);
    const int h = n / 2;
    const R *cb = coef + (int64_t)(b + 1) * N;
    const R *sl = sll + (int64_t)b * sll_stride_basis;
    R *o = out + (int64_t)b * out_stride_basis;
    for (int e = blockIdx.x * NT + threadIdx.x; e < n * n; e += gridDim.x * NT) {
        const int r = e / n, c = e % n;
        R s = 0;
        for (int k = (r & 1); k < F; k += 2) {
            const int i = ((r - k) % n + n) % n / 2;
            R av;
            if (c < h) av = sll_from_coef ? cb[(int64_t)i * L + c] : sl[i * h + c];
            else av = cb[(int64_t)i * L + c];
            const R dv = cb[(int64_t)(i + h) * L + c];
            s += filt<R>(b, k) * av + hfilt<R>(b, F, k) * dv;
        }
        o[e] = s;
    }
}

// synthesis along rows: out[r][m] from [a | d] of t (compact pitch n).
template <typename R>
__global__ void k_syn_rows(const R *__restrict__ t, int64_t t_stride_basis, int n, R *__restrict__ out,
                           int64_t out_stride_basis) {
    const int b = blockIdx.z, F = 2 * (b + 1);
    const int h = n / 2;
    const R *in = t + (int64_t)b * t_stride_basis;
    R *o = out + (int64_t)b * out_stride_basis;
    for (int e = blockIdx.x * NT + threadIdx.x; e < n * n; e += gridDim.x * NT) {
        const int r = e / n, m = e % n;
        const R *row = in + (int64_t)r * n;
        R s = 0;
        for (int k = (m & 1); k < F; k += 2) {
            const int i = ((m - k) % n + n) % n / 2;
            s += filt<R>(b, k) * row[i] + hfilt<R>(b, F, k) * row[i + h];
        }
        o[e] = s;
    }
}

// last synthesis row pass for all bases together:
// out = scale * (dirac + sum_b W_b^T u_b), summed in basis order.
template <typename R>
__global__ void k_syn_rows_sum(const R *__restrict__ t, int64_t t_stride_basis, int n, const R *__restrict__ dirac,
                               R scale, R *__restrict__ out) {
    const int h = n / 2;
    for (int e = blockIdx.x * NT + threadIdx.x; e < n * n; e += gridDim.x * NT) {
        const int r = e / n, m = e % n;
        R tot = dirac ? dirac[e] : R(0);
        for (int b = 0; b < N_WAVELETS; ++b) {
            const int F = 2 * (b + 1);
            const R *row = t + (int64_t)b * t_stride_basis + (int64_t)r * n;
            R s = 0;
            for (int k = (m & 1); k < F; k += 2) {
                const int i = ((m - k) % n + n) % n / 2;
                s += filt<R>(b, k) * row[i] + hfilt<R>(b, F, k) * row[i + h];
            }
            tot += s;
        }
        out[e] = scale * tot;
    }
}

template <typename R> __global__ void k_scale_copy(const R *__restrict__ in, R *__restrict__ out, int64_t n, R a) {
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) out[e] = a * in[e];
}

inline unsigned nblk(int64_t work) { return (unsigned)std::min<int64_t>((work + NT - 1) / NT, 152 * 8); }

// Psi_b^dagger for b = 1..8 (times 1/3) into coef[b] (mode 0), or the fused
// clip update of u (mode 1).  x has pitch L.
template <typename R> int analysis_core(ppd_ctx *c, const R *x, R *coef, int mode, cudaStream_t s) {
    const int L = c->L0;
    const int64_t N = c->N;
    R *tmp = static_cast<R *>(c->wtmp);          // 8 x L^2
    R *ll = static_cast<R *>(c->wtmp2);          // 8 x (L/2)^2
    const int64_t ll_stride = (int64_t)(L / 2) * (L / 2);
    int site;
    for (int l = 0; l < c->levels; ++l) {
        const int n = L >> l;
        const bool last = (l == c->levels - 1);
        PPD_CHECK(launch_begin(c, "sara_ana_rows", s, &site));
        if (l == 0) k_ana_rows<R><<<dim3(nblk((int64_t)n * n), 1, N_WAVELETS), NT, 0, s>>>(x, L, 0, tmp, n, N);
        else k_ana_rows<R><<<dim3(nblk((int64_t)n * n), 1, N_WAVELETS), NT, 0, s>>>(ll, n, (int)ll_stride, tmp, n, N);
        PPD_CHECK(launch_end(c, site, s));
        PPD_CHECK(launch_begin(c, "sara_ana_cols", s, &site));
        k_ana_cols<R><<<dim3(nblk((int64_t)n * n), 1, N_WAVELETS), NT, 0, s>>>(tmp, N, n, ll, ll_stride, last, coef, L,
                                                                               N, mode, (R)c->kappa);
        PPD_CHECK(launch_end(c, site, s));
    }
    return PPD_OK;
}

// sum over wavelet bases of W_b^T coef[b+1], plus scale*dirac -> out
template <typename R> int synthesis_core(ppd_ctx *c, const R *coef, const R *dirac, R scale, R *out, cudaStream_t s) {
    const int L = c->L0;
    const int64_t N = c->N;
    R *tmp = static_cast<R *>(c->wtmp);                          // 8 x L^2
    R *sl = static_cast<R *>(c->wtmp2) + (int64_t)N_WAVELETS * (L / 2) * (L / 2);   // 8 x (L/2)^2
    const int64_t sl_stride = (int64_t)(L / 2) * (L / 2);
    int site;
    for (int l = c->levels - 1; l >= 0; --l) {
        const int n = L >> l;
        const bool coarsest = (l == c->levels - 1);
        PPD_CHECK(launch_begin(c, "sara_syn_cols", s, &site));
        k_syn_cols<R><<<dim3(nblk((int64_t)n * n), 1, N_WAVELETS), NT, 0, s>>>(coef, L, N, sl, coarsest ? 1 : 0,
                                                                               sl_stride, n, tmp, N);
        PPD_CHECK(launch_end(c, site, s));
        PPD_CHECK(launch_begin(c, "sara_syn_rows", s, &site));
        if (l > 0) k_syn_rows<R><<<dim3(nblk((int64_t)n * n), 1, N_WAVELETS), NT, 0, s>>>(tmp, N, n, sl, sl_stride);
        else k_syn_rows_sum<R><<<nblk((int64_t)n * n), NT, 0, s>>>(tmp, N, n, dirac, scale, out);
        PPD_CHECK(launch_end(c, site, s));
    }
    return PPD_OK;
}

// Durand-Kerner roots of the polynomial with real coefficients a (ascending).
std::vector<std::complex<double>> poly_roots(const std::vector<double> &a) {
    using cd = std::complex<double>;
    const int n = (int)a.size() - 1;
    std::vector<cd> r(n);
    const cd seed(0.4, 0.9);
    for (int i = 0; i < n; ++i) r[i] = std::pow(seed, i);
    auto eval = [&](cd z) {
        cd s = 0;
        for (int k = n; k >= 0; --k) s = s * z + a[k];
        return s / a[n];
    };
    for (int it = 0; it < 2000; ++it) {
        double delta = 0;
        for (int i = 0; i < n; ++i) {
            cd den = 1;
            for (int j = 0; j < n; ++j)
                if (j != i) den *= (r[i] - r[j]);
            cd step = eval(r[i]) / den;
            r[i] -= step;
            delta = std::max(delta, std::abs(step));
        }
        if (delta < 1e-15) break;
    }
    // Newton polish on the original polynomial
    for (int i = 0; i < n; ++i) {
        for (int it = 0; it < 5; ++it) {
            cd p = 0, dp = 0;
            for (int k = n; k >= 0; --k) {
                dp = dp * r[i] + p;
                p = p * r[i] + a[k];
            }
            if (std::abs(dp) > 0) r[i] -= p / dp;
        }
    }
    return r;
}

}  // namespace

// db_p low-pass filter: |m0|^2 = cos^{2p} P(sin^2), P(y) = sum_{k<p} C(p-1+k,k) y^k;
// roots y of P -> z from sin^2(xi/2) = (2 - z - 1/z)/4 keeping |z| < 1;
// h = coefficients of (1+z)^p prod (z - z_r), scaled to sum sqrt(2), larger end first.
std::vector<double> daubechies(int p) {
    using cd = std::complex<double>;
    if (p == 1) return {1.0 / std::sqrt(2.0), 1.0 / std::sqrt(2.0)};
    std::vector<double> a(p);
    for (int k = 0; k < p; ++k) {
        double cb = 1.0;   // C(p-1+k, k)
        for (int i = 1; i <= k; ++i) cb = cb * (p - 1 + i) / i;
        a[k] = cb;
    }
    std::vector<cd> poly{1.0};
    auto mul = [&](cd c0, cd c1) {   // poly *= (c0 + c1 X) in coefficient-sequence form
        std::vector<cd> out(poly.size() + 1, 0.0);
        for (size_t i = 0; i < poly.size(); ++i) {
            out[i] += poly[i] * c0;
            out[i + 1] += poly[i] * c1;
        }
        poly.swap(out);
    };
    for (int i = 0; i < p; ++i) mul(1.0, 1.0);
    for (cd y : poly_roots(a)) {
        cd aa = 1.0 - 2.0 * y;
        cd disc = std::sqrt(aa * aa - 1.0);
        cd z1 = aa + disc, z2 = aa - disc;
        cd zr = std::abs(z1) < std::abs(z2) ? z1 : z2;
        mul(1.0, -zr);
    }
    std::vector<double> h(poly.size());
    double sum = 0;
    for (size_t i = 0; i < poly.size(); ++i) {
        h[i] = poly[i].real();
        sum += h[i];
    }
    for (double &v : h) v *= std::sqrt(2.0) / sum;
    if (std::abs(h.front()) < std::abs(h.back())) std::reverse(h.begin(), h.end());
    return h;
}

int make_filters(ppd_ctx *c) {
    (void)c;
    double hd[N_WAVELETS][MAX_TAPS] = {};
    float hf[N_WAVELETS][MAX_TAPS] = {};
    for (int b = 0; b < N_WAVELETS; ++b) {
        std::vector<double> h = daubechies(b + 1);
        for (size_t k = 0; k < h.size(); ++k) {
            hd[b][k] = h[k];
            hf[b][k] = (float)h[k];
        }
    }
    PPD_CUDA(cudaMemcpyToSymbol(c_filt_d, hd, sizeof(hd)));
    PPD_CUDA(cudaMemcpyToSymbol(c_filt_f, hf, sizeof(hf)));
    return PPD_OK;
}

template <typename R> int psi_analysis(ppd_ctx *c, const R *x, R *coef, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "sara_dirac", s, &site));
    k_scale_copy<R><<<nblk(c->N), NT, 0, s>>>(x, coef, c->N, R(1.0 / 3.0));
    PPD_CHECK(launch_end(c, site, s));
    return analysis_core<R>(c, x, coef, 0, s);
}

template <typename R> int psi_synthesis(ppd_ctx *c, const R *coef, R *x, cudaStream_t s) {
    return synthesis_core<R>(c, coef, coef, R(1.0 / 3.0), x, s);
}

// Prior dual step for the 8 wavelet bases and synthesis of their sum:
// u_b <- clip(u_b + Psi_b^dagger xt, kappa); ut <- sum_b W_b^T u_b (the Dirac
// basis and the 1/3 are applied in the primal step).
template <typename R> int sara_dual_step(ppd_ctx *c, cudaStream_t s) {
    R *u = static_cast<R *>(c->u);
    PPD_CHECK(analysis_core<R>(c, static_cast<const R *>(c->xt), u, 1, s));
    return synthesis_core<R>(c, u, nullptr, R(1), static_cast<R *>(c->ut), s);
}

template int psi_analysis<float>(ppd_ctx *, const float *, float *, cudaStream_t);
template int psi_analysis<double>(ppd_ctx *, const double *, double *, cudaStream_t);
template int psi_synthesis<float>(ppd_ctx *, const float *, float *, cudaStream_t);
template int psi_synthesis<double>(ppd_ctx *, const double *, double *, cudaStream_t);
template int sara_dual_step<float>(ppd_ctx *, cudaStream_t);
template int sara_dual_step<double>(ppd_ctx *, cudaStream_t);

}  // namespace ppd
