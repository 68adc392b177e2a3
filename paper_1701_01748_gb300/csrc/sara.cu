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
constexpr int TSA = 16;                       // analysis: quadrant positions per tile side
constexpr int TS = 8;                         // synthesis: quadrant positions per tile side
constexpr int AEXT = 2 * TSA + MAX_TAPS - 2;  // analysis input tile side (46)
constexpr int SEXT = TS + MAX_TAPS / 2 - 1;   // synthesis quadrant tile side (15)

// periodic index for power-of-two n (two's complement makes the mask exact
// for negative i)
__device__ __forceinline__ int wrap(int i, int n) { return i & (n - 1); }

// low-pass h and high-pass g[k] = (-1)^k h[F-1-k] of basis b, staged in shared memory
template <typename R> __device__ __forceinline__ void stage_filters(R *fh, R *fg, int b, int F) {
    if (threadIdx.x < MAX_TAPS) {
        const int k = threadIdx.x;
        fh[k] = k < F ? filt<R>(b, k) : R(0);
        fg[k] = k < F ? hfilt<R>(b, F, k) : R(0);
    }
}

// One analysis level for all 8 wavelet bases (grid.y = basis), one tile of
// ts x ts positions of each of the 4 quadrants per CTA.  Rows (axis 1) are
// filtered into shared memory, then columns (axis 0).
//   in:   level input, basis b at in + b*in_bstride, row pitch in_pitch
//   LL:   next level's input (compact, pitch h) unless last
//   coef: coefficient images (basis b+1 at coef + (b+1)*N, pitch L), written
//         (mode 0: c = W x / 3) or clip-updated (mode 1: u = clip(u + W x / 3, kappa))
template <typename R>
__global__ void __launch_bounds__(NT) k_sara_ana(const R *__restrict__ in, int in_pitch, int64_t in_bstride, int n,
                                                 int ts, R *__restrict__ ll, int64_t ll_bstride, int last,
                                                 R *__restrict__ coef, int L, int64_t N, int mode, R kappa) {
    __shared__ R tin[AEXT * AEXT];
    __shared__ R rowf[AEXT * 2 * TSA];
    __shared__ R fh[MAX_TAPS], fg[MAX_TAPS];
    const int b = blockIdx.y, F = 2 * (b + 1);
    const int h = n / 2, tpd = h / ts;
    const int R0 = (blockIdx.x / tpd) * ts, C0 = (blockIdx.x % tpd) * ts;
    const int ext = 2 * ts + F - 2;
    const R *src = in + (int64_t)b * in_bstride;
    stage_filters(fh, fg, b, F);
    for (int e = threadIdx.x; e < ext * ext; e += NT) {
        const int i = e / ext, j = e % ext;
        tin[i * AEXT + j] = src[(int64_t)wrap(2 * R0 + i, n) * in_pitch + wrap(2 * C0 + j, n)];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ext * 2 * ts; e += NT) {
        const int i = e / (2 * ts), q = e % (2 * ts);
        const int cc = q % ts;
        const bool hi = q >= ts;
        const R *row = tin + i * AEXT + 2 * cc;
        const R *f = hi ? fg : fh;
        R acc = 0;
        for (int k = 0; k < F; ++k) acc += f[k] * row[k];
        rowf[i * 2 * TSA + q] = acc;
    }
    __syncthreads();
    R *cb = coef + (int64_t)(b + 1) * N;
    for (int e = threadIdx.x; e < 4 * ts * ts; e += NT) {
        const int rq = e / (2 * ts), q = e % (2 * ts);
        const int rr = rq % ts, cc = q % ts;
        const bool hi0 = rq >= ts, hi1 = q >= ts;
        const R *f = hi0 ? fg : fh;
        const R *col = rowf + 2 * rr * 2 * TSA + q;
        R acc = 0;
        for (int k = 0; k < F; ++k) acc += f[k] * col[k * 2 * TSA];
        if (!hi0 && !hi1 && !last) {
            ll[(int64_t)b * ll_bstride + (R0 + rr) * h + C0 + cc] = acc;
        } else {
            R *dst = cb + (int64_t)((hi0 ? h : 0) + R0 + rr) * L + (hi1 ? h : 0) + C0 + cc;
            const R cv = acc * R(1.0 / 3.0);
            if (mode == 0) {
                *dst = cv;
            } else {
                const R u = *dst + cv;
                *dst = fmin(fmax(u, -kappa), kappa);
            }
        }
    }
}

// Load the four quadrant tiles of basis b for the synthesis of the tile whose
// quadrant positions start at (R0, C0): rows/cols R0 - F/2 + 1 ... R0 + ts - 1.
template <typename R>
__device__ __forceinline__ void syn_load(R *qs, const R *cb, const R *sl, int from_coef, int L, int h, int R0,
                                         int C0, int ext, int F) {
    for (int e = threadIdx.x; e < 4 * ext * ext; e += NT) {
        const int qd = e / (ext * ext), r = e % (ext * ext);
        const int i = r / ext, j = r % ext;
        const int gi = wrap(R0 - F / 2 + 1 + i, h), gj = wrap(C0 - F / 2 + 1 + j, h);
        R v;
        if (qd == 0) v = from_coef ? cb[(int64_t)gi * L + gj] : sl[gi * h + gj];
        else if (qd == 1) v = cb[(int64_t)gi * L + h + gj];
        else if (qd == 2) v = cb[(int64_t)(h + gi) * L + gj];
        else v = cb[(int64_t)(h + gi) * L + h + gj];
        qs[qd * SEXT * SEXT + i * SEXT + j] = v;
    }
}

// Inverse along axis 0: tl/th[mm][j] (mm < 2 ts, j < ext) from the quadrants.
template <typename R>
__device__ __forceinline__ void syn_cols(const R *qs, R *tl, R *th, const R *fh, const R *fg, int F, int n, int h,
                                         int R0, int ts, int ext) {
    for (int e = threadIdx.x; e < 2 * ts * ext; e += NT) {
        const int mm = e / ext, j = e % ext;
        const int m = 2 * R0 + mm;
        R sl = 0, sh = 0;
        for (int k = (m & 1); k < F; k += 2) {
            const int ig = wrap(m - k, n) >> 1;
            const int il = wrap(ig - (R0 - F / 2 + 1), h);
            const R a = fh[k], c = fg[k];
            sl += a * qs[0 * SEXT * SEXT + il * SEXT + j] + c * qs[2 * SEXT * SEXT + il * SEXT + j];
            sh += a * qs[1 * SEXT * SEXT + il * SEXT + j] + c * qs[3 * SEXT * SEXT + il * SEXT + j];
        }
        tl[mm * SEXT + j] = sl;
        th[mm * SEXT + j] = sh;
    }
}

// Inverse along axis 1 for output (mm, nn') of the tile.
template <typename R>
__device__ __forceinline__ R syn_row(const R *tl, const R *th, const R *fh, const R *fg, int F, int n, int h, int C0,
                                     int mm, int nnl) {
    const int nn = 2 * C0 + nnl;
    R s = 0;
    for (int j = (nn & 1); j < F; j += 2) {
        const int jg = wrap(nn - j, n) >> 1;
        const int jl = wrap(jg - (C0 - F / 2 + 1), h);
        s += fh[j] * tl[mm * SEXT + jl] + fg[j] * th[mm * SEXT + jl];
    }
    return s;
}

// One synthesis level l > 0 for all 8 bases: out_b (compact pitch n) = W_b^T of
// (LL' block, detail quadrants).  LL' comes from the coefficients at the
// coarsest level (from_coef) or from the coarser level's output sl.
template <typename R>
__global__ void __launch_bounds__(NT) k_sara_syn(const R *__restrict__ coef, int L, int64_t N, const R *__restrict__ sll,
                                                 int from_coef, int64_t sll_bstride, int n, int ts, R *__restrict__ out,
                                                 int64_t out_bstride) {
    __shared__ R qs[4 * SEXT * SEXT];
    __shared__ R tl[2 * TS * SEXT], th[2 * TS * SEXT];
    __shared__ R fh[MAX_TAPS], fg[MAX_TAPS];
    const int b = blockIdx.y, F = 2 * (b + 1);
    const int h = n / 2, tpd = h / ts;
    const int R0 = (blockIdx.x / tpd) * ts, C0 = (blockIdx.x % tpd) * ts;
    const int ext = ts + F / 2 - 1;
    stage_filters(fh, fg, b, F);
    syn_load(qs, coef + (int64_t)(b + 1) * N, sll + (int64_t)b * sll_bstride, from_coef, L, h, R0, C0, ext, F);
    __syncthreads();
    syn_cols(qs, tl, th, fh, fg, F, n, h, R0, ts, ext);
    __syncthreads();
    R *o = out + (int64_t)b * out_bstride;
    for (int e = threadIdx.x; e < 4 * ts * ts; e += NT) {
        const int mm = e / (2 * ts), nnl = e % (2 * ts);
        o[(int64_t)(2 * R0 + mm) * n + 2 * C0 + nnl] = syn_row(tl, th, fh, fg, F, n, h, C0, mm, nnl);
    }
}

// Finest synthesis level, all 8 bases summed in order per output sample.
// mode 0 (operator):  out = scale * (dirac + sum_b W_b^T c_b)
// mode 1 (PPD step):  u0 <- clip(u0 + xt/3, kappa); ut = (u0 + sum_b W_b^T u_b)/3;
//                     xbar = max(0, x - tau (eta g + zeta ut)); xt = 2 xbar - x; x = xbar
//                     with FP64 partial sums (||dx||^2, ||xbar||^2, ||xbar - x0||^2) per CTA.
template <typename R> struct PrimalArgs {
    R *x, *xt, *u0;
    const R *g, *xtrue;
    R tau, eta, zeta, kappa;
    double *part;
};

template <typename R>
__global__ void __launch_bounds__(NT) k_sara_syn0(const R *__restrict__ coef, int L, int64_t N, const R *__restrict__ sll,
                                                  int from_coef, int64_t sll_bstride, int ts, int mode,
                                                  const R *__restrict__ dirac, R scale, R *__restrict__ out,
                                                  PrimalArgs<R> P) {
    __shared__ R qs[4 * SEXT * SEXT];
    __shared__ R tl[2 * TS * SEXT], th[2 * TS * SEXT];
    __shared__ R fh[MAX_TAPS], fg[MAX_TAPS];
    __shared__ double red[3][NT / 32];
    const int n = L, h = n / 2, tpd = h / ts;
    const int R0 = (blockIdx.x / tpd) * ts, C0 = (blockIdx.x % tpd) * ts;
    constexpr int PER = (4 * TS * TS + NT - 1) / NT;
    R acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0;
    for (int b = 0; b < N_WAVELETS; ++b) {
        const int F = 2 * (b + 1), ext = ts + F / 2 - 1;
        stage_filters(fh, fg, b, F);
        syn_load(qs, coef + (int64_t)(b + 1) * N, sll + (int64_t)b * sll_bstride, from_coef, L, h, R0, C0, ext, F);
        __syncthreads();
        syn_cols(qs, tl, th, fh, fg, F, n, h, R0, ts, ext);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + k * NT;
            if (e < 4 * ts * ts) acc[k] += syn_row(tl, th, fh, fg, F, n, h, C0, e / (2 * ts), e % (2 * ts));
        }
        __syncthreads();
    }
    double sd = 0, sx = 0, se = 0;
    const R third = R(1.0 / 3.0);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * NT;
        if (e >= 4 * ts * ts) continue;
        const int64_t idx = (int64_t)(2 * R0 + e / (2 * ts)) * L + 2 * C0 + e % (2 * ts);
        if (mode == 0) {
            out[idx] = scale * ((dirac ? dirac[idx] : R(0)) + acc[k]);
        } else {
            const R xo = P.x[idx], xte = P.xt[idx];
            R un = P.u0[idx] + xte * third;
            un = fmin(fmax(un, -P.kappa), P.kappa);
            P.u0[idx] = un;
            const R utot = (un + acc[k]) * third;
            const R xb = fmax(R(0), xo - P.tau * (P.eta * P.g[idx] + P.zeta * utot));
            P.xt[idx] = R(2) * xb - xo;
            P.x[idx] = xb;
            const double dd = (double)xb - (double)xo;
            sd += dd * dd;
            sx += (double)xb * (double)xb;
            if (P.xtrue) {
                const double de = (double)xb - (double)P.xtrue[idx];
                se += de * de;
            }
        }
    }
    if (mode == 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sd += __shfl_down_sync(0xffffffffu, sd, o);
            sx += __shfl_down_sync(0xffffffffu, sx, o);
            se += __shfl_down_sync(0xffffffffu, se, o);
        }
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            red[0][wid] = sd;
            red[1][wid] = sx;
            red[2][wid] = se;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a0 = 0, a1 = 0, a2 = 0;
            for (int i = 0; i < NT / 32; ++i) {
                a0 += red[0][i];
                a1 += red[1][i];
                a2 += red[2][i];
            }
            P.part[3 * (int64_t)blockIdx.x] = a0;
            P.part[3 * (int64_t)blockIdx.x + 1] = a1;
            P.part[3 * (int64_t)blockIdx.x + 2] = a2;
        }
    }
}

template <typename R> __global__ void k_scale_copy(const R *__restrict__ in, R *__restrict__ out, int64_t n, R a) {
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) out[e] = a * in[e];
}

inline unsigned nblk(int64_t work) { return (unsigned)std::min<int64_t>((work + NT - 1) / NT, 152 * 8); }
inline int tile_side(int h) { return h < TS ? h : TS; }

inline int tile_side_ana(int h) { return h < TSA ? h : TSA; }

// Analysis of all levels (tiled).  mode 0 writes c = W x / 3, mode 1
// clip-updates u.
template <typename R> int analysis_all(ppd_ctx *c, const R *x, R *coef, int mode, cudaStream_t s) {
    const int L = c->L0;
    const int64_t N = c->N;
    R *ll[2] = {static_cast<R *>(c->wtmp), static_cast<R *>(c->wtmp) + (int64_t)N_WAVELETS * (L / 2) * (L / 2)};
    const int64_t ll_stride = (int64_t)(L / 2) * (L / 2);
    int site;
    for (int l = 0; l < c->levels; ++l) {
        const int n = L >> l, h = n / 2, ts = tile_side_ana(h);
        const bool last = (l == c->levels - 1);
        const R *in = l == 0 ? x : ll[(l - 1) & 1];
        const int pitch = l == 0 ? L : n;
        const int64_t bstride = l == 0 ? 0 : ll_stride;
        PPD_CHECK(launch_begin(c, "sara_analysis", s, &site));
        k_sara_ana<R><<<dim3((h / ts) * (h / ts), N_WAVELETS), NT, 0, s>>>(in, pitch, bstride, n, ts, ll[l & 1],
                                                                           ll_stride, last, coef, L, N, mode,
                                                                           (R)c->kappa);
        PPD_CHECK(launch_end(c, site, s));
    }
    return PPD_OK;
}

// Synthesis of the 8 wavelet bases, levels coarsest .. 1 (tiled); returns
// the buffer holding the LL' block of level 0.
template <typename R> int synthesis_levels(ppd_ctx *c, const R *coef, const R **ll0, cudaStream_t s) {
    const int L = c->L0;
    const int64_t N = c->N;
    const int64_t st = (int64_t)(L / 2) * (L / 2);
    R *buf[2] = {static_cast<R *>(c->wtmp2), static_cast<R *>(c->wtmp2) + (int64_t)N_WAVELETS * st};
    const R *prev = nullptr;
    int site, k = 0;
    for (int l = c->levels - 1; l >= 1; --l, ++k) {
        const int n = L >> l, h = n / 2, ts = tile_side(h);
        const bool coarsest = (l == c->levels - 1);
        PPD_CHECK(launch_begin(c, "sara_synthesis", s, &site));
        k_sara_syn<R><<<dim3((h / ts) * (h / ts), N_WAVELETS), NT, 0, s>>>(coef, L, N, coarsest ? coef : prev,
                                                                           coarsest ? 1 : 0, st, n, ts, buf[k & 1],
                                                                           st);
        PPD_CHECK(launch_end(c, site, s));
        prev = buf[k & 1];
    }
    *ll0 = prev;
    return PPD_OK;
}

template <typename R>
int synthesis_final(ppd_ctx *c, const R *coef, const R *ll0, int mode, const R *dirac, R scale, R *out,
                    cudaStream_t s) {
    const int L = c->L0;
    const int h = L / 2, ts = tile_side(h);
    const int64_t st = (int64_t)(L / 2) * (L / 2);
    PrimalArgs<R> P{};
    if (mode == 1) {
        P.x = static_cast<R *>(c->x);
        P.xt = static_cast<R *>(c->xt);
        P.u0 = static_cast<R *>(c->u);
        P.g = static_cast<const R *>(c->g);
        P.xtrue = static_cast<const R *>(c->xtrue);
        P.tau = (R)c->tau;
        P.eta = (R)c->eta;
        P.zeta = (R)c->zeta;
        P.kappa = (R)c->kappa;
        P.part = c->prim_part;
    }
    const bool from_coef = ll0 == nullptr;   // levels == 1: LL' straight from the coefficients
    int site;
    PPD_CHECK(launch_begin(c, mode == 1 ? "sara_synthesis_primal" : "sara_synthesis", s, &site));
    k_sara_syn0<R><<<(h / ts) * (h / ts), NT, 0, s>>>(coef, L, c->N, from_coef ? coef : ll0, from_coef ? 1 : 0, st, ts,
                                                        mode, dirac, scale, out, P);
    return launch_end(c, site, s);
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
    return analysis_all<R>(c, x, coef, 0, s);
}

template <typename R> int psi_synthesis(ppd_ctx *c, const R *coef, R *x, cudaStream_t s) {
    const R *ll0 = nullptr;
    PPD_CHECK(synthesis_levels<R>(c, coef, &ll0, s));
    return synthesis_final<R>(c, coef, ll0, 0, coef, R(1.0 / 3.0), x, s);
}

// Prior dual step of Algorithm 3 for the 8 wavelet bases up to the level-0
// synthesis: u_b <- clip(u_b + Psi_b^dagger xt, kappa), then the synthesis of
// levels coarsest .. 1.  Needs only xt and u, so it can run beside the data
// branch of the iteration.
template <typename R> int sara_prior_branch(ppd_ctx *c, const R **ll0, cudaStream_t s) {
    R *u = static_cast<R *>(c->u);
    PPD_CHECK(analysis_all<R>(c, static_cast<const R *>(c->xt), u, 1, s));
    return synthesis_levels<R>(c, u, ll0, s);
}

// Level-0 synthesis summed over the bases with the Dirac basis, fused with
// the primal step (needs g = Phi^dagger v from the data branch).
template <typename R> int sara_primal(ppd_ctx *c, const R *ll0, cudaStream_t s) {
    return synthesis_final<R>(c, static_cast<const R *>(c->u), ll0, 1, nullptr, R(1), nullptr, s);
}

int sara_primal_blocks(ppd_ctx *c) {
    const int h = c->L0 / 2, ts = tile_side(h);
    return (h / ts) * (h / ts);
}

template int psi_analysis<float>(ppd_ctx *, const float *, float *, cudaStream_t);
template int psi_analysis<double>(ppd_ctx *, const double *, double *, cudaStream_t);
template int psi_synthesis<float>(ppd_ctx *, const float *, float *, cudaStream_t);
template int psi_synthesis<double>(ppd_ctx *, const double *, double *, cudaStream_t);
template int sara_prior_branch<float>(ppd_ctx *, const float **, cudaStream_t);
template int sara_prior_branch<double>(ppd_ctx *, const double **, cudaStream_t);
template int sara_primal<float>(ppd_ctx *, const float *, cudaStream_t);
template int sara_primal<double>(ppd_ctx *, const double *, cudaStream_t);

}  // namespace ppd
