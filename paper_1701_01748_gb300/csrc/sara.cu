// SARA dictionary Psi = (1/3) [Dirac, db1, ..., db8] (Section 2.2, Section
// 5.1): separable periodic 2-D DWT, 4 levels, rows then columns per level,
// Mallat quadrant layout per basis; and the prior dual step of Algorithm 3,
// u_i <- (I - S_alpha)(u_i + W_i Psi_i^dagger xt) = clip(u_i + W_i Psi_i^dagger xt, +-alpha),
// fused into the analysis output, with the prior weights W_i of the
// re-weighted scheme (Algorithm 1; W = I unless set) and the clip level
// alpha = kappa ||Psi W||_S^2.  D_b below is the orthonormal DWT of basis b.
//
// The eight wavelet bases run together (grid.y = basis); the filter taps
// sit in registers, the level tiles in shared memory.  Each filter pass
// reads an input window once for every output that uses it: the analysis
// forms the low (h) and high (g) half of a position together, the synthesis
// an even and an odd output sample together (they read the same inputs with
// the even and the odd taps).  Filters are derived on the host by
// minimum-phase spectral factorisation (Daubechies 1988) with a
// Durand-Kerner root finder.
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
static_assert(NT == 4 * TS * TS, "one synthesis output per thread");
static_assert(TSA % (NT / 32) == 0 && AEXT % 2 == 0, "analysis: row pairs per warp, even tile pitch");

// periodic index i mod n (i may be negative); indices inside [0, n) are
// the common case and skip the division
__device__ __forceinline__ int wrap(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Filter taps of basis b in registers: h[k] and g[k] = (-1)^k h[F-1-k].
template <typename R, int F> struct Taps {
    R h[F], g[F];
    __device__ __forceinline__ explicit Taps(int b) {
#pragma unroll
        for (int k = 0; k < F; ++k) {
            h[k] = filt<R>(b, k);
            g[k] = hfilt<R>(b, F, k);
        }
    }
};

// ------------------------------------------------------------- analysis
// One tile of TSA x TSA positions of each of the 4 quadrants of one level,
// one basis (filter length F); the level input is n0 x n1, its quadrants
// h0 x h1.  Rows (axis 1) are filtered into shared memory, then columns
// (axis 0).  Tiles reaching past h0 or h1 (levels smaller than a tile, or
// sides that are not multiples of TSA) skip the positions outside.
template <typename R, int F>
__device__ __forceinline__ void ana_tile(const R *__restrict__ src, int in_pitch, int n0, int n1, int R0, int C0,
                                         R *__restrict__ ll, int last, R *__restrict__ cb,
                                         const R *__restrict__ wb, int L1, int mode, R kappa, int b, R *tin,
                                         R *rowf) {
    constexpr int EXT = 2 * TSA + F - 2;
    constexpr int NQ = 2 * TSA / (NT / 32);   // output rows per warp in the column pass
    const Taps<R, F> f(b);
    const int h0 = n0 >> 1, h1 = n1 >> 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cc = lane & (TSA - 1);
    const bool hi1 = lane >= TSA;
    // the coefficients this thread clip-updates (and their weights) are
    // loaded before the input tile, so both global round trips overlap
    R pu[NQ], pw[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int rq = warp + k * (NT / 32), rr = rq & (TSA - 1);
        const bool hi0 = rq >= TSA;
        pu[k] = R(0);
        pw[k] = R(1);
        if (mode != 0 && R0 + rr < h0 && C0 + cc < h1 && (hi0 || hi1 || last)) {
            const int64_t off = (int64_t)((hi0 ? h0 : 0) + R0 + rr) * L1 + (hi1 ? h1 : 0) + C0 + cc;
            pu[k] = cb[off];
            if (wb) pw[k] = wb[off];
        }
    }
    // the input tile: every load issued before the first store
    constexpr int NR = (EXT + NT / 32 - 1) / (NT / 32);
    R tv[NR][2];
    const int j1 = wrap(2 * C0 + lane, n1), j2 = wrap(2 * C0 + lane + 32, n1);
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int i = warp + k * (NT / 32);
        if (i < EXT) {
            const R *row = src + (int64_t)wrap(2 * R0 + i, n0) * in_pitch;
            tv[k][0] = row[j1];
            if (lane + 32 < EXT) tv[k][1] = row[j2];
        }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int i = warp + k * (NT / 32);
        if (i < EXT) {
            tin[i * AEXT + lane] = tv[k][0];
            if (lane + 32 < EXT) tin[i * AEXT + lane + 32] = tv[k][1];
        }
    }
    __syncthreads();
    {   // rows: thread (row i, position q) forms both halves, low (h) into
        // column q and high (g) into column TSA + q, from one pass over its F
        // inputs, read two at a time (even offsets: 8-byte / 16-byte aligned)
        const int q = threadIdx.x & (TSA - 1);
        for (int i = threadIdx.x / TSA; i < EXT; i += NT / TSA) {
            const R *row = tin + i * AEXT + 2 * q;
            R lo = 0, hi = 0;
#pragma unroll
            for (int k = 0; k < F; k += 2) {
                const auto v = *reinterpret_cast<const typename Cplx<R>::T *>(row + k);
                lo += f.h[k] * v.x;
                hi += f.g[k] * v.x;
                lo += f.h[k + 1] * v.y;
                hi += f.g[k + 1] * v.y;
            }
            rowf[i * 2 * TSA + q] = lo;
            rowf[i * 2 * TSA + TSA + q] = hi;
        }
    }
    __syncthreads();
    // columns: warp = output row rr of both halves (low h: quadrant row rr,
    // high g: row TSA + rr), lane = column of the row-filtered tile
    auto emit = [&](int rr, bool hi0, R acc, R u0, R w0) {
        if (R0 + rr >= h0 || C0 + cc >= h1) return;   // outside the quadrant
        if (!hi0 && !hi1 && !last) {
            ll[(R0 + rr) * h1 + C0 + cc] = acc;
        } else {
            const int64_t off = (int64_t)((hi0 ? h0 : 0) + R0 + rr) * L1 + (hi1 ? h1 : 0) + C0 + cc;
            R *dst = cb + off;
            const R cv = acc * R(1.0 / 3.0);
            if (mode == 0) {
                *dst = cv;
            } else {
                const R u = u0 + (wb ? w0 * cv : cv);
                *dst = fmin(fmax(u, -kappa), kappa);
            }
        }
    };
#pragma unroll
    for (int kq = 0; kq < NQ / 2; ++kq) {
        const int rr = warp + kq * (NT / 32);
        const R *col = rowf + 2 * rr * 2 * TSA + lane;
        R lo = 0, hi = 0;
#pragma unroll
        for (int k = 0; k < F; ++k) {
            const R v = col[k * 2 * TSA];
            lo += f.h[k] * v;
            hi += f.g[k] * v;
        }
        emit(rr, false, lo, pu[kq], pw[kq]);
        emit(rr, true, hi, pu[kq + NQ / 2], pw[kq + NQ / 2]);
    }
}

// One analysis level for all 8 wavelet bases (grid.y = basis).
//   in:   level input n0 x n1, basis b at in + b*in_bstride, row pitch in_pitch
//   ll:   next level's input (compact, pitch h1) unless last
//   coef: coefficient images (basis b+1 at coef + (b+1)*N, pitch L1), written
//         (mode 0: c = D x / 3) or clip-updated (mode 1: u = clip(u + w D x / 3, kappa))
//   wgt:  prior weights (same layout as coef) or null (w = 1)
//   pmask: active set P of Algorithm 3 (9 flags, Dirac first) or null; in
//         mode 1 a basis outside P keeps u_b and is skipped at every level
template <typename R>
__global__ void __launch_bounds__(NT) k_sara_ana(const R *__restrict__ in, int in_pitch, int64_t in_bstride, int n0,
                                                 int n1, R *__restrict__ ll, int64_t ll_bstride, int last,
                                                 R *__restrict__ coef, const R *__restrict__ wgt, int L1, int64_t N,
                                                 int mode, R kappa, const uint8_t *__restrict__ pmask) {
    __shared__ __align__(16) R tin[AEXT * AEXT];
    __shared__ R rowf[AEXT * 2 * TSA];
    const int b = blockIdx.y;
    pdl_enter();
    if (mode == 1 && pmask && !pmask[b + 1]) return;
    const int tpd1 = (n1 / 2 + TSA - 1) / TSA;
    const int R0 = (blockIdx.x / tpd1) * TSA, C0 = (blockIdx.x % tpd1) * TSA;
    const R *src = in + (int64_t)b * in_bstride;
    R *lb = ll + (int64_t)b * ll_bstride;
    R *cb = coef + (int64_t)(b + 1) * N;
    const R *wb = wgt ? wgt + (int64_t)(b + 1) * N : nullptr;
    switch (b) {
        case 0: ana_tile<R, 2>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
        case 1: ana_tile<R, 4>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
        case 2: ana_tile<R, 6>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
        case 3: ana_tile<R, 8>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
        case 4: ana_tile<R, 10>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
        case 5: ana_tile<R, 12>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
        case 6: ana_tile<R, 14>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
        default: ana_tile<R, 16>(src, in_pitch, n0, n1, R0, C0, lb, last, cb, wb, L1, mode, kappa, b, tin, rowf); break;
    }
}

// ------------------------------------------------------------- synthesis
// Inverse of one level (output n0 x n1, quadrants h0 x h1) for one basis on
// one output tile of 2TS x 2TS samples whose quadrant positions start at
// (R0, C0).  The quadrant tiles cover rows R0 - F/2 + 1 ... R0 + TS - 1
// (mod h0) and the same columns (mod h1), EXT = TS + F/2 - 1 <= 15 of each:
// thread t holds tile position (t / 16, t % 16) of the 4 quadrants.  An
// output sample m of a row takes quadrant row (m - k)/2 for its taps k of the
// same parity, so the tile row is (m - k)/2 - (R0 - F/2 + 1) with no wrap.
static_assert(NT == 16 * 16 && SEXT <= 16, "one quadrant-tile position per thread");

// This thread's quadrant-tile values of basis filter length F (loads only;
// the prior weights multiply them when they are stored).
template <typename R> struct SynVals {
    R v[4], w[4];
};

template <typename R>
__device__ __forceinline__ void syn_load(SynVals<R> &o, const R *__restrict__ cb, const R *__restrict__ wb,
                                         const R *__restrict__ sl, int from_coef, int L1, int h0, int h1, int R0,
                                         int C0, int F) {
    const int ext = TS + F / 2 - 1, i = threadIdx.x >> 4, j = threadIdx.x & 15;
    if (i >= ext || j >= ext) return;
    const int gi = wrap(R0 - F / 2 + 1 + i, h0), gj = wrap(C0 - F / 2 + 1 + j, h1);
#pragma unroll
    for (int qd = 0; qd < 4; ++qd) {
        o.w[qd] = R(1);
        if (qd == 0 && !from_coef) {
            o.v[qd] = sl[gi * h1 + gj];
        } else {
            const int64_t off = (int64_t)((qd & 2) ? h0 + gi : gi) * L1 + ((qd & 1) ? h1 : 0) + gj;
            o.v[qd] = cb[off];
            if (wb) o.w[qd] = wb[off];
        }
    }
}

template <typename R> __device__ __forceinline__ void syn_store(const SynVals<R> &o, R *qs, int F) {
    const int ext = TS + F / 2 - 1, i = threadIdx.x >> 4, j = threadIdx.x & 15;
    if (i >= ext || j >= ext) return;
#pragma unroll
    for (int qd = 0; qd < 4; ++qd) qs[qd * SEXT * SEXT + i * SEXT + j] = o.v[qd] * o.w[qd];
}

// Output sample of this thread in the 2TS x 2TS tile: row mm, column nnl,
// the column parity the same for a whole warp (odd warps: odd columns), so
// that the axis-1 pass below takes its taps as compile-time operands.
__device__ __forceinline__ void syn_pos(int &mm, int &nnl) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    mm = (w >> 1) * 4 + (l >> 3);
    nnl = 2 * (l & 7) + (w & 1);
}
static_assert(NT == 256 && TS == 8, "syn_pos covers the 16 x 16 tile with 8 warps");

// Row pitch of the axis-0 results: the 4 rows x 8 columns a warp reads in
// the axis-1 pass fall in disjoint banks.
constexpr int TP = 24;

// The two filter passes over the stored quadrant tiles (barrier first);
// returns this thread's output (position syn_pos; NT == 4 TS^2) and leaves
// the shared tiles free for reuse.  An output pair 2p, 2p + 1 reads the same
// F/2 inputs (quadrant row p + F/2 - 1 - kk for tap pair kk): the even
// sample takes the even taps, the odd one the odd taps.
template <typename R, int F>
__device__ __forceinline__ R syn_compute(int b, const R *qs, R *tl, R *th) {
    constexpr int EXT = TS + F / 2 - 1;
    const Taps<R, F> f(b);
    __syncthreads();
    if (threadIdx.x < TS * EXT) {   // inverse along axis 0: rows 2p and 2p + 1, column j
        const int p = threadIdx.x / EXT, j = threadIdx.x % EXT;
        R le = 0, he = 0, lo = 0, ho = 0;
#pragma unroll
        for (int kk = 0; kk < F / 2; ++kk) {
            const int il = p + F / 2 - 1 - kk;
            const R q0 = qs[0 * SEXT * SEXT + il * SEXT + j], q1 = qs[1 * SEXT * SEXT + il * SEXT + j];
            const R q2 = qs[2 * SEXT * SEXT + il * SEXT + j], q3 = qs[3 * SEXT * SEXT + il * SEXT + j];
            le += f.h[2 * kk] * q0 + f.g[2 * kk] * q2;
            he += f.h[2 * kk] * q1 + f.g[2 * kk] * q3;
            lo += f.h[2 * kk + 1] * q0 + f.g[2 * kk + 1] * q2;
            ho += f.h[2 * kk + 1] * q1 + f.g[2 * kk + 1] * q3;
        }
        tl[2 * p * TP + j] = le;
        th[2 * p * TP + j] = he;
        tl[(2 * p + 1) * TP + j] = lo;
        th[(2 * p + 1) * TP + j] = ho;
    }
    __syncthreads();
    int mm, nnl;   // inverse along axis 1
    syn_pos(mm, nnl);
    const R *rl = tl + mm * TP + (nnl >> 1) + F / 2 - 1, *rh = th + mm * TP + (nnl >> 1) + F / 2 - 1;
    R out = 0;
    if (nnl & 1) {
#pragma unroll
        for (int kk = 0; kk < F / 2; ++kk) out += f.h[2 * kk + 1] * rl[-kk] + f.g[2 * kk + 1] * rh[-kk];
    } else {
#pragma unroll
        for (int kk = 0; kk < F / 2; ++kk) out += f.h[2 * kk] * rl[-kk] + f.g[2 * kk] * rh[-kk];
    }
    __syncthreads();
    return out;
}

template <typename R> __device__ __forceinline__ R syn_compute_b(int b, const R *qs, R *tl, R *th) {
    switch (b) {
        case 0: return syn_compute<R, 2>(b, qs, tl, th);
        case 1: return syn_compute<R, 4>(b, qs, tl, th);
        case 2: return syn_compute<R, 6>(b, qs, tl, th);
        case 3: return syn_compute<R, 8>(b, qs, tl, th);
        case 4: return syn_compute<R, 10>(b, qs, tl, th);
        case 5: return syn_compute<R, 12>(b, qs, tl, th);
        case 6: return syn_compute<R, 14>(b, qs, tl, th);
        default: return syn_compute<R, 16>(b, qs, tl, th);
    }
}

// One synthesis level l > 0 for all 8 bases (grid.y = basis): out_b (n0 x n1,
// compact pitch n1) = D_b^T of (LL' block, detail quadrants), coefficients
// times the prior weights when wgt is set.  LL' comes from the coefficients
// at the coarsest level (from_coef) or from the coarser level's output sll.
template <typename R>
__global__ void __launch_bounds__(NT) k_sara_syn(const R *__restrict__ coef, const R *__restrict__ wgt, int L1,
                                                 int64_t N, const R *__restrict__ sll, int from_coef,
                                                 int64_t sll_bstride, int n0, int n1, R *__restrict__ out,
                                                 int64_t out_bstride) {
    __shared__ R qs[4 * SEXT * SEXT];
    __shared__ R tl[2 * TS * TP], th[2 * TS * TP];
    const int b = blockIdx.y;
    const int tpd1 = (n1 / 2 + TS - 1) / TS;
    const int R0 = (blockIdx.x / tpd1) * TS, C0 = (blockIdx.x % tpd1) * TS;
    pdl_enter();
    SynVals<R> q;
    syn_load(q, coef + (int64_t)(b + 1) * N, wgt ? wgt + (int64_t)(b + 1) * N : nullptr,
             sll + (int64_t)b * sll_bstride, from_coef, L1, n0 >> 1, n1 >> 1, R0, C0, 2 * b + 2);
    syn_store(q, qs, 2 * b + 2);
    const R v = syn_compute_b<R>(b, qs, tl, th);
    int mm, nnl;
    syn_pos(mm, nnl);
    if (2 * R0 + mm < n0 && 2 * C0 + nnl < n1)
        out[(int64_t)b * out_bstride + (int64_t)(2 * R0 + mm) * n1 + 2 * C0 + nnl] = v;
}

// Finest synthesis level, the 8 wavelet bases summed in order per output
// sample: out = scale * (dirac + sum_b D_b^T (w_b c_b)) (dirac may be null).
// The quadrant tiles of basis b + 1 are loaded into registers while basis b
// is filtered.
template <typename R>
__global__ void __launch_bounds__(NT) k_sara_syn0(const R *__restrict__ coef, const R *__restrict__ wgt, int L0,
                                                  int L1, int64_t N, const R *__restrict__ sll, int from_coef,
                                                  int64_t sll_bstride, const R *__restrict__ dirac, R scale,
                                                  R *__restrict__ out) {
    __shared__ R qs[4 * SEXT * SEXT];
    __shared__ R tl[2 * TS * TP], th[2 * TS * TP];
    const int tpd1 = (L1 / 2 + TS - 1) / TS;
    const int R0 = (blockIdx.x / tpd1) * TS, C0 = (blockIdx.x % tpd1) * TS;
    const int h0 = L0 >> 1, h1 = L1 >> 1;
    pdl_enter();
    auto load = [&](SynVals<R> &q, int b) {
        syn_load(q, coef + (int64_t)(b + 1) * N, wgt ? wgt + (int64_t)(b + 1) * N : nullptr,
                 sll + (int64_t)b * sll_bstride, from_coef, L1, h0, h1, R0, C0, 2 * b + 2);
    };
    SynVals<R> q;
    load(q, 0);
    R acc = 0;
#pragma unroll
    for (int b = 0; b < N_WAVELETS; ++b) {
        syn_store(q, qs, 2 * b + 2);
        if (b + 1 < N_WAVELETS) load(q, b + 1);
        acc += syn_compute_b<R>(b, qs, tl, th);
    }
    int mm, nnl;
    syn_pos(mm, nnl);
    if ((2 * R0 + mm < L0) && (2 * C0 + nnl < L1)) {
        const int64_t idx = (int64_t)(2 * R0 + mm) * L1 + 2 * C0 + nnl;
        out[idx] = scale * ((dirac ? dirac[idx] : R(0)) + acc);
    }
}

template <typename R> __global__ void k_scale_copy(const R *__restrict__ in, R *__restrict__ out, int64_t n, R a) {
    for (int64_t e = blockIdx.x * (int64_t)NT + threadIdx.x; e < n; e += (int64_t)gridDim.x * NT) out[e] = a * in[e];
}

inline unsigned nblk(int64_t work) { return (unsigned)std::min<int64_t>((work + NT - 1) / NT, 152 * 8); }
// tiles of ts x ts quadrant positions covering an h0 x h1 quadrant
inline unsigned tiles(int h0, int h1, int ts) { return (unsigned)(((h0 + ts - 1) / ts) * ((h1 + ts - 1) / ts)); }

// Analysis of all levels (tiled).  mode 0 writes c = D x / 3, mode 1
// clip-updates u with the prior weights and the clip level kappa ||Psi W||^2.
template <typename R> int analysis_all(ppd_ctx *c, const R *x, R *coef, int mode, cudaStream_t s) {
    const R *wgt = mode == 1 ? static_cast<const R *>(c->wgt) : nullptr;
    const uint8_t *pmask = (mode == 1 && c->rand_on) ? c->mask_cur + c->d : nullptr;
    const R alpha = (R)(c->kappa * c->psiw2);
    const int L0 = c->L0, L1 = c->L1;
    const int64_t N = c->N;
    const int64_t ll_stride = (int64_t)(L0 / 2) * (L1 / 2);
    R *ll[2] = {static_cast<R *>(c->wtmp), static_cast<R *>(c->wtmp) + (int64_t)N_WAVELETS * ll_stride};
    int site;
    for (int l = 0; l < c->levels; ++l) {
        const int n0 = L0 >> l, n1 = L1 >> l;
        const bool last = (l == c->levels - 1);
        const R *in = l == 0 ? x : ll[(l - 1) & 1];
        const int pitch = l == 0 ? L1 : n1;
        const int64_t bstride = l == 0 ? 0 : ll_stride;
        PPD_CHECK(launch_begin(c, "sara_analysis", s, &site));
        // level 0 starts its sequence (in the iteration: after the fork)
        launch(c, l > 0, k_sara_ana<R>, dim3(tiles(n0 / 2, n1 / 2, TSA), N_WAVELETS), NT, 0, s, in, pitch, bstride,
               n0, n1, ll[l & 1], ll_stride, (int)last, coef, wgt, L1, N, mode, alpha, pmask);
        PPD_CHECK(launch_end(c, site, s));
    }
    return PPD_OK;
}

// Synthesis of the 8 wavelet bases, levels coarsest .. 1 (tiled); returns
// the buffer holding the LL' block of level 0.
template <typename R>
int synthesis_levels(ppd_ctx *c, const R *coef, const R *wgt, const R **ll0, cudaStream_t s) {
    const int L0 = c->L0, L1 = c->L1;
    const int64_t N = c->N;
    const int64_t st = (int64_t)(L0 / 2) * (L1 / 2);
    R *buf[2] = {static_cast<R *>(c->wtmp2), static_cast<R *>(c->wtmp2) + (int64_t)N_WAVELETS * st};
    const R *prev = nullptr;
    int site, k = 0;
    for (int l = c->levels - 1; l >= 1; --l, ++k) {
        const int n0 = L0 >> l, n1 = L1 >> l;
        const bool coarsest = (l == c->levels - 1);
        PPD_CHECK(launch_begin(c, "sara_synthesis", s, &site));
        launch(c, true, k_sara_syn<R>, dim3(tiles(n0 / 2, n1 / 2, TS), N_WAVELETS), NT, 0, s, coef, wgt, L1, N,
               coarsest ? coef : prev, coarsest ? 1 : 0, st, n0, n1, buf[k & 1], st);
        PPD_CHECK(launch_end(c, site, s));
        prev = buf[k & 1];
    }
    *ll0 = prev;
    return PPD_OK;
}

template <typename R>
int synthesis_final(ppd_ctx *c, const R *coef, const R *wgt, const R *ll0, const R *dirac, R scale, R *out,
                    cudaStream_t s) {
    const int L0 = c->L0, L1 = c->L1;
    const int64_t st = (int64_t)(L0 / 2) * (L1 / 2);
    const bool from_coef = ll0 == nullptr;   // levels == 1: LL' straight from the coefficients
    int site;
    PPD_CHECK(launch_begin(c, "sara_synthesis", s, &site));
    launch(c, true, k_sara_syn0<R>, tiles(L0 / 2, L1 / 2, TS), NT, 0, s, coef, wgt, L0, L1, c->N,
           from_coef ? coef : ll0, from_coef ? 1 : 0, st, dirac, scale, out);
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
    PPD_CHECK(synthesis_levels<R>(c, coef, nullptr, &ll0, s));
    return synthesis_final<R>(c, coef, nullptr, ll0, coef, R(1.0 / 3.0), x, s);
}

// Prior dual step of Algorithm 3 for the 8 wavelet bases up to the level-0
// synthesis: u_b <- clip(u_b + W_b Psi_b^dagger xt, alpha), then the synthesis
// of W_b u_b for levels coarsest .. 1.  Needs only xt and u, so it can run
// beside the data branch of the iteration.
template <typename R> int sara_prior_branch(ppd_ctx *c, const R **ll0, cudaStream_t s) {
    R *u = static_cast<R *>(c->u);
    PPD_CHECK(analysis_all<R>(c, static_cast<const R *>(c->xt), u, 1, s));
    return synthesis_levels<R>(c, u, static_cast<const R *>(c->wgt), ll0, s);
}

// Level-0 synthesis summed over the 8 wavelet bases: ut = sum_b D_b^T (W_b u_b)
// (the Dirac basis and the 1/3 are applied in the primal step).
template <typename R> int sara_level0(ppd_ctx *c, const R *ll0, cudaStream_t s) {
    return synthesis_final<R>(c, static_cast<const R *>(c->u), static_cast<const R *>(c->wgt), ll0, nullptr, R(1),
                              static_cast<R *>(c->ut), s);
}



template int psi_analysis<float>(ppd_ctx *, const float *, float *, cudaStream_t);
template int psi_analysis<double>(ppd_ctx *, const double *, double *, cudaStream_t);
template int psi_synthesis<float>(ppd_ctx *, const float *, float *, cudaStream_t);
template int psi_synthesis<double>(ppd_ctx *, const double *, double *, cudaStream_t);
template int sara_prior_branch<float>(ppd_ctx *, const float **, cudaStream_t);
template int sara_prior_branch<double>(ppd_ctx *, const double **, cudaStream_t);
template int sara_level0<float>(ppd_ctx *, const float *, cudaStream_t);
template int sara_level0<double>(ppd_ctx *, const double *, cudaStream_t);

}  // namespace ppd
