// Oversampled 2-D FFT with the zero-padding / scaling operator Z fused in
// (Section 2: Phi = Theta G F Z; F is the unnormalised n-oversampled DFT).
//
// Forward  a = F Z x:  row pass   x (L x L real)  -> tmp (L x K complex)
//                      column pass tmp            -> grid (K x K complex)
// Inverse  Re(Z^T F^H grid): column pass grid -> tmp, row pass tmp -> image.
//
// Every pass is a batched Stockham radix-4 (one radix-2 stage when log2 K is
// odd) FFT in shared memory: a CTA loads B whole rows (row pass) or a strip of
// W columns (column pass), runs log K stages with one shared buffer (each
// thread keeps its butterflies in registers between the read and the write
// half of a stage) and writes the result.  Only the L nonzero rows/columns of
// the padded image are read or produced; the grid is stored with the zero
// frequency at the centre (plain index k at (k + K/2) mod K).
#include <cmath>

#include "common.cuh"

namespace ppd {

namespace {

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }

__host__ __device__ constexpr int ilog2_(int k) { return k <= 1 ? 0 : 1 + ilog2_(k / 2); }

// In-place batched Stockham FFT (forward sign) of NSEQ sequences of length K
// held in shared memory.  INTERLEAVED: element (s, i) at i*NSEQ + s;
// otherwise at s*K + i.  tw[m] = exp(-2 pi i m / K).
template <typename R, int K, int NSEQ, int NT, bool INTERLEAVED>
__device__ void fft_smem(cplx_t<R> *buf, const cplx_t<R> *tw) {
    using C = cplx_t<R>;
    const int tid = threadIdx.x;
    constexpr int LOG2K = ilog2_(K);
    int Ns = 1;
    auto idx = [](int s, int i) { return INTERLEAVED ? i * NSEQ + s : s * K + i; };
    if (LOG2K & 1) {   // one radix-2 stage (Ns = 1: no twiddles)
        constexpr int NB = NSEQ * K / 2 / NT;
        static_assert(NB >= 1 && NSEQ * K / 2 % NT == 0, "radix-2 work split");
        C v[NB][2];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int bf = tid + b * NT;
            int s = INTERLEAVED ? bf % NSEQ : bf / (K / 2);
            int j = INTERLEAVED ? bf / NSEQ : bf % (K / 2);
            C a0 = buf[idx(s, j)], a1 = buf[idx(s, j + K / 2)];
            v[b][0] = cadd(a0, a1);
            v[b][1] = csub(a0, a1);
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int bf = tid + b * NT;
            int s = INTERLEAVED ? bf % NSEQ : bf / (K / 2);
            int j = INTERLEAVED ? bf / NSEQ : bf % (K / 2);
            buf[idx(s, 2 * j)] = v[b][0];
            buf[idx(s, 2 * j + 1)] = v[b][1];
        }
        __syncthreads();
        Ns = 2;
    }
    constexpr int NB = NSEQ * K / 4 / NT;
    static_assert(NB >= 1 && NSEQ * K / 4 % NT == 0, "radix-4 work split");
    for (; Ns < K; Ns *= 4) {
        C v[NB][4];
        const int twstep = K / (Ns * 4);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int bf = tid + b * NT;
            int s = INTERLEAVED ? bf % NSEQ : bf / (K / 4);
            int j = INTERLEAVED ? bf / NSEQ : bf % (K / 4);
            int k = j & (Ns - 1);
            C a0 = buf[idx(s, j)];
            C a1 = buf[idx(s, j + K / 4)];
            C a2 = buf[idx(s, j + K / 2)];
            C a3 = buf[idx(s, j + 3 * K / 4)];
            if (Ns > 1) {
                a1 = cmul(a1, tw[(1 * k * twstep) & (K - 1)]);
                a2 = cmul(a2, tw[(2 * k * twstep) & (K - 1)]);
                a3 = cmul(a3, tw[(3 * k * twstep) & (K - 1)]);
            }
            C t0 = cadd(a0, a2), t1 = csub(a0, a2);
            C t2 = cadd(a1, a3), t3 = csub(a1, a3);
            // X1 = t1 - i t3, X3 = t1 + i t3
            v[b][0] = cadd(t0, t2);
            v[b][1] = C{t1.x + t3.y, t1.y - t3.x};
            v[b][2] = csub(t0, t2);
            v[b][3] = C{t1.x - t3.y, t1.y + t3.x};
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int bf = tid + b * NT;
            int s = INTERLEAVED ? bf % NSEQ : bf / (K / 4);
            int j = INTERLEAVED ? bf / NSEQ : bf % (K / 4);
            int k = j & (Ns - 1);
            int d = (j / Ns) * Ns * 4 + k;
            buf[idx(s, d)] = v[b][0];
            buf[idx(s, d + Ns)] = v[b][1];
            buf[idx(s, d + 2 * Ns)] = v[b][2];
            buf[idx(s, d + 3 * Ns)] = v[b][3];
        }
        __syncthreads();
    }
}

constexpr int NT = 256;

// rows per CTA in a row pass: enough butterflies for 256 threads
template <typename R> __host__ __device__ constexpr int rows_per_cta(int K) { return 1024 / K > 0 ? 1024 / K : 1; }
// columns per CTA in a column pass.  K <= 2048: the strips are read from
// L2 (grid and row-pass output of these sizes stay cached between the
// passes), so the fewest columns the 256-thread butterfly split allows
// (1024 / K, at least 1) give the most CTAs for these latency-bound passes.
// Larger K: at least 32 contiguous bytes per grid row (one DRAM sector:
// 4 float / 2 double columns), at most 128 KB of strip.
template <typename R> __host__ __device__ constexpr int cols_per_cta(int K) {
    constexpr int csz = 2 * (int)sizeof(R);
    if (K <= 2048) return 1024 / K > 1 ? 1024 / K : 1;
    const int w32 = (32 * 1024) / (K * csz), wmin = 32 / csz;
    int w = w32 > wmin ? w32 : wmin;
    while (w > 1 && (long long)w * K * csz > 128 * 1024) w /= 2;
    return w < K ? w : K;
}
// twiddles go to shared memory beside nseq sequences when a CTA then stays
// within 100 KB (two or more CTAs per SM), else they are read through the
// L1 from global memory (8192-point rows: 64 KB per CTA, three per SM)
template <typename R> __host__ __device__ constexpr bool tw_smem(int nseq, int K) {
    return (long long)(nseq + 1) * K * 2 * (int)sizeof(R) <= 100 * 1024;
}
template <typename R> constexpr size_t pass_smem(int nseq, int K) {
    return (size_t)(nseq + (tw_smem<R>(nseq, K) ? 1 : 0)) * K * 2 * sizeof(R);
}
template <typename R, int NSEQ, int K>
__device__ __forceinline__ const cplx_t<R> *stage_twiddles(cplx_t<R> *buf, const cplx_t<R> *__restrict__ tw) {
    if constexpr (tw_smem<R>(NSEQ, K)) {
        cplx_t<R> *tws = buf + NSEQ * K;
        for (int e = threadIdx.x; e < K; e += NT) tws[e] = tw[e];
        return tws;
    } else {
        return tw;
    }
}

// forward row pass: tmp[n0][c] = FFT_axis1(Z x)[n0][(c + K/2) mod K]
template <typename R, int K>
__global__ void __launch_bounds__(NT) k_rows_fwd(const R *__restrict__ x, cplx_t<R> *__restrict__ tmp,
                                                 const cplx_t<R> *__restrict__ tw, const R *__restrict__ s0,
                                                 const R *__restrict__ s1, int L, const uint8_t *__restrict__ colmask) {
    using C = cplx_t<R>;
    constexpr int B = rows_per_cta<R>(K);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const C *tws = stage_twiddles<R, B, K>(buf, tw);
    const int row0 = blockIdx.x * B;
    for (int e = threadIdx.x; e < B * K; e += NT) buf[e] = C{0, 0};
    __syncthreads();
    for (int e = threadIdx.x; e < B * L; e += NT) {
        int s = e / L, n1 = e % L, n0 = row0 + s;
        if (n0 < L) {
            int pos = (n1 - L / 2 + K) & (K - 1);
            buf[s * K + pos] = C{s0[n0] * s1[n1] * x[(int64_t)n0 * L + n1], R(0)};
        }
    }
    __syncthreads();
    fft_smem<R, K, B, NT, false>(buf, tws);
    for (int e = threadIdx.x; e < B * K; e += NT) {
        int s = e / K, c = e % K, n0 = row0 + s;
        if (n0 < L && colmask[c]) tmp[(int64_t)n0 * K + c] = buf[s * K + ((c + K / 2) & (K - 1))];
    }
}

// forward column pass: grid[r][c] = FFT_axis0(tmp padded)[(r + K/2) mod K][c]
template <typename R, int K>
__global__ void __launch_bounds__(NT) k_cols_fwd(const cplx_t<R> *__restrict__ tmp, cplx_t<R> *__restrict__ grid,
                                                 const cplx_t<R> *__restrict__ tw, int L,
                                                 const int32_t *__restrict__ strips,
                                                 const uint8_t *__restrict__ rowmask) {
    using C = cplx_t<R>;
    constexpr int W = cols_per_cta<R>(K);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const C *tws = stage_twiddles<R, W, K>(buf, tw);
    const int c0 = strips[blockIdx.x];
    for (int e = threadIdx.x; e < W * K; e += NT) buf[e] = C{0, 0};
    __syncthreads();
    for (int e = threadIdx.x; e < W * L; e += NT) {
        int s = e % W, n0 = e / W;
        int pos = (n0 - L / 2 + K) & (K - 1);
        buf[pos * W + s] = tmp[(int64_t)n0 * K + c0 + s];
    }
    __syncthreads();
    fft_smem<R, K, W, NT, true>(buf, tws);
    for (int e = threadIdx.x; e < W * K; e += NT) {
        int s = e % W, r = e / W;
        if (rowmask[r]) grid[(int64_t)r * K + c0 + s] = buf[((r + K / 2) & (K - 1)) * W + s];
    }
}

// inverse column pass: tmp[n0][c] = (F^H along axis 0 of grid)[(n0 - L/2) mod K][c]
template <typename R, int K>
__global__ void __launch_bounds__(NT) k_cols_inv(const cplx_t<R> *__restrict__ grid, cplx_t<R> *__restrict__ tmp,
                                                 const cplx_t<R> *__restrict__ tw, int L,
                                                 const int32_t *__restrict__ strips,
                                                 const uint8_t *__restrict__ rowmask) {
    using C = cplx_t<R>;
    constexpr int W = cols_per_cta<R>(K);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const C *tws = stage_twiddles<R, W, K>(buf, tw);
    const int c0 = strips[blockIdx.x];
    for (int e = threadIdx.x; e < W * K; e += NT) {
        int s = e % W, r = e / W;   // r: stored (centred) row; natural frequency (r + K/2) mod K
        buf[((r + K / 2) & (K - 1)) * W + s] = rowmask[r] ? cconj(grid[(int64_t)r * K + c0 + s]) : C{0, 0};
    }
    __syncthreads();
    fft_smem<R, K, W, NT, true>(buf, tws);
    for (int e = threadIdx.x; e < W * L; e += NT) {
        int s = e % W, n0 = e / W;
        int pos = (n0 - L / 2 + K) & (K - 1);
        tmp[(int64_t)n0 * K + c0 + s] = cconj(buf[pos * W + s]);
    }
}

// inverse column pass reading the gridding's per-chunk partial tiles
// directly: each cell of the strip is the fixed-order sum that the combine
// pass would write (its tile's chunks, then the halo rows/columns of the
// tiles above, left and above-left), so the combined grid never goes to HBM.
template <typename R, int K, int T>
__global__ void __launch_bounds__(NT) k_cols_inv_part(const cplx_t<R> *__restrict__ gpart,
                                                      const int32_t *__restrict__ tile_first,
                                                      const int32_t *__restrict__ tile_n, cplx_t<R> *__restrict__ tmp,
                                                      const cplx_t<R> *__restrict__ tw, int L,
                                                      const int32_t *__restrict__ strips,
                                                      const uint8_t *__restrict__ rowmask) {
    using C = cplx_t<R>;
    constexpr int W = cols_per_cta<R>(K);
    constexpr int E = T + 8, NTL = K / T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const C *tws = stage_twiddles<R, W, K>(buf, tw);
    const int c0 = strips[blockIdx.x];
    for (int e = threadIdx.x; e < W * K; e += NT) {
        const int s = e % W, r = e / W;   // r: stored (centred) row
        C acc{0, 0};
        if (rowmask[r]) {
            const int t0 = r / T, up = (t0 + NTL - 1) % NTL;
            const int t1 = (c0 + s) / T, left = (t1 + NTL - 1) % NTL;
            const int lr = r % T, lc = (c0 + s) % T;
            auto add = [&](int tt0, int tt1, int rr, int cc) {
                const int t = tt0 * NTL + tt1;
                const int f = tile_first[t], n = tile_n[t];
#pragma unroll 4
                for (int k = 0; k < n; ++k) {
                    const C g = gpart[(int64_t)(f + k) * E * E + rr * E + cc];
                    acc.x += g.x;
                    acc.y += g.y;
                }
            };
            add(t0, t1, lr, lc);
            if (lr < 8) add(up, t1, lr + T, lc);
            if (lc < 8) add(t0, left, lr, lc + T);
            if (lr < 8 && lc < 8) add(up, left, lr + T, lc + T);
        }
        buf[((r + K / 2) & (K - 1)) * W + s] = cconj(acc);
    }
    __syncthreads();
    fft_smem<R, K, W, NT, true>(buf, tws);
    for (int e = threadIdx.x; e < W * L; e += NT) {
        int s = e % W, n0 = e / W;
        int pos = (n0 - L / 2 + K) & (K - 1);
        tmp[(int64_t)n0 * K + c0 + s] = cconj(buf[pos * W + s]);
    }
}

// inverse row pass: img[n0][n1] = s0 s1 Re(F^H along axis 1 of tmp)[n0][(n1 - L/2) mod K]
template <typename R, int K>
__global__ void __launch_bounds__(NT) k_rows_inv(const cplx_t<R> *__restrict__ tmp, R *__restrict__ img,
                                                 const cplx_t<R> *__restrict__ tw, const R *__restrict__ s0,
                                                 const R *__restrict__ s1, int L) {
    using C = cplx_t<R>;
    constexpr int B = rows_per_cta<R>(K);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const C *tws = stage_twiddles<R, B, K>(buf, tw);
    const int row0 = blockIdx.x * B;
    for (int e = threadIdx.x; e < B * K; e += NT) {
        int s = e / K, c = e % K, n0 = row0 + s;
        C val = C{0, 0};
        if (n0 < L) val = cconj(tmp[(int64_t)n0 * K + c]);
        buf[s * K + ((c + K / 2) & (K - 1))] = val;
    }
    __syncthreads();
    fft_smem<R, K, B, NT, false>(buf, tws);
    for (int e = threadIdx.x; e < B * L; e += NT) {
        int s = e / L, n1 = e % L, n0 = row0 + s;
        if (n0 < L) {
            int pos = (n1 - L / 2 + K) & (K - 1);
            img[(int64_t)n0 * L + n1] = s0[n0] * s1[n1] * buf[s * K + pos].x;
        }
    }
}

// The end of one PPD iteration and the start of the next, B rows per CTA:
// the inverse row pass g = s0 s1 Re(F^H along axis 1 of tmp_inv) (the rows'
// Phi^dagger v, kept on chip), the primal step of Algorithm 3 on those
// pixels (primal_pixel), and the forward row pass of the new xt into
// tmp_fwd (the next iteration's first FFT pass), with the FP64 statistics
// partials of the CTA.  The join of the prior branch precedes it (ut, u0).
template <typename R, int K>
__global__ void __launch_bounds__(NT) k_rows_primal(const cplx_t<R> *__restrict__ tmp_inv, cplx_t<R> *__restrict__ tmp_fwd,
                                                    const cplx_t<R> *__restrict__ tw, const R *__restrict__ s0,
                                                    const R *__restrict__ s1, const uint8_t *__restrict__ colmask,
                                                    PrimalArgs<R> P, double *__restrict__ part) {
    using C = cplx_t<R>;
    constexpr int B = rows_per_cta<R>(K), L = K / 2, PER = B * L / NT;
    static_assert(B * L % NT == 0, "pixels per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const C *tws = stage_twiddles<R, B, K>(buf, tw);
    const int row0 = blockIdx.x * B;
    for (int e = threadIdx.x; e < B * K; e += NT) {
        const int s = e / K, c = e % K, n0 = row0 + s;
        buf[s * K + ((c + K / 2) & (K - 1))] = n0 < L ? cconj(tmp_inv[(int64_t)n0 * K + c]) : C{0, 0};
    }
    __syncthreads();
    fft_smem<R, K, B, NT, false>(buf, tws);
    PrimalSums<R> acc;
    R xtn[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * NT, s = e / L, n1 = e % L, n0 = row0 + s;
        xtn[k] = R(0);
        if (n0 < L) {
            const R g = s0[n0] * s1[n1] * buf[s * K + ((n1 - L / 2 + K) & (K - 1))].x;
            xtn[k] = primal_pixel(P, (int64_t)n0 * L + n1, g, acc);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < B * K; e += NT) buf[e] = C{0, 0};
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * NT, s = e / L, n1 = e % L, n0 = row0 + s;
        if (n0 < L) buf[s * K + ((n1 - L / 2 + K) & (K - 1))] = C{s0[n0] * s1[n1] * xtn[k], R(0)};
    }
    __syncthreads();
    fft_smem<R, K, B, NT, false>(buf, tws);
    for (int e = threadIdx.x; e < B * K; e += NT) {
        const int s = e / K, c = e % K, n0 = row0 + s;
        if (n0 < L && colmask[c]) tmp_fwd[(int64_t)n0 * K + c] = buf[s * K + ((c + K / 2) & (K - 1))];
    }
    acc.write(part + 3 * (int64_t)blockIdx.x);
}

template <typename R, int K> struct Pass {
    static constexpr int B = rows_per_cta<R>(K), W = cols_per_cta<R>(K);
    // dynamic shared memory of the row and column passes (per device)
    static int attrs() {
        const int shr = (int)pass_smem<R>(B, K), shc = (int)pass_smem<R>(W, K);
        PPD_CHECK(smem_attr((const void *)k_rows_fwd<R, K>, shr));
        PPD_CHECK(smem_attr((const void *)k_rows_inv<R, K>, shr));
        PPD_CHECK(smem_attr((const void *)k_rows_primal<R, K>, shr));
        PPD_CHECK(smem_attr((const void *)k_cols_fwd<R, K>, shc));
        PPD_CHECK(smem_attr((const void *)k_cols_inv<R, K>, shc));
        PPD_CHECK(smem_attr((const void *)k_cols_inv_part<R, K, 16>, shc));
        return smem_attr((const void *)k_cols_inv_part<R, K, 32>, shc);
    }
    static int rows_fwd(ppd_ctx *c, const R *x, cudaStream_t s) {
        PPD_CHECK(attrs());
        int site;
        PPD_CHECK(launch_begin(c, "fft_fwd_rows", s, &site));
        k_rows_fwd<R, K><<<(c->L0 + B - 1) / B, NT, pass_smem<R>(B, K), s>>>(
            x, static_cast<cplx_t<R> *>(c->fft_tmp), static_cast<const cplx_t<R> *>(c->tw0),
            static_cast<const R *>(c->deap0), static_cast<const R *>(c->deap1), c->L0, c->col_fwd);
        return launch_end(c, site, s);
    }
    static int cols_fwd(ppd_ctx *c, cplx_t<R> *grid, cudaStream_t s) {
        PPD_CHECK(attrs());
        if (c->n_fwd_strips == 0) return PPD_OK;
        int site;
        PPD_CHECK(launch_begin(c, "fft_fwd_cols", s, &site));
        k_cols_fwd<R, K><<<c->n_fwd_strips, NT, pass_smem<R>(W, K), s>>>(
            static_cast<const cplx_t<R> *>(c->fft_tmp), grid, static_cast<const cplx_t<R> *>(c->tw0), c->L0,
            c->fwd_strips, c->row_fwd);
        return launch_end(c, site, s);
    }
    static int cols_inv(ppd_ctx *c, const cplx_t<R> *grid, cudaStream_t s) {
        PPD_CHECK(attrs());
        if (c->n_inv_strips == 0) return PPD_OK;
        int site;
        PPD_CHECK(launch_begin(c, "fft_inv_cols", s, &site));
        k_cols_inv<R, K><<<c->n_inv_strips, NT, pass_smem<R>(W, K), s>>>(
            grid, static_cast<cplx_t<R> *>(c->fft_tmp_inv), static_cast<const cplx_t<R> *>(c->tw0), c->L0,
            c->inv_strips, c->row_inv);
        return launch_end(c, site, s);
    }
    static int cols_inv_part(ppd_ctx *c, cudaStream_t s) {
        PPD_CHECK(attrs());
        if (c->n_inv_strips == 0) return PPD_OK;
        int site;
        PPD_CHECK(launch_begin(c, "fft_inv_cols", s, &site));
        const cplx_t<R> *gp = static_cast<const cplx_t<R> *>(c->gpart);
        cplx_t<R> *out = static_cast<cplx_t<R> *>(c->fft_tmp_inv);
        const cplx_t<R> *tw = static_cast<const cplx_t<R> *>(c->tw0);
        if (c->T == 16)
            k_cols_inv_part<R, K, 16><<<c->n_inv_strips, NT, pass_smem<R>(W, K), s>>>(
                gp, c->ch.tile_first, c->ch.tile_n, out, tw, c->L0, c->inv_strips, c->row_inv);
        else
            k_cols_inv_part<R, K, 32><<<c->n_inv_strips, NT, pass_smem<R>(W, K), s>>>(
                gp, c->ch.tile_first, c->ch.tile_n, out, tw, c->L0, c->inv_strips, c->row_inv);
        return launch_end(c, site, s);
    }
    static int rows_inv(ppd_ctx *c, R *img, cudaStream_t s) {
        PPD_CHECK(attrs());
        int site;
        PPD_CHECK(launch_begin(c, "fft_inv_rows", s, &site));
        k_rows_inv<R, K><<<(c->L0 + B - 1) / B, NT, pass_smem<R>(B, K), s>>>(
            static_cast<const cplx_t<R> *>(c->fft_tmp_inv), img, static_cast<const cplx_t<R> *>(c->tw0),
            static_cast<const R *>(c->deap0), static_cast<const R *>(c->deap1), c->L0);
        return launch_end(c, site, s);
    }
    static int rows_primal(ppd_ctx *c, cudaStream_t s) {
        PPD_CHECK(attrs());
        int site;
        PPD_CHECK(launch_begin(c, "rows_primal", s, &site));
        const int n = (c->L0 + B - 1) / B;
        k_rows_primal<R, K><<<n, NT, pass_smem<R>(B, K), s>>>(
            static_cast<const cplx_t<R> *>(c->fft_tmp_inv), static_cast<cplx_t<R> *>(c->fft_tmp),
            static_cast<const cplx_t<R> *>(c->tw0), static_cast<const R *>(c->deap0),
            static_cast<const R *>(c->deap1), c->col_fwd, primal_args<R>(c), c->prim_part);
        c->n_stat_parts = n;
        return launch_end(c, site, s);
    }
};

}  // namespace

#define PPD_FFT_SIZES(X) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)
#define PPD_FFT_CASE(KK, CALL) case KK: return Pass<R, KK>::CALL;

// forward row pass of x into the FFT temporary (first half of F Z x)
template <typename R> int fft_forward_rows(ppd_ctx *c, const R *x, cudaStream_t s) {
    c->xt_rows_valid = false;
    switch (c->K0) {
#define X(KK) PPD_FFT_CASE(KK, rows_fwd(c, x, s))
        PPD_FFT_SIZES(X)
#undef X
        default: return fail(PPD_ERR_UNSUPPORTED, "FFT size not supported");
    }
}

// forward column pass from the FFT temporary to the grid (second half of F Z x)
template <typename R> int fft_forward_cols(ppd_ctx *c, cplx_t<R> *grid, cudaStream_t s) {
    switch (c->K0) {
#define X(KK) PPD_FFT_CASE(KK, cols_fwd(c, grid, s))
        PPD_FFT_SIZES(X)
#undef X
        default: return fail(PPD_ERR_UNSUPPORTED, "FFT size not supported");
    }
}

// inverse column pass of a combined grid into the inverse temporary
template <typename R> int fft_inverse_cols(ppd_ctx *c, const cplx_t<R> *grid, cudaStream_t s) {
    switch (c->K0) {
#define X(KK) PPD_FFT_CASE(KK, cols_inv(c, grid, s))
        PPD_FFT_SIZES(X)
#undef X
        default: return fail(PPD_ERR_UNSUPPORTED, "FFT size not supported");
    }
}

// inverse column pass summing the gridding's partial tiles while loading
// (the combine pass fused in)
template <typename R> int fft_inverse_cols_partials(ppd_ctx *c, cudaStream_t s) {
    switch (c->K0) {
#define X(KK) PPD_FFT_CASE(KK, cols_inv_part(c, s))
        PPD_FFT_SIZES(X)
#undef X
        default: return fail(PPD_ERR_UNSUPPORTED, "FFT size not supported");
    }
}

// inverse row pass into an image (second half of Z^T F^H)
template <typename R> int fft_inverse_rows(ppd_ctx *c, R *img, cudaStream_t s) {
    switch (c->K0) {
#define X(KK) PPD_FFT_CASE(KK, rows_inv(c, img, s))
        PPD_FFT_SIZES(X)
#undef X
        default: return fail(PPD_ERR_UNSUPPORTED, "FFT size not supported");
    }
}

// inverse row pass + primal step + forward row pass of the new xt
template <typename R> int rows_primal(ppd_ctx *c, cudaStream_t s) {
    switch (c->K0) {
#define X(KK) PPD_FFT_CASE(KK, rows_primal(c, s))
        PPD_FFT_SIZES(X)
#undef X
        default: return fail(PPD_ERR_UNSUPPORTED, "FFT size not supported");
    }
}

template <typename R> int fft_forward(ppd_ctx *c, const R *x, cplx_t<R> *grid, cudaStream_t s) {
    PPD_CHECK(fft_forward_rows<R>(c, x, s));
    return fft_forward_cols<R>(c, grid, s);
}

template <typename R> int fft_inverse(ppd_ctx *c, const cplx_t<R> *grid, R *img, cudaStream_t s) {
    PPD_CHECK(fft_inverse_cols<R>(c, grid, s));
    return fft_inverse_rows<R>(c, img, s);
}

#undef PPD_FFT_CASE
#undef PPD_FFT_SIZES

#define PPD_FFT_INST(R)                                                                                         \
    template int fft_forward<R>(ppd_ctx *, const R *, cplx_t<R> *, cudaStream_t);                              \
    template int fft_inverse<R>(ppd_ctx *, const cplx_t<R> *, R *, cudaStream_t);                              \
    template int fft_forward_rows<R>(ppd_ctx *, const R *, cudaStream_t);                                       \
    template int fft_forward_cols<R>(ppd_ctx *, cplx_t<R> *, cudaStream_t);                                     \
    template int fft_inverse_cols<R>(ppd_ctx *, const cplx_t<R> *, cudaStream_t);                              \
    template int fft_inverse_cols_partials<R>(ppd_ctx *, cudaStream_t);                                         \
    template int fft_inverse_rows<R>(ppd_ctx *, R *, cudaStream_t);                                             \
    template int rows_primal<R>(ppd_ctx *, cudaStream_t);
PPD_FFT_INST(float)
PPD_FFT_INST(double)
#undef PPD_FFT_INST

// Column strips (W columns each, W as the column passes use) that contain a
// marked column, and the row / column masks, uploaded for the pruned passes.
int fft_plan_pruning(ppd_ctx *c, const std::vector<char> &rows_fwd, const std::vector<char> &cols_fwd,
                     const std::vector<char> &rows_inv, const std::vector<char> &cols_inv) {
    const int K = c->K0;
    const int W = c->is_f32 ? cols_per_cta<float>(K) : cols_per_cta<double>(K);
    std::vector<int32_t> fs, is;
    for (int s0 = 0; s0 < K; s0 += W) {
        bool f = false, i = false;
        for (int j = s0; j < s0 + W; ++j) {
            f = f || cols_fwd[j];
            i = i || cols_inv[j];
        }
        if (f) fs.push_back(s0);
        if (i) is.push_back(s0);
    }
    std::vector<uint8_t> rf(rows_fwd.begin(), rows_fwd.end()), ri(rows_inv.begin(), rows_inv.end()),
        cf(cols_fwd.begin(), cols_fwd.end());
    c->n_fwd_strips = (int)fs.size();
    c->n_inv_strips = (int)is.size();
    if (!fs.empty()) PPD_CUDA(cudaMemcpy(c->fwd_strips, fs.data(), fs.size() * 4, cudaMemcpyHostToDevice));
    if (!is.empty()) PPD_CUDA(cudaMemcpy(c->inv_strips, is.data(), is.size() * 4, cudaMemcpyHostToDevice));
    PPD_CUDA(cudaMemcpy(c->row_fwd, rf.data(), K, cudaMemcpyHostToDevice));
    PPD_CUDA(cudaMemcpy(c->row_inv, ri.data(), K, cudaMemcpyHostToDevice));
    PPD_CUDA(cudaMemcpy(c->col_fwd, cf.data(), K, cudaMemcpyHostToDevice));
    // the inverse column pass writes only its strips: the rest of its output
    // stays zero; the forward row pass writes only marked columns
    PPD_CUDA(cudaMemset(c->fft_tmp_inv, 0, (size_t)c->L0 * K * 2 * c->rsz));
    PPD_CUDA(cudaMemset(c->fft_tmp, 0, (size_t)c->L0 * K * 2 * c->rsz));
    return PPD_OK;
}

// Twiddles exp(-2 pi i m / K), m < K, computed in double on the host.
int make_twiddles(ppd_ctx *c) {
    const int K = c->K0;
    std::vector<double> t(2 * (size_t)K);
    for (int m = 0; m < K; ++m) {
        double a = -2.0 * M_PI * (double)m / (double)K;
        t[2 * m] = std::cos(a);
        t[2 * m + 1] = std::sin(a);
    }
    if (c->is_f32) {
        std::vector<float> f(t.begin(), t.end());
        PPD_CUDA(cudaMemcpy(c->tw0, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        PPD_CUDA(cudaMemcpy(c->tw0, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return PPD_OK;
}

// Z's scaling s(n) = 1 / psi_hat((n - L/2)/K), psi_hat(f) = (J / I0(beta)) sinh(q)/q,
// q = sqrt(beta^2 - (pi J f)^2): the Fourier transform of the Kaiser-Bessel kernel.
int make_deapodisation(ppd_ctx *c) {
    const int L = c->L0, K = c->K0;
    const double J = KB_J, beta = c->beta, i0b = std::cyl_bessel_i(0.0, beta);
    std::vector<double> s(L);
    for (int n = 0; n < L; ++n) {
        double f = ((double)n - L / 2) / (double)K;
        double q = std::sqrt(beta * beta - (M_PI * J * f) * (M_PI * J * f));
        s[n] = 1.0 / ((J / i0b) * std::sinh(q) / q);
    }
    if (c->is_f32) {
        std::vector<float> f(s.begin(), s.end());
        PPD_CUDA(cudaMemcpy(c->deap0, f.data(), L * sizeof(float), cudaMemcpyHostToDevice));
        PPD_CUDA(cudaMemcpy(c->deap1, f.data(), L * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        PPD_CUDA(cudaMemcpy(c->deap0, s.data(), L * sizeof(double), cudaMemcpyHostToDevice));
        PPD_CUDA(cudaMemcpy(c->deap1, s.data(), L * sizeof(double), cudaMemcpyHostToDevice));
    }
    return PPD_OK;
}

}  // namespace ppd
