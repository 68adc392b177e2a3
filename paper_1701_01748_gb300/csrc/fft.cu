// Oversampled 2-D FFT with the zero-padding / scaling operator Z fused in
// (Section 2: Phi = Theta G F Z; F is the unnormalised n-oversampled DFT).
//
// Image L0 x L1 (rows x columns), grid K0 x K1 (K = 2L per axis).
// Forward  a = F Z x:  row pass    x (L0 x L1 real) -> tmp (L0 x K1 complex)
//                      column pass tmp              -> grid (K0 x K1 complex)
// Inverse  Re(Z^T F^H grid): column pass grid -> tmp, row pass tmp -> image.
//
// Every pass is a batched Stockham FFT in shared memory: a CTA loads B whole
// rows (row pass, length K1) or a strip of W columns (column pass, length
// K0), runs the stages and writes the result.  Only the L nonzero rows /
// columns of the padded image are read or produced; the grid is stored with
// the zero frequency at the centre (plain index k at (k + K/2) mod K).
//
// Two cores: lengths that are powers of two use a compile-time radix-4 (and
// one radix-2) core with one shared buffer; any other length whose prime
// factors are 2, 3 and 5 uses a run-time mixed-radix core (radices 5, 3, 4,
// 2 from a plan made on the host) that ping-pongs between two buffers.  The
// pass kernels are templated on KT = the length for the first core, 0 for
// the second.
#include <cmath>
#include <vector>

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

// v mod K for v in [0, 2K)
__device__ __forceinline__ int wrapK(int v, int K) { return v >= K ? v - K : v; }

constexpr int NT = 256;

// ------------------------------------------------------------ power-of-two core
// In-place batched Stockham FFT (forward sign) of NSEQ sequences of length K
// held in shared memory.  INTERLEAVED: element (s, i) at i*NSEQ + s;
// otherwise at s*K + i.  tw: the twiddles stage by stage (upload_stage_twiddles):
// for the radix-4 stage of span Ns, w^(q k K / (4 Ns)) at (q - 1) Ns + k, so
// that the butterflies of a warp (consecutive k) read consecutive words.
template <typename R, int K, int NSEQ, bool INTERLEAVED>
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
    const C *tws = tw;   // this stage's table (stages with Ns = 1 have none)
    for (; Ns < K; Ns *= 4) {
        C v[NB][4];
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
                a1 = cmul(a1, tws[k]);
                a2 = cmul(a2, tws[Ns + k]);
                a3 = cmul(a3, tws[2 * Ns + k]);
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
        if (Ns > 1) tws += 3 * Ns;
    }
}

// ------------------------------------------------------------ mixed-radix core
// Forward DFT of RAD points in place (sign -), written out per radix.
template <typename C> __device__ __forceinline__ void dft(C (&a)[2]) {
    const C t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
}
template <typename C> __device__ __forceinline__ void dft(C (&a)[3]) {
    using R = decltype(a[0].x);
    const R h = R(0.8660254037844386);   // sin(2 pi / 3)
    const C s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
    const C m{a[0].x - R(0.5) * s.x, a[0].y - R(0.5) * s.y};
    const C e{h * d.y, -h * d.x};   // -i sin(2 pi/3) (a1 - a2)
    a[0] = cadd(a[0], s);
    a[1] = cadd(m, e);
    a[2] = csub(m, e);
}
template <typename C> __device__ __forceinline__ void dft(C (&a)[4]) {
    const C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    const C t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
    a[0] = cadd(t0, t2);
    a[1] = C{t1.x + t3.y, t1.y - t3.x};
    a[2] = csub(t0, t2);
    a[3] = C{t1.x - t3.y, t1.y + t3.x};
}
template <typename C> __device__ __forceinline__ void dft(C (&a)[5]) {
    using R = decltype(a[0].x);
    const R c1 = R(0.30901699437494745), c2 = R(-0.8090169943749475);   // cos(2 pi/5), cos(4 pi/5)
    const R s1 = R(0.9510565162951535), s2 = R(0.5877852522924731);     // sin(2 pi/5), sin(4 pi/5)
    const C t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    const C t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
    const C u1{a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y};
    const C u2{a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y};
    const C v1{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
    const C v2{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
    a[0] = cadd(a[0], cadd(t1, t2));
    a[1] = C{u1.x + v1.y, u1.y - v1.x};   // u1 - i v1
    a[4] = C{u1.x - v1.y, u1.y + v1.x};   // u1 + i v1
    a[2] = C{u2.x + v2.y, u2.y - v2.x};
    a[3] = C{u2.x - v2.y, u2.y + v2.x};
}

// One Stockham stage of radix RAD from src to dst: for butterfly j (k = j mod
// Ns) the inputs j + q K/RAD, twiddled by w^(q k K/(Ns RAD)), go to
// (j - k) RAD + k + p Ns.
template <typename R, int RAD, bool INTERLEAVED>
__device__ __forceinline__ void stage_any(const cplx_t<R> *__restrict__ src, cplx_t<R> *__restrict__ dst, int K,
                                          int nseq, int Ns, const cplx_t<R> *__restrict__ tw) {
    using C = cplx_t<R>;
    const int m = K / RAD, tstep = K / (Ns * RAD), nbf = nseq * m;
    for (int bf = threadIdx.x; bf < nbf; bf += NT) {
        int s, j;
        if (INTERLEAVED) {
            j = bf / nseq;
            s = bf - j * nseq;
        } else {
            s = bf / m;
            j = bf - s * m;
        }
        const int k = j % Ns;
        C a[RAD];
#pragma unroll
        for (int q = 0; q < RAD; ++q) a[q] = src[INTERLEAVED ? (j + q * m) * nseq + s : s * K + j + q * m];
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < RAD; ++q) a[q] = cmul(a[q], tw[q * k * tstep]);
        }
        dft(a);
        const int d = (j - k) * RAD + k;
#pragma unroll
        for (int p = 0; p < RAD; ++p) dst[INTERLEAVED ? (d + p * Ns) * nseq + s : s * K + d + p * Ns] = a[p];
    }
}

// Batched mixed-radix FFT of nseq sequences of length pl.K in a (layout as
// fft_smem), ping-ponging with b; returns the buffer holding the result.
// Callers synchronise before (the input is complete) and the last stage
// ends with a barrier.
template <typename R, bool INTERLEAVED>
__device__ cplx_t<R> *fft_any(cplx_t<R> *a, cplx_t<R> *b, int nseq, const FftPlan &pl, const cplx_t<R> *tw) {
    int Ns = 1;
    for (int st = 0; st < pl.ns; ++st) {
        const int r = pl.rad[st];
        if (r == 4) stage_any<R, 4, INTERLEAVED>(a, b, pl.K, nseq, Ns, tw);
        else if (r == 2) stage_any<R, 2, INTERLEAVED>(a, b, pl.K, nseq, Ns, tw);
        else if (r == 3) stage_any<R, 3, INTERLEAVED>(a, b, pl.K, nseq, Ns, tw);
        else stage_any<R, 5, INTERLEAVED>(a, b, pl.K, nseq, Ns, tw);
        __syncthreads();
        Ns *= r;
        cplx_t<R> *t = a;
        a = b;
        b = t;
    }
    return a;
}

// ------------------------------------------------------------ pass geometry
// rows per CTA in a row pass of the power-of-two core: enough butterflies for 256 threads
template <typename R> __host__ __device__ constexpr int rows_per_cta(int K) { return 1024 / K > 0 ? 1024 / K : 1; }
// columns per CTA in a column pass of the power-of-two core.  K <= 1024:
// the fewest columns the 256-thread butterfly split allows (1024 / K, at
// least 1), the most CTAs for these latency-bound passes (measured: four
// columns per CTA at K = 1024 made both column passes 40 % slower).  At
// K = 2048 every row of a strip is one 32-byte sector (4 float / 2 double
// columns; measured: forward pass 41 -> 31 us).  Longer columns: one per
// CTA (the column-major inputs make its reads contiguous; 64 KB of strip in
// FP32 at K = 8192 leaves room for three CTAs per SM, where two columns took
// 128 KB and one CTA: 7.27 -> 6.96 ms per 4096^2 iteration).
template <typename R> __host__ __device__ constexpr int cols_per_cta(int K) {
    constexpr int csz = 2 * (int)sizeof(R);
    if (K <= 1024) return 1024 / K > 1 ? 1024 / K : 1;
    return K == 2048 ? 32 / csz : 1;
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
// sequences per CTA as a compile-time constant (power-of-two core) or 1
template <typename R, int KT> constexpr int rows_ct() { return KT ? rows_per_cta<R>(KT) : 1; }
template <typename R, int KT> constexpr int cols_ct() { return KT ? cols_per_cta<R>(KT) : 1; }

// The FFT of a pass: the compile-time core in place, or the mixed-radix core
// (buf2 the second buffer); returns the buffer holding the result.
template <typename R, int KT, int NSEQ, bool IL>
__device__ __forceinline__ cplx_t<R> *run_fft(cplx_t<R> *buf, cplx_t<R> *buf2, const cplx_t<R> *tws, int nseq,
                                              const FftPlan &pl, const cplx_t<R> *tw) {
    if constexpr (KT != 0) {
        fft_smem<R, KT, NSEQ, IL>(buf, tws);
        return buf;
    } else {
        return fft_any<R, IL>(buf, buf2, nseq, pl, tw);
    }
}

// Run-time arguments of a pass: the FFT plan of its length and the
// sequences per CTA (used by the mixed-radix core only).
struct PassArgs {
    FftPlan pl;
    int nseq;
};

// Row passes of the power-of-two core transform two real rows (a, b) as one
// complex sequence.  Forward: z = a + i b, and after the FFT
// A[k] = (Z[k] + conj(Z[-k]))/2, B[k] = (Z[k] - conj(Z[-k]))/(2i).
template <typename C> __device__ __forceinline__ void split_two_real(C z, C zr, C &A, C &B) {
    using R = decltype(z.x);
    A = C{R(0.5) * (z.x + zr.x), R(0.5) * (z.y - zr.y)};
    B = C{R(0.5) * (z.y + zr.y), R(0.5) * (zr.x - z.x)};
}
// Inverse to real parts: Re(F^H X) = F^H H with H[k] = (X[k] + conj(X[-k]))/2
// (the Hermitian part of X), so the pair is Y = Ha + i Hb, F^H Y = ha + i hb;
// returns Y[k] and Y[-k] from Xa[k], Xa[-k], Xb[k], Xb[-k].
template <typename C> __device__ __forceinline__ void pack_two_real(C xa, C xar, C xb, C xbr, C &y, C &yr) {
    using R = decltype(xa.x);
    const C ha{R(0.5) * (xa.x + xar.x), R(0.5) * (xa.y - xar.y)};
    const C hb{R(0.5) * (xb.x + xbr.x), R(0.5) * (xb.y - xbr.y)};
    y = C{ha.x - hb.y, ha.y + hb.x};    // ha + i hb
    yr = C{ha.x + hb.y, hb.x - ha.y};   // conj(ha) + i conj(hb)
}

// Loads the spectra of rows (row0 + 2s, row0 + 2s + 1), s < NSEQ, of tmp
// (stored centred: natural frequency k at column (k + K/2) mod K) and writes
// conj(Y) in natural order into buf, so that the forward FFT of buf gives
// conj(F^H Y): row a's real inverse in .x, row b's in -.y.
template <typename R, int K, int NSEQ>
__device__ __forceinline__ void load_two_real_inverse(const cplx_t<R> *__restrict__ tmp, int row0, int L0,
                                                      cplx_t<R> *buf) {
    using C = cplx_t<R>;
    constexpr int H = K / 2 + 1;   // pairs (k, -k), k = 0 .. K/2
    for (int e = threadIdx.x; e < NSEQ * H; e += NT) {
        const int s = e / H, k = e - s * H, kr = (K - k) & (K - 1);
        const int ra = row0 + 2 * s, rb = ra + 1;
        const int ck = (k + K / 2) & (K - 1), ckr = (kr + K / 2) & (K - 1);
        C xa{0, 0}, xar{0, 0}, xb{0, 0}, xbr{0, 0};
        if (ra < L0) {
            xa = tmp[(int64_t)ra * K + ck];
            xar = tmp[(int64_t)ra * K + ckr];
        }
        if (rb < L0) {
            xb = tmp[(int64_t)rb * K + ck];
            xbr = tmp[(int64_t)rb * K + ckr];
        }
        C y, yr;
        pack_two_real(xa, xar, xb, xbr, y, yr);
        buf[s * K + k] = cconj(y);
        buf[s * K + kr] = cconj(yr);
    }
}

// Writes the spectra of rows (row0 + 2s, row0 + 2s + 1) from the FFT of
// a + i b in buf (natural order) to the column-major tmp (column c at
// c L0, stored centred, marked columns): the two rows are adjacent there.
template <typename R, int K, int NSEQ>
__device__ __forceinline__ void store_two_real_forward(const cplx_t<R> *out, int row0, int L0,
                                                       const uint8_t *__restrict__ colmask,
                                                       cplx_t<R> *__restrict__ tmp) {
    using C = cplx_t<R>;
    for (int e = threadIdx.x; e < NSEQ * K; e += NT) {
        const int s = e / K, c = e % K, ra = row0 + 2 * s, rb = ra + 1;
        if (!colmask[c] || ra >= L0) continue;
        const int kk = (c + K / 2) & (K - 1), kr = (K - kk) & (K - 1);
        C A, B;
        split_two_real(out[s * K + kk], out[s * K + kr], A, B);
        C *dst = tmp + (int64_t)c * L0 + ra;   // ra and L0 even: rb < L0, 16-byte aligned pair
        if constexpr (sizeof(R) == 4) {
            *reinterpret_cast<float4 *>(dst) = make_float4(A.x, A.y, B.x, B.y);
        } else {
            dst[0] = A;
            dst[1] = B;
        }
    }
}

// forward row pass: tmp[n0][c] = FFT_axis1(Z x)[n0][(c + K1/2) mod K1],
// tmp column-major (element (n0, c) at c L0 + n0) for the column pass
template <typename R, int KT>
__global__ void __launch_bounds__(NT) k_rows_fwd(const R *__restrict__ x, cplx_t<R> *__restrict__ tmp,
                                                 const cplx_t<R> *__restrict__ tw, const R *__restrict__ s0,
                                                 const R *__restrict__ s1, int L0, int L1,
                                                 const uint8_t *__restrict__ colmask, PassArgs pa) {
    using C = cplx_t<R>;
    constexpr int BT = rows_ct<R, KT>();
    const int K = KT ? KT : pa.pl.K, B = KT ? BT : pa.nseq;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *buf2 = buf + B * K;
    const C *tws = KT ? stage_twiddles<R, BT, KT ? KT : 1>(buf, tw) : tw;
    pdl_enter();   // the twiddles are static: staged while the previous kernel drains
    if constexpr (KT != 0) {   // two rows per sequence
        const int row0 = blockIdx.x * 2 * BT;
        for (int e = threadIdx.x; e < BT * KT; e += NT) {
            const int s = e / KT, p = e % KT, ra = row0 + 2 * s, rb = ra + 1;
            const int n1 = p < L1 / 2 ? p + L1 / 2 : (p >= KT - L1 / 2 ? p - KT + L1 / 2 : -1);
            R va = 0, vb = 0;
            if (n1 >= 0 && ra < L0) va = s0[ra] * s1[n1] * x[(int64_t)ra * L1 + n1];
            if (n1 >= 0 && rb < L0) vb = s0[rb] * s1[n1] * x[(int64_t)rb * L1 + n1];
            buf[e] = C{va, vb};
        }
        __syncthreads();
        fft_smem<R, KT ? KT : 1, BT, false>(buf, tws);
        store_two_real_forward<R, KT ? KT : 1, BT>(buf, row0, L0, colmask, tmp);
        return;
    }
    const int row0 = blockIdx.x * B;
    // one pass over the padded rows: position p holds pixel p + L1/2 (p <
    // L1/2) or p - K + L1/2 (p >= K - L1/2), zero in between
    for (int e = threadIdx.x; e < B * K; e += NT) {
        const int s = e / K, p = e - s * K, n0 = row0 + s;
        const int n1 = p < L1 / 2 ? p + L1 / 2 : (p >= K - L1 / 2 ? p - K + L1 / 2 : -1);
        buf[e] = (n1 >= 0 && n0 < L0) ? C{s0[n0] * s1[n1] * x[(int64_t)n0 * L1 + n1], R(0)} : C{0, 0};
    }
    __syncthreads();
    const C *out = run_fft<R, KT, BT, false>(buf, buf2, tws, B, pa.pl, tw);
    for (int e = threadIdx.x; e < B * K; e += NT) {
        const int s = e / K, c = e - s * K, n0 = row0 + s;
        if (n0 < L0 && colmask[c]) tmp[(int64_t)c * L0 + n0] = out[s * K + wrapK(c + K / 2, K)];
    }
}

// forward column pass: grid[r][c] = FFT_axis0(tmp padded)[(r + K0/2) mod K0][c]
template <typename R, int KT>
__global__ void __launch_bounds__(NT) k_cols_fwd(const cplx_t<R> *__restrict__ tmp, cplx_t<R> *__restrict__ grid,
                                                 const cplx_t<R> *__restrict__ tw, int L0, int K1,
                                                 const int32_t *__restrict__ strips,
                                                 const uint8_t *__restrict__ rowmask, PassArgs pa) {
    using C = cplx_t<R>;
    constexpr int WT = cols_ct<R, KT>();
    const int K = KT ? KT : pa.pl.K, W = KT ? WT : pa.nseq;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *buf2 = buf + W * K;
    const C *tws = KT ? stage_twiddles<R, WT, KT ? KT : 1>(buf, tw) : tw;
    pdl_enter();
    const int c0 = strips[blockIdx.x];
    // one pass over the padded strip: position p holds image row p + L0/2
    // (p < L0/2) or p - K + L0/2 (p >= K - L0/2), zero in between; the
    // column-major tmp makes consecutive threads read consecutive rows
    (void)K1;
    for (int e = threadIdx.x; e < W * K; e += NT) {
        const int s = e / K, p = e - s * K;
        const int n0 = p < L0 / 2 ? p + L0 / 2 : (p >= K - L0 / 2 ? p - K + L0 / 2 : -1);
        buf[p * W + s] = n0 >= 0 ? tmp[(int64_t)(c0 + s) * L0 + n0] : C{0, 0};
    }
    __syncthreads();
    const C *out = run_fft<R, KT, WT, true>(buf, buf2, tws, W, pa.pl, tw);
    for (int e = threadIdx.x; e < W * K; e += NT) {
        const int r = e / W, s = e - r * W;
        if (rowmask[r]) grid[(int64_t)r * K1 + c0 + s] = out[wrapK(r + K / 2, K) * W + s];
    }
}

// inverse column pass: tmp[n0][c] = (F^H along axis 0 of grid)[(n0 - L0/2) mod K0][c],
// the grid column-major (element (r, c) at c K0 + r, written by the combine
// pass), so that consecutive threads read consecutive rows
template <typename R, int KT>
__global__ void __launch_bounds__(NT) k_cols_inv(const cplx_t<R> *__restrict__ grid, cplx_t<R> *__restrict__ tmp,
                                                 const cplx_t<R> *__restrict__ tw, int L0, int K1,
                                                 const int32_t *__restrict__ strips,
                                                 const uint8_t *__restrict__ rowmask, PassArgs pa) {
    using C = cplx_t<R>;
    constexpr int WT = cols_ct<R, KT>();
    const int K = KT ? KT : pa.pl.K, W = KT ? WT : pa.nseq;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *buf2 = buf + W * K;
    const C *tws = KT ? stage_twiddles<R, WT, KT ? KT : 1>(buf, tw) : tw;
    pdl_enter();
    const int c0 = strips[blockIdx.x];
    for (int e = threadIdx.x; e < W * K; e += NT) {
        const int s = e / K, r = e - s * K;   // r: stored (centred) row; natural frequency (r + K/2) mod K
        buf[wrapK(r + K / 2, K) * W + s] = rowmask[r] ? cconj(grid[(int64_t)(c0 + s) * K + r]) : C{0, 0};
    }
    __syncthreads();
    const C *out = run_fft<R, KT, WT, true>(buf, buf2, tws, W, pa.pl, tw);
    for (int e = threadIdx.x; e < W * L0; e += NT) {
        const int n0 = e / W, s = e - n0 * W;
        tmp[(int64_t)n0 * K1 + c0 + s] = cconj(out[wrapK(n0 - L0 / 2 + K, K) * W + s]);
    }
}

// inverse row pass: img[n0][n1] = s0 s1 Re(F^H along axis 1 of tmp)[n0][(n1 - L1/2) mod K1]
template <typename R, int KT>
__global__ void __launch_bounds__(NT) k_rows_inv(const cplx_t<R> *__restrict__ tmp, R *__restrict__ img,
                                                 const cplx_t<R> *__restrict__ tw, const R *__restrict__ s0,
                                                 const R *__restrict__ s1, int L0, int L1, PassArgs pa) {
    using C = cplx_t<R>;
    constexpr int BT = rows_ct<R, KT>();
    const int K = KT ? KT : pa.pl.K, B = KT ? BT : pa.nseq;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *buf2 = buf + B * K;
    const C *tws = KT ? stage_twiddles<R, BT, KT ? KT : 1>(buf, tw) : tw;
    pdl_enter();
    if constexpr (KT != 0) {   // two rows per sequence
        const int row0 = blockIdx.x * 2 * BT;
        load_two_real_inverse<R, KT ? KT : 1, BT>(tmp, row0, L0, buf);
        __syncthreads();
        fft_smem<R, KT ? KT : 1, BT, false>(buf, tws);
        for (int e = threadIdx.x; e < BT * L1; e += NT) {
            const int s = e / L1, n1 = e % L1, ra = row0 + 2 * s, rb = ra + 1;
            const C v = buf[s * KT + ((n1 - L1 / 2 + KT) & (KT - 1))];
            if (ra < L0) img[(int64_t)ra * L1 + n1] = s0[ra] * s1[n1] * v.x;
            if (rb < L0) img[(int64_t)rb * L1 + n1] = -s0[rb] * s1[n1] * v.y;
        }
        return;
    }
    const int row0 = blockIdx.x * B;
    for (int e = threadIdx.x; e < B * K; e += NT) {
        const int s = e / K, c = e - s * K, n0 = row0 + s;
        buf[s * K + wrapK(c + K / 2, K)] = n0 < L0 ? cconj(tmp[(int64_t)n0 * K + c]) : C{0, 0};
    }
    __syncthreads();
    const C *out = run_fft<R, KT, BT, false>(buf, buf2, tws, B, pa.pl, tw);
    for (int e = threadIdx.x; e < B * L1; e += NT) {
        const int s = e / L1, n1 = e - s * L1, n0 = row0 + s;
        if (n0 < L0) img[(int64_t)n0 * L1 + n1] = s0[n0] * s1[n1] * out[s * K + wrapK(n1 - L1 / 2 + K, K)].x;
    }
}

// The end of one PPD iteration and the start of the next, B rows per CTA:
// the inverse row pass g = s0 s1 Re(F^H along axis 1 of tmp_inv) (the rows'
// Phi^dagger v, kept on chip), the primal step of Algorithm 3 on those
// pixels (primal_pixel), and the forward row pass of the new xt into
// tmp_fwd (the next iteration's first FFT pass), with the FP64 statistics
// partials of the CTA.  The join of the prior branch precedes it (ut, u0).
template <typename R, int KT>
__global__ void __launch_bounds__(NT) k_rows_primal(const cplx_t<R> *__restrict__ tmp_inv,
                                                    cplx_t<R> *__restrict__ tmp_fwd, const cplx_t<R> *__restrict__ tw,
                                                    const R *__restrict__ s0, const R *__restrict__ s1,
                                                    const uint8_t *__restrict__ colmask, PrimalArgs<R> P,
                                                    double *__restrict__ part, int L0, int L1, PassArgs pa) {
    using C = cplx_t<R>;
    constexpr int BT = rows_ct<R, KT>();
    const int K = KT ? KT : pa.pl.K, B = KT ? BT : pa.nseq;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *buf2 = buf + B * K;
    const C *tws = KT ? stage_twiddles<R, BT, KT ? KT : 1>(buf, tw) : tw;
    pdl_enter();
    PrimalSums<R> acc;
    if constexpr (KT != 0) {
        // two rows per sequence (rows row0 + 2s and row0 + 2s + 1)
        constexpr int KK = KT ? KT : 1, LT = KK / 2, PER = BT * LT / NT;
        static_assert(BT * LT % NT == 0, "pixel pairs per thread");
        const int row0 = blockIdx.x * 2 * BT;
        load_two_real_inverse<R, KK, BT>(tmp_inv, row0, L0, buf);
        // the primal step's pixel inputs, in flight during the inverse FFT
        // (up to K = 1024; longer rows keep them for later: at K = 2048 the
        // registers cost more than the overlap gains, 43 -> 49 us measured)
        constexpr bool PRE = KK <= 1024;
        PrimalIn<R> ina[PER], inb[PER];
        if constexpr (PRE) {
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int e = threadIdx.x + k * NT, s = e / LT, n1 = e % LT, ra = row0 + 2 * s, rb = ra + 1;
                if (ra < L0) ina[k] = primal_load(P, (int64_t)ra * LT + n1);
                if (rb < L0) inb[k] = primal_load(P, (int64_t)rb * LT + n1);
            }
        }
        __syncthreads();
        fft_smem<R, KK, BT, false>(buf, tws);
        // the new xt of both rows stays in registers while the buffer is rewritten
        R xa[PER], xb[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + k * NT, s = e / LT, n1 = e % LT, ra = row0 + 2 * s, rb = ra + 1;
            const C v = buf[s * KK + ((n1 - LT / 2 + KK) & (KK - 1))];
            xa[k] = xb[k] = R(0);
            const int64_t ea = (int64_t)ra * LT + n1, eb = (int64_t)rb * LT + n1;
            if (ra < L0) xa[k] = primal_pixel(P, ea, s0[ra] * s1[n1] * v.x, PRE ? ina[k] : primal_load(P, ea), acc);
            if (rb < L0) xb[k] = primal_pixel(P, eb, -s0[rb] * s1[n1] * v.y, PRE ? inb[k] : primal_load(P, eb), acc);
        }
        __syncthreads();
        // the new rows a + i b in place, each thread also clearing the padding
        // position K/2 away from its pixel's (the padding is [LT/2, K - LT/2))
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + k * NT, s = e / LT, n1 = e % LT, ra = row0 + 2 * s, rb = ra + 1;
            const int pos = (n1 - LT / 2 + KK) & (KK - 1);
            buf[s * KK + pos] = C{ra < L0 ? s0[ra] * s1[n1] * xa[k] : R(0), rb < L0 ? s0[rb] * s1[n1] * xb[k] : R(0)};
            buf[s * KK + ((pos + LT) & (KK - 1))] = C{0, 0};
        }
        __syncthreads();
        fft_smem<R, KK, BT, false>(buf, tws);
        store_two_real_forward<R, KK, BT>(buf, row0, L0, colmask, tmp_fwd);
        acc.write(part + 3 * (int64_t)blockIdx.x);
        return;
    }
    const int row0 = blockIdx.x * B;
    for (int e = threadIdx.x; e < B * K; e += NT) {
        const int s = e / K, c = e - s * K, n0 = row0 + s;
        buf[s * K + wrapK(c + K / 2, K)] = n0 < L0 ? cconj(tmp_inv[(int64_t)n0 * K + c]) : C{0, 0};
    }
    __syncthreads();
    C *out = run_fft<R, KT, BT, false>(buf, buf2, tws, B, pa.pl, tw);
    {
        // the mixed-radix core leaves the result in one buffer: the forward
        // input is built in the other one
        C *fin = out == buf ? buf2 : buf;
        for (int e = threadIdx.x; e < B * K; e += NT) fin[e] = C{0, 0};
        __syncthreads();
        for (int e = threadIdx.x; e < B * L1; e += NT) {
            const int s = e / L1, n1 = e - s * L1, n0 = row0 + s;
            if (n0 < L0) {
                const int pos = wrapK(n1 - L1 / 2 + K, K);
                const R g = s0[n0] * s1[n1] * out[s * K + pos].x;
                const R xtn = primal_pixel(P, (int64_t)n0 * L1 + n1, g, acc);
                fin[s * K + pos] = C{s0[n0] * s1[n1] * xtn, R(0)};
            }
        }
        __syncthreads();
        buf = fin;
        buf2 = out;
    }
    const C *res = run_fft<R, KT, BT, false>(buf, buf2, tws, B, pa.pl, tw);
    for (int e = threadIdx.x; e < B * K; e += NT) {
        const int s = e / K, c = e - s * K, n0 = row0 + s;
        if (n0 < L0 && colmask[c]) tmp_fwd[(int64_t)c * L0 + n0] = res[s * K + wrapK(c + K / 2, K)];
    }
    acc.write(part + 3 * (int64_t)blockIdx.x);
}

// ------------------------------------------------------------ launchers
// Sequences per CTA of the mixed-radix passes: rows: enough for ~1024
// points; columns: the largest power of two <= 1024 / K (at most 32, so
// that it divides K1, a multiple of 32).
int any_rows(int K) { return std::max(1, 1024 / K); }
int any_cols(int K) {
    int w = 1;
    while (w < 32 && 2 * w * K <= 1024) w *= 2;
    return w;
}

// Row passes have the row length K1, column passes the column length K0.
// RowPass / ColPass hold the launches of one core (KT) and precision.
template <typename R, int KT> struct RowPass {
    static constexpr int BT = rows_ct<R, KT>();
    static int nseq(const ppd_ctx *c) { return KT ? BT : any_rows(c->K1); }
    static size_t smem(const ppd_ctx *c) {
        return KT ? pass_smem<R>(BT, KT) : (size_t)2 * nseq(c) * c->K1 * 2 * sizeof(R);
    }
    static PassArgs args(const ppd_ctx *c) { return PassArgs{c->plan1, nseq(c)}; }
    // rows per CTA: two per sequence in the power-of-two core
    static int rows(const ppd_ctx *c) { return KT ? 2 * BT : nseq(c); }
    static unsigned blocks(const ppd_ctx *c) { return (unsigned)((c->L0 + rows(c) - 1) / rows(c)); }
    static const cplx_t<R> *tw(const ppd_ctx *c) {
        return static_cast<const cplx_t<R> *>(KT ? c->twst1 : c->tw1);
    }
    static int fwd(ppd_ctx *c, const R *x, cudaStream_t s) {
        const int sh = (int)smem(c);
        PPD_CHECK(smem_attr((const void *)k_rows_fwd<R, KT>, sh));
        int site;
        PPD_CHECK(launch_begin(c, "fft_fwd_rows", s, &site));
        // mostly the first kernel of its sequence: an ordinary launch
        launch(c, false, k_rows_fwd<R, KT>, blocks(c), NT, sh, s, x, static_cast<cplx_t<R> *>(c->fft_tmp), tw(c),
               static_cast<const R *>(c->deap0), static_cast<const R *>(c->deap1), c->L0, c->L1,
               (const uint8_t *)c->col_fwd, args(c));
        return launch_end(c, site, s);
    }
    static int inv(ppd_ctx *c, R *img, cudaStream_t s) {
        const int sh = (int)smem(c);
        PPD_CHECK(smem_attr((const void *)k_rows_inv<R, KT>, sh));
        int site;
        PPD_CHECK(launch_begin(c, "fft_inv_rows", s, &site));
        launch(c, true, k_rows_inv<R, KT>, blocks(c), NT, sh, s, static_cast<const cplx_t<R> *>(c->fft_tmp_inv),
               img, tw(c), static_cast<const R *>(c->deap0), static_cast<const R *>(c->deap1), c->L0, c->L1,
               args(c));
        return launch_end(c, site, s);
    }
    static int primal(ppd_ctx *c, cudaStream_t s) {
        const int sh = (int)smem(c);
        PPD_CHECK(smem_attr((const void *)k_rows_primal<R, KT>, sh));
        int site;
        PPD_CHECK(launch_begin(c, "rows_primal", s, &site));
        const unsigned n = blocks(c);
        // it follows the join of the two branches: an ordinary launch
        launch(c, false, k_rows_primal<R, KT>, n, NT, sh, s, static_cast<const cplx_t<R> *>(c->fft_tmp_inv),
               static_cast<cplx_t<R> *>(c->fft_tmp), tw(c), static_cast<const R *>(c->deap0),
               static_cast<const R *>(c->deap1), (const uint8_t *)c->col_fwd, primal_args<R>(c), c->prim_part, c->L0,
               c->L1, args(c));
        c->n_stat_parts = (int)n;
        return launch_end(c, site, s);
    }
};

template <typename R, int KT> struct ColPass {
    static constexpr int WT = cols_ct<R, KT>();
    static int nseq(const ppd_ctx *c) { return KT ? WT : any_cols(c->K0); }
    static size_t smem(const ppd_ctx *c) {
        return KT ? pass_smem<R>(WT, KT) : (size_t)2 * nseq(c) * c->K0 * 2 * sizeof(R);
    }
    static PassArgs args(const ppd_ctx *c) { return PassArgs{c->plan0, nseq(c)}; }
    static const cplx_t<R> *tw(const ppd_ctx *c) {
        return static_cast<const cplx_t<R> *>(KT ? c->twst0 : c->tw0);
    }
    static int fwd(ppd_ctx *c, cplx_t<R> *grid, cudaStream_t s) {
        if (c->n_fwd_strips == 0) return PPD_OK;
        const int sh = (int)smem(c);
        PPD_CHECK(smem_attr((const void *)k_cols_fwd<R, KT>, sh));
        int site;
        PPD_CHECK(launch_begin(c, "fft_fwd_cols", s, &site));
        launch(c, true, k_cols_fwd<R, KT>, (unsigned)c->n_fwd_strips, NT, sh, s,
               static_cast<const cplx_t<R> *>(c->fft_tmp), grid, tw(c), c->L0, c->K1,
               (const int32_t *)c->fwd_strips, (const uint8_t *)c->row_fwd, args(c));
        return launch_end(c, site, s);
    }
    static int inv(ppd_ctx *c, const cplx_t<R> *grid, cudaStream_t s) {
        if (c->n_inv_strips == 0) return PPD_OK;
        const int sh = (int)smem(c);
        PPD_CHECK(smem_attr((const void *)k_cols_inv<R, KT>, sh));
        int site;
        PPD_CHECK(launch_begin(c, "fft_inv_cols", s, &site));
        launch(c, true, k_cols_inv<R, KT>, (unsigned)c->n_inv_strips, NT, sh, s, grid,
               static_cast<cplx_t<R> *>(c->fft_tmp_inv), tw(c), c->L0, c->K1, (const int32_t *)c->inv_strips,
               (const uint8_t *)c->row_inv, args(c));
        return launch_end(c, site, s);
    }
};

}  // namespace

// Power-of-two lengths take the compile-time core; other 5-smooth lengths
// the mixed-radix one (KT = 0).
#define PPD_FFT_DISPATCH(KLEN, PASS, CALL)                  \
    switch (KLEN) {                                         \
        case 32: return PASS<R, 32>::CALL;                  \
        case 64: return PASS<R, 64>::CALL;                  \
        case 128: return PASS<R, 128>::CALL;                \
        case 256: return PASS<R, 256>::CALL;                \
        case 512: return PASS<R, 512>::CALL;                \
        case 1024: return PASS<R, 1024>::CALL;              \
        case 2048: return PASS<R, 2048>::CALL;              \
        case 4096: return PASS<R, 4096>::CALL;              \
        case 8192: return PASS<R, 8192>::CALL;              \
        default: return PASS<R, 0>::CALL;                   \
    }

// forward row pass of x into the FFT temporary (first half of F Z x)
template <typename R> int fft_forward_rows(ppd_ctx *c, const R *x, cudaStream_t s) {
    c->xt_rows_valid = false;
    PPD_FFT_DISPATCH(c->K1, RowPass, fwd(c, x, s))
}

// forward column pass from the FFT temporary to the grid (second half of F Z x)
template <typename R> int fft_forward_cols(ppd_ctx *c, cplx_t<R> *grid, cudaStream_t s) {
    PPD_FFT_DISPATCH(c->K0, ColPass, fwd(c, grid, s))
}

// inverse column pass of a combined grid into the inverse temporary
template <typename R> int fft_inverse_cols(ppd_ctx *c, const cplx_t<R> *grid, cudaStream_t s) {
    PPD_FFT_DISPATCH(c->K0, ColPass, inv(c, grid, s))
}

// inverse row pass into an image (second half of Z^T F^H)
template <typename R> int fft_inverse_rows(ppd_ctx *c, R *img, cudaStream_t s) {
    PPD_FFT_DISPATCH(c->K1, RowPass, inv(c, img, s))
}

// inverse row pass + primal step + forward row pass of the new xt
template <typename R> int rows_primal(ppd_ctx *c, cudaStream_t s) {
    PPD_FFT_DISPATCH(c->K1, RowPass, primal(c, s))
}

template <typename R> int fft_forward(ppd_ctx *c, const R *x, cplx_t<R> *grid, cudaStream_t s) {
    PPD_CHECK(fft_forward_rows<R>(c, x, s));
    return fft_forward_cols<R>(c, grid, s);
}

template <typename R> int fft_inverse(ppd_ctx *c, const cplx_t<R> *grid, R *img, cudaStream_t s) {
    PPD_CHECK(fft_inverse_cols<R>(c, grid, s));
    return fft_inverse_rows<R>(c, img, s);
}

#undef PPD_FFT_DISPATCH

#define PPD_FFT_INST(R)                                                                                         \
    template int fft_forward<R>(ppd_ctx *, const R *, cplx_t<R> *, cudaStream_t);                              \
    template int fft_inverse<R>(ppd_ctx *, const cplx_t<R> *, R *, cudaStream_t);                              \
    template int fft_forward_rows<R>(ppd_ctx *, const R *, cudaStream_t);                                       \
    template int fft_forward_cols<R>(ppd_ctx *, cplx_t<R> *, cudaStream_t);                                     \
    template int fft_inverse_cols<R>(ppd_ctx *, const cplx_t<R> *, cudaStream_t);                              \
    template int fft_inverse_rows<R>(ppd_ctx *, R *, cudaStream_t);                                             \
    template int rows_primal<R>(ppd_ctx *, cudaStream_t);
PPD_FFT_INST(float)
PPD_FFT_INST(double)
#undef PPD_FFT_INST

// FFT plan of length K: radices 5, 3, then 4, then a last 2 (an empty plan
// if K has another prime factor).
FftPlan make_fft_plan(int K) {
    FftPlan p{};
    p.K = K;
    int k = K;
    for (int r : {5, 3})
        while (k % r == 0 && p.ns < FftPlan::MAX_STAGES) {
            p.rad[p.ns++] = r;
            k /= r;
        }
    while (k % 4 == 0 && p.ns < FftPlan::MAX_STAGES) {
        p.rad[p.ns++] = 4;
        k /= 4;
    }
    if (k == 2 && p.ns < FftPlan::MAX_STAGES) {
        p.rad[p.ns++] = 2;
        k = 1;
    }
    if (k != 1) p.ns = 0;
    return p;
}

bool fft_length_supported(int K, bool fp64) {
    if (K < 32 || K > 8192 || make_fft_plan(K).ns == 0) return false;
    const bool pow2 = (K & (K - 1)) == 0;
    // two buffers of the mixed-radix core per CTA: at most 128 KB
    return pow2 || (size_t)2 * K * 2 * (fp64 ? 8 : 4) <= 128 * 1024;
}

// Column strips (W columns each, W as the column passes use) that contain a
// marked column, and the row / column masks, uploaded for the pruned passes.
int fft_plan_pruning(ppd_ctx *c, const std::vector<char> &rows_fwd, const std::vector<char> &cols_fwd,
                     const std::vector<char> &rows_inv, const std::vector<char> &cols_inv) {
    const int K0 = c->K0, K1 = c->K1;
    const bool p2 = (K0 & (K0 - 1)) == 0;
    const int W = !p2 ? any_cols(K0) : c->is_f32 ? cols_per_cta<float>(K0) : cols_per_cta<double>(K0);
    std::vector<int32_t> fs, is;
    for (int s0 = 0; s0 < K1; s0 += W) {
        bool f = false, i = false;
        for (int j = s0; j < s0 + W && j < K1; ++j) {
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
    PPD_CUDA(cudaMemcpy(c->row_fwd, rf.data(), K0, cudaMemcpyHostToDevice));
    PPD_CUDA(cudaMemcpy(c->row_inv, ri.data(), K0, cudaMemcpyHostToDevice));
    PPD_CUDA(cudaMemcpy(c->col_fwd, cf.data(), K1, cudaMemcpyHostToDevice));
    // the inverse column pass writes only its strips: the rest of its output
    // stays zero; the forward row pass writes only marked columns
    PPD_CUDA(cudaMemset(c->fft_tmp_inv, 0, (size_t)c->L0 * K1 * 2 * c->rsz));
    PPD_CUDA(cudaMemset(c->fft_tmp, 0, (size_t)c->L0 * K1 * 2 * c->rsz));
    return PPD_OK;
}

// Twiddles exp(-2 pi i m / K), m < K, computed in double on the host, for
// the column length K0 (tw0) and the row length K1 (tw1).
static int upload_twiddles(ppd_ctx *c, int K, void *dst) {
    std::vector<double> t(2 * (size_t)K);
    for (int m = 0; m < K; ++m) {
        double a = -2.0 * M_PI * (double)m / (double)K;
        t[2 * m] = std::cos(a);
        t[2 * m + 1] = std::sin(a);
    }
    if (c->is_f32) {
        std::vector<float> f(t.begin(), t.end());
        PPD_CUDA(cudaMemcpy(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        PPD_CUDA(cudaMemcpy(dst, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return PPD_OK;
}

// Twiddles of the power-of-two core stage by stage (K entries, zero padded):
// the radix-4 stages of span Ns = 2 or 4, then x4 up to K/4, each with
// w^(q k K / (4 Ns)) at (q - 1) Ns + k, q = 1..3, k < Ns.
static int upload_stage_twiddles(ppd_ctx *c, int K, void *dst) {
    std::vector<double> t(2 * (size_t)K, 0.0);
    if ((K & (K - 1)) == 0) {
        size_t off = 0;
        for (int Ns = (ilog2_(K) & 1) ? 2 : 4; Ns < K; Ns *= 4)
            for (int q = 1; q <= 3; ++q)
                for (int k = 0; k < Ns; ++k, ++off) {
                    const double a = -2.0 * M_PI * (double)q * k / (4.0 * Ns);
                    t[2 * off] = std::cos(a);
                    t[2 * off + 1] = std::sin(a);
                }
    }
    if (c->is_f32) {
        std::vector<float> f(t.begin(), t.end());
        PPD_CUDA(cudaMemcpy(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        PPD_CUDA(cudaMemcpy(dst, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return PPD_OK;
}

int make_twiddles(ppd_ctx *c) {
    c->plan0 = make_fft_plan(c->K0);
    c->plan1 = make_fft_plan(c->K1);
    PPD_CHECK(upload_twiddles(c, c->K0, c->tw0));
    PPD_CHECK(upload_twiddles(c, c->K1, c->tw1));
    PPD_CHECK(upload_stage_twiddles(c, c->K0, c->twst0));
    return upload_stage_twiddles(c, c->K1, c->twst1);
}

// Z's scaling s(n) = 1 / psi_hat((n - L/2)/K), psi_hat(f) = (J / I0(beta)) sinh(q)/q,
// q = sqrt(beta^2 - (pi J f)^2): the Fourier transform of the Kaiser-Bessel kernel.
static int upload_deapodisation(ppd_ctx *c, int L, int K, void *dst) {
    const double J = KB_J, beta = c->beta, i0b = std::cyl_bessel_i(0.0, beta);
    std::vector<double> s(L);
    for (int n = 0; n < L; ++n) {
        double f = ((double)n - L / 2) / (double)K;
        double q = std::sqrt(beta * beta - (M_PI * J * f) * (M_PI * J * f));
        s[n] = 1.0 / ((J / i0b) * std::sinh(q) / q);
    }
    if (c->is_f32) {
        std::vector<float> f(s.begin(), s.end());
        PPD_CUDA(cudaMemcpy(dst, f.data(), L * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        PPD_CUDA(cudaMemcpy(dst, s.data(), L * sizeof(double), cudaMemcpyHostToDevice));
    }
    return PPD_OK;
}

int make_deapodisation(ppd_ctx *c) {
    PPD_CHECK(upload_deapodisation(c, c->L0, c->K0, c->deap0));
    return upload_deapodisation(c, c->L1, c->K1, c->deap1);
}

}  // namespace ppd
