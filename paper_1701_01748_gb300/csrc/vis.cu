// Visibility-side kernels of PPD.
//
//  * binning (Section 2: G's 8 x 8 Kaiser-Bessel taps, Section 5: n = 4
//    oversampling; Section 4.3 / Section 5: sampling density per grid cell)
//  * degridding G with the data step of Algorithm 3 fused in (z = U^-1 v +
//    Theta G a, first forward-backward step of Algorithm 2, block norms)
//  * extra Algorithm 2 sub-iterations and the per-block l2-ball scale
//  * gridding G^dagger Theta^dagger v with the dual update fused in
//    (vbar = U (z - P_B(w))), accumulated per tile in shared memory and
//    summed across work items in a fixed order (deterministic, no atomics)
//
// Work decomposition: visibilities are sorted by (tile of the centred grid
// holding the first tap, block, base cell); a "chunk" is a run of at most C
// visibilities of one tile and one block, and each CTA owns one chunk.  The
// CTA stages the (T+8) x (T+8) extended grid tile in shared memory (TMA for
// interior tiles, wrapped plain loads at the grid edge) for degridding, or
// accumulates into it for gridding.
#include <cmath>

#include "common.cuh"
#include "tma.cuh"

namespace ppd {

namespace {

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }

// ----------------------------------------------------------------- binning
// kappa = (omega * K) * (1/(2 pi)) with correctly rounded multiplies (no FMA
// contraction possible), f = floor(kappa), first tap (f - 3) mod K, fraction
// kappa - f, nearest cell floor(kappa + 0.5) mod K.
__global__ void k_bin(const double *__restrict__ uv, const int32_t *__restrict__ blk, int64_t M, int K0, int K1,
                      int T, int d, uint64_t *__restrict__ key, int32_t *__restrict__ base,
                      double *__restrict__ frac, int32_t *__restrict__ cell, int32_t *__restrict__ count_grid,
                      int *__restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const double om0 = uv[2 * i], om1 = uv[2 * i + 1];
        const int b = blk[i];
        if (!(om0 >= -M_PI && om0 <= M_PI && om1 >= -M_PI && om1 <= M_PI) || b < 0 || b >= d) {
            atomicOr(bad, 1);
            key[i] = 0;
            base[2 * i] = base[2 * i + 1] = 0;
            frac[2 * i] = frac[2 * i + 1] = 0.0;
            cell[i] = 0;   // a valid cell for k_cell_count; the call fails on `bad`
            continue;
        }
        const double k0 = __dmul_rn(__dmul_rn(om0, (double)K0), INV_TWO_PI);
        const double k1 = __dmul_rn(__dmul_rn(om1, (double)K1), INV_TWO_PI);
        const double f0 = floor(k0), f1 = floor(k1);
        const int64_t i0 = (int64_t)f0, i1 = (int64_t)f1;
        const int b0 = (int)(((i0 - 3) % K0 + K0) % K0);
        const int b1 = (int)(((i1 - 3) % K1 + K1) % K1);
        const int cb0 = (b0 + K0 / 2) % K0, cb1 = (b1 + K1 / 2) % K1;
        const int64_t n0 = (((int64_t)floor(__dadd_rn(k0, 0.5))) % K0 + K0) % K0;
        const int64_t n1 = (((int64_t)floor(__dadd_rn(k1, 0.5))) % K1 + K1) % K1;
        const uint64_t tile = (uint64_t)(cb0 / T) * (uint64_t)(K1 / T) + (uint64_t)(cb1 / T);
        key[i] = ((tile * (uint64_t)d + (uint64_t)b) * (uint64_t)K0 + (uint64_t)cb0) * (uint64_t)K1 + (uint64_t)cb1;
        base[2 * i] = b0;
        base[2 * i + 1] = b1;
        frac[2 * i] = __dsub_rn(k0, f0);
        frac[2 * i + 1] = __dsub_rn(k1, f1);
        const int c = (int)(n0 * K1 + n1);
        cell[i] = c;
        atomicAdd(&count_grid[c], 1);
    }
}

__global__ void k_cell_count(const int32_t *__restrict__ cell, const int32_t *__restrict__ count_grid, int64_t M,
                             int32_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = count_grid[cell[i]];
}

// ----------------------------------------------------------------- weights
// FP32: per tap j a degree-KB_DEG polynomial in t = 2 frac - 1 (Chebyshev fit
// of psi(frac + 3 - j) made on the host); coefficients p[k*8 + j].  p is a
// kernel argument, so with the loops unrolled every coefficient is a
// constant-bank operand of its FMA: no load instruction.
constexpr int KB_NC = (KB_DEG + 1) * KB_J;
__device__ __forceinline__ void kb_weights(float frac, float (&w)[KB_J], const float (&p)[KB_NC], double, double) {
    const float t = fmaf(2.0f, frac, -1.0f);
#pragma unroll
    for (int j = 0; j < KB_J; ++j) w[j] = p[KB_DEG * KB_J + j];
#pragma unroll
    for (int k = KB_DEG - 1; k >= 0; --k)
#pragma unroll
        for (int j = 0; j < KB_J; ++j) w[j] = fmaf(w[j], t, p[k * KB_J + j]);
}

// FP64: the kernel itself, psi(d) = I0(beta sqrt(1 - (d/4)^2)) / I0(beta), d = frac + 3 - j.
__device__ __forceinline__ void kb_weights(double frac, double (&w)[KB_J], const float (&)[KB_NC], double beta,
                                           double inv_i0b) {
#pragma unroll
    for (int j = 0; j < KB_J; ++j) {
        const double dd = (frac + (double)(3 - j)) * 0.25;
        const double x = 1.0 - dd * dd;
        w[j] = x >= 0.0 ? cyl_bessel_i0(beta * sqrt(x)) * inv_i0b : 0.0;
    }
}

template <typename R> struct VisArgs {
    const VisRec<R> *rec;
    const R *theta_v;
    R theta_s;
    const int32_t *ch_start, *ch_count, *ch_tile, *ch_block;
    const int32_t *ch_order;   // chunks by decreasing size: the gridding's CTA order
    // work units of the degridding and sub-iteration kernels: runs of at
    // most DG_NT visibilities of one chunk, each with its partial slot
    const int32_t *u_start, *u_count, *u_chunk, *u_order;
    // the degridding's work counters: [0] next position in u_order to claim,
    // [1] CTAs finished (both back to zero after every launch)
    int *claim;
    int K0, K1, ntile1;
    float kbp[KB_NC];   // the FP32 weight polynomials (kb_weights)
    double beta, inv_i0b;
    const cplx_t<R> *y;
    cplx_t<R> *v, *z, *w, *p;
    const double *mu, *scale;
    double *partials;            // this launch's chunk partials
    const double *part_in;       // previous step's chunk partials (P_B scale)
    // partials live in block-major slots: work unit u writes slot
    // u_pos[u]; block b's slots are blk_ptr[b] .. blk_ptr[b+1] - 1
    const int32_t *blk_ptr, *u_pos;
    const double *eps;
    int *err;
    // randomised active sets (null: every block active): the current
    // iteration's block flags, per-block "has a prox output" flags, and the
    // flag that makes the gridding redo the partial tiles of inactive blocks
    const uint8_t *bmask;
    uint8_t *seen;
    const int *regrid;
    // operator mode I/O (caller order through perm when non-null)
    const cplx_t<R> *op_in;
    cplx_t<R> *op_out;
    const int64_t *perm;
    // Algorithm 2 stopping test (inner_tol > 0): this launch's step number
    // (0: the step that forms the start P_B(z); 1 .. n_itr - 1: sub-iterations;
    // n_itr: the gridding), whether part_in holds the previous step's test
    // partials, per block the step at which the test held (0: running) and
    // the steps taken
    double inner_tol;
    int step, test_in, n_itr;
    int *inner_state, *inner_steps;
};

// Deterministic CTA sum of two doubles per thread (fixed shuffle tree, then
// warps in order).
template <int NT> __device__ void cta_sum2(double a, double b, double *out2) {
    __shared__ double red[2][NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][wid] = a;
        red[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0;
        for (int i = 0; i < NT / 32; ++i) {
            s0 += red[0][i];
            s1 += red[1][i];
        }
        out2[0] = s0;
        out2[1] = s1;
    }
}

// Kahan-compensated FP32 accumulator (FP64 accumulation in the FP64 path).
template <typename R> struct Acc {
    R s = 0, c = 0;
    __device__ void add(R x) {
        R y = x - c;
        R t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ double get() const { return (double)s - (double)c; }
};

constexpr int DG_NT = 256;

// P_B scale of block `blk` (Section 3.3, Eq. "proj-L2" as a radial scale):
// eps / ||w - y|| if that norm exceeds eps, else 1, from the previous step's
// chunk partials summed in a fixed order (the same result in every CTA).
// With `test`, *stop also receives Algorithm 2's stopping test of the
// previous step, ||zbar^t - zbar^(t-1)|| <= inner_tol ||zbar^t||, in FP64.
// Every thread of the CTA loads a strided share of the block's contiguous
// slots (one round trip), then a fixed-order tree and warp order sum them.
template <typename R> __device__ double block_scale(const VisArgs<R> &A, int blk, bool test = false,
                                                   bool *stop = nullptr) {
    __shared__ double sc_s;
    __shared__ int st_s;
    __shared__ double red[3][32];
    double a = 0, dd = 0, nn = 0;
    for (int k = A.blk_ptr[blk] + threadIdx.x; k < A.blk_ptr[blk + 1]; k += blockDim.x) {
        const double *q = A.part_in + NPART * (int64_t)k;
        a += q[0];
        if (test) {
            dd += q[2];
            nn += q[3];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        dd += __shfl_down_sync(0xffffffffu, dd, o);
        nn += __shfl_down_sync(0xffffffffu, nn, o);
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][wid] = a;
        red[1][wid] = dd;
        red[2][wid] = nn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0, sd = 0, sn = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sa += red[0][w];
            sd += red[1][w];
            sn += red[2][w];
        }
        const double nrm = sqrt(sa);
        if (!isfinite(nrm)) atomicOr(A.err, ERR_NONFINITE);
        sc_s = (nrm > A.eps[blk]) ? A.eps[blk] / nrm : 1.0;
        st_s = test && sqrt(sd) <= A.inner_tol * sqrt(sn);
    }
    __syncthreads();
    if (stop) *stop = st_s != 0;
    return sc_s;
}

// Step at which block `blk` stopped Algorithm 2 in this iteration (0: still
// running), read once per CTA so that every thread takes the same branch.
template <typename R> __device__ int inner_stopped(const VisArgs<R> &A, int blk) {
    __shared__ int s_state;
    if (threadIdx.x == 0) s_state = (A.inner_tol > 0) ? *(volatile const int *)(A.inner_state + blk) : 0;
    __syncthreads();
    return s_state;
}

// ----------------------------------------------------------------- degrid
// mode DG_OP:    op_out[perm[i]] = Theta G a
// mode DG_DUAL:  z = v/U + Theta G a;  w = p - mu U (p - z)
// mode DG_FIRST: z = v/U + Theta G a;  w = z   (Algorithm 2 then starts from P_B(z))
// partial slot of the unit = (||w - y||^2, ||Theta G a - y||^2)
//
// Persistent CTAs walk the work units (the chunks) in the order u_order
// (largest first): CTA b starts at position b, then every CTA claims its
// next position from a counter when it starts a unit (so the light units
// of the tail go to whichever CTAs finish first); the last CTA to finish
// resets the counters for the next launch.  Which CTA computes a unit does
// not change any result.
// The (T+8)^2 grid tile of the next unit is fetched by TMA into the other of
// two shared buffers while the current unit is computed (interior tiles;
// tiles that wrap around the grid edge are loaded with plain loads when they
// are used); each thread loads its first visibility of the next unit before
// the current one is computed, and one visibility ahead inside a unit.
template <typename R> struct VisIn {
    VisRec<R> rc;
    cplx_t<R> v, y, p;
    R th;
};

template <typename R, int MODE>
__device__ __forceinline__ void load_vis(const VisArgs<R> &A, int gi, VisIn<R> &o) {
    o.rc = A.rec[gi];
    o.th = A.theta_v ? A.theta_v[gi] : A.theta_s;
    if (MODE != DG_OP) {
        o.v = A.v[gi];
        o.y = A.y[gi];
        if (MODE == DG_DUAL) o.p = A.p[gi];
    }
}

// NTD threads per CTA (256 or 128; FP64: 256): the autotuner picks per
// problem, fewer threads giving more CTAs per SM and shorter barriers.
template <typename R, int T, int MODE, int NTD>
__global__ void __launch_bounds__(NTD, sizeof(R) == 4 ? 768 / NTD : 1)
    k_degrid(const __grid_constant__ CUtensorMap tmap, int use_tma, const cplx_t<R> *__restrict__ grid, VisArgs<R> A,
             int n_units, long long spin_first) {
    using C = cplx_t<R>;
    constexpr int E = T + HALO;
    constexpr int TILE_BYTES = E * E * (int)sizeof(C);
    constexpr int TILE_STRIDE = (TILE_BYTES + 127) / 128 * 128;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar[2];
    __shared__ int ok_s;

    if (threadIdx.x == 0) {
        ok_s = 1;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    pdl_enter();   // the grid, v and p come from the kernels before
    auto origin = [&](int u, int &row0, int &col0) {
        const int tl = A.ch_tile[A.u_chunk[u]];
        row0 = (tl / A.ntile1) * T;
        col0 = (tl % A.ntile1) * T;
    };
    auto interior = [&](int row0, int col0) { return use_tma && row0 + E <= A.K0 && col0 + E <= A.K1; };
    auto issue = [&](int u, int buf) {   // thread 0 only
        int r0, c0;
        origin(u, r0, c0);
        if (interior(r0, c0)) {
            mbar_expect_tx(&bar[buf], (uint32_t)TILE_BYTES);
            tma_load_2d(smem_raw + buf * TILE_STRIDE, &tmap, 2 * c0, r0, &bar[buf]);
        }
    };
    uint32_t ph = 0u;   // bit b: parity of the next completion of bar[b]
    const int32_t *ord = A.u_order;
    __shared__ int claim_s;
    auto claim = [&](int from) {   // thread 0: the next position after `from` (n_units: none)
        claim_s = from < n_units ? (int)gridDim.x + atomicAdd(A.claim, 1) : n_units;
    };
    if (threadIdx.x == 0) {
        if ((int)blockIdx.x < n_units) issue(ord[blockIdx.x], 0);
        claim(blockIdx.x);
    }
    VisIn<R> cur;
    if ((int)blockIdx.x < n_units && (int)threadIdx.x < A.u_count[ord[blockIdx.x]])
        load_vis<R, MODE>(A, A.u_start[ord[blockIdx.x]] + threadIdx.x, cur);
    __syncthreads();
    int nxt_pos = min(claim_s, n_units);
    int it = 0;
    for (int iu = blockIdx.x; iu < n_units; iu = nxt_pos, nxt_pos = min(claim_s, n_units), ++it) {
        const int buf = it & 1;
        C *tile = reinterpret_cast<C *>(smem_raw + buf * TILE_STRIDE);
        const int u = ord[iu];
        const int nxt = nxt_pos < n_units ? ord[nxt_pos] : n_units;
        if (threadIdx.x == 0 && nxt < n_units) issue(nxt, buf ^ 1);
        const int start = A.u_start[u], count = A.u_count[u], ch = A.u_chunk[u];
        int row0, col0;
        origin(u, row0, col0);
        if (interior(row0, col0)) {
            // spin_first bounds the first wait (SPIN_LIMIT unless a test shortens
            // it); the waits for copies in flight before leaving keep SPIN_LIMIT
            if (!mbar_wait(&bar[buf], (ph >> buf) & 1u, spin_first)) {
                atomicOr(A.err, ERR_TMA_TIMEOUT);
                ok_s = 0;
                mbar_wait(&bar[buf], (ph >> buf) & 1u, SPIN_LIMIT);   // second bounded wait for the copy in flight
            }
            ph ^= 1u << buf;
            __syncthreads();
            if (!ok_s) {
                // the next unit's copy may be in flight: wait for it (bounded) before leaving
                if (nxt < n_units) {
                    int r1, c1;
                    origin(nxt, r1, c1);
                    if (interior(r1, c1)) mbar_wait(&bar[buf ^ 1], (ph >> (buf ^ 1)) & 1u, SPIN_LIMIT);
                }
                break;
            }
        } else {
            for (int e = threadIdx.x; e < E * E; e += NTD) {
                const int r = e / E, cc = e % E;
                tile[e] = grid[(int64_t)((row0 + r) % A.K0) * A.K1 + (col0 + cc) % A.K1];
            }
            __syncthreads();
        }
        const int blk = A.ch_block[ch];
        const double mu = (MODE != DG_OP) ? A.mu[blk] : 0.0;
        // block outside the active set D: z, w untouched (only the residual
        // statistic is formed); block without a prox output yet: w = z, so
        // that the next Algorithm 2 step starts from P_B(z)
        const bool act = MODE == DG_OP || !A.bmask || A.bmask[blk];
        const bool first_blk = MODE == DG_FIRST || (A.seen && !A.seen[blk]);
        if (MODE != DG_OP && threadIdx.x == 0) {
            if (A.inner_tol > 0) A.inner_state[blk] = 0;
            if (A.inner_steps) A.inner_steps[blk] = act ? A.n_itr : 0;
        }
        // with the stopping test the start zbar^(0) = z of a block without a
        // prox output is kept in p, the previous point of the first test
        const bool keep_start = first_blk && A.inner_tol > 0;
        Acc<R> s_w, s_r;
        for (int i = threadIdx.x; i < count; i += NTD) {
            const int gi = start + i;
            VisIn<R> nx;   // the next visibility: of this unit, else the next unit's first
            if (i + NTD < count) load_vis<R, MODE>(A, gi + NTD, nx);
            const int lb0 = (cur.rc.packed & 0xffff) - row0, lb1 = ((cur.rc.packed >> 16) & 0xffff) - col0;
            R w0[KB_J], w1[KB_J];
            kb_weights(cur.rc.f0, w0, A.kbp, A.beta, A.inv_i0b);
            kb_weights(cur.rc.f1, w1, A.kbp, A.beta, A.inv_i0b);
            C q{0, 0};
#pragma unroll
            for (int a = 0; a < KB_J; ++a) {
                const C *row = tile + (lb0 + a) * E + lb1;
                C r{0, 0};
#pragma unroll
                for (int b = 0; b < KB_J; ++b) {
                    const C g = row[b];
                    r.x += w1[b] * g.x;
                    r.y += w1[b] * g.y;
                }
                q.x += w0[a] * r.x;
                q.y += w0[a] * r.y;
            }
            const C phix{cur.th * q.x, cur.th * q.y};
            if (MODE == DG_OP) {
                A.op_out[A.perm ? A.perm[gi] : gi] = phix;
            } else {
                if (act) {
                    const R invU = R(1) / cur.rc.U;
                    const C zz{cur.v.x * invU + phix.x, cur.v.y * invU + phix.y};
                    A.z[gi] = zz;
                    C ww;
                    if (first_blk) {
                        ww = zz;
                        if (keep_start) A.p[gi] = zz;
                    } else {
                        const R mu_u = (R)mu * cur.rc.U;
                        ww = C{cur.p.x - mu_u * (cur.p.x - zz.x), cur.p.y - mu_u * (cur.p.y - zz.y)};
                    }
                    A.w[gi] = ww;
                    const R dx = ww.x - cur.y.x, dy = ww.y - cur.y.y;
                    s_w.add(dx * dx + dy * dy);
                }
                const R ex = phix.x - cur.y.x, ey = phix.y - cur.y.y;
                s_r.add(ex * ex + ey * ey);
            }
            if (i + NTD < count) cur = nx;
        }
        // this thread's first visibility of the next unit (loaded during the
        // unit's reduction and barrier below)
        if (nxt < n_units && (int)threadIdx.x < A.u_count[nxt]) load_vis<R, MODE>(A, A.u_start[nxt] + threadIdx.x, cur);
        if (MODE != DG_OP) cta_sum2<NTD>(s_w.get(), s_r.get(), A.partials + NPART * (int64_t)A.u_pos[u]);
        // the position after the next unit (read after the barrier below;
        // rewritten only after the next unit's first barrier)
        if (threadIdx.x == 0) claim(nxt_pos);
        __syncthreads();   // the tile buffer is refilled two units later
    }
    // no claim follows this CTA's exit: the last CTA out resets the counters
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(A.claim + 1, 1) == (int)gridDim.x - 1) {
            A.claim[0] = 0;
            A.claim[1] = 0;
        }
    }
}

// ----------------------------------------------------------------- sub-iteration
// Algorithm 2 step with the block scale c of the previous step:
//   p = P_B(w) = y + c (w - y);  w = q - mu U (q - z);  partial ||w - y||^2
// with q = p (Algorithm 2) or, for the accelerated form, the extrapolated
// point q = p + beta (p - p_prev), p_prev read from and p written to the
// warm-start array (beta = 0: p_prev is not read; write_p = 0: p not written).
// only_first: the extra step that moves the start of a block with no prox
// output yet from z to P_B(z) (randomised active sets); chunks of other
// blocks, and of blocks outside D, pass their partial through unchanged.
// Stopping test (inner_tol > 0): p is kept every step; a step k >= 1 also
// forms the partials ||p - p_prev||^2 and ||p||^2; a block whose test held
// for the previous step (or earlier) stops, its p being the prox output.
template <typename R>
__global__ void __launch_bounds__(DG_NT) k_subiter(VisArgs<R> A, int only_first, R beta, int write_p) {
    using C = cplx_t<R>;
    const int u = blockIdx.x;   // one work unit (at most DG_NT visibilities)
    const int start = A.u_start[u], count = A.u_count[u], blk = A.ch_block[A.u_chunk[u]];
    pdl_enter();
    const bool act = !A.bmask || A.bmask[blk];
    const bool first_blk = A.seen && !A.seen[blk];
    if (!act || (only_first && !first_blk)) {
        if (threadIdx.x == 0) {
            const int64_t slot = NPART * (int64_t)A.u_pos[u];
            A.partials[slot] = A.part_in[slot];
        }
        return;
    }
    const bool tol_on = A.inner_tol > 0;
    if (inner_stopped(A, blk)) return;   // stopped at an earlier step of this iteration
    bool stop = false;
    const R c = (R)block_scale(A, blk, tol_on && A.test_in, &stop);
    if (stop) {   // the previous step's output is the prox
        if (threadIdx.x == 0) A.inner_state[blk] = A.step - 1;
        return;
    }
    const R mu = (R)A.mu[blk];
    const bool test_out = tol_on && A.step > 0;
    const bool keep = write_p || tol_on;
    Acc<R> s_w, s_d, s_n;
    for (int i = threadIdx.x; i < count; i += DG_NT) {
        const int gi = start + i;
        const R U = A.rec[gi].U;
        const C yy = A.y[gi], ww = A.w[gi], zz = A.z[gi];
        const C pp{yy.x + c * (ww.x - yy.x), yy.y + c * (ww.y - yy.y)};
        C q = pp;
        if (beta != R(0) || test_out) {
            const C pm = A.p[gi];
            if (beta != R(0)) q = C{pp.x + beta * (pp.x - pm.x), pp.y + beta * (pp.y - pm.y)};
            if (test_out) {
                const R ex = pp.x - pm.x, ey = pp.y - pm.y;
                s_d.add(ex * ex + ey * ey);
                s_n.add(pp.x * pp.x + pp.y * pp.y);
            }
        }
        if (keep) A.p[gi] = pp;
        const R mu_u = mu * U;
        const C wn{q.x - mu_u * (q.x - zz.x), q.y - mu_u * (q.y - zz.y)};
        A.w[gi] = wn;
        const R dx = wn.x - yy.x, dy = wn.y - yy.y;
        s_w.add(dx * dx + dy * dy);
    }
    __shared__ double o3[3];
    cta_sum3<DG_NT>(s_w.get(), s_d.get(), s_n.get(), o3);
    if (threadIdx.x == 0) {
        double *out = A.partials + NPART * (int64_t)A.u_pos[u];
        out[0] = o3[0];
        out[2] = o3[1];
        out[3] = o3[2];
    }
}

// ----------------------------------------------------------------- block norms
// One warp per block j: n2 = sum of the block's chunk partials (fixed order),
// scale_j = eps_j / ||w_j - y_j|| if that norm exceeds eps_j, else 1 (the
// l2-ball projection P_B of Section 3.3 as a radial scale).
__global__ void k_block_norms(const double *__restrict__ partials, const int32_t *__restrict__ blk_ptr,
                              const double *__restrict__ eps, int d,
                              int with_resid, double *__restrict__ scale, double *__restrict__ resid2,
                              int *__restrict__ err) {
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= d) return;
    double a = 0, b = 0;
    for (int k = blk_ptr[j] + lane; k < blk_ptr[j + 1]; k += 32) {
        a += partials[NPART * (int64_t)k];
        if (with_resid) b += partials[NPART * (int64_t)k + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        const double n = sqrt(a);
        if (!isfinite(n)) atomicOr(err, ERR_NONFINITE);
        scale[j] = (n > eps[j]) ? eps[j] / n : 1.0;
        if (with_resid) resid2[j] = b;
    }
}

// ----------------------------------------------------------------- gridding
// Per warp, in rounds of 32 visibilities of its slice of the chunk: phase 1
// (lane per visibility) forms Theta v, the 8 products w0[a] Theta v and the 8
// weights w1[b] into the warp's staging area; phase 2 (the warp per
// visibility) adds the 8 x 8 footprint w1[b] (w0[a] Theta v) into the warp's
// private (T+8)^2 tile.  Finally the CTA sums the private tiles in warp order
// and writes the chunk's partial tile.  GR_DUAL fuses the
// end of the data step: p = P_B(w) = y + c (w - y), v = U (z - p).
// Lane l of the scattering warp owns footprint column l mod 8 of rows l/8
// and l/8 + 4; with the private-tile pitch T + 8 = 8 mod 16 (in 8-byte
// words) the two rows a half-warp touches fall in disjoint bank halves, so
// the read-modify-write of the tile is free of bank conflicts.
constexpr int GRID_MINV = 16;   // least visibilities per scattering warp
// NW warps per CTA (4 or 8; FP64: 4): eight split a chunk finer, four
// leave room for more CTAs per SM (the autotuner picks per problem).
template <typename R, int T, int MODE, int NW>
__global__ void __launch_bounds__(NW * 32) k_grid(VisArgs<R> A, cplx_t<R> *__restrict__ gpart) {
    using C = cplx_t<R>;
    constexpr int NT = NW * 32;
    constexpr int E = T + HALO, P = E;   // P: pitch of the private tiles (8 mod 16 words)
    static_assert(P % 16 == 8, "private-tile pitch");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // per-warp staging of 32 visibilities, component-major with a pitch of
    // 33 so that the stores of a warp's lanes and their reads of one
    // visibility both hit distinct banks
    constexpr int SP = 33, SW = 2 * 4 * SP;   // complex words per warp: 4 x SP pairs
    C *priv = reinterpret_cast<C *>(smem_raw);                          // NW * E * P
    C *sa_all = priv + NW * E * P;                                      // NW x 4 x SP pairs (w0[a] Theta v, w0[a+4] Theta v)
    R *sb_all = reinterpret_cast<R *>(sa_all + NW * SW);                // NW x 8 x SP: w1[b]

    // largest chunks first, so that the last wave holds the small ones
    const int ch = A.ch_order[blockIdx.x];
    const int start = A.ch_start[ch], count = A.ch_count[ch], tl = A.ch_tile[ch];
    const int row0 = (tl / A.ntile1) * T, col0 = (tl % A.ntile1) * T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int blk = A.ch_block[ch];
    // warps that scatter: at least GRID_MINV visibilities each, so that a
    // small chunk clears and sums only as many private tiles as it fills
    const int nwu = min(NW, max(1, (count + GRID_MINV - 1) / GRID_MINV));
    for (int e = threadIdx.x; e < nwu * E * P; e += NT) priv[e] = C{0, 0};
    pdl_enter();
    // a block outside the active set D keeps v_j, so its chunks' partial
    // tiles from the last gridding still hold G^dagger Theta^dagger v_j
    const bool act = MODE != GR_DUAL || !A.bmask || A.bmask[blk];
    if (!act && !(A.regrid && *A.regrid)) return;
    R c = 0;
    // Algorithm 2 stopped early (stopping test): the prox output is the p
    // the stopping step kept, not P_B of the current w
    bool done = false;
    if (MODE == GR_DUAL && act) {
        const bool tol_on = A.inner_tol > 0 && A.n_itr > 1;
        int steps = A.n_itr;
        const int stopped = tol_on ? inner_stopped(A, blk) : 0;
        if (stopped) {
            done = true;
            steps = stopped;
        } else {
            bool stop = false;
            c = (R)block_scale(A, blk, tol_on && A.test_in, &stop);
            if (stop) {
                done = true;
                steps = A.n_itr - 1;
            }
        }
        if (threadIdx.x == 0 && A.inner_steps) A.inner_steps[blk] = steps;
    }
    if (MODE == GR_DUAL && act && A.seen && threadIdx.x == 0) A.seen[blk] = 1;
    __syncthreads();

    C *mine = priv + warp * E * P;
    const int bcol = lane & 7, a0 = lane >> 3;   // rows a0 and a0 + 4
    // a lane's visibility of the current round, loaded one round ahead so
    // that the loads of round r + 1 are in flight during the scatter of r
    struct In {
        VisRec<R> rc;
        C a, b, z;   // GR_DUAL active: y, w, z (stopped early: p, -, z); inactive: v; operator modes: input
        R th;
    };
    auto load_in = [&](int gi, In &o) {
        o.rc = A.rec[gi];
        if (MODE == GR_DUAL && act) {
            if (done) {
                o.a = A.p[gi];
            } else {
                o.a = A.y[gi];
                o.b = A.w[gi];
            }
            o.z = A.z[gi];
        } else if (MODE == GR_DUAL) {
            o.a = A.v[gi];
        } else {
            o.a = A.op_in[A.perm ? A.perm[gi] : gi];
        }
        o.th = A.theta_v ? A.theta_v[gi] : A.theta_s;
    };
    // warp w owns a contiguous slice of the chunk (the sort order makes runs
    // of visibilities share a first tap) and works through it in rounds of
    // 32: each lane stages one visibility (dual update, Theta v, weights) in
    // the warp's staging area, then the warp adds the 32 footprints one after
    // the other, each lane accumulating its two cells in registers and
    // writing the private tile only when the base cell changes.  Warps never
    // wait for one another inside the loop.
    C *sa = sa_all + warp * SW;
    R *sb = sb_all + warp * KB_J * SP;
    const int seg = (count + nwu - 1) / nwu;
    const int v0 = warp < nwu ? min(count, warp * seg) : count, v1 = min(count, v0 + seg);
    In cur;
    if (v0 + lane < v1) load_in(start + v0 + lane, cur);
    int run = -1;   // base cell (packed local row | col << 16) of the run being accumulated
    C acc0{0, 0}, acc1{0, 0};
    auto fetch = [&](int i, C &pa, C &pb, R &wb) {   // w0[a0] Theta v, w0[a0+4] Theta v, w1[bcol]
        if constexpr (sizeof(R) == 4) {
            const float4 q = *reinterpret_cast<const float4 *>(sa + 2 * (a0 * SP + i));
            pa = C{q.x, q.y};
            pb = C{q.z, q.w};
        } else {
            pa = sa[2 * (a0 * SP + i)];
            pb = sa[2 * (a0 * SP + i) + 1];
        }
        wb = sb[bcol * SP + i];
    };
    auto accumulate = [&](const C &pa, const C &pb, R wb) {
        acc0.x += wb * pa.x;
        acc0.y += wb * pa.y;
        acc1.x += wb * pb.x;
        acc1.y += wb * pb.y;
    };
    auto flush = [&]() {   // add the run's two cells of this lane into the private tile
        C *cell = mine + ((run & 0xffff) + a0) * P + (run >> 16) + bcol;
        const C g0 = cell[0], g1 = cell[4 * P];
        cell[0] = cadd(g0, acc0);
        cell[4 * P] = cadd(g1, acc1);
    };
    for (int base = v0; base < v1; base += 32) {
        const int n = min(32, v1 - base);
        int mylb = -1;
        if (lane < n) {
            const int gi = start + base + lane;
            const VisRec<R> rc = cur.rc;
            C vv;
            if (MODE == GR_DUAL && act) {
                const C zz = cur.z;
                C pp;
                if (done) {
                    pp = cur.a;
                } else {
                    const C yy = cur.a, ww = cur.b;
                    pp = C{yy.x + c * (ww.x - yy.x), yy.y + c * (ww.y - yy.y)};
                    A.p[gi] = pp;
                }
                vv = C{rc.U * (zz.x - pp.x), rc.U * (zz.y - pp.y)};
                A.v[gi] = vv;
            } else if (MODE == GR_DUAL) {
                vv = cur.a;
            } else {
                vv = cur.a;
                if (MODE == GR_OP_U) vv = C{rc.U * vv.x, rc.U * vv.y};
            }
            const R th = cur.th;
            const C tv{th * vv.x, th * vv.y};
            R w0[KB_J], w1[KB_J];
            kb_weights(rc.f0, w0, A.kbp, A.beta, A.inv_i0b);
            kb_weights(rc.f1, w1, A.kbp, A.beta, A.inv_i0b);
#pragma unroll
            for (int a = 0; a < KB_J / 2; ++a) {   // lane rows (a, a+4) read one pair
                C *da = sa + 2 * (a * SP + lane);
                if constexpr (sizeof(R) == 4) {
                    *reinterpret_cast<float4 *>(da) =
                        make_float4(w0[a] * tv.x, w0[a] * tv.y, w0[a + 4] * tv.x, w0[a + 4] * tv.y);
                } else {
                    da[0] = C{w0[a] * tv.x, w0[a] * tv.y};
                    da[1] = C{w0[a + 4] * tv.x, w0[a + 4] * tv.y};
                }
            }
#pragma unroll
            for (int j = 0; j < KB_J; ++j) sb[j * SP + lane] = w1[j];
            mylb = ((rc.packed & 0xffff) - row0) | ((((rc.packed >> 16) & 0xffff) - col0) << 16);
        }
        // the visibilities of the round that start a new run (the order is
        // sorted by base cell): lane 0 compares with the run carried over
        const int prev = __shfl_up_sync(0xffffffffu, mylb, 1);
        unsigned starts = __ballot_sync(0xffffffffu, lane < n && mylb != (lane == 0 ? run : prev));
        __syncwarp();
        if (base + 32 + lane < v1) load_in(start + base + 32 + lane, cur);   // next round, in flight during the scatter
        // the warp walks the round run by run (uniform control flow): at a
        // run start the finished run is added to the tile, inside a run the
        // footprints accumulate in registers, four at a time
        int i = 0;
        while (i < n) {
            const int e = starts ? __ffs(starts) - 1 : n;
            if (e == i) {
                if (run >= 0) flush();
                run = __shfl_sync(0xffffffffu, mylb, i);
                acc0 = C{0, 0};
                acc1 = C{0, 0};
                starts &= starts - 1;
                continue;
            }
            for (; i + 4 <= e; i += 4) {
                C pa[4], pb[4];
                R wb[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) fetch(i + q, pa[q], pb[q], wb[q]);
#pragma unroll
                for (int q = 0; q < 4; ++q) accumulate(pa[q], pb[q], wb[q]);
            }
            for (; i < e; ++i) {
                C pa, pb;
                R wb;
                fetch(i, pa, pb, wb);
                accumulate(pa, pb, wb);
            }
        }
        __syncwarp();   // the staging is rewritten by the next round
    }
    if (run >= 0) flush();
    __syncthreads();
    C *out = gpart + (int64_t)ch * E * E;
    for (int e = threadIdx.x; e < E * E; e += NT) {
        const int r = e / E, cc = e % E;
        C s{0, 0};
        for (int k = 0; k < nwu; ++k) s = cadd(s, priv[k * E * P + r * P + cc]);
        out[e] = s;
    }
}

// ----------------------------------------------------------------- combine
// One CTA per active tile (a tile with chunks, or below/right of one):
// grid[r][c] = sum of the partial tiles covering the cell, in a fixed order:
// the cell's own tile's chunks, then the halo rows/columns of the tiles
// above, left and above-left (periodic grid).  The grid is column-major
// (element (r, c) at c K0 + r, the layout the inverse column pass reads):
// the T x T sums, formed from row-major partial-tile reads, are transposed
// in shared memory and written as whole column segments.  Tiles never
// touched by any visibility stay zero from the initial clear.
template <typename R, int T>
__global__ void __launch_bounds__(256) k_combine(const cplx_t<R> *__restrict__ gpart,
                                                 const int32_t *__restrict__ tile_first,
                                                 const int32_t *__restrict__ tile_n,
                                                 const int32_t *__restrict__ active, int K0, int nt0, int nt1,
                                                 cplx_t<R> *__restrict__ grid) {
    using C = cplx_t<R>;
    constexpr int E = T + HALO;
    __shared__ int f_s[4], n_s[4];
    __shared__ C tr[T][T + 1];
    const int t = active[blockIdx.x];
    const int t0 = t / nt1, t1 = t - t0 * nt1;
    if (threadIdx.x < 4) {
        const int up = (t0 + nt0 - 1) % nt0, left = (t1 + nt1 - 1) % nt1;
        const int tt = threadIdx.x == 0 ? t : threadIdx.x == 1 ? up * nt1 + t1
                       : threadIdx.x == 2 ? t0 * nt1 + left : up * nt1 + left;
        f_s[threadIdx.x] = tile_first[tt];
        n_s[threadIdx.x] = tile_n[tt];
    }
    __syncthreads();
    pdl_enter();
    for (int e = threadIdx.x; e < T * T; e += 256) {
        const int lr = e / T, lc = e % T;
        C acc{0, 0};
#pragma unroll 4
        for (int k = 0; k < n_s[0]; ++k) acc = cadd(acc, gpart[(int64_t)(f_s[0] + k) * E * E + lr * E + lc]);
        if (lr < HALO)
            for (int k = 0; k < n_s[1]; ++k)
                acc = cadd(acc, gpart[(int64_t)(f_s[1] + k) * E * E + (lr + T) * E + lc]);
        if (lc < HALO)
            for (int k = 0; k < n_s[2]; ++k)
                acc = cadd(acc, gpart[(int64_t)(f_s[2] + k) * E * E + lr * E + lc + T]);
        if (lr < HALO && lc < HALO)
            for (int k = 0; k < n_s[3]; ++k)
                acc = cadd(acc, gpart[(int64_t)(f_s[3] + k) * E * E + (lr + T) * E + lc + T]);
        tr[lc][lr] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < T * T; e += 256) {
        const int lc = e / T, lr = e % T;
        grid[(int64_t)(t1 * T + lc) * K0 + t0 * T + lr] = tr[lc][lr];
    }
}

template <typename R> VisArgs<R> make_args(ppd_ctx *c) {
    VisArgs<R> A{};
    A.rec = static_cast<const VisRec<R> *>(c->rec);
    A.theta_v = static_cast<const R *>(c->theta_v);
    A.theta_s = (R)c->theta_scalar;
    A.ch_start = c->ch.start;
    A.ch_count = c->ch.count;
    A.ch_tile = c->ch.tile;
    A.ch_block = c->ch.block;
    A.ch_order = c->ch.order;
    A.K0 = c->K0;
    A.K1 = c->K1;
    A.ntile1 = c->K1 / c->T;
    for (int i = 0; i < KB_NC; ++i) A.kbp[i] = c->kbpoly_h.empty() ? 0.f : c->kbpoly_h[i];
    A.beta = c->beta;
    A.inv_i0b = 1.0 / std::cyl_bessel_i(0.0, c->beta);
    A.y = static_cast<const cplx_t<R> *>(c->y);
    A.v = static_cast<cplx_t<R> *>(c->v);
    A.z = static_cast<cplx_t<R> *>(c->z);
    A.w = static_cast<cplx_t<R> *>(c->w);
    A.p = static_cast<cplx_t<R> *>(c->p);
    A.mu = c->mu_d;
    A.scale = c->scale;
    A.partials = c->part_out;
    A.part_in = c->part_in;
    A.blk_ptr = c->ch.blk_ptr;
    A.u_pos = c->ch.u_pos;
    A.u_start = c->ch.u_start;
    A.u_count = c->ch.u_count;
    A.u_chunk = c->ch.u_chunk;
    A.u_order = c->ch.u_order;
    A.claim = c->dg_claim;
    A.eps = c->eps_d;
    A.err = c->err;
    A.bmask = c->rand_on ? c->mask_cur : nullptr;
    A.seen = c->rand_on ? c->blk_seen : nullptr;
    A.regrid = c->rand_on ? c->regrid_d : nullptr;
    A.inner_tol = c->cfg.inner_tol;
    A.step = c->next_step;
    A.test_in = c->next_test_in;
    A.n_itr = c->cfg.n_itr;
    A.inner_state = c->inner_state;
    A.inner_steps = c->inner_steps;
    return A;
}

template <typename R, int T, int NW> size_t grid_smem() {
    constexpr int E = T + HALO, P = E, SP = 33;
    return (size_t)NW * E * P * sizeof(cplx_t<R>) + (size_t)NW * 8 * SP * sizeof(cplx_t<R>) +
           (size_t)NW * KB_J * SP * sizeof(R);
}

template <typename R, int T, int NTD>
int degrid_t(ppd_ctx *c, int mode, const cplx_t<R> *grid, cplx_t<R> *out, const int64_t *perm, cudaStream_t s) {
    VisArgs<R> A = make_args<R>(c);
    A.op_out = out;
    A.perm = perm;
    constexpr int E = T + HALO;
    const size_t tile_stride = ((size_t)E * E * sizeof(cplx_t<R>) + 127) / 128 * 128;
    const size_t sh = 2 * tile_stride;
    PPD_CHECK(smem_attr((const void *)k_degrid<R, T, DG_OP, NTD>, (int)sh));
    PPD_CHECK(smem_attr((const void *)k_degrid<R, T, DG_DUAL, NTD>, (int)sh));
    PPD_CHECK(smem_attr((const void *)k_degrid<R, T, DG_FIRST, NTD>, (int)sh));
    const int use_tma = (c->tma_ok && grid == c->grid_a) ? 1 : 0;
    if (c->ch.nu == 0) return PPD_OK;
    int per_sm = 0;
    PPD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_degrid<R, T, DG_DUAL, NTD>, NTD, sh));
    if (per_sm < 1) per_sm = 1;
    int sms = 0;
    PPD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int nch = (int)c->ch.nu;   // work units
    const unsigned nb = (unsigned)std::min<int64_t>(nch, (int64_t)sms * per_sm);
    int site;
    PPD_CHECK(launch_begin(c, mode == DG_OP ? "degrid_op" : "degrid_dual", s, &site));
    const long long sf = c->wait_first;
    auto k = mode == DG_OP     ? k_degrid<R, T, DG_OP, NTD>
             : mode == DG_DUAL ? k_degrid<R, T, DG_DUAL, NTD>
                               : k_degrid<R, T, DG_FIRST, NTD>;
    launch(c, true, k, nb, NTD, sh, s, c->tmap_a, use_tma, grid, A, nch, sf);
    return launch_end(c, site, s);
}

template <typename R, int T, int NW> int grid_launch(ppd_ctx *c, int mode, const VisArgs<R> &A, cudaStream_t s) {
    const size_t sh = grid_smem<R, T, NW>();
    PPD_CHECK(smem_attr((const void *)k_grid<R, T, GR_OP, NW>, (int)sh));
    PPD_CHECK(smem_attr((const void *)k_grid<R, T, GR_OP_U, NW>, (int)sh));
    PPD_CHECK(smem_attr((const void *)k_grid<R, T, GR_DUAL, NW>, (int)sh));
    int site;
    PPD_CHECK(launch_begin(c, mode == GR_DUAL ? "grid_dual" : "grid_op", s, &site));
    auto k = mode == GR_OP     ? k_grid<R, T, GR_OP, NW>
             : mode == GR_OP_U ? k_grid<R, T, GR_OP_U, NW>
                               : k_grid<R, T, GR_DUAL, NW>;
    launch(c, true, k, (unsigned)c->ch.n, NW * 32, sh, s, A, static_cast<cplx_t<R> *>(c->gpart));
    return launch_end(c, site, s);
}

template <typename R, int T>
int grid_t(ppd_ctx *c, int mode, const cplx_t<R> *in, const int64_t *perm, cplx_t<R> *grid, cudaStream_t s,
           bool combine) {
    VisArgs<R> A = make_args<R>(c);
    A.op_in = in;
    A.perm = perm;
    cplx_t<R> *gp = static_cast<cplx_t<R> *>(c->gpart);
    int site;
    if (c->ch.n > 0) {
        if constexpr (sizeof(R) == 4) {
            PPD_CHECK((c->grid_nw == 4 ? grid_launch<R, T, 4>(c, mode, A, s) : grid_launch<R, T, 8>(c, mode, A, s)));
        } else {
            PPD_CHECK((grid_launch<R, T, 4>(c, mode, A, s)));
        }
    }
    if (c->ch.n_active == 0 || !combine) return PPD_OK;
    PPD_CHECK(launch_begin(c, "grid_combine", s, &site));
    launch(c, true, k_combine<R, T>, (unsigned)c->ch.n_active, 256, 0, s, (const cplx_t<R> *)gp,
           (const int32_t *)c->ch.tile_first, (const int32_t *)c->ch.tile_n, (const int32_t *)c->ch.active, c->K0,
           c->K0 / T, c->K1 / T, grid);
    return launch_end(c, site, s);
}

}  // namespace

// Binning entry used by the API: fills key, base (2 per vis), frac (2 per
// vis), per-visibility cell count.
int bin_all(ppd_ctx *c, const double *uv_d, const int32_t *blk_d, int64_t M, uint64_t *key_d, int32_t *base_d,
            double *frac_d, int32_t *count_d, int *bad_d) {
    int32_t *cell_d = nullptr, *cgrid = nullptr;
    PPD_CUDA(cudaMalloc(&cell_d, M * sizeof(int32_t)));
    PPD_CUDA(cudaMalloc(&cgrid, (size_t)c->K0 * c->K1 * sizeof(int32_t)));
    PPD_CUDA(cudaMemsetAsync(cgrid, 0, (size_t)c->K0 * c->K1 * sizeof(int32_t), c->stream));
    const int nb = (int)std::min<int64_t>((M + 255) / 256, 152 * 32);
    k_bin<<<nb, 256, 0, c->stream>>>(uv_d, blk_d, M, c->K0, c->K1, c->T, c->d, key_d, base_d, frac_d, cell_d, cgrid,
                                     bad_d);
    k_cell_count<<<nb, 256, 0, c->stream>>>(cell_d, cgrid, M, count_d);
    c->launches += 2;
    PPD_CUDA(cudaGetLastError());
    PPD_CUDA(cudaStreamSynchronize(c->stream));
    PPD_CUDA(cudaFree(cell_d));
    PPD_CUDA(cudaFree(cgrid));
    return PPD_OK;
}

// Chebyshev interpolation (degree KB_DEG, in t = 2 frac - 1) of each tap's
// weight psi(frac + 3 - j), converted to monomial coefficients for Horner.
int make_kb_poly(ppd_ctx *c) {
    const int n = KB_DEG + 1;
    const double beta = c->beta, i0b = std::cyl_bessel_i(0.0, beta);
    std::vector<float> out((size_t)n * KB_J);
    for (int j = 0; j < KB_J; ++j) {
        std::vector<double> fk(n), cheb(n, 0.0);
        for (int k = 0; k < n; ++k) {
            const double t = std::cos(M_PI * (k + 0.5) / n);
            const double d = (t + 1.0) * 0.5 + 3.0 - j;
            const double x = 1.0 - (d / 4.0) * (d / 4.0);
            fk[k] = x >= 0 ? std::cyl_bessel_i(0.0, beta * std::sqrt(x)) / i0b : 0.0;
        }
        for (int m = 0; m < n; ++m) {
            double s = 0;
            for (int k = 0; k < n; ++k) s += fk[k] * std::cos(M_PI * m * (k + 0.5) / n);
            cheb[m] = s * (m == 0 ? 1.0 : 2.0) / n;
        }
        // Chebyshev -> monomial: T_0 = 1, T_1 = t, T_{m+1} = 2 t T_m - T_{m-1}
        std::vector<double> mono(n, 0.0), Tm1(n, 0.0), Tm(n, 0.0), Tn(n, 0.0);
        Tm1[0] = 1.0;
        Tm[1] = 1.0;
        for (int k = 0; k < n; ++k) mono[k] += cheb[0] * Tm1[k];
        if (n > 1)
            for (int k = 0; k < n; ++k) mono[k] += cheb[1] * Tm[k];
        for (int m = 2; m < n; ++m) {
            for (int k = 0; k < n; ++k) Tn[k] = (k > 0 ? 2.0 * Tm[k - 1] : 0.0) - Tm1[k];
            for (int k = 0; k < n; ++k) mono[k] += cheb[m] * Tn[k];
            Tm1 = Tm;
            Tm = Tn;
        }
        for (int k = 0; k < n; ++k) out[(size_t)k * KB_J + j] = (float)mono[k];
    }
    PPD_CUDA(cudaMemcpy(c->kbpoly, out.data(), out.size() * sizeof(float), cudaMemcpyHostToDevice));
    c->kbpoly_h = out;
    return PPD_OK;
}

template <typename R>
int degrid(ppd_ctx *c, int mode, const cplx_t<R> *grid, cplx_t<R> *out, const int64_t *perm, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        if (c->degrid_nt == 128)
            return c->T == 16 ? degrid_t<R, 16, 128>(c, mode, grid, out, perm, s)
                              : degrid_t<R, 32, 128>(c, mode, grid, out, perm, s);
    }
    return c->T == 16 ? degrid_t<R, 16, 256>(c, mode, grid, out, perm, s)
                      : degrid_t<R, 32, 256>(c, mode, grid, out, perm, s);
}

template <typename R>
int grid_vis(ppd_ctx *c, int mode, const cplx_t<R> *in, const int64_t *perm, cplx_t<R> *grid, cudaStream_t s,
             bool combine) {
    return c->T == 16 ? grid_t<R, 16>(c, mode, in, perm, grid, s, combine)
                      : grid_t<R, 32>(c, mode, in, perm, grid, s, combine);
}

template <typename R> int subiter(ppd_ctx *c, cudaStream_t s, int only_first, double beta, int write_p) {
    if (c->ch.nu == 0) return PPD_OK;
    int site;
    PPD_CHECK(launch_begin(c, "subiter", s, &site));
    launch(c, true, k_subiter<R>, (unsigned)c->ch.nu, DG_NT, 0, s, make_args<R>(c), only_first, (R)beta, write_p);
    return launch_end(c, site, s);
}

int block_norms(ppd_ctx *c, int with_resid, cudaStream_t s) {
    int site;
    PPD_CHECK(launch_begin(c, "block_norms", s, &site));
    const int wpb = 8;
    k_block_norms<<<(c->d + wpb - 1) / wpb, wpb * 32, 0, s>>>(c->part_out, c->ch.blk_ptr, c->eps_d,
                                                               c->d, with_resid, c->scale, c->resid2, c->err);
    return launch_end(c, site, s);
}

// Same launches as grid_vis, with the per-chunk partial tiles written to a
// caller-supplied device buffer instead of the context's.
template <typename R>
int grid_vis_into(ppd_ctx *c, int mode, const cplx_t<R> *in, const int64_t *perm, cplx_t<R> *grid, void *gpart,
                  cudaStream_t s) {
    void *own = c->gpart;
    c->gpart = gpart;
    const int st = grid_vis<R>(c, mode, in, perm, grid, s);
    c->gpart = own;
    return st;
}

template int grid_vis_into<float>(ppd_ctx *, int, const float2 *, const int64_t *, float2 *, void *, cudaStream_t);
template int grid_vis_into<double>(ppd_ctx *, int, const double2 *, const int64_t *, double2 *, void *,
                                   cudaStream_t);
template int degrid<float>(ppd_ctx *, int, const float2 *, float2 *, const int64_t *, cudaStream_t);
template int degrid<double>(ppd_ctx *, int, const double2 *, double2 *, const int64_t *, cudaStream_t);
template int grid_vis<float>(ppd_ctx *, int, const float2 *, const int64_t *, float2 *, cudaStream_t, bool);
template int grid_vis<double>(ppd_ctx *, int, const double2 *, const int64_t *, double2 *, cudaStream_t, bool);
template int subiter<float>(ppd_ctx *, cudaStream_t, int, double, int);
template int subiter<double>(ppd_ctx *, cudaStream_t, int, double, int);

}  // namespace ppd
