// Image-side helpers: deterministic FP64 reductions for the statistics and
// the power iteration, and a scaled copy.  (The primal step of Algorithm 3
// runs fused into the finest SARA synthesis, csrc/sara.cu.)
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

}  // namespace

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

template int sumsq<float>(ppd_ctx *, const float *, int64_t, double *, cudaStream_t);
template int sumsq<double>(ppd_ctx *, const double *, int64_t, double *, cudaStream_t);
template int scale_copy<float>(ppd_ctx *, const float *, float *, int64_t, double, cudaStream_t);
template int scale_copy<double>(ppd_ctx *, const double *, double *, int64_t, double, cudaStream_t);

}  // namespace ppd
