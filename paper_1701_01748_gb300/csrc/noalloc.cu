// Phi^dagger without any device allocation during the call.
//
// Some callers cannot let a library call cudaMalloc while they run: an
// application with a fixed device-memory budget that reserves everything at
// start-up, or a real-time loop that must neither block on the allocator nor
// handle an out-of-memory error half-way through.  ppd_op_adjoint_noalloc
// serves them.  It computes the same result as ppd_op_adjoint, but the
// gridding kernel's scratch (one partial (T+8) x (T+8) tile per work item)
// lives in the fixed array below instead of memory the context allocated.
//
// The array is a file-scope __device__ object, so every GPU that loads this
// library holds its PPD_NOALLOC_SCRATCH_BYTES until the process exits.  In
// host code its name is only a host-side stand-in, never a device address:
// the device address is obtained once per device with cudaGetSymbolAddress
// (with that device current) on the first call made on that device.  The
// call runs on the device the context was created on, whichever device the
// caller has current.
// Every call shares the array and it keeps the last call's contents; the
// kernel writes every partial tile it later reads, so nothing needs clearing.
// Calls that overlap on the GPU (other streams, other contexts on the same
// device) race on the array.
#include <mutex>

#include "common.cuh"

namespace ppd {
namespace {

__device__ __align__(256) unsigned char g_grid_scratch[PPD_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_dev[MAX_DEVICES] = {};

// Device address of g_grid_scratch on device `dev`, which must be current
// (set-up on the first call made on that device).
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= MAX_DEVICES) return fail(PPD_ERR_UNSUPPORTED, "ppd_op_adjoint_noalloc: device index");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_grid_scratch);
        if (e != cudaSuccess || !p)
            return fail(PPD_ERR_CUDA, std::string("ppd_op_adjoint_noalloc: cudaGetSymbolAddress: ") +
                                          cudaGetErrorString(e));
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return PPD_OK;
}

}  // namespace
}  // namespace ppd

using namespace ppd;

extern "C" int ppd_op_adjoint_noalloc(ppd_ctx *c, const void *y_dev, void *x_dev, void *stream) {
    if (!c || !y_dev || !x_dev) return fail(PPD_ERR_INVALID_ARG, "ppd_op_adjoint_noalloc: NULL argument");
    if (!c->have_weights) return fail(PPD_ERR_NOT_READY, "ppd_op_adjoint_noalloc: call ppd_set_weights first");
    const size_t E = (size_t)(c->T + HALO);
    const size_t need = (size_t)c->ch.n * E * E * 2 * c->rsz;
    if (need > (size_t)PPD_NOALLOC_SCRATCH_BYTES)
        return fail(PPD_ERR_UNSUPPORTED,
                    "ppd_op_adjoint_noalloc: problem needs " + std::to_string(need) +
                        " bytes of gridding scratch, above the fixed " +
                        std::to_string((size_t)PPD_NOALLOC_SCRATCH_BYTES) + " bytes");
    // the context's device is current for the call, so the scratch address
    // and the kernels below belong to the GPU that holds the context's memory
    DeviceGuard dg_(c->device);
    void *scratch = nullptr;
    PPD_CHECK(scratch_address(c->device, &scratch));
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : c->stream;
    if (c->is_f32) {
        PPD_CHECK(grid_vis_into<float>(c, GR_OP, static_cast<const float2 *>(y_dev), c->perm,
                                       static_cast<float2 *>(c->grid_v), scratch, s));
        return fft_inverse<float>(c, static_cast<const float2 *>(c->grid_v), static_cast<float *>(x_dev), s);
    }
    PPD_CHECK(grid_vis_into<double>(c, GR_OP, static_cast<const double2 *>(y_dev), c->perm,
                                    static_cast<double2 *>(c->grid_v), scratch, s));
    return fft_inverse<double>(c, static_cast<const double2 *>(c->grid_v), static_cast<double *>(x_dev), s);
}
