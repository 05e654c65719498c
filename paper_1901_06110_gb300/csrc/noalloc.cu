// Allocation-free variant of the super-resolution data-term gradient.
//
// lpnp_gradient keeps its scratch (the low-resolution residual r = A x - y) in
// memory owned by a dsgnlm_t handle, which is allocated with cudaMalloc.  Some
// callers cannot allocate device memory at the point where they need the
// gradient: a plugin whose host framework owns every device allocation and hands
// out only the buffers it passes in, a real-time pipeline that forbids allocation
// after start-up, or code that runs while another component holds the device
// allocator.  lpnp_sr_gradient_noalloc serves them: its scratch is the file-scope
// array below, so a call allocates nothing; the caller passes x, y and grad.
//
// Limits and sharing:
// - r holds at most kMaxLowResPixels FP32 values (4 MiB), i.e. (H/2)(W/2) <=
//   1,048,576 (for example 2048 x 2048); larger images are rejected with
//   DSGNLM_EINVAL before any launch.  Every GPU that loads this library keeps the
//   array until the process exits.
// - All calls on one device share the array.  It keeps the last call's contents;
//   a call writes all of its (H/2)(W/2) entries before reading them, so nothing
//   has to start at zero.  Calls whose work overlaps on the GPU (different
//   streams, or host threads racing) race on the array and give wrong results;
//   serialise them on one stream.
// - The first call on a device resolves the array's device address with
//   cudaGetSymbolAddress (which may load this library's module onto that device).
//   Make that first call before any stream capture begins on the device.  The
//   address is cached for the life of the process, so the call must not be used
//   on a device after cudaDeviceReset or a teardown of its primary context.
// - The blur is always periodic: the result equals lpnp_gradient's only for a
//   problem with blur_boundary == LPNP_BC_PERIODIC.
#include <mutex>

#include "../../include/dsgnlm.h"
#include "internal.h"

namespace {

constexpr size_t kMaxLowResPixels = (size_t)1 << 20;
constexpr int kMaxDevices = 64;

// Scratch for r = A x - y on the low-resolution grid.  In host code this name is a
// host-side stand-in, not a device address: use the address resolved below.
static __device__ __align__(256) float g_sr_residual_scratch[kMaxLowResPixels];

std::mutex g_scratch_mutex;
float* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// Resolve (once per device, with that device current) the array's device address.
cudaError_t scratch_address(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sr_residual_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_scratch_addr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" dsgnlm_status lpnp_sr_gradient_noalloc(const float* x, const float* y, int H, int W,
                                                  float blur_sigma, int blur_r, float* grad,
                                                  void* stream) {
    if (!x || !y || !grad || H < 2 || W < 2 || (H & 1) || (W & 1)) return DSGNLM_EINVAL;
    if (blur_r < 0 || blur_r > 8 || !(blur_sigma > 0.f)) return DSGNLM_EINVAL;
    if ((size_t)(H / 2) * (size_t)(W / 2) > kMaxLowResPixels) return DSGNLM_EINVAL;
    float* r = nullptr;
    cudaError_t e = scratch_address(&r);
    if (e == cudaSuccess) {
        const dsg::BlurTaps taps = dsg::make_blur_taps(blur_sigma, blur_r);
        cudaStream_t st = (cudaStream_t)stream;
        e = dsg::launch_sr_forward(x, H, W, taps, y, -1.0f, r, st);
        if (e == cudaSuccess) e = dsg::launch_sr_adjoint(r, H, W, taps, grad, st);
    }
    if (e != cudaSuccess) {
        dsg::record_cuda_error(e);
        return DSGNLM_ECUDA;
    }
    return DSGNLM_OK;
}
