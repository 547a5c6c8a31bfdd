// btrt_noalloc.cu -- FP64 sum of a phi plane that allocates no device memory.
//
// For callers that cannot call cudaMalloc or hand the library a workspace: a
// serving process that reserves its whole device-memory budget at start-up and
// forbids allocations afterwards, or a plug-in running inside a host framework
// that owns the device allocator.  The partial sums live in a fixed array in the
// library's own device memory instead of a caller workspace.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/btrt.h"
#include "btrt_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// 1024 partial sums (the fixed grid of the library's FP64 sum) + the result:
// 8200 bytes, held by every GPU that loads the library until the process exits.
// Shared by all calls on a device.
__device__ __align__(256) double g_sum_scratch[btrt::kRedBlocks + 1];

std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in.
btrt_status scratch_for_current_device(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        btrt::set_last_error("btrt_phi_sum_static: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return BTRT_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        btrt::set_last_error("btrt_phi_sum_static: device ordinal %d >= %d", dev, kMaxDevices);
        return BTRT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_sum_scratch);
        if (e != cudaSuccess || !ptr) {
            btrt::set_last_error("btrt_phi_sum_static: cudaGetSymbolAddress failed: %s",
                                 cudaGetErrorString(e));
            return BTRT_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double *>(ptr);
    }
    *out = g_scratch_addr[dev];
    return BTRT_OK;
}

}  // namespace

extern "C" btrt_status btrt_phi_sum_static(const void *phi_dev, int32_t dtype, int32_t nx, int32_t ny,
                                           int64_t pitch, void *cuda_stream, double *out_host) {
    if (!phi_dev || !out_host) {
        btrt::set_last_error("btrt_phi_sum_static: null argument");
        return BTRT_EINVAL;
    }
    if (dtype != BTRT_F64 && dtype != BTRT_F32) {
        btrt::set_last_error("btrt_phi_sum_static: dtype must be BTRT_F64 or BTRT_F32");
        return BTRT_EINVAL;
    }
    if (nx < 1 || ny < 1 || nx > BTRT_PHI_SUM_STATIC_MAX_SIDE || ny > BTRT_PHI_SUM_STATIC_MAX_SIDE) {
        btrt::set_last_error("btrt_phi_sum_static: plane %d x %d outside [1, %d] per side", nx, ny,
                             BTRT_PHI_SUM_STATIC_MAX_SIDE);
        return BTRT_EINVAL;
    }
    if (pitch < nx) {
        btrt::set_last_error("btrt_phi_sum_static: pitch %lld < nx %d", (long long)pitch, nx);
        return BTRT_EINVAL;
    }
    double *scratch = nullptr;
    btrt_status st = scratch_for_current_device(&scratch);
    if (st != BTRT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // every partial slot is overwritten by its block, so nothing needs clearing; the
    // kernels are btrt_mass's own (btrt_reduce.cuh), so the sums agree bitwise
    cudaError_t e = dtype == BTRT_F64
                        ? btrt::enqueue_rows_sum<double>(static_cast<const double *>(phi_dev), nx, ny, pitch,
                                                         scratch, scratch + btrt::kRedBlocks, s)
                        : btrt::enqueue_rows_sum<float>(static_cast<const float *>(phi_dev), nx, ny, pitch,
                                                        scratch, scratch + btrt::kRedBlocks, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, scratch + btrt::kRedBlocks, sizeof(double),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        btrt::set_last_error("btrt_phi_sum_static: %s", cudaGetErrorString(e));
        return BTRT_ECUDA;
    }
    return BTRT_OK;
}
