// btrt_kernels.cu -- instantiations and launchers of the fused sweep.
#include "btrt_internal.h"
#include "../../include/btrt.h"

namespace btrt {

static inline dim3 sweep_block() { return dim3(32, 8, 1); }
static inline dim3 sweep_grid(int nx, int ny) {
    return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8), 1);
}

cudaError_t launch_sweep_f64(const SweepParams<double> &p, cudaStream_t s) {
    sweep_kernel<double, double><<<sweep_grid(p.nx, p.ny), sweep_block(), 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f32(const SweepParams<float> &p, int storage, cudaStream_t s) {
    const dim3 g = sweep_grid(p.nx, p.ny), b = sweep_block();
    switch (storage) {
    case BTRT_F32: sweep_kernel<float, float><<<g, b, 0, s>>>(p); break;
    case BTRT_F16: sweep_kernel<float, __half><<<g, b, 0, s>>>(p); break;
    case BTRT_BF16: sweep_kernel<float, __nv_bfloat16><<<g, b, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace btrt
