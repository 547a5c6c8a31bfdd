// btrt_kernels.cu -- instantiations and launchers of the fused sweep.
#include "btrt_internal.h"
#include "../../include/btrt.h"

namespace btrt {

// 32 x 8 threads; each thread sweeps RowsPerThread<Real> nodes of its column.
static inline dim3 sweep_block() { return dim3(32, 8, 1); }
static inline dim3 sweep_grid(int nx, int ny, int rows_per_thread) {
    const int rows = 8 * rows_per_thread;
    return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + rows - 1) / rows), 1);
}

long long sweep_blocks(int nx, int ny, int compute) {
    const dim3 g = sweep_grid(nx, ny, compute == BTRT_F64 ? RowsPerThread<double>::value
                                                          : RowsPerThread<float>::value);
    return (long long)g.x * g.y;
}

cudaError_t launch_sweep_f64(const SweepParams<double> &p, int mode, cudaStream_t s) {
    const dim3 g = sweep_grid(p.nx, p.ny, RowsPerThread<double>::value), b = sweep_block();
    switch (mode) {
    case kGeneral: sweep_kernel<double, double, kGeneral><<<g, b, 0, s>>>(p); break;
    case kLinear: sweep_kernel<double, double, kLinear><<<g, b, 0, s>>>(p); break;
    case kLinearK0One: sweep_kernel<double, double, kLinearK0One><<<g, b, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
static void launch_f32_mode(const SweepParams<float> &p, int mode, dim3 g, dim3 b, cudaStream_t s) {
    if (mode == kGeneral) sweep_kernel<float, S, kGeneral><<<g, b, 0, s>>>(p);
    else sweep_kernel<float, S, kLinear><<<g, b, 0, s>>>(p);
}

cudaError_t launch_sweep_f32(const SweepParams<float> &p, int storage, int mode, cudaStream_t s) {
    const dim3 g = sweep_grid(p.nx, p.ny, RowsPerThread<float>::value), b = sweep_block();
    switch (storage) {
    case BTRT_F32: launch_f32_mode<float>(p, mode, g, b, s); break;
    case BTRT_F16: launch_f32_mode<__half>(p, mode, g, b, s); break;
    case BTRT_BF16: launch_f32_mode<__nv_bfloat16>(p, mode, g, b, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace btrt
