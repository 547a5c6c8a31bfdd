// btrt_kernels.cu -- instantiations and launchers of the fused sweep.
#include <algorithm>

#include "btrt_internal.h"
#include "btrt_tma.cuh"
#include "../../include/btrt.h"

namespace btrt {

// 32 x 8 threads; each thread sweeps RowsPerThread<Real> nodes of its column.
static inline dim3 sweep_block() { return dim3(32, 8, 1); }
static inline dim3 sweep_grid(int nx, int ny, int rows_per_thread) {
    const int rows = 8 * rows_per_thread;
    return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + rows - 1) / rows), 1);
}

long long sweep_blocks(int nx, int ny, int compute, int storage) {
    const int r = compute == BTRT_F64    ? RowsPerThread<double, double>::value
                  : compute == BTRT_DF64 ? RowsPerThread<dw, dw>::value
                  : storage == BTRT_F32  ? RowsPerThread<float, float>::value
                                         : RowsPerThread<float, __half>::value;
    const dim3 g = sweep_grid(nx, ny, r);
    return (long long)g.x * g.y;
}

// Dispatch on the source kind so that each compiled sweep carries only its own
// source arithmetic.
template <typename Real, typename S, int MODE>
static void launch_src(const SweepParams<Real> &p, dim3 g, dim3 b, cudaStream_t s) {
    switch (p.src_kind) {
    case 0: sweep_kernel<Real, S, MODE, 0><<<g, b, 0, s>>>(p); break;
    case 1: sweep_kernel<Real, S, MODE, 1><<<g, b, 0, s>>>(p); break;
    case 2: sweep_kernel<Real, S, MODE, 2><<<g, b, 0, s>>>(p); break;
    default: sweep_kernel<Real, S, MODE, 3><<<g, b, 0, s>>>(p); break;
    }
}

template <typename Real>
static cudaError_t launch_mode3(const SweepParams<Real> &p, int mode, cudaStream_t s) {
    const dim3 g = sweep_grid(p.nx, p.ny, RowsPerThread<Real, Real>::value), b = sweep_block();
    switch (mode) {
    case kGeneral: launch_src<Real, Real, kGeneral>(p, g, b, s); break;
    case kLinear: launch_src<Real, Real, kLinear>(p, g, b, s); break;
    case kLinearK0One: launch_src<Real, Real, kLinearK0One>(p, g, b, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep_f64(const SweepParams<double> &p, int mode, cudaStream_t s) {
    return launch_mode3<double>(p, mode, s);
}

cudaError_t launch_sweep_dw(const SweepParams<dw> &p, int mode, cudaStream_t s) {
    return launch_mode3<dw>(p, mode, s);
}

template <typename S>
static void launch_f32_mode(const SweepParams<float> &p, int mode, cudaStream_t s) {
    const dim3 g = sweep_grid(p.nx, p.ny, RowsPerThread<float, S>::value), b = sweep_block();
    if (mode == kGeneral) launch_src<float, S, kGeneral>(p, g, b, s);
    else launch_src<float, S, kLinear>(p, g, b, s);
}

cudaError_t launch_sweep_f32(const SweepParams<float> &p, int storage, int mode, cudaStream_t s) {
    switch (storage) {
    case BTRT_F32: launch_f32_mode<float>(p, mode, s); break;
    case BTRT_F16: launch_f32_mode<__half>(p, mode, s); break;
    case BTRT_BF16: launch_f32_mode<__nv_bfloat16>(p, mode, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- TMA-staged sweep
template <typename S, int MODE, int SRC>
static cudaError_t launch_tma_src(const SweepParams<float> &p, const CUtensorMap *in_map,
                                  const CUtensorMap *out_map, cudaStream_t s) {
    using G = TmaGeom<S>;
    static bool configured = false;   // one attribute call per instantiation
    static int per_sm = 0, sms = 0;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(sweep_tma_kernel<S, MODE, SRC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_tma_kernel<S, MODE, SRC>, G::THREADS,
                                                              G::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        configured = true;
    }
    const int ntx = (p.nx + G::TX - 1) / G::TX;
    const int nty = (p.ny + G::TY - 1) / G::TY;
    const int ntiles = ntx * nty;
    const int grid = std::min(ntiles, per_sm * sms);
    sweep_tma_kernel<S, MODE, SRC><<<grid, G::THREADS, G::SMEM, s>>>(p, *in_map, *out_map, ntx, ntiles, 1u << 22);
    return cudaGetLastError();
}

template <typename S, int MODE>
static cudaError_t launch_tma_typed(const SweepParams<float> &p, const CUtensorMap *in_map,
                                    const CUtensorMap *out_map, cudaStream_t s) {
    switch (p.src_kind) {
    case 0: return launch_tma_src<S, MODE, 0>(p, in_map, out_map, s);
    case 1: return launch_tma_src<S, MODE, 1>(p, in_map, out_map, s);
    case 2: return launch_tma_src<S, MODE, 2>(p, in_map, out_map, s);
    default: return launch_tma_src<S, MODE, 3>(p, in_map, out_map, s);
    }
}

cudaError_t launch_sweep_tma(const SweepParams<float> &p, int storage, int mode, const CUtensorMap *in_map,
                             const CUtensorMap *out_map, cudaStream_t s) {
    const bool lin = mode != kGeneral;
    switch (storage) {
    case BTRT_F32: return lin ? launch_tma_typed<float, kLinear>(p, in_map, out_map, s)
                              : launch_tma_typed<float, kGeneral>(p, in_map, out_map, s);
    case BTRT_F16: return lin ? launch_tma_typed<__half, kLinear>(p, in_map, out_map, s)
                              : launch_tma_typed<__half, kGeneral>(p, in_map, out_map, s);
    case BTRT_BF16: return lin ? launch_tma_typed<__nv_bfloat16, kLinear>(p, in_map, out_map, s)
                               : launch_tma_typed<__nv_bfloat16, kGeneral>(p, in_map, out_map, s);
    }
    return cudaErrorInvalidValue;
}

void tma_box(int storage, int *box_in_x, int *box_in_y, int *box_out_x, int *box_out_y) {
    if (storage == BTRT_F32) {
        *box_in_x = TmaGeom<float>::BX; *box_in_y = TmaGeom<float>::BY;
        *box_out_x = TmaGeom<float>::TX; *box_out_y = TmaGeom<float>::TY;
    } else {
        *box_in_x = TmaGeom<__half>::BX; *box_in_y = TmaGeom<__half>::BY;
        *box_out_x = TmaGeom<__half>::TX; *box_out_y = TmaGeom<__half>::TY;
    }
}

}  // namespace btrt
