// btrt_launch3.cuh -- launch helpers of the D3Q19 sweep, instantiated per
// storage format in btrt3_kern_*.cu.
#pragma once

#include <cuda_runtime.h>

#include "btrt_sweep3.cuh"

namespace btrt {

// 32 x 8 threads per block, one node each; one grid layer per z.
inline dim3 sweep3_block() { return dim3(32, 8, 1); }
inline dim3 sweep3_grid(int nx, int ny, int nz) {
    return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8), (unsigned)nz);
}

template <typename Real, typename S, int SH, int MODE>
inline void launch3_src(const Sweep3Params<Real> &p, cudaStream_t s) {
    const dim3 g = sweep3_grid(p.nx, p.ny, p.nz), b = sweep3_block();
    switch (p.src_kind) {
    case kSrcNone: sweep3_kernel<Real, S, SH, MODE, kSrcNone><<<g, b, 0, s>>>(p); break;
    case kSrcConst: sweep3_kernel<Real, S, SH, MODE, kSrcConst><<<g, b, 0, s>>>(p); break;
    case kSrcField: sweep3_kernel<Real, S, SH, MODE, kSrcField><<<g, b, 0, s>>>(p); break;
    default: sweep3_kernel<Real, S, SH, MODE, kSrcReaction><<<g, b, 0, s>>>(p); break;
    }
}

template <typename Real, typename S, int SH>
inline cudaError_t launch3_mode(const Sweep3Params<Real> &p, int mode, cudaStream_t s) {
    if (mode == kGeneral) launch3_src<Real, S, SH, kGeneral>(p, s);
    else if (mode == kLinearK0One) launch3_src<Real, S, SH, kLinearK0One>(p, s);
    else launch3_src<Real, S, SH, kLinear>(p, s);
    return cudaGetLastError();
}

template <typename S>
inline cudaError_t launch3_f32_storage(const Sweep3Params<float> &p, int shift, int mode, cudaStream_t s) {
    return shift == kShiftLocal ? launch3_mode<float, S, kShiftLocal>(p, mode, s)
                                : launch3_mode<float, S, kShiftRef>(p, mode, s);
}

// Defined in btrt3_kern_*.cu.
cudaError_t launch_sweep3_f64(const Sweep3Params<double> &p, int mode, cudaStream_t s);
cudaError_t launch_sweep3_f32(const Sweep3Params<float> &p, int storage, int shift, int mode, cudaStream_t s);

}  // namespace btrt
