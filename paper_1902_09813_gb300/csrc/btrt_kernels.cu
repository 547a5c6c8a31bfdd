// btrt_kernels.cu -- FP64 and double-word sweep variants, and the dispatch of
// the FP32-compute variants to their per-storage translation units.
#include "btrt_internal.h"
#include "btrt_tma.cuh"
#include "../../include/btrt.h"

namespace btrt {

cudaError_t launch_sweep_f32_f32(const SweepParams<float> &, int, int, cudaStream_t);
cudaError_t launch_sweep_f32_f16(const SweepParams<float> &, int, int, cudaStream_t);
cudaError_t launch_sweep_f32_bf16(const SweepParams<float> &, int, int, cudaStream_t);
cudaError_t launch_sweep_tma_f32(const SweepParams<float> &, int, int, const CUtensorMap *, const CUtensorMap *,
                                 cudaStream_t);
cudaError_t launch_sweep_tma_f16(const SweepParams<float> &, int, int, const CUtensorMap *, const CUtensorMap *,
                                 cudaStream_t);
cudaError_t launch_sweep_tma_bf16(const SweepParams<float> &, int, int, const CUtensorMap *, const CUtensorMap *,
                                  cudaStream_t);

long long sweep_blocks(int nx, int ny, int compute, int storage) {
    const int r = compute == BTRT_F64    ? RowsPerThread<double, double>::value
                  : compute == BTRT_DF64 ? RowsPerThread<dw, dw>::value
                  : storage == BTRT_F32  ? RowsPerThread<float, float>::value
                                         : RowsPerThread<float, __half>::value;
    const dim3 g = sweep_grid(nx, ny, r);
    return (long long)g.x * g.y;
}

template <typename Real, int MODE>
static void launch_unshifted(const SweepParams<Real> &p, dim3 g, dim3 b, cudaStream_t s) {
    switch (p.src_kind) {
    case 0: sweep_kernel<Real, Real, kShiftNone, MODE, 0><<<g, b, 0, s>>>(p); break;
    case 1: sweep_kernel<Real, Real, kShiftNone, MODE, 1><<<g, b, 0, s>>>(p); break;
    case 2: sweep_kernel<Real, Real, kShiftNone, MODE, 2><<<g, b, 0, s>>>(p); break;
    case 3: sweep_kernel<Real, Real, kShiftNone, MODE, 3><<<g, b, 0, s>>>(p); break;
    default: sweep_kernel<Real, Real, kShiftNone, MODE, kSrcReaction><<<g, b, 0, s>>>(p); break;
    }
}

template <typename Real>
static cudaError_t launch_mode3(const SweepParams<Real> &p, int mode, cudaStream_t s) {
    const dim3 g = sweep_grid(p.nx, p.ny, RowsPerThread<Real, Real>::value), b = sweep_block();
    switch (mode) {
    case kGeneral: launch_unshifted<Real, kGeneral>(p, g, b, s); break;
    case kLinear: launch_unshifted<Real, kLinear>(p, g, b, s); break;
    case kLinearK0One: launch_unshifted<Real, kLinearK0One>(p, g, b, s); break;
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

cudaError_t launch_sweep_f32(const SweepParams<float> &p, int storage, int shift, int mode, cudaStream_t s) {
    switch (storage) {
    case BTRT_F32: return launch_sweep_f32_f32(p, shift, mode, s);
    case BTRT_F16: return launch_sweep_f32_f16(p, shift, mode, s);
    case BTRT_BF16: return launch_sweep_f32_bf16(p, shift, mode, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tb2v(const SweepParams<float> &pa, const SweepParams<float> &pb, int storage, int shift,
                              int mode, cudaStream_t s) {
    switch (storage) {
    case BTRT_F32: return launch_sweep_tb2v_f32(pa, pb, shift, mode, s);
    case BTRT_F16: return launch_sweep_tb2v_f16(pa, pb, shift, mode, s);
    case BTRT_BF16: return launch_sweep_tb2v_bf16(pa, pb, shift, mode, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_vec(const SweepParams<float> &p, int storage, int shift, int mode, cudaStream_t s) {
    switch (storage) {
    case BTRT_F32: return launch_sweep_vec_f32(p, shift, mode, s);
    case BTRT_F16: return launch_sweep_vec_f16(p, shift, mode, s);
    case BTRT_BF16: return launch_sweep_vec_bf16(p, shift, mode, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tma(const SweepParams<float> &p, int storage, int shift, int mode,
                             const CUtensorMap *in_map, const CUtensorMap *out_map, cudaStream_t s) {
    switch (storage) {
    case BTRT_F32: return launch_sweep_tma_f32(p, shift, mode, in_map, out_map, s);
    case BTRT_F16: return launch_sweep_tma_f16(p, shift, mode, in_map, out_map, s);
    case BTRT_BF16: return launch_sweep_tma_bf16(p, shift, mode, in_map, out_map, s);
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
