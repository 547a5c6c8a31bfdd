// btrt3_kern_f64.cu -- D3Q19 sweep, FP64 compute and storage; dispatch of the FP32 forms.
#include "../../include/btrt.h"
#include "btrt_launch3.cuh"

namespace btrt {

cudaError_t launch_sweep3_f32_f32(const Sweep3Params<float> &, int, int, cudaStream_t);
cudaError_t launch_sweep3_f32_h16(const Sweep3Params<float> &, int, int, int, cudaStream_t);

cudaError_t launch_sweep3_f64(const Sweep3Params<double> &p, int mode, cudaStream_t s) {
    return launch3_mode<double, double, kShiftNone>(p, mode, s);
}

cudaError_t launch_sweep3_f32(const Sweep3Params<float> &p, int storage, int shift, int mode, cudaStream_t s) {
    if (storage == BTRT_F32) return launch_sweep3_f32_f32(p, shift, mode, s);
    if (storage == BTRT_F16 || storage == BTRT_BF16) return launch_sweep3_f32_h16(p, storage, shift, mode, s);
    return cudaErrorInvalidValue;
}

}  // namespace btrt
