// btrt3_kern_f32.cu -- D3Q19 sweep, FP32 compute with FP32 storage (both shifts).
#include "btrt_launch3.cuh"

namespace btrt {

cudaError_t launch_sweep3_f32_f32(const Sweep3Params<float> &p, int shift, int mode, cudaStream_t s) {
    return launch3_f32_storage<float>(p, shift, mode, s);
}

}  // namespace btrt
