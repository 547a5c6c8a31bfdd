// btrt3_kern_h16.cu -- D3Q19 sweep, FP32 compute with FP16 or BF16 storage (both shifts).
#include "../../include/btrt.h"
#include "btrt_launch3.cuh"

namespace btrt {

cudaError_t launch_sweep3_f32_h16(const Sweep3Params<float> &p, int storage, int shift, int mode, cudaStream_t s) {
    return storage == BTRT_F16 ? launch3_f32_storage<__half>(p, shift, mode, s)
                               : launch3_f32_storage<__nv_bfloat16>(p, shift, mode, s);
}

}  // namespace btrt
