// btrt_vec_bf16.cu -- compiled variants of the vector-access FP32-compute sweep with
// bf16 storage (both storage shifts, both coefficient modes, every source kind),
// in a translation unit of their own so that they build in parallel.
#include "btrt_launch.cuh"

namespace btrt {

cudaError_t launch_sweep_vec_bf16(const SweepParams<float> &p, int shift, int mode, cudaStream_t s) {
    return launch_vec_storage<__nv_bfloat16>(p, shift, mode, s);
}

}  // namespace btrt
