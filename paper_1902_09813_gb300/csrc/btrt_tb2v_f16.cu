// btrt_tb2v_f16.cu -- compiled variants of the vector two-step FP32-compute sweep
// with f16 storage (both storage shifts, both coefficient modes, every source
// kind), in a translation unit of their own so that they build in parallel.
#include "btrt_launch.cuh"

namespace btrt {

cudaError_t launch_sweep_tb2v_f16(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                  cudaStream_t s) {
    return launch_tb2v_storage<__half>(pa, pb, shift, mode, s);
}

}  // namespace btrt
