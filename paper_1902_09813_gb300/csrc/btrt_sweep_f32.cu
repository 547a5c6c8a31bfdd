// btrt_sweep_f32.cu -- compiled variants of the FP32-compute sweep with f32 storage
// (plain and TMA-staged; both storage shifts, both coefficient modes, every source kind).
#include "btrt_launch.cuh"

namespace btrt {

cudaError_t launch_sweep_f32_f32(const SweepParams<float> &p, int shift, int mode, cudaStream_t s) {
    return launch_f32_storage<float>(p, shift, mode, s);
}

cudaError_t launch_sweep_tma_f32(const SweepParams<float> &p, int shift, int mode, const CUtensorMap *in_map,
                                const CUtensorMap *out_map, cudaStream_t s) {
    return launch_tma_storage<float>(p, shift, mode, in_map, out_map, s);
}

cudaError_t launch_sweep_tb2(const SweepParams<float> &pa, const SweepParams<float> &pb, int mode, cudaStream_t s) {
    return launch_tb2_storage<float>(pa, pb, mode, s);
}

}  // namespace btrt
