// btrt_sweep_f16.cu -- compiled variants of the FP32-compute sweep with f16 storage
// (plain, TMA-staged and two-step; both storage shifts, both coefficient modes, every
// source kind).
#include "btrt_launch.cuh"

namespace btrt {

cudaError_t launch_sweep_f32_f16(const SweepParams<float> &p, int shift, int mode, cudaStream_t s) {
    return launch_f32_storage<__half>(p, shift, mode, s);
}

cudaError_t launch_sweep_tma_f16(const SweepParams<float> &p, int shift, int mode, const CUtensorMap *in_map,
                                const CUtensorMap *out_map, cudaStream_t s) {
    return launch_tma_storage<__half>(p, shift, mode, in_map, out_map, s);
}

cudaError_t launch_sweep_tb2_f16(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                  cudaStream_t s) {
    return launch_tb2_storage<__half>(pa, pb, shift, mode, s);
}

}  // namespace btrt
