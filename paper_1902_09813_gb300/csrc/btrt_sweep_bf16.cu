// btrt_sweep_bf16.cu -- compiled variants of the FP32-compute sweep with bf16 storage
// (plain, TMA-staged and two-step; both storage shifts, both coefficient modes, every
// source kind).
#include "btrt_launch.cuh"

namespace btrt {

cudaError_t launch_sweep_f32_bf16(const SweepParams<float> &p, int shift, int mode, cudaStream_t s) {
    return launch_f32_storage<__nv_bfloat16>(p, shift, mode, s);
}

cudaError_t launch_sweep_tma_bf16(const SweepParams<float> &p, int shift, int mode, const CUtensorMap *in_map,
                                const CUtensorMap *out_map, cudaStream_t s) {
    return launch_tma_storage<__nv_bfloat16>(p, shift, mode, in_map, out_map, s);
}

cudaError_t launch_sweep_tb2_bf16(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                  cudaStream_t s) {
    return launch_tb2_storage<__nv_bfloat16>(pa, pb, shift, mode, s);
}

}  // namespace btrt
