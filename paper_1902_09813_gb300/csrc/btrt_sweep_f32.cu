// btrt_sweep_f32.cu -- compiled variants of the FP32-compute sweep with f32 storage
// (plain, TMA-staged and two-step; both storage shifts, both coefficient modes, every
// source kind).
#include "btrt_launch.cuh"

namespace btrt {

cudaError_t launch_sweep_f32_f32(const SweepParams<float> &p, int shift, int mode, cudaStream_t s) {
    return launch_f32_storage<float>(p, shift, mode, s);
}

cudaError_t launch_sweep_tma_f32(const SweepParams<float> &p, int shift, int mode, const CUtensorMap *in_map,
                                const CUtensorMap *out_map, cudaStream_t s) {
    return launch_tma_storage<float>(p, shift, mode, in_map, out_map, s);
}

cudaError_t launch_sweep_tb2_f32(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                  cudaStream_t s) {
    return launch_tb2_storage<float>(pa, pb, shift, mode, s);
}

cudaError_t launch_sweep_tb2(const SweepParams<float> &pa, const SweepParams<float> &pb, int storage, int shift,
                             int mode, cudaStream_t s) {
    switch (storage) {
    case BTRT_F16: return launch_sweep_tb2_f16(pa, pb, shift, mode, s);
    case BTRT_BF16: return launch_sweep_tb2_bf16(pa, pb, shift, mode, s);
    default: return launch_sweep_tb2_f32(pa, pb, shift, mode, s);
    }
}

}  // namespace btrt
