// btrt_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "btrt_sweep.cuh"

namespace btrt {

// Launch one sweep (or the initialising collision) for a (compute, storage) pair.
// compute: 0 = FP64, 1 = FP32; storage: BTRT_F64/F32/F16/BF16.
// mode: kGeneral, kLinear or kLinearK0One (FP64); kGeneral or kLinear (FP32).
cudaError_t launch_sweep_f64(const SweepParams<double> &p, int mode, cudaStream_t s);
cudaError_t launch_sweep_f32(const SweepParams<float> &p, int storage, int mode, cudaStream_t s);

// Record the thread-local message returned by btrt_last_error (printf format).
void set_last_error(const char *fmt, ...);

}  // namespace btrt
