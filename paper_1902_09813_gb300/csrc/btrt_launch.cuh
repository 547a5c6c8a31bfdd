// btrt_launch.cuh -- launch helpers of the FP32-compute sweeps, instantiated per
// storage format in their own translation units (btrt_sweep_*.cu) so that the
// many compiled variants build in parallel.
#pragma once

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "btrt_internal.h"
#include "btrt_tb.cuh"
#include "btrt_tma.cuh"
#include "btrt_tb2v.cuh"
#include "btrt_vec.cuh"

namespace btrt {

// Dispatch on the source kind so that each compiled sweep carries only its own
// source arithmetic.
template <typename Real, typename S, int SH, int MODE>
inline void launch_src(const SweepParams<Real> &p, dim3 g, dim3 b, cudaStream_t s) {
    switch (p.src_kind) {
    case 0: sweep_kernel<Real, S, SH, MODE, 0><<<g, b, 0, s>>>(p); break;
    case 1: sweep_kernel<Real, S, SH, MODE, 1><<<g, b, 0, s>>>(p); break;
    case 2: sweep_kernel<Real, S, SH, MODE, 2><<<g, b, 0, s>>>(p); break;
    case 3: sweep_kernel<Real, S, SH, MODE, 3><<<g, b, 0, s>>>(p); break;
    default: sweep_kernel<Real, S, SH, MODE, kSrcReaction><<<g, b, 0, s>>>(p); break;
    }
}

// Plain FP32-compute sweep for storage S: shift (reference, local, local with a
// double-word phi; for 16-bit storage also both local forms with stochastic
// rounding) x {kGeneral, kLinear} x source.
template <typename S>
cudaError_t launch_f32_storage(const SweepParams<float> &p, int shift, int mode, cudaStream_t s) {
    const dim3 g = sweep_grid(p.nx, p.ny, RowsPerThread<float, S>::value), b = sweep_block();
    const bool lin = mode != kGeneral;
    constexpr bool S16 = !std::is_same<S, float>::value;
    if (shift == kShiftLocal) {
        if (lin) launch_src<float, S, kShiftLocal, kLinear>(p, g, b, s);
        else launch_src<float, S, kShiftLocal, kGeneral>(p, g, b, s);
    } else if (shift == kShiftLocalDW) {
        if (lin) launch_src<float, S, kShiftLocalDW, kLinear>(p, g, b, s);
        else launch_src<float, S, kShiftLocalDW, kGeneral>(p, g, b, s);
    } else if (shift == kShiftLocalSR || shift == kShiftLocalDWSR || shift == kShiftMomentSR) {
        if constexpr (S16) {
            if (shift == kShiftLocalSR) {
                if (lin) launch_src<float, S, kShiftLocalSR, kLinear>(p, g, b, s);
                else launch_src<float, S, kShiftLocalSR, kGeneral>(p, g, b, s);
            } else if (shift == kShiftMomentSR) {
                if (lin) launch_src<float, S, kShiftMomentSR, kLinear>(p, g, b, s);
                else launch_src<float, S, kShiftMomentSR, kGeneral>(p, g, b, s);
            } else {
                if (lin) launch_src<float, S, kShiftLocalDWSR, kLinear>(p, g, b, s);
                else launch_src<float, S, kShiftLocalDWSR, kGeneral>(p, g, b, s);
            }
        } else {
            return cudaErrorInvalidValue;   // stochastic rounding serves 16-bit storage
        }
    } else {
        if (lin) launch_src<float, S, kShiftRef, kLinear>(p, g, b, s);
        else launch_src<float, S, kShiftRef, kGeneral>(p, g, b, s);
    }
    return cudaGetLastError();
}

// TMA-staged sweep: a persistent grid of at most (resident blocks per SM) x SMs.
template <typename S, int SH, int MODE, int SRC>
cudaError_t launch_tma_src(const SweepParams<float> &p, const CUtensorMap *in_map, const CUtensorMap *out_map,
                           cudaStream_t s) {
    using G = TmaGeom<S>;
    // The shared-memory attribute belongs to the current device's context, so it
    // is set, and the grid measured, once per instantiation and device, under a lock.
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static int per_sm_of[kMaxDev] = {}, sms_of[kMaxDev] = {};   // 0: not configured yet
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    int per_sm = 0, sms = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!per_sm_of[dev]) {
            e = cudaFuncSetAttribute(sweep_tma_kernel<S, SH, MODE, SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     G::SMEM);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_tma_kernel<S, SH, MODE, SRC>,
                                                                  G::THREADS, G::SMEM);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            sms_of[dev] = sms;
            per_sm_of[dev] = per_sm;
        }
        per_sm = per_sm_of[dev];
        sms = sms_of[dev];
    }
    const int ntx = (p.nx + G::TX - 1) / G::TX;
    const int nty = (p.ny + G::TY - 1) / G::TY;
    const int ntiles = ntx * nty;
    const int grid = std::min(ntiles, per_sm * sms);
    sweep_tma_kernel<S, SH, MODE, SRC><<<grid, G::THREADS, G::SMEM, s>>>(p, *in_map, *out_map, ntx, ntiles,
                                                                        1u << 22);
    return cudaGetLastError();
}

template <typename S, int SH, int MODE>
cudaError_t launch_tma_mode(const SweepParams<float> &p, const CUtensorMap *in_map, const CUtensorMap *out_map,
                            cudaStream_t s) {
    switch (p.src_kind) {
    case 0: return launch_tma_src<S, SH, MODE, 0>(p, in_map, out_map, s);
    case 1: return launch_tma_src<S, SH, MODE, 1>(p, in_map, out_map, s);
    case 2: return launch_tma_src<S, SH, MODE, 2>(p, in_map, out_map, s);
    case 3: return launch_tma_src<S, SH, MODE, 3>(p, in_map, out_map, s);
    default: return launch_tma_src<S, SH, MODE, kSrcReaction>(p, in_map, out_map, s);
    }
}

template <typename S>
cudaError_t launch_tma_storage(const SweepParams<float> &p, int shift, int mode, const CUtensorMap *in_map,
                               const CUtensorMap *out_map, cudaStream_t s) {
    const bool lin = mode != kGeneral;
    if (shift == kShiftLocal)
        return lin ? launch_tma_mode<S, kShiftLocal, kLinear>(p, in_map, out_map, s)
                   : launch_tma_mode<S, kShiftLocal, kGeneral>(p, in_map, out_map, s);
    return lin ? launch_tma_mode<S, kShiftRef, kLinear>(p, in_map, out_map, s)
               : launch_tma_mode<S, kShiftRef, kGeneral>(p, in_map, out_map, s);
}

// Two steps per launch: one block per output tile, 24-35 KB of shared memory.
template <typename S, int SH, int MODE, int SRC>
cudaError_t launch_tb2_src(const SweepParams<float> &pa, const SweepParams<float> &pb, cudaStream_t s) {
    using G = TbGeomFor<MODE>;
    const int ntx = (pa.nx + G::TX - 1) / G::TX;
    const int nty = (pa.ny + G::TY - 1) / G::TY;
    sweep_tb2_kernel<S, SH, MODE, SRC><<<ntx * nty, G::THREADS, G::SMEM, s>>>(pa, pb, ntx);
    return cudaGetLastError();
}

template <typename S, int SH, int MODE>
cudaError_t launch_tb2_mode(const SweepParams<float> &pa, const SweepParams<float> &pb, cudaStream_t s) {
    switch (pa.src_kind) {
    case kSrcNone: return launch_tb2_src<S, SH, MODE, kSrcNone>(pa, pb, s);
    case kSrcConst: return launch_tb2_src<S, SH, MODE, kSrcConst>(pa, pb, s);
    case kSrcTrig: return launch_tb2_src<S, SH, MODE, kSrcTrig>(pa, pb, s);
    case kSrcField: return launch_tb2_src<S, SH, MODE, kSrcField>(pa, pb, s);
    default: return launch_tb2_src<S, SH, MODE, kSrcReaction>(pa, pb, s);
    }
}

template <typename S>
cudaError_t launch_tb2_storage(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                               cudaStream_t s) {
    if (shift == kShiftLocal)
        return mode == kGeneral ? launch_tb2_mode<S, kShiftLocal, kGeneral>(pa, pb, s)
                                : launch_tb2_mode<S, kShiftLocal, kLinear>(pa, pb, s);
    return mode == kGeneral ? launch_tb2_mode<S, kShiftRef, kGeneral>(pa, pb, s)
                            : launch_tb2_mode<S, kShiftRef, kLinear>(pa, pb, s);
}

// Two steps per launch with vector memory access (btrt_tb2v.cuh): one block per
// 32 x TY output tile.
template <typename S, int SH, int MODE, int SRC>
cudaError_t launch_tb2v_src(const SweepParams<float> &pa, const SweepParams<float> &pb, cudaStream_t s) {
    using G = Tb2vGeom<S>;
    const int ntx = (pa.nx + G::TX - 1) / G::TX;
    const int nty = (pa.ny + G::TY - 1) / G::TY;
    sweep_tb2v_kernel<S, SH, MODE, SRC><<<ntx * nty, G::THREADS, G::SMEM, s>>>(pa, pb, ntx);
    return cudaGetLastError();
}

template <typename S, int SH, int MODE>
cudaError_t launch_tb2v_mode(const SweepParams<float> &pa, const SweepParams<float> &pb, cudaStream_t s) {
    switch (pa.src_kind) {
    case kSrcNone: return launch_tb2v_src<S, SH, MODE, kSrcNone>(pa, pb, s);
    case kSrcConst: return launch_tb2v_src<S, SH, MODE, kSrcConst>(pa, pb, s);
    case kSrcTrig: return launch_tb2v_src<S, SH, MODE, kSrcTrig>(pa, pb, s);
    case kSrcField: return launch_tb2v_src<S, SH, MODE, kSrcField>(pa, pb, s);
    default: return launch_tb2v_src<S, SH, MODE, kSrcReaction>(pa, pb, s);
    }
}

template <typename S>
cudaError_t launch_tb2v_storage(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                cudaStream_t s) {
    if (shift == kShiftLocal)
        return mode == kGeneral ? launch_tb2v_mode<S, kShiftLocal, kGeneral>(pa, pb, s)
                                : launch_tb2v_mode<S, kShiftLocal, kLinear>(pa, pb, s);
    return mode == kGeneral ? launch_tb2v_mode<S, kShiftRef, kGeneral>(pa, pb, s)
                            : launch_tb2v_mode<S, kShiftRef, kLinear>(pa, pb, s);
}

// One step per launch with vector memory access (btrt_vec.cuh).
template <typename S, int SH, int MODE>
inline void launch_vec_src(const SweepParams<float> &p, cudaStream_t s) {
    const dim3 g = sweep_vec_grid(p.nx, p.ny), b = sweep_block();
    switch (p.src_kind) {
    case kSrcNone: sweep_vec_kernel<S, SH, MODE, kSrcNone><<<g, b, 0, s>>>(p); break;
    case kSrcConst: sweep_vec_kernel<S, SH, MODE, kSrcConst><<<g, b, 0, s>>>(p); break;
    case kSrcTrig: sweep_vec_kernel<S, SH, MODE, kSrcTrig><<<g, b, 0, s>>>(p); break;
    case kSrcField: sweep_vec_kernel<S, SH, MODE, kSrcField><<<g, b, 0, s>>>(p); break;
    default: sweep_vec_kernel<S, SH, MODE, kSrcReaction><<<g, b, 0, s>>>(p); break;
    }
}

template <typename S>
cudaError_t launch_vec_storage(const SweepParams<float> &p, int shift, int mode, cudaStream_t s) {
    const bool lin = mode != kGeneral;
    if (shift == kShiftLocal) {
        if (lin) launch_vec_src<S, kShiftLocal, kLinear>(p, s);
        else launch_vec_src<S, kShiftLocal, kGeneral>(p, s);
    } else if (shift == kShiftLocalSR || shift == kShiftMomentSR) {
        if constexpr (!std::is_same<S, float>::value) {
            if (shift == kShiftLocalSR) {
                if (lin) launch_vec_src<S, kShiftLocalSR, kLinear>(p, s);
                else launch_vec_src<S, kShiftLocalSR, kGeneral>(p, s);
            } else {
                if (lin) launch_vec_src<S, kShiftMomentSR, kLinear>(p, s);
                else launch_vec_src<S, kShiftMomentSR, kGeneral>(p, s);
            }
        } else {
            return cudaErrorInvalidValue;
        }
    } else {
        if (lin) launch_vec_src<S, kShiftRef, kLinear>(p, s);
        else launch_vec_src<S, kShiftRef, kGeneral>(p, s);
    }
    return cudaGetLastError();
}

}  // namespace btrt
