// btrt_probe.cu -- throughput of GB300's FP64 pipe, measured on the device the
// caller has current.  The FP64 sweep is bound by this rate, not by HBM, so its
// roofline needs the rate of the GPU it runs on rather than the nominal figure.
//
// Every thread runs CHAINS independent chains of one FP64 operation kind (FMA,
// add or multiply) over `iters` iterations; the grid is a whole number of
// waves (blocks per SM x SMs).  Each operation counts as one FP64 operation, the
// unit of the sweep's operation count.  The sweep's own peak follows from its
// mix of kinds and their rates (the host combines them).
#include <cuda_runtime.h>

#include "../../include/btrt_probe.h"
#include "btrt_internal.h"

namespace {

constexpr int kProbeThreads = 256;

template <int KIND, int CHAINS>
__global__ void __launch_bounds__(kProbeThreads) fp64_chains(long long iters, double b, double c, double never,
                                                              double *sink) {
    double a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 0.1 + (double)(threadIdx.x + k) * 1e-6;
    for (long long n = 0; n < iters; ++n) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) {
            if constexpr (KIND == BTRT_PROBE_FMA) a[k] = fma(a[k], b, c);
            else if constexpr (KIND == BTRT_PROBE_ADD) a[k] = a[k] + c;
            else a[k] = a[k] * b;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    // never true for the arguments the host passes; keeps the chains live
    if (s == never) *sink = s;
}

template <int KIND, int CHAINS>
cudaError_t time_chains(cudaStream_t s, long long iters, double *sink, double *ops_per_s, double *ms) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_chains<KIND, CHAINS>,
                                                                            kProbeThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * sms;
    // values stay near 0.1: b slightly below 1 with c small for FMA; for adds and
    // multiplies they drift by iters * c or shrink by b^iters, far from overflow and subnormals
    const double b = 0.9999999, c = 1e-12, never = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        fp64_chains<KIND, CHAINS><<<grid, kProbeThreads, 0, s>>>(iters / 4 + 1, b, c, never, sink);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        fp64_chains<KIND, CHAINS><<<grid, kProbeThreads, 0, s>>>(iters, b, c, never, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    if (t <= 0.f) return cudaErrorUnknown;
    *ops_per_s = (double)grid * kProbeThreads * CHAINS * (double)iters / (t * 1e-3);
    *ms = t;
    return cudaSuccess;
}

template <int KIND>
cudaError_t time_kind(int chains, cudaStream_t s, long long iters, double *sink, double *r, double *ms) {
    switch (chains) {
    case 4: return time_chains<KIND, 4>(s, iters, sink, r, ms);
    case 8: return time_chains<KIND, 8>(s, iters, sink, r, ms);
    case 16: return time_chains<KIND, 16>(s, iters, sink, r, ms);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

extern "C" btrt_status btrt_probe_fp64_rate(void *cuda_stream, int32_t kind, int32_t chains, int64_t iters,
                                            void *dev_sink, double *ops_per_s, double *ms) {
    if (!dev_sink || !ops_per_s || iters < 1 || (chains != 4 && chains != 8 && chains != 16) ||
        (kind != BTRT_PROBE_FMA && kind != BTRT_PROBE_ADD && kind != BTRT_PROBE_MUL)) {
        btrt::set_last_error("btrt_probe_fp64_rate: null argument, iters < 1, chains not 4/8/16 or unknown kind");
        return BTRT_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *sink = static_cast<double *>(dev_sink);
    double t = 0.0;
    cudaError_t e = kind == BTRT_PROBE_FMA ? time_kind<BTRT_PROBE_FMA>(chains, s, iters, sink, ops_per_s, &t)
                    : kind == BTRT_PROBE_ADD ? time_kind<BTRT_PROBE_ADD>(chains, s, iters, sink, ops_per_s, &t)
                                             : time_kind<BTRT_PROBE_MUL>(chains, s, iters, sink, ops_per_s, &t);
    if (e != cudaSuccess) {
        btrt::set_last_error("btrt_probe_fp64_rate: %s", cudaGetErrorString(e));
        return BTRT_ECUDA;
    }
    if (ms) *ms = t;
    return BTRT_OK;
}
