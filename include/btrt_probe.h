/*
 * btrt_probe.h -- measurement aid of the B-TriRT library: the throughput of the
 * GPU's FP64 pipe.  The paper has no counterpart; it exists because the FP64
 * sweep is bound by that rate (GB300 issues FP64 at a small fraction of its FP32
 * rate), so the sweep's roofline needs the measured rate of the GPU it runs on.
 */
#ifndef BTRT_PROBE_H
#define BTRT_PROBE_H

#include <stdint.h>

#include "btrt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Operation kinds of the probe. */
enum { BTRT_PROBE_FMA = 0, BTRT_PROBE_ADD = 1, BTRT_PROBE_MUL = 2 };

/* FP64 operations per second of independent chains of one operation kind
 * (BTRT_PROBE_FMA, _ADD or _MUL; one operation each, the unit of the sweep's
 * operation count) on the current device: `chains` (4, 8 or 16) chains per
 * thread, a warm-up launch, then one timed launch of `iters` iterations per
 * chain over a whole number of waves, timed with CUDA events on cuda_stream
 * (NULL = default stream), which it synchronises.  dev_sink: caller-owned device
 * memory of at least 8 bytes that the kernel may write (it keeps the chains from
 * being optimised away).  Writes the rate to *ops_per_s and the timed launch's
 * duration in milliseconds to *ms (ms may be NULL).  BTRT_EINVAL for null
 * arguments, iters < 1, another chain count or an unknown kind, BTRT_ECUDA when
 * a CUDA call fails. */
btrt_status btrt_probe_fp64_rate(void *cuda_stream, int32_t kind, int32_t chains, int64_t iters, void *dev_sink,
                                 double *ops_per_s, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* BTRT_PROBE_H */
