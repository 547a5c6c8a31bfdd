// btrt_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/btrt.h"
#include "btrt_reduce.cuh"
#include "btrt_sweep.cuh"

namespace btrt {

size_t elem_size(int fmt);
// A stored FP16 (IEEE binary16, by its definition) or BF16 value as a double.
double half_bits_to_double(int fmt, const unsigned char *p);

// Where each part of a lattice lives in its workspace (byte offsets).
struct Layout {
    long long pitch = 0;     // elements per row (f planes and phi plane)
    long long plane = 0;     // elements per plane
    size_t fbuf_bytes = 0;   // one buffer of 9 planes
    size_t off_f[2] = {0, 0};
    size_t off_phi[2] = {0, 0};   // phi planes, double-buffered with the populations
    size_t off_tab = 0, off_wall = 0, off_red = 0, off_resid = 0, total = 0;
    size_t off_srcf = 0, off_af = 0;   // optional field planes (0 when absent)
    int maxside = 0;
    long long resid_blocks = 0;   // partial slots of a residual sweep (one per block)
};

// Lattices whose phi is a double-word pair (a plane of low words after each phi plane).
inline bool has_phi_lo(const btrt_grid_desc &g) {
    return g.shift == BTRT_SHIFT_LOCAL_DW || g.shift == BTRT_SHIFT_LOCAL_DW_SR;
}
// Lattices whose 16-bit stored deviations are rounded stochastically.
inline bool stochastic_store(const btrt_grid_desc &g) {
    return g.shift == BTRT_SHIFT_LOCAL_SR || g.shift == BTRT_SHIFT_LOCAL_DW_SR || g.shift == BTRT_SHIFT_MOMENT_SR;
}
// Lattices that keep the writers' first moments (two planes of the storage format
// after the phi plane of each buffer).
inline bool has_j(const btrt_grid_desc &g) { return g.shift == BTRT_SHIFT_MOMENT_SR; }

// Stochastic-rounding seed of the step that produces step index n: the SplitMix64
// output function (Steele, Lea and Flood, 2014) of the step index.  Host and
// device (the batch kernels derive each step's seed from the member's step count)
// compute the same value.
__host__ __device__ inline unsigned int sr_step_seed(long long n) {
    unsigned long long z = (unsigned long long)n * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (unsigned int)(z ^ (z >> 31));
}

}  // namespace btrt

// The host-side lattice object behind btrt_lattice.
struct btrt_lattice_s {
    btrt_grid_desc g;
    btrt_coeffs c;
    btrt::Layout lay;
    unsigned char *ws = nullptr;
    cudaStream_t stream = nullptr;
    int cur = 0;              // buffer holding the current post-collision populations
    int64_t step = 0;
    double t0 = 0.0;
    bool have_coeffs = false, ready = false;
    int batch_refs = 0;       // batches that reference this lattice
    // lattice-unit constants derived from the coefficients
    double ux = 0, uy = 0, b2 = 0, A0[3] = {0, 0, 0}, K1[3] = {0, 0, 0}, k2 = 1;
    double bgx = 0, bgy = 0, bq = 2;   // power-law flux in lattice units: B^ += bg phi^q
    bool nonlin_A = false;
    double wall_const[4] = {0, 0, 0, 0};
    bool wall_is_arr[4] = {false, false, false, false};
    // TMA descriptors of the two population buffers (FP32-compute lattices)
    CUtensorMap tma_in[2];
    CUtensorMap tma_out[2];
    bool have_tma = false;
    int sweep_variant = 0;    // BTRT_SWEEP_AUTO / PLAIN / TMA
    bool have_srcf = false, have_af = false;   // fields uploaded

    // phi plane k; phi<Real>() is the current one (written with the populations of buffer cur)
    template <typename Real> Real *phi(int k) { return reinterpret_cast<Real *>(ws + lay.off_phi[k]); }
    template <typename Real> Real *phi() { return phi<Real>(cur); }
    // low words of phi plane k (BTRT_SHIFT_LOCAL_DW lattices: the plane after the high words)
    float *phi_lo(int k) {
        return btrt::has_phi_lo(g) ? reinterpret_cast<float *>(ws + lay.off_phi[k]) + lay.plane : nullptr;
    }
    void *fbuf(int k) { return ws + lay.off_f[k]; }
    // first-moment planes x, y of buffer k (BTRT_SHIFT_MOMENT_SR; after the phi plane)
    void *jplanes(int k) {
        return btrt::has_j(g) ? ws + lay.off_phi[k] + (size_t)lay.plane * sizeof(float) : nullptr;
    }
    template <typename Real> Real *tab() { return reinterpret_cast<Real *>(ws + lay.off_tab); }
    template <typename Real> Real *wall(int side) {
        return reinterpret_cast<Real *>(ws + lay.off_wall) + (size_t)side * lay.maxside;
    }
    double *partials() { return reinterpret_cast<double *>(ws + lay.off_red); }
    double *resid_partials() { return reinterpret_cast<double *>(ws + lay.off_resid); }
    template <typename Real> Real *srcf() { return lay.off_srcf ? reinterpret_cast<Real *>(ws + lay.off_srcf) : nullptr; }
    template <typename Real> Real *af() { return lay.off_af ? reinterpret_cast<Real *>(ws + lay.off_af) : nullptr; }
    double *red_out() { return partials() + btrt::kRedBlocks; }
    int *flags() { return reinterpret_cast<int *>(partials() + btrt::kRedBlocks + 2); }
};

namespace btrt {

// Sweep parameters of lattice L for the step that produces step index n
// (first: the initialising collision at t0).
template <typename Real> void fill_params(btrt_lattice L, SweepParams<Real> &p, int64_t n, bool first);
// Source factor dt (3 T_n - T_{n-1})/2 (or the constant's dt S) and wall factor
// exp(wall_lam t_n) of the step producing step index n.
void step_scalars(btrt_lattice L, int64_t n, bool first, double *src_val, double *wall_fac);
// Compiled variant (kGeneral / kLinear / kLinearK0One) that serves L's coefficients.
int sweep_mode(btrt_lattice L);
// Kernel form of L's ordinary steps (BTRT_SWEEP_AUTO resolved; PLAIN for FP64 and
// double-word lattices).
int effective_sweep_variant(btrt_lattice L);

// Threads of a single-lattice sweep block, and its grid: 32 x 8 threads, each
// sweeping rows_per_thread nodes of its column.
inline dim3 sweep_block() { return dim3(32, 8, 1); }
inline dim3 sweep_grid(int nx, int ny, int rows_per_thread) {
    const int rows = 8 * rows_per_thread;
    return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + rows - 1) / rows), 1);
}

// Exponent q as n + h/2 (n in [0, 8], h in {0, 1}) when it has that form, so the
// kernels take products and one square root; otherwise n = -1 (pow).
inline void half_split(double q, int *n, int *h) {
    const double t = 2.0 * q;
    if (q >= 0.0 && q <= 8.5 && t == (double)(long long)t) {
        *n = (int)(t / 2);
        *h = (int)((long long)t % 2);
    } else {
        *n = -1;
        *h = 0;
    }
}

// Storage shift of a lattice (kShiftNone for FP64 / double-word storage).
inline int shift_of(const btrt_grid_desc &g) {
    if (g.storage == BTRT_F64 || g.storage == BTRT_DF64) return kShiftNone;
    switch (g.shift) {
    case BTRT_SHIFT_LOCAL: return kShiftLocal;
    case BTRT_SHIFT_LOCAL_DW: return kShiftLocalDW;
    case BTRT_SHIFT_LOCAL_SR: return kShiftLocalSR;
    case BTRT_SHIFT_LOCAL_DW_SR: return kShiftLocalDWSR;
    case BTRT_SHIFT_MOMENT_SR: return kShiftMomentSR;
    default: return kShiftRef;
    }
}

// TMA-staged sweep (FP32 compute) and the box sizes its tensor maps need.
cudaError_t launch_sweep_tma(const SweepParams<float> &p, int storage, int shift, int mode,
                             const CUtensorMap *in_map, const CUtensorMap *out_map, cudaStream_t s);
void tma_box(int storage, int *box_in_x, int *box_in_y, int *box_out_x, int *box_out_y);

// Two steps in one launch (FP32 compute; storage BTRT_F32, F16 or BF16; shift
// kShiftRef or kShiftLocal): pa holds the parameters of the first step (its
// inputs), pb those of the second (its outputs).
cudaError_t launch_sweep_tb2(const SweepParams<float> &pa, const SweepParams<float> &pb, int storage, int shift,
                             int mode, cudaStream_t s);
cudaError_t launch_sweep_tb2_f32(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                 cudaStream_t s);
cudaError_t launch_sweep_tb2_f16(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                 cudaStream_t s);
cudaError_t launch_sweep_tb2_bf16(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                  cudaStream_t s);

// Two steps per launch with vector memory access (FP32 compute; arguments as
// launch_sweep_tb2).
cudaError_t launch_sweep_tb2v(const SweepParams<float> &pa, const SweepParams<float> &pb, int storage, int shift,
                              int mode, cudaStream_t s);
cudaError_t launch_sweep_tb2v_f32(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                  cudaStream_t s);
cudaError_t launch_sweep_tb2v_f16(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                  cudaStream_t s);
cudaError_t launch_sweep_tb2v_bf16(const SweepParams<float> &pa, const SweepParams<float> &pb, int shift, int mode,
                                   cudaStream_t s);

// One step per launch with vector memory access (FP32 compute; storage BTRT_F32,
// F16 or BF16; shift kShiftRef or kShiftLocal); never the initialising collision
// or a residual step.
cudaError_t launch_sweep_vec(const SweepParams<float> &p, int storage, int shift, int mode, cudaStream_t s);
cudaError_t launch_sweep_vec_f32(const SweepParams<float> &p, int shift, int mode, cudaStream_t s);
cudaError_t launch_sweep_vec_f16(const SweepParams<float> &p, int shift, int mode, cudaStream_t s);
cudaError_t launch_sweep_vec_bf16(const SweepParams<float> &p, int shift, int mode, cudaStream_t s);

// Blocks of one single-lattice sweep (32 x 8 threads, RowsPerThread nodes each).
long long sweep_blocks(int nx, int ny, int compute, int storage);

// Launch one sweep (or the initialising collision) for a (compute, storage) pair.
// compute: 0 = FP64, 1 = FP32; storage: BTRT_F64/F32/F16/BF16.
// mode: kGeneral, kLinear or kLinearK0One (FP64); kGeneral or kLinear (FP32).
cudaError_t launch_sweep_f64(const SweepParams<double> &p, int mode, cudaStream_t s);
cudaError_t launch_sweep_dw(const SweepParams<dw> &p, int mode, cudaStream_t s);
cudaError_t launch_sweep_f32(const SweepParams<float> &p, int storage, int shift, int mode, cudaStream_t s);

// Record the thread-local message returned by btrt_last_error (printf format).
void set_last_error(const char *fmt, ...);

// NVTX range around a host entry point (visible in Nsight timelines; no cost
// beyond a function-pointer test when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace btrt
