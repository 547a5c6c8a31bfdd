// btrt_batch.cu -- many independent lattices of uneven size in one persistent launch.
//
// A batch owns a descriptor per member (its sweep parameters and step counter),
// a table of tiles covering every member, a per-step table of source and wall
// factors, and two kernel forms over the same tile code:
//  - persistent: one cooperative launch per call; all resident blocks walk the
//    tile table for one time step, meet at a grid barrier (bounded wait) and go
//    on with the next step;
//  - step-per-launch: one launch per step over all tiles.
//  - two-step: FP32 compute only; one launch per pair of steps over a table of
//    the two-step kernel's output tiles (btrt_tb.cuh), the last step of a slice
//    that wants the residual (or an odd one) in the step-per-launch form.
//  - vector: FP32 compute only; one launch per step over tiles swept four
//    x-consecutive nodes per thread (btrt_vec.cuh).
// Each form is captured in a CUDA graph per (steps, residual) pair and
// replayed.  Members keep their own workspaces; the batch workspace holds only
// the descriptors, tables and reduction scratch.  btrt_batch_autotune times the
// candidate tile shapes in every form on real steps and keeps the fastest.
// Tables go up from pinned staging memory, so no call waits for work already
// queued on the batch stream: a serving loop can queue slice k + 1 before it
// reads slice k's flags.  With freezing on, btrt_batch_step_tol marks every
// member it flags in the member's own device flags, and launches of any batch
// skip marked members (btrt_settle rewinds the member's step count afterwards).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/btrt.h"
#include "btrt_internal.h"
#include "btrt_tb.cuh"
#include "btrt_vec.cuh"

using namespace btrt;

namespace {

template <typename Real>
struct BatchMember {
    SweepParams<Real> p;       // fin, phi_in = buffers 0; fout, phi_out = buffers 1; first = 0
    long long step;            // completed steps at the start of the launch
    int cur;                   // buffer holding the current populations at the start
    int mode;                  // kGeneral or kLinear
};

// Resident blocks per SM the FP32 constant-coefficient step-per-launch form is
// compiled for (0: the compiler's choice).  Five (48 registers, a few spilled
// words) measured 73.7 GLUPS on the 512-instance FP16 batch against 68.6 with
// the compiler's 58-61 registers and four blocks.
#ifndef BTRT_BATCH_LIN_MINBLOCKS
#define BTRT_BATCH_LIN_MINBLOCKS 5
#endif

constexpr int kMaxSliceSteps = 4096;   // steps per launch (the step table holds this many)

template <typename Real>
struct BatchArgs {
    const BatchMember<Real> *members;
    const int4 *tiles;         // {member, x0, y0, 0}
    int ntiles;
    const int4 *tiles2;        // the two-step kernel's output tiles {member, x0, y0, 0}
    int ntiles2;
    const int4 *tilesv;        // the vector form's tiles {member, x0, y0, 0}: (4 bx) x (by rows) nodes
    int ntilesv;
    int rows;                  // nodes per thread along y
    int nsteps;
    int want_resid;
    double *tile_partials;     // sum (phi^n - phi^{n-1})^2 per tile, last step
    unsigned int *barrier;     // arrivals, zeroed before the launch
    int *err;                  // bit 1: a barrier wait gave up
    unsigned long long wait_limit;
    unsigned int barrier_extra;  // added to every barrier target (0; >0 only to test the timeout path)
    const Real *step_vals;     // [member][table_steps][2]: source factor, wall factor of each step of the launch
    int table_steps;
};

// Grid-wide barrier with a bounded wait.  All blocks are co-resident (cooperative
// launch).  Returns false after raising err bit 1 when the wait gave up.
__device__ __forceinline__ bool grid_barrier(unsigned int *count, unsigned int target, int *err,
                                             unsigned long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        int good = 1;
        unsigned long long polls = 0;
        while (atomicAdd(count, 0u) < target) {
            if (++polls > limit) {
                atomicOr(err, 2);
                good = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Member m was frozen by an earlier btrt_batch_step_tol (word 1 of its lattice's
// device flags): launches leave it as it is.  The mark changes only between
// launches, so every thread of a block reads the same value.
template <typename Real>
__device__ __forceinline__ bool member_frozen(const BatchArgs<Real> &a, int m) {
    return (a.members[m].p.flags[1] & 1) != 0;
}

// One tile of one step: load the member's parameters into shared memory, patch
// the step-dependent ones (buffer parity, source and wall time factors from the
// host-computed step table) and sweep the tile's nodes.  LIN: every member of
// the batch takes the constant-coefficient collision and a source other than
// the reaction term, so only that collision and those sources are compiled
// (fewer registers than the form that can take any member).
// Copy member M's parameters into shared memory and patch the step-dependent
// ones: buffer parity (flips since the slice began) and the source and wall time
// factors of step k of the slice from the host-computed step table.  The caller
// places no barrier before reading sp; this function ends with one.
template <typename Real>
__device__ __forceinline__ void stage_member(const BatchArgs<Real> &a, int member, int k, int flip,
                                             SweepParams<Real> &sp) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    const BatchMember<Real> &M = a.members[member];
    __syncthreads();   // the previous tile is done with sp
    {
        const int *src = reinterpret_cast<const int *>(&M.p);
        int *dst = reinterpret_cast<int *>(&sp);
        for (int w = tid; w < (int)(sizeof(SweepParams<Real>) / 4); w += nthr) dst[w] = src[w];
    }
    __syncthreads();
    if (tid == 0) {
        const int cur = (M.cur + flip) & 1;  // buffer flips since the slice began
        const void *b0 = M.p.fin;            // buffer 0
        void *b1 = M.p.fout;                 // buffer 1
        sp.fin = cur ? b1 : b0;
        sp.fout = cur ? const_cast<void *>(b0) : b1;
        const Real *q0 = M.p.phi_in;         // phi plane 0
        Real *q1 = M.p.phi_out;              // phi plane 1
        sp.phi_in = cur ? q1 : q0;
        sp.phi_out = cur ? const_cast<Real *>(q0) : q1;
    } else if (tid == 32) {
        const Real *v = a.step_vals + ((size_t)member * a.table_steps + k) * 2;
        sp.src_val = v[0];
        sp.wall_fac = v[1];
        sp.first = 0;
        sp.sr_seed = sr_step_seed(M.step + k + 1);   // stochastic rounding: the seed of this step
    }
    __syncthreads();
}

// One tile of one step: stage the member's parameters (stage_member) and sweep
// the tile's nodes.  LIN: every member of the batch takes the constant-coefficient
// collision and a source other than the reaction term, so only that collision and
// those sources are compiled (fewer registers than the form that can take any member).
template <typename Real, typename S, int SH, bool L2ONLY, bool LIN>
__device__ __forceinline__ void batch_tile(const BatchArgs<Real> &a, int t, int k, int flip, bool resid,
                                           SweepParams<Real> &sp, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    const int4 tile = a.tiles[t];
    if (member_frozen(a, tile.x)) return;
    const BatchMember<Real> &M = a.members[tile.x];
    stage_member(a, tile.x, k, flip, sp);
    const SweepParams<Real> &lp = sp;
    const int x = tile.y + threadIdx.x;
    double r = 0.0;
    if (x < lp.nx) {
        const int y0 = tile.z + threadIdx.y;
        if (!LIN && M.mode == kGeneral) {
            if (resid) r = sweep_rows<Real, S, SH, kGeneral, kSrcRuntime, L2ONLY, true>(lp, x, y0, blockDim.y, a.rows);
            else sweep_rows<Real, S, SH, kGeneral, kSrcRuntime, L2ONLY, false>(lp, x, y0, blockDim.y, a.rows);
        } else {
            constexpr int SRC = LIN ? kSrcRuntimeNR : kSrcRuntime;
            if (resid) r = sweep_rows<Real, S, SH, kLinear, SRC, L2ONLY, true>(lp, x, y0, blockDim.y, a.rows);
            else sweep_rows<Real, S, SH, kLinear, SRC, L2ONLY, false>(lp, x, y0, blockDim.y, a.rows);
        }
    }
    if (resid) {
        red[tid] = r;
        __syncthreads();
        for (int s = nthr / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        if (tid == 0) a.tile_partials[t] = red[0];
    }
}

// Persistent form: every resident block walks the tile table each step; a
// bounded grid barrier separates the steps.  Population and phi loads go
// through L2 only, since other SMs rewrote them in the previous step.
template <typename Real, typename S, int SH, bool LIN>
__global__ void __launch_bounds__(256) batch_kernel(const __grid_constant__ BatchArgs<Real> a) {
    __shared__ SweepParams<Real> sp;
    __shared__ double red[256];
    for (int k = 0; k < a.nsteps; ++k) {
        const bool resid = a.want_resid && (k == a.nsteps - 1);
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) batch_tile<Real, S, SH, true, LIN>(a, t, k, k, resid, sp, red);
        if (!grid_barrier(a.barrier, (unsigned)(k + 1) * gridDim.x + a.barrier_extra, a.err, a.wait_limit))
            return;
    }
}

// Step-per-launch form: one launch per step (all of them in one CUDA graph);
// kernel boundaries order the steps, so no barrier and ordinary cached loads.
template <typename Real, typename S, int SH, bool LIN>
__global__ void __launch_bounds__(256, (LIN && sizeof(Real) == 4) ? BTRT_BATCH_LIN_MINBLOCKS : 0)
    batch_step_kernel(const __grid_constant__ BatchArgs<Real> a, int k, int flip) {
    __shared__ SweepParams<Real> sp;
    __shared__ double red[256];
    const bool resid = a.want_resid && (k == a.nsteps - 1);
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x)
        batch_tile<Real, S, SH, false, LIN>(a, t, k, flip, resid, sp, red);
}

// Vector form (FP32 compute): one launch per step (all of them in one CUDA
// graph), one block per tile of (4 bx) x (by rows) nodes; each thread owns four
// x-consecutive nodes of `rows` rows and sweeps them with the single-lattice
// vector sweep's code (btrt_vec.cuh), so every node's arithmetic is that of the
// plain form.  Resident blocks per SM it is compiled for: BatchVecMinBlocks for the
// constant-coefficient form (16-bit storage: BTRT_BATCH_VEC_MINBLOCKS_S16; FP32
// storage two), two for the form that takes any member, which spills 700-900
// bytes at four.  On the 512-instance FP16 batch (32 x 4 threads, 4 rows) three
// blocks of 256 threads (85 registers) measured 104.6 GLUPS, four (64 registers,
// spilling) 98.2 and two 87.4.
#ifndef BTRT_BATCH_VEC_MINBLOCKS_S16
#define BTRT_BATCH_VEC_MINBLOCKS_S16 3
#endif
template <typename S> struct BatchVecMinBlocks { static constexpr int value = BTRT_BATCH_VEC_MINBLOCKS_S16; };
template <> struct BatchVecMinBlocks<float> { static constexpr int value = 2; };
// The members' folded collision constants travel in the launch's parameter
// block: the kernel reads them from the constant bank, as the single-lattice
// kernels read theirs, instead of holding them in registers loaded from shared
// memory.  One launch serves at most kParamMembers members (a contiguous range
// of the vector form's tile table); larger batches take several launches a step.
constexpr int kParamMembers = 256;
struct BatchVecArgs {
    BatchArgs<float> a;
    int m0;                                   // first member of this launch
    int t0;                                   // its first tile in the vector form's tile table
    FoldConsts<float> lin[kParamMembers];     // constants of members m0, m0 + 1, ...
};

template <typename S, int SH, bool LIN>
__global__ void __launch_bounds__(256, LIN ? BatchVecMinBlocks<S>::value : 2)
    batch_vec_kernel(const __grid_constant__ BatchVecArgs va, int k, int flip) {
    __shared__ SweepParams<float> sp;
    const BatchArgs<float> &a = va.a;
    const int4 tile = a.tilesv[va.t0 + blockIdx.x];
    if (member_frozen(a, tile.x)) return;
    const int mode = a.members[tile.x].mode;
    const FoldConsts<float> *Lc = &va.lin[tile.x - va.m0];
    stage_member(a, tile.x, k, flip, sp);
    const SweepParams<float> &lp = sp;
    const int x0 = tile.y + threadIdx.x * kVec;
    bool bad = false;
    // interior groups on the vector path, then the tile's edge nodes spread over the block
    const int tw = kVec * blockDim.x, th = blockDim.y * a.rows;
    if (LIN || mode != kGeneral) {
        constexpr int SRC = LIN ? kSrcRuntimeNR : kSrcRuntime;
        if (x0 < lp.nx)
            for (int r = 0; r < a.rows; ++r) {
                const int y = tile.z + threadIdx.y + r * blockDim.y;
                if (y >= lp.ny) break;
                bad |= vec_group_inner<S, SH, kLinear, SRC>(lp, x0, y, Lc);
            }
        bad |= vec_tile_edges<S, SH, kLinear, SRC>(lp, tile.y, tile.z, tw, th, Lc);
    } else {
        if (x0 < lp.nx)
            for (int r = 0; r < a.rows; ++r) {
                const int y = tile.z + threadIdx.y + r * blockDim.y;
                if (y >= lp.ny) break;
                bad |= vec_group_inner<S, SH, kGeneral, kSrcRuntime>(lp, x0, y, Lc);
            }
        bad |= vec_tile_edges<S, SH, kGeneral, kSrcRuntime>(lp, tile.y, tile.z, tw, th, Lc);
    }
    if (bad) atomicOr(lp.flags, 1);
}

// Two-step form (FP32 compute): steps k and k + 1 of the slice in one launch, one
// block per two-step output tile; flip = buffer flips since the slice began.
// Resident blocks per SM the two-step batch form is compiled for: four (64
// registers) for the constant-coefficient collision, three for the per-node one.
// On the 512-instance FP16 batch four blocks measured 73.3 GLUPS, five (48
// registers, 200 spilled bytes) 58.5 and the compiler's 80-128 registers 63.2.
#ifndef BTRT_BATCH_TB2_MINBLOCKS_LIN
#define BTRT_BATCH_TB2_MINBLOCKS_LIN 4
#endif
#ifndef BTRT_BATCH_TB2_MINBLOCKS_GEN
#define BTRT_BATCH_TB2_MINBLOCKS_GEN 3
#endif
template <typename S, int SH, bool LIN>
__global__ void __launch_bounds__(256, LIN ? BTRT_BATCH_TB2_MINBLOCKS_LIN : BTRT_BATCH_TB2_MINBLOCKS_GEN)
    batch_tb2_kernel(const __grid_constant__ BatchArgs<float> a, int k, int flip) {
    __shared__ SweepParams<float> spa, spb;
    extern __shared__ float tb_smem[];
    const int tid = threadIdx.x;
    const int4 tile = a.tiles2[blockIdx.x];
    if (member_frozen(a, tile.x)) return;
    const BatchMember<float> &M = a.members[tile.x];
    {
        const int *src = reinterpret_cast<const int *>(&M.p);
        int *da = reinterpret_cast<int *>(&spa), *db = reinterpret_cast<int *>(&spb);
        for (int w = tid; w < (int)(sizeof(SweepParams<float>) / 4); w += blockDim.x) {
            const int v = src[w];
            da[w] = v;
            db[w] = v;
        }
    }
    __syncthreads();
    if (tid == 0) {
        // both steps read buffer cur and write the other one (the first step's
        // output stays in shared memory)
        const int cur = (M.cur + flip) & 1;
        const void *b0 = M.p.fin;
        void *b1 = M.p.fout;
        const float *q0 = M.p.phi_in;
        float *q1 = M.p.phi_out;
        spa.fin = spb.fin = cur ? b1 : b0;
        spa.fout = spb.fout = cur ? const_cast<void *>(b0) : b1;
        spa.phi_in = spb.phi_in = cur ? q1 : q0;
        spa.phi_out = spb.phi_out = cur ? const_cast<float *>(q0) : q1;
        const float *v = a.step_vals + ((size_t)tile.x * a.table_steps + k) * 2;
        spa.src_val = v[0];
        spa.wall_fac = v[1];
        spa.first = 0;
    } else if (tid == 32) {
        const float *v = a.step_vals + ((size_t)tile.x * a.table_steps + k + 1) * 2;
        spb.src_val = v[0];
        spb.wall_fac = v[1];
        spb.first = 0;
    }
    __syncthreads();
    bool bad;
    if (LIN || M.mode != kGeneral)
        bad = tb2_tile<S, SH, kLinear, LIN ? kSrcRuntimeNR : kSrcRuntime, TbGeom::TY>(spa, spb, tile.y, tile.z,
                                                                                       tb_smem);
    else
        bad = tb2_tile<S, SH, kGeneral, kSrcRuntime, TbGeom::TY>(spa, spb, tile.y, tile.z, tb_smem);
    if (bad) atomicOr(spb.flags, 1);
}

// Each member's device flags (bit 0: non-finite phi) gathered into one array.
template <typename Real>
__global__ void gather_member_flags(const BatchMember<Real> *members, int n, int *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = *members[k].p.flags;
}

// Per-member stop flags after a residual slice: bit 0 residual < tol, bit 1 a
// non-finite phi in the member (its device flag bit 0), bit 2 the member was
// frozen before this slice (its residual is then not that of a step: NaN).
// resid_out (optional) receives the residuals.  freeze: a member flagged here is
// marked in words 1-3 of its lattice's flags: word 1 = 1 | (buffer index << 1),
// words 2-3 = the step count, both as after this slice (chunk steps, `flips`
// buffer flips since the member descriptors' step and buffer index).
template <typename Real>
__global__ void member_done(const BatchMember<Real> *members, const double *resid, int n, double tol, int *out,
                            double *resid_out, int freeze, int chunk, int flips) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const BatchMember<Real> &M = members[k];
    int *lf = M.p.flags;
    if (lf[1] & 1) {
        out[k] = 4;
        if (resid_out) resid_out[k] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int f = (resid[k] < tol ? 1 : 0) | ((lf[0] & 1) ? 2 : 0);
    out[k] = f;
    if (resid_out) resid_out[k] = resid[k];
    if (freeze && f) {
        *reinterpret_cast<long long *>(lf + 2) = M.step + chunk;
        lf[1] = 1 | (((M.cur + flips) & 1) << 1);
    }
}

// Per-member residual: fixed-order sum of its tiles' partials, then sqrt.
__global__ void __launch_bounds__(256) member_residual(const double *tile_partials, const int *tile_begin,
                                                       const int *tile_count, double *out) {
    __shared__ double sh[256];
    const int m = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < tile_count[m]; k += blockDim.x) acc += tile_partials[tile_begin[m] + k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[m] = sqrt(sh[0]);
}

thread_local std::string t_err;

btrt_status bfail(btrt_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error("%s", buf);
    return code;
}

#define BCUDA(expr)                                                                       \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bfail(BTRT_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),   \
                         __FILE__, __LINE__);                                             \
    } while (0)

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct Shape {
    int bx, by, rows;
    int per_step;   // 0: persistent launch per call; 1: one launch per step; 2: two steps per launch
                    // (FP32 compute; its odd or residual last step in the form of 1); 3: one launch
                    // per step in the vector form (FP32 compute; its residual step in the form of 1)
};
const Shape kShapes[] = {{32, 8, 1, 0}, {32, 8, 2, 0}, {32, 8, 4, 0}, {64, 4, 1, 0},  {64, 4, 2, 0},
                         {32, 4, 2, 0}, {16, 16, 1, 0}, {8, 32, 1, 0}, {32, 4, 4, 0}, {16, 8, 2, 0}};
constexpr int kForms = 4;   // launch forms 0 .. 3 (FP64 batches: 0 and 1)

// Grid sizes of the members: all the batch tables depend on.
struct MemberGeom {
    int nx, ny;
};

std::vector<MemberGeom> geoms_of(const std::vector<btrt_lattice> &m) {
    std::vector<MemberGeom> g;
    for (auto L : m) g.push_back(MemberGeom{L->g.nx, L->g.ny});
    return g;
}

long long tiles_for(const std::vector<MemberGeom> &m, int bx, int by, int rows) {
    long long t = 0;
    for (const MemberGeom &g : m) t += (long long)((g.nx + bx - 1) / bx) * ((g.ny + by * rows - 1) / (by * rows));
    return t;
}

long long max_tiles(const std::vector<MemberGeom> &m) {
    long long t = 0;
    for (const Shape &s : kShapes) t = std::max(t, tiles_for(m, s.bx, s.by, s.rows));
    return t;
}

size_t member_bytes(int compute) {
    return compute == BTRT_F64 ? sizeof(BatchMember<double>) : sizeof(BatchMember<float>);
}

struct BatchLayout {
    size_t off_members, off_tiles, off_tiles2, off_tilesv, off_partials, off_resid, off_tbeg, off_tcnt, off_vals,
        off_mflags, off_sync, total;
};

BatchLayout batch_layout(const std::vector<MemberGeom> &m, int compute) {
    BatchLayout b;
    const size_t n = m.size();
    const size_t T = (size_t)max_tiles(m);
    size_t off = 0;
    b.off_members = off;
    off += up256(n * member_bytes(compute));
    b.off_tiles = off;
    off += up256(T * sizeof(int4));
    b.off_tiles2 = off;
    off += up256((size_t)tiles_for(m, TbGeom::TX, TbGeom::TY, 1) * sizeof(int4));
    b.off_tilesv = off;   // vector-form tiles are four times wider: never more than T
    off += up256(T * sizeof(int4));
    b.off_partials = off;
    off += up256(T * sizeof(double));
    b.off_resid = off;
    off += up256(n * sizeof(double));
    b.off_tbeg = off;
    off += up256(n * sizeof(int));
    b.off_tcnt = off;
    off += up256(n * sizeof(int));
    b.off_vals = off;
    off += up256(n * (size_t)kMaxSliceSteps * 2 * (compute == BTRT_F64 ? 8 : 4));
    b.off_mflags = off;
    off += up256(n * sizeof(int));
    b.off_sync = off;
    off += 256;
    b.total = off;
    return b;
}

btrt_status check_members(const btrt_lattice *members, int32_t n, std::vector<btrt_lattice> &out) {
    if (!members || n <= 0) return bfail(BTRT_EINVAL, "a batch needs at least one member");
    out.assign(members, members + n);
    for (int k = 0; k < n; ++k) {
        if (!out[k]) return bfail(BTRT_EINVAL, "member %d is null", k);
        if (!out[k]->ready) return bfail(BTRT_ESTATE, "member %d is not initialised", k);
        if (out[k]->g.compute == BTRT_DF64)
            return bfail(BTRT_EINVAL, "member %d: batches take FP64 or FP32 members", k);
        if (has_phi_lo(out[k]->g))
            return bfail(BTRT_EINVAL, "member %d: batches take no double-word phi planes (BTRT_SHIFT_LOCAL_DW)", k);
        if (out[k]->g.shift == BTRT_SHIFT_LOCAL_DW_SR || has_j(out[k]->g))
            return bfail(BTRT_EINVAL, "member %d: batches take no double-word phi or first-moment planes", k);
        if (out[k]->g.compute != out[0]->g.compute || out[k]->g.storage != out[0]->g.storage ||
            shift_of(out[k]->g) != shift_of(out[0]->g))
            return bfail(BTRT_EINVAL, "member %d: all members need the same compute and storage formats and shift", k);
        for (int j = 0; j < k; ++j)
            if (out[j] == out[k]) return bfail(BTRT_EINVAL, "member %d appears twice", k);
    }
    return BTRT_OK;
}

// autotuner cache: (members, total nodes in millions, compute, storage, shift) -> shape
std::mutex g_tune_mu;
std::map<std::tuple<int, long long, int, int, int>, Shape> g_tune_cache;

// Pinned host staging for the batch tables.  Copies from pinned memory are
// asynchronous, so uploading a slice's tables never waits for the work already
// queued on the batch stream.  Blocks are shared by the process's batches and
// reused once the copy that last read a block has completed (its event).
struct PinnedBlock {
    unsigned char *p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
};
std::mutex g_pin_mu;
std::vector<PinnedBlock> g_pin_free;

PinnedBlock pin_acquire(size_t bytes) {
    {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        size_t best = g_pin_free.size();
        for (size_t k = 0; k < g_pin_free.size(); ++k)
            if (g_pin_free[k].cap >= bytes && (best == g_pin_free.size() || g_pin_free[k].cap < g_pin_free[best].cap))
                best = k;
        if (best < g_pin_free.size()) {
            PinnedBlock b = g_pin_free[best];
            g_pin_free.erase(g_pin_free.begin() + (long)best);
            return b;
        }
    }
    PinnedBlock b;
    const size_t cap = std::max<size_t>(size_t(64) << 10, (bytes + 65535) & ~size_t(65535));
    if (cudaHostAlloc(reinterpret_cast<void **>(&b.p), cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return PinnedBlock{};
    }
    if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(b.p);
        return PinnedBlock{};
    }
    b.cap = cap;
    return b;
}

void pin_release(PinnedBlock &b) {
    if (!b.p) return;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back(b);
    b = PinnedBlock{};
}

}  // namespace

struct btrt_batch_s {
    std::vector<btrt_lattice> members;
    int compute = 0, storage = 0, shift = 0;
    unsigned char *ws = nullptr;
    cudaStream_t stream = nullptr;
    BatchLayout lay{};
    Shape shape{32, 8, 1, 0};
    int ntiles = 0;
    int ntiles2 = 0;           // output tiles of the two-step form
    int ntilesv = 0;           // tiles of the vector form
    std::vector<int2> vchunks; // vector form: per launch {first member, first tile}; tiles run to the next entry
    std::vector<FoldConsts<float>> graph_lin;   // members' constants inside the captured graphs
    int grid = 0;              // persistent grid (co-resident blocks), form that takes either collision
    int grid_lin = 0;          // the same for the constant-coefficient-only form
    bool all_linear = false;   // every member takes the constant-coefficient collision and no reaction term (set per slice)
    unsigned long long wait_limit = 1ull << 24;
    unsigned int barrier_extra = 0;
    bool use_graph = true;
    bool have_resid = false;
    std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;
    cudaStream_t cap_stream = nullptr;   // the graphs are captured here (the caller's stream may be the legacy one)
    PinnedBlock stg[2];                  // staging of the table uploads, used in turn
    int stg_next = 0;
    cudaEvent_t last_ev = nullptr;       // recorded after the batch's latest work on its stream
    bool freeze = false;                 // btrt_batch_step_tol freezes the members it flags
    int last_chunk = 0, last_flips = 0;  // steps and buffer flips of the latest chunk of btrt_batch_step
    std::vector<unsigned char> host_members, host_vals;

    unsigned int *barrier() { return reinterpret_cast<unsigned int *>(ws + lay.off_sync); }
    int *err() { return reinterpret_cast<int *>(ws + lay.off_sync + 16); }

    void drop_graphs() {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
    }

    // Pinned staging of `bytes` for the next upload (nullptr if none can be had);
    // the upload's copies are followed by staged() on the batch stream.
    unsigned char *stage(size_t bytes) {
        PinnedBlock &b = stg[stg_next];
        if (b.p && b.cap < bytes) pin_release(b);
        if (!b.p) b = pin_acquire(bytes);
        if (!b.p) return nullptr;
        if (cudaEventSynchronize(b.ev) != cudaSuccess) return nullptr;   // its previous copy has read it
        return b.p;
    }
    cudaError_t staged() {
        cudaError_t e = cudaEventRecord(stg[stg_next].ev, stream);
        stg_next ^= 1;
        return e;
    }
    cudaError_t mark() {
        if (!last_ev) {
            cudaError_t e = cudaEventCreateWithFlags(&last_ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        return cudaEventRecord(last_ev, stream);
    }
};

namespace {

template <int SH, bool LIN>
void *persistent_kernel_sh(int storage) {
    switch (storage) {
    case BTRT_F32: return reinterpret_cast<void *>(&batch_kernel<float, float, SH, LIN>);
    case BTRT_F16: return reinterpret_cast<void *>(&batch_kernel<float, __half, SH, LIN>);
    case BTRT_BF16: return reinterpret_cast<void *>(&batch_kernel<float, __nv_bfloat16, SH, LIN>);
    }
    return nullptr;
}

template <bool LIN>
void *persistent_kernel_for(int compute, int storage, int shift) {
    if (compute == BTRT_F64) return reinterpret_cast<void *>(&batch_kernel<double, double, kShiftNone, LIN>);
    if (shift == kShiftLocalSR)   // 16-bit storage only
        return storage == BTRT_F16 ? reinterpret_cast<void *>(&batch_kernel<float, __half, kShiftLocalSR, LIN>)
                                   : reinterpret_cast<void *>(&batch_kernel<float, __nv_bfloat16, kShiftLocalSR, LIN>);
    return shift == kShiftLocal ? persistent_kernel_sh<kShiftLocal, LIN>(storage)
                                : persistent_kernel_sh<kShiftRef, LIN>(storage);
}

// Two-step launches of a slice of nsteps steps in the two-step form (0 in the
// others): every pair but the residual step, which runs alone.
int pairs_in_slice(btrt_batch B, int nsteps, int want_resid) {
    return B->shape.per_step == 2 ? (nsteps - (want_resid ? 1 : 0)) / 2 : 0;
}

// Tile table for the current shape; also sizes the persistent grid.
btrt_status build_tiles(btrt_batch B) {
    const Shape s = B->shape;
    std::vector<int4> tiles;
    std::vector<int> beg(B->members.size()), cnt(B->members.size());
    for (size_t m = 0; m < B->members.size(); ++m) {
        btrt_lattice L = B->members[m];
        beg[m] = (int)tiles.size();
        const int th = s.by * s.rows;
        for (int y0 = 0; y0 < L->g.ny; y0 += th)
            for (int x0 = 0; x0 < L->g.nx; x0 += s.bx) tiles.push_back(make_int4((int)m, x0, y0, 0));
        cnt[m] = (int)tiles.size() - beg[m];
    }
    B->ntiles = (int)tiles.size();
    // output tiles of the two-step form
    std::vector<int4> tiles2;
    for (size_t m = 0; m < B->members.size(); ++m) {
        btrt_lattice L = B->members[m];
        for (int y0 = 0; y0 < L->g.ny; y0 += TbGeom::TY)
            for (int x0 = 0; x0 < L->g.nx; x0 += TbGeom::TX) tiles2.push_back(make_int4((int)m, x0, y0, 0));
    }
    B->ntiles2 = (int)tiles2.size();
    // tiles of the vector form: (4 bx) x (by rows) nodes, in member order, split into
    // launches of at most kParamMembers members
    std::vector<int4> tilesv;
    B->vchunks.clear();
    for (size_t m = 0; m < B->members.size(); ++m) {
        if (m % kParamMembers == 0) B->vchunks.push_back(make_int2((int)m, (int)tilesv.size()));
        btrt_lattice L = B->members[m];
        for (int y0 = 0; y0 < L->g.ny; y0 += s.by * s.rows)
            for (int x0 = 0; x0 < L->g.nx; x0 += kVec * s.bx) tilesv.push_back(make_int4((int)m, x0, y0, 0));
    }
    B->ntilesv = (int)tilesv.size();
    // one pinned staging block, five copies in stream order (after any launch still
    // reading the previous tables)
    const struct { const void *src; size_t bytes; size_t dst; } parts[] = {
        {tiles.data(), tiles.size() * sizeof(int4), B->lay.off_tiles},
        {tiles2.data(), tiles2.size() * sizeof(int4), B->lay.off_tiles2},
        {tilesv.data(), tilesv.size() * sizeof(int4), B->lay.off_tilesv},
        {beg.data(), beg.size() * sizeof(int), B->lay.off_tbeg},
        {cnt.data(), cnt.size() * sizeof(int), B->lay.off_tcnt}};
    size_t total = 0;
    for (const auto &q : parts) total += (q.bytes + 15) & ~size_t(15);
    unsigned char *h = B->stage(total);
    if (!h) return bfail(BTRT_ECUDA, "no pinned staging memory for the tile tables");
    size_t off = 0;
    for (const auto &q : parts) {
        std::memcpy(h + off, q.src, q.bytes);
        BCUDA(cudaMemcpyAsync(B->ws + q.dst, h + off, q.bytes, cudaMemcpyHostToDevice, B->stream));
        off += (q.bytes + 15) & ~size_t(15);
    }
    BCUDA(B->staged());
    int dev = 0, sms = 0, per_sm = 0, per_sm_lin = 0;
    BCUDA(cudaGetDevice(&dev));
    BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, persistent_kernel_for<false>(B->compute, B->storage, B->shift), s.bx * s.by, 0));
    BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm_lin, persistent_kernel_for<true>(B->compute, B->storage, B->shift), s.bx * s.by, 0));
    if (per_sm < 1 || per_sm_lin < 1) return bfail(BTRT_ECUDA, "batch kernel cannot be resident");
    B->grid = per_sm * sms;
    B->grid_lin = per_sm_lin * sms;
    B->drop_graphs();
    return BTRT_OK;
}

// Member descriptors (from the members' host state) and the per-step table of
// source and wall factors, computed by the same host code as single-lattice steps.
template <typename Real>
btrt_status upload_members(btrt_batch B, int nsteps) {
    const size_t n = B->members.size();
    B->host_members.resize(n * sizeof(BatchMember<Real>));
    B->host_vals.resize(n * (size_t)nsteps * 2 * sizeof(Real));
    BatchMember<Real> *hm = reinterpret_cast<BatchMember<Real> *>(B->host_members.data());
    Real *hv = reinterpret_cast<Real *>(B->host_vals.data());
    B->all_linear = true;
    for (size_t m = 0; m < n; ++m) {
        btrt_lattice L = B->members[m];
        BatchMember<Real> d;
        std::memset(&d, 0, sizeof d);
        // parameters of the next step with buffer 0 as input; the kernel swaps per parity
        const int saved = L->cur;
        L->cur = 0;
        fill_params<Real>(L, d.p, L->step + 1, false);
        L->cur = saved;
        d.step = L->step;
        d.cur = L->cur;
        d.mode = sweep_mode(L) == kGeneral ? kGeneral : kLinear;
        B->all_linear = B->all_linear && d.mode == kLinear && d.p.src_kind != kSrcReaction;
        hm[m] = d;
        for (int k = 0; k < nsteps; ++k) {
            double sv = 0.0, wf = 1.0;
            step_scalars(L, L->step + 1 + k, false, &sv, &wf);
            hv[(m * nsteps + k) * 2] = (Real)sv;
            hv[(m * nsteps + k) * 2 + 1] = (Real)wf;
        }
    }
    const size_t mb = n * sizeof(BatchMember<Real>), vb = n * (size_t)nsteps * 2 * sizeof(Real);
    const size_t voff = (mb + 15) & ~size_t(15);
    unsigned char *h = B->stage(voff + vb);
    if (!h) return bfail(BTRT_ECUDA, "no pinned staging memory for the member tables");
    std::memcpy(h, hm, mb);
    std::memcpy(h + voff, hv, vb);
    BCUDA(cudaMemcpyAsync(B->ws + B->lay.off_members, h, mb, cudaMemcpyHostToDevice, B->stream));
    BCUDA(cudaMemcpyAsync(B->ws + B->lay.off_vals, h + voff, vb, cudaMemcpyHostToDevice, B->stream));
    BCUDA(B->staged());
    return BTRT_OK;
}

template <typename Real>
BatchArgs<Real> make_args(btrt_batch B, int nsteps, int want_resid) {
    BatchArgs<Real> a;
    std::memset(&a, 0, sizeof a);
    a.members = reinterpret_cast<const BatchMember<Real> *>(B->ws + B->lay.off_members);
    a.tiles = reinterpret_cast<const int4 *>(B->ws + B->lay.off_tiles);
    a.ntiles = B->ntiles;
    a.tiles2 = reinterpret_cast<const int4 *>(B->ws + B->lay.off_tiles2);
    a.ntiles2 = B->ntiles2;
    a.tilesv = reinterpret_cast<const int4 *>(B->ws + B->lay.off_tilesv);
    a.ntilesv = B->ntilesv;
    a.rows = B->shape.rows;
    a.nsteps = nsteps;
    a.want_resid = want_resid;
    a.tile_partials = reinterpret_cast<double *>(B->ws + B->lay.off_partials);
    a.barrier = B->barrier();
    a.err = B->err();
    a.wait_limit = B->wait_limit;
    a.barrier_extra = B->barrier_extra;
    a.step_vals = reinterpret_cast<const Real *>(B->ws + B->lay.off_vals);
    a.table_steps = nsteps;   // rows of the step table: [member][nsteps][2]
    return a;
}

template <typename Real, typename S, int SH, bool LIN>
btrt_status enqueue_form(btrt_batch B, int nsteps, int want_resid) {
    BatchArgs<Real> a = make_args<Real>(B, nsteps, want_resid);
    const dim3 block(B->shape.bx, B->shape.by);
    if (B->shape.per_step) {
        int k = 0, flip = 0;
        if constexpr (std::is_same<Real, float>::value) {
            if constexpr (!StoreSR<SH>::value) {   // the two-step form stores round-to-nearest only
                if (B->shape.per_step == 2)
                    for (int j = 0; j < pairs_in_slice(B, nsteps, want_resid); ++j, k += 2, ++flip)
                        batch_tb2_kernel<S, SH, LIN><<<(unsigned)B->ntiles2, TbGeom::THREADS, TbGeom::SMEM,
                                                       B->stream>>>(a, k, flip);
            }
            if (B->shape.per_step == 3) {
                // one parameter block per member range, reused by every step
                const BatchMember<float> *hm = reinterpret_cast<const BatchMember<float> *>(B->host_members.data());
                std::vector<BatchVecArgs> va(B->vchunks.size());
                for (size_t c = 0; c < B->vchunks.size(); ++c) {
                    std::memset(&va[c], 0, sizeof(BatchVecArgs));
                    va[c].a = a;
                    va[c].m0 = B->vchunks[c].x;
                    va[c].t0 = B->vchunks[c].y;
                    const int m1 = c + 1 < B->vchunks.size() ? B->vchunks[c + 1].x : (int)B->members.size();
                    for (int m = va[c].m0; m < m1; ++m) va[c].lin[m - va[c].m0] = hm[m].p.lin;
                }
                for (; k < nsteps - (want_resid ? 1 : 0); ++k, ++flip)
                    for (size_t c = 0; c < va.size(); ++c) {
                        const int t1 = c + 1 < B->vchunks.size() ? B->vchunks[c + 1].y : B->ntilesv;
                        batch_vec_kernel<S, SH, LIN><<<(unsigned)(t1 - va[c].t0), block, 0, B->stream>>>(va[c], k,
                                                                                                      flip);
                    }
            }
        }
        for (; k < nsteps; ++k, ++flip)
            batch_step_kernel<Real, S, SH, LIN><<<(unsigned)B->ntiles, block, 0, B->stream>>>(a, k, flip);
        BCUDA(cudaGetLastError());
        return BTRT_OK;
    }
    void *args[] = {&a};
    BCUDA(cudaMemsetAsync(B->barrier(), 0, sizeof(unsigned int), B->stream));
    BCUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(&batch_kernel<Real, S, SH, LIN>),
                                      dim3(LIN ? B->grid_lin : B->grid), block, args, 0, B->stream));
    return BTRT_OK;
}

template <typename Real, typename S, int SH>
btrt_status enqueue_typed(btrt_batch B, int nsteps, int want_resid) {
    return B->all_linear ? enqueue_form<Real, S, SH, true>(B, nsteps, want_resid)
                         : enqueue_form<Real, S, SH, false>(B, nsteps, want_resid);
}

template <int SH>
btrt_status enqueue_sh(btrt_batch B, int nsteps, int want_resid) {
    switch (B->storage) {
    case BTRT_F32: return enqueue_typed<float, float, SH>(B, nsteps, want_resid);
    case BTRT_F16: return enqueue_typed<float, __half, SH>(B, nsteps, want_resid);
    case BTRT_BF16: return enqueue_typed<float, __nv_bfloat16, SH>(B, nsteps, want_resid);
    }
    return bfail(BTRT_EINVAL, "unsupported storage format");
}

btrt_status enqueue(btrt_batch B, int nsteps, int want_resid) {
    if (B->compute == BTRT_F64) return enqueue_typed<double, double, kShiftNone>(B, nsteps, want_resid);
    if (B->shift == kShiftLocalSR)   // 16-bit storage only (checked when the batch is made)
        return B->storage == BTRT_F16 ? enqueue_typed<float, __half, kShiftLocalSR>(B, nsteps, want_resid)
                                      : enqueue_typed<float, __nv_bfloat16, kShiftLocalSR>(B, nsteps, want_resid);
    return B->shift == kShiftLocal ? enqueue_sh<kShiftLocal>(B, nsteps, want_resid)
                                   : enqueue_sh<kShiftRef>(B, nsteps, want_resid);
}

// Replay (or capture, then replay) the slice graph; falls back to direct
// launches if the launch cannot be captured.  With launch == false the graph is
// only captured and instantiated (nothing runs).
btrt_status run_slice(btrt_batch B, int nsteps, int want_resid, bool launch = true) {
    if (B->compute == BTRT_F32) {
        // the vector form's graphs hold the members' collision constants in their
        // launch parameters: a change of coefficients invalidates them
        const BatchMember<float> *hm = reinterpret_cast<const BatchMember<float> *>(B->host_members.data());
        const size_t n = B->members.size();
        bool same = B->graph_lin.size() == n;
        for (size_t m = 0; same && m < n; ++m)
            same = std::memcmp(&B->graph_lin[m], &hm[m].p.lin, sizeof(FoldConsts<float>)) == 0;
        if (!same) {
            B->drop_graphs();
            B->graph_lin.resize(n);
            for (size_t m = 0; m < n; ++m) B->graph_lin[m] = hm[m].p.lin;
        }
    }
    if (B->use_graph) {
        auto key = std::make_pair((long long)nsteps, want_resid | (B->all_linear ? 2 : 0));
        auto it = B->graphs.find(key);
        if (it == B->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            // capture on a private stream: the legacy default stream cannot be captured,
            // and the graph replays on whichever stream the batch runs on
            bool ok = B->cap_stream || cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
            const cudaStream_t run_stream = B->stream;
            if (ok) ok = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            btrt_status st = BTRT_OK;
            if (ok) {
                B->stream = B->cap_stream;   // enqueue() issues on B->stream
                st = enqueue(B, nsteps, want_resid);
                B->stream = run_stream;
                ok = cudaStreamEndCapture(B->cap_stream, &g) == cudaSuccess && st == BTRT_OK;
            }
            if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            if (!ok) {
                cudaGetLastError();
                if (ge) cudaGraphExecDestroy(ge);
                B->use_graph = false;   // capture unsupported here: launch directly from now on
                return launch ? enqueue(B, nsteps, want_resid) : BTRT_OK;
            }
            it = B->graphs.emplace(key, ge).first;
        }
        if (launch) BCUDA(cudaGraphLaunch(it->second, B->stream));
        return BTRT_OK;
    }
    return launch ? enqueue(B, nsteps, want_resid) : BTRT_OK;
}

}  // namespace

extern "C" {

size_t btrt_batch_workspace_bytes(const btrt_lattice *members, int32_t n) {
    std::vector<btrt_lattice> m;
    if (check_members(members, n, m) != BTRT_OK) return 0;
    return batch_layout(geoms_of(m), m[0]->g.compute).total;
}

size_t btrt_batch_workspace_bytes_desc(const btrt_grid_desc *descs, int32_t n) {
    if (!descs || n <= 0) {
        bfail(BTRT_EINVAL, "a batch needs at least one member");
        return 0;
    }
    std::vector<MemberGeom> g;
    for (int k = 0; k < n; ++k) {
        if (btrt_workspace_bytes(&descs[k]) == 0) return 0;   // the message says why
        if ((has_phi_lo(descs[k]) || has_j(descs[k])) && descs[k].storage != BTRT_F64 && descs[k].storage != BTRT_DF64) {
            bfail(BTRT_EINVAL, "member %d: batches take no double-word phi or first-moment planes", k);
            return 0;
        }
        if (descs[k].compute != descs[0].compute || descs[k].compute == BTRT_DF64) {
            bfail(BTRT_EINVAL, "member %d: batches take FP64 or FP32 members of one compute format", k);
            return 0;
        }
        g.push_back(MemberGeom{descs[k].nx, descs[k].ny});
    }
    return batch_layout(g, descs[0].compute).total;
}

btrt_status btrt_batch_create(const btrt_lattice *members, int32_t n, void *dev_workspace, size_t bytes,
                              void *cuda_stream, btrt_batch *out) {
    if (!out) return bfail(BTRT_EINVAL, "null output handle");
    *out = nullptr;
    std::vector<btrt_lattice> m;
    btrt_status st = check_members(members, n, m);
    if (st != BTRT_OK) return st;
    if (!dev_workspace || ((uintptr_t)dev_workspace) % 256)
        return bfail(BTRT_EINVAL, "batch workspace must be a 256-byte aligned device pointer");
    BatchLayout lay = batch_layout(geoms_of(m), m[0]->g.compute);
    if (bytes < lay.total) return bfail(BTRT_ENOMEM, "batch workspace of %zu bytes < required %zu", bytes, lay.total);
    int coop = 0, dev = 0;
    BCUDA(cudaGetDevice(&dev));
    BCUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return bfail(BTRT_ECUDA, "device does not support cooperative launches");
    btrt_batch B = new (std::nothrow) btrt_batch_s();
    if (!B) return bfail(BTRT_ENOMEM, "host allocation failed");
    B->members = m;
    B->compute = m[0]->g.compute;
    B->storage = m[0]->g.storage;
    B->shift = shift_of(m[0]->g);
    B->ws = static_cast<unsigned char *>(dev_workspace);
    B->stream = static_cast<cudaStream_t>(cuda_stream);
    B->lay = lay;
    // every member's own stream work must be ordered before the batch's
    for (auto L : m) {
        cudaError_t e = cudaStreamSynchronize(L->stream);
        if (e != cudaSuccess) {
            delete B;
            return bfail(BTRT_ECUDA, "member stream: %s", cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaMemsetAsync(B->ws + lay.off_sync, 0, 256, B->stream);
    if (e != cudaSuccess) {
        delete B;
        return bfail(BTRT_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    st = build_tiles(B);
    if (st != BTRT_OK) {
        delete B;
        return st;
    }
    for (auto L : m) L->batch_refs++;
    *out = B;
    return BTRT_OK;
}

btrt_status btrt_batch_set_tiles(btrt_batch B, int32_t block_x, int32_t block_y, int32_t rows,
                                 int32_t per_step_launch) {
    if (!B) return bfail(BTRT_EINVAL, "null batch");
    bool known = false;
    for (const Shape &s : kShapes) known |= (s.bx == block_x && s.by == block_y && s.rows == rows);
    if (!known) return bfail(BTRT_EINVAL, "tile shape %dx%dx%d is not one of the compiled candidates",
                             block_x, block_y, rows);
    if (per_step_launch < 0 || per_step_launch > 3)
        return bfail(BTRT_EINVAL, "per_step_launch must be 0, 1, 2 or 3");
    if (per_step_launch >= 2 && B->compute != BTRT_F32)
        return bfail(BTRT_EINVAL, "the two-step and vector forms serve FP32-compute batches");
    if (per_step_launch == 2 && B->shift == kShiftLocalSR)
        return bfail(BTRT_EINVAL, "the two-step form stores round-to-nearest values only (no BTRT_SHIFT_LOCAL_SR)");
    B->shape = Shape{block_x, block_y, rows, per_step_launch};
    return build_tiles(B);
}

btrt_status btrt_batch_step(btrt_batch B, int64_t nsteps, int32_t want_residual) {
    NvtxRange range("btrt_batch_step");
    if (!B) return bfail(BTRT_EINVAL, "null batch");
    if (nsteps < 0) return bfail(BTRT_EINVAL, "negative step count");
    while (nsteps > 0) {
        const int chunk = (int)std::min<int64_t>(nsteps, kMaxSliceSteps);
        const int resid = (want_residual && chunk == nsteps) ? 1 : 0;
        btrt_status st = B->compute == BTRT_F64 ? upload_members<double>(B, chunk) : upload_members<float>(B, chunk);
        if (st != BTRT_OK) return st;
        st = run_slice(B, chunk, resid);
        if (st != BTRT_OK) return st;
        // buffer flips: one per launch (a two-step launch flips once for two steps)
        const int flips = chunk - pairs_in_slice(B, chunk, resid);
        if (resid) {
            member_residual<<<(unsigned)B->members.size(), 256, 0, B->stream>>>(
                reinterpret_cast<const double *>(B->ws + B->lay.off_partials),
                reinterpret_cast<const int *>(B->ws + B->lay.off_tbeg),
                reinterpret_cast<const int *>(B->ws + B->lay.off_tcnt),
                reinterpret_cast<double *>(B->ws + B->lay.off_resid));
            BCUDA(cudaGetLastError());
            B->have_resid = true;
        }
        for (auto L : B->members) {
            L->step += chunk;
            L->cur = (L->cur + flips) & 1;
        }
        B->last_chunk = chunk;
        B->last_flips = flips;
        nsteps -= chunk;
    }
    BCUDA(B->mark());
    return BTRT_OK;
}

btrt_status btrt_batch_prepare(btrt_batch B, int64_t nsteps, int32_t want_residual) {
    NvtxRange range("btrt_batch_prepare");
    if (!B) return bfail(BTRT_EINVAL, "null batch");
    if (nsteps < 1) return bfail(BTRT_EINVAL, "btrt_batch_prepare needs at least one step");
    // the same chunks as btrt_batch_step; the member tables are uploaded again by the step
    for (int64_t left = nsteps; left > 0;) {
        const int chunk = (int)std::min<int64_t>(left, kMaxSliceSteps);
        const int resid = (want_residual && chunk == left) ? 1 : 0;
        btrt_status st = B->compute == BTRT_F64 ? upload_members<double>(B, chunk) : upload_members<float>(B, chunk);
        if (st != BTRT_OK) return st;
        st = run_slice(B, chunk, resid, false);
        if (st != BTRT_OK) return st;
        left -= chunk;
    }
    return BTRT_OK;
}

btrt_status btrt_batch_step_tol(btrt_batch B, int64_t nsteps, double tol, int32_t *done, double *resid,
                                int32_t on_device) {
    if (!B || !done) return bfail(BTRT_EINVAL, "null argument");
    if (nsteps < 1) return bfail(BTRT_EINVAL, "btrt_batch_step_tol needs at least one step");
    btrt_status st = btrt_batch_step(B, nsteps, 1);
    if (st != BTRT_OK) return st;
    const int n = (int)B->members.size();
    int *dflags = on_device ? done : reinterpret_cast<int *>(B->ws + B->lay.off_mflags);
    double *dres = reinterpret_cast<double *>(B->ws + B->lay.off_resid);
    double *rout = on_device ? resid : dres;   // host copies come from the residual array itself
    const unsigned grid = (unsigned)((n + 255) / 256);
    const int fz = B->freeze ? 1 : 0;
    if (B->compute == BTRT_F64)
        member_done<double><<<grid, 256, 0, B->stream>>>(
            reinterpret_cast<const BatchMember<double> *>(B->ws + B->lay.off_members), dres, n, tol, dflags, rout, fz,
            B->last_chunk, B->last_flips);
    else
        member_done<float><<<grid, 256, 0, B->stream>>>(
            reinterpret_cast<const BatchMember<float> *>(B->ws + B->lay.off_members), dres, n, tol, dflags, rout, fz,
            B->last_chunk, B->last_flips);
    BCUDA(cudaGetLastError());
    if (!on_device) {
        BCUDA(cudaMemcpyAsync(done, dflags, n * sizeof(int), cudaMemcpyDeviceToHost, B->stream));
        if (resid) BCUDA(cudaMemcpyAsync(resid, rout, n * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
    }
    BCUDA(B->mark());
    return BTRT_OK;
}

btrt_status btrt_batch_set_freeze(btrt_batch B, int32_t enable) {
    if (!B) return bfail(BTRT_EINVAL, "null batch");
    B->freeze = enable != 0;
    return BTRT_OK;
}

btrt_status btrt_settle(btrt_lattice L, int32_t clear, int64_t *frozen_step) {
    if (!L || !frozen_step) return bfail(BTRT_EINVAL, "null argument");
    int w[4] = {0, 0, 0, 0};
    BCUDA(cudaMemcpyAsync(w, L->flags(), sizeof w, cudaMemcpyDeviceToHost, L->stream));
    BCUDA(cudaStreamSynchronize(L->stream));
    *frozen_step = -1;
    if (!(w[1] & 1)) return BTRT_OK;
    long long s = 0;
    std::memcpy(&s, &w[2], sizeof s);
    L->step = s;
    L->cur = (w[1] >> 1) & 1;
    *frozen_step = s;
    if (clear) BCUDA(cudaMemsetAsync(L->flags() + 1, 0, 3 * sizeof(int), L->stream));
    return BTRT_OK;
}

btrt_status btrt_batch_residuals(btrt_batch B, double *out_host) {
    if (!B || !out_host) return bfail(BTRT_EINVAL, "null argument");
    if (!B->have_resid) return bfail(BTRT_ESTATE, "no step with want_residual has run");
    BCUDA(cudaMemcpyAsync(out_host, B->ws + B->lay.off_resid, B->members.size() * sizeof(double),
                          cudaMemcpyDeviceToHost, B->stream));
    BCUDA(cudaStreamSynchronize(B->stream));
    return BTRT_OK;
}

btrt_status btrt_batch_check(btrt_batch B, int32_t *flags) {
    if (!B || !flags) return bfail(BTRT_EINVAL, "null argument");
    int e = 0;
    BCUDA(cudaMemcpyAsync(&e, B->err(), sizeof(int), cudaMemcpyDeviceToHost, B->stream));
    BCUDA(cudaStreamSynchronize(B->stream));
    int f = 0;
    for (auto L : B->members) {
        int v = 0;
        BCUDA(cudaMemcpyAsync(&v, L->flags(), sizeof(int), cudaMemcpyDeviceToHost, B->stream));
        BCUDA(cudaStreamSynchronize(B->stream));
        f |= v;
    }
    *flags = f | e;
    if (f & 8) return bfail(BTRT_ECUDA, "an index check of the debug build failed (flag bit 3)");
    if (e & 2) return bfail(BTRT_ETIMEOUT, "a grid barrier wait gave up (limit %llu polls)", B->wait_limit);
    if (f & 1) return bfail(BTRT_EUNSTABLE, "non-finite phi in a batch member");
    return BTRT_OK;
}

btrt_status btrt_batch_member_flags(btrt_batch B, int32_t *out_host) {
    if (!B || !out_host) return bfail(BTRT_EINVAL, "null argument");
    const int n = (int)B->members.size();
    int *dflags = reinterpret_cast<int *>(B->ws + B->lay.off_mflags);
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (B->compute == BTRT_F64)
        gather_member_flags<double><<<grid, 256, 0, B->stream>>>(
            reinterpret_cast<const BatchMember<double> *>(B->ws + B->lay.off_members), n, dflags);
    else
        gather_member_flags<float><<<grid, 256, 0, B->stream>>>(
            reinterpret_cast<const BatchMember<float> *>(B->ws + B->lay.off_members), n, dflags);
    BCUDA(cudaGetLastError());
    BCUDA(cudaMemcpyAsync(out_host, dflags, n * sizeof(int), cudaMemcpyDeviceToHost, B->stream));
    BCUDA(cudaStreamSynchronize(B->stream));
    return BTRT_OK;
}

btrt_status btrt_batch_set_wait_limit(btrt_batch B, uint64_t polls, int32_t never_release) {
    if (!B) return bfail(BTRT_EINVAL, "null batch");
    if (polls == 0) return bfail(BTRT_EINVAL, "wait limit must be positive");
    B->wait_limit = polls;
    B->barrier_extra = never_release ? 1u : 0u;
    B->drop_graphs();
    return BTRT_OK;
}

btrt_status btrt_batch_autotune(btrt_batch B, int32_t steps_per_trial, int32_t *block_x, int32_t *block_y,
                                int32_t *rows, int32_t *per_step_launch) {
    NvtxRange range("btrt_batch_autotune");
    if (!B) return bfail(BTRT_EINVAL, "null batch");
    if (steps_per_trial < 1) return bfail(BTRT_EINVAL, "steps_per_trial must be >= 1");
    long long nodes = 0;
    for (auto L : B->members) nodes += (long long)L->g.nx * L->g.ny;
    const auto key = std::make_tuple((int)B->members.size(), nodes / 1000000, B->compute, B->storage, B->shift);
    Shape best{0, 0, 0, 0};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) best = it->second;
    }
    if (best.bx == 0) {
        cudaEvent_t e0, e1;
        BCUDA(cudaEventCreate(&e0));
        BCUDA(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        for (int mode = 0; mode < (B->compute == BTRT_F32 ? kForms : 2); ++mode) {
            if (mode == 2 && B->shift == kShiftLocalSR) continue;   // no two-step form for stochastic rounding
            for (const Shape &s : kShapes) {
                btrt_status st = btrt_batch_set_tiles(B, s.bx, s.by, s.rows, mode);
                if (st != BTRT_OK) return st;
                st = btrt_batch_step(B, 1, 0);   // warm-up for this candidate
                if (st != BTRT_OK) return st;
                st = btrt_batch_prepare(B, steps_per_trial, 0);   // its graph, captured outside the timing
                if (st != BTRT_OK) return st;
                BCUDA(cudaEventRecord(e0, B->stream));
                st = btrt_batch_step(B, steps_per_trial, 0);
                if (st != BTRT_OK) return st;
                BCUDA(cudaEventRecord(e1, B->stream));
                BCUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                BCUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best = Shape{s.bx, s.by, s.rows, mode};
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    btrt_status st = btrt_batch_set_tiles(B, best.bx, best.by, best.rows, best.per_step);
    if (st != BTRT_OK) return st;
    if (block_x) *block_x = best.bx;
    if (block_y) *block_y = best.by;
    if (rows) *rows = best.rows;
    if (per_step_launch) *per_step_launch = best.per_step;
    return BTRT_OK;
}

btrt_status btrt_batch_graphs(btrt_batch B, int32_t *n_graphs) {
    if (!B || !n_graphs) return bfail(BTRT_EINVAL, "null argument");
    *n_graphs = B->use_graph ? (int32_t)B->graphs.size() : -1;
    return BTRT_OK;
}

btrt_status btrt_batch_destroy(btrt_batch B) {
    if (!B) return BTRT_OK;
    // the batch's own work only: later work queued on the stream (another batch's
    // slice) keeps running
    if (B->last_ev) cudaEventSynchronize(B->last_ev);
    for (auto &b : B->stg) {
        if (b.p) cudaEventSynchronize(b.ev);
        pin_release(b);
    }
    B->drop_graphs();
    if (B->last_ev) cudaEventDestroy(B->last_ev);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    for (auto L : B->members) L->batch_refs--;
    delete B;
    return BTRT_OK;
}

}  // extern "C"
