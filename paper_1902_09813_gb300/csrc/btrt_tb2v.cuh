// btrt_tb2v.cuh -- two time steps per launch with vector memory access (the
// BTRT_SWEEP_TB2V form) for FP32 compute with FP32, FP16 or BF16 storage in
// either shifted form.
//
// The scheme of the two-step kernel (btrt_tb.cuh): a block owns an output tile of
// 32 x TY nodes, computes the first step on the tile grown by one node on every
// side and keeps it in shared memory, then the second step on the tile from
// there.  Here both steps move four x-consecutive nodes per thread:
//  - first step: the grown tile's 32 core columns in groups of four pulled from
//    global memory with the vector sweep's loads (vec_interior), its two halo
//    columns and every group that touches the domain edge node by node;
//  - the intermediate populations are kept in shared memory in the storage format
//    itself (16 bits for FP16/BF16: half the shared memory of FP32 copies), in
//    rows of 40 values whose column 4 is the tile's first, so every group of the
//    second step reads one aligned vector per plane (64 bits for 16-bit storage)
//    plus one edge value, and its phi with one 128-bit load per row;
//  - second step: groups of four written to the other buffer with vector stores.
// Per node the arithmetic, and its order, is that of the one-step sweep, so the
// results equal the plain sweep's (and the two-step kernel's) bitwise.
#pragma once

#include "btrt_tb.cuh"
#include "btrt_vec.cuh"

namespace btrt {

// Output tile height: 32 rows for 16-bit storage (30 KB of shared memory), 24 for
// FP32 storage (42 KB, within the default per-block limit).
#ifndef BTRT_TB2V_TY_S16
#define BTRT_TB2V_TY_S16 32
#endif
#ifndef BTRT_TB2V_TY_S32
#define BTRT_TB2V_TY_S32 24
#endif
template <typename S> struct Tb2vRows { static constexpr int value = BTRT_TB2V_TY_S16; };
template <> struct Tb2vRows<float> { static constexpr int value = BTRT_TB2V_TY_S32; };

template <typename S>
struct Tb2vGeom {
    static constexpr int TX = 32, TY = Tb2vRows<S>::value;   // output tile
    static constexpr int MY = TY + 2;                        // first-step rows y0 - 1 .. y0 + TY
    static constexpr int C0 = kVec;                          // local column of x0
    static constexpr int MXA = TX + 2 * kVec;                // local columns x0 - 4 .. x0 + TX + 3
    static constexpr int PL = MY * MXA;                      // values per plane
    static constexpr int GROUPS = TX / kVec;                 // column groups of a row
    static constexpr int THREADS = 256;
    static constexpr int MID_BYTES = 9 * PL * (int)sizeof(S);
    static constexpr int PHI_OFF = (MID_BYTES + 15) / 16 * 16;
    static constexpr int SMEM = PHI_OFF + PL * (int)sizeof(float);
    static_assert(SMEM <= 48 * 1024, "the vector two-step kernel's shared memory fits the default per-block limit");
    static_assert((MXA * (int)sizeof(S)) % 16 == 0 && (C0 * (int)sizeof(float)) % 16 == 0, "aligned rows");
};

// Resident blocks per SM the vector two-step kernel is compiled for.
#ifndef BTRT_TB2V_MINBLOCKS_S16
#define BTRT_TB2V_MINBLOCKS_S16 4
#endif
#ifndef BTRT_TB2V_MINBLOCKS_S32
#define BTRT_TB2V_MINBLOCKS_S32 2
#endif
template <typename S> struct Tb2vMinBlocks { static constexpr int value = BTRT_TB2V_MINBLOCKS_S16; };
template <> struct Tb2vMinBlocks<float> { static constexpr int value = BTRT_TB2V_MINBLOCKS_S32; };

// First step of one node of the grown tile (global coordinates gx, gy inside the
// domain) into shared memory at local index `at` (row * MXA + column).
template <typename S, int SH, int MODE, int SRC, typename G>
__device__ __forceinline__ void tb2v_first_node(const SweepParams<float> &pa, int gx, int gy, int at, S *mid,
                                                float *phm, bool &bad) {
    float d[9], phi_prev;
    pull_node<float, S, SH, false>(pa, gx, gy, gx > 0 && gx < pa.nx - 1, d, phi_prev);
    const int node = gy * pa.pitch + gx;
    float xs = 0.f, xc = 0.f;
    if (SRC == kSrcTrig || ((SRC == kSrcRuntime || SRC == kSrcRuntimeNR) && pa.src_kind == kSrcTrig)) {
        xs = pa.Xs[BTRT_IX(pa.flags, gx, pa.nx)];
        xc = pa.Xc[BTRT_IX(pa.flags, gx, pa.nx)];
    }
    const float src = source_at<float, SRC>(pa, xs, xc, gy, node);
    const float rs = SH == kShiftLocal ? phi_prev : pa.phi_ref;
    float phid;
    const float phi = collide_fold<float, MODE, SRC, SH>(pa, d, rs, phi_prev, src, false, node, phid);
#pragma unroll
    for (int i = 0; i < 9; ++i) mid[i * G::PL + at] = store_value<float, S, SH>(i, d[i], phid);
    phm[at] = phi;
    bad |= not_finite(phi);
}

// Second step of one node of the output tile from shared memory (the two-step
// kernel's pull), written to the output buffer.
template <typename S, int SH, int MODE, int SRC, typename G>
__device__ __forceinline__ void tb2v_second_node(const SweepParams<float> &pb, int gx, int gy, int lx, int ly,
                                                 const S *mid, const float *phm, bool &bad) {
    S *__restrict__ fout = static_cast<S *>(pb.fout);
    const float phi_prev = phm[ly * G::MXA + lx];
    float d[9];
    tb_pull<SH, S>(pb, mid, phm, G::MXA, G::MY, lx, ly, gx, gy, phi_prev, d);
    const int node = gy * pb.pitch + gx;
    float xs = 0.f, xc = 0.f;
    if (SRC == kSrcTrig || ((SRC == kSrcRuntime || SRC == kSrcRuntimeNR) && pb.src_kind == kSrcTrig)) {
        xs = pb.Xs[BTRT_IX(pb.flags, gx, pb.nx)];
        xc = pb.Xc[BTRT_IX(pb.flags, gx, pb.nx)];
    }
    const float src = source_at<float, SRC>(pb, xs, xc, gy, node);
    const float rs = SH == kShiftLocal ? phi_prev : pb.phi_ref;
    float phid;
    const float phi = collide_fold<float, MODE, SRC, SH>(pb, d, rs, phi_prev, src, false, node, phid);
#pragma unroll
    for (int i = 0; i < 9; ++i)
        fout[BTRT_IX(pb.flags, i * pb.plane + node, 9 * pb.plane)] = store_value<float, S, SH>(i, d[i], phid);
    pb.phi_out[BTRT_IX(pb.flags, node, pb.plane)] = phi;
    bad |= not_finite(phi);
}

// The two steps of the output tile with origin (x0, y0) by the whole block.
// Returns true when a non-finite phi appeared in this thread's nodes.
template <typename S, int SH, int MODE, int SRC>
__device__ __forceinline__ bool tb2v_tile(const SweepParams<float> &pa, const SweepParams<float> &pb, int x0, int y0,
                                          unsigned char *smem) {
    using G = Tb2vGeom<S>;
    using V = Vec4<S>;
    using W = typename V::W;
    constexpr bool TRIG = SRC == kSrcTrig || SRC == kSrcRuntime || SRC == kSrcRuntimeNR;
    S *mid = reinterpret_cast<S *>(smem);                       // [9][MY][MXA]: after the first step
    float *phm = reinterpret_cast<float *>(smem + G::PHI_OFF);   // [MY][MXA]: phi^{n+1}
    bool bad = false;

    // first step: core groups of four (GROUPS per row), then the two halo columns
    constexpr int NCORE = G::GROUPS * G::MY;
    for (int k = threadIdx.x; k < NCORE + 2 * G::MY; k += G::THREADS) {
        if (k < NCORE) {
            const int my = k / G::GROUPS, g = k % G::GROUPS;
            int gy = y0 - 1 + my;
            if (!tb_coord(gy, pa.ny, pa.hbb_y)) continue;   // beyond a wall: never pulled
            const int gx0 = x0 + g * kVec;
            const int at = my * G::MXA + G::C0 + g * kVec;
            if (gx0 >= 1 && gx0 + kVec <= pa.nx - 1 && gy >= 1 && gy <= pa.ny - 2) {
                bad |= vec_interior<S, SH, MODE, SRC, false>(
                    pa, gx0, gy, [&](const float (&outv)[9][kVec], const float (&phi_o)[kVec]) {
#pragma unroll
                        for (int i = 0; i < 9; ++i)
                            *reinterpret_cast<W *>(mid + i * G::PL + at) =
                                V::put(outv[i][0], outv[i][1], outv[i][2], outv[i][3]);
                        *reinterpret_cast<float4 *>(phm + at) = make_float4(phi_o[0], phi_o[1], phi_o[2], phi_o[3]);
                    });
            } else {
                // next to the domain edge: node by node, columns beyond it wrapped or skipped
#pragma unroll 1
                for (int v = 0; v < kVec; ++v) {
                    int gx = gx0 + v;
                    if (!tb_coord(gx, pa.nx, pa.hbb_x)) continue;
                    tb2v_first_node<S, SH, MODE, SRC, G>(pa, gx, gy, at + v, mid, phm, bad);
                }
            }
        } else {
            const int h = k - NCORE;
            const int my = h >> 1, side = h & 1;
            int gy = y0 - 1 + my;
            int gx = side ? x0 + G::TX : x0 - 1;
            if (!tb_coord(gy, pa.ny, pa.hbb_y) || !tb_coord(gx, pa.nx, pa.hbb_x)) continue;
            tb2v_first_node<S, SH, MODE, SRC, G>(pa, gx, gy, my * G::MXA + (side ? G::C0 + G::TX : G::C0 - 1), mid,
                                                 phm, bad);
        }
    }
    __syncthreads();

    // second step on the tile, written to the other buffer
    S *__restrict__ fout = static_cast<S *>(pb.fout);
    for (int k = threadIdx.x; k < G::GROUPS * G::TY; k += G::THREADS) {
        const int oy = k / G::GROUPS, g = k % G::GROUPS;
        const int gy = y0 + oy, gx0 = x0 + g * kVec;
        if (gy >= pb.ny || gx0 >= pb.nx) continue;
        const int ly = oy + 1, lx = G::C0 + g * kVec;
        // no link of these nodes crosses a bounce-back wall, and all four exist
        const bool inner = gx0 + kVec <= pb.nx && (!pb.hbb_x || (gx0 > 0 && gx0 + kVec < pb.nx)) &&
                           (!pb.hbb_y || (gy > 0 && gy < pb.ny - 1));
        if (!inner) {
#pragma unroll 1
            for (int v = 0; v < kVec && gx0 + v < pb.nx; ++v)
                tb2v_second_node<S, SH, MODE, SRC, G>(pb, gx0 + v, gy, lx + v, ly, mid, phm, bad);
            continue;
        }
        W raw[9];
        float edge[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int at = i * G::PL + (ly - ey_of(i)) * G::MXA + lx;
            raw[i] = *reinterpret_cast<const W *>(mid + at);
            edge[i] = 0.f;
            if (ex_of(i) == 1) edge[i] = Storage<S>::load(mid[at - 1]);
            if (ex_of(i) == -1) edge[i] = Storage<S>::load(mid[at + kVec]);
        }
        float ph[3][kVec + 2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            if (SH != kShiftLocal && r != 1) continue;
            const int at = (ly + r - 1) * G::MXA + lx;
            const float4 m = *reinterpret_cast<const float4 *>(phm + at);
            ph[r][1] = m.x;
            ph[r][2] = m.y;
            ph[r][3] = m.z;
            ph[r][4] = m.w;
            if constexpr (SH == kShiftLocal) {
                ph[r][0] = phm[at - 1];
                ph[r][kVec + 1] = phm[at + kVec];
            }
        }
        const int node = gy * pb.pitch + gx0;
        float outv[9][kVec];
        float phi_o[kVec];
#pragma unroll
        for (int v = 0; v < kVec; ++v) {
            const int x = gx0 + v;
            const float phi_prev = ph[1][v + 1];
            float f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = seg_value<S>(raw[i], edge[i], v - ex_of(i));
            if constexpr (SH == kShiftLocal) {
#pragma unroll
                for (int i = 1; i < 9; ++i)
                    f[i] = fma(wgt<float>(i), ph[1 - ey_of(i)][v - ex_of(i) + 1] - phi_prev, f[i]);
            }
            float xs = 0.f, xc = 0.f;
            if (SRC == kSrcTrig || (TRIG && SRC != kSrcTrig && pb.src_kind == kSrcTrig)) {
                xs = pb.Xs[BTRT_IX(pb.flags, x, pb.nx)];
                xc = pb.Xc[BTRT_IX(pb.flags, x, pb.nx)];
            }
            const float src = source_at<float, SRC>(pb, xs, xc, gy, node + v);
            const float rs = SH == kShiftLocal ? phi_prev : pb.phi_ref;
            float phid;
            const float phi = collide_fold<float, MODE, SRC, SH>(pb, f, rs, phi_prev, src, false, node + v, phid);
#pragma unroll
            for (int i = 0; i < 9; ++i) outv[i][v] = SH == kShiftLocal ? fma(-wgt<float>(i), phid, f[i]) : f[i];
            phi_o[v] = phi;
            bad |= not_finite(phi);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i)
            *reinterpret_cast<W *>(fout + BTRT_IX(pb.flags, i * pb.plane + node, 9 * pb.plane)) =
                V::put(outv[i][0], outv[i][1], outv[i][2], outv[i][3]);
        *reinterpret_cast<float4 *>(pb.phi_out + BTRT_IX(pb.flags, node, pb.plane)) =
            make_float4(phi_o[0], phi_o[1], phi_o[2], phi_o[3]);
    }
    return bad;
}

template <typename S, int SH, int MODE, int SRC>
__global__ void __launch_bounds__(256, Tb2vMinBlocks<S>::value)
    sweep_tb2v_kernel(const __grid_constant__ SweepParams<float> pa, const __grid_constant__ SweepParams<float> pb,
                      int ntx) {
    extern __shared__ __align__(16) unsigned char tb2v_smem[];
    using G = Tb2vGeom<S>;
    const int x0 = (blockIdx.x % ntx) * G::TX, y0 = (blockIdx.x / ntx) * G::TY;
    if (tb2v_tile<S, SH, MODE, SRC>(pa, pb, x0, y0, tb2v_smem)) atomicOr(pb.flags, 1);
}

}  // namespace btrt
