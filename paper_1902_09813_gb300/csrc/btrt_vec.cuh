// btrt_vec.cuh -- one step per launch of the FP32-compute sweep with vector
// memory access (the BTRT_SWEEP_VEC form).
//
// Each thread owns kVec = 4 x-consecutive nodes x0 .. x0 + 3 of one row.  The pull
// of Eq. 38 reads, for population i, the values at x - e_ix of row y - e_iy: one
// aligned vector load of the four stored values at x0 .. x0 + 3 of that row
// (64 bits for FP16/BF16 storage, 128 bits for FP32) gives them all for e_ix = 0
// and three of four otherwise; the fourth (x0 - 1 for e_ix = +1, x0 + 4 for
// e_ix = -1) is one scalar load, which L1 serves since the neighbouring thread
// loads it in its own vector.  With the local shift the eight neighbours' phi
// arrive the same way: per row y - 1, y, y + 1 one 128-bit load and two scalar
// ones.  The results leave in nine vector stores and one 128-bit phi store.  So a
// node costs about a quarter of the plain sweep's memory instructions and address
// arithmetic, while every node's arithmetic, and its order, is that of pull_node,
// collide_fold and store_value: the results equal the plain sweep's bitwise.
//
// Groups that touch the domain edge (x0 = 0, x0 + 4 > nx - 1, y = 0 or
// y = ny - 1: periodic wrap or bounce-back links) take the plain per-node path.
// Alignment: rows are padded to 64 elements and planes are whole rows, so
// x0 * sizeof(S) is a multiple of the vector size in every plane.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "btrt_sweep.cuh"

namespace btrt {

constexpr int kVec = 4;

// Four stored values in one machine word, and their conversion to and from FP32
// (exact widening; RN narrowing, as Storage<S>::pack).
template <typename S> struct Vec4;
template <> struct Vec4<__half> {
    using W = uint2;
    static __device__ __forceinline__ float get(const W &w, int k) {
        const unsigned int u = k < 2 ? w.x : w.y;
        return __half2float(__ushort_as_half((unsigned short)((k & 1) ? (u >> 16) : (u & 0xffffu))));
    }
    static __device__ __forceinline__ W put(float a, float b, float c, float d) {
        const __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
        W w;
        w.x = *reinterpret_cast<const unsigned int *>(&lo);
        w.y = *reinterpret_cast<const unsigned int *>(&hi);
        return w;
    }
    // stochastic rounding (pack_sr; pack_sr_sub with SUB) with the random bits of each value
    template <bool SUB = false>
    static __device__ __forceinline__ W put_sr(const float (&v)[kVec], unsigned int ra, unsigned int rb,
                                               unsigned int rc, unsigned int rd) {
        auto pk = [](float x, unsigned int r) {
            return (unsigned int)__half_as_ushort(SUB ? pack_sr_sub<__half>(x, r) : pack_sr<__half>(x, r));
        };
        W w;
        w.x = pk(v[0], ra) | (pk(v[1], rb) << 16);
        w.y = pk(v[2], rc) | (pk(v[3], rd) << 16);
        return w;
    }
    // four stored values, unchanged
    static __device__ __forceinline__ W pack_raw(const __half (&s)[kVec]) {
        W w;
        w.x = (unsigned int)__half_as_ushort(s[0]) | ((unsigned int)__half_as_ushort(s[1]) << 16);
        w.y = (unsigned int)__half_as_ushort(s[2]) | ((unsigned int)__half_as_ushort(s[3]) << 16);
        return w;
    }
};
template <> struct Vec4<__nv_bfloat16> {
    using W = uint2;
    static __device__ __forceinline__ float get(const W &w, int k) {
        const unsigned int u = k < 2 ? w.x : w.y;
        return __uint_as_float((k & 1) ? (u & 0xffff0000u) : (u << 16));
    }
    static __device__ __forceinline__ W put(float a, float b, float c, float d) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
        W w;
        w.x = *reinterpret_cast<const unsigned int *>(&lo);
        w.y = *reinterpret_cast<const unsigned int *>(&hi);
        return w;
    }
    template <bool SUB = false>   // BF16 has no subnormal issue: SUB changes nothing
    static __device__ __forceinline__ W put_sr(const float (&v)[kVec], unsigned int ra, unsigned int rb,
                                               unsigned int rc, unsigned int rd) {
        W w;
        w.x = (unsigned int)__bfloat16_as_ushort(pack_sr<__nv_bfloat16>(v[0], ra)) |
              ((unsigned int)__bfloat16_as_ushort(pack_sr<__nv_bfloat16>(v[1], rb)) << 16);
        w.y = (unsigned int)__bfloat16_as_ushort(pack_sr<__nv_bfloat16>(v[2], rc)) |
              ((unsigned int)__bfloat16_as_ushort(pack_sr<__nv_bfloat16>(v[3], rd)) << 16);
        return w;
    }
    static __device__ __forceinline__ W pack_raw(const __nv_bfloat16 (&s)[kVec]) {
        W w;
        w.x = (unsigned int)__bfloat16_as_ushort(s[0]) | ((unsigned int)__bfloat16_as_ushort(s[1]) << 16);
        w.y = (unsigned int)__bfloat16_as_ushort(s[2]) | ((unsigned int)__bfloat16_as_ushort(s[3]) << 16);
        return w;
    }
};
template <> struct Vec4<float> {
    using W = float4;
    static __device__ __forceinline__ float get(const W &w, int k) {
        return k == 0 ? w.x : (k == 1 ? w.y : (k == 2 ? w.z : w.w));
    }
    static __device__ __forceinline__ W put(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};

// Value k (-1 .. 4) of a row segment: k in [0, 4) from the vector, else the edge value.
template <typename S>
__device__ __forceinline__ float seg_value(const typename Vec4<S>::W &w, float edge, int k) {
    return (k < 0 || k >= kVec) ? edge : Vec4<S>::get(w, k);
}

// Resident blocks per SM the vector sweep is compiled for.  FP16/BF16 storage:
// four (64 registers, a few spilled words); measured at 8192^2 against the
// compiler's 70-96 registers (two blocks) and three blocks: manufactured solution
// 141 / 137 / 138 GLUPS with the local shift, 153 / 147 / 147 with the reference
// shift; nonlinear workload 118 / 99 / 117 and 130 / 100 / 122.  FP32 storage
// spills 160-240 bytes at 64 registers and keeps two blocks.
#ifndef BTRT_VEC_MINBLOCKS_S16
#define BTRT_VEC_MINBLOCKS_S16 4
#endif
#ifndef BTRT_VEC_MINBLOCKS_S32
#define BTRT_VEC_MINBLOCKS_S32 2
#endif
template <typename S> struct VecMinBlocks { static constexpr int value = BTRT_VEC_MINBLOCKS_S16; };
template <> struct VecMinBlocks<float> { static constexpr int value = BTRT_VEC_MINBLOCKS_S32; };

// Pull and collide the four nodes x0 .. x0 + 3 of row y when all of them are
// interior (x0 >= 1, x0 + 4 <= nx - 1, 1 <= y <= ny - 2: no pull wraps or crosses
// a wall), and hand the stored-form outputs (FP32 values before the narrowing
// to S) and the four phi to `put(outv, phi_o)`.  Returns true when a
// non-finite phi appeared.  L2ONLY: loads of data other SMs rewrite during a
// persistent launch go through L2 only (as in pull_node).
template <typename S, int SH, int MODE, int SRC, bool L2ONLY, typename Put>
__device__ __forceinline__ bool vec_interior(const SweepParams<float> &p, int x0, int y, Put &&put,
                                             const FoldConsts<float> *Lc = nullptr) {
    using W = typename Vec4<S>::W;
    constexpr bool TRIG = SRC == kSrcTrig || SRC == kSrcRuntime || SRC == kSrcRuntimeNR;
    constexpr int SC = CollShift<SH>::value;   // kShiftLocalSR pulls and collides as kShiftLocal
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    const int node = y * p.pitch + x0;

    // populations: per plane the vector of the source row and, for e_x != 0, the edge value
    W raw[9];
    float edge[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int at = i * p.plane + node - ey_of(i) * p.pitch;
        raw[i] = ldg<L2ONLY>(reinterpret_cast<const W *>(fin + BTRT_IX(p.flags, at, 9 * p.plane)));
        edge[i] = 0.f;
        if (ex_of(i) == 1) edge[i] = Storage<S>::load(ldg<L2ONLY>(fin + BTRT_IX(p.flags, at - 1, 9 * p.plane)));
        if (ex_of(i) == -1) edge[i] = Storage<S>::load(ldg<L2ONLY>(fin + BTRT_IX(p.flags, at + kVec, 9 * p.plane)));
    }
    // phi^{n-1}: own row always; rows y - 1, y + 1 and the row edges for the local shift
    float ph[3][kVec + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (SC != kShiftLocal && r != 1) continue;
        const int at = node + (r - 1) * p.pitch;
        const float4 m = ldg<L2ONLY>(reinterpret_cast<const float4 *>(p.phi_in + BTRT_IX(p.flags, at, p.plane)));
        ph[r][1] = m.x;
        ph[r][2] = m.y;
        ph[r][3] = m.z;
        ph[r][4] = m.w;
        if constexpr (SC == kShiftLocal) {
            ph[r][0] = ldg<L2ONLY>(p.phi_in + BTRT_IX(p.flags, at - 1, p.plane));
            ph[r][kVec + 1] = ldg<L2ONLY>(p.phi_in + BTRT_IX(p.flags, at + kVec, p.plane));
        }
    }

    constexpr bool MOMENT = PullShift<SH>::value == kShiftMomentSR;
    bool bad = false;
    float outv[9][kVec];
    float phi_o[kVec];
    S jxo[kVec], jyo[kVec];   // the first moments stored by the first-moment form
#pragma unroll
    for (int v = 0; v < kVec; ++v) {
        const int x = x0 + v;
        const float phi_prev = ph[1][v + 1];
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = seg_value<S>(raw[i], edge[i], v - ex_of(i));
        if constexpr (DevScaled<S, SH>::value) {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] *= 1.f / kSrScaleF16;
        }
        if constexpr (SC == kShiftLocal) {
#pragma unroll
            for (int i = 1; i < 9; ++i) f[i] = fma(wgt<float>(i), ph[1 - ey_of(i)][v - ex_of(i) + 1] - phi_prev, f[i]);
        }
        if constexpr (MOMENT) {
            // the writers' first-moment terms, as pull_node adds them (scalar loads: L1 hits)
            const S *jin = static_cast<const S *>(p.j_in);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int nb = node + v - ey_of(i) * p.pitch - ex_of(i);
                const float jx = dev_load<float, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, nb, 2 * p.plane)));
                const float jy = dev_load<float, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, p.plane + nb, 2 * p.plane)));
                f[i] = fma(w3<float>(i), e_dot<float>(i, jx, jy), f[i]);
            }
        }
        float xs = 0.f, xc = 0.f;
        if (SRC == kSrcTrig || (TRIG && SRC != kSrcTrig && p.src_kind == kSrcTrig)) {
            xs = p.Xs[BTRT_IX(p.flags, x, p.nx)];
            xc = p.Xc[BTRT_IX(p.flags, x, p.nx)];
        }
        const float src = source_at<float, SRC>(p, xs, xc, y, node + v);
        const float rs = SC == kShiftLocal ? phi_prev : p.phi_ref;
        float phid;
        const float phi = collide_fold<float, MODE, SRC, SC>(p, f, rs, phi_prev, src, false, node + v, phid, Lc);
        if constexpr (MOMENT) {
            // as finish_node: the first moment stored rounded, the deviations taken from
            // w_i (phi + 3 e_i . j) with the stored j, phi rounded stochastically
            const float jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
            const float jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
            jxo[v] = j_pack<S, SH>(jx);
            jyo[v] = j_pack<S, SH>(jy);
            const float jxv = dev_load<float, S, SH>(jxo[v]), jyv = dev_load<float, S, SH>(jyo[v]);
#pragma unroll
            for (int i = 0; i < 9; ++i)
                outv[i][v] = i == 0 ? fma(-wgt<float>(i), phid, f[i])
                                    : fma(-w3<float>(i), e_dot<float>(i, jxv, jyv), fma(-wgt<float>(i), phid, f[i]));
            phi_o[v] = phi_sr(phi, phid, rs, sr_bits(sr_node_bits(p.sr_seed, node + v), 9));
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                outv[i][v] = SC == kShiftLocal ? fma(-wgt<float>(i), phid, f[i]) : f[i];
            phi_o[v] = phi;
        }
        bad |= not_finite(phi_o[v]);
    }
    if constexpr (MOMENT) {
        S *jout = static_cast<S *>(p.j_out);
        *reinterpret_cast<W *>(jout + BTRT_IX(p.flags, node, 2 * p.plane)) = Vec4<S>::pack_raw(jxo);
        *reinterpret_cast<W *>(jout + BTRT_IX(p.flags, p.plane + node, 2 * p.plane)) = Vec4<S>::pack_raw(jyo);
    }
    put(outv, phi_o);
    return bad;
}

// One step of the four nodes x0 .. x0 + 3 (those below nx) of row y, written to
// the output buffer.  Returns true when a non-finite phi appeared.  Lc: the folded
// collision constants when not p.lin (see collide_fold).
template <typename S, int SH, int MODE, int SRC, bool L2ONLY = false>
__device__ __forceinline__ bool vec_group(const SweepParams<float> &p, int x0, int y,
                                          const FoldConsts<float> *Lc = nullptr) {
    using V = Vec4<S>;
    using W = typename V::W;
    constexpr bool TRIG = SRC == kSrcTrig || SRC == kSrcRuntime || SRC == kSrcRuntimeNR;
    const bool interior = x0 >= 1 && x0 + kVec <= p.nx - 1 && y >= 1 && y <= p.ny - 2;
    if (!interior) {
        // the plain sweep's per-node path (periodic wrap, bounce-back links)
        bool bad = false;
#pragma unroll 1
        for (int v = 0; v < kVec && x0 + v < p.nx; ++v) {
            const int x = x0 + v;
            float xs = 0.f, xc = 0.f;
            if (SRC == kSrcTrig || (TRIG && SRC != kSrcTrig && p.src_kind == kSrcTrig)) {
                xs = p.Xs[BTRT_IX(p.flags, x, p.nx)];
                xc = p.Xc[BTRT_IX(p.flags, x, p.nx)];
            }
            float f[9], phi_prev;
            pull_node<float, S, SH, L2ONLY>(p, x, y, x > 0 && x < p.nx - 1, f, phi_prev);
            finish_node<float, S, SH, MODE, SRC, false>(p, x, y, xs, xc, f, phi_prev, bad, 0.f, Lc);
        }
        return bad;
    }
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const int node = y * p.pitch + x0;
    return vec_interior<S, SH, MODE, SRC, L2ONLY>(p, x0, y, [&](const float (&outv)[9][kVec], const float (&phi_o)[kVec]) {
        if constexpr (StoreSR<SH>::value) {
            unsigned int h[kVec];
#pragma unroll
            for (int v = 0; v < kVec; ++v) h[v] = sr_node_bits(p.sr_seed, node + v);
#pragma unroll
            for (int i = 0; i < 9; ++i)
                *reinterpret_cast<W *>(fout + BTRT_IX(p.flags, i * p.plane + node, 9 * p.plane)) =
                    V::template put_sr<PullShift<SH>::value == kShiftMomentSR>(
                        outv[i], sr_bits(h[0], i), sr_bits(h[1], i), sr_bits(h[2], i), sr_bits(h[3], i));
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                *reinterpret_cast<W *>(fout + BTRT_IX(p.flags, i * p.plane + node, 9 * p.plane)) =
                    V::put(outv[i][0], outv[i][1], outv[i][2], outv[i][3]);
        }
        *reinterpret_cast<float4 *>(p.phi_out + BTRT_IX(p.flags, node, p.plane)) =
            make_float4(phi_o[0], phi_o[1], phi_o[2], phi_o[3]);
    }, Lc);
}

// True when the group x0 .. x0 + 3 of row y takes the vector path (no pull wraps
// or crosses a wall).
__device__ __forceinline__ bool vec_interior_group(const SweepParams<float> &p, int x0, int y) {
    return x0 >= 1 && x0 + kVec <= p.nx - 1 && y >= 1 && y <= p.ny - 2;
}

// One step of the group x0 .. x0 + 3 of row y when it is interior (vector path,
// written to the output buffer); nothing otherwise (vec_tile_edges takes those
// nodes).  Returns true when a non-finite phi appeared.
template <typename S, int SH, int MODE, int SRC, bool L2ONLY = false>
__device__ __forceinline__ bool vec_group_inner(const SweepParams<float> &p, int x0, int y,
                                                const FoldConsts<float> *Lc = nullptr) {
    if (!vec_interior_group(p, x0, y)) return false;
    return vec_group<S, SH, MODE, SRC, L2ONLY>(p, x0, y, Lc);
}

// The nodes of the tile [tx0, tx0 + tw) x [ty0, ty0 + th) (clipped to the grid;
// tx0 a multiple of four) whose groups are not interior -- the columns 0 .. 3 and
// from the last interior group's end to nx - 1, and the whole of rows 0 and
// ny - 1 -- one node per thread of the block, by the plain sweep's per-node path.
// Spreading them over the block keeps the slow path out of the warps that run the
// vector path (a warp holding one edge group otherwise runs both paths).
template <typename S, int SH, int MODE, int SRC, bool L2ONLY = false>
__device__ __forceinline__ bool vec_tile_edges(const SweepParams<float> &p, int tx0, int ty0, int tw, int th,
                                               const FoldConsts<float> *Lc = nullptr) {
    constexpr bool TRIG = SRC == kSrcTrig || SRC == kSrcRuntime || SRC == kSrcRuntimeNR;
    // first column of the right-hand non-interior groups: groups start at multiples
    // of four, and x0 + 4 > nx - 1 leaves the vector path
    const int xr = p.nx - kVec > 0 ? (p.nx - 1) & ~(kVec - 1) : 0;
    const int xrs = max(xr, kVec);                 // [0, 4) is the left range
    // most tiles have no such node: leave at once
    if (tx0 >= kVec && tx0 + tw <= xrs && ty0 > 0 && ty0 + th < p.ny) return false;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    const int tx1 = min(tx0 + tw, p.nx), ty1 = min(ty0 + th, p.ny);
    if (tx0 >= tx1 || ty0 >= ty1) return false;
    const int l0 = tx0, l1 = min(tx1, kVec);       // left columns in the tile (empty if l0 >= l1)
    const int r0 = max(tx0, xrs), r1 = tx1;        // right columns in the tile
    const int nl = max(0, l1 - l0), nr = max(0, r1 - r0);
    const int width = tx1 - tx0;
    bool bad = false;
    auto node = [&](int x, int y) {
        float xs = 0.f, xc = 0.f;
        if (SRC == kSrcTrig || (TRIG && SRC != kSrcTrig && p.src_kind == kSrcTrig)) {
            xs = p.Xs[BTRT_IX(p.flags, x, p.nx)];
            xc = p.Xc[BTRT_IX(p.flags, x, p.nx)];
        }
        float f[9], phi_prev;
        pull_node<float, S, SH, L2ONLY>(p, x, y, x > 0 && x < p.nx - 1, f, phi_prev);
        finish_node<float, S, SH, MODE, SRC, false>(p, x, y, xs, xc, f, phi_prev, bad, 0.f, Lc);
    };
    // whole rows 0 and ny - 1, then the edge columns of the rows between
    int nedge = 0;
    const bool has_top = ty0 == 0, has_bot = ty1 == p.ny && p.ny - 1 > 0;
    nedge = (has_top ? 1 : 0) + (has_bot ? 1 : 0);
    for (int k = tid; k < nedge * width; k += nthr) {
        const int row = k / width, x = tx0 + k % width;
        const int y = (row == 0 && has_top) ? 0 : p.ny - 1;
        node(x, y);
    }
    const int iy0 = max(ty0, 1), iy1 = min(ty1, p.ny - 1);   // rows with interior groups
    const int per_row = nl + nr;
    if (per_row > 0 && iy0 < iy1) {
        const int items = (iy1 - iy0) * per_row;
        for (int k = tid; k < items; k += nthr) {
            const int y = iy0 + k / per_row, j = k % per_row;
            node(j < nl ? l0 + j : r0 + (j - nl), y);
        }
    }
    return bad;
}

// One step of one lattice, 32 x 8 threads per block: thread (tx, ty) owns nodes
// x0 = 4 (32 bx + tx) .. x0 + 3 of row y = 8 by + ty.  Never the initialising
// collision and never a residual step (the host runs those in the plain form).
template <typename S, int SH, int MODE, int SRC>
// The first-moment form (more live values) is compiled for two blocks per SM.
__global__ void __launch_bounds__(256, SH == kShiftMomentSR ? 2 : VecMinBlocks<S>::value)
    sweep_vec_kernel(const __grid_constant__ SweepParams<float> p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * kVec;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    bool bad = false;
    if (x0 < p.nx && y < p.ny) bad = vec_group_inner<S, SH, MODE, SRC>(p, x0, y);
    bad |= vec_tile_edges<S, SH, MODE, SRC>(p, blockIdx.x * blockDim.x * kVec, blockIdx.y * blockDim.y,
                                            blockDim.x * kVec, blockDim.y);
    if (bad) atomicOr(p.flags, 1);
}

// 32 x 8 threads, 128 x 8 nodes per block.
inline dim3 sweep_vec_grid(int nx, int ny) {
    const int groups = (nx + kVec - 1) / kVec;
    return dim3((unsigned)((groups + 31) / 32), (unsigned)((ny + 7) / 8), 1);
}

}  // namespace btrt
