// btrt_tb.cuh -- two time steps per launch (temporal blocking) for FP32 compute
// with FP32, FP16 or BF16 storage in either shifted form.
//
// A block owns an output tile of TX x TY nodes.  It computes the first step on
// the tile grown by one node on every side, pulling its populations straight
// from global memory as the one-step sweep does (the grown tile's halo comes
// from L1/L2, its interior once from DRAM), and keeps the post-collision
// populations and phi in shared memory, rounded to the storage format exactly as
// a stored step would be; then it computes the second step on the tile itself
// from shared memory and writes it to the other buffer.  Per node and step the
// arithmetic, and the order of it, is that of the one-step sweep (`pull_node`,
// `pull_boundary` and `collide_fold`), so two steps here equal two ordinary
// steps bitwise.  DRAM traffic per node and step is about half of the one-step
// sweep's: the populations are read and written once per two steps, at the cost
// of recomputing the ring of first-step nodes around each tile (612 first-step
// collisions per 512 nodes).
//
// Domain edges: on a periodic axis the ring wraps (a node may appear twice in a
// small domain; every copy computes the same values); on a bounce-back axis
// nodes beyond the wall do not exist and links that cross the wall take the
// bounce-back rule of Eqs. 54-56, as in the one-step sweep.
#pragma once

#include "btrt_sweep.cuh"

namespace btrt {

// Output tile height.  Swept on GB300 at 8192^2 (GLUPS, FP32 storage MMS /
// nonlinear, FP16 local-shift MMS / nonlinear): 8 rows 116.7 / 95.8 / 107.7 / 87.8,
// 16 rows 125.3 / 111.1 / 120.6 / 97.8, 24 rows 85.5 / 114.1 / 104.2 / 103.4 (the
// constant-coefficient collision runs six blocks per SM, which then leave little L1
// for the first step's halo), 32 rows 115.7 / 108.9 / 117.4 / 101.1.  So 16 rows
// for the constant-coefficient collision and 24 for the per-node one.
#ifndef BTRT_TB2_TY
#define BTRT_TB2_TY 16
#endif
#ifndef BTRT_TB2_TY_GEN
#define BTRT_TB2_TY_GEN 24
#endif
template <int TYV>
struct TbGeomT {
    static constexpr int TX = 32, TY = TYV;        // output tile
    static constexpr int MX = TX + 2, MY = TY + 2; // first-step region
    static constexpr int THREADS = 256;
    static constexpr int MID_VALS = 9 * MY * MX;
    static constexpr int SMEM = (MID_VALS + MY * MX) * (int)sizeof(float);
    static_assert(SMEM <= 48 * 1024, "the two-step kernel's shared memory fits the default per-block limit");
};
using TbGeom = TbGeomT<BTRT_TB2_TY>;   // the batch form's tiles
template <int MODE> using TbGeomFor = TbGeomT<MODE == kGeneral ? BTRT_TB2_TY_GEN : BTRT_TB2_TY>;

// Global coordinate -> wrapped coordinate on a periodic axis; false beyond a wall.
__device__ __forceinline__ bool tb_coord(int &g, int n, int wall) {
    if (g >= 0 && g < n) return true;
    if (wall) return false;
    g = g < 0 ? g + n : g - n;
    return g >= 0 && g < n;
}

// Pull of one node from a shared-memory region: `reg` holds 9 planes of
// `rw` x `rh` stored-form values (FP32 copies of them, or the stored format T
// itself) and `phr` the phi of the same region, the node sits at (lx, ly) of the
// region; (gx, gy) are its global coordinates (inside the domain) and phi_prev
// its own phi.  The same arithmetic as `pull_node` and `pull_boundary`: links
// that cross a bounce-back wall take the node's own opposite population and the
// wall term; with the local shift a value stored relative to the writer's phi is
// moved to this node's (w_i (phi_writer - phi_prev)).
template <int SH, typename T>
__device__ __forceinline__ void tb_pull(const SweepParams<float> &p, const T *reg, const float *phr, int rw,
                                        int rh, int lx, int ly, int gx, int gy, float phi_prev, float (&d)[9]) {
    const int plane = rw * rh;
    // no link of a node one or more nodes away from every bounce-back wall crosses one
    const bool inner = (!p.hbb_x || (gx > 0 && gx < p.nx - 1)) && (!p.hbb_y || (gy > 0 && gy < p.ny - 1));
    if (inner) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            d[i] = Storage<T>::load(reg[BTRT_IX(p.flags, i * plane + (ly - ey_of(i)) * rw + (lx - ex_of(i)), 9 * plane)]);
        if constexpr (SH == kShiftLocal) {
#pragma unroll
            for (int i = 1; i < 9; ++i)
                d[i] = fma(wgt<float>(i), phr[BTRT_IX(p.flags, (ly - ey_of(i)) * rw + (lx - ex_of(i)), plane)] - phi_prev,
                           d[i]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = gx - ex_of(i), sy = gy - ey_of(i);
        int wx = -1, wy = -1;   // crossed wall side, if any
        if (p.hbb_x) {
            if (sx < 0) wx = 0;
            if (sx >= p.nx) wx = 1;
        }
        if (p.hbb_y) {
            if (sy < 0) wy = 2;
            if (sy >= p.ny) wy = 3;
        }
        if (wx < 0 && wy < 0) {
            const int at = (ly - ey_of(i)) * rw + (lx - ex_of(i));
            d[i] = Storage<T>::load(reg[BTRT_IX(p.flags, i * plane + at, 9 * plane)]);
            if constexpr (SH == kShiftLocal)
                if (i != 0) d[i] = fma(wgt<float>(i), phr[BTRT_IX(p.flags, at, plane)] - phi_prev, d[i]);
        } else {
            const int o = opp_of(i);
            float phi_w;
            if (wx >= 0 && wy >= 0)
                phi_w = 0.5f * (wall_value(p, wx, gy) + wall_value(p, wy, gx));
            else if (wy >= 0)
                phi_w = wall_value(p, wy, gx);
            else
                phi_w = wall_value(p, wx, gy);
            const float dout = Storage<T>::load(reg[BTRT_IX(p.flags, o * plane + ly * rw + lx, 9 * plane)]);
            float wt = wall_term(p, o, phi_w);
            if constexpr (SH == kShiftRef) wt = wt - 2.0f * p.wref[i];
            if constexpr (SH == kShiftLocal) wt = fma(-2.0f * wgt<float>(i), phi_prev, wt);
            d[i] = wt - dout;
        }
    }
}

// Resident blocks per SM the two-step kernel is compiled for: six (40 registers)
// for the constant-coefficient collision, five (48) for the per-node one, which
// spills at six.  On the 8192^2 FP32-storage workloads these measured 125.8 and
// 111.4 GLUPS against 113.2 and 82.0 with the compiler's 64 and 75-80 registers.
#ifndef BTRT_TB2_MINBLOCKS_LIN
#define BTRT_TB2_MINBLOCKS_LIN 6
#endif
#ifndef BTRT_TB2_MINBLOCKS_GEN
#define BTRT_TB2_MINBLOCKS_GEN 5
#endif

// The two steps of one output tile with origin (x0, y0), by the whole block
// (G::THREADS threads, G::SMEM bytes of shared memory at `smem`, G = TbGeomT<TYV>).  pa:
// parameters of the first step, pb: of the second (the same buffers: inputs of
// the first, outputs of the second).  Returns true when a non-finite phi appeared
// in this thread's nodes.  Other threads may still read `smem` when one returns:
// the caller places a barrier before reusing it.
template <typename S, int SH, int MODE, int SRC, int TYV>
__device__ __forceinline__ bool tb2_tile(const SweepParams<float> &pa, const SweepParams<float> &pb, int x0, int y0,
                                         float *smem) {
    using G = TbGeomT<TYV>;
    float *mid = smem;                       // [9][MY][MX]: after the first step (stored form)
    float *phi_m = mid + G::MID_VALS;        // [MY][MX]: phi^{n+1}
    S *__restrict__ fout = static_cast<S *>(pb.fout);
    const int tid = threadIdx.x;
    bool bad = false;

    // first step on the grown tile, pulled from global memory
    auto pull_a = [&](int k, int &gx, int &gy, float (&d)[9], float &phi_prev) -> bool {
        const int mx = k % G::MX, my = k / G::MX;
        gx = x0 - 1 + mx;
        gy = y0 - 1 + my;
        if (!tb_coord(gx, pa.nx, pa.hbb_x) || !tb_coord(gy, pa.ny, pa.hbb_y)) return false;
        pull_node<float, S, SH, false>(pa, gx, gy, gx > 0 && gx < pa.nx - 1, d, phi_prev);
        return true;
    };
    auto finish_a = [&](int k, int gx, int gy, float (&d)[9], float phi_prev) {
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
        for (int i = 0; i < 9; ++i)
            mid[i * G::MX * G::MY + k] = Storage<S>::load(store_value<float, S, SH>(i, d[i], phid));
        phi_m[k] = phi;
        bad |= not_finite(phi);
    };
    for (int k = tid; k < G::MX * G::MY; k += G::THREADS) {
        int gx, gy;
        float d[9], phi_prev;
        if (pull_a(k, gx, gy, d, phi_prev)) finish_a(k, gx, gy, d, phi_prev);
    }
    __syncthreads();

    // second step on the tile, written to the other buffer
    for (int k = tid; k < G::TX * G::TY; k += G::THREADS) {
        const int ox = k % G::TX, oy = k / G::TX;
        const int gx = x0 + ox, gy = y0 + oy;
        if (gx >= pb.nx || gy >= pb.ny) continue;
        const float phi_prev = phi_m[(oy + 1) * G::MX + ox + 1];
        float d[9];
        tb_pull<SH, float>(pb, mid, phi_m, G::MX, G::MY, ox + 1, oy + 1, gx, gy, phi_prev, d);
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
    return bad;
}

template <typename S, int SH, int MODE, int SRC>
__global__ void __launch_bounds__(256, MODE == kGeneral ? BTRT_TB2_MINBLOCKS_GEN : BTRT_TB2_MINBLOCKS_LIN)
    sweep_tb2_kernel(const __grid_constant__ SweepParams<float> pa, const __grid_constant__ SweepParams<float> pb,
                     int ntx) {
    extern __shared__ float tb_smem[];
    using G = TbGeomFor<MODE>;
    const int x0 = (blockIdx.x % ntx) * G::TX, y0 = (blockIdx.x / ntx) * G::TY;
    if (tb2_tile<S, SH, MODE, SRC, G::TY>(pa, pb, x0, y0, tb_smem)) atomicOr(pb.flags, 1);
}

}  // namespace btrt
