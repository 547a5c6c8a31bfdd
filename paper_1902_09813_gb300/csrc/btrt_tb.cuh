// btrt_tb.cuh -- two time steps per launch (temporal blocking) for FP32 compute
// with FP32 storage in the reference-shifted form.
//
// A block owns an output tile of TX x TY nodes.  It loads the populations of
// the tile grown by two nodes on every side (the inputs of both steps) and phi
// of the tile grown by one node into shared memory, computes the first step on
// the tile grown by one node (keeping its post-collision populations and phi in
// shared memory, rounded to the storage format exactly as a stored step would
// be), and the second step on the tile itself, which it writes to the other
// buffer.  Per node and step the arithmetic, and the order of it, is that of the
// one-step sweep (`pull_boundary` and `collide_fold`), so two steps here equal
// two ordinary steps bitwise.  DRAM traffic per node and step is about half of
// the one-step sweep's: the populations are read and written once per two steps
// (plus the halo, mostly served by L2), at the cost of recomputing the ring of
// first-step nodes around each tile (612 first-step collisions per 512 nodes).
//
// Domain edges: on a periodic axis the halo is loaded from the wrapped
// positions (a node may appear twice in a small domain; every copy computes the
// same values); on a bounce-back axis nodes beyond the wall do not exist and
// links that cross the wall take the bounce-back rule of Eqs. 54-56, as in the
// one-step sweep.
#pragma once

#include "btrt_sweep.cuh"

namespace btrt {

struct TbGeom {
    static constexpr int TX = 32, TY = 16;        // output tile
    static constexpr int MX = TX + 2, MY = TY + 2; // first-step region
    static constexpr int RX = TX + 4, RY = TY + 4; // input region
    static constexpr int THREADS = 256;
    static constexpr int IN_VALS = 9 * RY * RX;
    static constexpr int MID_VALS = 9 * MY * MX;
    static constexpr int SMEM = (IN_VALS + MID_VALS + 2 * MY * MX) * (int)sizeof(float);
};

// Global coordinate -> wrapped coordinate on a periodic axis; false beyond a wall.
__device__ __forceinline__ bool tb_coord(int &g, int n, int wall) {
    if (g >= 0 && g < n) return true;
    if (wall) return false;
    g = g < 0 ? g + n : g - n;
    return g >= 0 && g < n;
}

// Pull of one node from a shared-memory region: `reg` holds 9 planes of
// `rw` x `rh` values, the node sits at (lx, ly) of the region; (gx, gy) are its
// global coordinates (inside the domain).  Links that cross a bounce-back wall
// take the node's own opposite population, as `pull_boundary` does.
__device__ __forceinline__ void tb_pull(const SweepParams<float> &p, const float *reg, int rw, int rh, int lx,
                                        int ly, int gx, int gy, float (&d)[9]) {
    const int plane = rw * rh;
    // no link of a node one or more nodes away from every bounce-back wall crosses one
    const bool inner = (!p.hbb_x || (gx > 0 && gx < p.nx - 1)) && (!p.hbb_y || (gy > 0 && gy < p.ny - 1));
    if (inner) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            d[i] = reg[BTRT_IX(p.flags, i * plane + (ly - ey_of(i)) * rw + (lx - ex_of(i)), 9 * plane)];
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
            d[i] = reg[BTRT_IX(p.flags, i * plane + (ly - ey_of(i)) * rw + (lx - ex_of(i)), 9 * plane)];
        } else {
            const int o = opp_of(i);
            float phi_w;
            if (wx >= 0 && wy >= 0)
                phi_w = 0.5f * (wall_value(p, wx, gy) + wall_value(p, wy, gx));
            else if (wy >= 0)
                phi_w = wall_value(p, wy, gx);
            else
                phi_w = wall_value(p, wx, gy);
            const float dout = reg[BTRT_IX(p.flags, o * plane + ly * rw + lx, 9 * plane)];
            float wt = wall_term(p, o, phi_w);
            wt = wt - 2.0f * p.wref[i];
            d[i] = wt - dout;
        }
    }
}

template <typename S, int MODE, int SRC>
__global__ void __launch_bounds__(256) sweep_tb2_kernel(const __grid_constant__ SweepParams<float> pa,
                                                        const __grid_constant__ SweepParams<float> pb, int ntx) {
    using G = TbGeom;
    extern __shared__ float tb_smem[];
    float *in = tb_smem;                     // [9][RY][RX]: step-n populations (stored form)
    float *mid = in + G::IN_VALS;            // [9][MY][MX]: after the first step
    float *phi_p = mid + G::MID_VALS;        // [MY][MX]: phi^n on the first-step region
    float *phi_m = phi_p + G::MY * G::MX;    // [MY][MX]: phi^{n+1}
    const S *__restrict__ fin = static_cast<const S *>(pa.fin);
    S *__restrict__ fout = static_cast<S *>(pb.fout);
    const int x0 = (blockIdx.x % ntx) * G::TX, y0 = (blockIdx.x / ntx) * G::TY;
    const int tid = threadIdx.x;
    bool bad = false;

    // inputs: populations on the grown tile, phi on the first-step region
    for (int k = tid; k < G::RX * G::RY; k += G::THREADS) {
        const int lx = k % G::RX, ly = k / G::RX;
        int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        if (!tb_coord(gx, pa.nx, pa.hbb_x) || !tb_coord(gy, pa.ny, pa.hbb_y)) continue;
        const int node = gy * pa.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            in[i * G::RX * G::RY + k] = Storage<S>::load(fin[BTRT_IX(pa.flags, i * pa.plane + node, 9 * pa.plane)]);
    }
    for (int k = tid; k < G::MX * G::MY; k += G::THREADS) {
        const int lx = k % G::MX, ly = k / G::MX;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        if (!tb_coord(gx, pa.nx, pa.hbb_x) || !tb_coord(gy, pa.ny, pa.hbb_y)) continue;
        phi_p[k] = pa.phi_in[BTRT_IX(pa.flags, gy * pa.pitch + gx, pa.plane)];
    }
    __syncthreads();

    // first step on the grown tile
    for (int k = tid; k < G::MX * G::MY; k += G::THREADS) {
        const int mx = k % G::MX, my = k / G::MX;
        int gx = x0 - 1 + mx, gy = y0 - 1 + my;
        if (!tb_coord(gx, pa.nx, pa.hbb_x) || !tb_coord(gy, pa.ny, pa.hbb_y)) continue;
        float d[9];
        tb_pull(pa, in, G::RX, G::RY, mx + 1, my + 1, gx, gy, d);
        const int node = gy * pa.pitch + gx;
        float xs = 0.f, xc = 0.f;
        if (SRC == kSrcTrig) {
            xs = pa.Xs[BTRT_IX(pa.flags, gx, pa.nx)];
            xc = pa.Xc[BTRT_IX(pa.flags, gx, pa.nx)];
        }
        const float src = source_at<float, SRC>(pa, xs, xc, gy, node);
        const float phi_prev = phi_p[k];
        float phid;
        const float phi = collide_fold<float, MODE, SRC, kShiftRef>(pa, d, pa.phi_ref, phi_prev, src, false, node, phid);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            mid[i * G::MX * G::MY + k] = Storage<S>::load(store_value<float, S, kShiftRef>(i, d[i], phid));
        phi_m[k] = phi;
        bad |= not_finite(phi);
    }
    __syncthreads();

    // second step on the tile, written to the other buffer
    for (int k = tid; k < G::TX * G::TY; k += G::THREADS) {
        const int ox = k % G::TX, oy = k / G::TX;
        const int gx = x0 + ox, gy = y0 + oy;
        if (gx >= pb.nx || gy >= pb.ny) continue;
        float d[9];
        tb_pull(pb, mid, G::MX, G::MY, ox + 1, oy + 1, gx, gy, d);
        const int node = gy * pb.pitch + gx;
        float xs = 0.f, xc = 0.f;
        if (SRC == kSrcTrig) {
            xs = pb.Xs[BTRT_IX(pb.flags, gx, pb.nx)];
            xc = pb.Xc[BTRT_IX(pb.flags, gx, pb.nx)];
        }
        const float src = source_at<float, SRC>(pb, xs, xc, gy, node);
        const float phi_prev = phi_m[(oy + 1) * G::MX + ox + 1];
        float phid;
        const float phi = collide_fold<float, MODE, SRC, kShiftRef>(pb, d, pb.phi_ref, phi_prev, src, false, node, phid);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            fout[BTRT_IX(pb.flags, i * pb.plane + node, 9 * pb.plane)] = store_value<float, S, kShiftRef>(i, d[i], phid);
        pb.phi_out[BTRT_IX(pb.flags, node, pb.plane)] = phi;
        bad |= not_finite(phi);
    }
    if (bad) atomicOr(pb.flags, 1);
}

}  // namespace btrt
