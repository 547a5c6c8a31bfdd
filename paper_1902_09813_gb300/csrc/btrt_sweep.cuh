// btrt_sweep.cuh -- device side of the fused B-TriRT D2Q9 stream-and-collide sweep.
//
// Lattice units throughout (c = 1, cs^2 = 1/3): B^ = B dt/dx, A^ = A dt/dx^2,
// S^ = S dt.  One thread owns one node; the sweep pulls f_i(x) = f_i^+(x - e_i)
// (Eq. 38 read backwards), replaces links that cross a bounce-back wall by
// -f_opp^+(x) + 2 w_i phi_w (Eqs. 54-56), collides with the moment-space form
// of Eq. 6 (Eqs. 94-95, 99) and writes f^+ back to its own slot of the other
// buffer, together with phi.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace btrt {

// ---------------------------------------------------------------- storage types
template <typename S> struct Storage;
template <> struct Storage<double> {
    static __device__ __forceinline__ double load(double v) { return v; }
    static __device__ __forceinline__ double pack(double v) { return v; }
};
template <> struct Storage<float> {
    static __device__ __forceinline__ float load(float v) { return v; }
    static __device__ __forceinline__ float pack(float v) { return v; }
};
template <> struct Storage<__half> {
    static __device__ __forceinline__ float load(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half pack(float v) { return __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 pack(float v) { return __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------- parameters
// Per-lattice constants of the linear fast path (see collide_linear).
template <typename Real>
struct LinearConsts {
    Real ux, uy;           // u^ (lattice units)
    Real ux3, uy3;         // 3 k0 u^
    Real Qxx, Qxy, Qyy;    // 3 (K1 - k0 I)
    Real gx, gy;           // 3 (I - K1/2) u^
    Real k0;
    Real c0;               // w0 kap / 3,           kap = (9/2)(k2 - k0)
    Real k6, k6x3;         // -w1 kap / 6, 3 k6
    Real kd, kdx3;         // -(2/3) w5 kap, 3 kd
};

// Everything one launch of the sweep needs, passed by value.
template <typename Real>
struct SweepParams {
    const void *fin;       // post-collision populations at step n-1: 9 planes, `plane` apart
    void *fout;            // post-collision populations at step n
    Real *phi;             // phi plane: phi^{n-1} on entry, phi^n on exit
    int nx, ny;
    int pitch;             // elements between rows
    int plane;             // elements between population planes; 9 * plane < 2^31
    int hbb_x, hbb_y;      // 1: bounce-back walls on that axis, 0: periodic
    Real wref[9];          // w_i phi_ref (storage shift)

    // walls (phi_w per side; arrays may be null) and the time factor of this step
    Real wall_const[4];
    const Real *wall_arr[4];
    Real wall_fac;

    // coefficients in lattice units
    Real ux, uy, b2, c3;   // B = u phi + b2 phi^2/2 (1,1); C = phi + c3 phi^3
    Real A0xx, A0xy, A0yy, a2;
    Real k0;
    int nonlin_A;          // 1: A depends on phi -> K1, k2 built per node
    int k2_hbb;            // 1: k2 from Eq. 62 at k1_eff
    Real k2c;              // constant k2
    Real K1xx, K1xy, K1yy; // K1 when A is constant (symmetric)
    Real k2;               // k2 when A is constant
    Real cond_limit;       // FP32: tr^2/det above this -> invert in FP64

    // source
    int src_kind;          // 0 none, 1 const, 2 trig
    Real src_val;          // const: S^ ; trig: dt (3 T_n - T_{n-1}) / 2
    const Real *Xs, *Xc, *Ys, *Yc;   // trig tables: sin/cos(k x_i), alpha folded into Ys/Yc

    int first;             // 1: initialisation (f = f_eq(phi), no streaming)
    int *flags;            // bit 0: non-finite phi
    double *resid_partials;  // non-null: per-block sum of (phi^n - phi^{n-1})^2 (single-lattice sweep)
    LinearConsts<Real> lin;
};

// D2Q9 velocity components and opposite directions, order of the rows of Eq. 85.
__host__ __device__ constexpr int ex_of(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int ey_of(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }

template <typename Real> __device__ __forceinline__ Real wgt(int i) {
    return i == 0 ? Real(4) / Real(9) : (i <= 4 ? Real(1) / Real(9) : Real(1) / Real(36));
}

// 2 x even part of f^eq at the wall value: 2 w_i [phi_w + (C(phi_w) - phi_w)(3|e_i|^2 - 2)/2]
template <typename Real>
__device__ __forceinline__ Real wall_term(const SweepParams<Real> &p, int i, Real phi_w) {
    Real e2 = (i == 0) ? Real(0) : (i <= 4 ? Real(1) : Real(2));
    Real dC = p.c3 * phi_w * phi_w * phi_w;
    return Real(2) * wgt<Real>(i) * (phi_w + dC * (Real(3) * e2 - Real(2)) * Real(0.5));
}

template <typename Real>
__device__ __forceinline__ Real wall_value(const SweepParams<Real> &p, int side, int idx) {
    const Real *a = p.wall_arr[side];
    return (a ? a[idx] : p.wall_const[side]) * p.wall_fac;
}

// Division: IEEE in FP64; the fast reciprocal-based quotient (about 2 ulp) in FP32,
// well inside the FP32 path's tolerance.
__device__ __forceinline__ double quot(double a, double b) { return a / b; }
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }

// ---------------------------------------------------------------- the collision
// Moment-space form of Eq. 6 (Eqs. 94, 95, 99 with K2 = k2 Ihat), expanded back
// into populations.  f: pre-collision populations; on return f^+.
template <typename Real>
__device__ __forceinline__ void collide(const SweepParams<Real> &p, Real (&f)[9], Real phi,
                                        Real phi_prev, Real src_spatial) {
    // first and second moments of f
    const Real d57 = f[5] - f[7];
    const Real d68 = f[6] - f[8];
    const Real jx = (f[1] - f[3]) + d57 - d68;
    const Real jy = (f[2] - f[4]) + d57 + d68;
    const Real sd = (f[5] + f[7]) + (f[6] + f[8]);
    const Real pxx = (f[1] + f[3]) + sd;
    const Real pyy = (f[2] + f[4]) + sd;
    const Real pxy = (f[5] + f[7]) - (f[6] + f[8]);

    // coefficients at phi (Eq. 1 families)
    const Real hb = Real(0.5) * p.b2 * phi * phi;
    const Real Bx = p.ux * phi + hb, By = p.uy * phi + hb;
    const Real hbp = Real(0.5) * p.b2 * phi_prev * phi_prev;
    const Real dBx = Bx - (p.ux * phi_prev + hbp);
    const Real dBy = By - (p.uy * phi_prev + hbp);
    const Real Cm = p.c3 * phi * phi * phi;          // C(phi) - phi

    // first-order block K1 (Eq. 30) and k2 (Eq. 62)
    Real K1xx = p.K1xx, K1xy = p.K1xy, K1yy = p.K1yy, k2 = p.k2;
    if (p.nonlin_A) {
        const Real s3 = Real(3) * (Real(1) + p.a2 * phi * phi);
        const Real mxx = s3 * p.A0xx + Real(0.5);
        const Real mxy = s3 * p.A0xy;
        const Real myy = s3 * p.A0yy + Real(0.5);
        const Real tr = mxx + myy;
        const Real det = mxx * myy - mxy * mxy;
        if (sizeof(Real) == 4 && tr * tr > p.cond_limit * det) {
            // ill-conditioned block: invert in FP64
            const double dxx = (double)mxx, dxy = (double)mxy, dyy = (double)myy;
            const double id = 1.0 / (dxx * dyy - dxy * dxy);
            K1xx = (Real)(dyy * id);
            K1xy = (Real)(-dxy * id);
            K1yy = (Real)(dxx * id);
        } else {
            const Real id = quot(Real(1), det);
            K1xx = myy * id;
            K1xy = -mxy * id;
            K1yy = mxx * id;
        }
        if (p.k2_hbb) {
            // Eq. 62 at k1_eff = 2/tr:  k2 = 8 (k1 - 2) / (3 (k1 - 4)) = (8/3)(tr - 1) / (2 tr - 1)
            k2 = quot(Real(8) / Real(3) * (tr - Real(1)), Real(2) * tr - Real(1));
        } else {
            k2 = p.k2c;
        }
    }
    const Real k0 = p.k0;

    // non-equilibrium moments: M1 - B, M2 - C/3 I (Eq. 9 gives the equilibrium parts)
    const Real mx = jx - Bx, my = jy - By;
    const Real c3rd = (phi + Cm) * (Real(1) / Real(3));
    const Real nxx = pxx - c3rd, nyy = pyy - c3rd, nxy = pxy;

    // (K1 - k0 I) M1neq and (I - K1/2) dB (Eq. 11)
    const Real qx = (K1xx - k0) * mx + K1xy * my;
    const Real qy = K1xy * mx + (K1yy - k0) * my;
    const Real gx = (Real(1) - Real(0.5) * K1xx) * dBx - Real(0.5) * K1xy * dBy;
    const Real gy = -Real(0.5) * K1xy * dBx + (Real(1) - Real(0.5) * K1yy) * dBy;
    const Real Vx = Real(3) * (k0 * Bx - qx + gx);
    const Real Vy = Real(3) * (k0 * By - qy + gy);

    // second-order block: -(9/2)(k2 - k0) H_i
    const Real kap = Real(4.5) * (k2 - k0);
    const Real tn = (nxx + nyy) * (Real(1) / Real(3));
    const Real h0 = kap * tn;
    const Real hx = -kap * (nxx - tn);             // -(kap)(2 nxx - nyy)/3
    const Real hy = -kap * (nyy - tn);
    const Real hdp = -kap * (Real(2) * tn + Real(2) * nxy);
    const Real hdm = -kap * (Real(2) * tn - Real(2) * nxy);

    // isotropic part: k0 phi + source;  C term: k0 (3/2)(C - phi)(|e|^2 - 2/3)
    const Real a = k0 * phi + p.src_val * src_spatial;
    const Real cc = k0 * Real(1.5) * Cm;
    const Real om = Real(1) - k0;
    const Real w0 = Real(4) / Real(9), w1 = Real(1) / Real(9), w5 = Real(1) / Real(36);

    const Real a0 = a - cc * (Real(2) / Real(3)) + h0;
    const Real a1 = a + cc * (Real(1) / Real(3));
    const Real a5 = a + cc * (Real(4) / Real(3));
    Real r[9];
    r[0] = w0 * a0;
    r[1] = w1 * (a1 + hx + Vx);
    r[3] = w1 * (a1 + hx - Vx);
    r[2] = w1 * (a1 + hy + Vy);
    r[4] = w1 * (a1 + hy - Vy);
    r[5] = w5 * (a5 + hdp + Vx + Vy);
    r[7] = w5 * (a5 + hdp - Vx - Vy);
    r[6] = w5 * (a5 + hdm - Vx + Vy);
    r[8] = w5 * (a5 + hdm + Vx - Vy);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = om * f[i] + r[i];
}

// Equilibrium populations (Eq. 7) in lattice units, D = C(phi) I.
template <typename Real>
__device__ __forceinline__ void equilibrium(const SweepParams<Real> &p, Real phi, Real (&f)[9]) {
    const Real hb = Real(0.5) * p.b2 * phi * phi;
    const Real Bx = Real(3) * (p.ux * phi + hb), By = Real(3) * (p.uy * phi + hb);
    const Real cc = Real(1.5) * p.c3 * phi * phi * phi;
    const Real w0 = Real(4) / Real(9), w1 = Real(1) / Real(9), w5 = Real(1) / Real(36);
    const Real a0 = phi - cc * (Real(2) / Real(3));
    const Real a1 = phi + cc * (Real(1) / Real(3));
    const Real a5 = phi + cc * (Real(4) / Real(3));
    f[0] = w0 * a0;
    f[1] = w1 * (a1 + Bx);
    f[3] = w1 * (a1 - Bx);
    f[2] = w1 * (a1 + By);
    f[4] = w1 * (a1 - By);
    f[5] = w5 * (a5 + Bx + By);
    f[7] = w5 * (a5 - Bx - By);
    f[6] = w5 * (a5 - Bx + By);
    f[8] = w5 * (a5 + Bx - By);
}

// ---------------------------------------------------------------- linear fast path
// For B = u phi, C = phi and constant A (so constant K1 and k2) the collision
// needs far fewer operations: the equilibrium moments are linear in phi and the
// weights fold into per-lattice constants (LinearConsts, computed on the host in
// FP64).  With K2 = k2 Ihat and sigma = nxx + nyy, delta = nxx - nyy:
//   w_i (a - (9/2)(k2 - k0) H_i) = w_i a + c0 sigma            (rest)
//                                   w_i a + k6 (sigma +- 3 delta)   (axes)
//                                   w_i a + kd (sigma +- 3 nxy)     (diagonals)
// and the first-order and correction terms combine into V = 3(k0 B - (K1 - k0 I) M1neq
// + (I - K1/2) u dphi).
template <typename Real, bool K0ONE>
__device__ __forceinline__ Real collide_linear(const SweepParams<Real> &p, Real (&f)[9], Real phi_prev,
                                               Real src_spatial, bool first) {
    const LinearConsts<Real> &L = p.lin;
    const Real a13 = f[1] + f[3], a24 = f[2] + f[4];
    const Real s57 = f[5] + f[7], s68 = f[6] + f[8];
    const Real sd = s57 + s68;
    const Real phi = (f[0] + sd) + (a13 + a24);
    const Real b13 = f[1] - f[3], b24 = f[2] - f[4];
    const Real d57 = f[5] - f[7], d68 = f[6] - f[8];
    const Real jx = b13 + (d57 - d68);
    const Real jy = b24 + (d57 + d68);
    const Real pxy = s57 - s68;
    const Real sig = fma(Real(-2) / Real(3), phi, fma(Real(2), sd, a13 + a24));
    const Real del = a13 - a24;
    const Real mx = fma(-L.ux, phi, jx), my = fma(-L.uy, phi, jy);
    const Real dphi = first ? Real(0) : phi - phi_prev;
    const Real Vx = fma(L.gx, dphi, fma(L.ux3, phi, -fma(L.Qxy, my, L.Qxx * mx)));
    const Real Vy = fma(L.gy, dphi, fma(L.uy3, phi, -fma(L.Qyy, my, L.Qxy * mx)));
    const Real a = K0ONE ? fma(p.src_val, src_spatial, phi) : fma(p.src_val, src_spatial, L.k0 * phi);
    const Real w0 = Real(4) / Real(9), w1 = Real(1) / Real(9), w5 = Real(1) / Real(36);
    Real r[9];
    r[0] = fma(L.c0, sig, w0 * a);
    const Real k6s = L.k6 * sig;
    const Real hx = fma(L.k6x3, del, k6s), hy = fma(-L.k6x3, del, k6s);
    const Real wa1 = w1 * a;
    const Real A1 = wa1 + hx, A2 = wa1 + hy;
    r[1] = fma(w1, Vx, A1);
    r[3] = fma(-w1, Vx, A1);
    r[2] = fma(w1, Vy, A2);
    r[4] = fma(-w1, Vy, A2);
    const Real kds = L.kd * sig;
    const Real hp = fma(L.kdx3, pxy, kds), hm = fma(-L.kdx3, pxy, kds);
    const Real wa5 = w5 * a;
    const Real P = wa5 + hp, M = wa5 + hm;
    const Real Vp = Vx + Vy, Vm = Vx - Vy;
    r[5] = fma(w5, Vp, P);
    r[7] = fma(-w5, Vp, P);
    r[6] = fma(-w5, Vm, M);
    r[8] = fma(w5, Vm, M);
    if (K0ONE) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = r[i];
    } else {
        const Real om = Real(1) - L.k0;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fma(om, f[i], r[i]);
    }
    return phi;
}

// Non-finite test without touching the FP64 pipe: exponent field all ones.
__device__ __forceinline__ bool not_finite(double v) {
    return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool not_finite(float v) {
    return (__float_as_int(v) & 0x7f800000) == 0x7f800000;
}

// ---------------------------------------------------------------- the sweep kernel
// MODE: kGeneral (every coefficient family, runtime flags), kLinear (B = u phi,
// C = phi, A constant; any k0), kLinearK0One (the same with k0 = 1).
enum { kGeneral = 0, kLinear = 1, kLinearK0One = 2 };
// Nodes per thread of the single-lattice sweep: the FP64 sweep is ALU-bound and
// amortises per-thread set-up over a column of 4 nodes; the HBM-bound FP32
// sweeps keep one node per thread for more loads in flight.
template <typename Real> struct RowsPerThread { static constexpr int value = 1; };
template <> struct RowsPerThread<double> { static constexpr int value = 4; };

template <typename S> struct Shifted { static constexpr bool value = true; };
template <> struct Shifted<double> { static constexpr bool value = false; };  // FP64 storage is never shifted

// Global loads of data that other SMs rewrite during a persistent launch go
// through L2 only (L1 is not coherent across SMs); ordinary loads otherwise.
template <bool L2ONLY, typename T>
__device__ __forceinline__ T ldg(const T *ptr) {
    if (L2ONLY) return __ldcg(ptr);
    return *ptr;
}

// Sweep `nrows` nodes of column x, rows ybase, ybase + ystride, ...: pull,
// collide, write back.  Returns the sum over those nodes of (phi^n - phi^{n-1})^2
// when RESID (steady-state residual), else 0.  RESID is a template argument so
// that no FP64 arithmetic is ever issued (or speculated) in ordinary sweeps.
template <typename Real, typename S, int MODE, bool L2ONLY, bool RESID>
__device__ __forceinline__ double sweep_rows(const SweepParams<Real> &p, int x, int ybase, int ystride,
                                             int nrows) {
    constexpr bool kShift = Shifted<S>::value;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    Real xs = Real(0), xc = Real(0);
    if (p.src_kind == 2) { xs = p.Xs[x]; xc = p.Xc[x]; }
    const bool x_inner = (x > 0) && (x < p.nx - 1);
    double resid = 0.0;

#pragma unroll 1
    for (int r = 0; r < nrows; ++r) {
        const int y = ybase + r * ystride;
        if (y >= p.ny) break;
        const int node = y * p.pitch + x;
        Real f[9];
        const Real phi_prev = ldg<L2ONLY>(p.phi + node);
        if (p.first) {
            equilibrium(p, phi_prev, f);
        } else if (x_inner && y > 0 && y < p.ny - 1) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = Storage<S>::load(ldg<L2ONLY>(fin + (i * p.plane + node - ey_of(i) * p.pitch - ex_of(i))));
                if (kShift) f[i] += p.wref[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                int sx = x - ex_of(i), sy = y - ey_of(i);
                int wx = -1, wy = -1;   // crossed wall side, if any
                if (sx < 0) { if (p.hbb_x) wx = 0; else sx += p.nx; }
                if (sx >= p.nx) { if (p.hbb_x) wx = 1; else sx -= p.nx; }
                if (sy < 0) { if (p.hbb_y) wy = 2; else sy += p.ny; }
                if (sy >= p.ny) { if (p.hbb_y) wy = 3; else sy -= p.ny; }
                if (wx < 0 && wy < 0) {
                    f[i] = Storage<S>::load(ldg<L2ONLY>(fin + (i * p.plane + sy * p.pitch + sx)));
                    if (kShift) f[i] += p.wref[i];
                } else {
                    // the node's own population leaving towards the wall (direction opp(i))
                    // comes back as direction i (Eqs. 54-56)
                    const int o = opp_of(i);
                    Real phi_w;
                    if (wx >= 0 && wy >= 0)
                        phi_w = Real(0.5) * (wall_value(p, wx, y) + wall_value(p, wy, x));
                    else if (wy >= 0)
                        phi_w = wall_value(p, wy, x);
                    else
                        phi_w = wall_value(p, wx, y);
                    Real fo = Storage<S>::load(ldg<L2ONLY>(fin + (o * p.plane + node)));
                    if (kShift) fo += p.wref[o];
                    f[i] = -fo + wall_term(p, o, phi_w);
                }
            }
        }

        Real src = Real(0);
        if (p.src_kind == 1) src = Real(1);
        else if (p.src_kind == 2) src = fma(xs, p.Ys[y], xc * p.Yc[y]);

        Real phi;
        if (MODE == kGeneral) {
            phi = p.first ? phi_prev
                          : ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            collide(p, f, phi, p.first ? phi : phi_prev, src);
        } else {
            phi = collide_linear<Real, MODE == kLinearK0One>(p, f, phi_prev, src, p.first != 0);
        }

#pragma unroll
        for (int i = 0; i < 9; ++i) fout[i * p.plane + node] = Storage<S>::pack(kShift ? f[i] - p.wref[i] : f[i]);
        p.phi[node] = phi;
        if (not_finite(phi)) atomicOr(p.flags, 1);
        if (RESID) {
            const double d = (double)phi - (double)phi_prev;
            resid = fma(d, d, resid);
        }
    }
    return resid;
}

// One sweep of one lattice: 32 x 8 threads per block, each thread sweeps
// RowsPerThread nodes of its column, rows blockDim.y apart.
template <typename Real, typename S, int MODE>
__global__ void __launch_bounds__(256) sweep_kernel(const __grid_constant__ SweepParams<Real> p) {
    constexpr int R = RowsPerThread<Real>::value;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int ybase = blockIdx.y * blockDim.y * R + threadIdx.y;
    if (!p.resid_partials) {
        if (x < p.nx) sweep_rows<Real, S, MODE, false, false>(p, x, ybase, blockDim.y, R);
        return;
    }
    // residual step: every thread joins the fixed-order block reduction
    __shared__ double red[256];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    red[tid] = x < p.nx ? sweep_rows<Real, S, MODE, false, true>(p, x, ybase, blockDim.y, R) : 0.0;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0) p.resid_partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

}  // namespace btrt
