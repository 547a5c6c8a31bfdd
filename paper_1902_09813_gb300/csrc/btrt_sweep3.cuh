// btrt_sweep3.cuh -- device side of the fused B-TriRT sweep on the D3Q19 lattice.
//
// Same scheme as the D2Q9 sweep in three dimensions (the appendix's D3Q19
// relaxation matrix S_f = diag(k0, K1, k2 I_6, k0 I_9) with a 3x3 first-order
// block K1 = (3 A^ + I/2)^-1 from Eq. 30, k2 from Eq. 62 at the mean rate
// 1/k1_eff = tr(K1^-1)/3, the correction of Eq. 11 and scheme-2 sources).  One
// thread owns one node; the sweep pulls f_i(x) = f_i^+(x - c_i), replaces links
// that cross bounce-back faces (one face, or two at an edge: mean of their
// values) by -f_opp^+(x) + wall term, collides in moment space and writes f^+
// and phi to the other buffers.  Lattice units (c = 1, cs^2 = 1/3).
//
// Velocity order (columns of Eq. 86): 0 rest; 1, 2 = +-x; 3, 4 = +-y; 5, 6 = +-z;
// 7 (1,1,0) 8 (-1,1,0) 9 (1,-1,0) 10 (-1,-1,0); 11 (1,0,1) 12 (-1,0,1)
// 13 (1,0,-1) 14 (-1,0,-1); 15 (0,1,1) 16 (0,-1,1) 17 (0,1,-1) 18 (0,-1,-1).
// Weights 1/3, 1/18, 1/36.  Populations are stored in the forms of the D2Q9
// sweep (unshifted FP64, or FP32/FP16/BF16 shifted by w_i phi_ref or by w_i phi
// of the writing node).
#pragma once

#include "btrt_sweep.cuh"

namespace btrt {

__host__ __device__ constexpr int cx3(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy3(int i) {
    return (i == 3 || i == 7 || i == 8 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz3(int i) {
    return (i == 5 || i == 11 || i == 12 || i == 15 || i == 16) ? 1
           : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18) ? -1 : 0;
}
// opposite directions (checked against cx3/cy3/cz3 by a static assertion below)
__host__ __device__ constexpr int opposite3(int i) {
    constexpr int o[19] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15};
    return o[i];
}
__host__ __device__ constexpr bool opposites_ok() {
    for (int i = 0; i < 19; ++i) {
        const int o = opposite3(i);
        if (cx3(o) != -cx3(i) || cy3(o) != -cy3(i) || cz3(o) != -cz3(i)) return false;
    }
    return true;
}
static_assert(opposites_ok(), "D3Q19 opposite table");

template <typename Real> __device__ __forceinline__ Real wgt3(int i) {
    return i == 0 ? cst<Real>(1, 3) : (i <= 6 ? cst<Real>(1, 18) : cst<Real>(1, 36));
}

template <typename Real>
struct Sweep3Params {
    const void *fin;       // post-collision populations of the previous step: 19 planes, `plane` apart
    void *fout;
    const Real *phi_in;    // phi of the nodes that wrote fin
    Real *phi_out;
    int nx, ny, nz;
    int pitch;             // elements between rows
    int slab;              // elements between z layers (pitch * ny)
    int plane;             // elements between population planes; 19 * plane < 2^31
    int hbb_x, hbb_y, hbb_z;
    Real wall[6];          // wall value per face (x-, x+, y-, y+, z-, z+), times wall_fac
    Real wall_fac;
    Real wref[3];          // w phi_ref for |c|^2 = 0, 1, 2 (reference shift)
    Real phi_ref;

    Real ux, uy, uz;       // B = u phi + bg phi^q
    Real bgx, bgy, bgz, bq;
    int bq2;
    int bq_n, bq_h;        // q = bq_n + bq_h / 2 when bq_n >= 0 (products and a square root)
    Real c3;               // C = phi + c3 phi^3
    Real A0[6];            // xx, xy, xz, yy, yz, zz (lattice units)
    Real a2;
    Real k0, om;           // k0, 1 - k0
    int nonlin;            // 1: A depends on phi (K1, k2 per node) or B, C nonlinear
    int k2_hbb;
    Real k2c;
    Real K1[6];            // constant K1 (symmetric) and k2 when A is constant
    Real k2;
    Real Q[3];             // diagonal of K1 - k0 I (constant K1)
    Real ka[3];            // w_i kap, kap = (9/2)(k2 - k0), for |c|^2 = 0, 1, 2 (constant k2)
    Real kak[3];           // -(3/2) k0, -k0/4, -k0/8: w_i kap = (3/2, 1/4, 1/8) k2 + kak (k2 per node)
    Real a2x3, k0x15;      // 3 a2, (3/2) k0
    int k0_one;            // 1: k0 == 1
    Real Ku[3];            // constant-coefficient fold: K1 u (B = u phi)
    Real gu[3];            //   and (I - K1/2) u
    Real cond_limit;       // FP32: tr^3 > cond_limit det -> build and invert the block in FP64
    double A0d[6], a2d;    // A0^ and a2 in FP64 for that path

    int src_kind;          // 0 none, 1 const, 3 per-node field, 4 reaction
    Real src_val;          // dt S (const), dt (3 T_n - T_{n-1}) / 2 (field), dt (reaction)
    const Real *srcF;      // field: F(x) per node (pitched)
    Real react_rate, react_exp;
    int react2;
    int re_n, re_h;

    int first;
    int *flags;            // bit 0: non-finite phi
};

template <typename Real>
__device__ __forceinline__ Real wall3_term(const Sweep3Params<Real> &p, int n2, Real phi_w) {
    // 2 x even part of f^eq at phi_w: 2 w [phi_w + (C - phi_w)(3/2)(|c|^2 - 1)]
    const Real w = n2 == 0 ? cst<Real>(1, 3) : (n2 == 1 ? cst<Real>(1, 18) : cst<Real>(1, 36));
    const Real dC = p.c3 * phi_w * phi_w * phi_w;
    return Real(2) * w * fma(dC, Real(1.5) * Real(n2 - 1), phi_w);
}

// Shifted equilibrium (Eq. 7, D = C I) for the initialising collision.
template <typename Real, int SH>
__device__ __forceinline__ void equilibrium3(const Sweep3Params<Real> &p, Real phi, Real (&f)[19]) {
    const Real g = p.bq2 ? phi * phi : pow_half(phi, p.bq, p.bq_n, p.bq_h);
    const Real Bx = Real(3) * fma(p.ux, phi, p.bgx * g);
    const Real By = Real(3) * fma(p.uy, phi, p.bgy * g);
    const Real Bz = Real(3) * fma(p.uz, phi, p.bgz * g);
    const Real Cm = Real(1.5) * p.c3 * phi * phi * phi;   // (3/2)(C - phi)
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int n2 = cx3(i) * cx3(i) + cy3(i) * cy3(i) + cz3(i) * cz3(i);
        Real v = fma(Cm, Real(n2 - 1), phi);
        v = v + Real(cx3(i)) * Bx + Real(cy3(i)) * By + Real(cz3(i)) * Bz;
        f[i] = wgt3<Real>(i) * v;
        if constexpr (SH == kShiftRef) f[i] = f[i] - p.wref[n2];
        if constexpr (SH == kShiftLocal) f[i] = fma(-wgt3<Real>(i), phi, f[i]);
    }
}

// K1 = (3 A^ + I/2)^-1 (Eq. 30) for A^ = (1 + a2 phi^2) A0^ (xx, xy, xz, yy, yz,
// zz), built and inverted in FP64 by cofactors and rounded to FP32: the FP32
// sweep's path for ill-conditioned blocks, not inlined so that well-conditioned
// nodes issue none of its FP64 instructions.
struct K1f3 {
    float v[6];
};
static __device__ __noinline__ K1f3 k1_fp64_3(double phi, double a2, const double *A0) {
    const double s3d = 3.0 + 3.0 * a2 * phi * phi;
    const double dxx = s3d * A0[0] + 0.5, dxy = s3d * A0[1], dxz = s3d * A0[2];
    const double dyy = s3d * A0[3] + 0.5, dyz = s3d * A0[4], dzz = s3d * A0[5] + 0.5;
    const double ex = dyy * dzz - dyz * dyz, exy = dxz * dyz - dxy * dzz, exz = dxy * dyz - dxz * dyy;
    const double ey = dxx * dzz - dxz * dxz, eyz = dxy * dxz - dxx * dyz, ez = dxx * dyy - dxy * dxy;
    const double id = 1.0 / (dxx * ex + dxy * exy + dxz * exz);
    return K1f3{{(float)(ex * id), (float)(exy * id), (float)(exz * id), (float)(ey * id), (float)(eyz * id),
                 (float)(ez * id)}};
}

// Moment-space collision of one node in shifted form d_i = f_i - w_i rs
// (rs = 0, phi_ref or phi^{n-1} of the node):
//   d_i^+ = (1 - k0) d_i + w_i [a + cC_i + 3 c_i.V - kap H_i],
//   a = k0 (phi - rs) + source, cC_i = (3/2) k0 (C - phi)(|c_i|^2 - 1),
//   V = k0 B - (K1 - k0 I)(M1) + (I - K1/2) dB, M1 = j - B,
//   H_i = c_i c_i : M2 - tr(M2)/3, M2 = Pi - (C - rs)/3 I, kap = (9/2)(k2 - k0).
// Returns phi; phid = phi - rs.
template <typename Real, int MODE, int SRC, int SH>
__device__ __forceinline__ Real collide3(const Sweep3Params<Real> &p, Real (&d)[19], Real rs, Real phi_prev,
                                         Real srcv, bool first, Real &phid_out) {
    // moments of the shifted populations
    const Real ax = d[1] + d[2], ay = d[3] + d[4], az = d[5] + d[6];
    const Real sxy = (d[7] + d[8]) + (d[9] + d[10]);
    const Real sxz = (d[11] + d[12]) + (d[13] + d[14]);
    const Real syz = (d[15] + d[16]) + (d[17] + d[18]);
    const Real phid = ((d[0] + (ax + ay)) + (az + sxy)) + (sxz + syz);
    phid_out = phid;
    Real phi = phid;
    if constexpr (SH != kShiftNone) phi = phid + rs;
    const Real jx = (d[1] - d[2]) + ((d[7] - d[8]) + (d[9] - d[10])) + ((d[11] - d[12]) + (d[13] - d[14]));
    const Real jy = (d[3] - d[4]) + ((d[7] + d[8]) - (d[9] + d[10])) + ((d[15] - d[16]) + (d[17] - d[18]));
    const Real jz = (d[5] - d[6]) + ((d[11] + d[12]) - (d[13] + d[14])) + ((d[15] + d[16]) - (d[17] + d[18]));
    const Real Pxx = (ax + sxy) + sxz, Pyy = (ay + sxy) + syz, Pzz = (az + sxz) + syz;
    const Real Pxy = (d[7] - d[8]) - (d[9] - d[10]);
    const Real Pxz = (d[11] - d[12]) - (d[13] - d[14]);
    const Real Pyz = (d[15] - d[16]) - (d[17] - d[18]);
    const Real dphi = first ? Real(0) : (SH == kShiftLocal ? phid : phi - phi_prev);

    // coefficients
    Real Bx, By, Bz, dBx, dBy, dBz, Cm = Real(0);
    Real Kxx, Kxy, Kxz, Kyy, Kyz, Kzz, k2 = Real(0);
    if constexpr (MODE == kGeneral) {
        const Real p2 = phi * phi;
        if (p.bq2) {
            Bx = fma(p.ux, phi, p.bgx * p2);
            By = fma(p.uy, phi, p.bgy * p2);
            Bz = fma(p.uz, phi, p.bgz * p2);
            const Real sp = phi + phi_prev;
            dBx = fma(p.bgx, sp, p.ux) * dphi;
            dBy = fma(p.bgy, sp, p.uy) * dphi;
            dBz = fma(p.bgz, sp, p.uz) * dphi;
        } else {
            const Real gq = pow_half(phi, p.bq, p.bq_n, p.bq_h);
            const Real dg = first ? Real(0) : gq - pow_half(phi_prev, p.bq, p.bq_n, p.bq_h);
            Bx = fma(p.ux, phi, p.bgx * gq);
            By = fma(p.uy, phi, p.bgy * gq);
            Bz = fma(p.uz, phi, p.bgz * gq);
            dBx = fma(p.ux, dphi, p.bgx * dg);
            dBy = fma(p.uy, dphi, p.bgy * dg);
            dBz = fma(p.uz, dphi, p.bgz * dg);
        }
        Cm = p.c3 * p2 * phi;
        // K1 = (3 A^ + I/2)^-1, A^ = (1 + a2 phi^2) A0^ (Eq. 30), symmetric 3x3 by cofactors
        const Real s3 = fma(p.a2x3, p2, Real(3));
        const Real mxx = fma(s3, p.A0[0], Real(0.5)), mxy = s3 * p.A0[1], mxz = s3 * p.A0[2];
        const Real myy = fma(s3, p.A0[3], Real(0.5)), myz = s3 * p.A0[4];
        const Real mzz = fma(s3, p.A0[5], Real(0.5));
        const Real cxx = fma(myy, mzz, -(myz * myz));
        const Real cxy = fma(mxz, myz, -(mxy * mzz));
        const Real cxz = fma(mxy, myz, -(mxz * myy));
        const Real cyy = fma(mxx, mzz, -(mxz * mxz));
        const Real cyz = fma(mxy, mxz, -(mxx * myz));
        const Real czz = fma(mxx, myy, -(mxy * mxy));
        const Real det = fma(mxx, cxx, fma(mxy, cxy, mxz * cxz));
        const Real tr = (mxx + myy) + mzz;
        bool ill = false;
        if constexpr (sizeof(Real) == 4) ill = tr * tr * tr > p.cond_limit * det;
        if (ill) {
            // ill-conditioned FP32 block: rebuilt from FP64 coefficients (FP32-rounded
            // entries carry errors the condition number amplifies), inverted in FP64
            const K1f3 k = k1_fp64_3(static_cast<double>(phi), p.a2d, p.A0d);
            Kxx = (Real)k.v[0]; Kxy = (Real)k.v[1]; Kxz = (Real)k.v[2];
            Kyy = (Real)k.v[3]; Kyz = (Real)k.v[4]; Kzz = (Real)k.v[5];
        } else {
            const Real id = quot(Real(1), det);
            Kxx = cxx * id; Kxy = cxy * id; Kxz = cxz * id;
            Kyy = cyy * id; Kyz = cyz * id; Kzz = czz * id;
        }
        // Eq. 62 at k1_eff = 3/tr:  k2 = (8/3)(2 tr - 3) / (4 tr - 3)
        k2 = p.k2_hbb ? quot(cst<Real>(8, 3) * fma(Real(2), tr, Real(-3)), fma(Real(4), tr, Real(-3))) : p.k2c;
    } else {
        Bx = By = Bz = dBx = dBy = dBz = Real(0);   // folded into Ku, gu below
        Kxx = p.K1[0]; Kxy = p.K1[1]; Kxz = p.K1[2]; Kyy = p.K1[3]; Kyz = p.K1[4]; Kzz = p.K1[5];
    }
    // V = k0 B - (K1 - k0 I)(j - B) + (I - K1/2) dB = K1 (B - j - dB/2) + k0 j + dB,
    // dB = B^n - B^{n-1} (its first form takes 36 operations, the second 18); for
    // B = u phi it is K1 u phi - (K1 - k0 I) j + (I - K1/2) u dphi
    Real Vx, Vy, Vz;
    if constexpr (MODE == kGeneral) {
        const Real ex = fma(Real(-0.5), dBx, Bx - jx);
        const Real ey = fma(Real(-0.5), dBy, By - jy);
        const Real ez = fma(Real(-0.5), dBz, Bz - jz);
        Vx = fma(Kxx, ex, fma(Kxy, ey, fma(Kxz, ez, fma(p.k0, jx, dBx))));
        Vy = fma(Kxy, ex, fma(Kyy, ey, fma(Kyz, ez, fma(p.k0, jy, dBy))));
        Vz = fma(Kxz, ex, fma(Kyz, ey, fma(Kzz, ez, fma(p.k0, jz, dBz))));
    } else {
        (void)Bx; (void)By; (void)Bz; (void)dBx; (void)dBy; (void)dBz;
        const Real qx = fma(p.Q[0], jx, fma(Kxy, jy, Kxz * jz));
        const Real qy = fma(Kxy, jx, fma(p.Q[1], jy, Kyz * jz));
        const Real qz = fma(Kxz, jx, fma(Kyz, jy, p.Q[2] * jz));
        Vx = fma(p.gu[0], dphi, fma(p.Ku[0], phi, -qx));
        Vy = fma(p.gu[1], dphi, fma(p.Ku[1], phi, -qy));
        Vz = fma(p.gu[2], dphi, fma(p.Ku[2], phi, -qz));
    }

    // second-order non-equilibrium moments M2 = Pi - (C - rs)/3 I: the deviatoric
    // parts h_a = Pi_aa - tr(Pi)/3 (C and the shift cancel from them) and
    // t3 = tr(M2)/3; H_i = c_i c_i : M2 - t3 is then h_a (axis a), t3 - h_c (the
    // face diagonals normal to axis c, from h_x + h_y + h_z = 0) +- 2 M_ab
    const Real third = cst<Real>(1, 3);
    const Real tP3 = third * ((Pxx + Pyy) + Pzz);
    const Real hx = Pxx - tP3, hy = Pyy - tP3, hz = Pzz - tP3;
    const Real cmid = MODE == kGeneral ? phid + Cm : phid;       // C - rs
    const Real t3 = fma(-third, cmid, tP3);
    // w_i kap for the three speeds, kap = (9/2)(k2 - k0)
    Real ka0, ka1, ka2;
    if constexpr (MODE == kGeneral) {
        ka0 = fma(Real(1.5), k2, p.kak[0]);
        ka1 = fma(Real(0.25), k2, p.kak[1]);
        ka2 = fma(Real(0.125), k2, p.kak[2]);
    } else {
        ka0 = p.ka[0];
        ka1 = p.ka[1];
        ka2 = p.ka[2];
    }

    Real a = MODE == kLinearK0One ? phid : p.k0 * phid;
    if constexpr (SRC == kSrcReaction || SRC == kSrcRuntime) {
        if (SRC == kSrcReaction || p.src_kind == kSrcReaction) {
            const Real Sn =
                p.react_rate * phi * (Real(1) - (p.react2 ? phi * phi : pow_half(phi, p.react_exp, p.re_n, p.re_h)));
            const Real Sp = first ? Sn
                                  : p.react_rate * phi_prev *
                                        (Real(1) - (p.react2 ? phi_prev * phi_prev
                                                             : pow_half(phi_prev, p.react_exp, p.re_n, p.re_h)));
            srcv = fma(Real(1.5), Sn, Real(-0.5) * Sp);
        }
    }
    if constexpr (SRC != kSrcNone) a = fma(p.src_val, srcv, a);
    const Real cC = MODE == kGeneral ? p.k0x15 * Cm : Real(0);   // (3/2) k0 (C - phi)

    const Real w0 = cst<Real>(1, 3), w1 = cst<Real>(1, 18), w2 = cst<Real>(1, 36);
    const Real v1 = cst<Real>(1, 6), v2 = cst<Real>(1, 12);      // 3 w1, 3 w2
    Real r[19];
    r[0] = fma(ka0, t3, w0 * (MODE == kGeneral ? a - cC : a));
    // axis directions: w1 (a - kap h_a) +- 3 w1 V_a
    const Real w1a = w1 * a;
    const Real bx = fma(-ka1, hx, w1a), by = fma(-ka1, hy, w1a), bz = fma(-ka1, hz, w1a);
    r[1] = fma(v1, Vx, bx); r[2] = fma(-v1, Vx, bx);
    r[3] = fma(v1, Vy, by); r[4] = fma(-v1, Vy, by);
    r[5] = fma(v1, Vz, bz); r[6] = fma(-v1, Vz, bz);
    // face diagonals: w2 (a + cC - kap (t3 - h_c)) -+ 2 w2 kap M_ab (2 w2 = w1) + 3 w2 c_i . V
    const Real G = fma(-ka2, t3, w2 * (MODE == kGeneral ? a + cC : a));
    const Real bxy = fma(ka2, hz, G), bxz = fma(ka2, hy, G), byz = fma(ka2, hx, G);
    const Real bxym = fma(-ka1, Pxy, bxy), bxyp = fma(ka1, Pxy, bxy);
    const Real bxzm = fma(-ka1, Pxz, bxz), bxzp = fma(ka1, Pxz, bxz);
    const Real byzm = fma(-ka1, Pyz, byz), byzp = fma(ka1, Pyz, byz);
    const Real sxyp = Vx + Vy, sxym = Vx - Vy;
    const Real sxzp = Vx + Vz, sxzm = Vx - Vz;
    const Real syzp = Vy + Vz, syzm = Vy - Vz;
    r[7] = fma(v2, sxyp, bxym);  r[10] = fma(-v2, sxyp, bxym);
    r[8] = fma(-v2, sxym, bxyp); r[9] = fma(v2, sxym, bxyp);
    r[11] = fma(v2, sxzp, bxzm); r[14] = fma(-v2, sxzp, bxzm);
    r[12] = fma(-v2, sxzm, bxzp); r[13] = fma(v2, sxzm, bxzp);
    r[15] = fma(v2, syzp, byzm); r[18] = fma(-v2, syzp, byzm);
    r[16] = fma(-v2, syzm, byzp); r[17] = fma(v2, syzm, byzp);
    // k0 = 1 (bitwise the same as (1 - k0) d_i + r_i); constant coefficients have their own variant
    if (MODE == kLinearK0One || (MODE == kGeneral && p.k0_one)) {
#pragma unroll
        for (int i = 0; i < 19; ++i) d[i] = r[i];
    } else {
#pragma unroll
        for (int i = 0; i < 19; ++i) d[i] = fma(p.om, d[i], r[i]);
    }
    return phi;
}

// Pull of a node with at least one neighbour across the domain boundary.
template <typename Real, typename S, int SH>
__device__ __forceinline__ void pull3_boundary(const Sweep3Params<Real> &p, const S *__restrict__ fin, int x, int y,
                                               int z, int node, Real phi_prev, Real (&d)[19]) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        int sx = x - cx3(i), sy = y - cy3(i), sz = z - cz3(i);
        Real wsum = Real(0);
        int crossed = 0;
        if (sx < 0) { if (p.hbb_x) { wsum += p.wall[0]; ++crossed; } else sx += p.nx; }
        if (sx >= p.nx) { if (p.hbb_x) { wsum += p.wall[1]; ++crossed; } else sx -= p.nx; }
        if (sy < 0) { if (p.hbb_y) { wsum += p.wall[2]; ++crossed; } else sy += p.ny; }
        if (sy >= p.ny) { if (p.hbb_y) { wsum += p.wall[3]; ++crossed; } else sy -= p.ny; }
        if (sz < 0) { if (p.hbb_z) { wsum += p.wall[4]; ++crossed; } else sz += p.nz; }
        if (sz >= p.nz) { if (p.hbb_z) { wsum += p.wall[5]; ++crossed; } else sz -= p.nz; }
        if (!crossed) {
            const int src = sz * p.slab + sy * p.pitch + sx;
            d[i] = Storage<S>::load(fin[BTRT_IX(p.flags, i * p.plane + src, 19 * p.plane)]);
            if constexpr (SH == kShiftLocal)
                if (i != 0) d[i] = fma(wgt3<Real>(i), p.phi_in[BTRT_IX(p.flags, src, p.plane)] - phi_prev, d[i]);
        } else {
            const int o = opposite3(i);
            const int n2 = cx3(i) * cx3(i) + cy3(i) * cy3(i) + cz3(i) * cz3(i);
            const Real phi_w = (crossed == 1 ? wsum : Real(0.5) * wsum) * p.wall_fac;
            const Real dout = Storage<S>::load(fin[BTRT_IX(p.flags, o * p.plane + node, 19 * p.plane)]);
            Real wt = wall3_term(p, n2, phi_w);
            if constexpr (SH == kShiftRef) wt = wt - Real(2) * p.wref[n2];
            if constexpr (SH == kShiftLocal) wt = fma(Real(-2) * wgt3<Real>(i), phi_prev, wt);
            d[i] = wt - dout;
        }
    }
}

template <typename Real, typename S, int SH, int MODE, int SRC>
__global__ void __launch_bounds__(256) sweep3_kernel(const __grid_constant__ Sweep3Params<Real> p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const int node = z * p.slab + y * p.pitch + x;
    const Real phi_prev = p.phi_in[BTRT_IX(p.flags, node, p.plane)];
    Real d[19];
    if (p.first) {
        equilibrium3<Real, SH>(p, phi_prev, d);
    } else if (x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1 && z > 0 && z < p.nz - 1) {
#pragma unroll
        for (int i = 0; i < 19; ++i)
            d[i] = Storage<S>::load(
                fin[BTRT_IX(p.flags, i * p.plane + node - cz3(i) * p.slab - cy3(i) * p.pitch - cx3(i), 19 * p.plane)]);
        if constexpr (SH == kShiftLocal) {
#pragma unroll
            for (int i = 1; i < 19; ++i)
                d[i] = fma(wgt3<Real>(i),
                           p.phi_in[BTRT_IX(p.flags, node - cz3(i) * p.slab - cy3(i) * p.pitch - cx3(i), p.plane)] -
                               phi_prev,
                           d[i]);
        }
    } else {
        pull3_boundary<Real, S, SH>(p, fin, x, y, z, node, phi_prev, d);
    }
    Real srcv = Real(0);
    if constexpr (SRC == kSrcConst) srcv = Real(1);
    if constexpr (SRC == kSrcField) srcv = p.srcF[BTRT_IX(p.flags, node, p.plane)];
    const Real rs = SH == kShiftLocal ? phi_prev : p.phi_ref;
    Real phid;
    const Real phi = collide3<Real, MODE, SRC, SH>(p, d, rs, phi_prev, srcv, p.first != 0, phid);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        Real v = d[i];
        if constexpr (SH == kShiftLocal) v = fma(-wgt3<Real>(i), phid, v);
        fout[BTRT_IX(p.flags, i * p.plane + node, 19 * p.plane)] = Storage<S>::pack(v);
    }
    p.phi_out[BTRT_IX(p.flags, node, p.plane)] = phi;
    if (not_finite(phi)) atomicOr(p.flags, 1);
}

}  // namespace btrt
