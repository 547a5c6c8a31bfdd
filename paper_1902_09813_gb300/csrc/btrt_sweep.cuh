// btrt_sweep.cuh -- device side of the fused B-TriRT D2Q9 stream-and-collide sweep.
//
// Lattice units throughout (c = 1, cs^2 = 1/3): B^ = B dt/dx, A^ = A dt/dx^2,
// S^ = S dt.  One thread owns one node; the sweep pulls f_i(x) = f_i^+(x - e_i)
// (Eq. 38 read backwards), replaces links that cross a bounce-back wall by
// -f_opp^+(x) + 2 w_i phi_w (Eqs. 54-56), collides with the moment-space form
// of Eq. 6 (Eqs. 94-95, 99) and writes f^+ back to its own slot of the other
// buffer, together with phi (the phi plane is double-buffered like f).
//
// Stored form of the populations (SH):
//   kShiftNone   FP64 and double-word storage: f_i itself;
//   kShiftRef    f_i - w_i phi_ref with one reference value per lattice;
//   kShiftLocal  f_i^+(x) - w_i phi^n(x), the deviation from w_i times the phi of
//                the node that wrote it.  The puller adds w_i phi^n(x - e_i) back
//                from the previous phi plane.  What is rounded to the storage
//                format is then of the size of the non-equilibrium and convective
//                parts only, not of phi itself.
//   kShiftLocalDW the same with phi kept as a double-word pair (hi + lo, FP32
//                each): the planes are never rounded to FP32, so a step that
//                changes phi by a few FP32 ulps (diffusive scaling on fine grids)
//                is not lost.  The collision and the stored deviations are those
//                of kShiftLocal; only the neighbour differences phi(x - e_i) -
//                phi(x) and the new phi take the low words along.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "btrt_dw.cuh"

namespace btrt {

// A rational constant in the compute type: folded at compile time for
// float/double, split into its double-word form for dw.
template <typename Real> __device__ __forceinline__ Real cst(int num, int den) { return Real(num) / Real(den); }
template <> __device__ __forceinline__ dw cst<dw>(int num, int den) { return dw((double)num / (double)den); }

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
template <> struct Storage<dw> {
    static __device__ __forceinline__ dw load(dw v) { return v; }
    static __device__ __forceinline__ dw pack(dw v) { return v; }
};
template <> struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 pack(float v) { return __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------- debug index checks
// Built with -DBTRT_DEBUG_BOUNDS, every global access of the sweeps checks its
// element index against the array's extent; an index outside it raises flag
// bit 3 and the access goes to element 0 instead (no fault, no trap).  The
// ordinary build compiles the check away.
#ifdef BTRT_DEBUG_BOUNDS
__device__ __forceinline__ long long checked_index(int *flags, long long idx, long long n) {
    if (idx < 0 || idx >= n) {
        atomicOr(flags, 8);
        return 0;
    }
    return idx;
}
#define BTRT_IX(flags, idx, n) ::btrt::checked_index((flags), (long long)(idx), (long long)(n))
#else
#define BTRT_IX(flags, idx, n) (idx)
#endif

// ---------------------------------------------------------------- parameters
// Per-lattice constants of the folded collision (see collide_fold), computed on
// the host in FP64.  kap = (9/2)(k2 - k0).
template <typename Real>
struct FoldConsts {
    Real Px, Py;           // K1 u^                  (constant K1)
    Real Qxx, Qxy, Qyy;    // K1 - k0 I
    Real gx, gy;           // (I - K1/2) u^
    Real Pgx, Pgy;         // K1 u^ + (I - K1/2) u^
    Real k0, om, k0x15;    // k0, 1 - k0, 1.5 k0
    Real c0;               // w0 kap / 3 = (2/3)(k2 - k0)   (constant k2)
    Real k6, k6x3;         // -w1 kap / 6 = -(k2 - k0) / 12, 3 k6
    Real c0k, k6k, k6x3k;  // -(2/3) k0, k0 / 12, k0 / 4   (k2 built per node)
    Real a2x3;             // 3 a2                   (phi-dependent coefficients)
};

// Everything one launch of the sweep needs, passed by value.
template <typename Real>
struct SweepParams {
    const void *fin;       // post-collision populations at step n-1: 9 planes, `plane` apart
    void *fout;            // post-collision populations at step n
    const Real *phi_in;    // phi^{n-1} (the phi of the nodes that wrote fin)
    Real *phi_out;         // phi^n (equal to phi_in for the initialising collision)
    const Real *phi_in_lo; // kShiftLocalDW: low words of phi_in and phi_out (null otherwise)
    Real *phi_out_lo;
    const void *j_in;      // kShiftMomentSR: first moments of the writers (planes x, y; storage format)
    void *j_out;
    int nx, ny;
    int pitch;             // elements between rows
    int plane;             // elements between population planes; 9 * plane < 2^31
    int hbb_x, hbb_y;      // 1: bounce-back walls on that axis, 0: periodic
    Real wref[9];          // w_i phi_ref (kShiftRef storage)

    // walls (phi_w per side; arrays may be null) and the time factor of this step
    Real wall_const[4];
    const Real *wall_arr[4];
    Real wall_fac;

    // coefficients in lattice units
    Real ux, uy, b2, c3;   // B = u phi + b2 (phi^q / q) d; C = phi + c3 phi^3
    Real bgx, bgy;         // b2 d / q: B = u phi + bg phi^q
    Real bq;               // q
    int bq2;               // 1: q == 2 (phi^q = phi phi)
    int bq_n, bq_h;        // q = bq_n + bq_h / 2 (bq_n >= 0) -> products and a square root; bq_n < 0: pow
    Real A0xx, A0xy, A0yy, a2;
    Real k0;
    int k0_one;            // 1: k0 == 1
    int nonlin_A;          // 1: A depends on phi -> K1, k2 built per node
    int k2_hbb;            // 1: k2 from Eq. 62 at k1_eff
    Real k2c;              // constant k2
    Real K1xx, K1xy, K1yy; // K1 when A is constant (symmetric)
    Real k2;               // k2 when A is constant
    Real cond_limit;       // FP32: tr^2/det above this -> build and invert the block in FP64
    double A0d[3], a2d;    // A0^ and a2 in FP64 for that path

    // source
    int src_kind;          // 0 none, 1 const, 2 trig, 3 per-node field, 4 reaction
    Real src_val;          // const: S^ ; trig, field: dt (3 T_n - T_{n-1}) / 2; reaction: dt
    Real react_rate, react_exp;   // reaction: S = rate phi (1 - phi^exp)
    int react2;                   // 1: exp == 2 (phi^exp = phi phi)
    int re_n, re_h;               // exp = re_n + re_h / 2 as for the flux exponent
    const Real *Xs, *Xc, *Ys, *Yc;   // trig tables: sin/cos(k x_i), alpha folded into Ys/Yc
    const Real *srcF;      // field: S(x) per node (pitched plane)
    const Real *Af;        // non-null: per-node lattice diffusion tensor, planes xx, xy, yy (`plane` apart)

    int first;             // 1: initialisation (f = f_eq(phi), no streaming)
    int *flags;            // bit 0: non-finite phi
    double *resid_partials;  // non-null: per-block sum of (phi^n - phi^{n-1})^2 (single-lattice sweep)
    Real phi_ref;          // kShiftRef: the reference value (0 otherwise)
    unsigned int sr_seed;  // stochastic rounding: the step's seed (sr_step_seed of its step index)
    FoldConsts<Real> lin;
};

// D2Q9 velocity components and opposite directions, order of the rows of Eq. 85.
__host__ __device__ constexpr int ex_of(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int ey_of(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }

template <typename Real> __device__ __forceinline__ Real wgt(int i) {
    return i == 0 ? cst<Real>(4, 9) : (i <= 4 ? cst<Real>(1, 9) : cst<Real>(1, 36));
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
    return (a ? a[BTRT_IX(p.flags, idx, side < 2 ? p.ny : p.nx)] : p.wall_const[side]) * p.wall_fac;
}

// Division: IEEE in FP64; the fast reciprocal-based quotient (about 2 ulp) in FP32,
// well inside the FP32 path's tolerance.
__device__ __forceinline__ double quot(double a, double b) { return a / b; }
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ dw quot(dw a, dw b) { return a / b; }

// ---------------------------------------------------------------- the collision
// Compiled variants: every coefficient family evaluated per node (kGeneral), or
// B = u phi, C = phi and constant A with any k0 (kLinear) or k0 = 1 (kLinearK0One).
enum { kGeneral = 0, kLinear = 1, kLinearK0One = 2 };
// Stored form of the populations (see the top of this file).
// kShiftLocalSR and kShiftLocalDWSR are kShiftLocal and kShiftLocalDW with the
// stored 16-bit deviations rounded stochastically (see pack_sr).  kShiftMomentSR
// also subtracts the writer's first-moment term: it stores f_i^+ - w_i (phi +
// 3 e_i . j), j the writer's post-collision first moment kept in two planes of the
// storage format, stochastically rounded.
enum { kShiftNone = 0, kShiftRef = 1, kShiftLocal = 2, kShiftLocalDW = 3, kShiftLocalSR = 4, kShiftLocalDWSR = 5,
       kShiftMomentSR = 6 };
// The collision and the stored deviations of the local variants are those of kShiftLocal.
template <int SH> struct CollShift {
    static constexpr int value =
        (SH == kShiftLocalDW || SH == kShiftLocalSR || SH == kShiftLocalDWSR || SH == kShiftMomentSR) ? kShiftLocal : SH;
};
// The pull (neighbour phi, low words, first moments) of each stored form.
template <int SH> struct PullShift {
    static constexpr int value = SH == kShiftLocalSR ? kShiftLocal : (SH == kShiftLocalDWSR ? kShiftLocalDW : SH);
};
// Stochastic rounding of the stored values.
template <int SH> struct StoreSR {
    static constexpr bool value = SH == kShiftLocalSR || SH == kShiftLocalDWSR || SH == kShiftMomentSR;
};
// Source kinds (compile-time SRC); kSrcRuntime decides per lattice at run time,
// kSrcRuntimeNR the same among the kinds other than the reaction term (whose
// power-law code then stays out of the kernel).
enum { kSrcNone = 0, kSrcConst = 1, kSrcTrig = 2, kSrcField = 3, kSrcReaction = 4, kSrcRuntime = 5, kSrcRuntimeNR = 6 };

// max(x, 0)^q for the power-law flux (q != 2) and the reaction term: those
// terms are defined for phi >= 0, and an undershoot next to a steep front must
// not turn into a non-finite value.
__device__ __forceinline__ float powr(float x, float q) { return powf(fmaxf(x, 0.0f), q); }
__device__ __forceinline__ double powr(double x, double q) { return pow(fmax(x, 0.0), q); }
__device__ __forceinline__ dw powr(dw x, dw q) {
    return dw(pow(fmax(static_cast<double>(x), 0.0), static_cast<double>(q)));
}

// max(x, 0)^(n + h/2) for a whole or half-whole exponent: n products and one
// square root (the exponents of Eq. 67 in the paper's tests are 1.5 and 2.5);
// n < 0 falls back to powr.
__device__ __forceinline__ float not_negative(float x) { return fmaxf(x, 0.0f); }
__device__ __forceinline__ double not_negative(double x) { return fmax(x, 0.0); }
__device__ __forceinline__ dw not_negative(dw x) { return x.hi > 0.0f ? x : dw(0.0f, 0.0f); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ dw sqrt_r(dw x) { return dw(sqrt(static_cast<double>(x))); }
template <typename Real>
__device__ __forceinline__ Real pow_half(Real x, Real q, int n, int h) {
    if (n < 0) return powr(x, q);
    const Real xp = not_negative(x);
    Real r = Real(1);
    for (int k = 0; k < n; ++k) r = r * xp;
    if (h) r = r * sqrt_r(xp);
    return r;
}

// phi^q / q times q, i.e. phi^q (q == 2: one product).
template <typename Real>
__device__ __forceinline__ Real flux_pow(const SweepParams<Real> &p, Real phi) {
    return p.bq2 ? phi * phi : pow_half(phi, p.bq, p.bq_n, p.bq_h);
}

// Reaction term S = rate phi (1 - phi^exp) (Eq. 67); exp == 2 takes phi phi.
template <typename Real>
__device__ __forceinline__ Real reaction(const SweepParams<Real> &p, Real phi) {
    const Real pe = p.react2 ? phi * phi : pow_half(phi, p.react_exp, p.re_n, p.re_h);
    return p.react_rate * phi * (Real(1) - pe);
}

// K1 = (3 A^ + I/2)^-1 (Eq. 30) for A^ = (1 + a2 phi^2) A0^, built and inverted
// in FP64 and rounded to FP32: the FP32 sweep's path for ill-conditioned blocks.
// Not inlined, so that the FP32 sweeps issue none of its FP64 instructions at
// well-conditioned nodes.
struct K1f {
    float xx, xy, yy;
};
static __device__ __noinline__ K1f k1_fp64(double phi, double a2, double bxx, double bxy, double byy) {
    const double s3d = 3.0 + 3.0 * a2 * phi * phi;
    const double dxx = s3d * bxx + 0.5, dxy = s3d * bxy, dyy = s3d * byy + 0.5;
    const double id = 1.0 / (dxx * dyy - dxy * dxy);
    return K1f{(float)(dyy * id), (float)(-dxy * id), (float)(dxx * id)};
}

// FP64 operations (add, multiply or FMA: one each) per node of the FP64 sweep in
// its k0 = 1 constant-coefficient form with the trig source
// (sweep_kernel<double, double, kShiftNone, kLinearK0One, kSrcTrig>), counted
// from collide_fold and source_at below: the moments 18 adds (a13, a24, s57,
// s68, sd, a1324, phid, b13, b24, d57, d68, jx: 2, jy: 2, pxy, del), V 2 adds
// (Vp, Vm); qx, qy 2 FMAs + 2 multiplies, Vx, Vy 4 FMAs, sig 2 FMAs, r0 1 FMA +
// 1 multiply, ks 1 multiply, T1, T5 2 FMAs, A1, A2, P, M 4 FMAs, r1..r8 8 FMAs,
// the trig source 1 FMA + 1 multiply and a = ... + src 1 FMA: 20 adds, 25 FMAs,
// 5 multiplies.  ncu counts 50.6 per node (DADD 20.5, DFMA 25.0, DMUL 5.0).
constexpr int kFp64AddsPerNodeLinearTrig = 20;
constexpr int kFp64FmasPerNodeLinearTrig = 25;
constexpr int kFp64MulsPerNodeLinearTrig = 5;
constexpr int kFp64OpsPerNodeLinearTrig = 50;

// Moment-space form of Eq. 6 (Eqs. 94, 95, 99 with K2 = k2 Ihat), expanded back
// into populations and written for shifted values d_i = f_i - w_i rs: rs = 0
// (kShiftNone), rs = phi_ref (kShiftRef) or rs = phi^{n-1} of this node
// (kShiftLocal).  The shift cancels from the first moments and from M2xx - M2yy,
// enters the trace as rs, and in the outputs only as -k0 w_i rs, which folds into
// the isotropic term; so the shift costs one add per node instead of eighteen.
//
// With sigma = nxx + nyy and delta = nxx - nyy of the non-equilibrium second
// moments, kap = (9/2)(k2 - k0) and a = k0 (phi - rs) + source:
//   d_i^+ = (1 - k0) d_i + w_i (a + cC_i) + 3 w_i e_i . V - w_i kap H_i
//   w0 kap H_0 = -(w0 kap/3) sigma,  w1 kap H_x,y = (w1 kap/6)(sigma +- 3 delta),
//   w5 kap H_d = (2/3) w5 kap (sigma +- 3 nxy)   (w1 kap / 6 = (2/3) w5 kap = (k2 - k0) / 12),
//   V = k0 B - (K1 - k0 I)(M1 - B) + (I - K1/2)(B^n - B^{n-1})    (Eq. 11)
//     = K1 (B - M1 - dB/2) + k0 M1 + dB,   dB = B^n - B^{n-1},
//   cC_i = (3/2) k0 (C - phi)(|e_i|^2 - 2/3)   (zero when C = phi).
// The second form of V takes ten operations where the first takes twenty-one;
// for B = u phi it is K1 u phi - (K1 - k0 I) M1 + (I - K1/2) u dphi, three
// per-lattice vectors and a matrix.
// MODE selects per-lattice constants (B = u phi, C = phi, constant A: kLinear,
// kLinearK0One) or per-node coefficient evaluation (kGeneral: nonlinear B, C and
// A(x, phi) with the first-order block K1 = (3 A^ + I/2)^-1 of Eq. 30 and k2 from
// Eq. 62 built at every node).  SRC: 0 none, 1 constant, 2 trig table, 3 field,
// 4 decided at run time.  Returns phi; phid_out = phi - rs as summed from the d_i.
template <typename Real, int MODE, int SRC, int SH>
__device__ __forceinline__ Real collide_fold(const SweepParams<Real> &p, Real (&d)[9], Real rs, Real phi_prev,
                                             Real srcv, bool first, int node, Real &phid_out,
                                             const FoldConsts<Real> *Lc = nullptr) {
    // the folded constants: p.lin, or the copy at Lc (a batch keeps its members'
    // copies in the kernel's parameter space)
    const FoldConsts<Real> &L = Lc ? *Lc : p.lin;
    constexpr bool K0ONE = MODE == kLinearK0One;
    const Real a13 = d[1] + d[3], a24 = d[2] + d[4];
    const Real s57 = d[5] + d[7], s68 = d[6] + d[8];
    const Real sd = s57 + s68;
    const Real a1324 = a13 + a24;
    const Real phid = (d[0] + sd) + a1324;            // phi - rs
    phid_out = phid;
    Real phi = phid;
    if constexpr (SH != kShiftNone) phi = phid + rs;
    const Real b13 = d[1] - d[3], b24 = d[2] - d[4];
    const Real d57 = d[5] - d[7], d68 = d[6] - d[8];
    const Real jx = b13 + (d57 - d68);
    const Real jy = b24 + (d57 + d68);
    const Real pxy = s57 - s68;
    const Real del = a13 - a24;
    // phi^n - phi^{n-1}; with the local shift rs = phi^{n-1}, so it is phid itself
    const Real dphi = first ? Real(0) : (SH == kShiftLocal ? phid : phi - phi_prev);

    Real Vx, Vy, c0, k6, k6x3;
    Real cmid = phid;                                   // C - rs
    Real cc = Real(0);                                  // (3/2) k0 (C - phi)
    if constexpr (MODE != kGeneral) {
        const Real qx = fma(L.Qxy, jy, L.Qxx * jx), qy = fma(L.Qyy, jy, L.Qxy * jx);   // (K1 - k0 I) M1
        if constexpr (SH == kShiftLocal) {
            Vx = fma(L.gx, dphi, fma(L.Px, phi, -qx));
            Vy = fma(L.gy, dphi, fma(L.Py, phi, -qy));
        } else {
            // g dphi = g phi - g phi^{n-1}: the first term joins the coefficient of phi
            const Real cx = first ? L.Px : L.Pgx, cy = first ? L.Py : L.Pgy;
            const Real gx = first ? Real(0) : L.gx, gy = first ? Real(0) : L.gy;
            Vx = fma(-gx, phi_prev, fma(cx, phi, -qx));
            Vy = fma(-gy, phi_prev, fma(cy, phi, -qy));
        }
        c0 = L.c0;
        k6 = L.k6;
        k6x3 = L.k6x3;
    } else {
        // coefficients at phi (Eq. 1 families): B = u phi + bg phi^q and
        // dB = B(phi) - B(phi_prev) = u dphi + bg (phi^q - phi_prev^q), for q = 2
        // factored as bg (phi + phi_prev) dphi
        const Real p2 = phi * phi;
        Real Bx, By, dBx, dBy;
        if (p.bq2) {
            Bx = fma(p.ux, phi, p.bgx * p2);
            By = fma(p.uy, phi, p.bgy * p2);
            const Real sp = phi + phi_prev;
            dBx = fma(p.bgx, sp, p.ux) * dphi;
            dBy = fma(p.bgy, sp, p.uy) * dphi;
        } else {
            const Real gq = pow_half(phi, p.bq, p.bq_n, p.bq_h);
            const Real dg = first ? Real(0) : gq - pow_half(phi_prev, p.bq, p.bq_n, p.bq_h);
            Bx = fma(p.ux, phi, p.bgx * gq);
            By = fma(p.uy, phi, p.bgy * gq);
            dBx = fma(p.ux, dphi, p.bgx * dg);
            dBy = fma(p.uy, dphi, p.bgy * dg);
        }
        const Real Cm = p.c3 * p2 * phi;                 // C(phi) - phi
        cmid = phid + Cm;
        cc = L.k0x15 * Cm;
        // first-order block K1 = (3 A^ + I/2)^-1 (Eq. 30), A^ = (1 + a2 phi^2) A0^
        const Real s3 = fma(L.a2x3, p2, Real(3));
        Real a0xx = p.A0xx, a0xy = p.A0xy, a0yy = p.A0yy;
        if (p.Af) {   // spatially varying tensor A(x)
            a0xx = p.Af[BTRT_IX(p.flags, node, p.plane)];
            a0xy = p.Af[BTRT_IX(p.flags, p.plane + node, 3 * p.plane)];
            a0yy = p.Af[BTRT_IX(p.flags, 2 * p.plane + node, 3 * p.plane)];
        }
        const Real mxx = fma(s3, a0xx, Real(0.5));
        const Real mxy = s3 * a0xy;
        const Real myy = fma(s3, a0yy, Real(0.5));
        const Real tr = mxx + myy;
        const Real det = fma(mxx, myy, -(mxy * mxy));
        Real K1xx, K1xy, K1yy;
        bool ill = false;
        if constexpr (sizeof(Real) == 4) ill = tr * tr > p.cond_limit * det;
        if (ill) {
            // ill-conditioned FP32 block: build it again from FP64 coefficients (the
            // FP32-rounded entries would carry errors the condition number amplifies)
            // and invert it in FP64
            const K1f k = p.Af ? k1_fp64(static_cast<double>(phi), p.a2d, (double)a0xx, (double)a0xy, (double)a0yy)
                               : k1_fp64(static_cast<double>(phi), p.a2d, p.A0d[0], p.A0d[1], p.A0d[2]);
            K1xx = (Real)k.xx;
            K1xy = (Real)k.xy;
            K1yy = (Real)k.yy;
        } else {
            const Real id = quot(Real(1), det);
            K1xx = myy * id;
            K1xy = -mxy * id;
            K1yy = mxx * id;
        }
        // Eq. 62 at k1_eff = 2/tr:  k2 = 8 (k1 - 2) / (3 (k1 - 4)) = (8/3)(tr - 1) / (2 tr - 1)
        const Real k2 = p.k2_hbb ? quot(cst<Real>(8, 3) * (tr - Real(1)), fma(Real(2), tr, Real(-1))) : p.k2c;
        c0 = fma(cst<Real>(2, 3), k2, L.c0k);            // (2/3)(k2 - k0) = w0 kap / 3
        k6 = fma(cst<Real>(-1, 12), k2, L.k6k);          // -(k2 - k0) / 12
        k6x3 = fma(cst<Real>(-1, 4), k2, L.k6x3k);       // 3 k6
        const Real ex = fma(Real(-0.5), dBx, Bx - jx), ey = fma(Real(-0.5), dBy, By - jy);
        Vx = fma(K1xx, ex, fma(K1xy, ey, fma(L.k0, jx, dBx)));
        Vy = fma(K1xy, ex, fma(K1yy, ey, fma(L.k0, jy, dBy)));
    }
    const Real sig = fma(cst<Real>(-2, 3), cmid, fma(Real(2), sd, a1324));
    Real a = K0ONE ? phid : L.k0 * phid;
    if constexpr (SRC == kSrcReaction || SRC == kSrcRuntime) {
        // phi-dependent source: (3 S(phi^n) - S(phi^{n-1})) / 2 (scheme 2), S^{-1} = S^0 at start
        if (SRC == kSrcReaction || p.src_kind == kSrcReaction) {
            const Real Sn = reaction(p, phi);
            const Real Sp = first ? Sn : reaction(p, phi_prev);
            srcv = fma(Real(1.5), Sn, Real(-0.5) * Sp);
        }
    }
    if constexpr (SRC != 0) a = fma(p.src_val, srcv, a);
    const Real w0 = cst<Real>(4, 9), w1 = cst<Real>(1, 9), w5 = cst<Real>(1, 36);
    const Real v1 = cst<Real>(1, 3), v5 = cst<Real>(1, 12);   // 3 w1, 3 w5
    Real r[9];
    if constexpr (MODE == kGeneral) {
        r[0] = fma(c0, sig, w0 * fma(cst<Real>(-2, 3), cc, a));
    } else {
        r[0] = fma(c0, sig, w0 * a);
    }
    const Real ks = k6 * sig;   // the sigma term of the axis and diagonal directions (equal weights)
    const Real T1 = MODE == kGeneral ? fma(w1, fma(cst<Real>(1, 3), cc, a), ks) : fma(w1, a, ks);
    const Real A1 = fma(k6x3, del, T1), A2 = fma(-k6x3, del, T1);
    r[1] = fma(v1, Vx, A1);
    r[3] = fma(-v1, Vx, A1);
    r[2] = fma(v1, Vy, A2);
    r[4] = fma(-v1, Vy, A2);
    const Real T5 = MODE == kGeneral ? fma(w5, fma(cst<Real>(4, 3), cc, a), ks) : fma(w5, a, ks);
    const Real P = fma(k6x3, pxy, T5), M = fma(-k6x3, pxy, T5);
    const Real Vp = Vx + Vy, Vm = Vx - Vy;
    r[5] = fma(v5, Vp, P);
    r[7] = fma(-v5, Vp, P);
    r[6] = fma(-v5, Vm, M);
    r[8] = fma(v5, Vm, M);
    // k0 = 1: nothing of d_i is kept (bitwise the same as (1 - k0) d_i + r_i).  A
    // run-time test where it saves more than it costs: the per-node coefficient
    // path and the double-word sweep (an FMA is a dozen instructions there); the
    // FP64 sweep has its own variant for k0 = 1, and the FP32 constant-coefficient
    // sweep is bound by memory, where the test's extra registers cost occupancy.
    constexpr bool K0RT = MODE == kGeneral || std::is_same<Real, dw>::value;
    if (K0ONE || (K0RT && p.k0_one)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = r[i];
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = fma(L.om, d[i], r[i]);
    }
    return phi;
}

// Equilibrium populations (Eq. 7) in lattice units, D = C(phi) I, shifted by
// w_i rs as the collision expects (rs = phi for the local shift).
template <typename Real, int SH>
__device__ __forceinline__ void equilibrium(const SweepParams<Real> &p, Real phi, Real (&f)[9]) {
    const Real g = flux_pow(p, phi);
    const Real Bx = Real(3) * fma(p.ux, phi, p.bgx * g), By = Real(3) * fma(p.uy, phi, p.bgy * g);
    const Real cc = Real(1.5) * p.c3 * phi * phi * phi;
    const Real w0 = cst<Real>(4, 9), w1 = cst<Real>(1, 9), w5 = cst<Real>(1, 36);
    const Real a0 = phi - cc * cst<Real>(2, 3);
    const Real a1 = phi + cc * cst<Real>(1, 3);
    const Real a5 = phi + cc * cst<Real>(4, 3);
    f[0] = w0 * a0;
    f[1] = w1 * (a1 + Bx);
    f[3] = w1 * (a1 - Bx);
    f[2] = w1 * (a1 + By);
    f[4] = w1 * (a1 - By);
    f[5] = w5 * (a5 + Bx + By);
    f[7] = w5 * (a5 - Bx - By);
    f[6] = w5 * (a5 - Bx + By);
    f[8] = w5 * (a5 + Bx - By);
    if constexpr (SH == kShiftRef) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = f[i] - p.wref[i];
    } else if constexpr (SH == kShiftLocal) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fma(-wgt<Real>(i), phi, f[i]);
    }
}

// Non-finite test without touching the FP64 pipe: exponent field all ones.
__device__ __forceinline__ bool not_finite(double v) {
    return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool not_finite(float v) {
    return (__float_as_int(v) & 0x7f800000) == 0x7f800000;
}

// ---------------------------------------------------------------- stochastic rounding
// Under diffusive scaling a step changes the state by much less than a 16-bit
// last place, and round-to-nearest then makes nearly the same error in the same
// direction step after step.  Stochastic rounding rounds up with probability
// equal to the fraction of the last place that is cut off, so every stored
// value is right on average and the errors of successive steps do not add up.
// Random bits: the 32-bit finalizer of MurmurHash3 (Appleby) of the node index
// mixed with the step's seed, then one multiply per population by a distinct
// odd constant (the product's high bits are used).  They depend only on the
// node, the step index and the population, so every kernel form stores the same
// values.
__device__ __forceinline__ unsigned int sr_node_bits(unsigned int seed, int node) {
    unsigned int h = (unsigned int)node ^ seed;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ unsigned int sr_bits(unsigned int h, int i) {
    return h * (0x9e3779b1u + 0x3c6ef372u * (unsigned int)i);
}
// FP32 -> BF16: add 16 random bits below BF16's last place to the FP32 pattern and
// truncate (BF16 has FP32's exponent range, so this holds for every finite value).
// FP32 -> FP16: the deviations are stored scaled by kSrScaleF16 = 2^12, which keeps
// them in FP16's normal range (on fine grids they are 1e-5 and below, where FP16's
// subnormal spacing 2^-24 would be a large part of each value; FP16's largest
// value, 65504, still allows deviations up to 16); then 13 random bits below FP16's
// last place are added to the FP32 pattern and the value converted toward zero.
// Both scalings are exact (powers of two).  Scaled values below FP16's normal range
// (deviations below 1.5e-8) are cut toward zero.
constexpr float kSrScaleF16 = 4096.f;
template <typename S> __device__ __forceinline__ S pack_sr(float v, unsigned int r);
template <> __device__ __forceinline__ __nv_bfloat16 pack_sr<__nv_bfloat16>(float v, unsigned int r) {
    const unsigned int b = __float_as_uint(v) + (r >> 16);
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
}
template <> __device__ __forceinline__ __half pack_sr<__half>(float v, unsigned int r) {
    return __float2half_rz(__uint_as_float(__float_as_uint(v * kSrScaleF16) + (r >> 19)));
}
// The same with FP16's subnormal range rounded stochastically too: the random bits
// cover all the FP32 mantissa bits below FP16's last place there (13 in the normal
// range, up to 23 below it; scaled values under 2^-24 are cut toward zero).  The
// first-moment form needs it: its stored values are O(dx^2) and, even scaled,
// reach FP16's subnormal range on fine grids.
template <typename S> __device__ __forceinline__ S pack_sr_sub(float v, unsigned int r) { return pack_sr<S>(v, r); }
template <> __device__ __forceinline__ __half pack_sr_sub<__half>(float v, unsigned int r) {
    const unsigned int u = __float_as_uint(v * kSrScaleF16);
    const int e = (int)((u >> 23) & 0xffu);
    const int k = e >= 113 ? 13 : min(23, 126 - e);
    return __float2half_rz(__uint_as_float(u + ((r >> 9) & ((1u << k) - 1u))));
}
// The new phi of the first-moment form, rounded stochastically to FP32 as well:
// phi = fl(phid + rs) and the TwoSum error e (phid + rs = phi + e exactly) move it
// one FP32 place towards e with probability |e| / place.  Under diffusive scaling
// a step changes phi by a few FP32 places, and round-to-nearest would repeat nearly
// the same error step after step; with the local shift the stochastically rounded
// 16-bit deviations dither that rounding, the first-moment form's far smaller ones
// do not.  r: random bits (the node's population-9 bits).
__device__ __forceinline__ float phi_sr(float phi, float phid, float rs, unsigned int r) {
    const float bb = phi - rs;
    const float e = (rs - (phi - bb)) + (phid - bb);
    // the neighbouring FP32 value on e's side (for phi = 0, e is 0 and phi stays;
    // a non-finite phi makes e NaN and stays too)
    const float nb = __int_as_float(__float_as_int(phi) + (((e > 0.f) == (phi > 0.f)) ? 1 : -1));
    const float u = __uint_as_float(0x3f800000u | (r >> 9)) - 1.f;   // uniform in [0, 1)
    return fabsf(e) > u * fabsf(nb - phi) ? nb : phi;
}

// The stored deviation back in the compute type: FP16 values of the stochastically
// rounded forms carry the 2^12 scale.
template <typename S, int SH> struct DevScaled {
    static constexpr bool value = StoreSR<SH>::value && std::is_same<S, __half>::value;
};
template <typename Real, typename S, int SH> __device__ __forceinline__ Real dev_load(S v) {
    if constexpr (DevScaled<S, SH>::value) return Storage<S>::load(v) * (1.f / kSrScaleF16);
    else return Storage<S>::load(v);
}
// kShiftMomentSR: the writer's first moment j in the storage format (with the
// deviations' scale), rounded to nearest; reader and writer both use the stored
// value, so its rounding changes only what is subtracted, not the result.
template <typename S, int SH> __device__ __forceinline__ S j_pack(float v) {
    if constexpr (DevScaled<S, SH>::value) return Storage<S>::pack(v * kSrScaleF16);
    else return Storage<S>::pack(v);
}
// e_i . j for the compile-time direction i, and 3 w_i (1/3 on the axes, 1/12 on the diagonals)
template <typename Real> __device__ __forceinline__ Real e_dot(int i, Real jx, Real jy) {
    const int ex = ex_of(i), ey = ey_of(i);
    if (ey == 0) return ex > 0 ? jx : -jx;
    if (ex == 0) return ey > 0 ? jy : -jy;
    return (ex > 0 ? jx : -jx) + (ey > 0 ? jy : -jy);
}
template <typename Real> __device__ __forceinline__ Real w3(int i) {
    return i <= 4 ? cst<Real>(1, 3) : cst<Real>(1, 12);
}

// FP64 and double-word storage are never shifted; the other formats take the
// shift the lattice was created with.
template <typename S, int SH> struct ShiftOf { static constexpr int value = SH; };
template <int SH> struct ShiftOf<double, SH> { static constexpr int value = kShiftNone; };
template <int SH> struct ShiftOf<dw, SH> { static constexpr int value = kShiftNone; };

// Nodes per thread of the single-lattice sweep: the FP64 sweep is ALU-bound and
// amortises per-thread set-up over a column of 4 nodes; the HBM-bound FP32-storage
// sweep takes two nodes with both pulls issued before the collisions (loads in
// flight together, set-up shared); the FP16/BF16-storage sweeps, limited by
// registers and issue, keep one node per thread.  The BTRT_ROWS_* macros
// override the counts at build time (tuning).
#ifndef BTRT_ROWS_S32
#define BTRT_ROWS_S32 2
#endif
#ifndef BTRT_UNROLL_S32
#define BTRT_UNROLL_S32 1
#endif
#ifndef BTRT_ROWS_S16
#define BTRT_ROWS_S16 1
#endif
#ifndef BTRT_UNROLL_S16
#define BTRT_UNROLL_S16 0
#endif
template <typename Real, typename S> struct RowsPerThread {
    static constexpr int value = BTRT_ROWS_S16;
    static constexpr bool unroll = BTRT_UNROLL_S16 != 0;
};
template <> struct RowsPerThread<float, float> {
    static constexpr int value = BTRT_ROWS_S32;
    static constexpr bool unroll = BTRT_UNROLL_S32 != 0;
};
#ifndef BTRT_ROWS_F64
#define BTRT_ROWS_F64 4
#endif
#ifndef BTRT_MINBLOCKS_F64
#define BTRT_MINBLOCKS_F64 0
#endif
#ifndef BTRT_UNROLL_F64
#define BTRT_UNROLL_F64 0
#endif
template <> struct RowsPerThread<double, double> {
    static constexpr int value = BTRT_ROWS_F64;
    static constexpr bool unroll = BTRT_UNROLL_F64 != 0;
};
#ifndef BTRT_MINBLOCKS_F32
#define BTRT_MINBLOCKS_F32 0
#endif
// 16-bit storage: six blocks (40 registers) measured +11 % on the nonlinear
// workload with the reference shift and +2 % with the local shift against the
// compiler's 48 registers and five blocks; FP32 storage would spill heavily.
#ifndef BTRT_MINBLOCKS_S16
#define BTRT_MINBLOCKS_S16 6
#endif
// Minimum resident blocks per SM requested from the compiler (register budget);
// 0 leaves the choice to the compiler.
// FP64 per-node coefficient sweeps: the compiler's 96 registers (two blocks);
// four blocks (64 registers) measured 5.14 GLUPS against 5.57 on the nonlinear
// workload.
#ifndef BTRT_MINBLOCKS_F64_GEN
#define BTRT_MINBLOCKS_F64_GEN 0
#endif
// Double-word constant-coefficient sweeps: five blocks (48 registers, 12 spilled
// bytes) measured 36.9 GLUPS against 33.5 with the compiler's 64 registers; the
// per-node coefficient form would spill hundreds of bytes there.
#ifndef BTRT_MINBLOCKS_DW
#define BTRT_MINBLOCKS_DW 5
#endif
template <typename Real, typename S, int MODE> struct MinBlocks { static constexpr int value = 0; };
template <int MODE> struct MinBlocks<double, double, MODE> {
    static constexpr int value = MODE == kGeneral ? BTRT_MINBLOCKS_F64_GEN : BTRT_MINBLOCKS_F64;
};
template <int MODE> struct MinBlocks<float, float, MODE> { static constexpr int value = BTRT_MINBLOCKS_F32; };
template <int MODE> struct MinBlocks<float, __half, MODE> { static constexpr int value = BTRT_MINBLOCKS_S16; };
template <int MODE> struct MinBlocks<float, __nv_bfloat16, MODE> { static constexpr int value = BTRT_MINBLOCKS_S16; };
template <int MODE> struct MinBlocks<dw, dw, MODE> {
    static constexpr int value = MODE == kGeneral ? 0 : BTRT_MINBLOCKS_DW;
};
template <> struct RowsPerThread<dw, dw> { static constexpr int value = 1; static constexpr bool unroll = false; };

// Global loads of data that other SMs rewrite during a persistent launch go
// through L2 only (L1 is not coherent across SMs); ordinary loads otherwise.
template <bool L2ONLY, typename T>
__device__ __forceinline__ T ldg(const T *ptr) {
    if constexpr (L2ONLY) return __ldcg(ptr);
    else return *ptr;
}

// Pull of a node on the domain boundary: periodic wrap or, for a link that
// crosses a wall, the node's own population leaving towards it comes back as
// direction i (half-way bounce-back, Eqs. 54-56).  Out: d_i = f_i - w_i rs with
// rs = phi_prev (the node's phi^{n-1}) for the local shift.
template <typename Real, typename S, int SH, bool L2ONLY>
__device__ __forceinline__ void pull_boundary(const SweepParams<Real> &p, const S *__restrict__ fin, int x,
                                              int y, int node, Real phi_prev, Real (&d)[9], Real phi_lo = Real(0)) {
    constexpr int PS = PullShift<SH>::value;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - ex_of(i), sy = y - ey_of(i);
        int wx = -1, wy = -1;   // crossed wall side, if any
        if (sx < 0) { if (p.hbb_x) wx = 0; else sx += p.nx; }
        if (sx >= p.nx) { if (p.hbb_x) wx = 1; else sx -= p.nx; }
        if (sy < 0) { if (p.hbb_y) wy = 2; else sy += p.ny; }
        if (sy >= p.ny) { if (p.hbb_y) wy = 3; else sy -= p.ny; }
        if (wx < 0 && wy < 0) {
            const int src = sy * p.pitch + sx;
            d[i] = dev_load<Real, S, SH>(ldg<L2ONLY>(fin + BTRT_IX(p.flags, i * p.plane + src, 9 * p.plane)));
            if constexpr (PS == kShiftLocal || PS == kShiftMomentSR)
                if (i != 0) d[i] = fma(wgt<Real>(i), ldg<L2ONLY>(p.phi_in + BTRT_IX(p.flags, src, p.plane)) - phi_prev, d[i]);
            if constexpr (PS == kShiftMomentSR)
                if (i != 0) {
                    const S *jin = static_cast<const S *>(p.j_in);
                    const Real jx = dev_load<Real, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, src, 2 * p.plane)));
                    const Real jy = dev_load<Real, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, p.plane + src, 2 * p.plane)));
                    d[i] = fma(w3<Real>(i), e_dot<Real>(i, jx, jy), d[i]);
                }
            if constexpr (PS == kShiftLocalDW)
                if (i != 0)
                    d[i] = fma(wgt<Real>(i),
                               (ldg<L2ONLY>(p.phi_in + BTRT_IX(p.flags, src, p.plane)) - phi_prev) +
                                   (ldg<L2ONLY>(p.phi_in_lo + BTRT_IX(p.flags, src, p.plane)) - phi_lo),
                               d[i]);
        } else {
            const int o = opp_of(i);
            Real phi_w;
            if (wx >= 0 && wy >= 0)
                phi_w = Real(0.5) * (wall_value(p, wx, y) + wall_value(p, wy, x));
            else if (wy >= 0)
                phi_w = wall_value(p, wy, x);
            else
                phi_w = wall_value(p, wx, y);
            const Real dout = dev_load<Real, S, SH>(ldg<L2ONLY>(fin + BTRT_IX(p.flags, o * p.plane + node, 9 * p.plane)));
            // f_i = -f_o^+ + wall term; in shifted form the two shifts add up to -2 w_i rs
            // (for the local shift f_o^+ was stored relative to this node's own phi^{n-1} = rs)
            Real wt = wall_term(p, o, phi_w);
            if constexpr (PS == kShiftRef) wt = wt - Real(2) * p.wref[i];
            if constexpr (PS == kShiftLocal || PS == kShiftLocalDW || PS == kShiftMomentSR)
                wt = fma(Real(-2) * wgt<Real>(i), phi_prev, wt);
            if constexpr (PS == kShiftLocalDW) wt = fma(Real(-2) * wgt<Real>(i), phi_lo, wt);
            d[i] = wt - dout;
            if constexpr (PS == kShiftMomentSR) {
                // f_o^+ was stored relative to this node's own first-moment term: with
                // e_o = -e_i it returns as + 3 w_i e_i . j
                const S *jin = static_cast<const S *>(p.j_in);
                const Real jx = dev_load<Real, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, node, 2 * p.plane)));
                const Real jy = dev_load<Real, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, p.plane + node, 2 * p.plane)));
                d[i] = fma(w3<Real>(i), e_dot<Real>(i, jx, jy), d[i]);
            }
        }
    }
}

// Spatial part of the source at node (x, y) for the compile-time source kind
// (the reaction term depends on phi and is evaluated in the collision).
template <typename Real, int SRC>
__device__ __forceinline__ Real source_at(const SweepParams<Real> &p, Real xs, Real xc, int y, int node) {
    if constexpr (SRC == kSrcConst) return Real(1);
    else if constexpr (SRC == kSrcTrig) return fma(xs, p.Ys[BTRT_IX(p.flags, y, p.ny)], xc * p.Yc[BTRT_IX(p.flags, y, p.ny)]);
    else if constexpr (SRC == kSrcField) return p.srcF[BTRT_IX(p.flags, node, p.plane)];
    else if constexpr (SRC == kSrcRuntime || SRC == kSrcRuntimeNR) {
        if (p.src_kind == kSrcConst) return Real(1);
        if (p.src_kind == kSrcTrig) return fma(xs, p.Ys[BTRT_IX(p.flags, y, p.ny)], xc * p.Yc[BTRT_IX(p.flags, y, p.ny)]);
        if (p.src_kind == kSrcField) return p.srcF[BTRT_IX(p.flags, node, p.plane)];
        return Real(0);
    } else return Real(0);
}

// Pull of one node's populations (shifted form, see collide_fold) and of phi^{n-1}.
template <typename Real, typename S, int SH, bool L2ONLY>
__device__ __forceinline__ void pull_node(const SweepParams<Real> &p, int x, int y, bool x_inner, Real (&f)[9],
                                          Real &phi_prev, Real *phi_lo_out = nullptr) {
    constexpr int PS = PullShift<SH>::value;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    const int node = y * p.pitch + x;
    phi_prev = ldg<L2ONLY>(p.phi_in + BTRT_IX(p.flags, node, p.plane));
    Real phi_lo = Real(0);
    if constexpr (PS == kShiftLocalDW) {
        phi_lo = ldg<L2ONLY>(p.phi_in_lo + BTRT_IX(p.flags, node, p.plane));
        *phi_lo_out = phi_lo;
    }
    if (p.first) {
        equilibrium<Real, CollShift<SH>::value>(p, phi_prev, f);
    } else if (x_inner && y > 0 && y < p.ny - 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i] = dev_load<Real, S, SH>(
                ldg<L2ONLY>(fin + BTRT_IX(p.flags, i * p.plane + node - ey_of(i) * p.pitch - ex_of(i), 9 * p.plane)));
        if constexpr (PS == kShiftLocal || PS == kShiftMomentSR) {
#pragma unroll
            for (int i = 1; i < 9; ++i)
                f[i] = fma(wgt<Real>(i),
                           ldg<L2ONLY>(p.phi_in + BTRT_IX(p.flags, node - ey_of(i) * p.pitch - ex_of(i), p.plane)) -
                               phi_prev,
                           f[i]);
        }
        if constexpr (PS == kShiftMomentSR) {
            const S *jin = static_cast<const S *>(p.j_in);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int nb = node - ey_of(i) * p.pitch - ex_of(i);
                const Real jx = dev_load<Real, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, nb, 2 * p.plane)));
                const Real jy = dev_load<Real, S, SH>(ldg<L2ONLY>(jin + BTRT_IX(p.flags, p.plane + nb, 2 * p.plane)));
                f[i] = fma(w3<Real>(i), e_dot<Real>(i, jx, jy), f[i]);
            }
        }
        if constexpr (PS == kShiftLocalDW) {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int nb = node - ey_of(i) * p.pitch - ex_of(i);
                f[i] = fma(wgt<Real>(i),
                           (ldg<L2ONLY>(p.phi_in + BTRT_IX(p.flags, nb, p.plane)) - phi_prev) +
                               (ldg<L2ONLY>(p.phi_in_lo + BTRT_IX(p.flags, nb, p.plane)) - phi_lo),
                           f[i]);
            }
        }
    } else {
        pull_boundary<Real, S, SH, L2ONLY>(p, fin, x, y, node, phi_prev, f, phi_lo);
    }
}

// Shifted post-collision value d_i^+ = f_i^+ - w_i rs -> the stored form.
template <typename Real, typename S, int SH>
__device__ __forceinline__ S store_value(int i, Real d, Real phid) {
    if constexpr (SH == kShiftLocal) return Storage<S>::pack(fma(-wgt<Real>(i), phid, d));
    else return Storage<S>::pack(d);
}

// Collision and write-back of one pulled node.  Returns (phi^n - phi^{n-1})^2
// when RESID.  A non-finite phi sets `bad` (one atomic per thread at the end).
template <typename Real, typename S, int SH, int MODE, int SRC, bool RESID>
__device__ __forceinline__ double finish_node(const SweepParams<Real> &p, int x, int y, Real xs, Real xc,
                                              Real (&f)[9], Real phi_prev, bool &bad, Real phi_lo = Real(0),
                                              const FoldConsts<Real> *Lc = nullptr) {
    constexpr int SC = CollShift<SH>::value;
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const int node = y * p.pitch + x;
    const Real src = source_at<Real, SRC>(p, xs, xc, y, node);
    const Real rs = SC == kShiftLocal ? phi_prev : p.phi_ref;
    Real phid;
    const Real phi = collide_fold<Real, MODE, SRC, SC>(p, f, rs, phi_prev, src, p.first != 0, node, phid, Lc);
    if constexpr (PullShift<SH>::value == kShiftMomentSR) {
        // the writer's first moment sum_i e_i d_i^+ (the w_i rs terms cancel), stored
        // rounded; the deviations are taken from w_i (phi + 3 e_i . j) with the stored j
        const Real jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
        const Real jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
        S *jout = static_cast<S *>(p.j_out);
        const S jxs = j_pack<S, SH>(jx), jys = j_pack<S, SH>(jy);
        jout[BTRT_IX(p.flags, node, 2 * p.plane)] = jxs;
        jout[BTRT_IX(p.flags, p.plane + node, 2 * p.plane)] = jys;
        const Real jxv = dev_load<Real, S, SH>(jxs), jyv = dev_load<Real, S, SH>(jys);
        const unsigned int h = sr_node_bits(p.sr_seed, node);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const Real v = i == 0 ? fma(-wgt<Real>(i), phid, f[i])
                                  : fma(-w3<Real>(i), e_dot<Real>(i, jxv, jyv), fma(-wgt<Real>(i), phid, f[i]));
            fout[BTRT_IX(p.flags, i * p.plane + node, 9 * p.plane)] = pack_sr_sub<S>(v, sr_bits(h, i));
        }
    } else if constexpr (StoreSR<SH>::value) {
        const unsigned int h = sr_node_bits(p.sr_seed, node);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            fout[BTRT_IX(p.flags, i * p.plane + node, 9 * p.plane)] = pack_sr<S>(fma(-wgt<Real>(i), phid, f[i]), sr_bits(h, i));
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) fout[BTRT_IX(p.flags, i * p.plane + node, 9 * p.plane)] = store_value<Real, S, SC>(i, f[i], phid);
    }
    if constexpr (PullShift<SH>::value == kShiftLocalDW) {
        // phi^n = (phi_prev + phi_lo) + phid as a double-word pair: TwoSum of the high
        // word and phid (its sum is the collision's phi), the error into the low word,
        // then Fast2Sum to renormalise
        const Real bb = phi - phi_prev;
        const Real e = (phi_prev - (phi - bb)) + (phid - bb);
        const Real lo = phi_lo + e;
        const Real hi_n = phi + lo;
        const Real lo_n = lo - (hi_n - phi);
        p.phi_out[BTRT_IX(p.flags, node, p.plane)] = hi_n;
        p.phi_out_lo[BTRT_IX(p.flags, node, p.plane)] = lo_n;
        bad |= not_finite(hi_n);
        if (RESID) {
            const double dd = (static_cast<double>(hi_n) - static_cast<double>(phi_prev)) +
                              (static_cast<double>(lo_n) - static_cast<double>(phi_lo));
            return dd * dd;
        }
        return 0.0;
    } else {
        Real phis = phi;
        if constexpr (SH == kShiftMomentSR) phis = phi_sr(phi, phid, rs, sr_bits(sr_node_bits(p.sr_seed, node), 9));
        p.phi_out[BTRT_IX(p.flags, node, p.plane)] = phis;
        bad |= not_finite(phis);
        if (RESID) {
            const double dd = static_cast<double>(phis) - static_cast<double>(phi_prev);
            return dd * dd;
        }
        return 0.0;
    }
}

// Sweep nodes of column x, rows ybase, ybase + ystride, ...: NR > 0 nodes, with
// all NR pulls issued before the first collision when UNROLL (their loads are in
// flight together), or one node after the other; NR == 0: `nrows` nodes decided
// at run time.  Returns the sum of the nodes' (phi^n - phi^{n-1})^2 when RESID
// (steady-state residual), else 0.  RESID is a template argument so that no FP64
// arithmetic is issued (or speculated) in ordinary sweeps.
template <typename Real, typename S, int SH, int MODE, int SRC, bool L2ONLY, bool RESID, int NR = 0,
          bool UNROLL = false>
__device__ __forceinline__ double sweep_rows(const SweepParams<Real> &p, int x, int ybase, int ystride,
                                             int nrows) {
    Real xs = Real(0), xc = Real(0);
    if (SRC == kSrcTrig || ((SRC == kSrcRuntime || SRC == kSrcRuntimeNR) && p.src_kind == kSrcTrig)) {
        xs = p.Xs[BTRT_IX(p.flags, x, p.nx)];
        xc = p.Xc[BTRT_IX(p.flags, x, p.nx)];
    }
    const bool x_inner = (x > 0) && (x < p.nx - 1);
    double resid = 0.0;
    bool bad = false;
    if constexpr (NR > 0 && UNROLL) {
        Real f[NR][9], phi_prev[NR], phi_lo[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int y = ybase + r * ystride;
            if (y < p.ny) pull_node<Real, S, SH, L2ONLY>(p, x, y, x_inner, f[r], phi_prev[r], &phi_lo[r]);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int y = ybase + r * ystride;
            if (y < p.ny)
                resid += finish_node<Real, S, SH, MODE, SRC, RESID>(p, x, y, xs, xc, f[r], phi_prev[r], bad,
                                                                    phi_lo[r]);
        }
    } else {
        const int n = NR > 0 ? NR : nrows;
#pragma unroll 1
        for (int r = 0; r < n; ++r) {
            const int y = ybase + r * ystride;
            if (y >= p.ny) break;
            Real f[9], phi_prev, phi_lo = Real(0);
            pull_node<Real, S, SH, L2ONLY>(p, x, y, x_inner, f, phi_prev, &phi_lo);
            resid += finish_node<Real, S, SH, MODE, SRC, RESID>(p, x, y, xs, xc, f, phi_prev, bad, phi_lo);
        }
    }
    if (bad) atomicOr(p.flags, 1);
    return resid;
}

// One sweep of one lattice: 32 x 8 threads per block, each thread sweeps
// RowsPerThread nodes of its column, rows blockDim.y apart.
template <typename Real, typename S, int SH, int MODE, int SRC>
__global__ void __launch_bounds__(256, MinBlocks<Real, S, MODE>::value) sweep_kernel(const __grid_constant__ SweepParams<Real> p) {
    constexpr int R = RowsPerThread<Real, S>::value;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int ybase = blockIdx.y * blockDim.y * R + threadIdx.y;
    constexpr bool U = RowsPerThread<Real, S>::unroll;
    if (!p.resid_partials) {
        if (x < p.nx) sweep_rows<Real, S, SH, MODE, SRC, false, false, R, U>(p, x, ybase, blockDim.y, R);
        return;
    }
    // residual step: every thread joins the fixed-order block reduction
    __shared__ double red[256];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    red[tid] = x < p.nx ? sweep_rows<Real, S, SH, MODE, SRC, false, true, R, U>(p, x, ybase, blockDim.y, R) : 0.0;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0) p.resid_partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

}  // namespace btrt
