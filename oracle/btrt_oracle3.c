/*
 * btrt_oracle3.c -- reference implementation of the B-TriRT scheme on the D3Q19
 * lattice (the three-dimensional variant of the appendix: Eqs. 77, 80, 81, 84,
 * 86, 89 and the D3Q19 form of S_f).  TEST INFRASTRUCTURE ONLY: imported by the
 * tests, never by the library.
 *
 * Plain, slow and literal: FP64, physical units, population space.  The
 * collision is Eq. 6 written with the relaxation matrices of Eq. 77,
 *     f_i^+ = f_i - k0 g_i - sum_j R_ij g_j - sum_j P_ij g_j + dt G_i + dt S_i
 *             + dt^2/2 D S_i,
 *     R_ij = w_i c_i.[(K1 - k0 I) c_j] / cs^2,
 *     P_ij = w_i (c_i c_i - cs^2 I):[(K2 - k0 Ihat) o (c_j c_j)] / (2 cs^4),
 * with g = f - f^eq, the equilibrium of Eq. 7 in three dimensions, K1 from
 * Eq. 30 (a 3x3 inverse), K2 = k2 Ihat, and G, S as in Eqs. 8 and 11.  The
 * readings that the two-dimensional oracle documents carry over: the backward
 * difference of B for d_t B, zero time derivatives at the first step, wall
 * values at t_{n+1}, and a link that crosses two walls (an edge) takes the mean
 * of their values.  k2 in the "HBB" mode follows Eq. 62 at the mean first-order
 * rate, 1/k1_eff = tr(K1^{-1}) / 3.
 *
 * Velocity order (columns of C_D3Q19, Eq. 86):
 *   0 (0,0,0); 1,2 (+-1,0,0); 3,4 (0,+-1,0); 5,6 (0,0,+-1);
 *   7 (1,1,0) 8 (-1,1,0) 9 (1,-1,0) 10 (-1,-1,0);
 *   11 (1,0,1) 12 (-1,0,1) 13 (1,0,-1) 14 (-1,0,-1);
 *   15 (0,1,1) 16 (0,-1,1) 17 (0,1,-1) 18 (0,-1,-1).
 * Weights 1/3, 1/18 (axis), 1/36 (face diagonals).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define Q3 19

static const int CX[Q3] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q3] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q3] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};

static double weight3(int i)
{
    int n2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    return n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

static int opposite3(int i)
{
    for (int j = 0; j < Q3; ++j)
        if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) return j;
    return -1;
}

enum { BC3_PERIODIC = 0, BC3_HBB = 1 };
enum { K2_3_HBB = 0, K2_3_CONST = 1 };
enum { SRC3_NONE = 0, SRC3_CONST = 1, SRC3_FIELD = 3, SRC3_REACTION = 4 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t bc[6];            /* faces x-, x+, y-, y+, z-, z+ */
    double dx, dt, x0, y0, z0;
    double u[3], b2, b_dir[3], b_q;   /* B(phi) = u phi + b2 (phi^q / q) d */
    double c3;                /* C(phi) = phi + c3 phi^3 */
    double A0[6];             /* A(phi) = (1 + a2 phi^2) A0; xx, xy, xz, yy, yz, zz */
    double a2;
    double k0;
    int32_t k2_mode, src_kind;
    double k2;
    double src_const, src_lam;          /* const: S; field: exp(src_lam t) F(x) */
    double react_rate, react_exp;       /* reaction: rate phi (1 - phi^exp) */
    double wall[6];           /* constant wall value per face */
    double wall_lam;          /* times exp(wall_lam t) */
    const double *src_field;  /* [nz][ny][nx] */
} oracle3_problem;

/* ---------------------------------------------------------------- coefficients */

static double phi_pow3(double phi, double q)
{
    if (q == 2.0) return phi * phi;
    return pow(phi > 0.0 ? phi : 0.0, q);
}

void btrt3_oracle_B(const oracle3_problem *p, double phi, double B[3])
{
    double g = phi_pow3(phi, p->b_q) / p->b_q;
    for (int a = 0; a < 3; ++a) B[a] = p->u[a] * phi + p->b2 * p->b_dir[a] * g;
}

double btrt3_oracle_C(const oracle3_problem *p, double phi)
{
    return phi + p->c3 * phi * phi * phi;
}

/* A(phi) as a full symmetric 3x3 matrix, row major. */
void btrt3_oracle_A(const oracle3_problem *p, double phi, double A[9])
{
    double s = 1.0 + p->a2 * phi * phi;
    const double *a = p->A0;
    double M[9] = {a[0], a[1], a[2], a[1], a[3], a[4], a[2], a[4], a[5]};
    for (int k = 0; k < 9; ++k) A[k] = s * M[k];
}

/* Inverse of a 3x3 matrix by cofactors; returns the determinant. */
static double inverse3(const double M[9], double Inv[9])
{
    double c00 = M[4] * M[8] - M[5] * M[7];
    double c01 = M[5] * M[6] - M[3] * M[8];
    double c02 = M[3] * M[7] - M[4] * M[6];
    double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    Inv[0] = c00 / det;
    Inv[1] = (M[2] * M[7] - M[1] * M[8]) / det;
    Inv[2] = (M[1] * M[5] - M[2] * M[4]) / det;
    Inv[3] = c01 / det;
    Inv[4] = (M[0] * M[8] - M[2] * M[6]) / det;
    Inv[5] = (M[2] * M[3] - M[0] * M[5]) / det;
    Inv[6] = c02 / det;
    Inv[7] = (M[1] * M[6] - M[0] * M[7]) / det;
    Inv[8] = (M[0] * M[4] - M[1] * M[3]) / det;
    return det;
}

/* K1 from Eq. 30: K1^{-1} = A / (cs^2 dt) + I/2. */
void btrt3_oracle_K1(const oracle3_problem *p, double phi, double K1[9])
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double A[9], M[9];
    btrt3_oracle_A(p, phi, A);
    for (int k = 0; k < 9; ++k) M[k] = A[k] / (cs2 * p->dt);
    M[0] += 0.5;
    M[4] += 0.5;
    M[8] += 0.5;
    inverse3(M, K1);
}

/* Eq. 62 at the mean first-order rate: 1/k1_eff = tr(K1^{-1}) / 3. */
double btrt3_oracle_k2(const oracle3_problem *p, const double K1[9])
{
    if (p->k2_mode == K2_3_CONST) return p->k2;
    double Kinv[9];
    inverse3(K1, Kinv);
    double k1 = 3.0 / (Kinv[0] + Kinv[4] + Kinv[8]);
    return 8.0 * (k1 - 2.0) / (3.0 * (k1 - 4.0));
}

static size_t cells3(const oracle3_problem *p) { return (size_t)p->nx * p->ny * p->nz; }

static long node3_of(const oracle3_problem *p, int ix, int iy, int iz)
{
    return ((long)iz * p->ny + iy) * p->nx + ix;
}

double btrt3_oracle_source(const oracle3_problem *p, long node, double t, double phi)
{
    if (p->src_kind == SRC3_CONST) return p->src_const;
    if (p->src_kind == SRC3_FIELD) return exp(p->src_lam * t) * p->src_field[node];
    if (p->src_kind == SRC3_REACTION) return p->react_rate * phi * (1.0 - phi_pow3(phi, p->react_exp));
    return 0.0;
}

/* ---------------------------------------------------------------- local scheme */

/* Eq. 7 in three dimensions with D = C(phi) I. */
void btrt3_oracle_feq(const oracle3_problem *p, double phi, double feq[Q3])
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double B[3];
    btrt3_oracle_B(p, phi, B);
    double D = btrt3_oracle_C(p, phi);
    for (int i = 0; i < Q3; ++i) {
        double ci[3] = {c * CX[i], c * CY[i], c * CZ[i]};
        double cB = ci[0] * B[0] + ci[1] * B[1] + ci[2] * B[2];
        double second = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double Dm = (a == b) ? (D - phi) : 0.0;
                double Qab = ci[a] * ci[b] - ((a == b) ? cs2 : 0.0);
                second += Dm * Qab;
            }
        feq[i] = weight3(i) * (phi + cB / cs2 + second / (2.0 * cs2));
    }
}

/*
 * sum_j (R_ij + P_ij) g_j of Eq. 77, built entry by entry: general K1 (row
 * major 3x3), K2 (3x3, Hadamard product with c_j c_j), lattice speed c.
 */
void btrt3_oracle_RP(double k0, const double K1[9], const double K2[9], double c, const double g[Q3],
                     double out[Q3])
{
    double cs2 = c * c / 3.0;
    for (int i = 0; i < Q3; ++i) {
        double ci[3] = {c * CX[i], c * CY[i], c * CZ[i]};
        double acc = 0.0;
        for (int j = 0; j < Q3; ++j) {
            double cj[3] = {c * CX[j], c * CY[j], c * CZ[j]};
            double Rij = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Rij += ci[a] * (K1[3 * a + b] - (a == b ? k0 : 0.0)) * cj[b];
            Rij *= weight3(i) / cs2;
            double Pij = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    Pij += (ci[a] * ci[b] - (a == b ? cs2 : 0.0)) * (K2[3 * a + b] - k0) * cj[a] * cj[b];
            Pij *= weight3(i) / (2.0 * cs2 * cs2);
            acc += (Rij + Pij) * g[j];
        }
        out[i] = acc;
    }
}

/*
 * One collision at a node (Eq. 6 with Eqs. 7, 8, 11, 30, 62, 77 and scheme 2 for
 * the source derivative).  f: pre-collision populations at time t.
 */
void btrt3_oracle_collide(const oracle3_problem *p, const double f[Q3], double phi_prev, long node,
                          double t, double t_prev, double fpost[Q3])
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double dt = p->dt;
    double phi = 0.0;
    for (int i = 0; i < Q3; ++i) phi += f[i];

    double feq[Q3], g[Q3];
    btrt3_oracle_feq(p, phi, feq);
    for (int i = 0; i < Q3; ++i) g[i] = f[i] - feq[i];

    double K1[9];
    btrt3_oracle_K1(p, phi, K1);
    double k2 = btrt3_oracle_k2(p, K1);
    double K2[9];
    for (int k = 0; k < 9; ++k) K2[k] = k2;     /* K2 = k2 Ihat */

    double rp[Q3];
    btrt3_oracle_RP(p->k0, K1, K2, c, g, rp);

    double Bn[3], Bp[3], dtB[3], Gv[3];
    btrt3_oracle_B(p, phi, Bn);
    btrt3_oracle_B(p, phi_prev, Bp);
    for (int a = 0; a < 3; ++a) dtB[a] = (Bn[a] - Bp[a]) / dt;
    for (int a = 0; a < 3; ++a) {
        Gv[a] = 0.0;
        for (int b = 0; b < 3; ++b) Gv[a] += ((a == b ? 1.0 : 0.0) - 0.5 * K1[3 * a + b]) * dtB[b];
    }
    double S = btrt3_oracle_source(p, node, t, phi);
    double Sprev = btrt3_oracle_source(p, node, t_prev, phi_prev);

    for (int i = 0; i < Q3; ++i) {
        double ci[3] = {c * CX[i], c * CY[i], c * CZ[i]};
        double G = weight3(i) * (ci[0] * Gv[0] + ci[1] * Gv[1] + ci[2] * Gv[2]) / cs2;  /* Eq. 11 */
        double Si = weight3(i) * S, Si_prev = weight3(i) * Sprev;                      /* Eq. 8 */
        double DSi = (Si - Si_prev) / dt;
        fpost[i] = f[i] - p->k0 * g[i] - rp[i] + dt * G + dt * Si + 0.5 * dt * dt * DSi;
    }
}

/* ---------------------------------------------------------------- walls */

static double wall3_term(const oracle3_problem *p, int i, double phi_w)
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double c2 = c * c * (double)(CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i]);
    double Cw = btrt3_oracle_C(p, phi_w);
    /* 2 x the even part of f_i^eq at phi_w: trace term (|c|^2 - 3 cs^2) in 3-D */
    return 2.0 * weight3(i) * (phi_w + (Cw - phi_w) * (c2 - 3.0 * cs2) / (2.0 * cs2));
}

/* Target of the link leaving (ix,iy,iz) along i: 1 and the (wrapped) node, or 0
 * and the mean of the crossed faces' wall values at t_wall. */
static int link3_target(const oracle3_problem *p, int ix, int iy, int iz, int i, double t_wall, long *target,
                        double *phi_w)
{
    int r[3] = {ix + CX[i], iy + CY[i], iz + CZ[i]};
    const int n[3] = {p->nx, p->ny, p->nz};
    double sum = 0.0;
    int crossed = 0;
    for (int a = 0; a < 3; ++a) {
        int face = -1;
        if (r[a] < 0) { if (p->bc[2 * a] == BC3_PERIODIC) r[a] += n[a]; else face = 2 * a; }
        else if (r[a] >= n[a]) { if (p->bc[2 * a + 1] == BC3_PERIODIC) r[a] -= n[a]; else face = 2 * a + 1; }
        if (face >= 0) {
            sum += p->wall[face] * exp(p->wall_lam * t_wall);
            ++crossed;
        }
    }
    if (!crossed) {
        *target = node3_of(p, r[0], r[1], r[2]);
        return 1;
    }
    *phi_w = sum / crossed;
    return 0;
}

/* ---------------------------------------------------------------- lattice */

void btrt3_oracle_init(const oracle3_problem *p, const double *phi0, double *f, double *phi_prev)
{
    size_t P = cells3(p);
    for (size_t n = 0; n < P; ++n) {
        double feq[Q3];
        btrt3_oracle_feq(p, phi0[n], feq);
        for (int i = 0; i < Q3; ++i) f[i * P + n] = feq[i];
        phi_prev[n] = phi0[n];
    }
}

void btrt3_oracle_phi(const oracle3_problem *p, const double *f, double *phi)
{
    size_t P = cells3(p);
    for (size_t n = 0; n < P; ++n) {
        double s = 0.0;
        for (int i = 0; i < Q3; ++i) s += f[i * P + n];
        phi[n] = s;
    }
}

/* One step: collide at t, then stream with bounce-back (same contract as the
 * two-dimensional oracle's step). */
int btrt3_oracle_step(const oracle3_problem *p, double *f, double *fpost, double *phi_prev, double t,
                      int first, int nthreads)
{
    const size_t P = cells3(p);
    const double t_prev = first ? t : t - p->dt;
    const long ncell = (long)P;
    (void)nthreads;

#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (long n = 0; n < ncell; ++n) {
        double fl[Q3], fp[Q3];
        double phi = 0.0;
        for (int i = 0; i < Q3; ++i) {
            fl[i] = f[i * P + n];
            phi += fl[i];
        }
        btrt3_oracle_collide(p, fl, phi_prev[n], n, t, t_prev, fp);
        for (int i = 0; i < Q3; ++i) fpost[i * P + n] = fp[i];
        phi_prev[n] = phi;
    }

#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (long n = 0; n < ncell; ++n) {
        int ix = (int)(n % p->nx), iy = (int)((n / p->nx) % p->ny), iz = (int)(n / ((long)p->nx * p->ny));
        for (int i = 0; i < Q3; ++i) {
            long tgt;
            double phi_w = 0.0;
            if (link3_target(p, ix, iy, iz, i, t + p->dt, &tgt, &phi_w))
                f[i * P + tgt] = fpost[i * P + n];
            else
                f[opposite3(i) * P + n] = -fpost[i * P + n] + wall3_term(p, i, phi_w);
        }
    }
    return 0;
}

int btrt3_oracle_run(const oracle3_problem *p, double *f, double *fpost, double *phi_prev, double t0,
                     int64_t step0, int64_t nsteps, int nthreads)
{
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t n = step0 + s;
        btrt3_oracle_step(p, f, fpost, phi_prev, t0 + (double)n * p->dt, n == 0, nthreads);
    }
    return 0;
}

/* Velocities and weights, for the tests. */
void btrt3_oracle_lattice(int *cx, int *cy, int *cz, double *w)
{
    for (int i = 0; i < Q3; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        cz[i] = CZ[i];
        w[i] = weight3(i);
    }
}
