/*
 * btrt_oracle.c -- plain FP64 CPU oracle of the block triple-relaxation-time
 * (B-TriRT) lattice Boltzmann scheme for nonlinear anisotropic
 * convection-diffusion equations on the D2Q9 lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library; it is
 * loaded by the tests, by the package smoke check and by the CPU-baseline leg of
 * the benchmark, never by the library itself.  It shares no code with the CUDA
 * path.
 *
 * Everything is written in physical units and in population space, literally
 * following the paper's equations:
 *   - lattice:         D2Q9, c_i = c e_i, weights 4/9, 1/9, 1/36, cs^2 = c^2/3 (Sec. 3, Eq. 85 rows)
 *   - equilibrium:     Eq. 7      f_i^eq = w_i [phi + c_i.B/cs^2 + (D - phi I):(c_i c_i - cs^2 I)/(2 cs^2)]
 *   - source:          Eq. 8      S_i = w_i S
 *   - correction:      Eq. 11     G_i = w_i c_i.(I - K1/2) d_t B / cs^2
 *   - evolution:       Eq. 6      f_i^+ = f_i - k0 fneq_i - w_i c_i.(K1 - k0 I) M1 / cs^2
 *                                         - w_i (c_i c_i - cs^2 I):((K2 - k0 Ihat) o M2) / (2 cs^4)
 *                                         + dt G_i + dt S_i + dt^2/2 Dbar_i S_i
 *   - source derivative, scheme 2 (gamma = 0, Remark III): Dbar_i S_i = [S_i(t) - S_i(t - dt)] / dt
 *   - K1 from A:       Eq. 30     A = cs^2 (K1^{-1} - I/2) dt
 *   - k2 from k1:      Eq. 62     k2 = 8 (k1 - 2) / (3 (k1 - 4))
 *   - streaming:       Eq. 38     f_i(x + c_i dt, t + dt) = f_i^+(x, t)
 *   - half-way bounce-back Dirichlet walls: Eqs. 54-56
 *
 * Readings where the paper is silent (each one is listed with its reason in the
 * design notes of the repository):
 *   - d_t B in G_i is the backward difference [B(phi^n) - B(phi^{n-1})] / dt,
 *     the same scheme the paper uses for d_t S (Remark III); at the first step
 *     phi^{n-1} = phi^0 and S(t - dt) = S(t), i.e. both derivatives start at zero.
 *   - K2 = k2 Ihat with k2 from Eq. 62 evaluated at k1_eff = 2 / tr(K1^{-1}),
 *     the isotropic part of K1 (exact for K1 = k1 I); or a constant k2.
 *   - The bounce-back wall term is 2 x the even part of f^eq at the wall value,
 *     2 w_i [phi_w + (C(phi_w) - phi_w)(|c_i|^2 - 2 cs^2)/(2 cs^2)]; for C = phi this
 *     is the paper's 2 w_i phi_w.  A link that crosses two walls (a corner) uses
 *     the mean of the two sides' wall values.  The wall value is taken at the
 *     time the reflected population arrives, t + dt.
 *   - Nodes are cell centred, x_i = x0 + (i + 1/2) dx.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 9

/* D2Q9 velocity set in the order of the rows of C_D2Q9 (Eq. 85). */
static const int EX[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

static double weight(int i)
{
    /* Sec. 3: w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36 */
    if (i == 0) return 4.0 / 9.0;
    if (i <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

static int opposite(int i)
{
    for (int j = 0; j < NQ; ++j)
        if (EX[j] == -EX[i] && EY[j] == -EY[i]) return j;
    return -1;
}

enum { BC_PERIODIC = 0, BC_HBB = 1 };
enum { K2_HBB = 0, K2_CONST = 1 };
enum { SRC_NONE = 0, SRC_CONST = 1, SRC_TRIG = 2, SRC_FIELD = 3, SRC_REACTION = 4 };

typedef struct {
    int32_t nx, ny;
    int32_t bc[4];            /* sides x-, x+, y-, y+ */
    double dx, dt, x0, y0;
    double u[2], b2;          /* B(phi) = u phi + b2 (phi^q / q) (d_x, d_y) */
    double c3;                /* C(phi) = phi + c3 phi^3           */
    double A0[3], a2;         /* A(phi) = (1 + a2 phi^2) A0, (xx, xy, yy) */
    double k0;
    int32_t k2_mode;
    int32_t src_kind;
    double k2;
    double src_const, src_lam, src_k;
    double src_alpha[4];      /* ss, sc, cs, cc */
    double wall[4];           /* constant wall value per side */
    double wall_lam;          /* wall values carry the time factor exp(wall_lam t) */
    const double *wall_arr[4];/* optional per-node wall values (NULL: constant) */
    const double *src_field;  /* SRC_FIELD: S = exp(src_lam t) src_field[node] */
    const double *A_field[3]; /* optional per-node diffusion tensor (xx, xy, yy): A = (1 + a2 phi^2) A(x) */
    double b_dir[2];          /* direction (d_x, d_y) of the power-law flux term */
    double b_q;               /* its exponent q (2: the quadratic family)      */
    double react_rate, react_exp; /* SRC_REACTION: S = rate phi (1 - phi^exp)  */
} oracle_problem;

/* ---------------------------------------------------------------- coefficients */

/* Row-major index of the node whose cell centre is (x, y). */
static long node_of(const oracle_problem *p, double x, double y)
{
    long ix = lround((x - p->x0) / p->dx - 0.5);
    long iy = lround((y - p->y0) / p->dx - 0.5);
    return iy * p->nx + ix;
}


/* phi^q; for q != 2 the power is taken of max(phi, 0): the power-law terms of
 * Eq. 67 are defined for phi >= 0 and an undershoot below 0 next to a steep
 * front would otherwise give a non-finite value. */
static double phi_pow(double phi, double q)
{
    if (q == 2.0) return phi * phi;
    return pow(phi > 0.0 ? phi : 0.0, q);
}

/* Eq. 1 flux family: B(phi) = u phi + b2 (phi^q / q) (d_x, d_y); q = 2 with
 * d = (1, 1) is the quadratic flux of the nonlinear tests, q = delta + 1 with
 * d = (1, 0) the Burgers-Fisher flux of Eq. 67 in conservative form. */
void btrt_oracle_B(const oracle_problem *p, double phi, double B[2])
{
    double g = phi_pow(phi, p->b_q) / p->b_q;
    B[0] = p->u[0] * phi + p->b2 * p->b_dir[0] * g;
    B[1] = p->u[1] * phi + p->b2 * p->b_dir[1] * g;
}

double btrt_oracle_C(const oracle_problem *p, double phi)
{
    return phi + p->c3 * phi * phi * phi;
}

/* A(phi) as a full 2x2 matrix, row major. */
void btrt_oracle_A(const oracle_problem *p, double phi, double A[4])
{
    double s = 1.0 + p->a2 * phi * phi;
    A[0] = s * p->A0[0];
    A[1] = s * p->A0[1];
    A[2] = s * p->A0[1];
    A[3] = s * p->A0[2];
}

/* K1 from Eq. 30: K1^{-1} = A / (cs^2 dt) + I/2, inverted as a 2x2 matrix. */
static void k1_of_A(const oracle_problem *p, const double A[4], double K1[4])
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double M[4];
    for (int k = 0; k < 4; ++k) M[k] = A[k] / (cs2 * p->dt);
    M[0] += 0.5;
    M[3] += 0.5;
    double det = M[0] * M[3] - M[1] * M[2];
    K1[0] = M[3] / det;
    K1[1] = -M[1] / det;
    K1[2] = -M[2] / det;
    K1[3] = M[0] / det;
}

/* K1 of Eq. 30 for the uniform tensor A(phi). */
void btrt_oracle_K1(const oracle_problem *p, double phi, double K1[4])
{
    double A[4];
    btrt_oracle_A(p, phi, A);
    k1_of_A(p, A, K1);
}

/* A(x, phi) at the node centred at (x, y): the per-node tensor when one is given. */
void btrt_oracle_A_at(const oracle_problem *p, double phi, double x, double y, double A[4])
{
    if (!p->A_field[0]) {
        btrt_oracle_A(p, phi, A);
        return;
    }
    long n = node_of(p, x, y);
    double s = 1.0 + p->a2 * phi * phi;
    A[0] = s * p->A_field[0][n];
    A[1] = s * p->A_field[1][n];
    A[2] = s * p->A_field[1][n];
    A[3] = s * p->A_field[2][n];
}

/* K1 from Eq. 30 at the node centred at (x, y). */
void btrt_oracle_K1_at(const oracle_problem *p, double phi, double x, double y, double K1[4])
{
    double A[4];
    btrt_oracle_A_at(p, phi, x, y, A);
    k1_of_A(p, A, K1);
}

/* Eq. 62 */
double btrt_oracle_k2_from_k1(double k1)
{
    return 8.0 * (k1 - 2.0) / (3.0 * (k1 - 4.0));
}

double btrt_oracle_k2(const oracle_problem *p, const double K1[4])
{
    if (p->k2_mode == K2_CONST) return p->k2;
    /* k1_eff: 1/k1_eff = tr(K1^{-1}) / 2 */
    double det = K1[0] * K1[3] - K1[1] * K1[2];
    double tr_inv = (K1[3] + K1[0]) / det;
    return btrt_oracle_k2_from_k1(2.0 / tr_inv);
}

/* S(x, t, phi); the reaction kind is the logistic-type term of Eq. 67. */
double btrt_oracle_source(const oracle_problem *p, double x, double y, double t, double phi)
{
    if (p->src_kind == SRC_NONE) return 0.0;
    if (p->src_kind == SRC_CONST) return p->src_const;
    if (p->src_kind == SRC_REACTION) return p->react_rate * phi * (1.0 - phi_pow(phi, p->react_exp));
    if (p->src_kind == SRC_FIELD) return exp(p->src_lam * t) * p->src_field[node_of(p, x, y)];
    double sx = sin(p->src_k * x), cx = cos(p->src_k * x);
    double sy = sin(p->src_k * y), cy = cos(p->src_k * y);
    return exp(p->src_lam * t) * (p->src_alpha[0] * sx * sy + p->src_alpha[1] * sx * cy +
                                  p->src_alpha[2] * cx * sy + p->src_alpha[3] * cx * cy);
}

/* ---------------------------------------------------------------- local scheme */

/* Eq. 7 with D = C(phi) I. */
void btrt_oracle_feq(const oracle_problem *p, double phi, double feq[NQ])
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double B[2];
    btrt_oracle_B(p, phi, B);
    double D = btrt_oracle_C(p, phi);
    for (int i = 0; i < NQ; ++i) {
        double ci[2] = {c * EX[i], c * EY[i]};
        double cB = ci[0] * B[0] + ci[1] * B[1];
        /* (D - phi I):(c_i c_i - cs^2 I) with D - phi I = (C - phi) I */
        double second = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double Dm = (a == b) ? (D - phi) : 0.0;
                double Q = ci[a] * ci[b] - ((a == b) ? cs2 : 0.0);
                second += Dm * Q;
            }
        feq[i] = weight(i) * (phi + cB / cs2 + second / (2.0 * cs2));
    }
}

/*
 * The relaxation part of Eq. 6 as a function of f^neq:
 *   out_i = k0 fneq_i + w_i c_i.(K1 - k0 I) M1 / cs^2
 *         + w_i (c_i c_i - cs^2 I):((K2 - k0 Ihat) o M2) / (2 cs^4)
 * with M1 = sum_j c_j fneq_j, M2 = sum_j c_j c_j fneq_j.  K1, K2 are general
 * 2x2 matrices (row major), as allowed by Eq. 98.
 */
void btrt_oracle_relax(double k0, const double K1[4], const double K2[4], double c,
                       const double fneq[NQ], double out[NQ])
{
    double cs2 = c * c / 3.0;
    double M1[2] = {0.0, 0.0};
    double M2[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int j = 0; j < NQ; ++j) {
        double cj[2] = {c * EX[j], c * EY[j]};
        for (int a = 0; a < 2; ++a) {
            M1[a] += cj[a] * fneq[j];
            for (int b = 0; b < 2; ++b) M2[a][b] += cj[a] * cj[b] * fneq[j];
        }
    }
    double QM1[2];
    for (int a = 0; a < 2; ++a) {
        QM1[a] = 0.0;
        for (int b = 0; b < 2; ++b) QM1[a] += (K1[2 * a + b] - ((a == b) ? k0 : 0.0)) * M1[b];
    }
    double HM2[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) HM2[a][b] = (K2[2 * a + b] - k0) * M2[a][b];
    for (int i = 0; i < NQ; ++i) {
        double ci[2] = {c * EX[i], c * EY[i]};
        double first = (ci[0] * QM1[0] + ci[1] * QM1[1]) / cs2;
        double second = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                second += (ci[a] * ci[b] - ((a == b) ? cs2 : 0.0)) * HM2[a][b];
        second /= (2.0 * cs2 * cs2);
        out[i] = k0 * fneq[i] + weight(i) * first + weight(i) * second;
    }
}

/*
 * One collision at a node (Eq. 6 with Eqs. 7, 8, 11, 30, 62 and scheme 2 for
 * the source derivative).  f: pre-collision populations at time t; phi_prev:
 * phi at t - dt; t_prev: time at which the previous source is evaluated.
 */
void btrt_oracle_collide(const oracle_problem *p, const double f[NQ], double phi_prev,
                         double x, double y, double t, double t_prev, double fpost[NQ])
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double dt = p->dt;
    double phi = 0.0;
    for (int i = 0; i < NQ; ++i) phi += f[i];

    double feq[NQ], fneq[NQ];
    btrt_oracle_feq(p, phi, feq);
    for (int i = 0; i < NQ; ++i) fneq[i] = f[i] - feq[i];

    double K1[4];
    btrt_oracle_K1_at(p, phi, x, y, K1);
    double k2 = btrt_oracle_k2(p, K1);
    double K2[4] = {k2, k2, k2, k2}; /* K2 = k2 Ihat */

    double relax[NQ];
    btrt_oracle_relax(p->k0, K1, K2, c, fneq, relax);

    /* d_t B by a backward difference */
    double Bn[2], Bp[2], dtB[2];
    btrt_oracle_B(p, phi, Bn);
    btrt_oracle_B(p, phi_prev, Bp);
    for (int a = 0; a < 2; ++a) dtB[a] = (Bn[a] - Bp[a]) / dt;
    /* (I - K1/2) d_t B */
    double Gv[2];
    for (int a = 0; a < 2; ++a) {
        Gv[a] = 0.0;
        for (int b = 0; b < 2; ++b) Gv[a] += (((a == b) ? 1.0 : 0.0) - 0.5 * K1[2 * a + b]) * dtB[b];
    }

    double S = btrt_oracle_source(p, x, y, t, phi);
    double Sprev = btrt_oracle_source(p, x, y, t_prev, phi_prev);

    for (int i = 0; i < NQ; ++i) {
        double ci[2] = {c * EX[i], c * EY[i]};
        double G = weight(i) * (ci[0] * Gv[0] + ci[1] * Gv[1]) / cs2;       /* Eq. 11 */
        double Si = weight(i) * S;                                           /* Eq. 8  */
        double Si_prev = weight(i) * Sprev;
        double DSi = (Si - Si_prev) / dt;                                    /* scheme 2 */
        fpost[i] = f[i] - relax[i] + dt * G + dt * Si + 0.5 * dt * dt * DSi;
    }
}

/* ---------------------------------------------------------------- walls */

/* Wall value of `side` next to node index `idx` along that side, at time t. */
static double wall_value(const oracle_problem *p, int side, int idx, double t)
{
    double v = p->wall_arr[side] ? p->wall_arr[side][idx] : p->wall[side];
    return v * exp(p->wall_lam * t);
}

/* 2 x even part of f_i^eq at the wall value (bounce-back source term, Eqs. 54-56). */
static double wall_term(const oracle_problem *p, int i, double phi_w)
{
    double c = p->dx / p->dt;
    double cs2 = c * c / 3.0;
    double c2 = c * c * (double)(EX[i] * EX[i] + EY[i] * EY[i]);
    double Cw = btrt_oracle_C(p, phi_w);
    return 2.0 * weight(i) * (phi_w + (Cw - phi_w) * (c2 - 2.0 * cs2) / (2.0 * cs2));
}

/*
 * Where does the population leaving node (ix, iy) in direction i go?
 * Returns 1 and the (wrapped) target node if it stays in the domain; returns 0
 * and the wall value if it crosses a bounce-back wall.
 */
static int link_target(const oracle_problem *p, int ix, int iy, int i, double t_wall,
                       int *tx, int *ty, double *phi_w)
{
    int x = ix + EX[i], y = iy + EY[i];
    int cross_x = 0, cross_y = 0;
    int side_x = -1, side_y = -1;
    if (x < 0) { if (p->bc[0] == BC_PERIODIC) x += p->nx; else { cross_x = 1; side_x = 0; } }
    if (x >= p->nx) { if (p->bc[1] == BC_PERIODIC) x -= p->nx; else { cross_x = 1; side_x = 1; } }
    if (y < 0) { if (p->bc[2] == BC_PERIODIC) y += p->ny; else { cross_y = 1; side_y = 2; } }
    if (y >= p->ny) { if (p->bc[3] == BC_PERIODIC) y -= p->ny; else { cross_y = 1; side_y = 3; } }
    if (!cross_x && !cross_y) {
        *tx = x;
        *ty = y;
        return 1;
    }
    if (cross_x && cross_y)
        *phi_w = 0.5 * (wall_value(p, side_x, iy, t_wall) + wall_value(p, side_y, ix, t_wall));
    else if (cross_y)
        *phi_w = wall_value(p, side_y, ix, t_wall);
    else
        *phi_w = wall_value(p, side_x, iy, t_wall);
    return 0;
}

/* ---------------------------------------------------------------- lattice */

static size_t plane(const oracle_problem *p) { return (size_t)p->nx * (size_t)p->ny; }

static double node_x(const oracle_problem *p, int ix) { return p->x0 + (ix + 0.5) * p->dx; }
static double node_y(const oracle_problem *p, int iy) { return p->y0 + (iy + 0.5) * p->dx; }

/* f = f^eq(phi0) (Sec. 4, initialisation); phi_prev = phi0. */
void btrt_oracle_init(const oracle_problem *p, const double *phi0, double *f, double *phi_prev)
{
    size_t P = plane(p);
    for (size_t n = 0; n < P; ++n) {
        double feq[NQ];
        btrt_oracle_feq(p, phi0[n], feq);
        for (int i = 0; i < NQ; ++i) f[i * P + n] = feq[i];
        phi_prev[n] = phi0[n];
    }
}

void btrt_oracle_phi(const oracle_problem *p, const double *f, double *phi)
{
    size_t P = plane(p);
    for (size_t n = 0; n < P; ++n) {
        double s = 0.0;
        for (int i = 0; i < NQ; ++i) s += f[i * P + n];
        phi[n] = s;
    }
}

/*
 * One time step: collide every node at time t (Eq. 6), then stream (Eq. 38)
 * with half-way bounce-back at walls (Eqs. 54-56).  f holds the pre-collision
 * populations at t on entry and at t + dt on return; fpost receives the
 * post-collision populations at t; phi_prev holds phi at t - dt on entry and
 * phi at t on return.  first != 0 marks the first step (zero time derivatives).
 */
int btrt_oracle_step(const oracle_problem *p, double *f, double *fpost, double *phi_prev,
                     double t, int first, int nthreads)
{
    const size_t P = plane(p);
    const int nx = p->nx, ny = p->ny;
    const double t_prev = first ? t : t - p->dt;
    (void)nthreads;

#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int iy = 0; iy < ny; ++iy) {
        for (int ix = 0; ix < nx; ++ix) {
            size_t n = (size_t)iy * nx + ix;
            double fl[NQ], fp[NQ];
            double phi = 0.0;
            for (int i = 0; i < NQ; ++i) {
                fl[i] = f[i * P + n];
                phi += fl[i];
            }
            btrt_oracle_collide(p, fl, phi_prev[n], node_x(p, ix), node_y(p, iy), t, t_prev, fp);
            for (int i = 0; i < NQ; ++i) fpost[i * P + n] = fp[i];
            phi_prev[n] = phi;
        }
    }

#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int iy = 0; iy < ny; ++iy) {
        for (int ix = 0; ix < nx; ++ix) {
            size_t n = (size_t)iy * nx + ix;
            for (int i = 0; i < NQ; ++i) {
                int tx, ty;
                double phi_w = 0.0;
                if (link_target(p, ix, iy, i, t + p->dt, &tx, &ty, &phi_w)) {
                    f[i * P + (size_t)ty * nx + tx] = fpost[i * P + n];
                } else {
                    int o = opposite(i);
                    f[o * P + n] = -fpost[i * P + n] + wall_term(p, i, phi_w);
                }
            }
        }
    }
    return 0;
}

/* Run nsteps from the current state (convenience loop around btrt_oracle_step). */
int btrt_oracle_run(const oracle_problem *p, double *f, double *fpost, double *phi_prev,
                    double t0, int64_t step0, int64_t nsteps, int nthreads)
{
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t n = step0 + s;
        btrt_oracle_step(p, f, fpost, phi_prev, t0 + (double)n * p->dt, n == 0, nthreads);
    }
    return 0;
}

/*
 * The same step for one node, in pull form, from a 3x3 window of post-collision
 * populations at t: win[(dy+1)*3 + (dx+1)][i] holds f_i^+ at (ix+dx, iy+dy)
 * (periodically wrapped by the caller; entries beyond a wall are ignored).
 * Produces the post-collision populations at t + dt and phi at t + dt.
 */
void btrt_oracle_node_step(const oracle_problem *p, const double *win, int ix, int iy,
                           double phi_prev, double t_next, double fpost[NQ], double *phi_out)
{
    double fl[NQ];
    for (int i = 0; i < NQ; ++i) {
        /* the population arriving in direction i left the node x - e_i in direction i;
           seen from this node, that is the link in direction opposite(i) */
        int o = opposite(i);
        int tx, ty;
        double phi_w = 0.0;
        if (link_target(p, ix, iy, o, t_next, &tx, &ty, &phi_w)) {
            fl[i] = win[((1 - EY[i]) * 3 + (1 - EX[i])) * NQ + i];
        } else {
            /* this node's own population leaving in direction o hits the wall and
               comes back in direction i (Eqs. 54-56) */
            fl[i] = -win[(1 * 3 + 1) * NQ + o] + wall_term(p, o, phi_w);
        }
    }
    double phi = 0.0;
    for (int i = 0; i < NQ; ++i) phi += fl[i];
    btrt_oracle_collide(p, fl, phi_prev, node_x(p, ix), node_y(p, iy), t_next, t_next - p->dt, fpost);
    *phi_out = phi;
}

int btrt_oracle_num_velocities(void) { return NQ; }
