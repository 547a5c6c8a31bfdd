/*
 * btrt3.h -- C ABI of the D3Q19 (three-dimensional) B-TriRT solver on GB300.
 *
 * The same equation, coefficient families and scheme as btrt.h in three
 * dimensions (the D3Q19 variant of the appendix: velocity set of Eq. 86,
 * relaxation matrix S_f = diag(k0, K1, k2 I_6, k0 I_9) of the D3Q19 form of
 * Eq. 96 with a 3x3 first-order block K1 = (A / (cs^2 dt) + I/2)^{-1} from
 * Eq. 30, and k2 from Eq. 62 at the mean rate 1/k1_eff = tr(K1^{-1}) / 3):
 *     d_t phi + div B(phi) = div( A(phi) grad C(phi) ) + S,
 *     B = u phi + b2 (phi^q / q) d,  C = phi + c3 phi^3,  A = (1 + a2 phi^2) A0,
 *     S = 0 | const | exp(lam t) F(x) | react_rate phi (1 - phi^react_exp).
 *
 * Conventions (as btrt.h): physical inputs, cell-centred nodes
 * x_i = x0 + (i + 1/2) dx (same spacing in y and z), arrays [nz][ny][nx] with x
 * fastest, caller-owned device workspace, status codes and btrt_last_error(),
 * device problems reported through flags read by the host, all work on the
 * stream given at creation.  Faces x-, x+, y-, y+, z-, z+ are periodic or
 * half-way bounce-back walls with one value each (times exp(wall_lam t),
 * evaluated at the end time of the step); a link that crosses two walls (an
 * edge of the box) takes the mean of the two values.
 *
 * Number formats: BTRT_F64 compute with F64 storage, or BTRT_F32 compute with
 * F32, F16 or BF16 storage in the shifted forms of btrt.h (BTRT_SHIFT_REF,
 * BTRT_SHIFT_LOCAL).  The nineteen population planes of a buffer are one array
 * with 32-bit element offsets: 19 * roundup(nx, 64) * ny * nz < 2^31.
 */
#ifndef BTRT3_H
#define BTRT3_H

#include <stddef.h>
#include <stdint.h>

#include "btrt.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct btrt3_lattice_s *btrt3_lattice;

typedef struct {
    int32_t nx, ny, nz;    /* nodes; each >= 3, 19 roundup(nx, 64) ny nz < 2^31          */
    int32_t bc[6];         /* BTRT_BC_* for faces x-, x+, y-, y+, z-, z+; opposite faces match */
    int32_t compute;       /* BTRT_F64 or BTRT_F32                                        */
    int32_t storage;       /* F64 (F64 compute) or F32, F16, BF16 (F32 compute)           */
    int32_t shift;         /* BTRT_SHIFT_REF or BTRT_SHIFT_LOCAL (F32/F16/BF16 storage)   */
    int32_t fields;        /* BTRT_FIELD_SOURCE: reserve a per-node source plane          */
    double dx, dt;         /* spacing (all axes) and time step                           */
    double x0, y0, z0;     /* lower corner of the box                                     */
    double phi_ref;        /* BTRT_SHIFT_REF: storage holds f_i - w_i phi_ref             */
} btrt3_grid_desc;

typedef struct {
    double u[3];           /* B(phi) = u phi + b2 (phi^q / q) d                           */
    double b2;
    double b_dir[3];       /* d; {0, 0, 0} selects (1, 1, 1)                              */
    double b_q;            /* q >= 1 (0 selects 2); for q != 2 the power is of max(phi, 0) */
    double c3;             /* C(phi) = phi + c3 phi^3                                     */
    double A0[6];          /* A(phi) = (1 + a2 phi^2) A0, A0 = {xx, xy, xz, yy, yz, zz}, SPD */
    double a2;
    double k0;             /* in (0, 2)                                                   */
    int32_t k2_mode;       /* BTRT_K2_HBB (Eq. 62 at 1/k1_eff = tr(K1^-1)/3) or BTRT_K2_CONST */
    int32_t src_kind;      /* BTRT_SRC_NONE, _CONST, _FIELD or _REACTION                  */
    double k2;             /* BTRT_K2_CONST, in (0, 2)                                    */
    double src_const;      /* BTRT_SRC_CONST: S                                           */
    double src_lam;        /* BTRT_SRC_FIELD: S = exp(src_lam t) F(x)                     */
    double react_rate, react_exp;   /* BTRT_SRC_REACTION: S = rate phi (1 - phi^exp)      */
    double wall[6];        /* wall value per face                                         */
    double wall_lam;       /* wall values carry exp(wall_lam t)                           */
} btrt3_coeffs;

/* Bytes of device workspace a lattice with this description needs (0: invalid). */
size_t btrt3_workspace_bytes(const btrt3_grid_desc *g);

/* Create a lattice in the caller's device workspace (>= 256-byte aligned). */
btrt_status btrt3_create(const btrt3_grid_desc *g, void *dev_workspace, size_t workspace_bytes,
                         void *cuda_stream, btrt3_lattice *out);

/* Coefficients (physical units); checked: A0 SPD, k0 and a constant k2 in (0, 2),
 * known source kind, finite values. */
btrt_status btrt3_set_coeffs(btrt3_lattice L, const btrt3_coeffs *c);

/* Per-node source field F (host, nx*ny*nz doubles, [nz][ny][nx]); needs
 * BTRT_FIELD_SOURCE in the grid description.  Synchronises the stream. */
btrt_status btrt3_set_source_field(btrt3_lattice L, const double *F_host);

/* f = f^eq(phi0) followed by the initialising collision at t0.  phi0: nx*ny*nz
 * values of dtype BTRT_F64 or BTRT_F32, on the device or the host. */
btrt_status btrt3_init_phi(btrt3_lattice L, const void *phi0, int32_t dtype, int32_t on_device, double t0);

/* Advance nsteps time steps (asynchronous on the lattice stream). */
btrt_status btrt3_step(btrt3_lattice L, int64_t nsteps);

/* phi at the current time into dst (nx*ny*nz values of dtype F64 or F32, on the
 * device or the host; a host read synchronises the stream). */
btrt_status btrt3_read_phi(btrt3_lattice L, void *dst, int32_t dtype, int32_t on_device);

/* The current post-collision populations of the box [x0, x0+w) x [y0, y0+h) x
 * [z0, z0+d) as FP64, unshifted, layout [19][d][h][w].  Synchronises. */
btrt_status btrt3_read_f(btrt3_lattice L, double *dst, int32_t x0, int32_t y0, int32_t z0, int32_t w, int32_t h,
                         int32_t d);

/* FP64 sum of phi over the box (fixed-order reduction).  Synchronises. */
btrt_status btrt3_mass(btrt3_lattice L, double *out);

/* Device flags (bit 0: a non-finite phi was produced -> BTRT_EUNSTABLE; bit 3: an
 * index check of a -DBTRT_DEBUG_BOUNDS build failed -> BTRT_ECUDA).  Synchronises. */
btrt_status btrt3_check(btrt3_lattice L, int32_t *flags);

/* Checkpoint: bytes of a saved state (header, the current populations in their
 * stored form, phi), the save (synchronises) and the load into a lattice of the
 * same grid, formats and shift (coefficients must be set first).  A resumed run
 * continues bitwise as the uninterrupted one. */
size_t btrt3_state_bytes(btrt3_lattice L);
btrt_status btrt3_save(btrt3_lattice L, void *host_buf, size_t n);
btrt_status btrt3_load(btrt3_lattice L, const void *host_buf, size_t n);

/* Steps taken since btrt3_init_phi and the current time t0 + step dt. */
btrt_status btrt3_get_time(btrt3_lattice L, int64_t *step, double *t);

/* Release the host-side handle (the workspace stays with the caller). */
btrt_status btrt3_destroy(btrt3_lattice L);

#ifdef __cplusplus
}
#endif

#endif /* BTRT3_H */
