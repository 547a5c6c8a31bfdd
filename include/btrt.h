/*
 * btrt.h -- C ABI of the GB300 (sm_103a) block triple-relaxation-time (B-TriRT)
 * lattice Boltzmann solver for nonlinear anisotropic convection-diffusion
 * equations on the D2Q9 lattice.
 *
 * The equation solved is
 *     d_t phi + div B(phi) = div( A(phi) grad C(phi) ) + S(x, t)            (Eq. 1, Eq. 29)
 * with B(phi) = u phi + b2 (phi^q/q) d (q = 2 and d = (1,1) by default),
 * C(phi) = phi + c3 phi^3 (the paper's D = C I), A(phi) = (1 + a2 phi^2) A0, and
 * S = 0, a constant, a separable trigonometric field exp(lam t) sum_pq
 * alpha_pq X_p(k x) Y_q(k y), a per-node field exp(lam t) F(x), or the reaction
 * term rate phi (1 - phi^exp) of the Burgers-Fisher equation (Eq. 67).
 *
 * One time step is one fused sweep (stream + collide, Eq. 38 with Eq. 6):
 * pull the nine populations, take phi, evaluate B, C, A, build the first-order
 * relaxation block K1 = (A / (cs^2 dt) + I/2)^{-1} from Eq. 30, take k2 from
 * Eq. 62, relax the three blocks (Eqs. 94-95, 99), add the convective correction
 * (Eq. 11) and the source (Eq. 8, scheme 2 of Remark III), write back, and apply
 * half-way bounce-back Dirichlet walls (Eqs. 54-56).
 *
 * Conventions
 *  - All inputs are physical; the library converts to lattice units internally.
 *  - Nodes are cell centred: x_i = x0 + (i + 1/2) dx, y_j = y0 + (j + 1/2) dx.
 *  - Arrays of nodes are row major [ny][nx] (x fastest).
 *  - Velocity order: c0 = (0,0), c1 = (1,0), c2 = (0,1), c3 = (-1,0), c4 = (0,-1),
 *    c5 = (1,1), c6 = (-1,1), c7 = (-1,-1), c8 = (1,-1) (rows of Eq. 85).
 *  - Every function returns a btrt_status; on failure btrt_last_error() returns a
 *    thread-local message.  No function aborts, throws or traps; device-side
 *    problems are reported through flags that the host reads.
 *  - Device memory is owned by the caller: btrt_create borrows a workspace of
 *    btrt_workspace_bytes() bytes and never frees it.  The library itself never
 *    allocates device memory.
 *  - All work is enqueued on the CUDA stream given at creation (0 = legacy
 *    default stream); functions that return host values synchronise that stream.
 */
#ifndef BTRT_H
#define BTRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BTRT_OK = 0,
    BTRT_EINVAL = -1,     /* invalid argument or unstable parameter set */
    BTRT_ENOMEM = -2,     /* workspace or host buffer too small           */
    BTRT_ECUDA = -3,      /* a CUDA runtime call failed                   */
    BTRT_EUNSTABLE = -4,  /* non-finite phi detected on the device        */
    BTRT_ETIMEOUT = -5,   /* a bounded device wait gave up                */
    BTRT_ESTATE = -6      /* call out of order (e.g. step before init)    */
} btrt_status;

enum { BTRT_BC_PERIODIC = 0, BTRT_BC_HBB = 1 };                 /* boundary kinds     */
/* number formats; BTRT_DF64 is double-word arithmetic and storage (a value is
 * the unevaluated sum of two FP32 numbers, ~48 significant bits) */
enum { BTRT_F64 = 0, BTRT_F32 = 1, BTRT_F16 = 2, BTRT_BF16 = 3, BTRT_DF64 = 4 };
enum { BTRT_K2_HBB = 0, BTRT_K2_CONST = 1 };                    /* second-order block */
enum { BTRT_SRC_NONE = 0, BTRT_SRC_CONST = 1, BTRT_SRC_TRIG = 2, BTRT_SRC_FIELD = 3, BTRT_SRC_REACTION = 4 };
enum { BTRT_FIELD_SOURCE = 1, BTRT_FIELD_DIFFUSION = 2 };      /* btrt_grid_desc.fields bits */
enum { BTRT_SIDE_XMIN = 0, BTRT_SIDE_XMAX = 1, BTRT_SIDE_YMIN = 2, BTRT_SIDE_YMAX = 3 };
/* Stored form of F32/F16/BF16 populations (btrt_grid_desc.shift):
 *  BTRT_SHIFT_REF    f_i - w_i phi_ref, one reference value per lattice;
 *  BTRT_SHIFT_LOCAL  f_i^+(x) - w_i phi(x), relative to the phi of the node that
 *                    wrote the population; the sweep adds w_i phi(x - e_i) back
 *                    from the previous phi plane.  What is rounded is then of the
 *                    size of the non-equilibrium part only, which keeps F16/BF16
 *                    storage far closer to the FP32-storage result.
 *  BTRT_SHIFT_LOCAL_DW as BTRT_SHIFT_LOCAL, with phi kept as a double-word pair
 *                    (two FP32 planes, high and low word; 8 more bytes per update):
 *                    phi is never rounded to FP32, which under diffusive scaling on
 *                    fine grids (a step changes phi by a few FP32 ulps) keeps FP32
 *                    storage within the FP64 discretisation error.  Plain kernel
 *                    form only (BTRT_SWEEP_AUTO / PLAIN); not in batches.
 *  BTRT_SHIFT_LOCAL_SR as BTRT_SHIFT_LOCAL, F16/BF16 storage only, with the stored
 *                    deviations rounded stochastically: up with probability equal to
 *                    the fraction of the last place cut off, from random bits that
 *                    depend only on the node, the step index and the population.
 *                    Under diffusive scaling a step changes the state by far less
 *                    than a 16-bit last place, and round-to-nearest then repeats
 *                    nearly the same error step after step; stochastic rounding
 *                    makes each stored value right on average.  FP16 deviations
 *                    are stored scaled by 2^12 (exact), which keeps the small
 *                    deviations of fine grids out of FP16's subnormal range; their
 *                    magnitude must stay below 16.  Plain and vector kernel forms
 *                    (AUTO takes the vector form from 2^21 nodes on); in batches
 *                    every form but two steps per launch.
 *  BTRT_SHIFT_LOCAL_DW_SR both: double-word phi and stochastically rounded F16/BF16
 *                    deviations.  Plain kernel form only; not in batches.
 *  BTRT_SHIFT_MOMENT_SR F16/BF16: f_i^+(x) - w_i (phi(x) + 3 e_i . j(x)), j the
 *                    writer's post-collision first moment, kept in two more planes
 *                    of the storage format (8 more bytes per update), the value
 *                    rounded stochastically.  What is stored is then about 1/dx
 *                    smaller than with the local shift (the first-moment part of
 *                    the non-equilibrium populations is taken out); the new phi is
 *                    rounded to its FP32 plane stochastically as well (its exact
 *                    value is phi + the TwoSum error of the collision's sum).
 *                    Plain and vector kernel forms (AUTO: the vector form from
 *                    2^21 nodes on); not in batches.
 * FP64 and double-word storage are never shifted. */
enum { BTRT_SHIFT_REF = 0, BTRT_SHIFT_LOCAL = 1, BTRT_SHIFT_LOCAL_DW = 2, BTRT_SHIFT_LOCAL_SR = 3,
       BTRT_SHIFT_LOCAL_DW_SR = 4, BTRT_SHIFT_MOMENT_SR = 5 };

typedef struct btrt_lattice_s *btrt_lattice;

/* Grid, number formats and the shift of reduced-precision storage. */
typedef struct {
    int32_t nx, ny;        /* nodes; 3 <= nx, ny <= 65536 and 9 ny roundup(nx, 64) < 2^31 */
    int32_t bc[4];         /* BTRT_BC_* for sides x-, x+, y-, y+; opposite sides match  */
    int32_t compute;       /* BTRT_F64, BTRT_DF64 or BTRT_F32: arithmetic of the sweep  */
    int32_t storage;       /* populations: F64 (F64 compute), DF64 (DF64 compute), or
                              F32, F16, BF16 (F32 compute)                               */
    double dx, dt;         /* physical spacing and time step (c = dx/dt, cs^2 = c^2/3)  */
    double x0, y0;         /* physical position of the lower-left domain corner         */
    double phi_ref;        /* BTRT_SHIFT_REF: F32/F16/BF16 storage holds f_i - w_i phi_ref  */
    int32_t fields;        /* BTRT_FIELD_* bits: reserve per-node source / diffusion planes */
    int32_t shift;         /* BTRT_SHIFT_* (F32/F16/BF16 storage; _SR forms F16/BF16)     */
} btrt_grid_desc;

/* Coefficients of Eq. 1 and the relaxation parameters (physical units). */
typedef struct {
    double u[2];           /* B(phi) = u phi + b2 (phi^q / q) (d_x, d_y)         */
    double b2;
    double c3;             /* C(phi) = phi + c3 phi^3                             */
    double A0[3];          /* A(phi) = (1 + a2 phi^2) A0; A0 = {xx, xy, yy}, SPD  */
    double a2;
    double k0;             /* relaxation of the remaining moments, in (0, 2)      */
    int32_t k2_mode;       /* BTRT_K2_HBB: Eq. 62 at k1_eff = 2/tr(K1^-1); CONST   */
    int32_t src_kind;      /* BTRT_SRC_*                                          */
    double k2;             /* used when k2_mode == BTRT_K2_CONST, in (0, 2)       */
    double src_const;      /* BTRT_SRC_CONST: S = src_const                       */
    double src_lam, src_k; /* BTRT_SRC_TRIG: S = exp(lam t) sum alpha_pq X_p Y_q;
                              BTRT_SRC_FIELD: S = exp(lam t) F(x) (btrt_set_source_field) */
    double src_alpha[4];   /*   {ss, sc, cs, cc}: X_s = sin(k x), X_c = cos(k x)  */
    double wall_lam;       /* wall values carry the factor exp(wall_lam t)        */
    double b_dir[2];       /* d of the power-law flux term; {0, 0} selects (1, 1) */
    double b_q;            /* its exponent q >= 1 (0 selects 2); for q != 2 the power
                              is taken of max(phi, 0)                              */
    double react_rate;     /* BTRT_SRC_REACTION: S = react_rate phi (1 - phi^react_exp),
                              with the same scheme-2 time derivative as the other
                              sources, S^{n-1} taken at phi^{n-1}                 */
    double react_exp;      /*   > 0; for an exponent other than 2 the power is taken
                              of max(phi, 0)                                       */
} btrt_coeffs;

/* Bytes of device workspace a lattice with this description needs.  Returns 0
 * for an invalid description (see btrt_last_error). */
size_t btrt_workspace_bytes(const btrt_grid_desc *g);

/* Create a lattice in the caller's workspace (device pointer, >= 256-byte
 * aligned, btrt_workspace_bytes(g) bytes).  cuda_stream is a cudaStream_t (may
 * be NULL for the default stream).  The workspace stays owned by the caller and
 * must outlive the lattice. */
btrt_status btrt_create(const btrt_grid_desc *g, void *dev_workspace, size_t workspace_bytes,
                        void *cuda_stream, btrt_lattice *out);

/* Set the coefficients (Eq. 1), k0 and the k2 rule.  Checks that A0 is SPD, k0
 * and k2 are in (0, 2) and that the first-order block is stable at phi = 0;
 * otherwise BTRT_EINVAL.  May be called again between steps. */
btrt_status btrt_set_coeffs(btrt_lattice L, const btrt_coeffs *c);

/* Dirichlet value phi_w of a bounce-back side (Eqs. 54-56).  n == 1: one value
 * for the whole side; n == side length (nx for y sides, ny for x sides): one
 * value per boundary node, read from host memory and copied.  The value used at
 * a step is phi_w * exp(wall_lam * t_{n+1}). */
btrt_status btrt_set_boundary(btrt_lattice L, int32_t side, const double *phi_w_host, int32_t n);

/* Per-node source field F(x) for BTRT_SRC_FIELD: nx*ny values in host memory,
 * row major; needs BTRT_FIELD_SOURCE in the grid description. */
btrt_status btrt_set_source_field(btrt_lattice L, const double *F_host);

/* Spatially varying diffusion tensor (physical units, nx*ny values each, row
 * major, host memory): A(x, phi) = (1 + a2 phi^2) A(x) replaces A0.  Every node's
 * tensor must be symmetric positive definite.  Needs BTRT_FIELD_DIFFUSION; the
 * first-order block K1 (Eq. 30) and k2 are then built at every node. */
btrt_status btrt_set_diffusion_field(btrt_lattice L, const double *Axx, const double *Axy, const double *Ayy);

/* Initial state f_i = f_i^eq(phi0) at time t0 (Sec. 4).  phi0: nx*ny values of
 * dtype BTRT_F64 or BTRT_F32, in host memory (on_device = 0) or device memory
 * (on_device = 1), row major without padding.  The first collision (at t0) is
 * performed here; afterwards the lattice is at step 0. */
btrt_status btrt_init_phi(btrt_lattice L, const void *phi0, int32_t dtype, int32_t on_device,
                          double t0);

/* Advance nsteps time steps (asynchronous on the lattice's stream). */
btrt_status btrt_step(btrt_lattice L, int64_t nsteps);

/* Advance nsteps >= 1 steps and return ||phi^n - phi^{n-1}||_2 of the last one
 * (FP64, fixed reduction order; the steady-state measure of the serving loop,
 * cf. Eq. 64).  Synchronises. */
btrt_status btrt_step_residual(btrt_lattice L, int64_t nsteps, double *residual);

/* Copy phi (nx*ny values, dtype F64 or F32) to host (on_device = 0, synchronises)
 * or device memory (on_device = 1, asynchronous). */
btrt_status btrt_read_phi(btrt_lattice L, void *dst, int32_t dtype, int32_t on_device);

/* Copy the current post-collision populations of a window [x0, x0+w) x [y0, y0+h)
 * to host memory as FP64, layout [9][h][w] (undone storage shift).  Synchronises. */
btrt_status btrt_read_f(btrt_lattice L, double *dst_host, int32_t x0, int32_t y0, int32_t w,
                        int32_t h);

/* Sum of phi over all nodes, in FP64 with a fixed reduction order (deterministic).
 * Synchronises. */
btrt_status btrt_mass(btrt_lattice L, double *out);

/* Flags raised by the sweep since the last btrt_init_phi: bit 0 = some node
 * produced a NaN/Inf phi (returns BTRT_EUNSTABLE), bit 2 = a bounded wait for a
 * tile copy gave up (returns BTRT_ETIMEOUT), bit 3 = an index check of a
 * -DBTRT_DEBUG_BOUNDS build failed (returns BTRT_ECUDA).  Synchronises. */
btrt_status btrt_check(btrt_lattice L, int32_t *flags);

/* Kernel form of the ordinary FP32-compute sweep: BTRT_SWEEP_AUTO (default: the
 * faster form as measured on GB300: BTRT_SWEEP_VEC for F16/BF16 storage on
 * lattices of 2^21 nodes or more, BTRT_SWEEP_TB2 otherwise), BTRT_SWEEP_PLAIN
 * (one step per launch, direct global loads served by L1/L2), BTRT_SWEEP_TMA
 * (persistent tiles staged in shared memory by TMA with mbarrier pipelining) or
 * BTRT_SWEEP_TB2 (two time steps per launch: the first step's populations stay
 * in shared memory, halving the DRAM bytes per step; btrt_step runs pairs of
 * steps this way and an odd last step, and btrt_step_residual its last step, in
 * the plain form), or BTRT_SWEEP_VEC (one step per launch; each thread owns four
 * x-consecutive nodes and moves each population plane with one vector load and
 * one vector store, 64 bits for F16/BF16 storage and 128 for F32; the
 * initialising collision and btrt_step_residual's last step run in the plain
 * form), or BTRT_SWEEP_TB2V (two steps per launch as BTRT_SWEEP_TB2, with the
 * vector access of BTRT_SWEEP_VEC in both steps and the intermediate step kept
 * in shared memory in the storage format).  Every storage format and shift of
 * an FP32-compute lattice.  All forms give bitwise identical results.  FP64 and
 * double-word lattices always use the plain form (BTRT_SWEEP_TMA, _TB2, _VEC and
 * _TB2V: BTRT_EINVAL). */
enum {
    BTRT_SWEEP_AUTO = 0, BTRT_SWEEP_PLAIN = 1, BTRT_SWEEP_TMA = 2, BTRT_SWEEP_TB2 = 3, BTRT_SWEEP_VEC = 4,
    BTRT_SWEEP_TB2V = 5
};
btrt_status btrt_set_sweep_variant(btrt_lattice L, int32_t variant);

/* Number of completed steps and the current time t0 + n dt. */
btrt_status btrt_get_time(btrt_lattice L, int64_t *step, double *t);

/* Checkpoint: bytes needed, save the full state (populations, phi, step) to
 * host memory, load it back.  A resumed run is bitwise equal to an
 * uninterrupted one.  Synchronises. */
size_t btrt_state_bytes(btrt_lattice L);
btrt_status btrt_save(btrt_lattice L, void *host_buf, size_t n);
btrt_status btrt_load(btrt_lattice L, const void *host_buf, size_t n);

/* Release the host-side handle (the workspace stays with the caller).
 * BTRT_ESTATE while a batch still references the lattice. */
btrt_status btrt_destroy(btrt_lattice L);

/* ---------------------------------------------------------------- batches
 * Many independent lattices of uneven size advanced together: one persistent
 * cooperative kernel per call (all members, all tiles, every step; a bounded
 * grid barrier between steps), or one launch per step over all tiles, either
 * captured in a CUDA graph per (steps, residual) pair and replayed.  Members keep their own workspaces and stay usable with the
 * single-lattice calls; they must be initialised, share compute and storage
 * formats and outlive the batch.  Each member's results are bitwise identical to
 * stepping it alone (the per-node arithmetic does not depend on the tiling). */
typedef struct btrt_batch_s *btrt_batch;

/* Device workspace (descriptors, tile table, reduction scratch) for a batch of
 * these members; 0 if the member list is invalid. */
size_t btrt_batch_workspace_bytes(const btrt_lattice *members, int32_t n);

/* The same size for a batch of lattices with these n grid descriptions (no
 * lattice needed): lets an admission policy count the batch tables of a
 * membership before it creates the lattices.  0 if a description is invalid or
 * they mix compute formats. */
size_t btrt_batch_workspace_bytes_desc(const btrt_grid_desc *descs, int32_t n);

/* Create a batch over n members in a caller-owned, 256-byte aligned device
 * workspace.  Synchronises the members' streams; the batch's own work goes to
 * cuda_stream (it may be the legacy default stream: slice graphs are captured on
 * a private stream and replayed on this one).  Members take FP64 or FP32 compute
 * of one format and one storage shift; no double-word phi or first-moment planes
 * (BTRT_SHIFT_LOCAL_DW, _DW_SR, _MOMENT_SR: BTRT_EINVAL).  Requires
 * cooperative-launch support. */
btrt_status btrt_batch_create(const btrt_lattice *members, int32_t n, void *dev_workspace, size_t bytes,
                              void *cuda_stream, btrt_batch *out);

/* Tile shape: block_x x block_y threads, each sweeping `rows` nodes of its
 * column.  Candidates: 32x8x1, 32x8x2, 32x8x4, 64x4x1, 64x4x2, 32x4x2, 16x16x1,
 * 8x32x1, 32x4x4, 16x8x2.  per_step_launch = 0: persistent launch per call; 1: one launch per
 * step; 2 (FP32-compute batches only, else BTRT_EINVAL): two steps per launch on
 * 32 x 16 output tiles (the form of BTRT_SWEEP_TB2), an odd last step and the
 * residual step of btrt_batch_step in the form of 1 with the given shape;
 * 3 (FP32-compute batches only): one launch per step in the vector form of
 * BTRT_SWEEP_VEC on tiles of (4 block_x) x (block_y rows) nodes, the residual
 * step in the form of 1.  Stochastically rounded members (BTRT_SHIFT_LOCAL_SR)
 * take forms 0, 1 and 3 (2: BTRT_EINVAL).  Results are bitwise the same in every
 * form and shape, and equal to the members' results stepped alone. */
btrt_status btrt_batch_set_tiles(btrt_batch B, int32_t block_x, int32_t block_y, int32_t rows,
                                 int32_t per_step_launch);

/* Pick the fastest candidate (10 tile shapes x 2 launch forms, x 4 for FP32
 * compute with the two-step and vector forms, x 3 for stochastically rounded
 * members) by timing steps_per_trial steps of each after one warm-up step (its
 * graph captured before the timing).  These are real steps: on a first tuning every
 * member advances by 20 (FP32: 40; stochastically rounded members: 30) x
 * (steps_per_trial + 1) steps.
 * The choice is cached per (members, total nodes, formats) in the process and
 * reused without timing.  Writes the choice (any pointer may be NULL). */
btrt_status btrt_batch_autotune(btrt_batch B, int32_t steps_per_trial, int32_t *block_x, int32_t *block_y,
                                int32_t *rows, int32_t *per_step_launch);

/* Advance every member nsteps steps (asynchronous; one launch or graph per 4096
 * steps).  want_residual != 0: also compute each member's ||phi^n - phi^{n-1}||_2
 * at the last step (fixed order). */
btrt_status btrt_batch_step(btrt_batch B, int64_t nsteps, int32_t want_residual);

/* Capture and instantiate, without running anything, the CUDA graphs that
 * btrt_batch_step(B, nsteps, want_residual) (and btrt_batch_step_tol with nsteps)
 * will replay: lets a caller take the capture's host time while the device is busy
 * elsewhere or outside a timed region.  Uploads the member tables on the batch
 * stream (asynchronous); advances no member.  No-op for a batch that launches
 * directly.  nsteps >= 1 (BTRT_EINVAL otherwise). */
btrt_status btrt_batch_prepare(btrt_batch B, int64_t nsteps, int32_t want_residual);

/* Number of slice graphs the batch holds (each (steps, residual) pair captured
 * once and replayed), or -1 if capture failed and the batch launches directly. */
btrt_status btrt_batch_graphs(btrt_batch B, int32_t *n_graphs);

/* Advance every member nsteps >= 1 steps (as btrt_batch_step with want_residual)
 * and compare, on the device, each member's residual ||phi^n - phi^{n-1}||_2 of
 * the last step with tol (the steady-state test of a serving loop, cf. Eq. 64):
 * done[k] bit 0 = residual < tol, bit 1 = member k produced a non-finite phi,
 * bit 2 = member k was frozen before this call (see btrt_batch_set_freeze; its
 * residual is then NaN and bits 0-1 are clear).  done: n int32 values; resid
 * (may be NULL): the n residuals.  Both in host memory (on_device = 0; pinned
 * memory keeps the copies asynchronous) or device memory (on_device = 1).
 * Nothing synchronises: the results are written in the batch stream's order, so
 * read them after synchronising that stream or an event recorded after this
 * call.  Table uploads use pinned staging, so the call does not wait for work
 * already queued on the stream: a caller may queue the next call before reading
 * this one's results. */
btrt_status btrt_batch_step_tol(btrt_batch B, int64_t nsteps, double tol, int32_t *done, double *resid,
                                int32_t on_device);

/* enable != 0: btrt_batch_step_tol freezes every member it flags (done bit 0 or
 * 1).  The mark lives in the member lattice's device flags, so launches of this
 * and of any later batch leave a frozen member unchanged, while the host's step
 * count of the member still advances with its batch; btrt_settle restores it.
 * Lets a serving loop queue slice k + 1 before it has read slice k's flags and
 * still take each retired member exactly as it was when flagged. */
btrt_status btrt_batch_set_freeze(btrt_batch B, int32_t enable);

/* Read lattice L's freeze mark (synchronises L's stream; call it once the batch
 * launch that flagged L has completed).  If L is frozen: *frozen_step = the step
 * count at which it froze, L's step count and buffer index are set back to that
 * step, and clear != 0 also removes the mark (do that only when no queued batch
 * launch still includes L, which would then step it).  Otherwise *frozen_step = -1. */
btrt_status btrt_settle(btrt_lattice L, int32_t clear, int64_t *frozen_step);

/* Residuals of the last step with want_residual, one per member (host, synchronises). */
btrt_status btrt_batch_residuals(btrt_batch B, double *out_host);

/* flags: bit 0 non-finite phi in some member, bit 1 a barrier wait gave up,
 * bit 3 an index check of a -DBTRT_DEBUG_BOUNDS build failed (BTRT_ECUDA).
 * Returns BTRT_ETIMEOUT or BTRT_EUNSTABLE accordingly.  Synchronises. */
btrt_status btrt_batch_check(btrt_batch B, int32_t *flags);

/* Each member's device flags (bit 0: non-finite phi), in member order, into
 * out_host[n]: lets a caller retire only the members that failed.  Synchronises
 * the batch stream. */
btrt_status btrt_batch_member_flags(btrt_batch B, int32_t *out_host);

/* Bound of every grid-barrier wait, in polls of about 0.1 us (default 2^24).  A
 * wait that reaches it raises flag bit 1 and ends the launch early.
 * never_release != 0 makes every barrier unreachable (for testing the timeout). */
btrt_status btrt_batch_set_wait_limit(btrt_batch B, uint64_t polls, int32_t never_release);

/* Release the batch (synchronises its stream; members stay with the caller). */
btrt_status btrt_batch_destroy(btrt_batch B);

/* FP64 sum of a phi plane that allocates no device memory -- for callers that
 * cannot call cudaMalloc or lend a workspace: a serving process that reserves
 * its whole device-memory budget at start-up and forbids later allocations, or a
 * plug-in inside a host framework that owns the device allocator.  The paper has
 * no counterpart; it runs btrt_mass's own reduction kernels (same fixed order,
 * bitwise the same result for the same values) on any device plane.
 *   phi_dev: device array of dtype BTRT_F64 or BTRT_F32, ny rows of `pitch`
 *   elements, the first nx of each row summed; 1 <= nx, ny <= 65536, pitch >= nx;
 *   larger planes are rejected with BTRT_EINVAL.  out_host: host double.
 * The partial sums live in a fixed 8200-byte array of the library's own device
 * memory (held by every GPU that loads the library until the process exits), not
 * in caller memory; no cudaMalloc/cudaFree or allocating library call is made.
 * The first call on a device looks up that array's device address for the
 * current device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls on a device share the array: calls that overlap on the GPU
 * (different streams, or host threads without ordering) race and may return
 * wrong sums.  Enqueued on cuda_stream (NULL = default stream); synchronises it. */
#define BTRT_PHI_SUM_STATIC_MAX_SIDE 65536
btrt_status btrt_phi_sum_static(const void *phi_dev, int32_t dtype, int32_t nx, int32_t ny,
                                int64_t pitch, void *cuda_stream, double *out_host);

/* Thread-local description of the last error ("" if none). */
const char *btrt_last_error(void);

/* Library build identification (architecture, version). */
const char *btrt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BTRT_H */
