/*
 * mm.h -- C ABI of the GB300 microscale kinetic step of the micro-macro
 * gliding-motility-assay model (Cook & Shinar, arXiv:1908.04279).
 *
 * One handle holds one simulation instance resident on one GPU: the bound-
 * motor density Mb(x, theta, s) (Sec. 2, the high-dimensional density of
 * Eq. 4), the filament density Psi(x, theta) (Eq. 1), the free, coarse and
 * total motor densities (Eq. 5-6), the prescribed in-plane fluid velocity and
 * the substep dt. Every step of the path runs in the library's CUDA kernels;
 * there is no CPU fallback: without a usable CUDA device every call that
 * needs one returns MM_ERR_CUDA.
 *
 * Grid and layouts (all row-major, float64 at this boundary in both
 * precisions):
 *   the unit periodic square with nx * ny cells, dx = 1/nx, dy = 1/ny, cell
 *   centres at ((i + 1/2) dx, (j + 1/2) dy);
 *   orientations theta_k = k * 2 pi / ntheta (Sec. 2: theta and s uniform);
 *   arclength nodes s_j = -L/2 + (j + 1/2) L / ns on the filament.
 *   psi  [ny][nx][ntheta]         mb [ny][nx][ntheta][ns]
 *   u    [2][ny][nx]   (u_x then u_y)
 *   mtot, mf, c [ny][nx]
 *
 * Memory: the caller owns every buffer it passes; the handle owns its device
 * state (allocated in mm_create, released in mm_destroy). A flag on_device
 * says whether a pointer is a device pointer (read or written in stream
 * order on the handle's stream) or a host pointer (the call synchronises the
 * stream before it returns). A handle is not thread-safe; distinct handles
 * may be used from distinct threads.
 *
 * Errors: every call returns an mm_status; no exception crosses the ABI.
 * mm_last_error(h) gives a human-readable message for the last failing call
 * on h (for a NULL handle: the last failure of mm_create or
 * mm_moments_static on this thread).
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_handle mm_handle;

/* Resolution (Sec. 2: x, y on a regular square grid; theta and s uniform).
 * Limits: nx, ny >= 1; 1 <= ntheta <= 1024; L > 0; one s-row is spread over
 * at most one warp, so ns <= 128 (multiple of 4) or <= 32 (otherwise) in
 * MM_FP32_MIXED, and ns <= 64 (even) or <= 32 (odd) in MM_FP64. Other sizes
 * return MM_ERR_UNSUPPORTED. */
typedef struct {
  int nx, ny, ntheta, ns;
  double L;
} mm_grid;

/* Nondimensional parameters.
 *   v_walk  walking speed of bound motor heads (Eq. 4, the d_s term); >= 0
 *   k_on    binding rate (Eq. 4)          k_off  unbinding rate (Eq. 4)
 *   glide, v_sp  gliding speed V = v_sp + glide * n_b of a filament carrying
 *           n_b = sum_j Mb ds bound motors (Eq. 2's -V_sp p term, with the
 *           motor dependence read into it)
 *   force_scale, ell  F and l/L of the motor force, Eq. 10
 *   cfl     Courant number of the adaptive substep */
typedef struct {
  double v_walk, k_on, k_off;
  double glide, v_sp;
  double force_scale, ell;
  double cfl;
} mm_rates;

typedef enum {
  MM_FP64 = 0,       /* every array and every operation in float64 */
  MM_FP32_MIXED = 1  /* Mb, psi, u and the per-cell motor densities stored
                        and stepped in float32 (the paper's mixed precision,
                        Sec. 3.1); the s-reductions feeding the force and
                        force dipole and the moments in compensated
                        float-float (about 48 bits), returned in float64;
                        the global sums of the substep and the mass
                        correction in float64 */
} mm_precision;

typedef enum {
  MM_OK = 0,
  MM_ERR_INVALID = 1,     /* bad argument: NULL, non-positive size, NaN rate */
  MM_ERR_OOM = 2,         /* the device has not enough free memory */
  MM_ERR_CUDA = 3,        /* a CUDA runtime call failed (see mm_last_error) */
  MM_ERR_UNSUPPORTED = 4, /* valid but not supported (v_walk < 0, ns too large) */
  MM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  MM_ERR_NONFINITE = 6,   /* a global sum came out NaN or infinite */
  MM_ERR_STATE = 7        /* call out of order (no state or velocity yet,
                             adjoint without a matching recording) */
} mm_status;

/* Create an instance (Sec. 3.1: all microscale data resident on the GPU).
 * stream: a cudaStream_t (NULL = the legacy default stream) on which every
 * kernel of this handle runs. The state starts as psi = 1/(2 pi), Mb = 0,
 * M = 1 (Mf = 1) with zero velocity and no dt; call mm_set_state and
 * mm_set_velocity before stepping. */
mm_status mm_create(const mm_grid* grid, const mm_rates* rates, mm_precision prec,
                    void* stream, mm_handle** out);
mm_status mm_destroy(mm_handle* h);
mm_status mm_set_stream(mm_handle* h, void* stream);
/* Replace the rates (checked as in mm_create). Synchronises the handle's
 * stream. New rates end an adjoint recording (mm_set_checkpointing): the
 * substeps recorded so far ran with the old rates, so a later mm_adjoint_step
 * returns MM_ERR_STATE until a new recording is made. */
mm_status mm_set_rates(mm_handle* h, const mm_rates* rates);

/* Load a state. psi (required), mb (NULL: all zero), mtot (NULL: all one).
 * Computes n_b and the coarse density C = sum_k psi n_b dtheta (Eq. 5),
 * applies the scale-down of Alg. 2 where C > M, and sets Mf = M - C (Eq. 6). */
mm_status mm_set_state(mm_handle* h, const double* psi, const double* mb, const double* mtot,
                       int on_device);
/* Export the state; any output pointer may be NULL. In MM_FP32_MIXED the
 * pending mass-correction factor is applied to psi on export. */
mm_status mm_get_state(mm_handle* h, double* psi, double* mb, double* mf, double* c,
                       int on_device);

/* Bitwise checkpoint and restart (checkpoint/resume of a long run). A
 * snapshot holds the state exactly as the substep kernels left it, in the
 * state precision (psi, n_b, Mb, Mf, C, M), the device scalars the next
 * substep reads (dt, the float32 form's pending mass-correction factor and
 * its reference filament number) and the velocity in effect, so that a handle
 * of the same grid and precision loaded from it continues the uninterrupted
 * run bit for bit (mm_get_state / mm_set_state re-derive n_b, C, Mf and the
 * reference filament number, which continues the same physics but not the
 * same bits). The buffer is caller-owned, host (on_device = 0) or device
 * memory of at least mm_snapshot_bytes; its format is private to this
 * library version. mm_save_snapshot and mm_load_snapshot synchronise the
 * handle's stream. Loading ends an adjoint recording, as mm_set_state does.
 * MM_ERR_INVALID for a buffer that is too small, not a snapshot, or of another
 * grid or precision; MM_ERR_STATE when saving a handle without a state;
 * MM_ERR_UNSUPPORTED with non-local anchors on. */
mm_status mm_snapshot_bytes(mm_handle* h, size_t* bytes);
mm_status mm_save_snapshot(mm_handle* h, void* buf, size_t bytes, int on_device);
mm_status mm_load_snapshot(mm_handle* h, const void* buf, size_t bytes, int on_device);

/* Prescribe the in-plane velocity u (held fixed over the following substeps)
 * and recompute the adaptive substep from the current state (Sec. 2: the
 * outer step is limited by the advective fluxes of Eq. 1, the inner one by the
 * motor speed and the binding and unbinding rates of Eq. 4):
 *   dt = cfl / max(v_walk/ds, max(|ax|/dx + |ay|/dy), max|omega|/dtheta,
 *                  k_off + k_on L max_cell sum_k psi dtheta),
 * with a = u - V p and omega the Jeffery rotation rate at theta faces. */
mm_status mm_set_velocity(mm_handle* h, const double* u, int on_device);
mm_status mm_get_dt(mm_handle* h, double* dt);
/* Override the substep (e.g. to compare runs at the same dt). dt > 0. */
mm_status mm_set_dt(mm_handle* h, double dt);

/* Advance n_substeps substeps (Alg. 1 inner loop, with psi advanced inside
 * each substep). Each substep:
 *   1. psi by Eq. 1 in donor-cell flux form in x, y and theta;
 *   2. every s-row of Mb by Eq. 4, Superbee-limited walking flux plus binding
 *      and unbinding, midpoint RK2 with Mf frozen (Alg. 2 half and full
 *      stage);
 *   3. n_b, the coarse density (Eq. 5) with psi at the new time, the
 *      scale-down of Alg. 2, and Mf = M - C (Eq. 6).
 * Asynchronous on the handle's stream; launched as a captured CUDA graph. */
mm_status mm_micro_step(mm_handle* h, int n_substeps);

/* Macroscale moments (Alg. 1 after the inner loop), all float64.
 * fields (may be NULL) receives [12][ny][nx]:
 *   0 rho = sum psi dtheta    1,2 P = sum psi p dtheta
 *   3,4 Q = sum psi (p p - I/2) dtheta (xx, xy)    5 C (Eq. 5)   6 Mf (Eq. 6)
 *   7,8 F = F sum_k p psi n_b dtheta (Eq. 10 with anchors in the cell)
 *   9,10,11 sigma_a = F ell sum_k p p psi m1 dtheta (xx, xy, yy),
 *           m1 = sum_j s_j Mb ds (force dipole of an s-row)
 * scalars (always written, host memory):
 *   0 total filament number sum psi dx dy dtheta   1 bound sum C dx dy
 *   2 free sum Mf dx dy   3 bound + free   4 polar order |sum psi e^{i theta}|
 *   / sum psi   5 mean over cells of tr sigma_a   6 sum psi cos  7 sum psi sin.
 * Returns MM_ERR_NONFINITE if a global sum is not finite. */
typedef struct {
  double* fields;
  int fields_on_device;
  double scalars[8];
} mm_moments_out;
mm_status mm_moments(mm_handle* h, mm_moments_out* out);

/* ---- Adjoint (reverse mode) of the substeps, with checkpointing ----------
 *
 * mm_set_checkpointing(h, K, max_substeps) starts a recording at the current
 * state: the following mm_micro_step calls (up to max_substeps substeps in
 * total, with any number of mm_set_velocity calls in between) save the state
 * every K substeps; the memory for ceil(max_substeps / K) + 1 checkpoints and
 * for the K + 1 states of one recomputed segment is reserved here
 * (MM_ERR_OOM if it does not fit), in one device allocation that a later
 * recording with the same K and max_substeps reuses. mm_set_state ends a
 * recording and keeps that memory; K = 0 ends it and frees the memory
 * (mm_destroy frees it too). While recording, substeps run as individual
 * launches (no graph) so that checkpoints can be taken between them.
 *
 * mm_adjoint_step(h, n, seed, out) runs the reverse sweep over the n substeps
 * recorded since mm_set_checkpointing (n must equal that count): for each
 * segment, last first, it restores the checkpoint, recomputes the segment's
 * states, and applies the transposed substep (discrete adjoint of Eq. 1, of
 * the midpoint RK2 of Eq. 4 with the Superbee branch the forward took, of
 * Eq. 5, the Alg. 2 scale-down and Eq. 6) from the last substep to the first.
 * dt and the velocities are held fixed (not differentiated). The seed is the
 * gradient of a loss L with respect to the final state, given either as
 * arrays in moment form or as one of the built-in observables. The live state
 * of the handle is left as it was. */
typedef enum {
  MM_OBS_NONE = 0,         /* seed given by the arrays below */
  MM_OBS_POLAR_ORDER = 1,  /* L = |sum psi e^{i theta}| / sum psi */
  MM_OBS_MEAN_STRESS = 2   /* L = mean over cells of tr sigma_a */
} mm_observable;
typedef struct {
  int observable;
  const double* dL_dpsi; /* [ny][nx][ntheta] or NULL */
  const double* dL_dnb;  /* [ny][nx][ntheta] or NULL: through n_b = sum_j Mb ds */
  const double* dL_dm1;  /* [ny][nx][ntheta] or NULL: through m1 = sum_j s_j Mb ds */
  const double* dL_dmf;  /* [ny][nx] or NULL: through the free motors Mf */
  int on_device;         /* all seed arrays are device (1) or host (0) pointers */
  const double* dL_dmb;  /* [ny][nx][ntheta][ns] or NULL: the bound-motor density itself,
                            added to the rows' seed from dL_dnb and dL_dm1 (for a loss on
                            the motor field that its first two s-moments do not carry) */
} mm_adjoint_seed;
typedef struct {
  double* dL_du;         /* [du_capacity][2][ny][nx] or NULL, in prescription order */
  int du_capacity;       /* velocity blocks dL_du holds; MM_ERR_INVALID if fewer than
                            the recording's velocity fields */
  double* dL_dpsi0;      /* [ny][nx][ntheta] or NULL: w.r.t. psi at the recording start */
  int on_device;
  double dL_drates[3];   /* written: dL/dk_off, dL/dv_walk, dL/dk_on */
  double value;          /* written for a built-in observable: L at the final state */
  int n_velocities;      /* written: velocity fields in effect during the recording */
} mm_adjoint_out;
mm_status mm_set_checkpointing(mm_handle* h, int K, int max_substeps);
/* Two-level form (for runs whose single-level memory would not fit): outer
 * checkpoints every K substeps during the recording, and, in the reverse
 * sweep, each outer segment is first recomputed once to store inner
 * checkpoints every K_inner substeps, then its inner segments are recomputed
 * into K_inner slots and reversed. Device memory: ceil(max_substeps / K) + 1
 * outer checkpoints + ceil(K / K_inner) - 1 inner checkpoints + max(K_inner, 2)
 * slots (one state each), against K + ceil(max_substeps / K) + 1 for one level;
 * one extra recomputation of the run. mm_set_checkpointing(h, K, n) is
 * mm_set_checkpointing_levels(h, K, K, n). MM_ERR_INVALID unless
 * 1 <= K_inner <= K. */
mm_status mm_set_checkpointing_levels(mm_handle* h, int K, int K_inner, int max_substeps);
mm_status mm_adjoint_step(mm_handle* h, int n_substeps, const mm_adjoint_seed* seed,
                          mm_adjoint_out* out);

/* ---- Tangent-linear mode (forward-mode derivative along a direction of the rates)
 *
 * mm_set_tangent(h, dparams): dparams = {d k_off, d v_walk, d k_on} (finite)
 * switches the tangent mode on: from then on every substep (mm_micro_step)
 * advances, in one launch, the state and its tangent -- the derivative of
 * the state along that direction of the rates, starting from zero at the
 * current state and again at every mm_set_state. The map differentiated is
 * the substep as the forward computes it at a fixed dt (dt and the velocities
 * are held fixed, as in the reverse sweep), on the branches the forward takes,
 * the float32 form's mass-correction factor a constant of the map. Costs one
 * pass of about twice the forward's memory traffic per substep and needs no
 * checkpoints: the tool for the derivative with respect to one scalar
 * parameter (mm_adjoint_step gives many at once). NULL switches it off and
 * frees its memory (one more state of Mb, psi and n_b). While it is on,
 * mm_set_checkpointing, mm_diffuse, mm_motor_local and mm_fluid_solve return
 * MM_ERR_STATE (their effect on the tangent is not followed). MM_ERR_UNSUPPORTED:
 * a batch or member, non-local anchors or a capture radius; MM_ERR_OOM.
 *
 * mm_get_tangent(h, dpsi, dmb, dmf, on_device): the tangent of psi (with the
 * pending float32 correction factor, as mm_get_state), Mb and Mf; any output
 * may be NULL. mm_tangent_observable(h, observable, &value, &dvalue): a
 * built-in observable (MM_OBS_POLAR_ORDER or MM_OBS_MEAN_STRESS) of the current
 * state and its derivative along the direction; synchronises the stream.
 * MM_ERR_STATE when the tangent mode is off. */
mm_status mm_set_tangent(mm_handle* h, const double* dparams);
mm_status mm_get_tangent(mm_handle* h, double* dpsi, double* dmb, double* dmf, int on_device);
mm_status mm_tangent_observable(mm_handle* h, int observable, double* value, double* dvalue);

/* ---- Filament diffusion --------------------------------------------------------
 *
 * mm_diffuse(h, D_t, D_r, dt): one step of the diffusive fluxes of Eq. 2-3,
 * -D_t grad ln psi and -D_r d_theta ln psi, i.e. d_t psi = D_t (d_xx + d_yy) psi
 * + D_r d_theta^2 psi on the periodic grid (dx = 1/nx, dy = 1/ny,
 * dtheta = 2 pi / ntheta), by Crank-Nicolson (the scheme Sec. 2 and Alg. 1
 * give the diffusive terms of the psi update) applied one direction at a time:
 * theta, then x, then y, each (I - a/2 L) psi' = (I + a/2 L) psi with L the
 * periodic second difference and a = D dt / h^2 (unconditionally stable,
 * second order; the one-dimensional operators commute). Meant once per macro
 * step with the macro step's dt, before its substeps (Alg. 1 updates psi before
 * the motor loop). Then recomputes the coarse density C = sum psi n_b dtheta,
 * the Alg. 2 scale-down and Mf = M - C for the new psi. Not differentiated:
 * MM_ERR_STATE while an adjoint recording is active. MM_ERR_INVALID for a
 * negative or non-finite diffusivity or a non-positive dt. No counterpart in
 * the microscale step of the paper's GPU code (the paper solves this on the
 * CPU). */
mm_status mm_diffuse(mm_handle* h, double D_t, double D_r, double dt);

/* ---- Local substeps with psi frozen -------------------------------------------
 *
 * mm_motor_local(h, T, nsteps_in, nsteps_out, on_device): advance the motor
 * densities over a macro interval T with psi held fixed and a substep of its
 * own in every cell -- the independent time steps of Sec. 3.1, Alg. 2's
 * "while t* < t*_end" loop run per anchor (anchors in the filament's own
 * cell). Per cell i:
 *   rho_i = sum_k psi dtheta, rate_i = max(v_walk/ds, k_off + k_on L rho_i),
 *   n_i = max(1, ceil(T rate_i / cfl)) (evaluated in float64, left to right,
 *   with no fused operations), dt_i = T / n_i;
 * then n_i times: every s-row by the midpoint RK2 of Eq. 4 (Mf frozen over the
 * two stages), C = sum_k psi n_b dtheta (Eq. 5, psi frozen), the Alg. 2
 * scale-down where C > M, Mf = M - C (Eq. 6). psi and the substep dt of
 * mm_micro_step are not touched; n_b, C and Mf are left consistent with the new
 * Mb. nsteps_in (NULL: the rule above) imposes n_i per cell ([ny][nx] ints,
 * each in 1..2^20); nsteps_out (may be NULL) receives the n_i used. on_device
 * says whether these two are device pointers (stream order) or host pointers
 * (then the call synchronises). A computed count above 2^20 (T far beyond the
 * cell's stable step) leaves the whole motor state unchanged and is reported as
 * MM_ERR_INVALID by this call (host nsteps_out) or by the next synchronising
 * call. MM_ERR_INVALID for T <= 0 or not finite or a host count out of range;
 * MM_ERR_STATE without a state or while an adjoint recording is active (not
 * differentiated); MM_ERR_UNSUPPORTED when one cell's ntheta * ns values do not
 * fit in shared memory (about 200 KB); MM_ERR_TIMEOUT (at the next synchronising
 * call) if a bounded device wait gave up. */
mm_status mm_motor_local(mm_handle* h, double T, const int* nsteps_in, int* nsteps_out,
                         int on_device);

/* ---- Non-local motor anchors ----------------------------------------------------
 *
 * mm_set_anchors(h, enable): with enable = 1 every bound-motor configuration
 * (cell i, theta_k, s_j) is anchored in the cell under its motor head,
 * x_i + (l/L) s_j p_k with l/L = rates.ell (the delta of Eq. 10), instead of
 * in the filament's own cell -- Eq. 4-6 and Eq. 10 with the anchor r0 kept and
 * the capture radius of Eq. 4 taken to zero. The anchor of (i, k, j) is cell
 * (ix + ox, iy + oy) (periodic) with
 *   ox = floor(((l/L) L (2j + 1 - ns) / (2 ns)) cos(theta_k) nx + 1/2),
 *   oy = floor(((l/L) L (2j + 1 - ns) / (2 ns)) sin(theta_k) ny + 1/2),
 * evaluated in float64 (products and quotients, then one add). Then in every
 * substep the binding term of node j takes the free motors of its anchor,
 * k_on Mf(r0) (Mf frozen over both RK2 stages); the coarse density of Eq. 5,
 * the Alg. 2 scale-down and Eq. 6 are formed per anchor cell, C(r0) = sum of
 * psi Mb ds dtheta over the configurations anchored at r0 (psi at the new
 * time); mm_moments' force fields Fx, Fy become the force of Eq. 10 acting in
 * the anchor cells, F(r0) = F sum p psi Mb ds dtheta. psi transport, n_b and
 * the substep rule are unchanged. enable = 0 returns to anchors in the
 * filament's own cell. Either way the call re-derives C, the scale-down and Mf
 * of the current state under the chosen rule; mm_set_rates re-derives them when
 * l/L changes. The coarse density is accumulated with float64 atomics: its last
 * bits depend on the schedule. MM_ERR_UNSUPPORTED on a batch or a batch
 * member; with anchors on, mm_set_checkpointing and mm_motor_local return
 * MM_ERR_UNSUPPORTED (the adjoint and the independent-cell local step are not
 * available) and mm_set_anchors returns MM_ERR_STATE during a recording. */
mm_status mm_set_anchors(mm_handle* h, int enable);

/* ---- Finite capture radius (Sec. 2's B_rc(r0), Eq. 4's indicator, Alg. 2 per r0)
 *
 * mm_set_capture(h, r_c): r_c >= 0 keeps the anchor r0 of a bound motor as an
 * axis of the motor density: Mb(r0, x, theta, s) is tracked where the motor
 * head x + (l/L) s p (l/L = rates.ell) is within reach of r0, a cell being in
 * reach when the distance from the head to the cell's square is at most r_c
 * (physical units of the unit square); at r_c = 0 the reach is the cell under
 * the head. Each substep runs Alg. 2 per anchor: every configuration by the
 * RK2 of Eq. 4 with Mf(r0) frozen, a motor keeping its anchor while it walks
 * (so the nodes in reach of one anchor form walking lines: no inflow at a
 * line's first node, donor-cell outflow at its last, the motor rejoining the
 * free pool through Eq. 6), binding k_on Mf(r0) / n_a shared among the n_a
 * anchors in reach of the node; then Eq. 5 at r0 with psi at the new time,
 * the scale-down at r0 and Eq. 6 at r0. n_b sums over anchors and nodes; the
 * force of Eq. 10 (mm_moments fields 7, 8) acts in the cell under each head.
 * r_c < 0 switches back to the models above. Either switch discards the
 * motors (Mb = 0, Mf = M; psi is kept).
 *
 * With a capture radius, the mb arrays of mm_set_state / mm_get_state are
 * [ny][nx][nconf] (float64 at this boundary): for each anchor cell, its
 * configurations in template order. mm_capture_template returns the template,
 * the same for every anchor: nlines lines of 6 ints (k, dx, dy, j0, len, off)
 * -- the motors of anchor r0 bound to a filament of orientation k centred at
 * r0 - (dx, dy) cells, at nodes j0 .. j0 + len - 1, stored from entry off --
 * when max_lines >= nlines (lines may be NULL), nconf, and w [ntheta][ns] =
 * 1 / n_a (may be NULL). Lines are sorted by k, then j0, dy, dx.
 *
 * MM_ERR_UNSUPPORTED: a batch or batch member; ns > 256; a reach wider than the
 * periodic grid (two offsets would name one cell). MM_ERR_STATE: during an
 * adjoint recording, or with mm_set_anchors on. MM_ERR_OOM: the state (cells x
 * nconf values) does not fit. With a capture radius set, mm_set_checkpointing,
 * mm_motor_local and mm_save_snapshot return MM_ERR_UNSUPPORTED, the fluid
 * solve refuses the dipole term, and mm_set_rates refuses a new l/L. */
mm_status mm_set_capture(mm_handle* h, double r_c);
mm_status mm_capture_template(mm_handle* h, int* lines, int max_lines, int* nlines, int* nconf,
                              double* w);

/* ---- Thin-gap fluid solve (Eq. 7-9, Alg. 1 after the inner loop) --------------
 *
 * The fluid fills the gap 0 <= z <= 1 between two no-slip plates and is
 * periodic in x and y over the unit square (Sec. 2); the filaments lie on the
 * plane z = z0 (Sec. 2: a Dirac delta in z about that plane), so the right side
 * of Eq. 7 is (F_2 + div_2 Sigma) delta(z - z0). The solve returns u_2 on that
 * plane, the velocity that advects the filaments (Eq. 2-3).
 *
 * mm_fluid_setup(h, eps, z0): eps of Eq. 7-8 (> 0, finite), the plane's height
 * z0 (0 < z0 < 1). Builds, on the device, the in-plane response per Fourier
 * mode of the half spectrum, (g_T, g_L) at |k| = 2 pi sqrt(jx^2 + my^2), the
 * velocity at z0 per unit force on the plane across and along k, each the exact
 * solution in z of the transformed Eq. 7-9 (the limit of the paper's z-grid).
 * P0 scales the pressure only and does not enter. Needs nx, ny >= 2
 * (MM_ERR_UNSUPPORTED otherwise, and on a batch member); plans three batched
 * float64 cuFFT transforms and allocates about 176 bytes per mode of the half
 * spectrum plus 80 bytes per cell, all or nothing (MM_ERR_OOM if they do not
 * fit). May be called again with new eps, z0 (the buffers are kept).
 *
 * mm_fluid_solve(h, sigma, sigma_on_device, dipole, u_out, u_out_on_device):
 *   1. the moments of the current state (as mm_moments; F = fields 7, 8);
 *   2. per mode of the 2D DFT of the cell values, f = F^ + i k . S^ with
 *      S = Sigma - dipole sigma_a: sigma (float64 [3][ny][nx], xx, xy, yy, host
 *      or device, may be NULL) is the extra stress sigma_f S_f - sigma_t S_t of
 *      Eq. 7 (its constitutive law is the caller's); dipole = 1 adds the
 *      first-order term of Eq. 10's spreading in s, F_2 ~ F - div sigma_a
 *      (moment fields 9-11; not with anchors, whose force already acts in the
 *      anchor cells: MM_ERR_UNSUPPORTED);
 *   3. u^ = g_T f + (g_L - g_T) k (k . f) / |k|^2 (g_T = g_L at k = 0, the mean
 *      flow); at a Nyquist index of an even nx or ny the map is the mean of its
 *      values for +k and -k of that component (the output stays real);
 *   4. the inverse DFT; u_2 [2][ny][nx] becomes the velocity in effect, as
 *      mm_set_velocity (the adaptive substep is recomputed), and is copied to
 *      u_out (float64 [2][ny][nx], host or device) if u_out is not NULL.
 * All in float64 in either precision. MM_ERR_STATE without mm_fluid_setup or a
 * state, or during an adjoint recording (not differentiated). Asynchronous on
 * the handle's stream unless u_out is a host pointer.
 *
 * mm_fluid_response(h, out, on_device): copies the response table, float64
 * [ny][nx/2 + 1][2] (g_T, g_L), index (jy, jx) at wavenumber (jx, my) with
 * my = jy for jy <= ny/2 and jy - ny above. */
mm_status mm_fluid_setup(mm_handle* h, double eps, double z0);
mm_status mm_fluid_solve(mm_handle* h, const double* sigma, int sigma_on_device, int dipole,
                         double* u_out, int u_out_on_device);
mm_status mm_fluid_response(mm_handle* h, double* out, int on_device);

/* ---- Batched ensemble --------------------------------------------------------
 *
 * An ensemble of n independent instances (an instance as above: its own grid,
 * rates, state, velocity and dt; e.g. a sweep of k_off or v_walk) advanced
 * together: mm_micro_step on the batch handle runs each substep as ONE launch
 * over all instances (a table of tiles, each a run of cells of one instance
 * holding about the same number of motor values), and the n_substeps of one
 * call as one captured CUDA graph. No counterpart in the paper, which runs one
 * instance at a time.
 *
 * mm_create_batch(n, grids, rates, prec, stream, &batch): grids[i], rates[i]
 * for instance i; every instance needs ns divisible by 4 (MM_FP32_MIXED) or 2
 * (MM_FP64) (MM_ERR_UNSUPPORTED otherwise). mm_batch_member(batch, i, &m)
 * returns instance i's handle, owned by the batch (mm_destroy on it fails;
 * mm_destroy on the batch frees all): mm_set_state, mm_set_velocity,
 * mm_set_dt, mm_get_state, mm_moments, mm_set_checkpointing and
 * mm_adjoint_step go to the members (on the batch, they fail with
 * MM_ERR_INVALID). A member recording an adjoint takes its checkpoints during
 * the batched substeps; its reverse sweep (mm_adjoint_step on the member)
 * replays with the single-instance kernel. mm_micro_step on a member advances
 * that member alone. mm_set_stream and mm_debug_set on the batch apply to
 * every member; mm_sync on the batch checks every member.
 *
 * mm_batch_autotune(batch, substeps, results, max_results, &n_results): times
 * `substeps` batched substeps for each (tile_work, chunk_bytes) in
 * {1024 .. 32768} x {2048, 4096, 8192} (motor values per tile, bytes per
 * s-row chunk) from the current state, restores the state, and keeps the
 * fastest; results (may be NULL) receives up to max_results timings. The
 * choice is cached for the process: a later batch with the same member grids
 * and precision starts with it.
 *
 * The candidates also try members with at most 16 orientations (and an even
 * row length) two cells to a warp (cells_per_warp 2: one chunk holds both
 * cells' rows, half-warps take psi and the close) and one cell to a warp (1).
 *
 * mm_get_launch_info on a batch: grid, block, shared memory, 1, ring stages,
 * largest chunk (values), tiles, values per lane, tile_work, chunk_bytes,
 * tuned (0/1), two cells per warp where possible (0/1). */
typedef struct {
  int tile_work;
  int chunk_bytes;
  double ms_per_substep;
  int cells_per_warp;
} mm_batch_tune;
mm_status mm_create_batch(int n, const mm_grid* grids, const mm_rates* rates, mm_precision prec,
                          void* stream, mm_handle** out);
mm_status mm_batch_member(mm_handle* batch, int i, mm_handle** member);
mm_status mm_batch_autotune(mm_handle* batch, int substeps, mm_batch_tune* results,
                            int max_results, int* n_results);

/* Wait for the handle's stream and report a failure recorded by a kernel
 * since the last check (MM_ERR_TIMEOUT: a bounded device-side wait gave up and
 * the state is no longer valid). mm_get_state and mm_moments check too. */
mm_status mm_sync(mm_handle* h);

/* Test and tuning knobs of the substep kernel (no counterpart in the paper).
 * wait_limit: polls of an mbarrier before a device wait gives up (default
 * 4194304); flags bit 0: wait on a barrier nothing completes, so that
 * every wait runs out -- used by tests of the timeout path, never in production. */
mm_status mm_debug_set(mm_handle* h, unsigned int wait_limit, unsigned int flags);

/* Launch plan of the substep kernel, for tests and profiling: info[0..9] =
 * grid, block, dynamic shared bytes, uses bulk copies (0/1), ring stages,
 * s-rows per stage, stages per cell, values per lane, lanes per s-row, SMs. */
mm_status mm_get_launch_info(mm_handle* h, int* info, int n);

const char* mm_last_error(const mm_handle* h);

/* Moments of a state held by the caller, with no device allocation (this
 * entry point has no counterpart in the paper). For callers that cannot call
 * cudaMalloc -- an application that reserved the GPU's memory for its own
 * pool and forbids allocations it does not manage, or a time-critical loop
 * that must not pay the synchronisation an allocation may imply.
 *   psi, mb, mf, c: float64 device arrays in the layouts above (inputs);
 *   fields: float64 device array [12][ny][nx] as in mm_moments, or NULL;
 *   scalars: float64 device array [8] as in mm_moments (output);
 *   stream: cudaStream_t for the two kernels (asynchronous; the caller
 *   synchronises before reading the outputs).
 * Scratch is one file-scope device array of 65536 cell records (4 MiB) that
 * every GPU loading the library holds until exit: grids above 65536 cells are
 * rejected with MM_ERR_UNSUPPORTED. The array is placed on a device when the
 * library's device code is loaded there: with CUDA's default lazy module
 * loading that is the first call on that device (with
 * CUDA_MODULE_LOADING=EAGER, when the process first uses the device), and
 * that first placement does take 4 MiB of device memory. A caller that
 * reserves the GPU's memory for its own pool should therefore make one call
 * before reserving it; later calls allocate nothing. The first call on a
 * device also looks up the array's device address (once per device, with that
 * device current), so it should come before any stream capture. All calls
 * share the array: calls that overlap on the GPU race. Errors:
 * mm_last_error(NULL). */
mm_status mm_moments_static(const mm_grid* grid, const mm_rates* rates, const double* psi,
                            const double* mb, const double* mf, const double* c, double* fields,
                            double* scalars, void* stream);

/* Measured arithmetic roof of the current device (a measurement aid with no
 * counterpart in the paper; the rooflines of the kernels bound by arithmetic
 * issue rather than memory are stated against it). kind 0: float64 fused
 * multiply-adds; 1: scalar float32; 2: packed two-value float32 (each packed
 * instruction counts as two). A grid of full blocks on every SM runs
 * independent chains of fused multiply-adds; the call times five launches
 * with CUDA events on `stream` after one warm-up launch and synchronises.
 * *fma_per_s: fused multiply-adds per second (flops = 2x); *ms_per_launch
 * (may be NULL): the average launch time. Allocates nothing beyond two CUDA
 * events. Errors: MM_ERR_INVALID (bad kind or NULL output), MM_ERR_CUDA;
 * mm_last_error(NULL). */
mm_status mm_alu_peak(int kind, double* fma_per_s, double* ms_per_launch, void* stream);

/* A short description of the build (library name and target architecture). */
const char* mm_build_info(void);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
