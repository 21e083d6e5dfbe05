/*
 * mm_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the
 * microscale kinetic step of the micro-macro gliding-assay model
 * (Cook & Shinar, arXiv:1908.04279).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library. It shares no
 * code, header, table or constant with the CUDA path: every trigonometric
 * table and every formula is computed here from its definition.
 *
 * What one substep computes (Alg. 1 inner loop with Alg. 2 inside it):
 *   1. filament transport, Eq. 1 (with Eq. 2-3 for the velocities), donor-cell
 *      flux form in x, y and theta, forward Euler over one substep;
 *   2. bound-motor kinetics, Eq. 4: walking advection in s with a Superbee
 *      limited flux (Sec. 2) and binding/unbinding, midpoint RK2 (Sec. 3.1
 *      "Numerical Integration Scheme"; Alg. 2 half and full stage);
 *   3. coarsened bound motors, Eq. 5, and the scale-down clip of Alg. 2;
 *   4. free motors, Eq. 6.
 * It also computes the adaptive substep (Sec. 2), the macroscale moments that
 * the motor force of Eq. 10 reduces to when motor anchors sit in the
 * filament's own cell, and the tangent-linear and adjoint maps of one substep.
 *
 * Layouts (row-major):
 *   psi  [ny][nx][nth]        mb [ny][nx][nth][ns]     u [2][ny][nx]
 *   mf, c, mtot [ny][nx]
 * theta_k = k dth (dth = 2 pi / nth); s_j = -L/2 + (j + 1/2) ds (ds = L/ns);
 * the domain is the periodic square of sides lx, ly (the unit square unless a
 * patch is being evaluated), dx = lx/nx, dy = ly/ny.
 *
 * Readings of the paper taken where it is silent (each is listed in the
 * design notes): motor anchors collapse to the filament-centre cell and the
 * capture indicator of Eq. 4 is 1 (the *_anchor functions keep the anchors
 * instead: each configuration is anchored in the cell under its motor head); the gliding speed is v_sp + glide * n_b;
 * the rotation rate of Eq. 3 is Jeffery's rod rotation p_perp . grad(u) . p;
 * the substep is global per instance; psi is advanced first in each substep.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* lx, ly: side lengths of the periodic domain (1 for the unit square). A
 * 3x3 periodic patch with lx = 3/N reproduces exactly the substep of its
 * centre cell on an N-cell grid, since one substep reads only the 4
 * neighbour cells. */
typedef struct {
  int nx, ny, nth, ns;
  double L, lx, ly;
} or_grid;

typedef struct {
  double v_walk, k_on, k_off;
  double glide, v_sp;
  double force_scale, ell;
  double cfl;
} or_rates;

enum { OR_OK = 0, OR_ERR_INVALID = 1, OR_ERR_NOMEM = 2 };

/* ------------------------------------------------------------------ helpers */

static const double OR_PI = 3.14159265358979323846264338327950288;

static int grid_ok(const or_grid* g) {
  return g && g->nx > 0 && g->ny > 0 && g->nth > 0 && g->ns > 0 && g->L > 0.0 && g->lx > 0.0 &&
         g->ly > 0.0;
}
static double dx_of(const or_grid* g) { return g->lx / g->nx; }
static double dy_of(const or_grid* g) { return g->ly / g->ny; }

static size_t ncell(const or_grid* g) { return (size_t)g->nx * (size_t)g->ny; }
static size_t cidx(const or_grid* g, int ix, int iy) { return (size_t)iy * g->nx + ix; }
static size_t pidx(const or_grid* g, int ix, int iy, int k) {
  return cidx(g, ix, iy) * g->nth + k;
}
static int wrap(int i, int n) { return ((i % n) + n) % n; }

static double dth_of(const or_grid* g) { return 2.0 * OR_PI / g->nth; }
static double ds_of(const or_grid* g) { return g->L / g->ns; }
static double s_node(const or_grid* g, int j) { return -0.5 * g->L + (j + 0.5) * ds_of(g); }

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

/* minmod and maxmod of two slopes: zero unless both have the same sign. */
static double minmod(double x, double y) {
  if (x * y <= 0.0) return 0.0;
  return fabs(x) < fabs(y) ? x : y;
}
static double maxmod(double x, double y) {
  if (x * y <= 0.0) return 0.0;
  return fabs(x) > fabs(y) ? x : y;
}

/* Superbee limited slope (Roe's limiter, the flux limiter named in Sec. 2):
 * sigma = maxmod(minmod(2a, b), minmod(a, 2b)), with a the backward and b the
 * forward difference. The value is always ca*a + cb*b for the returned
 * coefficients, which are also the derivative of the branch taken. */
static double superbee(double a, double b, double* ca, double* cb) {
  double x1 = minmod(2.0 * a, b), x2 = minmod(a, 2.0 * b);
  double x1a, x1b, x2a, x2b;
  if (x1 == 0.0) { x1a = 0.0; x1b = 0.0; }
  else if (x1 == 2.0 * a && fabs(2.0 * a) < fabs(b)) { x1a = 2.0; x1b = 0.0; }
  else { x1a = 0.0; x1b = 1.0; }
  if (x2 == 0.0) { x2a = 0.0; x2b = 0.0; }
  else if (fabs(a) < fabs(2.0 * b)) { x2a = 1.0; x2b = 0.0; }
  else { x2a = 0.0; x2b = 2.0; }
  double s = maxmod(x1, x2);
  if (s == 0.0) { *ca = 0.0; *cb = 0.0; }
  else if (x1 * x2 > 0.0 && fabs(x1) > fabs(x2)) { *ca = x1a; *cb = x1b; }
  else { *ca = x2a; *cb = x2b; }
  return s;
}

/* ----------------------------------------------------- filament kinematics */

/* Velocity gradient G_ab = d u_a / d x_b at cell (ix,iy) by periodic central
 * differences: G[0]=Gxx, G[1]=Gxy, G[2]=Gyx, G[3]=Gyy. */
static void vel_grad(const or_grid* g, const double* u, int ix, int iy, double G[4]) {
  const double* ux = u;
  const double* uy = u + ncell(g);
  double dx = dx_of(g), dy = dy_of(g);
  int xp = wrap(ix + 1, g->nx), xm = wrap(ix - 1, g->nx);
  int yp = wrap(iy + 1, g->ny), ym = wrap(iy - 1, g->ny);
  G[0] = (ux[cidx(g, xp, iy)] - ux[cidx(g, xm, iy)]) / (2.0 * dx);
  G[1] = (ux[cidx(g, ix, yp)] - ux[cidx(g, ix, ym)]) / (2.0 * dy);
  G[2] = (uy[cidx(g, xp, iy)] - uy[cidx(g, xm, iy)]) / (2.0 * dx);
  G[3] = (uy[cidx(g, ix, yp)] - uy[cidx(g, ix, ym)]) / (2.0 * dy);
}

/* Rotation rate of Eq. 3, read as Jeffery's rod rotation p_perp . G . p with
 * p = (cos phi, sin phi), p_perp = (-sin phi, cos phi). */
static double omega_at(const double G[4], double phi) {
  double c = cos(phi), s = sin(phi);
  return -s * (G[0] * c + G[1] * s) + c * (G[2] * c + G[3] * s);
}
/* d omega / d G at angle phi, same component order as G. */
static void omega_dG(double phi, double d[4]) {
  double c = cos(phi), s = sin(phi);
  d[0] = -s * c; d[1] = -s * s; d[2] = c * c; d[3] = c * s;
}

/* Translational velocity of Eq. 2 kept on the hot path: u - V p with gliding
 * speed V = v_sp + glide * n_b (motor-driven gliding). comp 0 = x, 1 = y. */
static double glide_vel(const or_grid* g, const or_rates* r, const double* u,
                        const double* nb, int ix, int iy, int k, int comp) {
  double th = k * dth_of(g);
  double p = comp == 0 ? cos(th) : sin(th);
  double V = r->v_sp + r->glide * nb[pidx(g, ix, iy, k)];
  return u[(size_t)comp * ncell(g) + cidx(g, ix, iy)] - V * p;
}

/* Bound motors per filament row: n_b = sum_j Mb_j ds (the s-integral of Eq. 5). */
static void rows_nb(const or_grid* g, const double* mb, double* nb) {
  double ds = ds_of(g);
  size_t rows = ncell(g) * g->nth;
  for (size_t r = 0; r < rows; ++r) {
    double acc = 0.0;
    for (int j = 0; j < g->ns; ++j) acc += mb[r * g->ns + j] * ds;
    nb[r] = acc;
  }
}

/* Donor-cell flux through a face with face velocity A between a left state
 * pl and a right state pr. */
static double donor(double A, double pl, double pr) { return dmax(A, 0.0) * pl + dmin(A, 0.0) * pr; }

/* Eq. 1 in flux form, one forward-Euler substep:
 * psi' = psi - dt [dFx/dx + dFy/dy + dFth/dth]. */
static void psi_transport(const or_grid* g, const or_rates* r, double dt, const double* u,
                          const double* psi, const double* nb, double* out) {
  double dx = dx_of(g), dy = dy_of(g), dth = dth_of(g);
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix) {
      double G[4];
      vel_grad(g, u, ix, iy, G);
      int xp = wrap(ix + 1, g->nx), xm = wrap(ix - 1, g->nx);
      int yp = wrap(iy + 1, g->ny), ym = wrap(iy - 1, g->ny);
      for (int k = 0; k < g->nth; ++k) {
        int kp = wrap(k + 1, g->nth), km = wrap(k - 1, g->nth);
        double ax = glide_vel(g, r, u, nb, ix, iy, k, 0);
        double ay = glide_vel(g, r, u, nb, ix, iy, k, 1);
        double Ae = 0.5 * (ax + glide_vel(g, r, u, nb, xp, iy, k, 0));
        double Aw = 0.5 * (glide_vel(g, r, u, nb, xm, iy, k, 0) + ax);
        double An = 0.5 * (ay + glide_vel(g, r, u, nb, ix, yp, k, 1));
        double As = 0.5 * (glide_vel(g, r, u, nb, ix, ym, k, 1) + ay);
        double pc = psi[pidx(g, ix, iy, k)];
        double Fe = donor(Ae, pc, psi[pidx(g, xp, iy, k)]);
        double Fw = donor(Aw, psi[pidx(g, xm, iy, k)], pc);
        double Fn = donor(An, pc, psi[pidx(g, ix, yp, k)]);
        double Fs = donor(As, psi[pidx(g, ix, ym, k)], pc);
        double wp = omega_at(G, (k + 0.5) * dth);
        double wm = omega_at(G, (k - 0.5) * dth);
        double Fp = donor(wp, pc, psi[pidx(g, ix, iy, kp)]);
        double Fm = donor(wm, psi[pidx(g, ix, iy, km)], pc);
        out[pidx(g, ix, iy, k)] =
            pc - dt * ((Fe - Fw) / dx + (Fn - Fs) / dy + (Fp - Fm) / dth);
      }
    }
}

/* ---------------------------------------------------- bound-motor kinetics */

/* Walking fluxes of one s-row (Eq. 4, d_s term at walking speed v):
 * Phi[0] = Phi_{-1/2} = 0 (nothing walks on at the minus end),
 * Phi[j+1] = Phi_{j+1/2} = v (M_j + sigma_j / 2) for j < ns-1 with the
 * Superbee slope sigma_j (ghost M_{-1} = 0), and the plus-end outflow
 * Phi[ns] = v M_{ns-1}. */
static void walk_fluxes(int ns, double v, const double* M, double* Phi) {
  Phi[0] = 0.0;
  for (int j = 0; j + 1 < ns; ++j) {
    double mm = j > 0 ? M[j - 1] : 0.0;
    double ca, cb;
    double sig = superbee(M[j] - mm, M[j + 1] - M[j], &ca, &cb);
    Phi[j + 1] = v * (M[j] + 0.5 * sig);
  }
  Phi[ns] = v * M[ns - 1];
}

/* Right-hand side of Eq. 4 on one row:
 * R_j = -(Phi_{j+1/2} - Phi_{j-1/2}) / ds - k_off M_j + k_on Mf. */
static void motor_rhs(const or_grid* g, const or_rates* r, const double* M, double mf,
                      double* Phi, double* R) {
  double ds = ds_of(g);
  walk_fluxes(g->ns, r->v_walk, M, Phi);
  for (int j = 0; j < g->ns; ++j)
    R[j] = -(Phi[j + 1] - Phi[j]) / ds - r->k_off * M[j] + r->k_on * mf;
}

/* ------------------------------------------------------------- public API */

/* Adaptive substep (Sec. 2: dt* limited by the motor speed and the binding and
 * unbinding rates; here also by the filament advection of Eq. 1):
 * dt = cfl / max(v/ds, max(|ax|/dx + |ay|/dy), max|omega|/dth,
 *                k_off + k_on L max_cell sum_k psi dth). */
int or_dt(const or_grid* g, const or_rates* r, const double* psi, const double* mb,
          const double* u, double* dt_out) {
  if (!grid_ok(g) || !r || !psi || !mb || !u || !dt_out) return OR_ERR_INVALID;
  double dx = dx_of(g), dy = dy_of(g), dth = dth_of(g);
  double* nb = (double*)malloc(sizeof(double) * ncell(g) * g->nth);
  if (!nb) return OR_ERR_NOMEM;
  rows_nb(g, mb, nb);
  double adv = 0.0, rot = 0.0, rho_max = 0.0;
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix) {
      double G[4];
      vel_grad(g, u, ix, iy, G);
      double rho = 0.0;
      for (int k = 0; k < g->nth; ++k) {
        double ax = glide_vel(g, r, u, nb, ix, iy, k, 0);
        double ay = glide_vel(g, r, u, nb, ix, iy, k, 1);
        adv = dmax(adv, fabs(ax) / dx + fabs(ay) / dy);
        rot = dmax(rot, fabs(omega_at(G, (k + 0.5) * dth)) / dth);
        rho += psi[pidx(g, ix, iy, k)] * dth;
      }
      rho_max = dmax(rho_max, rho);
    }
  free(nb);
  double rate = dmax(dmax(r->v_walk / ds_of(g), adv),
                     dmax(rot, r->k_off + r->k_on * g->L * rho_max));
  if (!(rate > 0.0)) return OR_ERR_INVALID;
  *dt_out = r->cfl / rate;
  return OR_OK;
}

/* Coarsened bound motors (Eq. 5 with anchors in the filament's own cell)
 * C = sum_k psi n_b dth, the scale-down clip of Alg. 2 when C exceeds the
 * total M, and the free motors of Eq. 6, Mf = M - C. Used to set up a state;
 * mb is scaled in place where the clip applies. */
int or_init_free(const or_grid* g, const double* psi, double* mb, const double* mtot,
                 double* mf, double* c) {
  if (!grid_ok(g) || !psi || !mb || !mtot || !mf || !c) return OR_ERR_INVALID;
  double dth = dth_of(g);
  double* nb = (double*)malloc(sizeof(double) * ncell(g) * g->nth);
  if (!nb) return OR_ERR_NOMEM;
  rows_nb(g, mb, nb);
  for (size_t i = 0; i < ncell(g); ++i) {
    double C = 0.0;
    for (int k = 0; k < g->nth; ++k) C += psi[i * g->nth + k] * nb[i * g->nth + k] * dth;
    if (mtot[i] < C) {
      double f = mtot[i] / C;
      for (size_t q = i * g->nth * g->ns; q < (i + 1) * g->nth * g->ns; ++q) mb[q] *= f;
      C = mtot[i];
    }
    c[i] = C;
    mf[i] = mtot[i] - C;
  }
  free(nb);
  return OR_OK;
}

/* One substep (Alg. 1 inner loop): psi by Eq. 1, then for every cell the
 * Alg. 2 body -- RK2 half and full stage of Eq. 4 on every (theta, s), the
 * coarse reduction of Eq. 5 (using psi at the new time), the clip, and
 * Eq. 6. psi, mb, mf, c are updated in place. */
int or_substep(const or_grid* g, const or_rates* r, double dt, const double* u,
               double* psi, double* mb, double* mf, double* c, const double* mtot) {
  if (!grid_ok(g) || !r || !u || !psi || !mb || !mf || !c || !mtot) return OR_ERR_INVALID;
  size_t rows = ncell(g) * g->nth;
  int ns = g->ns;
  double ds = ds_of(g), dth = dth_of(g);
  double* nb = (double*)malloc(sizeof(double) * rows);
  double* pn = (double*)malloc(sizeof(double) * rows);
  double* buf = (double*)malloc(sizeof(double) * (5 * (size_t)ns + 2));
  if (!nb || !pn || !buf) { free(nb); free(pn); free(buf); return OR_ERR_NOMEM; }
  double *R = buf, *Ms = buf + ns, *Mss = buf + 2 * ns, *Phi = buf + 3 * ns;

  rows_nb(g, mb, nb);                       /* n_b at the start of the substep */
  psi_transport(g, r, dt, u, psi, nb, pn);  /* Eq. 1 */

  for (size_t i = 0; i < ncell(g); ++i) {
    double Cpre = 0.0;
    for (int k = 0; k < g->nth; ++k) {
      double* M = mb + (i * g->nth + k) * ns;
      /* Alg. 2: half stage to t+dt/2, then full stage to t+dt; Mf frozen. */
      motor_rhs(g, r, M, mf[i], Phi, R);
      for (int j = 0; j < ns; ++j) Ms[j] = M[j] + 0.5 * dt * R[j];
      motor_rhs(g, r, Ms, mf[i], Phi, R);
      for (int j = 0; j < ns; ++j) Mss[j] = M[j] + dt * R[j];
      double nbk = 0.0;
      for (int j = 0; j < ns; ++j) { M[j] = Mss[j]; nbk += Mss[j] * ds; }
      Cpre += pn[i * g->nth + k] * nbk * dth; /* Eq. 5 */
    }
    double C = Cpre;
    if (mtot[i] < Cpre) { /* Alg. 2 scale-down */
      double f = mtot[i] / Cpre;
      for (size_t q = i * g->nth * ns; q < (i + 1) * g->nth * ns; ++q) mb[q] *= f;
      C = mtot[i];
    }
    c[i] = C;
    mf[i] = mtot[i] - C; /* Eq. 6 */
  }
  memcpy(psi, pn, sizeof(double) * rows);
  free(nb); free(pn); free(buf);
  return OR_OK;
}

/* Motor kinetics over a macro interval T with psi frozen and a local substep
 * in every cell -- Alg. 2's "while t* < t*_end" loop per anchor with the
 * independent time steps of Sec. 3.1 (anchors in the filament's own cell).
 * With psi frozen the cells are independent and only the motor rates of
 * Eq. 4 bound the step: rate_i = max(v/ds, k_off + k_on L rho_i),
 * rho_i = sum_k psi dtheta (summed in k order), n_i = max(1, ceil(T rate_i /
 * cfl)) equal substeps of dt_i = T / n_i, each the Alg. 2 body (the RK2 half
 * and full stage of Eq. 4 with Mf frozen over the stages, Eq. 5 with the
 * frozen psi, the scale-down, Eq. 6). nsteps_in (may be NULL) imposes n_i per
 * cell instead; nsteps_out (may be NULL) receives the n_i used. mb, mf, c are
 * updated in place. */
int or_motor_local(const or_grid* g, const or_rates* r, double T, const double* psi, double* mb,
                   double* mf, double* c, const double* mtot, const int* nsteps_in,
                   int* nsteps_out) {
  if (!grid_ok(g) || !r || !psi || !mb || !mf || !c || !mtot) return OR_ERR_INVALID;
  if (!(T > 0.0)) return OR_ERR_INVALID;
  int ns = g->ns;
  double ds = ds_of(g), dth = dth_of(g);
  double* buf = (double*)malloc(sizeof(double) * (5 * (size_t)ns + 2));
  if (!buf) return OR_ERR_NOMEM;
  double *R = buf, *Ms = buf + ns, *Mss = buf + 2 * ns, *Phi = buf + 3 * ns;
  for (size_t i = 0; i < ncell(g); ++i) {
    int n;
    if (nsteps_in) {
      n = nsteps_in[i];
    } else {
      double rho = 0.0;
      for (int k = 0; k < g->nth; ++k) rho += psi[i * g->nth + k] * dth;
      double rate = dmax(r->v_walk / ds, r->k_off + r->k_on * g->L * rho);
      double q = ceil(T * rate / r->cfl);
      n = q < 1.0 ? 1 : (int)q;
    }
    if (nsteps_out) nsteps_out[i] = n;
    double dt = T / n;
    for (int step = 0; step < n; ++step) {
      double Cpre = 0.0;
      for (int k = 0; k < g->nth; ++k) {
        double* M = mb + (i * g->nth + k) * ns;
        motor_rhs(g, r, M, mf[i], Phi, R);
        for (int j = 0; j < ns; ++j) Ms[j] = M[j] + 0.5 * dt * R[j];
        motor_rhs(g, r, Ms, mf[i], Phi, R);
        for (int j = 0; j < ns; ++j) Mss[j] = M[j] + dt * R[j];
        double nbk = 0.0;
        for (int j = 0; j < ns; ++j) { M[j] = Mss[j]; nbk += Mss[j] * ds; }
        Cpre += psi[i * g->nth + k] * nbk * dth; /* Eq. 5, psi frozen */
      }
      double C = Cpre;
      if (mtot[i] < Cpre) { /* Alg. 2 scale-down */
        double f = mtot[i] / Cpre;
        for (size_t q = i * g->nth * ns; q < (i + 1) * g->nth * ns; ++q) mb[q] *= f;
        C = mtot[i];
      }
      c[i] = C;
      mf[i] = mtot[i] - C; /* Eq. 6 */
    }
  }
  free(buf);
  return OR_OK;
}

/* ------------------------------------------------ non-local motor anchors */

/* Anchor of a bound-motor configuration (the next row f2 of the hot path,
 * Eq. 4-6 and Eq. 10 with r0 kept). A motor bound at arclength s of a filament
 * centred at x with orientation theta has its head at x + (l/L) s p (the point
 * where Eq. 10 spreads its force); with the capture radius r_c of Eq. 4 taken
 * to zero its tail r0 sits directly beneath the head, so each configuration
 * (cell i, theta_k, s_j) has exactly one anchor cell: the cell containing
 * x_i + (l/L) s_j p_k. Its offset from cell i, in cells, is
 *   ox = floor(((l/L) L (2j + 1 - ns) / (2 ns)) cos(theta_k) / dx + 1/2)
 *   oy = floor(((l/L) L (2j + 1 - ns) / (2 ns)) sin(theta_k) / dy + 1/2)
 * (s_j written as L (2j + 1 - ns) / (2 ns): products and quotients only, so
 * no compiler fuses a multiply with an add). ox, oy are [nth][ns]. */
static void anchor_offsets(const or_grid* g, const or_rates* r, int* ox, int* oy) {
  double dx = dx_of(g), dy = dy_of(g), dth = dth_of(g);
  for (int k = 0; k < g->nth; ++k) {
    double th = k * dth, ct = cos(th), st = sin(th);
    for (int j = 0; j < g->ns; ++j) {
      double disp = r->ell * g->L * (double)(2 * j + 1 - g->ns) / (2.0 * g->ns);
      ox[k * g->ns + j] = (int)floor(disp * ct / dx + 0.5);
      oy[k * g->ns + j] = (int)floor(disp * st / dy + 0.5);
    }
  }
}

static size_t anchor_of(const or_grid* g, const int* ox, const int* oy, int ix, int iy, int k,
                        int j) {
  return cidx(g, wrap(ix + ox[k * g->ns + j], g->nx), wrap(iy + oy[k * g->ns + j], g->ny));
}

/* Eq. 5 at the anchors, C(r0) = sum over the configurations anchored at r0
 * of psi Mb ds dth (cells i, then k, then j in order), the Alg. 2 scale-down
 * of every configuration anchored where C exceeds the total M, and Eq. 6. */
static int anchor_close(const or_grid* g, const int* ox, const int* oy, const double* psi,
                        double* mb, const double* mtot, double* mf, double* c) {
  size_t nc = ncell(g);
  double ds = ds_of(g), dth = dth_of(g);
  double* cpre = (double*)calloc(nc, sizeof(double));
  double* f = (double*)malloc(sizeof(double) * nc);
  if (!cpre || !f) { free(cpre); free(f); return OR_ERR_NOMEM; }
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix)
      for (int k = 0; k < g->nth; ++k) {
        double p = psi[pidx(g, ix, iy, k)];
        const double* M = mb + pidx(g, ix, iy, k) * g->ns;
        for (int j = 0; j < g->ns; ++j)
          cpre[anchor_of(g, ox, oy, ix, iy, k, j)] += p * M[j] * ds * dth;
      }
  for (size_t a = 0; a < nc; ++a) {
    f[a] = 1.0;
    c[a] = cpre[a];
    if (mtot[a] < cpre[a]) { /* Alg. 2 scale-down */
      f[a] = mtot[a] / cpre[a];
      c[a] = mtot[a];
    }
    mf[a] = mtot[a] - c[a]; /* Eq. 6 */
  }
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix)
      for (int k = 0; k < g->nth; ++k) {
        double* M = mb + pidx(g, ix, iy, k) * g->ns;
        for (int j = 0; j < g->ns; ++j) {
          double fa = f[anchor_of(g, ox, oy, ix, iy, k, j)];
          if (fa != 1.0) M[j] *= fa;
        }
      }
  free(cpre);
  free(f);
  return OR_OK;
}

/* State set-up with anchors: C at the anchors, the scale-down, Mf. */
int or_init_free_anchor(const or_grid* g, const or_rates* r, const double* psi, double* mb,
                        const double* mtot, double* mf, double* c) {
  if (!grid_ok(g) || !r || !psi || !mb || !mtot || !mf || !c) return OR_ERR_INVALID;
  int* ox = (int*)malloc(sizeof(int) * 2 * (size_t)g->nth * g->ns);
  if (!ox) return OR_ERR_NOMEM;
  int* oy = ox + (size_t)g->nth * g->ns;
  anchor_offsets(g, r, ox, oy);
  int rc = anchor_close(g, ox, oy, psi, mb, mtot, mf, c);
  free(ox);
  return rc;
}

/* One substep with non-local anchors: psi by Eq. 1 (unchanged), then every
 * s-row by the RK2 half and full stage of Eq. 4 where the binding term of
 * node j takes the free motors of its own anchor, k_on Mf(r0(i, k, j)) (Mf
 * frozen over both stages), then Eq. 5 at the anchors with psi at the new time,
 * the scale-down per anchor and Eq. 6. */
int or_substep_anchor(const or_grid* g, const or_rates* r, double dt, const double* u,
                      double* psi, double* mb, double* mf, double* c, const double* mtot) {
  if (!grid_ok(g) || !r || !u || !psi || !mb || !mf || !c || !mtot) return OR_ERR_INVALID;
  size_t rows = ncell(g) * g->nth;
  int ns = g->ns;
  double ds = ds_of(g);
  double* nb = (double*)malloc(sizeof(double) * rows);
  double* pn = (double*)malloc(sizeof(double) * rows);
  double* buf = (double*)malloc(sizeof(double) * (6 * (size_t)ns + 2));
  int* ox = (int*)malloc(sizeof(int) * 2 * (size_t)g->nth * ns);
  if (!nb || !pn || !buf || !ox) { free(nb); free(pn); free(buf); free(ox); return OR_ERR_NOMEM; }
  int* oy = ox + (size_t)g->nth * ns;
  double *R = buf, *Ms = buf + ns, *Mss = buf + 2 * ns, *Phi = buf + 3 * ns, *mfj = buf + 5 * ns + 2;
  anchor_offsets(g, r, ox, oy);
  rows_nb(g, mb, nb);
  psi_transport(g, r, dt, u, psi, nb, pn); /* Eq. 1 */
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix)
      for (int k = 0; k < g->nth; ++k) {
        double* M = mb + pidx(g, ix, iy, k) * ns;
        for (int j = 0; j < ns; ++j) mfj[j] = mf[anchor_of(g, ox, oy, ix, iy, k, j)];
        /* Alg. 2 half and full stage, R_j = -dPhi/ds - k_off M_j + k_on Mf(r0) */
        walk_fluxes(ns, r->v_walk, M, Phi);
        for (int j = 0; j < ns; ++j)
          R[j] = -(Phi[j + 1] - Phi[j]) / ds - r->k_off * M[j] + r->k_on * mfj[j];
        for (int j = 0; j < ns; ++j) Ms[j] = M[j] + 0.5 * dt * R[j];
        walk_fluxes(ns, r->v_walk, Ms, Phi);
        for (int j = 0; j < ns; ++j)
          R[j] = -(Phi[j + 1] - Phi[j]) / ds - r->k_off * Ms[j] + r->k_on * mfj[j];
        for (int j = 0; j < ns; ++j) Mss[j] = M[j] + dt * R[j];
        memcpy(M, Mss, sizeof(double) * ns);
      }
  int rc = anchor_close(g, ox, oy, pn, mb, mtot, mf, c); /* Eq. 5, Alg. 2, Eq. 6 */
  memcpy(psi, pn, sizeof(double) * rows);
  free(nb); free(pn); free(buf); free(ox);
  return rc;
}

/* The motor force of Eq. 10 with the anchors kept: the force of a bound
 * configuration acts at its head, i.e. in its anchor cell,
 * F(r0) = F sum over the configurations anchored at r0 of p psi Mb ds dth.
 * F is [2][ny][nx] (x then y component). */
int or_anchor_force(const or_grid* g, const or_rates* r, const double* psi, const double* mb,
                    double* F) {
  if (!grid_ok(g) || !r || !psi || !mb || !F) return OR_ERR_INVALID;
  size_t nc = ncell(g);
  double ds = ds_of(g), dth = dth_of(g);
  int* ox = (int*)malloc(sizeof(int) * 2 * (size_t)g->nth * g->ns);
  if (!ox) return OR_ERR_NOMEM;
  int* oy = ox + (size_t)g->nth * g->ns;
  anchor_offsets(g, r, ox, oy);
  for (size_t a = 0; a < 2 * nc; ++a) F[a] = 0.0;
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix)
      for (int k = 0; k < g->nth; ++k) {
        double th = k * dth_of(g), ct = cos(th), st = sin(th);
        double p = psi[pidx(g, ix, iy, k)];
        const double* M = mb + pidx(g, ix, iy, k) * g->ns;
        for (int j = 0; j < g->ns; ++j) {
          size_t a = anchor_of(g, ox, oy, ix, iy, k, j);
          F[a] += r->force_scale * ct * p * M[j] * ds * dth;
          F[nc + a] += r->force_scale * st * p * M[j] * ds * dth;
        }
      }
  free(ox);
  return OR_OK;
}

/* The anchor offsets themselves ([nth][ns] each), for tests. */
int or_anchor_offsets(const or_grid* g, const or_rates* r, int* ox, int* oy) {
  if (!grid_ok(g) || !r || !ox || !oy) return OR_ERR_INVALID;
  anchor_offsets(g, r, ox, oy);
  return OR_OK;
}

/* ------------------------------------ finite capture radius (the r0 axis) */

/* Eq. 4-6 with the anchor r0 of Sec. 2 kept as an axis of the bound-motor
 * density and a finite capture radius rc: Mb(r0, x, theta, s) is tracked only
 * where the motor head x + (l/L) s p is within reach of r0 (the set B_rc(r0)),
 * and Alg. 2 runs per r0 -- every configuration of B_rc(r0) by the RK2 of
 * Eq. 4, the coarse reduction of Eq. 5 at r0, the scale-down at r0, Eq. 6 at
 * r0. Readings (listed in the design notes):
 *   - r0 ranges over the grid's cells; the cell at offset d from the
 *     filament's cell is within reach of a head when the distance from the
 *     head to the cell's square is at most rc (so at rc = 0 the reach is the
 *     cell under the head, as on the rc -> 0 path);
 *   - a motor keeps its tail while it walks: the walking flux of Eq. 4 acts
 *     along s at fixed r0, so for each (x, theta, r0) the nodes within reach
 *     form walking lines (runs of consecutive nodes), with no inflow at a
 *     line's first node and donor-cell outflow at its last (a head that walks
 *     out of reach lets go, and its motor rejoins the free pool through
 *     Eq. 6), as at the filament's plus end;
 *   - the binding term k_on Mf(r0) of Eq. 4 is shared among the anchors in
 *     reach of the node: k_on Mf(r0) / n_a(k, j), n_a the number of anchors
 *     within reach, so that k_on keeps its meaning of the one-anchor model
 *     (the binding rate against the free motors under the filament) and a
 *     uniform Mf binds the same total at any rc;
 *   - the motors per filament are n_b = sum over anchors and nodes of Mb ds;
 *     the force of Eq. 10 acts at the head, in the cell under it.
 * Storage is the paper's (Sec. 3.2 "Reordering Storage"): anchor-major,
 * mb[r0][c] with c running over the configurations of B_rc(r0) line by line
 * (the template below, the same for every r0), s contiguous within a line. */

/* One walking line of the template: motors of anchor r0 bound to a filament
 * of orientation k centred at x = r0 - (dx, dy) cells, at nodes
 * j0 .. j0 + len - 1; off is the line's first entry in mb[r0][]. */
typedef struct {
  int k, dx, dy, j0, len, off;
} rc_line;

/* Whether the cell at offset (ex, ey) from the filament's cell is within reach
 * of a head at (hx, hy) cells from that cell's lower-left corner: the gap from
 * the head to the cell's square in each direction, in physical units, then
 * the squared distance against rc^2 (evaluated without fused operations). */
static int rc_reach(double hx, double hy, int ex, int ey, double dx, double dy, double rc2) {
  double gx = dmax(dmax((double)ex - hx, hx - (double)(ex + 1)), 0.0);
  double gy = dmax(dmax((double)ey - hy, hy - (double)(ey + 1)), 0.0);
  double px = gx * dx, py = gy * dy;
  return px * px + py * py <= rc2;
}

static int cmp_line(const void* a, const void* b) {
  const rc_line *x = (const rc_line*)a, *y = (const rc_line*)b;
  if (x->j0 != y->j0) return x->j0 < y->j0 ? -1 : 1;
  if (x->dy != y->dy) return x->dy < y->dy ? -1 : 1;
  if (x->dx != y->dx) return x->dx < y->dx ? -1 : 1;
  return 0;
}

/* The template: for each orientation k (in order), every anchor offset in
 * reach of some node, split into runs of consecutive nodes in reach; the lines
 * of one k sorted by (first node, dy, dx). w[k][j] = 1 / n_a(k, j). Returns
 * OR_ERR_INVALID if two offsets of the template could name the same cell of
 * the periodic grid (the reach spans the grid). */
static int rc_build(const or_grid* g, const or_rates* r, double rc, rc_line** out, int* nl_out,
                    int* nconf_out, double* w) {
  if (!(rc >= 0.0) || !isfinite(rc)) return OR_ERR_INVALID;
  int ns = g->ns;
  double dx = dx_of(g), dy = dy_of(g), dth = dth_of(g), rc2 = rc * rc;
  double* hx = (double*)malloc(sizeof(double) * 2 * (size_t)ns);
  int* cnt = (int*)malloc(sizeof(int) * (size_t)ns);
  int cap = 256, nl = 0;
  rc_line* L = (rc_line*)malloc(sizeof(rc_line) * (size_t)cap);
  if (!hx || !cnt || !L) { free(hx); free(cnt); free(L); return OR_ERR_NOMEM; }
  double* hy = hx + ns;
  int minx = 0, maxx = 0, miny = 0, maxy = 0;
  for (int k = 0; k < g->nth; ++k) {
    double th = k * dth, ct = cos(th), st = sin(th);
    double lo_x = 1e300, hi_x = -1e300, lo_y = 1e300, hi_y = -1e300;
    for (int j = 0; j < ns; ++j) {
      double disp = r->ell * g->L * (double)(2 * j + 1 - ns) / (2.0 * ns);
      hx[j] = disp * ct / dx + 0.5;
      hy[j] = disp * st / dy + 0.5;
      lo_x = dmin(lo_x, hx[j]); hi_x = dmax(hi_x, hx[j]);
      lo_y = dmin(lo_y, hy[j]); hi_y = dmax(hi_y, hy[j]);
    }
    int x0 = (int)floor(lo_x - rc / dx) - 1, x1 = (int)floor(hi_x + rc / dx) + 1;
    int y0 = (int)floor(lo_y - rc / dy) - 1, y1 = (int)floor(hi_y + rc / dy) + 1;
    int first = nl;
    for (int ey = y0; ey <= y1; ++ey)
      for (int ex = x0; ex <= x1; ++ex) {
        int j = 0;
        while (j < ns) {
          if (!rc_reach(hx[j], hy[j], ex, ey, dx, dy, rc2)) { ++j; continue; }
          int j0 = j;
          while (j < ns && rc_reach(hx[j], hy[j], ex, ey, dx, dy, rc2)) ++j;
          if (nl == cap) {
            cap *= 2;
            rc_line* L2 = (rc_line*)realloc(L, sizeof(rc_line) * (size_t)cap);
            if (!L2) { free(hx); free(cnt); free(L); return OR_ERR_NOMEM; }
            L = L2;
          }
          rc_line ln = {k, ex, ey, j0, j - j0, 0};
          L[nl++] = ln;
          if (ex < minx) minx = ex;
          if (ex > maxx) maxx = ex;
          if (ey < miny) miny = ey;
          if (ey > maxy) maxy = ey;
        }
      }
    qsort(L + first, (size_t)(nl - first), sizeof(rc_line), cmp_line);
    for (int j = 0; j < ns; ++j) cnt[j] = 0;
    for (int l = first; l < nl; ++l)
      for (int j = L[l].j0; j < L[l].j0 + L[l].len; ++j) cnt[j] += 1;
    if (w)
      for (int j = 0; j < ns; ++j) w[(size_t)k * ns + j] = 1.0 / cnt[j];
  }
  int off = 0;
  for (int l = 0; l < nl; ++l) {
    L[l].off = off;
    off += L[l].len;
  }
  free(hx);
  free(cnt);
  if (maxx - minx >= g->nx || maxy - miny >= g->ny) { free(L); return OR_ERR_INVALID; }
  *out = L;
  *nl_out = nl;
  *nconf_out = off;
  return OR_OK;
}

/* Filament cell x of a line of anchor r0 = (ax, ay). */
static size_t rc_fil(const or_grid* g, const rc_line* l, int ax, int ay) {
  return cidx(g, wrap(ax - l->dx, g->nx), wrap(ay - l->dy, g->ny));
}

/* Motors per filament n_b = sum over anchors and nodes of Mb ds, and the force
 * dipole m1 = sum s_j Mb ds (m1 may be NULL), per (x, theta): a gather over
 * the anchors of every line of each row, in template order. */
static void rc_rows(const or_grid* g, const rc_line* L, int nl, int nconf, const double* mb,
                    double* nb, double* m1) {
  double ds = ds_of(g);
  size_t rows = ncell(g) * g->nth;
  for (size_t q = 0; q < rows; ++q) {
    nb[q] = 0.0;
    if (m1) m1[q] = 0.0;
  }
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix)
      for (int l = 0; l < nl; ++l) {
        size_t a = cidx(g, wrap(ix + L[l].dx, g->nx), wrap(iy + L[l].dy, g->ny));
        const double* M = mb + a * (size_t)nconf + L[l].off;
        double acc = 0.0, acc1 = 0.0;
        for (int q = 0; q < L[l].len; ++q) {
          acc += M[q] * ds;
          acc1 += s_node(g, L[l].j0 + q) * M[q] * ds;
        }
        nb[pidx(g, ix, iy, L[l].k)] += acc;
        if (m1) m1[pidx(g, ix, iy, L[l].k)] += acc1;
      }
}

/* Eq. 5 at every anchor, C(r0) = sum over B_rc(r0) of psi Mb ds dth (lines in
 * template order), the Alg. 2 scale-down of B_rc(r0) where C exceeds the
 * total M, and Eq. 6. */
static void rc_close(const or_grid* g, const rc_line* L, int nl, int nconf, const double* psi,
                     double* mb, const double* mtot, double* mf, double* c) {
  double ds = ds_of(g), dth = dth_of(g);
  for (int ay = 0; ay < g->ny; ++ay)
    for (int ax = 0; ax < g->nx; ++ax) {
      size_t a = cidx(g, ax, ay);
      double* Ma = mb + a * (size_t)nconf;
      double C = 0.0;
      for (int l = 0; l < nl; ++l) {
        double nbl = 0.0;
        for (int q = 0; q < L[l].len; ++q) nbl += Ma[L[l].off + q] * ds;
        C += psi[rc_fil(g, &L[l], ax, ay) * g->nth + L[l].k] * nbl * dth;
      }
      if (mtot[a] < C) { /* Alg. 2 scale-down */
        double f = mtot[a] / C;
        for (int q = 0; q < nconf; ++q) Ma[q] *= f;
        C = mtot[a];
      }
      c[a] = C;
      mf[a] = mtot[a] - C; /* Eq. 6 */
    }
}

/* The template, for tests: lines as 6 ints each (k, dx, dy, j0, len, off)
 * when max_lines allows; the number of lines and of configurations per anchor;
 * w [nth][ns] = 1 / n_a (may be NULL). */
int or_rc_template(const or_grid* g, const or_rates* r, double rc, int* lines, int max_lines,
                   int* nlines, int* nconf, double* w) {
  if (!grid_ok(g) || !r || !nlines || !nconf) return OR_ERR_INVALID;
  rc_line* L;
  int nl, nconf_, st = rc_build(g, r, rc, &L, &nl, &nconf_, w);
  if (st) return st;
  *nlines = nl;
  *nconf = nconf_;
  if (lines && max_lines >= nl)
    for (int l = 0; l < nl; ++l) {
      int* o = lines + 6 * (size_t)l;
      o[0] = L[l].k; o[1] = L[l].dx; o[2] = L[l].dy; o[3] = L[l].j0; o[4] = L[l].len;
      o[5] = L[l].off;
    }
  free(L);
  return OR_OK;
}

/* State set-up with the capture radius: C at every anchor, the scale-down, Mf.
 * mb is [cells][nconf] (anchor-major, template order). */
int or_init_free_rc(const or_grid* g, const or_rates* r, double rc, const double* psi,
                    double* mb, const double* mtot, double* mf, double* c) {
  if (!grid_ok(g) || !r || !psi || !mb || !mtot || !mf || !c) return OR_ERR_INVALID;
  rc_line* L;
  int nl, nconf, st = rc_build(g, r, rc, &L, &nl, &nconf, NULL);
  if (st) return st;
  rc_close(g, L, nl, nconf, psi, mb, mtot, mf, c);
  free(L);
  return OR_OK;
}

/* n_b and m1 per (x, theta) of a state with the capture radius ([cells][nth]). */
int or_rc_rows(const or_grid* g, const or_rates* r, double rc, const double* mb, double* nb,
               double* m1) {
  if (!grid_ok(g) || !r || !mb || !nb) return OR_ERR_INVALID;
  rc_line* L;
  int nl, nconf, st = rc_build(g, r, rc, &L, &nl, &nconf, NULL);
  if (st) return st;
  rc_rows(g, L, nl, nconf, mb, nb, m1);
  free(L);
  return OR_OK;
}

/* One substep with the capture radius: n_b of the state (the gliding speed),
 * psi by Eq. 1, then Alg. 2 per anchor r0: every line of B_rc(r0) by the RK2
 * half and full stage of Eq. 4 (walking along the line; binding
 * k_on Mf(r0) / n_a(k, j) with Mf(r0) frozen over both stages), the coarse
 * reduction of Eq. 5 with psi at the new time, the scale-down at r0, Eq. 6. */
int or_substep_rc(const or_grid* g, const or_rates* r, double rc, double dt, const double* u,
                  double* psi, double* mb, double* mf, double* c, const double* mtot) {
  if (!grid_ok(g) || !r || !u || !psi || !mb || !mf || !c || !mtot) return OR_ERR_INVALID;
  rc_line* L;
  int nl, nconf;
  double* w = (double*)malloc(sizeof(double) * (size_t)g->nth * g->ns);
  if (!w) return OR_ERR_NOMEM;
  int st = rc_build(g, r, rc, &L, &nl, &nconf, w);
  if (st) { free(w); return st; }
  size_t rows = ncell(g) * g->nth;
  int ns = g->ns;
  double ds = ds_of(g), dth = dth_of(g);
  double* nb = (double*)malloc(sizeof(double) * rows);
  double* pn = (double*)malloc(sizeof(double) * rows);
  double* buf = (double*)malloc(sizeof(double) * (5 * (size_t)ns + 2));
  if (!nb || !pn || !buf) { free(w); free(L); free(nb); free(pn); free(buf); return OR_ERR_NOMEM; }
  double *R = buf, *Ms = buf + ns, *Mss = buf + 2 * ns, *Phi = buf + 3 * ns;
  rc_rows(g, L, nl, nconf, mb, nb, NULL);   /* n_b at the start of the substep */
  psi_transport(g, r, dt, u, psi, nb, pn);  /* Eq. 1 */
  for (int ay = 0; ay < g->ny; ++ay)
    for (int ax = 0; ax < g->nx; ++ax) {
      size_t a = cidx(g, ax, ay);
      double* Ma = mb + a * (size_t)nconf;
      double mfa = mf[a], Cpre = 0.0;
      for (int l = 0; l < nl; ++l) {
        const rc_line* ln = &L[l];
        double* M = Ma + ln->off;
        const double* wl = w + (size_t)ln->k * ns + ln->j0;
        int n = ln->len;
        /* Alg. 2: half stage to t+dt/2, then full stage to t+dt; Mf frozen */
        walk_fluxes(n, r->v_walk, M, Phi);
        for (int q = 0; q < n; ++q)
          R[q] = -(Phi[q + 1] - Phi[q]) / ds - r->k_off * M[q] + r->k_on * mfa * wl[q];
        for (int q = 0; q < n; ++q) Ms[q] = M[q] + 0.5 * dt * R[q];
        walk_fluxes(n, r->v_walk, Ms, Phi);
        for (int q = 0; q < n; ++q)
          R[q] = -(Phi[q + 1] - Phi[q]) / ds - r->k_off * Ms[q] + r->k_on * mfa * wl[q];
        for (int q = 0; q < n; ++q) Mss[q] = M[q] + dt * R[q];
        double nbl = 0.0;
        for (int q = 0; q < n; ++q) { M[q] = Mss[q]; nbl += Mss[q] * ds; }
        Cpre += pn[rc_fil(g, ln, ax, ay) * g->nth + ln->k] * nbl * dth; /* Eq. 5 */
      }
      double C = Cpre;
      if (mtot[a] < Cpre) { /* Alg. 2 scale-down at r0 */
        double f = mtot[a] / Cpre;
        for (int q = 0; q < nconf; ++q) Ma[q] *= f;
        C = mtot[a];
      }
      c[a] = C;
      mf[a] = mtot[a] - C; /* Eq. 6 */
    }
  memcpy(psi, pn, sizeof(double) * rows);
  free(w); free(L); free(nb); free(pn); free(buf);
  return OR_OK;
}

/* The motor force of Eq. 10 with the capture radius: every configuration's
 * force F p psi Mb ds dth acts at its head, in the cell under
 * x + (l/L) s_j p_k (the cell offset of the rc -> 0 anchors). F [2][ny][nx]. */
int or_rc_force(const or_grid* g, const or_rates* r, double rc, const double* psi,
                const double* mb, double* F) {
  if (!grid_ok(g) || !r || !psi || !mb || !F) return OR_ERR_INVALID;
  rc_line* L;
  int nl, nconf, st = rc_build(g, r, rc, &L, &nl, &nconf, NULL);
  if (st) return st;
  size_t nc = ncell(g);
  double ds = ds_of(g), dth = dth_of(g);
  int* ox = (int*)malloc(sizeof(int) * 2 * (size_t)g->nth * g->ns);
  if (!ox) { free(L); return OR_ERR_NOMEM; }
  int* oy = ox + (size_t)g->nth * g->ns;
  anchor_offsets(g, r, ox, oy);
  for (size_t q = 0; q < 2 * nc; ++q) F[q] = 0.0;
  for (int ay = 0; ay < g->ny; ++ay)
    for (int ax = 0; ax < g->nx; ++ax) {
      const double* Ma = mb + cidx(g, ax, ay) * (size_t)nconf;
      for (int l = 0; l < nl; ++l) {
        int k = L[l].k;
        int fx = wrap(ax - L[l].dx, g->nx), fy = wrap(ay - L[l].dy, g->ny);
        double th = k * dth, ct = cos(th), stn = sin(th);
        double p = psi[pidx(g, fx, fy, k)];
        for (int q = 0; q < L[l].len; ++q) {
          int j = L[l].j0 + q;
          size_t h = anchor_of(g, ox, oy, fx, fy, k, j);
          double m = Ma[L[l].off + q];
          F[h] += r->force_scale * ct * p * m * ds * dth;
          F[nc + h] += r->force_scale * stn * p * m * ds * dth;
        }
      }
    }
  free(ox);
  free(L);
  return OR_OK;
}

int or_run(const or_grid* g, const or_rates* r, double dt, const double* u, double* psi,
           double* mb, double* mf, double* c, const double* mtot, int nsub) {
  for (int n = 0; n < nsub; ++n) {
    int rc = or_substep(g, r, dt, u, psi, mb, mf, c, mtot);
    if (rc) return rc;
  }
  return OR_OK;
}

/* Macroscale moments (Alg. 1, after the inner loop).
 * Per cell, fields[f][ny][nx] for f =
 *   0 rho = sum psi dth          1,2 P = sum psi p dth
 *   3,4 Q = sum psi (pp - I/2) dth (xx, xy)
 *   5 C (coarse bound motors, Eq. 5)      6 Mf (Eq. 6)
 *   7,8 F = F_m sum_k p psi n_b dth       (Eq. 10 with anchors in the cell)
 *   9,10,11 sigma_a = F_m ell sum_k p p psi m1 dth (xx, xy, yy), with the
 *           force dipole m1 = sum_j s_j Mb_j ds (first moment of Eq. 10's
 *           spreading in s).
 * scalars[8]: total filament number sum psi dx dy dth, total bound
 *   sum C dx dy, total free sum Mf dx dy, total motors (bound + free),
 *   polar order |sum psi e^{i theta}| / sum psi, mean over cells of
 *   tr sigma_a, sum psi cos, sum psi sin (over all cells and angles). */
/* The moments from the per-row sums n_b and m1 ([cells][nth]); F (may be
 * NULL) replaces fields 7, 8 (the force acting elsewhere than in the
 * filament's cell). */
static void moments_rows(const or_grid* g, const or_rates* r, const double* psi,
                         const double* nb, const double* m1, const double* mf, const double* c,
                         const double* F, double* fields, double* scalars) {
  size_t nc = ncell(g);
  double dth = dth_of(g), dA = dx_of(g) * dy_of(g);
  double Ntot = 0.0, bound = 0.0, freem = 0.0, sc = 0.0, ss = 0.0, spsi = 0.0, tr = 0.0;
  for (size_t i = 0; i < nc; ++i) {
    double f[12] = {0};
    for (int k = 0; k < g->nth; ++k) {
      double th = k * dth, ct = cos(th), st = sin(th);
      double p = psi[i * g->nth + k];
      double nbk = nb[i * g->nth + k], m1k = m1[i * g->nth + k];
      f[0] += p * dth;
      f[1] += p * ct * dth;
      f[2] += p * st * dth;
      f[3] += p * (ct * ct - 0.5) * dth;
      f[4] += p * ct * st * dth;
      f[7] += r->force_scale * ct * p * nbk * dth;
      f[8] += r->force_scale * st * p * nbk * dth;
      f[9] += r->force_scale * r->ell * ct * ct * p * m1k * dth;
      f[10] += r->force_scale * r->ell * ct * st * p * m1k * dth;
      f[11] += r->force_scale * r->ell * st * st * p * m1k * dth;
      sc += p * ct;
      ss += p * st;
      spsi += p;
    }
    f[5] = c[i];
    f[6] = mf[i];
    if (F) {
      f[7] = F[i];
      f[8] = F[nc + i];
    }
    for (int q = 0; q < 12; ++q) fields[(size_t)q * nc + i] = f[q];
    Ntot += f[0] * dA;
    bound += c[i] * dA;
    freem += mf[i] * dA;
    tr += f[9] + f[11];
  }
  scalars[0] = Ntot;
  scalars[1] = bound;
  scalars[2] = freem;
  scalars[3] = bound + freem;
  scalars[4] = sqrt(sc * sc + ss * ss) / spsi;
  scalars[5] = tr / (double)nc;
  scalars[6] = sc;
  scalars[7] = ss;
}

int or_moments(const or_grid* g, const or_rates* r, const double* psi, const double* mb,
               const double* mf, const double* c, double* fields, double* scalars) {
  if (!grid_ok(g) || !r || !psi || !mb || !mf || !c || !fields || !scalars) return OR_ERR_INVALID;
  size_t rows = ncell(g) * g->nth;
  double ds = ds_of(g);
  double* nb = (double*)malloc(sizeof(double) * 2 * rows);
  if (!nb) return OR_ERR_NOMEM;
  double* m1 = nb + rows;
  for (size_t q = 0; q < rows; ++q) {
    const double* M = mb + q * g->ns;
    double nbk = 0.0, m1k = 0.0;
    for (int j = 0; j < g->ns; ++j) {
      nbk += M[j] * ds;
      m1k += s_node(g, j) * M[j] * ds;
    }
    nb[q] = nbk;
    m1[q] = m1k;
  }
  moments_rows(g, r, psi, nb, m1, mf, c, NULL, fields, scalars);
  free(nb);
  return OR_OK;
}

/* The moments of a state with the capture radius: n_b and m1 summed over the
 * anchors, C and Mf per anchor, and the force of Eq. 10 at the heads. */
int or_moments_rc(const or_grid* g, const or_rates* r, double rc, const double* psi,
                  const double* mb, const double* mf, const double* c, double* fields,
                  double* scalars) {
  if (!grid_ok(g) || !r || !psi || !mb || !mf || !c || !fields || !scalars) return OR_ERR_INVALID;
  size_t rows = ncell(g) * g->nth;
  double* nb = (double*)malloc(sizeof(double) * (2 * rows + 2 * ncell(g)));
  if (!nb) return OR_ERR_NOMEM;
  double *m1 = nb + rows, *F = nb + 2 * rows;
  int st = or_rc_rows(g, r, rc, mb, nb, m1);
  if (!st) st = or_rc_force(g, r, rc, psi, mb, F);
  if (!st) moments_rows(g, r, psi, nb, m1, mf, c, F, fields, scalars);
  free(nb);
  return st;
}

/* ------------------------------------------------- tangent-linear substep */

/* Directional derivative of the walking fluxes of one row, at state M, along
 * dM, with walking speed v and speed perturbation dv. */
static void walk_fluxes_tl(int ns, double v, double dv, const double* M, const double* dM,
                           double* dPhi) {
  dPhi[0] = 0.0;
  for (int j = 0; j + 1 < ns; ++j) {
    double mm = j > 0 ? M[j - 1] : 0.0, dmm = j > 0 ? dM[j - 1] : 0.0;
    double ca, cb;
    double sig = superbee(M[j] - mm, M[j + 1] - M[j], &ca, &cb);
    double dsig = ca * (dM[j] - dmm) + cb * (dM[j + 1] - dM[j]);
    dPhi[j + 1] = v * (dM[j] + 0.5 * dsig) + dv * (M[j] + 0.5 * sig);
  }
  dPhi[ns] = v * dM[ns - 1] + dv * M[ns - 1];
}

/* dp = {d k_off, d v_walk, d k_on}. */
static void motor_rhs_tl(const or_grid* g, const or_rates* r, const double* dp,
                         const double* M, const double* dM, double mf, double dmf,
                         double* dPhi, double* dR) {
  double ds = ds_of(g);
  walk_fluxes_tl(g->ns, r->v_walk, dp[1], M, dM, dPhi);
  for (int j = 0; j < g->ns; ++j)
    dR[j] = -(dPhi[j + 1] - dPhi[j]) / ds - r->k_off * dM[j] - dp[0] * M[j] +
            r->k_on * dmf + dp[2] * mf;
}

/* Derivative of the face flux donor(A, pl, pr) along (dA, dpl, dpr), taking
 * the branch the forward pass takes (A > 0 upwinds from the left). */
static double donor_tl(double A, double pl, double pr, double dA, double dpl, double dpr) {
  return dmax(A, 0.0) * dpl + dmin(A, 0.0) * dpr + dA * (A > 0.0 ? pl : pr);
}

/* Tangent of one substep. (psi, mb, mf) is the state at step n (read only);
 * (dpsi, dmb, dmf) enter as the tangent at step n and leave as the tangent at
 * step n+1. du is the velocity perturbation, dp = {d k_off, d v_walk, d k_on};
 * dt is held fixed. */
int or_tangent_substep(const or_grid* g, const or_rates* r, double dt, const double* u,
                       const double* du, const double* dp, const double* psi,
                       const double* mb, const double* mf, const double* mtot,
                       double* dpsi, double* dmb, double* dmf) {
  if (!grid_ok(g) || !r || !u || !du || !dp || !psi || !mb || !mf || !mtot || !dpsi || !dmb ||
      !dmf)
    return OR_ERR_INVALID;
  size_t rows = ncell(g) * g->nth, nc = ncell(g);
  int ns = g->ns;
  double dx = dx_of(g), dy = dy_of(g), dth = dth_of(g), ds = ds_of(g);
  double* nb = (double*)malloc(sizeof(double) * rows);
  double* dnb = (double*)malloc(sizeof(double) * rows);
  double* pn = (double*)malloc(sizeof(double) * rows);
  double* dpn = (double*)malloc(sizeof(double) * rows);
  double* buf = (double*)malloc(sizeof(double) * (10 * (size_t)ns + 4));
  if (!nb || !dnb || !pn || !dpn || !buf) {
    free(nb); free(dnb); free(pn); free(dpn); free(buf);
    return OR_ERR_NOMEM;
  }
  double *R = buf, *Ms = buf + ns, *Mss = buf + 2 * ns, *Phi = buf + 3 * ns;
  double *dR = buf + 4 * ns + 1, *dMs = buf + 5 * ns + 1, *dMss = buf + 6 * ns + 1,
         *dPhi = buf + 7 * ns + 1;

  rows_nb(g, mb, nb);
  rows_nb(g, dmb, dnb);
  psi_transport(g, r, dt, u, psi, nb, pn);

  /* tangent of Eq. 1 */
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix) {
      double G[4], dG[4];
      vel_grad(g, u, ix, iy, G);
      vel_grad(g, du, ix, iy, dG);
      int xp = wrap(ix + 1, g->nx), xm = wrap(ix - 1, g->nx);
      int yp = wrap(iy + 1, g->ny), ym = wrap(iy - 1, g->ny);
      for (int k = 0; k < g->nth; ++k) {
        int kp = wrap(k + 1, g->nth), km = wrap(k - 1, g->nth);
        double th = k * dth, ct = cos(th), st = sin(th);
        /* a = u - (v_sp + glide nb) p ; da = du - glide dnb p */
#define AX(X, Y) glide_vel(g, r, u, nb, X, Y, k, 0)
#define AY(X, Y) glide_vel(g, r, u, nb, X, Y, k, 1)
#define DAX(X, Y) (du[cidx(g, X, Y)] - r->glide * dnb[pidx(g, X, Y, k)] * ct)
#define DAY(X, Y) (du[nc + cidx(g, X, Y)] - r->glide * dnb[pidx(g, X, Y, k)] * st)
        double Ae = 0.5 * (AX(ix, iy) + AX(xp, iy)), dAe = 0.5 * (DAX(ix, iy) + DAX(xp, iy));
        double Aw = 0.5 * (AX(xm, iy) + AX(ix, iy)), dAw = 0.5 * (DAX(xm, iy) + DAX(ix, iy));
        double An = 0.5 * (AY(ix, iy) + AY(ix, yp)), dAn = 0.5 * (DAY(ix, iy) + DAY(ix, yp));
        double As = 0.5 * (AY(ix, ym) + AY(ix, iy)), dAs = 0.5 * (DAY(ix, ym) + DAY(ix, iy));
#undef AX
#undef AY
#undef DAX
#undef DAY
        double pc = psi[pidx(g, ix, iy, k)], dpc = dpsi[pidx(g, ix, iy, k)];
        double dFe = donor_tl(Ae, pc, psi[pidx(g, xp, iy, k)], dAe, dpc, dpsi[pidx(g, xp, iy, k)]);
        double dFw = donor_tl(Aw, psi[pidx(g, xm, iy, k)], pc, dAw, dpsi[pidx(g, xm, iy, k)], dpc);
        double dFn = donor_tl(An, pc, psi[pidx(g, ix, yp, k)], dAn, dpc, dpsi[pidx(g, ix, yp, k)]);
        double dFs = donor_tl(As, psi[pidx(g, ix, ym, k)], pc, dAs, dpsi[pidx(g, ix, ym, k)], dpc);
        double phip = (k + 0.5) * dth, phim = (k - 0.5) * dth;
        double wp = omega_at(G, phip), wm = omega_at(G, phim);
        double dwp = omega_at(dG, phip), dwm = omega_at(dG, phim); /* omega is linear in G */
        double dFp = donor_tl(wp, pc, psi[pidx(g, ix, iy, kp)], dwp, dpc, dpsi[pidx(g, ix, iy, kp)]);
        double dFm = donor_tl(wm, psi[pidx(g, ix, iy, km)], pc, dwm, dpsi[pidx(g, ix, iy, km)], dpc);
        dpn[pidx(g, ix, iy, k)] = dpc - dt * ((dFe - dFw) / dx + (dFn - dFs) / dy + (dFp - dFm) / dth);
      }
    }

  /* tangent of Eq. 4-6 */
  for (size_t i = 0; i < nc; ++i) {
    double Cpre = 0.0, dCpre = 0.0;
    for (int k = 0; k < g->nth; ++k) {
      const double* M = mb + (i * g->nth + k) * ns;
      double* dM = dmb + (i * g->nth + k) * ns;
      motor_rhs(g, r, M, mf[i], Phi, R);
      motor_rhs_tl(g, r, dp, M, dM, mf[i], dmf[i], dPhi, dR);
      for (int j = 0; j < ns; ++j) {
        Ms[j] = M[j] + 0.5 * dt * R[j];
        dMs[j] = dM[j] + 0.5 * dt * dR[j];
      }
      motor_rhs(g, r, Ms, mf[i], Phi, R);
      motor_rhs_tl(g, r, dp, Ms, dMs, mf[i], dmf[i], dPhi, dR);
      double nbk = 0.0, dnbk = 0.0;
      for (int j = 0; j < ns; ++j) {
        Mss[j] = M[j] + dt * R[j];
        dMss[j] = dM[j] + dt * dR[j];
        nbk += Mss[j] * ds;
        dnbk += dMss[j] * ds;
        dM[j] = dMss[j]; /* unclipped tangent, fixed below if the clip applies */
      }
      Cpre += pn[i * g->nth + k] * nbk * dth;
      dCpre += (dpn[i * g->nth + k] * nbk + pn[i * g->nth + k] * dnbk) * dth;
    }
    if (mtot[i] < Cpre) {
      /* Mb' = f Mb** with f = M / Cpre: dMb' = f dMb** - f (dCpre / Cpre) Mb** */
      double f = mtot[i] / Cpre, df = -f * dCpre / Cpre;
      for (int k = 0; k < g->nth; ++k) {
        const double* M = mb + (i * g->nth + k) * ns;
        double* dM = dmb + (i * g->nth + k) * ns;
        motor_rhs(g, r, M, mf[i], Phi, R);
        for (int j = 0; j < ns; ++j) Ms[j] = M[j] + 0.5 * dt * R[j];
        motor_rhs(g, r, Ms, mf[i], Phi, R);
        for (int j = 0; j < ns; ++j) dM[j] = f * dM[j] + df * (M[j] + dt * R[j]);
      }
      dmf[i] = 0.0;
    } else {
      dmf[i] = -dCpre;
    }
  }
  memcpy(dpsi, dpn, sizeof(double) * rows);
  free(nb); free(dnb); free(pn); free(dpn); free(buf);
  return OR_OK;
}

/* ---------------------------------------------------------- adjoint substep */

/* Transpose of the walking-flux part of R at state M: given y = adjoint of R,
 * add J^T y to z and the v-derivative to *gv. Includes only the d_s term. */
static void walk_adj(const or_grid* g, const or_rates* r, const double* M, const double* y,
                     double* z, double* gv) {
  int ns = g->ns;
  double ds = ds_of(g), v = r->v_walk;
  /* Phi_{j+1/2} enters R_j with -1/ds and R_{j+1} with +1/ds. */
  for (int j = 0; j + 1 < ns; ++j) {
    double lphi = (y[j + 1] - y[j]) / ds;
    double mm = j > 0 ? M[j - 1] : 0.0;
    double ca, cb;
    double sig = superbee(M[j] - mm, M[j + 1] - M[j], &ca, &cb);
    *gv += lphi * (M[j] + 0.5 * sig);
    double la = 0.5 * v * lphi * ca, lb = 0.5 * v * lphi * cb;
    z[j] += v * lphi + la - lb;
    if (j > 0) z[j - 1] -= la;
    z[j + 1] += lb;
  }
  double lout = -y[ns - 1] / ds;
  *gv += lout * M[ns - 1];
  z[ns - 1] += v * lout;
}

/* Transpose of R: z += J_R(M)^T y; grads {k_off, v_walk, k_on} += dR/dp^T y;
 * *lmf += dR/dMf^T y. */
static void motor_rhs_adj(const or_grid* g, const or_rates* r, const double* M, double mf,
                          const double* y, double* z, double* gp, double* lmf) {
  walk_adj(g, r, M, y, z, &gp[1]);
  for (int j = 0; j < g->ns; ++j) {
    z[j] += -r->k_off * y[j];
    gp[0] += -M[j] * y[j];
    gp[2] += mf * y[j];
    *lmf += r->k_on * y[j];
  }
}

/* Adjoint of one substep (reverse of or_substep at fixed dt).
 * (psi, mb, mf) is the state at step n (read only). (lpsi, lmb, lmf) enter as
 * the adjoint at step n+1 and leave as the adjoint at step n. lu [2][ny][nx]
 * and lp = {k_off, v_walk, k_on} are accumulated (+=). */
int or_adjoint_substep(const or_grid* g, const or_rates* r, double dt, const double* u,
                       const double* psi, const double* mb, const double* mf,
                       const double* mtot, double* lpsi, double* lmb, double* lmf,
                       double* lu, double* lp) {
  if (!grid_ok(g) || !r || !u || !psi || !mb || !mf || !mtot || !lpsi || !lmb || !lmf || !lu ||
      !lp)
    return OR_ERR_INVALID;
  size_t rows = ncell(g) * g->nth, nc = ncell(g);
  int ns = g->ns;
  double dx = dx_of(g), dy = dy_of(g), dth = dth_of(g), ds = ds_of(g);
  double* nb = (double*)malloc(sizeof(double) * rows);
  double* pn = (double*)malloc(sizeof(double) * rows);
  double* lpn = (double*)malloc(sizeof(double) * rows);  /* adjoint of psi^{n+1} */
  double* lpo = (double*)calloc(rows, sizeof(double));   /* adjoint of psi^n */
  double* lnb = (double*)calloc(rows, sizeof(double));   /* adjoint of nb^n */
  double* lG = (double*)calloc(4 * nc, sizeof(double));  /* adjoint of grad u */
  double* lmfo = (double*)calloc(nc, sizeof(double));    /* adjoint of Mf^n */
  double* buf = (double*)malloc(sizeof(double) * (10 * (size_t)ns + 4));
  if (!nb || !pn || !lpn || !lpo || !lnb || !lG || !lmfo || !buf) {
    free(nb); free(pn); free(lpn); free(lpo); free(lnb); free(lG); free(lmfo); free(buf);
    return OR_ERR_NOMEM;
  }
  double *R = buf, *Ms = buf + ns, *Mss = buf + 2 * ns, *Phi = buf + 3 * ns;
  double *lMss = buf + 4 * ns + 1, *lMs = buf + 5 * ns + 1, *lM = buf + 6 * ns + 1,
         *y = buf + 7 * ns + 1;

  rows_nb(g, mb, nb);
  psi_transport(g, r, dt, u, psi, nb, pn);
  memcpy(lpn, lpsi, sizeof(double) * rows);

  /* Reverse of Eq. 4-6 for every cell. */
  for (size_t i = 0; i < nc; ++i) {
    double Cpre = 0.0;
    for (int k = 0; k < g->nth; ++k) {
      const double* M = mb + (i * g->nth + k) * ns;
      motor_rhs(g, r, M, mf[i], Phi, R);
      for (int j = 0; j < ns; ++j) Ms[j] = M[j] + 0.5 * dt * R[j];
      motor_rhs(g, r, Ms, mf[i], Phi, R);
      double nbk = 0.0;
      for (int j = 0; j < ns; ++j) nbk += (M[j] + dt * R[j]) * ds;
      Cpre += pn[i * g->nth + k] * nbk * dth;
    }
    int clip = mtot[i] < Cpre;
    double f = clip ? mtot[i] / Cpre : 1.0;
    /* adjoint of Cpre: from Mf' = M - Cpre (no clip) or from Mb' = f Mb** */
    double lC;
    if (clip) {
      double dot = 0.0; /* sum lMb' * Mb** */
      for (int k = 0; k < g->nth; ++k) {
        const double* M = mb + (i * g->nth + k) * ns;
        motor_rhs(g, r, M, mf[i], Phi, R);
        for (int j = 0; j < ns; ++j) Ms[j] = M[j] + 0.5 * dt * R[j];
        motor_rhs(g, r, Ms, mf[i], Phi, R);
        for (int j = 0; j < ns; ++j) dot += lmb[(i * g->nth + k) * ns + j] * (M[j] + dt * R[j]);
      }
      lC = -f * dot / Cpre;
    } else {
      lC = -lmf[i];
    }
    for (int k = 0; k < g->nth; ++k) {
      const double* M = mb + (i * g->nth + k) * ns;
      double* lrow = lmb + (i * g->nth + k) * ns;
      /* forward recompute of the row */
      motor_rhs(g, r, M, mf[i], Phi, R);
      for (int j = 0; j < ns; ++j) Ms[j] = M[j] + 0.5 * dt * R[j];
      motor_rhs(g, r, Ms, mf[i], Phi, R);
      double nbk = 0.0;
      for (int j = 0; j < ns; ++j) { Mss[j] = M[j] + dt * R[j]; nbk += Mss[j] * ds; }
      /* Cpre = sum_k psi' nb** dth */
      lpn[i * g->nth + k] += lC * nbk * dth;
      double lnbk = lC * pn[i * g->nth + k] * dth;
      for (int j = 0; j < ns; ++j) lMss[j] = f * lrow[j] + lnbk * ds;
      /* Mss = M + dt R(Ms) */
      for (int j = 0; j < ns; ++j) { y[j] = dt * lMss[j]; lMs[j] = 0.0; lM[j] = lMss[j]; }
      motor_rhs_adj(g, r, Ms, mf[i], y, lMs, lp, &lmfo[i]);
      /* Ms = M + dt/2 R(M) */
      for (int j = 0; j < ns; ++j) { lM[j] += lMs[j]; y[j] = 0.5 * dt * lMs[j]; }
      motor_rhs_adj(g, r, M, mf[i], y, lM, lp, &lmfo[i]);
      for (int j = 0; j < ns; ++j) lrow[j] = lM[j];
    }
  }

  /* Reverse of Eq. 1: psi' = psi - dt (dFx/dx + dFy/dy + dFth/dth).
   * Each face flux F = donor(A, pl, pr) with adjoint lF = dt/h (l_right - l_left). */
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix) {
      double G[4];
      vel_grad(g, u, ix, iy, G);
      int xp = wrap(ix + 1, g->nx), yp = wrap(iy + 1, g->ny);
      for (int k = 0; k < g->nth; ++k) {
        double th = k * dth, ct = cos(th), st = sin(th);
        size_t c0 = pidx(g, ix, iy, k);
        lpo[c0] += lpn[c0];
        /* east face of (ix,iy): left = (ix,iy), right = (xp,iy) */
        {
          size_t c1 = pidx(g, xp, iy, k);
          double A = 0.5 * (glide_vel(g, r, u, nb, ix, iy, k, 0) + glide_vel(g, r, u, nb, xp, iy, k, 0));
          double lF = dt / dx * (lpn[c1] - lpn[c0]);
          lpo[c0] += dmax(A, 0.0) * lF;
          lpo[c1] += dmin(A, 0.0) * lF;
          double lA = (A > 0.0 ? psi[c0] : psi[c1]) * lF;
          lu[cidx(g, ix, iy)] += 0.5 * lA;
          lu[cidx(g, xp, iy)] += 0.5 * lA;
          lnb[c0] += -0.5 * lA * r->glide * ct;
          lnb[c1] += -0.5 * lA * r->glide * ct;
        }
        /* north face: left = (ix,iy), right = (ix,yp) */
        {
          size_t c1 = pidx(g, ix, yp, k);
          double A = 0.5 * (glide_vel(g, r, u, nb, ix, iy, k, 1) + glide_vel(g, r, u, nb, ix, yp, k, 1));
          double lF = dt / dy * (lpn[c1] - lpn[c0]);
          lpo[c0] += dmax(A, 0.0) * lF;
          lpo[c1] += dmin(A, 0.0) * lF;
          double lA = (A > 0.0 ? psi[c0] : psi[c1]) * lF;
          lu[nc + cidx(g, ix, iy)] += 0.5 * lA;
          lu[nc + cidx(g, ix, yp)] += 0.5 * lA;
          lnb[c0] += -0.5 * lA * r->glide * st;
          lnb[c1] += -0.5 * lA * r->glide * st;
        }
        /* theta face k+1/2: left = k, right = k+1 */
        {
          size_t c1 = pidx(g, ix, iy, wrap(k + 1, g->nth));
          double phi = (k + 0.5) * dth;
          double w = omega_at(G, phi);
          double lF = dt / dth * (lpn[c1] - lpn[c0]);
          lpo[c0] += dmax(w, 0.0) * lF;
          lpo[c1] += dmin(w, 0.0) * lF;
          double lw = (w > 0.0 ? psi[c0] : psi[c1]) * lF;
          double dw[4];
          omega_dG(phi, dw);
          for (int q = 0; q < 4; ++q) lG[(size_t)q * nc + cidx(g, ix, iy)] += lw * dw[q];
        }
      }
    }
  /* central-difference transpose: G from u */
  for (int iy = 0; iy < g->ny; ++iy)
    for (int ix = 0; ix < g->nx; ++ix) {
      size_t ci = cidx(g, ix, iy);
      int xp = wrap(ix + 1, g->nx), xm = wrap(ix - 1, g->nx);
      int yp = wrap(iy + 1, g->ny), ym = wrap(iy - 1, g->ny);
      double lxx = lG[ci], lxy = lG[nc + ci], lyx = lG[2 * nc + ci], lyy = lG[3 * nc + ci];
      lu[cidx(g, xp, iy)] += lxx / (2.0 * dx);
      lu[cidx(g, xm, iy)] -= lxx / (2.0 * dx);
      lu[cidx(g, ix, yp)] += lxy / (2.0 * dy);
      lu[cidx(g, ix, ym)] -= lxy / (2.0 * dy);
      lu[nc + cidx(g, xp, iy)] += lyx / (2.0 * dx);
      lu[nc + cidx(g, xm, iy)] -= lyx / (2.0 * dx);
      lu[nc + cidx(g, ix, yp)] += lyy / (2.0 * dy);
      lu[nc + cidx(g, ix, ym)] -= lyy / (2.0 * dy);
    }
  /* nb^n = sum_j Mb^n ds feeds the gliding speed */
  for (size_t q = 0; q < rows; ++q)
    for (int j = 0; j < ns; ++j) lmb[q * ns + j] += lnb[q] * ds;
  memcpy(lpsi, lpo, sizeof(double) * rows);
  memcpy(lmf, lmfo, sizeof(double) * nc);
  free(nb); free(pn); free(lpn); free(lpo); free(lnb); free(lG); free(lmfo); free(buf);
  return OR_OK;
}
