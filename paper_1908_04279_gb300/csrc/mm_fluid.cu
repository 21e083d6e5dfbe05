// Thin-gap fluid solve (mm_fluid_setup, mm_fluid_solve): the in-plane velocity
// u_2 on the filament plane z = z0 from Eq. 7-9, with no-slip plates at z = 0
// and z = 1 and periodic x, y over the unit square (Sec. 2). The filaments and
// bound motors sit on the plane z = z0 (Sec. 2), so the right side of Eq. 7 is
// (F_2 + div_2 Sigma) delta(z - z0): F_2 the motor force of Eq. 10 from the
// moments (with, optionally, the first-order term of its spreading in s,
// -div sigma_a), Sigma the caller's extra stress sigma_f S_f - sigma_t S_t.
//
// Per Fourier mode k, |k| = kappa, the transformed Eq. 7-9 are linear ODEs in
// z with constant coefficients and are solved exactly in z:
//   across k:  (kappa^2 - eps^-2 d_zz) u_T = f_T delta(z - z0): the Dirichlet
//              Green's function, g_T = eps^2 sinh(mu z0) sinh(mu (1 - z0)) /
//              (mu sinh mu), mu = eps kappa;
//   along k:   eliminating q and u_L = i w' / kappa from Eq. 7-9 leaves
//              (kappa^2 - eps^-2 d_zz)(d_zz - kappa^2) w = -i kappa f_L delta'(z - z0)
//              with w = w' = 0 at both plates: on each side of z0 a sum of
//              exp(+-kappa z), exp(+-mu z); w, w', w''' continuous and
//              [w''] = i kappa eps^2 f_L at z0. With w = i kappa eps^2 f_L W the
//              eight coefficients of W solve a real 8 x 8 system and
//              g_L = -eps^2 W'(z0).
// The velocity does not depend on P0 (it only scales q). The paper resolves z
// on an adaptive grid; the exact per-mode solve is that grid's limit.
//
// The table (g_T, g_L) per mode of the half spectrum is built once on the
// device (k_fluid_table); each solve is three batched cuFFT transforms and one
// per-mode kernel (k_fluid_modes), all in float64, and writes u_2 into the
// handle's velocity (the substep's adaptive dt is recomputed from it).
#include <cufft.h>

#include "mm_host.h"

static_assert(sizeof(cufftHandle) == sizeof(int), "cuFFT plan handles are stored as int");

namespace mm {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Basis functions of W on one side of z0, in t = kappa s (s >= 0 the distance
// from the function's anchor point, the plate or z0), as n-th derivatives in s
// divided by kappa^n:
//   fl_e:  exp(-kappa s)                                 -> (-1)^n e^{-t}
//   fl_dd: kappa (exp(-mu s) - exp(-kappa s)) / (kappa - mu), rho = mu/kappa = eps,
//          the divided difference that stays independent of exp(-kappa s) as
//          eps -> 1 (limit kappa s exp(-kappa s)):
//          (-1)^n (rho^n e^{-rho t} - e^{-t}) / (1 - rho)
//          = (-1)^n e^{-t} (rho^n expm1((1 - rho) t) / (1 - rho) - sum_{j<n} rho^j).
// The first form is used where |(1 - rho) t| >= 1 (no cancellation), the
// second below (no overflow of expm1).
__host__ __device__ inline double fl_e(int n, double t) {
  const double v = exp(-t);
  return (n & 1) ? -v : v;
}

__host__ __device__ inline double fl_dd(int n, double t, double rho) {
  const double d = 1.0 - rho;
  double rn = 1.0;
  for (int j = 0; j < n; ++j) rn *= rho;
  double v;
  if (fabs(d * t) >= 1.0) {
    v = (rn * exp(-rho * t) - exp(-t)) / d;
  } else {
    const double q = (d == 0.0) ? t : expm1(d * t) / d;
    double sum = 0.0, rj = 1.0;
    for (int j = 0; j < n; ++j) {
      sum += rj;
      rj *= rho;
    }
    v = exp(-t) * (rn * q - sum);
  }
  return (n & 1) ? -v : v;
}

// (g_T, g_L) of one mode: the in-plane velocity at z0 per unit force on the
// plane, across and along k.
__host__ __device__ inline double2 fl_mode_response(double kappa, double eps, double z0) {
  const double e2 = eps * eps;
  if (kappa == 0.0) {
    const double g = e2 * z0 * (1.0 - z0);  // -eps^-2 u'' = f delta: the mean flow
    return make_double2(g, g);
  }
  const double mu = eps * kappa;
  const double gT = e2 * (-expm1(-2.0 * mu * z0)) * (-expm1(-2.0 * mu * (1.0 - z0))) /
                    (2.0 * mu * (-expm1(-2.0 * mu)));
  // Columns: lower side 0..3 (anchors 0, 0, z0, z0), upper side 4..7 (z0, z0,
  // 1, 1); even columns exp, odd columns the divided difference; a function
  // anchored below its interval runs in s = z - a (sign +1), above it in
  // s = a - z (sign -1, so its n-th z-derivative carries (-1)^n).
  const double anchor[8] = {0.0, 0.0, z0, z0, z0, z0, 1.0, 1.0};
  const int sgn[8] = {1, 1, -1, -1, 1, 1, -1, -1};
  auto basis = [&](int c, int n, double z) {
    const double t = kappa * sgn[c] * (z - anchor[c]);
    const double v = (c & 1) ? fl_dd(n, t, eps) : fl_e(n, t);
    return (sgn[c] < 0 && (n & 1)) ? -v : v;
  };
  // Rows (derivative order n scaled by kappa^-n): W = W' = 0 at z = 0 (lower)
  // and z = 1 (upper); upper minus lower at z0 for n = 0..3, right side 1 for
  // n = 2 (the solution is kappa^2 W).
  double A[8][9];
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < 9; ++c) A[r][c] = 0.0;
  for (int n = 0; n < 2; ++n) {
    for (int c = 0; c < 4; ++c) A[n][c] = basis(c, n, 0.0);
    for (int c = 4; c < 8; ++c) A[2 + n][c] = basis(c, n, 1.0);
  }
  for (int n = 0; n < 4; ++n) {
    for (int c = 0; c < 4; ++c) A[4 + n][c] = -basis(c, n, z0);
    for (int c = 4; c < 8; ++c) A[4 + n][c] = basis(c, n, z0);
  }
  A[6][8] = 1.0;
  // Gaussian elimination with partial pivoting
  for (int p = 0; p < 8; ++p) {
    int best = p;
    for (int r = p + 1; r < 8; ++r)
      if (fabs(A[r][p]) > fabs(A[best][p])) best = r;
    if (best != p)
      for (int c = p; c < 9; ++c) {
        const double tmp = A[p][c];
        A[p][c] = A[best][c];
        A[best][c] = tmp;
      }
    const double inv = 1.0 / A[p][p];
    for (int r = p + 1; r < 8; ++r) {
      const double m = A[r][p] * inv;
      if (m != 0.0)
        for (int c = p; c < 9; ++c) A[r][c] -= m * A[p][c];
    }
  }
  double x[8];
  for (int p = 7; p >= 0; --p) {
    double v = A[p][8];
    for (int c = p + 1; c < 8; ++c) v -= A[p][c] * x[c];
    x[p] = v / A[p][p];
  }
  // W'(z0) = (kappa^2 W)'(z0) / kappa^2 = (scaled first derivative) / kappa
  double d1 = 0.0;
  for (int c = 4; c < 8; ++c) d1 += x[c] * basis(c, 1, z0);
  return make_double2(gT, -e2 * d1 / kappa);
}

// Signed integer wavenumber of DFT index j of a length-n axis: j for j <= n/2,
// j - n above.
__host__ __device__ inline int fl_wavenumber(int j, int n) { return j <= n / 2 ? j : j - n; }

__global__ void k_fluid_table(double2* __restrict__ tab, int nx, int ny, int nxh, double eps,
                              double z0) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)ny * nxh) return;
  const int jy = (int)(idx / nxh), jx = (int)(idx % nxh);
  const double my = fl_wavenumber(jy, ny);
  const double kappa = kTwoPi * sqrt((double)jx * jx + my * my);
  tab[idx] = fl_mode_response(kappa, eps, z0);
}

// One mode of the half spectrum: f = F^ + i k . S^ with S = Sigma - dipole
// sigma_a, then u^ = g_T f + (g_L - g_T) k^ (k^ . f), scaled by 1/(nx ny) for
// the inverse transform. At a Nyquist index (jx = nx/2 of an even nx, and
// likewise in y) the map is the mean over both signs of that wavenumber, which
// keeps the output real.
__global__ void k_fluid_modes(const double2* __restrict__ fh, const double2* __restrict__ sh,
                              const double2* __restrict__ tab, double2* __restrict__ uh, int nx,
                              int ny, int nxh, double dipole, double inv_n) {
  const long long nm = (long long)ny * nxh;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nm) return;
  const int jy = (int)(idx / nxh), jx = (int)(idx % nxh);
  const double2 Fx = fh[idx], Fy = fh[nm + idx];
  double2 S[3];
  for (int c = 0; c < 3; ++c) {
    const double2 a = fh[(2 + c) * nm + idx];
    S[c] = make_double2(-dipole * a.x, -dipole * a.y);
    if (sh) {
      const double2 b = sh[c * nm + idx];
      S[c].x += b.x;
      S[c].y += b.y;
    }
  }
  const double2 g = tab[idx];
  const int nsx = (nx % 2 == 0 && jx == nx / 2) ? 2 : 1;
  const int nsy = (ny % 2 == 0 && jy == ny / 2) ? 2 : 1;
  const double kx0 = kTwoPi * jx, ky0 = kTwoPi * fl_wavenumber(jy, ny);
  double2 ux = make_double2(0.0, 0.0), uy = make_double2(0.0, 0.0);
  for (int a = 0; a < nsx; ++a)
    for (int b = 0; b < nsy; ++b) {
      const double kx = a ? -kx0 : kx0, ky = b ? -ky0 : ky0;
      // f = F + i (k . S): i (p + i q) = -q + i p
      const double px = kx * S[0].x + ky * S[1].x, qx = kx * S[0].y + ky * S[1].y;
      const double py = kx * S[1].x + ky * S[2].x, qy = kx * S[1].y + ky * S[2].y;
      const double2 fx = make_double2(Fx.x - qx, Fx.y + px);
      const double2 fy = make_double2(Fy.x - qy, Fy.y + py);
      const double k2 = kx * kx + ky * ky;
      ux.x += g.x * fx.x;
      ux.y += g.x * fx.y;
      uy.x += g.x * fy.x;
      uy.y += g.x * fy.y;
      if (k2 > 0.0) {
        const double c = (g.y - g.x) / k2;  // (g_L - g_T) k k^T / kappa^2
        const double prx = kx * fx.x + ky * fy.x, pry = kx * fx.y + ky * fy.y;
        ux.x += c * kx * prx;
        ux.y += c * kx * pry;
        uy.x += c * ky * prx;
        uy.y += c * ky * pry;
      }
    }
  const double s = inv_n / (nsx * nsy);
  uh[idx] = make_double2(ux.x * s, ux.y * s);
  uh[nm + idx] = make_double2(uy.x * s, uy.y * s);
}

}  // namespace mm

using namespace mmh;

namespace {

mm_status fft_fail(mm_handle* h, const char* what, cufftResult r) {
  return fail(h, MM_ERR_CUDA, std::string(what) + ": cuFFT error " + std::to_string((int)r));
}

#define CKF(what, ...)                                        \
  do {                                                        \
    cufftResult r_ = (__VA_ARGS__);                           \
    if (r_ != CUFFT_SUCCESS) return fft_fail(h, what, r_);    \
  } while (0)

long long fluid_modes(const mm_handle* h) { return (long long)h->g.ny * (h->g.nx / 2 + 1); }

// Cells per field in the transforms' real buffers, rounded up to even: every
// batch of a batched transform then starts on a 16-byte boundary.
size_t fluid_pitch(const mm_handle* h) { return ((size_t)h->ncells + 1) & ~(size_t)1; }

}  // namespace

namespace mmh {

void fluid_free(mm_handle* h) {
  for (int& p : h->fl_plan) {
    if (p >= 0) cufftDestroy((cufftHandle)p);
    p = -1;
  }
  void* ptrs[3] = {h->fl_tab, h->fl_hat, h->fl_real};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->fl_tab = h->fl_hat = h->fl_real = nullptr;
  h->fluid = false;
}

}  // namespace mmh

extern "C" {

mm_status mm_fluid_setup(mm_handle* h, double eps, double z0) {
  MM_TRACE("mm_fluid_setup");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (h->owner) return fail(h, MM_ERR_UNSUPPORTED, "the fluid solve is not available to batch members");
  if (!finite_pos(eps)) return fail(h, MM_ERR_INVALID, "eps must be finite and > 0");
  if (!(z0 > 0.0 && z0 < 1.0)) return fail(h, MM_ERR_INVALID, "z0 must lie strictly between the plates (0, 1)");
  if (h->g.nx < 2 || h->g.ny < 2)
    return fail(h, MM_ERR_UNSUPPORTED, "the fluid solve needs nx >= 2 and ny >= 2");
  DeviceGuard dg(h->device);
  const int nx = h->g.nx, ny = h->g.ny, nxh = nx / 2 + 1;
  const long long nm = fluid_modes(h);
  const int np = (int)fluid_pitch(h);
  if (!h->fl_tab) {
    // all or nothing: a failure frees what this call allocated
    const size_t need = (size_t)nm * 16 * 11 + (size_t)np * 8 * 10;
    size_t freeb = 0, totalb = 0;
    CK(cudaMemGetInfo(&freeb, &totalb));
    if (need + (64u << 20) > freeb) return fail(h, MM_ERR_OOM, "fluid buffers do not fit");
    cudaError_t ae = cudaMalloc((void**)&h->fl_tab, (size_t)nm * 16);
    if (ae == cudaSuccess) ae = cudaMalloc((void**)&h->fl_hat, (size_t)nm * 16 * 10);
    if (ae == cudaSuccess) ae = cudaMalloc((void**)&h->fl_real, (size_t)np * 8 * 10);
    if (ae != cudaSuccess) {
      fluid_free(h);
      return cuda_fail(h, "cudaMalloc (fluid buffers)", ae);
    }
    // explicit embeddings: with NULL ones cuFFT takes the packed layout and
    // ignores the distances between batches
    int n[2] = {ny, nx}, real_e[2] = {ny, nx}, cplx_e[2] = {ny, nxh};
    const int kinds[3] = {CUFFT_D2Z, CUFFT_D2Z, CUFFT_Z2D};
    const int batch[3] = {5, 3, 2};
    for (int i = 0; i < 3; ++i) {
      cufftHandle p;
      const bool fwd = kinds[i] == CUFFT_D2Z;
      cufftResult r = cufftPlanMany(&p, 2, n, fwd ? real_e : cplx_e, 1, fwd ? np : (int)nm,
                                    fwd ? cplx_e : real_e, 1, fwd ? (int)nm : np,
                                    (cufftType)kinds[i], batch[i]);
      if (r != CUFFT_SUCCESS) {
        fluid_free(h);
        return fft_fail(h, "cufftPlanMany", r);
      }
      h->fl_plan[i] = (int)p;
    }
  }
  const int tb = 128;
  mm::k_fluid_table<<<(unsigned)((nm + tb - 1) / tb), tb, 0, h->stream>>>(
      (double2*)h->fl_tab, nx, ny, nxh, eps, z0);
  CK(cudaGetLastError());
  h->fl_eps = eps;
  h->fl_z0 = z0;
  h->fluid = true;
  return MM_OK;
}

mm_status mm_fluid_solve(mm_handle* h, const double* sigma, int sigma_on_device, int dipole,
                         double* u_out, int u_out_on_device) {
  MM_TRACE("mm_fluid_solve");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!h->fluid) return fail(h, MM_ERR_STATE, "no fluid set-up: call mm_fluid_setup first");
  if (!h->have_state) return fail(h, MM_ERR_STATE, "no state: call mm_set_state first");
  if (h->rec.active)
    return fail(h, MM_ERR_STATE, "the fluid solve is not differentiated: end the adjoint recording first");
  if (h->tangent)
    return fail(h, MM_ERR_STATE,
                "the fluid solve is not differentiated (the velocity would carry a tangent): "
                "end the tangent first");
  if (dipole && (h->anchors || h->capture))
    return fail(h, MM_ERR_UNSUPPORTED,
                "with anchors the force already acts in the anchor cells: dipole must be 0");
  DeviceGuard dg(h->device);
  const long long nm = fluid_modes(h);
  const size_t nc = (size_t)h->ncells, np = fluid_pitch(h);
  double2* hat = (double2*)h->fl_hat;
  // real buffers, np values per field: 0-4 force and dipole stress, 5-7 the
  // caller's stress, 8-9 the velocity
  double* re = h->fl_real;
  mm_status st;
  if ((st = run_moments(h)) != MM_OK) return st;
  for (int p : h->fl_plan) CKF("cufftSetStream", cufftSetStream((cufftHandle)p, h->stream));
  if (sigma) {
    CK(cudaMemcpy2DAsync(re + 5 * np, np * 8, sigma, nc * 8, nc * 8, 3,
                         sigma_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         h->stream));
    CKF("cufftExecD2Z (stress)",
        cufftExecD2Z((cufftHandle)h->fl_plan[1], re + 5 * np, (cufftDoubleComplex*)(hat + 5 * nm)));
  }
  // moment fields 7..11: Fx, Fy, sigma_a xx, xy, yy
  CK(cudaMemcpy2DAsync(re, np * 8, h->fields + 7 * nc, nc * 8, nc * 8, 5, cudaMemcpyDeviceToDevice,
                       h->stream));
  CKF("cufftExecD2Z (force)", cufftExecD2Z((cufftHandle)h->fl_plan[0], re, (cufftDoubleComplex*)hat));
  const int tb = 128;
  mm::k_fluid_modes<<<(unsigned)((nm + tb - 1) / tb), tb, 0, h->stream>>>(
      hat, sigma ? hat + 5 * nm : nullptr, (const double2*)h->fl_tab, hat + 8 * nm, h->g.nx,
      h->g.ny, h->g.nx / 2 + 1, dipole ? 1.0 : 0.0, 1.0 / (double)nc);
  CK(cudaGetLastError());
  CKF("cufftExecZ2D", cufftExecZ2D((cufftHandle)h->fl_plan[2], (cufftDoubleComplex*)(hat + 8 * nm),
                                   re + 8 * np));
  CK(cudaMemcpy2DAsync(h->u64, nc * 8, re + 8 * np, np * 8, nc * 8, 2, cudaMemcpyDeviceToDevice,
                       h->stream));
  if ((st = velocity_update(h)) != MM_OK) return st;
  if (u_out) {
    CK(cudaMemcpyAsync(u_out, h->u64, nc * 2 * 8,
                       u_out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!u_out_on_device) return check_status(h);
  }
  return MM_OK;
}

mm_status mm_fluid_response(mm_handle* h, double* out, int on_device) {
  if (!h || !out) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!h->fluid) return fail(h, MM_ERR_STATE, "no fluid set-up: call mm_fluid_setup first");
  DeviceGuard dg(h->device);
  CK(cudaMemcpyAsync(out, h->fl_tab, (size_t)fluid_modes(h) * 16,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (!on_device) return check_status(h);
  return MM_OK;
}

}  // extern "C"
