// Filament diffusion (the -D_t grad ln psi and -D_r d_theta ln psi fluxes of
// Eq. 2-3: d_t psi = D_t lap_x psi + D_r d_theta^2 psi) by Crank-Nicolson, the
// scheme Sec. 2 / Alg. 1 use for the diffusive terms of the psi update, taken
// one direction at a time (theta, x, y). Each direction is a batch of
// constant-coefficient periodic tridiagonal systems
//   (I - a/2 L) psi' = (I + a/2 L) psi,  (L psi)_i = psi_{i-1} - 2 psi_i + psi_{i+1},
// one per line, solved by one thread per line: a Thomas sweep for the
// tridiagonal part with the periodic corners folded in by the Sherman-Morrison
// formula (the factors are the same for every line). Arithmetic in float64,
// storage in the state precision; the line is overwritten in place (forward
// sweep, back substitution, correction). The factors are computed on the
// device too, so a call needs no host round trip.
#include "mm_internal.cuh"

namespace mm {

namespace {

// Factors of one periodic direction of n >= 2 points with a = D dt / h^2
// (one thread per direction): the matrix I - a/2 L (diagonal b = 1 + a,
// off-diagonals and corners c = -a/2) is T + u v^T with T tridiagonal
// (corners removed, T_00 = b - gamma, T_{n-1,n-1} = b - c^2 / gamma,
// gamma = -b), u = (gamma, 0, .., 0, c), v = (1, 0, .., 0, c / gamma).
// tab: cp[n], 1/m[n] of T's Thomas elimination, z[n] = T^{-1} u, then
// r = c / gamma and vzf = 1 / (1 + v.z).
__global__ void k_cn_factors(double* tab0, int n0, double a0, double* tab1, int n1, double a1,
                             double* tab2, int n2, double a2) {
  const int d = threadIdx.x;
  if (d > 2 || blockIdx.x != 0) return;
  double* tab = d == 0 ? tab0 : d == 1 ? tab1 : tab2;
  const int n = d == 0 ? n0 : d == 1 ? n1 : n2;
  const double a = d == 0 ? a0 : d == 1 ? a1 : a2;
  if (!(a > 0.0) || n < 2) return;
  const double b = 1.0 + a, c = -0.5 * a, gamma = -b;
  double* cp = tab;
  double* im = tab + n;
  double* z = tab + 2 * n;
  for (int i = 0; i < n; ++i) {
    double diag = b;
    if (i == 0) diag = b - gamma;
    if (i == n - 1) diag = b - c * c / gamma;
    const double m = i == 0 ? diag : diag - c * cp[i - 1];
    im[i] = 1.0 / m;
    cp[i] = c / m;
  }
  for (int i = 0; i < n; ++i) {  // T z = u
    const double ui = i == 0 ? gamma : (i == n - 1 ? c : 0.0);
    z[i] = (ui - (i == 0 ? 0.0 : c * z[i - 1])) * im[i];
  }
  for (int i = n - 2; i >= 0; --i) z[i] -= cp[i] * z[i + 1];
  const double r = c / gamma;
  tab[3 * n] = r;
  tab[3 * n + 1] = 1.0 / (1.0 + z[0] + r * z[n - 1]);
}

// One direction for every line: c = -a/2, ha = a/2, the factors in tab.
template <typename T>
__global__ void k_cn_lines(T* psi, int mode, int nx, int ny, int nth, const double* tab, int n,
                           double c, double ha, const double* scale) {
  const long long nlines = mode == 0 ? (long long)nx * ny : mode == 1 ? (long long)ny * nth
                                                                      : (long long)nx * nth;
  const double g = scale ? *scale : 1.0;
  const double* cp = tab;
  const double* im = tab + n;
  const double* z = tab + 2 * n;
  const double r = tab[3 * n], vzf = tab[3 * n + 1];
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < nlines;
       L += (long long)gridDim.x * blockDim.x) {
    size_t base, stride;
    if (mode == 0) {  // theta: a row of the cell, contiguous
      base = (size_t)L * nth;
      stride = 1;
    } else if (mode == 1) {  // x: line (y, k), stride nth
      const long long y = L / nth, k = L - y * nth;
      base = (size_t)y * nx * nth + (size_t)k;
      stride = (size_t)nth;
    } else {  // y: line (x, k), stride nx nth
      const long long x = L / nth, k = L - x * nth;
      base = (size_t)x * nth + (size_t)k;
      stride = (size_t)nx * nth;
    }
    T* p = psi + base;
    // forward sweep with the explicit half step as right-hand side
    const double first = g * (double)p[0];
    double prev = g * (double)p[(size_t)(n - 1) * stride], cur = first, yp = 0.0;
    for (int i = 0; i < n; ++i) {
      const double next = i + 1 < n ? g * (double)p[(size_t)(i + 1) * stride] : first;
      const double d = fma(ha, prev + next, (1.0 - 2.0 * ha) * cur);
      yp = (d - c * yp) * im[i];
      p[(size_t)i * stride] = (T)yp;
      prev = cur;
      cur = next;
    }
    // back substitution (y_{n-1} = y'_{n-1})
    const double ylast = yp;
    double y = yp;
    for (int i = n - 2; i >= 0; --i) {
      y = (double)p[(size_t)i * stride] - cp[i] * y;
      p[(size_t)i * stride] = (T)y;
    }
    // periodic corners: x = y - (v.y) / (1 + v.z) z, v = (1, 0, .., 0, r)
    const double beta = (y + r * ylast) * vzf;
    for (int i = 0; i < n; ++i)
      p[(size_t)i * stride] = (T)((double)p[(size_t)i * stride] - beta * z[i]);
  }
}

__global__ void k_set_scale_one(double* scale) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *scale = 1.0;
}

}  // namespace

cudaError_t launch_cn_factors(double* tab0, int n0, double a0, double* tab1, int n1, double a1,
                              double* tab2, int n2, double a2, cudaStream_t s) {
  k_cn_factors<<<1, 32, 0, s>>>(tab0, n0, a0, tab1, n1, a1, tab2, n2, a2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cn_lines(T* psi, int mode, int nx, int ny, int nth, const double* tab, int n,
                            double c, double ha, const double* scale, cudaStream_t s) {
  const long long nlines = mode == 0 ? (long long)nx * ny : mode == 1 ? (long long)ny * nth
                                                                      : (long long)nx * nth;
  long long g = (nlines + 127) / 128;
  if (g > 152LL * 32) g = 152LL * 32;
  k_cn_lines<T><<<(int)g, 128, 0, s>>>(psi, mode, nx, ny, nth, tab, n, c, ha, scale);
  return cudaGetLastError();
}

cudaError_t launch_set_scale_one(double* scale, cudaStream_t s) {
  k_set_scale_one<<<1, 32, 0, s>>>(scale);
  return cudaGetLastError();
}

template cudaError_t launch_cn_lines<float>(float*, int, int, int, int, const double*, int, double,
                                            double, const double*, cudaStream_t);
template cudaError_t launch_cn_lines<double>(double*, int, int, int, int, const double*, int,
                                             double, double, const double*, cudaStream_t);

}  // namespace mm
