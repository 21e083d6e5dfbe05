// Filament diffusion (the -D_t grad ln psi and -D_r d_theta ln psi fluxes of
// Eq. 2-3: d_t psi = D_t lap_x psi + D_r d_theta^2 psi) by Crank-Nicolson, the
// scheme Sec. 2 / Alg. 1 use for the diffusive terms of the psi update, taken
// one direction at a time (theta, x, y). Each direction is a batch of
// constant-coefficient periodic tridiagonal systems
//   (I - a/2 L) psi' = (I + a/2 L) psi,  (L psi)_i = psi_{i-1} - 2 psi_i + psi_{i+1},
// one per line, solved by one thread per line: a Thomas sweep for the
// tridiagonal part with the periodic corners folded in by the Sherman-Morrison
// formula (the factors, the same for every line, come precomputed from the
// host). Arithmetic in float64, storage in the state precision; the line is
// overwritten in place (forward sweep, back substitution, correction).
#include "mm_internal.cuh"

namespace mm {

namespace {

// Per-direction constants: cp[n], inv_m[n], z[n] (host-computed), then
// c = -a/2, ha = a/2, r = c / gamma, vzf = 1 / (1 + v.z).
template <typename T>
__global__ void k_cn_lines(T* psi, int mode, int nx, int ny, int nth, const double* tab, int n,
                           double c, double ha, double r, double vzf, const double* scale) {
  const long long nlines = mode == 0 ? (long long)nx * ny : mode == 1 ? (long long)ny * nth
                                                                      : (long long)nx * nth;
  const double g = scale ? *scale : 1.0;
  const double* cp = tab;
  const double* im = tab + n;
  const double* z = tab + 2 * n;
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

template <typename T>
cudaError_t launch_cn_lines(T* psi, int mode, int nx, int ny, int nth, const double* tab, int n,
                            double c, double ha, double r, double vzf, const double* scale,
                            cudaStream_t s) {
  const long long nlines = mode == 0 ? (long long)nx * ny : mode == 1 ? (long long)ny * nth
                                                                      : (long long)nx * nth;
  long long g = (nlines + 127) / 128;
  if (g > 152LL * 32) g = 152LL * 32;
  k_cn_lines<T><<<(int)g, 128, 0, s>>>(psi, mode, nx, ny, nth, tab, n, c, ha, r, vzf, scale);
  return cudaGetLastError();
}

cudaError_t launch_set_scale_one(double* scale, cudaStream_t s) {
  k_set_scale_one<<<1, 32, 0, s>>>(scale);
  return cudaGetLastError();
}

template cudaError_t launch_cn_lines<float>(float*, int, int, int, int, const double*, int, double,
                                            double, double, double, const double*, cudaStream_t);
template cudaError_t launch_cn_lines<double>(double*, int, int, int, int, const double*, int,
                                             double, double, double, double, const double*,
                                             cudaStream_t);

}  // namespace mm
