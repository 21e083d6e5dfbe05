// Auxiliary kernels: precision conversion, state set-up (Eq. 5-6 with the
// Alg. 2 scale-down), the maxima of the adaptive-substep rule, and the
// macroscale moments (Alg. 1 after the inner loop; Eq. 10's force and force
// dipole with anchors in the filament's own cell).
#include "mm_internal.cuh"

namespace mm {

namespace {

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Sum over the block of one value per thread; result valid in thread 0.
// `red` holds at least 32 doubles. Ends with a barrier so `red` can be reused.
__device__ double block_sum(double x, double* red) {
  x = warp_sum(x);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

template <typename TO, typename TI>
__global__ void k_convert(TO* out, const TI* in, size_t n, const double* scale) {
  const double sc = scale ? *scale : 1.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    if (scale)
      out[i] = (TO)((double)in[i] * sc);
    else
      out[i] = (TO)in[i];
  }
}

// Per cell: n_b of every row (sequential sum over s in float64, stored in the
// state precision), C = sum_k psi n_b dtheta, the Alg. 2 scale-down where
// C > M, Mf = M - C.
template <typename T>
__global__ void k_init_cells(T* mb, const T* psi, T* nb, double* mf, double* c,
                             const double* mtot, long long ncells, int nth, int ns, double ds,
                             double dth) {
  __shared__ double red[32];
  __shared__ double s_f;
  for (long long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nth; k += blockDim.x) {
      const T* row = mb + ((size_t)cell * nth + k) * ns;
      double s0 = 0.0;
      for (int j = 0; j < ns; ++j) s0 += (double)row[j] * ds;
      nb[cell * nth + k] = (T)s0;
      acc += (double)psi[cell * nth + k] * s0 * dth;
    }
    const double C = block_sum(acc, red);
    if (threadIdx.x == 0) {
      const double M = mtot[cell];
      double f = 1.0, Cc = C;
      if (M < C) {
        f = M / C;
        Cc = M;
      }
      s_f = f;
      c[cell] = Cc;
      mf[cell] = M - Cc;
    }
    __syncthreads();
    const double f = s_f;
    if (f != 1.0) {
      for (int k = threadIdx.x; k < nth; k += blockDim.x) {
        T* row = mb + ((size_t)cell * nth + k) * ns;
        for (int j = 0; j < ns; ++j) row[j] = (T)((double)row[j] * f);
        nb[cell * nth + k] = (T)((double)nb[cell * nth + k] * f);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // Non-negative doubles order like their bit patterns as unsigned integers.
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Maxima of the adaptive-substep rule: max(|ax|/dx + |ay|/dy),
// max |omega(theta_{k+1/2})| / dtheta, and max_cell sum_k psi dtheta.
template <typename T>
__global__ void k_dt_max(const T* psi, const T* nb, const double* u64, const double* trig,
                         long long ncells, int nx, int ny, int nth, double inv_dx, double inv_dy,
                         double inv_dth, double dth, double glide, double vsp, DevParams* prm) {
  __shared__ double red[32];
  const double psi_scale = prm->psi_scale;
  double adv = 0.0, rot = 0.0, rhomax = 0.0;
  const double* ux = u64;
  const double* uy = u64 + ncells;
  for (long long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
    const int ix = (int)(cell % nx), iy = (int)(cell / nx);
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const double Gxx = (ux[(long long)iy * nx + xp] - ux[(long long)iy * nx + xm]) * 0.5 * inv_dx;
    const double Gxy = (ux[(long long)yp * nx + ix] - ux[(long long)ym * nx + ix]) * 0.5 * inv_dy;
    const double Gyx = (uy[(long long)iy * nx + xp] - uy[(long long)iy * nx + xm]) * 0.5 * inv_dx;
    const double Gyy = (uy[(long long)yp * nx + ix] - uy[(long long)ym * nx + ix]) * 0.5 * inv_dy;
    double rho = 0.0;
    for (int k = threadIdx.x; k < nth; k += blockDim.x) {
      const double V = vsp + glide * (double)nb[cell * nth + k];
      const double ax = ux[cell] - V * trig[k], ay = uy[cell] - V * trig[nth + k];
      adv = fmax(adv, fabs(ax) * inv_dx + fabs(ay) * inv_dy);
      const double cp = trig[2 * nth + k], sp = trig[3 * nth + k];
      const double w = -sp * (Gxx * cp + Gxy * sp) + cp * (Gyx * cp + Gyy * sp);
      rot = fmax(rot, fabs(w) * inv_dth);
      rho += (double)psi[cell * nth + k] * psi_scale * dth;
    }
    const double r = block_sum(rho, red);
    if (threadIdx.x == 0) rhomax = fmax(rhomax, r);
  }
  adv = warp_max(adv);
  rot = warp_max(rot);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&prm->dtmax[0], adv);
    atomic_max_nonneg(&prm->dtmax[1], rot);
  }
  if (threadIdx.x == 0) atomic_max_nonneg(&prm->dtmax[2], rhomax);
}

// Moments per cell (one CTA per cell, threads over theta) and per-CTA
// partial global sums; the last CTA adds the partials in a fixed order. The
// s-reductions feeding the force and the force dipole -- n_b = sum_j Mb ds and
// m1 = sum_j s_j Mb ds -- are recomputed here from Mb in float64 sequential
// sums, in both precisions.
template <typename T>
__global__ void k_moments(const T* psi, const T* mb, const double* mf, const double* c,
                          const double* trig, long long ncells, int nth, int ns, double dth,
                          double ds, double L, double dA, double* fields, double* partial,
                          DevParams* prm) {
  __shared__ double red[32];
  __shared__ unsigned int s_last;
  const double g = prm->psi_scale;
  const double Fm = prm->force_scale, ell = prm->ell;
  // global accumulators: N_psi, bound, free, sum psi cos, sum psi sin, sum psi, sum tr
  double gs[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
    double f[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < nth; k += blockDim.x) {
      const double ct = trig[k], st = trig[nth + k];
      const double p = (double)psi[cell * nth + k] * g;
      const T* row = mb + ((size_t)cell * nth + k) * ns;
      double nbk = 0.0, m1k = 0.0;
      for (int j = 0; j < ns; ++j) {
        const double mj = (double)row[j];
        nbk += mj * ds;
        m1k += (-0.5 * L + (j + 0.5) * ds) * mj * ds;
      }
      f[0] += p * dth;
      f[1] += p * ct * dth;
      f[2] += p * st * dth;
      f[3] += p * (ct * ct - 0.5) * dth;
      f[4] += p * ct * st * dth;
      f[5] += Fm * ct * p * nbk * dth;
      f[6] += Fm * st * p * nbk * dth;
      f[7] += Fm * ell * ct * ct * p * m1k * dth;
      f[8] += Fm * ell * ct * st * p * m1k * dth;
      f[9] += Fm * ell * st * st * p * m1k * dth;
      gs[3] += p * ct;
      gs[4] += p * st;
      gs[5] += p;
    }
    double tot[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) tot[q] = block_sum(f[q], red);
    if (threadIdx.x == 0) {
      const double cc = c[cell], ff = mf[cell];
      fields[0 * ncells + cell] = tot[0];
      fields[1 * ncells + cell] = tot[1];
      fields[2 * ncells + cell] = tot[2];
      fields[3 * ncells + cell] = tot[3];
      fields[4 * ncells + cell] = tot[4];
      fields[5 * ncells + cell] = cc;
      fields[6 * ncells + cell] = ff;
      fields[7 * ncells + cell] = tot[5];
      fields[8 * ncells + cell] = tot[6];
      fields[9 * ncells + cell] = tot[7];
      fields[10 * ncells + cell] = tot[8];
      fields[11 * ncells + cell] = tot[9];
      gs[0] += tot[0] * dA;
      gs[1] += cc * dA;
      gs[2] += ff * dA;
      gs[6] += tot[7] + tot[9];
    }
  }
  double tot[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) tot[q] = block_sum(gs[q], red);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 7; ++q) partial[(size_t)blockIdx.x * 8 + q] = tot[q];
    __threadfence();
    const unsigned int prev = atomicInc(&prm->counter2, gridDim.x - 1);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (threadIdx.x == 0) {
      double t[7] = {0, 0, 0, 0, 0, 0, 0};
      for (unsigned int b = 0; b < gridDim.x; ++b)
        for (int q = 0; q < 7; ++q) t[q] += __ldcg(partial + (size_t)b * 8 + q);
      prm->scalars[0] = t[0];
      prm->scalars[1] = t[1];
      prm->scalars[2] = t[2];
      prm->scalars[3] = t[1] + t[2];
      prm->scalars[4] = sqrt(t[3] * t[3] + t[4] * t[4]) / t[5];
      prm->scalars[5] = t[6] / (double)ncells;
      prm->scalars[6] = t[3];
      prm->scalars[7] = t[4];
      prm->sum_psi = t[5];
    }
  }
}

// Per-cell velocity data of the psi transport: the cell's own u, the x
// component at the east/west neighbours, the y component at the north/south
// neighbours, and the central-difference velocity gradient G_ab = du_a/dx_b.
template <typename T>
__global__ void k_prep_ucell(T* ucell, const double* u64, long long ncells, int nx, int ny,
                             double inv_dx, double inv_dy) {
  const double* ux = u64;
  const double* uy = u64 + ncells;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ncells;
       cell += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(cell % nx), iy = (int)(cell / nx);
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const long long ce = (long long)iy * nx + xp, cw = (long long)iy * nx + xm;
    const long long cn = (long long)yp * nx + ix, cs = (long long)ym * nx + ix;
    T* o = ucell + cell * 12;
    o[0] = (T)ux[cell];
    o[1] = (T)uy[cell];
    o[2] = (T)ux[ce];
    o[3] = (T)ux[cw];
    o[4] = (T)uy[cn];
    o[5] = (T)uy[cs];
    // differences of the stored (precision T) velocities, as the oracle
    // differences its own velocity array
    o[6] = ((T)ux[ce] - (T)ux[cw]) * (T)(0.5 * inv_dx);
    o[7] = ((T)ux[cn] - (T)ux[cs]) * (T)(0.5 * inv_dy);
    o[8] = ((T)uy[ce] - (T)uy[cw]) * (T)(0.5 * inv_dx);
    o[9] = ((T)uy[cn] - (T)uy[cs]) * (T)(0.5 * inv_dy);
    o[10] = T(0);
    o[11] = T(0);
  }
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <typename TO, typename TI>
cudaError_t launch_convert(TO* out, const TI* in, size_t n, const double* scale, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_convert<TO, TI><<<grid_for((long long)n, 256), 256, 0, s>>>(out, in, n, scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prep_ucell(T* ucell, const double* u64, long long ncells, int nx, int ny,
                              double inv_dx, double inv_dy, cudaStream_t s) {
  k_prep_ucell<T><<<grid_for(ncells, 256), 256, 0, s>>>(ucell, u64, ncells, nx, ny, inv_dx, inv_dy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_cells(T* mb, const T* psi, T* nb, double* mf, double* c,
                              const double* mtot, long long ncells, int nth, int ns, double ds,
                              double dth, cudaStream_t s) {
  int block = nth >= 128 ? 128 : (nth >= 64 ? 64 : 32);
  long long g = ncells < 152 * 16 ? ncells : 152 * 16;
  k_init_cells<T><<<(int)g, block, 0, s>>>(mb, psi, nb, mf, c, mtot, ncells, nth, ns, ds, dth);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dt_max(const T* psi, const T* nb, const double* u64, const double* trig,
                          long long ncells, int nx, int ny, int nth, double inv_dx,
                          double inv_dy, double inv_dth, double dth, double glide, double vsp,
                          DevParams* prm, cudaStream_t s) {
  int block = nth >= 128 ? 128 : (nth >= 64 ? 64 : 32);
  long long g = ncells < 152 * 8 ? ncells : 152 * 8;
  k_dt_max<T><<<(int)g, block, 0, s>>>(psi, nb, u64, trig, ncells, nx, ny, nth, inv_dx, inv_dy,
                                       inv_dth, dth, glide, vsp, prm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(const T* psi, const T* mb, const double* mf, const double* c,
                           const double* trig, long long ncells, int nth, int ns, double dth,
                           double ds, double L, double dA, double* fields, double* partial,
                           int nblocks, DevParams* prm, cudaStream_t s) {
  int block = nth >= 128 ? 128 : (nth >= 64 ? 64 : 32);
  k_moments<T><<<nblocks, block, 0, s>>>(psi, mb, mf, c, trig, ncells, nth, ns, dth, ds, L, dA,
                                         fields, partial, prm);
  return cudaGetLastError();
}

template cudaError_t launch_convert<float, double>(float*, const double*, size_t, const double*,
                                                   cudaStream_t);
template cudaError_t launch_convert<double, float>(double*, const float*, size_t, const double*,
                                                   cudaStream_t);
template cudaError_t launch_convert<double, double>(double*, const double*, size_t,
                                                    const double*, cudaStream_t);
template cudaError_t launch_prep_ucell<float>(float*, const double*, long long, int, int, double,
                                              double, cudaStream_t);
template cudaError_t launch_prep_ucell<double>(double*, const double*, long long, int, int,
                                               double, double, cudaStream_t);
template cudaError_t launch_init_cells<float>(float*, const float*, float*, double*, double*,
                                              const double*, long long, int, int, double, double,
                                              cudaStream_t);
template cudaError_t launch_init_cells<double>(double*, const double*, double*, double*, double*,
                                               const double*, long long, int, int, double, double,
                                               cudaStream_t);
template cudaError_t launch_dt_max<float>(const float*, const float*, const double*,
                                          const double*, long long, int, int, int, double, double,
                                          double, double, double, double, DevParams*,
                                          cudaStream_t);
template cudaError_t launch_dt_max<double>(const double*, const double*, const double*,
                                           const double*, long long, int, int, int, double,
                                           double, double, double, double, double,
                                           DevParams*, cudaStream_t);
template cudaError_t launch_moments<float>(const float*, const float*, const double*,
                                           const double*, const double*, long long, int, int,
                                           double, double, double, double, double*, double*, int,
                                           DevParams*, cudaStream_t);
template cudaError_t launch_moments<double>(const double*, const double*, const double*,
                                            const double*, const double*, long long, int, int,
                                            double, double, double, double, double*, double*, int,
                                            DevParams*, cudaStream_t);

}  // namespace mm
