// Fused microscale substep kernel (forward).
//
// One CTA owns one spatial cell at a time (grid-stride over cells) and
// performs the whole substep for it:
//   1. psi^{n+1}(cell, :) by Eq. 1 in donor-cell flux form (x, y faces from the
//      4 neighbour cells, theta faces inside the cell), one thread per theta;
//   2. every s-row Mb(cell, k, :) by Eq. 4 with midpoint RK2 (Alg. 2 half and
//      full stage): the row is spread over `seg` lanes of a warp with V
//      consecutive s-nodes per lane (16-byte vector loads and stores), the
//      Superbee stencil reaches across lanes with warp shuffles, and the row
//      is updated in place;
//   3. n_b and the force dipole m1 of every row by a warp-shuffle reduction
//      over s, the coarse density C = sum_k psi^{n+1} n_b dtheta (Eq. 5), the
//      scale-down of Alg. 2 and Mf = M - C (Eq. 6).
// psi and n_b are double-buffered (neighbour cells read the old values); Mb,
// Mf and C are cell-local and updated in place. Each CTA also sums psi^{n+1}
// in float64; the last CTA to finish adds the partial sums in a fixed order
// (deterministic) and, in the float32 form, stores the mass-correction factor
// applied to psi on the next load.
#include "mm_internal.cuh"

namespace mm {

template <typename T, int V>
struct alignas(sizeof(T) * V) Pack {
  T v[V];
};

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// Donor-cell face flux: upwind state times face velocity. Written with an
// explicit fma so that both cells sharing a face compute the same bits and
// the flux differences telescope exactly.
template <typename T>
__device__ __forceinline__ T donor(T A, T pl, T pr) {
  return fma_t(tmax(A, T(0)), pl, tmin(A, T(0)) * pr);
}

// Half of the Superbee slope, sigma/2 with sigma = maxmod(minmod(2a,b),
// minmod(a,2b)), on magnitudes: with s = sign(b), A = s a, B = |b|,
// sigma/2 = s max(0, max(min(A, B/2), min(A/2, B))). Zero when a and b differ
// in sign or either vanishes.
template <typename T>
__device__ __forceinline__ T half_superbee(T a, T b) {
  const T s = copysign(T(1), b);
  const T A = a * s;
  const T B = fabs(b);
  T r = tmax(tmin(A, T(0.5) * B), tmin(T(0.5) * A, B));
  r = tmax(r, T(0));
  return s * r;
}

template <typename T, int V>
__device__ __forceinline__ void load_row(const T* p, T (&m)[V]) {
  const Pack<T, V> q = *reinterpret_cast<const Pack<T, V>*>(p);
#pragma unroll
  for (int v = 0; v < V; ++v) m[v] = q.v[v];
}
template <typename T, int V>
__device__ __forceinline__ void store_row(T* p, const T (&m)[V]) {
  Pack<T, V> q;
#pragma unroll
  for (int v = 0; v < V; ++v) q.v[v] = m[v];
  *reinterpret_cast<Pack<T, V>*>(p) = q;
}

// Right-hand side of Eq. 4 for the V nodes a lane holds:
// R_j = (v/ds) (F_{j-1} - F_j) - k_off M_j + k_on Mf, F_j = M_j + sigma_j/2
// (walking flux / v through the right face of node j), F_{-1} = 0 (no inflow
// at the minus end), F_{ns-1} = M_{ns-1} (donor-cell outflow at the plus end),
// ghost M_{-1} = 0 in the first slope.
template <typename T, int V>
__device__ __forceinline__ void motor_rhs(const T (&M)[V], T (&R)[V], bool first, bool last,
                                          int seg, T cw, T koff, T src) {
  T ml = __shfl_up_sync(0xffffffffu, M[V - 1], 1, seg);
  const T mr = __shfl_down_sync(0xffffffffu, M[0], 1, seg);
  if (first) ml = T(0);
  T F[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const T mm = v == 0 ? ml : M[v - 1];
    const T mp = v == V - 1 ? mr : M[v + 1];
    F[v] = M[v] + half_superbee(M[v] - mm, mp - M[v]);
  }
  if (last) F[V - 1] = M[V - 1];
  T fl = __shfl_up_sync(0xffffffffu, F[V - 1], 1, seg);
  if (first) fl = T(0);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const T fin = v == 0 ? fl : F[v - 1];
    R[v] = cw * (fin - F[v]) - koff * M[v] + src;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum_seg(T x, int seg) {
  for (int o = seg >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, seg);
  return x;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <typename T>
size_t substep_smem(int nth) {
  return sizeof(double) * (2 * (size_t)nth + 34) + sizeof(T) * 2 * (size_t)nth + 16;
}

template <typename T, int V, bool MASSCORR>
__global__ void __launch_bounds__(256) k_substep(const StepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nth = a.nth, ns = a.ns, seg = a.seg;
  double* s_nb = reinterpret_cast<double*>(smem_raw);
  double* s_m1 = s_nb + nth;
  double* s_red = s_m1 + nth;  // [32] + 2 flags
  T* s_pold = reinterpret_cast<T*>(s_red + 34);
  T* s_pnew = s_pold + nth;

  const int tid = threadIdx.x, NT = blockDim.x;
  const int lane = tid & (seg - 1);
  const int slot = tid / seg, slots = NT / seg;
  const int nl = ns / V;
  const bool first = lane == 0, last = lane == nl - 1;
  const bool lane_ok = lane < nl;

  const DevParams* P = a.prm;
  const double dt64 = P->dt;
  const T dt = (T)dt64, hdt = (T)(0.5 * dt64);
  const T cw = (T)(P->v_walk / a.ds);
  const T koff = (T)P->k_off;
  const double kon64 = P->k_on;
  const T glide = (T)P->glide, vsp = (T)P->v_sp;
  const T g = MASSCORR ? (T)P->psi_scale : T(1);
  const T inv_dx = (T)a.inv_dx, inv_dy = (T)a.inv_dy, inv_dth = (T)a.inv_dth;
  const T hinv_dx = (T)(0.5 * a.inv_dx), hinv_dy = (T)(0.5 * a.inv_dy);
  const T* cosk = a.trig;
  const T* sink = a.trig + nth;
  const T* cosf = a.trig + 2 * nth;
  const T* sinf = a.trig + 3 * nth;
  const long long nc = a.ncells;
  const T* ux = a.u;
  const T* uy = a.u + nc;

  // s_j of this lane's nodes, for the force dipole m1 = sum_j s_j Mb_j ds.
  T sj[V];
#pragma unroll
  for (int v = 0; v < V; ++v) sj[v] = (T)(-0.5 * a.L + ((double)(lane * V + v) + 0.5) * a.ds);

  double mass_acc = 0.0;

  for (long long cell = blockIdx.x; cell < nc; cell += gridDim.x) {
    const int ix = (int)(cell % a.nx), iy = (int)(cell / a.nx);
    // (1) psi^n of this cell into shared memory
    for (int k = tid; k < nth; k += NT) s_pold[k] = g * a.psi_in[cell * nth + k];
    const double mf_n = a.mf[cell];
    const double mtot = a.mtot[cell];
    __syncthreads();

    // (2) Eq. 1: psi^{n+1} = psi^n - dt (dFx/dx + dFy/dy + dFth/dth)
    {
      const int xp = ix + 1 == a.nx ? 0 : ix + 1, xm = ix == 0 ? a.nx - 1 : ix - 1;
      const int yp = iy + 1 == a.ny ? 0 : iy + 1, ym = iy == 0 ? a.ny - 1 : iy - 1;
      const long long ce = (long long)iy * a.nx + xp, cwc = (long long)iy * a.nx + xm;
      const long long cn = (long long)yp * a.nx + ix, cs = (long long)ym * a.nx + ix;
      const T uxc = ux[cell], uxe = ux[ce], uxw = ux[cwc], uxn = ux[cn], uxs = ux[cs];
      const T uyc = uy[cell], uye = uy[ce], uyw = uy[cwc], uyn = uy[cn], uys = uy[cs];
      const T Gxx = (uxe - uxw) * hinv_dx, Gxy = (uxn - uxs) * hinv_dy;
      const T Gyx = (uye - uyw) * hinv_dx, Gyy = (uyn - uys) * hinv_dy;
      for (int k = tid; k < nth; k += NT) {
        const T ck = cosk[k], sk = sink[k];
        const T Vc = vsp + glide * (T)a.nb_in[cell * nth + k];
        const T Ve = vsp + glide * (T)a.nb_in[ce * nth + k];
        const T Vw = vsp + glide * (T)a.nb_in[cwc * nth + k];
        const T Vn = vsp + glide * (T)a.nb_in[cn * nth + k];
        const T Vs = vsp + glide * (T)a.nb_in[cs * nth + k];
        const T axc = fma_t(-Vc, ck, uxc), axe = fma_t(-Ve, ck, uxe), axw = fma_t(-Vw, ck, uxw);
        const T ayc = fma_t(-Vc, sk, uyc), ayn = fma_t(-Vn, sk, uyn), ays = fma_t(-Vs, sk, uys);
        const T Ae = T(0.5) * (axc + axe), Aw = T(0.5) * (axw + axc);
        const T An = T(0.5) * (ayc + ayn), As = T(0.5) * (ays + ayc);
        const T pc = s_pold[k];
        const T pe = g * a.psi_in[ce * nth + k], pw = g * a.psi_in[cwc * nth + k];
        const T pn = g * a.psi_in[cn * nth + k], ps = g * a.psi_in[cs * nth + k];
        const int kp = k + 1 == nth ? 0 : k + 1, km = k == 0 ? nth - 1 : k - 1;
        const T cp = cosf[k], sp = sinf[k], cm = cosf[km], sm = sinf[km];
        // Jeffery rotation p_perp . G . p at the faces k +- 1/2
        const T wp = -sp * (Gxx * cp + Gxy * sp) + cp * (Gyx * cp + Gyy * sp);
        const T wm = -sm * (Gxx * cm + Gxy * sm) + cm * (Gyx * cm + Gyy * sm);
        const T Fe = donor(Ae, pc, pe), Fw = donor(Aw, pw, pc);
        const T Fn = donor(An, pc, pn), Fs = donor(As, ps, pc);
        const T Fp = donor(wp, pc, s_pold[kp]), Fm = donor(wm, s_pold[km], pc);
        const T pnew = pc - dt * ((Fe - Fw) * inv_dx + (Fn - Fs) * inv_dy + (Fp - Fm) * inv_dth);
        s_pnew[k] = pnew;
        a.psi_out[cell * nth + k] = pnew;
        mass_acc += (double)pnew;
      }
    }

    // (3) Eq. 4 on every s-row of the cell, midpoint RK2 with Mf frozen
    const T src = (T)(kon64 * mf_n);
    for (int p = 0; p < a.rpt; ++p) {
      const int k = slot + p * slots;
      const bool row_ok = k < nth;
      const bool act = row_ok && lane_ok;
      T M[V], R[V], Ms[V];
      T* rowp = a.mb + ((size_t)cell * nth + (row_ok ? k : 0)) * ns + (size_t)lane * V;
      if (act) {
        load_row<T, V>(rowp, M);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) M[v] = T(0);
      }
      motor_rhs<T, V>(M, R, first, last, seg, cw, koff, src);
#pragma unroll
      for (int v = 0; v < V; ++v) Ms[v] = M[v] + hdt * R[v];
      motor_rhs<T, V>(Ms, R, first, last, seg, cw, koff, src);
#pragma unroll
      for (int v = 0; v < V; ++v) M[v] = M[v] + dt * R[v];
      if (act) store_row<T, V>(rowp, M);
      T snb = T(0), sm1 = T(0);
      if (act) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          snb += M[v];
          sm1 = fma_t(sj[v], M[v], sm1);
        }
      }
      snb = warp_sum_seg(snb, seg);
      sm1 = warp_sum_seg(sm1, seg);
      if (first && row_ok) {
        s_nb[k] = (double)snb * a.ds;
        s_m1[k] = (double)sm1 * a.ds;
      }
    }
    __syncthreads();

    // (4) Eq. 5 with psi^{n+1}, scale-down of Alg. 2, Eq. 6
    if (tid < 32) {
      double acc = 0.0;
      for (int k = tid; k < nth; k += 32) acc += (double)s_pnew[k] * s_nb[k] * a.dth;
      acc = warp_sum(acc);
      if (tid == 0) {
        double f = 1.0, C = acc;
        if (mtot < acc) {
          f = mtot / acc;
          C = mtot;
        }
        s_red[32] = f;
        a.c[cell] = C;
        a.mf[cell] = mtot - C;
      }
    }
    __syncthreads();
    const double f = s_red[32];
    if (f != 1.0) {  // rare: rescale the rows just written (visible after the barrier)
      const T ft = (T)f;
      for (int p = 0; p < a.rpt; ++p) {
        const int k = slot + p * slots;
        if (k < nth && lane_ok) {
          T* rowp = a.mb + ((size_t)cell * nth + k) * ns + (size_t)lane * V;
          T M[V];
#pragma unroll
          for (int v = 0; v < V; ++v) M[v] = __ldcg(rowp + v) * ft;
          store_row<T, V>(rowp, M);
        }
      }
    }
    for (int k = tid; k < nth; k += NT) {
      a.nb_out[cell * nth + k] = s_nb[k] * f;
      if (a.write_m1) a.m1[cell * nth + k] = s_m1[k] * f;
    }
    __syncthreads();
  }

  // (5) sum psi^{n+1} over the grid: per-CTA partial, last CTA finalises
  __shared__ unsigned int s_last;
  mass_acc = warp_sum(mass_acc);
  if ((tid & 31) == 0) s_red[tid >> 5] = mass_acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (NT + 31) / 32; ++w) t += s_red[w];
    a.partial[blockIdx.x] = t;
    __threadfence();
    const unsigned int prev = atomicInc(&a.prm->counter, gridDim.x - 1);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double t = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += NT) t += __ldcg(a.partial + b);
    t = warp_sum(t);
    if ((tid & 31) == 0) s_red[tid >> 5] = t;
    __syncthreads();
    if (tid == 0) {
      double m = 0.0;
      for (int w = 0; w < (NT + 31) / 32; ++w) m += s_red[w];
      a.prm->mass = m;
      if (MASSCORR && a.mass_correct) a.prm->psi_scale = a.prm->mass0 / m;
    }
  }
}

template <typename T, int V>
cudaError_t launch_substep(const StepArgs<T>& a, int grid, int block, size_t smem,
                           cudaStream_t s) {
  if (a.mass_correct)
    k_substep<T, V, true><<<grid, block, smem, s>>>(a);
  else
    k_substep<T, V, false><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int V>
cudaError_t substep_occupancy(int block, size_t smem, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_substep<T, V, true>,
                                                       block, smem);
}

template size_t substep_smem<float>(int);
template size_t substep_smem<double>(int);
template cudaError_t launch_substep<float, 4>(const StepArgs<float>&, int, int, size_t,
                                              cudaStream_t);
template cudaError_t launch_substep<float, 1>(const StepArgs<float>&, int, int, size_t,
                                              cudaStream_t);
template cudaError_t launch_substep<double, 2>(const StepArgs<double>&, int, int, size_t,
                                               cudaStream_t);
template cudaError_t launch_substep<double, 1>(const StepArgs<double>&, int, int, size_t,
                                               cudaStream_t);
template cudaError_t substep_occupancy<float, 4>(int, size_t, int*);
template cudaError_t substep_occupancy<float, 1>(int, size_t, int*);
template cudaError_t substep_occupancy<double, 2>(int, size_t, int*);
template cudaError_t substep_occupancy<double, 1>(int, size_t, int*);

}  // namespace mm
