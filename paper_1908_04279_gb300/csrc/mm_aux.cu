// Auxiliary kernels: precision conversion, state set-up (Eq. 5-6 with the
// Alg. 2 scale-down), the maxima of the adaptive-substep rule, and the
// macroscale moments (Alg. 1 after the inner loop; Eq. 10's force and force
// dipole with anchors in the filament's own cell).
#include "mm_walk.cuh"

namespace mm {

namespace {


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

// The copies of a CopySegs: 16-byte vectors where both addresses are 16-byte
// aligned, then the remaining bytes one by one; every thread of the grid takes
// its share of each segment in turn.
__global__ void k_copy_multi(const CopySegs c) {
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int q = 0; q < c.n; ++q) {
    const unsigned char* s = static_cast<const unsigned char*>(c.src[q]);
    unsigned char* d = static_cast<unsigned char*>(c.dst[q]);
    const size_t b = c.bytes[q];
    const bool vec = ((reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(d)) & 15) == 0;
    const size_t nv = vec ? b / 16 : 0;
    const uint4* s4 = reinterpret_cast<const uint4*>(s);
    uint4* d4 = reinterpret_cast<uint4*>(d);
    for (size_t i = tid; i < nv; i += stride) d4[i] = s4[i];
    for (size_t i = nv * 16 + tid; i < b; i += stride) d[i] = s[i];
  }
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
__global__ void k_init_cells(T* mb, const T* psi, T* nb, T* mf, T* c, const T* mtot,
                             long long ncells, int nth, int ns, double ds, double dth) {
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
      const double M = (double)mtot[cell];
      double f = 1.0, Cc = C;
      if (M < C) {
        f = M / C;
        Cc = M;
      }
      s_f = f;
      c[cell] = (T)Cc;
      mf[cell] = (T)(M - Cc);
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
// max |omega(theta_{k+1/2})| / dtheta, and max_cell sum_k psi dtheta. One warp
// per cell, lanes over theta, in the state precision (float64 in the float64
// form, whose dt must agree with a float64 evaluation; float32 in the float32
// form, whose state is float32 anyway); the maxima are exact.
template <typename T>
__device__ __forceinline__ T warp_max_t(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = tmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

template <typename T>
__global__ void k_dt_max(const T* psi, const T* nb, const T* u, const T* trig, long long ncells,
                         int nx, int ny, int nth, double inv_dx64, double inv_dy64,
                         double inv_dth64, double dth64, double glide64, double vsp64,
                         DevParams* prm) {
  const int lane = threadIdx.x & 31;
  const long long gw = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  const T g = (T)prm->psi_scale;
  const T inv_dx = (T)inv_dx64, inv_dy = (T)inv_dy64, inv_dth = (T)inv_dth64, dth = (T)dth64;
  const T glide = (T)glide64, vsp = (T)vsp64, h = T(0.5);
  T adv = T(0), rot = T(0), rhomax = T(0);
  const T* ux = u;
  const T* uy = u + ncells;
  for (long long cell = gw; cell < ncells; cell += W) {
    const int ix = (int)(cell % nx), iy = (int)(cell / nx);
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const T Gxx = (ux[(long long)iy * nx + xp] - ux[(long long)iy * nx + xm]) * h * inv_dx;
    const T Gxy = (ux[(long long)yp * nx + ix] - ux[(long long)ym * nx + ix]) * h * inv_dy;
    const T Gyx = (uy[(long long)iy * nx + xp] - uy[(long long)iy * nx + xm]) * h * inv_dx;
    const T Gyy = (uy[(long long)yp * nx + ix] - uy[(long long)ym * nx + ix]) * h * inv_dy;
    const T uxc = ux[cell], uyc = uy[cell];
    T rho = T(0);
    for (int k = lane; k < nth; k += 32) {
      const T V = vsp + glide * nb[cell * nth + k];
      const T ax = uxc - V * trig[k], ay = uyc - V * trig[nth + k];
      adv = tmax(adv, fabs(ax) * inv_dx + fabs(ay) * inv_dy);
      const T cp = trig[2 * nth + k], sp = trig[3 * nth + k];
      const T w = -sp * (Gxx * cp + Gxy * sp) + cp * (Gyx * cp + Gyy * sp);
      rot = tmax(rot, fabs(w) * inv_dth);
      rho += psi[cell * nth + k] * g * dth;
    }
    rhomax = tmax(rhomax, warp_sum_t(rho));
  }
  adv = warp_max_t(adv);
  rot = warp_max_t(rot);
  if (lane == 0) {
    atomic_max_nonneg(&prm->dtmax[0], (double)adv);
    atomic_max_nonneg(&prm->dtmax[1], (double)rot);
    atomic_max_nonneg(&prm->dtmax[2], (double)rhomax);
  }
}

// ---- s-row sums for the moments: n_b = sum_j Mb_j ds and m1 = sum_j s_j Mb_j ds

// Compensated float32 accumulator (hi + lo), error-free transformations of
// Knuth (TwoSum) and of the fused multiply-add (TwoProduct).
struct FF {
  float hi, lo;
};
__device__ __forceinline__ void ff_add(FF& a, float x) {
  const float s = a.hi + x;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (x - bb);
  a.hi = s;
  a.lo += e;
}
__device__ __forceinline__ void ff_add_prod(FF& a, float u, float v) {
  const float p = __fmul_rn(u, v);  // not contracted into the sum below
  const float pe = __fmaf_rn(u, v, -p);
  ff_add(a, p);
  a.lo += pe;
}
__device__ __forceinline__ void ff_merge(FF& a, const FF& b) {
  const float lo = a.lo + b.lo;
  a.lo = 0.0f;
  ff_add(a, b.hi);
  a.lo += lo;
}
// a + b (TwoSum of the high parts, low parts added)
__device__ __forceinline__ FF ff_sum(const FF& a, const FF& b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return FF{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
// p w for a float p and a float-float w (TwoProduct of the high part)
__device__ __forceinline__ FF ff_scale(float p, const FF& w) {
  const float h = __fmul_rn(p, w.hi);
  return FF{h, __fmaf_rn(p, w.lo, __fmaf_rn(p, w.hi, -h))};
}
// a w for float-float a and w (the lo * lo term dropped)
__device__ __forceinline__ FF ff_prod(const FF& a, const FF& w) {
  const float h = __fmul_rn(a.hi, w.hi);
  return FF{h, __fmaf_rn(a.hi, w.lo, __fmaf_rn(a.lo, w.hi, __fmaf_rn(a.hi, w.hi, -h)))};
}

// Row sums of the V values a lane holds, reduced over the row's `seg` lanes;
// every lane of the segment gets (n_b / ds, m1 / ds) in float64.
template <int V>
__device__ __forceinline__ void row_sums(const double (&m)[V], const double (&sj)[V], int seg,
                                         double& nb, double& m1) {
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    a += m[v];
    b += sj[v] * m[v];
  }
  for (int o = seg >> 1; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o, seg);
    b += __shfl_xor_sync(0xffffffffu, b, o, seg);
  }
  nb = a;
  m1 = b;
}

// Float32 form: the float-float row sums (n_b / ds and m1 / ds) left
// unconverted; every lane of the segment gets them.
template <int V>
__device__ __forceinline__ void row_sums_ff(const float (&m)[V], const float (&sj)[V], int seg,
                                            FF& a, FF& b) {
  a = FF{0.f, 0.f};
  b = FF{0.f, 0.f};
#pragma unroll
  for (int v = 0; v < V; ++v) {
    ff_add(a, m[v]);
    ff_add_prod(b, sj[v], m[v]);
  }
  for (int o = seg >> 1; o > 0; o >>= 1) {
    FF ao{__shfl_xor_sync(0xffffffffu, a.hi, o, seg), __shfl_xor_sync(0xffffffffu, a.lo, o, seg)};
    FF bo{__shfl_xor_sync(0xffffffffu, b.hi, o, seg), __shfl_xor_sync(0xffffffffu, b.lo, o, seg)};
    ff_merge(a, ao);
    ff_merge(b, bo);
  }
}

// Sums over the warp of 16 values per lane by reduce-scatter (16 float64
// additions instead of 16 x 5): at each step a lane keeps half of its values
// and adds its partner's copies of them. Returns the total of value
// f(lane) = 8 b4 + 4 b3 + 2 b2 + b1 (b_i the bits of the lane index), which
// lanes 2 f and 2 f + 1 both hold.
__device__ __forceinline__ double warp_sum16_scatter(double (&v)[16], int lane) {
#pragma unroll
  for (int step = 0; step < 4; ++step) {
    const int o = 16 >> step, half = 8 >> step;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double keep = up ? v[half + i] : v[i];
      const double give = up ? v[i] : v[half + i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
// The same reduce-scatter in float-float.
__device__ __forceinline__ FF warp_sum16_scatter_ff(FF (&v)[16], int lane) {
#pragma unroll
  for (int step = 0; step < 4; ++step) {
    const int o = 16 >> step, half = 8 >> step;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const FF keep = up ? v[half + i] : v[i];
      const FF give = up ? v[i] : v[half + i];
      const FF got{__shfl_xor_sync(0xffffffffu, give.hi, o), __shfl_xor_sync(0xffffffffu, give.lo, o)};
      v[i] = ff_sum(keep, got);
    }
  }
  const FF got{__shfl_xor_sync(0xffffffffu, v[0].hi, 1), __shfl_xor_sync(0xffffffffu, v[0].lo, 1)};
  return ff_sum(v[0], got);
}
__device__ __forceinline__ int scatter_field(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

constexpr int kMomPasses = 4;

template <typename T, int V>
struct alignas(sizeof(T) * V) VPack {
  T v[V];
};

// Moments, one warp per cell, no block barriers before the final sums. The s-rows of the cell are
// read with the substep kernel's lane mapping (a row over `seg` lanes, V
// consecutive nodes per lane, vector loads) and reduced to n_b and m1: in
// float64 in the float64 form, compensated float32 (float-float) converted to
// float64 per row in the float32 form -- these are the s-reductions feeding
// the force and the force dipole. Then lanes over theta form the 12 fields.
// Each warp keeps partial global sums, added per block at the end; the last
// block to finish adds the block partials in a fixed order.
template <typename T, int V>
__global__ void k_moments(const T* psi, const T* mb, const T* mf, const T* c,
                          const double* trig, long long ncells, int nth, int ns, int seg,
                          double dth, double ds, double L, double dA, float hds, double* fields,
                          double* partial, DevParams* prm) {
  extern __shared__ double msm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* s_nb = msm + (size_t)wib * 2 * nth;
  double* s_m1 = s_nb + nth;
  // float32 form: the rows' float-float sums, converted once per row below
  float4* s_ff = reinterpret_cast<float4*>(msm + (size_t)(blockDim.x >> 5) * 2 * nth) +
                 (size_t)wib * nth;
  const long long gw = blockIdx.x * (long long)(blockDim.x >> 5) + wib;
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  const double g = prm->psi_scale;
  const double Fm = prm->force_scale, ell = prm->ell;
  const int sl = lane & (seg - 1), rslot = lane / seg, rpp = 32 / seg;
  const int nl = ns / V;
  const bool lane_ok = sl < nl;
  T sj[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    // s_j = (2j + 1 - ns) ds / 2; the float32 form in float32 (one rounding)
    if constexpr (sizeof(T) == 4)
      sj[v] = (float)(2 * (sl * V + v) + 1 - ns) * hds;
    else
      sj[v] = -0.5 * L + ((double)(sl * V + v) + 0.5) * ds;
  }
  // global accumulators: N_psi, bound, free, sum psi cos, sum psi sin, sum psi, sum tr
  double gs[7] = {0, 0, 0, 0, 0, 0, 0};
  const int fq = scatter_field(lane);
  // float32 form: every float64 warp instruction costs the float64 pipe as
  // much as a full warp's, so the per-cell bookkeeping stays in float-float:
  // acc is the lane's field total summed over its cells, acc2 (lanes 1, 3) the
  // sum of C and of Mf; each field total is scaled by its constant (psi_scale,
  // ds F, ds F ell) split into a float pair
  FF acc{0.f, 0.f}, acc2{0.f, 0.f};
  FF scf{0.f, 0.f};
  if constexpr (sizeof(T) == 4) {
    const double sc = fq < 5 ? g : (fq < 7 ? g * (ds * Fm) : g * (ds * Fm * ell));
    scf.hi = (float)sc;
    scf.lo = (float)(sc - (double)scf.hi);
  }
  for (long long cell = gw; cell < ncells; cell += W) {
    // kMomPasses passes of rows loaded before they are reduced (more bytes in
    // flight per warp)
    for (int r0 = 0; r0 < nth; r0 += kMomPasses * rpp) {
      T m[kMomPasses][V];
#pragma unroll
      for (int u = 0; u < kMomPasses; ++u) {
        const int k = r0 + u * rpp + rslot;
        if (k < nth && lane_ok) {
          const VPack<T, V> q =
              *reinterpret_cast<const VPack<T, V>*>(mb + ((size_t)cell * nth + k) * ns + sl * V);
#pragma unroll
          for (int v = 0; v < V; ++v) m[u][v] = q.v[v];
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) m[u][v] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < kMomPasses; ++u) {
        const int k = r0 + u * rpp + rslot;
        if constexpr (sizeof(T) == 4) {
          FF a, b;
          row_sums_ff<V>(m[u], sj, seg, a, b);
          if (sl == 0 && k < nth) s_ff[k] = make_float4(a.hi, a.lo, b.hi, b.lo);
        } else {
          double nbk, m1k;
          row_sums<V>(m[u], sj, seg, nbk, m1k);
          if (sl == 0 && k < nth) {
            s_nb[k] = nbk * ds;
            s_m1[k] = m1k * ds;
          }
        }
      }
    }
    __syncwarp();
    // ten field sums over theta (weights w[q][k] built on the host: dth,
    // cos dth, sin dth, (cos^2 - 1/2) dth, cos sin dth, cos, sin, cos^2 dth,
    // cos sin dth, sin^2 dth); slots 10..15 stay zero. Lane pair (2q, 2q + 1)
    // gets the total of field q.
    if constexpr (sizeof(T) == 4) {
      // Float32 form: the sums in float-float on the float32 pipe (each product
      // exact to about 2^-48 of itself, the weights split into float pairs on
      // the host); psi_scale and the constant factors ds F, ds F ell multiply
      // each total once, in float64.
      const float2* wf = reinterpret_cast<const float2*>(trig + 14 * (size_t)nth);
      FF f[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) f[q] = FF{0.f, 0.f};
      for (int k = lane; k < nth; k += 32) {
        const float4 q4 = s_ff[k];
        const float p = (float)psi[cell * nth + k];
        const FF pn = ff_scale(p, FF{q4.x, q4.y}), pm = ff_scale(p, FF{q4.z, q4.w});
        FF wq[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) {
          const float2 t = wf[(size_t)q * nth + k];
          wq[q] = FF{t.x, t.y};
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) f[q] = ff_sum(f[q], ff_scale(p, wq[q]));
        f[5] = ff_sum(f[5], ff_prod(pn, wq[1]));
        f[6] = ff_sum(f[6], ff_prod(pn, wq[2]));
#pragma unroll
        for (int q = 7; q < 10; ++q) f[q] = ff_sum(f[q], ff_prod(pm, wq[q]));
      }
      __syncwarp();
      const FF t = warp_sum16_scatter_ff(f, lane);
      acc = ff_sum(acc, t);
      const FF ts = ff_prod(t, scf);
      const double tot = (double)ts.hi + (double)ts.lo;
      if ((lane & 1) == 0 && fq < 10) fields[(size_t)(fq < 5 ? fq : fq + 2) * ncells + cell] = tot;
      // C and Mf as they are (lanes 1 and 3: one conversion for both)
      if (lane == 1 || lane == 3) {
        const float v = lane == 1 ? (float)c[cell] : (float)mf[cell];
        fields[(size_t)(lane == 1 ? 5 : 6) * ncells + cell] = (double)v;
        ff_add(acc2, v);
      }
    } else {
      double f[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      const double* w = trig + 4 * (size_t)nth;
      for (int k = lane; k < nth; k += 32) {
        const double nbk = s_nb[k], m1k = s_m1[k];
        const double p = (double)psi[cell * nth + k] * g;
        const double pn = p * nbk * Fm, pm = p * m1k * (Fm * ell);
        f[0] = fma(p, w[k], f[0]);
        f[1] = fma(p, w[nth + k], f[1]);
        f[2] = fma(p, w[2 * nth + k], f[2]);
        f[3] = fma(p, w[3 * nth + k], f[3]);
        f[4] = fma(p, w[4 * nth + k], f[4]);
        f[5] = fma(pn, w[nth + k], f[5]);
        f[6] = fma(pn, w[2 * nth + k], f[6]);
        f[7] = fma(pm, w[7 * nth + k], f[7]);
        f[8] = fma(pm, w[8 * nth + k], f[8]);
        f[9] = fma(pm, w[9 * nth + k], f[9]);
        gs[3] = fma(p, w[5 * nth + k], gs[3]);
        gs[4] = fma(p, w[6 * nth + k], gs[4]);
        gs[5] += p;
      }
      __syncwarp();
      const double tot = warp_sum16_scatter(f, lane);
      // output slot of field q: 0-4 as is, 5-9 to 7-11 (5 and 6 are C and Mf)
      if ((lane & 1) == 0 && fq < 10) fields[(size_t)(fq < 5 ? fq : fq + 2) * ncells + cell] = tot;
      const double f0 = __shfl_sync(0xffffffffu, tot, 0);   // field 0 (lane 0)
      const double f7 = __shfl_sync(0xffffffffu, tot, 14);  // field 7: bits 3, 2, 1 set
      if (lane == 0) {
        const double cc = (double)c[cell], ff = (double)mf[cell];
        fields[5 * ncells + cell] = cc;
        fields[6 * ncells + cell] = ff;
        gs[0] += f0 * dA;
        gs[1] += cc * dA;
        gs[2] += ff * dA;
      }
      // tr sigma_a = f7 + f9
      const double f9 = __shfl_sync(0xffffffffu, tot, 18);  // field 9: bits 4, 1 set
      if (lane == 0) gs[6] += f7 + f9;
    }
  }
  __shared__ double s_g[32 * 8];
  __shared__ unsigned int s_last;
  const int nw = (int)(blockDim.x >> 5);
  if constexpr (sizeof(T) == 4) {
    // The warp's quantities in float-float, lane q holding quantity q:
    // 0 N_psi (field 0), 1 C, 2 Mf, 3 sum psi cos (field 1), 4 sum psi sin
    // (field 2), 5 sum psi (field 0), 6 tr sigma_a (fields 7 + 9); unscaled.
    const int sa = lane == 3 ? 2 : lane == 4 ? 4 : lane == 6 ? 14 : 0;
    const int sb = lane == 2 ? 3 : 1;
    FF v{__shfl_sync(0xffffffffu, acc.hi, sa), __shfl_sync(0xffffffffu, acc.lo, sa)};
    const FF w2{__shfl_sync(0xffffffffu, acc2.hi, sb), __shfl_sync(0xffffffffu, acc2.lo, sb)};
    const FF a9{__shfl_sync(0xffffffffu, acc.hi, 18), __shfl_sync(0xffffffffu, acc.lo, 18)};
    if (lane == 1 || lane == 2) v = w2;
    if (lane == 6) v = ff_sum(v, a9);
    // per block in warp order, then the last block adds the block partials
    // (float pairs in the 8-byte slots) in a fixed order
    float2* s_ff2 = reinterpret_cast<float2*>(s_g);
    if (lane < 7) s_ff2[wib * 8 + lane] = make_float2(v.hi, v.lo);
    __syncthreads();
    float2* pf = reinterpret_cast<float2*>(partial);
    if (wib == 0 && lane < 7) {
      FF b{s_ff2[lane].x, s_ff2[lane].y};
      for (int w2i = 1; w2i < nw; ++w2i) b = ff_sum(b, FF{s_ff2[w2i * 8 + lane].x, s_ff2[w2i * 8 + lane].y});
      pf[(size_t)blockIdx.x * 8 + lane] = make_float2(b.hi, b.lo);
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int prev = atomicInc(&prm->counter2, gridDim.x - 1);
      s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // scales: psi_scale dA, dA, dA, psi_scale / dth (x3), psi_scale ds F ell
    for (int q = wib; q < 7; q += nw) {
      FF b{0.f, 0.f};
      for (int i = lane; i < (int)gridDim.x; i += 32) {
        const float2 t = __ldcg(pf + (size_t)i * 8 + q);
        b = ff_sum(b, FF{t.x, t.y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        b = ff_sum(b, FF{__shfl_xor_sync(0xffffffffu, b.hi, o), __shfl_xor_sync(0xffffffffu, b.lo, o)});
      if (lane == 0) {
        const double sq = q == 0 ? g * dA : q < 3 ? dA : q < 6 ? g / dth : g * (ds * Fm * ell);
        s_g[8 * 8 + q] = ((double)b.hi + (double)b.lo) * sq;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t[7];
      for (int q = 0; q < 7; ++q) t[q] = s_g[8 * 8 + q];
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
  } else {
#pragma unroll
    for (int q = 0; q < 7; ++q) gs[q] = warp_sum(gs[q]);
    // per block in warp order, then the last block adds the block partials in a
    // fixed order (warp q of that block sums quantities q, q + nw, ...)
    if (lane == 0)
      for (int q = 0; q < 7; ++q) s_g[wib * 8 + q] = gs[q];
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 0; q < 7; ++q) {
        double b = s_g[q];
        for (int w2 = 1; w2 < nw; ++w2) b += s_g[w2 * 8 + q];
        partial[(size_t)blockIdx.x * 8 + q] = b;
      }
      __threadfence();
      const unsigned int prev = atomicInc(&prm->counter2, gridDim.x - 1);
      s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      for (int q = wib; q < 7; q += nw) {
        const double tq = warp_sum_ldcg(partial + q, (int)gridDim.x, 8, lane);
        if (lane == 0) s_g[q] = tq;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double t[7];
        for (int q = 0; q < 7; ++q) t[q] = s_g[q];
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
}

// The adaptive-substep rule, evaluated on the device in float64 from the
// maxima of k_dt_max: dt = cfl / max(v/ds, adv, rot, k_off + k_on L rho_max).
// A non-finite or non-positive rate leaves dt unchanged and sets status bit 1.
__global__ void k_dt_finalize(DevParams* prm, double ds, double L, double cfl) {
  const double rate = fmax(fmax(prm->v_walk / ds, prm->dtmax[0]),
                           fmax(prm->dtmax[1], prm->k_off + prm->k_on * L * prm->dtmax[2]));
  if (rate > 0.0 && isfinite(rate))
    prm->dt = cfl / rate;
  else
    atomicOr(&prm->status, 2);
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

cudaError_t launch_copy_multi(const CopySegs& c, cudaStream_t s) {
  size_t most = 0;
  for (int q = 0; q < c.n; ++q) most = c.bytes[q] > most ? c.bytes[q] : most;
  if (most == 0) return cudaSuccess;
  k_copy_multi<<<grid_for((long long)((most + 15) / 16), 256), 256, 0, s>>>(c);
  return cudaGetLastError();
}

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
cudaError_t launch_init_cells(T* mb, const T* psi, T* nb, T* mf, T* c, const T* mtot,
                              long long ncells, int nth, int ns, double ds, double dth,
                              cudaStream_t s) {
  int block = nth >= 128 ? 128 : (nth >= 64 ? 64 : 32);
  long long g = ncells < 152 * 16 ? ncells : 152 * 16;
  k_init_cells<T><<<(int)g, block, 0, s>>>(mb, psi, nb, mf, c, mtot, ncells, nth, ns, ds, dth);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dt_max(const T* psi, const T* nb, const T* u, const T* trig, long long ncells,
                          int nx, int ny, int nth, double inv_dx, double inv_dy, double inv_dth,
                          double dth, double glide, double vsp, DevParams* prm, cudaStream_t s) {
  long long g = (ncells + 3) / 4;  // warp per cell, 4 warps per block
  if (g > 152 * 8) g = 152 * 8;
  k_dt_max<T><<<(int)g, 128, 0, s>>>(psi, nb, u, trig, ncells, nx, ny, nth, inv_dx, inv_dy,
                                     inv_dth, dth, glide, vsp, prm);
  return cudaGetLastError();
}

cudaError_t launch_dt_finalize(DevParams* prm, double ds, double L, double cfl, cudaStream_t s) {
  k_dt_finalize<<<1, 1, 0, s>>>(prm, ds, L, cfl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(const T* psi, const T* mb, const T* mf, const T* c,
                           const double* trig, long long ncells, int nth, int ns, int V, int seg,
                           double dth, double ds, double L, double dA, double* fields,
                           double* partial, int nblocks, DevParams* prm, cudaStream_t s) {
  // nblocks blocks of 4 warps; the partial buffer holds 8 doubles per warp
  const int block = 128;
  // per warp: n_b and m1 of the rows (float64), and their float-float sums
  const size_t smem = (size_t)4 * 2 * nth * sizeof(double) + (size_t)4 * nth * 16;
  auto go = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = mm::raise_smem_limit(kern, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<nblocks, block, smem, s>>>(psi, mb, mf, c, trig, ncells, nth, ns, seg, dth, ds, L, dA,
                                      (float)(0.5 * ds), fields, partial, prm);
    return cudaGetLastError();
  };
  if constexpr (sizeof(T) == 4)
    if (V == 8) return go(k_moments<T, 8>);
  if (V == 4) return go(k_moments<T, 4>);
  if (V == 2) return go(k_moments<T, 2>);
  return go(k_moments<T, 1>);
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
template cudaError_t launch_init_cells<float>(float*, const float*, float*, float*, float*,
                                              const float*, long long, int, int, double, double,
                                              cudaStream_t);
template cudaError_t launch_init_cells<double>(double*, const double*, double*, double*, double*,
                                               const double*, long long, int, int, double, double,
                                               cudaStream_t);
template cudaError_t launch_dt_max<float>(const float*, const float*, const float*, const float*,
                                          long long, int, int, int, double, double, double,
                                          double, double, double, DevParams*, cudaStream_t);
template cudaError_t launch_dt_max<double>(const double*, const double*, const double*,
                                           const double*, long long, int, int, int, double, double,
                                           double, double, double, double, DevParams*, cudaStream_t);
template cudaError_t launch_moments<float>(const float*, const float*, const float*,
                                           const float*, const double*, long long, int, int, int,
                                           int, double, double, double, double, double*, double*,
                                           int, DevParams*, cudaStream_t);
template cudaError_t launch_moments<double>(const double*, const double*, const double*,
                                            const double*, const double*, long long, int, int,
                                            int, int, double, double, double, double, double*,
                                            double*, int, DevParams*, cudaStream_t);

}  // namespace mm
