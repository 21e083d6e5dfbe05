// Tangent-linear (forward-mode) derivative of the substep along a direction
// of the rates (d k_off, d v_walk, d k_on), carried alongside the state
// (mm_set_tangent): every substep advances the state and its tangent
// (dpsi, dMb, dMf, dn_b) together, in one launch, so the derivative of an
// observable with respect to one scalar parameter costs one pass of about
// twice the forward's memory traffic and needs no checkpoints -- the reverse
// sweep (mm_adjoint_step) is the tool for many parameters at once (the
// velocity field, the initial psi).
//
// The map differentiated is the discrete substep exactly as the forward
// computes it, at a fixed dt, on the branches the forward takes (donor-cell
// upwinding, the Superbee limiter, the Alg. 2 scale-down), the float32 form's
// mass-correction factor a constant of the map: the same readings as the
// reverse sweep and the oracle's tangent substep. The forward part of the
// kernel is the plain substep's device code (psi_cell, walk_dflux), so the
// state advances as in the plain path up to the rounding of the row loads.
#include <algorithm>

#include "mm_cell.cuh"
#include "mm_host.h"

namespace mm {

template <typename T>
struct TanArgs {
  StepArgs<T> a;
  const T* dpsi_in;
  T* dpsi_out;
  const T* dnb_in;
  T* dnb_out;
  T* dmb;       // [cells][nth][ns] in place
  T* dmf;       // [cells] in place
  double dkoff, dvw, dkon;
};

// Per-warp shared memory of the tangent substep: psi, n_b, dpsi, dn_b of the
// cell and its four neighbours ([5][nth] each), the new psi and dpsi of the
// cell, and the new rows' n_b and dn_b.
__host__ __device__ inline size_t tan_warp_smem(int nth, int tsz) {
  return (size_t)24 * nth * tsz;
}

// d of the donor-cell flux max(A, 0) pl + min(A, 0) pr on the branch taken
// (the right state when A = 0).
template <typename T>
__device__ __forceinline__ T donor_tl(T A, T pl, T pr, T dA, T dpl, T dpr) {
  return fma_t(tmax(A, T(0)), dpl, tmin(A, T(0)) * dpr) + dA * (A > T(0) ? pl : pr);
}

// dpsi^{n+1} of the cell (lanes over theta), with no velocity perturbation:
// the face velocities change through dn_b (the gliding speed), the fluxes
// through them and through dpsi.
template <typename T>
__device__ __forceinline__ void psi_cell_tl(const PsiConst<T>& q, const CellVel<T>& u,
                                            const T* psi5, const T* nb5, const T* dpsi5,
                                            const T* dnb5, int nth, int lane, T* dpsi_new) {
  const T* cosk = q.trig;
  const T* sink = q.trig + nth;
  const T* cosf = q.trig + 2 * nth;
  const T* sinf = q.trig + 3 * nth;
  const T g = q.g;
  for (int k = lane; k < nth; k += 32) {
    const T Pc = g * psi5[k], Pe = g * psi5[nth + k], Pw = g * psi5[2 * nth + k];
    const T Pn = g * psi5[3 * nth + k], Ps = g * psi5[4 * nth + k];
    const T dPc = g * dpsi5[k], dPe = g * dpsi5[nth + k], dPw = g * dpsi5[2 * nth + k];
    const T dPn = g * dpsi5[3 * nth + k], dPs = g * dpsi5[4 * nth + k];
    const T ck = cosk[k], sk = sink[k];
    const T Vc = fma_t(q.glide, nb5[k], q.vsp), Ve = fma_t(q.glide, nb5[nth + k], q.vsp);
    const T Vw = fma_t(q.glide, nb5[2 * nth + k], q.vsp);
    const T Vn = fma_t(q.glide, nb5[3 * nth + k], q.vsp);
    const T Vs = fma_t(q.glide, nb5[4 * nth + k], q.vsp);
    const T axc = fma_t(-Vc, ck, u.uxc), axe = fma_t(-Ve, ck, u.uxe), axw = fma_t(-Vw, ck, u.uxw);
    const T ayc = fma_t(-Vc, sk, u.uyc), ayn = fma_t(-Vn, sk, u.uyn), ays = fma_t(-Vs, sk, u.uys);
    const T Ae = T(0.5) * (axc + axe), Aw = T(0.5) * (axw + axc);
    const T An = T(0.5) * (ayc + ayn), As = T(0.5) * (ays + ayc);
    // d(u - (v_sp + glide n_b) p) = -glide dn_b p
    const T gc = -q.glide * ck, gs = -q.glide * sk;
    const T daxc = gc * dnb5[k], daxe = gc * dnb5[nth + k], daxw = gc * dnb5[2 * nth + k];
    const T dayc = gs * dnb5[k], dayn = gs * dnb5[3 * nth + k], days = gs * dnb5[4 * nth + k];
    const T dAe = T(0.5) * (daxc + daxe), dAw = T(0.5) * (daxw + daxc);
    const T dAn = T(0.5) * (dayc + dayn), dAs = T(0.5) * (days + dayc);
    const int kp = k + 1 == nth ? 0 : k + 1, km = k == 0 ? nth - 1 : k - 1;
    const T cp = cosf[k], sp = sinf[k], cm = cosf[km], sm = sinf[km];
    // (the forward substep's fused form: the same upwind sides)
    const T wp = fma_t(-sp, fma_t(u.Gxx, cp, u.Gxy * sp), cp * fma_t(u.Gyx, cp, u.Gyy * sp));
    const T wm = fma_t(-sm, fma_t(u.Gxx, cm, u.Gxy * sm), cm * fma_t(u.Gyx, cm, u.Gyy * sm));
    const T dFe = donor_tl(Ae, Pc, Pe, dAe, dPc, dPe), dFw = donor_tl(Aw, Pw, Pc, dAw, dPw, dPc);
    const T dFn = donor_tl(An, Pc, Pn, dAn, dPc, dPn), dFs = donor_tl(As, Ps, Pc, dAs, dPs, dPc);
    const T dFp = donor_tl(wp, Pc, g * psi5[kp], T(0), dPc, g * dpsi5[kp]);
    const T dFm = donor_tl(wm, g * psi5[km], Pc, T(0), g * dpsi5[km], dPc);
    dpsi_new[k] =
        dPc - q.dt * ((dFe - dFw) * q.inv_dx + (dFn - dFs) * q.inv_dy + (dFp - dFm) * q.inv_dth);
  }
}

// The walking term and its tangent on a lane's V nodes: D as walk_dflux, and
// dD = dF_{j-1} - dF_j with dF = dM + ga da + gb db on the Superbee branch
// the forward takes (ga, gb from walk_dflux).
//
// The branch is chosen with the comparisons of walk_dflux<..., true> and its
// term taken at once: sigma/2 is one of a, b/2, a/2, b or 0, so its
// derivative is the same one of da, db/2, da/2, db or 0 (each exact), and
// dF = dM + that term rounds once, as dM + ga da + gb db does.
template <typename T, int V>
__device__ __forceinline__ void walk_tl(const T (&M)[V], const T (&dM)[V], T (&D)[V], T (&dD)[V],
                                        bool first, bool last, int seg) {
  T ml = __shfl_up_sync(0xffffffffu, M[V - 1], 1, seg);
  const T mr = __shfl_down_sync(0xffffffffu, M[0], 1, seg);
  T dml = __shfl_up_sync(0xffffffffu, dM[V - 1], 1, seg);
  const T dmr = __shfl_down_sync(0xffffffffu, dM[0], 1, seg);
  if (first) {
    ml = T(0);
    dml = T(0);
  }
  // d[i] = M_i - M_{i-1} and dd[i] = dM_i - dM_{i-1}, i = 0..V
  T d[V + 1], hd[V + 1], dd[V + 1];
  d[0] = M[0] - ml;
  dd[0] = dM[0] - dml;
#pragma unroll
  for (int v = 1; v < V; ++v) {
    d[v] = M[v] - M[v - 1];
    dd[v] = dM[v] - dM[v - 1];
  }
  d[V] = mr - M[V - 1];
  dd[V] = dmr - dM[V - 1];
#pragma unroll
  for (int i = 0; i <= V; ++i) hd[i] = T(0.5) * d[i];
  T F[V], dF[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    bool pos, p1, x1a, x2a;
    if constexpr (sizeof(T) == 8) {
      // the flux and decisions of walk_dflux<double, V, true> (bit patterns)
      const Lim64 q = superbee64(d[v], hd[v], d[v + 1], hd[v + 1], v == V - 1 && last, M[v]);
      F[v] = q.F;
      pos = q.pos;
      p1 = q.p1;
      x1a = q.x1a;
      x2a = q.x2a;
    } else {
      T sgn = copysign(T(1), d[v + 1]);
      if (v == V - 1 && last) sgn = T(0);  // plus end: F = M, no slope
      const T A = d[v] * sgn, hA = hd[v] * sgn;
      const T hB = fabs(hd[v + 1]), B = fabs(d[v + 1]);
      const T t1 = tmin(A, hB), t2 = tmin(hA, B);
      const T r = max3_t(t1, t2, T(0));
      F[v] = fma_t(r, sgn, M[v]);
      pos = r > T(0);
      p1 = t1 > t2;
      x1a = A < hB;
      x2a = hA < B;
    }
    const T e1 = x1a ? dd[v] : T(0.5) * dd[v + 1];   // t1 = a (sigma/2 = a) or |b|/2
    const T e2 = x2a ? T(0.5) * dd[v] : dd[v + 1];   // t2 = a/2 or |b|
    const T g = pos ? (p1 ? e1 : e2) : T(0);
    dF[v] = dM[v] + g;
  }
  T fl = __shfl_up_sync(0xffffffffu, F[V - 1], 1, seg);
  T dfl = __shfl_up_sync(0xffffffffu, dF[V - 1], 1, seg);
  if (first) {
    fl = T(0);
    dfl = T(0);
  }
  D[0] = fl - F[0];
  dD[0] = dfl - dF[0];
#pragma unroll
  for (int v = 1; v < V; ++v) {
    D[v] = F[v - 1] - F[v];
    dD[v] = dF[v - 1] - dF[v];
  }
}

// One substep of the state and its tangent (warp per cell, persistent grid).
// Per cell: psi^{n+1} by Eq. 1 (the plain substep's code) and dpsi^{n+1};
// every s-row by the RK2 of Eq. 4 and its tangent,
//   dR = (v/ds) dD + (dv/ds) D - k_off dM - dk_off M + k_on dMf + dk_on Mf,
// n_b and dn_b of the new rows; C = sum psi n_b dtheta and dC; where the
// scale-down acts, Mb' = f Mb and dMb' = f dMb + df Mb with df = -f dC / C
// (then C = M, dMf = 0), else dMf = -dC. Rows are read with plain vector
// loads, the next pass's rows while the current one is computed.
template <typename T, int V, bool MASSCORR>
__global__ void __launch_bounds__(128) k_substep_tl(const TanArgs<T> t) {
  extern __shared__ __align__(16) unsigned char tl_smem[];
  const StepArgs<T>& a = t.a;
  const int nth = a.nth, ns = a.ns, seg = a.seg, nx = a.nx, ny = a.ny;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* psi5 = reinterpret_cast<T*>(tl_smem + (size_t)wib * tan_warp_smem(nth, sizeof(T)));
  T* nb5 = psi5 + 5 * nth;
  T* dpsi5 = nb5 + 5 * nth;
  T* dnb5 = dpsi5 + 5 * nth;
  T* pnew = dnb5 + 5 * nth;
  T* dpnew = pnew + nth;
  T* s_nb = dpnew + nth;
  T* s_dnb = s_nb + nth;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  const StepScalars<T> sc = step_scalars<T, MASSCORR>(a.prm, a, lane);
  const PsiConst<T> pq{sc.dt, sc.g, sc.glide, sc.vsp, sc.inv_dx, sc.inv_dy, sc.inv_dth, sc.dth,
                       a.trig};
  const T dkoff = (T)t.dkoff, dkon = (T)t.dkon, dcw = (T)(t.dvw / a.ds);
  const T hdt = sc.hdt, dt = sc.dt;
  const LaneGeom lg = lane_geom(lane, seg, ns, V);
  const LaneTrig<T> lt = lane_trig(a.trig, nth, lane);
  T mass_hi = T(0), mass_lo = T(0);
  for (int cell = gw; cell < nc; cell += W) {
    const int iy = cell / nx, ix = cell - iy * nx;
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const int nbr[5] = {cell, iy * nx + xp, iy * nx + xm, yp * nx + ix, ym * nx + ix};
    for (int q = 0; q < 5; ++q)
      for (int k = lane; k < nth; k += 32) {
        const size_t o = (size_t)nbr[q] * nth + k;
        psi5[q * nth + k] = a.psi_in[o];
        nb5[q * nth + k] = a.nb_in[o];
        dpsi5[q * nth + k] = t.dpsi_in[o];
        dnb5[q * nth + k] = t.dnb_in[o];
      }
    __syncwarp();
    const CellVel<T> uv = load_cell_vel(a.ucell, cell);
    T cell_mass = T(0), unused = T(0);
    psi_cell(pq, uv, psi5, nb5, nb5, nth, lane, pnew, cell_mass, unused, &lt);
    psi_cell_tl(pq, uv, psi5, nb5, dpsi5, dnb5, nth, lane, dpnew);
    two_sum_acc(mass_hi, mass_lo, cell_mass);
    __syncwarp();
    for (int k = lane; k < nth; k += 32) {
      a.psi_out[(size_t)cell * nth + k] = pnew[k];
      t.dpsi_out[(size_t)cell * nth + k] = dpnew[k];
    }
    const T mf = a.mf_in[cell], dmf = t.dmf[cell];
    // the rows: Mf frozen over both stages
    const T c3 = sc.hdt * sc.kon * mf, e3 = dt * sc.kon * mf;
    const T dsrc = fma_t(sc.kon, dmf, dkon * mf);  // d(k_on Mf)
    Pack<T, V> qn, dqn;
    auto load_pass = [&](int r0) {
      const int k = r0 + lg.rslot;
      if (k < nth && lg.lane_ok) {
        const size_t off = ((size_t)cell * nth + k) * ns + lg.sl * V;
        qn = *reinterpret_cast<const Pack<T, V>*>(a.mb_in + off);
        dqn = *reinterpret_cast<const Pack<T, V>*>(t.dmb + off);
      }
    };
    load_pass(0);
    for (int r0 = 0; r0 < nth; r0 += lg.rpp) {
      const int k = r0 + lg.rslot;
      const bool row_ok = k < nth, act = row_ok && lg.lane_ok;
      const size_t roff = ((size_t)cell * nth + (row_ok ? k : 0)) * ns + lg.sl * V;
      T M[V], dM[V], D[V], dD[V], Ms[V], dMs[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        M[v] = act ? qn.v[v] : T(0);
        dM[v] = act ? dqn.v[v] : T(0);
      }
      if (r0 + lg.rpp < nth) load_pass(r0 + lg.rpp);
      // half stage: Ms = M + dt/2 R(M), dMs = dM + dt/2 dR(M, dM)
      walk_tl<T, V>(M, dM, D, dD, lg.first, lg.last, seg);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        Ms[v] = fma_t(hdt * sc.cw, D[v], fma_t(T(1) - hdt * sc.koff, M[v], c3));
        const T dR = fma_t(sc.cw, dD[v], fma_t(dcw, D[v], fma_t(-sc.koff, dM[v],
                                                                 fma_t(-dkoff, M[v], dsrc))));
        dMs[v] = fma_t(hdt, dR, dM[v]);
      }
      // full stage from M with R(Ms)
      walk_tl<T, V>(Ms, dMs, D, dD, lg.first, lg.last, seg);
      T snb = T(0), sdnb = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T dR = fma_t(sc.cw, dD[v], fma_t(dcw, D[v], fma_t(-sc.koff, dMs[v],
                                                                 fma_t(-dkoff, Ms[v], dsrc))));
        M[v] = fma_t(dt * sc.cw, D[v], fma_t(-dt * sc.koff, Ms[v], M[v] + e3));
        dM[v] = fma_t(dt, dR, dM[v]);
        snb += M[v];
        sdnb += dM[v];
      }
      if (act) {
        Pack<T, V> q, dq;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          q.v[v] = M[v];
          dq.v[v] = dM[v];
        }
        *reinterpret_cast<Pack<T, V>*>(a.mb_out + roff) = q;
        *reinterpret_cast<Pack<T, V>*>(t.dmb + roff) = dq;
      } else {
        snb = T(0);
        sdnb = T(0);
      }
      snb = seg_sum(snb, seg);
      sdnb = seg_sum(sdnb, seg);
      if (lg.first && row_ok) {
        s_nb[k] = snb * sc.ds;
        s_dnb[k] = sdnb * sc.ds;
      }
    }
    __syncwarp();
    // Eq. 5, the scale-down of Alg. 2, Eq. 6 and their tangents
    T acc = T(0), dacc = T(0);
    for (int k = lane; k < nth; k += 32) {
      acc = fma_t(pnew[k] * s_nb[k], sc.dth, acc);
      dacc = fma_t(fma_t(dpnew[k], s_nb[k], pnew[k] * s_dnb[k]), sc.dth, dacc);
    }
    const T Cpre = warp_sum_t(acc), dC = warp_sum_t(dacc);
    const T mtot = a.mtot[cell];
    const size_t cb = (size_t)cell * nth;
    if (mtot < Cpre) {
      const T f = mtot / Cpre, df = -f * dC / Cpre;
      T* base = a.mb_out + cb * ns;
      T* dbase = t.dmb + cb * ns;
      for (int e = lane; e < nth * ns; e += 32) {
        const T m = __ldcg(base + e);
        dbase[e] = fma_t(f, __ldcg(dbase + e), df * m);
        base[e] = m * f;
      }
      for (int k = lane; k < nth; k += 32) {
        a.nb_out[cb + k] = s_nb[k] * f;
        t.dnb_out[cb + k] = fma_t(f, s_dnb[k], df * s_nb[k]);
      }
      if (lane == 0) {
        a.c[cell] = mtot;
        a.mf_out[cell] = T(0);
        t.dmf[cell] = T(0);
      }
    } else {
      for (int k = lane; k < nth; k += 32) {
        a.nb_out[cb + k] = s_nb[k];
        t.dnb_out[cb + k] = s_dnb[k];
      }
      if (lane == 0) {
        a.c[cell] = Cpre;
        a.mf_out[cell] = mtot - Cpre;
        t.dmf[cell] = -dC;
      }
    }
    __syncwarp();
  }
  // sum psi^{n+1} (fixed order) and the float32 form's correction factor, as
  // in the plain substep
  __shared__ double s_red[32];
  __shared__ unsigned int s_last;
  const double m = warp_sum_ff(mass_hi, mass_lo);
  if (lane == 0) s_red[wib] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = s_red[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) b += s_red[q];
    a.partial[blockIdx.x] = b;
    __threadfence();
    const unsigned int prev = atomicInc(&a.prm->counter, gridDim.x - 1);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && wib == 0) {
    __threadfence();
    const double tot = warp_sum_ldcg(a.partial, (int)gridDim.x, 1, lane);
    if (lane == 0) {
      a.prm->mass = tot;
      if (MASSCORR && a.mass_correct) a.prm->psi_scale = a.prm->mass0 / tot;
    }
  }
}

// Per cell, the sums an observable and its tangent need (float64): sum psi cos,
// sum psi sin, sum psi, sum psi m1, and the same of the tangent (psi taken
// with the pending correction factor g, dpsi with g as a constant), into
// out[cell][8] (warp per cell, lanes over theta).
template <typename T>
__global__ void k_tan_cells(const T* psi, const T* mb, const T* dpsi, const T* dmb,
                            const double* trig64, const DevParams* prm, long long ncells, int nth,
                            int ns, double ds, double L, double* out) {
  const int lane = threadIdx.x & 31;
  const double g = prm->psi_scale;
  for (long long cell = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
       cell < ncells; cell += (long long)gridDim.x * (blockDim.x >> 5)) {
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = lane; k < nth; k += 32) {
      const size_t r = (size_t)cell * nth + k;
      const double p = g * (double)psi[r], dp = g * (double)dpsi[r];
      double m1 = 0.0, dm1 = 0.0;
      for (int j = 0; j < ns; ++j) {
        const double sj = -0.5 * L + (j + 0.5) * ds;
        m1 += sj * (double)mb[r * ns + j] * ds;
        dm1 += sj * (double)dmb[r * ns + j] * ds;
      }
      const double ck = trig64[k], sk = trig64[nth + k];
      s[0] += p * ck;
      s[1] += p * sk;
      s[2] += p;
      s[3] += p * m1;
      s[4] += dp * ck;
      s[5] += dp * sk;
      s[6] += dp;
      s[7] += dp * m1 + p * dm1;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = warp_sum(s[q]);
    if (lane < 8) {
      double v = s[0];
#pragma unroll
      for (int q = 1; q < 8; ++q)
        if (lane == q) v = s[q];
      out[(size_t)cell * 8 + lane] = v;
    }
  }
}

// One warp adds the per-cell sums in a fixed order: tot[8].
__global__ void k_tan_total(const double* cells, long long ncells, double* tot) {
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < 8; ++q) {
    double s = 0.0;
    for (long long c = lane; c < ncells; c += 32) s += cells[(size_t)c * 8 + q];
    s = warp_sum(s);
    if (lane == 0) tot[q] = s;
  }
}

}  // namespace mm

using namespace mmh;

namespace {

template <typename T, int V>
cudaError_t tan_launch_t(mm_handle* h, int parity, cudaStream_t s) {
  mm::TanArgs<T> t;
  t.a = step_args<T>(h, parity);
  t.a.seg = h->tan_seg;
  t.dpsi_in = (const T*)h->tan_psi[parity];
  t.dpsi_out = (T*)h->tan_psi[parity ^ 1];
  t.dnb_in = (const T*)h->tan_nb[parity];
  t.dnb_out = (T*)h->tan_nb[parity ^ 1];
  t.dmb = (T*)h->tan_mb;
  t.dmf = (T*)h->tan_mf;
  t.dkoff = h->tan_dp[0];
  t.dvw = h->tan_dp[1];
  t.dkon = h->tan_dp[2];
  const size_t smem = 4 * mm::tan_warp_smem(h->g.ntheta, sizeof(T));
  if (t.a.mass_correct)
    mm::k_substep_tl<T, V, true><<<h->tan_grid, 128, smem, s>>>(t);
  else
    mm::k_substep_tl<T, V, false><<<h->tan_grid, 128, smem, s>>>(t);
  return cudaGetLastError();
}

template <typename T, int V>
cudaError_t tan_prepare_t(mm_handle* h, int* per_sm) {
  const size_t smem = 4 * mm::tan_warp_smem(h->g.ntheta, sizeof(T));
  const void* fns[2] = {(const void*)mm::k_substep_tl<T, V, true>,
                        (const void*)mm::k_substep_tl<T, V, false>};
  for (const void* f : fns) {
    cudaError_t e = mm::raise_smem_limit(f, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, mm::k_substep_tl<T, V, true>, 128,
                                                       smem);
}

// Vector width of the tangent kernel: the registers hold the row and its
// tangent, so at most 4 float32 (2 float64) values per lane.
int tan_width(const mm_handle* h) {
  const int ns = h->g.ns;
  if (h->prec == MM_FP64) return (ns % 2 == 0 && ns / 2 <= 32) ? 2 : 1;
  if (ns % 4 == 0 && ns / 4 <= 32) return 4;
  if (ns % 2 == 0 && ns / 2 <= 32) return 2;
  return 1;
}

template <template <typename, int> class F, typename... A>
cudaError_t tan_by_width(mm_handle* h, A... args) {
  const int V = tan_width(h);
  if (h->prec == MM_FP64) return V == 2 ? F<double, 2>::run(h, args...) : F<double, 1>::run(h, args...);
  if (V == 4) return F<float, 4>::run(h, args...);
  return V == 2 ? F<float, 2>::run(h, args...) : F<float, 1>::run(h, args...);
}
template <typename T, int V>
struct TanLaunchF {
  static cudaError_t run(mm_handle* h, int parity, cudaStream_t s) {
    return tan_launch_t<T, V>(h, parity, s);
  }
};
template <typename T, int V>
struct TanPrepareF {
  static cudaError_t run(mm_handle* h, int* per_sm) { return tan_prepare_t<T, V>(h, per_sm); }
};

}  // namespace

namespace mmh {

void tangent_free(mm_handle* h) {
  void* p[6] = {h->tan_mb, h->tan_psi[0], h->tan_psi[1], h->tan_nb[0], h->tan_nb[1], h->tan_mf};
  for (void* q : p)
    if (q) cudaFree(q);
  h->tan_mb = h->tan_psi[0] = h->tan_psi[1] = h->tan_nb[0] = h->tan_nb[1] = h->tan_mf = nullptr;
  h->tangent = false;
}

cudaError_t launch_tangent_substep(mm_handle* h, int parity, cudaStream_t s) {
  return tan_by_width<TanLaunchF>(h, parity, s);
}

// A new state starts the tangent from zero (the direction is in the rates).
mm_status tangent_zero(mm_handle* h) {
  const size_t t = h->tsz;
  CK(cudaMemsetAsync(h->tan_mb, 0, h->mbn * t, h->stream));
  for (int p = 0; p < 2; ++p) {
    CK(cudaMemsetAsync(h->tan_psi[p], 0, h->rows * t, h->stream));
    CK(cudaMemsetAsync(h->tan_nb[p], 0, h->rows * t, h->stream));
  }
  CK(cudaMemsetAsync(h->tan_mf, 0, (size_t)h->ncells * t, h->stream));
  return MM_OK;
}

}  // namespace mmh

extern "C" {

mm_status mm_set_tangent(mm_handle* h, const double* dparams) {
  MM_TRACE("mm_set_tangent");
  if (!h) return MM_ERR_INVALID;
  if (h->batch || h->owner) return fail(h, MM_ERR_UNSUPPORTED, "the tangent is not available in a batch");
  if (h->rec.active)
    return fail(h, MM_ERR_STATE, "an adjoint recording is active: end it first");
  if (dparams && (h->anchors || h->capture))
    return fail(h, MM_ERR_UNSUPPORTED,
                "the tangent is not available with non-local anchors or a capture radius");
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream));
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  if (!dparams) {
    tangent_free(h);
    return MM_OK;
  }
  for (int q = 0; q < 3; ++q)
    if (!std::isfinite(dparams[q])) return fail(h, MM_ERR_INVALID, "dparams must be finite");
  if (!h->tan_mb) {
    const size_t t = h->tsz;
    size_t freeb = 0, totalb = 0;
    CK(cudaMemGetInfo(&freeb, &totalb));
    const size_t need = h->mbn * t + 4 * h->rows * t + (size_t)h->ncells * t;
    if (need + (64u << 20) > freeb) return fail(h, MM_ERR_OOM, "the tangent state does not fit");
    CK(cudaMalloc(&h->tan_mb, h->mbn * t));
    for (int p = 0; p < 2; ++p) {
      CK(cudaMalloc(&h->tan_psi[p], h->rows * t));
      CK(cudaMalloc(&h->tan_nb[p], h->rows * t));
    }
    CK(cudaMalloc(&h->tan_mf, (size_t)h->ncells * t));
  }
  const int V = tan_width(h);
  int seg = 1;
  while (seg < h->g.ns / V) seg <<= 1;
  if (seg > 32) return fail(h, MM_ERR_UNSUPPORTED, "ns too large for the tangent kernel");
  h->tan_seg = seg;
  if (4 * mm::tan_warp_smem(h->g.ntheta, (int)h->tsz) > kSmemBudget)
    return fail(h, MM_ERR_UNSUPPORTED, "ntheta too large for the tangent kernel");
  int per_sm = 0;
  CK(tan_by_width<TanPrepareF>(h, &per_sm));
  if (per_sm < 1) return fail(h, MM_ERR_UNSUPPORTED, "the tangent kernel cannot be resident");
  h->tan_grid = (int)std::max<long long>(
      1, std::min<long long>((h->ncells + 3) / 4, (long long)per_sm * h->sms));
  // the per-block partial sums of psi share the plain substep's buffer
  h->tan_grid = std::min(h->tan_grid, h->npartial);
  h->tan_dp[0] = dparams[0];
  h->tan_dp[1] = dparams[1];
  h->tan_dp[2] = dparams[2];
  h->tangent = true;
  return tangent_zero(h);
}

mm_status mm_get_tangent(mm_handle* h, double* dpsi, double* dmb, double* dmf, int on_device) {
  MM_TRACE("mm_get_tangent");
  if (!h) return MM_ERR_INVALID;
  if (!h->tangent) return fail(h, MM_ERR_STATE, "no tangent (mm_set_tangent)");
  DeviceGuard dg(h->device);
  mm_status st;
  const double* scale = h->prec == MM_FP32_MIXED ? &h->prm->psi_scale : nullptr;
  if (dpsi && (st = get_array(h, dpsi, h->tan_psi[h->parity], h->rows, on_device, scale)) != MM_OK)
    return st;
  if (dmb && (st = get_array(h, dmb, h->tan_mb, h->mbn, on_device, nullptr)) != MM_OK) return st;
  if (dmf && (st = get_array(h, dmf, h->tan_mf, (size_t)h->ncells, on_device, nullptr)) != MM_OK)
    return st;
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

mm_status mm_tangent_observable(mm_handle* h, int observable, double* value, double* dvalue) {
  MM_TRACE("mm_tangent_observable");
  if (!h || !value || !dvalue) return MM_ERR_INVALID;
  if (!h->tangent) return fail(h, MM_ERR_STATE, "no tangent (mm_set_tangent)");
  if (observable != MM_OBS_POLAR_ORDER && observable != MM_OBS_MEAN_STRESS)
    return fail(h, MM_ERR_INVALID, "observable must be MM_OBS_POLAR_ORDER or MM_OBS_MEAN_STRESS");
  DeviceGuard dg(h->device);
  const long long nc = h->ncells;
  const double ds = h->g.L / h->g.ns, dth = 2.0 * kPi / h->g.ntheta;
  // per-cell sums in the moments' field buffer (12 doubles per cell available)
  double* cells = h->fields;
  double* tot = h->partial;  // 8 doubles; the partial sums are free between substeps
  const int grid = (int)std::max<long long>(1, std::min<long long>((nc + 3) / 4, 8LL * h->sms));
  if (h->prec == MM_FP64)
    mm::k_tan_cells<double><<<grid, 128, 0, h->stream>>>(
        (const double*)h->psi[h->parity], (const double*)h->mb, (const double*)h->tan_psi[h->parity],
        (const double*)h->tan_mb, h->trig64, h->prm, nc, h->g.ntheta, h->g.ns, ds, h->g.L, cells);
  else
    mm::k_tan_cells<float><<<grid, 128, 0, h->stream>>>(
        (const float*)h->psi[h->parity], (const float*)h->mb, (const float*)h->tan_psi[h->parity],
        (const float*)h->tan_mb, h->trig64, h->prm, nc, h->g.ntheta, h->g.ns, ds, h->g.L, cells);
  CK(cudaGetLastError());
  mm::k_tan_total<<<1, 32, 0, h->stream>>>(cells, nc, tot);
  CK(cudaGetLastError());
  double s[8];
  CK(cudaMemcpyAsync(s, tot, sizeof s, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (observable == MM_OBS_POLAR_ORDER) {
    // L = |S| / N with S = sum psi e^{i theta}, N = sum psi
    const double S = std::sqrt(s[0] * s[0] + s[1] * s[1]), N = s[2];
    *value = S / N;
    const double dS = S > 0.0 ? (s[0] * s[4] + s[1] * s[5]) / S : 0.0;
    *dvalue = dS / N - S * s[6] / (N * N);
  } else {
    // L = mean over cells of tr sigma_a = F_m ell dth sum psi m1 / cells
    const double c = h->r.force_scale * h->r.ell * dth / (double)nc;
    *value = c * s[3];
    *dvalue = c * s[7];
  }
  return check_status(h);
}

}  // extern "C"
