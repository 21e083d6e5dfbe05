// Adjoint (reverse mode) of one microscale substep, and its seed and finish
// kernels.
//
// The forward substep maps (psi^n, Mb^n, Mf^n) to (psi^{n+1}, Mb^{n+1},
// Mf^{n+1}) at fixed dt and velocity: Eq. 1 for psi in donor-cell flux form,
// Eq. 4 for every s-row by midpoint RK2 (Alg. 2), the coarse density Eq. 5
// with psi^{n+1}, the scale-down of Alg. 2 and Eq. 6. Its adjoint is applied
// here in gather form, one warp per cell:
//   * lam_C, the adjoint of the coarse density before the scale-down, is
//     -lam_Mf^{n+1} where the cell did not clip and -D / C where it did
//     (D = sum over the cell of lam_Mb^{n+1} Mb^{n+1}, from the previous
//     reverse step), and enters the psi adjoint through C = sum psi n_b dtheta;
//   * the psi part transposes every face flux F = max(A,0) psi_L + min(A,0) psi_R
//     taking the branch the forward took (A > 0 upwinds from the left),
//     giving lam_psi^n, the adjoint of n_b^n through the gliding speed, and
//     accumulated adjoints of u (directly and through the velocity gradient);
//   * the motor part recomputes the RK2 stage of every row in registers and
//     applies the transposed Jacobians of both stages, with the Superbee
//     derivative of the branch the forward took, and accumulates the adjoints
//     of k_off, v_walk and k_on.
// Limits, order of operations and branch choices follow the oracle's adjoint.
#include "mm_internal.cuh"
#include "mm_walk.cuh"

namespace mm {

namespace {

// z = (d walk-term / dM)^T y for the V nodes a lane holds, where the walk
// term of R_j is (v/ds) (F_{j-1} - F_j) with F_j = M_j + sigma_j / 2
// (F_{ns-1} = M_{ns-1}, F_{-1} = 0, ghost M_{-1} = 0) and
// sigma_j / 2 = ga_j (M_j - M_{j-1}) + gb_j (M_{j+1} - M_j) on the branch the
// forward took (walk_dflux with COEF). With
// lam_F_j = (v/ds)(y_{j+1} - y_j) (lam_F_{ns-1} = -(v/ds) y_{ns-1}),
// P_j = ga_j lam_F_j and Q_j = gb_j lam_F_j:
// z_j = lam_F_j + P_j - Q_j - P_{j+1} + Q_{j-1}.
template <typename T, int V>
__device__ __forceinline__ void walk_adj(const T (&ga)[V], const T (&gb)[V], const T (&y)[V],
                                         T (&z)[V], bool first, bool last, int seg, T cw) {
  const T yr = __shfl_down_sync(0xffffffffu, y[0], 1, seg);
  T lF[V], P[V], Q[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const T yn = v == V - 1 ? yr : y[v + 1];
    lF[v] = cw * (yn - y[v]);
  }
  if (last) lF[V - 1] = -cw * y[V - 1];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    P[v] = ga[v] * lF[v];
    Q[v] = gb[v] * lF[v];
  }
  T Pr = __shfl_down_sync(0xffffffffu, P[0], 1, seg);
  T Ql = __shfl_up_sync(0xffffffffu, Q[V - 1], 1, seg);
  if (last) Pr = T(0);
  if (first) Ql = T(0);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const T pn = v == V - 1 ? Pr : P[v + 1];
    const T qp = v == 0 ? Ql : Q[v - 1];
    z[v] = lF[v] + P[v] - Q[v] - pn + qp;
  }
}

#ifndef MM_ADJ_V8_MIN_BLOCKS
#define MM_ADJ_V8_MIN_BLOCKS 3
#endif

// Resident blocks the register budget is sized for: float32 rows of up to 4
// values per lane fit 128 registers; 8 values per lane and float64 need more.
template <typename T, int V>
constexpr int adj_min_blocks() {
  return sizeof(T) == 8 ? 1 : (V == 8 ? MM_ADJ_V8_MIN_BLOCKS : 4);
}

// Adjoint of one substep, one warp per cell (grid-stride over cells).
// Per-warp shared memory: lam_psi_total and psi^n of the cell, and lam_n_b^n
// of its rows (3 nth values).
template <typename T, int V>
__global__ void __launch_bounds__(128, adj_min_blocks<T, V>()) k_adjoint(const AdjArgs<T> a) {
  extern __shared__ __align__(16) unsigned char adj_smem[];
  const int nth = a.nth, ns = a.ns, seg = a.seg;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* s_lt = reinterpret_cast<T*>(adj_smem) + (size_t)wib * 3 * nth;
  T* s_psi = s_lt + nth;
  T* s_lnb = s_psi + nth;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells, nx = a.nx, ny = a.ny;
  const int sl = lane & (seg - 1), rslot = lane / seg, rpp = 32 / seg;
  const int nl = ns / V;
  const bool first = sl == 0, last = sl == nl - 1, lane_ok = sl < nl;

  const T dt = (T)a.dt, hdt = (T)(0.5 * a.dt);
  const T cw = (T)(a.v_walk / a.ds), koff = (T)a.k_off, kon = (T)a.k_on;
  const T glide = (T)a.glide, vsp = (T)a.v_sp;
  const T c1 = hdt * cw, c2 = T(1) - hdt * koff;
  const T dtv = dt * (T)a.inv_dx, dtw = dt * (T)a.inv_dy, dtt = dt * (T)a.inv_dth;
  const T ds = (T)a.ds, dth = (T)a.dth, inv_ds = (T)(1.0 / a.ds);
  const T* cosk = a.trig;
  const T* sink = a.trig + nth;
  const T* cosf = a.trig + 2 * nth;
  const T* sinf = a.trig + 3 * nth;

  double g_koff = 0.0, g_v = 0.0, g_kon = 0.0;

  for (int cell = gw; cell < nc; cell += W) {
    const int iy = cell / nx, ix = cell - iy * nx;
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const int nbr[5] = {cell, iy * nx + xp, iy * nx + xm, yp * nx + ix, ym * nx + ix};
    // adjoint of the pre-scale-down coarse density and the scale factor, for
    // the cell and its 4 neighbours
    T lamC[5], fsc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int j = nbr[q];
      const T M = a.mtot[j], Cp = a.cpre_np[j];
      if (M < Cp) {
        fsc[q] = M / Cp;
        lamC[q] = -a.D_in[j] / Cp;
      } else {
        fsc[q] = T(1);
        lamC[q] = -a.lmf_in[j];
      }
    }
    // lam_psi_total = lam_psi^{n+1} + lam_C n_b** dtheta (n_b** = n_b^{n+1} / f)
    auto lam_tot = [&](int q, int k) -> T {
      const size_t r = (size_t)nbr[q] * nth + k;
      return a.lpsi_in[r] + lamC[q] * (a.nb_np[r] / fsc[q]) * dth;
    };
    for (int k = lane; k < nth; k += 32) {
      s_lt[k] = lam_tot(0, k);
      s_psi[k] = a.psi_n[(size_t)cell * nth + k];
    }
    __syncwarp();

    // ---- transpose of Eq. 1 (donor-cell flux form)
    const T* uc = a.ucell + (size_t)cell * 12;
    const T uxc = uc[0], uyc = uc[1], uxe = uc[2], uxw = uc[3], uyn = uc[4], uys = uc[5];
    const T Gxx = uc[6], Gxy = uc[7], Gyx = uc[8], Gyy = uc[9];
    T lux = T(0), luy = T(0), lG0 = T(0), lG1 = T(0), lG2 = T(0), lG3 = T(0);
    for (int k = lane; k < nth; k += 32) {
      const size_t rc = (size_t)cell * nth + k;
      const T pc = s_psi[k];
      const T pe = a.psi_n[(size_t)nbr[1] * nth + k], pw = a.psi_n[(size_t)nbr[2] * nth + k];
      const T pn = a.psi_n[(size_t)nbr[3] * nth + k], ps = a.psi_n[(size_t)nbr[4] * nth + k];
      const T ck = cosk[k], sk = sink[k];
      const T Vc = vsp + glide * a.nb_n[rc];
      const T Ve = vsp + glide * a.nb_n[(size_t)nbr[1] * nth + k];
      const T Vw = vsp + glide * a.nb_n[(size_t)nbr[2] * nth + k];
      const T Vn = vsp + glide * a.nb_n[(size_t)nbr[3] * nth + k];
      const T Vs = vsp + glide * a.nb_n[(size_t)nbr[4] * nth + k];
      const T axc = fma_t(-Vc, ck, uxc), axe = fma_t(-Ve, ck, uxe), axw = fma_t(-Vw, ck, uxw);
      const T ayc = fma_t(-Vc, sk, uyc), ayn = fma_t(-Vn, sk, uyn), ays = fma_t(-Vs, sk, uys);
      const T Ae = T(0.5) * (axc + axe), Aw = T(0.5) * (axw + axc);
      const T An = T(0.5) * (ayc + ayn), As = T(0.5) * (ays + ayc);
      const int kp = k + 1 == nth ? 0 : k + 1, km = k == 0 ? nth - 1 : k - 1;
      const T cp = cosf[k], sp = sinf[k], cm = cosf[km], sm = sinf[km];
      const T wp = -sp * (Gxx * cp + Gxy * sp) + cp * (Gyx * cp + Gyy * sp);
      const T wm = -sm * (Gxx * cm + Gxy * sm) + cm * (Gyx * cm + Gyy * sm);
      const T ltc = s_lt[k];
      const T lte = lam_tot(1, k), ltw = lam_tot(2, k), ltn = lam_tot(3, k), lts = lam_tot(4, k);
      // face adjoints lam_F = dt/h (lam_right - lam_left)
      const T lFe = dtv * (lte - ltc), lFw = dtv * (ltc - ltw);
      const T lFn = dtw * (ltn - ltc), lFs = dtw * (ltc - lts);
      const T lFp = dtt * (s_lt[kp] - ltc), lFm = dtt * (ltc - s_lt[km]);
      T lp = ltc + tmax(Ae, T(0)) * lFe + tmin(Aw, T(0)) * lFw + tmax(An, T(0)) * lFn +
             tmin(As, T(0)) * lFs + tmax(wp, T(0)) * lFp + tmin(wm, T(0)) * lFm;
      a.lpsi_out[rc] = lp;
      // face velocities: lam_A = psi_upwind lam_F, half to each side's a
      const T lAe = (Ae > T(0) ? pc : pe) * lFe, lAw = (Aw > T(0) ? pw : pc) * lFw;
      const T lAn = (An > T(0) ? pc : pn) * lFn, lAs = (As > T(0) ? ps : pc) * lFs;
      const T lax = T(0.5) * (lAe + lAw), lay = T(0.5) * (lAn + lAs);
      lux += lax;
      luy += lay;
      s_lnb[k] = -glide * (ck * lax + sk * lay);
      // rotation at the face k+1/2 owned by this orientation
      const T lw = (wp > T(0) ? pc : s_psi[kp]) * lFp;
      lG0 += lw * (-sp * cp);
      lG1 += lw * (-sp * sp);
      lG2 += lw * (cp * cp);
      lG3 += lw * (cp * sp);
    }
    {
      const double dlux = (double)warp_sum_t(lux), dluy = (double)warp_sum_t(luy);
      const double d0 = (double)warp_sum_t(lG0), d1 = (double)warp_sum_t(lG1);
      const double d2 = (double)warp_sum_t(lG2), d3 = (double)warp_sum_t(lG3);
      if (lane == 0) {
        a.lamu[cell] += dlux;
        a.lamu[nc + cell] += dluy;
        a.lamG[(size_t)cell * 4 + 0] += d0;
        a.lamG[(size_t)cell * 4 + 1] += d1;
        a.lamG[(size_t)cell * 4 + 2] += d2;
        a.lamG[(size_t)cell * 4 + 3] += d3;
      }
    }
    __syncwarp();

    // ---- transpose of Eq. 4 (midpoint RK2) on every row of the cell
    const T mf_n = a.mf_n[cell];
    const T c3 = hdt * kon * mf_n;
    const T lamC_c = lamC[0], f_c = fsc[0];
    T lmf_acc = T(0), D_acc = T(0);
    T gk = T(0), gv = T(0), gn = T(0);
    // rows of the next group are loaded one iteration ahead
    T Mq[V], Lq[V];
    auto load_rows = [&](int r0) {
      const int k = r0 + rslot;
      const bool act = k < nth && lane_ok;
      if (act) {
        const size_t off = ((size_t)cell * nth + k) * ns + (size_t)sl * V;
        const Pack<T, V> qm = *reinterpret_cast<const Pack<T, V>*>(a.mb_n + off);
        const Pack<T, V> ql = *reinterpret_cast<const Pack<T, V>*>(a.lmb + off);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          Mq[v] = qm.v[v];
          Lq[v] = ql.v[v];
        }
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          Mq[v] = T(0);
          Lq[v] = T(0);
        }
      }
    };
    load_rows(0);
    for (int r0 = 0; r0 < nth; r0 += rpp) {
      const int k = r0 + rslot;
      const bool row_ok = k < nth, act = row_ok && lane_ok;
      const size_t off = ((size_t)cell * nth + (row_ok ? k : 0)) * ns + (size_t)sl * V;
      T M[V], L[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        M[v] = Mq[v];
        L[v] = Lq[v];
      }
      const T psi1 = row_ok ? a.psi_np[(size_t)cell * nth + k] : T(0);
      const T lnb = row_ok ? s_lnb[k] * ds : T(0);
      if (r0 + rpp < nth) load_rows(r0 + rpp);
      // forward recompute: Ms = M + (dt/2) R(M), with the Superbee branch of
      // both stages
      T Dn[V], Ds[V], Ms[V], gan[V], gbn[V], gas[V], gbs[V];
      walk_dflux<T, V, true>(M, Dn, first, last, seg, gan, gbn);
#pragma unroll
      for (int v = 0; v < V; ++v) Ms[v] = fma_t(c1, Dn[v], fma_t(c2, M[v], c3));
      walk_dflux<T, V, true>(Ms, Ds, first, last, seg, gas, gbs);
      // lam_Mb** = f lam_Mb' + lam_C psi^{n+1} dtheta ds (through C and the scale-down)
      const T add = act ? lamC_c * psi1 * dth * ds : T(0);
      T y1[V], zs[V], y2[V], zn[V];
      T sy1 = T(0), sy2 = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        L[v] = f_c * L[v] + add;  // lam_Mb**
        y1[v] = dt * L[v];
        sy1 += y1[v];
      }
      walk_adj<T, V>(gas, gbs, y1, zs, first, last, seg, cw);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        zs[v] -= koff * y1[v];  // lam_Ms = J_R(Ms)^T y1
        gk -= Ms[v] * y1[v];
        gv += Ds[v] * inv_ds * y1[v];
        y2[v] = hdt * zs[v];
        sy2 += y2[v];
      }
      walk_adj<T, V>(gan, gbn, y2, zn, first, last, seg, cw);
      Pack<T, V> qo;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        gk -= M[v] * y2[v];
        gv += Dn[v] * inv_ds * y2[v];
        const T lm = L[v] + zs[v] + zn[v] - koff * y2[v] + lnb;
        qo.v[v] = lm;
        D_acc = fma_t(lm, M[v], D_acc);
      }
      if (act) *reinterpret_cast<Pack<T, V>*>(a.lmb + off) = qo;
      if (act) {
        lmf_acc += kon * (sy1 + sy2);
        gn += mf_n * (sy1 + sy2);
      }
    }
    const T lmf = warp_sum_t(lmf_acc);
    const T Dsum = warp_sum_t(D_acc);
    if (lane == 0) {
      a.lmf_out[cell] = lmf;
      a.D_out[cell] = Dsum;
    }
    g_koff += (double)gk;
    g_v += (double)gv;
    g_kon += (double)gn;
    __syncwarp();
  }
  g_koff = warp_sum(g_koff);
  g_v = warp_sum(g_v);
  g_kon = warp_sum(g_kon);
  if (lane == 0) {
    a.gpart[(size_t)gw * 4 + 0] += g_koff;
    a.gpart[(size_t)gw * 4 + 1] += g_v;
    a.gpart[(size_t)gw * 4 + 2] += g_kon;
  }
}

// Seeds of the reverse sweep at the final state.
//   kind 0: user seeds (float64 arrays, any may be NULL): lam_psi = dpsi,
//           lam_Mb(k, j) = dnb(k) ds + dm1(k) s_j ds, lam_Mf = dmf.
//   kind 1: polar order |P| / S with P = sum psi p, S = sum psi:
//           lam_psi(k) = coef[0] + coef[1] cos theta_k + coef[2] sin theta_k.
//   kind 2: mean of tr sigma_a = (F ell / cells) sum psi m1 dtheta:
//           lam_psi = coef[0] m1, lam_Mb(k, j) = coef[0] psi(k) s_j ds.
// Also D = sum over the cell of lam_Mb Mb. One warp per cell.
template <typename T>
__global__ void k_adj_seed(int kind, const double* coef, const T* psi, const T* mb,
                           const double* dpsi, const double* dnb, const double* dm1,
                           const double* dmf, T* lpsi, T* lmb, T* lmf, T* D, long long ncells,
                           int nth, int ns, double ds, double L, const T* trig) {
  const int lane = threadIdx.x & 31;
  const long long gw = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long cell = gw; cell < ncells; cell += W) {
    double dsum = 0.0;
    // one row at a time, the s-nodes across the lanes
    for (int k = 0; k < nth; ++k) {
      const size_t r = (size_t)cell * nth + k;
      const T* row = mb + r * ns;
      T* lrow = lmb + r * ns;
      double lp = 0.0, a_nb = 0.0, a_m1 = 0.0;
      if (kind == 0) {
        lp = dpsi ? dpsi[r] : 0.0;
        a_nb = dnb ? dnb[r] : 0.0;
        a_m1 = dm1 ? dm1[r] : 0.0;
      } else if (kind == 1) {
        lp = coef[0] + coef[1] * (double)trig[k] + coef[2] * (double)trig[nth + k];
      } else {
        double m1 = 0.0;
        for (int j = lane; j < ns; j += 32)
          m1 += (-0.5 * L + (j + 0.5) * ds) * (double)row[j] * ds;
        lp = coef[0] * warp_sum(m1);
        a_m1 = coef[0] * (double)psi[r];
      }
      if (lane == 0) lpsi[r] = (T)lp;
      for (int j = lane; j < ns; j += 32) {
        const double sj = -0.5 * L + (j + 0.5) * ds;
        const T lm = (T)(a_nb * ds + a_m1 * sj * ds);
        lrow[j] = lm;
        if (lm != T(0)) dsum += (double)lm * (double)row[j];
      }
    }
    dsum = warp_sum(dsum);
    if (lane == 0) {
      lmf[cell] = (T)((kind == 0 && dmf) ? dmf[cell] : 0.0);
      D[cell] = (T)dsum;
    }
  }
}

// dL/du = direct adjoint + transpose of the periodic central differences
// G_xx = (ux_e - ux_w)/(2dx), G_xy = (ux_n - ux_s)/(2dy), G_yx, G_yy likewise.
__global__ void k_adj_finish(const double* lamG, const double* lamu, double* dLdu, int nx, int ny,
                             double inv_dx, double inv_dy) {
  const long long nc = (long long)nx * ny;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < nc;
       cell += (long long)gridDim.x * blockDim.x) {
    const int iy = (int)(cell / nx), ix = (int)(cell - (long long)iy * nx);
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    // cell is the east neighbour of xm (enters G(xm) with +) and the west
    // neighbour of xp (with -); likewise in y
    const long long cw = (long long)iy * nx + xm, ce = (long long)iy * nx + xp;
    const long long cs = (long long)ym * nx + ix, cn = (long long)yp * nx + ix;
    const double hx = 0.5 * inv_dx, hy = 0.5 * inv_dy;
    dLdu[cell] = lamu[cell] + hx * (lamG[cw * 4 + 0] - lamG[ce * 4 + 0]) +
                 hy * (lamG[cs * 4 + 1] - lamG[cn * 4 + 1]);
    dLdu[nc + cell] = lamu[nc + cell] + hx * (lamG[cw * 4 + 2] - lamG[ce * 4 + 2]) +
                      hy * (lamG[cs * 4 + 3] - lamG[cn * 4 + 3]);
  }
}

// dL/dpsi0 = lam_psi^0 - lam_Mf^0 n_b^0 dtheta (Mf^0 = M - sum psi^0 n_b^0 dtheta).
template <typename T>
__global__ void k_adj_psi0(const T* lpsi, const T* lmf, const T* nb, double dth, long long rows,
                           int nth, double* out) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x)
    out[r] = (double)lpsi[r] - (double)lmf[r / nth] * (double)nb[r] * dth;
}

}  // namespace

template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T>& a, int V, int grid, cudaStream_t s) {
  const int block = 128;
  const size_t smem = (size_t)4 * 3 * a.nth * sizeof(T);
  auto go = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
  };
  if constexpr (sizeof(T) == 4)
    if (V == 8) return go(k_adjoint<T, 8>);
  if (V == 4) return go(k_adjoint<T, 4>);
  if (V == 2) return go(k_adjoint<T, 2>);
  return go(k_adjoint<T, 1>);
}

template <typename T>
cudaError_t launch_adj_seed(int kind, const double* coef, const T* psi, const T* mb,
                            const double* dpsi, const double* dnb, const double* dm1,
                            const double* dmf, T* lpsi, T* lmb, T* lmf, T* D, long long ncells,
                            int nth, int ns, double ds, double L, const T* trig, cudaStream_t s) {
  long long g = (ncells + 3) / 4;
  if (g > 152 * 8) g = 152 * 8;
  k_adj_seed<T><<<(int)g, 128, 0, s>>>(kind, coef, psi, mb, dpsi, dnb, dm1, dmf, lpsi, lmb, lmf,
                                       D, ncells, nth, ns, ds, L, trig);
  return cudaGetLastError();
}

cudaError_t launch_adj_finish(const double* lamG, const double* lamu, double* dLdu, int nx, int ny,
                              double inv_dx, double inv_dy, cudaStream_t s) {
  const long long nc = (long long)nx * ny;
  long long g = (nc + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_adj_finish<<<(int)g, 256, 0, s>>>(lamG, lamu, dLdu, nx, ny, inv_dx, inv_dy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_psi0(const T* lpsi, const T* lmf, const T* nb, double dth, long long rows,
                            int nth, double* out, cudaStream_t s) {
  long long g = (rows + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_adj_psi0<T><<<(int)g, 256, 0, s>>>(lpsi, lmf, nb, dth, rows, nth, out);
  return cudaGetLastError();
}

#define MM_ADJ_INST(T)                                                                          \
  template cudaError_t launch_adjoint<T>(const AdjArgs<T>&, int, int, cudaStream_t);            \
  template cudaError_t launch_adj_seed<T>(int, const double*, const T*, const T*, const double*, \
                                          const double*, const double*, const double*, T*, T*,  \
                                          T*, T*, long long, int, int, double, double, const T*, \
                                          cudaStream_t);                                        \
  template cudaError_t launch_adj_psi0<T>(const T*, const T*, const T*, double, long long, int,  \
                                          double*, cudaStream_t);
MM_ADJ_INST(float)
MM_ADJ_INST(double)

}  // namespace mm
