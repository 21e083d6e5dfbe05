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
#include "mm_async.cuh"
#include "mm_cell.cuh"

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

// The reverse kernels are launched overlapped (launch_overlapped): every block
// first waits in griddep_wait for the kernel before it in the stream.

// Resident blocks the staged psi reverse kernel is sized for (registers) in
// float32 (float64 keeps its natural register count).
#ifndef MM_ADJ_PSI_MIN_BLOCKS
#define MM_ADJ_PSI_MIN_BLOCKS 8
#endif
template <typename T>
constexpr int adj_psi_min_blocks() {
  return sizeof(T) == 8 ? 3 : MM_ADJ_PSI_MIN_BLOCKS;
}
#ifndef MM_ADJ_MOTOR_MIN_BLOCKS
#define MM_ADJ_MOTOR_MIN_BLOCKS 4
#endif

// Resident blocks the register budget of the motor kernel is sized for:
// float32 rows of up to 4 values per lane; 8 values per lane and float64 need
// more registers.
template <typename T, int V>
constexpr int adj_min_blocks() {
  return sizeof(T) == 8 ? 1 : (V == 8 ? 3 : MM_ADJ_MOTOR_MIN_BLOCKS);
}

// lam_C (the adjoint of the coarse density before the scale-down) and the
// scale-down factor f of a cell at n+1 (Alg. 2): lam_C = -D / C where the cell
// clipped (D = sum lam_Mb Mb), else -lam_Mf.
template <typename T>
__device__ __forceinline__ void cell_lamc(const AdjArgs<T>& a, int cell, T& lamC, T& f) {
  const T M = a.mtot[cell], Cp = a.cpre_np[cell];
  const size_t nc = (size_t)a.ncells;
  // both sums are loaded (independent of the branch, so the loads overlap)
  T D = T(0), lmf = T(0);
  for (int u = 0; u < a.units; ++u) {
    D += a.D_in[u * nc + cell];
    lmf += a.lmf_in[u * nc + cell];
  }
  if (M < Cp) {
    f = M / Cp;
    lamC = -D / Cp;
  } else {
    f = T(1);
    lamC = -lmf;
  }
}

// Where the psi adjoint of a cell reads the columns of the cell and its four
// neighbours (q = 0 cell, 1 east, 2 west, 3 north, 4 south): psi^n, n_b^n,
// lam_psi^{n+1}, n_b^{n+1}, and the cell's velocity block. ColsGlobal reads
// them in place; ColsSmem from a stage [psi 5][n_b 5][lam_psi 5][n_b' 5][u 12].
template <typename T>
struct ColsGlobal {
  const AdjArgs<T>* a;
  int nbr[5];
  int cell;
  __device__ T psi(int q, int k) const { return a->psi_n[(size_t)nbr[q] * a->nth + k]; }
  __device__ T nb(int q, int k) const { return a->nb_n[(size_t)nbr[q] * a->nth + k]; }
  __device__ T lp(int q, int k) const { return a->lpsi_in[(size_t)nbr[q] * a->nth + k]; }
  __device__ T nbp(int q, int k) const { return a->nb_np[(size_t)nbr[q] * a->nth + k]; }
  __device__ T u(int i) const { return a->ucell[(size_t)cell * 12 + i]; }
};
template <typename T>
struct ColsSmem {
  const T* st;
  int nth;
  __device__ T psi(int q, int k) const { return st[q * nth + k]; }
  __device__ T nb(int q, int k) const { return st[(5 + q) * nth + k]; }
  __device__ T lp(int q, int k) const { return st[(10 + q) * nth + k]; }
  __device__ T nbp(int q, int k) const { return st[(15 + q) * nth + k]; }
  __device__ T u(int i) const { return st[20 * nth + i]; }
};

// The psi adjoint of one cell (lanes over theta): transposes every donor-cell
// face flux on the branch the forward took, giving lam_psi^n, the adjoint of
// n_b^n through the gliding speed (stored, times ds, for part 2), and the
// cell's accumulated adjoints of u and of its velocity gradient (acc_old: the
// accumulator lane j < 6 holds, read earlier); stores lam_C and f of the cell.
// s_lt: nth values of shared memory for the cell's lam_psi_total.
// The scalars of the psi part in the state precision. In float32 the eight
// float64 values are converted by one instruction for the warp (lane q
// converts value q, then shuffles): conversions from float64 run on the narrow
// float64 pipe, and the cell loop needs them once per launch, not per cell.
template <typename T>
struct PsiAdjConst {
  T dt, glide, vsp, dtv, dtw, dtt, ds, dth;
};
template <typename T>
__device__ __forceinline__ PsiAdjConst<T> psi_adj_const(const AdjArgs<T>& a, int lane) {
  PsiAdjConst<T> c;
  if constexpr (sizeof(T) == 4) {
    const double v = lane == 0 ? *a.dt : lane == 1 ? a.glide : lane == 2 ? a.v_sp
                   : lane == 3 ? a.inv_dx : lane == 4 ? a.inv_dy : lane == 5 ? a.inv_dth
                   : lane == 6 ? a.ds : a.dth;
    const float x = (float)v;
    c.dt = __shfl_sync(0xffffffffu, x, 0);
    c.glide = __shfl_sync(0xffffffffu, x, 1);
    c.vsp = __shfl_sync(0xffffffffu, x, 2);
    c.dtv = c.dt * __shfl_sync(0xffffffffu, x, 3);
    c.dtw = c.dt * __shfl_sync(0xffffffffu, x, 4);
    c.dtt = c.dt * __shfl_sync(0xffffffffu, x, 5);
    c.ds = __shfl_sync(0xffffffffu, x, 6);
    c.dth = __shfl_sync(0xffffffffu, x, 7);
  } else {
    c.dt = *a.dt;
    c.glide = a.glide;
    c.vsp = a.v_sp;
    c.dtv = c.dt * a.inv_dx;
    c.dtw = c.dt * a.inv_dy;
    c.dtt = c.dt * a.inv_dth;
    c.ds = a.ds;
    c.dth = a.dth;
  }
  return c;
}

template <typename T, class Cols>
__device__ __forceinline__ void psi_adj_cell(const AdjArgs<T>& a, const PsiAdjConst<T>& pc0,
                                             const Cols& C, int cell, const T (&lamC)[5],
                                             const T (&fsc)[5], T* s_lt, double acc_old,
                                             int lane) {
  const int nth = a.nth, nc = (int)a.ncells;
  const T glide = pc0.glide, vsp = pc0.vsp;
  const T dtv = pc0.dtv, dtw = pc0.dtw, dtt = pc0.dtt;
  const T ds = pc0.ds, dth = pc0.dth;
  const T* cosk = a.trig;
  const T* sink = a.trig + nth;
  const T* cosf = a.trig + 2 * nth;
  const T* sinf = a.trig + 3 * nth;
  // lam_psi_total = lam_psi^{n+1} + lam_C n_b** dtheta (n_b** = n_b^{n+1} / f)
  auto lam_tot = [&](int q, int k) -> T { return C.lp(q, k) + lamC[q] * (C.nbp(q, k) / fsc[q]) * dth; };
  for (int k = lane; k < nth; k += 32) s_lt[k] = lam_tot(0, k);
  __syncwarp();
  const T uxc = C.u(0), uyc = C.u(1), uxe = C.u(2), uxw = C.u(3), uyn = C.u(4), uys = C.u(5);
  const T Gxx = C.u(6), Gxy = C.u(7), Gyx = C.u(8), Gyy = C.u(9);
  T lux = T(0), luy = T(0), lG0 = T(0), lG1 = T(0), lG2 = T(0), lG3 = T(0);
  for (int k = lane; k < nth; k += 32) {
    const size_t rc = (size_t)cell * nth + k;
    const T pc = C.psi(0, k), pe = C.psi(1, k), pw = C.psi(2, k), pn = C.psi(3, k),
            ps = C.psi(4, k);
    const T ck = cosk[k], sk = sink[k];
    const T Vc = fma_t(glide, C.nb(0, k), vsp), Ve = fma_t(glide, C.nb(1, k), vsp);
    const T Vw = fma_t(glide, C.nb(2, k), vsp), Vn = fma_t(glide, C.nb(3, k), vsp);
    const T Vs = fma_t(glide, C.nb(4, k), vsp);
    const T axc = fma_t(-Vc, ck, uxc), axe = fma_t(-Ve, ck, uxe), axw = fma_t(-Vw, ck, uxw);
    const T ayc = fma_t(-Vc, sk, uyc), ayn = fma_t(-Vn, sk, uyn), ays = fma_t(-Vs, sk, uys);
    const T Ae = T(0.5) * (axc + axe), Aw = T(0.5) * (axw + axc);
    const T An = T(0.5) * (ayc + ayn), As = T(0.5) * (ays + ayc);
    const int kp = k + 1 == nth ? 0 : k + 1, km = k == 0 ? nth - 1 : k - 1;
    const T cp = cosf[k], sp = sinf[k], cm = cosf[km], sm = sinf[km];
    // (the forward substep's fused form: the same upwind sides)
    const T wp = fma_t(-sp, fma_t(Gxx, cp, Gxy * sp), cp * fma_t(Gyx, cp, Gyy * sp));
    const T wm = fma_t(-sm, fma_t(Gxx, cm, Gxy * sm), cm * fma_t(Gyx, cm, Gyy * sm));
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
    a.lnb[rc] = -glide * (ck * lax + sk * lay) * ds;
    // rotation at the face k+1/2 owned by this orientation
    const T lw = (wp > T(0) ? pc : C.psi(0, kp)) * lFp;
    lG0 += lw * (-sp * cp);
    lG1 += lw * (-sp * sp);
    lG2 += lw * (cp * cp);
    lG3 += lw * (cp * sp);
  }
  const T s_ux = warp_sum_t(lux), s_uy = warp_sum_t(luy);
  const T s_g0 = warp_sum_t(lG0), s_g1 = warp_sum_t(lG1);
  const T s_g2 = warp_sum_t(lG2), s_g3 = warp_sum_t(lG3);
  // lane j < 6 adds the j-th of (ux, uy, G0..G3) to its accumulator
  const T mine = lane == 0 ? s_ux : lane == 1 ? s_uy : lane == 2 ? s_g0
               : lane == 3 ? s_g1 : lane == 4 ? s_g2 : s_g3;
  if (lane < 2)
    a.lamu[(size_t)lane * nc + cell] = acc_old + (double)mine;
  else if (lane < 6)
    a.lamG[(size_t)cell * 4 + (lane - 2)] = acc_old + (double)mine;
  if (lane == 0) {
    a.cellc[(size_t)cell * 2 + 0] = lamC[0];
    a.cellc[(size_t)cell * 2 + 1] = fsc[0];
  }
  __syncwarp();
}

__device__ __forceinline__ void cell_nbrs(int cell, int nx, int ny, int (&nbr)[5]) {
  const int iy = cell / nx, ix = cell - iy * nx;
  const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
  const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
  nbr[0] = cell;
  nbr[1] = iy * nx + xp;
  nbr[2] = iy * nx + xm;
  nbr[3] = yp * nx + ix;
  nbr[4] = ym * nx + ix;
}

// Adjoint of one substep, part 1: Eq. 1 and the coupling through C, one warp
// per cell (grid-stride), columns read in place (any ntheta). Per-warp shared
// memory: the cell's lam_psi_total (nth values).
template <typename T>
__global__ void __launch_bounds__(128) k_adj_psi(const AdjArgs<T> a) {
  griddep_wait();
  extern __shared__ __align__(16) unsigned char adj_smem[];
  const int nth = a.nth;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* s_lt = reinterpret_cast<T*>(adj_smem) + (size_t)wib * nth;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  const PsiAdjConst<T> pc0 = psi_adj_const(a, lane);
  for (int cell = gw; cell < nc; cell += W) {
    ColsGlobal<T> C;
    C.a = &a;
    C.cell = cell;
    cell_nbrs(cell, a.nx, a.ny, C.nbr);
    double acc_old = 0.0;
    if (lane < 2)
      acc_old = a.lamu[(size_t)lane * nc + cell];
    else if (lane < 6)
      acc_old = a.lamG[(size_t)cell * 4 + (lane - 2)];
    T lamC[5], fsc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) cell_lamc(a, C.nbr[q], lamC[q], fsc[q]);
    psi_adj_cell(a, pc0, C, cell, lamC, fsc, s_lt, acc_old, lane);
  }
}

// Stage bytes of the staged psi adjoint: 20 columns and the velocity block.
__host__ __device__ inline size_t psi_stage_bytes(int nth, int tsz) {
  return ((size_t)(20 * nth + 12) * tsz + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t psi_ring_warp_bytes(int nth, int tsz) {
  return 128 + 2 * psi_stage_bytes(nth, tsz) + (((size_t)nth * tsz + 15) & ~(size_t)15);
}

// The same with the columns of the next cell staged by bulk copies while the
// current one is computed (two stages per warp; needs nth * sizeof(T) a
// multiple of 16). Lane 0 posts the expected bytes, lanes 0-20 each issue
// one copy. Waits are bounded; a warp whose wait runs out records the
// failure, drains its copy and leaves.
template <typename T>
__global__ void __launch_bounds__(128, adj_psi_min_blocks<T>()) k_adj_psi_ring(const AdjArgs<T> a) {
  griddep_wait();
  extern __shared__ __align__(128) unsigned char psr_smem[];
  const int nth = a.nth, nx = a.nx, ny = a.ny;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t stb = psi_stage_bytes(nth, (int)sizeof(T));
  unsigned char* wbase = psr_smem + (size_t)wib * psi_ring_warp_bytes(nth, (int)sizeof(T));
  uint64_t* bars = reinterpret_cast<uint64_t*>(wbase);  // [2] stages, [2] never
  T* stage[2] = {reinterpret_cast<T*>(wbase + 128), reinterpret_cast<T*>(wbase + 128 + stb)};
  T* s_lt = reinterpret_cast<T*>(wbase + 128 + 2 * stb);
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  const uint32_t wait_limit = a.prm->wait_limit;
  const bool wait_never = (a.prm->debug_flags & 1u) != 0;
  const PsiAdjConst<T> pc0 = psi_adj_const(a, lane);
  const uint32_t colb = (uint32_t)(nth * sizeof(T));
  const uint32_t ub = (uint32_t)(12 * sizeof(T));
  auto issue = [&](int cell, int sidx) {
    int nbr[5];
    cell_nbrs(cell, nx, ny, nbr);
    if (lane == 0) mbar_expect_tx(&bars[sidx], 20 * colb + ub);
    __syncwarp();
    if (lane < 20) {
      const int f = lane / 5, q = lane - 5 * f;
      const T* src = f == 0 ? a.psi_n : f == 1 ? a.nb_n : f == 2 ? a.lpsi_in : a.nb_np;
      bulk_g2s(stage[sidx] + (size_t)lane * nth, src + (size_t)nbr[q] * nth, colb, &bars[sidx]);
    } else if (lane == 20) {
      bulk_g2s(stage[sidx] + (size_t)20 * nth, a.ucell + (size_t)cell * 12, ub, &bars[sidx]);
    }
  };
  if (lane == 0) {
    for (int q = 0; q < 3; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (gw < nc) issue(gw, 0);
  int sidx = 0;
  uint32_t par[2] = {0u, 0u};
  bool timed_out = false, pending_next = false;
  for (int cell = gw; cell < nc; cell += W) {
    const int next = cell + W;
    // scalar inputs of this cell (independent of the copies in flight)
    int nbr[5];
    cell_nbrs(cell, nx, ny, nbr);
    double acc_old = 0.0;
    if (lane < 2)
      acc_old = a.lamu[(size_t)lane * nc + cell];
    else if (lane < 6)
      acc_old = a.lamG[(size_t)cell * 4 + (lane - 2)];
    T lamC[5], fsc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) cell_lamc(a, nbr[q], lamC[q], fsc[q]);
    // the next cell's columns into the other stage
    if (next < nc) issue(next, sidx ^ 1);
    const bool ok = __all_sync(0xffffffffu, wait_never ? mbar_wait(&bars[2], 0u, wait_limit)
                                                       : mbar_wait(&bars[sidx], par[sidx], wait_limit));
    if (!ok) {
      timed_out = true;
      pending_next = next < nc;
      break;
    }
    par[sidx] ^= 1u;
    ColsSmem<T> C{stage[sidx], nth};
    psi_adj_cell(a, pc0, C, cell, lamC, fsc, s_lt, acc_old, lane);
    sidx ^= 1;
  }
  if (timed_out) {
    // record the failure; wait (bounded) for the copies this warp issued
    if (lane == 0) {
      atomicOr(&a.prm->status, 1);
      drain_wait(&bars[sidx], par[sidx], &a.prm->status);
      if (pending_next) drain_wait(&bars[sidx ^ 1], par[sidx ^ 1], &a.prm->status);
    }
    __syncwarp();
  }
}

// Constants of the motor part of one reverse substep.
template <typename T>
struct MotorConst {
  T dt, hdt, cw, koff, kon, c1, c2, ds, dth;
};

// Per-warp accumulators of the motor part: the unit's sums of lam_Mf and D,
// and the parameter adjoints (k_off, v_walk times ds, k_on).
template <typename T>
struct MotorAcc {
  T lmf, D, gk, gv, gn;
};

// ---- float32 rows of V = 4 or 8 nodes per lane as register pairs (nodes
// 2k, 2k + 1): the element-wise arithmetic of motor_rows as packed two-value
// instructions; shifted differences, the limiter and its branch decisions
// stay scalar. The same values as the scalar form (the accumulations over a
// lane's nodes run in two interleaved sums).

// One node of the COEF walk: the Superbee value r (sigma/2 = sgn r) and the
// branch coefficients, with the comparisons of walk_dflux<..., true>.
__device__ __forceinline__ void coef_node(float A, float hA, float hB, float B, float& r,
                                          float& ga, float& gb) {
  const float t1 = fminf(A, hB), t2 = fminf(hA, B);
  r = max3_t(t1, t2, 0.0f);
  const bool pos = r > 0.0f, p1 = t1 > t2, x1a = A < hB, x2a = hA < B;
  const float a1 = x1a ? 1.0f : 0.0f, b1 = x1a ? 0.0f : 0.5f;
  const float a2 = x2a ? 0.5f : 0.0f, b2 = x2a ? 0.0f : 1.0f;
  ga = pos ? (p1 ? a1 : a2) : 0.0f;
  gb = pos ? (p1 ? b1 : b2) : 0.0f;
}

template <int V>
__device__ __forceinline__ void walk_coef_x2(const float2 (&M)[V / 2], float2 (&D)[V / 2],
                                             float2 (&ga)[V / 2], float2 (&gb)[V / 2], bool first,
                                             bool last, int seg) {
  constexpr int H = V / 2;
  float ml = __shfl_up_sync(0xffffffffu, M[H - 1].y, 1, seg);
  const float mr = __shfl_down_sync(0xffffffffu, M[0].x, 1, seg);
  if (first) ml = 0.0f;
  float2 d[H], hd[H];
  d[0] = make_float2(M[0].x - ml, M[0].y - M[0].x);
#pragma unroll
  for (int k = 1; k < H; ++k) d[k] = make_float2(M[k].x - M[k - 1].y, M[k].y - M[k].x);
  const float dV = mr - M[H - 1].y, hdV = 0.5f * dV;
  const float2 half2 = make_float2(0.5f, 0.5f);
#pragma unroll
  for (int k = 0; k < H; ++k) hd[k] = __fmul2_rn(half2, d[k]);
  float2 F[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float b1 = k + 1 < H ? d[k + 1].x : dV, hb1 = k + 1 < H ? hd[k + 1].x : hdV;
    float2 sg = make_float2(copysignf(1.0f, d[k].y), copysignf(1.0f, b1));
    if (k == H - 1 && last) sg.y = 0.0f;  // plus end: F = M, no slope
    const float2 A = __fmul2_rn(d[k], sg), hA = __fmul2_rn(hd[k], sg);
    float2 r;
    coef_node(A.x, hA.x, fabsf(hd[k].y), fabsf(d[k].y), r.x, ga[k].x, gb[k].x);
    coef_node(A.y, hA.y, fabsf(hb1), fabsf(b1), r.y, ga[k].y, gb[k].y);
    F[k] = __ffma2_rn(r, sg, M[k]);
  }
  float fl = __shfl_up_sync(0xffffffffu, F[H - 1].y, 1, seg);
  if (first) fl = 0.0f;
  D[0] = make_float2(fl - F[0].x, F[0].x - F[0].y);
#pragma unroll
  for (int k = 1; k < H; ++k) D[k] = make_float2(F[k - 1].y - F[k].x, F[k].x - F[k].y);
}

// walk_adj on register pairs.
template <int V>
__device__ __forceinline__ void walk_adj_x2(const float2 (&ga)[V / 2], const float2 (&gb)[V / 2],
                                            const float2 (&y)[V / 2], float2 (&z)[V / 2],
                                            bool first, bool last, int seg, float cw) {
  constexpr int H = V / 2;
  const float yr = __shfl_down_sync(0xffffffffu, y[0].x, 1, seg);
  const float2 cw2 = make_float2(cw, cw);
  float2 lF[H], P[H], Q[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float yn1 = k + 1 < H ? y[k + 1].x : yr;
    lF[k] = __fmul2_rn(cw2, make_float2(y[k].y - y[k].x, yn1 - y[k].y));
  }
  if (last) lF[H - 1].y = -cw * y[H - 1].y;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    P[k] = __fmul2_rn(ga[k], lF[k]);
    Q[k] = __fmul2_rn(gb[k], lF[k]);
  }
  float Pr = __shfl_down_sync(0xffffffffu, P[0].x, 1, seg);
  float Ql = __shfl_up_sync(0xffffffffu, Q[H - 1].y, 1, seg);
  if (last) Pr = 0.0f;
  if (first) Ql = 0.0f;
  const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float2 t = __ffma2_rn(Q[k], m1, __fadd2_rn(lF[k], P[k]));  // lF + P - Q
    const float pn1 = k + 1 < H ? P[k + 1].x : Pr, qp0 = k > 0 ? Q[k - 1].y : Ql;
    z[k] = make_float2((t.x - P[k].y) + qp0, (t.y - pn1) + Q[k].x);
  }
}

template <int V>
__device__ __forceinline__ void motor_rows_x2(const float (&Mv)[V], float (&Lv)[V], float psi1,
                                              float lnb, bool act, bool first, bool last, int seg,
                                              const MotorConst<float>& m, float c3, float mf_n,
                                              float lamC_c, float f_c, MotorAcc<float>& acc,
                                              Pack<float, V>& out) {
  constexpr int H = V / 2;
  float2 M[H], L[H], Dn[H], Ds[H], Ms[H], gan[H], gbn[H], gas[H], gbs[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    M[k] = make_float2(Mv[2 * k], Mv[2 * k + 1]);
    L[k] = make_float2(Lv[2 * k], Lv[2 * k + 1]);
  }
  walk_coef_x2<V>(M, Dn, gan, gbn, first, last, seg);
  const float2 c1 = make_float2(m.c1, m.c1), c2 = make_float2(m.c2, m.c2);
  const float2 c32 = make_float2(c3, c3);
#pragma unroll
  for (int k = 0; k < H; ++k) Ms[k] = __ffma2_rn(c1, Dn[k], __ffma2_rn(c2, M[k], c32));
  walk_coef_x2<V>(Ms, Ds, gas, gbs, first, last, seg);
  // lam_Mb** = f lam_Mb' + lam_C psi^{n+1} dtheta ds (through C and the scale-down)
  const float add = act ? lamC_c * psi1 * m.dth * m.ds : 0.0f;
  const float2 f2 = make_float2(f_c, f_c), add2 = make_float2(add, add);
  const float2 dt2 = make_float2(m.dt, m.dt), hdt2 = make_float2(m.hdt, m.hdt);
  const float2 nk2 = make_float2(-m.koff, -m.koff), z2 = make_float2(0.0f, 0.0f);
  float2 y1[H], zs[H], y2[H], zn[H];
  float2 sy1 = z2, sy2 = z2, gk = z2, gv = z2, Dacc = z2;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    L[k] = __ffma2_rn(f2, L[k], add2);  // lam_Mb**
    y1[k] = __fmul2_rn(dt2, L[k]);
    sy1 = __fadd2_rn(sy1, y1[k]);
  }
  walk_adj_x2<V>(gas, gbs, y1, zs, first, last, seg, m.cw);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    zs[k] = __ffma2_rn(nk2, y1[k], zs[k]);  // lam_Ms = J_R(Ms)^T y1
    gk = __ffma2_rn(make_float2(-Ms[k].x, -Ms[k].y), y1[k], gk);
    gv = __ffma2_rn(Ds[k], y1[k], gv);
    y2[k] = __fmul2_rn(hdt2, zs[k]);
    sy2 = __fadd2_rn(sy2, y2[k]);
  }
  walk_adj_x2<V>(gan, gbn, y2, zn, first, last, seg, m.cw);
  const float2 lnb2 = make_float2(lnb, lnb);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    gk = __ffma2_rn(make_float2(-M[k].x, -M[k].y), y2[k], gk);
    gv = __ffma2_rn(Dn[k], y2[k], gv);
    float2 lm = __fadd2_rn(__fadd2_rn(L[k], zs[k]), zn[k]);
    lm = __fadd2_rn(__ffma2_rn(nk2, y2[k], lm), lnb2);
    out.v[2 * k] = lm.x;
    out.v[2 * k + 1] = lm.y;
    Dacc = __ffma2_rn(lm, M[k], Dacc);
  }
  acc.gk += gk.x + gk.y;
  acc.gv += gv.x + gv.y;
  acc.D += Dacc.x + Dacc.y;
  if (act) {
    const float sy = (sy1.x + sy1.y) + (sy2.x + sy2.y);
    acc.lmf += m.kon * sy;
    acc.gn += mf_n * sy;
  }
  (void)Lv;
}

// The reverse of Eq. 4 on one group of rows (V nodes per lane): M = Mb^n and
// L = lam_Mb^{n+1} of the lane's nodes, psi1 = psi^{n+1} and lnb = lam_n_b^n ds
// of the lane's row; returns lam_Mb^n of the nodes in `out`. Recomputes the
// RK2 stage with the forward's arithmetic and Superbee branches, then applies
// the transposed Jacobians of both stages.
template <typename T, int V>
__device__ __forceinline__ void motor_rows(const T (&M)[V], T (&L)[V], T psi1, T lnb, bool act,
                                           bool first, bool last, int seg, const MotorConst<T>& m,
                                           T c3, T mf_n, T lamC_c, T f_c, MotorAcc<T>& acc,
                                           Pack<T, V>& out) {
  if constexpr (sizeof(T) == 4 && (V == 4 || V == 8)) {
    motor_rows_x2<V>(M, L, psi1, lnb, act, first, last, seg, m, c3, mf_n, lamC_c, f_c, acc, out);
  } else {
  T Dn[V], Ds[V], Ms[V], gan[V], gbn[V], gas[V], gbs[V];
  walk_dflux<T, V, true>(M, Dn, first, last, seg, gan, gbn);
#pragma unroll
  for (int v = 0; v < V; ++v) Ms[v] = fma_t(m.c1, Dn[v], fma_t(m.c2, M[v], c3));
  walk_dflux<T, V, true>(Ms, Ds, first, last, seg, gas, gbs);
  // lam_Mb** = f lam_Mb' + lam_C psi^{n+1} dtheta ds (through C and the scale-down)
  const T add = act ? lamC_c * psi1 * m.dth * m.ds : T(0);
  T y1[V], zs[V], y2[V], zn[V];
  T sy1 = T(0), sy2 = T(0);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    L[v] = f_c * L[v] + add;  // lam_Mb**
    y1[v] = m.dt * L[v];
    sy1 += y1[v];
  }
  walk_adj<T, V>(gas, gbs, y1, zs, first, last, seg, m.cw);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    zs[v] -= m.koff * y1[v];  // lam_Ms = J_R(Ms)^T y1
    acc.gk -= Ms[v] * y1[v];
    acc.gv = fma_t(Ds[v], y1[v], acc.gv);
    y2[v] = m.hdt * zs[v];
    sy2 += y2[v];
  }
  walk_adj<T, V>(gan, gbn, y2, zn, first, last, seg, m.cw);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    acc.gk -= M[v] * y2[v];
    acc.gv = fma_t(Dn[v], y2[v], acc.gv);
    const T lm = L[v] + zs[v] + zn[v] - m.koff * y2[v] + lnb;
    out.v[v] = lm;
    acc.D = fma_t(lm, M[v], acc.D);
  }
  if (act) {
    acc.lmf += m.kon * (sy1 + sy2);
    acc.gn += mf_n * (sy1 + sy2);
  }
  }
}

// In float32 the six float64 scalars are converted by one instruction for the
// warp (lane q converts value q, then shuffles), as in psi_adj_const; dt / 2
// is formed after the conversion (halving is exact either way). Called by the
// whole warp.
template <typename T>
__device__ __forceinline__ MotorConst<T> motor_const(const AdjArgs<T>& a) {
  MotorConst<T> m;
  if constexpr (sizeof(T) == 4) {
    const int lane = threadIdx.x & 31;
    const double v = lane == 0 ? *a.dt : lane == 1 ? a.cw : lane == 2 ? a.k_off
                   : lane == 3 ? a.k_on : lane == 4 ? a.ds : a.dth;
    const float x = (float)v;
    m.dt = __shfl_sync(0xffffffffu, x, 0);
    m.hdt = 0.5f * m.dt;
    m.cw = __shfl_sync(0xffffffffu, x, 1);
    m.koff = __shfl_sync(0xffffffffu, x, 2);
    m.kon = __shfl_sync(0xffffffffu, x, 3);
    m.ds = __shfl_sync(0xffffffffu, x, 4);
    m.dth = __shfl_sync(0xffffffffu, x, 5);
  } else {
    const double dt64 = *a.dt;
    m.dt = dt64;
    m.hdt = 0.5 * dt64;
    m.cw = a.cw;
    m.koff = a.k_off;
    m.kon = a.k_on;
    m.ds = a.ds;
    m.dth = a.dth;
  }
  m.c1 = m.hdt * m.cw;
  m.c2 = T(1) - m.hdt * m.koff;
  return m;
}

// End of a unit: its partial sums of lam_Mf and D.
template <typename T>
__device__ __forceinline__ void close_unit(const AdjArgs<T>& a, MotorAcc<T>& acc, int lane, int u,
                                           int cell) {
  const T lmf = warp_sum_t(acc.lmf);
  const T Dsum = warp_sum_t(acc.D);
  if (lane == 0) {
    a.lmf_out[(size_t)u * a.ncells + cell] = lmf;
    a.D_out[(size_t)u * a.ncells + cell] = Dsum;
  }
  acc.lmf = T(0);
  acc.D = T(0);
}

// The warp's parameter adjoints into its float64 slot (reduced over the warp
// in the state precision, then added in float64; dR/dv_walk = D / ds). Lane q
// adds parameter q, so each float64 operation is one instruction for all three.
template <typename T>
__device__ __forceinline__ void flush_params(const AdjArgs<T>& a, const MotorAcc<T>& acc, int lane,
                                             int gw) {
  const T gk = warp_sum_t(acc.gk), gv = warp_sum_t(acc.gv), gn = warp_sum_t(acc.gn);
  if (lane < 3) {
    const T x = lane == 0 ? gk : lane == 1 ? gv : gn;
    const double d = lane == 1 ? (double)x * a.inv_ds : (double)x;
    a.gpart[(size_t)gw * 4 + lane] += d;
  }
}

// Adjoint of one substep, part 2: Eq. 4 (midpoint RK2) on the rows, with the
// coupling through C and the scale-down, rows read with plain loads (any ns).
// One warp per (cell, block of rows_per_unit rows) unit, grid-stride; the
// items (unit, group of rows) of a warp form one flat loop whose loads run
// one item ahead. The unit's partial sums of lam_Mf and D go to slot u of the
// [units][cells] partials; the parameter adjoints accumulate per warp.
template <typename T, int V>
__global__ void __launch_bounds__(128, adj_min_blocks<T, V>()) k_adj_motor(const AdjArgs<T> a) {
  griddep_wait();
  const int nth = a.nth, ns = a.ns, seg = a.seg;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  const int U = a.units, RU = a.rows_per_unit;
  const int nunits = nc * U;
  int lgU = 0;
  while ((1 << lgU) < U) ++lgU;
  const int sl = lane & (seg - 1), rslot = lane / seg, rpp = 32 / seg;
  const int nl = ns / V;
  const bool first = sl == 0, last = sl == nl - 1, lane_ok = sl < nl;
  const MotorConst<T> m = motor_const(a);

  const int G = (RU + rpp - 1) / rpp;
  const int my_units = gw < nunits ? (nunits - 1 - gw) / W + 1 : 0;
  const int nitems = my_units * G;
  MotorAcc<T> acc{T(0), T(0), T(0), T(0), T(0)};
  T Mq[V], Lq[V], psiq = T(0), lnbq = T(0), mfq = T(0), lcq = T(0), fq = T(1);
  int q_unit = gw, q_g = 0;  // item whose loads are in flight
  auto load_item = [&]() {
    const int cell = q_unit >> lgU, u = q_unit & (U - 1);
    const int k0 = u * RU, k1 = min(nth, k0 + RU);
    const int k = k0 + q_g * rpp + rslot;
    const bool row_ok = k < k1, act = row_ok && lane_ok;
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
    psiq = row_ok ? a.psi_np[(size_t)cell * nth + k] : T(0);
    lnbq = row_ok ? a.lnb[(size_t)cell * nth + k] : T(0);
    if (q_g == 0) {
      mfq = a.mf_n[cell];
      lcq = a.cellc[(size_t)cell * 2];
      fq = a.cellc[(size_t)cell * 2 + 1];
    }
  };
  if (nitems > 0) load_item();
  T mf_n = T(0), c3 = T(0), lamC_c = T(0), f_c = T(1);
  for (int it = 0; it < nitems; ++it) {
    const int unit = q_unit, g = q_g;
    const int cell = unit >> lgU, u = unit & (U - 1);
    const int k0 = u * RU, k1 = min(nth, k0 + RU);
    const int k = k0 + g * rpp + rslot;
    const bool row_ok = k < k1, act = row_ok && lane_ok;
    const size_t off = ((size_t)cell * nth + (row_ok ? k : k0)) * ns + (size_t)sl * V;
    T M[V], L[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      M[v] = Mq[v];
      L[v] = Lq[v];
    }
    const T psi1 = psiq, lnb = lnbq;
    if (g == 0) {
      mf_n = mfq;
      c3 = m.hdt * m.kon * mf_n;
      lamC_c = lcq;
      f_c = fq;
    }
    if (++q_g == G) {
      q_g = 0;
      q_unit += W;
    }
    if (it + 1 < nitems) load_item();
    Pack<T, V> qo;
    motor_rows<T, V>(M, L, psi1, lnb, act, first, last, seg, m, c3, mf_n, lamC_c, f_c, acc, qo);
    if (act) *reinterpret_cast<Pack<T, V>*>(a.lmb + off) = qo;
    if (g == G - 1) close_unit(a, acc, lane, u, cell);
  }
  flush_params(a, acc, lane, gw);
}

// The same, with the rows streamed by bulk copies (needs 16-byte rows and
// columns: ns * sizeof(T) and RC * sizeof(T) multiples of 16). Each unit is
// CH chunks of RC rows; a chunk is one ring stage holding the rows of Mb^n and
// lam_Mb^{n+1} and the RC values of psi^{n+1} and lam_n_b of its rows, all
// completing on the stage's mbarrier; lane 0 keeps up to S chunks in flight
// ahead of the warp, across unit boundaries. The cell scalars of the next
// unit are loaded one unit ahead. Waits are bounded (DevParams::wait_limit);
// a warp whose wait runs out records the failure, drains its copies and
// leaves. Per-warp shared memory: S + 1 mbarriers and S stages.
template <typename T, int V>
__global__ void __launch_bounds__(128, adj_min_blocks<T, V>())
    k_adj_motor_ring(const AdjArgs<T> a, int RC, int CH, int S) {
  griddep_wait();
  extern __shared__ __align__(128) unsigned char ring_smem[];
  const int nth = a.nth, ns = a.ns, seg = a.seg;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int rows_elems = RC * ns;
  const size_t stage_bytes = (size_t)(2 * rows_elems + 2 * RC) * sizeof(T);
  const size_t bars_bytes = ((size_t)(S + 1) * 8 + 127) & ~(size_t)127;
  const size_t warp_bytes = bars_bytes + (size_t)S * stage_bytes;
  unsigned char* wbase = ring_smem + (size_t)wib * warp_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wbase);
  uint64_t* never = bars + S;
  unsigned char* stages = wbase + bars_bytes;

  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  const int U = a.units, RU = a.rows_per_unit;
  const int nunits = nc * U;
  int lgU = 0;
  while ((1 << lgU) < U) ++lgU;
  const int sl = lane & (seg - 1), rslot = lane / seg, rpp = 32 / seg;
  const int nl = ns / V;
  const bool first = sl == 0, last = sl == nl - 1, lane_ok = sl < nl;
  const MotorConst<T> m = motor_const(a);
  const uint32_t wait_limit = a.prm->wait_limit;
  const bool wait_never = (a.prm->debug_flags & 1u) != 0;

  const int my_units = gw < nunits ? (nunits - 1 - gw) / W + 1 : 0;
  const int nchunks = my_units * CH;
  const uint32_t rows_bytes = (uint32_t)(rows_elems * sizeof(T));
  const uint32_t col_bytes = (uint32_t)(RC * sizeof(T));

  // producer cursor (lane 0): unit and chunk of the next copy
  int p_unit = gw, p_c = 0, istage = 0, issued = 0;
  auto issue_next = [&]() {
    const int cell = p_unit >> lgU, u = p_unit & (U - 1);
    const int k = u * RU + p_c * RC;  // first row of the chunk
    const size_t roff = ((size_t)cell * nth + k) * ns;
    const size_t coff = (size_t)cell * nth + k;
    unsigned char* st = stages + (size_t)istage * stage_bytes;
    mbar_expect_tx(&bars[istage], 2 * rows_bytes + 2 * col_bytes);
    bulk_g2s(st, a.mb_n + roff, rows_bytes, &bars[istage]);
    bulk_g2s(st + rows_bytes, a.lmb + roff, rows_bytes, &bars[istage]);
    bulk_g2s(st + 2 * (size_t)rows_bytes, a.psi_np + coff, col_bytes, &bars[istage]);
    bulk_g2s(st + 2 * (size_t)rows_bytes + col_bytes, a.lnb + coff, col_bytes, &bars[istage]);
    ++issued;
    if (++p_c == CH) {
      p_c = 0;
      p_unit += W;
    }
    if (++istage == S) istage = 0;
  };
  if (lane == 0) {
    for (int q = 0; q <= S; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    while (issued < S && issued < nchunks) issue_next();
  }
  __syncwarp();

  MotorAcc<T> acc{T(0), T(0), T(0), T(0), T(0)};
  // cell scalars of the current and the next unit
  T mfq = T(0), lcq = T(0), fq = T(1);
  auto load_scalars = [&](int unit) {
    const int cell = unit >> lgU;
    mfq = a.mf_n[cell];
    lcq = a.cellc[(size_t)cell * 2];
    fq = a.cellc[(size_t)cell * 2 + 1];
  };
  if (my_units > 0) load_scalars(gw);
  int unit = gw - W, c = CH - 1, s = 0;
  uint32_t par = 0;
  bool timed_out = false;
  int fail_stage = 0, fail_left = 0;
  uint32_t fail_par = 0;
  T mf_n = T(0), c3 = T(0), lamC_c = T(0), f_c = T(1);
  for (int t = 0; t < nchunks; ++t) {
    if (++c == CH) {
      c = 0;
      unit += W;
      mf_n = mfq;
      c3 = m.hdt * m.kon * mf_n;
      lamC_c = lcq;
      f_c = fq;
      if (unit + W < nunits) load_scalars(unit + W);
    }
    const int cell = unit >> lgU, u = unit & (U - 1);
    const bool ok = __all_sync(0xffffffffu, wait_never ? mbar_wait(never, 0u, wait_limit)
                                                       : mbar_wait(&bars[s], par, wait_limit));
    if (!ok) {
      timed_out = true;
      fail_stage = s;
      fail_par = par;
      fail_left = issued - t;
      break;
    }
    const unsigned char* st = stages + (size_t)s * stage_bytes;
    const T* sM = reinterpret_cast<const T*>(st);
    const T* sL = reinterpret_cast<const T*>(st + rows_bytes);
    const T* sP = reinterpret_cast<const T*>(st + 2 * (size_t)rows_bytes);
    const T* sN = reinterpret_cast<const T*>(st + 2 * (size_t)rows_bytes + col_bytes);
    const int kc = u * RU + c * RC;  // first row of the chunk
    for (int p = 0; p * rpp < RC; ++p) {
      const int r = p * rpp + rslot;
      const bool row_ok = r < RC, act = row_ok && lane_ok;
      const int off = (row_ok ? r : 0) * ns + sl * V;
      T M[V], L[V];
      if (act) {
        const Pack<T, V> qm = *reinterpret_cast<const Pack<T, V>*>(sM + off);
        const Pack<T, V> ql = *reinterpret_cast<const Pack<T, V>*>(sL + off);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          M[v] = qm.v[v];
          L[v] = ql.v[v];
        }
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          M[v] = T(0);
          L[v] = T(0);
        }
      }
      const T psi1 = row_ok ? sP[r] : T(0);
      const T lnb = row_ok ? sN[r] : T(0);
      Pack<T, V> qo;
      motor_rows<T, V>(M, L, psi1, lnb, act, first, last, seg, m, c3, mf_n, lamC_c, f_c, acc, qo);
      if (act)
        *reinterpret_cast<Pack<T, V>*>(a.lmb + ((size_t)cell * nth + kc + r) * ns + sl * V) = qo;
    }
    __syncwarp();
    // the stage is consumed: refill it with the chunk S ahead
    if (lane == 0 && issued < nchunks) issue_next();
    if (++s == S) {
      s = 0;
      par ^= 1u;
    }
    if (c == CH - 1) close_unit(a, acc, lane, u, cell);
  }
  if (timed_out) {
    if (lane == 0) {
      atomicOr(&a.prm->status, 1);
      int st = fail_stage;
      uint32_t pp = fail_par;
      for (int i = 0; i < fail_left; ++i) {
        drain_wait(&bars[st], pp, &a.prm->status);
        if (++st == S) {
          st = 0;
          pp ^= 1u;
        }
      }
    }
    __syncwarp();
  }
  flush_params(a, acc, lane, gw);
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
                           int nth, int ns, double ds, double L, const T* trig, bool mb_seeded) {
  const int lane = threadIdx.x & 31;
  const long long gw = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  if (kind == 1 || (kind == 0 && !dnb && !dm1 && !mb_seeded)) {
    // no seed on the rows (lam_Mb was cleared by the caller, so D = 0): lanes
    // over theta for lam_psi
    for (long long cell = gw; cell < ncells; cell += W) {
      for (int k = lane; k < nth; k += 32) {
        const size_t r = (size_t)cell * nth + k;
        const double lp = kind == 1 ? coef[0] + coef[1] * (double)trig[k] +
                                          coef[2] * (double)trig[nth + k]
                                    : (dpsi ? dpsi[r] : 0.0);
        lpsi[r] = (T)lp;
      }
      if (lane == 0) {
        lmf[cell] = (T)((kind == 0 && dmf) ? dmf[cell] : 0.0);
        D[cell] = T(0);
      }
    }
    return;
  }
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
        // with a seed on the motor density itself, lam_Mb already holds it
        const double base = mb_seeded ? (double)lrow[j] : 0.0;
        const T lm = (T)(base + a_nb * ds + a_m1 * sj * ds);
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

// dL/dpsi0 = lam_psi^0 - lam_Mf^0 n_b^0 dtheta (Mf^0 = M - sum psi^0 n_b^0 dtheta),
// lam_Mf^0 the sum of its `units` partials.
template <typename T>
__global__ void k_adj_psi0(const T* lpsi, const T* lmf, int units, const T* nb, double dth,
                           long long rows, int nth, double* out) {
  const long long nc = rows / nth;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    const long long cell = r / nth;
    T l = T(0);
    for (int u = 0; u < units; ++u) l += lmf[u * nc + cell];
    out[r] = (double)lpsi[r] - (double)l * (double)nb[r] * dth;
  }
}

// Seed coefficients of a built-in observable (one thread).
__global__ void k_adj_observable(int kind, const DevParams* prm, double stress_coef,
                                 double* coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double c0 = 0.0, c1 = 0.0, c2 = 0.0, v = 0.0;
  if (kind == 1) {
    // L = |P| / S, P = sum psi e^{i theta}, S = sum psi
    const double px = prm->scalars[6], py = prm->scalars[7], S = prm->sum_psi;
    const double pn = sqrt(px * px + py * py);
    v = pn / S;
    c0 = -v / S;
    c1 = pn > 0.0 ? px / pn / S : 0.0;
    c2 = pn > 0.0 ? py / pn / S : 0.0;
  } else if (kind == 2) {
    v = prm->scalars[5];
    c0 = stress_coef;
  }
  coef[0] = c0;
  coef[1] = c1;
  coef[2] = c2;
  coef[3] = v;
}

// Sum of the per-warp parameter adjoints in warp order (one warp).
__global__ void k_adj_params(const double* gpart, int nwarps, double* out) {
  const int lane = threadIdx.x & 31;
  double g[3] = {0.0, 0.0, 0.0};
  for (int w = lane; w < nwarps; w += 32)
    for (int q = 0; q < 3; ++q) g[q] += gpart[(size_t)w * 4 + q];
  for (int q = 0; q < 3; ++q) {
    const double r = warp_sum(g[q]);
    if (lane == 0) out[q] = r;
  }
}

}  // namespace

cudaError_t launch_adj_observable(int kind, const DevParams* prm, double stress_coef, double* coef,
                                  cudaStream_t s) {
  k_adj_observable<<<1, 32, 0, s>>>(kind, prm, stress_coef, coef);
  return cudaGetLastError();
}

cudaError_t launch_adj_params(const double* gpart, int nwarps, double* out, cudaStream_t s) {
  k_adj_params<<<1, 32, 0, s>>>(gpart, nwarps, out);
  return cudaGetLastError();
}

// Shared memory per warp of the ring kernel.
size_t adj_ring_warp_bytes(int rc, int ns, int S, int tsz) {
  const size_t bars = ((size_t)(S + 1) * 8 + 127) & ~(size_t)127;
  return bars + (size_t)S * (size_t)(2 * rc * ns + 2 * rc) * tsz;
}

// Resident 4-warp blocks per SM of the motor kernel the plan will launch.
template <typename T>
cudaError_t adj_motor_occupancy(int V, int ring_rc, int ns, int S, int* bps) {
  const size_t rs =
      ring_rc > 0 ? 4 * adj_ring_warp_bytes(ring_rc, ns, S, (int)sizeof(T)) : 0;
  auto occ = [&](auto plain, auto ring) -> cudaError_t {
    if (ring_rc > 0) {
      cudaError_t e = mm::raise_smem_limit(ring, (int)rs);
      if (e != cudaSuccess) return e;
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, ring, 128, rs);
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, plain, 128, 0);
  };
  if constexpr (sizeof(T) == 4)
    if (V == 8) return occ(k_adj_motor<T, 8>, k_adj_motor_ring<T, 8>);
  if (V == 4) return occ(k_adj_motor<T, 4>, k_adj_motor_ring<T, 4>);
  if (V == 2) return occ(k_adj_motor<T, 2>, k_adj_motor_ring<T, 2>);
  return occ(k_adj_motor<T, 1>, k_adj_motor_ring<T, 1>);
}

template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T>& a, int V, int grid_psi, int grid_motor,
                           cudaStream_t s) {
  const int block = 128;
  const size_t ring_smem = 4 * psi_ring_warp_bytes(a.nth, (int)sizeof(T));
  if ((a.nth * sizeof(T)) % 16 == 0 && ring_smem <= 200 * 1024) {
    if (ring_smem > 48 * 1024) {
      cudaError_t e = mm::raise_smem_limit(k_adj_psi_ring<T>, (int)ring_smem);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e0 = launch_overlapped(k_adj_psi_ring<T>, grid_psi, block, ring_smem, s, a);
    if (e0 != cudaSuccess) return e0;
  } else {
    const size_t smem = (size_t)4 * a.nth * sizeof(T);
    if (smem > 48 * 1024) {
      cudaError_t e = mm::raise_smem_limit(k_adj_psi<T>, (int)smem);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e0 = launch_overlapped(k_adj_psi<T>, grid_psi, block, smem, s, a);
    if (e0 != cudaSuccess) return e0;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto go = [&](auto plain, auto ring) -> cudaError_t {
    if (a.ring_rc > 0) {
      const size_t rs = 4 * adj_ring_warp_bytes(a.ring_rc, a.ns, a.ring_s, (int)sizeof(T));
      if (rs > 48 * 1024) {
        cudaError_t e2 =
            mm::raise_smem_limit(ring, (int)rs);
        if (e2 != cudaSuccess) return e2;
      }
      cudaError_t e1 =
          launch_overlapped(ring, grid_motor, block, rs, s, a, a.ring_rc, a.ring_ch, a.ring_s);
      if (e1 != cudaSuccess) return e1;
    } else {
      cudaError_t e1 = launch_overlapped(plain, grid_motor, block, (size_t)0, s, a);
      if (e1 != cudaSuccess) return e1;
    }
    return cudaGetLastError();
  };
  if constexpr (sizeof(T) == 4)
    if (V == 8) return go(k_adj_motor<T, 8>, k_adj_motor_ring<T, 8>);
  if (V == 4) return go(k_adj_motor<T, 4>, k_adj_motor_ring<T, 4>);
  if (V == 2) return go(k_adj_motor<T, 2>, k_adj_motor_ring<T, 2>);
  return go(k_adj_motor<T, 1>, k_adj_motor_ring<T, 1>);
}

template <typename T>
cudaError_t launch_adj_seed(int kind, const double* coef, const T* psi, const T* mb,
                            const double* dpsi, const double* dnb, const double* dm1,
                            const double* dmf, T* lpsi, T* lmb, T* lmf, T* D, long long ncells,
                            int nth, int ns, double ds, double L, const T* trig, bool mb_seeded,
                            cudaStream_t s) {
  long long g = (ncells + 3) / 4;
  if (g > 152 * 8) g = 152 * 8;
  if (kind == 1 || (kind == 0 && !dnb && !dm1 && !mb_seeded)) {
    // a seed without motor rows: lam_Mb = 0 by a fill, the kernel skips the rows
    const cudaError_t e = cudaMemsetAsync(lmb, 0, (size_t)ncells * nth * ns * sizeof(T), s);
    if (e != cudaSuccess) return e;
  }
  k_adj_seed<T><<<(int)g, 128, 0, s>>>(kind, coef, psi, mb, dpsi, dnb, dm1, dmf, lpsi, lmb, lmf,
                                       D, ncells, nth, ns, ds, L, trig, mb_seeded);
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
cudaError_t launch_adj_psi0(const T* lpsi, const T* lmf, int units, const T* nb, double dth,
                            long long rows, int nth, double* out, cudaStream_t s) {
  long long g = (rows + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_adj_psi0<T><<<(int)g, 256, 0, s>>>(lpsi, lmf, units, nb, dth, rows, nth, out);
  return cudaGetLastError();
}

#define MM_ADJ_INST(T)                                                                          \
  template cudaError_t launch_adjoint<T>(const AdjArgs<T>&, int, int, int, cudaStream_t);       \
  template cudaError_t adj_motor_occupancy<T>(int, int, int, int, int*);                        \
  template cudaError_t launch_adj_seed<T>(int, const double*, const T*, const T*, const double*, \
                                          const double*, const double*, const double*, T*, T*,  \
                                          T*, T*, long long, int, int, double, double, const T*, \
                                          bool, cudaStream_t);                                  \
  template cudaError_t launch_adj_psi0<T>(const T*, const T*, int, const T*, double, long long,  \
                                          int, double*, cudaStream_t);
MM_ADJ_INST(float)
MM_ADJ_INST(double)

}  // namespace mm
