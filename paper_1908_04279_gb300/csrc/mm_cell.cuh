// Device pieces of the fused substep shared by the single-instance kernel
// (mm_step.cu) and the batched-ensemble kernel (mm_batch.cu): the bulk-copy
// and mbarrier primitives, the per-warp shared-memory plan, one chunk of
// s-rows by Eq. 4 (midpoint RK2 of Alg. 2) and the end-of-cell update of psi
// by Eq. 1 with the coarse density of Eq. 5.
#pragma once

#include <cstddef>

#include "mm_internal.cuh"
#include "mm_walk.cuh"

namespace mm {

// ---------------------------------------------------------------- TMA / mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i >= limit) return false;
  }
}

constexpr uint32_t kDrainLimit = 1u << 24;  // polls while draining after a timeout

// After a timeout: wait (bounded) for a copy still in flight into this block's
// shared memory. If that wait gives up too, the copy may land after the block
// has left, in shared memory the next block on the SM may own: status bit 3
// records it, so the host can report that later launches are suspect too.
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity, int* status) {
  if (!mbar_wait(bar, parity, kDrainLimit)) atomicOr(status, 8);
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}


// Occupancy target (resident 4-warp blocks per SM, caps registers per thread)
// and unroll depth of the s-row pass loop.
#ifndef MM_STEP_MIN_BLOCKS
#define MM_STEP_MIN_BLOCKS 4
#endif
#ifndef MM_STEP_UNROLL
#define MM_STEP_UNROLL 2
#endif
constexpr int kStepUnroll = MM_STEP_UNROLL;

// ------------------------------------------------------------------- layout

// Per-warp shared memory: S + 2 mbarriers (S ring stages, 1 neighbourhood, 1
// that never completes, waited on by the timeout test knob), S stages of
// chunk_elems values, the psi and n_b columns of the cell and its east, west,
// north and south neighbours (2 x 5 nth values), and n_b of the cell's new
// rows (nth values), all in the state precision.
struct WarpSmem {
  size_t bars, stages, psi5, nb5, nbm, total;
};
__host__ __device__ inline WarpSmem warp_smem_layout(int S, int chunk_elems, int nth, int tsz) {
  WarpSmem w;
  w.bars = 0;
  size_t off = 8 * (size_t)(S + 2);
  off = (off + 127) & ~(size_t)127;
  w.stages = off;
  off += (size_t)S * chunk_elems * tsz;
  off = (off + 15) & ~(size_t)15;
  w.psi5 = off;
  off += 5 * (size_t)nth * tsz;
  off = (off + 15) & ~(size_t)15;
  w.nb5 = off;
  off += 5 * (size_t)nth * tsz;
  off = (off + 15) & ~(size_t)15;
  w.nbm = off;
  off += (size_t)nth * tsz;
  off = (off + 127) & ~(size_t)127;
  w.total = off;
  return w;
}

// ------------------------------------------------------------ launch scalars

// The scalars of a substep in the state precision: dt and dt / 2, the psi
// correction factor g (1 without mass correction), k_on, k_off, glide, v_sp,
// v/ds and the grid spacings. In float32 the seven float64 scalars of
// DevParams (dt, psi_scale, k_on, k_off, glide, v_sp, cw) are converted by one
// instruction for the whole warp -- lane q converts scalar q, the lanes then
// exchange them by shuffles -- because conversions from float64 run on the
// narrow float64 pipe; the spacings arrive converted in the launch arguments.
template <typename T>
struct StepScalars {
  T dt, hdt, g, kon, koff, glide, vsp, cw, inv_dx, inv_dy, inv_dth, dth, ds;
};
template <typename T, bool MASSCORR>
__device__ __forceinline__ StepScalars<T> step_scalars(const DevParams* P, const StepArgs<T>& a,
                                                       int lane) {
  StepScalars<T> s;
  if constexpr (sizeof(T) == 4) {
    const double* pd = reinterpret_cast<const double*>(P);
    constexpr int kCw = (int)(offsetof(DevParams, cw) / sizeof(double));
    static_assert(offsetof(DevParams, psi_scale) == 8 && offsetof(DevParams, k_on) == 40 &&
                      offsetof(DevParams, v_sp) == 64,
                  "lane q reads the q-th of dt, psi_scale, k_on, k_off, glide, v_sp");
    const int idx = lane < 2 ? lane : (lane < 6 ? lane + 3 : kCw);
    const float x = lane < 7 ? (float)pd[idx] : 0.0f;
    s.dt = __shfl_sync(0xffffffffu, x, 0);
    s.g = MASSCORR ? __shfl_sync(0xffffffffu, x, 1) : 1.0f;
    s.kon = __shfl_sync(0xffffffffu, x, 2);
    s.koff = __shfl_sync(0xffffffffu, x, 3);
    s.glide = __shfl_sync(0xffffffffu, x, 4);
    s.vsp = __shfl_sync(0xffffffffu, x, 5);
    s.cw = __shfl_sync(0xffffffffu, x, 6);
    s.hdt = 0.5f * s.dt;  // = (float)(dt / 2): halving commutes with the rounding
    s.inv_dx = a.f_inv_dx;
    s.inv_dy = a.f_inv_dy;
    s.inv_dth = a.f_inv_dth;
    s.dth = a.f_dth;
    s.ds = a.f_ds;
  } else {
    s.dt = P->dt;
    s.hdt = 0.5 * P->dt;
    s.g = MASSCORR ? P->psi_scale : 1.0;
    s.kon = P->k_on;
    s.koff = P->k_off;
    s.glide = P->glide;
    s.vsp = P->v_sp;
    s.cw = P->cw;
    s.inv_dx = a.inv_dx;
    s.inv_dy = a.inv_dy;
    s.inv_dth = a.inv_dth;
    s.dth = a.dth;
    s.ds = a.ds;
  }
  return s;
}

// Sum over the warp of a float-float pair (compensated: TwoSum at every level),
// returned as float64 in every lane.
__device__ __forceinline__ double warp_sum_ff(float hi, float lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = hi + h2, bb = s - hi;
    lo = (lo + l2) + ((hi - (s - bb)) + (h2 - bb));
    hi = s;
  }
  return (double)hi + (double)lo;
}
__device__ __forceinline__ double warp_sum_ff(double hi, double lo) {
  return warp_sum(hi + lo);
}

// ------------------------------------------------------------- s-row chunk

// Where a lane sits in the s-rows of a pass: `seg` lanes per row (V nodes
// each), rpp = 32 / seg rows per pass.
struct LaneGeom {
  int sl, rslot, rpp;
  bool first, last, lane_ok;
};
__device__ __forceinline__ LaneGeom lane_geom(int lane, int seg, int ns, int V) {
  LaneGeom g;
  g.sl = lane & (seg - 1);
  g.rslot = lane / seg;
  g.rpp = 32 / seg;
  const int nl = ns / V;
  g.first = g.sl == 0;
  g.last = g.sl == nl - 1;
  g.lane_ok = g.sl < nl;
  return g;
}

// RK2 constants of one cell: Eq. 4's right-hand side is
// R = (v/ds) D - k_off M + k_on Mf; the half step is
// Ms = c1 D(M) + c2 M + c3 and the full step M' = e1 D(Ms) + e2 Ms + M + e3.
// With SPLIT (rows_chunk), rows from rsplit on take c3b and e3b instead: the
// rows of a second cell, with its own Mf, in the same chunk.
template <typename T>
struct RkConst {
  T c1, c2, c3, e1, e2, e3;
  T c3b, e3b;
  int rsplit;
};

// Float32 rows with V = 4 or 8 nodes per lane as register pairs: the stage
// updates and the n_b sum as packed two-value instructions (walk_dflux_x2).
template <int V, bool SPLIT = false>
__device__ __forceinline__ void rows_chunk_x2(const float* src_rows, float* dst, int RC, int ns,
                                              int seg, const LaneGeom& lg,
                                              const RkConst<float>& k, float ds,
                                              float* s_nb_chunk) {
  constexpr int H = V / 2;
  const int passes = (RC + lg.rpp - 1) / lg.rpp;
  const float2 c1 = make_float2(k.c1, k.c1), c2 = make_float2(k.c2, k.c2);
  const float2 e1 = make_float2(k.e1, k.e1), e2 = make_float2(k.e2, k.e2);
#pragma unroll kStepUnroll
  for (int p = 0; p < passes; ++p) {
    const int r = p * lg.rpp + lg.rslot;  // row within the chunk
    const bool hi = SPLIT && r >= k.rsplit;
    const float c3s = hi ? k.c3b : k.c3, e3s = hi ? k.e3b : k.e3;
    const float2 c3 = make_float2(c3s, c3s), e3 = make_float2(e3s, e3s);
    const bool row_ok = r < RC;
    const bool act = row_ok && lg.lane_ok;
    const int off = (row_ok ? r : 0) * ns + lg.sl * V;
    float2 M[H], D[H], Ms[H];
    if (act) {
      const float4* q = reinterpret_cast<const float4*>(src_rows + off);
#pragma unroll
      for (int h = 0; h < H / 2; ++h) {
        const float4 v4 = q[h];
        M[2 * h] = make_float2(v4.x, v4.y);
        M[2 * h + 1] = make_float2(v4.z, v4.w);
      }
    } else {
#pragma unroll
      for (int h = 0; h < H; ++h) M[h] = make_float2(0.0f, 0.0f);
    }
    walk_dflux_x2<V>(M, D, lg.first, lg.last, seg);
#pragma unroll
    for (int h = 0; h < H; ++h) Ms[h] = __ffma2_rn(c1, D[h], __ffma2_rn(c2, M[h], c3));
    walk_dflux_x2<V>(Ms, D, lg.first, lg.last, seg);
#pragma unroll
    for (int h = 0; h < H; ++h)
      M[h] = __ffma2_rn(e1, D[h], __ffma2_rn(e2, Ms[h], __fadd2_rn(M[h], e3)));
    float2 acc = M[0];
#pragma unroll
    for (int h = 1; h < H; ++h) acc = __fadd2_rn(acc, M[h]);
    float snb = act ? acc.x + acc.y : 0.0f;
    if (act) {
      float4* q = reinterpret_cast<float4*>(dst + off);
#pragma unroll
      for (int h = 0; h < H / 2; ++h)
        q[h] = make_float4(M[2 * h].x, M[2 * h].y, M[2 * h + 1].x, M[2 * h + 1].y);
    }
    snb = seg_sum(snb, seg);
    if (lg.first && row_ok) s_nb_chunk[r] = snb * ds;
  }
}

// One chunk of RC s-rows (src_rows: the rows at step n, in shared or global
// memory; dst: global rows at step n+1, in place allowed), with n_b of each
// new row written to s_nb_chunk[r].
template <typename T, int V, bool SPLIT = false>
__device__ __forceinline__ void rows_chunk(const T* src_rows, T* dst, int RC, int ns, int seg,
                                           const LaneGeom& lg, const RkConst<T>& k, T ds,
                                           T* s_nb_chunk) {
  if constexpr (sizeof(T) == 4 && (V == 4 || V == 8)) {
    rows_chunk_x2<V, SPLIT>(src_rows, dst, RC, ns, seg, lg, k, ds, s_nb_chunk);
    return;
  }
  const int passes = (RC + lg.rpp - 1) / lg.rpp;
#pragma unroll kStepUnroll
  for (int p = 0; p < passes; ++p) {
    const int r = p * lg.rpp + lg.rslot;  // row within the chunk
    const bool hi = SPLIT && r >= k.rsplit;
    const T c3 = hi ? k.c3b : k.c3, e3 = hi ? k.e3b : k.e3;
    const bool row_ok = r < RC;
    const bool act = row_ok && lg.lane_ok;
    const int off = (row_ok ? r : 0) * ns + lg.sl * V;
    T M[V], D[V], Ms[V];
    if (act) {
      const Pack<T, V> q = *reinterpret_cast<const Pack<T, V>*>(src_rows + off);
#pragma unroll
      for (int v = 0; v < V; ++v) M[v] = q.v[v];
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) M[v] = T(0);
    }
    // midpoint RK2 with the constants folded
    walk_dflux<T, V>(M, D, lg.first, lg.last, seg);
#pragma unroll
    for (int v = 0; v < V; ++v) Ms[v] = fma_t(k.c1, D[v], fma_t(k.c2, M[v], c3));
    walk_dflux<T, V>(Ms, D, lg.first, lg.last, seg);
    T snb = T(0);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      M[v] = fma_t(k.e1, D[v], fma_t(k.e2, Ms[v], add_rn(M[v], e3)));
      snb += M[v];
    }
    if (!act) snb = T(0);
    if (act) {
      Pack<T, V> q;
#pragma unroll
      for (int v = 0; v < V; ++v) q.v[v] = M[v];
      *reinterpret_cast<Pack<T, V>*>(dst + off) = q;
    }
    snb = seg_sum(snb, seg);
    if (lg.first && row_ok) s_nb_chunk[r] = snb * ds;
  }
}

// The psi and n_b columns of a cell and its east, west, north and south
// neighbours into psi5 / nb5 ([5][nth]), completing on `nbar`: lane 0 posts
// the expected bytes, then lanes 0-9 each issue one of the 10 bulk copies.
template <typename T>
__device__ __forceinline__ void stage_neighbourhood(uint64_t* nbar, T* psi5, T* nb5,
                                                    const T* psi_in, const T* nb_in, int c0,
                                                    int c1, int c2, int c3, int c4, int nth,
                                                    int lane) {
  const uint32_t pb = (uint32_t)(nth * sizeof(T));
  if (lane == 0) mbar_expect_tx(nbar, 10 * pb);
  __syncwarp();
  if (lane < 10) {
    const int q = lane >> 1;
    const int cq = q == 0 ? c0 : q == 1 ? c1 : q == 2 ? c2 : q == 3 ? c3 : c4;
    if (lane & 1)
      bulk_g2s(nb5 + q * nth, nb_in + (size_t)cq * nth, pb, nbar);
    else
      bulk_g2s(psi5 + q * nth, psi_in + (size_t)cq * nth, pb, nbar);
  }
}

// ------------------------------------------------------------ end of a cell

// Velocity data of one cell: the cell's own and its east/west (x) and
// north/south (y) neighbours' velocities and the central-difference gradient.
template <typename T>
struct CellVel {
  T uxc, uyc, uxe, uxw, uyn, uys, Gxx, Gxy, Gyx, Gyy;
};
template <typename T>
__device__ __forceinline__ CellVel<T> load_cell_vel(const T* ucell, int cell) {
  const T* uc = ucell + (size_t)cell * 12;
  CellVel<T> u;
  u.uxc = uc[0]; u.uyc = uc[1]; u.uxe = uc[2]; u.uxw = uc[3]; u.uyn = uc[4]; u.uys = uc[5];
  u.Gxx = uc[6]; u.Gxy = uc[7]; u.Gyx = uc[8]; u.Gyy = uc[9];
  return u;
}

// Constants of the psi transport of one instance.
template <typename T>
struct PsiConst {
  T dt, g, glide, vsp, inv_dx, inv_dy, inv_dth, dth;
  const T* trig;  // [4][nth]
};

// psi^{n+1} of the cell (lane = theta) by Eq. 1 in donor-cell flux form from
// the staged columns psi5 / nb5 ([5][nth]: cell, east, west, north, south;
// psi scaled by g on load), written to psi_out[cell]. Returns, per lane, the
// partial sums of psi^{n+1} (cell_mass) and of psi^{n+1} n_b dtheta (the
// coarse density of Eq. 5, acc) over the lane's orientations.
// Trigonometric values of the orientation a lane handles when nth <= 32
// (k = lane): cos, sin of theta_k and of the faces theta_{k +- 1/2}.
template <typename T>
struct LaneTrig {
  T ck, sk, cp, sp, cm, sm;
};
template <typename T>
__device__ __forceinline__ LaneTrig<T> lane_trig(const T* trig, int nth, int lane) {
  LaneTrig<T> t{};
  if (lane < nth) {
    const int km = lane == 0 ? nth - 1 : lane - 1;
    t.ck = trig[lane];
    t.sk = trig[nth + lane];
    t.cp = trig[2 * nth + lane];
    t.sp = trig[3 * nth + lane];
    t.cm = trig[2 * nth + km];
    t.sm = trig[3 * nth + km];
  }
  return t;
}

template <typename T>
__device__ __forceinline__ void psi_cell(const PsiConst<T>& q, const CellVel<T>& u,
                                         const T* psi5, const T* nb5, const T* s_nb, int nth,
                                         int lane, T* psi_out_cell, T& cell_mass, T& acc,
                                         const LaneTrig<T>* lt = nullptr) {
  const T* cosk = q.trig;
  const T* sink = q.trig + nth;
  const T* cosf = q.trig + 2 * nth;
  const T* sinf = q.trig + 3 * nth;
  const T g = q.g;
  const bool cached = lt != nullptr && nth <= 32;
  for (int k = lane; k < nth; k += 32) {
    const T Pc = g * psi5[k], Pe = g * psi5[nth + k], Pw = g * psi5[2 * nth + k];
    const T Pn = g * psi5[3 * nth + k], Ps = g * psi5[4 * nth + k];
    const T ck = cached ? lt->ck : cosk[k], sk = cached ? lt->sk : sink[k];
    // (every sum of products below is written as explicit fused operations,
    // so that each kernel inlining this function rounds it the same way)
    const T Vc = fma_t(q.glide, nb5[k], q.vsp), Ve = fma_t(q.glide, nb5[nth + k], q.vsp);
    const T Vw = fma_t(q.glide, nb5[2 * nth + k], q.vsp);
    const T Vn = fma_t(q.glide, nb5[3 * nth + k], q.vsp);
    const T Vs = fma_t(q.glide, nb5[4 * nth + k], q.vsp);
    const T axc = fma_t(-Vc, ck, u.uxc), axe = fma_t(-Ve, ck, u.uxe), axw = fma_t(-Vw, ck, u.uxw);
    const T ayc = fma_t(-Vc, sk, u.uyc), ayn = fma_t(-Vn, sk, u.uyn), ays = fma_t(-Vs, sk, u.uys);
    const T Ae = T(0.5) * (axc + axe), Aw = T(0.5) * (axw + axc);
    const T An = T(0.5) * (ayc + ayn), As = T(0.5) * (ays + ayc);
    const int kp = k + 1 == nth ? 0 : k + 1, km = k == 0 ? nth - 1 : k - 1;
    const T cp = cached ? lt->cp : cosf[k], sp = cached ? lt->sp : sinf[k];
    const T cm = cached ? lt->cm : cosf[km], sm = cached ? lt->sm : sinf[km];
    // Jeffery rotation p_perp . G . p at the faces k +- 1/2
    const T wp = fma_t(-sp, fma_t(u.Gxx, cp, u.Gxy * sp), cp * fma_t(u.Gyx, cp, u.Gyy * sp));
    const T wm = fma_t(-sm, fma_t(u.Gxx, cm, u.Gxy * sm), cm * fma_t(u.Gyx, cm, u.Gyy * sm));
    const T Fe = donor(Ae, Pc, Pe), Fw = donor(Aw, Pw, Pc);
    const T Fn = donor(An, Pc, Pn), Fs = donor(As, Ps, Pc);
    const T Fp = donor(wp, Pc, g * psi5[kp]), Fm = donor(wm, g * psi5[km], Pc);
    const T div =
        fma_t(Fp - Fm, q.inv_dth, fma_t(Fn - Fs, q.inv_dy, (Fe - Fw) * q.inv_dx));
    const T pnew = fma_t(-q.dt, div, Pc);
    psi_out_cell[k] = pnew;
    cell_mass += pnew;
    acc = fma_t(pnew * s_nb[k], q.dth, acc);
  }
}

// TwoSum: hi + lo += x without rounding loss.
template <typename T>
__device__ __forceinline__ void two_sum_acc(T& hi, T& lo, T x) {
  const T s2 = hi + x, bb = s2 - hi;
  lo += (hi - (s2 - bb)) + (x - bb);
  hi = s2;
}

// Eq. 5 to Eq. 6 for the cell: the coarse density Cpre = sum_k psi n_b dtheta,
// the scale-down of Alg. 2 where the total motors fall short (the warp
// rescales the rows it has just written), n_b of the new rows, C and Mf.
template <typename T>
__device__ __forceinline__ void cell_motor_close(T acc, T mtot, const T* s_nb, int nth, int ns,
                                                 int lane, int cell, T* mb_out, T* nb_out, T* c,
                                                 T* mf_out, T* cpre_out) {
  const T Cpre = warp_sum_t(acc);
  T f = T(1), C = Cpre;
  if (mtot < Cpre) {
    f = mtot / Cpre;
    C = mtot;
  }
  const size_t cbase = (size_t)cell * nth;
  if (f != T(1)) {
    const T ft = f;
    T* base = mb_out + cbase * ns;
    for (int e = lane; e < nth * ns; e += 32) base[e] = __ldcg(base + e) * ft;
    for (int k = lane; k < nth; k += 32) nb_out[cbase + k] = s_nb[k] * ft;
  } else {
    for (int k = lane; k < nth; k += 32) nb_out[cbase + k] = s_nb[k];
  }
  if (lane == 0) {
    c[cell] = C;
    mf_out[cell] = mtot - C;
    if (cpre_out) cpre_out[cell] = Cpre;
  }
}

}  // namespace mm
