// Fused microscale substep kernel (forward), warp-per-cell with a TMA ring.
//
// Every warp owns whole spatial cells (cells gw, gw + W, gw + 2W, ... for
// global warp gw of W) and performs the whole substep for each of them, with
// no block-level barrier:
//   1. every s-row Mb(cell, k, :) by Eq. 4 with midpoint RK2 (Alg. 2 half and
//      full stage). The cell's rows stream through a ring of shared-memory
//      stages filled by bulk asynchronous copies (cp.async.bulk, the Tensor
//      Memory Accelerator) that complete on mbarriers; lane 0 keeps up to S
//      chunks in flight ahead of the warp. A row is spread over `seg` lanes
//      with V consecutive s-nodes per lane; the Superbee stencil reaches across
//      lanes with warp shuffles; the new row goes straight back to global
//      memory in place (16-byte vector stores);
//   2. n_b and the force dipole m1 of every row by a shuffle reduction over s;
//   3. psi^{n+1}(cell, :) by Eq. 1 in donor-cell flux form (lane = theta), from
//      psi^n and n_b^n of the cell and its 4 neighbours (loaded when the cell
//      starts, so their latency overlaps the motor rows);
//   4. the coarse density C = sum_k psi^{n+1} n_b dtheta (Eq. 5) by a warp
//      reduction, the scale-down of Alg. 2 (rare: the warp rescales the rows
//      it has just written) and Mf = M - C (Eq. 6).
// psi and n_b are double-buffered (neighbour cells read the old values); Mb,
// Mf and C are cell-local. Each warp also sums psi^{n+1} in float64; the last
// warp to finish adds the per-warp sums in a fixed order and, in the float32
// form, stores the mass-correction factor applied to psi on the next load.
//
// Every mbarrier wait is bounded (DevParams::wait_limit polls). A warp whose
// wait runs out records MM_ERR_TIMEOUT in DevParams::status, waits (bounded)
// for the copies it still has in flight and leaves.
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

// Donor-cell face flux: upwind state times face velocity, with an explicit fma
// so that both cells sharing a face compute the same bits (exact telescoping).
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
__device__ __forceinline__ T seg_sum(T x, int seg) {
  for (int o = seg >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, seg);
  return x;
}
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

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

constexpr uint32_t kDrainLimit = 1u << 24;  // polls while draining after a timeout

// ------------------------------------------------------------------- layout

// Per-warp shared memory: S + 2 mbarriers (S ring stages, 1 neighbourhood, 1
// that never completes, waited on by the timeout test knob),
// S stages of chunk_elems values, the psi columns of the cell and its east,
// west, north and south neighbours (5 nth values of T), their n_b columns
// (5 nth doubles), and n_b, m1 of the cell's new rows (2 nth doubles).
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
  off += 5 * (size_t)nth * 8;
  w.nbm = off;
  off += 2 * (size_t)nth * 8;
  off = (off + 127) & ~(size_t)127;
  w.total = off;
  return w;
}

size_t step_smem_per_warp(int S, int chunk_elems, int nth, int tsz) {
  return warp_smem_layout(S, chunk_elems, nth, tsz).total;
}

template <typename T, int V, bool TMA, bool MASSCORR>
__global__ void __launch_bounds__(128, 4) k_substep(const StepArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nth = a.nth, ns = a.ns, seg = a.seg;
  const int S = a.stages, RC = a.chunk_rows, CH = a.chunks_per_cell;
  const int chunk_elems = RC * ns;
  // the ring exists only with bulk copies (the host sizes shared memory alike)
  const WarpSmem L = warp_smem_layout(S, TMA ? chunk_elems : 0, nth, (int)sizeof(T));
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* wbase = smem_raw + (size_t)wib * L.total;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + L.bars);
  T* stages = reinterpret_cast<T*>(wbase + L.stages);
  T* psi5 = reinterpret_cast<T*>(wbase + L.psi5);          // [5][nth]: c, e, w, n, s
  double* nb5 = reinterpret_cast<double*>(wbase + L.nb5);  // [5][nth]
  double* s_nb = reinterpret_cast<double*>(wbase + L.nbm);
  double* s_m1 = s_nb + nth;
  uint64_t* nbar = bars + S;      // neighbourhood barrier
  uint64_t* never = bars + S + 1;  // no copy or arrival ever completes it
  const bool nb_tma = TMA && a.nb_tma;

  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const long long nc = a.ncells;
  const long long my_cells = gw < nc ? (nc - 1 - gw) / W + 1 : 0;
  const long long nchunks = my_cells * CH;

  const int sl = lane & (seg - 1);      // lane within its row
  const int rslot = lane / seg;         // row within a pass
  const int rpp = 32 / seg;             // rows per pass
  const int passes = (RC + rpp - 1) / rpp;
  const int nl = ns / V;
  const bool first = sl == 0, last = sl == nl - 1, lane_ok = sl < nl;

  const DevParams* P = a.prm;
  const double dt64 = P->dt;
  const T dt = (T)dt64, hdt = (T)(0.5 * dt64);
  const T cw = (T)(P->v_walk / a.ds);
  const T koff = (T)P->k_off;
  const double kon64 = P->k_on;
  const T glide = (T)P->glide, vsp = (T)P->v_sp;
  const T g = MASSCORR ? (T)P->psi_scale : T(1);
  const uint32_t wait_limit = P->wait_limit;
  const bool wait_never = (P->debug_flags & 1u) != 0;  // test knob: every wait runs out
  const T inv_dx = (T)a.inv_dx, inv_dy = (T)a.inv_dy, inv_dth = (T)a.inv_dth;
  const T* cosk = a.trig;
  const T* sink = a.trig + nth;
  const T* cosf = a.trig + 2 * nth;
  const T* sinf = a.trig + 3 * nth;

  T sj[V];
#pragma unroll
  for (int v = 0; v < V; ++v) sj[v] = (T)(-0.5 * a.L + ((double)(sl * V + v) + 0.5) * a.ds);

  auto chunk_src = [&](long long t) -> const T* {
    const long long cell = gw + (t / CH) * (long long)W;
    const int part = (int)(t % CH);
    return a.mb + ((size_t)cell * nth + (size_t)part * RC) * ns;
  };

  if (TMA) {
    if (lane == 0) {
      for (int s = 0; s <= S + 1; ++s) mbar_init(&bars[s], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      for (int s = 0; s < S && s < nchunks; ++s) {
        mbar_expect_tx(&bars[s], (uint32_t)(chunk_elems * sizeof(T)));
        bulk_g2s(stages + (size_t)s * chunk_elems, chunk_src(s), (uint32_t)(chunk_elems * sizeof(T)),
                 &bars[s]);
      }
    }
    __syncwarp();
  }

  double mass_acc = 0.0;
  bool timed_out = false, nb_pending = false;
  long long t_fail = 0;
  T uxc = 0, uyc = 0, uxe = 0, uxw = 0, uyn = 0, uys = 0, Gxx = 0, Gxy = 0, Gyx = 0, Gyy = 0;
  long long ce = 0, cwc = 0, cn = 0, cs = 0, cell = 0, jc = -1;
  double mf_n = 0.0, mtot = 0.0;
  T src = 0;

  for (long long t = 0; t < nchunks && !timed_out; ++t) {
    const int part = (int)(t % CH);
    const int s = (int)(t % S);
    if (part == 0) {
      // a new cell: per-cell scalars and the psi-transport inputs
      cell = gw + (t / CH) * (long long)W;
      const int ix = (int)(cell % a.nx), iy = (int)(cell / a.nx);
      const int xp = ix + 1 == a.nx ? 0 : ix + 1, xm = ix == 0 ? a.nx - 1 : ix - 1;
      const int yp = iy + 1 == a.ny ? 0 : iy + 1, ym = iy == 0 ? a.ny - 1 : iy - 1;
      ce = (long long)iy * a.nx + xp;
      cwc = (long long)iy * a.nx + xm;
      cn = (long long)yp * a.nx + ix;
      cs = (long long)ym * a.nx + ix;
      mf_n = a.mf[cell];
      mtot = a.mtot[cell];
      src = (T)(kon64 * mf_n);
      const T* uc = a.ucell + cell * 12;
      uxc = uc[0]; uyc = uc[1]; uxe = uc[2]; uxw = uc[3]; uyn = uc[4]; uys = uc[5];
      Gxx = uc[6]; Gxy = uc[7]; Gyx = uc[8]; Gyy = uc[9];
      ++jc;
      if (nb_tma && lane == 0) {
        // stage the psi^n and n_b^n columns of the cell and its 4 neighbours
        const uint32_t pb = (uint32_t)(nth * sizeof(T)), nbb = (uint32_t)(nth * 8);
        mbar_expect_tx(nbar, 5 * (pb + nbb));
        const long long src_cells[5] = {cell, ce, cwc, cn, cs};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          bulk_g2s(psi5 + q * nth, a.psi_in + src_cells[q] * nth, pb, nbar);
          bulk_g2s(nb5 + q * nth, a.nb_in + src_cells[q] * nth, nbb, nbar);
        }
      }
    }

    // ---- motor rows of this chunk
    const T* stg = stages + (size_t)s * chunk_elems;
    const T* gsrc = TMA ? nullptr : chunk_src(t);
    if (TMA) {
      const uint32_t par = (uint32_t)((t / S) & 1);
      const bool ok = __all_sync(0xffffffffu, wait_never ? mbar_wait(never, 0u, wait_limit)
                                                         : mbar_wait(&bars[s], par, wait_limit));
      if (!ok) {
        timed_out = true;
        t_fail = t;
        nb_pending = nb_tma && jc >= 0;
        break;
      }
    }
    T* dst = a.mb + ((size_t)cell * nth + (size_t)part * RC) * ns;
    for (int p = 0; p < passes; ++p) {
      const int r = p * rpp + rslot;  // row within the chunk
      const bool row_ok = r < RC;
      const bool act = row_ok && lane_ok;
      const size_t off = (size_t)(row_ok ? r : 0) * ns + (size_t)sl * V;
      T M[V], R[V], Ms[V];
      if (act) {
        const Pack<T, V> q = TMA ? *reinterpret_cast<const Pack<T, V>*>(stg + off)
                                 : *reinterpret_cast<const Pack<T, V>*>(gsrc + off);
#pragma unroll
        for (int v = 0; v < V; ++v) M[v] = q.v[v];
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) M[v] = T(0);
      }
      motor_rhs<T, V>(M, R, first, last, seg, cw, koff, src);
#pragma unroll
      for (int v = 0; v < V; ++v) Ms[v] = M[v] + hdt * R[v];
      motor_rhs<T, V>(Ms, R, first, last, seg, cw, koff, src);
      T snb = T(0), sm1 = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        M[v] = M[v] + dt * R[v];
        snb += act ? M[v] : T(0);
        sm1 = fma_t(sj[v], act ? M[v] : T(0), sm1);
      }
      if (act) {
        Pack<T, V> q;
#pragma unroll
        for (int v = 0; v < V; ++v) q.v[v] = M[v];
        *reinterpret_cast<Pack<T, V>*>(dst + off) = q;
      }
      snb = seg_sum(snb, seg);
      sm1 = seg_sum(sm1, seg);
      if (first && row_ok) {
        const int k = part * RC + r;
        s_nb[k] = (double)snb * a.ds;
        s_m1[k] = (double)sm1 * a.ds;
      }
    }
    __syncwarp();
    // the stage is consumed: refill it with the chunk S ahead
    if (TMA && lane == 0 && t + S < nchunks) {
      mbar_expect_tx(&bars[s], (uint32_t)(chunk_elems * sizeof(T)));
      bulk_g2s(stages + (size_t)s * chunk_elems, chunk_src(t + S),
               (uint32_t)(chunk_elems * sizeof(T)), &bars[s]);
    }
    if (part != CH - 1) continue;

    // ---- end of the cell: Eq. 1 for psi, then Eq. 5, Alg. 2 and Eq. 6
    if (nb_tma) {
      const bool ok = __all_sync(0xffffffffu, wait_never ? mbar_wait(never, 0u, wait_limit)
                                                         : mbar_wait(nbar, (uint32_t)(jc & 1),
                                                                     wait_limit));
      if (!ok) {
        timed_out = true;
        t_fail = t + 1;  // ring chunks t+1 .. t+S and this neighbourhood are in flight
        nb_pending = true;
        break;
      }
    } else {
      const long long src_cells[5] = {cell, ce, cwc, cn, cs};
      for (int q = 0; q < 5; ++q)
        for (int k = lane; k < nth; k += 32) {
          psi5[q * nth + k] = a.psi_in[src_cells[q] * nth + k];
          nb5[q * nth + k] = a.nb_in[src_cells[q] * nth + k];
        }
      __syncwarp();
    }
    double acc = 0.0;
    for (int k = lane; k < nth; k += 32) {
      const T Pc = g * psi5[k], Pe = g * psi5[nth + k], Pw = g * psi5[2 * nth + k];
      const T Pn = g * psi5[3 * nth + k], Ps = g * psi5[4 * nth + k];
      const T ck = cosk[k], sk = sink[k];
      const T Vc = vsp + glide * (T)nb5[k], Ve = vsp + glide * (T)nb5[nth + k];
      const T Vw = vsp + glide * (T)nb5[2 * nth + k], Vn = vsp + glide * (T)nb5[3 * nth + k];
      const T Vs = vsp + glide * (T)nb5[4 * nth + k];
      const T axc = fma_t(-Vc, ck, uxc), axe = fma_t(-Ve, ck, uxe), axw = fma_t(-Vw, ck, uxw);
      const T ayc = fma_t(-Vc, sk, uyc), ayn = fma_t(-Vn, sk, uyn), ays = fma_t(-Vs, sk, uys);
      const T Ae = T(0.5) * (axc + axe), Aw = T(0.5) * (axw + axc);
      const T An = T(0.5) * (ayc + ayn), As = T(0.5) * (ays + ayc);
      const int kp = k + 1 == nth ? 0 : k + 1, km = k == 0 ? nth - 1 : k - 1;
      const T cp = cosf[k], sp = sinf[k], cm = cosf[km], sm = sinf[km];
      // Jeffery rotation p_perp . G . p at the faces k +- 1/2
      const T wp = -sp * (Gxx * cp + Gxy * sp) + cp * (Gyx * cp + Gyy * sp);
      const T wm = -sm * (Gxx * cm + Gxy * sm) + cm * (Gyx * cm + Gyy * sm);
      const T Fe = donor(Ae, Pc, Pe), Fw = donor(Aw, Pw, Pc);
      const T Fn = donor(An, Pc, Pn), Fs = donor(As, Ps, Pc);
      const T Fp = donor(wp, Pc, g * psi5[kp]), Fm = donor(wm, g * psi5[km], Pc);
      const T pnew = Pc - dt * ((Fe - Fw) * inv_dx + (Fn - Fs) * inv_dy + (Fp - Fm) * inv_dth);
      a.psi_out[cell * nth + k] = pnew;
      mass_acc += (double)pnew;
      acc += (double)pnew * s_nb[k] * a.dth;
    }
    const double Cpre = warp_sum(acc);
    double f = 1.0, C = Cpre;
    if (mtot < Cpre) {
      f = mtot / Cpre;
      C = mtot;
    }
    if (f != 1.0) {
      // rare: rescale the rows of this cell just written (own writes, ordered
      // by the __syncwarp above)
      const T ft = (T)f;
      T* base = a.mb + (size_t)cell * nth * ns;
      for (size_t e = lane; e < (size_t)nth * ns; e += 32) base[e] = __ldcg(base + e) * ft;
    }
    if (lane == 0) {
      a.c[cell] = C;
      a.mf[cell] = mtot - C;
    }
    for (int k = lane; k < nth; k += 32) {
      a.nb_out[cell * nth + k] = s_nb[k] * f;
      if (a.write_m1) a.m1[cell * nth + k] = s_m1[k] * f;
    }
    __syncwarp();
  }

  if (TMA && timed_out) {
    // record the failure, then wait (bounded) for the copies this warp still
    // has in flight -- chunks t_fail .. t_fail + S - 1 -- before leaving
    if (lane == 0) {
      atomicOr(&a.prm->status, 1);
      const long long hi = t_fail + S < nchunks ? t_fail + S : nchunks;
      for (long long t2 = t_fail; t2 < hi; ++t2)
        (void)mbar_wait(&bars[t2 % S], (uint32_t)((t2 / S) & 1), kDrainLimit);
      if (nb_pending) (void)mbar_wait(nbar, (uint32_t)(jc & 1), kDrainLimit);
    }
    __syncwarp();
  }

  // sum psi^{n+1}: per-warp partial, the last warp finalises in a fixed order
  mass_acc = warp_sum(mass_acc);
  unsigned int is_last = 0;
  if (lane == 0) {
    a.partial[gw] = mass_acc;
    __threadfence();
    const unsigned int prev = atomicInc(&a.prm->counter, (unsigned int)W - 1);
    is_last = prev == (unsigned int)W - 1;
  }
  is_last = __shfl_sync(0xffffffffu, is_last, 0);
  if (is_last) {
    __threadfence();
    double m = 0.0;
    for (int b = lane; b < W; b += 32) m += __ldcg(a.partial + b);
    m = warp_sum(m);
    if (lane == 0) {
      a.prm->mass = m;
      if (MASSCORR && a.mass_correct) a.prm->psi_scale = a.prm->mass0 / m;
    }
  }
}

template <typename T, int V>
cudaError_t launch_substep(const StepArgs<T>& a, int grid, int block, size_t smem, bool tma,
                           cudaStream_t s) {
  if (tma) {
    if (a.mass_correct)
      k_substep<T, V, true, true><<<grid, block, smem, s>>>(a);
    else
      k_substep<T, V, true, false><<<grid, block, smem, s>>>(a);
  } else {
    if (a.mass_correct)
      k_substep<T, V, false, true><<<grid, block, smem, s>>>(a);
    else
      k_substep<T, V, false, false><<<grid, block, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int V>
cudaError_t substep_prepare(int block, size_t smem, bool tma, int* blocks_per_sm) {
  const void* fns[4] = {(const void*)k_substep<T, V, true, true>,
                        (const void*)k_substep<T, V, true, false>,
                        (const void*)k_substep<T, V, false, true>,
                        (const void*)k_substep<T, V, false, false>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, tma ? k_substep<T, V, true, true> : k_substep<T, V, false, true>, block, smem);
}

template cudaError_t launch_substep<float, 4>(const StepArgs<float>&, int, int, size_t, bool,
                                              cudaStream_t);
template cudaError_t launch_substep<float, 1>(const StepArgs<float>&, int, int, size_t, bool,
                                              cudaStream_t);
template cudaError_t launch_substep<double, 2>(const StepArgs<double>&, int, int, size_t, bool,
                                               cudaStream_t);
template cudaError_t launch_substep<double, 1>(const StepArgs<double>&, int, int, size_t, bool,
                                               cudaStream_t);
template cudaError_t substep_prepare<float, 4>(int, size_t, bool, int*);
template cudaError_t substep_prepare<float, 1>(int, size_t, bool, int*);
template cudaError_t substep_prepare<double, 2>(int, size_t, bool, int*);
template cudaError_t substep_prepare<double, 1>(int, size_t, bool, int*);

}  // namespace mm
