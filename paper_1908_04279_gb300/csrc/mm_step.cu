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
//   2. n_b of every row by a shuffle reduction over s (the force and force
//      dipole are reduced in float64 by the moments kernel instead);
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

size_t step_smem_per_warp(int S, int chunk_elems, int nth, int tsz) {
  return warp_smem_layout(S, chunk_elems, nth, tsz).total;
}

template <typename T, int V, bool TMA, bool MASSCORR>
__global__ void __launch_bounds__(128, MM_STEP_MIN_BLOCKS) k_substep(const StepArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nth = a.nth, ns = a.ns, seg = a.seg;
  const int S = a.stages, RC = a.chunk_rows, CH = a.chunks_per_cell;
  const int chunk_elems = RC * ns;
  const uint32_t chunk_bytes = (uint32_t)(chunk_elems * sizeof(T));
  // the ring exists only with bulk copies (the host sizes shared memory alike)
  const WarpSmem L = warp_smem_layout(S, TMA ? chunk_elems : 0, nth, (int)sizeof(T));
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* wbase = smem_raw + (size_t)wib * L.total;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + L.bars);
  T* stages = reinterpret_cast<T*>(wbase + L.stages);
  T* psi5 = reinterpret_cast<T*>(wbase + L.psi5);  // [5][nth]: c, e, w, n, s
  T* nb5 = reinterpret_cast<T*>(wbase + L.nb5);    // [5][nth]
  T* s_nb = reinterpret_cast<T*>(wbase + L.nbm);   // n_b of the new rows
  uint64_t* nbar = bars + S;       // neighbourhood barrier
  uint64_t* never = bars + S + 1;  // no copy or arrival ever completes it
  const bool nb_tma = TMA && a.nb_tma;

  // Cells fit in 32 bits (checked on the host); all loop bookkeeping below is
  // incremental, with no 64-bit integer division.
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  const int nx = a.nx, ny = a.ny;
  const int my_cells = gw < nc ? (nc - 1 - gw) / W + 1 : 0;
  const int nchunks = my_cells * CH;

  const int sl = lane & (seg - 1);  // lane within its row
  const int rslot = lane / seg;     // row within a pass
  const int rpp = 32 / seg;         // rows per pass
  const int passes = (RC + rpp - 1) / rpp;
  const int nl = ns / V;
  const bool first = sl == 0, last = sl == nl - 1, lane_ok = sl < nl;

  const DevParams* P = a.prm;
  const double dt64 = P->dt;
  const T dt = (T)dt64, hdt = (T)(0.5 * dt64);
  const T cw = (T)(P->v_walk / a.ds);
  const T koff = (T)P->k_off;
  const T kon = (T)P->k_on;
  const T glide = (T)P->glide, vsp = (T)P->v_sp;
  const T g = MASSCORR ? (T)P->psi_scale : T(1);
  const uint32_t wait_limit = P->wait_limit;
  const bool wait_never = (P->debug_flags & 1u) != 0;  // test knob: every wait runs out
  const T inv_dx = (T)a.inv_dx, inv_dy = (T)a.inv_dy, inv_dth = (T)a.inv_dth;
  const T* cosk = a.trig;
  const T* sink = a.trig + nth;
  const T* cosf = a.trig + 2 * nth;
  const T* sinf = a.trig + 3 * nth;
  const T ds = (T)a.ds, dth_t = (T)a.dth;
  const T c1 = hdt * cw, c2 = T(1) - hdt * koff;
  const T e1 = dt * cw, e2 = -dt * koff;

  // producer cursor: next chunk to issue (cell, part, stage)
  int icell = gw, ipart = 0, istage = 0, issued = 0;
  auto issue_next = [&]() {
    mbar_expect_tx(&bars[istage], chunk_bytes);
    bulk_g2s(stages + (size_t)istage * chunk_elems,
             a.mb_in + ((size_t)icell * nth + (size_t)ipart * RC) * ns, chunk_bytes, &bars[istage]);
    ++issued;
    if (++ipart == CH) { ipart = 0; icell += W; }
    if (++istage == S) istage = 0;
  };

  if (TMA) {
    if (lane == 0) {
      for (int q = 0; q <= S + 1; ++q) mbar_init(&bars[q], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      while (issued < S && issued < nchunks) issue_next();
    }
    __syncwarp();
  }

  double mass_acc = 0.0;
  bool timed_out = false, nb_pending = false;
  int fail_stage = 0, fail_left = 0;
  uint32_t fail_par = 0;
  T uxc = 0, uyc = 0, uxe = 0, uxw = 0, uyn = 0, uys = 0, Gxx = 0, Gxy = 0, Gyx = 0, Gyy = 0;
  int cell = gw - W, ce = 0, cwc = 0, cn = 0, cs = 0;
  uint32_t nb_par = 1;  // parity of the neighbourhood phase of the current cell
  T mtot = 0;
  T c3 = 0, e3 = 0;
  T mass_hi = T(0), mass_lo = T(0);  // compensated sum of psi^{n+1} over this warp's cells
  int part = 0, s = 0;
  uint32_t par = 0;  // parity of the phase chunk t waits for on stage s

  for (int t = 0; t < nchunks; ++t) {
    if (part == 0) {
      // a new cell: per-cell scalars and the psi-transport inputs
      cell += W;
      nb_par ^= 1u;
      const int iy = cell / nx, ix = cell - iy * nx;
      const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
      const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
      ce = iy * nx + xp;
      cwc = iy * nx + xm;
      cn = yp * nx + ix;
      cs = ym * nx + ix;
      const T mf_n = a.mf_in[cell];
      mtot = a.mtot[cell];
      // stage constants: c for the half step, e for the full step
      c3 = hdt * kon * mf_n;
      e3 = dt * kon * mf_n;
      const T* uc = a.ucell + (size_t)cell * 12;
      uxc = uc[0]; uyc = uc[1]; uxe = uc[2]; uxw = uc[3]; uyn = uc[4]; uys = uc[5];
      Gxx = uc[6]; Gxy = uc[7]; Gyx = uc[8]; Gyy = uc[9];
      if (nb_tma && lane == 0) {
        // stage the psi^n and n_b^n columns of the cell and its 4 neighbours
        const uint32_t pb = (uint32_t)(nth * sizeof(T));
        mbar_expect_tx(nbar, 10 * pb);
        const int src_cells[5] = {cell, ce, cwc, cn, cs};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          bulk_g2s(psi5 + q * nth, a.psi_in + (size_t)src_cells[q] * nth, pb, nbar);
          bulk_g2s(nb5 + q * nth, a.nb_in + (size_t)src_cells[q] * nth, pb, nbar);
        }
      }
    }

    // ---- motor rows of this chunk
    const size_t chunk_off = ((size_t)cell * nth + (size_t)part * RC) * ns;
    const T* src_rows = TMA ? stages + (size_t)s * chunk_elems : a.mb_in + chunk_off;
    if (TMA) {
      const bool ok = __all_sync(0xffffffffu, wait_never ? mbar_wait(never, 0u, wait_limit)
                                                         : mbar_wait(&bars[s], par, wait_limit));
      if (!ok) {
        // chunks t .. t + S - 1 (as many as were issued) are in flight
        timed_out = true;
        fail_stage = s;
        fail_par = par;
        fail_left = issued - t;
        nb_pending = nb_tma;
        break;
      }
    }
    T* dst = a.mb_out + chunk_off;
#pragma unroll kStepUnroll
    for (int p = 0; p < passes; ++p) {
      const int r = p * rpp + rslot;  // row within the chunk
      const bool row_ok = r < RC;
      const bool act = row_ok && lane_ok;
      const int off = (row_ok ? r : 0) * ns + sl * V;
      T M[V], D[V], Ms[V];
      if (act) {
        const Pack<T, V> q = *reinterpret_cast<const Pack<T, V>*>(src_rows + off);
#pragma unroll
        for (int v = 0; v < V; ++v) M[v] = q.v[v];
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) M[v] = T(0);
      }
      // Eq. 4 right-hand side R = (v/ds) D - k_off M + k_on Mf; midpoint RK2
      // Ms = M + (dt/2) R(M), M' = M + dt R(Ms), with the constants folded
      walk_dflux<T, V>(M, D, first, last, seg);
#pragma unroll
      for (int v = 0; v < V; ++v) Ms[v] = fma_t(c1, D[v], fma_t(c2, M[v], c3));
      walk_dflux<T, V>(Ms, D, first, last, seg);
      T snb = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        M[v] = fma_t(e1, D[v], fma_t(e2, Ms[v], M[v] + e3));
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
      if (first && row_ok) s_nb[part * RC + r] = snb * ds;
    }
    __syncwarp();
    // the stage is consumed: refill it with the chunk S ahead
    if (TMA && lane == 0 && issued < nchunks) issue_next();
    if (++s == S) { s = 0; par ^= 1u; }
    if (++part != CH) continue;
    part = 0;

    // ---- end of the cell: Eq. 1 for psi, then Eq. 5, Alg. 2 and Eq. 6
    if (nb_tma) {
      const bool ok = __all_sync(0xffffffffu, wait_never ? mbar_wait(never, 0u, wait_limit)
                                                         : mbar_wait(nbar, nb_par, wait_limit));
      if (!ok) {
        timed_out = true;
        fail_stage = s;
        fail_par = par;
        fail_left = issued - (t + 1);
        nb_pending = true;
        break;
      }
    } else {
      const int src_cells[5] = {cell, ce, cwc, cn, cs};
      for (int q = 0; q < 5; ++q)
        for (int k = lane; k < nth; k += 32) {
          psi5[q * nth + k] = a.psi_in[(size_t)src_cells[q] * nth + k];
          nb5[q * nth + k] = a.nb_in[(size_t)src_cells[q] * nth + k];
        }
      __syncwarp();
    }
    T acc = T(0), cell_mass = T(0);
    const size_t cbase = (size_t)cell * nth;
    for (int k = lane; k < nth; k += 32) {
      const T Pc = g * psi5[k], Pe = g * psi5[nth + k], Pw = g * psi5[2 * nth + k];
      const T Pn = g * psi5[3 * nth + k], Ps = g * psi5[4 * nth + k];
      const T ck = cosk[k], sk = sink[k];
      const T Vc = vsp + glide * nb5[k], Ve = vsp + glide * nb5[nth + k];
      const T Vw = vsp + glide * nb5[2 * nth + k], Vn = vsp + glide * nb5[3 * nth + k];
      const T Vs = vsp + glide * nb5[4 * nth + k];
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
      a.psi_out[cbase + k] = pnew;
      cell_mass += pnew;
      acc = fma_t(pnew * s_nb[k], dth_t, acc);
    }
    {
      // TwoSum: mass_hi + mass_lo += cell_mass without rounding loss
      const T s2 = mass_hi + cell_mass, bb = s2 - mass_hi;
      mass_lo += (mass_hi - (s2 - bb)) + (cell_mass - bb);
      mass_hi = s2;
    }
    const T Cpre = warp_sum_t(acc);
    T f = T(1), C = Cpre;
    if (mtot < Cpre) {
      f = mtot / Cpre;
      C = mtot;
    }
    if (f != T(1)) {
      // rare: rescale the rows of this cell just written (own writes, ordered
      // by the __syncwarp above)
      const T ft = f;
      T* base = a.mb_out + cbase * ns;
      for (int e = lane; e < nth * ns; e += 32) base[e] = __ldcg(base + e) * ft;
      for (int k = lane; k < nth; k += 32) a.nb_out[cbase + k] = s_nb[k] * ft;
    } else {
      for (int k = lane; k < nth; k += 32) a.nb_out[cbase + k] = s_nb[k];
    }
    if (lane == 0) {
      a.c[cell] = C;
      a.mf_out[cell] = mtot - C;
      if (a.cpre_out) a.cpre_out[cell] = Cpre;
    }
    __syncwarp();
  }

  if (TMA && timed_out) {
    // record the failure, then wait (bounded) for the copies this warp still
    // has in flight before leaving
    if (lane == 0) {
      atomicOr(&a.prm->status, 1);
      int st = fail_stage;
      uint32_t pp = fail_par;
      for (int i = 0; i < fail_left; ++i) {
        (void)mbar_wait(&bars[st], pp, kDrainLimit);
        if (++st == S) { st = 0; pp ^= 1u; }
      }
      if (nb_pending) (void)mbar_wait(nbar, nb_par, kDrainLimit);
    }
    __syncwarp();
  }

  // sum psi^{n+1}: per-warp partial in float64, the last warp finalises in a
  // fixed order
  mass_acc = warp_sum((double)mass_hi + (double)mass_lo);
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

template cudaError_t launch_substep<float, 8>(const StepArgs<float>&, int, int, size_t, bool,
                                              cudaStream_t);
template cudaError_t launch_substep<float, 4>(const StepArgs<float>&, int, int, size_t, bool,
                                              cudaStream_t);
template cudaError_t launch_substep<float, 1>(const StepArgs<float>&, int, int, size_t, bool,
                                              cudaStream_t);
template cudaError_t launch_substep<double, 2>(const StepArgs<double>&, int, int, size_t, bool,
                                               cudaStream_t);
template cudaError_t launch_substep<double, 1>(const StepArgs<double>&, int, int, size_t, bool,
                                               cudaStream_t);
template cudaError_t substep_prepare<float, 8>(int, size_t, bool, int*);
template cudaError_t substep_prepare<float, 4>(int, size_t, bool, int*);
template cudaError_t substep_prepare<float, 1>(int, size_t, bool, int*);
template cudaError_t substep_prepare<double, 2>(int, size_t, bool, int*);
template cudaError_t substep_prepare<double, 1>(int, size_t, bool, int*);

}  // namespace mm
