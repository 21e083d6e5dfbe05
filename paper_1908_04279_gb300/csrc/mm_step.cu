// Fused microscale substep kernel (forward), warp-per-cell with a TMA ring.
//
// Every warp owns whole spatial cells (cells gw, gw + W, gw + 2W, ... for
// global warp gw of W) and performs the whole substep for each of them, with
// no block-level barrier before the final sum:
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
// Mf and C are cell-local. Each warp also sums psi^{n+1} in float64, the
// warps of a block add their sums at the end; the last block to finish adds
// the block sums in a fixed order and, in the float32 form, stores the
// mass-correction factor applied to psi on the next load.
//
// Every mbarrier wait is bounded (DevParams::wait_limit polls). A warp whose
// wait runs out records MM_ERR_TIMEOUT in DevParams::status, waits (bounded)
// for the copies it still has in flight and leaves.
#include "mm_async.cuh"
#include "mm_cell.cuh"

namespace mm {

size_t step_smem_per_warp(int S, int chunk_elems, int nth, int tsz) {
  return warp_smem_layout(S, chunk_elems, nth, tsz).total;
}

template <typename T, int V, bool TMA, bool MASSCORR>
__global__ void __launch_bounds__(128, MM_STEP_MIN_BLOCKS) k_substep(const StepArgs<T> a) {
  griddep_wait();  // launched overlapped outside graphs (recording, replays)
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

  const LaneGeom lg = lane_geom(lane, seg, ns, V);

  const DevParams* P = a.prm;
  const StepScalars<T> sc = step_scalars<T, MASSCORR>(P, a, lane);
  const T dt = sc.dt, hdt = sc.hdt, kon = sc.kon;
  const uint32_t wait_limit = P->wait_limit;
  const bool wait_never = (P->debug_flags & 1u) != 0;  // test knob: every wait runs out
  const PsiConst<T> pq{dt, sc.g, sc.glide, sc.vsp, sc.inv_dx, sc.inv_dy, sc.inv_dth, sc.dth,
                       a.trig};
  const T ds = sc.ds;
  RkConst<T> rk{hdt * sc.cw, T(1) - hdt * sc.koff, T(0), dt * sc.cw, -dt * sc.koff, T(0)};

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
  CellVel<T> uv{};
  int cell = gw - W, ce = 0, cwc = 0, cn = 0, cs = 0;
  // cell coordinates, advanced by W cells at a time without a division
  const int Wy = W / nx, Wx = W - Wy * nx;
  int ix = -1, iy = 0;
  const LaneTrig<T> lt = lane_trig(a.trig, nth, lane);
  uint32_t nb_par = 1;  // parity of the neighbourhood phase of the current cell
  T mtot = 0;
  // Mf and M of this warp's next cell (cell + W), loaded while the current
  // cell is computed: the RK2 constants need them as soon as a cell starts.
  // A cell's Mf is written only when that cell is done, by this warp.
  T mf_next = gw < (int)a.ncells ? a.mf_in[gw] : T(0);
  T mtot_next = gw < (int)a.ncells ? a.mtot[gw] : T(0);
  T mass_hi = T(0), mass_lo = T(0);  // compensated sum of psi^{n+1} over this warp's cells
  int part = 0, s = 0;
  uint32_t par = 0;  // parity of the phase chunk t waits for on stage s

  for (int t = 0; t < nchunks; ++t) {
    if (part == 0) {
      // a new cell: per-cell scalars and the psi-transport inputs
      cell += W;
      nb_par ^= 1u;
      if (ix < 0) {
        iy = cell / nx;
        ix = cell - iy * nx;
      } else {
        ix += Wx;
        iy += Wy;
        if (ix >= nx) {
          ix -= nx;
          ++iy;
        }
      }
      const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
      const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
      ce = iy * nx + xp;
      cwc = iy * nx + xm;
      cn = yp * nx + ix;
      cs = ym * nx + ix;
      const T mf_n = mf_next;
      mtot = mtot_next;
      if (cell + W < (int)a.ncells) {
        mf_next = a.mf_in[cell + W];
        mtot_next = a.mtot[cell + W];
      }
      // stage constants: c for the half step, e for the full step
      rk.c3 = hdt * kon * mf_n;
      rk.e3 = dt * kon * mf_n;
      uv = load_cell_vel(a.ucell, cell);
      if (nb_tma)  // stage the psi^n and n_b^n columns of the cell and its 4 neighbours
        stage_neighbourhood(nbar, psi5, nb5, a.psi_in, a.nb_in, cell, ce, cwc, cn, cs, nth, lane);
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
    rows_chunk<T, V>(src_rows, a.mb_out + chunk_off, RC, ns, seg, lg, rk, ds, s_nb + part * RC);
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
    psi_cell(pq, uv, psi5, nb5, s_nb, nth, lane, a.psi_out + (size_t)cell * nth, cell_mass, acc,
             &lt);
    two_sum_acc(mass_hi, mass_lo, cell_mass);
    cell_motor_close(acc, mtot, s_nb, nth, ns, lane, cell, a.mb_out, a.nb_out, a.c, a.mf_out,
                     a.cpre_out);
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
        drain_wait(&bars[st], pp, &a.prm->status);
        if (++st == S) { st = 0; pp ^= 1u; }
      }
      if (nb_pending) drain_wait(nbar, nb_par, &a.prm->status);
    }
    __syncwarp();
  }

  // sum psi^{n+1}: per-warp partial, added per block in warp order; the last
  // block adds the block partials in a fixed order. Float64 in the float64
  // form; float-float (float pairs in the partial slots) in the float32 form,
  // converted to float64 once.
  __shared__ double s_red[32];
  __shared__ unsigned int s_last;
  if constexpr (sizeof(T) == 4) {
    float2* s_red2 = reinterpret_cast<float2*>(s_red);
    const float2 wsum = warp_sum_ff2(make_float2(mass_hi, mass_lo));
    if (lane == 0) s_red2[wib] = wsum;
    __syncthreads();
    float2* part2 = reinterpret_cast<float2*>(a.partial);
    if (threadIdx.x == 0) {
      float2 b = s_red2[0];
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q) b = ff2_add(b, s_red2[q]);
      part2[blockIdx.x] = b;
      __threadfence();
      const unsigned int prev = atomicInc(&a.prm->counter, gridDim.x - 1);
      s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && wib == 0) {
      __threadfence();
      const float2 m2 = warp_sum_ldcg_ff2(part2, (int)gridDim.x, lane);
      if (lane == 0) {
        const double m = (double)m2.x + (double)m2.y;
        a.prm->mass = m;
        if (MASSCORR && a.mass_correct) a.prm->psi_scale = a.prm->mass0 / m;
      }
    }
  } else {
    mass_acc = warp_sum_ff(mass_hi, mass_lo);
    if (lane == 0) s_red[wib] = mass_acc;
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
      const double m = warp_sum_ldcg(a.partial, (int)gridDim.x, 1, lane);
      if (lane == 0) {
        a.prm->mass = m;
        if (MASSCORR && a.mass_correct) a.prm->psi_scale = a.prm->mass0 / m;
      }
    }
  }
}

template <typename T, int V>
cudaError_t launch_substep_impl(const StepArgs<T>& a, int grid, int block, size_t smem, bool tma,
                                cudaStream_t s, bool overlap) {
  void (*k)(StepArgs<T>) = tma ? (a.mass_correct ? k_substep<T, V, true, true>
                                                 : k_substep<T, V, true, false>)
                               : (a.mass_correct ? k_substep<T, V, false, true>
                                                 : k_substep<T, V, false, false>);
  if (overlap) return launch_overlapped(k, grid, block, smem, s, a);
  k<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int V>
cudaError_t launch_substep(const StepArgs<T>& a, int grid, int block, size_t smem, bool tma,
                           cudaStream_t s) {
  return launch_substep_impl<T, V>(a, grid, block, smem, tma, s, false);
}
// The same launched overlapped with the previous kernel of the stream (direct
// launches: the recording's last segment, the replays of the reverse sweep).
template <typename T, int V>
cudaError_t launch_substep_overlapped(const StepArgs<T>& a, int grid, int block, size_t smem,
                                      bool tma, cudaStream_t s) {
  return launch_substep_impl<T, V>(a, grid, block, smem, tma, s, true);
}

template <typename T, int V>
cudaError_t substep_prepare(int block, size_t smem, bool tma, int* blocks_per_sm) {
  const void* fns[4] = {(const void*)k_substep<T, V, true, true>,
                        (const void*)k_substep<T, V, true, false>,
                        (const void*)k_substep<T, V, false, true>,
                        (const void*)k_substep<T, V, false, false>};
  for (const void* f : fns) {
    cudaError_t e = mm::raise_smem_limit(f, (int)smem);
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
template cudaError_t launch_substep_overlapped<float, 8>(const StepArgs<float>&, int, int, size_t,
                                                         bool, cudaStream_t);
template cudaError_t substep_prepare<float, 8>(int, size_t, bool, int*);
template cudaError_t launch_substep_overlapped<float, 4>(const StepArgs<float>&, int, int, size_t,
                                                         bool, cudaStream_t);
template cudaError_t substep_prepare<float, 4>(int, size_t, bool, int*);
template cudaError_t launch_substep_overlapped<float, 1>(const StepArgs<float>&, int, int, size_t,
                                                         bool, cudaStream_t);
template cudaError_t substep_prepare<float, 1>(int, size_t, bool, int*);
template cudaError_t launch_substep_overlapped<double, 2>(const StepArgs<double>&, int, int, size_t,
                                                          bool, cudaStream_t);
template cudaError_t substep_prepare<double, 2>(int, size_t, bool, int*);
template cudaError_t launch_substep_overlapped<double, 1>(const StepArgs<double>&, int, int, size_t,
                                                          bool, cudaStream_t);
template cudaError_t substep_prepare<double, 1>(int, size_t, bool, int*);

}  // namespace mm
