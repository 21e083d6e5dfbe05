// Batched-ensemble substep: one persistent launch advances every instance of
// an ensemble (each with its own grid, rates, dt and velocity) by one
// substep.
//
// The work is a table of tiles, each a run of consecutive cells of one
// instance sized to about the same number of motor values; warp gw of W takes
// tiles gw, gw + W, ... and performs, cell by cell, exactly the fused substep
// of the single-instance kernel (Eq. 4 by midpoint RK2 on the s-rows streamed
// through the warp's bulk-copy ring, Eq. 1 for psi, Eq. 5, the scale-down of
// Alg. 2 and Eq. 6), with the instance's arguments read from a device table.
// The ring runs across tile boundaries: lane 0's producer cursor walks the
// same tile sequence ahead of the consumer.
//
// The sum of psi^{n+1} is kept per tile (compensated, then float64); the warp
// that completes the last tile of an instance adds that instance's tile sums
// in tile order (deterministic for any schedule) and, in the float32 form,
// stores the instance's mass-correction factor.
#include "mm_cell.cuh"

namespace mm {

// float64 rows need more registers than the float32 occupancy target allows
#ifndef MM_BATCH_MIN_BLOCKS
#define MM_BATCH_MIN_BLOCKS MM_STEP_MIN_BLOCKS
#endif
template <typename T>
constexpr int batch_min_blocks() {
  return sizeof(T) == 8 ? 3 : MM_BATCH_MIN_BLOCKS;
}

// The psi and n_b columns of two cells of one row (x0 and x0 + 1, y0; nx is
// even and x0 is even, so both lie in the row) and of the four neighbours of
// each into psi5 / nb5 ([2][5][nth], the layout of stage_neighbourhood per
// cell), completing on `nbar`: lane 0 posts the expected bytes, then lanes
// 0-19 each issue one of the 20 bulk copies.
template <typename T>
__device__ __forceinline__ void stage_pair_neighbourhood(uint64_t* nbar, T* psi5, T* nb5,
                                                         const T* psi_in, const T* nb_in, int x0,
                                                         int y0, int nx, int ny, int nth,
                                                         int lane) {
  const uint32_t pb = (uint32_t)(nth * sizeof(T));
  if (lane == 0) mbar_expect_tx(nbar, 20 * pb);
  __syncwarp();
  if (lane < 20) {
    const int h = lane >= 10 ? 1 : 0, q = (lane - 10 * h) >> 1;
    const int x = x0 + h;
    const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
    const int yp = y0 + 1 == ny ? 0 : y0 + 1, ym = y0 == 0 ? ny - 1 : y0 - 1;
    const int cq = q == 0   ? y0 * nx + x
                   : q == 1 ? y0 * nx + xp
                   : q == 2 ? y0 * nx + xm
                   : q == 3 ? yp * nx + x
                            : ym * nx + x;
    const size_t d = (size_t)(5 * h + q) * nth;
    if (lane & 1)
      bulk_g2s(nb5 + d, nb_in + (size_t)cq * nth, pb, nbar);
    else
      bulk_g2s(psi5 + d, psi_in + (size_t)cq * nth, pb, nbar);
  }
}

// cell_motor_close for the two cells of a unit, one per half-warp (lane
// 16 h + k holds orientation k of cell h): the same sums in the same order
// (a cell's orientations sit in lanes 0-15 of its half, as in lanes 0-15 of a
// warp of its own), the same scale-down and writes.
template <typename T>
__device__ __forceinline__ void pair_motor_close(T acc, T mtot, const T* s_nb, int nth, int ns,
                                                 int lane, int cell, T* mb_out, T* nb_out, T* c,
                                                 T* mf_out, T* cpre_out) {
  T Cpre = acc;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) Cpre += __shfl_xor_sync(0xffffffffu, Cpre, o);
  T f = T(1), C = Cpre;
  if (mtot < Cpre) {
    f = mtot / Cpre;
    C = mtot;
  }
  const int hl = lane & 15;
  const size_t cbase = (size_t)cell * nth;
  if (f != T(1)) {
    const T ft = f;
    T* base = mb_out + cbase * ns;
    for (int e = hl; e < nth * ns; e += 16) base[e] = __ldcg(base + e) * ft;
    for (int k = hl; k < nth; k += 16) nb_out[cbase + k] = s_nb[k] * ft;
  } else {
    for (int k = hl; k < nth; k += 16) nb_out[cbase + k] = s_nb[k];
  }
  if (hl == 0) {
    c[cell] = C;
    mf_out[cell] = mtot - C;
    if (cpre_out) cpre_out[cell] = Cpre;
  }
}

template <typename T, int V, bool MASSCORR>
__global__ void __launch_bounds__(128, batch_min_blocks<T>())
    k_substep_batch(const StepArgs<T>* __restrict__ insts, const BatchTile* __restrict__ tiles,
                    int ntiles, double* tile_mass, int S, int stage_elems, int nth_max) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const WarpSmem L = warp_smem_layout(S, stage_elems, nth_max, (int)sizeof(T));
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* wbase = smem_raw + (size_t)wib * L.total;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + L.bars);
  T* stages = reinterpret_cast<T*>(wbase + L.stages);
  T* psi5 = reinterpret_cast<T*>(wbase + L.psi5);
  T* nb5 = reinterpret_cast<T*>(wbase + L.nb5);
  T* s_nb = reinterpret_cast<T*>(wbase + L.nbm);
  uint64_t* nbar = bars + S;
  uint64_t* never = bars + S + 1;

  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  int nchunks = 0;
  for (int t = gw; t < ntiles; t += W) nchunks += tiles[t].ncell * tiles[t].ch;

  // producer cursor (lane 0): tile, cell within it, chunk within the cell
  int ptile = gw, pcell = 0, ppart = 0, istage = 0, issued = 0;
  BatchTile pt{};
  const T* pmb = nullptr;
  int pnth = 0, pns = 0;
  auto producer_tile = [&]() {
    pt = tiles[ptile];
    pmb = insts[pt.inst].mb_in;
    pnth = insts[pt.inst].nth;
    pns = insts[pt.inst].ns;
  };
  auto issue_next = [&]() {
    const uint32_t bytes = (uint32_t)(pt.rc * pns * sizeof(T));
    mbar_expect_tx(&bars[istage], bytes);
    bulk_g2s(stages + (size_t)istage * stage_elems,
             pmb + ((size_t)(pt.cell0 + pcell * pt.cpu) * pnth + (size_t)ppart * pt.rc) * pns, bytes,
             &bars[istage]);
    ++issued;
    if (++ppart == pt.ch) {
      ppart = 0;
      if (++pcell == pt.ncell) {
        pcell = 0;
        ptile += W;
        if (ptile < ntiles) producer_tile();
      }
    }
    if (++istage == S) istage = 0;
  };
  if (lane == 0) {
    for (int q = 0; q <= S + 1; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (ptile < ntiles) producer_tile();
    while (issued < S && issued < nchunks) issue_next();
  }
  __syncwarp();

  bool timed_out = false, nb_pending = false;
  int fail_stage = 0, fail_left = 0;
  uint32_t fail_par = 0;
  int s = 0;
  uint32_t par = 0;
  uint32_t nb_par = 1;

  // consumer: current tile and instance
  int tix = gw - W, ccell = 0, part = 0;
  BatchTile ct{};
  ct.ncell = 0;
  const StepArgs<T>* A = nullptr;
  int nth = 1, ns = 1, seg = 1, nx = 1, ny = 1;
  bool nb_tma = false;
  uint32_t wait_limit = 0;
  bool wait_never = false;
  T hdt = 0, dt = 0, kon = 0, ds = 0;
  PsiConst<T> pq{};
  RkConst<T> rk{};
  LaneGeom lg{};
  T mass_hi = T(0), mass_lo = T(0);
  int cell = 0, ix = 0, iy = 0;
  // the cell at (ix, iy) and its east, west, north and south neighbours
  // (recomputed where needed rather than kept across the rows)
  auto nbrs = [&](int (&c)[5]) {
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    c[0] = iy * nx + ix;
    c[1] = iy * nx + xp;
    c[2] = iy * nx + xm;
    c[3] = yp * nx + ix;
    c[4] = ym * nx + ix;
  };
  T mtot = 0;
  CellVel<T> uv{};
  // the next cell's free and total motors, loaded while the current cell is
  // computed (the RK2 constants need them as soon as a cell starts)
  T mf_next = 0;
  bool have_next = false;

  // sum of the finished tile; the last tile of an instance finalises it
  auto close_tile = [&]() {
    const double m = warp_sum_ff(mass_hi, mass_lo);
    mass_hi = T(0);
    mass_lo = T(0);
    unsigned int is_last = 0;
    if (lane == 0) {
      tile_mass[tix] = m;
      __threadfence();
      const unsigned int prev = atomicInc(&A->prm->counter, (unsigned int)ct.inst_tiles - 1);
      is_last = prev == (unsigned int)ct.inst_tiles - 1;
    }
    is_last = __shfl_sync(0xffffffffu, is_last, 0);
    if (is_last) {
      __threadfence();
      const double acc = warp_sum_ldcg(tile_mass + ct.tile0, ct.inst_tiles, 1, lane);
      if (lane == 0) {
        A->prm->mass = acc;
        if (MASSCORR && A->mass_correct) A->prm->psi_scale = A->prm->mass0 / acc;
      }
    }
  };

  for (int t = 0; t < nchunks; ++t) {
    if (part == 0) {
      if (ccell == ct.ncell) {
        // next tile (and its instance's constants)
        tix += W;
        ct = tiles[tix];
        ccell = 0;
        A = insts + ct.inst;
        nth = A->nth;
        ns = A->ns;
        seg = A->seg;
        nx = A->nx;
        ny = A->ny;
        nb_tma = A->nb_tma != 0;
        const DevParams* P = A->prm;
        const StepScalars<T> sc = step_scalars<T, MASSCORR>(P, *A, lane);
        dt = sc.dt;
        hdt = sc.hdt;
        kon = sc.kon;
        wait_limit = P->wait_limit;
        wait_never = (P->debug_flags & 1u) != 0;
        pq = PsiConst<T>{dt, sc.g, sc.glide, sc.vsp, sc.inv_dx, sc.inv_dy, sc.inv_dth, sc.dth,
                         A->trig};
        ds = sc.ds;
        rk = RkConst<T>{hdt * sc.cw, T(1) - hdt * sc.koff, T(0), dt * sc.cw, -dt * sc.koff, T(0),
                        T(0), T(0), nth};
        lg = lane_geom(lane, seg, ns, V);
        iy = ct.cell0 / nx;
        ix = ct.cell0 - iy * nx;
      } else if ((ix += ct.cpu) >= nx) {  // consecutive units of the tile
        ix -= nx;
        ++iy;
      }
      // the unit's first cell; Mf of the first cell and the total motors of
      // the half-warp's cell
      cell = ct.cell0 + ccell * ct.cpu;
      // the half-warp's cell in a unit of 2 with at most 16 orientations
      const int half = (ct.cpu == 2 && nth <= 16) ? lane >> 4 : 0;
      // (the total motors are needed at the unit's end only)
      const T mf_n = have_next && ccell > 0 ? mf_next : A->mf_in[cell];
      mtot = A->mtot[cell + half];
      have_next = ccell + 1 < ct.ncell;
      // Mf of the next unit is written only when that unit is done
      if (have_next) mf_next = A->mf_in[cell + ct.cpu];
      if (nb_tma) nb_par ^= 1u;  // members differ in whether they stage by bulk copy
      rk.c3 = hdt * kon * mf_n;
      rk.e3 = dt * kon * mf_n;
      {  // a unit of 2: the second cell's rows (from row nth on) bind to its own Mf
         // (a unit of 1 has no row nth in a chunk, and its c3b, e3b are c3, e3)
        const T mf2 = ct.cpu == 2 ? A->mf_in[cell + 1] : mf_n;
        rk.c3b = hdt * kon * mf2;
        rk.e3b = dt * kon * mf2;
      }
      uv = load_cell_vel(A->ucell, cell + half);
      if (nb_tma && ct.cpu == 2)
        stage_pair_neighbourhood(nbar, psi5, nb5, A->psi_in, A->nb_in, ix, iy, nx, ny, nth, lane);
      else if (nb_tma) {
        int c[5];
        nbrs(c);
        stage_neighbourhood(nbar, psi5, nb5, A->psi_in, A->nb_in, c[0], c[1], c[2], c[3], c[4],
                            nth, lane);
      }
    }

    // ---- motor rows of this chunk
    const size_t chunk_off = ((size_t)cell * nth + (size_t)part * ct.rc) * ns;
    {
      const bool ok = __all_sync(0xffffffffu, wait_never ? mbar_wait(never, 0u, wait_limit)
                                                         : mbar_wait(&bars[s], par, wait_limit));
      if (!ok) {
        timed_out = true;
        fail_stage = s;
        fail_par = par;
        fail_left = issued - t;
        nb_pending = nb_tma;
        break;
      }
    }
    // (rows from the unit's row nth on -- the second cell of a unit of 2 --
    // bind to that cell's Mf; a chunk may hold rows of either or both)
    rk.rsplit = nth - part * ct.rc;
    rows_chunk<T, V, true>(stages + (size_t)s * stage_elems, A->mb_out + chunk_off, ct.rc, ns, seg,
                           lg, rk, ds, s_nb + part * ct.rc);
    __syncwarp();
    if (lane == 0 && issued < nchunks) issue_next();
    if (++s == S) { s = 0; par ^= 1u; }
    if (++part != ct.ch) continue;
    part = 0;

    // ---- end of the cell
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
      int src_cells[5];
      nbrs(src_cells);
      for (int q = 0; q < 5; ++q)
        for (int k = lane; k < nth; k += 32) {
          psi5[q * nth + k] = A->psi_in[(size_t)src_cells[q] * nth + k];
          nb5[q * nth + k] = A->nb_in[(size_t)src_cells[q] * nth + k];
        }
      __syncwarp();
    }
    if (ct.cpu == 2 && nth > 16) {
      // a unit of 2 with more than 16 orientations: the warp takes the two
      // cells' psi transport and close one after the other
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        if (h) {  // the second cell's velocity block and total motors
          uv = load_cell_vel(A->ucell, cell + 1);
          mtot = A->mtot[cell + 1];
        }
        T acc = T(0), cell_mass = T(0);
        const size_t h5 = (size_t)h * 5 * nth;
        psi_cell(pq, uv, psi5 + h5, nb5 + h5, s_nb + h * nth, nth, lane,
                 A->psi_out + (size_t)(cell + h) * nth, cell_mass, acc);
        two_sum_acc(mass_hi, mass_lo, cell_mass);
        cell_motor_close(acc, mtot, s_nb + h * nth, nth, ns, lane, cell + h, A->mb_out,
                         A->nb_out, A->c, A->mf_out, A->cpre_out);
        __syncwarp();
      }
    } else {
      T acc = T(0), cell_mass = T(0);
      // (in a unit of 2, half-warp h takes cell h with lane 16 h + k on orientation k)
      const int half = ct.cpu == 2 ? lane >> 4 : 0;
      const size_t h5 = (size_t)half * 5 * nth;
      psi_cell(pq, uv, psi5 + h5, nb5 + h5, s_nb + half * nth, nth,
               ct.cpu == 2 ? lane & 15 : lane, A->psi_out + (size_t)(cell + half) * nth, cell_mass,
               acc);
      two_sum_acc(mass_hi, mass_lo, cell_mass);
      if (ct.cpu == 2)
        pair_motor_close(acc, mtot, s_nb + half * nth, nth, ns, lane, cell + half, A->mb_out,
                         A->nb_out, A->c, A->mf_out, A->cpre_out);
      else
        cell_motor_close(acc, mtot, s_nb, nth, ns, lane, cell, A->mb_out, A->nb_out, A->c,
                         A->mf_out, A->cpre_out);
      __syncwarp();
    }
    if (++ccell == ct.ncell) close_tile();
  }

  if (timed_out) {
    if (lane == 0) {
      atomicOr(&A->prm->status, 1);
      int st = fail_stage;
      uint32_t pp = fail_par;
      for (int i = 0; i < fail_left; ++i) {
        drain_wait(&bars[st], pp, &A->prm->status);
        if (++st == S) { st = 0; pp ^= 1u; }
      }
      if (nb_pending) drain_wait(nbar, nb_par, &A->prm->status);
    }
    __syncwarp();
  }
}

template <typename T, int V>
cudaError_t launch_substep_batch(const StepArgs<T>* insts, const BatchTile* tiles, int ntiles,
                                 double* tile_mass, int S, int stage_elems, int nth_max,
                                 bool masscorr, int grid, int block, size_t smem, cudaStream_t s) {
  if (masscorr)
    k_substep_batch<T, V, true><<<grid, block, smem, s>>>(insts, tiles, ntiles, tile_mass, S,
                                                          stage_elems, nth_max);
  else
    k_substep_batch<T, V, false><<<grid, block, smem, s>>>(insts, tiles, ntiles, tile_mass, S,
                                                           stage_elems, nth_max);
  return cudaGetLastError();
}

template <typename T, int V>
cudaError_t substep_batch_prepare(int block, size_t smem, int* blocks_per_sm) {
  const void* fns[2] = {(const void*)k_substep_batch<T, V, true>,
                        (const void*)k_substep_batch<T, V, false>};
  for (const void* f : fns) {
    cudaError_t e = mm::raise_smem_limit(f, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_substep_batch<T, V, true>,
                                                       block, smem);
}

#define MM_BATCH_INST(T, V)                                                                    \
  template cudaError_t launch_substep_batch<T, V>(const StepArgs<T>*, const BatchTile*, int,   \
                                                  double*, int, int, int, bool, int, int,      \
                                                  size_t, cudaStream_t);                       \
  template cudaError_t substep_batch_prepare<T, V>(int, size_t, int*);
MM_BATCH_INST(float, 8)
MM_BATCH_INST(float, 4)
MM_BATCH_INST(double, 2)

}  // namespace mm
