// Motor kinetics over a macro interval with psi frozen and a local substep in
// every cell: the independent time steps of Sec. 3.1, i.e. Alg. 2's
// "while t* < t*_end" loop run per anchor (anchors in the filament's own cell)
// with the step each anchor's own rates allow.
//
// With psi frozen the cells are independent, so a block owns one whole cell at
// a time and keeps the cell's motor rows in shared memory for all of the
// cell's substeps: the rows arrive by one bulk copy (issued a cell ahead into a
// second buffer), every substep is the midpoint RK2 of Eq. 4 (half and full
// stage, Mf frozen over the stages) on rows spread over the block's warps, a
// block barrier, then the coarse density of Eq. 5 with the frozen psi (each
// warp reduces all of the cell's n_b in the same order, so every warp holds the
// same bits without a second barrier), the Alg. 2 scale-down and Eq. 6. The
// last substep writes the rows straight back to global memory. The motor
// density therefore crosses HBM once per call, whatever the number of
// substeps: the kernel is bound by the float arithmetic of the row updates,
// not by memory.
//
// k_local_nsteps runs first: per cell, rho = sum_k psi dtheta (in k order),
// rate = max(v/ds, k_off + k_on L rho) and n = max(1, ceil(T rate / cfl)),
// every operation in float64 with explicit rounding (no contraction), so the
// count is the one a float64 evaluation of the same formula gives; or the
// caller's counts. A count outside 1..kMaxLocalSteps sets status bit 2 and the
// motor kernel then leaves the whole state unchanged.
#include "mm_cell.cuh"
#include "mm_host.h"

namespace mm {

constexpr int kMaxLocalSteps = 1 << 20;
constexpr int kLocalStatusBit = 4;  // status bit 2: a local step count out of range

template <typename T>
struct LocalArgs {
  int nth, ns, seg;
  int rows_per_warp;  // consecutive s-rows of a cell per warp (multiple of 32 / seg)
  int nbuf;           // shared-memory row buffers (2: the next cell's copy overlaps)
  int bulk;           // 1: the cell's rows arrive by one bulk copy
  long long ncells;
  double T_int;       // the macro interval
  double ds, dth;
  T* mb;              // [cells][nth][ns], in place
  const T* psi;       // [cells][nth], frozen (times psi_scale in the float32 form)
  T* nb_out;          // [cells][nth] n_b of the new rows
  T* mf;              // [cells] in place
  T* c;               // [cells]
  const T* mtot;      // [cells]
  const int* nsteps;  // [cells] substeps per cell
  DevParams* prm;
  int masscorr;       // 1: psi is scaled by prm->psi_scale on load
};

template <typename T>
__global__ void k_local_nsteps(const T* psi, int* nsteps, const int* nsteps_in, long long ncells,
                               int nth, double dth, double L, double T_int, double cfl,
                               int masscorr, DevParams* prm) {
  const double g = masscorr ? prm->psi_scale : 1.0;
  const double cw = prm->cw, koff = prm->k_off, konL = __dmul_rn(prm->k_on, L);
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ncells;
       cell += (long long)gridDim.x * blockDim.x) {
    int n;
    if (nsteps_in) {
      n = nsteps_in[cell];
      if (n < 1 || n > kMaxLocalSteps) {
        atomicOr(&prm->status, kLocalStatusBit);
        n = 0;
      }
    } else {
      double rho = 0.0;
      const T* p = psi + cell * nth;
      for (int k = 0; k < nth; ++k) {
        double v = (double)p[k];
        if (masscorr) v = __dmul_rn(v, g);
        rho = __dadd_rn(rho, __dmul_rn(v, dth));
      }
      const double rate = fmax(cw, __dadd_rn(koff, __dmul_rn(konL, rho)));
      const double q = ceil(__ddiv_rn(__dmul_rn(T_int, rate), cfl));
      if (!(q <= (double)kMaxLocalSteps)) {  // also catches NaN
        atomicOr(&prm->status, kLocalStatusBit);
        n = 0;
      } else {
        n = q < 1.0 ? 1 : (int)q;
      }
    }
    nsteps[cell] = n;
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared memory of the motor kernel: nbuf + 1 mbarriers (the last one never
// completes: the timeout test waits on it), nbuf row buffers of nth * ns
// values, the scaled psi column and two n_b columns (substeps alternate).
struct LocalSmem {
  size_t bars, rows, w, nb, total;
};
__host__ __device__ inline LocalSmem local_smem_layout(int nbuf, int nth, int ns, int tsz) {
  LocalSmem L;
  L.bars = 0;
  size_t off = 8 * (size_t)(nbuf + 1);
  off = (off + 127) & ~(size_t)127;
  L.rows = off;
  off += (size_t)nbuf * nth * ns * tsz;
  off = (off + 15) & ~(size_t)15;
  L.w = off;
  off += (size_t)nth * tsz;
  off = (off + 15) & ~(size_t)15;
  L.nb = off;
  off += 2 * (size_t)nth * tsz;
  off = (off + 127) & ~(size_t)127;
  L.total = off;
  return L;
}

template <typename T, int V>
__global__ void __launch_bounds__(256, 2) k_motor_local(const LocalArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nth = a.nth, ns = a.ns, seg = a.seg, nbuf = a.nbuf;
  const size_t cvals = (size_t)nth * ns;
  const LocalSmem Ls = local_smem_layout(nbuf, nth, ns, (int)sizeof(T));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + Ls.bars);
  T* rowbuf = reinterpret_cast<T*>(smem_raw + Ls.rows);
  T* wcol = reinterpret_cast<T*>(smem_raw + Ls.w);   // psi of the cell (scaled)
  T* nbcol = reinterpret_cast<T*>(smem_raw + Ls.nb);  // [2][nth]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const DevParams* P = a.prm;
  if (P->status & kLocalStatusBit) return;  // a step count out of range: change nothing

  const long long nc = a.ncells;
  const int first = blockIdx.x;
  const int G = gridDim.x;
  const int my_cells = first < nc ? (int)((nc - 1 - first) / G + 1) : 0;
  const uint32_t cbytes = (uint32_t)(cvals * sizeof(T));
  const bool bulk = a.bulk != 0;
  const uint32_t wait_limit = P->wait_limit;
  const bool wait_never = (P->debug_flags & 1u) != 0;
  uint64_t* never = bars + nbuf;

  int issued = 0;  // cells whose copy tid 0 has issued
  auto issue = [&](int it) {
    const long long cell = first + (long long)it * G;
    uint64_t* bar = &bars[it % nbuf];
    mbar_expect_tx(bar, cbytes);
    bulk_g2s(rowbuf + (size_t)(it % nbuf) * cvals, a.mb + (size_t)cell * cvals, cbytes, bar);
  };
  if (bulk && tid == 0) {
    for (int q = 0; q <= nbuf; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    while (issued < nbuf && issued < my_cells) issue(issued++);
  }
  __syncthreads();

  const LaneGeom lg = lane_geom(lane, seg, ns, V);
  const int r0 = w * a.rows_per_warp;
  const int cnt = max(0, min(a.rows_per_warp, nth - r0));
  const T ds = (T)a.ds, dth = (T)a.dth;
  const T cw = (T)P->cw, koff = (T)P->k_off, kon = (T)P->k_on;
  const T g = a.masscorr ? (T)P->psi_scale : T(1);

  for (int it = 0; it < my_cells; ++it) {
    const long long cell = first + (long long)it * G;
    T* rows = rowbuf + (size_t)(it % nbuf) * cvals;
    const int n = a.nsteps[cell];
    const T mt = a.mtot[cell];
    T mfc = a.mf[cell];
    for (int k = tid; k < nth; k += blockDim.x) wcol[k] = g * a.psi[(size_t)cell * nth + k];
    bool ok = true;
    if (bulk) {
      ok = wait_never ? mbar_wait(never, 0u, wait_limit)
                      : mbar_wait(&bars[it % nbuf], (uint32_t)((it / nbuf) & 1), wait_limit);
    } else {
      const T* src = a.mb + (size_t)cell * cvals;
      for (size_t e = tid; e < cvals; e += blockDim.x) rows[e] = src[e];
    }
    if (!__syncthreads_and(ok)) {
      // a bounded wait gave up: record it, wait (bounded) for the copies still
      // in flight, leave the rest of this block's cells untouched
      if (tid == 0) {
        atomicOr(&a.prm->status, 1);
        for (int j = it; j < issued; ++j)
          drain_wait(&bars[j % nbuf], (uint32_t)((j / nbuf) & 1), &a.prm->status);
      }
      return;
    }

    // substeps of this cell: dt = T / n, Eq. 4 by midpoint RK2 with Mf frozen
    const double dt64 = a.T_int / n;
    const T dt = (T)dt64, hdt = (T)(0.5 * dt64);
    RkConst<T> rk{hdt * cw, T(1) - hdt * koff, hdt * kon * mfc,
                  dt * cw, -dt * koff, dt * kon * mfc};
    T* gdst = a.mb + (size_t)cell * cvals;
    T f = T(1), C = T(0);
    for (int step = 0; step < n; ++step) {
      const bool last = step == n - 1;
      T* nbs = nbcol + (step & 1) * nth;
      T* dst = last ? gdst : rows;
      if (cnt > 0)
        rows_chunk<T, V>(rows + (size_t)r0 * ns, dst + (size_t)r0 * ns, cnt, ns, seg, lg, rk, ds,
                         nbs + r0);
      __syncthreads();
      // Eq. 5 with the frozen psi: every warp forms the same sum
      T acc = T(0);
      for (int k = lane; k < nth; k += 32) acc = fma_t(wcol[k] * nbs[k], dth, acc);
      const T Cpre = warp_sum_t(acc);
      f = T(1);
      C = Cpre;
      if (mt < Cpre) {  // Alg. 2 scale-down
        f = mt / Cpre;
        C = mt;
      }
      mfc = mt - C;  // Eq. 6
      if (f != T(1) && cnt > 0) {
        __syncwarp();
        T* base = dst + (size_t)r0 * ns;
        for (int e = lane; e < cnt * ns; e += 32) base[e] = base[e] * f;
        __syncwarp();
      }
      rk.c3 = hdt * kon * mfc;
      rk.e3 = dt * kon * mfc;
    }
    // n_b of the new rows (after the last scale-down), C and Mf
    const T* nbs = nbcol + ((n - 1) & 1) * nth;
    for (int k = lane; k < cnt; k += 32)
      a.nb_out[(size_t)cell * nth + r0 + k] = f != T(1) ? nbs[r0 + k] * f : nbs[r0 + k];
    if (tid == 0) {
      a.c[cell] = C;
      a.mf[cell] = mfc;
    }
    // the buffer is free: the cell nbuf ahead may be copied into it (the
    // generic-proxy writes above are ordered before the bulk copy's)
    fence_proxy_async_smem();
    __syncthreads();
    if (bulk && tid == 0 && issued < my_cells) issue(issued++);
  }
}

template <typename T, int V>
cudaError_t local_prepare(int block, size_t smem, int* bps) {
  cudaError_t e = mm::raise_smem_limit(k_motor_local<T, V>, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_motor_local<T, V>, block, smem);
}

template <typename T, int V>
cudaError_t launch_motor_local(const LocalArgs<T>& a, int grid, int block, size_t smem,
                               cudaStream_t s) {
  k_motor_local<T, V><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mm

using namespace mmh;

namespace {

// Block shape of the motor kernel: rows in groups of rpp = 32 / seg (one warp
// pass), at most 8 warps, each warp owning `passes` consecutive groups.
struct LocalPlan {
  int block, rows_per_warp, nbuf, bulk, grid;
  size_t smem;
};

template <typename T, int V>
mm_status local_plan(mm_handle* h, LocalPlan* p) {
  const int nth = h->g.ntheta, ns = h->g.ns;
  const int rpp = 32 / h->seg;
  const int groups = (nth + rpp - 1) / rpp;
  const int passes = (groups + 7) / 8;
  const int nw = (groups + passes - 1) / passes;
  p->block = 32 * nw;
  p->rows_per_warp = passes * rpp;
  p->bulk = ((size_t)nth * ns * sizeof(T)) % 16 == 0 ? 1 : 0;
  p->nbuf = 2;
  p->smem = mm::local_smem_layout(2, nth, ns, (int)sizeof(T)).total;
  if (!p->bulk || p->smem > kSmemBudget) {
    p->nbuf = 1;
    p->smem = mm::local_smem_layout(1, nth, ns, (int)sizeof(T)).total;
  }
  if (p->smem > kSmemBudget)
    return fail(h, MM_ERR_UNSUPPORTED,
                "ntheta * ns too large: one cell's motor rows must fit in shared memory");
  int bps = 0;
  CK((mm::local_prepare<T, V>(p->block, p->smem, &bps)));
  if (bps < 1) return fail(h, MM_ERR_UNSUPPORTED, "local-step kernel cannot be resident");
  long long g = (long long)bps * h->sms;
  if (g > h->ncells) g = h->ncells;
  p->grid = (int)g;
  return MM_OK;
}

template <typename T, int V>
mm_status run_local(mm_handle* h, double Tint, const int* nin) {
  LocalPlan p;
  mm_status st = local_plan<T, V>(h, &p);
  if (st != MM_OK) return st;
  const double dth = 2.0 * kPi / h->g.ntheta;
  const int masscorr = h->prec == MM_FP32_MIXED ? 1 : 0;
  const long long nc = h->ncells;
  const int tb = 256;
  long long gb = (nc + tb - 1) / tb;
  if (gb > 8LL * h->sms) gb = 8LL * h->sms;
  mm::k_local_nsteps<T><<<(int)gb, tb, 0, h->stream>>>(
      (const T*)h->psi[h->parity], h->local_n, nin, nc, h->g.ntheta, dth, h->g.L, Tint, h->r.cfl,
      masscorr, h->prm);
  CK(cudaGetLastError());
  mm::LocalArgs<T> a{};
  a.nth = h->g.ntheta;
  a.ns = h->g.ns;
  a.seg = h->seg;
  a.rows_per_warp = p.rows_per_warp;
  a.nbuf = p.nbuf;
  a.bulk = p.bulk;
  a.ncells = nc;
  a.T_int = Tint;
  a.ds = h->g.L / h->g.ns;
  a.dth = dth;
  a.mb = (T*)h->mb;
  a.psi = (const T*)h->psi[h->parity];
  a.nb_out = (T*)h->nb[h->parity];
  a.mf = (T*)h->mf;
  a.c = (T*)h->c;
  a.mtot = (const T*)h->mtot;
  a.nsteps = h->local_n;
  a.prm = h->prm;
  a.masscorr = masscorr;
  CK((mm::launch_motor_local<T, V>(a, p.grid, p.block, p.smem, h->stream)));
  return MM_OK;
}

}  // namespace

extern "C" {

mm_status mm_motor_local(mm_handle* h, double T, const int* nsteps_in, int* nsteps_out,
                         int on_device) {
  MM_TRACE("mm_motor_local");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!finite_pos(T)) return fail(h, MM_ERR_INVALID, "T must be finite and > 0");
  if (!h->have_state) return fail(h, MM_ERR_STATE, "no state: call mm_set_state first");
  if (h->rec.active)
    return fail(h, MM_ERR_STATE,
                "the local-step motor update is not differentiated: end the adjoint recording first");
  if (h->tangent)
    return fail(h, MM_ERR_STATE, "the local-step motor update is not differentiated: end the tangent first");
  if (h->anchors || h->capture)
    return fail(h, MM_ERR_UNSUPPORTED,
                "local substeps need independent cells: not available with non-local anchors "
                "or a capture radius");
  DeviceGuard dg(h->device);
  const size_t nc = (size_t)h->ncells;
  if (!h->local_n) CK(cudaMalloc((void**)&h->local_n, nc * sizeof(int)));
  const int* nin = nullptr;
  if (nsteps_in) {
    if (on_device) {
      nin = nsteps_in;
    } else {
      for (size_t i = 0; i < nc; ++i)
        if (nsteps_in[i] < 1 || nsteps_in[i] > mm::kMaxLocalSteps)
          return fail(h, MM_ERR_INVALID, "a substep count is outside 1..2^20");
      CK(cudaMemcpyAsync(h->local_n, nsteps_in, nc * sizeof(int), cudaMemcpyHostToDevice,
                         h->stream));
      nin = h->local_n;  // read and rewritten in place by the same thread
    }
  }
  mm_status st;
  if (h->prec == MM_FP64)
    st = h->V == 2 ? run_local<double, 2>(h, T, nin) : run_local<double, 1>(h, T, nin);
  else
    st = h->V == 8   ? run_local<float, 8>(h, T, nin)
         : h->V == 4 ? run_local<float, 4>(h, T, nin)
                     : run_local<float, 1>(h, T, nin);
  if (st != MM_OK) return st;
  if (nsteps_out) {
    CK(cudaMemcpyAsync(nsteps_out, h->local_n, nc * sizeof(int),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!on_device) return check_status(h);
  }
  return MM_OK;
}

}  // extern "C"
