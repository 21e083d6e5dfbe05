// Host side of the C ABI (include/mm.h): handle life cycle, state transfer,
// velocity and adaptive substep, the substep launch plan (captured CUDA
// graphs), the moments, and the adjoint recording and reverse sweep.
#include <array>

#include "mm_host.h"

using namespace mmh;

void mm::set_thread_error(const char* msg) { g_create_error = msg; }

namespace mmh {

mm_status check_rates(const mm_rates* r, mm_handle* h) {
  if (!r) return fail(h, MM_ERR_INVALID, "rates is NULL");
  const double v[8] = {r->v_walk, r->k_on, r->k_off, r->glide,
                       r->v_sp, r->force_scale, r->ell, r->cfl};
  for (double x : v)
    if (!std::isfinite(x)) return fail(h, MM_ERR_INVALID, "a rate is not finite");
  if (r->k_on < 0.0 || r->k_off < 0.0) return fail(h, MM_ERR_INVALID, "k_on and k_off must be >= 0");
  if (!(r->cfl > 0.0)) return fail(h, MM_ERR_INVALID, "cfl must be > 0");
  if (r->v_walk < 0.0)
    return fail(h, MM_ERR_UNSUPPORTED, "v_walk < 0 (walking toward the minus end) is not supported");
  return MM_OK;
}

void free_recording(mm_handle* h) {
  Recording& R = h->rec;
  if (R.slab) cudaFree(R.slab);
  for (void* p : R.vblocks) cudaFree(p);
  if (R.rstream) cudaStreamDestroy(R.rstream);
  cudaEvent_t evs[5] = {R.ev_start, R.ev_rep[0], R.ev_rep[1], R.ev_rev[0], R.ev_rev[1]};
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  h->rec = Recording();
}

mm_status free_all(mm_handle* h) {
  free_recording(h);
  fluid_free(h);
  capture_free(h);
  tangent_free(h);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  if (h->diff_tab) cudaFree(h->diff_tab);
  if (h->local_n) cudaFree(h->local_n);
  void* anc[8] = {h->anc_off,  h->anc_cacc,  h->anc_fsc,    h->anc_flags,
                  h->anc_widx, h->anc_wtab,  h->anc_runend, h->anc_rtab};
  for (void* p : anc)
    if (p) cudaFree(p);
  void* ptrs[] = {h->mb,  h->psi[0], h->psi[1], h->nb[0],   h->nb[1],
                  h->mf,  h->c,      h->mtot,   h->u,       h->u64,    h->trig,
                  h->trig64, h->partial, h->fields, h->staging, h->prm, h->ucell};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->cap) cudaStreamDestroy(h->cap);
  return MM_OK;
}

mm_status upload_params(mm_handle* h) {
  DevParams p{};
  p.dt = h->dt;
  p.psi_scale = 1.0;
  p.v_walk = h->r.v_walk;
  p.cw = walk_cw(h);
  p.k_on = h->r.k_on;
  p.k_off = h->r.k_off;
  p.glide = h->r.glide;
  p.v_sp = h->r.v_sp;
  p.force_scale = h->r.force_scale;
  p.ell = h->r.ell;
  p.wait_limit = 1u << 22;
  p.debug_flags = 0;
  CK(cudaMemcpy(h->prm, &p, sizeof(p), cudaMemcpyHostToDevice));
  return MM_OK;
}

template <typename T>
StepArgs<T> step_args(mm_handle* h, int parity) {
  StepArgs<T> a{};
  a.nx = h->g.nx;
  a.ny = h->g.ny;
  a.nth = h->g.ntheta;
  a.ns = h->g.ns;
  a.seg = h->seg;
  a.stages = h->stages;
  a.chunk_rows = h->chunk_rows;
  a.chunks_per_cell = h->chunks_per_cell;
  a.nb_tma = h->tma && ((size_t)h->g.ntheta * h->tsz) % 16 == 0;
  a.ncells = h->ncells;
  a.inv_dx = (double)h->g.nx;
  a.inv_dy = (double)h->g.ny;
  a.dth = 2.0 * kPi / h->g.ntheta;
  a.inv_dth = 1.0 / a.dth;
  a.ds = h->g.L / h->g.ns;
  a.L = h->g.L;
  a.f_inv_dx = (float)a.inv_dx;
  a.f_inv_dy = (float)a.inv_dy;
  a.f_inv_dth = (float)a.inv_dth;
  a.f_dth = (float)a.dth;
  a.f_ds = (float)a.ds;
  a.mb_in = (const T*)h->mb;
  a.mb_out = (T*)h->mb;
  a.psi_in = (const T*)h->psi[parity];
  a.psi_out = (T*)h->psi[parity ^ 1];
  a.nb_in = (const T*)h->nb[parity];
  a.nb_out = (T*)h->nb[parity ^ 1];
  a.mf_in = (const T*)h->mf;
  a.mf_out = (T*)h->mf;
  a.c = (T*)h->c;
  a.cpre_out = nullptr;
  a.mtot = (const T*)h->mtot;
  a.ucell = (const T*)h->ucell;
  a.trig = (const T*)h->trig;
  a.partial = h->partial;
  a.prm = h->prm;
  a.mass_correct = h->prec == MM_FP32_MIXED ? 1 : 0;
  return a;
}

template StepArgs<float> step_args<float>(mm_handle*, int);
template StepArgs<double> step_args<double>(mm_handle*, int);

cudaError_t launch_one(mm_handle* h, int parity, cudaStream_t s) {
  if (h->anchors) return launch_anchor_substep(h, parity, s);
  if (h->capture) return launch_capture_substep(h, parity, s);
  if (h->tangent) return launch_tangent_substep(h, parity, s);
  if (h->prec == MM_FP64) {
    StepArgs<double> a = step_args<double>(h, parity);
    return h->V == 2 ? mm::launch_substep<double, 2>(a, h->grid_step, h->block, h->smem, h->tma, s)
                     : mm::launch_substep<double, 1>(a, h->grid_step, h->block, h->smem, h->tma, s);
  }
  StepArgs<float> a = step_args<float>(h, parity);
  if (h->V == 8) return mm::launch_substep<float, 8>(a, h->grid_step, h->block, h->smem, h->tma, s);
  return h->V == 4 ? mm::launch_substep<float, 4>(a, h->grid_step, h->block, h->smem, h->tma, s)
                   : mm::launch_substep<float, 1>(a, h->grid_step, h->block, h->smem, h->tma, s);
}

// Launch plan of the substep kernel: one warp per cell, the cell's rows
// streamed in chunks of chunk_rows rows (at most kChunkBytes) through a ring of
// `stages` shared-memory stages per warp filled by bulk copies (TMA) when an
// s-row is a whole number of 16-byte vectors; otherwise rows are read from
// global memory directly.

// One substep with explicit state buffers (recomputing a recorded segment).
struct StepPtrs {
  const void *psi_in, *nb_in, *mb_in, *mf_in, *ucell;
  void *psi_out, *nb_out, *mb_out, *mf_out, *c, *cpre;
};
template <typename T>
StepArgs<T> step_args_ptrs(mm_handle* h, const StepPtrs& p) {
  StepArgs<T> a = step_args<T>(h, 0);
  a.psi_in = (const T*)p.psi_in;
  a.psi_out = (T*)p.psi_out;
  a.nb_in = (const T*)p.nb_in;
  a.nb_out = (T*)p.nb_out;
  a.mb_in = (const T*)p.mb_in;
  a.mb_out = (T*)p.mb_out;
  a.mf_in = (const T*)p.mf_in;
  a.mf_out = (T*)p.mf_out;
  a.c = (T*)p.c;
  a.cpre_out = (T*)p.cpre;
  a.ucell = (const T*)p.ucell;
  return a;
}
// (direct launches of the recording and the reverse sweep: overlapped with
// the previous kernel of the stream)
cudaError_t launch_ptrs(mm_handle* h, const StepPtrs& p, cudaStream_t s) {
  const int g = h->grid_step, b = h->block;
  const size_t sm = h->smem;
  if (h->prec == MM_FP64) {
    StepArgs<double> a = step_args_ptrs<double>(h, p);
    return h->V == 2 ? mm::launch_substep_overlapped<double, 2>(a, g, b, sm, h->tma, s)
                     : mm::launch_substep_overlapped<double, 1>(a, g, b, sm, h->tma, s);
  }
  StepArgs<float> a = step_args_ptrs<float>(h, p);
  if (h->V == 8) return mm::launch_substep_overlapped<float, 8>(a, g, b, sm, h->tma, s);
  return h->V == 4 ? mm::launch_substep_overlapped<float, 4>(a, g, b, sm, h->tma, s)
                   : mm::launch_substep_overlapped<float, 1>(a, g, b, sm, h->tma, s);
}

mm_status configure(mm_handle* h) {
  const int ns = h->g.ns, nth = h->g.ntheta;
  // values per lane: the widest instantiated vector that divides ns -- float64
  // {2, 1}, float32 {8, 4, 1} (two 16-byte vectors, one, or scalar lanes)
  h->V = 1;
  if (h->prec == MM_FP64) {
    if (ns % 2 == 0) h->V = 2;
  } else if (MM_FP32_VMAX >= 8 && ns % 8 == 0) {
    h->V = 8;
  } else if (ns % 4 == 0) {
    h->V = 4;
  }
  const int nl = ns / h->V;
  if (nl > 32)
    return fail(h, MM_ERR_UNSUPPORTED, "ns too large: one s-row must fit in one warp");
  int seg = 1;
  while (seg < nl) seg <<= 1;
  h->seg = seg;
  h->tma = ((size_t)h->V * h->tsz) % 16 == 0;
  const size_t row_bytes = (size_t)ns * h->tsz;
  int ch = 1;
  while (ch < nth && (nth % ch != 0 || (size_t)(nth / ch) * row_bytes > kChunkBytes)) ++ch;
  h->chunks_per_cell = ch;
  h->chunk_rows = nth / ch;
  const size_t chunk_bytes = (size_t)h->chunk_rows * row_bytes;
  int S = (int)(kWarpInflightBytes / std::max<size_t>(chunk_bytes, 1));
  S = std::max(2, std::min(8, S));
  h->stages = h->tma ? S : 1;
  const size_t per_warp =
      mm::step_smem_per_warp(h->stages, h->tma ? h->chunk_rows * ns : 0, nth, (int)h->tsz);
  const int wpb = (int)std::min<size_t>(kMaxWarpsPerBlock, kSmemBudget / per_warp);
  if (wpb < 1) return fail(h, MM_ERR_UNSUPPORTED, "ntheta too large for the shared-memory plan");
  h->block = 32 * wpb;
  h->smem = (size_t)wpb * per_warp;
  int bps = 0;
  cudaError_t e;
  if (h->prec == MM_FP64)
    e = h->V == 2 ? mm::substep_prepare<double, 2>(h->block, h->smem, h->tma, &bps)
                  : mm::substep_prepare<double, 1>(h->block, h->smem, h->tma, &bps);
  else
    e = h->V == 8 ? mm::substep_prepare<float, 8>(h->block, h->smem, h->tma, &bps)
        : h->V == 4 ? mm::substep_prepare<float, 4>(h->block, h->smem, h->tma, &bps)
                    : mm::substep_prepare<float, 1>(h->block, h->smem, h->tma, &bps);
  CK(e);
  if (bps < 1) return fail(h, MM_ERR_UNSUPPORTED, "substep kernel cannot be resident");
  long long g = (long long)bps * h->sms;
  const long long need = (h->ncells + wpb - 1) / wpb;
  if (g > need) g = need;
  h->grid_step = (int)g;
  long long gm = 8LL * h->sms;  // blocks of 4 warps, one warp per cell
  if (gm > (h->ncells + 3) / 4) gm = (h->ncells + 3) / 4;
  h->grid_mom = (int)gm;
  h->npartial = std::max(h->grid_step * wpb, 4 * h->grid_mom);
  return MM_OK;
}

// Read and clear the device status word; a set bit means a bounded device
// wait gave up during an earlier kernel.
mm_status check_status(mm_handle* h) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, &h->prm->status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st) {
    // clear the status, and the last-warp counters a warp that gave up early
    // may have left part-way
    const int zero = 0;
    const unsigned int zeros[2] = {0u, 0u};
    CK(cudaMemcpy(&h->prm->status, &zero, sizeof zero, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(&h->prm->counter, zeros, sizeof zeros, cudaMemcpyHostToDevice));
    if (st & 8)
      return fail(h, MM_ERR_TIMEOUT,
                  "a bounded wait in the substep kernel gave up and so did the wait for its copies "
                  "in flight; the state is invalid and later launches on this device are suspect");
    if (st & 1)
      return fail(h, MM_ERR_TIMEOUT, "a bounded wait in the substep kernel gave up; the state is invalid");
    if (st & 4)
      return fail(h, MM_ERR_INVALID,
                  "mm_motor_local: a substep count came out of 1..2^20; the motor state was left unchanged");
    return fail(h, MM_ERR_NONFINITE, "the substep rule found no positive finite rate");
  }
  return MM_OK;
}

// Copy a float64 array of n elements from (host or device) src into the
// device array dst of the handle's precision, in staging chunks for host src.
mm_status put_array(mm_handle* h, void* dst, const double* src, size_t n, int on_device) {
  if (h->prec == MM_FP64) {
    CK(cudaMemcpyAsync(dst, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream));
    return MM_OK;
  }
  float* d = (float*)dst;
  if (on_device) {
    CK(mm::launch_convert<float, double>(d, src, n, nullptr, h->stream));
    return MM_OK;
  }
  for (size_t off = 0; off < n; off += h->staging_n) {
    size_t m = std::min(h->staging_n, n - off);
    CK(cudaMemcpyAsync(h->staging, src + off, m * 8, cudaMemcpyHostToDevice, h->stream));
    CK(mm::launch_convert<float, double>(d + off, h->staging, m, nullptr, h->stream));
  }
  return MM_OK;
}

// Inverse of put_array; scale (device pointer or NULL) multiplies on export.
mm_status get_array(mm_handle* h, double* dst, const void* src, size_t n, int on_device,
                    const double* scale) {
  if (h->prec == MM_FP64 && !scale) {
    CK(cudaMemcpyAsync(dst, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    return MM_OK;
  }
  if (on_device) {
    if (h->prec == MM_FP64)
      CK(mm::launch_convert<double, double>(dst, (const double*)src, n, scale, h->stream));
    else
      CK(mm::launch_convert<double, float>(dst, (const float*)src, n, scale, h->stream));
    return MM_OK;
  }
  for (size_t off = 0; off < n; off += h->staging_n) {
    size_t m = std::min(h->staging_n, n - off);
    if (h->prec == MM_FP64)
      CK(mm::launch_convert<double, double>(h->staging, (const double*)src + off, m, scale, h->stream));
    else
      CK(mm::launch_convert<double, float>(h->staging, (const float*)src + off, m, scale, h->stream));
    CK(cudaMemcpyAsync(dst + off, h->staging, m * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  return MM_OK;
}

mm_status run_init(mm_handle* h) {
  if (h->anchors) return run_init_anchor(h);
  if (h->capture) return run_init_capture(h);
  const double ds = h->g.L / h->g.ns, dth = 2.0 * kPi / h->g.ntheta;
  cudaError_t e;
  if (h->prec == MM_FP64)
    e = mm::launch_init_cells<double>((double*)h->mb, (const double*)h->psi[h->parity],
                                      (double*)h->nb[h->parity], (double*)h->mf, (double*)h->c,
                                      (const double*)h->mtot, h->ncells,
                                      h->g.ntheta, h->g.ns, ds, dth, h->stream);
  else
    e = mm::launch_init_cells<float>((float*)h->mb, (const float*)h->psi[h->parity],
                                     (float*)h->nb[h->parity], (float*)h->mf, (float*)h->c,
                                     (const float*)h->mtot, h->ncells,
                                     h->g.ntheta, h->g.ns, ds, dth, h->stream);
  CK(e);
  return MM_OK;
}

mm_status run_moments(mm_handle* h) {
  // with a capture radius the rows are the per-node totals over the anchors
  mm_status st;
  if (h->capture && (st = capture_rows(h)) != MM_OK) return st;
  const double dth = 2.0 * kPi / h->g.ntheta, ds = h->g.L / h->g.ns;
  const double dA = (1.0 / h->g.nx) * (1.0 / h->g.ny);
  // the moments kernel reads rows with at most 4 values per lane
  const int mV = h->V;  // the substep's vector width (float32 8 or 4, float64 2 or 1)
  int mseg = 1;
  while (mseg < h->g.ns / mV) mseg <<= 1;
  cudaError_t e;
  if (h->prec == MM_FP64)
    e = mm::launch_moments<double>((const double*)h->psi[h->parity], (const double*)h->mb,
                                   (const double*)h->mf, (const double*)h->c, h->trig64, h->ncells, h->g.ntheta, h->g.ns, mV,
                                   mseg, dth, ds,
                                   h->g.L, dA, h->fields, h->partial, h->grid_mom, h->prm,
                                   h->stream);
  else
    e = mm::launch_moments<float>((const float*)h->psi[h->parity], (const float*)h->mb,
                                  (const float*)h->mf, (const float*)h->c, h->trig64, h->ncells, h->g.ntheta, h->g.ns, mV,
                                  mseg, dth, ds,
                                  h->g.L, dA, h->fields, h->partial, h->grid_mom, h->prm,
                                  h->stream);
  CK(e);
  // with anchors (or a capture radius) the motor force of Eq. 10 acts in the
  // cells under the heads
  if (h->anchors || h->capture) return anchor_force(h);
  return MM_OK;
}

mm_status rec_push_version(mm_handle* h);
mm_status rec_micro_step(mm_handle* h, int n);
int rec_tail_start(const Recording& R);

}  // namespace mmh

extern "C" {

mm_status mm_create(const mm_grid* grid, const mm_rates* rates, mm_precision prec, void* stream,
                    mm_handle** out) {
  MM_TRACE("mm_create");
  g_create_error.clear();
  if (!grid || !out) return fail(nullptr, MM_ERR_INVALID, "grid or out is NULL");
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->ntheta < 1 || grid->ns < 1 || !finite_pos(grid->L))
    return fail(nullptr, MM_ERR_INVALID, "grid sizes must be >= 1 and L > 0");
  if (prec != MM_FP64 && prec != MM_FP32_MIXED)
    return fail(nullptr, MM_ERR_INVALID, "unknown precision");
  if (grid->ntheta > 1024) return fail(nullptr, MM_ERR_UNSUPPORTED, "ntheta > 1024");
  {
    mm_status st = check_rates(rates, nullptr);
    if (st != MM_OK) return st;
  }
  const int vmax = prec == MM_FP64 ? 2 : 4;
  if (grid->ns > 32 * vmax)
    return fail(nullptr, MM_ERR_UNSUPPORTED, prec == MM_FP64 ? "ns > 64 in MM_FP64" : "ns > 128 in MM_FP32_MIXED");
  if ((long long)grid->nx * grid->ny > 0x7fffffffLL)
    return fail(nullptr, MM_ERR_UNSUPPORTED, "more than 2^31 - 1 cells");

  mm_handle* h = new mm_handle();
  h->g = *grid;
  h->r = *rates;
  h->prec = prec;
  h->stream = (cudaStream_t)stream;
  h->tsz = prec == MM_FP64 ? 8 : 4;
  h->ncells = (long long)grid->nx * grid->ny;
  h->rows = (size_t)h->ncells * grid->ntheta;
  h->mbn = h->rows * grid->ns;
  auto bail = [&](mm_status st) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return st;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    cuda_fail(h, "cudaGetDevice", e);
    return bail(MM_ERR_CUDA);
  }
  e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    cuda_fail(h, "cudaDeviceGetAttribute", e);
    return bail(MM_ERR_CUDA);
  }
  {
    mm_status st = configure(h);
    if (st != MM_OK) return bail(st);
  }
  const size_t nc = (size_t)h->ncells;
  // float64 staging of host transfers: the largest array, up to 32 MiB
  h->staging_n = std::min(kStagingDoubles, std::max(h->mbn, 12 * nc));
  const size_t need = h->mbn * h->tsz + 2 * h->rows * h->tsz + 3 * h->rows * 8 + 3 * nc * 8 +
                      2 * nc * (h->tsz + 8) + 12 * nc * (8 + h->tsz) + h->staging_n * 8 +
                      (size_t)h->npartial * 8 * 8 + 4 * grid->ntheta * (h->tsz + 8) + 4096;
  size_t freeb = 0, totalb = 0;
  e = cudaMemGetInfo(&freeb, &totalb);
  if (e != cudaSuccess) {
    cuda_fail(h, "cudaMemGetInfo", e);
    return bail(MM_ERR_CUDA);
  }
  if (need > freeb) {
    char buf[160];
    snprintf(buf, sizeof buf, "needs %zu bytes of device memory, %zu free", need, freeb);
    fail(h, MM_ERR_OOM, buf);
    return bail(MM_ERR_OOM);
  }
#define ALLOC(ptr, bytes)                                        \
  do {                                                           \
    e = cudaMalloc((void**)&(ptr), (bytes));                     \
    if (e != cudaSuccess) {                                      \
      cuda_fail(h, "cudaMalloc " #ptr, e);                       \
      return bail(e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA); \
    }                                                            \
  } while (0)
  ALLOC(h->mb, h->mbn * h->tsz);
  ALLOC(h->psi[0], h->rows * h->tsz);
  ALLOC(h->psi[1], h->rows * h->tsz);
  ALLOC(h->nb[0], h->rows * h->tsz);
  ALLOC(h->nb[1], h->rows * h->tsz);
  ALLOC(h->mf, nc * h->tsz);
  ALLOC(h->c, nc * h->tsz);
  ALLOC(h->mtot, nc * h->tsz);
  ALLOC(h->u, 2 * nc * h->tsz);
  ALLOC(h->ucell, 12 * nc * h->tsz);
  ALLOC(h->u64, 2 * nc * 8);
  ALLOC(h->trig, 4 * (size_t)grid->ntheta * h->tsz);
  ALLOC(h->trig64, 24 * (size_t)grid->ntheta * 8);
  ALLOC(h->partial, (size_t)h->npartial * 8 * 8);
  ALLOC(h->fields, 12 * nc * 8);
  ALLOC(h->staging, h->staging_n * 8);
  ALLOC(h->prm, sizeof(DevParams));
#undef ALLOC
  e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cuda_fail(h, "cudaStreamCreate", e);
    return bail(MM_ERR_CUDA);
  }
  // trigonometric tables: cos, sin at theta_k and at the faces theta_{k+1/2}
  const int nth = grid->ntheta;
  std::vector<double> tr(4 * (size_t)nth);
  const double dth = 2.0 * kPi / nth;
  for (int k = 0; k < nth; ++k) {
    tr[k] = std::cos(k * dth);
    tr[nth + k] = std::sin(k * dth);
    tr[2 * nth + k] = std::cos((k + 0.5) * dth);
    tr[3 * nth + k] = std::sin((k + 0.5) * dth);
  }
  // moment weights after the four trigonometric rows (see k_moments), then
  // the same ten weights split into float pairs (hi, lo) for the float32 form
  std::vector<double> tw(24 * (size_t)nth);
  std::copy(tr.begin(), tr.end(), tw.begin());
  for (int k = 0; k < nth; ++k) {
    const double c = tr[k], s = tr[nth + k];
    double* w = tw.data() + 4 * (size_t)nth;
    w[k] = dth;
    w[nth + k] = c * dth;
    w[2 * nth + k] = s * dth;
    w[3 * nth + k] = (c * c - 0.5) * dth;
    w[4 * nth + k] = c * s * dth;
    w[5 * nth + k] = c;
    w[6 * nth + k] = s;
    w[7 * nth + k] = c * c * dth;
    w[8 * nth + k] = c * s * dth;
    w[9 * nth + k] = s * s * dth;
  }
  {
    float* wf = reinterpret_cast<float*>(tw.data() + 14 * (size_t)nth);
    const double* w = tw.data() + 4 * (size_t)nth;
    for (size_t i = 0; i < 10 * (size_t)nth; ++i) {
      const float hi = (float)w[i];
      wf[2 * i] = hi;
      wf[2 * i + 1] = (float)(w[i] - (double)hi);
    }
  }
  e = cudaMemcpy(h->trig64, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (prec == MM_FP64) {
      e = cudaMemcpy(h->trig, tr.data(), tr.size() * 8, cudaMemcpyHostToDevice);
    } else {
      std::vector<float> tf(tr.begin(), tr.end());
      e = cudaMemcpy(h->trig, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) {
    cuda_fail(h, "upload trig tables", e);
    return bail(MM_ERR_CUDA);
  }
  if (upload_params(h) != MM_OK) return bail(MM_ERR_CUDA);
  // default state: psi = 1/(2 pi), Mb = 0, M = 1, u = 0
  {
    std::vector<double> zeros(2 * nc, 0.0);
    e = cudaMemcpy(h->u64, zeros.data(), 2 * nc * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->u, 0, 2 * nc * h->tsz);
    if (e == cudaSuccess) e = cudaMemset(h->ucell, 0, 12 * nc * h->tsz);
    if (e == cudaSuccess) e = cudaMemset(h->mb, 0, h->mbn * h->tsz);
    if (e == cudaSuccess) e = cudaMemset(h->partial, 0, (size_t)h->npartial * 64);
    if (e != cudaSuccess) {
      cuda_fail(h, "initial state", e);
      return bail(MM_ERR_CUDA);
    }
    std::vector<double> p0(h->rows, 1.0 / (2.0 * kPi));
    if (mm_set_state(h, p0.data(), nullptr, nullptr, 0) != MM_OK) return bail(MM_ERR_CUDA);
    h->have_state = false;
  }
  *out = h;
  return MM_OK;
}

mm_status mm_destroy(mm_handle* h) {
  if (!h) return MM_ERR_INVALID;
  if (h->owner) return fail(h, MM_ERR_INVALID, "a batch member: destroy its batch instead");
  DeviceGuard dg(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  batch_free(h);
  free_all(h);
  delete h;
  return MM_OK;
}

mm_status mm_set_stream(mm_handle* h, void* stream) {
  if (!h) return MM_ERR_INVALID;
  h->stream = (cudaStream_t)stream;
  if (h->batch)
    for (mm_handle* m : batch_members(h)) m->stream = (cudaStream_t)stream;
  return MM_OK;
}

mm_status mm_set_rates(mm_handle* h, const mm_rates* rates) {
  MM_TRACE("mm_set_rates");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  mm_status st = check_rates(rates, h);
  if (st != MM_OK) return st;
  if (h->capture && rates->ell != h->r.ell)
    return fail(h, MM_ERR_STATE,
                "l/L fixes the capture template: switch the capture radius off, change l/L, set it again");
  DeviceGuard dg(h->device);
  // the substeps recorded so far ran with the old rates, while the replays and
  // the reverse kernels would read the new ones: new rates end a recording
  h->rec.active = false;
  h->r = *rates;
  CK(cudaStreamSynchronize(h->stream));
  double v[7] = {rates->v_walk, rates->k_on, rates->k_off, rates->glide,
                 rates->v_sp, rates->force_scale, rates->ell};
  CK(cudaMemcpy(&h->prm->v_walk, v, sizeof v, cudaMemcpyHostToDevice));
  const double cw = walk_cw(h);
  CK(cudaMemcpy(&h->prm->cw, &cw, sizeof cw, cudaMemcpyHostToDevice));
  if (h->anchors) {  // l/L moves the anchors: new table, C and Mf of the state under it
    if ((st = anchor_table(h)) != MM_OK) return st;
    if (h->have_state) return run_init_anchor(h);
  }
  return MM_OK;
}

mm_status mm_set_state(mm_handle* h, const double* psi, const double* mb, const double* mtot,
                       int on_device) {
  MM_TRACE("mm_set_state");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!psi) return fail(h, MM_ERR_INVALID, "psi is NULL");
  DeviceGuard dg(h->device);
  mm_status st;
  h->rec.active = false;  // a new state ends an adjoint recording (its memory is kept)
  h->parity = 0;
  if ((st = put_array(h, h->psi[0], psi, h->rows, on_device)) != MM_OK) return st;
  // with a capture radius Mb is [cells][nconf] (anchor-major, template order)
  void* mbd = h->capture ? h->rc_mb : h->mb;
  const size_t mbn = h->capture ? (size_t)h->ncells * h->rc_nconf : h->mbn;
  if (mb) {
    if ((st = put_array(h, mbd, mb, mbn, on_device)) != MM_OK) return st;
  } else {
    CK(cudaMemsetAsync(mbd, 0, mbn * h->tsz, h->stream));
  }
  if (mtot) {
    if ((st = put_array(h, h->mtot, mtot, (size_t)h->ncells, on_device)) != MM_OK) return st;
  } else {
    std::vector<double> ones((size_t)h->ncells, 1.0);
    if ((st = put_array(h, h->mtot, ones.data(), ones.size(), 0)) != MM_OK) return st;
    CK(cudaStreamSynchronize(h->stream));
  }
  const double one = 1.0;
  CK(cudaMemcpyAsync(&h->prm->psi_scale, &one, 8, cudaMemcpyHostToDevice, h->stream));
  if (h->tangent && (st = tangent_zero(h)) != MM_OK) return st;  // the tangent starts at zero
  if ((st = run_init(h)) != MM_OK) return st;
  // reference filament number for the float32 mass correction
  if ((st = run_moments(h)) != MM_OK) return st;
  double sum_psi = 0.0;
  CK(cudaMemcpyAsync(&sum_psi, &h->prm->sum_psi, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (!std::isfinite(sum_psi)) return fail(h, MM_ERR_NONFINITE, "psi sums to a non-finite value");
  CK(cudaMemcpy(&h->prm->mass0, &sum_psi, 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(&h->prm->mass, &sum_psi, 8, cudaMemcpyHostToDevice));
  h->have_state = true;
  return MM_OK;
}

mm_status mm_get_state(mm_handle* h, double* psi, double* mb, double* mf, double* c,
                       int on_device) {
  MM_TRACE("mm_get_state");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  DeviceGuard dg(h->device);
  mm_status st;
  const double* scale = h->prec == MM_FP32_MIXED ? &h->prm->psi_scale : nullptr;
  if (psi && (st = get_array(h, psi, h->psi[h->parity], h->rows, on_device, scale)) != MM_OK)
    return st;
  if (mb && (st = get_array(h, mb, h->capture ? h->rc_mb : h->mb,
                            h->capture ? (size_t)h->ncells * h->rc_nconf : h->mbn, on_device,
                            nullptr)) != MM_OK)
    return st;
  if (mf && (st = get_array(h, mf, h->mf, (size_t)h->ncells, on_device, nullptr)) != MM_OK) return st;
  if (c && (st = get_array(h, c, h->c, (size_t)h->ncells, on_device, nullptr)) != MM_OK) return st;
  return check_status(h);
}

mm_status mm_set_velocity(mm_handle* h, const double* u, int on_device) {
  MM_TRACE("mm_set_velocity");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!u) return fail(h, MM_ERR_INVALID, "u is NULL");
  DeviceGuard dg(h->device);
  const size_t n = 2 * (size_t)h->ncells;
  CK(cudaMemcpyAsync(h->u64, u, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     h->stream));
  return velocity_update(h);
}

}  // extern "C"

namespace mmh {

// The velocity in h->u64 becomes the one in effect: its state-precision copy,
// the cell velocities and gradients, and the adaptive substep.
mm_status velocity_update(mm_handle* h) {
  const size_t n = 2 * (size_t)h->ncells;
  if (h->prec == MM_FP64)
    CK(cudaMemcpyAsync(h->u, h->u64, n * 8, cudaMemcpyDeviceToDevice, h->stream));
  else
    CK(mm::launch_convert<float, double>((float*)h->u, h->u64, n, nullptr, h->stream));
  if (h->prec == MM_FP64)
    CK(mm::launch_prep_ucell<double>((double*)h->ucell, h->u64, h->ncells, h->g.nx, h->g.ny,
                                     (double)h->g.nx, (double)h->g.ny, h->stream));
  else
    CK(mm::launch_prep_ucell<float>((float*)h->ucell, h->u64, h->ncells, h->g.nx, h->g.ny,
                                    (double)h->g.nx, (double)h->g.ny, h->stream));
  // maxima of the substep rule on the device, the rule itself in float64 here
  CK(cudaMemsetAsync(h->prm->dtmax, 0, sizeof(h->prm->dtmax), h->stream));
  const double dth = 2.0 * kPi / h->g.ntheta;
  cudaError_t e;
  if (h->prec == MM_FP64)
    e = mm::launch_dt_max<double>((const double*)h->psi[h->parity], (const double*)h->nb[h->parity],
                                  (const double*)h->u, (const double*)h->trig, h->ncells, h->g.nx,
                                  h->g.ny, h->g.ntheta, (double)h->g.nx, (double)h->g.ny, 1.0 / dth,
                                  dth, h->r.glide, h->r.v_sp, h->prm, h->stream);
  else
    e = mm::launch_dt_max<float>((const float*)h->psi[h->parity], (const float*)h->nb[h->parity],
                                 (const float*)h->u, (const float*)h->trig, h->ncells, h->g.nx,
                                 h->g.ny, h->g.ntheta, (double)h->g.nx, (double)h->g.ny, 1.0 / dth,
                                 dth, h->r.glide, h->r.v_sp, h->prm, h->stream);
  CK(e);
  CK(mm::launch_dt_finalize(h->prm, h->g.L / h->g.ns, h->g.L, h->r.cfl, h->stream));
  h->have_vel = true;
  h->have_dt = true;
  if (h->rec.active) return rec_push_version(h);
  return MM_OK;
}

}  // namespace mmh

extern "C" {

mm_status mm_get_dt(mm_handle* h, double* dt) {
  if (!h || !dt) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!h->have_dt) return fail(h, MM_ERR_STATE, "no dt yet: call mm_set_velocity or mm_set_dt");
  DeviceGuard dg(h->device);
  CK(cudaMemcpyAsync(&h->dt, &h->prm->dt, 8, cudaMemcpyDeviceToHost, h->stream));
  mm_status st = check_status(h);
  if (st != MM_OK) return st;
  *dt = h->dt;
  return MM_OK;
}

mm_status mm_set_dt(mm_handle* h, double dt) {
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!finite_pos(dt)) return fail(h, MM_ERR_INVALID, "dt must be finite and > 0");
  DeviceGuard dg(h->device);
  h->dt = dt;
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(&h->prm->dt, &h->dt, 8, cudaMemcpyHostToDevice));
  h->have_dt = true;
  if (h->rec.active) return rec_push_version(h);
  return MM_OK;
}

mm_status mm_micro_step(mm_handle* h, int n) {
  MM_TRACE("mm_micro_step");
  if (!h) return MM_ERR_INVALID;
  if (n < 0) return fail(h, MM_ERR_INVALID, "n_substeps < 0");
  if (n == 0) return MM_OK;
  if (h->batch) return batch_micro_step(h, n);
  if (!h->have_state) return fail(h, MM_ERR_STATE, "no state: call mm_set_state first");
  if (!h->have_vel) return fail(h, MM_ERR_STATE, "no velocity: call mm_set_velocity first");
  if (!h->have_dt) return fail(h, MM_ERR_STATE, "no dt");
  DeviceGuard dg(h->device);
  if (h->rec.active) return rec_micro_step(h, n);
  return launch_substeps(h, n);
}

}  // extern "C"

namespace mmh {

// n substeps on the live state: one captured CUDA graph per (n, parity),
// replayed (direct launches if graphs are off).
mm_status launch_substeps(mm_handle* h, int n) {
  if (!h->use_graphs) {
    for (int i = 0; i < n; ++i) {
      CK(launch_one(h, h->parity, h->stream));
      h->parity ^= 1;
    }
    return MM_OK;
  }
  const long long key = (long long)n * 2 + h->parity;
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int par = h->parity;
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < n && le == cudaSuccess; ++i) {
      le = launch_one(h, par, h->cap);
      par ^= 1;
    }
    cudaError_t ce = cudaStreamEndCapture(h->cap, &graph);
    if (le != cudaSuccess) return cuda_fail(h, "substep launch during capture", le);
    CK(ce);
    cudaGraphExec_t exec;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    it = h->graphs.emplace(key, exec).first;
  }
  CK(cudaGraphLaunch(it->second, h->stream));
  h->parity ^= (n & 1);
  return MM_OK;
}

}  // namespace mmh

extern "C" {

mm_status mm_diffuse(mm_handle* h, double D_t, double D_r, double dt) {
  MM_TRACE("mm_diffuse");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  if (!std::isfinite(D_t) || !std::isfinite(D_r) || D_t < 0.0 || D_r < 0.0)
    return fail(h, MM_ERR_INVALID, "diffusivities must be finite and >= 0");
  if (!finite_pos(dt)) return fail(h, MM_ERR_INVALID, "dt must be finite and > 0");
  if (!h->have_state) return fail(h, MM_ERR_STATE, "no state: call mm_set_state first");
  if (h->rec.active || h->tangent)
    return fail(h, MM_ERR_STATE,
                "diffusion is not differentiated: end the adjoint recording or the tangent first");
  DeviceGuard dg(h->device);
  const int nx = h->g.nx, ny = h->g.ny, nth = h->g.ntheta;
  if (!h->diff_tab) CK(cudaMalloc((void**)&h->diff_tab, (size_t)(3 * (nth + nx + ny) + 6) * 8));
  struct Dir {
    int mode, n;
    double hh, D;
    double* tab;
  };
  const Dir dirs[3] = {{0, nth, 2.0 * kPi / nth, D_r, h->diff_tab},
                       {1, nx, 1.0 / nx, D_t, h->diff_tab + 3 * nth + 2},
                       {2, ny, 1.0 / ny, D_t, h->diff_tab + 3 * (nth + nx) + 4}};
  double a[3];
  for (int d = 0; d < 3; ++d) a[d] = dirs[d].D * dt / (dirs[d].hh * dirs[d].hh);
  CK(mm::launch_cn_factors(dirs[0].tab, nth, a[0], dirs[1].tab, nx, a[1], dirs[2].tab, ny, a[2],
                           h->stream));
  bool first = true;
  for (int d = 0; d < 3; ++d) {
    if (!(dirs[d].D > 0.0) || dirs[d].n < 2) continue;  // a single point: L = 0
    // the float32 form folds the pending mass-correction factor into psi
    const double* sc = (first && h->prec == MM_FP32_MIXED) ? &h->prm->psi_scale : nullptr;
    cudaError_t e =
        h->prec == MM_FP64
            ? mm::launch_cn_lines<double>((double*)h->psi[h->parity], dirs[d].mode, nx, ny, nth,
                                          dirs[d].tab, dirs[d].n, -0.5 * a[d], 0.5 * a[d], sc,
                                          h->stream)
            : mm::launch_cn_lines<float>((float*)h->psi[h->parity], dirs[d].mode, nx, ny, nth,
                                         dirs[d].tab, dirs[d].n, -0.5 * a[d], 0.5 * a[d], sc,
                                         h->stream);
    CK(e);
    first = false;
  }
  if (!first && h->prec == MM_FP32_MIXED) CK(mm::launch_set_scale_one(&h->prm->psi_scale, h->stream));
  // the coarse density, the Alg. 2 scale-down and the free motors of the new psi
  return run_init(h);
}

mm_status mm_moments(mm_handle* h, mm_moments_out* out) {
  MM_TRACE("mm_moments");
  if (!h || !out) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  DeviceGuard dg(h->device);
  mm_status st;
  if ((st = run_moments(h)) != MM_OK) return st;
  if (out->fields)
    CK(cudaMemcpyAsync(out->fields, h->fields, 12 * (size_t)h->ncells * 8,
                       out->fields_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
  CK(cudaMemcpyAsync(out->scalars, h->prm->scalars, sizeof out->scalars, cudaMemcpyDeviceToHost,
                     h->stream));
  if ((st = check_status(h)) != MM_OK) return st;
  for (double x : out->scalars)
    if (!std::isfinite(x)) return fail(h, MM_ERR_NONFINITE, "a global moment is not finite");
  return MM_OK;
}

mm_status mm_sync(mm_handle* h) {
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return batch_sync(h);
  DeviceGuard dg(h->device);
  return check_status(h);
}

mm_status mm_debug_set(mm_handle* h, unsigned int wait_limit, unsigned int flags) {
  if (!h) return MM_ERR_INVALID;
  if (h->batch) {
    for (mm_handle* m : batch_members(h)) {
      const mm_status st = mm_debug_set(m, wait_limit, flags);
      if (st != MM_OK) {
        h->err = m->err;
        return st;
      }
    }
    return MM_OK;
  }
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(&h->prm->wait_limit, &wait_limit, sizeof wait_limit, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(&h->prm->debug_flags, &flags, sizeof flags, cudaMemcpyHostToDevice));
  return MM_OK;
}

mm_status mm_get_launch_info(mm_handle* h, int* info, int n) {
  if (!h || !info || n < 1) return MM_ERR_INVALID;
  if (h->batch) return batch_launch_info(h, info, n);
  const int v[10] = {h->grid_step, h->block, (int)h->smem, h->tma ? 1 : 0, h->stages,
                     h->chunk_rows, h->chunks_per_cell, h->V, h->seg, h->sms};
  for (int i = 0; i < n && i < 10; ++i) info[i] = v[i];
  return MM_OK;
}

const char* mm_last_error(const mm_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

const char* mm_build_info(void) { return "libmm sm_103a (tcgen05-free streaming stencil path)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint recording and reverse sweep

namespace mmh {

// Sub-buffers of one allocation at 256-byte alignment: a first pass with a
// null base only adds up the size.
struct Carver {
  unsigned char* base = nullptr;
  size_t off = 0;
  void* take(size_t bytes) {
    void* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  }
};

// Velocity block: per-cell velocity data, dt, and the adjoint accumulators.
size_t vblock_bytes(const mm_handle* h) {
  Carver c;
  const size_t nc = (size_t)h->ncells;
  c.take(12 * nc * h->tsz);
  c.take(8);
  c.take(4 * nc * 8);
  c.take(2 * nc * 8);
  return c.off;
}

// Copy the live state into checkpoint i.
mm_status rec_save_checkpoint(mm_handle* h, int i) {
  Recording& R = h->rec;
  const size_t t = h->tsz, nc = (size_t)h->ncells;
  // one launch for the five arrays
  mm::CopySegs c{};
  c.n = 5;
  const void* src[5] = {h->mb, h->psi[h->parity], h->nb[h->parity], h->mf, &h->prm->psi_scale};
  void* dst[5] = {R.ck_mb[i], R.ck_psi[i], R.ck_nb[i], R.ck_mf[i], R.ck_scale + i};
  const size_t bytes[5] = {h->mbn * t, h->rows * t, h->rows * t, nc * t, 8};
  for (int q = 0; q < 5; ++q) {
    c.src[q] = src[q];
    c.dst[q] = dst[q];
    c.bytes[q] = bytes[q];
  }
  CK(mm::launch_copy_multi(c, h->stream));
  return MM_OK;
}

// Remember the velocity (its per-cell block) and dt now in effect.
mm_status rec_push_version(mm_handle* h) {
  Recording& R = h->rec;
  const size_t nc = (size_t)h->ncells;
  const size_t ver = R.v_ucell.size();
  if (ver == R.vblocks.size()) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, vblock_bytes(h));
    if (e != cudaSuccess) return cuda_fail(h, "recording: velocity buffers", e);
    R.vblocks.push_back(p);
  }
  Carver c;
  c.base = (unsigned char*)R.vblocks[ver];
  void* uc = c.take(12 * nc * h->tsz);
  double* dt = (double*)c.take(8);
  R.v_lamG.push_back((double*)c.take(4 * nc * 8));
  R.v_lamu.push_back((double*)c.take(2 * nc * 8));
  CK(cudaMemcpyAsync(uc, h->ucell, 12 * nc * h->tsz, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(dt, &h->prm->dt, 8, cudaMemcpyDeviceToDevice, h->stream));
  R.v_ucell.push_back(uc);
  R.v_dt.push_back(dt);
  return MM_OK;
}

// Substeps while recording: direct launches, a checkpoint every K substeps.
mm_status rec_micro_step(mm_handle* h, int n) {
  Recording& R = h->rec;
  if (R.nsub + n > R.max_sub)
    return fail(h, MM_ERR_STATE, "recording: more substeps than mm_set_checkpointing reserved");
  // The substeps between checkpoints run as captured graphs. With one level,
  // the segment the reverse sweep starts with (the last one the reservation
  // allows) runs out of place into the recomputation slots instead, so that
  // the sweep need not recompute it; the live state is then copied from the
  // last slot at the end of the call.
  const int tail = rec_tail_start(R);
  mm_status st;
  bool in_tail = false;
  for (int i = 0; i < n;) {
    if (R.nsub >= tail) {
      if ((st = rec_push_substep(h)) != MM_OK) return st;
      const int j = R.nsub - 1 - tail, c = tail / R.K;
      StepPtrs p{j == 0 ? R.ck_psi[c] : R.sl_psi[j], j == 0 ? R.ck_nb[c] : R.sl_nb[j],
                 j == 0 ? R.ck_mb[c] : R.sl_mb[j],   j == 0 ? R.ck_mf[c] : R.sl_mf[j],
                 h->ucell, R.sl_psi[j + 1], R.sl_nb[j + 1], R.sl_mb[j + 1], R.sl_mf[j + 1],
                 h->c, R.sl_cpre[j + 1]};
      CK(launch_ptrs(h, p, h->stream));
      h->parity ^= 1;
      ++R.tail_done;
      in_tail = true;
      ++i;
      continue;
    }
    int m = std::min(std::min(n - i, R.K - R.nsub % R.K), tail - R.nsub);
    for (int j = 0; j < m; ++j)
      if ((st = rec_push_substep(h)) != MM_OK) return st;
    if ((st = launch_substeps(h, m)) != MM_OK) return st;
    i += m;
  }
  if (in_tail) {
    const int j = R.nsub - tail;  // slot of the current state
    const size_t t = h->tsz, nc = (size_t)h->ncells;
    mm::CopySegs c{};
    c.n = 4;
    const void* src[4] = {R.sl_mb[j], R.sl_psi[j], R.sl_nb[j], R.sl_mf[j]};
    void* dst[4] = {h->mb, h->psi[h->parity], h->nb[h->parity], h->mf};
    const size_t bytes[4] = {h->mbn * t, h->rows * t, h->rows * t, nc * t};
    for (int q = 0; q < 4; ++q) {
      c.src[q] = src[q];
      c.dst[q] = dst[q];
      c.bytes[q] = bytes[q];
    }
    CK(mm::launch_copy_multi(c, h->stream));
  }
  return MM_OK;
}

// First substep of the segment recorded straight into the slots (one level
// only; none with two levels).
int rec_tail_start(const Recording& R) {
  if (R.K2 != R.K) return INT32_MAX;
  return ((R.max_sub - 1) / R.K) * R.K;
}

// Before a recorded substep: the checkpoint due at its start and its velocity.
mm_status rec_push_substep(mm_handle* h) {
  Recording& R = h->rec;
  if (R.nsub >= R.max_sub)
    return fail(h, MM_ERR_STATE, "recording: more substeps than mm_set_checkpointing reserved");
  mm_status st;
  if (R.nsub > 0 && R.nsub % R.K == 0)
    if ((st = rec_save_checkpoint(h, R.nsub / R.K)) != MM_OK) return st;
  R.sub_vel.push_back((int)R.v_ucell.size() - 1);
  ++R.nsub;
  return MM_OK;
}

// The reverse kernel reads rows with at most MM_ADJ_FP32_VMAX values per lane.
int adj_V(const mm_handle* h) { return std::min(h->V, MM_ADJ_FP32_VMAX); }
int adj_seg(const mm_handle* h) {
  int sg = 1;
  while (sg < h->g.ns / adj_V(h)) sg <<= 1;
  return sg;
}

template <typename T>
mm::AdjArgs<T> adj_args(mm_handle* h, int slot, int ver, int cur) {
  Recording& R = h->rec;
  mm::AdjArgs<T> a{};
  a.nx = h->g.nx;
  a.ny = h->g.ny;
  a.nth = h->g.ntheta;
  a.ns = h->g.ns;
  a.seg = adj_seg(h);
  a.ncells = h->ncells;
  a.inv_dx = (double)h->g.nx;
  a.inv_dy = (double)h->g.ny;
  a.dth = 2.0 * kPi / h->g.ntheta;
  a.inv_dth = 1.0 / a.dth;
  a.ds = h->g.L / h->g.ns;
  a.L = h->g.L;
  a.dt = R.v_dt[ver];
  a.v_walk = h->r.v_walk;
  a.cw = walk_cw(h);
  a.inv_ds = 1.0 / a.ds;
  a.k_on = h->r.k_on;
  a.k_off = h->r.k_off;
  a.glide = h->r.glide;
  a.v_sp = h->r.v_sp;
  a.psi_n = (const T*)R.sl_psi[slot];
  a.nb_n = (const T*)R.sl_nb[slot];
  a.mb_n = (const T*)R.sl_mb[slot];
  a.mf_n = (const T*)R.sl_mf[slot];
  a.psi_np = (const T*)R.sl_psi[slot + 1];
  a.nb_np = (const T*)R.sl_nb[slot + 1];
  a.cpre_np = (const T*)R.sl_cpre[slot + 1];
  a.mtot = (const T*)h->mtot;
  a.ucell = (const T*)R.v_ucell[ver];
  a.trig = (const T*)h->trig;
  a.lpsi_in = (const T*)R.lpsi[cur];
  a.lmf_in = (const T*)R.lmf[cur];
  a.D_in = (const T*)R.Dd[cur];
  a.lpsi_out = (T*)R.lpsi[cur ^ 1];
  a.lmb = (T*)R.lmb;
  a.lmf_out = (T*)R.lmf[cur ^ 1];
  a.D_out = (T*)R.Dd[cur ^ 1];
  a.lamG = R.v_lamG[ver];
  a.lamu = R.v_lamu[ver];
  a.gpart = R.gpart;
  a.units = R.units;
  a.rows_per_unit = R.rows_per_unit;
  a.lnb = (T*)R.lnb;
  a.cellc = (T*)R.cellc;
  a.prm = h->prm;
  a.ring_rc = R.ring_rc;
  a.ring_ch = R.ring_ch;
  a.ring_s = R.ring_s;
  return a;
}

// Lay the recording's fixed buffers out in the slab (c.base may be null to
// size it).
void rec_layout(mm_handle* h, Carver& c) {
  Recording& R = h->rec;
  const size_t t = h->tsz, nc = (size_t)h->ncells, rows = h->rows;
  const int K = R.K;  // outer checkpoint spacing
  R.ck_mb.resize(R.nck);
  R.ck_psi.resize(R.nck);
  R.ck_nb.resize(R.nck);
  R.ck_mf.resize(R.nck);
  for (int i = 0; i < R.nck; ++i) {
    R.ck_mb[i] = c.take(h->mbn * t);
    R.ck_psi[i] = c.take(rows * t);
    R.ck_nb[i] = c.take(rows * t);
    R.ck_mf[i] = c.take(nc * t);
  }
  R.ck_scale = (double*)c.take((size_t)R.nck * 8);
  // inner checkpoints (two levels): states K2, 2 K2, ... of an outer segment
  const int nick = (K + R.K2 - 1) / R.K2 - 1;
  R.ick_mb.resize(nick);
  R.ick_psi.resize(nick);
  R.ick_nb.resize(nick);
  R.ick_mf.resize(nick);
  for (int i = 0; i < nick; ++i) {
    R.ick_mb[i] = c.take(h->mbn * t);
    R.ick_psi[i] = c.take(rows * t);
    R.ick_nb[i] = c.take(rows * t);
    R.ick_mf[i] = c.take(nc * t);
  }
  R.ick_scale = (double*)c.take((size_t)std::max(nick, 1) * 8);
  // slot 0 of a segment is its checkpoint (read in place); slots 1..nslots
  // hold the recomputed states (and, with two levels, the march between inner
  // checkpoints ping-pongs through slots 1 and 2)
  R.nslots = nick > 0 ? std::max(R.K2, 2) : R.K2;
  const int NS = R.nslots;
  R.sl_mb.resize(NS + 1);
  R.sl_psi.resize(NS + 1);
  R.sl_nb.resize(NS + 1);
  R.sl_mf.resize(NS + 1);
  R.sl_cpre.resize(NS + 1);
  R.sl_mb[0] = R.sl_psi[0] = R.sl_nb[0] = R.sl_mf[0] = R.sl_cpre[0] = nullptr;
  for (int i = 1; i <= NS; ++i) {
    R.sl_mb[i] = c.take(h->mbn * t);
    R.sl_psi[i] = c.take(rows * t);
    R.sl_nb[i] = c.take(rows * t);
    R.sl_mf[i] = c.take(nc * t);
    R.sl_cpre[i] = c.take(nc * t);
  }
  // the second slot set of the overlapped one-level sweep
  std::vector<void*>* s2[5] = {&R.sl2_mb, &R.sl2_psi, &R.sl2_nb, &R.sl2_mf, &R.sl2_cpre};
  for (auto* v : s2) v->assign(R.overlap ? NS + 1 : 0, nullptr);
  for (int i = 1; R.overlap && i <= NS; ++i) {
    R.sl2_mb[i] = c.take(h->mbn * t);
    R.sl2_psi[i] = c.take(rows * t);
    R.sl2_nb[i] = c.take(rows * t);
    R.sl2_mf[i] = c.take(nc * t);
    R.sl2_cpre[i] = c.take(nc * t);
  }
  R.sl_c = c.take(nc * t);
  R.lmb = c.take(h->mbn * t);
  for (int i = 0; i < 2; ++i) {
    R.lpsi[i] = c.take(rows * t);
    R.lmf[i] = c.take((size_t)R.units * nc * t);
    R.Dd[i] = c.take((size_t)R.units * nc * t);
  }
  R.lnb = c.take(rows * t);
  R.cellc = c.take(2 * nc * t);
  R.gpart = (double*)c.take((size_t)R.grid_motor * 4 * 4 * 8);
  for (int i = 0; i < 3; ++i) R.seed[i] = (double*)c.take(rows * 8);
  R.seed[3] = (double*)c.take(nc * 8);
  R.coef = (double*)c.take(128);
  R.work = (double*)c.take(std::max(rows, 2 * nc) * 8);
}

}  // namespace mmh

extern "C" {

mm_status mm_set_checkpointing(mm_handle* h, int K, int max_substeps) {
  return mm_set_checkpointing_levels(h, K, K, max_substeps);
}

mm_status mm_set_checkpointing_levels(mm_handle* h, int K, int K_inner, int max_substeps) {
  MM_TRACE("mm_set_checkpointing_levels");
  if (!h) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream));
  Recording& R = h->rec;
  R.active = false;
  if (K == 0) {
    free_recording(h);
    return MM_OK;
  }
  if (K < 0 || max_substeps < 1) return fail(h, MM_ERR_INVALID, "K >= 1 and max_substeps >= 1");
  if (h->capture)
    return fail(h, MM_ERR_UNSUPPORTED, "the adjoint is not available with a capture radius");
  if (h->tangent)
    return fail(h, MM_ERR_STATE, "the tangent mode is on: switch it off (mm_set_tangent(h, NULL)) first");
  if (h->anchors)
    return fail(h, MM_ERR_UNSUPPORTED, "the adjoint is not available with non-local anchors");
  if (K_inner < 1 || K_inner > K) return fail(h, MM_ERR_INVALID, "1 <= K_inner <= K");
  if (!h->have_state || !h->have_vel || !h->have_dt)
    return fail(h, MM_ERR_STATE, "set the state and the velocity before recording");
  if (!R.slab || R.K != K || R.K2 != K_inner || R.max_sub != max_substeps) {
    if (R.slab) cudaFree(R.slab);
    R.slab = nullptr;
    R.K = K;
    R.K2 = K_inner;
    R.max_sub = max_substeps;
    R.nck = (max_substeps + K - 1) / K + 1;
    // reverse kernels: the psi part one warp per cell; the motor part one warp
    // per block of rows, with enough blocks per cell (a power of two, at least
    // one pass of rows each) for about six waves of warps
    const int rpp = 32 / adj_seg(h);
    int U = 1;
    const int umax = h->prec == MM_FP64 ? MM_ADJ_MAX_UNITS : MM_ADJ_MAX_UNITS_F32;
    while (U < umax && h->ncells * U < 6LL * 16 * h->sms &&
           h->g.ntheta / (2 * U) >= rpp)
      U *= 2;
    R.units = U;
    R.rows_per_unit = (h->g.ntheta + U - 1) / U;
    R.grid_psi = (int)std::min<long long>((h->ncells + 3) / 4, 16LL * h->sms);
    // bulk-copy ring for the motor kernel: 16-byte rows and row-column slices,
    // chunks of RC rows (dividing a unit) of at most 2 KB per array
    R.ring_rc = R.ring_ch = R.ring_s = 0;
    const size_t row_b = (size_t)h->g.ns * h->tsz;
    if (MM_ADJ_RING && ((size_t)adj_V(h) * h->tsz) % 16 == 0 && h->g.ntheta % U == 0) {
      for (int rc = R.rows_per_unit; rc >= 1; --rc)
        if (R.rows_per_unit % rc == 0 && (rc * h->tsz) % 16 == 0 && rc * row_b <= 2048) {
          R.ring_rc = rc;
          break;
        }
      if (R.ring_rc > 0) {
        R.ring_ch = R.rows_per_unit / R.ring_rc;
        R.ring_s = (int)std::max<size_t>(2, std::min<size_t>(8, 8192 / (2 * R.ring_rc * row_b)));
        if (4 * mm::adj_ring_warp_bytes(R.ring_rc, h->g.ns, R.ring_s, (int)h->tsz) > kSmemBudget)
          R.ring_rc = R.ring_ch = R.ring_s = 0;
      }
    }
    // persistent motor grid: the resident blocks (each warp fills its ring once)
    int bps = 0;
    const cudaError_t oe =
        h->prec == MM_FP64
            ? mm::adj_motor_occupancy<double>(adj_V(h), R.ring_rc, h->g.ns, R.ring_s, &bps)
            : mm::adj_motor_occupancy<float>(adj_V(h), R.ring_rc, h->g.ns, R.ring_s, &bps);
    CK(oe);
    if (bps < 1) return fail(h, MM_ERR_UNSUPPORTED, "reverse kernel cannot be resident");
    R.grid_motor = (int)std::min<long long>((h->ncells * U + 3) / 4, (long long)bps * h->sms);
    size_t freeb = 0, totalb = 0;
    CK(cudaMemGetInfo(&freeb, &totalb));
    // one level with more than one segment: a second slot set lets the replay
    // of a segment overlap the reverse of the next one, where it takes at most
    // a quarter of the free memory
    R.overlap = K_inner == K && max_substeps > K;
    Carver sz;
    rec_layout(h, sz);
    if (R.overlap && sz.off > freeb / 4) {
      R.overlap = false;
      sz = Carver();
      rec_layout(h, sz);
    }
    if (R.overlap && !R.rstream) {
      CK(cudaStreamCreateWithFlags(&R.rstream, cudaStreamNonBlocking));
      cudaEvent_t* evs[5] = {&R.ev_start, &R.ev_rep[0], &R.ev_rep[1], &R.ev_rev[0], &R.ev_rev[1]};
      for (cudaEvent_t* ev : evs) CK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    }
    const size_t need = sz.off + 2 * vblock_bytes(h) + (1 << 20);
    if (need > freeb) {
      free_recording(h);
      char buf[160];
      snprintf(buf, sizeof buf, "recording needs %zu bytes of device memory, %zu free", need, freeb);
      return fail(h, MM_ERR_OOM, buf);
    }
    cudaError_t e = cudaMalloc(&R.slab, sz.off);
    if (e != cudaSuccess) {
      R.slab = nullptr;
      free_recording(h);
      return cuda_fail(h, "recording: cudaMalloc", e);
    }
    R.slab_bytes = sz.off;
    Carver c;
    c.base = (unsigned char*)R.slab;
    rec_layout(h, c);
  }
  R.nsub = 0;
  R.tail_done = 0;
  R.sub_vel.clear();
  R.v_ucell.clear();
  R.v_dt.clear();
  R.v_lamG.clear();
  R.v_lamu.clear();
  R.active = true;
  mm_status st;
  if ((st = rec_push_version(h)) != MM_OK || (st = rec_save_checkpoint(h, 0)) != MM_OK) {
    R.active = false;
    return st;
  }
  return MM_OK;
}

mm_status mm_adjoint_step(mm_handle* h, int n, const mm_adjoint_seed* seed, mm_adjoint_out* out) {
  MM_TRACE("mm_adjoint_step");
  if (!h || !seed || !out) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  Recording& R = h->rec;
  if (!R.active) return fail(h, MM_ERR_STATE, "no recording: call mm_set_checkpointing first (mm_set_state and mm_set_rates end one)");
  if (n != R.nsub || n < 1)
    return fail(h, MM_ERR_STATE, "n_substeps must equal the substeps recorded");
  if (out->dL_du && out->du_capacity < (int)R.v_ucell.size())
    return fail(h, MM_ERR_INVALID, "dL_du holds fewer velocity fields than were recorded");
  DeviceGuard dg(h->device);
  mm_status st;
  const size_t t = h->tsz, nc = (size_t)h->ncells, rows = h->rows;
  const double dth = 2.0 * kPi / h->g.ntheta, ds = h->g.L / h->g.ns;
  const bool f64 = h->prec == MM_FP64;
  const int nv = (int)R.v_ucell.size();
  // live scalars (psi correction factor, dt) kept on the device, restored at
  // the end; the whole sweep is enqueued without a host round trip
  CK(cudaMemcpyAsync(R.coef + 8, &h->prm->psi_scale, 8, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(R.coef + 9, &h->prm->dt, 8, cudaMemcpyDeviceToDevice, h->stream));

  // ---- seed at the final (live) state: coef[0..2] seed coefficients, coef[3]
  // the observable's value, coef[4..6] the parameter adjoints at the end
  int kind = seed->observable;
  out->value = 0.0;
  CK(cudaMemsetAsync(R.coef, 0, 8 * 8, h->stream));
  if (kind == MM_OBS_POLAR_ORDER || kind == MM_OBS_MEAN_STRESS) {
    if ((st = run_moments(h)) != MM_OK) return st;
    CK(mm::launch_adj_observable(kind, h->prm, h->r.force_scale * h->r.ell * dth / (double)nc,
                                 R.coef, h->stream));
  } else if (kind != MM_OBS_NONE) {
    return fail(h, MM_ERR_INVALID, "unknown observable");
  }
  const double* sp[4] = {nullptr, nullptr, nullptr, nullptr};
  if (kind == MM_OBS_NONE) {
    const double* src[4] = {seed->dL_dpsi, seed->dL_dnb, seed->dL_dm1, seed->dL_dmf};
    for (int i = 0; i < 4; ++i) {
      if (!src[i]) continue;
      const size_t cnt = i < 3 ? rows : nc;
      if (seed->on_device) {
        sp[i] = src[i];
      } else {
        CK(cudaMemcpyAsync(R.seed[i], src[i], cnt * 8, cudaMemcpyHostToDevice, h->stream));
        sp[i] = R.seed[i];
      }
    }
  }
  // a seed on the motor density itself goes straight into lam_Mb (in the
  // state precision); the seed kernel adds the moment seeds to it
  const bool mb_seeded = kind == MM_OBS_NONE && seed->dL_dmb;
  if (mb_seeded && (st = put_array(h, R.lmb, seed->dL_dmb, h->mbn, seed->on_device)) != MM_OK)
    return st;
  // the seed fills partial 0 of lam_Mf and D; the other partials start at 0
  CK(cudaMemsetAsync(R.lmf[0], 0, (size_t)R.units * nc * t, h->stream));
  CK(cudaMemsetAsync(R.Dd[0], 0, (size_t)R.units * nc * t, h->stream));
  cudaError_t e;
  if (f64)
    e = mm::launch_adj_seed<double>(kind, R.coef, (const double*)h->psi[h->parity],
                                    (const double*)h->mb, sp[0], sp[1], sp[2], sp[3],
                                    (double*)R.lpsi[0], (double*)R.lmb, (double*)R.lmf[0],
                                    (double*)R.Dd[0], h->ncells, h->g.ntheta, h->g.ns, ds, h->g.L,
                                    (const double*)h->trig, mb_seeded, h->stream);
  else
    e = mm::launch_adj_seed<float>(kind, R.coef, (const float*)h->psi[h->parity],
                                   (const float*)h->mb, sp[0], sp[1], sp[2], sp[3],
                                   (float*)R.lpsi[0], (float*)R.lmb, (float*)R.lmf[0],
                                   (float*)R.Dd[0], h->ncells, h->g.ntheta, h->g.ns, ds, h->g.L,
                                   (const float*)h->trig, mb_seeded, h->stream);
  CK(e);
  for (int v = 0; v < nv; ++v) {
    CK(cudaMemsetAsync(R.v_lamG[v], 0, 4 * nc * 8, h->stream));
    CK(cudaMemsetAsync(R.v_lamu[v], 0, 2 * nc * 8, h->stream));
  }
  CK(cudaMemsetAsync(R.gpart, 0, (size_t)R.grid_motor * 4 * 4 * 8, h->stream));

  // ---- outer segments (checkpoints every K), last first; with two levels
  // each is first marched through to store its inner checkpoints (every K2),
  // then its inner segments are recomputed into the slots and reversed, last
  // first
  int cur = 0, dt_ver = -1;
  auto set_dt = [&](int ver) -> mm_status {
    if (ver != dt_ver)
      CK(cudaMemcpyAsync(&h->prm->dt, R.v_dt[ver], 8, cudaMemcpyDeviceToDevice, h->stream));
    dt_ver = ver;
    return MM_OK;
  };
  const int nseg = (n + R.K - 1) / R.K;
  auto reverse_range = [&](int a0, int a1) -> mm_status {
    for (int tt = a1 - 1; tt >= a0; --tt) {
      const int i = tt - a0, ver = R.sub_vel[tt];
      if (f64)
        e = mm::launch_adjoint<double>(adj_args<double>(h, i, ver, cur), adj_V(h), R.grid_psi,
                                       R.grid_motor, h->stream);
      else
        e = mm::launch_adjoint<float>(adj_args<float>(h, i, ver, cur), adj_V(h), R.grid_psi,
                                      R.grid_motor, h->stream);
      CK(e);
      cur ^= 1;
    }
    return MM_OK;
  };
  if (R.overlap && R.K2 == R.K && nseg > 1) {
    // One level, two slot sets: segment s uses set (nseg - 1 - s) & 1 (the
    // last segment set 0, which the recording may have filled already). The
    // replay of segment s - 1 runs on the replay stream while segment s is
    // reversed on the handle's stream; a set is replayed into only after the
    // reverse that read it has finished (ev_rev), and reversed only after its
    // replay (ev_rep). Only the replay touches the device dt and the psi
    // correction factor; the reverse kernels read the recorded dt.
    cudaStream_t rs = R.rstream;
    CK(cudaEventRecord(R.ev_start, h->stream));
    CK(cudaStreamWaitEvent(rs, R.ev_start, 0));
    int live_set = 0;  // the set R.sl_* holds now (the other is in R.sl2_*)
    auto vecs = [&](int set) {
      const bool here = set == live_set;
      return std::array<std::vector<void*>*, 5>{here ? &R.sl_mb : &R.sl2_mb,
                                                here ? &R.sl_psi : &R.sl2_psi,
                                                here ? &R.sl_nb : &R.sl2_nb,
                                                here ? &R.sl_mf : &R.sl2_mf,
                                                here ? &R.sl_cpre : &R.sl2_cpre};
    };
    auto set_of = [&](int sg) { return (nseg - 1 - sg) & 1; };
    int rs_dt = -1;
    auto replay = [&](int sg) -> mm_status {
      const int set = set_of(sg), s0 = sg * R.K, s1 = std::min(s0 + R.K, n);
      auto v = vecs(set);
      std::vector<void*>&vmb = *v[0], &vpsi = *v[1], &vnb = *v[2], &vmf = *v[3], &vcp = *v[4];
      vmb[0] = R.ck_mb[sg];
      vpsi[0] = R.ck_psi[sg];
      vnb[0] = R.ck_nb[sg];
      vmf[0] = R.ck_mf[sg];
      CK(cudaMemcpyAsync(&h->prm->psi_scale, R.ck_scale + sg, 8, cudaMemcpyDeviceToDevice, rs));
      for (int tt = s0; tt < s1; ++tt) {
        const int i = tt - s0, ver = R.sub_vel[tt];
        if (ver != rs_dt)
          CK(cudaMemcpyAsync(&h->prm->dt, R.v_dt[ver], 8, cudaMemcpyDeviceToDevice, rs));
        rs_dt = ver;
        StepPtrs p{vpsi[i], vnb[i], vmb[i], vmf[i], R.v_ucell[ver], vpsi[i + 1], vnb[i + 1],
                   vmb[i + 1], vmf[i + 1], R.sl_c, vcp[i + 1]};
        CK(launch_ptrs(h, p, rs));
      }
      CK(cudaEventRecord(R.ev_rep[set], rs));
      return MM_OK;
    };
    const int tail = rec_tail_start(R);
    const bool last_in_slots = (nseg - 1) * R.K == tail && R.tail_done == n - tail;
    if (!last_in_slots && (st = replay(nseg - 1)) != MM_OK) return st;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
      if (sgi >= 1) {
        // the set of segment sgi - 1 was last read by the reverse of sgi + 1
        if (sgi + 1 <= nseg - 1) CK(cudaStreamWaitEvent(rs, R.ev_rev[set_of(sgi - 1)], 0));
        if ((st = replay(sgi - 1)) != MM_OK) return st;
      }
      const int set = set_of(sgi);
      if (sgi < nseg - 1 || !last_in_slots) CK(cudaStreamWaitEvent(h->stream, R.ev_rep[set], 0));
      if (set != live_set) {
        std::swap(R.sl_mb, R.sl2_mb);
        std::swap(R.sl_psi, R.sl2_psi);
        std::swap(R.sl_nb, R.sl2_nb);
        std::swap(R.sl_mf, R.sl2_mf);
        std::swap(R.sl_cpre, R.sl2_cpre);
        live_set = set;
      }
      R.sl_mb[0] = R.ck_mb[sgi];
      R.sl_psi[0] = R.ck_psi[sgi];
      R.sl_nb[0] = R.ck_nb[sgi];
      R.sl_mf[0] = R.ck_mf[sgi];
      const int s0 = sgi * R.K;
      if ((st = reverse_range(s0, std::min(s0 + R.K, n))) != MM_OK) return st;
      CK(cudaEventRecord(R.ev_rev[set], h->stream));
    }
    if (live_set != 0) {  // set 0 is the one the next recording writes into
      std::swap(R.sl_mb, R.sl2_mb);
      std::swap(R.sl_psi, R.sl2_psi);
      std::swap(R.sl_nb, R.sl2_nb);
      std::swap(R.sl_mf, R.sl2_mf);
      std::swap(R.sl_cpre, R.sl2_cpre);
    }
  }
  for (int sgi = (R.overlap && R.K2 == R.K && nseg > 1) ? -1 : nseg - 1; sgi >= 0; --sgi) {
    const int s0 = sgi * R.K, s1 = std::min(s0 + R.K, n);
    const int nin = (s1 - s0 + R.K2 - 1) / R.K2;
    if (nin > 1) {
      CK(cudaMemcpyAsync(&h->prm->psi_scale, R.ck_scale + sgi, 8, cudaMemcpyDeviceToDevice,
                         h->stream));
      const void *in_psi = R.ck_psi[sgi], *in_nb = R.ck_nb[sgi], *in_mb = R.ck_mb[sgi],
                 *in_mf = R.ck_mf[sgi];
      int tmp = 1;
      for (int tt = s0; tt < s0 + (nin - 1) * R.K2; ++tt) {
        const int ver = R.sub_vel[tt], done = tt + 1 - s0;
        if ((st = set_dt(ver)) != MM_OK) return st;
        const bool ick = done % R.K2 == 0;
        const int j = done / R.K2 - 1;
        void* o_psi = ick ? R.ick_psi[j] : R.sl_psi[tmp];
        void* o_nb = ick ? R.ick_nb[j] : R.sl_nb[tmp];
        void* o_mb = ick ? R.ick_mb[j] : R.sl_mb[tmp];
        void* o_mf = ick ? R.ick_mf[j] : R.sl_mf[tmp];
        StepPtrs p{in_psi, in_nb, in_mb, in_mf, R.v_ucell[ver], o_psi, o_nb, o_mb, o_mf, R.sl_c,
                   R.sl_cpre[1]};
        CK(launch_ptrs(h, p, h->stream));
        if (ick)
          CK(cudaMemcpyAsync(R.ick_scale + j, &h->prm->psi_scale, 8, cudaMemcpyDeviceToDevice,
                             h->stream));
        else
          tmp = 3 - tmp;
        in_psi = o_psi;
        in_nb = o_nb;
        in_mb = o_mb;
        in_mf = o_mf;
      }
    }
    // the segment the recording wrote straight into the slots needs no replay
    const int tail = rec_tail_start(R);
    const bool tail_in_slots = s0 == tail && R.tail_done == n - tail;
    for (int ig = nin - 1; ig >= 0; --ig) {
      const int a0 = s0 + ig * R.K2, a1 = std::min(a0 + R.K2, s1);
      R.sl_mb[0] = ig == 0 ? R.ck_mb[sgi] : R.ick_mb[ig - 1];
      R.sl_psi[0] = ig == 0 ? R.ck_psi[sgi] : R.ick_psi[ig - 1];
      R.sl_nb[0] = ig == 0 ? R.ck_nb[sgi] : R.ick_nb[ig - 1];
      R.sl_mf[0] = ig == 0 ? R.ck_mf[sgi] : R.ick_mf[ig - 1];
      CK(cudaMemcpyAsync(&h->prm->psi_scale, ig == 0 ? R.ck_scale + sgi : R.ick_scale + ig - 1,
                         8, cudaMemcpyDeviceToDevice, h->stream));
      for (int tt = a0; tt < a1 && !tail_in_slots; ++tt) {
        const int i = tt - a0, ver = R.sub_vel[tt];
        if ((st = set_dt(ver)) != MM_OK) return st;
        StepPtrs p{R.sl_psi[i], R.sl_nb[i], R.sl_mb[i], R.sl_mf[i], R.v_ucell[ver],
                   R.sl_psi[i + 1], R.sl_nb[i + 1], R.sl_mb[i + 1], R.sl_mf[i + 1], R.sl_c,
                   R.sl_cpre[i + 1]};
        CK(launch_ptrs(h, p, h->stream));
      }
      if ((st = reverse_range(a0, a1)) != MM_OK) return st;
    }
  }
  // restore the live scalars
  CK(cudaMemcpyAsync(&h->prm->psi_scale, R.coef + 8, 8, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(&h->prm->dt, R.coef + 9, 8, cudaMemcpyDeviceToDevice, h->stream));

  // ---- outputs
  out->n_velocities = nv;
  if (out->dL_du && out->du_capacity < nv)
    return fail(h, MM_ERR_INVALID, "dL_du holds fewer velocity fields than were recorded");
  if (out->dL_du) {
    for (int v = 0; v < nv; ++v) {
      double* dst = out->on_device ? out->dL_du + (size_t)v * 2 * nc : R.work;
      CK(mm::launch_adj_finish(R.v_lamG[v], R.v_lamu[v], dst, h->g.nx, h->g.ny, (double)h->g.nx,
                               (double)h->g.ny, h->stream));
      if (!out->on_device)
        CK(cudaMemcpyAsync(out->dL_du + (size_t)v * 2 * nc, R.work, 2 * nc * 8,
                           cudaMemcpyDeviceToHost, h->stream));
    }
  }
  if (out->dL_dpsi0) {
    double* dst = out->on_device ? out->dL_dpsi0 : R.work;
    if (f64)
      e = mm::launch_adj_psi0<double>((const double*)R.lpsi[cur], (const double*)R.lmf[cur], R.units,
                                      (const double*)R.ck_nb[0], dth, (long long)rows,
                                      h->g.ntheta, dst, h->stream);
    else
      e = mm::launch_adj_psi0<float>((const float*)R.lpsi[cur], (const float*)R.lmf[cur], R.units,
                                     (const float*)R.ck_nb[0], dth, (long long)rows, h->g.ntheta,
                                     dst, h->stream);
    CK(e);
    if (!out->on_device)
      CK(cudaMemcpyAsync(out->dL_dpsi0, R.work, rows * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(mm::launch_adj_params(R.gpart, R.grid_motor * 4, R.coef + 4, h->stream));
  double res[8];
  CK(cudaMemcpyAsync(res, R.coef, sizeof res, cudaMemcpyDeviceToHost, h->stream));
  if ((st = check_status(h)) != MM_OK) return st;
  out->value = res[3];
  for (int q = 0; q < 3; ++q) out->dL_drates[q] = res[4 + q];
  return MM_OK;
}

}  // extern "C"
