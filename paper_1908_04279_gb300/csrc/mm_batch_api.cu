// Host side of the batched ensemble (mm_create_batch, mm_batch_member,
// mm_batch_autotune, and mm_micro_step / mm_sync on a batch handle).
//
// A batch owns one ordinary handle per instance (its state, velocity, dt,
// moments and adjoint recording go through the single-instance calls on that
// member). Stepping the batch launches the batched substep kernel once per
// substep over a device table of every member's kernel arguments and a table
// of tiles; the substeps of one mm_micro_step call are captured in a CUDA
// graph. The tile size (motor values per tile) and the s-row chunk size are
// the tuning parameters; mm_batch_autotune times a grid of them on the live
// ensemble (restoring its state afterwards) and keeps the fastest, cached per
// process for batches of the same shape.
#include "mm_host.h"

using namespace mmh;

// Widest vector (values per lane) of the float32 batched kernel (8 or 4).
#ifndef MM_BATCH_FP32_VMAX
#define MM_BATCH_FP32_VMAX 8
#endif

namespace mmh {

struct BatchPlan {
  std::vector<mm_handle*> members;
  int V = 1;                  // values per lane, common to all members
  int tile_work = 8192;       // target motor values (rows x ns) per tile
  int chunk_bytes = kChunkBytes;
  int pairs = 1;              // members that can go two cells to a warp do
  int S = 2, stage_elems = 0, nth_max = 0, block = 128, grid = 1, ntiles = 0;
  size_t smem = 0;
  void* d_args = nullptr;     // [2][n] StepArgs: members at their parities, and flipped
  mm::BatchTile* d_tiles = nullptr;
  double* tile_mass = nullptr;
  std::vector<int> args_par;  // member parities the argument tables were built for
  std::map<int, cudaGraphExec_t> graphs;
  int tuned = 0;
};

namespace {

// Tuned (tile_work, chunk_bytes, two cells per warp) per batch shape, for this
// process.
struct TuneChoice {
  int tile_work, chunk_bytes, pairs;
};
std::map<std::string, TuneChoice> g_tune_cache;

std::string batch_signature(const mm_handle* h) {
  std::string sig = h->prec == MM_FP64 ? "f64" : "f32";
  for (const mm_handle* m : h->batch->members) {
    char buf[64];
    snprintf(buf, sizeof buf, ";%d,%d,%d,%d", m->g.nx, m->g.ny, m->g.ntheta, m->g.ns);
    sig += buf;
  }
  return sig;
}

void clear_graphs(BatchPlan* B) {
  for (auto& kv : B->graphs) cudaGraphExecDestroy(kv.second);
  B->graphs.clear();
}

// Rows per chunk of a member under the chunk limit (the largest divisor of
// nth whose rows fit), as for the single-instance plan.
void member_chunks(const mm_handle* m, int chunk_bytes, int* rc, int* ch) {
  const size_t row_bytes = (size_t)m->g.ns * m->tsz;
  const int nth = m->g.ntheta;
  int c = 1;
  while (c < nth && (nth % c != 0 || (size_t)(nth / c) * row_bytes > (size_t)chunk_bytes)) ++c;
  *ch = c;
  *rc = nth / c;
}

// Whether a member's cells go two to a warp: at most 16 orientations (one
// half-warp per cell for psi and the close) or at most 32 (the warp takes the
// two cells' psi and close in turn), with one cell's rows in at most 4 KB (a
// unit is one chunk or two); the rows of a cell a whole number of row passes
// (32 / seg rows each), an even row length (the two cells of a unit share a
// row) and neighbourhood columns that bulk copies can stage.
bool member_pairs(const mm_handle* m, int V) {
  int seg = 1;
  while (seg < m->g.ns / V) seg <<= 1;
  const int nth = m->g.ntheta;
  const bool fits = nth <= 32 && (size_t)nth * m->g.ns * m->tsz <= 4096;
  return fits && nth % (32 / seg) == 0 && m->g.nx % 2 == 0 && ((size_t)nth * m->tsz) % 16 == 0;
}

template <typename T>
cudaError_t prepare(int V, int block, size_t smem, int* bps) {
  if constexpr (sizeof(T) == 8) {
    (void)V;
    return mm::substep_batch_prepare<double, 2>(block, smem, bps);
  } else {
    return V == 8 ? mm::substep_batch_prepare<float, 8>(block, smem, bps)
                  : mm::substep_batch_prepare<float, 4>(block, smem, bps);
  }
}

// Tiles, shared-memory plan and grid for (tile_work, chunk_bytes).
mm_status make_plan(mm_handle* h, int tile_work, int chunk_bytes) {
  BatchPlan* B = h->batch;
  const int n = (int)B->members.size();
  std::vector<mm::BatchTile> tiles;
  int max_chunk_elems = 1, nth_max = 1;
  for (int i = 0; i < n; ++i) {
    const mm_handle* m = B->members[i];
    // units of 1 cell (rows in ch chunks of rc) or of 2 cells (one chunk of
    // both cells' rows); tiles of about tile_work motor values, whole units
    const int cpu = B->pairs && member_pairs(m, B->V) ? 2 : 1;
    int rc, ch;
    if (cpu == 2) {
      // the unit's 2 ntheta rows in chunks of at most 4 KB (a divisor of the
      // unit's rows: one chunk, or one cell's rows per chunk)
      const int rows = 2 * m->g.ntheta;
      const size_t row_bytes = (size_t)m->g.ns * m->tsz;
      ch = 1;
      while (ch < rows && (rows % ch != 0 || (size_t)(rows / ch) * row_bytes > 4096)) ++ch;
      rc = rows / ch;
    } else {
      member_chunks(m, chunk_bytes, &rc, &ch);
    }
    max_chunk_elems = std::max(max_chunk_elems, rc * m->g.ns);
    nth_max = std::max(nth_max, cpu * m->g.ntheta);  // a pair stages two neighbourhoods
    const long long nu = m->ncells / cpu;             // nx even for pairs: ncells is too
    const long long per_unit = (long long)cpu * m->g.ntheta * m->g.ns;
    long long tu = std::max(1LL, (long long)tile_work / per_unit);
    tu = std::min(tu, nu);
    const int nt = (int)((nu + tu - 1) / tu);
    const int tile0 = (int)tiles.size();
    for (int t = 0; t < nt; ++t) {
      mm::BatchTile bt{};
      bt.inst = i;
      bt.cell0 = (int)(t * tu * cpu);
      bt.ncell = (int)std::min(tu, nu - t * tu);
      bt.tile0 = tile0;
      bt.inst_tiles = nt;
      bt.ch = ch;
      bt.rc = rc;
      bt.cpu = cpu;
      tiles.push_back(bt);
    }
  }
  const size_t chunk_max_bytes = (size_t)max_chunk_elems * h->tsz;
  int S = (int)(kWarpInflightBytes / std::max<size_t>(chunk_max_bytes, 1));
  S = std::max(2, std::min(8, S));
  const size_t per_warp = mm::step_smem_per_warp(S, max_chunk_elems, nth_max, (int)h->tsz);
  const int wpb = (int)std::min<size_t>(kMaxWarpsPerBlock, kSmemBudget / per_warp);
  if (wpb < 1) return fail(h, MM_ERR_UNSUPPORTED, "batch: ntheta too large for the shared-memory plan");
  const int block = 32 * wpb;
  const size_t smem = (size_t)wpb * per_warp;
  int bps = 0;
  cudaError_t e = h->prec == MM_FP64 ? prepare<double>(B->V, block, smem, &bps)
                                     : prepare<float>(B->V, block, smem, &bps);
  CK(e);
  if (bps < 1) return fail(h, MM_ERR_UNSUPPORTED, "batch: the substep kernel cannot be resident");
  long long grid = (long long)bps * h->sms;
  const long long need = ((long long)tiles.size() + wpb - 1) / wpb;
  grid = std::min(grid, need);

  // device tables
  if (B->d_tiles) cudaFree(B->d_tiles);
  if (B->tile_mass) cudaFree(B->tile_mass);
  B->d_tiles = nullptr;
  B->tile_mass = nullptr;
  CK(cudaMalloc((void**)&B->d_tiles, tiles.size() * sizeof(mm::BatchTile)));
  CK(cudaMalloc((void**)&B->tile_mass, tiles.size() * sizeof(double)));
  CK(cudaMemcpy(B->d_tiles, tiles.data(), tiles.size() * sizeof(mm::BatchTile),
                cudaMemcpyHostToDevice));
  B->tile_work = tile_work;
  B->chunk_bytes = chunk_bytes;
  B->S = S;
  B->stage_elems = max_chunk_elems;
  B->nth_max = nth_max;
  B->block = block;
  B->smem = smem;
  B->grid = (int)grid;
  B->ntiles = (int)tiles.size();
  clear_graphs(B);
  return MM_OK;
}

// Kernel-argument tables for the members' current parities (table 0) and the
// flipped ones (table 1); rebuilt when a member's parity changed since.
template <typename T>
mm_status upload_args_t(mm_handle* h) {
  BatchPlan* B = h->batch;
  const int n = (int)B->members.size();
  std::vector<StepArgs<T>> a(2 * (size_t)n);
  for (int p = 0; p < 2; ++p)
    for (int i = 0; i < n; ++i) {
      mm_handle* m = B->members[i];
      StepArgs<T> x = step_args<T>(m, m->parity ^ p);
      int seg = 1;
      while (seg < m->g.ns / B->V) seg <<= 1;
      x.seg = seg;
      x.nb_tma = ((size_t)m->g.ntheta * m->tsz) % 16 == 0;
      a[(size_t)p * n + i] = x;
    }
  // stream-ordered after every launch that still reads the old tables; the
  // pageable source is staged before the call returns
  CK(cudaMemcpyAsync(B->d_args, a.data(), a.size() * sizeof(StepArgs<T>), cudaMemcpyHostToDevice,
                     h->stream));
  B->args_par.resize(n);
  for (int i = 0; i < n; ++i) B->args_par[i] = B->members[i]->parity;
  return MM_OK;
}

mm_status upload_args(mm_handle* h) {
  BatchPlan* B = h->batch;
  bool same = B->args_par.size() == B->members.size();
  for (size_t i = 0; same && i < B->members.size(); ++i)
    same = B->args_par[i] == B->members[i]->parity;
  if (same) return MM_OK;
  return h->prec == MM_FP64 ? upload_args_t<double>(h) : upload_args_t<float>(h);
}

// One batched substep with argument table `table` (0: current parities).
cudaError_t launch_batch(mm_handle* h, int table, cudaStream_t s) {
  BatchPlan* B = h->batch;
  const int n = (int)B->members.size();
  if (h->prec == MM_FP64) {
    const StepArgs<double>* a = (const StepArgs<double>*)B->d_args + (size_t)table * n;
    return mm::launch_substep_batch<double, 2>(a, B->d_tiles, B->ntiles, B->tile_mass, B->S,
                                               B->stage_elems, B->nth_max, false, B->grid,
                                               B->block, B->smem, s);
  }
  const StepArgs<float>* a = (const StepArgs<float>*)B->d_args + (size_t)table * n;
  if (B->V == 8)
    return mm::launch_substep_batch<float, 8>(a, B->d_tiles, B->ntiles, B->tile_mass, B->S,
                                              B->stage_elems, B->nth_max, true, B->grid, B->block,
                                              B->smem, s);
  return mm::launch_substep_batch<float, 4>(a, B->d_tiles, B->ntiles, B->tile_mass, B->S,
                                            B->stage_elems, B->nth_max, true, B->grid, B->block,
                                            B->smem, s);
}

// Device snapshot of every member's evolving state (for the autotuner).
struct Snapshot {
  void* buf = nullptr;
  std::vector<int> parity;
};
size_t member_state_bytes(const mm_handle* m) {
  const size_t t = m->tsz, nc = (size_t)m->ncells;
  return m->mbn * t + 4 * m->rows * t + 2 * nc * t + sizeof(DevParams);
}
mm_status snapshot(mm_handle* h, Snapshot& sn, bool save) {
  BatchPlan* B = h->batch;
  size_t total = 0;
  for (mm_handle* m : B->members) total += (member_state_bytes(m) + 255) & ~(size_t)255;
  if (save) {
    CK(cudaMalloc(&sn.buf, total));
    sn.parity.clear();
  }
  unsigned char* p = (unsigned char*)sn.buf;
  for (size_t i = 0; i < B->members.size(); ++i) {
    mm_handle* m = B->members[i];
    const size_t t = m->tsz, nc = (size_t)m->ncells;
    void* parts[8] = {m->mb, m->psi[0], m->psi[1], m->nb[0], m->nb[1], m->mf, m->c, m->prm};
    const size_t sizes[8] = {m->mbn * t, m->rows * t, m->rows * t, m->rows * t, m->rows * t,
                             nc * t, nc * t, sizeof(DevParams)};
    unsigned char* q = p;
    for (int k = 0; k < 8; ++k) {
      if (save)
        CK(cudaMemcpyAsync(q, parts[k], sizes[k], cudaMemcpyDeviceToDevice, h->stream));
      else
        CK(cudaMemcpyAsync(parts[k], q, sizes[k], cudaMemcpyDeviceToDevice, h->stream));
      q += sizes[k];
    }
    p += (member_state_bytes(m) + 255) & ~(size_t)255;
    if (save)
      sn.parity.push_back(m->parity);
    else
      m->parity = sn.parity[i];
  }
  CK(cudaStreamSynchronize(h->stream));
  return MM_OK;
}

}  // namespace

mm_status batch_micro_step(mm_handle* h, int n) {
  BatchPlan* B = h->batch;
  for (mm_handle* m : B->members) {
    if (!m->have_state) return fail(h, MM_ERR_STATE, "a member has no state");
    if (!m->have_vel) return fail(h, MM_ERR_STATE, "a member has no velocity");
    if (!m->have_dt) return fail(h, MM_ERR_STATE, "a member has no dt");
  }
  DeviceGuard dg(h->device);
  mm_status st;
  if ((st = upload_args(h)) != MM_OK) return st;
  bool recording = false;
  for (mm_handle* m : B->members) {
    recording = recording || m->rec.active;
    if (m->rec.active && m->rec.nsub + n > m->rec.max_sub)
      return fail(h, MM_ERR_STATE, "a member's recording: more substeps than reserved");
  }
  if (recording || !h->use_graphs) {
    // direct launches; recording members take their checkpoints between them
    for (int i = 0; i < n; ++i) {
      for (mm_handle* m : B->members)
        if (m->rec.active && (st = rec_push_substep(m)) != MM_OK) {
          h->err = m->err;
          return st;
        }
      CK(launch_batch(h, i & 1, h->stream));
      for (mm_handle* m : B->members) m->parity ^= 1;
    }
    return MM_OK;
  }
  auto it = B->graphs.find(n);
  if (it == B->graphs.end()) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < n && le == cudaSuccess; ++i) le = launch_batch(h, i & 1, h->cap);
    cudaError_t ce = cudaStreamEndCapture(h->cap, &graph);
    if (le != cudaSuccess) return cuda_fail(h, "batched substep launch during capture", le);
    CK(ce);
    cudaGraphExec_t exec;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    it = B->graphs.emplace(n, exec).first;
  }
  CK(cudaGraphLaunch(it->second, h->stream));
  for (mm_handle* m : B->members) m->parity ^= (n & 1);
  return MM_OK;
}

// Checks (and clears) every member's device status; reports the first failure.
mm_status batch_sync(mm_handle* h) {
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream));
  mm_status first = MM_OK;
  for (size_t i = 0; i < h->batch->members.size(); ++i) {
    mm_handle* m = h->batch->members[i];
    const mm_status st = check_status(m);
    if (st != MM_OK && first == MM_OK) {
      first = st;
      h->err = "member " + std::to_string(i) + ": " + m->err;
    }
  }
  return first;
}

const std::vector<mm_handle*>& batch_members(mm_handle* h) { return h->batch->members; }

// grid, block, shared memory, bulk copies (always), ring stages, largest
// chunk (values), tiles, V, tile_work, chunk_bytes, tuned, two cells per warp
mm_status batch_launch_info(mm_handle* h, int* info, int n) {
  const BatchPlan* B = h->batch;
  const int v[12] = {B->grid,    B->block, (int)B->smem,   1,         B->S,     B->stage_elems,
                     B->ntiles,  B->V,     B->tile_work,   B->chunk_bytes, B->tuned, B->pairs};
  for (int i = 0; i < n && i < 12; ++i) info[i] = v[i];
  return MM_OK;
}

void batch_free(mm_handle* h) {
  BatchPlan* B = h->batch;
  if (!B) return;
  clear_graphs(B);
  for (mm_handle* m : B->members) {
    m->owner = nullptr;
    mm_destroy(m);
  }
  if (B->d_args) cudaFree(B->d_args);
  if (B->d_tiles) cudaFree(B->d_tiles);
  if (B->tile_mass) cudaFree(B->tile_mass);
  delete B;
  h->batch = nullptr;
}

}  // namespace mmh

extern "C" {

mm_status mm_create_batch(int n, const mm_grid* grids, const mm_rates* rates, mm_precision prec,
                          void* stream, mm_handle** out) {
  MM_TRACE("mm_create_batch");
  g_create_error.clear();
  if (!out) return fail(nullptr, MM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || !grids || !rates) return fail(nullptr, MM_ERR_INVALID, "n >= 1, grids and rates");
  if (prec != MM_FP64 && prec != MM_FP32_MIXED)
    return fail(nullptr, MM_ERR_INVALID, "unknown precision");
  // one vector width for every member: float32 8 (or 4) nodes per lane,
  // float64 2, each a whole number of 16-byte vectors for the bulk copies
  int V = prec == MM_FP64 ? 2 : MM_BATCH_FP32_VMAX;
  for (int i = 0; i < n; ++i) {
    if (prec == MM_FP32_MIXED && grids[i].ns % 8 != 0) V = 4;
    if (grids[i].ns % V != 0 || (prec == MM_FP32_MIXED && grids[i].ns % 4 != 0))
      return fail(nullptr, MM_ERR_UNSUPPORTED,
                  prec == MM_FP64 ? "batch members need an even ns in MM_FP64"
                                  : "batch members need ns divisible by 4 in MM_FP32_MIXED");
  }
  mm_handle* h = new mm_handle();
  h->prec = prec;
  h->stream = (cudaStream_t)stream;
  h->tsz = prec == MM_FP64 ? 8 : 4;
  h->batch = new BatchPlan();
  h->batch->V = V;
  auto bail = [&](mm_status st) {
    if (g_create_error.empty()) g_create_error = h->err;
    batch_free(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
    return st;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cuda_fail(h, "batch setup", e);
    return bail(MM_ERR_CUDA);
  }
  for (int i = 0; i < n; ++i) {
    mm_handle* m = nullptr;
    mm_status st = mm_create(&grids[i], &rates[i], prec, stream, &m);
    if (st != MM_OK) {
      char buf[96];
      snprintf(buf, sizeof buf, "member %d: ", i);
      g_create_error = std::string(buf) + g_create_error;
      return bail(st);
    }
    m->owner = h;
    h->batch->members.push_back(m);
    h->ncells += m->ncells;
  }
  e = cudaMalloc(&h->batch->d_args, 2 * (size_t)n *
                                        (prec == MM_FP64 ? sizeof(StepArgs<double>)
                                                         : sizeof(StepArgs<float>)));
  if (e != cudaSuccess) {
    cuda_fail(h, "cudaMalloc batch arguments", e);
    return bail(MM_ERR_OOM);
  }
  int tw = 8192, cb = kChunkBytes;
  auto c = g_tune_cache.find(batch_signature(h));
  if (c != g_tune_cache.end()) {
    tw = c->second.tile_work;
    cb = c->second.chunk_bytes;
    h->batch->pairs = c->second.pairs;
    h->batch->tuned = 1;
  }
  mm_status st = make_plan(h, tw, cb);
  if (st != MM_OK) return bail(st);
  *out = h;
  return MM_OK;
}

mm_status mm_batch_member(mm_handle* h, int i, mm_handle** member) {
  if (!h || !member) return MM_ERR_INVALID;
  if (!h->batch) return fail(h, MM_ERR_INVALID, "not a batch handle");
  if (i < 0 || i >= (int)h->batch->members.size())
    return fail(h, MM_ERR_INVALID, "member index out of range");
  *member = h->batch->members[i];
  return MM_OK;
}

mm_status mm_batch_autotune(mm_handle* h, int substeps, mm_batch_tune* results, int max_results,
                            int* n_results) {
  MM_TRACE("mm_batch_autotune");
  if (!h) return MM_ERR_INVALID;
  if (!h->batch) return fail(h, MM_ERR_INVALID, "not a batch handle");
  if (substeps < 1) return fail(h, MM_ERR_INVALID, "substeps >= 1");
  BatchPlan* B = h->batch;
  for (mm_handle* m : B->members)
    if (!m->have_state || !m->have_vel || !m->have_dt || m->rec.active)
      return fail(h, MM_ERR_STATE, "autotune needs every member set up and not recording");
  DeviceGuard dg(h->device);
  Snapshot sn;
  mm_status st;
  if ((st = snapshot(h, sn, true)) != MM_OK) return st;
  const int works[] = {1024, 2048, 4096, 8192, 16384, 32768};
  const int chunks[] = {2048, 4096, 8192};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_w = B->tile_work, best_c = B->chunk_bytes, best_p = B->pairs, nres = 0;
  for (int pr = 1; pr >= 0 && st == MM_OK; --pr)
    for (int cb : chunks)
    for (int tw : works) {
      B->pairs = pr;
      if ((st = make_plan(h, tw, cb)) != MM_OK) break;
      B->args_par.clear();
      if ((st = upload_args(h)) != MM_OK) break;
      // one warm-up substep, then the timed ones, all from the saved state
      CK(launch_batch(h, 0, h->stream));
      CK(cudaEventRecord(e0, h->stream));
      for (int i = 0; i < substeps; ++i) CK(launch_batch(h, (i + 1) & 1, h->stream));
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if ((st = snapshot(h, sn, false)) != MM_OK) break;
      if (results && nres < max_results) {
        results[nres].tile_work = tw;
        results[nres].chunk_bytes = cb;
        results[nres].ms_per_substep = ms / substeps;
        results[nres].cells_per_warp = pr ? 2 : 1;
      }
      ++nres;
      if (ms < best) {
        best = ms;
        best_w = tw;
        best_c = cb;
        best_p = pr;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sn.buf);
  if (st != MM_OK) return st;
  B->pairs = best_p;
  if ((st = make_plan(h, best_w, best_c)) != MM_OK) return st;
  B->args_par.clear();
  B->tuned = 1;
  g_tune_cache[batch_signature(h)] = {best_w, best_c, best_p};
  if (n_results) *n_results = std::min(nres, max_results);
  return batch_sync(h);
}

}  // extern "C"
