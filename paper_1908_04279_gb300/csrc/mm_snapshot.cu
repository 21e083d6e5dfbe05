// Bitwise checkpoint and restart of one instance.
//
// mm_get_state / mm_set_state exchange the physical state in float64, and
// mm_set_state re-derives everything else from it (n_b, C, the scale-down,
// Mf, and in the float32 form the filament number the mass correction holds
// fixed). A run restarted that way continues the same physics but not the
// same bits: the re-derived sums round in another order, psi is exported with
// the pending mass-correction factor applied in float64, and the reference
// filament number becomes that of the restored state. A snapshot instead
// copies the arrays exactly as the substep kernel left them, in the state
// precision, together with the device scalars the next substep reads (dt,
// the pending correction factor, the reference and current filament numbers)
// and the velocity in effect, so that a handle loaded from it continues the
// uninterrupted run bit for bit.
//
// Layout (every block starts on a 256-byte boundary): a 256-byte header
// {magic, version, precision, nx, ny, ntheta, ns, flags, L, dt, psi_scale,
// mass0, mass}, then psi, n_b, Mb, Mf, C, M in the state precision, then the
// velocity [2][ny][nx] in float64.
#include <cstddef>
#include <cstdint>
#include <cstring>

#include "mm_host.h"

using namespace mmh;

namespace {

constexpr char kMagic[8] = {'M', 'M', 'S', 'N', 'A', 'P', '0', '1'};
constexpr int kVersion = 1;
constexpr size_t kAlign = 256;

struct SnapHeader {
  char magic[8];
  int32_t version, precision, nx, ny, ntheta, ns, flags, pad;
  double L;
  double dev[4];  // dt, psi_scale, mass0, mass: the first four DevParams fields
};
static_assert(sizeof(SnapHeader) <= kAlign, "snapshot header");
static_assert(offsetof(DevParams, psi_scale) == 8 && offsetof(DevParams, mass) == 24,
              "DevParams starts with dt, psi_scale, mass0, mass");

constexpr int kHaveVel = 1, kHaveDt = 2;

size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

struct Blocks {
  size_t off[8];  // psi, nb, mb, mf, c, mtot, u64, end
};

Blocks blocks_of(const mm_handle* h) {
  Blocks b;
  const size_t t = h->tsz, nc = (size_t)h->ncells;
  const size_t sz[7] = {h->rows * t, h->rows * t, h->mbn * t, nc * t, nc * t, nc * t, 2 * nc * 8};
  size_t o = kAlign;
  for (int i = 0; i < 7; ++i) {
    b.off[i] = o;
    o += up(sz[i]);
  }
  b.off[7] = o;
  return b;
}

mm_status snap_check(mm_handle* h, size_t bytes) {
  if (h->anchors || h->capture)
    return fail(h, MM_ERR_UNSUPPORTED,
                "snapshots of a handle with non-local anchors or a capture radius are not supported");
  if (bytes < blocks_of(h).off[7]) return fail(h, MM_ERR_INVALID, "snapshot buffer too small");
  return MM_OK;
}

}  // namespace

extern "C" {

mm_status mm_snapshot_bytes(mm_handle* h, size_t* bytes) {
  if (!h || !bytes) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  *bytes = blocks_of(h).off[7];
  return MM_OK;
}

mm_status mm_save_snapshot(mm_handle* h, void* buf, size_t bytes, int on_device) {
  MM_TRACE("mm_save_snapshot");
  if (!h || !buf) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  mm_status st = snap_check(h, bytes);
  if (st != MM_OK) return st;
  if (!h->have_state) return fail(h, MM_ERR_STATE, "no state: call mm_set_state first");
  DeviceGuard dg(h->device);
  const Blocks b = blocks_of(h);
  const size_t t = h->tsz, nc = (size_t)h->ncells;
  SnapHeader hd{};
  memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.precision = (int32_t)h->prec;
  hd.nx = h->g.nx;
  hd.ny = h->g.ny;
  hd.ntheta = h->g.ntheta;
  hd.ns = h->g.ns;
  hd.flags = (h->have_vel ? kHaveVel : 0) | (h->have_dt ? kHaveDt : 0);
  hd.L = h->g.L;
  char* base = (char*)buf;
  const cudaMemcpyKind to = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // the header's static part, then its device scalars, then the arrays, in
  // stream order after every substep already enqueued
  if (on_device) {
    CK(cudaMemcpyAsync(base, &hd, sizeof hd, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));  // hd lives on this stack frame
  } else {
    memcpy(base, &hd, sizeof hd);
  }
  CK(cudaMemcpyAsync(base + offsetof(SnapHeader, dev), &h->prm->dt, 4 * 8, to, h->stream));
  const void* src[7] = {h->psi[h->parity], h->nb[h->parity], h->mb, h->mf, h->c, h->mtot, h->u64};
  const size_t sz[7] = {h->rows * t, h->rows * t, h->mbn * t, nc * t, nc * t, nc * t, 2 * nc * 8};
  for (int i = 0; i < 7; ++i) CK(cudaMemcpyAsync(base + b.off[i], src[i], sz[i], to, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

mm_status mm_load_snapshot(mm_handle* h, const void* buf, size_t bytes, int on_device) {
  MM_TRACE("mm_load_snapshot");
  if (!h || !buf) return MM_ERR_INVALID;
  if (h->batch) return not_for_batch(h);
  mm_status st = snap_check(h, bytes);
  if (st != MM_OK) return st;
  DeviceGuard dg(h->device);
  const char* base = (const char*)buf;
  SnapHeader hd{};
  if (on_device)
    CK(cudaMemcpy(&hd, base, sizeof hd, cudaMemcpyDeviceToHost));
  else
    memcpy(&hd, base, sizeof hd);
  if (memcmp(hd.magic, kMagic, 8) != 0 || hd.version != kVersion)
    return fail(h, MM_ERR_INVALID, "not a snapshot of this library version");
  if (hd.precision != (int32_t)h->prec || hd.nx != h->g.nx || hd.ny != h->g.ny ||
      hd.ntheta != h->g.ntheta || hd.ns != h->g.ns || hd.L != h->g.L)
    return fail(h, MM_ERR_INVALID, "the snapshot's grid or precision differs from the handle's");
  const Blocks b = blocks_of(h);
  const size_t t = h->tsz, nc = (size_t)h->ncells;
  const cudaMemcpyKind from = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  h->rec.active = false;  // a new state ends an adjoint recording (its memory is kept)
  h->parity = 0;
  void* dst[7] = {h->psi[0], h->nb[0], h->mb, h->mf, h->c, h->mtot, h->u64};
  const size_t sz[7] = {h->rows * t, h->rows * t, h->mbn * t, nc * t, nc * t, nc * t, 2 * nc * 8};
  for (int i = 0; i < 7; ++i) CK(cudaMemcpyAsync(dst[i], base + b.off[i], sz[i], from, h->stream));
  h->have_state = true;
  h->have_vel = h->have_dt = false;
  if (hd.flags & kHaveVel) {
    // the velocity's state-precision copy and per-cell block, derived as
    // mm_set_velocity derives them; the substep rule it also evaluates is
    // overwritten by the saved dt below
    if ((st = velocity_update(h)) != MM_OK) return st;
  }
  CK(cudaMemcpyAsync(&h->prm->dt, hd.dev, 4 * 8, cudaMemcpyHostToDevice, h->stream));
  h->have_dt = (hd.flags & kHaveDt) != 0;
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

}  // extern "C"
