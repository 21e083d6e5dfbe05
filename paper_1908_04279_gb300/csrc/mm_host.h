// Host-side internals of libmm shared by the C-ABI translation units
// (mm_api.cu: single instances and the adjoint; mm_batch_api.cu: the batched
// ensemble): the handle, error helpers and the substep launch constants.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define MM_HAVE_NVTX 1
#else
#define MM_HAVE_NVTX 0
#endif

#include "mm_internal.cuh"

using mm::DevParams;
using mm::StepArgs;

// Widest vector (values per lane) of the float32 substep kernel.
#ifndef MM_FP32_VMAX
#define MM_FP32_VMAX 8
#endif
// 1: the motor reverse kernel streams rows by bulk copies where they allow it.
#ifndef MM_ADJ_RING
#define MM_ADJ_RING 1
#endif
// Most row blocks per cell of the motor reverse kernel (float64, float32).
#ifndef MM_ADJ_MAX_UNITS
#define MM_ADJ_MAX_UNITS 8
#endif
#ifndef MM_ADJ_MAX_UNITS_F32
#define MM_ADJ_MAX_UNITS_F32 2
#endif
// Widest vector of the float32 adjoint kernel.
#ifndef MM_ADJ_FP32_VMAX
#define MM_ADJ_FP32_VMAX 8
#endif

namespace mm {
// The substep launched overlapped with the previous kernel of its stream
// (mm_step.cu; direct launches only).
template <typename T, int V>
cudaError_t launch_substep_overlapped(const StepArgs<T>& a, int grid, int block, size_t smem,
                                      bool tma, cudaStream_t s);
}  // namespace mm

namespace mmh {
inline thread_local std::string g_create_error;
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr size_t kStagingDoubles = size_t(1) << 22;  // 32 MiB of float64 staging
}  // namespace mmh

// State of an adjoint recording (mm_set_checkpointing / mm_adjoint_step).
// The checkpoints, the recomputed segment and the reverse-sweep buffers live
// in one device allocation (`slab`), kept after the recording ends so that a
// new recording with the same K and max_substeps reuses it; the per-velocity
// blocks are pooled the same way.
struct Recording {
  bool active = false;
  int K = 0, max_sub = 0, nsub = 0, nck = 0;
  int K2 = 0;  // inner checkpoint spacing (two levels when K2 < K; K2 = K: one level)
  int tail_done = 0;  // substeps of the last segment recorded straight into the slots
  int nslots = 0;  // recomputed-state slots (1..nslots; slot 0 is the segment's start)
  std::vector<void*> ick_mb, ick_psi, ick_nb, ick_mf;  // inner checkpoints of one outer segment
  double* ick_scale = nullptr;
  void* slab = nullptr;
  size_t slab_bytes = 0;
  std::vector<void*> vblocks;  // velocity blocks, reused across recordings
  std::vector<void*> ck_mb, ck_psi, ck_nb, ck_mf;  // checkpoints (states 0, K, 2K, ...)
  double* ck_scale = nullptr;                      // psi mass-correction factor per checkpoint
  std::vector<void*> sl_mb, sl_psi, sl_nb, sl_mf, sl_cpre;  // K + 1 recomputed states
  void* sl_c = nullptr;
  // velocity fields (and dt) in effect, in prescription order
  std::vector<void*> v_ucell;
  std::vector<double*> v_dt, v_lamG, v_lamu;
  std::vector<int> sub_vel;  // velocity index of every recorded substep
  // reverse-sweep buffers
  void* lpsi[2] = {nullptr, nullptr};
  void* lmf[2] = {nullptr, nullptr};
  void* Dd[2] = {nullptr, nullptr};
  void* lmb = nullptr;
  double* gpart = nullptr;
  double* seed[4] = {nullptr, nullptr, nullptr, nullptr};
  double* coef = nullptr;
  double* work = nullptr;  // [rows] float64 scratch for dL/dpsi0
  void* lnb = nullptr;    // [rows] adjoint of n_b (times ds) between the two reverse kernels
  void* cellc = nullptr;  // [cells][2] lam_C and f per cell
  int units = 1, rows_per_unit = 1;  // row blocks per cell of the motor reverse kernel
  int grid_psi = 1, grid_motor = 1;  // blocks of 4 warps of the two reverse kernels
  int ring_rc = 0, ring_ch = 0, ring_s = 0;  // bulk-copy ring of the motor kernel (0: off)
  // One level: a second set of K slots, so that the replay of the next segment
  // (on rstream) runs while the current segment is reversed (on the handle's
  // stream); ev_rep / ev_rev order the two per slot set.
  bool overlap = false;
  std::vector<void*> sl2_mb, sl2_psi, sl2_nb, sl2_mf, sl2_cpre;
  cudaStream_t rstream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_rep[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
};

namespace mmh {
struct BatchPlan;
}

struct mm_handle {
  Recording rec;
  // batched ensemble: a batch handle owns its member handles (one per
  // instance, each an ordinary handle with its own state); a member points
  // back to its batch
  mmh::BatchPlan* batch = nullptr;
  mm_handle* owner = nullptr;
  mm_grid g{};
  mm_rates r{};
  mm_precision prec = MM_FP64;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream used only for graph capture
  int device = 0, sms = 0;
  long long ncells = 0;
  size_t rows = 0, mbn = 0, tsz = 8;
  void* mb = nullptr;
  void* psi[2] = {nullptr, nullptr};
  void* nb[2] = {nullptr, nullptr};
  void* mf = nullptr;    // free, coarse and total motors per cell, state precision
  void* c = nullptr;
  void* mtot = nullptr;
  void* u = nullptr;
  void* ucell = nullptr;
  double* u64 = nullptr;
  void* trig = nullptr;
  double* trig64 = nullptr;
  double* partial = nullptr;
  double* fields = nullptr;
  double* staging = nullptr;
  double* diff_tab = nullptr;  // Crank-Nicolson factors of the three directions (mm_diffuse)
  int* local_n = nullptr;      // [cells] substeps per cell of mm_motor_local
  // non-local motor anchors (mm_set_anchors)
  bool anchors = false;
  int anc_wpb = 4;              // warps per block of the anchor substep
  void* anc_off = nullptr;      // [nth][ns] int2 anchor cell offsets
  int* anc_widx = nullptr;      // [nth][ns] index of each node's anchor in the window
  unsigned short* anc_wtab = nullptr;  // [2][nth][ns] block-window entry and run place of each node
  bool anc_bw = false;          // the block's 4 warps share one window
  unsigned* anc_runend = nullptr;  // [nth][ns / V] run ends of each lane slot
  unsigned* anc_rtab = nullptr;    // block window: per-entry sum indices, lane end marks and counts
  int anc_nsr = 0;                 // slot runs per cell
  int anc_sg[4] = {0, 0, 0, 0};    // block window: places, lane chunk, mark words, entries
  int anc_win[4] = {0, 0, 0, 0};  // window: first x and y offset, width, height (0: none)
  double* anc_cacc = nullptr;   // [cells] float64 accumulators of C
  double* anc_fsc = nullptr;    // [cells] scale-down factors
  int* anc_flags = nullptr;     // [4] scale-down flags
  // tangent-linear mode (mm_set_tangent): the tangent of the state along a
  // direction of the rates, advanced with it by every substep
  bool tangent = false;
  double tan_dp[3] = {0.0, 0.0, 0.0};  // d k_off, d v_walk, d k_on
  void* tan_mb = nullptr;
  void* tan_psi[2] = {nullptr, nullptr};
  void* tan_nb[2] = {nullptr, nullptr};
  void* tan_mf = nullptr;
  int tan_seg = 1, tan_grid = 1;
  // finite capture radius (mm_set_capture): the anchor axis of Mb
  bool capture = false;
  double rc = 0.0;
  int rc_nconf = 0, rc_nlines = 0, rc_nchunks = 0, rc_motor_grid = 1;
  void* rc_mb = nullptr;   // [cells][nconf] motor density, anchor-major (template order)
  void* rc_ls = nullptr;   // [cells][nlines] line sums of Mb ds
  void* rc_tab = nullptr;  // the template's device tables (one block)
  size_t rc_tab_off[7] = {0, 0, 0, 0, 0, 0, 0};
  std::vector<int> rc_host_lines;  // [nlines][6] (k, dx, dy, j0, len, off)
  std::vector<double> rc_host_w;   // [nth][ns] 1 / n_a
  // thin-gap fluid solve (mm_fluid_setup)
  bool fluid = false;
  double fl_eps = 0.0, fl_z0 = 0.0;
  int fl_plan[3] = {-1, -1, -1};  // cuFFT plans: 5 forward, 3 forward, 2 inverse transforms
  double* fl_tab = nullptr;       // [ny][nx/2+1] (g_T, g_L) per mode
  double* fl_hat = nullptr;       // [10][ny][nx/2+1] complex: 5 force/dipole, 3 stress, 2 velocity
  double* fl_real = nullptr;      // [10][cells rounded up to even] real inputs and outputs
  size_t staging_n = 0;  // float64 values the staging buffer holds
  DevParams* prm = nullptr;
  int npartial = 0;
  int parity = 0;
  double dt = 0.0;
  bool have_state = false, have_vel = false, have_dt = false;
  // substep launch configuration
  int V = 1, seg = 1, block = 128, grid_step = 1, grid_mom = 1;
  int stages = 1, chunk_rows = 1, chunks_per_cell = 1;
  bool tma = false;
  size_t smem = 0;
  std::map<long long, cudaGraphExec_t> graphs;
  bool use_graphs = true;
  std::string err;
};

namespace mmh {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline mm_status fail(mm_handle* h, mm_status st, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_create_error = msg;
  return st;
}

inline mm_status cuda_fail(mm_handle* h, const char* what, cudaError_t e) {
  return fail(h, MM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                                  cudaGetErrorString(e) + ")");
}

// NVTX range over one ABI call, for Nsight tools' timelines and range filters
// (header-only NVTX 3; a no-op when no tool is attached, and compiled out
// where the toolkit has no NVTX headers).
struct TraceRange {
#if MM_HAVE_NVTX
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
#else
  explicit TraceRange(const char*) {}
#endif
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define MM_TRACE(name) ::mmh::TraceRange mm_trace_range_(name)

#define CK(...)                                               \
  do {                                                        \
    cudaError_t e_ = (__VA_ARGS__);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, #__VA_ARGS__, e_); \
  } while (0)

inline bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }


// Substep launch plan: s-rows stream through each warp's ring in chunks of at
// most kChunkBytes, with up to kWarpInflightBytes in flight per warp.
constexpr int kChunkBytes = 4096;
constexpr int kWarpInflightBytes = 8192;
constexpr int kMaxWarpsPerBlock = 4;
constexpr size_t kSmemBudget = 200 * 1024;  // dynamic shared memory per block at most
constexpr long long kAnchorWindowMax = 1024;   // anchor window entries kept in shared memory
constexpr long long kAnchorBlockWindowMax = 4096;  // entries of a window shared by a block

// Defined in mm_api.cu.
mm_status check_rates(const mm_rates* r, mm_handle* h);
mm_status check_status(mm_handle* h);
mm_status rec_save_checkpoint(mm_handle* h, int i);
template <typename T>
StepArgs<T> step_args(mm_handle* h, int parity);
mm_status rec_push_substep(mm_handle* h);  // checkpoint bookkeeping of one recorded substep
mm_status launch_substeps(mm_handle* h, int n);  // n substeps on the live state (graphs)
mm_status run_init(mm_handle* h);  // n_b, C, the scale-down and Mf of the live state
mm_status run_moments(mm_handle* h);  // the 12 moment fields and the scalars of the live state
mm_status velocity_update(mm_handle* h);  // h->u64 becomes the velocity in effect (and dt)

// Defined in mm_fluid.cu (thin-gap fluid solve).
void fluid_free(mm_handle* h);

// Defined in mm_anchor.cu (non-local motor anchors).
mm_status anchor_alloc(mm_handle* h);  // the anchor tables and accumulators
mm_status anchor_table(mm_handle* h);
cudaError_t launch_anchor_substep(mm_handle* h, int parity, cudaStream_t s);
mm_status run_init_anchor(mm_handle* h);
mm_status anchor_force(mm_handle* h);

// Defined in mm_capture.cu (finite capture radius).
void capture_free(mm_handle* h);
cudaError_t launch_capture_substep(mm_handle* h, int parity, cudaStream_t s);
mm_status run_init_capture(mm_handle* h);
mm_status capture_rows(mm_handle* h);  // per-node totals over the anchors into h->mb

// Defined in mm_tangent.cu (tangent-linear mode).
void tangent_free(mm_handle* h);
cudaError_t launch_tangent_substep(mm_handle* h, int parity, cudaStream_t s);
mm_status tangent_zero(mm_handle* h);
mm_status get_array(mm_handle* h, double* dst, const void* src, size_t n, int on_device,
                    const double* scale);

// Defined in mm_batch_api.cu.
mm_status batch_micro_step(mm_handle* h, int n);
void batch_free(mm_handle* h);
mm_status batch_sync(mm_handle* h);
const std::vector<mm_handle*>& batch_members(mm_handle* h);
mm_status batch_launch_info(mm_handle* h, int* info, int n);
// Walking rate v / ds of Eq. 4, evaluated once on the host for every kernel.
inline double walk_cw(const mm_handle* h) { return h->r.v_walk / (h->g.L / h->g.ns); }

inline mm_status not_for_batch(mm_handle* h) {
  return fail(h, MM_ERR_INVALID,
              "a batch handle: per-instance calls go to its members (mm_batch_member)");
}

}  // namespace mmh
