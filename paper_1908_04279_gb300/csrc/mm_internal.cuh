// Internal declarations shared by the CUDA translation units of libmm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "mm.h"

namespace mm {

// Raises a kernel's dynamic shared-memory limit to at least `bytes`. The limit
// belongs to the kernel function, shared by every handle of the process: a
// handle that needs less must not lower it under another handle's launches.
inline cudaError_t raise_smem_limit(const void* f, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
template <typename F, typename = std::enable_if_t<std::is_function<F>::value>>
inline cudaError_t raise_smem_limit(F* f, size_t bytes) {
  return raise_smem_limit(reinterpret_cast<const void*>(f), bytes);
}

// Device-resident per-handle scalars. Kernels read dt and the rates from here
// (not from launch arguments) so that captured graphs stay valid when dt or
// the rates change.
struct DevParams {
  double dt;
  double psi_scale;   // mass-correction factor applied to psi on load (FP32)
  double mass0;       // target sum(psi) for the mass correction
  double mass;        // sum(psi) after the last substep (float64)
  double v_walk, k_on, k_off, glide, v_sp;
  double force_scale, ell;
  double dtmax[4];    // [adv, rot, rho_max, spare] for the dt rule (bits as u64)
  double scalars[8];  // global moments
  double sum_psi;     // sum of psi over all cells and angles (moments kernel)
  unsigned int counter;   // last-warp-done counter of the substep kernel
  unsigned int counter2;  // last-block-done counter of the moments kernel
  int status;             // bit 0: a bounded device wait gave up; bit 1: no valid dt;
                          // bit 2: a local substep count out of range; bit 3: the drain
                          // after a timeout gave up too (copies may still be in flight)
  unsigned int wait_limit;   // polls of an mbarrier before a wait gives up
  unsigned int debug_flags;  // bit 0: wait on a phase nothing completes (tests)
  int pad;
  double cw;  // v_walk / ds (evaluated on the host; the kernels only convert it)
};

// Everything a substep kernel touches, by value as a launch argument.
template <typename T>
struct StepArgs {
  int nx, ny, nth, ns;
  int seg;            // lanes per s-row segment (power of two <= 32)
  int stages;         // shared-memory ring depth per warp
  int chunk_rows;     // s-rows per ring stage (divides nth)
  int chunks_per_cell;
  int nb_tma;         // 1: stage the psi / n_b neighbourhood by bulk copies
  long long ncells;
  double inv_dx, inv_dy, inv_dth, dth, ds, L;
  float f_inv_dx, f_inv_dy, f_inv_dth, f_dth, f_ds;  // the same in float32
  const T* mb_in;     // [cells][nth][ns] Mb at step n (may equal mb_out: in place)
  T* mb_out;          // Mb at step n+1
  const T* psi_in;    // [cells][nth]
  T* psi_out;
  const T* nb_in;     // [cells][nth] n_b = sum_j Mb ds (precision T)
  T* nb_out;
  const T* mf_in;     // [cells] free motors (Eq. 6) at step n, state precision
  T* mf_out;          // free motors at step n+1 (may equal mf_in)
  T* c;               // [cells] coarse bound motors (Eq. 5)
  T* cpre_out;        // [cells] coarse density before the Alg. 2 scale-down, or NULL
  const T* mtot;      // [cells] total motors
  const T* ucell;     // [cells][12]: ux, uy, ux east, ux west, uy north, uy south,
                      //   Gxx, Gxy, Gyx, Gyy (central differences), 2 spare
  const T* trig;      // [4][nth]: cos th_k, sin th_k, cos th_{k+1/2}, sin th_{k+1/2}
  double* partial;    // [warps in the grid] per-warp sum(psi)
  DevParams* prm;
  int mass_correct;   // 1: compute psi_scale = mass0 / mass after the substep
};

// Everything the adjoint of one substep touches (mm_adjoint.cu). State n is
// the substep's input, state n+1 its output (both from the recomputed
// segment); lam_* are the adjoint variables. The per-cell sums over the rows
// (lam_Mf and D) are kept as `units` partials per cell, [units][cells], one per
// block of rows the motor kernel assigns to a warp; readers add them in order.
template <typename T>
struct AdjArgs {
  int nx, ny, nth, ns, seg;
  int units;          // row blocks per cell (power of two)
  int rows_per_unit;  // rows of one block (the last may be shorter)
  long long ncells;
  double inv_dx, inv_dy, inv_dth, dth, ds, L;
  const double* dt; // the substep's dt (device)
  double v_walk, k_on, k_off, glide, v_sp;
  double cw;        // v_walk / ds, the same value as DevParams::cw
  double inv_ds;    // 1 / ds
  const T* psi_n;   // [cells][nth]
  const T* nb_n;    // [cells][nth]
  const T* mb_n;    // [cells][nth][ns]
  const T* mf_n;    // [cells]
  const T* psi_np;  // psi at n+1
  const T* nb_np;   // n_b at n+1 (after the scale-down)
  const T* cpre_np; // coarse density before the scale-down at n+1
  const T* mtot;    // [cells]
  const T* ucell;   // [cells][12]
  const T* trig;    // [4][nth]
  const T* lpsi_in; // adjoint of psi at n+1
  const T* lmf_in;  // [units][cells] partials of the adjoint of Mf at n+1
  const T* D_in;    // [units][cells] partials of sum lam_Mb * Mb at n+1
  T* lpsi_out;      // adjoint of psi at n
  T* lnb;           // [cells][nth] adjoint of n_b^n (times ds), psi kernel -> motor kernel
  T* cellc;         // [cells][2] lam_C and the scale-down factor f of the cell at n+1
  T* lmb;           // adjoint of Mb: n+1 in, n out (in place)
  T* lmf_out;       // [units][cells] partials of the adjoint of Mf at n
  T* D_out;         // [units][cells] partials of sum lam_Mb * Mb at n
  double* lamG;     // [cells][4] accumulated adjoint of the velocity gradient
  double* lamu;     // [2][cells] accumulated direct adjoint of u
  double* gpart;    // [warps][4] accumulated k_off, v_walk, k_on adjoints
  DevParams* prm;   // status word and wait limit of the bounded waits
  int ring_rc;      // bulk-copy ring: rows per chunk (0: rows read with plain loads)
  int ring_ch;      // chunks per unit
  int ring_s;       // ring stages per warp
};

// One tile of the batched-ensemble substep: a run of consecutive cells of one
// instance (mm_batch.cu).
struct BatchTile {
  int inst;        // instance (index into the StepArgs table)
  int cell0;       // first cell
  int ncell;       // units (of cpu cells) in the tile
  int tile0;       // index of the instance's first tile
  int inst_tiles;  // tiles of the instance
  int ch, rc;      // chunks per unit, s-rows per chunk
  int cpu;         // cells per unit: 1, or 2 (two cells of one row: one chunk holds both
                   // cells' rows; a half-warp each takes psi and the close)
};

// Kernel launchers (defined in mm_step.cu); V = values per lane.
template <typename T, int V>
cudaError_t launch_substep(const StepArgs<T>& a, int grid, int block, size_t smem, bool tma,
                           cudaStream_t s);
size_t step_smem_per_warp(int S, int chunk_elems, int nth, int tsz);
template <typename T, int V>
cudaError_t substep_prepare(int block, size_t smem, bool tma, int* blocks_per_sm);

// Batched-ensemble launchers (mm_batch.cu): every instance's arguments in a
// device table, tiles in a device table, per-tile float64 sums of psi.
template <typename T, int V>
cudaError_t launch_substep_batch(const StepArgs<T>* insts, const BatchTile* tiles, int ntiles,
                                 double* tile_mass, int S, int stage_elems, int nth_max,
                                 bool masscorr, int grid, int block, size_t smem, cudaStream_t s);
template <typename T, int V>
cudaError_t substep_batch_prepare(int block, size_t smem, int* blocks_per_sm);

// Auxiliary kernels (mm_aux.cu).
template <typename TO, typename TI>
cudaError_t launch_convert(TO* out, const TI* in, size_t n, const double* scale, cudaStream_t s);
template <typename T>
cudaError_t launch_prep_ucell(T* ucell, const double* u64, long long ncells, int nx, int ny,
                              double inv_dx, double inv_dy, cudaStream_t s);
template <typename T>
cudaError_t launch_init_cells(T* mb, const T* psi, T* nb, T* mf, T* c, const T* mtot,
                              long long ncells, int nth, int ns, double ds, double dth,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_dt_max(const T* psi, const T* nb, const T* u, const T* trig, long long ncells,
                          int nx, int ny, int nth, double inv_dx, double inv_dy, double inv_dth,
                          double dth, double glide, double vsp, DevParams* prm, cudaStream_t s);
cudaError_t launch_dt_finalize(DevParams* prm, double ds, double L, double cfl, cudaStream_t s);
template <typename T>
cudaError_t launch_moments(const T* psi, const T* mb, const T* mf, const T* c,
                           const double* trig, long long ncells, int nth, int ns, int V, int seg,
                           double dth, double ds, double L, double dA, double* fields,
                           double* partial, int nblocks, DevParams* prm, cudaStream_t s);

// Adjoint kernels (mm_adjoint.cu).
template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T>& a, int V, int grid_psi, int grid_motor,
                           cudaStream_t s);
size_t adj_ring_warp_bytes(int rc, int ns, int S, int tsz);
template <typename T>
cudaError_t adj_motor_occupancy(int V, int ring_rc, int ns, int S, int* bps);
template <typename T>
cudaError_t launch_adj_seed(int kind, const double* coef, const T* psi, const T* mb,
                            const double* dpsi, const double* dnb, const double* dm1,
                            const double* dmf, T* lpsi, T* lmb, T* lmf, T* D, long long ncells,
                            int nth, int ns, double ds, double L, const T* trig, bool mb_seeded,
                            cudaStream_t s);
cudaError_t launch_adj_finish(const double* lamG, const double* lamu, double* dLdu, int nx, int ny,
                              double inv_dx, double inv_dy, cudaStream_t s);
// The seed coefficients and value of a built-in observable from the moments'
// global scalars (kind 1: polar order, 2: mean tr sigma_a with `stress_coef`):
// coef[0..2] and coef[3] = value.
cudaError_t launch_adj_observable(int kind, const DevParams* prm, double stress_coef, double* coef,
                                  cudaStream_t s);
// Fixed-order sum of the per-warp parameter adjoints: out[0..2].
cudaError_t launch_adj_params(const double* gpart, int nwarps, double* out, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_psi0(const T* lpsi, const T* lmf, int units, const T* nb, double dth,
                            long long rows, int nth, double* out, cudaStream_t s);

// Filament diffusion (mm_diffuse.cu): the Crank-Nicolson factors of the three
// directions (3 n + 2 values each), then one direction (mode 0 theta, 1 x,
// 2 y) for every line of psi; scale (device, may be NULL) multiplies psi on
// load.
cudaError_t launch_cn_factors(double* tab0, int n0, double a0, double* tab1, int n1, double a1,
                              double* tab2, int n2, double a2, cudaStream_t s);
template <typename T>
cudaError_t launch_cn_lines(T* psi, int mode, int nx, int ny, int nth, const double* tab, int n,
                            double c, double ha, const double* scale, cudaStream_t s);
cudaError_t launch_set_scale_one(double* scale, cudaStream_t s);
// Up to kMaxCopySegs device-to-device copies in one launch (a checkpoint of the
// state: one launch instead of one copy operation per array).
constexpr int kMaxCopySegs = 6;
struct CopySegs {
  const void* src[kMaxCopySegs];
  void* dst[kMaxCopySegs];
  size_t bytes[kMaxCopySegs];
  int n;
};
cudaError_t launch_copy_multi(const CopySegs& c, cudaStream_t s);

// Message returned by mm_last_error(NULL) on this thread.
void set_thread_error(const char* msg);

}  // namespace mm
