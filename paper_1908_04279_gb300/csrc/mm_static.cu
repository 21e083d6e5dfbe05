// Allocation-free variant of the macroscale moments reduction.
//
// Some callers cannot call cudaMalloc: a host application that reserved the
// GPU's memory for its own pool and forbids allocations it does not manage,
// or a time-critical loop that must not pay the device-wide synchronisation
// an allocation may imply. mm_moments_static serves them: it takes the state
// as caller-owned float64 device arrays, writes caller-owned outputs, and
// keeps its only scratch -- one float64 partial-sum record per cell -- in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits. The array is placed on a device when this module is
// loaded there, which under CUDA's default lazy module loading is the first
// call on that device: a caller that reserves the GPU's memory for its own
// pool makes one call before reserving it.
//
// The per-cell records are reduced in a fixed order by a single block, so the
// scalars do not depend on the launch shape. Every record is rewritten by each
// call before it is read, so nothing in the array has to be cleared; calls
// that overlap on the GPU (on different streams, or from different threads)
// share the array and race.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "mm_internal.cuh"

namespace {

constexpr long long kStaticMaxCells = 65536;  // e.g. a 256 x 256 grid
constexpr int kRecord = 8;                     // doubles per cell record
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_cell_partials[kStaticMaxCells * kRecord];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

mm_status static_fail(mm_status st, const char* what, const char* detail = "") {
  char buf[256];
  snprintf(buf, sizeof buf, "mm_moments_static: %s%s", what, detail);
  mm::set_thread_error(buf);
  return st;
}

__device__ __forceinline__ double warp_sum_s(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Sum over the block; valid in thread 0. red holds >= 32 doubles.
__device__ double block_sum_s(double x, double* red) {
  x = warp_sum_s(x);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Per cell (one block, threads over theta): the 12 moment fields of the
// handle path's moments, and the cell's record of the global sums
// {N_psi, bound, free, sum psi cos, sum psi sin, sum psi, tr sigma_a}.
__global__ void k_moments_cells(const double* psi, const double* mb, const double* mf,
                                const double* c, long long ncells, int nth, int ns, double dth,
                                double ds, double L, double dA, double Fm, double ell,
                                double* fields, double* records) {
  __shared__ double red[32];
  for (long long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
    double f[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < nth; k += blockDim.x) {
      const double ct = cos(k * dth), st = sin(k * dth);
      const double p = psi[cell * nth + k];
      const double* row = mb + ((size_t)cell * nth + k) * ns;
      double nbk = 0.0, m1k = 0.0;
      for (int j = 0; j < ns; ++j) {
        nbk += row[j] * ds;
        m1k += (-0.5 * L + (j + 0.5) * ds) * row[j] * ds;
      }
      f[0] += p * dth;
      f[1] += p * ct * dth;
      f[2] += p * st * dth;
      f[3] += p * (ct * ct - 0.5) * dth;
      f[4] += p * ct * st * dth;
      f[5] += Fm * ct * p * nbk * dth;
      f[6] += Fm * st * p * nbk * dth;
      f[7] += Fm * ell * ct * ct * p * m1k * dth;
      f[8] += Fm * ell * ct * st * p * m1k * dth;
      f[9] += Fm * ell * st * st * p * m1k * dth;
      f[10] += p * ct;
      f[11] += p * st;
      f[12] += p;
    }
    double tot[13];
#pragma unroll
    for (int q = 0; q < 13; ++q) tot[q] = block_sum_s(f[q], red);
    if (threadIdx.x == 0) {
      const double cc = c[cell], ff = mf[cell];
      if (fields) {
        const int order[12] = {0, 1, 2, 3, 4, -1, -2, 5, 6, 7, 8, 9};
        for (int q = 0; q < 12; ++q)
          fields[(size_t)q * ncells + cell] =
              order[q] >= 0 ? tot[order[q]] : (order[q] == -1 ? cc : ff);
      }
      double* rec = records + (size_t)cell * kRecord;
      rec[0] = tot[0] * dA;
      rec[1] = cc * dA;
      rec[2] = ff * dA;
      rec[3] = tot[10];
      rec[4] = tot[11];
      rec[5] = tot[12];
      rec[6] = tot[7] + tot[9];
      rec[7] = 0.0;
    }
  }
}

// One block adds the cell records in a fixed order (thread t takes cells
// t, t + blockDim, ...; then a fixed tree) and writes the 8 scalars.
__global__ void k_moments_finalize(const double* records, long long ncells, double* scalars) {
  __shared__ double red[32];
  double t[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long long cell = threadIdx.x; cell < ncells; cell += blockDim.x)
    for (int q = 0; q < 7; ++q) t[q] += records[(size_t)cell * kRecord + q];
  double s[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) s[q] = block_sum_s(t[q], red);
  if (threadIdx.x == 0) {
    scalars[0] = s[0];
    scalars[1] = s[1];
    scalars[2] = s[2];
    scalars[3] = s[1] + s[2];
    scalars[4] = sqrt(s[3] * s[3] + s[4] * s[4]) / s[5];
    scalars[5] = s[6] / (double)ncells;
    scalars[6] = s[3];
    scalars[7] = s[4];
  }
}

}  // namespace

extern "C" mm_status mm_moments_static(const mm_grid* grid, const mm_rates* rates,
                                       const double* psi, const double* mb, const double* mf,
                                       const double* c, double* fields, double* scalars,
                                       void* stream) {
  if (!grid || !rates || !psi || !mb || !mf || !c || !scalars)
    return static_fail(MM_ERR_INVALID, "a required pointer is NULL");
  if (grid->nx < 1 || grid->ny < 1 || grid->ntheta < 1 || grid->ns < 1 || !(grid->L > 0.0))
    return static_fail(MM_ERR_INVALID, "grid sizes must be >= 1 and L > 0");
  const long long ncells = (long long)grid->nx * grid->ny;
  if (ncells > kStaticMaxCells) {
    char buf[160];
    snprintf(buf, sizeof buf,
             "%lld cells exceed the static scratch limit of %lld cells "
             "(use mm_moments on a handle instead)",
             ncells, kStaticMaxCells);
    return static_fail(MM_ERR_UNSUPPORTED, buf);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(MM_ERR_CUDA, "cudaGetDevice: ", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return static_fail(MM_ERR_UNSUPPORTED, "device ordinal out of range");
  void* records = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name of
    // the array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_cell_partials);
      if (e != cudaSuccess) return static_fail(MM_ERR_CUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    records = g_scratch_addr[dev];
  }
  const int nth = grid->ntheta;
  const double dth = 2.0 * 3.14159265358979323846264338327950288 / nth;
  const double ds = grid->L / grid->ns;
  const double dA = (1.0 / grid->nx) * (1.0 / grid->ny);
  const int block = nth >= 128 ? 128 : (nth >= 64 ? 64 : 32);
  const long long g = ncells < 1216 ? ncells : 1216;
  cudaStream_t s = (cudaStream_t)stream;
  k_moments_cells<<<(int)g, block, 0, s>>>(psi, mb, mf, c, ncells, nth, grid->ns, dth, ds,
                                           grid->L, dA, rates->force_scale, rates->ell, fields,
                                           (double*)records);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(MM_ERR_CUDA, "moments launch: ", cudaGetErrorString(e));
  k_moments_finalize<<<1, 256, 0, s>>>((const double*)records, ncells, scalars);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(MM_ERR_CUDA, "finalize launch: ", cudaGetErrorString(e));
  return MM_OK;
}
