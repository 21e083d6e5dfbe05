// Finite capture radius (mm_set_capture): the anchor r0 of a bound motor kept
// as an axis of the motor density, Mb(r0, x, theta, s), tracked only where
// the motor head x + (l/L) s p is within reach of r0 (Sec. 2's B_rc(r0), the
// indicator of Eq. 4), and Alg. 2 run per r0: every configuration of
// B_rc(r0) by the RK2 of Eq. 4, the coarse reduction of Eq. 5 at r0, the
// scale-down at r0, Eq. 6 at r0.
//
// Model (the same readings as the oracle): r0 ranges over the grid's cells; a
// cell is within reach of a head when the distance from the head to the
// cell's square is at most rc; a motor keeps its anchor while it walks, so
// for each (x, theta, r0) the nodes in reach form walking lines with no
// inflow at a line's first node and donor-cell outflow at its last; the
// binding term k_on Mf(r0) is shared among the n_a anchors in reach of the
// node, k_on Mf(r0) / n_a; n_b sums over anchors and nodes; the force of
// Eq. 10 acts in the cell under the head.
//
// Layout (the paper's, Sec. 3.2 "Reordering Storage"): anchor-major,
// mb[r0][c], c over B_rc(r0) in template order -- the lines sorted by
// orientation, then first node, dy, dx -- the same for every r0, s contiguous
// within a line. One substep is three launches:
//   k_rc_psi    warp per cell: psi by Eq. 1 (velocities from n_b and u), the
//               float32 form's mass sums;
//   k_rc_motor  warp per anchor r0 (Alg. 2's loop over r0): the anchor's
//               configurations in chunks of whole lines, positions across the
//               lanes (p = 32 v + lane, coalesced loads), the walking stencil
//               by shuffles with per-position line-start / line-end flags; the
//               line sums of Mb ds (kept per (r0, line) for n_b), the coarse
//               density C(r0) with psi^{n+1} of each line's filament cell, the
//               scale-down and Mf(r0) -- all local to the warp, no atomics;
//   k_rc_nb     thread per (x, theta): n_b = the line sums of its lines over
//               the anchors, in template order (deterministic).
#include <algorithm>
#include <vector>

#include "mm_async.cuh"
#include "mm_cell.cuh"
#include "mm_host.h"

namespace mm {

// Everything the capture-radius kernels touch.
template <typename T>
struct RcArgs {
  int nx, ny, nth, ns, nconf, nlines, nchunks;
  long long ncells;
  T* mb;                       // [cells][nconf] motor density, anchor-major
  T* ls;                       // [cells][nlines] sum of Mb ds of every line
  const int4* line;            // [nlines] {dx, dy, k, len}: filament cell = r0 - (dx, dy)
  const int* loff;             // [nlines] first entry of the line in mb[r0][]
  const int4* chunk;           // [nchunks] {first entry, entries, first line, lines}
  const unsigned char* meta;   // [nconf] bit 0: a line's first node, bit 1: its last
  const T* w;                  // [nconf] binding weight 1 / n_a of the entry's node
  const int* krange;           // [nth + 1] first line of each orientation
  const unsigned* cmask;       // [nchunks][32] per lane of a chunk: its 8 entries' line-start
                               // flags (bits 0-7), line-end flags (8-15), valid (16-23)
  const T* cw;                 // [nchunks][256] the chunk's weights, entry 8 lane + v
  const T* mtot;
  T* mf;
  T* c;
  const DevParams* prm;
  double ds, dth;
};

constexpr int kRcV = 8;                 // entries per lane of a chunk
constexpr int kRcChunk = 32 * kRcV;     // entries of a chunk at most

// (asynchronous copies: mm_async.cuh)

// A lane's 8 consecutive entries of a shared-memory stage (16-byte vectors).
template <typename T>
__device__ __forceinline__ void lds8(const T* p, T (&v)[kRcV]) {
  constexpr int P = 16 / sizeof(T);
#pragma unroll
  for (int h = 0; h < kRcV / P; ++h) {
    if constexpr (sizeof(T) == 4) {
      const float4 q = reinterpret_cast<const float4*>(p)[h];
      v[4 * h] = q.x; v[4 * h + 1] = q.y; v[4 * h + 2] = q.z; v[4 * h + 3] = q.w;
    } else {
      const double2 q = reinterpret_cast<const double2*>(p)[h];
      v[2 * h] = q.x; v[2 * h + 1] = q.y;
    }
  }
}
template <typename T>
__device__ __forceinline__ void sts8(T* p, const T (&v)[kRcV]) {
  constexpr int P = 16 / sizeof(T);
#pragma unroll
  for (int h = 0; h < kRcV / P; ++h) {
    if constexpr (sizeof(T) == 4)
      reinterpret_cast<float4*>(p)[h] = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
    else
      reinterpret_cast<double2*>(p)[h] = make_double2(v[2 * h], v[2 * h + 1]);
  }
}

// The walking term of Eq. 4 on a lane's 8 consecutive entries of a chunk:
// D = F_{p-1} - F_p with F_p = M_p + sigma_p / 2 (Superbee slope of the
// backward and forward differences), F_p = M_p at a line's last node
// (donor-cell outflow), F_{p-1} = 0 and M_{p-1} = 0 at a line's first node;
// mask bit v: entry v starts a line, bit 8 + v: it ends one. The arithmetic is
// that of the row kernels' walk (walk_dflux), entry by entry; the neighbours
// across lanes come by one shuffle each way.
template <typename T>
__device__ __forceinline__ void rc_walk(const T (&M)[kRcV], unsigned mask, T (&D)[kRcV]) {
  const T ml = __shfl_up_sync(0xffffffffu, M[kRcV - 1], 1);
  const T mr = __shfl_down_sync(0xffffffffu, M[0], 1);
  T F[kRcV];
#pragma unroll
  for (int v = 0; v < kRcV; ++v) {
    const T left = ((mask >> v) & 1u) ? T(0) : (v > 0 ? M[v - 1] : ml);
    const T right = v + 1 < kRcV ? M[v + 1] : mr;
    const T a = M[v] - left, b = right - M[v];
    const T ha = T(0.5) * a, hb = T(0.5) * b;
    const bool last = ((mask >> (8 + v)) & 1u) != 0;
    if constexpr (sizeof(T) == 4) {
      float r = max3_t(min_xorsign_abs(a, hb), min_xorsign_abs(ha, b), 0.0f);
      if (last) r = 0.0f;
      F[v] = M[v] + copysignf(r, b);
    } else {
      F[v] = superbee64(a, ha, b, hb, last, M[v]).F;  // the limiter on the bit patterns
    }
  }
  const T fl = __shfl_up_sync(0xffffffffu, F[kRcV - 1], 1);
#pragma unroll
  for (int v = 0; v < kRcV; ++v) {
    const T fprev = ((mask >> v) & 1u) ? T(0) : (v > 0 ? F[v - 1] : fl);
    D[v] = fprev - F[v];
  }
}

// Alg. 2 per anchor r0 (warp per anchor, grid-strided): the RK2 of Eq. 4 on
// every configuration of B_rc(r0) (Mf(r0) frozen over both stages, binding
// k_on Mf(r0) w), the line sums of Mb ds, C(r0) = sum over lines of
// psi(filament cell, k) (line sum) dtheta with psi = psi_c (psi^{n+1}), the
// scale-down where C exceeds M (the warp rescales the entries and line sums it
// wrote) and Mf = M - C. init = 1: dt = 0 (the set-up: C, the scale-down, Mf
// and the line sums of a loaded state).
// The warp's (anchor, chunk) items stream through a ring of S shared-memory
// stages filled by asynchronous copies S items ahead (coalesced 4/8-byte
// copies: a chunk may start anywhere); lane l computes the chunk's entries
// 8 l .. 8 l + 7, and the new values go back through the stage so that the
// global stores are coalesced too.
#ifndef MM_RC_MIN_BLOCKS
#define MM_RC_MIN_BLOCKS 8
#endif
template <typename T, int S>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? MM_RC_MIN_BLOCKS : 1)
    k_rc_motor(const RcArgs<T> x, const T* psi_c, int init) {
  extern __shared__ __align__(16) unsigned char rc_ring_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = blockIdx.x * 4LL + wib, W = (long long)gridDim.x * 4;
  T* ring = reinterpret_cast<T*>(rc_ring_raw) + (size_t)wib * S * kRcChunk;
  const double dt64 = init ? 0.0 : x.prm->dt;
  const T dt = (T)dt64, hdt = (T)(0.5 * dt64);
  const T cw = (T)x.prm->cw, kon = (T)x.prm->k_on, koff = (T)x.prm->k_off;
  const T c1 = hdt * cw, c2 = T(1) - hdt * koff, e1 = dt * cw, e2 = -dt * koff;
  const T hk = hdt * kon, fk = dt * kon;
  const T ds = (T)x.ds, dth = (T)x.dth;
  const int nx = x.nx, ny = x.ny, nth = x.nth, nch = x.nchunks;
  const long long na = gw < x.ncells ? (x.ncells - gw + W - 1) / W : 0;
  const long long nitems = na * nch;
  auto issue = [&](long long q) {
    if (q < nitems) {
      const long long a = gw + (q / nch) * W;
      const int4 cd = x.chunk[(int)(q % nch)];
      T* st = ring + (size_t)(q % S) * kRcChunk;
      const T* src = x.mb + (size_t)a * x.nconf + cd.x;
#pragma unroll
      for (int v = 0; v < kRcV; ++v) {
        const int p = 32 * v + lane;
        if (p < cd.y) cp_async_t(st + p, src + p);
      }
    }
    cp_async_commit();  // one group per item, empty past the end
  };
#pragma unroll
  for (int q = 0; q < S; ++q) issue(q);
  T cacc = T(0), mfa = T(0);
  for (long long q = 0; q < nitems; ++q) {
    const int ch = (int)(q % nch);
    const long long a = gw + (q / nch) * W;
    if (ch == 0) {
      mfa = x.mf[a];
      cacc = T(0);
    }
    const int4 cd = x.chunk[ch];
    const unsigned mask = x.cmask[ch * 32 + lane];
    T wv[kRcV];
    lds8(x.cw + (size_t)ch * kRcChunk + 8 * lane, wv);  // 16-byte vector loads (global)
    cp_async_wait<S - 1>();
    __syncwarp();
    T* st = ring + (size_t)(q % S) * kRcChunk;
    T M[kRcV], D[kRcV], Ms[kRcV];
    lds8(st + 8 * lane, M);
#pragma unroll
    for (int v = 0; v < kRcV; ++v)
      if (!((mask >> (16 + v)) & 1u)) M[v] = T(0);
    rc_walk<T>(M, mask, D);
    if constexpr (sizeof(T) == 4) {
      // the element-wise stage updates as packed two-value float32 operations
      const float2 c1_ = make_float2(c1, c1), c2_ = make_float2(c2, c2);
      const float2 e1_ = make_float2(e1, e1), e2_ = make_float2(e2, e2);
      const float2 hm = make_float2(hk * mfa, hk * mfa), fm = make_float2(fk * mfa, fk * mfa);
      float2 bh[kRcV / 2], bf[kRcV / 2];
#pragma unroll
      for (int h = 0; h < kRcV / 2; ++h) {
        const float2 w2 = make_float2(wv[2 * h], wv[2 * h + 1]);
        bh[h] = __fmul2_rn(hm, w2);
        bf[h] = __fmul2_rn(fm, w2);
        const float2 r = __ffma2_rn(c1_, make_float2(D[2 * h], D[2 * h + 1]),
                                    __ffma2_rn(c2_, make_float2(M[2 * h], M[2 * h + 1]), bh[h]));
        Ms[2 * h] = r.x;
        Ms[2 * h + 1] = r.y;
      }
      rc_walk<T>(Ms, mask, D);
#pragma unroll
      for (int h = 0; h < kRcV / 2; ++h) {
        const float2 r = __ffma2_rn(
            e1_, make_float2(D[2 * h], D[2 * h + 1]),
            __ffma2_rn(e2_, make_float2(Ms[2 * h], Ms[2 * h + 1]),
                       __fadd2_rn(make_float2(M[2 * h], M[2 * h + 1]), bf[h])));
        M[2 * h] = r.x;
        M[2 * h + 1] = r.y;
      }
    } else {
#pragma unroll
      for (int v = 0; v < kRcV; ++v) Ms[v] = fma_t(c1, D[v], fma_t(c2, M[v], hk * (mfa * wv[v])));
      rc_walk<T>(Ms, mask, D);
#pragma unroll
      for (int v = 0; v < kRcV; ++v)
        M[v] = fma_t(e1, D[v], fma_t(e2, Ms[v], M[v] + fk * (mfa * wv[v])));
    }
    __syncwarp();
    sts8(st + 8 * lane, M);
    __syncwarp();
    T* Ma = x.mb + (size_t)a * x.nconf + cd.x;
    if (!init) {
#pragma unroll
      for (int v = 0; v < kRcV; ++v) {
        const int p = 32 * v + lane;
        if (p < cd.y) Ma[p] = st[p];
      }
    }
    // each lane's running sums of the new values, restarted at every line
    // start, into the stage (entry 8 lane + v): a line's sum is then its last
    // entry's running sum plus the lane-end sums of the lanes it leaves
    {
      T r = T(0);
#pragma unroll
      for (int v = 0; v < kRcV; ++v) {
        r = ((mask >> v) & 1u) ? M[v] : r + M[v];
        M[v] = r;
      }
      __syncwarp();  // every lane has read the stage for the stores above
      sts8(st + 8 * lane, M);
      __syncwarp();
    }
    // lanes over the chunk's lines: the line sum of Mb ds, and the line's
    // part of the coarse density
    const int ay = (int)(a / nx), ax = (int)(a - (long long)ay * nx);
    T* La = x.ls + (size_t)a * x.nlines;
    for (int li = lane; li < cd.w; li += 32) {
      const int l = cd.z + li;
      const int4 ln = x.line[l];
      int fx = ax - ln.x, fy = ay - ln.y;
      fx += fx < 0 ? nx : (fx >= nx ? -nx : 0);
      fy += fy < 0 ? ny : (fy >= ny ? -ny : 0);
      const T pf = psi_c[((size_t)fy * nx + fx) * nth + ln.z];
      const int b0 = x.loff[l] - cd.x, e = b0 + ln.w - 1;
      T s0 = T(0);
      for (int q2 = (b0 >> 3) * 8 + 7; q2 < e; q2 += 8) s0 += st[q2];
      const T s = (s0 + st[e]) * ds;
      La[l] = s;
      cacc = fma_t(pf * s, dth, cacc);
    }
    __syncwarp();
    issue(q + S);
    if (ch == nch - 1) {
      const T C = warp_sum_t(cacc);
      const T Mt = x.mtot[a];
      T Cc = C;
      if (Mt < C) {  // Alg. 2 scale-down at r0 (rare): the warp rescales what it wrote
        const T f = Mt / C;
        T* Mall = x.mb + (size_t)a * x.nconf;
        for (int e = lane; e < x.nconf; e += 32) Mall[e] = __ldcg(Mall + e) * f;
        for (int l = lane; l < x.nlines; l += 32) La[l] = __ldcg(La + l) * f;
        Cc = Mt;
      }
      if (lane == 0) {
        x.c[a] = Cc;
        x.mf[a] = Mt - Cc;
      }
    }
  }
  cp_async_wait<0>();
}

// n_b(x, k) = sum over the lines of orientation k, in template order, of the
// line sum at the anchor r0 = x + (dx, dy) (thread per (x, k)).
template <typename T>
__global__ void k_rc_nb(const RcArgs<T> x, T* nb) {
  const long long n = x.ncells * x.nth;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long cell = t / x.nth;
    const int k = (int)(t - cell * x.nth);
    const int fy = (int)(cell / x.nx), fx = (int)(cell - (long long)fy * x.nx);
    // four loads in flight, added in template order
    T s = T(0);
    const int l1 = x.krange[k + 1];
    int l = x.krange[k];
    auto at = [&](int li) {
      const int4 ln = x.line[li];
      int ax = fx + ln.x, ay = fy + ln.y;
      ax += ax < 0 ? x.nx : (ax >= x.nx ? -x.nx : 0);
      ay += ay < 0 ? x.ny : (ay >= x.ny ? -x.ny : 0);
      return __ldcg(x.ls + ((size_t)ay * x.nx + ax) * x.nlines + li);
    };
    for (; l + 3 < l1; l += 4) {
      const T v0 = at(l), v1 = at(l + 1), v2 = at(l + 2), v3 = at(l + 3);
      s += v0;
      s += v1;
      s += v2;
      s += v3;
    }
    for (; l < l1; ++l) s += at(l);
    nb[t] = s;
  }
}

// Per-node totals over the anchors, NN[x][k][j] = sum over the anchors in
// reach of Mb (the one-anchor row layout: the moments and the force at the
// heads are formed from these rows). Warp per (x, k), lanes over nodes, the
// lines of k in template order.
template <typename T>
__global__ void k_rc_nodes(const RcArgs<T> x, T* nn) {
  const int lane = threadIdx.x & 31;
  const long long n = x.ncells * x.nth;
  for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < n;
       r += (long long)gridDim.x * (blockDim.x >> 5)) {
    const long long cell = r / x.nth;
    const int k = (int)(r - cell * x.nth);
    const int fy = (int)(cell / x.nx), fx = (int)(cell - (long long)fy * x.nx);
    T* row = nn + (size_t)r * x.ns;
    for (int j = lane; j < x.ns; j += 32) row[j] = T(0);
    __syncwarp();
    for (int l = x.krange[k]; l < x.krange[k + 1]; ++l) {
      const int4 ln = x.line[l];
      int ax = fx + ln.x, ay = fy + ln.y;
      ax += ax < 0 ? x.nx : (ax >= x.nx ? -x.nx : 0);
      ay += ay < 0 ? x.ny : (ay >= x.ny ? -x.ny : 0);
      const T* src = x.mb + ((size_t)ay * x.nx + ax) * x.nconf + x.loff[l];
      // the line's first node, from its entry: j0 is kept in the line sums'
      // table as the position of the line within its orientation's nodes
      const int j0 = x.loff[l + x.nlines];
      for (int q = lane; q < ln.w; q += 32) row[j0 + q] += src[q];
      __syncwarp();
    }
  }
}

// psi^{n+1} of every cell by Eq. 1 (warp per cell, lanes over theta), with the
// float32 form's mass sums and correction factor as in the fused substep.
template <typename T, bool MASSCORR>
__global__ void __launch_bounds__(128) k_rc_psi(const StepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char rc_smem[];
  const int nth = a.nth, nx = a.nx, ny = a.ny;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  T* psi5 = reinterpret_cast<T*>(rc_smem) + (size_t)wib * 10 * nth;
  T* nb5 = psi5 + 5 * nth;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  const StepScalars<T> sc = step_scalars<T, MASSCORR>(a.prm, a, lane);
  const PsiConst<T> pq{sc.dt, sc.g, sc.glide, sc.vsp, sc.inv_dx, sc.inv_dy, sc.inv_dth, sc.dth,
                       a.trig};
  const LaneTrig<T> lt = lane_trig(a.trig, nth, lane);
  T mass_hi = T(0), mass_lo = T(0);
  for (int cell = gw; cell < nc; cell += W) {
    const int iy = cell / nx, ix = cell - iy * nx;
    const int xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const int nbr[5] = {cell, iy * nx + xp, iy * nx + xm, yp * nx + ix, ym * nx + ix};
    for (int q = 0; q < 5; ++q)
      for (int k = lane; k < nth; k += 32) {
        psi5[q * nth + k] = a.psi_in[(size_t)nbr[q] * nth + k];
        nb5[q * nth + k] = a.nb_in[(size_t)nbr[q] * nth + k];
      }
    __syncwarp();
    const CellVel<T> uv = load_cell_vel(a.ucell, cell);
    T cell_mass = T(0), unused = T(0);
    psi_cell(pq, uv, psi5, nb5, nb5, nth, lane, a.psi_out + (size_t)cell * nth, cell_mass, unused,
             &lt);
    two_sum_acc(mass_hi, mass_lo, cell_mass);
    __syncwarp();
  }
  // sum psi^{n+1}: per warp, per block, then the last block, in a fixed order
  // (float-float in the float32 form), and the correction factor
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
        const double tot = (double)m2.x + (double)m2.y;
        a.prm->mass = tot;
        if (MASSCORR && a.mass_correct) a.prm->psi_scale = a.prm->mass0 / tot;
      }
    }
  } else {
    const double m = warp_sum_ff(mass_hi, mass_lo);
    if (lane == 0) s_red[wib] = m;
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
      const double tot = warp_sum_ldcg(a.partial, (int)gridDim.x, 1, lane);
      if (lane == 0) {
        a.prm->mass = tot;
        if (MASSCORR && a.mass_correct) a.prm->psi_scale = a.prm->mass0 / tot;
      }
    }
  }
}

}  // namespace mm

using namespace mmh;

namespace {

struct RcLine {
  int k, dx, dy, j0, len, off;
};

// The capture template (the same rule and order as the definition above):
// head of node j of orientation k at (hx, hy) cells from the filament cell's
// lower-left corner; the cell at offset (ex, ey) is in reach when the gap from
// the head to its square, in physical units, has squared length at most rc^2.
// Every value here decides integers, so it is evaluated by plain products,
// quotients, sums and comparisons in float64 without fused operations (the
// library's host code is compiled with contraction off).
mm_status rc_build(mm_handle* h, double rc, std::vector<RcLine>& L, int& nconf,
                   std::vector<double>& w) {
  const int nth = h->g.ntheta, ns = h->g.ns, nx = h->g.nx, ny = h->g.ny;
  const double dx = 1.0 / nx, dy = 1.0 / ny, dth = 2.0 * kPi / nth, rc2 = rc * rc;
  std::vector<double> hx(ns), hy(ns);
  std::vector<int> cnt(ns);
  w.assign((size_t)nth * ns, 0.0);
  L.clear();
  int minx = 0, maxx = 0, miny = 0, maxy = 0;
  auto reach = [&](int j, int ex, int ey) {
    const double gx = std::max(std::max((double)ex - hx[j], hx[j] - (double)(ex + 1)), 0.0);
    const double gy = std::max(std::max((double)ey - hy[j], hy[j] - (double)(ey + 1)), 0.0);
    const double px = gx * dx, py = gy * dy;
    const double px2 = px * px, py2 = py * py;
    return px2 + py2 <= rc2;
  };
  for (int k = 0; k < nth; ++k) {
    const double th = k * dth, ct = std::cos(th), st = std::sin(th);
    double lox = 1e300, hix = -1e300, loy = 1e300, hiy = -1e300;
    for (int j = 0; j < ns; ++j) {
      const double disp = h->r.ell * h->g.L * (double)(2 * j + 1 - ns) / (2.0 * ns);
      hx[j] = disp * ct / dx + 0.5;
      hy[j] = disp * st / dy + 0.5;
      lox = std::min(lox, hx[j]);
      hix = std::max(hix, hx[j]);
      loy = std::min(loy, hy[j]);
      hiy = std::max(hiy, hy[j]);
    }
    const double bx0 = std::floor(lox - rc / dx) - 1, bx1 = std::floor(hix + rc / dx) + 1;
    const double by0 = std::floor(loy - rc / dy) - 1, by1 = std::floor(hiy + rc / dy) + 1;
    if (!(bx1 - bx0 < 4.0 * nx + 8 && by1 - by0 < 4.0 * ny + 8))
      return fail(h, MM_ERR_UNSUPPORTED, "the reach of the heads spans the periodic grid");
    const size_t first = L.size();
    for (int ey = (int)by0; ey <= (int)by1; ++ey)
      for (int ex = (int)bx0; ex <= (int)bx1; ++ex) {
        int j = 0;
        while (j < ns) {
          if (!reach(j, ex, ey)) {
            ++j;
            continue;
          }
          const int j0 = j;
          while (j < ns && reach(j, ex, ey)) ++j;
          L.push_back(RcLine{k, ex, ey, j0, j - j0, 0});
          minx = std::min(minx, ex);
          maxx = std::max(maxx, ex);
          miny = std::min(miny, ey);
          maxy = std::max(maxy, ey);
        }
      }
    std::sort(L.begin() + first, L.end(), [](const RcLine& a, const RcLine& b) {
      if (a.j0 != b.j0) return a.j0 < b.j0;
      if (a.dy != b.dy) return a.dy < b.dy;
      return a.dx < b.dx;
    });
    std::fill(cnt.begin(), cnt.end(), 0);
    for (size_t l = first; l < L.size(); ++l)
      for (int j = L[l].j0; j < L[l].j0 + L[l].len; ++j) ++cnt[j];
    for (int j = 0; j < ns; ++j) w[(size_t)k * ns + j] = 1.0 / cnt[j];
  }
  if (maxx - minx >= nx || maxy - miny >= ny)
    return fail(h, MM_ERR_UNSUPPORTED,
                "the reach of the heads spans the periodic grid (two offsets name one cell)");
  long long off = 0;
  for (RcLine& l : L) {
    l.off = (int)off;
    off += l.len;
  }
  if (off > (1LL << 30)) return fail(h, MM_ERR_UNSUPPORTED, "too many configurations per anchor");
  nconf = (int)off;
  return MM_OK;
}

template <typename T>
mm::RcArgs<T> rc_args(mm_handle* h) {
  mm::RcArgs<T> x;
  x.nx = h->g.nx;
  x.ny = h->g.ny;
  x.nth = h->g.ntheta;
  x.ns = h->g.ns;
  x.nconf = h->rc_nconf;
  x.nlines = h->rc_nlines;
  x.nchunks = h->rc_nchunks;
  x.ncells = h->ncells;
  x.mb = (T*)h->rc_mb;
  x.ls = (T*)h->rc_ls;
  x.line = (const int4*)h->rc_tab;
  x.loff = (const int*)((const char*)h->rc_tab + h->rc_tab_off[0]);
  x.chunk = (const int4*)((const char*)h->rc_tab + h->rc_tab_off[1]);
  x.meta = (const unsigned char*)h->rc_tab + h->rc_tab_off[2];
  x.w = (const T*)((const char*)h->rc_tab + h->rc_tab_off[3]);
  x.krange = (const int*)((const char*)h->rc_tab + h->rc_tab_off[4]);
  x.cmask = (const unsigned*)((const char*)h->rc_tab + h->rc_tab_off[5]);
  x.cw = (const T*)((const char*)h->rc_tab + h->rc_tab_off[6]);
  x.mtot = (const T*)h->mtot;
  x.mf = (T*)h->mf;
  x.c = (T*)h->c;
  x.prm = h->prm;
  x.ds = h->g.L / h->g.ns;
  x.dth = 2.0 * kPi / h->g.ntheta;
  return x;
}

// Ring stages of the motor kernel per warp, and its dynamic shared memory.
constexpr int kRcStages = 4;
template <typename T>
constexpr size_t rc_ring_bytes() {
  return (size_t)4 * kRcStages * mm::kRcChunk * sizeof(T);
}

int rc_grid(mm_handle* h, long long work, int per_block) {
  long long b = (work + per_block - 1) / per_block;
  return (int)std::max<long long>(1, std::min<long long>(b, 16LL * h->sms));
}

template <typename T>
cudaError_t rc_substep_t(mm_handle* h, int parity, cudaStream_t s) {
  const StepArgs<T> a = step_args<T>(h, parity);
  const size_t smem = 4 * 10 * (size_t)h->g.ntheta * sizeof(T);
  const int gp = std::min(rc_grid(h, h->ncells, 4), h->npartial);  // a partial sum per block
  if (a.mass_correct)
    mm::k_rc_psi<T, true><<<gp, 128, smem, s>>>(a);
  else
    mm::k_rc_psi<T, false><<<gp, 128, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const mm::RcArgs<T> x = rc_args<T>(h);
  mm::k_rc_motor<T, kRcStages><<<h->rc_motor_grid, 128, rc_ring_bytes<T>(), s>>>(
      x, (const T*)h->psi[parity ^ 1], 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mm::k_rc_nb<T><<<rc_grid(h, h->ncells * h->g.ntheta, 256), 256, 0, s>>>(x, (T*)h->nb[parity ^ 1]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t rc_init_t(mm_handle* h) {
  const mm::RcArgs<T> x = rc_args<T>(h);
  mm::k_rc_motor<T, kRcStages><<<h->rc_motor_grid, 128, rc_ring_bytes<T>(), h->stream>>>(
      x, (const T*)h->psi[h->parity], 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mm::k_rc_nb<T><<<rc_grid(h, h->ncells * h->g.ntheta, 256), 256, 0, h->stream>>>(
      x, (T*)h->nb[h->parity]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t rc_nodes_t(mm_handle* h) {
  const mm::RcArgs<T> x = rc_args<T>(h);
  mm::k_rc_nodes<T><<<rc_grid(h, h->ncells * h->g.ntheta, 4), 128, 0, h->stream>>>(x, (T*)h->mb);
  return cudaGetLastError();
}

}  // namespace

namespace mmh {

void capture_free(mm_handle* h) {
  void* p[3] = {h->rc_mb, h->rc_ls, h->rc_tab};
  for (void* q : p)
    if (q) cudaFree(q);
  h->rc_mb = h->rc_ls = h->rc_tab = nullptr;
  h->capture = false;
}

cudaError_t launch_capture_substep(mm_handle* h, int parity, cudaStream_t s) {
  return h->prec == MM_FP64 ? rc_substep_t<double>(h, parity, s) : rc_substep_t<float>(h, parity, s);
}

// State set-up: C at every anchor, the scale-down, Mf, the line sums, n_b.
mm_status run_init_capture(mm_handle* h) {
  CK(h->prec == MM_FP64 ? rc_init_t<double>(h) : rc_init_t<float>(h));
  return MM_OK;
}

// The per-node totals over the anchors into h->mb (the one-anchor row layout)
// for the moments kernel and the force at the heads.
mm_status capture_rows(mm_handle* h) {
  CK(h->prec == MM_FP64 ? rc_nodes_t<double>(h) : rc_nodes_t<float>(h));
  return MM_OK;
}

}  // namespace mmh

extern "C" {

mm_status mm_set_capture(mm_handle* h, double rc) {
  MM_TRACE("mm_set_capture");
  if (!h) return MM_ERR_INVALID;
  if (h->batch || h->owner)
    return fail(h, MM_ERR_UNSUPPORTED, "a capture radius is not available in a batch");
  if (h->rec.active)
    return fail(h, MM_ERR_STATE, "the capture radius is not differentiated: end the adjoint recording first");
  if (h->anchors)
    return fail(h, MM_ERR_STATE, "non-local anchors are on: switch them off (mm_set_anchors) first");
  if (h->tangent && rc >= 0.0)
    return fail(h, MM_ERR_STATE, "the tangent mode is on: switch it off (mm_set_tangent) first");
  if (std::isnan(rc) || std::isinf(rc))
    return fail(h, MM_ERR_INVALID, "the capture radius must be finite (negative: off)");
  DeviceGuard dg(h->device);
  mm_status st;
  // everything that can refuse runs before the current state is touched
  std::vector<RcLine> L;
  std::vector<double> w;
  int nconf = 0;
  if (rc >= 0.0) {
    if (h->g.ns > mm::kRcChunk)
      return fail(h, MM_ERR_UNSUPPORTED, "a capture radius needs ns <= 256");
    if (40 * (size_t)h->g.ntheta * h->tsz > 48 * 1024)  // the psi kernel's staged columns
      return fail(h, MM_ERR_UNSUPPORTED, "a capture radius needs ntheta * 40 * value size <= 48 KB");
    if ((st = rc_build(h, rc, L, nconf, w)) != MM_OK) return st;
  }
  CK(cudaStreamSynchronize(h->stream));
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  const bool was_on = h->capture;
  const size_t held = was_on ? (size_t)h->ncells * ((size_t)h->rc_nconf + h->rc_nlines) * h->tsz : 0;
  if (rc < 0.0) {
    // back to the one-anchor models: the motor state is discarded (the plain
    // Mb held the per-node totals of the moments meanwhile)
    capture_free(h);
    CK(cudaMemsetAsync(h->mb, 0, h->mbn * h->tsz, h->stream));
    if (h->have_state) return run_init(h);
    return MM_OK;
  }
  const int nl = (int)L.size(), nth = h->g.ntheta, ns = h->g.ns;
  // chunks: consecutive whole lines, at most kRcChunk entries
  std::vector<int4> chunks;
  {
    int l = 0;
    while (l < nl) {
      const int l0 = l, pos0 = L[l].off;
      int npos = 0;
      while (l < nl && npos + L[l].len <= mm::kRcChunk) npos += L[l++].len;
      chunks.push_back(make_int4(pos0, npos, l0, l - l0));
    }
  }
  std::vector<int4> lines(nl);
  std::vector<int> loff(2 * (size_t)nl);  // first entry of each line, then its first node
  std::vector<unsigned char> meta(nconf);
  std::vector<int> krange(nth + 1, nl);
  for (int l = nl - 1; l >= 0; --l) krange[L[l].k] = l;
  for (int k = nth - 1; k >= 0; --k) krange[k] = std::min(krange[k], krange[k + 1]);
  std::vector<double> wpos(nconf);
  for (int l = 0; l < nl; ++l) {
    lines[l] = make_int4(L[l].dx, L[l].dy, L[l].k, L[l].len);
    loff[l] = L[l].off;
    loff[nl + l] = L[l].j0;
    for (int q = 0; q < L[l].len; ++q) {
      meta[L[l].off + q] = (unsigned char)((q == 0 ? 1 : 0) | (q == L[l].len - 1 ? 2 : 0));
      wpos[L[l].off + q] = w[(size_t)L[l].k * ns + L[l].j0 + q];
    }
  }
  // one device block for the tables, 256-byte aligned pieces
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t t = h->tsz, nc = (size_t)h->ncells;
  size_t o = up(nl * sizeof(int4));
  h->rc_tab_off[0] = o;
  o += up(2 * (size_t)nl * sizeof(int));
  h->rc_tab_off[1] = o;
  o += up(chunks.size() * sizeof(int4));
  h->rc_tab_off[2] = o;
  o += up((size_t)nconf);
  h->rc_tab_off[3] = o;
  o += up((size_t)nconf * t);
  h->rc_tab_off[4] = o;
  o += up((nth + 1) * sizeof(int));
  h->rc_tab_off[5] = o;
  o += up(chunks.size() * 32 * sizeof(unsigned));
  h->rc_tab_off[6] = o;
  o += up(chunks.size() * mm::kRcChunk * t);
  const size_t tab_bytes = o;
  const size_t need = nc * nconf * t + nc * nl * t + tab_bytes;
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  if (need + (64u << 20) > freeb + held)
    return fail(h, MM_ERR_OOM, "the capture-radius state does not fit");
  capture_free(h);
  // the head cells' offsets (the force of Eq. 10 at the heads), as for the
  // one-anchor model
  if (!h->anc_off && (st = anchor_alloc(h)) != MM_OK) return st;
  if ((st = anchor_table(h)) != MM_OK) return st;
  CK(cudaMalloc(&h->rc_mb, nc * nconf * t));
  CK(cudaMalloc(&h->rc_ls, std::max<size_t>(nc * nl * t, 16)));
  CK(cudaMalloc(&h->rc_tab, tab_bytes));
  std::vector<unsigned char> host(tab_bytes, 0);
  memcpy(host.data(), lines.data(), nl * sizeof(int4));
  memcpy(host.data() + h->rc_tab_off[0], loff.data(), loff.size() * sizeof(int));
  memcpy(host.data() + h->rc_tab_off[1], chunks.data(), chunks.size() * sizeof(int4));
  memcpy(host.data() + h->rc_tab_off[2], meta.data(), meta.size());
  if (h->prec == MM_FP64) {
    memcpy(host.data() + h->rc_tab_off[3], wpos.data(), (size_t)nconf * 8);
  } else {
    std::vector<float> wf(wpos.begin(), wpos.end());
    memcpy(host.data() + h->rc_tab_off[3], wf.data(), (size_t)nconf * 4);
  }
  memcpy(host.data() + h->rc_tab_off[4], krange.data(), (nth + 1) * sizeof(int));
  // per chunk and lane: the flags of the lane's 8 entries (entry 8 lane + v),
  // and the chunk's weights in the same order (0 past the chunk's end)
  {
    std::vector<unsigned> cmask(chunks.size() * 32, 0u);
    std::vector<double> cwd(chunks.size() * mm::kRcChunk, 0.0);
    for (size_t c = 0; c < chunks.size(); ++c)
      for (int lane = 0; lane < 32; ++lane) {
        unsigned m = 0;
        for (int v = 0; v < mm::kRcV; ++v) {
          const int pch = mm::kRcV * lane + v;
          if (pch < chunks[c].y) {
            const int e = chunks[c].x + pch;
            m |= (meta[e] & 1u) << v;
            m |= ((meta[e] >> 1) & 1u) << (8 + v);
            m |= 1u << (16 + v);
            cwd[c * mm::kRcChunk + pch] = wpos[e];
          } else {
            m |= (1u << v) | (1u << (8 + v));  // an isolated empty entry
          }
        }
        cmask[c * 32 + lane] = m;
      }
    memcpy(host.data() + h->rc_tab_off[5], cmask.data(), cmask.size() * sizeof(unsigned));
    if (h->prec == MM_FP64) {
      memcpy(host.data() + h->rc_tab_off[6], cwd.data(), cwd.size() * 8);
    } else {
      std::vector<float> cwf(cwd.begin(), cwd.end());
      memcpy(host.data() + h->rc_tab_off[6], cwf.data(), cwf.size() * 4);
    }
  }
  CK(cudaMemcpy(h->rc_tab, host.data(), tab_bytes, cudaMemcpyHostToDevice));
  CK(cudaMemset(h->rc_mb, 0, nc * nconf * t));
  h->rc = rc;
  h->rc_nconf = nconf;
  h->rc_nlines = nl;
  h->rc_nchunks = (int)chunks.size();
  h->rc_host_lines.assign(6 * (size_t)nl, 0);
  for (int l = 0; l < nl; ++l) {
    int* q = h->rc_host_lines.data() + 6 * (size_t)l;
    q[0] = L[l].k;
    q[1] = L[l].dx;
    q[2] = L[l].dy;
    q[3] = L[l].j0;
    q[4] = L[l].len;
    q[5] = L[l].off;
  }
  h->rc_host_w = w;
  int per_sm = 0;
  CK(h->prec == MM_FP64
         ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &per_sm, mm::k_rc_motor<double, kRcStages>, 128, rc_ring_bytes<double>())
         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &per_sm, mm::k_rc_motor<float, kRcStages>, 128, rc_ring_bytes<float>()));
  h->rc_motor_grid = (int)std::max<long long>(
      1, std::min<long long>((h->ncells + 3) / 4, (long long)std::max(per_sm, 1) * h->sms));
  h->capture = true;
  // a new layout: the motors are discarded (Mb = 0, Mf = M); psi is kept
  if (h->have_state) return run_init_capture(h);
  return MM_OK;
}

mm_status mm_capture_template(mm_handle* h, int* lines, int max_lines, int* nlines, int* nconf,
                              double* w) {
  if (!h || !nlines || !nconf) return MM_ERR_INVALID;
  if (!h->capture) return fail(h, MM_ERR_STATE, "no capture radius is set (mm_set_capture)");
  *nlines = h->rc_nlines;
  *nconf = h->rc_nconf;
  if (lines && max_lines >= h->rc_nlines)
    memcpy(lines, h->rc_host_lines.data(), h->rc_host_lines.size() * sizeof(int));
  if (w) memcpy(w, h->rc_host_w.data(), h->rc_host_w.size() * sizeof(double));
  return MM_OK;
}

}  // extern "C"
