// Non-local motor anchors (mm_set_anchors): every bound-motor configuration
// (cell i, theta_k, s_j) is anchored in the cell under its motor head,
// x_i + (l/L) s_j p_k -- Eq. 4-6 and Eq. 10 with the anchor r0 kept and the
// capture radius of Eq. 4 taken to zero. Binding at a node takes the free
// motors of its anchor (a gather), and the coarse density of Eq. 5, the Alg. 2
// scale-down, Eq. 6 and the motor force of Eq. 10 are formed per anchor (a
// scatter). One substep is three launches:
//   k_substep_anchor  warp per cell: psi by Eq. 1 first (its new values weight
//                     the scatter), then every s-row by the RK2 of Eq. 4 with
//                     the per-node binding term, n_b of the row, and the row's
//                     contributions psi ds dtheta Mb added into the anchors'
//                     float64 accumulators (runs of nodes with the same anchor
//                     summed in registers first; with a block window each
//                     warp sums its cell's run sums per window entry and the
//                     block adds its 4 cells' sums, one atomic per entry; else
//                     one atomic per run);
//   k_anchor_close    thread per anchor: C, the scale-down factor f, Mf = M - C,
//                     accumulator reset; a flag if any anchor scaled down;
//   k_anchor_fix      only where the flag is set (the scale-down is rare):
//                     scales every node by its anchor's f and recomputes n_b.
// The paper spreads the force to nearby anchors with atomics in the final
// reduction only (Sec. 2); here the coarse density and the force are
// accumulated that way, in float64. Atomic order makes the last bits of C
// depend on the schedule.
#include <algorithm>
#include <utility>

#include "mm_async.cuh"
#include "mm_cell.cuh"
#include "mm_host.h"

// Resident 4-warp blocks per SM the anchor substep's registers are sized for
// (more blocks force spills and measured slower).
#ifndef MM_ANCHOR_MIN_BLOCKS
#define MM_ANCHOR_MIN_BLOCKS 4
#endif

namespace mm {

// Anchor data of one instance: offsets [nth][ns] (reduced into [0, nx) and
// [0, ny)), float64 accumulators and scale-down factors per cell, flags.
template <typename T>
struct AnchorArgs {
  const int2* off;
  double* cacc;  // [cells] sum of psi Mb ds dth anchored in each cell (reset after use)
  double* fsc;   // [cells] scale-down factor of each anchor cell
  int* flags;    // [3]: 0, 1 alternate with the substep parity; 2 for the set-up
  int flag;      // the flag this launch sets or reads
  // The window of anchor cells around a filament cell: offsets wox..wox+wx-1,
  // woy..woy+wy-1; widx [nth][ns] is each node's index in it (wx * wy entries).
  const int* widx;
  int wox, woy, wx, wy;
  // [nth][ns / V]: per orientation and lane slot, bits 0-7: bit v set where
  // the slot's node v is the last of a run of nodes with one anchor (the same
  // in every cell: the anchors' offsets depend on (k, j) only)
  const unsigned* runend;
  // The block-window form: the block's 4 warps take 4 consecutive cells of a
  // row and share one window of wx + 3 columns; went [nth][ns] is each node's
  // entry in it for the group's first cell (cell c of the group adds c). A
  // cell's nsr slot runs (runs of a lane slot's nodes with one anchor) are
  // ordered by window entry, the same order in every cell: wpos [nth][ns] is
  // the place of each node's slot run in it. Each warp stores its cell's run
  // sums in that order (nsrp = 32 ch places, zeros past nsr) and sums them per
  // entry: lane l takes places l ch .. l ch + ch - 1; sgbits [nw][32] marks
  // the places that end an entry's sums and sgrank [32] counts such ends
  // before a lane's first place (nkeys in all). m4 [(wx + 3) wy] gives, per
  // entry of the block's window, the index of its sum among each of the 4
  // cells' per-entry sums (0xffff: none).
  const unsigned short* went;
  const unsigned short* wpos;
  const unsigned* sgbits;
  const unsigned* sgrank;
  const uint2* m4;
  int nsr, nsrp, ch, nw, nkeys;
};

__device__ __forceinline__ int anchor_cell(int ix, int iy, int2 o, int nx, int ny) {
  int ax = ix + o.x, ay = iy + o.y;
  if (ax >= nx) ax -= nx;
  if (ay >= ny) ay -= ny;
  return ay * nx + ax;
}

// V 16-bit table values of a lane slot, two to a 32-bit word.
template <int V>
struct U16Pack {
  unsigned w[(V + 1) / 2];
};
template <int V>
__device__ __forceinline__ U16Pack<V> ld_u16(const unsigned short* p) {
  U16Pack<V> r;
  if constexpr (V == 8) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    r.w[0] = q.x, r.w[1] = q.y, r.w[2] = q.z, r.w[3] = q.w;
  } else if constexpr (V == 4) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    r.w[0] = q.x, r.w[1] = q.y;
  } else if constexpr (V == 2) {
    r.w[0] = __ldg(reinterpret_cast<const unsigned*>(p));
  } else {
    r.w[0] = __ldg(p);
  }
  return r;
}
template <int V>
__device__ __forceinline__ unsigned u16_at(const U16Pack<V>& p, int v) {
  return (v & 1) ? p.w[v >> 1] >> 16 : p.w[v >> 1] & 0xffffu;
}

// A lane's V values of the motor density, loaded and stored with the streaming
// (evict-first) cache policy: the density is read and written once per
// substep, and the anchor tables the kernel re-reads for every cell stay in L1.
template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ld_stream(const T* p) {
  Pack<T, V> r;
  if constexpr (sizeof(T) == 4 && V % 4 == 0) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i) {
      const float4 f = __ldcs(reinterpret_cast<const float4*>(p) + i);
      r.v[4 * i] = f.x, r.v[4 * i + 1] = f.y, r.v[4 * i + 2] = f.z, r.v[4 * i + 3] = f.w;
    }
  } else if constexpr (sizeof(T) == 8 && V == 2) {
    const double2 d = __ldcs(reinterpret_cast<const double2*>(p));
    r.v[0] = d.x, r.v[1] = d.y;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) r.v[v] = __ldcs(p + v);
  }
  return r;
}
template <typename T, int V>
__device__ __forceinline__ void st_stream(T* p, const T (&M)[V]) {
  if constexpr (sizeof(T) == 4 && V % 4 == 0) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i)
      __stcs(reinterpret_cast<float4*>(p) + i,
             make_float4(M[4 * i], M[4 * i + 1], M[4 * i + 2], M[4 * i + 3]));
  } else if constexpr (sizeof(T) == 8 && V == 2) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(M[0], M[1]));
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) __stcs(p + v, M[v]);
  }
}

// Adds w M[v] of the lane's nodes into the accumulators of their anchors: a
// run of consecutive nodes with the same anchor is summed first.
template <typename T, int V>
__device__ __forceinline__ void scatter_runs(double* acc, const int (&anc)[V], const T (&M)[V],
                                             T w) {
  int cur = anc[0];
  T s = w * M[0];
#pragma unroll
  for (int v = 1; v < V; ++v) {
    if (anc[v] == cur) {
      s += w * M[v];
    } else {
      atomicAdd(acc + cur, (double)s);
      cur = anc[v];
      s = w * M[v];
    }
  }
  atomicAdd(acc + cur, (double)s);
}

// The same driven by the run-end mask of the lane's slot: one shared atomic
// per run, no comparison of anchors.
template <typename T, int V>
__device__ __forceinline__ void scatter_runs_mask(T* acc, const int (&widx)[V], const T (&M)[V],
                                                  T w, unsigned ends) {
  T s = T(0);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    s = fma_t(w, M[v], s);
    if ((ends >> v) & 1u) {
      atomicAdd(acc + widx[v], s);
      s = T(0);
    }
  }
}

// Per-warp shared memory: psi and n_b columns of the cell and its four
// neighbours ([5][nth] each) and psi^{n+1} of the cell.
__host__ __device__ inline size_t anchor_warp_smem(int nth, int tsz, int W = 0) {
  const size_t cols = ((size_t)11 * nth * tsz + 15) & ~(size_t)15;
  // the window: Mf and the coarse-density accumulator (state precision) and
  // the global cell of every entry
  return cols + (((size_t)W * (2 * tsz + 4) + 15) & ~(size_t)15);
}

// WIN: the anchors of a cell's nodes lie in a small window of cells around it;
// the window's free motors are gathered into shared memory when the cell
// starts and the rows' contributions to C are summed there (shared-memory
// atomics), then added to the global accumulators once per window entry.
// BW (with WIN): the block's 4 warps take 4 consecutive cells of one row and
// share one window of wx + 3 columns. Each warp stores its cell's slot-run sums
// ordered by window entry, sums them per entry right after its rows (lanes
// take equal runs of places; an entry's sum that spans lanes is completed by a
// segmented scan over the lanes), and after a block barrier the block adds
// the 4 cells' per-entry sums of each window entry and issues one float64
// atomic per entry (no shared atomics: those retried under contention at the
// window centre, where the middle nodes of every orientation land). The next
// group's window is copied in while that sum runs.
template <typename T, int V, bool MASSCORR, bool WIN, bool BW = false>
__global__ void __launch_bounds__(128, MM_ANCHOR_MIN_BLOCKS) k_substep_anchor(const StepArgs<T> a, const AnchorArgs<T> x) {
  extern __shared__ __align__(16) unsigned char asm_raw[];
  const int nth = a.nth, ns = a.ns, seg = a.seg, nx = a.nx, ny = a.ny;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int Wn = WIN ? (BW ? (x.wx + 3) * x.wy : x.wx * x.wy) : 0;
  unsigned char* wbase =
      asm_raw + (size_t)wib * anchor_warp_smem(nth, sizeof(T), BW ? 0 : Wn);
  T* psi5 = reinterpret_cast<T*>(wbase);
  T* nb5 = psi5 + 5 * nth;
  T* pnew = nb5 + 5 * nth;
  // the window: per warp after its columns, or (BW) one for the block after
  // the 4 warps' columns
  unsigned char* winbase =
      BW ? asm_raw + 4 * anchor_warp_smem(nth, sizeof(T), 0)
         : wbase + (((size_t)11 * nth * sizeof(T) + 15) & ~(size_t)15);
  T* wmf = reinterpret_cast<T*>(winbase);
  T* wacc = wmf + Wn;                                   // WIN: the window's sums
  int* wcell = reinterpret_cast<int*>(wacc + Wn);       // WIN: the window's cells
  // BW: after the window's free motors, the 4 warps' ordered run sums [nsrp]
  // and then their per-entry sums [nkeys]
  T* rb0 = reinterpret_cast<T*>(winbase + (((size_t)Wn * sizeof(T) + 15) & ~(size_t)15));
  T* rbw = rb0 + (size_t)wib * x.nsrp;
  T* sw0 = rb0 + 4 * (size_t)x.nsrp;
  T* sw = sw0 + (size_t)wib * x.nkeys;
  if (BW)  // the places past nsr stay zero (no run is stored there)
    for (int p = x.nsr + lane; p < x.nsrp; p += 32) rbw[p] = T(0);
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  const int W = gridDim.x * (blockDim.x >> 5);
  const int nc = (int)a.ncells;
  // the flag of the other parity was read by the previous substep's fix-up:
  // clear it for the next substep
  if (blockIdx.x == 0 && threadIdx.x == 0) x.flags[x.flag ^ 1] = 0;
  const StepScalars<T> sc = step_scalars<T, MASSCORR>(a.prm, a, lane);
  const PsiConst<T> pq{sc.dt, sc.g, sc.glide, sc.vsp, sc.inv_dx, sc.inv_dy, sc.inv_dth, sc.dth,
                       a.trig};
  const T c1 = sc.hdt * sc.cw, c2 = T(1) - sc.hdt * sc.koff, e1 = sc.dt * sc.cw, e2 = -sc.dt * sc.koff;
  const T hk = sc.hdt * sc.kon, fk = sc.dt * sc.kon;
  const T dsdth = sc.ds * sc.dth;
  const LaneGeom lg = lane_geom(lane, seg, ns, V);
  const LaneTrig<T> lt = lane_trig(a.trig, nth, lane);
  T mass_hi = T(0), mass_lo = T(0);
  // BW: block-strided groups of 4 consecutive cells (nx is a multiple of 4,
  // so the 4 warps of a block run the same iterations and all reach the block
  // barriers); else warp-strided cells
  const int cstart = BW ? (int)blockIdx.x * 4 + wib : gw;
  const int cstep = BW ? (int)gridDim.x * 4 : W;
  // The psi and n_b columns of a cell and its four neighbours into psi5 / nb5
  // by asynchronous copies (16 bytes each where a column is a whole number of
  // 16-byte pieces), one group: a cell's columns are issued as soon as the
  // previous cell's psi transport has read the buffer, and land while that
  // cell's rows are computed.
  auto stage_cols = [&](int c) {
    const int cy = c / nx, cx = c - cy * nx;
    const int xp = cx + 1 == nx ? 0 : cx + 1, xm = cx == 0 ? nx - 1 : cx - 1;
    const int yp = cy + 1 == ny ? 0 : cy + 1, ym = cy == 0 ? ny - 1 : cy - 1;
    // (a select chain: a dynamically indexed array would live in local memory)
    auto nbr = [&](int q) {
      return q == 0 ? c : q == 1 ? cy * nx + xp : q == 2 ? cy * nx + xm : q == 3 ? yp * nx + cx
                                                                                  : ym * nx + cx;
    };
    if ((nth * sizeof(T)) % 16 == 0) {
      constexpr int P = 16 / sizeof(T);  // values per piece
      const int per = nth / P;           // pieces per column
      for (int i = lane; i < 10 * per; i += 32) {
        const int col = i / per, p = i - col * per, q = col >> 1;
        const T* src = ((col & 1) ? a.nb_in : a.psi_in) + (size_t)nbr(q) * nth + p * P;
        T* dst = ((col & 1) ? nb5 : psi5) + (size_t)q * nth + p * P;
        cp_async16(dst, src);
      }
    } else {
      for (int i = lane; i < 10 * nth; i += 32) {
        const int col = i / nth, k = i - col * nth, q = col >> 1;
        if (col & 1)
          cp_async_t(nb5 + (size_t)q * nth + k, a.nb_in + (size_t)nbr(q) * nth + k);
        else
          cp_async_t(psi5 + (size_t)q * nth + k, a.psi_in + (size_t)nbr(q) * nth + k);
      }
    }
    cp_async_commit();
  };
  // BW: the window of the group whose first cell is c0, copied asynchronously
  // (the block waits for it with the next cell's columns); entries run over
  // the window row-major, the block's threads striding by 128 (the window is
  // no wider than the grid, so one wrap of each coordinate suffices)
  const int wxb = x.wx + 3;
  const int wdq = BW ? (int)blockDim.x / wxb : 0, wdr = BW ? (int)blockDim.x - wdq * wxb : 0;
  auto wrap = [](int g, int n) { return g < 0 ? g + n : g >= n ? g - n : g; };
  auto fill_window = [&](int c0) {
    const int iy0 = c0 / nx, ix0 = c0 - iy0 * nx;
    int wyi = (int)threadIdx.x / wxb, wxi = (int)threadIdx.x - wyi * wxb;
    for (int w = threadIdx.x; w < Wn; w += blockDim.x) {
      const int gc = wrap(iy0 + x.woy + wyi, ny) * nx + wrap(ix0 + x.wox + wxi, nx);
      cp_async_t(wmf + w, a.mf_in + gc);
      wxi += wdr;
      wyi += wdq;
      if (wxi >= wxb) wxi -= wxb, ++wyi;
    }
    cp_async_commit();
  };
  if (BW && cstart < nc) fill_window(cstart - wib);
  if (cstart < nc) stage_cols(cstart);
  // the next pass's motor density and table values (loaded while the current
  // pass is computed; the first pass of a warp's next cell while its last
  // cell's sums are formed)
  Pack<T, V> qn;
  Pack<int, V> wn;          // WIN: window entries
  U16Pack<V> wen, wps;      // BW: window entries and run places
  unsigned en = 0;          // the slot's run ends
  auto load_pass = [&](int cl, int r0) {
    const int k = r0 + lg.rslot;
    if (k < nth && lg.lane_ok) {
      qn = ld_stream<T, V>(a.mb_in + ((size_t)cl * nth + k) * ns + lg.sl * V);
      if (BW) {
        wen = ld_u16<V>(x.went + (size_t)k * ns + lg.sl * V);
        wps = ld_u16<V>(x.wpos + (size_t)k * ns + lg.sl * V);
      } else if (WIN) {
        wn = *reinterpret_cast<const Pack<int, V>*>(x.widx + (size_t)k * ns + lg.sl * V);
      }
      if (WIN) en = x.runend[(size_t)k * (ns / V) + lg.sl];
    }
  };
  if (cstart < nc) load_pass(cstart, 0);
  for (int cell = cstart; cell < nc; cell += cstep) {
    const int iy = cell / nx, ix = cell - iy * nx;
    if (WIN && !BW) {
      for (int w = lane; w < Wn; w += 32) {
        const int wyi = w / x.wx, wxi = w - wyi * x.wx;
        int gx = (ix + x.wox + wxi) % nx, gy = (iy + x.woy + wyi) % ny;
        if (gx < 0) gx += nx;
        if (gy < 0) gy += ny;
        const int gc = gy * nx + gx;
        wcell[w] = gc;
        wmf[w] = a.mf_in[gc];
        wacc[w] = T(0);
      }
    }
    // Eq. 1 first: psi^{n+1} of the cell weights the scatter of its rows
    const CellVel<T> uv = load_cell_vel(a.ucell, cell);
    cp_async_wait<0>();  // this cell's columns (BW: and the group's window)
    if (BW)
      __syncthreads();
    else
      __syncwarp();
    T cell_mass = T(0), unused = T(0);
    psi_cell(pq, uv, psi5, nb5, nb5, nth, lane, pnew, cell_mass, unused, &lt);
    two_sum_acc(mass_hi, mass_lo, cell_mass);
    __syncwarp();
    if (cell + cstep < nc) stage_cols(cell + cstep);
    for (int k = lane; k < nth; k += 32) a.psi_out[(size_t)cell * nth + k] = pnew[k];
    // Eq. 4 on every row, binding against the anchors' free motors
    for (int r0 = 0; r0 < nth; r0 += lg.rpp) {
      const int k = r0 + lg.rslot;
      const bool row_ok = k < nth, act = row_ok && lg.lane_ok;
      const size_t roff = ((size_t)cell * nth + (row_ok ? k : 0)) * ns + lg.sl * V;
      T M[V], D[V], Ms[V], mfv[V];
      int anc[V];
      unsigned ends = 0;
      U16Pack<V> pos = wps;
      if (act) {
        const Pack<T, V> q = qn;
        if (BW) {
          // the free motors of each node's anchor (a read per node: cheaper
          // than selecting the runs' first nodes)
          ends = en & 0xffu;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            M[v] = q.v[v];
            anc[v] = (int)u16_at<V>(wen, v) + wib;
            mfv[v] = wmf[anc[v]];
          }
        } else if (WIN) {
          // the free motors of each run's anchor, read once at the run's
          // first node
          ends = en & 0xffu;
          const unsigned starts = (ends << 1) | 1u;
          T cur = T(0);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            M[v] = q.v[v];
            anc[v] = wn.v[v];
            if ((starts >> v) & 1u) cur = wmf[anc[v]];
            mfv[v] = cur;
          }
        } else {
          const int2* o = x.off + (size_t)k * ns + lg.sl * V;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            M[v] = q.v[v];
            anc[v] = anchor_cell(ix, iy, o[v], nx, ny);
            mfv[v] = a.mf_in[anc[v]];
          }
        }
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          M[v] = T(0);
          mfv[v] = T(0);
          anc[v] = cell;
        }
      }
      if (r0 + lg.rpp < nth) load_pass(cell, r0 + lg.rpp);
      T snb = T(0);
      if constexpr (sizeof(T) == 4 && (V == 4 || V == 8)) {
        // register pairs, packed two-value arithmetic: the same nodal values,
        // bit for bit, as the scalar form below (the lane's n_b part is summed
        // in pairs)
        constexpr int H = V / 2;
        float2 M2[H], D2[H], Ms2[H], b2[H];
        const float2 c1_ = make_float2(c1, c1), c2_ = make_float2(c2, c2);
        const float2 e1_ = make_float2(e1, e1), e2_ = make_float2(e2, e2);
        const float2 hk_ = make_float2(hk, hk), fk_ = make_float2(fk, fk);
#pragma unroll
        for (int h = 0; h < H; ++h) {
          M2[h] = make_float2(M[2 * h], M[2 * h + 1]);
          b2[h] = make_float2(mfv[2 * h], mfv[2 * h + 1]);
        }
        walk_dflux_x2<V>(M2, D2, lg.first, lg.last, seg);
#pragma unroll
        for (int h = 0; h < H; ++h)
          Ms2[h] = __ffma2_rn(c1_, D2[h], __ffma2_rn(c2_, M2[h], __fmul2_rn(hk_, b2[h])));
        walk_dflux_x2<V>(Ms2, D2, lg.first, lg.last, seg);
        float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < H; ++h) {
          M2[h] = __ffma2_rn(e1_, D2[h],
                             __ffma2_rn(e2_, Ms2[h], __ffma2_rn(fk_, b2[h], M2[h])));
          acc2 = __fadd2_rn(acc2, M2[h]);
          M[2 * h] = M2[h].x;
          M[2 * h + 1] = M2[h].y;
        }
        snb = acc2.x + acc2.y;
      } else {
        walk_dflux<T, V>(M, D, lg.first, lg.last, seg);
#pragma unroll
        for (int v = 0; v < V; ++v) Ms[v] = fma_t(c1, D[v], fma_t(c2, M[v], hk * mfv[v]));
        walk_dflux<T, V>(Ms, D, lg.first, lg.last, seg);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          M[v] = fma_t(e1, D[v], fma_t(e2, Ms[v], fma_t(fk, mfv[v], M[v])));
          snb += M[v];
        }
      }
      if (act) {
        st_stream<T, V>(a.mb_out + roff, M);
        if (BW) {
          // each slot run's sum into its place among the cell's ordered sums
          const T w = pnew[k] * dsdth;
          T s = T(0);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            s = fma_t(w, M[v], s);
            if ((ends >> v) & 1u) {
              rbw[u16_at<V>(pos, v)] = s;
              s = T(0);
            }
          }
        } else if (WIN)
          scatter_runs_mask<T, V>(wacc, anc, M, pnew[k] * dsdth, ends);
        else
          scatter_runs<T, V>(x.cacc, anc, M, pnew[k] * dsdth);
      } else {
        snb = T(0);
      }
      snb = seg_sum(snb, seg);
      if (lg.first && row_ok) a.nb_out[(size_t)cell * nth + k] = snb * sc.ds;
    }
    __syncwarp();
    if (cell + cstep < nc) load_pass(cell + cstep, 0);
    if (BW) {
      // this cell's run sums per window entry: lane l adds its places in
      // order and stores the sum at each place that ends an entry
      const int r0 = (int)__ldg(x.sgrank + lane);
      int r = r0;
      T acc = T(0);
      for (int w = 0; w < x.nw; ++w) {
        const unsigned m = __ldg(x.sgbits + 32 * w + lane);
        const T* src = rbw + lane * x.ch + 32 * w;
        if (32 * w + 32 <= x.ch) {  // a whole word of places: constant bit masks
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            acc += src[i];
            if (m & (1u << i)) {
              sw[r++] = acc;
              acc = T(0);
            }
          }
        } else {
          const int n = x.ch - 32 * w;
#pragma unroll 4
          for (int i = 0; i < n; ++i) {
            acc += src[i];
            if ((m >> i) & 1u) {
              sw[r++] = acc;
              acc = T(0);
            }
          }
        }
      }
      // the places of an entry in earlier lanes: a segmented scan of the
      // lanes' open sums (a lane that ended an entry starts the next one)
      const unsigned had = __ballot_sync(0xffffffffu, r != r0);
      T v = acc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) {
          const unsigned span = ((2u << lane) - 1u) & ~((1u << (lane - d + 1)) - 1u);
          if (!(had & span)) v += u;
        }
      }
      const T cin = __shfl_up_sync(0xffffffffu, v, 1);
      if (lane > 0 && r != r0) sw[r0] += cin;
      __syncthreads();
      // the next group's window; then the 4 cells' sums of each window entry
      // into its global accumulator, one atomic per entry
      const int c0 = cell - wib;
      if (c0 + cstep < nc) fill_window(c0 + cstep);
      const int iy0 = c0 / nx, ix0 = c0 - iy0 * nx;
      int wyi = (int)threadIdx.x / wxb, wxi = (int)threadIdx.x - wyi * wxb;
      for (int w = threadIdx.x; w < Wn; w += blockDim.x) {
        const uint2 m = __ldg(x.m4 + w);
        const unsigned rr[4] = {m.x & 0xffffu, m.x >> 16, m.y & 0xffffu, m.y >> 16};
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (rr[c] != 0xffffu) s += sw0[(size_t)c * x.nkeys + rr[c]];
        if (s != T(0))
          atomicAdd(x.cacc + wrap(iy0 + x.woy + wyi, ny) * nx + wrap(ix0 + x.wox + wxi, nx),
                    (double)s);
        wxi += wdr;
        wyi += wdq;
        if (wxi >= wxb) wxi -= wxb, ++wyi;
      }
    } else if (WIN) {  // the window's sums into the global accumulators
      for (int w = lane; w < Wn; w += 32) {
        const T v = wacc[w];
        if (v != T(0)) atomicAdd(x.cacc + wcell[w], (double)v);
      }
      __syncwarp();
    }
  }
  // sum psi^{n+1} as in k_substep: per warp, per block, then the last block
  // (float-float in the float32 form)
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

// Eq. 5 at the anchors, the Alg. 2 scale-down and Eq. 6 (thread per cell).
template <typename T>
__global__ void k_anchor_close(const AnchorArgs<T> x, const T* mtot, T* mf, T* c, long long ncells) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < ncells;
       r += (long long)gridDim.x * blockDim.x) {
    const double C = x.cacc[r];
    x.cacc[r] = 0.0;
    const double M = (double)mtot[r];
    double f = 1.0, Cc = C;
    if (M < C) {
      f = M / C;
      Cc = M;
    }
    x.fsc[r] = f;
    c[r] = (T)Cc;
    mf[r] = (T)(M - Cc);
    if (f != 1.0) atomicOr(x.flags + x.flag, 1);
  }
}

// Where an anchor scaled down: every node times its anchor's factor, n_b of
// the row recomputed (warp per cell; nothing to do without the flag).
template <typename T, int V>
__global__ void __launch_bounds__(128) k_anchor_fix(const AnchorArgs<T> x, T* mb, T* nb, int nx,
                                                    int ny, int nth, int ns, int seg, double ds,
                                                    long long ncells) {
  if (x.flags[x.flag] == 0) return;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int W = gridDim.x * (blockDim.x >> 5);
  const LaneGeom lg = lane_geom(lane, seg, ns, V);
  for (int cell = gw; cell < (int)ncells; cell += W) {
    const int iy = cell / nx, ix = cell - iy * nx;
    for (int r0 = 0; r0 < nth; r0 += lg.rpp) {
      const int k = r0 + lg.rslot;
      const bool row_ok = k < nth, act = row_ok && lg.lane_ok;
      const size_t roff = ((size_t)cell * nth + (row_ok ? k : 0)) * ns + lg.sl * V;
      T snb = T(0);
      if (act) {
        Pack<T, V> q = *reinterpret_cast<const Pack<T, V>*>(mb + roff);
        const int2* o = x.off + (size_t)k * ns + lg.sl * V;
        bool any = false;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const double f = x.fsc[anchor_cell(ix, iy, o[v], nx, ny)];
          if (f != 1.0) {
            q.v[v] = (T)((double)q.v[v] * f);
            any = true;
          }
          snb += q.v[v];
        }
        if (any) *reinterpret_cast<Pack<T, V>*>(mb + roff) = q;
      }
      snb = seg_sum(snb, seg);
      if (lg.first && row_ok) nb[(size_t)cell * nth + k] = snb * (T)ds;
    }
  }
}

// Row sums and the scatter of a given state: mode 0 n_b and psi ds dth Mb into
// the coarse accumulators (state set-up); mode 1 the motor force of Eq. 10,
// F p psi Mb ds dth, into fx, fy (float64, [cells] each). psi is scaled by g.
template <typename T, int V>
__global__ void __launch_bounds__(128) k_anchor_scatter(const AnchorArgs<T> x, const T* mb,
                                                        const T* psi, T* nb, double* fx,
                                                        double* fy, const double* trig64,
                                                        const DevParams* prm, int mode, int nx,
                                                        int ny, int nth, int ns, int seg,
                                                        double ds, double dth, long long ncells) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int W = gridDim.x * (blockDim.x >> 5);
  const LaneGeom lg = lane_geom(lane, seg, ns, V);
  const double g = prm->psi_scale;
  const double Fm = prm->force_scale;
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) x.flags[x.flag] = 0;
  for (int cell = gw; cell < (int)ncells; cell += W) {
    const int iy = cell / nx, ix = cell - iy * nx;
    for (int r0 = 0; r0 < nth; r0 += lg.rpp) {
      const int k = r0 + lg.rslot;
      const bool row_ok = k < nth, act = row_ok && lg.lane_ok;
      const size_t roff = ((size_t)cell * nth + (row_ok ? k : 0)) * ns + lg.sl * V;
      T snb = T(0);
      if (act) {
        const Pack<T, V> q = *reinterpret_cast<const Pack<T, V>*>(mb + roff);
        const int2* o = x.off + (size_t)k * ns + lg.sl * V;
        const double w = (double)psi[(size_t)cell * nth + k] * g * ds * dth;
        int anc[V];
        double Mv[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          anc[v] = anchor_cell(ix, iy, o[v], nx, ny);
          Mv[v] = (double)q.v[v];
          snb += q.v[v];
        }
        if (mode == 0) {
          scatter_runs<double, V>(x.cacc, anc, Mv, w);
        } else {
          scatter_runs<double, V>(fx, anc, Mv, Fm * trig64[k] * w);
          scatter_runs<double, V>(fy, anc, Mv, Fm * trig64[nth + k] * w);
        }
      }
      if (mode == 0) {
        snb = seg_sum(snb, seg);
        if (lg.first && row_ok) nb[(size_t)cell * nth + k] = snb * (T)ds;
      }
    }
  }
}

}  // namespace mm

using namespace mmh;

namespace {

template <typename T>
mm::AnchorArgs<T> anchor_args(mm_handle* h, int flag) {
  mm::AnchorArgs<T> x;
  x.off = (const int2*)h->anc_off;
  x.cacc = h->anc_cacc;
  x.fsc = h->anc_fsc;
  x.flags = h->anc_flags;
  x.flag = flag;
  x.widx = h->anc_widx;
  x.runend = h->anc_runend;
  x.wox = h->anc_win[0];
  x.woy = h->anc_win[1];
  x.wx = h->anc_win[2];
  x.wy = h->anc_win[3];
  const size_t nn = (size_t)h->g.ntheta * h->g.ns, wnb = (size_t)(x.wx + 3) * x.wy;
  x.went = h->anc_wtab;
  x.wpos = h->anc_wtab + nn;
  x.m4 = reinterpret_cast<const uint2*>(h->anc_rtab);
  x.sgbits = h->anc_rtab ? h->anc_rtab + 2 * wnb : nullptr;
  x.sgrank = h->anc_rtab ? x.sgbits + 32 * (size_t)h->anc_sg[2] : nullptr;
  x.nsr = h->anc_nsr;
  x.nsrp = h->anc_sg[0];
  x.ch = h->anc_sg[1];
  x.nw = h->anc_sg[2];
  x.nkeys = h->anc_sg[3];
  return x;
}

int blocks_for(long long work, int per_block, int cap) {
  long long b = (work + per_block - 1) / per_block;
  if (b > cap) b = cap;
  return (int)std::max<long long>(b, 1);
}

// Shared memory of the block-window form: the 4 warps' columns, then the
// window's free motors ((wx + 3) x wy entries), then the 4 cells' ordered run
// sums and their per-entry sums.
template <typename T>
size_t anchor_bw_smem(const mm_handle* h) {
  const size_t wn = (size_t)(h->anc_win[2] + 3) * h->anc_win[3];
  return 4 * mm::anchor_warp_smem(h->g.ntheta, sizeof(T), 0) + ((wn * sizeof(T) + 15) & ~(size_t)15) +
         4 * ((size_t)h->anc_sg[0] + h->anc_sg[3]) * sizeof(T);
}

// Warps per block of the anchor substep (shared memory of 11 ntheta values per
// warp) and the kernels' shared-memory limit.
template <typename T, int V>
cudaError_t anchor_prepare_t(mm_handle* h) {
  const int W = h->anc_win[2] * h->anc_win[3];
  const size_t per_warp = mm::anchor_warp_smem(h->g.ntheta, sizeof(T), W);
  h->anc_wpb = (int)std::min<size_t>(4, kSmemBudget / per_warp);
  if (h->anc_wpb < 1) return cudaErrorInvalidValue;
  const int smem = (int)(h->anc_wpb * per_warp);
  const void* fns[4] = {(const void*)mm::k_substep_anchor<T, V, true, true>,
                        (const void*)mm::k_substep_anchor<T, V, false, true>,
                        (const void*)mm::k_substep_anchor<T, V, true, false>,
                        (const void*)mm::k_substep_anchor<T, V, false, false>};
  for (const void* f : fns) {
    cudaError_t e = mm::raise_smem_limit(f, smem);
    if (e != cudaSuccess) return e;
  }
  if (h->anc_bw) {
    const size_t bsm = anchor_bw_smem<T>(h);
    if (bsm > kSmemBudget) {
      h->anc_bw = false;
    } else {
      const void* bfns[2] = {(const void*)mm::k_substep_anchor<T, V, true, true, true>,
                             (const void*)mm::k_substep_anchor<T, V, false, true, true>};
      for (const void* f : bfns) {
        cudaError_t e =
            mm::raise_smem_limit(f, (int)bsm);
        if (e != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

template <typename T, int V>
cudaError_t anchor_substep_t(mm_handle* h, int parity, cudaStream_t s) {
  const StepArgs<T> a = step_args<T>(h, parity);
  const mm::AnchorArgs<T> x = anchor_args<T>(h, parity);
  const int wpb = h->anc_wpb;
  const bool win = x.wx > 0;
  const size_t smem = wpb * mm::anchor_warp_smem(h->g.ntheta, sizeof(T), x.wx * x.wy);
  const int grid = blocks_for(h->ncells, wpb, 8 * h->sms);
  if (win && h->anc_bw) {  // 4 consecutive cells of a row per block, one window
    const int bgrid = blocks_for(h->ncells / 4, 1, 8 * h->sms);
    const size_t bsm = anchor_bw_smem<T>(h);
    if (a.mass_correct)
      mm::k_substep_anchor<T, V, true, true, true><<<bgrid, 128, bsm, s>>>(a, x);
    else
      mm::k_substep_anchor<T, V, false, true, true><<<bgrid, 128, bsm, s>>>(a, x);
  } else if (win) {
    if (a.mass_correct)
      mm::k_substep_anchor<T, V, true, true><<<grid, 32 * wpb, smem, s>>>(a, x);
    else
      mm::k_substep_anchor<T, V, false, true><<<grid, 32 * wpb, smem, s>>>(a, x);
  } else if (a.mass_correct) {
    mm::k_substep_anchor<T, V, true, false><<<grid, 32 * wpb, smem, s>>>(a, x);
  } else {
    mm::k_substep_anchor<T, V, false, false><<<grid, 32 * wpb, smem, s>>>(a, x);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mm::k_anchor_close<T><<<blocks_for(h->ncells, 256, 8 * h->sms), 256, 0, s>>>(
      x, (const T*)h->mtot, (T*)h->mf, (T*)h->c, h->ncells);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mm::k_anchor_fix<T, V><<<grid, 128, 0, s>>>(x, (T*)h->mb, (T*)h->nb[parity ^ 1], h->g.nx,
                                             h->g.ny, h->g.ntheta, h->g.ns, h->seg,
                                             h->g.L / h->g.ns, h->ncells);
  return cudaGetLastError();
}

template <typename T, int V>
cudaError_t anchor_scatter_t(mm_handle* h, int mode, double* fx, double* fy) {
  const mm::AnchorArgs<T> x = anchor_args<T>(h, 2);
  const int grid = blocks_for(h->ncells, 4, 8 * h->sms);
  const double ds = h->g.L / h->g.ns, dth = 2.0 * kPi / h->g.ntheta;
  mm::k_anchor_scatter<T, V><<<grid, 128, 0, h->stream>>>(
      x, (const T*)h->mb, (const T*)h->psi[h->parity], (T*)h->nb[h->parity], fx, fy, h->trig64,
      h->prm, mode, h->g.nx, h->g.ny, h->g.ntheta, h->g.ns, h->seg, ds, dth, h->ncells);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || mode != 0) return e;
  mm::k_anchor_close<T><<<blocks_for(h->ncells, 256, 8 * h->sms), 256, 0, h->stream>>>(
      x, (const T*)h->mtot, (T*)h->mf, (T*)h->c, h->ncells);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mm::k_anchor_fix<T, V><<<grid, 128, 0, h->stream>>>(x, (T*)h->mb, (T*)h->nb[h->parity],
                                                      h->g.nx, h->g.ny, h->g.ntheta, h->g.ns,
                                                      h->seg, ds, h->ncells);
  return cudaGetLastError();
}

// Dispatch on precision and the substep's vector width.
template <template <typename, int> class F, typename... A>
cudaError_t by_width(mm_handle* h, A... args) {
  if (h->prec == MM_FP64) return h->V == 2 ? F<double, 2>::run(h, args...) : F<double, 1>::run(h, args...);
  if (h->V == 8) return F<float, 8>::run(h, args...);
  return h->V == 4 ? F<float, 4>::run(h, args...) : F<float, 1>::run(h, args...);
}
template <typename T, int V>
struct SubstepF {
  static cudaError_t run(mm_handle* h, int parity, cudaStream_t s) {
    return anchor_substep_t<T, V>(h, parity, s);
  }
};
template <typename T, int V>
struct PrepareF {
  static cudaError_t run(mm_handle* h) { return anchor_prepare_t<T, V>(h); }
};
template <typename T, int V>
struct ScatterF {
  static cudaError_t run(mm_handle* h, int mode, double* fx, double* fy) {
    return anchor_scatter_t<T, V>(h, mode, fx, fy);
  }
};

}  // namespace

namespace mmh {

// The anchor tables ([nth][ns] offsets and window indices) and the per-cell
// float64 accumulators and factors.
mm_status anchor_alloc(mm_handle* h) {
  const size_t nc = (size_t)h->ncells;
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  const size_t need = (size_t)h->g.ntheta * h->g.ns * sizeof(int2) + 2 * nc * 8 + 64;
  if (need + (1 << 20) > freeb) return fail(h, MM_ERR_OOM, "anchor buffers do not fit");
  CK(cudaMalloc((void**)&h->anc_off, (size_t)h->g.ntheta * h->g.ns * sizeof(int2)));
  CK(cudaMalloc((void**)&h->anc_widx, (size_t)h->g.ntheta * h->g.ns * sizeof(int)));
  CK(cudaMalloc((void**)&h->anc_wtab, 2 * (size_t)h->g.ntheta * h->g.ns * sizeof(unsigned short)));
  CK(cudaMalloc((void**)&h->anc_runend, (size_t)h->g.ntheta * h->g.ns * sizeof(unsigned)));
  CK(cudaMalloc((void**)&h->anc_cacc, nc * 8));
  CK(cudaMalloc((void**)&h->anc_fsc, nc * 8));
  CK(cudaMalloc((void**)&h->anc_flags, 4 * sizeof(int)));
  CK(cudaMemset(h->anc_cacc, 0, nc * 8));
  CK(cudaMemset(h->anc_flags, 0, 4 * sizeof(int)));
  return MM_OK;
}

// The anchor offsets of the current grid and l/L, reduced into [0, nx) and
// [0, ny), with the formula of the definition evaluated in float64 by products
// and quotients only (no operation a compiler could fuse).
mm_status anchor_table(mm_handle* h) {
  const int nth = h->g.ntheta, ns = h->g.ns, nx = h->g.nx, ny = h->g.ny;
  const double dx = 1.0 / nx, dy = 1.0 / ny, dth = 2.0 * kPi / nth;
  std::vector<int2> off((size_t)nth * ns), raw((size_t)nth * ns);
  long long xmin = 0, xmax = 0, ymin = 0, ymax = 0;
  for (int k = 0; k < nth; ++k) {
    const double th = k * dth, ct = std::cos(th), st = std::sin(th);
    for (int j = 0; j < ns; ++j) {
      const double disp = h->r.ell * h->g.L * (double)(2 * j + 1 - ns) / (2.0 * ns);
      const double qx = std::floor(disp * ct / dx + 0.5), qy = std::floor(disp * st / dy + 0.5);
      if (!(std::fabs(qx) < 1e9 && std::fabs(qy) < 1e9))
        return fail(h, MM_ERR_UNSUPPORTED, "anchor offsets out of range");
      const long long rx = (long long)qx, ry = (long long)qy;
      if (k == 0 && j == 0) xmin = xmax = rx, ymin = ymax = ry;
      xmin = std::min(xmin, rx);
      xmax = std::max(xmax, rx);
      ymin = std::min(ymin, ry);
      ymax = std::max(ymax, ry);
      raw[(size_t)k * ns + j] = make_int2((int)rx, (int)ry);
      long long ox = rx % nx, oy = ry % ny;
      if (ox < 0) ox += nx;
      if (oy < 0) oy += ny;
      off[(size_t)k * ns + j] = make_int2((int)ox, (int)oy);
    }
  }
  // the window of anchor cells around a filament cell, when it is small
  const long long wx = xmax - xmin + 1, wy = ymax - ymin + 1;
  std::vector<int> widx((size_t)nth * ns), widxb((size_t)nth * ns);
  h->anc_win[0] = h->anc_win[1] = h->anc_win[2] = h->anc_win[3] = 0;
  // a block's 4 warps share one window when they take 4 consecutive cells of a
  // row (nx a multiple of 4), the widened window fits and the window is no
  // wider or taller than the grid (a window coordinate then wraps at most once)
  h->anc_bw = nx % 4 == 0 && (wx + 3) * wy <= kAnchorBlockWindowMax && wx * wy <= kAnchorWindowMax &&
              wx <= nx && wy <= ny;
  if (wx * wy <= kAnchorWindowMax) {
    for (size_t q = 0; q < widx.size(); ++q) {
      widx[q] = (int)((raw[q].y - ymin) * wx + (raw[q].x - xmin));
      widxb[q] = (int)((raw[q].y - ymin) * (wx + 3) + (raw[q].x - xmin));
    }
    h->anc_win[0] = (int)xmin;
    h->anc_win[1] = (int)ymin;
    h->anc_win[2] = (int)wx;
    h->anc_win[3] = (int)wy;
  }
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(h->anc_off, off.data(), off.size() * sizeof(int2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->anc_widx, widx.data(), widx.size() * sizeof(int), cudaMemcpyHostToDevice));
  // the run ends of each lane slot of V nodes: a node whose successor in the
  // slot has another anchor, and the slot's last node (the window indices of
  // two nodes are equal exactly when their offsets are); the block window's
  // entry of each slot run and each node's slot run
  const int V = h->V, nsl = ns / V;
  const size_t nn = (size_t)nth * ns;
  std::vector<unsigned> runend((size_t)nth * nsl, 0);
  std::vector<int> sr_w, node_run(nn);
  for (int k = 0; k < nth; ++k)
    for (int sl = 0; sl < nsl; ++sl) {
      unsigned m = 0;
      for (int v = 0; v < V; ++v) {
        const size_t q = (size_t)k * ns + sl * V + v;
        node_run[q] = (int)sr_w.size();
        if (v == V - 1 || raw[q].x != raw[q + 1].x || raw[q].y != raw[q + 1].y) {
          m |= 1u << v;
          sr_w.push_back(widxb[q]);
        }
      }
      runend[(size_t)k * nsl + sl] = m;
    }
  CK(cudaMemcpy(h->anc_runend, runend.data(), runend.size() * sizeof(unsigned),
                cudaMemcpyHostToDevice));
  // The block-window form: the slot runs ordered (stably) by window entry, the
  // same order in every cell; nsrp = 32 ch places (an odd ch: the lanes' reads
  // of their places fall in distinct banks), the last entry's places running
  // on over the zeros past nsr. Places, entries and per-entry indices must fit
  // 16 bits.
  const long long nsr = (long long)sr_w.size();
  const long long ch = ((nsr + 31) / 32) | 1, nsrp = 32 * ch;
  const long long wnb = (wx + 3) * wy;
  if (h->anc_rtab) cudaFree(h->anc_rtab);
  h->anc_rtab = nullptr;
  h->anc_nsr = (int)nsr;
  h->anc_sg[0] = h->anc_sg[1] = h->anc_sg[2] = h->anc_sg[3] = 0;
  if (h->anc_bw && (nsrp >= 0xffff || wnb >= 0xffff)) h->anc_bw = false;
  if (h->anc_bw) {
    std::vector<int> ord((size_t)nsr);
    for (long long r = 0; r < nsr; ++r) ord[r] = (int)r;
    std::stable_sort(ord.begin(), ord.end(), [&](int p, int q) { return sr_w[p] < sr_w[q]; });
    std::vector<int> place((size_t)nsr);
    for (long long p = 0; p < nsr; ++p) place[ord[p]] = (int)p;
    // node tables: each node's window entry and its slot run's place
    std::vector<unsigned short> wt(2 * nn);
    for (size_t q = 0; q < nn; ++q) {
      wt[q] = (unsigned short)widxb[q];
      wt[nn + q] = (unsigned short)place[node_run[q]];
    }
    // the places that end an entry's places, and each entry's index among a
    // cell's per-entry sums (in place order)
    std::vector<char> end((size_t)nsrp, 0);
    for (long long p = 0; p + 1 < nsr; ++p) end[p] = sr_w[ord[p]] != sr_w[ord[p + 1]];
    end[nsrp - 1] = 1;
    std::vector<int> key_rank((size_t)wnb, 0xffff);
    int nk = 0;
    for (long long p = 0; p < nsrp; ++p)
      if (end[p]) key_rank[sr_w[ord[std::min(p, nsr - 1)]]] = nk++;
    // lane chunks: end marks per lane ([nw][32] words) and ends before each lane
    const int nw = (int)((ch + 31) / 32);
    std::vector<unsigned> tab(2 * (size_t)wnb + 32 * (size_t)nw + 32, 0);
    unsigned* bits = tab.data() + 2 * wnb;
    unsigned* rank0 = bits + 32 * nw;
    int before = 0;
    for (int l = 0; l < 32; ++l) {
      rank0[l] = (unsigned)before;
      for (long long i = 0; i < ch; ++i)
        if (end[l * ch + i]) {
          bits[(i / 32) * 32 + l] |= 1u << (i % 32);
          ++before;
        }
    }
    // per block-window entry, the per-entry sum index of entry e - c in cell c
    const long long wxb = wx + 3;
    for (long long e = 0; e < wnb; ++e) {
      const long long wxi = e % wxb;
      unsigned r4[4];
      for (int c = 0; c < 4; ++c)
        r4[c] = (wxi - c >= 0 && wxi - c < wx) ? (unsigned)key_rank[e - c] : 0xffffu;
      tab[2 * e] = r4[0] | (r4[1] << 16);
      tab[2 * e + 1] = r4[2] | (r4[3] << 16);
    }
    CK(cudaMemcpy(h->anc_wtab, wt.data(), wt.size() * sizeof(unsigned short), cudaMemcpyHostToDevice));
    CK(cudaMalloc((void**)&h->anc_rtab, tab.size() * sizeof(unsigned)));
    CK(cudaMemcpy(h->anc_rtab, tab.data(), tab.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    h->anc_sg[0] = (int)nsrp;
    h->anc_sg[1] = (int)ch;
    h->anc_sg[2] = nw;
    h->anc_sg[3] = nk;
  }
  // captured substep graphs hold the window and block shape as launch arguments
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  const cudaError_t e = by_width<PrepareF>(h);
  if (e == cudaErrorInvalidValue)
    return fail(h, MM_ERR_UNSUPPORTED, "ntheta too large for the anchor kernel's shared memory");
  CK(e);
  return MM_OK;
}

cudaError_t launch_anchor_substep(mm_handle* h, int parity, cudaStream_t s) {
  return by_width<SubstepF>(h, parity, s);
}

// State set-up with anchors: n_b, C at the anchors, the scale-down, Mf.
mm_status run_init_anchor(mm_handle* h) {
  CK(cudaMemsetAsync(h->anc_cacc, 0, (size_t)h->ncells * 8, h->stream));
  CK(by_width<ScatterF>(h, 0, (double*)nullptr, (double*)nullptr));
  return MM_OK;
}

// The motor force of Eq. 10 at the anchors into fields 7 and 8.
mm_status anchor_force(mm_handle* h) {
  const size_t nc = (size_t)h->ncells;
  CK(cudaMemsetAsync(h->fields + 7 * nc, 0, 2 * nc * 8, h->stream));
  CK(by_width<ScatterF>(h, 1, h->fields + 7 * nc, h->fields + 8 * nc));
  return MM_OK;
}

}  // namespace mmh

extern "C" {

mm_status mm_set_anchors(mm_handle* h, int enable) {
  MM_TRACE("mm_set_anchors");
  if (!h) return MM_ERR_INVALID;
  if (h->batch || h->owner)
    return fail(h, MM_ERR_UNSUPPORTED, "non-local anchors are not available in a batch");
  if (h->rec.active)
    return fail(h, MM_ERR_STATE, "non-local anchors are not differentiated: end the adjoint recording first");
  if (enable && h->capture)
    return fail(h, MM_ERR_STATE, "a capture radius is set: switch it off (mm_set_capture < 0) first");
  if (enable && h->tangent)
    return fail(h, MM_ERR_STATE, "the tangent mode is on: switch it off (mm_set_tangent) first");
  DeviceGuard dg(h->device);
  CK(cudaStreamSynchronize(h->stream));
  mm_status st;
  if (enable && !h->anc_off && (st = anchor_alloc(h)) != MM_OK) return st;
  if (enable && (st = anchor_table(h)) != MM_OK) return st;
  h->anchors = enable != 0;
  // substep graphs were captured for the other kernels
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  // C, the scale-down and Mf of the current state under the new rule
  if (h->have_state) return h->anchors ? run_init_anchor(h) : run_init(h);
  return MM_OK;
}

}  // extern "C"
