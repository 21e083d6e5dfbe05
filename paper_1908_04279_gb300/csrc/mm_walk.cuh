// Device helpers shared by the forward substep kernel and its adjoint: the
// Superbee-limited walking flux of Eq. 4 on lane-distributed s-rows, min/max,
// fused multiply-add and warp reductions.
#pragma once

#include "mm_internal.cuh"

namespace mm {

template <typename T, int V>
struct alignas(sizeof(T) * V) Pack {
  T v[V];
};

// Single min/max instructions (the operands are never NaN here).
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
// An addition the compiler may not fuse with a product feeding it (the same
// bits wherever the addend's product is computed).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Donor-cell face flux: upwind state times face velocity, with an explicit fma
// so that both cells sharing a face compute the same bits (exact telescoping).
template <typename T>
__device__ __forceinline__ T donor(T A, T pl, T pr) {
  return fma_t(tmax(A, T(0)), pl, tmin(A, T(0)) * pr);
}

__device__ __forceinline__ float max3_t(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double max3_t(double a, double b, double c) {
  return fmax(fmax(a, b), c);
}

// The sign bit of a float64 pattern.
constexpr long long kSign64 = (long long)0x8000000000000000ull;

// The float64 Superbee flux F = M + sigma/2 of one node (the general form of
// walk_dflux below) and its branch decisions, with the sign flips, magnitudes,
// minima and maximum on the bit patterns (integer pipe instead of the float64
// one, whose rate is a small fraction of float32's), the same values bit for
// bit: A = a sgn and hA = a/2 sgn take the sign bit of b, |b| and |b|/2 drop
// it; for hB, B >= 0 the signed 64-bit patterns order as the values do and a
// negative A (sign bit set, -0 included) orders below them, so min(A, hB) is
// the smaller pattern; max(t1, t2, 0) is the largest pattern, a negative one
// giving +0 (fmin and fmax order -0 below +0 alike); F = M + sgn r is one
// rounded addition, as the fma with sgn = +-1 is (+0 added at the plus end,
// where sgn = 0 made the product +0). The decisions: r > 0, t1 > t2, A < hB,
// hA < B (where -0 and +0 would differ, r = 0).
struct Lim64 {
  double F;
  bool pos, p1, x1a, x2a;
};
__device__ __forceinline__ Lim64 superbee64(double a, double ha, double b, double hb, bool endp,
                                            double M) {
  const long long ib = __double_as_longlong(b);
  const long long sb = ib & kSign64;
  const long long iA = __double_as_longlong(a) ^ sb, ihA = __double_as_longlong(ha) ^ sb;
  const long long iB = ib & ~kSign64, ihB = __double_as_longlong(hb) & ~kSign64;
  const long long it1 = iA < ihB ? iA : ihB, it2 = ihA < iB ? ihA : iB;
  long long ir = it1 > it2 ? it1 : it2;
  if (ir < 0 || endp) ir = 0;
  Lim64 q;
  q.F = __dadd_rn(M, __longlong_as_double(endp ? 0ll : ir ^ sb));
  q.pos = ir > 0;
  q.p1 = it1 > it2;
  q.x1a = iA < ihB;
  q.x2a = ihA < iB;
  return q;
}

// min(|a|, |b|) carrying the sign sign(a) xor sign(b): positive where a and b
// agree in sign, negative where they disagree (one instruction).
__device__ __forceinline__ float min_xorsign_abs(float a, float b) {
  float r;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Walking-flux differences of the V nodes a lane holds (the d_s term of
// Eq. 4 divided by v/ds): D_v = F_{j-1} - F_j with F_j = M_j + sigma_j/2 the
// flux / v through the right face of node j = lane*V + v, F_{-1} = 0 (nothing
// walks on at the minus end) and F_{ns-1} = M_{ns-1} (donor-cell outflow at
// the plus end). sigma_j is the Superbee slope
// maxmod(minmod(2a, b), minmod(a, 2b)) of the backward and forward
// differences a, b (ghost M_{-1} = 0), evaluated on magnitudes: with
// s = sign(b), sigma/2 = s max(min(s a, |b|/2), min(s a/2, |b|), 0).
// Neighbouring nodes of other lanes come by warp shuffles within the row's
// `seg`-lane segment.
//
// With COEF, also the derivative of sigma_j/2 on the branch taken:
// sigma/2 = ga a + gb b with (ga, gb) one of (1, 0) [2a], (0, 1/2) [b],
// (1/2, 0) [a], (0, 1) [2b] or (0, 0). The comparisons follow the Superbee
// definition with strict inequalities (minmod keeps the second argument and
// maxmod the second on ties), so that the branch is the one the forward map
// takes; the value of D is the same bits as without COEF.
template <typename T, int V, bool COEF = false>
__device__ __forceinline__ void walk_dflux(const T (&M)[V], T (&D)[V], bool first, bool last,
                                           int seg, T* ga = nullptr, T* gb = nullptr) {
  T ml = __shfl_up_sync(0xffffffffu, M[V - 1], 1, seg);
  const T mr = __shfl_down_sync(0xffffffffu, M[0], 1, seg);
  if (first) ml = T(0);
  T d[V + 1], hd[V + 1];  // d[i] = M_i - M_{i-1}, i = 0..V, with M_{-1} = ml, M_V = mr
  d[0] = M[0] - ml;
#pragma unroll
  for (int v = 1; v < V; ++v) d[v] = M[v] - M[v - 1];
  d[V] = mr - M[V - 1];
#pragma unroll
  for (int i = 0; i <= V; ++i) hd[i] = T(0.5) * d[i];
  T F[V];
  if constexpr (sizeof(T) == 4 && !COEF) {
    // float32 forward: sigma/2 = sign(b) max(min(|a|, |b|/2), min(|a|/2, |b|))
    // where a and b agree in sign, else 0 -- the two minima with the agreement
    // in their sign, so that the maximum with 0 drops the disagreeing case
    // (the same value, bit for bit, as the general form below)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T r = max3_t(min_xorsign_abs(d[v], hd[v + 1]), min_xorsign_abs(hd[v], d[v + 1]), T(0));
      if (v == V - 1 && last) r = T(0);  // plus end: F = M, no slope
      F[v] = M[v] + copysignf(r, d[v + 1]);
    }
  } else if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const Lim64 q = superbee64(d[v], hd[v], d[v + 1], hd[v + 1], v == V - 1 && last, M[v]);
      F[v] = q.F;
      if constexpr (COEF) {
        const T a1 = q.x1a ? T(1) : T(0), b1 = q.x1a ? T(0) : T(0.5);
        const T a2 = q.x2a ? T(0.5) : T(0), b2 = q.x2a ? T(0) : T(1);
        ga[v] = q.pos ? (q.p1 ? a1 : a2) : T(0);
        gb[v] = q.pos ? (q.p1 ? b1 : b2) : T(0);
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T sgn = copysign(T(1), d[v + 1]);
      if (v == V - 1 && last) sgn = T(0);  // plus end: F = M, no slope
      const T A = d[v] * sgn, hA = hd[v] * sgn;
      const T hB = fabs(hd[v + 1]), B = fabs(d[v + 1]);
      const T t1 = tmin(A, hB), t2 = tmin(hA, B);
      const T r = max3_t(t1, t2, T(0));
      F[v] = fma_t(r, sgn, M[v]);
      if constexpr (COEF) {
        const bool pos = r > T(0), p1 = t1 > t2, x1a = A < hB, x2a = hA < B;
        const T a1 = x1a ? T(1) : T(0), b1 = x1a ? T(0) : T(0.5);
        const T a2 = x2a ? T(0.5) : T(0), b2 = x2a ? T(0) : T(1);
        ga[v] = pos ? (p1 ? a1 : a2) : T(0);
        gb[v] = pos ? (p1 ? b1 : b2) : T(0);
      }
    }
  }
  T fl = __shfl_up_sync(0xffffffffu, F[V - 1], 1, seg);
  if (first) fl = T(0);
  D[0] = fl - F[0];
#pragma unroll
  for (int v = 1; v < V; ++v) D[v] = F[v - 1] - F[v];
}

// The float32 walk of walk_dflux for V = 4 or 8 nodes per lane, with the
// lane's values held as V/2 register pairs (nodes 2k, 2k + 1), so that the
// element-wise steps (the halved differences, the fluxes) run as packed
// two-value float32 instructions; the differences, the limiter's minima and
// maxima and the flux differences stay scalar. Same value, bit for bit, as
// walk_dflux<float, V>.
template <int V>
__device__ __forceinline__ void walk_dflux_x2(const float2 (&M)[V / 2], float2 (&D)[V / 2],
                                              bool first, bool last, int seg) {
  constexpr int H = V / 2;
  float ml = __shfl_up_sync(0xffffffffu, M[H - 1].y, 1, seg);
  const float mr = __shfl_down_sync(0xffffffffu, M[0].x, 1, seg);
  if (first) ml = 0.0f;
  // d_v = M_v - M_{v-1} as pairs (d_2k, d_2k+1), and d_V
  float2 d[H], hd[H];
  d[0] = make_float2(M[0].x - ml, M[0].y - M[0].x);
#pragma unroll
  for (int k = 1; k < H; ++k) d[k] = make_float2(M[k].x - M[k - 1].y, M[k].y - M[k].x);
  const float dV = mr - M[H - 1].y, hdV = 0.5f * dV;
  const float2 half2 = make_float2(0.5f, 0.5f);
#pragma unroll
  for (int k = 0; k < H; ++k) hd[k] = __fmul2_rn(half2, d[k]);
  float2 F[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float b1 = k + 1 < H ? d[k + 1].x : dV, hb1 = k + 1 < H ? hd[k + 1].x : hdV;
    const float r0 =
        max3_t(min_xorsign_abs(d[k].x, hd[k].y), min_xorsign_abs(hd[k].x, d[k].y), 0.0f);
    float r1 = max3_t(min_xorsign_abs(d[k].y, hb1), min_xorsign_abs(hd[k].y, b1), 0.0f);
    if (k == H - 1 && last) r1 = 0.0f;  // plus end: F = M, no slope
    F[k] = __fadd2_rn(M[k], make_float2(copysignf(r0, d[k].y), copysignf(r1, b1)));
  }
  float fl = __shfl_up_sync(0xffffffffu, F[H - 1].y, 1, seg);
  if (first) fl = 0.0f;
  D[0] = make_float2(fl - F[0].x, F[0].x - F[0].y);
#pragma unroll
  for (int k = 1; k < H; ++k) D[k] = make_float2(F[k - 1].y - F[k].x, F[k].x - F[k].y);
}

template <typename T>
__device__ __forceinline__ T seg_sum(T x, int seg) {
  for (int o = seg >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o, seg);
  return x;
}
template <typename T>
__device__ __forceinline__ T warp_sum_t(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Fixed-order float64 sum, by one warp, of p[0], p[stride], ...,
// p[(n - 1) stride], values other blocks wrote (read through L2). Lane l adds
// the values l, l + 32, ... into eight interleaved partial sums, so that eight
// loads are in flight per lane instead of one dependent load per value; the
// partials and the lanes then combine in a fixed tree. The result does not
// depend on the order in which blocks ran.
__device__ __forceinline__ double warp_sum_ldcg(const double* p, int n, int stride, int lane) {
  double s[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) s[q] = 0.0;
  int b = lane;
  for (; b + 7 * 32 < n; b += 8 * 32) {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcg(p + (size_t)(b + q * 32) * stride);
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] += v[q];
  }
#pragma unroll
  for (int q = 0; q < 7; ++q)
    if (b + q * 32 < n) s[q] += __ldcg(p + (size_t)(b + q * 32) * stride);
  return warp_sum(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])));
}


// Float-float values carried in a float2 (x: high part, y: low part), for the
// float32 form's end-of-launch sums: GB300's float64 pipe runs at 1/64 of the
// float32 rate and a float64 warp instruction costs it the same however few
// lanes are active, so a serial tail of float64 additions on one SM delays
// every launch; these run on the float32 pipe (TwoSum of the high parts).
__device__ __forceinline__ float2 ff2_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  return make_float2(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 warp_sum_ff2(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = ff2_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o),
                               __shfl_xor_sync(0xffffffffu, v.y, o)));
  return v;
}
// warp_sum_ldcg for float-float pairs p[0..n-1] (stride 1): the same loads in
// flight and the same fixed combination order.
__device__ __forceinline__ float2 warp_sum_ldcg_ff2(const float2* p, int n, int lane) {
  float2 s[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) s[q] = make_float2(0.f, 0.f);
  int b = lane;
  for (; b + 7 * 32 < n; b += 8 * 32) {
    float2 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcg(p + b + q * 32);
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = ff2_add(s[q], v[q]);
  }
#pragma unroll
  for (int q = 0; q < 7; ++q)
    if (b + q * 32 < n) s[q] = ff2_add(s[q], __ldcg(p + b + q * 32));
  return warp_sum_ff2(ff2_add(ff2_add(ff2_add(s[0], s[1]), ff2_add(s[2], s[3])),
                              ff2_add(ff2_add(s[4], s[5]), ff2_add(s[6], s[7]))));
}

}  // namespace mm
