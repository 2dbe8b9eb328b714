// Device-side helpers shared by the RP-Tuning kernels.
//
// Distances are squared Euclidean (§4.1 uses Euclidean distance for every
// dataset; squared distances order identically and avoid square roots).
//
// Exactness contract with the binary64 reading of the method:
//   uint8  : every distance is an exact integer, every decision exact.
//   float32: a distance is first computed in single precision in difference
//            form, s += (x_i - y_i)^2, and carried with a rigorous relative
//            error bound E(d) = (d + 8) * 2^-24 plus an absolute allowance for
//            gradual underflow.  When a comparison cannot be settled inside
//            that bound, both sides are recomputed in binary64 exactly as the
//            canonical reading defines them (index order, separate multiply
//            and add, round to nearest) and compared there.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rpk {

constexpr int kU8 = 1;
constexpr int kF32 = 2;
constexpr int kMaxTargets = 16;

// Status word and counters shared by all kernels of one context.
struct DevStatus {
  int code;             // 0 = fine; first error code raised wins
  int pad;
  long long info;       // first offending index / detail
  unsigned long long fp64_decisions;
  unsigned long long fp64_sort_keys;
  unsigned long long fp64_search;
  unsigned long long generic_nodes;
  unsigned long long nodes_pruned;
  unsigned long long spare[3];  // [0] self loops, [1] duplicates, [2] single-precision rechecks
};

enum DevCode : int {
  kDevOk = 0,
  kDevBadId = 1,        // an id outside [0, n) in an input graph
  kDevTieUnresolved = 2,// a near-tie run ran past the kept candidates (kNN)
  kDevOverflow = 3,     // a per-query scratch structure ran out of room
  kDevBadDegree = 4,    // a node with more candidates than its kernel handles
};

__device__ __forceinline__ void raise_status(DevStatus* st, int code, long long info) {
  if (atomicCAS(&st->code, 0, code) == 0) atomicExch(reinterpret_cast<unsigned long long*>(&st->info),
                                                     static_cast<unsigned long long>(info));
}

// ---------------------------------------------------------------------------
// canonical binary64 squared distance (float32 inputs)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double canon_d2_f32(const float* __restrict__ a,
                                               const float* __restrict__ b, int d) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) {
    double t = __dsub_rn(static_cast<double>(a[i]), static_cast<double>(b[i]));
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// Decision of the canonical reading: fl(A^2 * d2a) <= fl(1e6 * d2b).
__device__ __forceinline__ bool canon_dominates(double A2, double d2a, double d2b) {
  return __dmul_rn(A2, d2a) <= __dmul_rn(1.0e6, d2b);
}

// ---------------------------------------------------------------------------
// single-precision error model
// ---------------------------------------------------------------------------
// Relative bound for a single-precision difference-form squared distance over
// d dimensions, including the bound of the binary64 canonical value itself
// (folded in generously: (d + 8) ulps instead of (d + 2)).
__device__ __forceinline__ float rel_bound(int d) { return (float)(d + 8) * 5.9604645e-08f; }
// The same for a difference-form squared distance summed per 32-dimension
// slice (index order within a slice, then the slice sums in order):
// (min(d, 32) + ceil(d / 32) + 8) ulps.  Every single-precision distance of
// the float paths is summed this way.
__device__ __forceinline__ float slice_rel_bound(int d) {
  return float((d < 32 ? d : 32) + (d + 31) / 32 + 8) * 5.9604645e-08f;
}
// Absolute allowance for terms that underflow (at most 2^-149 each).
__device__ __forceinline__ float abs_bound(int d) { return (float)(d + 1) * 1.4012985e-45f * 4.0f; }

// Sure-ordering test for two single-precision distances carrying the bound:
// returns true only if every pair of values inside the two intervals orders
// a strictly below b.
__device__ __forceinline__ bool sure_less(float a, float b, float E, float Eabs) {
  return a * (1.0f + E) + Eabs < b * (1.0f - E) - Eabs;
}

// Domination test with three outcomes: 1 dominated for sure, 0 not dominated
// for sure, -1 undecided (recompute in binary64).  d2a = D(p*, v), d2b =
// D(p, v), A2 = A^2 as float (exact below 2^24).
__device__ __forceinline__ int sure_dominates(float A2, float d2a, float d2b, float E, float Eabs) {
  float lhs_hi = A2 * (d2a * (1.0f + E) + Eabs);
  float lhs_lo = A2 * (d2a * (1.0f - E) - Eabs);
  float rhs_hi = 1.0e6f * (d2b * (1.0f + E) + Eabs);
  float rhs_lo = 1.0e6f * (d2b * (1.0f - E) - Eabs);
  // the four products above carry one more rounding each; E has 6 ulps of slack
  if (!(isfinite(lhs_hi) && isfinite(rhs_hi))) return -1;
  if (lhs_hi < rhs_lo) return 1;
  if (lhs_lo > rhs_hi) return 0;
  return -1;
}

// ---------------------------------------------------------------------------
// float-float tier
// ---------------------------------------------------------------------------
// Float-float squared distance: each difference split exactly (two-sum), its
// square with the fused multiply-add error term, summed into a renormalised
// (high, low) pair.  |ff - d2| <= (3d + 13) 2^-48 d2 + (4d + 4) 2^-149: each
// term is off by at most 4u^2 of itself (u = 2^-24: the rounded cross term and
// the dropped low square), each step of the low sum by u^2 (3 S + 8 term), and
// the final conversion by 2^-53.  Only intrinsics (never contracted) are used.
__device__ __forceinline__ void ff_step(float x, float y, float& sh, float& sl) {
  const float th = __fsub_rn(x, y);  // two-sum of x and -y
  const float bv = __fsub_rn(th, x);
  const float tl = __fadd_rn(__fsub_rn(x, __fsub_rn(th, bv)), __fsub_rn(__fsub_rn(0.f, y), bv));
  const float ph = __fmul_rn(th, th);
  const float pl = __fmaf_rn(th, th, -ph);
  const float xt = __fmaf_rn(__fmul_rn(2.f, th), tl, pl);  // pl + 2 th tl
  const float s1 = __fadd_rn(sh, ph);                      // two-sum of sh and ph
  const float b1 = __fsub_rn(s1, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s1, b1)), __fsub_rn(ph, b1));
  const float l1 = __fadd_rn(sl, __fadd_rn(e, xt));
  sh = __fadd_rn(s1, l1);  // renormalise: |sl| <= u |sh|
  sl = __fsub_rn(l1, __fsub_rn(sh, s1));
}

// `q` may be in shared memory (plain loads); `x` is a global row.  Both are
// 16-byte aligned and zero-padded to row_bytes; a zero pair adds exactly
// nothing, so the bound for d holds over the padded length.  Used by the
// search's ordering and by the prune's decisions between the single-precision
// and the binary64 tiers.
__device__ __forceinline__ double ff_d2(const float* q, const float* __restrict__ x, int64_t row_bytes) {
  const float4* pq = reinterpret_cast<const float4*>(q);
  const float4* px = reinterpret_cast<const float4*>(x);
  float sh = 0.f, sl = 0.f;
  for (int64_t c = 0; c < row_bytes / 16; ++c) {
    const float4 a = pq[c], b = __ldg(px + c);
    ff_step(a.x, b.x, sh, sl);
    ff_step(a.y, b.y, sh, sl);
    ff_step(a.z, b.z, sh, sl);
    ff_step(a.w, b.w, sh, sl);
  }
  return __dadd_rn(double(sh), double(sl));
}

// Cached distance slots of float entries: NaN = not computed yet, sign bit
// set = a float-float value (its magnitude), else the canonical binary64 one.
// Order of two slots when their intervals allow it: 1 = a first, 0 = b first,
// -1 = undecided.  A float-float f stands for a binary64 value within
// [f (1 - E2) - A2, f (1 + E2) + A2], E2 = its bound plus the canonical sum's
// (d + 4) 2^-53 with room to spare, ends rounded outwards.
struct FFBound {
  double E2, A2;
};
__device__ __forceinline__ FFBound ff_bound(int d) {
  const double u2 = 3.552713678800501e-15;  // 2^-48
  const double u53 = 1.1102230246251565e-16;
  FFBound b;
  b.E2 = ((3.0 * d + 13.0) * u2 + (d + 4.0) * u53) * 1.01 + 4.0 * u53;
  b.A2 = (4.0 * d + 4.0) * 1.401298464324817e-45 * 2.0;
  return b;
}
__device__ __forceinline__ void slot_interval(double v, const FFBound& b, double* lo, double* hi) {
  if (signbit(v)) {
    const double f = -v;
    if (!(f <= 1.0e300)) {  // not finite: no bound (decided in binary64)
      *lo = 0.0;
      *hi = INFINITY;
      return;
    }
    *lo = __dsub_rd(__dmul_rd(f, 1.0 - b.E2), b.A2);
    *hi = __dadd_ru(__dmul_ru(f, 1.0 + b.E2), b.A2);
  } else {
    *lo = *hi = v;
  }
}
__device__ __forceinline__ int slot_order(double va, double vb, const FFBound& b) {
  double la, ha, lb, hb;
  slot_interval(va, b, &la, &ha);
  slot_interval(vb, b, &lb, &hb);
  if (ha < lb) return 1;
  if (hb < la) return 0;
  return -1;
}

// ---------------------------------------------------------------------------
// uint8 helpers
// ---------------------------------------------------------------------------
// Sum over four byte lanes of (a_i - b_i)^2, added to acc.
__device__ __forceinline__ unsigned sqdiff4_u8(unsigned a, unsigned b, unsigned acc) {
  unsigned t = __vabsdiffu4(a, b);
  return __dp4a(t, t, acc);
}

__device__ __forceinline__ unsigned long long f32_key_bits(float x) {
  return static_cast<unsigned long long>(__float_as_uint(x));
}

__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Named barrier over `count` threads (a multiple of 32) with id `id` (1..15).
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 16-byte asynchronous global -> shared copy (L2 only), zero-filling when
// src_bytes == 0.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace rpk
