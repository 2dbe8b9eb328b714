// RP-Tuning prune kernels (§3, "RP-Tuning": RobustPrune(p, N_out(p), alpha, R)
// for every node p, each reading only the input graph) and the CSR emit.
//
// Per node p with m = |N_out(p)| candidates (Algorithm 1):
//   a2 gather    each thread loads its candidate's row (and p's row) with
//                16-byte vector loads and writes it as an f16 MMA operand;
//   a3 keys      d2(p, v) for every candidate v, exactly / single precision;
//   a5 Gram      G = A A^T for the candidates on the tensor cores (tcgen05,
//                accumulator in TMEM), d2(u, v) = |u|^2 + |v|^2 - 2 G(u, v);
//   a4 sort      processing order = ascending (d2(p, v), id) -- the argmin of
//                Algorithm 1 taken in one go, ties to the smaller id -- or the
//                stored order for UnsortedRobustPrune;
//   a6 decide    for every target t and every pair u before v in that order,
//                bit "u removes v": alpha_t * D(u, v) <= D(p, v);
//   a7 scan      per target: keep the first live candidate, stop at R_t, drop
//                every candidate the kept one removes (warp ballots over
//                64-bit live masks; a6 is evaluated lazily inside this loop,
//                only for rows some target keeps);
//   a8 emit      kept ids in kept order into per-target scratch, then counts
//                -> row_ptr (scan) -> compacted col.
// Because removal is only ever done by kept points, "take the argmin of the
// live set" (Algorithm 1) and "walk the sorted order, skipping removed
// points" pick the same sequence; the bit scan is the latter.
//
// Tensor-core path: m <= 64 (two nodes per 128-thread CTA, one 128 x 128
// MMA) and 64 < m <= 128 (one node per CTA).  Larger degrees take the generic
// path (one node per 256-thread CTA, lazy CUDA-core distances).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"
#include "tc.cuh"

namespace rpk {

namespace {


struct PruneArgs {
  const uint8_t* X;
  int64_t row_bytes;
  int d;
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* nodes;
  const int32_t* count;
  unsigned int* work;
  int T;
  int variant;
  int32_t A[kMaxTargets];
  int32_t R[kMaxTargets];
  float inv_A2[kMaxTargets];  // 1 / A^2 rounded: a starting estimate for exact_threshold
  // Float rows: R only matters in the scan (a7), so targets that share alpha
  // share one domination mask.  TA distinct A values Ad[0..TA) ascending;
  // target u uses mask amap[u].
  int TA;
  int32_t Ad[kMaxTargets];
  int32_t amap[kMaxTargets];
  float kappa[kMaxTargets];   // 1e6 / Ad^2 rounded to nearest (float thresholds)
  float scale;                // float rows enter the f16 Gram as scale * x (a power of two: exact)
  float inv_s;                // 1 / scale
  float inv_s2;               // 1 / scale^2: the Gram back in the rows' units (exact)
  float sqrt_d;               // sqrt(d), rounded up
  int32_t* out_col[kMaxTargets];
  int32_t* out_cnt[kMaxTargets];
  DevStatus* status;
  const int32_t* point_of;  // row p holds the candidates of point point_of[p] (nullptr: of point p)
};

// The point whose candidates row p holds.
__device__ __forceinline__ int32_t point_of_row(const PruneArgs& a, int p) {
  return a.point_of ? a.point_of[p] : p;
}

template <int DT>
struct Acc;
template <>
struct Acc<kU8> {
  using T = unsigned;
  __device__ static __forceinline__ T step(uint2 x, uint2 y, T acc) {
    acc = sqdiff4_u8(x.x, y.x, acc);
    return sqdiff4_u8(x.y, y.y, acc);
  }
  __device__ static __forceinline__ T step4(uint4 x, uint4 y, T acc) {
    acc = sqdiff4_u8(x.x, y.x, acc);
    acc = sqdiff4_u8(x.y, y.y, acc);
    acc = sqdiff4_u8(x.z, y.z, acc);
    return sqdiff4_u8(x.w, y.w, acc);
  }
  __device__ static __forceinline__ unsigned long long bits(T v) { return v; }
  // inner product of 8 bytes (exact): the u8 Gram is built from <x, y>
  __device__ static __forceinline__ T gram(uint2 x, uint2 y, T acc) {
    return __dp4a(x.y, y.y, __dp4a(x.x, y.x, acc));
  }
  __device__ static __forceinline__ T dot4(uint4 x, uint4 y, T acc) {
    acc = __dp4a(x.x, y.x, acc);
    acc = __dp4a(x.y, y.y, acc);
    acc = __dp4a(x.z, y.z, acc);
    return __dp4a(x.w, y.w, acc);
  }
};
template <>
struct Acc<kF32> {
  using T = float;
  __device__ static __forceinline__ float sq(unsigned a, unsigned b, float acc) {
    float t = __uint_as_float(a) - __uint_as_float(b);
    return fmaf(t, t, acc);
  }
  __device__ static __forceinline__ T step(uint2 x, uint2 y, T acc) {
    acc = sq(x.x, y.x, acc);
    return sq(x.y, y.y, acc);
  }
  __device__ static __forceinline__ T step4(uint4 x, uint4 y, T acc) {
    acc = sq(x.x, y.x, acc);
    acc = sq(x.y, y.y, acc);
    acc = sq(x.z, y.z, acc);
    return sq(x.w, y.w, acc);
  }
  __device__ static __forceinline__ unsigned long long bits(T v) { return __float_as_uint(v); }
  // float Gram entries stay in difference form (rigorous relative bound)
  __device__ static __forceinline__ T gram(uint2 x, uint2 y, T acc) { return step(x, y, acc); }
  __device__ static __forceinline__ T dot4(uint4, uint4, T acc) { return acc; }
};

// Full single-precision difference-form d2 between two global rows.
// Float rows are summed per 32-dimension slice (slice_rel_bound).
template <int DT>
__device__ __forceinline__ typename Acc<DT>::T row_d2(const uint8_t* a, const uint8_t* b,
                                                       int64_t row_bytes) {
  typename Acc<DT>::T acc = 0;
  const uint4* pa = reinterpret_cast<const uint4*>(a);
  const uint4* pb = reinterpret_cast<const uint4*>(b);
  const int64_t nv = row_bytes / 16;
  for (int64_t c0 = 0; c0 < nv; c0 += 8) {
    typename Acc<DT>::T part = 0;
    for (int64_t c = c0; c < (c0 + 8 < nv ? c0 + 8 : nv); ++c) part = Acc<DT>::step4(__ldg(pa + c), __ldg(pb + c), part);
    acc += part;
  }
  return acc;
}

// The tiers past single precision for float rows.  First float-float
// distances (error (3d + 13) 2^-48 relative, ff_bound), whose intervals settle
// the canonical decision fl(A^2 d2a) <= fl(1e6 d2b) unless the two products'
// roundings could meet; only then both distances in binary64, exactly as the
// canonical reading computes them.  `key64_v` caches d2(p, v) for column v as
// the search's slots do: NaN, a float-float value (sign bit set) or the
// binary64 value.  Every writer of a slot stores a valid value of its kind.
__device__ __forceinline__ bool fine_dominates(const PruneArgs& a, int32_t u, int32_t v, int32_t p,
                                               double* key64_v, double A2) {
  const float* X = reinterpret_cast<const float*>(a.X);
  const int64_t stride = a.row_bytes / 4;
  const float* xv = X + int64_t(v) * stride;
  double sb = *key64_v;
  if (isnan(sb)) {
    sb = -ff_d2(X + int64_t(p) * stride, xv, a.row_bytes);
    *key64_v = sb;
  }
  const double fa = -ff_d2(X + int64_t(u) * stride, xv, a.row_bytes);
  const FFBound B = ff_bound(a.d);
  double la, ha, lb, hb;
  slot_interval(fa, B, &la, &ha);
  slot_interval(sb, B, &lb, &hb);
  // rounding is monotone: fl(A2 d2a) <= fl(A2 ha) and fl(1e6 lb) <= fl(1e6 d2b)
  if (__dmul_rn(A2, ha) <= __dmul_rn(1.0e6, lb)) return true;
  if (__dmul_rn(A2, la) > __dmul_rn(1.0e6, hb)) return false;
  const double d2a = canon_d2_f32(X + int64_t(u) * stride, xv, a.d);
  double d2b = sb;
  if (signbit(d2b)) {
    d2b = canon_d2_f32(X + int64_t(p) * stride, xv, a.d);
    *key64_v = d2b;
  }
  atomicAdd(&a.status->fp64_decisions, 1ull);
  return canon_dominates(A2, d2a, d2b);
}

// An open pair of the float decision pass: row `t` against column `c` for the
// distinct alphas u0 .. TA - 1 (ascending; the Gram tier found u0 of them
// surely removing).  One single-precision difference-form distance from the
// rows serves every alpha; a test inside its bound goes on to float-float and
// binary64.  Removal is monotone in alpha (removed at a larger alpha means
// removed at every smaller one), so the alphas that remove the column are a
// prefix: returns u1, the first that keeps it (TA if none), after
// recheck_tests(u0, u1, TA) tests.  Inlined into the queue's resolution
// loop; the in-place use below is out of line, since inlining it there let
// the mask loop unroll fully and the larger code ran slower.
__device__ __forceinline__ int recheck_prefix(const PruneArgs& a, const int32_t* ids, const float* key,
                                              double* key64, int t, int c, int u0, int TA, int p, float E_rel,
                                              float E_abs) {
  const float d2a = row_d2<kF32>(a.X + int64_t(ids[t]) * a.row_bytes, a.X + int64_t(ids[c]) * a.row_bytes,
                                 a.row_bytes);
  int u = u0;
  for (; u < TA; ++u) {
    const int64_t A2 = int64_t(a.Ad[u]) * a.Ad[u];
    const int rr = sure_dominates(float(A2), d2a, key[c], E_rel, E_abs);
    if (!(rr >= 0 ? (rr == 1) : fine_dominates(a, ids[t], ids[c], p, &key64[c], double(A2)))) break;
  }
  return u;
}
__device__ __forceinline__ int recheck_tests(int u0, int u1, int TA) { return u1 - u0 + (u1 < TA ? 1 : 0); }

// The same, out of line, for the rare pairs decided in place when the queue is full.
__device__ __noinline__ int recheck_prefix_cold(const PruneArgs& a, const int32_t* ids, const float* key,
                                                double* key64, int t, int c, int u0, int TA, int p, float E_rel,
                                                float E_abs) {
  return recheck_prefix(a, ids, key, key64, t, c, u0, TA, p, E_rel, E_abs);
}

// ---------------------------------------------------------------------------
// tensor-core path: the candidate Gram on tcgen05
// ---------------------------------------------------------------------------
// One CTA of 128 threads stacks the candidates of NG = 128 / MAXM nodes as the
// 128 rows of one MMA (M = N = 128): D = A A^T, A = candidates x dims in f16,
// accumulated in f32 in TMEM.  Row r of the CTA is candidate r % MAXM of node
// group r / MAXM, and TMEM lane r holds its Gram row; the diagonal MAXM x MAXM
// blocks are the nodes' Grams.
//   uint8: values 0..255 are exact in f16, products exact in f32, and every
//          partial sum is an integer below 2^24 (d <= 256), so G is exact and
//          d2(u, v) = |u|^2 + |v|^2 - 2 G(u, v) is the exact integer.
//   float: each candidate row enters centred on the pivot p, y = x - p (one
//          f32 subtraction per value, as in the pivot key's difference form),
//          scaled by a power of two into [-1, 1] and split into f16 hi and lo
//          (y = hi + 2^-11 lo up to 2^-22 relative); G~ = hi hi^T + 2^-11
//          (hi lo^T + lo hi^T) from two accumulators, with |G~ - <y_u, y_v>|
//          <= eps_ip |y_u||y_v| + 2^-36 sqrt(d) (|y_u| + |y_v|) / scale,
//          eps_ip = 5 2^-22 + 2^-23 + d 2^-22 (the subtractions, the split, the
//          dropped lo lo^T term, the last sum, f32 accumulation with a factor
//          4 allowance).  Then d2(u, v) = |y_u|^2 + |y_v|^2 - 2 <y_u, y_v>,
//          where |y|^2 = d2(p, x) is the pivot key: the bound scales with the
//          candidates' distances from p, not with their norms.  A domination
//          test whose margin is inside it is redone in single-precision
//          difference form from the rows (rigorous relative bound), and if
//          still inside, in float-float, then binary64.
// Eight float values of one row (dimensions 8c .. 8c+7 of a 128-dimension
// slice), scaled by a power of two and split into f16 hi and lo, stored at
// CTA row `orow` of the two operands (hi at opnd, lo 32 KB further) in the
// K-major core-matrix layout of tc.cuh.
__device__ __forceinline__ void store_split8(unsigned char* opnd, int orow, int c, const float (&xv)[8], float scale) {
  uint4 hi, lo;
  split_f16x2(xv[0] * scale, xv[1] * scale, hi.x, lo.x);
  split_f16x2(xv[2] * scale, xv[3] * scale, hi.y, lo.y);
  split_f16x2(xv[4] * scale, xv[5] * scale, hi.z, lo.z);
  split_f16x2(xv[6] * scale, xv[7] * scale, hi.w, lo.w);
  const size_t at = size_t(c * 16 + orow / 8) * 128 + (orow % 8) * 16;
  *reinterpret_cast<uint4*>(opnd + at) = hi;
  *reinterpret_cast<uint4*>(opnd + 128 * 128 * 2 + at) = lo;
}

// The same for a row centred on the pivot: xv - pv in f32, then scaled and split.
__device__ __forceinline__ void store_split8_centred(unsigned char* opnd, int orow, int c, const float (&xv)[8],
                                                     const float (&pv)[8], float scale) {
  float y[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) y[q] = xv[q] - pv[q];
  store_split8(opnd, orow, c, y, scale);
}

// One 128-dimension slice (kd dimensions) of the 128 x 128 candidate Gram,
// issued by one thread: hi hi^T into the accumulator at TMEM column 0 and, for
// split float rows, hi lo^T + lo hi^T into the one at column 128.
template <bool SPLIT>
__device__ __forceinline__ void issue_gram_slice(uint32_t tmem, const unsigned char* opnd, int kd, bool accumulate) {
  constexpr uint32_t idesc = umma_idesc_f16(128, 128);
#pragma unroll 1
  for (int kk = 0; kk < kd / 16; ++kk) {
    const uint64_t dsc = umma_desc(smem_addr(opnd) + uint32_t(kk) * 2u * 16u * 128u, 16u * 128u, 128u);
    umma_f16(tmem, dsc, dsc, idesc, accumulate || kk > 0);
    if constexpr (SPLIT) {  // the cross terms with the low halves into the second accumulator
      const uint64_t dlo = umma_desc(smem_addr(opnd + 128 * 128 * 2) + uint32_t(kk) * 2u * 16u * 128u, 16u * 128u, 128u);
      umma_f16(tmem + 128u, dsc, dlo, idesc, accumulate || kk > 0);
      umma_f16(tmem + 128u, dlo, dsc, idesc, true);
    }
  }
}

// A split Gram entry from its two accumulators, back in the rows' units
// (scalings by powers of two: exact).
__device__ __forceinline__ float split_gram_value(uint32_t acc0, uint32_t acc1, float inv_s2) {
  return fmaf(__uint_as_float(acc1), 4.8828125e-04f, __uint_as_float(acc0)) * inv_s2;
}

// Shared-memory plan of prune_tc_kernel.  Per node group the producer warps
// keep norms and thresholds; per pipeline slot (2) and group they hand the
// consumer warp the candidate ids, keys, binary64 key cache and masks.
template <int MAXM, int TB, int NOP>
struct TcLayout {
  static constexpr int NG = 128 / MAXM;
  static constexpr int MW = MAXM / 64;
  static constexpr size_t off_opnd = 0;  // NOP operands of 128 rows x 128 dims f16 = 32 KB each
  // per (slot, group)
  static constexpr size_t s_key64 = 0;
  static constexpr size_t s_masks = s_key64 + size_t(MAXM) * 8;  // [TB][MAXM][MW] u64
  static constexpr size_t s_ids = s_masks + size_t(TB) * MAXM * MW * 8;
  static constexpr size_t s_key = s_ids + size_t(MAXM) * 4;
  static constexpr size_t s_bytes = s_key + size_t(MAXM) * 4;
  static constexpr size_t off_slots = size_t(NOP) * 128 * 128 * 2;
  // per group, producer side
  static constexpr size_t p_norm = 0;
  static constexpr size_t p_sn = p_norm + size_t(MAXM) * 4;
  // thresholds: [TB][MAXM] for uint8; [MAXM][TB4] for float (distinct alphas of a
  // column contiguous, padded to a multiple of 4 for 16-byte reads)
  static constexpr int TB4 = (TB + 3) / 4 * 4;
  static constexpr size_t p_qlo = p_sn + size_t(MAXM) * 4;
  static constexpr size_t p_qhi = p_qlo + size_t(TB4) * MAXM * 4;
  static constexpr size_t p_sk = p_qhi + size_t(TB4) * MAXM * 4;  // [MAXM] (key, id) in stored order
  static constexpr size_t p_k64 = p_sk + size_t(MAXM) * 8;       // [MAXM] binary64 keys in stored order
  static constexpr size_t p_cq = p_k64 + size_t(MAXM) * 8;        // [MAXM] float4 per column (float rows)
  static constexpr size_t p_srt = p_cq + size_t(MAXM) * 16;       // [MAXM] float keys by rank (float rows)
  static constexpr size_t p_rk = p_srt + size_t(MAXM) * 4;        // [MAXM] rank of each stored position (float rows)
  static constexpr size_t p_bytes = p_rk + size_t(MAXM) * 4;
  static_assert(p_qlo % 16 == 0 && p_qhi % 16 == 0 && p_cq % 16 == 0 && p_rk % 16 == 0 && p_bytes % 16 == 0,
                "16-byte reads");
  static constexpr size_t off_prod = off_slots + 2 * NG * s_bytes;
  // small words: node/degree/row start per (slot, group), the claim queue's
  // head, mbarrier, TMEM address; then the claim queue (node, degree, row start)
  static constexpr size_t off_misc = off_prod + NG * p_bytes;
  static constexpr size_t q_node = 256, q_deg = q_node + 32 * 4, q_e0 = q_deg + 32 * 4;
  static constexpr size_t misc_bytes = q_e0 + 32 * 8;
  // float rows: per slot, the undecided (row, column, first alpha) entries,
  // resolved by the consumer warp before its scan of the slot
  static constexpr int rq_cap = NOP == 2 ? 1024 : 0;
  static constexpr size_t off_rq = off_misc + misc_bytes;
  static constexpr size_t bytes = (off_rq + 2 * size_t(rq_cap) * 4 + 127) & ~size_t(127);
  // float rows: a group's Gram staged in shared memory over the operands (which
  // the MMA has read by then), MAXM x MAXM floats in rank order, each row
  // rotated by its index so that a warp's accesses spread over the banks
  static_assert(NOP == 1 || size_t(NG) * MAXM * MAXM * 4 <= off_slots, "staged Gram fits over the operands");
};

// floor(1e6 k / A2) for integers, exactly: a single-precision estimate (off
// by a few units at most) corrected with 64-bit products.
__device__ __forceinline__ unsigned exact_threshold(unsigned k, unsigned long long A2, float inv_A2) {
  const unsigned long long num = 1000000ull * k;
  long long q = static_cast<long long>(floorf(1.0e6f * float(k) * inv_A2));
  if (q < 0) q = 0;
  while (static_cast<unsigned long long>(q) * A2 > num) --q;
  while (static_cast<unsigned long long>(q + 1) * A2 <= num) ++q;
  return static_cast<unsigned>(q);
}

// Nodes claimed at a time by a prune_tc_kernel CTA (one per lane of warp 0).
constexpr int kClaim = 32;

// Named barriers of prune_tc_kernel (0 is __syncthreads, unused in the loop).
constexpr int kBarProd = 1;       // the 128 producer threads
constexpr int kBarFull = 2;       // + slot: producers arrive, the consumer waits (160)
constexpr int kBarFree = 4;       // + slot: the consumer arrives, producers wait (160)

__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// Producer barrier that also ORs a flag over the 128 producer threads.
__device__ __forceinline__ bool prod_sync_or(bool flag) {
  uint32_t res;
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred p, 1, 128, p;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(res)
      : "r"(static_cast<uint32_t>(flag))
      : "memory");
  return res != 0;
}

// One CTA = 4 producer warps + 1 consumer warp.  The producers handle NG =
// 128 / MAXM nodes at a time, one candidate per thread: gather, pivot keys and
// norms, the rank of each candidate in the processing order (a4), its f16
// operand row, the tcgen05 Gram, per-column thresholds and one domination mask
// per target (uint8) or distinct alpha (float) for every rank.  uint8 operand
// rows sit at CTA row (group, rank) = TMEM lane, and each lane turns its Gram row
// into mask bits straight from TMEM.  Float operand rows stay at the stored
// position, so the MMA starts before the ranks are known; the Gram is then
// staged in shared memory in rank order and decided with the pairs spread
// evenly over the producers.  They hand ids and masks over through one of two
// slots; the consumer warp resolves the slot's open float pairs and runs the
// greedy loop per node and target (a7) while the producers work on the next
// nodes.  4 CTAs per SM (the TMEM limit) need at most 96 registers per thread;
// the kernels with more targets per launch, float rows (256 TMEM columns), or
// one 128-candidate node per MMA (more shared memory per CTA) trade that for
// registers.
template <int DT, int MAXM, int TB>
constexpr int tc_min_ctas() { return (DT == kU8 && MAXM == 64 && TB <= 4) ? 4 : 2; }

template <int DT, int MAXM, int TB>
__global__ void __launch_bounds__(160, tc_min_ctas<DT, MAXM, TB>()) prune_tc_kernel(PruneArgs a) {
  // float rows: two f16 operands (hi, lo) and two accumulators (256 TMEM columns)
  constexpr int kNop = DT == kF32 ? 2 : 1;
  constexpr uint32_t kTmemCols = DT == kF32 ? 256u : 128u;
  using L = TcLayout<MAXM, TB, kNop>;
  using AT = typename Acc<DT>::T;
  constexpr int NG = L::NG;
  constexpr int MW = L::MW;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int T = a.T;
  const int r = threadIdx.x;
  const int warp = r >> 5;
  const int lane = r & 31;
  unsigned char* opnd = smem_raw + L::off_opnd;
  int* misc = reinterpret_cast<int*>(smem_raw + L::off_misc);
  // misc ints: [0..3] slot node (s*2+g), [4..7] slot degree, [12] claim queue head
  int64_t* misc64 = reinterpret_cast<int64_t*>(smem_raw + L::off_misc + 64);  // [0..3] slot row start
  int* qnode = reinterpret_cast<int*>(smem_raw + L::off_misc + L::q_node);
  int* qdeg = reinterpret_cast<int*>(smem_raw + L::off_misc + L::q_deg);
  int64_t* qe0 = reinterpret_cast<int64_t*>(smem_raw + L::off_misc + L::q_e0);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + L::off_misc + 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + L::off_misc + 144);
  int* rq_count = misc + 14;  // [2]: per slot parity
  uint32_t* rq = reinterpret_cast<uint32_t*>(smem_raw + L::off_rq);
  auto slot_base = [&](int s, int g) { return smem_raw + L::off_slots + (size_t(s) * NG + g) * L::s_bytes; };
  const float E_rel = slice_rel_bound(a.d), E_abs = abs_bound(a.d);
  const int count = *a.count;

  if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);  // of the SM's 512 TMEM columns, for the kernel's life
  if (r == 0) {
    mbar_init(mbar, 1);
    misc[12] = kClaim;  // empty claim queue
    rq_count[0] = rq_count[1] = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp < 4) {
    // =========================== producers ===========================
    const int g = r / MAXM;
    const int t = r % MAXM;
    unsigned char* pb = smem_raw + L::off_prod + g * L::p_bytes;
    AT* norm = reinterpret_cast<AT*>(pb + L::p_norm);
    float* sn = reinterpret_cast<float*>(pb + L::p_sn);
    float* qlo = reinterpret_cast<float*>(pb + L::p_qlo);
    float* qhi = reinterpret_cast<float*>(pb + L::p_qhi);
    float4* cq = reinterpret_cast<float4*>(pb + L::p_cq);
    const uint32_t tmem = *tmem_slot;
    // operands go in as f16: uint8 values exactly, float rows centred on the
    // pivot, scaled by a power of two into [-1, 1] and split (issue_gram_slice)
    const int64_t elems = a.row_bytes / (DT == kU8 ? 1 : 4);  // padded dims per row
    const int nslices = int((elems + 127) / 128);
    // Split f16 Gram of the scaled centred rows y = x - p, G' = hi hi^T + 2^-11
    // (hi lo^T + lo hi^T): |G~ - <y_u, y_v>| <= eps_ip |y_u||y_v| + 2^-36 sqrt(d)
    // (|y_u| + |y_v|) / scale (the f32 subtractions 2^-23 relative to
    // |y_u||y_v|, the split 2^-22 per operand, the dropped lo lo^T term 2^-22,
    // the last sum 2^-23, f32 accumulation d 2^-24 with a factor 4 allowance;
    // subnormal lo).  The squared norms |y|^2 are the pivot keys, whose
    // single-precision bound is E_rel relative (+ E_abs); eps_n adds the
    // roundings that form d2 and its two bounds.
    const float eps_ip = 5.f * 2.384185791015625e-07f + 1.1920929e-07f + float(a.d) * 2.384185791015625e-07f;
    const float sub_abs = a.sqrt_d * 1.001f * 2.910383e-11f * a.inv_s;  // twice 2^-36 sqrt(d) / scale
    const float eps_n = E_rel + 6.f * 5.9604645e-08f;
    const float err_abs = 2.f * E_abs + float(a.d) * 2.3509887e-38f;  // + underflowed products, 2^-125 each
    uint32_t phase = 0;
    bool dead = false;
    unsigned long long n_rechecks = 0;  // single-precision rechecks, added to the status once at the end
    for (int k = 0;; ++k) {
      const int s = k & 1;
      named_sync(kBarFree + s, 160);  // the consumer is done with this slot
      // the consumer has resolved this slot's queue of two rounds ago: empty it
      if (DT == kF32 && r == 0) rq_count[s] = 0;
      if (warp == 0) {
        // next NG nodes from the claim queue; warp 0 refills it kClaim nodes at
        // a time (one atomic, the row bounds loaded by all lanes at once)
        int head = misc[12];
        if (head >= kClaim) {
          unsigned base = 0;
          if (lane == 0) base = atomicAdd(a.work, unsigned(kClaim));
          base = __shfl_sync(0xffffffffu, base, 0);
          const unsigned idx = base + unsigned(lane);
          const int pn = idx < unsigned(count) ? a.nodes[idx] : -1;
          int deg = 0;
          int64_t e0n = 0;
          if (pn >= 0) {
            e0n = a.row_ptr[pn];
            deg = int(a.row_ptr[pn + 1] - e0n);
          }
          if (deg > MAXM) {  // bucketing never sends such a node here; skip it, report it
            raise_status(a.status, kDevBadDegree, pn);
            deg = 0;
          }
          qnode[lane] = pn;
          qdeg[lane] = deg;
          qe0[lane] = e0n;
          __syncwarp();
          head = 0;
        }
        if (lane < NG) {
          misc[s * 2 + lane] = dead ? -1 : qnode[head + lane];
          misc[4 + s * 2 + lane] = dead ? 0 : qdeg[head + lane];
          misc64[s * 2 + lane] = qe0[head + lane];
        }
        __syncwarp();
        if (lane == 0) misc[12] = head + NG;
      }
      named_sync(kBarProd, 128);
      bool any = false;
#pragma unroll
      for (int q = 0; q < NG; ++q) any |= misc[s * 2 + q] >= 0;
      if (!any) {  // tell the consumer there is nothing more, and stop
        bar_arrive(kBarFull + s, 160);
        break;
      }
      unsigned char* sb = slot_base(s, g);
      double* key64 = reinterpret_cast<double*>(sb + L::s_key64);
      unsigned long long* masks = reinterpret_cast<unsigned long long*>(sb + L::s_masks);
      int32_t* ids = reinterpret_cast<int32_t*>(sb + L::s_ids);
      AT* key = reinterpret_cast<AT*>(sb + L::s_key);
      const int p = misc[s * 2 + g];
      const int m = misc[4 + s * 2 + g];
      const int64_t e0 = misc64[s * 2 + g];
      const bool live_row = t < m;  // thread t holds stored candidate t
      int32_t my_id = 0;
      if (live_row) my_id = a.col[e0 + t];
      // The next slot's node of this group, if the claim queue already holds it:
      // its candidate ids are loaded now and their rows prefetched into L2 while
      // this slot waits on its Gram, so the next gather finds them there.
      int32_t next_id = -1;
      {
        const int nh = misc[12] + g;
        if (nh < kClaim && t < qdeg[nh]) next_id = a.col[qe0[nh] + t];
      }
      const uint8_t* xrow = a.X + int64_t(my_id) * a.row_bytes;
      const int32_t ppt = p >= 0 ? point_of_row(a, p) : 0;  // the point being pruned
      const uint8_t* prow = a.X + int64_t(ppt) * a.row_bytes;
      // ---- a2 gather, a3 pivot key d2(p, x) and norm |x|^2 of candidate t
      AT kacc = 0, nacc = 0;
      uint4 xs[8];  // uint8, one slice: the row stays here for the operand pass
      if constexpr (DT == kU8) {
        // d2(p, x) = |p|^2 + |x|^2 - 2 <p, x>: an identity of integers, exact in
        // 32-bit modular arithmetic since d2 < 2^32; |p|^2 is summed across the warp
        unsigned dacc = 0, pacc = 0;
        for (int64_t w4 = lane; w4 < elems / 4; w4 += 32) {
          const unsigned pw = __ldg(reinterpret_cast<const unsigned*>(prow) + w4);
          pacc = __dp4a(pw, pw, pacc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pacc += __shfl_xor_sync(0xffffffffu, pacc, o);
        for (int sl = 0; sl < nslices; ++sl) {
          const int64_t rem = elems - int64_t(sl) * 128;
          const int kd = int(rem < 128 ? rem : 128);  // a multiple of 16 here
          uint4 ys[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            xs[c] = make_uint4(0, 0, 0, 0);
            ys[c] = make_uint4(0, 0, 0, 0);
            if (live_row && c < kd / 16) {
              xs[c] = __ldg(reinterpret_cast<const uint4*>(xrow + sl * 128) + c);
              ys[c] = __ldg(reinterpret_cast<const uint4*>(prow + sl * 128) + c);
            }
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            dacc = Acc<kU8>::dot4(xs[c], ys[c], dacc);
            nacc = Acc<kU8>::dot4(xs[c], xs[c], nacc);
          }
        }
        kacc = pacc + nacc - 2u * dacc;
      } else {
        // Rows of one 128-dimension slice also write their split f16 operand
        // here, at the stored position, so the row is read once.
        const bool one_slice = nslices == 1;
        if (live_row || one_slice) {
          // The key is summed per 32-dimension slice (slice_rel_bound), each
          // slice as two interleaved running sums of 16 squares added at its
          // end: a bound of 17 roundings per slice, within the 32 allowed, and
          // half the dependent chain.
          float part = 0.f, part1 = 0.f;
#pragma unroll 4
          for (int c = 0; c < int(elems / 8); ++c) {
            uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0, y0 = x0, y1 = x0;
            if (live_row) {
              const uint4* xq = reinterpret_cast<const uint4*>(xrow) + 2 * c;
              const uint4* pq = reinterpret_cast<const uint4*>(prow) + 2 * c;
              x0 = __ldg(xq);
              x1 = __ldg(xq + 1);
              y0 = __ldg(pq);
              y1 = __ldg(pq + 1);
            }
            part = Acc<kF32>::step4(x0, y0, part);
            part1 = Acc<kF32>::step4(x1, y1, part1);
            if ((c & 3) == 3 || c == int(elems / 8) - 1) {
              kacc += part + part1;
              part = part1 = 0.f;
            }
            if (one_slice) {  // rows past the degree: zeros
              const float xv[8] = {__uint_as_float(x0.x), __uint_as_float(x0.y), __uint_as_float(x0.z),
                                   __uint_as_float(x0.w), __uint_as_float(x1.x), __uint_as_float(x1.y),
                                   __uint_as_float(x1.z), __uint_as_float(x1.w)};
              const float pv[8] = {__uint_as_float(y0.x), __uint_as_float(y0.y), __uint_as_float(y0.z),
                                   __uint_as_float(y0.w), __uint_as_float(y1.x), __uint_as_float(y1.y),
                                   __uint_as_float(y1.z), __uint_as_float(y1.w)};
              store_split8_centred(opnd, g * MAXM + t, c, xv, pv, a.scale);
            }
          }
        }
      }
      // ---- a4 processing order: the rank of (d2(p, x), id) among the m
      // candidates is x's place in Algorithm 1's argmin sequence (stored order
      // for the unsorted variant).  Ids, keys, thresholds and masks below are
      // laid out by rank; uint8 operand rows too, float operand rows stay at
      // the stored position.
      unsigned long long* sk = reinterpret_cast<unsigned long long*>(pb + L::p_sk);  // stored order
      const unsigned long long my_sk = live_row ? (Acc<DT>::bits(kacc) << 32) | unsigned(my_id) : ~0ull;
      sk[t] = my_sk;
      // Float rows of one slice have their operands in place: the Gram (a5)
      // starts now and runs while the ranks are found.
      const bool early_mma = DT == kF32 && nslices == 1;
      if (early_mma) {
        fence_async_smem();
        tc_fence_before();
      }
      named_sync(kBarProd, 128);
      if (early_mma) {
        tc_fence_after();
        if (r == 0) {
          issue_gram_slice<true>(tmem, opnd, int(elems), false);
          umma_commit(mbar);
        }
      }
      int rank = t;
      // A list that Algorithm 1 wrote is already in its processing order
      // ((d2, id) ascending): then every rank is the stored position.  Checked,
      // not assumed: each candidate against the one before it (for float keys,
      // "surely less", which chains, so no two keys of the list can be near).
      bool in_order = true;
      if (a.variant == 0) {
        bool inv = false;
        if (live_row && t > 0) {
          if constexpr (DT == kU8) inv = !(sk[t - 1] < my_sk);
          else inv = !sure_less(__uint_as_float(unsigned(sk[t - 1] >> 32)), kacc, E_rel, E_abs);
        }
        in_order = !prod_sync_or(inv);
      }
      if (!in_order && live_row) {
        // entries past the degree hold ~0 and never count
        const ulonglong2* sk2 = reinterpret_cast<const ulonglong2*>(sk);
        int cnt0 = 0, cnt1 = 0;  // two sums, so the adds of successive entries overlap
#pragma unroll 4
        for (int j2 = 0; j2 < (m + 1) / 2; ++j2) {
          const ulonglong2 v = sk2[j2];
          cnt0 += int(v.x < my_sk);
          cnt1 += int(v.y < my_sk);
        }
        rank = cnt0 + cnt1;
      }
      double my64 = __longlong_as_double(0x7ff8000000000000ll);
      if constexpr (DT == kF32) {
        // single-precision keys that might be out of order (intervals overlap):
        // both ends of every such pair take a float-float key, and those pairs
        // are ordered by it; only if two float-float intervals still meet do
        // all such keys take their binary64 value (ties by id), as Algorithm 1
        // reads d2 in binary64
        // A key has a near partner iff a neighbour in single-precision order has
        // one: sure_less is monotone, so every key between two near keys is near
        // both.  The keys are laid out by rank (that order) and each thread looks
        // at its two neighbours.
        bool near = false;
        if (!in_order) {
          float* srt = reinterpret_cast<float*>(pb + L::p_srt);
          if (live_row) srt[rank] = kacc;
          named_sync(kBarProd, 128);
          if (live_row)
            near = (rank > 0 && !sure_less(srt[rank - 1], kacc, E_rel, E_abs)) ||
                   (rank + 1 < m && !sure_less(kacc, srt[rank + 1], E_rel, E_abs));
        }
        if (!in_order && prod_sync_or(near)) {
          double* k64s = reinterpret_cast<double*>(pb + L::p_k64);  // stored order
          const FFBound fb = ff_bound(a.d);
          if (near) my64 = -ff_d2(reinterpret_cast<const float*>(prow), reinterpret_cast<const float*>(xrow), a.row_bytes);
          k64s[t] = my64;
          named_sync(kBarProd, 128);
          int cnt = 0;
          bool open = false;
          if (near) {
            for (int j = 0; j < m; ++j) {
              const float kj = __uint_as_float(unsigned(sk[j] >> 32));
              if (sure_less(kj, kacc, E_rel, E_abs)) {
                ++cnt;
              } else if (j != t && !sure_less(kacc, kj, E_rel, E_abs)) {
                const int o = slot_order(k64s[j], my64, fb);  // 1: j first
                if (o < 0) open = true;
                else cnt += o;
              }
            }
          }
          if (prod_sync_or(open)) {  // every reader of k64s has passed the barrier
            if (near) {
              my64 = canon_d2_f32(reinterpret_cast<const float*>(prow), reinterpret_cast<const float*>(xrow), a.d);
              atomicAdd(&a.status->fp64_sort_keys, 1ull);
            }
            k64s[t] = my64;
            named_sync(kBarProd, 128);
            if (near) {
              cnt = 0;
              for (int j = 0; j < m; ++j) {
                const float kj = __uint_as_float(unsigned(sk[j] >> 32));
                if (sure_less(kj, kacc, E_rel, E_abs)) {
                  ++cnt;
                } else if (j != t && !sure_less(kacc, kj, E_rel, E_abs)) {
                  const double dj = k64s[j];
                  const int32_t idj = int32_t(unsigned(sk[j]));
                  cnt += (dj < my64 || (dj == my64 && idj < my_id)) ? 1 : 0;
                }
              }
            }
          }
          if (near) rank = cnt;
        }
      }
      if (live_row) {
        ids[rank] = my_id;
        key[rank] = kacc;
        if constexpr (DT == kF32) {
          // the centred rows' squared norms are the pivot keys
          norm[rank] = kacc;
          sn[rank] = sqrtf(kacc);
          key64[rank] = my64;
        } else {
          norm[rank] = nacc;
        }
      }
      if constexpr (DT == kU8) {
        // ---- f16 operand row at position rank (rows past the degree stay zero);
        // a5 Gram on tcgen05, one MMA chain per 128-dim slice
        const int orow = g * MAXM + rank;
        for (int sl = 0; sl < nslices; ++sl) {
          const int64_t rem = elems - int64_t(sl) * 128;
          const int kd = int(rem < 128 ? rem : 128);  // a multiple of 16 here
          if (nslices > 1) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              xs[c] = make_uint4(0, 0, 0, 0);
              if (live_row && c < kd / 16) xs[c] = __ldg(reinterpret_cast<const uint4*>(xrow + sl * 128) + c);
            }
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (c >= kd / 16) break;
            const uint4 x = xs[c];
            const unsigned w4[4] = {x.x, x.y, x.z, x.w};
            uint32_t o[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              o[2 * q] = u8x2_f16x2(w4[q], 0x4140u);      // bytes 0, 1
              o[2 * q + 1] = u8x2_f16x2(w4[q], 0x4342u);  // bytes 2, 3
            }
            const int kc0 = 2 * c;
            *reinterpret_cast<uint4*>(opnd + (kc0 * 16 + orow / 8) * 128 + (orow % 8) * 16) =
                make_uint4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<uint4*>(opnd + ((kc0 + 1) * 16 + orow / 8) * 128 + (orow % 8) * 16) =
                make_uint4(o[4], o[5], o[6], o[7]);
          }
          const bool last = sl == nslices - 1;
          fence_async_smem();
          tc_fence_before();
          named_sync(kBarProd, 128);
          tc_fence_after();
          if (r == 0) {
            issue_gram_slice<false>(tmem, opnd, kd, sl > 0);
            umma_commit(mbar);
          }
          if (last && live_row) {
            // while the MMA runs: the thresholds of column `rank` for every target (a6)
#pragma unroll
            for (int u = 0; u < TB; ++u) {
              if (u >= T) break;
              const unsigned long long A2 = static_cast<unsigned long long>(a.A[u]) * a.A[u];
              // v is removed by row u'  <=>  A2 d2(u', v) <= 1e6 d2(p, v)
              //   <=>  2 G(u', v) - |u'|^2 >= |v|^2 - floor(1e6 d2(p, v) / A2)
              // (every quantity an integer below 2^24, exact in f32)
              const unsigned thr = exact_threshold(kacc, A2, a.inv_A2[u]);
              qlo[u * MAXM + rank] = float(int(nacc) - int(thr));
            }
          }
          if (last && next_id >= 0) {
            const char* nrow = reinterpret_cast<const char*>(a.X + int64_t(next_id) * a.row_bytes);
            for (int64_t off = 0; off < a.row_bytes; off += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(nrow + off));
          }
          const bool ok = mbar_wait(mbar, phase, 1 << 24);
          if (prod_sync_or(!ok)) {  // the MMA never completed: report, stop after this slot (uniform)
            if (r == 0) raise_status(a.status, kDevOverflow, -2);
            dead = true;
          }
          phase ^= 1u;
          tc_fence_after();
        }

        // ---- a6: thread t turns Gram row t (TMEM lane t: the candidate of rank
        // t) into one mask per target of the ranks it would remove.
        // tcgen05.ld is warp-collective: every lane issues it, live rows use it.
        if (!dead) {
          unsigned long long mk[TB][MW];
#pragma unroll
          for (int u = 0; u < TB; ++u)
#pragma unroll
            for (int w = 0; w < MW; ++w) mk[u][w] = 0;
          const float nt = live_row ? float(norm[t]) : 0.f;
          // A row only removes candidates after it in the processing order (the
          // scan has decided every earlier one), so a warp whose rows all come
          // after a 32-column chunk skips it (a uniform choice: the TMEM read is
          // warp-collective).  Bits set for earlier columns are harmless too.
          const int first_col = 32 * (warp % (MAXM / 32));
          // Columns at or past the degree hold no candidate: the bits set there
          // can never meet a live bit in the scan, so they are not tested for.
#pragma unroll
          for (int c0 = 0; c0 < MAXM; c0 += 32) {
            if (c0 < first_col) continue;
            uint32_t v[32];
            tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + uint32_t(g * MAXM + c0), v);
            tmem_ld_wait();
            if (live_row) {
              // x = 2 G - |t|^2 lies in [-|t|^2, |c|^2], an integer below 2^24,
              // exact; q too.  x - q keeps its sign when rounded and is +0 when
              // x = q, so its sign bit is exactly "x < q": not removed.  Columns
              // go in last to first, so column c0 + j ends at bit j.
              uint32_t nb[TB];
#pragma unroll
              for (int u = 0; u < TB; ++u) nb[u] = 0u;
#pragma unroll
              for (int j4 = 28; j4 >= 0; j4 -= 4) {
                float x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) x[q] = fmaf(2.f, __uint_as_float(v[j4 + q]), -nt);
#pragma unroll
                for (int u = 0; u < TB; ++u) {
                  if (u >= T) break;
                  const float4 q4 = *reinterpret_cast<const float4*>(qlo + u * MAXM + c0 + j4);
                  nb[u] = __funnelshift_l(__float_as_uint(x[3] - q4.w), nb[u], 1);
                  nb[u] = __funnelshift_l(__float_as_uint(x[2] - q4.z), nb[u], 1);
                  nb[u] = __funnelshift_l(__float_as_uint(x[1] - q4.y), nb[u], 1);
                  nb[u] = __funnelshift_l(__float_as_uint(x[0] - q4.x), nb[u], 1);
                }
              }
#pragma unroll
              for (int u = 0; u < TB; ++u) mk[u][c0 >> 6] |= static_cast<unsigned long long>(~nb[u]) << (c0 & 63);
            }
          }
          if (live_row) {
#pragma unroll
            for (int u = 0; u < TB; ++u) {
              if (u >= T) break;
#pragma unroll
              for (int w = 0; w < MW; ++w) masks[(u * MAXM + t) * MW + w] = mk[u][w];
            }
          }
        }
        if (dead && t == 0) misc[s * 2 + g] = -1;  // nothing valid in this slot
        tc_fence_before();
        named_sync(kBarProd, 128);  // every producer's masks and TMEM reads are done
        tc_fence_after();
      } else {
        // ---- float rows: the operands stay at the stored position, so the
        // Gram is in stored order; it is staged in shared memory in rank order
        // and every pair (row before column) is decided from there, the pairs
        // spread evenly over the 128 producer threads.
        int* rank_of = reinterpret_cast<int*>(pb + L::p_rk);  // rank of each stored position
        if (live_row) rank_of[t] = rank;
        // rows of several 128-dimension slices: one MMA chain per slice, a
        // slice's operands written once the previous MMA has read its own
        for (int sl = 0; !early_mma && sl < nslices; ++sl) {
          const int64_t rem = elems - int64_t(sl) * 128;
          const int kd = int(rem < 128 ? rem : 128);  // a multiple of 16 here
          if (sl > 0) {
            const bool ok = mbar_wait(mbar, phase, 1 << 24);
            if (prod_sync_or(!ok)) {  // the MMA never completed: report, stop after this slot (uniform)
              if (r == 0) raise_status(a.status, kDevOverflow, -2);
              dead = true;
            }
            phase ^= 1u;
            tc_fence_after();
            if (dead) break;
          }
#pragma unroll 4
          for (int c = 0; c < kd / 8; ++c) {
            uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0, y0 = x0, y1 = x0;
            if (live_row) {  // rows past the degree stay zero
              const uint4* xq = reinterpret_cast<const uint4*>(xrow + int64_t(sl) * 512) + 2 * c;
              const uint4* pq = reinterpret_cast<const uint4*>(prow + int64_t(sl) * 512) + 2 * c;
              x0 = __ldg(xq);
              x1 = __ldg(xq + 1);
              y0 = __ldg(pq);
              y1 = __ldg(pq + 1);
            }
            const float xv[8] = {__uint_as_float(x0.x), __uint_as_float(x0.y), __uint_as_float(x0.z),
                                 __uint_as_float(x0.w), __uint_as_float(x1.x), __uint_as_float(x1.y),
                                 __uint_as_float(x1.z), __uint_as_float(x1.w)};
            const float pv[8] = {__uint_as_float(y0.x), __uint_as_float(y0.y), __uint_as_float(y0.z),
                                 __uint_as_float(y0.w), __uint_as_float(y1.x), __uint_as_float(y1.y),
                                 __uint_as_float(y1.z), __uint_as_float(y1.w)};
            store_split8_centred(opnd, g * MAXM + t, c, xv, pv, a.scale);
          }
          fence_async_smem();
          tc_fence_before();
          named_sync(kBarProd, 128);
          tc_fence_after();
          if (r == 0) {
            issue_gram_slice<true>(tmem, opnd, kd, sl > 0);
            umma_commit(mbar);
          }
        }
        // while the MMA runs: the thresholds of column `rank` for every distinct
        // alpha (a6).  The last factor of each (1 -+ 1e-6) covers the roundings
        // of the pair's d2 - err and d2 + err, compared against them directly.
        // a column's thresholds are TA4 = TA rounded up to 4 floats apart, so
        // that consecutive columns' 16-byte reads are consecutive
        const int TA4 = (a.TA + 3) & ~3;
        if (live_row) {
#pragma unroll
          for (int u = 0; u < TB; ++u) {
            if (u >= a.TA) break;
            // kappa = 1e6 / A^2 carries one rounding and the product two more; the
            // last factor (1 -+ 2e-6) covers them with room to spare, and the
            // roundings of the pair's d2 - err and d2 + err, compared against
            // these thresholds directly
            qlo[rank * TA4 + u] = (kacc * (1.0f - E_rel) - E_abs) * a.kappa[u] * 0.999998f;
            qhi[rank * TA4 + u] = (kacc * (1.0f + E_rel) + E_abs) * a.kappa[u] * 1.000002f;
          }
          // padding past the last alpha never counts (hi < -inf, lo > -inf)
          for (int u = a.TA; u < TA4; ++u) qlo[rank * TA4 + u] = qhi[rank * TA4 + u] = -INFINITY;
          cq[rank] = make_float4(kacc, sqrtf(kacc), 0.f, 0.f);  // the column's centred norm^2 and its root
        }
        if (next_id >= 0) {
          const char* nrow = reinterpret_cast<const char*>(a.X + int64_t(next_id) * a.row_bytes);
          for (int64_t off = 0; off < a.row_bytes; off += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(nrow + off));
        }
        // the Gram's MMA (dead is uniform; a slot that is already dead has none
        // outstanding)
        const bool waited = !dead;
        const bool ok = waited ? mbar_wait(mbar, phase, 1 << 24) : true;
        // one barrier: every rank-indexed array is complete, and the wait's outcome is known to all
        if (prod_sync_or(!ok)) {  // the MMA never completed: report, stop after this slot (uniform)
          if (r == 0) raise_status(a.status, kDevOverflow, -2);
          dead = true;
        }
        if (waited) phase ^= 1u;
        tc_fence_after();
        // The group's Gram, MAXM x MAXM in rank order over the operands (read by
        // now), row R rotated by R: G~(R, c) at [R * MAXM + (c + R) % MAXM], the
        // entries with R < c, in the operands' scaled units (G~ / inv_s2).
        // tcgen05.ld is warp-collective: every lane issues it, live rows store.
        float* Gs = reinterpret_cast<float*>(opnd) + size_t(g) * MAXM * MAXM;
        if (!dead) {
          const int cend = (m + 15) & ~15;  // the same for every lane of the warp (one node)
          const uint32_t lane_base = tmem + (uint32_t(32 * warp) << 16) + uint32_t(g * MAXM);
          float* grow = Gs + size_t(rank) * MAXM;
          const int4* rk4 = reinterpret_cast<const int4*>(rank_of);
#pragma unroll 1
          for (int c0 = 0; c0 < cend; c0 += 16) {
            uint32_t v[16], v2[16];
            tmem_ld8(lane_base + uint32_t(c0), *reinterpret_cast<uint32_t(*)[8]>(v));
            tmem_ld8(lane_base + uint32_t(c0 + 8), *reinterpret_cast<uint32_t(*)[8]>(v + 8));
            tmem_ld8(lane_base + uint32_t(128 + c0), *reinterpret_cast<uint32_t(*)[8]>(v2));
            tmem_ld8(lane_base + uint32_t(128 + c0 + 8), *reinterpret_cast<uint32_t(*)[8]>(v2 + 8));
            tmem_ld_wait();
            if (live_row) {
#pragma unroll
              for (int j4 = 0; j4 < 16; j4 += 4) {
                const int4 r4 = rk4[(c0 + j4) / 4];  // ranks of four stored columns (past m: not used)
                const int rc[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  if (c0 + j4 + j < m && rc[j] > rank)  // in the scaled units (inv_s2 goes into the decision)
                    grow[(rc[j] + rank) & (MAXM - 1)] = fmaf(__uint_as_float(v2[j4 + j]), 4.8828125e-04f,
                                                             __uint_as_float(v[j4 + j]));
              }
            }
          }
          // rank row t's masks start empty (the rows of the group, one per thread)
#pragma unroll
          for (int u = 0; u < TB; ++u) {
            if (u >= a.TA) break;
#pragma unroll
            for (int w = 0; w < MW; ++w) masks[(u * MAXM + t) * MW + w] = 0ull;
          }
        }
        tc_fence_before();
        named_sync(kBarProd, 128);  // the staged Gram, the cleared masks; TMEM read
        tc_fence_after();
        if (!dead) {
          // Rows pair up as (q, MAXM - 1 - q): row q has MAXM - 1 - q later
          // columns and row MAXM - 1 - q has q, MAXM - 1 in all, and the two
          // threads of a pair take half each.  Thread h = 0 takes row q's first
          // Q columns; thread h = 1 the rest of row q, then row MAXM - 1 - q.
          // Item k of a thread is one (row, column) pair.
          constexpr int Q = MAXM / 2;
          const int q = t % Q, h = t / Q;
          const int rA = q, rB = MAXM - 1 - q;
          const int nItems = h == 0 ? Q : Q - 1;
          const int nA = h == 0 ? Q : Q - 1 - q;        // items on row rA, the rest on row rB
          const int cA = h == 0 ? rA + 1 : rA + Q + 1;  // row rA's first column
          const int cB = rB + 1;                         // row rB's first column
          // the d2 error bound as two multiply-adds: err = |c| At + |c|^2 eps_n + Bt
          const float ntA = rA < m ? float(norm[rA]) : 0.f, stA = rA < m ? sn[rA] : 0.f;
          const float ntB = rB < m ? float(norm[rB]) : 0.f, stB = rB < m ? sn[rB] : 0.f;
          const float AtA = 2.f * eps_ip * stA * 1.0009765625f + sub_abs, BtA = sub_abs * stA + eps_n * ntA + err_abs;
          const float AtB = 2.f * eps_ip * stB * 1.0009765625f + sub_abs, BtB = sub_abs * stB + eps_n * ntB + err_abs;
          const int TA = a.TA;
          const float m2inv_s2 = -2.f * a.inv_s2;
          const float4* ql4 = reinterpret_cast<const float4*>(qlo);
          const float4* qh4 = reinterpret_cast<const float4*>(qhi);
          // Per distinct alpha u, bit k of mk[u] says that item k's column is
          // surely removed at alpha u: hi < qlo(column, u).  Those tests are a
          // prefix over u (the alphas ascend, the thresholds fall), so they are
          // the row masks' bits as they stand.  "May be removed", !(lo >
          // qhi(column, u)), is a prefix too; an item is open when some alpha may
          // remove its column without surely doing so.
          using IW = typename std::conditional<(Q <= 32), unsigned, unsigned long long>::type;
          IW mk[TB], open = 0;
#pragma unroll
          for (int u = 0; u < TB; ++u) mk[u] = 0;
          // straight-line items (the open ones are only marked), so that the
          // reads of several items overlap
#pragma unroll 2
          for (int k = 0; k < Q; ++k) {
            const bool onA = k < nA;
            const int R = onA ? rA : rB;
            const int c = onA ? cA + k : cB + (k - nA);
            const bool valid = k < nItems && c < m;  // c > R, so the row is live too
            const int ci = valid ? c : 0;            // the reads stay in range for every k
            const float G = Gs[R * MAXM + ((ci + R) & (MAXM - 1))];
            const float4 qc = cq[ci];
            const float dv = fmaf(G, m2inv_s2, (onA ? ntA : ntB) + qc.x);  // G~ = G * inv_s2: exact scaling
            const float err = fmaf(qc.y, onA ? AtA : AtB, fmaf(qc.x, eps_n, onA ? BtA : BtB));
            const float lo = dv - err, hi = dv + err;
            bool op = false;
#pragma unroll
            for (int u4 = 0; u4 < L::TB4; u4 += 4) {
              if (u4 < TA) {  // uniform
                const float4 l4 = ql4[(ci * TA4 + u4) / 4];
                const float4 h4 = qh4[(ci * TA4 + u4) / 4];
                const float lv[4] = {l4.x, l4.y, l4.z, l4.w}, hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  if (u4 + e >= TB) break;
                  const bool sure = valid && hi < lv[e];  // padding past TA: -inf, never
                  if (sure) mk[u4 + e] |= IW(1) << k;
                  op |= valid && !sure && !(lo > hv[e]);
                }
              }
            }
            if (op) open |= IW(1) << k;
          }
          // open pairs (rare): the alphas from ts (the surely-removing count) on
          // are decided exactly by the consumer warp before its scan; here if the
          // slot's queue is full
          while (open) {
            const int k = int(__ffsll(static_cast<long long>(open))) - 1;
            open &= open - 1;
            const bool onA = k < nA;
            const int R = onA ? rA : rB;
            const int c = onA ? cA + k : cB + (k - nA);
            int ts = 0;
#pragma unroll
            for (int u = 0; u < TB; ++u) ts += int((mk[u] >> k) & 1u);
            const int qi = atomicAdd(rq_count + s, 1);
            if (qi < L::rq_cap) {
              rq[s * L::rq_cap + qi] = (unsigned(g * MAXM + R) << 16) | (unsigned(c) << 5) | unsigned(ts);
            } else {
              // removal is monotone in alpha: the alphas before the first that keeps the pair remove it
              const int u1 = recheck_prefix_cold(a, ids, key, key64, R, c, ts, TA, ppt, E_rel, E_abs);
              n_rechecks += recheck_tests(ts, u1, TA);
#pragma unroll
              for (int u = 0; u < TB; ++u)
                if (u >= ts && u < u1) mk[u] |= IW(1) << k;
            }
          }
          // item masks -> row masks: row rA's items are [0, nA) from column cA,
          // row rB's [nA, nItems) from column cB
          auto or_run = [&](unsigned long long* row, unsigned long long bits, int col) {
            const int w0 = col >> 6, sh = col & 63;
            if (bits << sh) atomicOr(row + w0, bits << sh);
            if (MW > 1 && sh && w0 + 1 < MW && (bits >> (64 - sh))) atomicOr(row + w0 + 1, bits >> (64 - sh));
          };
#pragma unroll
          for (int u = 0; u < TB; ++u) {
            if (u >= TA) break;
            const unsigned long long gt = mk[u];
            const unsigned long long mA = nA >= 64 ? gt : (gt & ((1ull << nA) - 1));
            const unsigned long long mB = nA >= 64 ? 0ull : (gt >> nA);
            if (mA) or_run(masks + (u * MAXM + rA) * MW, mA, cA);
            if (mB) or_run(masks + (u * MAXM + rB) * MW, mB, cB);
          }
        }
        if (dead && t == 0) misc[s * 2 + g] = -1;  // nothing valid in this slot
      }
      bar_arrive(kBarFull + s, 160);
    }
    if constexpr (DT == kF32) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n_rechecks += __shfl_xor_sync(0xffffffffu, n_rechecks, o);
      if (lane == 0 && n_rechecks) atomicAdd(&a.status->spare[2], n_rechecks);
    }
  } else {
    // =========================== consumer warp ===========================
    bar_arrive(kBarFree + 0, 160);  // both slots start free
    bar_arrive(kBarFree + 1, 160);
    long long done = 0;
    unsigned long long n_rechecks = 0;  // single-precision rechecks of the queued pairs
    for (int k = 0;; ++k) {
      const int s = k & 1;
      named_sync(kBarFull + s, 160);
      bool any = false;
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        any |= misc[s * 2 + q] >= 0;
        done += misc[s * 2 + q] >= 0;
      }
      if (!any) break;
      if constexpr (DT == kF32) {
        // the slot's open pairs, one per lane: each alpha that removes the
        // column sets its bit in the row's mask for that alpha
        const int nq = min(rq_count[s], L::rq_cap);
        for (int i = lane; i < nq; i += 32) {
          const uint32_t e = rq[s * L::rq_cap + i];
          const int tr = int(e >> 16), c = int((e >> 5) & 0x7ffu), u0 = int(e & 31u);
          const int gq = tr / MAXM, tq = tr % MAXM;
          unsigned char* sbq = slot_base(s, gq);
          const int u1 = recheck_prefix(a, reinterpret_cast<const int32_t*>(sbq + L::s_ids),
                                        reinterpret_cast<const float*>(sbq + L::s_key),
                                        reinterpret_cast<double*>(sbq + L::s_key64), tq, c, u0, a.TA,
                                        point_of_row(a, misc[s * 2 + gq]), E_rel, E_abs);
          n_rechecks += recheck_tests(u0, u1, a.TA);
          unsigned long long* mrow = reinterpret_cast<unsigned long long*>(sbq + L::s_masks) + tq * MW + (c >> 6);
          for (int u = u0; u < u1; ++u) atomicOr(mrow + u * MAXM * MW, 1ull << (c & 63));
        }
        __syncwarp();
      }
      // ---- a7 greedy scan: lane (g * 16 + u) runs Algorithm 1's loop for node
      // g and target u.  Candidates are laid out by rank, so the next argmin of
      // the live set is its lowest set bit.
      {
        const int g = NG == 2 ? lane >> 4 : 0;
        const int u = NG == 2 ? (lane & 15) : lane;
        const int p = misc[s * 2 + g];
        if (p >= 0 && u < T) {
          const int m = misc[4 + s * 2 + g];
          const int64_t e0 = misc64[s * 2 + g];
          unsigned char* sb = slot_base(s, g);
          const unsigned long long* masks = reinterpret_cast<const unsigned long long*>(sb + L::s_masks);
          const int32_t* ids = reinterpret_cast<const int32_t*>(sb + L::s_ids);
          unsigned long long al[MW];
#pragma unroll
          for (int w = 0; w < MW; ++w) {
            const int lo = 64 * w;
            al[w] = m > lo ? ((m - lo >= 64) ? ~0ull : ((1ull << (m - lo)) - 1)) : 0ull;
          }
          const int R = a.R[u];
          const int mu = DT == kF32 ? a.amap[u] : u;  // the target's domination mask
          int32_t* out = a.out_col[u] + e0;
          int kept = 0;
          if constexpr (MW == 1) {
            // Two steps per round: the mask of the next live candidate is read
            // together with that of the one after it, which is the next argmin
            // too unless the first removes it (then the round takes one step).
            unsigned long long live = al[0];
            const unsigned long long* mrow = masks + mu * MAXM;
            while (kept < R && live) {
              const int p1 = __ffsll(static_cast<long long>(live)) - 1;
              const unsigned long long rest = live & (live - 1);  // live without p1
              const int p2 = rest ? __ffsll(static_cast<long long>(rest)) - 1 : p1;
              const unsigned long long m1 = mrow[p1], m2 = mrow[p2];
              out[kept++] = ids[p1];
              live = rest & ~m1;
              if (kept < R && ((live >> p2) & 1ull)) {  // p2 outlived p1: the next argmin
                out[kept++] = ids[p2];
                live &= ~(m2 | (1ull << p2));
              }
            }
          }
          while (MW > 1 && kept < R) {
            int pos = -1;
#pragma unroll
            for (int w = MW - 1; w >= 0; --w)
              if (al[w]) pos = 64 * w + __ffsll(static_cast<long long>(al[w])) - 1;
            if (pos < 0) break;
            out[kept++] = ids[pos];
            const unsigned long long pb = 1ull << (pos & 63);
            if (MW == 1 || pos < 64) al[0] &= ~pb;  // taken (its own mask bit is set too)
            else al[MW - 1] &= ~pb;
#pragma unroll
            for (int q = 0; q < MW; ++q) al[q] &= ~masks[(mu * MAXM + pos) * MW + q];
          }
          a.out_cnt[u][p] = kept;
        }
      }
      __syncwarp();
      bar_arrive(kBarFree + s, 160);
    }
    if (lane == 0 && done) atomicAdd(&a.status->nodes_pruned, static_cast<unsigned long long>(done) * T);
    if constexpr (DT == kF32) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n_rechecks += __shfl_xor_sync(0xffffffffu, n_rechecks, o);
      if (lane == 0 && n_rechecks) atomicAdd(&a.status->spare[2], n_rechecks);
    }
  }
  // the TMEM columns go back once the producers are finished with them
  if (warp < 4) {
    tc_fence_before();
    named_sync(kBarProd, 128);
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tmem_slot, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// generic path: one node per CTA, any degree up to RP_MAX_DEGREE
// ---------------------------------------------------------------------------
struct GenericLayout {
  // sort keys and, once sorted, the binary64 pivot-key cache share one array
  __host__ __device__ static size_t bytes(int M2) { return size_t(M2) * 22 + 64; }
};

template <int DT>
__global__ void __launch_bounds__(256) prune_generic_kernel(PruneArgs a, int M2) {
  using AT = typename Acc<DT>::T;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(smem_raw);
  double* key64 = reinterpret_cast<double*>(smem_raw);  // valid after the sort
  int32_t* ids = reinterpret_cast<int32_t*>(smem_raw + size_t(M2) * 8);
  int32_t* perm = reinterpret_cast<int32_t*>(smem_raw + size_t(M2) * 12);
  AT* key = reinterpret_cast<AT*>(smem_raw + size_t(M2) * 16);
  unsigned char* alive = smem_raw + size_t(M2) * 20;
  unsigned char* lnk = smem_raw + size_t(M2) * 21;
  int* misc = reinterpret_cast<int*>(smem_raw + size_t(M2) * 22);
  const int t = threadIdx.x, NT = blockDim.x;
  const int count = *a.count;
  const float E = rel_bound(a.d), Eabs = abs_bound(a.d);
  long long done = 0;

  for (;;) {
    if (t == 0) {
      unsigned idx = atomicAdd(a.work, 1u);
      misc[0] = idx < unsigned(count) ? a.nodes[idx] : -1;
      misc[2] = 0;
    }
    __syncthreads();
    const int p = misc[0];
    if (p < 0) break;
    const int64_t e0 = a.row_ptr[p];
    const int m = int(a.row_ptr[p + 1] - e0);
    if (m > M2) {  // bucketing guarantees m <= M2; keep the kernel safe regardless
      if (t == 0) raise_status(a.status, kDevBadDegree, p);
      __syncthreads();
      continue;
    }
    const int32_t ppt = point_of_row(a, p);  // the point being pruned
    const uint8_t* xp = a.X + int64_t(ppt) * a.row_bytes;
    // this node's sort width: the smallest power of two >= m (M2 is the launch's
    // largest, sized for its longest list; the others sort no more than their own)
    int Mp = 1;
    while (Mp < m) Mp <<= 1;
    for (int j = t; j < Mp; j += NT) {
      if (j < m) {
        const int32_t v = a.col[e0 + j];
        ids[j] = v;
        const AT kv = row_d2<DT>(xp, a.X + int64_t(v) * a.row_bytes, a.row_bytes);
        key[j] = kv;
        skey[j] = a.variant == 0 ? (Acc<DT>::bits(kv) << 32) | unsigned(v) : (unsigned long long)j;
      } else {
        skey[j] = ~0ull;
      }
      perm[j] = j;
    }
    __syncthreads();
    if (a.variant == 0) {
      for (int k = 2; k <= Mp; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int idx = t; idx < Mp / 2; idx += NT) {
            const int i = (idx / j) * 2 * j + (idx % j);
            const int l = i + j;
            const bool up = (i & k) == 0;
            const unsigned long long x = skey[i], y = skey[l];
            if ((x > y) == up) {
              skey[i] = y;
              skey[l] = x;
              const int tmp = perm[i];
              perm[i] = perm[l];
              perm[l] = tmp;
            }
          }
          __syncthreads();
        }
      }
      for (int j = t; j < Mp; j += NT) key64[j] = __longlong_as_double(0x7ff8000000000000ll);
      __syncthreads();
      if constexpr (DT == kF32) {
        for (int i = t; i < m; i += NT) {
          lnk[i] = 0;
          if (i + 1 < m && !sure_less(key[perm[i]], key[perm[i + 1]], E, Eabs)) {
            lnk[i] = 1;
            misc[2] = 1;
          }
        }
        __syncthreads();
        if (misc[2]) {
          const float* X = reinterpret_cast<const float*>(a.X);
          const int64_t stride = a.row_bytes / 4;
          for (int i = t; i < m; i += NT) {
            if (lnk[i] || (i > 0 && lnk[i - 1])) {
              key64[perm[i]] = canon_d2_f32(X + int64_t(ppt) * stride, X + int64_t(ids[perm[i]]) * stride, a.d);
              atomicAdd(&a.status->fp64_sort_keys, 1ull);
            }
          }
          __syncthreads();
          for (int s0 = t; s0 < m; s0 += NT) {
            const bool head = (lnk[s0] || (s0 > 0 && lnk[s0 - 1])) && !(s0 > 0 && lnk[s0 - 1]);
            if (!head) continue;
            int end = s0;
            while (end + 1 < m && lnk[end]) ++end;
            for (int i = s0 + 1; i <= end; ++i) {
              const int v = perm[i];
              int j = i - 1;
              while (j >= s0 && (key64[perm[j]] > key64[v] ||
                                 (key64[perm[j]] == key64[v] && ids[perm[j]] > ids[v]))) {
                perm[j + 1] = perm[j];
                --j;
              }
              perm[j + 1] = v;
            }
          }
        }
      }
    } else {
      for (int j = t; j < Mp; j += NT) key64[j] = __longlong_as_double(0x7ff8000000000000ll);
    }
    __syncthreads();

    for (int tt = 0; tt < a.T; ++tt) {
      const int64_t A2 = int64_t(a.A[tt]) * a.A[tt];
      const int R = a.R[tt];
      int32_t* out = a.out_col[tt] + e0;
      for (int j = t; j < m; j += NT) alive[j] = 1;
      if (t == 0) misc[1] = 0;  // cursor
      __syncthreads();
      int kept = 0;
      for (;;) {
        if (t == 0) {
          int c = misc[1];
          while (c < m && !alive[c]) ++c;
          misc[1] = c;
          misc[3] = c;
          if (c < m) {
            out[kept] = ids[perm[c]];
            alive[c] = 0;
          }
        }
        __syncthreads();
        const int i = misc[3];
        if (i >= m) break;
        ++kept;
        if (kept == R) break;
        const int32_t ui = ids[perm[i]];
        const uint8_t* xu = a.X + int64_t(ui) * a.row_bytes;
        for (int j = i + 1 + t; j < m; j += NT) {
          if (!alive[j]) continue;
          const int pj = perm[j];
          const AT d2a = row_d2<DT>(xu, a.X + int64_t(ids[pj]) * a.row_bytes, a.row_bytes);
          bool dom;
          if constexpr (DT == kU8) {
            dom = static_cast<unsigned long long>(A2) * d2a <= 1000000ull * static_cast<unsigned long long>(key[pj]);
          } else {
            const int r = sure_dominates(float(A2), d2a, key[pj], E, Eabs);
            dom = r >= 0 ? (r == 1) : fine_dominates(a, ui, ids[pj], ppt, &key64[pj], double(A2));
          }
          if (dom) alive[j] = 0;
        }
        __syncthreads();
      }
      if (t == 0) a.out_cnt[tt][p] = kept;
      __syncthreads();
    }
    ++done;
  }
  if (t == 0 && done) {
    atomicAdd(&a.status->nodes_pruned, static_cast<unsigned long long>(done) * a.T);
    atomicAdd(&a.status->generic_nodes, static_cast<unsigned long long>(done));
  }
}

__global__ void bucket_nodes_kernel(const int64_t* __restrict__ row_ptr, int64_t n,
                                    int32_t* __restrict__ lists, int32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = base + threadIdx.x;
    const bool valid = p < n;
    int b = -1;
    if (valid) {
      const int64_t deg = row_ptr[p + 1] - row_ptr[p];
      b = deg <= 64 ? 0 : (deg <= 128 ? 1 : 2);
    }
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      const unsigned msk = __ballot_sync(0xffffffffu, b == bb);
      if (!msk) continue;
      const int leader = __ffs(msk) - 1;
      int off = 0;
      if (lane == leader) off = atomicAdd(&counts[bb], __popc(msk));
      off = __shfl_sync(0xffffffffu, off, leader);
      if (b == bb) lists[int64_t(bb) * n + off + __popc(msk & ((1u << lane) - 1))] = int32_t(p);
    }
  }
}

// ---------------------------------------------------------------------------
// counts -> row_ptr -> compacted col (a8)
// ---------------------------------------------------------------------------
constexpr int kScanChunk = 4096;  // nodes per block
constexpr int kScanThreads = 256;
constexpr int kPerThread = kScanChunk / kScanThreads;

struct EmitArgs {
  int64_t n;
  int64_t nblk;
  const int64_t* src_row_ptr;
  int32_t* scratch[kMaxTargets];
  int32_t* cnt[kMaxTargets];
  int64_t* dst_row_ptr[kMaxTargets];
  int32_t* dst_col[kMaxTargets];
  int64_t* bsum;
};

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* warp_tot, int64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < int(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < int(blockDim.x >> 5)) warp_tot[lane] = s;  // inclusive per warp
    if (lane == int(blockDim.x >> 5) - 1) *total = s;
  }
  __syncthreads();
  const int64_t before = w > 0 ? warp_tot[w - 1] : 0;
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) emit_block_sums(EmitArgs e) {
  const int tt = blockIdx.y;
  const int64_t b0 = int64_t(blockIdx.x) * kScanChunk;
  int64_t s = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += kScanThreads) {
    const int64_t p = b0 + i;
    if (p < e.n) s += e.cnt[tt][p];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ int64_t ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t tot = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) tot += ws[w];
    e.bsum[int64_t(tt) * e.nblk + blockIdx.x] = tot;
  }
}

__global__ void __launch_bounds__(1024) emit_scan_sums(EmitArgs e) {
  const int tt = blockIdx.x;
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t total;
  int64_t carry = 0;
  for (int64_t base = 0; base < e.nblk; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < e.nblk ? e.bsum[int64_t(tt) * e.nblk + i] : 0;
    const int64_t ex = block_excl_scan(v, warp_tot, &total);
    if (i < e.nblk) e.bsum[int64_t(tt) * e.nblk + i] = carry + ex;
    carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) emit_write(EmitArgs e) {
  const int tt = blockIdx.y;
  const int64_t b0 = int64_t(blockIdx.x) * kScanChunk;
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t total;
  __shared__ int64_t off[kScanChunk];
  int local[kPerThread];
  int64_t mine = 0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const int64_t p = b0 + int64_t(threadIdx.x) * kPerThread + i;
    local[i] = p < e.n ? e.cnt[tt][p] : 0;
    mine += local[i];
  }
  int64_t run = block_excl_scan(mine, warp_tot, &total) + e.bsum[int64_t(tt) * e.nblk + blockIdx.x];
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const int li = threadIdx.x * kPerThread + i;
    const int64_t p = b0 + li;
    off[li] = run;
    run += local[i];
    if (p < e.n) e.dst_row_ptr[tt][p + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) e.dst_row_ptr[tt][0] = 0;
  __syncthreads();
  if (e.dst_col[tt] == nullptr) return;
  // A warp takes 32 consecutive rows: their counts and offsets in one coalesced
  // load, then the rows' ids four rows at a time (independent loads in flight).
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t* scr = e.scratch[tt];
  int32_t* dcol = e.dst_col[tt];
  for (int base = w * 32; base < kScanChunk; base += kScanThreads) {
    const int64_t p = b0 + base + lane;
    const bool valid = p < e.n;
    const int c_l = valid ? e.cnt[tt][p] : 0;
    const int64_t s_l = valid ? e.src_row_ptr[p] : 0;
    const int64_t o_l = off[base + lane];
    for (int r0 = 0; r0 < 32; r0 += 4) {
      int c[4];
      int64_t so[4], dof[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        c[q] = __shfl_sync(0xffffffffu, c_l, r0 + q);
        so[q] = __shfl_sync(0xffffffffu, s_l, r0 + q);
        dof[q] = __shfl_sync(0xffffffffu, o_l, r0 + q);
      }
      const int cmax = max(max(c[0], c[1]), max(c[2], c[3]));
      for (int j = lane; j < cmax; j += 32) {
        int32_t v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j < c[q]) v[q] = scr[so[q] + j];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j < c[q]) dcol[dof[q] + j] = v[q];
      }
    }
  }
}

}  // namespace

int64_t emit_csr_blocks(int64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

cudaError_t launch_emit_csr(int64_t n, int T, const int64_t* src_row_ptr, int32_t* const* scratch_col,
                            int32_t* const* cnt, int64_t* const* dst_row_ptr, int32_t* const* dst_col,
                            int64_t* block_sums, cudaStream_t s) {
  EmitArgs e{};
  e.n = n;
  e.nblk = emit_csr_blocks(n);
  e.src_row_ptr = src_row_ptr;
  e.bsum = block_sums;
  for (int t = 0; t < T; ++t) {
    e.scratch[t] = scratch_col ? scratch_col[t] : nullptr;
    e.cnt[t] = cnt[t];
    e.dst_row_ptr[t] = dst_row_ptr[t];
    e.dst_col[t] = dst_col ? dst_col[t] : nullptr;
  }
  const dim3 grid(unsigned(e.nblk), unsigned(T));
  emit_block_sums<<<grid, kScanThreads, 0, s>>>(e);
  emit_scan_sums<<<T, 1024, 0, s>>>(e);
  emit_write<<<grid, kScanThreads, 0, s>>>(e);
  return cudaGetLastError();
}

cudaError_t launch_bucket_nodes(const int64_t* row_ptr, int64_t n, int32_t* lists, int32_t* counts,
                                cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(counts, 0, 3 * sizeof(int32_t), s);
  if (err != cudaSuccess) return err;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 65535 * 4);
  bucket_nodes_kernel<<<unsigned(std::max<int64_t>(blocks, 1)), 256, 0, s>>>(row_ptr, n, lists, counts);
  return cudaGetLastError();
}

// CTAs of `kern` that fit on one SM, from its registers and dynamic shared
// memory (computed directly: the occupancy query under-reports it for these
// kernels when called while a stream is being captured).
template <typename K>
static cudaError_t resident_ctas(K kern, int threads, size_t dyn_smem, int cap, int* out) {
  cudaFuncAttributes fa;
  cudaError_t err = cudaFuncGetAttributes(&fa, kern);
  if (err != cudaSuccess) return err;
  int dev = 0, smem_sm = 0, regs_sm = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return err;
  if ((err = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess)
    return err;
  const size_t per_cta_smem = dyn_smem + fa.sharedSizeBytes + 1024;  // 1 KB reserved per CTA
  const int regs_per_warp = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;
  const int by_smem = int(size_t(smem_sm) / per_cta_smem);
  const int by_regs = regs_sm / (regs_per_warp * ((threads + 31) / 32));
  *out = std::max(1, std::min({cap, by_smem, by_regs}));
  return cudaSuccess;
}

template <int DT, int MAXM, int TB>
static cudaError_t run_fast_t(const PruneArgs& args, int num_sms, int64_t host_count, int ctas_cap, cudaStream_t s) {
  const size_t bytes = TcLayout<MAXM, TB, DT == kF32 ? 2 : 1>::bytes;
  auto kern = prune_tc_kernel<DT, MAXM, TB>;
  constexpr int kThreadsTc = 160;  // 4 producer warps + 1 consumer warp
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (err != cudaSuccess) return err;
  // ask for the largest shared-memory carveout so the launch sees the whole 228 KB per SM
  err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  // 128 (uint8) or 256 (float) of the SM's 512 TMEM columns per CTA
  err = resident_ctas(kern, kThreadsTc, bytes, DT == kF32 ? 2 : 4, &per_sm);
  if (err != cudaSuccess) return err;
  if (ctas_cap > 0) per_sm = std::min(per_sm, ctas_cap);
  const int64_t groups_needed = (host_count + (128 / MAXM) - 1) / (128 / MAXM);
  const int64_t grid = std::min<int64_t>(int64_t(num_sms) * per_sm, groups_needed);
  kern<<<unsigned(grid), kThreadsTc, bytes, s>>>(args);
  return cudaGetLastError();
}

// Picks the kernel instance whose per-node target slots cover T.
template <int DT, int MAXM>
static cudaError_t run_fast(const PruneArgs& args, int num_sms, int64_t host_count, int ctas_cap, cudaStream_t s) {
  if (host_count <= 0) return cudaSuccess;
  // TB bounds what the kernel keeps per target: one mask and threshold set per
  // target for uint8 rows, per distinct alpha for float rows (targets sharing
  // alpha share them; the consumer's lanes cover every target either way)
  const int nb = DT == kF32 ? args.TA : args.T;
  if (nb <= 1) return run_fast_t<DT, MAXM, 1>(args, num_sms, host_count, ctas_cap, s);
  if (nb <= 2) return run_fast_t<DT, MAXM, 2>(args, num_sms, host_count, ctas_cap, s);
  if (nb <= 4) return run_fast_t<DT, MAXM, 4>(args, num_sms, host_count, ctas_cap, s);
  if (nb <= 8) return run_fast_t<DT, MAXM, 8>(args, num_sms, host_count, ctas_cap, s);
  return run_fast_t<DT, MAXM, kMaxTargets>(args, num_sms, host_count, ctas_cap, s);
}

template <int DT>
static cudaError_t run_generic(const PruneArgs& args, int num_sms, int64_t host_count, int max_degree,
                               cudaStream_t s) {
  if (host_count <= 0) return cudaSuccess;
  int M2 = 256;
  while (M2 < max_degree) M2 <<= 1;
  const size_t bytes = GenericLayout::bytes(M2);
  auto kern = prune_generic_kernel<DT>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = resident_ctas(kern, 256, bytes, 8, &per_sm);
  if (err != cudaSuccess) return err;
  const int64_t grid = std::min<int64_t>(int64_t(num_sms) * per_sm, host_count);
  kern<<<unsigned(grid), 256, bytes, s>>>(args, M2);
  return cudaGetLastError();
}

namespace {

// Test support: the split-f16 tcgen05 Gram of 128 float rows per CTA, through
// the prune kernel's own operand stores, MMA sequence and combination, written
// out so that a test can hold every entry against the exact inner product and
// the bound the float decision tiers rely on.  With `centres`, each 64-row half
// of a group enters centred on its own pivot row, as the prune's nodes do.
__global__ void __launch_bounds__(128, 1) gram_probe_kernel(const uint8_t* X, int64_t row_bytes, float scale,
                                                           float inv_s2, const int32_t* rows, const int32_t* centres,
                                                           int64_t groups, float* out, DevStatus* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* opnd = smem_raw;  // hi and lo operands: 2 x 128 rows x 128 dims of f16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + 2 * 128 * 128 * 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + 2 * 128 * 128 * 2 + 16);
  const int r = threadIdx.x, warp = r >> 5;
  if (warp == 0) tmem_alloc(tmem_slot, 256u);
  if (r == 0) mbar_init(mbar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t elems = row_bytes / 4;
  const int nslices = int((elems + 127) / 128);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t gi = blockIdx.x; gi < groups && ok; gi += gridDim.x) {
    const float* xr = reinterpret_cast<const float*>(X + int64_t(rows[gi * 128 + r]) * row_bytes);
    const float* pr = centres ? reinterpret_cast<const float*>(X + int64_t(centres[gi * 2 + r / 64]) * row_bytes)
                              : nullptr;
    for (int sl = 0; sl < nslices && ok; ++sl) {
      const int64_t rem = elems - int64_t(sl) * 128;
      const int kd = int(rem < 128 ? rem : 128);
      for (int c = 0; c < kd / 8; ++c) {
        float xv[8], pv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          xv[q] = xr[int64_t(sl) * 128 + c * 8 + q];
          pv[q] = pr ? pr[int64_t(sl) * 128 + c * 8 + q] : 0.f;
        }
        store_split8_centred(opnd, r, c, xv, pv, scale);
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (r == 0) {
        issue_gram_slice<true>(tmem, opnd, kd, sl > 0);
        umma_commit(mbar);
      }
      ok = mbar_wait(mbar, phase, 1 << 24);
      phase ^= 1u;
      tc_fence_after();
      if (!__syncthreads_and(ok)) {
        if (r == 0) raise_status(status, kDevOverflow, -3);
        ok = false;
      }
    }
    if (!ok) break;
    for (int c0 = 0; c0 < 128; c0 += 8) {
      uint32_t v[8], v2[8];
      tmem_ld8(tmem + (uint32_t(32 * warp) << 16) + uint32_t(c0), v);
      tmem_ld8(tmem + (uint32_t(32 * warp) << 16) + uint32_t(128 + c0), v2);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 8; ++j) out[(gi * 128 + r) * 128 + c0 + j] = split_gram_value(v[j], v2[j], inv_s2);
    }
    tc_fence_before();
    __syncthreads();  // TMEM read before the next group's MMA overwrites it
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 256u);
}

}  // namespace

cudaError_t launch_gram_probe(const DevData& D, const int32_t* rows, const int32_t* centres, int64_t groups,
                              float* out, DevStatus* status, int num_sms, cudaStream_t s) {
  if (groups <= 0) return cudaSuccess;
  // 64 KB of operands, requested as 120 KB so that one CTA (256 TMEM columns) runs per SM
  const size_t bytes = 120 * 1024;
  cudaError_t err = cudaFuncSetAttribute(gram_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (err != cudaSuccess) return err;
  const float scale = centres ? 0.5f * D.scale : D.scale;  // the prune's scale for centred rows
  const float inv_s = 1.f / scale;
  const int64_t grid = std::min<int64_t>(groups, num_sms);
  gram_probe_kernel<<<unsigned(grid), 128, bytes, s>>>(D.X, D.row_bytes, scale, inv_s * inv_s, rows, centres, groups,
                                                       out, status);
  return cudaGetLastError();
}

cudaError_t launch_prune(const PruneLaunch& L, cudaStream_t s) {
  PruneArgs a{};
  a.X = L.data.X;
  a.row_bytes = L.data.row_bytes;
  // float rows enter centred on the pivot, |x - p| <= 2 max |x|: half the
  // data's power-of-two scale keeps them in [-1, 1]
  a.scale = L.data.dtype == kF32 ? 0.5f * L.data.scale : L.data.scale;
  a.inv_s = 1.f / a.scale;
  a.inv_s2 = a.inv_s * a.inv_s;
  a.sqrt_d = std::sqrt(float(L.data.d)) * 1.0001f;
  a.d = L.data.d;
  a.row_ptr = L.row_ptr;
  a.col = L.col;
  a.T = L.T;
  a.variant = L.variant;
  a.status = L.status;
  a.point_of = L.point_of;
  // Targets go to the kernel in ascending A (each with its own outputs), so
  // that the float pass may stop at the first target where a pair is surely
  // not removed: it is then surely not removed at every later one.
  int order[kMaxTargets];
  for (int t = 0; t < L.T; ++t) order[t] = t;
  std::stable_sort(order, order + L.T, [&](int x, int y) { return L.A[x] < L.A[y]; });
  for (int t = 0; t < L.T; ++t) {
    const int o = order[t];
    a.A[t] = L.A[o];
    a.R[t] = L.R[o];
    a.inv_A2[t] = float(1.0 / (double(L.A[o]) * double(L.A[o])));
    a.out_col[t] = L.out_col[o];
    a.out_cnt[t] = L.out_cnt[o];
  }
  // distinct alphas (ascending, as the targets now are) and each target's index among them
  a.TA = 0;
  for (int t = 0; t < L.T; ++t) {
    if (a.TA == 0 || a.Ad[a.TA - 1] != a.A[t]) {
      a.kappa[a.TA] = float(1.0e6 / (double(a.A[t]) * double(a.A[t])));
      a.Ad[a.TA++] = a.A[t];
    }
    a.amap[t] = a.TA - 1;
  }
  cudaError_t err = cudaSuccess;
  for (int b = 0; b < 3 && err == cudaSuccess; ++b) {
    a.nodes = L.bucket_nodes[b];
    a.count = L.bucket_count + b;
    a.work = L.work + b;
    const int64_t hc = L.host_bucket_count[b];
    if (L.data.dtype == kU8) {
      // The f16 Gram is exact for uint8 only while every partial sum stays
      // below 2^24 (d <= 256 here); wider rows take the exact CUDA-core path.
      const bool exact_tc = L.data.d <= 256;
      if (b == 0 && exact_tc && L.tile0 == 0) err = run_fast<kU8, 64>(a, L.num_sms, hc, L.ctas_per_sm, s);
      else if (b <= 1 && exact_tc) err = run_fast<kU8, 128>(a, L.num_sms, hc, L.ctas_per_sm, s);
      else err = run_generic<kU8>(a, L.num_sms, hc, L.host_max_degree, s);
    } else {
      if (b == 0 && L.tile0 == 0) err = run_fast<kF32, 64>(a, L.num_sms, hc, L.ctas_per_sm, s);
      else if (b <= 1) err = run_fast<kF32, 128>(a, L.num_sms, hc, L.ctas_per_sm, s);
      else err = run_generic<kF32>(a, L.num_sms, hc, L.host_max_degree, s);
    }
  }
  return err;
}

}  // namespace rpk
