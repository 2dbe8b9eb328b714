// Exact k nearest neighbours by brute force, ordered by (distance, id): the
// ground truth of k-recall@k (§4) and the candidate lists of kNN-candidate
// base graphs.
//
// A CTA owns 32 queries and streams every base point past them in tiles of
// 128 points, one 128-byte slice of every row at a time (cp.async into padded
// shared rows).  Each thread accumulates a 4 x 4 block of squared distances.
// A distance enters the query's candidate buffer only if its (distance, id)
// key is below the query's current threshold (the KEEP-th best so far); when
// a buffer could overflow on the next tile, each warp sorts the buffers of
// its queries in shared memory and keeps the best KEEP.
//
// uint8 distances are exact.  float32 keys are summed per 128-byte slice (32
// dimensions, in index order) and the slice sums added in order, which keeps
// their rigorous error bound at (min(d, 32) + ceil(d / 32) + 8) ulps instead
// of (d + 8) for one running sum (the difference matters at d = 960, where
// the distances of the 128-th and 160-th neighbours can lie that close).  At
// the end, runs of keys whose intervals overlap are re-ordered by binary64
// distances, and the list is accepted only if the k-th entry's run ends
// strictly before the last kept entry (so no discarded point can belong to
// the true top k); otherwise the device status reports kDevTieUnresolved.
#include <cmath>
#include <cstring>

#include "internal.h"
#include "tc.cuh"

namespace rpk {

namespace {

constexpr int QB = 32;        // queries per CTA
constexpr int PB = 128;       // points per tile
constexpr int CAP = 512;      // candidate buffer per query
constexpr int kPitch = 144;   // shared row pitch for one 128-byte slice
constexpr int kThreads = 256;

struct KnnArgs {
  const uint8_t* X;
  int64_t row_bytes;
  int64_t n;
  int d;
  const uint8_t* Q;  // nullptr: queries are base points 0..nq-1 (self excluded)
  int64_t nq;
  int64_t q_base;    // this launch handles queries q_base .. q_end-1
  int64_t q_end;
  int k;
  int keep;  // entries kept per query between merges (k for exact data, k + 32 for float)
  int32_t* out_ids;
  float* out_dists;
  DevStatus* status;
};

struct KnnSmem {
  unsigned long long buf[QB][CAP];
  unsigned long long thr[QB];
  int cnt[QB];
  int flag;
  alignas(16) unsigned char qs[QB * kPitch];
  alignas(16) unsigned char ps[PB * kPitch];
};

template <int DT>
__device__ __forceinline__ void acc_pair(uint2 x, uint2 y, unsigned& acc) {
  if constexpr (DT == kU8) {
    acc = sqdiff4_u8(x.x, y.x, acc);
    acc = sqdiff4_u8(x.y, y.y, acc);
  } else {
    float f = __uint_as_float(acc);
    float t = __uint_as_float(x.x) - __uint_as_float(y.x);
    f = fmaf(t, t, f);
    t = __uint_as_float(x.y) - __uint_as_float(y.y);
    f = fmaf(t, t, f);
    acc = __float_as_uint(f);
  }
}

// Runs of single-precision keys in b[0, m) (sorted ascending) whose intervals
// overlap are re-ordered by (binary64 distance, id); lane 0 alone, runs are
// rare.  Returns the end of the run holding position k - 1 (or -1).
__device__ int fix_near_ties(const uint8_t* Xb, int64_t row_bytes, int d, DevStatus* status,
                             unsigned long long* b, int m, const float* qv, int64_t qg, int k = 0) {
  const float E = slice_rel_bound(d), Eabs = abs_bound(d);
  const float* X = reinterpret_cast<const float*>(Xb);
  const int64_t stride = row_bytes / 4;
  int i = 0;
  int kth_run_end = -1;
  while (i < m) {
    int e = i;
    while (e + 1 < m && !sure_less(__uint_as_float(unsigned(b[e] >> 32)), __uint_as_float(unsigned(b[e + 1] >> 32)), E,
                                   Eabs))
      ++e;
    if (e > i) {
      // insertion sort of b[i..e] by (binary64 distance, id)
      double dd[64];
      const int len = min(e - i + 1, 64);
      if (e - i + 1 > 64) raise_status(status, kDevTieUnresolved, qg);
      for (int r = 0; r < len; ++r) dd[r] = canon_d2_f32(qv, X + int64_t(unsigned(b[i + r])) * stride, d);
      atomicAdd(&status->fp64_sort_keys, static_cast<unsigned long long>(len));
      for (int r = 1; r < len; ++r) {
        const unsigned long long kv = b[i + r];
        const double dv = dd[r];
        int z = r - 1;
        while (z >= 0 && (dd[z] > dv || (dd[z] == dv && unsigned(b[i + z]) > unsigned(kv)))) {
          b[i + z + 1] = b[i + z];
          dd[z + 1] = dd[z];
          --z;
        }
        b[i + z + 1] = kv;
        dd[z + 1] = dv;
      }
    }
    if (i <= k - 1 && k - 1 <= e) kth_run_end = e;
    i = e + 1;
  }
  return kth_run_end;
}

// Sort the first `len` (padded to a power of two) keys of one buffer with one warp.
__device__ void warp_sort(unsigned long long* b, int len) {
  int P = 32;
  while (P < len) P <<= 1;
  const int lane = threadIdx.x & 31;
  for (int i = len + lane; i < P; i += 32) b[i] = ~0ull;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int idx = lane; idx < P / 2; idx += 32) {
        const int i = (idx / j) * 2 * j + (idx % j);
        const int l = i + j;
        const bool up = (i & k) == 0;
        const unsigned long long x = b[i], y = b[l];
        if ((x > y) == up) {
          b[i] = y;
          b[l] = x;
        }
      }
      __syncwarp();
    }
  }
}

template <int DT>
__device__ void merge_buffers(KnnSmem& S, int keep) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = w; q < QB; q += kThreads / 32) {
    const int c = S.cnt[q];
    if (c > keep || (c == keep && S.thr[q] == ~0ull)) {
      warp_sort(S.buf[q], c);
      if (lane == 0) {
        const int nc = min(c, keep);
        S.cnt[q] = nc;
        if (nc == keep) S.thr[q] = S.buf[q][keep - 1];
      }
    }
    __syncwarp();
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads) knn_kernel(KnnArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  KnnSmem& S = *reinterpret_cast<KnnSmem*>(smem_raw);
  const int t = threadIdx.x;
  const int64_t q0 = a.q_base + int64_t(blockIdx.x) * QB;
  const int nqb = int(a.q_end - q0 < QB ? a.q_end - q0 : QB);
  for (int q = t; q < QB; q += kThreads) {
    S.cnt[q] = 0;
    S.thr[q] = ~0ull;
  }
  const int tq = t & 7, tp = t >> 3;  // thread rows: queries tq + 8j, points tp + 32i
  const int nslices = int(a.row_bytes / 128);
  __syncthreads();

  for (int64_t p0 = 0; p0 < a.n; p0 += PB) {
    const int npb = int(a.n - p0 < PB ? a.n - p0 : PB);
    unsigned acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[j][i] = 0u;
    for (int s = 0; s < nslices; ++s) {
      unsigned part[4][4];  // this slice's sums
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) part[j][i] = 0u;
      for (int c = t; c < (QB + PB) * 8; c += kThreads) {
        const int r = c >> 3, part = c & 7;
        unsigned char* dst;
        const uint8_t* src = nullptr;
        if (r < QB) {
          dst = S.qs + r * kPitch + part * 16;
          if (r < nqb) {
            const int64_t qg = q0 + r;
            src = (a.Q ? a.Q + qg * a.row_bytes : a.X + qg * a.row_bytes) + s * 128 + part * 16;
          }
        } else {
          const int pr = r - QB;
          dst = S.ps + pr * kPitch + part * 16;
          if (pr < npb) src = a.X + (p0 + pr) * a.row_bytes + s * 128 + part * 16;
        }
        if (src) cp_async16(dst, src, 16);
        else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
      }
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
#pragma unroll 4
      for (int wd = 0; wd < 16; ++wd) {
        uint2 qv[4], pv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) qv[j] = *reinterpret_cast<const uint2*>(S.qs + (tq + 8 * j) * kPitch + wd * 8);
#pragma unroll
        for (int i = 0; i < 4; ++i) pv[i] = *reinterpret_cast<const uint2*>(S.ps + (tp + 32 * i) * kPitch + wd * 8);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int i = 0; i < 4; ++i) acc_pair<DT>(qv[j], pv[i], part[j][i]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if constexpr (DT == kU8) acc[j][i] += part[j][i];
          else acc[j][i] = __float_as_uint(__uint_as_float(acc[j][i]) + __uint_as_float(part[j][i]));
        }
      __syncthreads();
    }
    // candidates below the thresholds
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ql = tq + 8 * j;
      if (ql >= nqb) continue;
      const int64_t self = a.Q ? -1 : q0 + ql;
      const unsigned long long thr = S.thr[ql];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int pl = tp + 32 * i;
        const int64_t pid = p0 + pl;
        if (pl >= npb || pid == self) continue;
        const unsigned long long key = (static_cast<unsigned long long>(acc[j][i]) << 32) | unsigned(pid);
        if (key < thr) {
          const int at = atomicAdd(&S.cnt[ql], 1);
          S.buf[ql][at] = key;  // at < CAP: buffers are merged while they hold <= CAP - PB entries
        }
      }
    }
    __syncthreads();
    if (t == 0) {
      int f = 0;
      for (int q = 0; q < QB; ++q) f |= S.cnt[q] > CAP - PB;
      S.flag = f;
    }
    __syncthreads();
    if (S.flag) {
      merge_buffers<DT>(S, a.keep);
      __syncthreads();
    }
  }
  // final ordering
  const int w = t >> 5, lane = t & 31;
  for (int q = w; q < nqb; q += kThreads / 32) {
    const int c = S.cnt[q];
    warp_sort(S.buf[q], c);
    const int nc = min(c, a.keep);
    const int64_t qg = q0 + q;
    unsigned long long* b = S.buf[q];
    if constexpr (DT == kF32) {
      // near-tie runs: re-order by binary64 distances (serial in lane 0; rare)
      if (lane == 0) {
        const float* X = reinterpret_cast<const float*>(a.X);
        const int64_t stride = a.row_bytes / 4;
        const float* qv = a.Q ? reinterpret_cast<const float*>(a.Q + qg * a.row_bytes) : X + qg * stride;
        const int kth_run_end = fix_near_ties(a.X, a.row_bytes, a.d, a.status, b, nc, qv, qg, a.k);
        // a full list whose k-th run reaches the last kept entry may miss points
        if (nc == a.keep && kth_run_end >= nc - 1 && a.keep > a.k) raise_status(a.status, kDevTieUnresolved, qg);
      }
      __syncwarp();
    }
    for (int j = lane; j < a.k; j += 32) {
      const bool have = j < nc;
      a.out_ids[qg * a.k + j] = have ? int32_t(unsigned(b[j])) : -1;
      if (a.out_dists) {
        const unsigned kb = unsigned(b[j] >> 32);
        a.out_dists[qg * a.k + j] = !have ? __int_as_float(0x7f800000) : (DT == kU8 ? float(kb) : __uint_as_float(kb));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tensor-core path: exact kNN with an f16 Gram filter
// ---------------------------------------------------------------------------
// Points and queries are packed once as f16 rows in tiles of 128 rows, each
// tile already in the core-matrix order of the tcgen05 operand layout: uint8
// values as they are (exact), float rows scaled by a power of two so that
// |x| <= 1 and split into two f16 operands, hi = f16(x) and lo =
// f16(2^11 (x - hi)), the tile holding hi then lo.  A CTA of 4 warps owns 128
// queries (thread t = query t = TMEM lane t) and streams every point tile past
// them: D = Q P^T on tcgen05 into one of two TMEM accumulator sets (float rows:
// hi hi^T in one accumulator, hi lo^T + lo hi^T in a second, G~ = the first +
// 2^-11 the second), the next tile's copy in flight meanwhile.  The split keeps
// the Gram error near 2^-22 |q||p| instead of f16's 2^-11, so the candidate
// window stays narrow on data whose neighbours lie close together.
//
// From G~ the thread forms d2~ = |q|^2 + |p|^2 - 2 G~ (scaled units) and a
// rigorous error bound err (zero for uint8 rows of d <= 128, where every
// quantity is an exact integer below 2^24).  Point p is kept as a candidate
// when its lower bound d2~ - err is at most tau, the k-th smallest upper bound
// d2~ + err met so far: at least k points have d2 <= tau, so every true k
// nearest neighbour passes when it is met (tau only decreases).  A query's
// candidates live in a global buffer; when it could overflow, the query's
// warp sorts the upper bounds, lowers tau and drops the candidates above it.
// At the end the candidates are ranked by their exact keys (uint8: exact
// integers; float: sums per 32-dim slice with near-tie runs re-ordered in
// binary64), as the CUDA-core kernel ranks its lists.
constexpr int kTcQ = 128;  // queries per CTA (rows of the MMA)
constexpr int kTcP = 128;  // points per tile (columns of the MMA)

struct KnnTcArgs {
  const uint8_t* X;          // raw rows (exact ranking)
  int64_t row_bytes;
  int64_t n;
  int d;
  const uint8_t* Qraw;       // raw query rows, or nullptr: queries are base points
  int64_t nq;
  int k;
  const uint8_t* qtiles;     // packed query tiles (the point tiles for base-point queries)
  const uint8_t* ptiles;     // packed point tiles
  int64_t tile_bytes;        // kTcP * dpad * 2 per operand: uint8 one (f16), float two (hi, lo)
  int ksteps;                // dpad / 16
  const float* qnorm;        // |q'|^2 per query (scaled)
  const float* pnorm;        // |p'|^2 per point, padded to whole tiles with 0
  const float2* tmax;        // per point tile: (max |p'|^2, max |p'|)
  int exact;                 // 1: G~ and d2~ are exact
  float eps_ip, eps_n, sub_abs;  // sub_abs: the subnormal-rounding term per unit of |q| + |p|
  uint4* cand;               // per CTA: kTcQ x capc entries {lb, ub, id, 0}
  int capc;
  int32_t* out_ids;
  float* out_dists;
  unsigned* work;            // zeroed: next query tile
  DevStatus* status;
};

// Total order on floats as unsigned keys (negatives included).
__device__ __forceinline__ unsigned fkey(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Bound on |d2~ - d2'| for one (query, point) pair in scaled units: twice the
// Gram error (eps_ip |q'||p'| plus the subnormal roundings, sub_abs (|q'| +
// |p'|) in all), the single-precision norms, and the roundings that form d2~
// and its two bounds (2^-21 (|q'|^2 + |p'|^2) covers them).
__device__ __forceinline__ float tc_err(const KnnTcArgs& a, float nq, float sq, float np, float sp) {
  return (2.f * a.eps_ip * sq * sp * 1.001f + a.sub_abs * (sq + sp) + (a.eps_n + 4.7683716e-07f) * (nq + np)) *
             1.0001f +
         1e-30f;
}

// Operands per tile: uint8 rows one f16 operand, float rows two (hi, lo).
__host__ __device__ constexpr int tc_nop(int dtype) { return dtype == kF32 ? 2 : 1; }

size_t knn_tc_smem(int dtype, int64_t tile_bytes, int capc) {
  // A tile, two B tiles, two point-norm rows, per-warp sort buffers, misc.
  // uint8: at least a third of an SM's shared memory, so that at most two CTAs
  // (each holding 256 of the SM's 512 TMEM columns) share an SM; float: more
  // than half, one CTA holding all 512 (two sets of two accumulators).
  const size_t need = size_t(tile_bytes) * 3 + 2 * kTcP * 4 + size_t(4) * capc * 8 + 256;
  return std::max(need, dtype == kF32 ? size_t(228 * 1024 / 2 + 1024) : size_t(228 * 1024 / 3 + 1024));
}

template <int DT>
__global__ void __launch_bounds__(128) knn_tc_kernel(KnnTcArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // float rows: hi and lo operands, two accumulators per set (acc0 at column
  // 0 of the set, acc1 at 128)
  constexpr bool kSplit = DT == kF32;
  constexpr uint32_t kSetCols = kSplit ? 256u : 128u;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  unsigned char* sA = smem_raw;
  unsigned char* sB0 = smem_raw + a.tile_bytes;
  unsigned char* sB1 = smem_raw + 2 * a.tile_bytes;
  float* sPn = reinterpret_cast<float*>(smem_raw + 3 * a.tile_bytes);                 // [2][kTcP]
  unsigned long long* sSort = reinterpret_cast<unsigned long long*>(sPn + 2 * kTcP);  // [4][capc]
  unsigned char* misc = reinterpret_cast<unsigned char*>(sSort + size_t(4) * a.capc);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc);  // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(misc + 16);
  int* qt_slot = reinterpret_cast<int*>(misc + 32);
  const int64_t npt = (a.n + kTcP - 1) / kTcP;
  const int64_t nqt = (a.nq + kTcQ - 1) / kTcQ;
  constexpr uint32_t idesc = umma_idesc_f16(128, 128);
  constexpr uint32_t lbo = 16u * 128u;  // 16 row-groups of 128 bytes per k-chunk

  if (warp == 0) tmem_alloc(tmem_slot, 2 * kSetCols);  // two accumulator sets
  if (t == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t phase0 = 0u, phase1 = 0u;
  unsigned long long* wsort = sSort + size_t(warp) * a.capc;
  const float inf = __int_as_float(0x7f800000);
  bool dead = false;

  for (;;) {
    if (t == 0) *qt_slot = int(atomicAdd(a.work, 1u));
    __syncthreads();
    const int64_t qt = *qt_slot;
    __syncthreads();
    if (qt >= nqt) break;
    // ---- the query tile (operand A), resident for the whole scan
    {
      const uint4* src = reinterpret_cast<const uint4*>(a.qtiles + qt * a.tile_bytes);
      uint4* dst = reinterpret_cast<uint4*>(sA);
      for (int64_t i = t; i < a.tile_bytes / 16; i += 128) dst[i] = src[i];
    }
    const int64_t qi = qt * kTcQ + t;
    const bool qlive = qi < a.nq;
    const float nqq = qlive ? a.qnorm[qi] : 0.f;
    const float sq = sqrtf(nqq);
    float tau = inf;
    int cnt = 0;
    uint4* cbuf = a.cand + (int64_t(blockIdx.x) * kTcQ + t) * a.capc;
    auto load_tile = [&](int64_t j, unsigned char* dstB, float* dstN) {
      const unsigned char* src = a.ptiles + j * a.tile_bytes;
      for (int64_t i = t; i < a.tile_bytes / 16; i += 128) cp_async16(dstB + i * 16, src + i * 16, 16);
      if (t < kTcP / 4) cp_async16(dstN + 4 * t, a.pnorm + j * kTcP + 4 * t, 16);
      cp_async_commit();
    };
    load_tile(0, sB0, sPn);
    for (int64_t j = 0; j < npt; ++j) {
      const int b = int(j & 1);
      unsigned char* sB = b ? sB1 : sB0;
      const float* pnb = sPn + b * kTcP;
      cp_async_wait<0>();
      fence_async_smem();
      tc_fence_before();
      __syncthreads();  // tile j in smem; every read of accumulator b (tile j - 2) finished
      tc_fence_after();
      if (t == 0) {
        const uint32_t acc = tmem + uint32_t(b) * kSetCols;
        const uint32_t lo_off = uint32_t(a.tile_bytes / 2);  // float tiles: lo after hi
        for (int kk = 0; kk < a.ksteps; ++kk) {
          const uint64_t da = umma_desc(smem_addr(sA) + uint32_t(kk) * 2u * lbo, lbo, 128u);
          const uint64_t db = umma_desc(smem_addr(sB) + uint32_t(kk) * 2u * lbo, lbo, 128u);
          umma_f16(acc, da, db, idesc, kk > 0);
          if constexpr (kSplit) {  // the cross terms with the low halves
            const uint64_t dal = umma_desc(smem_addr(sA) + lo_off + uint32_t(kk) * 2u * lbo, lbo, 128u);
            const uint64_t dbl = umma_desc(smem_addr(sB) + lo_off + uint32_t(kk) * 2u * lbo, lbo, 128u);
            umma_f16(acc + 128u, da, dbl, idesc, kk > 0);
            umma_f16(acc + 128u, dal, db, idesc, true);
          }
        }
        umma_commit(&mbar[b]);
      }
      // B[b ^ 1] held tile j - 1, whose MMA finished before its candidates were read
      if (j + 1 < npt) load_tile(j + 1, b ? sB0 : sB1, sPn + (b ^ 1) * kTcP);
      const bool ok = mbar_wait(&mbar[b], b ? phase1 : phase0, 1 << 24);
      if (b) phase1 ^= 1u;
      else phase0 ^= 1u;
      if (!__syncthreads_and(ok)) {  // the MMA never completed: report, stop (uniform)
        if (t == 0) raise_status(a.status, kDevOverflow, -3);
        dead = true;
        break;
      }
      tc_fence_after();
      // ---- this tile's candidates
      float thr = tau;
      if (!a.exact) {
        const float2 tm = a.tmax[j];
        thr = (tau + tc_err(a, nqq, sq, tm.x, tm.y)) * 1.000001f;  // never below tau + err of a point
      }
      const int64_t p0 = j * kTcP;
#pragma unroll 1
      for (int c0 = 0; c0 < kTcP; c0 += 32) {
        uint32_t v[32], v2[kSplit ? 32 : 1];
        const uint32_t acc = tmem + (uint32_t(32 * warp) << 16) + uint32_t(b) * kSetCols + uint32_t(c0);
        tmem_ld32(acc, v);
        if constexpr (kSplit) tmem_ld32(acc + 128u, *reinterpret_cast<uint32_t(*)[32]>(v2));
        tmem_ld_wait();
        if (!qlive) continue;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int c = c0 + jj;
          const float pn = pnb[c];
          // float rows: hi hi^T + 2^-11 (hi lo^T + lo hi^T), scaled units
          const float G = kSplit ? fmaf(__uint_as_float(v2[jj]), 4.8828125e-04f, __uint_as_float(v[jj]))
                                 : __uint_as_float(v[jj]);
          const float d2 = fmaf(-2.f, G, nqq + pn);
          if (d2 <= thr) {
            const int64_t pid = p0 + c;
            if (pid >= a.n || (!a.Qraw && pid == qi)) continue;
            float lb = d2, ub = d2;
            if (!a.exact) {
              const float err = tc_err(a, nqq, sq, pn, sqrtf(pn));
              lb = d2 - err;
              ub = d2 + err;
            }
            if (lb <= tau) {
              if (cnt < a.capc) cbuf[cnt++] = make_uint4(__float_as_uint(lb), __float_as_uint(ub), unsigned(pid), 0u);
              else raise_status(a.status, kDevOverflow, qi);
            }
          }
        }
      }
      // ---- buffers that could overflow on the next tile: lower tau, drop what lies above it
      unsigned need = __ballot_sync(0xffffffffu, cnt > a.capc - kTcP);
      __syncwarp();  // candidates written by one lane are read by the whole warp below
      while (need) {
        const int L = __ffs(need) - 1;
        need &= need - 1;
        const int cL = __shfl_sync(0xffffffffu, cnt, L);
        uint4* bL = a.cand + (int64_t(blockIdx.x) * kTcQ + warp * 32 + L) * a.capc;
        for (int i = lane; i < cL; i += 32)
          wsort[i] = (static_cast<unsigned long long>(fkey(__uint_as_float(bL[i].y))) << 32) | unsigned(i);
        __syncwarp();
        warp_sort(wsort, cL);
        const float tnew = cL >= a.k ? fkey_inv(unsigned(wsort[a.k - 1] >> 32)) : inf;
        __syncwarp();
        int w = 0;
        for (int i0 = 0; i0 < cL; i0 += 32) {
          const int i = i0 + lane;
          uint4 e = make_uint4(0, 0, 0, 0);
          bool keep = false;
          if (i < cL) {
            e = bL[i];
            keep = __uint_as_float(e.x) <= tnew;
          }
          const unsigned km = __ballot_sync(0xffffffffu, keep);
          __syncwarp();
          if (keep) bL[w + __popc(km & ((1u << lane) - 1))] = e;
          w += __popc(km);
          __syncwarp();
        }
        if (lane == L) {
          cnt = w;
          tau = fminf(tau, tnew);
          if (cnt > a.capc - kTcP) raise_status(a.status, kDevOverflow, qi);
        }
        __syncwarp();
      }
    }
    if (dead) break;
    // ---- exact ranking of each query's candidates, one warp per query in turn
    for (int L = 0; L < 32; ++L) {
      const int64_t qg = qt * kTcQ + warp * 32 + L;
      if (qg >= a.nq) break;
      const int cL = __shfl_sync(0xffffffffu, cnt, L);
      const float tL = __shfl_sync(0xffffffffu, tau, L);
      const uint4* bL = a.cand + (int64_t(blockIdx.x) * kTcQ + warp * 32 + L) * a.capc;
      const uint8_t* qrow = a.Qraw ? a.Qraw + qg * a.row_bytes : a.X + qg * a.row_bytes;
      int m = 0;
      for (int i0 = 0; i0 < cL; i0 += 32) {
        const int i = i0 + lane;
        bool keep = false;
        unsigned long long key = 0;
        if (i < cL) {
          const uint4 e = bL[i];
          keep = __uint_as_float(e.x) <= tL;
          if (keep) {
            const uint2* x2 = reinterpret_cast<const uint2*>(qrow);
            const uint2* y2 = reinterpret_cast<const uint2*>(a.X + int64_t(e.z) * a.row_bytes);
            unsigned acc = 0;
            for (int64_t s0 = 0; s0 < a.row_bytes / 8; s0 += 16) {  // per 128-byte slice, as the CUDA-core kernel
              unsigned part = 0;
              for (int w8 = 0; w8 < 16; ++w8) acc_pair<DT>(x2[s0 + w8], y2[s0 + w8], part);
              if constexpr (DT == kU8) acc += part;
              else acc = __float_as_uint(__uint_as_float(acc) + __uint_as_float(part));
            }
            key = (static_cast<unsigned long long>(acc) << 32) | e.z;
          }
        }
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) wsort[m + __popc(km & ((1u << lane) - 1))] = key;
        m += __popc(km);
      }
      __syncwarp();
      warp_sort(wsort, m);
      const int nc = min(m, a.k);
      if constexpr (DT == kF32) {
        if (lane == 0) fix_near_ties(a.X, a.row_bytes, a.d, a.status, wsort, m, reinterpret_cast<const float*>(qrow), qg);
        __syncwarp();
      }
      for (int j = lane; j < a.k; j += 32) {
        const bool have = j < nc;
        a.out_ids[qg * a.k + j] = have ? int32_t(unsigned(wsort[j])) : -1;
        if (a.out_dists) {
          const unsigned kb = unsigned(wsort[j] >> 32);
          a.out_dists[qg * a.k + j] = !have ? inf : (DT == kU8 ? float(kb) : __uint_as_float(kb));
        }
      }
      __syncwarp();
    }
  }
  cp_async_wait<0>();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * kSetCols);
}

// ---- packing: f16 operand tiles, scaled squared norms, per-tile maxima

// max |x| over n rows of float data (bits of a non-negative float, atomicMax)
__global__ void maxabs_kernel(const uint8_t* __restrict__ X, int64_t row_bytes, int64_t n, int d,
                              unsigned* __restrict__ out) {
  float m = 0.f;
  const int64_t total = n * d;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / d, c = i % d;
    m = fmaxf(m, fabsf(reinterpret_cast<const float*>(X + r * row_bytes)[c]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Row i -> tile i / 128, row i % 128 of the core-matrix layout: uint8 values
// as f16 (exact); float rows scaled by s (a power of two: exact) and split
// into f16 hi and lo (split_f16x2), lo kTcP * dpad * 2 bytes after hi; the
// norm |x'|^2 in single precision in index order.
template <int DT>
__global__ void pack_f16_kernel(const uint8_t* __restrict__ X, int64_t row_bytes, int64_t n, int d, int dpad,
                                float s, uint8_t* __restrict__ tiles, float* __restrict__ norms) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t ntile = (n + kTcP - 1) / kTcP;
  if (i >= ntile * kTcP) return;
  const int64_t tile = i / kTcP;
  const int r = int(i % kTcP);
  const int64_t op_bytes = int64_t(kTcP) * dpad * 2;
  uint8_t* tb = tiles + tile * op_bytes * tc_nop(DT);
  float acc = 0.f;
  for (int kc = 0; kc < dpad / 8; ++kc) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = kc * 8 + e;
      float x = 0.f;
      if (i < n && c < d) {
        if constexpr (DT == kU8) x = float(X[i * row_bytes + c]);
        else x = reinterpret_cast<const float*>(X + i * row_bytes)[c] * s;
      }
      v[e] = x;
      acc = fmaf(x, x, acc);
    }
    const int64_t at = (int64_t(kc) * 16 + r / 8) * 128 + (r % 8) * 16;
    if constexpr (DT == kF32) {
      uint4 hi, lo;
      split_f16x2(v[0], v[1], hi.x, lo.x);
      split_f16x2(v[2], v[3], hi.y, lo.y);
      split_f16x2(v[4], v[5], hi.z, lo.z);
      split_f16x2(v[6], v[7], hi.w, lo.w);
      *reinterpret_cast<uint4*>(tb + at) = hi;
      *reinterpret_cast<uint4*>(tb + op_bytes + at) = lo;
    } else {
      *reinterpret_cast<uint4*>(tb + at) = make_uint4(pack_f16x2(v[0], v[1]), pack_f16x2(v[2], v[3]),
                                                      pack_f16x2(v[4], v[5]), pack_f16x2(v[6], v[7]));
    }
  }
  norms[i] = acc;
}

// per tile: (max |x'|^2, max |x'|), the latter rounded up
__global__ void tile_max_kernel(const float* __restrict__ norms, int64_t ntile, float2* __restrict__ out) {
  const int64_t tile = int64_t(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= ntile) return;
  float m = 0.f;
  for (int r = lane; r < kTcP; r += 32) m = fmaxf(m, norms[tile * kTcP + r]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) out[tile] = make_float2(m, sqrtf(m) * 1.000001f);
}

}  // namespace

cudaError_t launch_knn(const KnnLaunch& K, cudaStream_t s) {
  KnnArgs a{};
  a.X = K.data.X;
  a.row_bytes = K.data.row_bytes;
  a.n = K.data.n;
  a.d = K.data.d;
  a.Q = K.Q;
  a.nq = K.nq;
  a.k = K.k;
  a.keep = K.data.dtype == kF32 ? K.k + 32 : K.k;
  a.out_ids = K.out_ids;
  a.out_dists = K.out_dists;
  a.status = K.status;
  if (a.keep > CAP - PB) return cudaErrorInvalidValue;
  const size_t bytes = sizeof(KnnSmem);
  cudaError_t err = cudaFuncSetAttribute(knn_kernel<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(knn_kernel<kU8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (err != cudaSuccess) return err;
  // launches of at most kChunk queries each, so that long scans proceed in bounded steps
  constexpr int64_t kChunk = 65536;
  for (int64_t c0 = 0; c0 < K.nq; c0 += kChunk) {
    a.q_base = c0;
    a.q_end = std::min(K.nq, c0 + kChunk);
    const unsigned grid = unsigned((a.q_end - c0 + QB - 1) / QB);
    if (K.data.dtype == kF32) knn_kernel<kF32><<<grid, kThreads, bytes, s>>>(a);
    else knn_kernel<kU8><<<grid, kThreads, bytes, s>>>(a);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaGetLastError();
}

cudaError_t launch_maxabs_f32(const uint8_t* X, int64_t row_bytes, int64_t n, int d, unsigned* out, cudaStream_t s) {
  if (n > 0) maxabs_kernel<<<1024, 256, 0, s>>>(X, row_bytes, n, d, out);
  return cudaGetLastError();
}

bool knn_tc_eligible(int dtype, int d, int k) {
  if (k < 1 || k > 128) return false;
  const int dpad = (d + 15) / 16 * 16;
  return dtype == kU8 ? d <= 128 : dpad <= 128;  // float: three split tiles fit in shared memory
}

namespace {
struct TcPlan {
  int dpad, capc, ctas, grid;
  int64_t ntile, nqtile, tile_bytes;
  size_t off_ptiles, off_pnorm, off_tmax, off_qtiles, off_qnorm, off_cand, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

TcPlan tc_plan(int dtype, int d, int64_t n, int64_t nq_ext, int num_sms) {
  TcPlan P{};
  P.dpad = (d + 15) / 16 * 16;
  P.capc = 512;
  P.tile_bytes = int64_t(kTcP) * P.dpad * 2 * tc_nop(dtype);
  const size_t smem = knn_tc_smem(dtype, P.tile_bytes, P.capc);
  P.ctas = int(std::max<size_t>(1, std::min<size_t>(2, size_t(228 * 1024) / (smem + 1024))));
  P.grid = num_sms * P.ctas;
  P.ntile = (n + kTcP - 1) / kTcP;
  P.nqtile = (nq_ext + kTcQ - 1) / kTcQ;
  size_t o = 256;  // header: max |x| bits at 0, query-tile counter at 64
  P.off_ptiles = o;
  o = align256(o + size_t(P.ntile) * P.tile_bytes);
  P.off_pnorm = o;
  o = align256(o + size_t(P.ntile) * kTcP * 4);
  P.off_tmax = o;
  o = align256(o + size_t(P.ntile) * 8);
  P.off_qtiles = o;
  o = align256(o + size_t(P.nqtile) * P.tile_bytes);
  P.off_qnorm = o;
  o = align256(o + size_t(P.nqtile) * kTcQ * 4);
  P.off_cand = o;
  o = align256(o + size_t(P.grid) * kTcQ * P.capc * 16);
  P.total = o;
  return P;
}
}  // namespace

size_t knn_tc_scratch_bytes(int dtype, int d, int64_t n, int64_t nq_ext, int num_sms) {
  return tc_plan(dtype, d, n, nq_ext, num_sms).total;
}

cudaError_t launch_knn_tc(const KnnTcLaunch& K, cudaStream_t s) {
  const bool f32 = K.data.dtype == kF32;
  const TcPlan P = tc_plan(K.data.dtype, K.data.d, K.data.n, K.Q ? K.nq : 0, K.num_sms);
  uint8_t* base = K.scratch;
  unsigned* maxbits = reinterpret_cast<unsigned*>(base);
  unsigned* work = reinterpret_cast<unsigned*>(base + 64);
  cudaError_t err = cudaMemsetAsync(base, 0, 256, s);
  if (err != cudaSuccess) return err;
  // the scale: a power of two that brings max |x| (points and queries) to at most 1
  float scale = 1.f;
  if (f32) {
    maxabs_kernel<<<1024, 256, 0, s>>>(K.data.X, K.data.row_bytes, K.data.n, K.data.d, maxbits);
    if (K.Q) maxabs_kernel<<<256, 256, 0, s>>>(K.Q, K.data.row_bytes, K.nq, K.data.d, maxbits);
    unsigned mb = 0;
    if ((err = cudaMemcpyAsync(&mb, maxbits, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return err;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
    float mx = 0.f;
    memcpy(&mx, &mb, 4);
    int e = 0;
    if (mx > 0.f && std::isfinite(mx)) std::frexp(mx, &e);  // mx < 2^e
    scale = std::ldexp(1.f, -e);
  }
  uint8_t* ptiles = base + P.off_ptiles;
  float* pnorm = reinterpret_cast<float*>(base + P.off_pnorm);
  float2* tmax = reinterpret_cast<float2*>(base + P.off_tmax);
  const int64_t rows = P.ntile * kTcP;
  if (f32)
    pack_f16_kernel<kF32><<<unsigned((rows + 255) / 256), 256, 0, s>>>(K.data.X, K.data.row_bytes, K.data.n, K.data.d,
                                                                      P.dpad, scale, ptiles, pnorm);
  else
    pack_f16_kernel<kU8><<<unsigned((rows + 255) / 256), 256, 0, s>>>(K.data.X, K.data.row_bytes, K.data.n, K.data.d,
                                                                     P.dpad, 1.f, ptiles, pnorm);
  tile_max_kernel<<<unsigned((P.ntile + 7) / 8), 256, 0, s>>>(pnorm, P.ntile, tmax);
  const uint8_t* qtiles = ptiles;
  const float* qnorm = pnorm;
  if (K.Q) {
    uint8_t* qt = base + P.off_qtiles;
    float* qn = reinterpret_cast<float*>(base + P.off_qnorm);
    const int64_t qrows = P.nqtile * kTcQ;
    if (f32)
      pack_f16_kernel<kF32><<<unsigned((qrows + 255) / 256), 256, 0, s>>>(K.Q, K.data.row_bytes, K.nq, K.data.d,
                                                                         P.dpad, scale, qt, qn);
    else
      pack_f16_kernel<kU8><<<unsigned((qrows + 255) / 256), 256, 0, s>>>(K.Q, K.data.row_bytes, K.nq, K.data.d,
                                                                        P.dpad, 1.f, qt, qn);
    qtiles = qt;
    qnorm = qn;
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  KnnTcArgs a{};
  a.X = K.data.X;
  a.row_bytes = K.data.row_bytes;
  a.n = K.data.n;
  a.d = K.data.d;
  a.Qraw = K.Q;
  a.nq = K.nq;
  a.k = K.k;
  a.qtiles = qtiles;
  a.ptiles = ptiles;
  a.tile_bytes = P.tile_bytes;
  a.ksteps = P.dpad / 16;
  a.qnorm = qnorm;
  a.pnorm = pnorm;
  a.tmax = tmax;
  a.exact = f32 ? 0 : 1;
  // Split Gram of scaled rows: |G~ - G| <= eps_ip |q'||p'| + 2^-36 sqrt(d) (|q'| + |p'|):
  // 2^-22 left by the split of each operand, 2^-22 for the dropped lo lo^T, 2^-23 for
  // the last sum, f32 accumulation d 2^-24 with a factor 4 allowance; the lo halves
  // that fall below f16's normal range round to 2^-25 in their units, 2^-36 here.
  a.eps_ip = 4.f * 2.384185791015625e-07f + 1.1920929e-07f + float(K.data.d) * 2.384185791015625e-07f;
  a.eps_n = float(K.data.d + 2) * 5.9604645e-08f;
  a.sub_abs = std::sqrt(float(K.data.d)) * 1.001f * 2.910383e-11f;  // twice 2^-36 sqrt(d)
  a.cand = reinterpret_cast<uint4*>(base + P.off_cand);
  a.capc = P.capc;
  a.out_ids = K.out_ids;
  a.out_dists = K.out_dists;
  a.work = work;
  a.status = K.status;
  const size_t smem = knn_tc_smem(K.data.dtype, P.tile_bytes, P.capc);
  if (f32) {
    if ((err = cudaFuncSetAttribute(knn_tc_kernel<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) !=
        cudaSuccess)
      return err;
    knn_tc_kernel<kF32><<<unsigned(P.grid), 128, smem, s>>>(a);
  } else {
    if ((err = cudaFuncSetAttribute(knn_tc_kernel<kU8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) !=
        cudaSuccess)
      return err;
    knn_tc_kernel<kU8><<<unsigned(P.grid), 128, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace rpk
