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
// uint8 distances are exact.  float32 keys carry a rigorous error bound; at
// the end, runs of keys whose intervals overlap are re-ordered by binary64
// distances, and the list is accepted only if the k-th entry's run ends
// strictly before the last kept entry (so no discarded point can belong to
// the true top k); otherwise the device status reports kDevTieUnresolved.
#include "internal.h"

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
  const int64_t q0 = int64_t(blockIdx.x) * QB;
  const int nqb = int(a.nq - q0 < QB ? a.nq - q0 : QB);
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
          for (int i = 0; i < 4; ++i) acc_pair<DT>(qv[j], pv[i], acc[j][i]);
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
        const float E = rel_bound(a.d), Eabs = abs_bound(a.d);
        const float* X = reinterpret_cast<const float*>(a.X);
        const int64_t stride = a.row_bytes / 4;
        const float* qv = a.Q ? reinterpret_cast<const float*>(a.Q + qg * a.row_bytes) : X + qg * stride;
        int i = 0;
        int kth_run_end = -1;
        while (i < nc) {
          int e = i;
          while (e + 1 < nc && !sure_less(__uint_as_float(unsigned(b[e] >> 32)),
                                          __uint_as_float(unsigned(b[e + 1] >> 32)), E, Eabs))
            ++e;
          if (e > i) {
            // insertion sort of b[i..e] by (binary64 distance, id)
            double dd[64];
            const int len = min(e - i + 1, 64);
            if (e - i + 1 > 64) raise_status(a.status, kDevTieUnresolved, qg);
            for (int r = 0; r < len; ++r)
              dd[r] = canon_d2_f32(qv, X + int64_t(unsigned(b[i + r])) * stride, a.d);
            atomicAdd(&a.status->fp64_sort_keys, static_cast<unsigned long long>(len));
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
          if (i <= a.k - 1 && a.k - 1 <= e) kth_run_end = e;
          i = e + 1;
        }
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
  const unsigned grid = unsigned((K.nq + QB - 1) / QB);
  cudaError_t err;
  if (K.data.dtype == kF32) {
    err = cudaFuncSetAttribute(knn_kernel<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (err != cudaSuccess) return err;
    knn_kernel<kF32><<<grid, kThreads, bytes, s>>>(a);
  } else {
    err = cudaFuncSetAttribute(knn_kernel<kU8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (err != cudaSuccess) return err;
    knn_kernel<kU8><<<grid, kThreads, bytes, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace rpk
