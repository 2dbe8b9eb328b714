// Load and preparation kernels (a1): padded device rows, input validation,
// graph cleaning and the search start vertex.
//
// Cleaning follows the first step of Algorithm 1, V <- (V u N_out(p)) \ {p}:
// the candidate set is a set that never holds p, so self loops are dropped and
// a repeated id keeps only its first occurrence (which fixes the stored order
// UnsortedRobustPrune walks).
//
// Start vertex (§4.1 starts every search at the medoid): the data point
// nearest to the binary64 mean vector, every sum taken in index order in
// binary64, ties to the smaller id.
#include <cfloat>

#include "internal.h"

namespace rpk {

namespace {

__global__ void pad_rows_kernel(const uint8_t* __restrict__ src, int64_t n, int64_t src_rb,
                                uint8_t* __restrict__ dst, int64_t dst_rb) {
  const int64_t total = n * dst_rb;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / dst_rb, c = i % dst_rb;
    dst[i] = c < src_rb ? src[r * src_rb + c] : 0;
  }
}

__global__ void check_finite_kernel(const float* __restrict__ X, int64_t n, int64_t stride, int d,
                                    DevStatus* st) {
  const int64_t total = n * d;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / d, c = i % d;
    if (!isfinite(X[r * stride + c])) raise_status(st, kDevBadId, -1 - r);
  }
}

__global__ void validate_csr_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                    int64_t n, int64_t nnz, DevStatus* st) {
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = row_ptr[p], b = row_ptr[p + 1];
    if (a < 0 || b < a || b > nnz) {
      raise_status(st, kDevBadId, p);
      continue;
    }
    if (b - a > 1000000) {
      raise_status(st, kDevBadDegree, p);
      continue;
    }
  }
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = col[e];
    if (v < 0 || int64_t(v) >= n) raise_status(st, kDevBadId, e);
  }
}

// One warp per row: entry j is kept if it is not p and no earlier entry of
// the row holds the same id.
__device__ __forceinline__ bool keep_entry(const int32_t* __restrict__ row, int j, int64_t p) {
  const int32_t v = row[j];
  if (int64_t(v) == p) return false;
  for (int i = 0; i < j; ++i)
    if (row[i] == v) return false;
  return true;
}

__global__ void clean_count_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   int64_t n, int32_t* __restrict__ cnt, unsigned long long* dropped) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  unsigned long long self_loops = 0, dups = 0;
  for (int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    const int64_t a = row_ptr[p];
    const int m = int(row_ptr[p + 1] - a);
    const int32_t* row = col + a;
    int kept = 0;
    for (int j = lane; j < m; j += 32) {
      const bool self = int64_t(row[j]) == p;
      const bool k = keep_entry(row, j, p);
      kept += k;
      if (!k) {
        if (self) ++self_loops;
        else ++dups;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(0xffffffffu, kept, o);
    if (lane == 0) cnt[p] = kept;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    self_loops += __shfl_down_sync(0xffffffffu, self_loops, o);
    dups += __shfl_down_sync(0xffffffffu, dups, o);
  }
  if (lane == 0 && (self_loops || dups)) {
    atomicAdd(&dropped[0], self_loops);
    atomicAdd(&dropped[1], dups);
  }
}

__global__ void clean_write_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   int64_t n, const int64_t* __restrict__ new_row_ptr,
                                   int32_t* __restrict__ new_col) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    const int64_t a = row_ptr[p];
    const int m = int(row_ptr[p + 1] - a);
    const int32_t* row = col + a;
    int64_t out = new_row_ptr[p];
    for (int j0 = 0; j0 < m; j0 += 32) {
      const int j = j0 + lane;
      const bool k = j < m && keep_entry(row, j, p);
      const unsigned msk = __ballot_sync(0xffffffffu, k);
      if (k) new_col[out + __popc(msk & ((1u << lane) - 1))] = row[j];
      out += __popc(msk);
    }
  }
}

// counts -> exclusive row_ptr (one level per 4096-node block), plus max count
constexpr int kChunk = 4096;
constexpr int kThreads = 256;

__global__ void count_block_sums(const int32_t* __restrict__ cnt, int64_t n, int64_t* bsum, int32_t* maxd) {
  const int64_t b0 = int64_t(blockIdx.x) * kChunk;
  int64_t s = 0;
  int mx = 0;
  for (int i = threadIdx.x; i < kChunk; i += kThreads) {
    const int64_t p = b0 + i;
    if (p < n) {
      s += cnt[p];
      mx = max(mx, cnt[p]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  __shared__ int64_t ws[kThreads / 32];
  __shared__ int wm[kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    ws[threadIdx.x >> 5] = s;
    wm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t tot = 0;
    int m2 = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      tot += ws[w];
      m2 = max(m2, wm[w]);
    }
    bsum[blockIdx.x] = tot;
    atomicMax(maxd, m2);
  }
}

__global__ void __launch_bounds__(1024) scan_sums_serial(int64_t* bsum, int64_t nblk) {
  // exclusive scan of the (few thousand) block sums in one block
  __shared__ int64_t buf[1024];
  int64_t carry = 0;
  for (int64_t base = 0; base < nblk; base += 1024) {
    const int64_t i = base + threadIdx.x;
    buf[threadIdx.x] = i < nblk ? bsum[i] : 0;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int64_t v = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += v;
      __syncthreads();
    }
    const int64_t incl = buf[threadIdx.x];
    const int64_t v = i < nblk ? bsum[i] : 0;
    if (i < nblk) bsum[i] = carry + incl - v;
    __syncthreads();
    carry += buf[1023];
    __syncthreads();
  }
}

__global__ void count_write(const int32_t* __restrict__ cnt, int64_t n, const int64_t* __restrict__ bsum,
                            int64_t* __restrict__ row_ptr) {
  __shared__ int64_t part[kThreads];
  const int64_t b0 = int64_t(blockIdx.x) * kChunk;
  constexpr int per = kChunk / kThreads;
  int64_t mine = 0;
  for (int i = 0; i < per; ++i) {
    const int64_t p = b0 + int64_t(threadIdx.x) * per + i;
    if (p < n) mine += cnt[p];
  }
  part[threadIdx.x] = mine;
  __syncthreads();
  for (int o = 1; o < kThreads; o <<= 1) {
    const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = bsum[blockIdx.x] + part[threadIdx.x] - mine;
  for (int i = 0; i < per; ++i) {
    const int64_t p = b0 + int64_t(threadIdx.x) * per + i;
    if (p < n) {
      run += cnt[p];
      row_ptr[p + 1] = run;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[0] = 0;
}

// ---- medoid -----------------------------------------------------------------
// uint8: exact integer column sums in any order (they equal the index-order
// binary64 sums, which are exact below 2^53).
__global__ void mean_u8_sum_kernel(const uint8_t* __restrict__ X, int64_t n, int64_t row_bytes, int d,
                                   unsigned long long* __restrict__ sums) {
  const int64_t rows_per_block = 4096;
  const int64_t r0 = int64_t(blockIdx.y) * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    unsigned long long s = 0;
    for (int64_t i = r0; i < r1; ++i) s += X[i * row_bytes + j];
    atomicAdd(&sums[j], s);
  }
}

__global__ void mean_u8_finish_kernel(const unsigned long long* __restrict__ sums, int64_t n, int d,
                                      double* __restrict__ mean) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
    mean[j] = __ddiv_rn(double(sums[j]), double(n));
}

// float32: each column's rows are added in index order in binary64, exactly as
// the sequential loop s <- fl(s + x_i) rounds them, but 64 rows per warp step.
//
// While s stays in one binade [2^E, 2^(E+1)) every addition rounds to the grid
// u = 2^(E-52): fl(s + x) = s + u * rne(x / u), unless x / u is exactly halfway
// (the tie then goes by the parity of the result). So with s = S * u (S the
// 53-bit significand) the step converts each x to integer units q = rne(x/u),
// takes the warp's inclusive prefix sum T = S + (q_0 + ... + q_e), and keeps
// every leading element for which T stays in [2^52 + 1, 2^53] and x was no tie.
// An element with T in that range had an exact sum in binade E (or rounding to
// 2^(E+1)), where this rounding is the IEEE one. The first element outside it is
// added with a real binary64 addition and the next step starts after it; a T of
// exactly 2^53 ends the step (s moves up a binade). s = +0 stays +0 over zeros
// and takes the first nonzero value exactly; a subnormal s takes real additions.
// Every step consumes at least one row, so the loop ends.
//
// One warp per column (grid = d). Rows arrive in blocks of kMeanBlock through
// shared memory, the next block loaded into registers while this one is summed.
constexpr int kMeanBlock = 1024;

// q = rne(x / 2^e52) in the sign frame of s (neg), or false when x / 2^e52 is a
// tie or too large to be kept anyway (the caller then adds x in binary64).
__device__ __forceinline__ bool mean_units(float x, int e52, unsigned neg, long long& q) {
  const unsigned xb = __float_as_uint(x);
  const int ex = int((xb >> 23) & 0xff);
  const unsigned m = (xb & 0x7fffffu) | (ex ? 0x800000u : 0u);  // x = m * 2^((ex ? ex : 1) - 150)
  const int k = (ex ? ex : 1) - 150 - e52;
  long long v = 0;
  bool ok = true;
  if (m != 0) {
    if (k >= 0) {
      ok = k <= 30;  // |x| >= 2^30 u: past the top of the binade before the sum could keep it
      v = ok ? (long long)m << k : 0;
    } else if (-k < 26) {  // -k >= 26: x / u < 1/4 rounds to 0, no tie
      const int sh = -k;
      const unsigned rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
      v = (long long)(m >> sh) + (rem > half ? 1 : 0);
      ok = rem != half;
    }
  }
  q = (xb >> 31) != neg ? -v : v;
  return ok;
}

__global__ void __launch_bounds__(32) mean_f32_kernel(const uint8_t* __restrict__ X, int64_t n,
                                                      int64_t row_bytes, int d, double* __restrict__ mean) {
  __shared__ float buf[kMeanBlock];
  const int j = blockIdx.x;
  const int lane = threadIdx.x;
  const float* F = reinterpret_cast<const float*>(X) + j;
  const int64_t stride = row_bytes / 4;
  const long long kLo = (1ll << 52) + 1, kHi = 1ll << 53;
  float nxt[kMeanBlock / 32];
#pragma unroll
  for (int t = 0; t < kMeanBlock / 32; ++t) {
    const int64_t r = int64_t(32 * t + lane);
    nxt[t] = r < n ? __ldg(F + r * stride) : 0.f;
  }
  double s = 0.0;
  for (int64_t base = 0; base < n; base += kMeanBlock) {
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kMeanBlock / 32; ++t) buf[32 * t + lane] = nxt[t];
    __syncwarp();
    if (base + kMeanBlock < n) {
#pragma unroll
      for (int t = 0; t < kMeanBlock / 32; ++t) {
        const int64_t r = base + kMeanBlock + 32 * t + lane;
        nxt[t] = r < n ? __ldg(F + r * stride) : 0.f;
      }
    }
    const int64_t bend = n < base + kMeanBlock ? n : base + kMeanBlock;
    int64_t i = base;
    while (i < bend) {  // s, i and every branch below are uniform over the warp
      const int avail = bend - i < 64 ? int(bend - i) : 64;
      const int off = int(i - base);
      const bool ha = 2 * lane < avail, hb = 2 * lane + 1 < avail;
      const float xa = ha ? buf[off + 2 * lane] : 0.f;
      const float xb = hb ? buf[off + 2 * lane + 1] : 0.f;
      const unsigned long long sb = (unsigned long long)__double_as_longlong(s);
      const int eb = int((sb >> 52) & 0x7ff);
      if (sb == 0) {  // s = +0
        const unsigned nza = __ballot_sync(0xffffffffu, ha && (__float_as_uint(xa) & 0x7fffffffu) != 0);
        const unsigned nzb = __ballot_sync(0xffffffffu, hb && (__float_as_uint(xb) & 0x7fffffffu) != 0);
        if ((nza | nzb) == 0) {
          i += avail;
          continue;
        }
        const int l = __ffs(int(nza | nzb)) - 1;
        const bool at_a = (nza >> l) & 1u;
        s = double(__shfl_sync(0xffffffffu, at_a ? xa : xb, l));  // 0 + x = x exactly
        i += 2 * l + (at_a ? 0 : 1) + 1;
        continue;
      }
      if (eb == 0 || eb == 0x7ff) {  // subnormal s (or a non-finite one): a real addition
        s = __dadd_rn(s, double(__shfl_sync(0xffffffffu, xa, 0)));
        i += 1;
        continue;
      }
      const int e52 = eb - 1075;
      const unsigned neg = unsigned(sb >> 63);
      const long long S = (long long)((sb & ((1ull << 52) - 1)) | (1ull << 52));
      long long qa, qb;
      const bool oka = mean_units(xa, e52, neg, qa) && ha;
      const bool okb = mean_units(xb, e52, neg, qb) && hb;
      if (!ha) qa = 0;
      if (!hb) qb = 0;
      long long pre = qa + qb;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
      }
      const long long Tb = S + pre, Ta = Tb - qb;
      const bool va = oka && Ta >= kLo && Ta <= kHi;
      const bool vb = okb && Tb >= kLo && Tb <= kHi;
      const unsigned inva = __ballot_sync(0xffffffffu, !va), invb = __ballot_sync(0xffffffffu, !vb);
      const unsigned enda = __ballot_sync(0xffffffffu, va && Ta == kHi);
      const unsigned endb = __ballot_sync(0xffffffffu, vb && Tb == kHi);
      int fi = 64, fe = 64;  // first element kept by no T, first element at 2^53
      if (inva | invb) {
        const int l = __ffs(int(inva | invb)) - 1;
        fi = 2 * l + (((inva >> l) & 1u) ? 0 : 1);
      }
      if (enda | endb) {
        const int l = __ffs(int(enda | endb)) - 1;
        fe = 2 * l + (((enda >> l) & 1u) ? 0 : 1);
      }
      const int c = fi < fe + 1 ? fi : fe + 1;  // elements kept, c <= fi <= avail
      if (c > 0) {
        const int e = c - 1;
        const long long T = __shfl_sync(0xffffffffu, (e & 1) ? Tb : Ta, e >> 1);
        const unsigned long long sign = (unsigned long long)neg << 63;
        s = __longlong_as_double((long long)(T == kHi ? sign | ((unsigned long long)(eb + 1) << 52)
                                                     : sign | ((unsigned long long)eb << 52) |
                                                           (unsigned long long)(T - (1ll << 52))));
      }
      int used = c;
      if (c < avail && c == fi) {
        s = __dadd_rn(s, double(__shfl_sync(0xffffffffu, (c & 1) ? xb : xa, c >> 1)));
        used = c + 1;
      }
      i += used;
    }
  }
  if (lane == 0) mean[j] = __ddiv_rn(s, double(n));
}

__global__ void nearest_mean_kernel(const uint8_t* __restrict__ X, int64_t n, int64_t row_bytes, int d,
                                    int dtype, const double* __restrict__ mean, double* best) {
  double bd = DBL_MAX;
  int64_t bi = -1;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
      const double x = dtype == kU8 ? double(X[i * row_bytes + j])
                                    : double(reinterpret_cast<const float*>(X + i * row_bytes)[j]);
      const double t = __dsub_rn(x, mean[j]);
      s = __dadd_rn(s, __dmul_rn(t, t));
    }
    if (bi < 0 || s < bd) {  // i increases along the loop: earlier ids win ties
      bd = s;
      bi = i;
    }
  }
  __shared__ double sd[256];
  __shared__ long long si[256];
  sd[threadIdx.x] = bd;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double d2 = sd[threadIdx.x + o];
      const long long i2 = si[threadIdx.x + o];
      if (i2 >= 0 && (si[threadIdx.x] < 0 || d2 < sd[threadIdx.x] ||
                      (d2 == sd[threadIdx.x] && i2 < si[threadIdx.x]))) {
        sd[threadIdx.x] = d2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    best[2 * blockIdx.x] = sd[0];
    best[2 * blockIdx.x + 1] = __longlong_as_double(si[0]);
  }
}

__global__ void pick_medoid_kernel(const double* __restrict__ best, int64_t nb, int64_t* medoid) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double bd = DBL_MAX;
  long long bi = -1;
  for (int64_t b = 0; b < nb; ++b) {
    const double d2 = best[2 * b];
    const long long i2 = __double_as_longlong(best[2 * b + 1]);
    if (i2 < 0) continue;
    if (bi < 0 || d2 < bd || (d2 == bd && i2 < bi)) {
      bd = d2;
      bi = i2;
    }
  }
  *medoid = bi;
}

unsigned grid_for(int64_t work, int threads) {
  return unsigned(std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 64)));
}

}  // namespace

cudaError_t launch_pad_rows(const void* src, int64_t n, int64_t src_rb, uint8_t* dst, int64_t dst_rb,
                            cudaStream_t s) {
  if (src_rb == dst_rb) return cudaMemcpyAsync(dst, src, size_t(n * dst_rb), cudaMemcpyDeviceToDevice, s);
  pad_rows_kernel<<<grid_for(n * dst_rb, 256), 256, 0, s>>>(static_cast<const uint8_t*>(src), n, src_rb, dst,
                                                            dst_rb);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const DevData& D, DevStatus* st, cudaStream_t s) {
  if (D.dtype != kF32) return cudaSuccess;
  check_finite_kernel<<<grid_for(D.n * D.d, 256), 256, 0, s>>>(reinterpret_cast<const float*>(D.X), D.n,
                                                               D.row_bytes / 4, D.d, st);
  return cudaGetLastError();
}

cudaError_t launch_validate_csr(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz,
                                DevStatus* st, cudaStream_t s) {
  validate_csr_kernel<<<grid_for(std::max(n, nnz), 256), 256, 0, s>>>(row_ptr, col, n, nnz, st);
  return cudaGetLastError();
}

cudaError_t launch_clean_count(const int64_t* row_ptr, const int32_t* col, int64_t n, int32_t* cnt,
                               unsigned long long* dropped, cudaStream_t s) {
  clean_count_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(row_ptr, col, n, cnt, dropped);
  return cudaGetLastError();
}

cudaError_t launch_clean_write(const int64_t* row_ptr, const int32_t* col, int64_t n,
                               const int64_t* new_row_ptr, int32_t* new_col, cudaStream_t s) {
  clean_write_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(row_ptr, col, n, new_row_ptr, new_col);
  return cudaGetLastError();
}

cudaError_t launch_scan_counts(const int32_t* cnt, int64_t n, int64_t* row_ptr, int64_t* block_sums,
                               int32_t* max_deg, cudaStream_t s) {
  const int64_t nblk = (n + kChunk - 1) / kChunk;
  cudaError_t err = cudaMemsetAsync(max_deg, 0, sizeof(int32_t), s);
  if (err != cudaSuccess) return err;
  count_block_sums<<<unsigned(nblk), kThreads, 0, s>>>(cnt, n, block_sums, max_deg);
  scan_sums_serial<<<1, 1024, 0, s>>>(block_sums, nblk);
  count_write<<<unsigned(nblk), kThreads, 0, s>>>(cnt, n, block_sums, row_ptr);
  return cudaGetLastError();
}

int64_t medoid_blocks(int64_t n) { return std::min<int64_t>((n + 255) / 256, 2048); }

// Candidate rows of width kk + nr: the kk nearest neighbours of p, then nr ids
// drawn uniformly from the other points by a counter-based generator
// (splitmix64 of seed, p and j), repeated ids left for the cleaning pass.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void add_random_candidates_kernel(const int32_t* __restrict__ knn, int kk, int64_t n, int nr,
                                             uint64_t seed, int32_t* __restrict__ out) {
  const int w = kk + nr;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * w; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = i / w;
    const int j = int(i % w);
    if (j < kk) {
      out[i] = knn[p * kk + j];
    } else {
      const uint64_t h = splitmix64(seed ^ splitmix64(uint64_t(p) * 131ull + uint64_t(j - kk)));
      int64_t v = int64_t(h % uint64_t(n - 1));
      if (v >= p) ++v;  // every point but p
      out[i] = int32_t(v);
    }
  }
}

cudaError_t launch_add_random_candidates(const int32_t* knn, int kk, int64_t n, int nr, uint64_t seed, int32_t* out,
                                         cudaStream_t s) {
  add_random_candidates_kernel<<<1024, 256, 0, s>>>(knn, kk, n, nr, seed, out);
  return cudaGetLastError();
}

// row_ptr of the slice of a graph that keeps the rows of [lo, hi): every row
// outside is empty and the kept rows keep their edges (col starts at lo's).
__global__ void slice_row_ptr_kernel(const int64_t* __restrict__ row_ptr, int64_t n, int64_t lo, int64_t hi,
                                     int64_t* __restrict__ out) {
  const int64_t e_lo = row_ptr[lo], e_hi = row_ptr[hi];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = row_ptr[i];
    out[i] = (e < e_lo ? e_lo : (e > e_hi ? e_hi : e)) - e_lo;
  }
}

cudaError_t launch_slice_row_ptr(const int64_t* row_ptr, int64_t n, int64_t lo, int64_t hi, int64_t* out,
                                 cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 256) / 256, 4096);
  slice_row_ptr_kernel<<<unsigned(blocks), 256, 0, s>>>(row_ptr, n, lo, hi, out);
  return cudaGetLastError();
}

cudaError_t launch_medoid(const DevData& D, double* mean, double* block_best, int64_t* medoid,
                          cudaStream_t s) {
  if (D.dtype == kU8) {
    // block_best has room for 2 * medoid_blocks(n) >= d doubles of scratch only when n is
    // large; the column sums live in `mean` reinterpreted, finished in place.
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(mean);
    cudaError_t err = cudaMemsetAsync(sums, 0, size_t(D.d) * 8, s);
    if (err != cudaSuccess) return err;
    const dim3 grid(unsigned((D.d + 127) / 128), unsigned((D.n + 4095) / 4096));
    mean_u8_sum_kernel<<<grid, 128, 0, s>>>(D.X, D.n, D.row_bytes, D.d, sums);
    mean_u8_finish_kernel<<<unsigned((D.d + 127) / 128), 128, 0, s>>>(sums, D.n, D.d, mean);
  } else {
    mean_f32_kernel<<<unsigned(D.d), 32, 0, s>>>(D.X, D.n, D.row_bytes, D.d, mean);
  }
  const int64_t nb = medoid_blocks(D.n);
  nearest_mean_kernel<<<unsigned(nb), 256, 0, s>>>(D.X, D.n, D.row_bytes, D.d, D.dtype, mean, block_best);
  pick_medoid_kernel<<<1, 32, 0, s>>>(block_best, nb, medoid);
  return cudaGetLastError();
}

}  // namespace rpk
