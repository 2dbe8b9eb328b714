// Batched GreedySearch (Algorithm 2) and k-recall@k (§4).
//
// One warp runs one query at a time; warps take queries from an atomic
// counter.  The search list is kept sorted by (distance, id) in shared
// memory, so "the closest unexpanded member" of Algorithm 2 is the first
// member without its visited bit, and "retain the closest L" is a cut after
// a merge.
//
// Algorithm 2 keeps a set: adding a point that is already in the list has
// no effect.  A point that was in the list and was cut may be added again by
// a later neighbour list, and then it is cut again at once: from the first cut
// on the list holds L members and its L-th (distance, id) only decreases, so
// the point still lies behind it.  (An expanded point that is cut is the same
// case: it comes back behind the L-th and is never the closest unexpanded
// member.)  So the only membership test the search needs is "is v in the
// list now?", which a binary search of the sorted list answers exactly at the
// position where v would be merged.  A small direct-mapped cache of recently
// met ids in shared memory skips most repeated distance computations; a miss
// only costs one more distance, never a different result.
//
// Neighbours are added 32 at a time, each batch merged and cut to L before the
// next; the L closest of a union are the L closest of the L closest of its
// parts, so this equals adding the whole list and cutting once.
//
// Ordering: uint8 distances are exact integers.  float32 distances (summed
// per 32-dimension slice) carry a rigorous single-precision error bound; when
// two intervals overlap, both distances are recomputed in float-float
// arithmetic (bound about d 2^-46 relative), and only if those intervals still
// overlap in binary64 (index order, no fused multiply-add), so every
// comparison agrees with the binary64 reading.
#include <cfloat>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace rpk {

namespace {

constexpr int kWarps = 4;  // warps (queries in flight) per CTA
constexpr unsigned kVisited = 0x80000000u;
constexpr unsigned kIdMask = 0x7fffffffu;

struct SearchArgs {
  const uint8_t* X;
  int64_t row_bytes;
  int d;
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  int64_t start;
  const SearchGraph* graphs;  // per-query graphs (with q_graph), or nullptr
  const int32_t* q_graph;     // index into graphs per query, or nullptr
  const int32_t* q_L;         // list size per query (k <= q_L <= L), or nullptr
  const uint8_t* Q;
  int64_t nq;
  int L;                      // largest list size; sizes the shared memory
  int k;
  int32_t* out_ids;
  float* out_dists;
  int cache_bits;             // log2 of the id-cache entries per warp
  unsigned int* work;
  DevStatus* status;
  // graph construction (Vamana): query i is base point q_point[i]; the graph
  // is held as adj_deg[v] ids at col + v * adj_stride; the expanded points of
  // query i go to visited[i * visited_cap ..] (the first visited_cap of them),
  // their number to visited_cnt[i]
  const int32_t* q_point;
  const int32_t* adj_deg;
  int64_t adj_stride;
  int32_t* visited;
  int32_t* visited_cnt;
  int visited_cap;
};

struct WarpSmem {
  unsigned* key;   // the list: distance bits, sorted by (distance, id)
  unsigned* idv;   // its ids (| kVisited once expanded)
  double* d64;     // float data: binary64 distances of the list (NaN until computed)
  unsigned* ckey;  // a batch's new members, then
  unsigned* cid;
  int* clo;        // their insertion points (sorted: the merge's shift table)
  double* cd64;
  uint8_t* q;
  unsigned* cache;  // direct-mapped ids met by this query (0xffffffff = empty)
};

__host__ __device__ inline size_t list_cap(int L) { return (size_t(L) + 3) & ~size_t(3); }

__host__ __device__ inline size_t warp_bytes(int L, int64_t row_bytes, bool f32, int cache_bits) {
  const size_t cap = list_cap(L);
  size_t b = cap * 8 + 32 * 12;  // list keys + ids; batch keys, ids, insertion points
  if (f32) b += cap * 8 + 32 * 8;
  b += size_t(row_bytes);
  b += size_t(4) << cache_bits;
  return (b + 127) & ~size_t(127);
}

__device__ inline WarpSmem carve(unsigned char* base, int L, int64_t row_bytes, bool f32, int cache_bits) {
  WarpSmem w;
  const size_t cap = list_cap(L);
  unsigned char* p = base;
  w.cache = reinterpret_cast<unsigned*>(p);
  p += size_t(4) << cache_bits;
  if (f32) {
    w.d64 = reinterpret_cast<double*>(p);
    p += cap * 8;
    w.cd64 = reinterpret_cast<double*>(p);
    p += 32 * 8;
  } else {
    w.d64 = w.cd64 = nullptr;
  }
  w.q = p;  // 16-byte aligned: cap is a multiple of 4 and row_bytes of 16
  p += row_bytes;
  w.key = reinterpret_cast<unsigned*>(p);
  p += cap * 4;
  w.idv = reinterpret_cast<unsigned*>(p);
  p += cap * 4;
  w.ckey = reinterpret_cast<unsigned*>(p);
  p += 32 * 4;
  w.cid = reinterpret_cast<unsigned*>(p);
  p += 32 * 4;
  w.clo = reinterpret_cast<int*>(p);
  return w;
}

// d2(q, v) in the search's working precision, as order-preserving bits.
// uint8: d2 = |q|^2 + |x|^2 - 2 <q, x> from dp4a alone, `qn` = |q|^2 (an
// identity of integers, exact in 32-bit modular arithmetic since d2 < 2^32).
template <int DT>
__device__ __forceinline__ unsigned dist_bits(const uint8_t* __restrict__ q, const uint8_t* __restrict__ x,
                                              int64_t row_bytes, unsigned qn) {
  const uint4* pq = reinterpret_cast<const uint4*>(q);
  const uint4* px = reinterpret_cast<const uint4*>(x);
  if constexpr (DT == kU8) {
    unsigned dot = 0, xn = 0;
    for (int64_t c = 0; c < row_bytes / 16; ++c) {
      const uint4 a = pq[c], b = __ldg(px + c);
      dot = __dp4a(a.x, b.x, dot);
      dot = __dp4a(a.y, b.y, dot);
      dot = __dp4a(a.z, b.z, dot);
      dot = __dp4a(a.w, b.w, dot);
      xn = __dp4a(b.x, b.x, xn);
      xn = __dp4a(b.y, b.y, xn);
      xn = __dp4a(b.z, b.z, xn);
      xn = __dp4a(b.w, b.w, xn);
    }
    return qn + xn - 2u * dot;
  } else {
    // summed per 32-dimension slice (slice_rel_bound)
    float acc = 0.f;
    for (int64_t c0 = 0; c0 < row_bytes / 16; c0 += 8) {
      float part = 0.f;
      const int64_t c1 = c0 + 8 < row_bytes / 16 ? c0 + 8 : row_bytes / 16;
      for (int64_t c = c0; c < c1; ++c) {
        const uint4 a = pq[c], b = __ldg(px + c);
        float t;
        t = __uint_as_float(a.x) - __uint_as_float(b.x); part = fmaf(t, t, part);
        t = __uint_as_float(a.y) - __uint_as_float(b.y); part = fmaf(t, t, part);
        t = __uint_as_float(a.z) - __uint_as_float(b.z); part = fmaf(t, t, part);
        t = __uint_as_float(a.w) - __uint_as_float(b.w); part = fmaf(t, t, part);
      }
      acc += part;
    }
    return __float_as_uint(acc);
  }
}

// Total order on (distance, id) entries.  For float data `d64a`/`d64b` point to
// the slots caching the binary64 distances (NaN until computed).
template <int DT>
__device__ __forceinline__ bool entry_less(unsigned ka, unsigned ia, double* d64a, unsigned kb, unsigned ib,
                                           double* d64b, const SearchArgs& a, const uint8_t* q, float E,
                                           float Eabs) {
  if constexpr (DT == kU8) {
    return ka < kb || (ka == kb && ia < ib);
  } else {
    if (ia == ib) return false;  // the same point: never less than itself (no binary64 needed)
    const float fa = __uint_as_float(ka), fb = __uint_as_float(kb);
    if (sure_less(fa, fb, E, Eabs)) return true;
    if (sure_less(fb, fa, E, Eabs)) return false;
    const float* qf = reinterpret_cast<const float*>(q);
    const int64_t stride = a.row_bytes / 4;
    const float* X = reinterpret_cast<const float*>(a.X);
    double xa = *d64a, xb = *d64b;
    // float-float first (cached, sign-marked), binary64 only if still undecided
    if (isnan(xa)) *d64a = xa = -ff_d2(qf, X + int64_t(ia) * stride, a.row_bytes);
    if (isnan(xb)) *d64b = xb = -ff_d2(qf, X + int64_t(ib) * stride, a.row_bytes);
    const int o = slot_order(xa, xb, ff_bound(a.d));
    if (o >= 0) return o == 1;
    if (signbit(xa)) {
      xa = canon_d2_f32(qf, X + int64_t(ia) * stride, a.d);
      *d64a = xa;
      atomicAdd(&a.status->fp64_search, 1ull);
    }
    if (signbit(xb)) {
      xb = canon_d2_f32(qf, X + int64_t(ib) * stride, a.d);
      *d64b = xb;
      atomicAdd(&a.status->fp64_search, 1ull);
    }
    return xa < xb || (xa == xb && ia < ib);
  }
}

template <int DT>
__global__ void __launch_bounds__(kWarps * 32, 9) search_kernel(SearchArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool f32 = DT == kF32;
  WarpSmem S = carve(smem_raw + size_t(w) * warp_bytes(a.L, a.row_bytes, f32, a.cache_bits), a.L, a.row_bytes, f32,
                     a.cache_bits);
  const int cshift = 32 - a.cache_bits;
  const int centries = 1 << a.cache_bits;
  const float E = slice_rel_bound(a.d), Eabs = abs_bound(a.d);
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);

  for (;;) {
    unsigned qi = 0;
    if (lane == 0) qi = atomicAdd(a.work, 1u);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    if (qi >= a.nq) break;
    const int64_t* __restrict__ row_ptr = a.row_ptr;
    const int32_t* __restrict__ col = a.col;
    int64_t start = a.start;
    if (a.q_graph) {
      const SearchGraph g = a.graphs[a.q_graph[qi]];
      row_ptr = g.row_ptr;
      col = g.col;
      start = g.start;
    }
    const int L = a.q_L ? a.q_L[qi] : a.L;
    // stage the query row
    const uint4* src = reinterpret_cast<const uint4*>(
        a.q_point ? a.X + int64_t(a.q_point[qi]) * a.row_bytes : a.Q + int64_t(qi) * a.row_bytes);
    for (int c = lane; c < a.row_bytes / 16; c += 32) reinterpret_cast<uint4*>(S.q)[c] = src[c];
    for (int c = lane; c < centries; c += 32) S.cache[c] = 0xffffffffu;
    __syncwarp();
    unsigned qn = 0;  // uint8: |q|^2
    if constexpr (DT == kU8) {
      for (int w4 = lane; w4 < a.row_bytes / 4; w4 += 32) {
        const unsigned qw = reinterpret_cast<const unsigned*>(S.q)[w4];
        qn = __dp4a(qw, qw, qn);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) qn += __shfl_xor_sync(0xffffffffu, qn, o);
    }

    unsigned* const keyc = S.key;
    unsigned* const idc = S.idv;
    double* const dc = S.d64;
    int size = 1;
    int f = 0;  // the members before index f are all expanded
    if (lane == 0) {
      const unsigned s = unsigned(start);
      keyc[0] = dist_bits<DT>(S.q, a.X + int64_t(s) * a.row_bytes, a.row_bytes, qn);
      idc[0] = s;
      if (f32) dc[0] = qnan;
      S.cache[(s * 0x9E3779B1u) >> cshift] = s;
    }
    __syncwarp();

    int64_t iters = 0;
    for (;;) {
      // the closest member not yet expanded
      int pos = -1;
      for (int c0 = f & ~31; c0 < size; c0 += 32) {
        const int i = c0 + lane;
        const bool open = i < size && !(idc[i] & kVisited);
        const unsigned b = __ballot_sync(0xffffffffu, open);
        if (b) {
          pos = c0 + __ffs(b) - 1;
          break;
        }
      }
      if (pos < 0) break;
      if (++iters > a.n + 1) {  // cannot happen: each point is expanded at most once
        if (lane == 0) raise_status(a.status, kDevOverflow, qi);
        break;
      }
      const unsigned ps = idc[pos] & kIdMask;
      __syncwarp();
      if (lane == 0) idc[pos] |= kVisited;
      __syncwarp();
      f = pos + 1;
      if (a.visited && lane == 0 && iters <= a.visited_cap) a.visited[int64_t(qi) * a.visited_cap + iters - 1] = int32_t(ps);
      int64_t e0, e1;
      if (a.adj_deg) {
        e0 = int64_t(ps) * a.adj_stride;
        e1 = e0 + a.adj_deg[ps];
      } else {
        e0 = row_ptr[ps];
        e1 = row_ptr[ps + 1];
      }
      for (int64_t eb = e0; eb < e1; eb += 32) {
        // ---- new neighbours of this batch
        const int64_t e = eb + lane;
        bool fresh = false;
        unsigned v = 0;
        if (e < e1) {
          v = unsigned(col[e]);
          // a row holds distinct ids, so lanes that share a cache entry hold
          // different ids: whichever write lands, no lane skips a new id
          const unsigned h = (v * 0x9E3779B1u) >> cshift;
          fresh = S.cache[h] != v;
          if (fresh) S.cache[h] = v;
        }
        if (!__any_sync(0xffffffffu, fresh)) continue;
        unsigned kv = 0xffffffffu;
        if (fresh) kv = dist_bits<DT>(S.q, a.X + int64_t(v) * a.row_bytes, a.row_bytes, qn);
        // A full list keeps only entries before its L-th: a point behind it
        // would be cut right after the merge, so it skips the merge.
        bool enters = fresh;
        double cand_d64 = qnan;
        if (enters && size == L) {
          enters = entry_less<DT>(kv, v, f32 ? &cand_d64 : nullptr, keyc[L - 1],
                                  idc[L - 1] & kIdMask, f32 ? &dc[L - 1] : nullptr, a, S.q,
                                  E, Eabs);
        }
        // Already in the list?  Its entry sits exactly where v would be
        // merged; otherwise `lo` (the members before v) is v's insertion point.
        int lo = 0;
        if (enters) {
          int hi = size;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const bool bl = entry_less<DT>(keyc[mid], idc[mid] & kIdMask,
                                           f32 ? &dc[mid] : nullptr, kv, v, f32 ? &cand_d64 : nullptr, a,
                                           S.q, E, Eabs);
            if (bl) lo = mid + 1;
            else hi = mid;
          }
          if (lo < size && (idc[lo] & kIdMask) == v) enters = false;
        }
        const unsigned fm = __ballot_sync(0xffffffffu, enters);
        const int nf = __popc(fm);
        if (nf == 0) continue;
        // ---- the new members, compacted into lanes 0..nf-1
        if (enters) {
          const int r = __popc(fm & ((1u << lane) - 1u));
          S.ckey[r] = kv;
          S.cid[r] = v;
          S.clo[r] = lo;
          if (f32) S.cd64[r] = cand_d64;
        }
        __syncwarp();
        unsigned myk = 0xffffffffu, myid = 0xffffffffu;
        int mylo = 0x7fffffff;
        double myd = qnan;
        if (lane < nf) {
          myk = S.ckey[lane];
          myid = S.cid[lane];
          mylo = S.clo[lane];
          if (f32) myd = S.cd64[lane];
        }
        // ---- sort them: bitonic over the smallest power of two >= nf lanes
        // (empty lanes sort last).  Different insertion points order two new
        // members without a distance: a list member lies between them.
        if (nf > 1) {
          const int w = 1 << (32 - __clz(nf - 1));
          for (int kk = 2; kk <= w; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
              const unsigned ok = __shfl_xor_sync(0xffffffffu, myk, j);
              const unsigned oi = __shfl_xor_sync(0xffffffffu, myid, j);
              const int olo = __shfl_xor_sync(0xffffffffu, mylo, j);
              // dec: 1 = my entry comes first, 0 = the partner's, -1 = undecided
              int dec;
              const bool me_empty = myid == 0xffffffffu, o_empty = oi == 0xffffffffu;
              if (me_empty && o_empty) dec = lane < (lane ^ j) ? 1 : 0;
              else if (me_empty) dec = 0;
              else if (o_empty) dec = 1;
              else if (mylo != olo) dec = mylo < olo ? 1 : 0;
              else if (DT == kU8) dec = (myk < ok || (myk == ok && myid < oi)) ? 1 : 0;
              else {
                const float fa = __uint_as_float(myk), fb = __uint_as_float(ok);
                dec = sure_less(fa, fb, E, Eabs) ? 1 : (sure_less(fb, fa, E, Eabs) ? 0 : -1);
              }
              double od = 0.0;
              if constexpr (DT == kF32) {
                // an undecided pair is undecided for both lanes: each brings its
                // own float-float distance, then (still undecided) its binary64
                // one, and both lanes compare the same pair of values
                const float* rowp = reinterpret_cast<const float*>(a.X + int64_t(myid) * a.row_bytes);
                if (dec < 0 && isnan(myd)) myd = -ff_d2(reinterpret_cast<const float*>(S.q), rowp, a.row_bytes);
                od = __shfl_xor_sync(0xffffffffu, myd, j);
                if (dec < 0) dec = slot_order(myd, od, ff_bound(a.d));
                if (dec < 0 && signbit(myd)) {
                  myd = canon_d2_f32(reinterpret_cast<const float*>(S.q), rowp, a.d);
                  atomicAdd(&a.status->fp64_search, 1ull);
                }
                od = __shfl_xor_sync(0xffffffffu, myd, j);
                if (dec < 0) dec = (myd < od || (myd == od && myid < oi)) ? 1 : 0;
              }
              const bool less_me = dec == 1;
              const bool up = (lane & kk) == 0;
              const bool lower = (lane & j) == 0;
              const bool take_partner = (lower == up) ? !less_me : less_me;
              if (take_partner) {
                myk = ok;
                myid = oi;
                mylo = olo;
                myd = od;
              }
            }
          }
          if (lane < nf) S.clo[lane] = mylo;
          __syncwarp();
        }
        // ---- merge in place, back to front: member i moves to i + #{r : clo[r] <= i}
        // and new member r to clo[r] + r; positions from L on are cut.  New
        // positions only grow and never meet, so a chunk read before any write
        // to its range is never clobbered.  Members before clo[0] stay.
        const int first = __shfl_sync(0xffffffffu, mylo, 0);
        for (int c0 = (size - 1) & ~31; c0 >= (first & ~31) && first < size; c0 -= 32) {
          const int i = c0 + lane;
          const bool mv = i >= first && i < size;
          unsigned bk = 0, bi = 0;
          double bd = 0.0;
          int np = L;
          if (mv) {
            bk = keyc[i];
            bi = idc[i];
            if (f32) bd = dc[i];
            int l2 = 1, h2 = nf;  // clo[0] = first <= i
            while (l2 < h2) {
              const int mid = (l2 + h2) >> 1;
              if (S.clo[mid] <= i) l2 = mid + 1;
              else h2 = mid;
            }
            np = i + l2;
          }
          __syncwarp();
          if (mv && np < L) {
            keyc[np] = bk;
            idc[np] = bi;
            if (f32) dc[np] = bd;
          }
          __syncwarp();
        }
        if (lane < nf && mylo + lane < L) {
          keyc[mylo + lane] = myk;
          idc[mylo + lane] = myid;
          if (f32) dc[mylo + lane] = myd;
        }
        __syncwarp();
        size = min(L, size + nf);
        f = min(f, first);
      }
    }
    if (a.visited_cnt && lane == 0) a.visited_cnt[qi] = int32_t(iters < INT32_MAX ? iters : INT32_MAX);
    // ---- the k closest members
    for (int j = lane; j < a.k; j += 32) {
      const bool have = j < size;
      a.out_ids[int64_t(qi) * a.k + j] = have ? int32_t(idc[j] & kIdMask) : -1;
      if (a.out_dists) {
        float dv;
        if (!have) dv = __int_as_float(0x7f800000);
        else if (DT == kU8) dv = float(keyc[j]);
        else dv = __uint_as_float(keyc[j]);
        a.out_dists[int64_t(qi) * a.k + j] = dv;
      }
    }
    __syncwarp();
  }
}

__global__ void recall_kernel(const int32_t* __restrict__ found, int ld_found, const int32_t* __restrict__ truth,
                              int ld_truth, int64_t nq, int k, unsigned long long* hits) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = int64_t(blockIdx.x) * (blockDim.x >> 5) + w;
  if (q >= nq) return;
  const int32_t* f = found + q * ld_found;
  const int32_t* t = truth + q * ld_truth;
  unsigned long long h = 0;
  for (int i = lane; i < k; i += 32) {
    const int32_t v = f[i];
    if (v < 0) continue;
    for (int j = 0; j < k; ++j)
      if (t[j] == v) {
        ++h;
        break;
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
  if (lane == 0 && h) atomicAdd(hits, h);
}

}  // namespace

// The CTAs per SM a configured plan may ask for.
constexpr int kMaxCtasPerSmCap = 16;
constexpr int kMinCacheBits = 8, kMaxCacheBits = 12;
// The default plan stops at 512 entries: a larger cache takes shared memory
// that L1 would otherwise give to the neighbour rows and vectors, and measured
// slower on 1M x 128 uint8 at L = 128 (1,024 entries 6% slower, 4,096 50%).
constexpr int kDefaultMaxCacheBits = 9;

// CTAs of search_kernel<DT> one SM holds with `bytes` of dynamic shared memory
// (registers and shared memory both count), from the occupancy calculator.
template <int DT>
cudaError_t resident_ctas(size_t bytes, size_t max_bytes, int* out) {
  cudaError_t err = cudaFuncSetAttribute(search_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(max_bytes));
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, search_kernel<DT>, kWarps * 32, bytes);
}

// Default plan: the queries in flight hide the latency of each expansion, so
// the search first maximises the CTAs per SM, then takes the largest id cache
// (256 or 512 entries per warp) that keeps that many.  Plans are remembered
// per (dtype, L, row bytes); the occupancy queries run once for each.
struct SearchPlan {
  int bits = kMinCacheBits;
  int ctas = 1;
};

cudaError_t default_plan(bool f32, int L, int64_t row_bytes, SearchPlan* plan) {
  static std::mutex mu;
  static std::map<std::tuple<bool, int, int64_t>, SearchPlan> memo;
  const auto key = std::make_tuple(f32, L, row_bytes);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = memo.find(key);
    if (it != memo.end()) {
      *plan = it->second;
      return cudaSuccess;
    }
  }
  const size_t max_bytes = warp_bytes(L, row_bytes, f32, kMaxCacheBits) * kWarps;
  SearchPlan best;
  int best_ctas = 0;
  for (int b = kMinCacheBits; b <= kDefaultMaxCacheBits; ++b) {
    int nb = 0;
    const size_t bytes = warp_bytes(L, row_bytes, f32, b) * kWarps;
    cudaError_t err = f32 ? resident_ctas<kF32>(bytes, max_bytes, &nb) : resident_ctas<kU8>(bytes, max_bytes, &nb);
    if (err != cudaSuccess) return err;
    if (nb >= best_ctas && nb > 0) {  // ties go to the larger cache
      best_ctas = nb;
      best.bits = b;
      best.ctas = nb;
    }
  }
  if (best_ctas == 0) return cudaErrorInvalidConfiguration;
  best.ctas = std::min(best.ctas, kMaxCtasPerSmCap);
  std::lock_guard<std::mutex> g(mu);
  memo[key] = best;
  *plan = best;
  return cudaSuccess;
}

cudaError_t launch_search(const SearchLaunch& L, cudaStream_t s) {
  SearchArgs a{};
  a.X = L.data.X;
  a.row_bytes = L.data.row_bytes;
  a.d = L.data.d;
  a.n = L.data.n;
  a.row_ptr = L.row_ptr;
  a.col = L.col;
  a.start = L.start;
  a.graphs = L.graphs;
  a.q_graph = L.q_graph;
  a.q_L = L.q_L;
  a.Q = L.Q;
  a.nq = L.nq;
  a.L = L.L;
  a.k = L.k;
  a.out_ids = L.out_ids;
  a.out_dists = L.out_dists;
  a.work = L.work;
  a.status = L.status;
  a.q_point = L.q_point;
  a.adj_deg = L.adj_deg;
  a.adj_stride = L.adj_stride;
  a.visited = L.visited;
  a.visited_cnt = L.visited_cnt;
  a.visited_cap = L.visited_cap;
  const bool f32 = L.data.dtype == kF32;
  SearchPlan plan;
  if (L.cache_bits >= kMinCacheBits && L.cache_bits <= kMaxCacheBits) {  // a configured plan (rp_set_search_config)
    plan.bits = L.cache_bits;
    const size_t bytes = warp_bytes(L.L, L.data.row_bytes, f32, plan.bits) * kWarps;
    cudaError_t err = f32 ? resident_ctas<kF32>(bytes, bytes, &plan.ctas) : resident_ctas<kU8>(bytes, bytes, &plan.ctas);
    if (err != cudaSuccess) return err;
    plan.ctas = std::min(plan.ctas, kMaxCtasPerSmCap);
  } else {
    cudaError_t err = default_plan(f32, L.L, L.data.row_bytes, &plan);
    if (err != cudaSuccess) return err;
  }
  int base_ctas = plan.ctas;
  if (L.ctas_per_sm > 0) base_ctas = std::min(base_ctas, L.ctas_per_sm);
  base_ctas = std::max(base_ctas, 1);
  a.cache_bits = plan.bits;
  const size_t bytes = warp_bytes(L.L, L.data.row_bytes, f32, plan.bits) * kWarps;
  const int64_t want = int64_t(L.num_sms) * base_ctas;
  const int64_t need = (L.nq + kWarps - 1) / kWarps;
  const int grid = int(std::max<int64_t>(1, std::min(want, need)));
  cudaError_t err;
  if (f32) {
    err = cudaFuncSetAttribute(search_kernel<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (err != cudaSuccess) return err;
    search_kernel<kF32><<<grid, kWarps * 32, bytes, s>>>(a);
  } else {
    err = cudaFuncSetAttribute(search_kernel<kU8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (err != cudaSuccess) return err;
    search_kernel<kU8><<<grid, kWarps * 32, bytes, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_recall(const int32_t* found, int ld_found, const int32_t* truth, int ld_truth, int64_t nq, int k,
                          unsigned long long* hits, cudaStream_t s) {
  const int per = 8;
  const int64_t blocks = (nq + per - 1) / per;
  recall_kernel<<<unsigned(blocks), per * 32, 0, s>>>(found, ld_found, truth, ld_truth, nq, k, hits);
  return cudaGetLastError();
}

}  // namespace rpk
