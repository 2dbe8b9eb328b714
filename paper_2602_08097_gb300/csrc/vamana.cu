// Vamana graph construction on the GPU (§2.1, the "fast preprocessing"
// construction; §4.1 builds every base index with it, alpha1 = 1.2,
// L_build = 75).  The paper treats the construction as a black box; this is
// the batched reading the oracle states:
//
//   The graph starts empty.  Points are inserted in the caller's order, in
//   batches of 1, 2, 4, ... points (at most max_batch).  Every point p of a
//   batch searches the graph as it stood when the batch began (Algorithm 2,
//   list size L; its first vcap visited points V_p, in expansion order) and
//   gets N_out(p) <- RobustPrune(p, V_p, alpha, R) (Algorithm 1, sorted; its
//   first step adds the current N_out(p) and drops p).  Then every point j
//   kept by some p of the batch takes those p as back edges, ascending by id
//   (at most 512 of them, the smallest ids), after its current list; a list
//   that grows past R is pruned again, N_out(j) <- RobustPrune(j, merged,
//   alpha, R).
//
// One batch on the device: the search kernel (queries are the batch's own
// rows, the graph is read from the fixed-capacity adjacency, the visited
// points are recorded), a candidate kernel (visited minus p, then the current
// list minus the visited ones: the union without repeats), the library's
// prune kernels over these batch-local rows, a write-back, and the back-edge
// kernels (count per target, scatter, sort each target's senders, merge,
// prune the lists that overflow, write back).
#include <algorithm>
#include <vector>

#include "internal.h"

namespace rpk {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kMaxSenders = 512;  // back edges a point takes per batch (the smallest sender ids)

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Candidate row i of the batch: V_i without the point itself (expansion
// order), then the point's current out-neighbours that are not in V_i.  V_i
// holds distinct points and so does a list, so the row holds no repeat.
__global__ void candidates_kernel(const int32_t* __restrict__ pts, int64_t nb, const int32_t* __restrict__ visited,
                                  const int32_t* __restrict__ vis_cnt, int vcap, const int32_t* __restrict__ nbr,
                                  const int32_t* __restrict__ deg, int R, int32_t* __restrict__ cand,
                                  int32_t* __restrict__ cnt, unsigned long long* __restrict__ cut) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < nb; i += warps) {
    const int32_t p = pts[i];
    const int vc = vis_cnt[i];
    const int nv = vc < vcap ? vc : vcap;
    if (vc > vcap && lane == 0) atomicAdd(cut, 1ull);
    const int32_t* V = visited + i * int64_t(vcap);
    int32_t* row = cand + i * int64_t(vcap + R);
    int out = 0;
    for (int j0 = 0; j0 < nv; j0 += 32) {
      const int j = j0 + lane;
      const int32_t v = j < nv ? V[j] : -1;
      const bool keep = j < nv && v != p;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) row[out + __popc(m & lanemask_lt())] = v;
      out += __popc(m);
    }
    const int dp = deg[p];
    const int32_t* np = nbr + int64_t(p) * R;
    for (int e0 = 0; e0 < dp; e0 += 32) {
      const int e = e0 + lane;
      const int32_t v = e < dp ? np[e] : -1;
      bool keep = e < dp;
      for (int j = 0; keep && j < nv; ++j) keep = V[j] != v;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) row[out + __popc(m & lanemask_lt())] = v;
      out += __popc(m);
    }
    if (lane == 0) cnt[i] = out;
  }
}

// Row i of a padded buffer (stride `stride`, cnt[i] entries) -> CSR at row_ptr[i].
__global__ void compact_rows_kernel(const int32_t* __restrict__ src, int64_t stride, const int64_t* __restrict__ src_off,
                                    const int32_t* __restrict__ cnt, int64_t rows, const int64_t* __restrict__ row_ptr,
                                    int32_t* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < rows; i += warps) {
    const int32_t* a = src + (src_off ? src_off[i] : i * stride);
    int32_t* b = col + row_ptr[i];
    for (int j = lane; j < cnt[i]; j += 32) b[j] = a[j];
  }
}

// The pruned rows back into the adjacency: N_out(pts[i]) <- row i.
__global__ void write_back_kernel(const int32_t* __restrict__ pts, int64_t rows, const int64_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ kept_col, const int32_t* __restrict__ kept_cnt,
                                  int32_t* __restrict__ nbr, int32_t* __restrict__ deg, int R) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < rows; i += warps) {
    const int32_t p = pts[i];
    const int k = kept_cnt[i];
    const int32_t* a = kept_col + row_ptr[i];
    for (int j = lane; j < k; j += 32) nbr[int64_t(p) * R + j] = a[j];
    if (lane == 0) deg[p] = k;
  }
}

// Back edges, step 1: how many batch points name each j; every j met for
// the first time gets a slot in jlist.
__global__ void back_count_kernel(const int32_t* __restrict__ pts, int64_t nb, const int32_t* __restrict__ nbr,
                                  const int32_t* __restrict__ deg, int R, int32_t* __restrict__ pend,
                                  int32_t* __restrict__ slot, int32_t* __restrict__ jlist, int32_t* __restrict__ nj) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nb * R; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t / R;
    const int e = int(t % R);
    const int32_t p = pts[i];
    if (e >= deg[p]) continue;
    const int32_t j = nbr[int64_t(p) * R + e];
    if (atomicAdd(&pend[j], 1) == 0) {
      const int s = atomicAdd(nj, 1);
      jlist[s] = j;
      slot[j] = s;
    }
  }
}

__global__ void slot_counts_kernel(const int32_t* __restrict__ jlist, int64_t nj, const int32_t* __restrict__ pend,
                                   int32_t* __restrict__ out) {
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nj; s += int64_t(gridDim.x) * blockDim.x)
    out[s] = pend[jlist[s]];
}

// Back edges, step 2: each sender p into its target's segment (any order).
__global__ void back_scatter_kernel(const int32_t* __restrict__ pts, int64_t nb, const int32_t* __restrict__ nbr,
                                    const int32_t* __restrict__ deg, int R, const int32_t* __restrict__ slot,
                                    const int64_t* __restrict__ seg_ptr, int32_t* __restrict__ cursor,
                                    int32_t* __restrict__ seg) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nb * R; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t / R;
    const int e = int(t % R);
    const int32_t p = pts[i];
    if (e >= deg[p]) continue;
    const int32_t j = nbr[int64_t(p) * R + e];
    const int s = slot[j];
    seg[seg_ptr[s] + atomicAdd(&cursor[s], 1)] = p;
  }
}

// Back edges, step 3, one warp per target j: its kMaxSenders smallest senders
// in ascending order, the merged list N_out(j) followed by those not already
// in it; a list of at most R points is written at once, a longer one is
// queued (ov_*) for RobustPrune.  pend[j] is reset.  The senders of j are
// distinct points.  Up to kMaxSenders of them are ordered by rank (the count
// of smaller ones); from more, a bisection on the id value first finds the
// bound below which exactly kMaxSenders lie and moves those to the front of
// the segment (in place, in their order there), which are then ranked.
__global__ void back_merge_kernel(const int32_t* __restrict__ jlist, int64_t nj, const int64_t* __restrict__ seg_ptr,
                                  int32_t* __restrict__ seg, int32_t* __restrict__ sorted,
                                  int32_t* __restrict__ nbr, int32_t* __restrict__ deg, int R,
                                  int32_t* __restrict__ pend, int32_t* __restrict__ ov_raw,
                                  int32_t* __restrict__ ov_slot, int32_t* __restrict__ ov_cnt,
                                  int32_t* __restrict__ n_ov) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t s = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < nj; s += warps) {
    const int32_t j = jlist[s];
    const int64_t a = seg_ptr[s];
    const int m = int(seg_ptr[s + 1] - a);
    // a point takes at most kMaxSenders back edges per batch (the smallest
    // sender ids), which bounds every list the prune sees
    const int ms = m < kMaxSenders ? m : kMaxSenders;
    if (m > ms) {
      // the least bound t with #{senders < t} >= ms: then exactly ms lie below it
      long long lo = 0, hi = 0x80000000ll;  // #{< lo} < ms <= #{< hi}
      while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        int cnt = 0;
        for (int x = lane; x < m; x += 32) cnt += seg[a + x] < mid;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (cnt >= ms) hi = mid;
        else lo = mid;
      }
      int w = 0;  // move the ms senders below hi to the front (w <= x: in place)
      for (int x0 = 0; x0 < m; x0 += 32) {
        const int x = x0 + lane;
        const int32_t v = x < m ? seg[a + x] : 0;
        const bool take = x < m && v < hi;
        const unsigned msk = __ballot_sync(0xffffffffu, take);
        __syncwarp();
        if (take) seg[a + w + __popc(msk & lanemask_lt())] = v;
        w += __popc(msk);
        __syncwarp();
      }
    }
    for (int x = lane; x < ms; x += 32) {
      const int32_t v = seg[a + x];
      int r = 0;
      for (int y = 0; y < ms; ++y) r += seg[a + y] < v;
      sorted[a + r] = v;
    }
    __syncwarp();
    const int dj = deg[j];
    int32_t* nj_row = nbr + int64_t(j) * R;
    // the senders not already in N_out(j), in ascending order
    int fresh = 0;
    for (int x0 = 0; x0 < ms; x0 += 32) {
      const int x = x0 + lane;
      const int32_t v = x < ms ? sorted[a + x] : -1;
      bool keep = x < ms;
      for (int e = 0; keep && e < dj; ++e) keep = nj_row[e] != v;
      const unsigned msk = __ballot_sync(0xffffffffu, keep);
      if (keep) sorted[a + fresh + __popc(msk & lanemask_lt())] = v;  // in place: fresh <= x
      fresh += __popc(msk);
      __syncwarp();
    }
    if (dj + fresh <= R) {
      for (int x = lane; x < fresh; x += 32) nj_row[dj + x] = sorted[a + x];
      __syncwarp();
      if (lane == 0) deg[j] = dj + fresh;
    } else {
      int o = 0;
      if (lane == 0) o = atomicAdd(n_ov, 1);
      o = __shfl_sync(0xffffffffu, o, 0);
      // room for R + m ids per target: seg_ptr[s] + s * R
      int32_t* row = ov_raw + a + s * int64_t(R);
      for (int e = lane; e < dj; e += 32) row[e] = nj_row[e];
      for (int x = lane; x < fresh; x += 32) row[dj + x] = sorted[a + x];
      if (lane == 0) {
        ov_slot[o] = int32_t(s);
        ov_cnt[o] = dj + fresh;
      }
    }
    if (lane == 0) pend[j] = 0;
  }
}

__global__ void ov_prep_kernel(const int32_t* __restrict__ ov_slot, int64_t no, const int32_t* __restrict__ jlist,
                               const int64_t* __restrict__ seg_ptr, int R, int32_t* __restrict__ ov_pts,
                               int64_t* __restrict__ ov_src) {
  for (int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; o < no; o += int64_t(gridDim.x) * blockDim.x) {
    const int s = ov_slot[o];
    ov_pts[o] = jlist[s];
    ov_src[o] = seg_ptr[s] + int64_t(s) * R;
  }
}

unsigned grid_warps(int64_t rows) {
  const int64_t b = (rows + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return unsigned(std::max<int64_t>(1, std::min<int64_t>(b, 65535)));
}
unsigned grid_threads(int64_t items) {
  const int64_t b = (items + 255) / 256;
  return unsigned(std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20)));
}

}  // namespace

cudaError_t launch_vamana_candidates(const int32_t* pts, int64_t nb, const int32_t* visited, const int32_t* vis_cnt,
                                     int vcap, const int32_t* nbr, const int32_t* deg, int R, int32_t* cand,
                                     int32_t* cnt, unsigned long long* cut, cudaStream_t s) {
  candidates_kernel<<<grid_warps(nb), kWarpsPerBlock * 32, 0, s>>>(pts, nb, visited, vis_cnt, vcap, nbr, deg, R, cand,
                                                                  cnt, cut);
  return cudaGetLastError();
}

cudaError_t launch_compact_rows(const int32_t* src, int64_t stride, const int64_t* src_off, const int32_t* cnt,
                                int64_t rows, const int64_t* row_ptr, int32_t* col, cudaStream_t s) {
  compact_rows_kernel<<<grid_warps(rows), kWarpsPerBlock * 32, 0, s>>>(src, stride, src_off, cnt, rows, row_ptr, col);
  return cudaGetLastError();
}

cudaError_t launch_vamana_write_back(const int32_t* pts, int64_t rows, const int64_t* row_ptr, const int32_t* kept_col,
                                     const int32_t* kept_cnt, int32_t* nbr, int32_t* deg, int R, cudaStream_t s) {
  write_back_kernel<<<grid_warps(rows), kWarpsPerBlock * 32, 0, s>>>(pts, rows, row_ptr, kept_col, kept_cnt, nbr, deg,
                                                                    R);
  return cudaGetLastError();
}

cudaError_t launch_back_count(const int32_t* pts, int64_t nb, const int32_t* nbr, const int32_t* deg, int R,
                              int32_t* pend, int32_t* slot, int32_t* jlist, int32_t* nj, cudaStream_t s) {
  back_count_kernel<<<grid_threads(nb * R), 256, 0, s>>>(pts, nb, nbr, deg, R, pend, slot, jlist, nj);
  return cudaGetLastError();
}

cudaError_t launch_slot_counts(const int32_t* jlist, int64_t nj, const int32_t* pend, int32_t* out, cudaStream_t s) {
  slot_counts_kernel<<<grid_threads(nj), 256, 0, s>>>(jlist, nj, pend, out);
  return cudaGetLastError();
}

cudaError_t launch_back_scatter(const int32_t* pts, int64_t nb, const int32_t* nbr, const int32_t* deg, int R,
                                const int32_t* slot, const int64_t* seg_ptr, int32_t* cursor, int32_t* seg,
                                cudaStream_t s) {
  back_scatter_kernel<<<grid_threads(nb * R), 256, 0, s>>>(pts, nb, nbr, deg, R, slot, seg_ptr, cursor, seg);
  return cudaGetLastError();
}

cudaError_t launch_back_merge(const int32_t* jlist, int64_t nj, const int64_t* seg_ptr, int32_t* seg,
                              int32_t* sorted, int32_t* nbr, int32_t* deg, int R, int32_t* pend, int32_t* ov_raw,
                              int32_t* ov_slot, int32_t* ov_cnt, int32_t* n_ov, cudaStream_t s) {
  back_merge_kernel<<<grid_warps(nj), kWarpsPerBlock * 32, 0, s>>>(jlist, nj, seg_ptr, seg, sorted, nbr, deg, R, pend,
                                                                  ov_raw, ov_slot, ov_cnt, n_ov);
  return cudaGetLastError();
}

cudaError_t launch_ov_prep(const int32_t* ov_slot, int64_t no, const int32_t* jlist, const int64_t* seg_ptr, int R,
                           int32_t* ov_pts, int64_t* ov_src, cudaStream_t s) {
  ov_prep_kernel<<<grid_threads(no), 256, 0, s>>>(ov_slot, no, jlist, seg_ptr, R, ov_pts, ov_src);
  return cudaGetLastError();
}

}  // namespace rpk
