// Internal host-side declarations shared by the library's translation units.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace rpk {

// Vectors on the device: rows padded to a multiple of 128 bytes with zeros
// (padding changes no distance).
struct DevData {
  const uint8_t* X = nullptr;
  int64_t row_bytes = 0;
  int64_t n = 0;
  int d = 0;
  int dtype = 0;
  float scale = 1.f;  // a power of two with max |x| * scale <= 1 (float rows; 1 for uint8)
};

// A source graph for the prune kernels.
struct PruneLaunch {
  DevData data;
  const int64_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const int32_t* bucket_nodes[3] = {nullptr, nullptr, nullptr};  // deg<=64, <=128, >128
  const int32_t* bucket_count = nullptr;                          // device int[3]
  int64_t host_bucket_count[3] = {0, 0, 0};
  int host_max_degree = 0;
  int T = 0;
  int variant = 0;
  int32_t A[kMaxTargets];
  int32_t R[kMaxTargets];
  int32_t* out_col[kMaxTargets];  // scratch, same offsets as row_ptr
  int32_t* out_cnt[kMaxTargets];  // per node
  unsigned int* work = nullptr;   // device unsigned[3], zeroed before the launch
  DevStatus* status = nullptr;
  int num_sms = 0;
  // tile of the degree <= 64 bucket: 0 = two nodes per 128-row MMA, 1 = one
  // node per MMA; CTAs per SM of the tensor-core kernels (0 = all that fit)
  int tile0 = 0;
  int ctas_per_sm = 0;
  // row p of row_ptr/col holds the candidates of point point_of[p] (graph
  // construction prunes batch-local rows); nullptr: row p is point p
  const int32_t* point_of = nullptr;
};

// prune.cu
cudaError_t launch_bucket_nodes(const int64_t* row_ptr, int64_t n, int32_t* lists /* 3*n */,
                                int32_t* counts /* 3 */, cudaStream_t s);
cudaError_t launch_prune(const PruneLaunch& L, cudaStream_t s);
// counts -> row_ptr (per target) and compaction of kept ids into col.
cudaError_t launch_emit_csr(int64_t n, int T, const int64_t* src_row_ptr,
                            int32_t* const* scratch_col, int32_t* const* cnt,
                            int64_t* const* dst_row_ptr, int32_t* const* dst_col,
                            int64_t* block_sums /* T * nblk */, cudaStream_t s);
int64_t emit_csr_blocks(int64_t n);

// Test support: the split-f16 Gram of float rows, 128 rows (rows[g*128 ..]) per group,
// out[(g*128 + i)*128 + j] = G~(row i, row j) of group g, the rows of each 64-row half
// centred on centres[2g + half] when centres is not null (prune.cu)
cudaError_t launch_gram_probe(const DevData& D, const int32_t* rows, const int32_t* centres, int64_t groups,
                              float* out, DevStatus* status, int num_sms, cudaStream_t s);

// prep.cu
cudaError_t launch_pad_rows(const void* src, int64_t n, int64_t src_row_bytes, uint8_t* dst,
                            int64_t dst_row_bytes, cudaStream_t s);
cudaError_t launch_check_finite(const DevData& D, DevStatus* st, cudaStream_t s);
cudaError_t launch_validate_csr(const int64_t* row_ptr, const int32_t* col, int64_t n,
                                int64_t nnz, DevStatus* st, cudaStream_t s);
cudaError_t launch_clean_count(const int64_t* row_ptr, const int32_t* col, int64_t n,
                               int32_t* cnt, unsigned long long* dropped /* [2] */,
                               cudaStream_t s);
cudaError_t launch_clean_write(const int64_t* row_ptr, const int32_t* col, int64_t n,
                               const int64_t* new_row_ptr, int32_t* new_col, cudaStream_t s);
cudaError_t launch_scan_counts(const int32_t* cnt, int64_t n, int64_t* row_ptr,
                               int64_t* block_sums, int32_t* max_deg, cudaStream_t s);
cudaError_t launch_add_random_candidates(const int32_t* knn, int kk, int64_t n, int nr, uint64_t seed, int32_t* out,
                                         cudaStream_t s);
cudaError_t launch_slice_row_ptr(const int64_t* row_ptr, int64_t n, int64_t lo, int64_t hi, int64_t* out,
                                 cudaStream_t s);
cudaError_t launch_medoid(const DevData& D, double* mean /* d */, double* block_best /* 2*nb */,
                          int64_t* medoid, cudaStream_t s);
int64_t medoid_blocks(int64_t n);

// search.cu
// One graph of a mixed search launch (all graphs share the vectors).
struct SearchGraph {
  const int64_t* row_ptr;
  const int32_t* col;
  int64_t start;
  int64_t pad;
};

struct SearchLaunch {
  DevData data;
  const int64_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  int64_t start = 0;
  const SearchGraph* graphs = nullptr;  // device; with q_graph, replaces row_ptr/col/start
  const int32_t* q_graph = nullptr;     // device, per query; validated by the caller
  const int32_t* q_L = nullptr;         // device, per query, k <= q_L[i] <= L; validated by the caller
  const uint8_t* Q = nullptr;  // padded rows like data
  int64_t nq = 0;
  int L = 0;
  int k = 0;
  int32_t* out_ids = nullptr;
  float* out_dists = nullptr;
  int num_sms = 0;
  int cache_bits = 0;   // id-cache entries per warp as a power of two (8..12); 0 = chosen by the launcher
  int ctas_per_sm = 0;  // CTAs per SM cap; 0 = as many as shared memory allows (<= 16)
  unsigned int* work = nullptr;   // zeroed
  DevStatus* status = nullptr;
  int max_degree = 0;
  // graph construction: query i = base point q_point[i] (Q unused); graph as
  // adj_deg[v] ids at col + v * adj_stride (row_ptr unused); expanded points
  // recorded per query (first visited_cap) with their count
  const int32_t* q_point = nullptr;
  const int32_t* adj_deg = nullptr;
  int64_t adj_stride = 0;
  int32_t* visited = nullptr;
  int32_t* visited_cnt = nullptr;
  int visited_cap = 0;
};
cudaError_t launch_search(const SearchLaunch& S, cudaStream_t s);
cudaError_t launch_recall(const int32_t* found, int ld_found, const int32_t* truth, int ld_truth,
                          int64_t nq, int k, unsigned long long* hits, cudaStream_t s);

// Per-node terms of alpha-reachability (Definition 2.1) at nodes[0..n_nodes)
// (nodes == nullptr: node i), into out[n_nodes] (reach.cu).
cudaError_t launch_reach(const DevData& D, const int64_t* row_ptr, const int32_t* col, const int64_t* nodes,
                         int64_t n_nodes, double* out, cudaStream_t s);

// knn.cu
struct KnnLaunch {
  DevData data;
  const uint8_t* Q = nullptr;  // padded query rows, or nullptr for base points 0..nq-1
  int64_t nq = 0;
  int k = 0;
  int32_t* out_ids = nullptr;
  float* out_dists = nullptr;
  DevStatus* status = nullptr;
  int num_sms = 0;
};
cudaError_t launch_knn(const KnnLaunch& K, cudaStream_t s);

// Exact kNN with the candidate filter on tcgen05 (uint8 rows of d <= 128,
// float rows of at most 256 dimensions, k <= 128).
struct KnnTcLaunch {
  DevData data;
  const uint8_t* Q = nullptr;  // padded query rows, or nullptr for base points 0..nq-1
  int64_t nq = 0;
  int k = 0;
  int32_t* out_ids = nullptr;
  float* out_dists = nullptr;
  DevStatus* status = nullptr;
  int num_sms = 0;
  uint8_t* scratch = nullptr;  // knn_tc_scratch_bytes(), 256-byte aligned
};
bool knn_tc_eligible(int dtype, int d, int k);
// max |x| over n float rows, as the bits of a non-negative float (atomicMax into *out)
cudaError_t launch_maxabs_f32(const uint8_t* X, int64_t row_bytes, int64_t n, int d, unsigned* out, cudaStream_t s);
size_t knn_tc_scratch_bytes(int dtype, int d, int64_t n, int64_t nq_ext, int num_sms);
cudaError_t launch_knn_tc(const KnnTcLaunch& K, cudaStream_t s);

// vamana.cu: batched Vamana construction (graph held as nbr[p * R ..], deg[p])
cudaError_t launch_vamana_candidates(const int32_t* pts, int64_t nb, const int32_t* visited, const int32_t* vis_cnt,
                                     int vcap, const int32_t* nbr, const int32_t* deg, int R, int32_t* cand,
                                     int32_t* cnt, unsigned long long* cut, cudaStream_t s);
cudaError_t launch_compact_rows(const int32_t* src, int64_t stride, const int64_t* src_off, const int32_t* cnt,
                                int64_t rows, const int64_t* row_ptr, int32_t* col, cudaStream_t s);
cudaError_t launch_vamana_write_back(const int32_t* pts, int64_t rows, const int64_t* row_ptr, const int32_t* kept_col,
                                     const int32_t* kept_cnt, int32_t* nbr, int32_t* deg, int R, cudaStream_t s);
cudaError_t launch_back_count(const int32_t* pts, int64_t nb, const int32_t* nbr, const int32_t* deg, int R,
                              int32_t* pend, int32_t* slot, int32_t* jlist, int32_t* nj, cudaStream_t s);
cudaError_t launch_slot_counts(const int32_t* jlist, int64_t nj, const int32_t* pend, int32_t* out, cudaStream_t s);
cudaError_t launch_back_scatter(const int32_t* pts, int64_t nb, const int32_t* nbr, const int32_t* deg, int R,
                                const int32_t* slot, const int64_t* seg_ptr, int32_t* cursor, int32_t* seg,
                                cudaStream_t s);
cudaError_t launch_back_merge(const int32_t* jlist, int64_t nj, const int64_t* seg_ptr, int32_t* seg,
                              int32_t* sorted, int32_t* nbr, int32_t* deg, int R, int32_t* pend, int32_t* ov_raw,
                              int32_t* ov_slot, int32_t* ov_cnt, int32_t* n_ov, cudaStream_t s);
cudaError_t launch_ov_prep(const int32_t* ov_slot, int64_t no, const int32_t* jlist, const int64_t* seg_ptr, int R,
                           int32_t* ov_pts, int64_t* ov_src, cudaStream_t s);

}  // namespace rpk
