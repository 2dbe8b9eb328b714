// C ABI and host runtime of librp.so: contexts, resident graphs, the HBM
// budget, stream-ordered allocation and CUDA-graph replay of batched tuning.
// The public contract of every function is documented in include/rp.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "rp.h"

using namespace rpk;

namespace {

struct Dataset {
  uint8_t* X = nullptr;
  int64_t row_bytes = 0;
  int64_t n = 0;
  int d = 0;
  int dtype = 0;
  float scale = 1.f;  // power of two bringing max |x| to at most 1 (float rows)
  size_t bytes = 0;
  DevData dev() const {
    DevData D;
    D.X = X;
    D.row_bytes = row_bytes;
    D.n = n;
    D.d = d;
    D.dtype = dtype;
    D.scale = scale;
    return D;
  }
};

// Tensor-core prune configuration picked for one source graph, per target-count
// class (1, 2, 4, 8, 16) and variant.
struct TuneChoice {
  int tclass = 0, variant = 0, tile0 = 0, ctas = 0;
};

struct Graph {
  std::shared_ptr<Dataset> data;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  int64_t n = 0;
  int64_t col_cap = 0;
  int64_t nnz = -1;         // known on the host after a sync, else -1
  int max_deg_bound = 0;    // an upper bound of the largest out-degree
  int64_t start = 0;
  int32_t* buckets = nullptr;  // 3 * n node lists + 3 counts, built on first use as a source
  size_t bytes = 0;
  size_t bucket_bytes = 0;
  int64_t bucket0 = -1;  // nodes of degree <= 64, read back for the autotuner
  int64_t bucket_cnt[3] = {-1, -1, -1};  // every bucket's size, read back for chunked tuning
  std::vector<TuneChoice> choices;
};

struct BatchPlan {
  rp_graph src = 0;
  int64_t kernels = 0;  // kernels in the captured graph
  int T = 0;
  int variant = 0;
  int32_t A[kMaxTargets];
  int32_t R[kMaxTargets];
  int tile0 = 0, ctas = 0;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct rp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  uint64_t budget = 0;
  uint64_t used = 0;
  uint64_t peak = 0;
  std::map<rp_graph, Graph*> graphs;
  rp_graph next_id = 1;
  std::string err;
  std::mutex mu;
  DevStatus* status = nullptr;        // device
  unsigned long long* dropped = nullptr;  // device [2]
  // prune scratch, grown on demand
  int32_t* scratch_col = nullptr;
  int64_t scratch_col_elems = 0;
  int32_t* scratch_cnt = nullptr;
  int64_t scratch_cnt_elems = 0;
  int64_t* scratch_bsum = nullptr;
  int64_t scratch_bsum_elems = 0;
  unsigned int* work = nullptr;       // device [8]
  // search scratch
  uint8_t* qbuf = nullptr;
  int64_t qbuf_bytes = 0;
  unsigned long long* hits = nullptr;  // device [1]
  std::vector<BatchPlan> plans;
  // prune configuration: autotuned per source graph, or fixed by rp_set_tuning
  int tuning_mode = RP_TUNING_AUTO;
  int fixed_tile0 = 0, fixed_ctas = 0;
  int last_tile0 = 0, last_ctas = 0;
  int knn_method = RP_KNN_AUTO;
  int search_cache_bits = 0, search_ctas = 0;  // rp_set_search_config
  int last_knn_method = 0;
  int32_t* trial_count = nullptr;  // device int[4]: bucket sizes of a trial launch
  // asynchronous tuning (rp_tune_batch_async): a lowest-priority stream that
  // runs one job at a time in node-range chunks, with scratch of its own
  cudaStream_t tune_stream = nullptr;
  cudaEvent_t tune_ready = nullptr;   // the outputs of the job in flight are in place
  cudaEvent_t tune_inputs = nullptr;  // its allocations on the ctx stream are done
  int64_t tune_ticket = 0;            // last job started (tickets count from 1)
  int32_t* a_col = nullptr;
  int64_t a_col_elems = 0;
  int32_t* a_cnt = nullptr;
  int64_t a_cnt_elems = 0;
  int64_t* a_bsum = nullptr;
  int64_t a_bsum_elems = 0;
  int32_t* a_chunk = nullptr;  // per chunk: 3 bucket counts, then 4 work counters
  int64_t a_chunk_elems = 0;
  int64_t graph_replays = 0;
  int64_t kernel_launches = 0;
  // phase timing: 0/1 prune, 1/2 emit, 3/4 search
  cudaEvent_t ev[5] = {};
  bool ev_tune = false, ev_search = false;
};

namespace {

rp_status fail(rp_ctx* c, rp_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CUDA_TRY(ctx, expr)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, RP_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),      \
                  __FILE__, __LINE__);                                                        \
  } while (0)

size_t elem_size(int dtype) { return dtype == RP_U8 ? 1 : 4; }
int64_t padded_row_bytes(int d, int dtype) {
  const int64_t raw = int64_t(d) * int64_t(elem_size(dtype));
  return (raw + 127) / 128 * 128;
}

// Stream-ordered allocation against the context budget.
rp_status dalloc(rp_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->budget && c->used + bytes > c->budget)
    return fail(c, RP_ENOMEM, "allocation of %zu bytes exceeds the HBM budget (%llu of %llu in use)", bytes,
                (unsigned long long)c->used, (unsigned long long)c->budget);
  cudaError_t e = cudaMallocAsync(p, bytes, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? RP_ENOMEM : RP_ECUDA, "cudaMallocAsync(%zu): %s", bytes,
                cudaGetErrorString(e));
  }
  c->used += bytes;
  c->peak = std::max(c->peak, c->used);
  return RP_OK;
}

void dfree(rp_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  cudaFreeAsync(p, c->stream);
  c->used -= std::min<uint64_t>(c->used, bytes);
}

template <typename T>
rp_status grow(rp_ctx* c, T** buf, int64_t* have, int64_t need) {
  if (*have >= need) return RP_OK;
  dfree(c, *buf, size_t(*have) * sizeof(T));
  *buf = nullptr;
  *have = 0;
  const int64_t want = std::max<int64_t>(need, 1);
  rp_status s = dalloc(c, reinterpret_cast<void**>(buf), size_t(want) * sizeof(T));
  if (s != RP_OK) return s;
  *have = want;
  return RP_OK;
}

rp_status check_device_status(rp_ctx* c) {
  DevStatus h;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->status, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (h.code != 0) {
    const int zero = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&c->status->code, &zero, sizeof zero, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const char* what = h.code == kDevBadId        ? "an id outside [0, n), a malformed row_ptr or a non-finite value"
                       : h.code == kDevTieUnresolved ? "a near-tie run longer than the kept candidates"
                       : h.code == kDevOverflow      ? "a per-query scratch structure ran out of room"
                       : h.code == kDevBadDegree     ? "a degree above the kernel's limit"
                                                     : "unknown";
    return fail(c, RP_EDEVICE, "device status %d (%s) at index %lld", h.code, what, (long long)h.info);
  }
  return RP_OK;
}

// Records a timing event; inside a stream capture it becomes an event-record
// node of the graph (cudaEventRecordExternal), so replays time themselves.
cudaError_t record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &st);
  if (err != cudaSuccess) return err;
  return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

Graph* find_graph(rp_ctx* c, rp_graph g) {
  auto it = c->graphs.find(g);
  return it == c->graphs.end() ? nullptr : it->second;
}

rp_graph add_graph(rp_ctx* c, Graph* G) {
  const rp_graph id = c->next_id++;
  c->graphs[id] = G;
  return id;
}

void free_graph_mem(rp_ctx* c, Graph* G) {
  dfree(c, G->row_ptr, size_t(G->n + 1) * 8);
  dfree(c, G->col, size_t(std::max<int64_t>(G->col_cap, 1)) * 4);
  if (G->buckets) dfree(c, G->buckets, G->bucket_bytes);
  if (G->data && G->data.use_count() == 1) dfree(c, G->data->X, G->data->bytes);
  G->data.reset();
  delete G;
}

bool alpha_to_milli(double alpha, int32_t* A) {
  if (!(alpha >= 1.0) || !(alpha <= 100.0)) return false;
  const double m = alpha * 1000.0;
  const double r = std::nearbyint(m);
  if (std::fabs(m - r) > 1e-6) return false;
  *A = int32_t(r);
  return true;
}

// Copy rows (packed, d * esz bytes each) into a padded device buffer.
rp_status upload_rows(rp_ctx* c, uint8_t* dst, int64_t dst_rb, const void* src, int64_t n, int d, int dtype,
                      int mem_flags) {
  const size_t w = size_t(d) * elem_size(dtype);
  CUDA_TRY(c, cudaMemsetAsync(dst, 0, size_t(n * dst_rb), c->stream));
  if (n == 0) return RP_OK;
  CUDA_TRY(c, cudaMemcpy2DAsync(dst, size_t(dst_rb), src, w, w, size_t(n),
                                mem_flags == RP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                c->stream));
  return RP_OK;
}

rp_status ensure_buckets(rp_ctx* c, Graph* G) {
  if (G->buckets) return RP_OK;
  G->bucket_bytes = size_t(3 * G->n + 4) * 4;
  rp_status s = dalloc(c, reinterpret_cast<void**>(&G->buckets), G->bucket_bytes);
  if (s != RP_OK) return s;
  CUDA_TRY(c, launch_bucket_nodes(G->row_ptr, G->n, G->buckets, G->buckets + 3 * G->n, c->stream));
  return RP_OK;
}

// Enqueue the whole tuning pipeline for `T` targets of `src` into `outs`.
rp_status enqueue_tune(rp_ctx* c, Graph* S, int T, const int32_t* A, const int32_t* R, int variant, int tile0,
                       int ctas, Graph* const* outs, int64_t* kernels) {
  PruneLaunch L;
  L.tile0 = tile0;
  L.ctas_per_sm = ctas;
  L.data = S->data->dev();
  L.row_ptr = S->row_ptr;
  L.col = S->col;
  for (int b = 0; b < 3; ++b) {
    L.bucket_nodes[b] = S->buckets + int64_t(b) * S->n;
    L.host_bucket_count[b] = S->n;  // upper bound; kernels stop at the device count
  }
  const bool generic_all = S->data->dtype == RP_U8 && S->data->d > 256;  // see launch_prune
  if (S->max_deg_bound <= 128 && !generic_all) L.host_bucket_count[2] = 0;
  if (S->max_deg_bound <= 64) L.host_bucket_count[1] = 0;
  L.bucket_count = S->buckets + 3 * S->n;
  L.host_max_degree = S->max_deg_bound;
  L.T = T;
  L.variant = variant;
  L.work = c->work;
  L.status = c->status;
  L.num_sms = c->num_sms;
  int32_t* dst_col[kMaxTargets];
  int64_t* dst_rp[kMaxTargets];
  int32_t* scr[kMaxTargets];
  int32_t* cnt[kMaxTargets];
  for (int t = 0; t < T; ++t) {
    L.A[t] = A[t];
    L.R[t] = R[t];
    scr[t] = c->scratch_col + int64_t(t) * std::max<int64_t>(S->col_cap, 1);
    cnt[t] = c->scratch_cnt + int64_t(t) * S->n;
    L.out_col[t] = scr[t];
    L.out_cnt[t] = cnt[t];
    dst_col[t] = outs[t]->col;
    dst_rp[t] = outs[t]->row_ptr;
  }
  CUDA_TRY(c, cudaMemsetAsync(c->work, 0, 8 * sizeof(unsigned), c->stream));
  CUDA_TRY(c, record(c->ev[0], c->stream));
  CUDA_TRY(c, launch_prune(L, c->stream));
  CUDA_TRY(c, record(c->ev[1], c->stream));
  CUDA_TRY(c, launch_emit_csr(S->n, T, S->row_ptr, scr, cnt, dst_rp, dst_col, c->scratch_bsum, c->stream));
  CUDA_TRY(c, record(c->ev[2], c->stream));
  c->ev_tune = true;
  int64_t k = 3;
  for (int b = 0; b < 3; ++b) k += L.host_bucket_count[b] > 0;
  *kernels = k;
  return RP_OK;
}

// The tensor-core prune configuration for T targets of S: fixed by
// rp_set_tuning, or chosen once per (source, target-count class, variant) by
// timing every candidate on a sample of the degree <= 64 nodes.  Runs before
// any stream capture (it synchronises).
constexpr int64_t kAutotuneMinNodes = 65536;
constexpr int64_t kAutotuneSample = 32768;

rp_status choose_config(rp_ctx* c, Graph* S, int T, const int32_t* A, const int32_t* R, int variant, int* tile0,
                        int* ctas) {
  *tile0 = 0;
  *ctas = 0;
  if (c->tuning_mode == RP_TUNING_FIXED) {
    *tile0 = c->fixed_tile0;
    *ctas = c->fixed_ctas;
    return RP_OK;
  }
  if (S->data->dtype == RP_U8 && S->data->d > 256) return RP_OK;  // all nodes take the CUDA-core path
  const int tclass = T <= 1 ? 1 : T <= 2 ? 2 : T <= 4 ? 4 : T <= 8 ? 8 : 16;
  for (const TuneChoice& ch : S->choices)
    if (ch.tclass == tclass && ch.variant == variant) {
      *tile0 = ch.tile0;
      *ctas = ch.ctas;
      return RP_OK;
    }
  if (S->bucket0 < 0) {
    int32_t cnt[3] = {0, 0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(cnt, S->buckets + 3 * S->n, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    S->bucket0 = cnt[0];
  }
  TuneChoice best;
  best.tclass = tclass;
  best.variant = variant;
  if (S->bucket0 >= kAutotuneMinNodes) {
    rp_status st;
    if (!c->trial_count && (st = dalloc(c, reinterpret_cast<void**>(&c->trial_count), 16)) != RP_OK) return st;
    const int32_t sample[4] = {int32_t(std::min(S->bucket0, kAutotuneSample)), 0, 0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(c->trial_count, sample, sizeof sample, cudaMemcpyHostToDevice, c->stream));
    PruneLaunch L;
    L.data = S->data->dev();
    L.row_ptr = S->row_ptr;
    L.col = S->col;
    for (int b = 0; b < 3; ++b) L.bucket_nodes[b] = S->buckets + int64_t(b) * S->n;
    L.host_bucket_count[0] = sample[0];
    L.bucket_count = c->trial_count;
    L.host_max_degree = S->max_deg_bound;
    L.T = T;
    L.variant = variant;
    L.work = c->work;
    L.status = c->status;
    L.num_sms = c->num_sms;
    for (int t = 0; t < T; ++t) {
      L.A[t] = A[t];
      L.R[t] = R[t];
      L.out_col[t] = c->scratch_col + int64_t(t) * std::max<int64_t>(S->col_cap, 1);
      L.out_cnt[t] = c->scratch_cnt + int64_t(t) * S->n;
    }
    const int cand[6][2] = {{0, 0}, {0, 3}, {0, 2}, {1, 0}, {1, 3}, {1, 2}};
    float best_ms = 0.f;
    for (int i = 0; i < 6; ++i) {
      L.tile0 = cand[i][0];
      L.ctas_per_sm = cand[i][1];
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the first run loads the kernel
        CUDA_TRY(c, cudaMemsetAsync(c->work, 0, 8 * sizeof(unsigned), c->stream));
        CUDA_TRY(c, cudaEventRecord(c->ev[0], c->stream));
        CUDA_TRY(c, launch_prune(L, c->stream));
        CUDA_TRY(c, cudaEventRecord(c->ev[1], c->stream));
        CUDA_TRY(c, cudaEventSynchronize(c->ev[1]));
        CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->kernel_launches += 1;
      }
      if (i == 0 || ms < best_ms) {
        best_ms = ms;
        best.tile0 = cand[i][0];
        best.ctas = cand[i][1];
      }
    }
    if ((st = check_device_status(c)) != RP_OK) return st;
  }
  S->choices.push_back(best);
  *tile0 = best.tile0;
  *ctas = best.ctas;
  return RP_OK;
}

rp_status tune_impl(rp_ctx* c, rp_graph src, const double* alphas, const int32_t* Rs, int32_t T, int32_t variant,
                    rp_graph* outs, bool use_graph) {
  if (!outs || !alphas || !Rs) return fail(c, RP_EINVAL, "null argument");
  if (T < 1 || T > kMaxTargets) return fail(c, RP_EINVAL, "T=%d outside [1, %d]", T, kMaxTargets);
  if (variant != RP_SORTED && variant != RP_UNSORTED) return fail(c, RP_EINVAL, "bad variant %d", variant);
  Graph* S = find_graph(c, src);
  if (!S) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)src);
  int32_t A[kMaxTargets], R[kMaxTargets];
  for (int t = 0; t < T; ++t) {
    if (!alpha_to_milli(alphas[t], &A[t]))
      return fail(c, RP_EINVAL, "alpha=%.17g must lie in [1, 100] on the 0.001 grid", alphas[t]);
    if (Rs[t] < 1) return fail(c, RP_EINVAL, "R=%d must be >= 1", Rs[t]);
    R[t] = Rs[t];
  }
  rp_status s = ensure_buckets(c, S);
  if (s != RP_OK) return s;
  const int64_t cap = std::max<int64_t>(S->col_cap, 1);
  if ((s = grow(c, &c->scratch_col, &c->scratch_col_elems, cap * T)) != RP_OK) return s;
  if ((s = grow(c, &c->scratch_cnt, &c->scratch_cnt_elems, S->n * T)) != RP_OK) return s;
  if ((s = grow(c, &c->scratch_bsum, &c->scratch_bsum_elems, emit_csr_blocks(S->n) * T)) != RP_OK) return s;
  int tile0 = 0, ctas = 0;
  if ((s = choose_config(c, S, T, A, R, variant, &tile0, &ctas)) != RP_OK) return s;
  c->last_tile0 = tile0;
  c->last_ctas = ctas;
  Graph* G[kMaxTargets] = {};
  for (int t = 0; t < T; ++t) {
    G[t] = new Graph;
    G[t]->data = S->data;
    G[t]->n = S->n;
    G[t]->col_cap = S->col_cap;
    G[t]->start = S->start;
    G[t]->max_deg_bound = std::min(S->max_deg_bound, R[t]);
    G[t]->bytes = size_t(S->n + 1) * 8 + size_t(cap) * 4;
    s = dalloc(c, reinterpret_cast<void**>(&G[t]->row_ptr), size_t(S->n + 1) * 8);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&G[t]->col), size_t(cap) * 4);
    if (s != RP_OK) {
      for (int u = 0; u <= t; ++u) free_graph_mem(c, G[u]);
      return s;
    }
  }
  int64_t nk = 0;
  if (!use_graph) {
    s = enqueue_tune(c, S, T, A, R, variant, tile0, ctas, G, &nk);
    c->kernel_launches += nk;
  } else {
    // Replay: capture this call's launches and update the cached executable
    // graph of the same (source, targets, variant) in place.
    BatchPlan* plan = nullptr;
    for (auto& pl : c->plans)
      if (pl.src == src && pl.T == T && pl.variant == variant && pl.tile0 == tile0 && pl.ctas == ctas &&
          !memcmp(pl.A, A, 4 * T) && !memcmp(pl.R, R, 4 * T))
        plan = &pl;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) s = fail(c, RP_ECUDA, "begin capture: %s", cudaGetErrorString(ce));
    if (s == RP_OK) {
      s = enqueue_tune(c, S, T, A, R, variant, tile0, ctas, G, &nk);
      ce = cudaStreamEndCapture(c->stream, &graph);
      if (s == RP_OK && ce != cudaSuccess) s = fail(c, RP_ECUDA, "end capture: %s", cudaGetErrorString(ce));
    }
    if (s == RP_OK) {
      bool ok = false;
      if (plan && plan->exec) {
        cudaGraphExecUpdateResultInfo info;
        ok = cudaGraphExecUpdate(plan->exec, graph, &info) == cudaSuccess;
        if (!ok) cudaGetLastError();
        else ++c->graph_replays;
      }
      if (!ok) {
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess) s = fail(c, RP_ECUDA, "instantiate: %s", cudaGetErrorString(ce));
        else {
          if (!plan) {
            c->plans.push_back(BatchPlan{});
            plan = &c->plans.back();
            plan->src = src;
            plan->T = T;
            plan->variant = variant;
            plan->tile0 = tile0;
            plan->ctas = ctas;
            memcpy(plan->A, A, 4 * T);
            memcpy(plan->R, R, 4 * T);
          } else if (plan->exec) {
            cudaGraphExecDestroy(plan->exec);
          }
          plan->exec = exec;
        }
      }
      if (s == RP_OK) {
        plan->kernels = nk;
        ce = cudaGraphLaunch(plan->exec, c->stream);
        if (ce != cudaSuccess) s = fail(c, RP_ECUDA, "graph launch: %s", cudaGetErrorString(ce));
        else c->kernel_launches += nk;
      }
    }
    if (graph) cudaGraphDestroy(graph);
  }
  if (s != RP_OK) {
    for (int t = 0; t < T; ++t) free_graph_mem(c, G[t]);
    return s;
  }
  for (int t = 0; t < T; ++t) outs[t] = add_graph(c, G[t]);
  return RP_OK;
}

// Asynchronous tuning: the pipeline of enqueue_tune on the ctx's lowest-
// priority stream, each bucket's nodes cut into `chunks` launches so that work
// on the ctx stream (searches) gets the SMs between them.  Outputs are
// allocated on the ctx stream before any chunk runs; they may be used once
// tune_ready has completed (rp_tune_wait).  One job at a time: a new one waits
// for the previous to finish.
rp_status tune_async_impl(rp_ctx* c, rp_graph src, const double* alphas, const int32_t* Rs, int32_t T,
                          int32_t variant, int32_t chunks, rp_graph* outs, int64_t* ticket) {
  if (!outs || !alphas || !Rs || !ticket) return fail(c, RP_EINVAL, "null argument");
  if (T < 1 || T > kMaxTargets) return fail(c, RP_EINVAL, "T=%d outside [1, %d]", T, kMaxTargets);
  if (variant != RP_SORTED && variant != RP_UNSORTED) return fail(c, RP_EINVAL, "bad variant %d", variant);
  if (chunks < 1 || chunks > 4096) return fail(c, RP_EINVAL, "chunks=%d outside [1, 4096]", chunks);
  Graph* S = find_graph(c, src);
  if (!S) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)src);
  int32_t A[kMaxTargets], R[kMaxTargets];
  for (int t = 0; t < T; ++t) {
    if (!alpha_to_milli(alphas[t], &A[t]))
      return fail(c, RP_EINVAL, "alpha=%.17g must lie in [1, 100] on the 0.001 grid", alphas[t]);
    if (Rs[t] < 1) return fail(c, RP_EINVAL, "R=%d must be >= 1", Rs[t]);
    R[t] = Rs[t];
  }
  if (!c->tune_stream) {
    int least = 0, greatest = 0;
    CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CUDA_TRY(c, cudaStreamCreateWithPriority(&c->tune_stream, cudaStreamNonBlocking, least));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->tune_ready, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->tune_inputs, cudaEventDisableTiming));
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->tune_stream));  // the previous job is finished with the scratch
  rp_status s = ensure_buckets(c, S);
  if (s != RP_OK) return s;
  if (S->bucket_cnt[0] < 0) {
    int32_t cnt[3] = {0, 0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(cnt, S->buckets + 3 * S->n, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int b = 0; b < 3; ++b) S->bucket_cnt[b] = cnt[b];
  }
  const int64_t cap = std::max<int64_t>(S->col_cap, 1);
  if ((s = grow(c, &c->a_col, &c->a_col_elems, cap * T)) != RP_OK) return s;
  if ((s = grow(c, &c->a_cnt, &c->a_cnt_elems, S->n * T)) != RP_OK) return s;
  if ((s = grow(c, &c->a_bsum, &c->a_bsum_elems, emit_csr_blocks(S->n) * T)) != RP_OK) return s;
  // the launches: every bucket cut into `chunks` contiguous ranges of its node list
  std::vector<int32_t> host;  // per launch: 3 counts (only its bucket's nonzero), 4 work counters
  std::vector<std::pair<int, int64_t>> launches;  // (bucket, first list entry)
  for (int b = 0; b < 3; ++b) {
    const int64_t nb = S->bucket_cnt[b];
    if (nb <= 0) continue;
    const int64_t per = (nb + chunks - 1) / chunks;
    for (int64_t lo = 0; lo < nb; lo += per) {
      const int64_t hi = std::min(nb, lo + per);
      launches.emplace_back(b, lo);
      for (int q = 0; q < 3; ++q) host.push_back(q == b ? int32_t(hi - lo) : 0);
      for (int q = 0; q < 4; ++q) host.push_back(0);
    }
  }
  if ((s = grow(c, &c->a_chunk, &c->a_chunk_elems, std::max<int64_t>(int64_t(host.size()), 7))) != RP_OK) return s;
  if (!host.empty())
    CUDA_TRY(c, cudaMemcpyAsync(c->a_chunk, host.data(), host.size() * 4, cudaMemcpyHostToDevice, c->stream));
  int tile0 = 0, ctas = 0;  // a configuration chosen earlier for this source, else the default
  const int tclass = T <= 1 ? 1 : T <= 2 ? 2 : T <= 4 ? 4 : T <= 8 ? 8 : 16;
  if (c->tuning_mode == RP_TUNING_FIXED) {
    tile0 = c->fixed_tile0;
    ctas = c->fixed_ctas;
  } else {
    for (const TuneChoice& ch : S->choices)
      if (ch.tclass == tclass && ch.variant == variant) {
        tile0 = ch.tile0;
        ctas = ch.ctas;
      }
  }
  Graph* G[kMaxTargets] = {};
  for (int t = 0; t < T; ++t) {
    G[t] = new Graph;
    G[t]->data = S->data;
    G[t]->n = S->n;
    G[t]->col_cap = S->col_cap;
    G[t]->start = S->start;
    G[t]->max_deg_bound = std::min(S->max_deg_bound, R[t]);
    G[t]->bytes = size_t(S->n + 1) * 8 + size_t(cap) * 4;
    s = dalloc(c, reinterpret_cast<void**>(&G[t]->row_ptr), size_t(S->n + 1) * 8);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&G[t]->col), size_t(cap) * 4);
    if (s != RP_OK) {
      for (int u = 0; u <= t; ++u) free_graph_mem(c, G[u]);
      return s;
    }
  }
  // the tuning stream starts once the ctx stream has made the allocations and copies
  CUDA_TRY(c, cudaEventRecord(c->tune_inputs, c->stream));
  CUDA_TRY(c, cudaStreamWaitEvent(c->tune_stream, c->tune_inputs, 0));
  PruneLaunch L;
  L.tile0 = tile0;
  L.ctas_per_sm = ctas;
  L.data = S->data->dev();
  L.row_ptr = S->row_ptr;
  L.col = S->col;
  L.host_max_degree = S->max_deg_bound;
  L.T = T;
  L.variant = variant;
  L.status = c->status;
  L.num_sms = c->num_sms;
  int32_t* scr[kMaxTargets];
  int32_t* cnt[kMaxTargets];
  int32_t* dst_col[kMaxTargets];
  int64_t* dst_rp[kMaxTargets];
  for (int t = 0; t < T; ++t) {
    L.A[t] = A[t];
    L.R[t] = R[t];
    scr[t] = c->a_col + int64_t(t) * cap;
    cnt[t] = c->a_cnt + int64_t(t) * S->n;
    L.out_col[t] = scr[t];
    L.out_cnt[t] = cnt[t];
    dst_col[t] = G[t]->col;
    dst_rp[t] = G[t]->row_ptr;
  }
  cudaError_t ce = cudaSuccess;
  for (size_t i = 0; i < launches.size() && ce == cudaSuccess; ++i) {
    const int b = launches[i].first;
    int32_t* blk = c->a_chunk + 7 * int64_t(i);
    for (int q = 0; q < 3; ++q) {
      L.bucket_nodes[q] = S->buckets + int64_t(q) * S->n + (q == b ? launches[i].second : 0);
      L.host_bucket_count[q] = q == b ? host[7 * i + size_t(q)] : 0;
    }
    L.bucket_count = blk;
    L.work = reinterpret_cast<unsigned int*>(blk + 3) - b;  // launch_prune adds the bucket index
    ce = launch_prune(L, c->tune_stream);
  }
  if (ce == cudaSuccess) ce = launch_emit_csr(S->n, T, S->row_ptr, scr, cnt, dst_rp, dst_col, c->a_bsum, c->tune_stream);
  if (ce == cudaSuccess) ce = cudaEventRecord(c->tune_ready, c->tune_stream);
  if (ce != cudaSuccess) {
    cudaStreamSynchronize(c->tune_stream);
    for (int t = 0; t < T; ++t) free_graph_mem(c, G[t]);
    return fail(c, RP_ECUDA, "asynchronous tuning: %s", cudaGetErrorString(ce));
  }
  c->kernel_launches += int64_t(launches.size()) + 3;
  for (int t = 0; t < T; ++t) outs[t] = add_graph(c, G[t]);
  *ticket = ++c->tune_ticket;
  return RP_OK;
}

// Exact kNN of nq queries (padded device rows Q, or base points 0..nq-1 when
// Q is null) by the tensor-core filter where it applies, else the CUDA-core scan.
rp_status run_knn(rp_ctx* c, const Dataset& D, const uint8_t* Q, int64_t nq, int32_t k, int32_t* ids, float* dists) {
  const bool tc_ok = knn_tc_eligible(D.dtype, D.d, k);
  if (c->knn_method == RP_KNN_TENSOR && !tc_ok)
    return fail(c, RP_EINVAL, "the tensor-core kNN needs k <= 128 and uint8 rows of d <= 128 or float rows of d <= 128");
  if (tc_ok && c->knn_method != RP_KNN_CUDA_CORE) {
    const size_t bytes = knn_tc_scratch_bytes(D.dtype, D.d, D.n, Q ? nq : 0, c->num_sms);
    void* scratch = nullptr;
    rp_status st = dalloc(c, &scratch, bytes);
    if (st != RP_OK) return st;
    KnnTcLaunch K;
    K.data = D.dev();
    K.Q = Q;
    K.nq = nq;
    K.k = k;
    K.out_ids = ids;
    K.out_dists = dists;
    K.status = c->status;
    K.num_sms = c->num_sms;
    K.scratch = static_cast<uint8_t*>(scratch);
    const cudaError_t ce = launch_knn_tc(K, c->stream);
    dfree(c, scratch, bytes);
    if (ce != cudaSuccess) return fail(c, RP_ECUDA, "tensor-core kNN: %s", cudaGetErrorString(ce));
    c->kernel_launches += D.dtype == RP_F32 ? 5 : 3;
    c->last_knn_method = RP_KNN_TENSOR;
    return RP_OK;
  }
  KnnLaunch K;
  K.data = D.dev();
  K.Q = Q;
  K.nq = nq;
  K.k = k;
  K.out_ids = ids;
  K.out_dists = dists;
  K.status = c->status;
  K.num_sms = c->num_sms;
  CUDA_TRY(c, launch_knn(K, c->stream));
  c->kernel_launches += (nq + 65535) / 65536;
  c->last_knn_method = RP_KNN_CUDA_CORE;
  return RP_OK;
}

// GreedySearch over `nq` queries.  With q_graph == nullptr every query runs on
// graphs[0] with list size L; otherwise query i runs on graphs[q_graph[i]] with
// list size q_L[i] (both validated by the caller, L = their maximum).
rp_status search_impl(rp_ctx* c, const rp_graph* graphs, int32_t ngraphs, const int32_t* q_graph,
                      const int32_t* q_L, const void* queries, int64_t nq, int32_t L, int32_t k, int32_t* ids,
                      float* dists, int32_t mem_flags) {
  std::vector<Graph*> Gs(static_cast<size_t>(ngraphs));
  for (int32_t j = 0; j < ngraphs; ++j) {
    Gs[j] = find_graph(c, graphs[j]);
    if (!Gs[j]) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)graphs[j]);
    if (Gs[j]->data != Gs[0]->data) return fail(c, RP_EINVAL, "graphs of one search must share their vectors");
  }
  if (nq < 0 || k < 1 || L < k || L > RP_MAX_L)
    return fail(c, RP_EINVAL, "need nq >= 0 and 1 <= k <= L <= %d (nq=%lld L=%d k=%d)", RP_MAX_L, (long long)nq, L, k);
  if (mem_flags != RP_MEM_HOST && mem_flags != RP_MEM_DEVICE) return fail(c, RP_EINVAL, "bad mem_flags %d", mem_flags);
  if (nq == 0) return RP_OK;
  if (!queries || !ids) return fail(c, RP_EINVAL, "null argument");
  const Dataset& D = *Gs[0]->data;
  rp_status s;
  const int64_t qbytes = nq * D.row_bytes;
  const int64_t out_bytes = mem_flags == RP_MEM_HOST ? nq * k * 8 : 0;
  // per-query tables of a mixed launch: graph refs, then graph index and L per query
  const int64_t table_off = (qbytes + out_bytes + 255) / 256 * 256;
  const int64_t table_bytes = q_graph ? int64_t(ngraphs) * int64_t(sizeof(SearchGraph)) + 8 * nq + 16 : 0;
  if ((s = grow(c, &c->qbuf, &c->qbuf_bytes, table_off + table_bytes)) != RP_OK) return s;
  if ((s = upload_rows(c, c->qbuf, D.row_bytes, queries, nq, D.d, D.dtype, mem_flags)) != RP_OK) return s;
  SearchLaunch S;
  S.data = D.dev();
  S.row_ptr = Gs[0]->row_ptr;
  S.col = Gs[0]->col;
  S.start = Gs[0]->start;
  S.max_degree = 0;
  for (Graph* G : Gs) S.max_degree = std::max(S.max_degree, G->max_deg_bound);
  if (q_graph) {
    std::vector<SearchGraph> tab(static_cast<size_t>(ngraphs));
    for (int32_t j = 0; j < ngraphs; ++j) tab[j] = SearchGraph{Gs[j]->row_ptr, Gs[j]->col, Gs[j]->start, 0};
    uint8_t* t = c->qbuf + table_off;
    const size_t gb = size_t(ngraphs) * sizeof(SearchGraph);
    CUDA_TRY(c, cudaMemcpyAsync(t, tab.data(), gb, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(t + gb, q_graph, size_t(nq) * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(t + gb + size_t(nq) * 4, q_L, size_t(nq) * 4, cudaMemcpyHostToDevice, c->stream));
    S.graphs = reinterpret_cast<const SearchGraph*>(t);
    S.q_graph = reinterpret_cast<const int32_t*>(t + gb);
    S.q_L = reinterpret_cast<const int32_t*>(t + gb + size_t(nq) * 4);
  }
  S.Q = c->qbuf;
  S.nq = nq;
  S.L = L;
  S.k = k;
  int32_t* dev_ids = ids;
  float* dev_d = dists;
  if (mem_flags == RP_MEM_HOST) {
    dev_ids = reinterpret_cast<int32_t*>(c->qbuf + qbytes);
    dev_d = reinterpret_cast<float*>(c->qbuf + qbytes + nq * k * 4);
  }
  S.out_ids = dev_ids;
  S.out_dists = dev_d;
  S.num_sms = c->num_sms;
  S.cache_bits = c->search_cache_bits;
  S.ctas_per_sm = c->search_ctas;
  S.work = c->work;
  S.status = c->status;
  CUDA_TRY(c, cudaMemsetAsync(c->work, 0, 8 * sizeof(unsigned), c->stream));
  CUDA_TRY(c, record(c->ev[3], c->stream));
  CUDA_TRY(c, launch_search(S, c->stream));
  CUDA_TRY(c, record(c->ev[4], c->stream));
  c->ev_search = true;
  c->kernel_launches += 1;
  if (mem_flags == RP_MEM_HOST) {
    CUDA_TRY(c, cudaMemcpyAsync(ids, dev_ids, size_t(nq * k) * 4, cudaMemcpyDeviceToHost, c->stream));
    if (dists) CUDA_TRY(c, cudaMemcpyAsync(dists, dev_d, size_t(nq * k) * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return check_device_status(c);
  }
  if (q_graph) {
    // the host tables were read by stream-ordered copies; finish them before returning
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  return RP_OK;
}

rp_status build_base(rp_ctx* c, rp_graph data, int32_t kcand, int32_t nrand, uint64_t seed, double alpha, int32_t R,
                     rp_graph* out) {
  Graph* G = find_graph(c, data);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)data);
  if (!out) return fail(c, RP_EINVAL, "null out");
  if (kcand < 1 || kcand > 128) return fail(c, RP_EINVAL, "kcand=%d outside [1, 128]", kcand);
  if (nrand < 0 || nrand > 128) return fail(c, RP_EINVAL, "nrand=%d outside [0, 128]", nrand);
  const int64_t n = G->n;
  const int kk = int(std::min<int64_t>(kcand, n - 1));
  const int nr = n > 1 ? nrand : 0;
  Graph* K = new Graph;
  K->data = G->data;
  K->n = n;
  K->col_cap = std::max<int64_t>(n * kk, 1);
  K->start = G->start;
  K->max_deg_bound = kk + nr;
  K->nnz = n * kk;
  rp_status s = dalloc(c, reinterpret_cast<void**>(&K->row_ptr), size_t(n + 1) * 8);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&K->col), size_t(K->col_cap) * 4);
  if (s != RP_OK) {
    free_graph_mem(c, K);
    return s;
  }
  if (kk > 0 && (s = run_knn(c, *G->data, nullptr, n, kk, K->col, nullptr)) != RP_OK) {
    free_graph_mem(c, K);
    return s;
  }
  std::vector<int64_t> hrp(size_t(n + 1));
  for (int64_t p = 0; p <= n; ++p) hrp[size_t(p)] = p * kk;
  cudaError_t ce = cudaMemcpyAsync(K->row_ptr, hrp.data(), size_t(n + 1) * 8, cudaMemcpyHostToDevice, c->stream);
  if (ce == cudaSuccess && nr > 0) {
    // rows of kNN ids followed by nr seeded random ids, then repeated ids dropped
    const int w = kk + nr;
    int32_t* raw = nullptr;
    int64_t* rp_raw = nullptr;
    int32_t* cnt = nullptr;
    int64_t* bsum = nullptr;
    int32_t* maxd = nullptr;
    unsigned long long* dropped = nullptr;
    int32_t* col2 = nullptr;
    const int64_t nblk = (n + 4095) / 4096;
    auto release = [&]() {
      dfree(c, raw, size_t(n * w) * 4);
      dfree(c, rp_raw, size_t(n + 1) * 8);
      dfree(c, cnt, size_t(n) * 4);
      dfree(c, bsum, size_t(nblk) * 8);
      dfree(c, maxd, 8);
      dfree(c, dropped, 16);
    };
    s = dalloc(c, reinterpret_cast<void**>(&raw), size_t(n * w) * 4);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&rp_raw), size_t(n + 1) * 8);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&cnt), size_t(n) * 4);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&bsum), size_t(nblk) * 8);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&maxd), 8);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&dropped), 16);
    if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&col2), size_t(n * w) * 4);
    if (s != RP_OK) {
      release();
      free_graph_mem(c, K);
      return s;
    }
    for (int64_t p = 0; p <= n; ++p) hrp[size_t(p)] = p * w;
    ce = cudaMemcpyAsync(rp_raw, hrp.data(), size_t(n + 1) * 8, cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess) ce = launch_add_random_candidates(K->col, kk, n, nr, seed, raw, c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(dropped, 0, 16, c->stream);
    if (ce == cudaSuccess) ce = launch_clean_count(rp_raw, raw, n, cnt, dropped, c->stream);
    if (ce == cudaSuccess) ce = launch_scan_counts(cnt, n, K->row_ptr, bsum, maxd, c->stream);
    if (ce == cudaSuccess) ce = launch_clean_write(rp_raw, raw, n, K->row_ptr, col2, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    release();
    dfree(c, K->col, size_t(K->col_cap) * 4);
    K->col = col2;
    K->col_cap = std::max<int64_t>(n * w, 1);
    K->nnz = -1;
    c->kernel_launches += 5;
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) {
    free_graph_mem(c, K);
    return fail(c, RP_ECUDA, "knn graph: %s", cudaGetErrorString(ce));
  }
  if ((s = check_device_status(c)) != RP_OK) {
    free_graph_mem(c, K);
    return s;
  }
  const rp_graph kid = add_graph(c, K);
  rp_graph res = 0;
  s = tune_impl(c, kid, &alpha, &R, 1, RP_SORTED, &res, false);
  auto it = c->graphs.find(kid);
  free_graph_mem(c, it->second);
  c->graphs.erase(it);
  if (s != RP_OK) return s;
  // The result holds the candidate graph's capacity (n x kcand ids); keep only
  // its edges, since every graph tuned from it takes its capacity too.
  Graph* B = find_graph(c, res);
  CUDA_TRY(c, cudaMemcpyAsync(&B->nnz, B->row_ptr + B->n, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int64_t cap = std::max<int64_t>(B->nnz, 1);
  if (cap < B->col_cap) {
    int32_t* col = nullptr;
    if (dalloc(c, reinterpret_cast<void**>(&col), size_t(cap) * 4) == RP_OK) {
      CUDA_TRY(c, cudaMemcpyAsync(col, B->col, size_t(cap) * 4, cudaMemcpyDeviceToDevice, c->stream));
      dfree(c, B->col, size_t(B->col_cap) * 4);
      B->col = col;
      B->col_cap = cap;
      B->bytes = size_t(B->n + 1) * 8 + size_t(cap) * 4;
    }
  }
  *out = res;
  return RP_OK;
}

}  // namespace

namespace {

// Device buffers of one Vamana build, freed together.
struct VamanaBufs {
  rp_ctx* c;
  std::vector<std::pair<void*, size_t>> held;
  explicit VamanaBufs(rp_ctx* ctx) : c(ctx) {}
  template <typename T>
  rp_status get(T** p, int64_t elems) {
    const size_t b = size_t(std::max<int64_t>(elems, 1)) * sizeof(T);
    rp_status s = dalloc(c, reinterpret_cast<void**>(p), b);
    if (s == RP_OK) held.emplace_back(static_cast<void*>(*p), b);
    return s;
  }
  ~VamanaBufs() {
    for (auto& h : held) dfree(c, h.first, h.second);
  }
};

// Batch k of a pass holds min(2^k, max_batch) points (the last one the rest).
int64_t vamana_batch(int64_t k, int64_t max_batch) {
  int64_t b = 1;
  for (int64_t i = 0; i < k && b < max_batch; ++i) b *= 2;
  return std::min(b, max_batch);
}

// RobustPrune(point_of[i], row i of (row_ptr, col), A, R) for `rows` rows,
// kept ids to kept_col at the rows' offsets, counts to kept_cnt.
rp_status vamana_prune(rp_ctx* c, const Dataset& D, const int64_t* row_ptr, const int32_t* col, int64_t rows,
                       int max_deg, const int32_t* point_of, int32_t A, int32_t R, int32_t* lists, int32_t* kept_col,
                       int32_t* kept_cnt) {
  CUDA_TRY(c, launch_bucket_nodes(row_ptr, rows, lists, lists + 3 * rows, c->stream));
  PruneLaunch P;
  P.data = D.dev();
  P.row_ptr = row_ptr;
  P.col = col;
  for (int b = 0; b < 3; ++b) {
    P.bucket_nodes[b] = lists + int64_t(b) * rows;
    P.host_bucket_count[b] = rows;  // upper bound; the kernels stop at the device count
  }
  if (max_deg <= 128 && !(D.dtype == RP_U8 && D.d > 256)) P.host_bucket_count[2] = 0;
  if (max_deg <= 64) P.host_bucket_count[1] = 0;
  P.bucket_count = lists + 3 * rows;
  P.host_max_degree = max_deg;
  P.T = 1;
  P.A[0] = A;
  P.R[0] = R;
  P.variant = RP_SORTED;
  P.out_col[0] = kept_col;
  P.out_cnt[0] = kept_cnt;
  P.work = c->work;
  P.status = c->status;
  P.num_sms = c->num_sms;
  P.point_of = point_of;
  CUDA_TRY(c, cudaMemsetAsync(c->work, 0, 8 * sizeof(unsigned), c->stream));
  CUDA_TRY(c, launch_prune(P, c->stream));
  c->kernel_launches += 4;
  return RP_OK;
}

int32_t read_i32(rp_ctx* c, const int32_t* d, rp_status* st) {
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) *st = fail(c, RP_ECUDA, "read back: %s", cudaGetErrorString(e));
  return h;
}

rp_status build_vamana(rp_ctx* c, rp_graph data, const int32_t* perm, int32_t npass, const double* alphas, int32_t R,
                       int32_t L, int32_t vcap, int64_t max_batch, int64_t* visited_cut, rp_graph* out) {
  Graph* G = find_graph(c, data);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)data);
  if (!out || !alphas) return fail(c, RP_EINVAL, "null argument");
  if (npass < 1 || npass > 8) return fail(c, RP_EINVAL, "npass=%d outside [1, 8]", npass);
  if (R < 1 || R > 1024) return fail(c, RP_EINVAL, "R=%d outside [1, 1024]", R);
  if (L < 1 || L > RP_MAX_L) return fail(c, RP_EINVAL, "L=%d outside [1, %d]", L, RP_MAX_L);
  if (vcap < 1 || vcap > 4096) return fail(c, RP_EINVAL, "vcap=%d outside [1, 4096]", vcap);
  if (max_batch < 1) return fail(c, RP_EINVAL, "max_batch=%lld", (long long)max_batch);
  std::vector<int32_t> A(static_cast<size_t>(npass));
  for (int i = 0; i < npass; ++i)
    if (!alpha_to_milli(alphas[i], &A[size_t(i)]))
      return fail(c, RP_EINVAL, "alpha=%.17g must lie in [1, 100] on the 0.001 grid", alphas[i]);
  const Dataset& D = *G->data;
  const int64_t n = G->n;
  std::vector<int32_t> hperm(static_cast<size_t>(n));
  if (perm) {
    std::vector<char> seen(static_cast<size_t>(n), 0);
    for (int64_t i = 0; i < n; ++i) {
      const int32_t v = perm[i];
      if (v < 0 || v >= n || seen[size_t(v)]) return fail(c, RP_EINVAL, "perm is not a permutation of 0 .. n-1");
      seen[size_t(v)] = 1;
      hperm[size_t(i)] = v;
    }
  } else {
    for (int64_t i = 0; i < n; ++i) hperm[size_t(i)] = int32_t(i);
  }
  const int64_t B = std::min<int64_t>(max_batch, n);
  const int64_t W = int64_t(vcap) + R;          // candidate row width
  const int64_t J = std::min<int64_t>(n, B * R);  // distinct back-edge targets per batch
  VamanaBufs buf(c);
  int32_t *nbr, *deg, *pend, *slot, *dperm, *vis, *vis_cnt, *sids, *cand, *ccnt, *ccol, *lists, *kept_col, *kept_cnt;
  int32_t *maxd, *jlist, *nj, *scnt, *cursor, *seg, *sorted, *ov_raw, *ov_slot, *ov_cnt, *n_ov, *ov_pts, *ov_col;
  int32_t *ov_kept, *ov_kcnt;
  int64_t *crp, *bsum, *seg_ptr, *ov_src, *ov_rp;
  unsigned long long* cut;
  rp_status s = RP_OK;
  const int64_t nblk = (std::max(n, J + 1) + 4095) / 4096 + 1;
  if (s == RP_OK) s = buf.get(&nbr, n * R);
  if (s == RP_OK) s = buf.get(&deg, n);
  if (s == RP_OK) s = buf.get(&pend, n);
  if (s == RP_OK) s = buf.get(&slot, n);
  if (s == RP_OK) s = buf.get(&dperm, n);
  if (s == RP_OK) s = buf.get(&vis, B * vcap);
  if (s == RP_OK) s = buf.get(&vis_cnt, B);
  if (s == RP_OK) s = buf.get(&sids, B);
  if (s == RP_OK) s = buf.get(&cand, B * W);
  if (s == RP_OK) s = buf.get(&ccnt, B);
  if (s == RP_OK) s = buf.get(&ccol, B * W);
  if (s == RP_OK) s = buf.get(&crp, B + 1);
  if (s == RP_OK) s = buf.get(&bsum, nblk);
  if (s == RP_OK) s = buf.get(&maxd, 2);
  if (s == RP_OK) s = buf.get(&lists, 3 * std::max(B, J) + 3);
  if (s == RP_OK) s = buf.get(&kept_col, B * W);
  if (s == RP_OK) s = buf.get(&kept_cnt, B);
  if (s == RP_OK) s = buf.get(&jlist, J);
  if (s == RP_OK) s = buf.get(&nj, 2);
  if (s == RP_OK) s = buf.get(&scnt, J);
  if (s == RP_OK) s = buf.get(&seg_ptr, J + 1);
  if (s == RP_OK) s = buf.get(&cursor, J);
  if (s == RP_OK) s = buf.get(&seg, B * R);
  if (s == RP_OK) s = buf.get(&sorted, B * R);
  if (s == RP_OK) s = buf.get(&ov_raw, B * R + J * R);
  if (s == RP_OK) s = buf.get(&ov_slot, J);
  if (s == RP_OK) s = buf.get(&ov_cnt, J);
  if (s == RP_OK) s = buf.get(&n_ov, 2);
  if (s == RP_OK) s = buf.get(&ov_pts, J);
  if (s == RP_OK) s = buf.get(&ov_src, J);
  if (s == RP_OK) s = buf.get(&ov_rp, J + 1);
  if (s == RP_OK) s = buf.get(&ov_col, B * R + J * R);
  if (s == RP_OK) s = buf.get(&ov_kept, B * R + J * R);
  if (s == RP_OK) s = buf.get(&ov_kcnt, J);
  if (s == RP_OK) s = buf.get(&cut, 1);
  if (s != RP_OK) return s;
  CUDA_TRY(c, cudaMemsetAsync(deg, 0, size_t(n) * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(pend, 0, size_t(n) * 4, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(cut, 0, 8, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(dperm, hperm.data(), size_t(n) * 4, cudaMemcpyHostToDevice, c->stream));
  for (int pass = 0; pass < npass; ++pass) {
    int64_t b0 = 0;
    for (int64_t k = 0; b0 < n; ++k) {
      const int64_t nb = std::min(vamana_batch(k, max_batch), n - b0);
      const int32_t* pts = dperm + b0;
      // Algorithm 2 for every point of the batch on the graph as it stands
      SearchLaunch S;
      S.data = D.dev();
      S.col = nbr;
      S.adj_deg = deg;
      S.adj_stride = R;
      S.q_point = pts;
      S.start = G->start;
      S.nq = nb;
      S.L = L;
      S.k = 1;
      S.out_ids = sids;
      S.visited = vis;
      S.visited_cnt = vis_cnt;
      S.visited_cap = vcap;
      S.num_sms = c->num_sms;
      S.cache_bits = c->search_cache_bits;
      S.ctas_per_sm = c->search_ctas;
      S.work = c->work;
      S.status = c->status;
      CUDA_TRY(c, cudaMemsetAsync(c->work, 0, 8 * sizeof(unsigned), c->stream));
      CUDA_TRY(c, launch_search(S, c->stream));
      // candidates V_p u N_out(p) \ {p}, Algorithm 1 over them, write back
      CUDA_TRY(c, launch_vamana_candidates(pts, nb, vis, vis_cnt, vcap, nbr, deg, R, cand, ccnt, cut, c->stream));
      CUDA_TRY(c, launch_scan_counts(ccnt, nb, crp, bsum, maxd, c->stream));
      CUDA_TRY(c, launch_compact_rows(cand, W, nullptr, ccnt, nb, crp, ccol, c->stream));
      if ((s = vamana_prune(c, D, crp, ccol, nb, int(W), pts, A[size_t(pass)], R, lists, kept_col, kept_cnt)) !=
          RP_OK)
        return s;
      CUDA_TRY(c, launch_vamana_write_back(pts, nb, crp, kept_col, kept_cnt, nbr, deg, R, c->stream));
      // back edges
      CUDA_TRY(c, cudaMemsetAsync(nj, 0, 4, c->stream));
      CUDA_TRY(c, launch_back_count(pts, nb, nbr, deg, R, pend, slot, jlist, nj, c->stream));
      c->kernel_launches += 8;
      const int64_t nJ = read_i32(c, nj, &s);
      if (s != RP_OK) return s;
      if (nJ > 0) {
        CUDA_TRY(c, launch_slot_counts(jlist, nJ, pend, scnt, c->stream));
        CUDA_TRY(c, launch_scan_counts(scnt, nJ, seg_ptr, bsum, maxd, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(cursor, 0, size_t(nJ) * 4, c->stream));
        CUDA_TRY(c, launch_back_scatter(pts, nb, nbr, deg, R, slot, seg_ptr, cursor, seg, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(n_ov, 0, 4, c->stream));
        CUDA_TRY(c, launch_back_merge(jlist, nJ, seg_ptr, seg, sorted, nbr, deg, R, pend, ov_raw, ov_slot, ov_cnt,
                                      n_ov, c->stream));
        c->kernel_launches += 6;
        const int64_t nO = read_i32(c, n_ov, &s);
        if (s != RP_OK) return s;
        if (nO > 0) {
          CUDA_TRY(c, launch_ov_prep(ov_slot, nO, jlist, seg_ptr, R, ov_pts, ov_src, c->stream));
          CUDA_TRY(c, launch_scan_counts(ov_cnt, nO, ov_rp, bsum, maxd, c->stream));
          CUDA_TRY(c, launch_compact_rows(ov_raw, 0, ov_src, ov_cnt, nO, ov_rp, ov_col, c->stream));
          int32_t mx = 0;
          CUDA_TRY(c, cudaMemcpyAsync(&mx, maxd, 4, cudaMemcpyDeviceToHost, c->stream));
          CUDA_TRY(c, cudaStreamSynchronize(c->stream));
          if ((s = vamana_prune(c, D, ov_rp, ov_col, nO, mx, ov_pts, A[size_t(pass)], R, lists, ov_kept, ov_kcnt)) !=
              RP_OK)
            return s;
          CUDA_TRY(c, launch_vamana_write_back(ov_pts, nO, ov_rp, ov_kept, ov_kcnt, nbr, deg, R, c->stream));
          c->kernel_launches += 6;
        }
      }
      b0 += nb;
    }
  }
  // the adjacency as a CSR graph
  Graph* V = new Graph;
  V->data = G->data;
  V->n = n;
  V->start = G->start;
  V->max_deg_bound = R;
  if ((s = dalloc(c, reinterpret_cast<void**>(&V->row_ptr), size_t(n + 1) * 8)) != RP_OK) {
    free_graph_mem(c, V);
    return s;
  }
  cudaError_t ce = launch_scan_counts(deg, n, V->row_ptr, bsum, maxd, c->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&V->nnz, V->row_ptr + n, 8, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) {
    free_graph_mem(c, V);
    return fail(c, RP_ECUDA, "vamana graph: %s", cudaGetErrorString(ce));
  }
  V->col_cap = std::max<int64_t>(V->nnz, 1);
  V->bytes = size_t(n + 1) * 8 + size_t(V->col_cap) * 4;
  if ((s = dalloc(c, reinterpret_cast<void**>(&V->col), size_t(V->col_cap) * 4)) != RP_OK) {
    free_graph_mem(c, V);
    return s;
  }
  ce = launch_compact_rows(nbr, R, nullptr, deg, n, V->row_ptr, V->col, c->stream);
  unsigned long long hcut = 0;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hcut, cut, 8, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  c->kernel_launches += 4;
  if (ce != cudaSuccess) {
    free_graph_mem(c, V);
    return fail(c, RP_ECUDA, "vamana graph: %s", cudaGetErrorString(ce));
  }
  if ((s = check_device_status(c)) != RP_OK) {
    free_graph_mem(c, V);
    return s;
  }
  if (visited_cut) *visited_cut = int64_t(hcut);
  *out = add_graph(c, V);
  return RP_OK;
}

}  // namespace

// The CSR part of loading a graph over G->data (G->n rows): copy, validate
// (ids in [0, n), row_ptr monotone), drop self loops and repeated ids, exact
// degrees, and the start vertex (the medoid if start < 0).  On failure G keeps
// whatever it allocated; the caller frees it.
rp_status attach_csr(rp_ctx* c, Graph* G, const int64_t* row_ptr, const int32_t* col, int64_t start,
                     int32_t mem_flags) {
  const int64_t n = G->n;
  const int d = G->data->d;
  rp_status s = RP_OK;
  int64_t nnz_in = 0;
  if (row_ptr) {
    if (mem_flags == RP_MEM_HOST) {
      nnz_in = row_ptr[n];
      if (row_ptr[0] != 0 || nnz_in < 0) return fail(c, RP_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
    } else {
      int64_t ends[2];
      cudaMemcpyAsync(&ends[0], row_ptr, 8, cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(&ends[1], row_ptr + n, 8, cudaMemcpyDeviceToHost, c->stream);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess || ends[0] != 0 || ends[1] < 0)
        return fail(c, RP_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
      nnz_in = ends[1];
    }
  }
  // device copies of the input CSR
  int64_t* rp_in = nullptr;
  int32_t* col_in = nullptr;
  int32_t* cnt = nullptr;
  int64_t* bsum = nullptr;
  int32_t* maxd = nullptr;
  int64_t* med = nullptr;
  double* mean = nullptr;
  double* best = nullptr;
  const int64_t nblk = (n + 4095) / 4096;
  auto cleanup = [&]() {
    dfree(c, rp_in, size_t(n + 1) * 8);
    dfree(c, col_in, size_t(std::max<int64_t>(nnz_in, 1)) * 4);
    dfree(c, cnt, size_t(n) * 4);
    dfree(c, bsum, size_t(nblk) * 8);
    dfree(c, maxd, 8);
    dfree(c, med, 8);
    dfree(c, mean, size_t(d) * 8);
    dfree(c, best, size_t(2 * medoid_blocks(n)) * 8);
  };
  G->col_cap = std::max<int64_t>(nnz_in, 1);
  s = dalloc(c, reinterpret_cast<void**>(&G->row_ptr), size_t(n + 1) * 8);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&G->col), size_t(G->col_cap) * 4);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&rp_in), size_t(n + 1) * 8);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&col_in), size_t(std::max<int64_t>(nnz_in, 1)) * 4);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&cnt), size_t(n) * 4);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&bsum), size_t(nblk) * 8);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&maxd), 8);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&med), 8);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&mean), size_t(d) * 8);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&best), size_t(2 * medoid_blocks(n)) * 8);
  if (s != RP_OK) {
    cleanup();
    return s;
  }
  const cudaMemcpyKind kind = mem_flags == RP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t ce = cudaSuccess;
  if (row_ptr) {
    ce = cudaMemcpyAsync(rp_in, row_ptr, size_t(n + 1) * 8, kind, c->stream);
    if (ce == cudaSuccess && nnz_in > 0) ce = cudaMemcpyAsync(col_in, col, size_t(nnz_in) * 4, kind, c->stream);
  } else {
    ce = cudaMemsetAsync(rp_in, 0, size_t(n + 1) * 8, c->stream);
  }
  const unsigned long long zero2[2] = {0, 0};
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(c->dropped, zero2, 16, cudaMemcpyHostToDevice, c->stream);
  if (ce == cudaSuccess) ce = launch_validate_csr(rp_in, col_in, n, nnz_in, c->status, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) {
    cleanup();
    return fail(c, RP_ECUDA, "graph upload/validate: %s", cudaGetErrorString(ce));
  }
  if ((s = check_device_status(c)) != RP_OK) {
    cleanup();
    return fail(c, RP_EINVAL, "invalid input: %s", c->err.c_str());
  }
  ce = launch_clean_count(rp_in, col_in, n, cnt, c->dropped, c->stream);
  if (ce == cudaSuccess) ce = launch_scan_counts(cnt, n, G->row_ptr, bsum, maxd, c->stream);
  if (ce == cudaSuccess) ce = launch_clean_write(rp_in, col_in, n, G->row_ptr, G->col, c->stream);
  if (ce == cudaSuccess && start < 0) ce = launch_medoid(G->data->dev(), mean, best, med, c->stream);
  int64_t nnz = 0, medoid = start;
  int32_t maxdeg = 0;
  unsigned long long dropped[2] = {0, 0};
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&nnz, G->row_ptr + n, 8, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&maxdeg, maxd, 4, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess && start < 0) ce = cudaMemcpyAsync(&medoid, med, 8, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(dropped, c->dropped, 16, cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  cleanup();
  if (ce != cudaSuccess) return fail(c, RP_ECUDA, "graph cleaning: %s", cudaGetErrorString(ce));
  if ((s = check_device_status(c)) != RP_OK) return s;
  if (maxdeg > RP_MAX_DEGREE)
    return fail(c, RP_EINVAL, "out-degree %d after cleaning exceeds RP_MAX_DEGREE=%d", maxdeg, RP_MAX_DEGREE);
  G->nnz = nnz;
  G->max_deg_bound = maxdeg;
  G->start = medoid;
  G->bytes = size_t(n + 1) * 8 + size_t(G->col_cap) * 4;
  static_assert(sizeof(unsigned long long) == 8, "");
  // stats carry the cleaning counters in the spare slots of the status word
  unsigned long long add[2] = {dropped[0], dropped[1]};
  DevStatus hs;
  cudaMemcpyAsync(&hs, c->status, sizeof hs, cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  hs.spare[0] += add[0];
  hs.spare[1] += add[1];
  cudaMemcpyAsync(c->status, &hs, sizeof hs, cudaMemcpyHostToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  return RP_OK;
}

extern "C" {

rp_status rp_create(rp_ctx** out, int32_t device, uint64_t hbm_budget_bytes, void* cuda_stream) {
  if (!out) return RP_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return RP_EINVAL;
  }
  std::unique_ptr<rp_ctx> c(new rp_ctx);
  c->device = device;
  c->budget = hbm_budget_bytes;
  if (cudaSetDevice(device) != cudaSuccess) return RP_ECUDA;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return RP_ECUDA;
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    // searches on this stream run ahead of asynchronous tuning (lowest priority)
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return RP_ECUDA;
    if (cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, greatest) != cudaSuccess) return RP_ECUDA;
    c->own_stream = true;
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached in this process
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (dalloc(c.get(), reinterpret_cast<void**>(&c->status), sizeof(DevStatus)) != RP_OK) return RP_ECUDA;
  if (dalloc(c.get(), reinterpret_cast<void**>(&c->dropped), 2 * sizeof(unsigned long long)) != RP_OK)
    return RP_ECUDA;
  if (dalloc(c.get(), reinterpret_cast<void**>(&c->work), 8 * sizeof(unsigned)) != RP_OK) return RP_ECUDA;
  if (dalloc(c.get(), reinterpret_cast<void**>(&c->hits), sizeof(unsigned long long)) != RP_OK) return RP_ECUDA;
  if (cudaMemsetAsync(c->status, 0, sizeof(DevStatus), c->stream) != cudaSuccess) return RP_ECUDA;
  if (cudaMemsetAsync(c->dropped, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess) return RP_ECUDA;
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return RP_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RP_ECUDA;
  *out = c.release();
  return RP_OK;
}

rp_status rp_destroy(rp_ctx* c) {
  if (!c) return RP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& kv : c->graphs) free_graph_mem(c, kv.second);
    c->graphs.clear();
    for (auto& pl : c->plans)
      if (pl.exec) cudaGraphExecDestroy(pl.exec);
    dfree(c, c->scratch_col, size_t(c->scratch_col_elems) * 4);
    dfree(c, c->scratch_cnt, size_t(c->scratch_cnt_elems) * 4);
    dfree(c, c->scratch_bsum, size_t(c->scratch_bsum_elems) * 8);
    dfree(c, c->qbuf, size_t(c->qbuf_bytes));
    dfree(c, c->status, sizeof(DevStatus));
    dfree(c, c->dropped, 16);
    dfree(c, c->work, 32);
    dfree(c, c->hits, 8);
    if (c->trial_count) dfree(c, c->trial_count, 16);
    if (c->tune_stream) cudaStreamSynchronize(c->tune_stream);
    dfree(c, c->a_col, size_t(c->a_col_elems) * 4);
    dfree(c, c->a_cnt, size_t(c->a_cnt_elems) * 4);
    dfree(c, c->a_bsum, size_t(c->a_bsum_elems) * 8);
    dfree(c, c->a_chunk, size_t(c->a_chunk_elems) * 4);
    cudaStreamSynchronize(c->stream);
    if (c->tune_ready) cudaEventDestroy(c->tune_ready);
    if (c->tune_inputs) cudaEventDestroy(c->tune_inputs);
    if (c->tune_stream) cudaStreamDestroy(c->tune_stream);
    for (auto& e : c->ev)
      if (e) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
  }
  delete c;
  return RP_OK;
}

const char* rp_last_error(const rp_ctx* c) { return c ? c->err.c_str() : "null context"; }

rp_status rp_sync(rp_ctx* c) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return check_device_status(c);
}

rp_status rp_load_graph(rp_ctx* c, const void* vectors, int32_t dtype, int64_t n, int32_t d, const int64_t* row_ptr,
                        const int32_t* col, int32_t start, int32_t mem_flags, rp_graph* base_out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (!base_out || !vectors) return fail(c, RP_EINVAL, "null argument");
  if (dtype != RP_U8 && dtype != RP_F32) return fail(c, RP_EINVAL, "bad dtype %d", dtype);
  if (n < 1 || n > INT32_MAX || d < 1 || d > 65536) return fail(c, RP_EINVAL, "bad shape n=%lld d=%d", (long long)n, d);
  if (start < -1 || start >= n) return fail(c, RP_EINVAL, "start=%d outside [-1, n)", start);
  if (mem_flags != RP_MEM_HOST && mem_flags != RP_MEM_DEVICE) return fail(c, RP_EINVAL, "bad mem_flags");
  if (dtype == RP_U8 && d > 4096) return fail(c, RP_EINVAL, "uint8 vectors are limited to d <= 4096");

  auto D = std::make_shared<Dataset>();
  D->n = n;
  D->d = d;
  D->dtype = dtype;
  D->row_bytes = padded_row_bytes(d, dtype);
  D->bytes = size_t(n * D->row_bytes);
  rp_status s = dalloc(c, reinterpret_cast<void**>(&D->X), D->bytes);
  if (s != RP_OK) return s;
  auto fail_free = [&](rp_status st) {
    dfree(c, D->X, D->bytes);
    D->X = nullptr;
    return st;
  };
  if ((s = upload_rows(c, D->X, D->row_bytes, vectors, n, d, dtype, mem_flags)) != RP_OK) return fail_free(s);
  if (launch_check_finite(D->dev(), c->status, c->stream) != cudaSuccess)
    return fail_free(fail(c, RP_ECUDA, "check_finite launch failed"));
  if (dtype == RP_F32) {
    // the power-of-two scale under which float rows enter the f16 Gram
    unsigned mb = 0;
    CUDA_TRY(c, cudaMemsetAsync(c->work, 0, 4, c->stream));
    CUDA_TRY(c, launch_maxabs_f32(D->X, D->row_bytes, n, d, c->work, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&mb, c->work, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    float mx = 0.f;
    memcpy(&mx, &mb, 4);
    c->kernel_launches += 1;
    // |x| <= 2^50 keeps every squared distance below 2^120 even at d = 65536,
    // so no single-precision sum on the path can overflow.
    if (std::isfinite(mx) && mx > 1125899906842624.f)  // non-finite rows: the status check below
      return fail_free(fail(c, RP_EINVAL, "float rows with |x| above 2^50 (max %g) are not supported", double(mx)));
    int e = 0;
    if (mx > 0.f && std::isfinite(mx)) std::frexp(mx, &e);  // mx < 2^e
    D->scale = std::ldexp(1.f, -e);
  }

  Graph* G = new Graph;
  G->data = D;
  G->n = n;
  D.reset();  // the graph owns the vectors now: freeing it on failure frees them
  if ((s = attach_csr(c, G, row_ptr, col, start, mem_flags)) != RP_OK) {
    free_graph_mem(c, G);
    return s;
  }
  *base_out = add_graph(c, G);
  return RP_OK;
}

rp_status rp_graph_attach(rp_ctx* c, rp_graph data, const int64_t* row_ptr, const int32_t* col, int32_t mem_flags,
                          rp_graph* out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (!out || !row_ptr) return fail(c, RP_EINVAL, "null argument");
  if (mem_flags != RP_MEM_HOST && mem_flags != RP_MEM_DEVICE) return fail(c, RP_EINVAL, "bad mem_flags");
  Graph* D = find_graph(c, data);
  if (!D) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)data);
  Graph* G = new Graph;
  G->data = D->data;
  G->n = D->n;
  const rp_status s = attach_csr(c, G, row_ptr, col, D->start, mem_flags);
  if (s != RP_OK) {
    free_graph_mem(c, G);
    return s;
  }
  *out = add_graph(c, G);
  return RP_OK;
}

rp_status rp_tune(rp_ctx* c, rp_graph src, double alpha, int32_t R, int32_t variant, rp_graph* out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return tune_impl(c, src, &alpha, &R, 1, variant, out, false);
}

rp_status rp_tune_batch(rp_ctx* c, rp_graph src, const double* alphas, const int32_t* Rs, int32_t T,
                        int32_t variant, rp_graph* outs) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return tune_impl(c, src, alphas, Rs, T, variant, outs, true);
}

rp_status rp_debug_gram(rp_ctx* c, rp_graph g, const int32_t* rows, const int32_t* centres, int64_t nrows,
                        float* out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  Graph* G = find_graph(c, g);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  if (G->data->dtype != RP_F32) return fail(c, RP_EINVAL, "the split Gram is for float rows");
  if (!rows || !out || nrows < 0 || nrows % 128 != 0) return fail(c, RP_EINVAL, "need rows and out, nrows a multiple of 128");
  for (int64_t i = 0; i < nrows; ++i)
    if (rows[i] < 0 || rows[i] >= G->n) return fail(c, RP_EINVAL, "rows[%lld]=%d outside [0, n)", (long long)i, rows[i]);
  const int64_t ncen = centres ? nrows / 64 : 0;
  for (int64_t i = 0; i < ncen; ++i)
    if (centres[i] < 0 || centres[i] >= G->n)
      return fail(c, RP_EINVAL, "centres[%lld]=%d outside [0, n)", (long long)i, centres[i]);
  if (nrows == 0) return RP_OK;
  int32_t* drows = nullptr;
  float* dout = nullptr;
  const size_t row_bytes = size_t(nrows + ncen) * 4;  // rows, then the centres
  rp_status s = dalloc(c, reinterpret_cast<void**>(&drows), row_bytes);
  if (s == RP_OK) s = dalloc(c, reinterpret_cast<void**>(&dout), size_t(nrows) * 128 * 4);
  cudaError_t ce = cudaSuccess;
  if (s == RP_OK) {
    ce = cudaMemcpyAsync(drows, rows, size_t(nrows) * 4, cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess && ncen)
      ce = cudaMemcpyAsync(drows + nrows, centres, size_t(ncen) * 4, cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess)
      ce = launch_gram_probe(G->data->dev(), drows, ncen ? drows + nrows : nullptr, nrows / 128, dout, c->status,
                             c->num_sms, c->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, dout, size_t(nrows) * 128 * 4, cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    c->kernel_launches += 1;
  }
  dfree(c, drows, row_bytes);
  dfree(c, dout, size_t(nrows) * 128 * 4);
  if (s != RP_OK) return s;
  if (ce != cudaSuccess) return fail(c, RP_ECUDA, "Gram probe: %s", cudaGetErrorString(ce));
  return check_device_status(c);
}

rp_status rp_tune_batch_async(rp_ctx* c, rp_graph src, const double* alphas, const int32_t* Rs, int32_t T,
                              int32_t variant, int32_t chunks, rp_graph* outs, int64_t* ticket) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return tune_async_impl(c, src, alphas, Rs, T, variant, chunks, outs, ticket);
}

rp_status rp_tune_wait(rp_ctx* c, int64_t ticket, int32_t timeout_ms) {
  if (!c) return RP_EINVAL;
  if (timeout_ms < 0) return fail(c, RP_EINVAL, "timeout_ms=%d", timeout_ms);
  const auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(c->mu);
      cudaSetDevice(c->device);
      if (ticket < 1 || ticket > c->tune_ticket) return fail(c, RP_ENOTFOUND, "unknown tuning ticket %lld", (long long)ticket);
      // jobs run one after another, so an earlier ticket is done once the latest is
      const cudaError_t e = cudaEventQuery(c->tune_ready);
      if (e == cudaSuccess) return check_device_status(c);
      if (e != cudaErrorNotReady) return fail(c, RP_ECUDA, "tuning: %s", cudaGetErrorString(e));
      if (ticket < c->tune_ticket) return RP_OK;  // a later job was started, so this one finished before it
    }
    if (std::chrono::steady_clock::now() >= t_end) return RP_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

rp_status rp_graph_info(rp_ctx* c, rp_graph g, int64_t* n, int64_t* nnz, int32_t* max_deg, int64_t* start) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  Graph* G = find_graph(c, g);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  if (G->nnz < 0 || max_deg) {
    std::vector<int64_t> h(size_t(G->n + 1));
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), G->row_ptr, size_t(G->n + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    G->nnz = h[size_t(G->n)];
    int64_t mx = 0;
    for (int64_t p = 0; p < G->n; ++p) mx = std::max(mx, h[size_t(p + 1)] - h[size_t(p)]);
    G->max_deg_bound = int(mx);
    if (max_deg) *max_deg = int32_t(mx);
  }
  if (n) *n = G->n;
  if (nnz) *nnz = G->nnz;
  if (start) *start = G->start;
  return check_device_status(c);
}

rp_status rp_graph_export(rp_ctx* c, rp_graph g, int64_t* row_ptr, int32_t* col, int64_t col_cap,
                          int32_t mem_flags) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  Graph* G = find_graph(c, g);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  if (!row_ptr || (!col && col_cap > 0)) return fail(c, RP_EINVAL, "null argument");
  if (G->nnz < 0) {
    CUDA_TRY(c, cudaMemcpyAsync(&G->nnz, G->row_ptr + G->n, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  if (col_cap < G->nnz) return fail(c, RP_EINVAL, "col_cap=%lld < nnz=%lld", (long long)col_cap, (long long)G->nnz);
  const cudaMemcpyKind kind = mem_flags == RP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CUDA_TRY(c, cudaMemcpyAsync(row_ptr, G->row_ptr, size_t(G->n + 1) * 8, kind, c->stream));
  if (G->nnz > 0) CUDA_TRY(c, cudaMemcpyAsync(col, G->col, size_t(G->nnz) * 4, kind, c->stream));
  if (mem_flags == RP_MEM_HOST) {
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return check_device_status(c);
  }
  return RP_OK;
}

rp_status rp_graph_slice(rp_ctx* c, rp_graph g, int64_t lo, int64_t hi, rp_graph* out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  Graph* G = find_graph(c, g);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  if (!out || lo < 0 || hi < lo || hi > G->n)
    return fail(c, RP_EINVAL, "need 0 <= lo <= hi <= n (lo=%lld hi=%lld n=%lld)", (long long)lo, (long long)hi,
                (long long)G->n);
  int64_t e[2] = {0, 0};
  CUDA_TRY(c, cudaMemcpyAsync(&e[0], G->row_ptr + lo, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&e[1], G->row_ptr + hi, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int64_t nnz = e[1] - e[0];
  Graph* S = new Graph;
  S->data = G->data;
  S->n = G->n;
  S->col_cap = std::max<int64_t>(nnz, 1);
  S->nnz = nnz;
  S->start = G->start;
  S->max_deg_bound = G->max_deg_bound;
  S->bytes = size_t(G->n + 1) * 8 + size_t(S->col_cap) * 4;
  rp_status st = dalloc(c, reinterpret_cast<void**>(&S->row_ptr), size_t(G->n + 1) * 8);
  if (st == RP_OK) st = dalloc(c, reinterpret_cast<void**>(&S->col), size_t(S->col_cap) * 4);
  if (st != RP_OK) {
    free_graph_mem(c, S);
    return st;
  }
  CUDA_TRY(c, launch_slice_row_ptr(G->row_ptr, G->n, lo, hi, S->row_ptr, c->stream));
  c->kernel_launches += 1;
  if (nnz > 0) CUDA_TRY(c, cudaMemcpyAsync(S->col, G->col + e[0], size_t(nnz) * 4, cudaMemcpyDeviceToDevice, c->stream));
  *out = add_graph(c, S);
  return RP_OK;
}

rp_status rp_graph_shape(rp_ctx* c, rp_graph g, int32_t* d, int32_t* dtype, uint64_t* adj_bytes) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  Graph* G = find_graph(c, g);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  if (d) *d = G->data->d;
  if (dtype) *dtype = G->data->dtype;
  if (adj_bytes) *adj_bytes = uint64_t(G->n + 1) * 8 + uint64_t(std::max<int64_t>(G->col_cap, 1)) * 4;
  return RP_OK;
}

rp_status rp_graph_free(rp_ctx* c, rp_graph g) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  auto it = c->graphs.find(g);
  if (it == c->graphs.end()) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  for (auto pl = c->plans.begin(); pl != c->plans.end();) {
    if (pl->src == g) {
      if (pl->exec) cudaGraphExecDestroy(pl->exec);
      pl = c->plans.erase(pl);
    } else {
      ++pl;
    }
  }
  free_graph_mem(c, it->second);
  c->graphs.erase(it);
  return RP_OK;
}

rp_status rp_search(rp_ctx* c, rp_graph g, const void* queries, int64_t nq, int32_t L, int32_t k, int32_t* ids,
                    float* dists, int32_t mem_flags) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return search_impl(c, &g, 1, nullptr, nullptr, queries, nq, L, k, ids, dists, mem_flags);
}

rp_status rp_search_multi(rp_ctx* c, const rp_graph* graphs, int32_t ngraphs, const int32_t* q_graph,
                          const int32_t* q_L, const void* queries, int64_t nq, int32_t k, int32_t* ids, float* dists,
                          int32_t mem_flags) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (!graphs || ngraphs < 1 || (nq > 0 && (!q_graph || !q_L)))
    return fail(c, RP_EINVAL, "need ngraphs >= 1 and per-query graph indexes and list sizes");
  int32_t Lmax = k;
  for (int64_t i = 0; i < nq; ++i) {
    if (q_graph[i] < 0 || q_graph[i] >= ngraphs)
      return fail(c, RP_EINVAL, "query %lld: graph index %d outside [0, %d)", (long long)i, q_graph[i], ngraphs);
    if (q_L[i] < k || q_L[i] > RP_MAX_L)
      return fail(c, RP_EINVAL, "query %lld: need k <= L <= %d (L=%d k=%d)", (long long)i, RP_MAX_L, q_L[i], k);
    Lmax = std::max(Lmax, q_L[i]);
  }
  return search_impl(c, graphs, ngraphs, q_graph, q_L, queries, nq, Lmax, k, ids, dists, mem_flags);
}

rp_status rp_knn(rp_ctx* c, rp_graph g, const void* queries, int64_t nq, int32_t k, int32_t* ids, float* dists,
                 int32_t mem_flags) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  Graph* G = find_graph(c, g);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  const Dataset& D = *G->data;
  if (k < 1 || k > 1024 || nq < 0 || (!queries && nq > D.n))
    return fail(c, RP_EINVAL, "need 1 <= k <= 1024, nq >= 0 (nq <= n without queries)");
  if (nq == 0) return RP_OK;
  if (!ids) return fail(c, RP_EINVAL, "null ids");
  rp_status s;
  const int64_t qbytes = queries ? nq * D.row_bytes : 0;
  const int64_t out_bytes = nq * k * 8;
  if ((s = grow(c, &c->qbuf, &c->qbuf_bytes, qbytes + (mem_flags == RP_MEM_HOST ? out_bytes : 0))) != RP_OK) return s;
  if (queries && (s = upload_rows(c, c->qbuf, D.row_bytes, queries, nq, D.d, D.dtype, mem_flags)) != RP_OK) return s;
  int32_t* dev_ids = ids;
  float* dev_d = dists;
  if (mem_flags == RP_MEM_HOST) {
    dev_ids = reinterpret_cast<int32_t*>(c->qbuf + qbytes);
    dev_d = reinterpret_cast<float*>(c->qbuf + qbytes + nq * k * 4);
  }
  if ((s = run_knn(c, D, queries ? c->qbuf : nullptr, nq, k, dev_ids, dev_d)) != RP_OK) return s;
  if (mem_flags == RP_MEM_HOST) {
    CUDA_TRY(c, cudaMemcpyAsync(ids, dev_ids, size_t(nq * k) * 4, cudaMemcpyDeviceToHost, c->stream));
    if (dists) CUDA_TRY(c, cudaMemcpyAsync(dists, dev_d, size_t(nq * k) * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return check_device_status(c);
  }
  return RP_OK;
}

rp_status rp_recall(rp_ctx* c, const int32_t* found, int32_t ld_found, const int32_t* truth, int32_t ld_truth,
                    int64_t nq, int32_t k, int64_t* hits, int32_t mem_flags) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (!hits || k < 1 || ld_found < k || ld_truth < k || nq < 0 || k > 1024)
    return fail(c, RP_EINVAL, "need 1 <= k <= min(ld_found, ld_truth, 1024)");
  *hits = 0;
  if (nq == 0) return RP_OK;
  const int32_t* df = found;
  const int32_t* dt = truth;
  rp_status s;
  if (mem_flags == RP_MEM_HOST) {
    const int64_t need = nq * (int64_t(ld_found) + ld_truth) * 4;
    if ((s = grow(c, &c->qbuf, &c->qbuf_bytes, need)) != RP_OK) return s;
    int32_t* a = reinterpret_cast<int32_t*>(c->qbuf);
    int32_t* b = a + nq * ld_found;
    CUDA_TRY(c, cudaMemcpyAsync(a, found, size_t(nq * ld_found) * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(b, truth, size_t(nq * ld_truth) * 4, cudaMemcpyHostToDevice, c->stream));
    df = a;
    dt = b;
  }
  CUDA_TRY(c, cudaMemsetAsync(c->hits, 0, 8, c->stream));
  CUDA_TRY(c, launch_recall(df, ld_found, dt, ld_truth, nq, k, c->hits, c->stream));
  c->kernel_launches += 1;
  unsigned long long h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->hits, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *hits = int64_t(h);
  return check_device_status(c);
}

rp_status rp_reachability(rp_ctx* c, rp_graph g, const int64_t* nodes, int64_t n_nodes, double* per_node,
                          double* alpha_star) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  Graph* G = find_graph(c, g);
  if (!G) return fail(c, RP_ENOTFOUND, "unknown graph %lld", (long long)g);
  if (!alpha_star && !per_node) return fail(c, RP_EINVAL, "nothing to return: per_node and alpha_star are null");
  if (nodes && n_nodes < 0) return fail(c, RP_EINVAL, "n_nodes=%lld", (long long)n_nodes);
  const int64_t m = nodes ? n_nodes : G->n;
  for (int64_t i = 0; nodes && i < m; ++i)
    if (nodes[i] < 0 || nodes[i] >= G->n)
      return fail(c, RP_EINVAL, "nodes[%lld]=%lld outside [0, %lld)", (long long)i, (long long)nodes[i],
                  (long long)G->n);
  if (alpha_star) *alpha_star = INFINITY;
  if (m == 0) return RP_OK;
  rp_status s;
  const int64_t need = m * 8 * (nodes ? 2 : 1);
  if ((s = grow(c, &c->qbuf, &c->qbuf_bytes, need)) != RP_OK) return s;
  double* d_out = reinterpret_cast<double*>(c->qbuf);
  int64_t* d_nodes = nullptr;
  if (nodes) {
    d_nodes = reinterpret_cast<int64_t*>(d_out + m);
    CUDA_TRY(c, cudaMemcpyAsync(d_nodes, nodes, size_t(m) * 8, cudaMemcpyHostToDevice, c->stream));
  }
  CUDA_TRY(c, launch_reach(G->data->dev(), G->row_ptr, G->col, d_nodes, m, d_out, c->stream));
  c->kernel_launches += 1;
  std::vector<double> h(static_cast<size_t>(m));
  CUDA_TRY(c, cudaMemcpyAsync(h.data(), d_out, size_t(m) * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (per_node) std::memcpy(per_node, h.data(), size_t(m) * 8);
  if (alpha_star)
    for (double v : h) *alpha_star = std::min(*alpha_star, v);
  return check_device_status(c);
}

rp_status rp_build_knn_base(rp_ctx* c, rp_graph data, int32_t kcand, double alpha, int32_t R, rp_graph* out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return build_base(c, data, kcand, 0, 0, alpha, R, out);
}

rp_status rp_build_knn_random_base(rp_ctx* c, rp_graph data, int32_t kcand, int32_t nrand, uint64_t seed,
                                   double alpha, int32_t R, rp_graph* out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return build_base(c, data, kcand, nrand, seed, alpha, R, out);
}

rp_status rp_build_vamana(rp_ctx* c, rp_graph data, const int32_t* perm, int32_t npass, const double* alphas,
                          int32_t R, int32_t L, int32_t vcap, int64_t max_batch, int64_t* visited_cut,
                          rp_graph* out) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return build_vamana(c, data, perm, npass, alphas, R, L, vcap, max_batch, visited_cut, out);
}

rp_status rp_set_search_config(rp_ctx* c, int32_t cache_bits, int32_t ctas_per_sm) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (cache_bits != 0 && (cache_bits < 8 || cache_bits > 12))
    return fail(c, RP_EINVAL, "cache_bits=%d: use 0 or 8..12", cache_bits);
  if (ctas_per_sm < 0 || ctas_per_sm > 16) return fail(c, RP_EINVAL, "ctas_per_sm=%d outside 0..16", ctas_per_sm);
  c->search_cache_bits = cache_bits;
  c->search_ctas = ctas_per_sm;
  return RP_OK;
}

rp_status rp_set_knn_method(rp_ctx* c, int32_t method) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (method != RP_KNN_AUTO && method != RP_KNN_CUDA_CORE && method != RP_KNN_TENSOR)
    return fail(c, RP_EINVAL, "unknown kNN method %d", method);
  c->knn_method = method;
  return RP_OK;
}

rp_status rp_set_tuning(rp_ctx* c, int32_t mode, int32_t tile0, int32_t ctas_per_sm) {
  if (!c) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (mode != RP_TUNING_AUTO && mode != RP_TUNING_FIXED)
    return fail(c, RP_EINVAL, "tuning mode %d is neither RP_TUNING_AUTO nor RP_TUNING_FIXED", mode);
  if (mode == RP_TUNING_FIXED && (tile0 < 0 || tile0 > 1 || ctas_per_sm < 0 || ctas_per_sm > 4))
    return fail(c, RP_EINVAL, "need tile0 in {0, 1} and ctas_per_sm in 0..4 (got %d, %d)", tile0, ctas_per_sm);
  c->tuning_mode = mode;
  c->fixed_tile0 = mode == RP_TUNING_FIXED ? tile0 : 0;
  c->fixed_ctas = mode == RP_TUNING_FIXED ? ctas_per_sm : 0;
  return RP_OK;
}

rp_status rp_stats(rp_ctx* c, rp_stats_t* out, int32_t reset) {
  if (!c || !out) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  DevStatus h;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->status, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof *out);
  out->nodes_pruned = int64_t(h.nodes_pruned);
  out->fp64_decisions = int64_t(h.fp64_decisions);
  out->fp64_sort_keys = int64_t(h.fp64_sort_keys);
  out->fp64_search_dists = int64_t(h.fp64_search);
  out->generic_nodes = int64_t(h.generic_nodes);
  out->self_loops_dropped = int64_t(h.spare[0]);
  out->duplicates_dropped = int64_t(h.spare[1]);
  out->graph_replays = c->graph_replays;
  out->bytes_in_use = c->used;
  out->bytes_peak = c->peak;
  out->kernel_launches = c->kernel_launches;
  if (c->ev_tune) {
    cudaEventElapsedTime(&out->last_prune_ms, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&out->last_emit_ms, c->ev[1], c->ev[2]);
  }
  if (c->ev_search) cudaEventElapsedTime(&out->last_search_ms, c->ev[3], c->ev[4]);
  cudaGetLastError();
  out->tile0 = c->last_tile0;
  out->ctas_per_sm = c->last_ctas;
  out->knn_method = c->last_knn_method;
  out->f32_rechecks = int64_t(h.spare[2]);
  if (reset) {
    DevStatus z;
    memset(&z, 0, sizeof z);
    z.code = h.code;
    z.info = h.info;
    CUDA_TRY(c, cudaMemcpyAsync(c->status, &z, sizeof z, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->graph_replays = 0;
    c->kernel_launches = 0;
    c->peak = c->used;
  }
  return RP_OK;
}

}  // extern "C"
