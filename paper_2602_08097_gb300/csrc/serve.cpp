// Serving scheduler of librp.so: one thread per server runs scheduling rounds
// over the requests that have arrived (continuous batching), keeps tuned
// graphs resident under a byte budget with least-recently-used eviction, and
// records per-request timestamps.  All device work goes through an executor
// (rp_executor); rp_server_create builds one over an rp_ctx.  The public
// contract is documented in include/rp.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "rp.h"

namespace {

constexpr int kMaxTargets = 16;
constexpr int64_t kDefaultBatch = 65536;

// (A, R) with A = round(1000 alpha); A = 0 addresses the base graph.
using Key = std::pair<int32_t, int32_t>;

bool alpha_key(double alpha, int32_t* A) {
  if (alpha == 0.0) {
    *A = 0;
    return true;
  }
  if (!(alpha >= 1.0) || !(alpha <= 100.0)) return false;
  const double m = alpha * 1000.0;
  const double r = std::nearbyint(m);
  if (std::fabs(m - r) > 1e-6) return false;
  *A = int32_t(r);
  return true;
}

struct Req {
  int64_t id = 0;
  bool search = false;
  Key key{0, 0};
  std::vector<uint8_t> q;  // packed query rows
  int64_t nq = 0;
  int32_t L_eff = 0, k = 0;
  int32_t* ids = nullptr;
  float* dists = nullptr;
  rp_status status = RP_OK;  // written by the scheduler, published into info when done
  rp_graph graph = 0;
  rp_request_info info{};    // read by rp_poll under the server mutex
};

int64_t now_ns(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
}

// ---- executor over an rp_ctx
struct CtxExec {
  rp_ctx* ctx;
};

rp_status ctx_tune(void* u, rp_graph src, const double* a, const int32_t* R, int32_t T, rp_graph* outs) {
  return rp_tune_batch(static_cast<CtxExec*>(u)->ctx, src, a, R, T, RP_SORTED, outs);
}

rp_status ctx_search(void* u, const rp_graph* g, int32_t ng, const int32_t* qg, const int32_t* qL, const void* Q,
                     int64_t nq, int32_t k, int32_t* ids, float* dists) {
  return rp_search_multi(static_cast<CtxExec*>(u)->ctx, g, ng, qg, qL, Q, nq, k, ids, dists, RP_MEM_HOST);
}

rp_status ctx_free(void* u, rp_graph g) { return rp_graph_free(static_cast<CtxExec*>(u)->ctx, g); }

// Asynchronous tuning over the ctx: chunks of about 256K nodes, so that a
// search waits at most for one chunk.
rp_status ctx_tune_start(void* u, rp_graph src, const double* a, const int32_t* R, int32_t T, rp_graph* outs,
                         int64_t* ticket) {
  rp_ctx* ctx = static_cast<CtxExec*>(u)->ctx;
  int64_t n = 0, nnz = 0, start = 0;
  int32_t md = 0;
  rp_status st = rp_graph_info(ctx, src, &n, &nnz, &md, &start);
  if (st != RP_OK) return st;
  const int32_t chunks = int32_t(std::min<int64_t>(64, std::max<int64_t>(1, n / 262144)));
  return rp_tune_batch_async(ctx, src, a, R, T, RP_SORTED, chunks, outs, ticket);
}

rp_status ctx_tune_ready(void* u, int64_t ticket, int32_t timeout_ms) {
  return rp_tune_wait(static_cast<CtxExec*>(u)->ctx, ticket, timeout_ms);
}

}  // namespace

struct rp_server {
  rp_executor ex{};
  rp_server_config cfg{};
  CtxExec ctx_exec{};
  size_t row_bytes = 0;   // packed query row
  int64_t capacity = 0;   // tuned graphs that fit in the budget
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::unordered_map<int64_t, Req*> reqs;  // every request not yet reaped by rp_poll
  int64_t next_id = 1;
  bool stop = false;
  rp_server_stats_t stats{};
  std::string err;

  // scheduler-thread state
  struct Inflight {
    bool active = false;
    int64_t ticket = 0;
    std::vector<Key> keys;
    std::vector<rp_graph> outs;
  } inflight;                 // the asynchronous tuning job running now
  std::vector<Req*> parked;   // admitted requests waiting for a graph being tuned (or to be)
  std::list<std::pair<Key, rp_graph>> lru;  // front = least recently used
  std::map<Key, std::list<std::pair<Key, rp_graph>>::iterator> resident;
  std::vector<uint8_t> qbuf;
  std::vector<int32_t> ibuf;
  std::vector<float> dbuf;
  std::thread worker;

  void set_error(const char* fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(mu);
    err = b;
  }

  void run();
  void round(std::vector<Req*>& batch, int32_t round_no);
  void round_async(std::vector<Req*>& batch, int32_t* round_no);
  void run_searches(std::vector<Req*>& rs);
  void publish(std::vector<Req*>& rs);
  void evict_for(size_t nnew, const std::map<Key, int>& needed);
};

void rp_server::evict_for(size_t nnew, const std::map<Key, int>& needed) {
  auto it = lru.begin();
  while (int64_t(lru.size() + nnew) > capacity && it != lru.end()) {
    if (needed.count(it->first)) {
      ++it;
      continue;
    }
    const rp_status s = ex.graph_free(ex.user, it->second);
    if (s != RP_OK) set_error("freeing tuned graph (%d, %d) failed with status %d", it->first.first,
                              it->first.second, s);
    resident.erase(it->first);
    it = lru.erase(it);
    std::lock_guard<std::mutex> lk(mu);
    stats.evictions += 1;
  }
}

void rp_server::run_searches(std::vector<Req*>& rs) {
  auto graph_of = [&](const Key& k) -> rp_graph {
    if (k.first == 0) return cfg.base;
    auto it = resident.find(k);
    return it == resident.end() ? 0 : it->second->second;
  };
  for (Req* r : rs)
    if (r->status == RP_OK) r->graph = graph_of(r->key);
  // one mixed search launch per k
  std::map<int32_t, std::vector<Req*>> by_k;
  for (Req* r : rs)
    if (r->search && r->status == RP_OK) by_k[r->k].push_back(r);
  for (auto& kv : by_k) {
    const int32_t k = kv.first;
    std::vector<Req*>& group = kv.second;
    std::vector<rp_graph> graphs;
    std::map<rp_graph, int32_t> gidx;
    std::vector<int32_t> qg, qL;
    int64_t nq = 0;
    for (Req* r : group) nq += r->nq;
    qbuf.resize(size_t(nq) * row_bytes);
    ibuf.resize(size_t(nq) * size_t(k));
    dbuf.resize(size_t(nq) * size_t(k));
    qg.reserve(size_t(nq));
    qL.reserve(size_t(nq));
    int64_t off = 0;
    for (Req* r : group) {
      auto ins = gidx.emplace(r->graph, int32_t(graphs.size()));
      if (ins.second) graphs.push_back(r->graph);
      std::memcpy(qbuf.data() + size_t(off) * row_bytes, r->q.data(), size_t(r->nq) * row_bytes);
      for (int64_t i = 0; i < r->nq; ++i) {
        qg.push_back(ins.first->second);
        qL.push_back(r->L_eff);
      }
      off += r->nq;
    }
    const rp_status s = ex.search_multi(ex.user, graphs.data(), int32_t(graphs.size()), qg.data(), qL.data(),
                                        qbuf.data(), nq, k, ibuf.data(), dbuf.data());
    if (s != RP_OK) set_error("search launch over %lld queries failed with status %d", (long long)nq, s);
    off = 0;
    for (Req* r : group) {
      if (s == RP_OK) {
        const size_t m = size_t(r->nq) * size_t(k);
        std::memcpy(r->ids, ibuf.data() + size_t(off) * size_t(k), m * 4);
        if (r->dists) std::memcpy(r->dists, dbuf.data() + size_t(off) * size_t(k), m * 4);
      } else {
        r->status = s;
        r->graph = 0;
      }
      off += r->nq;
    }
    std::lock_guard<std::mutex> lk(mu);
    stats.search_launches += 1;
  }
}

void rp_server::publish(std::vector<Req*>& rs) {
  const int64_t t_done = now_ns(t0);
  std::lock_guard<std::mutex> lk(mu);
  for (Req* r : rs) {
    r->info.state = RP_REQ_DONE;
    r->info.status = r->status;
    r->info.graph = r->graph;
    r->info.done_ns = t_done;
    r->q.clear();
    r->q.shrink_to_fit();
    if (r->status == RP_OK) {
      stats.requests_done += 1;
      stats.queries_done += r->nq;
    } else {
      stats.requests_failed += 1;
    }
  }
  cv_done.notify_all();
}

void rp_server::round(std::vector<Req*>& batch, int32_t round_no) {
  const int64_t t_start = now_ns(t0);
  {
    std::lock_guard<std::mutex> lk(mu);
    for (Req* r : batch) {
      r->info.state = RP_REQ_RUNNING;
      r->info.start_ns = t_start;
      r->info.round = round_no;
    }
  }
  // graphs this round needs, in order of first use
  std::map<Key, int> needed;  // key -> order
  std::vector<Key> missing;
  for (Req* r : batch) {
    r->status = RP_OK;
    if (r->key.first == 0) continue;
    if (needed.emplace(r->key, int(needed.size())).second && !resident.count(r->key)) missing.push_back(r->key);
  }
  // mark use (most recent last)
  for (auto& kv : needed) {
    auto it = resident.find(kv.first);
    if (it != resident.end()) lru.splice(lru.end(), lru, it->second);
  }
  // Requests on graphs that are already resident (or on the base) run before
  // this round's tuning launch and complete at once: a search never waits for
  // a prune of the whole base that other requests of the round asked for.
  std::vector<Req*> rest;
  if (!missing.empty()) {
    std::vector<Req*> early;
    for (Req* r : batch) {
      const bool ready = r->key.first == 0 || resident.count(r->key);
      (ready ? early : rest).push_back(r);
    }
    if (!early.empty()) {
      run_searches(early);
      publish(early);
    }
  } else {
    rest = batch;
  }
  std::map<Key, rp_status> failed;
  evict_for(missing.size(), needed);
  const size_t chunk = cfg.serial ? 1 : size_t(kMaxTargets);
  for (size_t lo = 0; lo < missing.size(); lo += chunk) {
    const size_t T = std::min(chunk, missing.size() - lo);
    double alphas[kMaxTargets];
    int32_t Rs[kMaxTargets];
    rp_graph outs[kMaxTargets] = {};
    for (size_t t = 0; t < T; ++t) {
      alphas[t] = missing[lo + t].first / 1000.0;
      Rs[t] = missing[lo + t].second;
    }
    const rp_status s = ex.tune_batch(ex.user, cfg.base, alphas, Rs, int32_t(T), outs);
    {
      std::lock_guard<std::mutex> lk(mu);
      stats.tune_launches += 1;
      if (s == RP_OK) stats.targets_tuned += int64_t(T);
    }
    for (size_t t = 0; t < T; ++t) {
      const Key& key = missing[lo + t];
      if (s != RP_OK) {
        failed[key] = s;
        continue;
      }
      lru.emplace_back(key, outs[t]);
      resident[key] = std::prev(lru.end());
    }
    if (s != RP_OK) set_error("tuning %zu target(s) from the base failed with status %d", T, s);
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    stats.resident_graphs = int64_t(lru.size());
    stats.peak_resident_graphs = std::max(stats.peak_resident_graphs, stats.resident_graphs);
  }
  for (Req* r : rest) {
    auto f = failed.find(r->key);
    if (f != failed.end()) {
      r->status = f->second;
      r->graph = 0;
    }
  }
  run_searches(rest);
  {
    // counted before the last requests complete, so that a caller who has seen
    // them complete also sees the round in the statistics
    std::lock_guard<std::mutex> lk(mu);
    stats.rounds += 1;
    stats.busy_ns += now_ns(t0) - t_start;
  }
  publish(rest);
}

// One step of the scheduler with an asynchronous executor: take in the tuning
// job that finished, admit the new batch, run every request whose graph is
// resident, and start the next tuning job for the parked requests.
void rp_server::round_async(std::vector<Req*>& batch, int32_t* round_no) {
  const int64_t t_start = now_ns(t0);
  bool worked = false;
  std::map<Key, rp_status> failed;
  if (inflight.active) {
    const rp_status st = ex.tune_ready(ex.user, inflight.ticket, 0);
    if (st != RP_ETIMEOUT) {
      worked = true;
      for (size_t t = 0; t < inflight.keys.size(); ++t) {
        if (st == RP_OK) {
          lru.emplace_back(inflight.keys[t], inflight.outs[t]);
          resident[inflight.keys[t]] = std::prev(lru.end());
        } else {
          failed[inflight.keys[t]] = st;
          ex.graph_free(ex.user, inflight.outs[t]);
        }
      }
      if (st != RP_OK) set_error("tuning %zu target(s) from the base failed with status %d", inflight.keys.size(), st);
      std::lock_guard<std::mutex> lk(mu);
      if (st == RP_OK) stats.targets_tuned += int64_t(inflight.keys.size());
      stats.resident_graphs = int64_t(lru.size());
      stats.peak_resident_graphs = std::max(stats.peak_resident_graphs, stats.resident_graphs);
      inflight = Inflight{};
    }
  }
  if (!batch.empty()) {
    worked = true;
    ++*round_no;
    std::lock_guard<std::mutex> lk(mu);
    for (Req* r : batch) {
      r->status = RP_OK;
      r->info.state = RP_REQ_RUNNING;
      r->info.start_ns = t_start;
      r->info.round = *round_no;
    }
  }
  // mark use (most recent last) and split: ready now, or parked
  for (Req* r : batch) {
    auto it = resident.find(r->key);
    if (it != resident.end()) lru.splice(lru.end(), lru, it->second);
    parked.push_back(r);
  }
  std::vector<Req*> ready, still;
  for (Req* r : parked) {
    auto f = failed.find(r->key);
    if (f != failed.end()) {
      r->status = f->second;
      r->graph = 0;
      ready.push_back(r);
    } else if (r->key.first == 0 || resident.count(r->key)) {
      ready.push_back(r);
    } else {
      still.push_back(r);
    }
  }
  parked.swap(still);
  if (!ready.empty()) {
    run_searches(ready);
    publish(ready);
  }
  // the next tuning job: the graphs the parked requests need, in order of first use
  if (!inflight.active && !parked.empty()) {
    worked = true;
    std::map<Key, int> needed;
    std::vector<Key> missing;
    // at most what the budget holds (evict_for can free every resident graph:
    // no parked request uses one)
    const size_t cap = size_t(std::min<int64_t>(kMaxTargets, capacity));
    for (Req* r : parked)
      if (needed.emplace(r->key, int(needed.size())).second && missing.size() < cap) missing.push_back(r->key);
    evict_for(missing.size(), needed);
    double alphas[kMaxTargets];
    int32_t Rs[kMaxTargets];
    rp_graph outs[kMaxTargets] = {};
    for (size_t t = 0; t < missing.size(); ++t) {
      alphas[t] = missing[t].first / 1000.0;
      Rs[t] = missing[t].second;
    }
    int64_t ticket = 0;
    const rp_status st = ex.tune_start(ex.user, cfg.base, alphas, Rs, int32_t(missing.size()), outs, &ticket);
    {
      std::lock_guard<std::mutex> lk(mu);
      stats.tune_launches += 1;
    }
    if (st == RP_OK) {
      inflight.active = true;
      inflight.ticket = ticket;
      inflight.keys = missing;
      inflight.outs.assign(outs, outs + missing.size());
    } else {
      set_error("starting to tune %zu target(s) from the base failed with status %d", missing.size(), st);
      std::vector<Req*> bad, keep;
      std::map<Key, int> mk;
      for (const Key& k : missing) mk[k] = 0;
      for (Req* r : parked) (mk.count(r->key) ? bad : keep).push_back(r);
      for (Req* r : bad) {
        r->status = st;
        r->graph = 0;
      }
      parked.swap(keep);
      publish(bad);
    }
  }
  if (worked) {
    std::lock_guard<std::mutex> lk(mu);
    if (!batch.empty()) stats.rounds += 1;
    stats.busy_ns += now_ns(t0) - t_start;
  }
}

void rp_server::run() {
  int32_t round_no = 0;
  const bool async = ex.tune_start && ex.tune_ready && !cfg.serial;
  for (;;) {
    std::vector<Req*> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (async && (inflight.active || !parked.empty())) {
        // a tuning job runs: look at it again soon even if nothing arrives
        cv_work.wait_for(lk, std::chrono::microseconds(200), [&] { return !queue.empty(); });
      } else {
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        if (queue.empty()) break;  // stopping and drained
      }
      // admission in arrival order
      std::map<Key, int> keys;
      int64_t qsum = 0;
      while (!queue.empty()) {
        Req* r = queue.front();
        if (!batch.empty()) {
          if (cfg.serial) break;
          const bool new_key = r->key.first != 0 && !keys.count(r->key);
          if (new_key && int64_t(keys.size()) + 1 > capacity) break;
          if (r->nq > 0 && qsum + r->nq > cfg.max_batch_queries) break;
        }
        if (r->key.first != 0) keys.emplace(r->key, 0);
        qsum += r->nq;
        batch.push_back(r);
        queue.pop_front();
      }
    }
    if (async) {
      round_async(batch, &round_no);
    } else {
      round(batch, ++round_no);
    }
  }
}

namespace {

rp_status start_server(rp_server* s, rp_server** out) {
  s->t0 = std::chrono::steady_clock::now();
  const size_t esz = s->cfg.dtype == RP_U8 ? 1 : 4;
  s->row_bytes = size_t(s->cfg.d) * esz;
  if (s->cfg.max_batch_queries <= 0) s->cfg.max_batch_queries = kDefaultBatch;
  s->capacity = INT64_MAX;
  if (s->cfg.graph_budget_bytes > 0)
    s->capacity = std::max<int64_t>(1, int64_t(s->cfg.graph_budget_bytes / std::max<uint64_t>(s->cfg.graph_bytes, 1)));
  try {
    s->worker = std::thread([s] { s->run(); });
  } catch (...) {
    delete s;
    return RP_ENOMEM;
  }
  *out = s;
  return RP_OK;
}

rp_status submit(rp_server* s, Req* r, int64_t* request_id) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return RP_EINVAL;
  }
  r->id = s->next_id++;
  r->info.state = RP_REQ_QUEUED;
  r->info.L_eff = r->L_eff;
  r->info.submit_ns = now_ns(s->t0);
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  *request_id = r->id;
  s->cv_work.notify_one();
  return RP_OK;
}

}  // namespace

extern "C" {

rp_status rp_server_create_ex(const rp_executor* ex, const rp_server_config* cfg, rp_server** out) {
  if (!out) return RP_EINVAL;
  *out = nullptr;
  if (!ex || !cfg || !ex->tune_batch || !ex->search_multi || !ex->graph_free) return RP_EINVAL;
  if (cfg->d < 1 || (cfg->dtype != RP_U8 && cfg->dtype != RP_F32) || cfg->max_batch_queries < 0) return RP_EINVAL;
  rp_server* s = new (std::nothrow) rp_server();
  if (!s) return RP_ENOMEM;
  s->ex = *ex;
  s->cfg = *cfg;
  return start_server(s, out);
}

rp_status rp_server_create(rp_ctx* ctx, rp_graph base, uint64_t graph_budget_bytes, int64_t max_batch_queries,
                           int32_t serial, rp_server** out) {
  if (!out || !ctx || max_batch_queries < 0) return RP_EINVAL;
  *out = nullptr;
  rp_server_config cfg{};
  cfg.base = base;
  rp_status st = rp_graph_shape(ctx, base, &cfg.d, &cfg.dtype, &cfg.graph_bytes);
  if (st != RP_OK) return st;
  cfg.graph_budget_bytes = graph_budget_bytes;
  cfg.max_batch_queries = max_batch_queries;
  cfg.serial = serial ? 1 : 0;
  rp_server* s = new (std::nothrow) rp_server();
  if (!s) return RP_ENOMEM;
  s->ctx_exec.ctx = ctx;
  s->ex.user = &s->ctx_exec;
  s->ex.tune_batch = ctx_tune;
  s->ex.search_multi = ctx_search;
  s->ex.graph_free = ctx_free;
  s->ex.tune_start = ctx_tune_start;
  s->ex.tune_ready = ctx_tune_ready;
  s->cfg = cfg;
  return start_server(s, out);
}

rp_status rp_server_destroy(rp_server* s) {
  if (!s) return RP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  rp_status st = RP_OK;
  for (auto& e : s->lru) {
    const rp_status f = s->ex.graph_free(s->ex.user, e.second);
    if (f != RP_OK) st = f;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return st;
}

rp_status rp_submit_tune(rp_server* s, double alpha, int32_t R, int64_t* request_id) {
  if (!s || !request_id) return RP_EINVAL;
  int32_t A = 0;
  if (!alpha_key(alpha, &A) || A == 0 || R < 1) {
    s->set_error("rp_submit_tune: need alpha >= 1 on the 0.001 grid and R >= 1 (alpha=%g R=%d)", alpha, R);
    return RP_EINVAL;
  }
  Req* r = new (std::nothrow) Req();
  if (!r) return RP_ENOMEM;
  r->key = Key(A, R);
  return submit(s, r, request_id);
}

rp_status rp_submit_search(rp_server* s, double alpha, int32_t R, const void* queries, int64_t nq, int32_t L,
                           int32_t k, int32_t* ids, float* dists, int64_t* request_id) {
  if (!s || !request_id) return RP_EINVAL;
  int32_t A = 0;
  if (!alpha_key(alpha, &A) || (A != 0 && R < 1) || nq < 1 || k < 1 || k > RP_MAX_L || L > RP_MAX_L || !queries ||
      !ids) {
    s->set_error("rp_submit_search: bad argument (alpha=%g R=%d nq=%lld L=%d k=%d)", alpha, R, (long long)nq, L, k);
    return RP_EINVAL;
  }
  Req* r = new (std::nothrow) Req();
  if (!r) return RP_ENOMEM;
  r->search = true;
  r->key = A == 0 ? Key(0, 0) : Key(A, R);
  r->nq = nq;
  r->k = k;
  r->L_eff = std::max(L, k);
  r->ids = ids;
  r->dists = dists;
  try {
    r->q.assign(static_cast<const uint8_t*>(queries), static_cast<const uint8_t*>(queries) + size_t(nq) * s->row_bytes);
  } catch (...) {
    delete r;
    return RP_ENOMEM;
  }
  if (L < k) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.l_clamps += 1;
  }
  return submit(s, r, request_id);
}

rp_status rp_poll(rp_server* s, int64_t id, int32_t timeout_ms, rp_request_info* info) {
  if (!s || timeout_ms < 0) return RP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return RP_ENOTFOUND;
  Req* r = it->second;
  s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->info.state == RP_REQ_DONE; });
  if (info) *info = r->info;
  if (r->info.state != RP_REQ_DONE) return RP_ETIMEOUT;
  s->reqs.erase(it);
  delete r;
  return RP_OK;
}

rp_status rp_server_stats(rp_server* s, rp_server_stats_t* out) {
  if (!s || !out) return RP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return RP_OK;
}

const char* rp_server_last_error(rp_server* s) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  return s->err.c_str();
}

}  // extern "C"
