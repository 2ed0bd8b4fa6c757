// Request loop with continuous batching: clients submit (graph, parameters)
// requests; worker threads, each with its own CUDA stream, repeatedly take the
// oldest pending request plus the compatible ones behind it (same attribute
// layout and the same batch-wide parameters) up to the batch limits and the
// free part of the HBM budget, upload them as one stacked batch, solve it with
// abg_batch_cluster and hand each request its labels. Several batches are in
// flight at once (one per worker), so requests that arrive while others run
// are admitted as soon as a worker and memory free up, and their work overlaps
// on the device. A request whose estimated footprint exceeds the budget is
// rejected at submission.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace {

using clock_t_ = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  abg_graph_desc desc{};
  abg_params params{};
  int64_t bytes = 0;
  int status = ABG_PENDING;
  std::vector<int32_t> labels;
  abg_result result{};
  std::string error;  // message of a failed batch, handed to the poller
  abg::SideSwap swap; // storage behind desc when the request clusters V
  abg_graph* resident = nullptr;  // solve this caller-owned graph (no upload, runs alone)
  int64_t rows = 0;                // clustered nodes (labels)
  clock_t_::time_point t_submit, t_done;
};

// device bytes of one request: its graph (both edge orders, values, scales,
// attributes, schedules) plus one solve's workspaces
int64_t estimate_bytes(const abg_graph_desc& d, const abg_params& p) {
  const int64_t n = d.n_u, nv = d.n_v, nnz = d.nnz;
  const int dd = p.d == 0 ? d.d_u : p.d;
  int64_t g = nnz * 16 + (n + nv) * 32;
  if (d.x_kind == ABG_X_CSR_F32)
    g += (d.x_ptr ? d.x_ptr[d.n_u] : 0) * 20 + (int64_t)d.d_u * 16;
  else
    g += n * abg::round_up(d.d_u, 8) * (d.x_kind == ABG_X_DENSE_F32 ? 4 : 2);
  const int64_t ld = abg::round_up(dd, 4), ldr = abg::round_up(2 * dd, 4);
  const int64_t kk = abg::round_up(p.k, 4);
  const int64_t ll = abg::round_up(std::min(p.k + p.oversample, 2 * dd), 4);
  int64_t s = 4 * n * ld + 4 * nv * ld + 4 * n * ldr + 8 * n * ll + 16 * n * kk + 16 * n;
  s += 4 * (abg::ceil_div(n, 2048) + 1) * std::max<int64_t>(2 * dd, 128) * std::max(kk, ll);
  if (dd < d.d_u) s += 4 * n * (ld + 2 * abg::round_up(dd + p.oversample, 4));
  else if (d.x_kind == ABG_X_CSR_F32) s += 4 * n * ld;
  return g + s + (8 << 20);
}

bool compatible(const Job& a, const Job& b) {
  if (a.resident || b.resident) return false;  // a resident graph is solved on its own
  const abg_params &p = a.params, &q = b.params;
  return a.desc.d_u == b.desc.d_u && a.desc.x_kind == b.desc.x_kind && p.d == q.d &&
         p.alpha == q.alpha && p.gamma == q.gamma && p.t_f == q.t_f && p.t_g == q.t_g &&
         p.oversample == q.oversample && p.power_iters == q.power_iters &&
         p.nci_flags == q.nci_flags && p.precision == q.precision;
}

}  // namespace

struct abg_server {
  abg_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::map<uint64_t, Job*> jobs;
  uint64_t next_id = 1;
  int64_t inflight_bytes = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  abg_server_stats stats{};
};

namespace {

void worker_main(abg_server* sv, int wid) {
  cudaSetDevice(sv->opts.device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Job*> batch;
    int64_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop) break;
        if (!sv->pending.empty()) {
          Job* head = sv->pending.front();
          if (sv->inflight_bytes + head->bytes <= sv->opts.hbm_budget_bytes) break;
        }
        sv->cv_work.wait(lk);
      }
      if (sv->stop) break;
      // optionally wait a little for the batch to fill
      if (sv->opts.batch_window_us > 0 && (int)sv->pending.size() < sv->opts.max_batch_graphs) {
        const auto until = sv->pending.front()->t_submit +
                           std::chrono::microseconds(sv->opts.batch_window_us);
        sv->cv_work.wait_until(lk, until, [&] {
          return sv->stop || (int)sv->pending.size() >= sv->opts.max_batch_graphs;
        });
        if (sv->stop) break;
        if (sv->pending.empty()) continue;
      }
      // oldest request first, then compatible ones in arrival order within the limits
      Job* head = sv->pending.front();
      if (sv->inflight_bytes + head->bytes > sv->opts.hbm_budget_bytes) continue;
      int64_t rows = 0;
      for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        Job* j = *it;
        const bool fits = (int)batch.size() < sv->opts.max_batch_graphs &&
                          (batch.empty() || rows + j->rows <= sv->opts.max_batch_rows) &&
                          sv->inflight_bytes + bytes + j->bytes <= sv->opts.hbm_budget_bytes;
        if ((batch.empty() || compatible(*batch.front(), *j)) && fits) {
          batch.push_back(j);
          bytes += j->bytes;
          rows += j->rows;
          it = sv->pending.erase(it);
          if (j->resident) break;
        } else {
          ++it;
        }
      }
      sv->inflight_bytes += bytes;
      sv->stats.batches += 1;
      sv->stats.inflight_bytes = sv->inflight_bytes;
      sv->stats.max_batch = std::max<int64_t>(sv->stats.max_batch, (int64_t)batch.size());
    }
    // ---- run the batch (outside the lock) ----
    std::vector<abg_graph_desc> descs;
    std::vector<abg_params> params;
    int64_t rows = 0;
    for (Job* j : batch) {
      descs.push_back(j->desc);
      params.push_back(j->params);
      rows += j->rows;
    }
    abg_graph* g = nullptr;
    std::vector<int32_t> labels(rows);
    std::vector<abg_result> res(batch.size());
    int st;
    if (batch.front()->resident) {  // one request on a caller-owned resident graph
      st = abg_cluster(batch.front()->resident, &params[0], stream, labels.data(), res.data());
    } else {
      st = abg_batch_create(descs.data(), (int32_t)descs.size(), sv->opts.device, stream, &g);
      if (st == ABG_OK)
        st = abg_batch_cluster(g, params.data(), stream, labels.data(), res.data());
    }
    const std::string err = st == ABG_OK ? std::string() : std::string(abg_last_error());
    if (g) abg_destroy(g);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      int64_t off = 0;
      const auto now = clock_t_::now();
      for (size_t i = 0; i < batch.size(); ++i) {
        Job* j = batch[i];
        if (st == ABG_OK) {
          j->labels.assign(labels.begin() + off, labels.begin() + off + j->rows);
          j->result = res[i];
        } else {
          j->error = err;
        }
        off += j->rows;
        j->status = st;
        j->t_done = now;
        if (st == ABG_OK) sv->stats.completed += 1; else sv->stats.failed += 1;
        if (st == ABG_OK && res[i].reused_propagation) sv->stats.propagations_reused += 1;
      }
      sv->inflight_bytes -= bytes;
      sv->stats.inflight_bytes = sv->inflight_bytes;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
  cudaStreamDestroy(stream);
  (void)wid;
}

}  // namespace

extern "C" {

ABG_API void abg_server_opts_default(abg_server_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->device = 0;
  o->hbm_budget_bytes = int64_t(64) << 30;
  o->max_batch_graphs = 64;
  o->max_batch_rows = int64_t(4) << 20;
  o->workers = 3;
  o->batch_window_us = 0;
}

ABG_API int abg_server_create(const abg_server_opts* opts, abg_server** out) {
  using namespace abg;
  ABG_CHECK(out, "null output pointer");
  *out = nullptr;
  abg_server* sv = new abg_server();
  if (opts) sv->opts = *opts; else abg_server_opts_default(&sv->opts);
  if (sv->opts.workers < 1 || sv->opts.max_batch_graphs < 1 || sv->opts.hbm_budget_bytes <= 0 ||
      sv->opts.max_batch_rows < 1) {
    delete sv;
    set_error("server options: workers, max_batch_graphs, max_batch_rows, budget must be > 0");
    return ABG_EINVAL;
  }
  for (int i = 0; i < sv->opts.workers; ++i) sv->workers.emplace_back(worker_main, sv, i);
  *out = sv;
  return ABG_OK;
}

ABG_API void abg_server_destroy(abg_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (Job* j : sv->pending) j->status = ABG_ECANCELLED;
    sv->pending.clear();
  }
  sv->cv_work.notify_all();
  sv->cv_done.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->jobs) delete kv.second;
  delete sv;
}

ABG_API int abg_submit(abg_server* sv, const abg_graph_desc* graph, const abg_params* params,
                       uint64_t* req_id) {
  using namespace abg;
  ABG_CHECK(sv && graph && params && req_id, "null argument");
  Job* j = new Job();
  const abg_graph_desc* gd = nullptr;
  int st = swap_sides(graph, &j->swap, &gd);
  if (st == ABG_OK) st = validate_desc(gd);
  if (st == ABG_OK && !(params->k >= 1 && params->k <= kMaxK && params->k <= gd->n_u)) {
    set_error("need 1 <= k <= min(|U|, %d)", kMaxK);
    st = ABG_EINVAL;
  }
  if (st != ABG_OK) {
    delete j;
    return st;
  }
  j->desc = *gd;
  j->rows = gd->n_u;
  const abg_graph_desc* graph_eff = &j->desc;
  j->params = *params;
  j->bytes = estimate_bytes(*graph_eff, *params);
  j->t_submit = clock_t_::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
      delete j;
      set_error("server is shutting down");
      return ABG_ECANCELLED;
    }
    j->id = sv->next_id++;
    *req_id = j->id;
    sv->stats.submitted += 1;
    if (j->bytes > sv->opts.hbm_budget_bytes) {
      j->status = ABG_ENOTADMITTED;
      sv->stats.rejected += 1;
      sv->jobs[j->id] = j;
      set_error("request needs ~%lld bytes, budget is %lld", (long long)j->bytes,
                (long long)sv->opts.hbm_budget_bytes);
      return ABG_ENOTADMITTED;
    }
    sv->jobs[j->id] = j;
    sv->pending.push_back(j);
  }
  sv->cv_work.notify_one();
  return ABG_OK;
}

ABG_API int abg_submit_resident(abg_server* sv, abg_graph* g, const abg_params* params,
                                uint64_t* req_id) {
  using namespace abg;
  ABG_CHECK(sv && g && params && req_id, "null argument");
  ABG_CHECK(g->nseg == 1, "a resident request needs a graph from abg_create, not a batch");
  ABG_CHECK(g->device == sv->opts.device, "the graph lives on device %d, the server on %d",
            g->device, sv->opts.device);
  int d = 0;
  ABG_TRY(check_params(g, params, g->n_u, &d));
  Job* j = new Job();
  j->resident = g;
  j->params = *params;
  j->rows = g->n_u;
  j->bytes = abg_solve_footprint(g, params);
  j->t_submit = clock_t_::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
      delete j;
      set_error("server is shutting down");
      return ABG_ECANCELLED;
    }
    j->id = sv->next_id++;
    *req_id = j->id;
    sv->stats.submitted += 1;
    if (j->bytes > sv->opts.hbm_budget_bytes) {
      j->status = ABG_ENOTADMITTED;
      sv->stats.rejected += 1;
      sv->jobs[j->id] = j;
      set_error("request needs ~%lld bytes, budget is %lld", (long long)j->bytes,
                (long long)sv->opts.hbm_budget_bytes);
      return ABG_ENOTADMITTED;
    }
    sv->jobs[j->id] = j;
    sv->pending.push_back(j);
  }
  sv->cv_work.notify_one();
  return ABG_OK;
}

ABG_API int abg_poll(abg_server* sv, uint64_t req_id, int64_t timeout_us, int32_t* labels,
                     abg_result* res) {
  using namespace abg;
  ABG_CHECK(sv, "null server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(req_id);
  if (it == sv->jobs.end()) {
    set_error("unknown request %llu", (unsigned long long)req_id);
    return ABG_ENOTFOUND;
  }
  Job* j = it->second;
  if (j->status == ABG_PENDING && timeout_us != 0) {
    auto done = [&] { return j->status != ABG_PENDING; };
    if (timeout_us < 0)
      sv->cv_done.wait(lk, done);
    else
      sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  }
  if (j->status == ABG_PENDING) return timeout_us == 0 ? ABG_PENDING : ABG_ETIMEDOUT;
  const int st = j->status;
  const std::string err = j->error;
  if (st == ABG_OK) {
    if (labels) memcpy(labels, j->labels.data(), sizeof(int32_t) * j->labels.size());
    if (res) *res = j->result;
  }
  sv->stats.latency_us_last =
      std::chrono::duration_cast<std::chrono::microseconds>(j->t_done - j->t_submit).count();
  sv->jobs.erase(it);
  delete j;
  if (st != ABG_OK && st != ABG_ENOTADMITTED)
    set_error("request failed: %s (%s)", abg_strerror(st), err.c_str());
  return st;
}

ABG_API int abg_server_get_stats(abg_server* sv, abg_server_stats* out) {
  using namespace abg;
  ABG_CHECK(sv && out, "null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  out->pending = (int64_t)sv->pending.size();
  return ABG_OK;
}

}  // extern "C"
