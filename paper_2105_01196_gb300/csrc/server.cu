// Job server: continuous batching of independent EBIC runs on one GPU.
//
// Jobs (a matrix, parameters and a generation count) are queued as they arrive.  A scheduler
// thread admits queued jobs in arrival order, letting a later job that fits go ahead of a head
// job that does not (backfill), while the sum of the admitted jobs' device-memory footprints stays
// within the budget and at most `max_running` jobs run.  Each admitted job runs on a worker thread;
// a worker keeps one context (and stream) for all its jobs, so the kernels of different jobs
// overlap on the device and no job pays for creating or destroying a context.  A job's matrix,
// bitmap and population stay resident until it ends; finishing a job returns those buffers to
// the library's memory pool (stream-ordered, no device-wide synchronisation) and admits the
// next ones.  A worker whose job failed replaces its context.  A job's results do not depend on the other jobs: each context's
// computation is deterministic and shares nothing with the others.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// The evaluation form a job will use: the cost model of ebic_eval_population's AUTO mode.
int job_mode(int64_t rows, int32_t cols, const ebic_params &p, int32_t n_gen) {
  if (p.mode != EBIC_MODE_AUTO) return p.mode;
  if (p.last_kept) return EBIC_MODE_DIRECT;  // no bitmap form
  const double mean_len = 0.5 * (p.init_min_len + p.max_len);
  return cost_model_prefers_bitmap((double)round_up(rows, 128), (double)cols,
                                   code_bytes_for(cols), (double)p.pop_size, mean_len,
                                   (double)n_gen + 1.0)
             ? EBIC_MODE_BITMAP
             : EBIC_MODE_DIRECT;
}

struct Job {
  int64_t id = 0;
  std::vector<float> x;
  int64_t rows = 0;
  int32_t cols = 0, layout = 0, n_gen = 0, mode = 0;
  ebic_params p{};
  int64_t footprint = 0;
  Clock::time_point t_submit, t_start, t_end;
  bool done = false;
  int32_t status = EBIC_OK;
  ebic_run_report rep{};
  std::vector<int32_t> top_cols, top_lens, top_rows;
  std::vector<uint64_t> top_fit, top_keys;
  int32_t n_top = 0;
};

}  // namespace

struct ebic_server {
  int device = 0;
  int64_t budget = 0, reserved = 0;
  int max_running = 1, running = 0;
  int64_t next_id = 1;
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv_sched, cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queued, admitted;
  std::map<int64_t, std::shared_ptr<Job>> jobs;
  std::thread scheduler;
  std::vector<std::thread> workers;
};

namespace {

void schedule_loop(ebic_server *srv) {
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    srv->cv_sched.wait(lk, [&] { return srv->stopping || !srv->queued.empty(); });
    if (srv->stopping) return;
    bool admitted_any = false;
    for (auto it = srv->queued.begin(); it != srv->queued.end();) {
      if (srv->running >= srv->max_running) break;
      const std::shared_ptr<Job> &j = *it;
      if (srv->reserved + j->footprint <= srv->budget) {
        srv->reserved += j->footprint;
        srv->running += 1;
        srv->admitted.push_back(j);
        it = srv->queued.erase(it);
        admitted_any = true;
      } else {
        ++it;
      }
    }
    if (admitted_any) srv->cv_work.notify_all();
    // nothing more fits: wait for a job to finish (or a new one to arrive)
    srv->cv_sched.wait(lk);
  }
}

// Runs job j on the worker's context *pctx (created when null; destroyed and set to null when
// the job fails, so that the next job starts from a fresh context).
void run_job(ebic_server *srv, Job &j, ebic_ctx **pctx) {
  int st = *pctx ? EBIC_OK : ebic_create(pctx, srv->device, nullptr);
  ebic_ctx *ctx = *pctx;
  if (st == EBIC_OK) st = ebic_load_matrix(ctx, j.x.data(), j.rows, j.cols, j.layout);
  ebic_params p = j.p;
  p.mode = j.mode;
  if (st == EBIC_OK) st = ebic_run_generations(ctx, &p, j.n_gen, &j.rep);
  if (st == EBIC_OK) {
    const int K = p.n_biclusters;
    j.top_cols.assign((size_t)K * EBIC_MAX_LEN, 0);
    j.top_lens.assign(K, 0);
    j.top_rows.assign((size_t)K * 3, 0);
    j.top_fit.assign(K, 0);
    j.top_keys.assign(K, 0);
    st = ebic_get_toplist(ctx, K, &j.n_top, j.top_cols.data(), j.top_lens.data(),
                          j.top_fit.data(), j.top_keys.data(), j.top_rows.data());
  }
  if (ctx && st == EBIC_OK) {
    ctx_release_buffers(ctx);
  } else if (ctx) {
    ebic_destroy(ctx);
    *pctx = nullptr;
  }
  j.status = st;
  std::vector<float>().swap(j.x);  // the matrix is no longer needed
}

void worker_loop(ebic_server *srv) {
  ebic_ctx *ctx = nullptr;  // the worker's context, kept across its jobs
  struct Owner {
    ebic_ctx **c;
    ~Owner() {
      if (*c) ebic_destroy(*c);
    }
  } owner{&ctx};
  for (;;) {
    std::shared_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv_work.wait(lk, [&] { return srv->stopping || !srv->admitted.empty(); });
      if (srv->admitted.empty()) return;  // stopping
      j = srv->admitted.front();
      srv->admitted.pop_front();
      j->t_start = Clock::now();
    }
    run_job(srv, *j, &ctx);
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      j->t_end = Clock::now();
      j->done = true;
      srv->reserved -= j->footprint;
      srv->running -= 1;
    }
    srv->cv_done.notify_all();
    srv->cv_sched.notify_all();
  }
}

}  // namespace

extern "C" {

int64_t ebic_job_footprint(int64_t rows, int32_t cols, const ebic_params *p, int32_t n_gen) {
  if (!p || rows < 1 || cols < 2 || n_gen < 0) return -1;
  const int64_t R_pad = round_up(rows, 128);
  const int64_t P = p->pop_size;
  int64_t bytes = (int64_t)cols * R_pad * 4;              // order keys
  bytes += rows * (int64_t)cols * 4;                      // staged host matrix
  if (job_mode(rows, cols, *p, n_gen) == EBIC_MODE_BITMAP)
    bytes += ebic_bitmap_bytes(rows, cols);               // pair bitmap
  const int w = code_bytes_for(cols);
  if (w)  // rank codes and their bit planes (both forms build them)
    bytes += (int64_t)cols * code_stride_for(rows, w) * w +
             (int64_t)cols * code_plane_stride(code_plane_bits(cols)) * (R_pad / 32) * 4;
  bytes += 2 * P * (EBIC_MAX_LEN * 4 + 4 + 4 + 12 + 1 + 1 + 8 + 8);  // population buffers
  bytes += P * 12 + 64;                                   // evaluation scratch
  bytes += (int64_t)tabu_capacity(P * ((int64_t)n_gen + 2)) * 8;  // tabu list
  bytes += 2 * (int64_t)dedup_capacity(P) * 12;                   // duplicate tables
  bytes += (int64_t)pow2_at_least((uint64_t)P) * 20;              // top-list candidates
  bytes += (int64_t)p->n_biclusters * 288 + (int64_t)cols * 4 + 4096;
  return bytes + bytes / 16;                               // allocator slack
}

int ebic_server_create(ebic_server **out, int32_t device, int64_t hbm_budget_bytes,
                       int32_t max_running) {
  if (!out || hbm_budget_bytes <= 0 || max_running < 1 || max_running > 64) return EBIC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return EBIC_ECUDA;
  }
  if (device < 0 || device >= ndev) return EBIC_EINVAL;
  ebic_server *srv = new (std::nothrow) ebic_server();
  if (!srv) return EBIC_ENOMEM;
  srv->device = device;
  srv->budget = hbm_budget_bytes;
  srv->max_running = max_running;
  try {
    srv->scheduler = std::thread(schedule_loop, srv);
    for (int i = 0; i < max_running; ++i) srv->workers.emplace_back(worker_loop, srv);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->stopping = true;
    }
    srv->cv_sched.notify_all();
    srv->cv_work.notify_all();
    if (srv->scheduler.joinable()) srv->scheduler.join();
    for (auto &w : srv->workers)
      if (w.joinable()) w.join();
    delete srv;
    return EBIC_ENOMEM;
  }
  *out = srv;
  return EBIC_OK;
}

int ebic_server_destroy(ebic_server *srv) {
  if (!srv) return EBIC_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
    srv->queued.clear();  // jobs not yet admitted are dropped; admitted ones finish
  }
  srv->cv_sched.notify_all();
  srv->cv_work.notify_all();
  if (srv->scheduler.joinable()) srv->scheduler.join();
  for (auto &w : srv->workers)
    if (w.joinable()) w.join();
  delete srv;
  return EBIC_OK;
}

int ebic_server_submit(ebic_server *srv, const float *x, int64_t rows, int32_t cols,
                       int32_t layout, const ebic_params *p, int32_t n_gen, int64_t *job_id) {
  if (!srv || !x || !p || !job_id || rows < 1 || cols < 2 || n_gen < 0) return EBIC_EINVAL;
  if (layout != EBIC_LAYOUT_ROW_MAJOR && layout != EBIC_LAYOUT_COL_MAJOR) return EBIC_EINVAL;
  auto j = std::make_shared<Job>();
  try {
    j->x.resize((size_t)rows * cols);
  } catch (...) {
    return EBIC_ENOMEM;
  }
  if (ebic_is_device_ptr(x)) {
    if (cudaMemcpy(j->x.data(), x, (size_t)rows * cols * 4, cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      cudaGetLastError();
      return EBIC_ECUDA;
    }
  } else {
    memcpy(j->x.data(), x, (size_t)rows * cols * 4);
  }
  j->rows = rows;
  j->cols = cols;
  j->layout = layout;
  j->p = *p;
  j->n_gen = n_gen;
  j->mode = job_mode(rows, cols, *p, n_gen);
  j->footprint = ebic_job_footprint(rows, cols, p, n_gen);
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stopping) return EBIC_ESTATE;
  if (j->footprint > srv->budget) return EBIC_ENOMEM;  // could never be admitted
  j->id = srv->next_id++;
  *job_id = j->id;
  srv->jobs[j->id] = j;
  srv->queued.push_back(j);
  srv->cv_sched.notify_all();
  return EBIC_OK;
}

int ebic_server_wait(ebic_server *srv, int64_t job_id, int32_t timeout_ms, ebic_job_result *res,
                     int32_t capacity, int32_t *top_cols, int32_t *top_lens, uint64_t *top_fit,
                     uint64_t *top_keys, int32_t *top_rows) {
  if (!srv || !res) return EBIC_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(job_id);
  if (it == srv->jobs.end()) return EBIC_EINVAL;
  std::shared_ptr<Job> j = it->second;
  auto ready = [&] { return j->done; };
  if (timeout_ms < 0) {
    srv->cv_done.wait(lk, ready);
  } else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return EBIC_ETIMEOUT;
  }
  memset(res, 0, sizeof(*res));
  res->job_id = j->id;
  res->status = j->status;
  res->gens_done = j->rep.gens_done;
  res->stopped = j->rep.stopped;
  res->n_top = j->n_top;
  res->eval_mode = j->mode;
  res->n_evaluated = j->rep.n_evaluated;
  res->footprint_bytes = j->footprint;
  res->queued_ms = std::chrono::duration<double, std::milli>(j->t_start - j->t_submit).count();
  res->run_ms = std::chrono::duration<double, std::milli>(j->t_end - j->t_start).count();
  if (j->status == EBIC_OK && capacity >= j->n_top) {
    const size_t n = (size_t)j->n_top;
    if (top_cols) memcpy(top_cols, j->top_cols.data(), n * EBIC_MAX_LEN * 4);
    if (top_lens) memcpy(top_lens, j->top_lens.data(), n * 4);
    if (top_fit) memcpy(top_fit, j->top_fit.data(), n * 8);
    if (top_keys) memcpy(top_keys, j->top_keys.data(), n * 8);
    if (top_rows) memcpy(top_rows, j->top_rows.data(), n * 12);
  }
  srv->jobs.erase(it);
  return EBIC_OK;
}

int ebic_server_stats(ebic_server *srv, int32_t *queued, int32_t *running, int64_t *reserved) {
  if (!srv) return EBIC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (queued) *queued = (int32_t)srv->queued.size();
  if (running) *running = srv->running;
  if (reserved) *reserved = srv->reserved;
  return EBIC_OK;
}

}  // extern "C"
