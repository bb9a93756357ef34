// Serving loop: continuous batching of independent gravity solves.
//
// Requests join a FIFO queue. Each worker thread owns a plan, a CUDA stream
// and packed device buffers; when free it takes the longest prefix of the
// queue that fits the batch limit and the device-memory budget (the estimated
// footprint of every batch in flight counts against it; the estimate is
// calibrated from the device bytes that completed batches needed), copies the requests'
// particles into its packed buffers, builds one batched tree, solves, and
// copies each request's results back. With two or more workers, a batch that
// arrives while another is on the GPU is admitted as soon as memory allows and
// its work overlaps the other's on the device. A request's results equal its
// solve alone (batched solves reproduce single solves bit for bit).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hpm_internal.cuh"

namespace hpm {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  hpm_request req{};
  Clock::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done, -1 cancelled, -2 failed
  hpm_status status = HPM_OK;
};

struct Worker {
  std::thread th;
  hpm_plan_t plan = nullptr;
  cudaStream_t stream = nullptr;
  DevBuf pos, mass, phi, acc;
};

}  // namespace
}  // namespace hpm

struct hpm_server_s {
  hpm_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<hpm::Request *> queue;
  std::unordered_map<uint64_t, hpm::Request *> reqs;
  std::vector<hpm::Worker *> workers;
  bool stop = false;
  uint64_t next_id = 1;
  int64_t inflight_bytes = 0;
  int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, cancelled = 0, failed = 0;
  int64_t particles_done = 0;
  // latencies of the last kLatencyWindow completions (a ring), and the sum
  // and count of all completions since the last reset
  std::vector<double> latencies_ms;
  size_t lat_next = 0;
  double lat_sum = 0.0;
  int64_t lat_count = 0;
  int waiters = 0;                  // threads inside hpm_server_wait
  std::condition_variable cv_idle;  // signalled when waiters drops to zero while stopping
  hpm::Clock::time_point t_first, t_last;
  bool any_done = false;
  // device bytes per particle that completed batches needed (the largest
  // seen; 0 until the first batch completes)
  double bytes_per_particle = 0.0;
  bool large_running = false;  // a request over the particle bound is on the GPU
};

namespace hpm {
namespace {

// p50 / p99 are taken over this many most recent completions
constexpr size_t kLatencyWindow = 65536;

void record_latency(hpm_server_s *sv, double ms) {
  if (sv->latencies_ms.size() < kLatencyWindow) {
    sv->latencies_ms.push_back(ms);
  } else {
    sv->latencies_ms[sv->lat_next] = ms;
    sv->lat_next = (sv->lat_next + 1) % kLatencyWindow;
  }
  sv->lat_sum += ms;
  ++sv->lat_count;
}

// A request whose final state has been reported to the caller is forgotten.
void release_request(hpm_server_s *sv, Request *r) {
  sv->reqs.erase(r->id);
  delete r;
}

// Device bytes a request of n particles needs while its batch runs: a rate
// per particle times n plus kFixedBytes (per-level tiles of the dense
// source-to-target kernel, counters, scan control: about 2.5 MB at depth 12).
// The rate is the caller's, or else the largest per-particle need beyond
// kFixedBytes measured on a completed batch (its plan's work buffers and the
// worker's packed buffers) with a quarter in reserve for trees denser in
// boxes than those seen so far; before any batch has completed, 512 bytes
// (packed inputs and outputs, keys and permutation double buffered, sorted
// copies, and the boxes, gridlets and locals of about one box per five
// particles).
constexpr int64_t kFixedBytes = 8ll << 20;
int64_t footprint_of(const hpm_server_s *sv, int64_t n) {
  const double rate = sv->opts.bytes_per_particle > 0.0
                          ? sv->opts.bytes_per_particle
                          : (sv->bytes_per_particle > 0.0 ? 1.25 * sv->bytes_per_particle : 512.0);
  return (int64_t)(rate * (double)n) + kFixedBytes;
}

// Takes the next batch from the queue (caller holds the lock), or nothing if
// no request can start now. Requests join in arrival order while they fit
// the batch limit, the particle bound and the device-memory budget. A request
// over the particle bound is large: it runs alone, and only while no other
// large one runs (two on the GPU at once slow each other and everything
// queued behind them); while one runs, the small requests behind a waiting
// large one go ahead of it. A request over the whole memory budget (possible
// after a recalibration) runs alone when nothing else is in flight.
bool take_batch(hpm_server_s *sv, std::vector<Request *> &batch, int64_t &bytes, bool &large) {
  const int64_t bound = sv->opts.max_batch_particles;
  int64_t batch_n = 0;
  bytes = 0;
  large = false;
  for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)batch.size() < sv->opts.max_batch;) {
    Request *r = *it;
    if (r->state == -1) {
      it = sv->queue.erase(it);
      continue;
    }
    const int64_t fp = footprint_of(sv, r->req.n);
    const bool fits_mem = sv->inflight_bytes + bytes + fp <= sv->opts.hbm_budget_bytes ||
                          (batch.empty() && sv->inflight_bytes == 0);
    if (bound > 0 && r->req.n > bound) {
      if (batch.empty() && !sv->large_running && fits_mem) {
        it = sv->queue.erase(it);
        r->state = 1;
        bytes = fp;
        batch.push_back(r);
        large = true;
        break;
      }
      if (!sv->large_running) break;  // it waits at the front for a free worker or memory
      ++it;  // a large one runs: the small ones behind this one may go
      continue;
    }
    if ((bound > 0 && !batch.empty() && batch_n + r->req.n > bound) || !fits_mem) break;
    it = sv->queue.erase(it);
    r->state = 1;
    bytes += fp;
    batch_n += r->req.n;
    batch.push_back(r);
  }
  return !batch.empty();
}

void worker_loop(hpm_server_s *sv, Worker *w) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Request *> batch;
    int64_t bytes = 0;
    bool large = false;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop) return;
        if (take_batch(sv, batch, bytes, large)) break;
        sv->cv_work.wait(lk);
      }
      sv->inflight_bytes += bytes;
      if (large) sv->large_running = true;
      ++sv->batches;
    }
    // run the batch
    std::vector<int64_t> off(batch.size() + 1, 0);
    for (size_t k = 0; k < batch.size(); ++k) off[k + 1] = off[k] + batch[k]->req.n;
    const int64_t n = off.back();
    hpm_status s = HPM_OK;
    const size_t nn = n > 0 ? (size_t)n : 1;
    w->pos.used = w->mass.used = w->phi.used = w->acc.used = 0;  // this batch's need
    if (s == HPM_OK) s = w->pos.ensure(sizeof(double) * 3 * nn, w->stream);
    if (s == HPM_OK) s = w->mass.ensure(sizeof(double) * nn, w->stream);
    if (s == HPM_OK) s = w->phi.ensure(sizeof(float) * nn, w->stream);
    if (s == HPM_OK) s = w->acc.ensure(sizeof(float) * 3 * nn, w->stream);
    for (size_t k = 0; k < batch.size() && s == HPM_OK; ++k) {
      const hpm_request &q = batch[k]->req;
      if (q.n == 0) continue;
      if (cudaMemcpyAsync(w->pos.as<double>() + 3 * off[k], q.pos, sizeof(double) * 3 * q.n, cudaMemcpyDefault,
                          w->stream) != cudaSuccess ||
          cudaMemcpyAsync(w->mass.as<double>() + off[k], q.mass, sizeof(double) * q.n, cudaMemcpyDefault,
                          w->stream) != cudaSuccess)
        s = HPM_ERR_CUDA;
    }
    if (s == HPM_OK) s = hpm_build_tree_batch(w->plan, w->pos.as<double>(), off.data(), (int)batch.size(), w->stream);
    if (s == HPM_OK)
      s = hpm_solve(w->plan, w->pos.as<double>(), w->mass.as<double>(), w->phi.as<float>(), w->acc.as<float>(),
                    w->stream);
    for (size_t k = 0; k < batch.size() && s == HPM_OK; ++k) {
      const hpm_request &q = batch[k]->req;
      if (q.n == 0) continue;
      if ((q.phi && cudaMemcpyAsync(q.phi, w->phi.as<float>() + off[k], sizeof(float) * q.n, cudaMemcpyDefault,
                                    w->stream) != cudaSuccess) ||
          (q.acc && cudaMemcpyAsync(q.acc, w->acc.as<float>() + 3 * off[k], sizeof(float) * 3 * q.n,
                                    cudaMemcpyDefault, w->stream) != cudaSuccess))
        s = HPM_ERR_CUDA;
    }
    if (cudaStreamSynchronize(w->stream) != cudaSuccess && s == HPM_OK) s = HPM_ERR_CUDA;
    const Clock::time_point now = Clock::now();
    double need_pp = 0.0;
    if (s == HPM_OK && n > 0) {
      int64_t tables = 0, work = 0;
      plan_bytes(w->plan, &tables, &work);
      work += (int64_t)(w->pos.used + w->mass.used + w->phi.used + w->acc.used);
      need_pp = std::max(0.0, (double)(work - kFixedBytes) / (double)n);
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->inflight_bytes -= bytes;
      if (large) sv->large_running = false;
      sv->bytes_per_particle = std::max(sv->bytes_per_particle, need_pp);
      for (Request *r : batch) {
        r->t_done = now;
        r->status = s;
        r->state = s == HPM_OK ? 2 : -2;
        if (s == HPM_OK) {
          ++sv->completed;
          sv->particles_done += r->req.n;
          record_latency(sv, std::chrono::duration<double, std::milli>(now - r->t_submit).count());
          if (!sv->any_done) sv->t_first = r->t_submit;
          sv->any_done = true;
          sv->t_last = now;
        } else {
          ++sv->failed;
        }
      }
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace hpm

using namespace hpm;

extern "C" {

hpm_status hpm_server_create(const hpm_server_opts *opts, hpm_server_t *out) {
  if (!opts || !out) return HPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (opts->workers < 0 || opts->workers > 16 || opts->max_batch < 1 || opts->hbm_budget_bytes <= 0 ||
      !(opts->bytes_per_particle >= 0.0) || opts->max_batch_particles < 0)
    return HPM_ERR_INVALID_ARG;
  hpm_server_s *sv = new (std::nothrow) hpm_server_s();
  if (!sv) return HPM_ERR_OOM;
  sv->opts = *opts;
  cudaGetDevice(&sv->device);
  hpm_plan_opts po{opts->leaf_max, 0};
  for (int k = 0; k < opts->workers; ++k) {
    Worker *w = new Worker();
    hpm_status s = hpm_plan(&opts->dom, opts->max_depth, opts->gridlet_order, &opts->green, &po, &w->plan);
    if (s == HPM_OK && cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) s = HPM_ERR_CUDA;
    if (s != HPM_OK) {
      if (w->plan) hpm_destroy(w->plan);
      delete w;
      for (Worker *o : sv->workers) {
        hpm_destroy(o->plan);
        cudaStreamDestroy(o->stream);
        delete o;
      }
      delete sv;
      return s;
    }
    sv->workers.push_back(w);
  }
  for (Worker *w : sv->workers) w->th = std::thread(worker_loop, sv, w);
  *out = sv;
  return HPM_OK;
}

hpm_status hpm_server_submit(hpm_server_t sv, const hpm_request *req, uint64_t *ticket) {
  if (!sv || !req || !ticket || req->n < 0) return HPM_ERR_INVALID_ARG;
  if (req->n > 0 && (!req->pos || !req->mass)) return HPM_ERR_INVALID_ARG;
  Request *r = new (std::nothrow) Request();
  if (!r) return HPM_ERR_OOM;
  r->req = *req;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (footprint_of(sv, req->n) > sv->opts.hbm_budget_bytes) {
      ++sv->rejected;
      delete r;
      return HPM_ERR_OOM;
    }
    r->id = sv->next_id++;
    r->t_submit = Clock::now();
    sv->reqs[r->id] = r;
    sv->queue.push_back(r);
    ++sv->submitted;
    *ticket = r->id;
  }
  sv->cv_work.notify_one();
  return HPM_OK;
}

hpm_status hpm_server_poll(hpm_server_t sv, uint64_t ticket, int *done, double *latency_ms) {
  if (!sv || !done) return HPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return HPM_ERR_INVALID_ARG;
  Request *r = it->second;
  *done = r->state == 2 ? 1 : (r->state < 0 ? -1 : 0);
  if (latency_ms)
    *latency_ms = r->state == 2 ? std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count() : 0.0;
  const hpm_status s = r->state == -2 ? r->status : HPM_OK;
  if (*done != 0) release_request(sv, r);  // final state reported: the ticket ends here
  return s;
}

hpm_status hpm_server_wait(hpm_server_t sv, uint64_t ticket, int timeout_ms, double *latency_ms) {
  if (!sv) return HPM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return HPM_ERR_INVALID_ARG;
  Request *r = it->second;
  ++sv->waiters;
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                       [sv, r] { return sv->stop || r->state == 2 || r->state < 0; });
  if (--sv->waiters == 0 && sv->stop) sv->cv_idle.notify_all();
  if (sv->stop) return HPM_ERR_BUSY;  // the server is being destroyed
  if (!ok) return HPM_ERR_TIMEOUT;
  if (latency_ms)
    *latency_ms = r->state == 2 ? std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count() : 0.0;
  const hpm_status s = r->state == -1 ? HPM_ERR_INVALID_ARG : (r->state == 2 ? HPM_OK : r->status);
  release_request(sv, r);  // final state reported: the ticket ends here
  return s;
}

hpm_status hpm_server_cancel(hpm_server_t sv, uint64_t ticket) {
  if (!sv) return HPM_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return HPM_ERR_INVALID_ARG;
    Request *r = it->second;
    if (r->state != 0) return HPM_ERR_BUSY;  // already running or finished
    r->state = -1;
    // out of the queue now, so that the request can be freed once its state
    // has been reported
    sv->queue.erase(std::remove(sv->queue.begin(), sv->queue.end(), r), sv->queue.end());
    ++sv->cancelled;
  }
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
  return HPM_OK;
}

hpm_status hpm_server_get_stats(hpm_server_t sv, hpm_server_stats *st) {
  if (!sv || !st) return HPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  memset(st, 0, sizeof(*st));
  st->submitted = sv->submitted;
  st->completed = sv->completed;
  st->rejected = sv->rejected;
  st->cancelled = sv->cancelled;
  st->failed = sv->failed;
  st->batches = sv->batches;
  int64_t queued = 0;
  for (Request *r : sv->queue)
    if (r->state == 0) ++queued;
  st->queued = queued;
  st->in_flight_bytes = sv->inflight_bytes;
  st->bytes_per_particle = sv->bytes_per_particle;
  st->particles = sv->particles_done;
  st->p50_ms = percentile(sv->latencies_ms, 0.50);
  st->p99_ms = percentile(sv->latencies_ms, 0.99);
  st->mean_ms = sv->lat_count ? sv->lat_sum / (double)sv->lat_count : 0.0;
  if (sv->any_done) {
    const double span = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
    st->particles_per_s = span > 0 ? (double)sv->particles_done / span : 0.0;
  }
  return HPM_OK;
}

hpm_status hpm_server_reset_stats(hpm_server_t sv) {
  if (!sv) return HPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->latencies_ms.clear();
  sv->lat_next = 0;
  sv->lat_sum = 0.0;
  sv->lat_count = 0;
  sv->particles_done = 0;
  sv->completed = sv->submitted = sv->batches = sv->rejected = sv->cancelled = sv->failed = 0;
  sv->any_done = false;
  return HPM_OK;
}

hpm_status hpm_server_destroy(hpm_server_t sv) {
  if (!sv) return HPM_OK;
  {
    // wake the threads blocked in hpm_server_wait (they return HPM_ERR_BUSY)
    // and wait until none is left inside before anything is freed
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_done.notify_all();
    sv->cv_idle.wait(lk, [sv] { return sv->waiters == 0; });
  }
  sv->cv_work.notify_all();
  for (Worker *w : sv->workers)
    if (w->th.joinable()) w->th.join();
  for (Worker *w : sv->workers) {
    w->pos.release(w->stream);
    w->mass.release(w->stream);
    w->phi.release(w->stream);
    w->acc.release(w->stream);
    cudaStreamSynchronize(w->stream);
    hpm_destroy(w->plan);
    cudaStreamDestroy(w->stream);
    delete w;
  }
  for (auto &kv : sv->reqs) delete kv.second;
  delete sv;
  return HPM_OK;
}

}  // extern "C"
