// Zoom-window serving (continuous batching) for MinMaxLTTB.
//
// A plotting front end asks for (series, [start, end), n_out) windows of series
// that stay resident on the device.  Submitters enqueue requests; one scheduler
// thread forms batches from the queue (first come, first served) whenever one of
// `streams` slots is free, admitting requests while the batch's workspace still
// fits the slot's share of the device pool.  Each batch runs as one batched launch
// sequence on its slot's stream, followed by a copy of the indices into the slot's
// pinned host buffer and a host callback that marks the slot complete.  Requests
// arriving while batches are on the GPU join the next batch as soon as a slot
// frees up, so batches overlap on the device.  Latency = completion - submission.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.h"

using namespace mmlttb;
using Clock = std::chrono::steady_clock;

namespace {

struct Resident {
  const void* y;
  int32_t ydt;
  const void* x;
  int32_t xk;
  int64_t n;
};

enum ReqState : int { RQ_PENDING = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct Request {
  mmlttb_request q;
  int state = RQ_PENDING;
  int status = MMLTTB_OK;
  Clock::time_point t_submit, t_done;
  std::vector<int64_t> result;
  int64_t est_bytes = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  char* ws = nullptr;          // device workspace (slot share of the pool)
  size_t ws_bytes = 0;
  int64_t* out_dev = nullptr;  // max_batch * max_n_out indices
  int64_t* cnt_dev = nullptr;  // max_batch counts
  int64_t* out_host = nullptr; // pinned copies
  int64_t* cnt_host = nullptr;
  char* upload = nullptr;      // pinned plan image
  size_t upload_bytes = 0;
  std::vector<uint64_t> ids;
  bool busy = false;
  std::atomic<bool> done{false};
  struct mmlttb_server* srv = nullptr;
};

}  // namespace

struct mmlttb_server {
  mmlttb_server_config cfg;
  int device = 0;
  DevInfo dev;
  std::vector<Resident> series;
  std::mutex mu;
  std::condition_variable cv_sched;  // scheduler: work or completions
  std::condition_variable cv_done;   // waiters: a request finished
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Slot*> slots;
  std::thread sched;
  bool stop = false;
  uint64_t next_id = 1;
  int64_t in_flight_requests = 0;
  // statistics since the last reset
  std::vector<double> lat;
  int64_t batches = 0, batched_requests = 0, submitted = 0, rejected = 0;
  int64_t overlapped_batches = 0, max_in_flight = 0;
  unsigned long long launches = 0;
  int last_error = MMLTTB_OK;
};

namespace {

// Conservative workspace bytes one request adds to a batch (the batch planner's
// per-series sections, each rounded up to 256 bytes).
int64_t request_bytes(const Resident& r, const mmlttb_request& q) {
  const int64_t B = q.n_out * (int64_t)q.r_ps / 2;
  int64_t b = (int64_t)sizeof(SeriesPlan) + 4 * 8 + 8;  // plan, offset tables, m
  b += (B + 1) * 8 * (q.binmode == MMLTTB_BINS_XWIDTH ? 1 : 0);
  b += B * (int64_t)sizeof(Record);
  b += (2 * B + 2) * 8 * 3 + (2 * B + 2) + 15;  // preselected list, its x and y, tables
  b += ((B + kBinsPerCta - 1) / kBinsPerCta) * (kBinsPerCta * 16 + 16);  // compaction
  b += 16 * q.n_out;                    // means if the block engine is chosen
  return b + 12 * 256;
}

int64_t batch_fixed_bytes(const mmlttb_server* s) {
  const int64_t wcap = stream_warp_cap(s->dev);
  return (int64_t)kHeader + wcap * (int64_t)sizeof(Record) + 12 * 256;
}

void CUDART_CB on_batch_done(void* arg) {
  Slot* slot = (Slot*)arg;
  mmlttb_server* s = slot->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    slot->done.store(true);
  }
  s->cv_sched.notify_one();
}

// Called with the lock held: move a completed slot's results into its requests.
void finish_slot(mmlttb_server* s, Slot* slot) {
  const Clock::time_point now = Clock::now();
  const int64_t cap = s->cfg.max_n_out;
  for (size_t i = 0; i < slot->ids.size(); ++i) {
    auto it = s->reqs.find(slot->ids[i]);
    if (it == s->reqs.end()) continue;
    Request& r = it->second;
    const int64_t c = slot->cnt_host[i];
    const int64_t* src = slot->out_host + (int64_t)i * cap;
    r.result.resize((size_t)(c > 0 ? c : 0));
    for (int64_t k = 0; k < c; ++k) r.result[k] = src[k] + r.q.start;  // window -> series index
    r.state = RQ_DONE;
    r.t_done = now;
    s->lat.push_back(std::chrono::duration<double>(now - r.t_submit).count());
  }
  s->in_flight_requests -= (int64_t)slot->ids.size();
  slot->ids.clear();
  slot->busy = false;
  slot->done.store(false);
}

// Enqueue one batch on a slot (lock NOT held).  Returns an MMLTTB code.
int launch_batch(mmlttb_server* s, Slot* slot, std::vector<mmlttb_request>& qs) {
  BatchImpl b;
  b.n = (int64_t)qs.size();
  b.descs.resize(qs.size());
  const int64_t cap = s->cfg.max_n_out;
  for (size_t i = 0; i < qs.size(); ++i) {
    const mmlttb_request& q = qs[i];
    const Resident& r = s->series[q.series];
    const size_t es = r.ydt == MMLTTB_F32 ? 4 : 8;
    mmlttb_series_desc& d = b.descs[i];
    memset(&d, 0, sizeof(d));
    d.y = (const char*)r.y + (size_t)q.start * es;
    d.x = r.xk == MMLTTB_X_IMPLICIT ? nullptr : (const char*)r.x + (size_t)q.start * 8;
    d.op = MMLTTB_OP_MINMAXLTTB;
    d.ydtype = r.ydt;
    d.xkind = r.xk;
    d.binmode = q.binmode;
    d.r_ps = q.r_ps;
    d.n_in = q.end - q.start;
    d.n_out = q.n_out;
    d.out_idx = slot->out_dev + (int64_t)i * cap;
    d.out_cap = cap;
    d.out_count = slot->cnt_dev + i;
  }
  int rc = batch_plan(&b, s->dev, slot->upload, slot->upload_bytes);
  if (rc) return rc;
  if (b.total > slot->ws_bytes) return MMLTTB_ENOSPC;
  const unsigned long long before = g_launches;
  rc = batch_enqueue(&b, slot->ws, slot->stream);
  if (rc) return rc;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(slot->cnt_host, slot->cnt_dev, qs.size() * 8, cudaMemcpyDeviceToHost,
                           slot->stream)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaMemcpyAsync(slot->out_host, slot->out_dev, qs.size() * (size_t)cap * 8,
                           cudaMemcpyDeviceToHost, slot->stream)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaLaunchHostFunc(slot->stream, on_batch_done, slot)) != cudaSuccess) return cuda_fail(e);
  s->launches += g_launches - before;
  // The upload image normally lives in the slot's pinned buffer, untouched until the
  // slot is reused after this batch completed.  A batch that had to allocate its own
  // image frees it on return, so wait for the upload first.
  if (b.own_pinned && (e = cudaStreamSynchronize(slot->stream)) != cudaSuccess) return cuda_fail(e);
  return MMLTTB_OK;
}

void scheduler(mmlttb_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_sched.wait(lk, [&] {
      if (s->stop) return true;
      for (Slot* sl : s->slots)
        if (sl->busy && sl->done.load()) return true;
      if (s->pending.empty()) return false;
      for (Slot* sl : s->slots)
        if (!sl->busy) return true;
      return false;
    });
    bool finished = false;
    for (Slot* sl : s->slots)
      if (sl->busy && sl->done.load()) {
        finish_slot(s, sl);
        finished = true;
      }
    if (finished) s->cv_done.notify_all();
    bool any_busy = false;
    for (Slot* sl : s->slots) any_busy |= sl->busy;
    if (s->stop && s->pending.empty() && !any_busy) break;
    for (Slot* sl : s->slots) {
      if (sl->busy || s->pending.empty()) continue;
      // admission: FIFO while the batch fits the slot's workspace and size limit
      std::vector<uint64_t> ids;
      std::vector<mmlttb_request> qs;
      int64_t bytes = batch_fixed_bytes(s) +
                      (int64_t)batch_upload_bytes(std::min<int64_t>(s->cfg.max_batch, (int64_t)s->pending.size()));
      while (!s->pending.empty() && (int64_t)ids.size() < s->cfg.max_batch) {
        Request& r = s->reqs[s->pending.front()];
        if (!ids.empty() && bytes + r.est_bytes > (int64_t)sl->ws_bytes) break;
        bytes += r.est_bytes;
        ids.push_back(s->pending.front());
        qs.push_back(r.q);
        r.state = RQ_RUNNING;
        s->pending.pop_front();
      }
      // batches still in flight on the other slots when this one is admitted
      int64_t others = 0;
      for (Slot* o : s->slots) others += (o != sl && o->busy) ? 1 : 0;
      if (others > 0) s->overlapped_batches += 1;
      s->max_in_flight = std::max<int64_t>(s->max_in_flight, others + 1);
      sl->ids = ids;
      sl->busy = true;
      sl->done.store(false);
      s->in_flight_requests += (int64_t)ids.size();
      s->batches += 1;
      s->batched_requests += (int64_t)ids.size();
      lk.unlock();
      int rc = launch_batch(s, sl, qs);
      lk.lock();
      if (rc) {  // the batch never reached the GPU: fail its requests
        for (uint64_t id : ids) {
          Request& r = s->reqs[id];
          r.state = RQ_DONE;
          r.status = rc;
          r.t_done = Clock::now();
        }
        s->in_flight_requests -= (int64_t)ids.size();
        sl->ids.clear();
        sl->busy = false;
        s->last_error = rc;
        s->cv_done.notify_all();
      }
    }
  }
}

int validate(const mmlttb_server* s, const mmlttb_request& q) {
  if (q.series < 0 || q.series >= (int64_t)s->series.size()) return MMLTTB_EINVAL;
  const Resident& r = s->series[q.series];
  if (q.start < 0 || q.end > r.n || q.start >= q.end) return MMLTTB_EINVAL;
  if (q.n_out < 3 || q.n_out > s->cfg.max_n_out || q.r_ps < 2) return MMLTTB_EINVAL;
  if (q.binmode != MMLTTB_BINS_INDEX && q.binmode != MMLTTB_BINS_XWIDTH) return MMLTTB_EINVAL;
  if (q.binmode == MMLTTB_BINS_XWIDTH && r.xk == MMLTTB_X_IMPLICIT) return MMLTTB_EINVAL;
  int32_t br;
  int64_t B;
  return classify(MMLTTB_OP_MINMAXLTTB, r.ydt, r.xk, q.end - q.start, q.n_out, q.r_ps, q.binmode, &br, &B);
}

void free_slot(Slot* sl) {
  if (sl->stream) cudaStreamDestroy(sl->stream);
  if (sl->out_host) cudaFreeHost(sl->out_host);
  if (sl->cnt_host) cudaFreeHost(sl->cnt_host);
  if (sl->upload) cudaFreeHost(sl->upload);
  delete sl;
}

}  // namespace

extern "C" {

int mmlttb_server_pool_bytes(const mmlttb_server_config* cfg, size_t* bytes) {
  if (!cfg || !bytes || cfg->streams < 1 || cfg->max_batch < 1 || cfg->max_n_out < 3 ||
      cfg->workspace_bytes_per_stream < (int64_t)(64 << 10))
    return MMLTTB_EINVAL;
  const size_t per = align256((size_t)cfg->workspace_bytes_per_stream) +
                     align256((size_t)cfg->max_batch * (size_t)cfg->max_n_out * 8) +
                     align256((size_t)cfg->max_batch * 8);
  *bytes = per * (size_t)cfg->streams;
  return MMLTTB_OK;
}

int mmlttb_server_create(const mmlttb_server_config* cfg, void* device_pool, size_t pool_bytes,
                         mmlttb_server_t* out) {
  if (!out) return MMLTTB_EINVAL;
  *out = nullptr;
  size_t need = 0;
  int rc = mmlttb_server_pool_bytes(cfg, &need);
  if (rc) return rc;
  if (!device_pool || pool_bytes < need) return MMLTTB_ENOSPC;
  if (cfg->max_pending < 1) return MMLTTB_EINVAL;
  mmlttb_server* s = new (std::nothrow) mmlttb_server;
  if (!s) return MMLTTB_ENOMEM;
  s->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) { delete s; return cuda_fail(e); }
  rc = get_dev_info(&s->dev);
  if (rc) { delete s; return rc; }
  char* p = (char*)device_pool;
  const size_t up = batch_upload_bytes(cfg->max_batch);
  for (int i = 0; i < cfg->streams; ++i) {
    Slot* sl = new (std::nothrow) Slot;
    if (!sl) { mmlttb_server_destroy(s); return MMLTTB_ENOMEM; }
    sl->srv = s;
    s->slots.push_back(sl);
    sl->ws = p;
    sl->ws_bytes = align256((size_t)cfg->workspace_bytes_per_stream);
    p += sl->ws_bytes;
    sl->out_dev = (int64_t*)p;
    p += align256((size_t)cfg->max_batch * (size_t)cfg->max_n_out * 8);
    sl->cnt_dev = (int64_t*)p;
    p += align256((size_t)cfg->max_batch * 8);
    sl->upload_bytes = up;
    if ((e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&sl->out_host, (size_t)cfg->max_batch * cfg->max_n_out * 8, 0)) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&sl->cnt_host, (size_t)cfg->max_batch * 8, 0)) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&sl->upload, up, 0)) != cudaSuccess) {
      mmlttb_server_destroy(s);
      return cuda_fail(e);
    }
  }
  s->sched = std::thread(scheduler, s);
  *out = s;
  return MMLTTB_OK;
}

int mmlttb_server_add_series(mmlttb_server_t s, const void* y, int ydtype, const void* x, int xkind,
                             int64_t n, int64_t* series_id) {
  if (!s || !series_id || n < 1 || !y) return MMLTTB_EINVAL;
  if (ydtype != MMLTTB_F32 && ydtype != MMLTTB_F64) return MMLTTB_EINVAL;
  if (xkind != MMLTTB_X_IMPLICIT && xkind != MMLTTB_X_I64 && xkind != MMLTTB_X_F64) return MMLTTB_EINVAL;
  if (xkind != MMLTTB_X_IMPLICIT && !x) return MMLTTB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->series.push_back(Resident{y, ydtype, xkind == MMLTTB_X_IMPLICIT ? nullptr : x, xkind, n});
  *series_id = (int64_t)s->series.size() - 1;
  return MMLTTB_OK;
}

int mmlttb_server_submit(mmlttb_server_t s, const mmlttb_request* q, uint64_t* request_id) {
  if (!s || !q || !request_id) return MMLTTB_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  int rc = validate(s, *q);
  if (rc) { s->rejected++; return rc; }
  const Resident& res = s->series[q->series];
  Request r;
  r.q = *q;
  r.est_bytes = request_bytes(res, *q);
  if (batch_fixed_bytes(s) + (int64_t)batch_upload_bytes(1) + r.est_bytes > s->cfg.workspace_bytes_per_stream) {
    s->rejected++;
    return MMLTTB_ENOSPC;  // would not fit a slot even alone
  }
  if ((int64_t)s->pending.size() >= s->cfg.max_pending) {
    s->rejected++;
    return MMLTTB_EBUSY;
  }
  r.t_submit = Clock::now();
  const uint64_t id = s->next_id++;
  s->reqs.emplace(id, std::move(r));
  s->pending.push_back(id);
  s->submitted++;
  *request_id = id;
  lk.unlock();
  s->cv_sched.notify_one();
  return MMLTTB_OK;
}

int mmlttb_server_wait(mmlttb_server_t s, uint64_t id, int64_t* out_host, int64_t out_cap,
                       int64_t* count, double* latency_s) {
  if (!s) return MMLTTB_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MMLTTB_EINVAL;
  s->cv_done.wait(lk, [&] { return it->second.state == RQ_DONE; });
  Request& r = it->second;
  int rc = r.status;
  const int64_t c = (int64_t)r.result.size();
  if (count) *count = rc ? 0 : c;
  if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
  if (!rc && out_host) {
    if (out_cap < c) rc = MMLTTB_ERANGE;
    else memcpy(out_host, r.result.data(), (size_t)c * 8);
  }
  s->reqs.erase(it);
  return rc;
}

int mmlttb_server_drain(mmlttb_server_t s) {
  if (!s) return MMLTTB_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->pending.empty() && s->in_flight_requests == 0; });
  return s->last_error;
}

int mmlttb_server_replay(mmlttb_server_t s, const mmlttb_request* reqs, const double* t_offset_s,
                         int64_t n, uint64_t* ids, int* status) {
  if (!s || (n > 0 && (!reqs || !t_offset_s || !ids))) return MMLTTB_EINVAL;
  const Clock::time_point t0 = Clock::now();
  int first_err = MMLTTB_OK;
  for (int64_t i = 0; i < n; ++i) {
    const Clock::time_point due =
        t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t_offset_s[i]));
    while (Clock::now() < due) {
    }
    int rc = mmlttb_server_submit(s, &reqs[i], &ids[i]);
    if (status) status[i] = rc;
    if (rc) {
      ids[i] = 0;
      if (!first_err) first_err = rc;
    }
  }
  return first_err;
}

int mmlttb_server_get_stats(mmlttb_server_t s, mmlttb_server_stats* st) {
  if (!s || !st) return MMLTTB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = (int64_t)s->lat.size();
  st->rejected = s->rejected;
  st->batches = s->batches;
  st->mean_batch = s->batches ? (double)s->batched_requests / (double)s->batches : 0.0;
  st->gpu_launches = (int64_t)s->launches;
  st->overlapped_batches = s->overlapped_batches;
  st->max_batches_in_flight = s->max_in_flight;
  if (!s->lat.empty()) {
    std::vector<double> v = s->lat;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[(size_t)std::min<double>((double)v.size() - 1, f * (double)(v.size() - 1) + 0.5)]; };
    st->latency_p50_s = q(0.50);
    st->latency_p99_s = q(0.99);
    st->latency_max_s = v.back();
    double sum = 0;
    for (double d : v) sum += d;
    st->latency_mean_s = sum / (double)v.size();
  }
  return MMLTTB_OK;
}

int mmlttb_server_reset_stats(mmlttb_server_t s) {
  if (!s) return MMLTTB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat.clear();
  s->batches = s->batched_requests = s->submitted = s->rejected = 0;
  s->overlapped_batches = s->max_in_flight = 0;
  s->launches = 0;
  return MMLTTB_OK;
}

int mmlttb_server_destroy(mmlttb_server_t s) {
  if (!s) return MMLTTB_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->sched.joinable()) s->sched.join();
  for (Slot* sl : s->slots) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    free_slot(sl);
  }
  delete s;
  return MMLTTB_OK;
}

}  // extern "C"
