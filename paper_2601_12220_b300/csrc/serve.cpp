// Serving loop: continuous batching of batched-einsum requests.
//
// A request is a parsed batched einsum with device-resident operands and
// outputs (the operands stay on the device; only descriptors travel).  The
// caller submits requests at any time; a worker thread admits them in
// arrival order as long as the bytes pinned by requests in flight (their
// declared buffers and outputs) stay within the HBM budget, and launches each
// admitted request at once on one of several streams, so requests that
// arrive while others run overlap with them on the device.  An event is
// recorded behind each request's kernels; a completion thread polls the
// oldest event of every stream (events of one stream complete in order),
// stamps the completion time, releases the budget and wakes the worker,
// which then admits what was waiting.  Events do not hold the stream the
// way a host callback does, so a stream's next request starts as soon as
// the previous one's kernels finish.
// The configuration of each request comes from the tuning database under its
// normal form (Alg. 1 + lookup), memoized by the request's text.
// Requests repeat: the same einsum on the same resident buffers.  A request
// whose template has no graph yet launches directly, and a capture thread
// then records the template's launches into a CUDA graph, keyed by the
// einsum, its buffers, scalars and configuration; later requests of the
// template replay the graph (one launch call of a few microseconds instead of
// one per row with its parameter block), which keeps the single worker thread
// ahead of the arrivals.  The graph is built by recording the launches as
// kernel nodes (no stream capture, which would make the caller's device
// synchronizations fail while it lasts), on its own thread, so it never holds
// up admission.  Split-precision requests use the
// context's workspace, which can move, and always launch directly.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>

#include "handles.hpp"
#include "launch_rec.hpp"

namespace {

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

int sfail(int code, const std::string &m) {
  be::set_last_error(m);
  return code;
}

}  // namespace

struct ServeReq;

struct be_server {
  be_ctx *x = nullptr;
  int device = 0;
  int32_t precision = BE_PREC_FP64;
  size_t budget = 0;
  size_t inflight_bytes = 0, peak_bytes = 0;
  int64_t inflight = 0, max_inflight = 0;
  std::vector<cudaStream_t> streams;
  size_t next_stream = 0;
  std::vector<std::deque<std::pair<ServeReq *, cudaEvent_t>>> running;   // per stream, launch order
  std::vector<cudaEvent_t> free_events;
  std::atomic<uint64_t> launched{0};   // requests handed to the completion thread
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_reap;
  std::deque<ServeReq *> pending;
  std::unordered_map<int64_t, std::unique_ptr<ServeReq>> reqs;
  int64_t next_id = 1;
  std::vector<double> latencies;
  // per completed request: id, submit, admit, launched (the launch calls
  // returned), done, stream -- the tracing view of the latency
  std::vector<std::array<double, 6>> trace;
  int64_t completed = 0, failed = 0;
  double first_submit = -1, last_done = -1;
  std::unordered_map<std::string, be_config> cfg_memo;
  std::unordered_map<std::string, bool> cfg_have;
  bool stop = false;
  std::thread worker, reaper;
  // captured launches of request templates, filled by the capture thread
  struct CaptureJob {
    std::string key, text;
    bool have;
    be_config cfg;
    std::vector<be_buf> bufs, outs;
    std::vector<std::vector<int64_t>> strides;
    std::vector<double> scalars;
  };
  std::mutex gmu;
  std::condition_variable gcv;
  std::unordered_map<std::string, cudaGraphExec_t> graphs;
  std::unordered_map<std::string, bool> queued;
  std::deque<CaptureJob> jobs;
  bool gstop = false;
  cudaStream_t cap = nullptr;
  std::thread capturer;
};

struct ServeReq {
  be_server *srv;
  int64_t id;
  be_einsum *e;
  std::vector<be_buf> bufs, outs;
  std::vector<std::vector<int64_t>> strides;
  std::vector<double> scalars;
  size_t bytes = 0;
  double t_submit = 0, t_admit = 0, t_launched = 0, t_done = 0;
  int stream = -1;
  int state = 0;      // 0 queued, 1 running, 2 done
  int status = BE_OK;
};

// completion of a running request (the server's lock held)
static void finish(be_server *s, ServeReq *r, double t, int status) {
  r->t_done = t;
  r->state = 2;
  r->status = status;
  s->inflight_bytes -= r->bytes;
  s->inflight -= 1;
  if (status == BE_OK) {
    s->latencies.push_back(t - r->t_submit);
    s->trace.push_back({(double)r->id, r->t_submit, r->t_admit, r->t_launched, t, (double)r->stream});
    s->completed += 1;
    s->last_done = std::max(s->last_done, t);
  } else {
    s->failed += 1;
  }
}

// Completion thread: snapshots the oldest running request of each stream,
// then queries their events without the lock until one has finished or the
// worker has launched more, and retires every finished head under the
// lock.  While requests are in flight it spins (yielding) and falls back to
// short sleeps after a while without progress; with nothing in flight it
// waits for the worker.
static void reaper_loop(be_server *s) {
  cudaSetDevice(s->device);
  using Head = std::pair<ServeReq *, cudaEvent_t>;
  std::vector<Head> heads(s->streams.size());
  std::vector<cudaError_t> res(s->streams.size());
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool any = false;
    for (size_t k = 0; k < heads.size(); ++k) {
      heads[k] = s->running[k].empty() ? Head{nullptr, nullptr} : s->running[k].front();
      any |= heads[k].first != nullptr;
    }
    if (!any) {
      if (s->stop && s->pending.empty() && s->inflight == 0) break;
      s->cv_reap.wait(lk);
      continue;
    }
    const uint64_t seen = s->launched.load(std::memory_order_relaxed);
    lk.unlock();
    int idle = 0;
    bool progress = false;
    while (true) {
      for (size_t k = 0; k < heads.size(); ++k) {
        res[k] = heads[k].first ? cudaEventQuery(heads[k].second) : cudaErrorNotReady;
        progress |= res[k] != cudaErrorNotReady;
      }
      if (progress || s->launched.load(std::memory_order_relaxed) != seen) break;
      if (++idle < 4096) std::this_thread::yield();
      else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    const double t = now_s();
    lk.lock();
    if (!progress) continue;
    for (size_t k = 0; k < heads.size(); ++k) {
      if (res[k] == cudaErrorNotReady) continue;
      s->running[k].pop_front();
      s->free_events.push_back(heads[k].second);
      finish(s, heads[k].first, t, res[k] == cudaSuccess ? BE_OK : BE_ECUDA);
    }
    s->cv_work.notify_one();
    s->cv_done.notify_all();
  }
}

// key of a request template: einsum text, configuration, buffers (pointer,
// dtype, strides), outputs and scalars, as raw bytes
static std::string template_key(const ServeReq *r, const be_config *cfg) {
  std::string k = r->e->e.text;       // the einsum by its text: a handle's address can be reused
  k.push_back('\0');
  auto put = [&](const void *p, size_t n) { k.append((const char *)p, n); };
  const char has = cfg != nullptr;
  put(&has, 1);
  if (cfg) put(cfg, sizeof(*cfg));
  for (const auto *v : {&r->bufs, &r->outs}) {
    const size_t n = v->size();
    put(&n, sizeof(n));
    for (const be_buf &b : *v) {
      put(&b.ptr, sizeof(b.ptr));
      put(&b.ndim, sizeof(b.ndim));
      put(&b.dtype, sizeof(b.dtype));
      if (b.strides) put(b.strides, sizeof(int64_t) * (size_t)b.ndim);
    }
  }
  put(r->scalars.data(), sizeof(double) * r->scalars.size());
  return k;
}

// Capture thread: records each queued template's launches into a graph
// (launch_rec.hpp: the launches become kernel nodes, nothing runs and no
// stream is captured, so the caller's synchronizations are never affected)
// and publishes the instantiated graph
static void capture_loop(be_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->gmu);
  while (true) {
    s->gcv.wait(lk, [&] { return s->gstop || !s->jobs.empty(); });
    if (s->gstop) break;
    be_server::CaptureJob j = std::move(s->jobs.front());
    s->jobs.pop_front();
    lk.unlock();
    cudaGraphExec_t exec = nullptr;
    // a private parse of the template's text: the caller may free its handle
    // once its request is done
    be_einsum *e = nullptr;
    LaunchRecorder rec;
    if (be_parse(j.text.c_str(), &e) == BE_OK && cudaGraphCreate(&rec.graph, 0) == cudaSuccess) {
      launch_recorder() = &rec;
      const int rc = be::execute_internal(s->x, e, j.have ? &j.cfg : nullptr, s->precision, j.bufs.data(),
                                          (int32_t)j.bufs.size(), j.outs.data(), (int32_t)j.outs.size(),
                                          j.scalars.data(), (int32_t)j.scalars.size(), s->cap);
      launch_recorder() = nullptr;
      if (rc == BE_OK && rec.status == cudaSuccess && rec.nodes > 0 &&
          cudaGraphInstantiate(&exec, rec.graph, 0) != cudaSuccess)
        exec = nullptr;
      cudaGraphDestroy(rec.graph);
    }
    be_free_einsum(e);
    cudaGetLastError();   // a failed recording leaves no sticky error behind
    lk.lock();
    if (exec) s->graphs.emplace(j.key, exec);
  }
}

static void worker_loop(be_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    while (!s->pending.empty()) {
      ServeReq *r = s->pending.front();
      if (r->bytes > s->budget && s->budget > 0) {            // can never fit
        r->status = BE_EBUDGET;
        r->state = 2;
        r->t_done = now_s();
        s->failed += 1;
        s->pending.pop_front();
        s->cv_done.notify_all();
        continue;
      }
      if (s->budget > 0 && s->inflight > 0 && s->inflight_bytes + r->bytes > s->budget) break;   // wait for room
      s->pending.pop_front();
      // configuration under the normal form, memoized by text
      be_config cfg;
      bool have = false;
      auto it = s->cfg_have.find(r->e->e.text);
      if (it != s->cfg_have.end()) {
        have = it->second;
        if (have) cfg = s->cfg_memo[r->e->e.text];
      } else {
        std::string err;
        int st;
        const Canon *c = be::canon_cached(r->e, err, st);
        if (!st && s->x) {
          lk.unlock();
          double sec;
          be_canon bc;
          bc.c = *c;
          have = be_lookup(s->x, &bc, s->precision, &cfg, &sec) == BE_OK;
          lk.lock();
        }
        s->cfg_have[r->e->e.text] = have;
        if (have) s->cfg_memo[r->e->e.text] = cfg;
      }
      // the stream with the fewest requests in flight (from a rotating start,
      // so ties spread); the dense split strategy shares its context's
      // workspace: keep it on one stream
      size_t si = 0;
      if (s->precision != BE_PREC_SPLIT) {
        const size_t ns = s->streams.size();
        si = s->next_stream;
        for (size_t j = 1; j < ns; ++j) {
          const size_t c = (s->next_stream + j) % ns;
          if (s->running[c].size() < s->running[si].size()) si = c;
        }
        s->next_stream = (si + 1) % ns;
      }
      cudaStream_t st = s->streams[si];
      cudaEvent_t ev = nullptr;
      if (!s->free_events.empty()) {
        ev = s->free_events.back();
        s->free_events.pop_back();
      } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        ev = nullptr;
      }
      r->t_admit = now_s();
      r->state = 1;
      s->inflight_bytes += r->bytes;
      s->inflight += 1;
      s->peak_bytes = std::max(s->peak_bytes, s->inflight_bytes);
      s->max_inflight = std::max(s->max_inflight, s->inflight);
      lk.unlock();
      int rc = BE_OK;
      bool done_launch = false;
      const bool graphable = s->precision != BE_PREC_SPLIT && s->cap && !(s->x && s->x->timing);
      std::string key;
      if (graphable) {
        key = template_key(r, have ? &cfg : nullptr);
        std::lock_guard<std::mutex> g(s->gmu);
        auto it2 = s->graphs.find(key);
        if (it2 != s->graphs.end()) {
          rc = cudaGraphLaunch(it2->second, st) == cudaSuccess ? BE_OK : BE_ECUDA;
          done_launch = true;
        }
      }
      if (!done_launch) {
        rc = be::execute_internal(s->x, r->e, have ? &cfg : nullptr, s->precision, r->bufs.data(),
                                  (int32_t)r->bufs.size(), r->outs.data(), (int32_t)r->outs.size(),
                                  r->scalars.data(), (int32_t)r->scalars.size(), st);
        // queue the template for capture (once; at most 65536 templates)
        if (rc == BE_OK && graphable) {
          std::lock_guard<std::mutex> g(s->gmu);
          if (!s->queued.count(key) && s->queued.size() < 65536) {
            s->queued[key] = true;
            be_server::CaptureJob j;
            j.key = key;
            j.text = r->e->e.text;
            j.have = have;
            if (have) j.cfg = cfg;
            j.bufs = r->bufs;
            j.outs = r->outs;
            j.scalars = r->scalars;
            j.strides.reserve(j.bufs.size() + j.outs.size());
            for (auto *v : {&j.bufs, &j.outs})
              for (auto &b : *v)
                if (b.strides) {
                  j.strides.emplace_back(b.strides, b.strides + b.ndim);
                  b.strides = j.strides.back().data();
                }
            s->jobs.push_back(std::move(j));
            s->gcv.notify_one();
          }
        }
      }
      r->t_launched = now_s();
      r->stream = (int)si;
      if (rc == BE_OK && ev && cudaEventRecord(ev, st) == cudaSuccess) {
        lk.lock();
        s->running[si].emplace_back(r, ev);
        s->launched.fetch_add(1, std::memory_order_relaxed);
        s->cv_reap.notify_one();
        continue;
      }
      lk.lock();
      if (ev) s->free_events.push_back(ev);
      finish(s, r, now_s(), rc ? rc : BE_ECUDA);
      s->cv_done.notify_all();
    }
    if (s->stop && s->pending.empty() && s->inflight == 0) break;
    s->cv_work.wait(lk);
  }
}

static size_t decl_bytes(const Einsum &e) {
  size_t n = 0;
  for (auto &b : e.buffers) {
    size_t k = (size_t)dtype_size(b.dtype);
    for (auto d : b.shape) k *= (size_t)d;
    n += k;
  }
  size_t o = (size_t)dtype_size(e.out_dtype);
  for (auto d : e.out_shape()) o *= (size_t)d;
  return n + o * (size_t)e.b;
}

extern "C" {

int be_server_create(be_ctx *x, int32_t precision, int32_t n_streams, size_t hbm_budget_bytes, be_server **out) {
  if (!out || n_streams < 1 || n_streams > 64) return sfail(BE_EARG, "n_streams must be in 1..64");
  auto s = std::make_unique<be_server>();
  s->x = x;
  s->precision = precision;
  s->budget = hbm_budget_bytes ? hbm_budget_bytes : (x ? x->hbm_budget : 0);
  cudaGetDevice(&s->device);
  for (int k = 0; k < n_streams; ++k) {
    cudaStream_t st;
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
      for (auto q : s->streams) cudaStreamDestroy(q);
      return sfail(BE_ECUDA, std::string("stream: ") + cudaGetErrorString(ce));
    }
    s->streams.push_back(st);
  }
  s->running.resize(s->streams.size());
  if (cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess) s->cap = nullptr;
  // room for many requests up front: growing these under the server's lock
  // (a rehash of the request table, a copy of the latency records) stalled
  // admission and completion for milliseconds at the growth points
  s->reqs.reserve(1 << 20);
  s->latencies.reserve(1 << 20);
  s->trace.reserve(1 << 20);
  be_server *raw = s.get();
  raw->worker = std::thread(worker_loop, raw);
  raw->reaper = std::thread(reaper_loop, raw);
  if (raw->cap) raw->capturer = std::thread(capture_loop, raw);
  *out = s.release();
  return BE_OK;
}

int be_server_submit(be_server *s, const be_einsum *e, const be_buf *bufs, int32_t n_bufs, const be_buf *outs,
                     int32_t n_outs, const double *scalars, int32_t n_scalars, int64_t *id) {
  if (!s || !e || !id || n_bufs < 0 || n_outs < 0 || n_scalars < 0) return sfail(BE_EARG, "bad request");
  auto r = std::make_unique<ServeReq>();
  r->srv = s;
  r->e = const_cast<be_einsum *>(e);
  r->bufs.assign(bufs, bufs + n_bufs);
  r->outs.assign(outs, outs + n_outs);
  // keep copies of the caller's stride arrays (reserved: no reallocation)
  r->strides.reserve(r->bufs.size());
  for (auto &b : r->bufs)
    if (b.strides) {
      r->strides.emplace_back(b.strides, b.strides + b.ndim);
      b.strides = r->strides.back().data();
    }
  if (scalars) r->scalars.assign(scalars, scalars + n_scalars);
  r->bytes = decl_bytes(e->e);
  r->t_submit = now_s();
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return sfail(BE_EARG, "server is shutting down");
  if (s->first_submit < 0) s->first_submit = r->t_submit;
  r->id = s->next_id++;
  *id = r->id;
  s->pending.push_back(r.get());
  s->reqs.emplace(r->id, std::move(r));
  s->cv_work.notify_one();
  return BE_OK;
}

int be_server_wait(be_server *s, int64_t id, double timeout_s, int32_t *status, double *latency_s) {
  if (!s) return sfail(BE_EARG, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(BE_EARG, "unknown request id");
  ServeReq *r = it->second.get();
  auto pred = [&] { return r->state == 2; };
  if (timeout_s < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
    return sfail(BE_ETIMEOUT, "request not finished within the timeout");
  if (status) *status = r->status;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  s->reqs.erase(it);
  return BE_OK;
}

int be_server_drain(be_server *s, double timeout_s) {
  if (!s) return sfail(BE_EARG, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto pred = [&] { return s->pending.empty() && s->inflight == 0; };
  if (timeout_s < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
    return sfail(BE_ETIMEOUT, "requests still in flight after the timeout");
  for (auto it = s->reqs.begin(); it != s->reqs.end();)
    it = it->second->state == 2 ? s->reqs.erase(it) : std::next(it);
  return BE_OK;
}

int be_server_stats(be_server *s, int64_t *completed, int64_t *failed, double *p50_s, double *p99_s,
                    double *throughput, size_t *peak_bytes, int64_t *max_inflight) {
  if (!s) return sfail(BE_EARG, "NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto q = [&](double f) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(f * (double)(l.size() - 1) + 0.5))]; };
  if (completed) *completed = s->completed;
  if (failed) *failed = s->failed;
  if (p50_s) *p50_s = q(0.50);
  if (p99_s) *p99_s = q(0.99);
  if (throughput)
    *throughput = (s->completed > 0 && s->last_done > s->first_submit) ? s->completed / (s->last_done - s->first_submit) : 0.0;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  if (max_inflight) *max_inflight = s->max_inflight;
  return BE_OK;
}

int be_server_trace(be_server *s, double *rows, int64_t cap, int64_t *n) {
  if (!s || !n || (cap > 0 && !rows)) return sfail(BE_EARG, "bad arguments");
  std::lock_guard<std::mutex> g(s->mu);
  *n = (int64_t)s->trace.size();
  const int64_t m = std::min<int64_t>(cap, *n);
  for (int64_t k = 0; k < m; ++k)
    for (int c = 0; c < 6; ++c) rows[k * 6 + c] = s->trace[(size_t)k][(size_t)c];
  return BE_OK;
}

int be_server_reset_stats(be_server *s) {
  if (!s) return sfail(BE_EARG, "NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  s->latencies.clear();
  s->trace.clear();
  s->latencies.reserve(1 << 20);
  s->trace.reserve(1 << 20);
  s->completed = s->failed = 0;
  s->first_submit = s->last_done = -1;
  s->peak_bytes = s->inflight_bytes;
  s->max_inflight = s->inflight;
  return BE_OK;
}

void be_server_destroy(be_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->cv_work.notify_one();
    s->cv_reap.notify_one();
  }
  s->worker.join();
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->cv_reap.notify_one();
  }
  s->reaper.join();
  if (s->capturer.joinable()) {
    {
      std::lock_guard<std::mutex> g(s->gmu);
      s->gstop = true;
    }
    s->gcv.notify_one();
    s->capturer.join();
  }
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto ev : s->free_events) cudaEventDestroy(ev);
  for (auto &g : s->graphs) cudaGraphExecDestroy(g.second);
  if (s->cap) cudaStreamDestroy(s->cap);
  delete s;
}

}  // extern "C"
