// mc_serve.cu -- serving loop with continuous batching.
//
// Requests (AMR boxes of cells on any uploaded network) are queued by
// mc_request_submit and admitted in arrival order by a host thread while the
// bytes of admitted state stay within the HBM budget. An admitted request's
// state is copied into pooled device memory (the state then stays device
// resident until its burn ends), burned on one of the server's streams and
// copied back; requests that arrive while others are on the GPU are admitted as
// soon as memory allows and start at once on their own stream, so the work of
// several requests overlaps on the device. Completion is detected with events;
// no device code waits on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mc_internal.h"
#include "mc_kernels.cuh"

using namespace mc;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  const mc_network *net = nullptr;
  int64_t n = 0, ld = 0;
  double dt = 0.0;
  double *x = nullptr, *T = nullptr;
  const double *nd = nullptr;
  int32_t *status = nullptr;
  size_t bytes = 0;
  int state = MC_PENDING;
  int32_t n_failed = 0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  int stream = -1;
  char *dev = nullptr;          // pooled device state
  int32_t *hstatus = nullptr;   // pinned copy of the statuses (failure count)
  cudaEvent_t done = nullptr;
};

size_t request_bytes(const mc_network *net, int64_t n) {
  return (size_t)n * (sizeof(double) * (net->S + 2) + sizeof(int32_t)) + 4 * 256;
}

}  // namespace

struct mc_server {
  int device = 0;
  uint64_t budget = 0;
  mc_burn_opts opts;
  Clock::time_point t0;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_busy;
  std::mutex mu;
  std::condition_variable cv;       // wakes the loop (new work / stop)
  std::condition_variable done_cv;  // wakes drainers
  std::deque<uint64_t> pending;     // FIFO of request ids
  std::map<uint64_t, Request> reqs;
  std::vector<uint64_t> inflight;
  uint64_t next_id = 1;
  uint64_t used = 0;
  int64_t outstanding = 0;
  bool stop = false;
  std::thread loop;
  mc_status loop_error = MC_OK;
  std::string loop_msg;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Admit one request: device state from the pool, copies in, burn, copies out,
// completion event -- all on the request's stream. Runs on the server thread.
mc_status start_request(mc_server *s, Request &r) {
  const cudaStream_t st = s->streams[r.stream];
  const int64_t n = r.n;
  const int S = r.net->S;
  cudaError_t e = cudaMallocAsync((void **)&r.dev, r.bytes, st);
  if (e != cudaSuccess) return cuda_error(e, "server pool allocation");
  if (!r.hstatus) {
    e = cudaMallocHost((void **)&r.hstatus, sizeof(int32_t) * n);
    if (e != cudaSuccess) return cuda_error(e, "server pinned status");
  }
  size_t off = 0;
  auto take = [&](size_t b) { char *p = r.dev + off; off += (b + 255) & ~(size_t)255; return p; };
  CellArgs a{};
  a.n_cells = n;
  a.ld = n;
  a.dt = r.dt;
  a.x = (double *)take(sizeof(double) * S * n);
  a.T = r.T ? (double *)take(sizeof(double) * n) : nullptr;
  a.nd = r.nd ? (const double *)take(sizeof(double) * n) : nullptr;
  a.status = (int32_t *)take(sizeof(int32_t) * n);
  e = cudaMemcpy2DAsync(a.x, sizeof(double) * n, r.x, sizeof(double) * r.ld, sizeof(double) * n, S,
                        cudaMemcpyDefault, st);
  if (e == cudaSuccess && r.T) e = cudaMemcpyAsync(a.T, r.T, sizeof(double) * n, cudaMemcpyDefault, st);
  if (e == cudaSuccess && r.nd) e = cudaMemcpyAsync((void *)a.nd, r.nd, sizeof(double) * n, cudaMemcpyDefault, st);
  if (e != cudaSuccess) return cuda_error(e, "server copy in");
  mc_status ms = burn_device(r.net, s->opts, a, st);
  if (ms != MC_OK) return ms;
  e = cudaMemcpy2DAsync(r.x, sizeof(double) * r.ld, a.x, sizeof(double) * n, sizeof(double) * n, S,
                        cudaMemcpyDefault, st);
  if (e == cudaSuccess && r.T) e = cudaMemcpyAsync(r.T, a.T, sizeof(double) * n, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r.status, a.status, sizeof(int32_t) * n, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r.hstatus, a.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaFreeAsync(r.dev, st);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r.done, st);
  if (e != cudaSuccess) return cuda_error(e, "server copy out");
  r.dev = nullptr;
  return MC_OK;
}

void server_loop(mc_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // admissions: FIFO while the budget and a free stream allow
    while (!s->pending.empty()) {
      Request &r = s->reqs[s->pending.front()];
      if (s->used + r.bytes > s->budget) break;
      int k = -1;
      for (size_t i = 0; i < s->streams.size(); ++i)
        if (!s->stream_busy[i]) { k = (int)i; break; }
      if (k < 0) break;
      s->pending.pop_front();
      s->stream_busy[k] = 1;
      s->used += r.bytes;
      r.stream = k;
      r.t_admit = s->now();
      const mc_status ms = start_request(s, r);
      if (ms != MC_OK) {
        s->loop_error = ms;
        s->loop_msg = mc_last_error();
        r.state = ms;
        r.t_done = s->now();
        s->used -= r.bytes;
        s->stream_busy[k] = 0;
        s->outstanding -= 1;
        s->done_cv.notify_all();
        continue;
      }
      s->inflight.push_back(r.id);
    }
    // completions
    for (size_t i = 0; i < s->inflight.size();) {
      Request &r = s->reqs[s->inflight[i]];
      const cudaError_t q = cudaEventQuery(r.done);
      if (q == cudaErrorNotReady) { ++i; continue; }
      int32_t failed = 0;
      if (q == cudaSuccess) {
        for (int64_t c = 0; c < r.n; ++c) failed += (r.hstatus[c] != MC_CELL_OK);
        r.state = MC_OK;
      } else {
        r.state = cuda_error(q, "request");
      }
      r.n_failed = failed;
      r.t_done = s->now();
      cudaEventDestroy(r.done);
      r.done = nullptr;
      cudaFreeHost(r.hstatus);
      r.hstatus = nullptr;
      s->used -= r.bytes;
      s->stream_busy[r.stream] = 0;
      s->outstanding -= 1;
      s->inflight.erase(s->inflight.begin() + i);
      s->done_cv.notify_all();
    }
    if (s->stop && s->pending.empty() && s->inflight.empty()) break;
    if (s->inflight.empty() && (s->pending.empty() || s->stop))
      s->cv.wait_for(lk, std::chrono::milliseconds(50));
    else
      s->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace

extern "C" mc_status mc_server_create(int32_t device, uint64_t hbm_budget_bytes, const mc_burn_opts *opts,
                                      mc_server **out) {
  if (!out) return set_error(MC_E_INVALID, "mc_server_create: null out");
  *out = nullptr;
  mc_burn_opts o;
  mc_status st = check_opts(opts, &o);
  if (st != MC_OK) return st;
  if (hbm_budget_bytes == 0) return set_error(MC_E_INVALID, "mc_server_create: zero budget");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(e, "mc_server_create: device");
  mc_server *s = new (std::nothrow) mc_server();
  if (!s) return set_error(MC_E_NOMEM, "mc_server_create");
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->opts = o;
  s->t0 = Clock::now();
  const int nstreams = 8;
  for (int i = 0; i < nstreams; ++i) {
    cudaStream_t q;
    e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return cuda_error(e, "server stream");
    }
    s->streams.push_back(q);
    s->stream_busy.push_back(0);
  }
  s->loop = std::thread(server_loop, s);
  *out = s;
  return MC_OK;
}

extern "C" mc_status mc_request_submit(mc_server *s, const mc_network *net, int64_t n_cells, double dt, double *x,
                                       int64_t ld, double *T, const double *ndens, int32_t *status,
                                       uint64_t *req_id) {
  if (!s || !net || !req_id) return set_error(MC_E_INVALID, "mc_request_submit: null argument");
  if (n_cells <= 0 || ld < n_cells || n_cells > (int64_t)INT32_MAX || !x || !status || (net->energy && !T))
    return set_error(MC_E_INVALID, "mc_request_submit: bad cells");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(MC_E_INVALID, "mc_request_submit: dt must be positive");
  if (net->device != s->device) return set_error(MC_E_INVALID, "mc_request_submit: network on another device");
  const size_t b = request_bytes(net, n_cells);
  if (b > s->budget) return set_error(MC_E_BUDGET, "request of %zu bytes exceeds the budget of %llu", b,
                                      (unsigned long long)s->budget);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return set_error(MC_E_BUSY, "server is shutting down");
  Request r;
  r.id = s->next_id++;
  r.net = net;
  r.n = n_cells;
  r.ld = ld;
  r.dt = dt;
  r.x = x;
  r.T = T;
  r.nd = ndens;
  r.status = status;
  r.bytes = b;
  r.t_submit = s->now();
  s->reqs[r.id] = r;
  s->pending.push_back(r.id);
  s->outstanding += 1;
  *req_id = r.id;
  s->cv.notify_all();
  return MC_OK;
}

extern "C" mc_status mc_request_poll(mc_server *s, uint64_t req_id, mc_request_info *info) {
  if (!s) return set_error(MC_E_INVALID, "mc_request_poll: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return set_error(MC_E_NOTFOUND, "unknown request %llu", (unsigned long long)req_id);
  const Request &r = it->second;
  if (info) {
    info->state = r.state;
    info->n_failed = r.n_failed;
    info->n_cells = r.n;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
  }
  if (r.state < 0) return set_error(r.state, "request %llu failed: %s", (unsigned long long)req_id, s->loop_msg.c_str());
  return r.state == MC_OK ? MC_OK : MC_PENDING;
}

extern "C" mc_status mc_server_drain(mc_server *s, double timeout_s) {
  if (!s) return set_error(MC_E_INVALID, "mc_server_drain: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (s->outstanding > 0) {
    if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout && s->outstanding > 0)
      return set_error(MC_E_TIMEOUT, "%lld requests still outstanding", (long long)s->outstanding);
  }
  return MC_OK;
}

extern "C" mc_status mc_server_destroy(mc_server *s) {
  if (!s) return MC_OK;
  mc_status r = mc_server_drain(s, 600.0);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->loop.join();  // the loop leaves once nothing is pending or in flight
  for (cudaStream_t q : s->streams) {
    cudaStreamSynchronize(q);
    cudaStreamDestroy(q);
  }
  for (auto &kv : s->reqs)
    if (kv.second.hstatus) cudaFreeHost(kv.second.hstatus);
  delete s;
  return r;
}
