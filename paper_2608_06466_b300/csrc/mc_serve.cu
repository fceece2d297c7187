// mc_serve.cu -- serving loop with continuous batching.
//
// Requests (AMR boxes of cells on any uploaded network, each with its own
// options) are queued by mc_request_submit and admitted in arrival order by a
// host thread while the device bytes they need stay within the HBM budget:
// the request's state in pooled device memory plus the growth of the library
// scratch of the stream it runs on (retry list, cost order, straggler
// records; scratch is kept per stream and never shrinks, so each stream's
// high-water mark stays charged). An admitted request's state is copied into
// the pool (it then stays device resident until its burn ends), burned on one
// of the server's streams and copied back; requests that arrive while others
// are on the GPU are admitted as soon as memory and a stream allow and start
// at once on their own stream, so the work of several requests overlaps on
// the device. Failed cells are counted on the device; completion is detected
// with events (the results are copied back once a request's burn has ended),
// and each request records when its burn started and ended on the GPU. No device code waits on the host (paper: state resident in GPU
// memory, Software design section, paragraph 3).
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
constexpr int kStreams = 8;

struct Request {
  uint64_t id = 0;
  const mc_network *net = nullptr;
  mc_burn_opts opts{};
  int64_t n = 0, ld = 0;
  double dt = 0.0;
  double *x = nullptr, *T = nullptr;
  const double *nd = nullptr;
  int32_t *status = nullptr;
  size_t state_bytes = 0;     // pooled state
  size_t scratch_need = 0;    // the stream scratch its burn needs
  int state = MC_PENDING;
  int32_t n_failed = 0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0, gpu_start = 0.0, gpu_end = 0.0;
  int stream = -1;
  char *dev = nullptr;          // pooled device state
  CellArgs args{};              // the burn's view of the pooled state
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // timed: start and end of its burn on the stream
  std::string err;
};

size_t request_bytes(const mc_network *net, int64_t n) {
  return (size_t)n * (sizeof(double) * (net->S + 2) + sizeof(int32_t)) + 4 * 256;
}

// status != MC_CELL_OK over n cells, added to *count
__global__ void k_count_failed(const int32_t *status, int64_t n, uint32_t *count) {
  uint32_t c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += (status[i] != MC_CELL_OK) ? 1u : 0u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace

struct mc_server {
  int device = 0;
  uint64_t budget = 0;
  mc_burn_opts opts;
  Clock::time_point t0;
  cudaEvent_t ref = nullptr;            // GPU time origin (recorded at creation)
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_busy;
  std::vector<size_t> stream_scratch;   // each stream's scratch high-water mark
  uint32_t *fail_dev = nullptr;         // per stream: failed-cell count of its request
  uint32_t *fail_host = nullptr;        // pinned copies
  std::mutex mu;
  std::condition_variable cv;       // wakes the loop (new work / stop)
  std::condition_variable done_cv;  // wakes drainers
  std::deque<uint64_t> pending;     // FIFO of request ids
  std::map<uint64_t, Request> reqs;
  std::vector<uint64_t> inflight;
  uint64_t next_id = 1;
  uint64_t used = 0;                // pooled state of admitted requests
  uint64_t scratch_total = 0;       // sum of stream_scratch
  int64_t outstanding = 0;
  bool stop = false;
  std::thread loop;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Admit one request: device state from the pool, copies in, burn and the
// failed-cell count, then an event marking the end of its GPU work -- all on
// the request's stream. Runs on the server thread without the server lock and
// returns as soon as the work is queued; the results are copied out by
// finish_copies once that event has fired (a copy to pageable host memory
// would otherwise hold the server thread until the burn ends). On failure
// everything it allocated is released and the message is kept with the
// request.
mc_status start_request(mc_server *s, Request &r) {
  const cudaStream_t st = s->streams[r.stream];
  const int64_t n = r.n;
  const int S = r.net->S;
  cudaError_t e = cudaEventCreate(&r.ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&r.ev1);
  if (e == cudaSuccess) e = cudaEventRecord(r.ev0, st);
  if (e == cudaSuccess) e = dev_malloc_async((void **)&r.dev, r.state_bytes, st);
  if (e != cudaSuccess) {
    r.dev = nullptr;
    return cuda_error(e, "server pool allocation");
  }
  size_t off = 0;
  auto take = [&](size_t b) { char *p = r.dev + off; off += (b + 255) & ~(size_t)255; return p; };
  CellArgs &a = r.args;
  a = CellArgs{};
  a.n_cells = n;
  a.ld = n;
  a.dt = r.dt;
  a.x = (double *)take(sizeof(double) * S * n);
  a.T = r.T ? (double *)take(sizeof(double) * n) : nullptr;
  a.nd = r.nd ? (const double *)take(sizeof(double) * n) : nullptr;
  a.status = (int32_t *)take(sizeof(int32_t) * n);
  mc_status ms = MC_OK;
  e = cudaMemcpy2DAsync(a.x, sizeof(double) * n, r.x, sizeof(double) * r.ld, sizeof(double) * n, S,
                        cudaMemcpyDefault, st);
  if (e == cudaSuccess && r.T) e = cudaMemcpyAsync(a.T, r.T, sizeof(double) * n, cudaMemcpyDefault, st);
  if (e == cudaSuccess && r.nd) e = cudaMemcpyAsync((void *)a.nd, r.nd, sizeof(double) * n, cudaMemcpyDefault, st);
  if (e != cudaSuccess) ms = cuda_error(e, "server copy in");
  if (ms == MC_OK) ms = burn_device(r.net, r.opts, a, st);
  if (ms == MC_OK) {
    e = cudaMemsetAsync(s->fail_dev + r.stream, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) {
      const int blocks = (int)std::min<int64_t>(1184, (n + 255) / 256);
      k_count_failed<<<blocks, 256, 0, st>>>(a.status, n, s->fail_dev + r.stream);
      e = cudaGetLastError();
      count_launch(1);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->fail_host + r.stream, s->fail_dev + r.stream, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(r.ev1, st);
    if (e != cudaSuccess) ms = cuda_error(e, "server burn");
  }
  if (ms != MC_OK) {
    cudaFreeAsync(r.dev, st);
    r.dev = nullptr;
  }
  return ms;
}

// The results of a request whose GPU work has ended: copies out (pageable
// host destinations make these synchronous, now only for the copy itself),
// the pool memory back, and the stream drained of the copies.
mc_status finish_copies(mc_server *s, Request &r) {
  const cudaStream_t st = s->streams[r.stream];
  const int64_t n = r.n;
  const int S = r.net->S;
  const CellArgs &a = r.args;
  cudaError_t e = cudaMemcpy2DAsync(r.x, sizeof(double) * r.ld, a.x, sizeof(double) * n, sizeof(double) * n, S,
                                    cudaMemcpyDefault, st);
  if (e == cudaSuccess && r.T) e = cudaMemcpyAsync(r.T, a.T, sizeof(double) * n, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r.status, a.status, sizeof(int32_t) * n, cudaMemcpyDefault, st);
  cudaFreeAsync(r.dev, st);
  r.dev = nullptr;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? MC_OK : cuda_error(e, "server copy out");
}

double gpu_seconds(cudaEvent_t ref, cudaEvent_t ev) {
  float ms = 0.f;
  return cudaEventElapsedTime(&ms, ref, ev) == cudaSuccess ? ms * 1e-3 : -1.0;
}

void finish_request(mc_server *s, Request &r) {
  if (r.ev0) cudaEventDestroy(r.ev0);
  if (r.ev1) cudaEventDestroy(r.ev1);
  r.ev0 = r.ev1 = nullptr;
  s->used -= r.state_bytes;
  s->stream_busy[r.stream] = 0;
  s->outstanding -= 1;
  s->done_cv.notify_all();
}

void server_loop(mc_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // admissions: FIFO while the budget and a free stream allow
    while (!s->pending.empty()) {
      Request &r = s->reqs[s->pending.front()];
      // the free stream whose scratch already covers the most of this burn
      int k = -1;
      for (int i = 0; i < (int)s->streams.size(); ++i) {
        if (s->stream_busy[i]) continue;
        if (k < 0 || std::min(s->stream_scratch[i], r.scratch_need) > std::min(s->stream_scratch[k], r.scratch_need))
          k = i;
      }
      if (k < 0) break;
      const size_t grow = r.scratch_need > s->stream_scratch[k] ? r.scratch_need - s->stream_scratch[k] : 0;
      if (s->used + r.state_bytes + s->scratch_total + grow > s->budget) break;
      s->pending.pop_front();
      s->stream_busy[k] = 1;
      s->used += r.state_bytes;
      s->scratch_total += grow;
      s->stream_scratch[k] += grow;
      r.stream = k;
      r.t_admit = s->now();
      lk.unlock();
      const mc_status ms = start_request(s, r);
      const std::string msg = ms == MC_OK ? std::string() : std::string(mc_last_error());
      lk.lock();
      if (ms != MC_OK) {
        r.state = ms;
        r.err = msg;
        r.t_done = s->now();
        finish_request(s, r);
        continue;
      }
      s->inflight.push_back(r.id);
    }
    // completions
    for (size_t i = 0; i < s->inflight.size();) {
      Request &r = s->reqs[s->inflight[i]];
      const cudaError_t q = cudaEventQuery(r.ev1);
      if (q == cudaErrorNotReady) { ++i; continue; }
      if (q == cudaSuccess) {
        r.n_failed = (int32_t)s->fail_host[r.stream];
        r.gpu_start = gpu_seconds(s->ref, r.ev0);
        r.gpu_end = gpu_seconds(s->ref, r.ev1);
        lk.unlock();
        const mc_status ms = finish_copies(s, r);
        const std::string msg = ms == MC_OK ? std::string() : std::string(mc_last_error());
        lk.lock();
        r.state = ms;
        r.err = msg;
      } else {
        r.state = MC_E_CUDA;
        r.err = cudaGetErrorString(q);
      }
      r.t_done = s->now();
      finish_request(s, r);
      s->inflight.erase(s->inflight.begin() + i);
    }
    if (s->stop && s->pending.empty() && s->inflight.empty()) break;
    if (s->inflight.empty() && (s->pending.empty() || s->stop))
      s->cv.wait_for(lk, std::chrono::milliseconds(50));
    else
      s->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

void release(mc_server *s) {
  for (cudaStream_t q : s->streams) cudaStreamDestroy(q);
  if (s->ref) cudaEventDestroy(s->ref);
  cudaFree(s->fail_dev);
  cudaFreeHost(s->fail_host);
  delete s;
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
  e = dev_malloc((void **)&s->fail_dev, sizeof(uint32_t) * kStreams);
  if (e == cudaSuccess) e = host_malloc_pinned((void **)&s->fail_host, sizeof(uint32_t) * kStreams);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ref);
  if (e == cudaSuccess) e = cudaEventRecord(s->ref, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(s->ref);
  for (int i = 0; e == cudaSuccess && i < kStreams; ++i) {
    cudaStream_t q;
    e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      s->streams.push_back(q);
      s->stream_busy.push_back(0);
      s->stream_scratch.push_back(0);
    }
  }
  if (e != cudaSuccess) {
    release(s);
    return cuda_error(e, "mc_server_create");
  }
  s->loop = std::thread(server_loop, s);
  *out = s;
  return MC_OK;
}

extern "C" mc_status mc_request_bytes(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                                      uint64_t *state_bytes, uint64_t *scratch_bytes) {
  if (!net || n_cells <= 0) return set_error(MC_E_INVALID, "mc_request_bytes: bad arguments");
  mc_burn_opts o;
  mc_status st = check_opts(opts, &o);
  if (st != MC_OK) return st;
  if (state_bytes) *state_bytes = request_bytes(net, n_cells);
  if (scratch_bytes) *scratch_bytes = burn_scratch_bytes(net, o, n_cells);
  return MC_OK;
}

extern "C" mc_status mc_request_submit(mc_server *s, const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                                       double dt, double *x, int64_t ld, double *T, const double *ndens,
                                       int32_t *status, uint64_t *req_id) {
  if (!s || !net || !req_id) return set_error(MC_E_INVALID, "mc_request_submit: null argument");
  if (n_cells <= 0 || ld < n_cells || n_cells > (int64_t)INT32_MAX || !x || !status || (net->energy && !T))
    return set_error(MC_E_INVALID, "mc_request_submit: bad cells");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(MC_E_INVALID, "mc_request_submit: dt must be positive");
  if (net->device != s->device) return set_error(MC_E_INVALID, "mc_request_submit: network on another device");
  mc_burn_opts o = s->opts;
  if (opts) {
    mc_status st = check_opts(opts, &o);
    if (st != MC_OK) return st;
  }
  const size_t b = request_bytes(net, n_cells), sc = burn_scratch_bytes(net, o, n_cells);
  if (b + sc > s->budget)
    return set_error(MC_E_BUDGET, "request of %zu bytes (state %zu, scratch %zu) exceeds the budget of %llu", b + sc,
                     b, sc, (unsigned long long)s->budget);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return set_error(MC_E_BUSY, "server is shutting down");
  Request r;
  r.id = s->next_id++;
  r.net = net;
  r.opts = o;
  r.n = n_cells;
  r.ld = ld;
  r.dt = dt;
  r.x = x;
  r.T = T;
  r.nd = ndens;
  r.status = status;
  r.state_bytes = b;
  r.scratch_need = sc;
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
    info->gpu_start = r.gpu_start;
    info->gpu_end = r.gpu_end;
  }
  if (r.state < 0) return set_error(r.state, "request %llu failed: %s", (unsigned long long)req_id, r.err.c_str());
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
  for (cudaStream_t q : s->streams) cudaStreamSynchronize(q);
  release(s);
  return r;
}
