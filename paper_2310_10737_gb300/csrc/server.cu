// server.cu -- the serving loop: continuous batching of product-code decode
// requests (the decoder of Sec. VI run as a service).
//
// A request is a batch of square product frames of one registered code.  Its
// frames occupy slots of that code's device pool (channel LLRs, L_E state,
// hard decisions, counters: everything stays resident between half
// iterations).  One worker thread drives every pool independently: when a
// pool's previous launch has finished it retires the frames that stopped
// (their request completes when its last frame does: the outputs are copied
// to the caller's host buffers), admits waiting requests of that code in
// arrival order while free slots last (their LLRs are copied in), and
// launches the batched decoder over every resident frame for at most
// `epoch_halves` half iterations, frames that need more being parked in
// place.  The pools run on their own streams, so the codes' launches overlap
// on the GPU; a request that arrives while others are decoding joins at its
// pool's next epoch.  Each frame runs exactly the arithmetic of
// product_decode_persistent, so its results do not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "launch.h"
#include "sogrand.h"

// Internal helpers of abi.cu.
namespace sgi {
sg::DevCode dev_code_of(const sogrand_code *c);
int code_n(const sogrand_code *c);
int code_nm(const sogrand_code *c);
int code_m(const sogrand_code *c);
int ensure_code_cap(sogrand_code *c, int64_t cap);
cudaError_t launch_persistent_for(const sogrand_code *c, const sg::SisoParams &P, const sg::ProductArgs &a,
                                  cudaStream_t s);
int sm_count_of_device();
sg::SisoParams siso_params_of(int L, int64_t cap, float thr);
int32_t queue_wait_us();
int dp_slice(const sogrand_code *c);
int code_dp_global(const sogrand_code *c);
}  // namespace sgi

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t ticket = 0;
  int pool = 0;
  int64_t frames = 0;
  const float *llr = nullptr;  // host [frames][n][n]
  uint8_t *bits = nullptr;     // host outputs
  int32_t *half_iters = nullptr;
  uint8_t *status = nullptr;
  int64_t *queries = nullptr;
  int32_t first = -1;  // the request's frames occupy slots first .. first + frames - 1
  int64_t remaining = 0;
  double t_submit = 0, t_done = 0;
  int state = 0;  // 0 waiting, 1 resident, 2 done
  int rc = SOGRAND_OK;
};

struct Pool {
  sogrand_code *code = nullptr;
  int n = 0, nm = 0;
  int64_t slots = 0;
  char *mem = nullptr;
  float *llr = nullptr, *le = nullptr;
  uint64_t *hb = nullptr;
  uint8_t *bits = nullptr, *status = nullptr;
  int32_t *half_iters = nullptr, *hmax = nullptr, *half_cur = nullptr, *done_words = nullptr, *bad = nullptr;
  int32_t *half_stop = nullptr, *queue = nullptr, *ctrl = nullptr, *list = nullptr;
  unsigned char *dp_area = nullptr;  // the launch blocks' remaining-mass areas
  int dp_stride = 0, dp_blocks = 0;
  int64_t *queries = nullptr, *par_queries = nullptr;
  int32_t *h_list = nullptr;   // pinned [slots]
  uint8_t *h_status = nullptr; // pinned [slots]
  int32_t *h_ctrl = nullptr;   // pinned [4]
  cudaStream_t stream = nullptr;
  std::map<int32_t, int32_t> free_runs;  // free slot ranges: first -> length (coalesced)
  int64_t free_count = 0;
  std::vector<int32_t> active;  // resident frames: slot, or -(slot + 1) for one admitted since the last launch
  std::vector<Request *> owner;  // [slots]
  std::deque<Request *> waiting;
  bool running = false;
  int64_t launched_words = 0;
  // requests whose outputs are being copied out: done once the event has fired
  std::vector<std::pair<cudaEvent_t, std::vector<Request *>>> draining;
  std::vector<cudaEvent_t> spare_events;

  // first-fit allocation of `len` consecutive slots; -1 if no run is long enough
  int32_t alloc(int32_t len) {
    for (auto it = free_runs.begin(); it != free_runs.end(); ++it) {
      if (it->second < len) continue;
      const int32_t first = it->first, rest = it->second - len;
      free_runs.erase(it);
      if (rest > 0) free_runs[first + len] = rest;
      free_count -= len;
      return first;
    }
    return -1;
  }
  void release(int32_t first, int32_t len) {
    auto it = free_runs.emplace(first, len).first;
    free_count += len;
    auto nx = std::next(it);
    if (nx != free_runs.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_runs.erase(nx);
    }
    if (it != free_runs.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_runs.erase(it);
      }
    }
  }
};

}  // namespace

struct sogrand_server {
  int device = 0;
  int L = 4;
  int64_t cap = 10000;
  float thr = 0.f, alpha = 0.5f;
  int max_iter = 20, epoch_halves = 2;
  std::vector<std::unique_ptr<Pool>> pools;
  std::mutex mu;
  std::condition_variable cv;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  bool stop = false;
  int error = SOGRAND_OK;
  std::thread worker;
  // statistics
  int64_t launches = 0, frames_done = 0, requests_done = 0;
  double busy_since = 0;
};

namespace {

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Carve one pool's device arrays out of `mem` (or just count the bytes).
size_t carve(Pool &p, int max_iter, char *mem) {
  size_t off = 0;
  auto take = [&](size_t b) {
    char *r = mem ? mem + off : nullptr;
    off += round256(b);
    return r;
  };
  const size_t S = (size_t)p.slots;
  p.llr = (float *)take(S * p.n * p.n * sizeof(float));
  p.le = (float *)take(S * p.n * p.n * sizeof(float));
  p.hb = (uint64_t *)take(S * p.n * p.nm * 8);
  p.bits = (uint8_t *)take(S * (((size_t)p.n * p.n + 7) / 8));
  p.status = (uint8_t *)take(S);
  p.half_iters = (int32_t *)take(S * 4);
  p.hmax = (int32_t *)take(S * 4);
  p.half_cur = (int32_t *)take(S * 4);
  p.done_words = (int32_t *)take(S * 4);
  p.bad = (int32_t *)take(S * 4);
  p.half_stop = (int32_t *)take(S * 4);
  p.list = (int32_t *)take(S * 4);
  p.queries = (int64_t *)take(S * 8);
  p.par_queries = (int64_t *)take(S * 8);
  p.queue = (int32_t *)take(S * 2 * max_iter * 4);
  p.ctrl = (int32_t *)take(32);
  p.dp_area = (unsigned char *)take((size_t)p.dp_blocks * p.dp_stride);
  return off;
}

// Requests whose output copies have completed are reported done.
void finish_drained(sogrand_server *sv, Pool &p, bool wait) {
  std::vector<Request *> done;
  for (size_t i = 0; i < p.draining.size();) {
    cudaEvent_t ev = p.draining[i].first;
    const cudaError_t q = !ev ? cudaSuccess : (wait ? cudaEventSynchronize(ev) : cudaEventQuery(ev));
    if (q == cudaErrorNotReady) {
      i++;
      continue;
    }
    for (Request *r : p.draining[i].second) {
      if (q != cudaSuccess) r->rc = SOGRAND_ECUDA;
      done.push_back(r);
    }
    if (ev) p.spare_events.push_back(ev);
    p.draining.erase(p.draining.begin() + i);
  }
  if (done.empty()) return;
  const double t = now_ms();
  std::lock_guard<std::mutex> g(sv->mu);
  for (Request *r : done) {
    r->t_done = t;
    r->state = 2;
    sv->frames_done += r->frames;
    sv->requests_done++;
  }
  sv->cv.notify_all();
}

// Retire the frames of pool p that stopped in its last launch.  A request
// whose last frame stopped has its outputs (contiguous slots) copied to its
// host buffers on the pool's stream; its slots are free at once (later work
// on the stream runs after the copies), and it is reported done when the
// copies have completed.
void retire(sogrand_server *sv, Pool &p) {
  std::vector<int32_t> still;
  std::vector<Request *> completed;
  still.reserve(p.active.size());
  const bool failed = p.h_ctrl[3] != 0;
  for (int32_t e : p.active) {
    const int32_t slot = e < 0 ? -e - 1 : e;
    if (!failed && p.h_status[slot] == 255) {
      still.push_back(slot);
      continue;
    }
    Request *r = p.owner[slot];
    if (r && --r->remaining == 0) completed.push_back(r);
  }
  p.active.swap(still);
  if (completed.empty()) return;
  cudaError_t e = cudaSuccess;
  const size_t nb = ((size_t)p.n * p.n + 7) / 8;
  for (Request *r : completed) {
    const size_t F = (size_t)r->frames, f0 = (size_t)r->first;
    e = cudaMemcpyAsync(r->bits, p.bits + f0 * nb, F * nb, cudaMemcpyDeviceToHost, p.stream);
    if (e == cudaSuccess && r->half_iters)
      e = cudaMemcpyAsync(r->half_iters, p.half_iters + f0, F * 4, cudaMemcpyDeviceToHost, p.stream);
    if (e == cudaSuccess && r->status)
      e = cudaMemcpyAsync(r->status, p.status + f0, F, cudaMemcpyDeviceToHost, p.stream);
    if (e == cudaSuccess && r->queries)
      e = cudaMemcpyAsync(r->queries, p.queries + f0, F * 8, cudaMemcpyDeviceToHost, p.stream);
    r->rc = failed ? SOGRAND_ETIMEOUT : (e == cudaSuccess ? SOGRAND_OK : SOGRAND_ECUDA);
    for (int64_t j = 0; j < r->frames; j++) p.owner[r->first + j] = nullptr;
  }
  cudaEvent_t ev = nullptr;
  if (!p.spare_events.empty()) {
    ev = p.spare_events.back();
    p.spare_events.pop_back();
  } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    ev = nullptr;
  }
  if (ev && cudaEventRecord(ev, p.stream) == cudaSuccess) {
    p.draining.emplace_back(ev, completed);
  } else {  // no event: wait for the copies here
    if (cudaStreamSynchronize(p.stream) != cudaSuccess)
      for (Request *r : completed) r->rc = SOGRAND_ECUDA;
    if (ev) p.spare_events.push_back(ev);
    p.draining.emplace_back(nullptr, completed);
  }
  std::lock_guard<std::mutex> g(sv->mu);
  for (Request *r : completed) p.release(r->first, (int32_t)r->frames);
}

// Admit waiting requests of pool p in arrival order while a run of free
// slots is long enough; one copy of each request's LLRs into its slots.
void admit(sogrand_server *sv, Pool &p) {
  std::vector<Request *> in;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    while (!p.waiting.empty()) {
      Request *r = p.waiting.front();
      const int32_t first = p.alloc((int32_t)r->frames);
      if (first < 0) break;
      p.waiting.pop_front();
      r->first = first;
      r->remaining = r->frames;
      r->state = 1;
      in.push_back(r);
    }
  }
  const size_t fb = (size_t)p.n * p.n * sizeof(float);
  for (Request *r : in) {
    cudaMemcpyAsync((char *)p.llr + (size_t)r->first * fb, r->llr, (size_t)r->frames * fb, cudaMemcpyHostToDevice,
                    p.stream);
    for (int64_t j = 0; j < r->frames; j++) {
      p.owner[r->first + j] = r;
      p.active.push_back(-(r->first + (int32_t)j) - 1);
    }
  }
}

// Launch the batched decoder over every resident frame of pool p.
cudaError_t launch(sogrand_server *sv, Pool &p, int64_t total_words) {
  const int64_t F = (int64_t)p.active.size();
  std::memcpy(p.h_list, p.active.data(), F * sizeof(int32_t));
  cudaError_t e = cudaMemcpyAsync(p.list, p.h_list, F * sizeof(int32_t), cudaMemcpyHostToDevice, p.stream);
  sg::ProductArgs a{};
  a.n_frames = F;
  a.nr = a.nc = a.hbw = p.n;
  a.llr_ch = p.llr;
  a.alpha = sv->alpha;
  a.max_half = 2 * sv->max_iter;
  a.le = p.le;
  a.hb = p.hb;
  a.hmax = p.hmax;
  a.bits = p.bits;
  a.half_iters = p.half_iters;
  a.status = p.status;
  a.queries = p.queries;
  a.par_queries = p.par_queries;
  a.queue = p.queue;
  a.half_cur = p.half_cur;
  a.done_words = p.done_words;
  a.bad = p.bad;
  a.ctrl = p.ctrl;
  a.max_spin = sgi::queue_wait_us();
  a.dp_area = sgi::code_dp_global(p.code) ? p.dp_area : nullptr;
  a.dp_stride = p.dp_stride;
  a.dp_blocks = p.dp_blocks;
  a.half_stop = p.half_stop;
  a.frame_list = p.list;
  a.epoch_halves = sv->epoch_halves;
  // the GPU is shared by the pools' concurrent launches in proportion to their words
  const int64_t words = F * p.n;
  const int64_t full = (int64_t)sgi::sm_count_of_device() * sg::MAX_BLOCKS_PER_SM;
  a.grid_cap = (int)std::max<int64_t>(full / 8, total_words > 0 ? (full * words + total_words - 1) / total_words : full);
  const sg::SisoParams P = sgi::siso_params_of(sv->L, sv->cap, sv->thr);
  if (e == cudaSuccess) e = sgi::launch_persistent_for(p.code, P, a, p.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.h_status, p.status, p.slots, cudaMemcpyDeviceToHost, p.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.h_ctrl, p.ctrl, 16, cudaMemcpyDeviceToHost, p.stream);
  p.launched_words = words;
  return e;
}

void worker_main(sogrand_server *sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    bool progress = false;
    for (auto &pp : sv->pools) {
      Pool &p = *pp;
      if (!p.draining.empty()) {
        const size_t before = p.draining.size();
        finish_drained(sv, p, false);
        progress = progress || p.draining.size() != before;
      }
      if (p.running) {
        const cudaError_t q = cudaStreamQuery(p.stream);
        if (q == cudaErrorNotReady) continue;
        p.running = false;
        progress = true;
        if (q != cudaSuccess) {
          std::lock_guard<std::mutex> g(sv->mu);
          sv->error = SOGRAND_ECUDA;
        }
        retire(sv, p);
      }
      admit(sv, p);
    }
    // launch every idle pool with resident frames; the GPU is split by words
    int64_t total_words = 0;
    for (auto &pp : sv->pools) total_words += pp->running ? pp->launched_words : (int64_t)pp->active.size() * pp->n;
    for (auto &pp : sv->pools) {
      Pool &p = *pp;
      if (p.running || p.active.empty()) continue;
      if (launch(sv, p, total_words) != cudaSuccess) {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->error = SOGRAND_ECUDA;
      }
      p.running = true;
      progress = true;
      std::lock_guard<std::mutex> g(sv->mu);
      sv->launches++;
    }
    if (progress) continue;
    std::unique_lock<std::mutex> lk(sv->mu);
    bool busy = false, waiting = false;
    for (auto &pp : sv->pools) {
      busy = busy || pp->running || !pp->active.empty() || !pp->draining.empty();
      waiting = waiting || !pp->waiting.empty();
    }
    if (sv->stop && !busy && !waiting) return;
    if (busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));  // a launch is in flight
    } else {
      sv->cv.wait_for(lk, std::chrono::milliseconds(2));  // idle until a submission
    }
  }
}

}  // namespace

extern "C" {

int sogrand_server_create(int n_codes, sogrand_code *const *codes, const int64_t *slots, int L, int64_t query_cap,
                          float thr, float alpha, int max_iter, int epoch_halves, sogrand_server **out) {
  if (!out || n_codes < 1 || n_codes > 16 || !codes || !slots || L < 1 || L > sg::LMAX || query_cap < 1 ||
      query_cap > (int64_t(1) << 24) || !(thr >= 0.f && thr < 1.f) || !(alpha > 0.f && alpha < 1e6f) ||
      max_iter < 1 || max_iter > 1000 || epoch_halves < 1 || epoch_halves > 2 * max_iter)
    return SOGRAND_EINVAL;
  for (int i = 0; i < n_codes; i++) {
    if (!codes[i] || slots[i] < 1 || slots[i] > (int64_t(1) << 24)) return SOGRAND_EINVAL;
    const int n = sgi::code_n(codes[i]);
    if (n - 1 < 63 && query_cap >= (int64_t(1) << (n - 1))) return SOGRAND_EINVAL;
    if (slots[i] * 2 * (int64_t)max_iter * n >= (int64_t(1) << 31) - (int64_t(1) << 22)) return SOGRAND_EINVAL;
  }
  std::unique_ptr<sogrand_server> sv(new (std::nothrow) sogrand_server());
  if (!sv) return SOGRAND_ENOMEM;
  cudaGetDevice(&sv->device);
  sv->L = L;
  sv->cap = query_cap;
  sv->thr = thr;
  sv->alpha = alpha;
  sv->max_iter = max_iter;
  sv->epoch_halves = epoch_halves;
  int rc = SOGRAND_OK;
  for (int i = 0; i < n_codes && rc == SOGRAND_OK; i++) {
    rc = sgi::ensure_code_cap(codes[i], query_cap);
    if (rc != SOGRAND_OK) break;
    std::unique_ptr<Pool> p(new Pool());
    p->code = codes[i];
    p->n = sgi::code_n(codes[i]);
    p->nm = sgi::code_nm(codes[i]);
    p->slots = slots[i];
    p->dp_stride = sgi::dp_slice(codes[i]);
    p->dp_blocks = sgi::sm_count_of_device() * sg::MAX_BLOCKS_PER_SM;  // a slice for every block a launch can have resident
    const size_t bytes = carve(*p, max_iter, nullptr);
    if (cudaMalloc(&p->mem, bytes) != cudaSuccess) {
      rc = SOGRAND_ENOMEM;
      break;
    }
    carve(*p, max_iter, p->mem);
    if (cudaMallocHost(&p->h_list, p->slots * 4) != cudaSuccess ||
        cudaMallocHost(&p->h_status, p->slots) != cudaSuccess || cudaMallocHost(&p->h_ctrl, 16) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = SOGRAND_ECUDA;
    }
    p->free_runs[0] = (int32_t)p->slots;
    p->free_count = p->slots;
    p->owner.assign(p->slots, nullptr);
    sv->pools.push_back(std::move(p));
  }
  if (rc != SOGRAND_OK) {
    sogrand_server_destroy(sv.release());
    return rc;
  }
  sogrand_server *raw = sv.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return SOGRAND_OK;
}

int sogrand_server_submit(sogrand_server *sv, int code_index, int64_t n_frames, const float *llr, uint8_t *bits,
                          int32_t *half_iters, uint8_t *status, int64_t *queries, int64_t *ticket) {
  if (!sv || !ticket || code_index < 0 || code_index >= (int)sv->pools.size() || n_frames < 1 || !llr || !bits)
    return SOGRAND_EINVAL;
  Pool &p = *sv->pools[code_index];
  if (n_frames > p.slots) return SOGRAND_EINVAL;  // could never be admitted
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return SOGRAND_ENOMEM;
  r->pool = code_index;
  r->frames = n_frames;
  r->llr = llr;
  r->bits = bits;
  r->half_iters = half_iters;
  r->status = status;
  r->queries = queries;
  std::lock_guard<std::mutex> g(sv->mu);
  if (sv->stop) return SOGRAND_EINVAL;
  if (sv->error != SOGRAND_OK) return sv->error;
  r->t_submit = now_ms();
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  p.waiting.push_back(r.get());
  sv->reqs[r->ticket] = std::move(r);
  sv->cv.notify_all();
  return SOGRAND_OK;
}

int sogrand_server_wait(sogrand_server *sv, int64_t ticket, int timeout_ms, int *done, double *latency_ms) {
  if (!sv || !done) return SOGRAND_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return SOGRAND_EINVAL;
  Request *r = it->second.get();
  if (timeout_ms > 0)
    sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [r] { return r->state == 2; });
  *done = r->state == 2;
  if (!*done) return SOGRAND_OK;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  const int rc = r->rc;
  sv->reqs.erase(it);  // a completed request is reported once
  return rc;
}

int sogrand_server_stats(sogrand_server *sv, int64_t *launches, int64_t *frames_done, int64_t *requests_done,
                         int64_t *frames_resident, int64_t *requests_waiting) {
  if (!sv) return SOGRAND_EINVAL;
  std::lock_guard<std::mutex> g(sv->mu);
  int64_t res = 0, wait = 0;
  for (auto &p : sv->pools) {
    res += p->slots - p->free_count;
    wait += (int64_t)p->waiting.size();
  }
  if (launches) *launches = sv->launches;
  if (frames_done) *frames_done = sv->frames_done;
  if (requests_done) *requests_done = sv->requests_done;
  if (frames_resident) *frames_resident = res;
  if (requests_waiting) *requests_waiting = wait;
  return sv->error;
}

int sogrand_server_destroy(sogrand_server *sv) {
  if (!sv) return SOGRAND_EINVAL;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();  // drains every submitted request first
  for (auto &p : sv->pools) {
    if (p->stream) {
      cudaStreamSynchronize(p->stream);
      cudaStreamDestroy(p->stream);
    }
    for (auto &d : p->draining)
      if (d.first) cudaEventDestroy(d.first);
    for (cudaEvent_t ev : p->spare_events) cudaEventDestroy(ev);
    if (p->mem) cudaFree(p->mem);
    if (p->h_list) cudaFreeHost(p->h_list);
    if (p->h_status) cudaFreeHost(p->h_status);
    if (p->h_ctrl) cudaFreeHost(p->h_ctrl);
  }
  const int err = sv->error;
  delete sv;
  return err;
}

}  // extern "C"
