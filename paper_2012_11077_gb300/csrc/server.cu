// Serving runtime: continuous batching of radar frames from many sources.
//
// Frames arrive at any time (rcfar_server_submit), from host memory or
// already in device memory (a device frame is read in place and its
// decisions written to the caller's device buffer: no staging copies, only
// its batch workspace counts against the budget). A
// scheduler thread takes them in arrival order into a batch for a free slot
// while they fit that slot's share of the device-memory budget (workspace of
// the rcfar_run_batch chain, the raw inputs, the decisions) and enqueues on
// the slot's own stream: the host->device copies, the batch chain, the
// device->host copy of the decisions and an event. Up to `slots` batches are
// on the GPU at once, so frames that arrive while others run are admitted as
// soon as a slot and its memory free up and their copies and kernels overlap
// the batches already in flight. A completion thread waits for the slots'
// events in launch order, copies each frame's decisions to the caller's
// buffer and publishes its completion (arrival, admission and completion
// times).
//
// The chain itself is rcfar_run_batch: a frame's results do not depend on the
// other frames of its batch, so each decision equals the frame's decision run
// alone. Every slot owns one rcfar handle; the handle keeps the twiddle
// tables of every (N, band) it has seen on the device.
#include "rcfar_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

namespace {

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t clock_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Pending {
  rcfar_request r;
  int C = 0;            // stored band columns of the frame's decisions
  size_t ws = 0;        // rcfar_run_batch workspace bytes
  size_t in_b = 0;      // raw frame bytes on the device (packed rows; 0 for a device frame)
  size_t det_b = 0;     // decision bytes (packed rows; 0 for a device frame)
  bool device = false;  // x and det are device memory: no copies
};

struct Slot {
  rcfar_handle h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* dev_io = nullptr;          // inputs, then decisions, of the batch in flight
  unsigned char* host_det = nullptr;  // pinned staging of the decisions
  size_t ws_cap = 0, in_cap = 0, det_cap = 0;
  std::vector<Pending> batch;
  std::vector<size_t> in_off, det_off;
  std::vector<rcfar_frame_desc> descs;
  int64_t admit_ns = 0;
  rcfar_status launch_status = RCFAR_OK;
  bool busy = false;
};

}  // namespace

struct rcfar_server_s {
  rcfar_server_config cfg{};
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_sched, cv_comp, cv_poll;
  std::deque<Pending> pending;
  std::deque<int> inflight;  // slot indices in launch order
  std::deque<rcfar_completion> done;
  bool closing = false;      // destroy has begun: admit nothing new, finish the rest
  bool sched_exited = false;
  std::thread sched, comp;
  rcfar_server_stats stats{};
  int64_t inflight_frames = 0;

  void scheduler();
  void completer();
  void launch(int si);
};

void rcfar_server_s::launch(int si) {
  Slot& S = slots[si];
  const int n = (int)S.batch.size();
  cudaSetDevice(cfg.device);
  rcfar_status st = RCFAR_OK;
  S.descs.resize(n);
  bool any_host = false;
  for (int i = 0; i < n; ++i) {
    const rcfar_request& r = S.batch[i].r;
    rcfar_frame_desc& d = S.descs[i];
    std::memset(&d, 0, sizeof(d));
    d.M = r.M;
    d.N = r.N;
    d.window = r.window;
    if (S.batch[i].device) {  // read in place, decisions straight to the caller's buffer
      d.x = r.x;
      d.ldx = r.ldx;
      d.det = r.det;
      d.ld_det = r.ld_det;
      continue;
    }
    any_host = true;
    float* xin = reinterpret_cast<float*>(S.dev_io + S.in_off[i]);
    // packed on the device in the frame's own layout (rows of N, or of M for trace-major frames)
    const bool tm = cfg.params.x_layout == RCFAR_X_TRACE_MAJOR;
    const int width = tm ? r.M : r.N, height = tm ? r.N : r.M;
    // a frame stored without row padding goes as one linear copy: pitched copies of rows of
    // 1-16 KB reached about 120 GB/s on this path, linear ones about 187 GB/s
    const cudaError_t ce =
        r.ldx == (int64_t)width
            ? cudaMemcpyAsync(xin, r.x, (size_t)width * (size_t)height * sizeof(float), cudaMemcpyHostToDevice,
                              S.stream)
            : cudaMemcpy2DAsync(xin, (size_t)width * sizeof(float), r.x, (size_t)r.ldx * sizeof(float),
                                (size_t)width * sizeof(float), (size_t)height, cudaMemcpyHostToDevice, S.stream);
    if (ce != cudaSuccess) st = RCFAR_ERR_CUDA;
    d.x = xin;
    d.ldx = width;
    d.det = reinterpret_cast<uint8_t*>(S.dev_io + S.in_cap + S.det_off[i]);
    d.ld_det = S.batch[i].C;
  }
  if (st == RCFAR_OK) st = rcfar_run_batch(S.h, S.descs.data(), n, &cfg.params, (rcfar_stream)S.stream);
  if (st == RCFAR_OK && any_host) {
    size_t total = 0;
    for (int i = 0; i < n; ++i)
      if (!S.batch[i].device) total = std::max(total, S.det_off[i] + (size_t)S.batch[i].r.M * S.batch[i].C);
    // decisions are packed back to back: one copy for the batch
    if (cudaMemcpyAsync(S.host_det, S.dev_io + S.in_cap, total, cudaMemcpyDeviceToHost, S.stream) != cudaSuccess)
      st = RCFAR_ERR_CUDA;
  }
  if (cudaEventRecord(S.done, S.stream) != cudaSuccess && st == RCFAR_OK) st = RCFAR_ERR_CUDA;
  S.launch_status = st;
}

void rcfar_server_s::scheduler() {
  cudaSetDevice(cfg.device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    int si = -1;
    cv_sched.wait(lk, [&] {
      if (pending.empty()) return closing;
      for (int i = 0; i < (int)slots.size(); ++i)
        if (!slots[i].busy) return true;
      return false;
    });
    if (pending.empty()) break;  // closing and nothing left to admit
    for (int i = 0; i < (int)slots.size(); ++i)
      if (!slots[i].busy) {
        si = i;
        break;
      }
    Slot& S = slots[si];
    S.batch.clear();
    S.in_off.clear();
    S.det_off.clear();
    size_t ws = 0, in = 0, det = 0;
    // arrival order: the batch closes at the first frame that does not fit
    while (!pending.empty() && (int)S.batch.size() < cfg.max_batch_frames) {
      const Pending& q = pending.front();
      if (ws + q.ws > S.ws_cap || in + q.in_b > S.in_cap || det + q.det_b > S.det_cap) break;
      S.in_off.push_back(in);
      S.det_off.push_back(det);
      ws += q.ws;
      in += q.in_b;
      det += q.det_b;
      S.batch.push_back(q);
      pending.pop_front();
    }
    S.busy = true;
    S.admit_ns = clock_ns();
    inflight_frames += (int64_t)S.batch.size();
    stats.max_inflight_frames = std::max(stats.max_inflight_frames, inflight_frames);
    stats.max_batch_frames_seen = std::max<int64_t>(stats.max_batch_frames_seen, (int64_t)S.batch.size());
    stats.batches += 1;
    lk.unlock();
    launch(si);
    lk.lock();
    inflight.push_back(si);
    cv_comp.notify_one();
  }
  sched_exited = true;
  cv_comp.notify_one();
}

void rcfar_server_s::completer() {
  cudaSetDevice(cfg.device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv_comp.wait(lk, [&] { return !inflight.empty() || sched_exited; });
    if (inflight.empty()) break;  // the scheduler has exited and everything is done
    const int si = inflight.front();
    lk.unlock();
    Slot& S = slots[si];
    rcfar_status st = S.launch_status;
    if (cudaEventSynchronize(S.done) != cudaSuccess && st == RCFAR_OK) st = RCFAR_ERR_CUDA;
    if (st == RCFAR_OK) {
      const rcfar_status dev = rcfar_get_error(S.h, (rcfar_stream)S.stream);
      if (dev != RCFAR_OK) st = dev;
    }
    const int64_t t = clock_ns();
    std::vector<rcfar_completion> out(S.batch.size());
    for (size_t i = 0; i < S.batch.size(); ++i) {
      const Pending& q = S.batch[i];
      if (st == RCFAR_OK && !q.device) {
        const unsigned char* src = S.host_det + S.det_off[i];
        if (q.r.ld_det == q.C) {
          std::memcpy(q.r.det, src, (size_t)q.r.M * q.C);
        } else {
          for (int m = 0; m < q.r.M; ++m) std::memcpy(q.r.det + (size_t)m * q.r.ld_det, src + (size_t)m * q.C, q.C);
        }
      }
      rcfar_completion& c = out[i];
      std::memset(&c, 0, sizeof(c));
      c.tag = q.r.tag;
      c.status = st;
      c.batch_frames = (int32_t)S.batch.size();
      c.slot = si;
      c.arrival_ns = q.r.arrival_ns;
      c.admit_ns = S.admit_ns;
      c.done_ns = t;
    }
    lk.lock();
    for (auto& c : out) done.push_back(c);
    stats.completed += (int64_t)out.size();
    inflight_frames -= (int64_t)out.size();
    S.busy = false;
    inflight.pop_front();
    cv_sched.notify_one();
    cv_poll.notify_all();
  }
}

static void free_slots(rcfar_server srv) {
  for (Slot& S : srv->slots) {
    if (S.h) rcfar_destroy(S.h);
    if (S.done) cudaEventDestroy(S.done);
    if (S.stream) cudaStreamDestroy(S.stream);
    if (S.dev_io) cudaFree(S.dev_io);
    if (S.host_det) cudaFreeHost(S.host_det);
    S = Slot();
  }
}

extern "C" {

int64_t rcfar_server_now_ns(void) { return clock_ns(); }

rcfar_status rcfar_server_create(const rcfar_server_config* cfg, rcfar_server* out) {
  if (!cfg || !out) return RCFAR_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 8 || cfg->max_batch_frames < 1 || cfg->max_batch_frames > rcfar::kMaxBatch ||
      cfg->max_rows <= 0 || cfg->max_n <= 0 || cfg->max_window < 0 || cfg->budget_bytes <= 0 ||
      cfg->params.halo_c != -1)
    return RCFAR_ERR_INVALID_ARG;
  rcfar_pre_params pv = cfg->params;  // the band parameters must be valid for the largest N
  pv.halo_c = 0;
  rcfar_band b;
  if (rcfar_band_plan(cfg->max_n, &pv, &b) != RCFAR_OK) return RCFAR_ERR_INVALID_ARG;
  rcfar_server srv = new rcfar_server_s();
  srv->cfg = *cfg;
  srv->slots.resize(cfg->slots);
  const size_t share = (size_t)cfg->budget_bytes / (size_t)cfg->slots;
  // a slot's share: three quarters for the batch workspace, the rest for the
  // raw inputs (7/8 of it) and the decisions (1/8)
  const size_t ws_cap = share / 4 * 3, io = share - ws_cap;
  const size_t det_cap = a256(io / 8), in_cap = a256(io - det_cap);
  rcfar_status st = RCFAR_OK;
  int64_t dev_bytes = 0;
  for (Slot& S : srv->slots) {
    rcfar_config hc;
    std::memset(&hc, 0, sizeof(hc));
    hc.device = cfg->device;
    hc.max_rows = cfg->max_rows;
    hc.max_cols = cfg->max_n / 2 + 1;
    hc.max_n = cfg->max_n;
    hc.max_window = cfg->max_window;
    hc.max_frames = cfg->max_batch_frames;
    hc.batch_bytes = (int64_t)ws_cap;
    st = rcfar_create(&hc, &S.h);
    if (st != RCFAR_OK) break;
    if (cudaSetDevice(cfg->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&S.dev_io), in_cap + det_cap) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&S.host_det), det_cap) != cudaSuccess) {
      st = RCFAR_ERR_CUDA;
      break;
    }
    S.ws_cap = ws_cap;
    S.in_cap = in_cap;
    S.det_cap = det_cap;
    dev_bytes += (int64_t)(ws_cap + in_cap + det_cap);
  }
  if (st != RCFAR_OK) {
    free_slots(srv);
    delete srv;
    return st;
  }
  srv->stats.device_bytes = dev_bytes;
  srv->sched = std::thread([srv] { srv->scheduler(); });
  srv->comp = std::thread([srv] { srv->completer(); });
  *out = srv;
  return RCFAR_OK;
}

// Checks one request and sizes what it takes from a slot (no lock held).
static rcfar_status make_pending(rcfar_server srv, const rcfar_request* req, Pending* out) {
  if (!srv || !req) return RCFAR_ERR_INVALID_ARG;
  const rcfar_request& r = *req;
  const bool tm = srv->cfg.params.x_layout == RCFAR_X_TRACE_MAJOR;
  if (!r.x || !r.det || r.M <= 0 || r.N <= 0 || r.ldx < (tm ? r.M : r.N) || srv->cfg.params.mean_len > r.N ||
      (r.memory != RCFAR_MEM_HOST && r.memory != RCFAR_MEM_DEVICE))
    return RCFAR_ERR_INVALID_ARG;
  const bool device = r.memory == RCFAR_MEM_DEVICE;
  if (device) {  // both buffers must be memory the server's device can address as its own
    for (const void* p : {static_cast<const void*>(r.x), static_cast<const void*>(r.det)}) {
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return RCFAR_ERR_INVALID_ARG;
      }
      if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != srv->cfg.device)
        return RCFAR_ERR_INVALID_ARG;
    }
  }
  const rcfar_window& w = r.window;
  double factor = 0.0;
  if (rcfar_threshold_factor(&w, &factor, nullptr) != RCFAR_OK) return RCFAR_ERR_INVALID_ARG;
  if (r.M > srv->cfg.max_rows || r.N > srv->cfg.max_n || w.guard_r + w.train_r > srv->cfg.max_window ||
      w.guard_c + w.train_c > srv->cfg.max_window)
    return RCFAR_ERR_UNSUPPORTED;
  Pending q;
  q.r = r;
  rcfar_pre_params pf = srv->cfg.params;
  pf.halo_c = w.guard_c + w.train_c;
  rcfar_band b;
  rcfar_status st = rcfar_band_plan(r.N, &pf, &b);
  if (st != RCFAR_OK) return st;
  q.C = b.cols;
  if (r.ld_det < q.C) return RCFAR_ERR_INVALID_ARG;
  int64_t ws = 0;
  st = rcfar_batch_bytes(r.M, r.N, &srv->cfg.params, &w, &ws);
  if (st != RCFAR_OK) return st;
  q.ws = (size_t)ws;
  q.device = device;
  q.in_b = device ? 0 : a256((size_t)r.M * r.N * sizeof(float));
  q.det_b = device ? 0 : a256((size_t)r.M * q.C);
  const Slot& S0 = srv->slots[0];
  if (q.ws > S0.ws_cap || q.in_b > S0.in_cap || q.det_b > S0.det_cap) return RCFAR_ERR_UNSUPPORTED;
  *out = q;
  return RCFAR_OK;
}

rcfar_status rcfar_server_submit(rcfar_server srv, const rcfar_request* req) {
  int32_t n = 0;
  return rcfar_server_submit_many(srv, req, 1, &n);
}

rcfar_status rcfar_server_submit_many(rcfar_server srv, const rcfar_request* reqs, int32_t n, int32_t* n_queued) {
  if (n_queued) *n_queued = 0;
  if (!srv || n < 0 || (n > 0 && !reqs)) return RCFAR_ERR_INVALID_ARG;
  std::vector<Pending> qs;
  qs.reserve((size_t)n);
  rcfar_status st = RCFAR_OK;
  for (int32_t i = 0; i < n && st == RCFAR_OK; ++i) {
    Pending q;
    st = make_pending(srv, &reqs[i], &q);
    if (st == RCFAR_OK) qs.push_back(q);
  }
  const int64_t now = clock_ns();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->closing) return RCFAR_ERR_BAD_STATE;
    for (Pending& q : qs) {
      if (q.r.arrival_ns == 0) q.r.arrival_ns = now;
      srv->pending.push_back(q);
    }
    srv->stats.submitted += (int64_t)qs.size();
  }
  if (n_queued) *n_queued = (int32_t)qs.size();
  if (!qs.empty()) srv->cv_sched.notify_one();
  return st;
}

rcfar_status rcfar_server_prepare(rcfar_server srv, const int32_t* N, const rcfar_window* w, int32_t n) {
  if (!srv || n < 0 || (n > 0 && (!N || !w))) return RCFAR_ERR_INVALID_ARG;
  std::vector<rcfar_frame_desc> f(n);
  for (int i = 0; i < n; ++i) {
    std::memset(&f[i], 0, sizeof(rcfar_frame_desc));
    f[i].M = 1;
    f[i].N = N[i];
    f[i].window = w[i];
  }
  // a slot's handle is only used by the scheduler while the slot is busy;
  // preparing takes the lock so that no batch is formed meanwhile
  std::lock_guard<std::mutex> lk(srv->mu);
  for (Slot& S : srv->slots) {
    while (S.busy) {
      srv->mu.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(200));
      srv->mu.lock();
    }
    const rcfar_status st = rcfar_prepare(S.h, f.data(), n, &srv->cfg.params);
    if (st != RCFAR_OK) return st;
  }
  return RCFAR_OK;
}

rcfar_status rcfar_server_poll(rcfar_server srv, rcfar_completion* out, int32_t max, int32_t* n_out,
                               int32_t wait_ms) {
  if (!srv || !n_out || max < 0 || (max > 0 && !out) || wait_ms < 0) return RCFAR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  if (srv->done.empty() && wait_ms > 0)
    srv->cv_poll.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !srv->done.empty(); });
  int n = 0;
  while (n < max && !srv->done.empty()) {
    out[n++] = srv->done.front();
    srv->done.pop_front();
  }
  *n_out = n;
  return RCFAR_OK;
}

rcfar_status rcfar_server_get_stats(rcfar_server srv, rcfar_server_stats* out) {
  if (!srv || !out) return RCFAR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->stats;
  return RCFAR_OK;
}

rcfar_status rcfar_server_destroy(rcfar_server srv) {
  if (!srv) return RCFAR_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->closing = true;
  }
  srv->cv_sched.notify_all();
  if (srv->sched.joinable()) srv->sched.join();
  if (srv->comp.joinable()) srv->comp.join();
  free_slots(srv);
  delete srv;
  return RCFAR_OK;
}

}  // extern "C"
