// Serving loop for chemistry-step requests (host C++ scheduler over CUDA streams).
//
// The paper keeps the fields resident on the device (Sec. 2.1: only initialisation and
// output touch the CPU) and sizes its inference batches dynamically to bound GPU memory
// (Sec. 2.1).  This scheduler serves independent chemistry-step requests the same way:
//   * admission by device-memory budget: every (mechanism, ANN) class owns a structure-of-
//     arrays arena of cell columns in HBM; a request is admitted when a free column range of
//     its size exists (first fit), its state is copied in once and stays resident;
//   * continuous batching in pieces: whenever a stream is idle, it picks the kind (class,
//     mode, dt) of the ready request with the least work left (or of a request that has
//     waited past the starvation limit) and launches one kernel over pieces of every ready
//     request of that kind, smallest remainder first, through an index list; a direct-
//     integration request contributes at most di_chunk_cells per launch, so a large request
//     advances in bounded pieces and never holds a stream for its whole length while small
//     requests wait; requests keep being admitted while others run, and several streams
//     overlap on the device;
//   * completion: each piece's results are copied back as its launch ends; a request whose
//     last piece is back frees its columns and records its latency (submit -> results on the
//     host).
// Every per-cell result is independent of the batch composition and of the piece it runs in
// (the kernels are deterministic per cell), so a request's answer is the same alone or in any
// mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace chem;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kQueued = 0, kAdmitting, kReady, kRunning, kDone };

struct Request {
  int64_t id = 0;
  int cls = 0, mode = 0;
  double dt = 0;
  int64_t n = 0;
  const double *T = nullptr, *p = nullptr, *Y = nullptr;
  double *T_out = nullptr, *Y_out = nullptr;
  int32_t* status_out = nullptr;
  double t_submit = 0, t_done = 0;
  int64_t col0 = -1;
  int64_t launched = 0;   // cells handed to launches so far
  int64_t finished = 0;   // cells whose results are back on the host
  int state = kQueued;
  int result = 0;        // CHEM_OK or the API error of its launch
  cudaEvent_t admitted = nullptr;
};

// first-fit allocator of column ranges [start, start + len)
struct ColumnAllocator {
  std::map<int64_t, int64_t> free_;   // start -> length
  int64_t cap = 0;
  void init(int64_t c) { cap = c; free_.clear(); if (c > 0) free_[0] = c; }
  int64_t alloc(int64_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int64_t s = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[s + n] = len - n;
        return s;
      }
    }
    return -1;
  }
  void release(int64_t s, int64_t n) {
    auto it = free_.emplace(s, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
};

struct Class {
  chem_mech mech = nullptr;
  chem_ann ann = nullptr;
  int K = 0;
  int64_t cap = 0;
  double *T = nullptr, *p = nullptr, *Y = nullptr;
  ColumnAllocator cols;
};

// cells [off, off + len) of a request, run in one launch
struct Piece {
  Request* r;
  int64_t off, len;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr, copied = nullptr;
  int phase = 0;                    // 0 idle, 1 running, 2 copying back
  std::vector<Piece> pieces;
  int rc = 0;                       // API result of the slot's launch
  int32_t* d_idx = nullptr;
  int32_t* h_idx = nullptr;         // pinned staging of the index list
  int32_t* d_status = nullptr;
  void* di_ws = nullptr;
  void* ann_ws = nullptr;
  size_t ann_ws_bytes = 0;
};

}  // namespace

struct chem_server_s {
  chem_server_opts opts{};
  int device = 0;
  std::vector<std::unique_ptr<Class>> classes;
  std::vector<Slot> slots;
  size_t used_bytes = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;                      // waiting for admission (FIFO)
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<double> latencies_ms;
  int64_t next_id = 1, submitted = 0, completed = 0, failed = 0, cells_done = 0, batches = 0, batch_reqs = 0;
  double t_first = -1, t_last = 0;
  cudaStream_t copy_in = nullptr;
  std::thread th;
  std::atomic<bool> stop{false};
  std::atomic<bool> started{false};
  int error = 0;
};

namespace {

void free_slot(Slot& sl) {
  if (sl.s) cudaStreamDestroy(sl.s);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.copied) cudaEventDestroy(sl.copied);
  if (sl.d_idx) cudaFree(sl.d_idx);
  if (sl.h_idx) cudaFreeHost(sl.h_idx);
  if (sl.d_status) cudaFree(sl.d_status);
  if (sl.di_ws) cudaFree(sl.di_ws);
  if (sl.ann_ws) cudaFree(sl.ann_ws);
  sl = Slot{};
}

void finish_request(chem_server_s* sv, Request* r, double t) {
  r->t_done = t;
  r->state = kDone;
  if (r->admitted) { cudaEventDestroy(r->admitted); r->admitted = nullptr; }
  if (r->col0 >= 0) { sv->classes[r->cls]->cols.release(r->col0, r->n); r->col0 = -1; }
  sv->completed++;
  if (r->result != CHEM_OK) sv->failed++;
  sv->cells_done += r->n;
  sv->latencies_ms.push_back((r->t_done - r->t_submit) * 1e3);
  sv->t_last = std::max(sv->t_last, t);
}

// one pass of the scheduler; returns true if anything progressed.  Called with mu held.
bool schedule(chem_server_s* sv) {
  bool progress = false;
  const double t = now_s();
  // completions: copy each piece's results back, then account for them
  for (Slot& sl : sv->slots) {
    if (sl.phase == 1 && cudaEventQuery(sl.done) == cudaSuccess) {
      int64_t s0 = 0;
      for (const Piece& pc : sl.pieces) {
        Request* r = pc.r;
        Class& c = *sv->classes[r->cls];
        if (sl.rc == CHEM_OK) {
          cudaMemcpyAsync(r->T_out + pc.off, c.T + r->col0 + pc.off, pc.len * 8, cudaMemcpyDeviceToHost, sl.s);
          cudaMemcpy2DAsync(r->Y_out + pc.off, r->n * 8, c.Y + r->col0 + pc.off, c.cap * 8, pc.len * 8, c.K,
                            cudaMemcpyDeviceToHost, sl.s);
          cudaMemcpyAsync(r->status_out + pc.off, sl.d_status + s0, pc.len * 4, cudaMemcpyDeviceToHost, sl.s);
        }
        s0 += pc.len;
      }
      cudaEventRecord(sl.copied, sl.s);
      sl.phase = 2;
      progress = true;
    }
    if (sl.phase == 2 && cudaEventQuery(sl.copied) == cudaSuccess) {
      for (const Piece& pc : sl.pieces) {
        Request* r = pc.r;
        if (sl.rc != CHEM_OK) r->result = sl.rc;
        r->finished += pc.len;
        if (r->finished == r->n) finish_request(sv, r, now_s());
      }
      sl.pieces.clear();
      sl.phase = 0;
      progress = true;
      sv->cv.notify_all();
    }
  }
  // admission in arrival order; a request that does not fit waits, and once the oldest
  // request has waited for starvation_s nothing newer is admitted past it
  for (auto it = sv->queue.begin(); it != sv->queue.end();) {
    Request* r = *it;
    Class& c = *sv->classes[r->cls];
    const int64_t col = c.cols.alloc(r->n);
    if (col < 0) {
      if (sv->opts.starvation_s > 0 && it == sv->queue.begin() && t - r->t_submit > sv->opts.starvation_s) break;
      ++it;
      continue;
    }
    r->col0 = col;
    cudaMemcpyAsync(c.T + col, r->T, r->n * 8, cudaMemcpyHostToDevice, sv->copy_in);
    cudaMemcpyAsync(c.p + col, r->p, r->n * 8, cudaMemcpyHostToDevice, sv->copy_in);
    cudaMemcpy2DAsync(c.Y + col, c.cap * 8, r->Y, r->n * 8, r->n * 8, c.K, cudaMemcpyHostToDevice, sv->copy_in);
    cudaEventCreateWithFlags(&r->admitted, cudaEventDisableTiming);
    cudaEventRecord(r->admitted, sv->copy_in);
    r->state = kAdmitting;
    it = sv->queue.erase(it);
    progress = true;
  }
  // batching: every idle stream picks a kind and launches pieces of its ready requests
  const int64_t di_chunk = sv->opts.di_chunk_cells > 0 ? sv->opts.di_chunk_cells : 32768;
  for (Slot& sl : sv->slots) {
    if (sl.phase != 0) continue;
    std::vector<Request*> ready;
    for (auto& kv : sv->reqs) {
      Request* r = kv.second.get();
      if (r->state == kAdmitting && cudaEventQuery(r->admitted) == cudaSuccess) r->state = kReady;
      if (r->state == kReady && r->launched < r->n) ready.push_back(r);
    }
    if (ready.empty()) break;
    auto left = [](const Request* r) { return r->n - r->launched; };
    auto before = [&](const Request* a, const Request* b) {
      return left(a) != left(b) ? left(a) < left(b) : a->id < b->id;
    };
    // the kind: that of a request past the starvation limit (oldest first), else that of the
    // request with the least work left
    Request* pick = nullptr;
    if (sv->opts.starvation_s > 0)
      for (Request* r : ready)
        if (t - r->t_submit > sv->opts.starvation_s && (!pick || r->id < pick->id)) pick = r;
    if (!pick)
      for (Request* r : ready)
        if (!pick || before(r, pick)) pick = r;
    std::vector<Request*> kind;
    for (Request* r : ready)
      if (r->cls == pick->cls && r->mode == pick->mode && r->dt == pick->dt) kind.push_back(r);
    std::sort(kind.begin(), kind.end(), before);
    if (pick != kind.front()) {   // a starving request goes first within its kind
      kind.erase(std::find(kind.begin(), kind.end(), pick));
      kind.insert(kind.begin(), pick);
    }
    const int64_t cap = sv->opts.max_batch_cells;
    const int64_t piece_max = pick->mode == 0 ? std::min<int64_t>(di_chunk, cap) : cap;
    int64_t cells = 0;
    for (Request* r : kind) {
      if (cells >= cap) break;
      const int64_t len = std::min({left(r), piece_max, cap - cells});
      sl.pieces.push_back(Piece{r, r->launched, len});
      for (int64_t i = 0; i < len; ++i) sl.h_idx[cells + i] = (int32_t)(r->col0 + r->launched + i);
      r->launched += len;
      if (r->launched == r->n) r->state = kRunning;
      cells += len;
    }
    Class& c = *sv->classes[pick->cls];
    cudaMemcpyAsync(sl.d_idx, sl.h_idx, cells * 4, cudaMemcpyHostToDevice, sl.s);
    if (pick->mode == 1) {
      chem_ann_opts ao{};
      sl.rc = chem_step_ann(c.mech, c.ann, cells, c.cap, pick->dt, c.T, c.p, c.Y, sl.d_idx, &ao, sl.d_status,
                            sl.ann_ws, sl.ann_ws_bytes, (chem_stream)sl.s);
    } else {
      sl.rc = chem_step_di(c.mech, cells, c.cap, pick->dt, c.T, c.p, c.Y, sl.d_idx, nullptr, sl.d_status, nullptr,
                           sl.di_ws, chem_workspace_bytes(c.mech, cells), (chem_stream)sl.s);
    }
    cudaEventRecord(sl.done, sl.s);
    sl.phase = 1;
    sv->batches++;
    sv->batch_reqs += (int64_t)sl.pieces.size();
    progress = true;
  }
  return progress;
}

void run(chem_server_s* sv) {
  cudaSetDevice(sv->device);
  while (!sv->stop.load()) {
    bool progress;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      progress = schedule(sv);
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" {

int chem_server_create(const chem_server_opts* opts, chem_server* out) {
  if (!opts || !out || opts->n_streams < 1 || opts->n_streams > 16 || opts->max_batch_cells < 1 ||
      opts->hbm_budget_bytes == 0 || opts->di_chunk_cells < 0)
    return set_error(CHEM_E_ARG, "chem_server_create: bad options");
  *out = nullptr;
  chem_server_s* sv = new chem_server_s();
  sv->opts = *opts;
  int rc = cuda_check(cudaGetDevice(&sv->device), "cudaGetDevice");
  if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&sv->copy_in, cudaStreamNonBlocking), "stream");
  sv->slots.resize(opts->n_streams);
  for (Slot& sl : sv->slots) {
    if (rc) break;
    rc = cuda_check(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking), "stream");
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "event");
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming), "event");
    if (!rc) rc = cuda_check(cudaMalloc((void**)&sl.d_idx, (size_t)opts->max_batch_cells * 4), "idx alloc");
    if (!rc) rc = cuda_check(cudaMallocHost((void**)&sl.h_idx, (size_t)opts->max_batch_cells * 4), "idx staging");
    if (!rc) rc = cuda_check(cudaMalloc((void**)&sl.d_status, (size_t)opts->max_batch_cells * 4), "status alloc");
    if (!rc) rc = cuda_check(cudaMalloc(&sl.di_ws, 256), "workspace alloc");
    sv->used_bytes += (size_t)opts->max_batch_cells * 8 + 256;
  }
  if (rc) {
    for (Slot& sl : sv->slots) free_slot(sl);
    if (sv->copy_in) cudaStreamDestroy(sv->copy_in);
    delete sv;
    return rc;
  }
  *out = sv;
  return CHEM_OK;
}

int chem_server_add_class(chem_server sv, chem_mech mech, chem_ann ann, int64_t capacity_cells, int* class_id) {
  if (!sv || !mech || capacity_cells < 1 || !class_id) return set_error(CHEM_E_ARG, "chem_server_add_class: bad arguments");
  if (sv->started.load()) return set_error(CHEM_E_ARG, "chem_server_add_class: add classes before the first submit");
  int K = 0;
  chem_mech_info(mech, &K, nullptr, nullptr);
  auto c = std::make_unique<Class>();
  c->mech = mech;
  c->ann = ann;
  c->K = K;
  c->cap = capacity_cells;
  size_t need = (size_t)capacity_cells * (K + 2) * 8;
  size_t ann_ws = ann ? chem_ann_workspace_bytes(ann, sv->opts.max_batch_cells) : 0;
  need += ann_ws * sv->slots.size();
  if (sv->used_bytes + need > sv->opts.hbm_budget_bytes)
    return set_error(CHEM_E_NOMEM, "chem_server_add_class: the class does not fit in the HBM budget");
  int rc = cuda_check(cudaMalloc((void**)&c->T, (size_t)capacity_cells * 8), "arena");
  if (!rc) rc = cuda_check(cudaMalloc((void**)&c->p, (size_t)capacity_cells * 8), "arena");
  if (!rc) rc = cuda_check(cudaMalloc((void**)&c->Y, (size_t)capacity_cells * K * 8), "arena");
  if (ann)
    for (Slot& sl : sv->slots) {
      if (rc) break;
      if (ann_ws > sl.ann_ws_bytes) {
        if (sl.ann_ws) cudaFree(sl.ann_ws);
        sl.ann_ws = nullptr;
        rc = cuda_check(cudaMalloc(&sl.ann_ws, ann_ws), "ann workspace");
        sl.ann_ws_bytes = ann_ws;
      }
    }
  if (rc) {
    if (c->T) cudaFree(c->T);
    if (c->p) cudaFree(c->p);
    if (c->Y) cudaFree(c->Y);
    return rc;
  }
  c->cols.init(capacity_cells);
  sv->used_bytes += need;
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->classes.push_back(std::move(c));
  *class_id = (int)sv->classes.size() - 1;
  return CHEM_OK;
}

int chem_server_submit(chem_server sv, int class_id, int mode, double dt, int64_t n, const double* T, const double* p,
                       const double* Y, double* T_out, double* Y_out, int32_t* status_out, int64_t* request_id) {
  if (!sv || class_id < 0 || class_id >= (int)sv->classes.size() || (mode != 0 && mode != 1) || n < 1 ||
      !T || !p || !Y || !T_out || !Y_out || !status_out || !(dt >= 0))
    return set_error(CHEM_E_ARG, "chem_server_submit: bad arguments");
  if (mode == 1 && !sv->classes[class_id]->ann) return set_error(CHEM_E_ARG, "chem_server_submit: class has no ANN");
  if (n > sv->classes[class_id]->cap) return set_error(CHEM_E_ARG, "chem_server_submit: request larger than its class arena");
  auto r = std::make_unique<Request>();
  r->cls = class_id;
  r->mode = mode;
  r->dt = dt;
  r->n = n;
  r->T = T; r->p = p; r->Y = Y;
  r->T_out = T_out; r->Y_out = Y_out; r->status_out = status_out;
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lock(sv->mu);
  r->id = sv->next_id++;
  if (request_id) *request_id = r->id;
  if (sv->t_first < 0) sv->t_first = r->t_submit;
  sv->queue.push_back(r.get());
  sv->reqs[r->id] = std::move(r);
  sv->submitted++;
  if (!sv->started.exchange(true)) sv->th = std::thread(run, sv);
  return CHEM_OK;
}

// Wait until the request is complete (done = 1) or timeout_s elapsed (done = 0).  The
// request's result code (CHEM_OK or the launch error) is returned in *result.
int chem_server_wait(chem_server sv, int64_t request_id, double timeout_s, int* done, int* result) {
  if (!sv || !done) return set_error(CHEM_E_ARG, "chem_server_wait: bad arguments");
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return set_error(CHEM_E_ARG, "chem_server_wait: unknown request");
  Request* r = it->second.get();
  sv->cv.wait_for(lock, std::chrono::duration<double>(std::max(timeout_s, 0.0)), [&] { return r->state == kDone; });
  *done = r->state == kDone;
  if (result) *result = r->result;
  return CHEM_OK;
}

int chem_server_request_latency(chem_server sv, int64_t request_id, double* latency_ms) {
  if (!sv || !latency_ms) return set_error(CHEM_E_ARG, "chem_server_request_latency: bad arguments");
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return set_error(CHEM_E_ARG, "chem_server_request_latency: unknown request");
  const Request* r = it->second.get();
  *latency_ms = r->state == kDone ? (r->t_done - r->t_submit) * 1e3 : -1.0;
  return CHEM_OK;
}

int chem_server_get_stats(chem_server sv, chem_server_stats* st) {
  if (!sv || !st) return set_error(CHEM_E_ARG, "chem_server_get_stats: bad arguments");
  std::lock_guard<std::mutex> lock(sv->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = sv->submitted;
  st->completed = sv->completed;
  st->failed = sv->failed;
  st->cells = sv->cells_done;
  st->batches = sv->batches;
  st->mean_batch_requests = sv->batches ? (double)sv->batch_reqs / sv->batches : 0.0;
  std::vector<double> l = sv->latencies_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
      const double pos = q * (l.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - i;
      return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->max_ms = l.back();
    double s = 0;
    for (double v : l) s += v;
    st->mean_ms = s / l.size();
  }
  st->wall_s = sv->t_first >= 0 ? sv->t_last - sv->t_first : 0.0;
  st->cells_per_s = st->wall_s > 0 ? st->cells / st->wall_s : 0.0;
  st->hbm_bytes = (double)sv->used_bytes;
  return CHEM_OK;
}

void chem_server_free(chem_server sv) {
  if (!sv) return;
  sv->stop.store(true);
  if (sv->th.joinable()) sv->th.join();
  for (Slot& sl : sv->slots) {
    if (sl.s) cudaStreamSynchronize(sl.s);
    free_slot(sl);
  }
  if (sv->copy_in) {
    cudaStreamSynchronize(sv->copy_in);
    cudaStreamDestroy(sv->copy_in);
  }
  for (auto& kv : sv->reqs)
    if (kv.second->admitted) cudaEventDestroy(kv.second->admitted);
  for (auto& c : sv->classes) {
    cudaFree(c->T);
    cudaFree(c->p);
    cudaFree(c->Y);
  }
  delete sv;
}

}  // extern "C"
