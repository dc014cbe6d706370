// server.cu -- the serving layer: a request loop that admits QCL solves as
// they arrive (device memory from a caller-owned arena), keeps their ensembles
// resident, advances all admitted requests together in rounds, and reports
// latency percentiles beside throughput.
//
// Rounds (continuous batching): every active request advances by at most
// `quantum_steps` steps (a packed request also by at most 32 output times, one
// packed launch; the others' steps may span several persistent launches of
// their own, with no host turnaround between them).  Adiabatic two-state
// requests with at most 8 modes and too few walkers to fill the GPU alone are
// packed, per (mode bucket, model kind), into one
// persistent launch that reads a device table of (request, tile) work items;
// that part of a round is a fixed-shape CUDA graph [table uploads, packed
// kernels] captured once and replayed every round.  Other requests (many modes,
// more states) get their own persistent launches in the same round, spread
// over eight side streams so that small launches run side by side.  Requests
// that arrive meanwhile are admitted at the next round boundary.  A request's
// arithmetic depends only on its own descriptors, so its results are the same
// bits alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "model.h"

using namespace qcl;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

qcl_status fail(qcl_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return qcl::set_error(st, buf);
}

// First-fit allocator over the caller's arena (256-byte granules).
class Arena {
 public:
  void init(size_t base, size_t bytes) {
    free_.clear();
    free_[base] = bytes;
    total_ = bytes;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t total() const { return total_; }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t total_ = 0, used_ = 0;
};

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_ERROR = 3 };

struct Request {
  int64_t id = 0;
  int state = RQ_QUEUED;
  std::string err;
  // copies of the caller's descriptors
  int ns = 0, n = 0;
  double hbar = 1, hop = 1, pmax = 0.5;
  int32_t repr = QCL_REPR_ADIABATIC;
  std::vector<double> mass, omega, E, K, rho, R0, P0;
  double beta = INFINITY;
  int wigner = 1;
  qcl_ensemble_desc ens{};
  int64_t n_steps = 0;
  double dt = 0;
  int32_t stride = 1;
  // runtime
  qcl_model* model = nullptr;
  size_t ens_off = 0, ens_bytes = 0, obs_off = 0, obs_bytes = 0;
  int64_t n_out = 0, step = 0;
  bool observed0 = false;
  int skipped = 0;  // consecutive rounds without a step (round work budget)
  int64_t round_quantum = 0;  // steps this round may take
  int bucket = -1;  // packed bucket, -1 = own launches
  double t_submit = 0, t_admit = 0, t_done = 0;
  std::vector<double> result;
};

}  // namespace

struct qcl_server {
  qcl_server_desc d{};
  int device = 0;
  char* arena = nullptr;
  Arena alloc;
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  // requests with their own launches run on side streams, so that the small
  // ones' launches overlap; each round joins them back into `stream`
  static constexpr int kSide = 8;
  cudaStream_t side[kSide] = {};
  cudaEvent_t side_ev[kSide] = {};
  cudaEvent_t start_ev = nullptr;
  // device-time span of each busy period (first admission's work to the last
  // retirement's work, CUDA events on `stream`)
  cudaEvent_t busy_ev = nullptr, idle_ev = nullptr;
  bool busy = false;
  double device_busy_s = 0.0;
  int n_sm = 1;
  PackedTable* host_tab = nullptr;  // pinned, [2 kinds][buckets]
  PackedTable* dev_tab = nullptr;   // in the arena
  cudaGraphExec_t graph = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  // statistics
  std::vector<double> latencies;
  double first_submit = -1, last_done = -1, traj_steps = 0;
  int64_t rounds = 0, graph_replays = 0, n_error = 0;
  std::string fatal;
};

namespace {

constexpr int kTables = 2 * kPackedBuckets;

size_t table_bytes() { return align256(sizeof(PackedTable)) * kTables; }

PackedTable* htab(qcl_server* s, int kind, int bucket) { return s->host_tab + kind * kPackedBuckets + bucket; }
PackedTable* dtab(qcl_server* s, int kind, int bucket) {
  return (PackedTable*)((char*)s->dev_tab + align256(sizeof(PackedTable)) * (kind * kPackedBuckets + bucket));
}

// Enqueues every packed table upload and packed launch (the fixed-shape part of a round).
void enqueue_packed(qcl_server* s) {
  for (int kind = 0; kind < 2; ++kind)
    for (int b = 0; b < kPackedBuckets; ++b) {
      cudaMemcpyAsync(dtab(s, kind, b), htab(s, kind, b), sizeof(PackedTable), cudaMemcpyHostToDevice, s->stream);
      launch_packed(b, kind, dtab(s, kind, b), s->stream);
    }
}

// Admission: FIFO while the arena has room and fewer than max_active run.
void admit(qcl_server* s, std::vector<std::shared_ptr<Request>>& fresh) {
  std::lock_guard<std::mutex> lk(s->mu);
  while (!s->queue.empty() && (int)s->active.size() < s->d.max_active) {
    auto r = s->queue.front();
    size_t eo = 0, oo = 0;
    if (!s->alloc.alloc(r->ens_bytes, &eo)) break;
    if (!s->alloc.alloc(r->obs_bytes, &oo)) {
      s->alloc.release(eo, r->ens_bytes);
      break;
    }
    r->ens_off = eo;
    r->obs_off = oo;
    r->state = RQ_RUNNING;
    r->t_admit = now_s();
    s->queue.pop_front();
    s->active.push_back(r);
    fresh.push_back(r);
  }
}

void finish(qcl_server* s, const std::shared_ptr<Request>& r, int state, const std::string& err) {
  if (r->model) qcl_destroy_model(r->model);
  r->model = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  s->alloc.release(r->ens_off, r->ens_bytes);
  s->alloc.release(r->obs_off, r->obs_bytes);
  r->state = state;
  r->err = err;
  r->t_done = now_s();
  if (state == RQ_DONE) {
    s->latencies.push_back(r->t_done - r->t_submit);
    s->traj_steps += (double)r->ens.n_traj * (double)r->n_steps;
    s->last_done = r->t_done;
  } else {
    ++s->n_error;
  }
  s->active.erase(std::remove(s->active.begin(), s->active.end(), r), s->active.end());
  s->cv.notify_all();
}

// Chunk of request r for this round: steps [cs, ce), at most quantum steps
// and, for a packed request (one launch per round), at most 32 output times.
struct Chunk {
  int64_t cs, ce, k_first;
  int n_slots;
  bool first;
};

// Algorithmic flops of one walker step of a request's model (its relative
// cost): two-state models 10 per mode (12 in the general form) plus 26 scalar,
// more states 25 N_s^2 (400 at four states).
double step_flops(const Request& r) {
  if (r.ns > 2) return 25.0 * r.ns * r.ns;
  return (r.model && r.model->host.kind != 0 ? 12.0 : 10.0) * r.n + 26.0;
}

// Rounds skipped after which a request advances first, whatever its size.
constexpr int kMaxSkipped = 16;

Chunk plan(const Request& r, int64_t quantum, bool packed) {
  Chunk c{};
  c.cs = r.step;
  c.first = !r.observed0;
  const int64_t end = std::min(r.n_steps, r.step + quantum);
  const int64_t stride = r.stride;
  int n_slots = c.first ? 1 : 0;
  const int64_t next_out = (c.cs / stride + 1) * stride;
  const int64_t room = kChunkOut - n_slots;
  int64_t ce;
  if (packed && next_out + (room - 1) * stride <= end) {
    ce = next_out + (room - 1) * stride;
    n_slots += (int)room;
  } else {
    ce = end;
    if (end >= next_out) n_slots += (int)((end - next_out) / stride + 1);
  }
  c.ce = ce;
  c.n_slots = n_slots;
  c.k_first = c.first ? 0 : next_out / stride;
  return c;
}

void fill_bulk(const Request& r, const Chunk& c, int64_t n_tiles, BulkParams& bp) {
  const DevModel& h = r.model->host;
  bp = BulkParams{};
  bp.n_traj = r.ens.n_traj;
  bp.n_tiles = n_tiles;
  bp.traj_offset = r.ens.traj_id_offset;
  bp.seed = r.ens.seed;
  bp.step0 = c.cs;
  bp.stride = r.stride;
  bp.n = r.n;
  bulk_model_scalars(bp, h, r.dt);
  bp.cs = c.cs;
  bp.ce = c.ce;
  bp.k_first = c.k_first;
  bp.obs_first = c.first ? 1 : 0;
  bp.len = (int32_t)(c.ce - c.cs);
  bp.to_out0 = (int32_t)(r.stride - (c.cs % r.stride));
  bp.blk0 = (uint32_t)(c.cs >> 2);
  bp.widx0 = (int32_t)(c.cs & 3);
}

// Destroys the server's streams and events (after synchronising the side streams).
void release_streams(qcl_server* s) {
  for (int j = 0; j < qcl_server::kSide; ++j) {
    if (s->side[j]) {
      cudaStreamSynchronize(s->side[j]);
      cudaStreamDestroy(s->side[j]);
    }
    if (s->side_ev[j]) cudaEventDestroy(s->side_ev[j]);
    s->side[j] = nullptr;
    s->side_ev[j] = nullptr;
  }
  if (s->start_ev) cudaEventDestroy(s->start_ev);
  if (s->done_ev) cudaEventDestroy(s->done_ev);
  if (s->busy_ev) cudaEventDestroy(s->busy_ev);
  if (s->idle_ev) cudaEventDestroy(s->idle_ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  s->start_ev = s->done_ev = s->busy_ev = s->idle_ev = nullptr;
  s->stream = nullptr;
}

bool wait_stream(qcl_server* s, double timeout_s) {
  cudaEventRecord(s->done_ev, s->stream);
  const double t0 = now_s();
  while (true) {
    const cudaError_t e = cudaEventQuery(s->done_ev);
    if (e == cudaSuccess) return true;
    if (e != cudaErrorNotReady) return false;
    if (now_s() - t0 > timeout_s) return false;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// Ends a busy period: records an event after the work enqueued so far and adds
// the device time since the period's first event to the statistics.
void end_busy(qcl_server* s) {
  if (!s->busy) return;
  float ms = 0.0f;
  if (cudaEventRecord(s->idle_ev, s->stream) == cudaSuccess && cudaEventSynchronize(s->idle_ev) == cudaSuccess &&
      cudaEventElapsedTime(&ms, s->busy_ev, s->idle_ev) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->device_busy_s += 1e-3 * ms;
  }
  s->busy = false;
}

void run_round(qcl_server* s) {
  std::vector<std::shared_ptr<Request>> act;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    act = s->active;
  }
  if (act.empty()) return;
  for (int t = 0; t < kTables; ++t) {
    s->host_tab[t].n_req = 0;
    s->host_tab[t].n_work = 0;
  }
  struct Item {
    std::shared_ptr<Request> r;
    Chunk c;
  };
  std::vector<Item> items;
  // With a round work budget, requests advance in ascending order of remaining
  // work (those skipped kMaxSkipped rounds in a row first) until the budget is
  // spent: a full quantum each, a partial one (at least one step) for the
  // request that reaches the budget; the others wait for a later round.
  if (s->d.round_flops > 0.0) {
    std::vector<std::pair<double, std::shared_ptr<Request>>> order;
    for (auto& r : act) {
      const double rem = (double)r->ens.n_traj * (double)(r->n_steps - r->step) * step_flops(*r);
      order.push_back({r->skipped >= kMaxSkipped ? -1.0 : rem, r});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const auto& x, const auto& y) { return x.first < y.first; });
    double left = s->d.round_flops;
    act.clear();
    std::vector<int64_t> steps;
    for (auto& o : order) {
      Request& r = *o.second;
      if (left <= 0.0) {
        ++r.skipped;
        continue;
      }
      const double per_step = (double)r.ens.n_traj * step_flops(r);
      const int64_t k = std::min<int64_t>(s->d.quantum_steps, std::max<int64_t>(1, (int64_t)(left / per_step)));
      left -= (double)k * per_step;
      r.skipped = 0;
      act.push_back(o.second);
      steps.push_back(k);
    }
    for (size_t i = 0; i < act.size(); ++i) act[i]->round_quantum = steps[i];
  } else {
    for (auto& r : act) r->round_quantum = s->d.quantum_steps;
  }
  for (auto& r : act) {
    const Chunk c = plan(*r, r->round_quantum, r->bucket >= 0);
    items.push_back({r, c});
    if (r->bucket < 0) continue;
    PackedTable* T = htab(s, bulk_kind(r->model->host), r->bucket);
    if (T->n_req >= kMaxPacked) {  // table full: this request runs its own launch
      r->bucket = -2;
      continue;
    }
    PackedReq& e = T->req[T->n_req];
    const int64_t n_tiles = (r->ens.n_traj + kTile - 1) / kTile;
    fill_bulk(*r, c, n_tiles, e.bp);
    e.ens = s->arena + r->ens_off;
    e.part = (double*)(s->arena + r->obs_off + ObsLayout::make(r->ens.n_traj, 2, r->n_out).off_part);
    e.work0 = T->n_work;
    const DevModel& h = r->model->host;
    for (int j = 0; j < 8; ++j) {
      const bool on = j < r->n;
      e.hk[j] = on ? (float)(0.5 * r->dt * h.k[j]) : 0.f;
      e.hs[j] = on ? (float)(0.5 * r->dt * h.s[j]) : 0.f;
      e.dtm[j] = on ? (float)(r->dt / h.mass[j]) : 0.f;
      e.a[j] = on ? (float)h.a[j] : 0.f;
      e.b[j] = on ? (float)h.b[j] : 0.f;
      e.am[j] = on ? (float)(h.a[j] / h.mass[j]) : 0.f;
      e.bm[j] = on ? (float)(h.b[j] / h.mass[j]) : 0.f;
    }
    T->n_work += n_tiles;
    ++T->n_req;
  }
  // the side streams start after everything enqueued on `stream` so far
  // (admission sampling, the previous round)
  cudaEventRecord(s->start_ev, s->stream);
  // packed part: one fixed-shape graph (or the same launches directly), in
  // rounds that have packed requests
  bool any_packed = false;
  for (int t = 0; t < kTables; ++t) any_packed = any_packed || s->host_tab[t].n_req > 0;
  if (any_packed && s->graph) {
    cudaGraphLaunch(s->graph, s->stream);
    launches_add(kTables);
    ++s->graph_replays;
  } else if (any_packed) {
    enqueue_packed(s);
  }
  bool side_used[qcl_server::kSide] = {};
  int n_own = 0;
  for (auto& it : items) {
    Request& r = *it.r;
    char* ens_buf = s->arena + r.ens_off;
    char* obs_buf = s->arena + r.obs_off;
    if (r.bucket >= 0) {
      const ObsLayout OL = ObsLayout::make(r.ens.n_traj, 2, r.n_out);
      if (it.c.n_slots > 0)
        launch_fold((double*)(obs_buf + OL.off_part), (double*)(obs_buf + OL.off_rows) + (size_t)it.c.k_first * OL.q2,
                    (double*)(obs_buf + OL.off_fold), OL.n_tiles, OL.q2, it.c.n_slots, s->stream,
                    OL.n_fold_blocks > 1
                        ? (double*)(obs_buf + OL.off_chunk) + (size_t)it.c.k_first * OL.n_fold_blocks * OL.q2
                        : nullptr);
      launch_header_finish(ens_buf, it.c.cs, it.c.ce, s->stream);
    } else {
      if (r.bucket == -2) r.bucket = -1;
      const int j = n_own++ % qcl_server::kSide;
      if (!side_used[j]) {
        cudaStreamWaitEvent(s->side[j], s->start_ev, 0);
        side_used[j] = true;
      }
      const qcl_status st = qcl_propagate(r.model, &r.ens, ens_buf, r.ens_bytes, it.c.cs, it.c.ce - it.c.cs, r.dt,
                                          r.stride, obs_buf, r.obs_bytes, r.n_out, s->side[j]);
      if (st != QCL_OK) {
        finish(s, it.r, RQ_ERROR, qcl_last_error());
        it.r = nullptr;
      }
    }
  }
  for (int j = 0; j < qcl_server::kSide; ++j)
    if (side_used[j]) {
      cudaEventRecord(s->side_ev[j], s->side[j]);
      cudaStreamWaitEvent(s->stream, s->side_ev[j], 0);
    }
  if (!wait_stream(s, s->d.round_timeout_s > 0 ? s->d.round_timeout_s : 600.0)) {
    const cudaError_t e = cudaGetLastError();
    for (auto& it : items)
      if (it.r) finish(s, it.r, RQ_ERROR, std::string("round did not complete: ") + cudaGetErrorString(e));
    return;
  }
  ++s->rounds;
  struct Retire {
    std::shared_ptr<Request> r;
    int state;
    std::string err;
  };
  std::vector<Retire> retire;
  for (auto& it : items) {
    if (!it.r) continue;
    Request& r = *it.r;
    r.step = it.c.ce;
    r.observed0 = true;
    if (r.step >= r.n_steps) {
      const int nq = 4 * r.ns * r.ns;
      r.result.assign((size_t)r.n_out * (2 * nq + 3), 0.0);
      qcl_ens_status es{};
      qcl_status st = qcl_reduce_observables(r.model, &r.ens, s->arena + r.obs_off, r.obs_bytes, r.n_out, 0, r.n_out,
                                             r.result.data(), r.result.size(), s->stream);
      if (st == QCL_OK) st = qcl_ensemble_status(r.model, &r.ens, s->arena + r.ens_off, r.ens_bytes, &es, s->stream);
      if (st != QCL_OK)
        retire.push_back({it.r, RQ_ERROR, qcl_last_error()});
      else if (es.flags & (QCL_FLAG_NONFINITE | QCL_FLAG_STEP_MISMATCH))
        retire.push_back({it.r, RQ_ERROR, "non-finite value or step mismatch in the ensemble"});
      else
        retire.push_back({it.r, RQ_DONE, ""});
    }
  }
  // when every active request retires, the busy period ends here, before the
  // waiters are told (so statistics read after a wait include it)
  size_t n_active;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    n_active = s->active.size();
  }
  if (!retire.empty() && retire.size() == n_active) end_busy(s);
  for (auto& x : retire) finish(s, x.r, x.state, x.err);
}

void worker_main(qcl_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<std::shared_ptr<Request>> fresh;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::milliseconds(20), [s] { return s->stop || !s->queue.empty() || !s->active.empty(); });
      if (s->stop) break;
    }
    admit(s, fresh);
    if (!fresh.empty() && !s->busy) {  // an idle device starts a busy period
      cudaEventRecord(s->busy_ev, s->stream);
      s->busy = true;
    }
    for (auto& r : fresh) {
      qcl_model_desc md{r->ns, r->n, r->hbar, r->mass.data(), r->omega.data(), r->E.data(), r->K.data(), r->hop, r->pmax, r->repr, 0};
      qcl_status st = qcl_create_model(&md, &r->model);
      if (st == QCL_OK) {
        qcl_init_desc in{r->rho.data(), r->R0.data(), r->P0.data(), r->beta, r->wigner, 0};
        st = qcl_sample_initial(r->model, &r->ens, &in, s->arena + r->ens_off, r->ens_bytes, s->stream);
      }
      if (st != QCL_OK) finish(s, r, RQ_ERROR, qcl_last_error());
    }
    run_round(s);
    bool idle;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      idle = s->active.empty();
    }
    if (idle) end_busy(s);  // (requests that failed outside a round's retirement)
  }
}

}  // namespace

extern "C" {

qcl_status qcl_server_create(const qcl_server_desc* d, qcl_server** out) {
  if (!out) return fail(QCL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(QCL_ERR_INVALID_ARG, "server descriptor is NULL");
  if (!d->arena || ((uintptr_t)d->arena & 255) != 0) return fail(QCL_ERR_INVALID_ARG, "arena must be a 256-byte aligned device pointer");
  if (d->arena_bytes < table_bytes() + (1 << 20)) return fail(QCL_ERR_OUT_OF_MEMORY, "arena smaller than %zu bytes", table_bytes() + (1 << 20));
  if (d->max_active < 1 || d->quantum_steps < 1) return fail(QCL_ERR_INVALID_ARG, "max_active and quantum_steps must be >= 1");
  if (!(d->round_flops >= 0.0) || !std::isfinite(d->round_flops)) return fail(QCL_ERR_INVALID_ARG, "round_flops must be finite and >= 0");
  auto s = std::make_unique<qcl_server>();
  s->d = *d;
  cudaGetDevice(&s->device);
  s->arena = (char*)d->arena;
  s->dev_tab = (PackedTable*)s->arena;
  s->alloc.init(table_bytes(), d->arena_bytes - table_bytes());
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->done_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->start_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&s->busy_ev);
  if (e == cudaSuccess) e = cudaEventCreate(&s->idle_ev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device);
  for (int j = 0; j < qcl_server::kSide && e == cudaSuccess; ++j) {
    e = cudaStreamCreateWithFlags(&s->side[j], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->side_ev[j], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->host_tab, sizeof(PackedTable) * kTables, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    release_streams(s.get());
    return fail(QCL_ERR_CUDA, "server set-up failed: %s", cudaGetErrorString(e));
  }
  memset(s->host_tab, 0, sizeof(PackedTable) * kTables);
  // warm the launchers (occupancy queries) outside capture, then capture the
  // fixed-shape packed part of a round
  enqueue_packed(s.get());
  e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess && d->use_graphs) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_packed(s.get());
      e = cudaStreamEndCapture(s->stream, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph, g, 0);
    if (g) cudaGraphDestroy(g);
  }
  if (e != cudaSuccess) {
    cudaFreeHost(s->host_tab);
    release_streams(s.get());
    return fail(QCL_ERR_CUDA, "server set-up failed: %s", cudaGetErrorString(e));
  }
  qcl_server* raw = s.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return qcl::set_error(QCL_OK, "");
}

qcl_status qcl_server_submit(qcl_server* s, const qcl_request_desc* r, int64_t* id) {
  if (!s || !r || !id) return fail(QCL_ERR_INVALID_ARG, "NULL argument");
  if (!r->model || !r->init) return fail(QCL_ERR_INVALID_ARG, "request without model or initial condition");
  const qcl_model_desc& m = *r->model;
  if (m.n_states < 2 || m.n_states > QCL_MAX_STATES || m.n_modes < 1 || m.n_modes > QCL_MAX_MODES)
    return fail(QCL_ERR_UNSUPPORTED, "model size outside the built range");
  if (m.repr != QCL_REPR_ADIABATIC && m.repr != QCL_REPR_DIABATIC) return fail(QCL_ERR_INVALID_ARG, "unknown representation %d", m.repr);
  if (!m.mass || !m.omega || !m.E || !m.K || !r->init->rho_el0 || !r->init->R0 || !r->init->P0)
    return fail(QCL_ERR_INVALID_ARG, "a request array is NULL");
  if (r->n_traj < 1 || r->n_steps < 1 || r->out_stride < 1 || !(r->dt > 0.0))
    return fail(QCL_ERR_INVALID_ARG, "n_traj, n_steps, out_stride and dt must be positive");
  auto q = std::make_shared<Request>();
  const int ns = m.n_states, n = m.n_modes, nn = ns * ns;
  q->ns = ns;
  q->n = n;
  q->hbar = m.hbar;
  q->hop = m.hop_scale == 0.0 ? 1.0 : m.hop_scale;
  q->pmax = m.p_max == 0.0 ? 0.5 : m.p_max;
  q->repr = m.repr;
  q->mass.assign(m.mass, m.mass + n);
  q->omega.assign(m.omega, m.omega + n);
  q->E.assign(m.E, m.E + nn);
  q->K.assign(m.K, m.K + (size_t)nn * n);
  q->rho.assign(r->init->rho_el0, r->init->rho_el0 + nn);
  q->R0.assign(r->init->R0, r->init->R0 + n);
  q->P0.assign(r->init->P0, r->init->P0 + n);
  q->beta = r->init->beta;
  q->wigner = r->init->wigner;
  q->ens = qcl_ensemble_desc{r->n_traj, r->seed, r->traj_id_offset, QCL_PREC_FP32_BULK, 0};
  q->n_steps = r->n_steps;
  q->dt = r->dt;
  q->stride = r->out_stride;
  q->n_out = r->n_steps / r->out_stride + 1;
  q->ens_bytes = EnsLayout::make(r->n_traj, ns, n, QCL_PREC_FP32_BULK).total;
  q->obs_bytes = ObsLayout::make(r->n_traj, ns, q->n_out, tile_walkers(QCL_PREC_FP32_BULK, n, ns)).total;
  // the packed kernel runs adiabatic two-state models; others get their own
  // launches, and so do requests whose tiles fill two waves of the persistent
  // grid by themselves (three resident blocks per SM): packing gains them
  // nothing, and their own launch runs the single-solve kernel with two walkers
  // per thread.  Both routes give the same bits.
  q->bucket = (ns == 2 && m.repr == QCL_REPR_ADIABATIC) ? packed_bucket(n) : -1;
  if (q->bucket >= 0 && (r->n_traj + kTile - 1) / kTile >= 6 * (int64_t)s->n_sm) q->bucket = -1;
  q->t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  if (align256(q->ens_bytes) + align256(q->obs_bytes) > s->alloc.total())
    return fail(QCL_ERR_OUT_OF_MEMORY, "request needs %zu bytes, the arena holds %zu", q->ens_bytes + q->obs_bytes,
                s->alloc.total());
  if (s->d.max_queue > 0 && (int64_t)s->queue.size() >= s->d.max_queue) return fail(QCL_ERR_BUSY, "queue full");
  q->id = s->next_id++;
  s->queue.push_back(q);
  s->all[q->id] = q;
  if (s->first_submit < 0) s->first_submit = q->t_submit;
  s->cv.notify_all();
  *id = q->id;
  return qcl::set_error(QCL_OK, "");
}

qcl_status qcl_server_poll(qcl_server* s, int64_t id, int32_t* state, double* host_out, size_t host_len,
                           int64_t* n_rows) {
  if (!s || !state) return fail(QCL_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return fail(QCL_ERR_NOT_FOUND, "unknown request %lld", (long long)id);
  const Request& r = *it->second;
  *state = r.state;
  if (n_rows) *n_rows = r.n_out;
  if (r.state == RQ_ERROR) return fail(QCL_ERR_NUMERICAL, "request %lld failed: %s", (long long)id, r.err.c_str());
  if (r.state == RQ_DONE && host_out) {
    if (host_len < r.result.size()) return fail(QCL_ERR_INVALID_ARG, "host_out holds %zu doubles, needs %zu", host_len, r.result.size());
    memcpy(host_out, r.result.data(), sizeof(double) * r.result.size());
  }
  return qcl::set_error(QCL_OK, "");
}

qcl_status qcl_server_wait(qcl_server* s, int64_t id, double timeout_s, int32_t* state) {
  if (!s || !state) return fail(QCL_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return fail(QCL_ERR_NOT_FOUND, "unknown request %lld", (long long)id);
  auto r = it->second;
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                 [&] { return r->state == RQ_DONE || r->state == RQ_ERROR; });
  *state = r->state;
  if (!ok) return fail(QCL_ERR_TIMEOUT, "request %lld not finished after %.3f s", (long long)id, timeout_s);
  return qcl::set_error(QCL_OK, "");
}

qcl_status qcl_server_stats(qcl_server* s, qcl_server_statistics* out) {
  if (!s || !out) return fail(QCL_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  qcl_server_statistics st{};
  st.n_submitted = (int64_t)s->all.size();
  st.n_done = (int64_t)s->latencies.size();
  st.n_error = s->n_error;
  st.n_active = (int64_t)s->active.size();
  st.n_queued = (int64_t)s->queue.size();
  st.rounds = s->rounds;
  st.graph_replays = s->graph_replays;
  st.arena_used = s->alloc.used();
  st.traj_steps_done = s->traj_steps;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return 0.0;
    const double x = p * (l.size() - 1);
    const size_t i = (size_t)x;
    const double f = x - i;
    return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
  };
  st.latency_p50_s = pct(0.50);
  st.latency_p99_s = pct(0.99);
  double sum = 0;
  for (double v : l) sum += v;
  st.latency_mean_s = l.empty() ? 0.0 : sum / l.size();
  st.span_s = (s->first_submit >= 0 && s->last_done >= 0) ? s->last_done - s->first_submit : 0.0;
  st.throughput = st.span_s > 0 ? s->traj_steps / st.span_s : 0.0;
  st.device_busy_s = s->device_busy_s;
  st.device_throughput = s->device_busy_s > 0 ? s->traj_steps / s->device_busy_s : 0.0;
  *out = st;
  return qcl::set_error(QCL_OK, "");
}

qcl_status qcl_server_destroy(qcl_server* s) {
  if (!s) return qcl::set_error(QCL_OK, "");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaStreamSynchronize(s->stream);
  for (auto& r : s->active)
    if (r->model) qcl_destroy_model(r->model);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  cudaFreeHost(s->host_tab);
  release_streams(s);
  delete s;
  return qcl::set_error(QCL_OK, "");
}

}  // extern "C"
