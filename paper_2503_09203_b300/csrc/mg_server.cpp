// Serving loop of libmarinegym: continuous batching of rollout requests.
//
// A server owns one device arena split into a slot space (per-env parameter
// planes, hover target and return accumulators, indexed by slot) and a state
// space (per-request SoA state planes). A scheduler thread runs ticks; each
//   1. admits pending requests in FIFO order while both spaces have room
//      (first-fit allocators) and resets their envs on the device;
//   2. advances every admitted request by one control step in one shared
//      launch per thruster count (segments = requests, each with its own
//      class, K, seed and step counter; actions drawn on the device);
//   3. copies the final state and returns of the requests whose last step it
//      ran to pinned host memory.
// Ticks are pipelined: while tick t runs, the host prepares and enqueues tick
// t+1 (which requests finish with tick t is known in advance, and the space
// they free may be reused at once: the stream orders t+1's resets after t's
// copies), then waits for tick t and publishes its results. Requests that
// arrive while others run join the next tick, so their work shares launches
// with the running ones. Nothing on the device waits on the host or on
// another kernel: every device call is an ordinary launch or copy on the
// server's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/marinegym.h"
#include "mg_internal.h"

namespace mg {
cudaError_t launch_step(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                        bool dependent, bool shared_sm, cudaStream_t st);
cudaError_t launch_reset(const ResetArgs& a, cudaStream_t st);
cudaError_t prepare_tick_pm0(int nt, int var);
cudaError_t prepare_tick_pm1(int nt, int var);
}  // namespace mg

// Class tables built as the simulator builds them (mg_runtime.cpp).
void class_alloc_table(const mg_class_desc& c, double B[6][8]);
mg::ClassG class_generic_table(const mg_class_desc& c);
bool class_is_generic(const mg_class_desc& c);

using namespace mg;

namespace {

const double kG = 9.81;
const int kThreads = 128;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, capacity) in units.
class RangeAlloc {
 public:
  explicit RangeAlloc(int64_t cap = 0) { reset(cap); }
  void reset(int64_t cap) {
    free_.clear();
    if (cap > 0) free_[0] = cap;
    cap_ = cap;
  }
  int64_t alloc(int64_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[off + n] = len - n;
        return off;
      }
    }
    return -1;
  }
  void release(int64_t off, int64_t n) {
    auto it = free_.emplace(off, n).first;
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
  int64_t capacity() const { return cap_; }

 private:
  std::map<int64_t, int64_t> free_;
  int64_t cap_ = 0;
};

struct Req {
  int64_t id = 0;
  mg_request r{};
  int32_t status = MG_REQ_PENDING;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int64_t steps_done = 0;    // completed ticks (published)
  int64_t steps_sched = 0;   // ticks enqueued
  int32_t n_thr = 0, n4 = 0;
  int32_t dz = 0;            // the class has a nonzero dead zone
  int64_t slot_off = -1, st_off = -1;
  float h = 0;
  float alpha[8] = {0};
  std::vector<float> final_state, returns;
};

// Weighted quantile over (value, weight) samples.
double wquantile(std::vector<std::pair<double, double>> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  double tot = 0;
  for (auto& x : v) tot += x.second;
  double acc = 0;
  for (auto& x : v) {
    acc += x.second;
    if (acc >= q * tot) return x.first;
  }
  return v.back().first;
}

}  // namespace

// Host side of one tick in flight; two alternate, so that the next tick is
// prepared and enqueued while the current one runs.
struct TickBuf {
  SegDesc* h_segs = nullptr;      // pinned tick segment table
  SegDesc* h_rsegs = nullptr;     // pinned reset segment table
  int32_t* h_tile_seg = nullptr;  // pinned tile map
  float* h_stage = nullptr;       // pinned: final states and returns of retiring requests
  size_t stage_floats = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_done = nullptr;
};

// One tick: the requests it steps, those it admitted (first step) and those
// whose last step it runs.
struct Tick {
  bool valid = false;
  int par = 0;
  std::vector<Req*> act, fresh, done;
  int64_t envs = 0;
};

struct mg_server {
  mg_server_config cfg{};
  std::vector<mg_class_desc> classes;
  std::vector<int> class_var;   // step variant per class: 0 propellers, 1 generic actuators, 2 RK4
  int device = 0;
  int num_sms = 148;
  // device
  void* arena = nullptr;
  ClassF* d_cls = nullptr;
  ClassNominal* d_nominal = nullptr;
  SegDesc* d_segs = nullptr;     // tick segment table
  SegDesc* d_rsegs = nullptr;    // reset segment table
  float4* d_planes = nullptr;    // [N_PLANES][S]
  float* d_ret = nullptr;        // [S]
  float* d_state = nullptr;      // state space (floats)
  uint32_t* d_status = nullptr;
  int32_t* d_tile_seg = nullptr; // tick: segment of each tile
  int64_t tile_cap = 0;
  TickBuf buf[2];                // host side of the two ticks in flight
  int64_t S = 0, state_cap = 0;
  size_t budget = 0;             // arena budget (bytes)
  // Without DR and current every env of a class has the class's nominal
  // physics: ticks then read the class tables instead of per-env parameter
  // planes (the target plane only), and resets write only the target.
  bool class_const = false;
  RangeAlloc slots, states;
  // Device bytes held by admitted requests (slot planes, return and state
  // of their envs), and the most ever held at once: the admission rule keeps
  // it within the arena, and the statistic lets a caller check that.
  size_t resident = 0, peak_resident = 0;
  int32_t held = 0, peak_requests = 0;   // requests holding arena space
  cudaStream_t stream = nullptr;
  // scheduler
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  int64_t next_id = 1;
  std::deque<int64_t> pending;
  std::vector<Req*> active;   // admitted, not yet published as done (map nodes are stable)
  std::unordered_map<int64_t, Req> reqs;
  // stats
  int64_t requests_done = 0, env_steps = 0, ticks = 0;
  double busy = 0, last_tick_end = 0;
  std::vector<std::pair<double, double>> lat;   // (inter-step time, #requests)
  std::vector<std::pair<double, double>> qdel;  // (queue delay, 1)
  std::vector<std::pair<double, double>> tick;  // (device time, 1)
  std::string err;
  int32_t fatal = MG_OK;
};

static int sfail(mg_server* s, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  return code;
}

static int64_t state_units(int n_thr, int n4) { return (int64_t)n4 * (13 + n_thr); }

// Device bytes of an admitted request: its slots' parameter planes and return
// accumulator, and its state planes.
static size_t request_bytes(const Req& q) {
  return (size_t)q.n4 * (sizeof(float4) * N_PLANES + sizeof(float)) + sizeof(float) * (size_t)state_units(q.n_thr, q.n4);
}

// Admit pending requests in FIFO order while they fit; reset their envs.
static void admit_locked(mg_server* s, std::vector<Req*>& admitted) {
  while (!s->pending.empty() && (int)s->active.size() < s->cfg.max_requests) {
    Req& q = s->reqs[s->pending.front()];
    const int64_t so = s->slots.alloc(q.n4);
    if (so < 0) break;
    const int64_t st = s->states.alloc(state_units(q.n_thr, q.n4));
    if (st < 0) {
      s->slots.release(so, q.n4);
      break;
    }
    q.slot_off = so;
    q.st_off = st;
    s->resident += request_bytes(q);
    s->peak_resident = std::max(s->peak_resident, s->resident);
    s->peak_requests = std::max(s->peak_requests, ++s->held);
    q.status = MG_REQ_RUNNING;
    q.t_admit = now_s();
    s->qdel.push_back({q.t_admit - q.t_submit, 1.0});
    s->active.push_back(&q);
    admitted.push_back(&q);
    s->pending.pop_front();
  }
}

static SegDesc seg_of(const Req& q) {
  SegDesc sd;
  std::memset(&sd, 0, sizeof(sd));
  sd.n_envs = q.r.n_envs;
  sd.cls = q.r.cls;
  sd.n_thr = q.n_thr;
  sd.K = q.r.K;
  sd.step0 = (int32_t)q.steps_sched;
  sd.n4 = q.n4;
  sd.st_off = q.st_off;
  sd.slot_off = q.slot_off;
  sd.env_base = 0;
  sd.h = q.h;
  sd.dt = q.h * (float)q.r.K;
  sd.track = 0;
  sd.flags = q.dz ? 1 : 0;   // bit 0: the class has a dead zone
  for (int i = 0; i < 8; ++i) sd.alpha[i] = q.alpha[i];
  sd.seed = q.r.seed;
  return sd;
}

// Prepare the tick after `prev` (still running) into buffer `par`: free the
// space of the requests that finish with `prev`, admit pending requests, and
// list the requests this tick steps.
static Tick prepare_tick(mg_server* s, const Tick& prev, int par) {
  Tick t;
  t.par = par;
  std::lock_guard<std::mutex> lk(s->mu);
  for (Req* q : prev.done) {
    s->slots.release(q->slot_off, q->n4);
    s->states.release(q->st_off, state_units(q->n_thr, q->n4));
    s->resident -= request_bytes(*q);
    --s->held;
  }
  if (s->stop || s->fatal != MG_OK) return t;
  admit_locked(s, t.fresh);
  for (Req* q : s->active)
    if (q->steps_sched < q->r.horizon) t.act.push_back(q);
  t.valid = !t.act.empty();
  return t;
}

// Enqueue tick t on the server's stream: resets of its admitted requests,
// its tables, one launch per thruster count, and the copies of the finishing
// requests' results. Returns false (fatal set) if pinned staging is short.
static bool enqueue_tick(mg_server* s, Tick& t) {
  TickBuf& b = s->buf[t.par];
  cudaStream_t st = s->stream;
  if (!t.fresh.empty()) {
    for (size_t k = 0; k < t.fresh.size(); ++k) b.h_rsegs[k] = seg_of(*t.fresh[k]);
    cudaMemcpyAsync(s->d_rsegs, b.h_rsegs, sizeof(SegDesc) * t.fresh.size(), cudaMemcpyHostToDevice, st);
    for (size_t k = 0; k < t.fresh.size(); ++k) {
      const SegDesc& sd = b.h_rsegs[k];
      ResetArgs a;
      std::memset(&a, 0, sizeof(a));
      a.segs = s->d_rsegs + k;
      a.n_segs = 1;
      a.n_sel = sd.n_envs;
      a.nominal = s->d_nominal;
      a.per_env = s->class_const ? 0 : 1;
      a.serving = 1;
      a.state = s->d_state;
      a.planes = s->class_const ? s->d_planes + (size_t)TGT_PLANE * s->S : s->d_planes;
      a.n_slots = s->S;
      const mg_reset_cfg& r = s->cfg.reset;
      a.dr = r.dr_enabled; a.cur = r.current_enabled; a.cur3d = r.current_3d; a.init_mode = r.init_mode;
      a.mass_lo = r.mass_lo; a.mass_hi = r.mass_hi; a.added_lo = r.added_lo; a.added_hi = r.added_hi;
      a.damp_lo = r.damp_lo; a.damp_hi = r.damp_hi; a.cob_lo = r.cob_lo; a.cob_hi = r.cob_hi;
      a.cur_lo = r.cur_lo; a.cur_hi = r.cur_hi; a.target_half = r.target_half; a.pos_radius = r.pos_radius;
      a.max_angle = r.max_angle;
      launch_reset(a, st);
      cudaMemsetAsync(s->d_ret + sd.slot_off, 0, sizeof(float) * sd.n4, st);
    }
  }
  // Tick table in one pass: requests grouped by thruster count and step
  // variant (propellers, generic actuators, RK4), and the segment (within
  // its group) of every tile.
  struct G { int nt, var, lo, hi, tile_lo, tiles; };
  std::vector<G> groups;
  std::vector<const Req*> by_nt[3][MG_MAX_THR + 1];
  for (const Req* q : t.act) {
    by_nt[s->class_var[q->r.cls]][q->n_thr].push_back(q);
    t.envs += q->r.n_envs;
  }
  int n_seg = 0, tiles = 0;
  for (int key = 0; key < 3 * MG_MAX_THR; ++key) {
    const int var = key / MG_MAX_THR, nt = 1 + key % MG_MAX_THR;
    if (by_nt[var][nt].empty()) continue;
    G g{nt, var, n_seg, 0, tiles, 0};
    for (const Req* q : by_nt[var][nt]) {
      SegDesc& sd = b.h_segs[n_seg];
      sd = seg_of(*q);
      sd.tile_begin = tiles;
      const int qt = (q->n4 + kThreads - 1) / kThreads;
      for (int k = 0; k < qt; ++k) b.h_tile_seg[tiles + k] = n_seg - g.lo;
      tiles += qt;
      ++n_seg;
    }
    g.hi = n_seg;
    g.tiles = tiles - g.tile_lo;
    groups.push_back(g);
  }
  cudaMemcpyAsync(s->d_segs, b.h_segs, sizeof(SegDesc) * n_seg, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s->d_tile_seg, b.h_tile_seg, sizeof(int32_t) * tiles, cudaMemcpyHostToDevice, st);
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.segs = s->d_segs;
  a.classes = s->d_cls;
  a.state = s->d_state;
  a.n_steps = 1;
  a.act_mode = 1;
  a.planes = s->class_const ? s->d_planes + (size_t)TGT_PLANE * s->S : s->d_planes;
  a.per_env = s->class_const ? 0 : 1;
  a.obs_every = 0;
  a.n_slots = s->S;
  a.ret = s->d_ret;
  a.status = s->d_status;
  a.ckpt_every = 1;
  cudaEventRecord(b.ev0, st);
  bool first = true;
  for (const G& g : groups) {
    a.seg_lo = g.lo; a.seg_hi = g.hi; a.tile_lo = g.tile_lo; a.n_tiles = g.tiles;
    a.tile_seg = s->d_tile_seg + g.tile_lo;
    launch_step(a, nullptr, nullptr, g.nt, g.var, std::min(g.tiles, 4 * s->num_sms), !first, false, st);
    first = false;
  }
  cudaEventRecord(b.ev1, st);
  // Requests whose last step this is: results into the pinned staging buffer.
  size_t stage = 0;
  for (Req* q : t.act) {
    q->steps_sched++;
    if (q->steps_sched >= q->r.horizon) {
      t.done.push_back(q);
      stage += (size_t)q->n4 * (14 + q->n_thr);
    }
  }
  if (stage > b.stage_floats) {
    if (b.h_stage) cudaFreeHost(b.h_stage);   // its last copies were waited for with this buffer's tick
    b.h_stage = nullptr;
    b.stage_floats = 0;
    if (cudaMallocHost(&b.h_stage, sizeof(float) * stage * 2) != cudaSuccess) {
      cudaGetLastError();
      std::lock_guard<std::mutex> lk(s->mu);
      s->fatal = MG_ERR_OOM;
      s->err = "tick: pinned staging allocation failed";
      return false;
    }
    b.stage_floats = stage * 2;
  }
  size_t off = 0;
  for (Req* q : t.done) {
    const size_t n = (size_t)q->n4 * (13 + q->n_thr);
    cudaMemcpyAsync(b.h_stage + off, s->d_state + q->st_off, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(b.h_stage + off + n, s->d_ret + q->slot_off, sizeof(float) * q->n4, cudaMemcpyDeviceToHost, st);
    off += n + q->n4;
  }
  cudaEventRecord(b.ev_done, st);
  return true;
}

// Wait for tick t and publish it: step counts, latency samples, and the
// results of the requests it finished.
static bool finish_tick(mg_server* s, const Tick& t) {
  TickBuf& b = s->buf[t.par];
  cudaError_t e = cudaEventSynchronize(b.ev1);
  const double t_end = now_s();
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b.ev0, b.ev1);
  if (e == cudaSuccess) e = cudaEventSynchronize(b.ev_done);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = MG_ERR_CUDA;
    s->err = std::string("tick: ") + cudaGetErrorString(e);
    return false;
  }
  // Unpack the finished requests (env-major, 21 floats per env).
  std::vector<std::vector<float>> states(t.done.size()), rets(t.done.size());
  size_t off = 0;
  for (size_t d = 0; d < t.done.size(); ++d) {
    const Req& q = *t.done[d];
    const int SS = 13 + q.n_thr, NF4 = SS / 4;
    const float* src = b.h_stage + off;
    std::vector<float>& fs = states[d];
    fs.assign((size_t)q.r.n_envs * 21, 0.0f);
    for (int64_t i = 0; i < q.r.n_envs; ++i)
      for (int j = 0; j < SS; ++j) {
        const int64_t o = (j < NF4 * 4) ? ((int64_t)(j / 4) * q.n4 + i) * 4 + (j % 4)
                                        : (int64_t)NF4 * 4 * q.n4 + (int64_t)(j - NF4 * 4) * q.n4 + i;
        fs[i * 21 + j] = src[o];
      }
    const float* r = src + (size_t)q.n4 * SS;
    rets[d].assign(r, r + q.r.n_envs);
    off += (size_t)q.n4 * (SS + 1);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const double spacing = s->last_tick_end > 0 ? t_end - s->last_tick_end : ms * 1e-3;
  s->last_tick_end = t_end;
  s->ticks++;
  s->env_steps += t.envs;
  s->busy += ms * 1e-3;
  s->tick.push_back({ms * 1e-3, 1.0});
  int n_cont = 0;
  for (Req* q : t.act) {
    // First step of a request admitted with this tick is measured from admission.
    if (q->steps_done == 0) s->lat.push_back({t_end - q->t_admit, 1.0});
    else ++n_cont;
    q->steps_done++;
  }
  if (n_cont > 0) s->lat.push_back({spacing, (double)n_cont});
  for (size_t d = 0; d < t.done.size(); ++d) {
    Req& q = *t.done[d];
    q.final_state.swap(states[d]);
    q.returns.swap(rets[d]);
    q.t_done = now_s();
    q.status = MG_REQ_DONE;
    s->requests_done++;
  }
  if (!t.done.empty()) {
    std::vector<Req*> keep;
    keep.reserve(s->active.size());
    for (Req* q : s->active)
      if (q->status != MG_REQ_DONE) keep.push_back(q);
    s->active.swap(keep);
  }
  return true;
}

static void scheduler(mg_server* s) {
  cudaSetDevice(s->device);
  Tick cur;   // the tick in flight
  int par = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || cur.valid || !s->pending.empty() || !s->active.empty(); });
      if (s->fatal != MG_OK) return;
      if (s->stop && !cur.valid) return;
    }
    // Prepare and enqueue the next tick while the current one runs.
    Tick nxt = prepare_tick(s, cur, par);
    if (nxt.valid && !enqueue_tick(s, nxt)) { s->cv.notify_all(); return; }
    if (cur.valid && !finish_tick(s, cur)) { s->cv.notify_all(); return; }
    cur = nxt;
    if (nxt.valid) par ^= 1;
    if (!cur.valid) {
      // Nothing in flight: wait for a submission (or a timeout to retry admission).
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->active.empty()) s->last_tick_end = 0;
      s->cv.notify_all();
      s->cv.wait_for(lk, std::chrono::milliseconds(1));
    }
    s->cv.notify_all();
  }
}

// Pinned tables, staging and events of the two tick buffers.
static bool alloc_tick_bufs(mg_server* s) {
  for (TickBuf& b : s->buf) {
    if (cudaMallocHost(&b.h_segs, sizeof(SegDesc) * s->cfg.max_requests) != cudaSuccess ||
        cudaMallocHost(&b.h_rsegs, sizeof(SegDesc) * s->cfg.max_requests) != cudaSuccess ||
        cudaMallocHost(&b.h_tile_seg, sizeof(int32_t) * s->tile_cap) != cudaSuccess ||
        cudaEventCreate(&b.ev0) != cudaSuccess || cudaEventCreate(&b.ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.ev_done, cudaEventDisableTiming) != cudaSuccess)
      return false;
  }
  return true;
}
static void free_tick_bufs(mg_server* s) {
  for (TickBuf& b : s->buf) {
    if (b.h_segs) cudaFreeHost(b.h_segs);
    if (b.h_rsegs) cudaFreeHost(b.h_rsegs);
    if (b.h_tile_seg) cudaFreeHost(b.h_tile_seg);
    if (b.h_stage) cudaFreeHost(b.h_stage);
    if (b.ev0) cudaEventDestroy(b.ev0);
    if (b.ev1) cudaEventDestroy(b.ev1);
    if (b.ev_done) cudaEventDestroy(b.ev_done);
    b = TickBuf();
  }
}

extern "C" {

const char* mg_server_last_error(const mg_server* s) { return s ? s->err.c_str() : "null server handle"; }

int mg_server_create(const mg_server_config* cfg, const mg_class_desc* classes, int32_t n_classes,
                     mg_server** out) {
  if (!out || !cfg || !classes || n_classes < 1 || n_classes > MG_MAX_CLASSES) return MG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(cfg->dt > 0) || cfg->max_requests < 1 || cfg->max_requests > 4096 || cfg->max_queue < 1)
    return MG_ERR_INVALID_ARG;
  if (cfg->integrator != MG_INTEG_EULER && cfg->integrator != MG_INTEG_RK4) return MG_ERR_INVALID_ARG;
  for (int c = 0; c < n_classes; ++c) {
    const mg_class_desc& d = classes[c];
    if (d.n_thr < 1 || d.n_thr > 8 || !(d.mass > 0) || d.rg[0] != 0 || d.rg[1] != 0 || d.rg[2] != 0)
      return MG_ERR_INVALID_ARG;
  }
  mg_server* s = new mg_server();
  s->cfg = *cfg;
  s->classes.assign(classes, classes + n_classes);
  for (int c = 0; c < n_classes; ++c)
    s->class_var.push_back(cfg->integrator == MG_INTEG_RK4 ? 2 : class_is_generic(classes[c]) ? 1 : 0);
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
  size_t budget = cfg->budget_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    budget = fr / 2;
  }
  // Per slot: 10 float4 planes + return; per state unit one float. A slot
  // holds at most 21 state floats, so size the spaces in that ratio.
  const size_t per_slot = sizeof(float4) * N_PLANES + sizeof(float) + 21 * sizeof(float);   // hover task: 10 planes
  int64_t S = (int64_t)(budget / per_slot) & ~int64_t(3);
  if (S < 4) { delete s; return MG_ERR_OOM; }
  s->S = S;
  s->state_cap = S * 21;
  s->budget = budget;
  s->class_const = !cfg->reset.dr_enabled && !cfg->reset.current_enabled;
  const size_t bytes = sizeof(float4) * N_PLANES * S + sizeof(float) * S + sizeof(float) * s->state_cap;
  auto cleanup = [&](int code) {
    if (s->arena) cudaFree(s->arena);
    if (s->d_cls) cudaFree(s->d_cls);
    if (s->d_nominal) cudaFree(s->d_nominal);
    if (s->d_segs) cudaFree(s->d_segs);
    if (s->d_rsegs) cudaFree(s->d_rsegs);
    if (s->d_status) cudaFree(s->d_status);
    free_tick_bufs(s);
    if (s->d_tile_seg) cudaFree(s->d_tile_seg);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return code;
  };
  if (cudaMalloc(&s->arena, bytes) != cudaSuccess) { cudaGetLastError(); return cleanup(MG_ERR_OOM); }
  s->d_planes = (float4*)s->arena;
  s->d_ret = (float*)(s->d_planes + (size_t)N_PLANES * S);
  s->d_state = s->d_ret + S;
  s->slots.reset(S);
  s->states.reset(s->state_cap);
  // Tiles of a tick: each request's slots rounded up to whole tiles.
  s->tile_cap = S / kThreads + cfg->max_requests;
  if (cudaMalloc(&s->d_tile_seg, sizeof(int32_t) * s->tile_cap) != cudaSuccess ||
      cudaMalloc(&s->d_cls, sizeof(ClassF) * n_classes) != cudaSuccess ||
      cudaMalloc(&s->d_nominal, sizeof(ClassNominal) * n_classes) != cudaSuccess ||
      cudaMalloc(&s->d_segs, sizeof(SegDesc) * cfg->max_requests) != cudaSuccess ||
      cudaMalloc(&s->d_rsegs, sizeof(SegDesc) * cfg->max_requests) != cudaSuccess ||
      cudaMalloc(&s->d_status, sizeof(uint32_t)) != cudaSuccess ||
      !alloc_tick_bufs(s)) {
    cudaGetLastError();
    return cleanup(MG_ERR_OOM);
  }
  std::vector<ClassF> cf(n_classes);
  std::vector<ClassNominal> cn(n_classes);
  for (int c = 0; c < n_classes; ++c) {
    const mg_class_desc& d = classes[c];
    ClassF& f = cf[c];
    std::memset(&f, 0, sizeof(f));
    double B[6][8];
    class_alloc_table(d, B);   // fixed propellers; zero columns for servos, fins and tilted propellers
    for (int i = 0; i < d.n_thr; ++i) {
      for (int k = 0; k < 6; ++k) f.alloc[k][i] = (float)B[k][i];
      f.kf[i] = (float)d.k_f[i];
      f.dz[i] = (float)d.deadzone[i];
    }
    f.gen = class_generic_table(d);
    // Nominal physics block (class-constant ticks), in the order of the
    // per-env parameter block; no current.
    const double Mrb[6] = {d.mass, d.mass, d.mass, d.Ig[0], d.Ig[1], d.Ig[2]};
    for (int j = 0; j < 6; ++j) {
      f.phys[PAR_MINV + j] = (float)(1.0 / (Mrb[j] + d.Ma[j]));
      f.phys[PAR_A + j] = (float)d.Ma[j];
      f.phys[PAR_DL + j] = (float)d.dl[j];
      f.phys[PAR_DQ + j] = (float)d.dq[j];
    }
    f.phys[PAR_M] = (float)d.mass;
    for (int j = 0; j < 3; ++j) { f.phys[PAR_IG + j] = (float)d.Ig[j]; f.phys[PAR_RB + j] = (float)d.rb[j]; }
    f.phys[PAR_W] = (float)(d.mass * kG);
    f.phys[PAR_B] = (float)(d.buoy_ratio * d.mass * kG);
    ClassNominal& n = cn[c];
    n.mass = d.mass;
    for (int j = 0; j < 3; ++j) { n.Ig[j] = d.Ig[j]; n.rb[j] = d.rb[j]; }
    n.B = d.buoy_ratio * d.mass * kG;
    for (int j = 0; j < 6; ++j) { n.Ma[j] = d.Ma[j]; n.dl[j] = d.dl[j]; n.dq[j] = d.dq[j]; }
  }
  for (int c = 0; c < n_classes; ++c) {   // tick kernels loaded before the first request
    const cudaError_t e = s->class_const ? prepare_tick_pm0(classes[c].n_thr, s->class_var[c])
                                         : prepare_tick_pm1(classes[c].n_thr, s->class_var[c]);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cleanup(MG_ERR_CUDA);
    }
  }
  if (cudaMemcpy(s->d_cls, cf.data(), sizeof(ClassF) * n_classes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_nominal, cn.data(), sizeof(ClassNominal) * n_classes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->d_status, 0, sizeof(uint32_t)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(MG_ERR_CUDA);
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return MG_OK;
}

int mg_server_submit(mg_server* s, const mg_request* r, int64_t* id_out) {
  if (!s || !r) return MG_ERR_INVALID_ARG;
  if (r->cls < 0 || r->cls >= (int)s->classes.size() || r->n_envs < 1 || r->horizon < 1 || r->K < 1 || r->K > 64)
    return sfail(s, MG_ERR_INVALID_ARG, "submit: bad request (class %d, n_envs %d, horizon %d, K %d)", r->cls,
                 r->n_envs, r->horizon, r->K);
  Req q;
  q.r = *r;
  q.n_thr = s->classes[r->cls].n_thr;
  q.n4 = (r->n_envs + 3) & ~3;
  if (q.n4 > s->S || state_units(q.n_thr, q.n4) > s->state_cap)
    return sfail(s, MG_ERR_ADMISSION_REFUSED, "submit: %d envs can never fit the %lld-slot arena", r->n_envs,
                 (long long)s->S);
  const double h = s->cfg.dt / r->K;
  q.h = (float)h;
  const mg_class_desc& d = s->classes[r->cls];
  for (int i = 0; i < d.n_thr; ++i)
    if (d.deadzone[i] != 0.0) q.dz = 1;
  for (int i = 0; i < 8; ++i)
    q.alpha[i] = (i < d.n_thr && d.T_rotor[i] > 0) ? (float)(1.0 - std::exp(-h / d.T_rotor[i])) : 1.0f;
  q.t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != MG_OK) return sfail(s, s->fatal, "server stopped: %s", s->err.c_str());
  if ((int)s->pending.size() >= s->cfg.max_queue)
    return sfail(s, MG_ERR_ADMISSION_REFUSED, "submit: queue full (%d pending)", (int)s->pending.size());
  q.id = s->next_id++;
  s->reqs[q.id] = q;
  s->pending.push_back(q.id);
  if (id_out) *id_out = q.id;
  s->cv.notify_all();
  return MG_OK;
}

int mg_server_poll(mg_server* s, int64_t id, mg_request_result* out) {
  if (!s || !out) return MG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) {
    out->status = MG_REQ_UNKNOWN;
    return MG_OK;
  }
  const Req& q = it->second;
  out->status = q.status;
  out->n_envs = q.r.n_envs;
  out->t_submit = q.t_submit;
  out->t_admit = q.t_admit;
  out->t_done = q.t_done;
  out->steps_done = q.steps_done;
  if (q.status == MG_REQ_DONE) {
    out->final_state = q.final_state.data();
    out->returns = q.returns.data();
  }
  return MG_OK;
}

int mg_server_release(mg_server* s, int64_t id) {
  if (!s) return MG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.status != MG_REQ_DONE)
    return sfail(s, MG_ERR_STATE, "release: request %lld is not done", (long long)id);
  s->reqs.erase(it);
  return MG_OK;
}

int mg_server_wait_idle(mg_server* s, double timeout_s) {
  if (!s) return MG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return (s->pending.empty() && s->active.empty()) || s->fatal != MG_OK;
  });
  if (s->fatal != MG_OK) return s->fatal;
  return ok ? MG_OK : sfail(s, MG_ERR_TIMEOUT, "wait_idle: %d pending, %d active after %.1f s",
                            (int)s->pending.size(), (int)s->active.size(), timeout_s);
}

int mg_server_stats_get(mg_server* s, mg_server_stats* out) {
  if (!s || !out) return MG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->requests_done = s->requests_done;
  out->env_steps = s->env_steps;
  out->ticks = s->ticks;
  out->busy_seconds = s->busy;
  out->step_latency_p50 = wquantile(s->lat, 0.50);
  out->step_latency_p99 = wquantile(s->lat, 0.99);
  out->queue_delay_p50 = wquantile(s->qdel, 0.50);
  out->queue_delay_p99 = wquantile(s->qdel, 0.99);
  out->tick_p50 = wquantile(s->tick, 0.50);
  out->tick_p99 = wquantile(s->tick, 0.99);
  out->budget_bytes = s->budget;
  out->peak_resident_bytes = s->peak_resident;
  out->peak_requests = s->peak_requests;
  return MG_OK;
}

int mg_server_destroy(mg_server* s) {
  if (!s) return MG_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaStreamSynchronize(s->stream);
  cudaFree(s->arena);
  cudaFree(s->d_cls);
  cudaFree(s->d_nominal);
  cudaFree(s->d_segs);
  cudaFree(s->d_rsegs);
  cudaFree(s->d_status);
  free_tick_bufs(s);
  cudaFree(s->d_tile_seg);
  cudaStreamDestroy(s->stream);
  delete s;
  return MG_OK;
}

}  // extern "C"
