// Host runtime of libmarinegym: validation, layout, device buffers, launches,
// checkpoint/resume, CUDA-graph capture and the launch-shape autotuner. All
// per-class derived quantities (allocation matrix, rotor factor, inverse
// inertia) are computed here in FP64 and stored FP32 for the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/marinegym.h"
#include "mg_internal.h"
#include "mg_payload.h"

namespace mg {
cudaError_t launch_step(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                        bool dependent, bool shared_sm, cudaStream_t st);
cudaError_t launch_reset(const ResetArgs& a, cudaStream_t st);
cudaError_t launch_set_hydro(float4* planes, int64_t n_slots, const float* A, const float* dl, const float* dq,
                             cudaStream_t st);
cudaError_t launch_adjoint(const AdjArgs& a, const ClassK& kc, const ClassG* kg, int nt, int var, bool dependent,
                           cudaStream_t st, const void* jit_kernel);
cudaError_t step_kernel_occupancy(int nt, int pm, int var, bool kp, bool track, int* blocks_per_sm);
cudaError_t launch_pair(const StepArgs& a, const ClassK& kc, int nt, bool dependent, cudaStream_t st);
const void* jit_step_kernel(const ClassK& k, int nt, bool ms, int pm, int min_blocks, std::string* err);
int jit_step_min_blocks(int K, int n_tiles, int num_sms);
const void* jit_adjoint_kernel(const ClassK& k, int nt, std::string* err);
cudaError_t launch_step_jit(const void* kern, const StepArgs& a, const ClassK& kc, int nt, int pm, int grid, bool dependent,
                            bool shared_sm, cudaStream_t st);
size_t step_kernel_smem_jit(int nt, int pm);
}  // namespace mg

namespace mg {
cudaError_t launch_fp64(const Fp64Args& a, int nt, int var, int block, cudaStream_t st);
}  // namespace mg

using namespace mg;

static const double kG = 9.81;
static thread_local std::string g_create_err;

struct ClassLay {
  int32_t n_envs, n_thr, env_off, slot_off, n4;
  int64_t st_off, act_off;
};

// Segments with the same thruster count and step variant (0 propellers with
// Euler, 1 generic actuators with Euler, 2 RK4), launched by one kernel
// instantiation. A launch of the step plan with cls >= 0 holds envs of that
// one class and passes its class tables as the kernel parameter (the groups
// of the segment layout have cls = -1).
struct Group {
  int32_t nt, seg_lo, seg_hi, tile_lo, n_tiles, var, cls;
};

struct mg_sim {
  mg_config cfg;
  std::vector<int32_t> counts;
  std::vector<mg_class_desc> classes;
  std::vector<ClassLay> lay;
  int32_t n_classes = 0, n_envs = 0, n_slots = 0;
  int64_t act_floats = 0, state_floats = 0;
  int32_t threads = 128;
  int32_t blocks_per_sm = 0;   // persistent blocks per SM (0: occupancy limit)
  int32_t lanes = 1;           // lanes per env of eligible launches (1 or 2)
  int32_t specialise = 1;      // class-specialised kernels for one-class propeller launches (when available)
  int32_t num_sms = 148;
  int32_t n_tiles = 0, n_segs = 0;
  double h = 0.0;
  std::vector<SegDesc> segs;
  std::vector<Group> groups;
  // device
  float* d_state = nullptr;
  float4* d_planes = nullptr;
  int32_t n_planes = 0;
  ClassF* d_cls = nullptr;
  ClassG* d_gen = nullptr;
  ClassGD* d_gen64 = nullptr;   // the generic tables in FP64 (check path)
  ClassD* d_cls64 = nullptr;
  ClassNominal* d_nominal = nullptr;
  SegDesc* d_segs = nullptr;
  uint32_t* d_status = nullptr;
  float* d_ckpt = nullptr;
  float* d_scratch = nullptr;
  float* d_stage = nullptr;
  size_t stage_floats = 0;
  int32_t ckpt_every = 20;
  int32_t rec_T = 0;           // steps of the last recorded rollout (0: none)
  uint64_t rec_id = 0;         // identity of that recording (0: none)
  size_t bytes = 0;
  std::string err;
  // Launch plan of a step (grids, launch shape, carveouts), computed once per
  // segment layout and blocks_per_sm setting: a step only reads it.
  struct Plan {
    bool valid = false;
    int bps = -1;
    bool cores = false;
    std::vector<int> grid;
    std::vector<int> full_grid;   // persistent grid of each group launched alone
    std::vector<char> carve_max;
    std::vector<Group> groups;     // the launches of a step
    bool first_pdl = false;        // the first launch is a programmatic dependent too
    std::vector<ClassK> kc;        // constants of each launch with cls >= 0
    // Class-specialised kernels of each launch ([0] single-step, [1]
    // multi-step instantiation), compiled on first use; null: none.
    std::vector<const void*> jit[2];
    std::vector<char> jit_tried[2];
    std::vector<int> jit_grid[2];
  } plan, plan_ms;                 // single-step launches; multi-step launches
  std::string jit_err;             // why the last specialised kernel could not be had
  std::vector<ClassF> h_cls;       // host copies of the class tables
  std::vector<ClassG> h_gen;
  // mg_step_host: copy streams and events of the chunked pipeline.
  cudaStream_t s_in = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> host_ev;
};

struct mg_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  mg_sim* sim = nullptr;        // a replay advances this simulator's envs
};

// Recordings for mg_step_backward. A recording is valid only while the
// simulator still holds what produced it: every call that changes the state,
// the per-env parameters, the task or the payload (or runs a step, a reset or
// a graph replay) discards it, so that a backward pass never differentiates
// old checkpoints with new parameters. Each recording gets a process-unique
// identity that callers (the autograd wrapper) keep to detect a newer one.
static std::atomic<uint64_t> g_next_rec_id{1};
static void drop_recording(mg_sim* sim) {
  sim->rec_T = 0;
  sim->rec_id = 0;
}

static int fail(mg_sim* s, int code, const char* fmt, ...) {
  if (s) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    s->err = buf;
  }
  return code;
}

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(sim, MG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

static bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

static int validate_class(mg_sim* sim, const mg_class_desc& c, int ci) {
  if (c.n_thr < 1 || c.n_thr > MG_MAX_THR) return fail(sim, MG_ERR_INVALID_ARG, "class %d: n_thr %d not in 1..8", ci, c.n_thr);
  if (!(std::isfinite(c.mass) && c.mass > 0)) return fail(sim, MG_ERR_INVALID_ARG, "class %d: mass must be > 0", ci);
  for (int i = 0; i < 3; ++i) {
    if (!(std::isfinite(c.Ig[i]) && c.Ig[i] > 0)) return fail(sim, MG_ERR_INVALID_ARG, "class %d: inertia must be > 0", ci);
    if (c.rg[i] != 0.0) return fail(sim, MG_ERR_INVALID_ARG, "class %d: r_g != 0 is not supported", ci);
    if (!std::isfinite(c.rb[i])) return fail(sim, MG_ERR_INVALID_ARG, "class %d: r_b not finite", ci);
  }
  if (!finite_nonneg(c.buoy_ratio)) return fail(sim, MG_ERR_INVALID_ARG, "class %d: buoy_ratio", ci);
  for (int i = 0; i < 6; ++i)
    if (!finite_nonneg(c.Ma[i]) || !finite_nonneg(c.dl[i]) || !finite_nonneg(c.dq[i]))
      return fail(sim, MG_ERR_INVALID_ARG, "class %d: added mass / damping must be finite and >= 0", ci);
  for (int i = 0; i < c.n_thr; ++i) {
    if (!finite_nonneg(c.k_f[i]) || !finite_nonneg(c.T_rotor[i]) || !finite_nonneg(c.deadzone[i]))
      return fail(sim, MG_ERR_INVALID_ARG, "class %d thruster %d: k_f, T_rotor, deadzone must be >= 0", ci, i);
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(c.thr_pos[i][k]) || !std::isfinite(c.thr_dir[i][k]) || !std::isfinite(c.act_axis[i][k]) ||
          !std::isfinite(c.act_chord[i][k]))
        return fail(sim, MG_ERR_INVALID_ARG, "class %d thruster %d: geometry not finite", ci, i);
    const int kind = c.act_kind[i];
    if (kind < MG_ACT_PROP || kind > MG_ACT_TILT)
      return fail(sim, MG_ERR_INVALID_ARG, "class %d channel %d: unknown actuator kind %d", ci, i, kind);
    auto norm = [](const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); };
    auto unit = [&](const double* v) { return std::fabs(norm(v) - 1.0) <= 1e-9; };
    if (kind == MG_ACT_SERVO || kind == MG_ACT_FIN)
      if (!(std::isfinite(c.act_range[i]) && c.act_range[i] > 0.0))
        return fail(sim, MG_ERR_INVALID_ARG, "class %d channel %d: act_range must be > 0", ci, i);
    if (kind == MG_ACT_FIN) {
      const double* a = c.act_axis[i];
      const double* ch = c.act_chord[i];
      if (!unit(a) || !unit(ch) || std::fabs(a[0] * ch[0] + a[1] * ch[1] + a[2] * ch[2]) > 1e-9)
        return fail(sim, MG_ERR_INVALID_ARG, "class %d fin %d: span axis and chord must be orthogonal unit vectors", ci, i);
      if (!finite_nonneg(c.fin_area[i]) || !std::isfinite(c.fin_cl[i]) || !finite_nonneg(c.fin_cd0[i]) ||
          !finite_nonneg(c.fin_cda[i]) || !(std::isfinite(c.rho) && c.rho > 0.0))
        return fail(sim, MG_ERR_INVALID_ARG, "class %d fin %d: area, drag >= 0, lift slope finite, rho > 0", ci, i);
    }
    if (kind == MG_ACT_TILT) {
      const int j = c.act_link[i];
      if (j < 0 || j >= c.n_thr || c.act_kind[j] != MG_ACT_SERVO)
        return fail(sim, MG_ERR_INVALID_ARG, "class %d channel %d: act_link must name a servo channel", ci, i);
      if (!unit(c.act_axis[i])) return fail(sim, MG_ERR_INVALID_ARG, "class %d channel %d: tilt axis must be a unit vector", ci, i);
    }
  }
  return MG_OK;
}

// A class with any channel other than a fixed propeller.
static bool generic_class(const mg_class_desc& c) {
  for (int i = 0; i < c.n_thr; ++i)
    if (c.act_kind[i] != MG_ACT_PROP) return true;
  return false;
}

// Generic actuator table of a class (FP64 geometry, stored as GT: ClassG in
// FP32 for the kernels, ClassGD in FP64 for the check path): fins
// e1, e2 = a x e1, r x e1, r x e2, 1/2 rho S (C_L_alpha, C_D0, C_D_alpha),
// range; tilted propellers B0 = [d ; r x d], B1 = [a x d ; r x (a x d)],
// B2 = (a . d) [a ; r x a], servo channel, servo range.
template <typename GT>
static GT generic_table(const mg_class_desc& c) {
  using V = tt::decay_t<decltype(GT::v[0][0])>;
  GT g;
  std::memset(&g, 0, sizeof(g));
  auto crs = [](const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0];
  };
  for (int i = 0; i < c.n_thr; ++i) {
    g.kind[i] = c.act_kind[i];
    const double* r = c.thr_pos[i];
    const double* a = c.act_axis[i];
    if (c.act_kind[i] == MG_ACT_FIN) {
      const double* e1 = c.act_chord[i];
      double e2[3], re1[3], re2[3];
      crs(a, e1, e2);
      crs(r, e1, re1);
      crs(r, e2, re2);
      for (int k = 0; k < 3; ++k) {
        g.v[i][k] = (V)e1[k]; g.v[i][3 + k] = (V)e2[k];
        g.v[i][6 + k] = (V)re1[k]; g.v[i][9 + k] = (V)re2[k];
      }
      const double qS = 0.5 * c.rho * c.fin_area[i];
      g.v[i][12] = (V)(qS * c.fin_cl[i]);
      g.v[i][13] = (V)(qS * c.fin_cd0[i]);
      g.v[i][14] = (V)(qS * c.fin_cda[i]);
      g.v[i][15] = (V)c.act_range[i];
    } else if (c.act_kind[i] == MG_ACT_TILT) {
      const double* d = c.thr_dir[i];
      double rd[3], ad[3], rad[3], ra[3];
      crs(r, d, rd);
      crs(a, d, ad);
      crs(r, ad, rad);
      crs(r, a, ra);
      const double adot = a[0] * d[0] + a[1] * d[1] + a[2] * d[2];
      for (int k = 0; k < 3; ++k) {
        g.v[i][k] = (V)d[k]; g.v[i][3 + k] = (V)rd[k];
        g.v[i][6 + k] = (V)ad[k]; g.v[i][9 + k] = (V)rad[k];
        g.v[i][12 + k] = (V)(adot * a[k]); g.v[i][15 + k] = (V)(adot * ra[k]);
      }
      g.v[i][18] = (V)c.act_link[i];
      g.v[i][19] = (V)c.act_range[c.act_link[i]];
    }
  }
  return g;
}

static void alpha_of(const mg_class_desc& c, double h, double* a) {
  for (int i = 0; i < 8; ++i) a[i] = 1.0;
  for (int i = 0; i < c.n_thr; ++i) a[i] = c.T_rotor[i] > 0.0 ? 1.0 - std::exp(-h / c.T_rotor[i]) : 1.0;
}

// Allocation matrix B = [d_i ; r_i x d_i] of the fixed propellers (FP64);
// the columns of other channels are zero.
static void alloc_of(const mg_class_desc& c, double B[6][8]) {
  for (int k = 0; k < 6; ++k) for (int i = 0; i < 8; ++i) B[k][i] = 0.0;
  for (int i = 0; i < c.n_thr; ++i) {
    if (c.act_kind[i] != MG_ACT_PROP) continue;
    const double* r = c.thr_pos[i];
    const double* d = c.thr_dir[i];
    B[0][i] = d[0]; B[1][i] = d[1]; B[2][i] = d[2];
    B[3][i] = r[1] * d[2] - r[2] * d[1];
    B[4][i] = r[2] * d[0] - r[0] * d[2];
    B[5][i] = r[0] * d[1] - r[1] * d[0];
  }
}

// Class tables shared with the serving loop: the fixed-propeller allocation
// columns (zero for the other channels), the generic actuator table, and
// whether a class has channels other than fixed propellers.
void class_alloc_table(const mg_class_desc& c, double B[6][8]) { alloc_of(c, B); }
ClassG class_generic_table(const mg_class_desc& c) { return generic_table<ClassG>(c); }
bool class_is_generic(const mg_class_desc& c) { return generic_class(c); }

// Step variant of a class: 2 with the RK4 integrator, else 1 for a generic
// class, 0 for a propeller-only class.
static int class_var(const mg_sim* sim, int c) {
  if (sim->cfg.integrator == MG_INTEG_RK4) return 2;
  return generic_class(sim->classes[c]) ? 1 : 0;
}

// Segments ordered by step variant, then thruster count (then class); tiles
// are numbered in that order so that each group owns one contiguous tile range.
// Launches of a single class pass its class tables as the kernel parameter
// (0: always staged in shared memory).
#ifndef MG_CLASS_PARAMS
#define MG_CLASS_PARAMS 1
#endif

static void build_segs(mg_sim* sim) {
  sim->segs.clear();
  sim->groups.clear();
  sim->plan.valid = false;
  sim->plan_ms.valid = false;
  int tiles = 0;
  for (int var = 0; var < 3; ++var)
  for (int nt = 1; nt <= MG_MAX_THR; ++nt) {
    Group g;
    g.nt = nt;
    g.var = var;
    g.seg_lo = (int32_t)sim->segs.size();
    g.tile_lo = tiles;
    for (int c = 0; c < sim->n_classes; ++c) {
      const ClassLay& L = sim->lay[c];
      if (L.n_envs == 0 || L.n_thr != nt || class_var(sim, c) != var) continue;
      SegDesc sd;
      std::memset(&sd, 0, sizeof(sd));
      sd.tile_begin = tiles;
      sd.n_envs = L.n_envs;
      sd.cls = c;
      sd.n_thr = L.n_thr;
      sd.K = sim->cfg.K;
      sd.n4 = L.n4;
      sd.st_off = L.st_off;
      sd.act_off = L.act_off;
      sd.slot_off = L.slot_off;
      sd.env_base = L.env_off;
      sd.h = (float)sim->h;
      sd.dt = (float)sim->cfg.dt;
      sd.track = sim->cfg.task == 1;
      sd.flags = 0;
      for (int i = 0; i < L.n_thr; ++i)
        if (sim->classes[c].deadzone[i] != 0.0) sd.flags |= 1;
      double a[8];
      alpha_of(sim->classes[c], sim->h, a);
      for (int i = 0; i < 8; ++i) sd.alpha[i] = (float)a[i];
      tiles += (L.n4 + sim->threads - 1) / sim->threads;
      sim->segs.push_back(sd);
    }
    g.seg_hi = (int32_t)sim->segs.size();
    g.n_tiles = tiles - g.tile_lo;
    g.cls = -1;
    if (g.seg_hi > g.seg_lo) sim->groups.push_back(g);
  }
  sim->n_tiles = tiles;
  sim->n_segs = (int32_t)sim->segs.size();
}

static int upload_segs(mg_sim* sim) {
  build_segs(sim);
  CK(cudaMemcpy(sim->d_segs, sim->segs.data(), sizeof(SegDesc) * sim->segs.size(), cudaMemcpyHostToDevice));
  return MG_OK;
}

static int dev_alloc(mg_sim* sim, void** p, size_t bytes) {
  if (sim->cfg.mem_budget && sim->bytes + bytes > sim->cfg.mem_budget)
    return fail(sim, MG_ERR_OOM, "device memory budget of %zu bytes exceeded (%zu needed)", sim->cfg.mem_budget,
                sim->bytes + bytes);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(sim, MG_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  sim->bytes += bytes;
  return MG_OK;
}

static void free_all(mg_sim* sim) {
  void* ps[] = {sim->d_state, sim->d_planes, sim->d_cls, sim->d_gen, sim->d_gen64, sim->d_cls64, sim->d_nominal,
                sim->d_segs, sim->d_status, sim->d_ckpt, sim->d_scratch, sim->d_stage};
  for (void* p : ps)
    if (p) cudaFree(p);
}

static ResetArgs reset_args(mg_sim* sim, const mg_reset_cfg& r, uint64_t seed) {
  ResetArgs a;
  std::memset(&a, 0, sizeof(a));
  a.segs = sim->d_segs;
  a.n_segs = sim->n_segs;
  a.nominal = sim->d_nominal;
  a.per_env = sim->cfg.per_env_params;
  a.state = sim->d_state;
  a.planes = sim->d_planes;
  a.n_slots = sim->n_slots;
  a.seed = seed;
  a.dr = r.dr_enabled;
  a.cur = r.current_enabled;
  a.cur3d = r.current_3d;
  a.init_mode = r.init_mode;
  a.mass_lo = r.mass_lo; a.mass_hi = r.mass_hi;
  a.added_lo = r.added_lo; a.added_hi = r.added_hi;
  a.damp_lo = r.damp_lo; a.damp_hi = r.damp_hi;
  a.cob_lo = r.cob_lo; a.cob_hi = r.cob_hi;
  a.cur_lo = r.cur_lo; a.cur_hi = r.cur_hi;
  a.target_half = r.target_half; a.pos_radius = r.pos_radius; a.max_angle = r.max_angle;
  a.track = sim->cfg.task == 1;
  a.track_kind = r.track_kind;
  a.payload = sim->cfg.payload;
  a.payload_lo = r.payload_lo;
  a.payload_hi = r.payload_hi;
  return a;
}

extern "C" {

const char* mg_strerror(int code) {
  switch (code) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_OOM: return "out of device memory or over budget";
    case MG_ERR_CUDA: return "CUDA runtime error";
    case MG_ERR_NONFINITE: return "non-finite state";
    case MG_ERR_TIMEOUT: return "bounded wait timed out";
    case MG_ERR_ADMISSION_REFUSED: return "admission refused";
    case MG_ERR_STATE: return "invalid call order";
    default: return "unknown error";
  }
}

const char* mg_last_error(const mg_sim* sim) { return sim ? sim->err.c_str() : g_create_err.c_str(); }

int mg_create(const mg_config* cfg, const mg_class_desc* classes, mg_sim** out) {
  if (!out) return MG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || !classes || !cfg->class_counts) return MG_ERR_INVALID_ARG;
  mg_sim* sim = new mg_sim();
  sim->cfg = *cfg;
  auto bail = [&](int code) {
    // keep the handle alive only on success; report the message on stderr-free path
    free_all(sim);
    g_create_err = sim->err.empty() ? mg_strerror(code) : sim->err;
    delete sim;
    return code;
  };
  if (cfg->n_classes < 1 || cfg->n_classes > MG_MAX_CLASSES) return bail(MG_ERR_INVALID_ARG);
  if (!(std::isfinite(cfg->dt) && cfg->dt > 0)) return bail(MG_ERR_INVALID_ARG);
  if (cfg->K < 1 || cfg->K > 64) return bail(MG_ERR_INVALID_ARG);
  if (cfg->record_steps < 0 || cfg->ckpt_every < 0) return bail(MG_ERR_INVALID_ARG);
  if (!cfg->per_env_params && (cfg->reset.dr_enabled || cfg->reset.current_enabled || cfg->record_steps > 0))
    return bail(MG_ERR_INVALID_ARG);
  if (cfg->task < 0 || cfg->task > 1 || cfg->reset.track_kind < 0 || cfg->reset.track_kind > 1)
    return bail(MG_ERR_INVALID_ARG);
  if (cfg->payload < 0 || cfg->payload > 1) return bail(MG_ERR_INVALID_ARG);
  if (cfg->integrator != MG_INTEG_EULER && cfg->integrator != MG_INTEG_RK4) {
    sim->err = "integrator must be MG_INTEG_EULER or MG_INTEG_RK4";
    return bail(MG_ERR_INVALID_ARG);
  }
  if (cfg->payload) {
    if (!cfg->per_env_params) {
      sim->err = "payload runs need per_env_params";
      return bail(MG_ERR_INVALID_ARG);
    }
    const double lo = cfg->reset.payload_lo, hi = cfg->reset.payload_hi;
    if (!(std::isfinite(lo) && std::isfinite(hi) && lo >= 0.0 && hi >= lo)) {
      sim->err = "payload range must satisfy 0 <= payload_lo <= payload_hi";
      return bail(MG_ERR_INVALID_ARG);
    }
  }
  sim->n_classes = cfg->n_classes;
  sim->classes.assign(classes, classes + cfg->n_classes);
  sim->counts.assign(cfg->class_counts, cfg->class_counts + cfg->n_classes);
  for (int c = 0; c < sim->n_classes; ++c) {
    if (validate_class(sim, sim->classes[c], c) != MG_OK) return bail(MG_ERR_INVALID_ARG);
    if (sim->counts[c] < 0) return bail(MG_ERR_INVALID_ARG);
  }
  sim->h = cfg->dt / cfg->K;
  sim->ckpt_every = cfg->ckpt_every > 0 ? cfg->ckpt_every : 20;
  int64_t env = 0, slot = 0, st = 0, act = 0;
  for (int c = 0; c < sim->n_classes; ++c) {
    ClassLay L;
    L.n_envs = sim->counts[c];
    L.n_thr = sim->classes[c].n_thr;
    L.env_off = (int32_t)env;
    L.slot_off = (int32_t)slot;
    L.n4 = (L.n_envs + 3) & ~3;
    L.st_off = st;
    L.act_off = act;
    env += L.n_envs;
    slot += L.n4;
    st += (int64_t)L.n4 * (13 + L.n_thr);
    act += (int64_t)L.n4 * L.n_thr;
    sim->lay.push_back(L);
  }
  if (env == 0 || slot > (int64_t)1 << 30) return bail(MG_ERR_INVALID_ARG);
  sim->n_envs = (int32_t)env;
  sim->n_slots = (int32_t)slot;
  sim->state_floats = st;
  sim->act_floats = act;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) { fail(sim, MG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce)); return bail(MG_ERR_CUDA); }
  cudaDeviceGetAttribute(&sim->num_sms, cudaDevAttrMultiProcessorCount, dev);

  sim->n_planes = n_planes_of(cfg->per_env_params, cfg->task == 1, cfg->payload);
  int rc;
  if ((rc = dev_alloc(sim, (void**)&sim->d_state, sizeof(float) * st)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_planes, sizeof(float4) * sim->n_planes * slot)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_cls, sizeof(ClassF) * sim->n_classes)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_gen, sizeof(ClassG) * sim->n_classes)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_gen64, sizeof(ClassGD) * sim->n_classes)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_cls64, sizeof(ClassD) * sim->n_classes)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_nominal, sizeof(ClassNominal) * sim->n_classes)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_segs, sizeof(SegDesc) * MG_MAX_CLASSES)) != MG_OK) return bail(rc);
  if ((rc = dev_alloc(sim, (void**)&sim->d_status, sizeof(uint32_t))) != MG_OK) return bail(rc);
  if (cfg->record_steps > 0) {
    const int64_t n_ck = (cfg->record_steps + sim->ckpt_every - 1) / sim->ckpt_every;
    if ((rc = dev_alloc(sim, (void**)&sim->d_ckpt, sizeof(float) * n_ck * 21 * slot)) != MG_OK) return bail(rc);
    const size_t n_scr = adjoint_scratch_floats(sim->ckpt_every, cfg->K, slot);
    if ((rc = dev_alloc(sim, (void**)&sim->d_scratch, sizeof(float) * n_scr)) != MG_OK) return bail(rc);
  }
  {
    cudaError_t e1 = cudaMemset(sim->d_state, 0, sizeof(float) * st);
    cudaError_t e2 = cudaMemset(sim->d_planes, 0, sizeof(float4) * sim->n_planes * slot);
    cudaError_t e3 = cudaMemset(sim->d_status, 0, sizeof(uint32_t));
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
      fail(sim, MG_ERR_CUDA, "cudaMemset failed");
      return bail(MG_ERR_CUDA);
    }
  }
  // Class tables.
  std::vector<ClassF> cf(sim->n_classes);
  std::vector<ClassD> cd(sim->n_classes);
  std::vector<ClassNominal> cn(sim->n_classes);
  std::vector<ClassG> cg(sim->n_classes);
  std::vector<ClassGD> cgd(sim->n_classes);
  for (int c = 0; c < sim->n_classes; ++c) {
    const mg_class_desc& d = sim->classes[c];
    cg[c] = generic_table<ClassG>(d);
    cgd[c] = generic_table<ClassGD>(d);
    double B[6][8], al[8];
    alloc_of(d, B);
    alpha_of(d, sim->h, al);
    ClassF& f = cf[c];
    ClassD& g = cd[c];
    std::memset(&f, 0, sizeof(f));
    std::memset(&g, 0, sizeof(g));
    f.gen = cg[c];
    for (int k = 0; k < 6; ++k)
      for (int i = 0; i < 8; ++i) { f.alloc[k][i] = (float)B[k][i]; g.alloc[k][i] = B[k][i]; }
    for (int i = 0; i < 8; ++i) {
      const bool on = i < d.n_thr;
      f.kf[i] = on ? (float)d.k_f[i] : 0.0f; g.kf[i] = on ? d.k_f[i] : 0.0;
      f.dz[i] = on ? (float)d.deadzone[i] : 0.0f; g.dz[i] = on ? d.deadzone[i] : 0.0;
      g.alpha[i] = al[i];
    }
    const double Mrb[6] = {d.mass, d.mass, d.mass, d.Ig[0], d.Ig[1], d.Ig[2]};
    for (int j = 0; j < 6; ++j) {
      g.Mrb[j] = Mrb[j];
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
  sim->h_cls = cf;
  sim->h_gen = cg;
  ce = cudaMemcpy(sim->d_cls, cf.data(), sizeof(ClassF) * cf.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(sim->d_cls64, cd.data(), sizeof(ClassD) * cd.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(sim->d_nominal, cn.data(), sizeof(ClassNominal) * cn.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(sim->d_gen, cg.data(), sizeof(ClassG) * cg.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(sim->d_gen64, cgd.data(), sizeof(ClassGD) * cgd.size(), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) { fail(sim, MG_ERR_CUDA, "class upload: %s", cudaGetErrorString(ce)); return bail(MG_ERR_CUDA); }
  if ((rc = upload_segs(sim)) != MG_OK) return bail(rc);
  // Rest state with nominal parameters.
  mg_reset_cfg rest;
  std::memset(&rest, 0, sizeof(rest));
  ResetArgs ra = reset_args(sim, rest, 0);
  ra.n_sel = sim->n_envs;
  ce = launch_reset(ra, 0);
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) { fail(sim, MG_ERR_CUDA, "initial reset: %s", cudaGetErrorString(ce)); return bail(MG_ERR_CUDA); }
  *out = sim;
  return MG_OK;
}

int mg_destroy(mg_sim* sim) {
  if (!sim) return MG_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : sim->host_ev) cudaEventDestroy(e);
  if (sim->s_in) cudaStreamDestroy(sim->s_in);
  if (sim->s_out) cudaStreamDestroy(sim->s_out);
  free_all(sim);
  delete sim;
  return MG_OK;
}

static const mg_sim::Plan& step_plan(mg_sim* sim, bool ms = false);

int mg_get_layout(const mg_sim* sim, mg_layout* out) {
  if (!sim || !out) return MG_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->n_classes = sim->n_classes;
  out->n_envs = sim->n_envs;
  out->n_slots = sim->n_slots;
  out->launches_per_step = (int32_t)step_plan(const_cast<mg_sim*>(sim)).groups.size();
  out->action_floats = sim->act_floats;
  out->state_floats = sim->state_floats;
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    mg_class_layout& o = out->cls[c];
    o.n_envs = L.n_envs; o.n_thr = L.n_thr; o.env_offset = L.env_off; o.slot_offset = L.slot_off;
    o.state_offset = L.st_off; o.state_stride = 13 + L.n_thr; o.action_offset = L.act_off;
  }
  return MG_OK;
}

int mg_reset(mg_sim* sim, const int32_t* env_ids_dev, int32_t n, uint64_t seed, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (env_ids_dev && (n < 0 || n > sim->n_envs)) return fail(sim, MG_ERR_INVALID_ARG, "reset: bad env count %d", n);
  ResetArgs a = reset_args(sim, sim->cfg.reset, seed);
  a.env_ids = env_ids_dev;
  a.n_sel = env_ids_dev ? n : sim->n_envs;
  CK(launch_reset(a, (cudaStream_t)stream));
  drop_recording(sim);
  return MG_OK;
}

// Parameter source of the step kernel: 0 class constants, 1 per-env planes,
// 2 per-env planes plus the payload planes.
static int param_mode(const mg_sim* sim) { return sim->cfg.payload ? 2 : (sim->cfg.per_env_params ? 1 : 0); }

// Kernel-parameter constants of a one-class group: the class table, the lag
// coefficients and dead-zone flag of its segment, no current.
// Class tables of group g as the kernel parameter. Step kernels of
// class-constant and payload runs take allocation rows premultiplied by the
// thrust constants (as their Premul); the adjoint (for_adjoint) always takes
// plain rows, its product applies k itself.
static ClassK class_k(const mg_sim* sim, const Group& g, bool for_adjoint = false) {
  ClassK k;
  std::memset(&k, 0, sizeof(k));
  const ClassF& f = sim->h_cls[g.cls];
  const SegDesc& sd = sim->segs[g.seg_lo];
  std::memcpy(k.alloc, f.alloc, sizeof(k.alloc));
  if (!for_adjoint && MG_PREMUL && g.var == 0 && param_mode(sim) != 1)   // as the kernels' Premul: rows of B diag(k)
    for (int r = 0; r < 6; ++r)
      for (int i = 0; i < 8; ++i) k.alloc[r][i] = f.alloc[r][i] * f.kf[i];
  std::memcpy(k.kf, f.kf, sizeof(k.kf));
  std::memcpy(k.dz, f.dz, sizeof(k.dz));
  std::memcpy(k.alpha, sd.alpha, sizeof(k.alpha));
  std::memcpy(k.minv, f.phys, sizeof(float) * PAR_DIM);
  for (int j = 0; j < 3; ++j) k.Vc[j] = 0.0f;
  k.dz_on = (uint32_t)(sd.flags & 1);
  return k;
}

static StepArgs step_args(mg_sim* sim) {
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.segs = sim->d_segs;
  a.classes = sim->d_cls;
  a.state = sim->d_state;
  a.act_stride = sim->act_floats;
  a.planes = sim->d_planes;
  a.per_env = param_mode(sim);
  a.n_slots = sim->n_slots;
  a.status = sim->d_status;
  a.ckpt_every = sim->ckpt_every;
  a.track = sim->cfg.task == 1;
  a.pay_plane = pay_plane(a.track);
  a.gen = sim->d_gen;
  return a;
}

// Persistent grid: blocks_per_sm resident blocks per SM (0: the kernel's
// occupancy limit), never more blocks than tiles.
// Resident blocks per SM of a group's launches: blocks_per_sm, capped by the
// kernel's occupancy limit (which is the default).
static int blocks_of(const mg_sim* sim, const Group& g) {
  int occ = 1;
  if (step_kernel_occupancy(g.nt, param_mode(sim), g.var, g.cls >= 0, sim->cfg.task == 1, &occ) != cudaSuccess ||
      occ < 1)
    occ = 1;
  return sim->blocks_per_sm > 0 ? std::min(sim->blocks_per_sm, occ) : occ;
}

static int grid_of(mg_sim* sim, const Group& g) {
  return std::max(1, std::min(g.n_tiles, blocks_of(sim, g) * sim->num_sms));
}

static bool misaligned(const void* p) { return p && ((uintptr_t)p & 15u) != 0; }

// Launch the step kernel once per thruster-count group.
// The first group is an ordinary launch (it waits for everything before it in
// the stream); later groups touch disjoint envs and are programmatic
// dependents, so they fill the SMs that the previous group's tail leaves idle.
#ifndef MG_USE_PDL
#define MG_USE_PDL 1
#endif
// Up to this many waves of tiles per step, the groups of a step (one kernel
// per thruster count and variant) share one wave of resident blocks: group g
// gets a grid proportional to its estimated work (tiles x FLOPs per
// env-step; one block per tile when all tiles fit), every launch is a
// programmatic dependent of the one before, so the groups run side by side
// and finish together; the first launch waits for the previous kernel of the
// stream (the previous step, same envs) before it reads anything or lets the
// step's other launches start. Larger steps launch the groups one after the
// other with full persistent grids (each group alone on the SMs runs faster
// than three interleaved), later groups as programmatic dependents that fill
// the previous group's tail.
#ifndef MG_CORESIDENT_WAVES
#define MG_CORESIDENT_WAVES 6
#endif
static bool coresident_grids(mg_sim* sim, std::vector<int>& grid) {
  const int n = (int)sim->groups.size();
  grid.assign(n, 1);
  int64_t resident = INT64_MAX, tiles = 0;
  std::vector<double> w(n);
  double wsum = 0.0;
  for (int i = 0; i < n; ++i) {
    const Group& g = sim->groups[i];
    resident = std::min<int64_t>(resident, (int64_t)blocks_of(sim, g) * sim->num_sms);
    double sub = 0.0, obs = 0.0;
    mg_count_flops(g.nt, sim->cfg.per_env_params, &sub, &obs, nullptr);
    w[i] = (double)g.n_tiles * ((g.var == 2 ? 4.0 : 1.0) * sim->cfg.K * sub + obs);
    wsum += w[i];
    tiles += g.n_tiles;
  }
  if (!MG_USE_PDL || resident < n || tiles > MG_CORESIDENT_WAVES * resident) return false;
  if (tiles <= resident) {
    for (int i = 0; i < n; ++i) grid[i] = sim->groups[i].n_tiles;
    return true;
  }
  int64_t used = 0;
  for (int i = 0; i < n; ++i) {
    grid[i] = std::max(1, std::min(sim->groups[i].n_tiles, (int)(resident * w[i] / wsum)));
    used += grid[i];
  }
  // Hand out what rounding left (or take back what the minimum of one added)
  // by the estimated time of each group: tile rounds x work per tile.
  auto cost = [&](int i, int blocks) {
    const Group& g = sim->groups[i];
    return (double)((g.n_tiles + blocks - 1) / blocks) * (w[i] / g.n_tiles);
  };
  while (used > resident) {
    int best = -1;
    for (int i = 0; i < n; ++i)
      if (grid[i] > 1 && (best < 0 || cost(i, grid[i] - 1) < cost(best, grid[best] - 1))) best = i;
    if (best < 0) break;
    grid[best]--; used--;
  }
  while (used < resident) {
    int best = -1;
    for (int i = 0; i < n; ++i)
      if (grid[i] < sim->groups[i].n_tiles && (best < 0 || cost(i, grid[i]) > cost(best, grid[best]))) best = i;
    if (best < 0) break;
    grid[best]++; used++;
  }
  return true;
}

// Shared-memory carveout of a launch: the largest when the step's groups share
// SMs (side-by-side launches with more blocks than SMs: blocks of different
// launches must fit one SM configuration) and for class-constant propeller
// steps without tracking (measured faster: their class-group launches overlap
// at the tails); the driver's default otherwise (with the class tables as
// kernel parameters the largest measured no faster for per-env and tracking
// steps, and slower for generic-actuator steps: 180 -> 204 us at 1M envs).
static bool carveout_max(const mg_sim* sim, const Group& g, bool shared_sm) {
  return shared_sm || (param_mode(sim) == 0 && g.var == 0 && sim->cfg.task != 1);
}

// The launch plan of the current segment layout and blocks_per_sm setting
// (occupancy queries and FLOP counts stay off the per-step path).
// Launches run one after the other (the larger steps) split the class groups
// into one launch per class, which takes its class tables as the kernel
// parameter (class-constant hover, 1M envs, K=4: 77.0 -> 69.8 us; 512k: 42.9
// -> 39.1 us). Side-by-side launches keep one launch per group with the
// tables in shared memory: their grids are split by estimated work, which a
// faster one-class kernel unbalances (262k envs: 23.1 -> 23.6 us), and five
// launches instead of three cost 4 us at 65k envs.
static const mg_sim::Plan& step_plan(mg_sim* sim, bool ms) {
  mg_sim::Plan& p = ms ? sim->plan_ms : sim->plan;
  if (p.valid && p.bps == sim->blocks_per_sm) return p;
  p.cores = coresident_grids(sim, p.grid);
  int64_t blocks = 0, tiles = 0;
  for (int b : p.grid) blocks += b;
  for (const Group& g : sim->groups) tiles += g.n_tiles;
  // Multi-step launches whose tiles all fit one wave (one tile per block) are
  // latency bound: every step is a chain of dependent arithmetic per warp, and
  // class tables read as constant-bank operands instead of shared-memory loads
  // shorten it. They too take one launch per class.
  const bool one_wave = p.cores && blocks == tiles;
  const bool split = MG_CLASS_PARAMS && (!p.cores || (ms && one_wave));
  const bool shared_sm = p.cores && blocks > sim->num_sms;
  p.groups.clear();
  for (const Group& g : sim->groups) {
    if (!split) { p.groups.push_back(g); continue; }
    for (int s = g.seg_lo; s < g.seg_hi; ++s) {   // a segment holds envs of one class
      Group h = g;
      h.seg_lo = s;
      h.seg_hi = s + 1;
      h.tile_lo = sim->segs[s].tile_begin;
      h.n_tiles = (s + 1 < g.seg_hi ? sim->segs[s + 1].tile_begin : g.tile_lo + g.n_tiles) - h.tile_lo;
      h.cls = sim->segs[s].cls;
      if (h.n_tiles > 0) p.groups.push_back(h);
    }
  }
  // Launches one after the other: the heaviest classes first, so that the
  // launch whose tail ends the step (the next step's first launch waits for
  // it) has the shortest tiles. Measured at 1M envs, K=4: hover 58.85 -> 58.5
  // us, mixed propeller / fin / tilt classes 165 -> 150 us, tracking 72.2 ->
  // 70.4 us; RK4 and payload steps ran slower (457 -> 483 us, 126.7 -> 127.7
  // us) and keep the class order.
  bool heavy_first = !p.cores && split && param_mode(sim) != 2;
  for (const Group& g : p.groups) heavy_first = heavy_first && g.var != 2;
  if (heavy_first)
    std::stable_sort(p.groups.begin(), p.groups.end(), [](const Group& x, const Group& y) { return x.nt > y.nt; });
  const size_t n = p.groups.size();
  if (!p.cores || split) p.grid.assign(n, 1);
  p.carve_max.assign(n, 0);
  p.full_grid.assign(n, 1);
  p.kc.assign(n, ClassK());
  for (size_t i = 0; i < n; ++i) {
    const Group& g = p.groups[i];
    if (g.cls >= 0) p.kc[i] = class_k(sim, g);
    p.full_grid[i] = grid_of(sim, g);
    if (!p.cores) p.grid[i] = p.full_grid[i];
    else if (split) p.grid[i] = g.n_tiles;   // one wave: a block per tile
    p.carve_max[i] = carveout_max(sim, g, shared_sm) ? 1 : 0;
  }
  // Measured: a programmatic first launch helps side-by-side steps and
  // propeller steps run one launch after the other (1M envs K=4 70.0 -> 67.6
  // us, K=1 52.4 -> 50.5 us, per-env DR 106.0 -> 104.3 us) but slows a step
  // that mixes propeller and generic-actuator launches (184 -> 196 us).
  p.first_pdl = true;
  if (!p.cores)
    for (const Group& g : p.groups)
      if (g.var != 0) p.first_pdl = false;
  for (int v = 0; v < 2; ++v) {
    p.jit[v].assign(n, nullptr);
    p.jit_tried[v].assign(n, 0);
    p.jit_grid[v].assign(n, 1);
  }
  p.bps = sim->blocks_per_sm;
  p.valid = true;
  return p;
}

// Whether launch i of a plan may run a class-specialised kernel: one class
// with class-constant or per-env parameters (no payload), propellers with
// the Euler substep, the hover task.
static bool jit_eligible(const mg_sim* sim, const Group& g) {
  return sim->specialise && g.cls >= 0 && g.var == 0 && param_mode(sim) <= 1 && sim->cfg.task == 0;
}

// The class-specialised kernel of launch i (single- or multi-step
// instantiation), compiled on first use, and its persistent grid; null if
// there is none (not eligible, NVRTC missing, compile failed).
static const void* plan_jit(mg_sim* sim, mg_sim::Plan& p, size_t i, bool ms) {
  const Group& g = p.groups[i];
  const int v = ms ? 1 : 0;
  if (!jit_eligible(sim, g)) return nullptr;
  if (!p.jit_tried[v][i]) {
    p.jit_tried[v][i] = 1;
    std::string err;
    // Per-env kernels keep the 4-block bound (their parameter columns fill
    // shared memory at 4 blocks per SM).
    const int pm = param_mode(sim);
    const int mb = pm == 0 ? jit_step_min_blocks(sim->cfg.K, g.n_tiles, sim->num_sms) : 4;
    const void* k = jit_step_kernel(p.kc[i], g.nt, ms, pm, mb, &err);
    if (!k) sim->jit_err = err;
    int occ = 0;
    if (k && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 128, step_kernel_smem_jit(g.nt, pm)) !=
                 cudaSuccess) {
      cudaGetLastError();
      occ = 0;
    }
    if (k && occ >= 1) {
      const int bps = sim->blocks_per_sm > 0 ? std::min(sim->blocks_per_sm, occ) : occ;
      p.jit[v][i] = k;
      // Same launch shape as the kernel it replaces: a persistent grid, or
      // (one-wave plans) a block per tile.
      p.jit_grid[v][i] = p.grid[i] == p.full_grid[i] ? std::max(1, std::min(g.n_tiles, bps * sim->num_sms))
                                                      : p.grid[i];
    } else if (k) {
      sim->jit_err = "specialised kernel does not fit an SM";
    }
  }
  return p.jit[v][i];
}

// Launches of at least this many steps use the multi-step plan. Measured:
// the per-class split costs about 5 us per call (single steps at 16k and 65k
// envs, K=4: 10.8 -> 15.6 us) and saves about 0.3 us per step at 16k envs
// (100-step graph 193 -> 163 us), so it pays from about 17 steps on.
#ifndef MG_SPLIT_MIN_STEPS
#define MG_SPLIT_MIN_STEPS 16
#endif

// Whether a launch of the plan may run on the lane-pair kernel: one class
// (class tables as the kernel parameter), propellers with the Euler substep,
// class-constant or per-env parameters, the hover task, actions from memory.
static bool pair_eligible(const mg_sim* sim, const Group& g, const StepArgs& a) {
  return g.cls >= 0 && g.var == 0 && param_mode(sim) <= 1 && sim->cfg.task == 0 && !a.ret && a.act_mode == 0 &&
         a.n_steps >= 1;
}

static int launch_groups(mg_sim* sim, StepArgs a, cudaStream_t st) {
  const mg_sim::Plan& p = step_plan(sim, a.n_steps >= MG_SPLIT_MIN_STEPS);
  bool first = true;
  for (size_t i = 0; i < p.groups.size(); ++i) {
    const Group& g = p.groups[i];
    a.seg_lo = g.seg_lo;
    a.seg_hi = g.seg_hi;
    a.tile_lo = g.tile_lo;
    a.n_tiles = g.n_tiles;
    // Later launches are programmatic dependents of the one before. With
    // p.first_pdl the first is too: it waits for the kernel before it (the
    // previous step, or unrelated work) before it reads anything or lets the
    // step's other launches start, so its blocks only become resident and set
    // up early.
    a.wait_first = first && p.first_pdl;
    const bool ms = g.var == 0 && a.act_mode == 0 && a.n_steps > 1;   // the kernels' multi-step instantiation
    const void* jk = nullptr;
    if (sim->lanes == 2 && pair_eligible(sim, g, a))
      CK(launch_pair(a, p.kc[i], g.nt, !first || p.first_pdl, st));
    else if ((jk = plan_jit(sim, const_cast<mg_sim::Plan&>(p), i, ms)) != nullptr)
      CK(launch_step_jit(jk, a, p.kc[i], g.nt, param_mode(sim), p.jit_grid[ms ? 1 : 0][i], !first || p.first_pdl, p.carve_max[i] != 0,
                         st));
    else
      CK(launch_step(a, g.cls >= 0 ? &p.kc[i] : nullptr, g.cls >= 0 ? &sim->h_gen[g.cls] : nullptr, g.nt, g.var,
                     p.grid[i], !first || p.first_pdl, p.carve_max[i] != 0, st));
    first = false;
  }
  return MG_OK;
}

int mg_step(mg_sim* sim, const float* actions_dev, int32_t n_steps, float* obs_dev, float* reward_dev,
            mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (!actions_dev || n_steps < 1) return fail(sim, MG_ERR_INVALID_ARG, "step: need actions and n_steps >= 1");
  if (misaligned(actions_dev) || misaligned(obs_dev))
    return fail(sim, MG_ERR_INVALID_ARG, "step: actions and obs buffers must be 16-byte aligned");
  StepArgs a = step_args(sim);
  a.actions = actions_dev;
  a.n_steps = n_steps;
  a.obs = obs_dev;
  a.reward = reward_dev;
  a.obs_every = 0;
  drop_recording(sim);
  return launch_groups(sim, a, (cudaStream_t)stream);
}

int mg_rollout(mg_sim* sim, const float* actions_dev, int32_t n_steps, float* obs_dev, float* reward_dev,
               int32_t record, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (!actions_dev || n_steps < 1) return fail(sim, MG_ERR_INVALID_ARG, "rollout: need actions and n_steps >= 1");
  if (misaligned(actions_dev) || misaligned(obs_dev))
    return fail(sim, MG_ERR_INVALID_ARG, "rollout: actions and obs buffers must be 16-byte aligned");
  if (record && (!sim->d_ckpt || n_steps > sim->cfg.record_steps))
    return fail(sim, MG_ERR_INVALID_ARG, "rollout: record needs record_steps >= n_steps (have %d)", sim->cfg.record_steps);
  StepArgs a = step_args(sim);
  a.actions = actions_dev;
  a.n_steps = n_steps;
  a.obs = obs_dev;
  a.reward = reward_dev;
  a.obs_every = 1;
  a.ckpt = record ? sim->d_ckpt : nullptr;
  drop_recording(sim);
  int rc = launch_groups(sim, a, (cudaStream_t)stream);
  if (record && rc == MG_OK) {
    sim->rec_T = n_steps;
    sim->rec_id = g_next_rec_id.fetch_add(1);
  }
  return rc;
}

int mg_observe(mg_sim* sim, float* obs_dev, float* reward_dev, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (!obs_dev && !reward_dev) return fail(sim, MG_ERR_INVALID_ARG, "observe: obs and reward are both null");
  if (misaligned(obs_dev)) return fail(sim, MG_ERR_INVALID_ARG, "observe: obs buffer must be 16-byte aligned");
  StepArgs a = step_args(sim);
  a.n_steps = 0;
  a.obs = obs_dev;
  a.reward = reward_dev;
  return launch_groups(sim, a, (cudaStream_t)stream);
}

int mg_recording(const mg_sim* sim, int32_t* steps, uint64_t* id) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (steps) *steps = sim->rec_T;
  if (id) *id = sim->rec_id;
  return MG_OK;
}

int mg_env_order(const int32_t* env_class, int32_t n_envs, int32_t n_classes, int32_t* class_counts,
                 int32_t* lib_env) {
  if (!env_class || !class_counts || !lib_env || n_envs < 0 || n_classes < 1 || n_classes > MG_MAX_CLASSES) {
    g_create_err = "env_order: null buffer or bad sizes";
    return MG_ERR_INVALID_ARG;
  }
  std::vector<int64_t> start(n_classes + 1, 0);
  for (int32_t i = 0; i < n_envs; ++i) {
    const int32_t c = env_class[i];
    if (c < 0 || c >= n_classes) {
      g_create_err = "env_order: env " + std::to_string(i) + " has class " + std::to_string(c) + " outside [0, n_classes)";
      return MG_ERR_INVALID_ARG;
    }
    ++start[c + 1];
  }
  for (int c = 0; c < n_classes; ++c) {
    class_counts[c] = (int32_t)start[c + 1];
    start[c + 1] += start[c];
  }
  // Stable: envs of one class keep their relative order.
  for (int32_t i = 0; i < n_envs; ++i) lib_env[i] = (int32_t)start[env_class[i]]++;
  return MG_OK;
}

// mg_step_host pipeline: the step is cut into chunks of at most this many
// tiles (one thruster-count group, contiguous tiles); chunk c's actions are
// copied in on one stream while chunk c-1 steps on the caller's stream and
// chunk c-2's observations are copied out on a third (host-to-device and
// device-to-host copies overlap on the link).
#ifndef MG_HOST_CHUNK_TILES
#define MG_HOST_CHUNK_TILES 2048
#endif
// The first chunk is smaller: device-to-host copies (the larger direction:
// 52 B of observation and 4 B of reward per env against 4 NT B of actions)
// start once it has stepped, instead of after a full chunk's actions crossed.
// Measured at 1M envs, K=4 (ms per host-buffer step): first chunk 1639 tiles
// (the whole first group) 1.273, 1024 1.277, 768 1.267, 512 1.236, 384 1.236,
// 128 1.266, 32 1.277; chunks of 256-1024 tiles throughout were slower still
// (1.29-1.48).
#ifndef MG_HOST_FIRST_CHUNK_TILES
#define MG_HOST_FIRST_CHUNK_TILES 512
#endif

int mg_step_host(mg_sim* sim, const float* actions_host, int32_t n_steps, float* obs_host, float* reward_host,
                 mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (!actions_host || n_steps < 1) return fail(sim, MG_ERR_INVALID_ARG, "step_host: need actions and n_steps >= 1");
  const size_t need = (size_t)n_steps * sim->act_floats + (size_t)sim->n_slots * 14;
  if (need > sim->stage_floats) {
    if (sim->d_stage) { cudaFree(sim->d_stage); sim->bytes -= sim->stage_floats * sizeof(float); sim->d_stage = nullptr; }
    sim->stage_floats = 0;
    int rc = dev_alloc(sim, (void**)&sim->d_stage, need * sizeof(float));
    if (rc != MG_OK) return rc;
    sim->stage_floats = need;
  }
  float* d_act = sim->d_stage;
  float* d_obs = d_act + (size_t)n_steps * sim->act_floats;
  float* d_rew = d_obs + (size_t)sim->n_slots * 13;
  cudaStream_t st = (cudaStream_t)stream;
  if (!sim->s_in) CK(cudaStreamCreateWithFlags(&sim->s_in, cudaStreamNonBlocking));
  if (!sim->s_out) CK(cudaStreamCreateWithFlags(&sim->s_out, cudaStreamNonBlocking));
  // Chunks: (launch of the step plan, first tile, tiles).
  const mg_sim::Plan& plan = step_plan(sim);
  struct Chunk { int g, t0, nt; };
  std::vector<Chunk> chunks;
  for (int gi = 0; gi < (int)plan.groups.size(); ++gi)
    for (int t = 0; t < plan.groups[gi].n_tiles;) {
      const int n = std::min(chunks.empty() ? MG_HOST_FIRST_CHUNK_TILES : MG_HOST_CHUNK_TILES,
                             plan.groups[gi].n_tiles - t);
      chunks.push_back({gi, t, n});
      t += n;
    }
  const size_t n_ev = 2 * chunks.size() + 1;
  while (sim->host_ev.size() < n_ev) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    sim->host_ev.push_back(e);
  }
  cudaEvent_t ev_entry = sim->host_ev[0];
  CK(cudaEventRecord(ev_entry, st));   // earlier work on the caller's stream
  CK(cudaStreamWaitEvent(sim->s_in, ev_entry, 0));
  CK(cudaStreamWaitEvent(sim->s_out, ev_entry, 0));
  const size_t pitch = sizeof(float) * (size_t)sim->act_floats;
  StepArgs a = step_args(sim);
  a.actions = d_act;
  a.n_steps = n_steps;
  a.obs = obs_host ? d_obs : nullptr;
  a.reward = reward_host ? d_rew : nullptr;
  a.act_stride = sim->act_floats;
  for (size_t c = 0; c < chunks.size(); ++c) {
    const Chunk& ch = chunks[c];
    const Group& g = plan.groups[ch.g];
    const int tile_lo = g.tile_lo + ch.t0, tile_hi = tile_lo + ch.nt;
    cudaEvent_t ev_in = sim->host_ev[1 + 2 * c], ev_done = sim->host_ev[2 + 2 * c];
    // Env ranges of the chunk, per segment of the group.
    struct Range { int64_t act0, nact, slot0, nslot; };
    std::vector<Range> ranges;
    for (int si = g.seg_lo; si < g.seg_hi; ++si) {
      const SegDesc& sd = sim->segs[si];
      const int seg_tiles = (sd.n4 + sim->threads - 1) / sim->threads;
      const int lo = std::max(tile_lo, sd.tile_begin), hi = std::min(tile_hi, sd.tile_begin + seg_tiles);
      if (lo >= hi) continue;
      const int64_t s0 = (int64_t)(lo - sd.tile_begin) * sim->threads;
      const int64_t s1 = std::min<int64_t>((int64_t)(hi - sd.tile_begin) * sim->threads, sd.n4);
      ranges.push_back({sd.act_off + s0 * sd.n_thr, (s1 - s0) * sd.n_thr, sd.slot_off + s0, s1 - s0});
    }
    for (const Range& r : ranges)
      CK(cudaMemcpy2DAsync(d_act + r.act0, pitch, actions_host + r.act0, pitch, sizeof(float) * r.nact, n_steps,
                           cudaMemcpyHostToDevice, sim->s_in));
    CK(cudaEventRecord(ev_in, sim->s_in));
    CK(cudaStreamWaitEvent(st, ev_in, 0));
    a.seg_lo = g.seg_lo;
    a.seg_hi = g.seg_hi;
    a.tile_lo = tile_lo;
    a.n_tiles = ch.nt;
    a.wait_first = 0;
    const bool ms = g.var == 0 && n_steps > 1;
    const void* jk = plan_jit(sim, const_cast<mg_sim::Plan&>(plan), ch.g, ms);
    if (jk)
      CK(launch_step_jit(jk, a, plan.kc[ch.g], g.nt, param_mode(sim), std::max(1, std::min(ch.nt, plan.jit_grid[ms ? 1 : 0][ch.g])), false,
                         carveout_max(sim, g, false), st));
    else
      CK(launch_step(a, g.cls >= 0 ? &plan.kc[ch.g] : nullptr, g.cls >= 0 ? &sim->h_gen[g.cls] : nullptr, g.nt,
                     g.var, std::max(1, std::min(ch.nt, plan.full_grid[ch.g])), false, carveout_max(sim, g, false),
                     st));
    CK(cudaEventRecord(ev_done, st));
    CK(cudaStreamWaitEvent(sim->s_out, ev_done, 0));
    for (const Range& r : ranges) {
      if (obs_host)
        CK(cudaMemcpyAsync(obs_host + r.slot0 * 13, d_obs + r.slot0 * 13, sizeof(float) * r.nslot * 13,
                           cudaMemcpyDeviceToHost, sim->s_out));
      if (reward_host)
        CK(cudaMemcpyAsync(reward_host + r.slot0, d_rew + r.slot0, sizeof(float) * r.nslot,
                           cudaMemcpyDeviceToHost, sim->s_out));
    }
  }
  drop_recording(sim);
  CK(cudaStreamSynchronize(sim->s_out));
  CK(cudaStreamSynchronize(st));
  return MG_OK;
}

// Steps of one reverse unit of the adjoint: a checkpoint segment of more
// than MG_ADJ_UNIT_MAX steps splits into units of at most that many, each
// recomputed from the segment's checkpoint (the recompute warps pass over the
// earlier units of the segment again; the records of a unit are what the
// reverse warps read while the next unit is recomputed). At 8192 envs with
// 20-step checkpoints, whole segments measured 0.497 ms per backward, units
// of 10 and 7 steps 0.51 and 0.56 ms.
#ifndef MG_ADJ_UNIT_MAX
#define MG_ADJ_UNIT_MAX 20
#endif
static int adjoint_unit_steps(int ckpt_every) {
  const int m = (ckpt_every + MG_ADJ_UNIT_MAX - 1) / MG_ADJ_UNIT_MAX;
  return (ckpt_every + m - 1) / m;
}

// The adjoint launches of a backward pass: one per class segment, with that
// class's tables as the kernel parameter, each a programmatic dependent of
// the previous one so that they run side by side.
static int launch_backward(mg_sim* sim, AdjArgs a, cudaStream_t st) {
  a.tile_envs = sim->threads;
  a.unit_steps = adjoint_unit_steps(sim->ckpt_every);
  a.pay_plane = sim->cfg.payload ? pay_plane(sim->cfg.task == 1) : 0;
  bool first = true;
  for (const Group& grp : sim->groups) {
    for (int s = grp.seg_lo; s < grp.seg_hi; ++s) {
      const SegDesc& sd = sim->segs[s];
      Group g = grp;
      g.seg_lo = s;
      g.seg_hi = s + 1;
      g.tile_lo = sd.tile_begin;
      g.n_tiles = (sd.n4 + sim->threads - 1) / sim->threads;
      g.cls = sd.cls;
      const ClassK kc = class_k(sim, g, true);
      a.seg_lo = g.seg_lo; a.seg_hi = g.seg_hi; a.tile_lo = g.tile_lo; a.n_tiles = g.n_tiles;
      // The class-specialised kernel (its actuator tables as literals) when
      // it can be had; the library's otherwise.
      const void* jk = nullptr;
      const bool gen = g.var != 0;
      if (sim->specialise && !sim->cfg.payload && !gen) {
        std::string err;
        jk = jit_adjoint_kernel(kc, g.nt, &err);
        if (!jk) sim->jit_err = err;
      }
      CK(launch_adjoint(a, kc, gen ? &sim->h_gen[g.cls] : nullptr, g.nt, g.var, !first, st, jk));
      first = false;
    }
  }
  return MG_OK;
}

int mg_step_backward(mg_sim* sim, const float* actions_dev, const float* g_obs, const float* g_rew,
                     const float* g_state_T, float* g_actions, float* g_added_mass, float* g_damping,
                     float* g_state0, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (sim->rec_T <= 0)
    return fail(sim, MG_ERR_STATE,
                "backward: no recorded rollout (call mg_rollout with record=1; a later step, reset, graph replay "
                "or state / parameter / task / payload change discards the recording)");
  if (!actions_dev) return fail(sim, MG_ERR_INVALID_ARG, "backward: actions required");
  AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.segs = sim->d_segs;
  a.classes = sim->d_cls;
  a.planes = sim->d_planes;
  a.n_slots = sim->n_slots;
  a.actions = actions_dev;
  a.act_stride = sim->act_floats;
  a.T = sim->rec_T;
  a.ckpt_every = sim->ckpt_every;
  a.ckpt = sim->d_ckpt;
  a.scratch = sim->d_scratch;
  a.g_obs = g_obs;
  a.g_rew = g_rew;
  a.g_state_T = g_state_T;
  a.g_actions = g_actions;
  a.g_A = g_added_mass;
  a.g_D = g_damping;
  a.g_state0 = g_state0;
  cudaStream_t st = (cudaStream_t)stream;
  if (g_actions) CK(cudaMemsetAsync(g_actions, 0, sizeof(float) * sim->rec_T * sim->act_floats, st));
  return launch_backward(sim, a, st);
}

int mg_set_hydro(mg_sim* sim, const float* A_dev, const float* dl_dev, const float* dq_dev, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (!sim->cfg.per_env_params) return fail(sim, MG_ERR_INVALID_ARG, "set_hydro needs per_env_params");
  if (sim->cfg.payload) return fail(sim, MG_ERR_INVALID_ARG, "set_hydro: not available for payload runs (use mg_set_params)");
  CK(launch_set_hydro(sim->d_planes, sim->n_slots, A_dev, dl_dev, dq_dev, (cudaStream_t)stream));
  drop_recording(sim);
  return MG_OK;
}

int mg_rollout_fp64(mg_sim* sim, const float* actions_dev, int32_t n_steps, const double* dA, const double* ddl,
                    const double* ddq, double eps, double* reward_dev, double* state_dev, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (!sim->cfg.per_env_params) return fail(sim, MG_ERR_INVALID_ARG, "rollout_fp64 needs per_env_params");
  if (!actions_dev || !reward_dev || n_steps < 1) return fail(sim, MG_ERR_INVALID_ARG, "rollout_fp64: bad arguments");
  Fp64Args a;
  std::memset(&a, 0, sizeof(a));
  a.segs = sim->d_segs;
  a.classes = sim->d_cls64;
  a.state = sim->d_state;
  a.planes = sim->d_planes;
  a.n_slots = sim->n_slots;
  a.actions = actions_dev;
  a.act_stride = sim->act_floats;
  a.T = n_steps;
  a.dA = dA; a.ddl = ddl; a.ddq = ddq;
  a.eps = eps;
  a.dt = sim->cfg.dt;
  a.h = sim->h;
  a.reward = reward_dev;
  a.state_out = state_dev;
  a.gen = sim->d_gen64;
  a.pay_plane = sim->cfg.payload ? pay_plane(sim->cfg.task == 1) : 0;
  for (const Group& g : sim->groups) {
    a.seg_lo = g.seg_lo; a.seg_hi = g.seg_hi; a.tile_lo = g.tile_lo; a.n_tiles = g.n_tiles;
    CK(launch_fp64(a, g.nt, g.var, sim->threads, (cudaStream_t)stream));
  }
  return MG_OK;
}

// Canonical field j of env (class layout L, local index i) inside the SoA planes.
static int64_t field_off(const ClassLay& L, int64_t i, int j) {
  const int SS = 13 + L.n_thr, NF4 = SS / 4;
  if (j < NF4 * 4) return L.st_off + ((int64_t)(j / 4) * L.n4 + i) * 4 + (j % 4);
  return L.st_off + (int64_t)NF4 * 4 * L.n4 + (int64_t)(j - NF4 * 4) * L.n4 + i;
}

int mg_get_state(const mg_sim* csim, float* host, size_t bytes) {
  mg_sim* sim = const_cast<mg_sim*>(csim);
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (bytes < sizeof(float) * 21 * (size_t)sim->n_envs) return fail(sim, MG_ERR_INVALID_ARG, "get_state: buffer too small");
  std::vector<float> buf(sim->state_floats);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(buf.data(), sim->d_state, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      float* o = host + (L.env_off + i) * 21;
      for (int j = 0; j < 21; ++j) o[j] = (j < 13 + L.n_thr) ? buf[field_off(L, i, j)] : 0.0f;
    }
  }
  return MG_OK;
}

int mg_set_state(mg_sim* sim, const float* host, size_t bytes) {
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (bytes < sizeof(float) * 21 * (size_t)sim->n_envs) return fail(sim, MG_ERR_INVALID_ARG, "set_state: buffer too small");
  std::vector<float> buf(sim->state_floats, 0.0f);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(buf.data(), sim->d_state, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      const float* s = host + (L.env_off + i) * 21;
      for (int j = 0; j < 13 + L.n_thr; ++j) buf[field_off(L, i, j)] = s[j];
    }
  }
  CK(cudaMemcpy(sim->d_state, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice));
  drop_recording(sim);
  return MG_OK;
}

int mg_get_params(const mg_sim* csim, double* host, size_t bytes) {
  mg_sim* sim = const_cast<mg_sim*>(csim);
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (bytes < sizeof(double) * MG_ENV_PARAM_DIM * (size_t)sim->n_envs)
    return fail(sim, MG_ERR_INVALID_ARG, "get_params: buffer too small");
  std::vector<float4> pl((size_t)sim->n_planes * sim->n_slots);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(pl.data(), sim->d_planes, sizeof(float4) * pl.size(), cudaMemcpyDeviceToHost));
  std::vector<ClassF> cf(sim->n_classes);
  CK(cudaMemcpy(cf.data(), sim->d_cls, sizeof(ClassF) * cf.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      const int64_t slot = L.slot_off + i;
      float v[40];
      if (sim->cfg.per_env_params) {
        for (int k = 0; k < PAR_PLANES + 1; ++k) {
          const float4 x = pl[(size_t)k * sim->n_slots + slot];
          v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
        }
      } else {
        for (int k = 0; k < 36; ++k) v[k] = cf[c].phys[k];
        const float4 x = pl[slot];
        v[36] = x.x; v[37] = x.y; v[38] = x.z; v[39] = x.w;
      }
      double* o = host + (L.env_off + i) * MG_ENV_PARAM_DIM;
      int q = 0;
      o[q++] = v[PAR_M];
      for (int j = 0; j < 3; ++j) o[q++] = v[PAR_IG + j];
      for (int j = 0; j < 3; ++j) o[q++] = v[PAR_RB + j];
      o[q++] = v[PAR_W];
      o[q++] = v[PAR_B];
      for (int j = 0; j < 6; ++j) o[q++] = v[PAR_A + j];
      for (int j = 0; j < 6; ++j) o[q++] = v[PAR_DL + j];
      for (int j = 0; j < 6; ++j) o[q++] = v[PAR_DQ + j];
      for (int j = 0; j < 3; ++j) o[q++] = v[PAR_VC + j];
      for (int j = 0; j < 3; ++j) o[q++] = v[36 + j];
      o[q++] = 0.0;
    }
  }
  return MG_OK;
}

// Payload planes of one slot from the vehicle parameters and the payload
// (m_p, r_p), computed in FP64 on the host.
static int write_payload(mg_sim* sim, std::vector<float4>& pl, int64_t slot, double m, const double Ig[3],
                         const double Ma[6], double W, double mp, const double rp[3]) {
  float v[PAY_DIM];
  if (!payload_block(m, Ig, Ma, W, mp, rp, v)) return MG_ERR_INVALID_ARG;
  const int pp = pay_plane(sim->cfg.task == 1);
  for (int k = 0; k < PAY_PLANES; ++k)
    pl[(size_t)(pp + k) * sim->n_slots + slot] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  return MG_OK;
}

int mg_set_params(mg_sim* sim, const double* host, size_t bytes) {
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (bytes < sizeof(double) * MG_ENV_PARAM_DIM * (size_t)sim->n_envs)
    return fail(sim, MG_ERR_INVALID_ARG, "set_params: buffer too small");
  if (!sim->cfg.per_env_params) return fail(sim, MG_ERR_INVALID_ARG, "set_params needs per_env_params");
  std::vector<float4> pl((size_t)sim->n_planes * sim->n_slots);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(pl.data(), sim->d_planes, sizeof(float4) * pl.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      const double* s = host + (L.env_off + i) * MG_ENV_PARAM_DIM;
      const double m = s[0], Ig[3] = {s[1], s[2], s[3]};
      for (int j = 0; j < 31; ++j)
        if (!std::isfinite(s[j])) return fail(sim, MG_ERR_INVALID_ARG, "set_params: env %lld not finite", (long long)(L.env_off + i));
      if (m <= 0 || Ig[0] <= 0 || Ig[1] <= 0 || Ig[2] <= 0)
        return fail(sim, MG_ERR_INVALID_ARG, "set_params: env %lld mass/inertia must be > 0", (long long)(L.env_off + i));
      float v[40];
      const double Mrb[6] = {m, m, m, Ig[0], Ig[1], Ig[2]};
      for (int j = 0; j < 6; ++j) {
        const double A = s[9 + j];
        v[PAR_MINV + j] = (float)(1.0 / (Mrb[j] + A));
        v[PAR_A + j] = (float)A;
        v[PAR_DL + j] = (float)s[15 + j];
        v[PAR_DQ + j] = (float)s[21 + j];
      }
      v[PAR_M] = (float)m;
      for (int j = 0; j < 3; ++j) { v[PAR_IG + j] = (float)Ig[j]; v[PAR_RB + j] = (float)s[4 + j]; v[PAR_VC + j] = (float)s[27 + j]; }
      v[PAR_W] = (float)s[7];
      v[PAR_B] = (float)s[8];
      const int64_t slot = L.slot_off + i;
      // The target plane's w lane is the env's step counter: keep it.
      v[36] = (float)s[30]; v[37] = (float)s[31]; v[38] = (float)s[32];
      v[39] = pl[(size_t)TGT_PLANE * sim->n_slots + slot].w;
      for (int k = 0; k < PAR_PLANES + 1; ++k)
        pl[(size_t)k * sim->n_slots + slot] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
      if (sim->cfg.payload) {
        // The combined body follows the new vehicle parameters; the payload stays.
        const float4 q = pl[(size_t)(pay_plane(sim->cfg.task == 1) + PAY_MP / 4) * sim->n_slots + slot];
        const double Ma[6] = {s[9], s[10], s[11], s[12], s[13], s[14]};
        const double rp[3] = {q.y, q.z, q.w};
        if (write_payload(sim, pl, slot, m, Ig, Ma, s[7], q.x, rp) != MG_OK)
          return fail(sim, MG_ERR_INVALID_ARG, "set_params: env %lld inertia not positive definite", (long long)(L.env_off + i));
      }
    }
  }
  CK(cudaMemcpy(sim->d_planes, pl.data(), sizeof(float4) * pl.size(), cudaMemcpyHostToDevice));
  drop_recording(sim);
  return MG_OK;
}

int mg_get_payload(const mg_sim* csim, double* host, size_t bytes) {
  mg_sim* sim = const_cast<mg_sim*>(csim);
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (!sim->cfg.payload) return fail(sim, MG_ERR_INVALID_ARG, "get_payload: not a payload run");
  if (bytes < sizeof(double) * 4 * (size_t)sim->n_envs) return fail(sim, MG_ERR_INVALID_ARG, "get_payload: buffer too small");
  std::vector<float4> pl((size_t)sim->n_planes * sim->n_slots);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(pl.data(), sim->d_planes, sizeof(float4) * pl.size(), cudaMemcpyDeviceToHost));
  const int qp = pay_plane(sim->cfg.task == 1) + PAY_MP / 4;
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      const float4 q = pl[(size_t)qp * sim->n_slots + L.slot_off + i];
      double* o = host + (L.env_off + i) * 4;
      o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    }
  }
  return MG_OK;
}

int mg_set_payload(mg_sim* sim, const double* host, size_t bytes) {
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (!sim->cfg.payload) return fail(sim, MG_ERR_INVALID_ARG, "set_payload: not a payload run");
  if (bytes < sizeof(double) * 4 * (size_t)sim->n_envs) return fail(sim, MG_ERR_INVALID_ARG, "set_payload: buffer too small");
  std::vector<float4> pl((size_t)sim->n_planes * sim->n_slots);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(pl.data(), sim->d_planes, sizeof(float4) * pl.size(), cudaMemcpyDeviceToHost));
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      const int64_t env = L.env_off + i, slot = L.slot_off + i;
      const double* q = host + env * 4;
      for (int j = 0; j < 4; ++j)
        if (!std::isfinite(q[j])) return fail(sim, MG_ERR_INVALID_ARG, "set_payload: env %lld not finite", (long long)env);
      if (q[0] < 0.0) return fail(sim, MG_ERR_INVALID_ARG, "set_payload: env %lld payload mass < 0", (long long)env);
      float v[PAR_DIM];
      for (int k = 0; k < PAR_PLANES; ++k) {
        const float4 x = pl[(size_t)k * sim->n_slots + slot];
        v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
      }
      const double Ig[3] = {v[PAR_IG], v[PAR_IG + 1], v[PAR_IG + 2]};
      double Ma[6];
      for (int j = 0; j < 6; ++j) Ma[j] = v[PAR_A + j];
      const double rp[3] = {q[1], q[2], q[3]};
      if (write_payload(sim, pl, slot, v[PAR_M], Ig, Ma, v[PAR_W], q[0], rp) != MG_OK)
        return fail(sim, MG_ERR_INVALID_ARG, "set_payload: env %lld inertia not positive definite", (long long)env);
    }
  }
  CK(cudaMemcpy(sim->d_planes, pl.data(), sizeof(float4) * pl.size(), cudaMemcpyHostToDevice));
  drop_recording(sim);
  return MG_OK;
}

int mg_get_task(const mg_sim* csim, double* host, size_t bytes) {
  mg_sim* sim = const_cast<mg_sim*>(csim);
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (bytes < sizeof(double) * 16 * (size_t)sim->n_envs) return fail(sim, MG_ERR_INVALID_ARG, "get_task: buffer too small");
  std::vector<float4> pl((size_t)sim->n_planes * sim->n_slots);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(pl.data(), sim->d_planes, sizeof(float4) * pl.size(), cudaMemcpyDeviceToHost));
  const int tp = tgt_plane(sim->cfg.per_env_params);
  const bool track = sim->cfg.task == 1;
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      const int64_t slot = L.slot_off + i;
      double* o = host + (L.env_off + i) * 16;
      for (int j = 0; j < 16; ++j) o[j] = 0.0;
      const float4 g = pl[(size_t)tp * sim->n_slots + slot];
      o[0] = g.x; o[1] = g.y; o[2] = g.z; o[15] = g.w;
      if (track) {
        const float4 t0 = pl[(size_t)(tp + 1) * sim->n_slots + slot];
        const float4 t1 = pl[(size_t)(tp + 2) * sim->n_slots + slot];
        const float4 t2 = pl[(size_t)(tp + 3) * sim->n_slots + slot];
        const float r[12] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
        for (int j = 0; j < 12; ++j) o[3 + j] = r[j];
      }
    }
  }
  return MG_OK;
}

int mg_set_task(mg_sim* sim, const double* host, size_t bytes) {
  if (!sim || !host) return MG_ERR_INVALID_ARG;
  if (bytes < sizeof(double) * 16 * (size_t)sim->n_envs) return fail(sim, MG_ERR_INVALID_ARG, "set_task: buffer too small");
  const bool track = sim->cfg.task == 1;
  std::vector<float4> pl((size_t)sim->n_planes * sim->n_slots);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(pl.data(), sim->d_planes, sizeof(float4) * pl.size(), cudaMemcpyDeviceToHost));
  const int tp = tgt_plane(sim->cfg.per_env_params);
  for (int c = 0; c < sim->n_classes; ++c) {
    const ClassLay& L = sim->lay[c];
    for (int64_t i = 0; i < L.n_envs; ++i) {
      const double* s = host + (L.env_off + i) * 16;
      for (int j = 0; j < 16; ++j)
        if (!std::isfinite(s[j])) return fail(sim, MG_ERR_INVALID_ARG, "set_task: env %lld not finite", (long long)(L.env_off + i));
      if (!track)
        for (int j = 3; j < 15; ++j)
          if (s[j] != 0.0) return fail(sim, MG_ERR_INVALID_ARG, "set_task: a, w, phi, v must be 0 without tracking");
      if (s[15] < 0 || s[15] > 16777216.0 || s[15] != std::floor(s[15]))
        return fail(sim, MG_ERR_INVALID_ARG, "set_task: step counter must be an integer in [0, 2^24]");
      const int64_t slot = L.slot_off + i;
      pl[(size_t)tp * sim->n_slots + slot] = make_float4((float)s[0], (float)s[1], (float)s[2], (float)s[15]);
      if (track) {
        pl[(size_t)(tp + 1) * sim->n_slots + slot] = make_float4((float)s[3], (float)s[4], (float)s[5], (float)s[6]);
        pl[(size_t)(tp + 2) * sim->n_slots + slot] = make_float4((float)s[7], (float)s[8], (float)s[9], (float)s[10]);
        pl[(size_t)(tp + 3) * sim->n_slots + slot] = make_float4((float)s[11], (float)s[12], (float)s[13], (float)s[14]);
      }
    }
  }
  CK(cudaMemcpy(sim->d_planes, pl.data(), sizeof(float4) * pl.size(), cudaMemcpyHostToDevice));
  drop_recording(sim);
  return MG_OK;
}

// Failure-path test: one step launch in which no copies are issued, so every
// warp's first wait runs out after limit_ns and the warp leaves with bit 1 of
// the status word set; no state is touched.
int mg_test_wait_timeout(mg_sim* sim, uint64_t limit_ns, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (limit_ns == 0 || limit_ns > 2000000000ull) return fail(sim, MG_ERR_INVALID_ARG, "test_wait_timeout: limit in (0, 2 s]");
  const size_t need = (size_t)sim->act_floats;
  if (need > sim->stage_floats) {
    if (sim->d_stage) { cudaFree(sim->d_stage); sim->bytes -= sim->stage_floats * sizeof(float); sim->d_stage = nullptr; }
    sim->stage_floats = 0;
    int rc = dev_alloc(sim, (void**)&sim->d_stage, need * sizeof(float));
    if (rc != MG_OK) return rc;
    sim->stage_floats = need;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // The segment table of this one launch marks every segment "issue no
  // copies" with the given bound; the simulator's own table is put back after.
  std::vector<SegDesc> test = sim->segs;
  for (SegDesc& sd : test) { sd.flags |= 2; sd.wait_limit_ns = limit_ns; }
  CK(cudaMemcpyAsync(sim->d_segs, test.data(), sizeof(SegDesc) * test.size(), cudaMemcpyHostToDevice, st));
  StepArgs a = step_args(sim);
  a.actions = sim->d_stage;
  a.n_steps = 1;
  int rc = launch_groups(sim, a, st);
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpy(sim->d_segs, sim->segs.data(), sizeof(SegDesc) * sim->segs.size(), cudaMemcpyHostToDevice));
  drop_recording(sim);
  return rc;
}

int mg_status(mg_sim* sim, mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  uint32_t st = 0;
  CK(cudaMemcpy(&st, sim->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st) CK(cudaMemset(sim->d_status, 0, sizeof(uint32_t)));
  if (st & 2u) return fail(sim, MG_ERR_TIMEOUT, "a bounded wait in the step kernel gave up; results are invalid");
  if (st & 1u) return fail(sim, MG_ERR_NONFINITE, "a step produced a non-finite state");
  return MG_OK;
}

// Launch-shape autotuner. Candidates: one lane per env (128-env blocks) with
// every persistent grid from 1 resident block per SM to the kernels'
// occupancy limit, and, when some launch of the rollout can take it, a lane
// pair per env (64-env blocks, one block per half tile). Each candidate
// times the rollout shape it will serve: n_steps steps with the observation
// and reward of every step (one warm-up, then the best of three), from the
// same saved state, which is put back afterwards.
int mg_autotune(mg_sim* sim, int32_t n_steps, mg_stream_t stream, mg_launch_shape* out) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (n_steps < 0 || n_steps > 4096) return fail(sim, MG_ERR_INVALID_ARG, "autotune: n_steps %d not in 0..4096", n_steps);
  const int steps = n_steps > 0 ? n_steps : 20;
  cudaStream_t st = (cudaStream_t)stream;
  float *d_save = nullptr, *d_act = nullptr, *d_obs = nullptr;
  const size_t obs_floats = (size_t)steps * sim->n_slots * 14;
  auto release = [&]() {
    if (d_save) cudaFree(d_save);
    if (d_act) cudaFree(d_act);
    if (d_obs) cudaFree(d_obs);
  };
  if (cudaMalloc(&d_save, sizeof(float) * sim->state_floats) != cudaSuccess ||
      cudaMalloc(&d_act, sizeof(float) * sim->act_floats * steps) != cudaSuccess ||
      cudaMalloc(&d_obs, sizeof(float) * obs_floats) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(sim, MG_ERR_OOM, "autotune: scratch allocation failed");
  }
  CK(cudaMemcpyAsync(d_save, sim->d_state, sizeof(float) * sim->state_floats, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(d_act, 0, sizeof(float) * sim->act_floats * steps, st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int old_lanes = sim->lanes, old_bps = sim->blocks_per_sm;
  int occ = 1 << 30;
  bool pair_any = false;
  StepArgs probe = step_args(sim);
  probe.n_steps = steps;
  probe.obs_every = 1;
  for (const Group& g : step_plan(sim, steps >= MG_SPLIT_MIN_STEPS).groups) {
    int o = 0;
    if (step_kernel_occupancy(g.nt, param_mode(sim), g.var, g.cls >= 0, sim->cfg.task == 1, &o) != cudaSuccess) o = 1;
    occ = std::min(occ, std::max(o, 1));
    pair_any = pair_any || pair_eligible(sim, g, probe);
  }
  if (occ == (1 << 30)) occ = 1;
  std::vector<std::pair<int, int>> cand;   // (lanes, blocks per SM)
  for (int b = 1; b <= occ; ++b) cand.push_back({1, b});
  if (pair_any) cand.push_back({2, 0});
  float best = 1e30f;
  int best_lanes = 1, best_bps = 0;
  int rc = MG_OK;
  for (const auto& c : cand) {
    sim->lanes = c.first;
    sim->blocks_per_sm = c.second;
    float ms = 1e30f;
    for (int rep = 0; rep < 4 && rc == MG_OK; ++rep) {
      cudaMemcpyAsync(sim->d_state, d_save, sizeof(float) * sim->state_floats, cudaMemcpyDeviceToDevice, st);
      cudaEventRecord(e0, st);
      rc = mg_rollout(sim, d_act, steps, d_obs, d_obs + (size_t)steps * sim->n_slots * 13, 0, stream);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float x = 0.0f;
      cudaEventElapsedTime(&x, e0, e1);
      if (rep > 0) ms = std::min(ms, x);
    }
    if (rc != MG_OK) break;
    if (ms < best) { best = ms; best_lanes = c.first; best_bps = c.second; }
  }
  sim->lanes = rc == MG_OK ? best_lanes : old_lanes;
  sim->blocks_per_sm = rc == MG_OK ? best_bps : old_bps;
  cudaMemcpyAsync(sim->d_state, d_save, sizeof(float) * sim->state_floats, cudaMemcpyDeviceToDevice, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  drop_recording(sim);
  if (rc != MG_OK) return rc;
  if (e != cudaSuccess) return fail(sim, MG_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  CK(cudaGetLastError());
  if (out) {
    mg_get_launch_shape(sim, out);
    out->us_per_step = 1e3 * best / steps;
  }
  return MG_OK;
}

int mg_get_launch_shape(const mg_sim* sim, mg_launch_shape* out) {
  if (!sim || !out) return MG_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->lanes_per_env = sim->lanes;
  out->envs_per_block = sim->threads / sim->lanes;
  out->blocks_per_sm = sim->blocks_per_sm;
  out->specialised = sim->specialise;
  // Launches of a single step that run class-specialised kernels (compiled
  // here if they were not yet).
  mg_sim* s = const_cast<mg_sim*>(sim);
  mg_sim::Plan& p = const_cast<mg_sim::Plan&>(step_plan(s));
  for (size_t i = 0; i < p.groups.size(); ++i)
    if (plan_jit(s, p, i, false)) out->specialised_launches++;
  return MG_OK;
}

int mg_set_launch_shape(mg_sim* sim, const mg_launch_shape* shape) {
  if (!sim || !shape) return MG_ERR_INVALID_ARG;
  if (shape->lanes_per_env != 1 && shape->lanes_per_env != 2)
    return fail(sim, MG_ERR_INVALID_ARG, "set_launch_shape: lanes_per_env %d not 1 or 2", shape->lanes_per_env);
  if (shape->blocks_per_sm < 0)
    return fail(sim, MG_ERR_INVALID_ARG, "set_launch_shape: negative blocks_per_sm %d", shape->blocks_per_sm);
  if (shape->specialised != 0 && shape->specialised != 1)
    return fail(sim, MG_ERR_INVALID_ARG, "set_launch_shape: specialised %d not 0 or 1", shape->specialised);
  sim->lanes = shape->lanes_per_env;
  sim->blocks_per_sm = shape->blocks_per_sm;
  if (sim->specialise != shape->specialised) {
    sim->specialise = shape->specialised;
    sim->plan.valid = sim->plan_ms.valid = false;
  }
  return MG_OK;
}

int mg_set_blocks_per_sm(mg_sim* sim, int32_t blocks_per_sm) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (blocks_per_sm < 0) return fail(sim, MG_ERR_INVALID_ARG, "set_blocks_per_sm: negative count %d", blocks_per_sm);
  sim->blocks_per_sm = blocks_per_sm;   // the step plan is rebuilt for the new value
  return MG_OK;
}

int mg_graph_capture(mg_sim* sim, const float* actions_dev, int32_t n_steps, float* obs_dev, float* reward_dev,
                     mg_stream_t stream, mg_graph** out) {
  if (!sim || !out) return MG_ERR_INVALID_ARG;
  if (!stream) return fail(sim, MG_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = mg_rollout(sim, actions_dev, n_steps, obs_dev, reward_dev, 0, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != MG_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return fail(sim, MG_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  mg_graph* G = new mg_graph();
  G->graph = g;
  G->sim = sim;
  e = cudaGraphInstantiate(&G->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    delete G;
    return fail(sim, MG_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  *out = G;
  return MG_OK;
}

int mg_graph_launch(mg_graph* g, mg_stream_t stream) {
  if (!g) return MG_ERR_INVALID_ARG;
  if (g->sim) drop_recording(g->sim);
  return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

int mg_graph_destroy(mg_graph* g) {
  if (!g) return MG_ERR_INVALID_ARG;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return MG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free adjoint: as mg_step_backward, with the segment-recompute
// scratch taken from the library's fixed device array (mg_noalloc.cu).
// ---------------------------------------------------------------------------
namespace mg {
cudaError_t noalloc_scratch(float** ptr, size_t* capacity_floats);
}  // namespace mg

extern "C" int mg_step_backward_noalloc(mg_sim* sim, const float* actions_dev, const float* g_obs,
                                        const float* g_rew, const float* g_state_T, float* g_actions,
                                        float* g_added_mass, float* g_damping, float* g_state0,
                                        mg_stream_t stream) {
  if (!sim) return MG_ERR_INVALID_ARG;
  if (sim->rec_T <= 0)
    return fail(sim, MG_ERR_STATE,
                "backward: no recorded rollout (call mg_rollout with record=1; a later step, reset, graph replay "
                "or state / parameter / task / payload change discards the recording)");
  if (!actions_dev) return fail(sim, MG_ERR_INVALID_ARG, "backward: actions required");
  float* scratch = nullptr;
  size_t cap = 0;
  CK(noalloc_scratch(&scratch, &cap));
  const size_t need = adjoint_scratch_floats(sim->ckpt_every, sim->cfg.K, sim->n_slots);
  if (need > cap)
    return fail(sim, MG_ERR_INVALID_ARG,
                "backward_noalloc: scratch of %zu floats needed (2*(ckpt_every*K+1)*28*n_slots), the fixed array "
                "holds %zu; lower ckpt_every or the env count",
                need, cap);
  AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.segs = sim->d_segs;
  a.classes = sim->d_cls;
  a.planes = sim->d_planes;
  a.n_slots = sim->n_slots;
  a.actions = actions_dev;
  a.act_stride = sim->act_floats;
  a.T = sim->rec_T;
  a.ckpt_every = sim->ckpt_every;
  a.ckpt = sim->d_ckpt;
  a.scratch = scratch;
  a.g_obs = g_obs;
  a.g_rew = g_rew;
  a.g_state_T = g_state_T;
  a.g_actions = g_actions;
  a.g_A = g_added_mass;
  a.g_D = g_damping;
  a.g_state0 = g_state0;
  cudaStream_t st = (cudaStream_t)stream;
  if (g_actions) CK(cudaMemsetAsync(g_actions, 0, sizeof(float) * sim->rec_T * sim->act_floats, st));
  return launch_backward(sim, a, st);
}
