/*
 * marinegym.h - C-ABI of libmarinegym, the B300 (sm_103a) batched underwater
 * vehicle step of MarineGym (arXiv 2503.09203).
 *
 * One call advances many independent environments (one vehicle each) by the
 * Fossen equation of motion of Sec. III-B, Eq. 1:
 *     tau = M nu_dot + C(nu) nu + D(nu) nu + g(eta),
 * split as in Eq. 2 into the rigid-body term (M_RB, C_RB, g_RB) and the
 * hydrodynamic term of Eq. 3 (M_A, C_A, D, g_A), the latter evaluated at the
 * relative velocity nu_r = nu - nu_c against an ocean current (Sec. III-B,
 * paragraph after Eq. 3). Actuators follow Sec. III-D: a first-order rotor lag
 * (zero-order when the time constant is 0), quadratic thrust k n|n| with a
 * dead zone, and forces applied at fixed actuator frames (a 6 x n_thr
 * allocation matrix). Domain randomisation follows Sec. III-C and the ranges of
 * Table 2; the hover (station-keeping) observation and reward follow Sec. IV-B.
 *
 * Conventions. NED world frame (z down, gravity +z), body frame x forward,
 * y starboard, z down. Pose: position p (3) and unit quaternion q = (w,x,y,z),
 * Hamilton, body -> NED. Body velocity nu = (u,v,w,p,q,r). Added-mass and
 * damping coefficients are positive magnitudes. The integrator is
 * semi-implicit Euler over K substeps of h = dt/K per control step (the paper
 * names no integrator).
 *
 * Memory and errors. All pointers named *_dev are device pointers owned by the
 * caller; they must stay valid until the work queued on `stream` completes.
 * The library owns the simulator state and never frees caller memory. Every
 * call returns MG_OK (0) or a negative MG_ERR_* code; the text of the last
 * error is returned by mg_last_error(). Calls that take a stream are
 * asynchronous on it; a non-finite state produced by a step is reported by the
 * next mg_status() call (it synchronises the stream).
 *
 * Environment order. Environments are grouped by class: class 0 owns env
 * indices [0, n_0), class 1 owns [n_0, n_0 + n_1), and so on. Per-env arrays
 * (observations, rewards) are indexed by *slot*: each class's first slot is a
 * multiple of 4, so class c occupies slots [slot_offset_c, slot_offset_c +
 * n_c) and up to 3 padding slots may follow it. mg_get_layout() reports all
 * offsets. Grouping by class lets one kernel instantiation (one thruster
 * count, one class table) walk contiguous, 16-byte aligned SoA planes; a
 * caller whose environments carry an arbitrary class map env_class[i] gets
 * the library's order from mg_env_order() (a stable sort by class: library
 * env index lib_env[i] of its env i) and passes the resulting class_counts to
 * mg_create.
 */
#ifndef MARINEGYM_H
#define MARINEGYM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mg_stream_t; /* same type as cudaStream_t */

enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = -1,      /* bad handle, size, pointer or value */
  MG_ERR_OOM = -2,              /* device allocation failed or budget exceeded */
  MG_ERR_CUDA = -3,             /* a CUDA runtime call failed */
  MG_ERR_NONFINITE = -4,        /* a step produced a NaN or Inf state */
  MG_ERR_TIMEOUT = -5,          /* a bounded device wait gave up */
  MG_ERR_ADMISSION_REFUSED = -6,/* serving: request can never fit the budget */
  MG_ERR_STATE = -7             /* call order (e.g. backward with no recorded rollout) */
};

#define MG_MAX_THR 8
#define MG_MAX_CLASSES 16
#define MG_STATE_DIM 21   /* canonical host state record: p3 q4 nu6 n8 */
#define MG_OBS_DIM 13     /* hover observation: R^T(p-p*) 3, q 4 (w>=0), v 3, w 3 */
#define MG_ENV_PARAM_DIM 34 /* canonical host per-env parameter record (doubles) */

/* Actuator kinds (Sec. III-D: multirotor, rudder-propeller and tiltrotor
 * types). Every channel has a first-order state n in [-1, 1] driven by its
 * command with alpha = 1 - exp(-h/T_rotor) (rotor speed, or a servo / fin
 * angle n * act_range).
 * MG_ACT_PROP  propeller: thrust k_f n|n| (0 inside the dead zone) along thr_dir
 *              at thr_pos.
 * MG_ACT_SERVO servo: no force; tilts the MG_ACT_TILT propellers linked to it.
 * MG_ACT_FIN   fin at thr_pos with span axis act_axis and chord act_chord at
 *              zero deflection (unit, orthogonal), deflected by n * act_range
 *              about the span. With u = v_r + w x r (v_r relative to the water)
 *              projected on the plane normal to the span, U = |u|, and the
 *              angle of attack a of u from the deflected chord towards
 *              act_axis x chord: lift 1/2 rho S U^2 C_L(a) along -(act_axis x u)/U,
 *              drag 1/2 rho S U^2 C_D(a) along -u/U, C_L = fin_cl sin a cos a,
 *              C_D = fin_cd0 + fin_cda sin^2 a, S = fin_area.
 * MG_ACT_TILT  propeller whose direction thr_dir is turned about act_axis by
 *              the angle of servo channel act_link (Rodrigues). */
#define MG_ACT_PROP 0
#define MG_ACT_SERVO 1
#define MG_ACT_FIN 2
#define MG_ACT_TILT 3

/* A vehicle class (Sec. III-D model library): rigid body, hydrodynamic
 * coefficients and up to 8 actuator channels. FP64 on the host; the library
 * derives the allocation matrix B = [d_i ; r_i x d_i] of the fixed
 * propellers, the fin and tilt tables, the lag factor alpha = 1 - exp(-h/T)
 * and the inverse inertia in FP64 and stores them FP32. The class's own CoG
 * is the body origin (r_g = 0) and its added mass is diagonal; an off-origin
 * CoG arises from a payload (see mg_set_payload). A class with any channel
 * other than MG_ACT_PROP (a "generic" class) has the step, the adjoint
 * (Euler), the FP64 check path and serving, but no payload. */
typedef struct {
  int32_t n_thr;            /* 1..8 (the workloads use 4, 6, 8) */
  int32_t pad0;
  double mass;              /* kg */
  double Ig[3];             /* principal inertia about the CoG, kg m^2 */
  double rg[3];             /* CoG in body frame (must be 0; payloads move it) */
  double rb[3];             /* CoB in body frame, m */
  double buoy_ratio;        /* B / (mass g) at nominal volume (1 = neutral) */
  double Ma[6];             /* added mass diag (kg, kg m^2) */
  double dl[6];             /* linear damping diag */
  double dq[6];             /* quadratic damping diag */
  double thr_pos[8][3];     /* thruster positions, body frame, m */
  double thr_dir[8][3];     /* thruster unit directions, body frame */
  double k_f[8];            /* thrust at |n| = 1, N */
  double T_rotor[8];        /* rotor time constant, s; 0 = zero-order model */
  double deadzone[8];       /* |n| below which the thrust is 0 */
  int32_t act_kind[8];      /* MG_ACT_* (all 0: a propeller-only class) */
  int32_t act_link[8];      /* MG_ACT_TILT: its servo channel */
  double act_axis[8][3];    /* fin span axis / tilt axis (unit, body frame) */
  double act_chord[8][3];   /* fin chord at zero deflection (unit, normal to the axis) */
  double act_range[8];      /* servo / fin angle at |n| = 1, rad (> 0) */
  double fin_area[8];       /* m^2 */
  double fin_cl[8];         /* lift slope, 1/rad */
  double fin_cd0[8];        /* drag at zero angle of attack */
  double fin_cda[8];        /* drag growth with sin^2 of the angle of attack */
  double rho;               /* water density, kg/m^3 (> 0 with fins) */
} mg_class_desc;

/* Reset configuration: domain randomisation (Sec. III-C, Table 2 train
 * column shape) and the initial state. Uniform draws come from Philox4x64-10
 * (Salmon et al. 2011) keyed by (seed, stream) with counter (env, draw/4, 0, 0).
 * DR factors: mass (inertia scales with it), each added-mass coefficient, each
 * linear and quadratic damping coefficient, CoB offset; current speed
 * U[cur_lo, cur_hi] with heading U[0, 2 pi) (horizontal unless current_3d). */
typedef struct {
  int32_t dr_enabled;
  int32_t current_enabled;
  int32_t current_3d;
  int32_t init_mode;        /* 0: rest at the origin; 1: hover-task random pose */
  double mass_lo, mass_hi;
  double added_lo, added_hi;
  double damp_lo, damp_hi;
  double cob_lo, cob_hi;
  double cur_lo, cur_hi;
  double target_half;       /* hover target p* ~ U[-L, L]^3 */
  double pos_radius;        /* |p - p*| uniform in a ball of this radius */
  double max_angle;         /* attitude error angle ~ U[0, max_angle], rad */
  int32_t track_kind;       /* tracking runs: 0 helix, 1 Lissajous reference */
  int32_t pad0;
  double payload_lo, payload_hi;   /* payload runs: m_p / m ~ U[lo, hi] (Table 2: [0, 0.3]) */
} mg_reset_cfg;

typedef struct {
  int32_t n_classes;            /* 1..MG_MAX_CLASSES */
  const int32_t* class_counts;  /* host [n_classes]: envs per class (>= 0) */
  double dt;                    /* control step, s (> 0) */
  int32_t K;                    /* substeps per control step (1..64) */
  int32_t per_env_params;       /* 1: per-env parameter block (needed for DR,
                                   current and gradients); 0: class values */
  mg_reset_cfg reset;
  int32_t record_steps;         /* longest rollout mg_step_backward may
                                   differentiate (0: no gradient buffers) */
  int32_t ckpt_every;           /* checkpoint interval in steps (0: 20) */
  size_t mem_budget;            /* 0: none; else mg_create fails with
                                   MG_ERR_OOM above this many device bytes */
  int32_t task;                 /* 0: station keeping (fixed target p*);
                                   1: trajectory tracking (time-varying p*(t)) */
  int32_t payload;              /* 1: every env carries a point-mass payload
                                   (needs per_env_params) */
  int32_t integrator;           /* MG_INTEG_EULER (semi-implicit Euler per
                                   substep) or MG_INTEG_RK4 (classical RK4 on
                                   p, q, nu with the actuator states held over
                                   the substep; mg_step_backward reverses its
                                   four stages from the recorded substep
                                   start) */
  int32_t pad1;
} mg_config;

#define MG_INTEG_EULER 0
#define MG_INTEG_RK4 1

/* Placement of class c inside the device buffers. */
typedef struct {
  int32_t n_envs, n_thr, env_offset, slot_offset;
  int64_t state_offset;   /* floats, start of the class's AoS state block */
  int32_t state_stride;   /* floats per env: 13 + n_thr (p3 q4 nu6 n[n_thr]) */
  int32_t pad0;
  int64_t action_offset;  /* floats, start of the class's [n_slots_c][n_thr] actions */
} mg_class_layout;

typedef struct {
  int32_t n_classes, n_envs, n_slots;
  int32_t launches_per_step;  /* kernel launches one mg_step call makes (one per
                               * thruster count and step variant; large steps of
                               * class-constant propeller classes: one per class) */
  int64_t action_floats;  /* floats per control step in an actions buffer */
  int64_t state_floats;
  mg_class_layout cls[MG_MAX_CLASSES];
} mg_layout;

typedef struct mg_sim mg_sim;

/* Create a simulator: validates the classes (n_thr in 1..8, r_g = 0, positive
 * mass and inertia, non-negative coefficients) and allocates the device state,
 * parameter, target and (if record_steps > 0) checkpoint buffers on the
 * current device. The state starts at rest; call mg_reset to sample.
 * Errors: INVALID_ARG, OOM (allocation failed or above mem_budget), CUDA. */
int mg_create(const mg_config* cfg, const mg_class_desc* classes, mg_sim** out);
int mg_destroy(mg_sim* sim);
int mg_get_layout(const mg_sim* sim, mg_layout* out);

/* Reset envs (indices into [0, n_envs), device int32 array; NULL = all,
 * then n is ignored): sample DR parameters (if enabled), the current (if
 * enabled), the hover target and the initial state from `seed`
 * (Sec. III-C, Table 2; reading of the DR ranges as independent per-coefficient
 * factors). Inverse inertia is computed in FP64 on the GPU. */
int mg_reset(mg_sim* sim, const int32_t* env_ids_dev, int32_t n, uint64_t seed, mg_stream_t stream);

/* Advance all envs by n_steps control steps (K substeps each, zero-order hold
 * of clamp(action, -1, 1)). actions_dev: [n_steps][action_floats] floats laid
 * out per mg_layout (class c's [n_envs_c][n_thr_c] row-major block at
 * action_offset_c). obs_dev [n_slots][13] and reward_dev [n_slots] receive the
 * hover observation and reward r = -|p-p*|^2 - 0.1|nu|^2 - 0.01|c|^2 after
 * the last step; either may be NULL. Padding slots receive zeros. */
int mg_step(mg_sim* sim, const float* actions_dev, int32_t n_steps, float* obs_dev, float* reward_dev,
            mg_stream_t stream);

/* As mg_step, with observations and rewards written after EVERY step:
 * obs_dev [n_steps][n_slots][13], reward_dev [n_steps][n_slots] (either may be
 * NULL). The whole rollout is one persistent launch with the state held in
 * registers. record != 0 stores checkpoints every ckpt_every steps for
 * mg_step_backward (needs n_steps <= record_steps and per_env_params). */
int mg_rollout(mg_sim* sim, const float* actions_dev, int32_t n_steps, float* obs_dev, float* reward_dev,
               int32_t record, mg_stream_t stream);

/* Trajectory tracking (task = 1; Sec. IV-B tracking task). Every env follows
 * p*(t) = c + a o sin(w t + phi) + v t with t = k dt and k the env's step
 * counter (reset to 0 by mg_reset, advanced by every step). The observation
 * and reward of mg_step / mg_rollout / mg_observe use p*(t) in place of the
 * fixed target, evaluated at the step's end time. Reset draws (stream 2, draws
 * 9..): helix (track_kind 0): radius R ~ U[1, 3] m, rate W ~ U[0.2, 0.6]
 * rad/s, phase psi ~ U[0, 2 pi), climb v_z ~ U[-0.2, 0.2] m/s, so
 * p*(t) = c + (R cos(W t + psi), R sin(W t + psi), v_z t);
 * Lissajous (track_kind 1): a_i ~ U[1, 3] m, w_i ~ U[0.2, 0.6] rad/s,
 * phi_i ~ U[0, 2 pi), v = 0. The initial position is drawn around p*(0).
 * mg_get_task / mg_set_task read and write the reference as [n_envs][16]
 * doubles: c[3], a[3], w[3], phi[3], v[3], k (hover runs: c and k only,
 * the rest 0). Both synchronise the device. */
int mg_get_task(const mg_sim* sim, double* host, size_t bytes);
int mg_set_task(mg_sim* sim, const double* host, size_t bytes);

/* Payload disturbance (payload = 1; Sec. III-B mission payloads, Table 2
 * payload mass). A point mass m_p rigidly attached at r_p (body frame, m)
 * moves the CoG to r_g = m_p r_p / (m + m_p) and couples translation and
 * rotation: the step then uses the full 6x6 inverse of M_RB + M_A (Eq. 1,
 * M_RB about the body origin with the S(m r_g) blocks), C_RB with r_g and the
 * weight (m + m_p) g acting at r_g. The inverse is computed in FP64 (Cholesky)
 * at reset and whenever the parameters change. Reset draws (stream 1, draws
 * 23..26): m_p = U[payload_lo, payload_hi] x the env's vehicle mass, r_p with
 * x, y ~ U[-0.1, 0.1] and z ~ U[0.05, 0.15] (below the vehicle's CoG); drawn
 * whether or not DR is enabled. The payload's own volume is neglected.
 * mg_get_payload / mg_set_payload read and write [n_envs][4] doubles
 * (m_p, r_p x, y, z); mg_get_params / mg_set_params keep describing the
 * vehicle alone (mg_set_params recomputes the combined body). Both synchronise
 * the device. Errors: INVALID_ARG (not a payload run, buffer too small,
 * non-finite values, m_p < 0, an inertia that is not positive definite).
 * Payload runs reject mg_set_hydro (use mg_set_params). */
int mg_get_payload(const mg_sim* sim, double* host, size_t bytes);
int mg_set_payload(mg_sim* sim, const double* host, size_t bytes);

/* Observation of the current state (no step): obs_dev [n_slots][13] and
 * reward_dev [n_slots] (either may be NULL, not both). The reward is the hover
 * reward of the current state without a command term:
 * r = -|p - p*|^2 - 0.1 |nu|^2 (Sec. IV-B station keeping; the command term of
 * mg_step's reward belongs to the step that applied it). */
int mg_observe(mg_sim* sim, float* obs_dev, float* reward_dev, mg_stream_t stream);

/* Library order of an arbitrary env -> class map (no device work, no
 * simulator needed): class_counts [n_classes] receives the number of envs of
 * each class (the mg_config.class_counts to create the simulator with) and
 * lib_env [n_envs] the library env index of env i (envs sorted by class,
 * stable: envs of one class keep their order). Per-env data of env i lives at
 * library env lib_env[i] (slot: that env's class slot_offset + its index
 * within the class). Errors: INVALID_ARG (a class outside [0, n_classes), null
 * buffers); the message is read with mg_last_error(NULL). */
int mg_env_order(const int32_t* env_class, int32_t n_envs, int32_t n_classes, int32_t* class_counts,
                 int32_t* lib_env);

/* Host-buffer variant of mg_step for callers without device memory: copies
 * actions (host, as for mg_step) in, steps, copies obs/reward (host, may be
 * NULL) out, and returns when all of it is done. The envs are cut into chunks
 * of consecutive tiles: actions of chunk c are copied in on a library stream
 * while chunk c-1 steps on `stream` and chunk c-2's results are copied out on
 * another library stream, so that copies in both directions overlap. Work
 * queued on `stream` before the call completes first. Host buffers should be
 * pinned for asynchronous copies. */
int mg_step_host(mg_sim* sim, const float* actions_host, int32_t n_steps, float* obs_host, float* reward_host,
                 mg_stream_t stream);

/* Reverse-mode gradient of the last recorded mg_rollout (discretise-then-
 * differentiate: the exact adjoint of the discrete map, including the clamp,
 * rotor lag, quaternion renormalisation, and M^-1 = (M_RB + M_A)^-1 through
 * the added mass; in payload runs the combined body's full inverse, its
 * inertia about the origin and the off-origin centre-of-gravity terms, with
 * g_added_mass the gradient with respect to the diagonal added mass M_A).
 * Inputs: the same actions_dev (the library keeps no copy of
 * the caller's actions; the segments between checkpoints are recomputed from
 * them), cotangents g_obs [T][n_slots][13] and g_rew [T][n_slots] (either may
 * be NULL = 0) and g_state_T [n_slots][21] on the final state (NULL = 0).
 * Outputs (each may be NULL): g_actions [T][action_floats], g_added_mass
 * [n_slots][6], g_damping [n_slots][12] (6 linear then 6 quadratic),
 * g_state0 [n_slots][21] (the cotangent of the rollout's initial state, so
 * that a long rollout cut into recorded pieces chains its gradients through
 * g_state_T of the previous piece). Segments between checkpoints are
 * recomputed into library-owned scratch.
 * A recording stays valid only until the simulator changes: mg_step,
 * mg_rollout, mg_step_host, mg_reset, mg_set_state, mg_set_params,
 * mg_set_hydro, mg_set_task, mg_set_payload, mg_autotune, mg_graph_capture
 * and mg_graph_launch of a graph of this simulator all discard it.
 * Errors: STATE if nothing is recorded (never recorded, or discarded). */
int mg_step_backward(mg_sim* sim, const float* actions_dev, const float* g_obs, const float* g_rew,
                     const float* g_state_T, float* g_actions, float* g_added_mass, float* g_damping,
                     float* g_state0, mg_stream_t stream);

/* Allocation-free variant of mg_step_backward (the paper has no counterpart;
 * this is an interface for callers that cannot allocate device memory while
 * they run the backward pass: a host framework whose own pool owns the
 * device, a process whose memory budget is already committed, or a loop that
 * must not take cudaMalloc's implicit device synchronisation).
 * Same arguments, outputs and errors as mg_step_backward, but the segment-
 * recompute scratch is a fixed 32 MiB array compiled into the library (held
 * by every GPU that loads it until the process exits) instead of the
 * simulator's own scratch buffer; the call allocates nothing.
 * Limit: 2 * (ckpt_every * K + 1) * 28 * n_slots <= 8,388,608 floats, else
 * MG_ERR_INVALID_ARG with the sizes in mg_last_error(). Every entry of the
 * scratch that the kernel reads it writes earlier in the same call, so nothing
 * needs clearing between calls; the array keeps the last call's contents.
 * All calls share the one array: calls that overlap on the GPU (for example on
 * two streams) race. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and caches it with the current context; make
 * that first call before any stream capture. A call in a new context of the
 * device (after cudaDeviceReset) looks the address up again, so it too should
 * come before any capture. Also a backward pass: the recording rules of
 * mg_step_backward apply. */
int mg_step_backward_noalloc(mg_sim* sim, const float* actions_dev, const float* g_obs, const float* g_rew,
                             const float* g_state_T, float* g_actions, float* g_added_mass, float* g_damping,
                             float* g_state0, mg_stream_t stream);

/* The current recording: *steps = its length T (0: none) and *id = a
 * process-unique identity (0: none), which changes with every new recording.
 * A caller that keeps a recording across other work (an autograd graph)
 * stores the id and checks it before mg_step_backward. Either may be NULL. */
int mg_recording(const mg_sim* sim, int32_t* steps, uint64_t* id);

/* Overwrite the added-mass (A [n_slots][6]), linear damping (dl) and quadratic
 * damping (dq) of every env from device arrays (each may be NULL = keep) and
 * recompute M^-1 in FP64 on the GPU. Needs per_env_params. */
int mg_set_hydro(mg_sim* sim, const float* A_dev, const float* dl_dev, const float* dq_dev, mg_stream_t stream);

/* FP64 rollout used only for finite-difference checks: runs the double
 * instantiation of the step from the current state (not modified) with the
 * current parameters, the added mass and damping optionally perturbed by
 * eps * (dA, ddl, ddq) (device doubles [n_slots][6] each, NULL = 0), and writes
 * reward_dev [n_steps][n_slots] (double) and, if not NULL, the final state
 * state_dev [n_slots][21] (double). Inverse inertia is recomputed in FP64
 * (payload runs: the combined body's full inverse, by Cholesky). Every class
 * and integrator: fins and tilted propellers with their FP64 tables, RK4. */
int mg_rollout_fp64(mg_sim* sim, const float* actions_dev, int32_t n_steps, const double* dA,
                    const double* ddl, const double* ddq, double eps, double* reward_dev, double* state_dev,
                    mg_stream_t stream);

/* Checkpoint / resume: the state as [n_envs][21] floats (canonical record,
 * rotor entries beyond n_thr are 0), and the per-env parameters as
 * [n_envs][34] doubles: mass, Ig[3], rb[3], W, B, Ma[6], dl[6], dq[6], Vc[3],
 * target[3], pad. Setting parameters recomputes M^-1 in FP64 (the live
 * re-tuning interface of Sec. III-C). These calls synchronise the device. */
int mg_get_state(const mg_sim* sim, float* host, size_t bytes);
int mg_set_state(mg_sim* sim, const float* host, size_t bytes);
int mg_get_params(const mg_sim* sim, double* host, size_t bytes);
int mg_set_params(mg_sim* sim, const double* host, size_t bytes);

/* Synchronise `stream`; return MG_ERR_TIMEOUT if a bounded wait of a step
 * kernel gave up (its results are invalid), else MG_ERR_NONFINITE if any step
 * since the last call produced a non-finite state, else MG_OK; the flags are
 * cleared. Every wait of the step kernel on its own copies gives up after 2 s,
 * so a stalled copy ends the kernel with an error instead of a hang. */
int mg_status(mg_sim* sim, mg_stream_t stream);

/* Test hook for the failure path (no counterpart in the paper): one step
 * launch in which no copies are issued, so every warp's wait runs out after
 * limit_ns (0 < limit_ns <= 2 s) and the warp leaves with the timeout flag
 * set; the state is not touched. The next mg_status returns MG_ERR_TIMEOUT and
 * the simulator stays usable. Synchronises `stream`. */
int mg_test_wait_timeout(mg_sim* sim, uint64_t limit_ns, mg_stream_t stream);

/* Launch shape of the step launches (no counterpart in the paper: how the
 * batched step maps onto the GPU).
 * lanes_per_env 1: one env per thread, tiles of 128 envs per block, each
 *   launch a persistent grid of blocks_per_sm resident blocks per SM (0: the
 *   kernels' occupancy limit).
 * lanes_per_env 2: a lane pair per env (the linear-momentum and the
 *   angular-momentum rows of the equation of motion on two lanes), 64 envs
 *   per block, one block per half tile. It serves the launches of one class
 *   (those of large steps and of long rollouts) of propeller classes with the
 *   Euler substep, class-constant or per-env parameters and the hover task
 *   (recorded rollouts included); every other launch keeps one lane per env.
 *   Results agree with the one-lane kernel to rounding (the rows are summed
 *   in another order), not bit for bit.
 * specialised: the class-specialised kernels are the one-lane step kernel
 *   compiled again with the class's constants as literals, so that zero
 *   allocation entries, a restoring arm on the body axis and W = B fold away;
 *   the first launch of a class compiles its kernel (about half a second;
 *   kept for the process). Results agree with the library-built kernel to
 *   rounding.
 * The K substeps of a step (and the steps of a multi-step launch) always stay
 * in one launch with the state in registers: splitting them over launches
 * would only add state traffic. */
typedef struct {
  int32_t lanes_per_env;    /* 1 or 2 */
  int32_t envs_per_block;   /* 128 / lanes_per_env (output only) */
  int32_t blocks_per_sm;    /* one-lane launches: resident blocks per SM (0: occupancy limit) */
  int32_t specialised;      /* 1 (default): one-lane launches of one class (propellers, Euler,
                               hover task; class-constant or per-env parameters, no payload) run a
                               kernel compiled at run time (NVRTC) with that class's constants
                               (per-env runs: its actuator tables) as literals, when NVRTC is
                               available; 0: the kernels built with the library */
  double us_per_step;       /* mg_autotune: the chosen shape's measured time per step (output only) */
  int32_t specialised_launches; /* output: launches of one step that run specialised kernels */
  int32_t pad0;
} mg_launch_shape;

/* Choose the launch shape by timing candidates on `stream`: one lane per env
 * with every persistent grid from 1 resident block per SM to the occupancy
 * limit, and a lane pair per env when a launch can take it. Each candidate
 * runs a rollout of n_steps steps (0: 20) with observations and rewards every
 * step, the shape of the rollouts and graphs it will serve, from the current
 * state, which is restored afterwards (a recording is discarded). Allocates
 * scratch of about n_steps * n_slots * 56 bytes plus the state and the
 * actions of n_steps steps. Writes the choice into *out if not NULL. */
int mg_autotune(mg_sim* sim, int32_t n_steps, mg_stream_t stream, mg_launch_shape* out);
int mg_get_launch_shape(const mg_sim* sim, mg_launch_shape* out);
/* Fix the launch shape by hand (lanes_per_env 1 or 2, blocks_per_sm >= 0,
 * specialised 0 or 1); takes effect from the next launch. Errors:
 * INVALID_ARG. mg_get_launch_shape compiles the specialised kernels of the
 * current plan if they were not yet, to report specialised_launches. */
int mg_set_launch_shape(mg_sim* sim, const mg_launch_shape* shape);

/* Fix the persistent grid: blocks_per_sm resident blocks of each step launch
 * per SM (0: the kernel's occupancy limit, the default; values above it are
 * capped by it). Takes effect from the next launch on any stream; a captured
 * graph keeps the grid it was captured with. Errors: INVALID_ARG (negative). */
int mg_set_blocks_per_sm(mg_sim* sim, int32_t blocks_per_sm);

/* CUDA-graph capture of mg_rollout(actions, n_steps, obs, reward, record=0)
 * on `stream`; mg_graph_launch replays it. Buffers are bound at capture. */
typedef struct mg_graph mg_graph;
int mg_graph_capture(mg_sim* sim, const float* actions_dev, int32_t n_steps, float* obs_dev, float* reward_dev,
                     mg_stream_t stream, mg_graph** out);
int mg_graph_launch(mg_graph* g, mg_stream_t stream);
int mg_graph_destroy(mg_graph* g);

/* Algorithmic FP32 operations (FMA = 2, divide and square root = 1 each) for
 * a class with n_thr thrusters, counted by running the kernels' own templated
 * arithmetic with a counting scalar on the host: one substep (with_current:
 * including the ocean-current terms, which class-constant runs compile out),
 * the observation + reward, and one substep's adjoint as the reverse pass
 * runs it (the forward recompute that records the states, the tape rebuilt
 * from the records of the substep's start and end, and the vector-Jacobian
 * product). Any output may be NULL. */
int mg_count_flops(int32_t n_thr, int32_t with_current, double* substep_flops, double* observe_flops,
                   double* adjoint_flops);

const char* mg_last_error(const mg_sim* sim);
const char* mg_strerror(int code);

/* ------------------------------------------------------------------------
 * Serving loop (continuous batching). A server owns a device arena of
 * `budget_bytes` and a scheduler thread. Each request is a rollout of n_envs
 * envs of one class for `horizon` control steps of K substeps; its actions are
 * drawn on the device from Philox4x64-10 (key (seed, 3), counter
 * (env, step, thr/4, 0), top 24 bits: a = k 2^-23 - 1). Requests are admitted
 * as soon as the arena has room, their envs live on the device until done, and
 * every scheduler tick advances all admitted requests by one step in ONE
 * shared launch. A finished request's final state ([n_envs][21] floats) and
 * per-env return (sum of rewards, [n_envs] floats) are copied to host memory
 * owned by the server and read with mg_server_poll.
 * ------------------------------------------------------------------------ */
typedef struct mg_server mg_server;

typedef struct {
  double dt;
  size_t budget_bytes;      /* arena size; 0: 50% of free device memory */
  int32_t max_requests;     /* simultaneously admitted requests (<= 4096) */
  int32_t max_queue;        /* pending requests before submit refuses */
  mg_reset_cfg reset;       /* initial state / DR per request (seeded by request) */
  int32_t integrator;       /* MG_INTEG_EULER or MG_INTEG_RK4, for every request */
  int32_t pad0;
} mg_server_config;

typedef struct {
  int32_t cls, n_envs, horizon, K;
  uint64_t seed;            /* reset draws and actions */
} mg_request;

enum { MG_REQ_PENDING = 0, MG_REQ_RUNNING = 1, MG_REQ_DONE = 2, MG_REQ_UNKNOWN = -1 };

typedef struct {
  int32_t status;           /* MG_REQ_* */
  int32_t n_envs;
  double t_submit, t_admit, t_done;   /* seconds, steady clock */
  int64_t steps_done;
  const float* final_state; /* server-owned host [n_envs][21], valid until mg_server_release */
  const float* returns;     /* server-owned host [n_envs] */
} mg_request_result;

typedef struct {
  int64_t requests_done, env_steps, ticks;
  double busy_seconds;
  double step_latency_p50, step_latency_p99;   /* s, per request step (tick completion spacing) */
  double queue_delay_p50, queue_delay_p99;     /* s, submit -> admit */
  double tick_p50, tick_p99;                   /* s, device time of one shared launch */
  size_t budget_bytes;          /* the arena budget the server was created with */
  size_t peak_resident_bytes;   /* most device bytes ever held by admitted requests at once
                                   (their slot planes, returns and states); <= budget_bytes */
  int32_t peak_requests;        /* most requests ever holding arena space at once */
  int32_t pad0;
} mg_server_stats;

/* Errors of mg_server_create: INVALID_ARG (bad config, an integrator other
 * than MG_INTEG_EULER / MG_INTEG_RK4, a class with r_g != 0), OOM. Every
 * actuator type is served (fixed propellers, fins, servo-tilted propellers)
 * with either integrator. */
int mg_server_create(const mg_server_config* cfg, const mg_class_desc* classes, int32_t n_classes,
                     mg_server** out);
int mg_server_submit(mg_server* srv, const mg_request* req, int64_t* id_out);
int mg_server_poll(mg_server* srv, int64_t id, mg_request_result* out);
int mg_server_release(mg_server* srv, int64_t id);
int mg_server_wait_idle(mg_server* srv, double timeout_s);
int mg_server_stats_get(mg_server* srv, mg_server_stats* out);
int mg_server_destroy(mg_server* srv);
const char* mg_server_last_error(const mg_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* MARINEGYM_H */
