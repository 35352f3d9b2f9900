// Shared host/device records of libmarinegym (not part of the public C-ABI).
#pragma once

#include "mg_rtc.h"

namespace mg {

// One segment of a launch: envs of a single class (and, for serving, of a
// single request) that share K, the substep length and the actuator factors.
// Tiles of `threads` envs never straddle segments.
struct SegDesc {
  int32_t tile_begin;   // first tile of this segment
  int32_t n_envs;       // valid envs
  int32_t cls;          // class index
  int32_t n_thr;
  int32_t K;
  int32_t step0;        // serving: step counter of the request at launch
  int32_t n4;           // slots of the segment's storage (n_envs rounded up to 4)
  int32_t flags;        // bit 0: the class has a nonzero dead zone; bit 1: failure-path test, issue no copies
  int64_t st_off;       // float offset of the segment's state planes
  int64_t act_off;      // float offset of the segment's [n4][n_thr] actions
  int64_t slot_off;     // first slot (obs / reward / parameter planes)
  int64_t env_base;     // global env id of local env 0 (random draws)
  float h;
  float dt;             // control step (trajectory time = step counter * dt)
  int32_t track;        // 1: trajectory-tracking reference, 0: fixed hover target
  float pad1;
  float alpha[8];
  uint64_t seed;        // serving: action seed
  uint64_t wait_limit_ns;   // bound of the waits on this segment's copies (0: 2 s)
};
static_assert(sizeof(SegDesc) == 128, "SegDesc layout");

// Generic actuator table of a class (fins, servo-tilted propellers): the kind
// of each channel (as the bits of a float, so that the table stages into
// shared memory as one float array) and 20 values per channel (layout in the
// step arithmetic's header).
struct ClassG {
  int32_t kind[8];
  float v[8][20];
};
static_assert(sizeof(ClassG) == (8 + 160) * 4, "ClassG layout");

// Per-class constants in FP32 (staged into shared memory per tile).
struct ClassF {
  float alloc[6][8];
  float kf[8];
  float dz[8];
  float phys[36];       // nominal Phys block (current 0)
  float pad[4];
  ClassG gen;           // generic actuator table (serving ticks stage it per warp)
};
static_assert(sizeof(ClassF) == (104 + 168) * 4, "ClassF layout");

// Propeller steps with class-constant or payload parameters take allocation
// rows premultiplied by the thrust constants (rows of B diag(k)): the thrust
// per channel is then n|n|, one multiply less per thruster and substep.
#ifndef MG_PREMUL
#define MG_PREMUL 1
#endif

// One class's constants passed by value as a kernel parameter (propeller
// steps with class constants launch one class at a time): the kernel reads
// them as constant-bank operands, with no shared-memory load and no register
// to hold them. Members as the actuator table (alloc, kf, dz, alpha) and the
// nominal physical block (minv .. Vc; current 0) that the step reads.
struct ClassK {
  static constexpr bool kFull = false;   // diagonal inertia, CoG at the origin
  float alloc[6][8];
  float kf[8];
  float dz[8];
  float alpha[8];
  float minv[6], A[6], dl[6], dq[6];
  float m, Ig[3], W, B, rb[3], Vc[3];
  uint32_t dz_on;       // 0: no channel has a dead zone
  uint32_t pad[3];
};
static_assert(sizeof(ClassK) == 112 * 4, "ClassK layout");

// The same table in FP64 (the finite-difference check path).
struct ClassGD {
  int32_t kind[8];
  double v[8][20];
};

// Kernel parameter of a one-class launch of a generic-actuator or RK4 step.
struct ClassKG {
  ClassK k;
  ClassG g;
};

// Per-class constants in FP64 for the finite-difference check path.
struct ClassD {
  double alloc[6][8];
  double kf[8];
  double dz[8];
  double alpha[8];
  double Mrb[6];        // rigid-body diagonal inertia (m, m, m, Ig)
};

// Per-env physical parameter block (36 floats, 9 float4 planes) field offsets.
enum { PAR_MINV = 0, PAR_A = 6, PAR_DL = 12, PAR_DQ = 18, PAR_M = 24, PAR_IG = 25, PAR_W = 28,
       PAR_B = 29, PAR_RB = 30, PAR_VC = 33, PAR_DIM = 36 };
#ifndef __CUDACC_RTC__
static_assert(offsetof(ClassK, minv) == 4 * (72 + PAR_MINV) && offsetof(ClassK, m) == 4 * (72 + PAR_M) &&
                  offsetof(ClassK, Vc) == 4 * (72 + PAR_VC),
              "ClassK physical block follows the parameter block layout");
#endif

// Number of float4 parameter planes: 9 for the 36 physical floats + 1 target.
// The target plane holds (c_x, c_y, c_z, k): the reference centre and the
// env's step counter. Tracking runs add 3 planes right after the target:
// (a_x, a_y, a_z, w_x), (w_y, w_z, phi_x, phi_y), (phi_z, v_x, v_y, v_z) of the
// reference p*(t) = c + a o sin(w t + phi) + v t, t = k dt.
enum { PAR_PLANES = 9, TGT_PLANE = 9, N_PLANES = 10, TRAJ_PLANES = 3, PAY_PLANES = 9 };
// Index of the target plane (per-env runs keep the physics in planes 0..8).
__host__ __device__ inline int tgt_plane(int per_env) { return per_env ? TGT_PLANE : 0; }
// Payload runs (per-env only) add 9 planes after the target and trajectory
// planes: the combined body's inverse inertia (21 floats, upper triangle row
// by row), its inertia about the body origin I_o (6: xx xy xz yy yz zz), its
// first moment s = m_p r_p (3), total mass m' (1), total weight W' (1), and the
// payload itself: m_p (1), r_p (3).
enum { PAY_MINV = 0, PAY_IO = 21, PAY_S = 27, PAY_M = 30, PAY_W = 31, PAY_MP = 32, PAY_RP = 33, PAY_DIM = 36 };
__host__ __device__ inline int pay_plane(int track) { return TGT_PLANE + 1 + (track ? TRAJ_PLANES : 0); }
// Planes of a run.
inline int n_planes_of(int per_env, int track, int payload = 0) {
  return (per_env ? PAR_PLANES : 0) + 1 + (track ? TRAJ_PLANES : 0) + (payload ? PAY_PLANES : 0);
}

// A launch covers the segments [seg_lo, seg_hi) of one thruster count, whose
// tiles are tile_lo .. tile_lo + n_tiles - 1.
struct StepArgs {
  const SegDesc* segs;
  int32_t seg_lo, seg_hi;
  int32_t tile_lo;
  int32_t n_tiles;
  const ClassF* classes;
  float* state;
  const float* actions;       // [n_steps][act_stride]
  int64_t act_stride;
  int32_t n_steps;
  int32_t act_mode;           // 0: load actions; 1: serving tick (Philox actions, tile map in tile_seg)
  const float4* planes;       // [N_PLANES][n_slots] (per-env) or target plane only
  int32_t per_env;            // 0: class constants; 1: physical parameters from planes 0..8; 2: as 1 plus the payload planes
  int32_t obs_every;          // 1: obs/reward every step; 0: after the last step
  int64_t n_slots;
  float* obs;                 // [*][n_slots][13] or null
  float* reward;              // [*][n_slots] or null
  float* ret;                 // serving: per-slot sum of rewards (or null)
  float* ckpt;                // record: [n_ckpt][21][n_slots] or null
  int32_t ckpt_every;
  int32_t track;              // 1: every segment of the launch is a tracking run
  uint32_t* status;           // bit 0: non-finite state
  int32_t pay_plane;          // payload runs: first payload plane
  int32_t wait_first;         // 1: launched as a programmatic dependent of unrelated work; wait before reading
  // Generic actuator tables (launches of generic-actuator classes), or, in a
  // serving tick (act_mode 1, propeller classes only), the segment (from
  // seg_lo) of each tile of the launch. One slot: the kernel's parameter
  // block stays 152 B (measured: 8 more bytes cost 0.8 us per 65k-env step).
  union {
    const ClassG* gen;
    const int32_t* tile_seg;
  };
};
static_assert(sizeof(StepArgs) == 152, "StepArgs layout");

// Adjoint scratch: per recomputed substep boundary and env one record of at
// most ADJ_REC floats (the state q, nu, n and, at step boundaries, p, in
// whole 16-byte vectors). Each class segment owns 2 (ckpt_every K + 1)
// ADJ_REC floats per slot, from its first slot on: two buffers of one
// checkpoint segment's records that alternate between the forward recompute
// and the reverse pass.
enum { ADJ_REC = 24 };
inline size_t adjoint_scratch_floats(int64_t ckpt_every, int64_t K, int64_t n_slots) {
  return (size_t)2 * (size_t)(ckpt_every * K + 1) * ADJ_REC * (size_t)n_slots;
}

struct AdjArgs {
  const SegDesc* segs;
  int32_t seg_lo, seg_hi;
  int32_t tile_lo;
  int32_t n_tiles;
  const ClassF* classes;
  const float4* planes;
  int64_t n_slots;
  const float* actions;
  int64_t act_stride;
  int32_t T;
  int32_t ckpt_every;
  const float* ckpt;          // [n_ckpt][21][n_slots]
  float* scratch;             // per class segment: 2 (ckpt_every K + 1) ADJ_REC floats per slot
  const float* g_obs;         // [T][n_slots][13] or null
  const float* g_rew;         // [T][n_slots] or null
  const float* g_state_T;     // [n_slots][21] or null
  float* g_actions;           // [T][act_stride] or null
  float* g_A;                 // [n_slots][6] or null
  float* g_D;                 // [n_slots][12] or null
  float* g_state0;            // [n_slots][21] or null
  int32_t tile_envs;          // envs per tile (the launch's blocks cover a tile in tile_envs / blockDim parts)
  int32_t pay_plane;          // payload runs: first payload plane; 0: no payload
  int32_t unit_steps;         // steps of one reverse unit (a checkpoint segment splits into units)
  int32_t pad1;
};

// Class nominal record for the reset kernel (FP64).
struct ClassNominal {
  double mass, Ig[3], rb[3], B, Ma[6], dl[6], dq[6];
};

struct ResetArgs {
  const SegDesc* segs;
  int32_t n_segs;
  int32_t n_sel;              // number of env ids (or total envs when ids is null)
  const int32_t* env_ids;     // global env ids or null = all
  const ClassNominal* nominal;
  int32_t per_env;
  int32_t serving;            // 1: draws keyed by (segment seed, env id within the segment)
  float* state;
  float4* planes;
  int64_t n_slots;
  uint64_t seed;
  int32_t dr, cur, cur3d, init_mode;
  double mass_lo, mass_hi, added_lo, added_hi, damp_lo, damp_hi, cob_lo, cob_hi, cur_lo, cur_hi;
  double target_half, pos_radius, max_angle;
  int32_t track, track_kind;
  int32_t payload, pad1;
  double payload_lo, payload_hi;
};

// Arguments of the FP64 finite-difference rollout.
struct Fp64Args {
  const SegDesc* segs;
  int32_t seg_lo, seg_hi;
  int32_t tile_lo;
  int32_t n_tiles;
  const ClassD* classes;
  const float* state;
  const float4* planes;
  int64_t n_slots;
  const float* actions;
  int64_t act_stride;
  int32_t T;
  int32_t pay_plane;          // payload runs: first payload plane; 0: no payload
  const double* dA;
  const double* ddl;
  const double* ddq;
  double eps;
  double dt;                  // control step in FP64 (tracking time)
  double h;                   // dt / K in FP64
  double* reward;
  double* state_out;
  const ClassGD* gen;         // generic actuator tables per class in FP64 (variants 1 and 2)
};

}  // namespace mg
