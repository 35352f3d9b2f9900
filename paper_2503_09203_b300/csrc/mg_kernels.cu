// CUDA kernels of libmarinegym for sm_103a (B300).
//
// Data layout in HBM (one GPU, all resident):
//   * state: per class segment, SoA planes over the segment's n4 slots: the
//     13 + n_thr fields (p3 q4 nu6 n[n_thr]) grouped as float4 planes plus up
//     to three scalar planes for the remainder, so one env-step moves exactly
//     4 (13 + n_thr) bytes each way with 512-byte coalesced warp accesses;
//   * parameters: 10 float4 planes over all slots (9 planes = 36 physical
//     floats, 1 plane = hover target); class-constant runs read only the
//     target plane and take the physics from the class table;
//   * actions: per class, row-major [n4][n_thr] (a policy's natural output);
//   * observations: [slot][13] row-major, written through a shared-memory
//     tile so that global stores are full 16-byte vectors.
// One thread advances one env through all K substeps (and all steps of a
// multi-step launch) with the state in registers; class constants live in
// shared memory and are read as warp-uniform broadcasts. Nothing here is a
// dense contraction, so there are no tensor-core paths.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "marinegym.h"
#include "mg_internal.h"
#include "mg_device.cuh"
#include "mg_payload.h"

namespace mg {

template <int NT>
struct Lay {
  static constexpr int SS = 13 + NT;
  static constexpr int NF4 = SS / 4;
  static constexpr int REM = SS % 4;
};

template <int NT>
__device__ __forceinline__ void fields_to_state(const float (&f)[13 + NT], St<float, NT>& x) {
#pragma unroll
  for (int i = 0; i < 3; ++i) x.p[i] = f[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] = f[3 + i];
#pragma unroll
  for (int i = 0; i < 6; ++i) x.nu[i] = f[7 + i];
#pragma unroll
  for (int i = 0; i < NT; ++i) x.n[i] = f[13 + i];
}

template <int NT>
__device__ __forceinline__ void state_to_fields(const St<float, NT>& x, float (&f)[13 + NT]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) f[i] = x.p[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) f[3 + i] = x.q[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) f[7 + i] = x.nu[i];
#pragma unroll
  for (int i = 0; i < NT; ++i) f[13 + i] = x.n[i];
}

template <int NT>
__device__ __forceinline__ void load_state(const float* base, int64_t n4, int64_t i, St<float, NT>& x) {
  float f[13 + NT];
  const float4* p4 = reinterpret_cast<const float4*>(base);
#pragma unroll
  for (int k = 0; k < Lay<NT>::NF4; ++k) {
    const float4 v = p4[k * n4 + i];
    f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
  }
  const float* pr = base + (int64_t)Lay<NT>::NF4 * 4 * n4;
#pragma unroll
  for (int r = 0; r < Lay<NT>::REM; ++r) f[Lay<NT>::NF4 * 4 + r] = pr[r * n4 + i];
  fields_to_state<NT>(f, x);
}

template <int NT>
__device__ __forceinline__ void store_state(float* base, int64_t n4, int64_t i, const St<float, NT>& x) {
  float f[13 + NT];
  state_to_fields<NT>(x, f);
  float4* p4 = reinterpret_cast<float4*>(base);
#pragma unroll
  for (int k = 0; k < Lay<NT>::NF4; ++k)
    p4[k * n4 + i] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
  float* pr = base + (int64_t)Lay<NT>::NF4 * 4 * n4;
#pragma unroll
  for (int r = 0; r < Lay<NT>::REM; ++r) pr[r * n4 + i] = f[Lay<NT>::NF4 * 4 + r];
}

__device__ __forceinline__ void load_phys(const float4* planes, int64_t n_slots, int64_t slot, Phys<float>& P) {
  float v[36];
#pragma unroll
  for (int k = 0; k < PAR_PLANES; ++k) {
    const float4 a = __ldg(&planes[k * n_slots + slot]);
    v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    P.minv[j] = v[PAR_MINV + j]; P.A[j] = v[PAR_A + j]; P.dl[j] = v[PAR_DL + j]; P.dq[j] = v[PAR_DQ + j];
  }
  P.m = v[PAR_M];
#pragma unroll
  for (int j = 0; j < 3; ++j) { P.Ig[j] = v[PAR_IG + j]; P.rb[j] = v[PAR_RB + j]; P.Vc[j] = v[PAR_VC + j]; }
  P.W = v[PAR_W]; P.B = v[PAR_B];
}

// Segment of a tile: binary search over tile_begin (segments sorted). The
// table may live in global or in shared memory, so the loads are generic.
__device__ __forceinline__ int find_seg(const SegDesc* segs, int n_segs, int tile) {
  int lo = 0, hi = n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float clamp1(float a) { return a < -1.0f ? -1.0f : (a > 1.0f ? 1.0f : a); }

// Serving action from one 64-bit Philox output: top 24 bits k -> k 2^-23 - 1,
// exact in FP32, on [-1, 1).
__device__ __forceinline__ float action_of_bits(uint64_t bits) {
  return (float)(int)(bits >> 40) * (1.0f / 8388608.0f) - 1.0f;
}

template <int NT>
__device__ __forceinline__ void load_actions(const float* base, float (&a)[NT]) {
  if constexpr (NT % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NT / 4; ++k) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(base) + k);
      a[4 * k] = v.x; a[4 * k + 1] = v.y; a[4 * k + 2] = v.z; a[4 * k + 3] = v.w;
    }
  } else if constexpr (NT % 2 == 0) {
#pragma unroll
    for (int k = 0; k < NT / 2; ++k) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(base) + k);
      a[2 * k] = v.x; a[2 * k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NT; ++k) a[k] = __ldg(base + k);
  }
}

// ---------------------------------------------------------------------------
// Shared-memory views read at the point of use. Class constants and per-env
// parameters stay in shared memory (vector loads for the actuator table)
// instead of occupying registers across the substep loop. The loads are plain
// (non-volatile) inline PTX, free to be scheduled within a substep; the step
// loop passes them a base address made opaque once per substep, so that they
// are neither hoisted out of the loop nor moved above the barrier that
// follows a table rewrite.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float lds1(unsigned a) {
  float v;
  asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds4(unsigned a) {
  float4 v;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}

// Actuator table in shared memory: alloc[6][8] | kf[8] | dz[8] | alpha[8].
// dz_on = 0: the class has no dead zone (the thrust skips the test).
#ifndef MG_DZ_FLAG
#define MG_DZ_FLAG 1
#endif
// DZF: the kernel carries a dead-zone-free thrust path (class-constant
// propellers only: in the other variants the second path costs registers).
template <bool DZF>
struct ActSmemT {
  unsigned base;
  unsigned dz_on;
};
template <bool DZF>
__device__ __forceinline__ bool dz_active(const ActSmemT<DZF>& A) { return !(MG_DZ_FLAG && DZF) || A.dz_on != 0u; }
// Class constants as a kernel parameter: the dead-zone test is skipped for
// classes without one.
__device__ __forceinline__ bool dz_active(const ClassK& k) { return !MG_DZ_FLAG || k.dz_on != 0u; }
enum { SA_ALLOC = 0, SA_KF = 48, SA_DZ = 56, SA_ALPHA = 64, SA_DIM = 72 };

template <int NT>
__device__ __forceinline__ void lds_vec(unsigned a, float (&r)[NT]) {
#pragma unroll
  for (int q = 0; q < (NT + 3) / 4; ++q) {
    const float4 v = lds4(a + 16 * q);
    if (4 * q + 0 < NT) r[(4 * q + 0) % NT] = v.x;
    if (4 * q + 1 < NT) r[(4 * q + 1) % NT] = v.y;
    if (4 * q + 2 < NT) r[(4 * q + 2) % NT] = v.z;
    if (4 * q + 3 < NT) r[(4 * q + 3) % NT] = v.w;
  }
}
template <typename S, int NT, bool DZF>
__device__ __forceinline__ void act_row(const ActSmemT<DZF>& A, int k, S (&r)[NT]) {
  lds_vec<NT>(A.base + 4 * (SA_ALLOC + 8 * k), r);
}
template <typename S, int NT, bool DZF>
__device__ __forceinline__ void act_rotor(const ActSmemT<DZF>& A, S (&kf)[NT], S (&dz)[NT], S (&al)[NT]) {
  lds_vec<NT>(A.base + 4 * SA_KF, kf);
  lds_vec<NT>(A.base + 4 * SA_DZ, dz);
  lds_vec<NT>(A.base + 4 * SA_ALPHA, al);
}
template <typename S, int NT, bool DZF>
__device__ __forceinline__ void act_rotor_nodz(const ActSmemT<DZF>& A, S (&kf)[NT], S (&al)[NT]) {
  lds_vec<NT>(A.base + 4 * SA_KF, kf);
  lds_vec<NT>(A.base + 4 * SA_ALPHA, al);
}

// Physical parameters in shared memory, field f at base + 4 * f * STRIDE
// (STRIDE = 1: class block read as a broadcast; STRIDE = tile width: per-env
// columns, one per thread, bank-conflict free).
template <int OFF, int STRIDE>
struct SArr {
  unsigned base;
  __device__ __forceinline__ float operator[](int j) const { return lds1(base + 4u * (unsigned)((OFF + j) * STRIDE)); }
};
template <int OFF, int STRIDE>
struct SScl {
  unsigned base;
  __device__ __forceinline__ operator float() const { return lds1(base + 4u * (unsigned)(OFF * STRIDE)); }
};
template <int STRIDE>
struct PhysSmem {
  static constexpr bool kFull = false;
  SArr<PAR_MINV, STRIDE> minv;
  SArr<PAR_A, STRIDE> A;
  SArr<PAR_DL, STRIDE> dl;
  SArr<PAR_DQ, STRIDE> dq;
  SScl<PAR_M, STRIDE> m;
  SArr<PAR_IG, STRIDE> Ig;
  SScl<PAR_W, STRIDE> W;
  SScl<PAR_B, STRIDE> B;
  SArr<PAR_RB, STRIDE> rb;
  SArr<PAR_VC, STRIDE> Vc;
  __device__ __forceinline__ explicit PhysSmem(unsigned b)
      : minv{b}, A{b}, dl{b}, dq{b}, m{b}, Ig{b}, W{b}, B{b}, rb{b}, Vc{b} {}
};

// Payload runs: per-env columns staged from physics planes 1-5, 7, 8 (columns
// 0-27) and payload planes 0-7 (columns 28-59). The diagonal inverse, the
// vehicle's own mass and inertia and its weight are not needed: the combined
// body's full inverse, inertia about the origin, first moment, mass and
// weight replace them.
enum { PF_A = 2, PF_DL = 8, PF_DQ = 14, PF_B = 21, PF_RB = 22, PF_VC = 25, PF_PAY = 28, PF_DIM = 60 };
constexpr int PF_STD_PLANES = 7;                       // physics planes staged
constexpr int PF_PAY_PLANES = 8;                       // payload planes staged
__device__ __forceinline__ int pf_std_plane(int k) { return k < 5 ? k + 1 : k + 2; }   // 1..5, 7, 8
template <int STRIDE>
struct PhysSmemFull {
  static constexpr bool kFull = true;
  SArr<PF_A, STRIDE> A;
  SArr<PF_DL, STRIDE> dl;
  SArr<PF_DQ, STRIDE> dq;
  SScl<PF_B, STRIDE> B;
  SArr<PF_RB, STRIDE> rb;
  SArr<PF_VC, STRIDE> Vc;
  SArr<PF_PAY + PAY_MINV, STRIDE> Mi;
  SArr<PF_PAY + PAY_IO, STRIDE> Io;
  SArr<PF_PAY + PAY_S, STRIDE> s;
  SScl<PF_PAY + PAY_M, STRIDE> m;
  SScl<PF_PAY + PAY_W, STRIDE> W;
  __device__ __forceinline__ explicit PhysSmemFull(unsigned b)
      : A{b}, dl{b}, dq{b}, B{b}, rb{b}, Vc{b}, Mi{b}, Io{b}, s{b}, m{b}, W{b} {}
};
static_assert(PF_STD_PLANES * 4 == PF_PAY && PF_PAY + PF_PAY_PLANES * 4 == PF_DIM, "payload column map");
static_assert(PAY_W < PF_PAY_PLANES * 4, "staged payload planes hold the step's fields");

// Generic actuator table in shared memory: 8 kinds (float bits), then
// GEN_VALS values per channel (a copy of the class's ClassG).
constexpr int GEN_FLOATS = 8 + 8 * GEN_VALS;
static_assert(sizeof(ClassG) == GEN_FLOATS * sizeof(float), "generic table layout");
static_assert(KIND_PROP == MG_ACT_PROP && KIND_SERVO == MG_ACT_SERVO && KIND_FIN == MG_ACT_FIN &&
                  KIND_TILT == MG_ACT_TILT, "actuator kinds");
struct GenSmem {
  unsigned base;
  __device__ __forceinline__ int kind(int i) const { return __float_as_int(lds1(base + 4u * (unsigned)i)); }
  __device__ __forceinline__ float v(int i, int k) const {
    return lds1(base + 4u * (unsigned)(8 + i * GEN_VALS + k));
  }
};

constexpr int STEP_BLK = 128;
#ifndef MG_STEP_MIN_BLOCKS
#define MG_STEP_MIN_BLOCKS 4
#endif


// ---------------------------------------------------------------------------
// Bulk-copy (1-D TMA) and mbarrier helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Global -> shared bulk copy completing on `bar` (addresses 16-byte aligned,
// size a multiple of 16).
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Shared -> global bulk copy in the current bulk group.
__device__ __forceinline__ void bulk_store(void* dst, unsigned src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait on an mbarrier phase: gives up after `limit_ns` and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

// Per-warp stage buffer: the warp's 32 envs of one tile. State planes (NF4
// float4 planes, then REM float planes, 32 entries each), actions [32][NT],
// target [32] float4. Each warp of a block owns two stage buffers and one
// observation buffer [32][13] and runs its own copy pipeline.
#ifndef MG_OBS_ALIAS
#define MG_OBS_ALIAS 0
#endif
constexpr int WENV = 32;
constexpr int N_WARPS = STEP_BLK / WENV;
template <int NT>
struct Stage {
  static constexpr int SS = 13 + NT, NF4 = SS / 4, REM = SS % 4;
  static constexpr int ACT_OFF = WENV * SS;                     // floats
  static constexpr int TGT_OFF = ACT_OFF + WENV * NT;           // floats (16-byte aligned)
  static constexpr int TRJ_OFF = TGT_OFF + 4 * WENV;            // 3 trajectory planes (tracking runs only)
  static constexpr int OBS = WENV * 13;
  // Stage buffer and per-warp sizes (floats); smaller shared memory pays off,
  // so the trajectory section exists only in tracking runs.
  static __host__ __device__ constexpr int floats(bool track) { return TRJ_OFF + (track ? 12 * WENV : 0); }
#if MG_OBS_ALIAS
  // The observation tile reuses the tile's own stage buffer once its inputs
  // are in registers (rows 0..12 per env lie below the trajectory section).
  static __host__ __device__ constexpr int warp_floats(bool track) { return 2 * floats(track); }
  static_assert(OBS <= TRJ_OFF, "observation tile must fit below the trajectory section");
#else
  static __host__ __device__ constexpr int warp_floats(bool track) { return 2 * floats(track) + OBS; }
#endif
  static_assert((ACT_OFF % 4) == 0 && (TGT_OFF % 4) == 0 && (TRJ_OFF % 4) == 0 && (OBS % 4) == 0,
                "16-byte aligned sections");
};
constexpr int SEG_CACHE = 16;   // segments of a launch kept in shared memory

// Class tables of segment `sd` into act (SA_DIM) and phys (PAR_DIM), and its
// generic actuator table into gen (generic variants), by the block's threads.
template <int VAR>
__device__ __forceinline__ void stage_tables(const StepArgs& a, const SegDesc& sd, float* act, float* phys,
                                             float* gen, int tid) {
  const ClassF& cf = a.classes[sd.cls];
  for (int k = tid; k < SA_DIM + PAR_DIM; k += STEP_BLK) {
    if (k < 48) act[k] = cf.alloc[k / 8][k % 8];
    else if (k < 56) act[k] = cf.kf[k - 48];
    else if (k < 64) act[k] = cf.dz[k - 56];
    else if (k < 72) act[k] = sd.alpha[k - 64];
    else phys[k - 72] = cf.phys[k - 72];
  }
  if (VAR) {
    const float* g = reinterpret_cast<const float*>(a.gen + sd.cls);
    for (int k = tid; k < GEN_FLOATS; k += STEP_BLK) gen[k] = g[k];
  }
}

// Issue the bulk copies of one warp's slice of a tile (lane 0 only). `nvw`
// (a multiple of 4, > 0) envs start at local env index w0 of the segment.
template <int NT, int PM>
__device__ __forceinline__ void issue_warp_loads(const StepArgs& a, const SegDesc& sd, int64_t w0, unsigned nvw,
                                                 float* buf, unsigned bar) {
  constexpr bool PER_ENV = PM == 1 || PM == 2;
  using SG = Stage<NT>;
  const float* st = a.state + sd.st_off;
  unsigned bytes = SG::NF4 * nvw * 16 + SG::REM * nvw * 4 + nvw * 16;
  const bool load_act = a.n_steps > 0 && a.act_mode == 0;
  if (load_act) bytes += nvw * NT * 4;
  const bool trj = a.track != 0;   // the launch's layout has the trajectory section
  if (trj) bytes += 3 * nvw * 16;
  mbar_expect_tx(bar, bytes);
  const unsigned b = smem_addr(buf);
#pragma unroll
  for (int k = 0; k < SG::NF4; ++k) bulk_load(b + 16u * k * WENV, st + ((int64_t)k * sd.n4 + w0) * 4, nvw * 16, bar);
#pragma unroll
  for (int r = 0; r < SG::REM; ++r)
    bulk_load(b + 16u * SG::NF4 * WENV + 4u * r * WENV, st + (int64_t)SG::NF4 * 4 * sd.n4 + (int64_t)r * sd.n4 + w0,
              nvw * 4, bar);
  if (load_act) bulk_load(b + 4u * SG::ACT_OFF, a.actions + sd.act_off + w0 * NT, nvw * NT * 4, bar);
  bulk_load(b + 4u * SG::TGT_OFF, a.planes + tgt_plane(PER_ENV) * a.n_slots + sd.slot_off + w0, nvw * 16, bar);
  if (trj) {
#pragma unroll
    for (int q = 0; q < TRAJ_PLANES; ++q)
      bulk_load(b + 4u * (SG::TRJ_OFF + 4 * q * WENV),
                a.planes + (int64_t)(tgt_plane(PER_ENV) + 1 + q) * a.n_slots + sd.slot_off + w0, nvw * 16, bar);
  }
}

// Envs of warp `warp` in a tile that starts at local env local0 (0 if none).
__device__ __forceinline__ unsigned warp_envs(const SegDesc& sd, int64_t local0, int warp) {
  const int64_t n = (int64_t)sd.n4 - local0 - (int64_t)warp * WENV;
  return n <= 0 ? 0u : (unsigned)min((int64_t)WENV, n);
}

template <int NT, int PM, int VAR>
__device__ __forceinline__ bool step_tile(const StepArgs& a, const ClassK* kc, const SegDesc& sd, int tile,
                                          unsigned s_act, unsigned s_phys, unsigned s_gen, const float* buf,
                                          float* obs_w, float* s_par, int& n_emit) {
  constexpr bool PER_ENV = PM == 1 || PM == 2;
  using SG = Stage<NT>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t local0 = (int64_t)(tile - sd.tile_begin) * STEP_BLK;
  const int64_t w0 = local0 + warp * WENV;
  const int64_t i = w0 + lane;
  const bool valid = i < sd.n_envs;
  const bool in_storage = i < sd.n4;
  const unsigned nvw = warp_envs(sd, local0, warp);
  const int64_t slot = sd.slot_off + i;
  float* st_base = a.state + sd.st_off;
  using ActSmem = ActSmemT<PM == 0 && VAR == 0>;
  const ActSmem A{s_act, (unsigned)(sd.flags & 1)};

  // Per-env parameters: plain per-env runs prefetch their 9 planes into
  // registers here (their loads overlap the stage reads below); payload runs
  // copy 15 planes straight to shared memory afterwards.
  constexpr bool STAGE_PAR = PM == 1;
  float4 pv[STAGE_PAR ? PAR_PLANES : 1];
  if (STAGE_PAR && valid) {
#pragma unroll
    for (int k = 0; k < PAR_PLANES; ++k) pv[k % (STAGE_PAR ? PAR_PLANES : 1)] = __ldg(&a.planes[k * a.n_slots + slot]);
  }
  St<float, NT> x;
  float c[NT];
  float tgt[3] = {0.0f, 0.0f, 0.0f};
  float4 tg = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
  for (int j = 0; j < NT; ++j) c[j] = 0.0f;
  bool have_act0 = false;
  if (valid) {
    float f[13 + NT];
    const float4* p4 = reinterpret_cast<const float4*>(buf);
#pragma unroll
    for (int k = 0; k < SG::NF4; ++k) {
      const float4 v = p4[k * WENV + lane];
      f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int r = 0; r < SG::REM; ++r) f[(SG::NF4 * 4 + r) % (13 + NT)] = buf[SG::NF4 * 4 * WENV + r * WENV + lane];
    fields_to_state<NT>(f, x);
    tg = reinterpret_cast<const float4*>(buf + SG::TGT_OFF)[lane];
    tgt[0] = tg.x; tgt[1] = tg.y; tgt[2] = tg.z;
    if (a.n_steps > 0 && a.act_mode == 0) {
#pragma unroll
      for (int j = 0; j < NT; ++j) c[j] = clamp1(buf[SG::ACT_OFF + lane * NT + j]);
      have_act0 = true;
    }
  }
  if (STAGE_PAR && valid) {
#pragma unroll
    for (int k = 0; k < PAR_PLANES; ++k) {
      const float4 v = pv[k % (STAGE_PAR ? PAR_PLANES : 1)];
      s_par[(4 * k + 0) * STEP_BLK + tid] = v.x;
      s_par[(4 * k + 1) * STEP_BLK + tid] = v.y;
      s_par[(4 * k + 2) * STEP_BLK + tid] = v.z;
      s_par[(4 * k + 3) * STEP_BLK + tid] = v.w;
    }
  }
  if (PM == 2 && valid) {
#pragma unroll
    for (int k = 0; k < PF_STD_PLANES + PF_PAY_PLANES; ++k) {
      const int plane = k < PF_STD_PLANES ? pf_std_plane(k) : a.pay_plane + (k - PF_STD_PLANES);
      const float4 v = __ldg(&a.planes[(int64_t)plane * a.n_slots + slot]);
      s_par[(4 * k + 0) * STEP_BLK + tid] = v.x;
      s_par[(4 * k + 1) * STEP_BLK + tid] = v.y;
      s_par[(4 * k + 2) * STEP_BLK + tid] = v.z;
      s_par[(4 * k + 3) * STEP_BLK + tid] = v.w;
    }
  }
  // Each thread reads only its own parameter column: no barrier needed.
  using PV = std::conditional_t<PM == 2, PhysSmemFull<STEP_BLK>, PhysSmem<PER_ENV ? STEP_BLK : 1>>;
  const unsigned p_base = PER_ENV ? smem_addr(s_par) + 4u * tid : s_phys;
  const unsigned g_base = s_gen;
  const int n_out_steps = a.n_steps == 0 ? 1 : a.n_steps;
  for (int t = 0; t < n_out_steps; ++t) {
    if (valid && a.n_steps > 0) {
      if (a.act_mode == 0) {
        if (!(t == 0 && have_act0)) {
          float raw[NT];
          load_actions<NT>(a.actions + t * a.act_stride + sd.act_off + i * NT, raw);
#pragma unroll
          for (int j = 0; j < NT; ++j) c[j] = clamp1(raw[j]);
        }
      } else {
#pragma unroll
        for (int g = 0; g < (NT + 3) / 4; ++g) {
          uint64_t o[4];
          philox4x64((uint64_t)i, (uint64_t)(sd.step0 + t), (uint64_t)g, 0, sd.seed, STREAM_ACTION, o);
#pragma unroll
          for (int l = 0; l < 4; ++l)
            if (4 * g + l < NT) c[(4 * g + l) % NT] = clamp1(action_of_bits(o[l]));
        }
      }
      if (a.ckpt && (t % a.ckpt_every) == 0) {
        float f[13 + NT];
        state_to_fields<NT>(x, f);
        float* ck = a.ckpt + (int64_t)(t / a.ckpt_every) * 21 * a.n_slots + slot;
#pragma unroll
        for (int j = 0; j < 21; ++j) ck[j * a.n_slots] = (j < 13 + NT) ? f[j % (13 + NT)] : 0.0f;
      }
      // Shared-memory bases made opaque once per substep: loads may be
      // scheduled freely inside a substep but not hoisted out of the loop.
      for (int k = 0; k < sd.K; ++k) {
        if constexpr (PM == 3) {
          // Class constants are kernel parameters: read as operands.
          substep<float, NT, false, ClassK, ClassK, false>(x, c, *kc, *kc, sd.h, nullptr);
        } else {
          unsigned pb = p_base, ab = A.base, gb = g_base;
          asm volatile("" : "+r"(pb), "+r"(ab), "+r"(gb));
          const ActSmem Ak{ab, A.dz_on};
          // Class-constant physics carries no current (zero by construction).
          const PV Pk(pb);
          if constexpr (VAR == 0) {
            substep<float, NT, false, ActSmem, PV, PER_ENV>(x, c, Pk, Ak, sd.h, nullptr);
          } else if constexpr (VAR == 1) {
            substep<float, NT, false, ActSmem, PV, PER_ENV, GenSmem>(x, c, Pk, Ak, sd.h, nullptr, GenSmem{gb});
          } else {
            substep_rk4<float, NT, ActSmem, PV, PER_ENV, GenSmem>(x, c, Pk, Ak, sd.h, GenSmem{gb});
          }
        }
      }
    }
    const bool emit = a.obs_every || t == n_out_steps - 1;
    if (emit) {
      const int64_t out = a.obs_every ? t : 0;
      float o[13], r = 0.0f;
#pragma unroll
      for (int j = 0; j < 13; ++j) o[j] = 0.0f;
      if (valid) {
        if (a.track) {
          // Tracking reference at the end of this step (counter k0 + t + 1);
          // its parameters were staged with the tile.
          const float4* tp = reinterpret_cast<const float4*>(buf + SG::TRJ_OFF) + lane;
          const float kk = tg.w + (a.n_steps > 0 ? (float)(t + 1) : 0.0f);
          track_ref<float>(tg, tp[0], tp[WENV], tp[2 * WENV], sd.dt, kk, tgt);
        }
        observe<float, NT>(x, c, tgt, o, r);
      }
      if (a.obs && nvw > 0) {
        // The warp's previous observation store must have read its buffer.
        if (lane == 0 && n_emit > 0) bulk_wait_read0();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 13; ++j) obs_w[lane * 13 + j] = o[j];
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          bulk_store(a.obs + (out * a.n_slots + sd.slot_off + w0) * 13, smem_addr(obs_w), nvw * 52u);
          bulk_commit();
        }
        ++n_emit;
      }
      if (a.reward && in_storage) a.reward[out * a.n_slots + slot] = valid ? r : 0.0f;
      if (a.ret && valid && a.n_steps > 0) a.ret[slot] += r;
    }
  }
  if (valid && a.n_steps > 0) {
    store_state<NT>(st_base, sd.n4, i, x);
    if (a.track) {
      // Advance the env's step counter (w lane of its target plane entry).
      float* kp = reinterpret_cast<float*>(const_cast<float4*>(a.planes) + (int64_t)tgt_plane(PER_ENV) * a.n_slots + slot);
      kp[3] = tg.w + (float)a.n_steps;
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) s += x.p[j];
#pragma unroll
    for (int j = 0; j < 4; ++j) s += x.q[j];
#pragma unroll
    for (int j = 0; j < 6; ++j) s += x.nu[j];
#pragma unroll
    for (int j = 0; j < NT; ++j) s += x.n[j];
    if (!isfinite(s)) atomicOr(a.status, 1u);
  }
  return true;
}

// Persistent step kernel for envs with NT thrusters. Block b walks the tiles
// tile_lo + b, + gridDim.x, ...; a tile is 128 envs of one segment, 32 per
// warp. Every warp runs its own pipeline: while it computes its slice of tile
// j, its lane 0 has already issued the bulk copies of its slice of the next
// tile into the warp's other stage buffer, and observation rows leave through
// a per-warp bulk store. Warps never wait on one another except when the
// class constants change. Every wait is bounded (2 s); a warp that gives up
// sets bit 1 of the status word and skips the rest of its tiles (it keeps
// walking them, so every block barrier is still reached).
// The RK4 variant keeps the stage point, the running sum and the substep's
// start state live at once. It is compiled for 3 resident blocks per SM (168
// registers): measured at 1M envs, K=4, that beats both 4 blocks (heavy
// spills) and 2 blocks (too few warps to hide latency), although the tracking
// and per-env kernels still spill a few hundred bytes. The generic-actuator
// variant (fins, servo tilt) is also compiled for 3 blocks per SM: its extra
// live state otherwise costs 3% at K=4 and 8% at K=1.
#ifndef MG_RK4_MIN_BLOCKS
#define MG_RK4_MIN_BLOCKS 3
#endif
#ifndef MG_GEN_MIN_BLOCKS
#define MG_GEN_MIN_BLOCKS 3
#endif
#ifndef MG_KSTEP_MIN_BLOCKS
#define MG_KSTEP_MIN_BLOCKS MG_STEP_MIN_BLOCKS
#endif
template <int PM, int VAR>
struct StepMinBlocks {
  static constexpr int value = VAR == 2 ? MG_RK4_MIN_BLOCKS
                               : VAR == 1 ? MG_GEN_MIN_BLOCKS
                               : PM == 3  ? MG_KSTEP_MIN_BLOCKS
                                          : MG_STEP_MIN_BLOCKS;
};

// Second kernel parameter: the class constants (PM 3), else nothing.
struct NoClassK {};
template <int PM>
using KParam = std::conditional_t<PM == 3, ClassK, NoClassK>;

// PM: parameter source (0 class constants staged in shared memory, 1 per-env
// planes, 2 per-env planes with the payload, 3 class constants passed as the
// kernel parameter `kp`: one class per launch). The body stays in the kernel
// itself: moved into a function taking the parameters by reference, the
// per-env and payload instantiations spilled.
template <int NT, int PM, int VAR>
__global__ void __launch_bounds__(STEP_BLK, (StepMinBlocks<PM, VAR>::value))
    mg_step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ KParam<PM> kp) {
  using SG = Stage<NT>;
  const ClassK* kc = nullptr;
  if constexpr (PM == 3) kc = &kp;
  extern __shared__ __align__(16) float s_dyn[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int fl = SG::floats(a.track != 0), wfl = SG::warp_floats(a.track != 0);
  float* const w_base = s_dyn + warp * wfl;
  float* const buf0 = w_base;
  float* const buf1 = w_base + fl;
  float* const obs_sep = w_base + 2 * fl;   // separate observation tile (unless aliased)
  float* const s_par = s_dyn + N_WARPS * wfl;
  __shared__ __align__(16) float s_act[SA_DIM];
  __shared__ __align__(16) float s_phys[PAR_DIM];
  __shared__ __align__(16) float s_gen[VAR ? GEN_FLOATS : 4];
  __shared__ __align__(8) uint64_t s_bar[N_WARPS][2];
  __shared__ SegDesc s_seg[SEG_CACHE];
  // The next launch of a step (another thruster count, disjoint envs) may
  // start filling SMs as soon as this grid's blocks are resident.
  // The first launch of a step may become resident while the previous step
  // (same envs) finishes: it waits for that work to complete before it reads
  // anything or lets its own dependents start, so that every later launch of
  // the step also follows the whole previous step.
  if (a.wait_first) asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if ((int)blockIdx.x >= a.n_tiles) return;
  const int n_seg = a.seg_hi - a.seg_lo;
  const bool cached = n_seg <= SEG_CACHE;
  if (cached) {
    const int32_t* src = reinterpret_cast<const int32_t*>(a.segs + a.seg_lo);
    int32_t* dst = reinterpret_cast<int32_t*>(s_seg);
    for (int k = tid; k < n_seg * (int)(sizeof(SegDesc) / 4); k += STEP_BLK) dst[k] = src[k];
  }
  const SegDesc* segs = cached ? s_seg : a.segs + a.seg_lo;
  const unsigned full0 = smem_addr(&s_bar[warp][0]), full1 = smem_addr(&s_bar[warp][1]);
  if (lane == 0) {
    mbar_init(full0, 1);
    mbar_init(full1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Prologue: this warp's slice of the first tile.
  unsigned nvw_cur = 0;
  {
    const int tile0 = a.tile_lo + blockIdx.x;
    const SegDesc& s0 = segs[find_seg(segs, n_seg, tile0)];
    const int64_t local0 = (int64_t)(tile0 - s0.tile_begin) * STEP_BLK;
    nvw_cur = warp_envs(s0, local0, warp);
    if (lane == 0 && nvw_cur > 0 && !(s0.flags & 2))
      issue_warp_loads<NT, PM>(a, s0, local0 + warp * WENV, nvw_cur, buf0, full0);
  }
  int prev_seg = -1, n_emit = 0;
  unsigned use[2] = {0u, 0u};   // completed uses of each stage barrier
  bool failed = false;
  for (int j = 0, tt = blockIdx.x; tt < a.n_tiles; ++j, tt += gridDim.x) {
    const int tile = a.tile_lo + tt;
    const int b = j & 1;
    const int si = find_seg(segs, n_seg, tile);
    // Refill the other buffer (read during tile j - 1) with the next slice.
    const int tt_next = tt + gridDim.x;
    unsigned nvw_next = 0;
    if (tt_next < a.n_tiles) {
      const int tile_n = a.tile_lo + tt_next;
      const SegDesc& sn = segs[find_seg(segs, n_seg, tile_n)];
      const int64_t ln = (int64_t)(tile_n - sn.tile_begin) * STEP_BLK;
      nvw_next = warp_envs(sn, ln, warp);
      if (lane == 0 && nvw_next > 0 && !failed && !(sn.flags & 2)) {
#if MG_OBS_ALIAS
        // The buffer may still be the source of the previous tile's observation store.
        bulk_wait_read0();
#endif
        fence_async_smem();
        issue_warp_loads<NT, PM>(a, sn, ln + warp * WENV, nvw_next, b ? buf0 : buf1, b ? full0 : full1);
      }
    }
    const SegDesc& sd = segs[si];
    if (PM != 3 && si != prev_seg) {
      // Class constants change: rewrite them between two block barriers
      // (every warp of the block walks the same tiles).
      __syncthreads();
      stage_tables<VAR>(a, sd, s_act, s_phys, s_gen, tid);
      __syncthreads();
      prev_seg = si;
    }
    // A warp whose wait ran out stops computing and copying but stays in the
    // loop, so that it still reaches every block barrier of the launch.
    if (nvw_cur > 0 && !failed) {
      if (mbar_wait_bounded(b ? full1 : full0, use[b] & 1u, sd.wait_limit_ns ? sd.wait_limit_ns : kWaitLimitNs))
        use[b]++;
      else
        failed = true;
    }
    if (!failed)
      step_tile<NT, PM, VAR>(a, kc, sd, tile, smem_addr(s_act), smem_addr(s_phys), smem_addr(s_gen),
                             b ? buf1 : buf0, MG_OBS_ALIAS ? (b ? buf1 : buf0) : obs_sep, s_par, n_emit);
    // The warp has read its stage buffer b; lane 0 may refill it next round.
    __syncwarp();
    nvw_cur = nvw_next;
  }
  if (failed && lane == 0) atomicOr(a.status, 2u);
  // Observation stores must finish reading shared memory before the warp exits.
  if (lane == 0) bulk_wait0();
  // A grid launched as a programmatic dependent completes only after the grid
  // it depends on, so that completion stays ordered along the stream.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Reset: domain randomisation draws and initial state (FP64 arithmetic).
// ---------------------------------------------------------------------------
__global__ void mg_reset_kernel(const __grid_constant__ ResetArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_sel) return;
  const int64_t env = a.env_ids ? (int64_t)a.env_ids[k] : (int64_t)k;
  int si = -1;
  for (int s = 0; s < a.n_segs; ++s)
    if (env >= a.segs[s].env_base && env < a.segs[s].env_base + a.segs[s].n_envs) si = s;
  if (si < 0) return;
  const SegDesc& sd = a.segs[si];
  const ClassNominal& cn = a.nominal[sd.cls];
  const int64_t i = env - sd.env_base;
  const int64_t slot = sd.slot_off + i;
  const uint64_t id = a.serving ? (uint64_t)i : (uint64_t)env;
  const uint64_t seed = a.serving ? sd.seed : a.seed;
  auto fac = [&](int j, double lo, double hi) {
    return a.dr ? lo + (hi - lo) * uniform53(seed, STREAM_DR, id, j) : 1.0;
  };
  const double fm = fac(0, a.mass_lo, a.mass_hi);
  const double m = cn.mass * fm;
  double Ig[3], Ma[6], dl[6], dq[6], rb[3], Vc[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < 3; ++j) Ig[j] = cn.Ig[j] * fm;
  for (int j = 0; j < 6; ++j) {
    Ma[j] = cn.Ma[j] * fac(1 + j, a.added_lo, a.added_hi);
    dl[j] = cn.dl[j] * fac(7 + j, a.damp_lo, a.damp_hi);
    dq[j] = cn.dq[j] * fac(13 + j, a.damp_lo, a.damp_hi);
  }
  const double fb = fac(19, a.cob_lo, a.cob_hi);
  for (int j = 0; j < 3; ++j) rb[j] = cn.rb[j] * fb;
  if (a.cur) {
    const double sp = a.cur_lo + (a.cur_hi - a.cur_lo) * uniform53(seed, STREAM_DR, id, 20);
    const double psi = 6.283185307179586 * uniform53(seed, STREAM_DR, id, 21);
    if (a.cur3d) {
      const double zc = 2.0 * uniform53(seed, STREAM_DR, id, 22) - 1.0;
      const double rh = sqrt(1.0 - zc * zc);
      Vc[0] = sp * rh * cos(psi); Vc[1] = sp * rh * sin(psi); Vc[2] = sp * zc;
    } else {
      Vc[0] = sp * cos(psi); Vc[1] = sp * sin(psi);
    }
  }
  const double W = m * 9.81;
  double f[21];
  for (int j = 0; j < 21; ++j) f[j] = 0.0;
  f[3] = 1.0;
  double tgt[3] = {0.0, 0.0, 0.0};
  // Tracking reference (stream 2, draws 9..): a, w, phi, v of
  // p*(t) = c + a o sin(w t + phi) + v t.
  double ta[3] = {0.0, 0.0, 0.0}, tw[3] = {0.0, 0.0, 0.0}, tph[3] = {0.0, 0.0, 0.0}, tv[3] = {0.0, 0.0, 0.0};
  if (a.init_mode == 1 || a.track)
    for (int j = 0; j < 3; ++j) tgt[j] = a.target_half * (2.0 * uniform53(seed, STREAM_INIT, id, j) - 1.0);
  if (a.track) {
    const double two_pi = 6.283185307179586;
    if (a.track_kind == 0) {
      const double R = 1.0 + 2.0 * uniform53(seed, STREAM_INIT, id, 9);
      const double W = 0.2 + 0.4 * uniform53(seed, STREAM_INIT, id, 10);
      const double psi = two_pi * uniform53(seed, STREAM_INIT, id, 11);
      const double vz = -0.2 + 0.4 * uniform53(seed, STREAM_INIT, id, 12);
      ta[0] = R; ta[1] = R;
      tw[0] = W; tw[1] = W;
      tph[0] = psi + 0.5 * 3.141592653589793; tph[1] = psi;
      tv[2] = vz;
    } else {
      for (int j = 0; j < 3; ++j) {
        ta[j] = 1.0 + 2.0 * uniform53(seed, STREAM_INIT, id, 9 + j);
        tw[j] = 0.2 + 0.4 * uniform53(seed, STREAM_INIT, id, 12 + j);
        tph[j] = two_pi * uniform53(seed, STREAM_INIT, id, 15 + j);
      }
    }
  }
  if (a.init_mode == 1) {
    // Initial pose around the reference at t = 0.
    double p0[3];
    for (int j = 0; j < 3; ++j) p0[j] = tgt[j] + ta[j] * sin(tph[j]);
    const double rad = a.pos_radius * cbrt(uniform53(seed, STREAM_INIT, id, 3));
    const double zd = 2.0 * uniform53(seed, STREAM_INIT, id, 4) - 1.0;
    const double ph = 6.283185307179586 * uniform53(seed, STREAM_INIT, id, 5);
    const double rd = sqrt(1.0 - zd * zd);
    f[0] = p0[0] + rad * rd * cos(ph);
    f[1] = p0[1] + rad * rd * sin(ph);
    f[2] = p0[2] + rad * zd;
    const double za = 2.0 * uniform53(seed, STREAM_INIT, id, 6) - 1.0;
    const double pa = 6.283185307179586 * uniform53(seed, STREAM_INIT, id, 7);
    const double ra = sqrt(1.0 - za * za);
    const double ang = a.max_angle * uniform53(seed, STREAM_INIT, id, 8);
    const double sh = sin(0.5 * ang);
    f[3] = cos(0.5 * ang);
    f[4] = sh * ra * cos(pa);
    f[5] = sh * ra * sin(pa);
    f[6] = sh * za;
  }
  // State planes.
  const int NT = sd.n_thr;
  const int SS = 13 + NT, NF4 = SS / 4;
  float* base = a.state + sd.st_off;
  for (int j = 0; j < SS; ++j) {
    const int64_t off = (j < NF4 * 4) ? ((int64_t)(j / 4) * sd.n4 + i) * 4 + (j % 4)
                                      : (int64_t)NF4 * 4 * sd.n4 + (int64_t)(j - NF4 * 4) * sd.n4 + i;
    base[off] = (float)f[j];
  }
  if (a.per_env) {
    float v[36];
    const double Mrb[6] = {m, m, m, Ig[0], Ig[1], Ig[2]};
    for (int j = 0; j < 6; ++j) {
      v[PAR_MINV + j] = (float)(1.0 / (Mrb[j] + Ma[j]));
      v[PAR_A + j] = (float)Ma[j];
      v[PAR_DL + j] = (float)dl[j];
      v[PAR_DQ + j] = (float)dq[j];
    }
    v[PAR_M] = (float)m;
    for (int j = 0; j < 3; ++j) {
      v[PAR_IG + j] = (float)Ig[j]; v[PAR_RB + j] = (float)rb[j]; v[PAR_VC + j] = (float)Vc[j];
    }
    v[PAR_W] = (float)W;
    v[PAR_B] = (float)cn.B;
    for (int kk = 0; kk < PAR_PLANES; ++kk)
      a.planes[kk * a.n_slots + slot] = make_float4(v[4 * kk], v[4 * kk + 1], v[4 * kk + 2], v[4 * kk + 3]);
  }
  const int tp = tgt_plane(a.per_env);
  a.planes[tp * a.n_slots + slot] = make_float4((float)tgt[0], (float)tgt[1], (float)tgt[2], 0.0f);
  if (a.track) {
    a.planes[(tp + 1) * a.n_slots + slot] = make_float4((float)ta[0], (float)ta[1], (float)ta[2], (float)tw[0]);
    a.planes[(tp + 2) * a.n_slots + slot] = make_float4((float)tw[1], (float)tw[2], (float)tph[0], (float)tph[1]);
    a.planes[(tp + 3) * a.n_slots + slot] = make_float4((float)tph[2], (float)tv[0], (float)tv[1], (float)tv[2]);
  }
  if (a.payload) {
    // Payload (stream 1, draws 23-26): mass m_p = U[lo, hi] x (randomised)
    // vehicle mass, attachment point r_p with x, y ~ U[-0.1, 0.1] m and
    // z ~ U[0.05, 0.15] m (below the CoG). Drawn whether or not DR is on.
    const double mp = m * (a.payload_lo + (a.payload_hi - a.payload_lo) * uniform53(seed, STREAM_DR, id, 23));
    const double rp[3] = {-0.1 + 0.2 * uniform53(seed, STREAM_DR, id, 24), -0.1 + 0.2 * uniform53(seed, STREAM_DR, id, 25),
                          0.05 + 0.1 * uniform53(seed, STREAM_DR, id, 26)};
    float v[PAY_DIM];
    if (!payload_block(m, Ig, Ma, W, mp, rp, v)) {
      for (int j = 0; j < PAY_DIM; ++j) v[j] = __int_as_float(0x7fc00000);   // reported as non-finite by the step
    }
    const int pp = pay_plane(a.track);
    for (int kk = 0; kk < PAY_PLANES; ++kk)
      a.planes[(pp + kk) * a.n_slots + slot] = make_float4(v[4 * kk], v[4 * kk + 1], v[4 * kk + 2], v[4 * kk + 3]);
  }
}

// Overwrite added mass / damping planes and recompute M^-1 in FP64.
__global__ void mg_set_hydro_kernel(float4* planes, int64_t n_slots, const float* A, const float* dl,
                                    const float* dq) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  float v[36];
  for (int k = 0; k < PAR_PLANES; ++k) {
    const float4 x = planes[k * n_slots + s];
    v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
  }
  for (int j = 0; j < 6; ++j) {
    if (A) v[PAR_A + j] = A[s * 6 + j];
    if (dl) v[PAR_DL + j] = dl[s * 6 + j];
    if (dq) v[PAR_DQ + j] = dq[s * 6 + j];
  }
  const double Mrb[6] = {v[PAR_M], v[PAR_M], v[PAR_M], v[PAR_IG], v[PAR_IG + 1], v[PAR_IG + 2]};
  for (int j = 0; j < 6; ++j) v[PAR_MINV + j] = (float)(1.0 / (Mrb[j] + (double)v[PAR_A + j]));
  for (int k = 0; k < PAR_PLANES; ++k)
    planes[k * n_slots + s] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// ---------------------------------------------------------------------------
// Adjoint of a recorded rollout (one env per thread).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void ld21(const float* base, int64_t stride, St<float, NT>& x) {
  float f[13 + NT];
#pragma unroll
  for (int j = 0; j < 13 + NT; ++j) f[j] = base[j * stride];
  fields_to_state<NT>(f, x);
}

template <int NT>
__device__ __forceinline__ void st21(float* base, int64_t stride, const St<float, NT>& x) {
  float f[13 + NT];
  state_to_fields<NT>(x, f);
#pragma unroll
  for (int j = 0; j < 13 + NT; ++j) base[j * stride] = f[j];
}

template <int NT, typename ActT>
__device__ void adjoint_env(const AdjArgs& a, const SegDesc& sd, const ActT& A, int64_t i) {
  const int64_t slot = sd.slot_off + i;
  const int64_t ns = a.n_slots;
  Phys<float> P;
  load_phys(a.planes, ns, slot, P);
  const float4 tg = __ldg(&a.planes[TGT_PLANE * ns + slot]);
  float tgt[3] = {tg.x, tg.y, tg.z};
  float4 tr[3] = {tg, tg, tg};
  if (sd.track) {
    for (int q = 0; q < 3; ++q) tr[q] = __ldg(&a.planes[(TGT_PLANE + 1 + q) * ns + slot]);
  }
  // The recorded rollout advanced the counter by T.
  const float k_start = tg.w - (float)a.T;
  St<float, NT> lam;
#pragma unroll
  for (int j = 0; j < 3; ++j) lam.p[j] = a.g_state_T ? a.g_state_T[slot * 21 + j] : 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) lam.q[j] = a.g_state_T ? a.g_state_T[slot * 21 + 3 + j] : 0.0f;
#pragma unroll
  for (int j = 0; j < 6; ++j) lam.nu[j] = a.g_state_T ? a.g_state_T[slot * 21 + 7 + j] : 0.0f;
#pragma unroll
  for (int j = 0; j < NT; ++j) lam.n[j] = a.g_state_T ? a.g_state_T[slot * 21 + 13 + j] : 0.0f;
  HydroGrad<float> g;
#pragma unroll
  for (int j = 0; j < 6; ++j) { g.A[j] = 0.0f; g.dl[j] = 0.0f; g.dq[j] = 0.0f; }
  const int K = sd.K;
  const int n_seg = (a.T + a.ckpt_every - 1) / a.ckpt_every;
  float* scr = a.scratch + slot;
  for (int s = n_seg - 1; s >= 0; --s) {
    const int t0 = s * a.ckpt_every;
    const int t1 = min(a.T, t0 + a.ckpt_every);
    St<float, NT> x;
    ld21<NT>(a.ckpt + (int64_t)s * 21 * ns + slot, ns, x);
    int j = 0;
    for (int t = t0; t < t1; ++t) {
      float raw[NT], c[NT];
      load_actions<NT>(a.actions + t * a.act_stride + sd.act_off + i * NT, raw);
#pragma unroll
      for (int q = 0; q < NT; ++q) c[q] = clamp1(raw[q]);
      for (int k = 0; k < K; ++k, ++j) {
        st21<NT>(scr + (int64_t)j * 21 * ns, ns, x);
        substep<float, NT, false>(x, c, P, A, sd.h, nullptr);
      }
    }
    st21<NT>(scr + (int64_t)j * 21 * ns, ns, x);
    for (int t = t1 - 1; t >= t0; --t) {
      float raw[NT], c[NT], lc[NT];
      load_actions<NT>(a.actions + t * a.act_stride + sd.act_off + i * NT, raw);
#pragma unroll
      for (int q = 0; q < NT; ++q) { c[q] = clamp1(raw[q]); lc[q] = 0.0f; }
      const int jb = (t - t0) * K;
      St<float, NT> xe;
      ld21<NT>(scr + (int64_t)(jb + K) * 21 * ns, ns, xe);
      float go[13];
      const float* gop = nullptr;
      if (a.g_obs) {
#pragma unroll
        for (int q = 0; q < 13; ++q) go[q] = a.g_obs[((int64_t)t * ns + slot) * 13 + q];
        gop = go;
      }
      const float gr = a.g_rew ? a.g_rew[(int64_t)t * ns + slot] : 0.0f;
      if (sd.track) track_ref<float>(tg, tr[0], tr[1], tr[2], sd.dt, k_start + (float)(t + 1), tgt);
      observe_vjp<float, NT>(xe, c, tgt, gop, gr, lam, lc);
      for (int k = K - 1; k >= 0; --k) {
        St<float, NT> xs;
        ld21<NT>(scr + (int64_t)(jb + k) * 21 * ns, ns, xs);
        substep_vjp<float, NT>(xs, c, P, A, sd.h, lam, lc, g);
      }
      if (a.g_actions) {
        float* ga = a.g_actions + t * a.act_stride + sd.act_off + i * NT;
#pragma unroll
        for (int q = 0; q < NT; ++q) ga[q] = (raw[q] >= -1.0f && raw[q] <= 1.0f) ? lc[q] : 0.0f;
      }
    }
  }
  if (a.g_state0) {
    float* o = a.g_state0 + slot * 21;
#pragma unroll
    for (int j = 0; j < 3; ++j) o[j] = lam.p[j];
#pragma unroll
    for (int j = 0; j < 4; ++j) o[3 + j] = lam.q[j];
#pragma unroll
    for (int j = 0; j < 6; ++j) o[7 + j] = lam.nu[j];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[13 + j] = (j < NT) ? lam.n[j] : 0.0f;
  }
  if (a.g_A) {
#pragma unroll
    for (int j = 0; j < 6; ++j) a.g_A[slot * 6 + j] = g.A[j];
  }
  if (a.g_D) {
#pragma unroll
    for (int j = 0; j < 6; ++j) { a.g_D[slot * 12 + j] = g.dl[j]; a.g_D[slot * 12 + 6 + j] = g.dq[j]; }
  }
}

// One warp-sized block per part of a tile: a few thousand envs (the adjoint
// workload) then spread over all SMs instead of a few dozen. Class groups are
// launched as programmatic dependents of one another (disjoint envs and
// outputs) so that they run side by side.
constexpr int ADJ_BLK = 32;
template <int NT>
__global__ void __launch_bounds__(ADJ_BLK) mg_adjoint_kernel(const __grid_constant__ AdjArgs a) {
  __shared__ Act<float> act;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int parts = a.tile_envs / (int)blockDim.x;
  const int tile = a.tile_lo + (int)blockIdx.x / parts;
  if (tile < a.tile_lo + a.n_tiles) {
    const int si = a.seg_lo + find_seg(a.segs + a.seg_lo, a.seg_hi - a.seg_lo, tile);
    const SegDesc& sd = a.segs[si];
    const ClassF& cf = a.classes[sd.cls];
    for (int k = threadIdx.x; k < 72; k += blockDim.x) {
      if (k < 48) (&act.alloc[0][0])[k] = cf.alloc[k / 8][k % 8];
      else if (k < 56) act.kf[k - 48] = cf.kf[k - 48];
      else if (k < 64) act.dz[k - 56] = cf.dz[k - 56];
      else act.alpha[k - 64] = sd.alpha[k - 64];
    }
    __syncthreads();
    const int64_t i = (int64_t)(tile - sd.tile_begin) * a.tile_envs + ((int)blockIdx.x % parts) * blockDim.x +
                      threadIdx.x;
    if (i >= sd.n_envs) {
      // Padding slots of the segment: zero gradients.
      if (i < sd.n4) {
        const int64_t slot = sd.slot_off + i;
        if (a.g_A) for (int j = 0; j < 6; ++j) a.g_A[slot * 6 + j] = 0.0f;
        if (a.g_D) for (int j = 0; j < 12; ++j) a.g_D[slot * 12 + j] = 0.0f;
        if (a.g_state0) for (int j = 0; j < 21; ++j) a.g_state0[slot * 21 + j] = 0.0f;
      }
    } else {
      const volatile Act<float>& va = act;
      adjoint_env<NT>(a, sd, va, i);
    }
  }
  // Completion stays ordered along the stream (see the step kernel).
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// FP64 rollout for finite-difference checks (one env per thread).
// ---------------------------------------------------------------------------

template <int NT>
__device__ void fp64_env(const Fp64Args& a, const SegDesc& sd, int64_t i) {
  const int64_t slot = sd.slot_off + i;
  const int64_t ns = a.n_slots;
  const ClassD& cd = a.classes[sd.cls];
  Act<double> A;
  for (int k = 0; k < 6; ++k)
    for (int q = 0; q < 8; ++q) A.alloc[k][q] = cd.alloc[k][q];
  for (int q = 0; q < 8; ++q) { A.kf[q] = cd.kf[q]; A.dz[q] = cd.dz[q]; A.alpha[q] = cd.alpha[q]; }
  Phys<float> Pf;
  load_phys(a.planes, ns, slot, Pf);
  Phys<double> P;
  for (int j = 0; j < 6; ++j) {
    P.A[j] = (double)Pf.A[j] + (a.dA ? a.eps * a.dA[slot * 6 + j] : 0.0);
    P.dl[j] = (double)Pf.dl[j] + (a.ddl ? a.eps * a.ddl[slot * 6 + j] : 0.0);
    P.dq[j] = (double)Pf.dq[j] + (a.ddq ? a.eps * a.ddq[slot * 6 + j] : 0.0);
  }
  P.m = Pf.m; P.W = Pf.W; P.B = Pf.B;
  for (int j = 0; j < 3; ++j) { P.Ig[j] = Pf.Ig[j]; P.rb[j] = Pf.rb[j]; P.Vc[j] = Pf.Vc[j]; }
  const double Mrb[6] = {P.m, P.m, P.m, P.Ig[0], P.Ig[1], P.Ig[2]};
  for (int j = 0; j < 6; ++j) P.minv[j] = 1.0 / (Mrb[j] + P.A[j]);
  const float4 tg = __ldg(&a.planes[TGT_PLANE * ns + slot]);
  double tgt[3] = {tg.x, tg.y, tg.z};
  float4 tr[3] = {tg, tg, tg};
  if (sd.track) {
    for (int q = 0; q < 3; ++q) tr[q] = __ldg(&a.planes[(TGT_PLANE + 1 + q) * ns + slot]);
  }
  St<float, NT> xf;
  load_state<NT>(a.state + sd.st_off, sd.n4, i, xf);
  St<double, NT> x;
  for (int j = 0; j < 3; ++j) x.p[j] = xf.p[j];
  for (int j = 0; j < 4; ++j) x.q[j] = xf.q[j];
  for (int j = 0; j < 6; ++j) x.nu[j] = xf.nu[j];
  for (int j = 0; j < NT; ++j) x.n[j] = xf.n[j];
  for (int t = 0; t < a.T; ++t) {
    float raw[NT];
    load_actions<NT>(a.actions + t * a.act_stride + sd.act_off + i * NT, raw);
    double c[NT];
    for (int q = 0; q < NT; ++q) c[q] = raw[q] < -1.0f ? -1.0 : (raw[q] > 1.0f ? 1.0 : (double)raw[q]);
    for (int k = 0; k < sd.K; ++k) substep<double, NT, false>(x, c, P, A, a.h, nullptr);
    double o[13], r;
    if (sd.track) track_ref<double>(tg, tr[0], tr[1], tr[2], a.dt, (double)tg.w + (double)(t + 1), tgt);
    observe<double, NT>(x, c, tgt, o, r);
    a.reward[(int64_t)t * ns + slot] = r;
  }
  if (a.state_out) {
    double* so = a.state_out + slot * 21;
    for (int j = 0; j < 3; ++j) so[j] = x.p[j];
    for (int j = 0; j < 4; ++j) so[3 + j] = x.q[j];
    for (int j = 0; j < 6; ++j) so[7 + j] = x.nu[j];
    for (int j = 0; j < 8; ++j) so[13 + j] = j < NT ? x.n[j] : 0.0;
  }
}

template <int NT>
__global__ void __launch_bounds__(128) mg_fp64_kernel(const __grid_constant__ Fp64Args a) {
  if ((int)blockIdx.x >= a.n_tiles) return;
  const int tile = a.tile_lo + blockIdx.x;
  const int si = a.seg_lo + find_seg(a.segs + a.seg_lo, a.seg_hi - a.seg_lo, tile);
  const SegDesc& sd = a.segs[si];
  const int64_t i = (int64_t)(tile - sd.tile_begin) * blockDim.x + threadIdx.x;
  if (i >= sd.n_envs) return;
  fp64_env<NT>(a, sd, i);
}

// ---------------------------------------------------------------------------
// Host-side launchers (called by the runtime).
// ---------------------------------------------------------------------------
#define MG_NT_SWITCH(nt, CALL) \
  switch (nt) {                   \
    case 1: CALL(1); break;       \
    case 2: CALL(2); break;       \
    case 3: CALL(3); break;       \
    case 4: CALL(4); break;       \
    case 5: CALL(5); break;       \
    case 6: CALL(6); break;       \
    case 7: CALL(7); break;       \
    case 8: CALL(8); break;       \
    default: return cudaErrorInvalidValue; \
  }

// Dynamic shared memory of mg_step_kernel<NT, PM, *>.
template <int NT, int PM>
static size_t step_smem(bool track) {
  const int cols = PM == 2 ? PF_DIM : (PM == 1 ? PAR_DIM : 0);
  return sizeof(float) * (N_WARPS * Stage<NT>::warp_floats(track) + cols * STEP_BLK);
}

template <int NT, int PM, int VAR>
static const void* step_fn() {
  return reinterpret_cast<const void*>(&mg_step_kernel<NT, PM, VAR>);
}

// Kernel attributes of a step instantiation: the largest dynamic shared
// memory of its layouts (tracking).
template <int NT, int PM, int VAR>
static cudaError_t step_attrs() {
  static bool done = false;   // per instantiation, per process (one device)
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(step_fn<NT, PM, VAR>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)step_smem<NT, PM>(true));
  if (e == cudaSuccess) done = true;
  return e;
}

// Shared-memory carveout of the next launch of an instantiation: the largest
// (`shared_sm`) or the driver's default; set only when it changes.
template <int NT, int PM, int VAR>
static cudaError_t step_carveout(bool shared_sm) {
  static int current = -2;   // per instantiation, per process (one device)
  const int want = shared_sm ? (int)cudaSharedmemCarveoutMaxShared : (int)cudaSharedmemCarveoutDefault;
  if (want == current) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(step_fn<NT, PM, VAR>(), cudaFuncAttributePreferredSharedMemoryCarveout, want);
  if (e == cudaSuccess) current = want;
  return e;
}

// `dependent`: launch as a programmatic dependent of the previous kernel in
// the stream (the previous launch of the same step, on disjoint envs).
template <int NT, int PM, int VAR>
static cudaError_t launch_step_t(const StepArgs& a, const ClassK* kc, int grid, bool dependent, bool shared_sm,
                                 cudaStream_t st) {
  const size_t smem = step_smem<NT, PM>(a.track != 0);
  cudaError_t e = step_attrs<NT, PM, VAR>();
  if (e == cudaSuccess) e = step_carveout<NT, PM, VAR>(shared_sm);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(STEP_BLK);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (MG_USE_PDL && dependent) ? 1 : 0;
  if constexpr (PM == 3) return cudaLaunchKernelEx(&cfg, mg_step_kernel<NT, PM, VAR>, a, *kc);
  else return cudaLaunchKernelEx(&cfg, mg_step_kernel<NT, PM, VAR>, a, NoClassK{});
}

template <int PM, int VAR>
static cudaError_t launch_step_pv(const StepArgs& a, const ClassK* kc, int nt, int grid, bool dependent,
                                  bool shared_sm, cudaStream_t st) {
#define MG_L(N) return launch_step_t<N, PM, VAR>(a, kc, grid, dependent, shared_sm, st)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaErrorInvalidValue;
}

// Step launch of one class group: thruster count nt, parameter source
// a.per_env (0 class, 1 per-env, 2 payload), variant var (0 propellers with
// Euler, 1 generic actuators with Euler, 2 RK4). `kc` (class-constant
// propeller steps whose segments are all of one class, else null): that
// class's constants, passed as a kernel parameter.
cudaError_t launch_step(const StepArgs& a, const ClassK* kc, int nt, int var, int grid, bool dependent,
                        bool shared_sm, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (kc) {
    if (a.per_env != 0 || var != 0) return cudaErrorInvalidValue;
    return launch_step_pv<3, 0>(a, kc, nt, grid, dependent, shared_sm, st);
  }
  switch (a.per_env * 3 + var) {
    case 0: return launch_step_pv<0, 0>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 1: return launch_step_pv<0, 1>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 2: return launch_step_pv<0, 2>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 3: return launch_step_pv<1, 0>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 4: return launch_step_pv<1, 1>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 5: return launch_step_pv<1, 2>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 6: return launch_step_pv<2, 0>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 7: return launch_step_pv<2, 1>(a, nullptr, nt, grid, dependent, shared_sm, st);
    case 8: return launch_step_pv<2, 2>(a, nullptr, nt, grid, dependent, shared_sm, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reset(const ResetArgs& a, cudaStream_t st) {
  if (a.n_sel <= 0) return cudaSuccess;
  mg_reset_kernel<<<(a.n_sel + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_set_hydro(float4* planes, int64_t n_slots, const float* A, const float* dl, const float* dq,
                             cudaStream_t st) {
  mg_set_hydro_kernel<<<(unsigned)((n_slots + 127) / 128), 128, 0, st>>>(planes, n_slots, A, dl, dq);
  return cudaGetLastError();
}

// Adjoint launch of one class group (tiles of a.tile_envs envs, a multiple
// of ADJ_BLK); `dependent`: programmatic dependent of the previous launch.
template <int NT>
static cudaError_t launch_adjoint_t(const AdjArgs& a, bool dependent, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_tiles * (a.tile_envs / ADJ_BLK)));
  cfg.blockDim = dim3(ADJ_BLK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (MG_USE_PDL && dependent) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, mg_adjoint_kernel<NT>, a);
}

cudaError_t launch_adjoint(const AdjArgs& a, int nt, bool dependent, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (a.tile_envs <= 0 || a.tile_envs % ADJ_BLK != 0) return cudaErrorInvalidValue;
#define MG_L(N) return launch_adjoint_t<N>(a, dependent, st)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaErrorInvalidValue;
}

cudaError_t launch_fp64(const Fp64Args& a, int nt, int block, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
#define MG_L(N) mg_fp64_kernel<N><<<a.n_tiles, block, 0, st>>>(a)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaGetLastError();
}

template <int NT, int PM, int VAR>
static cudaError_t occupancy_t(bool track, int* blocks_per_sm) {
  cudaError_t e = step_attrs<NT, PM, VAR>();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, step_fn<NT, PM, VAR>(), STEP_BLK,
                                                       step_smem<NT, PM>(track));
}

template <int PM, int VAR>
static cudaError_t occupancy_pv(int nt, bool track, int* blocks_per_sm) {
#define MG_L(N) return occupancy_t<N, PM, VAR>(track, blocks_per_sm)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaErrorInvalidValue;
}

// pm 3: class constants as kernel parameters (var 0 only).
cudaError_t step_kernel_occupancy(int nt, int pm, int var, bool track, int* blocks_per_sm) {
  switch (pm * 3 + var) {
    case 0: return occupancy_pv<0, 0>(nt, track, blocks_per_sm);
    case 1: return occupancy_pv<0, 1>(nt, track, blocks_per_sm);
    case 2: return occupancy_pv<0, 2>(nt, track, blocks_per_sm);
    case 3: return occupancy_pv<1, 0>(nt, track, blocks_per_sm);
    case 4: return occupancy_pv<1, 1>(nt, track, blocks_per_sm);
    case 5: return occupancy_pv<1, 2>(nt, track, blocks_per_sm);
    case 6: return occupancy_pv<2, 0>(nt, track, blocks_per_sm);
    case 7: return occupancy_pv<2, 1>(nt, track, blocks_per_sm);
    case 8: return occupancy_pv<2, 2>(nt, track, blocks_per_sm);
    case 9: return occupancy_pv<3, 0>(nt, track, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mg
