// The batched step kernel of libmarinegym for sm_103a (B300) and its launch
// templates; instantiated per parameter source in mg_step_pm0/1/2.cu.
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
// multi-step launch) with the state in registers. Class tables are either
// passed by value as a kernel parameter (launches of one class: read as
// constant-bank operands) or staged in shared memory and read as warp-uniform
// broadcasts. Nothing here is a dense contraction, so there are no
// tensor-core paths.
#pragma once

#include "mg_rtc.h"
#ifndef __CUDACC_RTC__
#include <atomic>

#include "marinegym.h"
#endif
#include "mg_internal.h"
#include "mg_device.cuh"

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
// Segment of launch tile `tile`: from the launch's tile map (TM: serving ticks
// with thousands of segments, one load instead of a search of dependent
// loads), else by binary search (a few segments, cached in shared memory).
template <bool TM>
__device__ __forceinline__ int seg_of_tile(const StepArgs& a, const SegDesc* segs, int n_segs, int tile) {
  if constexpr (TM) return __ldg(a.tile_seg + (tile - a.tile_lo));
  else return find_seg(segs, n_segs, tile);
}

__device__ __forceinline__ float clamp1(float a) { return a < -1.0f ? -1.0f : (a > 1.0f ? 1.0f : a); }

// Serving action j of one Philox4x64 block: 24 bits k of word j % 4 (its top
// bits for j < 4, bits 31..8 for j = 4..7) -> k 2^-23 - 1, exact in FP32, on
// [-1, 1). One block serves up to 8 thrusters.
__device__ __forceinline__ float action_of_block(const uint64_t (&o)[4], int j) {
  const uint64_t w = o[j & 3];
  const unsigned k = j < 4 ? (unsigned)(w >> 40) : (unsigned)((w >> 8) & 0xFFFFFFull);
  return (float)(int)k * (1.0f / 8388608.0f) - 1.0f;
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

// Actions of one env from its row of the stage buffer (row stride NT floats,
// row start 16-byte aligned when NT % 4 == 0, 8-byte when NT % 2 == 0):
// vector loads, which also avoid the bank conflicts of NT scalar reads at a
// 4 NT-byte lane stride. VOL: the slot is refilled by cp.async between reads
// of the same address, so the reads must not be merged or cached.
template <int NT, bool VOL>
__device__ __forceinline__ void lds_actions(unsigned addr, float (&a)[NT]) {
  if constexpr (NT % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NT / 4; ++k) {
      if constexpr (VOL)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(a[4 * k]), "=f"(a[4 * k + 1]), "=f"(a[4 * k + 2]), "=f"(a[4 * k + 3])
                     : "r"(addr + 16u * k) : "memory");
      else
        asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
            : "=f"(a[4 * k]), "=f"(a[4 * k + 1]), "=f"(a[4 * k + 2]), "=f"(a[4 * k + 3]) : "r"(addr + 16u * k));
    }
  } else if constexpr (NT % 2 == 0) {
#pragma unroll
    for (int k = 0; k < NT / 2; ++k) {
      if constexpr (VOL)
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(a[2 * k]), "=f"(a[2 * k + 1]) : "r"(addr + 8u * k)
                     : "memory");
      else
        asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(a[2 * k]), "=f"(a[2 * k + 1]) : "r"(addr + 8u * k));
    }
  } else {
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      if constexpr (VOL)
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(a[k]) : "r"(addr + 4u * k) : "memory");
      else
        asm("ld.shared.f32 %0, [%1];" : "=f"(a[k]) : "r"(addr + 4u * k));
    }
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

// Whether propeller launches of parameter source PM take allocation rows
// premultiplied by the thrust constants (MG_PREMUL). Not for per-env steps
// (PM 1, serving included): there the 8-thruster kernel spilled and the step
// measured slower (104.0 -> 106.4 us at 1M envs); class-constant and payload
// steps gained (1M envs K=4 67.6 -> 66.9 us, K=8 96.8 -> 95.0 us). Every
// table source of a launch kind does the same, so results do not depend on
// the launch shape.
template <int PM, int VAR>
struct Premul {
  static constexpr bool value = MG_PREMUL && VAR == 0 && PM != 1;
};

// Actuator table in shared memory: alloc[6][8] | kf[8] | dz[8] | alpha[8].
// dz_on = 0: the class has no dead zone (the thrust skips the test).
#ifndef MG_DZ_FLAG
#define MG_DZ_FLAG 1
#endif
// DZF: the kernel carries a dead-zone-free thrust path (class-constant
// propellers only: in the other variants the second path costs registers).
// PRE: the staged rows carry the thrust constants (Premul).
template <bool DZF, bool PRE>
struct ActSmemT {
  unsigned base;
  unsigned dz_on;
};
template <bool DZF>
struct ActPremul<ActSmemT<DZF, true>> {
  static constexpr bool value = true;
};
template <bool DZF, bool PRE>
__device__ __forceinline__ bool dz_active(const ActSmemT<DZF, PRE>& A) {
  return !(MG_DZ_FLAG && DZF) || A.dz_on != 0u;
}
// Actuator table passed as the kernel parameter (KP launches): read as
// constant-bank operands. DZF and PRE as for the shared-memory view.
template <bool DZF, bool PRE>
struct ActK {
  const ClassK& k;
};
template <bool DZF>
struct ActPremul<ActK<DZF, true>> {
  static constexpr bool value = true;
};
template <bool DZF, bool PRE>
__device__ __forceinline__ bool dz_active(const ActK<DZF, PRE>& A) {
  return !(MG_DZ_FLAG && DZF) || A.k.dz_on != 0u;
}
template <typename S, int NT, bool DZF, bool PRE>
__device__ __forceinline__ void act_row(const ActK<DZF, PRE>& A, int k, S (&r)[NT]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) r[i] = A.k.alloc[k][i];
}
template <typename S, int NT, bool DZF, bool PRE>
__device__ __forceinline__ void act_rotor(const ActK<DZF, PRE>& A, S (&kf)[NT], S (&dz)[NT], S (&al)[NT]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) { kf[i] = A.k.kf[i]; dz[i] = A.k.dz[i]; al[i] = A.k.alpha[i]; }
}
template <typename S, int NT, bool DZF, bool PRE>
__device__ __forceinline__ void act_rotor_nodz(const ActK<DZF, PRE>& A, S (&kf)[NT], S (&al)[NT]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) { kf[i] = A.k.kf[i]; al[i] = A.k.alpha[i]; }
}
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
template <typename S, int NT, bool DZF, bool PRE>
__device__ __forceinline__ void act_row(const ActSmemT<DZF, PRE>& A, int k, S (&r)[NT]) {
  lds_vec<NT>(A.base + 4 * (SA_ALLOC + 8 * k), r);
}
template <typename S, int NT, bool DZF, bool PRE>
__device__ __forceinline__ void act_rotor(const ActSmemT<DZF, PRE>& A, S (&kf)[NT], S (&dz)[NT], S (&al)[NT]) {
  lds_vec<NT>(A.base + 4 * SA_KF, kf);
  lds_vec<NT>(A.base + 4 * SA_DZ, dz);
  lds_vec<NT>(A.base + 4 * SA_ALPHA, al);
}
template <typename S, int NT, bool DZF, bool PRE>
__device__ __forceinline__ void act_rotor_nodz(const ActSmemT<DZF, PRE>& A, S (&kf)[NT], S (&al)[NT]) {
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
#ifndef __CUDACC_RTC__
static_assert(KIND_PROP == MG_ACT_PROP && KIND_SERVO == MG_ACT_SERVO && KIND_FIN == MG_ACT_FIN &&
                  KIND_TILT == MG_ACT_TILT, "actuator kinds");
#endif
// Generic actuator table passed as the kernel parameter (KP launches).
struct GenK {
  const ClassG& g;
  __device__ __forceinline__ int kind(int i) const { return g.kind[i]; }
  __device__ __forceinline__ float v(int i, int k) const { return g.v[i][k]; }
};
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
// target [32] float4. Each warp of a block owns two stage buffers and runs
// its own copy pipeline. The observation tile [32][13] is a third buffer of
// the warp, or (aliased) rows 0..12 per env of the tile's own stage buffer,
// written once the tile's inputs are in registers (below the action slot and
// the trajectory section); lane 0 then waits for the observation store to
// read the buffer before refilling it. Aliased: the per-env propeller kernels
// (measured at 1M envs, DR + current, K=4: 94.9 -> 91.7 us; 262k envs 31.05
// -> 29.3 us: a fourth block then fits an SM's shared memory) and, with
// MG_OBS_ALIAS, every kernel (the class-specialised kernels are compiled so);
// not aliased: the others (no gain measured with class constants at 4
// blocks per SM, tracking 70.4 -> 70.9 us, payload 126.7 -> 127.0 us).
#ifndef MG_OBS_ALIAS
#define MG_OBS_ALIAS 0
#endif
template <int PM, int VAR, bool TM>
struct ObsAlias {
  static constexpr bool value = MG_OBS_ALIAS || (PM == 1 && VAR == 0 && !TM);
};
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
  static __host__ __device__ constexpr int warp_floats(bool track, bool alias) {
    return 2 * floats(track) + (alias ? 0 : OBS);
  }
  static_assert(OBS <= ACT_OFF, "an aliased observation tile lies below the action slot");
  static_assert((ACT_OFF % 4) == 0 && (TGT_OFF % 4) == 0 && (TRJ_OFF % 4) == 0 && (OBS % 4) == 0,
                "16-byte aligned sections");
};
constexpr int SEG_CACHE = 16;   // segments of a launch kept in shared memory

// Class tables of segment `sd` into act (SA_DIM) and phys (PAR_DIM), and its
// generic actuator table into gen (generic variants), by the block's threads.
template <int PM, int VAR>
__device__ __forceinline__ void stage_tables(const StepArgs& a, const SegDesc& sd, float* act, float* phys,
                                             float* gen, int tid) {
  const ClassF& cf = a.classes[sd.cls];
  for (int k = tid; k < SA_DIM + PAR_DIM; k += STEP_BLK) {
    if (k < 48) act[k] = Premul<PM, VAR>::value ? cf.alloc[k / 8][k % 8] * cf.kf[k % 8] : cf.alloc[k / 8][k % 8];
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

// Class tables of segment `sd` into one warp's copies (lanes of that warp):
// the actuator table, for class-constant ticks (PM = 0) the nominal physics
// block, and for generic classes (VAR = 1) the generic actuator table.
// Serving ticks: rows as staged above.
template <int PM, int VAR>
__device__ __forceinline__ void stage_tables_warp(const StepArgs& a, const SegDesc& sd, float* act, float* phys,
                                                  float* gen, int lane) {
  const ClassF& cf = a.classes[sd.cls];
  for (int k = lane; k < SA_DIM; k += WENV) {
    if (k < 48) act[k] = Premul<PM, VAR>::value ? cf.alloc[k / 8][k % 8] * cf.kf[k % 8] : cf.alloc[k / 8][k % 8];
    else if (k < 56) act[k] = cf.kf[k - 48];
    else if (k < 64) act[k] = cf.dz[k - 56];
    else act[k] = sd.alpha[k - 64];
  }
  if (PM == 0)
    for (int k = lane; k < PAR_DIM; k += WENV) phys[k] = cf.phys[k];
  if (VAR) {
    const float* g = reinterpret_cast<const float*>(&cf.gen);
    for (int k = lane; k < GEN_FLOATS; k += WENV) gen[k] = g[k];
  }
}

// Issue the bulk copies of one warp's slice of a tile (lane 0 only). `nvw`
// (a multiple of 4, > 0) envs start at local env index w0 of the segment.
template <int NT, int PM>
__device__ __forceinline__ void issue_warp_loads(const StepArgs& a, const SegDesc& sd, int64_t w0, unsigned nvw,
                                                 float* buf, unsigned bar) {
  constexpr bool PER_ENV = PM >= 1;
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

// KP: the class tables (actuators; physics for PM 0; the generic table for
// VAR >= 1) come from the kernel parameter (*kc, *kg) instead of shared memory.
// Per-env parameter planes of this thread's env of a tile into its own
// column of s_par (PA: per-env launches other than serving ticks), by
// cp.async: issued once the thread has finished with the previous tile's
// column, waited for when the tile starts. Measured at 1M envs: per-env DR
// 103.5 -> 100.3 us, actuated Euler 181 -> 167.5 us, RK4 500 -> 478 us (no
// registers hold the next tile's parameters, so the per-env kernels stopped
// spilling); 16k-env rollout graph 6.87e9 -> 9.25e9 env-steps/s. Serving
// ticks (short tiles) keep vector loads: 36 four-byte copies per thread cost
// them 4-6%; payload steps (60 copies) measured slower too (131.4 -> 133.9
// us) and keep their direct staging.
#ifndef MG_PAR_ASYNC
#define MG_PAR_ASYNC 1
#endif
__device__ __forceinline__ void issue_par_copies(const StepArgs& a, const SegDesc& sd, int64_t local0, int warp,
                                                 int lane, float* s_par, int tid) {
  const int64_t i = local0 + warp * WENV + lane;
  if (i < sd.n_envs) {
    const float* src = reinterpret_cast<const float*>(a.planes + sd.slot_off + i);
    const unsigned dst = smem_addr(s_par + tid);
#pragma unroll
    for (int k = 0; k < PAR_PLANES; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 4u * (4 * k + q) * STEP_BLK),
                     "l"(src + (int64_t)k * a.n_slots * 4 + q)
                     : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int NT, int PM, int VAR, bool KP, bool MS, bool PA>
__device__ __forceinline__ bool step_tile(const StepArgs& a, const ClassK* kc, const ClassG* kg, const SegDesc& sd,
                                          int tile, unsigned s_act, unsigned s_phys, unsigned s_gen,
                                          const float* buf, float* obs_w, float* s_par, int& n_emit) {
  constexpr bool PER_ENV = PM >= 1;
  constexpr bool DZF = PM == 0 && VAR == 0;
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
  constexpr bool PRE = Premul<PM, VAR>::value;
  // Propeller / Euler steps without a payload read their actions with vector
  // loads and check finiteness through the reward (fewer instructions per
  // step); the other variants measured faster with scalar reads and the plain
  // 21-field sum (their register allocation is tighter).
  constexpr bool LEAN = VAR == 0 && PM != 2;
  using ActSmem = ActSmemT<DZF, PRE>;
  const ActSmem A{s_act, (unsigned)(sd.flags & 1)};

  // Per-env parameters: plain per-env runs prefetch their 9 planes into
  // registers here (their loads overlap the stage reads below); payload runs
  // copy 15 planes straight to shared memory afterwards.
  constexpr bool STAGE_PAR = PM == 1 && !PA;
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
      if constexpr (LEAN) {
        float raw[NT];
        lds_actions<NT, false>(smem_addr(buf + SG::ACT_OFF + lane * NT), raw);
#pragma unroll
        for (int j = 0; j < NT; ++j) c[j] = clamp1(raw[j]);
      } else {
#pragma unroll
        for (int j = 0; j < NT; ++j) c[j] = clamp1(buf[SG::ACT_OFF + lane * NT + j]);
      }
      have_act0 = true;
    }
  }
  if (PA) asm volatile("cp.async.wait_group 0;" ::: "memory");
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
  using PV = tt::conditional_t<PM == 2, PhysSmemFull<STEP_BLK>, PhysSmem<PER_ENV ? STEP_BLK : 1>>;
  const unsigned p_base = PER_ENV ? smem_addr(s_par) + 4u * tid : s_phys;
  const unsigned g_base = s_gen;
  const int n_out_steps = a.n_steps == 0 ? 1 : a.n_steps;
  float r_last = 0.0f;   // reward of the last step (always emitted)
  for (int t = 0; t < n_out_steps; ++t) {
    if (valid && a.n_steps > 0) {
      if (a.act_mode == 0) {
        if constexpr (MS) {
          // Multi-step launches: the env's action slot of the stage buffer
          // (free once step 0 has read it) receives step t+1's actions by
          // cp.async while step t runs, so no step starts with a dependent
          // global load. Volatile reads: the slot's address repeats.
          const unsigned act_slot = smem_addr(buf + SG::ACT_OFF + lane * NT);
          if (!(t == 0 && have_act0)) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if constexpr (LEAN) {
              float raw[NT];
              lds_actions<NT, true>(act_slot, raw);
#pragma unroll
              for (int j = 0; j < NT; ++j) c[j] = clamp1(raw[j]);
            } else {
#pragma unroll
              for (int j = 0; j < NT; ++j) {
                float v;
                asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(act_slot + 4u * j) : "memory");
                c[j] = clamp1(v);
              }
            }
          }
          if (t + 1 < a.n_steps) {
            const float* src = a.actions + (int64_t)(t + 1) * a.act_stride + sd.act_off + i * NT;
#pragma unroll
            for (int j = 0; j < NT; ++j)
              asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(act_slot + 4u * j), "l"(src + j)
                           : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
          }
        } else if (!(t == 0 && have_act0)) {
          float raw[NT];
          load_actions<NT>(a.actions + t * a.act_stride + sd.act_off + i * NT, raw);
#pragma unroll
          for (int j = 0; j < NT; ++j) c[j] = clamp1(raw[j]);
        }
      } else {
        static_assert(NT <= 8, "one Philox block holds 8 actions");
        uint64_t o[4];
        philox4x64((uint64_t)i, (uint64_t)(sd.step0 + t), 0, 0, sd.seed, STREAM_ACTION, o);
#pragma unroll
        for (int j = 0; j < NT; ++j) c[j] = clamp1(action_of_block(o, j));
      }
      if (a.ckpt && (t % a.ckpt_every) == 0) {
        float f[13 + NT];
        state_to_fields<NT>(x, f);
        float* ck = a.ckpt + (int64_t)(t / a.ckpt_every) * 21 * a.n_slots + slot;
#pragma unroll
        for (int j = 0; j < 21; ++j) ck[j * a.n_slots] = (j < 13 + NT) ? f[j % (13 + NT)] : 0.0f;
      }
      // One substep with the parameter views P (physics), Av (actuators), G
      // (generic table). Class-constant physics carries no current (zero by
      // construction): CURRENT = PER_ENV.
      auto sub = [&](const auto& P, const auto& Av, const auto& G) {
        using PT = tt::decay_t<decltype(P)>;
        using AT = tt::decay_t<decltype(Av)>;
        using GT = tt::decay_t<decltype(G)>;
        if constexpr (VAR == 2) substep_rk4<float, NT, AT, PT, PER_ENV, GT>(x, c, P, Av, sd.h, G);
        else substep<float, NT, false, AT, PT, PER_ENV, GT>(x, c, P, Av, sd.h, nullptr, G);
      };
      // Shared-memory bases made opaque once per substep: loads may be
      // scheduled freely inside a substep but not hoisted out of the loop.
      // Kernel-parameter tables are read as operands where they are used.
      for (int k = 0; k < sd.K; ++k) {
        if constexpr (KP) {
          const ActK<DZF, PRE> Av{*kc};
          if constexpr (PM == 0) {
            if constexpr (VAR == 0) sub(*kc, Av, NoGen{});
            else sub(*kc, Av, GenK{*kg});
          } else {
            unsigned pb = p_base;
            asm volatile("" : "+r"(pb));
            const PV Pk(pb);
            if constexpr (VAR == 0) sub(Pk, Av, NoGen{});
            else sub(Pk, Av, GenK{*kg});
          }
        } else {
          unsigned pb = p_base, ab = A.base, gb = g_base;
          asm volatile("" : "+r"(pb), "+r"(ab), "+r"(gb));
          const ActSmem Ak{ab, A.dz_on};
          const PV Pk(pb);
          if constexpr (VAR == 0) sub(Pk, Ak, NoGen{});
          else sub(Pk, Ak, GenSmem{gb});
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
        r_last = r;
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
    // Non-finite state check. The last step's reward -|d|^2 - 0.1|nu|^2 -
    // 0.01|c|^2 is a sum of non-positive terms (no inf - inf), so it is finite
    // exactly when p, nu and c are; c is clamped to [-1, 1], so only a NaN
    // command is non-finite, and it makes n NaN as well. Lean kernels
    // therefore add only q and n to it.
    float s = LEAN ? r_last : 0.0f;
    if constexpr (!LEAN) {
#pragma unroll
      for (int j = 0; j < 3; ++j) s += x.p[j];
#pragma unroll
      for (int j = 0; j < 6; ++j) s += x.nu[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s += x.q[j];
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
// a per-warp bulk store. Warps never wait on one another except when a
// block's shared class table changes (not in launches with the tables as the
// kernel parameter, nor in serving ticks, whose warps keep their own table).
// Every wait is bounded (2 s); a warp that gives up
// sets bit 1 of the status word and skips the rest of its tiles (it keeps
// walking them, so every block barrier is still reached).
// The RK4 variant keeps the stage point, the running sum and the substep's
// start state live at once. It is compiled for 3 resident blocks per SM (168
// registers): measured at 1M envs, K=4, that beats both 4 blocks (heavy
// spills) and 2 blocks (too few warps to hide latency), although the payload
// instantiations still spill 52-160 bytes. The generic-actuator
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
// Serving-tick kernels (TM) are compiled for 3 blocks per SM: at 4 their
// 8-thruster instantiation spilled, and shared memory held it to 3 blocks
// anyway (10^4-request serving run: 5.66e9 -> 6.19e9 env-steps/s while busy).
#ifndef MG_TM_MIN_BLOCKS
#define MG_TM_MIN_BLOCKS 3
#endif
template <int PM, int VAR, bool KP, bool TM>
struct StepMinBlocks {
  static constexpr int value = VAR == 2               ? MG_RK4_MIN_BLOCKS
                               : VAR == 1             ? MG_GEN_MIN_BLOCKS
                               : TM                   ? MG_TM_MIN_BLOCKS
                               : (KP && PM == 0)      ? MG_KSTEP_MIN_BLOCKS
                                                      : MG_STEP_MIN_BLOCKS;
};

// Second kernel parameter: the class tables of a KP launch (ClassK, plus the
// generic table for VAR >= 1), else nothing.
struct NoClassK {};

// Class constants known when the kernel is compiled: the class-specialised
// step kernels that the library compiles at run time (NVRTC) for one-class
// propeller launches take a type whose make() returns the class's ClassK,
// so that the arithmetic sees literals (zero allocation entries and, with
// class-constant physics, a zero restoring arm and W = B drop out; per-env
// launches take only the actuator tables from it). NoLit: the constants come
// from the kernel parameter.
struct NoLit {
  MG_HD static constexpr ClassK make() { return ClassK{}; }
};
template <bool KP, int VAR>
using KParam = tt::conditional_t<!KP, NoClassK, tt::conditional_t<VAR == 0, ClassK, ClassKG>>;

// PM: parameter source (0 class constants, 1 per-env planes, 2 per-env planes
// with the payload). KP: the launch holds one class and its tables travel as
// the kernel parameter `kp` (otherwise they are staged in shared memory). TM:
// tiles find their segment through the launch's tile map (serving). MS: a
// launch of several steps prefetches each next step's actions. The
// body stays in the kernel itself: moved into a function taking the
// parameters by reference, the per-env and payload instantiations spilled.
template <int NT, int PM, int VAR, bool KP, bool TM, bool MS, class LIT = NoLit>
__global__ void __launch_bounds__(STEP_BLK, (StepMinBlocks<PM, VAR, KP, TM>::value))
    mg_step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ KParam<KP, VAR> kp) {
  using SG = Stage<NT>;
  constexpr bool PA = PM == 1 && !TM && MG_PAR_ASYNC;
  constexpr bool HAS_LIT = !tt::is_same<LIT, NoLit>::value;
  static_assert(!HAS_LIT || (KP && PM <= 1 && VAR == 0 && !TM), "literal class constants: one-class propeller launches");
  const ClassK* kc = nullptr;
  const ClassG* kg = nullptr;
  if constexpr (KP && VAR == 0) kc = &kp;
  if constexpr (KP && VAR != 0) { kc = &kp.k; kg = &kp.g; }
  [[maybe_unused]] constexpr ClassK klit = LIT::make();
  if constexpr (HAS_LIT) kc = &klit;
  extern __shared__ __align__(16) float s_dyn[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr bool ALIAS = ObsAlias<PM, VAR, TM>::value;
  const int fl = SG::floats(a.track != 0), wfl = SG::warp_floats(a.track != 0, ALIAS);
  float* const w_base = s_dyn + warp * wfl;
  float* const buf0 = w_base;
  float* const buf1 = w_base + fl;
  float* const obs_sep = w_base + 2 * fl;   // separate observation tile (unless aliased)
  float* const s_par = s_dyn + N_WARPS * wfl;
  // Serving ticks (TM) keep one actuator table (and, with class constants,
  // one physics block) per warp: their tiles change segment almost every
  // time. Other launches keep one per block.
  __shared__ __align__(16) float s_act[TM ? N_WARPS * SA_DIM : SA_DIM];
  __shared__ __align__(16) float s_phys[TM ? N_WARPS * PAR_DIM : PAR_DIM];
  __shared__ __align__(16) float s_gen[VAR ? (TM ? N_WARPS * GEN_FLOATS : GEN_FLOATS) : 4];
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
    const SegDesc& s0 = segs[seg_of_tile<TM>(a, segs, n_seg, tile0)];
    const int64_t local0 = (int64_t)(tile0 - s0.tile_begin) * STEP_BLK;
    nvw_cur = warp_envs(s0, local0, warp);
    if (lane == 0 && nvw_cur > 0 && !(s0.flags & 2))
      issue_warp_loads<NT, PM>(a, s0, local0 + warp * WENV, nvw_cur, buf0, full0);
    if (PA) issue_par_copies(a, s0, local0, warp, lane, s_par, tid);
  }
  int prev_seg = -1, n_emit = 0;
  // Completed uses of each stage barrier (two scalars: an array indexed by
  // the stage parity would live in local memory).
  unsigned use0 = 0u, use1 = 0u;
  bool failed = false;
  for (int j = 0, tt = blockIdx.x; tt < a.n_tiles; ++j, tt += gridDim.x) {
    const int tile = a.tile_lo + tt;
    const int b = j & 1;
    const int si = seg_of_tile<TM>(a, segs, n_seg, tile);
    // Refill the other buffer (read during tile j - 1) with the next slice.
    const int tt_next = tt + gridDim.x;
    unsigned nvw_next = 0;
    if (tt_next < a.n_tiles) {
      const int tile_n = a.tile_lo + tt_next;
      const SegDesc& sn = segs[seg_of_tile<TM>(a, segs, n_seg, tile_n)];
      const int64_t ln = (int64_t)(tile_n - sn.tile_begin) * STEP_BLK;
      nvw_next = warp_envs(sn, ln, warp);
      if (lane == 0 && nvw_next > 0 && !failed && !(sn.flags & 2)) {
        // The buffer may still be the source of the previous tile's observation store.
        if (ALIAS) bulk_wait_read0();
        fence_async_smem();
        issue_warp_loads<NT, PM>(a, sn, ln + warp * WENV, nvw_next, b ? buf0 : buf1, b ? full0 : full1);
      }
    }
    const SegDesc& sd = segs[si];
    if constexpr (TM) {
      // Per-env physics; the warp rewrites its own actuator table (its lanes
      // finished the previous tile at the warp barrier that ends each round).
      if (si != prev_seg) {
        stage_tables_warp<PM, VAR>(a, sd, s_act + warp * SA_DIM, s_phys + warp * PAR_DIM,
                                   s_gen + (TM && VAR ? warp * GEN_FLOATS : 0), lane);
        __syncwarp();
        prev_seg = si;
      }
    } else if (!KP && si != prev_seg) {
      // Class constants change: rewrite them between two block barriers
      // (every warp of the block walks the same tiles).
      __syncthreads();
      stage_tables<PM, VAR>(a, sd, s_act, s_phys, s_gen, tid);
      __syncthreads();
      prev_seg = si;
    }
    // A warp whose wait ran out stops computing and copying but stays in the
    // loop, so that it still reaches every block barrier of the launch.
    if (nvw_cur > 0 && !failed) {
      if (mbar_wait_bounded(b ? full1 : full0, (b ? use1 : use0) & 1u,
                            sd.wait_limit_ns ? sd.wait_limit_ns : kWaitLimitNs)) {
        if (b) ++use1;
        else ++use0;
      }
      else
        failed = true;
    }
    if (!failed)
      step_tile<NT, PM, VAR, KP, MS, PA>(a, kc, kg, sd, tile, smem_addr(s_act + (TM ? warp * SA_DIM : 0)),
                                 smem_addr(s_phys + (TM ? warp * PAR_DIM : 0)),
                                 smem_addr(s_gen + (TM && VAR ? warp * GEN_FLOATS : 0)), b ? buf1 : buf0,
                                 ALIAS ? (b ? buf1 : buf0) : obs_sep, s_par, n_emit);
    if (PA && !failed && tt_next < a.n_tiles) {
      // This thread is done with its parameter column: bring in the next tile's.
      const int tile_n = a.tile_lo + tt_next;
      const SegDesc& sn = segs[seg_of_tile<TM>(a, segs, n_seg, tile_n)];
      issue_par_copies(a, sn, (int64_t)(tile_n - sn.tile_begin) * STEP_BLK, warp, lane, s_par, tid);
    }
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

#ifndef __CUDACC_RTC__
// ---------------------------------------------------------------------------
// Host-side launch templates of the step kernel. Each parameter source is
// instantiated in its own translation unit (mg_step_pm0/1/2.cu) so that the
// 48 kernels of each compile in parallel.
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

// Dynamic shared memory of mg_step_kernel<NT, PM, VAR, *, TM>.
template <int NT, int PM, int VAR, bool TM>
static size_t step_smem(bool track) {
  const int cols = PM == 2 ? PF_DIM : (PM == 1 ? PAR_DIM : 0);
  return sizeof(float) * (N_WARPS * Stage<NT>::warp_floats(track, ObsAlias<PM, VAR, TM>::value) + cols * STEP_BLK);
}

template <int NT, int PM, int VAR, bool KP, bool TM, bool MS = false>
static const void* step_fn() {
  return reinterpret_cast<const void*>(&mg_step_kernel<NT, PM, VAR, KP, TM, MS>);
}

// Kernel attributes of a step instantiation: the largest dynamic shared
// memory of its layouts (tracking). A function attribute belongs to the
// function on each device, so it is set once per instantiation and device
// (bit d of `done`; devices beyond 63 set it on every launch); concurrent
// callers may both set it, which is harmless.
template <int NT, int PM, int VAR, bool KP, bool TM, bool MS = false>
static cudaError_t step_attrs() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(step_fn<NT, PM, VAR, KP, TM, MS>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_smem<NT, PM, VAR, TM>(true));
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// `dependent`: launch as a programmatic dependent of the previous kernel in
// the stream (the previous launch of the same step, on disjoint envs).
// `shared_sm`: the largest shared-memory carveout for this launch, else the
// driver's default preference; a launch attribute, so launches of the same kernel with
// different carveouts (two simulators, two devices, two threads) never
// rewrite a shared function attribute.
template <int NT, int PM, int VAR, bool KP, bool TM, bool MS = false>
static cudaError_t launch_step_t(const StepArgs& a, const ClassK* kc, const ClassG* kg, int grid, bool dependent,
                                 bool shared_sm, cudaStream_t st) {
  const size_t smem = step_smem<NT, PM, VAR, TM>(a.track != 0);
  cudaError_t e = step_attrs<NT, PM, VAR, KP, TM, MS>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(STEP_BLK);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (shared_sm) {   // otherwise the function's own (default) preference
    attr[na].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[na].val.sharedMemCarveout = (unsigned)cudaSharedmemCarveoutMaxShared;
    ++na;
  }
  if (MG_USE_PDL && dependent) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  if constexpr (!KP) {
    return cudaLaunchKernelEx(&cfg, mg_step_kernel<NT, PM, VAR, KP, TM, MS>, a, NoClassK{});
  } else if constexpr (VAR == 0) {
    return cudaLaunchKernelEx(&cfg, mg_step_kernel<NT, PM, VAR, KP, TM, MS>, a, *kc);
  } else {
    ClassKG t;
    t.k = *kc;
    t.g = *kg;
    return cudaLaunchKernelEx(&cfg, mg_step_kernel<NT, PM, VAR, KP, TM, MS>, a, t);
  }
}

template <int PM, int VAR, bool KP, bool TM = false, bool MS = false>
static cudaError_t launch_step_pv(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int grid,
                                  bool dependent, bool shared_sm, cudaStream_t st) {
#define MG_L(N) return launch_step_t<N, PM, VAR, KP, TM, MS>(a, kc, kg, grid, dependent, shared_sm, st)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaErrorInvalidValue;
}

// Step launch with parameter source PM: variant var, class tables from the
// kernel parameter when kc is given (and kg for var >= 1). A serving tick
// (act_mode 1: per-env propeller steps with a tile map) has its own
// instantiation.
template <int PM>
static cudaError_t launch_step_pm(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                                  bool dependent, bool shared_sm, cudaStream_t st) {
  if (kc && var != 0 && !kg) return cudaErrorInvalidValue;
  if (a.act_mode == 1) {
    // Serving ticks: per-env parameters (DR or current on), or class
    // constants; propeller classes (var 0), generic ones (var 1) or RK4
    // (var 2); variants 1 and 2 stage the actuator table per warp from the
    // class records.
    if constexpr (PM <= 1) {
      if (kc) return cudaErrorInvalidValue;
      if (var == 2) return launch_step_pv<PM, 2, false, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
      if (var == 1) return launch_step_pv<PM, 1, false, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
      return launch_step_pv<PM, 0, false, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  // Propeller launches of several steps with actions from memory: the
  // prefetching instantiation (measured: 16k-env 100-step rollout graph
  // 5.72e9 -> 6.89e9 env-steps/s; kept apart because the extra code made the
  // single-step kernels spill).
  if (var == 0 && a.act_mode == 0 && a.n_steps > 1) {
    if (kc) return launch_step_pv<PM, 0, true, false, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    return launch_step_pv<PM, 0, false, false, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
  }
  switch (var * 2 + (kc ? 1 : 0)) {
    case 0: return launch_step_pv<PM, 0, false>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    case 1: return launch_step_pv<PM, 0, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    case 2: return launch_step_pv<PM, 1, false>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    case 3: return launch_step_pv<PM, 1, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    case 4: return launch_step_pv<PM, 2, false>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    case 5: return launch_step_pv<PM, 2, true>(a, kc, kg, nt, grid, dependent, shared_sm, st);
    default: return cudaErrorInvalidValue;
  }
}

// Load the serving-tick kernel of thruster count nt (and set its attributes)
// ahead of the first tick: with lazy module loading the first launch of each
// kernel otherwise pays the load, and early requests queue behind it.
template <int PM>
static cudaError_t prepare_tick_pm(int nt, int var) {
  if (var == 2) {
#define MG_L(N) return step_attrs<N, PM, 2, false, true, false>()
    MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  }
  if (var == 1) {
#define MG_L(N) return step_attrs<N, PM, 1, false, true, false>()
    MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  }
#define MG_L(N) return step_attrs<N, PM, 0, false, true, false>()
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaErrorInvalidValue;
}

template <int NT, int PM, int VAR, bool KP, bool TM, bool MS = false>
static cudaError_t occupancy_t(bool track, int* blocks_per_sm) {
  cudaError_t e = step_attrs<NT, PM, VAR, KP, TM, MS>();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, step_fn<NT, PM, VAR, KP, TM, MS>(), STEP_BLK,
                                                       step_smem<NT, PM, VAR, TM>(track));
}

template <int PM, int VAR, bool KP>
static cudaError_t occupancy_pv(int nt, bool track, int* blocks_per_sm) {
#define MG_L(N) return occupancy_t<N, PM, VAR, KP, false>(track, blocks_per_sm)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaErrorInvalidValue;
}

template <int PM>
static cudaError_t occupancy_pm(int nt, int var, bool kp, bool track, int* blocks_per_sm) {
  switch (var * 2 + (kp ? 1 : 0)) {
    case 0: return occupancy_pv<PM, 0, false>(nt, track, blocks_per_sm);
    case 1: return occupancy_pv<PM, 0, true>(nt, track, blocks_per_sm);
    case 2: return occupancy_pv<PM, 1, false>(nt, track, blocks_per_sm);
    case 3: return occupancy_pv<PM, 1, true>(nt, track, blocks_per_sm);
    case 4: return occupancy_pv<PM, 2, false>(nt, track, blocks_per_sm);
    case 5: return occupancy_pv<PM, 2, true>(nt, track, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

#endif  // __CUDACC_RTC__

}  // namespace mg
