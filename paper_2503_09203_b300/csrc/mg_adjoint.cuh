// Adjoint kernel of libmarinegym for sm_103a (B300): the reverse pass over a
// recorded rollout (checkpointed segments recomputed, vector-Jacobian
// products of the substeps). Included by the library's kernels and compiled
// again at run time (NVRTC) with a class's tables as literals.
#pragma once

#include "mg_device.cuh"
#include "mg_internal.h"
#include "mg_step.cuh"

namespace mg {

// ---------------------------------------------------------------------------
// Adjoint of a recorded rollout: a block of four warps per 64 envs, one
// launch per class with the class tables as the kernel parameter
// (constant-bank operands in the vector-Jacobian product).
//
// The reverse pass walks the checkpoint segments from the last to the first.
// Warps 2-3 (the producer) recompute segment s - 1 from its checkpoint while
// warps 0-1 (the consumer) run the vector-Jacobian products of segment s, so
// the forward recompute leaves the consumer's dependent chain. Per substep
// and env the producer stores one record: the start state and the
// right-hand side M nu_dot of a4-a7 (ADJ_REC floats, seven 16-byte vectors;
// in the scratch buffer the records of four consecutive slots interleave by
// vector, so that a warp's stores and copies of one vector touch whole 64-byte
// runs);
// the consumer rebuilds the rest of the substep's tape from it (rotor
// states, R, current, the new velocity and attitude: a few dozen operations
// instead of the full substep) and applies its VJP. Two scratch buffers
// alternate between the warps, with one block barrier per segment. Each
// consumer lane prefetches its next record (and the next step's cotangents
// and actions) into shared memory by cp.async while it computes the current
// substep; record copies go through L2 only (the producer wrote them).
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

#ifndef MG_ADJ_ENVS
#define MG_ADJ_ENVS 64
#endif
constexpr int ADJ_ENVS = MG_ADJ_ENVS;        // envs per block
constexpr int ADJ_THREADS = 2 * ADJ_ENVS;    // first half: reverse pass, second half: forward recompute
static_assert(ADJ_ENVS % 32 == 0, "whole warps per role");

// The fields of the launch's segment that the adjoint reads, held in
// registers: read through a reference into global memory, each use after a
// global store (records, action gradients) would be a fresh dependent load.
struct AdjSeg {
  int64_t act_off, slot_off;
  float h, dt;
  int K, track;
};

// Payload runs: the env's combined-body parameters in a shared-memory
// column [PF_DIM][ADJ_ENVS] (too many to hold in registers next to the
// product).
using AdjPhysPay = PhysSmemFull<ADJ_ENVS>;
constexpr int ADJ_PAY_SMEM = PF_DIM * ADJ_ENVS * 4;
constexpr int ADJ_STEPF = 14 + 8;            // per-step slot: g_obs 13, g_rew 1, actions 8
static_assert(ADJ_REC % 4 == 0 && ADJ_REC >= 27, "record of whole 16-byte vectors");

__device__ __forceinline__ void cp4(unsigned dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp16_l2(unsigned dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// All but the most recent group complete.
__device__ __forceinline__ void cp_wait_but1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Record of one env: state fields (canonical order p3 q4 nu6 n[NT]), rhs at
// 21. In the scratch buffer, record j of slot s starts at
// j * n_slots * ADJ_REC + rec_off(s) and its vector k lies 16 k floats further.
__device__ __forceinline__ int64_t rec_off(int64_t s) { return (s >> 2) * (4 * ADJ_REC) + (s & 3) * 4; }
template <int NT>
__device__ __forceinline__ void store_record(float* rec, const St<float, NT>& x, const float* rhs) {
  float sf[13 + NT], f[ADJ_REC];
  state_to_fields<NT>(x, sf);
#pragma unroll
  for (int j = 0; j < 21; ++j) f[j] = j < 13 + NT ? sf[j % (13 + NT)] : 0.0f;
#pragma unroll
  for (int j = 0; j < 6; ++j) f[21 + j] = rhs ? rhs[j] : 0.0f;
#pragma unroll
  for (int j = 27; j < ADJ_REC; ++j) f[j] = 0.0f;
  float4* r4 = reinterpret_cast<float4*>(rec);
#pragma unroll
  for (int k = 0; k < ADJ_REC / 4; ++k) r4[4 * k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// Consumer-side prefetch slots of one lane: a ring of ADJ_RING records
// [ADJ_RING][ADJ_ENVS][ADJ_REC] (record j in slot j % ADJ_RING: while the reverse
// pass works on record j, records j - 1 and j - 2 stream in) and a ring of
// per-step data [ADJ_RING][ADJ_STEPF][ADJ_ENVS] (step t in slot t % ADJ_RING,
// issued two steps ahead). Every issue is its own cp.async group.
constexpr int ADJ_RING = 3;
struct AdjPrefetch {
  float* rec;
  float* stp;
  int lane;
  __device__ __forceinline__ float* rslot(int b) const { return rec + (b * ADJ_ENVS + lane) * ADJ_REC; }
  __device__ __forceinline__ float* sslot(int b) const { return stp + b * ADJ_STEPF * ADJ_ENVS + lane; }
  __device__ __forceinline__ void issue_rec(const float* src, int b) const {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(rslot(b));
#pragma unroll
    for (int k = 0; k < ADJ_REC / 4; ++k) cp16_l2(dst + 16u * k, src + 16 * k);
    cp_commit();
  }
  template <int NT>
  __device__ __forceinline__ void read(int b, St<float, NT>& x, float rhs[6]) const {
    float f[ADJ_REC];
    const float4* p = reinterpret_cast<const float4*>(rslot(b));
#pragma unroll
    for (int k = 0; k < ADJ_REC / 4; ++k) {
      const float4 v = p[k];
      f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
    float sf[13 + NT];
#pragma unroll
    for (int j = 0; j < 13 + NT; ++j) sf[j] = f[j];
    fields_to_state<NT>(sf, x);
    if (rhs) {
#pragma unroll
      for (int j = 0; j < 6; ++j) rhs[j] = f[21 + j];
    }
  }
  // Step t's cotangents and actions into per-step slot b.
  template <int NT>
  __device__ __forceinline__ void issue_step(const AdjArgs& a, const AdjSeg& sd, int64_t i, int t, int b) const {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(sslot(b));
    const int64_t slot = sd.slot_off + i;
    if (a.g_obs) {
      const float* go = a.g_obs + ((int64_t)t * a.n_slots + slot) * 13;
#pragma unroll
      for (int q = 0; q < 13; ++q) cp4(dst + 4u * ADJ_ENVS * q, go + q);
    }
    if (a.g_rew) cp4(dst + 4u * ADJ_ENVS * 13, a.g_rew + (int64_t)t * a.n_slots + slot);
    const float* ac = a.actions + (int64_t)t * a.act_stride + sd.act_off + i * NT;
#pragma unroll
    for (int q = 0; q < NT; ++q) cp4(dst + 4u * ADJ_ENVS * (14 + q), ac + q);
    cp_commit();
  }
};

// Producer: recompute segment s from its checkpoint into the records of
// buffer `buf`.
template <int NT, bool PAY, int VAR, typename ActT, typename GenT>
__device__ __forceinline__ void adj_produce(const AdjArgs& a, const AdjSeg& sd, const ActT& A, const GenT& G,
                                            const Phys<float>& P, unsigned p_base, int64_t i, int s, float* buf) {
  const int64_t ns = a.n_slots, slot = sd.slot_off + i;
  const int t0 = s * a.ckpt_every, t1 = min(a.T, t0 + a.ckpt_every);
  St<float, NT> x;
  ld21<NT>(a.ckpt + (int64_t)s * 21 * ns + slot, ns, x);
  float* rec = buf + rec_off(slot);
  const int64_t rstride = ns * ADJ_REC;
  for (int t = t0; t < t1; ++t) {
    float raw[NT], c[NT];
    load_actions<NT>(a.actions + (int64_t)t * a.act_stride + sd.act_off + i * NT, raw);
#pragma unroll
    for (int q = 0; q < NT; ++q) c[q] = clamp1(raw[q]);
    for (int k = 0; k < sd.K; ++k) {
      St<float, NT> x0 = x;
      if constexpr (VAR == 2) {
        // RK4: the record is the start state (the reverse pass recomputes the stages).
        if constexpr (PAY) {
          unsigned pb = p_base;
          asm volatile("" : "+r"(pb));
          substep_rk4<float, NT, ActT, AdjPhysPay, true, GenT>(x, c, AdjPhysPay(pb), A, sd.h, G);
        } else {
          substep_rk4<float, NT, ActT, Phys<float>, true, GenT>(x, c, P, A, sd.h, G);
        }
        store_record<NT>(rec, x0, nullptr);
      } else {
        Tape<float, NT> tp;
        if constexpr (PAY) {
          unsigned pb = p_base;
          asm volatile("" : "+r"(pb));
          substep<float, NT, true>(x, c, AdjPhysPay(pb), A, sd.h, &tp);
        } else {
          substep<float, NT, true, ActT, Phys<float>, true, GenT>(x, c, P, A, sd.h, &tp, G);
        }
        store_record<NT>(rec, x0, tp.rhs);
      }
      rec += rstride;
    }
  }
  store_record<NT>(rec, x, nullptr);
}

template <int NT, bool PAY, int VAR, typename ActT, typename GenT>
__device__ __forceinline__ void adjoint_env(const AdjArgs& a, const AdjSeg& sd, const ActT& A, const GenT& G,
                                            int64_t i, bool valid, float* s_rec, float* s_step, float* s_par) {
  const int role = threadIdx.x / ADJ_ENVS;   // 0: reverse pass, 1: forward recompute
  const int lane = threadIdx.x % ADJ_ENVS;
  const int64_t slot = sd.slot_off + i;
  const int64_t ns = a.n_slots;
  Phys<float> P;
  unsigned p_base = 0;
  if constexpr (PAY) {
    // The combined body's parameters (vehicle planes 1-5, 7, 8 and the
    // payload planes) into the env's shared-memory column, read where used.
    if (role == 0 && valid) {
#pragma unroll
      for (int k = 0; k < PF_STD_PLANES + PF_PAY_PLANES; ++k) {
        const int plane = k < PF_STD_PLANES ? pf_std_plane(k) : a.pay_plane + (k - PF_STD_PLANES);
        const float4 v = __ldg(&a.planes[(int64_t)plane * ns + slot]);
        s_par[(4 * k + 0) * ADJ_ENVS + lane] = v.x;
        s_par[(4 * k + 1) * ADJ_ENVS + lane] = v.y;
        s_par[(4 * k + 2) * ADJ_ENVS + lane] = v.z;
        s_par[(4 * k + 3) * ADJ_ENVS + lane] = v.w;
      }
    }
    __syncthreads();
    p_base = smem_addr(s_par) + 4u * (unsigned)lane;
  } else {
    if (valid) load_phys(a.planes, ns, slot, P);
  }
  const int K = sd.K;
  const int n_seg = (a.T + a.ckpt_every - 1) / a.ckpt_every;
  const int64_t buf_floats = (int64_t)(a.ckpt_every * K + 1) * ns * ADJ_REC;
  const int64_t rstride = ns * ADJ_REC;

  // Consumer state.
  St<float, NT> lam;
  HydroGrad<float> g;
  float4 tg = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float4 tr[3] = {tg, tg, tg};
  float k_start = 0.0f;
  AdjPrefetch pf{s_rec, s_step, lane};
  if (role == 0 && valid) {
    tg = __ldg(&a.planes[TGT_PLANE * ns + slot]);
    if (sd.track) {
      for (int q = 0; q < 3; ++q) tr[q] = __ldg(&a.planes[(TGT_PLANE + 1 + q) * ns + slot]);
    }
    k_start = tg.w - (float)a.T;   // the recorded rollout advanced the counter by T
#pragma unroll
    for (int j = 0; j < 3; ++j) lam.p[j] = a.g_state_T ? a.g_state_T[slot * 21 + j] : 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) lam.q[j] = a.g_state_T ? a.g_state_T[slot * 21 + 3 + j] : 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) lam.nu[j] = a.g_state_T ? a.g_state_T[slot * 21 + 7 + j] : 0.0f;
#pragma unroll
    for (int j = 0; j < NT; ++j) lam.n[j] = a.g_state_T ? a.g_state_T[slot * 21 + 13 + j] : 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) { g.A[j] = 0.0f; g.dl[j] = 0.0f; g.dq[j] = 0.0f; }
    // The first two steps back (the last steps of the rollout): their
    // cotangents and actions.
    pf.issue_step<NT>(a, sd, i, a.T - 1, (a.T - 1) % ADJ_RING);
    if (a.T >= 2) pf.issue_step<NT>(a, sd, i, a.T - 2, (a.T - 2) % ADJ_RING);
  }
  float tgt[3] = {tg.x, tg.y, tg.z};

  for (int it = 0; it <= n_seg; ++it) {
    if (role == 1 && it < n_seg && valid)
      adj_produce<NT, PAY, VAR>(a, sd, A, G, P, p_base, i, n_seg - 1 - it, a.scratch + (int64_t)(it & 1) * buf_floats);
    if (role == 0 && it >= 1 && valid) {
      const int s = n_seg - it;
      const int t0 = s * a.ckpt_every, t1 = min(a.T, t0 + a.ckpt_every);
      const float* rec0 = a.scratch + (int64_t)((it - 1) & 1) * buf_floats + rec_off(slot);
      int j = (t1 - t0) * K;   // record of the segment's end state (j >= 1)
      pf.issue_rec(rec0 + (int64_t)j * rstride, j % ADJ_RING);
      pf.issue_rec(rec0 + (int64_t)(j - 1) * rstride, (j - 1) % ADJ_RING);
      cp_wait_but1();   // record j (record j - 1 was committed after it)
      for (int t = t1 - 1; t >= t0; --t) {
        // Step t's cotangents and actions, issued two steps ahead: complete
        // after the last wait (at least one record group followed them).
        float go[13], raw[NT], c[NT], lc[NT];
        const float* sp = pf.sslot(t % ADJ_RING);
#pragma unroll
        for (int q = 0; q < 13; ++q) go[q] = a.g_obs ? sp[ADJ_ENVS * q] : 0.0f;
        const float gr = a.g_rew ? sp[ADJ_ENVS * 13] : 0.0f;
#pragma unroll
        for (int q = 0; q < NT; ++q) {
          raw[q] = sp[ADJ_ENVS * (14 + q)];
          c[q] = clamp1(raw[q]);
          lc[q] = 0.0f;
        }
        if (t >= 2) pf.issue_step<NT>(a, sd, i, t - 2, (t - 2) % ADJ_RING);
        // State at the end of step t: record j (the segment's end on the
        // first step back, else the first substep record of step t + 1).
        St<float, NT> xe;
        pf.read<NT>(j % ADJ_RING, xe, nullptr);
        // After reading record j, record j - 2 is issued (records j and
        // j - 1 were issued before): every record once, two ahead.
        if (t == t1 - 1 && j >= 2) pf.issue_rec(rec0 + (int64_t)(j - 2) * rstride, (j - 2) % ADJ_RING);
        if (sd.track) track_ref<float>(tg, tr[0], tr[1], tr[2], sd.dt, k_start + (float)(t + 1), tgt);
        observe_vjp<float, NT>(xe, c, tgt, a.g_obs ? go : nullptr, gr, lam, lc);
        for (int k = K - 1; k >= 0; --k) {
          --j;
          // Record j: record j - 1 was committed after it, except for j = 0.
          if (j >= 1) cp_wait_but1();
          else cp_wait_all();
          St<float, NT> xs;
          float rhs[6], q1[4];
          pf.read<NT>(j % ADJ_RING, xs, rhs);
          // Records j - 1 and j - 2 stream in while this substep's product runs.
          if (j >= 2) pf.issue_rec(rec0 + (int64_t)(j - 2) * rstride, (j - 2) % ADJ_RING);
          if constexpr (VAR == 2) {
            // RK4: the stages are recomputed from the substep's start state.
            if constexpr (PAY) {
              unsigned pb = p_base;
              asm volatile("" : "+r"(pb));
              substep_rk4_vjp<float, NT, ActT, AdjPhysPay, true, GenT>(xs, c, AdjPhysPay(pb), A, sd.h, lam, lc, g, G);
            } else {
              substep_rk4_vjp<float, NT, ActT, Phys<float>, true, GenT>(xs, c, P, A, sd.h, lam, lc, g, G);
            }
          } else {
            Tape<float, NT> tp;
            if constexpr (PAY) {
              unsigned pb = p_base;
              asm volatile("" : "+r"(pb));
              const AdjPhysPay Pv(pb);
              tape_from_rhs<float, NT>(xs, c, Pv, A, sd.h, rhs, tp, q1);
              vjp_from_tape<float, NT>(xs, q1, tp, c, Pv, A, sd.h, lam, lc, g);
            } else {
              tape_from_rhs<float, NT>(xs, c, P, A, sd.h, rhs, tp, q1);
              vjp_from_tape<float, NT>(xs, q1, tp, c, P, A, sd.h, lam, lc, g, G);
            }
          }
        }
        if (a.g_actions) {
          float* ga = a.g_actions + (int64_t)t * a.act_stride + sd.act_off + i * NT;
#pragma unroll
          for (int q = 0; q < NT; ++q) ga[q] = (raw[q] >= -1.0f && raw[q] <= 1.0f) ? lc[q] : 0.0f;
        }
      }
    }
    // The producer's records of this round are complete and the consumer is
    // done with the buffer the producer fills next.
    __syncthreads();
  }
  if (role != 0 || !valid) return;
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

// One block of four warps per 64 envs of a class segment (one segment per
// launch): the adjoint workload's 8192 envs are 130 blocks, one per SM, each
// warp on its own scheduler (measured against two-warp blocks of 32 envs,
// two per SM: backward 0.537 -> 0.526 ms at 8192 envs x 200 steps x K=4). The launches of a backward pass are programmatic dependents of one
// another (disjoint envs and outputs) so that they run side by side.
// LIT: NoLit (the class tables of the kernel parameter) or, for the kernels
// compiled at run time, a type whose make() returns the class's tables
// (literal operands: zero allocation entries and a zero dead zone drop out).
// PAY: payload runs (the combined body's full inverse and inertia, read
// from a shared-memory column per env: ADJ_PAY_SMEM bytes of dynamic shared
// memory). VAR: 0 propeller classes with Euler, 1 classes with fins or
// servo-tilted propellers with Euler, 2 RK4 runs (1 and 2: the kernel
// parameter carries the generic actuator table too).
template <int NT, bool PAY = false, class LIT = NoLit, int VAR = 0>
__global__ void __launch_bounds__(ADJ_THREADS)
    mg_adjoint_kernel(const __grid_constant__ AdjArgs a,
                      const __grid_constant__ tt::conditional_t<VAR != 0, ClassKG, ClassK> kp) {
  constexpr bool GEN = VAR != 0;
  static_assert(!(PAY && VAR == 1), "payload runs are propeller classes");
  constexpr bool HAS_LIT = !tt::is_same<LIT, NoLit>::value;
  [[maybe_unused]] constexpr ClassK klit = LIT::make();
  const ClassK* kt;
  if constexpr (GEN) kt = &kp.k;
  else kt = &kp;
  if constexpr (HAS_LIT) kt = &klit;
  __shared__ __align__(16) float s_rec[ADJ_RING * ADJ_ENVS * ADJ_REC];
  __shared__ __align__(16) float s_step[ADJ_RING * ADJ_STEPF * ADJ_ENVS];
  extern __shared__ __align__(16) float s_dyn[];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int parts = a.tile_envs / ADJ_ENVS;
  const int tile = a.tile_lo + (int)blockIdx.x / parts;
  if (tile < a.tile_lo + a.n_tiles) {
    const SegDesc& sd = a.segs[a.seg_lo];
    const int64_t i = (int64_t)(tile - sd.tile_begin) * a.tile_envs + ((int)blockIdx.x % parts) * ADJ_ENVS +
                      (threadIdx.x % ADJ_ENVS);
    const bool valid = i < sd.n_envs;
    if (!valid && i < sd.n4 && threadIdx.x < ADJ_ENVS) {
      // Padding slots of the segment: zero gradients.
      const int64_t slot = sd.slot_off + i;
      if (a.g_A) for (int j = 0; j < 6; ++j) a.g_A[slot * 6 + j] = 0.0f;
      if (a.g_D) for (int j = 0; j < 12; ++j) a.g_D[slot * 12 + j] = 0.0f;
      if (a.g_state0) for (int j = 0; j < 21; ++j) a.g_state0[slot * 21 + j] = 0.0f;
    }
    // Every thread of the block takes part in the per-segment barriers.
    const AdjSeg sr{sd.act_off, sd.slot_off, sd.h, sd.dt, sd.K, sd.track};
    if constexpr (GEN) adjoint_env<NT, PAY, VAR>(a, sr, *kt, GenK{kp.g}, i, valid, s_rec, s_step, s_dyn);
    else adjoint_env<NT, PAY, VAR>(a, sr, *kt, NoGen{}, i, valid, s_rec, s_step, s_dyn);
  }
  // Completion stays ordered along the stream (see the step kernel).
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace mg
