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
// The reverse pass walks the rollout in units (a checkpoint segment, or a
// part of one: AdjUnit) from the last to the first. Warps 2-3 (the producer)
// recompute unit u - 1 from its segment's checkpoint while warps 0-1 (the
// consumer) run the vector-Jacobian products of unit u, so the forward
// recompute leaves the consumer's dependent chain. The producer
// stores the state at every substep boundary (q, nu, n, and p at step
// boundaries: the records of Rec<NT>); the consumer rebuilds a substep's tape
// from the records of its start and end (the end gives the new actuator
// states, the new velocity and so M^-1 rhs, and the end attitude; R, the
// current, the relative velocity and the quaternion update are a few dozen
// operations) and applies its VJP. Two buffers per class segment alternate
// between the warps, with one block barrier per unit. Each consumer lane
// prefetches its next records (and the next step's cotangents and actions)
// into shared memory by cp.async while it computes the current
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
  int K, track, n4;
};

// Payload runs: the env's combined-body parameters in a shared-memory
// column [PF_DIM][ADJ_ENVS] (too many to hold in registers next to the
// product).
using AdjPhysPay = PhysSmemFull<ADJ_ENVS>;
constexpr int ADJ_PAY_SMEM = PF_DIM * ADJ_ENVS * 4;
constexpr int ADJ_STEPF = 14 + 8;            // per-step slot: g_obs 13, g_rew 1, actions 8

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

// Record of one env at one substep boundary: the state fields q4 nu6 n[NT]
// and, at step boundaries (substep 0 of a step, and the segment's end), p3
// after them, in whole 16-byte vectors (Rec<NT>::IN or Rec<NT>::ST). The
// reverse pass of a substep reads the records of its start and end: the end
// gives the new actuator states, the new velocity (so M^-1 rhs = (nu1 -
// nu0) / h) and the end attitude, and p is needed only where the
// observation is taken.
//
// Layout of a class segment's buffer: the records of one checkpoint segment
// in time order, record j a plane of V(j) vectors over the segment's n4
// slots, in which four consecutive slots interleave by vector (slot i at
// (i / 4) 16 V + (i % 4) 4 floats, vector k 16 k floats further), so that a
// warp's stores and copies of one vector touch whole 64-byte runs.
template <int NT>
struct Rec {
  static constexpr int IN = (10 + NT + 3) / 4;   // vectors of a record inside a step
  static constexpr int ST = (13 + NT + 3) / 4;   // vectors of a record at a step boundary
  // Floats per env of a shared-memory record slot: an odd number of
  // vectors, so that the lanes' 16-byte accesses fall in distinct banks.
  static constexpr int SLOT = 4 * (ST | 1);
  static_assert(4 * ST <= ADJ_REC, "records fit the scratch share");
};

// Float offset of slot i inside a record plane of V vectors.
__device__ __forceinline__ int64_t rec_in_plane(int64_t i, int V) { return (i >> 2) * (16 * V) + (i & 3) * 4; }

template <int NT, bool STEP>
__device__ __forceinline__ void store_record(float* rec, const St<float, NT>& x) {
  constexpr int V = STEP ? Rec<NT>::ST : Rec<NT>::IN;
  float f[4 * V];
#pragma unroll
  for (int j = 0; j < 4; ++j) f[j] = x.q[j];
#pragma unroll
  for (int j = 0; j < 6; ++j) f[4 + j] = x.nu[j];
#pragma unroll
  for (int j = 0; j < NT; ++j) f[10 + j] = x.n[j];
#pragma unroll
  for (int j = 10 + NT; j < 4 * V; ++j) f[j] = (STEP && j < 13 + NT) ? x.p[(j - 10 - NT) % 3] : 0.0f;
  float4* r4 = reinterpret_cast<float4*>(rec);
#pragma unroll
  for (int k = 0; k < V; ++k) r4[4 * k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// Records of one segment buffer as the consumer lane sees them: record
// (tl, k) (step tl of the segment, substep k) starts at its plane, then the
// lane's slot inside it.
template <int NT>
struct RecSrc {
  const float* buf;
  int64_t step4, off_st, off_in;   // floats per vector plane; slot offsets in step / inner planes
  int K;
  __device__ __forceinline__ const float* at(int tl, int k) const {
    const int64_t plane = (int64_t)tl * (Rec<NT>::ST + (K - 1) * Rec<NT>::IN) +
                          (k ? Rec<NT>::ST + (k - 1) * Rec<NT>::IN : 0);
    return buf + plane * step4 + (k ? off_in : off_st);
  }
};

// Consumer-side prefetch slots of one lane: a ring of four records
// [4][ADJ_ENVS][Rec<NT>::SLOT] (record j in slot j % 4: while the reverse pass
// works on the substep between records j and j + 1, records j - 1 and j - 2
// stream in) and a ring of per-step data [ADJ_RING][ADJ_STEPF][ADJ_ENVS]
// (step t in slot t % ADJ_RING, issued two steps ahead). Every issue is its
// own cp.async group.
constexpr int ADJ_RING = 3;
constexpr int ADJ_RREC = 4;
template <int NT>
struct AdjPrefetch {
  float* rec;
  float* stp;
  int lane;
  __device__ __forceinline__ float* rslot(int j) const {
    return rec + ((j & (ADJ_RREC - 1)) * ADJ_ENVS + lane) * Rec<NT>::SLOT;
  }
  __device__ __forceinline__ float* sslot(int b) const { return stp + b * ADJ_STEPF * ADJ_ENVS + lane; }
  template <bool STEP>
  __device__ __forceinline__ void issue_rec(const float* src, int j) const {
    constexpr int V = STEP ? Rec<NT>::ST : Rec<NT>::IN;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(rslot(j));
#pragma unroll
    for (int k = 0; k < V; ++k) cp16_l2(dst + 16u * k, src + 16 * k);
    cp_commit();
  }
  // Record (tl, k), record j of the segment, into its slot.
  __device__ __forceinline__ void issue(const RecSrc<NT>& r, int tl, int k, int j) const {
    if (k == 0) issue_rec<true>(r.at(tl, 0), j);
    else issue_rec<false>(r.at(tl, k), j);
  }
  // Record j - 2, given record j = (tl, k).
  __device__ __forceinline__ void issue_back2(const RecSrc<NT>& r, int tl, int k, int j) const {
    if (j < 2) return;
    k -= 2;
    while (k < 0) { k += r.K; --tl; }
    issue(r, tl, k, j - 2);
  }
  // q, nu and n of record j (and p if P3, a step-boundary record).
  template <bool P3>
  __device__ __forceinline__ void read(int j, St<float, NT>& x) const {
    constexpr int V = P3 ? Rec<NT>::ST : Rec<NT>::IN;
    float f[4 * V];
    const float4* p = reinterpret_cast<const float4*>(rslot(j));
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float4 v = p[k];
      f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) x.q[i] = f[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) x.nu[i] = f[4 + i];
#pragma unroll
    for (int i = 0; i < NT; ++i) x.n[i] = f[10 + i];
    if constexpr (P3) {
#pragma unroll
      for (int i = 0; i < 3; ++i) x.p[i] = f[10 + NT + i];
    }
  }
  // q and nu of record j (the start of a substep).
  __device__ __forceinline__ void read_qnu(int j, St<float, NT>& x) const {
    const float4* p = reinterpret_cast<const float4*>(rslot(j));
    const float4 v0 = p[0], v1 = p[1], v2 = p[2];
    x.q[0] = v0.x; x.q[1] = v0.y; x.q[2] = v0.z; x.q[3] = v0.w;
    x.nu[0] = v1.x; x.nu[1] = v1.y; x.nu[2] = v1.z; x.nu[3] = v1.w;
    x.nu[4] = v2.x; x.nu[5] = v2.y;
  }
  // Step t's cotangents and actions into per-step slot b.
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

// Record planes of a segment buffer: record j = tl K + k (step tl of the
// segment, substep k) starts rec_plane(tl, k) vectors per slot into the
// buffer; a step spans ST + (K - 1) IN.
template <int NT>
__device__ __forceinline__ int64_t rec_plane(int tl, int k, int K) {
  return (int64_t)tl * (Rec<NT>::ST + (K - 1) * Rec<NT>::IN) + (k ? Rec<NT>::ST + (k - 1) * Rec<NT>::IN : 0);
}

// Reverse units: checkpoint segment s (steps [s c, (s + 1) c), c =
// ckpt_every) splits into units of unit_steps steps; unit q (in time order)
// covers steps [t0, t1) of segment s.
struct AdjUnit {
  int s, t0, t1;
};
__device__ __forceinline__ int adj_units(const AdjArgs& a) {
  const int c = a.ckpt_every, L = a.unit_steps;
  const int n_seg = (a.T + c - 1) / c, per_seg = (c + L - 1) / L;
  return (n_seg - 1) * per_seg + (a.T - (n_seg - 1) * c + L - 1) / L;
}
__device__ __forceinline__ AdjUnit adj_unit(const AdjArgs& a, int q) {
  const int c = a.ckpt_every, L = a.unit_steps, per_seg = (c + L - 1) / L;
  AdjUnit r;
  r.s = q / per_seg;
  const int u = q - r.s * per_seg;
  r.t0 = r.s * c + u * L;
  r.t1 = min(min(r.t0 + L, (r.s + 1) * c), a.T);
  return r;
}

// Producer: recompute unit `un` from its segment's checkpoint (steps before
// the unit without records) into the records of buffer `buf` (the states at
// every substep boundary of the unit).
template <int NT, bool PAY, int VAR, typename ActT, typename GenT>
__device__ __forceinline__ void adj_produce(const AdjArgs& a, const AdjSeg& sd, const ActT& A, const GenT& G,
                                            const Phys<float>& P, unsigned p_base, int64_t i, const AdjUnit& un,
                                            float* buf) {
  const int64_t ns = a.n_slots, slot = sd.slot_off + i;
  const int t0 = un.t0, t1 = un.t1;
  St<float, NT> x;
  ld21<NT>(a.ckpt + (int64_t)un.s * 21 * ns + slot, ns, x);
  const int64_t step4 = 4 * sd.n4;   // floats per vector plane
  float* rs = buf + rec_in_plane(i, Rec<NT>::ST);
  float* ri = buf + rec_in_plane(i, Rec<NT>::IN);
  int64_t plane = 0;                  // floats to the current record's plane
  for (int t = un.s * a.ckpt_every; t < t1; ++t) {
    float raw[NT], c[NT];
    load_actions<NT>(a.actions + (int64_t)t * a.act_stride + sd.act_off + i * NT, raw);
#pragma unroll
    for (int q = 0; q < NT; ++q) c[q] = clamp1(raw[q]);
    const bool rec = t >= t0;
    for (int k = 0; k < sd.K; ++k) {
      if (rec) {
        if (k == 0) {
          store_record<NT, true>(rs + plane, x);
          plane += Rec<NT>::ST * step4;
        } else {
          store_record<NT, false>(ri + plane, x);
          plane += Rec<NT>::IN * step4;
        }
      }
      if constexpr (VAR == 2) {
        if constexpr (PAY) {
          unsigned pb = p_base;
          asm volatile("" : "+r"(pb));
          substep_rk4<float, NT, ActT, AdjPhysPay, true, GenT>(x, c, AdjPhysPay(pb), A, sd.h, G);
        } else {
          substep_rk4<float, NT, ActT, Phys<float>, true, GenT>(x, c, P, A, sd.h, G);
        }
      } else if constexpr (PAY) {
        unsigned pb = p_base;
        asm volatile("" : "+r"(pb));
        substep<float, NT, false>(x, c, AdjPhysPay(pb), A, sd.h, nullptr);
      } else {
        substep<float, NT, false, ActT, Phys<float>, true, GenT>(x, c, P, A, sd.h, nullptr, G);
      }
    }
  }
  store_record<NT, true>(rs + plane, x);
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
  const int n_units = adj_units(a);
  // The class segment's two buffers (one reverse unit each), in its share of
  // the scratch.
  const int64_t buf_floats = rec_plane<NT>(a.unit_steps, 0, K) * 4 * sd.n4 + Rec<NT>::ST * 4 * sd.n4;
  float* const seg_scratch = a.scratch + (int64_t)2 * (a.ckpt_every * K + 1) * ADJ_REC * sd.slot_off;
  const int64_t step4 = 4 * sd.n4;
  const int64_t off_st = rec_in_plane(i, Rec<NT>::ST), off_in = rec_in_plane(i, Rec<NT>::IN);
  const float inv_h = 1.0f / sd.h;

  // Consumer state.
  St<float, NT> lam;
  HydroGrad<float> g;
  float4 tg = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float4 tr[3] = {tg, tg, tg};
  float k_start = 0.0f;
  AdjPrefetch<NT> pf{s_rec, s_step, lane};
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
    pf.issue_step(a, sd, i, a.T - 1, (a.T - 1) % ADJ_RING);
    if (a.T >= 2) pf.issue_step(a, sd, i, a.T - 2, (a.T - 2) % ADJ_RING);
  }
  float tgt[3] = {tg.x, tg.y, tg.z};

  for (int it = 0; it <= n_units; ++it) {
    if (role == 1 && it < n_units && valid)
      adj_produce<NT, PAY, VAR>(a, sd, A, G, P, p_base, i, adj_unit(a, n_units - 1 - it),
                                seg_scratch + (int64_t)(it & 1) * buf_floats);
    if (role == 0 && it >= 1 && valid) {
      const AdjUnit un = adj_unit(a, n_units - it);
      const int t0 = un.t0, t1 = un.t1;
      const RecSrc<NT> rsrc{seg_scratch + (int64_t)((it - 1) & 1) * buf_floats, step4, off_st, off_in, K};
      const int n = t1 - t0;
      int j = n * K;   // record of the segment's end state (j >= 1)
      pf.issue(rsrc, n, 0, j);
      if (K == 1) pf.issue(rsrc, n - 1, 0, j - 1);
      else pf.issue(rsrc, n - 1, K - 1, j - 1);
      cp_wait_but1();   // record j (record j - 1 was committed after it)
      for (int t = t1 - 1; t >= t0; --t) {
        const int tl = t - t0;
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
        if (t >= 2) pf.issue_step(a, sd, i, t - 2, (t - 2) % ADJ_RING);
        // State at the end of step t: record j (a step-boundary record).
        {
          St<float, NT> xe;
          pf.template read<true>(j, xe);
          // After reading record j, record j - 2 is issued (records j and
          // j - 1 were issued before): every record once, two ahead.
          if (t == t1 - 1) pf.issue_back2(rsrc, tl + 1, 0, j);
          if (sd.track) track_ref<float>(tg, tr[0], tr[1], tr[2], sd.dt, k_start + (float)(t + 1), tgt);
          observe_vjp<float, NT>(xe, c, tgt, a.g_obs ? go : nullptr, gr, lam, lc);
        }
        for (int k = K - 1; k >= 0; --k) {
          --j;
          // Record j: record j - 1 was committed after it, except for j = 0.
          if (j >= 1) cp_wait_but1();
          else cp_wait_all();
          // The substep from record j to record j + 1 (still in its slot).
          St<float, NT> x0, x1;
          pf.read_qnu(j, x0);
          pf.template read<false>(j + 1, x1);
          // Records j - 1 and j - 2 stream in while this substep's product runs.
          pf.issue_back2(rsrc, tl, k, j);
          if constexpr (VAR == 2) {
            // RK4: the stages are recomputed from the substep's start state,
            // with the new actuator states of its end.
#pragma unroll
            for (int q = 0; q < NT; ++q) x0.n[q] = x1.n[q];
            if constexpr (PAY) {
              unsigned pb = p_base;
              asm volatile("" : "+r"(pb));
              substep_rk4_vjp<float, NT, ActT, AdjPhysPay, true, GenT, true>(x0, c, AdjPhysPay(pb), A, sd.h, lam,
                                                                           lc, g, G);
            } else {
              substep_rk4_vjp<float, NT, ActT, Phys<float>, true, GenT, true>(x0, c, P, A, sd.h, lam, lc, g, G);
            }
          } else {
            Tape<float, NT> tp;
            if constexpr (PAY) {
              unsigned pb = p_base;
              asm volatile("" : "+r"(pb));
              const AdjPhysPay Pv(pb);
              tape_from_states<float, NT>(x0, x1, Pv, sd.h, inv_h, tp);
              vjp_from_tape<float, NT>(x0, x1.q, tp, c, Pv, A, sd.h, lam, lc, g);
            } else {
              tape_from_states<float, NT>(x0, x1, P, sd.h, inv_h, tp);
              vjp_from_tape<float, NT>(x0, x1.q, tp, c, P, A, sd.h, lam, lc, g, G);
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
    // The producer's records of this unit are complete and the consumer is
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
  __shared__ __align__(16) float s_rec[ADJ_RREC * ADJ_ENVS * Rec<NT>::SLOT];
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
    const AdjSeg sr{sd.act_off, sd.slot_off, sd.h, sd.dt, sd.K, sd.track, sd.n4};
    if constexpr (GEN) adjoint_env<NT, PAY, VAR>(a, sr, *kt, GenK{kp.g}, i, valid, s_rec, s_step, s_dyn);
    else adjoint_env<NT, PAY, VAR>(a, sr, *kt, NoGen{}, i, valid, s_rec, s_step, s_dyn);
  }
  // Completion stays ordered along the stream (see the step kernel).
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace mg
