// CUDA kernels of libmarinegym for sm_103a (B300) other than the step kernel
// (mg_step.cuh): reset with domain randomisation, set_hydro, the adjoint and
// the FP64 check path, and the launch dispatchers the runtime calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "marinegym.h"
#include "mg_internal.h"
#include "mg_device.cuh"
#include "mg_payload.h"
#include "mg_step.cuh"

namespace mg {

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
// Adjoint of a recorded rollout: a block of two warps per 32 envs, one launch
// per class with the class tables as the kernel parameter (constant-bank
// operands in the vector-Jacobian product).
//
// The reverse pass walks the checkpoint segments from the last to the first.
// Warp 1 (the producer) recomputes segment s - 1 from its checkpoint while
// warp 0 (the consumer) runs the vector-Jacobian products of segment s, so
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
#define MG_ADJ_ENVS 32
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
// [ADJ_RING][32][ADJ_REC] (record j in slot j % ADJ_RING: while the reverse
// pass works on record j, records j - 1 and j - 2 stream in) and a ring of
// per-step data [ADJ_RING][ADJ_STEPF][32] (step t in slot t % ADJ_RING,
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
template <int NT, typename ActT>
__device__ __forceinline__ void adj_produce(const AdjArgs& a, const AdjSeg& sd, const ActT& A, const Phys<float>& P,
                                            int64_t i, int s, float* buf) {
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
      Tape<float, NT> tp;
      substep<float, NT, true>(x, c, P, A, sd.h, &tp);
      store_record<NT>(rec, x0, tp.rhs);
      rec += rstride;
    }
  }
  store_record<NT>(rec, x, nullptr);
}

template <int NT, typename ActT>
__device__ __forceinline__ void adjoint_env(const AdjArgs& a, const AdjSeg& sd, const ActT& A, int64_t i, bool valid,
                                            float* s_rec, float* s_step) {
  const int role = threadIdx.x / ADJ_ENVS;   // 0: reverse pass, 1: forward recompute
  const int lane = threadIdx.x % ADJ_ENVS;
  const int64_t slot = sd.slot_off + i;
  const int64_t ns = a.n_slots;
  Phys<float> P;
  if (valid) load_phys(a.planes, ns, slot, P);
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
      adj_produce<NT>(a, sd, A, P, i, n_seg - 1 - it, a.scratch + (int64_t)(it & 1) * buf_floats);
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
          Tape<float, NT> tp;
          tape_from_rhs<float, NT>(xs, c, P, A, sd.h, rhs, tp, q1);
          vjp_from_tape<float, NT>(xs, q1, tp, c, P, A, sd.h, lam, lc, g);
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

// One block of two warps per 32 envs of a class segment (one segment per
// launch): a few thousand envs (the adjoint workload) then spread over all
// SMs. The launches of a backward pass are programmatic dependents of one
// another (disjoint envs and outputs) so that they run side by side.
template <int NT>
__global__ void __launch_bounds__(ADJ_THREADS)
    mg_adjoint_kernel(const __grid_constant__ AdjArgs a, const __grid_constant__ ClassK kc) {
  __shared__ __align__(16) float s_rec[ADJ_RING * ADJ_ENVS * ADJ_REC];
  __shared__ __align__(16) float s_step[ADJ_RING * ADJ_STEPF * ADJ_ENVS];
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
    adjoint_env<NT>(a, sr, kc, i, valid, s_rec, s_step);
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

// Adjoint launch of one class segment (a.seg_hi == a.seg_lo + 1; tiles of
// a.tile_envs envs, a multiple of ADJ_ENVS) with that class's tables kc;
// `dependent`: programmatic dependent of the previous launch.
template <int NT>
static cudaError_t launch_adjoint_t(const AdjArgs& a, const ClassK& kc, bool dependent, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_tiles * (a.tile_envs / ADJ_ENVS)));
  cfg.blockDim = dim3(ADJ_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (MG_USE_PDL && dependent) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, mg_adjoint_kernel<NT>, a, kc);
}

cudaError_t launch_adjoint(const AdjArgs& a, const ClassK& kc, int nt, bool dependent, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (a.tile_envs <= 0 || a.tile_envs % ADJ_ENVS != 0 || a.seg_hi - a.seg_lo != 1) return cudaErrorInvalidValue;
#define MG_L(N) return launch_adjoint_t<N>(a, kc, dependent, st)
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

cudaError_t launch_step_pm0(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                            bool dependent, bool shared_sm, cudaStream_t st);
cudaError_t launch_step_pm1(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                            bool dependent, bool shared_sm, cudaStream_t st);
cudaError_t launch_step_pm2(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                            bool dependent, bool shared_sm, cudaStream_t st);
cudaError_t occupancy_pm0(int nt, int var, bool kp, bool track, int* blocks_per_sm);
cudaError_t occupancy_pm1(int nt, int var, bool kp, bool track, int* blocks_per_sm);
cudaError_t occupancy_pm2(int nt, int var, bool kp, bool track, int* blocks_per_sm);

// Step launch of one class group: thruster count nt, parameter source
// a.per_env (0 class, 1 per-env, 2 payload), variant var (0 propellers with
// Euler, 1 generic actuators with Euler, 2 RK4). kc (launches whose segments
// are all of one class, else null): that class's constants, and kg its
// generic actuator table (var >= 1), passed as the kernel parameter.
cudaError_t launch_step(const StepArgs& a, const ClassK* kc, const ClassG* kg, int nt, int var, int grid,
                        bool dependent, bool shared_sm, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (kc && a.seg_hi - a.seg_lo != 1) return cudaErrorInvalidValue;   // one class, one segment
  switch (a.per_env) {
    case 0: return launch_step_pm0(a, kc, kg, nt, var, grid, dependent, shared_sm, st);
    case 1: return launch_step_pm1(a, kc, kg, nt, var, grid, dependent, shared_sm, st);
    case 2: return launch_step_pm2(a, kc, kg, nt, var, grid, dependent, shared_sm, st);
    default: return cudaErrorInvalidValue;
  }
}

// Dynamic shared memory of the step kernels of thruster count nt and
// parameter source pm (the run-time compiled kernels use the same layout).
size_t step_kernel_smem(int nt, int pm, bool track) {
#define MG_S(N)                                     \
  case N:                                           \
    return pm == 0 ? step_smem<N, 0>(track)         \
                   : (pm == 1 ? step_smem<N, 1>(track) : step_smem<N, 2>(track));
  switch (nt) {
    MG_S(1) MG_S(2) MG_S(3) MG_S(4) MG_S(5) MG_S(6) MG_S(7) MG_S(8)
    default: return 0;
  }
#undef MG_S
}

// Resident blocks per SM of a step instantiation (kp: class tables as the
// kernel parameter).
cudaError_t step_kernel_occupancy(int nt, int pm, int var, bool kp, bool track, int* blocks_per_sm) {
  switch (pm) {
    case 0: return occupancy_pm0(nt, var, kp, track, blocks_per_sm);
    case 1: return occupancy_pm1(nt, var, kp, track, blocks_per_sm);
    case 2: return occupancy_pm2(nt, var, kp, track, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mg
