// Lane-pair step kernel of libmarinegym for sm_103a (B300): two lanes per
// environment, for launches that are latency bound (every tile of the launch
// resident at once, at most one warp per scheduler with one env per thread).
//
// The equation of motion splits by momentum: the even lane of a pair owns the
// linear rows (forces, v), the odd lane the angular rows (moments, w). Both
// lanes hold the whole state; each computes its three rows of the wrench
// B f (Sec. III-D), its half of Eq. 1-3
//   linear : tau_l - w x (m v + A_l v_r) - A_l o (w x v_c) - D_l(v_r) + (W - B) e
//   angular: tau_a - w x (I w + A_a w)   - v_r x (A_l v_r) - D_a(w)   - (B r_b) x e
// and its half of the velocity update, then the pair swaps the new halves
// (one shuffle per component) and both lanes advance the pose. Both halves
// are written as one instruction stream with lane-dependent operands,
//   rhs = tau_h - w x (M1 o s1 + M2 o s2) - P o (y x z) - (dl + dq o |u|) o u + y2 x e + alpha e,
// so the warp never diverges. A warp advances 16 envs; per lane the substep
// is about 60% of the one-lane instruction count, and twice as many warps
// share the schedulers, hiding each other's dependency latency.
//
// Scope: propeller classes with the semi-implicit Euler substep, class
// tables as the kernel parameter (one class per launch), class-constant
// (PM = 0) or per-env (PM = 1) parameters, hover observation and reward
// after every step or after the last, actions from memory, and the
// checkpoints of a recorded rollout. Other launches use the one-lane kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "marinegym.h"
#include "mg_internal.h"
#include "mg_device.cuh"

namespace mg {

constexpr int PAIR_BLK = 128;             // threads per block
constexpr int PAIR_ENVS = PAIR_BLK / 2;   // envs per block
constexpr int PAIR_TILE = 128;            // envs per tile of the segment layout

template <int NT>
__device__ __forceinline__ void pair_load_state(const float* base, int64_t n4, int64_t i, St<float, NT>& x) {
  constexpr int SS = 13 + NT, NF4 = SS / 4, REM = SS % 4;
  float f[SS];
  const float4* p4 = reinterpret_cast<const float4*>(base);
#pragma unroll
  for (int k = 0; k < NF4; ++k) {
    const float4 v = p4[k * n4 + i];
    f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
  }
  const float* pr = base + (int64_t)NF4 * 4 * n4;
#pragma unroll
  for (int r = 0; r < REM; ++r) f[(NF4 * 4 + r) % SS] = pr[r * n4 + i];
#pragma unroll
  for (int j = 0; j < 3; ++j) x.p[j] = f[j];
#pragma unroll
  for (int j = 0; j < 4; ++j) x.q[j] = f[3 + j];
#pragma unroll
  for (int j = 0; j < 6; ++j) x.nu[j] = f[7 + j];
#pragma unroll
  for (int j = 0; j < NT; ++j) x.n[j] = f[13 + j];
}

template <int NT>
__device__ __forceinline__ void pair_store_state(float* base, int64_t n4, int64_t i, const St<float, NT>& x) {
  constexpr int SS = 13 + NT, NF4 = SS / 4, REM = SS % 4;
  float f[SS];
#pragma unroll
  for (int j = 0; j < 3; ++j) f[j] = x.p[j];
#pragma unroll
  for (int j = 0; j < 4; ++j) f[3 + j] = x.q[j];
#pragma unroll
  for (int j = 0; j < 6; ++j) f[7 + j] = x.nu[j];
#pragma unroll
  for (int j = 0; j < NT; ++j) f[13 + j] = x.n[j];
  float4* p4 = reinterpret_cast<float4*>(base);
#pragma unroll
  for (int k = 0; k < NF4; ++k) p4[k * n4 + i] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
  float* pr = base + (int64_t)NF4 * 4 * n4;
#pragma unroll
  for (int r = 0; r < REM; ++r) pr[r * n4 + i] = f[(NF4 * 4 + r) % SS];
}

__device__ __forceinline__ float pclamp(float a) { return a < -1.0f ? -1.0f : (a > 1.0f ? 1.0f : a); }

template <int NT>
__device__ __forceinline__ void pair_actions(const float* src, float (&c)[NT]) {
#pragma unroll
  for (int j = 0; j < NT; ++j) c[j] = __ldg(src + j);
}

// The lane's half of the parameters: rows 3h..3h+2 of everything that is
// per row, and the operands of the uniform half-rhs above.
template <int NT>
struct PairHalf {
  float rows[3][NT];   // allocation rows (times k for class-constant launches)
  float hminv[3];      // h * M^-1 of the lane's rows
  float M1[3], M2[3];  // b = M1 o s1 + M2 o s2
  float P[3];          // X = P o (y x z)
  float dl[3], dq[3];  // damping of the lane's rows
  float y2[3], alpha;  // restoring: y2 x e + alpha e
  float Al[3];         // linear added mass (both lanes: a1 = A_l o v_r)
  float Vc[3];         // current (NED)
};

// PM: 0 class constants from kc; 1 per-env planes. PRE: the host's rows
// carry k (class-constant launches); per-env launches multiply their rows by
// k here, once, so that every launch's substep takes f = n|n|.
template <int NT, int PM, bool CURRENT>
__global__ void __launch_bounds__(PAIR_BLK, 1)
    mg_pair_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ ClassK kc) {
  constexpr bool PRE = PM == 0 && MG_PREMUL;
  if (a.wait_first) asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int hsel = lane & 1;   // 0: linear lane, 1: angular lane
  const SegDesc& sd = a.segs[a.seg_lo];
  const int tile = a.tile_lo + (int)(blockIdx.x >> 1);
  const int64_t i = (int64_t)(tile - sd.tile_begin) * PAIR_TILE + (int64_t)(blockIdx.x & 1) * PAIR_ENVS +
                    warp * 16 + (lane >> 1);
  const bool valid = (int)(blockIdx.x >> 1) < a.n_tiles && i < sd.n_envs;
  const bool in_storage = (int)(blockIdx.x >> 1) < a.n_tiles && i < sd.n4;
  const int64_t slot = sd.slot_off + i;
  float* st_base = a.state + sd.st_off;
  const float h = sd.h;
  // Per-step fields in registers (a reference into global memory would be
  // read again after every observation store).
  const int K = sd.K;
  const int64_t n4 = sd.n4;
  const float* act_env = a.actions + sd.act_off + i * NT;

  // Parameters of this lane's half.
  PairHalf<NT> Q;
  float m, Ig[3], A6[6], dl6[6], dq6[6], minv6[6], W, Bf, rb[3];
  float4 tg = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  Q.Vc[0] = Q.Vc[1] = Q.Vc[2] = 0.0f;
  if constexpr (PM == 1) {
    float v[36];
#pragma unroll
    for (int k = 0; k < PAR_PLANES; ++k) {
      const float4 p = valid ? __ldg(&a.planes[k * a.n_slots + slot]) : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
      v[4 * k] = p.x; v[4 * k + 1] = p.y; v[4 * k + 2] = p.z; v[4 * k + 3] = p.w;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) { minv6[j] = v[PAR_MINV + j]; A6[j] = v[PAR_A + j]; dl6[j] = v[PAR_DL + j]; dq6[j] = v[PAR_DQ + j]; }
    m = v[PAR_M];
#pragma unroll
    for (int j = 0; j < 3; ++j) { Ig[j] = v[PAR_IG + j]; rb[j] = v[PAR_RB + j]; Q.Vc[j] = v[PAR_VC + j]; }
    W = v[PAR_W];
    Bf = v[PAR_B];
    if (valid) tg = __ldg(&a.planes[TGT_PLANE * a.n_slots + slot]);
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) { minv6[j] = kc.minv[j]; A6[j] = kc.A[j]; dl6[j] = kc.dl[j]; dq6[j] = kc.dq[j]; }
    m = kc.m;
#pragma unroll
    for (int j = 0; j < 3; ++j) { Ig[j] = kc.Ig[j]; rb[j] = kc.rb[j]; }
    W = kc.W;
    Bf = kc.B;
    if (valid) tg = __ldg(&a.planes[slot]);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int q = 0; q < NT; ++q)
      Q.rows[j][q] = (hsel ? kc.alloc[3 + j][q] : kc.alloc[j][q]) * (PRE ? 1.0f : kc.kf[q]);
    Q.hminv[j] = h * (hsel ? minv6[3 + j] : minv6[j]);
    Q.M1[j] = hsel ? Ig[j] : m;
    Q.M2[j] = hsel ? A6[3 + j] : A6[j];
    Q.P[j] = hsel ? 1.0f : A6[j];
    Q.dl[j] = hsel ? dl6[3 + j] : dl6[j];
    Q.dq[j] = hsel ? dq6[3 + j] : dq6[j];
    Q.y2[j] = hsel ? -(Bf * rb[j]) : 0.0f;
    Q.Al[j] = A6[j];
  }
  Q.alpha = hsel ? 0.0f : W - Bf;

  St<float, NT> x;
#pragma unroll
  for (int j = 0; j < 3; ++j) x.p[j] = 0.0f;
  x.q[0] = 1.0f; x.q[1] = x.q[2] = x.q[3] = 0.0f;
#pragma unroll
  for (int j = 0; j < 6; ++j) x.nu[j] = 0.0f;
#pragma unroll
  for (int j = 0; j < NT; ++j) x.n[j] = 0.0f;
  if (valid) pair_load_state<NT>(st_base, n4, i, x);
  const float tgt[3] = {tg.x, tg.y, tg.z};

  float c[NT], cn[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) c[j] = cn[j] = 0.0f;
  if (valid) pair_actions<NT>(act_env, cn);
  float r_last = 0.0f;
  for (int t = 0; t < a.n_steps; ++t) {
    if (a.ckpt && (t % a.ckpt_every) == 0 && valid && hsel == 0) {
      // Recorded rollout: the state before step t into checkpoint t / ckpt_every.
      float* ck = a.ckpt + (int64_t)(t / a.ckpt_every) * 21 * a.n_slots + slot;
#pragma unroll
      for (int j = 0; j < 3; ++j) ck[j * a.n_slots] = x.p[j];
#pragma unroll
      for (int j = 0; j < 4; ++j) ck[(3 + j) * a.n_slots] = x.q[j];
#pragma unroll
      for (int j = 0; j < 6; ++j) ck[(7 + j) * a.n_slots] = x.nu[j];
#pragma unroll
      for (int j = 0; j < 8; ++j) ck[(13 + j) * a.n_slots] = j < NT ? x.n[j % NT] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) c[j] = pclamp(cn[j]);
    // The next step's actions are in flight while this step computes.
    if (valid && t + 1 < a.n_steps) pair_actions<NT>(act_env + (int64_t)(t + 1) * a.act_stride, cn);
    for (int k = 0; k < K; ++k) {
      // a1 + a2: every rotor in both lanes; the lane's three wrench rows.
      float f[NT];
      if (kc.dz_on) {
#pragma unroll
        for (int q = 0; q < NT; ++q) {
          x.n[q] = x.n[q] + kc.alpha[q] * (c[q] - x.n[q]);
          const float an = fabsf(x.n[q]);
          f[q] = (an < kc.dz[q]) ? 0.0f : x.n[q] * an;
        }
      } else {
#pragma unroll
        for (int q = 0; q < NT; ++q) {
          x.n[q] = x.n[q] + kc.alpha[q] * (c[q] - x.n[q]);
          f[q] = x.n[q] * fabsf(x.n[q]);
        }
      }
      float tau[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float s = Q.rows[j][0] * f[0];
#pragma unroll
        for (int q = 1; q < NT; ++q) s = s + Q.rows[j][q] * f[q];
        tau[j] = s;
      }
      // a3
      float R[3][3];
      rot(x.q, R);
      const float v[3] = {x.nu[0], x.nu[1], x.nu[2]};
      const float w[3] = {x.nu[3], x.nu[4], x.nu[5]};
      float vc[3], vr[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        vc[j] = CURRENT ? R[0][j] * Q.Vc[0] + R[1][j] * Q.Vc[1] + R[2][j] * Q.Vc[2] : 0.0f;
        vr[j] = CURRENT ? v[j] - vc[j] : v[j];
      }
      // a4-a7, the lane's half.
      float a1[3], b[3], wxb[3], y[3], z[3], yz[3], u[3], e[3], ye[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        a1[j] = Q.Al[j] * vr[j];
        const float s1 = hsel ? w[j] : v[j];
        const float s2 = hsel ? w[j] : vr[j];
        b[j] = Q.M1[j] * s1 + Q.M2[j] * s2;
        y[j] = hsel ? vr[j] : w[j];
        z[j] = hsel ? a1[j] : vc[j];
        u[j] = hsel ? w[j] : vr[j];
        e[j] = R[2][j];
      }
      cross3(w, b, wxb);
      cross3(y, z, yz);
      cross3(Q.y2, e, ye);
      float half[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float dmp = (Q.dl[j] + Q.dq[j] * fabsf(u[j])) * u[j];
        const float rhs = tau[j] - wxb[j] - Q.P[j] * yz[j] - dmp + (ye[j] + Q.alpha * e[j]);
        half[j] = (hsel ? w[j] : v[j]) + Q.hminv[j] * rhs;
      }
      // a8: swap the new halves, then both lanes advance the pose.
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float other = __shfl_xor_sync(0xffffffffu, half[j], 1);
        x.nu[j] = hsel ? other : half[j];
        x.nu[3 + j] = hsel ? half[j] : other;
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) x.p[j] = x.p[j] + h * (R[j][0] * x.nu[0] + R[j][1] * x.nu[1] + R[j][2] * x.nu[2]);
      const float hh = 0.5f * h;
      const float wn[3] = {x.nu[3], x.nu[4], x.nu[5]};
      float qd[4], qn[4];
      quat_rate(x.q, wn, qd);
#pragma unroll
      for (int j = 0; j < 4; ++j) qn[j] = x.q[j] + hh * qd[j];
      const float inv = minvsqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j) x.q[j] = qn[j] * inv;
    }
    const bool emit = a.obs_every || t == a.n_steps - 1;
    if (emit) {
      const int64_t out = a.obs_every ? t : 0;
      float o[13], r = 0.0f;
#pragma unroll
      for (int j = 0; j < 13; ++j) o[j] = 0.0f;
      if (valid) {
        observe<float, NT>(x, c, tgt, o, r);
        r_last = r;
      }
      if (a.obs && in_storage) {
        float* dst = a.obs + (out * a.n_slots + slot) * 13;
        // Even lane: entries 0..6; odd lane: 7..12.
#pragma unroll
        for (int j = 0; j < 7; ++j) {
          const int col = hsel ? 7 + j : j;
          if (col < 13) dst[col] = hsel ? o[(7 + j) % 13] : o[j];
        }
      }
      if (a.reward && in_storage && hsel == 0) a.reward[out * a.n_slots + slot] = valid ? r : 0.0f;
    }
  }
  if (valid && hsel == 0 && a.n_steps > 0) {
    pair_store_state<NT>(st_base, n4, i, x);
    // Finite exactly when the last reward (p, nu, c) and q, n are.
    float s = r_last;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += x.q[j];
#pragma unroll
    for (int j = 0; j < NT; ++j) s += x.n[j];
    if (!isfinite(s)) atomicOr(a.status, 1u);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int NT, int PM, bool CURRENT>
static cudaError_t launch_pair_t(const StepArgs& a, const ClassK& kc, bool dependent, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * a.n_tiles));
  cfg.blockDim = dim3(PAIR_BLK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (MG_USE_PDL && dependent) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, mg_pair_kernel<NT, PM, CURRENT>, a, kc);
}

// Lane-pair launch of one class segment (a.seg_hi == a.seg_lo + 1): 2 blocks
// of 64 envs per 128-env tile, every block resident at once. Refuses what the
// kernel does not cover.
cudaError_t launch_pair(const StepArgs& a, const ClassK& kc, int nt, bool dependent, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (a.seg_hi - a.seg_lo != 1 || a.act_mode != 0 || a.track || a.ret || a.n_steps < 1 ||
      (a.per_env != 0 && a.per_env != 1))
    return cudaErrorInvalidValue;
#define MG_P(N)                                                                              \
  return a.per_env ? launch_pair_t<N, 1, true>(a, kc, dependent, st)                         \
                   : launch_pair_t<N, 0, false>(a, kc, dependent, st)
  switch (nt) {
    case 1: MG_P(1);
    case 2: MG_P(2);
    case 3: MG_P(3);
    case 4: MG_P(4);
    case 5: MG_P(5);
    case 6: MG_P(6);
    case 7: MG_P(7);
    case 8: MG_P(8);
    default: return cudaErrorInvalidValue;
  }
#undef MG_P
}

}  // namespace mg
