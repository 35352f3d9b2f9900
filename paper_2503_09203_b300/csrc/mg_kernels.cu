// CUDA kernels of libmarinegym for sm_103a (B300) other than the step kernel
// (mg_step.cuh): reset with domain randomisation, set_hydro, the adjoint and
// the FP64 check path, and the launch dispatchers the runtime calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>

#include "marinegym.h"
#include "mg_internal.h"
#include "mg_device.cuh"
#include "mg_adjoint.cuh"
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
// FP64 rollout for finite-difference checks (one env per thread).
// ---------------------------------------------------------------------------

// A class's generic actuator table in FP64 (fins, tilted propellers).
struct GenD {
  const ClassGD& g;
  __device__ __forceinline__ int kind(int i) const { return g.kind[i]; }
  __device__ __forceinline__ double v(int i, int k) const { return g.v[i][k]; }
};

// The combined body of a payload run in FP64 (the members the full-inertia
// step reads): recomputed per env from the vehicle's parameters, the
// perturbed added mass and the payload, so that a finite difference in the
// added mass moves the full inverse.
struct PhysPayD {
  static constexpr bool kFull = true;
  double A[6], dl[6], dq[6], B, rb[3], Vc[3], Mi[21], Io[6], s[3], m, W;
};

// VAR: 0 propellers with Euler, 1 generic actuators with Euler, 2 RK4.
// PAY: payload runs.
template <int NT, int VAR, bool PAY>
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
  PhysPayD Q;
  if constexpr (PAY) {
    // Payload mass and position: plane PAY_MP / 4 of the payload block.
    const float4 pv = __ldg(&a.planes[(int64_t)(a.pay_plane + PAY_MP / 4) * ns + slot]);
    const double mp = pv.x, rp[3] = {pv.y, pv.z, pv.w};
    double mt, sv[3], Io[3][3], Wt, Mi[6][6];
    payload_body(P.m, P.Ig, P.A, P.W, mp, rp, &mt, sv, Io, &Wt, Mi);
    for (int j = 0; j < 6; ++j) { Q.A[j] = P.A[j]; Q.dl[j] = P.dl[j]; Q.dq[j] = P.dq[j]; }
    Q.B = P.B;
    for (int j = 0; j < 3; ++j) { Q.rb[j] = P.rb[j]; Q.Vc[j] = P.Vc[j]; Q.s[j] = sv[j]; }
    int q = 0;
    for (int r = 0; r < 6; ++r)
      for (int c = r; c < 6; ++c) Q.Mi[q++] = 0.5 * (Mi[r][c] + Mi[c][r]);
    Q.Io[0] = Io[0][0]; Q.Io[1] = Io[0][1]; Q.Io[2] = Io[0][2];
    Q.Io[3] = Io[1][1]; Q.Io[4] = Io[1][2]; Q.Io[5] = Io[2][2];
    Q.m = mt;
    Q.W = Wt;
  }
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
  auto sub = [&](const auto& PP, const double (&c)[NT]) {
    using PT = tt::decay_t<decltype(PP)>;
    if constexpr (VAR == 2)
      substep_rk4<double, NT, Act<double>, PT, true, GenD>(x, c, PP, A, a.h, GenD{a.gen[sd.cls]});
    else if constexpr (VAR == 1)
      substep<double, NT, false, Act<double>, PT, true, GenD>(x, c, PP, A, a.h, nullptr, GenD{a.gen[sd.cls]});
    else
      substep<double, NT, false>(x, c, PP, A, a.h, nullptr);
  };
  for (int t = 0; t < a.T; ++t) {
    float raw[NT];
    load_actions<NT>(a.actions + t * a.act_stride + sd.act_off + i * NT, raw);
    double c[NT];
    for (int q = 0; q < NT; ++q) c[q] = raw[q] < -1.0f ? -1.0 : (raw[q] > 1.0f ? 1.0 : (double)raw[q]);
    for (int k = 0; k < sd.K; ++k) {
      if constexpr (PAY) sub(Q, c);
      else sub(P, c);
    }
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

template <int NT, int VAR, bool PAY>
__global__ void __launch_bounds__(128) mg_fp64_kernel(const __grid_constant__ Fp64Args a) {
  if ((int)blockIdx.x >= a.n_tiles) return;
  const int tile = a.tile_lo + blockIdx.x;
  const int si = a.seg_lo + find_seg(a.segs + a.seg_lo, a.seg_hi - a.seg_lo, tile);
  const SegDesc& sd = a.segs[si];
  const int64_t i = (int64_t)(tile - sd.tile_begin) * blockDim.x + threadIdx.x;
  if (i >= sd.n_envs) return;
  fp64_env<NT, VAR, PAY>(a, sd, i);
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
// `dependent`: programmatic dependent of the previous launch; kern: the
// kernel (the library's, or one compiled at run time for this class).
static cudaError_t launch_adjoint_k(const void* kern, const AdjArgs& a, const ClassK& kc, const ClassG* kg,
                                    bool dependent, cudaStream_t st, size_t dyn_smem = 0) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_tiles * (a.tile_envs / ADJ_ENVS)));
  cfg.blockDim = dim3(ADJ_THREADS);
  cfg.dynamicSmemBytes = dyn_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (MG_USE_PDL && dependent) ? 1 : 0;
  AdjArgs aa = a;
  ClassKG kk;
  kk.k = kc;
  if (kg) kk.g = *kg;
  void* args[] = {&aa, kg ? static_cast<void*>(&kk) : static_cast<void*>(&kk.k)};
  return cudaLaunchKernelExC(&cfg, kern, args);
}

// var: 0 propeller classes with Euler, 1 classes with fins or tilted
// propellers with Euler, 2 RK4 runs; kg: the class's generic actuator table
// (var >= 1), else null. jit_kernel: a class-specialised adjoint kernel for
// nt thrusters compiled at run time (var 0 without a payload; null: the
// library's).
template <bool PAY, int VAR>
static const void* adjoint_fn(int nt) {
  switch (nt) {
    case 1: return reinterpret_cast<const void*>(&mg_adjoint_kernel<1, PAY, NoLit, VAR>);
    case 2: return reinterpret_cast<const void*>(&mg_adjoint_kernel<2, PAY, NoLit, VAR>);
    case 3: return reinterpret_cast<const void*>(&mg_adjoint_kernel<3, PAY, NoLit, VAR>);
    case 4: return reinterpret_cast<const void*>(&mg_adjoint_kernel<4, PAY, NoLit, VAR>);
    case 5: return reinterpret_cast<const void*>(&mg_adjoint_kernel<5, PAY, NoLit, VAR>);
    case 6: return reinterpret_cast<const void*>(&mg_adjoint_kernel<6, PAY, NoLit, VAR>);
    case 7: return reinterpret_cast<const void*>(&mg_adjoint_kernel<7, PAY, NoLit, VAR>);
    case 8: return reinterpret_cast<const void*>(&mg_adjoint_kernel<8, PAY, NoLit, VAR>);
    default: return nullptr;
  }
}

cudaError_t launch_adjoint(const AdjArgs& a, const ClassK& kc, const ClassG* kg, int nt, int var, bool dependent,
                           cudaStream_t st, const void* jit_kernel) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (a.tile_envs <= 0 || a.tile_envs % ADJ_ENVS != 0 || a.seg_hi - a.seg_lo != 1) return cudaErrorInvalidValue;
  if (var < 0 || var > 2 || (var != 0 && !kg)) return cudaErrorInvalidValue;
  const bool pay = a.pay_plane > 0;
  if (pay && var == 1) return cudaErrorInvalidValue;   // payload runs are propeller classes
  if (jit_kernel && var == 0 && !pay) return launch_adjoint_k(jit_kernel, a, kc, nullptr, dependent, st);
  const void* k = pay ? (var == 2 ? adjoint_fn<true, 2>(nt) : adjoint_fn<true, 0>(nt))
                      : (var == 2 ? adjoint_fn<false, 2>(nt) : var == 1 ? adjoint_fn<false, 1>(nt)
                                                                          : adjoint_fn<false, 0>(nt));
  if (!k) return cudaErrorInvalidValue;
  if (pay) {
    // Payload runs: the parameter column in dynamic shared memory (above the
    // default 48 KB with the static part: the attribute is set once per
    // device and kernel).
    static std::atomic<uint32_t> attr_set[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
    const uint32_t bit = 1u << (nt + (var == 2 ? 9 : 0));
    if (dev >= 0 && dev < 64 && !(attr_set[dev].load() & bit)) {
      const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, ADJ_PAY_SMEM);
      if (e != cudaSuccess) return e;
      attr_set[dev].fetch_or(bit);
    }
    return launch_adjoint_k(k, a, kc, var ? kg : nullptr, dependent, st, ADJ_PAY_SMEM);
  }
  return launch_adjoint_k(k, a, kc, var ? kg : nullptr, dependent, st);
}

// FP64 launch of one group: var 0 propellers with Euler, 1 generic
// actuators with Euler, 2 RK4; a.pay_plane > 0: payload run.
template <int VAR, bool PAY>
static cudaError_t launch_fp64_t(const Fp64Args& a, int nt, int block, cudaStream_t st) {
#define MG_L(N) mg_fp64_kernel<N, VAR, PAY><<<a.n_tiles, block, 0, st>>>(a)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaGetLastError();
}

cudaError_t launch_fp64(const Fp64Args& a, int nt, int var, int block, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  const bool pay = a.pay_plane > 0;
  if (var == 0) return pay ? launch_fp64_t<0, true>(a, nt, block, st) : launch_fp64_t<0, false>(a, nt, block, st);
  if (var == 1) return pay ? launch_fp64_t<1, true>(a, nt, block, st) : launch_fp64_t<1, false>(a, nt, block, st);
  if (var == 2) return pay ? launch_fp64_t<2, true>(a, nt, block, st) : launch_fp64_t<2, false>(a, nt, block, st);
  return cudaErrorInvalidValue;
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

// Dynamic shared memory of the class-specialised step kernels (compiled at
// run time with the observation tile aliased into the stage buffer: two
// stage buffers per warp, no trajectory section; per-env parameters (pm 1)
// add their shared-memory columns).
size_t step_kernel_smem_jit(int nt, int pm) {
  const size_t cols = pm == 1 ? sizeof(float) * PAR_DIM * STEP_BLK : 0;
#define MG_S(N) \
  case N: return cols + sizeof(float) * N_WARPS * 2 * (size_t)Stage<N>::floats(false);
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
