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

__device__ __forceinline__ void phys_from_array(const float* v, Phys<float>& P) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    P.minv[j] = v[PAR_MINV + j]; P.A[j] = v[PAR_A + j]; P.dl[j] = v[PAR_DL + j]; P.dq[j] = v[PAR_DQ + j];
  }
  P.m = v[PAR_M];
#pragma unroll
  for (int j = 0; j < 3; ++j) { P.Ig[j] = v[PAR_IG + j]; P.rb[j] = v[PAR_RB + j]; P.Vc[j] = v[PAR_VC + j]; }
  P.W = v[PAR_W]; P.B = v[PAR_B];
}

// Segment of a tile: binary search over tile_begin (segments sorted).
__device__ __forceinline__ int find_seg(const SegDesc* segs, int n_segs, int tile) {
  int lo = 0, hi = n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&segs[mid].tile_begin) <= tile) lo = mid; else hi = mid - 1;
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
// instead of occupying registers across the substep loop; the loads are
// volatile so that they are not hoisted out of the loop.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float lds1(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds4(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}

// Actuator table in shared memory: alloc[6][8] | kf[8] | dz[8] | alpha[8].
struct ActSmem {
  unsigned base;
};
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
template <typename S, int NT>
__device__ __forceinline__ void act_row(const ActSmem& A, int k, S (&r)[NT]) {
  lds_vec<NT>(A.base + 4 * (SA_ALLOC + 8 * k), r);
}
template <typename S, int NT>
__device__ __forceinline__ void act_rotor(const ActSmem& A, S (&kf)[NT], S (&dz)[NT], S (&al)[NT]) {
  lds_vec<NT>(A.base + 4 * SA_KF, kf);
  lds_vec<NT>(A.base + 4 * SA_DZ, dz);
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

constexpr int STEP_BLK = 128;

// Cooperative store of the observation tile (nv4 envs x 13 floats, 16-byte
// aligned on both sides) from shared memory to global memory.
__device__ __forceinline__ void store_obs_tile(const float* s_obs, float* g_obs, int nv4) {
  const int n = nv4 * 13 / 4;
  const float4* src = reinterpret_cast<const float4*>(s_obs);
  float4* dst = reinterpret_cast<float4*>(g_obs);
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

template <int NT, bool PER_ENV>
__device__ __forceinline__ void step_tile(const StepArgs& a, const SegDesc& sd, int tile, const float* s_act,
                                          const float* s_phys, float* s_obs, float* s_par) {
  const int64_t local0 = (int64_t)(tile - sd.tile_begin) * STEP_BLK;
  const int64_t i = local0 + threadIdx.x;
  const bool valid = i < sd.n_envs;
  const bool in_storage = i < sd.n4;
  const int nv4 = (int)min((int64_t)STEP_BLK, (int64_t)sd.n4 - local0);
  const int64_t slot = sd.slot_off + i;
  float* st_base = a.state + sd.st_off;
  const ActSmem A{smem_addr(s_act)};

  St<float, NT> x;
  if (valid) {
    load_state<NT>(st_base, sd.n4, i, x);
    if (PER_ENV) {
#pragma unroll
      for (int k = 0; k < PAR_PLANES; ++k) {
        const float4 v = __ldg(&a.planes[k * a.n_slots + slot]);
        s_par[(4 * k + 0) * STEP_BLK + threadIdx.x] = v.x;
        s_par[(4 * k + 1) * STEP_BLK + threadIdx.x] = v.y;
        s_par[(4 * k + 2) * STEP_BLK + threadIdx.x] = v.z;
        s_par[(4 * k + 3) * STEP_BLK + threadIdx.x] = v.w;
      }
    }
  }
  // Each thread reads only its own parameter column: no barrier needed.
  using PV = PhysSmem<PER_ENV ? STEP_BLK : 1>;
  const PV P(PER_ENV ? smem_addr(s_par) + 4u * threadIdx.x : smem_addr(s_phys));
  float c[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) c[j] = 0.0f;
  const int n_out_steps = a.n_steps == 0 ? 1 : a.n_steps;
  for (int t = 0; t < n_out_steps; ++t) {
    if (valid && a.n_steps > 0) {
      if (a.act_mode == 0) {
        float raw[NT];
        load_actions<NT>(a.actions + t * a.act_stride + sd.act_off + i * NT, raw);
#pragma unroll
        for (int j = 0; j < NT; ++j) c[j] = clamp1(raw[j]);
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
      for (int k = 0; k < sd.K; ++k) substep<float, NT, false>(x, c, P, A, sd.h, nullptr);
    }
    const bool emit = a.obs_every || t == n_out_steps - 1;
    if (emit) {
      const int64_t out = a.obs_every ? t : 0;
      float o[13], r = 0.0f;
#pragma unroll
      for (int j = 0; j < 13; ++j) o[j] = 0.0f;
      if (valid) {
        const float4 tg = __ldg(&a.planes[(PER_ENV ? TGT_PLANE : 0) * a.n_slots + slot]);
        const float tgt[3] = {tg.x, tg.y, tg.z};
        observe<float, NT>(x, c, tgt, o, r);
      }
      if (a.obs) {
#pragma unroll
        for (int j = 0; j < 13; ++j) s_obs[threadIdx.x * 13 + j] = o[j];
        __syncthreads();
        store_obs_tile(s_obs, a.obs + (out * a.n_slots + sd.slot_off + local0) * 13, nv4);
        __syncthreads();
      }
      if (a.reward && in_storage) a.reward[out * a.n_slots + slot] = valid ? r : 0.0f;
      if (a.ret && valid && a.n_steps > 0) a.ret[slot] += r;
    }
  }
  if (valid && a.n_steps > 0) {
    store_state<NT>(st_base, sd.n4, i, x);
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
}

// Persistent-capable step kernel for envs with NT thrusters: each block walks
// tiles tile_lo + blockIdx.x, + gridDim.x, ... A tile is 128 envs of one
// segment. One instantiation per thruster count (and parameter source) keeps
// each kernel's register allocation to its own arithmetic.
template <int NT, bool PER_ENV>
__global__ void __launch_bounds__(STEP_BLK, 6) mg_step_kernel(const __grid_constant__ StepArgs a) {
  __shared__ __align__(16) float s_act[SA_DIM];
  __shared__ __align__(16) float s_phys[PAR_DIM];
  __shared__ __align__(16) float s_obs[STEP_BLK * 13];
  __shared__ __align__(16) float s_par[PER_ENV ? PAR_DIM * STEP_BLK : 4];
  for (int tt = blockIdx.x; tt < a.n_tiles; tt += gridDim.x) {
    const int tile = a.tile_lo + tt;
    const int si = a.seg_lo + find_seg(a.segs + a.seg_lo, a.seg_hi - a.seg_lo, tile);
    const SegDesc& sd = a.segs[si];
    __syncthreads();
    const ClassF& cf = a.classes[sd.cls];
    for (int k = threadIdx.x; k < SA_DIM + PAR_DIM; k += STEP_BLK) {
      if (k < 48) s_act[k] = cf.alloc[k / 8][k % 8];
      else if (k < 56) s_act[k] = cf.kf[k - 48];
      else if (k < 64) s_act[k] = cf.dz[k - 56];
      else if (k < 72) s_act[k] = sd.alpha[k - 64];
      else s_phys[k - 72] = cf.phys[k - 72];
    }
    __syncthreads();
    step_tile<NT, PER_ENV>(a, sd, tile, s_act, s_phys, s_obs, s_par);
  }
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
  if (a.init_mode == 1) {
    for (int j = 0; j < 3; ++j) tgt[j] = a.target_half * (2.0 * uniform53(seed, STREAM_INIT, id, j) - 1.0);
    const double rad = a.pos_radius * cbrt(uniform53(seed, STREAM_INIT, id, 3));
    const double zd = 2.0 * uniform53(seed, STREAM_INIT, id, 4) - 1.0;
    const double ph = 6.283185307179586 * uniform53(seed, STREAM_INIT, id, 5);
    const double rd = sqrt(1.0 - zd * zd);
    f[0] = tgt[0] + rad * rd * cos(ph);
    f[1] = tgt[1] + rad * rd * sin(ph);
    f[2] = tgt[2] + rad * zd;
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
  a.planes[(a.per_env ? TGT_PLANE : 0) * a.n_slots + slot] =
      make_float4((float)tgt[0], (float)tgt[1], (float)tgt[2], 0.0f);
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
  const float tgt[3] = {tg.x, tg.y, tg.z};
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

template <int NT>
__global__ void __launch_bounds__(128) mg_adjoint_kernel(const __grid_constant__ AdjArgs a) {
  __shared__ Act<float> act;
  if ((int)blockIdx.x >= a.n_tiles) return;
  const int tile = a.tile_lo + blockIdx.x;
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
  const int64_t i = (int64_t)(tile - sd.tile_begin) * blockDim.x + threadIdx.x;
  if (i >= sd.n_envs) {
    // Padding slots of the segment: zero gradients.
    if (i < sd.n4) {
      const int64_t slot = sd.slot_off + i;
      if (a.g_A) for (int j = 0; j < 6; ++j) a.g_A[slot * 6 + j] = 0.0f;
      if (a.g_D) for (int j = 0; j < 12; ++j) a.g_D[slot * 12 + j] = 0.0f;
      if (a.g_state0) for (int j = 0; j < 21; ++j) a.g_state0[slot * 21 + j] = 0.0f;
    }
    return;
  }
  const volatile Act<float>& va = act;
  adjoint_env<NT>(a, sd, va, i);
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
  const double tgt[3] = {tg.x, tg.y, tg.z};
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

cudaError_t launch_step(const StepArgs& a, int nt, int grid, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (a.per_env) {
#define MG_L(N) mg_step_kernel<N, true><<<grid, STEP_BLK, 0, st>>>(a)
    MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  } else {
#define MG_L(N) mg_step_kernel<N, false><<<grid, STEP_BLK, 0, st>>>(a)
    MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  }
  return cudaGetLastError();
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

cudaError_t launch_adjoint(const AdjArgs& a, int nt, int block, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
#define MG_L(N) mg_adjoint_kernel<N><<<a.n_tiles, block, 0, st>>>(a)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaGetLastError();
}

cudaError_t launch_fp64(const Fp64Args& a, int nt, int block, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
#define MG_L(N) mg_fp64_kernel<N><<<a.n_tiles, block, 0, st>>>(a)
  MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  return cudaGetLastError();
}

cudaError_t step_kernel_occupancy(int nt, bool per_env, int* blocks_per_sm) {
  if (per_env) {
#define MG_L(N) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mg_step_kernel<N, true>, STEP_BLK, 0)
    MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  } else {
#define MG_L(N) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mg_step_kernel<N, false>, STEP_BLK, 0)
    MG_NT_SWITCH(nt, MG_L)
#undef MG_L
  }
  return cudaErrorInvalidValue;
}

}  // namespace mg
