// Per-environment step arithmetic of the batched UUV simulator, templated on
// the scalar (float for the hot kernels, double for the FP64 check path, a
// counting type on the host for the FLOP count) and on the thruster count.
//
// One substep (h = dt/K) of the discrete map, in the order a1..a8:
//   a1 rotor lag      n <- n + alpha (c - n)                 (Sec. III-D)
//   a2 thrust/alloc   f_i = k_i n_i |n_i| (0 in dead zone), tau = B f; generic
//                     tables add fins (lift/drag) and servo-tilted propellers
//   a3 kinematics     R(q), v_c = R^T V_c, v_r = v - v_c     (Sec. III-B, current)
//   a4 C_RB(nu) nu  = [m w x v ; w x (I_g w)]                 (Eq. 2, r_g = 0)
//   a5 C_A(nu_r)nu_r= [w x a1 ; v_r x a1 + w x a2], a1 = A_lin v_r, a2 = A_ang w,
//      plus the current-acceleration term M_A [w x v_c ; 0]  (Eq. 3 with nu_r)
//   a6 D(nu_r)nu_r  = d_l o nu_r + d_q o |nu_r| o nu_r
//   a7 g(q)         = [-(W-B) e ; B r_b x e], e = R^T e_3    (Eq. 1-2, r_g = 0)
//   a8 nu += h M^-1 (tau - a4 - a5 - a6 - a7); p += h R v; q <- |q + h/2 q(x)(0,w)|
//      (or the RK4 variant over a3-a8 with the actuator states held)
// The hover observation / reward (Sec. IV-B station keeping) and the exact
// vector-Jacobian products of both are here too.
#pragma once

#include "mg_rtc.h"

#define MG_HD __host__ __device__ __forceinline__

// Build switches of the hot path (0/1).
#ifndef MG_FAST_RSQRT
#define MG_FAST_RSQRT 1
#endif
#ifndef MG_USE_PDL
#define MG_USE_PDL 1
#endif

namespace mg {

MG_HD float mabs(float x) { return fabsf(x); }
MG_HD double mabs(double x) { return fabs(x); }
MG_HD float msqrt(float x) { return sqrtf(x); }
MG_HD double msqrt(double x) { return sqrt(x); }
// Reciprocal norm used to renormalise the quaternion. FP32: the hardware
// reciprocal square root (about 2 ulp), exactly 1 for an exactly unit input so
// that a vehicle at rest stays bit-identical; FP64: correctly rounded.
MG_HD float minvsqrt(float x) {
#if defined(__CUDA_ARCH__) && MG_FAST_RSQRT
  return x == 1.0f ? 1.0f : rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
MG_HD double minvsqrt(double x) { return 1.0 / sqrt(x); }
MG_HD float msin(float x) { return sinf(x); }
MG_HD double msin(double x) { return sin(x); }

// Reference point of the trajectory-tracking task at step counter k:
// p*(t) = c + a o sin(w t + phi) + v t, t = k dt. `c` is the target plane
// (centre; its w lane holds the counter), tr0..tr2 the three trajectory planes
// (a_x a_y a_z w_x | w_y w_z phi_x phi_y | phi_z v_x v_y v_z).
template <typename S>
MG_HD void track_ref(float4 c, float4 tr0, float4 tr1, float4 tr2, S dt, S k, S out[3]) {
  const S t = k * dt;
  const S a[3] = {S(tr0.x), S(tr0.y), S(tr0.z)};
  const S w[3] = {S(tr0.w), S(tr1.x), S(tr1.y)};
  const S ph[3] = {S(tr1.z), S(tr1.w), S(tr2.x)};
  const S v[3] = {S(tr2.y), S(tr2.z), S(tr2.w)};
  const S cc[3] = {S(c.x), S(c.y), S(c.z)};
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = cc[i] + a[i] * msin(w[i] * t + ph[i]) + v[i] * t;
}

// Actuator table of one (class, substep length).
template <typename S>
struct Act {
  S alloc[6][8];  // B = [d_i ; r_i x d_i]
  S kf[8];
  S dz[8];
  S alpha[8];
};

// Per-env physical parameters (device block of 36 floats in this order).
template <typename S>
struct Phys {
  static constexpr bool kFull = false;   // diagonal inertia, CoG at the origin
  S minv[6], A[6], dl[6], dq[6];
  S m, Ig[3], W, B, rb[3], Vc[3];
};

// Index of entry (i, j), i <= j, of a symmetric 6x6 matrix stored as its upper
// triangle row by row (21 entries).
MG_HD constexpr int sym6(int i, int j) { return i * 6 - (i * (i - 1)) / 2 + (j - i); }

template <typename S, int NT>
struct St {
  S p[3], q[4], nu[6], n[NT];
};

template <typename S>
struct HydroGrad {
  S A[6], dl[6], dq[6];
};

template <typename S>
MG_HD void cross3(const S a[3], const S b[3], S o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename S>
MG_HD void rot(const S q[4], S R[3][3]) {
  // Products with the doubled components: each off-diagonal entry is one sum
  // and each diagonal entry two fused multiply-adds.
  const S w = q[0], x = q[1], y = q[2], z = q[3];
  const S one = S(1.0f);
  const S x2 = x + x, y2 = y + y, z2 = z + z;
  const S xy = x * y2, xz = x * z2, yz = y * z2, wx = w * x2, wy = w * y2, wz = w * z2;
  R[0][0] = one - y * y2 - z * z2;
  R[0][1] = xy - wz;
  R[0][2] = xz + wy;
  R[1][0] = xy + wz;
  R[1][1] = one - x * x2 - z * z2;
  R[1][2] = yz - wx;
  R[2][0] = xz - wy;
  R[2][1] = yz + wx;
  R[2][2] = one - x * x2 - y * y2;
}

// Actuator-table access: row k of the allocation matrix, and the thrust
// constant, dead zone and rotor factor vectors. Generic versions index the
// arrays of an Act<S> (or a volatile view of one); the hot kernel supplies
// overloads for its shared-memory view that use vector loads.
template <typename S, int NT, typename ActT>
MG_HD void act_row(const ActT& A, int k, S (&r)[NT]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) r[i] = S(A.alloc[k][i]);
}
template <typename S, int NT, typename ActT>
MG_HD void act_rotor(const ActT& A, S (&kf)[NT], S (&dz)[NT], S (&al)[NT]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) { kf[i] = S(A.kf[i]); dz[i] = S(A.dz[i]); al[i] = S(A.alpha[i]); }
}
template <typename S, int NT, typename ActT>
MG_HD void act_rotor_nodz(const ActT& A, S (&kf)[NT], S (&al)[NT]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) { kf[i] = S(A.kf[i]); al[i] = S(A.alpha[i]); }
}


// Intermediates of one substep kept for the vector-Jacobian product.
// nd: the velocity rate M^-1 rhs of a4-a7.
template <typename S, int NT>
struct Tape {
  S n1[NT], R[3][3], vc[3], vr[3], w[3], nd[6], nu1[6], qn[4], inv;
};

// Actuator kinds (Sec. III-D): propeller with a fixed direction (its column
// of the allocation matrix), servo (no force), fin, propeller tilted by a servo.
enum { KIND_PROP = 0, KIND_SERVO = 1, KIND_FIN = 2, KIND_TILT = 3 };

// No generic actuators: every channel is a fixed propeller.
struct NoGen {};

// Per-channel values of a generic actuator table (20 floats per channel):
// fin  : e1 = chord at zero deflection (0..2), e2 = a x e1 (3..5), r x e1
//        (6..8), r x e2 (9..11), kL = rho S C_L_alpha / 2 (12), kD0 (13),
//        kDa (14), deflection range (15);
// tilt : B0 = [d ; r x d] (0..5), B1 = [a x d ; r x (a x d)] (6..11),
//        B2 = (a . d) [a ; r x a] (12..17), servo channel (18), its range (19).
enum { GEN_VALS = 20 };

MG_HD void msincos(float x, float* s, float* c) {
#if defined(__CUDA_ARCH__)
  sincosf(x, s, c);
#else
  *s = sinf(x); *c = cosf(x);
#endif
}
MG_HD void msincos(double x, double* s, double* c) { *s = sin(x); *c = cos(x); }

// a1 + a2: actuator states (rotor speed or servo / fin angle, first-order
// lag), propeller thrust f = k n|n| (0 in the dead zone; k = 0 for servos and
// fins) and the fixed-direction part of the wrench tau = B f.
// Whether the actuator table may hold a nonzero dead zone (the hot kernel's
// shared-memory view knows per class; other tables are always tested).
template <typename ActT>
MG_HD bool dz_active(const ActT&) { return true; }

// Whether a table's allocation rows already carry the thrust constants
// (rows of B diag(k)): then f below is n|n| and tau = (B diag(k)) f.
template <typename ActT>
struct ActPremul {
  static constexpr bool value = false;
};

// LAG = false: x.n already holds the new actuator states (the adjoint takes
// them from the recorded end state of the substep).
template <typename S, int NT, typename ActT, bool LAG = true>
MG_HD void actuate(St<S, NT>& x, const S (&c)[NT], const ActT& A, S (&f)[NT], S tau[6]) {
  constexpr bool PRE = ActPremul<ActT>::value;
  if (dz_active(A)) {
    S kf[NT], dz[NT], al[NT];
    act_rotor<S, NT>(A, kf, dz, al);
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      if (LAG) x.n[i] = x.n[i] + al[i] * (c[i] - x.n[i]);
      const S an = mabs(x.n[i]);
      f[i] = (an < dz[i]) ? S(0.0f) : (PRE ? x.n[i] * an : kf[i] * x.n[i] * an);
    }
  } else {
    // No dead zone in this class: |n| < 0 never holds.
    S kf[NT], al[NT];
    act_rotor_nodz<S, NT>(A, kf, al);
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      if (LAG) x.n[i] = x.n[i] + al[i] * (c[i] - x.n[i]);
      f[i] = PRE ? x.n[i] * mabs(x.n[i]) : kf[i] * x.n[i] * mabs(x.n[i]);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    S r[NT];
    act_row<S, NT>(A, k, r);
    S s = r[0] * f[0];
#pragma unroll
    for (int i = 1; i < NT; ++i) s = s + r[i] * f[i];
    tau[k] = s;
  }
}

// Wrench of the propellers tilted by servos (depends on the actuator states only):
// f_i [cos th B0 + sin th B1 + (1 - cos th) B2], th = n_servo * range (Rodrigues).
template <typename S, int NT, typename GenT>
MG_HD void tilt_wrench(const GenT& G, const S (&n)[NT], const S (&f)[NT], S tau[6]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    if (G.kind(i) != KIND_TILT) continue;
    const int link = (int)G.v(i, 18);
    S nl = S(0.0f);
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j == link) nl = n[j];
    S sn, cs;
    msincos(nl * S(G.v(i, 19)), &sn, &cs);
    const S omc = S(1.0f) - cs;
#pragma unroll
    for (int k = 0; k < 6; ++k) tau[k] = tau[k] + f[i] * (cs * S(G.v(i, k)) + sn * S(G.v(i, 6 + k)) + omc * S(G.v(i, 12 + k)));
  }
}

// Wrench of the fins. With x = u . e1, y = u . e2 the components of the fin's
// velocity through the water u = v_r + w x r in the plane normal to the span,
// deflection th, u_c = cos th x + sin th y (along the chord), u_n = cos th y -
// sin th x (along the fin normal) and U^2 = x^2 + y^2: lift
// -kL (u_n u_c / U) (a x u) = kL g (y e1 - x e2), g = u_n u_c / U, and drag
// -(kD0 U + kDa u_n^2 / U) u (the lift and drag of C_L = C_L_alpha sin a cos a,
// C_D = C_D0 + C_D_alpha sin^2 a at angle of attack a, written in x and y).
template <typename S, int NT, typename GenT>
MG_HD void fin_wrench(const GenT& G, const S (&n)[NT], const S vr[3], const S w[3], S tau[6]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    if (G.kind(i) != KIND_FIN) continue;
    S e1[3], e2[3], re1[3], re2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e1[k] = S(G.v(i, k)); e2[k] = S(G.v(i, 3 + k)); re1[k] = S(G.v(i, 6 + k)); re2[k] = S(G.v(i, 9 + k));
    }
    const S xx = vr[0] * e1[0] + vr[1] * e1[1] + vr[2] * e1[2] + w[0] * re1[0] + w[1] * re1[1] + w[2] * re1[2];
    const S yy = vr[0] * e2[0] + vr[1] * e2[1] + vr[2] * e2[2] + w[0] * re2[0] + w[1] * re2[1] + w[2] * re2[2];
    const S U2 = xx * xx + yy * yy;
    if (!(U2 > S(0.0f))) continue;
    S sn, cs;
    msincos(n[i] * S(G.v(i, 15)), &sn, &cs);
    const S uc = cs * xx + sn * yy, un = cs * yy - sn * xx;
    const S iU = minvsqrt(U2);
    const S U = U2 * iU;
    const S g = un * uc * iU;
    const S kL = S(G.v(i, 12)), D = S(G.v(i, 13)) * U + S(G.v(i, 14)) * un * un * iU;
    const S F1 = kL * g * yy - D * xx, F2 = -(kL * g * xx) - D * yy;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      tau[k] = tau[k] + F1 * e1[k] + F2 * e2[k];
      tau[3 + k] = tau[3 + k] + F1 * re1[k] + F2 * re2[k];
    }
  }
}

// Vector-Jacobian products of the two generic wrenches (the tilt wrench
// depends on the thrusts f and the servo states, the fin wrench on the fin
// states and the fin velocities u = v_r + w x r). ltau is the adjoint of the
// wrench; lf and ln (per channel) and lvr, lw accumulate.
template <typename S, int NT, typename GenT>
MG_HD void tilt_wrench_vjp(const GenT& G, const S (&n)[NT], const S (&f)[NT], const S ltau[6], S (&lf)[NT],
                           S (&ln)[NT]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    if (G.kind(i) != KIND_TILT) continue;
    const int link = (int)G.v(i, 18);
    S nl = S(0.0f);
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j == link) nl = n[j];
    const S rng = S(G.v(i, 19));
    S sn, cs;
    msincos(nl * rng, &sn, &cs);
    const S omc = S(1.0f) - cs;
    S dir = S(0.0f), dth = S(0.0f);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const S b0 = S(G.v(i, k)), b1 = S(G.v(i, 6 + k)), b2 = S(G.v(i, 12 + k));
      dir = dir + ltau[k] * (cs * b0 + sn * b1 + omc * b2);
      dth = dth + ltau[k] * (-sn * b0 + cs * b1 + sn * b2);
    }
    lf[i] = lf[i] + dir;
    const S lnl = f[i] * dth * rng;
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j == link) ln[j] = ln[j] + lnl;
  }
}

template <typename S, int NT, typename GenT>
MG_HD void fin_wrench_vjp(const GenT& G, const S (&n)[NT], const S vr[3], const S w[3], const S ltau[6],
                          S (&ln)[NT], S lvr[3], S lw[3]) {
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    if (G.kind(i) != KIND_FIN) continue;
    S e1[3], e2[3], re1[3], re2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e1[k] = S(G.v(i, k)); e2[k] = S(G.v(i, 3 + k)); re1[k] = S(G.v(i, 6 + k)); re2[k] = S(G.v(i, 9 + k));
    }
    const S xx = vr[0] * e1[0] + vr[1] * e1[1] + vr[2] * e1[2] + w[0] * re1[0] + w[1] * re1[1] + w[2] * re1[2];
    const S yy = vr[0] * e2[0] + vr[1] * e2[1] + vr[2] * e2[2] + w[0] * re2[0] + w[1] * re2[1] + w[2] * re2[2];
    const S U2 = xx * xx + yy * yy;
    if (!(U2 > S(0.0f))) continue;
    const S rng = S(G.v(i, 15));
    S sn, cs;
    msincos(n[i] * rng, &sn, &cs);
    const S uc = cs * xx + sn * yy, un = cs * yy - sn * xx;
    const S iU = minvsqrt(U2);
    const S U = U2 * iU;
    const S g = un * uc * iU;
    const S kL = S(G.v(i, 12)), kD0 = S(G.v(i, 13)), kDa = S(G.v(i, 14));
    const S D = kD0 * U + kDa * un * un * iU;
    // F1 = kL g yy - D xx, F2 = -kL g xx - D yy; tau += F1 [e1; r x e1] + F2 [e2; r x e2].
    S lF1 = S(0.0f), lF2 = S(0.0f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lF1 = lF1 + ltau[k] * e1[k] + ltau[3 + k] * re1[k];
      lF2 = lF2 + ltau[k] * e2[k] + ltau[3 + k] * re2[k];
    }
    const S lg = kL * (lF1 * yy - lF2 * xx);
    const S lD = -(lF1 * xx + lF2 * yy);
    S lxx = -kL * g * lF2 - D * lF1;
    S lyy = kL * g * lF1 - D * lF2;
    // D = kD0 U + kDa un^2 iU ; g = un uc iU ; U = U2 iU ; iU = U2^-1/2
    S lU = kD0 * lD;
    S lun = S(2.0f) * kDa * un * iU * lD + uc * iU * lg;
    S liU = kDa * un * un * lD + un * uc * lg;
    const S luc = un * iU * lg;
    S lU2 = iU * lU;
    liU = liU + U2 * lU;
    lU2 = lU2 - S(0.5f) * iU * iU * iU * liU;
    // uc = cs xx + sn yy, un = cs yy - sn xx, th = n rng
    lxx = lxx + cs * luc - sn * lun + S(2.0f) * xx * lU2;
    lyy = lyy + sn * luc + cs * lun + S(2.0f) * yy * lU2;
    const S lth = un * luc - uc * lun;
    ln[i] = ln[i] + lth * rng;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lvr[k] = lvr[k] + e1[k] * lxx + e2[k] * lyy;
      lw[k] = lw[k] + re1[k] * lxx + re2[k] * lyy;
    }
  }
}

// a3: body-frame current v_c = R^T V_c and relative velocity v_r = v - v_c.
template <typename S, typename PhysT, bool CURRENT>
MG_HD void rel_velocity(const S R[3][3], const S v[3], const PhysT& P, S vc[3], S vr[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    vc[j] = CURRENT ? R[0][j] * S(P.Vc[0]) + R[1][j] * S(P.Vc[1]) + R[2][j] * S(P.Vc[2]) : S(0.0f);
    vr[j] = CURRENT ? v[j] - vc[j] : v[j];
  }
}

// a4-a7: rhs = tau - C_RB(nu) nu - C_A(nu_r) nu_r - M_A [w x v_c ; 0] - D(nu_r) nu_r - g(q).
template <typename S, typename PhysT, bool CURRENT>
MG_HD void body_rhs(const S R[3][3], const S v[3], const S w[3], const S vc[3], const S vr[3], const S tau[6],
                    const PhysT& P, S rhs[6]) {
  // a4. With a payload (PhysT::kFull) the body origin is not the CoG: with the
  // first moment s = m' r_g and the inertia I_o about the origin,
  // C_RB(nu) nu = [m' w x v + w x (w x s) ; w x (I_o w) + s x (w x v)].
  S Iw[3];
  if constexpr (PhysT::kFull) {
    Iw[0] = S(P.Io[0]) * w[0] + S(P.Io[1]) * w[1] + S(P.Io[2]) * w[2];
    Iw[1] = S(P.Io[1]) * w[0] + S(P.Io[3]) * w[1] + S(P.Io[4]) * w[2];
    Iw[2] = S(P.Io[2]) * w[0] + S(P.Io[4]) * w[1] + S(P.Io[5]) * w[2];
  } else {
    Iw[0] = S(P.Ig[0]) * w[0]; Iw[1] = S(P.Ig[1]) * w[1]; Iw[2] = S(P.Ig[2]) * w[2];
  }
  // a5: a1 = A_lin v_r, a2 = A_ang w. The terms with w on the left share one
  // cross product each: m w x v + w x a1 = w x (m v + a1) (linear) and
  // w x (I w) + w x a2 = w x (I w + a2) (angular); v_r x a1 stays apart.
  S a1[3], bl[3], ba[3], wxbl[3], wxba[3], vrxa1[3], wxvc[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    a1[j] = S(P.A[j]) * vr[j];
    bl[j] = S(P.m) * v[j] + a1[j];
    ba[j] = S(P.A[3 + j]) * w[j] + Iw[j];
  }
  cross3(w, bl, wxbl);
  cross3(w, ba, wxba);
  cross3(vr, a1, vrxa1);
  if (CURRENT) {
    cross3(w, vc, wxvc);
  } else {
    wxvc[0] = wxvc[1] = wxvc[2] = S(0.0f);
  }
  // a6 (nu_r = [v_r ; w])
  S dmp[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dmp[j] = (S(P.dl[j]) + S(P.dq[j]) * mabs(vr[j])) * vr[j];
    dmp[3 + j] = (S(P.dl[3 + j]) + S(P.dq[3 + j]) * mabs(w[j])) * w[j];
  }
  // a7: e = R^T e_3 is the third row of R.
  const S e[3] = {R[2][0], R[2][1], R[2][2]};
  const S Pw = S(P.W), Pb = S(P.B);
  const S WmB = Pw - Pb;
  S Brb[3] = {Pb * S(P.rb[0]), Pb * S(P.rb[1]), Pb * S(P.rb[2])}, mb[3];
  S extra_lin[3] = {S(0.0f), S(0.0f), S(0.0f)}, extra_ang[3] = {S(0.0f), S(0.0f), S(0.0f)};
  if constexpr (PhysT::kFull) {
    // Weight acts at r_g: the moment arm is B r_b - W r_g = B r_b - (W/m') s.
    const S sv[3] = {S(P.s[0]), S(P.s[1]), S(P.s[2])};
    const S wpm = Pw / S(P.m);
#pragma unroll
    for (int j = 0; j < 3; ++j) Brb[j] = Brb[j] - wpm * sv[j];
    S wxv[3], wxs[3], wxwxs[3], sxwxv[3];
    cross3(w, v, wxv);
    cross3(w, sv, wxs);
    cross3(w, wxs, wxwxs);
    cross3(sv, wxv, sxwxv);
#pragma unroll
    for (int j = 0; j < 3; ++j) { extra_lin[j] = wxwxs[j]; extra_ang[j] = sxwxv[j]; }
  }
  cross3(Brb, e, mb);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    rhs[j] = CURRENT ? tau[j] - wxbl[j] - S(P.A[j]) * wxvc[j] - dmp[j] + WmB * e[j]
                     : tau[j] - wxbl[j] - dmp[j] + WmB * e[j];
    rhs[3 + j] = tau[3 + j] - wxba[j] - vrxa1[j] - dmp[3 + j] - mb[j];
    if constexpr (PhysT::kFull) {
      rhs[j] = rhs[j] - extra_lin[j];
      rhs[3 + j] = rhs[3 + j] - extra_ang[j];
    }
  }
}

// a8 (first half): nu_dot = M^-1 rhs (diagonal, or the full symmetric inverse).
template <typename S, typename PhysT>
MG_HD void apply_minv(const PhysT& P, const S rhs[6], S nd[6]) {
  if constexpr (PhysT::kFull) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      S acc = S(0.0f);
#pragma unroll
      for (int j = 0; j < 6; ++j) acc = acc + S(P.Mi[i <= j ? sym6(i, j) : sym6(j, i)]) * rhs[j];
      nd[i] = acc;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) nd[j] = S(P.minv[j]) * rhs[j];
  }
}

// q (x) (0, w) for the quaternion kinematics q_dot = 1/2 q (x) (0, w).
template <typename S>
MG_HD void quat_rate(const S q[4], const S w[3], S qd[4]) {
  qd[0] = -q[1] * w[0] - q[2] * w[1] - q[3] * w[2];
  qd[1] = q[0] * w[0] + q[2] * w[2] - q[3] * w[1];
  qd[2] = q[0] * w[1] - q[1] * w[2] + q[3] * w[0];
  qd[3] = q[0] * w[2] + q[1] * w[1] - q[2] * w[0];
}

// a1-a8. `x` is updated in place; `c` is the clamped command (zero-order hold).
// `A` is an Act<S> or a volatile view of one in shared memory (a volatile view
// keeps the class table in shared memory instead of hoisting it into registers).
// `P` is a Phys<S> or a view with the same members (arrays minv, A, dl, dq,
// Ig, rb, Vc and scalars m, W, B) that reads shared memory on use.
// CURRENT = false compiles the ocean-current terms out (parameter sources
// whose current is zero by construction). `G` is NoGen (propellers only) or a
// generic actuator table (fins, servo-tilted propellers).
template <typename S, int NT, bool TAPE, typename ActT, typename PhysT, bool CURRENT = true,
          typename GenT = NoGen>
MG_HD void substep(St<S, NT>& x, const S (&c)[NT], const PhysT& P, const ActT& A, S h,
                   Tape<S, NT>* tp, const GenT& G = GenT()) {
  constexpr bool GEN = !tt::is_same<GenT, NoGen>::value;
  S f[NT], tau[6];
  actuate<S, NT>(x, c, A, f, tau);
  if constexpr (GEN) tilt_wrench<S, NT>(G, x.n, f, tau);
  // a3
  S R[3][3];
  rot(x.q, R);
  const S v[3] = {x.nu[0], x.nu[1], x.nu[2]};
  const S w[3] = {x.nu[3], x.nu[4], x.nu[5]};
  S vc[3], vr[3];
  rel_velocity<S, PhysT, CURRENT>(R, v, P, vc, vr);
  if constexpr (GEN) fin_wrench<S, NT>(G, x.n, vr, w, tau);
  S rhs[6];
  body_rhs<S, PhysT, CURRENT>(R, v, w, vc, vr, tau, P, rhs);
  if constexpr (PhysT::kFull) {
    S nd[6];
    apply_minv<S>(P, rhs, nd);
#pragma unroll
    for (int j = 0; j < 6; ++j) x.nu[j] = x.nu[j] + h * nd[j];
    if (TAPE) {
#pragma unroll
      for (int j = 0; j < 6; ++j) tp->nd[j] = nd[j];
    }
  } else {
    if (TAPE) {
#pragma unroll
      for (int j = 0; j < 6; ++j) tp->nd[j] = S(P.minv[j]) * rhs[j];
    }
    // Diagonal M^-1: nu += (h M^-1_jj) rhs_j; h M^-1 is the same for every
    // substep of the step loop, so the compiler can keep it in registers.
#pragma unroll
    for (int j = 0; j < 6; ++j) x.nu[j] = x.nu[j] + (h * S(P.minv[j])) * rhs[j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    x.p[i] = x.p[i] + h * (R[i][0] * x.nu[0] + R[i][1] * x.nu[1] + R[i][2] * x.nu[2]);
  const S hh = S(0.5f) * h;
  const S wn[3] = {x.nu[3], x.nu[4], x.nu[5]};
  S qd[4], qn[4];
  quat_rate(x.q, wn, qd);
#pragma unroll
  for (int i = 0; i < 4; ++i) qn[i] = x.q[i] + hh * qd[i];
  const S inv = minvsqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] = qn[i] * inv;
  if (TAPE) {
#pragma unroll
    for (int i = 0; i < NT; ++i) tp->n1[i] = x.n[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      tp->vc[i] = vc[i]; tp->vr[i] = vr[i]; tp->w[i] = w[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) tp->R[i][j] = R[i][j];
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) tp->nu1[j] = x.nu[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) tp->qn[i] = qn[i];
    tp->inv = inv;
  }
}

// Time derivative of (p, q, nu) for the RK4 variant, with the actuator states
// and the state-independent part of the actuator wrench (tau_n) held over the
// substep; the attitude of a stage is that of its normalised quaternion.
template <typename S, int NT, typename PhysT, bool CURRENT, typename GenT>
MG_HD void rk4_stage(const S q[4], const S nu[6], const S (&n)[NT], const S tau_n[6], const PhysT& P,
                     const GenT& G, S dp[3], S dq[4], S dnu[6]) {
  constexpr bool GEN = !tt::is_same<GenT, NoGen>::value;
  const S iq = minvsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const S qh[4] = {q[0] * iq, q[1] * iq, q[2] * iq, q[3] * iq};
  S R[3][3];
  rot(qh, R);
  const S v[3] = {nu[0], nu[1], nu[2]};
  const S w[3] = {nu[3], nu[4], nu[5]};
  S vc[3], vr[3], tau[6];
  rel_velocity<S, PhysT, CURRENT>(R, v, P, vc, vr);
#pragma unroll
  for (int k = 0; k < 6; ++k) tau[k] = tau_n[k];
  if constexpr (GEN) fin_wrench<S, NT>(G, n, vr, w, tau);
  S rhs[6];
  body_rhs<S, PhysT, CURRENT>(R, v, w, vc, vr, tau, P, rhs);
  apply_minv<S>(P, rhs, dnu);
#pragma unroll
  for (int i = 0; i < 3; ++i) dp[i] = R[i][0] * v[0] + R[i][1] * v[1] + R[i][2] * v[2];
  S qd[4];
  quat_rate(q, w, qd);
#pragma unroll
  for (int i = 0; i < 4; ++i) dq[i] = S(0.5f) * qd[i];
}

// One substep of the classical fourth-order Runge-Kutta variant: actuator
// states first (as a1), then RK4 on (p, q, nu) over h with them held, then q
// normalised. Stage sums are accumulated in place to bound register use.
template <typename S, int NT, typename ActT, typename PhysT, bool CURRENT = true, typename GenT = NoGen>
MG_HD void substep_rk4(St<S, NT>& x, const S (&c)[NT], const PhysT& P, const ActT& A, S h,
                       const GenT& G = GenT()) {
  constexpr bool GEN = !tt::is_same<GenT, NoGen>::value;
  S f[NT], tau_n[6];
  actuate<S, NT>(x, c, A, f, tau_n);
  if constexpr (GEN) tilt_wrench<S, NT>(G, x.n, f, tau_n);
  S q0[4], nu0[6];
#pragma unroll
  for (int i = 0; i < 4; ++i) q0[i] = x.q[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) nu0[i] = x.nu[i];
  // x holds the running sum y0 + h/6 (k1 + 2 k2 + 2 k3 + k4); ys the stage point.
  S ys_q[4], ys_nu[6], dp[3], dq[4], dnu[6];
  const S h2 = S(0.5f) * h, h6 = h / S(6.0f), h3 = h / S(3.0f);
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    if (st == 0) {
      rk4_stage<S, NT, PhysT, CURRENT>(q0, nu0, x.n, tau_n, P, G, dp, dq, dnu);
    } else {
      rk4_stage<S, NT, PhysT, CURRENT>(ys_q, ys_nu, x.n, tau_n, P, G, dp, dq, dnu);
    }
    const S wsum = (st == 0 || st == 3) ? h6 : h3;
    const S hs = (st == 2) ? h : h2;   // step to the next stage point
#pragma unroll
    for (int i = 0; i < 3; ++i) x.p[i] = x.p[i] + wsum * dp[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) { x.q[i] = x.q[i] + wsum * dq[i]; ys_q[i] = q0[i] + hs * dq[i]; }
#pragma unroll
    for (int i = 0; i < 6; ++i) { x.nu[i] = x.nu[i] + wsum * dnu[i]; ys_nu[i] = nu0[i] + hs * dnu[i]; }
  }
  const S inv = minvsqrt(x.q[0] * x.q[0] + x.q[1] * x.q[1] + x.q[2] * x.q[2] + x.q[3] * x.q[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) x.q[i] = x.q[i] * inv;
}

// Hover observation and reward after a control step.
template <typename S, int NT>
MG_HD void observe(const St<S, NT>& x, const S (&c)[NT], const S tgt[3], S obs[13], S& rew) {
  S R[3][3];
  rot(x.q, R);
  const S d[3] = {x.p[0] - tgt[0], x.p[1] - tgt[1], x.p[2] - tgt[2]};
#pragma unroll
  for (int j = 0; j < 3; ++j) obs[j] = R[0][j] * d[0] + R[1][j] * d[1] + R[2][j] * d[2];
  const S sg = (x.q[0] < S(0.0f)) ? S(-1.0f) : S(1.0f);
#pragma unroll
  for (int i = 0; i < 4; ++i) obs[3 + i] = sg * x.q[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) obs[7 + i] = x.nu[i];
  S dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  S vv = x.nu[0] * x.nu[0];
#pragma unroll
  for (int i = 1; i < 6; ++i) vv = vv + x.nu[i] * x.nu[i];
  S cc = c[0] * c[0];
#pragma unroll
  for (int i = 1; i < NT; ++i) cc = cc + c[i] * c[i];
  rew = -dd - S(0.1) * vv - S(0.01) * cc;
}

// ---------------------------------------------------------------------------
// Vector-Jacobian products (discretise-then-differentiate).
// ---------------------------------------------------------------------------

// d R / d q contracted with an adjoint LR (3x3): returns LR : dR/dq_k.
template <typename S>
MG_HD void rot_vjp(const S q[4], const S LR[3][3], S lq[4]) {
  const S w = q[0], x = q[1], y = q[2], z = q[3];
  const S t = S(2.0f);
  // R00 = 1-2(y^2+z^2), R01 = 2(xy-wz), R02 = 2(xz+wy)
  // R10 = 2(xy+wz), R11 = 1-2(x^2+z^2), R12 = 2(yz-wx)
  // R20 = 2(xz-wy), R21 = 2(yz+wx), R22 = 1-2(x^2+y^2)
  lq[0] += t * (-z * LR[0][1] + y * LR[0][2] + z * LR[1][0] - x * LR[1][2] - y * LR[2][0] + x * LR[2][1]);
  lq[1] += t * (y * LR[0][1] + z * LR[0][2] + y * LR[1][0] - S(2.0f) * x * LR[1][1] - w * LR[1][2] +
                z * LR[2][0] + w * LR[2][1] - S(2.0f) * x * LR[2][2]);
  lq[2] += t * (-S(2.0f) * y * LR[0][0] + x * LR[0][1] + w * LR[0][2] + x * LR[1][0] + z * LR[1][2] -
                w * LR[2][0] + z * LR[2][1] - S(2.0f) * y * LR[2][2]);
  lq[3] += t * (-S(2.0f) * z * LR[0][0] - w * LR[0][1] + x * LR[0][2] + w * LR[1][0] - S(2.0f) * z * LR[1][1] +
                y * LR[1][2] + x * LR[2][0] + y * LR[2][1]);
}

// y = a x b:  l_a += b x l_y ;  l_b += l_y x a.
template <typename S>
MG_HD void cross_vjp(const S a[3], const S b[3], const S ly[3], S la[3], S lb[3]) {
  S t[3];
  cross3(b, ly, t);
  la[0] += t[0]; la[1] += t[1]; la[2] += t[2];
  cross3(ly, a, t);
  lb[0] += t[0]; lb[1] += t[1]; lb[2] += t[2];
}

// Observation/reward adjoint: adds to the state adjoint `lx` and the command
// adjoint `lc` the contribution of cotangents g_obs (13, may be null) and g_rew.
template <typename S, int NT>
MG_HD void observe_vjp(const St<S, NT>& x, const S (&c)[NT], const S tgt[3], const S* g_obs, S g_rew,
                       St<S, NT>& lx, S (&lc)[NT]) {
  S R[3][3];
  rot(x.q, R);
  const S d[3] = {x.p[0] - tgt[0], x.p[1] - tgt[1], x.p[2] - tgt[2]};
  S LR[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) LR[i][j] = S(0.0f);
  S lq[4] = {S(0.0f), S(0.0f), S(0.0f), S(0.0f)};
  if (g_obs) {
    // obs_j = sum_i R_ij d_i
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lx.p[i] = lx.p[i] + R[i][0] * g_obs[0] + R[i][1] * g_obs[1] + R[i][2] * g_obs[2];
#pragma unroll
      for (int j = 0; j < 3; ++j) LR[i][j] = d[i] * g_obs[j];
    }
    const S sg = (x.q[0] < S(0.0f)) ? S(-1.0f) : S(1.0f);
#pragma unroll
    for (int i = 0; i < 4; ++i) lq[i] = sg * g_obs[3 + i];
#pragma unroll
    for (int i = 0; i < 6; ++i) lx.nu[i] = lx.nu[i] + g_obs[7 + i];
    rot_vjp(x.q, LR, lq);
#pragma unroll
    for (int i = 0; i < 4; ++i) lx.q[i] = lx.q[i] + lq[i];
  }
  // r = -|d|^2 - 0.1|nu|^2 - 0.01|c|^2
#pragma unroll
  for (int i = 0; i < 3; ++i) lx.p[i] = lx.p[i] - S(2.0f) * d[i] * g_rew;
#pragma unroll
  for (int i = 0; i < 6; ++i) lx.nu[i] = lx.nu[i] - S(0.2) * x.nu[i] * g_rew;
#pragma unroll
  for (int i = 0; i < NT; ++i) lc[i] = lc[i] - S(0.02) * c[i] * g_rew;
}

// Adjoint of the body terms of rhs (a4-a7: C_RB, C_A with the current term,
// damping and restoring; the vehicle alone or, PhysT::kFull, the combined
// body of a payload run) given lrhs: accumulates the adjoints of v, w, v_r,
// v_c and e = R^T e_3 and of the added-mass and damping coefficients. The
// wrench tau enters rhs with +1 (its adjoint is lrhs).
template <typename S, typename PhysT>
MG_HD void body_rhs_vjp(const S lrhs[6], const S v[3], const S w[3], const S vr[3], const S vc[3], const PhysT& P,
                        S lv[3], S lw[3], S lvr[3], S lvc[3], S le[3], HydroGrad<S>& g) {
  const S z0 = S(0.0f);
  // (W-B) e  and  -(B rb) x e
  const S WmB = S(P.W) - S(P.B);
  S Brb[3] = {S(P.B) * S(P.rb[0]), S(P.B) * S(P.rb[1]), S(P.B) * S(P.rb[2])};
  if constexpr (PhysT::kFull) {
    // Weight at r_g = s / m: the moment arm is B r_b - (W / m) s.
    const S wpm = S(P.W) / S(P.m);
#pragma unroll
    for (int j = 0; j < 3; ++j) Brb[j] = Brb[j] - wpm * S(P.s[j]);
  }
  {
    // d/de of -(B rb) x e contracted with lrhs_ang: (-lrhs_ang) x (B rb).
    const S nl[3] = {-lrhs[3], -lrhs[4], -lrhs[5]};
    S t[3];
    cross3(nl, Brb, t);
#pragma unroll
    for (int j = 0; j < 3; ++j) le[j] = le[j] + t[j] + WmB * lrhs[j];
  }
  // damping on nu_r
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const S ldm = -lrhs[j];
    const S a = mabs(vr[j]);
    lvr[j] = lvr[j] + ldm * (P.dl[j] + S(2.0f) * P.dq[j] * a);
    g.dl[j] = g.dl[j] + ldm * vr[j];
    g.dq[j] = g.dq[j] + ldm * a * vr[j];
    const S ldw = -lrhs[3 + j];
    const S b = mabs(w[j]);
    lw[j] = lw[j] + ldw * (P.dl[3 + j] + S(2.0f) * P.dq[3 + j] * b);
    g.dl[3 + j] = g.dl[3 + j] + ldw * w[j];
    g.dq[3 + j] = g.dq[3 + j] + ldw * b * w[j];
  }
  // C_RB + C_A in the forward's merged form: rhs_lin -= w x bl with
  // bl = m v + a1; rhs_ang -= w x ba + vr x a1 with ba = A_ang o w + Iw
  // (Iw = Ig o w, or Io w about the origin with a payload); a1 = A_lin o vr.
  {
    S a1[3], bl[3], ba[3], Iw[3];
    if constexpr (PhysT::kFull) {
      Iw[0] = S(P.Io[0]) * w[0] + S(P.Io[1]) * w[1] + S(P.Io[2]) * w[2];
      Iw[1] = S(P.Io[1]) * w[0] + S(P.Io[3]) * w[1] + S(P.Io[4]) * w[2];
      Iw[2] = S(P.Io[2]) * w[0] + S(P.Io[4]) * w[1] + S(P.Io[5]) * w[2];
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j) Iw[j] = S(P.Ig[j]) * w[j];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      a1[j] = S(P.A[j]) * vr[j];
      bl[j] = S(P.m) * v[j] + a1[j];
      ba[j] = S(P.A[3 + j]) * w[j] + Iw[j];
    }
    S nl[3] = {-lrhs[0], -lrhs[1], -lrhs[2]};
    S na[3] = {-lrhs[3], -lrhs[4], -lrhs[5]};
    S lbl[3] = {z0, z0, z0}, lba[3] = {z0, z0, z0}, la1[3] = {z0, z0, z0};
    cross_vjp(w, bl, nl, lw, lbl);
    cross_vjp(w, ba, na, lw, lba);
    cross_vjp(vr, a1, na, lvr, la1);
    // d(Iw)/dw contracted with lba: Ig o lba, or Io lba (symmetric).
    S lIw[3];
    if constexpr (PhysT::kFull) {
      lIw[0] = S(P.Io[0]) * lba[0] + S(P.Io[1]) * lba[1] + S(P.Io[2]) * lba[2];
      lIw[1] = S(P.Io[1]) * lba[0] + S(P.Io[3]) * lba[1] + S(P.Io[4]) * lba[2];
      lIw[2] = S(P.Io[2]) * lba[0] + S(P.Io[4]) * lba[1] + S(P.Io[5]) * lba[2];
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j) lIw[j] = S(P.Ig[j]) * lba[j];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lv[j] = lv[j] + S(P.m) * lbl[j];
      la1[j] = la1[j] + lbl[j];
      lw[j] = lw[j] + S(P.A[3 + j]) * lba[j] + lIw[j];
      g.A[3 + j] = g.A[3 + j] + lba[j] * w[j];
      g.A[j] = g.A[j] + la1[j] * vr[j];
      lvr[j] = lvr[j] + la1[j] * S(P.A[j]);
    }
    if constexpr (PhysT::kFull) {
      // Off-origin centre of gravity: rhs_lin -= w x (w x s),
      // rhs_ang -= s x (w x v).
      const S sv[3] = {S(P.s[0]), S(P.s[1]), S(P.s[2])};
      S wxs[3], lwxs[3] = {z0, z0, z0}, t[3], lz[3];
      cross3(w, sv, wxs);
      cross_vjp(w, wxs, nl, lw, lwxs);
      cross3(sv, lwxs, t);
#pragma unroll
      for (int j = 0; j < 3; ++j) lw[j] = lw[j] + t[j];
      cross3(na, sv, lz);
      cross_vjp(w, v, lz, lw, lv);
    }
    // current-acceleration term A_lin o (w x vc)
    S wxvc[3];
    cross3(w, vc, wxvc);
    S lwv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      g.A[j] = g.A[j] - lrhs[j] * wxvc[j];
      lwv[j] = -lrhs[j] * S(P.A[j]);
    }
    cross_vjp(w, vc, lwv, lw, lvc);
  }
}

// Tape of one substep rebuilt from its start state x0 and its end state x1
// (consecutive records of the forward recompute): the new actuator states n1
// and velocity nu1 are those of x1, the velocity rate M^-1 rhs of a4-a7 is
// (nu1 - nu0) / h, and R, the current, the relative velocity and the
// quaternion update are recomputed from the start attitude in the same
// operations as the substep. The end attitude q1 is x1.q.
template <typename S, int NT, typename PhysT>
MG_HD void tape_from_states(const St<S, NT>& x0, const St<S, NT>& x1, const PhysT& P, S h, S inv_h,
                            Tape<S, NT>& tp) {
#pragma unroll
  for (int i = 0; i < NT; ++i) tp.n1[i] = x1.n[i];
  rot(x0.q, tp.R);
  const S v[3] = {x0.nu[0], x0.nu[1], x0.nu[2]};
#pragma unroll
  for (int i = 0; i < 3; ++i) tp.w[i] = x0.nu[3 + i];
  rel_velocity<S, PhysT, true>(tp.R, v, P, tp.vc, tp.vr);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    tp.nu1[j] = x1.nu[j];
    tp.nd[j] = (x1.nu[j] - x0.nu[j]) * inv_h;
  }
  const S hh = S(0.5f) * h;
  const S wn[3] = {tp.nu1[3], tp.nu1[4], tp.nu1[5]};
  S qd[4];
  quat_rate(x0.q, wn, qd);
#pragma unroll
  for (int i = 0; i < 4; ++i) tp.qn[i] = x0.q[i] + hh * qd[i];
  tp.inv = minvsqrt(tp.qn[0] * tp.qn[0] + tp.qn[1] * tp.qn[1] + tp.qn[2] * tp.qn[2] + tp.qn[3] * tp.qn[3]);
}

// Adjoint of one substep from its tape. x0 is the substep's start state and
// q1 its end attitude; `lx` holds the adjoint of its end state on entry and
// of its start state on exit. The command adjoint and the
// hydrodynamic-coefficient adjoints accumulate. `P` is a Phys<S> or a view
// with its members, or (PhysT::kFull, payload runs) a view of the combined
// body: full inverse Mi, inertia about the origin Io, first moment s, mass m
// and weight W of vehicle and payload.
// `G`: NoGen, or the generic actuator table of a class with fins or tilted
// propellers (their wrenches' products join the thrust and body terms).
template <typename S, int NT, typename ActT, typename PhysT, typename GenT = NoGen>
MG_HD void vjp_from_tape(const St<S, NT>& x0, const S q1[4], const Tape<S, NT>& tp, const S (&c)[NT],
                         const PhysT& P, const ActT& A, S h, St<S, NT>& lx, S (&lc)[NT], HydroGrad<S>& g,
                         const GenT& G = GenT()) {
  constexpr bool GEN = !tt::is_same<GenT, NoGen>::value;
  const S z0 = S(0.0f);
  // Generic wrenches: extra adjoints of the thrusts (tilt) and of the
  // actuator states (servo links, fin angles).
  S lfx[NT], lnx[NT];
#pragma unroll
  for (int i = 0; i < NT; ++i) { lfx[i] = z0; lnx[i] = z0; }

  // q1 = qn * inv
  S dot = q1[0] * lx.q[0] + q1[1] * lx.q[1] + q1[2] * lx.q[2] + q1[3] * lx.q[3];
  S lqn[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) lqn[i] = tp.inv * (lx.q[i] - q1[i] * dot);
  // qn = q + hh * W(w1) q ; W(w) q = q (x) (0, w)
  const S hh = S(0.5f) * h;
  const S qw = x0.q[0], qx = x0.q[1], qy = x0.q[2], qz = x0.q[3];
  const S P_ = tp.nu1[3], Q_ = tp.nu1[4], R_ = tp.nu1[5];
  S lq[4];
  lq[0] = lqn[0] + hh * (P_ * lqn[1] + Q_ * lqn[2] + R_ * lqn[3]);
  lq[1] = lqn[1] + hh * (-P_ * lqn[0] - R_ * lqn[2] + Q_ * lqn[3]);
  lq[2] = lqn[2] + hh * (-Q_ * lqn[0] + R_ * lqn[1] - P_ * lqn[3]);
  lq[3] = lqn[3] + hh * (-R_ * lqn[0] - Q_ * lqn[1] + P_ * lqn[2]);
  S lnu1[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) lnu1[j] = lx.nu[j];
  lnu1[3] = lnu1[3] + hh * (-qx * lqn[0] + qw * lqn[1] + qz * lqn[2] - qy * lqn[3]);
  lnu1[4] = lnu1[4] + hh * (-qy * lqn[0] - qz * lqn[1] + qw * lqn[2] + qx * lqn[3]);
  lnu1[5] = lnu1[5] + hh * (-qz * lqn[0] + qy * lqn[1] - qx * lqn[2] + qw * lqn[3]);
  // p1 = p + h R v1
  S LR[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      LR[i][j] = h * lx.p[i] * tp.nu1[j];
    }
  }
#pragma unroll
  for (int j = 0; j < 3; ++j)
    lnu1[j] = lnu1[j] + h * (tp.R[0][j] * lx.p[0] + tp.R[1][j] * lx.p[1] + tp.R[2][j] * lx.p[2]);
  // lp unchanged (identity).
  // nu1 = nu + h minv o rhs
  S lrhs[6];
  if constexpr (PhysT::kFull) {
    // nu1 = nu + h Mi rhs with Mi = (M_RB + diag(A))^-1 symmetric:
    // lrhs = h Mi lnu1, and d(Mi rhs)/dA_j = -Mi e_j (Mi rhs)_j, so
    // g.A_j -= lrhs_j (Mi rhs)_j = lrhs_j nd_j.
    S t[6];
    apply_minv<S>(P, lnu1, t);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      lrhs[j] = h * t[j];
      g.A[j] = g.A[j] - lrhs[j] * tp.nd[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      lrhs[j] = h * P.minv[j] * lnu1[j];
      // minv_j = 1/(M_RB,jj + A_j): d minv / dA = -minv^2, and
      // h minv^2 lnu1 rhs = lrhs (minv rhs) = lrhs nd.
      g.A[j] = g.A[j] - lrhs[j] * tp.nd[j];
    }
  }
  S lnu[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) lnu[j] = lnu1[j];
  // rhs_lin = tau - m w x v - w x a1 - A_lin o (w x vc) - dmp_lin + (W-B) e
  // rhs_ang = tau - w x Iw - vr x a1 - w x a2 - dmp_ang - (B rb) x e
  const S* vr = tp.vr;
  const S* w = tp.w;
  const S* vc = tp.vc;
  const S v[3] = {x0.nu[0], x0.nu[1], x0.nu[2]};
  S lv[3] = {z0, z0, z0}, lw[3] = {z0, z0, z0}, lvr[3] = {z0, z0, z0}, lvc[3] = {z0, z0, z0};
  S le[3] = {z0, z0, z0};
  body_rhs_vjp<S, PhysT>(lrhs, v, w, vr, vc, P, lv, lw, lvr, lvc, le, g);
  if constexpr (GEN) fin_wrench_vjp<S, NT>(G, tp.n1, vr, w, lrhs, lnx, lvr, lw);
  // vr = v - vc ; vc = R^T Vc
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lv[j] = lv[j] + lvr[j];
    lvc[j] = lvc[j] - lvr[j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) LR[i][j] = LR[i][j] + P.Vc[i] * lvc[j];
#pragma unroll
  for (int j = 0; j < 3; ++j) LR[2][j] = LR[2][j] + le[j];
  rot_vjp(x0.q, LR, lq);
  // tau = B f (+ the tilt wrench) ; f_i = k n1 |n1|
  if constexpr (GEN) {
    S f1[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const S an = mabs(tp.n1[i]);
      f1[i] = (an < S(A.dz[i])) ? z0 : S(A.kf[i]) * tp.n1[i] * an;
    }
    tilt_wrench_vjp<S, NT>(G, tp.n1, f1, lrhs, lfx, lnx);
  }
  S ln1[NT];
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    S lf = S(A.alloc[0][i]) * lrhs[0];
#pragma unroll
    for (int k = 1; k < 6; ++k) lf = lf + S(A.alloc[k][i]) * lrhs[k];
    lf = lf + lfx[i];
    const S an = mabs(tp.n1[i]);
    const S df = (an < S(A.dz[i])) ? z0 : S(2.0f) * S(A.kf[i]) * an;
    ln1[i] = lx.n[i] + lnx[i] + lf * df;
  }
  // n1 = n + alpha (c - n)
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    lc[i] = lc[i] + S(A.alpha[i]) * ln1[i];
    lx.n[i] = (S(1.0f) - S(A.alpha[i])) * ln1[i];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lx.nu[j] = lnu[j] + lv[j];
    lx.nu[3 + j] = lnu[3 + j] + lw[j];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) lx.q[i] = lq[i];
  // lx.p: identity through p1 = p + ...
}

// Adjoint of one RK4 stage derivative F(q, nu) = (R v, 1/2 q (x) (0, w),
// M^-1 rhs) at the stage point (q, nu) (R from the normalised q), with the
// actuator states n and the state-independent wrench tau_n held: from the
// adjoints ldp, ldq, ldnu of F it accumulates those of the stage point (lq,
// lnu), of tau_n (ltau), of the fin angles (ln) and of the coefficients (g).
template <typename S, int NT, typename PhysT, bool CURRENT, typename GenT>
MG_HD void rk4_stage_vjp(const S q[4], const S nu[6], const S (&n)[NT], const S tau_n[6], const PhysT& P,
                         const GenT& G, const S ldp[3], const S ldq[4], const S ldnu[6], S lq[4], S lnu[6],
                         S ltau[6], S (&ln)[NT], HydroGrad<S>& g) {
  constexpr bool GEN = !tt::is_same<GenT, NoGen>::value;
  const S z0 = S(0.0f);
  // Forward internals.
  const S iq = minvsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const S qh[4] = {q[0] * iq, q[1] * iq, q[2] * iq, q[3] * iq};
  S R[3][3];
  rot(qh, R);
  const S v[3] = {nu[0], nu[1], nu[2]};
  const S w[3] = {nu[3], nu[4], nu[5]};
  S vc[3], vr[3], tau[6];
  rel_velocity<S, PhysT, CURRENT>(R, v, P, vc, vr);
#pragma unroll
  for (int k = 0; k < 6; ++k) tau[k] = tau_n[k];
  if constexpr (GEN) fin_wrench<S, NT>(G, n, vr, w, tau);
  S rhs[6];
  body_rhs<S, PhysT, CURRENT>(R, v, w, vc, vr, tau, P, rhs);
  // dnu = M^-1 rhs.
  S lrhs[6];
  if constexpr (PhysT::kFull) {
    S nd[6];
    apply_minv<S>(P, ldnu, lrhs);
    apply_minv<S>(P, rhs, nd);
#pragma unroll
    for (int j = 0; j < 6; ++j) g.A[j] = g.A[j] - lrhs[j] * nd[j];
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      lrhs[j] = S(P.minv[j]) * ldnu[j];
      g.A[j] = g.A[j] - rhs[j] * lrhs[j] * S(P.minv[j]);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) ltau[k] = ltau[k] + lrhs[k];
  S lv[3] = {z0, z0, z0}, lw[3] = {z0, z0, z0}, lvr[3] = {z0, z0, z0}, lvc[3] = {z0, z0, z0};
  S le[3] = {z0, z0, z0};
  body_rhs_vjp<S, PhysT>(lrhs, v, w, vr, vc, P, lv, lw, lvr, lvc, le, g);
  if constexpr (GEN) fin_wrench_vjp<S, NT>(G, n, vr, w, lrhs, ln, lvr, lw);
  // dp = R v
  S LR[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) LR[i][j] = ldp[i] * v[j];
#pragma unroll
  for (int j = 0; j < 3; ++j) lv[j] = lv[j] + R[0][j] * ldp[0] + R[1][j] * ldp[1] + R[2][j] * ldp[2];
  // dq = 1/2 q (x) (0, w)
  const S qw = q[0], qx = q[1], qy = q[2], qz = q[3];
  const S hq = S(0.5f);
  lq[0] = lq[0] + hq * (w[0] * ldq[1] + w[1] * ldq[2] + w[2] * ldq[3]);
  lq[1] = lq[1] + hq * (-w[0] * ldq[0] - w[2] * ldq[2] + w[1] * ldq[3]);
  lq[2] = lq[2] + hq * (-w[1] * ldq[0] + w[2] * ldq[1] - w[0] * ldq[3]);
  lq[3] = lq[3] + hq * (-w[2] * ldq[0] - w[1] * ldq[1] + w[0] * ldq[2]);
  lw[0] = lw[0] + hq * (-qx * ldq[0] + qw * ldq[1] + qz * ldq[2] - qy * ldq[3]);
  lw[1] = lw[1] + hq * (-qy * ldq[0] - qz * ldq[1] + qw * ldq[2] + qx * ldq[3]);
  lw[2] = lw[2] + hq * (-qz * ldq[0] + qy * ldq[1] - qx * ldq[2] + qw * ldq[3]);
  // vr = v - vc ; vc = R^T Vc ; e = R^T e_3 ; R = R(q / |q|)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lv[j] = lv[j] + lvr[j];
    lvc[j] = lvc[j] - lvr[j];
  }
  if (CURRENT) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) LR[i][j] = LR[i][j] + S(P.Vc[i]) * lvc[j];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) LR[2][j] = LR[2][j] + le[j];
  S lqh[4] = {z0, z0, z0, z0};
  rot_vjp(qh, LR, lqh);
  const S dot = qh[0] * lqh[0] + qh[1] * lqh[1] + qh[2] * lqh[2] + qh[3] * lqh[3];
#pragma unroll
  for (int i = 0; i < 4; ++i) lq[i] = lq[i] + iq * (lqh[i] - qh[i] * dot);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lnu[j] = lnu[j] + lv[j];
    lnu[3 + j] = lnu[3 + j] + lw[j];
  }
}

// Adjoint of one RK4 substep (substep_rk4) from its start state x0: the
// stages are recomputed, then reversed. `lx` holds the adjoint of the end
// state on entry and of x0 on exit; lc and g accumulate. N1: x0.n holds the
// substep's new actuator states (those of its recorded end state) instead of
// the start ones.
template <typename S, int NT, typename ActT, typename PhysT, bool CURRENT = true, typename GenT = NoGen,
          bool N1 = false>
MG_HD void substep_rk4_vjp(const St<S, NT>& x0, const S (&c)[NT], const PhysT& P, const ActT& A, S h, St<S, NT>& lx,
                           S (&lc)[NT], HydroGrad<S>& g, const GenT& G = GenT()) {
  constexpr bool GEN = !tt::is_same<GenT, NoGen>::value;
  const S z0 = S(0.0f);
  // Forward: actuators, then the four stage points and the sum.
  St<S, NT> xa = x0;
  S f[NT], tau_n[6];
  actuate<S, NT, ActT, !N1>(xa, c, A, f, tau_n);
  if constexpr (GEN) tilt_wrench<S, NT>(G, xa.n, f, tau_n);
  const S h2 = S(0.5f) * h, h6 = h / S(6.0f), h3 = h / S(3.0f);
  S yq[4][4], ynu[4][6], sq[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) { yq[0][i] = x0.q[i]; sq[i] = x0.q[i]; }
#pragma unroll
  for (int i = 0; i < 6; ++i) ynu[0][i] = x0.nu[i];
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    S dp[3], dq[4], dnu[6];
    rk4_stage<S, NT, PhysT, CURRENT>(yq[st], ynu[st], xa.n, tau_n, P, G, dp, dq, dnu);
    const S wsum = (st == 0 || st == 3) ? h6 : h3;
#pragma unroll
    for (int i = 0; i < 4; ++i) sq[i] = sq[i] + wsum * dq[i];
    if (st < 3) {
      const S hs = (st == 2) ? h : h2;
#pragma unroll
      for (int i = 0; i < 4; ++i) yq[st + 1][i] = x0.q[i] + hs * dq[i];
#pragma unroll
      for (int i = 0; i < 6; ++i) ynu[st + 1][i] = x0.nu[i] + hs * dnu[i];
    }
  }
  const S inv = minvsqrt(sq[0] * sq[0] + sq[1] * sq[1] + sq[2] * sq[2] + sq[3] * sq[3]);
  // Reverse: q1 = sum_q / |sum_q|.
  S q1[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) q1[i] = sq[i] * inv;
  const S dot = q1[0] * lx.q[0] + q1[1] * lx.q[1] + q1[2] * lx.q[2] + q1[3] * lx.q[3];
  S lsq[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) lsq[i] = inv * (lx.q[i] - q1[i] * dot);
  // Adjoints of the stage derivatives k_s and of the stage points g_s:
  // k4 <- h/6 ly; k3 <- h/3 ly + h g4; k2 <- h/3 ly + h/2 g3; k1 <- h/6 ly + h/2 g2.
  S ltau[6] = {z0, z0, z0, z0, z0, z0};
  S lnx[NT];
#pragma unroll
  for (int i = 0; i < NT; ++i) lnx[i] = z0;
  S gq[4] = {z0, z0, z0, z0}, gnu[6] = {z0, z0, z0, z0, z0, z0};     // g of the later stage point
  S aq[4], anu[6];                                                   // sum of the stage points' g
#pragma unroll
  for (int i = 0; i < 4; ++i) aq[i] = z0;
#pragma unroll
  for (int i = 0; i < 6; ++i) anu[i] = z0;
#pragma unroll
  for (int st = 3; st >= 0; --st) {
    const S wsum = (st == 0 || st == 3) ? h6 : h3;
    const S hn = (st == 2) ? h : h2;   // the next stage point's step (stage st + 1 = y0 + hn k_st)
    S ldp[3], ldq[4], ldnu[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) ldp[i] = wsum * lx.p[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) ldq[i] = wsum * lsq[i] + (st < 3 ? hn * gq[i] : z0);
#pragma unroll
    for (int i = 0; i < 6; ++i) ldnu[i] = wsum * lx.nu[i] + (st < 3 ? hn * gnu[i] : z0);
    S nq[4] = {z0, z0, z0, z0}, nnu[6] = {z0, z0, z0, z0, z0, z0};
    rk4_stage_vjp<S, NT, PhysT, CURRENT>(yq[st], ynu[st], xa.n, tau_n, P, G, ldp, ldq, ldnu, nq, nnu, ltau, lnx, g);
#pragma unroll
    for (int i = 0; i < 4; ++i) { gq[i] = nq[i]; aq[i] = aq[i] + nq[i]; }
#pragma unroll
    for (int i = 0; i < 6; ++i) { gnu[i] = nnu[i]; anu[i] = anu[i] + nnu[i]; }
  }
  // y0 = (q0, nu0) enters the sum and every stage point; p enters only the sum.
#pragma unroll
  for (int i = 0; i < 4; ++i) lx.q[i] = lsq[i] + aq[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) lx.nu[i] = lx.nu[i] + anu[i];
  // tau_n = B f (+ the tilt wrench) ; f_i = k n1 |n1| ; n1 = n + alpha (c - n)
  S lfx[NT];
#pragma unroll
  for (int i = 0; i < NT; ++i) lfx[i] = z0;
  if constexpr (GEN) tilt_wrench_vjp<S, NT>(G, xa.n, f, ltau, lfx, lnx);
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    S lf = S(A.alloc[0][i]) * ltau[0];
#pragma unroll
    for (int k = 1; k < 6; ++k) lf = lf + S(A.alloc[k][i]) * ltau[k];
    lf = lf + lfx[i];
    const S an = mabs(xa.n[i]);
    const S df = (an < S(A.dz[i])) ? z0 : S(2.0f) * S(A.kf[i]) * an;
    const S ln1 = lx.n[i] + lnx[i] + lf * df;
    lc[i] = lc[i] + S(A.alpha[i]) * ln1;
    lx.n[i] = (S(1.0f) - S(A.alpha[i])) * ln1;
  }
}

// Adjoint of one substep with its forward recomputed in full.
template <typename S, int NT, typename ActT>
MG_HD void substep_vjp(const St<S, NT>& x0, const S (&c)[NT], const Phys<S>& P, const ActT& A, S h,
                       St<S, NT>& lx, S (&lc)[NT], HydroGrad<S>& g) {
  St<S, NT> x = x0;
  Tape<S, NT> tp;
  substep<S, NT, true>(x, c, P, A, h, &tp);
  vjp_from_tape<S, NT>(x0, x.q, tp, c, P, A, h, lx, lc, g);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): published multipliers
// and Weyl increments.
// ---------------------------------------------------------------------------
MG_HD void mulhilo64(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
  hi = __umul64hi(a, b);
  lo = a * b;
#else
  unsigned __int128 p = (unsigned __int128)a * b;
  hi = (uint64_t)(p >> 64);
  lo = (uint64_t)p;
#endif
}

MG_HD void philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1,
                      uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, hi0, lo0);
    mulhilo64(M1, c2, hi1, lo1);
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Draw j of (seed, stream, env): block j/4, lane j%4, top 53 bits -> [0,1).
MG_HD double uniform53(uint64_t seed, uint64_t stream, uint64_t env, uint32_t j) {
  uint64_t o[4];
  philox4x64(env, j / 4, 0, 0, seed, stream, o);
  return (double)(o[j % 4] >> 11) * (1.0 / 9007199254740992.0);
}

enum : uint64_t { STREAM_DR = 1, STREAM_INIT = 2, STREAM_ACTION = 3 };

}  // namespace mg
