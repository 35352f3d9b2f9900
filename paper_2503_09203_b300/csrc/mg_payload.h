// Payload block of one env: a point mass rigidly attached to the vehicle
// (Sec. III-B, mission payloads with configurable mass and attachment point;
// Table 2, payload mass as a fraction of the vehicle mass). Used by the reset
// kernel and by the host-side parameter setters, in FP64.
//
// With the vehicle's CoG at the body origin (mass m, principal inertia Ig,
// weight W) and a payload m_p at r_p, the combined body has mass m' = m + m_p,
// first moment s = m_p r_p (so r_g = s / m'), inertia about the origin
// I_o = diag(Ig) + m_p (|r_p|^2 1 - r_p r_p^T) and weight W' = W + m_p g.
// The rigid-body inertia about the origin is
// M_RB = [[m' 1, -S(s)], [S(s), I_o]] (Fossen 2011, Eq. 6.37 with m' r_g = s),
// symmetric positive definite, and M = M_RB + diag(M_A) is inverted by a
// Cholesky factorisation.
#pragma once

#include <math.h>

#include "mg_internal.h"

#ifdef __CUDACC__
#define MG_PAY_HD __host__ __device__ inline
#else
#define MG_PAY_HD inline
#endif

namespace mg {

constexpr double kPayloadGravity = 9.81;

// The combined body in FP64: mass mt, first moment s, inertia about the
// origin Io, weight Wt and Mi = (M_RB + diag(Ma))^-1. Returns false if M is
// not positive definite.
MG_PAY_HD bool payload_body(double m, const double Ig[3], const double Ma[6], double W, double mp,
                            const double rp[3], double* mt_out, double s[3], double Io[3][3], double* Wt,
                            double Mi[6][6]) {
  const double mt = m + mp;
  for (int j = 0; j < 3; ++j) s[j] = mp * rp[j];
  const double rp2 = rp[0] * rp[0] + rp[1] * rp[1] + rp[2] * rp[2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Io[i][j] = (i == j ? Ig[i] + mp * rp2 : 0.0) - mp * rp[i] * rp[j];
  // S(s) = [[0, -s_z, s_y], [s_z, 0, -s_x], [-s_y, s_x, 0]].
  const double Ss[3][3] = {{0.0, -s[2], s[1]}, {s[2], 0.0, -s[0]}, {-s[1], s[0], 0.0}};
  double M[6][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      M[i][j] = (i == j) ? mt + Ma[i] : 0.0;
      M[i][3 + j] = -Ss[i][j];
      M[3 + i][j] = Ss[i][j];
      M[3 + i][3 + j] = Io[i][j] + (i == j ? Ma[3 + i] : 0.0);
    }
  // Cholesky M = L L^T.
  double L[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = 0.0;
  for (int j = 0; j < 6; ++j) {
    double d = M[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) return false;
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double v = M[i][j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  // Column c of M^-1 solves L L^T x = e_c.
  for (int c = 0; c < 6; ++c) {
    double y[6], x[6];
    for (int i = 0; i < 6; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
      y[i] = v / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < 6; ++k) v -= L[k][i] * x[k];
      x[i] = v / L[i][i];
    }
    for (int i = 0; i < 6; ++i) Mi[i][c] = x[i];
  }
  *mt_out = mt;
  *Wt = W + mp * kPayloadGravity;
  return true;
}

// Writes the PAY_DIM floats of the payload planes (layout PAY_*). Returns
// false (and leaves `out` untouched) if M is not positive definite.
MG_PAY_HD bool payload_block(double m, const double Ig[3], const double Ma[6], double W, double mp,
                             const double rp[3], float out[PAY_DIM]) {
  double mt, s[3], Io[3][3], Wt, Mi[6][6];
  if (!payload_body(m, Ig, Ma, W, mp, rp, &mt, s, Io, &Wt, Mi)) return false;
  int q = PAY_MINV;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) out[q++] = (float)(0.5 * (Mi[i][j] + Mi[j][i]));
  out[PAY_IO + 0] = (float)Io[0][0];
  out[PAY_IO + 1] = (float)Io[0][1];
  out[PAY_IO + 2] = (float)Io[0][2];
  out[PAY_IO + 3] = (float)Io[1][1];
  out[PAY_IO + 4] = (float)Io[1][2];
  out[PAY_IO + 5] = (float)Io[2][2];
  for (int j = 0; j < 3; ++j) out[PAY_S + j] = (float)s[j];
  out[PAY_M] = (float)mt;
  out[PAY_W] = (float)Wt;
  out[PAY_MP] = (float)mp;
  for (int j = 0; j < 3; ++j) out[PAY_RP + j] = (float)rp[j];
  return true;
}

}  // namespace mg
