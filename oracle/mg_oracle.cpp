// FP64 CPU oracle of the MarineGym per-environment UUV step (arXiv 2503.09203).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference the CUDA
// path is checked against. Only the test-suite, the smoke check and the CPU
// baseline leg of the benchmark may load it; the product library never links,
// calls or includes it, and it includes nothing from the product.
//
// What it computes (paper, Sec. III-B and III-D):
//   * Fossen's equation of motion, Eq. 1, split as in Eq. 2 into a rigid-body
//     part (M_RB, C_RB, g_RB) and a hydrodynamic part (M_A, C_A, D, g_A).
//   * The hydrodynamic wrench of Eq. 3 evaluated at the relative velocity
//     nu_r = nu - nu_c of the ocean-current paragraph (Sec. III-B, after Eq. 3).
//   * Actuators (Sec. III-D): first-order rotor lag (zero-order when the time
//     constant is 0), quadratic thrust with a dead zone, each force applied as a
//     wrench at its own actuator frame.
//   * Domain randomisation draws (Sec. III-C, Table 2 ranges) and the hover
//     (station-keeping) task's observation and reward (Sec. IV-B).
// The matrices C_RB(nu), C_A(nu) and D(nu) are built as full 6x6 matrices from
// Fossen's parametrisations and M nu_dot = rhs is solved by Gaussian
// elimination, so the oracle does not share the product-form shortcuts that a
// fast kernel would take.
//
// Readings where the paper is silent (each is listed in the design notes):
//   R1 attitude is a unit quaternion (w,x,y,z), Hamilton, body->NED, z down.
//   R2 Eq. 3 is evaluated with nu_r everywhere, including M_A d(nu_r)/dt; the
//      current is constant and irrotational in NED, so d(nu_c)/dt = [-w x v_c; 0].
//   R6 integrator: semi-implicit Euler per substep h = dt/K: rotor, forces at
//      (nu_k, q_k, n_{k+1}), nu, then p with v+, then q with w+ and renormalise.
//   R7 alpha = 1 - exp(-h/T); thrust f = k n|n| outside |n| < deadzone, else 0.
//   R11 hover reward r = -|p-p*|^2 - 0.1|nu|^2 - 0.01|c|^2.
//
// Parity of this oracle with the paper's own plugin is unpinned (the paper
// prints no parameters, trajectories or intermediate values); it is pinned to
// closed forms and invariants by the CPU tests.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <omp.h>

namespace orc {

static const double kGravity = 9.81;   // m/s^2, NED +z
static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Scalar types: plain double, and a forward-mode dual number for JVPs.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual fabs(Dual a) { return a.v < 0 ? -a : (a.v > 0 ? a : Dual(0.0, 0.0)); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Dual atan2(Dual y, Dual x) {
  return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v));
}
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
using std::sqrt;
using std::fabs;
using std::sin;
using std::cos;
using std::atan2;

// ---------------------------------------------------------------------------
// C-ABI records (host, FP64).
// ---------------------------------------------------------------------------
}  // namespace orc

extern "C" {

// A vehicle class (Sec. III-D): rigid body, hydrodynamic coefficients as
// positive magnitudes (added mass diag, linear and quadratic damping diag),
// and up to 8 actuator channels. Every channel has a first-order state n in
// [-1, 1] driven by its command (rotor speed, or servo / fin angle n * range).
// Kinds (Sec. III-D actuator types): 0 propeller with fixed unit direction;
// 1 servo (no force; tilts the propellers linked to it); 2 fin (control
// surface: lift and drag from the local flow); 3 propeller whose direction is
// turned about act_axis by the angle of the servo act_link.
typedef struct {
  int32_t n_thr;
  int32_t pad0;
  double mass;          // kg
  double Ig[3];         // principal inertia about CoG, kg m^2
  double rg[3];         // CoG in body frame, m
  double rb[3];         // CoB in body frame, m (z down: "above" is negative z)
  double buoy_ratio;    // B / (mass g) at nominal volume
  double Ma[6];         // added mass diag
  double dl[6];         // linear damping diag
  double dq[6];         // quadratic damping diag
  double thr_pos[8][3];
  double thr_dir[8][3];
  double k_f[8];        // N at |n| = 1
  double T_rotor[8];    // s; 0 means zero-order rotor
  double deadzone[8];   // |n| below which thrust is 0
  int32_t act_kind[8];  // 0 propeller, 1 servo, 2 fin, 3 tilted propeller
  int32_t act_link[8];  // kind 3: channel index of its servo
  double act_axis[8][3];   // kind 2: span axis; kind 3: tilt axis (unit, body frame)
  double act_chord[8][3];  // kind 2: chord direction at zero deflection (unit, normal to the span axis)
  double act_range[8];     // kinds 1, 2: angle at |n| = 1, rad
  double fin_area[8];      // kind 2: planform area S, m^2
  double fin_cl[8];        // kind 2: lift slope C_L_alpha, 1/rad
  double fin_cd0[8];       // kind 2: drag at zero angle of attack
  double fin_cda[8];       // kind 2: drag growth C_D_alpha
  double rho;              // water density, kg/m^3 (fins)
} or_class;

// Per-environment physical parameters after domain randomisation.
typedef struct {
  int32_t cls;
  int32_t pad0;
  double mass, Ig[3], rg[3], rb[3], W, B;
  double Ma[6], dl[6], dq[6];
  double Vc[3];       // ocean current, NED, m/s
  double target[3];   // hover target p* (tracking: the reference centre c), NED, m
  double traj_a[3], traj_w[3], traj_phi[3], traj_v[3];   // tracking reference (zeros: hover)
  double k0;          // step counter at the start of the rollout
  double Ig_off[3];   // products of inertia about the CoG (Ixy, Ixz, Iyz): 0 without payload
} or_env;

// Reset configuration: domain-randomisation ranges (Table 2 train column
// shape) and the initial-state mode.
typedef struct {
  int32_t dr_enabled;
  int32_t current_enabled;
  int32_t current_3d;      // 0: horizontal current direction, 1: uniform on sphere
  int32_t init_mode;       // 0: rest at origin, 1: hover task random pose
  double mass_lo, mass_hi;
  double added_lo, added_hi;
  double damp_lo, damp_hi;
  double cob_lo, cob_hi;
  double cur_lo, cur_hi;   // current speed range, m/s
  double target_half;      // hover target p* ~ U[-L, L]^3
  double pos_radius;       // initial |p - p*| <= radius (uniform in ball)
  double max_angle;        // initial attitude error angle ~ U[0, max], rad
  int32_t track;           // 1: draw a tracking reference
  int32_t track_kind;      // 0 helix, 1 Lissajous
  int32_t payload;         // 1: attach a point-mass payload (Sec. III-B payloads, Table 2)
  int32_t pad1;
  double payload_lo, payload_hi;   // payload mass / vehicle mass ~ U[lo, hi]
} or_reset_cfg;

}  // extern "C"

namespace orc {

// ---------------------------------------------------------------------------
// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
// Published constants: multipliers and Weyl key increments of Philox4x64.
// ---------------------------------------------------------------------------
static void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    unsigned __int128 p0 = (unsigned __int128)M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0; k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Uniform double in [0,1) from draw number j of (seed, stream, env):
// block j/4 of the counter (env, j/4, 0, 0) under key (seed, stream), lane j%4,
// top 53 bits.
static double draw_u(uint64_t seed, uint64_t stream, uint64_t env, uint64_t j) {
  uint64_t ctr[4] = {env, j / 4, 0, 0}, key[2] = {seed, stream}, out[4];
  philox4x64_10(ctr, key, out);
  return (double)(out[j % 4] >> 11) * (1.0 / 9007199254740992.0);
}

// Streams of the counter-based generator.
static const uint64_t kStreamDR = 1, kStreamInit = 2, kStreamAction = 3;

// ---------------------------------------------------------------------------
// Small dense linear algebra.
// ---------------------------------------------------------------------------
template <class T> struct V3 { T x[3]; };
template <class T> static void cross(const T a[3], const T b[3], T out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}
// Skew-symmetric S(a) with S(a) b = a x b.
template <class T> static void skew(const T a[3], T S[3][3]) {
  S[0][0] = T(0.0); S[0][1] = -a[2]; S[0][2] = a[1];
  S[1][0] = a[2];  S[1][1] = T(0.0); S[1][2] = -a[0];
  S[2][0] = -a[1]; S[2][1] = a[0];  S[2][2] = T(0.0);
}
template <class T> static void matvec6(const T A[6][6], const T x[6], T y[6]) {
  for (int i = 0; i < 6; ++i) {
    T s = T(0.0);
    for (int j = 0; j < 6; ++j) s += A[i][j] * x[j];
    y[i] = s;
  }
}
// Solve A x = b (6x6) by Gaussian elimination with partial pivoting on the
// value part of the entries.
template <class T> static void solve6(const T A_in[6][6], const T b_in[6], T x[6]) {
  T A[6][6], b[6];
  for (int i = 0; i < 6; ++i) { b[i] = b_in[i]; for (int j = 0; j < 6; ++j) A[i][j] = A_in[i][j]; }
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (std::fabs(val(A[r][c])) > std::fabs(val(A[piv][c]))) piv = r;
    if (piv != c) {
      for (int j = 0; j < 6; ++j) { T t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
      T t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < 6; ++r) {
      T f = A[r][c] / A[c][c];
      for (int j = c; j < 6; ++j) A[r][j] -= f * A[c][j];
      b[r] -= f * b[c];
    }
  }
  for (int i = 5; i >= 0; --i) {
    T s = b[i];
    for (int j = i + 1; j < 6; ++j) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
}

// Rotation matrix of a unit quaternion q = (w,x,y,z), body -> NED (R1).
template <class T> static void rotation(const T q[4], T R[3][3]) {
  const T w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = T(1.0) - T(2.0) * (y * y + z * z);
  R[0][1] = T(2.0) * (x * y - w * z);
  R[0][2] = T(2.0) * (x * z + w * y);
  R[1][0] = T(2.0) * (x * y + w * z);
  R[1][1] = T(1.0) - T(2.0) * (x * x + z * z);
  R[1][2] = T(2.0) * (y * z - w * x);
  R[2][0] = T(2.0) * (x * z - w * y);
  R[2][1] = T(2.0) * (y * z + w * x);
  R[2][2] = T(1.0) - T(2.0) * (x * x + y * y);
}

// ---------------------------------------------------------------------------
// Fossen's matrices (Eq. 1 and Eq. 2 terms). Env parameters in T so that the
// added-mass and damping coefficients can carry tangents.
// ---------------------------------------------------------------------------
template <class T> struct EnvT {
  double mass, Ig[3], Ig_off[3], rg[3], rb[3], W, B;
  T Ma[6], dl[6], dq[6];
  double Vc[3], target[3];
  double ta[3], tw[3], tph[3], tv[3], k0;
};

// Station-keeping target / tracking reference at time t (Sec. IV-B tasks):
// a helix or Lissajous curve written as c + a o sin(w t + phi) + v t
// (all of a, w, phi, v zero for station keeping).
template <class T> static void reference(const EnvT<T>& e, double t, double out[3]) {
  for (int i = 0; i < 3; ++i) out[i] = e.target[i] + e.ta[i] * std::sin(e.tw[i] * t + e.tph[i]) + e.tv[i] * t;
}

// Inertia tensor about the CoG: principal moments on the diagonal, products
// of inertia (nonzero once a payload is attached) off it.
template <class T> static double inertia_cog(const EnvT<T>& e, int i, int j) {
  if (i == j) return e.Ig[i];
  const int k = (i + j == 1) ? 0 : (i + j == 2 ? 1 : 2);   // (0,1)->Ixy, (0,2)->Ixz, (1,2)->Iyz
  return e.Ig_off[k];
}

// Rigid-body inertia about the body origin with the CoG at r_g:
// M_RB = [[m I, -m S(r_g)], [m S(r_g), I_g - m S(r_g)^2]].
template <class T> static void mass_rb(const EnvT<T>& e, T M[6][6]) {
  T rg[3] = {T(e.rg[0]), T(e.rg[1]), T(e.rg[2])}, S[3][3];
  skew(rg, S);
  for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) M[i][j] = T(0.0);
  for (int i = 0; i < 3; ++i) {
    M[i][i] = T(e.mass);
    for (int j = 0; j < 3; ++j) {
      M[i][3 + j] = T(-e.mass) * S[i][j];
      M[3 + i][j] = T(e.mass) * S[i][j];
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s2 = T(0.0);
      for (int k = 0; k < 3; ++k) s2 += S[i][k] * S[k][j];
      M[3 + i][3 + j] = T(inertia_cog(e, i, j)) - T(e.mass) * s2;
    }
}

// Added mass as a 6x6 matrix (diagonal of positive magnitudes).
template <class T> static void mass_a(const EnvT<T>& e, T M[6][6]) {
  for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) M[i][j] = (i == j) ? e.Ma[i] : T(0.0);
}

// Rigid-body Coriolis-centripetal matrix, parametrisation independent of the
// linear velocity (Fossen 2011, Eq. 6.43, here with I_o the inertia about
// the body origin): C_RB = [[m S(w), -m S(w) S(r_g)], [m S(r_g) S(w), -S(I_o w)]].
template <class T> static void coriolis_rb(const EnvT<T>& e, const T nu[6], T C[6][6]) {
  T w[3] = {nu[3], nu[4], nu[5]};
  T rg[3] = {T(e.rg[0]), T(e.rg[1]), T(e.rg[2])};
  T Sw[3][3], Sr[3][3];
  skew(w, Sw);
  skew(rg, Sr);
  T Mrb[6][6];
  mass_rb(e, Mrb);
  T Iow[3];
  for (int i = 0; i < 3; ++i) {
    Iow[i] = T(0.0);
    for (int j = 0; j < 3; ++j) Iow[i] += Mrb[3 + i][3 + j] * w[j];
  }
  T SI[3][3];
  skew(Iow, SI);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T SwSr = T(0.0), SrSw = T(0.0);
      for (int k = 0; k < 3; ++k) { SwSr += Sw[i][k] * Sr[k][j]; SrSw += Sr[i][k] * Sw[k][j]; }
      C[i][j] = T(e.mass) * Sw[i][j];
      C[i][3 + j] = T(-e.mass) * SwSr;
      C[3 + i][j] = T(e.mass) * SrSw;
      C[3 + i][3 + j] = -SI[i][j];
    }
}

// Added-mass Coriolis-centripetal matrix (Fossen 2011, Eq. 6.44 with the
// positive-magnitude convention of M_A):
// C_A(nu) = [[0, -S(A11 v + A12 w)], [-S(A11 v + A12 w), -S(A21 v + A22 w)]].
template <class T> static void coriolis_a(const EnvT<T>& e, const T nu[6], T C[6][6]) {
  T MA[6][6];
  mass_a(e, MA);
  T a1[3], a2[3];
  for (int i = 0; i < 3; ++i) {
    a1[i] = T(0.0); a2[i] = T(0.0);
    for (int j = 0; j < 6; ++j) { a1[i] += MA[i][j] * nu[j]; a2[i] += MA[3 + i][j] * nu[j]; }
  }
  T S1[3][3], S2[3][3];
  skew(a1, S1);
  skew(a2, S2);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C[i][j] = T(0.0);
      C[i][3 + j] = -S1[i][j];
      C[3 + i][j] = -S1[i][j];
      C[3 + i][3 + j] = -S2[i][j];
    }
}

// Damping matrix D(nu) = D_l + diag(d_q |nu|).
template <class T> static void damping(const EnvT<T>& e, const T nu[6], T D[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) D[i][j] = (i == j) ? (e.dl[i] + e.dq[i] * fabs(nu[i])) : T(0.0);
}

// Restoring vectors of Eq. 2: g_RB from the weight W at r_g and g_A from the
// buoyancy B at r_b; each is -[f; r x f] with f the body-frame force.
template <class T> static void restoring(const EnvT<T>& e, const T R[3][3], T gRB[6], T gA[6]) {
  T fg[3], fb[3];
  for (int i = 0; i < 3; ++i) {
    fg[i] = R[2][i] * T(e.W);     // R^T [0,0,W]
    fb[i] = R[2][i] * T(-e.B);    // R^T [0,0,-B]
  }
  T rg[3] = {T(e.rg[0]), T(e.rg[1]), T(e.rg[2])}, rb[3] = {T(e.rb[0]), T(e.rb[1]), T(e.rb[2])};
  T mg[3], mb[3];
  cross(rg, fg, mg);
  cross(rb, fb, mb);
  for (int i = 0; i < 3; ++i) {
    gRB[i] = -fg[i]; gRB[3 + i] = -mg[i];
    gA[i] = -fb[i];  gA[3 + i] = -mb[i];
  }
}

// Actuator wrench: each thruster force f_i d_i applied at its frame r_i
// contributes [f_i d_i ; r_i x f_i d_i] (Sec. III-D, last paragraph).
// Rotation by angle th about the unit axis a (Rodrigues):
// Rot = cos th 1 + sin th S(a) + (1 - cos th) a a^T.
template <class T> static void axis_rotation(const double a[3], T th, T Rm[3][3]) {
  const T ct = cos(th), st = sin(th);
  T S[3][3];
  const T aa[3] = {T(a[0]), T(a[1]), T(a[2])};
  skew(aa, S);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rm[i][j] = (i == j ? ct : T(0.0)) + st * S[i][j] + (T(1.0) - ct) * aa[i] * aa[j];
}

// Actuator wrench at the body origin (Sec. III-D: every actuator force acts
// at its own frame). Propellers: thrust k n|n| (0 inside the dead zone) along
// their direction, turned by the linked servo's angle for kind 3. Fins: the
// fin moves through the water with u = v_r + w x r; in the plane normal to
// the span axis a the angle of attack alpha is the angle of u from the
// deflected chord c (towards the fin normal a x c); lift
// 1/2 rho S U^2 C_L(alpha) acts along -(a x u)/U and drag
// 1/2 rho S U^2 C_D(alpha) along -u/U, with C_L = C_L_alpha sin(alpha) cos(alpha),
// C_D = C_D0 + C_D_alpha sin^2(alpha) (reading R18).
template <class T>
static void actuator_wrench(const or_class& c, const T n[8], const T nur[6], T tau[6]) {
  for (int k = 0; k < 6; ++k) tau[k] = T(0.0);
  for (int i = 0; i < c.n_thr; ++i) {
    const int kind = c.act_kind[i];
    T F[3] = {T(0.0), T(0.0), T(0.0)}, r[3], m[3];
    for (int k = 0; k < 3; ++k) r[k] = T(c.thr_pos[i][k]);
    if (kind == 0 || kind == 3) {
      T f = T(0.0);
      if (!(fabs(n[i]) < T(c.deadzone[i]))) f = T(c.k_f[i]) * n[i] * fabs(n[i]);
      T d[3] = {T(c.thr_dir[i][0]), T(c.thr_dir[i][1]), T(c.thr_dir[i][2])};
      if (kind == 3) {
        const int j = c.act_link[i];
        T Rm[3][3];
        axis_rotation(c.act_axis[i], n[j] * T(c.act_range[j]), Rm);
        T d0[3] = {d[0], d[1], d[2]};
        for (int a = 0; a < 3; ++a) d[a] = Rm[a][0] * d0[0] + Rm[a][1] * d0[1] + Rm[a][2] * d0[2];
      }
      for (int k = 0; k < 3; ++k) F[k] = f * d[k];
    } else if (kind == 2) {
      const T w[3] = {nur[3], nur[4], nur[5]};
      T wxr[3], u[3];
      cross(w, r, wxr);
      for (int k = 0; k < 3; ++k) u[k] = nur[k] + wxr[k];
      const T ax[3] = {T(c.act_axis[i][0]), T(c.act_axis[i][1]), T(c.act_axis[i][2])};
      const T ua = u[0] * ax[0] + u[1] * ax[1] + u[2] * ax[2];
      T up[3];
      for (int k = 0; k < 3; ++k) up[k] = u[k] - ua * ax[k];
      const T U2 = up[0] * up[0] + up[1] * up[1] + up[2] * up[2];
      if (val(U2) > 0.0) {
        const T U = sqrt(U2);
        T Rm[3][3];
        axis_rotation(c.act_axis[i], n[i] * T(c.act_range[i]), Rm);
        T ch[3], nrm[3];
        for (int a = 0; a < 3; ++a)
          ch[a] = Rm[a][0] * T(c.act_chord[i][0]) + Rm[a][1] * T(c.act_chord[i][1]) + Rm[a][2] * T(c.act_chord[i][2]);
        cross(ax, ch, nrm);
        const T alpha = atan2(up[0] * nrm[0] + up[1] * nrm[1] + up[2] * nrm[2],
                              up[0] * ch[0] + up[1] * ch[1] + up[2] * ch[2]);
        const T sa = sin(alpha), ca = cos(alpha);
        const T CL = T(c.fin_cl[i]) * sa * ca;
        const T CD = T(c.fin_cd0[i]) + T(c.fin_cda[i]) * sa * sa;
        const T qS = T(0.5 * c.rho * c.fin_area[i]) * U2;
        T axu[3];
        cross(ax, up, axu);
        for (int k = 0; k < 3; ++k) F[k] = -qS * CL * axu[k] / U - qS * CD * up[k] / U;
      }
    }
    cross(r, F, m);
    for (int k = 0; k < 3; ++k) { tau[k] += F[k]; tau[3 + k] += m[k]; }
  }
}

template <class T> static T clamp1(T a) {
  if (a < T(-1.0)) return T(-1.0);
  if (a > T(1.0)) return T(1.0);
  return a;
}

// Body acceleration nu_dot at state (q, nu) with actuator wrench tau.
// form 0: Eq. 3 with nu_r substituted everywhere (reading R2):
//   M_RB nu_dot + C_RB(nu) nu + g_RB = tau + tau_hydro,
//   tau_hydro = -M_A nu_r_dot - C_A(nu_r) nu_r - D(nu_r) nu_r - g_A.
// form 1: the same law rewritten in nu_r alone,
//   M nu_r_dot + C_RB(nu_r) nu_r + C_A(nu_r) nu_r + D(nu_r) nu_r + g = tau,
//   nu_dot = nu_r_dot + nu_c_dot (used only to pin form 0).
template <class T>
static void acceleration(const EnvT<T>& e, const T q[4], const T nu[6], const T tau[6], int form,
                         T nu_dot[6]) {
  T R[3][3];
  rotation(q, R);
  // Current in the body frame and its body-frame derivative.
  T vc[3], w[3] = {nu[3], nu[4], nu[5]};
  for (int i = 0; i < 3; ++i) vc[i] = R[0][i] * T(e.Vc[0]) + R[1][i] * T(e.Vc[1]) + R[2][i] * T(e.Vc[2]);
  T wxvc[3];
  cross(w, vc, wxvc);
  T nuc[6] = {vc[0], vc[1], vc[2], T(0.0), T(0.0), T(0.0)};
  T nuc_dot[6] = {-wxvc[0], -wxvc[1], -wxvc[2], T(0.0), T(0.0), T(0.0)};
  T nur[6];
  for (int i = 0; i < 6; ++i) nur[i] = nu[i] - nuc[i];

  T Mrb[6][6], Ma[6][6], M[6][6];
  mass_rb(e, Mrb);
  mass_a(e, Ma);
  for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) M[i][j] = Mrb[i][j] + Ma[i][j];
  T gRB[6], gA[6];
  restoring(e, R, gRB, gA);
  T Ca[6][6], D[6][6], Crb[6][6];
  coriolis_a(e, nur, Ca);
  damping(e, nur, D);
  T Ca_nur[6], D_nur[6], Crb_x[6];

  T rhs[6];
  if (form == 0) {
    coriolis_rb(e, nu, Crb);
    matvec6(Crb, nu, Crb_x);
    matvec6(Ca, nur, Ca_nur);
    matvec6(D, nur, D_nur);
    T Ma_ncd[6];
    matvec6(Ma, nuc_dot, Ma_ncd);
    // (M_RB + M_A) nu_dot = tau - C_RB(nu)nu - g_RB - C_A(nu_r)nu_r - D(nu_r)nu_r - g_A + M_A nu_c_dot
    for (int i = 0; i < 6; ++i)
      rhs[i] = tau[i] - Crb_x[i] - gRB[i] - Ca_nur[i] - D_nur[i] - gA[i] + Ma_ncd[i];
    solve6(M, rhs, nu_dot);
  } else {
    coriolis_rb(e, nur, Crb);
    matvec6(Crb, nur, Crb_x);
    matvec6(Ca, nur, Ca_nur);
    matvec6(D, nur, D_nur);
    for (int i = 0; i < 6; ++i) rhs[i] = tau[i] - Crb_x[i] - Ca_nur[i] - D_nur[i] - gRB[i] - gA[i];
    T nur_dot[6];
    solve6(M, rhs, nur_dot);
    for (int i = 0; i < 6; ++i) nu_dot[i] = nur_dot[i] + nuc_dot[i];
  }
}

// State layout [21]: p[3] NED, q[4] (w,x,y,z), nu[6] = (u,v,w,p,q,r), n[8].
enum { SP = 0, SQ = 3, SNU = 7, SN = 13, SDIM = 21 };

// Relative velocity nu_r = nu - [R^T V_c ; 0] (Sec. III-B current).
template <class T> static void relative_velocity(const EnvT<T>& e, const T q[4], const T nu[6], T nur[6]) {
  T R[3][3];
  rotation(q, R);
  for (int i = 0; i < 3; ++i)
    nur[i] = nu[i] - (R[0][i] * T(e.Vc[0]) + R[1][i] * T(e.Vc[1]) + R[2][i] * T(e.Vc[2]));
  for (int i = 3; i < 6; ++i) nur[i] = nu[i];
}

// q (x) (0, w): the quaternion kinematics q_dot = 1/2 q (x) (0, w).
template <class T> static void quat_rate(const T q[4], const T nu[6], T qd[4]) {
  const T w = q[0], x = q[1], y = q[2], z = q[3];
  const T P = nu[3], Q = nu[4], Rr = nu[5];
  qd[0] = -x * P - y * Q - z * Rr;
  qd[1] = w * P + y * Rr - z * Q;
  qd[2] = w * Q - x * Rr + z * P;
  qd[3] = w * Rr + x * Q - y * P;
}

// One substep of the discrete map (reading R6: semi-implicit Euler).
template <class T>
static void substep_euler(const or_class& c, const EnvT<T>& e, double h, const T n[8], int form, T s[SDIM]) {
  T q[4] = {s[SQ], s[SQ + 1], s[SQ + 2], s[SQ + 3]};
  T nu[6];
  for (int i = 0; i < 6; ++i) nu[i] = s[SNU + i];
  T nur[6], tau[6];
  relative_velocity(e, q, nu, nur);
  actuator_wrench(c, n, nur, tau);
  T nu_dot[6];
  acceleration(e, q, nu, tau, form, nu_dot);
  for (int i = 0; i < 6; ++i) nu[i] = nu[i] + T(h) * nu_dot[i];
  T R[3][3];
  rotation(q, R);
  for (int i = 0; i < 3; ++i)
    s[SP + i] = s[SP + i] + T(h) * (R[i][0] * nu[0] + R[i][1] * nu[1] + R[i][2] * nu[2]);
  // q <- normalise(q + h/2 q (x) (0, w+)).
  T qd[4], qn[4];
  quat_rate(q, nu, qd);
  for (int i = 0; i < 4; ++i) qn[i] = q[i] + T(0.5 * h) * qd[i];
  T norm = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
  for (int i = 0; i < 4; ++i) s[SQ + i] = qn[i] / norm;
  for (int i = 0; i < 6; ++i) s[SNU + i] = nu[i];
}

// Time derivative of y = (p, q, nu) with the actuator states held (reading
// R19): the attitude of a stage is that of its normalised quaternion.
template <class T>
static void derivative(const or_class& c, const EnvT<T>& e, const T n[8], int form, const T y[13], T dy[13]) {
  const T* q = y + 3;
  const T* nu = y + 7;
  const T qq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const T qh[4] = {q[0] / qq, q[1] / qq, q[2] / qq, q[3] / qq};
  T R[3][3];
  rotation(qh, R);
  for (int i = 0; i < 3; ++i) dy[i] = R[i][0] * nu[0] + R[i][1] * nu[1] + R[i][2] * nu[2];
  T qd[4];
  quat_rate(q, nu, qd);
  for (int i = 0; i < 4; ++i) dy[3 + i] = T(0.5) * qd[i];
  T nur[6], tau[6];
  relative_velocity(e, qh, nu, nur);
  actuator_wrench(c, n, nur, tau);
  acceleration(e, qh, nu, tau, form, dy + 7);
}

// One substep of the classical fourth-order Runge-Kutta variant (reading R19):
// RK4 on (p, q, nu) over h with the actuator states n held, then q normalised.
template <class T>
static void substep_rk4(const or_class& c, const EnvT<T>& e, double h, const T n[8], int form, T s[SDIM]) {
  T y0[13], y[13], k1[13], k2[13], k3[13], k4[13];
  for (int i = 0; i < 13; ++i) y0[i] = s[i];
  derivative(c, e, n, form, y0, k1);
  for (int i = 0; i < 13; ++i) y[i] = y0[i] + T(0.5 * h) * k1[i];
  derivative(c, e, n, form, y, k2);
  for (int i = 0; i < 13; ++i) y[i] = y0[i] + T(0.5 * h) * k2[i];
  derivative(c, e, n, form, y, k3);
  for (int i = 0; i < 13; ++i) y[i] = y0[i] + T(h) * k3[i];
  derivative(c, e, n, form, y, k4);
  for (int i = 0; i < 13; ++i) s[i] = y0[i] + T(h / 6.0) * (k1[i] + T(2.0) * k2[i] + T(2.0) * k3[i] + k4[i]);
  T norm = sqrt(s[SQ] * s[SQ] + s[SQ + 1] * s[SQ + 1] + s[SQ + 2] * s[SQ + 2] + s[SQ + 3] * s[SQ + 3]);
  for (int i = 0; i < 4; ++i) s[SQ + i] = s[SQ + i] / norm;
}

// One substep: actuator states first (n <- n + alpha (c - n), rotor or servo
// lag), then the rigid body with integrator `integ` (0 Euler, 1 RK4).
template <class T>
static void substep(const or_class& c, const EnvT<T>& e, const double alpha[8], double h, const T cmd[8],
                    int form, T s[SDIM], int integ = 0) {
  T n[8];
  for (int i = 0; i < 8; ++i) n[i] = s[SN + i];
  for (int i = 0; i < c.n_thr; ++i) n[i] = n[i] + T(alpha[i]) * (cmd[i] - n[i]);
  if (integ == 1)
    substep_rk4(c, e, h, n, form, s);
  else
    substep_euler(c, e, h, n, form, s);
  for (int i = 0; i < 8; ++i) s[SN + i] = n[i];
}

// Hover-task observation (13) and reward after a control step.
template <class T>
static void observe(const or_class& c, const EnvT<T>& e, double t_ref, const T s[SDIM], const T cmd[8], T obs[13],
                    T* reward) {
  T q[4] = {s[SQ], s[SQ + 1], s[SQ + 2], s[SQ + 3]};
  T R[3][3];
  rotation(q, R);
  double pstar[3];
  reference(e, t_ref, pstar);
  T d[3];
  for (int i = 0; i < 3; ++i) d[i] = s[SP + i] - T(pstar[i]);
  for (int j = 0; j < 3; ++j) obs[j] = R[0][j] * d[0] + R[1][j] * d[1] + R[2][j] * d[2];
  T sgn = (val(q[0]) < 0.0) ? T(-1.0) : T(1.0);
  for (int i = 0; i < 4; ++i) obs[3 + i] = sgn * q[i];
  for (int i = 0; i < 6; ++i) obs[7 + i] = s[SNU + i];
  T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  T vv = T(0.0);
  for (int i = 0; i < 6; ++i) vv += s[SNU + i] * s[SNU + i];
  T cc = T(0.0);
  for (int i = 0; i < c.n_thr; ++i) cc += cmd[i] * cmd[i];
  *reward = -dd - T(0.1) * vv - T(0.01) * cc;
}

static void rotor_alpha(const or_class& c, double h, double alpha[8]) {
  for (int i = 0; i < 8; ++i) alpha[i] = 1.0;
  for (int i = 0; i < c.n_thr; ++i) alpha[i] = (c.T_rotor[i] > 0.0) ? 1.0 - std::exp(-h / c.T_rotor[i]) : 1.0;
}

template <class T> static EnvT<T> env_of(const or_env& in) {
  EnvT<T> e;
  e.mass = in.mass;
  for (int i = 0; i < 3; ++i) {
    e.Ig[i] = in.Ig[i]; e.rg[i] = in.rg[i]; e.rb[i] = in.rb[i];
    e.Vc[i] = in.Vc[i]; e.target[i] = in.target[i];
  }
  e.W = in.W; e.B = in.B;
  for (int i = 0; i < 6; ++i) { e.Ma[i] = T(in.Ma[i]); e.dl[i] = T(in.dl[i]); e.dq[i] = T(in.dq[i]); }
  for (int i = 0; i < 3; ++i) {
    e.ta[i] = in.traj_a[i]; e.tw[i] = in.traj_w[i]; e.tph[i] = in.traj_phi[i]; e.tv[i] = in.traj_v[i];
  }
  e.k0 = in.k0;
  for (int i = 0; i < 3; ++i) e.Ig_off[i] = in.Ig_off[i];
  return e;
}

}  // namespace orc

using namespace orc;

extern "C" {

int or_philox4x64(const uint64_t* ctr, const uint64_t* key, uint64_t* out) {
  philox4x64_10(ctr, key, out);
  return 0;
}

double or_uniform(uint64_t seed, uint64_t stream, uint64_t env, uint64_t j) {
  return draw_u(seed, stream, env, j);
}

// Serving-loop action: a(seed, env, step, thr) in [-1, 1), 24-bit grid, from
// one Philox4x64-10 block under key (seed, 3), counter (env, step, 0, 0):
// word thr % 4, its top 24 bits for thr < 4 and bits 31..8 for thr = 4..7;
// a = k/2^23 - 1.
float or_action(uint64_t seed, uint64_t env, uint64_t step, int thr) {
  uint64_t ctr[4] = {env, step, 0, 0}, key[2] = {seed, kStreamAction}, out[4];
  philox4x64_10(ctr, key, out);
  const uint64_t w = out[thr % 4];
  double k = (double)(thr < 4 ? (w >> 40) : ((w >> 8) & 0xFFFFFFull));
  return (float)(k * (1.0 / 8388608.0) - 1.0);
}

// Attach a point mass m_p at r_p (body frame) to an env whose CoG is at r_g
// (Sec. III-B mission payloads). The payload's volume is neglected. The
// combined body has mass m' = m + m_p, CoG r_g' = (m r_g + m_p r_p) / m' and,
// by the parallel-axis theorem, inertia about r_g'
// I' = I + m (|d|^2 1 - d d^T) + m_p (|d_p|^2 1 - d_p d_p^T),
// d = r_g - r_g', d_p = r_p - r_g'; the payload's weight m_p g adds to W.
void or_attach_payload(or_env* env, double mp, const double* rp) {
  or_env& e = *env;
  const double m = e.mass, mt = m + mp;
  double rg[3], d[3], dp[3];
  for (int i = 0; i < 3; ++i) rg[i] = (m * e.rg[i] + mp * rp[i]) / mt;
  for (int i = 0; i < 3; ++i) { d[i] = e.rg[i] - rg[i]; dp[i] = rp[i] - rg[i]; }
  const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double dp2 = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
  // Current inertia about the CoG as a full tensor (products from Ig_off).
  const double I0[3][3] = {{e.Ig[0], e.Ig_off[0], e.Ig_off[1]},
                           {e.Ig_off[0], e.Ig[1], e.Ig_off[2]},
                           {e.Ig_off[1], e.Ig_off[2], e.Ig[2]}};
  double I[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      I[i][j] = I0[i][j] + m * ((i == j ? d2 : 0.0) - d[i] * d[j]) + mp * ((i == j ? dp2 : 0.0) - dp[i] * dp[j]);
  e.mass = mt;
  for (int i = 0; i < 3; ++i) { e.Ig[i] = I[i][i]; e.rg[i] = rg[i]; }
  e.Ig_off[0] = I[0][1]; e.Ig_off[1] = I[0][2]; e.Ig_off[2] = I[1][2];
  e.W += mp * kGravity;
}

// Reset: domain-randomised parameters (Sec. III-C, Table 2) and initial state.
// Draw numbers of stream 1 (per env): 0 mass, 1-6 added mass, 7-12 linear
// damping, 13-18 quadratic damping, 19 CoB offset, 20 current speed,
// 21 current heading, 22 current vertical (3D variant).
// Draw numbers of stream 2: 0-2 target, 3 radius, 4-5 offset direction,
// 6-7 rotation axis, 8 rotation angle.
// env_ids (may be NULL): the env index each record's draws are keyed by
// (default: the record index).
int or_reset(const or_class* classes, int n_classes, const int32_t* env_class, int64_t n_envs,
             const or_reset_cfg* cfg, uint64_t seed, const int64_t* env_ids, or_env* envs, double* state) {
  for (int64_t ei = 0; ei < n_envs; ++ei) {
    const int ci = env_class[ei];
    if (ci < 0 || ci >= n_classes) return -1;
    const or_class& c = classes[ci];
    or_env& e = envs[ei];
    std::memset(&e, 0, sizeof(e));
    e.cls = ci;
    const uint64_t id = env_ids ? (uint64_t)env_ids[ei] : (uint64_t)ei;
    auto f = [&](int j, double lo, double hi) {
      return cfg->dr_enabled ? lo + (hi - lo) * draw_u(seed, kStreamDR, id, j) : 1.0;
    };
    const double fm = f(0, cfg->mass_lo, cfg->mass_hi);
    e.mass = c.mass * fm;
    for (int i = 0; i < 3; ++i) { e.Ig[i] = c.Ig[i] * fm; e.rg[i] = c.rg[i]; }
    for (int i = 0; i < 6; ++i) {
      e.Ma[i] = c.Ma[i] * f(1 + i, cfg->added_lo, cfg->added_hi);
      e.dl[i] = c.dl[i] * f(7 + i, cfg->damp_lo, cfg->damp_hi);
      e.dq[i] = c.dq[i] * f(13 + i, cfg->damp_lo, cfg->damp_hi);
    }
    const double fb = f(19, cfg->cob_lo, cfg->cob_hi);
    for (int i = 0; i < 3; ++i) e.rb[i] = c.rb[i] * fb;
    e.W = e.mass * kGravity;
    e.B = c.buoy_ratio * c.mass * kGravity;   // volume is not randomised
    if (cfg->payload) {
      // Payload (stream 1, draws 23-26): mass fraction of the vehicle's mass
      // U[lo, hi] (Table 2), position x, y ~ U[-0.1, 0.1] m, z ~ U[0.05, 0.15] m.
      const double mp = e.mass * (cfg->payload_lo + (cfg->payload_hi - cfg->payload_lo) *
                                                         draw_u(seed, kStreamDR, id, 23));
      const double rp[3] = {-0.1 + 0.2 * draw_u(seed, kStreamDR, id, 24), -0.1 + 0.2 * draw_u(seed, kStreamDR, id, 25),
                            0.05 + 0.1 * draw_u(seed, kStreamDR, id, 26)};
      or_attach_payload(&e, mp, rp);
    }
    if (cfg->current_enabled) {
      const double speed = cfg->cur_lo + (cfg->cur_hi - cfg->cur_lo) * draw_u(seed, kStreamDR, id, 20);
      const double psi = 2.0 * kPi * draw_u(seed, kStreamDR, id, 21);
      if (cfg->current_3d) {
        const double zc = 2.0 * draw_u(seed, kStreamDR, id, 22) - 1.0;
        const double rh = std::sqrt(1.0 - zc * zc);
        e.Vc[0] = speed * rh * std::cos(psi); e.Vc[1] = speed * rh * std::sin(psi); e.Vc[2] = speed * zc;
      } else {
        e.Vc[0] = speed * std::cos(psi); e.Vc[1] = speed * std::sin(psi); e.Vc[2] = 0.0;
      }
    }
    double* s = state + ei * SDIM;
    for (int i = 0; i < SDIM; ++i) s[i] = 0.0;
    s[SQ] = 1.0;
    if (cfg->init_mode == 1 || cfg->track)
      for (int i = 0; i < 3; ++i)
        e.target[i] = cfg->target_half * (2.0 * draw_u(seed, kStreamInit, id, i) - 1.0);
    if (cfg->track) {
      // Helix: c + (R cos(W t + psi), R sin(W t + psi), v_z t), written with
      // sin(x + pi/2) = cos(x). Lissajous: c + a o sin(w t + phi).
      if (cfg->track_kind == 0) {
        const double R = 1.0 + 2.0 * draw_u(seed, kStreamInit, id, 9);
        const double W = 0.2 + 0.4 * draw_u(seed, kStreamInit, id, 10);
        const double psi = 2.0 * kPi * draw_u(seed, kStreamInit, id, 11);
        const double vz = -0.2 + 0.4 * draw_u(seed, kStreamInit, id, 12);
        e.traj_a[0] = R; e.traj_a[1] = R;
        e.traj_w[0] = W; e.traj_w[1] = W;
        e.traj_phi[0] = psi + 0.5 * kPi; e.traj_phi[1] = psi;
        e.traj_v[2] = vz;
      } else {
        for (int i = 0; i < 3; ++i) {
          e.traj_a[i] = 1.0 + 2.0 * draw_u(seed, kStreamInit, id, 9 + i);
          e.traj_w[i] = 0.2 + 0.4 * draw_u(seed, kStreamInit, id, 12 + i);
          e.traj_phi[i] = 2.0 * kPi * draw_u(seed, kStreamInit, id, 15 + i);
        }
      }
    }
    if (cfg->init_mode == 1) {
      double p0[3];
      for (int i = 0; i < 3; ++i) p0[i] = e.target[i] + e.traj_a[i] * std::sin(e.traj_phi[i]);
      const double rad = cfg->pos_radius * std::cbrt(draw_u(seed, kStreamInit, id, 3));
      const double zd = 2.0 * draw_u(seed, kStreamInit, id, 4) - 1.0;
      const double ph = 2.0 * kPi * draw_u(seed, kStreamInit, id, 5);
      const double rd = std::sqrt(1.0 - zd * zd);
      const double dir[3] = {rd * std::cos(ph), rd * std::sin(ph), zd};
      for (int i = 0; i < 3; ++i) s[SP + i] = p0[i] + rad * dir[i];
      const double za = 2.0 * draw_u(seed, kStreamInit, id, 6) - 1.0;
      const double pa = 2.0 * kPi * draw_u(seed, kStreamInit, id, 7);
      const double ra = std::sqrt(1.0 - za * za);
      const double ax[3] = {ra * std::cos(pa), ra * std::sin(pa), za};
      const double ang = cfg->max_angle * draw_u(seed, kStreamInit, id, 8);
      s[SQ] = std::cos(0.5 * ang);
      for (int i = 0; i < 3; ++i) s[SQ + 1 + i] = std::sin(0.5 * ang) * ax[i];
    }
  }
  return 0;
}

// Roll out n_steps control steps of K substeps each (zero-order hold of the
// clamped command). actions: [n_steps][n_envs][8] float32 (entries beyond the
// class's thruster count are ignored). state: [n_envs][21] in/out.
// obs: [n_steps][n_envs][13] or NULL; reward: [n_steps][n_envs] or NULL.
int or_rollout(const or_class* classes, const or_env* envs, int64_t n_envs, double dt, int K, int n_steps,
               const float* actions, double* state, double* obs, double* reward, int form, int n_threads,
               int integ) {
  if (K < 1 || dt <= 0.0) return -1;
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
  for (int64_t ei = 0; ei < n_envs; ++ei) {
    const or_env& ein = envs[ei];
    const or_class& c = classes[ein.cls];
    const EnvT<double> e = env_of<double>(ein);
    const double h = dt / K;
    double alpha[8];
    rotor_alpha(c, h, alpha);
    double* s = state + ei * SDIM;
    for (int t = 0; t < n_steps; ++t) {
      double cmd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      const float* a = actions + ((int64_t)t * n_envs + ei) * 8;
      for (int i = 0; i < c.n_thr; ++i) cmd[i] = clamp1((double)a[i]);
      for (int k = 0; k < K; ++k) substep(c, e, alpha, h, cmd, form, s, integ);
      if (obs || reward) {
        double o[13], r;
        observe(c, e, (e.k0 + t + 1) * dt, s, cmd, o, &r);
        if (obs) for (int i = 0; i < 13; ++i) obs[((int64_t)t * n_envs + ei) * 13 + i] = o[i];
        if (reward) reward[(int64_t)t * n_envs + ei] = r;
      }
    }
  }
  return 0;
}

// Forward-mode directional derivative of a rollout (dual numbers). Tangent
// inputs: d_actions [n_steps][n_envs][8], d_state0 [n_envs][21],
// d_Ma/d_dl/d_dq [n_envs][6] (any may be NULL = 0). Outputs: values as in
// or_rollout plus tangents d_state [n_envs][21], d_obs, d_reward. integ: the
// integrator of the substep (0 semi-implicit Euler, 1 RK4), as in or_rollout.
int or_rollout_jvp(const or_class* classes, const or_env* envs, int64_t n_envs, double dt, int K, int n_steps,
                   const float* actions, const double* d_actions, double* state, const double* d_state0,
                   const double* d_Ma, const double* d_dl, const double* d_dq, double* d_state, double* obs,
                   double* d_obs, double* reward, double* d_reward, int n_threads, int integ) {
  if (K < 1 || dt <= 0.0 || integ < 0 || integ > 1) return -1;
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
  for (int64_t ei = 0; ei < n_envs; ++ei) {
    const or_env& ein = envs[ei];
    const or_class& c = classes[ein.cls];
    EnvT<Dual> e = env_of<Dual>(ein);
    for (int i = 0; i < 6; ++i) {
      if (d_Ma) e.Ma[i].d = d_Ma[ei * 6 + i];
      if (d_dl) e.dl[i].d = d_dl[ei * 6 + i];
      if (d_dq) e.dq[i].d = d_dq[ei * 6 + i];
    }
    const double h = dt / K;
    double alpha[8];
    rotor_alpha(c, h, alpha);
    Dual s[SDIM];
    for (int i = 0; i < SDIM; ++i) s[i] = Dual(state[ei * SDIM + i], d_state0 ? d_state0[ei * SDIM + i] : 0.0);
    for (int t = 0; t < n_steps; ++t) {
      Dual cmd[8];
      const int64_t ai = ((int64_t)t * n_envs + ei) * 8;
      for (int i = 0; i < c.n_thr; ++i)
        cmd[i] = clamp1(Dual((double)actions[ai + i], d_actions ? d_actions[ai + i] : 0.0));
      for (int k = 0; k < K; ++k) substep(c, e, alpha, h, cmd, 0, s, integ);
      Dual o[13], r;
      observe(c, e, (e.k0 + t + 1) * dt, s, cmd, o, &r);
      for (int i = 0; i < 13; ++i) {
        const int64_t oi = ((int64_t)t * n_envs + ei) * 13 + i;
        if (obs) obs[oi] = o[i].v;
        if (d_obs) d_obs[oi] = o[i].d;
      }
      if (reward) reward[(int64_t)t * n_envs + ei] = r.v;
      if (d_reward) d_reward[(int64_t)t * n_envs + ei] = r.d;
    }
    for (int i = 0; i < SDIM; ++i) {
      state[ei * SDIM + i] = s[i].v;
      if (d_state) d_state[ei * SDIM + i] = s[i].d;
    }
  }
  return 0;
}

// --- Pieces exposed for the CPU pins ---------------------------------------

int or_rotation(const double* q, double* R9) {
  double R[3][3];
  rotation(q, R);
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) R9[3 * i + j] = R[i][j];
  return 0;
}

// C_RB(nu), C_A(nu_r) as row-major 6x6 for the passivity pin.
int or_coriolis(const or_env* env, const double* nu, double* Crb36, double* Ca36) {
  EnvT<double> e = env_of<double>(*env);
  double Crb[6][6], Ca[6][6];
  coriolis_rb(e, nu, Crb);
  coriolis_a(e, nu, Ca);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) { Crb36[6 * i + j] = Crb[i][j]; Ca36[6 * i + j] = Ca[i][j]; }
  return 0;
}

// M = M_RB + M_A as row-major 6x6.
int or_mass(const or_env* env, double* M36) {
  EnvT<double> e = env_of<double>(*env);
  double Mrb[6][6], Ma[6][6];
  mass_rb(e, Mrb);
  mass_a(e, Ma);
  for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) M36[6 * i + j] = Mrb[i][j] + Ma[i][j];
  return 0;
}

// Total restoring vector g(eta) = g_RB + g_A at attitude q.
int or_restoring(const or_env* env, const double* q, double* g6) {
  EnvT<double> e = env_of<double>(*env);
  double R[3][3], gRB[6], gA[6];
  rotation(q, R);
  restoring(e, R, gRB, gA);
  for (int i = 0; i < 6; ++i) g6[i] = gRB[i] + gA[i];
  return 0;
}

// Actuator wrench for actuator states n[8] and relative velocity nu_r (NULL: at rest).
int or_actuator_wrench(const or_class* c, const double* n, const double* nur6, double* tau6) {
  const double zero[6] = {0, 0, 0, 0, 0, 0};
  actuator_wrench(*c, n, nur6 ? nur6 : zero, tau6);
  return 0;
}

// nu_dot for a given state s[21] and actuator wrench, either form.
int or_acceleration(const or_env* env, const double* s, const double* tau, int form, double* nu_dot) {
  EnvT<double> e = env_of<double>(*env);
  acceleration(e, s + SQ, s + SNU, tau, form, nu_dot);
  return 0;
}

int or_state_dim(void) { return SDIM; }
int or_sizeof_class(void) { return (int)sizeof(or_class); }
int or_sizeof_env(void) { return (int)sizeof(or_env); }
int or_sizeof_reset_cfg(void) { return (int)sizeof(or_reset_cfg); }

}  // extern "C"
