// Host check of the step kernel's vector-Jacobian product (vjp_from_tape in
// mg_device.cuh on the tape that tape_from_states rebuilds from a substep's
// start and end states: the arithmetic the adjoint kernel runs) in FP64: for random
// states, commands, parameters and directions d, the product's
// <vjp(lambda), d> must equal <lambda, J d> from central differences of the
// forward substep (h = 1e-6), over the state, the commands and the added-mass
// and damping coefficients (the inverse mass matrix follows the added mass).
// Prints the worst relative difference and, with a nonzero argument, the
// same for a product whose added-mass gradient is scaled by 1.01 (the check
// must see that). For the vehicle alone, with a point-mass payload, and for a
// class with fins and a servo-tilted propeller; the semi-implicit Euler substep
// (vjp_from_tape) and RK4 (substep_rk4_vjp).
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <random>
#include "mg_device.cuh"
using namespace mg;
template <int NT>
struct In { St<double, NT> x; double c[NT]; double A[6], dl[6], dq[6]; };
template <int NT, bool RK = false>
void fwd(const In<NT>& in, const Phys<double>& P0, const Act<double>& Ac, double h, St<double, NT>& out) {
  Phys<double> P = P0;
  const double Mrb[6] = {P0.m, P0.m, P0.m, P0.Ig[0], P0.Ig[1], P0.Ig[2]};
  for (int j = 0; j < 6; ++j) { P.A[j] = in.A[j]; P.dl[j] = in.dl[j]; P.dq[j] = in.dq[j]; P.minv[j] = 1.0 / (Mrb[j] + in.A[j]); }
  out = in.x;
  double c[NT]; for (int i = 0; i < NT; ++i) c[i] = in.c[i];
  if constexpr (RK) substep_rk4<double, NT>(out, c, P, Ac, h);
  else substep<double, NT, false>(out, c, P, Ac, h, nullptr);
}
static double g_scale = 1.0;

template <int NT, bool RK = false>
double run(std::mt19937_64& rng) {
  std::uniform_real_distribution<double> U(-1, 1), P01(0.2, 2.0);
  Phys<double> P; Act<double> Ac; In<NT> in;
  P.m = 12; P.W = 110; P.B = 113;
  for (int j = 0; j < 3; ++j) { P.Ig[j] = P01(rng); P.rb[j] = U(rng) * 0.05; P.Vc[j] = U(rng) * 0.4; }
  for (int j = 0; j < 6; ++j) { in.A[j] = P01(rng) * 3; in.dl[j] = P01(rng) * 5; in.dq[j] = P01(rng) * 10; }
  for (int r = 0; r < 6; ++r) for (int i = 0; i < 8; ++i) Ac.alloc[r][i] = i < NT ? U(rng) : 0;
  for (int i = 0; i < 8; ++i) { Ac.kf[i] = P01(rng) * 20; Ac.dz[i] = 0.0; Ac.alpha[i] = P01(rng) * 0.4; }
  const double h = 0.0025;
  for (int j = 0; j < 3; ++j) in.x.p[j] = U(rng);
  for (int j = 0; j < 4; ++j) in.x.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) in.x.nu[j] = U(rng);
  for (int j = 0; j < NT; ++j) in.x.n[j] = U(rng);
  for (int j = 0; j < NT; ++j) in.c[j] = U(rng);
  // VJP at the base point
  Phys<double> Pb = P;
  const double Mrb[6] = {P.m, P.m, P.m, P.Ig[0], P.Ig[1], P.Ig[2]};
  for (int j = 0; j < 6; ++j) { Pb.A[j] = in.A[j]; Pb.dl[j] = in.dl[j]; Pb.dq[j] = in.dq[j]; Pb.minv[j] = 1.0 / (Mrb[j] + in.A[j]); }
  St<double, NT> x = in.x; Tape<double, NT> tp;
  substep<double, NT, true>(x, in.c, Pb, Ac, h, &tp);
  St<double, NT> lam; for (int j = 0; j < 3; ++j) lam.p[j] = U(rng); for (int j = 0; j < 4; ++j) lam.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) lam.nu[j] = U(rng); for (int j = 0; j < NT; ++j) lam.n[j] = U(rng);
  // As the reverse pass: the tape from the start and end states.
  Tape<double, NT> tr;
  tape_from_states<double, NT>(in.x, x, Pb, h, 1.0 / h, tr);
  St<double, NT> xn = in.x;
  for (int j = 0; j < NT; ++j) xn.n[j] = x.n[j];
  St<double, NT> lx = lam; double lc[NT] = {}; HydroGrad<double> g{};
  if constexpr (RK) substep_rk4_vjp<double, NT, Act<double>, Phys<double>, true, NoGen, true>(xn, in.c, Pb, Ac, h, lx, lc, g);
  else vjp_from_tape<double, NT>(in.x, x.q, tr, in.c, Pb, Ac, h, lx, lc, g);
  // random direction
  In<NT> d;
  for (int j = 0; j < 3; ++j) d.x.p[j] = U(rng); for (int j = 0; j < 4; ++j) d.x.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) d.x.nu[j] = U(rng); for (int j = 0; j < NT; ++j) d.x.n[j] = U(rng);
  for (int j = 0; j < NT; ++j) d.c[j] = U(rng);
  for (int j = 0; j < 6; ++j) { d.A[j] = U(rng); d.dl[j] = U(rng); d.dq[j] = U(rng); }
  const double eps = 1e-6;
  auto shift = [&](double s) { In<NT> o = in;
    for (int j = 0; j < 3; ++j) o.x.p[j] += s * d.x.p[j]; for (int j = 0; j < 4; ++j) o.x.q[j] += s * d.x.q[j];
    for (int j = 0; j < 6; ++j) o.x.nu[j] += s * d.x.nu[j]; for (int j = 0; j < NT; ++j) o.x.n[j] += s * d.x.n[j];
    for (int j = 0; j < NT; ++j) o.c[j] += s * d.c[j];
    for (int j = 0; j < 6; ++j) { o.A[j] += s * d.A[j]; o.dl[j] += s * d.dl[j]; o.dq[j] += s * d.dq[j]; }
    return o; };
  St<double, NT> yp, ym; fwd<NT, RK>(shift(eps), P, Ac, h, yp); fwd<NT, RK>(shift(-eps), P, Ac, h, ym);
  double fd = 0;
  for (int j = 0; j < 3; ++j) fd += lam.p[j] * (yp.p[j] - ym.p[j]); for (int j = 0; j < 4; ++j) fd += lam.q[j] * (yp.q[j] - ym.q[j]);
  for (int j = 0; j < 6; ++j) fd += lam.nu[j] * (yp.nu[j] - ym.nu[j]); for (int j = 0; j < NT; ++j) fd += lam.n[j] * (yp.n[j] - ym.n[j]);
  fd /= 2 * eps;
  double an = 0;
  for (int j = 0; j < 3; ++j) an += lx.p[j] * d.x.p[j]; for (int j = 0; j < 4; ++j) an += lx.q[j] * d.x.q[j];
  for (int j = 0; j < 6; ++j) an += lx.nu[j] * d.x.nu[j]; for (int j = 0; j < NT; ++j) an += lx.n[j] * d.x.n[j];
  for (int j = 0; j < NT; ++j) an += lc[j] * d.c[j];
  for (int j = 0; j < 6; ++j) an += g_scale * g.A[j] * d.A[j] + g.dl[j] * d.dl[j] + g.dq[j] * d.dq[j];
  return std::fabs(fd - an) / std::max(1.0, std::fabs(fd));
}

// Payload runs: the combined body (vehicle + point mass) about the body
// origin, with its full inverse recomputed from M_RB + diag(A) for every
// perturbation of the added mass.
template <typename S>
struct PhysPay {
  static constexpr bool kFull = true;
  S A[6], dl[6], dq[6], B, rb[3], Vc[3], Mi[21], Io[6], s[3], m, W;
};

static bool invert6(double M[6][6], double Mi[6][6]) {
  double a[6][12];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 12; ++j) a[i][j] = j < 6 ? M[i][j] : (j - 6 == i ? 1.0 : 0.0);
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    if (std::fabs(a[piv][c]) < 1e-300) return false;
    for (int j = 0; j < 12; ++j) std::swap(a[c][j], a[piv][j]);
    const double d = a[c][c];
    for (int j = 0; j < 12; ++j) a[c][j] /= d;
    for (int r = 0; r < 6; ++r)
      if (r != c) {
        const double f = a[r][c];
        for (int j = 0; j < 12; ++j) a[r][j] -= f * a[c][j];
      }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Mi[i][j] = a[i][6 + j];
  return true;
}

static void pay_fill(PhysPay<double>& P, const double A[6]) {
  const double Ss[3][3] = {{0, -P.s[2], P.s[1]}, {P.s[2], 0, -P.s[0]}, {-P.s[1], P.s[0], 0}};
  const double Io[3][3] = {{P.Io[0], P.Io[1], P.Io[2]}, {P.Io[1], P.Io[3], P.Io[4]}, {P.Io[2], P.Io[4], P.Io[5]}};
  double M[6][6], Mi[6][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      M[i][j] = (i == j) ? P.m + A[i] : 0.0;
      M[i][3 + j] = -Ss[i][j];
      M[3 + i][j] = Ss[i][j];
      M[3 + i][3 + j] = Io[i][j] + (i == j ? A[3 + i] : 0.0);
    }
  invert6(M, Mi);
  int q = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) P.Mi[q++] = 0.5 * (Mi[i][j] + Mi[j][i]);
  for (int j = 0; j < 6; ++j) P.A[j] = A[j];
}

template <int NT, bool RK = false>
double run_pay(std::mt19937_64& rng) {
  std::uniform_real_distribution<double> U(-1, 1), P01(0.2, 2.0);
  PhysPay<double> P; Act<double> Ac; In<NT> in;
  const double mp = 3.0, rp[3] = {U(rng) * 0.3, U(rng) * 0.3, U(rng) * 0.3};
  const double m = 12, Ig[3] = {P01(rng), P01(rng), P01(rng)};
  P.m = m + mp; P.W = 110 + mp * 9.81; P.B = 113;
  for (int j = 0; j < 3; ++j) { P.s[j] = mp * rp[j]; P.rb[j] = U(rng) * 0.05; P.Vc[j] = U(rng) * 0.4; }
  const double rp2 = rp[0] * rp[0] + rp[1] * rp[1] + rp[2] * rp[2];
  P.Io[0] = Ig[0] + mp * (rp2 - rp[0] * rp[0]); P.Io[1] = -mp * rp[0] * rp[1]; P.Io[2] = -mp * rp[0] * rp[2];
  P.Io[3] = Ig[1] + mp * (rp2 - rp[1] * rp[1]); P.Io[4] = -mp * rp[1] * rp[2]; P.Io[5] = Ig[2] + mp * (rp2 - rp[2] * rp[2]);
  for (int j = 0; j < 6; ++j) { in.A[j] = P01(rng) * 3; in.dl[j] = P01(rng) * 5; in.dq[j] = P01(rng) * 10; }
  for (int r = 0; r < 6; ++r) for (int i = 0; i < 8; ++i) Ac.alloc[r][i] = i < NT ? U(rng) : 0;
  for (int i = 0; i < 8; ++i) { Ac.kf[i] = P01(rng) * 20; Ac.dz[i] = 0.0; Ac.alpha[i] = P01(rng) * 0.4; }
  const double h = 0.0025;
  for (int j = 0; j < 3; ++j) in.x.p[j] = U(rng);
  for (int j = 0; j < 4; ++j) in.x.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) in.x.nu[j] = U(rng);
  for (int j = 0; j < NT; ++j) in.x.n[j] = U(rng);
  for (int j = 0; j < NT; ++j) in.c[j] = U(rng);
  auto fwd_pay = [&](const In<NT>& i2, St<double, NT>& out) {
    PhysPay<double> Q = P;
    pay_fill(Q, i2.A);
    for (int j = 0; j < 6; ++j) { Q.dl[j] = i2.dl[j]; Q.dq[j] = i2.dq[j]; }
    out = i2.x;
    double c[NT]; for (int k = 0; k < NT; ++k) c[k] = i2.c[k];
    if constexpr (RK) substep_rk4<double, NT>(out, c, Q, Ac, h);
    else substep<double, NT, false>(out, c, Q, Ac, h, nullptr);
  };
  PhysPay<double> Pb = P;
  pay_fill(Pb, in.A);
  for (int j = 0; j < 6; ++j) { Pb.dl[j] = in.dl[j]; Pb.dq[j] = in.dq[j]; }
  St<double, NT> x = in.x; Tape<double, NT> tp;
  substep<double, NT, true>(x, in.c, Pb, Ac, h, &tp);
  St<double, NT> lam; for (int j = 0; j < 3; ++j) lam.p[j] = U(rng); for (int j = 0; j < 4; ++j) lam.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) lam.nu[j] = U(rng); for (int j = 0; j < NT; ++j) lam.n[j] = U(rng);
  // The reverse pass rebuilds the tape from the start and end states.
  Tape<double, NT> tr;
  tape_from_states<double, NT>(in.x, x, Pb, h, 1.0 / h, tr);
  St<double, NT> xn = in.x;
  for (int j = 0; j < NT; ++j) xn.n[j] = x.n[j];
  St<double, NT> lx = lam; double lc[NT] = {}; HydroGrad<double> g{};
  if constexpr (RK)
    substep_rk4_vjp<double, NT, Act<double>, PhysPay<double>, true, NoGen, true>(xn, in.c, Pb, Ac, h, lx, lc, g);
  else vjp_from_tape<double, NT>(in.x, x.q, tr, in.c, Pb, Ac, h, lx, lc, g);
  In<NT> d;
  for (int j = 0; j < 3; ++j) d.x.p[j] = U(rng); for (int j = 0; j < 4; ++j) d.x.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) d.x.nu[j] = U(rng); for (int j = 0; j < NT; ++j) d.x.n[j] = U(rng);
  for (int j = 0; j < NT; ++j) d.c[j] = U(rng);
  for (int j = 0; j < 6; ++j) { d.A[j] = U(rng); d.dl[j] = U(rng); d.dq[j] = U(rng); }
  const double eps = 1e-6;
  auto shift = [&](double sc) { In<NT> o = in;
    for (int j = 0; j < 3; ++j) o.x.p[j] += sc * d.x.p[j]; for (int j = 0; j < 4; ++j) o.x.q[j] += sc * d.x.q[j];
    for (int j = 0; j < 6; ++j) o.x.nu[j] += sc * d.x.nu[j]; for (int j = 0; j < NT; ++j) o.x.n[j] += sc * d.x.n[j];
    for (int j = 0; j < NT; ++j) o.c[j] += sc * d.c[j];
    for (int j = 0; j < 6; ++j) { o.A[j] += sc * d.A[j]; o.dl[j] += sc * d.dl[j]; o.dq[j] += sc * d.dq[j]; }
    return o; };
  St<double, NT> yp, ym; fwd_pay(shift(eps), yp); fwd_pay(shift(-eps), ym);
  double fd = 0;
  for (int j = 0; j < 3; ++j) fd += lam.p[j] * (yp.p[j] - ym.p[j]); for (int j = 0; j < 4; ++j) fd += lam.q[j] * (yp.q[j] - ym.q[j]);
  for (int j = 0; j < 6; ++j) fd += lam.nu[j] * (yp.nu[j] - ym.nu[j]); for (int j = 0; j < NT; ++j) fd += lam.n[j] * (yp.n[j] - ym.n[j]);
  fd /= 2 * eps;
  double an = 0;
  for (int j = 0; j < 3; ++j) an += lx.p[j] * d.x.p[j]; for (int j = 0; j < 4; ++j) an += lx.q[j] * d.x.q[j];
  for (int j = 0; j < 6; ++j) an += lx.nu[j] * d.x.nu[j]; for (int j = 0; j < NT; ++j) an += lx.n[j] * d.x.n[j];
  for (int j = 0; j < NT; ++j) an += lc[j] * d.c[j];
  for (int j = 0; j < 6; ++j) an += g_scale * g.A[j] * d.A[j] + g.dl[j] * d.dl[j] + g.dq[j] * d.dq[j];
  return std::fabs(fd - an) / std::max(1.0, std::fabs(fd));
}

// A generic class on the host: 4 fixed propellers, a servo, a propeller
// tilted by that servo and 2 fins (table values random; the check is about
// derivatives, not about a particular vehicle).
struct GenH {
  int k[8];
  double vals[8][20];
  int kind(int i) const { return k[i]; }
  double v(int i, int j) const { return vals[i][j]; }
};

template <int NT, bool RK = false>
double run_gen(std::mt19937_64& rng) {
  static_assert(NT == 8, "channel layout of the generic check");
  std::uniform_real_distribution<double> U(-1, 1), P01(0.2, 2.0);
  Phys<double> P; Act<double> Ac; In<NT> in; GenH G;
  P.m = 12; P.W = 110; P.B = 113;
  for (int j = 0; j < 3; ++j) { P.Ig[j] = P01(rng); P.rb[j] = U(rng) * 0.05; P.Vc[j] = U(rng) * 0.4; }
  for (int j = 0; j < 6; ++j) { in.A[j] = P01(rng) * 3; in.dl[j] = P01(rng) * 5; in.dq[j] = P01(rng) * 10; }
  for (int i = 0; i < 8; ++i) {
    G.k[i] = i < 4 ? KIND_PROP : (i == 4 ? KIND_SERVO : (i == 5 ? KIND_TILT : KIND_FIN));
    for (int j = 0; j < 20; ++j) G.vals[i][j] = U(rng);
    for (int r = 0; r < 6; ++r) Ac.alloc[r][i] = i < 4 ? U(rng) : 0.0;
    Ac.kf[i] = (i < 4 || i == 5) ? P01(rng) * 20 : 0.0;
    Ac.dz[i] = 0.0;
    Ac.alpha[i] = P01(rng) * 0.4;
  }
  G.vals[5][18] = 4;      // the tilted propeller follows the servo
  G.vals[5][19] = 0.8;    // tilt range (rad)
  for (int i = 6; i < 8; ++i) { G.vals[i][12] = 3.0; G.vals[i][13] = 0.5; G.vals[i][14] = 2.0; G.vals[i][15] = 0.5; }
  const double h = 0.0025;
  for (int j = 0; j < 3; ++j) in.x.p[j] = U(rng);
  for (int j = 0; j < 4; ++j) in.x.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) in.x.nu[j] = U(rng);
  for (int j = 0; j < NT; ++j) in.x.n[j] = U(rng);
  for (int j = 0; j < NT; ++j) in.c[j] = U(rng);
  auto phys_of = [&](const In<NT>& i2) {
    Phys<double> Q = P;
    const double Mrb[6] = {P.m, P.m, P.m, P.Ig[0], P.Ig[1], P.Ig[2]};
    for (int j = 0; j < 6; ++j) { Q.A[j] = i2.A[j]; Q.dl[j] = i2.dl[j]; Q.dq[j] = i2.dq[j]; Q.minv[j] = 1.0 / (Mrb[j] + i2.A[j]); }
    return Q;
  };
  auto fwd_gen = [&](const In<NT>& i2, St<double, NT>& out) {
    const Phys<double> Q = phys_of(i2);
    out = i2.x;
    double c[NT]; for (int k = 0; k < NT; ++k) c[k] = i2.c[k];
    if constexpr (RK) substep_rk4<double, NT, Act<double>, Phys<double>, true, GenH>(out, c, Q, Ac, h, G);
    else substep<double, NT, false, Act<double>, Phys<double>, true, GenH>(out, c, Q, Ac, h, nullptr, G);
  };
  const Phys<double> Pb = phys_of(in);
  St<double, NT> x = in.x; Tape<double, NT> tp;
  substep<double, NT, true, Act<double>, Phys<double>, true, GenH>(x, in.c, Pb, Ac, h, &tp, G);
  St<double, NT> lam; for (int j = 0; j < 3; ++j) lam.p[j] = U(rng); for (int j = 0; j < 4; ++j) lam.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) lam.nu[j] = U(rng); for (int j = 0; j < NT; ++j) lam.n[j] = U(rng);
  Tape<double, NT> tr;
  tape_from_states<double, NT>(in.x, x, Pb, h, 1.0 / h, tr);
  St<double, NT> xn = in.x;
  for (int j = 0; j < NT; ++j) xn.n[j] = x.n[j];
  St<double, NT> lx = lam; double lc[NT] = {}; HydroGrad<double> g{};
  if constexpr (RK)
    substep_rk4_vjp<double, NT, Act<double>, Phys<double>, true, GenH, true>(xn, in.c, Pb, Ac, h, lx, lc, g, G);
  else vjp_from_tape<double, NT>(in.x, x.q, tr, in.c, Pb, Ac, h, lx, lc, g, G);
  In<NT> d;
  for (int j = 0; j < 3; ++j) d.x.p[j] = U(rng); for (int j = 0; j < 4; ++j) d.x.q[j] = U(rng);
  for (int j = 0; j < 6; ++j) d.x.nu[j] = U(rng); for (int j = 0; j < NT; ++j) d.x.n[j] = U(rng);
  for (int j = 0; j < NT; ++j) d.c[j] = U(rng);
  for (int j = 0; j < 6; ++j) { d.A[j] = U(rng); d.dl[j] = U(rng); d.dq[j] = U(rng); }
  const double eps = 1e-6;
  auto shift = [&](double sc) { In<NT> o = in;
    for (int j = 0; j < 3; ++j) o.x.p[j] += sc * d.x.p[j]; for (int j = 0; j < 4; ++j) o.x.q[j] += sc * d.x.q[j];
    for (int j = 0; j < 6; ++j) o.x.nu[j] += sc * d.x.nu[j]; for (int j = 0; j < NT; ++j) o.x.n[j] += sc * d.x.n[j];
    for (int j = 0; j < NT; ++j) o.c[j] += sc * d.c[j];
    for (int j = 0; j < 6; ++j) { o.A[j] += sc * d.A[j]; o.dl[j] += sc * d.dl[j]; o.dq[j] += sc * d.dq[j]; }
    return o; };
  St<double, NT> yp, ym; fwd_gen(shift(eps), yp); fwd_gen(shift(-eps), ym);
  double fd = 0;
  for (int j = 0; j < 3; ++j) fd += lam.p[j] * (yp.p[j] - ym.p[j]); for (int j = 0; j < 4; ++j) fd += lam.q[j] * (yp.q[j] - ym.q[j]);
  for (int j = 0; j < 6; ++j) fd += lam.nu[j] * (yp.nu[j] - ym.nu[j]); for (int j = 0; j < NT; ++j) fd += lam.n[j] * (yp.n[j] - ym.n[j]);
  fd /= 2 * eps;
  double an = 0;
  for (int j = 0; j < 3; ++j) an += lx.p[j] * d.x.p[j]; for (int j = 0; j < 4; ++j) an += lx.q[j] * d.x.q[j];
  for (int j = 0; j < 6; ++j) an += lx.nu[j] * d.x.nu[j]; for (int j = 0; j < NT; ++j) an += g_scale * lx.n[j] * d.x.n[j];
  for (int j = 0; j < NT; ++j) an += lc[j] * d.c[j];
  for (int j = 0; j < 6; ++j) an += g.A[j] * d.A[j] + g.dl[j] * d.dl[j] + g.dq[j] * d.dq[j];
  return std::fabs(fd - an) / std::max(1.0, std::fabs(fd));
}

int main(int argc, char** argv) {
  for (int pass = 0; pass < (argc > 1 ? 2 : 1); ++pass) {
    g_scale = pass ? 1.01 : 1.0;
    std::mt19937_64 rng(11);
    double w = 0;
    double wp = 0;
    for (int k = 0; k < 300; ++k) { w = std::max(w, run<8>(rng)); w = std::max(w, run<5>(rng)); w = std::max(w, run<3>(rng)); }
    for (int k = 0; k < 300; ++k) { wp = std::max(wp, run_pay<8>(rng)); wp = std::max(wp, run_pay<4>(rng)); }
    double wg = 0;
    for (int k = 0; k < 300; ++k) wg = std::max(wg, run_gen<8>(rng));
    printf("%s %.6e\n", pass ? "scaled" : "worst", w);
    printf("%s %.6e\n", pass ? "scaled_payload" : "worst_payload", wp);
    printf("%s %.6e\n", pass ? "scaled_generic" : "worst_generic", wg);
    double wr = 0;
    for (int k = 0; k < 200; ++k) {
      wr = std::max(wr, run<8, true>(rng)); wr = std::max(wr, run<5, true>(rng));
      wr = std::max(wr, run_pay<8, true>(rng)); wr = std::max(wr, run_gen<8, true>(rng));
    }
    printf("%s %.6e\n", pass ? "scaled_rk4" : "worst_rk4", wr);
  }
  return 0;
}
