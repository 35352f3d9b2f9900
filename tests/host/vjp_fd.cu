// Host check of the step kernel's vector-Jacobian product (vjp_from_tape in
// mg_device.cuh, the arithmetic the adjoint kernel runs) in FP64: for random
// states, commands, parameters and directions d, the product's
// <vjp(lambda), d> must equal <lambda, J d> from central differences of the
// forward substep (h = 1e-6), over the state, the commands and the added-mass
// and damping coefficients (the inverse mass matrix follows the added mass).
// Prints the worst relative difference and, with a nonzero argument, the
// same for a product whose added-mass gradient is scaled by 1.01 (the check
// must see that).
#include <cstdio>
#include <random>
#include "mg_device.cuh"
using namespace mg;
template <int NT>
struct In { St<double, NT> x; double c[NT]; double A[6], dl[6], dq[6]; };
template <int NT>
void fwd(const In<NT>& in, const Phys<double>& P0, const Act<double>& Ac, double h, St<double, NT>& out) {
  Phys<double> P = P0;
  const double Mrb[6] = {P0.m, P0.m, P0.m, P0.Ig[0], P0.Ig[1], P0.Ig[2]};
  for (int j = 0; j < 6; ++j) { P.A[j] = in.A[j]; P.dl[j] = in.dl[j]; P.dq[j] = in.dq[j]; P.minv[j] = 1.0 / (Mrb[j] + in.A[j]); }
  out = in.x;
  double c[NT]; for (int i = 0; i < NT; ++i) c[i] = in.c[i];
  substep<double, NT, false>(out, c, P, Ac, h, nullptr);
}
static double g_scale = 1.0;

template <int NT>
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
  St<double, NT> lx = lam; double lc[NT] = {}; HydroGrad<double> g{};
  vjp_from_tape<double, NT>(in.x, x.q, tp, in.c, Pb, Ac, h, lx, lc, g);
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
  St<double, NT> yp, ym; fwd<NT>(shift(eps), P, Ac, h, yp); fwd<NT>(shift(-eps), P, Ac, h, ym);
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
int main(int argc, char** argv) {
  for (int pass = 0; pass < (argc > 1 ? 2 : 1); ++pass) {
    g_scale = pass ? 1.01 : 1.0;
    std::mt19937_64 rng(11);
    double w = 0;
    for (int k = 0; k < 300; ++k) { w = std::max(w, run<8>(rng)); w = std::max(w, run<5>(rng)); w = std::max(w, run<3>(rng)); }
    printf("%s %.6e\n", pass ? "scaled" : "worst", w);
  }
  return 0;
}
