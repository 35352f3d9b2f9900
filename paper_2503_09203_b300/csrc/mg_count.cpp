// FLOP count of the step arithmetic: the kernels' own templated substep and
// observation run on the host with a counting scalar. Convention: add, sub,
// mul = 1; a fused multiply-add is a mul and an add (2); divide, square root
// and reciprocal square root = 1 each; compare, abs and negate = 0.
#include <cstdint>

#include "../../include/marinegym.h"
#include "mg_internal.h"
#include "mg_device.cuh"

namespace mgcount {

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(float a) : v(a) {}
  Cnt(double a) : v(a) {}
};

static thread_local int64_t g_ops = 0;

inline Cnt operator+(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline Cnt mabs(Cnt a) { return Cnt(a.v < 0 ? -a.v : a.v); }
inline Cnt msqrt(Cnt a) { ++g_ops; return Cnt(__builtin_sqrt(a.v)); }
inline Cnt minvsqrt(Cnt a) { ++g_ops; return Cnt(1.0 / __builtin_sqrt(a.v)); }

}  // namespace mgcount

namespace mg {
using mgcount::Cnt;
using mgcount::mabs;
using mgcount::msqrt;
using mgcount::minvsqrt;
}  // namespace mg

template <int NT>
static void count(bool with_current, double* sub, double* obs, double* adj) {
  using mg::Cnt;
  mg::St<Cnt, NT> x;
  for (int i = 0; i < 3; ++i) x.p[i] = Cnt(0.1 * (i + 1));
  x.q[0] = Cnt(1.0);
  for (int i = 1; i < 4; ++i) x.q[i] = Cnt(0.0);
  for (int i = 0; i < 6; ++i) x.nu[i] = Cnt(0.1);
  for (int i = 0; i < NT; ++i) x.n[i] = Cnt(0.2);
  Cnt c[NT];
  for (int i = 0; i < NT; ++i) c[i] = Cnt(0.3);
  mg::Phys<Cnt> P;
  for (int j = 0; j < 6; ++j) { P.minv[j] = Cnt(0.1); P.A[j] = Cnt(1.0); P.dl[j] = Cnt(1.0); P.dq[j] = Cnt(1.0); }
  P.m = Cnt(10.0); P.W = Cnt(100.0); P.B = Cnt(100.0);
  for (int j = 0; j < 3; ++j) { P.Ig[j] = Cnt(0.2); P.rb[j] = Cnt(0.0); P.Vc[j] = Cnt(0.1); }
  mg::Act<Cnt> A;
  for (int k = 0; k < 6; ++k) for (int i = 0; i < 8; ++i) A.alloc[k][i] = Cnt(0.5);
  for (int i = 0; i < 8; ++i) { A.kf[i] = Cnt(40.0); A.dz[i] = Cnt(0.0); A.alpha[i] = Cnt(0.2); }
  mgcount::g_ops = 0;
  if (with_current)
    mg::substep<Cnt, NT, false, mg::Act<Cnt>, mg::Phys<Cnt>, true>(x, c, P, A, Cnt(0.01), nullptr);
  else
    mg::substep<Cnt, NT, false, mg::Act<Cnt>, mg::Phys<Cnt>, false>(x, c, P, A, Cnt(0.01), nullptr);
  *sub = (double)mgcount::g_ops;
  mgcount::g_ops = 0;
  Cnt tgt[3] = {Cnt(0.0), Cnt(0.0), Cnt(0.0)};
  Cnt o[13], r;
  mg::observe<Cnt, NT>(x, c, tgt, o, r);
  *obs = (double)mgcount::g_ops;
  // Adjoint of one substep as the reverse pass runs it: the forward
  // recompute (which records the states), the tape rebuilt from the records of
  // the substep's start and end, and the vector-Jacobian product.
  mg::St<Cnt, NT> lam = x;
  Cnt lc[NT];
  mg::HydroGrad<Cnt> g;
  mgcount::g_ops = 0;
  mg::St<Cnt, NT> xf = x;
  mg::substep<Cnt, NT, false>(xf, c, P, A, Cnt(0.01), nullptr);
  mg::Tape<Cnt, NT> tp;
  mg::tape_from_states<Cnt, NT>(x, xf, P, Cnt(0.01), Cnt(100.0), tp);
  mg::vjp_from_tape<Cnt, NT>(x, xf.q, tp, c, P, A, Cnt(0.01), lam, lc, g);
  *adj = (double)mgcount::g_ops;
}

extern "C" int mg_count_flops(int32_t n_thr, int32_t with_current, double* substep_flops, double* observe_flops,
                              double* adjoint_flops) {
  double s = 0, o = 0, a = 0;
  switch (n_thr) {
    case 1: count<1>(with_current != 0, &s, &o, &a); break;
    case 2: count<2>(with_current != 0, &s, &o, &a); break;
    case 3: count<3>(with_current != 0, &s, &o, &a); break;
    case 4: count<4>(with_current != 0, &s, &o, &a); break;
    case 5: count<5>(with_current != 0, &s, &o, &a); break;
    case 6: count<6>(with_current != 0, &s, &o, &a); break;
    case 7: count<7>(with_current != 0, &s, &o, &a); break;
    case 8: count<8>(with_current != 0, &s, &o, &a); break;
    default: return MG_ERR_INVALID_ARG;
  }
  if (substep_flops) *substep_flops = s;
  if (observe_flops) *observe_flops = o;
  if (adjoint_flops) *adjoint_flops = a;
  return MG_OK;
}
