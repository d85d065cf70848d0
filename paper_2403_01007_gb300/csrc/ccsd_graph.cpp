// Closed-shell CCSD energy and residual as a graph (Sec. 2.1, 2.4.2).
//
// The T1 transformation Hhat = exp(-T1) H exp(T1) is the one-index transform
// Lhat^J = (1 - t1) L^J (1 + t1), hhat = (1 - t1) h (1 + t1), where t1 sits in
// the virtual-occupied block. With it the projected equations keep only T2:
//   E0      = <HF|Hhat|HF> + sum_ijab (2 g_iajb - g_ibja) t_ij^ab
//   Omega_ai   = <ai~|Hhat + [Hhat,T2]|HF>
//   Omega_aibj = <aibj~|Hhat + [Hhat,T2] + 1/2 [[Hhat,T2],T2]|HF>
// written out below in the usual closed-shell intermediates (the paper gives
// no programmable expressions; these are checked term by term against a
// determinant-space evaluation of the defining projections).
//
// The particle-particle ladder sum_cd g_acbd t_ij^cd of the dressed integrals
// is split into the undressed vvvv ladder (a linear operator of t2 alone,
// computed on tensor cores from the Cholesky vectors) plus three terms with
// one or two powers of t1 through the ovvv and ovov integrals, because
// Lhat_vv = L_vv - t1 L_ov.
#include "ccsd_graph.h"

#include <stdexcept>

namespace sccsd {

namespace {
using V = std::vector<int64_t>;
}

EnergyResidual build_energy_residual(Graph& g, int t1, int t2, int L, int h, int delta) {
  const int64_t o = g.o, v = g.v, J = g.J;
  // blocks of the raw integrals
  int Loo = g.slice(L, {0, 0, 0}, {J, o, o});
  int Lov = g.slice(L, {0, 0, o}, {J, o, v});
  int Lvo = g.slice(L, {0, o, 0}, {J, v, o});
  int Lvv = g.slice(L, {0, o, o}, {J, v, v});
  int hoo = g.slice(h, {0, 0}, {o, o});
  int hov = g.slice(h, {0, o}, {o, v});
  int hvo = g.slice(h, {o, 0}, {v, o});
  int hvv = g.slice(h, {o, o}, {v, v});

  // T1-transformed Cholesky vectors and one-electron integrals
  int Lhoo = g.add("Jkl", {{Loo, "Jkl", 1.0}, {g.contract(Lov, "Jka", t1, "al", "Jkl", 1.0, true), "Jkl", 1.0}});
  int Lhvv = g.add("Jab", {{Lvv, "Jab", 1.0}, {g.contract(t1, "ak", Lov, "Jkb", "Jab", 1.0, true), "Jab", -1.0}});
  int Lhvo = g.add("Jai", {{Lvo, "Jai", 1.0},
                           {g.contract(Lvv, "Jac", t1, "ci", "Jai", 1.0, true), "Jai", 1.0},
                           {g.contract(t1, "ak", Lhoo, "Jki", "Jai", 1.0, true), "Jai", -1.0}});
  int hhoo = g.add("kl", {{hoo, "kl", 1.0}, {g.contract(hov, "ka", t1, "al", "kl", 1.0, true), "kl", 1.0}});
  int hhvo = g.add("ai", {{hvo, "ai", 1.0},
                          {g.contract(hvv, "ac", t1, "ci", "ai", 1.0, true), "ai", 1.0},
                          {g.contract(t1, "ak", hhoo, "ki", "ai", 1.0, true), "ai", -1.0}});
  int hhvv = g.add("ab", {{hvv, "ab", 1.0}, {g.contract(t1, "ak", hov, "kb", "ab", 1.0, true), "ab", -1.0}});

  // dressed Fock matrix F_pq = h_pq + sum_k (2 g_pqkk - g_pkkq)
  int s = g.contract(Lhoo, "Jkl", delta, "kl", "J");
  int Foo = g.add("kl", {{hhoo, "kl", 1.0},
                         {g.contract(Lhoo, "Jkl", s, "J", "kl", 1.0, true), "kl", 2.0},
                         {g.contract(Lhoo, "Jkm", Lhoo, "Jml", "kl", 1.0, true), "kl", -1.0}});
  int Fov = g.add("kc", {{hov, "kc", 1.0},
                         {g.contract(Lov, "Jkc", s, "J", "kc", 1.0, true), "kc", 2.0},
                         {g.contract(Lhoo, "Jkm", Lov, "Jmc", "kc", 1.0, true), "kc", -1.0}});
  int Fvo = g.add("ai", {{hhvo, "ai", 1.0},
                         {g.contract(Lhvo, "Jai", s, "J", "ai", 1.0, true), "ai", 2.0},
                         {g.contract(Lhvo, "Jam", Lhoo, "Jmi", "ai", 1.0, true), "ai", -1.0}});
  int Fvv = g.add("ab", {{hhvv, "ab", 1.0},
                         {g.contract(Lhvv, "Jab", s, "J", "ab", 1.0, true), "ab", 2.0},
                         {g.contract(Lhvo, "Jam", Lov, "Jmb", "ab", 1.0, true), "ab", -1.0}});

  // u_ij^ab = 2 t_ij^ab - t_ij^ba
  int u = g.add("ijab", {{t2, "ijab", 2.0}, {t2, "ijba", -1.0}});
  // g_iajb = sum_J L_ia L_jb stored as [i][j][a][b]
  int Govov = g.contract(Lov, "Jia", Lov, "Jjb", "ijab", 1.0, true);

  EnergyResidual r;
  // ---- energy
  int eh = g.contract(hhoo, "ij", delta, "ij", "");
  int ej = g.contract(s, "J", s, "J", "");
  int ek = g.contract(Lhoo, "Jij", Lhoo, "Jji", "");
  int et = g.contract(u, "ijab", Govov, "ijab", "");
  r.E0 = g.add("", {{eh, "", 2.0}, {ej, "", 2.0}, {ek, "", -1.0}, {et, "", 1.0}});

  // ---- singles
  int Z = g.contract(Lov, "Jkc", u, "kicd", "Jid", 1.0, true);
  int A1 = g.contract(Lhvv, "Jad", Z, "Jid", "ai", 1.0, true);
  int Gooov = g.contract(Lhoo, "Jki", Lov, "Jlc", "kilc", 1.0, true);
  int B1 = g.contract(u, "klac", Gooov, "kilc", "ai", 1.0, true);
  int C1 = g.contract(u, "ikac", Fov, "kc", "ai", 1.0, true);
  r.O1 = g.add("ai", {{Fvo, "ai", 1.0}, {A1, "ai", 1.0}, {B1, "ai", -1.0}, {C1, "ai", 1.0}});

  // ---- doubles
  int A2 = g.contract(Lhvo, "Jai", Lhvo, "Jbj", "ijab", 1.0, true);
  // ladder: undressed vvvv part plus the t1 corrections through ovvv / ovov
  int lad = g.ladder(t2, L);
  int Govvv = g.contract(Lov, "Jkc", Lvv, "Jbd", "kcbd", 1.0, true);
  int W0 = g.contract(t2, "ijcd", Govvv, "kcbd", "ijkb", 1.0, true);
  int l2 = g.contract(t1, "ak", W0, "ijkb", "ijab", 1.0, true);
  int l3 = g.contract(t1, "bl", W0, "jila", "ijab", 1.0, true);
  int Zl = g.contract(t2, "ijcd", Govov, "klcd", "ijkl", 1.0, true);
  int l4 = g.contract(g.contract(t1, "ak", Zl, "ijkl", "ijal", 1.0, true), "ijal", t1, "bl", "ijab", 1.0, true);
  // hole-hole ladder
  int Goooo = g.contract(Lhoo, "Jki", Lhoo, "Jlj", "kilj", 1.0, true);
  int Bint = g.add("ijkl", {{Goooo, "kilj", 1.0}, {Zl, "ijkl", 1.0}});
  int B2 = g.contract(Bint, "ijkl", t2, "klab", "ijab", 1.0, true);
  // C-type (exchange ring) terms
  int Goovv = g.contract(Lhoo, "Jki", Lhvv, "Jac", "kiac", 1.0, true);
  int c2a = g.contract(t2, "liad", Govov, "kldc", "kiac", 1.0, true);
  int X = g.add("kiac", {{Goovv, "kiac", 1.0}, {c2a, "kiac", -0.5}});
  int Q = g.contract(t2, "kjbc", X, "kiac", "jbia", 1.0, true);
  int C2 = g.add("ijab", {{Q, "jbia", -0.5}, {Q, "ibja", -1.0}});
  // D-type (direct ring) terms
  int Gvoov = g.contract(Lhvo, "Jai", Lov, "Jkc", "aikc", 1.0, true);
  int Lovov = g.add("lkdc", {{Govov, "lkdc", 2.0}, {Govov, "lkcd", -1.0}});
  int d2a = g.contract(u, "ilad", Lovov, "lkdc", "aikc", 1.0, true);
  int Y = g.add("aikc", {{Gvoov, "aikc", 2.0}, {Goovv, "kiac", -1.0}, {d2a, "aikc", 0.5}});
  int D2 = g.contract(u, "jkbc", Y, "aikc", "ijab", 0.5, true);
  // E-type (Fock-like) terms
  int Fvvi = g.add("bc", {{Fvv, "bc", 1.0},
                          {g.contract(u, "klbd", Govov, "lkdc", "bc", 1.0, true), "bc", -1.0}});
  int Fooi = g.add("kj", {{Foo, "kj", 1.0},
                          {g.contract(u, "ljcd", Govov, "kldc", "kj", 1.0, true), "kj", 1.0}});
  int E2 = g.add("ijab", {{g.contract(t2, "ijac", Fvvi, "bc", "ijab", 1.0, true), "ijab", 1.0},
                          {g.contract(t2, "ikab", Fooi, "kj", "ijab", 1.0, true), "ijab", -1.0}});
  r.Fvvi = Fvvi;
  r.Fooi = Fooi;
  r.Govov = Govov;
  int Pp = g.add("ijab", {{C2, "ijab", 1.0}, {D2, "ijab", 1.0}, {E2, "ijab", 1.0}});
  r.O2 = g.add("ijab", {{A2, "ijab", 1.0},
                        {lad, "ijab", 1.0},
                        {l2, "ijab", -1.0},
                        {l3, "ijab", -1.0},
                        {l4, "ijab", 1.0},
                        {B2, "ijab", 1.0},
                        {Pp, "ijab", 1.0},
                        {Pp, "jiba", 1.0}});
  return r;
}

static int get_or_zero(Graph& g, const std::map<int, int>& m, int id) {
  auto it = m.find(id);
  if (it != m.end()) return it->second;
  return g.zero(g.t[id].dims);
}

Xi build_xi(Graph& g, int t1, int t2zero, const EnergyResidual& er0,
            const Graph::Ranges& primal0, int x1, int y2) {
  // first derivative along T2 = u R2 at u = 0
  size_t b1 = g.ops.size();
  auto tu = g.tangent({{t2zero, y2}}, primal0);
  size_t b2 = g.ops.size();
  int e2 = get_or_zero(g, tu, er0.E0);   // <HF|Hhat R2|HF>
  int s1 = get_or_zero(g, tu, er0.O1);   // <kappa~|Hhat R2|HF>
  int dO2 = get_or_zero(g, tu, er0.O2);
  // mixed derivative along T1 = t1 + s R1
  Graph::Ranges r = primal0;
  r.push_back({b1, b2});
  auto ts = g.tangent({{t1, x1}}, r);
  int e1 = get_or_zero(g, ts, er0.E0);   // <HF|Hhat R1|HF>
  int d2O1 = get_or_zero(g, ts, s1);
  int d2O2 = get_or_zero(g, ts, dO2);
  Xi xi;
  xi.X1 = g.add("ai", {{d2O1, "ai", 1.0}, {g.contract(x1, "ai", e2, "", "ai"), "ai", 1.0}});
  int P = g.contract(x1, "ai", s1, "bj", "ijab");
  xi.X2 = g.add("ijab", {{d2O2, "ijab", 1.0},
                         {P, "ijab", 1.0},
                         {P, "jiba", 1.0},
                         {g.contract(y2, "ijab", e1, "", "ijab"), "ijab", 1.0}});
  return xi;
}

}  // namespace sccsd
