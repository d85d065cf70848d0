// Graph model of one context: the residual graph and the lazily built
// sections (transformations, densities, overlap, multiplier gradients).
#include "context.h"

using namespace sccsd;

namespace sccsd {

static int node_or_zero(Graph& g, const std::map<int, int>& m, int id) {
  auto it = m.find(id);
  return it != m.end() ? it->second : g.zero(g.t[id].dims);
}

std::unique_ptr<Model> build_model(Backend* be, int o, int v, int J, bool scc, int nslots) {
  auto M = std::make_unique<Model>();
  Graph& g = M->g;
  g.be = be;
  g.o = o;
  g.v = v;
  g.J = J;
  const int64_t n = o + v;
  M->scc = scc;
  M->t1 = g.input({v, o}, "t1");
  M->t2 = g.input({o, o, v, v}, "t2");
  M->L = g.input({J, n, n}, "L");
  M->h = g.input({n, n}, "h");
  M->delta = g.input({o, o}, "delta");
  M->R1 = g.input({v, o}, "R1");
  M->R2 = g.input({o, o, v, v}, "R2");
  M->Lb1 = g.input({v, o}, "Lbar1");
  M->Lb2 = g.input({o, o, v, v}, "Lbar2");
  M->s_l0r0 = g.input({}, "l0r0");
  M->s_l0 = g.input({}, "l0");
  M->s_r0 = g.input({}, "r0");

  M->er = build_energy_residual(g, M->t1, M->t2, M->L, M->h, M->delta);
  if (scc) {
    M->zeta = g.input({}, "zeta");
    M->Ra1 = g.input({v, o}, "Ra1");
    M->Ra2 = g.input({o, o, v, v}, "Ra2");
    M->Rb1 = g.input({v, o}, "Rb1");
    M->Rb2 = g.input({o, o, v, v}, "Rb2");
    M->t2zero = g.input({o, o, v, v}, "t2zero");
    size_t p0 = g.ops.size();
    EnergyResidual er0 = build_energy_residual(g, M->t1, M->t2zero, M->L, M->h, M->delta);
    Graph::Ranges r0 = {{p0, g.ops.size()}};
    Xi ab = build_xi(g, M->t1, M->t2zero, er0, r0, M->Ra1, M->Rb2);
    Xi ba = build_xi(g, M->t1, M->t2zero, er0, r0, M->Rb1, M->Ra2);
    int d1 = g.add("ai", {{ab.X1, "ai", 1.0}, {ba.X1, "ai", -1.0}});
    int d2 = g.add("ijab", {{ab.X2, "ijab", 1.0}, {ba.X2, "ijab", -1.0}});
    M->er.O1 = g.add("ai", {{M->er.O1, "ai", 1.0}, {g.contract(M->zeta, "", d1, "ai", "ai"), "ai", 1.0}});
    M->er.O2 = g.add("ijab", {{M->er.O2, "ijab", 1.0},
                              {g.contract(M->zeta, "", d2, "ijab", "ijab"), "ijab", 1.0}});
  } else if (nslots > 0) {
    // several constrained states: sum_{k<l} zeta_kl X_kl = sum_k R1^k Y2^k with
    // Y2^k = sum_l Z_kl R2^l (Z antisymmetric), so the X3 terms are a sum of
    // one bilinear term per state; the inputs are (R1^k, Y2^k)
    M->nslots = nslots;
    M->t2zero = g.input({o, o, v, v}, "t2zero");
    size_t p0 = g.ops.size();
    EnergyResidual er0 = build_energy_residual(g, M->t1, M->t2zero, M->L, M->h, M->delta);
    Graph::Ranges r0 = {{p0, g.ops.size()}};
    std::vector<Graph::Term> s1 = {{M->er.O1, "ai", 1.0}}, s2 = {{M->er.O2, "ijab", 1.0}};
    for (int k = 0; k < nslots; ++k) {
      const int x1 = g.input({v, o}, "X1_" + std::to_string(k));
      const int y2 = g.input({o, o, v, v}, "Y2_" + std::to_string(k));
      M->X1s.push_back(x1);
      M->Y2s.push_back(y2);
      Xi xk = build_xi(g, M->t1, M->t2zero, er0, r0, x1, y2);
      s1.push_back({xk.X1, "ai", 1.0});
      s2.push_back({xk.X2, "ijab", 1.0});
    }
    M->er.O1 = g.add("ai", s1);
    M->er.O2 = g.add("ijab", s2);
  }
  Graph::Ranges fwd = {{0, g.ops.size()}};
  M->fwd = fwd;

  // right transformation: forward-mode derivative along R
  size_t rb = g.ops.size();
  auto tan = g.tangent({{M->t1, M->R1}, {M->t2, M->R2}}, fwd);
  size_t re = g.ops.size();
  M->sig1 = node_or_zero(g, tan, M->er.O1);
  M->sig2 = node_or_zero(g, tan, M->er.O2);
  M->etaR = node_or_zero(g, tan, M->er.E0);

  // left transformation: gradient of Lbar . Omega
  auto adj = g.adjoint({{M->er.O1, M->Lb1}, {M->er.O2, M->Lb2}}, {M->t1, M->t2}, fwd);
  M->lt1 = adj[M->t1];
  M->lt2 = adj[M->t2];

  // densities: gradient w.r.t. (h, L) of
  //   <L|Hbar|R> = l0 r0 E0 + l0 eta.R + r0 L.Omega + L.(A R) + E0 L.R + L.(R1 x Omega1)
  int dot = g.add("", {{g.contract(M->Lb1, "ai", M->R1, "ai", ""), "", 1.0},
                       {g.contract(M->Lb2, "ijab", M->R2, "ijab", ""), "", 1.0}});
  int sE = g.add("", {{M->s_l0r0, "", 1.0}, {dot, "", 1.0}});
  int oB1 = g.add("ai", {{g.contract(M->s_r0, "", M->Lb1, "ai", "ai"), "ai", 1.0},
                         {g.contract(M->Lb2, "ijab", M->R1, "ai", "bj"), "ai", 2.0}});
  int oB2 = g.contract(M->s_r0, "", M->Lb2, "ijab", "ijab");
  Graph::Ranges dr = {{0, rb}, {rb, re}};
  auto dadj = g.adjoint({{M->er.E0, sE},
                         {M->er.O1, oB1},
                         {M->er.O2, oB2},
                         {M->etaR, M->s_l0},
                         {M->sig1, M->Lb1},
                         {M->sig2, M->Lb2}},
                        {M->h, M->L}, dr);
  M->D1 = dadj[M->h];
  M->Gam = dadj[M->L];
  M->sE = sE;
  M->oB1 = oB1;
  M->oB2 = oB2;
  M->dr = dr;
  M->vol_inputs = {M->R1, M->R2, M->Lb1, M->Lb2, M->s_l0r0, M->s_l0, M->s_r0};
  g.set_volatile_inputs(M->vol_inputs);
  return M;
}

// O_ab = <psi_a|P|psi_b>, P onto HF + singles + doubles, psi = exp(T)(R0 + R)|HF>
// with T without X3 (Sec. 2.4.2): the Hilbert-space inner product of
//   c0 = R0, c1 = r1 + R0 t1, c2 = r2 + (t1 x r1 + transpose) + R0 (t2 + t1 x t1)
// with <S|S'> = 2 sum c1 c1' and <D|D'> = sum c2 (2 c2' - c2' with i <-> j).
OverlapSec& overlap_section(Model& M) {
  if (M.ovl) return *M.ovl;
  Graph& g = M.g;
  const int64_t o = g.o, v = g.v;
  auto S = std::make_unique<OverlapSec>();
  S->op_begin = g.ops.size();
  S->ra0 = g.input({}, "Oa0");
  S->ra1 = g.input({v, o}, "Oa1");
  S->ra2 = g.input({o, o, v, v}, "Oa2");
  S->rb0 = g.input({}, "Ob0");
  S->rb1 = g.input({v, o}, "Ob1");
  S->rb2 = g.input({o, o, v, v}, "Ob2");
  int tt = g.contract(M.t1, "ai", M.t1, "bj", "ijab");
  auto state = [&](int r0, int r1, int r2, int& c1, int& c2) {
    c1 = g.add("ai", {{r1, "ai", 1.0}, {g.contract(r0, "", M.t1, "ai", "ai"), "ai", 1.0}});
    int tr = g.contract(M.t1, "ai", r1, "bj", "ijab");
    int tp = g.add("ijab", {{M.t2, "ijab", 1.0}, {tt, "ijab", 1.0}});
    c2 = g.add("ijab", {{r2, "ijab", 1.0},
                        {tr, "ijab", 1.0},
                        {tr, "jiba", 1.0},
                        {g.contract(r0, "", tp, "ijab", "ijab"), "ijab", 1.0}});
  };
  int ca1, ca2, cb1, cb2;
  state(S->ra0, S->ra1, S->ra2, ca1, ca2);
  state(S->rb0, S->rb1, S->rb2, cb1, cb2);
  S->ca1 = ca1;
  S->ca2 = ca2;
  S->cb1 = cb1;
  S->cb2 = cb2;
  int q = g.add("ijab", {{cb2, "ijab", 2.0}, {cb2, "jiab", -1.0}});
  S->O = g.add("", {{g.contract(S->ra0, "", S->rb0, "", ""), "", 1.0},
                    {g.contract(ca1, "ai", cb1, "ai", ""), "", 2.0},
                    {g.contract(ca2, "ijab", q, "ijab", ""), "", 1.0}});
  S->op_end = g.ops.size();
  for (int x : {S->ra0, S->ra1, S->ra2, S->rb0, S->rb1, S->rb2}) M.vol_inputs.push_back(x);
  g.set_volatile_inputs(M.vol_inputs);
  M.ovl = std::move(S);
  return *M.ovl;
}

OverlapKSec& overlap_k_section(Model& M) {
  if (M.ovk) return *M.ovk;
  OverlapSec& O = overlap_section(M);
  Graph& g = M.g;
  auto S = std::make_unique<OverlapKSec>();
  S->op_begin = g.ops.size();
  // <x|y> over HF+S+D kets: x0 y0 + 2 x1.y1 + x2.(2 y2 - y2 with j <-> i)
  auto metric = [&](int x0, int x1, int x2, int y0, int y1, int y2) {
    int q = g.add("ijab", {{y2, "ijab", 2.0}, {y2, "jiab", -1.0}});
    return g.add("", {{g.contract(x0, "", y0, "", ""), "", 1.0},
                      {g.contract(x1, "ai", y1, "ai", ""), "", 2.0},
                      {g.contract(x2, "ijab", q, "ijab", ""), "", 1.0}});
  };
  // the c0 part of exp(T)|R> is R0 itself
  S->maa = metric(O.ra0, O.ca1, O.ca2, O.ra0, O.ra1, O.ra2);
  S->mab = metric(O.ra0, O.ca1, O.ca2, O.rb0, O.rb1, O.rb2);
  S->nab = metric(O.ra0, O.ra1, O.ra2, O.rb0, O.cb1, O.cb2);
  S->nbb = metric(O.rb0, O.rb1, O.rb2, O.rb0, O.cb1, O.cb2);
  S->Saa = metric(O.ra0, O.ra1, O.ra2, O.ra0, O.ra1, O.ra2);
  S->Sab = metric(O.ra0, O.ra1, O.ra2, O.rb0, O.rb1, O.rb2);
  S->Sbb = metric(O.rb0, O.rb1, O.rb2, O.rb0, O.rb1, O.rb2);
  S->op_end = g.ops.size();
  M.ovk = std::move(S);
  return *M.ovk;
}

OvlKGradSec& overlap_k_grad_section(Model& M) {
  if (M.ovkg) return *M.ovkg;
  OverlapSec& O = overlap_section(M);
  OverlapKSec& K = overlap_k_section(M);
  Graph& g = M.g;
  auto S = std::make_unique<OvlKGradSec>();
  const int sc[7] = {K.maa, K.mab, K.nab, K.nbb, K.Saa, K.Sab, K.Sbb};
  std::map<int, int> seeds;
  for (int i = 0; i < 7; ++i) {
    S->w[i] = g.input({}, "wK" + std::to_string(i));
    seeds[sc[i]] = S->w[i];
  }
  auto adj = g.adjoint(seeds, {M.t1, M.t2, O.ra0, O.ra1, O.ra2, O.rb0, O.rb1, O.rb2},
                       {{O.op_begin, O.op_end}, {K.op_begin, K.op_end}});
  S->dt1 = adj[M.t1];
  S->dt2 = adj[M.t2];
  S->da0 = adj[O.ra0];
  S->da1 = adj[O.ra1];
  S->da2 = adj[O.ra2];
  S->db0 = adj[O.rb0];
  S->db1 = adj[O.rb1];
  S->db2 = adj[O.rb2];
  for (int i = 0; i < 7; ++i) M.vol_inputs.push_back(S->w[i]);
  g.set_volatile_inputs(M.vol_inputs);
  M.ovkg = std::move(S);
  return *M.ovkg;
}

// sigma = A R for nb trial vectors at once (forward mode with a batch label)
RightSec& right_section(Model& M, int64_t nb) {
  auto it = M.right.find(nb);
  if (it != M.right.end()) return it->second;
  Graph& g = M.g;
  const int64_t o = g.o, v = g.v;
  RightSec S;
  S.R1 = g.input({nb, v, o}, "R1b");
  S.R2 = g.input({nb, o, o, v, v}, "R2b");
  auto tan = g.tangent({{M.t1, S.R1}, {M.t2, S.R2}}, M.fwd, nb);
  auto pick = [&](int id, std::vector<int64_t> d) {
    auto f = tan.find(id);
    if (f != tan.end()) return f->second;
    d.insert(d.begin(), nb);
    return g.zero(d);
  };
  S.sig1 = pick(M.er.O1, g.t[M.er.O1].dims);
  S.sig2 = pick(M.er.O2, g.t[M.er.O2].dims);
  S.etaR = pick(M.er.E0, g.t[M.er.E0].dims);
  M.vol_inputs.push_back(S.R1);
  M.vol_inputs.push_back(S.R2);
  g.set_volatile_inputs(M.vol_inputs);
  return M.right[nb] = S;
}

// sigma = A^T L for nb bras at once (reverse mode with a batch label)
LeftSec& left_section(Model& M, int64_t nb) {
  auto it = M.left.find(nb);
  if (it != M.left.end()) return it->second;
  Graph& g = M.g;
  const int64_t o = g.o, v = g.v;
  LeftSec S;
  S.Lb1 = g.input({nb, v, o}, "Lbar1b");
  S.Lb2 = g.input({nb, o, o, v, v}, "Lbar2b");
  auto adj = g.adjoint({{M.er.O1, S.Lb1}, {M.er.O2, S.Lb2}}, {M.t1, M.t2}, M.fwd, nb);
  S.lt1 = adj[M.t1];
  S.lt2 = adj[M.t2];
  M.vol_inputs.push_back(S.Lb1);
  M.vol_inputs.push_back(S.Lb2);
  g.set_volatile_inputs(M.vol_inputs);
  return M.left[nb] = S;
}

// d<K|Hbar|R>/d(t, zeta, Ra, Rb, R) for the bra and ket of the density
// inputs: the seeds of the density section, differentiated with respect to
// the state instead of the integrals (reverse over forward mode)
LagSec& lag_section(Model& M) {
  if (M.lag) return *M.lag;
  if (!M.scc) throw std::logic_error("multipliers need the SCC model");
  Graph& g = M.g;
  auto adj = g.adjoint({{M.er.E0, M.sE},
                        {M.er.O1, M.oB1},
                        {M.er.O2, M.oB2},
                        {M.etaR, M.s_l0},
                        {M.sig1, M.Lb1},
                        {M.sig2, M.Lb2}},
                       {M.t1, M.t2, M.zeta, M.Ra1, M.Ra2, M.Rb1, M.Rb2, M.R1, M.R2}, M.dr);
  auto S = std::make_unique<LagSec>();
  S->gt1 = adj[M.t1];
  S->gt2 = adj[M.t2];
  S->gz = adj[M.zeta];
  S->gRa1 = adj[M.Ra1];
  S->gRa2 = adj[M.Ra2];
  S->gRb1 = adj[M.Rb1];
  S->gRb2 = adj[M.Rb2];
  S->gR1 = adj[M.R1];
  S->gR2 = adj[M.R2];
  g.set_volatile_inputs(M.vol_inputs);
  M.lag = std::move(S);
  return *M.lag;
}

OvlGradSec& overlap_grad_section(Model& M) {
  if (M.ovg) return *M.ovg;
  OverlapSec& O = overlap_section(M);
  Graph& g = M.g;
  auto S = std::make_unique<OvlGradSec>();
  S->gbar = g.input({}, "gbar");
  auto adj = g.adjoint({{O.O, S->gbar}}, {M.t1, M.t2, O.ra0, O.ra1, O.ra2, O.rb0, O.rb1, O.rb2},
                       {{O.op_begin, O.op_end}});
  S->dt1 = adj[M.t1];
  S->dt2 = adj[M.t2];
  S->da0 = adj[O.ra0];
  S->da1 = adj[O.ra1];
  S->da2 = adj[O.ra2];
  S->db0 = adj[O.rb0];
  S->db1 = adj[O.rb1];
  S->db2 = adj[O.rb2];
  M.vol_inputs.push_back(S->gbar);
  g.set_volatile_inputs(M.vol_inputs);
  M.ovg = std::move(S);
  return *M.ovg;
}

}  // namespace sccsd
