// C ABI of the SCCSD hot path: contexts, graph assembly and marshalling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/sccsd.h"
#include "backend.h"
#include "ccsd_graph.h"
#include "small_la.h"

namespace sccsd {

// Defined by the device backend translation unit.
std::unique_ptr<Backend> make_backend(void* stream, int precision);

// One graph holding the residual, both Jacobian transformations and the
// densities, with or without the SCC X3 terms.
struct RightSec {
  int R1, R2, sig1, sig2, etaR;
};
struct LeftSec {
  int Lb1, Lb2, lt1, lt2;
};

// O_ab of the natural projection for two states given as (R0, R1, R2)
struct OverlapSec {
  int ra0, ra1, ra2, rb0, rb1, rb2;
  int O;
  size_t op_begin = 0, op_end = 0;  // the section's ops
};

// Gradient of <K|Hbar|R> (bra (k0, K), ket (r0, R) in the density inputs) with
// respect to the state: t, zeta, the X3 vectors Ra, Rb and the ket R itself.
struct LagSec {
  int gt1, gt2, gz, gRa1, gRa2, gRb1, gRb2, gR1, gR2;
};

// Gradient of gbar * O_ab with respect to t and both states.
struct OvlGradSec {
  int gbar, dt1, dt2, da0, da1, da2, db0, db1, db2;
};

struct Model {
  Graph g;
  bool scc = false;
  std::unique_ptr<OverlapSec> ovl;
  Graph::Ranges fwd;
  std::vector<int> vol_inputs;
  std::map<int64_t, RightSec> right;  // batched right transformations by batch size
  std::map<int64_t, LeftSec> left;
  int t1, t2, L, h, delta;
  int R1, R2, Lb1, Lb2;
  int zeta = -1, Ra1 = -1, Ra2 = -1, Rb1 = -1, Rb2 = -1, t2zero = -1;
  int s_l0r0, s_l0, s_r0;
  EnergyResidual er;
  int sig1, sig2, etaR;
  int lt1, lt2;
  int D1, Gam;
  // seeds of the transition element and the op ranges they differentiate
  int sE = -1, oB1 = -1, oB2 = -1;
  Graph::Ranges dr;
  std::unique_ptr<LagSec> lag;
  std::unique_ptr<OvlGradSec> ovg;
};

static int node_or_zero(Graph& g, const std::map<int, int>& m, int id) {
  auto it = m.find(id);
  return it != m.end() ? it->second : g.zero(g.t[id].dims);
}

static std::unique_ptr<Model> build_model(Backend* be, int o, int v, int J, bool scc) {
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
static OverlapSec& overlap_section(Model& M) {
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

// sigma = A R for nb trial vectors at once (forward mode with a batch label)
static RightSec& right_section(Model& M, int64_t nb) {
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
static LeftSec& left_section(Model& M, int64_t nb) {
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
static LagSec& lag_section(Model& M) {
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

static OvlGradSec& overlap_grad_section(Model& M) {
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

using namespace sccsd;

struct sccsd_ctx {
  int o = 0, v = 0, J = 0, n = 0, precision = 0;
  int64_t dim = 0;
  std::unique_ptr<Backend> be;
  std::unique_ptr<Model> plain, scc;
  Model* cur = nullptr;
  double* L = nullptr;      // device copy of the Cholesky vectors
  double* h = nullptr;      // device one-electron integrals
  double* delta = nullptr;  // identity [o][o]
  double* stage = nullptr;  // one packed vector
  double* stage2 = nullptr;
  double e_hf = 0.0;
  int max_batch = 8;  // trial vectors per batched pass
  std::vector<double> eps_host;
  double* eps_dev = nullptr;  // orbital energies on the device
  double* D = nullptr;        // packed orbital-energy denominators
  double* Dprec = nullptr;    // user/learned preconditioner of the ground-state update
  bool use_dprec = false;
  std::vector<double*> sv;    // solver work buffers
  std::vector<int64_t> sv_n;  // their sizes (doubles)
  double* sv_small = nullptr; // small matrices and vectors
  int* sv_info = nullptr;
  std::string err;
  ~sccsd_ctx() {
    if (getenv("SCCSD_TRACE")) {
      for (Model* m : {plain.get(), scc.get()})
        if (m) fprintf(stderr, "%s", m->g.trace_report(std::max(60, atoi(getenv("SCCSD_TRACE")))).c_str());
    }
    plain.reset();
    scc.reset();
    if (be) {
      for (double* p : {L, h, delta, stage, stage2, eps_dev, D, Dprec, sv_small})
        if (p) be->release(p);
      for (double* p : sv)
        if (p) be->release(p);
      if (sv_info) be->release((double*)sv_info);
    }
  }
};

namespace {

int fail(sccsd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

template <class F>
int guarded(sccsd_ctx* c, F&& f) {
  try {
    f();
    return SCCSD_OK;
  } catch (const OomError& e) {
    return fail(c, SCCSD_ENOMEM, e.what());
  } catch (const CudaError& e) {
    return fail(c, SCCSD_ECUDA, e.what());
  } catch (const std::invalid_argument& e) {
    return fail(c, SCCSD_EINVAL, e.what());
  } catch (const std::domain_error& e) {
    return fail(c, SCCSD_ECOMPLEX, e.what());
  } catch (const std::logic_error& e) {
    return fail(c, SCCSD_ESTATE, e.what());
  } catch (const std::bad_alloc&) {
    return fail(c, SCCSD_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(c, SCCSD_EINTERNAL, e.what());
  }
}

Model& model(sccsd_ctx* c, bool scc) {
  std::unique_ptr<Model>& m = scc ? c->scc : c->plain;
  if (!m) {
    m = build_model(c->be.get(), c->o, c->v, c->J, scc);
    m->g.trace = getenv("SCCSD_TRACE") != nullptr;
    m->g.set_input(m->L, c->L, true);
    m->g.set_input(m->h, c->h, true);
    m->g.set_input(m->delta, c->delta, true);
    if (scc) {
      double* z = m->g.t[m->t2zero].data;
      if (!z) {
        m->g.t[m->t2zero].data = c->be->alloc(m->g.t[m->t2zero].numel());
        z = m->g.t[m->t2zero].data;
      }
      c->be->fill(z, m->g.t[m->t2zero].numel(), 0.0);
      m->g.touch(m->t2zero);
    }
  }
  return *m;
}

double* input_buffer(Graph& g, int id) {
  Tensor& x = g.t[id];
  if (!x.data) x.data = g.be->alloc(std::max<int64_t>(1, x.numel()));
  return x.data;
}

// packed vector (host or device) -> graph inputs (x1, x2)
void load_packed(sccsd_ctx* c, Graph& g, const double* src, int x1, int x2, bool bra) {
  const double* d = src;
  if (!c->be->is_device(src)) {
    c->be->upload(c->stage, src, c->dim, false);
    d = c->stage;
  }
  c->be->unpack(d, c->o, c->v, input_buffer(g, x1), input_buffer(g, x2), bra);
  g.touch(x1);
  g.touch(x2);
}

// nb packed vectors (host or device) -> batched graph inputs [nb][...]
void load_packed_batch(sccsd_ctx* c, Graph& g, const double* src, int64_t nb, int x1, int x2,
                       bool bra) {
  const int64_t ov = (int64_t)c->o * c->v, oovv = ov * ov;
  double* b1 = input_buffer(g, x1);
  double* b2 = input_buffer(g, x2);
  const bool dev = c->be->is_device(src);
  for (int64_t k = 0; k < nb; ++k) {
    const double* d = src + k * c->dim;
    if (!dev) {
      c->be->upload(c->stage, d, c->dim, false);
      d = c->stage;
    }
    c->be->unpack(d, c->o, c->v, b1 + k * ov, b2 + k * oovv, bra);
  }
  g.touch(x1);
  g.touch(x2);
}

void store_packed_batch(sccsd_ctx* c, Graph& g, int64_t nb, int y1, int y2, double* dst, bool bra) {
  const int64_t ov = (int64_t)c->o * c->v, oovv = ov * ov;
  if (g.is_zero(y1) || g.is_zero(y2)) throw std::runtime_error("zero output node");
  const bool dev = c->be->is_device(dst);
  for (int64_t k = 0; k < nb; ++k) {
    double* d = dev ? dst + k * c->dim : c->stage2;
    c->be->pack(g.data(y1) + k * ov, g.data(y2) + k * oovv, c->o, c->v, d, bra);
    if (!dev) c->be->download(dst + k * c->dim, d, c->dim, false);
  }
}

void store_packed(sccsd_ctx* c, Graph& g, int y1, int y2, double* dst, bool bra) {
  bool dev = c->be->is_device(dst);
  double* d = dev ? dst : c->stage2;
  if (g.is_zero(y1) || g.is_zero(y2)) throw std::runtime_error("zero output node");
  c->be->pack(g.data(y1), g.data(y2), c->o, c->v, d, bra);
  if (!dev) c->be->download(dst, d, c->dim, false);
}

void set_scalar(sccsd_ctx* c, Graph& g, int id, double v) { g.set_input(id, &v, false); }

double get_scalar(sccsd_ctx* c, Graph& g, int id) {
  double v = 0.0;
  if (g.is_zero(id)) return 0.0;
  c->be->download(&v, g.data(id), 1, false);
  return v;
}

}  // namespace

extern "C" {

long long sccsd_dim(int o, int v) {
  long long ov = (long long)o * v;
  return ov + ov * (ov + 1) / 2;
}

const char* sccsd_strerror(int code) {
  switch (code) {
    case SCCSD_OK: return "ok";
    case SCCSD_EINVAL: return "invalid argument";
    case SCCSD_ENOMEM: return "out of memory";
    case SCCSD_ECUDA: return "CUDA error";
    case SCCSD_ESTATE: return "invalid call order";
    case SCCSD_EINTERNAL: return "internal error";
    case SCCSD_ENOTCONV: return "not converged";
    case SCCSD_ECOMPLEX: return "complex roots";
    default: return "unknown error";
  }
}

const char* sccsd_last_error(sccsd_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int sccsd_init(sccsd_ctx** out, int o, int v, int J, const double* eps, const double* L,
               int precision, void* stream) {
  if (!out) return SCCSD_EINVAL;
  *out = nullptr;
  if (o < 1 || v < 1 || J < 1 || !eps || !L) return SCCSD_EINVAL;
  if (precision < SCCSD_FP64 || precision > SCCSD_BF16) return SCCSD_EINVAL;
  sccsd_ctx* c = new (std::nothrow) sccsd_ctx;
  if (!c) return SCCSD_ENOMEM;
  int rc = guarded(c, [&] {
    c->o = o;
    c->v = v;
    c->J = J;
    c->n = o + v;
    c->precision = precision;
    c->dim = sccsd_dim(o, v);
    c->be = make_backend(stream, precision);
    const int64_t n = c->n;
    c->L = c->be->alloc((int64_t)J * n * n);
    c->be->upload(c->L, L, (int64_t)J * n * n, c->be->is_device(L));
    std::vector<double> e(n);
    if (c->be->is_device(eps)) {
      c->be->download(e.data(), eps, n, false);
    } else {
      std::memcpy(e.data(), eps, sizeof(double) * n);
    }
    for (int k = 0; k < n; ++k)
      if (!std::isfinite(e[k])) throw std::invalid_argument("eps is not finite");
    for (int k = 1; k < o; ++k)
      if (e[k] < e[k - 1]) throw std::invalid_argument("occupied eps not ascending");
    for (int k = o + 1; k < n; ++k)
      if (e[k] < e[k - 1]) throw std::invalid_argument("virtual eps not ascending");
    if (e[o] <= e[o - 1]) throw std::invalid_argument("no gap between occupied and virtual eps");
    c->eps_host = e;
    c->eps_dev = c->be->alloc(n);
    c->be->upload(c->eps_dev, e.data(), n, false);
    c->D = c->be->alloc(c->dim);
    launch_denoms((cudaStream_t)c->be->stream(), o, v, c->eps_dev, c->D);
    std::vector<double> I(o * o, 0.0), E(n * n, 0.0);
    for (int k = 0; k < o; ++k) I[k * o + k] = 1.0;
    for (int k = 0; k < n; ++k) E[k * n + k] = e[k];
    c->delta = c->be->alloc(o * o);
    c->be->upload(c->delta, I.data(), o * o, false);
    c->stage = c->be->alloc(c->dim);
    c->stage2 = c->be->alloc(c->dim);
    // h_pq = eps_p d_pq - sum_k (2 g_pqkk - g_pkkq)  (canonical reference)
    {
      Graph g;
      g.be = c->be.get();
      int Ein = g.input({n, n}, "E");
      int Lin = g.input({J, n, n}, "L");
      int din = g.input({o, o}, "delta");
      int Loo = g.slice(Lin, {0, 0, 0}, {J, o, o});
      int Lpo = g.slice(Lin, {0, 0, 0}, {J, n, o});
      int Lop = g.slice(Lin, {0, 0, 0}, {J, o, n});
      int s = g.contract(Loo, "Jkl", din, "kl", "J");
      int hh = g.add("pq", {{Ein, "pq", 1.0},
                            {g.contract(Lin, "Jpq", s, "J", "pq"), "pq", -2.0},
                            {g.contract(Lpo, "Jpk", Lop, "Jkq", "pq"), "pq", 1.0}});
      g.set_input(Ein, E.data(), false);
      g.set_input(Lin, c->L, true);
      g.set_input(din, c->delta, true);
      g.run({hh});
      c->h = c->be->alloc(n * n);
      c->be->upload(c->h, g.data(hh), n * n, true);
      c->be->sync();
    }
    // HF energy = E0 at t = 0
    Model& m = model(c, false);
    c->be->fill(input_buffer(m.g, m.t1), (int64_t)v * o, 0.0);
    c->be->fill(input_buffer(m.g, m.t2), (int64_t)o * o * v * v, 0.0);
    m.g.touch(m.t1);
    m.g.touch(m.t2);
    m.g.run({m.er.E0});
    c->e_hf = get_scalar(c, m.g, m.er.E0);
    c->be->sync();
  });
  if (rc != SCCSD_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return SCCSD_OK;
}

int sccsd_residual(sccsd_ctx* c, const double* t, double zeta, const double* Ra,
                   const double* Rb, double* omega, double* e_corr) {
  if (!c) return SCCSD_EINVAL;
  if (!t) return fail(c, SCCSD_EINVAL, "t is NULL");
  if ((Ra == nullptr) != (Rb == nullptr)) return fail(c, SCCSD_EINVAL, "give both Ra and Rb or neither");
  if (!std::isfinite(zeta)) return fail(c, SCCSD_EINVAL, "zeta is not finite");
  return guarded(c, [&] {
    bool scc = Ra != nullptr;
    Model& m = model(c, scc);
    load_packed(c, m.g, t, m.t1, m.t2, false);
    if (scc) {
      load_packed(c, m.g, Ra, m.Ra1, m.Ra2, false);
      load_packed(c, m.g, Rb, m.Rb1, m.Rb2, false);
      set_scalar(c, m.g, m.zeta, zeta);
    }
    c->cur = &m;
    std::vector<int> targets = {m.er.E0};
    if (omega) {
      targets.push_back(m.er.O1);
      targets.push_back(m.er.O2);
    }
    m.g.run(targets);
    if (omega) store_packed(c, m.g, m.er.O1, m.er.O2, omega, false);
    if (e_corr) *e_corr = get_scalar(c, m.g, m.er.E0) - c->e_hf;
    c->be->sync();
  });
}

int sccsd_jacobian_right(sccsd_ctx* c, int nvec, const double* R, double* sigma, double* etaR) {
  if (!c) return SCCSD_EINVAL;
  if (nvec < 0 || (nvec > 0 && (!R || !sigma))) return fail(c, SCCSD_EINVAL, "bad vectors");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual first");
  return guarded(c, [&] {
    Model& m = *c->cur;
    std::vector<double> er(nvec, 0.0);
    for (int k0 = 0; k0 < nvec; k0 += c->max_batch) {
      const int nb = std::min(c->max_batch, nvec - k0);
      RightSec& S = right_section(m, nb);
      load_packed_batch(c, m.g, R + (int64_t)k0 * c->dim, nb, S.R1, S.R2, false);
      m.g.run({S.sig1, S.sig2, S.etaR});
      store_packed_batch(c, m.g, nb, S.sig1, S.sig2, sigma + (int64_t)k0 * c->dim, false);
      if (etaR && !m.g.is_zero(S.etaR)) c->be->download(er.data() + k0, m.g.data(S.etaR), nb, false);
    }
    if (etaR) {
      if (c->be->is_device(etaR))
        c->be->upload(etaR, er.data(), nvec, false);
      else
        std::memcpy(etaR, er.data(), sizeof(double) * nvec);
    }
    c->be->sync();
  });
}

int sccsd_jacobian_left(sccsd_ctx* c, int nvec, const double* L, double* sigma) {
  if (!c) return SCCSD_EINVAL;
  if (nvec < 0 || (nvec > 0 && (!L || !sigma))) return fail(c, SCCSD_EINVAL, "bad vectors");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual first");
  return guarded(c, [&] {
    Model& m = *c->cur;
    for (int k0 = 0; k0 < nvec; k0 += c->max_batch) {
      const int nb = std::min(c->max_batch, nvec - k0);
      LeftSec& S = left_section(m, nb);
      load_packed_batch(c, m.g, L + (int64_t)k0 * c->dim, nb, S.Lb1, S.Lb2, true);
      m.g.run({S.lt1, S.lt2});
      store_packed_batch(c, m.g, nb, S.lt1, S.lt2, sigma + (int64_t)k0 * c->dim, true);
    }
    c->be->sync();
  });
}

int sccsd_densities(sccsd_ctx* c, double l0, const double* L, double r0, const double* R,
                    double* D1, double* Gamma) {
  if (!c) return SCCSD_EINVAL;
  if (!L || !R || !D1) return fail(c, SCCSD_EINVAL, "NULL argument");
  if (!std::isfinite(l0) || !std::isfinite(r0)) return fail(c, SCCSD_EINVAL, "l0/r0 not finite");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual first");
  return guarded(c, [&] {
    Model& m = *c->cur;
    load_packed(c, m.g, L, m.Lb1, m.Lb2, true);
    load_packed(c, m.g, R, m.R1, m.R2, false);
    set_scalar(c, m.g, m.s_l0r0, l0 * r0);
    set_scalar(c, m.g, m.s_l0, l0);
    set_scalar(c, m.g, m.s_r0, r0);
    std::vector<int> targets = {m.D1};
    if (Gamma) targets.push_back(m.Gam);
    m.g.run(targets);
    const int64_t n = c->n;
    auto put = [&](int id, double* dst, int64_t cnt) {
      bool dev = c->be->is_device(dst);
      if (m.g.is_zero(id)) {
        if (dev)
          c->be->fill(dst, cnt, 0.0);
        else
          std::memset(dst, 0, sizeof(double) * cnt);
        return;
      }
      if (dev)
        c->be->upload(dst, m.g.data(id), cnt, true);
      else
        c->be->download(dst, m.g.data(id), cnt, false);
    };
    put(m.D1, D1, n * n);
    if (Gamma) put(m.Gam, Gamma, (int64_t)c->J * n * n);
    c->be->sync();
  });
}

void sccsd_destroy(sccsd_ctx* c) { delete c; }

int sccsd_profile(sccsd_ctx* c, int enable) {
  if (!c) return SCCSD_EINVAL;
  return guarded(c, [&] { c->be->profile(enable != 0); });
}

int sccsd_profile_read(sccsd_ctx* c, double* ladder_ms, long long* ladder_calls,
                       double* ladder_flops, long long* launches) {
  if (!c) return SCCSD_EINVAL;
  return guarded(c, [&] {
    long long calls = 0;
    double fl = 0.0;
    c->be->profile_read(ladder_ms, &calls, &fl, launches);
    if (ladder_calls) *ladder_calls = calls;
    if (ladder_flops) *ladder_flops = fl;
  });
}

int sccsd_gemm_tn(int precision, long long M, long long N, long long K, double alpha,
                  const double* A, const double* B, double* C, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C) return SCCSD_EINVAL;
  if (precision < SCCSD_FP64 || precision > SCCSD_BF16) return SCCSD_EINVAL;
  sccsd_ctx tmp;
  return guarded(&tmp, [&] {
    auto be = make_backend(stream, precision);
    for (const double* p : {A, B, (const double*)C})
      if (!be->is_device(p)) throw std::invalid_argument("sccsd_gemm_tn needs device pointers");
    be->gemm_tn(1, M, N, K, alpha, A, B, C, precision != SCCSD_FP64);
    be->sync();
  });
}

}  // extern "C"


// ======================================================================
// Solvers: ground state (Jacobi + DIIS) and EOM roots (Davidson), driven from
// the host with every vector on the device.
// ======================================================================
namespace {

constexpr int kDiis = 8;
constexpr int kMaxSpace = 48;

struct Dev {
  sccsd_ctx* c;
  cudaStream_t st() const { return (cudaStream_t)c->be->stream(); }
  double dot(const double* x, const double* y, int64_t n) {
    double* r = c->sv_small + 4 * kMaxSpace * kMaxSpace;
    c->be->gemm_tn(1, 1, 1, n, 1.0, x, y, r, false);
    double h = 0.0;
    c->be->download(&h, r, 1, false);
    return h;
  }
  void copy(double* dst, const double* src, int64_t n) { c->be->upload(dst, src, n, true); }
  // y = a x + b y
  void axpby(int64_t n, double a, const double* x, double b, double* y) {
    launch_axpby(st(), n, a, x, b, y);
  }
  // out[k][:] = sum_p coef[p][k] V[p][:], coef [m][nk] row-major on the device
  void combine(int nk, int m, const double* coef, const double* V, double* out) {
    MatView A;  // element (k, p) = coef[p * nk + k]
    A.p = coef;
    A.sr2 = 1;
    A.sk2 = nk;
    MatView B;  // element (j, p) = V[p * dim + j]
    B.p = V;
    B.sr2 = 1;
    B.sk2 = c->dim;
    c->be->gemm_view(1, nk, c->dim, m, 1.0, A, B, out, false);
  }
};

// solver work buffer i with room for at least n doubles (grown on demand)
double* solver_buf(sccsd_ctx* c, size_t i, int64_t n) {
  if (c->sv.size() <= i) {
    c->sv.resize(i + 1, nullptr);
    c->sv_n.resize(i + 1, 0);
  }
  if (c->sv[i] && c->sv_n[i] < n) {
    c->be->sync();
    c->be->release(c->sv[i]);
    c->sv[i] = nullptr;
  }
  if (!c->sv[i]) {
    c->sv[i] = c->be->alloc(n);
    c->sv_n[i] = n;
  }
  return c->sv[i];
}

void ensure_small(sccsd_ctx* c) {
  if (!c->sv_small) c->sv_small = c->be->alloc(6 * kMaxSpace * kMaxSpace + 16);
  if (!c->sv_info) c->sv_info = (int*)c->be->alloc(kMaxSpace + 4);
}

void switch_precision(sccsd_ctx* c, int p) {
  if (c->be->get_precision() == p) return;
  c->be->set_precision(p);
  for (Model* m : {c->plain.get(), c->scc.get()})
    if (m) m->g.invalidate();
}

// E0 and packed omega (device) at packed amplitudes t (device)
double eval_residual(sccsd_ctx* c, const double* t, double zeta, const double* Ra,
                     const double* Rb, double* om) {
  const bool scc = Ra != nullptr;
  Model& m = model(c, scc);
  load_packed(c, m.g, t, m.t1, m.t2, false);
  if (scc) {
    load_packed(c, m.g, Ra, m.Ra1, m.Ra2, false);
    load_packed(c, m.g, Rb, m.Rb1, m.Rb2, false);
    set_scalar(c, m.g, m.zeta, zeta);
  }
  c->cur = &m;
  m.g.run({m.er.E0, m.er.O1, m.er.O2});
  store_packed(c, m.g, m.er.O1, m.er.O2, om, false);
  return get_scalar(c, m.g, m.er.E0);
}

// sigma[k] = A V[k] (side 0) or A^T V[k] (side 1), all on the device
void transform(sccsd_ctx* c, int side, int nvec, const double* V, double* W) {
  Model& m = *c->cur;
  for (int k0 = 0; k0 < nvec; k0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nvec - k0);
    if (side == 0) {
      RightSec& S = right_section(m, nb);
      load_packed_batch(c, m.g, V + (int64_t)k0 * c->dim, nb, S.R1, S.R2, false);
      m.g.run({S.sig1, S.sig2});
      store_packed_batch(c, m.g, nb, S.sig1, S.sig2, W + (int64_t)k0 * c->dim, false);
    } else {
      LeftSec& S = left_section(m, nb);
      load_packed_batch(c, m.g, V + (int64_t)k0 * c->dim, nb, S.Lb1, S.Lb2, true);
      m.g.run({S.lt1, S.lt2});
      store_packed_batch(c, m.g, nb, S.lt1, S.lt2, W + (int64_t)k0 * c->dim, true);
    }
  }
}

}  // namespace

extern "C" {

int sccsd_overlap(sccsd_ctx* c, double ra0, const double* Ra, double rb0, const double* Rb,
                  double* O) {
  if (!c) return SCCSD_EINVAL;
  if (!Ra || !Rb || !O) return fail(c, SCCSD_EINVAL, "NULL argument");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual or a solver first");
  return guarded(c, [&] {
    Model& m = *c->cur;
    OverlapSec& S = overlap_section(m);
    set_scalar(c, m.g, S.ra0, ra0);
    set_scalar(c, m.g, S.rb0, rb0);
    load_packed(c, m.g, Ra, S.ra1, S.ra2, false);
    load_packed(c, m.g, Rb, S.rb1, S.rb2, false);
    m.g.run({S.O});
    *O = get_scalar(c, m.g, S.O);
    c->be->sync();
  });
}

int sccsd_set_precision(sccsd_ctx* c, int precision) {
  if (!c) return SCCSD_EINVAL;
  if (precision < SCCSD_FP64 || precision > SCCSD_BF16) return fail(c, SCCSD_EINVAL, "bad precision");
  return guarded(c, [&] {
    switch_precision(c, precision);
    c->precision = precision;
  });
}

int sccsd_solve_ground(sccsd_ctx* c, const double* t0, double zeta, const double* Ra,
                       const double* Rb, double tol, int maxit, double refine_tol, double* t_out,
                       double* e_corr, int* iterations) {
  if (!c) return SCCSD_EINVAL;
  if (!(tol > 0.0) || maxit < 1) return fail(c, SCCSD_EINVAL, "bad tolerance or iteration limit");
  if ((Ra == nullptr) != (Rb == nullptr)) return fail(c, SCCSD_EINVAL, "give both Ra and Rb or neither");
  int status = SCCSD_OK;
  int rc = guarded(c, [&] {
    Dev d{c};
    ensure_small(c);
    const int64_t dim = c->dim;
    double* t = solver_buf(c, 0, dim);
    double* om = solver_buf(c, 1, dim);
    double* tn = solver_buf(c, 2, dim);
    double* X = solver_buf(c, 3, kDiis * dim);
    double* Rr = solver_buf(c, 4, kDiis * dim);
    double* Bm = c->sv_small;
    double* cf = c->sv_small + kMaxSpace * kMaxSpace;
    // device copies of the SCC vectors (they may be host arrays)
    const double *ra = Ra, *rb = Rb;
    if (Ra) {
      double* a = solver_buf(c, 5, dim);
      double* b = solver_buf(c, 6, dim);
      c->be->upload(a, Ra, dim, c->be->is_device(Ra));
      c->be->upload(b, Rb, dim, c->be->is_device(Rb));
      ra = a;
      rb = b;
    }
    if (t0)
      c->be->upload(t, t0, dim, c->be->is_device(t0));
    else
      c->be->fill(t, dim, 0.0);
    const int p0 = c->be->get_precision();
    const bool refine = p0 != SCCSD_FP64 && refine_tol > 0.0;
    bool fp64_phase = !refine;
    int nh = 0, head = 0, it = 0;
    double E = 0.0, nrm = 0.0;
    double best = 1e300;
    int since_best = 0;
    // Update denominators: the dressed denominators D' from the diagonals of
    // the dressed Fock-like intermediates at the current amplitudes, refreshed
    // at iterations 3, 6, 12, 24, ... (DIIS restarts with each refresh) and
    // floored at 0.2 D. Before the first refresh: the caller's (or learned)
    // preconditioner when one is set, else the orbital-energy denominators D
    // (which D' equals at t = 0).
    double* Dp = solver_buf(c, 7, dim);
    double* fdg = solver_buf(c, 8, c->o + c->v);
    bool have_dp = false;
    int next_refresh = 3;
    for (it = 1; it <= maxit; ++it) {
      E = eval_residual(c, t, zeta, ra, rb, om);
      nrm = std::sqrt(d.dot(om, om, dim));
      if (getenv("SCCSD_LOG"))
        fprintf(stderr, "{\"solver\": \"ground\", \"iter\": %d, \"fp64\": %d, \"residual\": %.3e, \"e_corr\": %.12f}\n", it,
                (int)fp64_phase, nrm, E - c->e_hf);
      if (!std::isfinite(nrm)) throw std::runtime_error("ground state diverged (non-finite residual)");
      if (nrm < 0.9 * best) {
        best = nrm;
        since_best = 0;
      } else {
        ++since_best;
      }
      // the mixed phase ends below refine_tol, or when it stalls at its noise floor
      if (!fp64_phase && (nrm < refine_tol || since_best >= 6)) {
        // mixed-precision phase done: refine in FP64 from the current amplitudes
        switch_precision(c, SCCSD_FP64);
        fp64_phase = true;
        nh = 0;
        head = 0;
        --it;
        continue;
      }
      if (fp64_phase && nrm < tol) break;
      const double* Dstep = c->use_dprec ? c->Dprec : c->D;
      {
        if (it >= next_refresh) {
          Model& mdl = *c->cur;
          mdl.g.run({mdl.er.Fooi, mdl.er.Fvvi});
          const int o = c->o, v = c->v;
          int64_t d1[1] = {o}, os1[1] = {1}, is1[1] = {o + 1};
          c->be->copy_view(1, d1, fdg, os1, mdl.g.data(mdl.er.Fooi), is1, 1.0, false);
          int64_t d2[1] = {v}, os2[1] = {1}, is2[1] = {v + 1};
          c->be->copy_view(1, d2, fdg + o, os2, mdl.g.data(mdl.er.Fvvi), is2, 1.0, false);
          launch_denoms(d.st(), o, v, fdg, Dp);
          launch_floor(d.st(), dim, c->D, 0.2, Dp);
          have_dp = true;
          next_refresh *= 2;
          nh = 0;
          head = 0;
        }
        if (have_dp) Dstep = Dp;
      }
      launch_jacobi(d.st(), dim, t, om, Dstep, tn);
      const int slot = head;
      head = (head + 1) % kDiis;
      nh = std::min(nh + 1, kDiis);
      d.copy(X + (int64_t)slot * dim, tn, dim);
      d.copy(Rr + (int64_t)slot * dim, tn, dim);
      d.axpby(dim, -1.0, t, 1.0, Rr + (int64_t)slot * dim);
      if (nh >= 2) {
        c->be->gemm_tn(1, nh, nh, dim, 1.0, Rr, Rr, Bm, false);
        launch_diis(d.st(), nh, Bm, cf, c->sv_info);
        int info = 0;
        cudaMemcpyAsync(&info, c->sv_info, sizeof(int), cudaMemcpyDeviceToHost, d.st());
        c->be->sync();
        if (info == 0)
          d.combine(1, nh, cf, X, t);
        else
          d.copy(t, tn, dim);
      } else {
        d.copy(t, tn, dim);
      }
    }
    if (it > maxit) status = SCCSD_ENOTCONV;
    if (refine) switch_precision(c, p0);
    if (refine) eval_residual(c, t, zeta, ra, rb, om);  // fix the state for later transforms
    if (t_out) c->be->download(t_out, t, dim, c->be->is_device(t_out));
    if (e_corr) *e_corr = E - c->e_hf;
    if (iterations) *iterations = std::min(it, maxit);
    c->be->sync();
  });
  if (rc != SCCSD_OK) return rc;
  if (status != SCCSD_OK) return fail(c, status, "ground state not converged within maxit");
  return SCCSD_OK;
}

int sccsd_solve_states(sccsd_ctx* c, int nroots, int side, double tol, int maxit,
                       double refine_tol, double* omega, double* vecs, int* iterations) {
  if (!c) return SCCSD_EINVAL;
  if (nroots < 1 || nroots > 12 || (side != 0 && side != 1) || !(tol > 0.0) || maxit < 1 || !omega)
    return fail(c, SCCSD_EINVAL, "bad arguments");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual or sccsd_solve_ground first");
  int status = SCCSD_OK;
  int rc = guarded(c, [&] {
    Dev d{c};
    ensure_small(c);
    const int64_t dim = c->dim;
    const int mmax = kMaxSpace;
    if (dim < mmax) throw std::invalid_argument("problem too small for the requested roots");
    double* V = solver_buf(c, 10, (int64_t)kMaxSpace * dim);
    double* W = solver_buf(c, 11, (int64_t)kMaxSpace * dim);
    double* Xr = solver_buf(c, 12, 12 * dim);
    double* AX = solver_buf(c, 13, 12 * dim);
    double* Rz = solver_buf(c, 14, 13 * dim);
    double* Xp = solver_buf(c, 15, 12 * dim);   // Ritz vectors of the previous iteration
    double* AXp = solver_buf(c, 16, 12 * dim);
    bool have_prev = false;
    double* S = c->sv_small;
    double* Y = c->sv_small + kMaxSpace * kMaxSpace;
    double* wr = c->sv_small + 2 * kMaxSpace * kMaxSpace;
    double* wi = wr + kMaxSpace;
    double* cf = wi + kMaxSpace;
    double* G = c->sv_small + 3 * kMaxSpace * kMaxSpace;
    int* order = c->sv_info;
    int* info_d = c->sv_info + kMaxSpace;
    cudaStream_t st = d.st();
    auto get_info = [&]() {
      int h = 0;
      cudaMemcpyAsync(&h, info_d, sizeof(int), cudaMemcpyDeviceToHost, st);
      c->be->sync();
      return h;
    };
    // Gram-Schmidt of vec (and the same combination of its image) against V[0:m)
    auto orthogonalize = [&](double* vec, double* img, int m) {
      for (int pass = 0; pass < 2 && m > 0; ++pass) {
        c->be->gemm_tn(1, m, 1, dim, 1.0, V, vec, cf, false);     // cf[p] = v_p . vec
        double* tmp = Rz + 12 * dim;
        d.combine(1, m, cf, V, tmp);
        d.axpby(dim, -1.0, tmp, 1.0, vec);
        if (img) {
          d.combine(1, m, cf, W, tmp);
          d.axpby(dim, -1.0, tmp, 1.0, img);
        }
      }
    };
    // Preconditioner: dressed denominators D'_ai = f_a - f_i, D'_aibj = f_a + f_b
    // - f_i - f_j from the diagonals f of the Fock-like intermediates at the
    // fixed state (they carry most of the correlation shift of diag(A));
    // initial guesses: unit vectors on the lowest singles D'.
    const int o = c->o, v = c->v;
    Model& mdl = *c->cur;
    mdl.g.run({mdl.er.Fooi, mdl.er.Fvvi});
    double* fdiag = solver_buf(c, 17, o + v);
    double* Dp = solver_buf(c, 18, dim);
    {
      int64_t d1[1] = {o}, os1[1] = {1}, is1[1] = {o + 1};
      c->be->copy_view(1, d1, fdiag, os1, mdl.g.data(mdl.er.Fooi), is1, 1.0, false);
      int64_t d2[1] = {v}, os2[1] = {1}, is2[1] = {v + 1};
      c->be->copy_view(1, d2, fdiag + o, os2, mdl.g.data(mdl.er.Fvvi), is2, 1.0, false);
    }
    launch_denoms(st, o, v, fdiag, Dp);
    std::vector<double> fh(o + v);
    c->be->download(fh.data(), fdiag, o + v, false);
    std::vector<std::pair<double, int>> dd;
    for (int a = 0; a < v; ++a)
      for (int i = 0; i < o; ++i) dd.push_back({fh[o + a] - fh[i], a * o + i});
    std::sort(dd.begin(), dd.end());
    int m = std::min<int>(std::min<int>((int)dd.size(), 2 * nroots + 2), mmax);
    c->be->fill(V, (int64_t)m * dim, 0.0);
    for (int k = 0; k < m; ++k) {
      double one = 1.0;
      c->be->upload(V + (int64_t)k * dim + dd[k].second, &one, 1, false);
    }
    transform(c, side, m, V, W);
    const int p0 = c->be->get_precision();
    const bool refine = p0 != SCCSD_FP64 && refine_tol > 0.0;
    bool fp64_phase = !refine;
    std::vector<double> lam(nroots), res(nroots);
    int it = 0;
    bool converged = false;
    double best = 1e300;
    int since_best = 0;
    for (it = 1; it <= maxit; ++it) {
      // subspace matrix and its lowest roots
      c->be->gemm_tn(1, m, m, dim, 1.0, V, W, S, false);
      launch_small_eig(st, m, S, wr, wi, Y, nroots, order, info_d);
      int info = get_info();
      if (info == 3) throw std::domain_error("complex pair among the lowest roots");
      if (info != 0) throw std::runtime_error("subspace eigensolver failed");
      std::vector<int> ord(nroots);
      cudaMemcpyAsync(ord.data(), order, sizeof(int) * nroots, cudaMemcpyDeviceToHost, st);
      std::vector<double> w(m);
      cudaMemcpyAsync(w.data(), wr, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
      c->be->sync();
      for (int k = 0; k < nroots; ++k) lam[k] = w[ord[k]];
      // Ritz vectors, their images and residuals
      d.combine(nroots, m, Y, V, Xr);
      d.combine(nroots, m, Y, W, AX);
      launch_ritz_residual(st, nroots, dim, AX, Xr, wr, order, Rz);
      c->be->gemm_tn(1, nroots, nroots, dim, 1.0, Rz, Rz, G, false);
      c->be->gemm_tn(1, nroots, nroots, dim, 1.0, Xr, Xr, G + 144, false);
      std::vector<double> g1(nroots * nroots), g2(nroots * nroots);
      c->be->download(g1.data(), G, nroots * nroots, false);
      c->be->download(g2.data(), G + 144, nroots * nroots, false);
      double worst = 0.0;
      for (int k = 0; k < nroots; ++k) {
        res[k] = std::sqrt(g1[k * nroots + k] / g2[k * nroots + k]);
        worst = std::max(worst, res[k]);
      }
      if (getenv("SCCSD_LOG")) {
        fprintf(stderr, "{\"solver\": \"davidson\", \"iter\": %d, \"space\": %d, \"fp64\": %d, \"max_res\": %.3e, \"omega\": [", it, m,
                (int)fp64_phase, worst);
        for (int k = 0; k < nroots; ++k) fprintf(stderr, "%s%.12f", k ? ", " : "", lam[k]);
        fprintf(stderr, "]}\n");
      }
      if (worst < 0.9 * best) {
        best = worst;
        since_best = 0;
      } else {
        ++since_best;
      }
      if (!fp64_phase && (worst < refine_tol || since_best >= 8)) {
        // restart in FP64 from the current Ritz vectors
        switch_precision(c, SCCSD_FP64);
        fp64_phase = true;
        have_prev = false;
        d.copy(V, Xr, (int64_t)nroots * dim);
        m = 0;
        for (int k = 0; k < nroots; ++k) {
          double* vk = V + (int64_t)m * dim;
          if (k != m) d.copy(vk, Xr + (int64_t)k * dim, dim);
          orthogonalize(vk, nullptr, m);
          double nn = std::sqrt(d.dot(vk, vk, dim));
          if (nn < 1e-10) continue;
          d.axpby(dim, 0.0, vk, 1.0 / nn, vk);
          ++m;
        }
        transform(c, side, m, V, W);
        continue;
      }
      if (fp64_phase && worst < tol) {
        converged = true;
        break;
      }
      // preconditioned residuals of the unconverged roots
      std::vector<int> want;
      for (int k = 0; k < nroots; ++k)
        if (res[k] >= tol) want.push_back(k);
      if (m + (int)want.size() > mmax) {
        // thick restart: current and previous Ritz vectors, orthonormalised
        // (their images follow the same combinations)
        d.copy(V, Xr, (int64_t)nroots * dim);
        d.copy(W, AX, (int64_t)nroots * dim);
        int nk = nroots;
        if (have_prev) {
          d.copy(V + (int64_t)nroots * dim, Xp, (int64_t)nroots * dim);
          d.copy(W + (int64_t)nroots * dim, AXp, (int64_t)nroots * dim);
          nk = 2 * nroots;
        }
        int mm = 0;
        for (int k = 0; k < nk; ++k) {
          double* vk = V + (int64_t)mm * dim;
          double* wk = W + (int64_t)mm * dim;
          if (k != mm) {
            d.copy(vk, V + (int64_t)k * dim, dim);
            d.copy(wk, W + (int64_t)k * dim, dim);
          }
          orthogonalize(vk, wk, mm);
          double nn = std::sqrt(d.dot(vk, vk, dim));
          if (!(nn > 1e-10)) continue;
          d.axpby(dim, 0.0, vk, 1.0 / nn, vk);
          d.axpby(dim, 0.0, wk, 1.0 / nn, wk);
          ++mm;
        }
        m = mm;
      }
      d.copy(Xp, Xr, (int64_t)nroots * dim);
      d.copy(AXp, AX, (int64_t)nroots * dim);
      have_prev = true;
      int added = 0;
      for (int k : want) {
        double* nv = V + (int64_t)(m + added) * dim;
        launch_precond(st, dim, Rz + (int64_t)k * dim, Dp, lam[k], nv);
        double n0 = std::sqrt(d.dot(nv, nv, dim));
        orthogonalize(nv, nullptr, m + added);
        double nn = std::sqrt(d.dot(nv, nv, dim));
        if (!(nn > 1e-8 * n0) || nn == 0.0) continue;
        d.axpby(dim, 0.0, nv, 1.0 / nn, nv);
        ++added;
      }
      if (added == 0) throw std::runtime_error("Davidson subspace stagnated");
      transform(c, side, added, V + (int64_t)m * dim, W + (int64_t)m * dim);
      m += added;
    }
    if (!converged) status = SCCSD_ENOTCONV;
    if (refine) switch_precision(c, p0);
    for (int k = 0; k < nroots; ++k) omega[k] = lam[k];
    if (vecs) {
      // unit-norm Ritz vectors
      for (int k = 0; k < nroots; ++k) {
        double* xk = Xr + (int64_t)k * dim;
        double nn = std::sqrt(d.dot(xk, xk, dim));
        d.axpby(dim, 0.0, xk, 1.0 / nn, xk);
      }
      c->be->download(vecs, Xr, (int64_t)nroots * dim, c->be->is_device(vecs));
    }
    if (iterations) *iterations = std::min(it, maxit);
    c->be->sync();
  });
  if (rc != SCCSD_OK) return rc;
  if (status != SCCSD_OK) return fail(c, status, "roots not converged within maxit");
  return SCCSD_OK;
}

}  // extern "C"

extern "C" {

// Self-consistent SCCSD for the two lowest states (K = {a, b}, Sec. 2.4.2).
int sccsd_solve_scc(sccsd_ctx* c, double tol, int maxit, double ground_tol, double eom_tol,
                    double* zeta_out, double* e_corr, double* omega2, double* r0_2, double* Ra_out,
                    double* Rb_out, int* iterations) {
  if (!c) return SCCSD_EINVAL;
  if (!(tol > 0.0) || maxit < 1 || !(ground_tol > 0.0) || !(eom_tol > 0.0))
    return fail(c, SCCSD_EINVAL, "bad tolerances or iteration limit");
  int status = SCCSD_OK;
  int rc = guarded(c, [&] {
    const int64_t dim = c->dim;
    std::vector<double> t(dim), vecs(2 * dim), sig(2 * dim), Ra(dim), Rb(dim);
    double zeta = 0.0, E = 0.0, O = 0.0;
    double w[2] = {0.0, 0.0}, r0[2] = {0.0, 0.0};
    bool have_states = false, have_t = false;
    std::vector<std::pair<double, double>> hist;
    auto check = [&](int r) {
      if (r != SCCSD_OK) throw std::runtime_error("inner solver failed: " + c->err);
    };
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
      int gi = 0;
      if (have_states)
        check(sccsd_solve_ground(c, have_t ? t.data() : nullptr, zeta, Ra.data(), Rb.data(),
                                 ground_tol, 1000, 1e-5, t.data(), &E, &gi));
      else
        check(sccsd_solve_ground(c, nullptr, 0.0, nullptr, nullptr, ground_tol, 1000, 1e-5,
                                 t.data(), &E, &gi));
      have_t = true;
      int si = 0;
      check(sccsd_solve_states(c, 2, 0, eom_tol, 1000, 1e-4, w, vecs.data(), &si));
      // sign convention: largest |component| positive
      for (int k = 0; k < 2; ++k) {
        double* x = vecs.data() + k * dim;
        int64_t im = 0;
        for (int64_t q = 1; q < dim; ++q)
          if (std::fabs(x[q]) > std::fabs(x[im])) im = q;
        if (x[im] < 0)
          for (int64_t q = 0; q < dim; ++q) x[q] = -x[q];
      }
      double etaR[2];
      check(sccsd_jacobian_right(c, 2, vecs.data(), sig.data(), etaR));
      r0[0] = etaR[0] / w[0];
      r0[1] = etaR[1] / w[1];
      check(sccsd_overlap(c, r0[0], vecs.data(), r0[1], vecs.data() + dim, &O));
      if (getenv("SCCSD_LOG"))
        fprintf(stderr, "{\"solver\": \"scc\", \"iter\": %d, \"zeta\": %.12f, \"O_ab\": %.3e, \"omega\": [%.12f, %.12f]}\n",
                it, zeta, O, w[0], w[1]);
      hist.push_back({zeta, O});
      std::copy(vecs.begin(), vecs.begin() + dim, Ra.begin());
      std::copy(vecs.begin() + dim, vecs.end(), Rb.begin());
      have_states = true;
      if (std::fabs(O) < tol && hist.size() > 1 &&
          std::fabs(hist[hist.size() - 1].first - hist[hist.size() - 2].first) < 1e-8)
        break;
      if (hist.size() == 1) {
        zeta = zeta - O;
      } else {
        auto [z1, o1] = hist[hist.size() - 2];
        auto [z2, o2] = hist[hist.size() - 1];
        zeta = (o2 != o1) ? z2 - o2 * (z2 - z1) / (o2 - o1) : z2;
      }
    }
    if (it > maxit) status = SCCSD_ENOTCONV;
    if (zeta_out) *zeta_out = hist.back().first;
    if (e_corr) *e_corr = E;
    if (omega2) {
      omega2[0] = w[0];
      omega2[1] = w[1];
    }
    if (r0_2) {
      r0_2[0] = r0[0];
      r0_2[1] = r0[1];
    }
    for (auto pr : {std::make_pair(Ra_out, &Ra), std::make_pair(Rb_out, &Rb)}) {
      if (!pr.first) continue;
      if (c->be->is_device(pr.first))
        c->be->upload(pr.first, pr.second->data(), dim, false);
      else
        std::memcpy(pr.first, pr.second->data(), sizeof(double) * dim);
    }
    if (iterations) *iterations = std::min(it, maxit);
  });
  if (rc != SCCSD_OK) return rc;
  if (status != SCCSD_OK) return fail(c, status, "zeta iteration not converged within maxit");
  return SCCSD_OK;
}

}  // extern "C"

// ======================================================================
// Learned initial guess and preconditioner (per-amplitude MLP)
// ======================================================================
namespace {

// diagonals f of the dressed one-body intermediates at the fixed state
void dressed_diagonals(sccsd_ctx* c, double* f) {
  Model& m = *c->cur;
  m.g.run({m.er.Fooi, m.er.Fvvi});
  const int64_t o = c->o, v = c->v;
  int64_t d1[1] = {o}, os1[1] = {1}, is1[1] = {o + 1};
  c->be->copy_view(1, d1, f, os1, m.g.data(m.er.Fooi), is1, 1.0, false);
  int64_t d2[1] = {v}, os2[1] = {1}, is2[1] = {v + 1};
  c->be->copy_view(1, d2, f + o, os2, m.g.data(m.er.Fvvi), is2, 1.0, false);
}

struct Scales {
  double st, sg, sD;
};

// features at the MP2 amplitudes into X [o^2 v^2][10]; returns the scales
Scales learned_features(sccsd_ctx* c, float* X) {
  Dev d{c};
  ensure_small(c);
  const int64_t dim = c->dim, o = c->o, v = c->v, nf = o * o * v * v;
  double* tz = solver_buf(c, 30, dim);
  double* om = solver_buf(c, 31, dim);
  double* tm = solver_buf(c, 32, dim);
  double* t1 = solver_buf(c, 33, o * v);
  double* t2 = solver_buf(c, 34, nf);
  double* f = solver_buf(c, 35, o + v);
  c->be->fill(tz, dim, 0.0);
  eval_residual(c, tz, 0.0, nullptr, nullptr, om);
  launch_jacobi(d.st(), dim, tz, om, c->D, tm);          // MP2 first iterate
  eval_residual(c, tm, 0.0, nullptr, nullptr, om);
  dressed_diagonals(c, f);
  Model& m = *c->cur;
  m.g.run({m.er.Govov});
  const double* g = m.g.data(m.er.Govov);
  c->be->unpack(tm, c->o, c->v, t1, t2, false);
  Scales s;
  s.st = std::sqrt(d.dot(t2, t2, nf) / nf);
  s.sg = std::sqrt(d.dot(g, g, nf) / nf);
  double eo = 0, ev = 0;
  for (int i = 0; i < c->o; ++i) eo += c->eps_host[i];
  for (int a = 0; a < c->v; ++a) ev += c->eps_host[c->o + a];
  s.sD = 2.0 * (ev / c->v - eo / c->o);
  if (!(s.st > 0)) s.st = 1.0;
  if (!(s.sg > 0)) s.sg = 1.0;
  launch_learned_features(d.st(), c->o, c->v, t2, g, c->eps_dev, f, s.st, s.sg, s.sD, X);
  return s;
}

}  // namespace

extern "C" {

int sccsd_learned_features(sccsd_ctx* c, float* X, double* scales) {
  if (!c || !X) return SCCSD_EINVAL;
  if (!c->be->is_device(X)) return fail(c, SCCSD_EINVAL, "X must be device memory");
  return guarded(c, [&] {
    Scales s = learned_features(c, X);
    if (scales) {
      scales[0] = s.st;
      scales[1] = s.sg;
      scales[2] = s.sD;
    }
    c->be->sync();
  });
}

int sccsd_learned_targets(sccsd_ctx* c, const double* t, double st, float* Y) {
  if (!c || !t || !Y || !(st > 0)) return SCCSD_EINVAL;
  if (!c->be->is_device(Y)) return fail(c, SCCSD_EINVAL, "Y must be device memory");
  return guarded(c, [&] {
    const int64_t dim = c->dim, o = c->o, v = c->v, nf = o * o * v * v;
    double* tt = solver_buf(c, 30, dim);
    double* om = solver_buf(c, 31, dim);
    double* t1 = solver_buf(c, 33, o * v);
    double* t2 = solver_buf(c, 34, nf);
    double* f = solver_buf(c, 35, o + v);
    c->be->upload(tt, t, dim, c->be->is_device(t));
    eval_residual(c, tt, 0.0, nullptr, nullptr, om);
    dressed_diagonals(c, f);
    c->be->unpack(tt, c->o, c->v, t1, t2, false);
    launch_learned_targets((cudaStream_t)c->be->stream(), c->o, c->v, t2, c->eps_dev, f, st, Y);
    c->be->sync();
  });
}

int sccsd_mlp_forward(sccsd_mlp* net, const float* X, long long N, float* Y);

int sccsd_learned_guess(sccsd_ctx* c, sccsd_mlp* net, double* t0, double* Dprec) {
  if (!c || !net || !t0 || !Dprec) return SCCSD_EINVAL;
  return guarded(c, [&] {
    const int64_t dim = c->dim, o = c->o, v = c->v, nf = o * o * v * v;
    float* X = (float*)solver_buf(c, 36, nf * 5);   // nf x 10 floats
    float* Y = (float*)solver_buf(c, 37, nf);       // nf x 2 floats
    Scales s = learned_features(c, X);
    if (sccsd_mlp_forward(net, X, nf, Y) != SCCSD_OK) throw std::runtime_error("network forward failed");
    double* t2 = solver_buf(c, 34, nf);
    double* d2 = solver_buf(c, 38, nf);
    double* z1 = solver_buf(c, 39, o * v);
    double* f = solver_buf(c, 35, o + v);
    double* outt = solver_buf(c, 40, dim);
    double* outd = solver_buf(c, 41, dim);
    cudaStream_t st = (cudaStream_t)c->be->stream();
    launch_learned_apply(st, c->o, c->v, Y, c->eps_dev, s.st, t2, d2);
    c->be->fill(z1, o * v, 0.0);
    c->be->pack(z1, t2, c->o, c->v, outt, false);
    // singles of the preconditioner: dressed denominators at the MP2 amplitudes
    double* fd = solver_buf(c, 42, dim);
    launch_denoms(st, c->o, c->v, f, fd);
    c->be->pack(z1, d2, c->o, c->v, outd, false);
    c->be->upload(outd, fd, o * v, true);
    c->be->download(t0, outt, dim, c->be->is_device(t0));
    c->be->download(Dprec, outd, dim, c->be->is_device(Dprec));
    c->be->sync();
  });
}

int sccsd_set_preconditioner(sccsd_ctx* c, const double* Dprec) {
  if (!c) return SCCSD_EINVAL;
  return guarded(c, [&] {
    if (!Dprec) {
      c->use_dprec = false;
      return;
    }
    if (!c->Dprec) c->Dprec = c->be->alloc(c->dim);
    c->be->upload(c->Dprec, Dprec, c->dim, c->be->is_device(Dprec));
    c->use_dprec = true;
    c->be->sync();
  });
}

}  // extern "C"

// ======================================================================
// CUDA graphs of the right transformation (many instances in one launch)
// ======================================================================
extern "C" {

int sccsd_capture_transform(sccsd_ctx* c, int side, int nvec, const double* R, double* sigma,
                            void** graph) {
  if (!c) return SCCSD_EINVAL;
  if (!R || !sigma || !graph || nvec < 1 || (side != 0 && side != 1))
    return fail(c, SCCSD_EINVAL, "bad capture arguments");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual first");
  if (!c->be->is_device(R) || !c->be->is_device(sigma))
    return fail(c, SCCSD_EINVAL, "capture needs device vectors");
  if (c->be->stream() == nullptr)
    return fail(c, SCCSD_EINVAL, "capture needs a context created with a (non-default) stream");
  cudaStream_t st = (cudaStream_t)c->be->stream();
  return guarded(c, [&] {
    // warm-up with the same targets: sizes every buffer and pool slot the
    // captured launches use, converts the state-dependent operands once
    transform(c, side, nvec, R, sigma);
    c->be->sync();
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      throw CudaError("cudaStreamBeginCapture failed");
    cudaGraph_t g = nullptr;
    try {
      c->be->set_capturing(true);
      transform(c, side, nvec, R, sigma);
      c->be->set_capturing(false);
    } catch (...) {
      c->be->set_capturing(false);
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g) throw CudaError("cudaStreamEndCapture failed");
    *graph = (void*)g;
  });
}

int sccsd_graph_join(void** graphs, int n, void** exec) {
  if (!graphs || n < 1 || !exec) return SCCSD_EINVAL;
  cudaGraph_t parent = nullptr;
  if (cudaGraphCreate(&parent, 0) != cudaSuccess) return SCCSD_ECUDA;
  for (int k = 0; k < n; ++k) {
    cudaGraphNode_t node;
    if (!graphs[k] ||
        cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, (cudaGraph_t)graphs[k]) != cudaSuccess) {
      cudaGraphDestroy(parent);
      cudaGetLastError();
      return SCCSD_ECUDA;
    }
  }
  cudaGraphExec_t e = nullptr;
  cudaError_t r = cudaGraphInstantiate(&e, parent, 0);
  cudaGraphDestroy(parent);
  if (r != cudaSuccess) {
    cudaGetLastError();
    return SCCSD_ECUDA;
  }
  *exec = (void*)e;
  return SCCSD_OK;
}

int sccsd_graph_launch(void* exec, void* stream) {
  if (!exec) return SCCSD_EINVAL;
  if (cudaGraphLaunch((cudaGraphExec_t)exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return SCCSD_ECUDA;
  }
  return SCCSD_OK;
}

void sccsd_graph_destroy(void* graph) {
  if (graph) cudaGraphDestroy((cudaGraph_t)graph);
}

void sccsd_graph_exec_destroy(void* exec) {
  if (exec) cudaGraphExecDestroy((cudaGraphExec_t)exec);
}

}  // extern "C"

// ======================================================================
// Lagrangian multipliers of SCCSD gradients and couplings (Sec. 2.3.1-2.3.4)
//
// K = {a, b}, natural projection, fixed orbitals. Unknowns
// u = (zbar, Lb_a, Lb_b, gbar); lb0_k = gbar (dO_ab/dr0_k) / omega_k and
// Ebar_k = E_k (delta_kn - <Lbar_k|R_k>) are closed forms (Sec. 2.3.3), and
// with the bras K_k = (delta_kn - <Lbar_k|R_k>) L_k + Lb_k (Sec. 2.3.2; no
// delta_kn for a coupling) the stationarity residual is
//   r_t    = sum_k d<K_k|Hbar|R_k>/dt + d(zbar.Omega)/dt + gbar dO_ab/dt (+ dO_mn/dt)
//   r_Rk   = d<K_k|Hbar|R_k>/dR_k - omega_k K_k + sum_j d<K_j|Hbar|R_j>/dR_k|X3
//            + d(zbar.Omega)/dR_k + gbar dO_ab/dR_k (+ delta_kn L_m)
//   r_zeta = sum_k d<K_k|Hbar|R_k>/dzeta + d(zbar.Omega)/dzeta
// (zbar.Omega = <(0, zbar)|Hbar|(1, 0)>). The map u -> r is affine; it is
// solved by right-preconditioned restarted GMRES with the dressed diagonal
// denominators, and refined in FP64 when the context computes in a mixed
// precision: the FP64 residual drives correction solves in the mixed mode.
// ======================================================================
namespace {

struct MultSolver {
  sccsd_ctx* c;
  Model* m;
  int kind, ms, ns;  // 0 gradient of state ns; 1 coupling <psi_ms|d psi_ns>
  // The equations depend on Lb_k only through K_k, so Lb_k -> Lb_k + a L_k is
  // an exact null direction. The solver adds (Lb_k . R_k) L_k to the R_k
  // equations: their original part has no component along R_k at a solution,
  // so the solutions coincide, the gauge Lb_k . R_k = 0 is selected and the
  // system becomes nonsingular (a small inconsistency of a not fully
  // converged state no longer drives the iterate along the null direction).
  bool gauge_fix = false;
  int64_t dim, N;
  const double* vec[5];  // t, Ra, Rb, La, Lb (device, packed)
  double zeta, r0[2], omega[2], E0 = 0.0, dO[2] = {0.0, 0.0};
  double *tmp, *zero, *zero1, *zero2, *Kb[2], *Bc, *Ot, *Pd;
  cudaStream_t st() const { return (cudaStream_t)c->be->stream(); }

  double dot(const double* x, const double* y, int64_t n) {
    double* r = c->sv_small + 4 * kMaxSpace * kMaxSpace;
    c->be->gemm_tn(1, 1, 1, n, 1.0, x, y, r, false);
    double h = 0.0;
    c->be->download(&h, r, 1, false);
    return h;
  }
  double get(const double* p) {
    double h = 0.0;
    c->be->download(&h, p, 1, false);
    return h;
  }
  void put(double* p, double v) { c->be->upload(p, &v, 1, false); }
  double scalar_node(int id) { return m->g.is_zero(id) ? 0.0 : get(m->g.data(id)); }

  // dst += coef * packed bra-type gradient (y1, y2); a Zero part adds nothing
  void add_grad(int y1, int y2, double coef, double* dst) {
    Graph& g = m->g;
    if (g.is_zero(y1) && g.is_zero(y2)) return;
    const double* p1 = g.is_zero(y1) ? zero1 : g.data(y1);
    const double* p2 = g.is_zero(y2) ? zero2 : g.data(y2);
    c->be->pack(p1, p2, c->o, c->v, tmp, true);
    launch_axpby(st(), dim, coef, tmp, 1.0, dst);
  }

  // gradient of <(l0, Lbra)|Hbar|(r0, Rket)> with respect to the state
  void run_T(double l0, const double* Lbra, double r0v, const double* Rket) {
    Graph& g = m->g;
    LagSec& S = lag_section(*m);
    load_packed(c, g, Lbra, m->Lb1, m->Lb2, true);
    load_packed(c, g, Rket, m->R1, m->R2, false);
    set_scalar(c, g, m->s_l0r0, l0 * r0v);
    set_scalar(c, g, m->s_l0, l0);
    set_scalar(c, g, m->s_r0, r0v);
    std::vector<int> tg;
    for (int x : {S.gt1, S.gt2, S.gz, S.gRa1, S.gRa2, S.gRb1, S.gRb2, S.gR1, S.gR2})
      if (!g.is_zero(x)) tg.push_back(x);
    g.run(tg);
  }

  void load_state() {
    E0 = eval_residual(c, vec[0], zeta, vec[1], vec[2], tmp);
    m = c->cur;
    OverlapSec& O = overlap_section(*m);
    set_scalar(c, m->g, O.ra0, r0[0]);
    set_scalar(c, m->g, O.rb0, r0[1]);
    load_packed(c, m->g, vec[1], O.ra1, O.ra2, false);
    load_packed(c, m->g, vec[2], O.rb1, O.rb2, false);
  }

  // the full (affine) stationarity residual at u
  void residual(const double* u, double* out) {
    Graph& g = m->g;
    const double* zb = u;
    const double* Lbk[2] = {u + dim, u + 2 * dim};
    const double gbar = get(u + 3 * dim);
    double* rt = out;
    double* rR[2] = {out + dim, out + 2 * dim};
    c->be->fill(out, 3 * dim, 0.0);
    double rz = 0.0;
    double lb0[2], lr[2];
    for (int k = 0; k < 2; ++k) {
      lb0[k] = gbar * dO[k] / omega[k];
      lr[k] = dot(Lbk[k], vec[1 + k], dim);
      const double ck = lb0[k] * r0[k] + lr[k];
      const double dk = (kind == 0 && k == ns) ? 1.0 : 0.0;
      c->be->upload(Kb[k], Lbk[k], dim, true);
      launch_axpby(st(), dim, dk - ck, vec[3 + k], 1.0, Kb[k]);
    }
    LagSec& S = lag_section(*m);
    for (int k = 0; k < 2; ++k) {
      run_T(lb0[k], Kb[k], r0[k], vec[1 + k]);
      add_grad(S.gt1, S.gt2, 1.0, rt);
      add_grad(S.gRa1, S.gRa2, 1.0, rR[0]);
      add_grad(S.gRb1, S.gRb2, 1.0, rR[1]);
      add_grad(S.gR1, S.gR2, 1.0, rR[k]);
      rz += scalar_node(S.gz);
      launch_axpby(st(), dim, -omega[k], Kb[k], 1.0, rR[k]);
    }
    run_T(0.0, zb, 1.0, zero);
    add_grad(S.gt1, S.gt2, 1.0, rt);
    add_grad(S.gRa1, S.gRa2, 1.0, rR[0]);
    add_grad(S.gRb1, S.gRb2, 1.0, rR[1]);
    rz += scalar_node(S.gz);
    OvlGradSec& Og = overlap_grad_section(*m);
    set_scalar(c, g, Og.gbar, gbar);
    std::vector<int> tg;
    for (int x : {Og.dt1, Og.dt2, Og.da1, Og.da2, Og.db1, Og.db2})
      if (!g.is_zero(x)) tg.push_back(x);
    g.run(tg);
    add_grad(Og.dt1, Og.dt2, 1.0, rt);
    add_grad(Og.da1, Og.da2, 1.0, rR[0]);
    add_grad(Og.db1, Og.db2, 1.0, rR[1]);
    if (kind == 1) {
      launch_axpby(st(), dim, 1.0, Ot, 1.0, rt);
      launch_axpby(st(), dim, 1.0, vec[3 + ms], 1.0, rR[ns]);
    }
    if (gauge_fix)
      for (int k = 0; k < 2; ++k) launch_axpby(st(), dim, lr[k], vec[3 + k], 1.0, rR[k]);
    put(out + 3 * dim, rz);
  }

  void precompute() {
    Graph& g = m->g;
    OvlGradSec& Og = overlap_grad_section(*m);
    set_scalar(c, g, Og.gbar, 1.0);
    std::vector<int> tg;
    for (int x : {Og.da0, Og.db0})
      if (!g.is_zero(x)) tg.push_back(x);
    if (!tg.empty()) g.run(tg);
    dO[0] = scalar_node(Og.da0);
    dO[1] = scalar_node(Og.db0);
    if (kind == 1) {
      // dO_mn/dt = r0_n L_m + <L_m| tau R1_n>, the seeds of a transition element
      load_packed(c, g, vec[3 + ms], m->Lb1, m->Lb2, true);
      load_packed(c, g, vec[1 + ns], m->R1, m->R2, false);
      set_scalar(c, g, m->s_l0r0, 0.0);
      set_scalar(c, g, m->s_l0, 0.0);
      set_scalar(c, g, m->s_r0, r0[ns]);
      g.run({m->oB1, m->oB2});
      c->be->fill(Ot, dim, 0.0);
      add_grad(m->oB1, m->oB2, 1.0, Ot);
    }
    // diagonal preconditioner: dressed denominators D' (zbar), D' - omega_k (Lb_k)
    const int o = c->o, v = c->v;
    g.run({m->er.Fooi, m->er.Fvvi});
    double* fdiag = solver_buf(c, 40, o + v);
    double* Dp = solver_buf(c, 41, dim);
    int64_t d1[1] = {o}, os1[1] = {1}, is1[1] = {o + 1};
    c->be->copy_view(1, d1, fdiag, os1, g.data(m->er.Fooi), is1, 1.0, false);
    int64_t d2[1] = {v}, os2[1] = {1}, is2[1] = {v + 1};
    c->be->copy_view(1, d2, fdiag + o, os2, g.data(m->er.Fvvi), is2, 1.0, false);
    launch_denoms(st(), o, v, fdiag, Dp);
    // Pd = 1 / (D' - lam): precond gives 1 / (lam - D'), hence the sign
    c->be->fill(tmp, dim, 1.0);
    launch_precond(st(), dim, tmp, Dp, 0.0, Pd);
    launch_precond(st(), dim, tmp, Dp, omega[0], Pd + dim);
    launch_precond(st(), dim, tmp, Dp, omega[1], Pd + 2 * dim);
    launch_axpby(st(), 3 * dim, 0.0, Pd, -1.0, Pd);
    put(Pd + 3 * dim, 1.0);
  }
};

}  // namespace

namespace {

// Right-preconditioned restarted GMRES for lin(x) = rhs with
// lin(x) = S.residual(x) - B (the affine residual minus its constant), x
// accumulated in place. Krylov vectors live on the device; the small
// Hessenberg least-squares problem (Givens rotations) is solved on the host.
// Returns the number of operator applications.
int gmres(MultSolver& S, const double* B, const double* rhs, double* x, double abs_tol,
          double rel_tol, int max_apply, double* est_out) {
  sccsd_ctx* c = S.c;
  const int64_t N = S.N;
  // Krylov dimension between restarts: long enough for the indefinite
  // (A - omega_k) blocks, bounded to about 32 GB of basis vectors
  const int mk = (int)std::max<int64_t>(
      20, std::min<int64_t>(120, (int64_t)(32e9 / 8.0) / std::max<int64_t>(1, N) - 1));
  double* V = solver_buf(c, 50, (int64_t)(mk + 1) * N);
  double* W = solver_buf(c, 51, N);
  double* Z = solver_buf(c, 52, N);
  double* y_dev = c->sv_small + 5 * kMaxSpace * kMaxSpace;
  cudaStream_t st = S.st();
  auto combine = [&](int k, const double* coef_dev, double* out) {
    MatView A;  // element (0, p) = coef[p]
    A.p = coef_dev;
    A.sr2 = 1;
    A.sk2 = 1;
    MatView Bv;  // element (n, p) = V[p * N + n]
    Bv.p = V;
    Bv.sr2 = 1;
    Bv.sk2 = N;
    c->be->gemm_view(1, 1, N, k, 1.0, A, Bv, out, false);
  };
  auto lin = [&](const double* in, double* out) {
    S.residual(in, out);
    launch_axpby(st, N, -1.0, B, 1.0, out);
  };
  int applied = 0;
  double beta0 = -1.0, est = 0.0;
  while (applied < max_apply) {
    // R = rhs - lin(x)  (in V[0])
    lin(x, V);
    ++applied;
    launch_axpby(st, N, 1.0, rhs, -1.0, V);
    const double beta = std::sqrt(std::max(0.0, S.dot(V, V, N)));
    if (beta0 < 0) beta0 = beta;
    est = beta;
    if (beta <= std::max(abs_tol, rel_tol * beta0) || beta == 0.0) break;
    launch_axpby(st, N, 0.0, V, 1.0 / beta, V);
    std::vector<double> H((mk + 1) * mk, 0.0), cs(mk), sn(mk), g(mk + 1, 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < mk && applied < max_apply; ++j) {
      double* vj = V + (int64_t)j * N;
      double* vn = V + (int64_t)(j + 1) * N;
      launch_scale(st, N, S.Pd, vj, Z);
      lin(Z, W);
      ++applied;
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        double* cf = c->sv_small + 4 * kMaxSpace * kMaxSpace + 8;
        c->be->gemm_tn(1, j + 1, 1, N, 1.0, V, W, cf, false);
        std::vector<double> h(j + 1);
        c->be->download(h.data(), cf, j + 1, false);
        for (int i = 0; i <= j; ++i) H[i * mk + j] += h[i];
        combine(j + 1, cf, Z);
        launch_axpby(st, N, -1.0, Z, 1.0, W);
      }
      const double hn = std::sqrt(std::max(0.0, S.dot(W, W, N)));
      H[(j + 1) * mk + j] = hn;
      if (hn > 0.0) {
        c->be->upload(vn, W, N, true);
        launch_axpby(st, N, 0.0, vn, 1.0 / hn, vn);
      }
      for (int i = 0; i < j; ++i) {  // previous rotations
        const double a = H[i * mk + j], b = H[(i + 1) * mk + j];
        H[i * mk + j] = cs[i] * a + sn[i] * b;
        H[(i + 1) * mk + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[j * mk + j], b = H[(j + 1) * mk + j];
      const double r = std::hypot(a, b);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? b / r : 0.0;
      H[j * mk + j] = r;
      H[(j + 1) * mk + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      est = std::fabs(g[j + 1]);
      if (getenv("SCCSD_LOG") && (j + 1) % 10 == 0)
        fprintf(stderr, "  gmres: step %d estimate %.3e\n", j + 1, est);
      if (est <= std::max(abs_tol, rel_tol * beta0) || hn == 0.0) {
        ++j;
        break;
      }
    }
    // y = H^-1 g (upper triangular), x += Pd (V y)
    std::vector<double> yv(j, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[i * mk + k] * yv[k];
      yv[i] = H[i * mk + i] != 0.0 ? s / H[i * mk + i] : 0.0;
    }
    if (j > 0) {
      c->be->upload(y_dev, yv.data(), j, false);
      combine(j, y_dev, Z);
      launch_scale(st, N, S.Pd, Z, W);
      launch_axpby(st, N, 1.0, W, 1.0, x);
    }
    if (getenv("SCCSD_LOG"))
      fprintf(stderr, "  gmres: restart after %d applications, estimate %.3e\n", applied, est);
    if (est <= std::max(abs_tol, rel_tol * beta0)) break;
  }
  if (est_out) *est_out = est;
  return applied;
}

}  // namespace

namespace {

void mult_setup(sccsd_ctx* c, MultSolver& S, const double* vecs, const double* scal, int kind,
                int m_state, int n_state) {
    ensure_small(c);
    const int64_t dim = c->dim, N = 3 * dim + 1;
    const int64_t ov = (int64_t)c->o * c->v;
    S.c = c;
    S.kind = kind;
    S.ms = m_state;
    S.ns = n_state;
    S.dim = dim;
    S.N = N;
    double sc[5];
    if (c->be->is_device(scal))
      c->be->download(sc, scal, 5, false);
    else
      std::memcpy(sc, scal, sizeof sc);
    for (double x : sc)
      if (!std::isfinite(x)) throw std::invalid_argument("non-finite scalar input");
    if (sc[3] == 0.0 || sc[4] == 0.0) throw std::invalid_argument("zero excitation energy");
    S.zeta = sc[0];
    S.r0[0] = sc[1];
    S.r0[1] = sc[2];
    S.omega[0] = sc[3];
    S.omega[1] = sc[4];
    for (int k = 0; k < 5; ++k) {
      double* d = solver_buf(c, 30 + k, dim);
      c->be->upload(d, vecs + (int64_t)k * dim, dim, c->be->is_device(vecs));
      S.vec[k] = d;
    }
    S.tmp = solver_buf(c, 35, dim);
    S.zero = solver_buf(c, 36, dim);
    S.zero1 = solver_buf(c, 37, ov);
    S.zero2 = solver_buf(c, 38, ov * ov);
    c->be->fill(S.zero, dim, 0.0);
    c->be->fill(S.zero1, ov, 0.0);
    c->be->fill(S.zero2, ov * ov, 0.0);
    S.Kb[0] = solver_buf(c, 46, dim);
    S.Kb[1] = solver_buf(c, 47, dim);
    S.Bc = solver_buf(c, 48, N);
    S.Ot = solver_buf(c, 49, dim);
    S.Pd = solver_buf(c, 53, N);
}

}  // namespace

extern "C" {

int sccsd_solve_multipliers(sccsd_ctx* c, const double* vecs, const double* scal, int kind,
                            int m_state, int n_state, double tol, int maxit, double refine_tol,
                            double* zbar, double* K, double* out_scal, double* D1, double* Gamma,
                            int* iterations) {
  if (!c) return SCCSD_EINVAL;
  if (!vecs || !scal || !(tol > 0.0) || maxit < 1)
    return fail(c, SCCSD_EINVAL, "bad arguments");
  if (kind == 0 ? (n_state != 0 && n_state != 1)
                : (kind != 1 || m_state < 0 || m_state > 1 || n_state < 0 || n_state > 1 ||
                   m_state == n_state))
    return fail(c, SCCSD_EINVAL, "bad target");
  int status = SCCSD_OK;
  int rc = guarded(c, [&] {
    MultSolver S{};
    mult_setup(c, S, vecs, scal, kind, m_state, n_state);
    S.gauge_fix = true;
    const int64_t dim = c->dim, N = 3 * dim + 1;
    double* X = solver_buf(c, 54, N);
    double* DX = solver_buf(c, 55, N);
    double* RHS = solver_buf(c, 56, N);
    cudaStream_t st = (cudaStream_t)c->be->stream();

    const int p0 = c->be->get_precision();
    const bool refine = p0 != SCCSD_FP64 && refine_tol > 0.0;
    if (refine) switch_precision(c, SCCSD_FP64);
    S.load_state();
    S.precompute();
    c->be->fill(X, N, 0.0);
    int applied = 0;
    bool converged = false;
    const int max_outer = 12;
    for (int outer = 0; outer <= max_outer && applied < maxit; ++outer) {
      if (refine) {
        switch_precision(c, SCCSD_FP64);
        S.load_state();
      }
      S.residual(X, RHS);  // true residual (FP64 when refining)
      ++applied;
      const double rn = std::sqrt(S.dot(RHS, RHS, N));
      if (getenv("SCCSD_LOG"))
        fprintf(stderr, "multipliers: outer %d residual %.3e (%d applications)\n", outer, rn,
                applied);
      if (rn <= tol) {
        converged = true;
        break;
      }
      if (outer == max_outer) break;
      if (refine) {
        switch_precision(c, p0);
        S.load_state();
      }
      // B = residual(0) in the current precision; correction solve lin(DX) = -r
      c->be->fill(DX, N, 0.0);
      S.residual(DX, S.Bc);
      ++applied;
      launch_axpby(st, N, 0.0, RHS, -1.0, RHS);
      double est = 0.0;
      applied += gmres(S, S.Bc, RHS, DX, refine ? 0.0 : tol, refine ? 1e-3 : 0.0,
                       maxit - applied, &est);
      launch_axpby(st, N, 1.0, DX, 1.0, X);
    }
    if (refine) {
      switch_precision(c, SCCSD_FP64);
      S.load_state();
    }
    // outputs: zbar, the gauge-free bras K_k, and the scalars
    const double gbar = S.get(X + 3 * dim);
    double lb0[2], cst[2], Ebar[2];
    for (int k = 0; k < 2; ++k) {
      lb0[k] = gbar * S.dO[k] / S.omega[k];
      cst[k] = lb0[k] * S.r0[k] + S.dot(X + (1 + k) * dim, S.vec[1 + k], dim);
      const double dk = (kind == 0 && k == n_state) ? 1.0 : 0.0;
      c->be->upload(S.Kb[k], X + (1 + k) * dim, dim, true);
      launch_axpby(st, dim, dk - cst[k], S.vec[3 + k], 1.0, S.Kb[k]);
      // reported in the gauge Lbar_k . R_k = 0, where <Lbar_k|R_k> = lb0_k r0_k
      Ebar[k] = (S.E0 + S.omega[k]) * (dk - lb0[k] * S.r0[k]);
    }
    if (zbar) c->be->download(zbar, X, dim, c->be->is_device(zbar));
    if (K) {
      c->be->download(K, S.Kb[0], dim, c->be->is_device(K));
      c->be->download(K + dim, S.Kb[1], dim, c->be->is_device(K));
    }
    if (out_scal) {
      double o5[5] = {gbar, lb0[0], lb0[1], Ebar[0], Ebar[1]};
      if (c->be->is_device(out_scal))
        c->be->upload(out_scal, o5, 5, false);
      else
        std::memcpy(out_scal, o5, sizeof o5);
    }
    // densities of the Lagrangian: sum_k d(K_k; R_k) + d((0, zbar); (1, 0))
    if (D1) {
      Model& mm = *S.m;
      Graph& g = mm.g;
      const int64_t n = c->n, nJ = (int64_t)c->J * n * n;
      double* Dacc = solver_buf(c, 57, n * n);
      double* Gacc = Gamma ? solver_buf(c, 58, nJ) : nullptr;
      c->be->fill(Dacc, n * n, 0.0);
      if (Gacc) c->be->fill(Gacc, nJ, 0.0);
      struct Pair {
        double l0;
        const double* bra;
        double r0;
        const double* ket;
      };
      Pair pairs[3] = {{lb0[0], S.Kb[0], S.r0[0], S.vec[1]},
                       {lb0[1], S.Kb[1], S.r0[1], S.vec[2]},
                       {0.0, X, 1.0, S.zero}};
      for (const Pair& p : pairs) {
        load_packed(c, g, p.bra, mm.Lb1, mm.Lb2, true);
        load_packed(c, g, p.ket, mm.R1, mm.R2, false);
        set_scalar(c, g, mm.s_l0r0, p.l0 * p.r0);
        set_scalar(c, g, mm.s_l0, p.l0);
        set_scalar(c, g, mm.s_r0, p.r0);
        std::vector<int> tg;
        if (!g.is_zero(mm.D1)) tg.push_back(mm.D1);
        if (Gacc && !g.is_zero(mm.Gam)) tg.push_back(mm.Gam);
        if (!tg.empty()) g.run(tg);
        if (!g.is_zero(mm.D1)) launch_axpby(st, n * n, 1.0, g.data(mm.D1), 1.0, Dacc);
        if (Gacc && !g.is_zero(mm.Gam)) launch_axpby(st, nJ, 1.0, g.data(mm.Gam), 1.0, Gacc);
      }
      c->be->download(D1, Dacc, n * n, c->be->is_device(D1));
      if (Gamma) c->be->download(Gamma, Gacc, nJ, c->be->is_device(Gamma));
    }
    if (refine) switch_precision(c, p0);
    if (iterations) *iterations = applied;
    c->be->sync();
    if (!converged) status = SCCSD_ENOTCONV;
  });
  if (rc != SCCSD_OK) return rc;
  if (status != SCCSD_OK) return fail(c, status, "multiplier equations did not converge");
  return SCCSD_OK;
}

int sccsd_multiplier_residual(sccsd_ctx* c, const double* vecs, const double* scal, int kind,
                              int m_state, int n_state, const double* u, double* r) {
  if (!c) return SCCSD_EINVAL;
  if (!vecs || !scal || !u || !r) return fail(c, SCCSD_EINVAL, "NULL argument");
  if (kind == 0 ? (n_state != 0 && n_state != 1)
                : (kind != 1 || m_state < 0 || m_state > 1 || n_state < 0 || n_state > 1 ||
                   m_state == n_state))
    return fail(c, SCCSD_EINVAL, "bad target");
  return guarded(c, [&] {
    MultSolver S{};
    mult_setup(c, S, vecs, scal, kind, m_state, n_state);
    const int64_t N = 3 * c->dim + 1;
    double* U = solver_buf(c, 54, N);
    double* RR = solver_buf(c, 56, N);
    c->be->upload(U, u, N, c->be->is_device(u));
    S.load_state();
    S.precompute();
    S.residual(U, RR);
    c->be->download(r, RR, N, c->be->is_device(r));
    c->be->sync();
  });
}

int sccsd_state_amplitudes(sccsd_ctx* c, double* t) {
  if (!c) return SCCSD_EINVAL;
  if (!t) return fail(c, SCCSD_EINVAL, "t is NULL");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "no state yet");
  return guarded(c, [&] {
    Model& m = *c->cur;
    store_packed(c, m.g, m.t1, m.t2, t, false);
    c->be->sync();
  });
}

}  // extern "C"
