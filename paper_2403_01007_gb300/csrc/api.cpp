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

struct Model {
  Graph g;
  bool scc = false;
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
  M->vol_inputs = {M->R1, M->R2, M->Lb1, M->Lb2, M->s_l0r0, M->s_l0, M->s_r0};
  g.set_volatile_inputs(M->vol_inputs);
  return M;
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
  std::string err;
  ~sccsd_ctx() {
    if (getenv("SCCSD_TRACE")) {
      for (Model* m : {plain.get(), scc.get()})
        if (m) fprintf(stderr, "%s", m->g.trace_report(60).c_str());
    }
    plain.reset();
    scc.reset();
    if (be) {
      for (double* p : {L, h, delta, stage, stage2})
        if (p) be->release(p);
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
