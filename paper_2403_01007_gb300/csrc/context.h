// Internal declarations shared by the translation units of the C ABI (not
// part of the installed interface): the per-context graph model and its
// sections, the context itself, marshalling helpers and solver helpers.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
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

// sigma = A R and A^T L for a batch of nb vectors (graph node ids)
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
  int ca1, ca2, cb1, cb2;           // HF+S+D parts of exp(T)|R_a>, exp(T)|R_b>
  size_t op_begin = 0, op_end = 0;  // the section's ops
};

// The scalars of O_ab with the state projection over K = {a, b}:
// m_k = <psi_a|R_k>, n_l = <R_l|psi_b>, S_kl = <R_k|R_l> (same inputs as
// OverlapSec); O_ab = m^T S^-1 n is formed on the host.
struct OverlapKSec {
  int maa, mab, nab, nbb, Saa, Sab, Sbb;
  size_t op_begin = 0, op_end = 0;
};

// Gradient of sum_i w_i s_i over the seven scalars s of OverlapKSec, with
// respect to t and both states; with w_i = gbar dO_ab/ds_i (formed on the host
// at the state) it is the gradient of gbar O_ab of the state projection.
struct OvlKGradSec {
  int w[7];
  int dt1, dt2, da0, da1, da2, db0, db1, db2;
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

// One graph holding the residual, both Jacobian transformations and the
// densities, with or without the SCC X3 terms, plus its lazily built sections.
struct Model {
  Graph g;
  bool scc = false;
  std::unique_ptr<OverlapSec> ovl;
  std::unique_ptr<OverlapKSec> ovk;
  std::unique_ptr<OvlKGradSec> ovkg;
  Graph::Ranges fwd;
  std::vector<int> vol_inputs;
  std::map<int64_t, RightSec> right;  // batched right transformations by batch size
  std::map<int64_t, LeftSec> left;
  int t1, t2, L, h, delta;
  int R1, R2, Lb1, Lb2;
  int zeta = -1, Ra1 = -1, Ra2 = -1, Rb1 = -1, Rb2 = -1, t2zero = -1;
  // several constrained states: one (R1^k, Y2^k) input pair per state
  int nslots = 0;
  std::vector<int> X1s, Y2s;
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

// scc: the two-state X3 terms (zeta, Ra, Rb); nslots > 0 (with scc false):
// the X3 terms of nslots constrained states
std::unique_ptr<Model> build_model(Backend* be, int o, int v, int J, bool scc, int nslots = 0);
// lazily built graph sections (model.cpp)
OverlapSec& overlap_section(Model& M);
OverlapKSec& overlap_k_section(Model& M);
OvlKGradSec& overlap_k_grad_section(Model& M);

// O_ab = m^T S^-1 n of the state projection from its scalars
// s = (m_a, m_b, n_a, n_b, S_aa, S_ab, S_bb) (the 2 x 2 inverse written out),
// and its partial derivatives dO/ds_i; throws if S is singular.
inline double overlap_k_value(const double* s, double* w = nullptr) {
  const double maa = s[0], mab = s[1], nab = s[2], nbb = s[3];
  const double Saa = s[4], Sab = s[5], Sbb = s[6];
  const double det = Saa * Sbb - Sab * Sab;
  if (!(std::fabs(det) > 1e-14 * std::max(1.0, Saa * Sbb)))
    throw std::invalid_argument("R_a and R_b are linearly dependent");
  const double N = maa * (Sbb * nab - Sab * nbb) + mab * (Saa * nbb - Sab * nab);
  if (w) {
    w[0] = (Sbb * nab - Sab * nbb) / det;
    w[1] = (Saa * nbb - Sab * nab) / det;
    w[2] = (maa * Sbb - mab * Sab) / det;
    w[3] = (mab * Saa - maa * Sab) / det;
    w[4] = mab * nbb / det - N * Sbb / (det * det);
    w[5] = -(maa * nbb + mab * nab) / det + 2.0 * N * Sab / (det * det);
    w[6] = maa * nab / det - N * Saa / (det * det);
  }
  return N / det;
}
RightSec& right_section(Model& M, int64_t nb);
LeftSec& left_section(Model& M, int64_t nb);
LagSec& lag_section(Model& M);
OvlGradSec& overlap_grad_section(Model& M);

}  // namespace sccsd

struct sccsd_ctx {
  int o = 0, v = 0, J = 0, n = 0, precision = 0;
  int64_t dim = 0;
  std::unique_ptr<sccsd::Backend> be;
  std::unique_ptr<sccsd::Model> plain, scc;
  std::unique_ptr<sccsd::Model> multi;  // several constrained states (built for multi_n states)
  int multi_n = 0;
  bool multi_set = false;  // the packed (R1^k, Y2^k) of the multi-state X3 terms are loaded
  sccsd::Model* cur = nullptr;
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
  int projection = 0;  // SCC overlap: 0 natural, 1 state projection (Sec. 2.4.1)
  std::vector<double*> sv;    // solver work buffers
  std::vector<int64_t> sv_n;  // their sizes (doubles)
  double* sv_small = nullptr; // small matrices and vectors
  int* sv_info = nullptr;
  std::string err;
  ~sccsd_ctx() {
    if (getenv("SCCSD_TRACE")) {
      for (sccsd::Model* m : {plain.get(), scc.get(), multi.get()})
        if (m) fprintf(stderr, "%s", m->g.trace_report(std::max(60, atoi(getenv("SCCSD_TRACE")))).c_str());
    }
    plain.reset();
    scc.reset();
    multi.reset();
    if (be) {
      for (double* p : {L, h, delta, stage, stage2, eps_dev, D, Dprec, sv_small})
        if (p) be->release(p);
      for (double* p : sv)
        if (p) be->release(p);
      if (sv_info) be->release((double*)sv_info);
    }
  }
};

namespace sccsd {

inline int fail(sccsd_ctx* c, int code, const std::string& msg) {
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

// marshalling between packed vectors (host or device) and graph tensors (api.cpp)
Model& model(sccsd_ctx* c, bool scc);
// the model of n constrained states (rebuilt when n changes)
Model& model_states(sccsd_ctx* c, int n);
double* input_buffer(Graph& g, int id);
void load_packed(sccsd_ctx* c, Graph& g, const double* src, int x1, int x2, bool bra);
void load_packed_batch(sccsd_ctx* c, Graph& g, const double* src, int64_t nb, int x1, int x2,
                       bool bra);
void store_packed_batch(sccsd_ctx* c, Graph& g, int64_t nb, int y1, int y2, double* dst, bool bra);
void store_packed(sccsd_ctx* c, Graph& g, int y1, int y2, double* dst, bool bra);
void set_scalar(sccsd_ctx* c, Graph& g, int id, double v);
double get_scalar(sccsd_ctx* c, Graph& g, int id);

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

// solver helpers (solvers.cpp)
double* solver_buf(sccsd_ctx* c, size_t i, int64_t n);
void ensure_small(sccsd_ctx* c);
void switch_precision(sccsd_ctx* c, int p);
// E0 and packed omega at t; with multi the X3 terms of the states set by
// set_states, else those of (zeta, Ra, Rb) when Ra is given
double eval_residual(sccsd_ctx* c, const double* t, double zeta, const double* Ra,
                     const double* Rb, double* om, bool multi = false);
// the X3 terms of n states R[n][dim] (host or device) with zeta_kl, k < l, in
// the order (0,1), (0,2), ..., (1,2), ...: packed P_k = (R1^k, sum_l Z_kl R2^l)
void set_states(sccsd_ctx* c, int n, const double* zeta, const double* R);
int solve_ground_impl(sccsd_ctx* c, const double* t0, double zeta, const double* Ra,
                      const double* Rb, bool multi, double tol, int maxit, double refine_tol,
                      double* t_out, double* e_corr, int* iterations);
void transform(sccsd_ctx* c, int side, int nvec, const double* V, double* W);

}  // namespace sccsd
