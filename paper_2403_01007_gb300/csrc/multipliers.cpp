// C ABI of the Lagrangian multipliers of SCCSD gradients and couplings.
#include "context.h"

using namespace sccsd;

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
  int proj = 0;              // 0 natural, 1 state projection of O_ab
  double wK[7] = {0.0};      // dO_ab/ds for the state projection's scalars
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
    if (proj == 1) {
      OvlKGradSec& Og = overlap_k_grad_section(*m);
      for (int i = 0; i < 7; ++i) set_scalar(c, g, Og.w[i], gbar * wK[i]);
      std::vector<int> tg;
      for (int x : {Og.dt1, Og.dt2, Og.da1, Og.da2, Og.db1, Og.db2})
        if (!g.is_zero(x)) tg.push_back(x);
      g.run(tg);
      add_grad(Og.dt1, Og.dt2, 1.0, rt);
      add_grad(Og.da1, Og.da2, 1.0, rR[0]);
      add_grad(Og.db1, Og.db2, 1.0, rR[1]);
    } else {
      OvlGradSec& Og = overlap_grad_section(*m);
      set_scalar(c, g, Og.gbar, gbar);
      std::vector<int> tg;
      for (int x : {Og.dt1, Og.dt2, Og.da1, Og.da2, Og.db1, Og.db2})
        if (!g.is_zero(x)) tg.push_back(x);
      g.run(tg);
      add_grad(Og.dt1, Og.dt2, 1.0, rt);
      add_grad(Og.da1, Og.da2, 1.0, rR[0]);
      add_grad(Og.db1, Og.db2, 1.0, rR[1]);
    }
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
    if (proj == 1) {
      // the state projection's scalars at the state fix the weights dO/ds
      OverlapKSec& K = overlap_k_section(*m);
      const int ids[7] = {K.maa, K.mab, K.nab, K.nbb, K.Saa, K.Sab, K.Sbb};
      g.run(std::vector<int>(ids, ids + 7));
      double sv[7];
      for (int i = 0; i < 7; ++i) sv[i] = scalar_node(ids[i]);
      overlap_k_value(sv, wK);
      OvlKGradSec& Og = overlap_k_grad_section(*m);
      for (int i = 0; i < 7; ++i) set_scalar(c, g, Og.w[i], wK[i]);
      std::vector<int> tg;
      for (int x : {Og.da0, Og.db0})
        if (!g.is_zero(x)) tg.push_back(x);
      if (!tg.empty()) g.run(tg);
      dO[0] = scalar_node(Og.da0);
      dO[1] = scalar_node(Og.db0);
    } else {
      OvlGradSec& Og = overlap_grad_section(*m);
      set_scalar(c, g, Og.gbar, 1.0);
      std::vector<int> tg;
      for (int x : {Og.da0, Og.db0})
        if (!g.is_zero(x)) tg.push_back(x);
      if (!tg.empty()) g.run(tg);
      dO[0] = scalar_node(Og.da0);
      dO[1] = scalar_node(Og.db0);
    }
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
    S.proj = c->projection;
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
    // correction solves run in the context's precision while they pay: two
    // rounds in a row that cut the FP64 residual by less than a factor 10 mean
    // the mixed operator is too far from the FP64 one for this system, and the
    // remaining corrections are solved in FP64
    bool mixed = refine;
    int slow = 0;
    double prev = 0.0;
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
      if (mixed && outer > 0) {
        slow = rn > 0.1 * prev ? slow + 1 : 0;
        if (slow >= 2) {
          mixed = false;
          if (getenv("SCCSD_LOG"))
            fprintf(stderr, "multipliers: mixed corrections stalled, finishing in FP64\n");
        }
      }
      prev = rn;
      if (mixed) {
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

}  // extern "C"
