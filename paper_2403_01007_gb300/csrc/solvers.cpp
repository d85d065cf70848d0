// Solvers: ground state (Jacobi + DIIS with dressed denominators), EOM roots
// (Davidson) and the self-consistent SCC constraint, driven from the host
// with every vector on the device.
#include "context.h"

using namespace sccsd;

namespace sccsd {

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
  for (Model* m : {c->plain.get(), c->scc.get(), c->multi.get()})
    if (m) m->g.invalidate();
}

void set_states(sccsd_ctx* c, int n, const double* zeta, const double* R) {
  if (n < 2) throw std::invalid_argument("at least two constrained states");
  if (!zeta || !R) throw std::invalid_argument("zeta or R is NULL");
  const int np = n * (n - 1) / 2;
  for (int p = 0; p < np; ++p)
    if (!std::isfinite(zeta[p])) throw std::invalid_argument("zeta is not finite");
  const int64_t dim = c->dim, ov = (int64_t)c->o * c->v;
  Dev d{c};
  Model& m = model_states(c, n);
  double* Rd = solver_buf(c, 90, n * dim);
  c->be->upload(Rd, R, n * dim, c->be->is_device(R));
  // coef[l][k] = Z_kl with Z antisymmetric, Z_kl = zeta_kl for k < l
  std::vector<double> coef((size_t)n * n, 0.0);
  int p = 0;
  for (int k = 0; k < n; ++k)
    for (int l = k + 1; l < n; ++l, ++p) {
      coef[(size_t)l * n + k] = zeta[p];
      coef[(size_t)k * n + l] = -zeta[p];
    }
  double* cd = solver_buf(c, 91, (int64_t)n * n);
  c->be->upload(cd, coef.data(), (int64_t)n * n, false);
  // P_k = (R1^k, sum_l Z_kl R2^l): the doubles of the combination, the singles of R^k
  double* P = solver_buf(c, 92, n * dim);
  d.combine(n, n, cd, Rd, P);
  for (int k = 0; k < n; ++k) d.copy(P + k * dim, Rd + k * dim, ov);
  for (int k = 0; k < n; ++k) load_packed(c, m.g, P + k * dim, m.X1s[k], m.Y2s[k], false);
  c->multi_set = true;
}

// E0 and packed omega (device) at packed amplitudes t (device)
double eval_residual(sccsd_ctx* c, const double* t, double zeta, const double* Ra,
                     const double* Rb, double* om, bool multi) {
  if (multi) {
    if (!c->multi || !c->multi_set) throw std::logic_error("no constrained states set");
    Model& m = *c->multi;
    load_packed(c, m.g, t, m.t1, m.t2, false);
    c->cur = &m;
    m.g.run({m.er.E0, m.er.O1, m.er.O2});
    store_packed(c, m.g, m.er.O1, m.er.O2, om, false);
    return get_scalar(c, m.g, m.er.E0);
  }
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

}  // namespace sccsd

extern "C" {

int sccsd_solve_ground(sccsd_ctx* c, const double* t0, double zeta, const double* Ra,
                       const double* Rb, double tol, int maxit, double refine_tol, double* t_out,
                       double* e_corr, int* iterations) {
  if (!c) return SCCSD_EINVAL;
  if ((Ra == nullptr) != (Rb == nullptr)) return fail(c, SCCSD_EINVAL, "give both Ra and Rb or neither");
  return solve_ground_impl(c, t0, zeta, Ra, Rb, false, tol, maxit, refine_tol, t_out, e_corr,
                           iterations);
}

}  // extern "C"

int sccsd::solve_ground_impl(sccsd_ctx* c, const double* t0, double zeta, const double* Ra,
                             const double* Rb, bool multi, double tol, int maxit,
                             double refine_tol, double* t_out, double* e_corr, int* iterations) {
  if (!(tol > 0.0) || maxit < 1) return fail(c, SCCSD_EINVAL, "bad tolerance or iteration limit");
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
    int refine_fp64_evals = 0, inner_its = 0, refine_fail = 0;
    double gate = 1e300;
    int next_refresh = 3;
    for (it = 1; it <= maxit; ++it) {
      E = eval_residual(c, t, zeta, ra, rb, om, multi);
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
      // the mixed phase ends below refine_tol, or when it stalls at its noise
      // floor; after a refinement attempt that did not hold (strongly
      // correlated systems can stall far from the solution, where the
      // linearised correction overshoots) a stall counts only below 1% of
      // the residual of that attempt
      if (!fp64_phase && (nrm < refine_tol || (since_best >= 6 && nrm < gate))) {
        // Iterative refinement (defect correction): the FP64 residual
        // r = Omega(t) drives a correction solve A d = -r with the mixed
        // Jacobian (its error scales with d, not with t), t <- t + d. Each
        // round gains about the mixed arithmetic's relative accuracy, so a
        // few FP64 residuals replace the FP64 iteration tail. When a round
        // gains less than 3x, the remaining iterations run in FP64.
        const double* Dpre = have_dp ? Dp : (c->use_dprec ? c->Dprec : c->D);
        double* dl = solver_buf(c, 9, dim);
        double* Ad = solver_buf(c, 19, dim);
        double* rr = solver_buf(c, 20, dim);
        double* tp = solver_buf(c, 21, dim);   // amplitudes before the last correction
        // the correction solves start in the context's precision and move up
        // to the split BF16 form when a round gains too little
        int pc = p0;
        double inner_rtol = pc == SCCSD_BF16X3 ? 1e-4 : 1e-2;
        double prev = 1e300;
        bool done = false, worse = false;
        for (int round = 0; round < 12 && !done; ++round) {
          switch_precision(c, SCCSD_FP64);
          E = eval_residual(c, t, zeta, ra, rb, rr, multi);
          const double rn = std::sqrt(d.dot(rr, rr, dim));
          switch_precision(c, pc);
          ++refine_fp64_evals;
          if (getenv("SCCSD_LOG"))
            fprintf(stderr, "{\"solver\": \"ground_refine\", \"round\": %d, \"fp64_residual\": %.3e, \"e_corr\": %.12f}\n",
                    round, rn, E - c->e_hf);
          if (!std::isfinite(rn)) throw std::runtime_error("ground state diverged (non-finite residual)");
          nrm = rn;
          if (rn < tol) {
            done = true;
            break;
          }
          if (rn > prev) {
            // the last correction made things worse (too far from the
            // solution for the linearised step): undo it and let the mixed
            // iterations go on
            d.copy(t, tp, dim);
            worse = true;
            break;
          }
          if (rn > prev / 3.0) {
            if (pc == SCCSD_BF16) {
              // not gaining in BF16: the next corrections in the split form
              pc = SCCSD_BF16X3;
              inner_rtol = 1e-4;
              switch_precision(c, pc);
            } else {
              break;  // not gaining: finish in FP64
            }
          }
          prev = rn;
          // the mixed state at t for the Jacobian transforms
          eval_residual(c, t, zeta, ra, rb, om, multi);
          // A d = -r by the Jacobi-preconditioned linear iteration with DIIS
          c->be->fill(dl, dim, 0.0);
          int lh = 0, lhead = 0;
          const double goal = std::max(inner_rtol * rn, 0.3 * tol);
          for (int k = 0; k < 300; ++k) {
            transform(c, 0, 1, dl, Ad);
            d.axpby(dim, 1.0, rr, 1.0, Ad);      // rho = A d + r
            const double rho = std::sqrt(d.dot(Ad, Ad, dim));
            ++inner_its;
            if (!std::isfinite(rho)) throw std::runtime_error("correction solve diverged");
            if (rho < goal) break;
            launch_jacobi(d.st(), dim, dl, Ad, Dpre, tn);   // tn = d - rho / D
            const int sl = lhead;
            lhead = (lhead + 1) % kDiis;
            lh = std::min(lh + 1, kDiis);
            d.copy(X + (int64_t)sl * dim, tn, dim);
            d.copy(Rr + (int64_t)sl * dim, tn, dim);
            d.axpby(dim, -1.0, dl, 1.0, Rr + (int64_t)sl * dim);
            if (lh >= 2) {
              c->be->gemm_tn(1, lh, lh, dim, 1.0, Rr, Rr, Bm, false);
              launch_diis(d.st(), lh, Bm, cf, c->sv_info);
              int info = 0;
              cudaMemcpyAsync(&info, c->sv_info, sizeof(int), cudaMemcpyDeviceToHost, d.st());
              c->be->sync();
              if (info == 0)
                d.combine(1, lh, cf, X, dl);
              else
                d.copy(dl, tn, dim);
            } else {
              d.copy(dl, tn, dim);
            }
          }
          d.copy(tp, t, dim);
          d.axpby(dim, 1.0, dl, 1.0, t);
        }
        if (done) break;
        if (worse && ++refine_fail < 3) {
          // back to the mixed iterations from the best amplitudes, with a
          // lower gate for the next attempt
          switch_precision(c, p0);
          gate = std::min(gate, prev) * 1e-2;
          best = 1e300;
          since_best = 0;
          nh = 0;
          head = 0;
          continue;
        }
        // FP64 iterations from the current amplitudes
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
    if (getenv("SCCSD_LOG") && refine)
      fprintf(stderr, "{\"solver\": \"ground_done\", \"iterations\": %d, \"fp64_refine_residuals\": %d, \"correction_transforms\": %d, \"fp64_phase\": %d}\n",
              std::min(it, maxit), refine_fp64_evals, inner_its, (int)fp64_phase);
    if (refine) switch_precision(c, p0);
    if (refine) eval_residual(c, t, zeta, ra, rb, om, multi);  // fix the state for later transforms
    if (t_out) c->be->download(t_out, t, dim, c->be->is_device(t_out));
    if (e_corr) *e_corr = E - c->e_hf;
    if (iterations) *iterations = std::min(it, maxit);
    c->be->sync();
  });
  if (rc != SCCSD_OK) return rc;
  if (status != SCCSD_OK) return fail(c, status, "ground state not converged within maxit");
  return SCCSD_OK;
}

extern "C" {

int sccsd_normalize_left(sccsd_ctx* c, int nvec, const double* R, double* L) {
  if (!c) return SCCSD_EINVAL;
  if (nvec < 0) return fail(c, SCCSD_EINVAL, "nvec < 0");
  if (nvec == 0) return SCCSD_OK;
  if (!R || !L) return fail(c, SCCSD_EINVAL, "R or L is NULL");
  int status = SCCSD_OK;
  int k_bad = -1;
  int rc = guarded(c, [&] {
    Dev d{c};
    ensure_small(c);
    const int64_t dim = c->dim;
    const bool rdev = c->be->is_device(R), ldev = c->be->is_device(L);
    double* rb = solver_buf(c, 80, dim);
    double* lb = solver_buf(c, 81, dim);
    for (int k = 0; k < nvec && status == SCCSD_OK; ++k) {
      const double* rk = R + (int64_t)k * dim;
      double* lk = L + (int64_t)k * dim;
      const double* rd = rk;
      double* ld = lk;
      if (!rdev) {
        c->be->upload(rb, rk, dim, false);
        rd = rb;
      }
      if (!ldev) {
        c->be->upload(lb, lk, dim, false);
        ld = lb;
      }
      // <L_k|R_k> is the plain dot product in the biorthonormal bra basis
      const double s = d.dot(ld, rd, dim);
      if (!std::isfinite(s) || std::fabs(s) < 1e-300) {
        status = SCCSD_EINVAL;
        k_bad = k;
        break;
      }
      d.axpby(dim, 1.0 / s, ld, 0.0, ld);
      if (!ldev) c->be->download(lk, ld, dim, false);
    }
    c->be->sync();
  });
  if (rc != SCCSD_OK) return rc;
  if (status != SCCSD_OK)
    return fail(c, status, "L_k . R_k is zero or not finite for k = " + std::to_string(k_bad));
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
    // the subspace holds at most kMaxSpace vectors, and never more than dim
    const int mmax = (int)std::min<int64_t>(kMaxSpace, dim);
    if (2 * nroots + 2 > mmax) throw std::invalid_argument("problem too small for the requested roots");
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
    int anchors = 0;     // FP64 evaluations of the Ritz vectors' images
    int restarts = 0;    // of them, restarts of the subspace on FP64 images
    int pc = p0;         // precision of the expansion transforms
    int complex_run = 0; // consecutive iterations with a complex pair among the wanted roots
    std::vector<double> lam(nroots), res(nroots);
    double best = 1e300;
    int since_best = 0;
    double* AXf = solver_buf(c, 93, 12 * dim);
    double last_true = 1e300;   // FP64 residual at the previous check
    double target = std::max(tol, refine_tol);  // mixed residual that triggers the next check
    // Refinement in a mixed precision: the expansion vectors are transformed
    // in the mixed precision throughout; the FP64 images of the current Ritz
    // vectors decide convergence (their FP64 residuals must be below tol), and
    // when the mixed estimate of the residual proves too optimistic (the
    // subspace images carry more error than the residual is small), the
    // subspace restarts from the Ritz vectors with their FP64 images, after
    // which the mixed error scales with the size of the corrections, not of
    // the roots. Returns 1 when converged, 2 after a restart, 0 otherwise
    // (then res and Rz hold the FP64 residuals, which the expansion uses).
    auto anchor = [&](double mixed_worst) -> int {
      switch_precision(c, SCCSD_FP64);
      transform(c, side, nroots, Xr, AXf);
      switch_precision(c, pc);
      ++anchors;
      launch_ritz_residual(st, nroots, dim, AXf, Xr, wr, order, Rz);
      c->be->gemm_tn(1, nroots, nroots, dim, 1.0, Rz, Rz, G, false);
      c->be->gemm_tn(1, nroots, nroots, dim, 1.0, Xr, Xr, G + 144, false);
      std::vector<double> g1(nroots * nroots), g2(nroots * nroots);
      c->be->download(g1.data(), G, nroots * nroots, false);
      c->be->download(g2.data(), G + 144, nroots * nroots, false);
      double true_worst = 0.0;
      for (int k = 0; k < nroots; ++k) {
        res[k] = std::sqrt(g1[k * nroots + k] / g2[k * nroots + k]);
        true_worst = std::max(true_worst, res[k]);
      }
      if (getenv("SCCSD_LOG"))
        fprintf(stderr, "{\"solver\": \"davidson_anchor\", \"mixed_res\": %.3e, \"fp64_res\": %.3e}\n",
                mixed_worst, true_worst);
      if (true_worst < tol) return 1;
      best = std::min(best, true_worst);
      since_best = 0;
      // restart when the mixed estimate is off, or when the FP64 residual
      // gained less than 30 % since the previous check (a noise floor of the
      // mixed images)
      // (before the first restart every image in the subspace is a mixed one,
      // whose error does not shrink with the residual: always restart then)
      const bool restart = restarts == 0 || true_worst > 1.5 * mixed_worst ||
                           true_worst > 0.7 * last_true;
      // next check when the mixed estimate is below half the FP64 residual
      // this cycle is expected to reach (the last cycle's gain; 1e-3 before
      // one is known): deeper mixed iterations would only fit the noise
      const double gain = last_true < 1e300 ? std::min(1.0, true_worst / last_true) : 1e-3;
      target = std::max(tol, 0.5 * true_worst * std::max(gain, 1e-6));
      last_true = true_worst;
      if (restart) {
        // restart: V = orthonormalised Ritz vectors, W = their FP64 images
        have_prev = false;
        d.copy(V, Xr, (int64_t)nroots * dim);
        d.copy(W, AXf, (int64_t)nroots * dim);
        m = 0;
        for (int k = 0; k < nroots; ++k) {
          double* vk = V + (int64_t)m * dim;
          double* wk = W + (int64_t)m * dim;
          if (k != m) {
            d.copy(vk, V + (int64_t)k * dim, dim);
            d.copy(wk, W + (int64_t)k * dim, dim);
          }
          orthogonalize(vk, wk, m);
          double nn = std::sqrt(d.dot(vk, vk, dim));
          if (nn < 1e-10) continue;
          d.axpby(dim, 0.0, vk, 1.0 / nn, vk);
          d.axpby(dim, 0.0, wk, 1.0 / nn, wk);
          ++m;
        }
        ++restarts;
        // repeated restarts mean the expansions are too inexact: split BF16
        // after four, FP64 after sixteen
        if (restarts >= 16) pc = SCCSD_FP64;
        else if (restarts >= 4 && pc == SCCSD_BF16) pc = SCCSD_BF16X3;
        switch_precision(c, pc);
        best = 1e300;
        return 2;
      }
      return 0;
    };
    int it = 0;
    bool converged = false;
    for (it = 1; it <= maxit; ++it) {
      // subspace matrix and its lowest roots
      c->be->gemm_tn(1, m, m, dim, 1.0, V, W, S, false);
      launch_small_eig(st, m, S, wr, wi, Y, nroots, order, info_d, 1);
      int info = get_info();
      if (info != 0 && info != 4) throw std::runtime_error("subspace eigensolver failed");
      // A complex pair among the wanted Ritz values is followed through its
      // real invariant plane while the subspace grows; it is an error only
      // when it persists for 40 iterations or when the roots converge.
      complex_run = info == 4 ? complex_run + 1 : 0;
      if (complex_run >= 40) throw std::domain_error("complex pair among the lowest roots");
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
        fprintf(stderr, "{\"solver\": \"davidson\", \"iter\": %d, \"space\": %d, \"precision\": %d, \"max_res\": %.3e, \"omega\": [", it, m,
                pc, worst);
        for (int k = 0; k < nroots; ++k) fprintf(stderr, "%s%.12f", k ? ", " : "", lam[k]);
        fprintf(stderr, "]}\n");
      }
      if (worst < 0.9 * best) {
        best = worst;
        since_best = 0;
      } else {
        ++since_best;
      }
      if (worst < tol && complex_run > 0) throw std::domain_error("complex pair among the lowest roots");
      if (!refine && worst < tol) {
        converged = true;
        break;
      }
      // mixed estimate below the target (refine_tol at first, then from the
      // gain of the last cycle, never below tol), or a stall within 100x of
      // refine_tol: check on FP64 images (far from convergence a stall is a
      // slow Davidson, not the mixed precision's noise)
      if (refine && (worst < target || (since_best >= 20 && worst < 100.0 * refine_tol))) {
        const int a = anchor(worst);
        if (a == 1) {
          converged = true;
          break;
        }
        if (a == 2) continue;
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
    if (getenv("SCCSD_LOG") && refine)
      fprintf(stderr, "{\"solver\": \"davidson_done\", \"iterations\": %d, \"fp64_anchors\": %d, \"restarts\": %d}\n",
              std::min(it, maxit), anchors, restarts);
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

namespace {

// Runs in FP64 for its lifetime when the context computes in a mixed
// precision, and restores that precision on every exit.
struct Fp64Scope {
  sccsd_ctx* c;
  int p0;
  explicit Fp64Scope(sccsd_ctx* ctx) : c(ctx), p0(ctx->be->get_precision()) {
    if (p0 != SCCSD_FP64) switch_precision(c, SCCSD_FP64);
  }
  ~Fp64Scope() {
    if (p0 != SCCSD_FP64) switch_precision(c, p0);
  }
};

// eta.R_k for nb packed host kets at the fixed state (the eta part of the
// right-transformation section only)
void eta_dot(sccsd_ctx* c, int nb, const double* R, double* etaR) {
  Model& m = *c->cur;
  RightSec& S = right_section(m, nb);
  load_packed_batch(c, m.g, R, nb, S.R1, S.R2, false);
  m.g.run({S.etaR});
  if (m.g.is_zero(S.etaR))
    std::fill(etaR, etaR + nb, 0.0);
  else
    c->be->download(etaR, m.g.data(S.etaR), nb, false);
}

}  // namespace

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
    std::vector<double> t(dim), vecs(2 * dim), Ra(dim), Rb(dim);
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
      {
        // r0 = eta.R / omega and O_ab decide zeta: FP64 in a mixed context,
        // like the solves above, which finish in FP64
        Fp64Scope fp64(c);
        double etaR[2];
        eta_dot(c, 2, vecs.data(), etaR);
        r0[0] = etaR[0] / w[0];
        r0[1] = etaR[1] / w[1];
        check(c->projection == 1
                  ? sccsd_overlap_states(c, r0[0], vecs.data(), r0[1], vecs.data() + dim, &O)
                  : sccsd_overlap(c, r0[0], vecs.data(), r0[1], vecs.data() + dim, &O));
      }
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
// More than two constrained states (Sec. 2.2 with K of n states)
// ======================================================================
extern "C" {

int sccsd_residual_states(sccsd_ctx* c, const double* t, int nstates, const double* zeta,
                          const double* R, double* omega, double* e_corr) {
  if (!c) return SCCSD_EINVAL;
  if (!t || !zeta || !R) return fail(c, SCCSD_EINVAL, "NULL argument");
  if (nstates < 2) return fail(c, SCCSD_EINVAL, "at least two constrained states");
  return guarded(c, [&] {
    set_states(c, nstates, zeta, R);
    Model& m = *c->multi;
    load_packed(c, m.g, t, m.t1, m.t2, false);
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

int sccsd_solve_ground_states(sccsd_ctx* c, const double* t0, int nstates, const double* zeta,
                              const double* R, double tol, int maxit, double refine_tol,
                              double* t_out, double* e_corr, int* iterations) {
  if (!c) return SCCSD_EINVAL;
  if (!zeta || !R) return fail(c, SCCSD_EINVAL, "NULL argument");
  if (nstates < 2) return fail(c, SCCSD_EINVAL, "at least two constrained states");
  int rc = guarded(c, [&] { set_states(c, nstates, zeta, R); });
  if (rc != SCCSD_OK) return rc;
  return solve_ground_impl(c, t0, 0.0, nullptr, nullptr, true, tol, maxit, refine_tol, t_out,
                           e_corr, iterations);
}

// Self-consistent SCCSD for the n lowest states: zeta_kl for every pair k < l
// solves O_kl = 0 (the context's projection: natural, or the state projection
// over all n states) by Broyden's method from zeta = 0
// (plain CCSD) with the unit matrix as the first Jacobian estimate; at every
// zeta the ground state and the n lowest right roots are re-converged.
int sccsd_solve_scc_states(sccsd_ctx* c, int nstates, double tol, int maxit, double ground_tol,
                           double eom_tol, double* zeta_out, double* O_out, double* e_corr,
                           double* omega, double* r0_out, double* R_out, int* iterations) {
  if (!c) return SCCSD_EINVAL;
  if (nstates < 2 || nstates > 8) return fail(c, SCCSD_EINVAL, "nstates must be 2..8");
  if (!(tol > 0.0) || maxit < 1 || !(ground_tol > 0.0) || !(eom_tol > 0.0))
    return fail(c, SCCSD_EINVAL, "bad tolerances or iteration limit");
  int status = SCCSD_OK;
  int rc = guarded(c, [&] {
    const int n = nstates, np = n * (n - 1) / 2;
    const int64_t dim = c->dim;
    std::vector<double> t(dim), R((size_t)n * dim), w(n), r0(n), zeta(np, 0.0), O(np, 0.0);
    std::vector<double> Jb((size_t)np * np, 0.0), zprev(np), Oprev(np);
    for (int p = 0; p < np; ++p) Jb[(size_t)p * np + p] = 1.0;
    bool have_states = false, have_prev = false;
    double E = 0.0;
    auto check = [&](int r) {
      if (r != SCCSD_OK) throw std::runtime_error("inner solver failed: " + c->err);
    };
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
      int gi = 0;
      if (have_states)
        check(sccsd_solve_ground_states(c, t.data(), n, zeta.data(), R.data(), ground_tol, 1000,
                                        1e-5, t.data(), &E, &gi));
      else
        check(sccsd_solve_ground(c, nullptr, 0.0, nullptr, nullptr, ground_tol, 1000, 1e-5,
                                 t.data(), &E, &gi));
      int si = 0;
      check(sccsd_solve_states(c, n, 0, eom_tol, 1000, 1e-4, w.data(), R.data(), &si));
      for (int k = 0; k < n; ++k) {
        // sign convention: largest |component| positive
        double* x = R.data() + (size_t)k * dim;
        int64_t im = 0;
        for (int64_t q = 1; q < dim; ++q)
          if (std::fabs(x[q]) > std::fabs(x[im])) im = q;
        if (x[im] < 0)
          for (int64_t q = 0; q < dim; ++q) x[q] = -x[q];
      }
      {
        // r0 = eta.R / omega and the overlaps decide zeta: FP64 in a mixed context
        Fp64Scope fp64(c);
        std::vector<double> etaR(n);
        for (int k0 = 0; k0 < n; k0 += c->max_batch) {
          const int nb = std::min(c->max_batch, n - k0);
          eta_dot(c, nb, R.data() + (size_t)k0 * dim, etaR.data() + k0);
        }
        for (int k = 0; k < n; ++k) r0[k] = etaR[k] / w[k];
        check(sccsd_overlaps(c, n, r0.data(), R.data(), c->projection, O.data()));
      }
      have_states = true;
      double omax = 0.0, dz = 0.0;
      for (int p = 0; p < np; ++p) {
        omax = std::max(omax, std::fabs(O[p]));
        if (have_prev) dz = std::max(dz, std::fabs(zeta[p] - zprev[p]));
      }
      if (getenv("SCCSD_LOG")) {
        fprintf(stderr, "{\"solver\": \"scc_states\", \"iter\": %d, \"max_O\": %.3e, \"zeta\": [", it,
                omax);
        for (int p = 0; p < np; ++p) fprintf(stderr, "%s%.12f", p ? ", " : "", zeta[p]);
        fprintf(stderr, "]}\n");
      }
      if (omax < tol && have_prev && dz < 1e-8) break;
      if (have_prev) {
        // Broyden: Jb += (dO - Jb dz) dz^T / (dz . dz)
        std::vector<double> dzv(np), u(np);
        double zz = 0.0;
        for (int p = 0; p < np; ++p) {
          dzv[p] = zeta[p] - zprev[p];
          zz += dzv[p] * dzv[p];
        }
        if (zz > 0.0) {
          for (int p = 0; p < np; ++p) {
            double s = O[p] - Oprev[p];
            for (int q = 0; q < np; ++q) s -= Jb[(size_t)p * np + q] * dzv[q];
            u[p] = s / zz;
          }
          for (int p = 0; p < np; ++p)
            for (int q = 0; q < np; ++q) Jb[(size_t)p * np + q] += u[p] * dzv[q];
        }
      }
      zprev = zeta;
      Oprev = O;
      have_prev = true;
      // zeta -= Jb^-1 O (Gaussian elimination with partial pivoting)
      std::vector<double> A = Jb, b = O;
      for (int col = 0; col < np; ++col) {
        int piv = col;
        for (int r = col + 1; r < np; ++r)
          if (std::fabs(A[(size_t)r * np + col]) > std::fabs(A[(size_t)piv * np + col])) piv = r;
        if (!(std::fabs(A[(size_t)piv * np + col]) > 1e-300))
          throw std::runtime_error("Broyden Jacobian of the overlaps is singular");
        if (piv != col) {
          for (int q = 0; q < np; ++q) std::swap(A[(size_t)col * np + q], A[(size_t)piv * np + q]);
          std::swap(b[col], b[piv]);
        }
        for (int r = col + 1; r < np; ++r) {
          const double f = A[(size_t)r * np + col] / A[(size_t)col * np + col];
          for (int q = col; q < np; ++q) A[(size_t)r * np + q] -= f * A[(size_t)col * np + q];
          b[r] -= f * b[col];
        }
      }
      for (int r = np - 1; r >= 0; --r) {
        double s = b[r];
        for (int q = r + 1; q < np; ++q) s -= A[(size_t)r * np + q] * b[q];
        b[r] = s / A[(size_t)r * np + r];
      }
      for (int p = 0; p < np; ++p) zeta[p] -= b[p];
    }
    if (it > maxit) status = SCCSD_ENOTCONV;
    // the zeta of the last evaluation (after a non-converged loop, zeta holds an untried step)
    const std::vector<double>& zfinal = it > maxit ? zprev : zeta;
    if (zeta_out) std::copy(zfinal.begin(), zfinal.end(), zeta_out);
    if (O_out) std::copy(O.begin(), O.end(), O_out);
    if (e_corr) *e_corr = E;
    if (omega) std::copy(w.begin(), w.end(), omega);
    if (r0_out) std::copy(r0.begin(), r0.end(), r0_out);
    if (R_out) {
      if (c->be->is_device(R_out))
        c->be->upload(R_out, R.data(), (int64_t)n * dim, false);
      else
        std::memcpy(R_out, R.data(), sizeof(double) * n * dim);
    }
    if (iterations) *iterations = std::min(it, maxit);
  });
  if (rc != SCCSD_OK) return rc;
  if (status != SCCSD_OK) return fail(c, status, "zeta iteration not converged within maxit");
  return SCCSD_OK;
}

}  // extern "C"
