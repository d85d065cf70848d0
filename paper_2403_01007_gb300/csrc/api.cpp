// C ABI of the SCCSD hot path: contexts, residual, transformations,
// densities and marshalling (solvers, multipliers, learned part and CUDA-graph
// batching are in their own files).
#include "context.h"
#include "tc_tune.h"

#include <cstring>
#include <string>

using namespace sccsd;

namespace sccsd {

Model& model_states(sccsd_ctx* c, int n) {
  if (c->multi && c->multi_n != n) {
    if (c->cur == c->multi.get()) c->cur = nullptr;
    c->multi.reset();
    c->multi_set = false;
  }
  if (!c->multi) {
    c->multi = build_model(c->be.get(), c->o, c->v, c->J, false, n);
    c->multi_n = n;
    Model* m = c->multi.get();
    m->g.trace = getenv("SCCSD_TRACE") != nullptr;
    m->g.set_input(m->L, c->L, true);
    m->g.set_input(m->h, c->h, true);
    m->g.set_input(m->delta, c->delta, true);
    double* z = m->g.t[m->t2zero].data;
    if (!z) {
      m->g.t[m->t2zero].data = c->be->alloc(m->g.t[m->t2zero].numel());
      z = m->g.t[m->t2zero].data;
    }
    c->be->fill(z, m->g.t[m->t2zero].numel(), 0.0);
    m->g.touch(m->t2zero);
  }
  return *c->multi;
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

}  // namespace sccsd

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
    const bool L_dev = c->be->is_device(L);
    c->be->upload(c->L, L, (int64_t)J * n * n, L_dev);
    {
      // each L^J must be finite and symmetric in pq (to rounding)
      std::vector<double> hL;
      const double* Lh = L;
      if (L_dev) {
        hL.resize((size_t)J * n * n);
        c->be->download(hL.data(), c->L, (int64_t)J * n * n, false);
        Lh = hL.data();
      }
      double mx = 0.0;
      for (int64_t k = 0; k < (int64_t)J * n * n; ++k) {
        if (!std::isfinite(Lh[k])) throw std::invalid_argument("L is not finite");
        mx = std::max(mx, std::fabs(Lh[k]));
      }
      for (int64_t q = 0; q < J; ++q)
        for (int64_t a = 0; a < n; ++a)
          for (int64_t b = a + 1; b < n; ++b)
            if (std::fabs(Lh[(q * n + a) * n + b] - Lh[(q * n + b) * n + a]) > 1e-12 * mx)
              throw std::invalid_argument("L^J is not symmetric in pq");
    }
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
  if (M == 0 || N == 0) return SCCSD_OK;  // an empty C: nothing to write
  sccsd_ctx tmp;
  return guarded(&tmp, [&] {
    auto be = make_backend(stream, precision);
    for (const double* p : {A, B, (const double*)C})
      if (!be->is_device(p)) throw std::invalid_argument("sccsd_gemm_tn needs device pointers");
    if (K == 0)
      be->fill(C, M * N, 0.0);  // the empty sum
    else
      be->gemm_tn(1, M, N, K, alpha, A, B, C, precision != SCCSD_FP64);
    be->sync();
  });
}

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

int sccsd_overlap_states(sccsd_ctx* c, double ra0, const double* Ra, double rb0,
                         const double* Rb, double* O) {
  if (!c) return SCCSD_EINVAL;
  if (!Ra || !Rb || !O) return fail(c, SCCSD_EINVAL, "NULL argument");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual or a solver first");
  return guarded(c, [&] {
    Model& m = *c->cur;
    OverlapSec& S = overlap_section(m);
    OverlapKSec& K = overlap_k_section(m);
    set_scalar(c, m.g, S.ra0, ra0);
    set_scalar(c, m.g, S.rb0, rb0);
    load_packed(c, m.g, Ra, S.ra1, S.ra2, false);
    load_packed(c, m.g, Rb, S.rb1, S.rb2, false);
    m.g.run({K.maa, K.mab, K.nab, K.nbb, K.Saa, K.Sab, K.Sbb});
    const int ids[7] = {K.maa, K.mab, K.nab, K.nbb, K.Saa, K.Sab, K.Sbb};
    double sv[7];
    for (int i = 0; i < 7; ++i) sv[i] = get_scalar(c, m.g, ids[i]);
    *O = overlap_k_value(sv);
    c->be->sync();
  });
}

int sccsd_overlaps(sccsd_ctx* c, int nstates, const double* r0, const double* R, int projection,
                   double* O) {
  if (!c) return SCCSD_EINVAL;
  if (!r0 || !R || !O) return fail(c, SCCSD_EINVAL, "NULL argument");
  if (nstates < 2) return fail(c, SCCSD_EINVAL, "at least two states");
  if (projection != 0 && projection != 1) return fail(c, SCCSD_EINVAL, "projection must be 0 or 1");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual or a solver first");
  return guarded(c, [&] {
    const int n = nstates;
    const int64_t dim = c->dim;
    Model& m = *c->cur;
    OverlapSec& S = overlap_section(m);
    OverlapKSec* K = projection == 1 ? &overlap_k_section(m) : nullptr;
    // M[k][j] = <psi_k|R_j>, G[j][l] = <R_j|R_l> (state projection)
    std::vector<double> M((size_t)n * n, 0.0), G((size_t)n * n, 0.0);
    int p = 0;
    for (int k = 0; k < n; ++k)
      for (int l = k + 1; l < n; ++l, ++p) {
        set_scalar(c, m.g, S.ra0, r0[k]);
        set_scalar(c, m.g, S.rb0, r0[l]);
        load_packed(c, m.g, R + (int64_t)k * dim, S.ra1, S.ra2, false);
        load_packed(c, m.g, R + (int64_t)l * dim, S.rb1, S.rb2, false);
        if (!K) {
          m.g.run({S.O});
          O[p] = get_scalar(c, m.g, S.O);
          continue;
        }
        const int ids[7] = {K->maa, K->mab, K->nab, K->nbb, K->Saa, K->Sab, K->Sbb};
        m.g.run(std::vector<int>(ids, ids + 7));
        double sv[7];
        for (int i = 0; i < 7; ++i) sv[i] = get_scalar(c, m.g, ids[i]);
        M[(size_t)k * n + k] = sv[0];
        M[(size_t)k * n + l] = sv[1];
        M[(size_t)l * n + k] = sv[2];
        M[(size_t)l * n + l] = sv[3];
        G[(size_t)k * n + k] = sv[4];
        G[(size_t)k * n + l] = G[(size_t)l * n + k] = sv[5];
        G[(size_t)l * n + l] = sv[6];
      }
    if (K) {
      // O_kl = sum_jm M[k][j] (G^-1)_jm M[l][m]: W = G^-1 M^T by Gaussian
      // elimination with partial pivoting
      std::vector<double> A = G, W((size_t)n * n);
      for (int j = 0; j < n; ++j)
        for (int l = 0; l < n; ++l) W[(size_t)j * n + l] = M[(size_t)l * n + j];
      double scale = 0.0;
      for (double x : G) scale = std::max(scale, std::fabs(x));
      for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
          if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
        if (!(std::fabs(A[(size_t)piv * n + col]) > 1e-14 * std::max(1.0, scale)))
          throw std::invalid_argument("the states are linearly dependent");
        if (piv != col)
          for (int q = 0; q < n; ++q) {
            std::swap(A[(size_t)col * n + q], A[(size_t)piv * n + q]);
            std::swap(W[(size_t)col * n + q], W[(size_t)piv * n + q]);
          }
        for (int r = 0; r < n; ++r) {
          if (r == col) continue;
          const double f = A[(size_t)r * n + col] / A[(size_t)col * n + col];
          if (f == 0.0) continue;
          for (int q = 0; q < n; ++q) {
            A[(size_t)r * n + q] -= f * A[(size_t)col * n + q];
            W[(size_t)r * n + q] -= f * W[(size_t)col * n + q];
          }
        }
      }
      for (int r = 0; r < n; ++r)
        for (int q = 0; q < n; ++q) W[(size_t)r * n + q] /= A[(size_t)r * n + r];
      p = 0;
      for (int k = 0; k < n; ++k)
        for (int l = k + 1; l < n; ++l, ++p) {
          double o = 0.0;
          for (int j = 0; j < n; ++j) o += M[(size_t)k * n + j] * W[(size_t)j * n + l];
          O[p] = o;
        }
    }
    c->be->sync();
  });
}

int sccsd_set_projection(sccsd_ctx* c, int projection) {
  if (!c) return SCCSD_EINVAL;
  if (projection != 0 && projection != 1) return fail(c, SCCSD_EINVAL, "projection must be 0 or 1");
  c->projection = projection;
  return SCCSD_OK;
}

int sccsd_set_precision(sccsd_ctx* c, int precision) {
  if (!c) return SCCSD_EINVAL;
  if (precision < SCCSD_FP64 || precision > SCCSD_BF16) return fail(c, SCCSD_EINVAL, "bad precision");
  return guarded(c, [&] {
    switch_precision(c, precision);
    c->precision = precision;
  });
}

int sccsd_set_autotune(sccsd_ctx* c, int enable) {
  if (!c) return SCCSD_EINVAL;
  if (enable != 0 && enable != 1) return fail(c, SCCSD_EINVAL, "enable must be 0 or 1");
  return guarded(c, [&] { c->be->set_autotune(enable == 1); });
}

// these four have no context to report through: no exception leaves them
int sccsd_autotune_export(char* buf, long long cap, long long* len) {
  try {
    const std::string text = TcTuneTable::global().dump();
    const long long need = (long long)text.size() + 1;
    if (len) *len = need;
    if (!buf || cap < need) return SCCSD_EINVAL;
    std::memcpy(buf, text.c_str(), (size_t)need);
    return SCCSD_OK;
  } catch (const std::bad_alloc&) {
    return SCCSD_ENOMEM;
  } catch (...) {
    return SCCSD_EINTERNAL;
  }
}

int sccsd_autotune_import(const char* text) {
  if (!text) return SCCSD_EINVAL;
  try {
    return TcTuneTable::global().load(std::string(text)) == 0 ? SCCSD_OK : SCCSD_EINVAL;
  } catch (const std::bad_alloc&) {
    return SCCSD_ENOMEM;
  } catch (...) {
    return SCCSD_EINTERNAL;
  }
}

void sccsd_autotune_clear(void) {
  try {
    TcTuneTable::global().clear();
  } catch (...) {
  }
}

long long sccsd_autotune_entries(void) {
  try {
    return (long long)TcTuneTable::global().size();
  } catch (...) {
    return 0;
  }
}

int sccsd_integral_derivative(sccsd_ctx* c, const double* D1, const double* Gamma,
                              const double* h1, const double* L1, double* out) {
  if (!c) return SCCSD_EINVAL;
  if (!D1 || !h1 || !out || (Gamma == nullptr) != (L1 == nullptr))
    return fail(c, SCCSD_EINVAL, "NULL argument");
  return guarded(c, [&] {
    ensure_small(c);
    Dev d{c};
    const int64_t n2 = (int64_t)c->n * c->n, jn2 = (int64_t)c->J * n2;
    // host arrays are staged in solver buffers; device arrays are read in place
    auto on_device = [&](size_t slot, const double* x, int64_t len) -> const double* {
      if (c->be->is_device(x)) return x;
      double* b = solver_buf(c, slot, len);
      c->be->upload(b, x, len, false);
      return b;
    };
    double s = d.dot(on_device(70, D1, n2), on_device(71, h1, n2), n2);
    if (Gamma) s += d.dot(on_device(72, Gamma, jn2), on_device(73, L1, jn2), jn2);
    if (c->be->is_device(out))
      c->be->upload(out, &s, 1, false);
    else
      *out = s;
    c->be->sync();
  });
}

int sccsd_input_derivative(sccsd_ctx* c, const double* D1, const double* Gamma,
                           const double* deps, const double* dL, double* out) {
  if (!c) return SCCSD_EINVAL;
  if (!D1 || !deps || !out || (Gamma == nullptr) != (dL == nullptr))
    return fail(c, SCCSD_EINVAL, "NULL argument");
  double* dh = nullptr;
  const int rc = guarded(c, [&] {
    const int64_t o = c->o, n = c->n, J = c->J;
    // the change of h per unit of the perturbation: h = diag(eps) - 2 sum_J L^J s_J
    // + sum_Jk L^J_pk L^J_kq with s_J = sum_k L^J_kk (k occupied), to first order
    std::vector<double> de(n);
    if (c->be->is_device(deps))
      c->be->download(de.data(), deps, n, false);
    else
      std::copy(deps, deps + n, de.begin());
    std::vector<double> E((size_t)n * n, 0.0);
    for (int64_t p = 0; p < n; ++p) E[p * n + p] = de[p];
    Graph g;
    g.be = c->be.get();
    int Ein = g.input({n, n}, "dE");
    int hh = Ein;
    int Lin = -1, dLin = -1;
    if (dL) {
      Lin = g.input({J, n, n}, "L");
      dLin = g.input({J, n, n}, "dL");
      int din = g.input({o, o}, "delta");
      int s = g.contract(g.slice(Lin, {0, 0, 0}, {J, o, o}), "Jkl", din, "kl", "J");
      int ds = g.contract(g.slice(dLin, {0, 0, 0}, {J, o, o}), "Jkl", din, "kl", "J");
      hh = g.add("pq", {{Ein, "pq", 1.0},
                        {g.contract(dLin, "Jpq", s, "J", "pq"), "pq", -2.0},
                        {g.contract(Lin, "Jpq", ds, "J", "pq"), "pq", -2.0},
                        {g.contract(g.slice(dLin, {0, 0, 0}, {J, n, o}), "Jpk",
                                    g.slice(Lin, {0, 0, 0}, {J, o, n}), "Jkq", "pq"), "pq", 1.0},
                        {g.contract(g.slice(Lin, {0, 0, 0}, {J, n, o}), "Jpk",
                                    g.slice(dLin, {0, 0, 0}, {J, o, n}), "Jkq", "pq"), "pq", 1.0}});
      g.set_input(Lin, c->L, true);
      g.set_input(dLin, dL, c->be->is_device(dL));
      g.set_input(din, c->delta, true);
    }
    g.set_input(Ein, E.data(), false);
    g.run({hh});
    dh = solver_buf(c, 74, n * n);
    c->be->upload(dh, g.data(hh), n * n, true);
    c->be->sync();
  });
  if (rc != SCCSD_OK) return rc;
  return sccsd_integral_derivative(c, D1, Gamma, dh, dL, out);
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
