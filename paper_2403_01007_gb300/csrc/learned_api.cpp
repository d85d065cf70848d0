// C ABI of the learned initial guess and preconditioner.
#include "context.h"
#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <vector>

using namespace sccsd;

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
    // the update divides by these: every entry must be finite and positive
    const bool dev = c->be->is_device(Dprec);
    std::vector<double> h((size_t)c->dim);
    if (dev)
      c->be->download(h.data(), Dprec, c->dim, false);
    else
      std::copy(Dprec, Dprec + c->dim, h.begin());
    for (double x : h)
      if (!(x > 0.0) || !std::isfinite(x))
        throw std::invalid_argument("preconditioner entries must be finite and positive");
    if (!c->Dprec) c->Dprec = c->be->alloc(c->dim);
    c->be->upload(c->Dprec, h.data(), c->dim, false);
    c->use_dprec = true;
    c->be->sync();
  });
}

}  // extern "C"
