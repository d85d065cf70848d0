// Test double of the device backend (tests only; never linked into the
// library): every Backend method done with plain host loops, so that the
// graph construction, its forward/reverse differentiation and the C ABI
// marshalling can be checked on a machine without a GPU. The product library
// always uses the CUDA backend and fails when it cannot.
#include <cstring>
#include <memory>
#include <set>
#include <vector>
#include <cstdio>
#include <stdexcept>
#include <cuda_runtime.h>
#include "../../paper_2403_01007_gb300/csrc/backend.h"
#include "../../paper_2403_01007_gb300/csrc/graph.h"
namespace sccsd {
class HostBackend : public Backend {
 public:
  std::set<const void*> mine;
  std::vector<double*> slots = std::vector<double*>(8, nullptr);
  std::vector<int64_t> slot_n = std::vector<int64_t>(8, 0);
  std::vector<double> G; int64_t Gver = -1;
  double* alloc(int64_t n) override { double* p = new double[n]; std::memset(p, 0xff, n*8); mine.insert(p); return p; }
  void release(double* p) override { mine.erase(p); delete[] p; }
  void upload(double* d, const double* s, int64_t n, bool) override { std::memmove(d, s, n*8); }
  void download(double* d, const double* s, int64_t n, bool) override { std::memmove(d, s, n*8); }
  void fill(double* p, int64_t n, double v) override { for (int64_t i=0;i<n;++i) p[i]=v; }
  bool is_device(const void* p) override { return mine.count(p) > 0; }
  void sync() override {}
  void unpack(const double* x, int o, int v, double* t1, double* t2, bool bra) override {
    int64_t ov = (int64_t)o*v;
    for (int64_t k=0;k<ov;++k) t1[k]=x[k];
    for (int i=0;i<o;++i) for (int j=0;j<o;++j) for (int a=0;a<v;++a) for (int b=0;b<v;++b) {
      int64_t P=(int64_t)a*o+i, Q=(int64_t)b*o+j; int64_t lo=P<Q?P:Q, hi=P<Q?Q:P;
      double val = x[ov + hi*(hi+1)/2 + lo];
      if (bra && P!=Q) val *= 0.5;
      t2[((int64_t)(i*o+j)*v+a)*v+b] = val;
    }
  }
  void pack(const double* t1, const double* t2, int o, int v, double* x, bool bra) override {
    int64_t ov=(int64_t)o*v;
    for (int64_t k=0;k<ov;++k) x[k]=t1[k];
    for (int64_t Q=0;Q<ov;++Q) for (int64_t P=0;P<=Q;++P) {
      int a=P/o,i=P%o,b=Q/o,j=Q%o;
      double val = t2[((int64_t)(i*o+j)*v+a)*v+b];
      if (bra && P!=Q) val += t2[((int64_t)(j*o+i)*v+b)*v+a];
      x[ov + Q*(Q+1)/2 + P] = val;
    }
  }
  void copy_view(int rank, const int64_t* dims, double* out, const int64_t* ostr, const double* in, const int64_t* istr, double coef, bool acc) override {
    int64_t total=1; for (int k=0;k<rank;++k) total*=dims[k];
    for (int64_t lin=0; lin<total; ++lin) {
      int64_t r=lin, oo=0, ii=0;
      for (int k=rank-1;k>=0;--k){ int64_t c=r%dims[k]; r/=dims[k]; oo+=c*ostr[k]; ii+=c*istr[k]; }
      out[oo] = (acc? out[oo]:0.0) + coef*in[ii];
    }
  }
  void mul_view(int rank, const int64_t* dims, double* out, const int64_t* ostr, const double* a, const int64_t* astr, const double* b, const int64_t* bstr, double coef, bool acc) override {
    int64_t total=1; for (int k=0;k<rank;++k) total*=dims[k];
    for (int64_t lin=0; lin<total; ++lin) {
      int64_t r=lin, oo=0, ia=0, ib=0;
      for (int k=rank-1;k>=0;--k){ int64_t c=r%dims[k]; r/=dims[k]; oo+=c*ostr[k]; ia+=c*astr[k]; ib+=c*bstr[k]; }
      out[oo] = (acc? out[oo]:0.0) + coef*a[ia]*b[ib];
    }
  }
  static int64_t vr(const MatView& v, int64_t r){ return v.n2r ? (r / v.n2r) * v.sr1 + (r % v.n2r) * v.sr2 : r * v.sr2; }
  static int64_t vk(const MatView& v, int64_t k){ return v.n2k ? (k / v.n2k) * v.sk1 + (k % v.n2k) * v.sk2 : k * v.sk2; }
  void gemm_view(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const MatView& A, const MatView& B, double* C, bool) override {
    for (int64_t b=0;b<nb;++b) for (int64_t m=0;m<M;++m) for (int64_t n=0;n<N;++n) {
      double s=0; const double* a=A.p + b*A.sb + vr(A,m); const double* bb=B.p + b*B.sb + vr(B,n);
      for (int64_t k=0;k<K;++k) s+=a[vk(A,k)]*bb[vk(B,k)];
      C[(b*M+m)*N+n]=alpha*s;
    }
  }
  void* stream() override { return nullptr; }
  void set_precision(int) override {}
  int get_precision() const override { return 0; }
  void set_capturing(bool) override {}
  bool tc_will_use(int64_t, int64_t, int64_t, int64_t) override { return false; }
  bool tc_cached(const OperandKey&) override { return false; }
  void gemm_tc_keyed(int64_t, int64_t, int64_t, double, const MatView&, const OperandKey*, const MatView&, const OperandKey*, double*, const OutView*, bool) override {}
  double* scratch(int slot, int64_t n) override {
    if (slot_n[slot] < n) { delete[] slots[slot]; slots[slot]=new double[n]; slot_n[slot]=n; }
    return slots[slot];
  }
  void build_G(const Graph& g, const double* L) {
    int o=g.o, v=g.v, J=g.J, n=o+v; G.assign((size_t)v*v*v*v, 0.0);
    for (int a=0;a<v;++a) for (int b=0;b<v;++b) for (int c=0;c<v;++c) for (int d=0;d<v;++d) {
      double s=0; for (int q=0;q<J;++q) s += L[((int64_t)q*n+o+a)*n+o+c]*L[((int64_t)q*n+o+b)*n+o+d];
      G[((int64_t)(a*v+b)*v+c)*v+d]=s; }
  }
  void* record_event() override { return nullptr; }
  double elapsed_ms(void*, void*) override { return 0; }
  void profile(bool) override {}
  void profile_read(double*, long long*, double*, long long*) override {}
  double* pool_get(int64_t n) override { return alloc(n); }
  void pool_put(double* p, int64_t) override { release(p); }
  void ladder(const Graph& g, const double* L, int64_t ver, const double* X, double* Y, int64_t rows) override {
    if (ver != Gver) { build_G(g, L); Gver = ver; }
    int v=g.v; int64_t vv=(int64_t)v*v;
    for (int64_t ij=0; ij<rows; ++ij) for (int64_t ab=0; ab<vv; ++ab) {
      double s=0; for (int64_t cd=0; cd<vv; ++cd) s+=G[ab*vv+cd]*X[ij*vv+cd]; Y[ij*vv+ab]=s; }
  }
  void ladder_adj_l(const Graph& g, const double* L, const double* Yb, const double* X, double* out) override {
    int o=g.o, v=g.v, J=g.J, n=o+v; int64_t vv=(int64_t)v*v;
    // D_acbd = sum_ij Yb_ij^ab X_ij^cd ; out[J][a][c] = sum_bd (D_acbd + D_bdac) L_bd
    std::vector<double> D((size_t)vv*vv, 0.0);
    for (int a=0;a<v;++a) for (int b=0;b<v;++b) for (int c=0;c<v;++c) for (int d=0;d<v;++d) {
      double s=0; for (int64_t ij=0; ij<(int64_t)o*o; ++ij) s+=Yb[ij*vv+a*v+b]*X[ij*vv+c*v+d];
      D[((int64_t)(a*v+c)*v+b)*v+d]=s; }
    for (int q=0;q<J;++q) for (int a=0;a<v;++a) for (int c=0;c<v;++c) {
      double s=0; for (int b=0;b<v;++b) for (int d=0;d<v;++d) {
        double l=L[((int64_t)q*n+o+b)*n+o+d];
        s += (D[((int64_t)(a*v+c)*v+b)*v+d] + D[((int64_t)(b*v+d)*v+a)*v+c])*l; }
      out[((int64_t)q*v+a)*v+c]=s; }
  }
};
std::unique_ptr<Backend> make_backend(void*, int) { return std::make_unique<HostBackend>(); }
}

namespace sccsd {
// device-only solver kernels: not available in the test double
static void no_device() { throw std::runtime_error("solver kernels need the device backend"); }
void launch_small_solve(cudaStream_t, int, const double*, const double*, double*, int*) { no_device(); }
void launch_small_eig(cudaStream_t, int, const double*, double*, double*, double*, int, int*, int*) { no_device(); }
void launch_diis(cudaStream_t, int, const double*, double*, int*) { no_device(); }
void launch_denoms(cudaStream_t, int o, int v, const double* eps, double* D) {
  const int64_t ov = (int64_t)o * v;
  for (int64_t k = 0; k < ov; ++k) D[k] = eps[o + k / o] - eps[k % o];
  int64_t q = ov;
  for (int64_t Q = 0; Q < ov; ++Q)
    for (int64_t P = 0; P <= Q; ++P) D[q++] = D[P] + D[Q];
}
void launch_jacobi(cudaStream_t, int64_t, const double*, const double*, const double*, double*) { no_device(); }
void launch_precond(cudaStream_t, int64_t n, const double* r, const double* D, double lam, double* out) {
  for (int64_t k = 0; k < n; ++k) {
    double d = lam - D[k];
    if (d > -1e-4 && d < 1e-4) d = d < 0 ? -1e-4 : 1e-4;
    out[k] = r[k] / d;
  }
}
void launch_axpby(cudaStream_t, int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t k = 0; k < n; ++k) y[k] = a * x[k] + b * y[k];
}
void launch_floor(cudaStream_t, int64_t n, const double* ref, double frac, double* d) {
  for (int64_t k = 0; k < n; ++k) d[k] = d[k] > frac * ref[k] ? d[k] : frac * ref[k];
}
void launch_scale(cudaStream_t, int64_t n, const double* d, const double* x, double* y) {
  for (int64_t k = 0; k < n; ++k) y[k] = d[k] * x[k];
}
void launch_ritz_residual(cudaStream_t, int, int64_t, const double*, const double*, const double*, const int*, double*) { no_device(); }
}
extern "C" long long sccsd_gemm_tn_noalloc_capacity(void) { return 0; }
extern "C" int sccsd_gemm_tn_noalloc(long long, long long, long long, double, const double*, const double*, double*, void*) { return -1; }
namespace sccsd {
void launch_learned_features(cudaStream_t, int, int, const double*, const double*, const double*, const double*, double, double, double, float*) { no_device(); }
void launch_learned_targets(cudaStream_t, int, int, const double*, const double*, const double*, double, float*) { no_device(); }
void launch_learned_apply(cudaStream_t, int, int, const float*, const double*, double, double*, double*) { no_device(); }
}
extern "C" int sccsd_mlp_forward(struct sccsd_mlp*, const float*, long long, float*) { return -5; }
