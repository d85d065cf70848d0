// Test double of the device backend (tests only; never linked into the
// library): every Backend method done with plain host loops, so that the
// graph construction, its forward/reverse differentiation, the C ABI
// marshalling and the solvers' control flow (with host versions of the small
// dense solver kernels) can be checked on a machine without a GPU. The product
// library always uses the CUDA backend and fails when it cannot.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <set>
#include <vector>
#include <cstdio>
#include <cstdlib>
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
  // Stand-in for an expired bounded wait in a tensor-core kernel: the device
  // backend reads the kernel's error flag at a synchronisation and throws this
  // CudaError. SCCSD_HOST_FAKE_WAIT_EXPIRY=k makes the k-th synchronisation
  // after it is set (counting from 0) report it once.
  long long fake_syncs = 0;
  void sync() override {
    const char* e = getenv("SCCSD_HOST_FAKE_WAIT_EXPIRY");
    if (!e) {
      fake_syncs = 0;
      return;
    }
    if (fake_syncs++ == atoll(e))
      throw CudaError("tensor-core pipeline wait expired (code 3)");
  }
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
  // Mixed precision emulated on the host: the tensor-core route takes every
  // contraction with M, N >= 2 (the device adds a size threshold), operands
  // become BF16 slices (one, or two with the three leading products), each
  // slice product is accumulated in FP32 and the products are summed in FP64.
  int prec = 0;
  void set_precision(int p) override { prec = p; }
  int get_precision() const override { return prec; }
  void set_capturing(bool) override {}
  bool tc_will_use(int64_t nb, int64_t M, int64_t N, int64_t) override {
    return prec != 0 && nb == 1 && M >= 2 && N >= 2;
  }
  bool tc_cached(const OperandKey&) override { return false; }
  static float bf16(double x) {           // round to nearest even on the upper 16 bits
    float f = (float)x;
    uint32_t b;
    std::memcpy(&b, &f, 4);
    b += 0x7FFFu + ((b >> 16) & 1u);
    b &= 0xFFFF0000u;
    std::memcpy(&f, &b, 4);
    return f;
  }
  static double view_el(const MatView& v, int64_t r, int64_t k) {
    const int64_t R = v.n2r > 0 ? (r / v.n2r) * v.sr1 + (r % v.n2r) * v.sr2 : r * v.sr2;
    const int64_t Q = v.n2k > 0 ? (k / v.n2k) * v.sk1 + (k % v.n2k) * v.sk2 : k * v.sk2;
    return v.p[R + Q];
  }
  static int64_t level_off(int n, const int64_t* e, const int64_t* st, int64_t i) {
    int64_t off = 0;
    for (int l = n - 1; l > 0; --l) {
      off += (i % e[l]) * st[l];
      i /= e[l];
    }
    return off + i * st[0];
  }
  // slices of rows x K values
  void slices(int64_t rows, int64_t K, const std::function<double(int64_t, int64_t)>& get,
              std::vector<float>& out) const {
    const int sl = prec == 1 ? 2 : 1;
    out.assign((size_t)sl * rows * K, 0.0f);
    for (int64_t r = 0; r < rows; ++r)
      for (int64_t k = 0; k < K; ++k) {
        const double x = get(r, k);
        const float x0 = bf16(x);
        out[(size_t)r * K + k] = x0;
        if (sl == 2) out[(size_t)(rows + r) * K + k] = bf16(x - (double)x0);
      }
  }
  double sliced_dot(const std::vector<float>& a, int64_t Ma, int64_t m, const std::vector<float>& b,
                    int64_t Nb, int64_t n, int64_t K) const {
    const int sl = prec == 1 ? 2 : 1;
    double s = 0.0;
    for (int i = 0; i < sl; ++i)
      for (int j = 0; i + j < sl; ++j) {
        float f = 0.0f;
        const float* x = &a[(size_t)(i * Ma + m) * K];
        const float* y = &b[(size_t)(j * Nb + n) * K];
        for (int64_t k = 0; k < K; ++k) f += x[k] * y[k];
        s += (double)f;
      }
    return s;
  }
  void gemm_tc_keyed(int64_t M, int64_t N, int64_t K, double alpha, const MatView& A,
                     const OperandKey*, const MatView& B, const OperandKey*, double* C,
                     const OutView* ov, bool acc) override {
    std::vector<float> a, b;
    slices(M, K, [&](int64_t r, int64_t k) { return view_el(A, r, k); }, a);
    slices(N, K, [&](int64_t r, int64_t k) { return view_el(B, r, k); }, b);
    const OutView o = ov ? *ov : OutView::dense(N);
    for (int64_t m = 0; m < M; ++m)
      for (int64_t n = 0; n < N; ++n) {
        double& c = C[level_off(o.nr, o.re, o.rs, m) + level_off(o.nc, o.ce, o.cs, n)];
        c = (acc ? c : 0.0) + alpha * sliced_dot(a, M, m, b, N, n, K);
      }
  }
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
    {
      // the device ladder packs X by its pair symmetry X_ij^cd = X_ji^dc; every
      // operand the graph hands to the ladder must have it
      const int o = g.o;
      const int64_t oo = (int64_t)o * o, nb = rows / oo;
      double big = 0.0, bad = 0.0;
      for (int64_t z = 0; z < nb; ++z)
        for (int i = 0; i < o; ++i) for (int j = 0; j < o; ++j)
          for (int c = 0; c < v; ++c) for (int d = 0; d < v; ++d) {
            const double x = X[((z * oo) + (int64_t)i * o + j) * vv + (int64_t)c * v + d];
            const double y = X[((z * oo) + (int64_t)j * o + i) * vv + (int64_t)d * v + c];
            big = std::max(big, std::fabs(x));
            bad = std::max(bad, std::fabs(x - y));
          }
      if (bad > 1e-12 * std::max(1.0, big))
        throw std::runtime_error("ladder operand without pair symmetry");
    }
    if (prec != 0) {                      // the same BF16-slice emulation as gemm_tc_keyed
      std::vector<float> gs, xs;
      slices(vv, vv, [&](int64_t r, int64_t k) { return G[r * vv + k]; }, gs);
      slices(rows, vv, [&](int64_t r, int64_t k) { return X[r * vv + k]; }, xs);
      for (int64_t ij=0; ij<rows; ++ij) for (int64_t ab=0; ab<vv; ++ab)
        Y[ij*vv+ab] = sliced_dot(xs, rows, ij, gs, vv, ab, vv);
      return;
    }
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
std::unique_ptr<Backend> make_backend(void*, int precision) {
  auto b = std::make_unique<HostBackend>();
  b->prec = precision;
  return b;
}
}

namespace sccsd {
static void no_device() { throw std::runtime_error("this kernel needs the device backend"); }

// Host versions of the small dense solver kernels, written independently of
// the device ones (same contracts, different textbook algorithms), so that the
// solver control flow runs through the C ABI on the CPU.

// x = A^-1 b by Gaussian elimination with partial pivoting (A row-major m x m)
static int host_solve(int m, std::vector<double> A, std::vector<double>& b) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (std::fabs(A[(size_t)i * m + k]) > std::fabs(A[(size_t)p * m + k])) p = i;
    if (!(std::fabs(A[(size_t)p * m + k]) > 1e-300)) return 1;
    if (p != k) {
      for (int j = 0; j < m; ++j) std::swap(A[(size_t)k * m + j], A[(size_t)p * m + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < m; ++i) {
      const double f = A[(size_t)i * m + k] / A[(size_t)k * m + k];
      for (int j = k; j < m; ++j) A[(size_t)i * m + j] -= f * A[(size_t)k * m + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < m; ++j) s -= A[(size_t)i * m + j] * b[j];
    b[i] = s / A[(size_t)i * m + i];
  }
  return 0;
}

void launch_small_solve(cudaStream_t, int m, const double* A, const double* b, double* x,
                        int* info) {
  std::vector<double> a(A, A + (size_t)m * m), y(b, b + m);
  *info = host_solve(m, a, y);
  std::copy(y.begin(), y.end(), x);
}

// Pulay DIIS: minimise |sum c_k r_k| with sum c_k = 1 from B_pq = r_p . r_q
void launch_diis(cudaStream_t, int m, const double* B, double* c, int* info) {
  const int n = m + 1;
  double mx = 0.0;
  for (int k = 0; k < m; ++k) mx = std::max(mx, std::fabs(B[(size_t)k * m + k]));
  const double sc = mx > 0.0 ? 1.0 / mx : 1.0;
  std::vector<double> A((size_t)n * n, -1.0), y(n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * n + j] = B[(size_t)i * m + j] * sc;
  A[(size_t)m * n + m] = 0.0;
  y[m] = -1.0;
  *info = host_solve(n, A, y);
  std::copy(y.begin(), y.begin() + m, c);
}

// Eigenvalues of a real m x m matrix (row-major): Householder reduction to
// Hessenberg form, then complex QR steps with Wilkinson shifts and deflation
// (Golub & Van Loan, Sec. 7.4-7.5); eigenvectors of the wanted real roots by
// inverse iteration on the original matrix (Sec. 7.6.1).
void launch_small_eig(cudaStream_t, int m, const double* Hin, double* wr, double* wi, double* Y,
                      int nwant, int* order, int* info, int allow_complex) {
  typedef std::complex<double> cd;
  *info = 0;
  std::vector<double> H(Hin, Hin + (size_t)m * m);
  for (int k = 0; k + 2 < m; ++k) {
    double nrm = 0.0;
    for (int i = k + 1; i < m; ++i) nrm += H[(size_t)i * m + k] * H[(size_t)i * m + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    std::vector<double> v(m, 0.0);
    const double a = H[(size_t)(k + 1) * m + k];
    v[k + 1] = a + (a >= 0 ? nrm : -nrm);
    for (int i = k + 2; i < m; ++i) v[i] = H[(size_t)i * m + k];
    double vv = 0.0;
    for (int i = k + 1; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = 0; j < m; ++j) {          // H = (I - 2vv^T/vv) H
      double s = 0.0;
      for (int i = k + 1; i < m; ++i) s += v[i] * H[(size_t)i * m + j];
      s *= 2.0 / vv;
      for (int i = k + 1; i < m; ++i) H[(size_t)i * m + j] -= s * v[i];
    }
    for (int i = 0; i < m; ++i) {          // H = H (I - 2vv^T/vv)
      double s = 0.0;
      for (int j = k + 1; j < m; ++j) s += H[(size_t)i * m + j] * v[j];
      s *= 2.0 / vv;
      for (int j = k + 1; j < m; ++j) H[(size_t)i * m + j] -= s * v[j];
    }
  }
  std::vector<cd> T((size_t)m * m);
  for (size_t e = 0; e < T.size(); ++e) T[e] = H[e];
  auto at = [&](int i, int j) -> cd& { return T[(size_t)i * m + j]; };
  int hi = m - 1, iters = 0;
  while (hi > 0) {
    if (++iters > 100 * m) { *info = 2; break; }
    int lo = hi;
    while (lo > 0 && std::abs(at(lo, lo - 1)) >
                         1e-15 * (std::abs(at(lo, lo)) + std::abs(at(lo - 1, lo - 1))))
      --lo;
    if (lo == hi) { at(hi, hi - 1) = 0.0; --hi; continue; }
    if (lo > 0) at(lo, lo - 1) = 0.0;
    // Wilkinson shift: eigenvalue of the trailing 2 x 2 closer to its last entry
    const cd a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
    const cd tr = a + d, disc = std::sqrt((a - d) * (a - d) * 0.25 + b * c);
    cd mu1 = tr * 0.5 + disc, mu2 = tr * 0.5 - disc;
    cd mu = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
    if (iters % 11 == 0) mu += std::abs(at(hi, hi - 1));   // exceptional shift
    for (int i = lo; i <= hi; ++i) at(i, i) -= mu;
    std::vector<cd> cs(hi - lo), sn(hi - lo);
    for (int k = lo; k < hi; ++k) {        // QR of the active block by Givens rotations
      const cd x = at(k, k), y = at(k + 1, k);
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      cd cc = 1.0, ss = 0.0;
      if (r > 0.0) { cc = x / r; ss = y / r; }
      cs[k - lo] = cc;
      sn[k - lo] = ss;
      for (int j = k; j <= hi; ++j) {
        const cd u = at(k, j), w = at(k + 1, j);
        at(k, j) = std::conj(cc) * u + std::conj(ss) * w;
        at(k + 1, j) = -ss * u + cc * w;
      }
    }
    for (int k = lo; k < hi; ++k) {        // R Q
      const cd cc = cs[k - lo], ss = sn[k - lo];
      for (int i = lo; i <= std::min(hi, k + 2); ++i) {
        const cd u = at(i, k), w = at(i, k + 1);
        at(i, k) = u * cc + w * ss;
        at(i, k + 1) = -u * std::conj(ss) + w * std::conj(cc);
      }
    }
    for (int i = lo; i <= hi; ++i) at(i, i) += mu;
  }
  for (int i = 0; i < m; ++i) {
    const cd l = at(i, i);
    wr[i] = l.real();
    wi[i] = std::fabs(l.imag()) <= 1e-9 * std::max(1.0, std::abs(l)) ? 0.0 : l.imag();
  }
  std::vector<int> idx(m);
  for (int i = 0; i < m; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) { return wr[p] < wr[q]; });
  for (int k = 0; k < nwant && k < m; ++k) {
    order[k] = idx[k];
    if (wi[idx[k]] != 0.0 && *info == 0) *info = allow_complex ? 4 : 3;
  }
  if (*info != 0 && *info != 4) return;
  std::vector<double> prev(m, 0.0);
  for (int k = 0; k < nwant; ++k) {
    const int ik = order[k];
    if (k > 0 && wi[ik] != 0.0 && wi[order[k - 1]] == -wi[ik] && wr[order[k - 1]] == wr[ik]) {
      // second member of a complex pair: the other direction of its real
      // invariant plane, H y - Re(lambda) y of the first, orthonormalised
      std::vector<double> z(m);
      for (int i = 0; i < m; ++i) {
        double s = -wr[ik] * prev[i];
        for (int j = 0; j < m; ++j) s += Hin[(size_t)i * m + j] * prev[j];
        z[i] = s;
      }
      double dt = 0.0, nrm = 0.0;
      for (int i = 0; i < m; ++i) dt += z[i] * prev[i];
      for (int i = 0; i < m; ++i) { z[i] -= dt * prev[i]; nrm += z[i] * z[i]; }
      nrm = std::sqrt(nrm);
      for (int i = 0; i < m; ++i) Y[(size_t)i * nwant + k] = nrm > 0.0 ? z[i] / nrm : 0.0;
      continue;
    }
    const double lam = wr[order[k]] + 1e-10 * std::max(1.0, std::fabs(wr[order[k]]));
    std::vector<double> y(m);
    for (int i = 0; i < m; ++i) y[i] = 1.0 + 0.01 * i;
    for (int it = 0; it < 4; ++it) {
      std::vector<double> A(Hin, Hin + (size_t)m * m);
      for (int i = 0; i < m; ++i) A[(size_t)i * m + i] -= lam;
      if (host_solve(m, A, y) != 0) { *info = 2; return; }
      double nrm = 0.0;
      for (double e : y) nrm += e * e;
      nrm = std::sqrt(nrm);
      for (double& e : y) e /= nrm;
    }
    for (int i = 0; i < m; ++i) Y[(size_t)i * nwant + k] = y[i];
    prev = y;
  }
}
void launch_denoms(cudaStream_t, int o, int v, const double* eps, double* D) {
  const int64_t ov = (int64_t)o * v;
  for (int64_t k = 0; k < ov; ++k) D[k] = eps[o + k / o] - eps[k % o];
  int64_t q = ov;
  for (int64_t Q = 0; Q < ov; ++Q)
    for (int64_t P = 0; P <= Q; ++P) D[q++] = D[P] + D[Q];
}
void launch_jacobi(cudaStream_t, int64_t n, const double* t, const double* om, const double* D,
                   double* out) {
  for (int64_t k = 0; k < n; ++k) out[k] = t[k] - om[k] / D[k];
}
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
void launch_ritz_residual(cudaStream_t, int nr, int64_t n, const double* ax, const double* x,
                          const double* wr, const int* order, double* r) {
  for (int k = 0; k < nr; ++k)
    for (int64_t e = 0; e < n; ++e)
      r[(int64_t)k * n + e] = ax[(int64_t)k * n + e] - wr[order[k]] * x[(int64_t)k * n + e];
}
}
// The solver reads small results (info flags, root order, eigenvalues) with
// cudaMemcpyAsync; in the test double all "device" memory is host memory.
extern "C" cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t count,
                                       cudaMemcpyKind, cudaStream_t) {
  std::memmove(dst, src, count);
  return cudaSuccess;
}
extern "C" long long sccsd_gemm_tn_noalloc_capacity(void) { return 0; }
extern "C" int sccsd_gemm_tn_noalloc(long long, long long, long long, double, const double*, const double*, double*, void*) { return -1; }
namespace sccsd {
void launch_learned_features(cudaStream_t, int, int, const double*, const double*, const double*, const double*, double, double, double, float*) { no_device(); }
void launch_learned_targets(cudaStream_t, int, int, const double*, const double*, const double*, double, float*) { no_device(); }
void launch_learned_apply(cudaStream_t, int, int, const float*, const double*, double, double*, double*) { no_device(); }
}
extern "C" int sccsd_mlp_forward(struct sccsd_mlp*, const float*, long long, float*) { return -5; }
