// Device backend used by the graph executor. Every method launches kernels
// of this library on the context's CUDA stream; there is no host path.
#pragma once

#include <cstdint>
#include <stdexcept>

namespace sccsd {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct OomError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

class Graph;

// A strided (batch, row, k) matrix view of a tensor: element (b, r, k) is at
// p + b*sb + R(r) + K(k), with R(r) = (r / n2r) * sr1 + (r % n2r) * sr2 when
// n2r > 0 and R(r) = r * sr2 otherwise (K(k) likewise with n2k, sk1, sk2).
struct MatView {
  const double* p = nullptr;
  int64_t sb = 0;
  int64_t n2r = 0, sr1 = 0, sr2 = 0;
  int64_t n2k = 0, sk1 = 0, sk2 = 1;
  static MatView dense(const double* p, int64_t rows, int64_t K) {
    MatView v;
    v.p = p;
    v.sb = rows * K;
    v.sr2 = K;
    v.sk2 = 1;
    return v;
  }
};

// Output of a contraction as a strided multi-level view: the row index m of
// the M x N result is split into levels (outermost first) of extents re[] and
// strides rs[], i.e. row(m) = sum_l digit_l(m) * rs[l] with the digits of m
// in the mixed radix re[] (the outermost extent is not needed); the same for
// the column index n. Element (m, n) lives at C + row(m) + col(n), so that
// any permuted output layout is written directly by the GEMM epilogue.
constexpr int kOutLevels = 6;
struct OutView {
  int nr = 1, nc = 1;
  int64_t re[kOutLevels] = {0}, rs[kOutLevels] = {0};
  int64_t ce[kOutLevels] = {0}, cs[kOutLevels] = {0};
  static OutView dense(int64_t ldc) {
    OutView v;
    v.rs[0] = ldc;
    v.cs[0] = 1;
    return v;
  }
};

class Backend {
 public:
  virtual ~Backend() {}
  virtual double* alloc(int64_t n) = 0;
  virtual void release(double* p) = 0;
  // dst (device, n doubles) <- src (host or device)
  virtual void upload(double* dst, const double* src, int64_t n, bool src_on_device) = 0;
  virtual void fill(double* p, int64_t n, double v) = 0;
  // dst (host or device) <- src (device)
  virtual void download(double* dst, const double* src, int64_t n, bool dst_on_device) = 0;
  // true when p is a device (or managed) pointer usable by kernels
  virtual bool is_device(const void* p) = 0;
  virtual void sync() = 0;
  virtual void* stream() = 0;
  // Precision of the tensor-core-eligible contractions from now on
  // (SCCSD_FP64 / SCCSD_BF16X3 / SCCSD_BF16); cached operands are dropped.
  virtual void set_precision(int p) = 0;
  virtual int get_precision() const = 0;
  // While capturing a CUDA graph: no synchronisation, no allocation.
  virtual void set_capturing(bool on) = 0;
  // time the launch-shape candidates of each new tensor-core contraction shape
  // (no effect in FP64 mode)
  virtual void set_autotune(bool on) { (void)on; }
  // packed singles+doubles vector <-> t1[a][i], full t2[i][j][a][b].
  // ket: t2 = t_mu on both (P,Q) and (Q,P);  bra: off-diagonal pairs halved
  // on unpack and summed on pack, so that sum_packed L X = sum_full L~ X.
  virtual void unpack(const double* x, int o, int v, double* t1, double* t2, bool bra) = 0;
  virtual void pack(const double* t1, const double* t2, int o, int v, double* x, bool bra) = 0;
  // out[i] (+)= coef * in[i] over a rank-r index box; both sides strided.
  virtual void copy_view(int rank, const int64_t* dims, double* out, const int64_t* ostr,
                         const double* in, const int64_t* istr, double coef, bool accumulate) = 0;
  // out[i] (+)= coef * a[i] * b[i] over a rank-r index box, all three strided
  // (a stride 0 broadcasts): contractions with no contracted index.
  virtual void mul_view(int rank, const int64_t* dims, double* out, const int64_t* ostr,
                        const double* a, const int64_t* astr, const double* b,
                        const int64_t* bstr, double coef, bool accumulate) = 0;
  // C[b][m][n] = alpha * sum_k A(b,m,k) B(b,n,k); C dense and overwritten.
  // tc: the contraction may use tensor cores when the precision mode allows.
  virtual void gemm_view(int64_t batch, int64_t M, int64_t N, int64_t K, double alpha,
                         const MatView& A, const MatView& B, double* C, bool tc) = 0;
  void gemm_tn(int64_t batch, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
               const double* B, double* C, bool tc) {
    gemm_view(batch, M, N, K, alpha, MatView::dense(A, M, K), MatView::dense(B, N, K), C, tc);
  }
  // Pool of recyclable device buffers keyed by exact size.
  virtual double* pool_get(int64_t n) = 0;
  virtual void pool_put(double* p, int64_t n) = 0;
  // Tensor-core routing with a cache of converted operands. A key names an
  // operand (graph, node, layout) at a version; the backend keeps its
  // tensor-core form and reuses it while the version is unchanged.
  struct OperandKey {
    const void* graph;
    int id;
    int64_t version;
    uint64_t layout;
  };
  virtual bool tc_will_use(int64_t nb, int64_t M, int64_t N, int64_t K) = 0;
  virtual bool tc_cached(const OperandKey& k) = 0;
  // A.p or B.p may be NULL when its key is cached.
  // ov == NULL: C dense [M][N]. accumulate: C += alpha A B^T.
  virtual void gemm_tc_keyed(int64_t M, int64_t N, int64_t K, double alpha, const MatView& A,
                             const OperandKey* ka, const MatView& B, const OperandKey* kb,
                             double* C, const OutView* ov = nullptr, bool accumulate = false) = 0;
  // Reusable temporary device buffers (slot 0..7), grown on demand.
  virtual double* scratch(int slot, int64_t n) = 0;
  // Particle-particle ladder with the vv block of L (see Graph::ladder).
  // rows = number of (ij) rows of X, o^2 times the batch size
  virtual void ladder(const Graph& g, const double* L, int64_t L_version, const double* X,
                      double* Y, int64_t rows) = 0;
  // Profiling: CUDA-event timing of the ladder contractions and a count of
  // kernel launches since the last reset.
  virtual void profile(bool enable) = 0;
  // Per-operation tracing support: record an event on the stream, and the
  // elapsed milliseconds between two recorded events (synchronises).
  virtual void* record_event() = 0;
  virtual double elapsed_ms(void* a, void* b) = 0;
  virtual void profile_read(double* ladder_ms, long long* ladder_calls, double* ladder_flops,
                            long long* launches) = 0;
  virtual void ladder_adj_l(const Graph& g, const double* L, const double* Ybar,
                            const double* X, double* out) = 0;
};

}  // namespace sccsd
