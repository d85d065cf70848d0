// CUDA backend of the graph executor: FP64 kernels for strided copies,
// packing, reductions and contractions, plus dispatch of tensor-core
// eligible contractions to the tcgen05 path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "backend.h"
#include "graph.h"
#include "tc_gemm.h"

namespace sccsd {

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      throw CudaError(std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

static void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
}

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

// ------------------------------------------------------------------ copies

struct ViewArgs {
  int rank;
  int64_t dims[kMaxRank];
  int64_t ostr[kMaxRank];
  int64_t istr[kMaxRank];
};

__global__ void k_copy_view(ViewArgs a, int64_t total, double* __restrict__ out,
                            const double* __restrict__ in, double coef, int acc) {
  for (int64_t lin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lin < total;
       lin += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = lin, oo = 0, ii = 0;
    for (int k = a.rank - 1; k >= 0; --k) {
      int64_t c = r % a.dims[k];
      r /= a.dims[k];
      oo += c * a.ostr[k];
      ii += c * a.istr[k];
    }
    double v = coef * in[ii];
    out[oo] = acc ? out[oo] + v : v;
  }
}

// 32x32 shared-memory tile transpose for copies whose fastest output index is
// strided in the input while another output index is contiguous in the input.
// Tile axes: x = output dim px (unit output stride), y = output dim py (unit
// input stride); the remaining dims are walked by blockIdx.z.
struct TransArgs {
  int rank, px, py;
  int64_t dims[kMaxRank];
  int64_t ostr[kMaxRank];
  int64_t istr[kMaxRank];
  int64_t rest_total;
};

__global__ void k_copy_transpose(TransArgs a, double* __restrict__ out,
                                 const double* __restrict__ in, double coef, int acc) {
  __shared__ double tile[32][33];
  const int64_t nx = a.dims[a.px], ny = a.dims[a.py];
  for (int64_t rest = blockIdx.z; rest < a.rest_total; rest += gridDim.z) {
    int64_t r = rest, ob = 0, ib = 0;
    for (int k = a.rank - 1; k >= 0; --k) {
      if (k == a.px || k == a.py) continue;
      int64_t c = r % a.dims[k];
      r /= a.dims[k];
      ob += c * a.ostr[k];
      ib += c * a.istr[k];
    }
    const int64_t x0 = (int64_t)blockIdx.x * 32, y0 = (int64_t)blockIdx.y * 32;
    // read: consecutive threads walk the input-contiguous dim (py)
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      int64_t x = x0 + j, y = y0 + threadIdx.x;
      if (x < nx && y < ny) tile[j][threadIdx.x] = in[ib + x * a.istr[a.px] + y * a.istr[a.py]];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      int64_t y = y0 + j, x = x0 + threadIdx.x;
      if (x < nx && y < ny) {
        int64_t oo = ob + x * a.ostr[a.px] + y * a.ostr[a.py];
        double v = coef * tile[threadIdx.x][j];
        out[oo] = acc ? out[oo] + v : v;
      }
    }
    __syncthreads();
  }
}

__global__ void k_fill(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ------------------------------------------------------------------ packing

__global__ void k_unpack(const double* __restrict__ x, int o, int v, double* __restrict__ t1,
                         double* __restrict__ t2, int bra) {
  const int64_t ov = (int64_t)o * v;
  const int64_t total = ov * ov;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    // e indexes t2[i][j][a][b]
    int64_t b = e % v, r = e / v;
    int64_t a = r % v;
    r /= v;
    int64_t j = r % o, i = r / o;
    int64_t P = a * o + i, Q = b * o + j;
    int64_t lo = P < Q ? P : Q, hi = P < Q ? Q : P;
    double val = x[ov + hi * (hi + 1) / 2 + lo];
    if (bra && P != Q) val *= 0.5;
    t2[e] = val;
    if (e < ov) t1[e] = x[e];
  }
}

__global__ void k_pack(const double* __restrict__ t1, const double* __restrict__ t2, int o, int v,
                       double* __restrict__ x, int bra) {
  const int64_t ov = (int64_t)o * v;
  const int64_t np = ov * (ov + 1) / 2;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < np + ov;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < ov) {
      x[k] = t1[k];
      continue;
    }
    int64_t q = k - ov;
    // Q = largest with Q(Q+1)/2 <= q
    int64_t Q = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while (Q * (Q + 1) / 2 > q) --Q;
    while ((Q + 1) * (Q + 2) / 2 <= q) ++Q;
    int64_t P = q - Q * (Q + 1) / 2;
    int64_t a = P / o, i = P % o, b = Q / o, j = Q % o;
    double val = t2[((i * o + j) * v + a) * v + b];
    if (bra && P != Q) val += t2[((j * o + i) * v + b) * v + a];
    x[k] = val;
  }
}

// ------------------------------------------------------------------ FP64 GEMM

// C[b][m][n] = alpha * sum_k A[b][m][k] B[b][n][k], FP64 on CUDA cores.
// 64x64 output tile per block, 256 threads with a 4x4 register tile each.
constexpr int DBM = 64, DBN = 64, DBK = 16;

__global__ void __launch_bounds__(256) k_dgemm_tn(int64_t M, int64_t N, int64_t K, double alpha,
                                                  const double* __restrict__ A,
                                                  const double* __restrict__ B,
                                                  double* __restrict__ C) {
  __shared__ double As[DBK][DBM + 1];
  __shared__ double Bs[DBK][DBN + 1];
  const int64_t bz = blockIdx.z;
  A += bz * M * K;
  B += bz * N * K;
  C += bz * M * N;
  const int64_t m0 = (int64_t)blockIdx.y * DBM, n0 = (int64_t)blockIdx.x * DBN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += DBK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int row = e >> 4, kk = e & 15;
      int64_t gk = k0 + kk;
      int64_t gm = m0 + row, gn = n0 + row;
      As[kk][row] = (gm < M && gk < K) ? A[gm * K + gk] : 0.0;
      Bs[kk][row] = (gn < N && gk < K) ? B[gn * K + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn < N) C[gm * N + gn] = alpha * acc[i][j];
    }
  }
}

// Split-K dot products for outputs with few elements: partial sums per
// (output, chunk), then a fixed-order final sum (deterministic).
__global__ void k_dot_partial(int64_t M, int64_t N, int64_t K, const double* __restrict__ A,
                              const double* __restrict__ B, int64_t chunk, int chunks,
                              double* __restrict__ part) {
  const int64_t oidx = blockIdx.y;  // b*M*N + m*N + n
  const int64_t n = oidx % N, bm = oidx / N;
  const int64_t m = bm % M, b = bm / M;
  const double* a = A + (b * M + m) * K;
  const double* bb = B + (b * N + n) * K;
  const int64_t k0 = (int64_t)blockIdx.x * chunk, k1 = (K < k0 + chunk) ? K : k0 + chunk;
  double s = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) s = fma(a[k], bb[k], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) part[oidx * chunks + blockIdx.x] = s;
  }
}

__global__ void k_dot_final(int64_t outs, int chunks, const double* __restrict__ part, double alpha,
                            double* __restrict__ C) {
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= outs) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[o * chunks + c];
  C[o] = alpha * s;
}

// ------------------------------------------------------------------ backend

class CudaBackend : public Backend {
 public:
  cudaStream_t st;
  int precision;
  std::vector<double*> slots = std::vector<double*>(8, nullptr);
  std::vector<int64_t> slot_n = std::vector<int64_t>(8, 0);
  // ladder integrals G[(ab)][(cd)] = sum_J L^J_ac L^J_bd (FP64), and the
  // tensor-core operand form when a mixed precision mode is active
  double* G = nullptr;
  int64_t G_version = -1;
  const double* G_src = nullptr;
  std::unique_ptr<TcGemm> tc;
  TcOperand G_tc;

  CudaBackend(void* stream, int prec) : st((cudaStream_t)stream), precision(prec) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (precision != 0) tc = std::make_unique<TcGemm>(st, precision);
  }
  ~CudaBackend() override {
    for (double* p : slots)
      if (p) cudaFree(p);
    if (G) cudaFree(G);
    tc.reset();
  }

  double* alloc(int64_t n) override {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(double) * std::max<int64_t>(1, n));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw OomError("cudaMalloc of " + std::to_string(n * 8) + " bytes failed");
    }
    return (double*)p;
  }
  void release(double* p) override { cudaFree(p); }
  void upload(double* d, const double* s, int64_t n, bool src_dev) override {
    if (n <= 0) return;
    CK(cudaMemcpyAsync(d, s, sizeof(double) * n,
                       src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (!src_dev) CK(cudaStreamSynchronize(st));
  }
  void download(double* d, const double* s, int64_t n, bool dst_dev) override {
    if (n <= 0) return;
    CK(cudaMemcpyAsync(d, s, sizeof(double) * n,
                       dst_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!dst_dev) CK(cudaStreamSynchronize(st));
  }
  bool is_device(const void* p) override {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  }
  void sync() override { CK(cudaStreamSynchronize(st)); }
  void fill(double* p, int64_t n, double v) override {
    if (n <= 0) return;
    k_fill<<<grid_for(n, 256), 256, 0, st>>>(p, n, v);
    check_launch("fill");
  }
  void unpack(const double* x, int o, int v, double* t1, double* t2, bool bra) override {
    int64_t total = (int64_t)o * v * o * v;
    k_unpack<<<grid_for(total, 256), 256, 0, st>>>(x, o, v, t1, t2, bra ? 1 : 0);
    check_launch("unpack");
  }
  void pack(const double* t1, const double* t2, int o, int v, double* x, bool bra) override {
    int64_t ov = (int64_t)o * v;
    int64_t total = ov + ov * (ov + 1) / 2;
    k_pack<<<grid_for(total, 256), 256, 0, st>>>(t1, t2, o, v, x, bra ? 1 : 0);
    check_launch("pack");
  }

  void copy_view(int rank, const int64_t* dims, double* out, const int64_t* ostr, const double* in,
                 const int64_t* istr, double coef, bool acc) override {
    // merge adjacent dims that are contiguous on both sides; drop unit dims
    int64_t d[kMaxRank], os[kMaxRank], is[kMaxRank];
    int r = 0;
    int64_t total = 1;
    for (int k = 0; k < rank; ++k) {
      total *= dims[k];
      if (dims[k] == 1) continue;
      if (r > 0 && os[r - 1] == ostr[k] * dims[k] && is[r - 1] == istr[k] * dims[k]) {
        d[r - 1] *= dims[k];
        os[r - 1] = ostr[k];
        is[r - 1] = istr[k];
        continue;
      }
      d[r] = dims[k];
      os[r] = ostr[k];
      is[r] = istr[k];
      ++r;
    }
    if (total == 0) return;
    // transposing copy: fastest output dim not unit-stride in the input but
    // some other dim is
    int px = -1, py = -1;
    if (r >= 2 && os[r - 1] == 1 && is[r - 1] != 1) {
      for (int k = 0; k < r - 1; ++k)
        if (is[k] == 1) py = k;
      px = r - 1;
    }
    if (py >= 0 && d[px] >= 8 && d[py] >= 8) {
      TransArgs a;
      a.rank = r;
      a.px = px;
      a.py = py;
      a.rest_total = 1;
      for (int k = 0; k < r; ++k) {
        a.dims[k] = d[k];
        a.ostr[k] = os[k];
        a.istr[k] = is[k];
        if (k != px && k != py) a.rest_total *= d[k];
      }
      dim3 grid((unsigned)((d[px] + 31) / 32), (unsigned)((d[py] + 31) / 32),
                (unsigned)std::min<int64_t>(a.rest_total, 65535));
      k_copy_transpose<<<grid, dim3(32, 8), 0, st>>>(a, out, in, coef, acc ? 1 : 0);
      check_launch("copy_transpose");
      return;
    }
    ViewArgs a;
    a.rank = r;
    for (int k = 0; k < r; ++k) {
      a.dims[k] = d[k];
      a.ostr[k] = os[k];
      a.istr[k] = is[k];
    }
    k_copy_view<<<grid_for(total, 256), 256, 0, st>>>(a, total, out, in, coef, acc ? 1 : 0);
    check_launch("copy_view");
  }

  void dgemm(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
             const double* B, double* C) {
    if (nb * M * N == 0) return;
    if (K == 0) {
      fill(C, nb * M * N, 0.0);
      return;
    }
    if (nb * M * N <= 64 && K >= 4096) {
      int chunks = (int)std::min<int64_t>(256, (K + 8191) / 8192);
      int64_t chunk = (K + chunks - 1) / chunks;
      double* part = scratch(7, nb * M * N * chunks);
      k_dot_partial<<<dim3(chunks, (unsigned)(nb * M * N)), 256, 0, st>>>(M, N, K, A, B, chunk,
                                                                          chunks, part);
      check_launch("dot_partial");
      k_dot_final<<<(unsigned)((nb * M * N + 127) / 128), 128, 0, st>>>(nb * M * N, chunks, part,
                                                                       alpha, C);
      check_launch("dot_final");
      return;
    }
    for (int64_t b0 = 0; b0 < nb; b0 += 65535) {
      int64_t bc = std::min<int64_t>(65535, nb - b0);
      for (int64_t m0 = 0; m0 < M; m0 += 65535LL * DBM) {
        int64_t mc = std::min<int64_t>(65535LL * DBM, M - m0);
        dim3 grid((unsigned)((N + DBN - 1) / DBN), (unsigned)((mc + DBM - 1) / DBM), (unsigned)bc);
        if (nb == 1) {
          k_dgemm_tn<<<grid, 256, 0, st>>>(mc, N, K, alpha, A + m0 * K, B, C + m0 * N);
        } else {
          if (m0 != 0) throw std::runtime_error("batched GEMM with huge M");
          k_dgemm_tn<<<grid, 256, 0, st>>>(M, N, K, alpha, A + b0 * M * K, B + b0 * N * K,
                                           C + b0 * M * N);
        }
        check_launch("dgemm");
      }
    }
  }

  void gemm_tn(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
               const double* B, double* C, bool use_tc) override {
    if (use_tc && tc && tc->worthwhile(nb, M, N, K)) {
      tc->gemm(nb, M, N, K, alpha, A, B, C);
      return;
    }
    dgemm(nb, M, N, K, alpha, A, B, C);
  }

  double* scratch(int slot, int64_t n) override {
    if (slot_n[slot] < n) {
      if (slots[slot]) {
        CK(cudaStreamSynchronize(st));
        cudaFree(slots[slot]);
        slots[slot] = nullptr;
      }
      slots[slot] = alloc(n);
      slot_n[slot] = n;
    }
    return slots[slot];
  }

  // G[(ab)][(cd)] = sum_J L^J_ac L^J_bd over the virtual block of L
  void build_ladder_integrals(const Graph& g, const double* L) {
    const int64_t o = g.o, v = g.v, J = g.J, n = o + v, vv = v * v;
    // Lt[(ac)][J] = L[J][o+a][o+c]
    double* Lt = scratch(3, vv * J);
    {
      int64_t dims[3] = {v, v, J};
      int64_t ostr[3] = {v * J, J, 1};
      int64_t istr[3] = {n, 1, n * n};
      copy_view(3, dims, Lt, ostr, L + o * n + o, istr, 1.0, false);
    }
    if (!G) G = alloc(vv * vv);
    double* Gp = scratch(4, vv * vv);  // Gp[(ac)][(bd)]
    dgemm(1, vv, vv, J, 1.0, Lt, Lt, Gp);
    // G[a][b][c][d] = Gp[a][c][b][d]
    int64_t dims[4] = {v, v, v, v};
    int64_t ostr[4] = {v * vv, vv, v, 1};
    int64_t istr[4] = {v * vv, v, vv, 1};
    copy_view(4, dims, G, ostr, Gp, istr, 1.0, false);
    if (tc) tc->prepare_operand(G, vv, vv, G_tc);
  }

  void ladder(const Graph& g, const double* L, int64_t ver, const double* X, double* Y) override {
    if (!G || ver != G_version || L != G_src) {
      build_ladder_integrals(g, L);
      G_version = ver;
      G_src = L;
    }
    const int64_t o = g.o, v = g.v, vv = v * v;
    // Y[(ij)][(ab)] = sum_(cd) X[(ij)][(cd)] G[(ab)][(cd)]
    if (tc && precision != 0) {
      tc->gemm_prepared_b(o * o, vv, vv, 1.0, X, G_tc, Y);
      return;
    }
    dgemm(1, o * o, vv, vv, 1.0, X, G, Y);
  }

  void ladder_adj_l(const Graph& g, const double* L, const double* Yb, const double* X,
                    double* out) override {
    const int64_t o = g.o, v = g.v, J = g.J, n = o + v, vv = v * v, oo = o * o;
    // D[(ab)][(cd)] = sum_ij Yb[(ij)][(ab)] X[(ij)][(cd)]
    double* YT = scratch(3, vv * oo);
    double* XT = scratch(5, vv * oo);
    {
      int64_t dims[2] = {vv, oo}, ostr[2] = {oo, 1}, istr[2] = {1, vv};
      copy_view(2, dims, YT, ostr, Yb, istr, 1.0, false);
      copy_view(2, dims, XT, ostr, X, istr, 1.0, false);
    }
    double* D = scratch(4, vv * vv);
    gemm_tn(1, vv, vv, oo, 1.0, YT, XT, D, true);
    // M2[(ac)][(bd)] = D[(ab)][(cd)] + D[(ba)][(dc)]
    double* M2 = scratch(6, vv * vv);
    {
      int64_t dims[4] = {v, v, v, v};  // a c b d
      int64_t ostr[4] = {v * vv, vv, v, 1};
      int64_t i1[4] = {v * vv, v, vv, 1};  // D[a][b][c][d]
      int64_t i2[4] = {vv, 1, v * vv, v};  // D[b][a][d][c]
      copy_view(4, dims, M2, ostr, D, i1, 1.0, false);
      copy_view(4, dims, M2, ostr, D, i2, 1.0, true);
    }
    // out'[(ac)][J] = sum_(bd) M2[(ac)][(bd)] Lvv[J][(bd)]
    double* Lvv = scratch(5, J * vv);
    {
      int64_t dims[3] = {J, v, v}, ostr[3] = {vv, v, 1}, istr[3] = {n * n, n, 1};
      copy_view(3, dims, Lvv, ostr, L + o * n + o, istr, 1.0, false);
    }
    double* op = scratch(3, vv * J);
    gemm_tn(1, vv, J, vv, 1.0, M2, Lvv, op, true);
    int64_t dims[2] = {J, vv}, ostr[2] = {vv, 1}, istr[2] = {1, J};
    copy_view(2, dims, out, ostr, op, istr, 1.0, false);
  }
};

std::unique_ptr<Backend> make_backend(void* stream, int precision) {
  return std::make_unique<CudaBackend>(stream, precision);
}

}  // namespace sccsd
