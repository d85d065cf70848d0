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

static long long g_launches = 0;  // kernel launches issued by this library

void count_launch() { ++g_launches; }
long long launch_count() { return g_launches; }

static void check_launch(const char* what) {
  ++g_launches;
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

// same with 32-bit index arithmetic (all extents and offsets below 2^31)
struct ViewArgs32 {
  int rank;
  uint32_t dims[kMaxRank];
  uint32_t ostr[kMaxRank];
  uint32_t istr[kMaxRank];
};

__global__ void k_copy_view32(ViewArgs32 a, uint32_t total, double* __restrict__ out,
                              const double* __restrict__ in, double coef, int acc) {
  for (uint32_t lin = blockIdx.x * blockDim.x + threadIdx.x; lin < total;
       lin += gridDim.x * blockDim.x) {
    uint32_t r = lin, oo = 0, ii = 0;
    for (int k = a.rank - 1; k >= 0; --k) {
      uint32_t c = r % a.dims[k];
      r /= a.dims[k];
      oo += c * a.ostr[k];
      ii += c * a.istr[k];
    }
    double v = coef * in[ii];
    out[oo] = acc ? out[oo] + v : v;
  }
}

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

// Split-K variant for outputs with few tiles: blockIdx.z selects a K chunk,
// part[z][m][n] receives the chunk's sum.
__global__ void __launch_bounds__(256) k_dgemm_splitk(int64_t M, int64_t N, int64_t K, int64_t kc,
                                                      const double* __restrict__ A,
                                                      const double* __restrict__ B,
                                                      double* __restrict__ part) {
  __shared__ double As[DBK][DBM + 1];
  __shared__ double Bs[DBK][DBN + 1];
  const int64_t kbeg = (int64_t)blockIdx.z * kc;
  const int64_t kend = (K < kbeg + kc) ? K : kbeg + kc;
  const int64_t m0 = (int64_t)blockIdx.y * DBM, n0 = (int64_t)blockIdx.x * DBN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += DBK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int row = e >> 4, kk = e & 15;
      int64_t gk = k0 + kk;
      int64_t gm = m0 + row, gn = n0 + row;
      As[kk][row] = (gm < M && gk < kend) ? A[gm * K + gk] : 0.0;
      Bs[kk][row] = (gn < N && gk < kend) ? B[gn * K + gk] : 0.0;
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
  double* P = part + (int64_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn < N) P[gm * N + gn] = acc[i][j];
    }
  }
}

// Outputs of at most 32 x 32 with a long contraction: 32x32 tile, K chunk per
// block (blockIdx.z), each thread 2x2 outputs; partial tiles go to part[z].
__global__ void __launch_bounds__(256) k_dgemm_small(int64_t M, int64_t N, int64_t K, int64_t kc,
                                                     const double* __restrict__ A,
                                                     const double* __restrict__ B,
                                                     double* __restrict__ part) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int64_t kbeg = (int64_t)blockIdx.z * kc;
  const int64_t kend = (K < kbeg + kc) ? K : kbeg + kc;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc00 = 0, acc01 = 0, acc10 = 0, acc11 = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int row = e >> 5, kk = e & 31;
      int64_t gk = k0 + kk;
      As[kk][row] = (row < M && gk < kend) ? A[row * K + gk] : 0.0;
      Bs[kk][row] = (row < N && gk < kend) ? B[row * K + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      double a0 = As[kk][ty], a1 = As[kk][ty + 16], b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc00 = fma(a0, b0, acc00);
      acc01 = fma(a0, b1, acc01);
      acc10 = fma(a1, b0, acc10);
      acc11 = fma(a1, b1, acc11);
    }
    __syncthreads();
  }
  double* P = part + (int64_t)blockIdx.z * M * N;
  if (ty < M && tx < N) P[ty * N + tx] = acc00;
  if (ty < M && tx + 16 < N) P[ty * N + tx + 16] = acc01;
  if (ty + 16 < M && tx < N) P[(ty + 16) * N + tx] = acc10;
  if (ty + 16 < M && tx + 16 < N) P[(ty + 16) * N + tx + 16] = acc11;
}

__global__ void k_sum_parts(int64_t n, int splits, const double* __restrict__ part, double alpha,
                            double* __restrict__ C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * n + e];
    C[e] = alpha * s;
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
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  double prof_ms = 0.0;
  long long prof_calls = 0, launches0 = 0;

  CudaBackend(void* stream, int prec) : st((cudaStream_t)stream), precision(prec) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (precision != 0) tc = std::make_unique<TcGemm>(st, precision);
  }
  ~CudaBackend() override {
    for (auto& e : ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
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
  void sync() override {
    CK(cudaStreamSynchronize(st));
    if (tc) tc->check_error();
  }
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
    int64_t omax = 0, imax = 0;
    for (int k = 0; k < r; ++k) {
      omax += (d[k] - 1) * os[k];
      imax += (d[k] - 1) * is[k];
    }
    if (total < (1LL << 31) && omax < (1LL << 31) && imax < (1LL << 31)) {
      ViewArgs32 a;
      a.rank = r;
      for (int k = 0; k < r; ++k) {
        a.dims[k] = (uint32_t)d[k];
        a.ostr[k] = (uint32_t)os[k];
        a.istr[k] = (uint32_t)is[k];
      }
      k_copy_view32<<<grid_for(total, 256), 256, 0, st>>>(a, (uint32_t)total, out, in, coef,
                                                           acc ? 1 : 0);
      check_launch("copy_view32");
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
    if (nb == 1 && M <= 32 && N <= 32 && K >= 4096) {
      int64_t splits = std::min<int64_t>(1216, (K + 1023) / 1024);
      int64_t kc = (K + splits - 1) / splits;
      kc = (kc + 31) / 32 * 32;
      splits = (K + kc - 1) / kc;
      double* part = scratch(7, splits * M * N);
      k_dgemm_small<<<dim3(1, 1, (unsigned)splits), 256, 0, st>>>(M, N, K, kc, A, B, part);
      check_launch("dgemm_small");
      k_sum_parts<<<grid_for(M * N, 256), 256, 0, st>>>(M * N, (int)splits, part, alpha, C);
      check_launch("sum_parts");
      return;
    }
    const int64_t tiles = nb * ((M + DBM - 1) / DBM) * ((N + DBN - 1) / DBN);
    if (nb == 1 && tiles < 2 * 152 && K >= 4096) {
      // split K so that the grid fills the GPU; partial tiles are summed in a
      // fixed order afterwards (deterministic)
      int64_t splits = std::min<int64_t>((4 * 152 + tiles - 1) / tiles, K / 1024);
      splits = std::max<int64_t>(2, std::min<int64_t>(splits, 64));
      int64_t kc = (K + splits - 1) / splits;
      kc = (kc + DBK - 1) / DBK * DBK;
      splits = (K + kc - 1) / kc;
      double* part = scratch(7, splits * M * N);
      dim3 grid((unsigned)((N + DBN - 1) / DBN), (unsigned)((M + DBM - 1) / DBM), (unsigned)splits);
      k_dgemm_splitk<<<grid, 256, 0, st>>>(M, N, K, kc, A, B, part);
      check_launch("dgemm_splitk");
      k_sum_parts<<<grid_for(M * N, 256), 256, 0, st>>>(M * N, (int)splits, part, alpha, C);
      check_launch("sum_parts");
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
    gemm_tn(1, vv, vv, J, 1.0, Lt, Lt, Gp, true);
    // G[a][b][c][d] = Gp[a][c][b][d]
    int64_t dims[4] = {v, v, v, v};
    int64_t ostr[4] = {v * vv, vv, v, 1};
    int64_t istr[4] = {v * vv, v, vv, 1};
    copy_view(4, dims, G, ostr, Gp, istr, 1.0, false);
    if (tc) tc->prepare_operand(G, vv, vv, G_tc);
  }

  void* record_event() override {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    CK(cudaEventRecord(e, st));
    return (void*)e;
  }
  double elapsed_ms(void* a, void* b) override {
    CK(cudaEventSynchronize((cudaEvent_t)b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, (cudaEvent_t)a, (cudaEvent_t)b));
    cudaEventDestroy((cudaEvent_t)a);
    cudaEventDestroy((cudaEvent_t)b);
    return ms;
  }

  void profile(bool enable) override {
    sync();
    for (auto& e : ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    ev.clear();
    prof = enable;
    prof_ms = 0.0;
    prof_calls = 0;
    launches0 = g_launches;
  }
  void profile_read(double* ms, long long* calls, long long* launches) override {
    sync();
    for (auto& e : ev) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e.first, e.second));
      prof_ms += t;
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    ev.clear();
    if (ms) *ms = prof_ms;
    if (calls) *calls = prof_calls;
    if (launches) *launches = g_launches - launches0;
  }

  void ladder(const Graph& g, const double* L, int64_t ver, const double* X, double* Y) override {
    if (!G || ver != G_version || L != G_src) {
      build_ladder_integrals(g, L);
      G_version = ver;
      G_src = L;
    }
    const int64_t o = g.o, v = g.v, vv = v * v;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      CK(cudaEventRecord(e0, st));
    }
    // Y[(ij)][(ab)] = sum_(cd) X[(ij)][(cd)] G[(ab)][(cd)]
    if (tc && precision != 0)
      tc->gemm_prepared_b(o * o, vv, vv, 1.0, X, G_tc, Y, !prof);
    else
      dgemm(1, o * o, vv, vv, 1.0, X, G, Y);
    if (prof) {
      CK(cudaEventRecord(e1, st));
      ev.push_back({e0, e1});
      ++prof_calls;
    }
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
