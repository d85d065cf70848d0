// Learned initial guess / preconditioner: a small MLP with BF16 weights and
// activations, FP32 accumulation, trained and evaluated by these kernels.
//
// Network: x[F] -> (Linear + ReLU) x L_hidden -> Linear -> y[n_out].
// Loss: mean squared error over all outputs.
//
// Every layer product runs on the tensor cores (tcgen05 through
// TcGemm::mlp_gemm) with the elementwise work of the layer fused into the
// product's epilogue. With A_0 = x, Z_l = A_l W_l + b_l and G_l = dLoss/dZ_l:
//   forward   A_{l+1} = relu(Z_l), written as BF16 [rows][in] and, when
//             training, transposed [in][rows]; Y = Z_L in FP32
//   backward  G_L = dLoss/dY; G_{l-1} = (G_l W_l^T) * [A_l > 0] (BF16, both
//             layouts); dW_l = A_l^T G_l, a contraction over the rows split
//             across CTAs (FP32 partial sums, then reduced); db_l = sum_rows G_l
// Storage: FP32 master weights W_l [in][out] with the Adam moments; BF16
// copies Wt_l [out][in] (the forward operand) and Wk_l [in][out] (the
// backward operand), rows padded to 256 and the contraction index to 64,
// padding zero.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/sccsd.h"
#include "tc_gemm.h"

namespace {

int64_t up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint16_t u) {
  return __bfloat162float(__ushort_as_bfloat16(u));
}

// A[n][k] = bf16(X[n][k]) for k < n_in, 0 for n_in <= k < lda; when AT is
// given also AT[k][n] for n < N, and zeros for N <= n < max(N, 64) (the
// contraction over rows reads whole blocks of 64 there)
__global__ void k_input(int64_t N, int n_in, const float* __restrict__ X, uint16_t* A,
                        int64_t lda, uint16_t* AT, int64_t ldt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * lda; e += stride) {
    const int64_t n = e / lda, k = e % lda;
    const uint16_t b = k < n_in ? bf16_bits(X[n * n_in + k]) : (uint16_t)0;
    A[e] = b;
    if (AT && k < n_in) AT[k * ldt + n] = b;
  }
  if (AT) {
    const int64_t tail = N < 64 ? 64 - N : 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tail * n_in; e += stride)
      AT[(e / tail) * ldt + N + e % tail] = 0;
  }
}

// MSE: G[n][c] = 2 (Y - T) / (N n_out) as BF16 (zeros for n_out <= c < ldg),
// GT[c][n] likewise (zeros for N <= n < max(N, 64)); loss accumulated atomically
__global__ void k_mse(int64_t N, int n_out, const float* __restrict__ Y, const float* __restrict__ T,
                      uint16_t* G, int64_t ldg, uint16_t* GT, int64_t ldt, float* loss) {
  float s = 0.f;
  const float inv = 1.f / (float)(N * n_out);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * ldg; e += stride) {
    const int64_t n = e / ldg, c = e % ldg;
    uint16_t b = 0;
    if (c < n_out) {
      const float d = Y[n * n_out + c] - T[n * n_out + c];
      s += d * d * inv;
      b = bf16_bits(2.f * d * inv);
      GT[c * ldt + n] = b;
    }
    G[e] = b;
  }
  const int64_t tail = N < 64 ? 64 - N : 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tail * n_out; e += stride)
    GT[(e / tail) * ldt + N + e % tail] = 0;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

// db[c] = sum_{n < N} GT[c][n]
__global__ void k_rowsum(int64_t N, int rows, const uint16_t* __restrict__ GT, int64_t ldt,
                         float* db) {
  __shared__ float ws[32];
  for (int c = blockIdx.x; c < rows; c += gridDim.x) {
    float s = 0.f;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s += bf16_val(GT[c * ldt + n]);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.f;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (threadIdx.x == 0) db[c] = s;
    }
    __syncthreads();
  }
}

// out[e] = sum_z part[z][e] (the split partial sums of a weight gradient)
__global__ void k_reduce(int splits, int64_t n, const float* __restrict__ part, float* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * n + e];
    out[e] = s;
  }
}

// BF16 operand copies of W [din][dout]: Wt[o][i] (ld ldt) and Wk[i][o] (ld ldk)
__device__ __forceinline__ void put_w(int64_t e, int dout, float w, uint16_t* Wt, int64_t ldt,
                                      uint16_t* Wk, int64_t ldk) {
  const int64_t i = e / dout, o = e % dout;
  const uint16_t b = bf16_bits(w);
  Wt[o * ldt + i] = b;
  Wk[i * ldk + o] = b;
}

__global__ void k_refresh(int din, int dout, const float* W, uint16_t* Wt, int64_t ldt,
                          uint16_t* Wk, int64_t ldk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)din * dout;
       e += (int64_t)gridDim.x * blockDim.x)
    put_w(e, dout, W[e], Wt, ldt, Wk, ldk);
}

// Adam on FP32 master parameters; refreshes the BF16 operand copies of a weight
// matrix (din > 0) or of nothing (biases: din = 0)
__global__ void k_adam(int64_t n, int din, int dout, float* w, const float* g, float* m1, float* m2,
                       float lr, float b1, float b2, float eps, float c1, float c2, uint16_t* Wt,
                       int64_t ldt, uint16_t* Wk, int64_t ldk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    float gg = g[e];
    m1[e] = b1 * m1[e] + (1.f - b1) * gg;
    m2[e] = b2 * m2[e] + (1.f - b2) * gg * gg;
    float mh = m1[e] / c1, vh = m2[e] / c2;
    w[e] -= lr * mh / (sqrtf(vh) + eps);
    if (din > 0) put_w(e, dout, w[e], Wt, ldt, Wk, ldk);
  }
}

int grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

void check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

struct sccsd_mlp {
  cudaStream_t st = nullptr;
  std::unique_ptr<sccsd::TcGemm> tc;
  int n_in = 0, hidden = 0, layers = 0, n_out = 0;  // layers = number of Linear layers
  std::vector<int> din, dout;
  std::vector<int64_t> din_p, dout_p, din_r, dout_r;  // padded to 64 (contraction) and 256 (rows)
  std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;   // FP32 master, grads, Adam moments
  std::vector<uint16_t*> Wt, Wk;                     // BF16 operand copies
  int64_t cap = 0;                                   // rows the work buffers hold (multiple of 256)
  bool cap_train = false;                            // transposed and gradient buffers present
  std::vector<uint16_t*> A, AT, G, GT;               // per layer: input activations, output grads
  float *Y = nullptr, *part = nullptr, *loss = nullptr;
  size_t part_floats = 0;
  int64_t step = 0;
  std::string err;
  void free_rows() {
    for (auto* v : {&A, &AT, &G, &GT}) {
      for (uint16_t* p : *v) cudaFree(p);
      v->clear();
    }
    cudaFree(Y);
    Y = nullptr;
    cap = 0;
    cap_train = false;
  }
  ~sccsd_mlp() {
    free_rows();
    for (auto* v : {&W, &b, &gW, &gb, &mW, &vW, &mb, &vb})
      for (float* p : *v) cudaFree(p);
    for (auto* v : {&Wt, &Wk})
      for (uint16_t* p : *v) cudaFree(p);
    cudaFree(part);
    cudaFree(loss);
  }
};

namespace {

void* zalloc(size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    throw std::runtime_error("mlp allocation failed");
  }
  if (cudaMemset(p, 0, std::max<size_t>(bytes, 16)) != cudaSuccess)
    throw std::runtime_error("mlp allocation failed");
  return p;
}
float* falloc(int64_t n) { return (float*)zalloc(sizeof(float) * (size_t)std::max<int64_t>(1, n)); }
uint16_t* halloc(int64_t n) { return (uint16_t*)zalloc(2 * (size_t)std::max<int64_t>(1, n)); }

// work buffers for N rows (transposed copies and gradients only for training)
void ensure_rows(sccsd_mlp* net, int64_t N, bool train) {
  if (N <= net->cap && (!train || net->cap_train)) return;
  const int64_t cap = std::max(up(std::max<int64_t>(N, 1), 256), net->cap);
  const bool tr = train || net->cap_train;
  cudaStreamSynchronize(net->st);
  net->free_rows();
  for (int l = 0; l < net->layers; ++l) {
    net->A.push_back(halloc(cap * net->din_p[l]));
    if (tr) {
      net->AT.push_back(halloc(net->din_r[l] * cap));
      net->G.push_back(halloc(cap * net->dout_p[l]));
      net->GT.push_back(halloc(net->dout_r[l] * cap));
    }
  }
  net->Y = falloc(cap * net->n_out);
  net->cap = cap;
  net->cap_train = tr;
}

// forward pass for N rows of X (FP32 features, device); output in net->Y
void forward(sccsd_mlp* net, const float* X, int64_t N, bool train) {
  ensure_rows(net, N, train);
  cudaStream_t st = net->st;
  const int64_t cap = net->cap;
  k_input<<<grid1(N * net->din_p[0]), 256, 0, st>>>(N, net->n_in, X, net->A[0], net->din_p[0],
                                                    train ? net->AT[0] : nullptr, cap);
  check("mlp input");
  for (int l = 0; l < net->layers; ++l) {
    const bool last = l == net->layers - 1;
    sccsd::MlpEpi e;
    e.bias = net->b[l];
    if (last) {
      e.outf = net->Y;
      e.ldf = net->n_out;
    } else {
      e.out = net->A[l + 1];
      e.ldo = net->din_p[l + 1];
      e.outT = train ? net->AT[l + 1] : nullptr;
      e.ldt = cap;
    }
    net->tc->mlp_gemm(last ? sccsd::MLP_OUTPUT : sccsd::MLP_HIDDEN, net->A[l], cap, net->din_p[l],
                      net->Wt[l], net->dout_r[l], net->din_p[l], N, net->dout[l], net->din[l], 1, e);
  }
}

// gradients of the MSE loss w.r.t. all parameters into gW/gb; returns loss
float backward(sccsd_mlp* net, const float* T, int64_t N) {
  cudaStream_t st = net->st;
  const int64_t cap = net->cap;
  const int L = net->layers;
  cudaMemsetAsync(net->loss, 0, sizeof(float), st);
  k_mse<<<grid1(N * net->dout_p[L - 1]), 256, 0, st>>>(N, net->n_out, net->Y, T, net->G[L - 1],
                                                      net->dout_p[L - 1], net->GT[L - 1], cap,
                                                      net->loss);
  check("mlp loss");
  for (int l = L - 1; l >= 0; --l) {
    // dW_l = A_l^T G_l: a contraction over the N rows, split across CTAs
    const int64_t base = ((net->din[l] + 127) / 128) * ((net->dout[l] + 255) / 256);
    const int want = (int)std::max<int64_t>(1, net->tc->sm_count() / base);
    const size_t need = (size_t)want * net->din[l] * net->dout[l];
    if (net->part_floats < need) {
      cudaStreamSynchronize(st);
      cudaFree(net->part);
      net->part = nullptr;
      net->part_floats = 0;
      net->part = falloc((int64_t)need);
      net->part_floats = need;
    }
    sccsd::MlpEpi ep;
    ep.outf = net->part;
    ep.ldf = net->dout[l];
    const int splits = net->tc->mlp_gemm(sccsd::MLP_PARTIAL, net->AT[l], net->din_r[l], cap,
                                         net->GT[l], net->dout_r[l], cap, net->din[l],
                                         net->dout[l], N, want, ep);
    const int64_t nw = (int64_t)net->din[l] * net->dout[l];
    k_reduce<<<grid1(nw), 256, 0, st>>>(splits, nw, net->part, net->gW[l]);
    k_rowsum<<<std::min(net->dout[l], 1024), 256, 0, st>>>(N, net->dout[l], net->GT[l], cap,
                                                          net->gb[l]);
    check("mlp weight gradient");
    if (l > 0) {
      // G_{l-1} = (G_l W_l^T) * [A_l > 0]
      sccsd::MlpEpi eb;
      eb.out = net->G[l - 1];
      eb.ldo = net->dout_p[l - 1];
      eb.outT = net->GT[l - 1];
      eb.ldt = cap;
      eb.maskT = net->AT[l];
      eb.ldm = cap;
      net->tc->mlp_gemm(sccsd::MLP_RELU_BACK, net->G[l], cap, net->dout_p[l], net->Wk[l],
                        net->din_r[l], net->dout_p[l], N, net->din[l], net->dout[l], 1, eb);
    }
  }
  float h = 0.f;
  cudaMemcpyAsync(&h, net->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return h;
}

template <class F>
int mlp_guard(sccsd_mlp* net, F&& f) {
  try {
    f();
    cudaError_t e = cudaStreamSynchronize(net->st);
    if (e != cudaSuccess) throw std::runtime_error(cudaGetErrorString(e));
    if (net->tc) net->tc->check_error();
    return SCCSD_OK;
  } catch (const std::exception& e) {
    if (net) net->err = e.what();
    return SCCSD_ECUDA;
  }
}

void refresh(sccsd_mlp* net, int l) {
  k_refresh<<<grid1((int64_t)net->din[l] * net->dout[l]), 256, 0, net->st>>>(
      net->din[l], net->dout[l], net->W[l], net->Wt[l], net->din_p[l], net->Wk[l], net->dout_p[l]);
  check("mlp weights");
}

}  // namespace

extern "C" {

int sccsd_mlp_create(sccsd_mlp** out, int n_in, int hidden, int n_hidden_layers, int n_out,
                     unsigned long long seed, void* stream) {
  if (!out || n_in < 1 || hidden < 1 || n_hidden_layers < 0 || n_out < 1) return SCCSD_EINVAL;
  auto* net = new sccsd_mlp;
  net->st = (cudaStream_t)stream;
  net->n_in = n_in;
  net->hidden = hidden;
  net->layers = n_hidden_layers + 1;
  net->n_out = n_out;
  int rc = mlp_guard(net, [&] {
    // He-style initialisation from a simple counter-based generator
    // (splitmix64 -> uniform in [-s, s])
    uint64_t state = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
      uint64_t z = (state += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    net->tc.reset(new sccsd::TcGemm(net->st, 0));
    for (int l = 0; l < net->layers; ++l) {
      int din = l == 0 ? n_in : hidden;
      int dout = l == net->layers - 1 ? n_out : hidden;
      net->din.push_back(din);
      net->dout.push_back(dout);
      net->din_p.push_back(up(din, 64));
      net->dout_p.push_back(up(dout, 64));
      net->din_r.push_back(up(din, 256));
      net->dout_r.push_back(up(dout, 256));
      std::vector<float> w((size_t)din * dout);
      double s = std::sqrt(6.0 / din);
      for (auto& x : w) x = (float)((2.0 * next() - 1.0) * s);
      float* W = falloc((int64_t)din * dout);
      cudaMemcpy(W, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice);
      net->W.push_back(W);
      net->Wt.push_back(halloc(net->dout_r[l] * net->din_p[l]));
      net->Wk.push_back(halloc(net->din_r[l] * net->dout_p[l]));
      refresh(net, l);
      net->b.push_back(falloc(dout));
      net->gW.push_back(falloc((int64_t)din * dout));
      net->gb.push_back(falloc(dout));
      net->mW.push_back(falloc((int64_t)din * dout));
      net->vW.push_back(falloc((int64_t)din * dout));
      net->mb.push_back(falloc(dout));
      net->vb.push_back(falloc(dout));
    }
    net->loss = falloc(1);
  });
  if (rc != SCCSD_OK) {
    delete net;
    return rc;
  }
  *out = net;
  return SCCSD_OK;
}

void sccsd_mlp_destroy(sccsd_mlp* net) { delete net; }

const char* sccsd_mlp_last_error(sccsd_mlp* net) { return net ? net->err.c_str() : "no network"; }

long long sccsd_mlp_num_params(sccsd_mlp* net) {
  if (!net) return -1;
  long long n = 0;
  for (int l = 0; l < net->layers; ++l) n += (long long)net->din[l] * net->dout[l] + net->dout[l];
  return n;
}

// parameters as one FP32 array: per layer W[in][out] then b[out]
int sccsd_mlp_get_params(sccsd_mlp* net, float* host_out) {
  if (!net || !host_out) return SCCSD_EINVAL;
  return mlp_guard(net, [&] {
    int64_t off = 0;
    for (int l = 0; l < net->layers; ++l) {
      int64_t nw = (int64_t)net->din[l] * net->dout[l];
      cudaMemcpy(host_out + off, net->W[l], sizeof(float) * nw, cudaMemcpyDeviceToHost);
      off += nw;
      cudaMemcpy(host_out + off, net->b[l], sizeof(float) * net->dout[l], cudaMemcpyDeviceToHost);
      off += net->dout[l];
    }
  });
}

int sccsd_mlp_set_params(sccsd_mlp* net, const float* host_in) {
  if (!net || !host_in) return SCCSD_EINVAL;
  return mlp_guard(net, [&] {
    int64_t off = 0;
    for (int l = 0; l < net->layers; ++l) {
      int64_t nw = (int64_t)net->din[l] * net->dout[l];
      cudaMemcpy(net->W[l], host_in + off, sizeof(float) * nw, cudaMemcpyHostToDevice);
      refresh(net, l);
      off += nw;
      cudaMemcpy(net->b[l], host_in + off, sizeof(float) * net->dout[l], cudaMemcpyHostToDevice);
      off += net->dout[l];
    }
  });
}

// Y[N][n_out] = net(X[N][n_in]); X, Y device FP32
int sccsd_mlp_forward(sccsd_mlp* net, const float* X, long long N, float* Y) {
  if (!net || !X || !Y || N < 0) return SCCSD_EINVAL;
  return mlp_guard(net, [&] {
    if (N == 0) return;
    forward(net, X, N, false);
    cudaMemcpyAsync(Y, net->Y, sizeof(float) * N * net->n_out, cudaMemcpyDeviceToDevice, net->st);
  });
}

// gradient of the MSE loss at the current parameters (host FP32 array laid
// out like sccsd_mlp_get_params); loss in *loss
int sccsd_mlp_gradient(sccsd_mlp* net, const float* X, const float* T, long long N, float* grad,
                       float* loss) {
  if (!net || !X || !T || N < 1) return SCCSD_EINVAL;
  return mlp_guard(net, [&] {
    forward(net, X, N, true);
    float l = backward(net, T, N);
    if (loss) *loss = l;
    if (grad) {
      int64_t off = 0;
      for (int k = 0; k < net->layers; ++k) {
        int64_t nw = (int64_t)net->din[k] * net->dout[k];
        cudaMemcpy(grad + off, net->gW[k], sizeof(float) * nw, cudaMemcpyDeviceToHost);
        off += nw;
        cudaMemcpy(grad + off, net->gb[k], sizeof(float) * net->dout[k], cudaMemcpyDeviceToHost);
        off += net->dout[k];
      }
    }
  });
}

// one Adam step on the minibatch (X, T) of N rows; loss before the step in *loss
int sccsd_mlp_train_step(sccsd_mlp* net, const float* X, const float* T, long long N, float lr,
                         float* loss) {
  if (!net || !X || !T || N < 1 || !(lr > 0.f)) return SCCSD_EINVAL;
  return mlp_guard(net, [&] {
    forward(net, X, N, true);
    float l = backward(net, T, N);
    if (loss) *loss = l;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
    for (int k = 0; k < net->layers; ++k) {
      int64_t nw = (int64_t)net->din[k] * net->dout[k];
      k_adam<<<grid1(nw), 256, 0, net->st>>>(nw, net->din[k], net->dout[k], net->W[k], net->gW[k],
                                              net->mW[k], net->vW[k], lr, b1, b2, 1e-8f, c1, c2,
                                              net->Wt[k], net->din_p[k], net->Wk[k],
                                              net->dout_p[k]);
      k_adam<<<grid1(net->dout[k]), 256, 0, net->st>>>(net->dout[k], 0, net->dout[k], net->b[k],
                                                        net->gb[k], net->mb[k], net->vb[k], lr, b1,
                                                        b2, 1e-8f, c1, c2, nullptr, 0, nullptr, 0);
    }
    check("mlp adam");
  });
}

}  // extern "C"
