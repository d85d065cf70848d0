// Learned initial guess / preconditioner: a small MLP with BF16 weights and
// activations, FP32 accumulation, trained and evaluated by these kernels.
//
// Network: x[F] -> (Linear + ReLU) x L_hidden -> Linear -> y[n_out].
// Storage: weights W_l [in][out] BF16 (with FP32 master copies for Adam),
// biases FP32, activations BF16, pre-activations FP32 (kept for backward).
// Loss: mean squared error over all outputs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/sccsd.h"

namespace {

__device__ __forceinline__ float ld(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

// C[m][n] (+)= alpha * sum_k A(m,k) B(k,n), FP32 accumulation.
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], C row-major [M][N].
// blockIdx.z splits K into chunks of kc; with more than one chunk the
// results are added atomically (C must be zeroed first).
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gemm_f32(int64_t M, int64_t N, int64_t K, int64_t kc,
                                                  float alpha, const TA* __restrict__ A,
                                                  int64_t sam, int64_t sak,
                                                  const TB* __restrict__ B, int64_t sbk,
                                                  int64_t sbn, float* __restrict__ C,
                                                  int accumulate) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
  const int64_t kbeg = (int64_t)blockIdx.z * kc;
  const int64_t kend = (K < kbeg + kc) ? K : kbeg + kc;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      // A tile: rows fastest when sam == 1, else k fastest
      int r, kk;
      if (sam == 1) {
        r = e & 63;
        kk = e >> 6;
      } else {
        r = e >> 4;
        kk = e & 15;
      }
      int64_t gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < kend) ? ld(A, gm * sam + gk * sak) : 0.f;
      int c2, k2;
      if (sbn == 1) {
        c2 = e & 63;
        k2 = e >> 6;
      } else {
        c2 = e >> 4;
        k2 = e & 15;
      }
      int64_t gn = n0 + c2, gk2 = k0 + k2;
      Bs[k2][c2] = (gn < N && gk2 < kend) ? ld(B, gk2 * sbk + gn * sbn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool atomic = gridDim.z > 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float v = alpha * acc[i][j];
      float* p = C + gm * N + gn;
      if (atomic)
        atomicAdd(p, v);
      else
        *p = accumulate ? *p + v : v;
    }
  }
}

// Z[n][m] += b[m]; A = relu(Z) as BF16 (or Z copied to FP32 output for the last layer)
__global__ void k_bias_act(int64_t N, int64_t M, float* Z, const float* b, __nv_bfloat16* A,
                           float* Yout, int relu) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * M;
       e += (int64_t)gridDim.x * blockDim.x) {
    float z = Z[e] + b[e % M];
    Z[e] = z;
    if (relu)
      A[e] = __float2bfloat16(z > 0.f ? z : 0.f);
    else
      Yout[e] = z;
  }
}

// dZ = dA * relu'(Z) (in place on dA)
__global__ void k_relu_back(int64_t n, const float* Z, float* dA) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    if (Z[e] <= 0.f) dA[e] = 0.f;
}

// MSE: dY = 2 (Y - T) / (N * n_out); loss partials accumulated atomically
__global__ void k_mse(int64_t n, const float* Y, const float* T, float* dY, float* loss) {
  float s = 0.f;
  const float inv = 1.f / (float)n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    float d = Y[e] - T[e];
    dY[e] = 2.f * d * inv;
    s += d * d * inv;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

// db[m] = sum_n dZ[n][m]
__global__ void k_colsum(int64_t N, int64_t M, const float* dZ, float* db) {
  for (int64_t m = blockIdx.x; m < M; m += gridDim.x) {
    float s = 0.f;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) s += dZ[n * M + m];
    __shared__ float ws[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.f;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (threadIdx.x == 0) db[m] = s;
    }
    __syncthreads();
  }
}

// Adam on FP32 master weights; refreshes the BF16 copy
__global__ void k_adam(int64_t n, float* w, const float* g, float* m1, float* m2, float lr, float b1,
                       float b2, float eps, float c1, float c2, __nv_bfloat16* wb) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    float gg = g[e];
    m1[e] = b1 * m1[e] + (1.f - b1) * gg;
    m2[e] = b2 * m2[e] + (1.f - b2) * gg * gg;
    float mh = m1[e] / c1, vh = m2[e] / c2;
    w[e] -= lr * mh / (sqrtf(vh) + eps);
    if (wb) wb[e] = __float2bfloat16(w[e]);
  }
}

__global__ void k_to_bf16(int64_t n, const float* x, __nv_bfloat16* y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = __float2bfloat16(x[e]);
}

int grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

void check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename TA, typename TB>
void gemm(cudaStream_t st, int64_t M, int64_t N, int64_t K, float alpha, const TA* A, int64_t sam,
          int64_t sak, const TB* B, int64_t sbk, int64_t sbn, float* C, int accumulate,
          int64_t splits = 1) {
  if (M == 0 || N == 0) return;
  int64_t kc = (K + splits - 1) / splits;
  kc = (kc + 15) / 16 * 16;
  splits = (K + kc - 1) / kc;
  if (splits < 1) splits = 1;
  if (splits > 1 && !accumulate) cudaMemsetAsync(C, 0, sizeof(float) * M * N, st);
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), (unsigned)splits);
  k_gemm_f32<TA, TB><<<grid, 256, 0, st>>>(M, N, K, kc, alpha, A, sam, sak, B, sbk, sbn, C,
                                          accumulate);
  check("mlp gemm");
}

}  // namespace

struct sccsd_mlp {
  cudaStream_t st = nullptr;
  int n_in = 0, hidden = 0, layers = 0, n_out = 0;  // layers = number of Linear layers
  std::vector<int> din, dout;
  std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;   // FP32 master, grads, Adam moments
  std::vector<__nv_bfloat16*> Wb;                    // BF16 weights used by the kernels
  int64_t cap = 0;                                   // rows the work buffers hold
  std::vector<float*> Z;                             // pre-activations [cap][dout]
  std::vector<__nv_bfloat16*> Act;                   // activations [cap][din] (Act[0] = input)
  float *Y = nullptr, *dY = nullptr, *dA = nullptr, *dB = nullptr, *loss = nullptr;
  int64_t step = 0;
  std::string err;
  ~sccsd_mlp() {
    for (auto* v : {&W, &b, &gW, &gb, &mW, &vW, &mb, &vb, &Z})
      for (float* p : *v) cudaFree(p);
    for (auto* p : Wb) cudaFree(p);
    for (auto* p : Act) cudaFree(p);
    for (float* p : {Y, dY, dA, dB, loss}) cudaFree(p);
  }
};

namespace {

float* falloc(int64_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, sizeof(float) * std::max<int64_t>(1, n)) != cudaSuccess) {
    cudaGetLastError();
    throw std::runtime_error("mlp allocation failed");
  }
  cudaMemset(p, 0, sizeof(float) * std::max<int64_t>(1, n));
  return (float*)p;
}

__nv_bfloat16* balloc(int64_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, 2 * std::max<int64_t>(1, n)) != cudaSuccess) {
    cudaGetLastError();
    throw std::runtime_error("mlp allocation failed");
  }
  return (__nv_bfloat16*)p;
}

void ensure_rows(sccsd_mlp* net, int64_t N) {
  if (N <= net->cap) return;
  for (float* p : net->Z) cudaFree(p);
  for (auto* p : net->Act) cudaFree(p);
  for (float* p : {net->Y, net->dY, net->dA, net->dB}) cudaFree(p);
  net->Z.clear();
  net->Act.clear();
  int widest = net->n_in;
  for (int l = 0; l < net->layers; ++l) {
    net->Z.push_back(falloc(N * net->dout[l]));
    net->Act.push_back(balloc(N * net->din[l]));
    widest = std::max(widest, net->dout[l]);
  }
  net->Y = falloc(N * net->n_out);
  net->dY = falloc(N * net->n_out);
  net->dA = falloc(N * widest);
  net->dB = falloc(N * widest);
  net->cap = N;
}

// forward pass for N rows of X (FP32 features, device); output in net->Y
void forward(sccsd_mlp* net, const float* X, int64_t N) {
  ensure_rows(net, N);
  cudaStream_t st = net->st;
  k_to_bf16<<<grid1(N * net->n_in), 256, 0, st>>>(N * net->n_in, X, net->Act[0]);
  check("mlp input");
  for (int l = 0; l < net->layers; ++l) {
    const int K = net->din[l], M = net->dout[l];
    gemm(st, N, M, K, 1.f, net->Act[l], (int64_t)K, (int64_t)1, net->Wb[l], (int64_t)M,
         (int64_t)1, net->Z[l], 0);
    const bool last = l == net->layers - 1;
    k_bias_act<<<grid1(N * M), 256, 0, st>>>(N, M, net->Z[l], net->b[l],
                                               last ? nullptr : net->Act[l + 1],
                                               last ? net->Y : nullptr, last ? 0 : 1);
    check("mlp bias/act");
  }
}

// gradients of the MSE loss w.r.t. all parameters into gW/gb; returns loss
float backward(sccsd_mlp* net, const float* T, int64_t N) {
  cudaStream_t st = net->st;
  cudaMemsetAsync(net->loss, 0, sizeof(float), st);
  k_mse<<<grid1(N * net->n_out), 256, 0, st>>>(N * net->n_out, net->Y, T, net->dY, net->loss);
  check("mlp loss");
  float* g = net->dY;  // gradient w.r.t. Z of the current layer
  for (int l = net->layers - 1; l >= 0; --l) {
    const int K = net->din[l], M = net->dout[l];
    // dW = Act_l^T g  (K x M, reduction over N rows)
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(256, N / 2048));
    gemm(st, (int64_t)K, (int64_t)M, N, 1.f, net->Act[l], (int64_t)1, (int64_t)K, g, (int64_t)M,
         (int64_t)1, net->gW[l], 0, splits);
    k_colsum<<<std::min(M, 1024), 256, 0, st>>>(N, M, g, net->gb[l]);
    check("mlp db");
    if (l > 0) {
      // dAct_l = g W_l^T  (N x K), then through ReLU: multiply by [Z_{l-1} > 0]
      float* dst = (g == net->dA) ? net->dB : net->dA;
      gemm(st, N, (int64_t)K, (int64_t)M, 1.f, g, (int64_t)M, (int64_t)1, net->Wb[l], (int64_t)1,
           (int64_t)M, dst, 0);
      k_relu_back<<<grid1(N * K), 256, 0, st>>>(N * K, net->Z[l - 1], dst);
      check("mlp relu back");
      g = dst;
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
    return SCCSD_OK;
  } catch (const std::exception& e) {
    if (net) net->err = e.what();
    return SCCSD_ECUDA;
  }
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
    for (int l = 0; l < net->layers; ++l) {
      int din = l == 0 ? n_in : hidden;
      int dout = l == net->layers - 1 ? n_out : hidden;
      net->din.push_back(din);
      net->dout.push_back(dout);
      std::vector<float> w((size_t)din * dout);
      double s = std::sqrt(6.0 / din);
      for (auto& x : w) x = (float)((2.0 * next() - 1.0) * s);
      float* W = falloc((int64_t)din * dout);
      cudaMemcpy(W, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice);
      net->W.push_back(W);
      __nv_bfloat16* Wb = balloc((int64_t)din * dout);
      k_to_bf16<<<grid1(din * dout), 256, 0, net->st>>>((int64_t)din * dout, W, Wb);
      net->Wb.push_back(Wb);
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
      k_to_bf16<<<grid1(nw), 256, 0, net->st>>>(nw, net->W[l], net->Wb[l]);
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
    forward(net, X, N);
    cudaMemcpyAsync(Y, net->Y, sizeof(float) * N * net->n_out, cudaMemcpyDeviceToDevice, net->st);
  });
}

// gradient of the MSE loss at the current parameters (host FP32 array laid
// out like sccsd_mlp_get_params); loss in *loss
int sccsd_mlp_gradient(sccsd_mlp* net, const float* X, const float* T, long long N, float* grad,
                       float* loss) {
  if (!net || !X || !T || N < 1) return SCCSD_EINVAL;
  return mlp_guard(net, [&] {
    forward(net, X, N);
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
    forward(net, X, N);
    float l = backward(net, T, N);
    if (loss) *loss = l;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
    for (int k = 0; k < net->layers; ++k) {
      int64_t nw = (int64_t)net->din[k] * net->dout[k];
      k_adam<<<grid1(nw), 256, 0, net->st>>>(nw, net->W[k], net->gW[k], net->mW[k], net->vW[k], lr,
                                              b1, b2, 1e-8f, c1, c2, net->Wb[k]);
      k_adam<<<grid1(net->dout[k]), 256, 0, net->st>>>(net->dout[k], net->b[k], net->gb[k],
                                                        net->mb[k], net->vb[k], lr, b1, b2, 1e-8f,
                                                        c1, c2, nullptr);
    }
    check("mlp adam");
  });
}

}  // extern "C"
