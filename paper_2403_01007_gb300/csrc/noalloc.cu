// Contraction entry point that allocates no device memory.
//
// The regular entry points grow their scratch buffers (split-K partial sums,
// operand copies) with cudaMalloc on demand. Some callers cannot allow that:
// applications that hand all device memory to their own pool allocator up
// front and forbid further cudaMalloc calls, and latency-critical callers for
// which the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable. For them, sccsd_gemm_tn_noalloc runs the FP64 split-K
// contraction with its partial sums in a fixed file-scope device array
// instead of allocated scratch.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/sccsd.h"

namespace {

// Partial sums of the split-K contraction: [splits][M][N] doubles.
constexpr long long kNoallocCapacity = 1LL << 20;  // 8 MiB, held by every device that loads us
static __device__ __align__(256) double g_noalloc_partials[kNoallocCapacity];

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) k_splitk_noalloc(long long M, long long N, long long K,
                                                        long long kc, const double* __restrict__ A,
                                                        const double* __restrict__ B,
                                                        double* __restrict__ part) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const long long kbeg = (long long)blockIdx.z * kc;
  const long long kend = (K < kbeg + kc) ? K : kbeg + kc;
  const long long m0 = (long long)blockIdx.y * TM, n0 = (long long)blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (long long k0 = kbeg; k0 < kend; k0 += TK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int row = e >> 4, kk = e & 15;
      long long gk = k0 + kk, gm = m0 + row, gn = n0 + row;
      As[kk][row] = (gm < M && gk < kend) ? A[gm * K + gk] : 0.0;
      Bs[kk][row] = (gn < N && gk < kend) ? B[gn * K + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
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
  // every (z, m, n) slot of the used range is written here before it is read
  double* P = part + (long long)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long gn = n0 + tx + 16 * j;
      if (gn < N) P[gm * N + gn] = acc[i][j];
    }
  }
}

__global__ void k_reduce_noalloc(long long n, int splits, const double* __restrict__ part,
                                 double alpha, double* __restrict__ C) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(long long)z * n + e];
    C[e] = alpha * s;
  }
}

// K = 0: the empty sum
__global__ void k_zero_noalloc(long long n, double* __restrict__ C) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    C[e] = 0.0;
}

// Per device, looked up once with that device current: the device address of
// g_noalloc_partials and the number of multiprocessors (the split count is
// sized for it).
struct DeviceInfo {
  void* addr = nullptr;
  int sms = 0;
};
std::mutex g_mu;
DeviceInfo g_dev[256];

int device_info(double** out, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SCCSD_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceInfo& d = g_dev[dev];
  if (!d.addr) {
    void* p = nullptr;
    int n = 0;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return SCCSD_ECUDA;
    }
    d.addr = p;
    d.sms = n;
  }
  *out = (double*)d.addr;
  *sms = d.sms;
  return SCCSD_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" long long sccsd_gemm_tn_noalloc_capacity(void) { return kNoallocCapacity; }

extern "C" int sccsd_gemm_tn_noalloc(long long M, long long N, long long K, double alpha,
                                     const double* A, const double* B, double* C, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C) return SCCSD_EINVAL;
  if (M == 0 || N == 0) return SCCSD_OK;  // an empty C: nothing to write
  // M * N above the capacity (tested without forming the product, which could
  // overflow): even one K chunk would not fit
  if (N > kNoallocCapacity / M) return SCCSD_EINVAL;
  if ((M + TM - 1) / TM > 65535) return SCCSD_EINVAL;
  if (!on_device(A) || !on_device(B) || !on_device(C)) return SCCSD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = M * N;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (K == 0) {
    k_zero_noalloc<<<blocks, 256, 0, st>>>(n, C);
    return cudaGetLastError() == cudaSuccess ? SCCSD_OK : SCCSD_ECUDA;
  }
  double* part = nullptr;
  int sms = 0;
  int rc = device_info(&part, &sms);
  if (rc != SCCSD_OK) return rc;
  const long long tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  // about four CTAs per multiprocessor, at least 256 K values per split, and
  // never more partial sums than the shared array holds
  long long splits = (4LL * sms + tiles - 1) / tiles;
  if (splits > K / 256) splits = K / 256;
  if (splits > kNoallocCapacity / n) splits = kNoallocCapacity / n;
  if (splits > 1024) splits = 1024;
  if (splits < 1) splits = 1;
  long long kc = (K + splits - 1) / splits;
  kc = (kc + TK - 1) / TK * TK;
  splits = (K + kc - 1) / kc;  // never above the clamped value: kc only grew
  dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM), (unsigned)splits);
  k_splitk_noalloc<<<grid, 256, 0, st>>>(M, N, K, kc, A, B, part);
  if (cudaGetLastError() != cudaSuccess) return SCCSD_ECUDA;
  k_reduce_noalloc<<<blocks, 256, 0, st>>>(n, (int)splits, part, alpha, C);
  if (cudaGetLastError() != cudaSuccess) return SCCSD_ECUDA;
  return SCCSD_OK;
}
