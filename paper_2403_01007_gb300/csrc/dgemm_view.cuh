// FP64 CUDA-core contraction kernels reading operands through strided views.
//
// An operand is a (batch, row, k) matrix whose row and k indices each map to
// memory through at most two strided levels (see MatView), so most index
// permutations of a tensor contraction need no copy. Tiles are staged through
// shared memory; the loader walks whichever index is unit-stride so that the
// global loads stay coalesced.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "backend.h"

namespace sccsd {

__device__ __forceinline__ int64_t view_row(const MatView& v, int64_t r) {
  return v.n2r ? (r / v.n2r) * v.sr1 + (r % v.n2r) * v.sr2 : r * v.sr2;
}
__device__ __forceinline__ int64_t view_k(const MatView& v, int64_t k) {
  return v.n2k ? (k / v.n2k) * v.sk1 + (k % v.n2k) * v.sk2 : k * v.sk2;
}

// out (partial == 0): C[b][m][n] = alpha * sum_k A(b,m,k) B(b,n,k), b = blockIdx.z
// out (partial == 1): part[z][m][n] = sum over the z-th K chunk of length kc
// Tiles are enumerated by blockIdx.x (M tiles fastest).
template <int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_dgemm_view(int64_t M, int64_t N, int64_t K, int64_t kc,
                                                    double alpha, MatView A, MatView B,
                                                    double* __restrict__ out, int partial) {
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int64_t mt = (M + BM - 1) / BM;
  const int64_t m0 = (int64_t)(blockIdx.x % mt) * BM, n0 = (int64_t)(blockIdx.x / mt) * BN;
  const int64_t z = blockIdx.z;
  int64_t kbeg = 0, kend = K;
  const double* Ap = A.p;
  const double* Bp = B.p;
  double* O = out + z * M * N;
  if (partial) {
    kbeg = z * kc;
    kend = (K < kbeg + kc) ? K : kbeg + kc;
  } else {
    Ap += z * A.sb;
    Bp += z * B.sb;
  }
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool akf = A.n2k ? (A.sk2 == 1) : (A.sk2 == 1);
  const bool bkf = B.n2k ? (B.sk2 == 1) : (B.sk2 == 1);
  int64_t aro[LA], bro[LB];
  int arow[LA], akk[LA], brow[LB], bkk[LB];
#pragma unroll
  for (int q = 0; q < LA; ++q) {
    int e = tid + 256 * q;
    arow[q] = akf ? e / BK : e % BM;
    akk[q] = akf ? e % BK : e / BM;
    int64_t gm = m0 + arow[q];
    aro[q] = gm < M ? view_row(A, gm) : -1;
  }
#pragma unroll
  for (int q = 0; q < LB; ++q) {
    int e = tid + 256 * q;
    brow[q] = bkf ? e / BK : e % BN;
    bkk[q] = bkf ? e % BK : e / BN;
    int64_t gn = n0 + brow[q];
    bro[q] = gn < N ? view_row(B, gn) : -1;
  }
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int64_t gk = k0 + akk[q];
      As[akk[q]][arow[q]] = (aro[q] >= 0 && gk < kend) ? Ap[aro[q] + view_k(A, gk)] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int64_t gk = k0 + bkk[q];
      Bs[bkk[q]][brow[q]] = (bro[q] >= 0 && gk < kend) ? Bp[bro[q] + view_k(B, gk)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const double s = partial ? 1.0 : alpha;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn < N) O[gm * N + gn] = s * acc[i][j];
    }
  }
}

// Matrix-vector form for N == 1: C[b][m] = alpha * sum_k A(b,m,k) x(b,k).
// k contiguous in A: one warp per row; otherwise one thread per row.
__global__ void k_dgemv_view(int64_t M, int64_t K, double alpha, MatView A, MatView X,
                             double* __restrict__ C, int warp_per_row) {
  const int64_t b = blockIdx.z;
  const double* Ap = A.p + b * A.sb;
  const double* Xp = X.p + b * X.sb;
  double* Cb = C + b * M;
  if (warp_per_row) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t m = w; m < M; m += nw) {
      const int64_t ro = view_row(A, m);
      double s = 0.0;
      for (int64_t k = lane; k < K; k += 32) s = fma(Ap[ro + view_k(A, k)], Xp[view_k(X, k)], s);
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (lane == 0) Cb[m] = alpha * s;
    }
  } else {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
      const int64_t ro = view_row(A, m);
      double s = 0.0;
      for (int64_t k = 0; k < K; ++k) s = fma(Ap[ro + view_k(A, k)], Xp[view_k(X, k)], s);
      Cb[m] = alpha * s;
    }
  }
}

// Few outputs, long contraction: one block per (output, K chunk), no padding.
// part[o * chunks + c] = sum over chunk c of A(b,m,k) B(b,n,k), o = (b*M + m)*N + n.
__global__ void k_dot_view(int64_t M, int64_t N, int64_t K, int64_t kc, int chunks, MatView A,
                           MatView B, double* __restrict__ part) {
  const int64_t o = blockIdx.y;
  const int64_t n = o % N, bm = o / N;
  const int64_t m = bm % M, b = bm / M;
  const double* Ap = A.p + b * A.sb + view_row(A, m);
  const double* Bp = B.p + b * B.sb + view_row(B, n);
  const int64_t k0 = (int64_t)blockIdx.x * kc;
  const int64_t k1 = (K < k0 + kc) ? K : k0 + kc;
  double s = 0.0;
  if (!A.n2k && !B.n2k) {
    const int64_t sa = A.sk2, sb = B.sk2;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) s = fma(Ap[k * sa], Bp[k * sb], s);
  } else {
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x)
      s = fma(Ap[view_k(A, k)], Bp[view_k(B, k)], s);
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) part[o * chunks + blockIdx.x] = s;
  }
}

__global__ void k_dot_sum(int64_t outs, int chunks, const double* __restrict__ part, double alpha,
                          double* __restrict__ C) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= outs) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[o * chunks + c];
  C[o] = alpha * s;
}

}  // namespace sccsd
