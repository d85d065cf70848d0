// CUDA backend of the graph executor: FP64 kernels for strided copies,
// packing, reductions and contractions, plus dispatch of tensor-core
// eligible contractions to the tcgen05 path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <string>
#include <vector>

#include "backend.h"
#include "dgemm_view.cuh"
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

// Four elements per thread and round, their loads issued before any store, so
// that a thread keeps four (eight when accumulating) HBM reads in flight;
// consecutive threads take consecutive linear indices in each of the four
// slabs of a round. total < 2^31 and the grid holds fewer than 2^22 threads,
// so lin + 3 * stride cannot wrap.
__global__ void k_copy_view32(ViewArgs32 a, uint32_t total, double* __restrict__ out,
                              const double* __restrict__ in, double coef, int acc) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t lin = blockIdx.x * blockDim.x + threadIdx.x; lin < total; lin += 4 * stride) {
    uint32_t oo[4], ii[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t l = lin + (uint32_t)u * stride;
      ok[u] = l < total;
      uint32_t r = ok[u] ? l : 0, o = 0, i = 0;
      // compile-time indices keep the view in kernel parameters (no local copy)
#pragma unroll
      for (int k = kMaxRank - 1; k >= 0; --k) {
        if (k >= a.rank) continue;
        const uint32_t c = r % a.dims[k];
        r /= a.dims[k];
        o += c * a.ostr[k];
        i += c * a.istr[k];
      }
      oo[u] = o;
      ii[u] = i;
    }
    double v[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = ok[u] ? in[ii[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = (acc && ok[u]) ? out[oo[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u]) out[oo[u]] = w[u] + coef * v[u];
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

// out (+)= coef * a * b elementwise over a strided index box (no contracted
// index; a zero stride broadcasts)
struct MulArgs32 {
  int rank;
  uint32_t dims[kMaxRank];
  uint32_t ostr[kMaxRank];
  uint32_t astr[kMaxRank];
  uint32_t bstr[kMaxRank];
};
struct MulArgs {
  int rank;
  int64_t dims[kMaxRank];
  int64_t ostr[kMaxRank];
  int64_t astr[kMaxRank];
  int64_t bstr[kMaxRank];
};

template <class Args, class I>
__global__ void k_mul_view(Args m, I total, double* __restrict__ out, const double* __restrict__ a,
                           const double* __restrict__ b, double coef, int acc) {
  for (I lin = (I)blockIdx.x * blockDim.x + threadIdx.x; lin < total;
       lin += (I)gridDim.x * blockDim.x) {
    I r = lin, oo = 0, ia = 0, ib = 0;
    for (int k = m.rank - 1; k >= 0; --k) {
      const I c = r % (I)m.dims[k];
      r /= (I)m.dims[k];
      oo += c * (I)m.ostr[k];
      ia += c * (I)m.astr[k];
      ib += c * (I)m.bstr[k];
    }
    const double v = coef * a[ia] * b[ib];
    out[oo] = acc ? out[oo] + v : v;
  }
}

// 64x64 shared-memory tile transpose for copies whose fastest output index is
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

constexpr int TT = 64;  // transpose tile edge

__global__ void __launch_bounds__(256, 3) k_copy_transpose(TransArgs a, double* __restrict__ out,
                                                        const double* __restrict__ in,
                                                        double coef, int acc) {
  __shared__ double tile[TT][TT + 1];
  const int64_t nx = a.dims[a.px], ny = a.dims[a.py];
  const int64_t isx = a.istr[a.px], isy = a.istr[a.py], osx = a.ostr[a.px], osy = a.ostr[a.py];
  const int tx = threadIdx.x, ty = threadIdx.y;  // blockDim = (32, 8)
  for (int64_t rest = blockIdx.z; rest < a.rest_total; rest += gridDim.z) {
    int64_t r = rest, ob = 0, ib = 0;
    for (int k = a.rank - 1; k >= 0; --k) {
      if (k == a.px || k == a.py) continue;
      int64_t c = r % a.dims[k];
      r /= a.dims[k];
      ob += c * a.ostr[k];
      ib += c * a.istr[k];
    }
    const int64_t x0 = (int64_t)blockIdx.x * TT, y0 = (int64_t)blockIdx.y * TT;
    // read: consecutive lanes walk the input-contiguous dim (y); the loads of
    // a half tile are all issued before the shared-memory stores
    const double* ip = in + ib + (x0 + ty) * isx + (y0 + tx) * isy;
    const int64_t ix8 = 8 * isx, iy32 = 32 * isy;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int xi = ty + 8 * q, yj = tx + 32 * h;
        v[q] = (x0 + xi < nx && y0 + yj < ny) ? __ldg(ip + q * ix8 + h * iy32) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) tile[ty + 8 * q][tx + 32 * h] = v[q];
    }
    __syncthreads();
    // write: consecutive lanes walk the output-contiguous dim (x)
    double* op = out + ob + (x0 + tx) * osx + (y0 + ty) * osy;
    const int64_t oy8 = 8 * osy, ox32 = 32 * osx;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double old[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int yj = ty + 8 * q, xi = tx + 32 * h;
        old[q] = (acc && x0 + xi < nx && y0 + yj < ny) ? op[q * oy8 + h * ox32] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int yj = ty + 8 * q, xi = tx + 32 * h;
        if (x0 + xi < nx && y0 + yj < ny) op[q * oy8 + h * ox32] = old[q] + coef * tile[xi][yj];
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
    int64_t Q = (int64_t)((sqrtf((float)(8 * q + 1)) - 1.0f) * 0.5f);
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

__global__ void k_sum_parts(int64_t n, int splits, const double* __restrict__ part, double alpha,
                            double* __restrict__ C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * n + e];
    C[e] = alpha * s;
  }
}

// ------------------------------------------------------------------ ladder
//
// Sum_cd g_acbd X_ij^cd with g_acbd = sum_J L^J_ac L^J_bd (the vvvv block of
// the Hamiltonian, Sec. 2.4.2) in the symmetric / antisymmetric form: with
// G+-_(ab)(cd) = g_acbd +- g_adbc over pairs a <= b, c <= d, and
//   X~+_ij(cd) = X_ij^cd + X_ij^dc (c < d), X_ij^cc (c = d),
//   X-_ij(cd)  = X_ij^cd - X_ij^dc (c < d),
// the result is Y_ij^ab = P_ij(ab) + s M_ij(ab) with
//   P = 1/2 sum_(c<=d) G+ X~+,   M = 1/2 sum_(c<d) G- X-,
// s = +1 for a <= b and -1 for a > b. Every operand the residual graph hands
// to the ladder has the pair symmetry X_ij^cd = X_ji^dc, so X~+ is symmetric
// and X- antisymmetric in ij: P is needed for i <= j only and M for i < j.
// Pair indices are row-major over the upper triangle: p(a, b) = a (v - 1) -
// a (a - 1) / 2 + b for a <= b (likewise q(c, d) and the occupied pairs).

// X~+[(z, i<=j)][q] and X-[(z, i<j)][q] from X[(z, i, j)][(c, d)]; with the
// pair symmetry X_ij^dc is read as X_ji^cd, so both reads walk d. Written as
// FP64 rows of stride ld, or (Out = __nv_bfloat16) as `nsl` BF16 slices of a
// tensor-core operand (rows of stride ld, slices sstride apart; x = sum of the
// slices, each the BF16 rounding of what the previous ones left, formed in
// double so that the last slice keeps the remainder).
// values x[0], x[1] at i0, i0 + 1 (the second only when i0 + 1 < n); i0 even
template <class Out>
__device__ __forceinline__ void put_pair(Out* p, int64_t i0, const double* x, int64_t n, int nsl,
                                         int64_t sstride);
template <>
__device__ __forceinline__ void put_pair<double>(double* p, int64_t i0, const double* x, int64_t n,
                                                 int, int64_t) {
  p[i0] = x[0];
  if (i0 + 1 < n) p[i0 + 1] = x[1];
}
template <>
__device__ __forceinline__ void put_pair<__nv_bfloat16>(__nv_bfloat16* p, int64_t i0,
                                                        const double* x, int64_t n, int nsl,
                                                        int64_t sstride) {
  double r0 = x[0], r1 = x[1];
  for (int s = 0; s < nsl; ++s) {
    __nv_bfloat162 b;
    b.x = __float2bfloat16_rn((float)r0);
    b.y = __float2bfloat16_rn((float)r1);
    if (i0 + 1 < n)
      *reinterpret_cast<__nv_bfloat162*>(p + s * sstride + i0) = b;
    else
      p[s * sstride + i0] = b.x;
    r0 -= (double)__bfloat162float(b.x);
    r1 -= (double)__bfloat162float(b.y);
  }
}

template <class Out>
__global__ void k_ladder_pack_x(const double* __restrict__ X, int o, int v, int64_t nb,
                                const int* __restrict__ pairs, Out* __restrict__ Xp,
                                Out* __restrict__ Xm, int64_t ld, int nsl, int64_t sp_stride,
                                int64_t sm_stride) {
  const int64_t Po = (int64_t)o * (o + 1) / 2, Pm = (int64_t)o * (o - 1) / 2;
  const int64_t Pv = (int64_t)v * (v + 1) / 2, vv = (int64_t)v * v;
  for (int64_t blk = blockIdx.x; blk < nb * Po; blk += gridDim.x) {
    const int64_t z = blk / Po;
    int r = (int)(blk % Po), i = 0;
    while (r >= o - i) {
      r -= o - i;
      ++i;
    }
    const int j = i + r;
    const double* xij = X + ((z * o + i) * o + j) * vv;
    const double* xji = X + ((z * o + j) * o + i) * vv;
    Out* op = Xp + blk * ld;
    Out* om = i < j ? Xm + (z * Pm + (int64_t)i * (o - 1) - (int64_t)i * (i - 1) / 2 + (j - i - 1)) * ld
                    : nullptr;
    // two consecutive q per thread (one 4-byte store per BF16 slice)
    for (int64_t q0 = 2 * (int64_t)threadIdx.x; q0 < Pv; q0 += 2 * (int64_t)blockDim.x) {
      double pv[2], mv[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t q = q0 + h;
        pv[h] = mv[h] = 0.0;
        if (q < Pv) {
          const int cd = __ldg(pairs + q);
          const int c = cd >> 16, d = cd & 0xffff;
          const int64_t e = (int64_t)c * v + d;
          const double a = xij[e], b = xji[e];
          pv[h] = c == d ? 0.5 * (a + b) : a + b;
          mv[h] = c == d ? 0.0 : a - b;
        }
      }
      put_pair<Out>(op, q0, pv, Pv, nsl, sp_stride);
      if (om) put_pair<Out>(om, q0, mv, Pv, nsl, sm_stride);
    }
  }
}

// Y[(z, i, j)][(a, b)] from P[(z, i<=j)][p] and M[(z, i<j)][p]. A block takes
// one occupied pair i0 <= j0 and one 32 x 32 tile of (a, b) with a-tile <=
// b-tile: it reads the P and M entries of the tile once (b fastest), and
// writes Y_i0j0^ab = P + M, Y_j0i0^ab = P - M and, through shared memory, the
// transposed elements Y_i0j0^ba = P - M, Y_j0i0^ba = P + M (a fastest), so that
// every read and write walks consecutive addresses.
constexpr int UT = 32;  // unpack tile edge

__global__ void __launch_bounds__(256) k_ladder_unpack(const double* __restrict__ P,
                                                       const double* __restrict__ M, int64_t ld,
                                                       int o, int v, int64_t nb,
                                                       double* __restrict__ Y) {
  __shared__ double tp[UT][UT + 1], tm[UT][UT + 1];
  const int64_t vv = (int64_t)v * v, oo = (int64_t)o * o;
  const int64_t Po = (int64_t)o * (o + 1) / 2, Pm = (int64_t)o * (o - 1) / 2;
  const int nt = (v + UT - 1) / UT;
  const int64_t tiles = (int64_t)nt * (nt + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int64_t blk = blockIdx.x; blk < nb * Po * tiles; blk += gridDim.x) {
    const int64_t rowp = blk / tiles;
    int t = (int)(blk % tiles), ta = 0;
    while (t >= nt - ta) {
      t -= nt - ta;
      ++ta;
    }
    const int tb = ta + t;
    const int64_t z = rowp / Po;
    int r = (int)(rowp % Po), i0 = 0;
    while (r >= o - i0) {
      r -= o - i0;
      ++i0;
    }
    const int j0 = i0 + r;
    const double* pr = P + rowp * ld;
    const double* mr =
        i0 < j0 ? M + (z * Pm + (int64_t)i0 * (o - 1) - (int64_t)i0 * (i0 - 1) / 2 + (j0 - i0 - 1)) * ld
                : nullptr;
    double* y1 = Y + ((z * o + i0) * o + j0) * vv;   // row (i0, j0)
    double* y2 = Y + ((z * o + j0) * o + i0) * vv;   // row (j0, i0)
    const int a0 = ta * UT, b0 = tb * UT;
    // load the tile's P and M entries (a <= b), b fastest
    for (int k = ty; k < UT; k += 8) {
      const int a = a0 + k, b = b0 + tx;
      double pv = 0.0, mv = 0.0;
      if (a < v && b < v) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        const int64_t p = (int64_t)lo * (v - 1) - (int64_t)lo * (lo - 1) / 2 + hi;
        pv = pr[p];
        if (mr && lo < hi) mv = (a <= b ? 1.0 : -1.0) * mr[p];
      }
      tp[k][tx] = pv;
      tm[k][tx] = mv;
    }
    __syncthreads();
    // direct elements (a, b): Y_i0j0 = P + M, Y_j0i0 = P - M
    for (int k = ty; k < UT; k += 8) {
      const int a = a0 + k, b = b0 + tx;
      if (a < v && b < v && (ta < tb || a <= b)) {
        const int64_t e = (int64_t)a * v + b;
        y1[e] = tp[k][tx] + tm[k][tx];
        if (i0 < j0) y2[e] = tp[k][tx] - tm[k][tx];
      }
    }
    // transposed elements (b, a) of the tile, a fastest: Y_i0j0 = P - M, Y_j0i0 = P + M
    for (int k = ty; k < UT; k += 8) {
      const int b = b0 + k, a = a0 + tx;
      if (a < v && b < v && (ta < tb || a < b)) {
        const int64_t e = (int64_t)b * v + a;
        y1[e] = tp[tx][k] - tm[tx][k];
        if (i0 < j0) y2[e] = tp[tx][k] + tm[tx][k];
      }
    }
    __syncthreads();
  }
}

// G+ and G- rows of pairs from a block of the full integrals,
// Gc[((a - a0) v + c)][((b - a0) v + d)] = g_acbd (FP64 build)
__global__ void k_ladder_pack_g(const double* __restrict__ Gc, int64_t ldg, int v, int a0,
                                const int* __restrict__ pairs, int64_t p_begin, int64_t npairs,
                                double* __restrict__ Gp, double* __restrict__ Gm, int64_t ld) {
  const int64_t Pv = (int64_t)v * (v + 1) / 2;
  for (int64_t w = blockIdx.x; w < npairs; w += gridDim.x) {
    const int ab = __ldg(pairs + p_begin + w);
    const int a = ab >> 16, b = ab & 0xffff;
    const double* W = Gc + (int64_t)(a - a0) * v * ldg + (int64_t)(b - a0) * v;  // W[c][d] = W[c ldg + d]
    for (int64_t q = threadIdx.x; q < Pv; q += blockDim.x) {
      const int cd = __ldg(pairs + q);
      const int c = cd >> 16, d = cd & 0xffff;
      const double x = W[(int64_t)c * ldg + d], y = W[(int64_t)d * ldg + c];
      Gp[w * ld + q] = x + y;
      Gm[w * ld + q] = c == d ? 0.0 : x - y;
    }
  }
}

// ------------------------------------------------------------------ backend

class CudaBackend : public Backend {
 public:
  cudaStream_t st;
  int precision;
  std::vector<double*> slots = std::vector<double*>(8, nullptr);
  std::vector<int64_t> slot_n = std::vector<int64_t>(8, 0);
  std::unique_ptr<TcGemm> tc;
  // ladder: pair table of the current v (device, a << 16 | b), the virtual
  // block of L in tensor-core form (kept while L is unchanged), the packed
  // operands of one call and the G+- slabs of one chunk of pairs
  int* pairs_dev = nullptr;
  int pairs_v = -1;
  TcOperand lt_op, xp_op, xm_op, gp_op, gm_op;
  int64_t lt_version = -1;
  const double* lt_src = nullptr;
  int lt_slices = 0;
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  double prof_ms = 0.0, prof_flops = 0.0;
  long long prof_calls = 0, launches0 = 0;
  std::map<int64_t, std::vector<double*>> pool;
  struct CacheEntry {
    int64_t version;
    TcOperand op;
  };
  std::map<std::tuple<const void*, int, uint64_t>, CacheEntry> opcache;
  TcOperand tmpA, tmpB;

  CudaBackend(void* stream, int prec) : st((cudaStream_t)stream), precision(prec) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (precision != 0) tc = std::make_unique<TcGemm>(st, precision);
  }
  ~CudaBackend() override {
    if (tc) {
      for (auto& kv : opcache) tc->release(kv.second.op);
      tc->release(tmpA);
      tc->release(tmpB);
    }
    for (auto& kv : pool)
      for (double* p : kv.second) cudaFree(p);
    for (auto& e : ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    for (double* p : slots)
      if (p) cudaFree(p);
    if (tc)
      for (TcOperand* op : {&lt_op, &xp_op, &xm_op, &gp_op, &gm_op}) tc->release(*op);
    if (pairs_dev) cudaFree(pairs_dev);
    tc.reset();
  }

  bool autotune = false;
  void set_autotune(bool on) override {
    autotune = on;
    if (tc) tc->set_tune(on);
  }

  bool capturing = false, prof_saved = false;
  // profiling events stay out of captured graphs
  void set_capturing(bool on) override {
    if (on && !capturing) { prof_saved = prof; prof = false; }
    if (!on && capturing) prof = prof_saved;
    capturing = on;
  }

  double* alloc(int64_t n) override {
    if (capturing) throw std::runtime_error("device allocation during graph capture (warm-up missing)");
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
    if (capturing) return;
    CK(cudaStreamSynchronize(st));
    if (tc) tc->check_error();
  }
  void* stream() override { return (void*)st; }
  int get_precision() const override { return precision; }
  void set_precision(int p) override {
    if (p == precision) return;
    sync();
    precision = p;
    if (p != 0) {
      if (!tc) {
        tc = std::make_unique<TcGemm>(st, p);
        tc->set_tune(autotune);
      } else {
        tc->set_precision(p);
      }
    }
    if (tc)
      for (auto& kv : opcache) tc->release(kv.second.op);
    opcache.clear();
    lt_version = -1;
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
      dim3 grid((unsigned)((d[px] + TT - 1) / TT), (unsigned)((d[py] + TT - 1) / TT),
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

  void mul_view(int rank, const int64_t* dims, double* out, const int64_t* ostr, const double* a,
                const int64_t* astr, const double* b, const int64_t* bstr, double coef,
                bool acc) override {
    // merge adjacent dims contiguous on all three sides; drop unit dims
    int64_t d[kMaxRank], os[kMaxRank], as[kMaxRank], bs[kMaxRank];
    int r = 0;
    int64_t total = 1;
    for (int k = 0; k < rank; ++k) {
      total *= dims[k];
      if (dims[k] == 1) continue;
      if (r > 0 && os[r - 1] == ostr[k] * dims[k] && as[r - 1] == astr[k] * dims[k] &&
          bs[r - 1] == bstr[k] * dims[k]) {
        d[r - 1] *= dims[k];
        os[r - 1] = ostr[k];
        as[r - 1] = astr[k];
        bs[r - 1] = bstr[k];
        continue;
      }
      d[r] = dims[k];
      os[r] = ostr[k];
      as[r] = astr[k];
      bs[r] = bstr[k];
      ++r;
    }
    if (total == 0) return;
    int64_t omax = 0, amax = 0, bmax = 0;
    for (int k = 0; k < r; ++k) {
      omax += (d[k] - 1) * os[k];
      amax += (d[k] - 1) * as[k];
      bmax += (d[k] - 1) * bs[k];
    }
    const int64_t lim = 1LL << 31;
    if (total < lim && omax < lim && amax < lim && bmax < lim) {
      MulArgs32 m;
      m.rank = r;
      for (int k = 0; k < r; ++k) {
        m.dims[k] = (uint32_t)d[k];
        m.ostr[k] = (uint32_t)os[k];
        m.astr[k] = (uint32_t)as[k];
        m.bstr[k] = (uint32_t)bs[k];
      }
      k_mul_view<MulArgs32, uint32_t><<<grid_for(total, 256), 256, 0, st>>>(
          m, (uint32_t)total, out, a, b, coef, acc ? 1 : 0);
    } else {
      MulArgs m;
      m.rank = r;
      for (int k = 0; k < r; ++k) {
        m.dims[k] = d[k];
        m.ostr[k] = os[k];
        m.astr[k] = as[k];
        m.bstr[k] = bs[k];
      }
      k_mul_view<MulArgs, int64_t><<<grid_for(total, 256), 256, 0, st>>>(m, total, out, a, b,
                                                                           coef, acc ? 1 : 0);
    }
    check_launch("mul_view");
  }

  void dgemm(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
             const double* B, double* C) {
    dgemm_v(nb, M, N, K, alpha, MatView::dense(A, M, K), MatView::dense(B, N, K), C);
  }

  // FP64 contraction through strided views (see dgemm_view.cuh)
  void dgemm_v(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const MatView& A,
               const MatView& B, double* C) {
    if (nb * M * N == 0) return;
    if (K == 0) {
      fill(C, nb * M * N, 0.0);
      return;
    }
    // FP64 FMAs are scarce on this part: shapes are routed so that padding
    // wastes as few of them as possible
    const int64_t outs = nb * M * N;
    if (outs <= 4096 && K >= 512) {
      int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + outs - 1) / outs, K / 2048));
      int64_t kc = (K + chunks - 1) / chunks;
      chunks = (K + kc - 1) / kc;
      double* part = scratch(7, outs * chunks);
      k_dot_view<<<dim3((unsigned)chunks, (unsigned)outs), 256, 0, st>>>(M, N, K, kc, (int)chunks,
                                                                         A, B, part);
      check_launch("dot_view");
      k_dot_sum<<<(unsigned)((outs + 127) / 128), 128, 0, st>>>(outs, (int)chunks, part, alpha, C);
      check_launch("dot_sum");
      return;
    }
    if (N == 1 || M == 1) {
      // matrix-vector form; for M == 1 the roles swap (C^T has the same layout)
      const MatView& Mv = (N == 1) ? A : B;
      const MatView& Xv = (N == 1) ? B : A;
      const int64_t rows = (N == 1) ? M : N;
      const int wpr = Mv.sk2 == 1 ? 1 : 0;
      int64_t threads = wpr ? rows * 32 : rows;
      dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, 152 * 32)),
                1, (unsigned)nb);
      if (nb > 65535) throw std::runtime_error("gemv batch too large");
      k_dgemv_view<<<grid, 256, 0, st>>>(rows, K, alpha, Mv, Xv, C, wpr);
      check_launch("dgemv_view");
      return;
    }
    // tile shape: narrow tiles for skinny outputs
    int shape = 0;  // 0: 64x64, 1: 32x32, 2: 32x64, 3: 64x32
    if (M <= 32 && N <= 32)
      shape = 1;
    else if (M <= 32)
      shape = 2;
    else if (N <= 32)
      shape = 3;
    const int64_t bm = (shape == 1 || shape == 2) ? 32 : 64;
    const int64_t bn = (shape == 1 || shape == 3) ? 32 : 64;
    const int64_t bk = shape == 1 ? 32 : 16;
    const int64_t tiles = ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
    auto launch = [&](dim3 grid, int64_t kc, double* o, int partial) {
      switch (shape) {
        case 1: k_dgemm_view<32, 32, 32><<<grid, 256, 0, st>>>(M, N, K, kc, alpha, A, B, o, partial); break;
        case 2: k_dgemm_view<32, 64, 16><<<grid, 256, 0, st>>>(M, N, K, kc, alpha, A, B, o, partial); break;
        case 3: k_dgemm_view<64, 32, 16><<<grid, 256, 0, st>>>(M, N, K, kc, alpha, A, B, o, partial); break;
        default: k_dgemm_view<64, 64, 16><<<grid, 256, 0, st>>>(M, N, K, kc, alpha, A, B, o, partial);
      }
      check_launch("dgemm_view");
    };
    if (nb == 1 && tiles < 2 * 152 && K >= 256) {
      // split K so that the grid fills the GPU; the partial tiles are summed
      // in a fixed order afterwards (deterministic)
      int64_t splits = std::min<int64_t>((4 * 152 + tiles - 1) / tiles, K / 128);
      splits = std::max<int64_t>(2, std::min<int64_t>(splits, 1024));
      int64_t kc = (K + splits - 1) / splits;
      kc = (kc + bk - 1) / bk * bk;
      splits = (K + kc - 1) / kc;
      double* part = scratch(7, splits * M * N);
      launch(dim3((unsigned)tiles, 1, (unsigned)splits), kc, part, 1);
      k_sum_parts<<<grid_for(M * N, 256), 256, 0, st>>>(M * N, (int)splits, part, alpha, C);
      check_launch("sum_parts");
      return;
    }
    if (nb > 65535) throw std::runtime_error("batched GEMM: batch too large");
    if (tiles > (1LL << 31) - 1) throw std::runtime_error("GEMM: too many tiles");
    launch(dim3((unsigned)tiles, 1, (unsigned)nb), 0, C, 0);
  }

  void gemm_view(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const MatView& A,
                 const MatView& B, double* C, bool use_tc) override {
    if (use_tc && tc && precision != 0 && tc->worthwhile(nb, M, N, K)) {
      gemm_tc_keyed(M, N, K, alpha, A, nullptr, B, nullptr, C, nullptr, false);
      return;
    }
    dgemm_v(nb, M, N, K, alpha, A, B, C);
  }

  bool tc_will_use(int64_t nb, int64_t M, int64_t N, int64_t K) override {
    return tc && precision != 0 && tc->worthwhile(nb, M, N, K);
  }
  bool tc_cached(const OperandKey& k) override {
    auto it = opcache.find(std::make_tuple(k.graph, k.id, k.layout));
    return it != opcache.end() && it->second.version == k.version;
  }
  const TcOperand& tc_operand(const MatView& X, int64_t rows, int64_t K, const OperandKey* key,
                              TcOperand& tmp) {
    if (!key) {
      tc->prepare_operand_view(X, rows, K, tmp);
      return tmp;
    }
    CacheEntry& e = opcache[std::make_tuple(key->graph, key->id, key->layout)];
    if (e.op.data && e.version == key->version && e.op.rows == rows && e.op.k == K) return e.op;
    if (!X.p) throw std::runtime_error("tensor-core operand cache miss without data");
    tc->prepare_operand_view(X, rows, K, e.op);
    e.version = key->version;
    return e.op;
  }
  void gemm_tc_keyed(int64_t M, int64_t N, int64_t K, double alpha, const MatView& A,
                     const OperandKey* ka, const MatView& B, const OperandKey* kb,
                     double* C, const OutView* ov, bool accumulate) override {
    const TcOperand& a = tc_operand(A, M, K, ka, tmpA);
    const TcOperand& b = tc_operand(B, N, K, kb, tmpB);
    tc->gemm_ops(M, N, alpha, a, b, C, ov ? *ov : OutView::dense(N), accumulate);
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

  double* pool_get(int64_t n) override {
    auto it = pool.find(n);
    if (it != pool.end() && !it->second.empty()) {
      double* p = it->second.back();
      it->second.pop_back();
      return p;
    }
    return alloc(n);
  }
  void pool_put(double* p, int64_t n) override { pool[n].push_back(p); }

  void profile(bool enable) override {
    sync();
    for (auto& e : ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    ev.clear();
    prof = enable;
    prof_ms = 0.0;
    prof_flops = 0.0;
    prof_calls = 0;
    launches0 = g_launches;
  }
  void profile_read(double* ms, long long* calls, double* flops, long long* launches) override {
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
    if (flops) *flops = prof_flops;
    if (launches) *launches = g_launches - launches0;
  }

  // device table of the packed pairs (a, b), a <= b, of v indices
  const int* pair_table(int v) {
    if (pairs_v == v) return pairs_dev;
    const int64_t Pv = (int64_t)v * (v + 1) / 2;
    if (v > 65535) throw std::runtime_error("ladder: v too large for the pair table");
    std::vector<int> h((size_t)Pv);
    int64_t k = 0;
    for (int a = 0; a < v; ++a)
      for (int b = a; b < v; ++b) h[(size_t)k++] = (a << 16) | b;
    if (pairs_dev) {
      CK(cudaStreamSynchronize(st));
      cudaFree(pairs_dev);
      pairs_dev = nullptr;
      pairs_v = -1;
    }
    if (capturing) throw std::runtime_error("device allocation during graph capture (warm-up missing)");
    if (cudaMalloc(&pairs_dev, sizeof(int) * (size_t)Pv) != cudaSuccess) {
      cudaGetLastError();
      throw OomError("ladder pair table");
    }
    CK(cudaMemcpyAsync(pairs_dev, h.data(), sizeof(int) * (size_t)Pv, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    pairs_v = v;
    return pairs_dev;
  }

  // Y[(z ij)][(ab)] = sum_(cd) g_acbd X[(z ij)][(cd)], the ladder integrals
  // formed from the Cholesky vectors inside the call (never stored whole).
  void ladder(const Graph& g, const double* L, int64_t ver, const double* X, double* Y,
              int64_t rows) override {
    const int o = g.o, v = g.v, J = g.J;
    const int64_t n = (int64_t)o + v, oo = (int64_t)o * o, nb = rows / oo;
    const int64_t Pv = (int64_t)v * (v + 1) / 2;
    const int64_t Po = (int64_t)o * (o + 1) / 2, Pm = (int64_t)o * (o - 1) / 2;
    const int64_t np = nb * Po, nm = nb * Pm;
    const bool mixed = tc && precision != 0;
    const int* pairs = pair_table(v);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      CK(cudaEventRecord(e0, st));
    }
    // packed operands X~+, X- (FP64, or BF16 slices of tensor-core operands in
    // a mixed mode) and the results P, M [rows][Pv]
    double* Xp = nullptr;
    double* Xm = nullptr;
    double* Pr = scratch(2, np * Pv);
    double* Mr = scratch(3, std::max<int64_t>(1, nm) * Pv);
    if (mixed) {
      const int nsl = tc->slices();
      tc->alloc_operand(np, Pv, nsl, xp_op);
      tc->alloc_operand(std::max<int64_t>(1, nm), Pv, nsl, xm_op);
      xm_op.rows = nm;
      k_ladder_pack_x<__nv_bfloat16><<<grid_for(np * 256, 256), 256, 0, st>>>(
          X, o, v, nb, pairs, (__nv_bfloat16*)xp_op.data, (__nv_bfloat16*)xm_op.data, xp_op.k_pad,
          nsl, xp_op.rows_pad * xp_op.k_pad, xm_op.rows_pad * xm_op.k_pad);
    } else {
      Xp = scratch(0, np * Pv);
      Xm = scratch(1, std::max<int64_t>(1, nm) * Pv);
      k_ladder_pack_x<double><<<grid_for(np * 256, 256), 256, 0, st>>>(X, o, v, nb, pairs, Xp, Xm,
                                                                      Pv, 1, 0, 0);
    }
    check_launch("ladder_pack_x");
    if (mixed && v <= TcGemm::ladder_build_max_v()) {
      // fused build on the tensor cores, one chunk of pairs at a time
      if (lt_version != ver || lt_src != L || lt_slices != tc->slices()) {
        tc->prepare_ladder_lt(L, o, v, J, lt_op);
        lt_version = ver;
        lt_src = L;
        lt_slices = tc->slices();
      }
      // chunks of whole 256-pair tiles sized so that the contraction of one
      // chunk is about one wave of the persistent grid
      int sms = 152;
      {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      }
      const int64_t mt = std::max<int64_t>(1, (np + 127) / 128);
      int64_t nt = std::max<int64_t>(1, sms / mt);
      const int64_t chunk = std::min<int64_t>(nt * 256, ((Pv + 255) / 256) * 256);
      tc->alloc_operand(chunk, Pv, tc->slices(), gp_op);
      tc->alloc_operand(chunk, Pv, tc->slices(), gm_op);
      for (int64_t p0 = 0; p0 < Pv; p0 += chunk) {
        const int64_t cnt = std::min<int64_t>(chunk, Pv - p0);
        // the slabs as operands of this chunk's rows only (fewer N tiles in the
        // last chunk); the build writes its slices at the same row stride
        TcOperand gp = gp_op, gm = gm_op;
        gp.rows = gm.rows = cnt;
        gp.rows_pad = gm.rows_pad = (cnt + 255) / 256 * 256;
        tc->ladder_build(lt_op, v, pairs, p0, cnt, gp, gm);
        tc->gemm_ops(np, cnt, 0.5, xp_op, gp, Pr + p0, OutView::dense(Pv), false);
        if (nm > 0) tc->gemm_ops(nm, cnt, 0.5, xm_op, gm, Mr + p0, OutView::dense(Pv), false);
      }
    } else {
      // build g_acbd for a block of a values with FP64 GEMMs, form G+- of its
      // pairs, contract (FP64, or on the tensor cores in a mixed mode)
      const int64_t vv = (int64_t)v * v;
      double* Lt = scratch(4, vv * J);  // Lt[(a c)][J]
      {
        int64_t dims[3] = {v, v, J};
        int64_t ostr[3] = {(int64_t)v * J, J, 1};
        int64_t istr[3] = {n, 1, n * n};
        copy_view(3, dims, Lt, ostr, L + o * n + o, istr, 1.0, false);
      }
      const int64_t budget = (int64_t)1 << 27;  // doubles of one integral block (1 GiB)
      for (int a0 = 0; a0 < v;) {
        const int64_t cols = (int64_t)(v - a0) * v;
        int na = (int)std::max<int64_t>(1, std::min<int64_t>(v - a0, budget / (cols * v)));
        const int a1 = a0 + na;
        const int64_t p0 = (int64_t)a0 * (v - 1) - (int64_t)a0 * (a0 - 1) / 2 + a0;
        const int64_t p1 = a1 < v ? (int64_t)a1 * (v - 1) - (int64_t)a1 * (a1 - 1) / 2 + a1 : Pv;
        const int64_t cnt = p1 - p0;
        double* Gc = scratch(5, (int64_t)na * v * cols);
        gemm_tn(1, (int64_t)na * v, cols, J, 1.0, Lt + (int64_t)a0 * v * J, Lt + (int64_t)a0 * v * J,
                Gc, false);
        // (slot 7 holds the split-K partial sums of the FP64 GEMMs)
        double* Gp = scratch(6, 2 * cnt * Pv);
        double* Gm = Gp + cnt * Pv;
        k_ladder_pack_g<<<grid_for(cnt * 256, 256), 256, 0, st>>>(Gc, cols, v, a0, pairs, p0, cnt, Gp,
                                                                  Gm, Pv);
        check_launch("ladder_pack_g");
        if (mixed) {
          tc->prepare_operand(Gp, cnt, Pv, gp_op);
          tc->gemm_ops(np, cnt, 0.5, xp_op, gp_op, Pr + p0, OutView::dense(Pv), false);
          if (nm > 0) {
            tc->prepare_operand(Gm, cnt, Pv, gm_op);
            tc->gemm_ops(nm, cnt, 0.5, xm_op, gm_op, Mr + p0, OutView::dense(Pv), false);
          }
        } else {
          // C[n][w] for the pairs of this block, then into P[n][p0 + w]
          double* Cc = scratch(5, std::max(np, nm) * cnt);
          dgemm(1, np, cnt, Pv, 0.5, Xp, Gp, Cc);
          int64_t dims[2] = {np, cnt}, ostr[2] = {Pv, 1}, istr[2] = {cnt, 1};
          copy_view(2, dims, Pr + p0, ostr, Cc, istr, 1.0, false);
          if (nm > 0) {
            dgemm(1, nm, cnt, Pv, 0.5, Xm, Gm, Cc);
            int64_t dm[2] = {nm, cnt};
            copy_view(2, dm, Mr + p0, ostr, Cc, istr, 1.0, false);
          }
        }
        a0 = a1;
      }
    }
    {
      const int64_t ntl = (v + UT - 1) / UT;
      k_ladder_unpack<<<grid_for(np * ntl * (ntl + 1) / 2 * 256, 256), 256, 0, st>>>(Pr, Mr, Pv, o,
                                                                                      v, nb, Y);
    }
    check_launch("ladder_unpack");
    if (prof) {
      CK(cudaEventRecord(e1, st));
      ev.push_back({e0, e1});
      ++prof_calls;
      // algorithmic count: the (ac) <-> (bd) symmetric build v^2 (v^2 + 1) / 2 . 2J
      // plus the packed contraction 2 [Po Pv^2 + o(o-1)/2 (v(v-1)/2)^2] per vector
      const double vv = (double)v * v, pm = (double)v * (v - 1) / 2;
      prof_flops += vv * (vv + 1.0) / 2.0 * 2.0 * J +
                    2.0 * (double)nb * ((double)Po * Pv * Pv + (double)Pm * pm * pm);
    }
  }

  // adjoint of the ladder with respect to the Cholesky vectors (two-particle
  // density, vvvv block): out[J][(a c)] = sum_bd (D[a,b,c,d] + D[b,a,d,c]) L^J_bd
  // with D[a,b,c,d] = sum_n Yb[n][(a b)] X[n][(c d)], formed for a block of a
  // values at a time (the full v^4 D is never stored)
  void ladder_adj_l(const Graph& g, const double* L, const double* Yb, const double* X,
                    double* out) override {
    const int64_t o = g.o, v = g.v, J = g.J, n = o + v, vv = v * v, oo = o * o;
    double* Lvv = scratch(5, J * vv);  // Lvv[J][(b d)]
    {
      int64_t dims[3] = {J, v, v}, ostr[3] = {vv, v, 1}, istr[3] = {n * n, n, 1};
      copy_view(3, dims, Lvv, ostr, L + o * n + o, istr, 1.0, false);
    }
    const int64_t budget = (int64_t)1 << 26;  // doubles of one D block (512 MiB)
    for (int64_t a0 = 0; a0 < v;) {
      const int64_t na = std::max<int64_t>(1, std::min<int64_t>(v - a0, budget / (v * vv)));
      const int64_t rows = na * v;
      // D1[(a b)][(c d)] = sum_n Yb[n][(a b)] X[n][(c d)], a in the block
      MatView A1;
      A1.p = Yb + a0 * v;
      A1.sr2 = 1;
      A1.sk2 = vv;
      MatView B1;
      B1.p = X;
      B1.sr2 = 1;
      B1.sk2 = vv;
      double* D1 = scratch(3, rows * vv);
      gemm_view(1, rows, vv, oo, 1.0, A1, B1, D1, true);
      // D2[(a b)][(c d)] = sum_n Yb[n][(b a)] X[n][(d c)]
      MatView A2;
      A2.p = Yb + a0;
      A2.n2r = v;
      A2.sr1 = 1;
      A2.sr2 = v;
      A2.sk2 = vv;
      MatView B2;
      B2.p = X;
      B2.n2r = v;
      B2.sr1 = 1;
      B2.sr2 = v;
      B2.sk2 = vv;
      double* D2 = scratch(4, rows * vv);
      gemm_view(1, rows, vv, oo, 1.0, A2, B2, D2, true);
      {
        int64_t dims[1] = {rows * vv}, os[1] = {1};
        copy_view(1, dims, D1, os, D2, os, 1.0, true);
      }
      // op[(a c)][J] = sum_(b d) D[a][b][c][d] Lvv[J][(b d)]
      MatView A3;
      A3.p = D1;
      A3.n2r = v;
      A3.sr1 = v * vv;
      A3.sr2 = v;
      A3.n2k = v;
      A3.sk1 = vv;
      A3.sk2 = 1;
      double* op = scratch(6, rows * J);
      gemm_view(1, rows, J, vv, 1.0, A3, MatView::dense(Lvv, J, vv), op, true);
      int64_t dims[2] = {J, rows}, ostr[2] = {vv, 1}, istr[2] = {1, J};
      copy_view(2, dims, out + a0 * v, ostr, op, istr, 1.0, false);
      a0 += na;
    }
  }
};

std::unique_ptr<Backend> make_backend(void* stream, int precision) {
  return std::make_unique<CudaBackend>(stream, precision);
}

}  // namespace sccsd
