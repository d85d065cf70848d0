// Small dense FP64 linear algebra on the device, one thread block per problem:
// the DIIS equations and the Davidson subspace eigenproblem (dimension <= 48).
//
// * k_small_solve: Gaussian elimination with partial pivoting.
// * k_small_eig:   eigenvalues of a real non-symmetric matrix by reduction to
//   upper Hessenberg form (Householder reflections) followed by Francis
//   double-shift QR steps (implicit, with 3x3 reflectors chasing the bulge),
//   deflating converged 1x1 and 2x2 blocks (a complex-conjugate pair is
//   reported through wi != 0); right eigenvectors of the requested lowest real
//   eigenvalues by inverse iteration on the original matrix. These are the
//   textbook algorithms (Golub & Van Loan, Matrix Computations, Sec. 7.4-7.6).
#include <cuda_runtime.h>

#include <cstdint>

namespace sccsd {

constexpr int kSmallMax = 48;  // two matrices of this size fit the static shared memory

// x <- solution of A x = b (A is m x m row-major, overwritten); info = 1 if singular
__device__ void dev_solve(int m, double* A, double* b, int* info, double* piv_scratch) {
  __shared__ int s_piv;
  __shared__ double s_max;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double mx = fabs(A[k * m + k]);
      for (int i = k + 1; i < m; ++i)
        if (fabs(A[i * m + k]) > mx) {
          mx = fabs(A[i * m + k]);
          p = i;
        }
      s_piv = p;
      s_max = mx;
    }
    __syncthreads();
    if (s_max == 0.0) {
      if (threadIdx.x == 0) *info = 1;
      return;
    }
    const int p = s_piv;
    if (p != k) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double t = A[k * m + j];
        A[k * m + j] = A[p * m + j];
        A[p * m + j] = t;
      }
      if (threadIdx.x == 0) {
        double t = b[k];
        b[k] = b[p];
        b[p] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / A[k * m + k];
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) piv_scratch[i] = A[i * m + k] * inv;
    __syncthreads();
    for (int e = threadIdx.x; e < (m - k - 1) * (m - k); e += blockDim.x) {
      int i = k + 1 + e / (m - k), j = k + e % (m - k);
      A[i * m + j] -= piv_scratch[i] * A[k * m + j];
    }
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) b[i] -= piv_scratch[i] * b[k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int i = m - 1; i >= 0; --i) {
      double s = b[i];
      for (int j = i + 1; j < m; ++j) s -= A[i * m + j] * b[j];
      b[i] = s / A[i * m + i];
    }
    *info = 0;
  }
  __syncthreads();
}

__global__ void k_small_solve(int m, const double* __restrict__ A, const double* __restrict__ b,
                              double* __restrict__ x, int* info) {
  __shared__ double sA[kSmallMax * kSmallMax];
  __shared__ double sb[kSmallMax];
  __shared__ double sp[kSmallMax];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) sA[e] = A[e];
  for (int e = threadIdx.x; e < m; e += blockDim.x) sb[e] = b[e];
  __syncthreads();
  dev_solve(m, sA, sb, info, sp);
  for (int e = threadIdx.x; e < m; e += blockDim.x) x[e] = sb[e];
}

// Eigenvalues (wr, wi) of H (m x m, row-major) and unit right eigenvectors of
// the nwant real eigenvalues with the lowest real part (columns of Y, m x nwant,
// row-major [i][k]); order[k] = index into wr of the k-th wanted root.
// info: 0 ok, 2 = QR did not converge, 3 = a wanted root is complex. With
// allow_complex, a complex pair among the wanted roots gives info 4 instead,
// and the pair's two columns of Y span its real invariant plane: the first by
// inverse iteration at the real part, the second H x - Re(lambda) x of it,
// orthonormalised (a Davidson subspace can carry such pairs before its roots
// settle).
__global__ void k_small_eig(int m, const double* __restrict__ Hin, double* __restrict__ wr,
                            double* __restrict__ wi, double* __restrict__ Y, int nwant,
                            int* __restrict__ order, int* info, int allow_complex) {
  __shared__ double H[kSmallMax * kSmallMax];
  __shared__ double W[kSmallMax * kSmallMax];
  __shared__ double v[kSmallMax];
  __shared__ double x[kSmallMax];
  __shared__ double sp[kSmallMax];
  __shared__ double lr[kSmallMax], li[kSmallMax];
  __shared__ int sorder[kSmallMax];
  __shared__ int s_info;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * m; e += nt) H[e] = Hin[e];
  if (tid == 0) s_info = 0;
  __syncthreads();

  // --- Householder reduction to upper Hessenberg form
  for (int k = 0; k < m - 2; ++k) {
    __shared__ double s_alpha, s_vnorm2;
    if (tid == 0) {
      double nrm = 0.0;
      for (int i = k + 1; i < m; ++i) nrm += H[i * m + k] * H[i * m + k];
      nrm = sqrt(nrm);
      double a = H[(k + 1) * m + k];
      s_alpha = (a > 0) ? -nrm : nrm;
      for (int i = 0; i < m; ++i) v[i] = 0.0;
      if (nrm > 0.0) {
        v[k + 1] = a - s_alpha;
        for (int i = k + 2; i < m; ++i) v[i] = H[i * m + k];
      }
      double vn = 0.0;
      for (int i = k + 1; i < m; ++i) vn += v[i] * v[i];
      s_vnorm2 = vn;
    }
    __syncthreads();
    if (s_vnorm2 > 0.0) {
      const double beta = 2.0 / s_vnorm2;
      // H <- (I - beta v v^T) H
      for (int j = tid; j < m; j += nt) {
        double s = 0.0;
        for (int i = k + 1; i < m; ++i) s += v[i] * H[i * m + j];
        sp[j] = s;
      }
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {
        int i = e / m, j = e % m;
        if (i > k) H[e] -= beta * v[i] * sp[j];
      }
      __syncthreads();
      // H <- H (I - beta v v^T)
      for (int i = tid; i < m; i += nt) {
        double s = 0.0;
        for (int j = k + 1; j < m; ++j) s += H[i * m + j] * v[j];
        sp[i] = s;
      }
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {
        int i = e / m, j = e % m;
        if (j > k) H[e] -= beta * sp[i] * v[j];
      }
      __syncthreads();
    }
  }

  // --- Francis double-shift QR on the Hessenberg matrix (thread 0; m <= 48),
  // deflating 1x1 and 2x2 blocks; exceptional shifts every 10 iterations
  if (tid == 0) {
    int n = m;  // active rows/cols [l, n)
    int its = 0;
    const double eps = 2.220446049250313e-16;
    while (n > 0) {
      int l = n - 1;
      for (; l > 0; --l) {
        double s = fabs(H[(l - 1) * m + l - 1]) + fabs(H[l * m + l]);
        if (s == 0.0) s = 1.0;
        if (fabs(H[l * m + l - 1]) <= eps * s) {
          H[l * m + l - 1] = 0.0;
          break;
        }
      }
      if (l == n - 1) {  // 1x1 block
        lr[n - 1] = H[(n - 1) * m + n - 1];
        li[n - 1] = 0.0;
        n -= 1;
        its = 0;
        continue;
      }
      const double a = H[(n - 2) * m + n - 2], b = H[(n - 2) * m + n - 1];
      const double c = H[(n - 1) * m + n - 2], d = H[(n - 1) * m + n - 1];
      if (l == n - 2) {  // 2x2 block
        const double tr = a + d, det = a * d - b * c, disc = 0.25 * tr * tr - det;
        if (disc >= 0.0) {
          double r = sqrt(disc);
          lr[n - 2] = 0.5 * tr + r;
          lr[n - 1] = 0.5 * tr - r;
          li[n - 2] = li[n - 1] = 0.0;
        } else {
          double r = sqrt(-disc);
          lr[n - 2] = lr[n - 1] = 0.5 * tr;
          li[n - 2] = r;
          li[n - 1] = -r;
        }
        n -= 2;
        its = 0;
        continue;
      }
      if (++its > 60) {
        s_info = 2;
        break;
      }
      const int N = n - l;
      double s = a + d, t = a * d - b * c;
      if (its % 10 == 0) {  // exceptional shift
        double w = fabs(H[(n - 1) * m + n - 2]) + fabs(H[(n - 2) * m + n - 3]);
        double e = d + 0.75 * w;
        s = 2.0 * e;
        t = e * e - 0.4375 * w * w;
      }
      double x = H[l * m + l] * H[l * m + l] + H[l * m + l + 1] * H[(l + 1) * m + l] -
                 s * H[l * m + l] + t;
      double y = H[(l + 1) * m + l] * (H[l * m + l] + H[(l + 1) * m + l + 1] - s);
      double z = H[(l + 1) * m + l] * H[(l + 2) * m + l + 1];
      for (int k = 0; k < N - 2; ++k) {
        // Householder reflector sending (x, y, z) to a multiple of e1
        double nrm = sqrt(x * x + y * y + z * z);
        const int r0 = l + k, c0 = l + (k > 0 ? k - 1 : 0);
        if (nrm > 0.0) {
          double v0 = x + (x >= 0.0 ? nrm : -nrm), v1 = y, v2 = z;
          double beta = 2.0 / (v0 * v0 + v1 * v1 + v2 * v2);
          for (int j = c0; j < n; ++j) {
            double w = v0 * H[r0 * m + j] + v1 * H[(r0 + 1) * m + j] + v2 * H[(r0 + 2) * m + j];
            w *= beta;
            H[r0 * m + j] -= w * v0;
            H[(r0 + 1) * m + j] -= w * v1;
            H[(r0 + 2) * m + j] -= w * v2;
          }
          const int re = l + (k + 4 < N ? k + 4 : N);
          for (int i = l; i < re; ++i) {
            double w = H[i * m + r0] * v0 + H[i * m + r0 + 1] * v1 + H[i * m + r0 + 2] * v2;
            w *= beta;
            H[i * m + r0] -= w * v0;
            H[i * m + r0 + 1] -= w * v1;
            H[i * m + r0 + 2] -= w * v2;
          }
        }
        x = H[(r0 + 1) * m + r0];
        y = H[(r0 + 2) * m + r0];
        if (k < N - 3) z = H[(r0 + 3) * m + r0];
      }
      {
        double nrm = sqrt(x * x + y * y);
        if (nrm > 0.0) {
          double v0 = x + (x >= 0.0 ? nrm : -nrm), v1 = y;
          double beta = 2.0 / (v0 * v0 + v1 * v1);
          for (int j = n - 3; j < n; ++j) {
            double w = beta * (v0 * H[(n - 2) * m + j] + v1 * H[(n - 1) * m + j]);
            H[(n - 2) * m + j] -= w * v0;
            H[(n - 1) * m + j] -= w * v1;
          }
          for (int i = l; i < n; ++i) {
            double w = beta * (H[i * m + n - 2] * v0 + H[i * m + n - 1] * v1);
            H[i * m + n - 2] -= w * v0;
            H[i * m + n - 1] -= w * v1;
          }
        }
      }
    }
    // pick the nwant lowest real parts
    for (int i = 0; i < m; ++i) sorder[i] = i;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j)
        if (lr[sorder[j]] < lr[sorder[i]]) {
          int t = sorder[i];
          sorder[i] = sorder[j];
          sorder[j] = t;
        }
    for (int k = 0; k < nwant && s_info == 0; ++k)
      if (li[sorder[k]] != 0.0) s_info = allow_complex ? 4 : 3;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    wr[i] = lr[i];
    wi[i] = li[i];
  }
  for (int k = tid; k < nwant; k += nt) order[k] = sorder[k];
  if (s_info != 0 && s_info != 4) {
    if (tid == 0) *info = s_info;
    return;
  }
  // --- eigenvectors by inverse iteration on the original matrix
  for (int k = 0; k < nwant; ++k) {
    const double lam = lr[sorder[k]];
    const int ik = sorder[k];
    if (k > 0 && li[ik] != 0.0 && li[sorder[k - 1]] == -li[ik] && lr[sorder[k - 1]] == lam) {
      // second member of a complex pair: H x - lam x of the first (still in x)
      for (int i = tid; i < m; i += nt) {
        double y = -lam * x[i];
        for (int j = 0; j < m; ++j) y += Hin[i * m + j] * x[j];
        v[i] = y;
      }
      __syncthreads();
      if (tid == 0) {
        double dt = 0.0;
        for (int i = 0; i < m; ++i) dt += v[i] * x[i];
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) {
          v[i] -= dt * x[i];
          nrm += v[i] * v[i];
        }
        nrm = sqrt(nrm);
        int imax = 0;
        for (int i = 1; i < m; ++i)
          if (fabs(v[i]) > fabs(v[imax])) imax = i;
        const double sgn = v[imax] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < m; ++i) x[i] = nrm > 0.0 ? sgn * v[i] / nrm : 0.0;
      }
      __syncthreads();
      for (int i = tid; i < m; i += nt) Y[i * nwant + k] = x[i];
      __syncthreads();
      continue;
    }
    double scale = 0.0;
    for (int e = 0; e < m * m; ++e) scale = fmax(scale, fabs(Hin[e]));
    const double shift = lam + 1e-10 * fmax(1.0, scale);
    for (int i = tid; i < m; i += nt) x[i] = 1.0 / sqrt((double)m) * (1.0 + 0.01 * i);
    __syncthreads();
    for (int it = 0; it < 3; ++it) {
      for (int e = tid; e < m * m; e += nt) W[e] = Hin[e] - ((e / m == e % m) ? shift : 0.0);
      __syncthreads();
      __shared__ int sinfo;
      dev_solve(m, W, x, &sinfo, sp);
      __syncthreads();
      if (tid == 0) {
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
        nrm = sqrt(nrm);
        // sign convention: largest component positive
        int imax = 0;
        for (int i = 1; i < m; ++i)
          if (fabs(x[i]) > fabs(x[imax])) imax = i;
        double sgn = x[imax] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < m; ++i) x[i] = sgn * x[i] / nrm;
      }
      __syncthreads();
    }
    for (int i = tid; i < m; i += nt) Y[i * nwant + k] = x[i];
    __syncthreads();
  }
  if (tid == 0) *info = s_info;
}

}  // namespace sccsd

namespace sccsd {

// DIIS coefficients: minimise |sum c_k r_k| subject to sum c_k = 1, from the
// Gram matrix B_pq = r_p . r_q (Pulay): [B -1; -1 0] [c; l] = [0; -1].
// The matrix is scaled by its largest diagonal element for conditioning.
__global__ void k_diis(int m, const double* __restrict__ B, double* __restrict__ c, int* info) {
  __shared__ double A[(kSmallMax + 1) * (kSmallMax + 1)];
  __shared__ double b[kSmallMax + 1];
  __shared__ double sp[kSmallMax + 1];
  const int n = m + 1;
  __shared__ double scale;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < m; ++k) mx = fmax(mx, fabs(B[k * m + k]));
    scale = mx > 0.0 ? 1.0 / mx : 1.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    A[e] = (i < m && j < m) ? B[i * m + j] * scale : ((i == m && j == m) ? 0.0 : -1.0);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = (i == m) ? -1.0 : 0.0;
  __syncthreads();
  dev_solve(n, A, b, info, sp);
  for (int i = threadIdx.x; i < m; i += blockDim.x) c[i] = b[i];
}

void launch_small_solve(cudaStream_t st, int m, const double* A, const double* b, double* x,
                        int* info) {
  k_small_solve<<<1, 128, 0, st>>>(m, A, b, x, info);
}
void launch_small_eig(cudaStream_t st, int m, const double* H, double* wr, double* wi, double* Y,
                      int nwant, int* order, int* info, int allow_complex) {
  k_small_eig<<<1, 128, 0, st>>>(m, H, wr, wi, Y, nwant, order, info, allow_complex);
}
void launch_diis(cudaStream_t st, int m, const double* B, double* c, int* info) {
  k_diis<<<1, 128, 0, st>>>(m, B, c, info);
}

// ----------------------------------------------------------- vector kernels

// packed orbital-energy denominators: D_ai = e_a - e_i, D_aibj = D_ai + D_bj
__global__ void k_denoms(int o, int v, const double* __restrict__ eps, double* __restrict__ D) {
  const int64_t ov = (int64_t)o * v, np = ov * (ov + 1) / 2;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ov + np;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < ov) {
      D[k] = eps[o + k / o] - eps[k % o];
      continue;
    }
    int64_t q = k - ov;
    int64_t Q = (int64_t)((sqrtf((float)(8 * q + 1)) - 1.0f) * 0.5f);
    while (Q * (Q + 1) / 2 > q) --Q;
    while ((Q + 1) * (Q + 2) / 2 <= q) ++Q;
    int64_t P = q - Q * (Q + 1) / 2;
    D[k] = (eps[o + P / o] - eps[P % o]) + (eps[o + Q / o] - eps[Q % o]);
  }
}

// out = t - om / D
__global__ void k_jacobi(int64_t n, const double* __restrict__ t, const double* __restrict__ om,
                         const double* __restrict__ D, double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = t[k] - om[k] / D[k];
}

// out = r / (lam - D), the diagonal (Davidson) preconditioner with a floor
__global__ void k_precond(int64_t n, const double* __restrict__ r, const double* __restrict__ D,
                          double lam, double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double d = lam - D[k];
    if (fabs(d) < 1e-4) d = d < 0 ? -1e-4 : 1e-4;
    out[k] = r[k] / d;
  }
}

// y = a x + b y
__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b,
                        double* __restrict__ y) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    y[k] = a * x[k] + b * y[k];
}

// d = max(d, frac * ref) elementwise (a floor for refreshed denominators)
__global__ void k_floor(int64_t n, const double* __restrict__ ref, double frac,
                        double* __restrict__ d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double f = frac * ref[k];
    d[k] = d[k] > f ? d[k] : f;
  }
}

// y = d * x elementwise
__global__ void k_scale(int64_t n, const double* __restrict__ d, const double* __restrict__ x,
                        double* __restrict__ y) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    y[k] = d[k] * x[k];
}

// y_k = x_k - lam_k-weighted: r[k][:] = ax[k][:] - lam[order[k]] * x[k][:]
__global__ void k_ritz_residual(int nr, int64_t n, const double* __restrict__ ax,
                                const double* __restrict__ x, const double* __restrict__ wr,
                                const int* __restrict__ order, double* __restrict__ r) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nr * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(e / n);
    r[e] = ax[e] - wr[order[k]] * x[e];
  }
}

static int vgrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

void launch_denoms(cudaStream_t st, int o, int v, const double* eps, double* D) {
  int64_t ov = (int64_t)o * v;
  k_denoms<<<vgrid(ov + ov * (ov + 1) / 2), 256, 0, st>>>(o, v, eps, D);
}
void launch_jacobi(cudaStream_t st, int64_t n, const double* t, const double* om, const double* D,
                   double* out) {
  k_jacobi<<<vgrid(n), 256, 0, st>>>(n, t, om, D, out);
}
void launch_precond(cudaStream_t st, int64_t n, const double* r, const double* D, double lam,
                    double* out) {
  k_precond<<<vgrid(n), 256, 0, st>>>(n, r, D, lam, out);
}
void launch_axpby(cudaStream_t st, int64_t n, double a, const double* x, double b, double* y) {
  k_axpby<<<vgrid(n), 256, 0, st>>>(n, a, x, b, y);
}
void launch_floor(cudaStream_t st, int64_t n, const double* ref, double frac, double* d) {
  k_floor<<<vgrid(n), 256, 0, st>>>(n, ref, frac, d);
}
void launch_scale(cudaStream_t st, int64_t n, const double* d, const double* x, double* y) {
  k_scale<<<vgrid(n), 256, 0, st>>>(n, d, x, y);
}
void launch_ritz_residual(cudaStream_t st, int nr, int64_t n, const double* ax, const double* x,
                          const double* wr, const int* order, double* r) {
  k_ritz_residual<<<vgrid((int64_t)nr * n), 256, 0, st>>>(nr, n, ax, x, wr, order, r);
}

}  // namespace sccsd

namespace sccsd {

// Per-amplitude features of the learned guess, for every full doubles element
// (i, j, a, b) (row index ((i*o + j)*v + a)*v + b), all symmetric under
// (ia) <-> (jb):
//   0 t_MP2 / st   1 g_iajb / sg   2 g_ibja / sg   3 D / sD   4 log D
//   5 log(D'_MP2 / D)   6 (e_a + e_b)/2   7 (e_i + e_j)/2   8 |e_a - e_b|   9 |e_i - e_j|
// with D = e_a + e_b - e_i - e_j and D' the same from the diagonals f of the
// dressed intermediates at the MP2 amplitudes.
__global__ void k_learned_features(int o, int v, const double* __restrict__ tmp2,
                                   const double* __restrict__ govov, const double* __restrict__ eps,
                                   const double* __restrict__ f, double st, double sg, double sD,
                                   float* __restrict__ X) {
  const int64_t total = (int64_t)o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % v, r1 = e / v, a = r1 % v, r2 = r1 / v, j = r2 % o, i = r2 / o;
    const double ea = eps[o + a], eb = eps[o + b], ei = eps[i], ej = eps[j];
    const double D = ea + eb - ei - ej;
    const double Dp = f[o + a] + f[o + b] - f[i] - f[j];
    const double exch = govov[((i * o + j) * v + b) * v + a];
    float* x = X + e * 10;
    x[0] = (float)(tmp2[e] / st);
    x[1] = (float)(govov[e] / sg);
    x[2] = (float)(exch / sg);
    x[3] = (float)(D / sD);
    x[4] = (float)log(D);
    x[5] = (float)log(fmax(Dp, 1e-3) / D);
    x[6] = (float)(0.5 * (ea + eb));
    x[7] = (float)(0.5 * (ei + ej));
    x[8] = (float)fabs(ea - eb);
    x[9] = (float)fabs(ei - ej);
  }
}

// targets: y0 = t / st, y1 = log(D'/D) for every full doubles element
__global__ void k_learned_targets(int o, int v, const double* __restrict__ t,
                                  const double* __restrict__ eps, const double* __restrict__ f,
                                  double st, float* __restrict__ Y) {
  const int64_t total = (int64_t)o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % v, r1 = e / v, a = r1 % v, r2 = r1 / v, j = r2 % o, i = r2 / o;
    const double D = eps[o + a] + eps[o + b] - eps[i] - eps[j];
    const double Dp = f[o + a] + f[o + b] - f[i] - f[j];
    Y[e * 2] = (float)(t[e] / st);
    Y[e * 2 + 1] = (float)log(fmax(Dp, 1e-3) / D);
  }
}

// network outputs -> full doubles guess t = y0 * st and preconditioner
// D_prec = D * exp(y1) (clamped to [D/4, 8 D])
__global__ void k_learned_apply(int o, int v, const float* __restrict__ Y,
                                const double* __restrict__ eps, double st, double* __restrict__ t2,
                                double* __restrict__ d2) {
  const int64_t total = (int64_t)o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % v, r1 = e / v, a = r1 % v, r2 = r1 / v, j = r2 % o, i = r2 / o;
    const double D = eps[o + a] + eps[o + b] - eps[i] - eps[j];
    t2[e] = (double)Y[e * 2] * st;
    double s = exp((double)Y[e * 2 + 1]);
    d2[e] = D * fmin(8.0, fmax(0.25, s));
  }
}

void launch_learned_features(cudaStream_t st, int o, int v, const double* tmp2, const double* govov,
                             const double* eps, const double* f, double s_t, double s_g, double s_D,
                             float* X) {
  k_learned_features<<<vgrid((int64_t)o * o * v * v), 256, 0, st>>>(o, v, tmp2, govov, eps, f, s_t,
                                                                    s_g, s_D, X);
}
void launch_learned_targets(cudaStream_t st, int o, int v, const double* t, const double* eps,
                            const double* f, double s_t, float* Y) {
  k_learned_targets<<<vgrid((int64_t)o * o * v * v), 256, 0, st>>>(o, v, t, eps, f, s_t, Y);
}
void launch_learned_apply(cudaStream_t st, int o, int v, const float* Y, const double* eps, double s_t,
                          double* t2, double* d2) {
  k_learned_apply<<<vgrid((int64_t)o * o * v * v), 256, 0, st>>>(o, v, Y, eps, s_t, t2, d2);
}

}  // namespace sccsd
