// Launchers of the small dense linear algebra and vector kernels (small_la.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sccsd {

void launch_small_solve(cudaStream_t st, int m, const double* A, const double* b, double* x,
                        int* info);
void launch_small_eig(cudaStream_t st, int m, const double* H, double* wr, double* wi, double* Y,
                      int nwant, int* order, int* info, int allow_complex = 0);
void launch_diis(cudaStream_t st, int m, const double* B, double* c, int* info);
void launch_denoms(cudaStream_t st, int o, int v, const double* eps, double* D);
void launch_jacobi(cudaStream_t st, int64_t n, const double* t, const double* om, const double* D,
                   double* out);
void launch_precond(cudaStream_t st, int64_t n, const double* r, const double* D, double lam,
                    double* out);
void launch_axpby(cudaStream_t st, int64_t n, double a, const double* x, double b, double* y);
// d = max(d, frac * ref) elementwise
void launch_floor(cudaStream_t st, int64_t n, const double* ref, double frac, double* d);
// y = d * x elementwise
void launch_scale(cudaStream_t st, int64_t n, const double* d, const double* x, double* y);
void launch_ritz_residual(cudaStream_t st, int nr, int64_t n, const double* ax, const double* x,
                          const double* wr, const int* order, double* r);

}  // namespace sccsd

namespace sccsd {
void launch_learned_features(cudaStream_t st, int o, int v, const double* tmp2, const double* govov,
                             const double* eps, const double* f, double s_t, double s_g, double s_D,
                             float* X);
void launch_learned_targets(cudaStream_t st, int o, int v, const double* t, const double* eps,
                            const double* f, double s_t, float* Y);
void launch_learned_apply(cudaStream_t st, int o, int v, const float* Y, const double* eps, double s_t,
                          double* t2, double* d2);
}  // namespace sccsd
