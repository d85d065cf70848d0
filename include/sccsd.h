/* C ABI of the SCCSD hot path (closed-shell similarity constrained CCSD).
 *
 * Paper: "Nuclear gradients and nonadiabatic couplings for similarity
 * constrained coupled cluster singles and doubles" (arXiv 2403.01007).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * o, v, J  occupied and virtual spatial orbitals, Cholesky rank; n = o + v.
 * eps[n]   orbital energies of a canonical closed-shell HF reference, the o
 *          occupied first; the Fock matrix is diag(eps) (Brillouin condition
 *          F_ai = 0, the last constraint of the Lagrangian of Sec. 2.3.1).
 * L[J][n][n]  Cholesky vectors, g_pqrs = sum_J L^J_pq L^J_rs, each L^J
 *          symmetric in pq. The one-electron integrals are derived so that
 *          F = diag(eps):  h_pq = eps_p d_pq - sum_k (2 g_pqkk - g_pkkq).
 * packed vectors (length dim = ov + ov(ov+1)/2, double):
 *          singles first, x[a*o + i]; then the doubles over unique compound
 *          pairs P = a*o + i <= Q = b*o + j at x[ov + Q(Q+1)/2 + P].
 *          Kets (t, R): T = sum_ai t_ai E_ai + 1/2 sum_{ai,bj} t_aibj E_ai E_bj
 *          with t_aibj = t_bjai (= t_ij^ab = t_ji^ba).
 *          Bras (Omega, L, sigma of the left transform) live in the
 *          biorthonormal basis <mu~|nu> = d_mu,nu, so <L|R> = sum_mu L_mu R_mu.
 * pointers: every array argument may be host or device memory (detected per
 *          call); the caller owns all of them. The context owns its internal
 *          device buffers. Work is queued on the stream given to sccsd_init and
 *          every call returns after that stream has finished the call's work.
 * errors:  0 on success, a negative SCCSD_E* code otherwise; the text of the
 *          last failure is returned by sccsd_last_error(ctx). No exception
 *          crosses this interface. A failed call leaves the outputs undefined.
 */
#ifndef SCCSD_H
#define SCCSD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sccsd_ctx sccsd_ctx;

enum {
  SCCSD_OK = 0,
  SCCSD_EINVAL = -1,   /* bad size, NULL pointer, bad mode */
  SCCSD_ENOMEM = -2,   /* device allocation failed */
  SCCSD_ECUDA = -3,    /* a CUDA call or kernel failed */
  SCCSD_ESTATE = -4,   /* call order: e.g. a Jacobian before any residual */
  SCCSD_EINTERNAL = -5,
  SCCSD_ENOTCONV = -6, /* an iterative solver hit its iteration limit */
  SCCSD_ECOMPLEX = -7  /* a complex-conjugate pair among the wanted EOM roots */
};

/* Precision of the tensor-core-eligible contractions (ladder, rings,
 * integral products). SCCSD_FP64: all arithmetic in FP64 on CUDA cores.
 * SCCSD_BF16X3: each FP64 operand split into two BF16 slices x = x0 + x1 (x1
 * the BF16 rounding of x - x0), the three products x0 y0 + x0 y1 + x1 y0 on
 * tcgen05 tensor cores with FP32 accumulation, summed in FP64 (about 16
 * significant bits per product; FP32 accumulation over long contractions then
 * dominates the error). SCCSD_BF16: one BF16 slice per operand. */
enum { SCCSD_FP64 = 0, SCCSD_BF16X3 = 1, SCCSD_BF16 = 2 };

/* Create a context for one synthetic system (sizes, eps, L as above).
 * Computes h (the integrals of a canonical reference) and the HF energy.
 * stream: a cudaStream_t, or NULL for the default stream. SCCSD_EINVAL for
 * non-positive sizes, a bad precision, eps not finite, not ascending within
 * the occupied and virtual blocks or without a gap between them, and L not
 * finite or not symmetric in pq (to 1e-12 of its largest entry). */
int sccsd_init(sccsd_ctx** ctx, int o, int v, int J, const double* eps, const double* L,
               int precision, void* stream);

/* Ground-state energy and residual at amplitudes t (packed ket):
 *   E0 = <HF|Hbar|HF>,  omega_mu = <mu~|Hbar|HF>   (Sec. 2.1),
 * with Hbar = exp(-T) H exp(T). With Ra and Rb non-NULL (packed kets of the two
 * constrained states a, b) the cluster operator is T + zeta X3,
 * X3 = R1^a R2^b - R1^b R2^a (Sec. 2.4.1), which adds
 * zeta <mu~|[Hhat, X3]|HF> to omega (Sec. 2.4.2); E0 is unchanged by it.
 * Outputs: omega (packed bra, may be NULL), e_corr = E0 - E_HF (may be NULL).
 * The call also fixes t (and zeta, Ra, Rb) as the state at which the
 * Jacobians and densities below are evaluated. */
int sccsd_residual(sccsd_ctx* ctx, const double* t, double zeta, const double* Ra,
                   const double* Rb, double* omega, double* e_corr);

/* sigma_k = A R_k for nvec packed kets R[nvec][dim], with
 * A_mu,nu = <mu~|[Hbar, tau_nu]|HF> (Sec. 2.3.3), at the state fixed by the
 * last sccsd_residual call (SCC terms included when it had them).
 * Also returns eta.R_k in etaR[nvec] when etaR is non-NULL (eta of Sec. 2.3.3).
 * nvec = 0 does nothing and returns SCCSD_OK (R and sigma may then be NULL);
 * nvec < 0 is SCCSD_EINVAL. */
int sccsd_jacobian_right(sccsd_ctx* ctx, int nvec, const double* R, double* sigma,
                         double* etaR);

/* sigma_k = A^T L_k (the left transformation) for nvec packed bras: the
 * left EOM problem of Sec. 2.1 and the A^T products of the multiplier
 * equations (Sec. 2.3.3), at the fixed state. nvec = 0 does nothing (L and
 * sigma may be NULL); nvec < 0 is SCCSD_EINVAL; SCCSD_ESTATE before any
 * sccsd_residual. */
int sccsd_jacobian_left(sccsd_ctx* ctx, int nvec, const double* L, double* sigma);

/* One- and two-particle (transition) densities of Sec. 2.3.2 for the bra
 * (l0, L) and ket (r0, R) at the fixed state:
 *   D1[p][q]       = d_pq = <L|exp(-T) E_pq exp(T)|R>
 *   Gamma[J][p][q] = sum_rs d_pqrs L^J_rs,  d_pqrs = <L|exp(-T) e_pqrs exp(T)|R>
 * (with the SCC state the cluster operator includes zeta X3, which gives the
 * Delta d corrections of Sec. 2.4.2). Gamma may be NULL. */
int sccsd_densities(sccsd_ctx* ctx, double l0, const double* L, double r0, const double* R,
                    double* D1, double* Gamma);

/* Dense contraction utility on the library's own kernels:
 *   C[m][n] = alpha * sum_k A[m][k] B[n][k]   (row-major, FP64 in and out)
 * on CUDA cores (SCCSD_FP64) or on tcgen05 tensor cores with BF16 slices
 * (SCCSD_BF16X3 / SCCSD_BF16, used when the product is large enough). All three
 * pointers must be device memory; the call returns after the work finished.
 * This is the contraction primitive of the hot path, exposed for validation
 * (an interface of this library; the paper has no counterpart). SCCSD_EINVAL
 * for negative sizes, a NULL or host pointer or a bad precision; M or N = 0
 * writes nothing, K = 0 sets C to zero. */
int sccsd_gemm_tn(int precision, long long M, long long N, long long K, double alpha,
                  const double* A, const double* B, double* C, void* stream);

/* Profiling (instrumentation of this library; the paper has no counterpart).
 * sccsd_profile(ctx, 1) resets the counters and starts timing
 * every particle-particle ladder call (the vvvv integrals built from the
 * Cholesky vectors, packing, contraction) with CUDA events on the context's
 * stream; 0 stops it. sccsd_profile_read returns the summed ladder time in ms,
 * the number of ladder calls, their algorithmic flop count (the (ac) <-> (bd)
 * symmetric build v^2 (v^2 + 1) / 2 . 2J per call plus the +- packed
 * contraction 2 [P_o P_v^2 + o(o-1)/2 (v(v-1)/2)^2] per trial vector, P_x =
 * x(x+1)/2; trial vectors are batched up to 8 per call) and the number of
 * kernels this library launched since the reset (any output may be NULL).
 * Timing adds one stream synchronisation per read. */
int sccsd_profile(sccsd_ctx* ctx, int enable);
int sccsd_profile_read(sccsd_ctx* ctx, double* ladder_ms, long long* ladder_calls,
                       double* ladder_flops, long long* launches);

/* The same FP64 contraction, C[m][n] = alpha * sum_k A[m][k] B[n][k], for
 * callers that must not trigger device allocations: applications that give
 * all device memory to their own pool allocator up front and forbid further
 * cudaMalloc calls, and latency-critical callers that cannot take the implicit
 * device synchronisation of cudaMalloc/cudaFree. (The paper has no
 * counterpart; this is an interface of this library.)
 * It calls no cudaMalloc, cudaFree or allocating library routine: the split-K
 * partial sums live in a file-scope device array of
 * sccsd_gemm_tn_noalloc_capacity() doubles (8 MiB), which every device that
 * loads the library holds until exit. The first call on a device looks up that
 * array's device address and the device's multiprocessor count (with the
 * device current), so make it before any stream capture. Both are cached for
 * the life of the process: after cudaDeviceReset on a device the cached
 * address is stale, so do not call this entry point on that device again.
 * Sizes as for sccsd_gemm_tn: negative sizes or a NULL pointer give
 * SCCSD_EINVAL, M or N = 0 writes nothing, K = 0 sets C to zero. M*N above the
 * capacity is rejected with SCCSD_EINVAL before any CUDA call; larger K only
 * lowers the number of K chunks. A, B and C must be device memory.
 * All calls share the one array: calls that overlap on the GPU (two streams,
 * two host threads) race on it, so serialise them. Every partial sum is written
 * before it is read, so stale contents from the previous call do no harm.
 * The work is enqueued on `stream` in order and the call returns without
 * waiting for it: C is ready once the stream reaches that point. A launch
 * failure is returned as SCCSD_ECUDA; a fault during execution shows up at the
 * caller's next synchronisation of the stream. */
int sccsd_gemm_tn_noalloc(long long M, long long N, long long K, double alpha, const double* A,
                          const double* B, double* C, void* stream);
long long sccsd_gemm_tn_noalloc_capacity(void);

/* SCC orthogonality of the natural projection (Sec. 2.4.1, 2.4.2):
 *   O_ab = <psi_a|P|psi_b>,  psi = exp(T) (R0 |HF> + sum_mu R_mu |mu>),
 * P the projector onto HF, singles and doubles, T the cluster operator of the
 * fixed state without X3 (the triples part does not reach the projected
 * space). States a, b are given by (ra0, Ra) and (rb0, Rb), Ra/Rb packed kets.
 * The inner product is that of the Hilbert space (the metric of the singlet
 * singles and doubles kets included). Result in *O. */
int sccsd_overlap(sccsd_ctx* ctx, double ra0, const double* Ra, double rb0, const double* Rb,
                  double* O);

/* SCC orthogonality with the state projection P = sum_kl |R_k> (S^-1)_kl <R_l|
 * over K = {a, b} (Sec. 2.4.1), S_kl = <R_k|R_l>, |R_k> = R0_k |HF> + R_k:
 *   O_ab = sum_kl <psi_a|R_k> (S^-1)_kl <R_l|psi_b>,
 * with psi and the inner product as for sccsd_overlap. Result in *O;
 * SCCSD_EINVAL if R_a and R_b are linearly dependent. */
int sccsd_overlap_states(sccsd_ctx* ctx, double ra0, const double* Ra, double rb0,
                         const double* Rb, double* O);

/* The projection sccsd_solve_scc constrains: 0 the natural projection
 * (SCCSD(E), the default), 1 the state projection (SCCSD(K)), Sec. 2.4.1.
 * sccsd_solve_multipliers and sccsd_multiplier_residual use the same choice
 * for the gbar O_ab term of the Lagrangian. */
int sccsd_set_projection(sccsd_ctx* ctx, int projection);

/* Self-consistent SCCSD for the two lowest states, K = {a, b} (Sec. 2.4.2):
 * find zeta with O_ab = 0 (Sec. 2.2). For each zeta the ground state is
 * converged with zeta X3 built from the current R_a, R_b (ground_tol), the two
 * lowest right EOM roots of the SCC Jacobian follow (eom_tol), with
 * R0 = eta.R / omega (block form of the EOM matrix, Sec. 2.1) and state vectors
 * of unit norm with their largest component positive; zeta is updated by the
 * secant method on O_ab, starting from zeta = 0 (plain CCSD), which selects
 * the root connected to CCSD (the paper notes the equation may have several,
 * Sec. 3.1.1). Converged when |O_ab| < tol and the zeta step is below 1e-8.
 * In a mixed-precision context the inner solves finish in FP64, and r0 and
 * O_ab, which decide zeta, are evaluated in FP64.
 * Outputs (may be NULL): zeta, e_corr, omega2[2], r0_2[2], Ra/Rb (packed),
 * iterations. Afterwards the fixed state is the SCC state of the last zeta. */
int sccsd_solve_scc(sccsd_ctx* ctx, double tol, int maxit, double ground_tol, double eom_tol,
                    double* zeta, double* e_corr, double* omega2, double* r0_2, double* Ra,
                    double* Rb, int* iterations);

/* More than two constrained states (Sec. 2.2 with K = {1..n}; the X3 form of
 * Sec. 2.4.1 for every pair). The cluster operator is
 *   T + sum_{k<l} zeta_kl X_kl,   X_kl = R1^k R2^l - R1^l R2^k,
 * for n >= 2 packed kets R[n][dim] (host or device) and zeta[n(n-1)/2] (host)
 * in the pair order (0,1), (0,2), ..., (0,n-1), (1,2), ... Only
 * sum_{k<l} zeta_kl <mu~|[Hhat, X_kl]|HF> reaches omega; E0 is unchanged.
 * With n = 2 this is sccsd_residual with (zeta, Ra, Rb) = (zeta_01, R_0, R_1).
 * sccsd_residual_states fixes (t, the states) like sccsd_residual: the
 * transformations, densities and overlaps that follow use it. Errors:
 * SCCSD_EINVAL for n < 2, NULL arguments or a non-finite zeta. */
int sccsd_residual_states(sccsd_ctx* ctx, const double* t, int nstates, const double* zeta,
                          const double* R, double* omega, double* e_corr);
/* The ground state with the X3 terms of n states (otherwise as
 * sccsd_solve_ground, including refinement in a mixed precision). */
int sccsd_solve_ground_states(sccsd_ctx* ctx, const double* t0, int nstates, const double* zeta,
                              const double* R, double tol, int maxit, double refine_tol,
                              double* t_out, double* e_corr, int* iterations);
/* O_kl for every pair k < l of nstates states (R0_k = r0[k], packed kets
 * R[nstates][dim], host or device) at the fixed state, in the pair order of
 * sccsd_residual_states: projection 0 the natural projection (as
 * sccsd_overlap), 1 the state projection over all nstates states (Sec. 2.4.1),
 * O_kl = sum_jm <psi_k|R_j> (S^-1)_jm <R_m|psi_l>, S_jm = <R_j|R_m>, with
 * psi and the inner product as for sccsd_overlap. SCCSD_EINVAL for linearly
 * dependent states. */
int sccsd_overlaps(sccsd_ctx* ctx, int nstates, const double* r0, const double* R, int projection,
                   double* O);
/* Self-consistent SCCSD for the nstates (2..8) lowest states: zeta_kl for
 * every pair solves O_kl = 0 (the projection of sccsd_set_projection: natural,
 * or the state projection over all nstates states) by Broyden's method from
 * zeta = 0 (plain CCSD) with the unit matrix as the first Jacobian estimate;
 * at every zeta the ground state (ground_tol) and the n lowest right roots
 * (eom_tol, unit norm, largest component positive) are re-converged.
 * Converged when max |O_kl| < tol and the last zeta step is below 1e-8.
 * Outputs (may be NULL): zeta and O [n(n-1)/2], e_corr, omega [n], r0 [n],
 * R [n][dim] (host or device), iterations. Afterwards the fixed state is that
 * of the last zeta. */
int sccsd_solve_scc_states(sccsd_ctx* ctx, int nstates, double tol, int maxit, double ground_tol,
                           double eom_tol, double* zeta, double* O, double* e_corr, double* omega,
                           double* r0, double* R, int* iterations);

/* Switch the precision of the tensor-core-eligible contractions for later
 * calls (SCCSD_FP64 / SCCSD_BF16X3 / SCCSD_BF16). An implementation choice: the
 * paper's program is FP64 throughout. SCCSD_EINVAL for another value. */
int sccsd_set_precision(sccsd_ctx* ctx, int precision);

/* Launch-shape tuning of the tensor-core contractions (an implementation
 * choice, not part of the method: results are the same contraction up to the
 * FP32 summation order of split K ranges).
 * Each contraction has a fixed default launch shape: kernel variant (four or
 * eight epilogue warps), order of the output tiles, number of K ranges. With
 * tuning enabled on a context (enable = 1), the first contraction of each
 * new shape (M, padded N, K blocks, slices, output view, accumulate mode, SM
 * count) outside graph capture times every candidate shape on its operands,
 * into a scratch buffer, so the caller's outputs are not touched. The fastest
 * shape is recorded in a table shared by all contexts of the process and used
 * by every later contraction of that shape, whether or not tuning is enabled.
 * Tune before sccsd_capture_transform, which only reads the table. The
 * scratch buffer of the tuning runs (as large as the largest output tuned)
 * is held until tuning is switched off (enable = 0) or the context is
 * destroyed; do not switch tuning while a captured graph of the context runs.
 * No effect in SCCSD_FP64 mode.
 * sccsd_autotune_export writes the table as text, one line per shape, into
 * buf[cap] (NUL-terminated). *len receives the bytes needed, NUL included.
 * SCCSD_EINVAL if buf is NULL or cap is too small (*len is still set).
 * sccsd_autotune_import merges a text written by export. On a malformed line,
 * or a shape the library never launches, it merges nothing and returns
 * SCCSD_EINVAL. sccsd_autotune_clear empties the table;
 * sccsd_autotune_entries returns its size. These four take no context and
 * run on the host. */
int sccsd_set_autotune(sccsd_ctx* ctx, int enable);
int sccsd_autotune_export(char* buf, long long cap, long long* len);
int sccsd_autotune_import(const char* text);
void sccsd_autotune_clear(void);
long long sccsd_autotune_entries(void);

/* Ground state: converge Omega(t) = 0 (Sec. 2.1; with Ra/Rb non-NULL the SCC
 * residual of sccsd_residual at fixed zeta) by the preconditioned update
 * t <- t - Omega/D with DIIS (8 vectors). D starts as the orbital-energy
 * denominators D_ai = e_a - e_i, D_aibj = D_ai + D_bj (or the preconditioner
 * of sccsd_set_preconditioner) and is replaced after two iterations, and then
 * at doubling intervals, by the dressed denominators D' built the same way from
 * the diagonals of the dressed Fock-like intermediates at the current
 * amplitudes (floored at 0.2 D; DIIS restarts with each refresh). Starts from
 * t0 (packed ket) or from zero (whose first step is the MP2 guess). With a mixed precision and
 * refine_tol > 0 the iterations run in that precision until |Omega| <
 * refine_tol, or until they stall (no 10% improvement in 6 iterations: the
 * noise floor of the mixed arithmetic), and are then refined by defect
 * correction: the FP64 residual r = Omega(t) is formed, A d = -r is solved
 * with the mixed-precision Jacobian (Jacobi preconditioner with DIIS, to 1e-4
 * of |r| for SCCSD_BF16X3 and 1e-2 for SCCSD_BF16), and t <- t + d; each round
 * gains about the mixed arithmetic's relative accuracy. A round that gains
 * less than 3x hands the remaining iterations to FP64. The FP64 residual
 * decides convergence (|Omega|_2 < tol). Outputs (each may be NULL):
 * t_out (packed), e_corr, iterations. The converged state is fixed for the
 * Jacobian and density calls. SCCSD_ENOTCONV when maxit is reached (outputs
 * hold the last iterate). */
int sccsd_solve_ground(sccsd_ctx* ctx, const double* t0, double zeta, const double* Ra,
                       const double* Rb, double tol, int maxit, double refine_tol,
                       double* t_out, double* e_corr, int* iterations);

/* The nroots (<= 12) EOM roots omega of lowest real part (Sec. 2.1:
 * A R = omega R for side 0, L^T A = omega L^T for side 1) at the fixed state,
 * by the Davidson method with a subspace of at most 48 vectors and the
 * diagonal preconditioner (omega - D')^-1, D' built from the diagonals of the
 * dressed one-body intermediates (f_a - f_i for singles, f_a + f_b - f_i - f_j
 * for doubles); restarts keep the current and previous Ritz vectors. The
 * subspace eigenproblem and all vector work run on the device. Convergence: |A x - omega x| / |x| < tol for every
 * root. Mixed precisions refine once every residual is below refine_tol or the
 * residuals stall for 8 iterations (refine_tol <= 0: no refinement): the
 * subspace restarts from the Ritz vectors with their FP64 images (an FP64
 * anchor), later expansion vectors are transformed in the mixed precision
 * (their error scales with the corrections), and convergence is accepted
 * only on a subspace of FP64 images alone, i.e. after a fresh anchor. Outputs: omega[nroots],
 * vecs[nroots][dim] (unit-norm packed vectors, may be NULL), iterations.
 * The subspace holds min(48, dim) vectors and needs room for 2 nroots + 2,
 * else SCCSD_EINVAL.
 * SCCSD_ECOMPLEX if a complex pair appears among the wanted roots;
 * SCCSD_ENOTCONV when maxit is reached (outputs hold the last Ritz pairs). */
int sccsd_solve_states(sccsd_ctx* ctx, int nroots, int side, double tol, int maxit,
                       double refine_tol, double* omega, double* vecs, int* iterations);

/* Biorthonormal scaling of left eigenvectors (Sec. 2.1: the left and right
 * EOM vectors of a state satisfy <L_k|R_k> = 1; with the biorthonormal bra
 * basis the bracket is the plain dot product of the packed vectors):
 *   L_k <- L_k / (L_k . R_k),  k = 0 .. nvec-1,
 * R [nvec][dim] packed kets, L [nvec][dim] packed bras, overwritten in place;
 * host or device pointers; FP64 dot products on the device. nvec = 0 does
 * nothing. SCCSD_EINVAL for a NULL pointer, nvec < 0, or a dot product that is
 * zero or not finite (L is then left scaled up to the offending k). */
int sccsd_normalize_left(sccsd_ctx* ctx, int nvec, const double* R, double* L);

/* ---- Learned initial guess and preconditioner ----------------------------
 * A per-amplitude MLP (BF16 weights and activations, FP32 accumulation; every
 * layer product on the tcgen05 tensor cores with bias, ReLU and the backward
 * mask fused into the product's epilogue) maps MP2-level features of each
 * doubles amplitude to (t_ij^ab / s_t,
 * log(D'_ij^ab / D_ij^ab)): a guess for the converged amplitude and for the
 * dressed denominator D' (the diagonal of the Jacobian estimated from the
 * intermediates) used as the ground-state preconditioner. The plain solver
 * decides the result: the guess only sets the starting point and the update
 * preconditioner, and callers fall back to t0 = 0 (MP2 first step) and D.
 * (An extension of the method, not in the paper.) */
typedef struct sccsd_mlp sccsd_mlp;

/* Network with n_in inputs, n_hidden_layers hidden layers of width hidden
 * (ReLU), n_out outputs; He-uniform initialisation from a splitmix64 stream. */
int sccsd_mlp_create(sccsd_mlp** net, int n_in, int hidden, int n_hidden_layers, int n_out,
                     unsigned long long seed, void* stream);
void sccsd_mlp_destroy(sccsd_mlp* net);
const char* sccsd_mlp_last_error(sccsd_mlp* net);
long long sccsd_mlp_num_params(sccsd_mlp* net);
/* parameters as one host FP32 array, per layer W[in][out] then b[out] */
int sccsd_mlp_get_params(sccsd_mlp* net, float* params);
int sccsd_mlp_set_params(sccsd_mlp* net, const float* params);
/* Y[N][n_out] = net(X[N][n_in]); device FP32 arrays */
int sccsd_mlp_forward(sccsd_mlp* net, const float* X, long long N, float* Y);
/* gradient of the mean-squared error against T[N][n_out] (host FP32 array
 * laid out like the parameters) and the loss */
int sccsd_mlp_gradient(sccsd_mlp* net, const float* X, const float* T, long long N, float* grad,
                       float* loss);
/* one Adam step (beta 0.9/0.999) on the minibatch; loss before the step */
int sccsd_mlp_train_step(sccsd_mlp* net, const float* X, const float* T, long long N, float lr,
                         float* loss);

/* Features X[o^2 v^2][10] (device FP32) of every full doubles element
 * (i,j,a,b), evaluated at the MP2 amplitudes; scales[3] = (s_t, s_g, s_D).
 * Leaves the fixed state at the MP2 amplitudes. */
int sccsd_learned_features(sccsd_ctx* ctx, float* X, double* scales);
/* Training targets Y[o^2 v^2][2] (device FP32) from converged amplitudes t. */
int sccsd_learned_targets(sccsd_ctx* ctx, const double* t, double s_t, float* Y);
/* Packed initial amplitudes t0 and packed preconditioner Dprec proposed by net. */
int sccsd_learned_guess(sccsd_ctx* ctx, sccsd_mlp* net, double* t0, double* Dprec);
/* Initial denominators of sccsd_solve_ground's update (packed, positive), or
 * NULL for the orbital-energy denominators D. The solver replaces them by its
 * own dressed denominators D' (from the dressed Fock diagonals at the current
 * amplitudes) at its first refresh, after two iterations. SCCSD_EINVAL (and
 * the previous setting kept) if an entry is not finite and positive. */
int sccsd_set_preconditioner(sccsd_ctx* ctx, const double* Dprec);

/* ---- Lagrangian multipliers (gradients and couplings) ---------------------
 * sccsd_solve_multipliers solves the stationarity equations of the SCCSD
 * Lagrangian (Sec. 2.3.1 and 2.3.3 of the paper) for K = {a, b} with the
 * context's projection (sccsd_set_projection; natural by default), at fixed
 * orbitals (no orbital multipliers), for
 *   kind 0: the gradient of state n_state (0 = a, 1 = b), or
 *   kind 1: the derivative coupling <psi_m|d psi_n> from the bra-frozen
 *           overlap O_mn (Sec. 2.3.4), m_state != n_state.
 * Inputs describe the converged SCCSD solution:
 *   vecs [5][dim] packed: t, R_a, R_b (right EOM vectors, kets), L_a, L_b
 *        (left EOM vectors normalised so that L_k . R_k = 1, bras);
 *   scal [5]: zeta, r0_a, r0_b, omega_a, omega_b  (r0 = eta . R / omega).
 * Outputs (any may be NULL; host or device memory):
 *   zbar [dim]   ground-state multipliers (a bra);
 *   K [2][dim]   the gauge-free excited-state bras
 *                K_k = (delta_kn - <Lbar_k|R_k>) L_k + Lbar_k (no delta_kn for
 *                a coupling; Sec. 2.3.2); Lbar_k itself is fixed only up to
 *                multiples of L_k, which do not enter any result;
 *   out_scal [5] gbar, Lbar0_a, Lbar0_b, Ebar_a, Ebar_b (Ebar in the gauge
 *                Lbar_k . R_k = 0, i.e. Lbar_k = K_k - (delta_kn -
 *                Lbar0_k r0_k) L_k);
 *   D1 [n][n], Gamma [J][n][n]  derivatives of the Lagrangian with respect to
 *                h_pq and L^J_pq: the effective densities of the gradient or
 *                coupling (Gamma needs D1).
 * Solver: right-preconditioned restarted GMRES on the affine stationarity map,
 * with an FP64 residual driving correction solves in the context's precision
 * when that is mixed and refine_tol > 0 (after two correction rounds in a row
 * that cut the FP64 residual by less than a factor 10, the remaining ones are
 * solved in FP64); maxit bounds the number of applications of the map. Returns SCCSD_ENOTCONV (outputs hold the last
 * iterate) when the FP64 residual norm does not reach tol. */
int sccsd_solve_multipliers(sccsd_ctx* ctx, const double* vecs, const double* scal, int kind,
                            int m_state, int n_state, double tol, int maxit, double refine_tol,
                            double* zbar, double* K, double* out_scal, double* D1,
                            double* Gamma, int* iterations);
/* Derivative of a gradient or coupling along a perturbation of the
 * integrals (Sec. 2.3.2: the effective densities are the derivatives of the
 * Lagrangian with respect to h and L^J, so at fixed orbitals)
 *   *out = sum_pq D1[p][q] h1[p][q] + sum_Jpq Gamma[J][p][q] L1[J][p][q],
 * with D1, Gamma from sccsd_solve_multipliers and h1 [n][n], L1 [J][n][n] the
 * change of h and L^J per unit of the perturbation (Gamma and L1 may both be
 * NULL). Computed by FP64 reductions on the device in every precision mode.
 * For a perturbation of eps and L through sccsd_init, h1 includes the change
 * of h that L1 causes (h is derived from eps and L). */
int sccsd_integral_derivative(sccsd_ctx* ctx, const double* D1, const double* Gamma,
                              const double* h1, const double* L1, double* out);
/* The same along a perturbation of this library's inputs: deps [n] and dL
 * [J][n][n] (symmetric in pq; dL and Gamma may both be NULL) per unit of the
 * perturbation. h follows eps and L as in sccsd_init, so h1 = diag(deps) plus
 * the first-order change of -2 sum_J L^J s_J + sum_Jk L^J_pk L^J_kq
 * (s_J = sum_k L^J_kk over occupied k), formed by the library's kernels. */
int sccsd_input_derivative(sccsd_ctx* ctx, const double* D1, const double* Gamma,
                           const double* deps, const double* dL, double* out);
/* The packed amplitudes t (Sec. 2.1) of the context's current state (the
 * last sccsd_residual, or the result of a solver), e.g. the SCCSD ground state
 * after sccsd_solve_scc. SCCSD_ESTATE before any state exists. */
int sccsd_state_amplitudes(sccsd_ctx* ctx, double* t);
/* The stationarity residual r [3 dim + 1] = (d/dt, d/dR_a, d/dR_b, d/dzeta)
 * of the Lagrangian at the unknowns u [3 dim + 1] = (zbar, Lbar_a, Lbar_b,
 * gbar), with the closed forms for Lbar0_k and Ebar_k substituted: the
 * stationarity conditions of Sec. 2.3.3 (gradient) or Sec. 2.3.4 (coupling),
 * the map the solver drives to zero; same inputs as sccsd_solve_multipliers. */
int sccsd_multiplier_residual(sccsd_ctx* ctx, const double* vecs, const double* scal, int kind,
                              int m_state, int n_state, const double* u, double* r);

/* ---- CUDA graphs: many instances in one launch --------------------------
 * sccsd_capture_transform records W = A V (side 0, V packed kets, as
 * sccsd_jacobian_right) or W = A^T V (side 1, V packed bras, as
 * sccsd_jacobian_left) for nvec vectors at the fixed state of ctx into a CUDA
 * graph (cudaGraph_t, returned as void*); the call first runs the transform
 * once uncaptured, which sizes every buffer. Batching is an interface of this
 * library (the transforms are those of Sec. 2.1); the paper has no
 * counterpart. SCCSD_EINVAL for host vectors, a context on the default
 * stream or bad sizes; SCCSD_ESTATE before any sccsd_residual; the join and
 * launch calls return SCCSD_EINVAL for NULL arguments and SCCSD_ECUDA for a
 * failed CUDA call. V and W must be device memory and stay
 * valid while the graph is used; a launch reads V as it is then. The
 * context needs its own (non-default) stream. The graph reuses the context's
 * internal buffers: do not run other calls on the same context while a launch
 * of its graph is in flight.
 * sccsd_graph_join instantiates one executable graph with the n graphs as
 * independent child graphs (e.g. one per instance of a batch of uneven
 * systems), so that a single sccsd_graph_launch runs them all concurrently.
 * sccsd_graph_launch enqueues on the given stream and returns immediately. */
int sccsd_capture_transform(sccsd_ctx* ctx, int side, int nvec, const double* V, double* W,
                            void** graph);
int sccsd_graph_join(void** graphs, int n, void** exec);
int sccsd_graph_launch(void* exec, void* stream);
void sccsd_graph_destroy(void* graph);
void sccsd_graph_exec_destroy(void* exec);

/* Size of a packed vector, ov + ov(ov+1)/2 (the singles and doubles of
 * Sec. 2.1). */
long long sccsd_dim(int o, int v);
/* Text of the last failure on ctx (owned by ctx, valid until its next call),
 * the text of an error code, and the release of a context with every device
 * buffer it owns (NULL is ignored). */
const char* sccsd_last_error(sccsd_ctx* ctx);
const char* sccsd_strerror(int code);
void sccsd_destroy(sccsd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SCCSD_H */
