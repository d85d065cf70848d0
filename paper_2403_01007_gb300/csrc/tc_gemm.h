// Tensor-core (tcgen05 / TMEM / TMA) contraction path for sm_103a.
//
// FP64 operands are split into BF16 slices x = x_0 + x_1 + ... (each slice the
// BF16 rounding of what the previous ones left over); slice products run as
// BF16 x BF16 -> FP32 GEMMs on the tensor cores and are summed into the FP64
// result. One slice (SCCSD_BF16) keeps about 8 significant bits per operand;
// two slices with the three leading products x0 y0 + x0 y1 + x1 y0
// (SCCSD_BF16X3) about 16, at which point the FP32 accumulation over long
// contractions is the limiting error.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "backend.h"
#include "tc_tune.h"

namespace sccsd {

// A matrix already converted to BF16 slices, rows padded to 256 and K to 64.
struct TcOperand {
  void* data = nullptr;   // slices back to back, each [rows_pad][k_pad] bf16
  int64_t rows = 0, k = 0, rows_pad = 0, k_pad = 0;
  int slices = 0;
  size_t bytes = 0;
};

// Epilogue of the learned part's layers (mlp_gemm below): BF16 activations
// and gradients, FP32 outputs, all dense row-major with the given leading
// dimensions (elements).
enum MlpMode {
  MLP_HIDDEN = 1,   // out = relu(acc + bias) as BF16 in out[row][col] and outT[col][row]
  MLP_OUTPUT = 2,   // outf[row][col] = acc + bias (FP32)
  MLP_RELU_BACK = 3,// out = acc where maskT[col][row] > 0, else 0; BF16 in out and outT
  MLP_PARTIAL = 4,  // outf[z][row][col] = acc of K split z (FP32, split stride rows * ldf)
};
struct MlpEpi {
  const float* bias = nullptr;
  uint16_t* out = nullptr;          // BF16 bits; may be null (modes 1, 3)
  int64_t ldo = 0;
  uint16_t* outT = nullptr;         // BF16 bits, transposed; may be null (modes 1, 3)
  int64_t ldt = 0;
  const uint16_t* maskT = nullptr;  // BF16 bits, transposed activations (mode 3)
  int64_t ldm = 0;
  float* outf = nullptr;            // modes 2, 4
  int64_t ldf = 0;
};

class TcGemm {
 public:
  TcGemm(cudaStream_t st, int precision);
  ~TcGemm();
  bool worthwhile(int64_t nb, int64_t M, int64_t N, int64_t K) const;
  // C[m][n] = alpha * sum_k A[m][k] B[n][k]  (FP64 in and out)
  void gemm(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
            const double* B, double* C);
  void prepare_operand(const double* X, int64_t rows, int64_t K, TcOperand& out);
  // same from a strided view (the permutation is folded into the conversion)
  void prepare_operand_view(const MatView& X, int64_t rows, int64_t K, TcOperand& out);
  // check: read back the pipeline error flag (synchronises the stream)
  void gemm_prepared_b(int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                       const TcOperand& B, double* C, bool check = true);
  void check_error();
  // C (= or +=) alpha * A B^T for operands already in slice form; C through
  // the output view ov. Small output grids split K over extra CTAs. The launch
  // shape comes from the process-wide tuning table, else from the fixed rule
  // (and is timed and recorded first when tuning is on).
  void gemm_ops(int64_t M, int64_t N, double alpha, const TcOperand& A, const TcOperand& B,
                double* C, const OutView& ov, bool accumulate);
  // the same with an explicit launch shape
  void execute(const TcConfig& cfg, int64_t M, int64_t N, double alpha, const TcOperand& A,
               const TcOperand& B, double* C, const OutView& ov, bool accumulate);
  // tuning off also frees the scratch output of the tuning runs
  void set_tune(bool on);
  void release(TcOperand& op);
  // an operand of `rows` rows (K = k) in slice form, all zero; its rows are
  // written later by a kernel (the ladder build below)
  void alloc_operand(int64_t rows, int64_t k, int slices, TcOperand& out);
  // Lt[(p, q)][J] = L^J_{o+p, o+q} (the virtual block of the Cholesky vectors,
  // L [J][n][n]) in slice form, with 256 spare rows after the v^2 used ones so
  // that the build kernel's tiles past the last row stay inside the buffer
  void prepare_ladder_lt(const double* L, int o, int v, int J, TcOperand& out);
  // largest v the fused ladder build handles (its shared-memory triangle)
  static int ladder_build_max_v();
  // G+ and G- rows of the pairs p_begin .. p_begin + npairs - 1 (pair table:
  // a << 16 | b, a <= b) from Lt, as slices of Gp and Gm (rows 0 .. npairs-1,
  // K = v (v + 1) / 2 packed (c <= d)); see k_ladder_build
  void ladder_build(const TcOperand& Lt, int v, const int* pairs, int64_t p_begin,
                    int64_t npairs, TcOperand& Gp, TcOperand& Gm);
  // One layer product of the learned part, C[M][N] = sum_k A[m][k] B[n][k],
  // with A and B BF16 row-major (leading dimensions lda, ldb elements, a
  // multiple of 8) holding a_rows >= M and b_rows >= N allocated rows, and the
  // epilogue `mode` (MlpMode). Contraction columns at or past K are read as
  // zero when K >= 64; for K < 64 columns K .. 63 must hold zeros. `splits`
  // splits K over more CTAs (mode MLP_PARTIAL only); returns the split count
  // used.
  int mlp_gemm(int mode, const void* A, int64_t a_rows, int64_t lda, const void* B,
               int64_t b_rows, int64_t ldb, int64_t M, int64_t N, int64_t K, int splits,
               const MlpEpi& e);
  int sm_count() const { return sm_count_; }
  int slices() const { return nslices_; }
  void set_precision(int precision) { nslices_ = precision == 1 ? 2 : 1; }

 private:
  void convert(const MatView& X, int64_t rows, int64_t K, TcOperand& out, int64_t spare = 0);
  void run(const TcOperand& A, int sa, const TcOperand& B, int sb, int64_t M, int64_t N,
           double alpha, double* C, int64_t split_stride, const OutView& ov, bool accumulate,
           int splits, int kbs, int variant, int nfast);
  TcConfig tune(const TcShape& s, int64_t M, int64_t N, double alpha, const TcOperand& A,
                const TcOperand& B, const OutView& ov, const TcConfig& fallback);
  cudaStream_t st_;
  int nslices_;
  TcOperand a_tmp_, b_tmp_;
  int sm_count_ = 1;         // persistent grid size
  double* part_ = nullptr;   // split-K partial results
  size_t part_bytes_ = 0;
  int* d_err_ = nullptr;
  bool tune_ = false;
  double* tune_buf_ = nullptr;   // scratch output of the tuning runs
  size_t tune_bytes_ = 0;
};

}  // namespace sccsd
