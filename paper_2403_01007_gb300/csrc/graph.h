// Tensor-operation graph with forward- and reverse-mode differentiation.
//
// The CCSD ground-state functions E0(t) and Omega(t) are written once as a
// static graph of FP64 tensor operations (contractions, permuted sums,
// sub-block copies and the particle-particle ladder). The quantities of the
// hot path are derivatives of these functions:
//   A R    = directional derivative of Omega along R         (forward mode)
//   A^T L  = gradient of L . Omega                           (reverse mode)
//   d_pq, Gamma^J_pq = gradients of <L|Hbar|R> w.r.t. h, L^J  (reverse over forward)
//   SCC X3 terms     = mixed second derivatives              (forward over forward)
// so the graph transforms below produce them mechanically. All operations
// are executed by the CUDA backend on the device; this file is host logic.
#pragma once

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

namespace sccsd {

constexpr int kMaxRank = 6;

enum class Kind { Input, Node, Zero };

struct Tensor {
  std::vector<int64_t> dims;
  Kind kind = Kind::Node;
  double* data = nullptr;   // device buffer (owned by the graph)
  int64_t version = 0;      // bumped whenever the contents change
  std::string name;
  int64_t numel() const {
    int64_t n = 1;
    for (auto d : dims) n *= d;
    return n;
  }
};

enum class OpKind { Contract, Add, Slice, Embed, Ladder, LadderAdjL };

struct Op {
  OpKind kind;
  int out = -1;
  std::vector<int> in;
  // Contract: out[lc] = alpha * sum A[la] B[lb];  tc = may run on tensor cores
  std::string la, lb, lc;
  double alpha = 1.0;
  bool tc = false;
  // Add: out[lc] = sum_k coef[k] * in[k] labelled perm[k]
  std::vector<double> coef;
  std::vector<std::string> perm;
  // Slice / Embed: offsets of the sub-block inside the larger tensor
  std::vector<int64_t> off;
  // execution memo
  std::vector<int64_t> seen;
  bool ran = false;
  double trace_ms = 0.0;
  int64_t trace_calls = 0;
  // tracing: operands converted for the tensor cores (bit 0 A, bit 1 B)
  int trace_conv = 0;
};

class Backend;

class Graph {
 public:
  std::vector<Tensor> t;
  std::vector<Op> ops;
  Backend* be = nullptr;
  int64_t clock = 0;
  // ladder support: vv block offset o and Cholesky dims are needed by the
  // backend; stored here for the executor
  int o = 0, v = 0, J = 0;

  ~Graph();

  // --- construction -------------------------------------------------------
  int input(const std::vector<int64_t>& dims, const std::string& name);
  int zero(const std::vector<int64_t>& dims);
  bool is_zero(int id) const { return t[id].kind == Kind::Zero; }

  // out[lc] = alpha * sum A[la] B[lb]; returns a Zero node if A or B is zero
  int contract(int A, const std::string& la, int B, const std::string& lb,
               const std::string& lc, double alpha = 1.0, bool tc = false);
  // out[lc] = sum coef_k * X_k[perm_k]; zero terms are dropped
  struct Term { int id; std::string perm; double coef; };
  int add(const std::string& lc, const std::vector<Term>& terms);
  int slice(int X, const std::vector<int64_t>& off, const std::vector<int64_t>& dims);
  int embed(int X, const std::vector<int64_t>& off, const std::vector<int64_t>& dims);
  // Y_ij^ab = sum_cd g_acbd X_ij^cd with g_acbd = sum_J L^J_ac L^J_bd (vv block)
  int ladder(int X, int L);
  int ladder_adj_l(int Ybar, int X, int L);

  // --- differentiation ------------------------------------------------------
  // Tangents of every node produced by ops [begin, end) given tangents of some
  // nodes (seeds). Returns node -> tangent node for all nodes with a non-zero
  // tangent (seeds included).
  // With nb > 0 every tangent carries an extra leading dimension of size nb
  // (label 'Z'): nb directions are propagated at once, and contractions with
  // a primal operand fold the batch into their row dimension.
  using Ranges = std::vector<std::pair<size_t, size_t>>;
  std::map<int, int> tangent(const std::map<int, int>& seeds, const Ranges& ranges,
                             int64_t nb = 0);
  // Adjoints: seeds map output node -> adjoint node; returns adjoint nodes of
  // the requested wrt nodes (Zero node if it does not depend on the seeds).
  // With nb > 0 the seeds (and all adjoints) carry a leading batch dimension;
  // the ops in ranges must then be unbatched.
  std::map<int, int> adjoint(const std::map<int, int>& seeds, const std::vector<int>& wrt,
                             const Ranges& ranges, int64_t nb = 0);

  // --- execution ------------------------------------------------------------
  void set_input(int id, const double* src, bool src_on_device);
  void touch(int id) { t[id].version = ++clock; }
  // Run the ops among [begin, end) that the target nodes need, skipping ops
  // whose inputs did not change since their last execution.
  void run(const std::vector<int>& targets);
  // Nodes that depend on the given inputs are recomputed on every run and
  // their buffers are recycled after their last use (inputs that change on
  // every call: trial vectors, bras, seeds). Call after the graph is built.
  void set_volatile_inputs(const std::vector<int>& inputs);
  // Forget all memoised results (e.g. after a change of arithmetic precision).
  void invalidate() {
    for (auto& op : ops) op.ran = false;
  }
  double* data(int id) { return t[id].data; }
  // Tracing: when enabled, every executed op is bracketed by events and its
  // time accumulated per op; trace_report() lists the most expensive ops.
  bool trace = false;
  std::string trace_report(int top = 40);

 private:
  int new_tensor(const std::vector<int64_t>& dims, Kind k);
  void exec(Op& op);
  void exec_contract(Op& op, double* out_data, const int64_t* ostr, double coef, bool acc);
  // one term of a permuted sum after planning: node x labelled by perm (in
  // the sum's labels), scaled by coef; fused >= 0: x is the output of that
  // contraction op, which is evaluated straight into the sum
  struct SumTerm {
    int node;
    std::string perm;
    double coef;
    int fused;
  };
  void exec_add(Op& op, const std::vector<SumTerm>& terms);
  std::vector<char> vol_;
  std::vector<int> held_;  // volatile buffers kept alive for the caller
};

}  // namespace sccsd
