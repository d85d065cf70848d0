// Graph construction, differentiation and execution (host logic).
#include "graph.h"

#include <algorithm>
#include <cstdio>
#include <stdexcept>

#include "backend.h"

namespace sccsd {

namespace {

std::vector<int64_t> row_strides(const std::vector<int64_t>& d) {
  std::vector<int64_t> s(d.size());
  int64_t acc = 1;
  for (int k = (int)d.size() - 1; k >= 0; --k) {
    s[k] = acc;
    acc *= d[k];
  }
  return s;
}

void check_labels(const std::string& l, size_t rank, const char* what) {
  if (l.size() != rank) throw std::runtime_error(std::string("label/rank mismatch in ") + what);
  for (size_t a = 0; a < l.size(); ++a)
    for (size_t b = a + 1; b < l.size(); ++b)
      if (l[a] == l[b]) throw std::runtime_error(std::string("repeated label in ") + what);
}

}  // namespace

Graph::~Graph() {
  if (!be) return;
  for (auto& x : t)
    if (x.data) be->release(x.data);
}

int Graph::new_tensor(const std::vector<int64_t>& dims, Kind k) {
  if (dims.size() > (size_t)kMaxRank) throw std::runtime_error("rank too large");
  Tensor x;
  x.dims = dims;
  x.kind = k;
  t.push_back(x);
  return (int)t.size() - 1;
}

int Graph::input(const std::vector<int64_t>& dims, const std::string& name) {
  int id = new_tensor(dims, Kind::Input);
  t[id].name = name;
  return id;
}

int Graph::zero(const std::vector<int64_t>& dims) { return new_tensor(dims, Kind::Zero); }

int Graph::contract(int A, const std::string& la, int B, const std::string& lb,
                    const std::string& lc, double alpha, bool tc) {
  check_labels(la, t[A].dims.size(), "contract A");
  check_labels(lb, t[B].dims.size(), "contract B");
  std::vector<int64_t> dims;
  for (char c : lc) {
    size_t pa = la.find(c), pb = lb.find(c);
    if (pa == std::string::npos && pb == std::string::npos)
      throw std::runtime_error("output label missing from operands");
    dims.push_back(pa != std::string::npos ? t[A].dims[pa] : t[B].dims[pb]);
  }
  for (size_t pa = 0; pa < la.size(); ++pa) {
    size_t pb = lb.find(la[pa]);
    if (pb != std::string::npos && t[A].dims[pa] != t[B].dims[pb])
      throw std::runtime_error("contracted dimension mismatch");
    if (pb == std::string::npos && lc.find(la[pa]) == std::string::npos)
      throw std::runtime_error("label summed over one operand only");
  }
  for (char c : lb)
    if (la.find(c) == std::string::npos && lc.find(c) == std::string::npos)
      throw std::runtime_error("label summed over one operand only");
  check_labels(lc, dims.size(), "contract C");
  if (is_zero(A) || is_zero(B) || alpha == 0.0) return zero(dims);
  int out = new_tensor(dims, Kind::Node);
  Op op;
  op.kind = OpKind::Contract;
  op.out = out;
  op.in = {A, B};
  op.la = la;
  op.lb = lb;
  op.lc = lc;
  op.alpha = alpha;
  op.tc = tc;
  ops.push_back(op);
  return out;
}

int Graph::add(const std::string& lc, const std::vector<Term>& terms) {
  std::vector<int64_t> dims(lc.size(), -1);
  Op op;
  op.kind = OpKind::Add;
  op.lc = lc;
  for (auto& tm : terms) {
    check_labels(tm.perm, t[tm.id].dims.size(), "add term");
    if (tm.perm.size() != lc.size()) throw std::runtime_error("add: rank mismatch");
    for (size_t k = 0; k < lc.size(); ++k) {
      size_t p = tm.perm.find(lc[k]);
      if (p == std::string::npos) throw std::runtime_error("add: label mismatch");
      int64_t d = t[tm.id].dims[p];
      if (dims[k] >= 0 && dims[k] != d) throw std::runtime_error("add: dim mismatch");
      dims[k] = d;
    }
    if (is_zero(tm.id) || tm.coef == 0.0) continue;
    op.in.push_back(tm.id);
    op.coef.push_back(tm.coef);
    op.perm.push_back(tm.perm);
  }
  if (op.in.empty()) return zero(dims);
  int out = new_tensor(dims, Kind::Node);
  op.out = out;
  ops.push_back(op);
  return out;
}

int Graph::slice(int X, const std::vector<int64_t>& off, const std::vector<int64_t>& dims) {
  if (off.size() != t[X].dims.size() || dims.size() != off.size())
    throw std::runtime_error("slice rank");
  for (size_t k = 0; k < dims.size(); ++k)
    if (off[k] < 0 || off[k] + dims[k] > t[X].dims[k]) throw std::runtime_error("slice bounds");
  if (is_zero(X)) return zero(dims);
  int out = new_tensor(dims, Kind::Node);
  Op op;
  op.kind = OpKind::Slice;
  op.out = out;
  op.in = {X};
  op.off = off;
  ops.push_back(op);
  return out;
}

int Graph::embed(int X, const std::vector<int64_t>& off, const std::vector<int64_t>& dims) {
  if (off.size() != t[X].dims.size() || dims.size() != off.size())
    throw std::runtime_error("embed rank");
  for (size_t k = 0; k < dims.size(); ++k)
    if (off[k] < 0 || off[k] + t[X].dims[k] > dims[k]) throw std::runtime_error("embed bounds");
  if (is_zero(X)) return zero(dims);
  int out = new_tensor(dims, Kind::Node);
  Op op;
  op.kind = OpKind::Embed;
  op.out = out;
  op.in = {X};
  op.off = off;
  ops.push_back(op);
  return out;
}

int Graph::ladder(int X, int L) {
  const auto& d = t[X].dims;
  if (d.size() != 4 || d[0] != o || d[1] != o || d[2] != v || d[3] != v)
    throw std::runtime_error("ladder operand must be [o][o][v][v]");
  if (is_zero(X)) return zero(d);
  int out = new_tensor(d, Kind::Node);
  Op op;
  op.kind = OpKind::Ladder;
  op.out = out;
  op.in = {X, L};
  op.tc = true;
  ops.push_back(op);
  return out;
}

int Graph::ladder_adj_l(int Ybar, int X, int L) {
  std::vector<int64_t> d = {J, v, v};
  if (is_zero(Ybar) || is_zero(X)) return zero(d);
  int out = new_tensor(d, Kind::Node);
  Op op;
  op.kind = OpKind::LadderAdjL;
  op.out = out;
  op.in = {Ybar, X, L};
  op.tc = true;
  ops.push_back(op);
  return out;
}

// ---------------------------------------------------------------- tangents

std::map<int, int> Graph::tangent(const std::map<int, int>& seeds, const Ranges& ranges) {
  std::map<int, int> tan;
  for (auto& kv : seeds)
    if (!is_zero(kv.second)) tan[kv.first] = kv.second;
  auto T = [&](int id) -> int {
    auto it = tan.find(id);
    return it == tan.end() ? -1 : it->second;
  };
  std::vector<size_t> order;
  for (auto& r : ranges)
    for (size_t i = r.first; i < r.second; ++i) order.push_back(i);
  for (size_t i : order) {
    Op op = ops[i];  // copy: ops grows below
    int d = -1;
    switch (op.kind) {
      case OpKind::Contract: {
        int A = op.in[0], B = op.in[1];
        int dA = T(A), dB = T(B);
        int c1 = dA >= 0 ? contract(dA, op.la, B, op.lb, op.lc, op.alpha, op.tc) : -1;
        int c2 = dB >= 0 ? contract(A, op.la, dB, op.lb, op.lc, op.alpha, op.tc) : -1;
        if (c1 >= 0 && is_zero(c1)) c1 = -1;
        if (c2 >= 0 && is_zero(c2)) c2 = -1;
        if (c1 >= 0 && c2 >= 0)
          d = add(op.lc, {{c1, op.lc, 1.0}, {c2, op.lc, 1.0}});
        else
          d = c1 >= 0 ? c1 : c2;
        break;
      }
      case OpKind::Add: {
        std::vector<Term> terms;
        for (size_t k = 0; k < op.in.size(); ++k) {
          int dk = T(op.in[k]);
          if (dk >= 0) terms.push_back({dk, op.perm[k], op.coef[k]});
        }
        if (!terms.empty()) d = add(op.lc, terms);
        break;
      }
      case OpKind::Slice: {
        int dx = T(op.in[0]);
        if (dx >= 0) d = slice(dx, op.off, t[op.out].dims);
        break;
      }
      case OpKind::Embed: {
        int dx = T(op.in[0]);
        if (dx >= 0) d = embed(dx, op.off, t[op.out].dims);
        break;
      }
      case OpKind::Ladder: {
        if (T(op.in[1]) >= 0) throw std::runtime_error("ladder: tangent w.r.t. L not supported");
        int dx = T(op.in[0]);
        if (dx >= 0) d = ladder(dx, op.in[1]);
        break;
      }
      case OpKind::LadderAdjL:
        if (T(op.in[0]) >= 0 || T(op.in[1]) >= 0 || T(op.in[2]) >= 0)
          throw std::runtime_error("ladder_adj_l: tangent not supported");
        break;
    }
    if (d >= 0 && !is_zero(d)) tan[op.out] = d;
  }
  return tan;
}

// ---------------------------------------------------------------- adjoints

std::map<int, int> Graph::adjoint(const std::map<int, int>& seeds, const std::vector<int>& wrt,
                                  const Ranges& ranges) {
  std::vector<size_t> order;
  for (auto& r : ranges)
    for (size_t i = r.first; i < r.second; ++i) order.push_back(i);
  std::sort(order.begin(), order.end());
  std::vector<char> dep(t.size(), 0);
  for (int w : wrt) dep[w] = 1;
  for (size_t i : order)
    for (int x : ops[i].in)
      if (dep[x]) dep[ops[i].out] = 1;
  std::map<int, std::vector<int>> contrib;
  for (auto& kv : seeds)
    if (!is_zero(kv.second) && dep[kv.first]) contrib[kv.first].push_back(kv.second);

  auto total = [&](int id) -> int {
    auto it = contrib.find(id);
    if (it == contrib.end() || it->second.empty()) return -1;
    auto& v = it->second;
    if (v.size() == 1) return v[0];
    std::string l;
    for (size_t k = 0; k < t[id].dims.size(); ++k) l.push_back(char('A' + k));
    std::vector<Term> terms;
    for (int c : v) terms.push_back({c, l, 1.0});
    int s = add(l, terms);
    v.assign(1, s);
    return s;
  };
  auto push = [&](int id, int c) {
    if (c >= 0 && !is_zero(c)) contrib[id].push_back(c);
  };

  for (size_t q = order.size(); q-- > 0;) {
    Op op = ops[order[q]];
    if (!dep[op.out]) continue;
    int g = total(op.out);
    if (g < 0) continue;
    switch (op.kind) {
      case OpKind::Contract: {
        int A = op.in[0], B = op.in[1];
        if (dep[A]) push(A, contract(g, op.lc, B, op.lb, op.la, op.alpha, op.tc));
        if (dep[B]) push(B, contract(A, op.la, g, op.lc, op.lb, op.alpha, op.tc));
        break;
      }
      case OpKind::Add:
        for (size_t k = 0; k < op.in.size(); ++k)
          if (dep[op.in[k]]) push(op.in[k], add(op.perm[k], {{g, op.lc, op.coef[k]}}));
        break;
      case OpKind::Slice:
        if (dep[op.in[0]]) push(op.in[0], embed(g, op.off, t[op.in[0]].dims));
        break;
      case OpKind::Embed:
        if (dep[op.in[0]]) push(op.in[0], slice(g, op.off, t[op.in[0]].dims));
        break;
      case OpKind::Ladder: {
        int X = op.in[0], L = op.in[1];
        if (dep[X]) push(X, ladder(g, L));
        if (dep[L]) {
          int a = ladder_adj_l(g, X, L);
          push(L, embed(a, {0, (int64_t)o, (int64_t)o}, t[L].dims));
        }
        break;
      }
      case OpKind::LadderAdjL:
        throw std::runtime_error("ladder_adj_l: second adjoint not supported");
    }
  }
  std::map<int, int> res;
  for (int w : wrt) {
    int s = total(w);
    res[w] = s >= 0 ? s : zero(t[w].dims);
  }
  return res;
}

// ---------------------------------------------------------------- execution

void Graph::set_input(int id, const double* src, bool src_on_device) {
  Tensor& x = t[id];
  if (x.kind != Kind::Input) throw std::runtime_error("set_input on a non-input");
  if (!x.data) x.data = be->alloc(std::max<int64_t>(1, x.numel()));
  be->upload(x.data, src, x.numel(), src_on_device);
  touch(id);
}

void Graph::run(const std::vector<int>& targets) {
  // producer of each node
  std::vector<int> prod(t.size(), -1);
  for (size_t i = 0; i < ops.size(); ++i) prod[ops[i].out] = (int)i;
  std::vector<char> need_op(ops.size(), 0), seen_node(t.size(), 0);
  std::vector<int> stack;
  for (int x : targets)
    if (!seen_node[x]) {
      seen_node[x] = 1;
      stack.push_back(x);
    }
  while (!stack.empty()) {
    int x = stack.back();
    stack.pop_back();
    int p = prod[x];
    if (p < 0) continue;
    need_op[p] = 1;
    for (int y : ops[p].in)
      if (!seen_node[y]) {
        seen_node[y] = 1;
        stack.push_back(y);
      }
  }
  for (size_t i = 0; i < ops.size(); ++i) {
    if (!need_op[i]) continue;
    Op& op = ops[i];
    bool need = !op.ran;
    if (!need)
      for (size_t k = 0; k < op.in.size(); ++k)
        if (t[op.in[k]].version != op.seen[k]) {
          need = true;
          break;
        }
    if (!need) continue;
    for (int x : op.in)
      if (t[x].kind == Kind::Input && !t[x].data)
        throw std::runtime_error("graph input '" + t[x].name + "' was never set");
    void* e0 = trace ? be->record_event() : nullptr;
    exec(op);
    if (trace) {
      void* e1 = be->record_event();
      op.trace_ms += be->elapsed_ms(e0, e1);
      op.trace_calls += 1;
    }
    op.seen.resize(op.in.size());
    for (size_t k = 0; k < op.in.size(); ++k) op.seen[k] = t[op.in[k]].version;
    op.ran = true;
    touch(op.out);
  }
}

std::string Graph::trace_report(int top) {
  std::vector<size_t> idx;
  double total = 0.0;
  for (size_t i = 0; i < ops.size(); ++i)
    if (ops[i].trace_calls) {
      idx.push_back(i);
      total += ops[i].trace_ms;
    }
  std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return ops[a].trace_ms > ops[b].trace_ms; });
  static const char* names[] = {"contract", "add", "slice", "embed", "ladder", "ladder_adj_l"};
  std::string out = "op trace: total " + std::to_string(total) + " ms\n";
  for (int k = 0; k < top && k < (int)idx.size(); ++k) {
    const Op& op = ops[idx[k]];
    char line[512];
    std::string dims;
    for (int x : op.in) {
      dims += "[";
      for (auto d : t[x].dims) dims += std::to_string(d) + ",";
      dims += "]";
    }
    snprintf(line, sizeof line, "%8.3f ms %6lld x  op%-5zu %-12s %s,%s->%s tc=%d %s\n", op.trace_ms,
             (long long)op.trace_calls, idx[k], names[(int)op.kind], op.la.c_str(), op.lb.c_str(),
             op.lc.c_str(), (int)op.tc, dims.c_str());
    out += line;
  }
  return out;
}

void Graph::exec(Op& op) {
  Tensor& out = t[op.out];
  if (!out.data) out.data = be->alloc(std::max<int64_t>(1, out.numel()));
  const int rc = (int)out.dims.size();
  switch (op.kind) {
    case OpKind::Add: {
      auto ostr = row_strides(out.dims);
      for (size_t k = 0; k < op.in.size(); ++k) {
        const Tensor& x = t[op.in[k]];
        auto xs = row_strides(x.dims);
        int64_t istr[kMaxRank];
        for (int q = 0; q < rc; ++q) istr[q] = xs[op.perm[k].find(op.lc[q])];
        be->copy_view(rc, out.dims.data(), out.data, ostr.data(), x.data, istr, op.coef[k], k > 0);
      }
      if (rc == 0 && op.in.empty()) be->fill(out.data, 1, 0.0);
      break;
    }
    case OpKind::Slice: {
      const Tensor& x = t[op.in[0]];
      auto xs = row_strides(x.dims);
      int64_t base = 0;
      for (int q = 0; q < rc; ++q) base += op.off[q] * xs[q];
      auto ostr = row_strides(out.dims);
      be->copy_view(rc, out.dims.data(), out.data, ostr.data(), x.data + base, xs.data(), 1.0, false);
      break;
    }
    case OpKind::Embed: {
      const Tensor& x = t[op.in[0]];
      auto os = row_strides(out.dims);
      int64_t base = 0;
      for (int q = 0; q < rc; ++q) base += op.off[q] * os[q];
      be->fill(out.data, out.numel(), 0.0);
      auto xs = row_strides(x.dims);
      be->copy_view(rc, x.dims.data(), out.data + base, os.data(), x.data, xs.data(), 1.0, false);
      break;
    }
    case OpKind::Ladder:
      be->ladder(*this, t[op.in[1]].data, t[op.in[1]].version, t[op.in[0]].data, out.data);
      break;
    case OpKind::LadderAdjL:
      be->ladder_adj_l(*this, t[op.in[2]].data, t[op.in[0]].data, t[op.in[1]].data, out.data);
      break;
    case OpKind::Contract: {
      const Tensor& A = t[op.in[0]];
      const Tensor& B = t[op.in[1]];
      const std::string &la = op.la, &lb = op.lb, &lc = op.lc;
      std::string bat, ml, nl;
      for (char c : lc) {
        bool ia = la.find(c) != std::string::npos, ib = lb.find(c) != std::string::npos;
        if (ia && ib)
          bat.push_back(c);
        else if (ia)
          ml.push_back(c);
        else
          nl.push_back(c);
      }
      std::string ka, kb;  // contracted labels in A's order / in B's order
      for (char c : la)
        if (lb.find(c) != std::string::npos && lc.find(c) == std::string::npos) ka.push_back(c);
      for (char c : lb)
        if (la.find(c) != std::string::npos && lc.find(c) == std::string::npos) kb.push_back(c);
      // choose the contracted-label order that needs fewer operand copies
      auto cost = [&](const std::string& k) {
        int64_t c = 0;
        if (la != bat + ml + k) c += A.numel();
        if (lb != bat + nl + k) c += B.numel();
        return c;
      };
      std::string kl = cost(ka) <= cost(kb) ? ka : kb;
      auto dim_of = [&](char c) -> int64_t {
        size_t p = la.find(c);
        if (p != std::string::npos) return A.dims[p];
        return B.dims[lb.find(c)];
      };
      int64_t nb = 1, M = 1, N = 1, K = 1;
      for (char c : bat) nb *= dim_of(c);
      for (char c : ml) M *= dim_of(c);
      for (char c : nl) N *= dim_of(c);
      for (char c : kl) K *= dim_of(c);
      // bring an operand into [batch][rows][K] order
      auto arrange = [&](const Tensor& X, const std::string& lx, const std::string& want,
                         int slot) -> const double* {
        if (lx == want) return X.data;
        double* dst = be->scratch(slot, std::max<int64_t>(1, X.numel()));
        std::vector<int64_t> wd;
        for (char c : want) wd.push_back(X.dims[lx.find(c)]);
        auto ws = row_strides(wd);
        auto xs = row_strides(X.dims);
        int64_t istr[kMaxRank];
        for (size_t q = 0; q < want.size(); ++q) istr[q] = xs[lx.find(want[q])];
        be->copy_view((int)want.size(), wd.data(), dst, ws.data(), X.data, istr, 1.0, false);
        return dst;
      };
      const double* Ap = arrange(A, la, bat + ml + kl, 0);
      const double* Bp = arrange(B, lb, bat + nl + kl, 1);
      if (lc == bat + ml + nl) {
        be->gemm_tn(nb, M, N, K, op.alpha, Ap, Bp, out.data, op.tc);
      } else if (lc == bat + nl + ml) {
        be->gemm_tn(nb, N, M, K, op.alpha, Bp, Ap, out.data, op.tc);
      } else {
        double* Cp = be->scratch(2, std::max<int64_t>(1, nb * M * N));
        be->gemm_tn(nb, M, N, K, op.alpha, Ap, Bp, Cp, op.tc);
        std::string cl = bat + ml + nl;
        std::vector<int64_t> cd;
        for (char c : cl) cd.push_back(dim_of(c));
        auto cs = row_strides(cd);
        auto os = row_strides(out.dims);
        int64_t istr[kMaxRank];
        for (int q = 0; q < rc; ++q) istr[q] = cs[cl.find(lc[q])];
        be->copy_view(rc, out.dims.data(), out.data, os.data(), Cp, istr, 1.0, false);
      }
      break;
    }
  }
}

}  // namespace sccsd
