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
  const auto d = t[X].dims;
  const size_t r = d.size();
  if ((r != 4 && r != 5) || d[r - 4] != o || d[r - 3] != o || d[r - 2] != v || d[r - 1] != v)
    throw std::runtime_error("ladder operand must be [(nb)][o][o][v][v]");
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

std::map<int, int> Graph::tangent(const std::map<int, int>& seeds, const Ranges& ranges,
                                  int64_t nb) {
  const std::string Zs = nb > 0 ? "Z" : "";
  auto bdims = [&](const std::vector<int64_t>& d) {
    std::vector<int64_t> r;
    if (nb > 0) r.push_back(nb);
    r.insert(r.end(), d.begin(), d.end());
    return r;
  };
  auto boff = [&](const std::vector<int64_t>& d) {
    std::vector<int64_t> r;
    if (nb > 0) r.push_back(0);
    r.insert(r.end(), d.begin(), d.end());
    return r;
  };
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
        int c1 = dA >= 0 ? contract(dA, Zs + op.la, B, op.lb, Zs + op.lc, op.alpha, op.tc) : -1;
        int c2 = dB >= 0 ? contract(A, op.la, dB, Zs + op.lb, Zs + op.lc, op.alpha, op.tc) : -1;
        if (c1 >= 0 && is_zero(c1)) c1 = -1;
        if (c2 >= 0 && is_zero(c2)) c2 = -1;
        if (c1 >= 0 && c2 >= 0)
          d = add(Zs + op.lc, {{c1, Zs + op.lc, 1.0}, {c2, Zs + op.lc, 1.0}});
        else
          d = c1 >= 0 ? c1 : c2;
        break;
      }
      case OpKind::Add: {
        std::vector<Term> terms;
        for (size_t k = 0; k < op.in.size(); ++k) {
          int dk = T(op.in[k]);
          if (dk >= 0) terms.push_back({dk, Zs + op.perm[k], op.coef[k]});
        }
        if (!terms.empty()) d = add(Zs + op.lc, terms);
        break;
      }
      case OpKind::Slice: {
        int dx = T(op.in[0]);
        if (dx >= 0) d = slice(dx, boff(op.off), bdims(t[op.out].dims));
        break;
      }
      case OpKind::Embed: {
        int dx = T(op.in[0]);
        if (dx >= 0) d = embed(dx, boff(op.off), bdims(t[op.out].dims));
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
                                  const Ranges& ranges, int64_t nb) {
  const std::string Zs = nb > 0 ? "Z" : "";
  auto bdims = [&](const std::vector<int64_t>& d) {
    std::vector<int64_t> r;
    if (nb > 0) r.push_back(nb);
    r.insert(r.end(), d.begin(), d.end());
    return r;
  };
  auto boff = [&](const std::vector<int64_t>& d) {
    std::vector<int64_t> r;
    if (nb > 0) r.push_back(0);
    r.insert(r.end(), d.begin(), d.end());
    return r;
  };
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
    for (size_t k = 0; k < t[v[0]].dims.size(); ++k) l.push_back(char('A' + k));
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
        if (dep[A]) push(A, contract(g, Zs + op.lc, B, op.lb, Zs + op.la, op.alpha, op.tc));
        if (dep[B]) push(B, contract(A, op.la, g, Zs + op.lc, Zs + op.lb, op.alpha, op.tc));
        break;
      }
      case OpKind::Add:
        for (size_t k = 0; k < op.in.size(); ++k)
          if (dep[op.in[k]])
            push(op.in[k], add(Zs + op.perm[k], {{g, Zs + op.lc, op.coef[k]}}));
        break;
      case OpKind::Slice:
        if (dep[op.in[0]]) push(op.in[0], embed(g, boff(op.off), bdims(t[op.in[0]].dims)));
        break;
      case OpKind::Embed:
        if (dep[op.in[0]]) push(op.in[0], slice(g, boff(op.off), bdims(t[op.in[0]].dims)));
        break;
      case OpKind::Ladder: {
        int X = op.in[0], L = op.in[1];
        if (dep[X]) push(X, ladder(g, L));
        if (dep[L]) {
          if (nb > 0) throw std::runtime_error("batched adjoint w.r.t. L not supported");
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
    res[w] = s >= 0 ? s : zero(bdims(t[w].dims));
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

void Graph::set_volatile_inputs(const std::vector<int>& inputs) {
  vol_.assign(t.size(), 0);
  for (int x : inputs) vol_[x] = 1;
  for (auto& op : ops)
    for (int x : op.in)
      if (vol_[x]) vol_[op.out] = 1;
}

void Graph::run(const std::vector<int>& targets) {
  if (vol_.size() < t.size()) vol_.resize(t.size(), 0);
  // buffers of volatile results handed to the caller by the previous run
  for (int x : held_) {
    if (t[x].data && t[x].kind == Kind::Node) {
      be->pool_put(t[x].data, std::max<int64_t>(1, t[x].numel()));
      t[x].data = nullptr;
    }
  }
  held_.clear();
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
  // last use of each volatile node among the ops of this run
  std::vector<char> is_target(t.size(), 0);
  for (int x : targets) is_target[x] = 1;
  std::vector<size_t> last_use(t.size(), 0);
  for (size_t i = 0; i < ops.size(); ++i)
    if (need_op[i])
      for (int x : ops[i].in) last_use[x] = i;
  // Planning of the per-call permuted sums. A term produced by a contraction
  // whose result feeds nothing else is evaluated inside the sum, straight into
  // its output (the intermediate is never stored, the sum never re-reads it);
  // a term produced by another such single-use sum is replaced by that sum's
  // own terms (permutations composed, coefficients multiplied), recursively.
  std::vector<int> uses(t.size(), 0);
  for (size_t i = 0; i < ops.size(); ++i)
    if (need_op[i])
      for (int x : ops[i].in) uses[x]++;
  std::vector<char> fused_op(ops.size(), 0);
  std::map<size_t, std::vector<SumTerm>> add_plan;
  auto single_use = [&](int x) {
    const int p = prod[x];
    return p >= 0 && need_op[p] && vol_[x] && !is_target[x] && uses[x] == 1 &&
           t[x].kind == Kind::Node;
  };
  for (size_t i = 0; i < ops.size(); ++i) {
    const Op& a = ops[i];
    if (!need_op[i] || a.kind != OpKind::Add || !vol_[a.out] || t[a.out].dims.empty()) continue;
    std::vector<SumTerm> plan;
    bool changed = false;
    std::vector<SumTerm> stack;
    for (size_t k = a.in.size(); k-- > 0;) stack.push_back({a.in[k], a.perm[k], a.coef[k], -1});
    while (!stack.empty()) {
      SumTerm tm = stack.back();
      stack.pop_back();
      const int x = tm.node;
      if (single_use(x)) {
        const int p = prod[x];
        const Op& q = ops[p];
        if (q.kind == OpKind::Contract) {
          tm.fused = p;
          fused_op[p] = 1;
          for (int y : q.in) last_use[y] = std::max(last_use[y], i);
          plan.push_back(tm);
          changed = true;
          continue;
        }
        if (q.kind == OpKind::Add && !t[x].dims.empty()) {
          // x's dim j has label q.lc[j] in q and label tm.perm[j] here
          fused_op[p] = 1;
          changed = true;
          for (size_t r = q.in.size(); r-- > 0;) {
            std::string pr;
            for (char c : q.perm[r]) pr.push_back(tm.perm[q.lc.find(c)]);
            stack.push_back({q.in[r], pr, tm.coef * q.coef[r], -1});
          }
          continue;
        }
      }
      last_use[x] = std::max(last_use[x], i);
      plan.push_back(tm);
    }
    if (changed) add_plan[i] = plan;
  }
  std::vector<std::vector<int>> free_after(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) {
    if (!need_op[i]) continue;
    int x = ops[i].out;
    if (vol_[x] && !is_target[x]) free_after[std::max(last_use[x], i)].push_back(x);
  }
  for (size_t i = 0; i < ops.size(); ++i) {
    if (!need_op[i] || fused_op[i]) continue;
    Op& op = ops[i];
    bool need = !op.ran || vol_[op.out];
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
    if (vol_[op.out] && !t[op.out].data)
      t[op.out].data = be->pool_get(std::max<int64_t>(1, t[op.out].numel()));
    auto fz = add_plan.find(i);
    if (fz != add_plan.end())
      exec_add(op, fz->second);
    else
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
    for (int x : free_after[i]) {
      if (t[x].data) {
        be->pool_put(t[x].data, std::max<int64_t>(1, t[x].numel()));
        t[x].data = nullptr;
      }
    }
  }
  for (int x : targets)
    if (x < (int)vol_.size() && vol_[x] && t[x].kind == Kind::Node) held_.push_back(x);
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
    if (op.kind == OpKind::Contract && op.trace_conv) {
      // converted operands and their producers (c contract, a add, ... i input)
      std::string conv = "           converted:";
      for (int q = 0; q < 2; ++q) {
        if (!(op.trace_conv & (1 << q))) continue;
        char kc = 'i';
        for (size_t p = 0; p < ops.size(); ++p)
          if (ops[p].out == op.in[q]) {
            kc = "caselL"[(int)ops[p].kind];
            break;
          }
        const Tensor& x = t[op.in[q]];
        conv += std::string(" ") + (q ? "B" : "A") + "(" + kc + ", " +
                std::to_string(x.numel() * 8 / 1000000) + " MB)";
      }
      out += conv + "\n";
    }
    if (op.kind == OpKind::Add) {
      // the producer of every term: c contract, a add, s slice, e embed, l ladder, i input
      std::string terms = "           terms:";
      for (size_t q = 0; q < op.in.size(); ++q) {
        char kc = 'i';
        for (size_t p = 0; p < ops.size(); ++p)
          if (ops[p].out == op.in[q]) {
            kc = "caselL"[(int)ops[p].kind];
            break;
          }
        terms += std::string(" ") + kc + ":" + op.perm[q];
      }
      out += terms + "\n";
    }
  }
  return out;
}

void Graph::exec(Op& op) {
  Tensor& out = t[op.out];
  if (!out.data) out.data = be->alloc(std::max<int64_t>(1, out.numel()));
  const int rc = (int)out.dims.size();
  switch (op.kind) {
    case OpKind::Add:
      exec_add(op, {});
      break;
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
      be->ladder(*this, t[op.in[1]].data, t[op.in[1]].version, t[op.in[0]].data, out.data,
                 t[op.in[0]].numel() / ((int64_t)v * v));
      break;
    case OpKind::LadderAdjL:
      be->ladder_adj_l(*this, t[op.in[2]].data, t[op.in[0]].data, t[op.in[1]].data, out.data);
      break;
    case OpKind::Contract: {
      auto os = row_strides(out.dims);
      exec_contract(op, out.data, os.data(), 1.0, false);
      break;
    }
  }
}

// Permuted sum. fused[k] >= 0: term k is the output of contraction op
// fused[k], which is evaluated here straight into the sum (scaled, and
// accumulated after the first term) instead of through its own buffer.
void Graph::exec_add(Op& op, const std::vector<SumTerm>& terms_in) {
  Tensor& out = t[op.out];
  const int rc = (int)out.dims.size();
  auto ostr = row_strides(out.dims);
  std::vector<SumTerm> own;
  if (terms_in.empty())
    for (size_t k = 0; k < op.in.size(); ++k) own.push_back({op.in[k], op.perm[k], op.coef[k], -1});
  const std::vector<SumTerm>& terms = terms_in.empty() ? own : terms_in;
  for (size_t k = 0; k < terms.size(); ++k) {
    const SumTerm& tm = terms[k];
    const Tensor& x = t[tm.node];
    if (tm.fused >= 0) {
      int64_t cs[kMaxRank];
      for (size_t q = 0; q < x.dims.size(); ++q) cs[q] = ostr[op.lc.find(tm.perm[q])];
      void* e0 = trace ? be->record_event() : nullptr;
      exec_contract(ops[tm.fused], out.data, cs, tm.coef, k > 0);
      if (trace) {
        // the sum's own time includes this; the contraction is listed too
        ops[tm.fused].trace_ms += be->elapsed_ms(e0, be->record_event());
        ops[tm.fused].trace_calls += 1;
      }
      continue;
    }
    auto xs = row_strides(x.dims);
    int64_t istr[kMaxRank];
    for (int q = 0; q < rc; ++q) istr[q] = xs[tm.perm.find(op.lc[q])];
    be->copy_view(rc, out.dims.data(), out.data, ostr.data(), x.data, istr, tm.coef, k > 0);
  }
  if (rc == 0 && terms.empty()) be->fill(out.data, 1, 0.0);
}

// Contraction into out_data, whose dims are those of op's output and whose
// strides are ostr (per output label): out (= or +=) coef * result.
void Graph::exec_contract(Op& op, double* out_data, const int64_t* ostr, double coef, bool acc) {
  Tensor& out = t[op.out];
  const int rc = (int)out.dims.size();
  const std::vector<int64_t> ostrides(ostr, ostr + rc);
  const bool plain = !acc && coef == 1.0 && ostrides == row_strides(out.dims);
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
  auto dim_of = [&](char c) -> int64_t {
    size_t p = la.find(c);
    if (p != std::string::npos) return A.dims[p];
    return B.dims[lb.find(c)];
  };
  // nothing contracted (scalings, outer and elementwise products): one
  // elementwise pass over the output, no GEMM
  {
    bool all_out = true;
    for (char c : la + lb)
      if (lc.find(c) == std::string::npos) all_out = false;
    if (all_out) {
      auto as_ = row_strides(A.dims), bs_ = row_strides(B.dims);
      int64_t astr[kMaxRank], bstr[kMaxRank];
      for (int q = 0; q < rc; ++q) {
        size_t pa = la.find(lc[q]), pb = lb.find(lc[q]);
        astr[q] = pa == std::string::npos ? 0 : as_[pa];
        bstr[q] = pb == std::string::npos ? 0 : bs_[pb];
      }
      be->mul_view(rc, out.dims.data(), out_data, ostrides.data(), A.data, astr, B.data, bstr,
                   op.alpha * coef, acc);
      return;
    }
  }
  // a label group of X collapsed to at most two strided levels
  struct Grp {
    bool ok = true;
    int64_t n2 = 0, s1 = 0, s2 = 0;
  };
  // maximal runs (extent, innermost stride) of a label group, outermost first
  auto runs_of = [&](const std::vector<int64_t>& dims, const std::vector<int64_t>& xs,
                     const std::string& lx, const std::string& grp) {
    std::vector<std::pair<int64_t, int64_t>> runs;
    for (char c : grp) {
      size_t p = lx.find(c);
      int64_t d = dims[p], st = xs[p];
      if (d == 1) continue;
      if (!runs.empty() && runs.back().second == st * d) {
        runs.back().first *= d;
        runs.back().second = st;
      } else {
        runs.push_back({d, st});
      }
    }
    return runs;
  };
  auto collapse_s = [&](const std::vector<int64_t>& dims, const std::vector<int64_t>& xs,
                        const std::string& lx, const std::string& grp) {
    auto runs = runs_of(dims, xs, lx, grp);
    Grp g;
    if (runs.size() == 1) {
      g.s2 = runs[0].second;
    } else if (runs.size() == 2) {
      g.n2 = runs[1].first;
      g.s1 = runs[0].second;
      g.s2 = runs[1].second;
    } else if (runs.size() > 2) {
      g.ok = false;
    }
    return g;
  };
  auto collapse = [&](const Tensor& X, const std::string& lx, const std::string& grp) {
    return collapse_s(X.dims, row_strides(X.dims), lx, grp);
  };
  auto view_of = [&](const Tensor& X, const std::string& lx, const std::string& rows,
                     const std::string& kls, MatView& v) {
    Grp gb = collapse(X, lx, bat), gr = collapse(X, lx, rows), gk = collapse(X, lx, kls);
    if (!gb.ok || gb.n2 || !gr.ok || !gk.ok) return false;
    v.p = X.data;
    v.sb = gb.s2;
    v.n2r = gr.n2;
    v.sr1 = gr.s1;
    v.sr2 = gr.s2;
    v.n2k = gk.n2;
    v.sk1 = gk.s1;
    v.sk2 = gk.s2;
    // a K group of extent 1 has no stride of its own
    if (!gk.n2 && gk.s2 == 0) v.sk2 = 1;
    return true;
  };
  // contracted-label order: the one for which both operands are views
  MatView Av, Bv;
  std::string kl = ka;
  bool okA = view_of(A, la, ml, kl, Av), okB = view_of(B, lb, nl, kl, Bv);
  if (!(okA && okB)) {
    MatView A2, B2;
    bool a2 = view_of(A, la, ml, kb, A2), b2 = view_of(B, lb, nl, kb, B2);
    if ((int)a2 + (int)b2 > (int)okA + (int)okB) {
      kl = kb;
      okA = a2;
      okB = b2;
      Av = A2;
      Bv = B2;
    }
  }
  int64_t nb = 1, M = 1, N = 1, K = 1;
  for (char c : bat) nb *= dim_of(c);
  for (char c : ml) M *= dim_of(c);
  for (char c : nl) N *= dim_of(c);
  for (char c : kl) K *= dim_of(c);
  // dense [batch][rows][K] copy for operands that are not a two-level view
  auto arrange = [&](const Tensor& X, const std::string& lx, const std::string& want,
                     int slot, int64_t rows) -> MatView {
    if (lx == want) return MatView::dense(X.data, rows, K);
    double* dst = be->scratch(slot, std::max<int64_t>(1, X.numel()));
    std::vector<int64_t> wd;
    for (char c : want) wd.push_back(X.dims[lx.find(c)]);
    auto ws = row_strides(wd);
    auto xs = row_strides(X.dims);
    int64_t istr[kMaxRank];
    for (size_t q = 0; q < want.size(); ++q) istr[q] = xs[lx.find(want[q])];
    be->copy_view((int)want.size(), wd.data(), dst, ws.data(), X.data, istr, 1.0, false);
    return MatView::dense(dst, rows, K);
  };
  auto finish = [&](double* Cp) {
    std::string cl = bat + ml + nl;
    std::vector<int64_t> cd;
    for (char c : cl) cd.push_back(dim_of(c));
    auto cs = row_strides(cd);
    int64_t istr[kMaxRank];
    for (int q = 0; q < rc; ++q) istr[q] = cs[cl.find(lc[q])];
    be->copy_view(rc, out.dims.data(), out_data, ostrides.data(), Cp, istr, coef, acc);
  };
  // tensor-core route: converted operands are kept in the backend, keyed by
  // (node, layout, version)
  const bool use_tc = op.tc && be->tc_will_use(nb, M, N, K);
  if (use_tc) {
    auto hash = [](const std::string& a, const std::string& b) {
      uint64_t h = 1469598103934665603ull;
      for (char c : a + "|" + b) h = (h ^ (uint64_t)(unsigned char)c) * 1099511628211ull;
      return h;
    };
    Backend::OperandKey kA{this, op.in[0], A.version, hash(la, bat + ml + kl)};
    Backend::OperandKey kB{this, op.in[1], B.version, hash(lb, bat + nl + kl)};
    // every operand is keyed: a per-call tensor changes version on every run,
    // so its converted form is reused only by the other contractions of the
    // same run that read it in the same layout
    const bool cA = true, cB = true;
    if (trace) op.trace_conv = (be->tc_cached(kA) ? 0 : 1) | (be->tc_cached(kB) ? 0 : 2);
    if (cA && be->tc_cached(kA))
      Av.p = nullptr;
    else if (!okA)
      Av = arrange(A, la, bat + ml + kl, 0, M);
    if (cB && be->tc_cached(kB))
      Bv.p = nullptr;
    else if (!okB)
      Bv = arrange(B, lb, bat + nl + kl, 1, N);
    const Backend::OperandKey* pA = cA ? &kA : nullptr;
    const Backend::OperandKey* pB = cB ? &kB : nullptr;
    if (plain && lc == bat + ml + nl) {
      be->gemm_tc_keyed(M, N, K, op.alpha, Av, pA, Bv, pB, out_data);
    } else if (plain && lc == bat + nl + ml) {
      be->gemm_tc_keyed(N, M, K, op.alpha, Bv, pB, Av, pA, out_data);
    } else {
      // a permuted (or accumulated) output is written by the GEMM epilogue
      // through a multi-level view of the M and N label groups
      auto rm = runs_of(out.dims, ostrides, lc, ml), rn = runs_of(out.dims, ostrides, lc, nl);
      if ((int)rm.size() <= kOutLevels && (int)rn.size() <= kOutLevels) {
        OutView ov;
        ov.nr = std::max<int>(1, (int)rm.size());
        ov.nc = std::max<int>(1, (int)rn.size());
        for (size_t l = 0; l < rm.size(); ++l) {
          ov.re[l] = rm[l].first;
          ov.rs[l] = rm[l].second;
        }
        for (size_t l = 0; l < rn.size(); ++l) {
          ov.ce[l] = rn[l].first;
          ov.cs[l] = rn[l].second;
        }
        be->gemm_tc_keyed(M, N, K, op.alpha * coef, Av, pA, Bv, pB, out_data, &ov, acc);
      } else {
        double* Cp = be->scratch(2, std::max<int64_t>(1, nb * M * N));
        be->gemm_tc_keyed(M, N, K, op.alpha, Av, pA, Bv, pB, Cp);
        finish(Cp);
      }
    }
    return;
  }
  if (!okA) Av = arrange(A, la, bat + ml + kl, 0, M);
  if (!okB) Bv = arrange(B, lb, bat + nl + kl, 1, N);
  if (plain && lc == bat + ml + nl) {
    be->gemm_view(nb, M, N, K, op.alpha, Av, Bv, out_data, false);
  } else if (plain && lc == bat + nl + ml) {
    be->gemm_view(nb, N, M, K, op.alpha, Bv, Av, out_data, false);
  } else {
    double* Cp = be->scratch(2, std::max<int64_t>(1, nb * M * N));
    be->gemm_view(nb, M, N, K, op.alpha, Av, Bv, Cp, false);
    finish(Cp);
  }
}

}  // namespace sccsd
