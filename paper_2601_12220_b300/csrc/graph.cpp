// Induced graph of a batched einsum (Appendix B): construction (B.1), the
// compliance conditions and the reconstruction Steps (B.2).
//
// Readings taken where the appendix is garbled or loose:
//  * N_dim uses AllDims (argument dimensionalities and |I_out|); the dim
//    rank tournament spans all dim nodes 1..N_dim.
//  * The edge set E_access,in-to-arg links access (i, j, d) to A^{i,j}.
//  * Step 2 orders V_arg-pos (the text says V_dim).  The second line of the
//    output-access condition concerns V_access,out (the text repeats
//    V_access,in).  ArgLabel(i, j) is the argument succeeding an input
//    access whose predecessors include output i and position j.
//    LengthLabel is taken per dimension d through InputIndex(d, j).
//  * The list has thirty conditions (C1..C30).  The two "consecutive
//    dimensions" conditions (C29, C30) are vacuous for an empty dimension
//    set, so scalar outputs are allowed; 0-dimensional operands have no
//    access nodes and are rejected by the parser.
#include <algorithm>
#include <map>
#include <set>

#include "canon.hpp"

namespace be {

namespace {

// successor and predecessor lists, sorted and without repeated edges; an
// edge test is a binary search in the source's successors
struct Adj {
  std::vector<std::vector<int>> succ, pred;
  int n;
  explicit Adj(const Graph &g) : succ(g.n), pred(g.n), n(g.n) {
    std::vector<int> dout(g.n, 0), din(g.n, 0);
    for (auto &e : g.edges) {
      ++dout[e.first];
      ++din[e.second];
    }
    for (int v = 0; v < g.n; ++v) {
      succ[v].reserve(dout[v]);
      pred[v].reserve(din[v]);
    }
    for (auto &e : g.edges) {
      succ[e.first].push_back(e.second);
      pred[e.second].push_back(e.first);
    }
    for (auto *lists : {&succ, &pred})
      for (auto &v : *lists) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
      }
  }
  bool edge(int a, int b) const { return std::binary_search(succ[a].begin(), succ[a].end(), b); }
};

int count_color(const std::vector<int> &v, const std::vector<int> &color, int c) {
  int k = 0;
  for (int x : v) k += color[x] == c;
  return k;
}

bool all_in(const std::vector<int> &v, const std::vector<int> &color, std::initializer_list<int> cs) {
  for (int x : v) {
    bool ok = false;
    for (int c : cs) ok |= color[x] == c;
    if (!ok) return false;
  }
  return true;
}

// the subgraph on nodes of colour c is a transitive tournament
bool tournament(const Graph &g, const Adj &A, int c) {
  std::vector<int> vs;
  for (int v = 0; v < g.n; ++v)
    if (g.color[v] == c) vs.push_back(v);
  std::vector<std::pair<int, int>> deg;
  for (int v : vs) deg.push_back({-count_color(A.succ[v], g.color, c), v});
  std::sort(deg.begin(), deg.end());
  for (size_t a = 0; a < deg.size(); ++a)
    for (size_t b = 0; b < deg.size(); ++b) {
      if (a == b) continue;
      if (A.edge(deg[a].second, deg[b].second) != (a < b)) return false;
    }
  return true;
}

int only(const std::vector<int> &v, const std::vector<int> &color, int c) {
  for (int x : v)
    if (color[x] == c) return x;
  return -1;
}

}  // namespace

Graph to_induced_graph(const Einsum &e) {
  Graph g;
  const int n_arg = (int)e.args.size();
  std::vector<int> letters;
  for (int c = 0; c < 26; ++c)
    if (e.used[c]) letters.push_back(c);
  const int n_index = (int)letters.size();
  int n_acc_in = 0;
  for (int j = 0; j < e.n; ++j) n_acc_in += (int)e.in[j].size();
  n_acc_in *= e.b;
  const int n_acc_out = (int)e.out.size();
  std::set<int> dtypes;
  for (auto &a : e.args) dtypes.insert(a.dtype);   // ordered by DtypeRank value
  std::set<int64_t> lengths;
  for (auto &a : e.args)
    for (auto L : a.shape) lengths.insert(L);
  int n_dim = (int)e.out.size();
  for (auto &a : e.args) n_dim = std::max(n_dim, (int)a.shape.size());

  int base = 0;
  const int o_arg = base; base += n_arg;
  const int o_index = base; base += n_index;
  const int o_accin = base; base += n_acc_in;
  const int o_accout = base; base += n_acc_out;
  const int o_output = base; base += e.b;
  const int o_argpos = base; base += e.n;
  const int o_dtype = base; base += (int)dtypes.size();
  const int o_length = base; base += (int)lengths.size();
  const int o_dim = base; base += n_dim;
  g.n = base;   // Eq. for N^IDG
  g.color.assign(g.n, 0);
  g.dtype_of.assign(g.n, 0);
  g.length_of.assign(g.n, -1);
  for (int v = 0; v < n_arg; ++v) g.color[o_arg + v] = C_ARG;
  for (int v = 0; v < n_index; ++v) g.color[o_index + v] = C_INDEX;
  for (int v = 0; v < n_acc_in; ++v) g.color[o_accin + v] = C_ACC_IN;
  for (int v = 0; v < n_acc_out; ++v) g.color[o_accout + v] = C_ACC_OUT;
  for (int v = 0; v < e.b; ++v) g.color[o_output + v] = C_OUTPUT;
  for (int v = 0; v < e.n; ++v) g.color[o_argpos + v] = C_ARGPOS;
  std::map<int, int> dt_node;
  {
    int k = 0;
    for (int dt : dtypes) {
      g.color[o_dtype + k] = C_DTYPE;
      g.dtype_of[o_dtype + k] = dt;
      dt_node[dt] = o_dtype + k;
      ++k;
    }
  }
  std::map<int64_t, int> len_node;
  {
    int k = 0;
    for (int64_t L : lengths) {
      g.color[o_length + k] = C_LENGTH;
      g.length_of[o_length + k] = L;
      len_node[L] = o_length + k;
      ++k;
    }
  }
  for (int v = 0; v < n_dim; ++v) g.color[o_dim + v] = C_DIM;

  g.arg_node.resize(n_arg);
  for (int a = 0; a < n_arg; ++a) g.arg_node[a] = o_arg + a;
  g.index_node.assign(26, -1);
  for (int k = 0; k < n_index; ++k) g.index_node[letters[k]] = o_index + k;
  g.row_node.resize(e.b);
  for (int i = 0; i < e.b; ++i) g.row_node[i] = o_output + i;
  g.pos_node.resize(e.n);
  for (int j = 0; j < e.n; ++j) g.pos_node[j] = o_argpos + j;
  g.acc_out_node.resize(n_acc_out);
  for (int d = 0; d < n_acc_out; ++d) g.acc_out_node[d] = o_accout + d;

  // every node has few edges; a generous reservation avoids regrowing the list
  g.edges.reserve((size_t)g.n * 6 + 64);
  auto E = [&](int a, int b) { g.edges.push_back({a, b}); };
  int acc = o_accin;
  g.acc_in_node.assign(e.b, std::vector<std::vector<int>>(e.n));
  for (int i = 0; i < e.b; ++i)
    for (int j = 0; j < e.n; ++j)
      for (size_t d = 0; d < e.in[j].size(); ++d) {
        int v = acc++;
        g.acc_in_node[i][j].push_back(v);
        E(v, g.arg_node[e.rows[i][j]]);            // E_access,in-to-arg
        E(g.pos_node[j], v);                       // E_arg-pos-to-access,in
        E(g.row_node[i], v);                       // E_output-to-access,in
        E(g.index_node[e.in[j][d]], v);            // E_index-to-access,in
        E(o_dim + (int)d, v);                      // E_dim-to-access,in
      }
  for (int d = 0; d < n_acc_out; ++d) {
    E(g.index_node[e.out[d]], g.acc_out_node[d]);  // E_index-to-access,out
    E(o_dim + d, g.acc_out_node[d]);               // E_dim-to-access,out
  }
  for (int k = 0; k < n_index; ++k) E(len_node[e.len[letters[k]]], o_index + k);   // E_length
  for (int a = 0; a < n_arg; ++a) E(dt_node[e.args[a].dtype], g.arg_node[a]);      // E_dtype
  for (auto &x : len_node)                                                          // E_length ranks
    for (auto &y : len_node)
      if (y.first > x.first) E(x.second, y.second);
  for (auto &x : dt_node)                                                           // E_dtype ranks
    for (auto &y : dt_node)
      if (y.first > x.first) E(x.second, y.second);
  for (int a = 0; a < n_dim; ++a)                                                   // E_dim ranks
    for (int b = a + 1; b < n_dim; ++b) E(o_dim + a, o_dim + b);
  return g;
}

int graph_check(const Graph &g) {
  const auto &col = g.color;
  for (int v = 0; v < g.n; ++v)
    if (col[v] < 1 || col[v] > 9) return 1;
  Adj A(g);
  for (int v = 0; v < g.n; ++v) {
    const auto &S = A.succ[v], &P = A.pred[v];
    switch (col[v]) {
      case C_ARG:
        if (!S.empty()) return 2;
        if (!all_in(P, col, {C_ACC_IN, C_DTYPE})) return 3;
        if (count_color(P, col, C_DTYPE) != 1) return 4;
        break;
      case C_DTYPE:
        if (!all_in(P, col, {C_DTYPE})) return 5;
        if (!all_in(S, col, {C_ARG, C_DTYPE})) return 6;
        break;
      case C_ACC_IN:
        if (!all_in(S, col, {C_ARG})) return 7;
        if (P.size() != 4 || count_color(P, col, C_ARGPOS) != 1 || count_color(P, col, C_INDEX) != 1 ||
            count_color(P, col, C_OUTPUT) != 1 || count_color(P, col, C_DIM) != 1)
          return 8;
        break;
      case C_OUTPUT:
        if (!all_in(S, col, {C_ACC_IN})) return 9;
        if (!P.empty()) return 10;
        break;
      case C_ACC_OUT:
        if (!S.empty()) return 11;
        if (P.size() != 2 || count_color(P, col, C_INDEX) != 1 || count_color(P, col, C_DIM) != 1) return 12;
        break;
      case C_INDEX:
        if (!all_in(S, col, {C_ACC_IN, C_ACC_OUT})) return 13;
        if (P.size() != 1 || count_color(P, col, C_LENGTH) != 1) return 14;
        break;
      case C_LENGTH:
        if (!all_in(P, col, {C_LENGTH})) return 15;
        if (!all_in(S, col, {C_INDEX, C_LENGTH})) return 16;
        break;
      case C_DIM:
        if (!all_in(P, col, {C_DIM})) return 17;
        if (!all_in(S, col, {C_ACC_IN, C_ACC_OUT, C_DIM})) return 18;
        break;
      case C_ARGPOS:
        if (!P.empty()) return 19;
        if (!all_in(S, col, {C_ACC_IN})) return 20;
        break;
    }
  }
  if (!tournament(g, A, C_DIM)) return 21;
  if (!tournament(g, A, C_LENGTH)) return 22;
  if (!tournament(g, A, C_DTYPE)) return 23;
  std::vector<int> accin, accout, outputs, argpos;
  for (int v = 0; v < g.n; ++v) {
    if (col[v] == C_ACC_IN) accin.push_back(v);
    if (col[v] == C_ACC_OUT) accout.push_back(v);
    if (col[v] == C_OUTPUT) outputs.push_back(v);
    if (col[v] == C_ARGPOS) argpos.push_back(v);
  }
  // C24: same argument and same dimension -> indices of equal length
  {
    std::map<std::pair<int, int>, std::vector<int>> seen;
    for (int v : accin) {
      int arg = only(A.succ[v], col, C_ARG), dim = only(A.pred[v], col, C_DIM);
      int idx = only(A.pred[v], col, C_INDEX);
      auto &lp = seen[{arg, dim}];
      if (lp.empty()) lp = A.pred[idx];
      else if (lp != A.pred[idx]) return 24;
    }
  }
  // C25: an output index also indexes some input
  for (int v : accout) {
    int idx = only(A.pred[v], col, C_INDEX);
    if (count_color(A.succ[idx], col, C_ACC_IN) == 0) return 25;
  }
  // C26: the same (index, dim, position) access exists exactly once per output
  {
    std::map<std::tuple<int, int, int, int>, int> cnt;
    for (int v : accin) {
      int i = only(A.pred[v], col, C_INDEX), d = only(A.pred[v], col, C_DIM);
      int k = only(A.pred[v], col, C_ARGPOS), o = only(A.pred[v], col, C_OUTPUT);
      cnt[{i, d, k, o}]++;
    }
    for (int v : accin) {
      int i = only(A.pred[v], col, C_INDEX), d = only(A.pred[v], col, C_DIM);
      int k = only(A.pred[v], col, C_ARGPOS);
      for (int o : outputs) {
        auto it = cnt.find({i, d, k, o});
        if (it == cnt.end() || it->second != 1) return 26;
      }
    }
  }
  // C27: distinct output indices
  {
    std::set<int> s;
    for (int v : accout) s.insert(only(A.pred[v], col, C_INDEX));
    if (s.size() != accout.size()) return 27;
  }
  // C28, C29 per (position, output)
  std::map<std::pair<int, int>, std::vector<int>> acc_ko;
  for (int v : accin)
    acc_ko[{only(A.pred[v], col, C_ARGPOS), only(A.pred[v], col, C_OUTPUT)}].push_back(v);
  auto consecutive = [&](const std::set<int> &dims) {
    if (dims.empty()) return true;
    int roots = 0, inner = 0;
    for (int d : dims) {
      bool has_dim_pred = count_color(A.pred[d], col, C_DIM) > 0;
      roots += !has_dim_pred;
      bool pred_in = false;
      for (int p : A.pred[d]) pred_in |= dims.count(p) > 0;
      inner += pred_in;
    }
    return roots == 1 && inner == (int)dims.size() - 1;
  };
  for (int k : argpos)
    for (int o : outputs) {
      auto it = acc_ko.find({k, o});
      if (it == acc_ko.end()) return 28;
      std::set<int> args, dims;
      for (int a : it->second) {
        for (int s : A.succ[a]) args.insert(s);
        dims.insert(only(A.pred[a], col, C_DIM));
      }
      if (args.size() != 1) return 28;
      if (!consecutive(dims)) return 29;
    }
  {
    std::set<int> dims;
    for (int v : accout) dims.insert(only(A.pred[v], col, C_DIM));
    if (!consecutive(dims)) return 30;
  }
  return 0;
}

int to_batched_einsum(const Graph &g, Einsum &out, std::vector<int> &index_order,
                      std::vector<int> &arg_order, std::string &err) {
  const auto &col = g.color;
  Adj A(g);
  std::vector<int> V[10];
  for (int v = 0; v < g.n; ++v) V[col[v]].push_back(v);   // node order = inferred orderings
  if (V[C_INDEX].size() > 26) { err = "more than 26 indices"; return ETOOMANY; }
  std::vector<int> ord(g.n, -1);
  for (int c = 1; c <= 9; ++c)
    for (size_t k = 0; k < V[c].size(); ++k) ord[V[c][k]] = (int)k;   // Steps 2-5
  auto dimrank = [&](int d) { return 1 + count_color(A.pred[d], col, C_DIM); };   // Step 6
  index_order.assign(g.n, -1);
  arg_order.assign(g.n, -1);
  for (int v : V[C_INDEX]) index_order[v] = ord[v];
  for (int v : V[C_ARG]) arg_order[v] = ord[v];

  out = Einsum();
  out.b = (int)V[C_OUTPUT].size();
  out.n = (int)V[C_ARGPOS].size();
  // Step 7: output index list
  out.out.assign(V[C_ACC_OUT].size(), -1);
  for (int v : V[C_ACC_OUT]) {
    int d = only(A.pred[v], col, C_DIM), i = only(A.pred[v], col, C_INDEX);
    int k = dimrank(d);
    if (k < 1 || k > (int)out.out.size()) { err = "output dimension out of range"; return EINVALID; }
    out.out[k - 1] = (int8_t)ord[i];
  }
  // Steps 8-9: argument dimensions and input index lists
  out.in.assign(out.n, {});
  std::vector<std::vector<int>> in_idx_node(out.n);
  for (int jn : V[C_ARGPOS]) {
    int j = ord[jn];
    std::map<int, int> by_dim;   // dim rank -> index node
    for (int a : A.succ[jn]) {
      if (col[a] != C_ACC_IN) continue;
      int d = dimrank(only(A.pred[a], col, C_DIM));
      int i = only(A.pred[a], col, C_INDEX);
      auto it = by_dim.find(d);
      if (it != by_dim.end() && it->second != i) { err = "input indexing differs between outputs"; return EINVALID; }
      by_dim[d] = i;
    }
    int argdim = (int)by_dim.size();
    for (int d = 1; d <= argdim; ++d) {
      auto it = by_dim.find(d);
      if (it == by_dim.end()) { err = "argument dimensions are not consecutive"; return EINVALID; }
      out.in[j].push_back((int8_t)ord[it->second]);
      in_idx_node[j].push_back(it->second);
    }
  }
  // Step 10: arguments, dtypes and shapes
  out.args.resize(V[C_ARG].size());
  std::vector<bool> seen(V[C_ARG].size(), false);
  out.rows.assign(out.b, std::vector<int>(out.n, -1));
  for (int on : V[C_OUTPUT]) {
    int i = ord[on];
    for (int a : A.succ[on]) {
      if (col[a] != C_ACC_IN) continue;
      int j = ord[only(A.pred[a], col, C_ARGPOS)];
      int argn = only(A.succ[a], col, C_ARG);
      int k = ord[argn];
      if (out.rows[i][j] >= 0 && out.rows[i][j] != k) { err = "two arguments at one position"; return EINVALID; }
      out.rows[i][j] = k;
      if (!seen[k]) {
        seen[k] = true;
        Arg &arg = out.args[k];
        arg.name = "A" + std::to_string(k);
        arg.buffer = k;
        arg.dtype = g.dtype_of[only(A.pred[argn], col, C_DTYPE)];
        for (int idx : in_idx_node[j]) arg.shape.push_back(g.length_of[only(A.pred[idx], col, C_LENGTH)]);
      }
    }
  }
  for (auto &r : out.rows)
    for (int k : r)
      if (k < 0) { err = "missing argument"; return EINVALID; }
  for (auto &a : out.args) {
    Buffer bf;
    bf.name = a.name;
    bf.dtype = a.dtype;
    bf.shape = a.shape;
    out.buffers.push_back(bf);
  }
  int best = -1;
  for (auto &a : out.args)
    if (dtype_promote_rank(a.dtype) > best) { best = dtype_promote_rank(a.dtype); out.out_dtype = a.dtype; }
  return check_sound(out, err);
}

}  // namespace be
