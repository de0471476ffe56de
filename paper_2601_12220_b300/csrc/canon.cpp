// Alg. 1 (CanonicalizeBatchedEinsum) with an exact lexicographic canonical
// labeling.
//
// The paper leaves GetCanonLabel to an external graph canonizer and notes
// that the normal form then depends on which one is used.  Here the label
// is fixed by C_lex: among all operand orders sigma^j and row orders
// sigma^i, take the one whose token vector
//
//   T = [b, n, |I_out|, ids(I_out), |I_in,1|, ids(I_in,1), ..., lengths by
//        index id, argument ids row by row, DtypeRank by argument id]
//
// is lexicographically smallest, with index ids and argument ids given by
// first appearance (which minimizes each part for a fixed order).  The
// search is a depth-first walk that only ever extends a prefix by the
// smallest next segment (any other segment loses regardless of what
// follows), branching on ties; two tied rows whose fresh arguments occur
// nowhere else and agree in dtype are interchangeable, so only one of them
// is explored.  The labeling is then applied to the induced graph
// (Appendix B.1), the relabeled graph is turned back into a batched einsum
// (Appendix B.2) and sigma^A, sigma^I are read off as in Alg. 1.
#include <algorithm>
#include <cstdio>
#include <map>

#include "canon.hpp"

namespace be {

namespace {

typedef std::vector<int64_t> Tok;

// compare ``prefix`` with the same-length prefix of ``best``: -1, 0 or 1
int prefix_cmp(const Tok &prefix, const Tok &best) {
  for (size_t k = 0; k < prefix.size(); ++k) {
    if (prefix[k] < best[k]) return -1;
    if (prefix[k] > best[k]) return 1;
  }
  return 0;
}

struct IndexCand {
  std::vector<int> perm;   // canonical position p -> user position
  int id_of[26];           // user letter -> canonical index id
  int n_ids;
};

struct OpSearch {
  const Einsum &e;
  Tok best;
  bool have = false;
  std::vector<IndexCand> cands;
  explicit OpSearch(const Einsum &e_) : e(e_) {}

  void dfs(std::vector<int> &perm, std::vector<char> &used, int *id_of, int next_id, Tok &prefix) {
    if ((int)perm.size() == e.n) {
      if (!have || prefix < best) {
        best = prefix;
        have = true;
        cands.clear();
      }
      if (prefix == best) {
        IndexCand c;
        c.perm = perm;
        std::copy(id_of, id_of + 26, c.id_of);
        c.n_ids = next_id;
        cands.push_back(c);
      }
      return;
    }
    // segment of every unused operand
    std::vector<Tok> segs(e.n);
    Tok minseg;
    bool first = true;
    for (int j = 0; j < e.n; ++j) {
      if (used[j]) continue;
      int tmp[26];
      std::copy(id_of, id_of + 26, tmp);
      int nid = next_id;
      Tok s{(int64_t)e.in[j].size()};
      for (int8_t c : e.in[j]) {
        if (tmp[c] < 0) tmp[c] = nid++;
        s.push_back(tmp[c]);
      }
      segs[j] = s;
      if (first || s < minseg) { minseg = s; first = false; }
    }
    if (have && prefix_cmp(prefix, best) == 0) {
      // prune: the prefix extended by the smallest segment must not exceed the best
      size_t L = prefix.size();
      for (size_t k = 0; k < minseg.size(); ++k) {
        int64_t want = best[L + k];
        if (minseg[k] < want) break;
        if (minseg[k] > want) return;
      }
    }
    for (int j = 0; j < e.n; ++j) {
      if (used[j] || segs[j] != minseg) continue;
      int tmp[26];
      std::copy(id_of, id_of + 26, tmp);
      int nid = next_id;
      for (int8_t c : e.in[j])
        if (tmp[c] < 0) tmp[c] = nid++;
      used[j] = 1;
      perm.push_back(j);
      size_t L = prefix.size();
      prefix.insert(prefix.end(), minseg.begin(), minseg.end());
      dfs(perm, used, tmp, nid, prefix);
      prefix.resize(L);
      perm.pop_back();
      used[j] = 0;
    }
  }
};

struct RowSearch {
  const Einsum &e;
  const std::vector<int> &perm;          // canonical position -> user position
  std::vector<std::vector<int>> seq;     // user row -> args in canonical position order
  std::vector<int> owner;                // arg -> the only row holding it, or -1 if several
  Tok best_table, best_dt;
  bool have = false;
  std::vector<int> best_rows, best_argid;
  long leaves = 0;
  std::vector<int64_t> segs;             // [depth][row][position] segment scratch
  std::vector<int> fresh_args;           // a segment's arguments in order of first appearance
  RowSearch(const Einsum &e_, const std::vector<int> &perm_, const Tok *prev_table, const Tok *prev_dt)
      : e(e_), perm(perm_) {
    segs.assign((size_t)e.b * e.b * e.n, 0);
    fresh_args.assign((size_t)e.n, 0);
    seq.resize(e.b);
    owner.assign(e.args.size(), -2);
    for (int i = 0; i < e.b; ++i)
      for (int p = 0; p < e.n; ++p) {
        int a = e.rows[i][perm[p]];
        seq[i].push_back(a);
        if (owner[a] == -2) owner[a] = i;
        else if (owner[a] != i) owner[a] = -1;
      }
    if (prev_table) {
      best_table = *prev_table;
      best_dt = *prev_dt;
      have = true;
    }
  }
  bool improved = false;

  void dfs(std::vector<int> &rows, std::vector<char> &used, std::vector<int> &argid, int next_id, Tok &prefix) {
    if ((int)rows.size() == e.b) {
      ++leaves;
      Tok dt;
      std::vector<int> by_id(next_id);
      for (size_t a = 0; a < argid.size(); ++a)
        if (argid[a] >= 0) by_id[argid[a]] = (int)a;
      for (int k = 0; k < next_id; ++k) dt.push_back(e.args[by_id[k]].dtype);
      bool better = !have || prefix < best_table || (prefix == best_table && dt < best_dt);
      if (better) {
        best_table = prefix;
        best_dt = dt;
        best_rows = rows;
        best_argid = argid;
        have = true;
        improved = true;
      }
      return;
    }
    // the segment of every unused row (n ids each) in this depth's scratch
    // row of segs (allocated once per search), and the smallest of them
    const int n = e.n;
    const size_t depth = rows.size();
    int64_t *seg = segs.data() + depth * (size_t)e.b * n;
    int *fresh = fresh_args.data();
    int minrow = -1;
    for (int i = 0; i < e.b; ++i) {
      if (used[i]) continue;
      int64_t *s = seg + (size_t)i * n;
      int nid = next_id, nf = 0;
      for (int p = 0; p < n; ++p) {
        const int a = seq[i][p];
        int id = argid[a];
        if (id < 0) {
          for (int f = 0; f < nf; ++f)
            if (fresh[f] == a) id = next_id + f;
          if (id < 0) {
            id = nid++;
            fresh[nf++] = a;
          }
        }
        s[p] = id;
      }
      if (minrow < 0 || std::lexicographical_compare(s, s + n, seg + (size_t)minrow * n, seg + (size_t)minrow * n + n))
        minrow = i;
    }
    const int64_t *minseg = seg + (size_t)minrow * n;
    if (have && prefix_cmp(prefix, best_table) == 0) {
      size_t L = prefix.size();
      for (int k = 0; k < n; ++k) {
        int64_t want = best_table[L + k];
        if (minseg[k] < want) break;
        if (minseg[k] > want) return;
      }
    }
    std::vector<int> chosen;
    for (int i = 0; i < e.b; ++i) {
      if (used[i] || !std::equal(minseg, minseg + n, seg + (size_t)i * n)) continue;
      bool dup = false;
      for (int r : chosen)
        if (interchangeable(r, i, argid)) { dup = true; break; }
      if (!dup) chosen.push_back(i);
    }
    for (int i : chosen) {
      std::vector<int> saved;
      int nid = next_id;
      for (int a : seq[i])
        if (argid[a] < 0) {
          argid[a] = nid++;
          saved.push_back(a);
        }
      used[i] = 1;
      rows.push_back(i);
      size_t L = prefix.size();
      prefix.insert(prefix.end(), minseg, minseg + n);
      dfs(rows, used, argid, nid, prefix);
      prefix.resize(L);
      rows.pop_back();
      used[i] = 0;
      for (int a : saved) argid[a] = -1;
    }
  }

  // rows r1 and r2 give equal segments; swapping them together with their
  // private fresh arguments leaves the remaining problem unchanged
  bool interchangeable(int r1, int r2, const std::vector<int> &argid) const {
    for (int p = 0; p < e.n; ++p) {
      int a1 = seq[r1][p], a2 = seq[r2][p];
      bool n1 = argid[a1] >= 0, n2 = argid[a2] >= 0;
      if (n1 || n2) {
        if (!(n1 && n2 && a1 == a2)) return false;
        continue;
      }
      if (owner[a1] != r1 || owner[a2] != r2) return false;
      if (e.args[a1].dtype != e.args[a2].dtype) return false;
    }
    return true;
  }
};

}  // namespace

std::string key_text(const Einsum &f) {
  std::string s = "be1:" + std::to_string(f.b) + ";" + std::to_string(f.n) + ";";
  for (int8_t c : f.out) s += char('a' + c);
  s += "->";
  for (int j = 0; j < f.n; ++j) {
    if (j) s += ",";
    for (int8_t c : f.in[j]) s += char('a' + c);
  }
  s += ";";
  bool firstl = true;
  for (int c = 0; c < 26; ++c) {
    if (!f.used[c]) continue;
    if (!firstl) s += ",";
    s += std::to_string(f.len[c]);
    firstl = false;
  }
  s += ";";
  for (int i = 0; i < f.b; ++i) {
    if (i) s += "/";
    for (int j = 0; j < f.n; ++j) {
      if (j) s += ",";
      s += f.args[f.rows[i][j]].name;
    }
  }
  s += ";";
  for (size_t k = 0; k < f.args.size(); ++k) {
    if (k) s += ",";
    s += dtype_name(f.args[k].dtype);
  }
  return s;
}

int canonicalize(const Einsum &e, Canon &c, std::string &err) {
  // ---- GetCanonLabel: C_lex search ----
  OpSearch os(e);
  {
    std::vector<int> perm;
    std::vector<char> used(e.n, 0);
    int id_of[26];
    std::fill(id_of, id_of + 26, -1);
    int nid = 0;
    Tok prefix;
    for (int8_t ch : e.out) {
      if (id_of[ch] < 0) id_of[ch] = nid++;
    }
    os.dfs(perm, used, id_of, nid, prefix);
  }
  // lengths part decides among tied operand orders
  std::vector<const IndexCand *> tied;
  Tok best_len;
  for (auto &cand : os.cands) {
    Tok L(cand.n_ids);
    for (int ch = 0; ch < 26; ++ch)
      if (cand.id_of[ch] >= 0) L[cand.id_of[ch]] = e.len[ch];
    if (tied.empty() || L < best_len) {
      best_len = L;
      tied.clear();
    }
    if (L == best_len) tied.push_back(&cand);
  }
  const IndexCand *win = nullptr;
  std::vector<int> win_rows, win_argid;
  Tok bt, bd;
  bool have = false;
  for (const IndexCand *cand : tied) {
    RowSearch rs(e, cand->perm, have ? &bt : nullptr, have ? &bd : nullptr);
    std::vector<int> rows;
    std::vector<char> used(e.b, 0);
    std::vector<int> argid(e.args.size(), -1);
    Tok prefix;
    rs.dfs(rows, used, argid, 0, prefix);
    if (rs.improved) {
      win = cand;
      win_rows = rs.best_rows;
      win_argid = rs.best_argid;
      bt = rs.best_table;
      bd = rs.best_dt;
      have = true;
    }
  }
  if (!win) { err = "canonical search found no labeling"; return EINVALID; }

  // ---- RelabelingMap on the induced graph of e ----
  Graph g = to_induced_graph(e);
  const int n_arg = (int)e.args.size();
  const int n_index = e.n_index();
  std::vector<int> inv_row(e.b), inv_pos(e.n);
  for (int q = 0; q < e.b; ++q) inv_row[win_rows[q]] = q;
  for (int p = 0; p < e.n; ++p) inv_pos[win->perm[p]] = p;
  std::vector<int> R(g.n, -1);
  for (int a = 0; a < n_arg; ++a) R[g.arg_node[a]] = win_argid[a];
  for (int ch = 0; ch < 26; ++ch)
    if (g.index_node[ch] >= 0) R[g.index_node[ch]] = n_arg + win->id_of[ch];
  int acc_base = n_arg + n_index;
  std::vector<int> pos_off(e.n + 1, 0);     // canonical position offsets within a row
  for (int p = 0; p < e.n; ++p) pos_off[p + 1] = pos_off[p] + (int)e.in[win->perm[p]].size();
  const int row_len = pos_off[e.n];
  for (int i = 0; i < e.b; ++i)
    for (int j = 0; j < e.n; ++j)
      for (size_t d = 0; d < e.in[j].size(); ++d)
        R[g.acc_in_node[i][j][d]] = acc_base + inv_row[i] * row_len + pos_off[inv_pos[j]] + (int)d;
  for (int v = 0; v < g.n; ++v) {
    if (R[v] >= 0) continue;
    switch (g.color[v]) {
      case C_OUTPUT: R[v] = g.row_node[0] + inv_row[v - g.row_node[0]]; break;
      case C_ARGPOS: R[v] = g.pos_node[0] + inv_pos[v - g.pos_node[0]]; break;
      default: R[v] = v;   // output accesses, dtype, length and dim nodes are already canonical
    }
  }
  // ---- relabel (lines building A', c', iota'_dtype, iota'_length) ----
  Graph h;
  h.n = g.n;
  h.color.assign(g.n, 0);
  h.dtype_of.assign(g.n, 0);
  h.length_of.assign(g.n, -1);
  for (int v = 0; v < g.n; ++v) {
    h.color[R[v]] = g.color[v];
    h.dtype_of[R[v]] = g.dtype_of[v];
    h.length_of[R[v]] = g.length_of[v];
  }
  for (auto &ed : g.edges) h.edges.push_back({R[ed.first], R[ed.second]});
  // ---- ToBatchedEinsum ----
  std::vector<int> index_order, arg_order;
  int st = to_batched_einsum(h, c.form, index_order, arg_order, err);
  if (st) return st;
  c.form.text = key_text(c.form);
  c.key = c.form.text;
  // ---- sigma^A, sigma^I ----
  c.sigma_index.assign(n_index, -1);
  c.sigma_arg.assign(n_arg, -1);
  for (int ch = 0; ch < 26; ++ch)
    if (g.index_node[ch] >= 0) c.sigma_index[index_order[R[g.index_node[ch]]]] = ch;
  for (int a = 0; a < n_arg; ++a) c.sigma_arg[arg_order[R[g.arg_node[a]]]] = a;
  c.sigma_arg_name.clear();
  for (int k = 0; k < n_arg; ++k) c.sigma_arg_name.push_back(e.args[c.sigma_arg[k]].name);
  c.sigma_row = win_rows;
  c.sigma_pos = win->perm;
  c.relabel = R;
  c.graph_nodes = g.n;
  // ---- token vector of C(e) ----
  const Einsum &f = c.form;
  c.tokens = {f.b, f.n, (int64_t)f.out.size()};
  for (int8_t ch : f.out) c.tokens.push_back(ch);
  for (int j = 0; j < f.n; ++j) {
    c.tokens.push_back((int64_t)f.in[j].size());
    for (int8_t ch : f.in[j]) c.tokens.push_back(ch);
  }
  for (int ch = 0; ch < 26; ++ch)
    if (f.used[ch]) c.tokens.push_back(f.len[ch]);
  for (auto &r : f.rows)
    for (int a : r) c.tokens.push_back(a);
  for (auto &a : f.args) c.tokens.push_back(a.dtype);
  return OK;
}

}  // namespace be
