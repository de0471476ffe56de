// RaiseToBatchedEinsum (the first step of Alg. 2, Sec. "Integration with
// other frameworks"): a loop-nest kernel is read back as the functional
// batched einsum it computes.  The kernel language is a small loop-nest IR
// of our own, with the parts a raising needs:
//
//   { [i0,i1] : 0<=i0<96 and 0<=i1<4 }         loop domain (names, extents)
//   P:f64[96,4]                                  input array
//   u(i,j) := P[i,j]*P[i,j]                      substitution rule (a lambda)
//   for i0                                       loop nesting ... end
//     y1[i0] = sum([i1], u(i0,i1)*v(i1))         one statement per row
//   end
//
// Each statement y[..] = sum([..], f1(..)*f2(..)*..) (or a plain product)
// becomes one row: the output subscripts are the output indices, each factor
// (a rule call or an array access, subscripts loop names) one operand.  All
// statements must share one index structure up to a renaming of their loop
// names and the order of their factors; their factors then fill the rows.
// The result is written in the text grammar of be_parse and parsed, so the
// raised einsum goes through the same soundness checks, canonicalization and
// lookup as a textual one; the letters keep a map back to the loop names.
#include <algorithm>
#include <cctype>
#include <map>
#include <numeric>
#include <sstream>

#include "raise.hpp"

namespace be {

namespace {

std::string trim(const std::string &s) {
  size_t a = 0, b = s.size();
  while (a < b && std::isspace((unsigned char)s[a])) ++a;
  while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
  return s.substr(a, b - a);
}

bool is_name(const std::string &s) {
  if (s.empty() || !(std::isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
  for (char c : s)
    if (!(std::isalnum((unsigned char)c) || c == '_')) return false;
  return true;
}

std::vector<std::string> split_top(const std::string &s, char sep) {
  std::vector<std::string> out;
  int depth = 0;
  std::string cur;
  for (char c : s) {
    if (c == '(' || c == '[') ++depth;
    if (c == ')' || c == ']') --depth;
    if (c == sep && depth == 0) {
      out.push_back(trim(cur));
      cur.clear();
    } else {
      cur += c;
    }
  }
  out.push_back(trim(cur));
  return out;
}

// "name(a,b)" or "name[a,b]": name, bracket kind and subscript names
bool parse_call(const std::string &s, std::string &name, char &open, std::vector<std::string> &subs) {
  const size_t p = s.find_first_of("([");
  if (p == std::string::npos || s.empty()) return false;
  const char close = s[p] == '(' ? ')' : ']';
  if (s.back() != close) return false;
  name = trim(s.substr(0, p));
  open = s[p];
  subs.clear();
  const std::string inner = trim(s.substr(p + 1, s.size() - p - 2));
  if (!inner.empty())
    for (auto &t : split_top(inner, ',')) subs.push_back(t);
  return is_name(name);
}

struct Factor {
  std::string name;             // rule or array
  std::vector<std::string> subs;
};

struct Stmt {
  std::string out;
  std::vector<std::string> out_subs, red;
  std::vector<Factor> factors;
  int line = 0;
};

// loop names of a statement in order of first appearance (output, factors)
std::vector<std::string> first_appearance(const Stmt &s, const std::vector<int> &perm) {
  std::vector<std::string> order;
  auto add = [&](const std::string &n) {
    if (std::find(order.begin(), order.end(), n) == order.end()) order.push_back(n);
  };
  for (auto &n : s.out_subs) add(n);
  for (int k : perm)
    for (auto &n : s.factors[k].subs) add(n);
  return order;
}

// index structure of a statement under factor order perm: every subscript
// replaced by its first-appearance position
std::vector<std::vector<int>> structure(const Stmt &s, const std::vector<int> &perm) {
  const auto order = first_appearance(s, perm);
  auto pos = [&](const std::string &n) { return (int)(std::find(order.begin(), order.end(), n) - order.begin()); };
  std::vector<std::vector<int>> st;
  std::vector<int> o;
  for (auto &n : s.out_subs) o.push_back(pos(n));
  st.push_back(o);
  for (int k : perm) {
    std::vector<int> f;
    for (auto &n : s.factors[k].subs) f.push_back(pos(n));
    st.push_back(f);
  }
  return st;
}

// array references name[s0,s1,..] in a rule body: (array, subscripts)
std::vector<std::pair<std::string, std::vector<std::string>>> array_refs(const std::string &body,
                                                                          const std::map<std::string, int> &arrays) {
  std::vector<std::pair<std::string, std::vector<std::string>>> out;
  for (size_t i = 0; i < body.size();) {
    if (std::isalpha((unsigned char)body[i]) || body[i] == '_') {
      size_t j = i;
      while (j < body.size() && (std::isalnum((unsigned char)body[j]) || body[j] == '_')) ++j;
      const std::string name = body.substr(i, j - i);
      size_t k = j;
      while (k < body.size() && std::isspace((unsigned char)body[k])) ++k;
      if (k < body.size() && body[k] == '[' && arrays.count(name)) {
        const size_t close = body.find(']', k);
        if (close == std::string::npos) break;
        out.push_back({name, split_top(body.substr(k + 1, close - k - 1), ',')});
        i = close + 1;
        continue;
      }
      i = j;
    } else {
      ++i;
    }
  }
  return out;
}

}  // namespace

int raise_kernel(const std::string &text, Raised &r, std::string &err) {
  r = Raised();
  std::map<std::string, int64_t> extent;
  std::vector<std::string> domain_order;
  std::vector<std::string> arrays, array_decls, rule_decls;
  std::map<std::string, int> array_rank;
  std::map<std::string, std::string> array_dtype;
  std::map<std::string, int> rule_arity;
  std::map<std::string, std::vector<std::string>> rule_params;
  std::map<std::string, std::string> rule_body;
  std::vector<std::string> rule_order;
  std::vector<std::string> loop_stack;
  std::vector<Stmt> stmts;
  std::istringstream in(text);
  std::string raw;
  int ln = 0;
  auto bad = [&](int code, const std::string &m) {
    err = "line " + std::to_string(ln) + ": " + m;
    return code;
  };
  while (std::getline(in, raw)) {
    ++ln;
    const size_t hash = raw.find('#');
    std::string line = trim(hash == std::string::npos ? raw : raw.substr(0, hash));
    if (line.empty()) continue;
    if (line[0] == '{') {   // { [i0,i1] : 0<=i0<N and ... }
      if (line.back() != '}') return bad(EPARSE, "domain must end with '}'");
      const std::string body = trim(line.substr(1, line.size() - 2));
      const size_t colon = body.find(':');
      if (colon == std::string::npos) return bad(EPARSE, "domain needs ':'");
      std::string names = trim(body.substr(0, colon));
      if (names.size() < 2 || names.front() != '[' || names.back() != ']') return bad(EPARSE, "domain names in [..]");
      for (auto &n : split_top(names.substr(1, names.size() - 2), ',')) {
        if (!is_name(n)) return bad(EPARSE, "bad loop name '" + n + "'");
        if (extent.count(n)) return bad(EINVALID, "loop '" + n + "' declared twice");
        extent[n] = -1;
        domain_order.push_back(n);
      }
      std::string bounds = body.substr(colon + 1);
      size_t p;
      while ((p = bounds.find(" and ")) != std::string::npos) bounds.replace(p, 5, ",");
      for (auto &b : split_top(bounds, ',')) {
        // 0<=name<N
        std::string t;
        for (char c : b)
          if (!std::isspace((unsigned char)c)) t += c;
        if (t.rfind("0<=", 0) != 0) return bad(EPARSE, "bound must read 0<=name<N: '" + b + "'");
        const size_t lt = t.find('<', 3);
        if (lt == std::string::npos) return bad(EPARSE, "bound must read 0<=name<N: '" + b + "'");
        const std::string n = t.substr(3, lt - 3), v = t.substr(lt + 1);
        if (!extent.count(n)) return bad(EINVALID, "bound on an undeclared loop '" + n + "'");
        if (v.empty() || !std::all_of(v.begin(), v.end(), [](char c) { return std::isdigit((unsigned char)c); }))
          return bad(EPARSE, "extent must be a number: '" + v + "'");
        extent[n] = std::atoll(v.c_str());
      }
      continue;
    }
    if (line.rfind("for ", 0) == 0) {
      const std::string n = trim(line.substr(4));
      if (!extent.count(n)) return bad(EINVALID, "loop '" + n + "' is not in the domain");
      if (std::find(loop_stack.begin(), loop_stack.end(), n) != loop_stack.end())
        return bad(EINVALID, "loop '" + n + "' nested in itself");
      loop_stack.push_back(n);
      continue;
    }
    if (line == "end") {
      if (loop_stack.empty()) return bad(EPARSE, "'end' without 'for'");
      loop_stack.pop_back();
      continue;
    }
    const size_t def = line.find(":=");
    if (def != std::string::npos) {   // substitution rule
      std::string name;
      char open;
      std::vector<std::string> params;
      std::string head = trim(line.substr(0, def));
      const size_t ann = head.find(')');
      if (ann != std::string::npos && ann + 1 < head.size()) head = trim(head.substr(0, ann + 1));
      if (!parse_call(head, name, open, params) || open != '(') return bad(EPARSE, "rule must read name(p,..) := expr");
      if (rule_arity.count(name) || array_rank.count(name)) return bad(EINVALID, "name '" + name + "' defined twice");
      rule_arity[name] = (int)params.size();
      rule_params[name] = params;
      rule_body[name] = trim(line.substr(def + 2));
      rule_order.push_back(name);
      rule_decls.push_back(line);
      continue;
    }
    const size_t eq = line.find('=');
    if (eq == std::string::npos) {   // array declaration name:dtype[dims]
      const size_t colon = line.find(':');
      if (colon == std::string::npos) return bad(EPARSE, "expected a declaration, rule, loop or statement");
      const std::string name = trim(line.substr(0, colon));
      if (!is_name(name)) return bad(EPARSE, "bad array name '" + name + "'");
      if (rule_arity.count(name) || array_rank.count(name)) return bad(EINVALID, "name '" + name + "' defined twice");
      const std::string ty = trim(line.substr(colon + 1));
      const size_t lb = ty.find('[');
      if (lb == std::string::npos || ty.back() != ']') return bad(EPARSE, "array must read name:dtype[dims]");
      const std::string dims = trim(ty.substr(lb + 1, ty.size() - lb - 2));
      array_rank[name] = dims.empty() ? 0 : (int)split_top(dims, ',').size();
      array_dtype[name] = trim(ty.substr(0, lb));
      arrays.push_back(name);
      array_decls.push_back(name + ":" + ty);
      continue;
    }
    // statement
    Stmt st;
    st.line = ln;
    std::string name;
    char open;
    if (!parse_call(trim(line.substr(0, eq)), name, open, st.out_subs) || open != '[')
      return bad(EPARSE, "statement must read y[i,..] = ..");
    st.out = name;
    std::string rhs = trim(line.substr(eq + 1));
    if (rhs.rfind("sum(", 0) == 0 || rhs.rfind("sum (", 0) == 0) {
      const size_t lp = rhs.find('(');
      if (rhs.back() != ')') return bad(EPARSE, "sum(..) not closed");
      const auto parts = split_top(trim(rhs.substr(lp + 1, rhs.size() - lp - 2)), ',');
      if (parts.size() != 2) return bad(EPARSE, "sum must read sum([names], product)");
      const std::string &rl = parts[0];
      if (rl.size() < 2 || rl.front() != '[' || rl.back() != ']') return bad(EPARSE, "sum names in [..]");
      for (auto &n : split_top(rl.substr(1, rl.size() - 2), ','))
        if (!n.empty()) st.red.push_back(n);
      rhs = parts[1];
    }
    for (auto &f : split_top(rhs, '*')) {
      Factor fc;
      if (!parse_call(f, fc.name, open, fc.subs)) return bad(EPARSE, "factor must read r(i,..) or A[i,..]: '" + f + "'");
      if (open == '(' ? !rule_arity.count(fc.name) : !array_rank.count(fc.name))
        return bad(EINVALID, std::string(open == '(' ? "unknown rule '" : "unknown array '") + fc.name + "'");
      const int want = open == '(' ? rule_arity[fc.name] : array_rank[fc.name];
      if ((int)fc.subs.size() != want) return bad(EINVALID, "'" + fc.name + "' takes " + std::to_string(want) + " subscripts");
      st.factors.push_back(fc);
    }
    // subscripts: outputs from the enclosing loops, the rest reduced
    for (auto &n : st.out_subs)
      if (std::find(loop_stack.begin(), loop_stack.end(), n) == loop_stack.end())
        return bad(EINVALID, "output subscript '" + n + "' is not an enclosing loop");
    for (auto &n : st.red) {
      if (!extent.count(n)) return bad(EINVALID, "reduction over an undeclared loop '" + n + "'");
      if (std::find(loop_stack.begin(), loop_stack.end(), n) != loop_stack.end())
        return bad(EINVALID, "reduction over an enclosing loop '" + n + "'");
    }
    for (auto &fc : st.factors)
      for (auto &n : fc.subs) {
        const bool outer = std::find(st.out_subs.begin(), st.out_subs.end(), n) != st.out_subs.end();
        const bool red = std::find(st.red.begin(), st.red.end(), n) != st.red.end();
        if (!outer && !red) return bad(EINVALID, "subscript '" + n + "' of '" + fc.name + "' is neither an output index nor reduced");
      }
    stmts.push_back(st);
  }
  ln = 0;
  if (!loop_stack.empty()) return bad(EPARSE, "'for' without 'end'");
  if (stmts.empty()) return bad(EINVALID, "no statement");
  for (auto &kv : extent)
    if (kv.second < 0) return bad(EINVALID, "loop '" + kv.first + "' has no extent");
  // structure of statement 0; every other statement is matched under some
  // order of its factors
  const Stmt &s0 = stmts[0];
  const int n = (int)s0.factors.size();
  std::vector<int> id(n);
  std::iota(id.begin(), id.end(), 0);
  const auto st0 = structure(s0, id);
  const auto names0 = first_appearance(s0, id);
  std::vector<std::vector<int>> perms(stmts.size());
  perms[0] = id;
  for (size_t k = 1; k < stmts.size(); ++k) {
    const Stmt &s = stmts[k];
    if ((int)s.factors.size() != n) {
      err = "line " + std::to_string(s.line) + ": statements do not form one batched einsum (operand count)";
      return EINVALID;
    }
    std::vector<int> p = id;
    bool found = false;
    do {
      if (structure(s, p) == st0) {
        // lengths must agree too
        const auto nk = first_appearance(s, p);
        bool same = true;
        for (size_t q = 0; q < nk.size(); ++q) same = same && extent[nk[q]] == extent[names0[q]];
        if (same) { found = true; break; }
      }
    } while (std::next_permutation(p.begin(), p.end()));
    if (!found) {
      err = "line " + std::to_string(s.line) + ": statements do not form one batched einsum (index structure)";
      return EINVALID;
    }
    perms[k] = p;
  }
  if (names0.size() > 26) { err = "more than 26 loop indices"; return ETOOMANY; }
  // letters by first appearance in statement 0
  auto letter = [&](const std::string &nm) {
    return (char)('a' + (std::find(names0.begin(), names0.end(), nm) - names0.begin()));
  };
  std::string notation;
  for (int k = 0; k < n; ++k) {
    if (k) notation += ",";
    for (auto &nm : s0.factors[k].subs) notation += letter(nm);
  }
  notation += "->";
  for (auto &nm : s0.out_subs) notation += letter(nm);
  std::string spec = notation;
  for (size_t k = 0; k < stmts.size(); ++k) {
    spec += " | ";
    for (int q = 0; q < n; ++q) spec += (q ? "," : "") + stmts[k].factors[perms[k][q]].name;
  }
  for (auto &d : array_decls) spec += " ; " + d;
  // rules: a parameter that no array subscript of the body names gets its
  // extent from the loop it is called with (first call), through a domain
  // annotation whose dtype is the highest of the referenced arrays (f64 for none)
  std::map<std::string, std::vector<int64_t>> rule_dims;
  for (size_t k = 0; k < stmts.size(); ++k)
    for (auto &f : stmts[k].factors)
      if (rule_arity.count(f.name) && !rule_dims.count(f.name)) {
        std::vector<int64_t> d;
        for (auto &nm : f.subs) d.push_back(extent[nm]);
        rule_dims[f.name] = d;
      }
  static const char *rank_order[] = {"i8", "i32", "i64", "f16", "bf16", "f32", "f64", "c64", "c128"};
  for (size_t k = 0; k < rule_order.size(); ++k) {
    const std::string &nm = rule_order[k];
    const auto refs = array_refs(rule_body[nm], array_rank);
    bool inferable = true;
    for (auto &prm : rule_params[nm]) {
      bool named = false;
      for (auto &rf : refs)
        for (auto &sb : rf.second) named = named || trim(sb) == prm;
      inferable = inferable && named;
    }
    if (inferable || !rule_dims.count(nm)) {
      spec += " ; " + rule_decls[k];
      continue;
    }
    int best = -1;
    for (auto &rf : refs)
      for (int q = 0; q < 9; ++q)
        if (array_dtype[rf.first] == rank_order[q]) best = std::max(best, q);
    std::string ann = std::string(best < 0 ? "f64" : rank_order[best]) + "[";
    for (size_t q = 0; q < rule_dims[nm].size(); ++q) ann += (q ? "," : "") + std::to_string(rule_dims[nm][q]);
    ann += "]";
    std::string pl;
    for (size_t q = 0; q < rule_params[nm].size(); ++q) pl += (q ? "," : "") + rule_params[nm][q];
    spec += " ; " + nm + "(" + pl + "):" + ann + " := " + rule_body[nm];
  }
  r.spec = spec;
  r.loop_names = names0;
  for (auto &s : stmts) r.outputs.push_back(s.out);
  return OK;
}

}  // namespace be
