// Parser of the textual batched-einsum spec (be_parse).
//
//   spec     := notation ('|' row)+ (';' decl)*
//   notation := idx (',' idx)* '->' idx        idx := letters a..z
//   row      := name (',' name)*               one name per operand
//   decl     := name ':' dtype '[' dims ']'                     buffer
//             | name '(' params ')' [':' dtype ['[' dims ']']] ':=' expr
//
// Index letters follow the index grammar of Sec. "Preliminaries" (a..z).
// A name used in a row is an idealized argument: a declared buffer (the
// identity lambda) or a functional operand given by a producer expression
// (Def. "Functional Batched Einstein Summation").  Soundness follows the
// four rules listed after Eq. (1) and is checked for every row of the batch.
#include <cctype>
#include <cstdlib>
#include <map>

#include "ir.hpp"

namespace be {

const char *dtype_name(int dt) {
  switch (dt) {
    case I8: return "int8";
    case I32: return "int32";
    case I64: return "int64";
    case F16: return "float16";
    case F32: return "float32";
    case F64: return "float64";
    case C64: return "complex64";
    case C128: return "complex128";
    case BF16: return "bfloat16";
  }
  return "?";
}

int dtype_from_text(const std::string &s) {
  static const std::map<std::string, int> m = {
      {"i8", I8}, {"int8", I8}, {"i32", I32}, {"int32", I32}, {"i64", I64}, {"int64", I64},
      {"f16", F16}, {"float16", F16}, {"f32", F32}, {"float32", F32}, {"f64", F64},
      {"float64", F64}, {"c64", C64}, {"complex64", C64}, {"c128", C128},
      {"complex128", C128}, {"bf16", BF16}, {"bfloat16", BF16}};
  auto it = m.find(s);
  return it == m.end() ? 0 : it->second;
}

int dtype_size(int dt) {
  switch (dt) {
    case I8: return 1;
    case F16: case BF16: return 2;
    case I32: case F32: return 4;
    case I64: case F64: case C64: return 8;
    case C128: return 16;
  }
  return 0;
}

int dtype_promote_rank(int dt) {
  switch (dt) {
    case I8: return 0;
    case I32: return 1;
    case I64: return 2;
    case BF16: return 3;
    case F16: return 4;
    case F32: return 5;
    case F64: return 6;
    case C64: return 7;
    case C128: return 8;
  }
  return -1;
}

namespace {

std::string trim(const std::string &s) {
  size_t a = 0, b = s.size();
  while (a < b && std::isspace((unsigned char)s[a])) ++a;
  while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
  return s.substr(a, b - a);
}

std::vector<std::string> split(const std::string &s, char c) {
  std::vector<std::string> out;
  size_t start = 0;
  for (size_t i = 0; i <= s.size(); ++i) {
    if (i == s.size() || s[i] == c) {
      out.push_back(s.substr(start, i - start));
      start = i + 1;
    }
  }
  return out;
}

bool is_ident(const std::string &s) {
  if (s.empty() || !(std::isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
  for (char ch : s)
    if (!(std::isalnum((unsigned char)ch) || ch == '_')) return false;
  return true;
}

struct Lexer {
  std::string s;
  size_t p = 0;
  std::string tok;
  bool err = false;
  explicit Lexer(const std::string &t) : s(t) { next(); }
  void next() {
    while (p < s.size() && std::isspace((unsigned char)s[p])) ++p;
    if (p >= s.size()) { tok.clear(); return; }
    size_t st = p;
    char c = s[p];
    if (std::isdigit((unsigned char)c) || (c == '.' && p + 1 < s.size() && std::isdigit((unsigned char)s[p + 1]))) {
      char *end = nullptr;
      std::strtod(s.c_str() + p, &end);
      p = end - s.c_str();
    } else if (std::isalpha((unsigned char)c) || c == '_' || c == '$') {
      ++p;
      while (p < s.size() && (std::isalnum((unsigned char)s[p]) || s[p] == '_')) ++p;
    } else if ((c == '=' || c == '!') && p + 1 < s.size() && s[p + 1] == '=') {
      p += 2;
    } else if (std::string("+-*/()[],?:").find(c) != std::string::npos) {
      ++p;
    } else {
      err = true;
      tok = std::string(1, c);
      p = s.size();
      return;
    }
    tok = s.substr(st, p - st);
  }
};

struct ExprParser {
  Lexer lx;
  Einsum &e;
  Arg &a;
  std::string &err;
  bool bad = false;
  ExprParser(const std::string &t, Einsum &e_, Arg &a_, std::string &err_) : lx(t), e(e_), a(a_), err(err_) {}

  int add(XNode n) {
    a.nodes.push_back(std::move(n));
    return (int)a.nodes.size() - 1;
  }
  bool expect(const char *t) {
    if (lx.tok != t) {
      if (!bad) err = std::string("expected '") + t + "' near '" + lx.tok + "'";
      bad = true;
      return false;
    }
    lx.next();
    return true;
  }
  int expr() {
    int c = cmp();
    if (lx.tok == "?") {
      lx.next();
      int x = expr();
      expect(":");
      int y = expr();
      XNode n{X_SELECT};
      n.kids = {c, x, y};
      return add(n);
    }
    return c;
  }
  int cmp() {
    int x = sum();
    if (lx.tok == "==" || lx.tok == "!=") {
      XOp op = lx.tok == "==" ? X_EQ : X_NE;
      lx.next();
      int y = sum();
      XNode n{op};
      n.kids = {x, y};
      return add(n);
    }
    return x;
  }
  int sum() {
    int x = prod();
    while (lx.tok == "+" || lx.tok == "-") {
      XOp op = lx.tok == "+" ? X_ADD : X_SUB;
      lx.next();
      int y = prod();
      XNode n{op};
      n.kids = {x, y};
      x = add(n);
    }
    return x;
  }
  int prod() {
    int x = unary();
    while (lx.tok == "*" || lx.tok == "/") {
      XOp op = lx.tok == "*" ? X_MUL : X_DIV;
      lx.next();
      int y = unary();
      XNode n{op};
      n.kids = {x, y};
      x = add(n);
    }
    return x;
  }
  int unary() {
    if (lx.tok == "-") {
      lx.next();
      XNode n{X_NEG};
      n.kids = {unary()};
      return add(n);
    }
    if (lx.tok == "+") {
      lx.next();
      return unary();
    }
    return primary();
  }
  int primary() {
    if (bad) return add(XNode{X_NUM});
    std::string t = lx.tok;
    if (t.empty()) {
      err = "unexpected end of expression";
      bad = true;
      return add(XNode{X_NUM});
    }
    if (t == "(") {
      lx.next();
      int x = expr();
      expect(")");
      return x;
    }
    if (std::isdigit((unsigned char)t[0]) || t[0] == '.') {
      XNode n{X_NUM};
      n.num = std::strtod(t.c_str(), nullptr);
      lx.next();
      return add(n);
    }
    if (t[0] == '$') {
      std::string nm = t.substr(1);
      if (!is_ident(nm)) { err = "bad scalar name"; bad = true; return add(XNode{X_NUM}); }
      int id = -1;
      for (size_t k = 0; k < e.scalars.size(); ++k)
        if (e.scalars[k] == nm) id = (int)k;
      if (id < 0) { e.scalars.push_back(nm); id = (int)e.scalars.size() - 1; }
      XNode n{X_SCALAR};
      n.id = id;
      lx.next();
      return add(n);
    }
    if (!is_ident(t)) {
      err = "unexpected token '" + t + "'";
      bad = true;
      return add(XNode{X_NUM});
    }
    lx.next();
    if (lx.tok == "(") {
      XOp op;
      if (t == "sin") op = X_SIN;
      else if (t == "cos") op = X_COS;
      else if (t == "exp") op = X_EXP;
      else if (t == "abs") op = X_ABS;
      else { err = "unknown function " + t; bad = true; return add(XNode{X_NUM}); }
      lx.next();
      int x = expr();
      expect(")");
      XNode n{op};
      n.kids = {x};
      return add(n);
    }
    if (lx.tok == "[") {
      lx.next();
      int bid = -1;
      for (size_t k = 0; k < e.buffers.size(); ++k)
        if (e.buffers[k].name == t) bid = (int)k;
      if (bid < 0) { err = "unknown buffer " + t + " (declare buffers before lambdas)"; bad = true; return add(XNode{X_NUM}); }
      XNode n{X_REF};
      n.id = bid;
      while (true) {
        std::string s = lx.tok;
        if (!s.empty() && std::isdigit((unsigned char)s[0])) {
          n.sub.push_back(-(std::atoi(s.c_str()) + 1));
        } else if (is_ident(s)) {
          int pp = -1;
          for (size_t k = 0; k < a.params.size(); ++k)
            if (a.params[k] == s) pp = (int)k;
          if (pp < 0) { err = "unknown lambda parameter " + s; bad = true; return add(XNode{X_NUM}); }
          n.sub.push_back(pp);
        } else {
          err = "bad subscript '" + s + "'";
          bad = true;
          return add(XNode{X_NUM});
        }
        lx.next();
        if (lx.tok == ",") { lx.next(); continue; }
        if (!expect("]")) return add(XNode{X_NUM});
        break;
      }
      return add(n);
    }
    int pp = -1;
    for (size_t k = 0; k < a.params.size(); ++k)
      if (a.params[k] == t) pp = (int)k;
    if (pp < 0) { err = "unknown name " + t; bad = true; return add(XNode{X_NUM}); }
    XNode n{X_PARAM};
    n.id = pp;
    return add(n);
  }
};

int parse_dims(const std::string &s, std::vector<int64_t> &dims, std::string &err) {
  dims.clear();
  std::string t = trim(s);
  if (t.empty()) return OK;
  for (auto &part : split(t, ',')) {
    std::string q = trim(part);
    if (q.empty()) { err = "empty dimension"; return EPARSE; }
    for (char ch : q)
      if (!std::isdigit((unsigned char)ch)) { err = "bad dimension '" + q + "'"; return EPARSE; }
    dims.push_back(std::atoll(q.c_str()));
  }
  return OK;
}

}  // namespace

int check_sound(Einsum &e, std::string &err) {
  for (int c = 0; c < 26; ++c) { e.len[c] = -1; e.used[c] = false; }
  if (e.n == 0) { err = "n = 0: an einsum needs at least one operand"; return EINVALID; }
  for (int i = 0; i < e.b; ++i) {
    for (int j = 0; j < e.n; ++j) {
      const Arg &a = e.args[e.rows[i][j]];
      if (a.shape.size() != e.in[j].size()) {
        err = "Dim(" + a.name + ") differs from the length of index list " + std::to_string(j + 1);
        return EINVALID;
      }
      for (size_t d = 0; d < a.shape.size(); ++d) {
        int c = e.in[j][d];
        if (e.len[c] >= 0 && e.len[c] != a.shape[d]) {
          err = std::string("axis length of index '") + char('a' + c) + "' is inconsistent";
          return ESHAPE;
        }
        e.len[c] = a.shape[d];
        e.used[c] = true;
      }
    }
  }
  for (int8_t c : e.out)
    if (!e.used[c]) {
      err = std::string("output index '") + char('a' + c) + "' does not appear in any input";
      return EINVALID;
    }
  for (int c = 0; c < 26; ++c)
    if (!e.used[c]) e.len[c] = 0;
  return OK;
}

int parse(const std::string &text, Einsum &e, std::string &err) {
  e = Einsum();
  e.text = text;
  auto parts = split(text, ';');
  auto head = split(parts[0], '|');
  std::string notation;
  for (char ch : head[0])
    if (!std::isspace((unsigned char)ch)) notation += ch;
  size_t arrow = notation.find("->");
  if (arrow == std::string::npos) { err = "missing '->'"; return EPARSE; }
  std::string lhs = notation.substr(0, arrow), rhs = notation.substr(arrow + 2);
  auto parse_list = [&](const std::string &s, std::vector<int8_t> &v) -> bool {
    for (char ch : s) {
      if (ch < 'a' || ch > 'z') return false;
      v.push_back((int8_t)(ch - 'a'));
    }
    return true;
  };
  if (!parse_list(rhs, e.out)) { err = "bad output index list '" + rhs + "'"; return EPARSE; }
  {
    bool seen[26] = {false};
    for (int8_t c : e.out) {
      if (seen[c]) { err = "repeated output index"; return EINVALID; }
      seen[c] = true;
    }
  }
  if (!lhs.empty()) {
    for (auto &s : split(lhs, ',')) {
      std::vector<int8_t> v;
      if (!parse_list(s, v)) { err = "bad index list '" + s + "'"; return EPARSE; }
      e.in.push_back(v);
    }
  }
  e.n = (int)e.in.size();
  if (e.n == 0) { err = "n = 0: an einsum needs at least one operand"; return EINVALID; }
  if (e.n > 16) { err = "more than 16 operands"; return ETOOMANY; }
  for (size_t j = 0; j < e.in.size(); ++j)
    if (e.in[j].empty()) {
      err = "a 0-dimensional operand has no access nodes in the induced graph";
      return EUNSUPPORTED;
    }
  std::vector<std::vector<std::string>> row_names;
  for (size_t r = 1; r < head.size(); ++r) {
    std::vector<std::string> names;
    for (auto &x : split(head[r], ',')) {
      std::string nm = trim(x);
      if (!is_ident(nm)) { err = "bad argument name '" + nm + "'"; return EPARSE; }
      names.push_back(nm);
    }
    if ((int)names.size() != e.n) { err = "row arity differs from the notation"; return EINVALID; }
    row_names.push_back(names);
  }
  e.b = (int)row_names.size();
  if (e.b == 0) { err = "no rows"; return EINVALID; }
  if (e.b > 4096) { err = "more than 4096 rows"; return ETOOMANY; }

  struct FunDecl { std::string name, params, dtype, dims, body; bool has_dims; };
  std::vector<FunDecl> funs;
  for (size_t k = 1; k < parts.size(); ++k) {
    std::string d = trim(parts[k]);
    if (d.empty()) continue;
    size_t def = d.find(":=");
    if (def == std::string::npos) {
      size_t colon = d.find(':');
      size_t lb = d.find('['), rb = d.rfind(']');
      if (colon == std::string::npos || lb == std::string::npos || rb == std::string::npos || rb < lb || lb < colon) {
        err = "bad declaration '" + d + "'";
        return EPARSE;
      }
      Buffer bf;
      bf.name = trim(d.substr(0, colon));
      if (!is_ident(bf.name)) { err = "bad buffer name '" + bf.name + "'"; return EPARSE; }
      bf.dtype = dtype_from_text(trim(d.substr(colon + 1, lb - colon - 1)));
      if (!bf.dtype) { err = "unknown dtype in '" + d + "'"; return EDTYPE; }
      if (!trim(d.substr(rb + 1)).empty()) { err = "trailing text in '" + d + "'"; return EPARSE; }
      int st = parse_dims(d.substr(lb + 1, rb - lb - 1), bf.shape, err);
      if (st) return st;
      for (auto &b2 : e.buffers)
        if (b2.name == bf.name) { err = "buffer declared twice: " + bf.name; return EINVALID; }
      e.buffers.push_back(bf);
    } else {
      std::string lhs2 = d.substr(0, def), body = d.substr(def + 2);
      size_t lp = lhs2.find('('), rp = lhs2.find(')');
      if (lp == std::string::npos || rp == std::string::npos || rp < lp) { err = "bad lambda '" + d + "'"; return EPARSE; }
      FunDecl f;
      f.name = trim(lhs2.substr(0, lp));
      f.params = lhs2.substr(lp + 1, rp - lp - 1);
      std::string rest = trim(lhs2.substr(rp + 1));
      f.has_dims = false;
      if (!rest.empty()) {
        if (rest[0] != ':') { err = "bad lambda annotation '" + rest + "'"; return EPARSE; }
        rest = trim(rest.substr(1));
        size_t lb = rest.find('[');
        if (lb == std::string::npos) {
          f.dtype = rest;
        } else {
          size_t rb = rest.rfind(']');
          if (rb == std::string::npos) { err = "bad lambda annotation"; return EPARSE; }
          f.dtype = trim(rest.substr(0, lb));
          f.dims = rest.substr(lb + 1, rb - lb - 1);
          f.has_dims = true;
        }
      }
      f.body = body;
      if (!is_ident(f.name)) { err = "bad lambda name '" + f.name + "'"; return EPARSE; }
      funs.push_back(f);
    }
  }

  // idealized arguments in first-appearance order
  std::map<std::string, int> arg_id;
  for (int i = 0; i < e.b; ++i) {
    std::vector<int> row;
    for (int j = 0; j < e.n; ++j) {
      const std::string &nm = row_names[i][j];
      auto it = arg_id.find(nm);
      if (it == arg_id.end()) {
        Arg a;
        a.name = nm;
        int bid = -1;
        for (size_t k = 0; k < e.buffers.size(); ++k)
          if (e.buffers[k].name == nm) bid = (int)k;
        const FunDecl *fd = nullptr;
        for (auto &f : funs)
          if (f.name == nm) fd = &f;
        if (bid >= 0 && fd) { err = "name is both a buffer and a lambda: " + nm; return EINVALID; }
        if (bid >= 0) {
          a.buffer = bid;
          a.dtype = e.buffers[bid].dtype;
          a.shape = e.buffers[bid].shape;
        } else if (fd) {
          for (auto &p : split(fd->params, ',')) {
            std::string q = trim(p);
            if (q.empty()) continue;
            if (!is_ident(q)) { err = "bad lambda parameter '" + q + "'"; return EPARSE; }
            a.params.push_back(q);
          }
          ExprParser xp(fd->body, e, a, err);
          a.root = xp.expr();
          if (xp.bad) return EPARSE;
          if (xp.lx.err || !xp.lx.tok.empty()) { err = "trailing input in lambda " + nm; return EPARSE; }
          // domain: annotation, else extents of the buffer dims each parameter subscripts
          std::vector<int64_t> shape(a.params.size(), -1);
          if (fd->has_dims) {
            std::vector<int64_t> dd;
            int st = parse_dims(fd->dims, dd, err);
            if (st) return st;
            if (dd.size() != a.params.size()) { err = nm + ": annotated shape rank differs from its parameters"; return EINVALID; }
            shape = dd;
          }
          int best = -1;
          for (auto &nd : a.nodes) {
            if (nd.op != X_REF) continue;
            const Buffer &bf = e.buffers[nd.id];
            if (bf.shape.size() != nd.sub.size()) { err = nm + ": wrong subscript count for " + bf.name; return EINVALID; }
            if (dtype_promote_rank(bf.dtype) > best) { best = dtype_promote_rank(bf.dtype); a.dtype = bf.dtype; }
            for (size_t d = 0; d < nd.sub.size(); ++d) {
              int s = nd.sub[d];
              if (s >= 0) {
                if (shape[s] < 0) shape[s] = bf.shape[d];
                else if (shape[s] != bf.shape[d]) { err = nm + ": inconsistent extent of parameter " + a.params[s]; return ESHAPE; }
              } else if (-(s + 1) >= bf.shape[d]) {
                err = nm + ": constant subscript out of range for " + bf.name;
                return ESHAPE;
              }
            }
          }
          if (best < 0) a.dtype = F64;
          for (size_t k = 0; k < shape.size(); ++k)
            if (shape[k] < 0) { err = nm + ": cannot infer the extent of parameter " + a.params[k]; return EINVALID; }
          a.shape = shape;
          if (!fd->dtype.empty()) {
            a.dtype = dtype_from_text(fd->dtype);
            if (!a.dtype) { err = "unknown dtype " + fd->dtype; return EDTYPE; }
          }
        } else {
          err = "undeclared argument " + nm;
          return EINVALID;
        }
        e.args.push_back(a);
        it = arg_id.emplace(nm, (int)e.args.size() - 1).first;
      }
      row.push_back(it->second);
    }
    e.rows.push_back(row);
  }
  int best = -1;
  for (auto &a : e.args)
    if (dtype_promote_rank(a.dtype) > best) { best = dtype_promote_rank(a.dtype); e.out_dtype = a.dtype; }
  return check_sound(e, err);
}

}  // namespace be
