// Planner: turns a parsed batched einsum plus the caller's buffers into the
// parameter block of one strategy and launches it.
//
// Every argument at every operand position is resolved either to a strided
// view (the identity lambda of an idealized argument, or a lambda whose
// body is a single buffer reference, e.g. G[e,r,0]) or to a producer
// program in postfix form that the kernel evaluates at each access, so
// elementwise producers run inside the operand loads (Def. "Functional
// Batched Einstein Summation"; the fused listing of the Feinsum section).
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "plan.hpp"

namespace be {

namespace {

int esz(int dt) { return dtype_size(dt); }

// strides of declared buffer k as the caller passed them (row-major if none)
void strides_of(const BufIn &b, const Buffer &decl, std::vector<int64_t> &st) {
  st.assign(decl.shape.size(), 0);
  if (b.strides) {
    for (size_t d = 0; d < decl.shape.size(); ++d) st[d] = b.strides[d];
  } else {
    int64_t s = 1;
    for (int d = (int)decl.shape.size() - 1; d >= 0; --d) {
      st[d] = s;
      s *= decl.shape[d];
    }
  }
}

}  // namespace

bool arg_view(const Einsum &e, int arg, int pos, const std::vector<BufIn> &bufs, View &v) {
  const Arg &a = e.args[arg];
  std::fill(v.coef, v.coef + 26, 0);
  std::vector<int64_t> st;
  if (!a.functional()) {
    const Buffer &bf = e.buffers[a.buffer];
    strides_of(bufs[a.buffer], bf, st);
    for (size_t d = 0; d < bf.shape.size(); ++d) v.coef[e.in[pos][d]] += st[d];
    v.ptr = (const char *)bufs[a.buffer].ptr;
    v.dtype = bf.dtype;
    return true;
  }
  const XNode &root = a.nodes[a.root];
  if (root.op != X_REF) return false;
  const Buffer &bf = e.buffers[root.id];
  strides_of(bufs[root.id], bf, st);
  int64_t off = 0;
  for (size_t d = 0; d < root.sub.size(); ++d) {
    int s = root.sub[d];
    if (s >= 0) v.coef[e.in[pos][s]] += st[d];
    else off += (int64_t)(-(s + 1)) * st[d];
  }
  v.ptr = (const char *)bufs[root.id].ptr + off * esz(bf.dtype);
  v.dtype = bf.dtype;
  return true;
}

// view of a REF node of arg's body at position pos
static void ref_view(const Einsum &e, const XNode &nd, int pos, const std::vector<BufIn> &bufs, View &v) {
  const Buffer &bf = e.buffers[nd.id];
  std::vector<int64_t> st;
  strides_of(bufs[nd.id], bf, st);
  std::fill(v.coef, v.coef + 26, 0);
  int64_t off = 0;
  for (size_t d = 0; d < nd.sub.size(); ++d) {
    int s = nd.sub[d];
    if (s >= 0) v.coef[e.in[pos][s]] += st[d];
    else off += (int64_t)(-(s + 1)) * st[d];
  }
  v.ptr = (const char *)bufs[nd.id].ptr + off * esz(bf.dtype);
  v.dtype = bf.dtype;
}

int check_buffers(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                  std::string &err) {
  if (bufs.size() != e.buffers.size()) {
    err = "expected " + std::to_string(e.buffers.size()) + " buffers, got " + std::to_string(bufs.size());
    return EARG;
  }
  for (size_t k = 0; k < bufs.size(); ++k) {
    const Buffer &d = e.buffers[k];
    if (!bufs[k].ptr && !d.shape.empty()) {
      bool empty = false;
      for (auto x : d.shape) empty |= x == 0;
      if (!empty) { err = "buffer " + d.name + " is NULL"; return EARG; }
    }
    if (bufs[k].dtype != d.dtype) { err = "dtype of buffer " + d.name + " differs from its declaration"; return EDTYPE; }
    if (bufs[k].ndim != (int)d.shape.size()) { err = "rank of buffer " + d.name + " differs from its declaration"; return ESHAPE; }
    if (d.dtype != F64 && d.dtype != F32 && d.dtype != F16 && d.dtype != BF16 && d.dtype != I32 &&
        d.dtype != I64 && d.dtype != I8) {
      err = std::string("buffers of dtype ") + dtype_name(d.dtype) + " are not evaluated";
      return EUNSUPPORTED;
    }
  }
  if ((int)outs.size() != e.b) { err = "expected one output per row"; return EARG; }
  for (auto &o : outs) {
    if (o.dtype != e.out_dtype) { err = std::string("output dtype must be ") + dtype_name(e.out_dtype); return EDTYPE; }
    if (o.ndim != (int)e.out.size()) { err = "output rank differs from the notation"; return ESHAPE; }
    if (o.strides) { err = "outputs must be dense row-major (strides = NULL)"; return EARG; }
  }
  if (e.out_dtype != F64 && e.out_dtype != F32) {
    err = "outputs of dtype other than float64 / float32 are not evaluated";
    return EUNSUPPORTED;
  }
  return OK;
}

// ------------------------------------------------------------ generic

// Operands of a fast row that no contracted letter moves are constant over
// the whole sum: they go last (n_hoist of them) and multiply the sum once
// instead of every term (one multiply per term fewer for each).
static void hoist_invariants(GParams &p) {
  if (!p.fast || p.n_ops < 3 || p.n_con == 0) return;
  auto invariant = [&](const GOp &op) {
    for (int c = 0; c < p.n_con; ++c) {
      const int L = p.con_letter[c];
      if (p.len[L] > 1 && op.coef[L] != 0) return false;
    }
    return true;
  };
  GOp run[4], inv[4];
  int nr = 0, ni = 0;
  for (int k = 0; k < p.n_ops; ++k) (invariant(p.ops[k]) ? inv[ni++] : run[nr++]) = p.ops[k];
  if (nr == 0 || ni == 0) return;
  for (int k = 0; k < nr; ++k) p.ops[k] = run[k];
  for (int k = 0; k < ni; ++k) p.ops[nr + k] = inv[k];
  p.n_hoist = ni;
}

// Of the operands left in the sum of a fast row (modes 0-2), those that the
// innermost contracted letter does not move are constant within each run of
// it: they go after the others (n_inv of them) and multiply each run's sum
// once instead of every term (rows with at least three such operands).
static void split_run_invariants(GParams &p) {
  if (!p.fast || p.mode == 3 || p.n_con == 0) return;
  const int L = p.con_letter[p.n_con - 1];
  if (p.len[L] < 2) return;
  const int nr = p.n_ops - p.n_hoist;
  if (nr < 3) return;   // with two operands a term costs one multiply-add either way
  GOp var[4], inv[4];
  int nv = 0, ni = 0;
  for (int k = 0; k < nr; ++k) (p.ops[k].coef[L] == 0 ? inv[ni++] : var[nv++]) = p.ops[k];
  if (nv == 0 || ni == 0) return;
  for (int k = 0; k < nv; ++k) p.ops[k] = var[k];
  for (int k = 0; k < ni; ++k) p.ops[nv + k] = inv[k];
  p.n_inv = ni;
}

// Mode 3: the GEMM view of a fast row with two operands in its sum (plus at
// most one hoisted operand) whose M, N and K extents
// are all large enough to fill its tiles.  Letters within a role run
// outermost first, ordered by decreasing stride, so the fastest-varying
// letter of each role has the smallest stride; each operand is then loaded
// along the role (K or M / N) in which it is contiguous.
static void plan_gemm_view(GParams &p) {
  // two operands in the sum, and at most one hoisted operand (it multiplies
  // each output once, after its sum)
  if (!p.fast || p.n_ops - p.n_hoist != 2 || p.n_hoist > 1) return;
  GGemm g{};
  const int64_t *ca = p.ops[0].coef, *cb = p.ops[1].coef;
  int64_t oc = 1;
  for (int d = p.n_out - 1; d >= 0; --d) {
    g.out_coef[p.out_letter[d]] = oc;
    oc *= p.len[p.out_letter[d]];
  }
  std::vector<int> M, N, K, Bt;
  for (int d = 0; d < p.n_out; ++d) {
    const int L = p.out_letter[d];
    if (cb[L] == 0) M.push_back(L);
    else if (ca[L] == 0) N.push_back(L);
    else Bt.push_back(L);
  }
  for (int c = 0; c < p.n_con; ++c) K.push_back(p.con_letter[c]);
  auto ext = [&](const std::vector<int> &v) {
    int64_t n = 1;
    for (int L : v) n *= p.len[L];
    return n;
  };
  g.M = ext(M), g.N = ext(N), g.K = ext(K), g.B = ext(Bt);
  if (g.M < 32 || g.N < 32 || g.K < 8) return;
  auto by = [&](std::vector<int> &v, auto key) {
    std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return key(x) > key(y); });
  };
  by(M, [&](int L) { return std::abs(ca[L]); });
  by(N, [&](int L) { return std::abs(cb[L]); });
  by(K, [&](int L) { return std::abs(ca[L]) + std::abs(cb[L]); });
  g.nm = (int)M.size(), g.nn = (int)N.size(), g.nk = (int)K.size(), g.nb = (int)Bt.size();
  for (int q = 0; q < g.nm; ++q) g.m[q] = M[q];
  for (int q = 0; q < g.nn; ++q) g.n[q] = N[q];
  for (int q = 0; q < g.nk; ++q) g.k[q] = K[q];
  for (int q = 0; q < g.nb; ++q) g.b[q] = Bt[q];
  // the tile side is a launch choice (every output sums its terms in
  // increasing k whatever the tile): 64 for FP32, 32 for FP64 by default
  set_gemm_tile(g, p.out_dtype == F64 ? 32 : 64);
  const int lk = K.back(), lm = M.back(), ln = N.back();
  g.a_kmajor = std::abs(ca[lk]) < std::abs(ca[lm]);
  g.b_kmajor = std::abs(cb[lk]) < std::abs(cb[ln]);
  p.gemm = g;
  p.mode = 3;
}


int plan_generic_row(const Einsum &e, int row, const std::vector<BufIn> &bufs, const BufIn &out,
                     const std::vector<double> &scalars, GParams &p, std::string &err) {
  std::memset(&p, 0, sizeof(p));
  int compact[26];
  int nl = 0;
  for (int c = 0; c < 26; ++c) compact[c] = e.used[c] ? nl++ : -1;
  if (nl > GMAXL) { err = "more than 16 distinct indices on the generic path"; return EUNSUPPORTED; }
  if (e.n > GMAXOPS) { err = "more than 8 operands on the generic path"; return EUNSUPPORTED; }
  if (scalars.size() > 8) { err = "more than 8 runtime scalars"; return EUNSUPPORTED; }
  p.n_letters = nl;
  p.n_ops = e.n;
  for (int c = 0; c < 26; ++c)
    if (e.used[c]) p.len[compact[c]] = e.len[c];
  p.n_out = (int)e.out.size();
  bool is_out[26] = {false};
  p.total_out = 1;
  for (int d = 0; d < p.n_out; ++d) {
    p.out_letter[d] = compact[e.out[d]];
    is_out[e.out[d]] = true;
    p.total_out *= e.len[e.out[d]];
  }
  p.total_con = 1;
  for (int c = 0; c < 26; ++c)
    if (e.used[c] && !is_out[c]) {
      p.con_letter[p.n_con++] = compact[c];
      p.total_con *= e.len[c];
    }
  p.out = out.ptr;
  p.out_dtype = e.out_dtype;
  // a thread per output for short contractions (under 512 terms when there
  // are at least 32768 outputs, enough threads to fill the GPU, else under
  // 64: a warp's butterfly sum would cost more FP64 adds than its terms), a
  // warp for medium ones and a CTA for long ones, or for medium ones with too
  // few outputs to fill the GPU with warps (each virtual lane still takes at
  // least 8 terms)
  p.mode = (p.total_con < 64 || (p.total_con < 512 && p.total_out >= 32768))
               ? 0
               : ((p.total_con >= 16384 || (p.total_con >= 2048 && p.total_out < 1024)) ? 2 : 1);
  for (size_t k = 0; k < scalars.size(); ++k) p.scalars[k] = scalars[k];
  int n_ins = 0;
  for (int j = 0; j < e.n; ++j) {
    int a = e.rows[row][j];
    GOp &op = p.ops[j];
    View v;
    if (arg_view(e, a, j, bufs, v)) {
      op.kind = 0;
      op.ptr = v.ptr;
      op.dtype = v.dtype;
      for (int c = 0; c < 26; ++c)
        if (compact[c] >= 0) op.coef[compact[c]] = v.coef[c];
      continue;
    }
    // producer program: postfix walk of the lambda body
    const Arg &arg = e.args[a];
    op.kind = 1;
    op.prog_begin = n_ins;
    int depth = 0, max_depth = 0;
    std::vector<std::pair<int, bool>> stack{{arg.root, false}};
    while (!stack.empty()) {
      auto [id, done] = stack.back();
      stack.pop_back();
      const XNode &nd = arg.nodes[id];
      if (!done && nd.op != X_REF) {
        stack.push_back({id, true});
        for (int k = (int)nd.kids.size() - 1; k >= 0; --k) stack.push_back({nd.kids[k], false});
        continue;
      }
      if (n_ins >= GMAXINS) { err = "producer programs longer than 48 instructions"; return EUNSUPPORTED; }
      GIns &in = p.ins[n_ins++];
      in.op = nd.op;
      switch (nd.op) {
        case X_NUM: in.num = nd.num; ++depth; break;
        case X_SCALAR:
          if (nd.id >= (int)scalars.size()) { err = "missing value of scalar $" + e.scalars[nd.id]; return EARG; }
          in.letter = nd.id;
          ++depth;
          break;
        case X_PARAM: in.letter = compact[e.in[j][nd.id]]; ++depth; break;
        case X_REF: {
          View rv;
          ref_view(e, nd, j, bufs, rv);
          in.ptr = rv.ptr;
          in.dtype = rv.dtype;
          for (int c = 0; c < 26; ++c)
            if (compact[c] >= 0) in.coef[compact[c]] = rv.coef[c];
          ++depth;
          break;
        }
        case X_ADD: case X_SUB: case X_MUL: case X_DIV: case X_EQ: case X_NE: --depth; break;
        case X_SELECT: depth -= 2; break;
        default: break;
      }
      max_depth = std::max(max_depth, depth);
    }
    if (max_depth > GSTACK) { err = "producer expression deeper than 8"; return EUNSUPPORTED; }
    op.prog_len = n_ins - op.prog_begin;
    op.dtype = arg.dtype;
  }
  // the running-offset evaluator: plain views of the output's dtype only
  // (the contraction count and each operand's largest offset fit in 32 bits)
  p.fast = p.n_ops >= 1 && p.n_ops <= 4 && p.n_con <= 4 && p.total_con < ((int64_t)1 << 31);
  for (int j = 0; j < p.n_ops; ++j) {
    if (p.ops[j].kind != 0 || p.ops[j].dtype != p.out_dtype) p.fast = 0;
    int64_t span = 0;
    for (int L = 0; L < p.n_letters; ++L) span += std::abs(p.ops[j].coef[L]) * std::max<int64_t>(0, p.len[L] - 1);
    if (span >= ((int64_t)1 << 31)) p.fast = 0;
  }
  hoist_invariants(p);
  plan_gemm_view(p);
  split_run_invariants(p);
  return OK;
}

// ------------------------------------------------------------ element

static int plan_element_stacked(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                                const be_config_t &cfg, EParams &p, std::string &why);

// shared-memory tile: the configured element count, else the default shrunk
// (in steps of 4 elements) until the operator, one group's produced operand
// and the geometric factors fit the budget
static int element_tile(const EParams &p, const be_config_t &cfg, std::string &why) {
  auto bytes = [&](int te) {
    EParams q = p;
    q.tile_e = te;
    return sizeof(double) * element_smem_words(q);
  };
  int te = cfg.tile[0] > 0 ? cfg.tile[0] : (p.NI >= 16 ? 32 : 256);
  if (cfg.tile[2] != 1) te = (te + 3) / 4 * 4;   // the double-float kernel works on groups of 4 elements
  if (cfg.tile[0] <= 0)
    while (te > 4 && bytes(te) > EM_SMEM_BUDGET) te -= 4;
  if (bytes(te) > EM_SMEM_BUDGET) { why = "tile does not fit shared memory"; return 0; }
  return te;
}

static int plan_element_hoisted(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                                const be_config_t &cfg, EParams &p, std::string &why);

// the hoisted form (t = D u shared by the rows) where it applies, else the
// stacked form
int plan_element(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                 const be_config_t &cfg, EParams &p, std::string &why) {
  const int st = plan_element_hoisted(e, bufs, outs, cfg, p, why);
  if (st != EUNSUPPORTED || e.n != 3 || e.out_dtype != F64 || e.out.size() != 2) return st;
  std::string why_s;
  if (plan_element_stacked(e, bufs, outs, cfg, p, why_s) == OK) return OK;
  why += "; stacked form: " + why_s;
  return EUNSUPPORTED;
}

static int plan_element_hoisted(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                                const be_config_t &cfg, EParams &p, std::string &why) {
  std::memset(&p, 0, sizeof(p));
  if (e.out_dtype != F64) { why = "element strategy runs FP64 only"; return EUNSUPPORTED; }
  for (auto &a : e.args)
    if (a.dtype != F64) { why = "element strategy runs FP64 only"; return EUNSUPPORTED; }
  for (auto &b : e.buffers)
    if (b.dtype != F64) { why = "element strategy runs FP64 only"; return EUNSUPPORTED; }
  if (e.out.size() != 2 || (e.n != 2 && e.n != 3)) { why = "notation is not R[e,i] = sum D u (g)"; return EUNSUPPORTED; }
  if (e.b > EM_MAXROWS) { why = "more than 16 rows"; return EUNSUPPORTED; }
  const int le = e.out[0], li = e.out[1];
  // D: the operand without e that holds i
  int pD = -1, pU = -1, pG = -1;
  for (int j = 0; j < e.n; ++j) {
    bool has_e = std::find(e.in[j].begin(), e.in[j].end(), le) != e.in[j].end();
    bool has_i = std::find(e.in[j].begin(), e.in[j].end(), li) != e.in[j].end();
    if (!has_e && has_i) pD = j;
  }
  if (pD < 0) { why = "no shared operator operand"; return EUNSUPPORTED; }
  const auto &dl = e.in[pD];
  if ((e.n == 2 && dl.size() != 2) || (e.n == 3 && dl.size() != 3)) { why = "operator rank"; return EUNSUPPORTED; }
  int lj = -1, lr = -1;
  // identify u (e, j) and g (e, r); when n = 3 both are (e, x) operands
  std::vector<int> ex;
  for (int j = 0; j < e.n; ++j)
    if (j != pD) {
      if (e.in[j].size() != 2 || e.in[j][0] != le || e.in[j][1] == le) { why = "per-element operands must be (e, x)"; return EUNSUPPORTED; }
      ex.push_back(j);
    }
  std::vector<int8_t> others;
  for (int8_t c : dl)
    if (c != li) others.push_back(c);
  if (e.n == 2) {
    pU = ex[0];
    lj = e.in[pU][1];
    if (others.size() != 1 || others[0] != lj) { why = "u does not share j with D"; return EUNSUPPORTED; }
  } else {
    // two letters besides i in D: j (shared with u) and r (shared with g)
    if (others.size() != 2 || others[0] == others[1]) { why = "operator letters"; return EUNSUPPORTED; }
    int8_t x0 = e.in[ex[0]][1], x1 = e.in[ex[1]][1];
    if (x0 == x1) { why = "g and u index the same letter"; return EUNSUPPORTED; }
    // u is the operand with the larger extent (dofs), g the smaller one (dimension r)
    if (e.len[x0] >= e.len[x1]) { pU = ex[0]; pG = ex[1]; } else { pU = ex[1]; pG = ex[0]; }
    lj = e.in[pU][1];
    lr = e.in[pG][1];
    if (!((others[0] == lj && others[1] == lr) || (others[0] == lr && others[1] == lj))) { why = "operator letters"; return EUNSUPPORTED; }
  }
  p.NI = (int)e.len[li];
  p.NJ = (int)e.len[lj];
  p.R = lr >= 0 ? (int)e.len[lr] : 1;
  p.has_g = pG >= 0;
  p.E = e.len[le];
  if (p.NI > EM_MAXN || p.NJ > EM_MAXN || p.R > EM_MAXR || p.NI < 1 || p.NJ < 1) { why = "operator extents beyond 64 x 64 x 4"; return EUNSUPPORTED; }
  // D shared by every row
  int dArg = e.rows[0][pD];
  for (int i = 0; i < e.b; ++i)
    if (e.rows[i][pD] != dArg) { why = "operator differs between rows"; return EUNSUPPORTED; }
  View dv;
  if (!arg_view(e, dArg, pD, bufs, dv)) { why = "operator is not a plain view"; return EUNSUPPORTED; }
  p.D = (const double *)dv.ptr;
  p.si = dv.coef[li];
  p.sj = dv.coef[lj];
  p.sr = lr >= 0 ? dv.coef[lr] : 0;
  // per-row producers and geometric factors
  std::vector<int> uargs;
  p.n_rows = e.b;
  for (int i = 0; i < e.b; ++i) {
    int ua = e.rows[i][pU];
    int g = -1;
    for (size_t k = 0; k < uargs.size(); ++k)
      if (uargs[k] == ua) g = (int)k;
    if (g < 0) {
      EProd q;
      std::memset(&q, 0, sizeof(q));
      View v;
      if (arg_view(e, ua, pU, bufs, v)) {
        q.kind = 0;
        q.a = EView{(const double *)v.ptr, v.coef[le], v.coef[lj]};
      } else {
        const Arg &A = e.args[ua];
        const XNode &rt = A.nodes[A.root];
        int sin_kid = -1, ref_kid = -1;
        bool both_ref = false;
        if (rt.op == X_MUL && rt.kids.size() == 2) {
          both_ref = A.nodes[rt.kids[0]].op == X_REF && A.nodes[rt.kids[1]].op == X_REF;
          for (int k = 0; k < 2; ++k) {
            const XNode &kd = A.nodes[rt.kids[k]];
            if (kd.op == X_SIN && A.nodes[kd.kids[0]].op == X_REF) sin_kid = k;
            else if (kd.op == X_REF) ref_kid = k;
          }
        }
        View va, vb;
        if (both_ref) {
          ref_view(e, A.nodes[rt.kids[0]], pU, bufs, va);
          ref_view(e, A.nodes[rt.kids[1]], pU, bufs, vb);
          q.kind = 2;
        } else {
          if (sin_kid < 0 || ref_kid < 0 || sin_kid == ref_kid) { why = "producer is not a view, a*b or sin(a)*b"; return EUNSUPPORTED; }
          ref_view(e, A.nodes[A.nodes[rt.kids[sin_kid]].kids[0]], pU, bufs, va);
          ref_view(e, A.nodes[rt.kids[ref_kid]], pU, bufs, vb);
          q.kind = 1;
        }
        if (va.dtype != F64 || vb.dtype != F64) { why = "producer operands must be float64"; return EUNSUPPORTED; }
        q.a = EView{(const double *)va.ptr, va.coef[le], va.coef[lj]};
        q.b = EView{(const double *)vb.ptr, vb.coef[le], vb.coef[lj]};
      }
      uargs.push_back(ua);
      g = (int)uargs.size() - 1;
      p.groups[g] = q;
    }
    p.rows[i].group = g;
    p.rows[i].out = (double *)outs[i].ptr;
    if (pG >= 0) {
      View gv;
      if (!arg_view(e, e.rows[i][pG], pG, bufs, gv)) { why = "geometric factor is not a plain view"; return EUNSUPPORTED; }
      p.rows[i].g = EView{(const double *)gv.ptr, gv.coef[le], gv.coef[lr]};
    }
  }
  p.n_groups = (int)uargs.size();
  p.tile_e = element_tile(p, cfg, why);
  return p.tile_e > 0 ? OK : EUNSUPPORTED;
}

// Stacked form of the element strategy: three operands D (without e), A and
// B (with e) such that R[e, i] = sum_k D[i, k] v[e, k], k running over the
// one or two letters of D besides i (j, and s when present), with
//     v[e, s, j] = sum_x A[e, x, s, j] * B[e, x, s, j],
// where x is at most one letter shared by A and B only and each operand
// holds any subset of s and j.  The DG local divergence 'xre,rij,xej->ei'
// (v = sum_x J[x, r, e] F[x, e, j]) and the face mass 'fe,ifj,fej->ei'
// (v = J[f, e] U[f, e, j]) have this form (Sec. "Batched einsums in DG-FEM
// Operators", divergence and face-mass tuples).  A functional operand
// whose body selects on x (F(x, e, j) := x == 0 ? u : ...) is resolved to
// one view per value of x.

// body node of functional argument A with parameter px fixed to xv: selects
// whose condition compares that parameter with a number are resolved; -1
// when a condition is anything else
static int resolve_select(const Arg &A, int node, int px, int64_t xv) {
  while (node >= 0 && A.nodes[node].op == X_SELECT) {
    const XNode &sel = A.nodes[node];
    const XNode &c = A.nodes[sel.kids[0]];
    if (c.op != X_EQ && c.op != X_NE) return -1;
    const XNode &l = A.nodes[c.kids[0]], &r = A.nodes[c.kids[1]];
    double num;
    if (l.op == X_PARAM && l.id == px && r.op == X_NUM) num = r.num;
    else if (r.op == X_PARAM && r.id == px && l.op == X_NUM) num = l.num;
    else return -1;
    const bool eq = (double)xv == num;
    node = (c.op == X_EQ ? eq : !eq) ? sel.kids[1] : sel.kids[2];
  }
  return node;
}

// the view of operand position pos (argument arg) over (e, s, j) with the
// letter lx (if any) fixed to xv
static bool stacked_view(const Einsum &e, int arg, int pos, int lx, int64_t xv, const std::vector<BufIn> &bufs, int le,
                         int ls, int lj, ESView &out) {
  const Arg &A = e.args[arg];
  View v;
  if (!A.functional()) {
    arg_view(e, arg, pos, bufs, v);
  } else {
    int px = -1;
    for (size_t d = 0; d < e.in[pos].size(); ++d)
      if (lx >= 0 && e.in[pos][d] == lx) px = (int)d;
    const int nd = px >= 0 ? resolve_select(A, A.root, px, xv) : A.root;
    if (nd < 0 || A.nodes[nd].op != X_REF) return false;
    ref_view(e, A.nodes[nd], pos, bufs, v);
  }
  if (v.dtype != F64) return false;
  out.ptr = (const double *)v.ptr + (lx >= 0 ? v.coef[lx] * xv : 0);
  out.se = v.coef[le];
  out.ss = ls >= 0 ? v.coef[ls] : 0;
  out.sj = v.coef[lj];
  return true;
}

static int plan_element_stacked(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                                const be_config_t &cfg, EParams &p, std::string &why) {
  std::memset(&p, 0, sizeof(p));
  for (auto &a : e.args)
    if (a.dtype != F64) { why = "element strategy runs FP64 only"; return EUNSUPPORTED; }
  for (auto &b : e.buffers)
    if (b.dtype != F64) { why = "element strategy runs FP64 only"; return EUNSUPPORTED; }
  if (e.b > EM_MAXROWS) { why = "more than 16 rows"; return EUNSUPPORTED; }
  const int le = e.out[0], li = e.out[1];
  auto has = [&](int pos, int c) { return std::find(e.in[pos].begin(), e.in[pos].end(), c) != e.in[pos].end(); };
  int pD = -1;
  std::vector<int> pe;
  for (int j = 0; j < 3; ++j) {
    if (!has(j, le) && has(j, li)) pD = j;
    else if (has(j, le) && !has(j, li)) pe.push_back(j);
  }
  if (pD < 0 || pe.size() != 2) { why = "not D[i, ..] with two per-element operands"; return EUNSUPPORTED; }
  const int pA = pe[0], pB = pe[1];
  for (int j = 0; j < 3; ++j)
    for (size_t a = 0; a < e.in[j].size(); ++a)
      for (size_t b = a + 1; b < e.in[j].size(); ++b)
        if (e.in[j][a] == e.in[j][b]) { why = "repeated letter in an operand"; return EUNSUPPORTED; }
  std::vector<int8_t> dl;
  for (int8_t c : e.in[pD])
    if (c != li) dl.push_back(c);
  if (dl.empty() || dl.size() > 2) { why = "operator rank"; return EUNSUPPORTED; }
  int lx = -1;
  for (int8_t c : e.in[pA])
    if (c != le && has(pB, c) && !has(pD, c)) {
      if (lx >= 0) { why = "more than one stacking letter"; return EUNSUPPORTED; }
      lx = c;
    }
  for (int pos : {pA, pB})
    for (int8_t c : e.in[pos])
      if (c != le && c != lx && !has(pD, c)) { why = "letter summed outside the operator"; return EUNSUPPORTED; }
  for (int8_t c : dl)
    if (!has(pA, c) && !has(pB, c)) { why = "operator letter not in the per-element operands"; return EUNSUPPORTED; }
  int lj = dl[0], ls = -1;
  if (dl.size() == 2) {
    lj = e.len[dl[0]] >= e.len[dl[1]] ? dl[0] : dl[1];
    ls = lj == dl[0] ? dl[1] : dl[0];
  }
  const int X = lx >= 0 ? (int)e.len[lx] : 1;
  const int64_t S = ls >= 0 ? e.len[ls] : 1, NJ0 = e.len[lj];
  if (X < 1 || X > EM_MAXX) { why = "stacking extent beyond 4"; return EUNSUPPORTED; }
  if (e.len[li] < 1 || e.len[li] > EM_MAXN || NJ0 < 1 || S < 1 || S * NJ0 > EM_MAXK) {
    why = "operator extents beyond 64 x 128";
    return EUNSUPPORTED;
  }
  const int dArg = e.rows[0][pD];
  for (int i = 0; i < e.b; ++i)
    if (e.rows[i][pD] != dArg) { why = "operator differs between rows"; return EUNSUPPORTED; }
  View dv;
  if (!arg_view(e, dArg, pD, bufs, dv)) { why = "operator is not a plain view"; return EUNSUPPORTED; }
  p.D = (const double *)dv.ptr;
  p.si = dv.coef[li];
  p.sj = dv.coef[lj];
  p.sr = ls >= 0 ? dv.coef[ls] : 0;
  p.NI = (int)e.len[li];
  p.NJ0 = (int)NJ0;
  p.NJ = (int)(S * NJ0);
  p.R = 1;
  p.has_g = 0;
  p.E = e.len[le];
  p.n_rows = e.b;
  std::vector<std::pair<int, int>> keys;
  for (int i = 0; i < e.b; ++i) {
    const std::pair<int, int> key(e.rows[i][pA], e.rows[i][pB]);
    int g = -1;
    for (size_t k = 0; k < keys.size(); ++k)
      if (keys[k] == key) g = (int)k;
    if (g < 0) {
      EProd &q = p.groups[keys.size()];
      q.kind = 3;
      q.X = X;
      for (int x = 0; x < X; ++x)
        if (!stacked_view(e, key.first, pA, lx, x, bufs, le, ls, lj, q.A[x]) ||
            !stacked_view(e, key.second, pB, lx, x, bufs, le, ls, lj, q.B[x])) {
          why = "per-element operand is not a view or a select of views over the stacking letter";
          return EUNSUPPORTED;
        }
      keys.push_back(key);
      g = (int)keys.size() - 1;
    }
    p.rows[i].group = g;
    p.rows[i].out = (double *)outs[i].ptr;
  }
  p.n_groups = (int)keys.size();
  p.tile_e = element_tile(p, cfg, why);
  return p.tile_e > 0 ? OK : EUNSUPPORTED;
}

}  // namespace be

// ------------------------------------------------------------ dense split

namespace be {

// stride of the flattened letters ls (row-major over ls) in a view, or -1
static int64_t flat_stride(const Einsum &e, const View &v, const std::vector<int8_t> &ls) {
  if (ls.empty()) return 0;
  int64_t st = v.coef[ls.back()];
  int64_t expect = st;
  for (int k = (int)ls.size() - 1; k >= 0; --k) {
    if (v.coef[ls[k]] != expect) return -1;
    expect *= e.len[ls[k]];
  }
  return st;
}

// A functional body that is affine in a single buffer reference,
// f(x) = alpha * x + beta, with alpha and beta built from numbers and runtime
// scalars by + - * and division by a constant (the producers
// (alpha_1 A + beta_1)(alpha_2 B + beta_2) of Sec. "Evaluation", TCCG
// experiment).  ref receives the reference node; false for anything else.
static bool affine_of(const Arg &A, int node, const std::vector<double> *sc, double &alpha, double &beta, int &ref) {
  const XNode &n = A.nodes[node];
  switch (n.op) {
    case X_NUM: alpha = 0.0; beta = n.num; return true;
    case X_SCALAR:
      alpha = 0.0;
      beta = sc ? (n.id < (int)sc->size() ? (*sc)[n.id] : 0.0) : 1.0;
      return true;
    case X_REF:
      if (ref >= 0) return false;               // a second reference
      ref = node;
      alpha = 1.0;
      beta = 0.0;
      return true;
    case X_NEG: {
      if (!affine_of(A, n.kids[0], sc, alpha, beta, ref)) return false;
      alpha = -alpha;
      beta = -beta;
      return true;
    }
    case X_ADD: case X_SUB: case X_MUL: case X_DIV: {
      double a0, b0, a1, b1;
      const int r0 = ref;
      if (!affine_of(A, n.kids[0], sc, a0, b0, ref)) return false;
      const bool left_ref = ref != r0;
      const int r1 = ref;
      if (!affine_of(A, n.kids[1], sc, a1, b1, ref)) return false;
      const bool right_ref = ref != r1;
      if (n.op == X_ADD) { alpha = a0 + a1; beta = b0 + b1; return true; }
      if (n.op == X_SUB) { alpha = a0 - a1; beta = b0 - b1; return true; }
      if (n.op == X_MUL) {
        if (left_ref && right_ref) return false;
        if (right_ref) { alpha = b0 * a1; beta = b0 * b1; }
        else { alpha = a0 * b1; beta = b0 * b1; }
        return true;
      }
      if (right_ref) return false;              // division by the reference
      if (sc && b1 == 0.0) return false;
      const double d = sc ? b1 : 1.0;
      alpha = a0 / d;
      beta = b0 / d;
      return true;
    }
    default: return false;
  }
}

// view of operand position pos of argument arg, directly or through an
// affine producer (coefficients in alpha, beta)
static bool dense_operand(const Einsum &e, int arg, int pos, const std::vector<BufIn> &bufs,
                          const std::vector<double> *sc, View &v, double &alpha, double &beta) {
  alpha = 1.0;
  beta = 0.0;
  if (arg_view(e, arg, pos, bufs, v)) return true;
  const Arg &A = e.args[arg];
  int ref = -1;
  if (!affine_of(A, A.root, sc, alpha, beta, ref) || ref < 0) return false;
  ref_view(e, A.nodes[ref], pos, bufs, v);
  return v.dtype == F64;
}

int plan_dense(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs, DensePlan &p,
               std::string &why, const std::vector<double> *scalars) {
  p = DensePlan();
  if (e.n != 2) { why = "dense strategy needs two operands"; return EUNSUPPORTED; }
  if (e.out_dtype != F64) { why = "dense strategy evaluates float64"; return EUNSUPPORTED; }
  for (auto &a : e.args)
    if (a.dtype != F64) { why = "dense strategy evaluates float64"; return EUNSUPPORTED; }
  bool in0[26] = {false}, in1[26] = {false}, is_out[26] = {false};
  for (int j = 0; j < 2; ++j) {
    bool seen[26] = {false};
    for (int8_t c : e.in[j]) {
      if (seen[c]) { why = "repeated index inside an operand"; return EUNSUPPORTED; }
      seen[c] = true;
      (j ? in1 : in0)[c] = true;
    }
  }
  for (int8_t c : e.out) is_out[c] = true;
  // output = M letters (from the A operand) then N letters (from the B
  // operand); A is operand 0 when the output starts with operand 0's free
  // letters, else operand 1 (C = A B either way, with the roles swapped)
  for (int8_t c : e.out)
    if (in0[c] && in1[c]) { why = "batch index shared by both operands and the output"; return EUNSUPPORTED; }
  const int opA = (!e.out.empty() && !in0[e.out[0]]) ? 1 : 0, opB = 1 - opA;
  const bool *inA = opA ? in1 : in0, *inB = opA ? in0 : in1;
  std::vector<int8_t> Ml, Nl, Kl;
  for (int8_t c : e.out) (inA[c] ? Ml : Nl).push_back(c);
  for (size_t k = 0; k < e.out.size(); ++k)
    if (k < Ml.size() ? e.out[k] != Ml[k] : e.out[k] != Nl[k - Ml.size()]) {
      why = "output letters are not (free letters of one operand, free letters of the other)";
      return EUNSUPPORTED;
    }
  for (int8_t c : e.in[opA])
    if (!is_out[c]) {
      if (!inB[c]) { why = "index summed inside one operand"; return EUNSUPPORTED; }
      Kl.push_back(c);
    }
  for (int8_t c : e.in[opB])
    if (!is_out[c] && !inA[c]) { why = "index summed inside one operand"; return EUNSUPPORTED; }
  p.M = 1;
  for (auto c : Ml) p.M *= e.len[c];
  p.N = 1;
  for (auto c : Nl) p.N *= e.len[c];
  p.K = 1;
  for (auto c : Kl) p.K *= e.len[c];
  p.rows.clear();
  for (int i = 0; i < e.b; ++i) {
    View va, vb;
    DenseRow r;
    if (!dense_operand(e, e.rows[i][opA], opA, bufs, scalars, va, r.alA, r.beA) ||
        !dense_operand(e, e.rows[i][opB], opB, bufs, scalars, vb, r.alB, r.beB)) {
      why = "dense operands must be views or affine producers of one view";
      return EUNSUPPORTED;
    }
    r.argA = e.rows[i][opA];
    r.argB = e.rows[i][opB];
    r.A = (const double *)va.ptr;
    r.B = (const double *)vb.ptr;
    r.lda = flat_stride(e, va, Ml);
    r.ska = flat_stride(e, va, Kl);
    r.ldb = flat_stride(e, vb, Kl);
    r.snb = flat_stride(e, vb, Nl);
    if (r.lda < 0 || r.ska < 0 || r.ldb < 0 || r.snb < 0) {
      why = "operand letters cannot be flattened to a matrix";
      return EUNSUPPORTED;
    }
    r.C = (double *)outs[i].ptr;
    p.rows.push_back(r);
  }
  return OK;
}


// ------------------------------------------------------------ factored rows
//
// Eq. (1) sums the product of a row's n operands over the contracted
// letters as one loop nest.  Summing some contracted letters inside a pair
// of operands first (an intermediate over the letters still needed) gives
// the same sum with the terms grouped differently -- each pairwise step is
// itself a two-operand einsum -- and, for notations such as the triple
// product 'ik,kl,lj->ij' or Fig. 1's 'mnj,mni,kli->ijkl', far fewer
// multiply-adds than the full nest.  The order is chosen per notation and
// lengths; every step runs on the generic evaluator (as GEMM tiles when
// its form allows).

namespace {

double letters_volume(const Einsum &e, uint32_t mask) {
  double v = 1.0;
  for (int c = 0; c < 26; ++c)
    if (mask >> c & 1u) v *= (double)e.len[c];
  return v;
}

uint32_t mask_of(const std::vector<int8_t> &ls) {
  uint32_t m = 0;
  for (int8_t c : ls) m |= 1u << c;
  return m;
}

// exhaustive search over pairwise orders: slots holds the letter masks of
// the operands still to combine, path the steps taken so far
void search_orders(const Einsum &e, uint32_t out_mask, std::vector<uint32_t> &slots, std::vector<int> &ids,
                   int next_id, double cost, std::vector<std::array<int, 2>> &path, std::vector<uint32_t> &kept,
                   double &best, std::vector<std::array<int, 2>> &best_path, std::vector<uint32_t> &best_kept) {
  if (slots.size() == 1) {
    if (cost < best) {
      best = cost;
      best_path = path;
      best_kept = kept;
    }
    return;
  }
  // a unary step: an operand with letters that no other operand and not the
  // output uses sums them first (e.g. both sides of 'ij,ik->i')
  for (size_t a = 0; a < slots.size(); ++a) {
    uint32_t rest = out_mask;
    for (size_t k = 0; k < slots.size(); ++k)
      if (k != a) rest |= slots[k];
    const uint32_t keep = slots[a] & rest;
    if (keep == slots[a]) continue;
    const double c = cost + letters_volume(e, slots[a]);
    if (c >= best) continue;
    std::vector<uint32_t> ns = slots;
    std::vector<int> nid = ids;
    ns[a] = keep;
    nid[a] = next_id;
    path.push_back({ids[a], -1});
    kept.push_back(keep);
    search_orders(e, out_mask, ns, nid, next_id + 1, c, path, kept, best, best_path, best_kept);
    path.pop_back();
    kept.pop_back();
  }
  for (size_t a = 0; a < slots.size(); ++a)
    for (size_t b2 = a + 1; b2 < slots.size(); ++b2) {
      uint32_t rest = out_mask;
      for (size_t k = 0; k < slots.size(); ++k)
        if (k != a && k != b2) rest |= slots[k];
      const uint32_t both = slots[a] | slots[b2];
      const double c = cost + letters_volume(e, both);
      if (c >= best) continue;
      const uint32_t keep = both & rest;
      std::vector<uint32_t> ns;
      std::vector<int> nid;
      for (size_t k = 0; k < slots.size(); ++k)
        if (k != a && k != b2) {
          ns.push_back(slots[k]);
          nid.push_back(ids[k]);
        }
      ns.push_back(keep);
      nid.push_back(next_id);
      path.push_back({ids[a], ids[b2]});
      kept.push_back(keep);
      search_orders(e, out_mask, ns, nid, next_id + 1, c, path, kept, best, best_path, best_kept);
      path.pop_back();
      kept.pop_back();
    }
}

}  // namespace

bool factor_order(const Einsum &e, double min_gain, FactorOrder &fo) {
  if (e.n < 2 || e.n > 5) return false;
  uint32_t all = mask_of(e.out);
  std::vector<uint32_t> slots;
  std::vector<int> ids;
  for (int j = 0; j < e.n; ++j) {
    slots.push_back(mask_of(e.in[j]));
    ids.push_back(j);
    all |= slots.back();
  }
  fo.direct = letters_volume(e, all) * (double)(e.n - 1);
  double best = fo.direct / min_gain;
  std::vector<std::array<int, 2>> path, best_path;
  std::vector<uint32_t> kept, best_kept;
  search_orders(e, mask_of(e.out), slots, ids, e.n, 0.0, path, kept, best, best_path, best_kept);
  if (best_path.empty()) return false;
  fo.factored = best;
  fo.steps = best_path;
  fo.letters.clear();
  fo.inter_elems = 0;
  for (size_t s = 0; s < best_kept.size(); ++s) {
    std::vector<int8_t> ls;
    if (s + 1 == best_kept.size()) {
      ls = e.out;   // the last step writes the output, in its letter order
    } else {
      for (int c = 0; c < 26; ++c)
        if (best_kept[s] >> c & 1u) ls.push_back((int8_t)c);
      fo.inter_elems += (int64_t)letters_volume(e, best_kept[s]);
    }
    fo.letters.push_back(ls);
  }
  return true;
}

bool operand_fop(const Einsum &e, int row, int pos, const std::vector<BufIn> &bufs, FOp &f) {
  View v;
  if (!arg_view(e, e.rows[row][pos], pos, bufs, v)) return false;
  // the view's coefficients by letter; a letter repeated within the operand
  // (a diagonal) already carries the sum of its strides
  f.ptr = v.ptr;
  f.dtype = v.dtype;
  f.letters.clear();
  f.strides.clear();
  bool seen[26] = {false};
  for (int8_t c : e.in[pos]) {
    if (seen[c]) continue;
    seen[c] = true;
    f.letters.push_back(c);
    f.strides.push_back(v.coef[c]);
  }
  return true;
}

// a pairwise (or unary) step as a batched einsum of one row and one or two
// identity arguments X, Y over the operands' views, with a dense row-major
// output over out_letters
static void step_einsum(const Einsum &e, const FOp &x, const FOp *y, const std::vector<int8_t> &out_letters,
                        void *out, Einsum &s, std::vector<BufIn> &bufs, BufIn &bo) {
  // the step as a batched einsum of one row and one or two identity
  // arguments (one: a unary step summing the operand's own letters)
  const int n = y ? 2 : 1;
  s.b = 1;
  s.n = n;
  s.out = out_letters;
  s.in = {x.letters};
  s.rows = {{0}};
  if (y) {
    s.in.push_back(y->letters);
    s.rows[0].push_back(1);
  }
  for (int c = 0; c < 26; ++c) s.len[c] = e.len[c];
  for (int j = 0; j < n; ++j)
    for (int8_t c : s.in[j]) s.used[c] = true;
  for (int8_t c : out_letters) s.used[c] = true;
  s.out_dtype = e.out_dtype;
  const FOp *ops[2] = {&x, y};
  for (int k = 0; k < n; ++k) {
    Buffer bf;
    bf.name = k ? "Y" : "X";
    bf.dtype = ops[k]->dtype;
    for (int8_t c : ops[k]->letters) bf.shape.push_back(e.len[c]);
    s.buffers.push_back(bf);
    Arg a;
    a.name = bf.name;
    a.dtype = bf.dtype;
    a.shape = bf.shape;
    a.buffer = k;
    s.args.push_back(a);
    bufs.push_back(BufIn{const_cast<void *>(ops[k]->ptr), ops[k]->strides.data(), (int32_t)ops[k]->letters.size(),
                         ops[k]->dtype});
  }
  bo = BufIn{out, nullptr, (int32_t)out_letters.size(), e.out_dtype};
}

int plan_factor_step(const Einsum &e, const FOp &x, const FOp *y, const std::vector<int8_t> &out_letters, void *out,
                     GParams &p, std::string &err) {
  Einsum s;
  std::vector<BufIn> bufs;
  BufIn bo;
  step_einsum(e, x, y, out_letters, out, s, bufs, bo);
  return plan_generic_row(s, 0, bufs, bo, {}, p, err);
}

int plan_factor_step_dense(const Einsum &e, const FOp &x, const FOp &y, const std::vector<int8_t> &out_letters,
                           void *out, DensePlan &dp, std::string &why) {
  Einsum s;
  std::vector<BufIn> bufs;
  BufIn bo;
  step_einsum(e, x, &y, out_letters, out, s, bufs, bo);
  return plan_dense(s, bufs, {bo}, dp, why, nullptr);
}

}  // namespace be
