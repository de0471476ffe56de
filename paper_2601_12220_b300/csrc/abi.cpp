// C ABI of the engine (include/be.h): handles, error reporting, the
// tuning database keyed by the normal form, Alg. 2 (identify a reference
// einsum in a target's names) and strategy dispatch for be_execute.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <memory>
#include <mutex>
#include <algorithm>
#include <cmath>
#include <sstream>
#include <tuple>
#include <unordered_map>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "dense.hpp"
#include "launch_rec.hpp"
#include "handles.hpp"
#include "raise.hpp"

using namespace be;

static thread_local std::string g_err;

// NVTX range around one host step (parse, canonicalize, lookup, execute): a
// no-op unless a profiler that collects NVTX ranges is attached
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

namespace be {
// lets the other translation units of the library report through be_last_error()
void set_last_error(const std::string &msg) { g_err = msg; }
// the calling thread's launch recorder (launch_rec.hpp)
LaunchRecorder *&launch_recorder() {
  static thread_local LaunchRecorder *r = nullptr;
  return r;
}
}  // namespace be

static int ensure_status(be_ctx *x) {
  if (x->status) return BE_OK;
  cudaError_t ce = cudaMalloc(&x->status, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemset(x->status, 0, sizeof(int));
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("status word: ") + cudaGetErrorString(ce));
  return BE_OK;
}

static int ensure_ws(be_ctx *x, size_t need) {
  if (x->ws_size >= need) return BE_OK;
  if (x->ws) {
    cudaDeviceSynchronize();
    cudaFree(x->ws);
    x->ws = nullptr;
    x->ws_size = 0;
  }
  cudaError_t ce = cudaMalloc(&x->ws, need);
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("workspace (") + std::to_string(need) + " B): " + cudaGetErrorString(ce));
  x->ws_size = need;
  return BE_OK;
}

static std::string db_key(const std::string &nf, const std::string &dev, int prec) {
  return nf + "\t" + dev + "\t" + std::to_string(prec);
}

static int put_string(const std::string &s, char *buf, size_t len, size_t *needed) {
  if (needed) *needed = s.size() + 1;
  if (!buf || len < s.size() + 1) return fail(BE_EARG, "buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return BE_OK;
}

const Canon *be::canon_cached(be_einsum *e, std::string &err, int &st) {
  std::lock_guard<std::mutex> g(e->mu);
  if (!e->canon) {
    auto c = std::make_unique<Canon>();
    st = canonicalize(e->e, *c, err);
    if (st) return nullptr;
    e->canon = std::move(c);
  }
  st = BE_OK;
  return e->canon.get();
}

extern "C" {

int be_version(void) { return 10000; }

const char *be_last_error(void) { return g_err.c_str(); }

int be_parse(const char *text, be_einsum **out) {
  NvtxRange nv("be_parse");
  if (!text || !out) return fail(BE_EARG, "NULL argument");
  auto h = std::make_unique<be_einsum>();
  std::string err;
  int st = parse(text, h->e, err);
  if (st) return fail(st, err);
  *out = h.release();
  return BE_OK;
}

void be_free_einsum(be_einsum *e) { delete e; }

int be_raise(const char *kernel, be_einsum **out) {
  if (!kernel || !out) return fail(BE_EARG, "NULL argument");
  Raised r;
  std::string err;
  int st = raise_kernel(kernel, r, err);
  if (st) return fail(st, "raise: " + err);
  auto h = std::make_unique<be_einsum>();
  st = parse(r.spec, h->e, err);
  if (st) return fail(st, "raised einsum '" + r.spec + "': " + err);
  h->raised_spec = r.spec;
  h->loop_names = r.loop_names;
  h->outputs = r.outputs;
  *out = h.release();
  return BE_OK;
}

int be_raised_name(const be_einsum *h, int32_t kind, int32_t k, char *buf, size_t len, size_t *needed) {
  if (!h) return fail(BE_EARG, "NULL einsum");
  if (h->raised_spec.empty()) return fail(BE_ENOTFOUND, "einsum was not raised from a kernel");
  std::string s;
  if (kind == BE_RAISED_SPEC) {
    s = h->raised_spec;
  } else if (kind == BE_RAISED_LOOP) {
    if (k < 0 || k >= (int32_t)h->loop_names.size()) return fail(BE_ENOTFOUND, "no such index letter");
    s = h->loop_names[k];
  } else if (kind == BE_RAISED_OUTPUT) {
    if (k < 0 || k >= (int32_t)h->outputs.size()) return fail(BE_ENOTFOUND, "no such row");
    s = h->outputs[k];
  } else {
    return fail(BE_EARG, "unknown kind");
  }
  if (needed) *needed = s.size() + 1;
  if (buf && len > 0) {
    const size_t n = std::min(len - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return BE_OK;
}

int be_einsum_info(const be_einsum *h, int32_t *b, int32_t *n, int32_t *n_buffers, int32_t *n_args,
                   int32_t *n_scalars, int32_t *out_ndim, int32_t *out_dtype) {
  if (!h) return fail(BE_EARG, "NULL einsum");
  const Einsum &e = h->e;
  if (b) *b = e.b;
  if (n) *n = e.n;
  if (n_buffers) *n_buffers = (int32_t)e.buffers.size();
  if (n_args) *n_args = (int32_t)e.args.size();
  if (n_scalars) *n_scalars = (int32_t)e.scalars.size();
  if (out_ndim) *out_ndim = (int32_t)e.out.size();
  if (out_dtype) *out_dtype = e.out_dtype;
  return BE_OK;
}

int be_einsum_out_shape(const be_einsum *h, int64_t *shape) {
  if (!h || !shape) return fail(BE_EARG, "NULL argument");
  auto s = h->e.out_shape();
  for (size_t k = 0; k < s.size(); ++k) shape[k] = s[k];
  return BE_OK;
}

int be_einsum_buffer(const be_einsum *h, int32_t k, char *name, size_t len, size_t *needed, int32_t *dtype,
                     int32_t *ndim, int64_t *shape) {
  if (!h) return fail(BE_EARG, "NULL einsum");
  if (k < 0 || k >= (int)h->e.buffers.size()) return fail(BE_EARG, "buffer index out of range");
  const Buffer &bf = h->e.buffers[k];
  if (dtype) *dtype = bf.dtype;
  if (ndim) *ndim = (int32_t)bf.shape.size();
  if (shape)
    for (size_t d = 0; d < bf.shape.size(); ++d) shape[d] = bf.shape[d];
  if (name || needed) return put_string(bf.name, name, len, needed);
  return BE_OK;
}

int be_canonicalize(const be_einsum *h, be_canon **out) {
  NvtxRange nv("be_canonicalize");
  if (!h || !out) return fail(BE_EARG, "NULL argument");
  auto c = std::make_unique<be_canon>();
  std::string err;
  int st = canonicalize(h->e, c->c, err);
  if (st) return fail(st, err);
  *out = c.release();
  return BE_OK;
}

void be_free_canon(be_canon *c) { delete c; }

int be_canon_key(const be_canon *c, char *buf, size_t len, size_t *needed) {
  if (!c) return fail(BE_EARG, "NULL canon");
  return put_string(c->c.key, buf, len, needed);
}

int be_canon_sigma(const be_canon *c, int32_t kind, int32_t id, char *user, size_t len, size_t *needed) {
  if (!c) return fail(BE_EARG, "NULL canon");
  const Canon &k = c->c;
  std::string s;
  switch (kind) {
    case BE_SIGMA_INDEX:
      if (id < 0 || id >= (int)k.sigma_index.size()) return fail(BE_EARG, "index id out of range");
      s = std::string(1, char('a' + k.sigma_index[id]));
      break;
    case BE_SIGMA_ARG:
      if (id < 0 || id >= (int)k.sigma_arg_name.size()) return fail(BE_EARG, "argument id out of range");
      s = k.sigma_arg_name[id];
      break;
    case BE_SIGMA_ROW:
      if (id < 0 || id >= (int)k.sigma_row.size()) return fail(BE_EARG, "row out of range");
      s = std::to_string(k.sigma_row[id]);
      break;
    case BE_SIGMA_POS:
      if (id < 0 || id >= (int)k.sigma_pos.size()) return fail(BE_EARG, "position out of range");
      s = std::to_string(k.sigma_pos[id]);
      break;
    default:
      return fail(BE_EARG, "unknown sigma kind");
  }
  return put_string(s, user, len, needed);
}

int be_canon_tokens(const be_canon *c, int64_t *tokens, size_t cap, size_t *n_tokens) {
  if (!c) return fail(BE_EARG, "NULL canon");
  const auto &t = c->c.tokens;
  if (n_tokens) *n_tokens = t.size();
  if (!tokens || cap < t.size()) return fail(BE_EARG, "buffer too small");
  for (size_t k = 0; k < t.size(); ++k) tokens[k] = t[k];
  return BE_OK;
}

int be_induced_graph(const be_einsum *h, int32_t *n_nodes, int32_t *colors, int32_t cap_nodes, int32_t *edges,
                     int64_t cap_edges, int64_t *n_edges) {
  if (!h) return fail(BE_EARG, "NULL einsum");
  Graph g = to_induced_graph(h->e);
  if (n_nodes) *n_nodes = g.n;
  if (n_edges) *n_edges = (int64_t)g.edges.size();
  if (colors) {
    if (cap_nodes < g.n) return fail(BE_EARG, "colors buffer too small");
    for (int v = 0; v < g.n; ++v) colors[v] = g.color[v];
  }
  if (edges) {
    if (cap_edges < (int64_t)g.edges.size()) return fail(BE_EARG, "edges buffer too small");
    for (size_t k = 0; k < g.edges.size(); ++k) {
      edges[2 * k] = g.edges[k].first;
      edges[2 * k + 1] = g.edges[k].second;
    }
  }
  return BE_OK;
}

int be_graph_check(int32_t n_nodes, const int32_t *colors, const int32_t *edges, int64_t n_edges, int32_t *failed) {
  if (n_nodes < 0 || (!colors && n_nodes) || (!edges && n_edges) || !failed) return fail(BE_EARG, "bad graph");
  Graph g;
  g.n = n_nodes;
  g.color.assign(colors, colors + n_nodes);
  for (int64_t k = 0; k < n_edges; ++k) {
    int a = edges[2 * k], b = edges[2 * k + 1];
    if (a < 0 || b < 0 || a >= n_nodes || b >= n_nodes) return fail(BE_EARG, "edge endpoint out of range");
    g.edges.push_back({a, b});
  }
  *failed = graph_check(g);
  return BE_OK;
}

int be_identify(const be_einsum *ref, const be_einsum *target, char *buf, size_t len, size_t *needed) {
  if (!ref || !target) return fail(BE_EARG, "NULL einsum");
  Canon cr, ct;
  std::string err;
  int st = canonicalize(ref->e, cr, err);
  if (!st) st = canonicalize(target->e, ct, err);
  if (st) return fail(st, err);
  if (cr.key != ct.key) return fail(BE_EINVALID, "normal forms differ: " + cr.key + " vs " + ct.key);
  // sigma[canon_to_ref[(canon_to_target)^-1[x_target]]] = x_target, written ref -> target
  std::string s;
  for (size_t k = 0; k < cr.sigma_index.size(); ++k) {
    s += char('a' + cr.sigma_index[k]);
    s += "=";
    s += char('a' + ct.sigma_index[k]);
    s += ";";
  }
  for (size_t k = 0; k < cr.sigma_arg.size(); ++k)
    s += ref->e.args[cr.sigma_arg[k]].name + "=" + target->e.args[ct.sigma_arg[k]].name + ";";
  return put_string(s, buf, len, needed);
}

// ------------------------------------------------------------ database

static bool parse_record(const std::string &line, std::string &key, DbEntry &d) {
  std::vector<std::string> f;
  std::string cur;
  for (char ch : line) {
    if (ch == '\t') { f.push_back(cur); cur.clear(); }
    else cur += ch;
  }
  f.push_back(cur);
  // keys are normal forms of einsums ("be1:...") or of batches ("batch1:...")
  if (f.size() != 5 || (f[0].rfind("be1:", 0) != 0 && f[0].rfind("batch1:", 0) != 0)) return false;
  char *end = nullptr;
  long prec = std::strtol(f[2].c_str(), &end, 10);
  if (*end || f[2].empty()) return false;
  std::istringstream cs(f[3]);
  be_config c;
  std::memset(&c, 0, sizeof(c));
  if (!(cs >> c.strategy >> c.tile[0] >> c.tile[1] >> c.tile[2] >> c.tile[3] >> c.stages >> c.stage_mask >> c.vec >> c.split))
    return false;
  std::string rest;
  if (cs >> rest) return false;
  d.seconds = std::strtod(f[4].c_str(), &end);
  if (*end || f[4].empty() || !(d.seconds >= 0)) return false;
  d.cfg = c;
  key = db_key(f[0], f[1], (int)prec);
  return true;
}

int be_ctx_create(const char *db_path, const char *device_name, int32_t device, size_t hbm_budget, be_ctx **out) {
  if (!out) return fail(BE_EARG, "NULL out");
  auto x = std::make_unique<be_ctx>();
  x->device = device;
  x->hbm_budget = hbm_budget;
  if (device_name) {
    x->device_name = device_name;
  } else {
    cudaDeviceProp prop;
    cudaError_t ce = cudaGetDeviceProperties(&prop, device);
    if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(ce));
    x->device_name = prop.name;
  }
  for (auto &ch : x->device_name)
    if (ch == '\t' || ch == '\n') ch = ' ';
  if (db_path) {
    x->db_path = db_path;
    std::ifstream f(db_path);
    if (f) {
      std::string line;
      int lineno = 0;
      while (std::getline(f, line)) {
        ++lineno;
        if (line.empty()) continue;
        std::string key;
        DbEntry d;
        if (!parse_record(line, key, d))
          return fail(BE_EDB, std::string(db_path) + ":" + std::to_string(lineno) + ": malformed record");
        auto it = x->db.find(key);
        if (it == x->db.end() || d.seconds < it->second.seconds) x->db[key] = d;
      }
    }
  }
  *out = x.release();
  return BE_OK;
}

void be_ctx_destroy(be_ctx *x) {
  if (!x) return;
  for (void *p : x->stage)
    if (p) cudaFree(p);
  for (cudaStream_t q : x->pipe)
    if (q) cudaStreamDestroy(q);
  for (cudaEvent_t ev : x->pipe_ev) cudaEventDestroy(ev);
  if (x->ws) cudaFree(x->ws);
  if (x->status) cudaFree(x->status);
  for (auto &m : x->marks) {
    cudaEventDestroy(std::get<1>(m));
    cudaEventDestroy(std::get<2>(m));
  }
  delete x;
}

int be_lookup(be_ctx *x, const be_canon *c, int32_t precision, be_config *out, double *seconds) {
  NvtxRange nv("be_lookup");
  if (!x || !c || !out) return fail(BE_EARG, "NULL argument");
  std::lock_guard<std::mutex> g(x->mu);
  auto it = x->db.find(db_key(c->c.key, x->device_name, precision));
  if (it == x->db.end()) return fail(BE_ENOTFOUND, "no record for " + c->c.key);
  *out = it->second.cfg;
  if (seconds) *seconds = it->second.seconds;
  return BE_OK;
}

int be_record(be_ctx *x, const be_canon *c, int32_t precision, const be_config *cfg, double seconds) {
  if (!x || !c || !cfg) return fail(BE_EARG, "NULL argument");
  if (!(seconds >= 0)) return fail(BE_EARG, "seconds must be >= 0");
  std::lock_guard<std::mutex> g(x->mu);
  std::string key = db_key(c->c.key, x->device_name, precision);
  if (!x->db_path.empty()) {
    std::ofstream f(x->db_path, std::ios::app);
    if (!f) return fail(BE_EDB, "cannot append to " + x->db_path);
    char line[256];
    std::snprintf(line, sizeof line, "%d %d %d %d %d %d %u %d %d", cfg->strategy, cfg->tile[0], cfg->tile[1],
                  cfg->tile[2], cfg->tile[3], cfg->stages, cfg->stage_mask, cfg->vec, cfg->split);
    f << c->c.key << '\t' << x->device_name << '\t' << precision << '\t' << line << '\t';
    char sec[64];
    std::snprintf(sec, sizeof sec, "%.9e", seconds);
    f << sec << '\n';
    if (!f) return fail(BE_EDB, "write failed on " + x->db_path);
  }
  auto it = x->db.find(key);
  if (it == x->db.end() || seconds < it->second.seconds) x->db[key] = DbEntry{*cfg, seconds};
  return BE_OK;
}

int be_db_size(be_ctx *x, int64_t *n) {
  if (!x || !n) return fail(BE_EARG, "NULL argument");
  std::lock_guard<std::mutex> g(x->mu);
  *n = (int64_t)x->db.size();
  return BE_OK;
}

// ------------------------------------------------------------ execution

static int resolve_config(be_ctx *x, be_einsum *h, const be_config *cfg, int32_t precision, be_config_t &out) {
  std::memset(&out, 0, sizeof(out));
  if (cfg) {
    std::memcpy(&out, cfg, sizeof(out));
    return BE_OK;
  }
  if (x) {
    std::string err;
    int st;
    const Canon *c = be::canon_cached(h, err, st);
    if (st) return fail(st, err);
    std::lock_guard<std::mutex> g(x->mu);
    auto it = x->db.find(db_key(c->key, x->device_name, precision));
    if (it != x->db.end()) std::memcpy(&out, &it->second.cfg, sizeof(out));
  }
  return BE_OK;
}

static int choose(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                  const be_config_t &cfg, int32_t precision, int &strategy, EParams *ep, std::string &why) {
  strategy = cfg.strategy;
  EParams tmp;
  EParams &p = ep ? *ep : tmp;
  if (strategy == BE_STRAT_AUTO) {
    DensePlan dp;
    if (precision == BE_PREC_FP64 && plan_element(e, bufs, outs, cfg, p, why) == OK) strategy = BE_STRAT_ELEMENT;
    else if (precision == BE_PREC_SPLIT && plan_dense(e, bufs, outs, dp, why) == OK) strategy = BE_STRAT_DENSE_SPLIT;
    else strategy = BE_STRAT_GENERIC;
    return BE_OK;
  }
  if (strategy == BE_STRAT_ELEMENT) {
    int st = plan_element(e, bufs, outs, cfg, p, why);
    if (st) return st;
  } else if (strategy == BE_STRAT_DENSE_SPLIT) {
    DensePlan dp;
    int st = plan_dense(e, bufs, outs, dp, why);
    if (st) return st;
  } else if (strategy != BE_STRAT_GENERIC) {
    why = "unknown strategy";
    return EARG;
  }
  return BE_OK;
}

// the split, split and GEMM launches of every row of a dense plan, with the
// workspace ws (dense_workspace_bytes(M, N, K) bytes) and status word given
static cudaError_t run_dense_rows(be_ctx *x, const DensePlan &dp, const be_config_t &c, void *ws, int *status,
                                  long long wait_limit, cudaStream_t s) {
  cudaError_t ce = cudaSuccess;
  int prevB = -1;
  for (auto &r : dp.rows) {
    if (dp.K == 0) {
      ce = cudaMemsetAsync(r.C, 0, sizeof(double) * (size_t)(dp.M * dp.N), s);
    } else {
      if (r.argB != prevB) {
        KernelMark km(x, BE_KERNEL_SPLIT, s);
        ce = dense_split_b(DenseB{r.B, dp.K, dp.N, r.ldb, r.snb, dp.M, r.alB, r.beB}, ws, s);
        prevB = r.argB;
      }
      if (ce == cudaSuccess) {
        KernelMark km(x, BE_KERNEL_SPLIT, s);
        ce = dense_split_a(DenseA{r.A, dp.M, r.lda, r.ska, r.alA, r.beA}, dp.K, dp.M, dp.N, ws, s);
      }
      if (ce == cudaSuccess) {
        KernelMark km(x, BE_KERNEL_DENSE_GEMM, s);
        ce = dense_split_gemm(DenseA{r.A, dp.M, r.lda, r.ska}, dp.N, dp.K, dp.M, r.C, dp.N, ws, c.split >= 4,
                              c.tile[2] > 0 ? c.tile[2] : 1, status, wait_limit, s);
      }
    }
    if (ce != cudaSuccess) return ce;
  }
  return cudaSuccess;
}

static int do_execute(be_ctx *x, const be_einsum *hc, const be_config *cfg, int32_t precision, const be_buf *bufs,
                      int32_t n_bufs, const be_buf *outs, int32_t n_outs, const double *scalars, int32_t n_scalars,
                      void *stream) {
  be_einsum *h = const_cast<be_einsum *>(hc);
  if (!h) return fail(BE_EARG, "NULL einsum");
  if (n_bufs < 0 || n_outs < 0 || n_scalars < 0) return fail(BE_EARG, "negative count");
  const Einsum &e = h->e;
  std::vector<BufIn> bi(n_bufs), bo(n_outs);
  for (int k = 0; k < n_bufs; ++k) bi[k] = BufIn{bufs[k].ptr, bufs[k].strides, bufs[k].ndim, bufs[k].dtype};
  for (int k = 0; k < n_outs; ++k) bo[k] = BufIn{outs[k].ptr, outs[k].strides, outs[k].ndim, outs[k].dtype};
  std::string err;
  int st = check_buffers(e, bi, bo, err);
  if (st) return fail(st, err);
  if (n_scalars != (int)e.scalars.size()) return fail(BE_EARG, "scalar count differs from the spec");
  std::vector<double> sc(scalars, scalars + n_scalars);
  be_config_t c;
  st = resolve_config(x, h, cfg, precision, c);
  if (st) return st;
  int strategy;
  EParams ep;
  st = choose(e, bi, bo, c, precision, strategy, &ep, err);
  if (st) return fail(st, err);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t ce = cudaSuccess;
  if (strategy == BE_STRAT_DENSE_SPLIT) {
    if (!x) return fail(BE_EARG, "the dense split strategy needs a context (workspace)");
    DensePlan dp;
    st = plan_dense(e, bi, bo, dp, err, &sc);
    if (st) return fail(st, err);
    if (dp.M == 0 || dp.N == 0) return BE_OK;
    std::lock_guard<std::mutex> g(x->mu);
    if ((st = ensure_status(x)) || (st = ensure_ws(x, dense_workspace_bytes(dp.M, dp.N, dp.K)))) return st;
    ce = run_dense_rows(x, dp, c, x->ws, x->status, x->wait_limit, s);
    if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("dense split: ") + cudaGetErrorString(ce));
    return BE_OK;
  }
  if (strategy == BE_STRAT_ELEMENT) {
    // tile[2]: 1 = FP64 pipe, 2 = double-float on the FP32 pipe, 3 = tensor
    // cores; unset = tensor cores where the shape allows, else double-float.
    // The stacked form (divergence, face mass) defaults to double-float: its
    // tensor-core form measured slower at every order but face mass P4 (a
    // few thousand instructions per element leave the tile hand-offs
    // exposed); the autotuner times both.
    std::string why_tc;
    const bool tc_ok = element_tc_supported(ep, why_tc);
    const int variant = c.tile[2] > 0 ? c.tile[2] : (tc_ok && ep.NJ0 == 0 ? 3 : 2);
    if (variant == 3) {
      if (!tc_ok) return fail(BE_EUNSUPPORTED, "tensor-core element variant: " + why_tc);
      int *status = nullptr;
      if (x) {
        std::lock_guard<std::mutex> g(x->mu);
        if ((st = ensure_status(x))) return st;
        status = x->status;
      }
      KernelMark km(x, BE_KERNEL_ELEMENT, s);
      ce = launch_element_tc(ep, status, x ? x->wait_limit : 0, s);
      if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("launch: ") + cudaGetErrorString(ce));
      return BE_OK;
    }
    int block = c.tile[1] > 0 ? c.tile[1] : (variant == 1 ? 256 : element_df_block(ep));
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t smem = sizeof(double) * element_smem_words(ep);
    per_sm = (int)std::max<size_t>(1, std::min<size_t>(2048 / block, (220 * 1024) / (smem + 1024)));
    int64_t tiles = (ep.E + ep.tile_e - 1) / ep.tile_e;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * per_sm));
    if (ep.E > 0) {
      KernelMark km(x, BE_KERNEL_ELEMENT, s);
      if (variant == 1) ce = launch_element(ep, grid, block, s);
      else if (element_df_small(ep) && c.tile[1] <= 0)
        ce = launch_element_df_small(ep, c.tile[3] > 0 ? c.tile[3] - 1 : SMALL_FP64_SHARE16, s);
      else ce = launch_element_df(ep, grid, block, s);
    }
  } else {
    for (int i = 0; i < e.b && ce == cudaSuccess; ++i) {
      GParams p;
      st = plan_generic_row(e, i, bi, bo[i], sc, p, err);
      if (st) return fail(st, err);
      KernelMark km(x, BE_KERNEL_GENERIC, s);
      ce = launch_generic(p, s);
    }
  }
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("launch: ") + cudaGetErrorString(ce));
  return BE_OK;
}

int be_execute(be_ctx *x, const be_einsum *h, const be_config *cfg, int32_t precision, const be_buf *bufs,
               int32_t n_bufs, const be_buf *outs, int32_t n_outs, const double *scalars, int32_t n_scalars,
               void *stream) {
  NvtxRange nv("be_execute");
  return do_execute(x, h, cfg, precision, bufs, n_bufs, outs, n_outs, scalars, n_scalars, stream);
}

}  // extern "C"

int be::execute_internal(be_ctx *x, const be_einsum *h, const be_config *cfg, int32_t precision, const be_buf *bufs,
                         int32_t n_bufs, const be_buf *outs, int32_t n_outs, const double *scalars,
                         int32_t n_scalars, void *stream) {
  return do_execute(x, h, cfg, precision, bufs, n_bufs, outs, n_outs, scalars, n_scalars, stream);
}

extern "C" {

int be_plan_strategy(be_ctx *x, const be_einsum *hc, const be_config *cfg, int32_t precision, int32_t *strategy) {
  be_einsum *h = const_cast<be_einsum *>(hc);
  if (!h || !strategy) return fail(BE_EARG, "NULL argument");
  be_config_t c;
  int st = resolve_config(x, h, cfg, precision, c);
  if (st) return st;
  // plan on placeholder buffers (pointers are not dereferenced while planning)
  const Einsum &e = h->e;
  std::vector<BufIn> bi, bo;
  static double dummy;
  for (auto &b : e.buffers) bi.push_back(BufIn{&dummy, nullptr, (int32_t)b.shape.size(), b.dtype});
  for (int i = 0; i < e.b; ++i) bo.push_back(BufIn{&dummy, nullptr, (int32_t)e.out.size(), e.out_dtype});
  std::string why;
  int s;
  st = choose(e, bi, bo, c, precision, s, nullptr, why);
  if (st) return fail(st, why);
  *strategy = s;
  return BE_OK;
}

static size_t dense_bytes(const Buffer &b) {
  size_t n = (size_t)dtype_size(b.dtype);
  for (auto d : b.shape) n *= (size_t)d;
  return n;
}

// Chunking of be_execute_host along the output's outermost letter L: every
// buffer must either not involve L (copied whole) or have L as its outermost
// dimension in every access and nowhere else (a chunk of L is then one
// contiguous slice).  kind[k]: 0 whole, 1 sliced; false if any buffer fails.
static bool host_chunking(const Einsum &e, std::vector<int> &kind) {
  if (e.out.empty()) return false;
  const int L = e.out[0];
  kind.assign(e.buffers.size(), 0);
  std::vector<int> seen(e.buffers.size(), 0);   // bit 0: L outermost, bit 1: L elsewhere or outermost not L
  for (int i = 0; i < e.b; ++i)
    for (int j = 0; j < e.n; ++j) {
      const Arg &A = e.args[e.rows[i][j]];
      const auto &letters = e.in[j];
      if (!A.functional()) {
        int &f = seen[A.buffer];
        for (size_t d = 0; d < letters.size(); ++d)
          if (letters[d] == L) f |= d == 0 ? 1 : 2;
        if (!letters.empty() && letters[0] != L && std::find(letters.begin(), letters.end(), L) != letters.end()) f |= 2;
        continue;
      }
      for (const XNode &nd : A.nodes) {
        if (nd.op != X_REF) continue;
        int &f = seen[nd.id];
        bool has_l = false, outer_l = false;
        for (size_t d = 0; d < nd.sub.size(); ++d)
          if (nd.sub[d] >= 0 && letters[nd.sub[d]] == L) {
            has_l = true;
            if (d == 0) outer_l = true;
            else f |= 2;
          }
        if (has_l && outer_l) f |= 1;
        if (!has_l && (f & 1)) f |= 2;   // the same buffer also read without L
        if (!has_l) f |= 4;
      }
    }
  for (size_t k = 0; k < e.buffers.size(); ++k) {
    const int f = seen[k];
    if (f & 2) return false;
    if ((f & 1) && (f & 4)) return false;
    kind[k] = (f & 1) ? 1 : 0;
  }
  return true;
}

// the einsum with the extent of the output's outermost letter set to n
static void resize_outer(const Einsum &src, const std::vector<int> &kind, int64_t n, Einsum &dst) {
  dst = src;
  const int L = src.out[0];
  dst.len[L] = n;
  for (size_t k = 0; k < dst.buffers.size(); ++k)
    if (kind[k] == 1) dst.buffers[k].shape[0] = n;
  for (int i = 0; i < src.b; ++i)
    for (int j = 0; j < src.n; ++j) {
      Arg &A = dst.args[src.rows[i][j]];
      for (size_t d = 0; d < src.in[j].size() && d < A.shape.size(); ++d)
        if (src.in[j][d] == L) A.shape[d] = n;
    }
}

int be_execute_host(be_ctx *x, const be_einsum *h, const be_config *cfg, int32_t precision, const be_buf *bufs,
                    int32_t n_bufs, const be_buf *outs, int32_t n_outs, const double *scalars, int32_t n_scalars,
                    void *stream) {
  NvtxRange nv("be_execute_host");
  if (!x || !h) return fail(BE_EARG, "NULL argument");
  const Einsum &e = h->e;
  if (n_bufs != (int)e.buffers.size() || n_outs != e.b) return fail(BE_EARG, "buffer counts differ from the spec");
  std::vector<size_t> need;
  for (int k = 0; k < n_bufs; ++k) {
    if (bufs[k].strides) return fail(BE_EARG, "host buffers must be dense row-major");
    need.push_back(dense_bytes(e.buffers[k]));
  }
  size_t out_bytes = (size_t)dtype_size(e.out_dtype);
  for (auto d : e.out_shape()) out_bytes *= (size_t)d;
  for (int k = 0; k < n_outs; ++k) need.push_back(out_bytes);
  be_config_t c;
  int rst = resolve_config(x, const_cast<be_einsum *>(h), cfg, precision, c);
  if (rst) return rst;
  std::lock_guard<std::mutex> g(x->mu);
  cudaError_t ce = cudaSuccess;
  if (x->stage.size() < need.size()) {
    x->stage.resize(need.size(), nullptr);
    x->stage_size.resize(need.size(), 0);
  }
  for (size_t k = 0; k < need.size(); ++k) {
    if (x->stage_size[k] < need[k]) {
      if (x->stage[k]) cudaFree(x->stage[k]);
      x->stage[k] = nullptr;
      ce = cudaMalloc(&x->stage[k], need[k] ? need[k] : 16);
      if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("cudaMalloc: ") + cudaGetErrorString(ce));
      x->stage_size[k] = need[k];
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<be_buf> db(n_bufs), dout(n_outs);
  // Large inputs stream through in chunks of the output's outermost letter:
  // copy-in of chunk c + 1, the kernels of chunk c and copy-out of chunk
  // c - 1 run on three streams, so both PCIe directions and the GPU overlap.
  size_t total = 0;
  for (size_t v : need) total += v;
  std::vector<int> kind;
  const int64_t L_ext = e.out.empty() ? 0 : e.len[e.out[0]];
  const int n_chunks = (int)std::min<int64_t>(8, L_ext);
  if (total >= ((size_t)64 << 20) && n_chunks >= 2 && host_chunking(e, kind)) {
    for (int q = 0; q < 3; ++q)
      if (!x->pipe[q] && (ce = cudaStreamCreateWithFlags(&x->pipe[q], cudaStreamNonBlocking)) != cudaSuccess)
        return fail(BE_ECUDA, std::string("stream: ") + cudaGetErrorString(ce));
    while ((int)x->pipe_ev.size() < 2 * n_chunks + 1) {
      cudaEvent_t ev;
      if ((ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return fail(BE_ECUDA, std::string("event: ") + cudaGetErrorString(ce));
      x->pipe_ev.push_back(ev);
    }
    cudaStream_t s_in = x->pipe[0], s_run = x->pipe[1], s_out = x->pipe[2];
    // after the caller's earlier work on `stream`
    cudaEventRecord(x->pipe_ev[2 * n_chunks], s);
    cudaStreamWaitEvent(s_in, x->pipe_ev[2 * n_chunks], 0);
    for (int k = 0; k < n_bufs; ++k)
      if (kind[k] == 0 && need[k] &&
          (ce = cudaMemcpyAsync(x->stage[k], bufs[k].ptr, need[k], cudaMemcpyHostToDevice, s_in)) != cudaSuccess)
        return fail(BE_ECUDA, std::string("H2D: ") + cudaGetErrorString(ce));
    const int64_t chunk = (L_ext + n_chunks - 1) / n_chunks;
    const size_t out_row = L_ext ? out_bytes / (size_t)L_ext : 0;
    for (int ch = 0; ch < n_chunks; ++ch) {
      const int64_t e0 = ch * chunk, n = std::min<int64_t>(chunk, L_ext - e0);
      if (n <= 0) break;
      for (int k = 0; k < n_bufs; ++k) {
        const size_t row = need[k] / (size_t)L_ext;
        if (kind[k] == 1) {
          ce = cudaMemcpyAsync((char *)x->stage[k] + e0 * row, (const char *)bufs[k].ptr + e0 * row, n * row,
                               cudaMemcpyHostToDevice, s_in);
          if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("H2D: ") + cudaGetErrorString(ce));
        }
        db[k] = be_buf{(char *)x->stage[k] + (kind[k] == 1 ? e0 * row : 0), nullptr, bufs[k].ndim, bufs[k].dtype};
      }
      for (int k = 0; k < n_outs; ++k)
        dout[k] = be_buf{(char *)x->stage[n_bufs + k] + e0 * out_row, nullptr, outs[k].ndim, outs[k].dtype};
      cudaEventRecord(x->pipe_ev[2 * ch], s_in);
      cudaStreamWaitEvent(s_run, x->pipe_ev[2 * ch], 0);
      be_einsum part;
      resize_outer(e, kind, n, part.e);
      int st = do_execute(nullptr, &part, reinterpret_cast<const be_config *>(&c), precision, db.data(), n_bufs,
                          dout.data(), n_outs, scalars, n_scalars, s_run);
      if (st) return st;
      cudaEventRecord(x->pipe_ev[2 * ch + 1], s_run);
      cudaStreamWaitEvent(s_out, x->pipe_ev[2 * ch + 1], 0);
      for (int k = 0; k < n_outs; ++k)
        if (n * out_row &&
            (ce = cudaMemcpyAsync((char *)outs[k].ptr + e0 * out_row, (char *)x->stage[n_bufs + k] + e0 * out_row,
                                  n * out_row, cudaMemcpyDeviceToHost, s_out)) != cudaSuccess)
          return fail(BE_ECUDA, std::string("D2H: ") + cudaGetErrorString(ce));
    }
    ce = cudaStreamSynchronize(s_out);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s_run);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s_in);
    if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("sync: ") + cudaGetErrorString(ce));
    return BE_OK;
  }
  for (int k = 0; k < n_bufs; ++k) {
    if (need[k]) ce = cudaMemcpyAsync(x->stage[k], bufs[k].ptr, need[k], cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("H2D: ") + cudaGetErrorString(ce));
    db[k] = be_buf{x->stage[k], nullptr, bufs[k].ndim, bufs[k].dtype};
  }
  for (int k = 0; k < n_outs; ++k) dout[k] = be_buf{x->stage[n_bufs + k], nullptr, outs[k].ndim, outs[k].dtype};
  int st = do_execute(nullptr, h, reinterpret_cast<const be_config *>(&c), precision, db.data(), n_bufs, dout.data(),
                      n_outs, scalars, n_scalars, stream);
  if (st) return st;
  for (int k = 0; k < n_outs; ++k) {
    if (out_bytes) ce = cudaMemcpyAsync(outs[k].ptr, x->stage[n_bufs + k], out_bytes, cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("D2H: ") + cudaGetErrorString(ce));
  }
  ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("sync: ") + cudaGetErrorString(ce));
  return BE_OK;
}

int be_ctx_set_timing(be_ctx *x, int32_t enable) {
  if (!x) return fail(BE_EARG, "NULL context");
  std::lock_guard<std::mutex> g(x->mu);
  x->timing = enable != 0;
  return BE_OK;
}

int be_ctx_timing(be_ctx *x, int32_t kernel, int64_t *launches, double *total_ms) {
  if (!x || !launches || !total_ms) return fail(BE_EARG, "NULL argument");
  std::lock_guard<std::mutex> g(x->mu);
  *launches = 0;
  *total_ms = 0.0;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> keep;
  for (auto &m : x->marks) {
    if (std::get<0>(m) != kernel) {
      keep.push_back(m);
      continue;
    }
    float ms = 0.f;
    cudaError_t ce = cudaEventSynchronize(std::get<2>(m));
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, std::get<1>(m), std::get<2>(m));
    cudaEventDestroy(std::get<1>(m));
    cudaEventDestroy(std::get<2>(m));
    if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("timing: ") + cudaGetErrorString(ce));
    *launches += 1;
    *total_ms += ms;
  }
  x->marks.swap(keep);
  return BE_OK;
}

// ------------------------------------------------------------ autotuner

static void tune_candidates(const Einsum &e, const std::vector<BufIn> &bi, const std::vector<BufIn> &bo,
                            int32_t precision, std::vector<be_config_t> &out) {
  be_config_t c;
  std::string why;
  EParams ep;
  DensePlan dp;
  std::memset(&c, 0, sizeof(c));
  c.strategy = BE_STRAT_ELEMENT;
  if (precision == BE_PREC_FP64 && plan_element(e, bi, bo, c, ep, why) == OK) {
    if (element_tc_supported(ep, why)) {
      c.tile[2] = 3;                                   // the tensor-core variant has one launch shape
      out.push_back(c);
    }
    for (int variant : {2, 1})
      for (int te : {8, 16, 32, 64, 128})
        for (int blk : {128, 256}) {
          if (variant == 1 && te != 32) continue;      // the FP64-pipe variant: one candidate per block size
          c.tile[0] = te;
          c.tile[1] = blk;
          c.tile[2] = variant;
          if (plan_element(e, bi, bo, c, ep, why) == OK) out.push_back(c);
        }
  }
  std::memset(&c, 0, sizeof(c));
  if (precision == BE_PREC_SPLIT && plan_dense(e, bi, bo, dp, why) == OK) {
    // one drain interval: k-blocks of 64 between drains of the leading
    // accumulator beyond 1 would trade the a-priori 1e-6 bound for speed
    c.strategy = BE_STRAT_DENSE_SPLIT;
    c.tile[2] = 1;
    out.push_back(c);
  }
  std::memset(&c, 0, sizeof(c));
  c.strategy = BE_STRAT_GENERIC;
  out.push_back(c);
}

// ------------------------------------------------------------ persistent batch

}  // extern "C"

// largest workspace of a batch's factored intermediates (bytes)
static constexpr double FACTOR_WS_MAX = 4.0 * (1ull << 30);
// concurrent graph branches of a batch's dense instances
static constexpr int NDN = 4;

struct be_batch {
  be_ctx *x = nullptr;
  std::vector<GParams> rows;
  std::vector<PTile> tiles;
  GParams *d_rows = nullptr;
  PTile *d_tiles = nullptr;
  unsigned long long *d_counter = nullptr;
  // branch 0 runs the element instances, branches 1..NDN the dense ones
  // (round robin, each with its own split workspace)
  cudaStream_t cap = nullptr, branch[1 + NDN] = {};
  cudaEvent_t ev[2 + NDN] = {};
  size_t ws_stride = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid = 0, block = 256;
  double terms = 0;
  // instances per strategy, and the split workspace and status word of the
  // dense instances (owned by the batch: the graph holds their addresses)
  int32_t n_kind[3] = {0, 0, 0};
  void *ws = nullptr;
  int *status = nullptr;
  bool own_status = false;
  // factored instances: their pairwise steps, ordered by dependency depth
  // (phases) in the one tile list, with the intermediates in a workspace
  // owned by the batch
  int phases = 1;
  unsigned int *d_done = nullptr;   // finished tiles per row (factored batches)
  int32_t n_factored = 0;
  void *fws = nullptr;
  size_t fws_bytes = 0;
  // per instance: 0 loop nest, 1 element, 2 dense, 3 factored steps in the
  // persistent launch, 4 factored steps on a dense branch (be_batch_instance_kind)
  std::vector<int8_t> inst_kind;
  ~be_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    for (auto st : branch)
      if (st) cudaStreamDestroy(st);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    if (d_rows) cudaFree(d_rows);
    if (d_tiles) cudaFree(d_tiles);
    if (d_counter) cudaFree(d_counter);
    if (d_done) cudaFree(d_done);
    if (ws) cudaFree(ws);
    if (fws) cudaFree(fws);
    if (own_status && status) cudaFree(status);
  }
};

extern "C" {

// Key of a batch in the tuning database: the canonical keys of its
// instances (normal forms with their lengths, Alg. 1), sorted and hashed
// (FNV-1a, 64 bits), so that any renaming or reordering of the instances
// finds the same record.
static int batch_key(int32_t n, const be_einsum *const *es, std::string &key) {
  std::vector<std::string> ks;
  std::string err;
  int st;
  for (int k = 0; k < n; ++k) {
    if (!es[k]) return fail(BE_EARG, "NULL einsum in batch");
    const Canon *c = be::canon_cached(const_cast<be_einsum *>(es[k]), err, st);
    if (st) return fail(st, err);
    ks.push_back(c->key);
  }
  std::sort(ks.begin(), ks.end());
  uint64_t h = 1469598103934665603ull;
  for (auto &k : ks) {
    for (unsigned char ch : k) h = (h ^ ch) * 1099511628211ull;
    h = (h ^ '\n') * 1099511628211ull;
  }
  char buf[64];
  std::snprintf(buf, sizeof buf, "batch1:%d:%016llx", n, (unsigned long long)h);
  key = buf;
  return BE_OK;
}

int be_batch_create(be_ctx *x, int32_t n, const be_einsum *const *es, const be_buf *const *bufs,
                    const int32_t *n_bufs, const be_buf *const *outs, const int32_t *n_outs,
                    const double *const *scalars, const int32_t *n_scalars, const be_config *cfg, be_batch **out) {
  if (!out || n < 0 || (n > 0 && (!es || !bufs || !n_bufs || !outs || !n_outs))) return fail(BE_EARG, "bad batch arguments");
  auto b = std::make_unique<be_batch>();
  b->x = x;
  be_config_t c;
  std::memset(&c, 0, sizeof(c));
  if (cfg) {
    std::memcpy(&c, cfg, sizeof(c));
  } else if (x && n > 0) {
    // a configuration tuned for this batch (be_tune_batch), by the batch key
    std::string bk;
    if (batch_key(n, es, bk) == BE_OK) {
      std::lock_guard<std::mutex> g(x->mu);
      auto it = x->db.find(db_key(bk, x->device_name, BE_PREC_FP64));
      if (it != x->db.end()) std::memcpy(&c, &it->second.cfg, sizeof(c));
    }
  }
  b->block = c.tile[0] > 0 ? c.tile[0] : 256;
  if (b->block % 32 || b->block > 256) return fail(BE_EARG, "block size must be a multiple of 32 up to 256");
  const int cost_log2 = c.tile[1] > 0 ? c.tile[1] : 20;
  const int per_sm = c.tile[2] > 0 ? c.tile[2] : 4;
  const double cost_target = std::ldexp(1.0, cost_log2);
  // strategy policy: element-shaped FP64 instances take the element strategy
  // unless stage_mask bit 0 is set; with split >= 1, FP64 instances of GEMM
  // form with at least 2^tile[3] (default 2^23, the best of 2^16 .. 2^25 on
  // the uneven mix: smaller GEMMs spend more in the split kernels than they
  // save) multiply-adds take the split-precision tensor-core strategy
  const bool allow_element = !(c.stage_mask & 1u);
  const double dense_min = std::ldexp(1.0, c.tile[3] > 0 ? c.tile[3] : 23);
  // factored steps are two-operand rows, often GEMM tiles, which need the
  // 256-thread block
  const bool allow_factor = !(c.stage_mask & 2u) && b->block == 256;
  std::vector<int> el_inst, dn_inst;
  std::vector<be_config_t> el_cfg;
  std::vector<DensePlan> dn_plan;
  size_t ws_need = 0;
  std::string err;
  struct FacInst {
    int k = 0;
    FactorOrder fo;
    std::vector<std::vector<FOp>> ops;   // per row, the operand views
    std::vector<void *> outs;            // per row, the output
    // the split-precision route: two steps, the last a GEMM of the first
    // step's result (laid out as inter_letters) and user operand `user`
    // (permuted first into a dense user_letters layout when copy_user)
    bool dense = false, copy_user = false;
    int user = -1;
    std::vector<int8_t> inter_letters, user_letters;
  };
  std::vector<FacInst> fac_inst;
  // steps of the factored instances on the dense branches: a generic launch
  // (the first step, a permuted copy) or a split-precision GEMM
  struct DnStep {
    bool gemm = false;
    GParams gp;
    DensePlan dp;
  };
  std::vector<std::vector<DnStep>> dnf_steps;   // per dense-routed instance
  // the dense route of a factored FP64 instance (split >= 2; off at 1: on
  // the uneven mix it cost 6 %, since the persistent grid holds every SM
  // until its queue drains and the route's chain of small launches per
  // instance then runs in the tail): the order has
  // two steps, the last contracting the first step's result I with one
  // operand U into the output as a GEMM of at least dense_min multiply-adds
  // that carries at least half of the instance's multiply-adds; the output's
  // letters are those of one operand followed by those of the other (no
  // letter kept by both).  I is laid out (its output letters, K) and U, when
  // its own layout does not flatten that way, is first copied so
  auto dense_route = [&](const Einsum &e, FacInst &fi) {
    if (c.split < 2 || e.out_dtype != F64 || fi.fo.steps.size() != 2) return;
    for (auto &a : e.args)
      if (a.dtype != F64) return;
    const int n = e.n, sa = fi.fo.steps[1][0], sb = fi.fo.steps[1][1];
    if (sb < 0 || (sa == n) == (sb == n) || std::max(sa, sb) != n) return;
    const int user = sa == n ? sb : sa;
    const FOp &U0 = fi.ops[0][user];
    bool inU[26] = {false}, inI[26] = {false}, isOut[26] = {false};
    for (int8_t ch : U0.letters) inU[ch] = true;
    for (int8_t ch : fi.fo.letters[0]) inI[ch] = true;
    for (int8_t ch : e.out) isOut[ch] = true;
    if (e.out.empty()) return;
    const bool A_is_I = inI[e.out[0]];
    const bool *inA = A_is_I ? inI : inU, *inB = A_is_I ? inU : inI;
    size_t nm = 0;
    while (nm < e.out.size() && inA[e.out[nm]]) ++nm;
    for (size_t k2 = 0; k2 < e.out.size(); ++k2) {
      const int8_t ch = e.out[k2];
      if (inA[ch] && inB[ch]) return;                               // a letter kept by both
      if (k2 < nm ? !inA[ch] : !inB[ch]) return;
    }
    std::vector<std::pair<int64_t, int8_t>> kk;                      // K letters by U's stride
    double M = 1, N = 1, K = 1;
    for (size_t k2 = 0; k2 < U0.letters.size(); ++k2) {
      const int8_t ch = U0.letters[k2];
      if (isOut[ch]) continue;
      if (!inI[ch]) return;                                          // summed inside U alone
      kk.push_back({-std::llabs(U0.strides[k2]), ch});
      K *= (double)e.len[ch];
    }
    for (int8_t ch : fi.fo.letters[0])
      if (!isOut[ch] && !inU[ch]) return;                            // summed inside I alone
    if (kk.empty()) return;
    for (size_t k2 = 0; k2 < e.out.size(); ++k2) (k2 < nm ? M : N) *= (double)e.len[e.out[k2]];
    if (M * N * K * e.b < dense_min || M * N * K < 0.5 * fi.fo.factored) return;
    std::stable_sort(kk.begin(), kk.end());
    std::vector<int8_t> kl;
    for (auto &pr : kk) kl.push_back(pr.second);
    fi.user_letters.clear();
    fi.inter_letters.clear();
    for (int8_t ch : e.out) {
      if (inU[ch]) fi.user_letters.push_back(ch);
      if (inI[ch]) fi.inter_letters.push_back(ch);
    }
    fi.user_letters.insert(fi.user_letters.end(), kl.begin(), kl.end());
    fi.inter_letters.insert(fi.inter_letters.end(), kl.begin(), kl.end());
    // U in place when its output letters (in the output's order) and K each
    // flatten to one stride in every row
    auto flat = [&](const FOp &f, const std::vector<int8_t> &ls) {
      int64_t expect = 0;
      for (int k2 = (int)ls.size() - 1; k2 >= 0; --k2) {
        int64_t st = -1;
        for (size_t d = 0; d < f.letters.size(); ++d)
          if (f.letters[d] == ls[k2]) st = f.strides[d];
        if (k2 == (int)ls.size() - 1) expect = st;
        if (st != expect || st <= 0) return false;
        expect *= e.len[ls[k2]];
      }
      return true;
    };
    std::vector<int8_t> uo(fi.user_letters.begin(), fi.user_letters.end() - (long)kl.size());
    fi.copy_user = false;
    for (int i = 0; i < e.b; ++i)
      if (!flat(fi.ops[i][user], uo) || !flat(fi.ops[i][user], kl)) fi.copy_user = true;
    fi.user = user;
    fi.dense = true;
  };
  // a generic row (or a factored step) into the tile list of its group
  // (group 0: the factored steps without dependencies, 1: the unfactored
  // rows, q + 1: the factored steps of dependency depth q >= 1); outputs
  // per tile so that each tile costs about cost_target operand terms.  deps
  // are rows whose tiles must all finish first (-1: none); *row_out gets
  // the new row, or -1 for a row without outputs
  std::vector<std::vector<PTile>> ptiles(2);
  std::vector<int> row_tiles;
  auto add_row = [&](const GParams &p, int group, int k, const int deps[2], int *row_out) -> int {
    *row_out = -1;
    if (p.total_out == 0) return BE_OK;
    if (p.mode == 3 && b->block != 256)
      return fail(BE_EARG, "instance " + std::to_string(k) + ": rows evaluated as GEMM tiles need a block of 256 threads");
    if ((int)ptiles.size() <= group) ptiles.resize(group + 1);
    std::vector<PTile> &pt = ptiles[group];
    const int row = (int)b->rows.size();
    b->rows.push_back(p);
    row_tiles.push_back(0);
    *row_out = row;
    PTile base{row, 0, 0, 0, {-1, -1}, {0, 0}};
    for (int q = 0; q < 2; ++q)
      if (deps[q] >= 0) {
        base.dep[q] = deps[q];
        base.need[q] = row_tiles[deps[q]];
      }
    const double per_out = (double)std::max<int64_t>(1, p.total_con) * std::max(1, p.n_ops);
    b->terms += per_out * (double)p.total_out;
    int64_t tile, units;
    if (p.mode == 3) {   // units are GEMM tiles of tile x tile outputs
      const double per_tile = per_out * p.gemm.tile * p.gemm.tile;
      tile = std::max<int64_t>(1, std::min<int64_t>((int64_t)(cost_target / per_tile), 65536));
      units = p.gemm.tiles;
    } else {
      tile = (int64_t)(cost_target / per_out);
      if (p.mode == 0) {
        tile = std::max<int64_t>(32, std::min<int64_t>(tile, 65536));
        tile = (tile + 31) / 32 * 32;
      } else {
        tile = std::max<int64_t>(1, std::min<int64_t>(tile, 65536));
      }
      units = p.total_out;
    }
    for (int64_t s0 = 0; s0 < units; s0 += tile) {
      PTile t = base;
      t.start = s0;
      t.count = std::min(tile, units - s0);
      pt.push_back(t);
      ++row_tiles[row];
    }
    return BE_OK;
  };
  b->inst_kind.assign(n, 0);
  for (int k = 0; k < n; ++k) {
    if (!es[k]) return fail(BE_EARG, "NULL einsum in batch");
    const Einsum &e = es[k]->e;
    std::vector<BufIn> bi(n_bufs[k]), bo(n_outs[k]);
    for (int q = 0; q < n_bufs[k]; ++q) bi[q] = BufIn{bufs[k][q].ptr, bufs[k][q].strides, bufs[k][q].ndim, bufs[k][q].dtype};
    for (int q = 0; q < n_outs[k]; ++q) bo[q] = BufIn{outs[k][q].ptr, outs[k][q].strides, outs[k][q].ndim, outs[k][q].dtype};
    int st = check_buffers(e, bi, bo, err);
    if (st) return fail(st, "instance " + std::to_string(k) + ": " + err);
    const int ns = n_scalars ? n_scalars[k] : 0;
    if (ns != (int)e.scalars.size()) return fail(BE_EARG, "instance " + std::to_string(k) + ": scalar count");
    std::vector<double> sc(ns);
    for (int q = 0; q < ns; ++q) sc[q] = scalars[k][q];
    {
      // the instance's own configuration (database record, else defaults)
      be_config_t ci;
      st = resolve_config(x, const_cast<be_einsum *>(es[k]), nullptr, BE_PREC_FP64, ci);
      if (st) return st;
      std::string why;
      EParams ep;
      DensePlan dp;
      if (allow_element && plan_element(e, bi, bo, ci, ep, why) == OK) {
        ci.strategy = BE_STRAT_ELEMENT;
        el_inst.push_back(k);
        el_cfg.push_back(ci);
        ++b->n_kind[1];
        b->inst_kind[k] = 1;
        continue;
      }
      if (c.split >= 1 && plan_dense(e, bi, bo, dp, why, &sc) == OK &&
          (double)dp.M * (double)dp.N * (double)dp.K * (double)dp.rows.size() >= dense_min) {
        ws_need = std::max(ws_need, dense_workspace_bytes(dp.M, dp.N, dp.K));
        dn_inst.push_back(k);
        dn_plan.push_back(dp);
        ++b->n_kind[2];
        b->inst_kind[k] = 2;
        continue;
      }
    }
    // factored evaluation: an instance whose order of steps cuts the loop
    // nest's multiply-adds at least 1.5 times runs as one- and two-operand steps over
    // dense intermediates (stage_mask bit 1 turns this off)
    if (allow_factor) {
      FactorOrder fo;
      bool fac = factor_order(e, 1.5, fo) &&
                 (double)fo.inter_elems * e.b * dtype_size(e.out_dtype) <= FACTOR_WS_MAX;
      std::vector<std::vector<FOp>> ops;
      for (int i = 0; fac && i < e.b; ++i) {
        std::vector<FOp> r(e.n);
        for (int j = 0; fac && j < e.n; ++j) fac = operand_fop(e, i, j, bi, r[j]);
        ops.push_back(r);
      }
      if (fac) {
        FacInst fi;
        fi.k = k;
        fi.fo = fo;
        fi.ops = ops;
        for (int i = 0; i < e.b; ++i) fi.outs.push_back(bo[i].ptr);
        dense_route(e, fi);
        if (fi.dense) {
          ++b->n_kind[2];
          b->inst_kind[k] = 4;
        } else {
          ++b->n_kind[0];
          ++b->n_factored;
          b->inst_kind[k] = 3;
        }
        fac_inst.push_back(std::move(fi));
        continue;
      }
    }
    ++b->n_kind[0];
    for (int i = 0; i < e.b; ++i) {
      GParams p;
      st = plan_generic_row(e, i, bi, bo[i], sc, p, err);
      if (st) return fail(st, "instance " + std::to_string(k) + ": " + err);
      const int none[2] = {-1, -1};
      int row;
      st = add_row(p, 1, k, none, &row);
      if (st) return st;
    }
  }
  // the factored instances' steps: intermediates carved from one workspace,
  // each step in the phase after the steps it reads
  {
    size_t need = 0;
    for (auto &fi : fac_inst) {
      const Einsum &e = es[fi.k]->e;
      for (int i = 0; i < e.b; ++i) {
        for (size_t q = 0; q + 1 < fi.fo.steps.size(); ++q) {
          double elems = 1.0;
          for (int8_t c : fi.fo.letters[q]) elems *= (double)e.len[c];
          need += ((size_t)elems * dtype_size(e.out_dtype) + 255) / 256 * 256;
        }
        if (fi.dense && fi.copy_user) {
          double elems = 1.0;
          for (int8_t c : fi.user_letters) elems *= (double)e.len[c];
          need += ((size_t)elems * dtype_size(e.out_dtype) + 255) / 256 * 256;
        }
      }
    }
    if (need) {
      cudaError_t ce0 = cudaMalloc(&b->fws, need);
      if (ce0 != cudaSuccess) return fail(BE_ECUDA, std::string("batch workspace: ") + cudaGetErrorString(ce0));
      b->fws_bytes = need;
    }
    size_t off = 0;
    for (auto &fi : fac_inst) {
      const Einsum &e = es[fi.k]->e;
      const int n = e.n;
      if (fi.dense) {
        // the dense route: per row the permuted copy of U (if any), the
        // first step into I (generic launches) and the GEMM, in that order
        // on one dense branch
        auto dense_fop = [&](const std::vector<int8_t> &ls) {
          FOp r;
          r.dtype = e.out_dtype;
          r.letters = ls;
          r.ptr = (char *)b->fws + off;
          double elems = 1.0;
          for (int8_t ch : ls) elems *= (double)e.len[ch];
          off += ((size_t)elems * dtype_size(e.out_dtype) + 255) / 256 * 256;
          r.strides.assign(ls.size(), 1);
          for (int d = (int)ls.size() - 2; d >= 0; --d) r.strides[d] = r.strides[d + 1] * e.len[ls[d + 1]];
          return r;
        };
        std::vector<DnStep> steps;
        for (int i = 0; i < e.b; ++i) {
          FOp U = fi.ops[i][fi.user];
          int st;
          if (fi.copy_user) {
            const FOp Uc = dense_fop(fi.user_letters);
            DnStep d;
            st = plan_factor_step(e, U, nullptr, Uc.letters, const_cast<void *>(Uc.ptr), d.gp, err);
            if (st) return fail(st, "instance " + std::to_string(fi.k) + ", operand copy: " + err);
            steps.push_back(d);
            U = Uc;
          }
          const FOp I = dense_fop(fi.inter_letters);
          const int s0a = fi.fo.steps[0][0], s0b = fi.fo.steps[0][1];
          DnStep d0;
          st = plan_factor_step(e, fi.ops[i][s0a], s0b >= 0 ? &fi.ops[i][s0b] : nullptr, I.letters,
                                const_cast<void *>(I.ptr), d0.gp, err);
          if (st) return fail(st, "instance " + std::to_string(fi.k) + ", factored step: " + err);
          steps.push_back(d0);
          DnStep d1;
          std::string why;
          if (plan_factor_step_dense(e, I, U, e.out, fi.outs[i], d1.dp, why) == OK) {
            d1.gemm = true;
            ws_need = std::max(ws_need, dense_workspace_bytes(d1.dp.M, d1.dp.N, d1.dp.K));
          } else {   // the layouts were chosen for the GEMM; a generic step keeps the result correct
            st = plan_factor_step(e, I, &U, e.out, fi.outs[i], d1.gp, err);
            if (st) return fail(st, "instance " + std::to_string(fi.k) + ", factored step: " + err);
          }
          steps.push_back(d1);
        }
        dnf_steps.push_back(std::move(steps));
        continue;
      }
      for (int i = 0; i < e.b; ++i) {
        std::vector<FOp> slot = fi.ops[i];
        std::vector<int> slot_phase(n, -1), slot_row(n, -1);
        for (size_t q = 0; q < fi.fo.steps.size(); ++q) {
          const bool last = q + 1 == fi.fo.steps.size();
          const int sa = fi.fo.steps[q][0], sb = fi.fo.steps[q][1];   // sb < 0: a unary step
          const int phase = 1 + std::max(slot_phase[sa], sb >= 0 ? slot_phase[sb] : -1);
          FOp r;
          r.dtype = e.out_dtype;
          r.letters = fi.fo.letters[q];
          void *dst = fi.outs[i];
          if (!last) {
            dst = (char *)b->fws + off;
            double elems = 1.0;
            for (int8_t c : r.letters) elems *= (double)e.len[c];
            off += ((size_t)elems * dtype_size(e.out_dtype) + 255) / 256 * 256;
          }
          r.ptr = dst;
          r.strides.assign(r.letters.size(), 1);
          for (int d = (int)r.letters.size() - 2; d >= 0; --d) r.strides[d] = r.strides[d + 1] * e.len[r.letters[d + 1]];
          GParams p;
          int st = plan_factor_step(e, slot[sa], sb >= 0 ? &slot[sb] : nullptr, r.letters, dst, p, err);
          if (st) return fail(st, "instance " + std::to_string(fi.k) + ", factored step: " + err);
          const int deps[2] = {slot_row[sa], sb >= 0 ? slot_row[sb] : -1};
          int row;
          st = add_row(p, phase == 0 ? 0 : phase + 1, fi.k, deps, &row);
          if (st) return st;
          b->phases = std::max(b->phases, phase + 1);
          slot.push_back(r);
          slot_phase.push_back(phase);
          slot_row.push_back(row);
        }
      }
    }
  }
  // within each group, longest tiles first (cost = outputs x terms per
  // output; ties by position); the groups one after the other, so that
  // every tile comes after the tiles it depends on
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (auto &pt : ptiles) {
    std::vector<double> cost(pt.size());
    for (size_t t = 0; t < pt.size(); ++t) {
      const GParams &p = b->rows[pt[t].row];
      cost[t] = (double)pt[t].count * (double)std::max<int64_t>(1, p.total_con) * std::max(1, p.n_ops) *
                (p.mode == 3 ? (double)p.gemm.tile * p.gemm.tile : 1.0);
    }
    std::vector<size_t> order(pt.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](size_t a2, size_t c2) { return cost[a2] > cost[c2]; });
    for (size_t t : order) b->tiles.push_back(pt[t]);
  }
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->tiles.size(), (int64_t)sms * per_sm));
  cudaError_t ce = cudaMalloc(&b->d_rows, sizeof(GParams) * std::max<size_t>(1, b->rows.size()));
  if (ce == cudaSuccess) ce = cudaMalloc(&b->d_tiles, sizeof(PTile) * std::max<size_t>(1, b->tiles.size()));
  if (ce == cudaSuccess) ce = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
  if (ce == cudaSuccess && b->n_factored) ce = cudaMalloc(&b->d_done, sizeof(unsigned int) * std::max<size_t>(1, b->rows.size()));
  if (ce == cudaSuccess && !b->rows.empty())
    ce = cudaMemcpy(b->d_rows, b->rows.data(), sizeof(GParams) * b->rows.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess && !b->tiles.empty())
    ce = cudaMemcpy(b->d_tiles, b->tiles.data(), sizeof(PTile) * b->tiles.size(), cudaMemcpyHostToDevice);
  b->ws_stride = (ws_need + 255) / 256 * 256;
  if (ce == cudaSuccess && ws_need) ce = cudaMalloc(&b->ws, b->ws_stride * (size_t)NDN);
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("batch setup: ") + cudaGetErrorString(ce));
  if (!el_inst.empty() || !dn_inst.empty() || !dnf_steps.empty() || b->n_factored) {
    if (x) {
      std::lock_guard<std::mutex> g(x->mu);
      int st = ensure_status(x);
      if (st) return st;
      b->status = x->status;
    } else {
      ce = cudaMalloc(&b->status, sizeof(int));
      if (ce == cudaSuccess) ce = cudaMemset(b->status, 0, sizeof(int));
      if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("batch status word: ") + cudaGetErrorString(ce));
      b->own_status = true;
    }
  }
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int q = 0; q < 1 + NDN && ce == cudaSuccess; ++q) ce = cudaStreamCreateWithFlags(&b->branch[q], cudaStreamNonBlocking);
  for (int q = 0; q < 2 + NDN && ce == cudaSuccess; ++q) ce = cudaEventCreateWithFlags(&b->ev[q], cudaEventDisableTiming);
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("batch setup: ") + cudaGetErrorString(ce));
  const bool timing = x && x->timing;
  if (x) x->timing = false;   // no timing events inside the captured graph
  // element and dense instances: their launches, once outside the capture
  // (first-launch set-up such as kernel attributes happens here) and then
  // captured on their own branches
  const long long wl = x ? x->wait_limit : 0;
  auto launch_el = [&](cudaStream_t st) -> int {
    for (size_t q = 0; q < el_inst.size(); ++q) {
      const int k = el_inst[q];
      be_config cq;
      std::memcpy(&cq, &el_cfg[q], sizeof(cq));
      int r = be::execute_internal(x, es[k], &cq, BE_PREC_FP64, bufs[k], n_bufs[k], outs[k], n_outs[k],
                                   n_scalars && n_scalars[k] ? scalars[k] : nullptr, n_scalars ? n_scalars[k] : 0, st);
      if (r) return r;
    }
    return BE_OK;
  };
  auto launch_dn = [&](int br, cudaStream_t st) -> cudaError_t {
    be_config_t cd;
    std::memset(&cd, 0, sizeof(cd));
    for (size_t q = br; q < dn_inst.size(); q += NDN) {
      cudaError_t r = run_dense_rows(nullptr, dn_plan[q], cd, (char *)b->ws + b->ws_stride * br, b->status, wl, st);
      if (r != cudaSuccess) return r;
    }
    // the dense-routed factored instances continue the round robin
    for (size_t q = 0; q < dnf_steps.size(); ++q) {
      if ((dn_inst.size() + q) % NDN != (size_t)br) continue;
      for (const DnStep &d : dnf_steps[q]) {
        cudaError_t r = d.gemm ? run_dense_rows(nullptr, d.dp, cd, (char *)b->ws + b->ws_stride * br, b->status, wl, st)
                               : launch_generic(d.gp, st);
        if (r != cudaSuccess) return r;
      }
    }
    return cudaSuccess;
  };
  int est = launch_el(b->branch[0]);
  for (int q = 0; !est && q < NDN && ce == cudaSuccess; ++q) ce = launch_dn(q, b->branch[1 + q]);
  if (!est && ce == cudaSuccess) ce = cudaDeviceSynchronize();
  if (est || ce != cudaSuccess) {
    if (x) x->timing = timing;
    return est ? est : fail(BE_ECUDA, std::string("batch first launch: ") + cudaGetErrorString(ce));
  }
  // capture: counter reset + persistent launch on the capture stream; the
  // element and dense branches fork from it and join back
  ce = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    // the branches fork before the persistent launch, so that the three
    // parts are concurrent in the graph (the side kernels take SMs as the
    // persistent grid's CTAs leave) and join after it
    cudaError_t c1 = cudaSuccess;
    const bool side = !el_inst.empty() || !dn_inst.empty() || !dnf_steps.empty();
    if (side) {
      c1 = cudaEventRecord(b->ev[0], b->cap);
      for (int q = 0; q < 1 + NDN && c1 == cudaSuccess; ++q) c1 = cudaStreamWaitEvent(b->branch[q], b->ev[0], 0);
      if (c1 == cudaSuccess) {
        est = launch_el(b->branch[0]);
        if (est) c1 = cudaErrorUnknown;
      }
      for (int q = 0; q < NDN && c1 == cudaSuccess; ++q) c1 = launch_dn(q, b->branch[1 + q]);
    }
    // one persistent launch; factored steps wait in it for the steps they
    // read (left out, with its counter resets, when there are no generic
    // tiles and the branches hold all the work)
    if (!b->tiles.empty() || !side) {
      if (c1 == cudaSuccess) c1 = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), b->cap);
      if (c1 == cudaSuccess && b->d_done)
        c1 = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned int) * b->rows.size(), b->cap);
      if (c1 == cudaSuccess)
        c1 = launch_persistent(b->d_rows, b->d_tiles, (int64_t)b->tiles.size(), b->d_counter, b->d_done,
                               b->d_done ? b->status : nullptr, wl, b->grid, b->block, b->cap);
    }
    if (side) {
      for (int q = 0; q < 1 + NDN && c1 == cudaSuccess; ++q) c1 = cudaEventRecord(b->ev[1 + q], b->branch[q]);
      for (int q = 0; q < 1 + NDN && c1 == cudaSuccess; ++q) c1 = cudaStreamWaitEvent(b->cap, b->ev[1 + q], 0);
    }
    ce = cudaStreamEndCapture(b->cap, &b->graph);
    if (c1 != cudaSuccess) ce = c1;
  }
  if (x) x->timing = timing;
  if (est) return est;
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("batch setup: ") + cudaGetErrorString(ce));
  *out = b.release();
  return BE_OK;
}

int be_tune_batch(be_ctx *x, int32_t n, const be_einsum *const *es, const be_buf *const *bufs,
                  const int32_t *n_bufs, const be_buf *const *outs, const int32_t *n_outs,
                  const double *const *scalars, const int32_t *n_scalars, const be_config *base, int32_t reps,
                  void *stream, be_config *best, double *best_seconds, int32_t *n_tried) {
  if (!x || !best || n <= 0) return fail(BE_EARG, "bad arguments");
  if (n_tried) *n_tried = 0;
  std::string bk;
  int st = batch_key(n, es, bk);
  if (st) return st;
  be_canon bc;
  bc.c.key = bk;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a, e2;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&e2) != cudaSuccess) return fail(BE_ECUDA, "event");
  double best_t = -1;
  // the persistent part's launch shape: block size, CTAs per SM and the
  // operand terms per tile; the strategy policy (split, tile[3],
  // stage_mask) is the caller's
  for (int block : {128, 256})
    for (int per_sm : {2, 3, 4})
      for (int cost : {18, 20, 22}) {
        be_config cand;
        std::memset(&cand, 0, sizeof(cand));
        if (base) cand = *base;
        cand.tile[0] = block;
        cand.tile[1] = cost;
        cand.tile[2] = per_sm;
        be_batch *bt = nullptr;
        st = be_batch_create(x, n, es, bufs, n_bufs, outs, n_outs, scalars, n_scalars, &cand, &bt);
        if (st) { st = BE_OK; continue; }     // a candidate that cannot be planned is skipped
        double total = 0;
        int done = 0;
        bool okc = be_batch_run(bt, stream) == BE_OK;
        for (int r = 0; okc && r < std::max(1, reps); ++r) {
          cudaEventRecord(a, s);
          okc = be_batch_run(bt, stream) == BE_OK;
          cudaEventRecord(e2, s);
          if (!okc || cudaEventSynchronize(e2) != cudaSuccess) { okc = false; break; }
          float ms = 0;
          cudaEventElapsedTime(&ms, a, e2);
          total += ms * 1e-3;
          ++done;
        }
        be_batch_destroy(bt);
        if (!okc || !done) continue;
        const double sec = total / done;
        if (n_tried) ++*n_tried;
        const int rs = be_record(x, &bc, BE_PREC_FP64, &cand, sec);
        if (rs) { cudaEventDestroy(a); cudaEventDestroy(e2); return rs; }
        if (best_t < 0 || sec < best_t) {
          best_t = sec;
          *best = cand;
        }
      }
  cudaEventDestroy(a);
  cudaEventDestroy(e2);
  if (best_t < 0) return fail(BE_EUNSUPPORTED, "no candidate batch configuration ran");
  if (best_seconds) *best_seconds = best_t;
  return BE_OK;
}

int be_batch_kinds(const be_batch *b, int32_t *generic, int32_t *element, int32_t *dense) {
  if (!b) return fail(BE_EARG, "NULL batch");
  if (generic) *generic = b->n_kind[0];
  if (element) *element = b->n_kind[1];
  if (dense) *dense = b->n_kind[2];
  return BE_OK;
}

int be_batch_instance_kind(const be_batch *b, int32_t k, int32_t *kind) {
  if (!b || !kind) return fail(BE_EARG, "NULL argument");
  if (k < 0 || k >= (int32_t)b->inst_kind.size()) return fail(BE_EARG, "instance index out of range");
  *kind = b->inst_kind[k];
  return BE_OK;
}

int be_batch_factored(const be_batch *b, int32_t *instances, int32_t *phases, int64_t *workspace_bytes) {
  if (!b) return fail(BE_EARG, "NULL batch");
  if (instances) *instances = b->n_factored;
  if (phases) *phases = b->phases;
  if (workspace_bytes) *workspace_bytes = (int64_t)b->fws_bytes;
  return BE_OK;
}

int be_batch_run(be_batch *b, void *stream) {
  NvtxRange nv("be_batch_run");
  if (!b) return fail(BE_EARG, "NULL batch");
  cudaStream_t s = (cudaStream_t)stream;
  KernelMark km(b->x, BE_KERNEL_PERSISTENT, s);
  cudaError_t ce = cudaGraphLaunch(b->exec, s);
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
  return BE_OK;
}

int be_batch_info(const be_batch *b, int64_t *rows, int64_t *tiles, double *terms) {
  if (!b) return fail(BE_EARG, "NULL batch");
  if (rows) *rows = (int64_t)b->rows.size();
  if (tiles) *tiles = (int64_t)b->tiles.size();
  if (terms) *terms = b->terms;
  return BE_OK;
}

void be_batch_destroy(be_batch *b) { delete b; }

int be_tune(be_ctx *x, const be_einsum *hc, int32_t precision, const be_buf *bufs, int32_t n_bufs, const be_buf *outs,
            int32_t n_outs, const double *scalars, int32_t n_scalars, int32_t warmup, int32_t min_reps,
            double min_seconds, int32_t force, void *stream, be_config *best, double *best_seconds,
            int32_t *n_tried) {
  be_einsum *h = const_cast<be_einsum *>(hc);
  if (!x || !h || !best) return fail(BE_EARG, "NULL argument");
  if (n_tried) *n_tried = 0;
  std::string err;
  int st;
  const Canon *cn = be::canon_cached(h, err, st);
  if (st) return fail(st, err);
  const std::string key = db_key(cn->key, x->device_name, precision);
  if (!force) {
    std::lock_guard<std::mutex> g(x->mu);
    auto it = x->db.find(key);
    if (it != x->db.end()) {          // resume: a tuned key is not timed again
      *best = it->second.cfg;
      if (best_seconds) *best_seconds = it->second.seconds;
      return BE_OK;
    }
  }
  const Einsum &e = h->e;
  std::vector<BufIn> bi(n_bufs), bo(n_outs);
  for (int k = 0; k < n_bufs; ++k) bi[k] = BufIn{bufs[k].ptr, bufs[k].strides, bufs[k].ndim, bufs[k].dtype};
  for (int k = 0; k < n_outs; ++k) bo[k] = BufIn{outs[k].ptr, outs[k].strides, outs[k].ndim, outs[k].dtype};
  st = check_buffers(e, bi, bo, err);
  if (st) return fail(st, err);
  std::vector<be_config_t> cands;
  tune_candidates(e, bi, bo, precision, cands);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return fail(BE_ECUDA, "event");
  double best_t = -1;
  be_canon bc;
  bc.c = *cn;
  for (auto &c : cands) {
    const be_config *cfg = reinterpret_cast<const be_config *>(&c);
    for (int w = 0; w < warmup; ++w) {
      st = do_execute(x, h, cfg, precision, bufs, n_bufs, outs, n_outs, scalars, n_scalars, stream);
      if (st) break;
    }
    if (st) { st = BE_OK; continue; }     // a candidate that cannot run is skipped
    int reps = 0;
    double total = 0;
    while (reps < std::max(1, min_reps) || total < min_seconds) {
      cudaEventRecord(a, s);
      st = do_execute(x, h, cfg, precision, bufs, n_bufs, outs, n_outs, scalars, n_scalars, stream);
      cudaEventRecord(b, s);
      if (st) break;
      if (cudaEventSynchronize(b) != cudaSuccess) { st = BE_ECUDA; break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      total += ms * 1e-3;
      ++reps;
      if (reps > 100000) break;
    }
    if (st) { st = BE_OK; continue; }
    const double sec = total / reps;
    if (n_tried) ++*n_tried;
    int rs = be_record(x, &bc, precision, cfg, sec);
    if (rs) { cudaEventDestroy(a); cudaEventDestroy(b); return rs; }
    if (best_t < 0 || sec < best_t) {
      best_t = sec;
      *best = *cfg;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (best_t < 0) return fail(BE_EUNSUPPORTED, "no candidate configuration ran");
  if (best_seconds) *best_seconds = best_t;
  return BE_OK;
}

int be_ctx_set_wait_limit(be_ctx *x, int64_t cycles) {
  if (!x) return fail(BE_EARG, "NULL context");
  if (cycles < 0) return fail(BE_EARG, "negative wait limit");
  std::lock_guard<std::mutex> g(x->mu);
  x->wait_limit = cycles;
  return BE_OK;
}

int be_status(be_ctx *x, int32_t *device_status) {
  if (!x || !device_status) return fail(BE_EARG, "NULL argument");
  *device_status = BE_OK;
  if (!x->status) return BE_OK;
  cudaError_t ce = cudaDeviceSynchronize();
  int v = 0;
  if (ce == cudaSuccess) ce = cudaMemcpy(&v, x->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (ce == cudaSuccess) ce = cudaMemset(x->status, 0, sizeof(int));
  if (ce != cudaSuccess) return fail(BE_ECUDA, std::string("status: ") + cudaGetErrorString(ce));
  *device_status = v;
  return BE_OK;
}

}  // extern "C"
