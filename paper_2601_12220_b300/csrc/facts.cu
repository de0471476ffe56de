// record_facts and the transform library (Sec. "Integration with other
// frameworks", the transformation writer's view): a configuration is
// registered against an idealized reference batched einsum, timed on the
// device on synthetic operands of the reference's shapes (warm-up runs
// first), and the measured time is stored in the tuning database under the
// reference's normal form, so that every isomorphic einsum retrieves it.
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "handles.hpp"

namespace be {

namespace {

// counter-based synthetic values: splitmix64 of (seed, index), mapped to
// [-1, 1) for floating types and to -3..3 for integers
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void fill_kernel(void *p, int64_t n, int dtype, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64(seed * 0x100000001B3ull + (uint64_t)i);
    const double u = (double)(h >> 11) * 0x1p-52 - 1.0;   // [-1, 1)
    const int k = (int)(h % 7) - 3;
    switch (dtype) {
      case I8: ((int8_t *)p)[i] = (int8_t)k; break;
      case I32: ((int32_t *)p)[i] = k; break;
      case I64: ((int64_t *)p)[i] = k; break;
      case F16: ((__half *)p)[i] = __float2half((float)u); break;
      case BF16: ((__nv_bfloat16 *)p)[i] = __float2bfloat16((float)u); break;
      case F32: ((float *)p)[i] = (float)u; break;
      case F64: ((double *)p)[i] = u; break;
      case C64: ((float2 *)p)[i] = make_float2((float)u, (float)(-u)); break;
      case C128: ((double2 *)p)[i] = make_double2(u, -u); break;
      default: break;
    }
  }
}

struct DeviceBufs {
  std::vector<void *> ptrs;
  ~DeviceBufs() {
    for (void *p : ptrs) cudaFree(p);
  }
  void *alloc(size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
};

int set_error(int code, const std::string &msg) {
  set_last_error(msg);
  return code;
}

}  // namespace

// time cfg on synthetic operands of e's declared shapes and record it
int record_facts(be_ctx *x, be_einsum *h, const be_config *cfg, int32_t precision, int32_t warmup, int32_t reps,
                 double *seconds, std::string &err) {
  const Einsum &e = h->e;
  DeviceBufs mem;
  std::vector<be_buf> bufs, outs;
  for (size_t k = 0; k < e.buffers.size(); ++k) {
    const Buffer &b = e.buffers[k];
    int64_t n = 1;
    for (int64_t d : b.shape) n *= d;
    void *p = mem.alloc((size_t)n * dtype_size(b.dtype));
    if (!p) { err = "device allocation for the synthetic operands failed"; return ECUDA; }
    if (n > 0) fill_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256>>>(p, n, b.dtype, k + 1);
    bufs.push_back(be_buf{p, nullptr, (int32_t)b.shape.size(), b.dtype});
  }
  int64_t n_out = 1;
  for (int8_t c : e.out) n_out *= e.len[c];
  for (int r = 0; r < e.b; ++r) {
    void *p = mem.alloc((size_t)n_out * dtype_size(e.out_dtype));
    if (!p) { err = "device allocation for the outputs failed"; return ECUDA; }
    outs.push_back(be_buf{p, nullptr, (int32_t)e.out.size(), e.out_dtype});
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { err = "synthetic operand fill failed"; return ECUDA; }
  const std::vector<double> sc(e.scalars.size(), 1.0);   // every runtime scalar 1
  cudaStream_t s = nullptr;
  int st = OK;
  for (int w = 0; w < warmup && !st; ++w)
    st = execute_internal(x, h, cfg, precision, bufs.data(), (int32_t)bufs.size(), outs.data(), (int32_t)outs.size(),
                          sc.data(), (int32_t)sc.size(), s);
  if (st) { err = "the configuration does not run on the reference"; return st; }
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { err = "event"; return ECUDA; }
  cudaEventRecord(a, s);
  for (int r = 0; r < reps && !st; ++r)
    st = execute_internal(x, h, cfg, precision, bufs.data(), (int32_t)bufs.size(), outs.data(), (int32_t)outs.size(),
                          sc.data(), (int32_t)sc.size(), s);
  cudaEventRecord(b, s);
  const cudaError_t ce = cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st) { err = "the configuration failed while timed"; return st; }
  if (ce != cudaSuccess) { err = std::string("timing: ") + cudaGetErrorString(ce); return ECUDA; }
  *seconds = ms * 1e-3 / reps;
  return OK;
}

}  // namespace be

using namespace be;
using be::set_error;

extern "C" {

int be_record_facts(be_ctx *x, const be_einsum *ref, const be_config *cfg, int32_t precision, int32_t warmup,
                    int32_t reps, double *seconds) {
  if (!x || !ref || !cfg) return set_error(BE_EARG, "NULL argument");
  if (warmup < 0 || reps < 1) return set_error(BE_EARG, "warmup >= 0 and reps >= 1 required");
  be_einsum *h = const_cast<be_einsum *>(ref);
  std::string err;
  double sec = 0;
  int st = record_facts(x, h, cfg, precision, warmup, reps, &sec, err);
  if (st) return set_error(st, "record_facts: " + err);
  be_canon *c = nullptr;
  if ((st = be_canonicalize(ref, &c))) return st;
  st = be_record(x, c, precision, cfg, sec);
  be_free_canon(c);
  if (st) return st;
  if (seconds) *seconds = sec;
  return BE_OK;
}

// Transform library: one registration per line,
//   <be_parse text of the reference> => <strategy> <tile0> <tile1> <tile2> <tile3>
//                                       [<stages> <stage_mask> <vec> <split> [<precision>]]
// ('#' starts a comment line); every line is parsed before any is timed.
int be_load_transforms(be_ctx *x, const char *text, int32_t warmup, int32_t reps, int32_t *n_recorded) {
  if (!x || !text) return set_error(BE_EARG, "NULL argument");
  if (n_recorded) *n_recorded = 0;
  struct Item {
    be_einsum *e;
    be_config c;
    int32_t prec;
  };
  std::vector<Item> items;
  auto release = [&]() {
    for (auto &it : items) be_free_einsum(it.e);
  };
  std::istringstream in(text);
  std::string line;
  int ln = 0;
  while (std::getline(in, line)) {
    ++ln;
    size_t a = line.find_first_not_of(" \t\r");
    if (a == std::string::npos || line[a] == '#') continue;
    const size_t arrow = line.find("=>");
    if (arrow == std::string::npos) {
      release();
      return set_error(BE_EPARSE, "transform line " + std::to_string(ln) + ": expected '<reference> => <config>'");
    }
    Item it;
    std::memset(&it.c, 0, sizeof(it.c));
    it.prec = BE_PREC_FP64;
    std::istringstream cs(line.substr(arrow + 2));
    if (!(cs >> it.c.strategy >> it.c.tile[0] >> it.c.tile[1] >> it.c.tile[2] >> it.c.tile[3])) {
      release();
      return set_error(BE_EPARSE, "transform line " + std::to_string(ln) + ": config needs strategy and four tiles");
    }
    if (cs >> it.c.stages) {
      if (!(cs >> it.c.stage_mask >> it.c.vec >> it.c.split)) {
        release();
        return set_error(BE_EPARSE, "transform line " + std::to_string(ln) + ": stages, stage_mask, vec and split go together");
      }
      cs >> it.prec;
    }
    const std::string ref = line.substr(0, arrow);
    int st = be_parse(ref.c_str(), &it.e);
    if (st) {
      std::string m = be_last_error();
      release();
      return set_error(st, "transform line " + std::to_string(ln) + ": " + m);
    }
    items.push_back(it);
  }
  for (auto &it : items) {
    const int st = be_record_facts(x, it.e, &it.c, it.prec, warmup, reps, nullptr);
    if (st) {
      release();
      return st;
    }
    if (n_recorded) ++*n_recorded;
  }
  release();
  return BE_OK;
}

}  // extern "C"
