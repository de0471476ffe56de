// Library-internal definitions of the C-ABI handles, shared by the
// translation units that implement include/be.h.
#pragma once

#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/be.h"
#include "canon.hpp"
#include "plan.hpp"

using namespace be;

struct be_einsum {
  Einsum e;
  std::mutex mu;
  std::unique_ptr<Canon> canon;   // cached C(e) for lookups
  // raised from a loop-nest kernel (be_raise): the text it was written as,
  // the loop name of each index letter and the output array of each row
  std::string raised_spec;
  std::vector<std::string> loop_names, outputs;
};

struct be_canon {
  Canon c;
};

struct DbEntry {
  be_config cfg;
  double seconds;
};

struct be_ctx {
  std::string db_path, device_name;
  int device = -1;
  size_t hbm_budget = 0;
  std::mutex mu;
  std::unordered_map<std::string, DbEntry> db;
  // staging memory of be_execute_host, and its copy-in / compute / copy-out
  // streams and per-chunk events (created on first use)
  std::vector<void *> stage;
  std::vector<size_t> stage_size;
  cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> pipe_ev;
  // workspace of the dense split strategy and the device status word
  void *ws = nullptr;
  size_t ws_size = 0;
  int *status = nullptr;
  // limit of the tensor-core kernels' pipeline waits in SM cycles (0: about
  // one second); lowered only to exercise the BE_ETIMEOUT path
  long long wait_limit = 0;
  // optional per-kernel timing: (kernel id, start, stop) event pairs
  bool timing = false;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> marks;
};

// brackets one kernel launch with events when x has timing enabled
struct KernelMark {
  be_ctx *x;
  int id;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  KernelMark(be_ctx *x_, int id_, cudaStream_t s_) : x(x_), id(id_), s(s_) {
    if (x && x->timing && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, s);
  }
  ~KernelMark() {
    if (a && b) {
      cudaEventRecord(b, s);
      x->marks.emplace_back(id, a, b);
    }
  }
};


namespace be {
void set_last_error(const std::string &msg);
// be_execute without the C wrapper (x may be NULL; cfg NULL = database / defaults)
int execute_internal(be_ctx *x, const be_einsum *h, const be_config *cfg, int32_t precision, const be_buf *bufs,
                     int32_t n_bufs, const be_buf *outs, int32_t n_outs, const double *scalars, int32_t n_scalars,
                     void *stream);
// canonical form of a parsed einsum, computed once and cached in the handle
const Canon *canon_cached(be_einsum *e, std::string &err, int &st);
}  // namespace be
