// Kernel launches that can be recorded instead of issued.  A thread that
// installs a LaunchRecorder turns every launch made through be_launch into a
// kernel node of the recorder's graph (chained in launch order), with the
// same function, launch shape and argument values; no stream capture is
// involved, so other threads' stream or device synchronizations are never
// affected.  Without a recorder, be_launch is cudaLaunchKernel.
#pragma once

#include <tuple>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

namespace be {

struct LaunchRecorder {
  cudaGraph_t graph = nullptr;
  cudaGraphNode_t last = nullptr;
  cudaError_t status = cudaSuccess;
  int nodes = 0;
};

// the calling thread's recorder, or nullptr (defined in abi.cpp)
LaunchRecorder *&launch_recorder();

template <typename... KArgs, typename... Args>
cudaError_t be_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                      Args &&...args) {
  static_assert(sizeof...(KArgs) == sizeof...(Args), "argument count");
  std::tuple<std::decay_t<KArgs>...> vals(std::forward<Args>(args)...);
  void *ptrs[sizeof...(KArgs) > 0 ? sizeof...(KArgs) : 1];
  std::apply([&](auto &...v) {
    int k = 0;
    ((ptrs[k++] = (void *)&v), ...);
  }, vals);
  LaunchRecorder *rec = launch_recorder();
  if (!rec) return cudaLaunchKernel((const void *)kernel, grid, block, ptrs, smem, s);
  cudaKernelNodeParams p = {};
  p.func = (void *)kernel;
  p.gridDim = grid;
  p.blockDim = block;
  p.sharedMemBytes = (unsigned)smem;
  p.kernelParams = ptrs;
  cudaGraphNode_t node;
  const cudaError_t e = cudaGraphAddKernelNode(&node, rec->graph, rec->last ? &rec->last : nullptr, rec->last ? 1 : 0, &p);
  if (e != cudaSuccess) {
    rec->status = e;
    return e;
  }
  rec->last = node;
  ++rec->nodes;
  return cudaSuccess;
}

}  // namespace be
