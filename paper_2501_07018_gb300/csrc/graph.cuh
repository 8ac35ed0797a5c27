// Replay of captured launch sequences (CUDA graphs) for launch-bound loops.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace pdlp {

// A launch sequence captured once from a stream and replayed as a CUDA graph.  capture()
// returns false (nothing launched, no error left pending) where the stream cannot be
// captured; the caller then launches the sequence directly.
class Replay {
 public:
  Replay() = default;
  Replay(const Replay&) = delete;
  Replay& operator=(const Replay&) = delete;
  ~Replay() {
    if (exec_) cudaGraphExecDestroy(exec_);
  }
  template <class F>
  bool capture(cudaStream_t st, F&& body) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    cudaGraph_t g = nullptr;
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      throw;
    }
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      return false;
    }
    const cudaError_t ei = cudaGraphInstantiate(&exec_, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      exec_ = nullptr;
      (void)cudaGetLastError();
      return false;
    }
    return true;
  }
  void launch(cudaStream_t st) { PDLP_CUDA_CHECK(cudaGraphLaunch(exec_, st)); }

 private:
  cudaGraphExec_t exec_ = nullptr;
};

}  // namespace pdlp
