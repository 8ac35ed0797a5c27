// Shared device helpers of the PDLP library: error handling, deterministic block
// and grid reductions, and the device-resident solver state.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <stdexcept>
#include <string>

namespace pdlp {

// ---------------------------------------------------------------------------
// host-side error plumbing: every failure becomes a PdlpError carrying the ABI code
// ---------------------------------------------------------------------------
struct PdlpError : public std::runtime_error {
  int code;
  PdlpError(int c, const std::string& msg) : std::runtime_error(msg), code(c) {}
};

void set_last_error(const std::string& msg);
void set_last_error_cstr(const char* msg, const char* detail);  // never allocates

#define PDLP_CUDA_CHECK(expr)                                                          \
  do {                                                                                 \
    cudaError_t err__ = (expr);                                                        \
    if (err__ != cudaSuccess) {                                                        \
      if (err__ == cudaErrorMemoryAllocation)                                          \
        throw ::pdlp::PdlpError(-2, std::string("out of device memory at ") + #expr); \
      throw ::pdlp::PdlpError(-3, std::string(#expr) + ": " + cudaGetErrorString(err__)); \
    }                                                                                  \
  } while (0)

#define PDLP_LAUNCH_CHECK() PDLP_CUDA_CHECK(cudaGetLastError())

constexpr int kThreads = 256;           // threads per CTA of every grid kernel
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sums K values over the CTA of NW warps (fixed tree: lanes, then warps in order).
// The result is valid in thread 0.  `scratch` needs K * NW doubles of shared memory.
template <int K, int NW = kWarps>
__device__ __forceinline__ void block_sum(double (&v)[K], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k * NW + warp] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < NW; ++w) s += scratch[k * NW + w];
      v[k] = s;
    }
  }
  __syncthreads();
}

// "Last CTA" detection: every CTA calls this once after publishing its partials;
// exactly one CTA (the last to arrive) gets true, with all other CTAs' writes
// visible.  The counter is reset for the next launch.
__device__ __forceinline__ bool last_block_arrival(unsigned int* counter) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1);
    if (s_last) *counter = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// Fixed-order sum of partials[0..count) by one CTA of NW warps; result in thread 0.
template <int NW = kWarps>
__device__ __forceinline__ double block_sum_array(const double* partials, int count,
                                                  double* scratch) {
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < count; i += blockDim.x) v[0] += ((volatile const double*)partials)[i];
  block_sum<1, NW>(v, scratch);
  return v[0];
}

// Totals of per-CTA partials by one CTA: KS arrays to sum, then KM arrays of
// non-negative values to take the maximum of, each `count` long, stored one after the
// other from `part`.  Every thread reads its strided elements of all arrays (L2 loads,
// issued together), then fixed-order block trees; results valid in thread 0.  The
// partials must have been made visible (last_block_arrival).
// The shared scratch is taken as arrays of the exact sizes KS * NW and KM * NW, so a
// call with smaller arrays does not compile.
template <int KS, int KM, int NW = kWarps>
__device__ __forceinline__ void block_reduce_partials(const double* part, int count,
                                                      double (&sums)[KS], double (&maxs)[KM],
                                                      double (&sm_sum)[KS * NW],
                                                      double (&sm_max)[KM * NW]) {
#pragma unroll
  for (int k = 0; k < KS; ++k) sums[k] = 0.0;
#pragma unroll
  for (int k = 0; k < KM; ++k) maxs[k] = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < KS; ++k) sums[k] += __ldcg(part + (size_t)k * count + i);
#pragma unroll
    for (int k = 0; k < KM; ++k) maxs[k] = fmax(maxs[k], __ldcg(part + (size_t)(KS + k) * count + i));
  }
  block_sum<KS, NW>(sums, sm_sum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const double w = warp_max(maxs[k]);
    if (lane == 0) sm_max[k * NW + warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      double a = 0.0;
      for (int w = 0; w < NW; ++w) a = fmax(a, sm_max[k * NW + w]);
      maxs[k] = a;
    }
  }
  __syncthreads();
}

// Sums each of K arrays partials[k*count .. k*count+count) by one CTA in a single
// pass: a group of blockDim/K threads (a power of two <= 32) per array reads it
// strided, then shuffles; every thread of the group holds the result.  The order is
// fixed, so the result is deterministic.  Requires blockDim.x % K == 0 and K <= blockDim.x.
template <int K>
__device__ __forceinline__ double group_sum_arrays(const double* partials, int count) {
  constexpr int GS = (kThreads / K) >= 32 ? 32 : (kThreads / K);
  const int k = threadIdx.x / GS, r = threadIdx.x % GS;
  double v = 0.0;
  if (k < K)
    for (int i = r; i < count; i += GS) v += ((volatile const double*)partials)[k * count + i];
#pragma unroll
  for (int o = GS >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, GS);
  return v;
}

// ---------------------------------------------------------------------------
// device-resident scalar state of the PDHG loop (Algorithm 1 / Algorithm 2)
// ---------------------------------------------------------------------------
struct DevState {
  int32_t cur;        // which of the two iterate buffers holds z^{n,t}
  int32_t accepted;   // outcome of the last step attempt
  int32_t retries;    // consecutive rejected attempts of the current iteration
  int32_t error;      // 1: non-finite step quantities, 2: retry cap reached
  int64_t k;          // accepted iterations in total
  int64_t t;          // accepted iterations since the last restart
  int64_t attempts;   // all step attempts
  int64_t rejected;
  int64_t spmv_a;     // number of A x products (for KKT-pass accounting)
  int64_t spmv_at;
  double eta;         // step size of the next attempt
  double eta_hat;     // eta' returned by the last accepted step
  double eta_acc;     // eta of the last accepted step
  double omega;       // primal weight
  double W;           // sum of accepted etas since the last restart
  double last_dx2, last_dy2, last_inter, last_eta_bar;
  int32_t max_retries;
  int32_t pad_;
  double fixed_eta;   // > 0: constant step, every attempt accepted (no Algorithm 2)
};

struct Counters {
  unsigned int spmv_a_done;
  unsigned int misc_done[8];
};

}  // namespace pdlp
