// pdlp_kkt_products_noalloc: the optimality measures of pdlp_kkt for a point whose
// matrix products the caller already has, computed without allocating any memory.
//
// The reduction needs scratch for its per-CTA partial sums, an arrival counter and
// the final sums.  Here that scratch is one file-scope device array of fixed size
// (kNaDoubles doubles, about 74 KB), which every GPU that loads the library holds
// until the process exits.  Host code must not pass the array's name to a kernel
// (on the host it is only a stand-in symbol); its device address is looked up once
// per device with cudaGetSymbolAddress and cached.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/pdlp.h"
#include "common.cuh"

namespace pdlp {
namespace {

constexpr int kNaCtas = 1024;                    // most CTAs the reduction uses
constexpr int kNaSums = 9;                       // quantities reduced per CTA
constexpr int kNaDoubles = kNaSums * kNaCtas + kNaSums + 2;  // partials, result, counter
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

// Sums of one point (x, y) with products (ax = A x, aty = A'y), unscaled LP:
//   [0] ||Ax - proj_[lc,uc](Ax)||^2   [1] ||(c - A'y) - proj_R(c - A'y)||^2
//   [2] c'x   [3] lc'y+ - uc'y-   [4] lv'r+ - uv'r-   [5] ||c||^2   [6] ||Combine(lc,uc)||^2
//   [7] max |primal residual|   [8] max |dual residual|
__global__ void __launch_bounds__(kThreads)
    k_kkt_products(const double* c, const double* lc, const double* uc, const double* lv,
                   const double* uv, const double* x, const double* y, const double* ax,
                   const double* aty, int64_t m, int64_t n, double* scratch) {
  __shared__ double red[7 * kWarps];
  __shared__ double mred[2 * kWarps];
  double* part = scratch;
  double* result = scratch + kNaSums * kNaCtas;
  unsigned int* counter = reinterpret_cast<unsigned int*>(result + kNaSums);
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  double mx0 = 0.0, mx1 = 0.0;
  for (int64_t i = t0; i < m; i += st) {
    const double a = ax[i], l = lc[i], u = uc[i], yi = y[i];
    const double pr = a - fmin(fmax(a, l), u);
    v[0] += pr * pr;
    mx0 = fmax(mx0, fabs(pr));
    if (yi > 0.0)
      v[3] += l * yi;
    else if (yi < 0.0)
      v[3] += u * yi;
    const double b = fmax(0.0, fmax(isfinite(l) ? fabs(l) : 0.0, isfinite(u) ? fabs(u) : 0.0));
    v[6] += b * b;
  }
  for (int64_t j = t0; j < n; j += st) {
    const double g = c[j] - aty[j];
    const bool lf = isfinite(lv[j]), uf = isfinite(uv[j]);
    double r = g;
    if (lf && !uf) r = fmax(g, 0.0);
    if (!lf && uf) r = fmin(g, 0.0);
    if (!lf && !uf) r = 0.0;
    const double dr = g - r;
    v[1] += dr * dr;
    mx1 = fmax(mx1, fabs(dr));
    v[2] += c[j] * x[j];
    if (r > 0.0)
      v[4] += lv[j] * r;
    else if (r < 0.0)
      v[4] += uv[j] * r;
    v[5] += c[j] * c[j];
  }
  block_sum<7>(v, red);
  mx0 = warp_max(mx0);
  mx1 = warp_max(mx1);
  if ((threadIdx.x & 31) == 0) {
    mred[threadIdx.x >> 5] = mx0;
    mred[kWarps + (threadIdx.x >> 5)] = mx1;
  }
  __syncthreads();
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      a = fmax(a, mred[w]);
      b = fmax(b, mred[kWarps + w]);
    }
    for (int k = 0; k < 7; ++k) part[k * G + blockIdx.x] = v[k];
    part[7 * G + blockIdx.x] = a;
    part[8 * G + blockIdx.x] = b;
  }
  if (!last_block_arrival(counter)) return;
  double tot[7], mxt[2];
  block_reduce_partials<7, 2>(part, G, tot, mxt, red, mred);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 7; ++k) result[k] = tot[k];
    result[7] = mxt[0];
    result[8] = mxt[1];
  }
}

std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device
// index: the address in the context current at that first call (normally the primary one).
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

int fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  set_last_error_cstr(msg, e == cudaSuccess ? nullptr : cudaGetErrorString(e));
  return code;
}

}  // namespace
}  // namespace pdlp

extern "C" int pdlp_kkt_products_noalloc(int64_t m, int64_t n, const double* c,
                                         const double* lc, const double* uc, const double* lv,
                                         const double* uv, const double* x, const double* y,
                                         const double* ax, const double* aty, void* cuda_stream,
                                         double* out) {
  using namespace pdlp;
  if (m < 0 || n < 1 || m > INT32_MAX || n > INT32_MAX)
    return fail(PDLP_INVALID_ARGUMENT,
                "pdlp_kkt_products_noalloc: need 0 <= m <= 2^31-1 and 1 <= n <= 2^31-1");
  if (!c || !lv || !uv || !x || !aty || !out || (m > 0 && (!lc || !uc || !y || !ax)))
    return fail(PDLP_INVALID_ARGUMENT, "pdlp_kkt_products_noalloc: null argument");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PDLP_CUDA_ERROR, "pdlp_kkt_products_noalloc: cudaGetDevice", e);
  if (dev < 0 || dev >= kNaMaxDevices)
    return fail(PDLP_INVALID_ARGUMENT, "pdlp_kkt_products_noalloc: device index above 63");
  double* scratch = nullptr;
  e = scratch_address(dev, &scratch);
  if (e != cudaSuccess)
    return fail(PDLP_CUDA_ERROR, "pdlp_kkt_products_noalloc: cudaGetSymbolAddress", e);
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(PDLP_CUDA_ERROR, "pdlp_kkt_products_noalloc: SM count", e);
  const int64_t need = (std::max(m, n) + kThreads - 1) / kThreads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, std::min(4 * sms, kNaCtas)));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the arrival counter must start at zero; everything else is overwritten
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNaSums * kNaCtas + kNaSums);
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return fail(PDLP_CUDA_ERROR, "pdlp_kkt_products_noalloc: clear counter", e);
  k_kkt_products<<<grid, kThreads, 0, s>>>(c, lc, uc, lv, uv, x, y, ax, aty, m, n, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PDLP_CUDA_ERROR, "pdlp_kkt_products_noalloc: launch", e);
  double r[kNaSums];
  e = cudaMemcpyAsync(r, scratch + kNaSums * kNaCtas, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(PDLP_CUDA_ERROR, "pdlp_kkt_products_noalloc: result copy", e);
  // same measures and order as pdlp_kkt
  const double pres2 = std::sqrt(r[0]), dres2 = std::sqrt(r[1]);
  const double pobj = r[2], dobj = r[3] + r[4];
  const double rel_p = pres2 / (1.0 + std::sqrt(r[6]));
  const double rel_d = dres2 / (1.0 + std::sqrt(r[5]));
  const double rel_g = std::fabs(pobj - dobj) / (1.0 + std::fabs(pobj) + std::fabs(dobj));
  const double den = std::fabs(pobj) + std::fabs(dobj);
  out[0] = std::max(rel_p, std::max(rel_d, rel_g));
  out[1] = rel_p;
  out[2] = rel_d;
  out[3] = rel_g;
  out[4] = pres2;
  out[5] = dres2;
  out[6] = r[7];
  out[7] = r[8];
  out[8] = pobj;
  out[9] = dobj;
  out[10] = den > 0.0 ? std::fabs(pobj - dobj) / den : 0.0;
  return 0;
}
