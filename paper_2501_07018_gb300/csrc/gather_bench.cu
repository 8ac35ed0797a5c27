// The random-gather ceiling of this GPU for the access pattern of the fused SpMV kernels
// (pdhg.cu): a synthetic SELL-32 product y = M t, every entry gathering one element of a
// table t at a random index.  The paper names memory bandwidth as the bound of its
// parallel A x / A'y (Sec. 5, "Multithreading"); on GB300 the random gathers of the
// vector bound the products before DRAM does, and this measures by how much.
//
// Three ways to gather, each over the same data:
//   method 0  LSU: one ld.global per entry, 8 in flight per lane (the SpMV kernels' way);
//   method 1  TMA: cp.async.bulk.tensor tile::gather4 -- four 32-byte rows of the table
//             (viewed as [len/4][4]) per instruction into shared memory, completion on an
//             mbarrier, double-buffered per warp;
//   method 2  half the warps of each CTA gather through the LSU, half through TMA.
// Column indices are uniform on [0, len), or those of the entries of a matrix with
// power-law column degrees, columns numbered by decreasing degree (as the solver's
// renumbering leaves them).  The data are
// generated on the device from a counter-based hash; nothing here is part of the solver.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "pdlp.h"
#include "problem.cuh"
#include "tma.cuh"

namespace pdlp {
namespace {

constexpr int kGbWarps = 8;                 // warps per CTA of the gather kernels
constexpr int kGbThreads = 32 * kGbWarps;
constexpr int kGbBatch = 8;                 // LSU entries in flight per lane
constexpr uint32_t kSpinLimit = 1u << 22;   // bounded mbarrier waits

// SplitMix64 finaliser: a counter-based generator for the synthetic indices and values
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double unit(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }

// Entry e: column uniform on [0, len) (s <= 0), or, for s > 1, the column of a matrix
// whose len columns have degrees from the truncated power law P(d) ~ d^-s on [dmin,
// dmax], numbered by decreasing degree, each entry drawn with probability proportional
// to its column's degree.  Column j's degree is the law's quantile at u = 1 - (j + 1/2)
// / len, d(u) = (a + u b)^(1/(1-s)) with a = dmin^(1-s), b = dmax^(1-s) - a; the
// cumulative degree of the columns past u is len (F(1) - F(u)) with F(u) = (a + u b)^g
// / (b g), g = (2-s)/(1-s), so a uniform share of the total degree inverts in closed
// form.  Values are uniform in [-0.5, 0.5).
__global__ void k_gb_fill(int32_t* col, double* val64, float* val32, int64_t nnz, int64_t len,
                          double s, double dmin, double dmax, uint64_t seed) {
  const double a = pow(dmin, 1.0 - s), b = pow(dmax, 1.0 - s) - a, g = (2.0 - s) / (1.0 - s);
  const double F1 = pow(a + b, g) / (b * g), F0 = pow(a, g) / (b * g);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64(seed ^ (uint64_t)e);
    int64_t c;
    if (s <= 0.0) {
      c = (int64_t)(unit(h) * (double)len);
    } else {
      const double w = unit(mix64(h)) * (F1 - F0);  // degree share past the column
      const double u = (pow((F1 - w) * b * g, 1.0 / g) - a) / b;
      c = (int64_t)((1.0 - u) * (double)len);
    }
    c = c < 0 ? 0 : (c >= len ? len - 1 : c);
    col[e] = (int32_t)c;
    const double v = unit(mix64(h ^ 0x5DEECE66DULL)) - 0.5;
    if (val64) val64[e] = v;
    if (val32) val32[e] = (float)v;
  }
}

__global__ void k_gb_table(double* t64, float* t32, int64_t len, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = unit(mix64(seed + (uint64_t)i)) - 0.5;
    if (t64) t64[i] = v;
    if (t32) t32[i] = (float)v;
  }
}

// LSU gathers of one slice (32 rows x L entries, entry k of lane l at 32 k + l)
template <class T>
__device__ __forceinline__ T gb_slice_lsu(const int32_t* __restrict__ cp, const T* __restrict__ vp,
                                          const T* __restrict__ tab, int L) {
  T acc = (T)0;
  for (int k0 = 0; k0 < L; k0 += kGbBatch) {
    int c[kGbBatch];
    T v[kGbBatch], x[kGbBatch];
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) {
      const bool in = k0 + u < L;
      c[u] = in ? __ldcs(cp + 32 * (k0 + u)) : 0;  // streamed, evict-first
      v[u] = in ? __ldcs(vp + 32 * (k0 + u)) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) x[u] = (k0 + u < L) ? tab[c[u]] : (T)0;
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u)
      if (k0 + u < L) acc = fma(v[u], x[u], acc);
  }
  return acc;
}

// Waits for the phase with the given parity; gives up after kSpinLimit polls (error
// flag set), then polls as long again so that copies in flight land before the buffer
// is reused or the CTA exits.
__device__ __forceinline__ void gb_wait(uint64_t* bar, uint32_t parity, int* err) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > kSpinLimit) {
      atomicExch(err, 1);
      for (uint32_t again = 0; again < kSpinLimit && !mbar_try_wait(bar, parity); ++again) {
      }
      return;
    }
  }
}
// four 32-byte rows r0..r3 of the [len/4][4] view of the table into dst (128 bytes,
// 128-byte aligned); the x coordinate is 0, so every copy starts on a 32-byte boundary
__device__ __forceinline__ void tma_gather4(void* dst, const CUtensorMap* map, int r0, int r1,
                                            int r2, int r3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
      : "memory");
}

// TMA gathers of one slice: stages of four entries per lane, two buffers per warp
template <int L4>
__device__ __forceinline__ double gb_slice_tma(const int32_t* __restrict__ cp,
                                               const double* __restrict__ vp,
                                               const CUtensorMap* map, unsigned char* base,
                                               uint64_t* bars, uint32_t& ph0, uint32_t& ph1,
                                               int lane, int* err) {
  double acc = 0.0;
  int cl[4 * L4];
#pragma unroll
  for (int st = -1; st < L4; ++st) {
    const int nx = st + 1;
    if (nx < L4) {
      const int nb = nx & 1;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (lane == 0) mbar_expect_tx(&bars[nb], 32u * 128u);
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 4; ++u) cl[4 * nx + u] = __ldcs(cp + 32 * (4 * nx + u));
      tma_gather4(base + (size_t)(nb * 32 + lane) * 128, map, cl[4 * nx] >> 2,
                  cl[4 * nx + 1] >> 2, cl[4 * nx + 2] >> 2, cl[4 * nx + 3] >> 2, &bars[nb]);
    }
    if (st < 0) continue;
    const int b = st & 1;
    gb_wait(&bars[b], b ? ph1 : ph0, err);
    if (b)
      ph1 ^= 1u;
    else
      ph0 ^= 1u;
    const unsigned char* slot = base + (size_t)(b * 32 + lane) * 128;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = cl[4 * st + u];
      const double xv = *reinterpret_cast<const double*>(slot + 32 * u + 8 * (c & 3));
      acc = fma(__ldcs(vp + 32 * (4 * st + u)), xv, acc);
    }
    __syncwarp();
  }
  return acc;
}

// y = M t over SELL-32 slices of L entries per row, slices from a work queue (sched[0]
// next slice, sched[1] CTAs done; the last CTA out resets both).  Warps [0, kGbWarps -
// NT) gather through the LSU, the other NT warps through TMA (T = double only).
template <class T, int NT, int L4>
__global__ void __launch_bounds__(kGbThreads) k_gb(const __grid_constant__ CUtensorMap map,
                                                   const int32_t* __restrict__ col,
                                                   const T* __restrict__ val,
                                                   const T* __restrict__ tab, T* __restrict__ y,
                                                   int64_t nslices, int L,
                                                   unsigned int* sched, int* err) {
  extern __shared__ unsigned char gb_smem[];
  __shared__ __align__(8) uint64_t bars[kGbWarps][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool tma = w >= kGbWarps - NT;
  unsigned char* base = nullptr;
  uint32_t ph0 = 0, ph1 = 0;
  if (NT > 0 && tma) {
    const uint32_t a0 = smem_addr(gb_smem);
    unsigned char* al = gb_smem + (((a0 + 127u) & ~127u) - a0);
    base = al + (size_t)(w - (kGbWarps - NT)) * 2 * 32 * 128;
    if (lane == 0) {
      mbar_init(&bars[w][0]);
      mbar_init(&bars[w][1]);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
  }
  for (;;) {
    unsigned int sl = 0;
    if (lane == 0) sl = atomicAdd(&sched[0], 1u);
    sl = __shfl_sync(0xffffffffu, sl, 0);
    if ((int64_t)sl >= nslices) break;
    const int32_t* cp = col + (int64_t)sl * 32 * L + lane;
    const T* vp = val + (int64_t)sl * 32 * L + lane;
    T acc;
    if constexpr (NT > 0) {
      if (tma)
        acc = (T)gb_slice_tma<L4>(cp, (const double*)vp, &map, base, bars[w], ph0, ph1, lane, err);
      else
        acc = gb_slice_lsu<T>(cp, vp, tab, L);
    } else {
      acc = gb_slice_lsu<T>(cp, vp, tab, L);
    }
    y[(int64_t)sl * 32 + lane] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&sched[1], 1u) == gridDim.x - 1) {
      sched[0] = 0u;
      sched[1] = 0u;
      __threadfence();
    }
  }
}

}  // namespace
}  // namespace pdlp

namespace pdlp {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  PDLP_CUDA_CHECK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess)
    throw PdlpError(-3, "cuTensorMapEncodeTiled is not available");
  return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

// device buffers of one measurement, freed on every exit path
struct GbBuffers {
  void* p[8] = {};
  int n = 0;
  template <class U>
  U* alloc(size_t count) {
    void* q = nullptr;
    PDLP_CUDA_CHECK(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(U)));
    p[n++] = q;
    return static_cast<U*>(q);
  }
  ~GbBuffers() {
    for (int i = 0; i < n; ++i) cudaFree(p[i]);
  }
};

template <class T, int NT, int L4>
float time_gb(const CUtensorMap& map, const int32_t* col, const T* val, const T* tab, T* y,
              int64_t nslices, int L, unsigned int* sched, int* err, int reps, cudaStream_t s) {
  const size_t smem = NT > 0 ? (size_t)NT * 2 * 32 * 128 + 128 : 0;
  auto kern = k_gb<T, NT, L4>;
  PDLP_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  PDLP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGbThreads, smem));
  const int grid = num_sms() * std::max(1, occ);
  cudaEvent_t e0, e1;
  PDLP_CUDA_CHECK(cudaEventCreate(&e0));
  PDLP_CUDA_CHECK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int r = 0; r <= reps; ++r) {  // the first launch warms up
    PDLP_CUDA_CHECK(cudaEventRecord(e0, s));
    kern<<<grid, kGbThreads, smem, s>>>(map, col, val, tab, y, nslices, L, sched, err);
    PDLP_CUDA_CHECK(cudaGetLastError());
    PDLP_CUDA_CHECK(cudaEventRecord(e1, s));
    PDLP_CUDA_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    PDLP_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    if (r > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

template <class T>
double max_abs_diff(const T* a, const T* b, int64_t len) {
  double m = 0.0;
  for (int64_t i = 0; i < len; ++i) m = std::max(m, std::fabs((double)a[i] - (double)b[i]));
  return m;
}

}  // namespace
}  // namespace pdlp

extern "C" int pdlp_gather_bench(int method, int elem_bytes, int64_t table_len, int row_len,
                                 int64_t nnz, double degree_s, double dmin, double dmax,
                                 int reps, double* out) {
  using namespace pdlp;
  try {
    if (!out) throw PdlpError(-1, "pdlp_gather_bench: out is NULL");
    if (method < 0 || method > 2) throw PdlpError(-1, "pdlp_gather_bench: method must be 0, 1 or 2");
    if (elem_bytes != 8 && !(elem_bytes == 4 && method == 0))
      throw PdlpError(-1, "pdlp_gather_bench: elem_bytes must be 8 (or 4 with method 0)");
    if (table_len < 4 || table_len % 4 != 0 || table_len > ((int64_t)1 << 31))
      throw PdlpError(-1, "pdlp_gather_bench: table_len must be a multiple of 4 in [4, 2^31]");
    if (method > 0 ? (row_len != 8 && row_len != 24) : (row_len < 1 || row_len > 4096))
      throw PdlpError(-1, "pdlp_gather_bench: row_len must be 8 or 24 for TMA, 1..4096 for LSU");
    if (reps < 1 || std::isnan(degree_s) || (degree_s > 0.0 && !(degree_s > 1.0 && degree_s != 2.0 &&
                                                                  dmin >= 1.0 && dmax > dmin)))
      throw PdlpError(-1, "pdlp_gather_bench: reps >= 1; degree_s <= 0, or degree_s > 1, != 2 with "
                          "1 <= dmin < dmax");
    const int64_t nslices = nnz / (32 * (int64_t)row_len);
    if (nslices < 1 || nslices > ((int64_t)1 << 30))
      throw PdlpError(-1, "pdlp_gather_bench: nnz must hold 1 .. 2^30 slices of 32 rows");
    const int64_t ent = nslices * 32 * row_len, rows = nslices * 32;
    cudaStream_t s = nullptr;
    PDLP_CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamDone {
      cudaStream_t s;
      ~StreamDone() { cudaStreamDestroy(s); }
    } sd{s};
    GbBuffers B;
    int32_t* col = B.alloc<int32_t>(ent);
    unsigned int* sched = B.alloc<unsigned int>(2);
    int* err = B.alloc<int>(1);
    PDLP_CUDA_CHECK(cudaMemsetAsync(sched, 0, 2 * sizeof(unsigned int), s));
    PDLP_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), s));
    const int fill_grid = num_sms() * 8;
    float ms = 0.f;
    double diff = 0.0;
    if (elem_bytes == 4) {
      float* val = B.alloc<float>(ent);
      float* tab = B.alloc<float>(table_len);
      float* y = B.alloc<float>(rows);
      k_gb_fill<<<fill_grid, 256, 0, s>>>(col, nullptr, val, ent, table_len, degree_s, dmin, dmax,
                                           0x1234567ULL);
      k_gb_table<<<fill_grid, 256, 0, s>>>(nullptr, tab, table_len, 0x7654321ULL);
      PDLP_CUDA_CHECK(cudaGetLastError());
      CUtensorMap none{};
      ms = time_gb<float, 0, 1>(none, col, val, tab, y, nslices, row_len, sched, err, reps, s);
    } else {
      double* val = B.alloc<double>(ent);
      double* tab = B.alloc<double>(table_len);
      double* y = B.alloc<double>(rows);
      double* yref = B.alloc<double>(rows);
      k_gb_fill<<<fill_grid, 256, 0, s>>>(col, val, nullptr, ent, table_len, degree_s, dmin, dmax,
                                           0x1234567ULL);
      k_gb_table<<<fill_grid, 256, 0, s>>>(tab, nullptr, table_len, 0x7654321ULL);
      PDLP_CUDA_CHECK(cudaGetLastError());
      CUtensorMap map{};
      if (method > 0) {
        // the table as [table_len / 4] rows of 4 doubles (32 bytes); gather4 boxes are one
        // row high
        cuuint64_t gdim[2] = {4, (cuuint64_t)(table_len / 4)};
        cuuint64_t gstride[1] = {32};
        cuuint32_t box[2] = {4, 1};
        cuuint32_t estr[2] = {1, 1};
        const CUresult r = tensor_map_encoder()(
            &map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, tab, gdim, gstride, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw PdlpError(-3, "cuTensorMapEncodeTiled failed");
      }
      // the LSU result is the reference of the other two methods
      time_gb<double, 0, 1>(map, col, val, tab, yref, nslices, row_len, sched, err, 1, s);
      if (method == 0) {
        ms = time_gb<double, 0, 1>(map, col, val, tab, y, nslices, row_len, sched, err, reps, s);
      } else if (method == 1) {
        ms = row_len == 24
                 ? time_gb<double, kGbWarps, 6>(map, col, val, tab, y, nslices, row_len, sched, err, reps, s)
                 : time_gb<double, kGbWarps, 2>(map, col, val, tab, y, nslices, row_len, sched, err, reps, s);
      } else {
        ms = row_len == 24
                 ? time_gb<double, kGbWarps / 2, 6>(map, col, val, tab, y, nslices, row_len, sched, err, reps, s)
                 : time_gb<double, kGbWarps / 2, 2>(map, col, val, tab, y, nslices, row_len, sched, err, reps, s);
      }
      if (method > 0) {
        std::vector<double> a(rows), b(rows);
        PDLP_CUDA_CHECK(cudaMemcpy(a.data(), y, rows * sizeof(double), cudaMemcpyDeviceToHost));
        PDLP_CUDA_CHECK(cudaMemcpy(b.data(), yref, rows * sizeof(double), cudaMemcpyDeviceToHost));
        diff = max_abs_diff(a.data(), b.data(), rows);
      }
    }
    int herr = 0;
    PDLP_CUDA_CHECK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) throw PdlpError(-3, "pdlp_gather_bench: an mbarrier wait gave up");
    out[0] = 1e3 * (double)ms;
    out[1] = (double)ent / (1e-3 * (double)ms);
    out[2] = diff;
    out[3] = (double)ent;
    return 0;
  } catch (const PdlpError& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("out of host memory");
    return PDLP_OUT_OF_MEMORY;
  } catch (...) {
    set_last_error("pdlp_gather_bench: unknown error");
    return PDLP_CUDA_ERROR;
  }
}
