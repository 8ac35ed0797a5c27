// Persistent batch of unrolled PDHG and its adjoint: one launch, one CTA per LP at a
// time (LPs taken from a device queue).  Per LP, the same computation as
// pdlp_unrolled_pdhg (adjoint.cu): K steps of Eq. (3) with fixed steps from
// (proj_X(0), 0), checkpoints every C steps, and -- with an upstream gradient -- the
// reverse pass that recomputes each segment from its checkpoint and walks it backwards.
//
// The LPs of a differentiable batch are small, so a CTA keeps an LP's whole forward
// state in shared memory and every step is three phases separated by CTA barriers:
//   columns     x <- clamp(x - tau (c - A'y), lv, uv)                     (in place)
//   A x         row epilogue: yh = y - sigma (2 A x - Ax_old),
//               y <- yh - clamp(yh, -sigma uc, -sigma lc), Ax <- A x      (in place)
//   A'y         row epilogue: A'y <- A'y
// the products gathering x and y from shared memory.  A reverse step is the row
// pre-step (which branches of the dual clamp were open), A'byh with the column adjoint
// fused into its row epilogue, and A bu with the row update fused; the gathered adjoints
// byh and bu sit in shared memory.  Each row's sum runs over its entries in SELL order
// with the even/odd chains of pdhg.cu's product, and rows of up to 4096 entries are
// summed as there, so the arithmetic is that of the single-call path.
#include <algorithm>

#include "unroll_batch.cuh"

namespace pdlp {
namespace {

constexpr int kNT = 1024;  // threads per CTA
constexpr int kB = 4;      // entries per lane in flight (64 registers per thread)
constexpr size_t kSmemMax = 200 * 1024;

// the clamp of the forward steps (fmin / fmax, as in adjoint.cu)
template <class T>
__device__ __forceinline__ T clamp_ad(T v, T lo, T hi) {
  return fmin(fmax(v, lo), hi);
}

// y = M src for the rows of M, calling epi(row, sum) once per row.  TV is the matrix
// type (the accumulation type), TS the gathered vector's.
template <class TV, class TS, class Epi>
__device__ __forceinline__ void cta_product(const Mat<TV>& M, const TS* src, const Epi& epi) {
  constexpr int NW = kNT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t R0 = M.R0;
  const int64_t items = R0 + M.nslices;
  for (int64_t it = w; it < items; it += NW) {
    if (it >= R0) {
      const int64_t sl = it - R0;
      const int64_t row = R0 + 32 * sl + lane;
      const int L = M.slice_len[sl];
      const int32_t* __restrict__ cp = M.sell_col + M.slice_ptr[sl] + lane;
      const TV* __restrict__ vp = M.sell_val + M.slice_ptr[sl] + lane;
      TV acc_e = (TV)0, acc_o = (TV)0;
      for (int k0 = 0; k0 < L; k0 += kB) {
        int cr[kB];
        TV vr[kB], xr[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const bool in = k0 + u < L;
          cr[u] = in ? __ldg(cp + 32 * (k0 + u)) : 0;
          vr[u] = in ? __ldg(vp + 32 * (k0 + u)) : (TV)0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) xr[u] = (k0 + u < L) ? (TV)src[cr[u]] : (TV)0;
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          if (k0 + u < L) {
            if (u & 1)
              acc_o = fma(vr[u], xr[u], acc_o);
            else
              acc_e = fma(vr[u], xr[u], acc_e);
          }
        }
      }
      if (row < M.rows) epi(row, acc_e + acc_o);
    } else {
      // a long row: lanes stride over its entries, then a fixed shuffle tree
      const int64_t row = it;
      const int64_t rb = M.row_ptr[row], re = M.row_ptr[row + 1];
      TV acc = (TV)0;
      for (int64_t p = rb + lane; p < re; p += 32) acc = fma(__ldg(M.val + p), (TV)src[__ldg(M.col + p)], acc);
      double sum = (double)acc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) epi(row, (TV)sum);
    }
  }
}

// the forward state of an LP in shared memory
template <class T>
struct FwdState {
  T *x, *aty, *y, *ax;
};

// one forward step of Eq. (3) on the shared state
template <class T>
__device__ void forward_step(const UnrollLP<T>& L, const FwdState<T>& z) {
  const T tau = L.tau_t, sigma = L.sigma_t;
  for (int64_t j = threadIdx.x; j < L.n; j += kNT)
    z.x[j] = clamp_ad<T>(z.x[j] - tau * (__ldg(L.c + j) - z.aty[j]), __ldg(L.lv + j), __ldg(L.uv + j));
  __syncthreads();
  cta_product<T, T>(L.A, z.x, [&](int64_t i, T v) {
    const T yh = z.y[i] - sigma * ((T)2 * v - z.ax[i]);
    z.y[i] = yh - clamp_ad<T>(yh, -sigma * __ldg(L.uc + i), -sigma * __ldg(L.lc + i));
    z.ax[i] = v;
  });
  __syncthreads();
  cta_product<T, T>(L.AT, z.y, [&](int64_t j, T v) { z.aty[j] = v; });
  __syncthreads();
}

// state k of a trajectory buffer: x, y, Ax, A'y at offsets 0, n, n+m, n+2m
template <class T>
__device__ __forceinline__ T* state_ptr(T* base, int64_t k, int64_t m, int64_t n) {
  return base + (size_t)k * 2 * (size_t)(m + n);
}

template <class T>
__device__ void save_state(const UnrollLP<T>& L, const FwdState<T>& z, T* dst) {
  const int64_t m = L.m, n = L.n;
  for (int64_t j = threadIdx.x; j < n; j += kNT) {
    dst[j] = z.x[j];
    dst[n + 2 * m + j] = z.aty[j];
  }
  for (int64_t i = threadIdx.x; i < m; i += kNT) {
    dst[n + i] = z.y[i];
    dst[n + m + i] = z.ax[i];
  }
}

template <class T>
__device__ void load_state(const UnrollLP<T>& L, const T* src, const FwdState<T>& z) {
  const int64_t m = L.m, n = L.n;
  for (int64_t j = threadIdx.x; j < n; j += kNT) {
    z.x[j] = src[j];
    z.aty[j] = src[n + 2 * m + j];
  }
  for (int64_t i = threadIdx.x; i < m; i += kNT) {
    z.y[i] = src[n + i];
    z.ax[i] = src[n + m + i];
  }
  __syncthreads();
}

// one reverse step from the states s (step i) and t (step i + 1) of the segment buffer
template <class T>
__device__ void reverse_step(const UnrollLP<T>& L, const T* s, const T* t, double* byh,
                             double* bu) {
  const int64_t m = L.m, n = L.n;
  const T tau_t = L.tau_t, sigma_t = L.sigma_t;
  const double tau = L.tau, sigma = L.sigma;
  const T* sx = s;
  const T* sy = s + n;
  const T* sax = s + n + m;
  const T* saty = s + n + 2 * m;
  const T* tax = t + n + m;
  // rows: the dual clamp's open branches; the bounds' gradients
  for (int64_t i = threadIdx.x; i < m; i += kNT) {
    const T yh = sy[i] - sigma_t * ((T)2 * tax[i] - sax[i]);
    const bool below = yh < -sigma_t * __ldg(L.uc + i), above = yh > -sigma_t * __ldg(L.lc + i);
    const double b = L.by[i];
    byh[i] = (below || above) ? b : 0.0;
    if (below) L.g[2][i] += sigma * b;
    if (above) L.g[1][i] += sigma * b;
  }
  __syncthreads();
  // q = A' byh, and per column the total adjoint of x', the primal clamp's branch, the
  // cost and bound gradients, bu, and the adjoint of x
  cta_product<double, double>(L.AT64, byh, [&](int64_t j, double q) {
    const double bxn = L.bx[j] - 2.0 * sigma * q;
    const T u = sx[j] - tau_t * (__ldg(L.c + j) - saty[j]);
    const bool lo = u < __ldg(L.lv + j), hi = u > __ldg(L.uv + j);
    const double b = (lo || hi) ? 0.0 : bxn;
    if (lo) L.g[3][j] += bxn;
    if (hi) L.g[4][j] += bxn;
    L.g[0][j] -= tau * b;
    bu[j] = b;
    L.bx[j] = sigma * q + b;
  });
  __syncthreads();
  // r = A bu, and the adjoint of y
  cta_product<double, double>(L.A64, bu, [&](int64_t i, double r) { L.by[i] = byh[i] + tau * r; });
  __syncthreads();
}

template <class T>
__device__ void run_lp(const UnrollLP<T>& L, unsigned char* dsm) {
  const int64_t m = L.m, n = L.n;
  // shared memory: x, A'y (n each), y, Ax (m each) in T; then byh (m) and bu (n) in FP64
  T* base = reinterpret_cast<T*>(dsm);
  const FwdState<T> z{base, base + n, base + 2 * n, base + 2 * n + m};
  const size_t fwd_bytes = (sizeof(T) * 2 * (size_t)(m + n) + 15) & ~(size_t)15;
  double* byh = reinterpret_cast<double*>(dsm + fwd_bytes);
  double* bu = byh + m;
  const int64_t C = L.C, K = L.K;

  // ---- forward: z_0 = (proj_X(0), 0), checkpoints every C steps ----
  for (int64_t j = threadIdx.x; j < n; j += kNT) {
    z.x[j] = clamp_ad<T>((T)0, L.lv[j], L.uv[j]);
    z.aty[j] = (T)0;
  }
  for (int64_t i = threadIdx.x; i < m; i += kNT) z.y[i] = (T)0;
  __syncthreads();
  cta_product<T, T>(L.A, z.x, [&](int64_t i, T v) { z.ax[i] = v; });
  __syncthreads();
  save_state(L, z, state_ptr(L.cp, 0, m, n));
  for (int64_t k = 1; k <= K; ++k) {
    forward_step(L, z);
    if (k % C == 0) save_state(L, z, state_ptr(L.cp, k / C, m, n));
  }
  for (int64_t j = threadIdx.x; j < n; j += kNT) L.x_out[L.perm_c[j]] = (double)z.x[j];
  for (int64_t i = threadIdx.x; i < m; i += kNT) L.y_out[L.perm_r[i]] = (double)z.y[i];
  if (!L.gx) return;

  // ---- reverse pass ----
  for (int64_t j = threadIdx.x; j < n; j += kNT) {
    L.bx[j] = L.gx[j];
    L.g[0][j] = L.g[3][j] = L.g[4][j] = 0.0;
  }
  for (int64_t i = threadIdx.x; i < m; i += kNT) {
    L.by[i] = L.gy ? L.gy[i] : 0.0;
    L.g[1][i] = L.g[2][i] = 0.0;
  }
  __syncthreads();
  for (int64_t sgi = K > 0 ? (K - 1) / C : -1; sgi >= 0; --sgi) {
    const int64_t k0 = sgi * C, steps = min(K, k0 + C) - k0;
    // recompute the segment's states from its checkpoint
    load_state(L, state_ptr(L.cp, sgi, m, n), z);
    save_state(L, z, state_ptr(L.seg, 0, m, n));
    for (int64_t i = 0; i < steps; ++i) {
      forward_step(L, z);
      save_state(L, z, state_ptr(L.seg, i + 1, m, n));
    }
    __syncthreads();
    for (int64_t i = steps - 1; i >= 0; --i)
      reverse_step(L, state_ptr(L.seg, i, m, n), state_ptr(L.seg, i + 1, m, n), byh, bu);
  }
  // x_0 = proj_X(0): the gradient reaches a bound where the start sits on it; infinite
  // bounds get 0; then the caller's numbering
  for (int64_t j = threadIdx.x; j < n; j += kNT) {
    const T lv = L.lv[j], uv = L.uv[j];
    if ((T)0 < lv) L.g[3][j] += L.bx[j];
    if ((T)0 > uv) L.g[4][j] += L.bx[j];
    if (!isfinite(lv)) L.g[3][j] = 0.0;
    if (!isfinite(uv)) L.g[4][j] = 0.0;
  }
  for (int64_t i = threadIdx.x; i < m; i += kNT) {
    if (!isfinite(L.lc[i])) L.g[1][i] = 0.0;
    if (!isfinite(L.uc[i])) L.g[2][i] = 0.0;
  }
  __syncthreads();
  const int64_t len[5] = {n, m, m, n, n};
  for (int q = 0; q < 5; ++q) {
    if (!L.gout[q]) continue;
    const int32_t* perm = (q == 1 || q == 2) ? L.perm_r : L.perm_c;
    for (int64_t i = threadIdx.x; i < len[q]; i += kNT) L.gout[q][perm[i]] = L.g[q][i];
  }
}

template <class T>
__global__ void __launch_bounds__(kNT, 1)
    k_unroll_batch(const UnrollLP<T>* lps, const int32_t* order, int count, unsigned int* queue) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ UnrollLP<T> lp;
  __shared__ int s_next;
  static_assert(sizeof(UnrollLP<T>) % sizeof(int) == 0, "descriptor size");
  for (;;) {
    if (threadIdx.x == 0) s_next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int q = s_next;
    if (q >= count) break;
    {
      const int words = (int)(sizeof(UnrollLP<T>) / sizeof(int));
      const int* srcw = reinterpret_cast<const int*>(lps + order[q]);
      int* dstw = reinterpret_cast<int*>(&lp);
      for (int w = threadIdx.x; w < words; w += kNT) dstw[w] = srcw[w];
    }
    __syncthreads();
    run_lp(lp, dsm);
    __syncthreads();
  }
}

}  // namespace

size_t unroll_smem_need(int64_t m, int64_t n, size_t t_bytes) {
  return ((t_bytes * 2 * (size_t)(m + n) + 15) & ~(size_t)15) + sizeof(double) * (size_t)(m + n);
}
size_t unroll_smem_max() { return kSmemMax; }

template <class T>
int unroll_resident_ctas() {
  static int cached = 0;
  if (cached) return cached;
  PDLP_CUDA_CHECK(cudaFuncSetAttribute(k_unroll_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSmemMax));
  int occ = 0;
  PDLP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_unroll_batch<T>, kNT, kSmemMax));
  if (occ < 1) throw PdlpError(-3, "unrolled batch kernel does not fit on an SM");
  cached = occ * num_sms();
  return cached;
}

template <class T>
void launch_unroll_batch(const UnrollLP<T>* lps, const int32_t* order, int count,
                         unsigned int* queue, int ctas, cudaStream_t s) {
  unroll_resident_ctas<T>();
  k_unroll_batch<T><<<ctas, kNT, kSmemMax, s>>>(lps, order, count, queue);
  PDLP_LAUNCH_CHECK();
}

template int unroll_resident_ctas<double>();
template int unroll_resident_ctas<float>();
template void launch_unroll_batch<double>(const UnrollLP<double>*, const int32_t*, int,
                                          unsigned int*, int, cudaStream_t);
template void launch_unroll_batch<float>(const UnrollLP<float>*, const int32_t*, int,
                                         unsigned int*, int, cudaStream_t);

}  // namespace pdlp
