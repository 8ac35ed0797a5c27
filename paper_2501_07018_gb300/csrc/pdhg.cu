// The PDHG iteration on the GPU (Sec. 2 Eq. (3), Algorithm 2, the running average of
// Algorithm 1), as three kernels per step attempt:
//   k_primal          x' = proj_X(x - tau (c - A'y))                       Eq. (3a)
//   k_spmv<kEpiDual>  A x', then per row y' = yhat - proj_[-s uc,-s lc](yhat),
//                     yhat = y - sigma (2 A x' - A x)                       Eq. (3b)
//                     + the step-size sums and, in the last CTA, the accept test
//   k_spmv<kEpiAverage>  A'y' and the running sums of eta * (x, y, Ax, A'y)
// Both sparse products share one engine over the SELL-32 layout of problem.cuh: a
// warp owns a slice of 32 rows of nearly equal length (rows are numbered by length),
// one row per lane; it streams the slice's entries k-major (coalesced), keeps a batch
// of loads and gathers in flight, accumulates its row with fused multiply-adds in
// entry order (deterministic) and applies the row epilogue with operands prefetched
// when the slice started.  Every FP64 instruction thus runs with all 32 lanes active,
// which matters on GB300 where the FP64 pipe is narrow.  Long rows go in chunks.
#include <algorithm>
#include <atomic>

#include "pdhg.cuh"

namespace pdlp {

__device__ __forceinline__ int64_t gtid2() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride2() { return (int64_t)gridDim.x * blockDim.x; }

// Monotone integer key of a non-NaN double: signed comparison of the keys orders the
// values like IEEE comparison (with -0 < +0).  Clamping doubles through the integer
// pipe keeps the scarce FP64 pipe of GB300 for arithmetic.
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// Sign tests of a non-NaN double on the integer pipe: v < 0 (-0 excluded) and v > 0.
__device__ __forceinline__ bool neg_strict(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && b != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool pos_strict(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool neg_strict(float v) { return v < 0.0f; }
__device__ __forceinline__ bool pos_strict(float v) { return v > 0.0f; }

template <class T>
__device__ __forceinline__ T clampv(T v, T lo, T hi);
template <>
__device__ __forceinline__ double clampv<double>(double v, double lo, double hi) {
  const long long kv = dkey(v);
  return kv < dkey(lo) ? lo : (kv > dkey(hi) ? hi : v);
}
template <>
__device__ __forceinline__ float clampv<float>(float v, float lo, float hi) {
  return fminf(fmaxf(v, lo), hi);
}

// Accumulator type of the per-lane step-size sums: FP64 for the FP64 path, FP32 for
// FP32 bulk (converted to FP64 for the cross-lane reduction).
template <class T>
struct AccT {
  using type = double;
};
template <>
struct AccT<float> {
  using type = float;
};

// ---------------------------------------------------------------------------
// Eq. (3a)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kThreads) k_primal(IterBuffers<T> b, DevState* st, double* part) {
  __shared__ double red[kWarps];
  const int cur = st->cur;
  const bool err = st->error != 0;
  const double eta = st->eta, omega = st->omega;
  using A = typename AccT<T>::type;
  A lacc = (A)0;
  if (!err) {
    const T tau = (T)(eta / omega);
    const T* __restrict__ x = b.X[cur];
    const T* __restrict__ aty = b.ATY[cur];
    const T* __restrict__ c = b.c;
    const T* __restrict__ lv = b.lv;
    const T* __restrict__ uv = b.uv;
    T* __restrict__ xn = b.X[cur ^ 1];
    constexpr int U = 4;
    const int64_t stride = gstride2();
    for (int64_t j0 = gtid2(); j0 < b.n; j0 += U * stride) {
      T xo[U], g[U], lo[U], hi[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = j0 + u * stride;
        if (j < b.n) {
          xo[u] = x[j];
          g[u] = c[j] - aty[j];
          lo[u] = lv[j];
          hi[u] = uv[j];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = j0 + u * stride;
        if (j < b.n) {
          const T v = clampv<T>(xo[u] - tau * g[u], lo[u], hi[u]);
          xn[j] = v;
          const A d = (A)v - (A)xo[u];
          lacc = fma(d, d, lacc);
        }
      }
    }
  }
  double acc[1] = {(double)lacc};
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

// ---------------------------------------------------------------------------
// tiled SpMV engine with fused row epilogues
// ---------------------------------------------------------------------------
template <class T>
struct SpmvArgs {
  Mat<T> M;
  const T* src;  // gathered vector
  T* dst;        // plain product output
  IterBuffers<T> b;
  DevState* st;
  const double* part_primal;
  int grid_primal;
  double* part_dual;
  unsigned int* counter;
  StepTable tab;
};

// Per-launch scalars and pointers every CTA reads once (kept in registers).
template <class T>
struct EpiCtx {
  int cur;
  T sigma;    // kEpiDual
  T eta_acc;  // kEpiAverage
  const T* src;
  T* out0;        // plain: dst; dual: A x'; average: A'y'
  T* out1;        // dual: y'
  const T* in0;   // dual: A x; average: x'
  const T* in1;   // dual: y
  const T* lo;    // dual: lc
  const T* hi;    // dual: uc
  T* acc0;        // average: S x
  T* acc1;        // average: S A'y
};

// Epilogue operands of one row, loaded before its product is formed.
template <class T>
struct EpiIn {
  T a, b, c, d;
};

template <class T, int EPI>
__device__ __forceinline__ EpiIn<T> load_epi(const EpiCtx<T>& e, int64_t row) {
  EpiIn<T> r;
  if (EPI == kEpiDual) {
    r.a = e.in0[row];
    r.b = e.in1[row];
    r.c = e.lo[row];
    r.d = e.hi[row];
  } else if (EPI == kEpiAverage) {
    r.a = e.in0[row];
    r.b = e.acc0[row];
    r.c = e.acc1[row];
    r.d = (T)0;
  } else {
    r.a = r.b = r.c = r.d = (T)0;
  }
  return r;
}

// Row epilogue.  Accumulates the two step-size contributions for kEpiDual.
template <class T, int EPI, class A>
__device__ __forceinline__ void row_epilogue(const EpiCtx<T>& e, const EpiIn<T>& in, int64_t row,
                                             T v, A& c0, A& c1) {
  if (EPI == kEpiPlain) {
    e.out0[row] = v;
  } else if (EPI == kEpiDual) {
    const T axo = in.a, yo = in.b;
    const T q = (T)2 * v - axo;
    const T yh = yo - e.sigma * q;
    // Sec. 2's case analysis of Eq. (3b): y' = yh + sigma uc if that is negative,
    // yh + sigma lc if that is positive, else 0 (a free row gives +-inf and lands on
    // 0); one rounding each and exact in sign
    const T tu = fma(e.sigma, in.d, yh);
    const T tl = fma(e.sigma, in.c, yh);
    const T yn = neg_strict(tu) ? tu : (pos_strict(tl) ? tl : (T)0);
    e.out0[row] = v;
    e.out1[row] = yn;
    const A dy = (A)yn - (A)yo;
    const A dax = (A)v - (A)axo;
    c0 = fma(dy, dy, c0);
    c1 = fma(dy, dax, c1);
  } else {
    e.out0[row] = v;
    e.acc0[row] = in.b + e.eta_acc * in.a;
    e.acc1[row] = in.c + e.eta_acc * v;
  }
}

constexpr int kSpmvWarps = 4;
constexpr int kSpmvThreads = 32 * kSpmvWarps;
#ifndef PDLP_SPMV_BATCH
#define PDLP_SPMV_BATCH 8
#endif
#ifndef PDLP_SPMV_FBATCH
#define PDLP_SPMV_FBATCH 8
#endif
// entries per lane whose loads and gathers are in flight together
template <class T>
__host__ __device__ constexpr int batch_of() {
  return sizeof(T) == 8 ? PDLP_SPMV_BATCH : PDLP_SPMV_FBATCH;
}
#ifndef PDLP_SPMV_GRAB
#define PDLP_SPMV_GRAB 2
#endif
#ifndef PDLP_SPMV_DYNAMIC
#define PDLP_SPMV_DYNAMIC 1
#endif
constexpr int kGrab = PDLP_SPMV_GRAB;  // items taken per visit of the dynamic work queue

// CTAs per SM the register budget must allow (8 = 32 warps): the gathers need the
// warps in flight to cover their latency
#ifndef PDLP_SPMV_MINB
#define PDLP_SPMV_MINB(T) 8
#endif

// Persistent kernel over work items: items [0, nchunks) are chunks of the long rows,
// the rest are SELL slices, in decreasing order of size.  kEpiDual assigns items
// statically (warp w of W takes w, w + W, ...) because its step-size sums are
// accumulated per warp and must not depend on timing; the other epilogues write
// per-row results only and take items from a work queue (largest first), which
// balances the power-law mix of item sizes.
template <class T, int EPI>
__global__ void __launch_bounds__(kSpmvThreads, PDLP_SPMV_MINB(T)) k_spmv(SpmvArgs<T> a) {
  __shared__ double red[2 * kSpmvWarps];
  using A = typename AccT<T>::type;

  EpiCtx<T> e;
  e.sigma = (T)0;
  e.eta_acc = (T)0;
  e.out1 = nullptr;
  e.in0 = e.in1 = e.lo = e.hi = nullptr;
  e.acc0 = e.acc1 = nullptr;
  if (EPI == kEpiPlain) {
    e.cur = 0;
    e.src = a.src;
    e.out0 = a.dst;
  } else {
    const int cur = a.st->cur;
    e.cur = cur;
    const bool err = a.st->error != 0;
    if (EPI == kEpiDual) {
      if (err) return;  // every CTA returns: the arrival counter stays consistent
      e.sigma = (T)(a.st->eta * a.st->omega);
      e.src = a.b.X[cur ^ 1];
      e.out0 = a.b.AX[cur ^ 1];
      e.out1 = a.b.Y[cur ^ 1];
      e.in0 = a.b.AX[cur];
      e.in1 = a.b.Y[cur];
      e.lo = a.b.lc;
      e.hi = a.b.uc;
    } else {
      if (err || a.st->accepted == 0) return;
      e.eta_acc = (T)a.st->eta_acc;
      e.src = a.b.Y[cur];
      e.out0 = a.b.ATY[cur];
      e.in0 = a.b.X[cur];
      e.acc0 = a.b.Sx;
      e.acc1 = a.b.SATy;
      // the m-side of the running sums (Algorithm 1): Sy += eta y', SAx += eta A x'
      const T* __restrict__ y = a.b.Y[cur];
      const T* __restrict__ ax = a.b.AX[cur];
      T* __restrict__ sy = a.b.Sy;
      T* __restrict__ sax = a.b.SAx;
      const T w = e.eta_acc;
      for (int64_t i = gtid2(); i < a.b.m; i += gstride2()) {
        sy[i] += w * y[i];
        sax[i] += w * ax[i];
      }
    }
  }

  const Mat<T>& M = a.M;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const T* __restrict__ src = e.src;
  A c0 = (A)0, c1 = (A)0;
  const int64_t items = M.nchunks + M.nslices;
  const int64_t W = (int64_t)gridDim.x * kSpmvWarps;
  constexpr bool kDynamic = PDLP_SPMV_DYNAMIC && EPI != kEpiDual;
  int64_t it = kDynamic ? 0 : (int64_t)blockIdx.x * kSpmvWarps + wib;
  int64_t grab_end = 0;
  for (;;) {
    if (kDynamic) {
      if (it >= grab_end) {
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(&M.sched[0], (unsigned int)kGrab);
        base = __shfl_sync(0xffffffffu, base, 0);
        it = base;
        grab_end = (int64_t)base + kGrab;
      }
      if (it >= items) break;
    } else if (it >= items) {
      break;
    }
    if (it >= M.nchunks) {
      // one SELL slice: 32 rows, one per lane, entries k-major
      const int64_t sl = it - M.nchunks;
      const int64_t row = (int64_t)M.R0 + 32 * sl + lane;
      const bool own = row < M.rows;
      EpiIn<T> ein{};
      if (own) ein = load_epi<T, EPI>(e, row);
      const int L = M.slice_len[sl];
      const int32_t* __restrict__ cp = M.sell_col + M.slice_ptr[sl] + lane;
      const T* __restrict__ vp = M.sell_val + M.slice_ptr[sl] + lane;
      // the matrix is streamed with evict-first loads (ld.global.cs), so that L1 and L2
      // keep the gathered vector; two independent FMA chains (even / odd entries) for
      // instruction-level parallelism
      T acc_e = (T)0, acc_o = (T)0;
      constexpr int kBatch = batch_of<T>();
      for (int k0 = 0; k0 < L; k0 += kBatch) {
        int cr[kBatch];
        T vr[kBatch], xr[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const bool in = k0 + u < L;
          cr[u] = in ? __ldcs(cp + 32 * (k0 + u)) : 0;
          vr[u] = in ? __ldcs(vp + 32 * (k0 + u)) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) xr[u] = (k0 + u < L) ? src[cr[u]] : (T)0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          if (k0 + u < L) {
            if (u & 1)
              acc_o = fma(vr[u], xr[u], acc_o);
            else
              acc_e = fma(vr[u], xr[u], acc_e);
          }
        }
      }
      const T acc = acc_e + acc_o;
      if (own) row_epilogue<T, EPI, A>(e, ein, row, acc, c0, c1);
    } else {
      // one chunk of a long row (CSR)
      const int64_t ci = it;
      const int64_t row = M.chunk_owner[ci];
      const int64_t first = M.chunk_ptr[row];
      const int64_t nch = M.chunk_ptr[row + 1] - first;
      const int64_t rb = M.row_ptr[row], re = M.row_ptr[row + 1];
      const int64_t pb = rb + (ci - first) * kChunk;
      const int64_t pe = min(pb + (int64_t)kChunk, re);
      const int32_t* __restrict__ colp = M.col;
      const T* __restrict__ valp = M.val;
      T acc = (T)0;
#pragma unroll 4
      for (int64_t p = pb + lane; p < pe; p += 32) acc = fma(__ldcs(valp + p), src[__ldcs(colp + p)], acc);
      const double part = warp_sum((double)acc);
      // a row of one chunk is finished here; otherwise the last of its chunks to
      // arrive adds the chunk sums (lane q holds chunk q; fixed tree over lanes)
      bool finish = nch == 1;
      double sum = part;
      if (!finish) {
        unsigned prev = 0;
        if (lane == 0) {
          M.long_part[ci] = part;
          __threadfence();
          prev = atomicAdd(&M.long_cnt[row], 1u);
        }
        prev = __shfl_sync(0xffffffffu, prev, 0);
        finish = prev == (unsigned)(nch - 1);
        if (finish) {
          __threadfence();
          double v = 0.0;
          for (int64_t q = lane; q < nch; q += 32) v += __ldcg(M.long_part + first + q);
          sum = warp_sum(v);
          if (lane == 0) M.long_cnt[row] = 0u;
        }
      }
      if (finish && lane == 0) {
        A d0 = (A)0, d1 = (A)0;
        const EpiIn<T> ein = load_epi<T, EPI>(e, row);
        row_epilogue<T, EPI, A>(e, ein, row, (T)sum, d0, d1);
        if (EPI == kEpiDual) {
          M.long_contrib[2 * row] = (double)d0;
          M.long_contrib[2 * row + 1] = (double)d1;
        }
      }
    }
    it += kDynamic ? 1 : W;
  }

  if (kDynamic) {
    // the last CTA out resets the queue for the next launch on the stream (every
    // warp's last visit precedes its CTA's arrival)
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&M.sched[1], 1u);
      if (prev == gridDim.x - 1) {
        M.sched[0] = 0u;
        M.sched[1] = 0u;
        __threadfence();
      }
    }
    return;
  }
  if (EPI != kEpiDual) return;  // only the A-side product feeds Algorithm 2

  // step-size sums: per CTA, then the last CTA reduces in fixed order and decides
  double v[2] = {(double)c0, (double)c1};
  block_sum<2, kSpmvWarps>(v, red);
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    a.part_dual[blockIdx.x] = v[0];
    a.part_dual[G + blockIdx.x] = v[1];
  }
  if (!last_block_arrival(a.counter)) return;
  // the per-CTA partials of both kernels and the long rows' contributions, read from
  // L2 four strides at a time (one latency per four loads), fixed-order sums
  double t5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // dx2, dy2, inter, long dy2, long inter
  {
    const int64_t n0 = a.grid_primal, n1 = G, n2 = M.R0;
    const int64_t nmax = max(n0, max(n1, n2));
    const int64_t B = blockDim.x;
    for (int64_t i0 = threadIdx.x; i0 < nmax; i0 += 4 * B) {
      double q[5][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + u * B;
        q[0][u] = i < n0 ? __ldcg(a.part_primal + i) : 0.0;
        q[1][u] = i < n1 ? __ldcg(a.part_dual + i) : 0.0;
        q[2][u] = i < n1 ? __ldcg(a.part_dual + G + i) : 0.0;
        q[3][u] = i < n2 ? __ldcg(M.long_contrib + 2 * i) : 0.0;
        q[4][u] = i < n2 ? __ldcg(M.long_contrib + 2 * i + 1) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < 5; ++j) t5[j] += q[j][u];
    }
  }
  __shared__ double red5[5 * kSpmvWarps];
  block_sum<5, kSpmvWarps>(t5, red5);
  if (threadIdx.x != 0) return;
  const double dx2 = t5[0];
  const double dy2 = t5[1] + t5[3];
  const double inter = t5[2] + t5[4];
  DevState* s = a.st;
  const double omega = s->omega, eta = s->eta;
  // Algorithm 2 with the interaction taken in magnitude (Eq. (5) for K = -A)
  const double num = omega * dx2 + dy2 / omega;
  const double den = 2.0 * fabs(inter);
  const double eta_bar = den > 0.0 ? num / den : INFINITY;
  double red_f, grow_f;
  if (s->k < a.tab.len) {
    red_f = a.tab.f[2 * s->k];
    grow_f = a.tab.f[2 * s->k + 1];
  } else {
    const double kf = (double)(s->k + 2);
    red_f = 1.0 - pow(kf, -0.3);
    grow_f = 1.0 + pow(kf, -0.6);
  }
  const double eta_new = s->fixed_eta > 0.0 ? s->fixed_eta : fmin(red_f * eta_bar, grow_f * eta);
  s->attempts += 1;
  s->last_dx2 = dx2;
  s->last_dy2 = dy2;
  s->last_inter = inter;
  s->last_eta_bar = eta_bar;
  const bool fixed = s->fixed_eta > 0.0;  // constant-step PDHG: accept as is
  if (!(isfinite(eta_new) && isfinite(num))) {
    s->error = 1;
    s->accepted = 0;
  } else if (fixed || eta <= eta_bar) {
    s->eta_acc = eta;
    s->eta_hat = eta_new;
    s->eta = eta_new;
    s->cur ^= 1;
    s->k += 1;
    s->t += 1;
    s->W += eta;
    s->accepted = 1;
    s->retries = 0;
  } else {
    s->eta = eta_new;
    s->accepted = 0;
    s->retries += 1;
    s->rejected += 1;
    if (s->retries >= s->max_retries) s->error = 2;
  }
}

__global__ void k_step_table(double* f, int64_t len) {
  for (int64_t k = gtid2(); k < len; k += gstride2()) {
    const double kf = (double)(k + 2);
    f[2 * k] = 1.0 - pow(kf, -0.3);
    f[2 * k + 1] = 1.0 + pow(kf, -0.6);
  }
}

void fill_step_table(double* f, int64_t len, cudaStream_t s) {
  const int64_t need = (len + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 8));
  k_step_table<<<grid, 256, 0, s>>>(f, len);
  PDLP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class T, int EPI>
static int spmv_grid_impl(const Mat<T>& M) {
  static std::atomic<int> occ_cache{0};  // same value from every thread
  int occ = occ_cache.load(std::memory_order_relaxed);
  if (occ == 0) {
    PDLP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv<T, EPI>, kSpmvThreads, 0));
    if (occ < 1) occ = 1;
    occ_cache.store(occ, std::memory_order_relaxed);
  }
  const int64_t items = (M.work_items() + kSpmvWarps - 1) / kSpmvWarps;  // warps -> CTAs
  const int64_t cap = (int64_t)num_sms() * occ;
  return (int)std::max<int64_t>(1, std::min(items, cap));
}

template <class T>
int spmv_grid(const Mat<T>& M, int epi) {
  if (epi == kEpiDual) return spmv_grid_impl<T, kEpiDual>(M);
  if (epi == kEpiAverage) return spmv_grid_impl<T, kEpiAverage>(M);
  return spmv_grid_impl<T, kEpiPlain>(M);
}

int primal_grid(int64_t n) {
  // resident CTAs only; each thread keeps four elements' loads in flight
  const int64_t need = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 8));
}

template <class T>
void launch_primal(const IterBuffers<T>& b, DevState* st, double* part, int grid, cudaStream_t s) {
  k_primal<T><<<grid, kThreads, 0, s>>>(b, st, part);
  PDLP_LAUNCH_CHECK();
}

template <class T>
void launch_spmv_dual(const Mat<T>& A, const IterBuffers<T>& b, DevState* st,
                      const double* part_primal, int grid_primal, double* part_dual,
                      unsigned int* counter, StepTable tab, int grid, cudaStream_t s) {
  SpmvArgs<T> a{};
  a.tab = tab;
  a.M = A;
  a.b = b;
  a.st = st;
  a.part_primal = part_primal;
  a.grid_primal = grid_primal;
  a.part_dual = part_dual;
  a.counter = counter;
  k_spmv<T, kEpiDual><<<grid, kSpmvThreads, 0, s>>>(a);
  PDLP_LAUNCH_CHECK();
}

template <class T>
void launch_spmv_avg(const Mat<T>& AT, const IterBuffers<T>& b, DevState* st, int grid,
                     cudaStream_t s) {
  SpmvArgs<T> a{};
  a.M = AT;
  a.b = b;
  a.st = st;
  k_spmv<T, kEpiAverage><<<grid, kSpmvThreads, 0, s>>>(a);
  PDLP_LAUNCH_CHECK();
}

template <class T>
void launch_spmv_plain(const Mat<T>& M, const T* src, T* dst, int grid, cudaStream_t s) {
  SpmvArgs<T> a{};
  a.M = M;
  a.src = src;
  a.dst = dst;
  k_spmv<T, kEpiPlain><<<grid, kSpmvThreads, 0, s>>>(a);
  PDLP_LAUNCH_CHECK();
}

#define PDLP_INST(T)                                                                        \
  template int spmv_grid<T>(const Mat<T>&, int);                                            \
  template void launch_primal<T>(const IterBuffers<T>&, DevState*, double*, int, cudaStream_t); \
  template void launch_spmv_dual<T>(const Mat<T>&, const IterBuffers<T>&, DevState*,        \
                                    const double*, int, double*, unsigned int*, StepTable,  \
                                    int, cudaStream_t);                                     \
  template void launch_spmv_avg<T>(const Mat<T>&, const IterBuffers<T>&, DevState*, int,    \
                                   cudaStream_t);                                           \
  template void launch_spmv_plain<T>(const Mat<T>&, const T*, T*, int, cudaStream_t);
PDLP_INST(double)
PDLP_INST(float)

}  // namespace pdlp
