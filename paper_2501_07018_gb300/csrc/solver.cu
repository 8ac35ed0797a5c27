// Host driver of the library: the C ABI of include/pdlp.h.
//
// pdlp_solve runs Algorithm 1 of the paper after the preconditioning of Sec. 3.  The
// step attempts run on the device without host round trips: each attempt is three
// kernel launches (primal step; A x' with the dual step and Algorithm 2's accept
// test; A'y' with the running averages), and the device-side state decides whether
// the attempt became the new iterate.  The host only synchronises at the iteration
// counts where something else happens -- every check_period accepted iterations
// (termination and restart evaluation), and whenever restart condition (iii) can fire
// -- which it computes in advance from (k, t).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/pdlp.h"
#include "adjoint.cuh"
#include "batch.cuh"
#include "unroll_batch.cuh"
#include "gap.cuh"
#include "graph.cuh"
#include "host_logic.h"
#include "infeas.cuh"
#include "pdhg.cuh"

namespace pdlp {

// message of the last failed call of this thread, in a fixed buffer so that recording
// an error never allocates
static thread_local char g_last_error[1024] = {0};
void set_last_error(const std::string& msg) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg.c_str());
}
void set_last_error_cstr(const char* msg, const char* detail) {
  if (detail)
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", msg, detail);
  else
    std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

// Set on the worker threads of a batch: their solves launch step attempts directly.
// With many LPs in flight the GPU, not the launching thread, sets the pace, and each
// graph instantiation (taken under a driver-wide lock) is pure cost: the 128-LP batch
// took 17.6 s with per-LP graphs against 13.9 s with direct launches.
static thread_local bool t_batch_worker = false;

__device__ __forceinline__ int64_t sgi() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t sgs() { return (int64_t)gridDim.x * blockDim.x; }

static unsigned vec_grid(int64_t len) {
  const int64_t need = (len + kThreads - 1) / kThreads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 8));
}

// ---------------------------------------------------------------------------
// small vector kernels of the driver
// ---------------------------------------------------------------------------
// Preconditioned vectors (Sec. 3): c~ = D2 c, (lc~, uc~) = D1 (lc, uc), (lv~, uv~) = D2^-1 (lv, uv),
// gathered into the renumbered order (column j' is original column perm_c[j'], row i' is
// original row perm_r[i']); the unscaled vectors and the scalings are gathered too.
template <class T>
__global__ void k_prep_vectors(const double* c, const double* lc, const double* uc,
                               const double* lv, const double* uv, const double* d1,
                               const double* d2, const int32_t* perm_r, const int32_t* perm_c,
                               int64_t m, int64_t n, T* sc, T* slc, T* suc, T* slv, T* suv,
                               double* oc, double* olc, double* ouc, double* olv, double* ouv,
                               double* d1p, double* d2p, double* inv_d1, double* inv_d2) {
  for (int64_t jp = sgi(); jp < n; jp += sgs()) {
    const int64_t j = perm_c ? perm_c[jp] : jp;
    sc[jp] = (T)(d2[j] * c[j]);
    slv[jp] = (T)(lv[j] / d2[j]);
    suv[jp] = (T)(uv[j] / d2[j]);
    oc[jp] = c[j];
    olv[jp] = lv[j];
    ouv[jp] = uv[j];
    d2p[jp] = d2[j];
    inv_d2[jp] = 1.0 / d2[j];
  }
  for (int64_t ip = sgi(); ip < m; ip += sgs()) {
    const int64_t i = perm_r ? perm_r[ip] : ip;
    slc[ip] = (T)(d1[i] * lc[i]);
    suc[ip] = (T)(d1[i] * uc[i]);
    olc[ip] = lc[i];
    ouc[ip] = uc[i];
    d1p[ip] = d1[i];
    inv_d1[ip] = 1.0 / d1[i];
  }
}

// sum of squares of c and of Combine(lc, uc) (Sec. 3, "Initialization of the primal
// weights"), deterministic: per-CTA partials, fixed-order final sum
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_norms(const T* c, const T* lc, const T* uc, int64_t m, int64_t n, double* part,
            unsigned int* counter, double* out) {
  __shared__ double red[2 * kWarps];
  double v[2] = {0, 0};
  for (int64_t j = sgi(); j < n; j += sgs()) {
    const double x = c[j];
    v[0] += x * x;
  }
  for (int64_t i = sgi(); i < m; i += sgs()) {
    const double l = lc[i], u = uc[i];
    const double lf = isfinite(l) ? fabs(l) : 0.0, uf = isfinite(u) ? fabs(u) : 0.0;
    const double b = fmax(0.0, fmax(lf, uf));
    v[1] += b * b;
  }
  block_sum<2>(v, red);
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[G + blockIdx.x] = v[1];
  }
  if (!last_block_arrival(counter)) return;
  const double a = block_sum_array(part, G, red);
  const double b = block_sum_array(part + G, G, red);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

template <class T>
__global__ void k_init_point(const T* lv, const T* uv, T* x, T* y, T* aty, T* x0, T* y0,
                             int64_t m, int64_t n) {
  for (int64_t j = sgi(); j < n; j += sgs()) {
    const T lo = lv[j], hi = uv[j];
    const T v = (T)0 < lo ? lo : ((T)0 > hi ? hi : (T)0);  // proj_X(0)
    x[j] = v;
    x0[j] = v;
    aty[j] = (T)0;
  }
  for (int64_t i = sgi(); i < m; i += sgs()) {
    y[i] = (T)0;
    y0[i] = (T)0;
  }
}

template <class T>
__global__ void k_set_point(const double* xs, const double* ys, T* x, T* y, T* x0, T* y0,
                            int64_t m, int64_t n) {
  for (int64_t j = sgi(); j < n; j += sgs()) {
    x[j] = (T)xs[j];
    x0[j] = (T)xs[j];
  }
  for (int64_t i = sgi(); i < m; i += sgs()) {
    y[i] = (T)ys[i];
    y0[i] = (T)ys[i];
  }
}

template <class T>
__global__ void k_copy2(const T* a, T* a_out, int64_t na, const T* b, T* b_out, int64_t nb) {
  for (int64_t j = sgi(); j < na; j += sgs()) a_out[j] = a[j];
  for (int64_t i = sgi(); i < nb; i += sgs()) b_out[i] = b[i];
}

// x = D2 x~ (kept inside [lv, uv] against the rounding of the product), y = D1 y~,
// scattered back to the caller's numbering
template <class T>
__global__ void k_unscale(const T* x, const T* y, const double* d1, const double* d2,
                          const double* lv, const double* uv, const int32_t* perm_r,
                          const int32_t* perm_c, double* xo, double* yo, int64_t m, int64_t n,
                          bool clamp) {
  for (int64_t j = sgi(); j < n; j += sgs())
    xo[perm_c[j]] = clamp ? fmin(fmax(d2[j] * (double)x[j], lv[j]), uv[j]) : d2[j] * (double)x[j];
  for (int64_t i = sgi(); i < m; i += sgs()) yo[perm_r[i]] = d1[i] * (double)y[i];
}

template <class T>
__global__ void k_to_double2(const T* x, double* xo, int64_t n, const T* y, double* yo, int64_t m) {
  for (int64_t j = sgi(); j < n; j += sgs()) xo[j] = (double)x[j];
  for (int64_t i = sgi(); i < m; i += sgs()) yo[i] = (double)y[i];
}

__global__ void k_fill(double* v, int64_t n, double val) {
  for (int64_t i = sgi(); i < n; i += sgs()) v[i] = val;
}

// ---------------------------------------------------------------------------
// inputs
// ---------------------------------------------------------------------------
struct Inputs {
  int64_t m, n, nnz;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double *c, *lc, *uc, *lv, *uv;
  bool on_device;
};

struct DevInputs {
  int64_t* row_ptr;
  int32_t* col;
  double* val;  // modifiable copy (scaled in place)
  double *c, *lc, *uc, *lv, *uv;
};

static void copy_in(void* dst, const void* src, size_t bytes, bool on_device, cudaStream_t s) {
  if (bytes == 0) return;
  PDLP_CUDA_CHECK(cudaMemcpyAsync(dst, src, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

static void check_args(const Inputs& in) {
  if (in.m < 0 || in.n < 1) throw PdlpError(-1, "need m >= 0 and n >= 1");
  if (in.n > INT32_MAX || in.m > INT32_MAX - 1)
    throw PdlpError(-1, "m and n must fit 32-bit indices");
  if (in.nnz < 0) throw PdlpError(-1, "nnz < 0");
  if (!in.row_ptr || (in.nnz > 0 && (!in.col || !in.val)))
    throw PdlpError(-1, "null matrix array");
  if (!in.c || !in.lv || !in.uv || (in.m > 0 && (!in.lc || !in.uc)))
    throw PdlpError(-1, "null vector argument");
}

static DevInputs stage_inputs(DeviceArena& arena, const Inputs& in, cudaStream_t s) {
  DevInputs d;
  d.row_ptr = arena.alloc<int64_t>(in.m + 1);
  d.col = arena.alloc<int32_t>(in.nnz);
  d.val = arena.alloc<double>(in.nnz);
  d.c = arena.alloc<double>(in.n);
  d.lv = arena.alloc<double>(in.n);
  d.uv = arena.alloc<double>(in.n);
  d.lc = arena.alloc<double>(in.m);
  d.uc = arena.alloc<double>(in.m);
  copy_in(d.row_ptr, in.row_ptr, sizeof(int64_t) * (in.m + 1), in.on_device, s);
  copy_in(d.col, in.col, sizeof(int32_t) * in.nnz, in.on_device, s);
  copy_in(d.val, in.val, sizeof(double) * in.nnz, in.on_device, s);
  copy_in(d.c, in.c, sizeof(double) * in.n, in.on_device, s);
  copy_in(d.lv, in.lv, sizeof(double) * in.n, in.on_device, s);
  copy_in(d.uv, in.uv, sizeof(double) * in.n, in.on_device, s);
  copy_in(d.lc, in.lc, sizeof(double) * in.m, in.on_device, s);
  copy_in(d.uc, in.uc, sizeof(double) * in.m, in.on_device, s);
  return d;
}

static void validate(DeviceArena& arena, const Inputs& in, const DevInputs& d, cudaStream_t s) {
  ValidateFlags* f = arena.alloc<ValidateFlags>(1);
  PDLP_CUDA_CHECK(cudaMemsetAsync(f, 0xff, sizeof(ValidateFlags), s));
  validate_rowptr(d.row_ptr, in.m, in.nnz, f, s);
  ValidateFlags h;
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, f, sizeof(h), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  const unsigned long long none = ~0ull;
  if (h.bad_rowptr != none)
    throw PdlpError(-1, "row_ptr invalid at index " + std::to_string(h.bad_rowptr) +
                            " (need row_ptr[0]=0, nondecreasing, row_ptr[m]=nnz)");
  validate_entries(d.row_ptr, d.col, d.val, in.m, in.n, f, s);
  validate_vectors(d.c, d.lc, d.uc, d.lv, d.uv, in.m, in.n, f, s);
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, f, sizeof(h), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  if (h.bad_col != none)
    throw PdlpError(-1, "column indices of row " + std::to_string(h.bad_col) +
                            " out of range or not strictly increasing");
  if (h.bad_val != none)
    throw PdlpError(-1, "non-finite matrix value at position " + std::to_string(h.bad_val));
  if (h.bad_c != none) throw PdlpError(-1, "non-finite c at index " + std::to_string(h.bad_c));
  if (h.bad_cols != none)
    throw PdlpError(-1, "variable bounds invalid at index " + std::to_string(h.bad_cols) +
                            " (NaN, lv > uv, lv = +inf or uv = -inf)");
  if (h.bad_rows != none)
    throw PdlpError(-1, "row bounds invalid at index " + std::to_string(h.bad_rows) +
                            " (NaN, lc > uc, lc = +inf or uc = -inf)");
}

// ---------------------------------------------------------------------------
// preconditioned problem
// ---------------------------------------------------------------------------
template <class T>
struct Problem {
  int64_t m = 0, n = 0, nnz = 0;
  Mat<T> A, AT;
  double* val64 = nullptr;   // A~ values in FP64
  double* valT64 = nullptr;  // A~' values in FP64
  double *d1 = nullptr, *d2 = nullptr, *inv_d1 = nullptr, *inv_d2 = nullptr;
  T *c = nullptr, *lc = nullptr, *uc = nullptr, *lv = nullptr, *uv = nullptr;  // scaled
  DevInputs orig;  // unscaled vectors (renumbered when renumber = true)
  int32_t *perm_r = nullptr, *inv_r = nullptr, *perm_c = nullptr, *inv_c = nullptr;
  double max_abs = 0.0;
  double c_norm = 0.0, b_norm = 0.0;          // ||c||, ||Combine(lc,uc)|| of the unscaled LP
  double c_norm_s = 0.0, b_norm_s = 0.0;      // same for the scaled LP
  double* norm_part = nullptr;
  unsigned int* norm_cnt = nullptr;
  double* norm_out = nullptr;
  int launches = 0;
};

template <class V, class T>
static void norms2(Problem<T>& P, const V* c, const V* lc, const V* uc, double* out2,
                   cudaStream_t s) {
  const int G = std::max(1, std::min(num_sms() * 4, (int)vec_grid(std::max(P.m, P.n))));
  k_norms<V><<<G, kThreads, 0, s>>>(c, lc, uc, P.m, P.n, P.norm_part, P.norm_cnt, P.norm_out);
  PDLP_LAUNCH_CHECK();
  P.launches++;
  PDLP_CUDA_CHECK(cudaMemcpyAsync(out2, P.norm_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
}

// Keeps the CSR prefix of a renumbered matrix that the kernels still read after setup
// (the long rows [0, R0), processed in chunks) in arrays of `arena`, so that the full
// renumbered CSR can be freed with the other setup temporaries.
template <class T>
static void keep_long_prefix(DeviceArena& arena, Mat<T>& M, cudaStream_t s) {
  const int64_t R0 = M.R0;
  int64_t ne = 0;
  if (R0) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(&ne, M.row_ptr + R0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  }
  int64_t* rp = arena.alloc<int64_t>(R0 + 1);
  int32_t* col = arena.alloc<int32_t>(ne);
  T* val = arena.alloc<T>(ne);
  if (R0) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(rp, M.row_ptr, sizeof(int64_t) * (R0 + 1), cudaMemcpyDeviceToDevice, s));
  } else {
    PDLP_CUDA_CHECK(cudaMemsetAsync(rp, 0, sizeof(int64_t), s));
  }
  if (ne) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(col, M.col, sizeof(int32_t) * ne, cudaMemcpyDeviceToDevice, s));
    PDLP_CUDA_CHECK(cudaMemcpyAsync(val, M.val, sizeof(T) * ne, cudaMemcpyDeviceToDevice, s));
  }
  M.row_ptr = rp;
  M.col = col;
  M.val = val;
}

// The preconditioned, renumbered problem of Sec. 3 with its SELL-32 / long-row layouts.
// With `tmp`, every setup temporary (the transpose, the preconditioner's scratch, the
// renumbered CSR copies, the scratch of sorts and scans) is allocated there and freed,
// in stream order, before returning; the problem then holds the layouts, the long-row
// prefixes, the permutations and the vectors only (P.val64 / P.valT64 are null).
template <class T>
static void build_problem(DeviceArena& arena, const Inputs& in, const DevInputs& d,
                          int ruiz_iters, double pc_alpha, Problem<T>& P, cudaStream_t s,
                          bool renumber = true, DeviceArena* tmp = nullptr) {
  DeviceArena& ta = tmp ? *tmp : arena;
  P.m = in.m;
  P.n = in.n;
  P.nnz = in.nnz;
  P.orig = d;
  const int64_t m = in.m, n = in.n, nnz = in.nnz;
  P.norm_part = arena.alloc<double>(2 * num_sms() * 4);
  P.norm_cnt = arena.alloc<unsigned int>(1);
  P.norm_out = arena.alloc<double>(2);
  PDLP_CUDA_CHECK(cudaMemsetAsync(P.norm_cnt, 0, sizeof(unsigned int), s));

  // CSR of A and of its transpose (FP64 values while preconditioning)
  P.A.rows = m;
  P.A.cols = n;
  P.A.nnz = nnz;
  P.A.row_ptr = d.row_ptr;
  P.A.col = d.col;
  P.val64 = d.val;
  P.AT.rows = n;
  P.AT.cols = m;
  P.AT.nnz = nnz;
  P.AT.row_ptr = ta.alloc<int64_t>(n + 1);
  P.AT.col = ta.alloc<int32_t>(nnz);
  P.valT64 = ta.alloc<double>(nnz);
  transpose_csr(ta, d.row_ptr, d.col, d.val, m, n, nnz, P.AT.row_ptr, P.AT.col, P.valT64, s);
  P.launches += 10;

  // Sec. 3: Ruiz passes, then Pock-Chambolle
  P.d1 = (renumber ? ta : arena).alloc<double>(m);  // renumbered copies are kept below
  P.d2 = (renumber ? ta : arena).alloc<double>(n);
  double* nr = ta.alloc<double>(m);
  double* nc = ta.alloc<double>(n);
  double* fr = ta.alloc<double>(m);
  double* fs = ta.alloc<double>(n);
  k_fill<<<vec_grid(m), kThreads, 0, s>>>(P.d1, m, 1.0);
  k_fill<<<vec_grid(n), kThreads, 0, s>>>(P.d2, n, 1.0);
  PDLP_LAUNCH_CHECK();
  auto pass = [&](int kind_r, double p_r, int kind_c, double p_c) {
    row_norms(P.A.row_ptr, P.val64, m, nnz, kind_r, p_r, nr, s);
    row_norms(P.AT.row_ptr, P.valT64, n, nnz, kind_c, p_c, nc, s);
    scale_factors(nr, m, fr, P.d1, s);
    scale_factors(nc, n, fs, P.d2, s);
    scale_values(P.A.row_ptr, P.A.col, P.val64, m, nnz, fr, fs, false, s);
    scale_values(P.AT.row_ptr, P.AT.col, P.valT64, n, nnz, fr, fs, true, s);
    P.launches += 6;
  };
  for (int it = 0; it < ruiz_iters; ++it) pass(0, 0.0, 0, 0.0);
  if (pc_alpha > 0.0) {
    const double pr = 2.0 - pc_alpha, pcl = pc_alpha;
    pass(pr == 1.0 ? 1 : 2, pr, pcl == 1.0 ? 1 : 2, pcl);
  }
  P.max_abs = max_abs(ta, P.val64, nnz, s);

  if (!renumber) return;  // the preconditioner alone (original numbering)

  // renumber rows and columns by decreasing length, then the SELL-32 / long-row layout
  P.perm_r = arena.alloc<int32_t>(m);
  P.inv_r = ta.alloc<int32_t>(m);
  P.perm_c = arena.alloc<int32_t>(n);
  P.inv_c = ta.alloc<int32_t>(n);
  sort_by_length_desc(ta, P.A.row_ptr, m, P.perm_r, P.inv_r, s);
  sort_by_length_desc(ta, P.AT.row_ptr, n, P.perm_c, P.inv_c, s);
  Mat<T> A2, AT2;
  A2.rows = m;
  A2.cols = n;
  A2.nnz = nnz;
  AT2.rows = n;
  AT2.cols = m;
  AT2.nnz = nnz;
  A2.row_ptr = ta.alloc<int64_t>(m + 1);
  A2.col = ta.alloc<int32_t>(nnz);
  double* aval = ta.alloc<double>(nnz);
  AT2.row_ptr = ta.alloc<int64_t>(n + 1);
  AT2.col = ta.alloc<int32_t>(nnz);
  double* atval = ta.alloc<double>(nnz);
  permute_csr(ta, P.A.row_ptr, P.A.col, P.val64, m, P.perm_r, P.inv_c, A2.row_ptr, A2.col,
              aval, s);
  permute_csr(ta, P.AT.row_ptr, P.AT.col, P.valT64, n, P.perm_c, P.inv_r, AT2.row_ptr,
              AT2.col, atval, s);
  if (sizeof(T) == sizeof(double)) {
    A2.val = reinterpret_cast<T*>(aval);
    AT2.val = reinterpret_cast<T*>(atval);
  } else {
    A2.val = ta.alloc<T>(nnz);
    AT2.val = ta.alloc<T>(nnz);
    convert_values<T>(aval, A2.val, nnz, s);
    convert_values<T>(atval, AT2.val, nnz, s);
  }
  build_sell<T>(arena, A2, aval, s);
  build_sell<T>(arena, AT2, atval, s);
  if (tmp) {
    keep_long_prefix<T>(arena, A2, s);
    keep_long_prefix<T>(arena, AT2, s);
  }
  P.A = A2;
  P.AT = AT2;

  P.c = arena.alloc<T>(n);
  P.lv = arena.alloc<T>(n);
  P.uv = arena.alloc<T>(n);
  P.lc = arena.alloc<T>(m);
  P.uc = arena.alloc<T>(m);
  DevInputs o = d;
  o.c = arena.alloc<double>(n);
  o.lv = arena.alloc<double>(n);
  o.uv = arena.alloc<double>(n);
  o.lc = arena.alloc<double>(m);
  o.uc = arena.alloc<double>(m);
  double* d1p = arena.alloc<double>(m);
  double* d2p = arena.alloc<double>(n);
  P.inv_d1 = arena.alloc<double>(m);
  P.inv_d2 = arena.alloc<double>(n);
  k_prep_vectors<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(
      d.c, d.lc, d.uc, d.lv, d.uv, P.d1, P.d2, P.perm_r, P.perm_c, m, n, P.c, P.lc, P.uc, P.lv,
      P.uv, o.c, o.lc, o.uc, o.lv, o.uv, d1p, d2p, P.inv_d1, P.inv_d2);
  PDLP_LAUNCH_CHECK();
  P.orig = o;
  P.d1 = d1p;
  P.d2 = d2p;
  double o2[2];
  norms2<double, T>(P, o.c, o.lc, o.uc, o2, s);
  P.c_norm = std::sqrt(o2[0]);
  P.b_norm = std::sqrt(o2[1]);
  norms2<T, T>(P, P.c, P.lc, P.uc, o2, s);
  P.c_norm_s = std::sqrt(o2[0]);
  P.b_norm_s = std::sqrt(o2[1]);
  if (tmp) {
    tmp->release();  // stream-ordered: after every launch above that reads them
    P.val64 = nullptr;
    P.valT64 = nullptr;
    P.inv_r = nullptr;
    P.inv_c = nullptr;
    P.orig.row_ptr = nullptr;
    P.orig.col = nullptr;
    P.orig.val = nullptr;
  }
}

// The FP32 copy of an FP64 layout: the same row order, long-row prefix and SELL slices
// (index arrays shared with M), values rounded to FP32, and long-row scratch of its own.
// Every FP32 value build_problem<float> stores is the rounding of the FP64 value that
// build_problem<double> stores, so the copy equals the FP32 build of the same LP.
static Mat<float> narrow_layout(DeviceArena& a, const Mat<double>& M, cudaStream_t s) {
  Mat<float> F;
  F.rows = M.rows;
  F.cols = M.cols;
  F.nnz = M.nnz;
  F.row_ptr = M.row_ptr;
  F.col = M.col;
  F.R0 = M.R0;
  F.nchunks = M.nchunks;
  F.chunk_ptr = M.chunk_ptr;
  F.chunk_owner = M.chunk_owner;
  F.nslices = M.nslices;
  F.slice_ptr = M.slice_ptr;
  F.slice_len = M.slice_len;
  F.sell_col = M.sell_col;
  F.sell_entries = M.sell_entries;
  int64_t ne = 0;  // entries of the long rows [0, R0)
  if (M.R0) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(&ne, M.row_ptr + M.R0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  }
  F.val = a.alloc<float>(ne);
  convert_values<float>(M.val, F.val, ne, s);
  F.sell_val = a.alloc<float>(M.sell_entries);
  convert_values<float>(M.sell_val, F.sell_val, M.sell_entries, s);
  const int64_t R0 = M.R0;
  F.long_cnt = a.alloc<unsigned int>(R0);
  F.long_part = a.alloc<double>(M.nchunks);
  F.long_contrib = a.alloc<double>(2 * R0);
  F.sched = a.alloc<unsigned int>(2);
  PDLP_CUDA_CHECK(cudaMemsetAsync(F.long_cnt, 0, sizeof(unsigned int) * std::max<int64_t>(1, R0), s));
  PDLP_CUDA_CHECK(cudaMemsetAsync(F.long_contrib, 0, sizeof(double) * 2 * std::max<int64_t>(1, R0), s));
  PDLP_CUDA_CHECK(cudaMemsetAsync(F.sched, 0, 2 * sizeof(unsigned int), s));
  return F;
}

// The FP32 forward problem of the unrolled iteration from its FP64 build (identity
// scaling): both layouts and the five vectors narrowed, the permutations shared.
static void narrow_problem(DeviceArena& a, const Problem<double>& P, Problem<float>& F,
                           cudaStream_t s) {
  F.m = P.m;
  F.n = P.n;
  F.nnz = P.nnz;
  F.A = narrow_layout(a, P.A, s);
  F.AT = narrow_layout(a, P.AT, s);
  F.perm_r = P.perm_r;
  F.perm_c = P.perm_c;
  auto vec = [&](const double* v, int64_t len) {
    float* out = a.alloc<float>(len);
    convert_values<float>(v, out, len, s);
    return out;
  };
  F.c = vec(P.c, P.n);
  F.lv = vec(P.lv, P.n);
  F.uv = vec(P.uv, P.n);
  F.lc = vec(P.lc, P.m);
  F.uc = vec(P.uc, P.m);
}

// ---------------------------------------------------------------------------
// the solver
// ---------------------------------------------------------------------------
struct KktResult {
  double rel_kkt, rel_primal, rel_dual, rel_gap, pres2, dres2, pres_inf, dres_inf, pobj, dobj,
      paper_gap;
  double pres_rel_inf, dres_rel_inf;  // Sec. 7, Eq. (10)
};

static KktResult kkt_finish(const KktSums& k, double c_norm, double b_norm) {
  KktResult r;
  r.pres2 = std::sqrt(k.pres2);
  r.dres2 = std::sqrt(k.dres2);
  r.pres_inf = k.pres_max;
  r.dres_inf = k.dres_max;
  r.pres_rel_inf = k.pres_rel_max;
  r.dres_rel_inf = k.dres_rel_max;
  r.pobj = k.pobj;
  r.dobj = k.dobj_rows + k.dobj_cols;
  r.rel_primal = r.pres2 / (1.0 + b_norm);
  r.rel_dual = r.dres2 / (1.0 + c_norm);
  r.rel_gap = std::fabs(r.pobj - r.dobj) / (1.0 + std::fabs(r.pobj) + std::fabs(r.dobj));
  r.rel_kkt = std::max(r.rel_primal, std::max(r.rel_dual, r.rel_gap));
  const double den = std::fabs(r.pobj) + std::fabs(r.dobj);
  r.paper_gap = den > 0.0 ? std::fabs(r.pobj - r.dobj) / den : 0.0;
  return r;
}

// the primal / dual halves of the termination criteria: relative KKT (mode 0), the l_inf
// residuals of Eq. (9) (mode 1), or those residuals scaled as in Eq. (10) (mode 2)
static bool primal_ok(const KktResult& r, const pdlp_params& p) {
  if (p.termination_mode == 0) return r.rel_primal <= p.eps_rel_kkt;
  return (p.termination_mode == 2 ? r.pres_rel_inf : r.pres_inf) <= p.eps_abs_feas;
}
static bool dual_ok(const KktResult& r, const pdlp_params& p) {
  if (p.termination_mode == 0) return r.rel_dual <= p.eps_rel_kkt;
  return (p.termination_mode == 2 ? r.dres_rel_inf : r.dres_inf) <= p.eps_abs_feas;
}

static bool converged(const KktResult& r, const pdlp_params& p) {
  if (p.termination_mode == 0) return r.rel_kkt <= p.eps_rel_kkt;
  return primal_ok(r, p) && dual_ok(r, p) && r.paper_gap <= p.eps_rel_gap;
}

using Clock = std::chrono::steady_clock;
static double secs_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

struct EventTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> pending;  // (pair index, bucket)
  size_t used = 0;
  double ms[4] = {0, 0, 0, 0};
  int64_t count[4] = {0, 0, 0, 0};
  ~EventTimer() {
    for (auto e : pool) cudaEventDestroy(e);
  }
  int begin(cudaStream_t s) {
    if (!on) return -1;
    if (used + 2 > pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        PDLP_CUDA_CHECK(cudaEventCreate(&e));
        pool.push_back(e);
      }
    }
    const int idx = (int)used;
    used += 2;
    PDLP_CUDA_CHECK(cudaEventRecord(pool[idx], s));
    return idx;
  }
  void end(int idx, int bucket, cudaStream_t s) {
    if (idx < 0) return;
    PDLP_CUDA_CHECK(cudaEventRecord(pool[idx + 1], s));
    pending.push_back({idx, bucket});
  }
  void collect() {  // after a stream synchronisation
    for (auto& pr : pending) {
      float t = 0.f;
      PDLP_CUDA_CHECK(cudaEventElapsedTime(&t, pool[pr.first], pool[pr.first + 1]));
      ms[pr.second] += t;
      count[pr.second] += 1;
    }
    pending.clear();
    used = 0;
  }
};

// Termination test of a run: Algorithm 1 uses the full criteria; the phases of
// Algorithm 4 use the primal or the dual half of them.
enum Goal { kGoalOptimal = 0, kGoalPrimalFeasible = 1, kGoalDualFeasible = 2 };

static bool goal_met(const KktResult& r, const pdlp_params& p, int goal) {
  if (goal == kGoalPrimalFeasible) return primal_ok(r, p);
  if (goal == kGoalDualFeasible) return dual_ok(r, p);
  return converged(r, p);
}

enum RunOutcome { kRunDone, kRunLimit, kRunError, kRunTime, kRunPaused, kRunPrimalInf, kRunDualInf };

// One PDLP run (Algorithm 1) on the device: its iterate slots and running sums, the
// LP vectors it solves, z^{n,0}, the device-side scalars and the host-side restart
// bookkeeping.  A paused run keeps all of it and continues where it stopped.
template <class T>
struct Run {
  IterBuffers<T> b{};
  T *X0 = nullptr, *Y0 = nullptr;
  DevState* dst = nullptr;
  DevState hs{};
  int goal = kGoalOptimal;
  int64_t max_iters = 0;
  bool trace = false;
  bool infeas = false;  // infeasibility detection at the checks (normal PDLP only)
  bool started = false, have_mu_ref = false;
  double mu_ref = 0.0, mu_c_prev = INFINITY;
  int64_t k = 0, t = 0, attempts_at_last = 0;
  int64_t restarts[3] = {0, 0, 0};
};

template <class T>
__global__ void k_start_point(const T* xs, const T* ys, T* x, T* y, T* x0, T* y0, int64_t m,
                              int64_t n) {
  for (int64_t j = sgi(); j < n; j += sgs()) {
    const T v = xs ? xs[j] : (T)0;
    x[j] = v;
    x0[j] = v;
  }
  for (int64_t i = sgi(); i < m; i += sgs()) {
    const T v = ys ? ys[i] : (T)0;
    y[i] = v;
    y0[i] = v;
  }
}

// finite entries -> 0, infinite ones kept (the bounds of the dual feasibility problem)
template <class T>
__global__ void k_zero_finite(const T* in, T* out, int64_t len) {
  for (int64_t i = sgi(); i < len; i += sgs()) out[i] = isfinite(in[i]) ? (T)0 : in[i];
}

template <class T>
struct Solver {
  const pdlp_params& prm;
  cudaStream_t s;
  DeviceArena arena;
  Problem<T> P;
  Run<T> main_run, pol_run;
  // scratch shared by the runs (they advance one at a time on one stream)
  T *Xa = nullptr, *Ya = nullptr, *AXa = nullptr, *ATYa = nullptr;
  double *part_primal = nullptr, *part_dual = nullptr;
  unsigned int* counters = nullptr;  // [0] spmv-A, [1] kkt, [2] gap, [3] dist2
  int g_primal = 1, g_a = 1, g_at = 1, g_plain_a = 1, g_plain_at = 1, g_red = 1;
  KktScratch kks{};
  GapScratch gsc{};
  double* dist_part = nullptr;
  double* dist_out = nullptr;
  double* step_tab = nullptr;  // Algorithm 2's factors by accepted count (StepTable)
  int64_t step_len = 0;
  InfeasScratch<T> isc{};      // infeasibility detection (Sec. 3, App. C)
  bool ray_output = false;     // the returned x is a dual-infeasibility ray (no clamp)
  EventTimer timer;
  GapStats gap_stats;
  int64_t launches = 0;
  size_t setup_peak = 0;  // device bytes held at the end of setup, its temporaries included
  double ms_checks = 0.0;
  double ms_gap = 0.0, ms_kkt = 0.0, ms_infeas = 0.0;
  int64_t evaluations = 0;
  Clock::time_point t_solve0;
  // feasibility polishing (Algorithm 4)
  T* c_zero = nullptr;                                     // objective of the primal problem
  T *zlc = nullptr, *zuc = nullptr, *zlv = nullptr, *zuv = nullptr;  // bounds of the dual one
  T *Xk = nullptr, *Yk = nullptr;                          // (x^k, y^k) of the pause
  T *Xt = nullptr, *AXt = nullptr, *Yt = nullptr, *ATYt = nullptr;  // polished pair

  Solver(const pdlp_params& p, cudaStream_t st) : prm(p), s(st), slot_graphs_ok(!t_batch_worker) {
    arena.set_stream(st);
  }

  void alloc_shared() {
    const int64_t m = P.m, n = P.n;
    Xa = arena.alloc<T>(n);
    ATYa = arena.alloc<T>(n);
    Ya = arena.alloc<T>(m);
    AXa = arena.alloc<T>(m);
    g_primal = primal_grid(n);
    g_a = spmv_grid<T>(P.A, kEpiDual);
    g_at = spmv_grid<T>(P.AT, kEpiAverage);
    g_plain_a = spmv_grid<T>(P.A, kEpiPlain);
    g_plain_at = spmv_grid<T>(P.AT, kEpiPlain);
    g_red = std::max(1, num_sms() * 4);
    part_primal = arena.alloc<double>(g_primal);
    part_dual = arena.alloc<double>(2 * (int64_t)g_a);
    counters = arena.alloc<unsigned int>(8);
    PDLP_CUDA_CHECK(cudaMemsetAsync(counters, 0, 8 * sizeof(unsigned int), s));
    kks.grid = g_red;
    kks.rc_mode = prm.reduced_costs;
    kks.part = arena.alloc<double>(kKktPartials * (int64_t)g_red);
    kks.counter = counters + 1;
    kks.out = arena.alloc<KktSums>(1);
    gsc.grid = g_red;
    gsc.ctx = static_cast<GapCtx*>(arena.alloc_bytes(gap_ctx_bytes()));
    gsc.part = arena.alloc<double>((int64_t)kGapPartials * g_red);
    gsc.counter = counters + 2;
    gsc.cand = arena.alloc<int64_t>(kGapCandCap);
    gsc.params = arena.alloc_bytes(gap_param_bytes(m, n));
    dist_part = arena.alloc<double>(2 * (int64_t)g_red);
    dist_out = arena.alloc<double>(2);
  }

  void alloc_run(Run<T>& r) {
    const int64_t m = P.m, n = P.n;
    for (int q = 0; q < 2; ++q) {
      r.b.X[q] = arena.alloc<T>(n);
      r.b.ATY[q] = arena.alloc<T>(n);
      r.b.Y[q] = arena.alloc<T>(m);
      r.b.AX[q] = arena.alloc<T>(m);
    }
    r.b.Sx = arena.alloc<T>(n);
    r.b.SATy = arena.alloc<T>(n);
    r.b.Sy = arena.alloc<T>(m);
    r.b.SAx = arena.alloc<T>(m);
    r.b.m = m;
    r.b.n = n;
    r.X0 = arena.alloc<T>(n);
    r.Y0 = arena.alloc<T>(m);
    r.dst = arena.alloc<DevState>(1);
  }

  void alloc_polishing() {
    const int64_t m = P.m, n = P.n;
    alloc_run(pol_run);
    c_zero = arena.alloc<T>(n);
    PDLP_CUDA_CHECK(cudaMemsetAsync(c_zero, 0, sizeof(T) * n, s));
    zlv = arena.alloc<T>(n);
    zuv = arena.alloc<T>(n);
    zlc = arena.alloc<T>(m);
    zuc = arena.alloc<T>(m);
    k_zero_finite<T><<<vec_grid(n), kThreads, 0, s>>>(P.lv, zlv, n);
    k_zero_finite<T><<<vec_grid(n), kThreads, 0, s>>>(P.uv, zuv, n);
    launches += 2;
    if (m) {
      k_zero_finite<T><<<vec_grid(m), kThreads, 0, s>>>(P.lc, zlc, m);
      k_zero_finite<T><<<vec_grid(m), kThreads, 0, s>>>(P.uc, zuc, m);
      launches += 2;
    }
    PDLP_LAUNCH_CHECK();
    Xk = arena.alloc<T>(n);
    Xt = arena.alloc<T>(n);
    ATYt = arena.alloc<T>(n);
    Yk = arena.alloc<T>(m);
    Yt = arena.alloc<T>(m);
    AXt = arena.alloc<T>(m);
  }

  void alloc_infeas() {
    const int64_t m = P.m, n = P.n;
    isc.yd = arena.alloc<T>(m);
    isc.atyd = arena.alloc<T>(n);
    isc.xb = arena.alloc<T>(3 * n);
    isc.axb = arena.alloc<T>(3 * m);
    isc.grid = g_red;
    isc.part = arena.alloc<double>(15 * (int64_t)g_red);
    isc.counter = counters + 4;
    isc.out = arena.alloc<double>(18);
  }

  // App. C's tests on the three candidates of this check (difference of the last two
  // iterates, current iterate, average in Xa..ATYa); on success out_pt is the returned
  // point: (current x, certificate y) or (certificate x, current y).
  int check_infeasibility(Run<T>& r, PointRef<T>& out_pt, KktResult& out_k) {
    const int64_t m = P.m, n = P.n;
    const int cur = r.hs.cur;
    const InfeasInputs<T> in{r.b.X[cur], r.b.Y[cur], r.b.ATY[cur], r.b.X[cur ^ 1], r.b.Y[cur ^ 1],
                             Xa, Ya, ATYa, r.b.lc, r.b.uc, r.b.lv, r.b.uv};
    int nl = 0;
    const auto t0 = Clock::now();
    const InfeasMeasures im = infeasibility_measures<T>(in, isc, origv(), P.A, P.AT, g_plain_a,
                                                        g_plain_at, m, n, s, &nl);
    launches += nl;
    const double ms = 1e3 * secs_since(t0);
    ms_checks += ms;
    ms_infeas += ms;
    const double eps = prm.eps_infeas;
    const T* ys[3] = {isc.yd, r.b.Y[cur], Ya};
    const T* atys[3] = {isc.atyd, r.b.ATY[cur], ATYa};
    for (int c = 0; c < 3; ++c) {
      if (im.y_obj[c] > 0.0 && im.y_res[c] <= eps * im.y_obj[c]) {
        out_pt = PointRef<T>{r.b.X[cur], ys[c], r.b.AX[cur], atys[c]};
        out_k = kkt(out_pt);
        return PDLP_PRIMAL_INFEASIBLE;
      }
    }
    for (int c = 0; c < 3; ++c) {
      if (im.cx[c] < 0.0 && im.x_res[c] <= eps * std::fabs(im.cx[c])) {
        out_pt = PointRef<T>{isc.xb + c * n, r.b.Y[cur], isc.axb + c * m, r.b.ATY[cur]};
        out_k = kkt(out_pt);
        ray_output = true;
        return PDLP_DUAL_INFEASIBLE;
      }
    }
    return 0;
  }

  void zero_sums(Run<T>& r) {
    PDLP_CUDA_CHECK(cudaMemsetAsync(r.b.Sx, 0, sizeof(T) * P.n, s));
    PDLP_CUDA_CHECK(cudaMemsetAsync(r.b.SATy, 0, sizeof(T) * P.n, s));
    if (P.m) {
      PDLP_CUDA_CHECK(cudaMemsetAsync(r.b.Sy, 0, sizeof(T) * P.m, s));
      PDLP_CUDA_CHECK(cudaMemsetAsync(r.b.SAx, 0, sizeof(T) * P.m, s));
    }
  }

  void push_state(Run<T>& r) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(r.dst, &r.hs, sizeof(DevState), cudaMemcpyHostToDevice, s));
  }
  void pull_state(Run<T>& r) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(&r.hs, r.dst, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    timer.collect();
  }

  PointRef<T> current(const Run<T>& r) const {
    return PointRef<T>{r.b.X[r.hs.cur], r.b.Y[r.hs.cur], r.b.AX[r.hs.cur], r.b.ATY[r.hs.cur]};
  }
  PointRef<T> average() const { return PointRef<T>{Xa, Ya, AXa, ATYa}; }
  static ScaledVecs<T> vecs(const Run<T>& r) {
    return ScaledVecs<T>{r.b.c, r.b.lc, r.b.uc, r.b.lv, r.b.uv, r.b.m, r.b.n};
  }
  OrigVecs origv() const {
    return OrigVecs{P.orig.c, P.orig.lc, P.orig.uc, P.orig.lv, P.orig.uv,
                    P.d1,     P.d2,      P.inv_d1,  P.inv_d2};
  }

  double gap(const Run<T>& r, const PointRef<T>& z, double omega) {
    auto t0 = Clock::now();
    int nl = 0;
    const double mu =
        normalized_gap<T>(z, r.X0, r.Y0, omega, vecs(r), gsc, s, &nl, &gap_stats);
    launches += nl;
    const double ms = 1e3 * secs_since(t0);
    ms_checks += ms;
    ms_gap += ms;
    return mu;
  }

  KktResult kkt(const PointRef<T>& z) {
    auto t0 = Clock::now();
    launch_kkt<T>(z, origv(), P.m, P.n, kks, s);
    launches++;
    KktSums h;
    PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, kks.out, sizeof(KktSums), cudaMemcpyDeviceToHost, s));
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    const double ms = 1e3 * secs_since(t0);
    ms_checks += ms;
    ms_kkt += ms;
    return kkt_finish(h, P.c_norm, P.b_norm);
  }

  // the step-factor table covers accepted counts [0, upto]; it grows by doubling
  void ensure_step_table(int64_t upto) {
    if (upto < step_len) return;
    int64_t len = std::max<int64_t>(4096, 2 * step_len);
    while (len <= upto) len *= 2;
    step_tab = arena.alloc<double>(2 * len);
    fill_step_table(step_tab, len, s);
    launches++;
    step_len = len;
  }

  // one step attempt = three launches (see file comment)
  void launch_slot(Run<T>& r) {
    int e0 = timer.begin(s);
    launch_primal<T>(r.b, r.dst, part_primal, g_primal, s);
    timer.end(e0, 2, s);
    int e1 = timer.begin(s);
    launch_spmv_dual<T>(P.A, r.b, r.dst, part_primal, g_primal, part_dual, counters,
                        StepTable{step_tab, step_len}, g_a, s);
    timer.end(e1, 0, s);
    int e2 = timer.begin(s);
    launch_spmv_avg<T>(P.AT, r.b, r.dst, g_at, s);
    timer.end(e2, 1, s);
    launches += 3;
  }

  // Step attempts replayed from captured graphs of 64 attempts (the span between two
  // checks; shorter spans launch directly) when per-kernel timing is off and the call is
  // not part of a batch: the three launches of an attempt take the same arguments
  // throughout a run (the device state picks the buffers and decides acceptance), so a
  // graph is keyed by the run's buffers and the step-factor table.
  static constexpr int64_t kSlotChunk = 64;
  struct SlotGraph {
    IterBuffers<T> b;
    DevState* dst;
    const double* tab;
    int64_t len;
    std::unique_ptr<Replay> replay;
  };
  std::vector<SlotGraph> slot_graphs;
  bool slot_graphs_ok;

  Replay* slot_graph(Run<T>& r) {
    for (auto& g : slot_graphs)
      if (g.dst == r.dst && g.tab == step_tab && g.len == step_len &&
          std::memcmp(&g.b, &r.b, sizeof(r.b)) == 0)
        return g.replay.get();
    std::unique_ptr<Replay> rp(new Replay);
    const int64_t saved = launches;  // captured launches run when the graph is replayed
    const bool ok = rp->capture(s, [&] {
      for (int64_t q = 0; q < kSlotChunk; ++q) launch_slot(r);
    });
    launches = saved;
    if (!ok) {
      slot_graphs_ok = false;
      return nullptr;
    }
    slot_graphs.push_back(SlotGraph{r.b, r.dst, step_tab, step_len, std::move(rp)});
    return slot_graphs.back().replay.get();
  }

  void launch_slots(Run<T>& r, int64_t count) {
    while (count >= kSlotChunk && !timer.on && slot_graphs_ok) {
      Replay* g = slot_graph(r);
      if (!g) break;
      g->launch(s);
      launches += 3 * kSlotChunk;
      count -= kSlotChunk;
    }
    for (int64_t q = 0; q < count; ++q) launch_slot(r);
  }

  // first n (>= 1) such that restart condition (iii) t+j >= beta (k+j) holds
  int64_t steps_to_artificial(int64_t k, int64_t t) const {
    return pdlp::steps_to_artificial(k, t, prm.beta_art);
  }

  // Starts run r on the LP with scaled vectors (c, lc, uc, lv, uv) from (x_start,
  // y_start) (device vectors of the renumbered LP; null = 0), or from z^{0,0} =
  // (proj_X(0), 0) when both are null, with primal weight omega and step eta_hat.
  void start_run(Run<T>& r, const T* x_start, const T* y_start, double omega, double eta_hat,
                 int64_t max_iters, int goal, const T* c, const T* lc, const T* uc,
                 const T* lv, const T* uv) {
    const int64_t m = P.m, n = P.n;
    r.b.c = c;
    r.b.lc = lc;
    r.b.uc = uc;
    r.b.lv = lv;
    r.b.uv = uv;
    if (!x_start && !y_start) {
      k_init_point<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(
          lv, uv, r.b.X[0], r.b.Y[0], r.b.ATY[0], r.X0, r.Y0, m, n);
      PDLP_LAUNCH_CHECK();
      launches++;
    } else {
      k_start_point<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(
          x_start, y_start, r.b.X[0], r.b.Y[0], r.X0, r.Y0, m, n);
      PDLP_LAUNCH_CHECK();
      launch_spmv_plain<T>(P.AT, r.b.Y[0], r.b.ATY[0], g_plain_at, s);
      launches += 2;
    }
    launch_spmv_plain<T>(P.A, r.b.X[0], r.b.AX[0], g_plain_a, s);
    launches++;
    zero_sums(r);
    std::memset(&r.hs, 0, sizeof(r.hs));
    r.hs.cur = 0;
    r.hs.eta = eta_hat;
    r.hs.eta_hat = eta_hat;
    r.hs.omega = omega;
    r.hs.max_retries = prm.max_step_retries;
    r.hs.fixed_eta = prm.fixed_step > 0.0 ? prm.fixed_step : 0.0;
    push_state(r);
    r.goal = goal;
    r.max_iters = max_iters;
    r.started = false;
    r.have_mu_ref = false;
    r.mu_ref = 0.0;
    r.mu_c_prev = INFINITY;
    r.k = r.t = r.attempts_at_last = 0;
    r.restarts[0] = r.restarts[1] = r.restarts[2] = 0;
  }

  // Advances run r (Algorithm 1 with device-side Algorithm 2 steps, the restart scheme
  // of Sec. 3 and Algorithm 3) until its goal is met on a restart candidate, its
  // iteration cap or the time limit is reached, a step fails, or -- pause_at >= 0 --
  // pause_at iterations are complete (with that iteration's check and restart done).
  // out_pt / out_k receive the point to return and its KKT measures (not for a pause).
  RunOutcome advance(Run<T>& r, int64_t pause_at, PointRef<T>& out_pt, KktResult& out_k) {
    const int64_t m = P.m, n = P.n;
    const int64_t period = std::max(1, prm.check_period);
    const int64_t trace_iters =
        (r.trace && prm.trace_out && prm.trace_iters > 0) ? prm.trace_iters : 0;
    const int64_t rec_len = PDLP_TRACE_HEADER + n + m;
    if (!r.started) {
      r.started = true;
      // termination test on the start point before the first step
      out_k = kkt(current(r));
      if (goal_met(out_k, prm, r.goal)) {
        out_pt = current(r);
        return kRunDone;
      }
    }
    for (;;) {
      if (pause_at >= 0 && r.k >= pause_at) return kRunPaused;
      const int64_t next_check = (r.k / period + 1) * period;
      int64_t target = std::min(next_check, r.max_iters);
      if (pause_at >= 0) target = std::min(target, pause_at);
      const int64_t j_art = steps_to_artificial(r.k, r.t);
      if (r.k + j_art < target) target = r.k + j_art;
      // launch attempts until `target` accepted iterations (rejections need more)
      ensure_step_table(target);
      bool error = false;
      while (r.k < target) {
        const int64_t need = (trace_iters > r.k) ? 1 : (target - r.k);
        launch_slots(r, need);
        const double omega_used = r.hs.omega;
        pull_state(r);
        if (r.hs.error) {
          error = true;
          break;
        }
        if (trace_iters > r.k && r.hs.k > r.k) record_trace(r, omega_used, rec_len);
        if (r.hs.k > r.k) r.attempts_at_last = r.hs.attempts;
        r.k = r.hs.k;
        r.t = r.hs.t;
      }
      if (error) {
        out_pt = current(r);
        out_k = kkt(out_pt);
        return kRunError;
      }
      const int64_t k = r.k, t = r.t;
      double* rec =
          (trace_iters >= k && k >= 1) ? prm.trace_out + (size_t)(k - 1) * rec_len : nullptr;
      const bool is_check = (k % period) == 0;
      const bool is_art = (double)t >= prm.beta_art * (double)k;
      const bool is_limit = k >= r.max_iters;
      if (!(is_check || is_art || is_limit)) continue;
      evaluations++;
      // GetRestartCandidate: current vs average since the restart
      launch_average<T>(r.b.Sx, r.b.Sy, r.b.SAx, r.b.SATy, 1.0 / r.hs.W, r.b.lv, r.b.uv, Xa, Ya,
                        AXa, ATYa, m, n, s);
      launches++;
      const double omega = r.hs.omega;
      const double mu_cur = gap(r, current(r), omega);
      const double mu_avg = gap(r, average(), omega);
      const bool cand_avg = !(mu_cur < mu_avg);
      const double mu_c = cand_avg ? mu_avg : mu_cur;
      const PointRef<T> cand = cand_avg ? average() : current(r);
      if (rec) {
        rec[6] = mu_cur;
        rec[7] = mu_avg;
      }
      if (is_check || is_limit) {
        out_k = kkt(cand);
        if (prm.verbose)
          std::fprintf(stderr,
                       "pdlp: goal=%d k=%lld rel_kkt=%.3e pres_inf=%.3e dres_inf=%.3e "
                       "pres_eq10=%.3e dres_eq10=%.3e gap8=%.3e pobj=%.10e omega=%.3e eta=%.3e "
                       "restarts=%lld/%lld/%lld\n",
                       r.goal, (long long)k, out_k.rel_kkt, out_k.pres_inf, out_k.dres_inf,
                       out_k.pres_rel_inf, out_k.dres_rel_inf, out_k.paper_gap, out_k.pobj, omega,
                       r.hs.eta_hat, (long long)r.restarts[0],
                       (long long)r.restarts[1], (long long)r.restarts[2]);
        if (goal_met(out_k, prm, r.goal)) {
          out_pt = cand;
          return kRunDone;
        }
        if (r.infeas) {  // after the termination test, before the restart decision
          const int inf = check_infeasibility(r, out_pt, out_k);
          if (inf == PDLP_PRIMAL_INFEASIBLE) return kRunPrimalInf;
          if (inf == PDLP_DUAL_INFEASIBLE) return kRunDualInf;
        }
        if (is_limit) {
          out_pt = cand;
          return kRunLimit;
        }
        if (secs_since(t_solve0) > prm.time_limit_s) {
          out_pt = cand;
          return kRunTime;
        }
      }
      const int kind = restart_kind(is_check, is_art, r.have_mu_ref, mu_c, r.mu_ref,
                                    r.mu_c_prev, prm.beta_suff, prm.beta_nec);
      if (is_check) r.mu_c_prev = mu_c;
      if (kind == 0) continue;
      // restart the outer loop at the candidate
      r.restarts[kind - 1]++;
      if (rec) rec[5] = (double)kind;
      const int cur = r.hs.cur;
      if (cand_avg) {
        k_copy2<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(Xa, r.b.X[cur], n, Ya, r.b.Y[cur], m);
        k_copy2<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(ATYa, r.b.ATY[cur], n, AXa, r.b.AX[cur], m);
        PDLP_LAUNCH_CHECK();
        launches += 2;
      }
      // Algorithm 3
      launch_dist2<T>(r.b.X[cur], r.X0, r.b.Y[cur], r.Y0, m, n, dist_part, counters + 3, dist_out,
                      g_red, s);
      launches++;
      double d2h[2];
      PDLP_CUDA_CHECK(cudaMemcpyAsync(d2h, dist_out, sizeof(d2h), cudaMemcpyDeviceToHost, s));
      PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
      const double dx = std::sqrt(d2h[0]), dy = std::sqrt(d2h[1]);
      const double om = prm.fixed_omega > 0.0 ? prm.fixed_omega
                                              : primal_weight(r.hs.omega, dx, dy, prm.theta, prm.eps_zero);
      r.mu_ref = gap(r, current(r), om);
      r.have_mu_ref = true;
      k_copy2<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(r.b.X[cur], r.X0, n, r.b.Y[cur], r.Y0, m);
      PDLP_LAUNCH_CHECK();
      launches++;
      zero_sums(r);
      r.mu_c_prev = INFINITY;
      r.hs.omega = om;
      r.hs.W = 0.0;
      r.hs.t = 0;
      r.t = 0;
      push_state(r);
    }
  }

  // trace record of accepted iteration r.hs.k (one slot per pull in trace mode)
  std::vector<T> hx, hy;
  std::vector<int32_t> hperm_c, hperm_r;
  void record_trace(Run<T>& r, double omega_used, int64_t rec_len) {
    const int64_t m = P.m, n = P.n;
    double* rec = prm.trace_out + (size_t)r.k * rec_len;
    rec[0] = (double)r.hs.k;
    rec[1] = r.hs.eta_acc;
    rec[2] = omega_used;
    rec[3] = r.hs.eta_hat;
    rec[4] = (double)(r.hs.attempts - r.attempts_at_last);
    rec[5] = 0.0;
    rec[6] = NAN;
    rec[7] = NAN;
    if (hperm_c.empty() && n) {
      hperm_c.resize(n);
      hperm_r.resize(m);
      PDLP_CUDA_CHECK(cudaMemcpyAsync(hperm_c.data(), P.perm_c, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
      if (m) PDLP_CUDA_CHECK(cudaMemcpyAsync(hperm_r.data(), P.perm_r, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
    }
    hx.resize(n);
    hy.resize(m);
    PDLP_CUDA_CHECK(cudaMemcpyAsync(hx.data(), r.b.X[r.hs.cur], sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    if (m) PDLP_CUDA_CHECK(cudaMemcpyAsync(hy.data(), r.b.Y[r.hs.cur], sizeof(T) * m, cudaMemcpyDeviceToHost, s));
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    for (int64_t j = 0; j < n; ++j) rec[PDLP_TRACE_HEADER + hperm_c[j]] = (double)hx[j];
    for (int64_t i = 0; i < m; ++i) rec[PDLP_TRACE_HEADER + n + hperm_r[i]] = (double)hy[i];
  }

  // status of a finished run
  static int status_of(RunOutcome o) {
    switch (o) {
      case kRunDone: return PDLP_OPTIMAL;
      case kRunLimit: return PDLP_ITERATION_LIMIT;
      case kRunTime: return PDLP_TIME_LIMIT;
      case kRunPrimalInf: return PDLP_PRIMAL_INFEASIBLE;
      case kRunDualInf: return PDLP_DUAL_INFEASIBLE;
      default: return PDLP_NUMERICAL_ERROR;
    }
  }

  struct PolishTotals {
    int64_t pauses = 0, primal_iters = 0, dual_iters = 0, accepted_k = 0;
  } pol;

  // The two phases of Algorithm 4 from (x^k, y^k) = (Xk, Yk), with primal weight omega
  // and step eta, each for at most `budget` iterations.  Returns 1 when the polished
  // pair meets the termination criteria (out_pt / out_k set to it), 2 when the time
  // limit ran out, 0 otherwise.  `row` (may be null) receives the phases' log entries.
  int polish_phases(int64_t budget, double omega, double eta, double* row, PointRef<T>& out_pt,
                    KktResult& out_k) {
    const int64_t m = P.m, n = P.n;
    // primal feasibility problem (objective 0) from (x^k, 0)
    start_run(pol_run, Xk, nullptr, omega, eta, budget, kGoalPrimalFeasible, c_zero, P.lc, P.uc,
              P.lv, P.uv);
    PointRef<T> pp;
    KktResult kpp;
    const RunOutcome op = advance(pol_run, -1, pp, kpp);
    pol.primal_iters += pol_run.k;
    if (row) {
      row[2] = (double)pol_run.k;
      row[3] = op == kRunDone ? 1.0 : 0.0;
    }
    if (op == kRunTime) return 2;
    if (op != kRunDone) return 0;
    k_copy2<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(pp.x, Xt, n, pp.ax, AXt, m);
    PDLP_LAUNCH_CHECK();
    launches++;
    // dual feasibility problem (finite bounds set to 0) from (0, y^k)
    start_run(pol_run, nullptr, Yk, omega, eta, budget, kGoalDualFeasible, P.c, zlc, zuc, zlv, zuv);
    PointRef<T> pd;
    KktResult kpd;
    const RunOutcome od = advance(pol_run, -1, pd, kpd);
    pol.dual_iters += pol_run.k;
    if (row) {
      row[4] = (double)pol_run.k;
      row[5] = od == kRunDone ? 1.0 : 0.0;
    }
    if (od == kRunTime) return 2;
    k_copy2<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(pd.aty, ATYt, n, pd.y, Yt, m);
    PDLP_LAUNCH_CHECK();
    launches++;
    const PointRef<T> pair{Xt, Yt, AXt, ATYt};
    const KktResult kf = kkt(pair);
    if (!converged(kf, prm)) return 0;
    if (row) row[6] = 1.0;
    out_pt = pair;
    out_k = kf;
    return 1;
  }

  // FP32 bulk: the phases run in FP64 on a second, FP64 copy of the preconditioned
  // problem (same scaling and numbering, from the unscaled staged inputs din_), built
  // at the first pause that needs it.
  const Inputs* in_ = nullptr;
  DevInputs din_{};
  std::unique_ptr<Solver<double>> aux64;
  bool out_from_aux = false;
  PointRef<double> aux_pt{};

  void prepare_phases(const Inputs& in, const DevInputs& d, Clock::time_point t0) {
    DeviceArena tmp;
    tmp.set_stream(s);
    build_problem<T>(arena, in, d, prm.ruiz_iters, prm.pc_alpha, P, s, true, &tmp);
    setup_peak = arena.total() + tmp.total();
    launches += P.launches;
    alloc_shared();
    alloc_polishing();
    t_solve0 = t0;
  }

  // Algorithm 4: normal PDLP (main_run) with pauses at k = 100, 200, 400, ...
  int solve_polished(PointRef<T>& out_pt, KktResult& out_k) {
    const int64_t m = P.m, n = P.n;
    for (int64_t kp = 100;; kp *= 2) {
      const RunOutcome o = advance(main_run, kp, out_pt, out_k);
      if (o != kRunPaused) return status_of(o);
      // (x^k, y^k): the average since the last restart (right after a restart, the
      // restart point)
      PointRef<T> zk = current(main_run);
      if (main_run.hs.W != 0.0) {
        launch_average<T>(main_run.b.Sx, main_run.b.Sy, main_run.b.SAx, main_run.b.SATy,
                          1.0 / main_run.hs.W, P.lv, P.uv, Xa, Ya, AXa, ATYa, m, n, s);
        launches++;
        zk = average();
      }
      const KktResult kz = kkt(zk);
      double* row = nullptr;
      if (prm.polish_log && pol.pauses < prm.polish_log_cap) {
        row = prm.polish_log + (size_t)pol.pauses * PDLP_POLISH_LOG_COLS;
        for (int q = 0; q < PDLP_POLISH_LOG_COLS; ++q) row[q] = 0.0;
        row[0] = (double)kp;
        row[1] = kz.paper_gap;
      }
      pol.pauses++;
      if (prm.verbose)
        std::fprintf(stderr, "pdlp: pause k=%lld average: gap8=%.3e pres_inf=%.3e dres_inf=%.3e\n",
                     (long long)kp, kz.paper_gap, kz.pres_inf, kz.dres_inf);
      if (!(kz.paper_gap < prm.eps_rel_gap)) continue;
      const double omega = main_run.hs.omega, eta = main_run.hs.eta_hat;
      const int64_t budget = kp / 8;
      int r;
      if constexpr (std::is_same<T, double>::value) {
        k_copy2<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(zk.x, Xk, n, zk.y, Yk, m);
        PDLP_LAUNCH_CHECK();
        launches++;
        r = polish_phases(budget, omega, eta, row, out_pt, out_k);
      } else {
        if (!aux64) {
          aux64.reset(new Solver<double>(prm, s));
          aux64->prepare_phases(*in_, din_, t_solve0);
        }
        k_to_double2<T><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(zk.x, aux64->Xk, n, zk.y,
                                                                      aux64->Yk, m);
        PDLP_LAUNCH_CHECK();
        launches++;
        r = aux64->polish_phases(budget, omega, eta, row, aux_pt, out_k);
        out_from_aux = r == 1;
      }
      if (r == 2) {
        out_from_aux = false;
        out_pt = current(main_run);
        out_k = kkt(out_pt);
        return PDLP_TIME_LIMIT;
      }
      if (r == 1) {
        pol.accepted_k = kp;
        return PDLP_OPTIMAL;
      }
    }
  }

  // x = D2 x~, y = D1 y~ of a point of problem Q, into the caller's numbering
  template <class U>
  void emit(const Problem<U>& Q, const PointRef<U>& pt, double* xo, double* yo) {
    const int64_t m = Q.m, n = Q.n;
    k_unscale<U><<<vec_grid(std::max(m, n)), kThreads, 0, s>>>(
        pt.x, pt.y, Q.d1, Q.d2, Q.orig.lv, Q.orig.uv, Q.perm_r, Q.perm_c, xo, yo, m, n,
        !ray_output);
    PDLP_LAUNCH_CHECK();
    launches++;
  }

  int run(const Inputs& in, double* x_out, double* y_out, pdlp_stats* st) {
    const auto t_start = Clock::now();
    // setup temporaries (the staged input included, unless the FP64 phase problem of
    // FP32-bulk polishing is built from it later) are freed once the layouts exist
    const bool keep_staged = prm.feasibility_polishing && !std::is_same<T, double>::value;
    DeviceArena tmp;
    tmp.set_stream(s);
    DeviceArena& stage_arena = keep_staged ? arena : tmp;
    DevInputs d = stage_inputs(stage_arena, in, s);
    validate(stage_arena, in, d, s);
    in_ = &in;
    din_ = d;
    if (keep_staged && in.nnz) {
      // build_problem scales the staged values in place; the FP64 phase problem is
      // built later from an unscaled copy
      double* v = arena.alloc<double>(in.nnz);
      PDLP_CUDA_CHECK(cudaMemcpyAsync(v, d.val, sizeof(double) * in.nnz, cudaMemcpyDeviceToDevice, s));
      din_.val = v;
    }
    build_problem<T>(arena, in, d, prm.ruiz_iters, prm.pc_alpha, P, s, true, &tmp);
    setup_peak = arena.total() + tmp.total();
    launches += P.launches;
    alloc_shared();
    alloc_run(main_run);
    if (prm.feasibility_polishing && std::is_same<T, double>::value) alloc_polishing();
    if (prm.detect_infeasibility) alloc_infeas();
    const int64_t m = P.m, n = P.n;

    double eta0 = P.max_abs > 0.0 ? 1.0 / P.max_abs : 1.0;
    double omega0 = (P.c_norm_s > 0.0 && P.b_norm_s > 0.0) ? P.c_norm_s / P.b_norm_s : 1.0;
    if (prm.fixed_step > 0.0) eta0 = prm.fixed_step;
    if (prm.fixed_omega > 0.0) omega0 = prm.fixed_omega;
    // z^{0,0} = (proj_X(0), 0)
    start_run(main_run, nullptr, nullptr, omega0, eta0, prm.max_iters, kGoalOptimal, P.c, P.lc,
              P.uc, P.lv, P.uv);
    main_run.trace = true;
    main_run.infeas = prm.detect_infeasibility != 0;
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    const double t_setup = secs_since(t_start);
    t_solve0 = Clock::now();
    timer.on = prm.profile != 0;

    PointRef<T> out_pt = current(main_run);
    KktResult out_k{};
    int status;
    if (prm.feasibility_polishing)
      status = solve_polished(out_pt, out_k);
    else
      status = status_of(advance(main_run, -1, out_pt, out_k));

    // output: the returned point, unscaled
    double* xo = x_out;
    double* yo = y_out;
    double* dx_out = nullptr;
    double* dy_out = nullptr;
    if (!in.on_device) {
      dx_out = arena.alloc<double>(n);
      dy_out = arena.alloc<double>(m);
      xo = dx_out;
      yo = dy_out;
    }
    if (out_from_aux)
      emit<double>(aux64->P, aux_pt, xo, yo);
    else
      emit<T>(P, out_pt, xo, yo);
    if (!in.on_device) {
      PDLP_CUDA_CHECK(cudaMemcpyAsync(x_out, dx_out, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
      if (m) PDLP_CUDA_CHECK(cudaMemcpyAsync(y_out, dy_out, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    }
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    timer.collect();
    if (st) {
      const DevState& hs = main_run.hs;
      std::memset(st, 0, sizeof(*st));
      st->status = status;
      st->iterations = hs.k;
      st->attempts = hs.attempts;
      st->rejected_steps = hs.rejected;
      for (int q = 0; q < 3; ++q) st->restarts[q] = main_run.restarts[q];
      st->kkt_passes = 0.5 * (double)(hs.attempts + hs.k);
      st->rel_kkt = out_k.rel_kkt;
      st->rel_primal = out_k.rel_primal;
      st->rel_dual = out_k.rel_dual;
      st->rel_gap = out_k.rel_gap;
      st->primal_res_l2 = out_k.pres2;
      st->dual_res_l2 = out_k.dres2;
      st->primal_res_inf = out_k.pres_inf;
      st->dual_res_inf = out_k.dres_inf;
      st->pobj = out_k.pobj;
      st->dobj = out_k.dobj;
      st->paper_gap = out_k.paper_gap;
      st->omega = hs.omega;
      st->eta_hat = hs.eta_hat;
      st->seconds_setup = t_setup;
      st->seconds_solve = secs_since(t_solve0);
      st->seconds_total = secs_since(t_start);
      st->ms_spmv_a = timer.ms[0];
      st->ms_spmv_at = timer.ms[1];
      st->ms_primal = timer.ms[2];
      st->primal_res_rel_inf = out_k.pres_rel_inf;
      st->dual_res_rel_inf = out_k.dres_rel_inf;
      st->ms_checks = ms_checks + (aux64 ? aux64->ms_checks : 0.0);
      st->ms_gap = ms_gap + (aux64 ? aux64->ms_gap : 0.0);
      st->ms_kkt = ms_kkt + (aux64 ? aux64->ms_kkt : 0.0);
      st->ms_infeas = ms_infeas + (aux64 ? aux64->ms_infeas : 0.0);
      st->evaluations = evaluations + (aux64 ? aux64->evaluations : 0);
      st->launches_spmv_a = timer.count[0];
      st->launches_spmv_at = timer.count[1];
      st->kernel_launches = launches + (aux64 ? aux64->launches : 0);
      const double v = (double)sizeof(T);
      st->gap_evals = gap_stats.evals;
      st->gap_fallbacks = gap_stats.fallbacks;
      st->gap_failures = gap_stats.failures;
      if (gap_stats.failures) set_last_error(gap_stats.last_failure);
      if (aux64) {
        st->gap_evals += aux64->gap_stats.evals;
        st->gap_fallbacks += aux64->gap_stats.fallbacks;
        st->gap_failures += aux64->gap_stats.failures;
        if (aux64->gap_stats.failures) set_last_error(aux64->gap_stats.last_failure);
      }
      st->bytes_spmv_a = (double)(m + 1) * 8 + (double)P.nnz * (4 + v) + (double)n * v + 6.0 * m * v;
      st->bytes_spmv_at = (double)(n + 1) * 8 + (double)P.nnz * (4 + v) + (double)m * v +
                          6.0 * (double)n * v + 6.0 * (double)m * v;
      st->polish_pauses = pol.pauses;
      st->polish_primal_iters = pol.primal_iters + (aux64 ? aux64->pol.primal_iters : 0);
      st->polish_dual_iters = pol.dual_iters + (aux64 ? aux64->pol.dual_iters : 0);
      st->polish_accepted_k = pol.accepted_k;
      st->device_bytes = (int64_t)(std::max(setup_peak, arena.total()) +
                                   (aux64 ? std::max(aux64->setup_peak, aux64->arena.total()) : 0));
    }
    return status;
  }
};

static int handle_exception() {
  try {
    throw;
  } catch (const PdlpError& e) {
    set_last_error(e.what());
    return e.code < 0 ? e.code : PDLP_NUMERICAL_ERROR;
  } catch (const std::bad_alloc&) {
    set_last_error("out of host memory");
    return PDLP_OUT_OF_MEMORY;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return PDLP_CUDA_ERROR;
  } catch (...) {
    set_last_error("unknown error");
    return PDLP_CUDA_ERROR;
  }
}

struct StreamGuard {
  cudaStream_t s = nullptr;
  bool own = false;
  explicit StreamGuard(void* user) {
    if (user) {
      s = (cudaStream_t)user;
    } else {
      PDLP_CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      own = true;
    }
  }
  ~StreamGuard() {
    if (own && s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
};

static void check_params(const pdlp_params& prm) {
  if (prm.pc_alpha >= 2.0) throw PdlpError(-1, "pc_alpha must be < 2");
  if (prm.max_iters < 1 || prm.check_period < 1 || prm.max_step_retries < 1)
    throw PdlpError(-1, "max_iters, check_period and max_step_retries must be >= 1");
  if (prm.termination_mode < 0 || prm.termination_mode > 2)
    throw PdlpError(-1, "termination_mode must be 0, 1 or 2");
  if (!(prm.beta_art >= 0.0) || std::isnan(prm.beta_suff) || std::isnan(prm.beta_nec))
    throw PdlpError(-1, "beta_art must be >= 0 (>= 1: criterion (iii) off); beta_suff and beta_nec not NaN");
  if (!(prm.fixed_step >= 0.0 && std::isfinite(prm.fixed_step)) ||
      !(prm.fixed_omega >= 0.0 && std::isfinite(prm.fixed_omega)))
    throw PdlpError(-1, "fixed_step and fixed_omega must be finite and >= 0");
}

static Inputs make_inputs(int64_t m, int64_t n, const pdlp_csr* A, const double* c,
                          const double* lc, const double* uc, const double* lv, const double* uv,
                          const pdlp_params* p) {
  if (!A) throw PdlpError(-1, "A is NULL");
  Inputs in;
  in.m = m;
  in.n = n;
  in.nnz = A->nnz;
  in.row_ptr = A->row_ptr;
  in.col = A->col_idx;
  in.val = A->val;
  in.c = c;
  in.lc = lc;
  in.uc = uc;
  in.lv = lv;
  in.uv = uv;
  in.on_device = p && p->inputs_on_device;
  check_args(in);
  return in;
}

}  // namespace pdlp

using namespace pdlp;

// Runs call(i, params with a worker stream) for i in [0, count) on `concurrency` host
// threads of the caller's device, each with its own non-blocking stream; records each
// return value and the message of the lowest failed index.
namespace pdlp {
template <class Call>
static int run_batch(const char* name, int64_t count, const pdlp_params& prm, int concurrency,
                     int* status_out, Call call) {
  int dev = 0;
  PDLP_CUDA_CHECK(cudaGetDevice(&dev));
  const int64_t workers =
      std::max<int64_t>(1, std::min<int64_t>(concurrency <= 0 ? 16 : concurrency, count));
  std::atomic<int64_t> next{0};
  std::mutex mu;
  std::string first_error;
  int64_t first_index = -1;
  auto work = [&]() {
    const bool was_worker = t_batch_worker;
    t_batch_worker = true;
    cudaStream_t s = nullptr;
    if (cudaSetDevice(dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      s = nullptr;
    }
    pdlp_params q = prm;
    q.cuda_stream = s;
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= count) break;
      int code;
      if (!s) {
        set_last_error(std::string(name) + ": could not create a stream for a worker");
        code = PDLP_CUDA_ERROR;
      } else {
        code = call(i, q);
      }
      status_out[i] = code;
      if (code < 0) {
        std::lock_guard<std::mutex> lock(mu);
        if (first_index < 0 || i < first_index) {
          first_index = i;
          first_error = std::string("problem ") + std::to_string(i) + ": " + pdlp_last_error();
        }
      }
    }
    if (s) cudaStreamDestroy(s);
    t_batch_worker = was_worker;
  };
  std::vector<std::thread> pool;
  for (int64_t w = 1; w < workers; ++w) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  if (first_index >= 0) set_last_error(first_error);
  return 0;
}
}  // namespace pdlp


// ---------------------------------------------------------------------------
// persistent batch: every LP set up by the single-LP code (staging, validation,
// preconditioning, SELL layouts) on worker streams, then one launch of k_batch
// ---------------------------------------------------------------------------
namespace pdlp {

constexpr int64_t kSetupWorkers = 16;  // host threads (each with a stream) setting LPs up

template <class T>
struct BatchItem {
  DeviceArena arena;
  Problem<T> P;
  BatchLP<T> d{};
  double *dx = nullptr, *dy = nullptr;  // device outputs when the caller's are on the host
  int code = 0;                         // negative: the LP failed before the launch
  std::string err;
  double setup_s = 0.0;
  int64_t launches = 0;
};

__global__ void k_narrow_u16(const int32_t* in, uint16_t* out, int64_t len) {
  for (int64_t i = sgi(); i < len; i += sgs()) out[i] = (uint16_t)in[i];
}

// 16-bit copy of a SELL layout's column indices (every index < cols <= 65536)
template <class T>
static const uint16_t* sell_col16(DeviceArena& a, const Mat<T>& M, cudaStream_t s) {
  uint16_t* out = a.alloc<uint16_t>(M.sell_entries);
  if (M.sell_entries) {
    k_narrow_u16<<<vec_grid(M.sell_entries), kThreads, 0, s>>>(M.sell_col, out, M.sell_entries);
    PDLP_LAUNCH_CHECK();
  }
  return out;
}

// LP i's problem, work buffers and descriptor, on stream s
template <class T>
static void batch_setup_one(BatchItem<T>& it, const pdlp_problem& pr, const pdlp_params& prm,
                            cudaStream_t s) {
  const auto t0 = Clock::now();
  it.arena.set_stream(s);
  const Inputs in = make_inputs(pr.m, pr.n, &pr.A, pr.c, pr.lc, pr.uc, pr.lv, pr.uv, &prm);
  if (!pr.x_out || (pr.m > 0 && !pr.y_out)) throw PdlpError(-1, "null output array");
  DeviceArena& a = it.arena;
  DeviceArena tmp;  // the staged input and the setup temporaries, freed after setup
  tmp.set_stream(s);
  DevInputs d = stage_inputs(tmp, in, s);
  validate(tmp, in, d, s);
  Problem<T>& P = it.P;
  build_problem<T>(a, in, d, prm.ruiz_iters, prm.pc_alpha, P, s, true, &tmp);
  const int64_t m = P.m, n = P.n;
  BatchLP<T>& L = it.d;
  L.A = P.A;
  L.AT = P.AT;
  L.m = m;
  L.n = n;
  L.c = P.c;
  L.lc = P.lc;
  L.uc = P.uc;
  L.lv = P.lv;
  L.uv = P.uv;
  L.o = OrigVecs{P.orig.c, P.orig.lc, P.orig.uc, P.orig.lv, P.orig.uv,
                 P.d1,     P.d2,      P.inv_d1,  P.inv_d2};
  L.perm_r = P.perm_r;
  L.perm_c = P.perm_c;
  L.c_norm = P.c_norm;
  L.b_norm = P.b_norm;
  L.eta0 = P.max_abs > 0.0 ? 1.0 / P.max_abs : 1.0;
  L.omega0 = (P.c_norm_s > 0.0 && P.b_norm_s > 0.0) ? P.c_norm_s / P.b_norm_s : 1.0;
  for (int q = 0; q < 2; ++q) {
    L.X[q] = a.alloc<T>(n);
    L.ATY[q] = a.alloc<T>(n);
    L.Y[q] = a.alloc<T>(m);
    L.AX[q] = a.alloc<T>(m);
  }
  using S = typename BatchSum<T>::type;
  L.Sx = a.alloc<S>(n);
  L.Sy = a.alloc<S>(m);
  L.a_col16 = n <= 65536 ? sell_col16(a, P.A, s) : nullptr;
  L.at_col16 = m <= 65536 ? sell_col16(a, P.AT, s) : nullptr;
  L.gp_row = a.alloc<float4>(m);
  L.gp_x = a.alloc<float>(3 * n);
  L.X0 = a.alloc<T>(n);
  L.Y0 = a.alloc<T>(m);
  L.Xa = a.alloc<T>(n);
  L.ATYa = a.alloc<T>(n);
  L.Ya = a.alloc<T>(m);
  L.AXa = a.alloc<T>(m);
  if (prm.detect_infeasibility) {
    L.yd = a.alloc<T>(m);
    L.atyd = a.alloc<T>(n);
    L.xb = a.alloc<T>(3 * n);
    L.axb = a.alloc<T>(3 * m);
  }
  if (in.on_device) {
    L.x_out = pr.x_out;
    L.y_out = pr.y_out;
  } else {
    it.dx = a.alloc<double>(n);
    it.dy = a.alloc<double>(m);
    L.x_out = it.dx;
    L.y_out = it.dy;
  }
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  it.launches = P.launches;
  it.setup_s = secs_since(t0);
}

// Work of one iteration of an LP (bytes of its two products and vectors, FP32 units),
// the key of the largest-first order and of the autotuner's throughput.
static double lp_work(int64_t m, int64_t n, int64_t nnz) {
  return 2.0 * 8.0 * (double)nnz + 11.0 * 4.0 * (double)(m + n);
}

template <class T>
static int batch_persistent(int64_t count, const pdlp_problem* problems, const pdlp_params& prm,
                            int tune, int* status_out, pdlp_stats* stats_out, int* tune_out) {
  const auto t_call = Clock::now();
  int dev = 0;
  PDLP_CUDA_CHECK(cudaGetDevice(&dev));
  StreamGuard sg(prm.cuda_stream);
  cudaStream_t s = sg.s;
  // ---- setup of every LP on worker streams ----
  std::vector<std::unique_ptr<BatchItem<T>>> items(count);
  for (auto& p : items) p.reset(new BatchItem<T>());
  {
    // the setup of one small LP is a chain of short launches and a few host
    // synchronisations, so many LPs are set up at once (48 workers instead of 16 changed
    // the 1024-LP uneven batch's setup by under 5%)
    const int64_t workers = std::max<int64_t>(1, std::min<int64_t>(kSetupWorkers, count));
    std::atomic<int64_t> next{0};
    auto work = [&]() {
      cudaStream_t ws = nullptr;
      const bool ok = cudaSetDevice(dev) == cudaSuccess &&
                      cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) == cudaSuccess;
      for (;;) {
        const int64_t i = next.fetch_add(1);
        if (i >= count) break;
        BatchItem<T>& it = *items[i];
        if (!ok) {
          it.code = PDLP_CUDA_ERROR;
          it.err = "could not create a stream for a worker";
          continue;
        }
        try {
          batch_setup_one<T>(it, problems[i], prm, ws);
        } catch (const PdlpError& e) {
          it.code = e.code < 0 ? e.code : PDLP_CUDA_ERROR;
          it.err = e.what();
        } catch (const std::exception& e) {
          it.code = PDLP_CUDA_ERROR;
          it.err = e.what();
        }
        // the arena is released on the launch stream once the batch is done
        if (ws) cudaStreamSynchronize(ws);
        it.arena.set_stream(s);
      }
      if (ws) cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int64_t w = 1; w < workers; ++w) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
  }
  std::vector<int32_t> order;
  for (int64_t i = 0; i < count; ++i)
    if (items[i]->code == 0) order.push_back((int32_t)i);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    const BatchLP<T>& x = items[a]->d;
    const BatchLP<T>& y = items[b]->d;
    return lp_work(x.m, x.n, x.A.nnz) > lp_work(y.m, y.n, y.A.nnz);
  });
  const int nv = (int)order.size();
  double t_setup = secs_since(t_call);

  DeviceArena arena;
  arena.set_stream(s);
  std::vector<BatchResult> hres(count);
  int chosen = 1;
  double tune_s = 0.0, launch_s = 0.0;
  if (nv > 0) {
    std::vector<BatchLP<T>> hd(count);
    for (int64_t i = 0; i < count; ++i) hd[i] = items[i]->d;
    BatchLP<T>* dl = arena.alloc<BatchLP<T>>(count);
    int32_t* dord = arena.alloc<int32_t>(nv);
    BatchResult* dres = arena.alloc<BatchResult>(count);
    unsigned int* queue = arena.alloc<unsigned int>(1);
    const int64_t tab_len = std::min<int64_t>(prm.max_iters + 1, (int64_t)1 << 16);
    double* tab = arena.alloc<double>(2 * tab_len);
    fill_step_table(tab, tab_len, s);
    PDLP_CUDA_CHECK(cudaMemcpyAsync(dl, hd.data(), sizeof(BatchLP<T>) * count, cudaMemcpyHostToDevice, s));
    PDLP_CUDA_CHECK(cudaMemcpyAsync(dord, order.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, s));
    PDLP_CUDA_CHECK(cudaMemsetAsync(dres, 0, sizeof(BatchResult) * count, s));
    BatchParams bp{};
    bp.eps_rel_kkt = prm.eps_rel_kkt;
    bp.eps_abs_feas = prm.eps_abs_feas;
    bp.eps_rel_gap = prm.eps_rel_gap;
    bp.termination_mode = prm.termination_mode;
    bp.reduced_costs = prm.reduced_costs;
    bp.check_period = prm.check_period;
    bp.max_retries = prm.max_step_retries;
    bp.detect_infeasibility = prm.detect_infeasibility;
    bp.max_iters = prm.max_iters;
    bp.time_limit_s = prm.time_limit_s;
    bp.beta_suff = prm.beta_suff;
    bp.beta_nec = prm.beta_nec;
    bp.beta_art = prm.beta_art;
    bp.theta = prm.theta;
    bp.eps_zero = prm.eps_zero;
    bp.fixed_step = prm.fixed_step;
    bp.fixed_omega = prm.fixed_omega;
    bp.eps_infeas = prm.eps_infeas;
    bp.step_tab = tab;
    bp.step_len = tab_len;

    if (tune == 0) {
      // Autotuner: time 192 iterations (termination off) of a sample of the batch spread
      // over its size order under every launch configuration, and keep the one with the
      // highest throughput (work of the iterations done divided by the time the LPs
      // occupied their CTAs, per CTA slot of the device).  Restart criterion (iii) is
      // off in the probe, so it evaluates at the periodic checks only -- one evaluation
      // per check_period iterations, the mix of a long solve (with (iii), the first 128
      // iterations of an LP hold 8 evaluations, which ranked the configurations by
      // their evaluation cost).
      const auto t0 = Clock::now();
      const int nconf = batch_config_count();
      int ns = 1;
      for (int c = 1; c <= nconf; ++c) ns = std::max(ns, batch_resident_ctas<T>(c));
      ns = std::min(ns, nv);
      std::vector<int32_t> samp(ns);
      for (int q = 0; q < ns; ++q) samp[q] = order[(int64_t)q * nv / ns];
      int32_t* dsamp = arena.alloc<int32_t>(ns);
      BatchResult* pres = arena.alloc<BatchResult>(count);
      PDLP_CUDA_CHECK(cudaMemcpyAsync(dsamp, samp.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
      BatchParams pp = bp;
      pp.max_iters = std::min<int64_t>(3 * (int64_t)std::max(1, prm.check_period), 512);
      pp.beta_art = 1.0;
      pp.eps_rel_kkt = -1.0;
      pp.termination_mode = 0;
      pp.detect_infeasibility = 0;
      pp.time_limit_s = INFINITY;
      double best = -1.0;
      std::vector<BatchResult> pr(count);
      for (int c = 1; c <= nconf; ++c) {
        PDLP_CUDA_CHECK(cudaMemsetAsync(queue, 0, sizeof(unsigned int), s));
        const int slots = std::min(ns, batch_resident_ctas<T>(c));
        launch_batch<T>(dl, dsamp, ns, pp, pres, queue, c, slots, s);
        PDLP_CUDA_CHECK(cudaMemcpyAsync(pr.data(), pres, sizeof(BatchResult) * count, cudaMemcpyDeviceToHost, s));
        PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
        double work = 0.0, secs = 0.0;
        for (int q = 0; q < ns; ++q) {
          const BatchLP<T>& L = hd[samp[q]];
          work += lp_work(L.m, L.n, L.A.nnz) * (double)pr[samp[q]].k;
          secs += pr[samp[q]].seconds;
        }
        // per CTA slot, times the LPs the real launch runs at once
        const double rate =
            secs > 0.0 ? work / secs * std::min(nv, batch_resident_ctas<T>(c)) : 0.0;
        if (rate > best) {
          best = rate;
          chosen = c;
        }
      }
      tune_s = secs_since(t0);
    } else {
      chosen = tune;
    }
    const int ctas = std::min(nv, batch_resident_ctas<T>(chosen));
    PDLP_CUDA_CHECK(cudaMemsetAsync(queue, 0, sizeof(unsigned int), s));
    cudaEvent_t ev[2];
    PDLP_CUDA_CHECK(cudaEventCreate(&ev[0]));
    PDLP_CUDA_CHECK(cudaEventCreate(&ev[1]));
    PDLP_CUDA_CHECK(cudaEventRecord(ev[0], s));
    launch_batch<T>(dl, dord, nv, bp, dres, queue, chosen, ctas, s);
    PDLP_CUDA_CHECK(cudaEventRecord(ev[1], s));
    PDLP_CUDA_CHECK(cudaMemcpyAsync(hres.data(), dres, sizeof(BatchResult) * count, cudaMemcpyDeviceToHost, s));
    for (int q = 0; q < nv; ++q) {
      const BatchItem<T>& it = *items[order[q]];
      if (!it.dx) continue;
      const pdlp_problem& pb = problems[order[q]];
      PDLP_CUDA_CHECK(cudaMemcpyAsync(pb.x_out, it.dx, sizeof(double) * pb.n, cudaMemcpyDeviceToHost, s));
      if (pb.m) PDLP_CUDA_CHECK(cudaMemcpyAsync(pb.y_out, it.dy, sizeof(double) * pb.m, cudaMemcpyDeviceToHost, s));
    }
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    float ms = 0.0f;
    PDLP_CUDA_CHECK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    launch_s = 1e-3 * ms;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  if (tune_out) *tune_out = chosen;
  const double t_total = secs_since(t_call);
  std::string first_error;
  for (int64_t i = 0; i < count; ++i) {
    const BatchItem<T>& it = *items[i];
    if (it.code != 0) {
      status_out[i] = it.code;
      if (first_error.empty()) first_error = "problem " + std::to_string(i) + ": " + it.err;
      if (stats_out) {
        std::memset(&stats_out[i], 0, sizeof(pdlp_stats));
        stats_out[i].status = it.code;
      }
      continue;
    }
    const BatchResult& r = hres[i];
    status_out[i] = r.status;
    if (!stats_out) continue;
    pdlp_stats* st = &stats_out[i];
    std::memset(st, 0, sizeof(*st));
    st->status = r.status;
    st->iterations = r.k;
    st->attempts = r.attempts;
    st->rejected_steps = r.rejected;
    for (int q = 0; q < 3; ++q) st->restarts[q] = r.restarts[q];
    st->kkt_passes = 0.5 * (double)(r.attempts + r.k);
    st->rel_kkt = r.rel_kkt;
    st->rel_primal = r.rel_primal;
    st->rel_dual = r.rel_dual;
    st->rel_gap = r.rel_gap;
    st->primal_res_l2 = r.pres2;
    st->dual_res_l2 = r.dres2;
    st->primal_res_inf = r.pres_inf;
    st->dual_res_inf = r.dres_inf;
    st->pobj = r.pobj;
    st->dobj = r.dobj;
    st->paper_gap = r.paper_gap;
    st->primal_res_rel_inf = r.pres_rel_inf;
    st->dual_res_rel_inf = r.dres_rel_inf;
    st->omega = r.omega;
    st->eta_hat = r.eta_hat;
    st->seconds_setup = it.setup_s;
    st->seconds_solve = r.seconds;
    st->seconds_total = t_total;
    st->evaluations = r.evaluations;
    st->gap_evals = r.gap_evals;
    st->gap_fallbacks = r.gap_fallbacks;
    st->gap_failures = r.gap_failures;
    st->kernel_launches = it.launches + 1;
    st->device_bytes = (int64_t)it.arena.total();
    const double v = (double)sizeof(T);
    const int64_t m = it.P.m, n = it.P.n, nnz = it.P.nnz;
    st->bytes_spmv_a = (double)(m + 1) * 8 + (double)nnz * (4 + v) + (double)n * v + 6.0 * m * v;
    st->bytes_spmv_at = (double)(n + 1) * 8 + (double)nnz * (4 + v) + (double)m * v +
                        6.0 * (double)n * v + 6.0 * (double)m * v;
    // device time by phase (the LP's time split by its SM cycles per phase)
    double cyc = 0.0;
    for (int q = 0; q < 8; ++q) cyc += (double)r.cycles[q];
    const double per = cyc > 0.0 ? 1e3 * r.seconds / cyc : 0.0;
    st->ms_primal = per * (double)r.cycles[0];
    st->ms_spmv_a = per * (double)r.cycles[1];
    st->ms_spmv_at = per * (double)r.cycles[2];
    st->ms_checks = per * (double)(r.cycles[3] + r.cycles[4] + r.cycles[5] + r.cycles[6] +
                                   r.cycles[7]);
    st->ms_gap = per * (double)r.cycles[5];
    st->ms_kkt = per * (double)r.cycles[6];
    st->ms_infeas = per * (double)r.cycles[7];
    st->batch_launch_s = launch_s;
    st->batch_sm = r.sm;
  }
  (void)tune_s;
  (void)t_setup;
  if (!first_error.empty()) set_last_error(first_error);
  return 0;
}

}  // namespace pdlp


// ---------------------------------------------------------------------------
// persistent unrolled-PDHG batch: every LP set up as pdlp_unrolled_pdhg sets it up
// (identity scaling, renumbered SELL layouts, FP32 copies for an FP32 forward) on worker
// streams, then one launch of k_unroll_batch
// ---------------------------------------------------------------------------
namespace pdlp {

template <class T>
struct UnrollItem {
  DeviceArena arena;
  Problem<double> P;
  Problem<float> P32;
  UnrollLP<T> d{};
  bool on_device = false;
  double* host_out[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* dev_out[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t out_len[7] = {0, 0, 0, 0, 0, 0, 0};
  int code = 0;
  std::string err;
  double setup_s[4] = {0.0, 0.0, 0.0, 0.0};  // host time: staging and validation, layouts,
                                             // FP32 copy, buffers and the closing sync
};

template <class T>
static void unroll_setup_one(UnrollItem<T>& it, const pdlp_unrolled_problem& u,
                             const pdlp_params& prm, cudaStream_t s) {
  it.arena.set_stream(s);
  const Inputs in = make_inputs(u.m, u.n, &u.A, u.c, u.lc, u.uc, u.lv, u.uv, &prm);
  if (u.K < 0) throw PdlpError(-1, "K < 0");
  if (!(u.eta > 0.0) || !std::isfinite(u.eta) || !(u.omega > 0.0) || !std::isfinite(u.omega))
    throw PdlpError(-1, "eta and omega must be positive and finite");
  if (!u.x_out || (u.m > 0 && !u.y_out)) throw PdlpError(-1, "null output");
  if (u.gx && u.m > 0 && !u.gy) throw PdlpError(-1, "gx without gy");
  if (unroll_smem_need(u.m, u.n, sizeof(T)) > unroll_smem_max())
    throw PdlpError(-1, "LP too large for the persistent unrolled batch (its state must fit "
                        "one CTA's shared memory: 2 (m + n) forward values and m + n FP64 "
                        "adjoints in " + std::to_string(unroll_smem_max()) +
                        " bytes); use pdlp_unrolled_pdhg_batch");
  DeviceArena& a = it.arena;
  const int64_t m = u.m, n = u.n;
  auto t0 = Clock::now();
  DevInputs d = stage_inputs(a, in, s);
  validate(a, in, d, s);
  it.setup_s[0] = secs_since(t0);
  t0 = Clock::now();
  build_problem<double>(a, in, d, 0, 0.0, it.P, s);  // identity scaling, renumbered
  it.setup_s[1] = secs_since(t0);
  t0 = Clock::now();
  UnrollLP<T>& L = it.d;
  L.m = m;
  L.n = n;
  L.K = u.K;
  L.C = u.checkpoint_every > 0 ? u.checkpoint_every : 50;
  L.tau = u.eta / u.omega;
  L.sigma = u.eta * u.omega;
  L.tau_t = (T)L.tau;
  L.sigma_t = (T)L.sigma;
  L.A64 = it.P.A;
  L.AT64 = it.P.AT;
  L.perm_r = it.P.perm_r;
  L.perm_c = it.P.perm_c;
  if constexpr (std::is_same<T, double>::value) {
    L.A = it.P.A;
    L.AT = it.P.AT;
    L.c = it.P.c;
    L.lc = it.P.lc;
    L.uc = it.P.uc;
    L.lv = it.P.lv;
    L.uv = it.P.uv;
  } else {
    // FP32 forward: the same renumbered LP with FP32 values and vectors
    narrow_problem(a, it.P, it.P32, s);
    L.A = it.P32.A;
    L.AT = it.P32.AT;
    L.c = it.P32.c;
    L.lc = it.P32.lc;
    L.uc = it.P32.uc;
    L.lv = it.P32.lv;
    L.uv = it.P32.uv;
  }
  it.setup_s[2] = secs_since(t0);
  t0 = Clock::now();
  const int64_t state = 2 * (m + n);
  L.cp = a.alloc<T>((L.K / L.C + 1) * state);
  L.seg = a.alloc<T>((L.C + 1) * state);
  it.on_device = in.on_device;
  // outputs: the caller's device arrays, or device arrays copied back after the launch
  double* outs[7] = {u.x_out, u.y_out, u.grad_c, u.grad_lc, u.grad_uc, u.grad_lv, u.grad_uv};
  const int64_t lens[7] = {n, m, n, m, m, n, n};
  for (int q = 0; q < 7; ++q) {
    it.out_len[q] = lens[q];
    if (!outs[q] || (q >= 2 && !u.gx)) continue;
    it.host_out[q] = outs[q];
    it.dev_out[q] = in.on_device ? outs[q] : a.alloc<double>(lens[q]);
  }
  L.x_out = it.dev_out[0];
  L.y_out = it.dev_out[1];
  for (int q = 0; q < 5; ++q) L.gout[q] = it.dev_out[2 + q];
  if (u.gx) {
    // upstream gradient into the renumbered order
    auto renumbered = [&](const double* src, int64_t len, const int32_t* perm) -> const double* {
      if (!src || len == 0) return nullptr;
      const double* dsrc = src;
      if (!in.on_device) {
        double* t = a.alloc<double>(len);
        copy_in(t, src, sizeof(double) * len, false, s);
        dsrc = t;
      }
      double* out = a.alloc<double>(len);
      gather_f64(dsrc, perm, out, len, s);
      return out;
    };
    L.gx = renumbered(u.gx, n, it.P.perm_c);
    L.gy = renumbered(u.gy, m, it.P.perm_r);
    L.bx = a.alloc<double>(n);
    L.by = a.alloc<double>(m);
    const int64_t glen[5] = {n, m, m, n, n};
    for (int q = 0; q < 5; ++q) L.g[q] = a.alloc<double>(glen[q]);
  }
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  it.setup_s[3] = secs_since(t0);
}

template <class T>
static int unroll_batch_persistent(int64_t count, const pdlp_unrolled_problem* problems,
                                   const pdlp_params& prm, int* status_out) {
  int dev = 0;
  PDLP_CUDA_CHECK(cudaGetDevice(&dev));
  StreamGuard sg(prm.cuda_stream);
  cudaStream_t s = sg.s;
  std::vector<std::unique_ptr<UnrollItem<T>>> items(count);
  for (auto& p : items) p.reset(new UnrollItem<T>());
  const auto t_setup = Clock::now();
  {
    // the setup of one small LP is a chain of short launches and a few host
    // synchronisations, so many LPs are set up at once (48 workers instead of 16 changed
    // the 1024-LP uneven batch's setup by under 5%)
    const int64_t workers = std::max<int64_t>(1, std::min<int64_t>(kSetupWorkers, count));
    std::atomic<int64_t> next{0};
    auto work = [&]() {
      cudaStream_t ws = nullptr;
      const bool ok = cudaSetDevice(dev) == cudaSuccess &&
                      cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) == cudaSuccess;
      for (;;) {
        const int64_t i = next.fetch_add(1);
        if (i >= count) break;
        UnrollItem<T>& it = *items[i];
        if (!ok) {
          it.code = PDLP_CUDA_ERROR;
          it.err = "could not create a stream for a worker";
          continue;
        }
        try {
          unroll_setup_one<T>(it, problems[i], prm, ws);
        } catch (const PdlpError& e) {
          it.code = e.code < 0 ? e.code : PDLP_CUDA_ERROR;
          it.err = e.what();
        } catch (const std::exception& e) {
          it.code = PDLP_CUDA_ERROR;
          it.err = e.what();
        }
        if (ws) cudaStreamSynchronize(ws);
        it.arena.set_stream(s);
      }
      if (ws) cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int64_t w = 1; w < workers; ++w) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
  }
  const double setup_s = secs_since(t_setup);
  const auto t_run = Clock::now();
  std::vector<int32_t> order;
  for (int64_t i = 0; i < count; ++i)
    if (items[i]->code == 0) order.push_back((int32_t)i);
  // the longest runs first: steps times the work of one step
  auto work_of = [&](int32_t i) {
    const UnrollLP<T>& L = items[i]->d;
    return (double)(L.K + 1) * (double)(L.A.nnz + L.m + L.n) * (L.gx ? 4.0 : 1.0);
  };
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return work_of(a) > work_of(b); });
  const int nv = (int)order.size();
  DeviceArena arena;
  arena.set_stream(s);
  if (nv > 0) {
    std::vector<UnrollLP<T>> hd(count);
    for (int64_t i = 0; i < count; ++i) hd[i] = items[i]->d;
    UnrollLP<T>* dl = arena.alloc<UnrollLP<T>>(count);
    int32_t* dord = arena.alloc<int32_t>(nv);
    unsigned int* queue = arena.alloc<unsigned int>(1);
    PDLP_CUDA_CHECK(cudaMemcpyAsync(dl, hd.data(), sizeof(UnrollLP<T>) * count, cudaMemcpyHostToDevice, s));
    PDLP_CUDA_CHECK(cudaMemcpyAsync(dord, order.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, s));
    PDLP_CUDA_CHECK(cudaMemsetAsync(queue, 0, sizeof(unsigned int), s));
    launch_unroll_batch<T>(dl, dord, nv, queue, std::min(nv, unroll_resident_ctas<T>()), s);
    for (int q = 0; q < nv; ++q) {
      const UnrollItem<T>& it = *items[order[q]];
      if (it.on_device) continue;
      for (int k = 0; k < 7; ++k)
        if (it.host_out[k] && it.out_len[k] > 0)
          PDLP_CUDA_CHECK(cudaMemcpyAsync(it.host_out[k], it.dev_out[k], sizeof(double) * it.out_len[k],
                                          cudaMemcpyDeviceToHost, s));
    }
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  }
  const double run_s = secs_since(t_run);
  std::string first_error;
  for (int64_t i = 0; i < count; ++i) {
    status_out[i] = items[i]->code;
    if (items[i]->code != 0 && first_error.empty())
      first_error = "problem " + std::to_string(i) + ": " + items[i]->err;
  }
  if (!first_error.empty()) set_last_error(first_error);
  if (prm.verbose) {
    double per[4] = {0.0, 0.0, 0.0, 0.0};  // summed over the LPs (the workers overlap)
    for (const auto& it : items)
      for (int q = 0; q < 4; ++q) per[q] += it->setup_s[q];
    const auto t_rel = Clock::now();
    arena.release();
    items.clear();
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    std::fprintf(stderr,
                 "pdlp: unrolled batch of %lld LPs: setup %.3f s (summed over LPs: staging %.3f, "
                 "layouts %.3f, FP32 copy %.3f, buffers %.3f), launch and copies %.3f s, "
                 "release %.3f s\n",
                 (long long)count, setup_s, per[0], per[1], per[2], per[3], run_s,
                 secs_since(t_rel));
  }
  return 0;
}

}  // namespace pdlp

extern "C" {

void pdlp_params_default(pdlp_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps_rel_kkt = 1e-8;
  p->termination_mode = 0;
  p->eps_abs_feas = 1e-8;
  p->eps_rel_gap = 1e-2;
  p->max_iters = 1000000000LL;
  p->time_limit_s = INFINITY;
  p->ruiz_iters = 10;
  p->pc_alpha = 1.0;
  p->check_period = 64;
  p->beta_suff = 0.1;
  p->beta_nec = 0.9;
  p->beta_art = 0.5;
  p->theta = 0.5;
  p->eps_zero = 1e-10;
  p->max_step_retries = 60;
  p->precision = PDLP_FP64;
  p->inputs_on_device = 0;
  p->cuda_stream = nullptr;
  p->trace_iters = 0;
  p->trace_out = nullptr;
  p->profile = 0;
  p->verbose = 0;
  p->feasibility_polishing = 0;
  p->detect_infeasibility = 1;
  p->eps_infeas = 1e-9;
  p->reduced_costs = 0;
  p->polish_log_cap = 0;
  p->polish_log = nullptr;
  p->fixed_step = 0.0;
  p->fixed_omega = 0.0;
}

const char* pdlp_last_error(void) { return g_last_error; }

int pdlp_unrolled_pdhg_batch_persistent(int64_t count, const pdlp_unrolled_problem* problems,
                                        const pdlp_params* p, int* status_out) {
  try {
    if (count < 0) throw PdlpError(-1, "pdlp_unrolled_pdhg_batch_persistent: count < 0");
    if (count > INT32_MAX)
      throw PdlpError(-1, "pdlp_unrolled_pdhg_batch_persistent: count > 2^31-1");
    if (count > 0 && (!problems || !status_out))
      throw PdlpError(-1, "pdlp_unrolled_pdhg_batch_persistent: null problems or status_out");
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    if (prm.precision == PDLP_FP32_BULK)
      return unroll_batch_persistent<float>(count, problems, prm, status_out);
    return unroll_batch_persistent<double>(count, problems, prm, status_out);
  } catch (...) {
    return handle_exception();
  }
}


int pdlp_solve(int64_t m, int64_t n, const pdlp_csr* A, const double* c, const double* lc,
               const double* uc, const double* lv, const double* uv, const pdlp_params* p,
               double* x_out, double* y_out, pdlp_stats* stats) {
  try {
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    const Inputs in = make_inputs(m, n, A, c, lc, uc, lv, uv, &prm);
    if (!x_out || (m > 0 && !y_out)) throw PdlpError(-1, "null output array");
    check_params(prm);
    StreamGuard sg(prm.cuda_stream);
    if (prm.precision == PDLP_FP32_BULK) {
      Solver<float> S(prm, sg.s);
      return S.run(in, x_out, y_out, stats);
    }
    Solver<double> S(prm, sg.s);
    return S.run(in, x_out, y_out, stats);
  } catch (...) {
    return handle_exception();
  }
}

int pdlp_solve_batch(int64_t count, const pdlp_problem* problems, const pdlp_params* p,
                     int concurrency, int* status_out, pdlp_stats* stats_out) {
  try {
    if (count < 0) throw PdlpError(-1, "pdlp_solve_batch: count < 0");
    if (count > 0 && (!problems || !status_out))
      throw PdlpError(-1, "pdlp_solve_batch: null problems or status_out");
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    prm.trace_iters = 0;
    prm.trace_out = nullptr;
    prm.polish_log = nullptr;
    prm.polish_log_cap = 0;
    return pdlp::run_batch("pdlp_solve_batch", count, prm, concurrency, status_out,
                     [&](int64_t i, const pdlp_params& q) {
                       const pdlp_problem& pb = problems[i];
                       return pdlp_solve(pb.m, pb.n, &pb.A, pb.c, pb.lc, pb.uc, pb.lv, pb.uv, &q,
                                         pb.x_out, pb.y_out, stats_out ? &stats_out[i] : nullptr);
                     });
  } catch (...) {
    return handle_exception();
  }
}

int pdlp_solve_batch_persistent(int64_t count, const pdlp_problem* problems, const pdlp_params* p,
                                int tune, int* status_out, pdlp_stats* stats_out, int* tune_out) {
  try {
    if (count < 0) throw PdlpError(-1, "pdlp_solve_batch_persistent: count < 0");
    if (count > INT32_MAX) throw PdlpError(-1, "pdlp_solve_batch_persistent: count > 2^31-1");
    if (count > 0 && (!problems || !status_out))
      throw PdlpError(-1, "pdlp_solve_batch_persistent: null problems or status_out");
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    check_params(prm);
    if (prm.feasibility_polishing)
      throw PdlpError(-1, "pdlp_solve_batch_persistent: feasibility polishing is not available "
                          "in the persistent batch (use pdlp_solve_batch)");
    if (tune < 0 || tune > batch_config_count())
      throw PdlpError(-1, "tune must be 0 (autotune) or a configuration 1.." +
                              std::to_string(batch_config_count()));
    if (prm.precision == PDLP_FP32_BULK)
      return batch_persistent<float>(count, problems, prm, tune, status_out, stats_out, tune_out);
    return batch_persistent<double>(count, problems, prm, tune, status_out, stats_out, tune_out);
  } catch (...) {
    return handle_exception();
  }
}

int pdlp_unrolled_pdhg_batch(int64_t count, const pdlp_unrolled_problem* problems,
                             const pdlp_params* p, int concurrency, int* status_out) {
  try {
    if (count < 0) throw PdlpError(-1, "pdlp_unrolled_pdhg_batch: count < 0");
    if (count > 0 && (!problems || !status_out))
      throw PdlpError(-1, "pdlp_unrolled_pdhg_batch: null problems or status_out");
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    return pdlp::run_batch("pdlp_unrolled_pdhg_batch", count, prm, concurrency, status_out,
                     [&](int64_t i, const pdlp_params& q) {
                       const pdlp_unrolled_problem& u = problems[i];
                       return pdlp_unrolled_pdhg(u.m, u.n, &u.A, u.c, u.lc, u.uc, u.lv, u.uv, u.K,
                                                 u.eta, u.omega, u.checkpoint_every, u.gx, u.gy,
                                                 &q, u.x_out, u.y_out, u.grad_c, u.grad_lc,
                                                 u.grad_uc, u.grad_lv, u.grad_uv);
                     });
  } catch (...) {
    return handle_exception();
  }
}

int pdlp_unrolled_pdhg(int64_t m, int64_t n, const pdlp_csr* A, const double* c,
                       const double* lc, const double* uc, const double* lv, const double* uv,
                       int64_t K, double eta, double omega, int64_t checkpoint_every,
                       const double* gx, const double* gy, const pdlp_params* p, double* x_out,
                       double* y_out, double* grad_c, double* grad_lc, double* grad_uc,
                       double* grad_lv, double* grad_uv) {
  try {
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    const Inputs in = make_inputs(m, n, A, c, lc, uc, lv, uv, &prm);
    if (K < 0) throw PdlpError(-1, "pdlp_unrolled_pdhg: K < 0");
    if (!(eta > 0.0) || !std::isfinite(eta) || !(omega > 0.0) || !std::isfinite(omega))
      throw PdlpError(-1, "pdlp_unrolled_pdhg: eta and omega must be positive and finite");
    if (!x_out || (m > 0 && !y_out)) throw PdlpError(-1, "pdlp_unrolled_pdhg: null output");
    if (gx && m > 0 && !gy) throw PdlpError(-1, "pdlp_unrolled_pdhg: gx without gy");
    StreamGuard sg(prm.cuda_stream);
    const cudaStream_t s = sg.s;
    DeviceArena arena;
    arena.set_stream(s);
    DevInputs d = stage_inputs(arena, in, s);
    validate(arena, in, d, s);
    Problem<double> P;
    build_problem<double>(arena, in, d, 0, 0.0, P, s);  // identity scaling, renumbered
    const UnrolledLp L{P.m, P.n, P.A, P.AT, P.c, P.lc, P.uc, P.lv, P.uv, P.perm_r, P.perm_c};
    const UnrolledProblem U{&L, eta / omega, eta * omega, spmv_grid<double>(P.A, kEpiPlain),
                            spmv_grid<double>(P.AT, kEpiPlain)};
    // device views of the caller's arrays
    auto dev_in = [&](const double* h, int64_t len) -> const double* {
      if (!h || in.on_device) return h;
      double* dptr = arena.alloc<double>(len);
      copy_in(dptr, h, sizeof(double) * len, false, s);
      return dptr;
    };
    auto dev_out = [&](double* h, int64_t len) -> double* {
      if (!h || in.on_device) return h;
      return arena.alloc<double>(len);
    };
    const double* dgx = dev_in(gx, n);
    const double* dgy = dev_in(gy, m);
    double* dx = dev_out(x_out, n);
    double* dy = dev_out(y_out, m);
    UnrolledGrads G{dev_out(grad_c, n), dev_out(grad_lc, m), dev_out(grad_uc, m),
                    dev_out(grad_lv, n), dev_out(grad_uv, n)};
    if (gx && m == 0) dgy = nullptr;
    const int64_t every = checkpoint_every > 0 ? checkpoint_every : 50;
    if (prm.precision == PDLP_FP32_BULK) {
      // FP32 forward: the same renumbered LP with FP32 values and vectors (identity
      // scaling leaves the staged values as given); the reverse pass stays FP64
      Problem<float> P32;
      narrow_problem(arena, P, P32, s);
      const UnrolledFwd<float> F{P32.A, P32.AT, P32.c, P32.lc, P32.uc, P32.lv, P32.uv,
                                 (float)(eta / omega), (float)(eta * omega),
                                 spmv_grid<float>(P32.A, kEpiPlain), spmv_grid<float>(P32.AT, kEpiPlain)};
      unrolled_pdhg_run<float>(arena, U, F, K, every, dgx, dgy, dx, dy, gx ? &G : nullptr, s);
    } else {
      const UnrolledFwd<double> F{P.A, P.AT, P.c, P.lc, P.uc, P.lv, P.uv, U.tau, U.sigma,
                                  U.grid_a, U.grid_at};
      unrolled_pdhg_run<double>(arena, U, F, K, every, dgx, dgy, dx, dy, gx ? &G : nullptr, s);
    }
    if (!in.on_device) {
      auto back = [&](double* h, const double* dptr, int64_t len) {
        if (h && len > 0)
          PDLP_CUDA_CHECK(cudaMemcpyAsync(h, dptr, sizeof(double) * len, cudaMemcpyDeviceToHost, s));
      };
      back(x_out, dx, n);
      back(y_out, dy, m);
      if (gx) {
        back(grad_c, G.c, n);
        back(grad_lc, G.lc, m);
        back(grad_uc, G.uc, m);
        back(grad_lv, G.lv, n);
        back(grad_uv, G.uv, n);
      }
    }
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    return 0;
  } catch (...) {
    return handle_exception();
  }
}

int pdlp_precondition(int64_t m, int64_t n, const pdlp_csr* A, const pdlp_params* p,
                      double* d1_out, double* d2_out, double* scaled_val_out) {
  try {
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    // the vectors are not needed: use n zeros / unit bounds as placeholders
    std::vector<double> zn((size_t)n, 0.0), on((size_t)n, 1.0), zm((size_t)m, 0.0);
    Inputs in = make_inputs(m, n, A, zn.data(), zm.data(), zm.data(), zn.data(), on.data(), &prm);
    StreamGuard sg(prm.cuda_stream);
    cudaStream_t s = sg.s;
    DeviceArena arena;
    arena.set_stream(s);
    // stage the matrix from its own memory space and the placeholder vectors from host
    Inputs mat = in;
    DevInputs d;
    d.row_ptr = arena.alloc<int64_t>(m + 1);
    d.col = arena.alloc<int32_t>(in.nnz);
    d.val = arena.alloc<double>(in.nnz);
    copy_in(d.row_ptr, in.row_ptr, sizeof(int64_t) * (m + 1), in.on_device, s);
    copy_in(d.col, in.col, sizeof(int32_t) * in.nnz, in.on_device, s);
    copy_in(d.val, in.val, sizeof(double) * in.nnz, in.on_device, s);
    mat.on_device = false;
    d.c = arena.alloc<double>(n);
    d.lv = arena.alloc<double>(n);
    d.uv = arena.alloc<double>(n);
    d.lc = arena.alloc<double>(m);
    d.uc = arena.alloc<double>(m);
    copy_in(d.c, zn.data(), sizeof(double) * n, false, s);
    copy_in(d.lv, zn.data(), sizeof(double) * n, false, s);
    copy_in(d.uv, on.data(), sizeof(double) * n, false, s);
    copy_in(d.lc, zm.data(), sizeof(double) * m, false, s);
    copy_in(d.uc, zm.data(), sizeof(double) * m, false, s);
    validate(arena, mat, d, s);
    Problem<double> P;
    build_problem<double>(arena, mat, d, prm.ruiz_iters, prm.pc_alpha, P, s, false);
    const cudaMemcpyKind k = in.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (d1_out && m) PDLP_CUDA_CHECK(cudaMemcpyAsync(d1_out, P.d1, sizeof(double) * m, k, s));
    if (d2_out) PDLP_CUDA_CHECK(cudaMemcpyAsync(d2_out, P.d2, sizeof(double) * n, k, s));
    if (scaled_val_out && in.nnz)
      PDLP_CUDA_CHECK(cudaMemcpyAsync(scaled_val_out, P.val64, sizeof(double) * in.nnz, k, s));
    PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
    return 0;
  } catch (...) {
    return handle_exception();
  }
}

// Shared by pdlp_normalized_gap and pdlp_kkt: stage the LP unscaled (no
// preconditioning) and a point, compute A x and A'y with the SpMV engine.
struct PointProblem {
  DeviceArena arena;
  Problem<double> P;
  double *x, *y, *ax, *aty, *xr, *yr;
};

static void stage_point_problem(PointProblem& pp, const Inputs& in, const double* x,
                                const double* y, const double* xr, const double* yr,
                                cudaStream_t s) {
  pp.arena.set_stream(s);
  DevInputs d = stage_inputs(pp.arena, in, s);
  validate(pp.arena, in, d, s);
  build_problem<double>(pp.arena, in, d, 0, 0.0, pp.P, s);
  const int64_t m = in.m, n = in.n;
  auto stage = [&](const double* src, int64_t len, const int32_t* perm) {
    double* tmp = pp.arena.alloc<double>(len);
    double* out = pp.arena.alloc<double>(len);
    copy_in(tmp, src, sizeof(double) * len, in.on_device, s);
    gather_f64(tmp, perm, out, len, s);
    return out;
  };
  pp.x = stage(x, n, pp.P.perm_c);
  pp.y = stage(y, m, pp.P.perm_r);
  pp.ax = pp.arena.alloc<double>(m);
  pp.aty = pp.arena.alloc<double>(n);
  pp.xr = pp.yr = nullptr;
  if (xr) {
    pp.xr = stage(xr, n, pp.P.perm_c);
    pp.yr = stage(yr, m, pp.P.perm_r);
  }
  launch_spmv_plain<double>(pp.P.A, pp.x, pp.ax, spmv_grid<double>(pp.P.A, kEpiPlain), s);
  if (m)
    launch_spmv_plain<double>(pp.P.AT, pp.y, pp.aty, spmv_grid<double>(pp.P.AT, kEpiPlain), s);
  else
    PDLP_CUDA_CHECK(cudaMemsetAsync(pp.aty, 0, sizeof(double) * n, s));
}

int pdlp_normalized_gap(int64_t m, int64_t n, const pdlp_csr* A, const double* c,
                        const double* lc, const double* uc, const double* lv,
                        const double* uv, const double* x, const double* y,
                        const double* x_ref, const double* y_ref, double omega,
                        const pdlp_params* p, double* mu_out) {
  try {
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    const Inputs in = make_inputs(m, n, A, c, lc, uc, lv, uv, &prm);
    if (!x || !x_ref || (m > 0 && (!y || !y_ref)) || !mu_out)
      throw PdlpError(-1, "null point argument");
    if (!(omega > 0.0) || !std::isfinite(omega)) throw PdlpError(-1, "omega must be positive");
    StreamGuard sg(prm.cuda_stream);
    PointProblem pp;
    stage_point_problem(pp, in, x, y, x_ref, y_ref, sg.s);
    const int g = std::max(1, num_sms() * 4);
    GapScratch gsc;
    gsc.grid = g;
    gsc.ctx = static_cast<GapCtx*>(pp.arena.alloc_bytes(gap_ctx_bytes()));
    gsc.part = pp.arena.alloc<double>((int64_t)kGapPartials * g);
    gsc.counter = pp.arena.alloc<unsigned int>(1);
    gsc.cand = pp.arena.alloc<int64_t>(kGapCandCap);
    gsc.params = pp.arena.alloc_bytes(gap_param_bytes(m, n));
    PDLP_CUDA_CHECK(cudaMemsetAsync(gsc.counter, 0, sizeof(unsigned int), sg.s));
    const ScaledVecs<double> sv{pp.P.c, pp.P.lc, pp.P.uc, pp.P.lv, pp.P.uv, m, n};
    GapStats gst;
    *mu_out = normalized_gap<double>(PointRef<double>{pp.x, pp.y, pp.ax, pp.aty}, pp.xr, pp.yr,
                                     omega, sv, gsc, sg.s, nullptr, &gst);
    if (gst.failures) throw PdlpError(-3, gst.last_failure);
    return 0;
  } catch (...) {
    return handle_exception();
  }
}

int pdlp_kkt(int64_t m, int64_t n, const pdlp_csr* A, const double* c, const double* lc,
             const double* uc, const double* lv, const double* uv, const double* x,
             const double* y, const pdlp_params* p, double* out) {
  try {
    pdlp_params prm;
    pdlp_params_default(&prm);
    if (p) prm = *p;
    const Inputs in = make_inputs(m, n, A, c, lc, uc, lv, uv, &prm);
    if (!x || (m > 0 && !y) || !out) throw PdlpError(-1, "null point argument");
    StreamGuard sg(prm.cuda_stream);
    PointProblem pp;
    stage_point_problem(pp, in, x, y, nullptr, nullptr, sg.s);
    const int g = std::max(1, num_sms() * 4);
    KktScratch ks;
    ks.grid = g;
    ks.rc_mode = prm.reduced_costs;
    ks.part = pp.arena.alloc<double>(kKktPartials * (int64_t)g);
    ks.counter = pp.arena.alloc<unsigned int>(1);
    ks.out = pp.arena.alloc<KktSums>(1);
    PDLP_CUDA_CHECK(cudaMemsetAsync(ks.counter, 0, sizeof(unsigned int), sg.s));
    const OrigVecs o{pp.P.orig.c, pp.P.orig.lc, pp.P.orig.uc, pp.P.orig.lv, pp.P.orig.uv,
                     pp.P.d1,     pp.P.d2,      pp.P.inv_d1,  pp.P.inv_d2};
    launch_kkt<double>(PointRef<double>{pp.x, pp.y, pp.ax, pp.aty}, o, m, n, ks, sg.s);
    KktSums h;
    PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, ks.out, sizeof(h), cudaMemcpyDeviceToHost, sg.s));
    PDLP_CUDA_CHECK(cudaStreamSynchronize(sg.s));
    const KktResult r = kkt_finish(h, pp.P.c_norm, pp.P.b_norm);
    const double vals[11] = {r.rel_kkt,  r.rel_primal, r.rel_dual, r.rel_gap,
                             r.pres2,    r.dres2,      r.pres_inf, r.dres_inf,
                             r.pobj,     r.dobj,       r.paper_gap};
    std::memcpy(out, vals, sizeof(vals));
    return 0;
  } catch (...) {
    return handle_exception();
  }
}

}  // extern "C"
