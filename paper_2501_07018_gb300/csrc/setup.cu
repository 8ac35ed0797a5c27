// One-time setup on the GPU: input validation, the CSR transpose, the diagonal
// preconditioning passes of Sec. 3 ("Diagonal Preconditioning") and the row tiling
// used by the fused SpMV kernels.
#include <algorithm>

#include "problem.cuh"

namespace pdlp {

static int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    PDLP_CUDA_CHECK(cudaGetDevice(&dev));
    PDLP_CUDA_CHECK(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return g_num_sms;
}

int grid_ctas(int per_sm) { return num_sms() * per_sm; }

static inline unsigned grid_for(int64_t items, int per_thread = 1, int cap_per_sm = 8) {
  int64_t need = (items + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  int64_t cap = (int64_t)grid_ctas(cap_per_sm);
  return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// ---------------------------------------------------------------------------
// validation: record the smallest offending index of each kind
// ---------------------------------------------------------------------------
__global__ void k_validate_rowptr(const int64_t* rp, int64_t m, int64_t nnz, ValidateFlags* f) {
  for (int64_t i = gtid(); i <= m; i += gstride()) {
    bool bad = false;
    if (i == 0) bad = rp[0] != 0;
    if (i == m) bad = bad || rp[m] != nnz;
    if (i < m) bad = bad || rp[i + 1] < rp[i];
    if (bad) atomicMin(&f->bad_rowptr, (unsigned long long)i);
  }
}

__global__ void k_validate_entries(const int64_t* rp, const int32_t* col, const double* val,
                                   int64_t m, int64_t n, ValidateFlags* f) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    const int64_t b = rp[i], e = rp[i + 1];
    for (int64_t p = b + lane; p < e; p += 32) {
      const int32_t j = col[p];
      if (j < 0 || j >= n || (p > b && col[p - 1] >= j))
        atomicMin(&f->bad_col, (unsigned long long)i);
      if (!isfinite(val[p])) atomicMin(&f->bad_val, (unsigned long long)p);
    }
  }
}

__global__ void k_validate_vectors(const double* c, const double* lc, const double* uc,
                                   const double* lv, const double* uv, int64_t m, int64_t n,
                                   ValidateFlags* f) {
  for (int64_t j = gtid(); j < n; j += gstride()) {
    if (!isfinite(c[j])) atomicMin(&f->bad_c, (unsigned long long)j);
    const double l = lv[j], u = uv[j];
    if (isnan(l) || isnan(u) || l > u || l == INFINITY || u == -INFINITY)
      atomicMin(&f->bad_cols, (unsigned long long)j);
  }
  for (int64_t i = gtid(); i < m; i += gstride()) {
    const double l = lc[i], u = uc[i];
    if (isnan(l) || isnan(u) || l > u || l == INFINITY || u == -INFINITY)
      atomicMin(&f->bad_rows, (unsigned long long)i);
  }
}

void validate_rowptr(const int64_t* rp, int64_t m, int64_t nnz, ValidateFlags* f,
                     cudaStream_t s) {
  k_validate_rowptr<<<grid_for(m + 1), kThreads, 0, s>>>(rp, m, nnz, f);
  PDLP_LAUNCH_CHECK();
}
void validate_entries(const int64_t* rp, const int32_t* col, const double* val, int64_t m,
                      int64_t n, ValidateFlags* f, cudaStream_t s) {
  if (m == 0) return;
  k_validate_entries<<<grid_for(m * 32), kThreads, 0, s>>>(rp, col, val, m, n, f);
  PDLP_LAUNCH_CHECK();
}
void validate_vectors(const double* c, const double* lc, const double* uc, const double* lv,
                      const double* uv, int64_t m, int64_t n, ValidateFlags* f,
                      cudaStream_t s) {
  k_validate_vectors<<<grid_for(std::max(m, n)), kThreads, 0, s>>>(c, lc, uc, lv, uv, m, n, f);
  PDLP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// exclusive scan of int64 (three phases: tile sums, scan of tile sums, apply)
// ---------------------------------------------------------------------------
constexpr int kScanPer = 16;
constexpr int kScanTile = kThreads * kScanPer;

__global__ void k_scan_tile_sums(const int64_t* in, int64_t len, int64_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  long long acc = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kThreads) {
    const int64_t e = base + i;
    if (e < len) acc += in[e];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ long long ws[kWarps];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kWarps; ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// exclusive block-wide scan of one value per thread; returns the block total too
__device__ __forceinline__ long long block_exscan(long long v, long long* total) {
  __shared__ long long ws[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  long long woff = 0, tot = 0;
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) woff += ws[w];
    tot += ws[w];
  }
  __syncthreads();
  *total = tot;
  return woff + inc - v;
}

// single CTA: in-place exclusive scan of `count` tile sums; writes the grand total
__global__ void k_scan_sums(int64_t* sums, int64_t count, int64_t* total_out) {
  long long carry = 0;
  for (int64_t base = 0; base < count; base += kThreads) {
    const int64_t i = base + threadIdx.x;
    long long v = (i < count) ? sums[i] : 0;
    long long tot;
    long long ex = block_exscan(v, &tot);
    if (i < count) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_apply(const int64_t* in, int64_t len, const int64_t* sums, int64_t* out) {
  __shared__ long long tile[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kThreads) {
    const int64_t e = base + i;
    tile[i] = (e < len) ? in[e] : 0;
  }
  __syncthreads();
  long long run = 0;
  long long loc[kScanPer];
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    loc[q] = run;
    run += tile[threadIdx.x * kScanPer + q];
  }
  long long tot;
  const long long ex = block_exscan(run, &tot);
  const long long off = sums[blockIdx.x] + ex;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) tile[threadIdx.x * kScanPer + q] = off + loc[q];
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += kThreads) {
    const int64_t e = base + i;
    if (e < len) out[e] = tile[i];
  }
}

void exclusive_scan_i64(DeviceArena& arena, const int64_t* in, int64_t* out, int64_t len,
                        cudaStream_t s) {
  const int64_t tiles = std::max<int64_t>(1, (len + kScanTile - 1) / kScanTile);
  int64_t* sums = arena.alloc<int64_t>(tiles);
  if (len > 0) {
    k_scan_tile_sums<<<(unsigned)tiles, kThreads, 0, s>>>(in, len, sums);
    PDLP_LAUNCH_CHECK();
  } else {
    PDLP_CUDA_CHECK(cudaMemsetAsync(sums, 0, sizeof(int64_t), s));
  }
  k_scan_sums<<<1, kThreads, 0, s>>>(sums, tiles, out + len);
  PDLP_LAUNCH_CHECK();
  if (len > 0) {
    k_scan_apply<<<(unsigned)tiles, kThreads, 0, s>>>(in, len, sums, out);
    PDLP_LAUNCH_CHECK();
  }
}

// ---------------------------------------------------------------------------
// CSR transpose: stable LSD radix sort of (column, original position)
// ---------------------------------------------------------------------------
constexpr int kRsPer = 16;
constexpr int kRsTile = kThreads * kRsPer;

__global__ void k_expand_rows(const int64_t* rp, int64_t m, int32_t* rowidx) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t i = warp; i < m; i += nwarps)
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) rowidx[p] = (int32_t)i;
}

__global__ void k_col_counts(const int32_t* col, int64_t nnz, unsigned long long* cnt) {
  for (int64_t e = gtid(); e < nnz; e += gstride()) atomicAdd(&cnt[col[e]], 1ull);
}

__global__ void k_rs_hist(const int32_t* keys, int64_t N, int shift, int64_t* hist,
                          int64_t ntiles) {
  __shared__ unsigned int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += kThreads) {
    const int64_t e = base + i;
    if (e < N) atomicAdd(&cnt[(keys[e] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one 8-bit digit: items are taken in 16 rounds of 256 consecutive
// positions; inside a round thread t holds position t, so rank order equals position
// order (warp ranks from __match_any_sync, warp offsets from per-warp digit counts).
__global__ void k_rs_scatter(const int32_t* kin, const int64_t* vin, int32_t* kout,
                             int64_t* vout, int64_t N, int shift, const int64_t* offs,
                             int64_t ntiles) {
  __shared__ unsigned int base[256];
  __shared__ unsigned int wcnt[kWarps][257];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  base[t] = 0;
  for (int w = 0; w < kWarps; ++w) wcnt[w][t] = 0;
  if (t < kWarps) wcnt[t][256] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  for (int round = 0; round < kRsPer; ++round) {
    const int64_t e = tile0 + (int64_t)round * kThreads + t;
    const bool valid = e < N;
    const int32_t key = valid ? kin[e] : 0;
    const int d = valid ? ((key >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank_w = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    if (lane == leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned int r = base[d] + rank_w;
      for (int w = 0; w < warp; ++w) r += wcnt[w][d];
      const int64_t dst = offs[(int64_t)d * ntiles + blockIdx.x] + r;
      kout[dst] = key;
      vout[dst] = vin ? vin[e] : e;
    }
    __syncthreads();
    {
      unsigned int sum = 0;
      for (int w = 0; w < kWarps; ++w) {
        sum += wcnt[w][t];
        wcnt[w][t] = 0;
      }
      base[t] += sum;
      if (t < kWarps) wcnt[t][256] = 0;
    }
    __syncthreads();
  }
}

__global__ void k_gather_transpose(const int64_t* perm, const int32_t* rowidx,
                                   const double* val, int64_t nnz, int32_t* t_col,
                                   double* t_val) {
  for (int64_t p = gtid(); p < nnz; p += gstride()) {
    const int64_t e = perm[p];
    t_col[p] = rowidx[e];
    t_val[p] = val[e];
  }
}

__global__ void k_iota64(int64_t* v, int64_t n) {
  for (int64_t i = gtid(); i < n; i += gstride()) v[i] = i;
}

void transpose_csr(DeviceArena& arena, const int64_t* row_ptr, const int32_t* col,
                   const double* val, int64_t m, int64_t n, int64_t nnz, int64_t* t_row_ptr,
                   int32_t* t_col, double* t_val, cudaStream_t s) {
  // row pointers of the transpose: column counts, then an exclusive scan
  unsigned long long* cnt = arena.alloc<unsigned long long>(n);
  PDLP_CUDA_CHECK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * n, s));
  if (nnz > 0) {
    k_col_counts<<<grid_for(nnz), kThreads, 0, s>>>(col, nnz, cnt);
    PDLP_LAUNCH_CHECK();
  }
  exclusive_scan_i64(arena, reinterpret_cast<const int64_t*>(cnt), t_row_ptr, n, s);
  if (nnz == 0) return;

  int32_t* rowidx = arena.alloc<int32_t>(nnz);
  k_expand_rows<<<grid_for(m * 32), kThreads, 0, s>>>(row_ptr, m, rowidx);
  PDLP_LAUNCH_CHECK();

  int bits = 0;
  while (bits < 63 && ((int64_t)1 << bits) < n) ++bits;
  const int passes = (bits + 7) / 8;
  const int64_t ntiles = (nnz + kRsTile - 1) / kRsTile;
  int32_t* kbuf[2] = {arena.alloc<int32_t>(nnz), arena.alloc<int32_t>(nnz)};
  int64_t* vbuf[2] = {arena.alloc<int64_t>(nnz), arena.alloc<int64_t>(nnz)};
  int64_t* hist = arena.alloc<int64_t>(256 * ntiles);
  int64_t* offs = arena.alloc<int64_t>(256 * ntiles + 1);
  const int32_t* kin = col;
  const int64_t* vin = nullptr;  // identity payload on the first pass
  int which = 0;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    k_rs_hist<<<(unsigned)ntiles, kThreads, 0, s>>>(kin, nnz, shift, hist, ntiles);
    PDLP_LAUNCH_CHECK();
    exclusive_scan_i64(arena, hist, offs, 256 * ntiles, s);
    k_rs_scatter<<<(unsigned)ntiles, kThreads, 0, s>>>(kin, vin, kbuf[which], vbuf[which], nnz,
                                                       shift, offs, ntiles);
    PDLP_LAUNCH_CHECK();
    kin = kbuf[which];
    vin = vbuf[which];
    which ^= 1;
  }
  if (passes == 0) {
    // n == 1: every key is 0 and the input order is already the stable order
    k_iota64<<<grid_for(nnz), kThreads, 0, s>>>(vbuf[0], nnz);
    PDLP_LAUNCH_CHECK();
    vin = vbuf[0];
  }
  k_gather_transpose<<<grid_for(nnz), kThreads, 0, s>>>(vin, rowidx, val, nnz, t_col, t_val);
  PDLP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// preconditioning passes
// ---------------------------------------------------------------------------
__global__ void k_row_norms(const int64_t* rp, const double* val, int64_t rows, int kind,
                            double p, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t i = warp; i < rows; i += nwarps) {
    double acc = 0.0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      const double a = fabs(val[e]);
      if (kind == 0)
        acc = fmax(acc, a);
      else if (kind == 1)
        acc += a;
      else
        acc += pow(a, p);
    }
    acc = (kind == 0) ? warp_max(acc) : warp_sum(acc);
    if (lane == 0) out[i] = (kind == 2 && acc > 0.0) ? pow(acc, 1.0 / p) : acc;
  }
}

__global__ void k_scale_factors(const double* norms, int64_t len, double* f, double* acc) {
  for (int64_t i = gtid(); i < len; i += gstride()) {
    const double v = norms[i];
    const double fi = (v > 0.0) ? 1.0 / sqrt(v) : 1.0;
    f[i] = fi;
    acc[i] = acc[i] * fi;
  }
}

// The entry in row `row`, column col[e] becomes (val * f_first[.]) * f_second[.] where
// f_first is indexed by the column (first_is_col) or the row, f_second by the other.
__global__ void k_scale_values(const int64_t* rp, const int32_t* col, double* val, int64_t rows,
                               const double* f_first, const double* f_second,
                               bool first_is_col) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t i = warp; i < rows; i += nwarps) {
    const double fr = first_is_col ? 0.0 : f_first[i];
    const double fs = first_is_col ? f_second[i] : 0.0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      const int32_t j = col[e];
      double v;
      if (first_is_col)
        v = __dmul_rn(__dmul_rn(val[e], f_first[j]), fs);
      else
        v = __dmul_rn(__dmul_rn(val[e], fr), f_second[j]);
      val[e] = v;
    }
  }
}

__global__ void k_max_abs_partial(const double* v, int64_t len, double* part) {
  double m = 0.0;
  for (int64_t i = gtid(); i < len; i += gstride()) m = fmax(m, fabs(v[i]));
  m = warp_max(m);
  __shared__ double ws[kWarps];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kWarps; ++w) r = fmax(r, ws[w]);
    part[blockIdx.x] = r;
  }
}

void row_norms(const int64_t* rp, const double* val, int64_t rows, int kind, double p,
               double* out, cudaStream_t s) {
  if (rows == 0) return;
  k_row_norms<<<grid_for(rows * 32), kThreads, 0, s>>>(rp, val, rows, kind, p, out);
  PDLP_LAUNCH_CHECK();
}
void scale_factors(const double* norms, int64_t len, double* f, double* acc, cudaStream_t s) {
  if (len == 0) return;
  k_scale_factors<<<grid_for(len), kThreads, 0, s>>>(norms, len, f, acc);
  PDLP_LAUNCH_CHECK();
}
void scale_values(const int64_t* rp, const int32_t* col, double* val, int64_t rows,
                  const double* f_first, const double* f_second, bool first_is_col,
                  cudaStream_t s) {
  if (rows == 0) return;
  k_scale_values<<<grid_for(rows * 32), kThreads, 0, s>>>(rp, col, val, rows, f_first, f_second,
                                                          first_is_col);
  PDLP_LAUNCH_CHECK();
}
double max_abs(DeviceArena& arena, const double* v, int64_t len, cudaStream_t s) {
  if (len == 0) return 0.0;
  const unsigned g = grid_for(len);
  double* part = arena.alloc<double>(g);
  k_max_abs_partial<<<g, kThreads, 0, s>>>(v, len, part);
  PDLP_LAUNCH_CHECK();
  std::vector<double> h(g);
  PDLP_CUDA_CHECK(cudaMemcpyAsync(h.data(), part, sizeof(double) * g, cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  double r = 0.0;
  for (double x : h) r = std::max(r, x);
  return r;
}

// ---------------------------------------------------------------------------
// row tiling for the fused SpMV kernels
// ---------------------------------------------------------------------------
__global__ void k_tile_rows(const int64_t* rp, int64_t rows, int64_t ntiles, int32_t* tile_row) {
  for (int64_t t = gtid(); t <= ntiles; t += gstride()) {
    if (t == ntiles) {
      tile_row[t] = (int32_t)rows;
      continue;
    }
    const int64_t target = t * kUnitDiag;
    int64_t lo = 0, hi = rows;  // first r with kUnitRowWeight * r + rp[r] >= target
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (kUnitRowWeight * mid + rp[mid] >= target)
        hi = mid;
      else
        lo = mid + 1;
    }
    tile_row[t] = (int32_t)lo;
  }
}

__global__ void k_long_flags(const int64_t* rp, int64_t rows, int64_t* flag, int64_t* nch) {
  for (int64_t i = gtid(); i < rows; i += gstride()) {
    const int64_t len = rp[i + 1] - rp[i];
    const bool lng = len > kLongRow;
    flag[i] = lng ? 1 : 0;
    nch[i] = lng ? (len + kChunk - 1) / kChunk : 0;
  }
}

__global__ void k_long_compact(const int64_t* flag, const int64_t* pos, const int64_t* nch,
                               const int64_t* nch_pos, int64_t rows, int32_t* long_rows,
                               int64_t* chunk_ptr, int32_t* chunk_owner) {
  for (int64_t i = gtid(); i < rows; i += gstride()) {
    if (!flag[i]) continue;
    const int64_t lr = pos[i];
    long_rows[lr] = (int32_t)i;
    chunk_ptr[lr] = nch_pos[i];
    for (int64_t c = 0; c < nch[i]; ++c) chunk_owner[nch_pos[i] + c] = (int32_t)lr;
  }
}

template <class T>
void build_tiles(DeviceArena& arena, Mat<T>& M, cudaStream_t s) {
  M.ntiles = 0;
  M.nlong = 0;
  M.nchunks = 0;
  if (M.rows == 0) {
    M.tile_row = arena.alloc<int32_t>(1);
    return;
  }
  int64_t last_start = 0;
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&last_start, M.row_ptr + (M.rows - 1), sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  const int64_t ntiles = (kUnitRowWeight * (M.rows - 1) + last_start) / kUnitDiag + 1;
  if (ntiles > INT32_MAX - 1) throw PdlpError(-1, "matrix too large for the row tiling");
  M.ntiles = (int32_t)ntiles;
  M.tile_row = arena.alloc<int32_t>(ntiles + 1);
  k_tile_rows<<<grid_for(ntiles + 1), kThreads, 0, s>>>(M.row_ptr, M.rows, ntiles, M.tile_row);
  PDLP_LAUNCH_CHECK();

  int64_t* flag = arena.alloc<int64_t>(M.rows);
  int64_t* pos = arena.alloc<int64_t>(M.rows + 1);
  int64_t* nch = arena.alloc<int64_t>(M.rows);
  int64_t* nch_pos = arena.alloc<int64_t>(M.rows + 1);
  k_long_flags<<<grid_for(M.rows), kThreads, 0, s>>>(M.row_ptr, M.rows, flag, nch);
  PDLP_LAUNCH_CHECK();
  exclusive_scan_i64(arena, flag, pos, M.rows, s);
  exclusive_scan_i64(arena, nch, nch_pos, M.rows, s);
  int64_t totals[2] = {0, 0};
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&totals[0], pos + M.rows, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&totals[1], nch_pos + M.rows, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  M.nlong = (int32_t)totals[0];
  M.nchunks = totals[1];
  M.long_rows = arena.alloc<int32_t>(M.nlong);
  M.chunk_ptr = arena.alloc<int64_t>(M.nlong + 1);
  M.chunk_owner = arena.alloc<int32_t>(M.nchunks);
  M.long_cnt = arena.alloc<unsigned int>(M.nlong);
  M.long_part = arena.alloc<double>(M.nchunks);
  M.long_contrib = arena.alloc<double>(2 * (int64_t)M.nlong);
  PDLP_CUDA_CHECK(cudaMemsetAsync(M.long_cnt, 0, sizeof(unsigned int) * std::max(1, M.nlong), s));
  PDLP_CUDA_CHECK(cudaMemsetAsync(M.long_contrib, 0, sizeof(double) * 2 * std::max(1, M.nlong), s));
  if (M.nlong > 0) {
    k_long_compact<<<grid_for(M.rows), kThreads, 0, s>>>(flag, pos, nch, nch_pos, M.rows,
                                                         M.long_rows, M.chunk_ptr,
                                                         M.chunk_owner);
    PDLP_LAUNCH_CHECK();
  }
  PDLP_CUDA_CHECK(cudaMemcpyAsync(M.chunk_ptr + M.nlong, &M.nchunks, sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
}

template <class T>
__global__ void k_convert(const double* src, T* dst, int64_t len) {
  for (int64_t i = gtid(); i < len; i += gstride()) dst[i] = (T)src[i];
}

template <class T>
void convert_values(const double* src, T* dst, int64_t len, cudaStream_t s) {
  if (len == 0) return;
  k_convert<T><<<grid_for(len), kThreads, 0, s>>>(src, dst, len);
  PDLP_LAUNCH_CHECK();
}

template void build_tiles<double>(DeviceArena&, Mat<double>&, cudaStream_t);
template void build_tiles<float>(DeviceArena&, Mat<float>&, cudaStream_t);
template void convert_values<double>(const double*, double*, int64_t, cudaStream_t);
template void convert_values<float>(const double*, float*, int64_t, cudaStream_t);

}  // namespace pdlp
