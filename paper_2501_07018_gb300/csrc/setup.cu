// One-time setup on the GPU: input validation, the CSR transpose, the diagonal
// preconditioning passes of Sec. 3 ("Diagonal Preconditioning") and the row tiling
// used by the fused SpMV kernels.
#include <algorithm>
#include <atomic>

#include "problem.cuh"

namespace pdlp {

static std::atomic<int> g_num_sms{0};  // same value from every thread (one GPU model)

int num_sms() {
  int v = g_num_sms.load(std::memory_order_relaxed);
  if (v == 0) {
    int dev = 0;
    PDLP_CUDA_CHECK(cudaGetDevice(&dev));
    PDLP_CUDA_CHECK(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    g_num_sms.store(v, std::memory_order_relaxed);
  }
  return v;
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

// Stable LSD radix sort of non-negative int32 keys < 2^bits; returns the sorted
// positions (the original index of each sorted entry) in a fresh array.
static int64_t* radix_sort_positions(DeviceArena& arena, const int32_t* keys, int64_t N, int bits,
                                     cudaStream_t s) {
  const int passes = (bits + 7) / 8;
  const int64_t ntiles = std::max<int64_t>(1, (N + kRsTile - 1) / kRsTile);
  int32_t* kbuf[2] = {arena.alloc<int32_t>(N), arena.alloc<int32_t>(N)};
  int64_t* vbuf[2] = {arena.alloc<int64_t>(N), arena.alloc<int64_t>(N)};
  if (N == 0) return vbuf[0];
  int64_t* hist = arena.alloc<int64_t>(256 * ntiles);
  int64_t* offs = arena.alloc<int64_t>(256 * ntiles + 1);
  const int32_t* kin = keys;
  const int64_t* vin = nullptr;  // identity payload on the first pass
  int which = 0;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    k_rs_hist<<<(unsigned)ntiles, kThreads, 0, s>>>(kin, N, shift, hist, ntiles);
    PDLP_LAUNCH_CHECK();
    exclusive_scan_i64(arena, hist, offs, 256 * ntiles, s);
    k_rs_scatter<<<(unsigned)ntiles, kThreads, 0, s>>>(kin, vin, kbuf[which], vbuf[which], N,
                                                       shift, offs, ntiles);
    PDLP_LAUNCH_CHECK();
    kin = kbuf[which];
    vin = vbuf[which];
    which ^= 1;
  }
  if (passes == 0) {
    k_iota64<<<grid_for(N), kThreads, 0, s>>>(vbuf[0], N);
    PDLP_LAUNCH_CHECK();
    return vbuf[0];
  }
  return const_cast<int64_t*>(vin);
}

static int bits_for(int64_t maxval) {
  int bits = 0;
  while (bits < 62 && ((int64_t)1 << bits) <= maxval) ++bits;
  return bits;
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
  const int64_t* perm = radix_sort_positions(arena, col, nnz, bits_for(n - 1), s);
  k_gather_transpose<<<grid_for(nnz), kThreads, 0, s>>>(perm, rowidx, val, nnz, t_col, t_val);
  PDLP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// renumbering by row length
// ---------------------------------------------------------------------------
__global__ void k_len_keys(const int64_t* rp, int64_t rows, int64_t maxlen, int32_t* key) {
  for (int64_t i = gtid(); i < rows; i += gstride()) key[i] = (int32_t)(maxlen - (rp[i + 1] - rp[i]));
}
__global__ void k_max_len(const int64_t* rp, int64_t rows, unsigned long long* out) {
  unsigned long long mx = 0;
  for (int64_t i = gtid(); i < rows; i += gstride()) {
    const unsigned long long l = (unsigned long long)(rp[i + 1] - rp[i]);
    mx = l > mx ? l : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}
__global__ void k_perm_from_positions(const int64_t* pos, int64_t n, int32_t* perm, int32_t* inv) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const int64_t o = pos[i];
    perm[i] = (int32_t)o;
    inv[o] = (int32_t)i;
  }
}

void sort_by_length_desc(DeviceArena& arena, const int64_t* rp, int64_t count, int32_t* perm,
                         int32_t* inv, cudaStream_t s) {
  if (count == 0) return;
  unsigned long long* mx = arena.alloc<unsigned long long>(1);
  PDLP_CUDA_CHECK(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
  k_max_len<<<grid_for(count), kThreads, 0, s>>>(rp, count, mx);
  PDLP_LAUNCH_CHECK();
  unsigned long long hmx = 0;
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  int32_t* key = arena.alloc<int32_t>(count);
  k_len_keys<<<grid_for(count), kThreads, 0, s>>>(rp, count, (int64_t)hmx, key);
  PDLP_LAUNCH_CHECK();
  const int64_t* pos = radix_sort_positions(arena, key, count, bits_for((int64_t)hmx), s);
  k_perm_from_positions<<<grid_for(count), kThreads, 0, s>>>(pos, count, perm, inv);
  PDLP_LAUNCH_CHECK();
}

__global__ void k_perm_lens(const int64_t* rp, const int32_t* perm, int64_t rows, int64_t* len) {
  for (int64_t i = gtid(); i < rows; i += gstride()) {
    const int32_t o = perm[i];
    len[i] = rp[o + 1] - rp[o];
  }
}
__global__ void k_perm_rows(const int64_t* rp, const int32_t* col, const double* val,
                            const int32_t* perm, const int32_t* inv_c, int64_t rows,
                            const int64_t* nrp, int32_t* ncol, double* nval) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t i = warp; i < rows; i += nwarps) {
    const int32_t o = perm[i];
    const int64_t b = rp[o], len = rp[o + 1] - b, nb = nrp[i];
    for (int64_t k = lane; k < len; k += 32) {
      ncol[nb + k] = inv_c[col[b + k]];
      nval[nb + k] = val[b + k];
    }
  }
}

void permute_csr(DeviceArena& arena, const int64_t* rp, const int32_t* col, const double* val,
                 int64_t rows, const int32_t* perm_r, const int32_t* inv_c, int64_t* nrp,
                 int32_t* ncol, double* nval, cudaStream_t s) {
  int64_t* len = arena.alloc<int64_t>(rows);
  if (rows) {
    k_perm_lens<<<grid_for(rows), kThreads, 0, s>>>(rp, perm_r, rows, len);
    PDLP_LAUNCH_CHECK();
  }
  exclusive_scan_i64(arena, len, nrp, rows, s);
  if (rows) {
    k_perm_rows<<<grid_for(rows * 32), kThreads, 0, s>>>(rp, col, val, perm_r, inv_c, rows, nrp,
                                                         ncol, nval);
    PDLP_LAUNCH_CHECK();
  }
}

__global__ void k_gather_f64(const double* in, const int32_t* perm, double* out, int64_t len) {
  for (int64_t i = gtid(); i < len; i += gstride()) out[i] = in[perm[i]];
}
void gather_f64(const double* in, const int32_t* perm, double* out, int64_t len, cudaStream_t s) {
  if (len == 0) return;
  k_gather_f64<<<grid_for(len), kThreads, 0, s>>>(in, perm, out, len);
  PDLP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// preconditioning passes
// ---------------------------------------------------------------------------
// One group of G lanes per row (G chosen from the mean row length); the loop trip
// count is uniform across a warp so the group shuffles are safe.  The max norm (kind 0)
// runs on the integer pipe: for the finite non-negative |a_ij| the IEEE bit patterns
// order as the values do, so the max of the patterns with the sign bit cleared is the
// pattern of the max, exactly.  On GB300 a double fmax per lane (one per entry and one
// per step of the group's shuffle tree) made the FP64 pipe the bound of this pass.
template <int G>
__global__ void k_row_max(const int64_t* rp, const double* val, int64_t rows, double* out) {
  const int lane = threadIdx.x & 31, lg = lane % G;
  const int64_t per_warp = 32 / G;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(val);
  constexpr unsigned long long kMag = 0x7fffffffffffffffULL;
  for (int64_t i0 = warp * per_warp; i0 < rows; i0 += nwarps * per_warp) {
    const int64_t i = i0 + lane / G;
    unsigned long long acc = 0;
    if (i < rows)
      for (int64_t e = rp[i] + lg; e < rp[i + 1]; e += G) {
        const unsigned long long a = bits[e] & kMag;
        acc = a > acc ? a : acc;
      }
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, acc, o, G);
      acc = t > acc ? t : acc;
    }
    if (i < rows && lg == 0) out[i] = __longlong_as_double((long long)acc);
  }
}

// Sums |a| (kind 1) or |a|^p (kind 2) per row, p-th root for kind 2.
template <int G>
__global__ void k_row_norms(const int64_t* rp, const double* val, int64_t rows, int kind,
                            double p, double* out) {
  const int lane = threadIdx.x & 31, lg = lane % G;
  const int64_t per_warp = 32 / G;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t i0 = warp * per_warp; i0 < rows; i0 += nwarps * per_warp) {
    const int64_t i = i0 + lane / G;
    double acc = 0.0;
    if (i < rows) {
      for (int64_t e = rp[i] + lg; e < rp[i + 1]; e += G) {
        const double a = fabs(val[e]);
        acc += kind == 1 ? a : pow(a, p);
      }
    }
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
    if (i < rows && lg == 0) out[i] = (kind == 2 && acc > 0.0) ? pow(acc, 1.0 / p) : acc;
  }
}

static int group_for(int64_t nnz, int64_t rows) {
  const double avg = rows > 0 ? (double)nnz / (double)rows : 1.0;
  int g = 1;
  while (g < 32 && g < avg) g <<= 1;
  return g;
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
// One group of G lanes per row, as in k_row_norms.
template <int G>
__global__ void k_scale_values(const int64_t* rp, const int32_t* col, double* val, int64_t rows,
                               const double* f_first, const double* f_second,
                               bool first_is_col) {
  const int lane = threadIdx.x & 31, lg = lane % G;
  const int64_t per_warp = 32 / G;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t i0 = warp * per_warp; i0 < rows; i0 += nwarps * per_warp) {
    const int64_t i = i0 + lane / G;
    if (i >= rows) continue;
    const double fr = first_is_col ? 0.0 : f_first[i];
    const double fs = first_is_col ? f_second[i] : 0.0;
    for (int64_t e = rp[i] + lg; e < rp[i + 1]; e += G) {
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

#define PDLP_GROUP_DISPATCH(G, CALL) \
  switch (G) {                          \
    case 1: CALL(1); break;             \
    case 2: CALL(2); break;             \
    case 4: CALL(4); break;             \
    case 8: CALL(8); break;             \
    case 16: CALL(16); break;           \
    default: CALL(32); break;           \
  }

void row_norms(const int64_t* rp, const double* val, int64_t rows, int64_t nnz, int kind,
               double p, double* out, cudaStream_t s) {
  if (rows == 0) return;
  const int g = group_for(nnz, rows);
  const unsigned grid = grid_for((rows * g + 31) / 32 * 32);
#define PDLP_MAX(G) k_row_max<G><<<grid, kThreads, 0, s>>>(rp, val, rows, out)
#define PDLP_NORMS(G) k_row_norms<G><<<grid, kThreads, 0, s>>>(rp, val, rows, kind, p, out)
  if (kind == 0) {
    PDLP_GROUP_DISPATCH(g, PDLP_MAX)
  } else {
    PDLP_GROUP_DISPATCH(g, PDLP_NORMS)
  }
#undef PDLP_NORMS
#undef PDLP_MAX
  PDLP_LAUNCH_CHECK();
}
void scale_factors(const double* norms, int64_t len, double* f, double* acc, cudaStream_t s) {
  if (len == 0) return;
  k_scale_factors<<<grid_for(len), kThreads, 0, s>>>(norms, len, f, acc);
  PDLP_LAUNCH_CHECK();
}
void scale_values(const int64_t* rp, const int32_t* col, double* val, int64_t rows,
                  int64_t nnz, const double* f_first, const double* f_second,
                  bool first_is_col, cudaStream_t s) {
  if (rows == 0) return;
  const int g = group_for(nnz, rows);
  const unsigned grid = grid_for((rows * g + 31) / 32 * 32);
#define PDLP_SCALE(G) \
  k_scale_values<G><<<grid, kThreads, 0, s>>>(rp, col, val, rows, f_first, f_second, first_is_col)
  PDLP_GROUP_DISPATCH(g, PDLP_SCALE)
#undef PDLP_SCALE
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
// long-row chunks and SELL-32 for the fused SpMV kernels
// ---------------------------------------------------------------------------
__global__ void k_count_long(const int64_t* rp, int64_t rows, unsigned long long* cnt) {
  unsigned long long c = 0;
  for (int64_t i = gtid(); i < rows; i += gstride()) c += (rp[i + 1] - rp[i] > kLongRow) ? 1ull : 0ull;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}
__global__ void k_chunk_counts(const int64_t* rp, int64_t R0, int64_t* nch) {
  for (int64_t i = gtid(); i < R0; i += gstride()) {
    const int64_t len = rp[i + 1] - rp[i];
    nch[i] = len > 0 ? (len + kChunk - 1) / kChunk : 1;
  }
}
__global__ void k_chunk_owner(const int64_t* chunk_ptr, int64_t R0, int32_t* owner) {
  for (int64_t i = gtid(); i < R0; i += gstride())
    for (int64_t c = chunk_ptr[i]; c < chunk_ptr[i + 1]; ++c) owner[c] = (int32_t)i;
}
__global__ void k_slice_len(const int64_t* rp, int64_t R0, int64_t rows, int64_t nslices,
                            int32_t* slen, int64_t* sent) {
  for (int64_t sl = gtid(); sl < nslices; sl += gstride()) {
    const int64_t r = R0 + 32 * sl;  // rows are sorted by decreasing length
    const int64_t len = rp[r + 1] - rp[r];
    slen[sl] = (int32_t)len;
    sent[sl] = 32 * len;
  }
}
template <class T>
__global__ void k_fill_sell(const int64_t* rp, const int32_t* col, const double* val, int64_t R0,
                            int64_t rows, int64_t nslices, const int64_t* sptr,
                            const int32_t* slen, int32_t* scol, T* sval) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
  for (int64_t sl = warp; sl < nslices; sl += nwarps) {
    const int64_t r = R0 + 32 * sl + lane;
    const int64_t L = slen[sl], base = sptr[sl];
    int64_t b = 0, len = 0;
    if (r < rows) {
      b = rp[r];
      len = rp[r + 1] - b;
    }
    int32_t last = len > 0 ? col[b + len - 1] : 0;
    for (int64_t k = 0; k < L; ++k) {
      const bool in = k < len;
      scol[base + 32 * k + lane] = in ? col[b + k] : last;
      sval[base + 32 * k + lane] = in ? (T)val[b + k] : (T)0;
    }
  }
}

template <class T>
void build_sell(DeviceArena& arena, Mat<T>& M, const double* val64, cudaStream_t s) {
  const int64_t rows = M.rows;
  // long rows: a prefix of the length-sorted rows, rounded up to whole slices
  unsigned long long* cnt = arena.alloc<unsigned long long>(1);
  PDLP_CUDA_CHECK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  if (rows) {
    k_count_long<<<grid_for(rows), kThreads, 0, s>>>(M.row_ptr, rows, cnt);
    PDLP_LAUNCH_CHECK();
  }
  unsigned long long nlong = 0;
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&nlong, cnt, sizeof(nlong), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  const int64_t R0 = nlong ? std::min<int64_t>(rows, ((int64_t)nlong + 31) / 32 * 32) : 0;
  M.R0 = (int32_t)R0;
  M.chunk_ptr = arena.alloc<int64_t>(R0 + 1);
  int64_t* nch = arena.alloc<int64_t>(R0);
  if (R0) {
    k_chunk_counts<<<grid_for(R0), kThreads, 0, s>>>(M.row_ptr, R0, nch);
    PDLP_LAUNCH_CHECK();
  }
  exclusive_scan_i64(arena, nch, M.chunk_ptr, R0, s);
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&M.nchunks, M.chunk_ptr + R0, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  M.chunk_owner = arena.alloc<int32_t>(M.nchunks);
  if (R0) {
    k_chunk_owner<<<grid_for(R0), kThreads, 0, s>>>(M.chunk_ptr, R0, M.chunk_owner);
    PDLP_LAUNCH_CHECK();
  }
  M.long_cnt = arena.alloc<unsigned int>(R0);
  M.long_part = arena.alloc<double>(M.nchunks);
  M.long_contrib = arena.alloc<double>(2 * R0);
  PDLP_CUDA_CHECK(cudaMemsetAsync(M.long_cnt, 0, sizeof(unsigned int) * std::max<int64_t>(1, R0), s));
  PDLP_CUDA_CHECK(cudaMemsetAsync(M.long_contrib, 0, sizeof(double) * 2 * std::max<int64_t>(1, R0), s));
  M.sched = arena.alloc<unsigned int>(2);
  PDLP_CUDA_CHECK(cudaMemsetAsync(M.sched, 0, 2 * sizeof(unsigned int), s));

  // SELL-32 of the remaining rows
  M.nslices = (rows - R0 + 31) / 32;
  M.slice_ptr = arena.alloc<int64_t>(M.nslices + 1);
  M.slice_len = arena.alloc<int32_t>(M.nslices);
  int64_t* sent = arena.alloc<int64_t>(M.nslices);
  if (M.nslices) {
    k_slice_len<<<grid_for(M.nslices), kThreads, 0, s>>>(M.row_ptr, R0, rows, M.nslices,
                                                         M.slice_len, sent);
    PDLP_LAUNCH_CHECK();
  }
  exclusive_scan_i64(arena, sent, M.slice_ptr, M.nslices, s);
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&M.sell_entries, M.slice_ptr + M.nslices, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  M.sell_col = arena.alloc<int32_t>(M.sell_entries);
  M.sell_val = arena.alloc<T>(M.sell_entries);
  if (M.nslices) {
    k_fill_sell<T><<<grid_for(M.nslices * 32), kThreads, 0, s>>>(
        M.row_ptr, M.col, val64, R0, rows, M.nslices, M.slice_ptr, M.slice_len, M.sell_col,
        M.sell_val);
    PDLP_LAUNCH_CHECK();
  }
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

template void build_sell<double>(DeviceArena&, Mat<double>&, const double*, cudaStream_t);
template void build_sell<float>(DeviceArena&, Mat<float>&, const double*, cudaStream_t);
template void convert_values<double>(const double*, double*, int64_t, cudaStream_t);
template void convert_values<float>(const double*, float*, int64_t, cudaStream_t);

}  // namespace pdlp
