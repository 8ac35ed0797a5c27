// Device-resident problem layout and the launcher interface between the host driver
// (solver.cu) and the kernel translation units (setup.cu, pdhg.cu, gap.cu).
#pragma once

#include <vector>

#include "common.cuh"

namespace pdlp {

// Storage of a (row- and column-renumbered) sparse matrix for the fused SpMV kernels.
//   Rows are numbered by decreasing length.  The first R0 rows (every row longer than
//   kLongRow, rounded up to a multiple of 32) stay in CSR and are processed in chunks
//   of kChunk entries, one warp per chunk; a row of several chunks is finished by the
//   last of its chunks to arrive, which adds the chunk sums in a fixed order.  The
//   remaining rows are stored as SELL-32: slice s holds rows R0 + 32 s ...
//   R0 + 32 s + 31, padded to the length of its first (longest) row, entry k of lane l
//   at slice_ptr[s] + 32 k + l; padding entries have value 0.  One warp processes one
//   slice, one row per lane.
#ifndef PDLP_CHUNK
#define PDLP_CHUNK 4096
#endif
constexpr int kLongRow = 256;
constexpr int kChunk = PDLP_CHUNK;

template <class T>
struct Mat {
  int64_t rows = 0, cols = 0, nnz = 0;
  // CSR of the renumbered matrix (only its first R0 rows are read by the kernels)
  int64_t* row_ptr = nullptr;  // [rows+1]
  int32_t* col = nullptr;      // [nnz]
  T* val = nullptr;            // [nnz]
  int32_t R0 = 0;
  int64_t nchunks = 0;
  int64_t* chunk_ptr = nullptr;      // [R0+1] first chunk of each long row
  int32_t* chunk_owner = nullptr;    // [nchunks] row of each chunk
  unsigned int* long_cnt = nullptr;  // [R0] arrival counters (kept at 0 between launches)
  double* long_part = nullptr;       // [nchunks] chunk partial sums
  double* long_contrib = nullptr;    // [R0 * 2] per-long-row reduction contributions
  unsigned int* sched = nullptr;     // [2] dynamic work queue: next item, CTAs done
                                     // (both back at 0 between launches)
  // SELL-32 of rows [R0, rows)
  int64_t nslices = 0;
  int64_t* slice_ptr = nullptr;  // [nslices+1]
  int32_t* slice_len = nullptr;  // [nslices]
  int32_t* sell_col = nullptr;
  T* sell_val = nullptr;
  int64_t sell_entries = 0;
  int64_t work_items() const { return nchunks + nslices; }
};

// Simple owning list of device allocations, freed together.  Allocations are
// stream-ordered (cudaMallocAsync / cudaFreeAsync on the arena's stream), so that solves
// running concurrently on different streams never synchronise the device to allocate
// or free.
class DeviceArena {
 public:
  ~DeviceArena() { release(); }
  void set_stream(cudaStream_t s) { stream_ = s; }
  void* alloc_bytes(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    PDLP_CUDA_CHECK(cudaMallocAsync(&p, (bytes + 255) & ~size_t(255), stream_));
    ptrs_.push_back(p);
    total_ += bytes;
    return p;
  }
  template <class U>
  U* alloc(int64_t count) {
    return static_cast<U*>(alloc_bytes(sizeof(U) * (size_t)(count > 0 ? count : 1)));
  }
  void release() {
    for (void* p : ptrs_) cudaFreeAsync(p, stream_);
    ptrs_.clear();
  }
  size_t total() const { return total_; }

 private:
  std::vector<void*> ptrs_;
  size_t total_ = 0;
  cudaStream_t stream_ = nullptr;
};

// Number of CTAs of the persistent / grid-stride kernels on this device.
int grid_ctas(int per_sm);
int num_sms();

// ---------------------------------------------------------------------------
// setup.cu
// ---------------------------------------------------------------------------
struct ValidateFlags {
  unsigned long long bad_rowptr, bad_col, bad_val, bad_c, bad_rows, bad_cols;
};
void validate_rowptr(const int64_t* row_ptr, int64_t m, int64_t nnz, ValidateFlags* flags,
                     cudaStream_t s);
void validate_entries(const int64_t* row_ptr, const int32_t* col, const double* val, int64_t m,
                      int64_t n, ValidateFlags* flags, cudaStream_t s);
void validate_vectors(const double* c, const double* lc, const double* uc, const double* lv,
                      const double* uv, int64_t m, int64_t n, ValidateFlags* flags,
                      cudaStream_t s);

// CSR transpose by a stable LSD radix sort of the column indices: within each row of
// the transpose, entries keep increasing original-row order.
void transpose_csr(DeviceArena& arena, const int64_t* row_ptr, const int32_t* col,
                   const double* val, int64_t m, int64_t n, int64_t nnz, int64_t* t_row_ptr,
                   int32_t* t_col, double* t_val, cudaStream_t s);

// kind: 0 = max |a| over the row, 1 = sum |a|, 2 = (sum |a|^p)^(1/p); nnz = row_ptr[rows]
// (sets the lanes per row).
void row_norms(const int64_t* row_ptr, const double* val, int64_t rows, int64_t nnz, int kind,
               double p, double* out, cudaStream_t s);
// out_i = (v_i > 0) ? 1/sqrt(v_i) : 1 ;  acc_i *= out_i
void scale_factors(const double* norms, int64_t len, double* factors, double* acc,
                   cudaStream_t s);
// val_e <- (val_e * f_col[col_e]) * f_row[row]   when col_first (A-side: f_col = row
// factor of A applied first ...).  See setup.cu for the exact operand order.
void scale_values(const int64_t* row_ptr, const int32_t* col, double* val, int64_t rows,
                  int64_t nnz, const double* f_first, const double* f_second,
                  bool first_is_col, cudaStream_t s);
double max_abs(DeviceArena& arena, const double* v, int64_t len, cudaStream_t s);

// Permutation sorting `count` rows by decreasing length (ties by index): perm[new] = old,
// inv[old] = new.  Lengths come from a row-pointer array.
void sort_by_length_desc(DeviceArena& arena, const int64_t* row_ptr, int64_t count,
                         int32_t* perm, int32_t* inv, cudaStream_t s);
// Renumbered CSR: new row r holds old row perm_r[r] with column c renamed inv_c[c]
// (entry order kept).
void permute_csr(DeviceArena& arena, const int64_t* row_ptr, const int32_t* col,
                 const double* val, int64_t rows, const int32_t* perm_r, const int32_t* inv_c,
                 int64_t* new_row_ptr, int32_t* new_col, double* new_val, cudaStream_t s);
// Chunk list of the long rows and the SELL-32 copy of the rest (values converted to T).
template <class T>
void build_sell(DeviceArena& arena, Mat<T>& M, const double* val64, cudaStream_t s);
// out[i] = in[perm[i]]
void gather_f64(const double* in, const int32_t* perm, double* out, int64_t len, cudaStream_t s);
template <class T>
void convert_values(const double* src, T* dst, int64_t len, cudaStream_t s);

// exclusive scan of int64 values (in place allowed); out[len] receives the total
void exclusive_scan_i64(DeviceArena& arena, const int64_t* in, int64_t* out, int64_t len,
                        cudaStream_t s);

}  // namespace pdlp
