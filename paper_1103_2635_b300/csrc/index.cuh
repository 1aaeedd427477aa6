// The index object behind the opaque rbc_index handle of the C ABI, shared by
// the search orchestration (api.cu) and the grouped multi-index search
// (group.cu).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <vector>

#include "common.cuh"

struct rbc_index {
  int64_t n = 0;
  int32_t d = 0, n_r = 0, s = 0, metric = 0, mode = 0, storage = 0, rerank_c = 0, plan = 0;
  int64_t list_entries = 0;
  int device = 0;             // CUDA device the index lives on
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t* reps = nullptr;    // [n_r] representative ids
  float* R32 = nullptr;       // [n_r, d] representative rows
  int* offsets = nullptr;     // [n_r + 1] list starts (entries)
  int* members = nullptr;     // [list_entries] database id of each entry
  float* X32 = nullptr;       // [list_entries, d] rows in list order
  float* psi = nullptr;       // [n_r] radius upper bounds
  float* xdist = nullptr;     // [list_entries] FP32 rho(x, r) of each entry (exact mode)
  int dpad = 0;               // low-precision row length (multiple of 64)
  void* Xlp = nullptr;        // [list_entries, dpad]
  float* xnorm = nullptr;     // [list_entries] |x~|^2
  void* xnblock = nullptr;    // [list_entries + NORM_PAD, 16] bf16 norm block (high, low)
  unsigned* lp_max = nullptr; // [4] float bits: max|x-x~|, max|x~|, max|r-r~|, max|r~|
  void* Rlp = nullptr;        // [n_r, dpad]
  float* rnorm = nullptr;     // [n_r]
  int norm_fold_col = -1;     // >= 0: Xlp carries -|x~|^2 / 2 in columns col, col + 1
  // windowed plan with representative offsets (bf16, l2): y~ = bf16(x - r)
  // of every list row (list r), its |y~|^2 and norm block; with
  // norm_fold_col >= 0 the rows carry -|y~|^2 / 2 in that column pair too
  void* Ylp = nullptr;        // [list_entries, dpad]
  float* ynorm = nullptr;     // [list_entries + NORM_PAD]
  void* ynblock = nullptr;    // [list_entries + NORM_PAD, 16]
  float* yerr_list = nullptr; // [n_r] largest |y - y~| of each list, rounded up
  float* xscale = nullptr;    // FP8: [list_entries + NORM_PAD] per-row power-of-two scales
  float* rscale = nullptr;    // FP8: [n_r]
  // device error flags of searches that could not report them when they
  // returned (searches recorded under stream capture): OR-ed in on the
  // device, read and cleared by rbc_search_check
  uint32_t* dev_status = nullptr;

  template <typename T>
  int alloc(T** out, int64_t count) {
    void* p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      rbc::set_error("index allocation of %lld bytes failed: %s",
                     (long long)(count * (int64_t)sizeof(T)), cudaGetErrorString(e));
      return RBC_ERR_OOM;
    }
    allocs.push_back(p);
    bytes += count * (int64_t)sizeof(T);
    *out = static_cast<T*>(p);
    return RBC_OK;
  }
  ~rbc_index() {
    for (void* p : allocs) cudaFree(p);
  }
};
