// Shared definitions of the dfmm library (CUDA side and host side).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <stdexcept>
#include <string>

namespace dfmm {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define DFMM_CUDA(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::dfmm::Error(e_ == cudaErrorMemoryAllocation ? -3 : -4,                       \
                          std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

constexpr int kLevelBits = 21;   // Morton bits per axis; deepest level
constexpr int kMaxLevels = 22;

// Device-side status word bits (written by kernels that check themselves).
constexpr unsigned kStatusBounds = 1u;
constexpr unsigned kStatusTimeout = 2u;

// ------------------------------------------------------------ plan kernels ---
// All take raw device pointers; launch on `stream`.

// q_d = floor((x_d + W/2) * 2^21 / W) clamped, interleaved into a 63-bit key.
void launch_morton_keys(const double* pts, int64_t n, double W, uint64_t* keys, int32_t* idx,
                        cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
// tmp buffers: keys2, vals2 of n entries; returns in keys/vals.
void radix_sort_pairs(uint64_t* keys, int32_t* vals, uint64_t* keys2, int32_t* vals2, int64_t n, int bits,
                      void* scratch, size_t scratch_bytes, cudaStream_t s);
size_t radix_sort_scratch_bytes(int64_t n);

// Exclusive scan of n int32 counts into offsets (n+1 entries; offsets[n] = total).
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* scratch, size_t scratch_bytes,
                        cudaStream_t s);
size_t scan_scratch_bytes(int64_t n);

}  // namespace dfmm
