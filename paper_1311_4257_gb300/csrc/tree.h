// Device octree and list construction (see tree.cu).
#pragma once
#include <cstdint>
#include <vector>

#include "common.h"

namespace dfmm {

// Owns device allocations; memory is released when the arena (or a mark
// taken on it) goes out of scope.
class DevArena {
 public:
  DevArena() = default;
  DevArena(const DevArena&) = delete;
  ~DevArena() { release(0); }
  template <class T>
  T* alloc(int64_t n) {
    void* p = nullptr;
    size_t bytes = (size_t)(n > 0 ? n : 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(-3, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    ptrs_.push_back(p);
    bytes_ += bytes;
    sizes_.push_back(bytes);
    return (T*)p;
  }
  size_t mark() const { return ptrs_.size(); }
  void release(size_t m) {
    while (ptrs_.size() > m) {
      cudaFree(ptrs_.back());
      bytes_ -= sizes_.back();
      ptrs_.pop_back();
      sizes_.pop_back();
    }
  }
  size_t bytes() const { return bytes_; }

 private:
  std::vector<void*> ptrs_;
  std::vector<size_t> sizes_;
  size_t bytes_ = 0;
};

struct ArenaMark {
  DevArena& a;
  size_t m;
  explicit ArenaMark(DevArena& ar) : a(ar), m(ar.mark()) {}
  ~ArenaMark() { a.release(m); }
};

struct LevelPtrs {
  const uint64_t* prefix;
  const int32_t* coords;
  const int32_t* first;
  const int32_t* count;
  const int32_t* parent;
  const int32_t* child_first;
  const int32_t* nchild;
  const uint8_t* leaf;
  int64_t n;
  int l;
  double w;
};

struct TreeLevel {
  int l = 0;
  double w = 0;
  int64_t n = 0;
  uint64_t* prefix = nullptr;
  int32_t* coords = nullptr;
  int32_t* first = nullptr;
  int32_t* count = nullptr;
  int32_t* parent = nullptr;
  int32_t* child_first = nullptr;
  int32_t* nchild = nullptr;
  uint8_t* leaf = nullptr;
  std::vector<uint64_t> h_prefix;
  std::vector<int32_t> h_coords, h_first, h_count, h_parent, h_child_first, h_nchild;
  std::vector<uint8_t> h_leaf;
  LevelPtrs ptrs() const { return {prefix, coords, first, count, parent, child_first, nchild, leaf, n, l, w}; }
  void download(cudaStream_t s);
};

struct PairList {
  int64_t n = 0;
  std::vector<int32_t> tgt, src, m, din, dout;
};

class TreeBuilder {
 public:
  std::vector<TreeLevel> levels;
  LevelPtrs* d_levels = nullptr;
  void build(const uint64_t* d_keys, int64_t N, double W, int leaf_max, cudaStream_t s, DevArena& ar);
  // Same-level pairs of level l from the template of parent offsets.
  // mode 0: HF (keep if not near at width w; lim = 4 w^2), mode 1: V list.
  PairList pairs(int l, const std::vector<int32_t>& tmpl, int mode, int64_t lim, bool dirs, int ncell,
                 cudaStream_t s, DevArena& ar);
  void uw_lists(int l_lf0, cudaStream_t s, DevArena& ar, std::vector<int32_t>& U, std::vector<int32_t>& W,
                unsigned* d_status);
};

}  // namespace dfmm
