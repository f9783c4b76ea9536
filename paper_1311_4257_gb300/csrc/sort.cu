// Morton keys (Sec. 2.2 octree), a hand-written stable LSD radix sort of
// (key, index) pairs, and a device exclusive scan.
#include "common.h"

namespace dfmm {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortChunks = 8;
constexpr int kSortTile = kSortThreads * kSortChunks;

__global__ void morton_kernel(const double* __restrict__ pts, int64_t n, double W, uint64_t* __restrict__ keys,
                              int32_t* __restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double scale = 2097152.0 / W;   // 2^21 / W, a power of two: exact
  uint64_t q[3];
  for (int d = 0; d < 3; ++d) {
    double t = __dmul_rn(__dadd_rn(pts[3 * i + d], 0.5 * W), scale);
    double f = floor(t);
    f = f < 0.0 ? 0.0 : f;
    f = f > 2097151.0 ? 2097151.0 : f;
    q[d] = (uint64_t)f;
  }
  uint64_t key = 0;
#pragma unroll
  for (int b = 0; b < kLevelBits; ++b) {
    key |= ((q[0] >> b) & 1ull) << (3 * b + 2);
    key |= ((q[1] >> b) & 1ull) << (3 * b + 1);
    key |= ((q[2] >> b) & 1ull) << (3 * b);
  }
  keys[i] = key;
  idx[i] = (int32_t)i;
}

// ----------------------------------------------------------------- scan ---

__global__ void scan_block_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                  int64_t* __restrict__ block_sums, int64_t n) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    sum += v[k];
  }
  // inclusive warp scan of thread sums
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;   // inclusive over warps
  }
  __syncthreads();
  int64_t excl = x - sum + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = excl;
    excl += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

__global__ void scan_add_kernel(int64_t* __restrict__ out, const int64_t* __restrict__ offs, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / kScanTile];
}

__global__ void scan_total_kernel(const int64_t* in, int64_t* out, int64_t n) {
  out[n] = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

// Scan without the trailing total, recursive over block sums.
void scan_rec(const int64_t* in, int64_t* out, int64_t n, int64_t* scratch, size_t scratch_elems,
              cudaStream_t s) {
  if (n <= 0) return;
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if ((size_t)(2 * nb) > scratch_elems) throw Error(-3, "scan scratch too small");
  int64_t* sums = scratch;
  int64_t* sums_scan = scratch + nb;
  scan_block_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, sums, n);
  if (nb > 1) {
    scan_rec(sums, sums_scan, nb, scratch + 2 * nb, scratch_elems - 2 * nb, s);
    scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, sums_scan, n);
  }
}

// ----------------------------------------------------------- radix sort ---

__global__ void radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                  int64_t* __restrict__ counts, int nblocks) {
  __shared__ unsigned hist[256];
  hist[threadIdx.x] = 0;
  __syncthreads();
  int64_t start = (int64_t)blockIdx.x * kSortTile;
  int64_t end = min(n, start + kSortTile);
  for (int64_t i = start + threadIdx.x; i < end; i += kSortThreads)
    atomicAdd(&hist[(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = hist[threadIdx.x];
}

__global__ void radix_scatter_kernel(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                     uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                                     int shift, const int64_t* __restrict__ offs, int nblocks) {
  __shared__ int64_t base[256];
  __shared__ int running[256];
  __shared__ int wcount[kSortThreads / 32][257];
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
  running[tid] = 0;
  for (int w = 0; w < kSortThreads / 32; ++w) wcount[w][tid] = 0;
  __syncthreads();
  int64_t start = (int64_t)blockIdx.x * kSortTile;
  for (int c = 0; c < kSortChunks; ++c) {
    int64_t i = start + (int64_t)c * kSortThreads + tid;
    bool ok = i < n;
    uint64_t key = ok ? kin[i] : 0;
    int digit = ok ? (int)((key >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) wcount[warp][digit] = __popc(peers);
    __syncthreads();
    if (ok) {
      int pre = 0;
      for (int w = 0; w < warp; ++w) pre += wcount[w][digit];
      int64_t pos = base[digit] + running[digit] + pre + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) {
      tot += wcount[w][tid];
      wcount[w][tid] = 0;
    }
    running[tid] += tot;
    if (tid == 0)
      for (int w = 0; w < kSortThreads / 32; ++w) wcount[w][256] = 0;
    __syncthreads();
  }
}

}  // namespace

void launch_morton_keys(const double* pts, int64_t n, double W, uint64_t* keys, int32_t* idx, cudaStream_t s) {
  if (n <= 0) return;
  morton_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, n, W, keys, idx);
  DFMM_CUDA(cudaGetLastError());
}

size_t scan_scratch_bytes(int64_t n) {
  size_t e = 0;
  int64_t m = n;
  while (m > 0) {
    int64_t nb = (m + kScanTile - 1) / kScanTile;
    e += 2 * nb;
    if (nb <= 1) break;
    m = nb;
  }
  return (e + 16) * sizeof(int64_t);
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* scratch, size_t scratch_bytes,
                        cudaStream_t s) {
  scan_rec(in, out, n, (int64_t*)scratch, scratch_bytes / sizeof(int64_t), s);
  scan_total_kernel<<<1, 1, 0, s>>>(in, out, n);
  DFMM_CUDA(cudaGetLastError());
}

size_t radix_sort_scratch_bytes(int64_t n) {
  int64_t nb = (n + kSortTile - 1) / kSortTile;
  int64_t m = 256 * nb;
  return (size_t)(2 * m + 1) * sizeof(int64_t) + scan_scratch_bytes(m) + 256;
}

void radix_sort_pairs(uint64_t* keys, int32_t* vals, uint64_t* keys2, int32_t* vals2, int64_t n, int bits,
                      void* scratch, size_t scratch_bytes, cudaStream_t s) {
  if (n <= 1) return;
  int nb = (int)((n + kSortTile - 1) / kSortTile);
  int64_t m = 256 * (int64_t)nb;
  int64_t* counts = (int64_t*)scratch;
  int64_t* offs = counts + m;
  void* sc = offs + m + 1;
  size_t sc_bytes = scratch_bytes - (size_t)(2 * m + 1) * sizeof(int64_t);
  uint64_t *ka = keys, *kb = keys2;
  int32_t *va = vals, *vb = vals2;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(ka, n, shift, counts, nb);
    exclusive_scan_i64(counts, offs, m, sc, sc_bytes, s);
    radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, offs, nb);
    DFMM_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    DFMM_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace dfmm
