// Device-side bounds checks of index tables (dfmm_validate): every entry of a
// table is compared with the extent it indexes, and the first entry out of
// range is recorded.  The kernels only read the tables.
#include "validate.h"

namespace dfmm {

namespace {

__global__ void range_check_kernel(RangeCheck c, unsigned long long* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.n) return;
  bool ok = true;
  if (c.mode == kCheckFields) {
    const int32_t* e = (const int32_t*)c.p + i * c.stride;
    const int64_t va = e[c.a];
    ok = va >= 0 && va < c.hi_a;
    if (c.b >= 0) {
      const int64_t vb = e[c.b];
      ok = ok && vb >= 0 && va + vb <= c.hi_ab;
    }
  } else if (c.mode == kCheckCsr32 || c.mode == kCheckCsr64) {
    // offsets[0 .. n]: nondecreasing, from 0 to hi_a; entry i checks offsets[i], offsets[i + 1]
    int64_t lo, hi;
    if (c.mode == kCheckCsr32) {
      lo = ((const int32_t*)c.p)[i];
      hi = ((const int32_t*)c.p)[i + 1];
    } else {
      lo = ((const int64_t*)c.p)[i];
      hi = ((const int64_t*)c.p)[i + 1];
    }
    ok = lo >= 0 && lo <= hi && hi <= c.hi_a && (i > 0 || lo == 0) && (i + 1 < c.n || hi == c.hi_a);
  } else {   // kCheckPacked: low 25 bits of a packed word
    const uint32_t v = ((const uint32_t*)c.p)[i] & 0x1FFFFFFu;
    ok = (int64_t)v < c.hi_a;
  }
  if (!ok) atomicMin(bad, (unsigned long long)i);
}

}  // namespace

std::vector<int64_t> run_range_checks(const std::vector<RangeCheck>& checks, cudaStream_t s) {
  std::vector<int64_t> out(checks.size(), -1);
  if (checks.empty()) return out;
  unsigned long long* bad = nullptr;
  DFMM_CUDA(cudaMallocAsync((void**)&bad, checks.size() * sizeof(unsigned long long), s));
  DFMM_CUDA(cudaMemsetAsync(bad, 0xFF, checks.size() * sizeof(unsigned long long), s));
  for (size_t k = 0; k < checks.size(); ++k) {
    const RangeCheck& c = checks[k];
    if (c.n <= 0) continue;
    range_check_kernel<<<(unsigned)((c.n + 255) / 256), 256, 0, s>>>(c, bad + k);
    DFMM_CUDA(cudaGetLastError());
  }
  std::vector<unsigned long long> h(checks.size());
  DFMM_CUDA(cudaMemcpyAsync(h.data(), bad, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaFreeAsync(bad, s));
  DFMM_CUDA(cudaStreamSynchronize(s));
  for (size_t k = 0; k < checks.size(); ++k)
    if (h[k] != ~0ull) out[k] = (int64_t)h[k];
  return out;
}

}  // namespace dfmm
