// Peak-rate probes of the GPU, for the rooflines of the benchmark report (the
// paper has no counterpart): FP32 and FP64 fused multiply-adds on the CUDA
// cores, the special-function unit (sine / cosine, reciprocal square root),
// and dense tcgen05 MMAs of kind::tf32 and kind::f16 from shared memory.
// Each probe is a short kernel with independent chains, timed with CUDA
// events on one stream; the rates are whole-GPU operations per second.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "common.h"
#include "dfmm.h"
#include "internal.h"

namespace dfmm {
namespace {

constexpr int kChains = 8;

__global__ void fma32_kernel(float* out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1234.5f) out[threadIdx.x] = s;   // keeps the chains alive
}

__global__ void fma64_kernel(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1234.5) out[threadIdx.x] = s;
}

// one fast sine and one fast cosine per chain and step
__global__ void sincos_kernel(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3f + 0.1f * k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __sinf(a[k]) + __cosf(a[k]);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void rsqrt_kernel(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.f + threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = rsqrtf(a[k]) + 1.f;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1234.5f) out[threadIdx.x] = s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no swizzle: 8-row x 16-byte core matrices, K-adjacent cores 128 B
// apart, 8-row groups 256 B apart (one MMA's 32 bytes of K per row)
__device__ __forceinline__ uint64_t probe_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

constexpr int PR_M = 128, PR_N = 256;
constexpr int PR_SMEM = 64 * 1024;

// kind = 0: tf32 (K = 8 per MMA), 1: f16 (K = 16); D f32, M = 128, N = 256.
// One thread per CTA issues `iters` MMAs into one accumulator from a zeroed
// 4 KB A tile and 8 KB B tile; the wait for their completion is time-limited.
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int kind, int iters, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  for (int i = threadIdx.x; i < PR_SMEM / 16; i += blockDim.x) ((uint4*)sm)[i] = make_uint4(0, 0, 0, 0);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(PR_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = (1u << 4) | ((kind == 0 ? 2u : 0u) << 7) | ((kind == 0 ? 2u : 0u) << 10) |
                           ((uint32_t)(PR_N >> 3) << 17) | ((uint32_t)(PR_M >> 4) << 24);
    const uint64_t da = probe_desc(smem_u32(sm)), db = probe_desc(smem_u32(sm + 32 * 1024));
    for (int i = 0; i < iters; ++i) {
      const uint32_t acc = i > 0 ? 1u : 0u;
      if (kind == 0)
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
      else
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
    // time-limited wait (1 s) for the MMAs to complete
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
      uint32_t ok;
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                   : "=r"(ok)
                   : "r"(smem_u32(&bar))
                   : "memory");
      if (ok) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) {
        atomicOr(status, kStatusTimeout);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PR_N));
}

template <class F>
double time_ms(cudaStream_t s, F&& launch) {
  cudaEvent_t a, b;
  DFMM_CUDA(cudaEventCreate(&a));
  DFMM_CUDA(cudaEventCreate(&b));
  launch();   // warm-up
  DFMM_CUDA(cudaGetLastError());
  DFMM_CUDA(cudaEventRecord(a, s));
  launch();
  DFMM_CUDA(cudaEventRecord(b, s));
  DFMM_CUDA(cudaEventSynchronize(b));
  DFMM_CUDA(cudaGetLastError());
  float ms = 0;
  DFMM_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

}  // namespace
}  // namespace dfmm

extern "C" int dfmm_measure_peaks(dfmm_peaks* out) {
  using namespace dfmm;
  if (!out) return set_error(DFMM_ERR_INVALID, "out is NULL");
  try {
    std::memset(out, 0, sizeof(*out));
    int dev = 0, nsm = 0;
    DFMM_CUDA(cudaGetDevice(&dev));
    DFMM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    out->sm_count = nsm;
    cudaStream_t s;
    DFMM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{s};
    void* scratch = nullptr;
    DFMM_CUDA(cudaMalloc(&scratch, 4096));
    struct MG { void* p; ~MG() { cudaFree(p); } } mg{scratch};
    unsigned* status = (unsigned*)scratch;
    DFMM_CUDA(cudaMemsetAsync(status, 0, 4, s));
    const int blocks = nsm * 8, threads = 256;
    const double lanes = (double)blocks * threads * kChains;
    {
      const int it = 32768;
      double ms = time_ms(s, [&] { fma32_kernel<<<blocks, threads, 0, s>>>((float*)scratch + 16, it, 0.999f, 1e-3f); });
      out->fp32_fma_tflops = 2.0 * lanes * it / (ms * 1e-3) / 1e12;
    }
    {
      const int it = 512;
      double ms = time_ms(s, [&] { fma64_kernel<<<blocks, threads, 0, s>>>((double*)scratch + 16, it, 0.999, 1e-3); });
      out->fp64_fma_tflops = 2.0 * lanes * it / (ms * 1e-3) / 1e12;
    }
    {
      const int it = 2048;
      double ms = time_ms(s, [&] { sincos_kernel<<<blocks, threads, 0, s>>>((float*)scratch + 16, it); });
      out->sincos_gops = lanes * it / (ms * 1e-3) / 1e9;   // sine + cosine pairs
    }
    {
      const int it = 4096;
      double ms = time_ms(s, [&] { rsqrt_kernel<<<blocks, threads, 0, s>>>((float*)scratch + 16, it); });
      out->rsqrt_gops = lanes * it / (ms * 1e-3) / 1e9;
    }
    DFMM_CUDA(cudaFuncSetAttribute(mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PR_SMEM));
    for (int kind = 0; kind < 2; ++kind) {
      const int it = 16384;
      double ms = time_ms(s, [&] { mma_probe_kernel<<<nsm, 128, PR_SMEM, s>>>(kind, it, status); });
      const double k = kind == 0 ? 8.0 : 16.0;
      const double tf = 2.0 * PR_M * PR_N * k * it * nsm / (ms * 1e-3) / 1e12;
      if (kind == 0) out->tf32_mma_tflops = tf;
      else out->f16_mma_tflops = tf;
    }
    unsigned st = 0;
    DFMM_CUDA(cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost));
    if (st) return set_error(DFMM_ERR_TIMEOUT, "an MMA probe's wait gave up");
    return DFMM_OK;
  } catch (const Error& e) {
    return set_error(e.code, e.what());
  }
}
