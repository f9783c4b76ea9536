// Tensor-core form of the translation stage  y[dst] += T_op x[src]  (M2L, and
// the other translations that share the gather / GEMM / scatter-add shape).
//
// One CTA computes D = X Tb^T for one tile: 128 gathered source rows (pairs x
// right-hand sides) against up to 256 real output components of one operator,
// on the 5th-generation tensor cores (tcgen05.mma, kind::tf32, accumulators in
// tensor memory).
//
//  * Complex arithmetic as a real GEMM: a state row is interleaved (re, im)
//    floats, so with K = 2 R_s and N = 2 R_t the real-block operator
//    Tb[2p][2q] = Re T, Tb[2p][2q+1] = -Im T, Tb[2p+1][2q] = Im T,
//    Tb[2p+1][2q+1] = Re T maps a source row directly to an interleaved
//    target row.
//  * Split TF32: every operand x = hi + lo with hi = x rounded to TF32 and
//    lo = (x - hi) rounded to TF32 (x is then represented to 2^-22 relative).
//    The tensor core's FP32 accumulation does not round to nearest, so its
//    error grows with the number of accumulation steps into one accumulator;
//    the large term Ahi Bhi goes to one accumulator (one step per K = 8) and
//    the small terms Ahi Blo + Alo Bhi to a second one, and the two are added
//    in FP32 in the epilogue (Alo Blo, below 2^-22, is left out).
//  * No conversion in the main loop: the operators are stored at plan time as
//    an image of their shared-memory tiles (real-block form, TF32 hi and lo,
//    canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
//    K-adjacent cores 128 B apart, 8-row groups 512 B apart), and the source
//    states are split into hi / lo arrays by an elementwise pass before the
//    stage.  Each stage's operator tile (hi and lo, contiguous in the image)
//    arrives by one bulk copy (cp.async.bulk, completing on an mbarrier), the
//    gathered state rows by 16-byte asynchronous copies (cp.async); 4 stages
//    of 16 K-floats.
//  * One thread issues the MMAs and commits them to an mbarrier; stage reuse
//    waits on it with a time limit.  The epilogue reads the accumulators with
//    tcgen05.ld (row = gathered column) and scatter-adds them into the target
//    states with float4 atomics.
#include "apply.h"

namespace dfmm {

namespace {

constexpr int TC_M = 128;
constexpr int TC_BK = 16;
constexpr int TC_NMAX = 256;
constexpr int TC_THREADS = 256;
constexpr int TC_STAGES = 4;
constexpr int A_BYTES = TC_M * TC_BK * 4;          // 8 KB
constexpr int B_BYTES = TC_NMAX * TC_BK * 4;       // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = TC_STAGES * STAGE_BYTES + 1024 + 128;
constexpr int TMEM_COLS = 512;   // two accumulators of up to 256 columns
constexpr int CORE_SBO = (TC_BK / 4) * 128;        // 512 B between 8-row groups
constexpr unsigned long long WAIT_NS = 200000000ull;    // 0.2 s bound on every wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in one stage tile (canonical K-major, no swizzle)
__host__ __device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
  return (uint32_t)((row >> 3) * CORE_SBO + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start, LBO = 128 B, SBO = 512 B,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((uint32_t)CORE_SBO >> 4) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

// instruction descriptor, kind::tf32: D f32, A and B tf32, K-major, M = 128
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete.  Gives up (false)
// after WAIT_NS, or as soon as another CTA has reported a timeout, and then
// reports the timeout itself.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* status) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > WAIT_NS || (*(volatile unsigned*)status & kStatusTimeout)) {
      atomicOr(status, kStatusTimeout);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
// 16 zero bytes (source size 0: nothing is read)
__device__ __forceinline__ void cp_async16_zero(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, 0;" ::"r"(saddr), "l"(g) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bulk global -> shared copy of `bytes` (multiple of 16), completing on `bar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// fire-and-forget vector add to global memory (no value returned)
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Operator image: for every (operator, N block b, K chunk c) two tiles (hi,
// then lo) of rows_b x 16 floats in the stage layout,
// rows_b = min(TC_NMAX, 2M - TC_NMAX b).
__global__ void op_image_kernel(const float2* __restrict__ ops, int M, int Kd, int nops, float* __restrict__ img) {
  const int nchunk = 2 * Kd / TC_BK;
  const int nb = (2 * M + TC_NMAX - 1) / TC_NMAX;
  const int64_t op_floats = (int64_t)2 * (2 * M) * (2 * Kd);
  int64_t g = blockIdx.x;          // (op, b, c)
  const int c = (int)(g % nchunk);
  g /= nchunk;
  const int b = (int)(g % nb);
  const int op = (int)(g / nb);
  if (op >= nops) return;
  const int rows = min(TC_NMAX, 2 * M - TC_NMAX * b);
  float* hi = img + op * op_floats + (int64_t)b * nchunk * 2 * TC_NMAX * TC_BK + (int64_t)c * 2 * rows * TC_BK;
  float* lo = hi + rows * TC_BK;
  const float2* T = ops + (size_t)op * M * Kd;
  for (int e = threadIdx.x; e < rows * TC_BK; e += blockDim.x) {
    const int row = e / TC_BK, kk = e % TC_BK;
    const int j = TC_NMAX * b + row, k = c * TC_BK + kk;
    const float2 tv = T[(size_t)(j >> 1) * Kd + (k >> 1)];
    const int cj = j & 1, ck = k & 1;
    const float v = (cj == ck) ? tv.x : (cj == 0 ? -tv.y : tv.y);
    const float h = tf32_rna(v);
    const uint32_t off = kmaj_off(row, kk) / 4;
    hi[off] = h;
    lo[off] = tf32_rna(v - h);
  }
}

__global__ void split_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ hi, float* __restrict__ lo) {
  int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i >= n) return;
  float4 v = *(const float4*)(x + i);
  float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
  float4 l = make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y), tf32_rna(v.z - h.z), tf32_rna(v.w - h.w));
  *(float4*)(hi + i) = h;
  *(float4*)(lo + i) = l;
}

__global__ __launch_bounds__(TC_THREADS, 1) void gemm_tc_kernel(GemmArgs a, TcArgs t, unsigned* status) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int srcrow[TC_M];
  __shared__ float2* dstp[TC_M];
  __shared__ int s_ok;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + TC_STAGES * STAGE_BYTES);   // MMAs of a stage done
  uint64_t* fullb = bars + TC_STAGES;                               // operator tile of a stage landed
  uint32_t* tmem_slot = (uint32_t*)(fullb + TC_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 tile = a.tiles[blockIdx.x];
  const int ncol = tile.z * a.nrhs;
  const int b = blockIdx.y;
  const int n0 = TC_NMAX * b;                        // first real output component
  const int n = min(TC_NMAX, 2 * a.M - n0);          // multiple of 16
  const int Kreal = 2 * a.Kd;                        // multiple of 16
  const int nchunk = Kreal / TC_BK;
  const int64_t op_floats = (int64_t)2 * (2 * a.M) * Kreal;
  const float* img = t.img + tile.x * op_floats + (int64_t)b * nchunk * 2 * TC_NMAX * TC_BK;

  if (tid < TC_M) {
    int sr = -1;
    float2* dp = nullptr;
    if (tid < ncol) {
      const int p = tile.y + tid / a.nrhs, k = tid % a.nrhs;
      const int2 pr = a.pairs[p];
      sr = pr.x * a.nrhs + k;
      dp = a.dst + ((int64_t)pr.y * a.nrhs + k) * a.dst_ld;
    }
    srcrow[tid] = sr;
    dstp[tid] = dp;
  }
  if (tid == 0) s_ok = (*(volatile unsigned*)status & kStatusTimeout) ? 0 : 1;
  __syncthreads();
  if (!s_ok) return;   // an earlier CTA gave up: skip the work, hold no tensor memory
  if (tid == 0) {
    for (int i = 0; i < TC_STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullb[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_tf32(n);
  const uint32_t sbase = smem_u32(smem);

  // asynchronous copies of chunk c into its stage: A hi/lo (128 rows x 4
  // pieces of 16 B each) and B hi/lo (n rows x 4 pieces, contiguous image)
  auto issue = [&](int c) {
    const int st = c % TC_STAGES;
    const uint32_t sA = sbase + st * STAGE_BYTES;
    const uint32_t sB = sA + 2 * A_BYTES;
    const int k0 = c * TC_BK;
    for (int e = tid; e < TC_M * 8; e += TC_THREADS) {
      const int row = e & (TC_M - 1), piece = (e >> 7) & 3, part = e >> 9;   // part 0 = hi, 1 = lo
      const int sr = srcrow[row];
      const uint32_t dsts = sA + part * A_BYTES + kmaj_off(row, 4 * piece);
      const float* base = part ? t.src_lo : t.src_hi;
      if (sr >= 0) cp_async16(dsts, base + (int64_t)sr * Kreal + k0 + 4 * piece);
      else cp_async16_zero(dsts, base);
    }
    if (tid == 0) {   // operator tile: hi then lo, n x 16 floats each, one bulk copy
      const uint32_t bytes = (uint32_t)(2 * n * TC_BK * 4);
      mbar_expect_tx(smem_u32(&fullb[st]), bytes);
      bulk_g2s(sB, img + (int64_t)c * 2 * n * TC_BK, bytes, smem_u32(&fullb[st]));
    }
  };

  for (int c = 0; c < TC_STAGES - 1; ++c) {
    if (c < nchunk) issue(c);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  int issued = 0;
  for (int c = 0; c < nchunk; ++c) {
    const int st = c % TC_STAGES;
    asm volatile("cp.async.wait_group %0;" ::"n"(TC_STAGES - 2) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) s_ok = mbar_wait(smem_u32(&fullb[st]), (c / TC_STAGES) & 1, status) ? 1 : 0;
    __syncthreads();
    if (!s_ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = sbase + st * STAGE_BYTES, al = ah + A_BYTES, bh = al + A_BYTES;
      const uint32_t bl = bh + (uint32_t)(n * TC_BK * 4);    // lo tile follows the hi tile
#pragma unroll
      for (int s = 0; s < TC_BK / 8; ++s) {
        const uint32_t off = 256u * s;
        const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bh + off), idesc, acc);
        mma_tf32(tmem + (uint32_t)TC_NMAX, smem_desc(ah + off), smem_desc(bl + off), idesc, acc);
        mma_tf32(tmem + (uint32_t)TC_NMAX, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bars[st]))
                   : "memory");
    }
    issued = c + 1;
    // refill the stage of chunk c - 1 with chunk c + STAGES - 1 once its MMAs are done
    const int cn = c + TC_STAGES - 1;
    if (cn < nchunk) {
      if (c >= 1) {
        const int cp = c - 1;
        if (tid == 0) s_ok = mbar_wait(smem_u32(&bars[cp % TC_STAGES]), (cp / TC_STAGES) & 1, status) ? 1 : 0;
        __syncthreads();
        if (!s_ok) break;
      }
      issue(cn);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  // wait (bounded) for the last issued chunk: MMAs complete in order
  if (tid == 0) {
    int ok = s_ok;
    if (issued > 0) {
      const int last = issued - 1;
      ok = mbar_wait(smem_u32(&bars[last % TC_STAGES]), (last / TC_STAGES) & 1, status) && ok;
    }
    s_ok = ok;
  }
  __syncthreads();
  const bool ok = s_ok != 0 && issued == nchunk;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: accumulator lane 32 (warp % 4) + lane is gathered column c;
  // warps w and w + 4 share the lane quarter and split the 16-column chunks
  const int quarter = warp & 3, half = warp >> 2;
  float2* dp = dstp[32 * quarter + lane];
  for (int j0 = 16 * half; j0 < n; j0 += 32) {
    float v[16], w[16];
    tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)j0, v);
    tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)TC_NMAX + (uint32_t)j0, w);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] += w[i];
    if (dp && ok) {
      float* out = (float*)dp + n0 + j0;
#pragma unroll
      for (int i = 0; i < 4; ++i) red_add4(out + 4 * i, v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

int gemm_tc_columns() { return TC_M; }

bool gemm_tc_supported(int M, int Kd) { return M % 8 == 0 && Kd % 8 == 0; }

int64_t tc_image_floats(int M, int Kd, int nops) { return (int64_t)nops * 2 * (2 * M) * (2 * Kd); }

void build_tc_image(const float2* ops, int M, int Kd, int nops, float* img, cudaStream_t s) {
  if (nops == 0) return;
  if (M % 8 != 0 || Kd % 8 != 0) throw Error(-5, "tensor-core stage needs ranks padded to a multiple of 8");
  const int nchunk = 2 * Kd / TC_BK;
  const int nb = (2 * M + TC_NMAX - 1) / TC_NMAX;
  int64_t blocks = (int64_t)nops * nb * nchunk;
  op_image_kernel<<<(unsigned)blocks, 256, 0, s>>>(ops, M, Kd, nops, img);
  DFMM_CUDA(cudaGetLastError());
}

void launch_split(const float2* x, int64_t rows, int ld, float* hi, float* lo, cudaStream_t s) {
  int64_t n = rows * ld * 2;   // floats, a multiple of 16
  if (n == 0) return;
  split_kernel<<<(unsigned)((n / 4 + 255) / 256), 256, 0, s>>>((const float*)x, n, hi, lo);
  DFMM_CUDA(cudaGetLastError());
}

void launch_gemm_stage_tc(const GemmArgs& a, const TcArgs& t, unsigned* status, cudaStream_t s) {
  if (a.ntiles == 0) return;
  if (!gemm_tc_supported(a.M, a.Kd) || a.src_ld != a.Kd)
    throw Error(-5, "tensor-core stage needs ranks padded to a multiple of 8 and dense source rows");
  static bool attr = false;
  if (!attr) {
    DFMM_CUDA(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  dim3 grid((unsigned)a.ntiles, (unsigned)((2 * a.M + TC_NMAX - 1) / TC_NMAX));
  gemm_tc_kernel<<<grid, TC_THREADS, SMEM_BYTES, s>>>(a, t, status);
  DFMM_CUDA(cudaGetLastError());
}

}  // namespace dfmm
