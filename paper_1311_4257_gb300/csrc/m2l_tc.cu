// Tensor-core form of the translation stage  y[dst] += T_op x[src]  (M2L, and
// the other translations that share the gather / GEMM / scatter-add shape).
//
// One CTA computes D = X Tb^T for one tile: 128 gathered source rows (pairs x
// right-hand sides) against up to 256 real output components of one operator,
// on the 5th-generation tensor cores (tcgen05.mma, kind::f16 with FP32
// accumulation in tensor memory).
//
//  * Complex arithmetic as a real GEMM: a state row is interleaved (re, im)
//    floats, so with K = 2 R_s and N = 2 R_t the real-block operator
//    Tb[2p][2q] = Re T, Tb[2p][2q+1] = -Im T, Tb[2p+1][2q] = Im T,
//    Tb[2p+1][2q+1] = Re T maps a source row directly to an interleaved
//    target row.
//  * Scaled FP16 split: each source row x is scaled by a power of two
//    s >= max |x| (exact), and x / s = hi + lo with hi = fp16(x / s) and
//    lo = fp16(x / s - hi); each operator likewise with one power of two t.
//    x is then represented to about 2^-22 of its row's largest entry (lo is
//    subnormal only where that bound is absolute anyway).  The products
//    hi hi, hi lo and lo hi are exact in FP32; the epilogue multiplies by s t.
//  * The tensor core's FP32 accumulation does not round to nearest, so its
//    error grows with the number of accumulation steps into one accumulator;
//    the large term Ahi Bhi goes to one accumulator (one step per K = 16) and
//    the small terms Ahi Blo + Alo Bhi to a second one, added in FP32 in the
//    epilogue (Alo Blo, below 2^-22, is left out).
//  * No conversion in the main loop: operators are stored at plan time as an
//    image of their shared-memory tiles (real-block form, scaled FP16 hi and
//    lo, canonical K-major layout without swizzle: 8-row x 16-byte core
//    matrices, K-adjacent cores 128 B apart, 8-row groups 512 B apart; as
//    many bytes as the complex64 operator), and the source states are split
//    by a pass before the stage.  Each stage's operator tile arrives by one
//    bulk copy (cp.async.bulk, completing on an mbarrier), the gathered state
//    rows by 16-byte asynchronous copies (cp.async), 8 lanes per row so that
//    one warp-wide copy reads 4 rows x 2 contiguous 64-byte segments instead of
//    32 scattered pieces; 4 stages of 32 K-values.
//  * One thread issues the MMAs and commits them to an mbarrier; stage reuse
//    waits on it with a time limit.  The epilogue reads the accumulators with
//    tcgen05.ld in the .16x256b shape (TMEM lane = gathered column; four lanes
//    of a warp hold 8 consecutive outputs of one column) and scatter-adds them
//    into the target states with return-free 8-byte reductions, so one warp
//    instruction covers 8 target rows x 32 contiguous bytes.
#include <cuda_fp16.h>

#include <algorithm>

#include "apply.h"
#include "tcgen05.cuh"

namespace dfmm {

namespace {

constexpr int TC_M = 128;
constexpr int TC_BK = 32;                          // K values (fp16) per stage
constexpr int TC_NMAX = 256;
constexpr int TC_PRODUCERS = 128;                 // warps 0-3: gather the 128 rows of a chunk
constexpr int TC_MMA_WARP = 8;                     // warps 4-7: epilogue; warp 8: MMA issuer
constexpr int TC_THREADS = 288;
constexpr int TC_STAGES = 4;
constexpr int A_BYTES = TC_M * TC_BK * 2;          // 8 KB
constexpr int B_BYTES = TC_NMAX * TC_BK * 2;       // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = TC_STAGES * STAGE_BYTES + 1024 + 256;   // stages, alignment, barriers
constexpr int TMEM_COLS = 512;                     // two accumulators of up to 256 columns
constexpr int CORE_SBO = (TC_BK / 8) * 128;        // 512 B between 8-row groups

using namespace tc;

// byte offset of fp16 element (row, k) in one stage tile
__host__ __device__ __forceinline__ uint32_t kmaj(int row, int k) { return tc::kmaj_off(row, k, CORE_SBO); }

// per-operator scale: power of two >= max |entry|
__global__ void op_scale_kernel(const float2* __restrict__ ops, int64_t per_op, float* __restrict__ scale) {
  __shared__ float red[256];
  const float2* T = ops + (size_t)blockIdx.x * per_op;
  float m = 0.f;
  for (int64_t e = threadIdx.x; e < per_op; e += blockDim.x) m = fmaxf(m, fmaxf(fabsf(T[e].x), fabsf(T[e].y)));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) scale[blockIdx.x] = pow2_above(red[0]);
}

// Operator image: for every (operator, N block b, K chunk c) two tiles (hi,
// then lo) of rows_b x 32 fp16 values in the stage layout,
// rows_b = min(TC_NMAX, 2M - TC_NMAX b); values scaled by 1 / scale[op].
__global__ void op_image_kernel(const float2* __restrict__ ops, const float* __restrict__ scale, int M, int Kd,
                                int nops, __half* __restrict__ img) {
  const int Kreal = 2 * Kd;
  const int nchunk = (Kreal + TC_BK - 1) / TC_BK;
  const int nb = (2 * M + TC_NMAX - 1) / TC_NMAX;
  const int64_t op_elems = (int64_t)2 * (2 * M) * (nchunk * TC_BK);
  int64_t g = blockIdx.x;          // (op, b, c)
  const int c = (int)(g % nchunk);
  g /= nchunk;
  const int b = (int)(g % nb);
  const int op = (int)(g / nb);
  if (op >= nops) return;
  const int rows = min(TC_NMAX, 2 * M - TC_NMAX * b);
  __half* hi = img + op * op_elems + (int64_t)b * nchunk * 2 * TC_NMAX * TC_BK + (int64_t)c * 2 * rows * TC_BK;
  __half* lo = hi + rows * TC_BK;
  const float2* T = ops + (size_t)op * M * Kd;
  const float inv = 1.f / scale[op];
  for (int e = threadIdx.x; e < rows * TC_BK; e += blockDim.x) {
    const int row = e / TC_BK, kk = e % TC_BK;
    const int j = TC_NMAX * b + row, k = c * TC_BK + kk;
    float v = 0.f;
    if (k < Kreal) {
      const float2 tv = T[(size_t)(j >> 1) * Kd + (k >> 1)];
      const int cj = j & 1, ck = k & 1;
      v = ((cj == ck) ? tv.x : (cj == 0 ? -tv.y : tv.y)) * inv;
    }
    __half h, l;
    split_h(v, h, l);
    const uint32_t off = kmaj(row, kk) / 2;
    hi[off] = h;
    lo[off] = l;
  }
}

// one warp per source row of len floats (a multiple of 16): scale and split
__global__ void split_kernel(const float* __restrict__ x, int64_t rows, int len, __half* __restrict__ hi,
                             __half* __restrict__ lo, float* __restrict__ scale) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float* xr = x + row * len;
  float m = 0.f;
  for (int k = lane * 4; k < len; k += 128) {
    const float4 v = *(const float4*)(xr + k);
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float s = pow2_above(m);
  const float inv = 1.f / s;
  if (lane == 0) scale[row] = s;
  for (int k = lane * 4; k < len; k += 128) {
    const float4 v = *(const float4*)(xr + k);
    __half h0, h1, h2, h3, l0, l1, l2, l3;
    split_h(v.x * inv, h0, l0);
    split_h(v.y * inv, h1, l1);
    split_h(v.z * inv, h2, l2);
    split_h(v.w * inv, h3, l3);
    __half2* ph = (__half2*)(hi + row * len + k);
    __half2* pl = (__half2*)(lo + row * len + k);
    ph[0] = __halves2half2(h0, h1);
    ph[1] = __halves2half2(h2, h3);
    pl[0] = __halves2half2(l0, l1);
    pl[1] = __halves2half2(l2, l3);
  }
}

__device__ __forceinline__ void named_bar_producers() { asm volatile("bar.sync 1, %0;" ::"n"(TC_PRODUCERS) : "memory"); }

// Persistent, warp-specialised stage kernel.  Work item = (tile, N block);
// CTA x takes items x, x + gridDim.x, ...  Roles:
//   warps 0-3  producers: 8 threads gather one row's K chunk (its 64-byte hi
//              and lo segments, 16 bytes each), 8 rows per thread (cp.async,
//              completion counted on the stage's full barrier),
//              thread 0 also bulk-copies the operator tile; they run up to
//              TC_STAGES chunks ahead, across items.
//   warp 8     one thread issues the MMAs of a chunk once its stage is full,
//              commits them to the stage's empty barrier, and after an
//              item's last chunk to acc_full; it waits for acc_empty before
//              it overwrites the accumulators with the next item.
//   warps 4-7  epilogue: read the accumulators (warp 4 + q reads TMEM lanes
//              32q..32q+31 = gathered columns, as two 16-lane blocks of the
//              .16x256b shape), scatter-add into the target states and then
//              release them (acc_empty).
// Every wait is time-limited; on a timeout the CTA reports it, stops issuing,
// lets its own copies and MMAs land, frees its tensor memory and returns.
__global__ __launch_bounds__(TC_THREADS, 1) void gemm_tc_kernel(GemmArgs a, TcArgs t, int64_t nitems, int nb,
                                                                unsigned* status) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_start;
  __shared__ int s_flag[2];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TC_STAGES * STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* acc_full = empty + TC_STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* never = acc_empty + 1;   // nothing arrives here (wait_test)
  uint32_t* tmem_slot = (uint32_t*)(never + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) s_start = (*(volatile unsigned*)status & kStatusTimeout) ? 0 : 1;
  __syncthreads();
  if (!s_start) return;   // an earlier CTA gave up: skip the work, hold no tensor memory
  if (tid == 0) {
    for (int i = 0; i < TC_STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "n"(TC_PRODUCERS + 1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(acc_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(acc_empty)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(never)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);
  const int Kreal = 2 * a.Kd;                        // multiple of 16
  const int nchunk = (Kreal + TC_BK - 1) / TC_BK;
  const int64_t op_elems = (int64_t)2 * (2 * a.M) * (nchunk * TC_BK);

  if (warp < TC_PRODUCERS / 32) {
    // ---------------- producers ----------------
    int64_t g = 0;   // chunks issued by this CTA
    bool ok = true;
    // thread tid copies 16-byte piece (tid & 3) of the hi (tid & 4 == 0) or lo
    // half-line of rows (tid >> 3) + 16 q: 8 lanes cover one row's chunk, so a
    // warp's copy touches 4 rows x 2 segments of 64 bytes.  The source rows of
    // the next item (tile record, then pair indices) are loaded while this
    // item's chunks are issued, off the gather's critical path.
    const int piece = tid & 3, which = (tid >> 2) & 1;
    const __half* sarr = (which ? t.src_lo : t.src_hi) + 8 * piece;
    const int64_t G = gridDim.x;
    auto load_rows = [&](const int4& tl, int* srcrow) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int row = (tid >> 3) + 16 * q;
        srcrow[q] = -1;
        if (row < tl.z * a.nrhs) {
          if (a.nrhs == 1) srcrow[q] = a.pairs[tl.y + row].x;
          else srcrow[q] = a.pairs[tl.y + row / a.nrhs].x * a.nrhs + row % a.nrhs;
        }
      }
    };
    int4 tile_n = blockIdx.x < nitems ? a.tiles[blockIdx.x / nb] : make_int4(0, 0, 0, 0);
    int rows_n[8];
    load_rows(tile_n, rows_n);
    int4 tile_nn = blockIdx.x + G < nitems ? a.tiles[(blockIdx.x + G) / nb] : make_int4(0, 0, 0, 0);
    for (int64_t it = blockIdx.x; it < nitems && ok; it += G) {
      const int4 tile = tile_n;
      int rows[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) rows[q] = rows_n[q];
      tile_n = tile_nn;
      load_rows(tile_n, rows_n);
      tile_nn = it + 2 * G < nitems ? a.tiles[(it + 2 * G) / nb] : make_int4(0, 0, 0, 0);
      const int b = (int)(it % nb);
      const int n = min(TC_NMAX, 2 * a.M - TC_NMAX * b);
      const __half* img = t.img + tile.x * op_elems + (int64_t)b * nchunk * 2 * TC_NMAX * TC_BK;
      const __half* srow[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) srow[q] = rows[q] >= 0 ? sarr + (int64_t)rows[q] * Kreal : nullptr;
      for (int c = 0; c < nchunk; ++c, ++g) {
        const int st = (int)(g % TC_STAGES);
        const int64_t j = g / TC_STAGES;
        if (j > 0) {   // the stage's previous chunk has been consumed by the MMAs
          if (tid == 0) s_flag[g & 1] = mbar_wait(smem_u32(&empty[st]), (uint32_t)((j - 1) & 1), status) ? 1 : 0;
          named_bar_producers();
          ok = s_flag[g & 1] != 0;
          if (!ok) break;
        }
        const uint32_t sA = sbase + st * STAGE_BYTES;
        const int k0 = c * TC_BK;
        const bool kin = k0 + 8 * piece < Kreal;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t dh = sA + (uint32_t)which * A_BYTES + kmaj((tid >> 3) + 16 * q, 8 * piece);
          if (srow[q] && kin)
            cp_async16(dh, srow[q] + k0);
          else
            cp_async16_zero(dh, t.src_hi);
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[st])) : "memory");
        if (tid == 0) {   // operator tile: hi then lo, n x 32 values each
          const uint32_t bytes = (uint32_t)(2 * n * TC_BK * 2);
          mbar_expect_tx(smem_u32(&full[st]), bytes);
          bulk_g2s(sA + 2 * A_BYTES, img + (int64_t)c * 2 * n * TC_BK, bytes, smem_u32(&full[st]));
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (tid == 0)   // the bulk copies of the last fills have landed
      for (int64_t q = (g > TC_STAGES ? g - TC_STAGES : 0); q < g; ++q)
        mbar_wait_drain(smem_u32(&full[q % TC_STAGES]), (uint32_t)((q / TC_STAGES) & 1));
  } else if (warp == TC_MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int64_t g = 0, last = -1;
      int i = 0;
      // wait_test: a wait that can only end by giving up (phase 0 of `never`
      // never completes); the CTA then takes the timeout path below
      bool ok = !(a.wait_test && blockIdx.x == 0) || mbar_wait(smem_u32(never), 0u, status);
      for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++i) {
        const int b = (int)(it % nb);
        const int n = min(TC_NMAX, 2 * a.M - TC_NMAX * b);
        const uint32_t idesc = idesc_f16(n);
        if (i > 0 && !mbar_wait(smem_u32(acc_empty), (uint32_t)((i - 1) & 1), status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < nchunk; ++c, ++g) {
          const int st = (int)(g % TC_STAGES);
          if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((g / TC_STAGES) & 1), status)) {
            ok = false;
            break;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // cp.async data -> async proxy
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int ksteps = min(TC_BK, Kreal - c * TC_BK) / 16;
          const uint32_t ah = sbase + st * STAGE_BYTES, al = ah + A_BYTES, bh = al + A_BYTES;
          const uint32_t bl = bh + (uint32_t)(n * TC_BK * 2);    // lo tile follows the hi tile
          for (int s = 0; s < ksteps; ++s) {
            const uint32_t off = 256u * s;
            const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
            mma_f16(tmem, smem_desc(ah + off, CORE_SBO), smem_desc(bh + off, CORE_SBO), idesc, acc);
            mma_f16(tmem + 256u, smem_desc(ah + off, CORE_SBO), smem_desc(bl + off, CORE_SBO), idesc, acc);
            mma_f16(tmem + 256u, smem_desc(al + off, CORE_SBO), smem_desc(bh + off, CORE_SBO), idesc, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty[st]))
                       : "memory");
          last = g;
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(acc_full))
                     : "memory");
      }
      // MMAs complete in order: once the last commit has arrived, all have
      if (last >= 0) mbar_wait_drain(smem_u32(&empty[last % TC_STAGES]), (uint32_t)((last / TC_STAGES) & 1));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    // Warp 4 + q reads TMEM lanes 32q..32q+31 as two blocks of 16 lanes with the
    // .16x256b shape: four lanes of the warp hold 8 consecutive outputs of one
    // gathered column, so each 8-byte reduction of a warp covers 8 target rows x
    // 32 contiguous bytes.
    const int quarter = warp & 3;
    int i = 0;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x, ++i) {
      const int4 tile = a.tiles[it / nb];
      const int b = (int)(it % nb);
      const int n0 = TC_NMAX * b;
      const int n = min(TC_NMAX, 2 * a.M - n0);
      float* out[4];
      float cs[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {   // columns 32q + 16 (h/2) + lane/4 + 8 (h%2)
        const int col = 32 * quarter + 16 * (h >> 1) + (lane >> 2) + 8 * (h & 1);
        out[h] = nullptr;
        cs[h] = 0.f;
        if (col < tile.z * a.nrhs) {
          const int2 pr = a.pairs[tile.y + col / a.nrhs];
          const int k = col % a.nrhs;
          cs[h] = t.src_scale[(int64_t)pr.x * a.nrhs + k] * t.op_scale[tile.x];
          out[h] = (float*)(a.dst + ((int64_t)pr.y * a.nrhs + k) * a.dst_ld) + n0 + 2 * (lane & 3);
        }
      }
      int okw = 0;
      if (lane == 0) okw = mbar_wait(smem_u32(acc_full), (uint32_t)(i & 1), status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int blk = 0; blk < 2; ++blk) {
        const uint32_t tb = tmem + ((uint32_t)(32 * quarter + 16 * blk) << 16);
        float* oA = out[2 * blk];
        float* oB = out[2 * blk + 1];
        const float cA = cs[2 * blk], cB = cs[2 * blk + 1];
        for (int j0 = 0; j0 < n; j0 += 32) {
          uint32_t v[16], w[16];
          tmem_ld16x256_x4(tb + (uint32_t)j0, v);
          tmem_ld16x256_x4(tb + 256u + (uint32_t)j0, w);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int c = j0 + 8 * j;   // this thread's columns c + 2 (lane % 4) + {0, 1}
            if (c < n) {
              const float a0 = (__uint_as_float(v[4 * j]) + __uint_as_float(w[4 * j])) * cA;
              const float a1 = (__uint_as_float(v[4 * j + 1]) + __uint_as_float(w[4 * j + 1])) * cA;
              const float b0 = (__uint_as_float(v[4 * j + 2]) + __uint_as_float(w[4 * j + 2])) * cB;
              const float b1 = (__uint_as_float(v[4 * j + 3]) + __uint_as_float(w[4 * j + 3])) * cB;
              if (a.store) {
                if (oA) *(float2*)(oA + c) = make_float2(a0, a1);
                if (oB) *(float2*)(oB + c) = make_float2(b0, b1);
              } else {
                if (oA) red_add2(oA + c, a0, a1);
                if (oB) red_add2(oB + c, b0, b1);
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acc_empty)) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == TC_MMA_WARP) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

void compute_op_scales(const float2* ops, int64_t per_op, int nops, float* scale, cudaStream_t s) {
  if (nops == 0) return;
  op_scale_kernel<<<nops, 256, 0, s>>>(ops, per_op, scale);
  DFMM_CUDA(cudaGetLastError());
}

int gemm_tc_columns() { return TC_M; }

bool gemm_tc_supported(int M, int Kd) { return M % 8 == 0 && Kd % 8 == 0; }

int64_t tc_image_elems(int M, int Kd, int nops) {
  const int nchunk = (2 * Kd + TC_BK - 1) / TC_BK;
  return (int64_t)nops * 2 * (2 * M) * (nchunk * TC_BK);
}

void build_tc_image(const float2* ops, int M, int Kd, int nops, __half* img, float* scale, cudaStream_t s) {
  if (nops == 0) return;
  if (!gemm_tc_supported(M, Kd)) throw Error(-5, "tensor-core stage needs ranks padded to a multiple of 8");
  op_scale_kernel<<<nops, 256, 0, s>>>(ops, (int64_t)M * Kd, scale);
  const int nchunk = (2 * Kd + TC_BK - 1) / TC_BK;
  const int nb = (2 * M + TC_NMAX - 1) / TC_NMAX;
  int64_t blocks = (int64_t)nops * nb * nchunk;
  op_image_kernel<<<(unsigned)blocks, 256, 0, s>>>(ops, scale, M, Kd, nops, img);
  DFMM_CUDA(cudaGetLastError());
}

void launch_split(const float2* x, int64_t rows, int ld, __half* hi, __half* lo, float* scale, cudaStream_t s) {
  if (rows == 0) return;
  const int64_t threads = rows * 32;
  split_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>((const float*)x, rows, 2 * ld, hi, lo, scale);
  DFMM_CUDA(cudaGetLastError());
}

void launch_gemm_stage_tc(const GemmArgs& a, const TcArgs& t, unsigned* status, cudaStream_t s) {
  if (a.ntiles == 0) return;
  if (!gemm_tc_supported(a.M, a.Kd) || a.src_ld != a.Kd)
    throw Error(-5, "tensor-core stage needs ranks padded to a multiple of 8 and dense source rows");
  static int nsm[64] = {0};
  int dev = 0;
  DFMM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(-1, "device ordinal out of range");
  if (!nsm[dev]) {
    DFMM_CUDA(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    DFMM_CUDA(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
  }
  const int nb = (2 * a.M + TC_NMAX - 1) / TC_NMAX;
  const int64_t nitems = a.ntiles * nb;
  const unsigned grid = (unsigned)std::min<int64_t>(nitems, nsm[dev]);
  gemm_tc_kernel<<<grid, TC_THREADS, SMEM_BYTES, s>>>(a, t, nitems, nb, status);
  DFMM_CUDA(cudaGetLastError());
}

}  // namespace dfmm
