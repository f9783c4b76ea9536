// Split-complex tensor-core form of the translation stage y[dst] += T_op x[src]
// (M2L and the other translations of the same gather / GEMM / scatter-add
// shape), for target ranks up to 128.
//
// A complex product y = T x is four real products,
//     Re y = Tr xr - Ti xi,     Im y = Ti xr + Tr xi,
// each a GEMM with N = r_t (the target rank) and K = r_s.  The operator is
// stored as its real and imaginary parts once each, half the bytes of the
// real-block form [[Tr, -Ti], [Ti, Tr]] that m2l_tc.cu streams per tile, and
// the source rows are split into their real and imaginary halves.  The minus
// sign is the MMA's negate-A flag.
//
//  * One CTA computes a tile of 128 gathered columns (pairs x right-hand
//    sides) against one operator, with tcgen05.mma kind::f16, M = 128,
//    N = r_t <= 128, K = 16, FP32 accumulation in tensor memory.
//  * Scaled split as in m2l_tc.cu: x / s = hi + lo per source row and
//    T / t = hi + lo per operator, in one of three element types (KIND):
//    FP16 (kind::f16, the default), BF16 (kind::f16 with BF16 operands:
//    "3xBF16", about 16 bits) or TF32 (kind::tf32: "3xTF32", about 22 bits,
//    half the FP16 rate).  Every tile is 64 bytes per row and K step 32
//    bytes whatever the type, so one layout serves all three.  12 MMAs per K
//    step.  The hi hi products go to the accumulators Re Y, Im Y, and the
//    cross terms hi lo + lo hi either to a second pair re y, im y, added in
//    FP32 by the epilogue (ONE = false: tensor-core accumulation truncates, so
//    the small terms keep their own accumulators; 4 r_t <= 512 tensor-memory
//    columns, one tile at a time), or into Re Y, Im Y as well (ONE = true, the
//    automatic choice at eps >= 1e-5: 2 r_t columns per buffer and two
//    buffers, so that a tile's MMAs overlap the previous tile's epilogue).
//  * Stage = one K chunk of 32: the gathered xr hi, xr lo, xi hi, xi lo tiles
//    (128 rows x 64 bytes each, 16-byte cp.async) and the operator's Tr hi,
//    Tr lo, Ti hi, Ti lo tiles (one bulk copy of its plan-time image); 3
//    stages of up to 64 KB.
//  * Epilogue: the .16x256b tensor-memory shape gives a thread two
//    consecutive outputs p, p + 1 of a column in each accumulator, i.e. the
//    interleaved target components 2p .. 2p + 3: one 16-byte reduction
//    (red.global.add.v4.f32), and one warp instruction covers 8 target rows x
//    64 contiguous bytes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "apply.h"
#include "tcgen05.cuh"

namespace dfmm {

namespace {

using namespace tc;

constexpr int CX_M = 128;                          // gathered columns per tile
constexpr int CX_SEG = 64;                         // bytes per row of a tile: one K chunk of one half
constexpr int CX_NMAX = 128;                       // target rank
constexpr int CX_PRODUCERS = 128;                  // warps 0-3: gather
constexpr int CX_MMA_WARP = 8;                     // warps 4-7: epilogue; warp 8: MMA issuer
constexpr int CX_THREADS = 288;
constexpr int CX_STAGES = 3;
constexpr int CX_A_TILE = CX_M * CX_SEG;          // 8 KB: one of xr hi, xr lo, xi hi, xi lo
constexpr int CX_B_MAX = 4 * CX_NMAX * CX_SEG;     // 32 KB: Tr hi, Tr lo, Ti hi, Ti lo
constexpr int CX_STAGE = 4 * CX_A_TILE + CX_B_MAX;
constexpr int CX_SMEM = CX_STAGES * CX_STAGE + 1024 + 256;
constexpr int CX_TMEM_COLS = 512;
constexpr uint32_t CX_SBO = (CX_SEG / 16) * 128;   // 512 B between 8-row groups

// byte offset of byte b (even) of row `row` of a tile in the stage layout
__host__ __device__ __forceinline__ uint32_t ckmaj(int row, int b) { return tc::kmaj_off(row, b / 2, CX_SBO); }

// element types: 0 = FP16, 1 = BF16, 2 = TF32 (stored as FP32 bit patterns)
template <int KIND> struct Elem;
template <> struct Elem<0> {
  using T = __half;
  static __device__ __forceinline__ void split(float v, T& h, T& l) {
    h = __float2half_rn(v);
    l = __float2half_rn(v - __half2float(h));
  }
};
template <> struct Elem<1> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ void split(float v, T& h, T& l) {
    h = __float2bfloat16_rn(v);
    l = __float2bfloat16_rn(v - __bfloat162float(h));
  }
};
__device__ __forceinline__ uint32_t to_tf32(float v) {   // round to the nearest TF32 (ties away)
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
template <> struct Elem<2> {
  using T = uint32_t;
  static __device__ __forceinline__ void split(float v, T& h, T& l) {
    h = to_tf32(v);
    l = to_tf32(v - __uint_as_float(h));
  }
};
template <int KIND> __host__ __device__ constexpr int elem_bytes() { return KIND == 2 ? 4 : 2; }
template <int KIND> __host__ __device__ constexpr int seg_elems() { return CX_SEG / elem_bytes<KIND>(); }   // K values per chunk
template <int KIND> __host__ __device__ constexpr int kstep_elems() { return 32 / elem_bytes<KIND>(); }    // K values per MMA

// instruction descriptor: D f32, both operands K-major, M = 128, N = n; A and
// B FP16 / BF16 (kind::f16) or TF32 (kind::tf32); neg_a negates A
template <int KIND>
__device__ __forceinline__ uint32_t idesc_cx(int n, bool neg_a) {
  const uint32_t ty = KIND == 0 ? 0u : (KIND == 1 ? 1u : 2u);
  return (1u << 4) | (ty << 7) | (ty << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma_cx(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND == 2)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  else
    mma_f16(d_tmem, a, b, idesc, acc);
}

// Source rows (interleaved complex, len = 2 r floats) -> scaled FP16 hi / lo
// rows with the real parts first and the imaginary parts second; one warp per
// row, one power-of-two scale per row.
template <int KIND>
__global__ void split_cx_kernel(const float* __restrict__ x, int64_t rows, int r, typename Elem<KIND>::T* __restrict__ hi,
                                typename Elem<KIND>::T* __restrict__ lo, float* __restrict__ scale) {
  using E = Elem<KIND>;
  using T = typename E::T;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const int len = 2 * r;
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
  T* h = hi + row * len;
  T* l = lo + row * len;
  for (int k = lane * 4; k < len; k += 128) {   // complex elements k/2 and k/2 + 1
    const float4 v = *(const float4*)(xr + k);
    T hr0, hi0, hr1, hi1, lr0, li0, lr1, li1;
    E::split(v.x * inv, hr0, lr0);
    E::split(v.y * inv, hi0, li0);
    E::split(v.z * inv, hr1, lr1);
    E::split(v.w * inv, hi1, li1);
    const int q = k >> 1;
    h[q] = hr0;
    h[q + 1] = hr1;
    h[r + q] = hi0;
    h[r + q + 1] = hi1;
    l[q] = lr0;
    l[q + 1] = lr1;
    l[r + q] = li0;
    l[r + q + 1] = li1;
  }
}

// Operator image: for every (operator, K chunk c) the four tiles Tr hi, Tr lo,
// Ti hi, Ti lo of M rows x 32 fp16 values (row p, column q = 32 c + kk holds
// T[p][q] / scale[op]), in the stage layout; zero beyond Kd.
template <int KIND>
__global__ void op_image_cx_kernel(const float2* __restrict__ ops, const float* __restrict__ scale, int M, int Kd,
                                   int nops, unsigned char* __restrict__ img) {
  using E = Elem<KIND>;
  using T = typename E::T;
  constexpr int BKE = seg_elems<KIND>(), EB = elem_bytes<KIND>();
  const int nchunk = (Kd + BKE - 1) / BKE;
  const int64_t g = blockIdx.x;   // (op, c)
  const int c = (int)(g % nchunk);
  const int op = (int)(g / nchunk);
  if (op >= nops) return;
  unsigned char* base = img + g * (int64_t)(4 * M * CX_SEG);
  const float2* Top = ops + (size_t)op * M * Kd;
  const float inv = 1.f / scale[op];
  for (int e = threadIdx.x; e < M * BKE; e += blockDim.x) {
    const int p = e / BKE, kk = e % BKE;
    const int q = c * BKE + kk;
    float2 t = make_float2(0.f, 0.f);
    if (q < Kd) t = Top[(size_t)p * Kd + q];
    T rh, rl, ih, il;
    E::split(t.x * inv, rh, rl);
    E::split(t.y * inv, ih, il);
    const uint32_t off = ckmaj(p, kk * EB);
    *(T*)(base + off) = rh;
    *(T*)(base + M * CX_SEG + off) = rl;
    *(T*)(base + 2 * M * CX_SEG + off) = ih;
    *(T*)(base + 3 * M * CX_SEG + off) = il;
  }
}

// The stage of a tile: from the launch's stage table (tile .w), or the single
// stage of GemmArgs / TcArgs.
__device__ __forceinline__ CxStage stage_of(const GemmArgs& a, const TcArgs& t, int w) {
  if (a.stages) return a.stages[w];
  CxStage s;
  s.pairs = a.pairs;
  s.src_hi = t.src_hi;
  s.src_lo = t.src_lo;
  s.src_scale = t.src_scale;
  s.img = t.img;
  s.op_scale = t.op_scale;
  s.dst = a.dst;
  s.nrhs = a.nrhs;
  s.store = a.store;
  return s;
}

__device__ __forceinline__ void named_bar_cx() { asm volatile("bar.sync 1, %0;" ::"n"(CX_PRODUCERS) : "memory"); }

// Persistent, warp-specialised stage kernel; CTA x takes tiles x, x + gridDim.x, ...
//   warps 0-3  producers: thread t copies 16-byte piece t % 4 of segment
//              (t / 4) % 4 (xr hi, xr lo, xi hi, xi lo) of rows t / 16 + 8 q
//              (cp.async, counted on the stage's full barrier); thread 0 also
//              bulk-copies the operator chunk; up to CX_STAGES chunks ahead.
//   warp 8     one thread issues the 12 MMAs per K step, commits each chunk to
//              its stage's empty barrier and each tile to acc_full; it waits
//              for acc_empty before it overwrites the accumulators.
//   warps 4-7  epilogue: warp 4 + q reads tensor-memory lanes 32 q .. 32 q + 31
//              (gathered columns), adds the two accumulator pairs, scales, and
//              scatter-adds 16 bytes per thread and step; then acc_empty.
// Every wait is time-limited; on a timeout the CTA reports it, stops issuing,
// lets its own copies and MMAs land, frees its tensor memory and returns.
//
// ONE = false: two accumulator pairs (hi hi terms apart from the cross terms),
// 4 r_t columns, one tile at a time.  ONE = true: one accumulator per
// component (2 r_t columns) and two tensor-memory buffers, so that the MMAs
// of a tile overlap the epilogue of the previous one; the cross terms then
// accumulate with the truncation of the large terms.
template <int KIND, bool ONE>
__global__ __launch_bounds__(CX_THREADS, 1) void gemm_cx_kernel(GemmArgs a, TcArgs t, unsigned* status) {
  constexpr int EB = elem_bytes<KIND>(), BKE = seg_elems<KIND>(), KSTEP = kstep_elems<KIND>();
  extern __shared__ unsigned char smem_raw[];
  __shared__ int s_start;
  __shared__ int s_flag[2];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + CX_STAGES * CX_STAGE);
  uint64_t* empty = full + CX_STAGES;
  uint64_t* acc_full = empty + CX_STAGES;    // [2]: one per tensor-memory buffer
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* never = acc_empty + 2;   // nothing arrives here (wait_test)
  uint32_t* tmem_slot = (uint32_t*)(never + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.M;     // target rank: the MMA's N
  const int Kh = a.Kd;   // source rank: K of each half
  const int nchunk = (Kh + BKE - 1) / BKE;
  const int64_t nitems = a.ntiles;
  const uint32_t b_bytes = (uint32_t)(4 * N * CX_SEG);
  const int64_t op_bytes = (int64_t)nchunk * 4 * N * CX_SEG;

  if (tid == 0) s_start = (*(volatile unsigned*)status & kStatusTimeout) ? 0 : 1;
  __syncthreads();
  if (!s_start) return;   // an earlier CTA gave up: skip the work, hold no tensor memory
  if (tid == 0) {
    for (int i = 0; i < CX_STAGES; ++i) {
      mbar_init(smem_u32(&full[i]), CX_PRODUCERS + 1);
      mbar_init(smem_u32(&empty[i]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 4);
    }
    mbar_init(smem_u32(never), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == CX_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(CX_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp < CX_PRODUCERS / 32) {
    // ---------------- producers ----------------
    const int piece = tid & 3, seg = (tid >> 2) & 3, rg = tid >> 4;
    int64_t g = 0;   // chunks issued by this CTA
    bool ok = true;
    // The source row of each gathered column: (pair, right-hand side) -> source
    // state row.  The tile records and pair indices of the next tile are loaded
    // while this tile's chunks are issued, so their latency stays off the
    // gather's critical path.
    const int G = gridDim.x;
    // per tile: this thread's source segment base and its 16 source rows
    auto load_rows = [&](const int4& tl, int* srcrow, const unsigned char*& sbase_arr, const unsigned char*& img_tile) {
      const CxStage sg = stage_of(a, t, tl.w);
      sbase_arr = (const unsigned char*)((seg & 1) ? sg.src_lo : sg.src_hi) + ((seg & 2) ? Kh * EB : 0) + 16 * piece;
      img_tile = (const unsigned char*)sg.img + tl.x * op_bytes;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int row = rg + 8 * q;
        srcrow[q] = -1;
        if (row < tl.z * sg.nrhs) {
          if (sg.nrhs == 1) srcrow[q] = sg.pairs[tl.y + row].x;
          else srcrow[q] = sg.pairs[tl.y + row / sg.nrhs].x * sg.nrhs + row % sg.nrhs;
        }
      }
    };
    int4 tile_n = blockIdx.x < nitems ? a.tiles[blockIdx.x] : make_int4(0, 0, 0, 0);
    int rows_n[16];
    const unsigned char *sarr_n = nullptr, *img_n = nullptr;
    if (blockIdx.x < nitems) load_rows(tile_n, rows_n, sarr_n, img_n);
    int4 tile_nn = blockIdx.x + G < nitems ? a.tiles[blockIdx.x + G] : make_int4(0, 0, 0, 0);
    for (int64_t it = blockIdx.x; it < nitems && ok; it += G) {
      int rows[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) rows[q] = rows_n[q];
      const unsigned char* sarr = sarr_n;
      const unsigned char* img = img_n;
      // prefetch: rows of the next tile, record of the one after
      tile_n = tile_nn;
      if (it + G < nitems) load_rows(tile_n, rows_n, sarr_n, img_n);
      tile_nn = it + 2 * (int64_t)G < nitems ? a.tiles[it + 2 * G] : make_int4(0, 0, 0, 0);
      const unsigned char* srow[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) srow[q] = rows[q] >= 0 ? sarr + (int64_t)rows[q] * (2 * Kh * EB) : nullptr;
      for (int c = 0; c < nchunk; ++c, ++g) {
        const int st = (int)(g % CX_STAGES);
        const int64_t j = g / CX_STAGES;
        if (j > 0) {   // the stage's previous chunk has been consumed by the MMAs
          if (tid == 0) s_flag[g & 1] = mbar_wait(smem_u32(&empty[st]), (uint32_t)((j - 1) & 1), status) ? 1 : 0;
          named_bar_cx();
          ok = s_flag[g & 1] != 0;
          if (!ok) break;
        }
        const uint32_t sA = sbase + st * CX_STAGE + seg * CX_A_TILE;
        const int b0 = c * CX_SEG;   // byte offset of the chunk within a row half
        const bool kin = b0 + 16 * piece < Kh * EB;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const uint32_t dst = sA + ckmaj(rg + 8 * q, 16 * piece);
          if (srow[q] && kin)
            cp_async16(dst, srow[q] + b0);
          else
            cp_async16_zero(dst, sarr);
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[st])) : "memory");
        if (tid == 0) {   // operator chunk: Tr hi, Tr lo, Ti hi, Ti lo
          mbar_expect_tx(smem_u32(&full[st]), b_bytes);
          bulk_g2s(sbase + st * CX_STAGE + 4 * CX_A_TILE, img + (int64_t)c * 4 * N * CX_SEG, b_bytes,
                   smem_u32(&full[st]));
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (tid == 0)   // the bulk copies of the last fills have landed
      for (int64_t q = (g > CX_STAGES ? g - CX_STAGES : 0); q < g; ++q)
        mbar_wait_drain(smem_u32(&full[q % CX_STAGES]), (uint32_t)((q / CX_STAGES) & 1));
  } else if (warp == CX_MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int64_t g = 0, last = -1;
      int i = 0;
      // wait_test: a wait that can only end by giving up; the CTA then takes the timeout path
      bool ok = !(a.wait_test && blockIdx.x == 0) || mbar_wait(smem_u32(never), 0u, status);
      const uint32_t ip = idesc_cx<KIND>(N, false), in = idesc_cx<KIND>(N, true);
      for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++i) {
        // buffer of this tile: ONE alternates two buffers of 2 r_t columns
        const int b = ONE ? (i & 1) : 0;
        const int use = ONE ? (i >> 1) : i;   // earlier tiles on this buffer
        const uint32_t base = tmem + (uint32_t)(b * 256);
        const uint32_t YR = base, YI = base + (uint32_t)N;
        const uint32_t yr = ONE ? YR : base + 2u * N, yi = ONE ? YI : base + 3u * N;
        if (use > 0 && !mbar_wait(smem_u32(&acc_empty[b]), (uint32_t)((use - 1) & 1), status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < nchunk; ++c, ++g) {
          const int st = (int)(g % CX_STAGES);
          if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((g / CX_STAGES) & 1), status)) {
            ok = false;
            break;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // cp.async data -> async proxy
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int ksteps = min(BKE, Kh - c * BKE) / KSTEP;
          const uint32_t xrh = sbase + st * CX_STAGE, xrl = xrh + CX_A_TILE, xih = xrl + CX_A_TILE,
                         xil = xih + CX_A_TILE;
          const uint32_t trh = xil + CX_A_TILE, trl = trh + (uint32_t)(N * CX_SEG), tih = trl + (uint32_t)(N * CX_SEG),
                         til = tih + (uint32_t)(N * CX_SEG);
          for (int s = 0; s < ksteps; ++s) {
            const uint32_t off = 256u * s;
            const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
            const uint64_t dxrh = smem_desc(xrh + off, CX_SBO), dxrl = smem_desc(xrl + off, CX_SBO),
                           dxih = smem_desc(xih + off, CX_SBO), dxil = smem_desc(xil + off, CX_SBO);
            const uint64_t dtrh = smem_desc(trh + off, CX_SBO), dtrl = smem_desc(trl + off, CX_SBO),
                           dtih = smem_desc(tih + off, CX_SBO), dtil = smem_desc(til + off, CX_SBO);
            // Re y = Tr xr - Ti xi, Im y = Ti xr + Tr xi; hi hi terms into Y, the rest into y
            mma_cx<KIND>(YR, dxrh, dtrh, ip, acc);
            mma_cx<KIND>(YR, dxih, dtih, in, 1u);
            mma_cx<KIND>(YI, dxrh, dtih, ip, acc);
            mma_cx<KIND>(YI, dxih, dtrh, ip, 1u);
            mma_cx<KIND>(yr, dxrh, dtrl, ip, ONE ? 1u : acc);
            mma_cx<KIND>(yr, dxrl, dtrh, ip, 1u);
            mma_cx<KIND>(yr, dxih, dtil, in, 1u);
            mma_cx<KIND>(yr, dxil, dtih, in, 1u);
            mma_cx<KIND>(yi, dxrh, dtil, ip, ONE ? 1u : acc);
            mma_cx<KIND>(yi, dxrl, dtih, ip, 1u);
            mma_cx<KIND>(yi, dxih, dtrl, ip, 1u);
            mma_cx<KIND>(yi, dxil, dtrh, ip, 1u);
          }
          mma_commit(smem_u32(&empty[st]));
          last = g;
        }
        if (!ok) break;
        mma_commit(smem_u32(&acc_full[b]));
      }
      // MMAs complete in order: once the last commit has arrived, all have
      if (last >= 0) mbar_wait_drain(smem_u32(&empty[last % CX_STAGES]), (uint32_t)((last / CX_STAGES) & 1));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int quarter = warp & 3;
    int i = 0;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x, ++i) {
      const int4 tile = a.tiles[it];
      const CxStage sg = stage_of(a, t, tile.w);
      float* out[4];
      float cs[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {   // columns 32q + 16 (h/2) + lane/4 + 8 (h%2)
        const int col = 32 * quarter + 16 * (h >> 1) + (lane >> 2) + 8 * (h & 1);
        out[h] = nullptr;
        cs[h] = 0.f;
        if (col < tile.z * sg.nrhs) {
          const int2 pr = sg.pairs[tile.y + col / sg.nrhs];
          const int k = col % sg.nrhs;
          cs[h] = sg.src_scale[(int64_t)pr.x * sg.nrhs + k] * sg.op_scale[tile.x];
          out[h] = (float*)(sg.dst + ((int64_t)pr.y * sg.nrhs + k) * a.dst_ld) + 4 * (lane & 3);
        }
      }
      const int b = ONE ? (i & 1) : 0;
      const int use = ONE ? (i >> 1) : i;
      int okw = 0;
      if (lane == 0) okw = mbar_wait(smem_u32(&acc_full[b]), (uint32_t)(use & 1), status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int blk = 0; blk < 2; ++blk) {
        const uint32_t tb = tmem + (uint32_t)(b * 256) + ((uint32_t)(32 * quarter + 16 * blk) << 16);
        float* oA = out[2 * blk];
        float* oB = out[2 * blk + 1];
        const float cA = cs[2 * blk], cB = cs[2 * blk + 1];
        for (int j0 = 0; j0 < N; j0 += 32) {
          uint32_t vr[16], vi[16], wr[16], wi[16];
          tmem_ld16x256_x4(tb + (uint32_t)j0, vr);
          tmem_ld16x256_x4(tb + (uint32_t)(N + j0), vi);
          if (!ONE) {
            tmem_ld16x256_x4(tb + (uint32_t)(2 * N + j0), wr);
            tmem_ld16x256_x4(tb + (uint32_t)(3 * N + j0), wi);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) wr[q] = wi[q] = 0u;
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // this thread's outputs p = j0 + 8 j + 2 (lane % 4) + {0, 1}: target floats 2p .. 2p + 3
            if (j0 + 8 * j < N) {
              const int f = 2 * j0 + 16 * j;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                float* o = h ? oB : oA;
                const float cc = h ? cB : cA;
                const int r = 4 * j + 2 * h;
                const float re0 = (__uint_as_float(vr[r]) + __uint_as_float(wr[r])) * cc;
                const float im0 = (__uint_as_float(vi[r]) + __uint_as_float(wi[r])) * cc;
                const float re1 = (__uint_as_float(vr[r + 1]) + __uint_as_float(wr[r + 1])) * cc;
                const float im1 = (__uint_as_float(vi[r + 1]) + __uint_as_float(wi[r + 1])) * cc;
                if (o) {
                  if (sg.store) *(float4*)(o + f) = make_float4(re0, im0, re1, im1);
                  else red_add4(o + f, re0, im0, re1, im1);
                }
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == CX_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CX_TMEM_COLS));
}

}  // namespace

int gemm_cx_columns() { return CX_M; }

bool gemm_cx_supported(int M, int Kd) { return M % 16 == 0 && Kd % 16 == 0 && M >= 16 && M <= CX_NMAX; }

int cx_elem_bytes(int kind) { return kind == 2 ? 4 : 2; }

int64_t cx_image_bytes(int M, int Kd, int nops, int kind) {
  const int bke = CX_SEG / cx_elem_bytes(kind);
  const int nchunk = (Kd + bke - 1) / bke;
  return (int64_t)nops * nchunk * 4 * M * CX_SEG;
}

void build_cx_image(const float2* ops, int M, int Kd, int nops, void* img, float* scale, int kind, cudaStream_t s) {
  if (nops == 0) return;
  if (!gemm_cx_supported(M, Kd)) throw Error(-5, "split-complex stage needs ranks that are multiples of 16, <= 128");
  compute_op_scales(ops, (int64_t)M * Kd, nops, scale, s);
  const int bke = CX_SEG / cx_elem_bytes(kind);
  const unsigned blocks = (unsigned)((int64_t)nops * ((Kd + bke - 1) / bke));
  unsigned char* p = (unsigned char*)img;
  if (kind == 0) op_image_cx_kernel<0><<<blocks, 256, 0, s>>>(ops, scale, M, Kd, nops, p);
  else if (kind == 1) op_image_cx_kernel<1><<<blocks, 256, 0, s>>>(ops, scale, M, Kd, nops, p);
  else op_image_cx_kernel<2><<<blocks, 256, 0, s>>>(ops, scale, M, Kd, nops, p);
  DFMM_CUDA(cudaGetLastError());
}

void launch_split_cx(const float2* x, int64_t rows, int r, void* hi, void* lo, float* scale, int kind, cudaStream_t s) {
  if (rows == 0) return;
  if (r % 16) throw Error(-5, "split-complex source rows need a rank that is a multiple of 16");
  const unsigned grid = (unsigned)((rows * 32 + 255) / 256);
  const float* xf = (const float*)x;
  if (kind == 0)
    split_cx_kernel<0><<<grid, 256, 0, s>>>(xf, rows, r, (__half*)hi, (__half*)lo, scale);
  else if (kind == 1)
    split_cx_kernel<1><<<grid, 256, 0, s>>>(xf, rows, r, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, scale);
  else
    split_cx_kernel<2><<<grid, 256, 0, s>>>(xf, rows, r, (uint32_t*)hi, (uint32_t*)lo, scale);
  DFMM_CUDA(cudaGetLastError());
}

template <int KIND, bool ONE>
void launch_cx(const GemmArgs& a, const TcArgs& t, unsigned* status, unsigned grid, cudaStream_t s) {
  static bool attr[64] = {false};
  int dev = 0;
  DFMM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(-1, "device ordinal out of range");
  if (!attr[dev]) {
    DFMM_CUDA(cudaFuncSetAttribute(gemm_cx_kernel<KIND, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, CX_SMEM));
    attr[dev] = true;
  }
  gemm_cx_kernel<KIND, ONE><<<grid, CX_THREADS, CX_SMEM, s>>>(a, t, status);
}

void launch_gemm_stage_cx(const GemmArgs& a, const TcArgs& t, unsigned* status, bool one_acc, int kind,
                          cudaStream_t s) {
  if (a.ntiles == 0) return;
  if (!gemm_cx_supported(a.M, a.Kd) || a.src_ld != a.Kd)
    throw Error(-5, "split-complex stage needs ranks that are multiples of 16, <= 128, and dense source rows");
  static int nsm[64] = {0};
  int dev = 0;
  DFMM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(-1, "device ordinal out of range");
  if (!nsm[dev]) DFMM_CUDA(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)std::min<int64_t>(a.ntiles, nsm[dev]);
  if (kind == 0) {
    if (one_acc) launch_cx<0, true>(a, t, status, grid, s);
    else launch_cx<0, false>(a, t, status, grid, s);
  } else if (kind == 1) {
    if (one_acc) launch_cx<1, true>(a, t, status, grid, s);
    else launch_cx<1, false>(a, t, status, grid, s);
  } else {
    if (one_acc) launch_cx<2, true>(a, t, status, grid, s);
    else launch_cx<2, false>(a, t, status, grid, s);
  }
  DFMM_CUDA(cudaGetLastError());
}

}  // namespace dfmm
