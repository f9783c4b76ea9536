// Apply-time kernels of the directional FMM matvec (FP32).
//
//  * gemm_stage_kernel: every translation of Alg. 1 (P2L projection,
//    LF/HF-M2M, HF-M2L, LF-M2L, HF/LF-L2L) is "y[dst] += T_op x[src]" over a
//    list of (src, dst) pairs grouped by operator.  One CTA computes a
//    64-row x 64-column block of T_op X, where the columns are the gathered
//    source states (pairs x right-hand sides), and scatter-adds the result
//    into the target states with vector atomics (targets of one operator are
//    distinct, different operators meet in L2).  This is the plain CUDA-core
//    form; the tensor-core forms are in m2l_cx.cu and m2l_tc.cu.
//  * p2c_kernel: potentials at check points from points (P2L, X lists), with
//    the phase 2 pi |x - y| reduced in a compensated form so that far check
//    points keep full FP32 accuracy.
//  * p2m_rows_kernel: P2M as a sum of FP64-formed per-point rows.
//  * l2p_kernel: L2P through precomputed per-point rows (flat row stream).
//  * rows_kernel: M2P (W lists) through precomputed rows.
//  * p2p_fast_kernel: the near field (U lists) on FP32 coordinates, with the
//    exact plan-time corrections of the close pairs (p2p_close_kernel,
//    p2p_close_apply_kernel); p2p_kernel: the same on double-float coordinates.
#include "apply.h"

#include <type_traits>

namespace dfmm {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// fire-and-forget vector adds to global memory (no value returned)
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}
__device__ __forceinline__ void red_add2(float* p, float a, float b) {
  asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

__global__ __launch_bounds__(256) void gemm_stage_kernel(GemmArgs a) {
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  __shared__ const float2* srcp[BN];
  __shared__ float2* dstp[BN];
  const int tid = threadIdx.x;
  const int4 tile = a.tiles[blockIdx.x];
  const float2* A = a.ops + (size_t)tile.x * a.M * a.Kd;
  const int row0 = blockIdx.y * BM;
  const int ncol = tile.z * a.nrhs;
  if (tid < BN) {
    const float2* sp = nullptr;
    float2* dp = nullptr;
    if (tid < ncol) {
      int p = tile.y + tid / a.nrhs, k = tid % a.nrhs;
      int2 pr = a.pairs[p];
      sp = a.src + ((int64_t)pr.x * a.nrhs + k) * a.src_ld;
      dp = a.dst + ((int64_t)pr.y * a.nrhs + k) * a.dst_ld;
    }
    srcp[tid] = sp;
    dstp[tid] = dp;
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < a.Kd; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int i = e / BK, kk = e % BK;
      int r = row0 + i, kc = k0 + kk;
      As[kk][i] = (r < a.M && kc < a.Kd) ? A[(size_t)r * a.Kd + kc] : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int c = e / BK, kk = e % BK;
      int kc = k0 + kk;
      Bs[kk][c] = (c < ncol && kc < a.Kd) ? srcp[c][kc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(av[i].x, bv[j].x, fmaf(-av[i].y, bv[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(av[i].x, bv[j].y, fmaf(av[i].y, bv[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int c = tx * 4 + j;
    if (c >= ncol) continue;
    float2* d = dstp[c] + row0 + ty * 4;
    int r = row0 + ty * 4;
    if (r + 3 < a.M) {
      red_add4((float*)d, acc[0][j].x, acc[0][j].y, acc[1][j].x, acc[1][j].y);
      red_add4((float*)(d + 2), acc[2][j].x, acc[2][j].y, acc[3][j].x, acc[3][j].y);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r + i < a.M) red_add2((float*)(d + i), acc[i][j].x, acc[i][j].y);
    }
  }
}

__global__ void permute_in_kernel(const float2* __restrict__ f, const int32_t* __restrict__ perm, int64_t N,
                                  int nrhs, float2* __restrict__ fs) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nrhs) return;
  int64_t k = e / nrhs;
  int r = (int)(e % nrhs);
  fs[e] = f[(int64_t)r * N + perm[k]];
}

__global__ void permute_out_kernel(const float2* __restrict__ us, const int32_t* __restrict__ perm, int64_t N,
                                   int nrhs, float2* __restrict__ u) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nrhs) return;
  int64_t k = e / nrhs;
  int r = (int)(e % nrhs);
  u[(int64_t)r * N + perm[k]] = us[e];
}

// x rounded to the nearest integer (ties to even) for |x| < 2^22: adding
// 1.5 * 2^23 moves x into the binade where the FP32 spacing is 1.  Two adds
// on the FMA pipe, where rintf would take a slot of the special-function unit
// that the sine, cosine and reciprocal square root already saturate.
__device__ __forceinline__ float round_near(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

// exp(2 pi i phase) / d with phase reduced to [-1/2, 1/2]
__device__ __forceinline__ float2 green_phase(float phase, float inv_d) {
  float ph = phase - round_near(phase);
  float s, c;
  __sincosf(6.28318530717958647f * ph, &s, &c);
  return make_float2(c * inv_d, s * inv_d);
}

constexpr int P2C_THREADS = 256;
constexpr int P2C_CHUNK = 128;
constexpr int P2C_JOBS = 8;   // rounds of side-by-side jobs per block

// Check-point potentials of leaf points (the sample of Eq. 6 that P2L
// projects).  A group of tpj threads (one per check point) takes one job; a
// block runs P2C_THREADS / tpj groups side by side, P2C_JOBS rounds in a row,
// and keeps its check points in registers across the rounds.  NR right-hand
// sides are accumulated per pass.
template <int NR>
__global__ __launch_bounds__(P2C_THREADS) void p2c_kernel(P2CArgs a, int tpj) {
  __shared__ float4 sp[P2C_CHUNK];
  __shared__ float2 sf[P2C_CHUNK][NR];
  const int jp = blockDim.x / tpj;
  const int slice = P2C_CHUNK / jp;
  const int grp = threadIdx.x / tpj, lane = threadIdx.x % tpj;
  const int64_t jb0 = (int64_t)blockIdx.x * jp * P2C_JOBS;
  const int64_t jb1 = min(a.njobs, jb0 + (int64_t)jp * P2C_JOBS);
  for (int p0 = 0; p0 < a.nchk; p0 += tpj) {
    const int p = p0 + lane;
    ChkPt c = {};
    if (p < a.nchk) c = a.chk[p];
    for (int64_t jb = jb0; jb < jb1; jb += jp) {
      const int64_t my = jb + grp;
      const bool has = my < jb1;
      const int4 job = has ? a.jobs[my] : make_int4(0, 0, 0, 0);
      int maxy = 0;
      for (int g = 0; g < jp && jb + g < jb1; ++g) maxy = max(maxy, a.jobs[jb + g].y);
      const float4 sh = has ? a.shifts[job.w] : make_float4(0.f, 0.f, 0.f, 0.f);
      float4* spg = sp + grp * slice;
      float2(*sfg)[NR] = sf + grp * slice;
      for (int r0 = 0; r0 < a.nrhs; r0 += NR) {
        const int nr = min(NR, a.nrhs - r0);
        float2 acc[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[k] = make_float2(0.f, 0.f);
        for (int i0 = 0; i0 < maxy; i0 += slice) {
          const int ni = max(0, min(slice, job.y - i0));
          __syncthreads();
          for (int e = lane; e < ni; e += tpj) {
            float4 v = a.pts[job.x + i0 + e];
            v.x += sh.x; v.y += sh.y; v.z += sh.z;
            v.w = v.x * v.x + v.y * v.y + v.z * v.z;
            spg[e] = v;
          }
          for (int e = lane; e < ni * NR; e += tpj) {
            int i = e / NR, k = e % NR;
            sfg[i][k] = k < nr ? a.fs[(int64_t)(job.x + i0 + i) * a.nrhs + r0 + k] : make_float2(0.f, 0.f);
          }
          __syncthreads();
          if (p < a.nchk) {
            for (int i = 0; i < ni; ++i) {
              float4 v = spg[i];
              // |x - v|^2 = |x|^2 + s,  s = |v|^2 - 2 x.v ; d - |x| = s / (d + |x|)
              float s = fmaf(-2.f, c.x * v.x + c.y * v.y + c.z * v.z, v.w);
              float d2 = c.nx2 + s;
              float inv_d = rsqrtf(d2);
              float d = d2 * inv_d;
              // d + |x| >= |x| ~ w: the fast division's 2 ulp change the phase by < 1e-6 rad
              float phase = c.fx + __fdividef(s, d + c.nx);
              float2 g = green_phase(phase, inv_d);
#pragma unroll
              for (int k = 0; k < NR; ++k) {
                float2 f = sfg[i][k];
                acc[k].x = fmaf(g.x, f.x, fmaf(-g.y, f.y, acc[k].x));
                acc[k].y = fmaf(g.x, f.y, fmaf(g.y, f.x, acc[k].y));
              }
            }
          }
        }
        if (has) {
          float2* out = a.out + (int64_t)job.z * a.nrhs * a.ld;
          if (p < a.nchk)
            for (int k = 0; k < nr; ++k) out[(int64_t)(r0 + k) * a.ld + p] = acc[k];
          if (p0 == 0)   // zero padding rows of the check-point sample
            for (int q = a.nchk + lane; q < a.ld; q += tpj)
              for (int k = 0; k < nr; ++k) out[(int64_t)(r0 + k) * a.ld + q] = make_float2(0.f, 0.f);
        }
      }
    }
  }
}

__global__ __launch_bounds__(256) void rows_kernel(RowsArgs a) {
  const int4 job = a.jobs[blockIdx.x];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const float2* st = a.state + (int64_t)job.w * a.nrhs * a.R;
  for (int i = warp; i < job.y; i += 8) {
    const float2* row = a.rows + (int64_t)(job.z + i) * a.R;
    float2 rv[8];
    const int nq = (a.R + 31) / 32;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      int q = lane + 32 * t;
      rv[t] = (t < nq && q < a.R) ? row[q] : make_float2(0.f, 0.f);
    }
    for (int k = 0; k < a.nrhs; ++k) {
      float2 sum = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        int q = lane + 32 * t;
        if (t < nq && q < a.R) {
          float2 v = st[(int64_t)k * a.R + q];
          sum.x = fmaf(rv[t].x, v.x, fmaf(-rv[t].y, v.y, sum.x));
          sum.y = fmaf(rv[t].x, v.y, fmaf(rv[t].y, v.x, sum.y));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
      }
      if (lane == 0) {
        float2* u = a.us + (int64_t)(job.x + i) * a.nrhs + k;
        if (a.atomic) atomicAdd(u, sum);
        else { float2 o = *u; *u = make_float2(o.x + sum.x, o.y + sum.y); }
      }
    }
  }
}

// L2P as a flat stream of rows: warp w evaluates the point rows 2w and 2w+1
// (1 KB each at rank 128, loaded together as float4 before any arithmetic);
// the state rows they dot with are shared by the points of a leaf and mostly
// hit in L1.  Two rows per warp keep the registers low and the warps many:
// 0.27 ms at K = 64 against 0.28 ms with four rows and 0.43 ms with eight.
constexpr int L2P_ROWS = 2;

template <int Q>
__global__ __launch_bounds__(256) void l2p_kernel(L2PArgs a) {
  const int64_t r0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * L2P_ROWS;
  const int lane = threadIdx.x & 31;
  if (r0 >= a.nrows) return;
  const int R2 = a.R / 2;
  float4 v[L2P_ROWS][Q];
  int2 m[L2P_ROWS];
#pragma unroll
  for (int j = 0; j < L2P_ROWS; ++j) {
    const int64_t r = r0 + j;
    const bool ok = r < a.nrows;
    m[j] = ok ? a.map[r] : make_int2(-1, 0);
    const float4* row = (const float4*)(a.rows + (ok ? r : r0) * a.R);
#pragma unroll
    for (int t = 0; t < Q; ++t) {
      const int q = lane + 32 * t;
      v[j][t] = (ok && q < R2) ? __ldcs(row + q) : make_float4(0.f, 0.f, 0.f, 0.f);   // streamed once
    }
  }
#pragma unroll
  for (int j = 0; j < L2P_ROWS; ++j) {
    if (m[j].x < 0) continue;   // warp-uniform
    const float4* st = (const float4*)(a.state + (int64_t)m[j].y * a.nrhs * a.R);
    for (int k = 0; k < a.nrhs; ++k) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < Q; ++t) {
        const int q = lane + 32 * t;
        if (q < R2) {
          const float4 sv = __ldg(st + (int64_t)k * R2 + q);
          acc.x = fmaf(v[j][t].x, sv.x, fmaf(-v[j][t].y, sv.y, acc.x));
          acc.y = fmaf(v[j][t].x, sv.y, fmaf(v[j][t].y, sv.x, acc.y));
          acc.x = fmaf(v[j][t].z, sv.z, fmaf(-v[j][t].w, sv.w, acc.x));
          acc.y = fmaf(v[j][t].z, sv.w, fmaf(v[j][t].w, sv.z, acc.y));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) {
        float2* u = a.us + (int64_t)m[j].x * a.nrhs + k;
        const float2 o = *u;
        *u = make_float2(o.x + acc.x, o.y + acc.y);
      }
    }
  }
}

// P2M through rows: one warp per leaf, lane l owns the state entries
// 2 (l + 32 t), 2 (l + 32 t) + 1 (float4 loads); the leaf's point rows are read
// 4 at a time (4 KB in flight per warp) and weighted by the points' densities
// (one broadcast load per point and right-hand side).  KB right-hand sides are
// accumulated per pass over the rows: 1 for a single right-hand side, whose
// accumulators then take a quarter of the registers, so that more warps
// (more rows in flight) fit on an SM.
template <int Q, int KB>
__global__ __launch_bounds__(256) void p2m_rows_kernel(P2MRowsArgs a) {
  const int64_t jw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (jw >= a.njobs) return;
  const int4 job = a.jobs[jw];
  const int R2 = a.R / 2;
  const float4* rows = (const float4*)a.rows;
  float4* st = (float4*)a.state;
  for (int k0 = 0; k0 < a.nrhs; k0 += KB) {
    const int nk = min(KB, a.nrhs - k0);
    float4 acc[KB][Q];
#pragma unroll
    for (int kk = 0; kk < KB; ++kk)
#pragma unroll
      for (int t = 0; t < Q; ++t) acc[kk][t] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < job.y; i += 4) {
      float4 r[4][Q];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int t = 0; t < Q; ++t) {
          const int q = lane + 32 * t;
          r[j][t] = (i + j < job.y && q < R2) ? __ldcs(rows + (int64_t)(job.z + i + j) * R2 + q)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (i + j >= job.y) break;
#pragma unroll
        for (int kk = 0; kk < KB; ++kk) {
          if (kk >= nk) break;
          const float2 f = __ldg(a.fs + (int64_t)(job.x + i + j) * a.nrhs + k0 + kk);
#pragma unroll
          for (int t = 0; t < Q; ++t) {
            float4& c = acc[kk][t];
            const float4 v = r[j][t];
            c.x = fmaf(v.x, f.x, fmaf(-v.y, f.y, c.x));
            c.y = fmaf(v.x, f.y, fmaf(v.y, f.x, c.y));
            c.z = fmaf(v.z, f.x, fmaf(-v.w, f.y, c.z));
            c.w = fmaf(v.z, f.y, fmaf(v.w, f.x, c.w));
          }
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < KB; ++kk) {
      if (kk >= nk) break;
#pragma unroll
      for (int t = 0; t < Q; ++t) {
        const int q = lane + 32 * t;
        if (q < R2) st[((int64_t)job.w * a.nrhs + k0 + kk) * R2 + q] = acc[kk][t];
      }
    }
  }
}

constexpr int P2P_THREADS = 128;
constexpr int P2P_CHUNK = 512;    // source points staged at a time
constexpr int P2P_LEAVES = 64;    // U-list entries staged at a time

// Exact sum a + b = s + e (Knuth's TwoSum; IEEE adds, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Near field (the U list of Sec. 2.4 and the HF near pairs of Sec. 3.2
// evaluated directly, Eq. 1).  Coordinates are box-local double-floats
// (hi + lo), so the difference of two nearby points keeps full single-precision
// relative accuracy however close they are (the 1/d amplitude of the closest
// pairs dominates their targets' potentials).  The leaf-centre shift is added
// exactly with TwoSum when a source point is staged.  One block per target
// leaf: up to P2P_LEAVES U-list entries are read at once and prefix-summed,
// then their points are gathered into shared memory in parallel, P2P_CHUNK at
// a time (each thread finds its point's leaf by binary search).  The threads
// are split into groups that each take every ngrp-th staged source; NR
// right-hand sides are accumulated per pass.
template <int NR>
__global__ __launch_bounds__(P2P_THREADS) void p2p_kernel(P2PArgs a) {
  __shared__ float4 syh[P2P_CHUNK];
  __shared__ float4 syl[P2P_CHUNK];
  __shared__ float2 sf[P2P_CHUNK][NR];
  __shared__ float2 red[P2P_THREADS][NR];
  __shared__ int4 su[P2P_LEAVES];
  __shared__ float4 ssh[P2P_LEAVES];
  __shared__ int soff[P2P_LEAVES + 1];
  const int2 lr = a.leaf_range[blockIdx.x];
  const int64_t u0 = a.u_off[blockIdx.x], u1 = a.u_off[blockIdx.x + 1];
  const int lane = threadIdx.x & 31;
  for (int t0 = 0; t0 < lr.y; t0 += P2P_THREADS) {
    const int nt = min(P2P_THREADS, lr.y - t0);
    const int ngrp = P2P_THREADS / nt;
    const int ti = threadIdx.x % nt, grp = threadIdx.x / nt;
    const bool active = grp < ngrp;
    const float4 xh = a.pts[lr.x + t0 + ti];
    const float4 xl = a.pts_lo[lr.x + t0 + ti];
    for (int r0 = 0; r0 < a.nrhs; r0 += NR) {
      const int nr = min(NR, a.nrhs - r0);
      float2 acc[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) acc[k] = make_float2(0.f, 0.f);
      for (int64_t ub = u0; ub < u1; ub += P2P_LEAVES) {
        const int nb = (int)(u1 - ub < P2P_LEAVES ? u1 - ub : P2P_LEAVES);
        __syncthreads();   // the previous batch has been consumed
        if (threadIdx.x < nb) {
          su[threadIdx.x] = a.u_src[ub + threadIdx.x];
          ssh[threadIdx.x] = a.u_shift[ub + threadIdx.x];
        }
        __syncthreads();
        if (threadIdx.x < 32) {   // exclusive prefix of the leaf sizes
          int v0 = lane < nb ? su[lane].y : 0;
          int v1 = lane + 32 < nb ? su[lane + 32].y : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, v0, o);
            int w = __shfl_up_sync(0xffffffffu, v1, o);
            if (lane >= o) { v0 += t; v1 += w; }
          }
          v1 += __shfl_sync(0xffffffffu, v0, 31);
          soff[lane + 1] = v0;
          soff[lane + 33] = v1;
          if (lane == 0) soff[0] = 0;
        }
        __syncthreads();
        const int total = soff[nb];
        for (int c0 = 0; c0 < total; c0 += P2P_CHUNK) {
          const int fill = min(P2P_CHUNK, total - c0);
          if (c0 > 0) __syncthreads();
          for (int e = threadIdx.x; e < fill; e += P2P_THREADS) {
            const int q = c0 + e;
            int lo = 0, hi = nb;   // soff[lo] <= q < soff[hi]
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (soff[mid] <= q) lo = mid; else hi = mid;
            }
            const int j = su[lo].x + (q - soff[lo]);
            const float4 sh = ssh[lo];
            const float4 vh = a.pts[j], vl = a.pts_lo[j];
            float hx, hy, hz, ex, ey, ez;
            two_sum(vh.x, sh.x, hx, ex);
            two_sum(vh.y, sh.y, hy, ey);
            two_sum(vh.z, sh.z, hz, ez);
            syh[e] = make_float4(hx, hy, hz, 0.f);
            syl[e] = make_float4(vl.x + ex, vl.y + ey, vl.z + ez, 0.f);
#pragma unroll
            for (int k = 0; k < NR; ++k)
              sf[e][k] = k < nr ? a.fs[(int64_t)j * a.nrhs + r0 + k] : make_float2(0.f, 0.f);
          }
          __syncthreads();
          if (active) {
#pragma unroll 4
            for (int j = grp; j < fill; j += ngrp) {
              const float4 yh = syh[j], yl = syl[j];
              float dx = (xh.x - yh.x) + (xl.x - yl.x);
              float dy = (xh.y - yh.y) + (xl.y - yl.y);
              float dz = (xh.z - yh.z) + (xl.z - yl.z);
              float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              // a coincident source (r2 == 0) contributes nothing: 1/d is set to 0.
              // rsqrtf's 2 ulp give |G| to 2e-7 and the phase to 1e-6 rad (d < 2).
              const float inv_d = r2 > 0.f ? rsqrtf(r2) : 0.f;
              float2 g = green_phase(r2 * inv_d, inv_d);
#pragma unroll
              for (int k = 0; k < NR; ++k) {
                float2 f = sf[j][k];
                acc[k].x = fmaf(g.x, f.x, fmaf(-g.y, f.y, acc[k].x));
                acc[k].y = fmaf(g.x, f.y, fmaf(g.y, f.x, acc[k].y));
              }
            }
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < NR; ++k) red[threadIdx.x][k] = active ? acc[k] : make_float2(0.f, 0.f);
      __syncthreads();
      if (threadIdx.x < nt) {
        for (int k = 0; k < nr; ++k) {
          float2 sum = make_float2(0.f, 0.f);
          for (int g = 0; g < ngrp; ++g) {
            float2 v = red[g * nt + threadIdx.x][k];
            sum.x += v.x;
            sum.y += v.y;
          }
          float2* uu = a.us + (int64_t)(lr.x + t0 + threadIdx.x) * a.nrhs + r0 + k;
          float2 o = *uu;
          *uu = make_float2(o.x + sum.x, o.y + sum.y);
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------
// FP32 form of the near field.  Coordinates are the high parts alone: a
// source point is shifted into the target leaf's frame once, when it is staged,
// and every pair then costs three subtractions for its difference.  Their
// rounding (about 1e-7 absolute) matters only for close pairs, whose 1/d
// amplitude it perturbs by 1e-7 / d relative: the plan lists every pair closer
// than delta and stores its exact correction G(p_i, p_j) - g32 (FP64 at plan
// time), added at the end.  Only points of the target leaf itself can
// coincide (equal points have equal Morton keys), so only that entry of the U
// list, kept first, takes the guarded form.

constexpr int PF_THREADS = 128;
constexpr int PF_CHUNK = 512;

// The FP32 form's kernel value for one pair: target x and source y in the target
// leaf's frame.  Every rounding is explicit, so the close-pair pass reproduces
// the main loop's value exactly.  guarded: a coincident pair gives 0.
template <bool guarded>
__device__ __forceinline__ float2 g32(float xx, float xy, float xz, float4 y) {
  const float dx = __fsub_rn(xx, y.x), dy = __fsub_rn(xy, y.y), dz = __fsub_rn(xz, y.z);
  const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
  const float inv = guarded ? (r2 > 0.f ? rsqrtf(r2) : 0.f) : rsqrtf(r2);
  const float d = __fmul_rn(r2, inv);
  const float ph = __fsub_rn(d, round_near(d));
  float sn, cs;
  __sincosf(__fmul_rn(6.28318530717958647f, ph), &sn, &cs);
  return make_float2(__fmul_rn(cs, inv), __fmul_rn(sn, inv));
}

__device__ __forceinline__ float4 shifted(float4 v, float4 sh) {
  return make_float4(__fadd_rn(v.x, sh.x), __fadd_rn(v.y, sh.y), __fadd_rn(v.z, sh.z), 0.f);
}

// One block per target leaf; each thread holds two targets (t and t + nth), so
// a staged source is read from shared memory once per two interactions; the
// threads form groups that split the staged sources.  NR right-hand sides per
// pass.
template <int NR>
__global__ __launch_bounds__(PF_THREADS) void p2p_fast_kernel(P2PArgs a) {
  __shared__ float4 sy[PF_CHUNK];
  __shared__ float2 sf[PF_CHUNK][NR];
  __shared__ float2 red[PF_THREADS][2][NR];
  __shared__ float4 stab[128];   // shift of each entry of the leaf's list
  const int2 lr = a.leaf_range[blockIdx.x];
  const int64_t u0 = a.u_off[blockIdx.x], u1 = a.u_off[blockIdx.x + 1];
  // the leaf's list: the flat staging list and the entry offsets are precomputed
  const int4 e0 = a.u_src[u0], el = a.u_src[u1 - 1];
  const int total = el.z + el.y - e0.z;
  const int self_end = e0.w ? e0.y : 0;   // staged indices of the own leaf's points
  for (int t = threadIdx.x; t < (int)(u1 - u0); t += PF_THREADS) stab[t] = a.u_shift[u0 + t];
  for (int t0 = 0; t0 < lr.y; t0 += 2 * PF_THREADS) {
    const int nt = min(2 * PF_THREADS, lr.y - t0);
    const int nth = (nt + 1) >> 1;
    // thread -> (group, target pair) without integer division: the operands are
    // below 256, so the correctly rounded reciprocal leaves a margin of 1 / 256
    const float rth = __frcp_rn((float)nth);
    const int ngrp = (int)(((float)PF_THREADS + 0.5f) * rth);
    const int grp = (int)(((float)threadIdx.x + 0.5f) * rth), ti = threadIdx.x - grp * nth;
    const float rgrp = __frcp_rn((float)ngrp);
    const bool active = grp < ngrp;
    const int i1 = ti + nth < nt ? ti + nth : ti;   // an odd count repeats the last target
    const float4 x0 = a.pts[lr.x + t0 + ti];
    const float4 x1 = a.pts[lr.x + t0 + i1];
    for (int r0 = 0; r0 < a.nrhs; r0 += NR) {
      const int nr = min(NR, a.nrhs - r0);
      float2 acc0[NR], acc1[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) acc0[k] = acc1[k] = make_float2(0.f, 0.f);
      for (int c0 = 0; c0 < total; c0 += PF_CHUNK) {
        const int fill = min(PF_CHUNK, total - c0);
        __syncthreads();   // the previous chunk (and the previous pass's sums) are consumed
        // one thread per staged source: its point, shifted into this leaf's frame
        for (int q = threadIdx.x; q < fill; q += PF_THREADS) {
          const uint32_t v = a.flat[e0.z + c0 + q];
          const int j = (int)(v & 0x1FFFFFFu);
          sy[q] = shifted(a.pts[j], stab[v >> 25]);
#pragma unroll
          for (int k = 0; k < NR; ++k)
            sf[q][k] = k < nr ? a.fs[(int64_t)j * a.nrhs + r0 + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (active) {
          // the own leaf's points (staged first) take the guarded form, spread
          // over the groups so that the lanes of a warp stay on one path; the
          // rest is split into contiguous shares
          const int self_hi = min(max(self_end - c0, 0), fill);
          const int per = (int)(((float)(fill - self_hi + ngrp) - 0.5f) * rgrp);   // ceil((fill - self_hi) / ngrp)
          const int jlo = min(fill, self_hi + grp * per), jhi = min(fill, jlo + per);
          auto body = [&](int j, auto guard) {
            const float4 y = sy[j];
            constexpr bool G = decltype(guard)::value;
            const float2 g0 = g32<G>(x0.x, x0.y, x0.z, y), g1 = g32<G>(x1.x, x1.y, x1.z, y);
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              const float2 f = sf[j][k];
              acc0[k].x = fmaf(g0.x, f.x, fmaf(-g0.y, f.y, acc0[k].x));
              acc0[k].y = fmaf(g0.x, f.y, fmaf(g0.y, f.x, acc0[k].y));
              acc1[k].x = fmaf(g1.x, f.x, fmaf(-g1.y, f.y, acc1[k].x));
              acc1[k].y = fmaf(g1.x, f.y, fmaf(g1.y, f.x, acc1[k].y));
            }
          };
          for (int j = grp; j < self_hi; j += ngrp) body(j, std::true_type());
          int j = jlo;
          for (; j + 3 < jhi; j += 4) {
            body(j, std::false_type());
            body(j + 1, std::false_type());
            body(j + 2, std::false_type());
            body(j + 3, std::false_type());
          }
          for (; j < jhi; ++j) body(j, std::false_type());
        }
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        red[threadIdx.x][0][k] = active ? acc0[k] : make_float2(0.f, 0.f);
        red[threadIdx.x][1][k] = active ? acc1[k] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      for (int tt = threadIdx.x; tt < nt; tt += PF_THREADS) {
        const int th = tt < nth ? tt : tt - nth, slot = tt < nth ? 0 : 1;
        const int64_t i = lr.x + t0 + tt;
        for (int k = 0; k < nr; ++k) {
          float2 sum = make_float2(0.f, 0.f);
          for (int g = 0; g < ngrp; ++g) {
            const float2 v = red[g * nth + th][slot][k];
            sum.x += v.x;
            sum.y += v.y;
          }
          red_add2((float*)(a.us + i * a.nrhs + r0 + k), sum.x, sum.y);   // no round trip
        }
      }
    }
  }
}

// Exact corrections of the close pairs of the FP32 form, one thread per
// target point: us[i] += sum_c w_c f[j_c].
__global__ void p2p_close_apply_kernel(P2PArgs a, int64_t npoints) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npoints) return;
  const int c0 = a.close_off[i], c1 = a.close_off[i + 1];
  if (c0 == c1) return;
  for (int k = 0; k < a.nrhs; ++k) {
    float2 sum = make_float2(0.f, 0.f);
    for (int c = c0; c < c1; ++c) {
      const float2 w = a.close_w[c];
      const float2 f = a.fs[(int64_t)a.close_j[c] * a.nrhs + k];
      sum.x = fmaf(w.x, f.x, fmaf(-w.y, f.y, sum.x));
      sum.y = fmaf(w.x, f.y, fmaf(w.y, f.x, sum.y));
    }
    float2* uu = a.us + i * a.nrhs + k;
    const float2 o = *uu;
    *uu = make_float2(o.x + sum.x, o.y + sum.y);
  }
}

// Close pairs of the FP32 form (plan time): one thread per target point walks
// its leaf's U list.  Pass 1 counts, pass 2 writes (j, G - g32) with G in FP64
// from the double-float coordinates.
__global__ void p2p_close_kernel(P2PArgs a, float delta2, int32_t* cnt, unsigned* degenerate,
                                 const int32_t* off, int32_t* cj, float2* cw) {
  const int64_t leaf = blockIdx.x;
  const int2 lr = a.leaf_range[leaf];
  const int64_t u0 = a.u_off[leaf], u1 = a.u_off[leaf + 1];
  for (int t = threadIdx.x; t < lr.y; t += blockDim.x) {
    const int64_t i = lr.x + t;
    const float4 x = a.pts[i], xl = a.pts_lo[i];
    int n = 0;
    for (int64_t e = u0; e < u1; ++e) {
      const int4 ue = a.u_src[e];
      const float4 sh = a.u_shift[e];
      for (int q = 0; q < ue.y; ++q) {
        const int j = ue.x + q;
        const float4 v = a.pts[j], vl = a.pts_lo[j];
        const float4 y = shifted(v, sh);
        const float dx = __fsub_rn(x.x, y.x), dy = __fsub_rn(x.y, y.y), dz = __fsub_rn(x.z, y.z);
        const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
        const bool same = ue.w && v.x == x.x && v.y == x.y && v.z == x.z && vl.x == xl.x && vl.y == xl.y &&
                          vl.z == xl.z;
        if (same || !(r2 < delta2)) continue;
        if (r2 == 0.f) atomicOr(degenerate, 1u);
        if (off) {
          const double ex = ((double)x.x + (double)xl.x) - ((double)v.x + (double)vl.x + (double)sh.x);
          const double ey = ((double)x.y + (double)xl.y) - ((double)v.y + (double)vl.y + (double)sh.y);
          const double ez = ((double)x.z + (double)xl.z) - ((double)v.z + (double)vl.z + (double)sh.z);
          const double d = sqrt(ex * ex + ey * ey + ez * ez);
          double sn, cs;
          sincospi(2.0 * d, &sn, &cs);
          const float2 g = g32<true>(x.x, x.y, x.z, y);
          const int64_t c = off[i] + n;
          cj[c] = j;
          cw[c] = make_float2((float)(cs / d - (double)g.x), (float)(sn / d - (double)g.y));
        }
        ++n;
      }
    }
    if (!off) cnt[i] = n;
  }
}

}  // namespace

void launch_gemm_stage(const GemmArgs& a, cudaStream_t s) {
  if (a.ntiles == 0) return;
  dim3 grid((unsigned)a.ntiles, (unsigned)((a.M + BM - 1) / BM));
  gemm_stage_kernel<<<grid, 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_permute_in(const float2* f, const int32_t* perm, int64_t N, int nrhs, float2* fs, cudaStream_t s) {
  int64_t n = N * nrhs;
  permute_in_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, perm, N, nrhs, fs);
  DFMM_CUDA(cudaGetLastError());
}

void launch_permute_out(const float2* us, const int32_t* perm, int64_t N, int nrhs, float2* u, cudaStream_t s) {
  int64_t n = N * nrhs;
  permute_out_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(us, perm, N, nrhs, u);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2c(const P2CArgs& a, cudaStream_t s) {
  if (a.njobs == 0) return;
  const int tpj = max(32, (min(a.nchk, P2C_THREADS) + 31) / 32 * 32);
  const int jp = P2C_THREADS / tpj;
  const unsigned grid = (unsigned)((a.njobs + (int64_t)jp * P2C_JOBS - 1) / ((int64_t)jp * P2C_JOBS));
  if (a.nrhs == 1) p2c_kernel<1><<<grid, jp * tpj, 0, s>>>(a, tpj);
  else if (a.nrhs == 2) p2c_kernel<2><<<grid, jp * tpj, 0, s>>>(a, tpj);
  else if (a.nrhs <= 4) p2c_kernel<4><<<grid, jp * tpj, 0, s>>>(a, tpj);
  else p2c_kernel<8><<<grid, jp * tpj, 0, s>>>(a, tpj);
  DFMM_CUDA(cudaGetLastError());
}

void launch_rows(const RowsArgs& a, cudaStream_t s) {
  if (a.njobs == 0) return;
  if (a.R > 256 || a.R % 2) throw Error(-5, "representation rank must be even and at most 256");
  rows_kernel<<<(unsigned)a.njobs, 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_l2p(const L2PArgs& a, cudaStream_t s) {
  if (a.nrows == 0) return;
  if (a.R > 256 || a.R % 2) throw Error(-5, "representation rank must be even and at most 256");
  const unsigned grid = (unsigned)((a.nrows + 8 * L2P_ROWS - 1) / (8 * L2P_ROWS));
  if (a.R <= 128) l2p_kernel<2><<<grid, 256, 0, s>>>(a);
  else l2p_kernel<4><<<grid, 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2m_rows(const P2MRowsArgs& a, cudaStream_t s) {
  if (a.njobs == 0) return;
  if (a.R > 256 || a.R % 2) throw Error(-5, "representation rank must be even and at most 256");
  const unsigned grid = (unsigned)((a.njobs + 7) / 8);
  if (a.nrhs == 1) {
    if (a.R <= 128) p2m_rows_kernel<2, 1><<<grid, 256, 0, s>>>(a);
    else p2m_rows_kernel<4, 1><<<grid, 256, 0, s>>>(a);
  } else {
    if (a.R <= 128) p2m_rows_kernel<2, 4><<<grid, 256, 0, s>>>(a);
    else p2m_rows_kernel<4, 4><<<grid, 256, 0, s>>>(a);
  }
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2p_fast(const P2PArgs& a, int64_t npoints, cudaStream_t s) {
  if (a.nleaves == 0) return;
  if (a.nrhs == 1) p2p_fast_kernel<1><<<(unsigned)a.nleaves, PF_THREADS, 0, s>>>(a);
  else if (a.nrhs == 2) p2p_fast_kernel<2><<<(unsigned)a.nleaves, PF_THREADS, 0, s>>>(a);
  else p2p_fast_kernel<4><<<(unsigned)a.nleaves, PF_THREADS, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
  p2p_close_apply_kernel<<<(unsigned)((npoints + 255) / 256), 256, 0, s>>>(a, npoints);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2p_close(const P2PArgs& a, float delta, int32_t* cnt, unsigned* degenerate, const int32_t* off,
                      int32_t* close_j, float2* close_w, cudaStream_t s) {
  if (a.nleaves == 0) return;
  p2p_close_kernel<<<(unsigned)a.nleaves, 64, 0, s>>>(a, delta * delta, cnt, degenerate, off, close_j, close_w);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2p(const P2PArgs& a, cudaStream_t s) {
  if (a.nleaves == 0) return;
  if (a.nrhs == 1) p2p_kernel<1><<<(unsigned)a.nleaves, P2P_THREADS, 0, s>>>(a);
  else if (a.nrhs == 2) p2p_kernel<2><<<(unsigned)a.nleaves, P2P_THREADS, 0, s>>>(a);
  else p2p_kernel<4><<<(unsigned)a.nleaves, P2P_THREADS, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

}  // namespace dfmm
