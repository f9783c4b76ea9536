// Apply-time kernels of the directional FMM matvec (FP32).
//
//  * gemm_stage_kernel: every translation of Alg. 1 (P2M/P2L projections,
//    LF/HF-M2M, HF-M2L, LF-M2L, HF/LF-L2L) is "y[dst] += T_op x[src]" over a
//    list of (src, dst) pairs grouped by operator.  One CTA computes a
//    64-row x 64-column block of T_op X, where the columns are the gathered
//    source states (pairs x right-hand sides), and scatter-adds the result
//    into the target states with vector atomics (targets of one operator are
//    distinct, different operators meet in L2).  This is the plain CUDA-core
//    form; the tensor-core form is in m2l_tc.cu.
//  * p2c_kernel: potentials at check points from points (P2M, P2L), with the
//    phase 2 pi |x - y| reduced in a compensated form so that far check
//    points keep full FP32 accuracy.
//  * rows_kernel: L2P and M2P through precomputed rows.
//  * p2p_kernel: the near field (U lists) in FP32 on box-local coordinates.
#include "apply.h"

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

// exp(2 pi i phase) / d with phase reduced to [-1/2, 1/2]
__device__ __forceinline__ float2 green_phase(float phase, float inv_d) {
  float ph = phase - rintf(phase);
  float s, c;
  __sincosf(6.28318530717958647f * ph, &s, &c);
  return make_float2(c * inv_d, s * inv_d);
}

constexpr int P2C_THREADS = 256;
constexpr int P2C_CHUNK = 128;
constexpr int P2C_RHS = 8;

__global__ __launch_bounds__(P2C_THREADS) void p2c_kernel(P2CArgs a) {
  __shared__ float4 sp[P2C_CHUNK];
  __shared__ float2 sf[P2C_CHUNK][P2C_RHS];
  const int4 job = a.jobs[blockIdx.x];
  const float4 sh = a.shifts[job.w];
  for (int r0 = 0; r0 < a.nrhs; r0 += P2C_RHS) {
    const int nr = min(P2C_RHS, a.nrhs - r0);
    for (int p0 = 0; p0 < a.ld; p0 += P2C_THREADS) {
      const int p = p0 + threadIdx.x;
      ChkPt c = {};
      if (p < a.nchk) c = a.chk[p];
      float2 acc[P2C_RHS];
#pragma unroll
      for (int k = 0; k < P2C_RHS; ++k) acc[k] = make_float2(0.f, 0.f);
      for (int i0 = 0; i0 < job.y; i0 += P2C_CHUNK) {
        const int ni = min(P2C_CHUNK, job.y - i0);
        __syncthreads();
        for (int e = threadIdx.x; e < ni; e += P2C_THREADS) {
          float4 v = a.pts[job.x + i0 + e];
          v.x += sh.x; v.y += sh.y; v.z += sh.z;
          v.w = v.x * v.x + v.y * v.y + v.z * v.z;
          sp[e] = v;
        }
        for (int e = threadIdx.x; e < ni * P2C_RHS; e += P2C_THREADS) {
          int i = e / P2C_RHS, k = e % P2C_RHS;
          sf[i][k] = k < nr ? a.fs[(int64_t)(job.x + i0 + i) * a.nrhs + r0 + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (p < a.nchk) {
          for (int i = 0; i < ni; ++i) {
            float4 v = sp[i];
            // |x - v|^2 = |x|^2 + s,  s = |v|^2 - 2 x.v ; d - |x| = s / (d + |x|)
            float s = fmaf(-2.f, c.x * v.x + c.y * v.y + c.z * v.z, v.w);
            float d2 = c.nx2 + s;
            float inv_d = rsqrtf(d2);
            float d = d2 * inv_d;
            float phase = c.fx + s / (d + c.nx);
            float2 g = green_phase(phase, inv_d);
#pragma unroll
            for (int k = 0; k < P2C_RHS; ++k) {
              float2 f = sf[i][k];
              acc[k].x = fmaf(g.x, f.x, fmaf(-g.y, f.y, acc[k].x));
              acc[k].y = fmaf(g.x, f.y, fmaf(g.y, f.x, acc[k].y));
            }
          }
        }
      }
      if (p < a.ld) {
        for (int k = 0; k < nr; ++k)
          a.out[((int64_t)job.z * a.nrhs + r0 + k) * a.ld + p] = p < a.nchk ? acc[k] : make_float2(0.f, 0.f);
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

constexpr int P2P_THREADS = 128;
constexpr int P2P_CHUNK = 256;
constexpr int P2P_RHS = 4;

// Exact sum a + b = s + e (Knuth's TwoSum; IEEE adds, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Near field.  Coordinates are box-local double-floats (hi + lo), so the
// difference of two nearby points keeps full single-precision relative
// accuracy however close they are (the 1/d amplitude of the closest pairs
// dominates their targets' potentials).  The leaf-centre shift is added
// exactly with TwoSum when the source chunk is staged.
__global__ __launch_bounds__(P2P_THREADS) void p2p_kernel(P2PArgs a) {
  __shared__ float4 syh[P2P_CHUNK];
  __shared__ float4 syl[P2P_CHUNK];
  __shared__ float2 sf[P2P_CHUNK][P2P_RHS];
  __shared__ float2 red[P2P_THREADS][P2P_RHS];
  const int2 lr = a.leaf_range[blockIdx.x];
  const int64_t u0 = a.u_off[blockIdx.x], u1 = a.u_off[blockIdx.x + 1];
  for (int t0 = 0; t0 < lr.y; t0 += P2P_THREADS) {
    const int nt = min(P2P_THREADS, lr.y - t0);
    const int ngrp = P2P_THREADS / nt;
    const int ti = threadIdx.x % nt, grp = threadIdx.x / nt;
    const bool active = grp < ngrp;
    const float4 xh = a.pts[lr.x + t0 + ti];
    const float4 xl = a.pts_lo[lr.x + t0 + ti];
    for (int r0 = 0; r0 < a.nrhs; r0 += P2P_RHS) {
      const int nr = min(P2P_RHS, a.nrhs - r0);
      float2 acc[P2P_RHS];
#pragma unroll
      for (int k = 0; k < P2P_RHS; ++k) acc[k] = make_float2(0.f, 0.f);
      for (int64_t u = u0; u < u1; ++u) {
        const int4 src = a.u_src[u];
        const float4 sh = a.shifts[src.z];
        for (int j0 = 0; j0 < src.y; j0 += P2P_CHUNK) {
          const int nj = min(P2P_CHUNK, src.y - j0);
          __syncthreads();
          for (int e = threadIdx.x; e < nj; e += P2P_THREADS) {
            float4 vh = a.pts[src.x + j0 + e], vl = a.pts_lo[src.x + j0 + e];
            float hx, hy, hz, ex, ey, ez;
            two_sum(vh.x, sh.x, hx, ex);
            two_sum(vh.y, sh.y, hy, ey);
            two_sum(vh.z, sh.z, hz, ez);
            syh[e] = make_float4(hx, hy, hz, 0.f);
            syl[e] = make_float4(vl.x + ex, vl.y + ey, vl.z + ez, 0.f);
          }
          for (int e = threadIdx.x; e < nj * P2P_RHS; e += P2P_THREADS) {
            int j = e / P2P_RHS, k = e % P2P_RHS;
            sf[j][k] = k < nr ? a.fs[(int64_t)(src.x + j0 + j) * a.nrhs + r0 + k] : make_float2(0.f, 0.f);
          }
          __syncthreads();
          if (active) {
            for (int j = grp; j < nj; j += ngrp) {
              const float4 yh = syh[j], yl = syl[j];
              float dx = (xh.x - yh.x) + (xl.x - yl.x);
              float dy = (xh.y - yh.y) + (xl.y - yl.y);
              float dz = (xh.z - yh.z) + (xl.z - yl.z);
              float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              if (r2 > 0.f) {
                float inv_d = rsqrtf(r2);
                inv_d = inv_d * fmaf(-0.5f * r2 * inv_d, inv_d, 1.5f);   // one Newton step
                float2 g = green_phase(r2 * inv_d, inv_d);
#pragma unroll
                for (int k = 0; k < P2P_RHS; ++k) {
                  float2 f = sf[j][k];
                  acc[k].x = fmaf(g.x, f.x, fmaf(-g.y, f.y, acc[k].x));
                  acc[k].y = fmaf(g.x, f.y, fmaf(g.y, f.x, acc[k].y));
                }
              }
            }
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < P2P_RHS; ++k) red[threadIdx.x][k] = active ? acc[k] : make_float2(0.f, 0.f);
      __syncthreads();
      if (threadIdx.x < nt) {
        for (int k = 0; k < nr; ++k) {
          float2 s = make_float2(0.f, 0.f);
          for (int g = 0; g < ngrp; ++g) {
            float2 v = red[g * nt + threadIdx.x][k];
            s.x += v.x;
            s.y += v.y;
          }
          float2* u = a.us + (int64_t)(lr.x + t0 + threadIdx.x) * a.nrhs + r0 + k;
          float2 o = *u;
          *u = make_float2(o.x + s.x, o.y + s.y);
        }
      }
      __syncthreads();
    }
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
  p2c_kernel<<<(unsigned)a.njobs, P2C_THREADS, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_rows(const RowsArgs& a, cudaStream_t s) {
  if (a.njobs == 0) return;
  if (a.R > 256) throw Error(-5, "representation rank above 256 is not supported");
  rows_kernel<<<(unsigned)a.njobs, 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2p(const P2PArgs& a, cudaStream_t s) {
  if (a.nleaves == 0) return;
  p2p_kernel<<<(unsigned)a.nleaves, P2P_THREADS, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

}  // namespace dfmm
