// FP64 forms of the apply-time kernels, for tolerances below what FP32
// arithmetic reaches (eps < 1e-6, down to the 1e-8 level of Table 1).
//
// The argument structs are those of the FP32 kernels (apply.h); in this form
// every complex array they name (operators, rows, states, densities,
// potentials) holds complex128 (double2) elements at the same indices.  Points
// are rebuilt in FP64 from their double-float local coordinates (hi + lo
// carries 48 significant bits, exact in a double), centre offsets are exact
// dyadic values, and the kernel exp(2 pi i d) / d of Eq. 1 is evaluated with
// sincospi, so no phase reduction is needed.  Plain CUDA-core kernels: the
// GB300 FP64 rate is far below its FP32 and tensor rates, so this form trades
// speed for the accuracy level.
#include "apply.h"

namespace dfmm {

namespace {

__device__ __forceinline__ const double2* c128(const float2* p) { return reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ double2* c128(float2* p) { return reinterpret_cast<double2*>(p); }

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// exp(2 pi i d) / d for the difference (dx, dy, dz); coincident points give 0
__device__ __forceinline__ double2 green64(double dx, double dy, double dz) {
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 > 0.0)) return make_double2(0.0, 0.0);
  const double d = sqrt(r2);
  const double inv = 1.0 / d;
  double sn, cs;
  sincospi(2.0 * d, &sn, &cs);
  return make_double2(cs * inv, sn * inv);
}

// FP64 local coordinates of sorted point j, shifted by sh
__device__ __forceinline__ double3 point64(const float4* hi, const float4* lo, int64_t j, float4 sh) {
  const float4 h = hi[j], l = lo[j];
  return make_double3(((double)h.x + (double)l.x) + (double)sh.x, ((double)h.y + (double)l.y) + (double)sh.y,
                      ((double)h.z + (double)l.z) + (double)sh.z);
}

__device__ __forceinline__ void add_to(double2* p, double2 v, bool atomic) {
  if (atomic) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
  } else {
    const double2 o = *p;
    *p = make_double2(o.x + v.x, o.y + v.y);
  }
}

// y[dst] += T_op x[src] over a stage's pairs: one CTA computes a 64-row x
// 64-column block of T_op X (columns = gathered source rows x right-hand
// sides) and adds it into the target rows with FP64 atomics.
constexpr int GM = 64, GN = 64, GK = 8;

__global__ __launch_bounds__(256) void gemm64_kernel(GemmArgs a) {
  __shared__ double2 As[GK][GM + 1];
  __shared__ double2 Bs[GK][GN + 1];
  __shared__ const double2* srcp[GN];
  __shared__ double2* dstp[GN];
  const int tid = threadIdx.x;
  const int4 tile = a.tiles[blockIdx.x];
  const double2* A = c128(a.ops) + (size_t)tile.x * a.M * a.Kd;
  const int row0 = blockIdx.y * GM;
  const int ncol = tile.z * a.nrhs;
  if (tid < GN) {
    const double2* sp = nullptr;
    double2* dp = nullptr;
    if (tid < ncol) {
      const int p = tile.y + tid / a.nrhs, k = tid % a.nrhs;
      const int2 pr = a.pairs[p];
      sp = c128(a.src) + ((int64_t)pr.x * a.nrhs + k) * a.src_ld;
      dp = c128(a.dst) + ((int64_t)pr.y * a.nrhs + k) * a.dst_ld;
    }
    srcp[tid] = sp;
    dstp[tid] = dp;
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < a.Kd; k0 += GK) {
    for (int e = tid; e < GM * GK; e += 256) {
      const int i = e / GK, kk = e % GK;
      const int r = row0 + i, kc = k0 + kk;
      As[kk][i] = (r < a.M && kc < a.Kd) ? A[(size_t)r * a.Kd + kc] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < GN * GK; e += 256) {
      const int c = e / GK, kk = e % GK;
      const int kc = k0 + kk;
      Bs[kk][c] = (c < ncol && kc < a.Kd) ? srcp[c][kc] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double2 av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], av[i], bv[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = tx * 4 + j;
    if (c >= ncol) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = row0 + ty * 4 + i;
      if (r < a.M) add_to(dstp[c] + r, acc[i][j], true);
    }
  }
}

__global__ void permute_in64_kernel(const double2* __restrict__ f, const int32_t* __restrict__ perm, int64_t N,
                                    int nrhs, double2* __restrict__ fs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nrhs) return;
  fs[e] = f[(e % nrhs) * N + perm[e / nrhs]];
}

__global__ void permute_out64_kernel(const double2* __restrict__ us, const int32_t* __restrict__ perm, int64_t N,
                                     int nrhs, double2* __restrict__ u) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nrhs) return;
  u[(e % nrhs) * N + perm[e / nrhs]] = us[e];
}

constexpr int C64_T = 128;   // threads of the check-point and near-field kernels
constexpr int C64_NR = 4;    // right-hand sides per pass

// Check-point potentials of a job's source points (the P2L sample of Eq. 6):
// one block per job, one thread per check point, sources staged in shared
// memory C64_T at a time; padding rows up to ld are written as zeros.
__global__ __launch_bounds__(C64_T) void p2c64_kernel(P2CArgs a) {
  __shared__ double3 sp[C64_T];
  __shared__ double2 sf[C64_T][C64_NR];
  const int4 job = a.jobs[blockIdx.x];
  const float4 sh = a.shifts[job.w];
  const double2* fs = c128(a.fs);
  double2* out = c128(a.out) + (int64_t)job.z * a.nrhs * a.ld;
  for (int r0 = 0; r0 < a.nrhs; r0 += C64_NR) {
    const int nr = min(C64_NR, a.nrhs - r0);
    for (int p0 = 0; p0 < a.ld; p0 += C64_T) {
      const int p = p0 + threadIdx.x;
      const bool live = p < a.nchk;
      const double cx = live ? a.chk64[3 * p] : 0.0, cy = live ? a.chk64[3 * p + 1] : 0.0,
                   cz = live ? a.chk64[3 * p + 2] : 0.0;
      double2 acc[C64_NR];
#pragma unroll
      for (int k = 0; k < C64_NR; ++k) acc[k] = make_double2(0.0, 0.0);
      for (int i0 = 0; i0 < job.y; i0 += C64_T) {
        const int ni = min(C64_T, job.y - i0);
        __syncthreads();
        if (threadIdx.x < ni) {
          const int64_t j = (int64_t)job.x + i0 + threadIdx.x;
          sp[threadIdx.x] = point64(a.pts, a.pts_lo, j, sh);
#pragma unroll
          for (int k = 0; k < C64_NR; ++k)
            sf[threadIdx.x][k] = k < nr ? fs[j * a.nrhs + r0 + k] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (live)
          for (int i = 0; i < ni; ++i) {
            const double3 v = sp[i];
            const double2 g = green64(cx - v.x, cy - v.y, cz - v.z);
#pragma unroll
            for (int k = 0; k < C64_NR; ++k) cfma(acc[k], g, sf[i][k]);
          }
      }
      if (p < a.ld)
        for (int k = 0; k < nr; ++k) out[(int64_t)(r0 + k) * a.ld + p] = live ? acc[k] : make_double2(0.0, 0.0);
    }
  }
}

// Dot products of point rows with states: row r (one warp) gives
// us[point][k] += sum_q rows[r][q] state[srow][k][q].  rows_kernel form (jobs
// of consecutive rows) for M2P, map form (one (point, state row) per row) for L2P.
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

constexpr int R64_MAX = 512;         // largest rank of the FP64 row kernels
constexpr int R64_Q = R64_MAX / 32;  // state entries per lane

__device__ __forceinline__ void row_dot(const double2* row, const double2* st, int R, int nrhs, double2* u,
                                        bool atomic) {
  const int lane = threadIdx.x & 31;
  double2 rv[R64_Q];
#pragma unroll
  for (int t = 0; t < R64_Q; ++t) {
    const int q = lane + 32 * t;
    rv[t] = q < R ? row[q] : make_double2(0.0, 0.0);
  }
  for (int k = 0; k < nrhs; ++k) {
    double2 sum = make_double2(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < R64_Q; ++t) {
      const int q = lane + 32 * t;
      if (q < R) cfma(sum, rv[t], st[(int64_t)k * R + q]);
    }
    sum = warp_sum(sum);
    if (lane == 0) add_to(u + k, sum, atomic);
  }
}

__global__ __launch_bounds__(256) void rows64_kernel(RowsArgs a) {
  const int4 job = a.jobs[blockIdx.x];
  const int warp = threadIdx.x / 32;
  const double2* st = c128(a.state) + (int64_t)job.w * a.nrhs * a.R;
  for (int i = warp; i < job.y; i += 8)
    row_dot(c128(a.rows) + (int64_t)(job.z + i) * a.R, st, a.R, a.nrhs, c128(a.us) + (int64_t)(job.x + i) * a.nrhs,
            a.atomic != 0);
}

__global__ __launch_bounds__(256) void l2p64_kernel(L2PArgs a) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= a.nrows) return;
  const int2 m = a.map[r];
  row_dot(c128(a.rows) + r * a.R, c128(a.state) + (int64_t)m.y * a.nrhs * a.R, a.R, a.nrhs,
          c128(a.us) + (int64_t)m.x * a.nrhs, false);
}

// P2M through rows, one warp per leaf: state[box][k][q] = sum_i rows[row + i][q] fs[first + i][k]
__global__ __launch_bounds__(256) void p2m64_kernel(P2MRowsArgs a) {
  const int64_t jw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (jw >= a.njobs) return;
  const int4 job = a.jobs[jw];
  const double2* rows = c128(a.rows);
  const double2* fs = c128(a.fs);
  double2* st = c128(a.state);
  for (int k = 0; k < a.nrhs; ++k) {
    double2 acc[R64_Q];
#pragma unroll
    for (int t = 0; t < R64_Q; ++t) acc[t] = make_double2(0.0, 0.0);
    for (int i = 0; i < job.y; ++i) {
      const double2 f = fs[(int64_t)(job.x + i) * a.nrhs + k];
      const double2* row = rows + (int64_t)(job.z + i) * a.R;
#pragma unroll
      for (int t = 0; t < R64_Q; ++t) {
        const int q = lane + 32 * t;
        if (q < a.R) cfma(acc[t], row[q], f);
      }
    }
#pragma unroll
    for (int t = 0; t < R64_Q; ++t) {
      const int q = lane + 32 * t;
      if (q < a.R) st[((int64_t)job.w * a.nrhs + k) * a.R + q] = acc[t];
    }
  }
}

// Near field (U lists, Eq. 1 directly): one block per target leaf, one thread
// per target point (C64_T at a time); each U-list entry's points are staged
// in shared memory in the target leaf's frame, C64_T at a time.
__global__ __launch_bounds__(C64_T) void p2p64_kernel(P2PArgs a) {
  __shared__ double3 sp[C64_T];
  __shared__ double2 sf[C64_T][C64_NR];
  const int2 lr = a.leaf_range[blockIdx.x];
  const int64_t u0 = a.u_off[blockIdx.x], u1 = a.u_off[blockIdx.x + 1];
  const double2* fs = c128(a.fs);
  double2* us = c128(a.us);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int t0 = 0; t0 < lr.y; t0 += C64_T) {
    const int t = t0 + threadIdx.x;
    const bool live = t < lr.y;
    const double3 x = point64(a.pts, a.pts_lo, lr.x + (live ? t : 0), zero);
    for (int r0 = 0; r0 < a.nrhs; r0 += C64_NR) {
      const int nr = min(C64_NR, a.nrhs - r0);
      double2 acc[C64_NR];
#pragma unroll
      for (int k = 0; k < C64_NR; ++k) acc[k] = make_double2(0.0, 0.0);
      for (int64_t e = u0; e < u1; ++e) {
        const int4 ue = a.u_src[e];
        const float4 sh = a.u_shift[e];
        for (int i0 = 0; i0 < ue.y; i0 += C64_T) {
          const int ni = min(C64_T, ue.y - i0);
          __syncthreads();
          if (threadIdx.x < ni) {
            const int64_t j = (int64_t)ue.x + i0 + threadIdx.x;
            sp[threadIdx.x] = point64(a.pts, a.pts_lo, j, sh);
#pragma unroll
            for (int k = 0; k < C64_NR; ++k)
              sf[threadIdx.x][k] = k < nr ? fs[j * a.nrhs + r0 + k] : make_double2(0.0, 0.0);
          }
          __syncthreads();
          if (live)
            for (int i = 0; i < ni; ++i) {
              const double3 v = sp[i];
              const double2 g = green64(x.x - v.x, x.y - v.y, x.z - v.z);
#pragma unroll
              for (int k = 0; k < C64_NR; ++k) cfma(acc[k], g, sf[i][k]);
            }
        }
      }
      if (live)
        for (int k = 0; k < nr; ++k) add_to(us + (int64_t)(lr.x + t) * a.nrhs + r0 + k, acc[k], false);
    }
  }
}

void check_rank(int R) {
  if (R > R64_MAX || R < 1) throw Error(-5, "representation rank of the FP64 form must be in [1, 512]");
}

}  // namespace

void launch_gemm_stage64(const GemmArgs& a, cudaStream_t s) {
  if (a.ntiles == 0) return;
  const dim3 grid((unsigned)a.ntiles, (unsigned)((a.M + GM - 1) / GM));
  gemm64_kernel<<<grid, 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_permute_in64(const float2* f, const int32_t* perm, int64_t N, int nrhs, float2* fs, cudaStream_t s) {
  const int64_t n = N * nrhs;
  permute_in64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2*)f, perm, N, nrhs, (double2*)fs);
  DFMM_CUDA(cudaGetLastError());
}

void launch_permute_out64(const float2* us, const int32_t* perm, int64_t N, int nrhs, float2* u, cudaStream_t s) {
  const int64_t n = N * nrhs;
  permute_out64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2*)us, perm, N, nrhs, (double2*)u);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2c64(const P2CArgs& a, cudaStream_t s) {
  if (a.njobs == 0) return;
  if (!a.chk64 || !a.pts_lo) throw Error(-5, "FP64 check-point evaluation needs FP64 check points");
  p2c64_kernel<<<(unsigned)a.njobs, C64_T, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_rows64(const RowsArgs& a, cudaStream_t s) {
  if (a.njobs == 0) return;
  check_rank(a.R);
  rows64_kernel<<<(unsigned)a.njobs, 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_l2p64(const L2PArgs& a, cudaStream_t s) {
  if (a.nrows == 0) return;
  check_rank(a.R);
  l2p64_kernel<<<(unsigned)((a.nrows + 7) / 8), 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2m_rows64(const P2MRowsArgs& a, cudaStream_t s) {
  if (a.njobs == 0) return;
  check_rank(a.R);
  p2m64_kernel<<<(unsigned)((a.njobs + 7) / 8), 256, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

void launch_p2p64(const P2PArgs& a, cudaStream_t s) {
  if (a.nleaves == 0) return;
  p2p64_kernel<<<(unsigned)a.nleaves, C64_T, 0, s>>>(a);
  DFMM_CUDA(cudaGetLastError());
}

}  // namespace dfmm
