// Pivot selection of the skeleton construction (Sec. 2.1, the randomized
// sampling and pivoted QR that pick the equivalent and check points of
// Eq. 2) on the GPU, for a batch of representation types at once.
//
//  * wkmat_kernel: weighted kernel matrices, |x| G(x, y) with the host
//    formula (cos 2 pi d, sin 2 pi d) / d in FP64.
//  * sign_kernel / sketch_kernel: Z = Omega A with Omega the +-1 sketch drawn
//    by SplitMix64 (Steele, Lea and Flood 2014) at the same counters as the
//    host (draw k = q S_X + i + 1 of the type's sketch seed, sign = top bit);
//    each Z entry is summed over i in ascending order, as on the host.
//  * pqr_coop_kernel: column-pivoted Householder QR of several matrices at
//    once (row-major complex128 in global memory), each spread over several
//    CTAs of one cooperative launch (GB300 runs FP64 at a few operations per
//    clock and SM, so one SM per matrix would take ten times longer).  Every
//    step takes the column of largest remaining norm (the first one among
//    equal norms), swaps it to position k, reflects the trailing columns and
//    recomputes their norms below row k, like the host form; it stops when
//    the largest norm is <= tol |R_00|, vanishes, or after kmax steps.  The
//    CTAs meet at grid syncs only (the cooperative launch keeps them all
//    resident), two per step.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "skeleton.h"
#include "tree.h"

namespace dfmm {

namespace {

namespace cg = cooperative_groups;

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr double kTwoPi = 6.283185307179586;

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// out[p][q] = w * G(P_p, Q_q), w = |P_p| (w_rows) or |Q_q| (else); G = e^{2 pi i d} / d
__global__ void wkmat_kernel(const double* __restrict__ P, int np, const double* __restrict__ Q, int nq,
                             const double* __restrict__ w, bool w_rows, double2* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)np * nq) return;
  const int p = (int)(e / nq), q = (int)(e % nq);
  const double dx = P[3 * p] - Q[3 * q], dy = P[3 * p + 1] - Q[3 * q + 1], dz = P[3 * p + 2] - Q[3 * q + 2];
  const double d = sqrt(dx * dx + dy * dy + dz * dz);
  double sn, cs;
  sincos(kTwoPi * d, &sn, &cs);
  const double wt = w_rows ? w[p] : w[q];
  out[e] = make_double2(wt * (cs / d), wt * (sn / d));
}

// bits[q][i / 32] bit i % 32 = 1 where draw (q S_X + i + 1) has its top bit set (sign -1)
__global__ void sign_kernel(uint64_t seed, int s, int SX, uint32_t* __restrict__ bits) {
  const int words = (SX + 31) / 32;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * words) return;
  const int q = (int)(e / words), wd = (int)(e % words);
  uint32_t b = 0;
  for (int t = 0; t < 32; ++t) {
    const int i = 32 * wd + t;
    if (i >= SX) break;
    const uint64_t kk = (uint64_t)q * SX + i + 1;
    if (splitmix64_dev(seed + kk * kGamma) >> 63) b |= 1u << t;
  }
  bits[e] = b;
}

constexpr int SK_QB = 8;   // sketch rows per thread

// Z[q][j] = sum_i sign(q, i) A[i][j], i ascending; thread: column j, SK_QB rows q
__global__ __launch_bounds__(128) void sketch_kernel(const double2* __restrict__ A, int SX, int SY, int s,
                                                     const uint32_t* __restrict__ bits, double2* __restrict__ Z) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int q0 = blockIdx.y * SK_QB;
  if (j >= SY) return;
  const int words = (SX + 31) / 32;
  double2 z[SK_QB];
#pragma unroll
  for (int u = 0; u < SK_QB; ++u) z[u] = make_double2(0.0, 0.0);
  for (int w0 = 0; w0 < words; ++w0) {
    uint32_t b[SK_QB];
#pragma unroll
    for (int u = 0; u < SK_QB; ++u) b[u] = q0 + u < s ? bits[(int64_t)(q0 + u) * words + w0] : 0u;
    const int i1 = min(SX, 32 * w0 + 32);
    for (int i = 32 * w0; i < i1; ++i) {
      const double2 a = A[(int64_t)i * SY + j];
      const int t = i & 31;
#pragma unroll
      for (int u = 0; u < SK_QB; ++u) {
        if ((b[u] >> t) & 1u) {
          z[u].x = __dsub_rn(z[u].x, a.x);
          z[u].y = __dsub_rn(z[u].y, a.y);
        } else {
          z[u].x = __dadd_rn(z[u].x, a.x);
          z[u].y = __dadd_rn(z[u].y, a.y);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < SK_QB; ++u)
    if (q0 + u < s) Z[(int64_t)(q0 + u) * SY + j] = z[u];
}

// out[q][c] = in[q][cols[c]]
__global__ void gather_cols_kernel(const double2* __restrict__ in, int rows, int ld_in, const int* __restrict__ cols,
                                   int ncols, double2* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * ncols) return;
  const int q = (int)(e / ncols), c = (int)(e % ncols);
  out[e] = in[(int64_t)q * ld_in + cols[c]];
}

struct QrTask {
  double2* A;      // m x n row-major (destroyed)
  int m, n;
  int kmax;
  double tol;
  int* cols;       // [n] scratch: original index of the column at each position
  double* norms;   // [n] scratch: squared norms of the trailing columns below row k
  double* cand_s;  // [G] scratch: each CTA's largest column norm
  int* cand_j;     // [G] scratch: and its position
  int* piv;        // [kmax] out: original column indices
  double* diag;    // [kmax] out: the chosen column norms
  int* nsteps;     // out
  int cta0, G;     // the task's CTAs: cta0 .. cta0 + G - 1
};

constexpr int QR_T = 1024;    // threads per CTA: 32 warps
constexpr int QR_CH = 4;      // 32-column chunks per column group (128 columns)
constexpr int QR_RP = 8;      // row phases: warp w takes chunk w % 4 and rows k + (w / 4) + 8 t
constexpr int QR_GROUP = 32 * QR_CH;

// Column-pivoted QR of several matrices at once; a cooperative launch in
// which task t owns CTAs cta0 .. cta0 + G - 1.  Column groups of 128 are dealt
// round-robin to the task's CTAs; inside a CTA, 8 warps share each 32-column
// chunk, one row phase each, and the partial sums meet in shared memory in a
// fixed order.  Per step: the task's CTAs combine the per-CTA column maxima
// (largest norm, then lowest position), swap the pivot column into place
// (rows dealt over the CTAs), sync the grid, each rebuild the Householder
// vector from column k, reflect their own columns, recompute those columns'
// norms and their own maximum for the next step, and sync the grid again.
// Every CTA runs the same number of steps (the largest kmax) so that all meet
// at every grid sync; finished tasks idle through them.
__global__ __launch_bounds__(QR_T, 1) void pqr_coop_kernel(const QrTask* __restrict__ tasks, const int* __restrict__ cta_task,
                                                        int kmax_all) {
  extern __shared__ double2 v[];   // Householder vector, m entries
  __shared__ double2 part[QR_RP][QR_CH][32];
  __shared__ double red_s[QR_T / 32];
  __shared__ int red_j[QR_T / 32];
  __shared__ double s_sc, s_best, s_r00;
  __shared__ int s_jb, s_state;   // state: 0 running, 1 stopped
  cg::grid_group grid = cg::this_grid();
  const QrTask t = tasks[cta_task[blockIdx.x]];
  const int g = blockIdx.x - t.cta0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cc = warp % QR_CH, rp = warp / QR_CH;
  const int m = t.m, n = t.n;
  const int ngroups = (n + QR_GROUP - 1) / QR_GROUP;
  const int kmax = min(t.kmax, min(m, n));
  double2* A = t.A;

  // this CTA's largest column norm over its columns j >= k0 (first position on ties)
  auto local_max = [&](int k0) {
    double best = -1.0;
    int jb = n;
    for (int gi = g; gi < ngroups; gi += t.G)
      for (int j = gi * QR_GROUP + tid; j < min(n, gi * QR_GROUP + QR_GROUP); j += QR_T)
        if (j >= k0) {
          const double sv = sqrt(t.norms[j]);
          if (sv > best) { best = sv; jb = j; }
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
      if (ob > best || (ob == best && oj < jb)) { best = ob; jb = oj; }
    }
    if (lane == 0) { red_s[warp] = best; red_j[warp] = jb; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < QR_T / 32; ++w)
        if (red_s[w] > red_s[0] || (red_s[w] == red_s[0] && red_j[w] < red_j[0])) { red_s[0] = red_s[w]; red_j[0] = red_j[w]; }
      t.cand_s[g] = red_s[0];
      t.cand_j[g] = red_j[0];
    }
    __syncthreads();
  };

  // squared norms of this CTA's columns over rows r0 .. m-1, 8 row phases per chunk
  auto column_norms = [&](int gi, int r0) {
    const int j = gi * QR_GROUP + 32 * cc + lane;
    double nn = 0.0;
    if (j < n)
      for (int i = r0 + rp; i < m; i += QR_RP) {
        const double2 a = A[(int64_t)i * n + j];
        nn += a.x * a.x + a.y * a.y;
      }
    part[rp][cc][lane].x = nn;
    __syncthreads();
    if (rp == 0 && j < n) {
      double s = 0.0;
      for (int q = 0; q < QR_RP; ++q) s += part[q][cc][lane].x;
      t.norms[j] = s;
    }
    __syncthreads();
  };

  if (tid == 0) s_state = 0;
  for (int gi = g; gi < ngroups; gi += t.G) {
    for (int j = gi * QR_GROUP + tid; j < min(n, gi * QR_GROUP + QR_GROUP); j += QR_T) t.cols[j] = j;
    column_norms(gi, 0);
  }
  local_max(0);
  grid.sync();

  for (int k = 0; k < kmax_all; ++k) {
    // every thread reads the task's state before thread 0 may change it below, so
    // that all threads of the CTA take the same branches (and barriers)
    const int state0 = s_state;
    __syncthreads();
    const bool active = k < kmax && state0 == 0;
    if (active) {
      if (tid == 0) {
        double best = t.cand_s[0];
        int jb = t.cand_j[0];
        for (int q = 1; q < t.G; ++q)
          if (t.cand_s[q] > best || (t.cand_s[q] == best && t.cand_j[q] < jb)) { best = t.cand_s[q]; jb = t.cand_j[q]; }
        if (k == 0) s_r00 = best;
        s_best = best;
        s_jb = jb;
        if (best <= t.tol * s_r00 || best == 0.0 || jb >= n) s_state = 1;
      }
    }
    __syncthreads();
    const bool go = active && s_state == 0;
    if (go) {
      const int jb = s_jb;
      if (jb != k)   // rows dealt over the task's CTAs
        for (int i = g * QR_T + tid; i < m; i += t.G * QR_T) {
          const double2 x = A[(int64_t)i * n + k];
          A[(int64_t)i * n + k] = A[(int64_t)i * n + jb];
          A[(int64_t)i * n + jb] = x;
        }
      if (g == 0 && tid == 0) {
        if (jb != k) {
          const int c = t.cols[k];
          t.cols[k] = t.cols[jb];
          t.cols[jb] = c;
        }
        t.piv[k] = t.cols[k];
        t.diag[k] = s_best;
      }
    }
    if (active && !go && g == 0 && tid == 0) *t.nsteps = k;
    grid.sync();
    if (go) {
      for (int i = k + tid; i < m; i += QR_T) v[i - k] = A[(int64_t)i * n + k];
      __syncthreads();
      if (tid == 0) {
        // v = A[k:, k] + phase(A_kk) |A[k:, k]| e_k
        const double best = s_best;
        const double2 alpha = v[0];
        const double aa = hypot(alpha.x, alpha.y);
        const double px = aa > 0.0 ? alpha.x / aa : 1.0, py = aa > 0.0 ? alpha.y / aa : 0.0;
        v[0] = make_double2(alpha.x + px * best, alpha.y + py * best);
        double vn = 0.0;
        for (int i = 0; i < m - k; ++i) vn += v[i].x * v[i].x + v[i].y * v[i].y;
        s_sc = 2.0 / vn;
      }
      __syncthreads();
      const double sc = s_sc;
      for (int gi = g; gi < ngroups; gi += t.G) {
        if (gi * QR_GROUP + QR_GROUP <= k + 1) continue;   // no column of the group beyond k (CTA-uniform)
        const int j = gi * QR_GROUP + 32 * cc + lane;
        const bool live = j > k && j < n;
        // w_j = v^H A[k:, j]: partial sums per row phase, added in phase order
        double wr = 0.0, wi = 0.0;
        if (live)
          for (int i = k + rp; i < m; i += QR_RP) {
            const double2 a = A[(int64_t)i * n + j];
            const double2 vv = v[i - k];
            wr += vv.x * a.x + vv.y * a.y;
            wi += vv.x * a.y - vv.y * a.x;
          }
        part[rp][cc][lane] = make_double2(wr, wi);
        __syncthreads();
        wr = 0.0;
        wi = 0.0;
        for (int q = 0; q < QR_RP; ++q) {
          wr += part[q][cc][lane].x;
          wi += part[q][cc][lane].y;
        }
        __syncthreads();
        // A[k:, j] -= (2 / |v|^2) v w_j; the norm below row k
        double nn = 0.0;
        if (live)
          for (int i = k + rp; i < m; i += QR_RP) {
            double2 a = A[(int64_t)i * n + j];
            const double vx = v[i - k].x * sc, vy = v[i - k].y * sc;
            a.x -= vx * wr - vy * wi;
            a.y -= vx * wi + vy * wr;
            A[(int64_t)i * n + j] = a;
            if (i > k) nn += a.x * a.x + a.y * a.y;
          }
        part[rp][cc][lane].x = nn;
        __syncthreads();
        if (rp == 0 && live) {
          double ss = 0.0;
          for (int q = 0; q < QR_RP; ++q) ss += part[q][cc][lane].x;
          t.norms[j] = ss;
        }
        __syncthreads();
      }
      local_max(k + 1);
    }
    grid.sync();
  }
  if (g == 0 && tid == 0 && s_state == 0) *t.nsteps = kmax;
}

unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

template <class T>
T* upload(DevArena& ar, const std::vector<T>& h, cudaStream_t s) {
  T* d = ar.alloc<T>((int64_t)h.size());
  if (!h.empty()) DFMM_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

// Cooperative launches of pqr_coop_kernel over `tasks` (up to one CTA per SM
// in all, shared out by column groups); results copied back into the host vectors.
void run_qr(std::vector<QrTask>& tasks, std::vector<std::vector<int>*>& piv, std::vector<std::vector<double>*>& diag,
            DevArena& ar, cudaStream_t s) {
  if (tasks.empty()) return;
  int dev = 0, nsm = 0, coop = 0;
  DFMM_CUDA(cudaGetDevice(&dev));
  DFMM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  DFMM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) throw Error(-5, "pivoted QR on the device needs cooperative launches");
  int mmax = 1;
  for (auto& t : tasks) mmax = std::max(mmax, t.m);
  const size_t smem = (size_t)mmax * sizeof(double2);
  if (smem > 160 * 1024) throw Error(-5, "pivoted QR: too many rows for the device form");
  DFMM_CUDA(cudaFuncSetAttribute(pqr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  DFMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pqr_coop_kernel, QR_T, smem));
  const int resident = std::max(1, per_sm) * nsm;
  for (size_t t0 = 0; t0 < tasks.size(); t0 += (size_t)resident) {
    const size_t t1 = std::min(tasks.size(), t0 + (size_t)resident);
    const int nt = (int)(t1 - t0);
    // CTAs per task: a share of the resident CTAs, at most one per column group
    std::vector<int> cta_task;
    int kmax_all = 0;
    for (size_t k = t0; k < t1; ++k) {
      QrTask& t = tasks[k];
      const int ngroups = (t.n + QR_GROUP - 1) / QR_GROUP;
      t.G = std::max(1, std::min(ngroups, resident / nt));
      t.cta0 = (int)cta_task.size();
      t.cand_s = ar.alloc<double>(t.G);
      t.cand_j = ar.alloc<int>(t.G);
      for (int q = 0; q < t.G; ++q) cta_task.push_back((int)(k - t0));
      kmax_all = std::max(kmax_all, std::min(t.kmax, std::min(t.m, t.n)));
    }
    std::vector<QrTask> part(tasks.begin() + t0, tasks.begin() + t1);
    QrTask* dt = upload(ar, part, s);
    int* dct = upload(ar, cta_task, s);
    void* args[] = {(void*)&dt, (void*)&dct, (void*)&kmax_all};
    DFMM_CUDA(cudaLaunchCooperativeKernel((const void*)pqr_coop_kernel, dim3((unsigned)cta_task.size()), dim3(QR_T),
                                          args, smem, s));
    DFMM_CUDA(cudaGetLastError());
    DFMM_CUDA(cudaStreamSynchronize(s));
  }
  for (size_t k = 0; k < tasks.size(); ++k) {
    int ns = 0;
    DFMM_CUDA(cudaMemcpy(&ns, tasks[k].nsteps, sizeof(int), cudaMemcpyDeviceToHost));
    piv[k]->resize(ns);
    if (diag[k]) diag[k]->resize(ns);
    if (ns > 0) {
      DFMM_CUDA(cudaMemcpy(piv[k]->data(), tasks[k].piv, ns * sizeof(int), cudaMemcpyDeviceToHost));
      if (diag[k]) DFMM_CUDA(cudaMemcpy(diag[k]->data(), tasks[k].diag, ns * sizeof(double), cudaMemcpyDeviceToHost));
    }
  }
}

QrTask make_task(double2* A, int m, int n, int kmax, DevArena& ar) {
  QrTask t{};
  t.A = A;
  t.m = m;
  t.n = n;
  t.kmax = std::min(kmax, std::min(m, n));
  t.tol = 0.0;
  t.cols = ar.alloc<int>(n);
  t.norms = ar.alloc<double>(n);
  t.piv = ar.alloc<int>(std::max(1, t.kmax));
  t.diag = ar.alloc<double>(std::max(1, t.kmax));
  t.nsteps = ar.alloc<int>(1);
  return t;
}

struct StreamGuard {
  cudaStream_t s = nullptr;
  StreamGuard() { DFMM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
  ~StreamGuard() { cudaStreamDestroy(s); }
};

}  // namespace

void sketch_pivots_device(std::vector<SketchJob>& jobs, const SkelParams& prm) {
  if (jobs.empty()) return;
  StreamGuard sg;
  cudaStream_t s = sg.s;
  DevArena keep;   // sketches and QR scratch of every job
  const int rows = prm.sketch;
  std::vector<QrTask> tasks;
  std::vector<std::vector<int>*> piv;
  std::vector<std::vector<double>*> diag;
  constexpr size_t kChunk = 16;   // kernel matrices alive at once (64 MB each at the default sizes)
  for (size_t c0 = 0; c0 < jobs.size(); c0 += kChunk) {
    DevArena tmp;
    for (size_t k = c0; k < std::min(jobs.size(), c0 + kChunk); ++k) {
      const Samples& sm = *jobs[k].sm;
      const double* dX = upload(tmp, sm.X, s);
      const double* dY = upload(tmp, sm.Y, s);
      const double* dW = upload(tmp, sm.Wx, s);
      double2* A = tmp.alloc<double2>((int64_t)sm.SX * sm.SY);
      wkmat_kernel<<<blocks_for((int64_t)sm.SX * sm.SY, 256), 256, 0, s>>>(dX, sm.SX, dY, sm.SY, dW, true, A);
      DFMM_CUDA(cudaGetLastError());
      const int words = (sm.SX + 31) / 32;
      uint32_t* bits = tmp.alloc<uint32_t>((int64_t)rows * words);
      sign_kernel<<<blocks_for((int64_t)rows * words, 256), 256, 0, s>>>(sm.sketch_seed, rows, sm.SX, bits);
      DFMM_CUDA(cudaGetLastError());
      double2* Z = keep.alloc<double2>((int64_t)rows * sm.SY);
      const dim3 grid(blocks_for(sm.SY, 128), blocks_for(rows, SK_QB));
      sketch_kernel<<<grid, 128, 0, s>>>(A, sm.SX, sm.SY, rows, bits, Z);
      DFMM_CUDA(cudaGetLastError());
      tasks.push_back(make_task(Z, rows, sm.SY, rows, keep));
      piv.push_back(&jobs[k].piv);
      diag.push_back(&jobs[k].diag);
    }
    DFMM_CUDA(cudaStreamSynchronize(s));   // before the chunk's kernel matrices are freed
  }
  run_qr(tasks, piv, diag, keep, s);
}

void check_pivots_device(std::vector<CheckJob>& jobs) {
  if (jobs.empty()) return;
  StreamGuard sg;
  cudaStream_t s = sg.s;
  DevArena ar;
  std::vector<double2*> A2(jobs.size());
  std::vector<QrTask> tasks;
  std::vector<std::vector<int>*> piv;
  std::vector<std::vector<double>*> nodiag(jobs.size(), nullptr);
  for (size_t k = 0; k < jobs.size(); ++k) {
    const Samples& sm = *jobs[k].sm;
    const int r = jobs[k].r;
    if (r < 1) throw Error(-5, "check-point selection needs a positive rank");
    const double* dX = upload(ar, sm.X, s);
    const double* dW = upload(ar, sm.Wx, s);
    const double* dB = upload(ar, jobs[k].b, s);
    // A2[q][i] = |x_i| G(x_i, b_q), r x SX (weights on the columns)
    A2[k] = ar.alloc<double2>((int64_t)r * sm.SX);
    wkmat_kernel<<<blocks_for((int64_t)r * sm.SX, 256), 256, 0, s>>>(dB, r, dX, sm.SX, dW, false, A2[k]);
    DFMM_CUDA(cudaGetLastError());
    double2* A2c = ar.alloc<double2>((int64_t)r * sm.SX);
    DFMM_CUDA(cudaMemcpyAsync(A2c, A2[k], (size_t)r * sm.SX * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    tasks.push_back(make_task(A2c, r, sm.SX, r, ar));
    piv.push_back(&jobs[k].p1);
  }
  run_qr(tasks, piv, nodiag, ar, s);
  tasks.clear();
  piv.clear();
  for (size_t k = 0; k < jobs.size(); ++k) {
    const Samples& sm = *jobs[k].sm;
    const int r = jobs[k].r;
    if ((int)jobs[k].p1.size() != r) throw Error(-5, "check-point selection failed");
    const std::vector<int> rest = rest_of(jobs[k].p1, sm.SX);
    const int* dR = upload(ar, rest, s);
    double2* A3 = ar.alloc<double2>((int64_t)r * rest.size());
    gather_cols_kernel<<<blocks_for((int64_t)r * rest.size(), 256), 256, 0, s>>>(A2[k], r, sm.SX, dR,
                                                                                    (int)rest.size(), A3);
    DFMM_CUDA(cudaGetLastError());
    tasks.push_back(make_task(A3, r, (int)rest.size(), r, ar));
    piv.push_back(&jobs[k].p2);
  }
  run_qr(tasks, piv, nodiag, ar, s);
}

}  // namespace dfmm
