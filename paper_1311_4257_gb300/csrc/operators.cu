// Plan-time formation of the translation operators (FP64 on the device).
//
// Every operator is a product of bounded factors (an orthonormal projection,
// the kernel matrix between check and equivalent points, and the inverse
// triangular factor of the source basis), formed in FP64 and rounded once to
// complex64 for the apply kernels (kept in complex128 for the FP64 form).  The
// kernel matrices and the products (a tiled FP64 complex GEMM) are the
// library's own kernels: the batched ZGEMM of the vendor library spends
// seconds on its first call in a process.
#include <cmath>

#include "operators.h"

namespace dfmm {

namespace {


__device__ __forceinline__ double2 green64(double x0, double x1, double x2, const double* y) {
  double dx = x0 - y[0], dy = x1 - y[1], dz = x2 - y[2];
  double d = sqrt(dx * dx + dy * dy + dz * dz);
  double sn, cs;
  sincospi(2.0 * d, &sn, &cs);
  return make_double2(cs / d, sn / d);
}

struct OpDev {
  int tgt, src;
  double shift[3];
};

__global__ void kmat_kernel(int kind, const OpDev* __restrict__ ops, const DevRep* __restrict__ reps, int Rt,
                            int Rs, double2* __restrict__ K) {
  const OpDev op = ops[blockIdx.x];
  const DevRep& t = reps[op.tgt];
  const DevRep& s = reps[op.src];
  const double* X = kind == kOpM2M ? t.a2 : t.b2;
  const double* Y = kind == kOpL2L ? s.a2 : s.b2;
  const double* wr = kind == kOpL2L ? s.wa2 : nullptr;
  int nx = 2 * t.r, ny = s.r;
  double2* Kk = K + (size_t)blockIdx.x * 2 * Rt * Rs;
  for (int e = threadIdx.x; e < 2 * Rt * Rs; e += blockDim.x) {
    int p = e / Rs, q = e % Rs;
    double2 v = make_double2(0.0, 0.0);
    if (p < nx && q < ny) {
      v = green64(X[3 * p] + op.shift[0], X[3 * p + 1] + op.shift[1], X[3 * p + 2] + op.shift[2], Y + 3 * q);
      if (wr) { v.x *= wr[q]; v.y *= wr[q]; }
    }
    Kk[e] = v;
  }
}

__global__ void rows_kmat_kernel(const double* __restrict__ pts, int64_t n, const double* __restrict__ Y,
                                 const double* __restrict__ wr, int r, int R, double2* __restrict__ K) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  int64_t i = e / R;
  int q = (int)(e % R);
  double2 v = make_double2(0.0, 0.0);
  if (q < r) {
    v = green64(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], Y + 3 * q);
    if (wr) { v.x *= wr[q]; v.y *= wr[q]; }
  }
  K[e] = v;
}

__global__ void to_c64_kernel(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// n FP64 results to elements [at, at + n) of out: rounded once to complex64,
// or copied as they are when the plan computes in FP64 (complex128 out)
void store_out(const double2* in, void* out, int64_t at, int64_t n, bool fp64, cudaStream_t s) {
  if (n <= 0) return;
  if (fp64) {
    DFMM_CUDA(cudaMemcpyAsync((double2*)out + at, in, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  } else {
    to_c64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, (float2*)out + at, n);
    DFMM_CUDA(cudaGetLastError());
  }
}

// Row-major complex128 products C_b = A_b op(B_b) for a batch of pointer
// triples: A_b is M x K (lda), B_b is K x N (ldb), or N x K with tb (then
// op(B) = B^T, no conjugation), C_b is M x N (ldc).  One CTA of 256 threads
// computes a 32 x 32 block of C (4 entries per thread, rows ty + 8 i), with
// K in steps of 16 through shared memory.
constexpr int ZT = 32, ZK = 16;

__global__ __launch_bounds__(256) void zgemm_kernel(const double2* const* __restrict__ Ap,
                                                    const double2* const* __restrict__ Bp, double2* const* __restrict__ Cp,
                                                    int M, int N, int K, int lda, int ldb, int ldc, bool tb) {
  __shared__ double2 As[ZT][ZK + 1];
  __shared__ double2 Bs[ZK][ZT + 1];
  const double2* A = Ap[blockIdx.z];
  const double2* B = Bp[blockIdx.z];
  double2* C = Cp[blockIdx.z];
  const int tid = threadIdx.x, tx = tid % ZT, ty = tid / ZT;
  const int row0 = blockIdx.y * ZT, col0 = blockIdx.x * ZT;
  double2 acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += ZK) {
    for (int e = tid; e < ZT * ZK; e += 256) {
      const int r = e / ZK, kk = e % ZK;
      const int gr = row0 + r, gk = k0 + kk;
      As[r][kk] = (gr < M && gk < K) ? A[(int64_t)gr * lda + gk] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < ZT * ZK; e += 256) {
      int kk, c;
      if (tb) { c = e / ZK; kk = e % ZK; } else { kk = e / ZT; c = e % ZT; }
      const int gk = k0 + kk, gc = col0 + c;
      double2 v = make_double2(0.0, 0.0);
      if (gk < K && gc < N) v = tb ? B[(int64_t)gc * ldb + gk] : B[(int64_t)gk * ldb + gc];
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZK; ++kk) {
      const double2 b = Bs[kk][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double2 a = As[ty + 8 * i][kk];
        acc[i].x = fma(a.x, b.x, fma(-a.y, b.y, acc[i].x));
        acc[i].y = fma(a.x, b.y, fma(a.y, b.x, acc[i].y));
      }
    }
    __syncthreads();
  }
  const int c = col0 + tx;
  if (c < N)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = row0 + ty + 8 * i;
      if (r < M) C[(int64_t)r * ldc + c] = acc[i];
    }
}

void zgemm(const double2* const* A, const double2* const* B, double2* const* C, int batch, int M, int N, int K,
           int lda, int ldb, int ldc, bool tb, cudaStream_t s) {
  if (batch <= 0 || M <= 0 || N <= 0) return;
  const dim3 grid((unsigned)((N + ZT - 1) / ZT), (unsigned)((M + ZT - 1) / ZT), (unsigned)batch);
  if (grid.y > 65535u || grid.z > 65535u) throw Error(-5, "operator formation: product too large for one launch");
  zgemm_kernel<<<grid, 256, 0, s>>>(A, B, C, M, N, K, lda, ldb, ldc, tb);
  DFMM_CUDA(cudaGetLastError());
}

// one product through a device pointer triple held in `ar`
void zgemm1(const double2* A, const double2* B, double2* C, int M, int N, int K, int lda, int ldb, int ldc, bool tb,
            DevArena& ar, cudaStream_t s) {
  const void* h[3] = {A, B, C};
  const void** d = ar.alloc<const void*>(3);
  DFMM_CUDA(cudaMemcpyAsync(d, h, sizeof h, cudaMemcpyHostToDevice, s));
  zgemm((const double2* const*)d, (const double2* const*)(d + 1), (double2* const*)(d + 2), 1, M, N, K, lda, ldb,
        ldc, tb, s);
  DFMM_CUDA(cudaStreamSynchronize(s));   // the pointer triple is released with the caller's mark
}

std::vector<double2> pad_matrix(const std::vector<cd>& M, int rows, int cols, int Rrows, int Rcols,
                                const double* colscale) {
  std::vector<double2> out((size_t)Rrows * Rcols, make_double2(0, 0));
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) {
      cd v = M[(size_t)i * cols + j];
      if (colscale) v *= colscale[j];
      out[(size_t)i * Rcols + j] = make_double2(v.real(), v.imag());
    }
  return out;
}

}  // namespace

DevRep upload_rep(const Rep& rep, int R, DevArena& ar, cudaStream_t s) {
  DevRep d;
  int r = rep.r;
  d.r = r;
  d.R = R;
  d.b2 = ar.alloc<double>(6 * r);
  d.a2 = ar.alloc<double>(6 * r);
  d.wa2 = ar.alloc<double>(2 * r);
  d.PoutH = ar.alloc<double2>((size_t)R * 2 * R);
  d.PinH = ar.alloc<double2>((size_t)R * 2 * R);
  d.Ro_inv = ar.alloc<double2>((size_t)R * R);
  d.Ri_inv = ar.alloc<double2>((size_t)R * R);
  // Qo^H W (r x 2r) and Qi^H (r x 2r), transposed conjugates of the 2r x r Q's
  std::vector<cd> QoH((size_t)r * 2 * r), QiH((size_t)r * 2 * r);
  for (int p = 0; p < 2 * r; ++p)
    for (int q = 0; q < r; ++q) {
      QoH[(size_t)q * 2 * r + p] = std::conj(rep.Qo[(size_t)p * r + q]);
      QiH[(size_t)q * 2 * r + p] = std::conj(rep.Qi[(size_t)p * r + q]);
    }
  auto po = pad_matrix(QoH, r, 2 * r, R, 2 * R, rep.wa2.data());
  auto pi = pad_matrix(QiH, r, 2 * r, R, 2 * R, nullptr);
  auto ro = pad_matrix(rep.Ro_inv, r, r, R, R, nullptr);
  auto ri = pad_matrix(rep.Ri_inv, r, r, R, R, nullptr);
  // PoutH / PinH are R x 2R but the padded column index must follow 2R:
  // pad_matrix placed column j of the r x 2r block at column j of 2R; correct.
  DFMM_CUDA(cudaMemcpyAsync(d.b2, rep.b2.data(), 6 * r * 8, cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaMemcpyAsync(d.a2, rep.a2.data(), 6 * r * 8, cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaMemcpyAsync(d.wa2, rep.wa2.data(), 2 * r * 8, cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaMemcpyAsync(d.PoutH, po.data(), po.size() * 16, cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaMemcpyAsync(d.PinH, pi.data(), pi.size() * 16, cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaMemcpyAsync(d.Ro_inv, ro.data(), ro.size() * 16, cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaMemcpyAsync(d.Ri_inv, ri.data(), ri.size() * 16, cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaStreamSynchronize(s));
  return d;
}

void form_ops(OpKind kind, const std::vector<OpSpec>& ops, const std::vector<DevRep>& reps, int Rt, int Rs,
              void* out, bool fp64, DevArena& ar, cudaStream_t s) {
  if (ops.empty()) return;
  ArenaMark mark(ar);
  DevRep* d_reps = ar.alloc<DevRep>(reps.size());
  DFMM_CUDA(cudaMemcpyAsync(d_reps, reps.data(), reps.size() * sizeof(DevRep), cudaMemcpyHostToDevice, s));
  size_t per_op = (size_t)(2 * Rt * Rs + Rt * Rs + Rt * Rs) * sizeof(double2);
  int64_t batch = std::max<int64_t>(1, std::min<int64_t>((int64_t)ops.size(), (int64_t)((768ull << 20) / per_op)));
  double2* K = ar.alloc<double2>((size_t)batch * 2 * Rt * Rs);
  double2* T1 = ar.alloc<double2>((size_t)batch * Rt * Rs);
  double2* T2 = ar.alloc<double2>((size_t)batch * Rt * Rs);
  OpDev* d_ops = ar.alloc<OpDev>(batch);
  const double2** pA = ar.alloc<const double2*>(batch);
  const double2** pB = ar.alloc<const double2*>(batch);
  double2** pC = ar.alloc<double2*>(batch);
  std::vector<OpDev> h_ops(batch);
  std::vector<const double2*> hA(batch), hB(batch);
  std::vector<double2*> hC(batch);
  for (size_t start = 0; start < ops.size(); start += batch) {
    int nb = (int)std::min<size_t>(batch, ops.size() - start);
    for (int k = 0; k < nb; ++k) {
      const OpSpec& o = ops[start + k];
      h_ops[k].tgt = o.tgt_rep;
      h_ops[k].src = o.src_rep;
      for (int d = 0; d < 3; ++d) h_ops[k].shift[d] = o.shift[d];
    }
    DFMM_CUDA(cudaMemcpyAsync(d_ops, h_ops.data(), nb * sizeof(OpDev), cudaMemcpyHostToDevice, s));
    kmat_kernel<<<nb, 256, 0, s>>>(kind, d_ops, d_reps, Rt, Rs, K);
    DFMM_CUDA(cudaGetLastError());
    // T1 = L (Rt x 2Rt) K (2Rt x Rs)
    for (int k = 0; k < nb; ++k) {
      const DevRep& t = reps[ops[start + k].tgt_rep];
      hA[k] = kind == kOpM2M ? t.PoutH : t.PinH;
      hB[k] = K + (size_t)k * 2 * Rt * Rs;
      hC[k] = T1 + (size_t)k * Rt * Rs;
    }
    DFMM_CUDA(cudaMemcpyAsync(pA, hA.data(), nb * sizeof(void*), cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(pB, hB.data(), nb * sizeof(void*), cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(pC, hC.data(), nb * sizeof(void*), cudaMemcpyHostToDevice, s));
    zgemm(pA, pB, pC, nb, Rt, Rs, 2 * Rt, 2 * Rt, Rs, Rs, false, s);
    // T2 = T1 (Rt x Rs) Rinv_s (Rs x Rs)
    DFMM_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nb; ++k) {
      const DevRep& sr = reps[ops[start + k].src_rep];
      hA[k] = T1 + (size_t)k * Rt * Rs;
      hB[k] = kind == kOpL2L ? sr.Ri_inv : sr.Ro_inv;
      hC[k] = T2 + (size_t)k * Rt * Rs;
    }
    DFMM_CUDA(cudaMemcpyAsync(pA, hA.data(), nb * sizeof(void*), cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(pB, hB.data(), nb * sizeof(void*), cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(pC, hC.data(), nb * sizeof(void*), cudaMemcpyHostToDevice, s));
    zgemm(pA, pB, pC, nb, Rt, Rs, Rs, Rs, Rs, Rs, false, s);
    store_out(T2, out, (int64_t)start * Rt * Rs, (int64_t)nb * Rt * Rs, fp64, s);
    DFMM_CUDA(cudaStreamSynchronize(s));
  }
}

void form_rows(bool incoming, const DevRep& rep, const double* d_pts, int64_t n, void* out, bool fp64,
               DevArena& ar, cudaStream_t s) {
  if (n <= 0) return;
  ArenaMark mark(ar);
  int R = rep.R;
  int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)((512ull << 20) / (2 * R * sizeof(double2)))));
  double2* K = ar.alloc<double2>((size_t)chunk * R);
  double2* T = ar.alloc<double2>((size_t)chunk * R);
  for (int64_t st = 0; st < n; st += chunk) {
    int64_t m = std::min(chunk, n - st);
    int64_t ne = m * R;
    rows_kmat_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(d_pts + 3 * st, m, incoming ? rep.a2 : rep.b2,
                                                                   incoming ? rep.wa2 : nullptr, rep.r, R, K);
    const double2* Rinv = incoming ? rep.Ri_inv : rep.Ro_inv;
    // row-major T (m x R) = K (m x R) Rinv (R x R)
    zgemm1(K, Rinv, T, (int)m, R, R, R, R, R, false, ar, s);
    store_out(T, out, st * R, ne, fp64, s);
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
}

void form_p2m_rows(const DevRep& rep, const double* d_pts, int64_t n, void* out, bool fp64, DevArena& ar,
                   cudaStream_t s) {
  if (n <= 0) return;
  ArenaMark mark(ar);
  const int R = rep.R, K2 = 2 * R;
  int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)((512ull << 20) / (3 * R * sizeof(double2)))));
  double2* K = ar.alloc<double2>((size_t)chunk * K2);
  double2* T = ar.alloc<double2>((size_t)chunk * R);
  for (int64_t st = 0; st < n; st += chunk) {
    const int64_t m = std::min(chunk, n - st);
    const int64_t ne = m * K2;
    // K (m x 2R, row-major): G(y_i - c, a2_p) for the 2r check points, zero padded
    rows_kmat_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(d_pts + 3 * st, m, rep.a2, nullptr, 2 * rep.r, K2,
                                                                   K);
    // row-major T (m x R) = K (m x 2R) PoutH^T, PoutH = Qo^H W (R x 2R, row-major)
    zgemm1(K, rep.PoutH, T, (int)m, R, K2, K2, K2, R, true, ar, s);
    store_out(T, out, st * R, m * R, fp64, s);
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dfmm
