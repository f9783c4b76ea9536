// Plan-time formation of the translation operators (FP64 on the device).
//
// Every operator is a product of bounded factors (an orthonormal projection,
// the kernel matrix between check and equivalent points, and the inverse
// triangular factor of the source basis), formed in FP64 and rounded once to
// complex64 for the apply kernels (kept in complex128 for the FP64 form).  The kernel matrices are evaluated by a
// hand-written FP64 kernel; the two small products per operator are plain
// batched ZGEMMs (cuBLAS).
#include <cmath>

#include "operators.h"

namespace dfmm {

namespace {

#define DFMM_CUBLAS(call)                                                             \
  do {                                                                                \
    cublasStatus_t st_ = (call);                                                      \
    if (st_ != CUBLAS_STATUS_SUCCESS) throw Error(-4, std::string(#call) + " failed"); \
  } while (0)

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

// row-major C (m x n) = A (m x k) B (k x n), batched through pointer arrays
void gemm_rm_batched(cublasHandle_t cb, int m, int n, int k, const double2** A, const double2** B, double2** C,
                     int batch) {
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  DFMM_CUBLAS(cublasZgemmBatched(cb, CUBLAS_OP_N, CUBLAS_OP_N, n, m, k, &one, (const cuDoubleComplex**)B, n,
                                 (const cuDoubleComplex**)A, k, &zero, (cuDoubleComplex**)C, n, batch));
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
              void* out, bool fp64, cublasHandle_t cb, DevArena& ar, cudaStream_t s) {
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
  DFMM_CUBLAS(cublasSetStream(cb, s));
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
    gemm_rm_batched(cb, Rt, Rs, 2 * Rt, pA, pB, pC, nb);
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
    gemm_rm_batched(cb, Rt, Rs, Rs, pA, pB, pC, nb);
    store_out(T2, out, (int64_t)start * Rt * Rs, (int64_t)nb * Rt * Rs, fp64, s);
    DFMM_CUDA(cudaStreamSynchronize(s));
  }
}

void form_rows(bool incoming, const DevRep& rep, const double* d_pts, int64_t n, void* out, bool fp64,
               cublasHandle_t cb, DevArena& ar, cudaStream_t s) {
  if (n <= 0) return;
  ArenaMark mark(ar);
  int R = rep.R;
  int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)((512ull << 20) / (2 * R * sizeof(double2)))));
  double2* K = ar.alloc<double2>((size_t)chunk * R);
  double2* T = ar.alloc<double2>((size_t)chunk * R);
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  DFMM_CUBLAS(cublasSetStream(cb, s));
  for (int64_t st = 0; st < n; st += chunk) {
    int64_t m = std::min(chunk, n - st);
    int64_t ne = m * R;
    rows_kmat_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(d_pts + 3 * st, m, incoming ? rep.a2 : rep.b2,
                                                                   incoming ? rep.wa2 : nullptr, rep.r, R, K);
    const double2* Rinv = incoming ? rep.Ri_inv : rep.Ro_inv;
    // row-major T (m x R) = K (m x R) Rinv (R x R)
    DFMM_CUBLAS(cublasZgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, R, (int)m, R, &one, (const cuDoubleComplex*)Rinv, R,
                            (const cuDoubleComplex*)K, R, &zero, (cuDoubleComplex*)T, R));
    store_out(T, out, st * R, ne, fp64, s);
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
}

void form_p2m_rows(const DevRep& rep, const double* d_pts, int64_t n, void* out, bool fp64, cublasHandle_t cb,
                   DevArena& ar, cudaStream_t s) {
  if (n <= 0) return;
  ArenaMark mark(ar);
  const int R = rep.R, K2 = 2 * R;
  int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)((512ull << 20) / (3 * R * sizeof(double2)))));
  double2* K = ar.alloc<double2>((size_t)chunk * K2);
  double2* T = ar.alloc<double2>((size_t)chunk * R);
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  DFMM_CUBLAS(cublasSetStream(cb, s));
  for (int64_t st = 0; st < n; st += chunk) {
    const int64_t m = std::min(chunk, n - st);
    const int64_t ne = m * K2;
    // K (m x 2R, row-major): G(y_i - c, a2_p) for the 2r check points, zero padded
    rows_kmat_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(d_pts + 3 * st, m, rep.a2, nullptr, 2 * rep.r, K2,
                                                                   K);
    // row-major T (m x R) = K (m x 2R) PoutH^T, PoutH = Qo^H W (R x 2R, row-major)
    DFMM_CUBLAS(cublasZgemm(cb, CUBLAS_OP_T, CUBLAS_OP_N, R, (int)m, K2, &one, (const cuDoubleComplex*)rep.PoutH,
                            K2, (const cuDoubleComplex*)K, K2, &zero, (cuDoubleComplex*)T, R));
    store_out(T, out, st * R, m * R, fp64, s);
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dfmm
