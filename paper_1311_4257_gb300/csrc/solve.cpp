// Iterative solve around the resident matvec: restarted GMRES for
//
//     (alpha I + beta G) x = b
//
// where G is the plan's operator (Eq. 1).  The paper's method is a fast matvec
// for the iterative solution of integral equations (Sec. 1: each iteration of a
// Krylov method applies G once); this is that outer loop, with the matvec
// through dfmm_apply on the caller's stream.  The Krylov basis lives on the
// device (complex64); each new vector is orthogonalised by classical
// Gram-Schmidt done twice (two GEMVs against the basis per pass), the small
// Hessenberg least-squares problem is solved on the host in double precision
// with Givens rotations.
#include <cublas_v2.h>

#include <cmath>
#include <complex>
#include <vector>

#include "common.h"
#include "dfmm.h"
#include "internal.h"

namespace {

using cd = std::complex<double>;

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

struct Blas {
  cublasHandle_t h = nullptr;
  ~Blas() {
    if (h) cublasDestroy(h);
  }
};

void check(cublasStatus_t st, const char* what) {
  if (st != CUBLAS_STATUS_SUCCESS) throw dfmm::Error(DFMM_ERR_CUDA, std::string("cuBLAS failed: ") + what);
}

cuComplex c32(cd z) { return make_cuComplex((float)z.real(), (float)z.imag()); }

}  // namespace

extern "C" int dfmm_solve(dfmm_plan_t plan, double alpha_re, double alpha_im, double beta_re, double beta_im,
                          const void* b, void* x, int restart, int maxit, double tol, cudaStream_t stream,
                          int* iters, double* relres) {
  try {
    if (!plan || !b || !x) return dfmm::set_error(DFMM_ERR_INVALID, "null argument");
    if (b == x) return dfmm::set_error(DFMM_ERR_INVALID, "b and x must not alias");
    if (restart < 1 || restart > 500) return dfmm::set_error(DFMM_ERR_INVALID, "restart must be in [1, 500]");
    if (maxit < 1) return dfmm::set_error(DFMM_ERR_INVALID, "maxit must be >= 1");
    if (!(tol > 0)) return dfmm::set_error(DFMM_ERR_INVALID, "tol must be positive");
    dfmm_stats st{};
    dfmm_plan_stats(plan, &st);
    if (st.arith != 32) return dfmm::set_error(DFMM_ERR_UNSUPPORTED, "dfmm_solve takes plans that compute in FP32");
    const int64_t N = st.N;
    const int m = restart;
    const cd alpha(alpha_re, alpha_im), beta(beta_re, beta_im);
    DevBuf Vb, wb, hb;
    if (cudaMalloc(&Vb.p, (size_t)(m + 1) * N * sizeof(cuComplex)) != cudaSuccess ||
        cudaMalloc(&wb.p, (size_t)N * sizeof(cuComplex)) != cudaSuccess ||
        cudaMalloc(&hb.p, (size_t)(m + 1) * sizeof(cuComplex)) != cudaSuccess) {
      cudaGetLastError();
      return dfmm::set_error(DFMM_ERR_OOM, "GMRES workspace allocation failed");
    }
    cuComplex* V = (cuComplex*)Vb.p;
    cuComplex* w = (cuComplex*)wb.p;
    cuComplex* hd = (cuComplex*)hb.p;
    cuComplex* xv = (cuComplex*)x;
    const cuComplex* bv = (const cuComplex*)b;
    Blas B;
    check(cublasCreate(&B.h), "create");
    check(cublasSetStream(B.h, stream), "set stream");
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f), mone = make_cuComplex(-1.f, 0.f);
    const cuComplex ca = c32(alpha), cb = c32(beta);

    // out = (alpha I + beta G) v
    auto matvec = [&](const cuComplex* v, cuComplex* out) {
      const int rc = dfmm_apply(plan, v, out, 1, stream);
      if (rc != DFMM_OK) throw dfmm::Error(rc, dfmm_last_error());
      check(cublasCscal(B.h, (int)N, &cb, out, 1), "scal");
      check(cublasCaxpy(B.h, (int)N, &ca, v, 1, out, 1), "axpy");
    };
    auto nrm = [&](const cuComplex* v) {
      float r = 0.f;
      check(cublasScnrm2(B.h, (int)N, v, 1, &r), "nrm2");
      return (double)r;
    };
    // r = b - A x into dst
    auto residual = [&](cuComplex* dst) {
      matvec(xv, w);
      DFMM_CUDA(cudaMemcpyAsync(dst, bv, (size_t)N * sizeof(cuComplex), cudaMemcpyDeviceToDevice, stream));
      check(cublasCaxpy(B.h, (int)N, &mone, w, 1, dst, 1), "axpy");
    };

    const double bnorm = nrm(bv);
    int done = 0;
    double rr = 0.0;
    if (bnorm == 0.0) {
      DFMM_CUDA(cudaMemsetAsync(xv, 0, (size_t)N * sizeof(cuComplex), stream));
    } else {
      std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), y(m);
      std::vector<cuComplex> hh(m + 1), yc(m);
      while (done < maxit) {
        residual(V);
        const double beta0 = nrm(V);
        rr = beta0 / bnorm;
        if (rr <= tol) break;
        const float inv0 = (float)(1.0 / beta0);
        check(cublasCsscal(B.h, (int)N, &inv0, V, 1), "scal");
        std::fill(H.begin(), H.end(), cd(0));
        std::fill(g.begin(), g.end(), cd(0));
        g[0] = beta0;
        int k = 0;
        for (int j = 0; j < m && done < maxit; ++j) {
          cuComplex* vj = V + (size_t)(j + 1) * N;
          matvec(V + (size_t)j * N, vj);
          for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
            check(cublasCgemv(B.h, CUBLAS_OP_C, (int)N, j + 1, &one, V, (int)N, vj, 1, &zero, hd, 1), "gemv");
            DFMM_CUDA(cudaMemcpyAsync(hh.data(), hd, (size_t)(j + 1) * sizeof(cuComplex), cudaMemcpyDeviceToHost,
                                      stream));
            DFMM_CUDA(cudaStreamSynchronize(stream));
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] += cd(hh[i].x, hh[i].y);
            check(cublasCgemv(B.h, CUBLAS_OP_N, (int)N, j + 1, &mone, V, (int)N, hd, 1, &one, vj, 1), "gemv");
          }
          const double hn = nrm(vj);
          H[(size_t)(j + 1) * m + j] = hn;
          // earlier rotations, then a new one that zeroes H[j+1][j]
          for (int i = 0; i < j; ++i) {
            const cd a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
            H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * c;
            H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
          }
          const cd a = H[(size_t)j * m + j];
          const double den = std::sqrt(std::norm(a) + hn * hn);
          cs[j] = den > 0 ? a / den : cd(1);
          sn[j] = den > 0 ? cd(hn / den) : cd(0);
          H[(size_t)j * m + j] = den;
          H[(size_t)(j + 1) * m + j] = 0;
          g[j + 1] = -sn[j] * g[j];
          g[j] = std::conj(cs[j]) * g[j];
          ++done;
          k = j + 1;
          rr = std::abs(g[j + 1]) / bnorm;
          if (rr <= tol || hn == 0.0) break;
          const float invn = (float)(1.0 / hn);
          check(cublasCsscal(B.h, (int)N, &invn, vj, 1), "scal");
        }
        // y = H[0:k, 0:k]^-1 g[0:k];  x += V[:, 0:k] y
        for (int i = k - 1; i >= 0; --i) {
          cd s = g[i];
          for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
          y[i] = s / H[(size_t)i * m + i];
        }
        for (int i = 0; i < k; ++i) yc[i] = c32(y[i]);
        DFMM_CUDA(cudaMemcpyAsync(hd, yc.data(), (size_t)k * sizeof(cuComplex), cudaMemcpyHostToDevice, stream));
        check(cublasCgemv(B.h, CUBLAS_OP_N, (int)N, k, &one, V, (int)N, hd, 1, &one, xv, 1), "gemv");
        DFMM_CUDA(cudaStreamSynchronize(stream));
        if (rr <= tol) break;
      }
      // the true residual of the returned x
      residual(V);
      rr = nrm(V) / bnorm;
    }
    DFMM_CUDA(cudaStreamSynchronize(stream));
    if (iters) *iters = done;
    if (relres) *relres = rr;
    return DFMM_OK;
  } catch (const dfmm::Error& e) {
    return dfmm::set_error(e.code, e.what());
  } catch (const std::exception& e) {
    return dfmm::set_error(DFMM_ERR_INVALID, e.what());
  }
}
