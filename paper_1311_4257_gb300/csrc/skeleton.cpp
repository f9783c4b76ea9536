// Host-side construction of the representations of Eq. 2 (see skeleton.h).
//
// Sampling (Sec. 2.1 "random sampling ... pivoted QR"): box samples are half
// uniform on the box surface, half uniform inside; far samples cover the
// region where the representation is evaluated:
//   HF (w, cell): boxes of width w that can enter the interaction list of a
//     width-w box in the closed wedge of `cell` (not near, parent near), and,
//     recursively up to w_top, the region of the parent's direction seen from
//     the child (the hierarchical wedges of Fig. 2);
//   LF (w): boxes of the V list, the exterior shell 1.5w <= |x|_inf <= 6w, and
//     the parent's region (LF parent, or every direction of the w = 1 box).
// Random numbers are SplitMix64 draws used as a counter-based generator; only
// +, *, floor and integer operations turn them into points.
#include "skeleton.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <thread>

namespace dfmm {

namespace {

const uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
const double TWO_PI = 6.283185307179586;

uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Stream {
  uint64_t seed, k = 0;
  explicit Stream(uint64_t s) : seed(s) {}
  double next() {
    k += 1;
    uint64_t z = splitmix64(seed + k * GAMMA);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  }
  int below(int n) {
    int v = (int)std::floor(next() * n);
    return v < n - 1 ? v : n - 1;
  }
};

uint64_t stream_seed(int64_t kind, double w, int64_t cell, double w_top, int64_t tol) {
  uint64_t h = 0x243F6A8885A308D3ull;
  int64_t vals[5] = {kind, (int64_t)std::llround(w * 1024), cell, (int64_t)std::llround(w_top * 1024), tol};
  for (int i = 0; i < 5; ++i) h = splitmix64(h ^ (uint64_t)vals[i]);
  return h;
}

int64_t floordiv(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

bool hf_near(const int64_t m[3], double w) {
  int64_t lim = (int64_t)std::llround(4.0 * w * w);
  int64_t s = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t t = 2 * std::llabs(m[d]) - 1;
    if (t < 0) t = 0;
    s += t * t;
  }
  return s <= lim;
}

struct P3 { double x[3]; };

P3 hf_box_point(Stream& st, double cw, int cell) {
  int n = n_cells(cw);
  int face = cell / (n * n), rem = cell % (n * n);
  int i = rem / n, j = rem % n;
  int a = face / 2, neg = face % 2;
  int others[2], no = 0;
  for (int d = 0; d < 3; ++d) if (d != a) others[no++] = d;
  int ks[2] = {i, j};
  int Mmax = 4 * (int)std::llround(cw) + 2;
  for (int it = 0; it < 100000; ++it) {
    int oB = st.below(8);
    int64_t M = 1 + st.below(Mmax);
    int64_t m[3] = {0, 0, 0};
    m[a] = neg ? -M : M;
    for (int q = 0; q < 2; ++q) {
      int64_t k = ks[q];
      int64_t lo = -floordiv(-(2 * M * k), n) - M;
      int64_t hi = floordiv(2 * M * (k + 1), n) - M;
      m[others[q]] = lo + st.below((int)(hi - lo + 1));
    }
    int64_t ob[3] = {(oB >> 2) & 1, (oB >> 1) & 1, oB & 1};
    if (hf_near(m, cw)) continue;
    int64_t pm[3];
    for (int d = 0; d < 3; ++d) pm[d] = floordiv(ob[d] + m[d], 2);
    if (!hf_near(pm, 2 * cw)) continue;
    P3 x;
    for (int d = 0; d < 3; ++d) x.x[d] = cw * (double)m[d] + (st.next() - 0.5) * cw;
    return x;
  }
  throw std::runtime_error("far-region rejection sampling did not terminate");
}

P3 hf_point(Stream& st, double w, int cell, double w_top) {
  int kmax = (int)std::llround(std::log2(w_top / w));
  double u = st.next();
  int k;
  if (kmax == 0 || u < 0.6) k = 0;
  else k = std::min(kmax, 1 + (int)std::floor((u - 0.6) * 2.5 * kmax));
  double shift[3] = {0, 0, 0};
  double cw = w;
  int n = n_cells(cw);
  for (int s = 0; s < k; ++s) {
    int o = st.below(8);
    double ob[3] = {(double)((o >> 2) & 1), (double)((o >> 1) & 1), (double)(o & 1)};
    for (int d = 0; d < 3; ++d) shift[d] = shift[d] - (ob[d] - 0.5) * cw;
    int face = cell / (n * n), rem = cell % (n * n);
    int i = rem / n, j = rem % n;
    int di = st.below(2), dj = st.below(2);
    int n2 = 2 * n;
    cell = (face * n2 + 2 * i + di) * n2 + 2 * j + dj;
    cw *= 2;
    n = n2;
  }
  P3 x = hf_box_point(st, cw, cell);
  for (int d = 0; d < 3; ++d) x.x[d] = shift[d] + x.x[d];
  return x;
}

P3 lf_point(Stream& st, double w, double w_top) {
  double u = st.next();
  if (u < 0.4) {
    for (;;) {
      int oB = st.below(8);
      int64_t ob[3] = {(oB >> 2) & 1, (oB >> 1) & 1, oB & 1};
      int64_t m[3];
      for (int d = 0; d < 3; ++d) m[d] = st.below(7) - 3;
      int64_t mx = std::max(std::llabs(m[0]), std::max(std::llabs(m[1]), std::llabs(m[2])));
      if (mx < 2) continue;
      bool ok = true;
      for (int d = 0; d < 3; ++d) if (std::llabs(floordiv(ob[d] + m[d], 2)) > 1) ok = false;
      if (!ok) continue;
      P3 x;
      for (int d = 0; d < 3; ++d) x.x[d] = w * (double)m[d] + (st.next() - 0.5) * w;
      return x;
    }
  }
  if (u < 0.6) {
    double R = 1.5 * w + st.next() * 4.5 * w;
    int face = st.below(6);
    int a = face / 2, neg = face % 2;
    P3 x;
    for (int d = 0; d < 3; ++d) x.x[d] = (2 * st.next() - 1) * R;
    x.x[a] = neg ? -R : R;
    return x;
  }
  int o = st.below(8);
  double ob[3] = {(double)((o >> 2) & 1), (double)((o >> 1) & 1), (double)(o & 1)};
  double shift[3];
  for (int d = 0; d < 3; ++d) shift[d] = -(ob[d] - 0.5) * w;
  P3 y;
  if (2 * w < 1.0) {
    y = lf_point(st, 2 * w, w_top);
  } else {
    int c = st.below(6);
    y = hf_point(st, 2 * w, c, w_top);
  }
  for (int d = 0; d < 3; ++d) y.x[d] = shift[d] + y.x[d];
  return y;
}

void box_samples_mixed(Stream& st, double w, int S, std::vector<double>& Y) {
  Y.assign((size_t)S * 3, 0.0);
  double h = 0.5 * w;
  int ns = S / 2;
  for (int q = 0; q < ns; ++q) {
    int face = st.below(6);
    int a = face / 2, neg = face % 2;
    for (int d = 0; d < 3; ++d) Y[q * 3 + d] = (2.0 * st.next() - 1.0) * h;
    Y[q * 3 + a] = neg ? -h : h;
  }
  for (int q = ns; q < S; ++q)
    for (int d = 0; d < 3; ++d) Y[q * 3 + d] = (st.next() - 0.5) * w;
}

inline double norm3(const double* x) { return std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]); }

inline cd kernel(const double* x, const double* y) {
  double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  double d = std::sqrt(dx * dx + dy * dy + dz * dz);
  double th = TWO_PI * d;
  return cd(std::cos(th) / d, std::sin(th) / d);
}

// Column-pivoted Householder QR of the m x n row-major matrix A (destroyed),
// norms recomputed at every step.  Pivots appended in order; stops when the
// largest remaining norm <= tol * |R_00| or after kmax steps.
void pivoted_qr(std::vector<cd>& A, int m, int n, double tol, int kmax,
                std::vector<int>& piv, std::vector<double>& diag) {
  std::vector<int> cols(n);
  for (int j = 0; j < n; ++j) cols[j] = j;
  kmax = std::min(kmax, std::min(m, n));
  std::vector<double> norms(n);
  std::vector<cd> v(m), wv(n);
  double r00 = -1;
  piv.clear();
  diag.clear();
  for (int k = 0; k < kmax; ++k) {
    std::fill(norms.begin() + k, norms.end(), 0.0);
    for (int i = k; i < m; ++i) {
      const cd* row = &A[(size_t)i * n];
      for (int j = k; j < n; ++j) norms[j] += row[j].real() * row[j].real() + row[j].imag() * row[j].imag();
    }
    int jb = k;
    double best = -1;
    for (int j = k; j < n; ++j) {
      double s = std::sqrt(norms[j]);
      if (s > best) { best = s; jb = j; }
    }
    if (r00 < 0) r00 = best;
    if (best <= tol * r00 || best == 0.0) break;
    if (jb != k) {
      for (int i = 0; i < m; ++i) std::swap(A[(size_t)i * n + k], A[(size_t)i * n + jb]);
      std::swap(cols[k], cols[jb]);
    }
    piv.push_back(cols[k]);
    diag.push_back(best);
    cd alpha = A[(size_t)k * n + k];
    double aa = std::abs(alpha);
    cd phase = aa > 0 ? alpha / aa : cd(1.0, 0.0);
    for (int i = k; i < m; ++i) v[i] = A[(size_t)i * n + k];
    v[k] += phase * best;
    double vn = 0;
    for (int i = k; i < m; ++i) vn += std::norm(v[i]);
    // w = v^H A[k:, k:]
    std::fill(wv.begin() + k, wv.end(), cd(0, 0));
    for (int i = k; i < m; ++i) {
      cd vc = std::conj(v[i]);
      const cd* row = &A[(size_t)i * n];
      for (int j = k; j < n; ++j) wv[j] += vc * row[j];
    }
    double sc = 2.0 / vn;
    for (int i = k; i < m; ++i) {
      cd vi = v[i] * sc;
      cd* row = &A[(size_t)i * n];
      for (int j = k; j < n; ++j) row[j] -= vi * wv[j];
    }
  }
}

// Thin QR (m >= n) by Householder, Q (m x n) and R (n x n) normalised so
// that diag(R) is real positive.
void thin_qr(const std::vector<cd>& A0, int m, int n, std::vector<cd>& Q, std::vector<cd>& R) {
  std::vector<cd> A = A0;
  std::vector<std::vector<cd>> vs(n);
  std::vector<double> vns(n);
  for (int k = 0; k < n; ++k) {
    double nk = 0;
    for (int i = k; i < m; ++i) nk += std::norm(A[(size_t)i * n + k]);
    nk = std::sqrt(nk);
    cd alpha = A[(size_t)k * n + k];
    double aa = std::abs(alpha);
    cd phase = aa > 0 ? alpha / aa : cd(1.0, 0.0);
    std::vector<cd> v(m - k);
    for (int i = k; i < m; ++i) v[i - k] = A[(size_t)i * n + k];
    v[0] += phase * nk;
    double vn = 0;
    for (auto& x : v) vn += std::norm(x);
    vs[k] = v;
    vns[k] = vn;
    if (vn == 0) continue;
    for (int j = k; j < n; ++j) {
      cd s(0, 0);
      for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * A[(size_t)i * n + j];
      s *= 2.0 / vn;
      for (int i = k; i < m; ++i) A[(size_t)i * n + j] -= v[i - k] * s;
    }
  }
  R.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) R[(size_t)i * n + j] = A[(size_t)i * n + j];
  // Q = H_0 H_1 ... H_{n-1} applied to the first n columns of I
  Q.assign((size_t)m * n, cd(0, 0));
  for (int j = 0; j < n; ++j) Q[(size_t)j * n + j] = cd(1, 0);
  for (int k = n - 1; k >= 0; --k) {
    const auto& v = vs[k];
    if (vns[k] == 0) continue;
    for (int j = 0; j < n; ++j) {
      cd s(0, 0);
      for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * Q[(size_t)i * n + j];
      s *= 2.0 / vns[k];
      for (int i = k; i < m; ++i) Q[(size_t)i * n + j] -= v[i - k] * s;
    }
  }
  // normalise: R_kk real positive
  for (int k = 0; k < n; ++k) {
    cd rk = R[(size_t)k * n + k];
    double ar = std::abs(rk);
    cd ph = ar > 0 ? rk / ar : cd(1, 0);
    for (int j = k; j < n; ++j) R[(size_t)k * n + j] *= std::conj(ph);
    for (int i = 0; i < m; ++i) Q[(size_t)i * n + k] *= ph;
  }
}

// Inverse of an upper-triangular n x n matrix.
std::vector<cd> tri_inv(const std::vector<cd>& R, int n) {
  std::vector<cd> X((size_t)n * n, cd(0, 0));
  for (int j = 0; j < n; ++j) {
    X[(size_t)j * n + j] = cd(1, 0) / R[(size_t)j * n + j];
    for (int i = j - 1; i >= 0; --i) {
      cd s(0, 0);
      for (int k = i + 1; k <= j; ++k) s += R[(size_t)i * n + k] * X[(size_t)k * n + j];
      X[(size_t)i * n + j] = -s / R[(size_t)i * n + i];
    }
  }
  return X;
}

}  // namespace

// Stage 1 of the selection (host form): Z = Omega (Wx G(X, Y)) with Omega the
// +-1 sketch from SplitMix draws (row-major order, draw k = q SX + i + 1),
// then its column-pivoted QR over all sketch rows.
void sketch_pivots_host(const Samples& sm, const SkelParams& prm, std::vector<int>& piv, std::vector<double>& diag) {
  const int SX = sm.SX, SY = sm.SY, s = prm.sketch;
  const std::vector<double>& X = sm.X;
  const std::vector<double>& Y = sm.Y;
  std::vector<cd> A((size_t)SX * SY);
  for (int i = 0; i < SX; ++i)
    for (int j = 0; j < SY; ++j) A[(size_t)i * SY + j] = sm.Wx[i] * kernel(&X[i * 3], &Y[j * 3]);
  std::vector<cd> Z((size_t)s * SY, cd(0, 0));
  for (int q = 0; q < s; ++q) {
    cd* zr = &Z[(size_t)q * SY];
    for (int i = 0; i < SX; ++i) {
      uint64_t kk = (uint64_t)q * SX + i + 1;
      uint64_t z = splitmix64(sm.sketch_seed + kk * GAMMA);
      const cd* ar = &A[(size_t)i * SY];
      if ((z >> 63) == 0) for (int j = 0; j < SY; ++j) zr[j] += ar[j];
      else for (int j = 0; j < SY; ++j) zr[j] -= ar[j];
    }
  }
  pivoted_qr(Z, s, SY, 0.0, s, piv, diag);
}

// Stage 2 (host form): the 2r far check points.  A2 = (Wx G(X, b))^T (r x SX);
// the first r are its pivots p1, the next r the pivots p2 of A2 restricted to
// the columns not in p1 (in ascending order).
void check_pivots_host(const Samples& sm, const std::vector<double>& b, int r, std::vector<int>& p1,
                       std::vector<int>& p2) {
  const int SX = sm.SX;
  std::vector<double> diag;
  std::vector<cd> A2((size_t)r * SX);
  for (int i = 0; i < SX; ++i)
    for (int q = 0; q < r; ++q) A2[(size_t)q * SX + i] = sm.Wx[i] * kernel(&sm.X[i * 3], &b[q * 3]);
  std::vector<cd> A2c = A2;
  pivoted_qr(A2c, r, SX, 0.0, r, p1, diag);
  const std::vector<int> rest = rest_of(p1, SX);
  std::vector<cd> A3((size_t)r * rest.size());
  for (int q = 0; q < r; ++q)
    for (size_t c = 0; c < rest.size(); ++c) A3[(size_t)q * rest.size() + c] = A2[(size_t)q * SX + rest[c]];
  pivoted_qr(A3, r, (int)rest.size(), 0.0, r, p2, diag);
}

Rep build_from_samples(const Samples& sm, const SkelParams& prm) {
  std::vector<int> piv, p1, p2;
  std::vector<double> diag;
  sketch_pivots_host(sm, prm, piv, diag);
  const int r = rank_from_pivots(diag, (int)piv.size(), prm);
  const std::vector<double> b = box_points(sm, piv, r);
  check_pivots_host(sm, b, r, p1, p2);
  return finish_rep(sm, piv, r, p1, p2);
}


const std::vector<Sym>& symmetries() {
  static std::vector<Sym> syms = [] {
    std::vector<Sym> v;
    int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (auto& p : perms)
      for (int s = 0; s < 8; ++s) {
        Sym y;
        for (int k = 0; k < 3; ++k) y.perm[k] = p[k];
        y.sign[0] = (s & 4) ? -1 : 1;
        y.sign[1] = (s & 2) ? -1 : 1;
        y.sign[2] = (s & 1) ? -1 : 1;
        v.push_back(y);
      }
    return v;
  }();
  return syms;
}

static void apply_sym(const Sym& s, const double* x, double* y) {
  for (int k = 0; k < 3; ++k) y[k] = s.sign[k] * x[s.perm[k]];
}

static void cell_center_dir(int cell, int n, double v[3]) {
  int face = cell / (n * n), rem = cell % (n * n);
  int i = rem / n, j = rem % n;
  int a = face / 2, neg = face % 2;
  int others[2], no = 0;
  for (int d = 0; d < 3; ++d) if (d != a) others[no++] = d;
  v[a] = neg ? -1.0 : 1.0;
  v[others[0]] = 2 * (i + 0.5) / n - 1;
  v[others[1]] = 2 * (j + 0.5) / n - 1;
}

static int cell_of_dir(const double v[3], int n) {
  int a = 0;
  for (int d = 1; d < 3; ++d) if (std::fabs(v[d]) > std::fabs(v[a])) a = d;
  double M = std::fabs(v[a]);
  int face = 2 * a + (v[a] < 0 ? 1 : 0);
  int others[2], no = 0;
  for (int d = 0; d < 3; ++d) if (d != a) others[no++] = d;
  int i = std::min(n - 1, (int)std::floor(n * (v[others[0]] / M + 1) / 2));
  int j = std::min(n - 1, (int)std::floor(n * (v[others[1]] / M + 1) / 2));
  return (face * n + i) * n + j;
}

void canonical_cells(int n, std::vector<int>& canon, std::vector<int>& which) {
  int nd = 6 * n * n;
  const auto& syms = symmetries();
  std::vector<int> img(syms.size() * nd);
  for (size_t s = 0; s < syms.size(); ++s)
    for (int c = 0; c < nd; ++c) {
      double v[3], u[3];
      cell_center_dir(c, n, v);
      apply_sym(syms[s], v, u);
      img[s * nd + c] = cell_of_dir(u, n);
    }
  canon.assign(nd, 0);
  which.assign(nd, 0);
  for (int c = 0; c < nd; ++c) {
    int k = nd;
    for (size_t s = 0; s < syms.size(); ++s) k = std::min(k, img[s * nd + c]);
    canon[c] = k;
    for (size_t s = 0; s < syms.size(); ++s)
      if (img[s * nd + k] == c) { which[c] = (int)s; break; }
  }
}

Samples make_samples(double w, int cell, double w_top, const SkelParams& prm) {
  int64_t tol = (int64_t)std::llround(-std::log10(prm.eps_op) * 100);
  bool lf = cell < 0;
  uint64_t seed = stream_seed(lf ? 2 : 1, w, lf ? 0 : cell, w_top, tol);
  Stream st(seed);
  Samples sm;
  sm.w = w;
  sm.cell = lf ? -1 : cell;
  sm.SY = prm.S_Y;
  sm.SX = prm.S_X;
  sm.X.resize((size_t)prm.S_X * 3);
  box_samples_mixed(st, w, prm.S_Y, sm.Y);
  for (int q = 0; q < prm.S_X; ++q) {
    P3 p = lf ? lf_point(st, w, w_top) : hf_point(st, w, cell, w_top);
    for (int d = 0; d < 3; ++d) sm.X[q * 3 + d] = p.x[d];
  }
  sm.Wx.resize(prm.S_X);
  for (int i = 0; i < prm.S_X; ++i) sm.Wx[i] = norm3(&sm.X[i * 3]);
  sm.sketch_seed = splitmix64(seed ^ 0x5DEECE66Dull);
  return sm;
}

int rank_from_pivots(const std::vector<double>& diag, int npiv, const SkelParams& prm) {
  int r = 0;
  for (double d : diag) if (d > prm.eps_op * diag[0]) ++r;
  if (2 * r > npiv) throw std::runtime_error("representation rank too large for the sketch");
  return r;
}

std::vector<double> box_points(const Samples& sm, const std::vector<int>& piv, int n) {
  std::vector<double> b((size_t)n * 3);
  for (int q = 0; q < n; ++q)
    for (int d = 0; d < 3; ++d) b[q * 3 + d] = sm.Y[piv[q] * 3 + d];
  return b;
}

std::vector<int> rest_of(const std::vector<int>& p1, int n) {
  std::vector<char> used(n, 0);
  for (int p : p1) used[p] = 1;
  std::vector<int> rest;
  for (int i = 0; i < n; ++i) if (!used[i]) rest.push_back(i);
  return rest;
}

Rep finish_rep(const Samples& sm, const std::vector<int>& piv, int r, const std::vector<int>& p1,
               const std::vector<int>& p2) {
  if ((int)p1.size() != r || (int)p2.size() != r) throw std::runtime_error("check-point selection failed");
  const std::vector<int> rest = rest_of(p1, sm.SX);
  Rep rep;
  rep.w = sm.w;
  rep.cell = sm.cell;
  rep.r = r;
  rep.b2 = box_points(sm, piv, 2 * r);
  rep.a2.resize((size_t)2 * r * 3);
  rep.wa2.resize(2 * r);
  for (int q = 0; q < 2 * r; ++q) {
    int idx = q < r ? p1[q] : rest[p2[q - r]];
    for (int d = 0; d < 3; ++d) rep.a2[q * 3 + d] = sm.X[idx * 3 + d];
    rep.wa2[q] = norm3(&rep.a2[q * 3]);
  }
  std::vector<cd> M((size_t)2 * r * r), Qm, Rm;
  for (int p = 0; p < 2 * r; ++p)
    for (int q = 0; q < r; ++q) M[(size_t)p * r + q] = rep.wa2[p] * kernel(&rep.a2[p * 3], &rep.b2[q * 3]);
  thin_qr(M, 2 * r, r, Qm, Rm);
  rep.Qo = Qm;
  rep.Ro_inv = tri_inv(Rm, r);
  for (int p = 0; p < 2 * r; ++p)
    for (int q = 0; q < r; ++q) M[(size_t)p * r + q] = kernel(&rep.b2[p * 3], &rep.a2[q * 3]) * rep.wa2[q];
  thin_qr(M, 2 * r, r, Qm, Rm);
  rep.Qi = Qm;
  rep.Ri_inv = tri_inv(Rm, r);
  return rep;
}

Rep build_rep(double w, int cell, double w_top, const SkelParams& prm) {
  return build_from_samples(make_samples(w, cell, w_top, prm), prm);
}

Rep map_rep(const Rep& base, const Sym& s, int cell) {
  Rep r = base;
  r.cell = cell;
  for (int q = 0; q < 2 * base.r; ++q) {
    apply_sym(s, &base.b2[q * 3], &r.b2[q * 3]);
    apply_sym(s, &base.a2[q * 3], &r.a2[q * 3]);
  }
  return r;
}

// ------------------------------------------------------------- RepSet ---

RepSet::RepSet(const SkelParams& prm, double w_top, int threads, const std::string& cache_dir, bool on_device)
    : prm_(prm), w_top_(w_top), threads_(threads), cache_dir_(cache_dir), on_device_(on_device) {}

Rep* RepSet::find(std::vector<std::pair<std::pair<double, int>, Rep>>& v, double w, int cell) {
  for (auto& e : v)
    if (e.first.first == w && e.first.second == cell) return &e.second;
  return nullptr;
}

static std::string cache_name(const std::string& dir, double w, int cell, double w_top, const SkelParams& p) {
  char buf[512];
  std::snprintf(buf, sizeof buf, "%s/rep_v1_w%g_c%d_t%g_e%.3e_%d_%d_%d.bin", dir.c_str(), w, cell, w_top, p.eps_op,
                p.S_Y, p.S_X, p.sketch);
  return buf;
}

static bool load_rep(const std::string& fn, Rep& r) {
  FILE* f = std::fopen(fn.c_str(), "rb");
  if (!f) return false;
  bool ok = std::fread(&r.w, sizeof r.w, 1, f) == 1 && std::fread(&r.cell, sizeof r.cell, 1, f) == 1 &&
            std::fread(&r.r, sizeof r.r, 1, f) == 1;
  if (ok) {
    size_t n2 = (size_t)2 * r.r, nn = (size_t)r.r * r.r;
    r.b2.resize(n2 * 3); r.a2.resize(n2 * 3); r.wa2.resize(n2);
    r.Qo.resize(n2 * r.r); r.Ro_inv.resize(nn); r.Qi.resize(n2 * r.r); r.Ri_inv.resize(nn);
    ok = std::fread(r.b2.data(), 8, n2 * 3, f) == n2 * 3 && std::fread(r.a2.data(), 8, n2 * 3, f) == n2 * 3 &&
         std::fread(r.wa2.data(), 8, n2, f) == n2 && std::fread(r.Qo.data(), 16, n2 * r.r, f) == n2 * r.r &&
         std::fread(r.Ro_inv.data(), 16, nn, f) == nn && std::fread(r.Qi.data(), 16, n2 * r.r, f) == n2 * r.r &&
         std::fread(r.Ri_inv.data(), 16, nn, f) == nn;
  }
  std::fclose(f);
  return ok;
}

static void save_rep(const std::string& fn, const Rep& r) {
  std::string tmp = fn + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return;
  size_t n2 = (size_t)2 * r.r, nn = (size_t)r.r * r.r;
  std::fwrite(&r.w, sizeof r.w, 1, f); std::fwrite(&r.cell, sizeof r.cell, 1, f); std::fwrite(&r.r, sizeof r.r, 1, f);
  std::fwrite(r.b2.data(), 8, n2 * 3, f); std::fwrite(r.a2.data(), 8, n2 * 3, f); std::fwrite(r.wa2.data(), 8, n2, f);
  std::fwrite(r.Qo.data(), 16, n2 * r.r, f); std::fwrite(r.Ro_inv.data(), 16, nn, f);
  std::fwrite(r.Qi.data(), 16, n2 * r.r, f); std::fwrite(r.Ri_inv.data(), 16, nn, f);
  std::fclose(f);
  std::rename(tmp.c_str(), fn.c_str());
}

void RepSet::prepare(const std::vector<std::pair<double, int>>& types) {
  // canonical work items
  std::vector<std::pair<double, int>> todo;
  for (auto& t : types) {
    int c0 = t.second;
    if (t.second >= 0) {
      std::vector<int> canon, which;
      canonical_cells(n_cells(t.first), canon, which);
      c0 = canon[t.second];
    }
    bool have = find(base_, t.first, c0) != nullptr;
    for (auto& x : todo) if (x.first == t.first && x.second == c0) have = true;
    if (!have) todo.push_back({t.first, c0});
  }
  const size_t n = todo.size();
  auto clock = [] { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); };
  double t0 = clock();
  std::vector<Rep> out(n);
  std::vector<char> have(n, 0);
  std::vector<std::string> fn(n);
  // fn(i) for i < count on up to threads_ host threads; the first error is rethrown
  auto parallel = [&](size_t count, const std::function<void(size_t)>& body) {
    std::atomic<size_t> next(0);
    std::string err;
    std::mutex mu;
    auto worker = [&]() {
      for (;;) {
        size_t i = next.fetch_add(1);
        if (i >= count) return;
        try {
          body(i);
        } catch (const std::exception& e) {
          std::lock_guard<std::mutex> g(mu);
          if (err.empty()) err = e.what();
        }
      }
    };
    int nt = threads_ > 0 ? threads_ : (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min<int>(nt, (int)count));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    if (!err.empty()) throw std::runtime_error(err);
  };
  parallel(n, [&](size_t i) {
    if (cache_dir_.empty()) return;
    fn[i] = cache_name(cache_dir_, todo[i].first, todo[i].second, w_top_, prm_);
    if (load_rep(fn[i], out[i])) have[i] = 1;
  });
  std::vector<size_t> miss;
  for (size_t i = 0; i < n; ++i)
    if (!have[i]) miss.push_back(i);
  seconds[0] += clock() - t0;
  t0 = clock();
  if (!on_device_) {
    parallel(miss.size(), [&](size_t k) {
      const size_t i = miss[k];
      out[i] = build_rep(todo[i].first, todo[i].second, w_top_, prm_);
      if (!fn[i].empty()) save_rep(fn[i], out[i]);
    });
    seconds[1] += clock() - t0;
  } else if (!miss.empty()) {
    // samples on the host, both pivot stages on the GPU for all missing types
    // at once, the least-squares factors on the host again
    std::vector<Samples> sm(miss.size());
    parallel(miss.size(), [&](size_t k) { sm[k] = make_samples(todo[miss[k]].first, todo[miss[k]].second, w_top_, prm_); });
    seconds[0] += clock() - t0;
    t0 = clock();
    std::vector<SketchJob> sj(miss.size());
    for (size_t k = 0; k < miss.size(); ++k) sj[k].sm = &sm[k];
    sketch_pivots_device(sj, prm_);
    seconds[1] += clock() - t0;
    t0 = clock();
    std::vector<CheckJob> cj(miss.size());
    for (size_t k = 0; k < miss.size(); ++k) {
      cj[k].sm = &sm[k];
      cj[k].r = rank_from_pivots(sj[k].diag, (int)sj[k].piv.size(), prm_);
      cj[k].b = box_points(sm[k], sj[k].piv, cj[k].r);
    }
    check_pivots_device(cj);
    seconds[2] += clock() - t0;
    t0 = clock();
    parallel(miss.size(), [&](size_t k) {
      const size_t i = miss[k];
      out[i] = finish_rep(sm[k], sj[k].piv, cj[k].r, cj[k].p1, cj[k].p2);
      if (!fn[i].empty()) save_rep(fn[i], out[i]);
    });
    seconds[3] += clock() - t0;
  }
  for (size_t i = 0; i < todo.size(); ++i) base_.push_back({todo[i], std::move(out[i])});
}

const Rep& RepSet::get(double w, int cell) {
  if (cell < 0) {
    Rep* r = find(base_, w, -1);
    if (!r) { prepare({{w, -1}}); r = find(base_, w, -1); }
    return *r;
  }
  Rep* m = find(mapped_, w, cell);
  if (m) return *m;
  std::vector<int> canon, which;
  canonical_cells(n_cells(w), canon, which);
  Rep* b = find(base_, w, canon[cell]);
  if (!b) { prepare({{w, cell}}); b = find(base_, w, canon[cell]); }
  mapped_.push_back({{w, cell}, map_rep(*b, symmetries()[which[cell]], cell)});
  return mapped_.back().second;
}

}  // namespace dfmm
