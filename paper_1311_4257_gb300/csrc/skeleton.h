// Host-side construction of the low-rank representations of Eq. 2.
//
// A representation type is (box width w, face cell) for w >= 1 (directional,
// Sec. 2.1-2.2) or (w, -1) for w < 1 (non-directional, the low-frequency
// regime).  Each type is built from random samples of the box and of the far
// region where it is evaluated, by pivoted QR (Sec. 2.1), and is stored in the
// least-squares form that keeps single-precision application stable:
//   outgoing: W G(a2, b) = Qo Ro,  state s = Qo^H W u(a2),  field G(x, b) Ro^{-1} s
//   incoming: G(b2, a_in) W = Qi Ri, state t = Qi^H v(b2),  field G(y, a_in) W Ri^{-1} t
// with b = b2[0:r] (equivalent points, in the box), a2 (2r far check points,
// a_in = a2[0:r]) and b2 (2r box check points).
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace dfmm {

using cd = std::complex<double>;

struct Rep {
  double w = 0;
  int cell = -1;
  int r = 0;
  std::vector<double> b2;      // [2r][3]
  std::vector<double> a2;      // [2r][3]
  std::vector<double> wa2;     // [2r]  |a2|
  std::vector<cd> Qo;          // [2r][r] row-major
  std::vector<cd> Ro_inv;      // [r][r]
  std::vector<cd> Qi;          // [2r][r]
  std::vector<cd> Ri_inv;      // [r][r]
};

struct SkelParams {
  double eps_op = 1e-6;
  int S_Y = 1024;
  int S_X = 4096;
  int sketch = 400;
};

// Number of face cells per side for width w (w >= 1).
inline int n_cells(double w) { return (int)(w + 0.5); }

// The 48 signed permutations of the cube: (Qx)_k = s_k x_{perm[k]}.
struct Sym { int perm[3]; int sign[3]; };
const std::vector<Sym>& symmetries();

// For every cell of the n x n face grids: the canonical cell of its orbit and
// the index of the symmetry that maps the canonical cell onto it.
void canonical_cells(int n, std::vector<int>& canon, std::vector<int>& which);

// Build one representation from scratch (HF if cell >= 0, LF if cell < 0).
// w_top: coarsest width whose representations are evaluated.
Rep build_rep(double w, int cell, double w_top, const SkelParams& prm);

// Apply a symmetry to a representation (points mapped, matrices unchanged).
Rep map_rep(const Rep& base, const Sym& s, int cell);

// Cache of representations: builds canonical types (in parallel) and maps.
class RepSet {
 public:
  RepSet(const SkelParams& prm, double w_top, int threads, const std::string& cache_dir);
  // Build every canonical type needed for the requested (w, cell) list.
  void prepare(const std::vector<std::pair<double, int>>& types);
  const Rep& get(double w, int cell);
  const SkelParams& params() const { return prm_; }
  double w_top() const { return w_top_; }

 private:
  SkelParams prm_;
  double w_top_;
  int threads_;
  std::string cache_dir_;
  std::vector<std::pair<std::pair<double, int>, Rep>> base_;   // canonical
  std::vector<std::pair<std::pair<double, int>, Rep>> mapped_;
  Rep* find(std::vector<std::pair<std::pair<double, int>, Rep>>& v, double w, int cell);
};

}  // namespace dfmm
