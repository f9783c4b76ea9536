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

// The stages of build_rep, so that the pivot selection can run on the GPU
// (skeleton_gpu.cu) for a batch of types:
//   make_samples       S_Y box samples Y, S_X far-region samples X, weights |x|
//                      and the sketch seed (host, counter-based draws);
//   sketch pivots      column-pivoted QR of the +-1 sketch of Wx G(X, Y) over
//                      all sketch rows: pivots and |R_kk| (Sec. 2.1);
//   rank_from_pivots   r = #{k : |R_kk| > eps_op |R_00|} (2r <= pivots);
//   check pivots       the 2r far check points: pivots p1 of A2 = (Wx G(X, b))^T
//                      (r x S_X, b = the r equivalent points), then pivots p2 of
//                      A2 restricted to the columns not in p1 (ascending);
//   finish_rep         points, weights and the least-squares factors.
struct Samples {
  double w = 0;
  int cell = -1;
  int SY = 0, SX = 0;
  std::vector<double> Y, X, Wx;   // [SY][3], [SX][3], [SX]
  uint64_t sketch_seed = 0;
};
Samples make_samples(double w, int cell, double w_top, const SkelParams& prm);
void sketch_pivots_host(const Samples& sm, const SkelParams& prm, std::vector<int>& piv, std::vector<double>& diag);
int rank_from_pivots(const std::vector<double>& diag, int npiv, const SkelParams& prm);
std::vector<double> box_points(const Samples& sm, const std::vector<int>& piv, int n);
std::vector<int> rest_of(const std::vector<int>& p1, int n);
void check_pivots_host(const Samples& sm, const std::vector<double>& b, int r, std::vector<int>& p1,
                       std::vector<int>& p2);
Rep finish_rep(const Samples& sm, const std::vector<int>& piv, int r, const std::vector<int>& p1,
               const std::vector<int>& p2);
Rep build_from_samples(const Samples& sm, const SkelParams& prm);

// GPU forms of the two pivot stages (skeleton_gpu.cu), for a batch of types on
// the current device.  Same draws, same pivot rule (largest remaining column
// norm, recomputed at every step, first index on ties); the floating-point
// rounding differs from the host's, so near-tied pivots may differ.
struct SketchJob {
  const Samples* sm = nullptr;
  std::vector<int> piv;          // out: one pivot per sketch row (fewer if a column norm vanishes)
  std::vector<double> diag;      // out: |R_kk|
};
void sketch_pivots_device(std::vector<SketchJob>& jobs, const SkelParams& prm);
struct CheckJob {
  const Samples* sm = nullptr;
  std::vector<double> b;         // the r equivalent points [r][3]
  int r = 0;
  std::vector<int> p1, p2;       // out
};
void check_pivots_device(std::vector<CheckJob>& jobs);

// Apply a symmetry to a representation (points mapped, matrices unchanged).
Rep map_rep(const Rep& base, const Sym& s, int cell);

// Cache of representations: builds canonical types (in parallel) and maps.
class RepSet {
 public:
  // on_device: pivot selection on the current GPU (skeleton_gpu.cu), else host threads
  RepSet(const SkelParams& prm, double w_top, int threads, const std::string& cache_dir, bool on_device = false);
  // Build every canonical type needed for the requested (w, cell) list.
  void prepare(const std::vector<std::pair<double, int>>& types);
  const Rep& get(double w, int cell);
  const SkelParams& params() const { return prm_; }
  size_t built() const { return base_.size(); }
  double w_top() const { return w_top_; }
  // wall seconds of the builds so far: 0 = disk cache and samples, 1 = sketch
  // pivots, 2 = check-point pivots, 3 = least-squares factors (1-3 summed over
  // the host threads' builds in the host form, where they are not separated: all in 1)
  double seconds[4] = {0, 0, 0, 0};

 private:
  SkelParams prm_;
  double w_top_;
  int threads_;
  std::string cache_dir_;
  bool on_device_ = false;
  std::vector<std::pair<std::pair<double, int>, Rep>> base_;   // canonical
  std::vector<std::pair<std::pair<double, int>, Rep>> mapped_;
  Rep* find(std::vector<std::pair<std::pair<double, int>, Rep>>& v, double w, int cell);
};

}  // namespace dfmm
