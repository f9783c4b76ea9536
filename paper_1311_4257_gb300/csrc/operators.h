// Plan-time formation of the translation operators in FP64 (see operators.cu).
#pragma once
#include <vector>

#include "common.h"
#include "skeleton.h"
#include "tree.h"

namespace dfmm {

// A representation type on the device, FP64, padded to the rank R of its
// width class.  All matrices row-major, zero outside the r x (.) block.
struct DevRep {
  int r = 0, R = 0;
  double* b2 = nullptr;      // [2r][3]
  double* a2 = nullptr;      // [2r][3]
  double* wa2 = nullptr;     // [2r]
  double2* PoutH = nullptr;  // [R][2R]  Qo^H diag(wa2)
  double2* PinH = nullptr;   // [R][2R]  Qi^H
  double2* Ro_inv = nullptr; // [R][R]
  double2* Ri_inv = nullptr; // [R][R]
};

DevRep upload_rep(const Rep& rep, int R, DevArena& ar, cudaStream_t s);

enum OpKind { kOpM2M = 0, kOpM2L = 1, kOpL2L = 2 };

// One translation operator T (R_t x R_s):
//   M2M: T = Qo_t^H W_t G(a2_t + shift, b_s) Ro_s^{-1}
//   M2L: T = Qi_t^H      G(b2_t + shift, b_s) Ro_s^{-1}
//   L2L: T = Qi_t^H      G(b2_t + shift, a_in_s) W_s Ri_s^{-1}
struct OpSpec {
  int tgt_rep, src_rep;
  double shift[3];
};

// Forms ops (all of one kind, one pair of width classes R_t, R_s) and writes
// them as complex64 [n][R_t][R_s] into out (device), or as complex128 when
// fp64 is set (the FP64 form of the apply).
void form_ops(OpKind kind, const std::vector<OpSpec>& ops, const std::vector<DevRep>& reps, int Rt, int Rs,
              void* out, bool fp64, DevArena& ar, cudaStream_t s);

// Rows for evaluating a representation at points:
//   L2P (incoming): row_i = G(y_i - c, a_in) W Ri^{-1}
//   M2P (outgoing): row_i = G(y_i - c, b) Ro^{-1}
// pts: device FP64 [n][3] of y_i - c (local), written as complex64 [n][R]
// (complex128 when fp64 is set).
void form_rows(bool incoming, const DevRep& rep, const double* d_local_pts, int64_t n, void* out, bool fp64,
               DevArena& ar, cudaStream_t s);

// Rows of P2M through the outgoing representation (Eq. 2 with the
// least-squares projection): row_i = Qo^H W G(a2, y_i - c), the outgoing
// state a unit source at y_i produces.  pts: device FP64 [n][3] of y_i - c;
// written as complex64 [n][R] (complex128 when fp64 is set).
void form_p2m_rows(const DevRep& rep, const double* d_local_pts, int64_t n, void* out, bool fp64, DevArena& ar,
                   cudaStream_t s);

}  // namespace dfmm
