// Apply-time kernels of the matvec (see apply.cu).
#pragma once
#include <cstdint>

#include <cuda_fp16.h>

#include "common.h"

namespace dfmm {

// Check point of an LF representation, for kernel evaluation with a
// compensated phase: x = local point, nx2 = |x|^2, nx = |x|, fx = frac(|x|).
struct ChkPt {
  float x, y, z, nx2;
  float nx, fx, pad0, pad1;
};

// One translation stage: y[dst] += T_op x[src] for every (src, dst) pair,
// columns = pairs x nrhs.  Operators complex64 [nops][M][Kd] row-major.
struct CxStage;

struct GemmArgs {
  const float2* ops;
  int M, Kd;
  const int4* tiles;        // (op, first pair, number of pairs, 0)
  int64_t ntiles;
  const int2* pairs;        // (src row, dst row)
  const float2* src;        // rows of src_ld complex, row index = src_row * nrhs + rhs
  float2* dst;              // rows of dst_ld complex
  int src_ld, dst_ld;
  int nrhs;
  int store;                // 1: every target row of the stage has one pair and nothing wrote it
                            //    earlier in the apply, so results are stored, not added
  int wait_test;            // tensor-core form: 1 = CTA 0 waits on a barrier nothing arrives at
                            //    (exercises the bounded-wait failure path)
  const CxStage* stages;    // split-complex form, several stages in one launch (device array), or
                            //    nullptr: one stage given by the fields above and TcArgs
};

void launch_gemm_stage(const GemmArgs& a, cudaStream_t s);

// One stage of a multi-stage split-complex launch (the batched form runs the
// same step of several plans in one launch): its tiles carry the stage's index
// in .w; all stages of a launch share M, Kd, dst_ld and the split's element type.
struct CxStage {
  const int2* pairs;        // (src row, dst row)
  const void* src_hi;       // split source rows (launch_split_cx)
  const void* src_lo;
  const float* src_scale;
  const void* img;          // operator image (build_cx_image)
  const float* op_scale;
  float2* dst;              // target states
  int nrhs;
  int store;
};

// Tensor-core form (tcgen05, scaled FP16 split) of the same stage; M and Kd
// must be multiples of 8, source rows dense (src_ld == Kd); tiles hold up to
// gemm_tc_columns() columns.  img / op_scale: operator image and per-operator
// power-of-two scales (build_tc_image); src_hi / src_lo / src_scale: the
// source buffer split by launch_split (one scale per source row).
struct TcArgs {
  const __half* img;
  const float* op_scale;
  const __half* src_hi;
  const __half* src_lo;
  const float* src_scale;
};
void launch_gemm_stage_tc(const GemmArgs& a, const TcArgs& t, unsigned* status, cudaStream_t s);
int gemm_tc_columns();
bool gemm_tc_supported(int M, int Kd);
int64_t tc_image_elems(int M, int Kd, int nops);
void build_tc_image(const float2* ops, int M, int Kd, int nops, __half* img, float* scale, cudaStream_t s);
void launch_split(const float2* x, int64_t rows, int ld, __half* hi, __half* lo, float* scale, cudaStream_t s);
// scale[op] = smallest power of two >= max |entry| of operator op (per_op complex entries each)
void compute_op_scales(const float2* ops, int64_t per_op, int nops, float* scale, cudaStream_t s);

// Split-complex tensor-core form (m2l_cx.cu): Re y = Tr xr - Ti xi, Im y =
// Ti xr + Tr xi as four real GEMMs with N = M (target rank, a multiple of 16,
// at most 128) and K = Kd (a multiple of 16); operator image of Tr and Ti
// (build_cx_image) and source rows split into real and imaginary halves
// (launch_split_cx, rank r = row length in complex values).  Tiles hold up to
// gemm_cx_columns() columns.
bool gemm_cx_supported(int M, int Kd);
int gemm_cx_columns();
// kind: element type of the split, 0 = FP16, 1 = BF16, 2 = TF32 (4 bytes)
int cx_elem_bytes(int kind);
int64_t cx_image_bytes(int M, int Kd, int nops, int kind);
void build_cx_image(const float2* ops, int M, int Kd, int nops, void* img, float* scale, int kind, cudaStream_t s);
void launch_split_cx(const float2* x, int64_t rows, int r, void* hi, void* lo, float* scale, int kind, cudaStream_t s);
// one_acc: one accumulator per component, double-buffered tensor memory (faster,
// the cross terms accumulate with the large terms' truncation)
void launch_gemm_stage_cx(const GemmArgs& a, const TcArgs& t, unsigned* status, bool one_acc, int kind,
                          cudaStream_t s);

// Permutes: fs[k][rhs] = f[rhs][perm[k]];  u[rhs][perm[k]] = us[k][rhs].
void launch_permute_in(const float2* f, const int32_t* perm, int64_t N, int nrhs, float2* fs, cudaStream_t s);
void launch_permute_out(const float2* us, const int32_t* perm, int64_t N, int nrhs, float2* u, cudaStream_t s);

// Kernel evaluation from points to check points (P2M, and P2L with the
// target box's check points): out[row][rhs][p] = sum_i G(c + x_p - y_i) f_i.
// jobs: (first point, count, row, ptsrc shift index) ; shifts: float4 c_tgt - c_src
// (zero for P2M).  pts: local coordinates relative to the source leaf centre.
struct P2CArgs {
  const int4* jobs;          // (first point, count, out row, shift index)
  int64_t njobs;
  const float4* shifts;      // (dx, dy, dz, 0): check-point frame minus point frame
  const ChkPt* chk;          // 2r check points
  int nchk, ld;              // number of check points, out row length (2R)
  const float4* pts;         // sorted local points (x, y, z, |x|^2)
  const float2* fs;          // [N][nrhs]
  float2* out;               // [rows][nrhs][ld]
  int nrhs;
  const double* chk64;       // FP64 form: the check points, [nchk][3]
  const float4* pts_lo;      // FP64 form: low parts of the local coordinates
};
void launch_p2c(const P2CArgs& a, cudaStream_t s);

// Rows applied to states: us[i][rhs] += sum_q rows[row_i][q] state[srow][rhs][q].
struct RowsArgs {
  const int4* jobs;          // (first point, count, first row, state row)
  int64_t njobs;
  const float2* rows;        // [..][R]
  const float2* state;       // [..][nrhs][R]
  int R, nrhs;
  float2* us;                // [N][nrhs]
  int atomic;
};
void launch_rows(const RowsArgs& a, cudaStream_t s);

// L2P, one warp per point: us[p_r][rhs] += sum_q rows[r][q] state[s_r][rhs][q]
// for every row r, with (p_r, s_r) = map[r] (each point has one row).
struct L2PArgs {
  const int2* map;           // (point, state row) per row
  int64_t nrows;
  const float2* rows;        // [nrows][R]
  const float2* state;       // [..][nrhs][R]
  int R, nrhs;               // R even, <= 256
  float2* us;                // [N][nrhs]
};
void launch_l2p(const L2PArgs& a, cudaStream_t s);

// P2M through per-point rows: for every leaf job (first point, count, first
// row, box) and right-hand side k, state[box][k][q] = sum_i rows[row + i][q]
// fs[first + i][k].
struct P2MRowsArgs {
  const int4* jobs;
  int64_t njobs;
  const float2* rows;        // [..][R]
  const float2* fs;          // [N][nrhs]
  float2* state;             // [boxes][nrhs][R]
  int R, nrhs;               // R <= 256
};
void launch_p2m_rows(const P2MRowsArgs& a, cudaStream_t s);

// Near field: us[i] += sum over U-list source leaves of G(p_i, p_j) f_j,
// skipping p_j == p_i.
struct P2PArgs {
  const int2* leaf_range;    // (first, count) per target leaf
  int64_t nleaves;
  const int64_t* u_off;      // CSR offsets per target leaf
  const int4* u_src;         // (first point, count, offset of its first point in the flat
                             //   list of all leaves' sources, self) per source leaf; the target
                             //   leaf's own entry comes first, with self = 1
  const float4* u_shift;     // c_src - c_tgt per source leaf
  const uint32_t* flat;      // FP32 form: the staged sources of every leaf in order, point index
                             //   | (entry within the leaf's list << 25), at the entries' .z
  const float4* pts;         // local (x, y, z, |x|^2), high parts
  const float4* pts_lo;      // low parts of the local coordinates
  const float2* fs;
  float2* us;
  int nrhs;
  // FP32 form only: close-pair corrections, CSR per sorted target point
  const int32_t* close_off;  // [N + 1]
  const int32_t* close_j;    // source point of each correction
  const float2* close_w;     // G(p_i, p_j) - (the FP32 form's value for the pair)
};
// Double-float coordinates throughout (any accuracy).
void launch_p2p(const P2PArgs& a, cudaStream_t s);
// FP32 coordinates (high parts) throughout, then the close-pair corrections.
void launch_p2p_fast(const P2PArgs& a, int64_t npoints, cudaStream_t s);
// Close pairs of the FP32 form: every (target i, source j) of the U lists with
// FP32 distance below delta and p_j != p_i.  Pass 1 (off == nullptr): counts per
// target point into cnt[N], and sets *degenerate if two distinct points have FP32
// distance 0.  Pass 2: fills j and w at the CSR offsets off[N + 1].
void launch_p2p_close(const P2PArgs& a, float delta, int32_t* cnt, unsigned* degenerate, const int32_t* off,
                      int32_t* close_j, float2* close_w, cudaStream_t s);

// FP64 forms (apply64.cu), for eps < 1e-6: the same argument structs, with
// every complex array (operators, rows, states, densities, potentials)
// holding complex128 (double2) elements at the same indices.  Representation
// ranks up to 512; the check-point form needs P2CArgs.chk64 and .pts_lo.
void launch_gemm_stage64(const GemmArgs& a, cudaStream_t s);
void launch_permute_in64(const float2* f, const int32_t* perm, int64_t N, int nrhs, float2* fs, cudaStream_t s);
void launch_permute_out64(const float2* us, const int32_t* perm, int64_t N, int nrhs, float2* u, cudaStream_t s);
void launch_p2c64(const P2CArgs& a, cudaStream_t s);
void launch_rows64(const RowsArgs& a, cudaStream_t s);
void launch_l2p64(const L2PArgs& a, cudaStream_t s);
void launch_p2m_rows64(const P2MRowsArgs& a, cudaStream_t s);
void launch_p2p64(const P2PArgs& a, cudaStream_t s);

}  // namespace dfmm
