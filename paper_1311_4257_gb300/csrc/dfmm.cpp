// C ABI of the directional FMM (include/dfmm.h): plan construction and the
// apply sequence of Alg. 1 plus the near field.
//
// Plan: Morton keys, radix sort, octree and list enumeration run on the
// device (sort.cu, tree.cu); the host groups the lists into per-operator work
// tables and draws the skeleton samples, the device selects the skeletons
// (skeleton_gpu.cu; host threads with options.skeleton_host) and forms the
// operators and evaluation rows in FP64 (operators.cu).
// Apply (one stream, no host synchronisation): permute in, P2M, LF-M2M, the
// top V list, then per HF level HF-M2M and HF-M2L, HF-L2L, HF->LF L2L, LF-L2L
// and LF-M2L (V), P2L (X), L2P, M2P (W), P2P (U), permute out.  The tensor-core
// (m2l_cx.cu, m2l_tc.cu), FP32 (apply.cu) and FP64 (apply64.cu) kernels serve
// the three arithmetic forms.  Also here: the allocation-free and captured
// applies, the batched forms, dfmm_validate and the live-plan registry.
#include "dfmm.h"

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_set>
#include <string>
#include <unordered_map>
#include <vector>

#include "apply.h"
#include "common.h"
#include "internal.h"
#include "operators.h"
#include "skeleton.h"
#include "validate.h"
#include "tree.h"

using namespace dfmm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// Live plans and the number of server requests that hold each one: a handle
// that is not in the map is not a plan (never created, or destroyed), and a
// plan with holders is not destroyed.
std::mutex g_plans_mu;
std::unordered_map<const void*, int64_t> g_plans;
int64_t g_next_plan_id = 1;   // under g_plans_mu

struct GemmPlan {
  int M = 0, Kd = 0, nops = 0;
  float2* ops = nullptr;
  std::vector<int4> groups;        // (op, first pair, count, 0)
  int2* pairs = nullptr;
  std::vector<int32_t> h_dst;      // target row of every pair (host), for tile ordering
  bool dst_unique = false;         // no two pairs share a target row
  int64_t npairs = 0;
  int fam = 0;                     // profiling family
  __half* img = nullptr;           // tensor-core operator image (tensor form only)
  float* op_scale = nullptr;       // its per-operator power-of-two scales
  double flops_rhs = 0;            // algorithmic flops per right-hand side
  double bytes_fixed = 0;          // operators (bytes once per launch)
  double bytes_rhs = 0;            // unique source rows + target rows (read and write), per rhs
  int64_t src_rows = 0;            // rows of the source buffer (pair .x < src_rows), for dfmm_validate
  int64_t dst_rows = 0;            // rows of the target buffer (pair .y < dst_rows)
};

enum Fam { F_M2L_HF, F_M2L_LF, F_M2M, F_L2L, F_P2L_PROJ, F_P2M_EVAL, F_P2L_EVAL, F_L2P, F_M2P, F_P2P,
           F_PERMUTE, F_ZERO, F_SPLIT, F_COUNT };
const char* kFamName[F_COUNT] = {"m2l_hf", "m2l_lf", "m2m", "l2l", "p2l_proj", "p2m_eval",
                                 "p2l_eval", "l2p", "m2p", "p2p", "permute", "zero", "split"};

// the translation families that m2l_mode 2 runs on the tensor cores (options.tc_stages)
constexpr int kTcFamBit[F_COUNT] = {1, 2, 4, 8, 16, 0, 0, 0, 0, 0, 0, 0, 0};

struct ProfRec {
  int fam;
  cudaEvent_t a, b;
  double flops, bytes;
};

struct HFLevel {
  int l = 0;
  double w = 0;
  int n = 0, nd = 0, R = 0;
  std::vector<int32_t> out_keys, in_keys;       // box * nd + dir, ascending
  std::vector<int32_t> out_map, in_map;         // dense -> slot (-1 if inactive)
  std::vector<int> out_cells, in_cells;         // distinct active directions
  PairList pairs;
  GemmPlan m2m, m2l, l2l;   // into this level: M2M from l+1, M2L, L2L from l-1
};

struct LFLevel {
  int l = 0;
  double w = 0;
  int R = 0, r = 0;
  int64_t nbox = 0;
  GemmPlan m2m, l2l, v, p2l;   // m2m from l+1, l2l from l-1 (LF or HF)
  ChkPt* chk_b2 = nullptr;
  double* chk64 = nullptr;         // FP64 form: the check points b2, [2r][3]
  int4* p2l_jobs = nullptr;
  float4* p2l_shifts = nullptr;
  int64_t n_p2l = 0;
  int4* l2p_jobs = nullptr;
  int64_t n_l2p = 0;
  float2* l2p_rows = nullptr;
  int2* l2p_map = nullptr;         // (point, state row) of every L2P row
  float2* p2m_rows = nullptr;      // outgoing-state rows of the leaf points (same row order as L2P)
  int64_t n_l2p_rows = 0;
  int64_t npts = 0;      // points in the leaves of this level
  int64_t npts_x = 0;    // source points over the X pairs of this level
};

struct M2PGroup {
  int src_level = 0;
  int R = 0;
  int4* jobs = nullptr;
  int64_t njobs = 0;
  float2* rows = nullptr;
  int64_t nrows = 0;
};

struct Workspace {
  int nrhs = 0;
  bool external = false;   // buffers carved from caller-provided memory
  DevArena ar;
  float2 *fs = nullptr, *us = nullptr, *p2l = nullptr;
  __half *ahi = nullptr, *alo = nullptr;                // split source buffer (tensor form)
  float* ascale = nullptr;                              // its per-row scales
  std::vector<float2*> S, T;                            // per level (LF or HF states)
  std::vector<std::pair<void*, size_t>> zero;           // reset before each apply
  std::vector<std::pair<void*, size_t>> zero_late;      // reset on the side stream, first read by HF M2M
  cudaStream_t side = nullptr;                          // for zero_late, beside P2M and the V list
  cudaEvent_t fork = nullptr, join = nullptr;
  std::map<std::pair<const void*, int>, std::pair<int4*, int64_t>> tiles;   // key (stage, nrhs * 1024 + columns)
  float2 *f_dev = nullptr, *u_dev = nullptr;            // staging for host applies
  unsigned* status = nullptr;
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  ~Workspace() {
    for (auto e : pool) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
  }
  cudaEvent_t ev() {
    if (pool_used == pool.size()) {
      cudaEvent_t e;
      DFMM_CUDA(cudaEventCreate(&e));
      pool.push_back(e);
    }
    return pool[pool_used++];
  }
};

struct ProfScope {
  Workspace* W;
  cudaStream_t s;
  ProfRec r{};
  ProfScope(Workspace* w, cudaStream_t st, int fam, double flops, double bytes) : W(w), s(st) {
    if (!W->prof) return;
    r.fam = fam;
    r.flops = flops;
    r.bytes = bytes;
    r.a = W->ev();
    r.b = W->ev();
    DFMM_CUDA(cudaEventRecord(r.a, s));
  }
  ~ProfScope() {
    if (!W->prof) return;
    cudaEventRecord(r.b, s);
    W->recs.push_back(r);
  }
};

}  // namespace

struct dfmm_plan_s {
  int device = 0;
  int64_t N = 0;
  double K = 0, W = 0, eps = 0, eps_op = 0;
  dfmm_options opt{};
  bool fp64 = false;   // FP64 form (options.arith 64): complex128 densities, states and operators
  int cw = 1;          // complex element width in float2 units (2 in the FP64 form)
  DevArena ar;
  TreeBuilder tree;
  int32_t* perm = nullptr;
  std::vector<int32_t> h_perm;
  std::vector<uint64_t> h_keys;
  float4* pts_local = nullptr;
  float4* pts_lo = nullptr;
  int l1 = -1, l_top = -1, l_lf0 = -1, nl = 0;
  std::vector<HFLevel> hf;
  std::vector<LFLevel> lf;
  std::vector<PairList> vlist;
  std::vector<int32_t> U, Wl, X;
  std::vector<M2PGroup> m2p;
  int2* p2p_range = nullptr;
  int64_t* p2p_off = nullptr;
  int4* p2p_src = nullptr;
  float4* p2p_shift = nullptr;
  uint32_t* p2p_flat = nullptr;   // FP32 near field: flat staging list
  int64_t n_flat = 0;
  int32_t* close_off = nullptr;   // FP32 near field: close-pair corrections (CSR per sorted point)
  int32_t* close_j = nullptr;
  float2* close_w = nullptr;
  int64_t n_close = 0;
  double close_delta = 0;
  std::unique_ptr<DevArena> close_keep;   // their storage (allocated after a scratch mark of the plan arena)
  int64_t n_leaves = 0;
  float4* zero_shift = nullptr;
  std::unique_ptr<RepSet> reps;
  std::vector<std::array<int64_t, 3>> rep_ranks;   // (level, cell, rank)
  dfmm_stats stats{};
  std::mutex ws_mu;
  std::map<cudaStream_t, std::unique_ptr<Workspace>> ws;
};

// A captured apply: the CUDA graph of run_apply on fixed buffers, with its own
// workspace (laid out once, reused by every launch).
struct dfmm_graph_s {
  dfmm_plan_s* plan = nullptr;
  DevArena ar;
  char* scratch = nullptr;
  size_t bytes = 0;
  Workspace W;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~dfmm_graph_s() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

namespace {

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// The 48 signed permutations of the skeleton code as a group: inverse,
// composition (mul[a][b] = a after b) and action on integer vectors, with
// y_k = sign_k x_perm_k.
struct SymTables {
  int inv[48];
  int mul[48][48];
  int perm[48][3], sign[48][3];
  void apply(int s, const int64_t* x, int64_t* y) const {
    for (int k = 0; k < 3; ++k) y[k] = sign[s][k] * x[perm[s][k]];
  }
};

const SymTables& sym_tables() {
  static SymTables T = [] {
    SymTables t;
    const auto& syms = symmetries();
    auto index_of = [&](const int* pm, const int* sg) {
      for (int s = 0; s < 48; ++s) {
        bool eq = true;
        for (int k = 0; k < 3; ++k) eq = eq && syms[s].perm[k] == pm[k] && syms[s].sign[k] == sg[k];
        if (eq) return s;
      }
      throw Error(DFMM_ERR_INVALID, "symmetry table is not closed");
    };
    for (int s = 0; s < 48; ++s)
      for (int k = 0; k < 3; ++k) { t.perm[s][k] = syms[s].perm[k]; t.sign[s][k] = syms[s].sign[k]; }
    for (int a = 0; a < 48; ++a) {
      int pm[3], sg[3];
      for (int k = 0; k < 3; ++k) { pm[t.perm[a][k]] = k; sg[t.perm[a][k]] = t.sign[a][k]; }
      t.inv[a] = index_of(pm, sg);
      for (int b = 0; b < 48; ++b) {
        int pc[3], sc[3];
        for (int k = 0; k < 3; ++k) { pc[k] = t.perm[b][t.perm[a][k]]; sc[k] = t.sign[a][k] * t.sign[b][t.perm[a][k]]; }
        t.mul[a][b] = index_of(pc, sc);
      }
    }
    return t;
  }();
  return T;
}

std::vector<int32_t> near_template(double w) {
  int R = (int)std::ceil(w) + 1;
  int64_t lim = std::llround(4 * w * w);
  std::vector<int32_t> t;
  for (int x = -R; x <= R; ++x)
    for (int y = -R; y <= R; ++y)
      for (int z = -R; z <= R; ++z) {
        int64_t a = std::max(0, 2 * std::abs(x) - 1), b = std::max(0, 2 * std::abs(y) - 1),
                c = std::max(0, 2 * std::abs(z) - 1);
        if (a * a + b * b + c * c <= lim) { t.push_back(x); t.push_back(y); t.push_back(z); }
      }
  return t;
}

std::vector<int32_t> colleague_template() {
  std::vector<int32_t> t;
  for (int x = -1; x <= 1; ++x)
    for (int y = -1; y <= 1; ++y)
      for (int z = -1; z <= 1; ++z) { t.push_back(x); t.push_back(y); t.push_back(z); }
  return t;
}

// Fig. 2 hierarchy: cell (f, i, j) of the parent grid lies in (f, i/2, j/2).
int parent_cell(int d, int n_parent) {
  int f = d / (n_parent * n_parent), rem = d % (n_parent * n_parent);
  int i = rem / n_parent, j = rem % n_parent;
  int nc = n_parent / 2;
  return (f * nc + i / 2) * nc + j / 2;
}

int octant_of(const int32_t* c) { return ((c[0] & 1) << 2) | ((c[1] & 1) << 1) | (c[2] & 1); }

// c_child - c_parent for octant o
void octant_delta(int o, double w_child, double out[3]) {
  out[0] = (((o >> 2) & 1) - 0.5) * w_child;
  out[1] = (((o >> 1) & 1) - 0.5) * w_child;
  out[2] = ((o & 1) - 0.5) * w_child;
}

// (op, src, dst) triples -> GemmPlan with pairs grouped by operator
void finish_gemm(GemmPlan& g, const std::vector<int32_t>& op, const std::vector<int2>& pr, DevArena& ar,
                 cudaStream_t s) {
  int64_t n = (int64_t)op.size();
  g.npairs = n;
  g.groups.clear();
  if (n == 0) return;
  {
    // unique rows touched, for the algorithmic byte count
    std::vector<int32_t> a(n), b(n);
    for (int64_t i = 0; i < n; ++i) { a[i] = pr[i].x; b[i] = pr[i].y; }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    int64_t ua = std::unique(a.begin(), a.end()) - a.begin(), ub = std::unique(b.begin(), b.end()) - b.begin();
    std::vector<uint8_t> used(g.nops, 0);
    for (int64_t i = 0; i < n; ++i) used[op[i]] = 1;
    int64_t uops = 0;
    for (auto u : used) uops += u;
    g.bytes_fixed = (double)uops * g.M * g.Kd * 8.0;
    g.bytes_rhs = (double)ua * g.Kd * 8.0 + 2.0 * (double)ub * g.M * 8.0;
    g.dst_unique = ub == n;
  }
  std::vector<int64_t> cnt(g.nops + 1, 0);
  for (int64_t i = 0; i < n; ++i) cnt[op[i] + 1]++;
  for (int k = 0; k < g.nops; ++k) cnt[k + 1] += cnt[k];
  std::vector<int2> sorted(n);
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  for (int64_t i = 0; i < n; ++i) sorted[pos[op[i]]++] = pr[i];
  for (int k = 0; k < g.nops; ++k)
    if (cnt[k + 1] > cnt[k]) g.groups.push_back(make_int4(k, (int)cnt[k], (int)(cnt[k + 1] - cnt[k]), 0));
  g.pairs = ar.alloc<int2>(n);
  DFMM_CUDA(cudaMemcpyAsync(g.pairs, sorted.data(), n * sizeof(int2), cudaMemcpyHostToDevice, s));
  g.h_dst.resize(n);
  for (int64_t i = 0; i < n; ++i) g.h_dst[i] = sorted[i].y;
  DFMM_CUDA(cudaStreamSynchronize(s));
}

template <class T>
T* upload(const std::vector<T>& v, DevArena& ar, cudaStream_t s) {
  T* d = ar.alloc<T>(std::max<size_t>(1, v.size()));
  if (!v.empty()) DFMM_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  DFMM_CUDA(cudaStreamSynchronize(s));
  return d;
}

// conjugate transpose of a 2r x r matrix, columns scaled, padded to R x 2R:
// complex64, or complex128 for the FP64 form
float2* upload_projection(const std::vector<cd>& Q, int r, const double* colscale, int R, bool fp64, DevArena& ar,
                          cudaStream_t s) {
  std::vector<double2> h((size_t)R * 2 * R, make_double2(0, 0));
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < 2 * r; ++j) {
      cd v = std::conj(Q[(size_t)j * r + i]);
      if (colscale) v *= colscale[j];
      h[(size_t)i * 2 * R + j] = make_double2(v.real(), v.imag());
    }
  if (fp64) return (float2*)upload(h, ar, s);
  std::vector<float2> f(h.size());
  for (size_t i = 0; i < h.size(); ++i) f[i] = make_float2((float)h[i].x, (float)h[i].y);
  return upload(f, ar, s);
}

ChkPt* upload_chk(const std::vector<double>& pts, int n, DevArena& ar, cudaStream_t s) {
  std::vector<ChkPt> h(n);
  for (int p = 0; p < n; ++p) {
    double x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
    double n2 = x * x + y * y + z * z, nn = std::sqrt(n2);
    h[p].x = (float)x; h[p].y = (float)y; h[p].z = (float)z;
    h[p].nx2 = (float)n2;
    h[p].nx = (float)nn;
    h[p].fx = (float)(nn - std::floor(nn));
    h[p].pad0 = h[p].pad1 = 0.f;
  }
  return upload(h, ar, s);
}

void build_plan(dfmm_plan_s* P, const double* d_points, cudaStream_t s) {
  double t0 = now();
  const int64_t N = P->N;
  DevArena& ar = P->ar;
  // ---- host copy of the points, domain check
  std::vector<double> hp((size_t)N * 3);
  DFMM_CUDA(cudaMemcpy(hp.data(), d_points, N * 24, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < 3 * N; ++i)
    if (!(std::fabs(hp[i]) <= 0.5 * P->K))
      throw Error(DFMM_ERR_DOMAIN, "point " + std::to_string(i / 3) + " lies outside |x|_inf <= K/2");
  // ---- Morton keys and stable radix sort (device)
  uint64_t* keys = ar.alloc<uint64_t>(N);
  P->perm = ar.alloc<int32_t>(N);
  {
    ArenaMark mk(ar);
    double* dp = ar.alloc<double>(3 * N);
    DFMM_CUDA(cudaMemcpyAsync(dp, d_points, N * 24, cudaMemcpyDeviceToDevice, s));
    uint64_t* k2 = ar.alloc<uint64_t>(N);
    int32_t* v2 = ar.alloc<int32_t>(N);
    size_t sb = radix_sort_scratch_bytes(N);
    void* scratch = ar.alloc<char>(sb);
    launch_morton_keys(dp, N, P->W, keys, P->perm, s);
    radix_sort_pairs(keys, P->perm, k2, v2, N, 63, scratch, sb, s);
    DFMM_CUDA(cudaStreamSynchronize(s));
  }
  P->h_perm.resize(N);
  P->h_keys.resize(N);
  DFMM_CUDA(cudaMemcpy(P->h_perm.data(), P->perm, N * 4, cudaMemcpyDeviceToHost));
  DFMM_CUDA(cudaMemcpy(P->h_keys.data(), keys, N * 8, cudaMemcpyDeviceToHost));
  // ---- octree (device)
  TreeBuilder& T = P->tree;
  T.build(keys, N, P->W, P->opt.leaf_max, s, ar);
  const int nl = (int)T.levels.size();
  const std::vector<TreeLevel>& LV = T.levels;
  P->nl = nl;
  P->stats.n_levels = nl;
  for (int l = 0; l < nl && l < 32; ++l) {
    P->stats.boxes[l] = LV[l].n;
    int64_t nleaf = 0;
    for (auto v : LV[l].h_leaf) nleaf += v;
    P->stats.leaves[l] = nleaf;
  }
  P->l1 = (int)std::llround(std::log2(P->W));
  P->stats.level_w1 = P->l1;
  P->l_lf0 = P->l1 + 1;
  if (P->l_lf0 >= nl) throw Error(DFMM_ERR_INVALID, "octree has no low-frequency level");
  unsigned* d_status = ar.alloc<unsigned>(1);
  DFMM_CUDA(cudaMemsetAsync(d_status, 0, 4, s));
  // ---- HF lists (device)
  P->hf.resize(nl);
  for (int l = 1; l <= P->l1; ++l) {
    HFLevel& H = P->hf[l];
    H.l = l;
    H.w = LV[l].w;
    H.n = n_cells(H.w);
    H.nd = 6 * H.n * H.n;
    // Prop. 1 with |p|_inf <= K/2: two data points are at most sqrt(3) K apart and
    // a box centre lies within sqrt(3) w / 2 of one of its points, so for
    // w^2 >= sqrt(3) (K + w / 2) every non-empty box is near and I^B is empty.
    if (H.w * H.w >= std::sqrt(3.0) * (P->K + 0.5 * H.w)) continue;
    H.pairs = T.pairs(l, near_template(2 * H.w), 0, std::llround(4 * H.w * H.w), true, H.n, s, ar);
    if (H.pairs.n > 0 && P->l_top < 0) P->l_top = l;
    P->stats.hf_pairs[l] = H.pairs.n;
  }
  P->stats.level_hf_top = P->l_top;
  // ---- LF lists (device)
  P->lf.resize(nl);
  P->vlist.resize(nl);
  for (int l = P->l_lf0; l < nl; ++l) {
    P->vlist[l] = T.pairs(l, colleague_template(), 1, 0, false, 0, s, ar);
    P->stats.v_pairs += P->vlist[l].n;
  }
  T.uw_lists(P->l_lf0, s, ar, P->U, P->Wl, d_status);
  {
    unsigned st = 0;
    DFMM_CUDA(cudaMemcpy(&st, d_status, 4, cudaMemcpyDeviceToHost));
    if (st) throw Error(DFMM_ERR_DEVICE, "list construction overflowed its descent stack");
  }
  const size_t nU = P->U.size() / 4, nW = P->Wl.size() / 4;
  P->X.resize(4 * nW);
  for (size_t q = 0; q < nW; ++q) {
    P->X[4 * q] = P->Wl[4 * q + 2];
    P->X[4 * q + 1] = P->Wl[4 * q + 3];
    P->X[4 * q + 2] = P->Wl[4 * q];
    P->X[4 * q + 3] = P->Wl[4 * q + 1];
  }
  P->stats.u_pairs = (int64_t)nU;
  P->stats.w_pairs = (int64_t)nW;
  P->stats.x_pairs = (int64_t)nW;
  // ---- active directions (closure under the wedge hierarchy)
  const bool has_hf = P->l_top >= 0;
  if (has_hf) {
    for (int l = P->l_top; l <= P->l1; ++l) {
      HFLevel& H = P->hf[l];
      const TreeLevel& L = LV[l];
      std::vector<uint8_t> fo((size_t)L.n * H.nd, 0), fi((size_t)L.n * H.nd, 0);
      for (int64_t q = 0; q < H.pairs.n; ++q) {
        fo[(size_t)H.pairs.src[q] * H.nd + H.pairs.dout[q]] = 1;
        fi[(size_t)H.pairs.tgt[q] * H.nd + H.pairs.din[q]] = 1;
      }
      if (l > P->l_top) {
        const HFLevel& Hp = P->hf[l - 1];
        const TreeLevel& Lp = LV[l - 1];
        for (int pass = 0; pass < 2; ++pass) {
          const std::vector<int32_t>& kp = pass == 0 ? Hp.out_keys : Hp.in_keys;
          std::vector<uint8_t>& f = pass == 0 ? fo : fi;
          for (int32_t key : kp) {
            int pb = key / Hp.nd, pd = key % Hp.nd;
            int cd = parent_cell(pd, Hp.n);
            for (int k = 0; k < Lp.h_nchild[pb]; ++k) f[(size_t)(Lp.h_child_first[pb] + k) * H.nd + cd] = 1;
          }
        }
      }
      H.out_map.assign(fo.size(), -1);
      H.in_map.assign(fi.size(), -1);
      std::vector<uint8_t> co(H.nd, 0), ci(H.nd, 0);
      for (size_t k = 0; k < fo.size(); ++k) {
        if (fo[k]) { H.out_map[k] = (int32_t)H.out_keys.size(); H.out_keys.push_back((int32_t)k); co[k % H.nd] = 1; }
        if (fi[k]) { H.in_map[k] = (int32_t)H.in_keys.size(); H.in_keys.push_back((int32_t)k); ci[k % H.nd] = 1; }
      }
      for (int d = 0; d < H.nd; ++d) {
        if (co[d]) H.out_cells.push_back(d);
        if (ci[d]) H.in_cells.push_back(d);
      }
      P->stats.slots_out[l] = (int64_t)H.out_keys.size();
      P->stats.slots_in[l] = (int64_t)H.in_keys.size();
    }
  }
  double* ph = P->stats.plan_phase_seconds;
  double tp = t0;
  auto phase = [&](int k) { const double t = now(); ph[k] += t - tp; tp = t; };
  phase(0);
  // ---- representations (host skeletons, built in parallel)
  double w_top = has_hf ? LV[P->l_top].w : 1.0;
  SkelParams sp;
  sp.eps_op = P->eps_op;
  sp.S_Y = P->opt.sample_box;
  sp.S_X = P->opt.sample_far;
  sp.sketch = P->opt.sketch_rows;
  P->reps.reset(new RepSet(sp, w_top, P->opt.host_threads, P->opt.cache_dir ? P->opt.cache_dir : "",
                           P->opt.skeleton_host == 0));
  std::vector<std::vector<int>> level_cells(nl);
  std::vector<std::pair<double, int>> need;
  for (int l = (has_hf ? P->l_top : P->l_lf0); l < nl; ++l) {
    if (l <= P->l1) {
      std::vector<uint8_t> used(P->hf[l].nd, 0);
      for (int d : P->hf[l].out_cells) used[d] = 1;
      for (int d : P->hf[l].in_cells) used[d] = 1;
      for (int d = 0; d < P->hf[l].nd; ++d) if (used[d]) level_cells[l].push_back(d);
    } else {
      level_cells[l].push_back(-1);
    }
    for (int c : level_cells[l]) need.push_back({LV[l].w, c});
  }
  P->reps->prepare(need);
  phase(1);
  for (int k = 0; k < 4; ++k) P->stats.skeleton_phase_seconds[k] = P->reps->seconds[k];
  P->stats.skeleton_types = (int64_t)P->reps->built();
  std::vector<DevRep> dreps;
  std::map<std::pair<int, int>, int> ridx;   // (level, cell) -> dreps index
  for (int l = (has_hf ? P->l_top : P->l_lf0); l < nl; ++l) {
    int rmax = 0;
    for (int c : level_cells[l]) rmax = std::max(rmax, P->reps->get(LV[l].w, c).r);
    // ranks padded to 8; to 16 for the split-complex tensor-core form (the MMA's N and K steps)
    const int pad = (P->opt.m2l_mode == 2 && P->opt.tc_layout != 1) ? 16 : 8;
    int R = round_up(std::max(rmax, pad), pad);
    // the FP32 row kernels take ranks up to 256, the FP64 form's up to 512
    if (R > (P->fp64 ? 512 : 256))
      throw Error(DFMM_ERR_UNSUPPORTED, P->fp64 ? "representation rank above 512" : "representation rank above 256");
    if (l <= P->l1) P->hf[l].R = R;
    else { P->lf[l].R = R; P->lf[l].r = rmax; }
    P->stats.rank[l] = R;
    for (int c : level_cells[l]) {
      const Rep& rp = P->reps->get(LV[l].w, c);
      ridx[{l, c}] = (int)dreps.size();
      dreps.push_back(upload_rep(rp, R, ar, s));
      P->rep_ranks.push_back({(int64_t)l, (int64_t)c, (int64_t)rp.r});
    }
  }
  // ranks per (level, cell), looked up once: the flop counts below take two per pair
  std::vector<std::vector<int>> rank_cache(nl);
  auto rank_of = [&](int l, int cell) {
    std::vector<int>& v = rank_cache[l];
    const size_t i = (size_t)(cell + 1);   // the LF type (cell -1) at 0
    if (i >= v.size()) v.resize(i + 1, -1);
    if (v[i] < 0) v[i] = P->reps->get(LV[l].w, cell).r;
    return v[i];
  };
  // operator formation on the device (FP64 kernel blocks and products), timed
  // apart within phase 3
  auto timed_form = [&](OpKind kind, const std::vector<OpSpec>& sp, const std::vector<DevRep>& dr, int Rt, int Rs,
                        void* out, bool fp64) {
    const double t = now();
    form_ops(kind, sp, dr, Rt, Rs, out, fp64, ar, s);
    ph[7] += now() - t;
  };
  double m2l_flops = 0, other_flops = 0;
  auto center = [&](int l, int64_t b, int d) { return -0.5 * P->W + (LV[l].h_coords[3 * b + d] + 0.5) * LV[l].w; };
  P->zero_shift = upload(std::vector<float4>{make_float4(0, 0, 0, 0)}, ar, s);

  phase(2);
  // ---- LF levels
  for (int l = P->l_lf0; l < nl; ++l) {
    LFLevel& F = P->lf[l];
    F.l = l;
    F.w = LV[l].w;
    F.nbox = LV[l].n;
    const Rep& rp = P->reps->get(F.w, -1);
    const int R = F.R;
    F.chk_b2 = upload_chk(rp.b2, 2 * rp.r, ar, s);
    if (P->fp64) F.chk64 = upload(rp.b2, ar, s);
    F.p2l.M = R; F.p2l.Kd = 2 * R; F.p2l.nops = 1;
    F.p2l.ops = upload_projection(rp.Qi, rp.r, nullptr, R, P->fp64, ar, s);
    std::vector<int4> jobs;
    std::vector<int32_t> op;
    std::vector<int2> pr;
    // P2M: leaves of this level, through per-point rows (formed with the L2P
    // rows below)
    for (int64_t b = 0; b < LV[l].n; ++b)
      if (LV[l].h_leaf[b]) F.npts += LV[l].h_count[b];
    other_flops += 8.0 * rp.r * F.npts;
    // P2L: X pairs whose target is at this level
    {
      std::vector<int4> xj;
      std::vector<float4> xs;
      op.clear(); pr.clear();
      for (size_t q = 0; q < nW; ++q) {
        int lb = P->X[4 * q], b = P->X[4 * q + 1], la = P->X[4 * q + 2], a = P->X[4 * q + 3];
        if (lb != l) continue;
        float sh[3];
        for (int d = 0; d < 3; ++d) sh[d] = (float)(center(la, a, d) - center(lb, b, d));
        xs.push_back(make_float4(sh[0], sh[1], sh[2], 0.f));
        xj.push_back(make_int4(LV[la].h_first[a], LV[la].h_count[a], (int)xj.size(), (int)xs.size() - 1));
        op.push_back(0);
        pr.push_back(make_int2((int)xj.size() - 1, b));
      }
      F.n_p2l = (int64_t)xj.size();
      for (auto& j : xj) F.npts_x += j.x >= 0 ? j.y : 0;
      F.p2l_jobs = upload(xj, ar, s);
      F.p2l_shifts = upload(xs, ar, s);
      F.p2l.fam = F_P2L_PROJ;
      F.p2l.flops_rhs = 8.0 * rp.r * 2 * rp.r * F.n_p2l;
      F.p2l.src_rows = F.n_p2l;
      F.p2l.dst_rows = LV[l].n;
      finish_gemm(F.p2l, op, pr, ar, s);
    }
    // LF-M2L over the V list: one operator per offset
    {
      const PairList& V = P->vlist[l];
      std::map<std::array<int, 3>, int> offs;
      std::vector<OpSpec> specs;
      op.clear(); pr.clear();
      for (int64_t q = 0; q < V.n; ++q) {
        std::array<int, 3> m = {V.m[3 * q], V.m[3 * q + 1], V.m[3 * q + 2]};
        auto it = offs.find(m);
        int id;
        if (it == offs.end()) {
          id = (int)specs.size();
          offs[m] = id;
          OpSpec o;
          o.tgt_rep = o.src_rep = ridx.at({l, -1});
          for (int d = 0; d < 3; ++d) o.shift[d] = -F.w * m[d];
          specs.push_back(o);
        } else id = it->second;
        op.push_back(id);
        pr.push_back(make_int2(V.src[q], V.tgt[q]));
      }
      F.v.M = R; F.v.Kd = R; F.v.nops = (int)specs.size();
      if (!specs.empty()) {
        F.v.ops = ar.alloc<float2>(((size_t)specs.size() * R * R) * P->cw);
        timed_form(kOpM2L, specs, dreps, R, R, F.v.ops, P->fp64);
      }
      F.v.fam = F_M2L_LF;
      F.v.flops_rhs = 8.0 * rp.r * rp.r * V.n;
      F.v.src_rows = F.v.dst_rows = LV[l].n;
      finish_gemm(F.v, op, pr, ar, s);
      m2l_flops += 8.0 * rp.r * rp.r * V.n;
    }
    // LF-M2M from level l+1 (LF children) and LF-L2L from level l-1 (LF parent)
    if (l + 1 < nl) {
      const LFLevel& C = P->lf[l + 1];
      const TreeLevel& Lc = LV[l + 1];
      std::vector<OpSpec> specs(8);
      for (int o = 0; o < 8; ++o) {
        double dl[3];
        octant_delta(o, Lc.w, dl);
        specs[o].tgt_rep = ridx.at({l, -1});
        specs[o].src_rep = ridx.at({l + 1, -1});
        for (int d = 0; d < 3; ++d) specs[o].shift[d] = -dl[d];
      }
      int Rc = P->lf[l + 1].R;
      (void)C;
      F.m2m.M = R; F.m2m.Kd = Rc; F.m2m.nops = 8;
      F.m2m.ops = ar.alloc<float2>(((size_t)8 * R * Rc) * P->cw);
      timed_form(kOpM2M, specs, dreps, R, Rc, F.m2m.ops, P->fp64);
      op.clear(); pr.clear();
      for (int64_t c = 0; c < Lc.n; ++c) {
        op.push_back(octant_of(&Lc.h_coords[3 * c]));
        pr.push_back(make_int2((int)c, Lc.h_parent[c]));
      }
      F.m2m.fam = F_M2M;
      F.m2m.flops_rhs = 8.0 * rp.r * P->lf[l + 1].r * Lc.n;
      F.m2m.src_rows = Lc.n;
      F.m2m.dst_rows = LV[l].n;
      finish_gemm(F.m2m, op, pr, ar, s);
      other_flops += F.m2m.flops_rhs;
    }
    if (l > P->l_lf0) {
      const TreeLevel& Lp = LV[l - 1];
      const int Rp = P->lf[l - 1].R;
      std::vector<OpSpec> specs(8);
      for (int o = 0; o < 8; ++o) {
        double dl[3];
        octant_delta(o, F.w, dl);
        specs[o].tgt_rep = ridx.at({l, -1});
        specs[o].src_rep = ridx.at({l - 1, -1});
        for (int d = 0; d < 3; ++d) specs[o].shift[d] = dl[d];
      }
      F.l2l.M = R; F.l2l.Kd = Rp; F.l2l.nops = 8;
      F.l2l.ops = ar.alloc<float2>(((size_t)8 * R * Rp) * P->cw);
      timed_form(kOpL2L, specs, dreps, R, Rp, F.l2l.ops, P->fp64);
      op.clear(); pr.clear();
      for (int64_t c = 0; c < LV[l].n; ++c) {
        op.push_back(octant_of(&LV[l].h_coords[3 * c]));
        pr.push_back(make_int2(LV[l].h_parent[c], (int)c));
      }
      F.l2l.fam = F_L2L;
      F.l2l.flops_rhs = 8.0 * rp.r * P->lf[l - 1].r * LV[l].n;
      F.l2l.src_rows = LV[l - 1].n;
      F.l2l.dst_rows = LV[l].n;
      finish_gemm(F.l2l, op, pr, ar, s);
      other_flops += F.l2l.flops_rhs;
      (void)Lp;
    }
  }

  // ---- HF levels
  if (has_hf) {
    for (int l = P->l_top; l <= P->l1; ++l) {
      HFLevel& H = P->hf[l];
      const TreeLevel& L = LV[l];
      const int R = H.R;
      std::vector<int32_t> op;
      std::vector<int2> pr;
      // HF-M2L, one operator per offset m up to the cube's symmetries.  The
      // skeleton of a cell is its orbit's canonical skeleton mapped by a
      // signed permutation tau (points in the same order), and G depends only
      // on distances, so the operator of (m, d_in, d_out) equals that of
      // (tau_in^-1 m, canonical d_in, tau_in^-1 tau_out applied to the
      // canonical d_out): pairs with equal keys share one operator exactly.
      {
        std::unordered_map<int64_t, int> offs;
        std::unordered_set<int64_t> distinct_m;
        std::vector<OpSpec> specs;
        const PairList& Pp = H.pairs;
        int64_t Rm = 8 * (int64_t)std::ceil(H.w) + 8;
        std::vector<int> canon, which;
        canonical_cells(n_cells(H.w), canon, which);
        const SymTables& ST = sym_tables();
        for (int64_t q = 0; q < Pp.n; ++q) {
          int64_t m0 = Pp.m[3 * q], m1 = Pp.m[3 * q + 1], m2 = Pp.m[3 * q + 2];
          distinct_m.insert(((m0 + Rm) * (2 * Rm + 1) + (m1 + Rm)) * (2 * Rm + 1) + (m2 + Rm));
          const int s_in = which[Pp.din[q]], s_out = which[Pp.dout[q]];
          const int inv_in = ST.inv[s_in];
          const int rho = ST.mul[inv_in][s_out];
          int64_t mm[3];
          const int64_t mv[3] = {m0, m1, m2};
          ST.apply(inv_in, mv, mm);
          int64_t key = ((mm[0] + Rm) * (2 * Rm + 1) + (mm[1] + Rm)) * (2 * Rm + 1) + (mm[2] + Rm);
          key = ((key * 48 + rho) * 2048 + canon[Pp.din[q]]) * 2048 + canon[Pp.dout[q]];
          auto it = offs.find(key);
          int id;
          if (it == offs.end()) {
            id = (int)specs.size();
            offs.emplace(key, id);
            OpSpec o;
            o.tgt_rep = ridx.at({l, Pp.din[q]});
            o.src_rep = ridx.at({l, Pp.dout[q]});
            o.shift[0] = -H.w * m0; o.shift[1] = -H.w * m1; o.shift[2] = -H.w * m2;
            specs.push_back(o);
          } else id = it->second;
          op.push_back(id);
          int ss = H.out_map[(size_t)Pp.src[q] * H.nd + Pp.dout[q]];
          int ts = H.in_map[(size_t)Pp.tgt[q] * H.nd + Pp.din[q]];
          pr.push_back(make_int2(ss, ts));
          H.m2l.flops_rhs += 8.0 * rank_of(l, Pp.din[q]) * rank_of(l, Pp.dout[q]);
        }
        m2l_flops += H.m2l.flops_rhs;
        H.m2l.fam = F_M2L_HF;
        P->stats.hf_offsets[l] = (int64_t)distinct_m.size();
        P->stats.hf_ops[l] = (int64_t)specs.size();
        H.m2l.M = R; H.m2l.Kd = R; H.m2l.nops = (int)specs.size();
        if (!specs.empty()) {
          H.m2l.ops = ar.alloc<float2>(((size_t)specs.size() * R * R) * P->cw);
          timed_form(kOpM2L, specs, dreps, R, R, H.m2l.ops, P->fp64);
        }
        H.m2l.src_rows = (int64_t)H.out_keys.size();
        H.m2l.dst_rows = (int64_t)H.in_keys.size();
        finish_gemm(H.m2l, op, pr, ar, s);
      }
      // HF-M2M into this level from its children (level l+1: HF or, at w = 1, LF)
      {
        const bool child_lf = (l == P->l1);
        const TreeLevel& Lc = LV[l + 1];
        const int Rc = child_lf ? P->lf[l + 1].R : P->hf[l + 1].R;
        std::vector<int> cell_id(H.nd, -1);
        for (size_t k = 0; k < H.out_cells.size(); ++k) cell_id[H.out_cells[k]] = (int)k;
        std::vector<OpSpec> specs;
        for (int d : H.out_cells)
          for (int o = 0; o < 8; ++o) {
            double dl[3];
            octant_delta(o, Lc.w, dl);
            OpSpec sp2;
            sp2.tgt_rep = ridx.at({l, d});
            sp2.src_rep = child_lf ? ridx.at({l + 1, -1}) : ridx.at({l + 1, parent_cell(d, H.n)});
            for (int q = 0; q < 3; ++q) sp2.shift[q] = -dl[q];
            specs.push_back(sp2);
          }
        H.m2m.M = R; H.m2m.Kd = Rc; H.m2m.nops = (int)specs.size();
        H.m2m.ops = ar.alloc<float2>((std::max<size_t>(1, specs.size()) * R * Rc) * P->cw);
        timed_form(kOpM2M, specs, dreps, R, Rc, H.m2m.ops, P->fp64);
        op.clear(); pr.clear();
        for (size_t k = 0; k < H.out_keys.size(); ++k) {
          int b = H.out_keys[k] / H.nd, d = H.out_keys[k] % H.nd;
          for (int c = 0; c < L.h_nchild[b]; ++c) {
            int ch = L.h_child_first[b] + c;
            int srow;
            if (child_lf) srow = ch;
            else {
              const HFLevel& Hc = P->hf[l + 1];
              srow = Hc.out_map[(size_t)ch * Hc.nd + parent_cell(d, H.n)];
            }
            op.push_back(cell_id[d] * 8 + octant_of(&Lc.h_coords[3 * ch]));
            pr.push_back(make_int2(srow, (int)k));
            H.m2m.flops_rhs += 8.0 * rank_of(l, d) * (child_lf ? P->lf[l + 1].r : rank_of(l + 1, parent_cell(d, H.n)));
          }
        }
        H.m2m.fam = F_M2M;
        H.m2m.src_rows = l == P->l1 ? LV[l + 1].n : (int64_t)P->hf[l + 1].out_keys.size();
        H.m2m.dst_rows = (int64_t)H.out_keys.size();
        finish_gemm(H.m2m, op, pr, ar, s);
        other_flops += H.m2m.flops_rhs;
      }
      // HF-L2L into this level from its parent (l > l_top)
      if (l > P->l_top) {
        const HFLevel& Hp = P->hf[l - 1];
        const TreeLevel& Lp = LV[l - 1];
        std::vector<int> cell_id(Hp.nd, -1);
        for (size_t k = 0; k < Hp.in_cells.size(); ++k) cell_id[Hp.in_cells[k]] = (int)k;
        std::vector<OpSpec> specs;
        for (int d : Hp.in_cells)
          for (int o = 0; o < 8; ++o) {
            double dl[3];
            octant_delta(o, H.w, dl);
            OpSpec sp2;
            sp2.tgt_rep = ridx.at({l, parent_cell(d, Hp.n)});
            sp2.src_rep = ridx.at({l - 1, d});
            for (int q = 0; q < 3; ++q) sp2.shift[q] = dl[q];
            specs.push_back(sp2);
          }
        H.l2l.M = R; H.l2l.Kd = Hp.R; H.l2l.nops = (int)specs.size();
        H.l2l.ops = ar.alloc<float2>((std::max<size_t>(1, specs.size()) * R * Hp.R) * P->cw);
        timed_form(kOpL2L, specs, dreps, R, Hp.R, H.l2l.ops, P->fp64);
        op.clear(); pr.clear();
        for (size_t k = 0; k < Hp.in_keys.size(); ++k) {
          int b = Hp.in_keys[k] / Hp.nd, d = Hp.in_keys[k] % Hp.nd;
          for (int c = 0; c < Lp.h_nchild[b]; ++c) {
            int ch = Lp.h_child_first[b] + c;
            int trow = H.in_map[(size_t)ch * H.nd + parent_cell(d, Hp.n)];
            op.push_back(cell_id[d] * 8 + octant_of(&L.h_coords[3 * ch]));
            pr.push_back(make_int2((int)k, trow));
            H.l2l.flops_rhs += 8.0 * rank_of(l, parent_cell(d, Hp.n)) * rank_of(l - 1, d);
          }
        }
        H.l2l.fam = F_L2L;
        H.l2l.src_rows = (int64_t)P->hf[l - 1].in_keys.size();
        H.l2l.dst_rows = (int64_t)H.in_keys.size();
        finish_gemm(H.l2l, op, pr, ar, s);
        other_flops += H.l2l.flops_rhs;
      }
    }
    // HF-L2L from w = 1 into the LF incoming states (summed over directions)
    {
      const int l = P->l_lf0;
      LFLevel& F = P->lf[l];
      const HFLevel& Hp = P->hf[P->l1];
      const TreeLevel& Lp = LV[P->l1];
      std::vector<int> cell_id(Hp.nd, -1);
      for (size_t k = 0; k < Hp.in_cells.size(); ++k) cell_id[Hp.in_cells[k]] = (int)k;
      std::vector<OpSpec> specs;
      for (int d : Hp.in_cells)
        for (int o = 0; o < 8; ++o) {
          double dl[3];
          octant_delta(o, F.w, dl);
          OpSpec sp2;
          sp2.tgt_rep = ridx.at({l, -1});
          sp2.src_rep = ridx.at({P->l1, d});
          for (int q = 0; q < 3; ++q) sp2.shift[q] = dl[q];
          specs.push_back(sp2);
        }
      F.l2l.M = F.R; F.l2l.Kd = Hp.R; F.l2l.nops = (int)specs.size();
      F.l2l.ops = ar.alloc<float2>((std::max<size_t>(1, specs.size()) * F.R * Hp.R) * P->cw);
      timed_form(kOpL2L, specs, dreps, F.R, Hp.R, F.l2l.ops, P->fp64);
      std::vector<int32_t> op;
      std::vector<int2> pr;
      for (size_t k = 0; k < Hp.in_keys.size(); ++k) {
        int b = Hp.in_keys[k] / Hp.nd, d = Hp.in_keys[k] % Hp.nd;
        for (int c = 0; c < Lp.h_nchild[b]; ++c) {
          int ch = Lp.h_child_first[b] + c;
          op.push_back(cell_id[d] * 8 + octant_of(&LV[l].h_coords[3 * ch]));
          pr.push_back(make_int2((int)k, ch));
          F.l2l.flops_rhs += 8.0 * F.r * rank_of(P->l1, d);
        }
      }
      F.l2l.fam = F_L2L;
      F.l2l.src_rows = (int64_t)Hp.in_keys.size();
      F.l2l.dst_rows = LV[l].n;
      finish_gemm(F.l2l, op, pr, ar, s);
      other_flops += F.l2l.flops_rhs;
    }
  }

  phase(3);
  // ---- per-point data: local coordinates, L2P rows, P2P lists, M2P rows
  std::vector<float4> loc(N), loc_lo(N);
  std::vector<int> leaf_level(N, -1);
  std::vector<int32_t> leaf_box(N, -1);
  std::vector<int64_t> gleaf_of_box;    // not used directly
  std::vector<int2> leaf_range;
  std::map<std::pair<int, int>, int> gleaf;   // (level, box) -> global leaf id
  std::vector<std::array<double, 3>> sorted_pts(N);
  for (int64_t k = 0; k < N; ++k)
    for (int d = 0; d < 3; ++d) sorted_pts[k][d] = hp[3 * (size_t)P->h_perm[k] + d];
  for (int l = P->l_lf0; l < nl; ++l)
    for (int64_t b = 0; b < LV[l].n; ++b) {
      if (!LV[l].h_leaf[b]) continue;
      gleaf[{l, (int)b}] = (int)leaf_range.size();
      leaf_range.push_back(make_int2(LV[l].h_first[b], LV[l].h_count[b]));
      double c[3] = {center(l, b, 0), center(l, b, 1), center(l, b, 2)};
      for (int64_t i = LV[l].h_first[b]; i < LV[l].h_first[b] + LV[l].h_count[b]; ++i) {
        double v[3] = {sorted_pts[i][0] - c[0], sorted_pts[i][1] - c[1], sorted_pts[i][2] - c[2]};
        loc[i] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
        loc_lo[i] = make_float4((float)(v[0] - (double)loc[i].x), (float)(v[1] - (double)loc[i].y),
                                (float)(v[2] - (double)loc[i].z), 0.f);
        leaf_level[i] = l;
        leaf_box[i] = (int32_t)b;
      }
    }
  P->n_leaves = (int64_t)leaf_range.size();
  P->pts_local = upload(loc, ar, s);
  P->pts_lo = upload(loc_lo, ar, s);
  // L2P rows per LF level (FP64 local coordinates -> rows)
  for (int l = P->l_lf0; l < nl; ++l) {
    LFLevel& F = P->lf[l];
    std::vector<double> lp;
    std::vector<int4> jobs;
    std::vector<int2> rmap;
    int64_t row = 0;
    for (int64_t b = 0; b < LV[l].n; ++b) {
      if (!LV[l].h_leaf[b]) continue;
      double c[3] = {center(l, b, 0), center(l, b, 1), center(l, b, 2)};
      jobs.push_back(make_int4(LV[l].h_first[b], LV[l].h_count[b], (int)row, (int)b));
      for (int64_t i = LV[l].h_first[b]; i < LV[l].h_first[b] + LV[l].h_count[b]; ++i) {
        for (int d = 0; d < 3; ++d) lp.push_back(sorted_pts[i][d] - c[d]);
        rmap.push_back(make_int2((int)i, (int)b));
        ++row;
      }
    }
    F.n_l2p = (int64_t)jobs.size();
    F.l2p_jobs = upload(jobs, ar, s);
    F.n_l2p_rows = row;
    F.l2p_map = upload(rmap, ar, s);
    F.l2p_rows = ar.alloc<float2>(std::max<int64_t>(1, row) * F.R * P->cw);
    F.p2m_rows = ar.alloc<float2>(std::max<int64_t>(1, row) * F.R * P->cw);
    if (row > 0) {
      ArenaMark mk(ar);
      double* dlp = ar.alloc<double>(lp.size());
      DFMM_CUDA(cudaMemcpyAsync(dlp, lp.data(), lp.size() * 8, cudaMemcpyHostToDevice, s));
      form_rows(true, dreps[ridx.at({l, -1})], dlp, row, F.l2p_rows, P->fp64, ar, s);
      form_p2m_rows(dreps[ridx.at({l, -1})], dlp, row, F.p2m_rows, P->fp64, ar, s);
    }
    other_flops += 8.0 * F.r * (double)row;
  }
  // M2P rows (W list), grouped by the source level
  for (int la = P->l_lf0; la < nl; ++la) {
    std::vector<double> lp;
    std::vector<int4> jobs;
    std::vector<int2> rmap;
    int64_t row = 0;
    for (size_t q = 0; q < nW; ++q) {
      int lb = P->Wl[4 * q], b = P->Wl[4 * q + 1], l2 = P->Wl[4 * q + 2], a = P->Wl[4 * q + 3];
      if (l2 != la) continue;
      double c[3] = {center(la, a, 0), center(la, a, 1), center(la, a, 2)};
      jobs.push_back(make_int4(LV[lb].h_first[b], LV[lb].h_count[b], (int)row, a));
      for (int64_t i = LV[lb].h_first[b]; i < LV[lb].h_first[b] + LV[lb].h_count[b]; ++i) {
        for (int d = 0; d < 3; ++d) lp.push_back(sorted_pts[i][d] - c[d]);
        rmap.push_back(make_int2((int)i, (int)b));
        ++row;
      }
    }
    if (jobs.empty()) continue;
    M2PGroup g;
    g.src_level = la;
    g.R = P->lf[la].R;
    g.njobs = (int64_t)jobs.size();
    g.nrows = row;
    g.jobs = upload(jobs, ar, s);
    g.rows = ar.alloc<float2>(row * g.R * P->cw);
    {
      ArenaMark mk(ar);
      double* dlp = ar.alloc<double>(lp.size());
      DFMM_CUDA(cudaMemcpyAsync(dlp, lp.data(), lp.size() * 8, cudaMemcpyHostToDevice, s));
      form_rows(false, dreps[ridx.at({la, -1})], dlp, row, g.rows, P->fp64, ar, s);
    }
    P->m2p.push_back(g);
  }
  phase(4);
  // P2P lists (U), CSR per target leaf: per source leaf (first point, count,
  // offset of its points within the leaf's list, self) and the exact centre
  // offset c_src - c_tgt (a multiple of the finest half-width, exact in FP32)
  {
    std::vector<std::vector<std::pair<int4, float4>>> per(leaf_range.size());
    int64_t inter = 0;
    for (size_t q = 0; q < nU; ++q) {
      int lb = P->U[4 * q], b = P->U[4 * q + 1], la = P->U[4 * q + 2], a = P->U[4 * q + 3];
      float sh[3];
      for (int d = 0; d < 3; ++d) sh[d] = (float)(center(la, a, d) - center(lb, b, d));
      const int self = (la == lb && a == b) ? 1 : 0;   // the leaf's own entry: may hold coincident points
      auto& lst = per[gleaf.at({lb, b})];
      lst.push_back({make_int4(LV[la].h_first[a], LV[la].h_count[a], 0, self), make_float4(sh[0], sh[1], sh[2], 0.f)});
      if (self) std::swap(lst.front(), lst.back());   // kept first
      inter += (int64_t)LV[lb].h_count[b] * LV[la].h_count[a];
    }
    std::vector<int64_t> off(leaf_range.size() + 1, 0);
    std::vector<int4> src;
    std::vector<float4> shifts;
    // the flat staging list of the FP32 form packs a point index (< 2^25) and
    // the entry within its leaf's list (< 128) into 32 bits; z = list offset
    bool flat_ok = N < ((int64_t)1 << 25) && inter < ((int64_t)1 << 62);
    std::vector<uint32_t> flat;
    int64_t zacc = 0;
    for (size_t g = 0; g < per.size(); ++g) {
      off[g + 1] = off[g] + (int64_t)per[g].size();
      if (per[g].size() > 127) flat_ok = false;
      for (size_t k = 0; k < per[g].size(); ++k) {
        auto& e = per[g][k];
        if (zacc >= ((int64_t)1 << 31)) flat_ok = false;
        e.first.z = (int)std::min<int64_t>(zacc, INT32_MAX);
        if (flat_ok)
          for (int q = 0; q < e.first.y; ++q) flat.push_back((uint32_t)(e.first.x + q) | ((uint32_t)k << 25));
        zacc += e.first.y;
        src.push_back(e.first);
        shifts.push_back(e.second);
      }
    }
    P->p2p_range = upload(leaf_range, ar, s);
    P->p2p_off = upload(off, ar, s);
    P->p2p_src = upload(src, ar, s);
    P->p2p_shift = upload(shifts, ar, s);
    if (P->opt.p2p_mode == 2 && !flat_ok) P->opt.p2p_mode = 1;   // beyond the packed list: double-float form
    if (P->opt.p2p_mode == 2) {
      P->p2p_flat = upload(flat, ar, s);
      P->n_flat = (int64_t)flat.size();
    }
    P->stats.p2p_interactions = inter;
    // FP32 form of the near field: its close pairs and their exact corrections
    // (the pairs closer than delta = 1e-6 / eps, at most 0.5; the FP32
    // coordinates' rounding perturbs a pair at distance d by about 1e-7 / d)
    if (P->opt.p2p_mode == 2 && P->n_leaves > 0) {
      P2PArgs pa{};
      pa.leaf_range = P->p2p_range;
      pa.nleaves = P->n_leaves;
      pa.u_off = P->p2p_off;
      pa.u_src = P->p2p_src;
      pa.u_shift = P->p2p_shift;
      pa.pts = P->pts_local;
      pa.pts_lo = P->pts_lo;
      const float delta = (float)std::min(0.5, 1e-6 / P->eps);
      ArenaMark mk(ar);
      int32_t* cnt = ar.alloc<int32_t>(N);
      unsigned* degen = ar.alloc<unsigned>(1);
      DFMM_CUDA(cudaMemsetAsync(degen, 0, 4, s));
      launch_p2p_close(pa, delta, cnt, degen, nullptr, nullptr, nullptr, s);
      std::vector<int32_t> hc(N);
      unsigned hd = 0;
      DFMM_CUDA(cudaMemcpyAsync(hc.data(), cnt, N * 4, cudaMemcpyDeviceToHost, s));
      DFMM_CUDA(cudaMemcpyAsync(&hd, degen, 4, cudaMemcpyDeviceToHost, s));
      DFMM_CUDA(cudaStreamSynchronize(s));
      P->close_delta = delta;
      if (hd) {
        P->opt.p2p_mode = 1;   // two distinct points share FP32 coordinates: double-float form
      } else {
        std::vector<int32_t> ho(N + 1, 0);
        for (int64_t i = 0; i < N; ++i) ho[i + 1] = ho[i] + hc[i];
        P->n_close = ho[N];
        P->close_keep.reset(new DevArena());
        DevArena& ca = *P->close_keep;
        P->close_off = upload(ho, ca, s);
        P->close_j = ca.alloc<int32_t>(std::max<int64_t>(1, P->n_close));
        P->close_w = ca.alloc<float2>(std::max<int64_t>(1, P->n_close));
        launch_p2p_close(pa, delta, nullptr, degen, P->close_off, P->close_j, P->close_w, s);
        DFMM_CUDA(cudaStreamSynchronize(s));
      }
    }
  }
  P->stats.m2l_flops = m2l_flops;
  P->stats.other_translation_flops = other_flops;
  P->stats.plan_bytes = (int64_t)ar.bytes() + (P->close_keep ? (int64_t)P->close_keep->bytes() : 0);
  P->stats.p2p_close_pairs = P->n_close;
  phase(5);
  P->stats.plan_seconds = now() - t0;
}

// ------------------------------------------------------------------- apply ---

// Most rows of a translation stage's source buffer, per RHS.
int64_t max_source_rows(const dfmm_plan_s* P) {
  int64_t m = 1;
  for (int l = 0; l < P->nl; ++l) {
    if (l >= P->l_lf0) {
      m = std::max({m, P->lf[l].nbox, P->lf[l].n_p2l});
    } else if (P->l_top >= 0 && l >= P->l_top) {
      m = std::max(m, (int64_t)std::max(P->hf[l].out_keys.size(), P->hf[l].in_keys.size()));
    }
  }
  return m;
}

// Largest source buffer of a translation stage, in complex elements per RHS
// (the tensor form splits it into FP16 hi / lo arrays).
int64_t max_source_elems(const dfmm_plan_s* P) {
  int64_t m = 0;
  for (int l = 0; l < P->nl; ++l) {
    if (l >= P->l_lf0) {
      const LFLevel& F = P->lf[l];
      m = std::max(m, F.nbox * (int64_t)F.R);
      m = std::max(m, F.n_p2l * 2 * (int64_t)F.R);
    } else if (P->l_top >= 0 && l >= P->l_top) {
      const HFLevel& H = P->hf[l];
      m = std::max(m, (int64_t)std::max(H.out_keys.size(), H.in_keys.size()) * H.R);
    }
  }
  return m;
}

Workspace* get_workspace(dfmm_plan_s* P, cudaStream_t s, int nrhs) {
  std::lock_guard<std::mutex> g(P->ws_mu);
  auto& slot = P->ws[s];
  if (slot && slot->nrhs >= nrhs) return slot.get();
  slot.reset(new Workspace());
  Workspace* W = slot.get();
  W->nrhs = nrhs;
  DevArena& ar = W->ar;
  const int64_t N = P->N;
  const int64_t cw = P->cw;   // float2 units per complex element
  W->fs = ar.alloc<float2>(N * nrhs * cw);
  W->us = ar.alloc<float2>(N * nrhs * cw);
  W->zero.push_back({W->us, (size_t)N * nrhs * cw * sizeof(float2)});
  W->S.assign(P->nl, nullptr);
  W->T.assign(P->nl, nullptr);
  int64_t p2l_rows = 1;
  for (int l = 0; l < P->nl; ++l) {
    int64_t rows = 0;
    int R = 0;
    if (l >= P->l_lf0) { rows = P->lf[l].nbox; R = P->lf[l].R; }
    else if (P->l_top >= 0 && l >= P->l_top) {
      R = P->hf[l].R;
      int64_t so = (int64_t)P->hf[l].out_keys.size(), si = (int64_t)P->hf[l].in_keys.size();
      if (so) { W->S[l] = ar.alloc<float2>(so * nrhs * R * cw); W->zero_late.push_back({W->S[l], (size_t)so * nrhs * R * 8 * cw}); }
      if (si) { W->T[l] = ar.alloc<float2>(si * nrhs * R * cw); W->zero_late.push_back({W->T[l], (size_t)si * nrhs * R * 8 * cw}); }
      continue;
    } else continue;
    W->S[l] = ar.alloc<float2>(rows * nrhs * R * cw);
    W->T[l] = ar.alloc<float2>(rows * nrhs * R * cw);
    W->zero.push_back({W->S[l], (size_t)rows * nrhs * R * 8 * cw});
    W->zero.push_back({W->T[l], (size_t)rows * nrhs * R * 8 * cw});
    p2l_rows = std::max(p2l_rows, P->lf[l].n_p2l * 2 * R);
  }
  W->p2l = ar.alloc<float2>(p2l_rows * nrhs * cw);
  if (P->opt.m2l_mode == 2) {
    // split arrays: 2 values per complex element, 2 bytes each (4 for the TF32 split)
    int64_t e = max_source_elems(P) * nrhs * 2 * (P->opt.tc_precision == 2 ? 2 : 1);
    W->ahi = ar.alloc<__half>(e);
    W->alo = ar.alloc<__half>(e);
    W->ascale = ar.alloc<float>(max_source_rows(P) * nrhs);
  }
  W->status = ar.alloc<unsigned>(1);
  W->zero.push_back({W->status, 4});   // reset by every apply; read by dfmm_sync_status
  DFMM_CUDA(cudaMemsetAsync(W->status, 0, 4, s));
  return W;
}

// Work tiles of a stage: runs of up to cols / nrhs pairs of one operator.
// Pairs of an operator are sorted by target, so an operator's tiles sweep the
// whole target array.  When the stage's operators are small enough to stay in
// L2 (<= 64 MB), tiles are ordered by block of target rows first and operator
// second, so that the tiles in flight together touch one block of targets
// (and the sources near them) and keep those rows in L2; blocks hold about
// 8 MB of target rows.  Otherwise tiles stay in operator order, so that an
// operator is read from DRAM once for all its tiles.
// whether a translation stage runs on the tensor cores (m2l_mode 2, ranks padded
// for the MMA, its family selected by options.tc_stages)
bool on_tensor_cores(const dfmm_plan_s* P, const GemmPlan& g) {
  // the BF16 and TF32 splits exist in the split-complex form only: other stages stay on the CUDA cores
  return P->opt.m2l_mode == 2 && gemm_tc_supported(g.M, g.Kd) && (P->opt.tc_stages & kTcFamBit[g.fam]) != 0 &&
         (P->opt.tc_precision == 0 || gemm_cx_supported(g.M, g.Kd));
}

// whether a tensor-core stage takes the split-complex form (m2l_cx.cu): target
// rank at most 128 and ranks that are multiples of 16; else the real-block form
bool split_complex(const dfmm_plan_s* P, const GemmPlan& g) {
  return on_tensor_cores(P, g) && P->opt.tc_layout != 1 && gemm_cx_supported(g.M, g.Kd);
}

// tile_order: 0 = by the 64 MB rule above, 1 = always by target block, 2 = always by operator.
// block_bytes: target rows per block in the blocked order (8 MB unless the
// batched form's autotuner tries another size).
std::vector<int4> make_tiles(const GemmPlan& g, int nrhs, int cols, int tile_order, int64_t block_bytes = (int64_t)8 << 20) {
  const int per = std::max(1, cols / nrhs);
  std::vector<int4> t;
  std::vector<int64_t> key;
  const int64_t row_bytes = (int64_t)g.M * 8 * nrhs;
  const bool blocked = tile_order == 1 || (tile_order == 0 && (double)g.nops * g.M * g.Kd * 8.0 <= 64.0 * (1 << 20));
  const int64_t block_rows = blocked ? std::max<int64_t>(1, block_bytes / std::max<int64_t>(1, row_bytes))
                                     : ((int64_t)1 << 40);
  for (const int4& grp : g.groups)
    for (int p = 0; p < grp.z; p += per) {
      t.push_back(make_int4(grp.x, grp.y + p, std::min(per, grp.z - p), 0));
      const int64_t blk = g.h_dst.empty() ? 0 : g.h_dst[grp.y + p] / block_rows;
      key.push_back(blk * (int64_t)(g.nops + 1) + grp.x);
    }
  std::vector<int64_t> order(t.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int64_t)i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  std::vector<int4> out(t.size());
  for (size_t i = 0; i < order.size(); ++i) out[i] = t[order[i]];
  return out;
}

std::pair<int4*, int64_t> tiles_for(const dfmm_plan_s* P, Workspace* W, const GemmPlan& g, int nrhs, int cols,
                                    cudaStream_t s) {
  auto key = std::make_pair((const void*)&g, nrhs * 1024 + cols);
  auto it = W->tiles.find(key);
  if (it != W->tiles.end()) return it->second;
  if (W->external) throw Error(DFMM_ERR_INVALID, "work tiles missing from the carved workspace");
  std::vector<int4> t = make_tiles(g, nrhs, cols, P->opt.tile_order);
  int4* d = W->ar.alloc<int4>(std::max<size_t>(1, t.size()));
  if (!t.empty()) DFMM_CUDA(cudaMemcpyAsync(d, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  W->tiles[key] = {d, (int64_t)t.size()};
  return W->tiles[key];
}

// A translation stage that the batched form runs in a merged launch.
struct WaveGemm {
  dfmm_plan_s* P;
  Workspace* W;
  const GemmPlan* g;
  const float2* src;
  int src_ld;
  int64_t src_rows;
  float2* dst;
  int dst_ld;
  int nrhs;
  bool split;   // the stage's source buffer must be split first
  int store;
};

// Wave filter of the batched form: run_apply acts only on the steps of one wave
// (the same step, by kind and box width, in every plan), and hands its
// split-complex translation stages to `collect` instead of launching them.
struct WaveCtl {
  int64_t wave;
  std::vector<WaveGemm>* collect;
  std::vector<int64_t>* keys;   // if set: the wave keys of the plan's steps are listed, nothing runs
};

struct Runner {
  dfmm_plan_s* P;
  Workspace* W;
  cudaStream_t s;
  int nrhs;
  int64_t* count;   // dry run: count launches only
  WaveCtl* ctl = nullptr;
  int64_t cur = 0;  // wave key of the next step

  Runner& at(int64_t key) {
    cur = key;
    return *this;
  }
  // whether the current step is skipped by the wave filter (after listing its key)
  bool skip() {
    if (!ctl) return false;
    if (ctl->keys) {
      ctl->keys->push_back(cur);
      return true;
    }
    return cur != ctl->wave;
  }

  template <class Fn>
  void launch(int fam, double flops, double bytes, Fn&& fn) {
    if (count) { ++*count; return; }
    if (skip()) return;
    ProfScope ps(W, s, fam, flops, bytes);
    fn();
  }

  int split_key = -1;   // source buffer that the split arrays hold (tensor form), -1: none

  // src_key names the source buffer (kSrcS / kSrcT + level, -1 for one used once); a
  // stage whose source is the buffer split for the previous stage reuses that split.
  // first: no earlier stage of the apply writes dst (it holds zeros), so a stage whose
  // target rows are all distinct may store its results instead of adding them.
  void gemm(const GemmPlan& g, const float2* src, int src_ld, int64_t src_rows, float2* dst, int dst_ld,
            int src_key, bool first = false) {
    if (g.npairs == 0) return;
    const bool tc = on_tensor_cores(P, g);
    const bool cx = tc && split_complex(P, g);
    // the split arrays hold one source buffer in one layout (interleaved or split-complex)
    const int key = src_key < 0 ? -1 : 2 * src_key + (cx ? 1 : 0);
    const bool split = tc && (key < 0 || key != split_key);
    if (tc) split_key = key;
    if (count) { count[0] += split ? 2 : 1; return; }
    if (skip()) return;
    if (ctl && ctl->collect && cx) {   // the batched form merges this stage with the other plans' same stage
      ctl->collect->push_back(WaveGemm{P, W, &g, src, src_ld, src_rows, dst, dst_ld, nrhs, split,
                                       (first && g.dst_unique) ? 1 : 0});
      return;
    }
    auto t = tiles_for(P, W, g, nrhs, tc ? gemm_tc_columns() : 64, s);
    GemmArgs a;
    a.ops = g.ops;
    a.M = g.M;
    a.Kd = g.Kd;
    a.tiles = t.first;
    a.ntiles = t.second;
    a.pairs = g.pairs;
    a.src = src;
    a.dst = dst;
    a.src_ld = src_ld;
    a.dst_ld = dst_ld;
    a.nrhs = nrhs;
    a.store = (first && g.dst_unique) ? 1 : 0;
    a.wait_test = P->opt.wait_test ? 1 : 0;
    a.stages = nullptr;
    if (tc) {
      if (split) {
        ProfScope ps(W, s, F_SPLIT, 0.0, (double)src_rows * nrhs * src_ld * 16);
        if (cx) launch_split_cx(src, src_rows * nrhs, src_ld, W->ahi, W->alo, W->ascale, P->opt.tc_precision, s);
        else launch_split(src, src_rows * nrhs, src_ld, W->ahi, W->alo, W->ascale, s);
      }
      ProfScope ps(W, s, g.fam, g.flops_rhs * nrhs, g.bytes_fixed + g.bytes_rhs * nrhs);
      TcArgs targs{g.img, g.op_scale, W->ahi, W->alo, W->ascale};
      if (cx) launch_gemm_stage_cx(a, targs, W->status, P->opt.tc_accumulate == 1, P->opt.tc_precision, s);
      else launch_gemm_stage_tc(a, targs, W->status, s);
    } else {
      ProfScope ps(W, s, g.fam, g.flops_rhs * nrhs, g.bytes_fixed + g.bytes_rhs * nrhs);
      if (P->fp64) launch_gemm_stage64(a, s);
      else launch_gemm_stage(a, s);
    }
  }
};

constexpr int kSrcS = 0, kSrcT = 64;   // source keys: outgoing / incoming states of a level

// Wave keys of the steps of an apply: the same step (kind, box width) of
// different plans gets the same key, and the keys of one plan's steps
// increase in the order the apply runs them, so the batched form can run the
// plans wave by wave.  lw = log2 of the box width.
constexpr int64_t kWaveStart = 0;
inline int64_t wave_p2m(int64_t lw) { return 1000 + (lw + 64) * 4; }
inline int64_t wave_lf_m2m(int64_t lw) { return 1000 + (lw + 64) * 4 + 1; }
constexpr int64_t kWaveTopV = 2000;
inline int64_t wave_hf_m2m(int64_t lw) { return 3000 + (lw + 64) * 4; }
inline int64_t wave_hf_m2l(int64_t lw) { return 3000 + (lw + 64) * 4 + 1; }
inline int64_t wave_hf_l2l(int64_t lw) { return 4000 + (64 - lw) * 4; }
inline int64_t wave_lf_down(int64_t lw, int k) { return 5000 + (64 - lw) * 8 + k; }
inline int64_t wave_l2p(int64_t lw) { return 6000 + (64 - lw); }
constexpr int64_t kWaveM2P = 6500, kWaveP2P = 7000, kWaveEnd = 8000;

void run_apply(dfmm_plan_s* P, const float2* f, float2* u, int nrhs, cudaStream_t s, int64_t* count = nullptr,
               Workspace* ext = nullptr, WaveCtl* ctl = nullptr) {
  Workspace* W = count ? nullptr : (ext ? ext : get_workspace(P, s, nrhs));
  Runner R{P, W, s, nrhs, count};
  R.ctl = ctl;
  const int64_t lW = (int64_t)std::llround(std::log2(P->W));
  auto lw = [&](int l) -> int64_t { return lW - l; };   // log2 of the width of level l
  const int64_t N = P->N;
  const int nl = P->nl;
  auto S = [&](int l) { return count ? (float2*)nullptr : W->S[l]; };
  auto T = [&](int l) { return count ? (float2*)nullptr : W->T[l]; };
  const bool late = !count && !ctl && !W->zero_late.empty();
  if (late) {   // HF states: reset on a side stream while P2M and the V list run
    if (!W->side) {
      DFMM_CUDA(cudaStreamCreateWithFlags(&W->side, cudaStreamNonBlocking));
      DFMM_CUDA(cudaEventCreateWithFlags(&W->fork, cudaEventDisableTiming));
      DFMM_CUDA(cudaEventCreateWithFlags(&W->join, cudaEventDisableTiming));
    }
    DFMM_CUDA(cudaEventRecord(W->fork, s));
    DFMM_CUDA(cudaStreamWaitEvent(W->side, W->fork, 0));
    for (auto& z : W->zero_late) DFMM_CUDA(cudaMemsetAsync(z.first, 0, z.second, W->side));
    DFMM_CUDA(cudaEventRecord(W->join, W->side));
  }
  if (!count && !R.at(kWaveStart).skip()) {
    ProfScope ps(W, s, F_ZERO, 0.0, 0.0);
    for (auto& z : W->zero) DFMM_CUDA(cudaMemsetAsync(z.first, 0, z.second, s));
    if (ctl)   // the batched form resets every state in line
      for (auto& z : W->zero_late) DFMM_CUDA(cudaMemsetAsync(z.first, 0, z.second, s));
  }
  R.at(kWaveStart).launch(F_PERMUTE, 0.0, 20.0 * N * nrhs, [&] {
    if (P->fp64) launch_permute_in64(f, P->perm, N, nrhs, W->fs, s);
    else launch_permute_in(f, P->perm, N, nrhs, W->fs, s);
  });
  // 1. LF upward: P2M at leaves, LF-M2M from the level below
  for (int l = nl - 1; l >= P->l_lf0; --l) {
    LFLevel& F = P->lf[l];
    if (F.n_l2p) {   // P2M: every leaf of this level, through its points' rows
      R.at(wave_p2m(lw(l))).launch(F_P2M_EVAL, 8.0 * F.r * F.npts * nrhs, F.npts * (8.0 * F.R + 8.0 * nrhs) + F.n_l2p * 8.0 * F.R * nrhs,
               [&] {
                 P2MRowsArgs a;
                 a.jobs = F.l2p_jobs;
                 a.njobs = F.n_l2p;
                 a.rows = F.p2m_rows;
                 a.fs = W->fs;
                 a.state = W->S[l];
                 a.R = F.R;
                 a.nrhs = nrhs;
                 if (P->fp64) launch_p2m_rows64(a, s);
                 else launch_p2m_rows(a, s);
               });
    }
    if (l + 1 < nl) R.at(wave_lf_m2m(lw(l))).gemm(F.m2m, S(l + 1), P->lf[l + 1].R, P->lf[l + 1].nbox, S(l), F.R, kSrcS + l + 1);
  }
  // M2L of each level as soon as its outgoing states are complete, so that the
  // next M2M, which reads the same states, reuses their split.  The V list of the
  // top LF level: its L2L (from HF, summed over directions) adds anyway.
  if (P->l_lf0 < nl)
    R.at(kWaveTopV).gemm(P->lf[P->l_lf0].v, S(P->l_lf0), P->lf[P->l_lf0].R, P->lf[P->l_lf0].nbox, T(P->l_lf0),
           P->lf[P->l_lf0].R, kSrcS + P->l_lf0);
  if (late) DFMM_CUDA(cudaStreamWaitEvent(s, W->join, 0));   // the HF states are reset
  // 2. HF upward: M2M, then that level's M2L
  if (P->l_top >= 0) {
    for (int l = P->l1; l >= P->l_top; --l) {
      HFLevel& H = P->hf[l];
      int sld = (l == P->l1) ? P->lf[l + 1].R : P->hf[l + 1].R;
      int64_t srows = (l == P->l1) ? P->lf[l + 1].nbox : (int64_t)P->hf[l + 1].out_keys.size();
      R.at(wave_hf_m2m(lw(l))).gemm(H.m2m, S(l + 1), sld, srows, S(l), H.R, kSrcS + l + 1);
      R.at(wave_hf_m2l(lw(l))).gemm(H.m2l, S(l), H.R, (int64_t)H.out_keys.size(), T(l), H.R, kSrcS + l);
    }
    // 3. HF downward: L2L from the parent level
    for (int l = P->l_top + 1; l <= P->l1; ++l) {
      HFLevel& H = P->hf[l];
      R.at(wave_hf_l2l(lw(l))).gemm(H.l2l, T(l - 1), P->hf[l - 1].R, (int64_t)P->hf[l - 1].in_keys.size(), T(l), H.R, kSrcT + l - 1);
    }
  }
  // 4. LF downward
  for (int l = P->l_lf0; l < nl; ++l) {
    LFLevel& F = P->lf[l];
    if (l == P->l_lf0) {
      if (P->l_top >= 0)
        R.at(wave_lf_down(lw(l), 0)).gemm(F.l2l, T(P->l1), P->hf[P->l1].R, (int64_t)P->hf[P->l1].in_keys.size(), T(l), F.R, kSrcT + P->l1);
    } else {
      R.at(wave_lf_down(lw(l), 0)).gemm(F.l2l, T(l - 1), P->lf[l - 1].R, P->lf[l - 1].nbox, T(l), F.R, kSrcT + l - 1,
                                        true);
      R.at(wave_lf_down(lw(l), 1)).gemm(F.v, S(l), F.R, F.nbox, T(l), F.R, kSrcS + l);
    }
    if (F.n_p2l) {
      double ev = (double)F.npts_x * 2 * F.r;
      R.at(wave_lf_down(lw(l), 2)).launch(F_P2L_EVAL, ev * (16 + 8.0 * nrhs), F.npts_x * (16.0 + 8.0 * nrhs) + F.n_p2l * 2.0 * F.R * 8 * nrhs, [&] {
        P2CArgs a{};
        a.jobs = F.p2l_jobs;
        a.njobs = F.n_p2l;
        a.shifts = F.p2l_shifts;
        a.chk = F.chk_b2;
        a.nchk = 2 * F.r;
        a.ld = 2 * F.R;
        a.pts = P->pts_local;
        a.fs = W->fs;
        a.out = W->p2l;
        a.nrhs = nrhs;
        a.chk64 = F.chk64;
        a.pts_lo = P->pts_lo;
        if (P->fp64) launch_p2c64(a, s);
        else launch_p2c(a, s);
      });
      R.at(wave_lf_down(lw(l), 3)).gemm(F.p2l, count ? nullptr : W->p2l, 2 * F.R, F.n_p2l, T(l), F.R, -1);
    }
  }
  // 5. L2P at every leaf, M2P over the W list
  for (int l = P->l_lf0; l < nl; ++l) {
    LFLevel& F = P->lf[l];
    if (!F.n_l2p) continue;
    R.at(wave_l2p(lw(l))).launch(F_L2P, 8.0 * F.r * F.npts * nrhs, F.npts * (8.0 * F.R + 16.0 * nrhs) + F.n_l2p * 8.0 * F.R * nrhs, [&] {
      L2PArgs a;
      a.map = F.l2p_map;
      a.nrows = F.n_l2p_rows;
      a.rows = F.l2p_rows;
      a.state = W->T[l];
      a.R = F.R;
      a.nrhs = nrhs;
      a.us = W->us;
      if (P->fp64) launch_l2p64(a, s);
      else launch_l2p(a, s);
    });
  }
  for (size_t k = 0; k < P->m2p.size(); ++k) {
    auto& g = P->m2p[k];
    R.at(kWaveM2P + (int64_t)k).launch(F_M2P, 8.0 * P->lf[g.src_level].r * g.nrows * nrhs, g.nrows * (8.0 * g.R + 16.0 * nrhs), [&] {
      RowsArgs a;
      a.jobs = g.jobs;
      a.njobs = g.njobs;
      a.rows = g.rows;
      a.state = W->S[g.src_level];
      a.R = g.R;
      a.nrhs = nrhs;
      a.us = W->us;
      a.atomic = 1;
      if (P->fp64) launch_rows64(a, s);
      else launch_rows(a, s);
    });
  }
  // 6. near field
  R.at(kWaveP2P).launch(F_P2P, (double)P->stats.p2p_interactions * (16.0 + 8.0 * nrhs), (double)N * (32.0 + 24.0 * nrhs), [&] {
    P2PArgs a;
    a.leaf_range = P->p2p_range;
    a.nleaves = P->n_leaves;
    a.u_off = P->p2p_off;
    a.u_src = P->p2p_src;
    a.u_shift = P->p2p_shift;
    a.flat = P->p2p_flat;
    a.pts = P->pts_local;
    a.pts_lo = P->pts_lo;
    a.fs = W->fs;
    a.us = W->us;
    a.nrhs = nrhs;
    a.close_off = P->close_off;
    a.close_j = P->close_j;
    a.close_w = P->close_w;
    if (P->fp64) launch_p2p64(a, s);
    else if (P->opt.p2p_mode == 2) launch_p2p_fast(a, N, s);
    else launch_p2p(a, s);
  });
  R.at(kWaveEnd).launch(F_PERMUTE, 0.0, 20.0 * N * nrhs, [&] {
    if (P->fp64) launch_permute_out64(W->us, P->perm, N, nrhs, u, s);
    else launch_permute_out(W->us, P->perm, N, nrhs, u, s);
  });
}

// Every translation stage of the plan, for laying out work tiles.
std::vector<const GemmPlan*> all_gemms(dfmm_plan_s* P) {
  std::vector<const GemmPlan*> v;
  for (auto& F : P->lf) { v.push_back(&F.m2m); v.push_back(&F.l2l); v.push_back(&F.v); v.push_back(&F.p2l); }
  for (auto& H : P->hf) { v.push_back(&H.m2m); v.push_back(&H.m2l); v.push_back(&H.l2l); }
  return v;
}

// Lays out the whole workspace of an apply with nrhs right-hand sides inside
// [base, base + bytes): the device status word (at offset 0), state buffers,
// staging buffers and the work tiles of every stage (copied in on `s`).  No device memory is allocated.  With
// base == nullptr nothing is laid out or copied: the return value is the
// number of bytes the layout needs.
size_t carve_workspace(dfmm_plan_s* P, int nrhs, char* base, size_t bytes, cudaStream_t s, Workspace& W) {
  size_t off = 0;
  auto take = [&](size_t n) -> char* {
    off = (off + 255) & ~(size_t)255;
    char* p = base + off;
    off += std::max<size_t>(n, 1);
    return p;
  };
  const int64_t N = P->N;
  const size_t cb = 8 * (size_t)P->cw;   // bytes per complex element
  W.external = true;
  W.nrhs = nrhs;
  // the device status word first, at offset 0 of the region (reset by every apply)
  W.status = (unsigned*)take(4);
  W.zero.push_back({W.status, 4});
  W.fs = (float2*)take((size_t)N * nrhs * cb);
  W.us = (float2*)take((size_t)N * nrhs * cb);
  W.zero.push_back({W.us, (size_t)N * nrhs * cb});
  W.S.assign(P->nl, nullptr);
  W.T.assign(P->nl, nullptr);
  size_t p2l_rows = 1;
  for (int l = 0; l < P->nl; ++l) {
    if (l >= P->l_lf0) {
      size_t b = (size_t)P->lf[l].nbox * nrhs * P->lf[l].R * cb;
      W.S[l] = (float2*)take(b);
      W.T[l] = (float2*)take(b);
      W.zero.push_back({W.S[l], b});
      W.zero.push_back({W.T[l], b});
      p2l_rows = std::max(p2l_rows, (size_t)P->lf[l].n_p2l * 2 * P->lf[l].R);
    } else if (P->l_top >= 0 && l >= P->l_top) {
      size_t so = P->hf[l].out_keys.size(), si = P->hf[l].in_keys.size();
      size_t R = P->hf[l].R;
      if (so) { W.S[l] = (float2*)take(so * nrhs * R * cb); W.zero.push_back({W.S[l], so * nrhs * R * cb}); }
      if (si) { W.T[l] = (float2*)take(si * nrhs * R * cb); W.zero.push_back({W.T[l], si * nrhs * R * cb}); }
    }
  }
  W.p2l = (float2*)take(p2l_rows * nrhs * cb);
  if (P->opt.m2l_mode == 2) {
    size_t e = (size_t)max_source_elems(P) * nrhs * 2 * (P->opt.tc_precision == 2 ? 2 : 1);
    W.ahi = (__half*)take(e * 2);
    W.alo = (__half*)take(e * 2);
    W.ascale = (float*)take((size_t)max_source_rows(P) * nrhs * 4);
  }
  std::vector<std::pair<const GemmPlan*, std::vector<int4>>> tl;
  std::vector<int> tl_cols;
  for (const GemmPlan* g : all_gemms(P)) {
    if (g->npairs == 0) continue;
    const int cols = on_tensor_cores(P, *g) ? gemm_tc_columns() : 64;
    tl_cols.push_back(cols);
    tl.push_back({g, make_tiles(*g, nrhs, cols, P->opt.tile_order)});
  }
  std::vector<int4*> dst(tl.size());
  for (size_t k = 0; k < tl.size(); ++k) dst[k] = (int4*)take(tl[k].second.size() * sizeof(int4));
  if (!base) return off;
  if (off > bytes)
    throw Error(DFMM_ERR_UNSUPPORTED, "apply needs " + std::to_string(off) + " bytes of scratch, more than the " +
                                          std::to_string(bytes) + " bytes of the static scratch array");
  for (size_t k = 0; k < tl.size(); ++k) {
    DFMM_CUDA(cudaMemcpyAsync(dst[k], tl[k].second.data(), tl[k].second.size() * sizeof(int4),
                              cudaMemcpyHostToDevice, s));
    W.tiles[std::make_pair((const void*)tl[k].first, nrhs * 1024 + tl_cols[k])] = {dst[k], (int64_t)tl[k].second.size()};
  }
  return off;
}

// Device bytes of one apply's workspace with nrhs right-hand sides.
int64_t workspace_bytes(dfmm_plan_s* P, int nrhs) {
  Workspace W;
  return (int64_t)carve_workspace(P, nrhs, nullptr, 0, nullptr, W);
}

// Operator images of every translation stage for the tensor-core form.
void build_images(dfmm_plan_s* P, cudaStream_t s) {
  for (const GemmPlan* gc : all_gemms(P)) {
    GemmPlan* g = const_cast<GemmPlan*>(gc);
    if (g->npairs == 0 || g->nops == 0 || !on_tensor_cores(P, *g)) continue;
    g->op_scale = P->ar.alloc<float>(g->nops);
    if (split_complex(P, *g)) {
      g->img = (__half*)P->ar.alloc<unsigned char>(cx_image_bytes(g->M, g->Kd, g->nops, P->opt.tc_precision));
      build_cx_image(g->ops, g->M, g->Kd, g->nops, g->img, g->op_scale, P->opt.tc_precision, s);
    } else {
      g->img = P->ar.alloc<__half>(tc_image_elems(g->M, g->Kd, g->nops));
      build_tc_image(g->ops, g->M, g->Kd, g->nops, g->img, g->op_scale, s);
    }
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
  P->stats.plan_bytes = (int64_t)P->ar.bytes() + (P->close_keep ? (int64_t)P->close_keep->bytes() : 0);
}

// Bounds checks of every index table of the plan and of the work tiles of
// every workspace laid out so far (dfmm_validate); names[k] names check k.  The
// caller holds P->ws_mu until the checks have run (a workspace replaced
// meanwhile would free its tile tables).
void plan_checks(dfmm_plan_s* P, std::vector<RangeCheck>& c, std::vector<std::string>& names) {
  const int64_t N = P->N;
  auto fields = [&](const std::string& nm, const void* p, int64_t n, int stride, int a, int64_t hi_a, int b = -1,
                    int64_t hi_ab = 0) {
    RangeCheck r;
    r.p = p;
    r.n = n;
    r.mode = kCheckFields;
    r.stride = stride;
    r.a = a;
    r.b = b;
    r.hi_a = hi_a;
    r.hi_ab = hi_ab;
    c.push_back(r);
    names.push_back(nm);
  };
  auto csr = [&](const std::string& nm, const void* p, int64_t n, bool i64, int64_t total) {
    RangeCheck r;
    r.p = p;
    r.n = n;
    r.mode = i64 ? kCheckCsr64 : kCheckCsr32;
    r.hi_a = total;
    c.push_back(r);
    names.push_back(nm);
  };
  fields("permutation", P->perm, N, 1, 0, N);
  int si = 0;
  for (const GemmPlan* gp : all_gemms(P)) {
    const std::string tag = std::string(kFamName[gp->fam]) + " stage " + std::to_string(si++);
    if (gp->npairs == 0) continue;
    fields(tag + " pair sources", gp->pairs, gp->npairs, 2, 0, gp->src_rows);
    fields(tag + " pair targets", gp->pairs, gp->npairs, 2, 1, gp->dst_rows);
    for (auto& ws : P->ws)
      for (auto& t : ws.second->tiles)
        if (t.first.first == (const void*)gp) {
          fields(tag + " tile operators", t.second.first, t.second.second, 4, 0, gp->nops);
          fields(tag + " tile pair ranges", t.second.first, t.second.second, 4, 1, gp->npairs, 2, gp->npairs);
        }
  }
  for (int l = P->l_lf0; l < P->nl; ++l) {
    const LFLevel& F = P->lf[l];
    const std::string tag = "level " + std::to_string(l);
    fields(tag + " L2P rows: points", F.l2p_map, F.n_l2p_rows, 2, 0, N);
    fields(tag + " L2P rows: boxes", F.l2p_map, F.n_l2p_rows, 2, 1, F.nbox);
    fields(tag + " leaf jobs: points", F.l2p_jobs, F.n_l2p, 4, 0, N, 1, N);
    fields(tag + " leaf jobs: rows", F.l2p_jobs, F.n_l2p, 4, 2, F.n_l2p_rows + 1, 1, F.n_l2p_rows);
    fields(tag + " leaf jobs: boxes", F.l2p_jobs, F.n_l2p, 4, 3, F.nbox);
    fields(tag + " X-list jobs: points", F.p2l_jobs, F.n_p2l, 4, 0, N, 1, N);
    fields(tag + " X-list jobs: rows", F.p2l_jobs, F.n_p2l, 4, 2, F.n_p2l);
    fields(tag + " X-list jobs: shifts", F.p2l_jobs, F.n_p2l, 4, 3, F.n_p2l);
  }
  for (size_t k = 0; k < P->m2p.size(); ++k) {
    const M2PGroup& m = P->m2p[k];
    const std::string tag = "W-list group " + std::to_string(k);
    fields(tag + ": points", m.jobs, m.njobs, 4, 0, N, 1, N);
    fields(tag + ": rows", m.jobs, m.njobs, 4, 2, m.nrows + 1, 1, m.nrows);
    fields(tag + ": states", m.jobs, m.njobs, 4, 3, P->lf[m.src_level].nbox);
  }
  int64_t n_src = 0;
  DFMM_CUDA(cudaMemcpy(&n_src, P->p2p_off + P->n_leaves, sizeof(int64_t), cudaMemcpyDeviceToHost));
  fields("near-field leaves", P->p2p_range, P->n_leaves, 2, 0, N, 1, N);
  csr("near-field list offsets", P->p2p_off, P->n_leaves, true, n_src);
  fields("near-field sources", P->p2p_src, n_src, 4, 0, N, 1, N);
  if (P->p2p_flat) {
    RangeCheck r;
    r.p = P->p2p_flat;
    r.n = P->n_flat;
    r.mode = kCheckPacked;
    r.hi_a = N;
    c.push_back(r);
    names.push_back("near-field staging list");
  }
  if (P->close_off) {
    csr("close-pair offsets", P->close_off, N, false, P->n_close);
    fields("close-pair sources", P->close_j, P->n_close, 1, 0, N);
  }
}

// The checks of plan_checks on `s`; with plant, also a scratch copy of the first
// non-empty pair table with the source row of its first pair set to its bound.
// Throws DFMM_ERR_DEVICE naming the first table with an entry out of range.
void validate_plan(dfmm_plan_s* P, cudaStream_t s, bool plant) {
  std::lock_guard<std::mutex> g(P->ws_mu);
  std::vector<RangeCheck> c;
  std::vector<std::string> names;
  plan_checks(P, c, names);
  DevArena ar;
  if (plant) {
    for (const GemmPlan* gp : all_gemms(P)) {
      if (gp->npairs == 0) continue;
      int2* copy = ar.alloc<int2>(gp->npairs);
      DFMM_CUDA(cudaMemcpyAsync(copy, gp->pairs, gp->npairs * sizeof(int2), cudaMemcpyDeviceToDevice, s));
      const int bad = (int)gp->src_rows;
      DFMM_CUDA(cudaMemcpyAsync(copy, &bad, sizeof(int), cudaMemcpyHostToDevice, s));
      RangeCheck r;
      r.p = copy;
      r.n = gp->npairs;
      r.stride = 2;
      r.a = 0;
      r.hi_a = gp->src_rows;
      c.push_back(r);
      names.push_back("planted copy of a pair table");
      break;
    }
  }
  const std::vector<int64_t> bad = run_range_checks(c, s);
  for (size_t k = 0; k < c.size(); ++k)
    if (bad[k] >= 0)
      throw Error(DFMM_ERR_DEVICE, names[k] + ": entry " + std::to_string(bad[k]) + " out of range");
}

template <class F>
int guarded(F&& fn) {
  try {
    return fn();
  } catch (const Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(DFMM_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(DFMM_ERR_INVALID, e.what());
  }
}

}  // namespace

namespace dfmm {

int set_error(int code, const char* msg) { return fail(code, msg); }

bool plan_acquire(const dfmm_plan_s* plan) {
  std::lock_guard<std::mutex> g(g_plans_mu);
  auto it = g_plans.find(plan);
  if (it == g_plans.end()) return false;
  ++it->second;
  return true;
}

void plan_release(const dfmm_plan_s* plan) {
  std::lock_guard<std::mutex> g(g_plans_mu);
  auto it = g_plans.find(plan);
  if (it != g_plans.end() && it->second > 0) --it->second;
}

int apply_with_scratch(dfmm_plan_s* P, const void* f, void* u, int nrhs, cudaStream_t stream, void* scratch,
                       size_t bytes) {
  return guarded([&]() -> int {
    if (!P || !f || !u) return fail(DFMM_ERR_INVALID, "null argument");
    if (nrhs < 1 || nrhs > 64) return fail(DFMM_ERR_INVALID, "nrhs must be in [1, 64]");
    if (f == u) return fail(DFMM_ERR_INVALID, "f and u must not alias");
    int dev = -1;
    DFMM_CUDA(cudaGetDevice(&dev));
    if (dev != P->device) return fail(DFMM_ERR_INVALID, "the plan belongs to another device");
    Workspace W;
    carve_workspace(P, nrhs, (char*)scratch, bytes, stream, W);
    run_apply(P, (const float2*)f, (float2*)u, nrhs, stream, nullptr, &W);
    return DFMM_OK;
  });
}

}  // namespace dfmm

namespace {

// Per-device pool of streams on which dfmm_apply_batched runs the geometries
// of a batch side by side (created on first use, kept for the process).
constexpr int kBatchStreams = 8;
struct BatchStreams {
  std::mutex mu;
  cudaStream_t s[kBatchStreams] = {};
  cudaEvent_t start = nullptr, done[kBatchStreams] = {};
};

BatchStreams& batch_streams(int dev) {
  static std::mutex mu;
  static std::map<int, std::unique_ptr<BatchStreams>> pools;
  std::lock_guard<std::mutex> g(mu);
  auto& slot = pools[dev];
  if (!slot) {
    std::unique_ptr<BatchStreams> B(new BatchStreams());
    for (int j = 0; j < kBatchStreams; ++j) {
      DFMM_CUDA(cudaStreamCreateWithFlags(&B->s[j], cudaStreamNonBlocking));
      DFMM_CUDA(cudaEventCreateWithFlags(&B->done[j], cudaEventDisableTiming));
    }
    DFMM_CUDA(cudaEventCreateWithFlags(&B->start, cudaEventDisableTiming));
    slot = std::move(B);
  }
  return *slot;
}

}  // namespace

// The batched form with merged stages: the plans of a batch run wave by wave
// (one wave = the same step of every plan, by kind and box width), and the
// split-complex translation stages of a wave run as one launch over a table of
// stages (tiles tagged with their stage).  Work tables and workspaces are laid
// out once, for fixed device buffers f and u, so that a replay can be one
// captured CUDA graph.
struct dfmm_batch_s {
  int device = 0;
  std::vector<dfmm_plan_s*> plans;
  std::vector<int> nrhs;
  std::vector<const float2*> f;
  std::vector<float2*> u;
  DevArena ar;
  std::vector<std::unique_ptr<Workspace>> ws;
  std::vector<int64_t> waves;             // sorted union of the plans' wave keys
  struct Merged {
    int64_t wave = 0;
    int M = 0, Kd = 0, kind = 0, one = 0;
    std::vector<const GemmPlan*> key;     // its stages, in order
    CxStage* stages = nullptr;
    int4* tiles[3] = {nullptr, nullptr, nullptr};   // tile orders: blocked 8 MB, blocked 2 MB, by operator
    int64_t ntiles[3] = {0, 0, 0};
    int choice = 0;
    double ms[3] = {0, 0, 0};
  };
  std::deque<Merged> merged;               // stable references while it grows
  unsigned* status = nullptr;
  int64_t launches = 0;                   // kernel launches of one run
  int tuned = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the plans' per-point kernels of a wave run side by side on these streams
  static constexpr int kSide = 8;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  ~dfmm_batch_s() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (int j = 0; j < kSide; ++j) {
      if (side[j]) cudaStreamDestroy(side[j]);
      if (join[j]) cudaEventDestroy(join[j]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

namespace {

constexpr int kBatchOrders = 3;

void batch_tiles(const GemmPlan& g, int nrhs, int v, std::vector<int4>& out, int stage) {
  std::vector<int4> t = v == 2 ? make_tiles(g, nrhs, gemm_cx_columns(), 2)
                               : make_tiles(g, nrhs, gemm_cx_columns(), 1, (int64_t)(v == 0 ? 8 : 2) << 20);
  for (int4 x : t) {
    x.w = stage;
    out.push_back(x);
  }
}

dfmm_batch_s::Merged& merged_for(dfmm_batch_s* B, int64_t wave, int M, int Kd, int kind, int one,
                                 const std::vector<WaveGemm>& list, cudaStream_t s) {
  std::vector<const GemmPlan*> key;
  for (auto& w : list) key.push_back(w.g);
  for (auto& m : B->merged)
    if (m.wave == wave && m.M == M && m.Kd == Kd && m.kind == kind && m.one == one && m.key == key) return m;
  if (B->exec || B->tuned > 1) throw Error(DFMM_ERR_INVALID, "batch stage tables missing after set-up");
  dfmm_batch_s::Merged m;
  m.wave = wave;
  m.M = M;
  m.Kd = Kd;
  m.kind = kind;
  m.one = one;
  m.key = key;
  std::vector<CxStage> st;
  std::vector<int4> tl[kBatchOrders];
  for (size_t i = 0; i < list.size(); ++i) {
    const WaveGemm& w = list[i];
    CxStage c;
    c.pairs = w.g->pairs;
    c.src_hi = w.W->ahi;
    c.src_lo = w.W->alo;
    c.src_scale = w.W->ascale;
    c.img = w.g->img;
    c.op_scale = w.g->op_scale;
    c.dst = w.dst;
    c.nrhs = w.nrhs;
    c.store = w.store;
    st.push_back(c);
    for (int v = 0; v < kBatchOrders; ++v) batch_tiles(*w.g, w.nrhs, v, tl[v], (int)i);
  }
  m.stages = B->ar.alloc<CxStage>((int64_t)st.size());
  DFMM_CUDA(cudaMemcpyAsync(m.stages, st.data(), st.size() * sizeof(CxStage), cudaMemcpyHostToDevice, s));
  for (int v = 0; v < kBatchOrders; ++v) {
    m.ntiles[v] = (int64_t)tl[v].size();
    m.tiles[v] = B->ar.alloc<int4>(std::max<int64_t>(1, m.ntiles[v]));
    DFMM_CUDA(cudaMemcpyAsync(m.tiles[v], tl[v].data(), tl[v].size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
  B->merged.push_back(m);
  return B->merged.back();
}

// One run of the batch on stream s.  force >= 0: every merged launch takes
// tile order `force` and its time is recorded into ms[force] (autotuning).
// Returns (stages merged, merged launches).
std::pair<int64_t, int64_t> batch_run(dfmm_batch_s* B, cudaStream_t s, int force = -1) {
  int64_t n_stages = 0, n_merged = 0;
  std::vector<std::pair<dfmm_batch_s::Merged*, std::pair<cudaEvent_t, cudaEvent_t>>> timed;
  int64_t launches = 0;
  const int nside = (int)std::min<size_t>(dfmm_batch_s::kSide, B->plans.size());
  for (int64_t wv : B->waves) {
    std::vector<WaveGemm> coll;
    // the plans' other steps of this wave (per-point kernels, stages outside the
    // merged form) on the side streams, after everything queued on s
    DFMM_CUDA(cudaEventRecord(B->fork, s));
    for (int j = 0; j < nside; ++j) DFMM_CUDA(cudaStreamWaitEvent(B->side[j], B->fork, 0));
    for (size_t k = 0; k < B->plans.size(); ++k) {
      WaveCtl c{wv, &coll, nullptr};
      run_apply(B->plans[k], B->f[k], B->u[k], B->nrhs[k], B->side[k % nside], nullptr, B->ws[k].get(), &c);
    }
    for (int j = 0; j < nside; ++j) {
      DFMM_CUDA(cudaEventRecord(B->join[j], B->side[j]));
      DFMM_CUDA(cudaStreamWaitEvent(s, B->join[j], 0));
    }
    // group the collected stages by launch shape, keeping the plans' order
    std::vector<std::pair<std::array<int, 4>, std::vector<WaveGemm>>> groups;
    for (auto& w : coll) {
      std::array<int, 4> sh = {w.g->M, w.g->Kd, w.P->opt.tc_precision, w.P->opt.tc_accumulate};
      auto it = std::find_if(groups.begin(), groups.end(), [&](const auto& g) { return g.first == sh; });
      if (it == groups.end()) groups.push_back({sh, {w}});
      else it->second.push_back(w);
    }
    for (auto& gr : groups) {
      const auto& sh = gr.first;
      auto& list = gr.second;
      dfmm_batch_s::Merged& m = merged_for(B, wv, sh[0], sh[1], sh[2], sh[3], list, s);
      for (auto& w : list)
        if (w.split) {
          launch_split_cx(w.src, w.src_rows * w.nrhs, w.src_ld, w.W->ahi, w.W->alo, w.W->ascale,
                          w.P->opt.tc_precision, s);
          ++launches;
        }
      const int v = force >= 0 ? force : m.choice;
      GemmArgs a{};
      a.M = m.M;
      a.Kd = m.Kd;
      a.tiles = m.tiles[v];
      a.ntiles = m.ntiles[v];
      a.src_ld = m.Kd;
      a.dst_ld = m.M;
      a.nrhs = 1;
      a.stages = m.stages;
      TcArgs t{};
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (force >= 0) {
        DFMM_CUDA(cudaEventCreate(&e0));
        DFMM_CUDA(cudaEventCreate(&e1));
        DFMM_CUDA(cudaEventRecord(e0, s));
      }
      launch_gemm_stage_cx(a, t, B->status, m.one == 1, m.kind, s);
      ++launches;
      ++n_merged;
      n_stages += (int64_t)list.size();
      if (force >= 0) {
        DFMM_CUDA(cudaEventRecord(e1, s));
        timed.push_back({&m, {e0, e1}});
      }
    }
  }
  if (force >= 0) {
    DFMM_CUDA(cudaStreamSynchronize(s));
    for (auto& t : timed) {
      float ms = 0;
      DFMM_CUDA(cudaEventElapsedTime(&ms, t.second.first, t.second.second));
      t.first->ms[force] = ms;
      cudaEventDestroy(t.second.first);
      cudaEventDestroy(t.second.second);
    }
  }
  (void)launches;
  return {n_stages, n_merged};
}

}  // namespace

// --------------------------------------------------------------- C ABI ---

extern "C" {

const char* dfmm_last_error(void) { return g_err.c_str(); }

int dfmm_plan(const double* points, int64_t N, double K, double eps, const dfmm_options* opts, dfmm_plan_t* out) {
  return guarded([&]() -> int {
    if (!out) return fail(DFMM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!points) return fail(DFMM_ERR_INVALID, "points is NULL");
    if (N < 1 || N > (int64_t)INT32_MAX / 2) return fail(DFMM_ERR_INVALID, "N must be in [1, 2^30]");
    if (!(K > 0) || K > 4096) return fail(DFMM_ERR_UNSUPPORTED, "K must be in (0, 4096]");
    if (!(eps >= 1e-8 && eps <= 1e-2)) return fail(DFMM_ERR_UNSUPPORTED, "eps must be in [1e-8, 1e-2]");
    dfmm_options o{};
    if (opts) o = *opts;
    if (o.leaf_max <= 0) o.leaf_max = 64;
    if (o.sample_box <= 0) o.sample_box = 1024;
    if (o.sample_far <= 0) o.sample_far = 4096;
    // eps below 1e-7 needs ranks up to about 320 (and 2r sketch rows)
    if (o.sketch_rows <= 0) o.sketch_rows = eps >= 1e-7 ? 400 : 800;
    // skeleton tolerance eps_op = factor * eps: 0.3 keeps the result within eps down to
    // eps 1e-6; below 1e-7 the errors of more levels add up relative to eps, and
    // 0.1 keeps it within eps at 1e-8
    if (!(o.eps_op_factor > 0)) o.eps_op_factor = eps >= 1e-7 ? 0.3 : 0.1;
    if (o.m2l_mode < 0 || o.m2l_mode > 2) return fail(DFMM_ERR_INVALID, "m2l_mode must be 0, 1 or 2");
    // automatic form: the split-FP16 tensor-core form adds about 2e-6
    // relative error, so it serves eps >= 1e-5; tighter tolerances use FP32
    // CUDA cores
    if (o.m2l_mode == 0) o.m2l_mode = eps >= 1e-5 ? 2 : 1;
    if (o.tc_stages < 0 || o.tc_stages > 31) return fail(DFMM_ERR_INVALID, "tc_stages must be a mask in [0, 31]");
    if (o.tc_stages == 0) o.tc_stages = 31;
    if (o.wait_test < 0 || o.wait_test > 1) return fail(DFMM_ERR_INVALID, "wait_test must be 0 or 1");
    if (o.tile_order < 0 || o.tile_order > 2) return fail(DFMM_ERR_INVALID, "tile_order must be 0, 1 or 2");
    if (o.p2p_mode < 0 || o.p2p_mode > 2) return fail(DFMM_ERR_INVALID, "p2p_mode must be 0, 1 or 2");
    if (o.tc_layout < 0 || o.tc_layout > 1) return fail(DFMM_ERR_INVALID, "tc_layout must be 0 or 1");
    if (o.tc_accumulate < 0 || o.tc_accumulate > 2) return fail(DFMM_ERR_INVALID, "tc_accumulate must be 0, 1 or 2");
    // automatic accumulation: one accumulator per component (the MMAs of a tile
    // overlap the previous tile's epilogue) within the tensor-core form's own
    // range (eps >= 1e-5); the separate cross-term accumulators below it
    if (o.tc_accumulate == 0) o.tc_accumulate = eps >= 1e-5 ? 1 : 2;
    if (o.tc_precision < 0 || o.tc_precision > 2) return fail(DFMM_ERR_INVALID, "tc_precision must be 0, 1 or 2");
    if (o.tc_precision != 0 && o.tc_layout == 1)
      return fail(DFMM_ERR_INVALID, "the BF16 and TF32 splits need the split-complex form (tc_layout 0)");
    if (o.arith != 0 && o.arith != 32 && o.arith != 64) return fail(DFMM_ERR_INVALID, "arith must be 0, 32 or 64");
    if (o.skeleton_host < 0 || o.skeleton_host > 1) return fail(DFMM_ERR_INVALID, "skeleton_host must be 0 or 1");
    // automatic arithmetic: the FP32 forms serve eps >= 1e-6; tighter
    // tolerances compute in FP64 throughout (complex128 densities and potentials)
    if (o.arith == 0) o.arith = eps >= 1e-6 ? 32 : 64;
    if (o.arith == 64) {
      if (opts && opts->m2l_mode == 2)
        return fail(DFMM_ERR_INVALID, "the tensor-core translations are not part of the FP64 form (arith 64)");
      o.m2l_mode = 1;   // translations on the CUDA cores, in FP64
      o.p2p_mode = 1;   // no FP32 near field (and no close-pair pass)
    }
    // automatic near field: FP32 coordinates with exact close-pair
    // corrections for eps >= 1e-5, double-float coordinates below
    if (o.p2p_mode == 0) o.p2p_mode = eps >= 1e-5 ? 2 : 1;
    std::unique_ptr<dfmm_plan_s> P(new dfmm_plan_s());
    DFMM_CUDA(cudaGetDevice(&P->device));
    P->N = N;
    P->K = K;
    P->W = std::pow(2.0, std::max(0.0, std::ceil(std::log2(K))));
    P->eps = eps;
    P->opt = o;
    P->fp64 = o.arith == 64;
    P->cw = P->fp64 ? 2 : 1;
    P->stats.arith = o.arith;
    P->eps_op = eps * o.eps_op_factor;
    P->stats.N = N;
    P->stats.K = K;
    P->stats.W = P->W;
    P->stats.eps = eps;
    P->stats.eps_op = P->eps_op;
    cudaStream_t s;
    DFMM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{s};
    build_plan(P.get(), points, s);
    if (P->opt.m2l_mode == 2) {
      const double ti = now();
      build_images(P.get(), s);
      DFMM_CUDA(cudaStreamSynchronize(s));
      P->stats.plan_phase_seconds[6] = now() - ti;
      P->stats.plan_seconds += P->stats.plan_phase_seconds[6];
    }
    DFMM_CUDA(cudaStreamSynchronize(s));
#ifdef DFMM_CHECK
    validate_plan(P.get(), s, false);   // the bounds-checking build checks every plan it makes
#endif
    {
      std::lock_guard<std::mutex> g(g_plans_mu);
      g_plans[P.get()] = 0;
      P->stats.plan_id = g_next_plan_id++;
    }
    *out = P.release();
    return DFMM_OK;
  });
}

int dfmm_apply(dfmm_plan_t plan, const void* f, void* u, int nrhs, cudaStream_t stream) {
  return guarded([&]() -> int {
    if (!plan || !f || !u) return fail(DFMM_ERR_INVALID, "null argument");
    if (nrhs < 1 || nrhs > 64) return fail(DFMM_ERR_INVALID, "nrhs must be in [1, 64]");
    if (f == u) return fail(DFMM_ERR_INVALID, "f and u must not alias");
    run_apply(plan, (const float2*)f, (float2*)u, nrhs, stream);
    return DFMM_OK;
  });
}

int dfmm_apply_host(dfmm_plan_t plan, const void* f_host, void* u_host, int nrhs, cudaStream_t stream) {
  return guarded([&]() -> int {
    if (!plan || !f_host || !u_host) return fail(DFMM_ERR_INVALID, "null argument");
    if (nrhs < 1 || nrhs > 64) return fail(DFMM_ERR_INVALID, "nrhs must be in [1, 64]");
    Workspace* W = get_workspace(plan, stream, nrhs);
    size_t bytes = (size_t)plan->N * nrhs * sizeof(float2) * plan->cw;
    if (!W->f_dev) {
      W->f_dev = W->ar.alloc<float2>(plan->N * W->nrhs * plan->cw);
      W->u_dev = W->ar.alloc<float2>(plan->N * W->nrhs * plan->cw);
    }
    DFMM_CUDA(cudaMemcpyAsync(W->f_dev, f_host, bytes, cudaMemcpyHostToDevice, stream));
    run_apply(plan, W->f_dev, W->u_dev, nrhs, stream);
    DFMM_CUDA(cudaMemcpyAsync(u_host, W->u_dev, bytes, cudaMemcpyDeviceToHost, stream));
    DFMM_CUDA(cudaStreamSynchronize(stream));
    return DFMM_OK;
  });
}

int dfmm_sync_status(dfmm_plan_t plan, cudaStream_t stream) {
  return guarded([&]() -> int {
    if (!plan) return fail(DFMM_ERR_INVALID, "null plan");
    DFMM_CUDA(cudaStreamSynchronize(stream));
    std::lock_guard<std::mutex> g(plan->ws_mu);
    auto it = plan->ws.find(stream);
    unsigned st = 0;
    if (it != plan->ws.end()) DFMM_CUDA(cudaMemcpy(&st, it->second->status, 4, cudaMemcpyDeviceToHost));
    if (const unsigned* na = noalloc_status_word(stream)) {   // the last allocation-free apply, if on this stream
      unsigned sn = 0;
      DFMM_CUDA(cudaMemcpy(&sn, na, 4, cudaMemcpyDeviceToHost));
      st |= sn;
    }
    if (st & kStatusTimeout) return fail(DFMM_ERR_TIMEOUT, "a device wait gave up");
    if (st) return fail(DFMM_ERR_DEVICE, "a device-side check failed");
    return DFMM_OK;
  });
}

int dfmm_validate(dfmm_plan_t plan, cudaStream_t stream, int flags) {
  return guarded([&]() -> int {
    if (!plan) return fail(DFMM_ERR_INVALID, "null plan");
    if (flags & ~DFMM_VALIDATE_PLANT) return fail(DFMM_ERR_INVALID, "unknown flags");
    validate_plan(plan, stream, (flags & DFMM_VALIDATE_PLANT) != 0);
    return DFMM_OK;
  });
}

int dfmm_destroy(dfmm_plan_t plan) {
  return guarded([&]() -> int {
    if (!plan) return DFMM_OK;
    {
      std::lock_guard<std::mutex> g(g_plans_mu);
      auto it = g_plans.find(plan);
      if (it == g_plans.end()) return fail(DFMM_ERR_INVALID, "not a live plan");
      if (it->second > 0) return fail(DFMM_ERR_INVALID, "the plan has requests queued or running in a server");
      g_plans.erase(it);
    }
    cudaDeviceSynchronize();
    delete plan;
    return DFMM_OK;
  });
}

int dfmm_plan_stats(dfmm_plan_t plan, dfmm_stats* out) {
  if (!plan || !out) return fail(DFMM_ERR_INVALID, "null argument");
  *out = plan->stats;
  return DFMM_OK;
}

int64_t dfmm_apply_workspace_bytes(dfmm_plan_t plan, int nrhs) {
  if (!plan || nrhs < 1 || nrhs > 64) return -1;
  try {
    return workspace_bytes(plan, nrhs);
  } catch (...) {
    return -1;
  }
}

int64_t dfmm_plan_bytes(dfmm_plan_t plan) { return plan ? plan->stats.plan_bytes : -1; }

int dfmm_graph_create(dfmm_plan_t plan, const void* f, void* u, int nrhs, cudaStream_t stream, dfmm_graph_t* out) {
  return guarded([&]() -> int {
    if (!out) return fail(DFMM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!plan || !f || !u) return fail(DFMM_ERR_INVALID, "null argument");
    if (nrhs < 1 || nrhs > 64) return fail(DFMM_ERR_INVALID, "nrhs must be in [1, 64]");
    if (f == u) return fail(DFMM_ERR_INVALID, "f and u must not alias");
    int dev = -1;
    DFMM_CUDA(cudaGetDevice(&dev));
    if (dev != plan->device) return fail(DFMM_ERR_INVALID, "the plan belongs to another device");
    std::unique_ptr<dfmm_graph_s> G(new dfmm_graph_s());
    G->bytes = (size_t)workspace_bytes(plan, nrhs);
    G->scratch = G->ar.alloc<char>(G->bytes);
    // work tables are copied in here, outside the capture
    carve_workspace(plan, nrhs, G->scratch, G->bytes, stream, G->W);
    // one ordinary run first: initialises per-kernel launch attributes
    run_apply(plan, (const float2*)f, (float2*)u, nrhs, stream, nullptr, &G->W);
    DFMM_CUDA(cudaStreamSynchronize(stream));
    cudaStream_t cs;
    DFMM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{cs};
    DFMM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
      run_apply(plan, (const float2*)f, (float2*)u, nrhs, cs, nullptr, &G->W);
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cs, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    DFMM_CUDA(cudaStreamEndCapture(cs, &G->graph));
    DFMM_CUDA(cudaGraphInstantiate(&G->exec, G->graph, 0));
    G->plan = plan;
    *out = G.release();
    return DFMM_OK;
  });
}

int dfmm_graph_launch(dfmm_graph_t graph, cudaStream_t stream) {
  return guarded([&]() -> int {
    if (!graph) return fail(DFMM_ERR_INVALID, "null graph");
    DFMM_CUDA(cudaGraphLaunch(graph->exec, stream));
    return DFMM_OK;
  });
}

int dfmm_graph_destroy(dfmm_graph_t graph) {
  if (!graph) return DFMM_OK;
  cudaDeviceSynchronize();
  delete graph;
  return DFMM_OK;
}

int dfmm_apply_batched(const dfmm_plan_t* plans, const void* const* f, void* const* u, const int* nrhs, int count,
                       cudaStream_t stream) {
  return guarded([&]() -> int {
    if (count < 0) return fail(DFMM_ERR_INVALID, "count must be >= 0");
    if (count == 0) return DFMM_OK;
    if (!plans || !f || !u || !nrhs) return fail(DFMM_ERR_INVALID, "null argument");
    int dev = -1;
    DFMM_CUDA(cudaGetDevice(&dev));
    for (int k = 0; k < count; ++k) {
      if (!plans[k] || !f[k] || !u[k]) return fail(DFMM_ERR_INVALID, "null plan or buffer in the batch");
      if (nrhs[k] < 1 || nrhs[k] > 64) return fail(DFMM_ERR_INVALID, "nrhs must be in [1, 64]");
      if (f[k] == u[k]) return fail(DFMM_ERR_INVALID, "f and u must not alias");
      if (plans[k]->device != dev) return fail(DFMM_ERR_INVALID, "a plan of the batch belongs to another device");
    }
    BatchStreams& B = batch_streams(dev);
    std::lock_guard<std::mutex> g(B.mu);
    // the batch starts after the work already queued on the caller's stream
    DFMM_CUDA(cudaEventRecord(B.start, stream));
    const int ns = std::min(count, kBatchStreams);
    for (int j = 0; j < ns; ++j) DFMM_CUDA(cudaStreamWaitEvent(B.s[j], B.start, 0));
    // geometries are independent: each runs its whole apply on one of the
    // pool's streams, so their stages overlap on the device
    for (int k = 0; k < count; ++k)
      run_apply(plans[k], (const float2*)f[k], (float2*)u[k], nrhs[k], B.s[k % ns]);
    for (int j = 0; j < ns; ++j) {
      DFMM_CUDA(cudaEventRecord(B.done[j], B.s[j]));
      DFMM_CUDA(cudaStreamWaitEvent(stream, B.done[j], 0));
    }
    return DFMM_OK;
  });
}

int dfmm_batch_create(const dfmm_plan_t* plans, const void* const* f, void* const* u, const int* nrhs, int count,
                      cudaStream_t stream, int flags, dfmm_batch_t* out) {
  return guarded([&]() -> int {
    if (!out) return fail(DFMM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (count < 1) return fail(DFMM_ERR_INVALID, "count must be >= 1");
    if (!plans || !f || !u || !nrhs) return fail(DFMM_ERR_INVALID, "null argument");
    if (flags & ~(DFMM_BATCH_GRAPH | DFMM_BATCH_TUNE)) return fail(DFMM_ERR_INVALID, "unknown batch flag");
    int dev = -1;
    DFMM_CUDA(cudaGetDevice(&dev));
    std::unique_ptr<dfmm_batch_s> B(new dfmm_batch_s());
    B->device = dev;
    for (int k = 0; k < count; ++k) {
      if (!plans[k] || !f[k] || !u[k]) return fail(DFMM_ERR_INVALID, "null plan or buffer in the batch");
      if (nrhs[k] < 1 || nrhs[k] > 64) return fail(DFMM_ERR_INVALID, "nrhs must be in [1, 64]");
      if (f[k] == u[k]) return fail(DFMM_ERR_INVALID, "f and u must not alias");
      if (plans[k]->device != dev) return fail(DFMM_ERR_INVALID, "a plan of the batch belongs to another device");
      if (plans[k]->opt.wait_test) return fail(DFMM_ERR_UNSUPPORTED, "wait_test plans cannot be batched");
      B->plans.push_back(plans[k]);
      B->nrhs.push_back(nrhs[k]);
      B->f.push_back((const float2*)f[k]);
      B->u.push_back((float2*)u[k]);
    }
    // one carved workspace per plan (work tables copied in here, before any capture)
    for (int k = 0; k < count; ++k) {
      std::unique_ptr<Workspace> W(new Workspace());
      const size_t bytes = (size_t)workspace_bytes(B->plans[k], B->nrhs[k]);
      char* base = B->ar.alloc<char>((int64_t)bytes);
      carve_workspace(B->plans[k], B->nrhs[k], base, bytes, stream, *W);
      B->ws.push_back(std::move(W));
    }
    B->status = B->ar.alloc<unsigned>(1);
    DFMM_CUDA(cudaMemsetAsync(B->status, 0, 4, stream));
    for (int j = 0; j < dfmm_batch_s::kSide; ++j) {
      DFMM_CUDA(cudaStreamCreateWithFlags(&B->side[j], cudaStreamNonBlocking));
      DFMM_CUDA(cudaEventCreateWithFlags(&B->join[j], cudaEventDisableTiming));
    }
    DFMM_CUDA(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
    // the waves: the union of the plans' wave keys
    for (int k = 0; k < count; ++k) {
      std::vector<int64_t> keys;
      WaveCtl c{0, nullptr, &keys};
      run_apply(B->plans[k], B->f[k], B->u[k], B->nrhs[k], stream, nullptr, B->ws[k].get(), &c);
      B->waves.insert(B->waves.end(), keys.begin(), keys.end());
    }
    std::sort(B->waves.begin(), B->waves.end());
    B->waves.erase(std::unique(B->waves.begin(), B->waves.end()), B->waves.end());
    // first run: lays out the merged stage tables; then the autotuner times each
    // tile order per merged launch and keeps the fastest
    auto nm = batch_run(B.get(), stream);
    if (flags & DFMM_BATCH_TUNE) {
      for (int v = 0; v < kBatchOrders; ++v) batch_run(B.get(), stream, v);
      for (auto& m : B->merged) {
        int best = 0;
        for (int v = 1; v < kBatchOrders; ++v)
          if (m.ms[v] < m.ms[best]) best = v;
        m.choice = best;
      }
      batch_run(B.get(), stream);   // the result of the chosen orders
    }
    B->tuned = 2;
    int64_t total = 0;
    for (int k = 0; k < count; ++k) {
      int64_t c = 0;
      run_apply(B->plans[k], nullptr, nullptr, B->nrhs[k], nullptr, &c);
      total += c;
    }
    B->launches = total - nm.first + nm.second;
    DFMM_CUDA(cudaStreamSynchronize(stream));
    if (flags & DFMM_BATCH_GRAPH) {
      cudaStream_t cs;
      DFMM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{cs};
      DFMM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      try {
        batch_run(B.get(), cs);
      } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      DFMM_CUDA(cudaStreamEndCapture(cs, &B->graph));
      DFMM_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
    }
    *out = B.release();
    return DFMM_OK;
  });
}

int dfmm_batch_launch(dfmm_batch_t batch, cudaStream_t stream) {
  return guarded([&]() -> int {
    if (!batch) return fail(DFMM_ERR_INVALID, "null batch");
    if (batch->exec) DFMM_CUDA(cudaGraphLaunch(batch->exec, stream));
    else batch_run(batch, stream);
    return DFMM_OK;
  });
}

int dfmm_batch_stats(dfmm_batch_t batch, dfmm_batch_report* out) {
  if (!batch || !out) return fail(DFMM_ERR_INVALID, "null argument");
  std::memset(out, 0, sizeof(*out));
  out->launches = batch->launches;
  out->waves = (int64_t)batch->waves.size();
  out->merged_launches = (int64_t)batch->merged.size();
  for (auto& m : batch->merged) {
    out->merged_stages += (int64_t)m.key.size();
    out->order_chosen[m.choice] += 1;
    for (int v = 0; v < kBatchOrders; ++v) out->tune_ms[v] += m.ms[v];
  }
  out->graph = batch->exec ? 1 : 0;
  return DFMM_OK;
}

int dfmm_batch_destroy(dfmm_batch_t batch) {
  if (!batch) return DFMM_OK;
  cudaDeviceSynchronize();
  delete batch;
  return DFMM_OK;
}

int dfmm_export(dfmm_plan_t plan, int what, void* buffer, int64_t* count) {
  return guarded([&]() -> int {
    if (!plan || !count) return fail(DFMM_ERR_INVALID, "null argument");
    std::vector<int64_t> v;
    const auto& LV = plan->tree.levels;
    switch (what) {
      case 0:
        for (auto p : plan->h_perm) v.push_back(p);
        break;
      case 1:
        for (auto k : plan->h_keys) v.push_back((int64_t)k);
        break;
      case 2:
        for (auto& L : LV)
          for (int64_t b = 0; b < L.n; ++b) {
            v.push_back(L.l); v.push_back((int64_t)L.h_prefix[b]); v.push_back(L.h_first[b]);
            v.push_back(L.h_count[b]); v.push_back(L.h_leaf[b]);
          }
        break;
      case 3:
        for (auto& H : plan->hf)
          for (int64_t q = 0; q < H.pairs.n; ++q) {
            v.push_back(H.l); v.push_back(H.pairs.tgt[q]); v.push_back(H.pairs.src[q]);
            v.push_back(H.pairs.din[q]); v.push_back(H.pairs.dout[q]);
          }
        break;
      case 4:
      case 5:
        for (auto& H : plan->hf)
          for (int32_t k : (what == 4 ? H.out_keys : H.in_keys)) {
            v.push_back(H.l); v.push_back(k / H.nd); v.push_back(k % H.nd);
          }
        break;
      case 6:
        for (size_t l = 0; l < plan->vlist.size(); ++l)
          for (int64_t q = 0; q < plan->vlist[l].n; ++q) {
            v.push_back((int64_t)l); v.push_back(plan->vlist[l].tgt[q]); v.push_back(plan->vlist[l].src[q]);
          }
        break;
      case 7:
        for (auto x : plan->U) v.push_back(x);
        break;
      case 8:
        for (auto x : plan->Wl) v.push_back(x);
        break;
      case 9:
        for (auto x : plan->X) v.push_back(x);
        break;
      case 10:
        for (auto& r : plan->rep_ranks) { v.push_back(r[0]); v.push_back(r[1]); v.push_back(r[2]); }
        break;
      default:
        return fail(DFMM_ERR_INVALID, "unknown export id");
    }
    int64_t n = (int64_t)v.size();
    if (buffer) {
      if (*count < n) return fail(DFMM_ERR_INVALID, "export buffer too small");
      std::memcpy(buffer, v.data(), n * sizeof(int64_t));
    }
    *count = n;
    return DFMM_OK;
  });
}

int dfmm_profile(dfmm_plan_t plan, cudaStream_t stream, int enable, dfmm_kernel_time* out, int cap, int* n) {
  return guarded([&]() -> int {
    if (!plan) return fail(DFMM_ERR_INVALID, "null plan");
    Workspace* W;
    {
      std::lock_guard<std::mutex> g(plan->ws_mu);
      auto it = plan->ws.find(stream);
      W = it == plan->ws.end() ? nullptr : it->second.get();
    }
    if (enable) {
      if (!W) W = get_workspace(plan, stream, 1);
      W->prof = true;
      W->recs.clear();
      W->pool_used = 0;
      return DFMM_OK;
    }
    if (n) *n = 0;
    if (!W) return DFMM_OK;
    W->prof = false;
    DFMM_CUDA(cudaStreamSynchronize(stream));
    std::vector<dfmm_kernel_time> tot(F_COUNT);
    for (int f = 0; f < F_COUNT; ++f) {
      std::memset(&tot[f], 0, sizeof(dfmm_kernel_time));
      std::snprintf(tot[f].name, sizeof tot[f].name, "%s", kFamName[f]);
    }
    for (auto& r : W->recs) {
      float ms = 0;
      DFMM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      tot[r.fam].launches += 1;
      tot[r.fam].ms += ms;
      tot[r.fam].flops += r.flops;
      tot[r.fam].bytes += r.bytes;
    }
    W->recs.clear();
    W->pool_used = 0;
    int k = 0;
    for (int f = 0; f < F_COUNT; ++f)
      if (tot[f].launches && out && k < cap) out[k++] = tot[f];
    if (n) *n = k;
    return DFMM_OK;
  });
}

int64_t dfmm_apply_launches(dfmm_plan_t plan, int nrhs) {
  if (!plan || nrhs < 1) return -1;
  int64_t c = 0;
  try {
    run_apply(plan, nullptr, nullptr, nrhs, nullptr, &c);
  } catch (...) {
    return -1;
  }
  return c;
}

}  // extern "C"

namespace {

int representation_impl(bool on_device, double w, int cell, double w_top, double eps_op, int sample_box,
                        int sample_far, int sketch_rows, int* r_out, double* b2, double* a2, int cap) {
  return guarded([&]() -> int {
    if (!r_out) return fail(DFMM_ERR_INVALID, "r_out is NULL");
    if (!(w > 0) || !(w_top >= 1) || !(eps_op > 0)) return fail(DFMM_ERR_INVALID, "bad representation arguments");
    if ((cell < 0) != (w < 1)) return fail(DFMM_ERR_INVALID, "cell must be -1 exactly for w < 1");
    if (cell >= 0 && cell >= 6 * n_cells(w) * n_cells(w)) return fail(DFMM_ERR_INVALID, "cell out of range");
    SkelParams sp;
    sp.eps_op = eps_op;
    sp.S_Y = sample_box > 0 ? sample_box : 1024;
    sp.S_X = sample_far > 0 ? sample_far : 4096;
    sp.sketch = sketch_rows > 0 ? sketch_rows : 400;
    Rep r;
    if (on_device) {
      const Samples sm = make_samples(w, cell, w_top, sp);
      std::vector<SketchJob> sj(1);
      sj[0].sm = &sm;
      sketch_pivots_device(sj, sp);
      std::vector<CheckJob> cj(1);
      cj[0].sm = &sm;
      cj[0].r = rank_from_pivots(sj[0].diag, (int)sj[0].piv.size(), sp);
      cj[0].b = box_points(sm, sj[0].piv, cj[0].r);
      check_pivots_device(cj);
      r = finish_rep(sm, sj[0].piv, cj[0].r, cj[0].p1, cj[0].p2);
    } else {
      r = build_rep(w, cell, w_top, sp);
    }
    *r_out = r.r;
    if (b2 || a2) {
      if (2 * r.r > cap) return fail(DFMM_ERR_INVALID, "buffer capacity below 2r");
      if (b2) std::memcpy(b2, r.b2.data(), r.b2.size() * 8);
      if (a2) std::memcpy(a2, r.a2.data(), r.a2.size() * 8);
    }
    return DFMM_OK;
  });
}

}  // namespace

extern "C" {

int dfmm_representation(double w, int cell, double w_top, double eps_op, int sample_box, int sample_far,
                        int sketch_rows, int* r_out, double* b2, double* a2, int cap) {
  return representation_impl(false, w, cell, w_top, eps_op, sample_box, sample_far, sketch_rows, r_out, b2, a2, cap);
}

int dfmm_representation_device(double w, int cell, double w_top, double eps_op, int sample_box, int sample_far,
                               int sketch_rows, int* r_out, double* b2, double* a2, int cap) {
  return representation_impl(true, w, cell, w_top, eps_op, sample_box, sample_far, sketch_rows, r_out, b2, a2, cap);
}

}  // extern "C"
