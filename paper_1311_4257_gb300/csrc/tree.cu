// Octree (Sec. 2.2) and interaction lists on the device.
//
// Tree: built level by level from the Morton-sorted keys.  A level-l box is
// split if it is a high-frequency box (w >= 1) holding a point, or a
// low-frequency box holding more than leaf_max points, and l < 21.
//
// Lists (all predicates in integer arithmetic):
//   HF (w >= 1, Sec. 2.2): A in I^B iff same width, parent(A) in N^{parent(B)}
//     and A not in N^B, where "A in N^B" reads: the closed box A has a point
//     within w^2 of B's centre, i.e.  sum_d max(0, 2|m_d| - 1)^2 <= 4 w^2  for
//     the offset m = (c_A - c_B) / w.  Direction of a pair (Alg. 1): B's
//     incoming direction is dir(m), A's outgoing direction dir(-m).
//   LF (kernel-independent FMM lists): V = children of the parent's colleagues
//     that do not touch B; U = leaves touching a leaf; W = descendants of a
//     leaf's colleagues that do not touch it while their parent does.
#include "tree.h"

#include <vector>

namespace dfmm {

namespace {

__device__ __forceinline__ uint64_t interleave3(int64_t x, int64_t y, int64_t z) {
  uint64_t k = 0;
#pragma unroll
  for (int b = 0; b < kLevelBits; ++b) {
    k |= ((uint64_t)(x >> b) & 1ull) << (3 * b + 2);
    k |= ((uint64_t)(y >> b) & 1ull) << (3 * b + 1);
    k |= ((uint64_t)(z >> b) & 1ull) << (3 * b);
  }
  return k;
}

__device__ __forceinline__ int64_t lookup(const LevelPtrs& L, int64_t x, int64_t y, int64_t z) {
  int64_t side = 1ll << L.l;
  if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) return -1;
  uint64_t key = interleave3(x, y, z);
  int64_t lo = 0, hi = L.n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (L.prefix[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < L.n && L.prefix[lo] == key) ? lo : -1;
}

__device__ __forceinline__ bool hf_near_dev(int64_t mx, int64_t my, int64_t mz, int64_t lim) {
  int64_t a = 2 * (mx < 0 ? -mx : mx) - 1, b = 2 * (my < 0 ? -my : my) - 1, c = 2 * (mz < 0 ? -mz : mz) - 1;
  a = a < 0 ? 0 : a; b = b < 0 ? 0 : b; c = c < 0 ? 0 : c;
  return a * a + b * b + c * c <= lim;
}

// closed boxes (integer coordinates at levels la, lb) touch or overlap
__device__ __forceinline__ bool touch(const int32_t* ca, int la, const int32_t* cb, int lb) {
  int L = la > lb ? la : lb;
  int64_t sa = 1ll << (L - la), sb = 1ll << (L - lb);
  for (int d = 0; d < 3; ++d) {
    int64_t alo = (int64_t)ca[d] * sa, ahi = alo + sa;
    int64_t blo = (int64_t)cb[d] * sb, bhi = blo + sb;
    if (alo > bhi || blo > ahi) return false;
  }
  return true;
}

// ---------------------------------------------------------------- tree ---

__global__ void box_of_points_kernel(const int32_t* first, const int32_t* count, int64_t nb, int32_t* box_of) {
  int64_t b = blockIdx.x;
  if (b >= nb) return;
  for (int64_t i = first[b] + threadIdx.x; i < first[b] + count[b]; i += blockDim.x) box_of[i] = (int32_t)b;
}

__global__ void split_flags_kernel(const int32_t* count, int64_t nb, int hf, int leaf_max, int at_max,
                                   uint8_t* leaf) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  bool split = hf ? count[b] > 0 : count[b] > leaf_max;
  if (at_max) split = false;
  leaf[b] = split ? 0 : 1;
}

__global__ void child_start_kernel(const uint64_t* keys, int64_t n, const int32_t* box_of, const int32_t* first,
                                   const uint8_t* leaf, int shift, int64_t* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t b = box_of[i];
  int64_t f = 0;
  if (b >= 0 && !leaf[b]) {
    if (i == first[b] || (keys[i] >> shift) != (keys[i - 1] >> shift)) f = 1;
  }
  flag[i] = f;
}

__global__ void child_fill_kernel(const uint64_t* keys, int64_t n, const int32_t* box_of, const int64_t* flag,
                                  const int64_t* pos, int shift, int child_level, uint64_t* cprefix,
                                  int32_t* cfirst, int32_t* cparent, int32_t* ccoords) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  int64_t c = pos[i];
  uint64_t p = keys[i] >> shift;
  cprefix[c] = p;
  cfirst[c] = (int32_t)i;
  cparent[c] = box_of[i];
  int32_t x = 0, y = 0, z = 0;
  for (int b = 0; b < child_level; ++b) {
    x |= (int32_t)((p >> (3 * b + 2)) & 1ull) << b;
    y |= (int32_t)((p >> (3 * b + 1)) & 1ull) << b;
    z |= (int32_t)((p >> (3 * b)) & 1ull) << b;
  }
  ccoords[3 * c] = x;
  ccoords[3 * c + 1] = y;
  ccoords[3 * c + 2] = z;
}

__global__ void child_count_kernel(const int32_t* cfirst, const int32_t* cparent, int64_t nc, const int32_t* pfirst,
                                   const int32_t* pcount, int32_t* ccount, int32_t* pchild_first,
                                   int32_t* pnchild) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int32_t p = cparent[c];
  bool last = (c + 1 == nc) || cparent[c + 1] != p;
  int64_t end = last ? (int64_t)pfirst[p] + pcount[p] : cfirst[c + 1];
  ccount[c] = (int32_t)(end - cfirst[c]);
  if (c == 0 || cparent[c - 1] != p) {
    int k = 1;
    while (c + k < nc && cparent[c + k] == p) ++k;
    pchild_first[p] = (int32_t)c;
    pnchild[p] = k;
  }
}

// ---------------------------------------------------------- pair lists ---

// One thread per (target box B, template entry t): the parent-level
// neighbour P' = parent(B) + T[t]; each child A of P' kept by the predicate.
template <bool FILL>
__global__ void pairs_kernel(const LevelPtrs* lv, int l, const int32_t* tmpl, int nt, int mode, int64_t lim,
                             int64_t* counts, const int64_t* offs, int32_t* tgt, int32_t* src, int32_t* mvec) {
  const LevelPtrs& L = lv[l];
  const LevelPtrs& P = lv[l - 1];
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n * nt) return;
  int64_t B = g / nt;
  int t = (int)(g % nt);
  int32_t pb = L.parent[B];
  int64_t pp = lookup(P, (int64_t)P.coords[3 * pb] + tmpl[3 * t], (int64_t)P.coords[3 * pb + 1] + tmpl[3 * t + 1],
                      (int64_t)P.coords[3 * pb + 2] + tmpl[3 * t + 2]);
  int64_t cnt = 0;
  int64_t o = FILL ? offs[g] : 0;
  if (pp >= 0) {
    int32_t cf = P.child_first[pp], nc = P.nchild[pp];
    for (int k = 0; k < nc; ++k) {
      int64_t A = cf + k;
      int64_t mx = (int64_t)L.coords[3 * A] - L.coords[3 * B];
      int64_t my = (int64_t)L.coords[3 * A + 1] - L.coords[3 * B + 1];
      int64_t mz = (int64_t)L.coords[3 * A + 2] - L.coords[3 * B + 2];
      bool keep;
      if (mode == 0) keep = !hf_near_dev(mx, my, mz, lim);
      else {
        int64_t ax = mx < 0 ? -mx : mx, ay = my < 0 ? -my : my, az = mz < 0 ? -mz : mz;
        int64_t mm = ax > ay ? ax : ay;
        mm = mm > az ? mm : az;
        keep = mm >= 2;
      }
      if (!keep) continue;
      if (FILL) {
        int64_t q = o + cnt;
        tgt[q] = (int32_t)B;
        src[q] = (int32_t)A;
        mvec[3 * q] = (int32_t)mx;
        mvec[3 * q + 1] = (int32_t)my;
        mvec[3 * q + 2] = (int32_t)mz;
      }
      ++cnt;
    }
  }
  if (!FILL) counts[g] = cnt;
}

// Direction index of a nonzero offset on the n x n face grids: closed cells,
// ties to the lexicographically first (face, i, j), faces +x,-x,+y,-y,+z,-z.
__device__ __forceinline__ int32_t direction_dev(int64_t m0, int64_t m1, int64_t m2, int64_t n) {
  int64_t a0 = m0 < 0 ? -m0 : m0, a1 = m1 < 0 ? -m1 : m1, a2 = m2 < 0 ? -m2 : m2;
  int64_t M = a0 > a1 ? a0 : a1;
  M = M > a2 ? M : a2;
  int a;
  int64_t ma, mb, mc;
  if (a0 == M) { a = 0; ma = m0; mb = m1; mc = m2; }
  else if (a1 == M) { a = 1; ma = m1; mb = m0; mc = m2; }
  else { a = 2; ma = m2; mb = m0; mc = m1; }
  int64_t face = 2 * a + (ma < 0 ? 1 : 0);
  int64_t q = 2 * M;
  int64_t pi = n * (mb + M), pj = n * (mc + M);
  int64_t i = (pi + q - 1) / q - 1;
  int64_t j = (pj + q - 1) / q - 1;
  i = i < 0 ? 0 : i;
  j = j < 0 ? 0 : j;
  return (int32_t)((face * n + i) * n + j);
}

__global__ void directions_kernel(const int32_t* mvec, int64_t np, int64_t n, int32_t* din, int32_t* dout) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  int64_t m0 = mvec[3 * q], m1 = mvec[3 * q + 1], m2 = mvec[3 * q + 2];
  din[q] = direction_dev(m0, m1, m2, n);
  dout[q] = direction_dev(-m0, -m1, -m2, n);
}

// U and W lists of the leaves of level l (one thread per leaf).
template <bool FILL>
__global__ void uw_kernel(const LevelPtrs* lv, int l, int l_lf0, const int32_t* leaves, int64_t nleaves,
                          int64_t* ucount, int64_t* wcount, const int64_t* uoffs, const int64_t* woffs,
                          int32_t* U, int32_t* Wl, unsigned* status) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nleaves) return;
  const LevelPtrs& L = lv[l];
  int64_t b = leaves[g];
  const int32_t* cb = L.coords + 3 * b;
  int64_t nu = 0, nw = 0;
  int64_t uo = FILL ? uoffs[g] : 0, wo = FILL ? woffs[g] : 0;
  auto emitU = [&](int la, int64_t a) {
    if (FILL) {
      int64_t q = uo + nu;
      U[4 * q] = l; U[4 * q + 1] = (int32_t)b; U[4 * q + 2] = la; U[4 * q + 3] = (int32_t)a;
    }
    ++nu;
  };
  auto emitW = [&](int la, int64_t a) {
    if (FILL) {
      int64_t q = wo + nw;
      Wl[4 * q] = l; Wl[4 * q + 1] = (int32_t)b; Wl[4 * q + 2] = la; Wl[4 * q + 3] = (int32_t)a;
    }
    ++nw;
  };
  // coarser leaves touching b: colleagues of b's LF ancestors
  int64_t anc = b;
  for (int la = l - 1; la >= l_lf0; --la) {
    anc = lv[la + 1].parent[anc];
    const LevelPtrs& A = lv[la];
    for (int t = 0; t < 27; ++t) {
      int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
      int64_t a = lookup(A, (int64_t)A.coords[3 * anc] + dx, (int64_t)A.coords[3 * anc + 1] + dy,
                         (int64_t)A.coords[3 * anc + 2] + dz);
      if (a >= 0 && A.leaf[a] && touch(A.coords + 3 * a, la, cb, l)) emitU(la, a);
    }
  }
  // same level and finer
  int64_t stk_l[192], stk_b[192];
  for (int t = 0; t < 27; ++t) {
    int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
    int64_t c = lookup(L, (int64_t)cb[0] + dx, (int64_t)cb[1] + dy, (int64_t)cb[2] + dz);
    if (c < 0) continue;
    if (L.leaf[c]) { emitU(l, c); continue; }
    int sp = 0;
    stk_l[sp] = l; stk_b[sp] = c; ++sp;
    while (sp > 0) {
      --sp;
      int lc = (int)stk_l[sp];
      int64_t bc = stk_b[sp];
      const LevelPtrs& Lc = lv[lc];
      const LevelPtrs& La = lv[lc + 1];
      for (int k = 0; k < Lc.nchild[bc]; ++k) {
        int64_t a = Lc.child_first[bc] + k;
        if (touch(La.coords + 3 * a, lc + 1, cb, l)) {
          if (La.leaf[a]) emitU(lc + 1, a);
          else if (sp < 192) { stk_l[sp] = lc + 1; stk_b[sp] = a; ++sp; }
          else atomicOr(status, kStatusBounds);
        } else {
          emitW(lc + 1, a);
        }
      }
    }
  }
  if (!FILL) { ucount[g] = nu; wcount[g] = nw; }
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// --------------------------------------------------------------- host side ---

void TreeBuilder::build(const uint64_t* d_keys, int64_t N, double W, int leaf_max, cudaStream_t s, DevArena& ar) {
  levels.clear();
  int32_t* box_of = ar.alloc<int32_t>(N);
  int64_t* flag = ar.alloc<int64_t>(N);
  int64_t* pos = ar.alloc<int64_t>(N + 1);
  void* scratch = ar.alloc<char>(scan_scratch_bytes(N));
  size_t scratch_bytes = scan_scratch_bytes(N);
  // level 0
  TreeLevel L0;
  L0.l = 0;
  L0.w = W;
  L0.n = 1;
  L0.prefix = ar.alloc<uint64_t>(1);
  L0.coords = ar.alloc<int32_t>(3);
  L0.first = ar.alloc<int32_t>(1);
  L0.count = ar.alloc<int32_t>(1);
  L0.parent = ar.alloc<int32_t>(1);
  {
    uint64_t p0 = 0;
    int32_t c3[3] = {0, 0, 0}, f0 = 0, n0 = (int32_t)N, pm = -1;
    DFMM_CUDA(cudaMemcpyAsync(L0.prefix, &p0, 8, cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(L0.coords, c3, 12, cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(L0.first, &f0, 4, cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(L0.count, &n0, 4, cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaMemcpyAsync(L0.parent, &pm, 4, cudaMemcpyHostToDevice, s));
    DFMM_CUDA(cudaStreamSynchronize(s));
  }
  levels.push_back(L0);
  for (int l = 0;; ++l) {
    TreeLevel& L = levels[l];
    L.leaf = ar.alloc<uint8_t>(L.n);
    L.child_first = ar.alloc<int32_t>(L.n);
    L.nchild = ar.alloc<int32_t>(L.n);
    DFMM_CUDA(cudaMemsetAsync(L.child_first, 0, L.n * 4, s));
    DFMM_CUDA(cudaMemsetAsync(L.nchild, 0, L.n * 4, s));
    split_flags_kernel<<<blocks(L.n, 256), 256, 0, s>>>(L.count, L.n, L.w >= 1.0 ? 1 : 0, leaf_max,
                                                         l == kLevelBits ? 1 : 0, L.leaf);
    DFMM_CUDA(cudaMemsetAsync(box_of, 0xff, N * 4, s));
    box_of_points_kernel<<<(unsigned)L.n, 128, 0, s>>>(L.first, L.count, L.n, box_of);
    int shift = 3 * (kLevelBits - (l + 1));
    if (l == kLevelBits) break;
    child_start_kernel<<<blocks(N, 256), 256, 0, s>>>(d_keys, N, box_of, L.first, L.leaf, shift, flag);
    exclusive_scan_i64(flag, pos, N, scratch, scratch_bytes, s);
    int64_t nc = 0;
    DFMM_CUDA(cudaMemcpyAsync(&nc, pos + N, 8, cudaMemcpyDeviceToHost, s));
    DFMM_CUDA(cudaStreamSynchronize(s));
    if (nc == 0) break;
    TreeLevel C;
    C.l = l + 1;
    C.w = W / (double)(1ll << (l + 1));
    C.n = nc;
    C.prefix = ar.alloc<uint64_t>(nc);
    C.coords = ar.alloc<int32_t>(3 * nc);
    C.first = ar.alloc<int32_t>(nc);
    C.count = ar.alloc<int32_t>(nc);
    C.parent = ar.alloc<int32_t>(nc);
    child_fill_kernel<<<blocks(N, 256), 256, 0, s>>>(d_keys, N, box_of, flag, pos, shift, l + 1, C.prefix,
                                                     C.first, C.parent, C.coords);
    child_count_kernel<<<blocks(nc, 256), 256, 0, s>>>(C.first, C.parent, nc, L.first, L.count, C.count,
                                                       L.child_first, L.nchild);
    DFMM_CUDA(cudaGetLastError());
    levels.push_back(C);
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
  // device table of level pointers
  std::vector<LevelPtrs> h(levels.size());
  for (size_t i = 0; i < levels.size(); ++i) h[i] = levels[i].ptrs();
  d_levels = ar.alloc<LevelPtrs>(levels.size());
  DFMM_CUDA(cudaMemcpyAsync(d_levels, h.data(), h.size() * sizeof(LevelPtrs), cudaMemcpyHostToDevice, s));
  // host copies
  for (auto& L : levels) L.download(s);
  DFMM_CUDA(cudaStreamSynchronize(s));
}

void TreeLevel::download(cudaStream_t s) {
  h_prefix.resize(n); h_coords.resize(3 * n); h_first.resize(n); h_count.resize(n); h_parent.resize(n);
  h_child_first.resize(n); h_nchild.resize(n); h_leaf.resize(n);
  DFMM_CUDA(cudaMemcpyAsync(h_prefix.data(), prefix, n * 8, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(h_coords.data(), coords, n * 12, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(h_first.data(), first, n * 4, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(h_count.data(), count, n * 4, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(h_parent.data(), parent, n * 4, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(h_child_first.data(), child_first, n * 4, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(h_nchild.data(), nchild, n * 4, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(h_leaf.data(), leaf, n, cudaMemcpyDeviceToHost, s));
}

PairList TreeBuilder::pairs(int l, const std::vector<int32_t>& tmpl, int mode, int64_t lim, bool dirs, int ncell,
                            cudaStream_t s, DevArena& ar) {
  PairList out;
  const TreeLevel& L = levels[l];
  int nt = (int)(tmpl.size() / 3);
  int64_t ng = L.n * nt;
  if (ng == 0) return out;
  ArenaMark mark(ar);
  int32_t* d_tmpl = ar.alloc<int32_t>(tmpl.size());
  DFMM_CUDA(cudaMemcpyAsync(d_tmpl, tmpl.data(), tmpl.size() * 4, cudaMemcpyHostToDevice, s));
  int64_t* counts = ar.alloc<int64_t>(ng);
  int64_t* offs = ar.alloc<int64_t>(ng + 1);
  size_t sb = scan_scratch_bytes(ng);
  void* scratch = ar.alloc<char>(sb);
  pairs_kernel<false><<<blocks(ng, 256), 256, 0, s>>>(d_levels, l, d_tmpl, nt, mode, lim, counts, nullptr,
                                                      nullptr, nullptr, nullptr);
  exclusive_scan_i64(counts, offs, ng, scratch, sb, s);
  int64_t np = 0;
  DFMM_CUDA(cudaMemcpyAsync(&np, offs + ng, 8, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaStreamSynchronize(s));
  out.n = np;
  if (np == 0) return out;
  int32_t* tgt = ar.alloc<int32_t>(np);
  int32_t* src = ar.alloc<int32_t>(np);
  int32_t* mv = ar.alloc<int32_t>(3 * np);
  pairs_kernel<true><<<blocks(ng, 256), 256, 0, s>>>(d_levels, l, d_tmpl, nt, mode, lim, nullptr, offs, tgt, src,
                                                     mv);
  out.tgt.resize(np); out.src.resize(np); out.m.resize(3 * np);
  DFMM_CUDA(cudaMemcpyAsync(out.tgt.data(), tgt, np * 4, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(out.src.data(), src, np * 4, cudaMemcpyDeviceToHost, s));
  DFMM_CUDA(cudaMemcpyAsync(out.m.data(), mv, np * 12, cudaMemcpyDeviceToHost, s));
  if (dirs) {
    int32_t* din = ar.alloc<int32_t>(np);
    int32_t* dout = ar.alloc<int32_t>(np);
    directions_kernel<<<blocks(np, 256), 256, 0, s>>>(mv, np, ncell, din, dout);
    out.din.resize(np); out.dout.resize(np);
    DFMM_CUDA(cudaMemcpyAsync(out.din.data(), din, np * 4, cudaMemcpyDeviceToHost, s));
    DFMM_CUDA(cudaMemcpyAsync(out.dout.data(), dout, np * 4, cudaMemcpyDeviceToHost, s));
  }
  DFMM_CUDA(cudaStreamSynchronize(s));
  return out;
}

void TreeBuilder::uw_lists(int l_lf0, cudaStream_t s, DevArena& ar, std::vector<int32_t>& U,
                           std::vector<int32_t>& Wl, unsigned* d_status) {
  U.clear();
  Wl.clear();
  for (size_t l = l_lf0; l < levels.size(); ++l) {
    const TreeLevel& L = levels[l];
    std::vector<int32_t> leaves;
    for (int64_t b = 0; b < L.n; ++b) if (L.h_leaf[b]) leaves.push_back((int32_t)b);
    int64_t nl = (int64_t)leaves.size();
    if (nl == 0) continue;
    ArenaMark mark(ar);
    int32_t* d_leaves = ar.alloc<int32_t>(nl);
    DFMM_CUDA(cudaMemcpyAsync(d_leaves, leaves.data(), nl * 4, cudaMemcpyHostToDevice, s));
    int64_t* uc = ar.alloc<int64_t>(nl);
    int64_t* wc = ar.alloc<int64_t>(nl);
    int64_t* uo = ar.alloc<int64_t>(nl + 1);
    int64_t* wo = ar.alloc<int64_t>(nl + 1);
    size_t sb = scan_scratch_bytes(nl);
    void* scratch = ar.alloc<char>(sb);
    uw_kernel<false><<<blocks(nl, 128), 128, 0, s>>>(d_levels, (int)l, l_lf0, d_leaves, nl, uc, wc, nullptr,
                                                     nullptr, nullptr, nullptr, d_status);
    exclusive_scan_i64(uc, uo, nl, scratch, sb, s);
    exclusive_scan_i64(wc, wo, nl, scratch, sb, s);
    int64_t nu = 0, nw = 0;
    DFMM_CUDA(cudaMemcpyAsync(&nu, uo + nl, 8, cudaMemcpyDeviceToHost, s));
    DFMM_CUDA(cudaMemcpyAsync(&nw, wo + nl, 8, cudaMemcpyDeviceToHost, s));
    DFMM_CUDA(cudaStreamSynchronize(s));
    int32_t* dU = ar.alloc<int32_t>(4 * (nu + 1));
    int32_t* dW = ar.alloc<int32_t>(4 * (nw + 1));
    uw_kernel<true><<<blocks(nl, 128), 128, 0, s>>>(d_levels, (int)l, l_lf0, d_leaves, nl, nullptr, nullptr, uo,
                                                    wo, dU, dW, d_status);
    size_t u0 = U.size(), w0 = Wl.size();
    U.resize(u0 + 4 * nu);
    Wl.resize(w0 + 4 * nw);
    DFMM_CUDA(cudaMemcpyAsync(U.data() + u0, dU, nu * 16, cudaMemcpyDeviceToHost, s));
    DFMM_CUDA(cudaMemcpyAsync(Wl.data() + w0, dW, nw * 16, cudaMemcpyDeviceToHost, s));
    DFMM_CUDA(cudaStreamSynchronize(s));
  }
}

}  // namespace dfmm
