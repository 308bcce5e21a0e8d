// lpa_fold.cuh -- device building blocks of the sweep: the register sketches (weighted
// Misra-Gries, weighted Boyer-Moore), the pipelined row fold, and the work decomposition
// over the binned graph (hub CTAs, mid-degree leaf groups, degree-sorted low rows).
#pragma once

#include "lpa_internal.cuh"

namespace lpa {

constexpr unsigned kFullMask = 0xffffffffu;

// ---------------------------------------------------------------- MG sketch

// k-slot weighted Misra-Gries sketch held in registers (Sec. 4.1, Alg. 2).  Empty slots
// hold key -1 and value 0; labels are >= 0, so a key only matches an occupied slot.
template <int K>
struct MGSketch {
  int key[K];
  float val[K];
  static constexpr int kSlots = K;

  __device__ __forceinline__ void init(int /*own*/) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      key[s] = -1;
      val[s] = 0.f;
    }
  }

  __device__ __forceinline__ unsigned empty_mask() const {
    unsigned em = 0;
#pragma unroll
    for (int s = 0; s < K; ++s) em |= (val[s] == 0.f ? 1u : 0u) << s;
    return em;
  }

  // (c, w) into the lowest free slot named by the non-zero mask em
  __device__ __forceinline__ void place(unsigned em, int c, float w) {
    const int s0 = __ffs(em) - 1;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      key[s] = (s == s0) ? c : key[s];
      val[s] = (s == s0) ? w : val[s];
    }
  }

  // sketchAccumulate with the clamped decrement: add to a matching slot, else fill the
  // lowest free slot, else lower every slot and w by min(w, smallest slot) and put a
  // positive remainder in the lowest slot that became free
  __device__ __forceinline__ void add(int c, float w) {
    bool hit = false;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const bool m = (key[s] == c);
      val[s] = m ? val[s] + w : val[s];
      hit = hit || m;
    }
    if (hit) return;
    unsigned em = empty_mask();
    if (em) {
      place(em, c, w);
      return;
    }
    float lo[K];
#pragma unroll
    for (int s = 0; s < K; ++s) lo[s] = val[s];
#pragma unroll
    for (int h = K / 2; h >= 1; h /= 2)
#pragma unroll
      for (int s = 0; s < h; ++s) lo[s] = fminf(lo[s], lo[s + h]);
    const float delta = fminf(w, lo[0]);
#pragma unroll
    for (int s = 0; s < K; ++s) {
      val[s] = val[s] - delta;
      key[s] = (val[s] == 0.f) ? -1 : key[s];
    }
    w = w - delta;
    if (w > 0.f) place(empty_mask(), c, w);
  }

  // merge(A = this, B): B's occupied slots in ascending slot order (Sec. 4.3)
  __device__ __forceinline__ void merge_from(const int* bk, const float* bv) {
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (bv[s] > 0.f) add(bk[s], bv[s]);
  }

  // receive lane + s's sketch; merge it when `take`
  __device__ __forceinline__ void shfl_merge(int s, bool take) {
    int bk[K];
    float bv[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      bk[q] = __shfl_down_sync(kFullMask, key[q], s);
      bv[q] = __shfl_down_sync(kFullMask, val[q], s);
    }
    if (take) merge_from(bk, bv);
  }

  // sketchMaxKey, single scan (Sec. 4.4): heaviest occupied slot, ties to the smallest
  // label; -1 when the sketch is empty
  __device__ __forceinline__ int choose() const {
    int best = -1;
    float bv = 0.f;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const bool better = (val[s] > bv) || (val[s] == bv && val[s] > 0.f && key[s] < best);
      best = better ? key[s] : best;
      bv = better ? val[s] : bv;
    }
    return best;
  }

  __device__ __forceinline__ void store(int* k, float* v) const {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      k[s] = key[s];
      v[s] = val[s];
    }
  }
  __device__ __forceinline__ void load(const int* k, const float* v) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      key[s] = k[s];
      val[s] = v[s];
    }
  }
};

// ---------------------------------------------------------------- BM state

// Weighted Boyer-Moore candidate (Sec. 4.7, Alg. 3) as printed: same label adds, a
// lighter other label subtracts, otherwise the other label replaces the candidate.
struct BMState {
  int c;
  float w;
  static constexpr int kSlots = 1;

  __device__ __forceinline__ void init(int own) {
    c = own;
    w = 0.f;
  }
  __device__ __forceinline__ void add(int lab, float wt) {
    if (lab == c) {
      w = w + wt;
    } else if (w > wt) {
      w = w - wt;
    } else {
      c = lab;
      w = wt;
    }
  }
  // pair max of partial results: larger w#, ties to the smaller label
  __device__ __forceinline__ void take_better(int oc, float ow) {
    const bool better = (ow > w) || (ow == w && oc < c);
    c = better ? oc : c;
    w = better ? ow : w;
  }
  __device__ __forceinline__ void shfl_merge(int s, bool take) {
    const int oc = __shfl_down_sync(kFullMask, c, s);
    const float ow = __shfl_down_sync(kFullMask, w, s);
    if (take) take_better(oc, ow);
  }
  __device__ __forceinline__ void merge_from(const int* k, const float* v) { take_better(k[0], v[0]); }
  __device__ __forceinline__ int choose() const { return w > 0.f ? c : -1; }
  __device__ __forceinline__ void store(int* k, float* v) const {
    k[0] = c;
    v[0] = w;
  }
  __device__ __forceinline__ void load(const int* k, const float* v) {
    c = k[0];
    w = v[0];
  }
};

// ------------------------------------------------------------ pipelined row fold

// Load the aligned group of four CSR positions starting at g (a multiple of 4).
// Positions outside [b, e) come back with index `self` and weight 0, so the caller
// skips them.  A group that would cross the end of the arrays is read element-wise.
template <bool WT>
__device__ __forceinline__ void load_group(const int32_t* __restrict__ idx,
                                           const float* __restrict__ wts, int64_t m, int64_t g,
                                           int64_t b, int64_t e, int self, int4& J, float4& W) {
  int j[4];
  float w[4];
  if (g + 3 < m) {
    const int4 jj = __ldg(reinterpret_cast<const int4*>(idx + g));
    j[0] = jj.x, j[1] = jj.y, j[2] = jj.z, j[3] = jj.w;
    if (WT) {
      const float4 ww = __ldg(reinterpret_cast<const float4*>(wts + g));
      w[0] = ww.x, w[1] = ww.y, w[2] = ww.z, w[3] = ww.w;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      j[u] = (g + u < m) ? __ldg(idx + g + u) : self;
      if (WT) w[u] = (g + u < m) ? __ldg(wts + g + u) : 0.f;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const bool in = (g + u >= b) && (g + u < e);
    if (!WT) w[u] = 1.f;
    j[u] = in ? j[u] : self;
    w[u] = in ? w[u] : 0.f;
  }
  J = make_int4(j[0], j[1], j[2], j[3]);
  W = make_float4(w[0], w[1], w[2], w[3]);
}

// Neighbour labels of a group: -1 where the position is skipped (outside the range, a
// self-loop when SKIP_SELF, or a weight that is not positive).
template <bool SKIP_SELF>
__device__ __forceinline__ int4 gather_group(const int32_t* __restrict__ lab, const int4& J,
                                             const float4& W, int self) {
  int c[4];
  const int j[4] = {J.x, J.y, J.z, J.w};
  const float w[4] = {W.x, W.y, W.z, W.w};
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const bool use = (w[u] > 0.f) && (!SKIP_SELF || j[u] != self);
    c[u] = use ? __ldg(lab + j[u]) : -1;
  }
  return make_int4(c[0], c[1], c[2], c[3]);
}

// Fold positions [b, e) of the CSR, in order, into st: st.add(C[j], w) for every kept
// position.  Software pipeline: the index/weight group two ahead is loaded and the label
// group one ahead is gathered before the current group is folded, so each lane keeps
// eight loads and four gathers in flight while it works.
template <class S, bool WT, bool SKIP_SELF>
__device__ __forceinline__ void fold_range(S& st, const int32_t* __restrict__ idx,
                                           const float* __restrict__ wts,
                                           const int32_t* __restrict__ lab, int64_t m,
                                           int self, int64_t b, int64_t e) {
  if (b >= e) return;
  int64_t g = b & ~(int64_t)3;
  int4 J0, J1 = make_int4(self, self, self, self);
  float4 W0, W1 = make_float4(0.f, 0.f, 0.f, 0.f);
  load_group<WT>(idx, wts, m, g, b, e, self, J0, W0);
  int4 C0 = gather_group<SKIP_SELF>(lab, J0, W0, self);
  if (g + 4 < e) load_group<WT>(idx, wts, m, g + 4, b, e, self, J1, W1);
  for (; g < e; g += 4) {
    int4 C1 = make_int4(-1, -1, -1, -1);
    if (g + 4 < e) C1 = gather_group<SKIP_SELF>(lab, J1, W1, self);
    int4 J2 = make_int4(self, self, self, self);
    float4 W2 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g + 8 < e) load_group<WT>(idx, wts, m, g + 8, b, e, self, J2, W2);
    if (C0.x >= 0) st.add(C0.x, W0.x);
    if (C0.y >= 0) st.add(C0.y, W0.y);
    if (C0.z >= 0) st.add(C0.z, W0.z);
    if (C0.w >= 0) st.add(C0.w, W0.w);
    C0 = C1;
    W0 = W1;
    J1 = J2;
    W1 = W2;
  }
}

// ------------------------------------------------------------ work decomposition

// Kernel work map over a binned graph: CTAs [0, nhubs) take one hub each; then
// mid_ctas CTAs whose warps take 32/L vertices of one mid class (L lanes per vertex,
// one leaf per lane); then low_ctas CTAs whose warps take 32 degree-sorted low rows of
// one window (one row per lane).
struct Work {
  int kind;    // 0 hub, 1 mid, 2 low, -1 none
  int v;       // vertex (or -1 for an idle lane)
  int leaf;    // leaf index of this lane (mid), 0 otherwise
  int L;       // leaves of the vertex (mid: the class's L; low: 1)
};

__device__ __forceinline__ Work lane_work(const WarpPlan& p, int cta, int warp, int lane) {
  Work w{-1, -1, 0, 1};
  if (cta < p.nhubs) {
    w.kind = 0;
    w.v = p.cls_list[p.cls_start[kHubClass] + cta];
    return w;
  }
  cta -= p.nhubs;
  if (cta < p.mid_ctas) {
    w.kind = 1;
    const int gw = cta * (kThreads / 32) + warp;
    if (gw >= p.cls_warp_start[kMidClasses]) return w;
    int c = 0;
    while (gw >= p.cls_warp_start[c + 1]) ++c;
    const int L = 32 >> (c / kMidSub);
    w.L = L;
    const int64_t slot = (int64_t)(gw - p.cls_warp_start[c]) * (32 / L) + lane / L;
    const int64_t cnt = p.cls_start[c + 1] - p.cls_start[c];
    w.leaf = lane % L;
    if (slot < cnt) w.v = p.cls_list[p.cls_start[c] + slot];
    return w;
  }
  cta -= p.mid_ctas;
  w.kind = 2;
  const int lw = cta * (kThreads / 32) + warp;
  const int win = lw / (kWinVerts / 32);
  if (win >= p.nwin) return w;
  const int pos = (lw % (kWinVerts / 32)) * 32 + lane;
  if (pos < p.cnt_low[win]) w.v = p.perm_low[(int64_t)win * kWinVerts + pos];
  return w;
}

}  // namespace lpa
