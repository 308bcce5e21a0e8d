// lpa_fold.cuh -- device building blocks of the sweep: the register sketches (weighted
// Misra-Gries as the paper uses it and as printed, weighted Boyer-Moore), the double-scan
// helpers and the pipelined row fold.
#pragma once

#include "lpa_internal.cuh"

namespace lpa {

constexpr unsigned kFullMask = 0xffffffffu;

// ---------------------------------------------------------------- MG sketch

// k-slot weighted Misra-Gries sketch held in registers (Sec. 4.1, Alg. 2).  Empty slots
// hold key -1 and value 0; labels are >= 0, so a key only matches an occupied slot.  em
// is the bitmask of empty slots, kept up to date so the insert path needs no scan.
template <int K>
struct MGSketch {
  int key[K];
  float val[K];
  unsigned em;
  static constexpr int kSlots = K;

  __device__ __forceinline__ void init(int /*own*/) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      key[s] = -1;
      val[s] = 0.f;
    }
    em = (K == 32) ? 0xffffffffu : ((1u << K) - 1u);
  }

  // (c, w) into the lowest free slot; em must be non-zero.  The slot is chosen by testing
  // bits of the one-hot lowest free bit, not by comparing slot numbers: fewer
  // instructions on the integer ALU pipe, which bounds the sweep.
  __device__ __forceinline__ void place(int c, float w) {
    const unsigned oh = em & (0u - em);
    em ^= oh;
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (oh & (1u << s)) {
        key[s] = c;
        val[s] = w;
      }
  }

  // sketchAccumulate with the clamped decrement: add to a matching slot, else fill the
  // lowest free slot, else lower every slot and w by min(w, smallest slot) and put a
  // positive remainder in the lowest slot that became free.  One insert site serves
  // both the free-slot and the after-decrement case, so diverged lanes share it.
  __device__ __forceinline__ void add(int c, float w) {
    bool hit = false;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const bool m = (key[s] == c);
      if (m) val[s] = val[s] + w;
      hit = hit || m;
    }
    if (hit) return;
    if (em == 0u) {
      float lo[K];
#pragma unroll
      for (int s = 0; s < K; ++s) lo[s] = val[s];
#pragma unroll
      for (int h = K / 2; h >= 1; h /= 2)
#pragma unroll
        for (int s = 0; s < h; ++s) lo[s] = fminf(lo[s], lo[s + h]);
      const float delta = fminf(w, lo[0]);
      // slots that drop to zero become empty; the mask is built with predicated adds,
      // which the compiler can put on the FMA pipe instead of the integer ALU pipe
      unsigned z = 0;
#pragma unroll
      for (int s = 0; s < K; ++s) {
        val[s] = val[s] - delta;
        if (val[s] == 0.f) {
          key[s] = -1;
          z = z + (1u << s);
        }
      }
      em = z;
      w = w - delta;
    }
    if (w > 0.f) place(c, w);
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
    em = 0;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      key[s] = k[s];
      val[s] = v[s];
      em |= (v[s] == 0.f ? 1u : 0u) << s;
    }
  }
};

// ------------------------------------------------------ paper-literal MG sketch

// sketchAccumulate as printed in Alg. 2 for a private sketch (the LPA_MG_UNCLAMPED
// ablation): a slot whose key equals c takes += w whatever its value; otherwise the
// lowest slot of value exactly 0 takes (c, w); otherwise every slot loses w and c is
// dropped.  Values may go negative; merges feed every slot of non-zero value; the
// choice is the largest positive value.
template <int K>
struct MGLiteral {
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
  __device__ __forceinline__ void add(int c, float w) {
    bool hit = false;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const bool m = (key[s] == c);
      if (m) val[s] = val[s] + w;
      hit = hit || m;
    }
    if (hit) return;
    unsigned em = 0;
#pragma unroll
    for (int s = 0; s < K; ++s) em |= (val[s] == 0.f ? 1u : 0u) << s;
    if (em != 0u) {
      const unsigned oh = em & (0u - em);  // the lowest slot of value 0, one-hot
#pragma unroll
      for (int s = 0; s < K; ++s)
        if (oh & (1u << s)) {
          key[s] = c;
          val[s] = w;
        }
    } else {
#pragma unroll
      for (int s = 0; s < K; ++s) val[s] = val[s] - w;
    }
  }
  __device__ __forceinline__ void merge_from(const int* bk, const float* bv) {
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (bv[s] != 0.f) add(bk[s], bv[s]);
  }
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

// ------------------------------------------------------------- double scan

// Second scan of Sec. 4.4 over one leaf: part[s] += w for every valid position whose
// neighbour label equals candidate ck[s] (ck[s] = -1: no candidate), in CSR order.
template <int K, bool WT>
__device__ __forceinline__ void rescan_range(float (&part)[K], const int (&ck)[K],
                                             const int32_t* __restrict__ idx,
                                             const float* __restrict__ wts,
                                             const int32_t* __restrict__ lab, int self,
                                             int64_t b, int64_t e) {
  for (int64_t p = b; p < e; ++p) {
    const int j = __ldg(idx + p);
    const float w = WT ? __ldg(wts + p) : 1.f;
    if (j == self || !(w > 0.f)) continue;
    const int c = __ldg(lab + j);
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (ck[s] == c) part[s] = part[s] + w;
  }
}

// The candidate of largest summed weight, ties to the smallest label; -1 if none.
template <int K>
__device__ __forceinline__ int rescan_pick(const float (&part)[K], const int (&ck)[K]) {
  int best = -1;
  float bk = 0.f;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    if (ck[s] < 0) continue;
    if (best < 0 || part[s] > bk || (part[s] == bk && ck[s] < best)) {
      best = ck[s];
      bk = part[s];
    }
  }
  return best;
}

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

// Load the aligned group of four CSR positions starting at g (a multiple of 4).  A group
// that would cross the end of the arrays is read element-wise; positions past the end
// come back as (self, 0).  Which positions belong to the range is decided by the caller.
template <bool WT>
__device__ __forceinline__ void load_group(const int32_t* __restrict__ idx,
                                           const float* __restrict__ wts, int64_t m, int64_t g,
                                           int self, int4& J, float4& W) {
  if (g + 3 < m) {
    J = __ldg(reinterpret_cast<const int4*>(idx + g));
    W = WT ? __ldg(reinterpret_cast<const float4*>(wts + g)) : make_float4(1.f, 1.f, 1.f, 1.f);
  } else {
    int j[4];
    float w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      j[u] = (g + u < m) ? __ldg(idx + g + u) : self;
      w[u] = (g + u < m) ? (WT ? __ldg(wts + g + u) : 1.f) : 0.f;
    }
    J = make_int4(j[0], j[1], j[2], j[3]);
    W = make_float4(w[0], w[1], w[2], w[3]);
  }
}

// 4-bit mask of the group's positions that lie in [b, e)
__device__ __forceinline__ unsigned group_mask(int64_t g, int64_t b, int64_t e) {
  const int64_t lo = b - g;  // > 0 only for the first group
  const int64_t hi = e - g;  // < 4 only for the last group
  unsigned mk = 0xFu;
  if (lo > 0) mk &= (0xFu << lo) & 0xFu;
  if (hi < 4) mk &= 0xFu >> (4 - hi);
  return mk;
}

// Neighbour labels of a group: -1 where the position is skipped (outside the range, a
// self-loop when SKIP_SELF, or a weight that is not positive).
template <bool SKIP_SELF>
__device__ __forceinline__ int4 gather_group(const int32_t* __restrict__ lab, const int4& J,
                                             const float4& W, unsigned mk, int self) {
  int c[4];
  const int j[4] = {J.x, J.y, J.z, J.w};
  const float w[4] = {W.x, W.y, W.z, W.w};
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const bool use = ((mk >> u) & 1u) && (w[u] > 0.f) && (!SKIP_SELF || j[u] != self);
    c[u] = use ? __ldg(lab + j[u]) : -1;
  }
  return make_int4(c[0], c[1], c[2], c[3]);
}

// Fold positions [b, e) of the CSR, in order, into st: st.add(C[j], w) for every kept
// position.  The range is read as aligned groups of four (16-byte index and weight
// loads); only the first and last group carry a mask.  Software pipeline with three
// register sets rotated by unrolling (no moves of registers with loads in flight): while
// group k is folded, the labels of group k+1 are being gathered and group k+2 is being
// loaded.
template <class S, bool WT, bool SKIP_SELF>
__device__ __forceinline__ void fold_range(S& st, const int32_t* __restrict__ idx,
                                           const float* __restrict__ wts,
                                           const int32_t* __restrict__ lab, int64_t m,
                                           int self, int64_t b, int64_t e) {
  if (b >= e) return;
  const int64_t g0 = b & ~(int64_t)3;
  const int ng = (int)((e - g0 + 3) >> 2);
  const unsigned first = (0xFu << (int)(b - g0)) & 0xFu;
  const unsigned lastm = 0xFu >> (int)(g0 + 4 * (int64_t)ng - e);
  const bool tail_unsafe = g0 + 4 * (int64_t)ng > m;  // last group crosses the array end
  const int4* __restrict__ ip = reinterpret_cast<const int4*>(idx + g0);
  const float4* __restrict__ wp = reinterpret_cast<const float4*>(wts + g0);

  auto load = [&](int k, int4& X, float4& W) {
    if (tail_unsafe && k == ng - 1) {
      load_group<WT>(idx, wts, m, g0 + 4 * (int64_t)k, self, X, W);
    } else {
      X = __ldg(ip + k);
      W = WT ? __ldg(wp + k) : make_float4(1.f, 1.f, 1.f, 1.f);
    }
  };
  auto gather = [&](int k, int4& X, const float4& W) {
    unsigned mk = 0xFu;
    if (k == 0) mk &= first;
    if (k == ng - 1) mk &= lastm;
    X = gather_group<SKIP_SELF>(lab, X, W, mk, self);
  };
  // one push site per step: the group's four pairs are shifted through lane x (its
  // registers hold finished gathers, so the moves wait on nothing), which keeps the
  // loop body, and the sketch code inlined into it, small for the instruction cache
  auto fold = [&](int4 C, float4 W) {
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
      if (C.x >= 0) st.add(C.x, W.x);
      C = make_int4(C.y, C.z, C.w, -1);
      W = make_float4(W.y, W.z, W.w, 0.f);
    }
  };
  int4 X0, X1 = make_int4(self, self, self, self), X2 = make_int4(self, self, self, self);
  float4 W0, W1 = make_float4(0.f, 0.f, 0.f, 0.f), W2 = make_float4(0.f, 0.f, 0.f, 0.f);
  load(0, X0, W0);
  gather(0, X0, W0);
  if (ng > 1) load(1, X1, W1);
  // step k: F = group k (gathered), G = group k+1 (loaded), L = free
#define LPA_STEP(XF, WF, XG, WG, XL, WL)   \
  if (k + 1 < ng) gather(k + 1, XG, WG);   \
  if (k + 2 < ng) load(k + 2, XL, WL);     \
  fold(XF, WF);                            \
  if (++k >= ng) break;
  for (int k = 0;;) {
    LPA_STEP(X0, W0, X1, W1, X2, W2)
    LPA_STEP(X1, W1, X2, W2, X0, W0)
    LPA_STEP(X2, W2, X0, W0, X1, W1)
  }
#undef LPA_STEP
}

// ---------------------------------------------------------------- sliced fold

// Where a lane's groups sit in its warp's slice (see WarpPlan): column k holds group k of
// every lane that has one, in lane order.  at(k) takes a warp vote, so every lane of the
// warp calls it for k = 0, 1, 2, ... in turn.
struct LaneSliceAddr {
  int64_t col;      // first element of the next column
  int groups;       // this lane's groups in the slice
  unsigned below;   // mask of the lanes below this one
  __device__ __forceinline__ int64_t at(int k) {
    const unsigned has = __ballot_sync(kFullMask, groups > k);
    const int64_t p = col + __popc(has & below);
    col += __popc(has);
    return p;
  }
};

// Where a hub leaf's groups sit: a fixed stride from its first one.
struct HubSliceAddr {
  int64_t first;
  int stride;
  __device__ __forceinline__ int64_t at(int k) const { return first + (int64_t)k * stride; }
};

// Neighbour labels of a group of the sliced copy: index -1 marks a position no vote
// comes from (a self-loop, a weight that is not positive, padding past the leaf's end).
// With SELF_LOOPS such a position of positive weight -- a self-loop -- counts under the
// vertex's own label (modularity: C_i = C_i), else it is skipped (-1).
template <bool SELF_LOOPS>
__device__ __forceinline__ int4 gather_slice(const int32_t* __restrict__ lab, const int4& J,
                                             const float4& W, int own) {
  int c[4];
  const int j[4] = {J.x, J.y, J.z, J.w};
  const float w[4] = {W.x, W.y, W.z, W.w};
#pragma unroll
  for (int u = 0; u < 4; ++u)
    c[u] = j[u] >= 0 ? __ldg(lab + j[u]) : (SELF_LOOPS && w[u] > 0.f ? own : -1);
  return make_int4(c[0], c[1], c[2], c[3]);
}

// Fold the positions of one leaf, in CSR order, from the sliced copy into st:
// st.add(C[j], w) for every position a vote comes from (the rule of fold_range; the
// sliced copy marks the others).  The leaf has ng groups (0: nothing to fold); the loop
// takes `iters` >= ng steps, the same on every lane when addr votes, and steps past ng
// only keep the vote going.  Same three-set pipeline as fold_range: while group k is
// folded, the labels of group k+1 are gathered and group k+2 is loaded; the loads of a
// warp's lanes are side by side in memory.
template <class S, int WF, bool SELF_LOOPS, class A>
__device__ __forceinline__ void fold_groups(S& st, const WarpPlan& pl,
                                            const int32_t* __restrict__ lab, int own, int ng,
                                            int iters, A& addr) {
  if (iters <= 0) return;
  const int4* __restrict__ si = pl.sl_idx;
  const float4* __restrict__ sw = pl.sl_w;
  // the sliced copy is read once per sweep, a warp's loads covering whole lines: mark it
  // first to leave L2 so that more of the gathered label array stays cached
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  auto stream = [&](const int4* q) {
    int4 r;
    asm("ld.global.nc.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(q), "l"(pol));
    return r;
  };
  auto load = [&](int k, int4& X, float4& W) {
    const int64_t p = addr.at(k);
    if (k < ng) {
      X = stream(si + p);
      if (WF == kSplitW) {
        const int4 t = stream(reinterpret_cast<const int4*>(sw + p));
        W = make_float4(__int_as_float(t.x), __int_as_float(t.y), __int_as_float(t.z),
                        __int_as_float(t.w));
      } else {
        W = make_float4(1.f, 1.f, 1.f, 1.f);
      }
    } else {
      X = make_int4(-1, -1, -1, -1);
      W = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto gather = [&](int4& X, const float4& W) { X = gather_slice<SELF_LOOPS>(lab, X, W, own); };
  // the four pushes of a group inlined (no register moves between them: measured faster
  // than one push site in a loop for the sliced layout)
  auto fold = [&](const int4& C, const float4& W) {
    if (C.x >= 0) st.add(C.x, W.x);
    if (C.y >= 0) st.add(C.y, W.y);
    if (C.z >= 0) st.add(C.z, W.z);
    if (C.w >= 0) st.add(C.w, W.w);
  };
  int4 X0, X1 = make_int4(-1, -1, -1, -1), X2 = make_int4(-1, -1, -1, -1);
  float4 W0, W1 = make_float4(0.f, 0.f, 0.f, 0.f), W2 = make_float4(0.f, 0.f, 0.f, 0.f);
  load(0, X0, W0);
  gather(X0, W0);
  if (iters > 1) load(1, X1, W1);
#define LPA_STEP(XF, WF_, XG, WG, XL, WL)  \
  if (k + 1 < iters) gather(XG, WG);       \
  if (k + 2 < iters) load(k + 2, XL, WL);  \
  fold(XF, WF_);                           \
  if (++k >= iters) break;
  for (int k = 0;;) {
    LPA_STEP(X0, W0, X1, W1, X2, W2)
    LPA_STEP(X1, W1, X2, W2, X0, W0)
    LPA_STEP(X2, W2, X0, W0, X1, W1)
  }
#undef LPA_STEP
}

}  // namespace lpa
