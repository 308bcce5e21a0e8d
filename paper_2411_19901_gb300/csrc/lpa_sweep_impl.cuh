// lpa_sweep_impl.cuh -- the label-choice sweep of the sketch modes (the move step of
// Alg. 1 / Alg. 3) as one warp-per-row kernel over the binned graph.
//
// One launch sweeps every vertex once: C_next[i] = choice(C_prev) (synchronous), with
// the pick-less commit rule (Sec. 4.5), and adds the changed-label count to dN.
//  * low rows (one leaf): each lane folds one whole row; the warp's 32 rows have (near)
//    equal degree because binning sorted each window's rows by degree, so lanes stay in
//    step and no CTA barrier waits on a straggler;
//  * mid rows (2..32 leaves): each lane folds one leaf; the L lanes of a vertex merge by
//    the stride-doubling tree with warp shuffles (Sec. 4.3, partial sketches merged);
//    mid and low vertices are packed lane by lane, so one warp may hold several L;
//  * hubs (longer rows, or more than 32 leaves): one CTA, one leaf per thread, shuffles
//    within warps, shared memory across warps (a kernel of their own, so the lane kernel
//    runs CTAs of single warps that retire independently).
// Every lane reads its leaf from the plan's sliced copy of the CSR with the pipelined fold
// of lpa_fold.cuh (16-byte index and weight loads two groups ahead, the lanes of a warp
// side by side; label gathers one group ahead).  The tree depends only on the row length,
// so results never depend on which of these paths a vertex takes.
#pragma once

#include "lpa_fold.cuh"

namespace lpa {

__device__ __forceinline__ int commit_label(int c, int old, int pick_less) {
  return (c >= 0 && c != old && (!pick_less || c < old)) ? c : old;
}

// Levels s >= 32 of the stride-doubling tree for a hub with L > 32 leaves: warp leaders
// deposit their sketches; the merges of one level are independent, so thread t of warp 0
// merges the pair starting at warp 2·s·t, level by level; thread 0 ends with S[0].
template <class S>
__device__ __forceinline__ void cross_warp_tree(S& st, int L, int tid, int* sk, float* sv) {
  const int nw = L / 32;
  if ((tid & 31) == 0 && (tid >> 5) < nw)
    st.store(sk + (tid >> 5) * S::kSlots, sv + (tid >> 5) * S::kSlots);
  __syncthreads();
  if (tid < 32) {
    for (int s = 1; s < nw; s <<= 1) {
      const int w = tid * 2 * s;
      if (w + s < nw) {
        S a;
        a.load(sk + w * S::kSlots, sv + w * S::kSlots);
        a.merge_from(sk + (w + s) * S::kSlots, sv + (w + s) * S::kSlots);
        a.store(sk + w * S::kSlots, sv + w * S::kSlots);
      }
      __syncwarp();
    }
    if (tid == 0) st.load(sk, sv);
  }
}

// Hub sweep: CTA c sweeps hub c, one leaf per thread, leaves merged by shuffles within
// warps and through shared memory across warps.  Launched per hub class with CTAs of
// max(32, L) threads, so every warp of a CTA holds leaves.
template <class S, int WF, bool RESCAN = false>
__global__ void __launch_bounds__(kThreads) sweep_hub_kernel(SweepArgs a, WarpPlan p) {
  constexpr bool WT = WF != kUnitW;
  if (a.done != nullptr && *a.done) return;
  __shared__ int sk[(kThreads / 32) * 32];
  __shared__ float sv[(kThreads / 32) * 32];
  const int tid = threadIdx.x, lane = tid & 31;
  const int4 h = __ldg(p.hub_desc + blockIdx.x);
  const int v = h.x;
  const int64_t base = (int64_t)(uint32_t)h.y | ((int64_t)h.z << 32);
  const int64_t d = h.w;
  const int L = leaf_count(d, a.e0, a.lmax);
  if ((a.act_in != nullptr && !a.act_in[v]) || (a.gid != nullptr && a.gdone[a.gid[v]])) {
    if (tid == 0) a.c_next[v] = a.c_prev[v];  // not swept: keep the label
    return;
  }
  const int own = a.c_prev[v];
  S st;
  st.init(own);
  if (tid < L) {
    const int64_t lo = base + (tid * d) / L, len = base + ((tid + 1) * d) / L - lo;
    const int W = L < 32 ? L : 32;
    const int64_t G = hub_leaf_groups(d, L);
    HubSliceAddr ad{p.hub_base[blockIdx.x] + (int64_t)(tid >> 5) * W * G + (tid & 31), W};
    const int ng = (int)((len + 3) >> 2);
    fold_groups<S, WF, false>(st, p, a.c_prev, -1, ng, ng, ad);
  }
  const int Lw = L < 32 ? L : 32;
  for (int s = 1; s < Lw; s <<= 1) st.shfl_merge(s, tid < L && (lane & (2 * s - 1)) == 0);
  if (L > 32) cross_warp_tree<S>(st, L, tid, sk, sv);
  int choice = -1;
  if constexpr (RESCAN) {
    // double scan: thread 0's candidates to every thread, per-leaf sums, the same tree
    constexpr int K = S::kSlots;
    if (tid == 0)
#pragma unroll
      for (int q = 0; q < K; ++q) sk[q] = st.val[q] > 0.f ? st.key[q] : -1;
    __syncthreads();
    int ck[K];
    float part[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      ck[q] = sk[q];
      part[q] = 0.f;
    }
    __syncthreads();
    if (tid < L)
      rescan_range<K, WT>(part, ck, a.idx, a.w, a.c_prev, v, base + (tid * d) / L,
                          base + ((tid + 1) * d) / L);
    for (int s = 1; s < Lw; s <<= 1)
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const float y = __shfl_down_sync(kFullMask, part[q], s);
        if (tid < L && (lane & (2 * s - 1)) == 0) part[q] = part[q] + y;
      }
    if (L > 32) {
      const int nw = L / 32;
      if (lane == 0 && (tid >> 5) < nw)
#pragma unroll
        for (int q = 0; q < K; ++q) sv[(tid >> 5) * K + q] = part[q];
      __syncthreads();
      if (tid == 0) {
        for (int s = 1; s < nw; s <<= 1)
          for (int w = 0; w + s < nw; w += 2 * s)
            for (int q = 0; q < K; ++q) sv[w * K + q] = sv[w * K + q] + sv[(w + s) * K + q];
#pragma unroll
        for (int q = 0; q < K; ++q) part[q] = sv[q];
      }
    }
    if (tid == 0) choice = rescan_pick<K>(part, ck);
  } else {
    if (tid == 0) choice = st.choose();
  }
  __shared__ int s_changed;
  if (tid == 0) {
    const int nl = commit_label(choice, own, a.gpl != nullptr ? a.gpl[a.gid[v]] : a.pick_less);
    a.c_next[v] = nl;
    s_changed = nl != own;
    if (nl != own) atomicAdd(a.dn + (blockIdx.x & (kDnSlots - 1)), 1ull);
    if (nl != own && a.gdn != nullptr) atomicAdd(a.gdn + a.gid[v], 1u);
    if (a.scanned) atomicAdd(a.scanned + (blockIdx.x & (kDnSlots - 1)), (unsigned long long)d);
  }
  if (a.act_out != nullptr) {  // a moved vertex marks its neighbours unprocessed
    __syncthreads();
    if (s_changed)
      for (int64_t q = base + tid; q < base + d; q += blockDim.x) a.act_out[__ldg(a.idx + q)] = 1;
  }
}

// Lane sweep: thread q of the grid takes lane descriptor q (a low row, or one leaf of a
// mid vertex whose L lanes are aligned inside the warp).  Lanes of one warp may belong to
// vertices of different L: every lane runs the warp's largest L, merging only below its
// own.  Warps are independent, so a CTA of kLaneThreads holds as few of them as possible.
// CTAs of 128 lane threads an SM should hold for sketch S: 7 (72 registers a thread) fits
// the sketches up to k = 8; the 16- and 32-slot sketches need more registers than that
// (they would spill), so fewer CTAs.
template <class S>
constexpr int lane_min_blocks() {
  return S::kSlots >= 32 ? 3 : (S::kSlots >= 16 ? 5 : 7);
}

template <class S, int WF, bool RESCAN = false, int TPB = kLaneThreads>
__global__ void __launch_bounds__(TPB, lane_min_blocks<S>() * 128 / TPB)
    sweep_lane_kernel(SweepArgs a, WarpPlan p) {
  constexpr bool WT = WF != kUnitW;
  if (a.done != nullptr && *a.done) return;
  const int64_t q = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int v = -1, leaf = 0, L = 1;
  int64_t lo = 0, len = 0;
  if (q < p.nlanes) {
    const int4 l = __ldg(p.lane_desc + q);
    v = l.x;
    lo = (int64_t)(uint32_t)l.y | ((int64_t)l.z << 32);
    len = l.w & ((1 << kLaneLeafShift) - 1);
    leaf = (l.w >> kLaneLeafShift) & 31;
    L = 1 << (l.w >> kLaneLgShift);
  }
  const int g = (v >= 0 && a.gid != nullptr) ? a.gid[v] : -1;
  const bool act = v >= 0 && (a.act_in == nullptr || a.act_in[v] != 0) &&
                   (g < 0 || !a.gdone[g]);
  S st;
  int own = -1;
  if (v >= 0) {
    own = a.c_prev[v];
    st.init(own);
  } else {
    st.init(-1);
  }
  // the leaf from the sliced copy: every lane of the warp runs the warp's longest leaf's
  // steps (the slice places are decided by warp votes)
  const int ngl = (int)((len + 3) >> 2);
  LaneSliceAddr ad{q < p.nlanes ? p.lane_base[q >> 5] : 0, ngl, (1u << lane) - 1u};
  fold_groups<S, WF, false>(st, p, a.c_prev, -1, act ? ngl : 0,
                            __reduce_max_sync(kFullMask, ngl), ad);
  const int Lw = __reduce_max_sync(kFullMask, L);
  for (int s = 1; s < Lw; s <<= 1) st.shfl_merge(s, v >= 0 && s < L && (leaf & (2 * s - 1)) == 0);
  int choice = -1;
  if constexpr (RESCAN) {
    // double scan: the leader's candidates to the vertex's lanes, per-leaf sums of
    // their exact weights, summed along the same stride-doubling tree
    constexpr int K = S::kSlots;
    int ck[K];
    float part[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      ck[q] = __shfl_sync(kFullMask, st.val[q] > 0.f ? st.key[q] : -1, lane - leaf);
      part[q] = 0.f;
    }
    if (act) rescan_range<K, WT>(part, ck, a.idx, a.w, a.c_prev, v, lo, lo + len);
    for (int s = 1; s < Lw; s <<= 1)
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const float y = __shfl_down_sync(kFullMask, part[q], s);
        if (v >= 0 && s < L && (leaf & (2 * s - 1)) == 0) part[q] = part[q] + y;
      }
    choice = rescan_pick<K>(part, ck);
  } else {
    choice = st.choose();
  }
  int changed = 0;
  if (v >= 0 && leaf == 0) {
    const int nl = commit_label(choice, own, a.gpl != nullptr ? a.gpl[g] : a.pick_less);
    a.c_next[v] = nl;
    changed = nl != own;
  }
  const int wsum = __reduce_add_sync(kFullMask, changed);
  if (lane == 0 && wsum > 0)
    atomicAdd(a.dn + ((q >> 5) & (kDnSlots - 1)), (unsigned long long)wsum);
  if (a.gdn != nullptr && wsum > 0) {  // batched: one atomic per graph present in the warp
    const unsigned same = __match_any_sync(kFullMask, changed ? g : -1 - lane);
    if (changed && lane == __ffs(same) - 1) atomicAdd(a.gdn + g, (unsigned)__popc(same));
  }
  if (a.act_out != nullptr) {
    // the vertex's leader knows whether it moved; each of its lanes marks its own leaf
    const int moved = __shfl_sync(kFullMask, changed, lane - leaf);
    if (v >= 0 && moved)
      for (int64_t p2 = lo; p2 < lo + len; ++p2) a.act_out[__ldg(a.idx + p2)] = 1;
    const unsigned sc = __reduce_add_sync(kFullMask, act ? (unsigned)len : 0u);
    if (lane == 0 && sc > 0) atomicAdd(a.scanned + ((q >> 5) & (kDnSlots - 1)), (unsigned long long)sc);
  }
}

// One sweep: the hub kernel on s_hub and the lane kernel on s (the caller orders the two
// streams; they may be the same stream).  Both write disjoint entries of c_next and add to
// the same dN counters.
template <class S, int WF, bool RESCAN = false, bool SIZES = false>
cudaError_t launch_warp_kernel(const SweepArgs& a, const WarpPlan& p, cudaStream_t s,
                               cudaStream_t s_hub) {
  for (int c = 0; c < kHubClasses; ++c) {  // one launch per hub class, CTAs of 256 >> c
    const int cnt = p.hub_start[c + 1] - p.hub_start[c];
    if (cnt <= 0) continue;
    WarpPlan q = p;
    q.hub_desc = p.hub_desc + p.hub_start[c];
    q.hub_base = p.hub_base + p.hub_start[c];
    sweep_hub_kernel<S, WF, RESCAN><<<(unsigned)cnt, kThreads >> c, 0, s_hub>>>(a, q);
    count_launch();
  }
  // lane CTAs of the tuned size (built for the sketches that take every tuning)
  const int tpb = SIZES ? p.lane_threads : kLaneThreads;
  const int64_t lane_ctas = (p.nlanes + tpb - 1) / tpb;
  if (lane_ctas > 0) {
    if constexpr (SIZES) {
      if (tpb == 64)
        sweep_lane_kernel<S, WF, RESCAN, 64><<<(unsigned)lane_ctas, 64, 0, s>>>(a, p);
      else if (tpb == 256)
        sweep_lane_kernel<S, WF, RESCAN, 256><<<(unsigned)lane_ctas, 256, 0, s>>>(a, p);
      else
        sweep_lane_kernel<S, WF, RESCAN><<<(unsigned)lane_ctas, kLaneThreads, 0, s>>>(a, p);
    } else {
      sweep_lane_kernel<S, WF, RESCAN><<<(unsigned)lane_ctas, kLaneThreads, 0, s>>>(a, p);
    }
    count_launch();
  }
  return cudaGetLastError();
}

// The instantiations of one sketch type: unit or fp32 weights; for the sketches that
// full_tuning_sketch names (FULL) every lane CTA size.
template <class S, bool FULL = false>
cudaError_t launch_warp_variants(const SweepArgs& a, const WarpPlan& p, cudaStream_t s,
                                 cudaStream_t s_hub) {
  return p.wfmt == kSplitW ? launch_warp_kernel<S, kSplitW, false, FULL>(a, p, s, s_hub)
                           : launch_warp_kernel<S, kUnitW, false, FULL>(a, p, s, s_hub);
}

// The MG ablation variants of one k: paper-literal accumulate and / or double scan.
template <int K>
cudaError_t launch_mg_variant(bool literal, bool rescan, const SweepArgs& a, const WarpPlan& p,
                              cudaStream_t s, cudaStream_t s_hub) {
  const bool weighted = p.wfmt == kSplitW;
  if (literal) {
    if (rescan)
      return weighted ? launch_warp_kernel<MGLiteral<K>, kSplitW, true>(a, p, s, s_hub)
                      : launch_warp_kernel<MGLiteral<K>, kUnitW, true>(a, p, s, s_hub);
    return weighted ? launch_warp_kernel<MGLiteral<K>, kSplitW, false>(a, p, s, s_hub)
                    : launch_warp_kernel<MGLiteral<K>, kUnitW, false>(a, p, s, s_hub);
  }
  return weighted ? launch_warp_kernel<MGSketch<K>, kSplitW, true>(a, p, s, s_hub)
                  : launch_warp_kernel<MGSketch<K>, kUnitW, true>(a, p, s, s_hub);
}

}  // namespace lpa
