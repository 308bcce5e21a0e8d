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
//  * hubs (longer rows, or more than 32 leaves): one CTA, one leaf per thread, shuffles
//    within warps, shared memory across warps.
// Every lane reads its range with the pipelined fold of lpa_fold.cuh (16-byte index and
// weight loads two groups ahead, label gathers one group ahead).  The tree depends only
// on the row length, so results never depend on which of these paths a vertex takes.
#pragma once

#include "lpa_fold.cuh"

namespace lpa {

__device__ __forceinline__ int commit_label(int c, int old, int pick_less) {
  return (c >= 0 && c != old && (!pick_less || c < old)) ? c : old;
}

// Levels s >= 32 of the stride-doubling tree for a hub with L > 32 leaves: warp leaders
// deposit their sketches, thread 0 merges them level by level; thread 0 ends with S[0].
template <class S>
__device__ __forceinline__ void cross_warp_tree(S& st, int L, int tid, int* sk, float* sv) {
  const int nw = L / 32;
  if ((tid & 31) == 0 && (tid >> 5) < nw)
    st.store(sk + (tid >> 5) * S::kSlots, sv + (tid >> 5) * S::kSlots);
  __syncthreads();
  if (tid == 0) {
    for (int s = 1; s < nw; s <<= 1) {
      for (int w = 0; w + s < nw; w += 2 * s) {
        S a;
        a.load(sk + w * S::kSlots, sv + w * S::kSlots);
        a.merge_from(sk + (w + s) * S::kSlots, sv + (w + s) * S::kSlots);
        a.store(sk + w * S::kSlots, sv + w * S::kSlots);
      }
    }
    st.load(sk, sv);
  }
}

// RUNS folds runs of equal consecutive labels as one add (MG only; the caller enables it
// when every sum of a row's weights is exact in fp32, so the bits do not change).
template <class S, bool WT, bool RUNS>
__global__ void __launch_bounds__(kThreads) sweep_warp_kernel(SweepArgs a, WarpPlan p) {
  constexpr bool kRuns = RUNS && S::kRunMergeable;
  if (a.done != nullptr && *a.done) return;
  __shared__ int sk[(kThreads / 32) * 32];
  __shared__ float sv[(kThreads / 32) * 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int cta = (int)blockIdx.x;
  int changed = 0;
  if (cta < p.nhubs) {  // hub: the whole CTA, one leaf per thread
    const int v = p.cls_list[p.cls_start[kHubClass] + cta];
    const int64_t base = a.off[v];
    const int64_t d = a.off[v + 1] - base;
    const int L = leaf_count(d, a.e0, a.lmax);
    const int own = a.c_prev[v];
    S st;
    st.init(own);
    if (tid < L)
      fold_range<S, WT, true, kRuns>(st, a.idx, a.w, a.c_prev, a.m, v, base + (tid * d) / L,
                                     base + ((tid + 1) * d) / L);
    const int Lw = L < 32 ? L : 32;
    for (int s = 1; s < Lw; s <<= 1) st.shfl_merge(s, tid < L && (lane & (2 * s - 1)) == 0);
    if (L > 32) cross_warp_tree<S>(st, L, tid, sk, sv);
    if (tid == 0) {
      const int nl = commit_label(st.choose(), own, a.pick_less);
      a.c_next[v] = nl;
      changed = nl != own;
    }
  } else {  // mid leaf group or low row: one lane per leaf
    const Work wk = lane_work(p, a.off, cta, warp, lane);
    S st;
    int own = -1;
    if (wk.v >= 0) {
      own = a.c_prev[wk.v];
      st.init(own);
      fold_range<S, WT, true, kRuns>(st, a.idx, a.w, a.c_prev, a.m, wk.v,
                                     wk.b + (wk.leaf * wk.d) / wk.L,
                                     wk.b + ((wk.leaf + 1) * wk.d) / wk.L);
    } else {
      st.init(-1);
    }
    for (int s = 1; s < wk.L; s <<= 1) st.shfl_merge(s, wk.v >= 0 && (wk.leaf & (2 * s - 1)) == 0);
    if (wk.v >= 0 && wk.leaf == 0) {
      const int nl = commit_label(st.choose(), own, a.pick_less);
      a.c_next[wk.v] = nl;
      changed = nl != own;
    }
  }
  const int wsum = __reduce_add_sync(kFullMask, changed);
  if (lane == 0 && wsum > 0)
    atomicAdd(a.dn + ((blockIdx.x * (kThreads / 32) + warp) & (kDnSlots - 1)), (unsigned long long)wsum);
}

inline unsigned sweep_grid(const WarpPlan& p) {
  return (unsigned)(p.nhubs + p.mid_ctas + p.low_ctas);
}

template <class S, bool WT, bool RUNS>
cudaError_t launch_warp_kernel(const SweepArgs& a, const WarpPlan& p, cudaStream_t s) {
  const unsigned grid = sweep_grid(p);
  if (grid == 0) return cudaSuccess;
  sweep_warp_kernel<S, WT, RUNS><<<grid, kThreads, 0, s>>>(a, p);
  count_launch();
  return cudaGetLastError();
}

// The four instantiations of one sketch type: weighted or not, runs folded or not.
template <class S>
cudaError_t launch_warp_variants(bool weighted, bool runs, const SweepArgs& a, const WarpPlan& p,
                                 cudaStream_t s) {
  if (weighted)
    return runs ? launch_warp_kernel<S, true, true>(a, p, s) : launch_warp_kernel<S, true, false>(a, p, s);
  return runs ? launch_warp_kernel<S, false, true>(a, p, s) : launch_warp_kernel<S, false, false>(a, p, s);
}

}  // namespace lpa
