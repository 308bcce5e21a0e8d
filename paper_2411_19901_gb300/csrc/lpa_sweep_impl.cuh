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

template <class S, bool WT>
__global__ void __launch_bounds__(kThreads) sweep_warp_kernel(SweepArgs a, WarpPlan p) {
  if (a.done != nullptr && *a.done) return;
  __shared__ int sk[(kThreads / 32) * 32];
  __shared__ float sv[(kThreads / 32) * 32];
  const int tid = threadIdx.x, lane = tid & 31;
  const Work wk = lane_work(p, (int)blockIdx.x, tid >> 5, lane);
  int changed = 0;
  if (wk.kind == 0) {  // hub: the whole CTA
    const int v = wk.v;
    const int64_t base = a.off[v];
    const int64_t d = a.off[v + 1] - base;
    const int L = leaf_count(d, a.e0, a.lmax);
    const int own = a.c_prev[v];
    S st;
    st.init(own);
    if (tid < L)
      fold_range<S, WT, true>(st, a.idx, a.w, a.c_prev, a.m, v, base + (tid * d) / L,
                              base + ((tid + 1) * d) / L);
    const int Lw = L < 32 ? L : 32;
    for (int s = 1; s < Lw; s <<= 1) st.shfl_merge(s, tid < L && (lane & (2 * s - 1)) == 0);
    if (L > 32) cross_warp_tree<S>(st, L, tid, sk, sv);
    if (tid == 0) {
      const int nl = commit_label(st.choose(), own, a.pick_less);
      a.c_next[v] = nl;
      changed = nl != own;
    }
  } else if (wk.kind > 0) {  // mid leaf group or low row: one lane per leaf
    S st;
    int own = -1;
    if (wk.v >= 0) {
      own = a.c_prev[wk.v];
      st.init(own);
      const int64_t base = a.off[wk.v];
      const int64_t d = a.off[wk.v + 1] - base;
      fold_range<S, WT, true>(st, a.idx, a.w, a.c_prev, a.m, wk.v, base + (wk.leaf * d) / wk.L,
                              base + ((wk.leaf + 1) * d) / wk.L);
    } else {
      st.init(-1);
    }
    for (int s = 1; s < wk.L; s <<= 1)
      st.shfl_merge(s, wk.v >= 0 && (wk.leaf & (2 * s - 1)) == 0);
    if (wk.v >= 0 && wk.leaf == 0) {
      const int nl = commit_label(st.choose(), own, a.pick_less);
      a.c_next[wk.v] = nl;
      changed = nl != own;
    }
  }
  const int cnt = __syncthreads_count(changed);
  if (tid == 0 && cnt > 0) atomicAdd(a.dn + (blockIdx.x & (kDnSlots - 1)), (unsigned long long)cnt);
}

inline unsigned sweep_grid(const WarpPlan& p) {
  return (unsigned)(p.nhubs + p.mid_ctas + p.low_ctas);
}

template <class S, bool WT>
cudaError_t launch_warp_kernel(const SweepArgs& a, const WarpPlan& p, cudaStream_t s) {
  const unsigned grid = sweep_grid(p);
  if (grid == 0) return cudaSuccess;
  sweep_warp_kernel<S, WT><<<grid, kThreads, 0, s>>>(a, p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lpa
