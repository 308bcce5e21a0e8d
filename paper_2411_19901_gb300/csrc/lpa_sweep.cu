// lpa_sweep.cu -- the label-choice sweep (the move step of Alg. 1 / Alg. 3) on sm_103a.
//
// One launch sweeps every vertex once: C_next[i] = choice(C_prev) (synchronous), with
// the pick-less commit rule (Sec. 4.5), and adds the number of changed labels to dN.
// CTAs [0, nhubs) take one hub vertex each; the remaining CTAs take one chunk of
// consecutive low-degree vertices.  This is a gather/reduce: no tensor cores.
//
// Sketch modes (MG, BM):
//   chunk CTA: (1) load the chunk's row starts and current labels; (2) stage the
//   chunk's CSR slice edge-parallel into shared memory as (C_prev[j], w) pairs --
//   coalesced index/weight loads, 16+ independent label gathers per thread, self-loops
//   and zero weights marked -1; (3) assign leaves to threads, sorted by leaf count then
//   degree octave so warps are balanced and a vertex's L leaves occupy L lanes aligned
//   to L; (4) each thread folds its leaf from shared memory into a register sketch;
//   (5) stride-doubling shuffle tree inside each L-lane group; (6) leaf 0 selects and
//   commits; labels are written back coalesced; one atomic per CTA adds dN.
//   hub CTA: thread l < L folds leaf l straight from global memory (batched loads),
//   then the same tree: shuffles up to 32 leaves, shared memory beyond.
// Exact mode (the nu-LPA baseline, Fig. 1): a per-vertex open-addressing table of
//   capacity = largest power of two <= 2d, in shared memory for chunk vertices and in
//   a global O(E) workspace for hubs.
#include "lpa_internal.cuh"

namespace lpa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- sketch states

// k-slot weighted Misra-Gries sketch in registers (Sec. 4.1).  Empty slots hold
// key -1 and value 0; labels are >= 0, so a key only ever matches an occupied slot.
template <int K>
struct MGSketch {
  int key[K];
  float val[K];

  __device__ __forceinline__ void init(int /*own*/) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      key[s] = -1;
      val[s] = 0.f;
    }
  }

  // first free slot gets (c, w); returns false if none is free
  __device__ __forceinline__ bool place(int c, float w) {
    bool placed = false;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      bool e = !placed && (val[s] == 0.f);
      key[s] = e ? c : key[s];
      val[s] = e ? w : val[s];
      placed = placed || e;
    }
    return placed;
  }

  // sketchAccumulate (Alg. 2) with the clamped decrement
  __device__ __forceinline__ void add(int c, float w) {
    bool hit = false;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      bool m = (key[s] == c);
      val[s] = m ? val[s] + w : val[s];
      hit = hit || m;
    }
    if (hit) return;
    if (place(c, w)) return;
    float delta = w;
#pragma unroll
    for (int s = 0; s < K; ++s) delta = fminf(delta, val[s]);
#pragma unroll
    for (int s = 0; s < K; ++s) {
      val[s] = val[s] - delta;
      key[s] = (val[s] == 0.f) ? -1 : key[s];
    }
    w = w - delta;
    if (w > 0.f) place(c, w);
  }

  // merge(A = this, B): B's occupied slots in ascending slot order
  __device__ __forceinline__ void merge_from(const int* bk, const float* bv) {
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (bv[s] > 0.f) add(bk[s], bv[s]);
  }

  // receive the sketch of lane + s; merge it when `take`
  __device__ __forceinline__ void shfl_merge(int s, bool take) {
    int bk[K];
    float bv[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      bk[q] = __shfl_down_sync(kFull, key[q], s);
      bv[q] = __shfl_down_sync(kFull, val[q], s);
    }
    if (take) merge_from(bk, bv);
  }

  // sketchMaxKey (single scan, Sec. 4.4): heaviest occupied slot, ties to the
  // smallest label; -1 when empty
  __device__ __forceinline__ int choose() const {
    int best = -1;
    float bv = 0.f;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      bool better = (val[s] > bv) || (val[s] == bv && val[s] > 0.f && key[s] < best);
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
  static constexpr int kSlots = K;
};

// Weighted Boyer-Moore candidate (Sec. 4.7, Alg. 3), as printed.
struct BMState {
  int c;
  float w;
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
  // pair max: larger w#, ties to the smaller label
  __device__ __forceinline__ void take_better(int oc, float ow) {
    bool better = (ow > w) || (ow == w && oc < c);
    c = better ? oc : c;
    w = better ? ow : w;
  }
  __device__ __forceinline__ void shfl_merge(int s, bool take) {
    int oc = __shfl_down_sync(kFull, c, s);
    float ow = __shfl_down_sync(kFull, w, s);
    if (take) take_better(oc, ow);
  }
  __device__ __forceinline__ int choose() const { return w > 0.f ? c : -1; }
  __device__ __forceinline__ void store(int* k, float* v) const {
    k[0] = c;
    v[0] = w;
  }
  __device__ __forceinline__ void load(const int* k, const float* v) {
    c = k[0];
    w = v[0];
  }
  __device__ __forceinline__ void merge_from(const int* k, const float* v) {
    take_better(k[0], v[0]);
  }
  static constexpr int kSlots = 1;
};

// ------------------------------------------------------------- shared helpers

// sort key of a chunk vertex: leaf count first (32..2), then degree octave (L = 1)
__device__ __forceinline__ int class_key(int d, int L) {
  if (L > 1) return 16 + (31 - __clz(L));         // 17..21
  return d == 0 ? 0 : min(32 - __clz(d), 15);     // 0..15
}

__device__ __forceinline__ int commit(int c, int old, int pick_less) {
  return (c >= 0 && c != old && (!pick_less || c < old)) ? c : old;
}

// Cross-warp part of the stride-doubling tree for a hub with L > 32 leaves: warp
// leaders deposit their sketches, thread 0 merges them level by level.
template <class S>
__device__ __forceinline__ void hub_cross_warp(S& st, int L, int tid, int* sk, float* sv) {
  const int nw = L / 32;
  if ((tid & 31) == 0 && (tid >> 5) < nw) st.store(sk + (tid >> 5) * S::kSlots, sv + (tid >> 5) * S::kSlots);
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

// --------------------------------------------------------- sketch sweep kernels

template <class S, bool WT>
__device__ __forceinline__ void fold_global(S& st, const SweepArgs& a, int v, int64_t b,
                                            int64_t e) {
  constexpr int B = 8;
  for (int64_t q = b; q < e; q += B) {
    int j[B];
    float w[B];
    int c[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const bool in = q + u < e;
      j[u] = in ? __ldg(a.idx + q + u) : v;
      w[u] = WT ? (in ? __ldg(a.w + q + u) : 0.f) : (in ? 1.f : 0.f);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) c[u] = (j[u] != v && w[u] > 0.f) ? __ldg(a.c_prev + j[u]) : -1;
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (c[u] >= 0) st.add(c[u], w[u]);
  }
}

template <class S, bool WT>
__device__ void hub_sketch(const SweepArgs& a, int v) {
  __shared__ int sk[(kMaxLeaves / 32) * 32];
  __shared__ float sv[(kMaxLeaves / 32) * 32];
  const int tid = threadIdx.x;
  const int64_t base = a.off[v];
  const int64_t d = a.off[v + 1] - base;
  const int L = leaf_count(d, a.e0, a.lmax);
  const int own = a.c_prev[v];
  S st;
  st.init(own);
  if (tid < L) fold_global<S, WT>(st, a, v, base + (tid * d) / L, base + ((tid + 1) * d) / L);
  const int lane = tid & 31;
  const int Lw = L < 32 ? L : 32;
  for (int s = 1; s < Lw; s <<= 1) st.shfl_merge(s, tid < L && (lane & (2 * s - 1)) == 0);
  if (L > 32) hub_cross_warp<S>(st, L, tid, sk, sv);
  if (tid == 0) {
    const int nl = commit(st.choose(), own, a.pick_less);
    a.c_next[v] = nl;
    if (nl != own) atomicAdd(a.dn, 1ull);
  }
}

template <class S, bool WT>
__device__ void chunk_sketch(const SweepArgs& a, int chunk, unsigned char* smem) {
  int* s_lab = reinterpret_cast<int*>(smem);
  float* s_w = reinterpret_cast<float*>(s_lab + kChunkCap);
  __shared__ int s_start[kThreads + 1];
  __shared__ int s_old[kThreads];
  __shared__ int s_new[kThreads];
  __shared__ int s_leaf[kThreads];
  __shared__ int s_cnt[32];
  __shared__ int s_base[32];
  __shared__ int s_total;

  const int tid = threadIdx.x;
  const int v0 = a.chunk_v0[chunk];
  const int nv = a.chunk_v1[chunk] - v0;
  const int64_t base = a.off[v0];
  if (tid < nv) {
    s_start[tid] = (int)(a.off[v0 + tid] - base);
    s_old[tid] = a.c_prev[v0 + tid];
  }
  if (tid == 0) s_start[nv] = (int)(a.off[v0 + nv] - base);
  if (tid < 32) s_cnt[tid] = 0;
  __syncthreads();

  // leaf counts per class
  int d = 0, L = 0, key = 0;
  if (tid < nv) {
    d = s_start[tid + 1] - s_start[tid];
    L = leaf_count(d, a.e0, a.lmax);
    key = class_key(d, L);
    atomicAdd(&s_cnt[key], L);
  }
  // stage (C_prev[j], w) for the chunk's CSR slice
  const int ne = s_start[nv];
  {
    constexpr int U = 4;
    for (int q0 = tid; q0 < ne; q0 += kThreads * U) {
      int j[U];
      float w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * kThreads;
        const bool in = q < ne;
        j[u] = in ? __ldg(a.idx + base + q) : 0;
        w[u] = WT ? (in ? __ldg(a.w + base + q) : 0.f) : 1.f;
      }
      int c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * kThreads;
        c[u] = (q < ne) ? __ldg(a.c_prev + j[u]) : -1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * kThreads;
        if (q < ne) {
          const unsigned r = (unsigned)(j[u] - v0);  // a self-loop lies in its own row
          const bool self = r < (unsigned)nv && s_start[r] <= q && q < s_start[r + 1];
          s_lab[q] = (self || !(w[u] > 0.f)) ? -1 : c[u];
          if (WT) s_w[q] = w[u];
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int c = 31; c >= 0; --c) {
      const int x = s_cnt[c];
      s_base[c] = run;
      run += x;
    }
    s_total = run;
  }
  __syncthreads();
  if (tid < nv) {
    // slots of one class start at a multiple of every smaller class's leaf count, so a
    // vertex's L leaves land on L lanes aligned to L inside one warp
    const int slot = atomicAdd(&s_base[key], L);
    for (int l = 0; l < L; ++l) s_leaf[slot + l] = (tid << 5) | l;
  }
  __syncthreads();

  // fold one leaf per thread
  S st;
  int t = 0, leaf = 0, Lt = 0;
  if (tid < s_total) {
    const int p = s_leaf[tid];
    t = p >> 5;
    leaf = p & 31;
    const int dt = s_start[t + 1] - s_start[t];
    Lt = leaf_count(dt, a.e0, a.lmax);
    st.init(s_old[t]);
    const int b = s_start[t] + (int)(((int64_t)leaf * dt) / Lt);
    const int e = s_start[t] + (int)(((int64_t)(leaf + 1) * dt) / Lt);
    for (int q = b; q < e; ++q) {
      const int c = s_lab[q];
      if (c >= 0) st.add(c, WT ? s_w[q] : 1.f);
    }
  } else {
    st.init(-1);
  }
  // merge the L leaves of each vertex (stride-doubling, within the warp)
  const int maxL = __reduce_max_sync(kFull, Lt);
  for (int s = 1; s < maxL; s <<= 1) st.shfl_merge(s, Lt > s && (leaf & (2 * s - 1)) == 0);
  int changed = 0;
  if (tid < s_total && leaf == 0) {
    const int nl = commit(st.choose(), s_old[t], a.pick_less);
    s_new[t] = nl;
    changed = nl != s_old[t];
  }
  const int cnt = __syncthreads_count(changed);
  if (tid < nv) a.c_next[v0 + tid] = s_new[tid];
  if (tid == 0 && cnt > 0) atomicAdd(a.dn, (unsigned long long)cnt);
}

template <class S, bool WT>
__global__ void __launch_bounds__(kThreads) sweep_sketch_kernel(SweepArgs a) {
  if (a.done != nullptr && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  if ((int)blockIdx.x < a.nhubs)
    hub_sketch<S, WT>(a, a.hubs[blockIdx.x]);
  else
    chunk_sketch<S, WT>(a, (int)blockIdx.x - a.nhubs, smem);
}

// ------------------------------------------------------------------ exact mode

__device__ __forceinline__ unsigned table_hash(int c, int lg) {
  return ((unsigned)c * 2654435761u) >> (32 - lg);
}

__device__ __forceinline__ bool better_kv(float v, int k, float bv, int bk) {
  return (v > bv) || (v == bv && v > 0.f && k < bk);
}

template <bool WT>
__device__ void hub_exact(const SweepArgs& a, int h) {
  __shared__ float s_bv[kThreads / 32];
  __shared__ int s_bk[kThreads / 32];
  const int tid = threadIdx.x;
  const int v = a.hubs[h];
  const int64_t base = a.off[v];
  const int64_t d = a.off[v + 1] - base;
  int lg = 1;
  while (((int64_t)1 << (lg + 1)) <= 2 * d) ++lg;
  const int64_t cap = (int64_t)1 << lg;  // largest power of two <= 2d (> d)
  int* tk = a.tab_keys + a.hub_tab[h];
  float* tv = a.tab_vals + a.hub_tab[h];
  for (int64_t s = tid; s < cap; s += kThreads) {
    tk[s] = -1;
    tv[s] = 0.f;
  }
  __syncthreads();
  for (int64_t q = base + tid; q < base + d; q += kThreads) {
    const int j = __ldg(a.idx + q);
    const float w = WT ? __ldg(a.w + q) : 1.f;
    if (j == v || !(w > 0.f)) continue;
    const int c = __ldg(a.c_prev + j);
    unsigned s = table_hash(c, lg);
    for (int64_t probe = 0; probe < cap; ++probe) {
      const int old = atomicCAS(tk + s, -1, c);
      if (old == -1 || old == c) {
        atomicAdd(tv + s, w);
        break;
      }
      s = (s + 1) & (unsigned)(cap - 1);
    }
  }
  __syncthreads();
  float bv = 0.f;
  int bk = -1;
  for (int64_t s = tid; s < cap; s += kThreads) {
    const int k = tk[s];
    const float x = tv[s];
    if (k >= 0 && better_kv(x, k, bv, bk)) {
      bv = x;
      bk = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_down_sync(kFull, bv, o);
    const int ok = __shfl_down_sync(kFull, bk, o);
    if (better_kv(ov, ok, bv, bk)) {
      bv = ov;
      bk = ok;
    }
  }
  if ((tid & 31) == 0) {
    s_bv[tid >> 5] = bv;
    s_bk[tid >> 5] = bk;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kThreads / 32; ++w)
      if (better_kv(s_bv[w], s_bk[w], bv, bk)) {
        bv = s_bv[w];
        bk = s_bk[w];
      }
    const int own = a.c_prev[v];
    const int nl = commit(bv > 0.f ? bk : -1, own, a.pick_less);
    a.c_next[v] = nl;
    if (nl != own) atomicAdd(a.dn, 1ull);
  }
}

template <bool WT>
__device__ void chunk_exact(const SweepArgs& a, int chunk, unsigned char* smem) {
  int* s_lab = reinterpret_cast<int*>(smem);
  float* s_w = reinterpret_cast<float*>(s_lab + kChunkCapExact);
  int* s_tk = reinterpret_cast<int*>(s_w + (WT ? kChunkCapExact : 0));
  float* s_tv = reinterpret_cast<float*>(s_tk + 2 * kChunkCapExact);
  __shared__ int s_start[kThreads + 1];
  __shared__ int s_old[kThreads];
  const int tid = threadIdx.x;
  const int v0 = a.chunk_v0[chunk];
  const int nv = a.chunk_v1[chunk] - v0;
  const int64_t base = a.off[v0];
  if (tid < nv) {
    s_start[tid] = (int)(a.off[v0 + tid] - base);
    s_old[tid] = a.c_prev[v0 + tid];
  }
  if (tid == 0) s_start[nv] = (int)(a.off[v0 + nv] - base);
  __syncthreads();
  const int ne = s_start[nv];
  for (int q = tid; q < ne; q += kThreads) {
    const int j = __ldg(a.idx + base + q);
    const float w = WT ? __ldg(a.w + base + q) : 1.f;
    const unsigned r = (unsigned)(j - v0);
    const bool self = r < (unsigned)nv && s_start[r] <= q && q < s_start[r + 1];
    s_lab[q] = (self || !(w > 0.f)) ? -1 : __ldg(a.c_prev + j);
    if (WT) s_w[q] = w;
  }
  __syncthreads();
  int changed = 0;
  int nl = 0;
  if (tid < nv) {
    const int b = s_start[tid], d = s_start[tid + 1] - b;
    int best = -1;
    if (d > 0) {
      int lg = 1;
      while ((1 << (lg + 1)) <= 2 * d) ++lg;
      const int cap = 1 << lg;
      int* tk = s_tk + 2 * b;
      float* tv = s_tv + 2 * b;
      for (int s = 0; s < cap; ++s) {
        tk[s] = -1;
        tv[s] = 0.f;
      }
      for (int q = b; q < b + d; ++q) {
        const int c = s_lab[q];
        if (c < 0) continue;
        const float w = WT ? s_w[q] : 1.f;
        unsigned s = table_hash(c, lg);
        while (tk[s] != -1 && tk[s] != c) s = (s + 1) & (unsigned)(cap - 1);
        tk[s] = c;
        tv[s] = tv[s] + w;
      }
      float bv = 0.f;
      for (int s = 0; s < cap; ++s)
        if (tk[s] >= 0 && better_kv(tv[s], tk[s], bv, best)) {
          bv = tv[s];
          best = tk[s];
        }
    }
    nl = commit(best, s_old[tid], a.pick_less);
    changed = nl != s_old[tid];
    a.c_next[v0 + tid] = nl;
  }
  const int cnt = __syncthreads_count(changed);
  if (tid == 0 && cnt > 0) atomicAdd(a.dn, (unsigned long long)cnt);
}

template <bool WT>
__global__ void __launch_bounds__(kThreads) sweep_exact_kernel(SweepArgs a) {
  if (a.done != nullptr && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  if ((int)blockIdx.x < a.nhubs)
    hub_exact<WT>(a, (int)blockIdx.x);
  else
    chunk_exact<WT>(a, (int)blockIdx.x - a.nhubs, smem);
}

template <class S, bool WT>
cudaError_t launch_sketch(const SweepArgs& a, size_t smem, cudaStream_t s) {
  auto kern = sweep_sketch_kernel<S, WT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)(a.nhubs + a.nchunks);
  if (grid == 0) return cudaSuccess;
  kern<<<grid, kThreads, smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_mg(bool weighted, const SweepArgs& a, size_t smem, cudaStream_t s) {
  return weighted ? launch_sketch<MGSketch<K>, true>(a, smem, s)
                  : launch_sketch<MGSketch<K>, false>(a, smem, s);
}

}  // namespace

size_t sweep_smem_bytes(int mode, bool weighted) {
  if (mode == kExact)
    return (size_t)kChunkCapExact * (weighted ? 8 : 4) + (size_t)2 * kChunkCapExact * 8;
  return (size_t)kChunkCap * (weighted ? 8 : 4);
}

cudaError_t launch_sweep(int mode, int k, bool weighted, const SweepArgs& a, cudaStream_t s) {
  const size_t smem = sweep_smem_bytes(mode, weighted);
  if (mode == kBM)
    return weighted ? launch_sketch<BMState, true>(a, smem, s)
                    : launch_sketch<BMState, false>(a, smem, s);
  if (mode == kExact) {
    auto kern = weighted ? sweep_exact_kernel<true> : sweep_exact_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)(a.nhubs + a.nchunks);
    if (grid == 0) return cudaSuccess;
    kern<<<grid, kThreads, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
  }
  switch (k) {
    case 1: return launch_mg<1>(weighted, a, smem, s);
    case 2: return launch_mg<2>(weighted, a, smem, s);
    case 4: return launch_mg<4>(weighted, a, smem, s);
    case 8: return launch_mg<8>(weighted, a, smem, s);
    case 16: return launch_mg<16>(weighted, a, smem, s);
    case 32: return launch_mg<32>(weighted, a, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lpa
