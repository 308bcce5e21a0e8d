// lpa_exact.cu -- the exact label choice (Eq. 3), the quality baseline of the paper's
// comparison (the nu-LPA per-vertex hashtable of Fig. 1).
//
// Chunk CTAs take runs of consecutive vertices whose rows fit the shared-memory stage:
// the CTA stages (C_prev[j], w) edge-parallel, then each thread builds its vertex's
// open-addressing table (capacity = largest power of two <= 2d, linear probing) in
// shared memory and takes the argmax, ties to the smallest label.  Hub CTAs (rows longer
// than a chunk) build the table in a global O(E) workspace with atomics.  Sums are exact
// for integer-valued weights, so the result does not depend on the atomic order.
#include "lpa_internal.cuh"

namespace lpa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int commit(int c, int old, int pick_less) {
  return (c >= 0 && c != old && (!pick_less || c < old)) ? c : old;
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
  __shared__ int s_changed;
  const int v = a.hubs[h];
  const int64_t base = a.off[v];
  const int64_t d = a.off[v + 1] - base;
  if ((a.act_in != nullptr && !a.act_in[v]) || (a.gid != nullptr && a.gdone[a.gid[v]])) {
    if (tid == 0) a.c_next[v] = a.c_prev[v];  // not swept: keep the label
    return;
  }
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
    const int nl = commit(bv > 0.f ? bk : -1, own, a.gpl != nullptr ? a.gpl[a.gid[v]] : a.pick_less);
    a.c_next[v] = nl;
    s_changed = nl != own;
    if (nl != own) atomicAdd(a.dn, 1ull);
    if (nl != own && a.gdn != nullptr) atomicAdd(a.gdn + a.gid[v], 1u);
    if (a.scanned) atomicAdd(a.scanned + (h & (kDnSlots - 1)), (unsigned long long)d);
  }
  if (a.act_out != nullptr) {  // a moved vertex marks its neighbours unprocessed
    __syncthreads();
    if (s_changed)
      for (int64_t q = base + tid; q < base + d; q += kThreads) a.act_out[__ldg(a.idx + q)] = 1;
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
  const bool act = tid < nv && (a.act_in == nullptr || a.act_in[v0 + tid] != 0) &&
                   (a.gid == nullptr || !a.gdone[a.gid[v0 + tid]]);
  if (tid < nv) {
    const int b = s_start[tid], d = act ? s_start[tid + 1] - b : 0;
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
    nl = commit(best, s_old[tid], a.gpl != nullptr ? a.gpl[a.gid[v0 + tid]] : a.pick_less);
    changed = nl != s_old[tid];
    a.c_next[v0 + tid] = nl;
    if (changed && a.gdn != nullptr) atomicAdd(a.gdn + a.gid[v0 + tid], 1u);
  }
  const int cnt = __syncthreads_count(changed);
  if (tid == 0 && cnt > 0) atomicAdd(a.dn, (unsigned long long)cnt);
  if (a.act_out != nullptr) {
    if (changed)
      for (int q = s_start[tid]; q < s_start[tid + 1]; ++q) a.act_out[__ldg(a.idx + base + q)] = 1;
    if (tid < 32) {
      unsigned part = 0;
      for (int t = tid; t < nv; t += 32)
        if (a.act_in[v0 + t]) part += (unsigned)(s_start[t + 1] - s_start[t]);
      part = __reduce_add_sync(kFull, part);
      if (tid == 0 && part > 0)
        atomicAdd(a.scanned + (chunk & (kDnSlots - 1)), (unsigned long long)part);
    }
  }
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

}  // namespace

size_t exact_smem_bytes(bool weighted) {
  return (size_t)kChunkCapExact * (weighted ? 8 : 4) + (size_t)2 * kChunkCapExact * 8;
}

cudaError_t launch_sweep_exact(bool weighted, const SweepArgs& a, cudaStream_t s) {
  const size_t smem = exact_smem_bytes(weighted);
  auto kern = weighted ? sweep_exact_kernel<true> : sweep_exact_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)(a.nhubs + a.nchunks);
  if (grid == 0) return cudaSuccess;
  kern<<<grid, kThreads, smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lpa
