// lpa_exact.cu -- the exact label choice (Eq. 3), the quality baseline of the paper's
// comparison (the nu-LPA per-vertex hashtable of Fig. 1).
//
// Every vertex gets an open-addressing table (capacity = largest power of two <= 2d,
// linear probing) of its neighbours' labels and their summed weights; the choice is the
// heaviest label, ties to the smallest.  Two kernels:
//  * chunk CTAs take runs of consecutive vertices whose rows fit the shared-memory stage.
//    The CTA stages (C_prev[j], w) entry-parallel, then inserts entry-parallel: a warp
//    takes 32 consecutive positions, sums runs of equal (row, label) with a segmented
//    scan across its lanes, and the run's last lane adds the sum with one shared-memory
//    atomic -- so rows of every length share the CTA's threads evenly, and a row whose
//    neighbours mostly share one label does not pile its atomics onto one slot.  The
//    argmax is slot-parallel too: (sum, label) packed so that a larger 64-bit value means
//    a heavier sum, then a smaller label, and reduced per row by a segmented warp
//    maximum and one shared atomic maximum per run.
//  * hub CTAs (rows longer than a chunk) build the row's table in shared memory when it
//    fits (kHubSmemSlots) and in a global O(E) workspace otherwise, with the same
//    warp-aggregated inserts.
// Sums are exact for integer-valued weights, so the result does not depend on the
// atomic order.
#include "lpa_internal.cuh"

namespace lpa {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Largest hub table kept in shared memory: 8192 slots (64 KB), three hub CTAs per SM.
constexpr int kHubSmemSlots = 8192;
// Positions a thread loads before it gathers their labels (memory-level parallelism).
constexpr int kStageBatch = 4;

__device__ __forceinline__ int commit(int c, int old, int pick_less) {
  return (c >= 0 && c != old && (!pick_less || c < old)) ? c : old;
}

__device__ __forceinline__ unsigned table_hash(int c, int lg) {
  return ((unsigned)c * 2654435761u) >> (32 - lg);
}

__device__ __forceinline__ bool better_kv(float v, int k, float bv, int bk) {
  return (v > bv) || (v == bv && v > 0.f && k < bk);
}

// log2 of a row's table capacity: the largest power of two <= 2d (> d)
__device__ __forceinline__ int table_lg(int64_t d) {
  return 63 - __clzll(2 * d);
}

// Runs of equal key among the warp's lanes (all 32 lanes call it): w becomes the sum of
// the run's weights up to this lane; returns true on the run's last lane.
template <class K>
__device__ __forceinline__ bool run_sum(K key, float& w) {
  const int lane = threadIdx.x & 31;
  const K kp = __shfl_up_sync(kFull, key, 1);
  const unsigned heads = __ballot_sync(kFull, lane == 0 || kp != key);
  const int run0 = 31 - __clz(heads & (kFull >> (31 - lane)));
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float y = __shfl_up_sync(kFull, w, d);
    if (lane - d >= run0) w += y;
  }
  return lane == 31 || ((heads >> (lane + 1)) & 1u);
}

// Add w to label c's slot of the table (tk, tv) of capacity 2^lg: linear probing from
// the label's hash, claiming an empty slot by compare-and-swap.  The table never fills
// (a row has fewer distinct labels than slots), so the probe ends.
__device__ __forceinline__ void table_add(int* tk, float* tv, int lg, int c, float w) {
  const unsigned mask = (1u << lg) - 1u;
  unsigned s = table_hash(c, lg);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int old = atomicCAS(tk + s, -1, c);
    if (old == -1 || old == c) {
      atomicAdd(tv + s, w);
      return;
    }
    s = (s + 1) & mask;
  }
}

// (sum, label) packed so that the larger value is the heavier sum, then the smaller label
// (sums are positive, so their bit patterns order like the values); 0 = no label
__device__ __forceinline__ unsigned long long pack_kv(float v, int k) {
  return ((unsigned long long)__float_as_uint(v) << 32) | (0xffffffffu - (unsigned)k);
}
__device__ __forceinline__ int unpack_label(unsigned long long p) {
  return (p >> 32) != 0 ? (int)(0xffffffffu - (unsigned)p) : -1;
}

// Hub CTA: one long row, its table in shared memory (capacity <= kHubSmemSlots) or in
// the global workspace.
template <bool WT>
__global__ void __launch_bounds__(kThreads) sweep_exact_hub_kernel(SweepArgs a) {
  if (a.done != nullptr && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_bv[kThreads / 32];
  __shared__ int s_bk[kThreads / 32];
  __shared__ int s_changed;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int h = blockIdx.x;
  const int v = a.hubs[h];
  const int64_t base = a.off[v];
  const int64_t d = a.off[v + 1] - base;
  if ((a.act_in != nullptr && !a.act_in[v]) || (a.gid != nullptr && a.gdone[a.gid[v]])) {
    if (tid == 0) a.c_next[v] = a.c_prev[v];  // not swept: keep the label
    return;
  }
  const int lg = table_lg(d);
  const int64_t cap = (int64_t)1 << lg;
  const bool in_smem = cap <= kHubSmemSlots;
  int* tk = in_smem ? reinterpret_cast<int*>(smem) : a.tab_keys + a.hub_tab[h];
  float* tv = in_smem ? reinterpret_cast<float*>(smem + sizeof(int) * kHubSmemSlots)
                      : a.tab_vals + a.hub_tab[h];
  for (int64_t s = tid; s < cap; s += kThreads) {
    tk[s] = -1;
    tv[s] = 0.f;
  }
  __syncthreads();
  // entries 32 at a time per warp, kStageBatch steps loaded and gathered together; runs
  // of equal labels are summed before their atomic
  for (int64_t q0 = base + 32 * warp; q0 < base + d; q0 += kStageBatch * kThreads) {
    int c[kStageBatch];
    float w[kStageBatch];
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const int64_t q = q0 + u * kThreads + lane;
      c[u] = q < base + d ? __ldg(a.idx + q) : v;
      w[u] = q < base + d ? (WT ? __ldg(a.w + q) : 1.f) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const bool use = c[u] != v && w[u] > 0.f;
      c[u] = use ? __ldg(a.c_prev + c[u]) : -1;
      w[u] = use ? w[u] : 0.f;
    }
#pragma unroll 1
    for (int u = 0; u < kStageBatch; ++u) {
      int cu = c[0];
      float wu = w[0];
#pragma unroll
      for (int t = 0; t + 1 < kStageBatch; ++t) {
        c[t] = c[t + 1];
        w[t] = w[t + 1];
      }
      if (run_sum(cu, wu) && cu >= 0) table_add(tk, tv, lg, cu, wu);
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
  if (lane == 0) {
    s_bv[warp] = bv;
    s_bk[warp] = bk;
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

// Chunk CTA: a run of consecutive vertices whose rows fit the stage (kChunkCapExact).
template <bool WT>
__global__ void __launch_bounds__(kThreads) sweep_exact_chunk_kernel(SweepArgs a) {
  if (a.done != nullptr && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  int* s_lab = reinterpret_cast<int*>(smem);
  float* s_w = reinterpret_cast<float*>(s_lab + kChunkCapExact);
  int* s_tk = reinterpret_cast<int*>(s_w + (WT ? kChunkCapExact : 0));
  float* s_tv = reinterpret_cast<float*>(s_tk + 2 * kChunkCapExact);
  __shared__ int s_start[kThreads + 1];
  __shared__ int s_old[kThreads];
  __shared__ unsigned char s_act[kThreads];
  __shared__ unsigned long long s_best[kThreads];
  __shared__ unsigned char s_row[kChunkCapExact];  // the row of each chunk position
  __shared__ int s_wmax[kThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int chunk = blockIdx.x;
  const int v0 = a.chunk_v0[chunk];
  const int nv = a.chunk_v1[chunk] - v0;
  const int64_t base = a.off[v0];
  if (tid < nv) {
    s_start[tid] = (int)(a.off[v0 + tid] - base);
    s_old[tid] = a.c_prev[v0 + tid];
    s_act[tid] = (a.act_in == nullptr || a.act_in[v0 + tid] != 0) &&
                 (a.gid == nullptr || !a.gdone[a.gid[v0 + tid]]);
    s_best[tid] = 0ull;
  }
  if (tid == 0) s_start[nv] = (int)(a.off[v0 + nv] - base);
  __syncthreads();
  const int ne = s_start[nv];
  // stage kStageBatch positions per thread at a time: their loads, then their gathers
  for (int q0 = tid; q0 < ne; q0 += kStageBatch * kThreads) {
    int j[kStageBatch];
    float w[kStageBatch];
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const int q = q0 + u * kThreads;
      j[u] = q < ne ? __ldg(a.idx + base + q) : -1;
      w[u] = q < ne ? (WT ? __ldg(a.w + base + q) : 1.f) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const int q = q0 + u * kThreads;
      if (q < ne) {
        const unsigned r = (unsigned)(j[u] - v0);
        const bool self = r < (unsigned)nv && s_start[r] <= q && q < s_start[r + 1];
        s_lab[q] = (self || !(w[u] > 0.f)) ? -1 : __ldg(a.c_prev + j[u]);
        if (WT) s_w[q] = w[u];
      }
    }
  }
  for (int s = tid; s < 2 * ne; s += kThreads) {
    s_tk[s] = -1;
    s_tv[s] = 0.f;
  }
  // the row of every position: each non-empty row marks its first position, then a
  // running maximum over the positions (rows are in position order)
  for (int q = tid; q < ne; q += kThreads) s_row[q] = 0;
  __syncthreads();
  if (tid < nv && s_start[tid] < s_start[tid + 1]) s_row[s_start[tid]] = (unsigned char)tid;
  __syncthreads();
  {
    constexpr int kPer = kChunkCapExact / kThreads;  // positions per thread, in a block
    const int q0 = tid * kPer;
    int m = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u)
      if (q0 + u < ne) m = max(m, (int)s_row[q0 + u]);
    // maximum over the threads below (exclusive): warp scan, then across warps
    int x = m;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(kFull, x, d);
      if (lane >= d) x = max(x, y);
    }
    if (lane == 31) s_wmax[warp] = x;
    __syncthreads();
    int before = __shfl_up_sync(kFull, x, 1);
    if (lane == 0) before = 0;
    for (int w = 0; w < warp; ++w) before = max(before, s_wmax[w]);
#pragma unroll
    for (int u = 0; u < kPer; ++u)
      if (q0 + u < ne) {
        before = max(before, (int)s_row[q0 + u]);
        s_row[q0 + u] = (unsigned char)before;
      }
  }
  __syncthreads();
  // inserts: 32 consecutive positions per warp step, runs of equal (row, label) summed
  for (int q0 = 32 * warp; q0 < ne; q0 += kThreads) {
    const int q = q0 + lane;
    int c = -1, r = 0;
    float w = 0.f;
    if (q < ne) {
      c = s_lab[q];
      if (c >= 0) {
        r = s_row[q];
        if (s_act[r]) w = WT ? s_w[q] : 1.f;
        else c = -1;
      }
    }
    const unsigned long long key =
        c >= 0 ? ((unsigned long long)(unsigned)r << 32) | (unsigned)c : ~0ull;
    if (run_sum(key, w) && c >= 0) {
      const int b = s_start[r];
      table_add(s_tk + 2 * b, s_tv + 2 * b, table_lg(s_start[r + 1] - b), c, w);
    }
  }
  __syncthreads();
  // argmax per row: slot-parallel, runs of one row reduced by a segmented warp maximum
  for (int i0 = 32 * warp; i0 < 2 * ne; i0 += kThreads) {
    const int i = i0 + lane;
    int r = nv;  // past the last row: no slot
    unsigned long long pk = 0ull;
    if (i < 2 * ne) {
      r = s_row[i >> 1];  // row r's table lies in slots [2 start_r, 2 start_{r+1})
      const int k = s_tk[i];
      if (k >= 0) pk = pack_kv(s_tv[i], k);
    }
    const int rp = __shfl_up_sync(kFull, r, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || rp != r);
    const int run0 = 31 - __clz(heads & (kFull >> (31 - lane)));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, pk, d);
      if (lane - d >= run0 && y > pk) pk = y;
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && pk != 0ull) atomicMax(s_best + r, pk);
  }
  __syncthreads();
  int changed = 0;
  if (tid < nv) {
    const int nl = commit(unpack_label(s_best[tid]), s_old[tid],
                          a.gpl != nullptr ? a.gpl[a.gid[v0 + tid]] : a.pick_less);
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

}  // namespace

size_t exact_smem_bytes(bool weighted) {
  return (size_t)kChunkCapExact * (weighted ? 8 : 4) + (size_t)2 * kChunkCapExact * 8;
}

cudaError_t launch_sweep_exact(bool weighted, const SweepArgs& a, cudaStream_t s) {
  if (a.nhubs > 0) {
    const size_t smem = (size_t)kHubSmemSlots * (sizeof(int) + sizeof(float));
    auto kern = weighted ? sweep_exact_hub_kernel<true> : sweep_exact_hub_kernel<false>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)a.nhubs, kThreads, smem, s>>>(a);
    count_launch();
  }
  if (a.nchunks > 0) {
    const size_t smem = exact_smem_bytes(weighted);
    auto kern = weighted ? sweep_exact_chunk_kernel<true> : sweep_exact_chunk_kernel<false>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)a.nchunks, kThreads, smem, s>>>(a);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace lpa
