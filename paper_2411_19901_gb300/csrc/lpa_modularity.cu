// lpa_modularity.cu -- modularity (Sec. 3.2, Eq. 1):
// Q = sum_c sigma_c / 2m - sum_c (Sigma_c / 2m)^2, accumulated in fp64.
//
// Two rows passes.  The one of a run reuses the sweep's work map (hub kernels per
// CTA-size class, packed lane descriptors) and its pipelined row reads, so it streams
// the CSR at the sweep's rate.  The standalone one (lpa_modularity*, no plan) needs no
// work map: a warp takes 32 consecutive vertices.  Per vertex both form K_i (all
// entries, self-loops included, as stored) and the weight of entries whose neighbour
// shares the label; Sigma_c receives K_i through one atomic per distinct label in a warp.
#include "lpa_fold.cuh"

namespace lpa {
namespace {

constexpr int kModSlots = 4096;
constexpr int kSqBlocks = 152 * 8;

// Row accumulator driven by fold_range: add(C[j], w) for every entry with w > 0.  Both
// sums (K_i and the intra-community weight) are kept as unevaluated fp32 pairs hi + lo
// updated by Knuth's TwoSum, which is exact: each pair holds its running sum to about
// 2^-48 relative, so a leaf's totals match an fp64 sum far inside the 1e-9 tolerance
// while every per-entry operation stays on the fp32 pipe (fp64 runs at a small fraction
// of its rate on this GPU).  The leaf totals continue in fp64.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float w) {
  const float s = hi + w;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (w - bb);
  hi = s;
  lo += err;
}

struct ModAcc {
  float kh, kl, ih, il;
  int cv;
  __device__ __forceinline__ void add(int c, float w) {
    two_sum_add(kh, kl, w);
    if (c == cv) two_sum_add(ih, il, w);
  }
  __device__ __forceinline__ double k() const { return (double)kh + (double)kl; }
  __device__ __forceinline__ double in() const { return (double)ih + (double)il; }
};

// Sum over the L lanes of an aligned group into its first lane.  Lanes of one warp may
// have different L (packed groups): all run the warp's largest L, adding only below their
// own; lanes that are not group leaders end with partial sums that are never read.
__device__ __forceinline__ double warp_down_sum(double x, int L, int Lw) {
  for (int s = 1; s < Lw; s <<= 1) {
    const double y = __shfl_down_sync(kFullMask, x, s);
    if (s < L) x += y;
  }
  return x;
}

// Per-graph totals of a batch (gid null for a single graph): 2m_g and the intra-community
// weight of graph g accumulate into g2m[g], gin[g].
struct ModGraphs {
  const int32_t* gid;
  double* g2m;
  double* gin;
};

// A block's vertex totals: Sigma_c through one atomic per distinct label among a warp's
// owners, per-graph totals (batches) through one atomic per graph in a warp, then the
// block's sums of K_i and of the intra-community weight into one of kModSlots
// accumulators.  s_k, s_in: blockDim.x doubles of shared memory each.
__device__ __forceinline__ void mod_commit(bool owner, int v, int cv, double kv, double in,
                                           double* sigma_c, double* slots, double* s_k,
                                           double* s_in, const ModGraphs& mg) {
  const int tid = threadIdx.x, lane = tid & 31;
  s_k[tid] = owner ? kv : 0.0;
  s_in[tid] = owner ? in : 0.0;
  __syncwarp();
  const unsigned grp = __match_any_sync(kFullMask, owner ? cv : -(lane + 2));
  if (owner && lane == __ffs(grp) - 1) {
    double sum = 0.0;
    for (unsigned g = grp; g; g &= g - 1) sum += s_k[(tid & ~31) + __ffs(g) - 1];
    if (sum != 0.0) atomicAdd(sigma_c + cv, sum);
  }
  if (mg.gid != nullptr) {
    const int gg = owner ? mg.gid[v] : -(lane + 2);
    const unsigned same = __match_any_sync(kFullMask, gg);
    if (owner && lane == __ffs(same) - 1) {
      double a = 0.0, b = 0.0;
      for (unsigned g = same; g; g &= g - 1) {
        a += s_k[(tid & ~31) + __ffs(g) - 1];
        b += s_in[(tid & ~31) + __ffs(g) - 1];
      }
      atomicAdd(mg.g2m + gg, a);
      atomicAdd(mg.gin + gg, b);
    }
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      s_k[tid] += s_k[tid + s];
      s_in[tid] += s_in[tid + s];
    }
    __syncthreads();
  }
  if (tid == 0 && (s_k[0] != 0.0 || s_in[0] != 0.0)) {
    const int slot = (blockIdx.x * 7919u) & (kModSlots - 1);
    atomicAdd(slots + 2 * slot, s_k[0]);
    atomicAdd(slots + 2 * slot + 1, s_in[0]);
  }
}

// Packed lanes (the sweep's lane descriptors): each lane sums its leaf, the L lanes of a
// vertex combine by shuffles, the vertex's first lane holds its totals.
template <int WF>
__global__ void __launch_bounds__(kLaneThreads) modularity_lane_kernel(
    const int32_t* __restrict__ idx, const float* __restrict__ wts, int64_t m,
    const int32_t* __restrict__ labels, WarpPlan p, double* sigma_c, double* slots, ModGraphs mg) {
  __shared__ double s_k[kLaneThreads], s_in[kLaneThreads];
  const int64_t q = (int64_t)blockIdx.x * kLaneThreads + threadIdx.x;
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
  ModAcc acc{0.f, 0.f, 0.f, 0.f, -1};
  if (v >= 0) acc.cv = labels[v];
  const int ngl = (int)((len + 3) >> 2);
  LaneSliceAddr ad{q < p.nlanes ? p.lane_base[q >> 5] : 0, ngl, (1u << (threadIdx.x & 31)) - 1u};
  fold_groups<ModAcc, WF, true>(acc, p, labels, acc.cv, ngl, __reduce_max_sync(kFullMask, ngl),
                                ad);
  double kv = acc.k(), in = acc.in();
  const int Lw = __reduce_max_sync(kFullMask, L);
  if (Lw > 1) {
    kv = warp_down_sum(kv, L, Lw);
    in = warp_down_sum(in, L, Lw);
  }
  mod_commit(v >= 0 && leaf == 0, v, acc.cv, kv, in, sigma_c, slots, s_k, s_in, mg);
}

// Hubs of one class (p.hub_desc, p.hub_base point at the class): leaf t on thread t, from
// the sliced copy.
template <int WF>
__global__ void __launch_bounds__(kThreads) modularity_hub_kernel(
    const int32_t* __restrict__ idx, const float* __restrict__ wts, int64_t m,
    const int32_t* __restrict__ labels, WarpPlan p, double* sigma_c, double* slots, ModGraphs mg) {
  __shared__ double s_k[kThreads], s_in[kThreads];
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const int4 h = __ldg(p.hub_desc + blockIdx.x);
  const int v = h.x;
  const int64_t base = (int64_t)(uint32_t)h.y | ((int64_t)h.z << 32);
  const int64_t d = h.w;
  const int L = leaf_count(d, p.e0, p.lmax);
  ModAcc acc{0.f, 0.f, 0.f, 0.f, labels[v]};
  if (tid < L) {  // leaf tid from the sliced copy
    const int64_t lo = base + (tid * d) / L, len = base + ((tid + 1) * d) / L - lo;
    const int W = L < 32 ? L : 32;
    const int64_t G = hub_leaf_groups(d, L);
    HubSliceAddr ad{p.hub_base[blockIdx.x] + (int64_t)(tid >> 5) * W * G + (tid & 31), W};
    const int ng = (int)((len + 3) >> 2);
    fold_groups<ModAcc, WF, true>(acc, p, labels, acc.cv, ng, ng, ad);
  }
  s_k[tid] = acc.k();
  s_in[tid] = acc.in();
  __syncthreads();
  for (int s = nt / 2; s > 0; s >>= 1) {  // fixed-order tree
    if (tid < s) {
      s_k[tid] += s_k[tid + s];
      s_in[tid] += s_in[tid + s];
    }
    __syncthreads();
  }
  const double kv = s_k[0], in = s_in[0];
  __syncthreads();
  mod_commit(tid == 0, v, acc.cv, kv, in, sigma_c, slots, s_k, s_in, mg);
}

__global__ void zero_f64_kernel(double* p, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) p[i] = 0.0;
}

__global__ void __launch_bounds__(256) sigma_sq_kernel(const double* sigma_c, int32_t n,
                                                      double* sq) {
  __shared__ double s[256];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * 256;
  for (int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x; c < n; c += stride)
    acc += sigma_c[c] * sigma_c[c];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) sq[blockIdx.x] = s[0];
}

// Fixed-order final sums; out4 = {2m, intra weight, sum_c Sigma_c^2, Q}.  a, b, c hold
// na, na, nc partial sums of 2m, the intra-community weight and Sigma_c^2 (a and b read
// with stride sa).
__global__ void __launch_bounds__(256) modularity_total_kernel(const double* a_part,
                                                              const double* b_part, int sa,
                                                              int na, const double* c_part,
                                                              int nc, double* out4) {
  __shared__ double sa_[256], sb_[256], sc_[256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < na; i += 256) {
    a += a_part[(int64_t)sa * i];
    b += b_part[(int64_t)sa * i];
  }
  for (int i = threadIdx.x; i < nc; i += 256) c += c_part[i];
  sa_[threadIdx.x] = a;
  sb_[threadIdx.x] = b;
  sc_[threadIdx.x] = c;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sa_[threadIdx.x] += sa_[threadIdx.x + h];
      sb_[threadIdx.x] += sb_[threadIdx.x + h];
      sc_[threadIdx.x] += sc_[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double two_m = sa_[0];
    out4[0] = two_m;
    out4[1] = sb_[0];
    out4[2] = sc_[0];
    out4[3] = two_m > 0.0 ? sb_[0] / two_m - sc_[0] / (two_m * two_m) : 0.0;
  }
}

// ------------------------------------------------------- standalone pass (no binning)
//
// A warp takes a tile of 32 consecutive vertices.  A row of at most kModShortRow
// positions is summed by its own lane with the pipelined 16-byte reads of the sweep.  A
// longer row is read by the whole warp: lane i folds the i-th of 32 contiguous pieces
// (cut at 4-entry group boundaries) with the same pipelined reads, and the lanes' sums
// are then combined.  Every sum is an fp32 TwoSum pair (fp64 runs at a small fraction of the
// fp32 rate on this GPU): per row, per lane across its rows, and in the combinations.
// Sigma_c receives K_i by one fp64 atomic per distinct label among the warp's rows (runs
// of equal labels summed by a segmented scan, run ends of one label joined by a warp
// match); the totals go through a fixed-order block tree into one partial per block.
// Only the order of the Sigma_c atomics depends on timing.

constexpr int kModThreads = 256;
constexpr int kModMaxBlocks = 152 * 3;  // one wave at 3 CTAs per SM
constexpr int kModShortRow = 64;

// (hi, lo) += (bh, bl), hi updated by TwoSum
__device__ __forceinline__ void two_sum_pair(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (bh - bb);
  hi = s;
  lo = lo + (bl + err);
}

// Lanes <= lane
__device__ __forceinline__ unsigned lanes_upto(int lane) { return 0xffffffffu >> (31 - lane); }

// Positions [b, e) of a row into acc by one lane: the pipelined 16-byte reads of the sweep
// when both arrays start on a 16-byte boundary (VEC), else one entry at a time.
template <bool WT, bool VEC>
__device__ __forceinline__ void mod_range(ModAcc& acc, const int32_t* __restrict__ idx,
                                          const float* __restrict__ wts,
                                          const int32_t* __restrict__ labels, int64_t m,
                                          int v, int64_t b, int64_t e) {
  if constexpr (VEC) {
    fold_range<ModAcc, WT, false>(acc, idx, wts, labels, m, v, b, e);
  } else {
    for (int64_t p = b; p < e; ++p) {
      const float x = WT ? __ldg(wts + p) : 1.f;
      if (x > 0.f) acc.add(__ldg(labels + __ldg(idx + p)), x);
    }
  }
}

// Sums of both pairs of acc over the warp (every lane gets them); the two chains are
// interleaved so their latencies overlap
__device__ __forceinline__ void warp_acc_sum(ModAcc& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float kh = __shfl_xor_sync(kFullMask, a.kh, o);
    const float kl = __shfl_xor_sync(kFullMask, a.kl, o);
    const float ih = __shfl_xor_sync(kFullMask, a.ih, o);
    const float il = __shfl_xor_sync(kFullMask, a.il, o);
    two_sum_pair(a.kh, a.kl, kh, kl);
    two_sum_pair(a.ih, a.il, ih, il);
  }
}

template <bool WT, bool VEC>
__global__ void __launch_bounds__(kModThreads, 3) modularity_rows_kernel(
    const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
    const float* __restrict__ wts, int64_t m, const int32_t* __restrict__ labels, int32_t n,
    double* sigma_c, double* part_k, double* part_in) {
  __shared__ double s_k[kModThreads], s_in[kModThreads];
  __shared__ float s_h[kModThreads], s_l[kModThreads];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t ntiles = ((int64_t)n + 31) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (kModThreads / 32);
  float tkh = 0.f, tkl = 0.f, tih = 0.f, til = 0.f;  // the lane's totals
  for (int64_t t = (int64_t)blockIdx.x * (kModThreads / 32) + (tid >> 5); t < ntiles;
       t += nwarps) {
    const int64_t v = t * 32 + lane;
    const bool own = v < n;
    int64_t b = 0, e = 0;
    int cv = -1;
    if (own) {
      b = __ldg(off + v);
      e = __ldg(off + v + 1);
      cv = __ldg(labels + v);
    }
    ModAcc acc{0.f, 0.f, 0.f, 0.f, cv};
    const bool longrow = e - b > kModShortRow;
    if (own && !longrow) mod_range<WT, VEC>(acc, idx, wts, labels, m, (int)v, b, e);
    for (unsigned lm = __ballot_sync(kFullMask, longrow); lm; lm &= lm - 1) {
      const int src = __ffs(lm) - 1;
      ModAcc pa{0.f, 0.f, 0.f, 0.f, __shfl_sync(kFullMask, cv, src)};
      // lane i folds the i-th of 32 contiguous pieces of the row, cut at 4-entry group
      // boundaries so that only the row's ends are partial groups
      const int64_t rb = __shfl_sync(kFullMask, b, src), re = __shfl_sync(kFullMask, e, src);
      const int64_t g0 = rb >> 2, ng = ((re + 3) >> 2) - g0;
      int64_t pb = (g0 + (lane * ng) / 32) << 2, pe = (g0 + ((lane + 1) * ng) / 32) << 2;
      pb = pb < rb ? rb : pb;
      pe = pe > re ? re : pe;
      mod_range<WT, VEC>(pa, idx, wts, labels, m, (int)(t * 32 + src), pb, pe);
      warp_acc_sum(pa);
      if (lane == src) acc = pa;
    }
    two_sum_pair(tkh, tkl, acc.kh, acc.kl);
    two_sum_pair(tih, til, acc.ih, acc.il);
    // Sigma_c: K_i summed over each run of equal labels among the warp's rows
    float kh = acc.kh, kl = acc.kl;
    const int cp = __shfl_up_sync(kFullMask, cv, 1);
    const unsigned heads = __ballot_sync(kFullMask, lane == 0 || cp != cv);
    const int run0 = 31 - __clz(heads & lanes_upto(lane));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const float yh = __shfl_up_sync(kFullMask, kh, d);
      const float yl = __shfl_up_sync(kFullMask, kl, d);
      if (lane - d >= run0) two_sum_pair(kh, kl, yh, yl);
    }
    // run ends of the same label (runs apart in the warp) join before the atomic: a large
    // community met in several runs costs one atomic on its hot address, not several
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    const bool put = own && tail && (kh != 0.f || kl != 0.f);
    const unsigned grp = __match_any_sync(kFullMask, put ? cv : -(lane + 2));
    if (put && __popc(grp) > 1) {
      s_h[tid] = kh;
      s_l[tid] = kl;
    }
    __syncwarp();
    if (put && lane == __ffs(grp) - 1) {
      for (unsigned g = grp & (grp - 1); g; g &= g - 1) {
        const int q = (tid & ~31) + __ffs(g) - 1;
        two_sum_pair(kh, kl, s_h[q], s_l[q]);
      }
      atomicAdd(sigma_c + cv, (double)kh + (double)kl);
    }
    __syncwarp();
  }
  s_k[tid] = (double)tkh + (double)tkl;
  s_in[tid] = (double)tih + (double)til;
  __syncthreads();
  for (int h = kModThreads / 2; h > 0; h >>= 1) {
    if (tid < h) {
      s_k[tid] += s_k[tid + h];
      s_in[tid] += s_in[tid + h];
    }
    __syncthreads();
  }
  if (tid == 0) {
    part_k[blockIdx.x] = s_k[0];
    part_in[blockIdx.x] = s_in[0];
  }
}

int mod_row_blocks(int32_t n) {
  const int64_t b = (((int64_t)n + 31) / 32 + kModThreads / 32 - 1) / (kModThreads / 32);
  return (int)(b < 1 ? 1 : (b > kModMaxBlocks ? kModMaxBlocks : b));
}

int mod_sq_blocks(int32_t n) {
  const int64_t b = ((int64_t)n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > kModMaxBlocks ? kModMaxBlocks : b));
}

template <bool WT, bool VEC>
void launch_rows(const int64_t* off, const int32_t* idx, const float* w, int64_t m,
                 const int32_t* labels, int32_t n, double* sigma_c, double* part_k,
                 double* part_in, cudaStream_t s) {
  modularity_rows_kernel<WT, VEC><<<mod_row_blocks(n), kModThreads, 0, s>>>(
      off, idx, w, m, labels, n, sigma_c, part_k, part_in);
  count_launch();
}

// Batch: Q of graph g from its totals and the Sigma_c of its label range (one block per
// graph; labels of graph g lie in [vb_g, vb_g + n_g)).
__global__ void __launch_bounds__(256) batch_q_kernel(const BatchGraph* __restrict__ gs,
                                                     const double* __restrict__ sigma_c,
                                                     const double* __restrict__ g2m,
                                                     const double* __restrict__ gin, double* gq) {
  __shared__ double s[256];
  const BatchGraph G = gs[blockIdx.x];
  double acc = 0.0;
  for (int64_t c = G.vb + threadIdx.x; c < G.vb + G.n; c += 256) acc += sigma_c[c] * sigma_c[c];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double two_m = g2m[blockIdx.x];
    gq[blockIdx.x] = two_m > 0.0 ? gin[blockIdx.x] / two_m - s[0] / (two_m * two_m) : 0.0;
  }
}

}  // namespace

cudaError_t launch_batch_q(const BatchGraph* gs, int count, const double* sigma_c, const double* g2m,
                           const double* gin, double* gq, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  batch_q_kernel<<<count, 256, 0, s>>>(gs, sigma_c, g2m, gin, gq);
  count_launch();
  return cudaGetLastError();
}

int64_t modularity_plan_partials(const WarpPlan& p, int32_t n) {
  (void)p;
  (void)n;
  return 2 * (int64_t)kModSlots + kSqBlocks;
}

cudaError_t launch_modularity_plan(const int64_t* off, const int32_t* idx, const float* w,
                                   int64_t m, const int32_t* labels, int32_t n,
                                   const WarpPlan& p, double* sigma_c, double* partials,
                                   int64_t npart, double* out4, cudaStream_t s,
                                   const int32_t* gid, double* g2m, double* gin) {
  (void)npart;
  const ModGraphs mg{gid, g2m, gin};
  double* slots = partials;
  double* sq = partials + 2 * kModSlots;
  zero_f64_kernel<<<152 * 4, 256, 0, s>>>(sigma_c, n);
  count_launch();
  zero_f64_kernel<<<16, 256, 0, s>>>(slots, 2 * kModSlots);
  count_launch();
  (void)off;
  for (int c = 0; c < kHubClasses; ++c) {
    const int cnt = p.hub_start[c + 1] - p.hub_start[c];
    if (cnt <= 0) continue;
    WarpPlan q = p;
    q.hub_desc = p.hub_desc + p.hub_start[c];
    q.hub_base = p.hub_base + p.hub_start[c];
    auto kern = p.wfmt == kSplitW ? modularity_hub_kernel<kSplitW> : modularity_hub_kernel<kUnitW>;
    kern<<<cnt, kThreads >> c, 0, s>>>(idx, w, m, labels, q, sigma_c, slots, mg);
    count_launch();
  }
  const int64_t lane_ctas = (p.nlanes + kLaneThreads - 1) / kLaneThreads;
  if (lane_ctas > 0) {
    auto kern = p.wfmt == kSplitW ? modularity_lane_kernel<kSplitW> : modularity_lane_kernel<kUnitW>;
    kern<<<(unsigned)lane_ctas, kLaneThreads, 0, s>>>(idx, w, m, labels, p, sigma_c, slots, mg);
    count_launch();
  }
  sigma_sq_kernel<<<kSqBlocks, 256, 0, s>>>(sigma_c, n, sq);
  count_launch();
  modularity_total_kernel<<<1, 256, 0, s>>>(slots, slots + 1, 2, kModSlots, sq, kSqBlocks,
                                             out4);
  count_launch();
  return cudaGetLastError();
}

int modularity_partials(int32_t n) {
  const int r = mod_row_blocks(n), q = mod_sq_blocks(n);
  return r > q ? r : q;
}

cudaError_t launch_modularity(const int64_t* off, const int32_t* idx, const float* w, int64_t m,
                              const int32_t* labels, int32_t n, double* sigma_c,
                              double* partials, int32_t npart, double* out4, cudaStream_t s) {
  double* part_k = partials;
  double* part_in = partials + npart;
  double* sq = partials + 2 * (int64_t)npart;
  int nr = 0, nq = 0;
  if (n > 0) {
    const int64_t zb = ((int64_t)n + 255) / 256;
    zero_f64_kernel<<<(unsigned)(zb < 152 * 8 ? zb : 152 * 8), 256, 0, s>>>(sigma_c, n);
    count_launch();
    const bool vec = ((uintptr_t)idx & 15) == 0 && ((uintptr_t)w & 15) == 0;
    if (w != nullptr && vec) launch_rows<true, true>(off, idx, w, m, labels, n, sigma_c, part_k, part_in, s);
    else if (w != nullptr) launch_rows<true, false>(off, idx, w, m, labels, n, sigma_c, part_k, part_in, s);
    else if (vec) launch_rows<false, true>(off, idx, w, m, labels, n, sigma_c, part_k, part_in, s);
    else launch_rows<false, false>(off, idx, w, m, labels, n, sigma_c, part_k, part_in, s);
    nr = mod_row_blocks(n);
    nq = mod_sq_blocks(n);
    sigma_sq_kernel<<<nq, 256, 0, s>>>(sigma_c, n, sq);
    count_launch();
  }
  modularity_total_kernel<<<1, 256, 0, s>>>(part_k, part_in, 1, nr, sq, nq, out4);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lpa
