// lpa_modularity.cu -- modularity (Sec. 3.2, Eq. 1) over the binned graph of a run:
// Q = sum_c sigma_c / 2m - sum_c (Sigma_c / 2m)^2, accumulated in fp64.
//
// The rows pass reuses the sweep's work map (hub kernels per CTA-size class, packed lane
// descriptors) and its pipelined row reads, so it streams the CSR at the sweep's rate.
// Per vertex it forms K_i (all entries, self-loops included, as stored) and the weight of
// entries whose neighbour shares the label; Sigma_c receives K_i through one atomic per
// run of equal labels in a warp.  Block sums go to kModSlots accumulators.
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
template <bool WT>
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
  if (v >= 0) {
    acc.cv = labels[v];
    fold_range<ModAcc, WT, false>(acc, idx, wts, labels, m, v, lo, lo + len);
  }
  double kv = acc.k(), in = acc.in();
  const int Lw = __reduce_max_sync(kFullMask, L);
  if (Lw > 1) {
    kv = warp_down_sum(kv, L, Lw);
    in = warp_down_sum(in, L, Lw);
  }
  mod_commit(v >= 0 && leaf == 0, v, acc.cv, kv, in, sigma_c, slots, s_k, s_in, mg);
}

// Hubs of one class (p.hub_desc points at the class): the row split evenly over the CTA.
template <bool WT>
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
  ModAcc acc{0.f, 0.f, 0.f, 0.f, labels[v]};
  fold_range<ModAcc, WT, false>(acc, idx, wts, labels, m, v, base + (tid * d) / nt,
                                base + ((tid + 1) * d) / nt);
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

// Fixed-order final sums; out4 = {2m, intra weight, sum_c Sigma_c^2, Q}.
__global__ void __launch_bounds__(256) modularity_total_kernel(const double* slots,
                                                              const double* sq, double* out4) {
  __shared__ double sa[256], sb[256], sc[256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < kModSlots; i += 256) {
    a += slots[2 * i];
    b += slots[2 * i + 1];
  }
  for (int i = threadIdx.x; i < kSqBlocks; i += 256) c += sq[i];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sa[threadIdx.x] += sa[threadIdx.x + h];
      sb[threadIdx.x] += sb[threadIdx.x + h];
      sc[threadIdx.x] += sc[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double two_m = sa[0];
    out4[0] = two_m;
    out4[1] = sb[0];
    out4[2] = sc[0];
    out4[3] = two_m > 0.0 ? sb[0] / two_m - sc[0] / (two_m * two_m) : 0.0;
  }
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
    if (w)
      modularity_hub_kernel<true><<<cnt, kThreads >> c, 0, s>>>(idx, w, m, labels, q, sigma_c, slots, mg);
    else
      modularity_hub_kernel<false><<<cnt, kThreads >> c, 0, s>>>(idx, w, m, labels, q, sigma_c, slots, mg);
    count_launch();
  }
  const int64_t lane_ctas = (p.nlanes + kLaneThreads - 1) / kLaneThreads;
  if (lane_ctas > 0) {
    if (w)
      modularity_lane_kernel<true><<<(unsigned)lane_ctas, kLaneThreads, 0, s>>>(idx, w, m, labels, p,
                                                                               sigma_c, slots, mg);
    else
      modularity_lane_kernel<false><<<(unsigned)lane_ctas, kLaneThreads, 0, s>>>(idx, w, m, labels, p,
                                                                                sigma_c, slots, mg);
    count_launch();
  }
  sigma_sq_kernel<<<kSqBlocks, 256, 0, s>>>(sigma_c, n, sq);
  count_launch();
  modularity_total_kernel<<<1, 256, 0, s>>>(slots, sq, out4);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lpa
