// lpa_setup.cu -- everything around the sweep: CSR validation, degree binning into
// chunks and hubs, label initialisation and the on-device convergence test (Alg. 1,
// `lpa`).
#include <algorithm>

#include "lpa_internal.cuh"

namespace lpa {
namespace {

constexpr int kScanThreads = 1024;

// ------------------------------------------------------------------ validation

__global__ void validate_offsets_kernel(const int64_t* off, int32_t n, int64_t m, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
    bool bad = false;
    if (v == 0 && off[0] != 0) bad = true;
    if (v == n && off[n] != m) bad = true;
    if (v < n && off[v + 1] < off[v]) bad = true;
    if (bad) atomicOr(err, kErrOffsets);
  }
}

__global__ void validate_edges_kernel(const int32_t* idx, const float* w, int32_t n, int64_t m,
                                      const int32_t* labels_in, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bits = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int32_t j = idx[e];
    if (j < 0 || j >= n) bits |= kErrIndex;
    if (w) {
      const float x = w[e];
      if (!(x >= 0.f) || isinf(x)) bits |= kErrWeight;  // !(x >= 0) also catches NaN
    }
  }
  if (labels_in)
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
      const int32_t c = labels_in[v];
      if (c < 0 || c >= n) bits |= kErrLabels;
    }
  if (bits) atomicOr(err, bits);
}

// ------------------------------------------------------------------ binning

// Greedy chunking of one segment of vertices.  A vertex is a hub if its row exceeds a
// chunk (d > cap) or it has more leaves than a warp has lanes.  Other vertices join the
// current chunk while its cost stays <= cap, with cost = max(d, floor * L, floor):
// so a chunk holds <= cap edges and <= cap / floor = kThreads vertices and leaves.
template <bool WRITE>
__device__ void greedy_segment(const BinArgs& b, int64_t seg, int64_t& nch, int64_t& nhub,
                               int64_t& hub_edges) {
  const int64_t v_begin = seg * kSegment;
  const int64_t v_end = min((int64_t)b.n, v_begin + kSegment);
  int64_t ch_out = WRITE ? b.seg_chunks[seg] : 0;
  int64_t hub_out = WRITE ? b.seg_hubs[seg] : 0;
  int64_t tab_out = WRITE ? 2 * b.seg_hub_edges[seg] : 0;
  nch = 0;
  nhub = 0;
  hub_edges = 0;
  int64_t cur_start = -1, cur_cost = 0;
  int64_t o_next = b.off[v_begin];
  for (int64_t v = v_begin; v < v_end; ++v) {
    const int64_t o = o_next;
    o_next = b.off[v + 1];
    const int64_t d = o_next - o;
    const int L = b.leaves ? leaf_count(d, b.e0, b.lmax) : 1;
    if (d > b.cap || L > kMaxWarpLeaves) {
      if (cur_start >= 0) {
        if (WRITE) {
          b.chunk_v0[ch_out] = (int32_t)cur_start;
          b.chunk_v1[ch_out] = (int32_t)v;
          ++ch_out;
        }
        ++nch;
        cur_start = -1;
      }
      if (WRITE) {
        b.hubs[hub_out] = (int32_t)v;
        if (b.hub_tab) b.hub_tab[hub_out] = tab_out;
        ++hub_out;
        tab_out += 2 * d;
      }
      ++nhub;
      hub_edges += d;
      continue;
    }
    int64_t cost = d;
    if (cost < (int64_t)b.cost_floor * L) cost = (int64_t)b.cost_floor * L;
    if (cur_start >= 0 && cur_cost + cost > b.cap) {
      if (WRITE) {
        b.chunk_v0[ch_out] = (int32_t)cur_start;
        b.chunk_v1[ch_out] = (int32_t)v;
        ++ch_out;
      }
      ++nch;
      cur_start = -1;
    }
    if (cur_start < 0) {
      cur_start = v;
      cur_cost = 0;
    }
    cur_cost += cost;
  }
  if (cur_start >= 0) {
    if (WRITE) {
      b.chunk_v0[ch_out] = (int32_t)cur_start;
      b.chunk_v1[ch_out] = (int32_t)v_end;
    }
    ++nch;
  }
}

__global__ void bin_count_kernel(BinArgs b, int64_t nseg) {
  const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (seg >= nseg) return;
  int64_t c, h, he;
  greedy_segment<false>(b, seg, c, h, he);
  b.seg_chunks[seg] = c;
  b.seg_hubs[seg] = h;
  b.seg_hub_edges[seg] = he;
}

__global__ void bin_write_kernel(BinArgs b, int64_t nseg) {
  const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (seg >= nseg) return;
  int64_t c, h, he;
  greedy_segment<true>(b, seg, c, h, he);
}

// Exclusive prefix sums of three int64 arrays (one block); totals go to the state.
__global__ void __launch_bounds__(kScanThreads) scan3_kernel(int64_t* a, int64_t* b, int64_t* c,
                                                             int64_t len, DevState* st) {
  __shared__ int64_t sa[kScanThreads], sb[kScanThreads], sc[kScanThreads];
  const int tid = threadIdx.x;
  const int64_t per = (len + kScanThreads - 1) / kScanThreads;
  const int64_t lo = min(len, tid * per), hi = min(len, lo + per);
  int64_t ta = 0, tb = 0, tc = 0;
  for (int64_t i = lo; i < hi; ++i) {
    ta += a[i];
    tb += b[i];
    tc += c[i];
  }
  sa[tid] = ta;
  sb[tid] = tb;
  sc[tid] = tc;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {  // Hillis-Steele inclusive scan
    int64_t xa = 0, xb = 0, xc = 0;
    if (tid >= o) {
      xa = sa[tid - o];
      xb = sb[tid - o];
      xc = sc[tid - o];
    }
    __syncthreads();
    sa[tid] += xa;
    sb[tid] += xb;
    sc[tid] += xc;
    __syncthreads();
  }
  int64_t ra = sa[tid] - ta, rb = sb[tid] - tb, rc = sc[tid] - tc;
  for (int64_t i = lo; i < hi; ++i) {
    const int64_t xa = a[i], xb = b[i], xc = c[i];
    a[i] = ra;
    b[i] = rb;
    c[i] = rc;
    ra += xa;
    rb += xb;
    rc += xc;
  }
  if (tid == kScanThreads - 1) {
    st->nchunks = sa[tid];
    st->nhubs = sb[tid];
    st->hub_edges = sc[tid];
  }
}

// ------------------------------------------------- binning for the warp sweep

// Sort key of a vertex with d positions inside its window: its class c < kHubClasses for a
// hub; kHubClasses + c for mid class c (larger L and longer leaves first); for a one-leaf
// row kHubClasses + kMidClasses + (kLowKeys - 1 - min(d, kLowKeys - 1)), so the rows of a
// warp have (nearly) the same number of groups in the sliced copy (longer rows first).
__device__ __forceinline__ int window_key(int64_t d, int e0, int lmax) {
  const int L = leaf_count(d, e0, lmax);
  if (d > kHubDegree || L > kMaxWarpLeaves)  // hub class c: CTA of 256 >> c threads
    return L >= 256 ? 0 : (L == 128 ? 1 : (L == 64 ? 2 : 3));
  if (L == 1)
    return kHubClasses + kMidClasses + (kLowKeys - 1 - (int)(d < kLowKeys ? d : kLowKeys - 1));
  const int lidx = 5 - (31 - __clz(L));  // L = 32 -> 0 ... L = 2 -> 4
  int sub = (int)(((d / L) * 4) / e0) - 4;  // leaf length quarter in [e0, 2 e0)
  sub = sub < 0 ? 0 : (sub > kMidSub - 1 ? kMidSub - 1 : sub);
  return kHubClasses + lidx * kMidSub + (kMidSub - 1 - sub);
}

constexpr int kSortThreads = 1024;
constexpr int kSortPad = 2 * kSortThreads;  // scan space: two keys per thread
static_assert(kSortKeys <= kSortPad, "sort keys exceed the scan space");

// One CTA per window of `win` vertices: counting sort of the window's vertices by
// window_key, writing each slot's descriptor {v, offset lo, offset hi, degree}, the window
// table, the window's hub count and its lane count rounded up to whole warps.  Order
// inside one key does not matter.
__global__ void __launch_bounds__(kSortThreads) window_sort_kernel(
    const int64_t* off, int32_t n, int e0, int lmax, int win, int32_t w_first, int64_t hstride,
    int4* desc, int32_t* wtab, int32_t* hcnt, int32_t* lcnt) {
  __shared__ int s_hist[kSortPad];
  __shared__ int s_wsum[kSortThreads / 32];
  __shared__ int s_grp[kHubClasses + kLaneGroups];  // hub classes, mid classes, low rows
  constexpr int kPer = kWinVerts / kSortThreads;
  const int tid = threadIdx.x;
  for (int i = tid; i < kSortPad; i += kSortThreads) s_hist[i] = 0;
  __syncthreads();
  const int64_t wi = (int64_t)w_first + blockIdx.x;  // the window this CTA sorts
  const int64_t v0 = wi * win;
  int key[kPer];
  int64_t b[kPer];
  int d[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int64_t v = v0 + tid + q * kSortThreads;
    key[q] = -1;
    if (tid + q * kSortThreads < win && v < n) {
      b[q] = off[v];
      const int64_t dd = off[v + 1] - b[q];
      d[q] = (int)dd;  // rows above INT32_MAX are refused after binning
      key[q] = window_key(dd, e0, lmax);
      atomicAdd(&s_hist[key[q]], 1);
    }
  }
  __syncthreads();
  if (tid < kHubClasses + kLaneGroups) {
    int c = 0;
    if (tid < kHubClasses + kMidClasses) {
      c = s_hist[tid];
    } else {
      for (int k = kHubClasses + kMidClasses; k < kSortKeys; ++k) c += s_hist[k];
    }
    s_grp[tid] = c;
  }
  // exclusive scan of the histogram, keys 2t and 2t+1 owned by thread t
  const int x0 = s_hist[2 * tid], x1 = s_hist[2 * tid + 1];
  int incl = x0 + x1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((tid & 31) >= o) incl += y;
  }
  if ((tid & 31) == 31) s_wsum[tid >> 5] = incl;
  __syncthreads();
  int wpre = 0;
  for (int w = 0; w < (tid >> 5); ++w) wpre += s_wsum[w];
  const int ex = wpre + incl - x0 - x1;
  s_hist[2 * tid] = ex;
  s_hist[2 * tid + 1] = ex + x0;
  if (tid == 0) {
    int32_t* t = wtab + wi * kWinTab;
    int nh = 0;
    for (int c = 0; c < kHubClasses; ++c) {
      t[kTabHub + c] = nh;
      hcnt[(int64_t)c * hstride + wi] = s_grp[c];
      nh += s_grp[c];
    }
    int lanes = 0, slot = nh;
    for (int g = 0; g < kLaneGroups; ++g) {
      t[kTabLane + g] = lanes;
      t[kTabVert + g] = slot;
      const int cnt = s_grp[kHubClasses + g];
      lanes += cnt * (g < kMidClasses ? 32 >> (g / kMidSub) : 1);
      slot += cnt;
    }
    t[0] = nh;
    t[kTabLanes] = lanes;
    lcnt[wi] = (lanes + 31) & ~31;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (key[q] < 0) continue;
    const int64_t v = v0 + tid + q * kSortThreads;
    const int pos = atomicAdd(&s_hist[key[q]], 1);
    desc[v0 + pos] = make_int4((int)v, (int)(uint32_t)(b[q] & 0xffffffffLL), (int)(b[q] >> 32), d[q]);
  }
}

// Exclusive prefix sum of len int32 counts into int64 prefix[0, len]; prefix[len] = total.
__global__ void __launch_bounds__(kScanThreads) scan_counts_kernel(const int32_t* cnt, int64_t len,
                                                                   int64_t* prefix) {
  __shared__ int64_t sv[kScanThreads];
  const int tid = threadIdx.x;
  const int64_t per = (len + kScanThreads - 1) / kScanThreads;
  const int64_t lo = min(len, tid * per), hi = min(len, lo + per);
  int64_t t = 0;
  for (int64_t i = lo; i < hi; ++i) t += cnt[i];
  sv[tid] = t;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {  // Hillis-Steele inclusive scan
    const int64_t x = tid >= o ? sv[tid - o] : 0;
    __syncthreads();
    sv[tid] += x;
    __syncthreads();
  }
  int64_t r = sv[tid] - t;
  for (int64_t i = lo; i < hi; ++i) {
    prefix[i] = r;
    r += cnt[i];
  }
  if (tid == kScanThreads - 1) prefix[len] = sv[tid];
}

// Multi-CTA exclusive scan for long count arrays: tiles of kScanTile counts; pass 1 sums
// each tile, scan_counts_kernel scans the tile sums, pass 2 scans each tile through
// shared memory (coalesced loads and stores) and adds its tile's base.
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t* warp_sums,
                                                        int64_t* total) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t w = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + incl - x;
  if (total) *total = warp_sums[31];
  return before;
}

__global__ void __launch_bounds__(kScanThreads) tile_sum_kernel(const int32_t* cnt, int64_t len,
                                                                int64_t* sums) {
  __shared__ int64_t ws[32];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  int64_t x = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    const int64_t i = t0 + q * kScanThreads + threadIdx.x;
    if (i < len) x += cnt[i];
  }
  int64_t total = 0;
  block_exclusive_scan(x, ws, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const int32_t* cnt, int64_t len,
                                                                 const int64_t* tile_base,
                                                                 int64_t* prefix) {
  __shared__ int32_t sc[kScanTile];
  __shared__ int64_t ws[32];
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {  // coalesced load of the tile
    const int64_t i = t0 + q * kScanThreads + threadIdx.x;
    sc[q * kScanThreads + threadIdx.x] = i < len ? cnt[i] : 0;
  }
  __syncthreads();
  int32_t v[kScanPer];
  int64_t x = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = sc[threadIdx.x * kScanPer + q];
    x += v[q];
  }
  int64_t r = tile_base[blockIdx.x] + block_exclusive_scan(x, ws, nullptr);
  __syncthreads();
  int64_t* out = reinterpret_cast<int64_t*>(sc);  // the tile's prefixes, half a tile at a time
  for (int half = 0; half < 2; ++half) {
    const int lo = half * (kScanThreads / 2);
    if (threadIdx.x >= lo && threadIdx.x < lo + kScanThreads / 2) {
      int64_t rr = r;
#pragma unroll
      for (int q = 0; q < kScanPer; ++q) {
        out[(threadIdx.x - lo) * kScanPer + q] = rr;
        rr += v[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kScanPer / 2; ++q) {  // coalesced store
      const int e = q * kScanThreads + threadIdx.x;
      const int64_t i = t0 + (int64_t)lo * kScanPer + e;
      if (i < len) prefix[i] = out[e];
    }
    __syncthreads();
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) prefix[len] = tile_base[gridDim.x];
}

// In-place exclusive prefix of len int64 values (len <= kScanThreads * kScanPer * 64 in
// practice: tile sums), a[len] = total.
__global__ void __launch_bounds__(kScanThreads) scan_i64_kernel(int64_t* a, int64_t len) {
  __shared__ int64_t ws[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < len; b0 += kScanThreads) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t x = i < len ? a[i] : 0;
    int64_t total = 0;
    const int64_t ex = block_exclusive_scan(x, ws, &total);
    const int64_t c = carry;
    if (i < len) a[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) a[len] = carry;
}

// One CTA per window: copy the window's hub descriptors to hub_desc[hub_prefix[w] + i]
// and write one lane descriptor per packed lane to lane_desc[lane_prefix[w] + q]:
// {v, leaf start lo, leaf start hi, leaf length | leaf << kLaneLeafShift | log2 L <<
// kLaneLgShift}, v = -1 for the padding lanes.  Writes past the capacities are skipped
// (the host then refuses the plan).
__global__ void __launch_bounds__(kSortThreads) expand_lanes_kernel(
    const int4* desc, const int32_t* wtab, const int64_t* hub_prefix, const int64_t* lane_prefix,
    int win, int64_t hstride, int32_t w_lanes, int4* hub_desc, int64_t hub_cap, int4* lane_desc,
    int64_t lane_cap) {
  __shared__ int32_t t[kWinTab];
  const int tid = threadIdx.x;
  const int64_t wi = blockIdx.x;
  if (tid < kWinTab) t[tid] = wtab[wi * kWinTab + tid];
  __syncthreads();
  const int4* wd = desc + blockIdx.x * (int64_t)win;
  const int nh = t[0];
  for (int i = tid; i < nh; i += kSortThreads) {
    int c = kHubClasses - 1;  // the class whose slots hold i
    while (c > 0 && t[kTabHub + c] > i) --c;
    const int64_t pos = hub_prefix[(int64_t)c * hstride + wi] + (i - t[kTabHub + c]);
    if (pos < hub_cap) hub_desc[pos] = wd[i];
  }
  if (wi < w_lanes) return;  // lanes of this window are kept from an earlier binning
  const int lanes = t[kTabLanes];
  const int64_t l0 = lane_prefix[wi];
  const int padded = (int)(lane_prefix[wi + 1] - l0);
  for (int q = tid; q < padded; q += kSortThreads) {
    if (l0 + q >= lane_cap) break;
    int4 out = make_int4(-1, 0, 0, 0);
    if (q < lanes) {
      int g = 0;  // last lane group whose first lane is <= q (first lanes ascend)
      for (int h = 16; h > 0; h >>= 1)
        if (g + h < kLaneGroups && t[kTabLane + g + h] <= q) g += h;
      const int lg = g < kMidClasses ? 5 - g / kMidSub : 0;
      const int r = q - t[kTabLane + g];
      const int L = 1 << lg, leaf = r & (L - 1);
      const int4 dv = wd[t[kTabVert + g] + (r >> lg)];
      const int64_t b = (int64_t)(uint32_t)dv.y | ((int64_t)dv.z << 32);
      const int64_t d = dv.w;
      const int64_t lo = b + (leaf * d) / L, hi = b + ((leaf + 1) * d) / L;
      out = make_int4(dv.x, (int)(uint32_t)(lo & 0xffffffffLL), (int)(lo >> 32),
                      (int)(hi - lo) | (leaf << kLaneLeafShift) | (lg << kLaneLgShift));
    }
    lane_desc[l0 + q] = out;
  }
}

// Profile of the weights and rows: out[0] stays 1 if every weight is an integer, out[1]
// gets the largest weight's bits and out[2] the longest row (w null: rows only).  The plan
// calls it with w null and refuses rows longer than 2^31 - 1.
__global__ void weight_profile_kernel(const int64_t* off, const float* w, int32_t n, int64_t m,
                                      unsigned long long* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool integral = true;
  unsigned wmax = 0;
  long long dmax = 0;
  if (w)
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
      const float x = w[e];
      integral = integral && (x == truncf(x));
      // weights are >= 0 (or -0): without the sign bit, bit order = value order
      const unsigned bits = __float_as_uint(x) & 0x7fffffffu;
      wmax = bits > wmax ? bits : wmax;
    }
  else
    wmax = __float_as_uint(1.f);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const long long d = off[v + 1] - off[v];
    dmax = d > dmax ? d : dmax;
  }
  if (!__all_sync(0xffffffffu, integral) && (threadIdx.x & 31) == 0) atomicAnd(out, 0ull);
  unsigned wm = wmax;
  long long dm = dmax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned a = __shfl_down_sync(0xffffffffu, wm, o);
    const long long b = __shfl_down_sync(0xffffffffu, dm, o);
    wm = a > wm ? a : wm;
    dm = b > dm ? b : dm;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + 1, (unsigned long long)wm);
    atomicMax(out + 2, (unsigned long long)dm);
  }
}

// ------------------------------------------------------------ driver helpers

__global__ void init_labels_kernel(int32_t* c, const int32_t* labels_in, int32_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    c[v] = labels_in ? labels_in[v] : (int32_t)v;
}

// Convergence test after sweep l (Alg. 1): dN is the sum of the sweep's counters; stop
// iff pick-less was off and dN/N < tau.
__global__ void converge_kernel(DevState* st, const unsigned long long* dn,
                                unsigned long long* dn_total, const unsigned long long* scanned,
                                unsigned long long* scan_total, int l, int pick_less, double tol,
                                int32_t n) {
  if (threadIdx.x != 0 || st->done) return;
  unsigned long long tot = 0;
  for (int i = 0; i < kDnSlots; ++i) tot += dn[(int64_t)l * kDnSlots + i];
  dn_total[l] = tot;
  if (scanned) {
    unsigned long long sc = 0;
    for (int i = 0; i < kDnSlots; ++i) sc += scanned[(int64_t)l * kDnSlots + i];
    scan_total[l] = sc;
  }
  st->iterations = l + 1;
  if (!pick_less && (double)tot / (double)n < tol) {
    st->done = 1;
    st->converged = 1;
  }
}

__global__ void dn_sum_kernel(const unsigned long long* slots, unsigned long long* out) {
  if (threadIdx.x != 0) return;
  unsigned long long tot = 0;
  for (int i = 0; i < kDnSlots; ++i) tot += slots[i];
  *out = tot;
}

// Iteration l writes buffer (l+1) & 1; buffer 0 is the caller's output.
__global__ void finalize_kernel(const DevState* st, int32_t* out, const int32_t* tmp, int32_t n) {
  if ((st->iterations & 1) == 0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    out[v] = tmp[v];
}

__global__ void fill_i32_kernel(int32_t* p, int32_t value, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) p[i] = value;
}

__global__ void fill_u8_kernel(uint8_t* p, uint8_t value, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    p[i] = value;
}

__global__ void fill_u64_kernel(unsigned long long* p, unsigned long long value, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) p[i] = value;
}

// ------------------------------------------------- sliced copy of the CSR

// Pass 1: the groups of each lane warp's slice (the sum of its lanes' ceil(len / 4)), for
// lane warps w_from .. nlanes / 32 - 1, and of each hub's slice (L leaves x the groups of
// its longest leaf).
__global__ void __launch_bounds__(256) slice_count_kernel(const int4* __restrict__ lane_desc,
                                                         int64_t lane_from, int64_t nlanes,
                                                         const int4* __restrict__ hub_desc,
                                                         int32_t nhubs, int e0, int lmax,
                                                         int32_t* lane_cnt, int32_t* hub_cnt) {
  const int64_t span = ((nlanes - lane_from + 255) >> 8) << 8;  // lane threads, whole CTAs
  const int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t q = lane_from + t;
  if (t < span && q < nlanes) {  // whole warps: lane_from and nlanes are multiples of 32
    const int4 l = __ldg(lane_desc + q);
    const int g = l.x >= 0 ? ((l.w & ((1 << kLaneLeafShift) - 1)) + 3) >> 2 : 0;
    const int sum = __reduce_add_sync(0xffffffffu, g);
    if ((threadIdx.x & 31) == 0) lane_cnt[(q - lane_from) >> 5] = sum;
  }
  const int64_t h = t - span;  // hubs after the lane CTAs
  if (h >= 0 && h < nhubs) {
    const int64_t d = __ldg(hub_desc + h).w;
    const int L = leaf_count(d, e0, lmax);
    hub_cnt[h] = (int32_t)(L * hub_leaf_groups(d, L));
  }
}

// base[w_from + i] = base[w_from] + scan[i] for i <= len (base[0] = 0 when w_from = 0):
// the lane warps from w_from on continue after the kept ones.
__global__ void lane_base_kernel(const int64_t* scan, int64_t len, int64_t w_from, int64_t* base) {
  const int64_t start = w_from > 0 ? base[w_from] : 0;  // unchanged by this kernel
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= len; i += stride)
    if (i > 0 || w_from == 0) base[w_from + i] = start + scan[i];
}

// Hub slices fill the top of the sliced copy downwards: hub h starts at
// cap - total + pre[h], so lanes can grow from the bottom without moving them.
__global__ void hub_base_kernel(const int64_t* pre, int32_t nhubs, int64_t cap, int64_t* hub_base) {
  const int64_t total = pre[nhubs];
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nhubs;
       h += (int64_t)gridDim.x * blockDim.x)
    hub_base[h] = cap - total + pre[h];
}

// The aligned block of four CSR positions starting at a (a multiple of 4); positions at
// or past m come back as 0.
__device__ __forceinline__ int4 load_block(const int32_t* __restrict__ a32, int64_t a, int64_t m) {
  if (a + 3 < m) return __ldg(reinterpret_cast<const int4*>(a32 + a));
  int r[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) r[u] = a + u < m ? __ldg(a32 + a + u) : 0;
  return make_int4(r[0], r[1], r[2], r[3]);
}

// Positions sh .. sh + 3 of the eight in (lo, hi).
__device__ __forceinline__ int4 funnel(const int4& lo, const int4& hi, int sh) {
  switch (sh) {
    case 0: return lo;
    case 1: return make_int4(lo.y, lo.z, lo.w, hi.x);
    case 2: return make_int4(lo.z, lo.w, hi.x, hi.y);
    default: return make_int4(lo.w, hi.x, hi.y, hi.z);
  }
}

// One group of the sliced copy at element p from positions u < valid of the leaf
// (indices j, weight bits x); an index of -1 marks what no vote comes from: a self-loop,
// a weight that is not positive, and the padding past the leaf's end (weight 0).
template <int WF>
__device__ __forceinline__ void store_group(const int (&j)[4], const int (&x)[4], int64_t valid,
                                            int self, int4* si, float4* sw, int64_t p) {
  int jo[4];
  float xo[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    xo[u] = u < valid ? (WF != kUnitW ? __int_as_float(x[u]) : 1.f) : 0.f;
    jo[u] = (u < valid && j[u] != self && xo[u] > 0.f) ? j[u] : -1;
  }
  si[p] = make_int4(jo[0], jo[1], jo[2], jo[3]);
  if (WF == kSplitW) sw[p] = make_float4(xo[0], xo[1], xo[2], xo[3]);
}

// Pass 2, lane warps: each lane copies its leaf into the columns of its warp's slice,
// reading its positions as aligned 16-byte blocks (each block once) and shifting them
// into groups that start at the leaf's first position.
template <int WF>
__global__ void __launch_bounds__(256) slice_fill_lanes_kernel(
    const int32_t* __restrict__ idx, const float* __restrict__ w, int64_t m,
    const int4* __restrict__ lane_desc, int64_t lane_from, int64_t nlanes,
    const int64_t* __restrict__ base, int4* si, float4* sw) {
  constexpr bool WT = WF != kUnitW;
  const int64_t t = lane_from + (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (t >= nlanes) return;  // whole warps
  const int lane = threadIdx.x & 31;
  const int4 l = __ldg(lane_desc + t);
  const int v = l.x;
  const int64_t lo = (int64_t)(uint32_t)l.y | ((int64_t)l.z << 32);
  const int64_t len = v >= 0 ? (l.w & ((1 << kLaneLeafShift) - 1)) : 0;
  const int ng = (int)((len + 3) >> 2);
  const int iters = __reduce_max_sync(0xffffffffu, ng);
  const int64_t a0 = lo & ~(int64_t)3;
  const int sh = (int)(lo & 3);
  const int32_t* wi = reinterpret_cast<const int32_t*>(w);
  int4 bi = make_int4(0, 0, 0, 0), bw = make_int4(0, 0, 0, 0);
  if (ng > 0) {
    bi = load_block(idx, a0, m);
    if (WT) bw = load_block(wi, a0, m);
  }
  int64_t col = base[t >> 5];
  for (int k = 0; k < iters; ++k) {
    const unsigned has = __ballot_sync(0xffffffffu, ng > k);
    if (ng > k) {
      int4 ni = make_int4(0, 0, 0, 0), nw = make_int4(0, 0, 0, 0);
      if (sh != 0 && 4 * (k + 1) < sh + len) {  // the next block holds part of group k
        ni = load_block(idx, a0 + 4 * (k + 1), m);
        if (WT) nw = load_block(wi, a0 + 4 * (k + 1), m);
      }
      int4 gi = funnel(bi, ni, sh), gw = funnel(bw, nw, sh);
      const int64_t valid = len - 4 * k;
      const int j[4] = {gi.x, gi.y, gi.z, gi.w};
      const int x[4] = {gw.x, gw.y, gw.z, gw.w};
      const int64_t p = col + __popc(has & ((1u << lane) - 1u));
      store_group<WF>(j, x, valid, v, si, sw, p);
      if (sh != 0) {
        bi = ni;
        bw = nw;
      } else if (ng > k + 1) {
        bi = load_block(idx, a0 + 4 * (k + 1), m);
        if (WT) bw = load_block(wi, a0 + 4 * (k + 1), m);
      }
    }
    col += __popc(has);
  }
}

// Pass 2, hubs: a CTA per hub, leaf t on thread t, read as aligned blocks as above.
template <int WF>
__global__ void __launch_bounds__(kThreads) slice_fill_hubs_kernel(
    const int32_t* __restrict__ idx, const float* __restrict__ w, int64_t m,
    const int4* __restrict__ hub_desc, const int64_t* __restrict__ base, int e0, int lmax,
    int4* si, float4* sw) {
  constexpr bool WT = WF != kUnitW;
  const int4 h = __ldg(hub_desc + blockIdx.x);
  const int64_t b = (int64_t)(uint32_t)h.y | ((int64_t)h.z << 32);
  const int64_t d = h.w;
  const int L = leaf_count(d, e0, lmax);
  const int64_t G = hub_leaf_groups(d, L);
  const int W = L < 32 ? L : 32;
  const int32_t* wi = reinterpret_cast<const int32_t*>(w);
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    const int64_t lo = b + (t * d) / L, len = b + ((t + 1) * d) / L - lo;
    const int64_t first = base[blockIdx.x] + (int64_t)(t >> 5) * W * G + (t & 31);
    const int64_t a0 = lo & ~(int64_t)3;
    const int sh = (int)(lo & 3);
    int4 bi = make_int4(0, 0, 0, 0), bw = make_int4(0, 0, 0, 0);
    if (len > 0) {
      bi = load_block(idx, a0, m);
      if (WT) bw = load_block(wi, a0, m);
    }
    for (int64_t k = 0; k < G; ++k) {
      const int64_t valid = len - 4 * k;
      int4 ni = make_int4(0, 0, 0, 0), nw = make_int4(0, 0, 0, 0);
      if (4 * (k + 1) < sh + len) {  // the next block holds positions of the leaf
        ni = load_block(idx, a0 + 4 * (k + 1), m);
        if (WT) nw = load_block(wi, a0 + 4 * (k + 1), m);
      }
      const int4 gi = funnel(bi, ni, sh), gw = funnel(bw, nw, sh);
      const int j[4] = {gi.x, gi.y, gi.z, gi.w};
      const int x[4] = {gw.x, gw.y, gw.z, gw.w};
      store_group<WF>(j, x, valid, h.x, si, sw, first + k * W);
      bi = ni;
      bw = nw;
    }
  }
}

inline unsigned grid_for(int64_t work, int threads, unsigned cap = 152 * 16) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  return (unsigned)(g < cap ? g : cap);
}

}  // namespace

cudaError_t launch_validate(const int64_t* off, const int32_t* idx, const float* w, int32_t n,
                            int64_t m, const int32_t* labels_in, int32_t* err, cudaStream_t s) {
  validate_offsets_kernel<<<grid_for((int64_t)n + 1, 256), 256, 0, s>>>(off, n, m, err);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  validate_edges_kernel<<<grid_for(m > n ? m : n, 256), 256, 0, s>>>(idx, w, n, m, labels_in, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bin(const BinArgs& b, DevState* st, cudaStream_t s, bool write_pass) {
  const int64_t nseg = num_segments(b.n);
  if (nseg == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((nseg + 127) / 128);
  if (!write_pass) {
    bin_count_kernel<<<grid, 128, 0, s>>>(b, nseg);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scan3_kernel<<<1, kScanThreads, 0, s>>>(b.seg_chunks, b.seg_hubs, b.seg_hub_edges, nseg, st);
    count_launch();
    return cudaGetLastError();
  }
  bin_write_kernel<<<grid, 128, 0, s>>>(b, nseg);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_init_labels(int32_t* c, const int32_t* labels_in, int32_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  init_labels_kernel<<<grid_for(n, 256), 256, 0, s>>>(c, labels_in, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_converge(DevState* st, const unsigned long long* dn,
                            unsigned long long* dn_total, const unsigned long long* scanned,
                            unsigned long long* scan_total, int l, int pick_less, double tol,
                            int32_t n, cudaStream_t s) {
  converge_kernel<<<1, 32, 0, s>>>(st, dn, dn_total, scanned, scan_total, l, pick_less, tol, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_finalize(const DevState* st, int32_t* out, const int32_t* tmp, int32_t n,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  finalize_kernel<<<grid_for(n, 256), 256, 0, s>>>(st, out, tmp, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t* p, int32_t value, int64_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  fill_i32_kernel<<<grid_for(count, 256), 256, 0, s>>>(p, value, count);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_u8(uint8_t* p, uint8_t value, int64_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  fill_u8_kernel<<<grid_for(count, 256), 256, 0, s>>>(p, value, count);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long* p, unsigned long long value, int64_t count,
                            cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  fill_u64_kernel<<<grid_for(count, 256), 256, 0, s>>>(p, value, count);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dn_sum(const unsigned long long* slots, unsigned long long* out,
                          cudaStream_t s) {
  dn_sum_kernel<<<1, 32, 0, s>>>(slots, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_weight_profile(const int64_t* off, const float* w, int32_t n, int64_t m,
                                  unsigned long long* out, cudaStream_t s) {
  weight_profile_kernel<<<grid_for(m > n ? m : n, 256), 256, 0, s>>>(off, w, n, m, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_window_sort(const int64_t* off, int32_t n, int e0, int lmax, int win,
                               int32_t w_first, int64_t hstride, int4* desc, int32_t* wtab,
                               int32_t* hcnt, int32_t* lcnt, cudaStream_t s) {
  const int64_t nwin = (n + (int64_t)win - 1) / win;
  if (nwin <= w_first) return cudaSuccess;
  window_sort_kernel<<<(unsigned)(nwin - w_first), kSortThreads, 0, s>>>(
      off, n, e0, lmax, win, w_first, hstride, desc, wtab, hcnt, lcnt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scan_counts(const int32_t* cnt, int64_t len, int64_t* prefix, cudaStream_t s,
                               int64_t* tiles) {
  if (tiles && len > kScanTile) {
    const int64_t ntiles = (len + kScanTile - 1) / kScanTile;
    tile_sum_kernel<<<(unsigned)ntiles, kScanThreads, 0, s>>>(cnt, len, tiles);
    count_launch();
    scan_i64_kernel<<<1, kScanThreads, 0, s>>>(tiles, ntiles);  // tiles[0, ntiles] in place
    count_launch();
    tile_scan_kernel<<<(unsigned)ntiles, kScanThreads, 0, s>>>(cnt, len, tiles, prefix);
    count_launch();
    return cudaGetLastError();
  }
  scan_counts_kernel<<<1, kScanThreads, 0, s>>>(cnt, len, prefix);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_expand_lanes(const int4* desc, const int32_t* wtab, const int64_t* hub_prefix,
                                const int64_t* lane_prefix, int32_t nwin, int win, int64_t hstride,
                                int32_t w_lanes, int4* hub_desc, int64_t hub_cap, int4* lane_desc,
                                int64_t lane_cap, cudaStream_t s) {
  if (nwin == 0) return cudaSuccess;
  expand_lanes_kernel<<<(unsigned)nwin, kSortThreads, 0, s>>>(
      desc, wtab, hub_prefix, lane_prefix, win, hstride, w_lanes, hub_desc, hub_cap, lane_desc,
      lane_cap);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_slice_count(const WarpPlan& p, int e0, int lmax, int64_t lane_from,
                               int32_t* lane_cnt, int32_t* hub_cnt, int64_t* scan_tmp,
                               int64_t* tiles, int64_t* lane_base, int64_t* hub_pre,
                               int64_t* hub_base, int64_t cap, cudaStream_t s) {
  const int64_t span = ((p.nlanes - lane_from + 255) >> 8) << 8;
  const int64_t threads = span + p.nhubs;
  if (threads > 0) {
    slice_count_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        p.lane_desc, lane_from, p.nlanes, p.hub_desc, p.nhubs, e0, lmax, lane_cnt, hub_cnt);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t nw = (p.nlanes - lane_from) / 32, w_from = lane_from / 32;
  cudaError_t e = launch_scan_counts(lane_cnt, nw, scan_tmp, s, tiles);
  if (e != cudaSuccess) return e;
  lane_base_kernel<<<(unsigned)std::min<int64_t>((nw + 256) / 256, 4096), 256, 0, s>>>(
      scan_tmp, nw, w_from, lane_base);
  count_launch();
  e = launch_scan_counts(hub_cnt, p.nhubs, hub_pre, s, tiles);
  if (e != cudaSuccess) return e;
  if (p.nhubs > 0) {
    hub_base_kernel<<<(unsigned)std::min<int64_t>((p.nhubs + 255) / 256, 4096), 256, 0, s>>>(
        hub_pre, p.nhubs, cap, hub_base);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_slice_fill(const int32_t* idx, const float* w, int64_t m, const WarpPlan& p,
                              int e0, int lmax, int64_t lane_from, int4* sl_idx, float4* sl_w,
                              cudaStream_t s) {
  if (p.nlanes > lane_from) {
    const unsigned grid = (unsigned)((p.nlanes - lane_from + 255) / 256);
    auto kern = p.wfmt == kSplitW ? slice_fill_lanes_kernel<kSplitW> : slice_fill_lanes_kernel<kUnitW>;
    kern<<<grid, 256, 0, s>>>(idx, w, m, p.lane_desc, lane_from, p.nlanes, p.lane_base, sl_idx,
                              sl_w);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (p.nhubs > 0) {
    auto kern = p.wfmt == kSplitW ? slice_fill_hubs_kernel<kSplitW> : slice_fill_hubs_kernel<kUnitW>;
    kern<<<p.nhubs, kThreads, 0, s>>>(idx, w, m, p.hub_desc, p.hub_base, e0, lmax, sl_idx, sl_w);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace lpa
