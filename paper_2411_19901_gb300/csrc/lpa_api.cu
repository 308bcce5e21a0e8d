// lpa_api.cu -- the C ABI declared in include/lpa.h: argument checks, workspace layout,
// plans (degree binning once per graph) and the iteration driver of Alg. 1 (`lpa`).
//
// The driver never waits on the host between iterations: it enqueues max_iter
// {sweep, convergence test} pairs; once the on-device test has fired, later sweeps exit
// on their first instruction.  The host synchronises once, at the end, to read the
// statistics.  Sketch modes (MG, BM) run the warp-per-row sweep over a class binning;
// the exact mode runs its chunk kernel over the chunk/hub binning.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/lpa.h"
#include "lpa_internal.cuh"

using namespace lpa;

std::atomic<unsigned long long> lpa::g_launches{0};

namespace {

thread_local std::string g_err;

lpa_status fail(lpa_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
lpa_status fail(lpa_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define LPA_CUDA(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? LPA_ENOMEM : LPA_ECUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
  } while (0)

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device memory of the library comes from one stream-ordered pool per device that keeps
// freed memory for the next call (release threshold: unlimited), so repeated calls do
// not map and unmap gigabytes of pages each time.  lpa_release_memory() trims the pools.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t lib_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

// Stream-ordered allocation from the library's pool (free with cudaFreeAsync).
cudaError_t lib_alloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool;
  cudaError_t e = lib_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

int64_t num_windows(int64_t n, int win) { return (n + win - 1) / win; }

// Page-locked host blocks of the plans (state, per-iteration counters, modularity and
// binning totals read back from the device), kept for reuse once a plan is destroyed:
// pinning memory costs an operating-system call, and the served form re-plans at every
// admission.
constexpr size_t kHostState = 256;  // >= sizeof(DevState)
constexpr size_t kHostBlock = kHostState + 2 * sizeof(unsigned long long) * LPA_MAX_ITER +
                              4 * sizeof(double) + 32 * sizeof(unsigned long long);
static_assert(sizeof(DevState) <= kHostState, "host block layout");
std::mutex g_host_mu;
std::vector<char*> g_host_free;

cudaError_t acquire_host_block(char** out) {
  {
    std::lock_guard<std::mutex> lock(g_host_mu);
    if (!g_host_free.empty()) {
      *out = g_host_free.back();
      g_host_free.pop_back();
      return cudaSuccess;
    }
  }
  return cudaMallocHost((void**)out, kHostBlock);
}

void release_host_block(void* p) {
  std::lock_guard<std::mutex> lock(g_host_mu);
  g_host_free.push_back((char*)p);
}

// Bounds of the warp-per-row binning for leaf parameter e0 (see lpa_internal.cuh).  A hub
// has more than kHubDegree positions or at least 64 leaves (so >= 64 e0 positions).  A mid
// vertex of L leaves has L e0 <= d positions and L <= 32, so the lanes, one per low
// vertex and L per mid vertex, number at most n + min(m / e0, 31 n), plus under a warp of
// padding per window.
int64_t hub_cap(int64_t n, int64_t m, int e0) {
  const int64_t dmin = std::min<int64_t>(kHubDegree + 1, 64 * (int64_t)e0);
  return std::min<int64_t>(n, m / dmin);
}
int64_t lane_cap(int64_t n, int64_t m, int e0, int win) {
  return n + std::min<int64_t>(m / e0, 31 * n) + 32 * num_windows(n, win);
}
// Elements (groups of four positions) of the sliced copy: a lane leaf of len positions
// takes ceil(len / 4) <= len / 4 + 3/4, a hub of d positions and L leaves L * G with
// G <= (d / L + 4) / 4, so L * G <= d / 4 + L; L <= 256, and L <= d / e0 once L > 1.
int64_t slice_cap(int64_t n, int64_t m, int e0, int win) {
  const int64_t hubs = hub_cap(n, m, e0);
  return m / 4 + 1 + lane_cap(n, m, e0, win) + std::min<int64_t>(256 * hubs, m / e0 + hubs);
}

// Workspace layout of a plan; offsets in bytes from the workspace base.
struct Layout {
  size_t state, dn, dn_total, tmp;
  size_t act, scanned, scan_total;  // pruning: two flag arrays, per-iteration counters
  // sketch modes
  size_t desc, wtab, hcnt, lcnt, hub_prefix, lane_prefix, hub_desc, lane_desc, counts;
  // the sliced copy of the CSR: lane warp counts and bases, hub counts, prefix and bases,
  // scan scratch, the copies of the indices and weights
  size_t sl_cnt, sl_base, sl_hcnt, sl_hpre, sl_hbase, sl_tmp, sl_tiles, sl_idx, sl_w;
  int64_t hub_cap, lane_cap, sl_cap, nwin_cap;
  // exact mode
  size_t cv0, cv1, hubs, hub_tab, seg;
  // modularity
  size_t sigma, partials, out4;
  size_t total_fixed, tab_keys, tab_vals, total;
};

Layout layout(int64_t n, int64_t m, int mode, int e0, int win, bool weighted,
              int64_t tab_slots) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.state = take(sizeof(DevState));
  L.dn = take(sizeof(unsigned long long) * LPA_MAX_ITER * kDnSlots);
  L.dn_total = take(sizeof(unsigned long long) * LPA_MAX_ITER);
  L.act = take(2 * (size_t)n);
  L.scanned = take(sizeof(unsigned long long) * LPA_MAX_ITER * kDnSlots);
  L.scan_total = take(sizeof(unsigned long long) * LPA_MAX_ITER);
  L.tmp = take(sizeof(int32_t) * (size_t)n);
  if (mode == kExact) {
    L.cv0 = take(sizeof(int32_t) * (size_t)(n + 1));
    L.cv1 = take(sizeof(int32_t) * (size_t)(n + 1));
    L.hubs = take(sizeof(int32_t) * (size_t)(n + 1));
    L.hub_tab = take(sizeof(int64_t) * (size_t)(n + 1));
    L.seg = take(3 * sizeof(int64_t) * (size_t)(num_segments(n) + 1));
    L.partials = take(sizeof(double) * 3 * (size_t)modularity_partials((int32_t)n));
  } else {
    const int64_t nwin = num_windows(n, win);
    L.nwin_cap = nwin;
    L.hub_cap = hub_cap(n, m, e0);
    L.lane_cap = lane_cap(n, m, e0, win);
    L.desc = take(sizeof(int4) * (size_t)(nwin * win));
    L.wtab = take(sizeof(int32_t) * (size_t)(nwin * kWinTab));
    L.hcnt = take(sizeof(int32_t) * (size_t)(kHubClasses * nwin));
    L.lcnt = take(sizeof(int32_t) * (size_t)nwin);
    L.hub_prefix = take(sizeof(int64_t) * (size_t)(kHubClasses * nwin + 1));
    L.lane_prefix = take(sizeof(int64_t) * (size_t)(nwin + 1));
    L.hub_desc = take(sizeof(int4) * (size_t)std::max<int64_t>(L.hub_cap, 1));
    L.lane_desc = take(sizeof(int4) * (size_t)std::max<int64_t>(L.lane_cap, 1));
    L.counts = take(sizeof(unsigned long long) * 8);
    L.sl_cap = slice_cap(n, m, e0, win);
    const int64_t nlw = L.lane_cap / 32 + 1, nmax = std::max<int64_t>(nlw, L.hub_cap) + 2;
    L.sl_cnt = take(sizeof(int32_t) * (size_t)nlw);
    L.sl_base = take(sizeof(int64_t) * (size_t)(nlw + 1));
    L.sl_hcnt = take(sizeof(int32_t) * (size_t)(L.hub_cap + 1));
    L.sl_hpre = take(sizeof(int64_t) * (size_t)(L.hub_cap + 2));
    L.sl_hbase = take(sizeof(int64_t) * (size_t)(L.hub_cap + 1));
    L.sl_tmp = take(sizeof(int64_t) * (size_t)nmax);
    L.sl_tiles = take(sizeof(int64_t) * (size_t)scan_tile_slots(nmax));
    L.sl_idx = take(sizeof(int4) * (size_t)L.sl_cap);
    L.sl_w = weighted ? take(sizeof(float4) * (size_t)L.sl_cap) : 0;
    WarpPlan dummy{};
    L.partials = take(sizeof(double) * (size_t)modularity_plan_partials(dummy, (int32_t)n));
  }
  L.sigma = take(sizeof(double) * (size_t)n);
  L.out4 = take(sizeof(double) * 4);
  L.total_fixed = o;
  L.tab_keys = take(sizeof(int32_t) * (size_t)tab_slots);
  L.tab_vals = take(sizeof(float) * (size_t)tab_slots);
  L.total = o;
  return L;
}

bool valid_k(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32; }

// The launch choices of o with the defaults filled in.
lpa_status resolve_tuning(const lpa_options& o, lpa_tuning* t) {
  lpa_tuning d{};
  if (o.tuning) d = *o.tuning;
  if (d.window == 0) d.window = kWinVerts;
  if (d.lane_threads == 0) d.lane_threads = kLaneThreads;
  if (d.window < kWinVertsMin || d.window > kWinVerts || (d.window & (d.window - 1)))
    return fail(LPA_EINVAL, "tuning.window = %d must be a power of two in [%d, %d]", d.window,
                kWinVertsMin, kWinVerts);
  if (d.lane_threads != 64 && d.lane_threads != 128 && d.lane_threads != 256)
    return fail(LPA_EINVAL, "tuning.lane_threads = %d must be 64, 128 or 256", d.lane_threads);
  if (d.serial_hubs != 0 && d.serial_hubs != 1)
    return fail(LPA_EINVAL, "tuning.serial_hubs must be 0 or 1");
  *t = d;
  return LPA_OK;
}

}  // namespace

int lpa::set_last_error(int s, const char* msg) {
  g_err = msg;
  return s;
}

struct lpa_plan_s {
  const int64_t* off = nullptr;
  const int32_t* idx = nullptr;
  const float* w = nullptr;
  int32_t n = 0;
  int64_t m = 0;
  int mode = kMG, k = 8;
  int e0 = 64, lmax = 256, rho = 8;
  lpa_tuning tune{};  // launch choices (all fields resolved: no zeros)
  int64_t cap_n = 0, cap_m = 0;  // largest graph the workspace layout holds
  uint32_t flags = 0;
  const int32_t* labels_in = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // sketch modes: the hub kernel runs here, beside the lanes
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  char* tab_ws = nullptr;  // exact-mode hub tables when the library allocates
  bool own_tab = false;
  Layout lay{};
  DevState* st = nullptr;
  unsigned long long* dn = nullptr;
  unsigned long long* dn_total = nullptr;
  int32_t* tmp = nullptr;
  WarpPlan wp{};  // sketch modes
  int32_t *cv0 = nullptr, *cv1 = nullptr, *hubs = nullptr;  // exact mode
  int64_t* hub_tab = nullptr;
  int32_t* tab_keys = nullptr;
  float* tab_vals = nullptr;
  int64_t nchunks = 0, nhubs = 0, hub_edges = 0;
  double setup_ms = 0.0;
  std::vector<cudaEvent_t> events;  // timing pairs, created on demand
  DevState* host_state = nullptr;   // page-locked mirrors
  unsigned long long* host_dn = nullptr;
  unsigned long long* host_scan = nullptr;
  double* host_q = nullptr;
  unsigned long long* host_cls = nullptr;
  // LPA_GRAPH: the recorded run (its launches as one CUDA graph), the arguments it was
  // recorded with, its kernel count, and the library's own stream it is recorded on
  cudaGraphExec_t gexec = nullptr;
  const int32_t* g_labels_out = nullptr;
  double g_tol = 0.0;
  int32_t g_max_iter = -1;
  uint32_t g_flags = 0;
  unsigned long long g_kernels = 0;
  cudaStream_t rec = nullptr;
};

namespace {

lpa_status check_graph_args(const int64_t* offsets, const int32_t* indices, int32_t n,
                            int64_t m) {
  if (n < 0) return fail(LPA_EINVAL, "n = %d is negative", n);
  if (m < 0 || m >= ((int64_t)1 << 62)) return fail(LPA_EINVAL, "m = %lld out of range", (long long)m);
  if (!offsets) return fail(LPA_EINVAL, "offsets is NULL");
  if (m > 0 && !indices) return fail(LPA_EINVAL, "indices is NULL with m > 0");
  return LPA_OK;
}

lpa_status ensure_events(lpa_plan_s* p, size_t count) {
  while (p->events.size() < count) {
    cudaEvent_t e;
    LPA_CUDA(cudaEventCreate(&e));
    p->events.push_back(e);
  }
  return LPA_OK;
}

SweepArgs sweep_args(const lpa_plan_s* p, const int32_t* c_prev, int32_t* c_next, int pick_less,
                     unsigned long long* dn, const int32_t* done) {
  SweepArgs a{};
  a.off = p->off;
  a.idx = p->idx;
  a.w = p->w;
  a.c_prev = c_prev;
  a.c_next = c_next;
  a.chunk_v0 = p->cv0;
  a.chunk_v1 = p->cv1;
  a.hubs = p->hubs;
  a.hub_tab = p->hub_tab;
  a.tab_keys = p->tab_keys;
  a.tab_vals = p->tab_vals;
  a.dn = dn;
  a.done = done;
  a.nchunks = (int32_t)p->nchunks;
  a.nhubs = (int32_t)p->nhubs;
  a.pick_less = pick_less;
  a.e0 = p->e0;
  a.lmax = p->lmax;
  a.m = p->m;
  return a;
}

cudaError_t launch_sketch_sweep(const lpa_plan_s* p, const SweepArgs& a, cudaStream_t s_hub) {
  const bool literal = (p->flags & LPA_MG_UNCLAMPED) != 0, rescan = (p->flags & LPA_RESCAN) != 0;
  if (p->mode == kMG && (literal || rescan))
    return launch_sweep_mg_variant(p->k, literal, rescan, a, p->wp, p->stream,
                                   s_hub);
  return launch_sweep_warp(p->mode, p->k, a, p->wp, p->stream, s_hub);
}

cudaError_t launch_one_sweep(const lpa_plan_s* p, const SweepArgs& a) {
  if (p->mode == kExact) return launch_sweep_exact(p->w != nullptr, a, p->stream);
  if (!p->side) return launch_sketch_sweep(p, a, p->stream);
  // fork: the hub kernel on the side stream, the lane kernel on the plan's stream; join
  cudaError_t e = cudaEventRecord(p->fork_ev, p->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->fork_ev, 0);
  if (e == cudaSuccess) e = launch_sketch_sweep(p, a, p->side);
  if (e == cudaSuccess) e = cudaEventRecord(p->join_ev, p->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->join_ev, 0);
  return e;
}

// LPA_GRAPH: run enqueue(stream) -- stream-ordered launches and copies only, no host
// synchronisation -- as one CUDA graph launched on the plan's stream.  The graph is
// recorded on a stream of the plan's own (capture is not possible on the legacy default
// stream) with the plan's stream field pointing at it meanwhile, instantiated, kept, and
// launched again while labels_out, tol, max_iter and the flags are those it was recorded
// with.  Capture-time launch counts are taken back and each launch of the graph adds its
// kernel count instead.
template <class F>
lpa_status run_recorded(lpa_plan_s* p, const int32_t* labels_out, double tol, int32_t max_iter,
                        F&& enqueue) {
  cudaStream_t s = p->stream;
  const bool same = p->gexec && p->g_labels_out == labels_out && p->g_tol == tol &&
                    p->g_max_iter == max_iter && p->g_flags == p->flags;
  if (!same) {
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    if (!p->rec) LPA_CUDA(cudaStreamCreateWithFlags(&p->rec, cudaStreamNonBlocking));
    LPA_CUDA(cudaStreamBeginCapture(p->rec, cudaStreamCaptureModeThreadLocal));
    p->stream = p->rec;
    lpa_status st = enqueue(p->rec);
    p->stream = s;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(p->rec, &g);  // ends it after a failure too
    size_t nodes = 0;
    unsigned long long kernels = 0;
    if (st == LPA_OK && ce == cudaSuccess && cudaGraphGetNodes(g, nullptr, &nodes) == cudaSuccess) {
      std::vector<cudaGraphNode_t> all(nodes);
      if (nodes > 0 && cudaGraphGetNodes(g, all.data(), &nodes) == cudaSuccess)
        for (cudaGraphNode_t nd : all) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
        }
    }
    g_launches.fetch_sub(kernels, std::memory_order_relaxed);
    if (st != LPA_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return st != LPA_OK ? st : fail(LPA_ECUDA, "recording the run: %s", cudaGetErrorString(ce));
    }
    const cudaError_t ie = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      p->gexec = nullptr;
      return fail(LPA_ECUDA, "instantiating the recorded run: %s", cudaGetErrorString(ie));
    }
    p->g_labels_out = labels_out;
    p->g_tol = tol;
    p->g_max_iter = max_iter;
    p->g_flags = p->flags;
    p->g_kernels = kernels;
  }
  LPA_CUDA(cudaGraphLaunch(p->gexec, s));
  g_launches.fetch_add(p->g_kernels, std::memory_order_relaxed);
  return LPA_OK;
}

void destroy_plan(lpa_plan_s* p) {
  if (!p) return;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->rec) cudaStreamDestroy(p->rec);
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  if (p->join_ev) cudaEventDestroy(p->join_ev);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->own_ws && p->ws) cudaFreeAsync(p->ws, p->stream);
  if (p->own_tab && p->tab_ws) cudaFreeAsync(p->tab_ws, p->stream);
  if (p->own_ws || p->own_tab) cudaStreamSynchronize(p->stream);
  if (p->host_state) release_host_block(p->host_state);
  delete p;
}

// Window binning of the sketch modes: sort each window's vertices into groups, lay out
// the hub and lane descriptors, and read back the totals.
lpa_status bin_classes(lpa_plan_s* p, int32_t keep_n) {
  cudaStream_t s = p->stream;
  const int32_t n = p->n;
  const Layout& ly = p->lay;
  WarpPlan& wp = p->wp;
  wp = WarpPlan{};
  wp.hub_desc = (const int4*)(p->ws + ly.hub_desc);
  wp.lane_desc = (const int4*)(p->ws + ly.lane_desc);
  if (n == 0) return LPA_OK;
  const int win = p->tune.window;
  const int32_t nwin = (int32_t)num_windows(n, win);
  const int64_t hstride = ly.nwin_cap;
  // windows before w0 hold only vertices below keep_n, binned before and unchanged
  const int32_t w0 = keep_n > 0 ? keep_n / win : 0;
  int4* desc = (int4*)(p->ws + ly.desc);
  int32_t* wtab = (int32_t*)(p->ws + ly.wtab);
  int32_t* hcnt = (int32_t*)(p->ws + ly.hcnt);
  int32_t* lcnt = (int32_t*)(p->ws + ly.lcnt);
  int64_t* hub_prefix = (int64_t*)(p->ws + ly.hub_prefix);
  int64_t* lane_prefix = (int64_t*)(p->ws + ly.lane_prefix);
  unsigned long long* counts = (unsigned long long*)(p->ws + ly.counts);
  // counts: [0, 3) weight profile
  LPA_CUDA(launch_fill_u64(counts, 0ull, 8, s));
  LPA_CUDA(launch_fill_u64(counts, 1ull, 1, s));  // profile: all integral until shown otherwise
  for (int c = 0; c < kHubClasses; ++c)  // hub counts of the windows sorted now, and past them
    LPA_CUDA(launch_fill_i32(hcnt + c * hstride + w0, 0, hstride - w0, s));
  LPA_CUDA(launch_window_sort(p->off, n, p->e0, p->lmax, win, w0, hstride, desc, wtab, hcnt,
                              lcnt, s));
  LPA_CUDA(launch_scan_counts(hcnt, (int64_t)kHubClasses * hstride, hub_prefix, s));
  LPA_CUDA(launch_scan_counts(lcnt, nwin, lane_prefix, s));
  LPA_CUDA(launch_expand_lanes(desc, wtab, hub_prefix, lane_prefix, nwin, win, hstride, w0,
                               (int4*)wp.hub_desc, ly.hub_cap, (int4*)wp.lane_desc, ly.lane_cap, s));
  // the longest row (the weights are not read: only row lengths matter here)
  LPA_CUDA(launch_weight_profile(p->off, nullptr, n, p->m, counts, s));
  LPA_CUDA(cudaMemcpyAsync(p->host_cls, counts, sizeof(unsigned long long) * 3,
                           cudaMemcpyDeviceToHost, s));
  for (int c = 0; c <= kHubClasses; ++c)  // first hub of each class, then the total
    LPA_CUDA(cudaMemcpyAsync(p->host_cls + 8 + c, hub_prefix + (int64_t)c * hstride,
                             sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaMemcpyAsync(p->host_cls + 4, lane_prefix + nwin, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaMemcpyAsync(p->host_cls + 5, lane_prefix + w0, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaStreamSynchronize(s));
  const double dmax = (double)p->host_cls[2];
  if (dmax > 2147483647.0) return fail(LPA_EUNSUPPORTED, "a row has more than 2^31 - 1 entries");
  const int64_t nhubs = (int64_t)p->host_cls[8 + kHubClasses], nlanes = (int64_t)p->host_cls[4];
  const int64_t lane_from = (int64_t)p->host_cls[5];
  if (nhubs < 0 || nhubs > ly.hub_cap || nlanes < 0 || nlanes > ly.lane_cap || lane_from < 0 ||
      lane_from > nlanes || (lane_from & 31))
    return fail(LPA_EINTERNAL, "window binning counted %lld hubs and %lld lanes", (long long)nhubs,
                (long long)nlanes);
  const int64_t nctas = nhubs + (nlanes + kThreads - 1) / kThreads;
  if (nctas > 0x7fffffffLL) return fail(LPA_EUNSUPPORTED, "graph too large for one launch grid");
  wp.nhubs = (int32_t)nhubs;
  for (int c = 0; c <= kHubClasses; ++c) wp.hub_start[c] = (int32_t)p->host_cls[8 + c];
  wp.nlanes = nlanes;
  wp.nctas = (int32_t)nctas;
  wp.e0 = p->e0;
  wp.lmax = p->lmax;
  wp.lane_threads = p->tune.lane_threads;
  p->nhubs = nhubs;
  p->nchunks = nctas - nhubs;
  // the sliced copy of the CSR that the sweeps read (lanes from lane_from on, every hub)
  wp.wfmt = p->w ? kSplitW : kUnitW;
  int64_t* lane_base = (int64_t*)(p->ws + ly.sl_base);
  int64_t* hub_pre = (int64_t*)(p->ws + ly.sl_hpre);
  wp.lane_base = lane_base;
  wp.hub_base = (int64_t*)(p->ws + ly.sl_hbase);
  LPA_CUDA(launch_slice_count(wp, p->e0, p->lmax, lane_from, (int32_t*)(p->ws + ly.sl_cnt),
                              (int32_t*)(p->ws + ly.sl_hcnt), (int64_t*)(p->ws + ly.sl_tmp),
                              (int64_t*)(p->ws + ly.sl_tiles), lane_base, hub_pre,
                              (int64_t*)wp.hub_base, ly.sl_cap, s));
  LPA_CUDA(cudaMemcpyAsync(p->host_cls + 16, lane_base + nlanes / 32, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaMemcpyAsync(p->host_cls + 17, hub_pre + nhubs, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaStreamSynchronize(s));
  const int64_t lane_groups = (int64_t)p->host_cls[16], hub_groups = (int64_t)p->host_cls[17];
  if (lane_groups < 0 || hub_groups < 0 || lane_groups + hub_groups > ly.sl_cap)
    return fail(LPA_EINTERNAL, "sliced copy of %lld + %lld groups exceeds its bound %lld",
                (long long)lane_groups, (long long)hub_groups, (long long)ly.sl_cap);
  wp.sl_idx = (const int4*)(p->ws + ly.sl_idx);
  wp.sl_w = p->w ? (const float4*)(p->ws + ly.sl_w) : nullptr;
  LPA_CUDA(launch_slice_fill(p->idx, p->w, p->m, wp, p->e0, p->lmax, lane_from, (int4*)wp.sl_idx,
                             (float4*)wp.sl_w, s));
  return LPA_OK;
}

// Chunk binning of the exact mode.
lpa_status bin_chunks(lpa_plan_s* p, const lpa_options& o) {
  cudaStream_t s = p->stream;
  const int32_t n = p->n;
  const int64_t nseg = num_segments(n);
  int64_t* seg = (int64_t*)(p->ws + p->lay.seg);
  BinArgs b{};
  b.off = p->off;
  b.n = n;
  b.cap = kChunkCapExact;
  b.cost_floor = b.cap / kThreads;
  b.e0 = p->e0;
  b.lmax = p->lmax;
  b.leaves = 0;
  b.seg_chunks = seg;
  b.seg_hubs = seg + (nseg + 1);
  b.seg_hub_edges = seg + 2 * (nseg + 1);
  b.chunk_v0 = p->cv0;
  b.chunk_v1 = p->cv1;
  b.hubs = p->hubs;
  b.hub_tab = p->hub_tab;
  if (n > 0) {
    LPA_CUDA(launch_bin(b, p->st, s, false));
    LPA_CUDA(cudaMemcpyAsync(p->host_state, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LPA_CUDA(cudaStreamSynchronize(s));
    p->nchunks = p->host_state->nchunks;
    p->nhubs = p->host_state->nhubs;
    p->hub_edges = p->host_state->hub_edges;
    if (p->nchunks + p->nhubs > 0x7fffffffLL || p->nchunks > n || p->nhubs > n)
      return fail(LPA_EINTERNAL, "binning produced %lld chunks and %lld hubs",
                  (long long)p->nchunks, (long long)p->nhubs);
    LPA_CUDA(launch_bin(b, p->st, s, true));
  }
  if (p->hub_edges > 0) {
    const int64_t slots = 2 * p->hub_edges;
    if (o.workspace) {
      p->tab_keys = (int32_t*)(p->ws + p->lay.tab_keys);
      p->tab_vals = (float*)(p->ws + p->lay.tab_vals);
    } else {
      const size_t kb = align256(sizeof(int32_t) * (size_t)slots);
      LPA_CUDA(lib_alloc((void**)&p->tab_ws, kb + sizeof(float) * (size_t)slots, s));
      p->own_tab = true;
      p->tab_keys = (int32_t*)p->tab_ws;
      p->tab_vals = (float*)(p->tab_ws + kb);
    }
  }
  return LPA_OK;
}

// A plan of the graph (offsets, indices, weights, n, m).  Its workspace is laid out for
// graphs of up to cap_n vertices and cap_m entries (at least n, m), so that the served
// form can re-bind it to its grown arena (plan_rebind) without allocating.
lpa_status plan_create(const int64_t* offsets, const int32_t* indices, const float* weights,
                       int32_t n, int64_t m, lpa_mode mode, int32_t k, const lpa_options* opt,
                       lpa_plan_s** out, int64_t cap_n = -1, int64_t cap_m = -1) {
  *out = nullptr;
  lpa_status s = check_graph_args(offsets, indices, n, m);
  if (s != LPA_OK) return s;
  if (mode != LPA_EXACT && mode != LPA_MG && mode != LPA_BM)
    return fail(LPA_EINVAL, "unknown mode %d", (int)mode);
  if (mode == LPA_MG && (k < 1 || k > 32)) return fail(LPA_EINVAL, "k = %d outside [1, 32]", k);
  if (mode == LPA_MG && !valid_k(k))
    return fail(LPA_EUNSUPPORTED, "k = %d: only 1, 2, 4, 8, 16, 32 are built", k);
  lpa_options defaults;
  lpa_options_init(&defaults);
  const lpa_options& o = opt ? *opt : defaults;
  if (o.pl_period < 0) return fail(LPA_EINVAL, "pl_period = %d is negative", o.pl_period);
  if (o.leaf_e0 < 1) return fail(LPA_EINVAL, "leaf_e0 = %d must be >= 1", o.leaf_e0);
  if ((o.flags & (LPA_MG_UNCLAMPED | LPA_RESCAN)) && mode != LPA_MG)
    return fail(LPA_EINVAL, "LPA_MG_UNCLAMPED and LPA_RESCAN apply to LPA_MG only");
  if ((o.flags & LPA_GRAPH) && (o.flags & LPA_TIMING))
    return fail(LPA_EINVAL, "LPA_GRAPH and LPA_TIMING cannot be combined: per-sweep events are "
                "not timed inside a graph");
  if (o.leaf_max < 1 || o.leaf_max > kMaxLeaves || (o.leaf_max & (o.leaf_max - 1)))
    return fail(LPA_EINVAL, "leaf_max = %d must be a power of two in [1, %d]", o.leaf_max, kMaxLeaves);
  if (((uintptr_t)indices & 15) != 0 || ((uintptr_t)weights & 15) != 0)
    return fail(LPA_EINVAL, "indices and weights must be 16-byte aligned");

  lpa_tuning tune;
  const lpa_status ts = resolve_tuning(o, &tune);
  if (ts != LPA_OK) return ts;

  lpa_plan_s* p = new lpa_plan_s();
  p->tune = tune;
  p->off = offsets;
  p->idx = indices;
  p->w = weights;
  p->n = n;
  p->m = m;
  p->mode = (int)mode;
  p->k = mode == LPA_MG ? k : 1;
  p->e0 = o.leaf_e0;
  p->lmax = o.leaf_max;
  p->rho = o.pl_period;
  p->flags = o.flags;
  p->labels_in = o.labels_in;
  p->stream = (cudaStream_t)o.stream;

  auto bail = [&](lpa_status st) {
    destroy_plan(p);
    return st;
  };
  char* hb = nullptr;
  cudaError_t ce = acquire_host_block(&hb);
  if (ce != cudaSuccess) return bail(fail(LPA_ECUDA, "cudaMallocHost: %s", cudaGetErrorString(ce)));
  p->host_state = (DevState*)hb;
  p->host_dn = (unsigned long long*)(hb + kHostState);
  p->host_scan = p->host_dn + LPA_MAX_ITER;
  p->host_q = (double*)(p->host_scan + LPA_MAX_ITER);
  p->host_cls = (unsigned long long*)(p->host_q + 4);

  // workspace: fixed part now; exact-mode hub tables once binning knows their size
  p->cap_n = std::max<int64_t>(cap_n, n);
  p->cap_m = std::max<int64_t>(cap_m, m);
  p->lay = layout(p->cap_n, p->cap_m, p->mode, p->e0, p->tune.window, weights != nullptr,
                  p->mode == kExact ? 2 * m : 0);
  if (o.workspace) {
    if (o.workspace_bytes < p->lay.total)
      return bail(fail(LPA_ENOMEM, "workspace of %zu bytes, %zu needed", o.workspace_bytes, p->lay.total));
    if (((uintptr_t)o.workspace & 255) != 0)
      return bail(fail(LPA_EINVAL, "workspace is not 256-byte aligned"));
    p->ws = (char*)o.workspace;
    p->ws_bytes = o.workspace_bytes;
  } else {
    p->ws_bytes = p->lay.total_fixed;
    ce = lib_alloc((void**)&p->ws, p->ws_bytes, p->stream);
    if (ce != cudaSuccess)
      return bail(fail(LPA_ENOMEM, "device allocation of %zu bytes: %s", p->ws_bytes, cudaGetErrorString(ce)));
    p->own_ws = true;
  }
  p->st = (DevState*)(p->ws + p->lay.state);
  p->dn = (unsigned long long*)(p->ws + p->lay.dn);
  p->dn_total = (unsigned long long*)(p->ws + p->lay.dn_total);
  p->tmp = (int32_t*)(p->ws + p->lay.tmp);
  if (p->mode == kExact) {
    p->cv0 = (int32_t*)(p->ws + p->lay.cv0);
    p->cv1 = (int32_t*)(p->ws + p->lay.cv1);
    p->hubs = (int32_t*)(p->ws + p->lay.hubs);
    p->hub_tab = (int64_t*)(p->ws + p->lay.hub_tab);
  }

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (p->flags & LPA_TIMING) {
    lpa_status es = ensure_events(p, 2);
    if (es != LPA_OK) return bail(es);
    ev0 = p->events[0];
    ev1 = p->events[1];
    ce = cudaEventRecord(ev0, p->stream);
    if (ce != cudaSuccess) return bail(fail(LPA_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(ce)));
  }
  ce = launch_fill_i32((int32_t*)p->st, 0, sizeof(DevState) / 4, p->stream);
  if (ce == cudaSuccess && (p->flags & LPA_VALIDATE))
    ce = launch_validate(offsets, indices, weights, n, m, p->labels_in, &p->st->err, p->stream);
  if (ce != cudaSuccess) return bail(fail(LPA_ECUDA, "validation launch: %s", cudaGetErrorString(ce)));
  if (p->flags & LPA_VALIDATE) {
    ce = cudaMemcpyAsync(p->host_state, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->stream);
    if (ce != cudaSuccess) return bail(fail(LPA_ECUDA, "validation: %s", cudaGetErrorString(ce)));
    const int err = p->host_state->err;
    if (err) {
      return bail(fail(LPA_EINVAL, "invalid input:%s%s%s%s", (err & kErrOffsets) ? " offsets" : "",
                       (err & kErrIndex) ? " index out of range" : "",
                       (err & kErrWeight) ? " negative/non-finite weight" : "",
                       (err & kErrLabels) ? " labels_in out of range" : ""));
    }
  }
  s = p->mode == kExact ? bin_chunks(p, o) : bin_classes(p, 0);
  if (s != LPA_OK) return bail(s);
  if (p->mode != kExact && p->wp.nhubs > 0 && p->wp.nlanes > 0 && !p->tune.serial_hubs) {
    ce = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(fail(LPA_ECUDA, "side stream: %s", cudaGetErrorString(ce)));
  }
  if (p->flags & LPA_TIMING) {
    ce = cudaEventRecord(ev1, p->stream);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(ev1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, ev0, ev1);
    if (ce != cudaSuccess) return bail(fail(LPA_ECUDA, "timing: %s", cudaGetErrorString(ce)));
    p->setup_ms = ms;
  }
  *out = p;
  return LPA_OK;
}

// Re-bind a sketch-mode plan to a grown graph whose first keep_n vertices (and their rows)
// are unchanged: only the binning windows from the one holding vertex keep_n on, their
// lanes and their slices, and the hubs are redone (keep_n = 0: everything).  The graph
// must fit the plan's capacity and weight format; no validation, no timing.
lpa_status plan_rebind(lpa_plan_s* p, const int64_t* offsets, const int32_t* indices,
                       const float* weights, int32_t n, int64_t m, int32_t keep_n) {
  if (p->mode == kExact || n > p->cap_n || m > p->cap_m || (weights && !p->lay.sl_w))
    return fail(LPA_EINTERNAL, "plan cannot take this graph");
  p->off = offsets;
  p->idx = indices;
  p->w = weights;
  p->n = n;
  p->m = m;
  lpa_status s = bin_classes(p, keep_n);
  if (s != LPA_OK) return s;
  if (!p->side && p->wp.nhubs > 0 && p->wp.nlanes > 0 && !p->tune.serial_hubs) {
    cudaError_t ce = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return fail(LPA_ECUDA, "side stream: %s", cudaGetErrorString(ce));
  }
  return LPA_OK;
}

cudaError_t launch_plan_modularity(const lpa_plan_s* p, const int32_t* labels) {
  double* sigma = (double*)(p->ws + p->lay.sigma);
  double* partials = (double*)(p->ws + p->lay.partials);
  double* out4 = (double*)(p->ws + p->lay.out4);
  if (p->mode == kExact)
    return launch_modularity(p->off, p->idx, p->w, p->m, labels, p->n, sigma, partials,
                             modularity_partials(p->n), out4, p->stream);
  return launch_modularity_plan(p->off, p->idx, p->w, p->m, labels, p->n, p->wp, sigma, partials,
                                modularity_plan_partials(p->wp, p->n), out4, p->stream);
}

lpa_status plan_run(lpa_plan_s* p, double tol, int32_t max_iter, int32_t* labels_out,
                    lpa_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  if (max_iter < 0 || max_iter > LPA_MAX_ITER)
    return fail(LPA_EINVAL, "max_iter = %d outside [0, %d]", max_iter, LPA_MAX_ITER);
  if (!(tol == tol)) return fail(LPA_EINVAL, "tol is NaN");
  if (p->n > 0 && !labels_out) return fail(LPA_EINVAL, "labels_out is NULL");
  cudaStream_t s = p->stream;
  const int32_t n = p->n;
  if (n == 0) {  // nothing to do; matches the definition of convergence on an empty graph
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->converged = 1;
      stats->device_bytes = p->ws_bytes;
    }
    return LPA_OK;
  }
  const bool timing = (p->flags & LPA_TIMING) != 0;
  if (timing && (p->flags & LPA_GRAPH))
    return fail(LPA_EINVAL, "LPA_GRAPH and LPA_TIMING cannot be combined");
  if (timing) {
    lpa_status es = ensure_events(p, 2 + 2 * (size_t)max_iter);
    if (es != LPA_OK) return es;
  }
  const bool prune = (p->flags & LPA_PRUNE) != 0;
  const bool want_q = (p->flags & LPA_MODULARITY) != 0;
  // every launch and copy of the run, stream-ordered on s with no host synchronisation
  // (so that LPA_GRAPH can record it as one graph)
  auto enqueue = [&](cudaStream_t s) -> lpa_status {
    LPA_CUDA(launch_fill_i32((int32_t*)p->st, 0, 4, s));  // done, iterations, converged, err
    LPA_CUDA(launch_fill_u64(p->dn, 0ull, (int64_t)max_iter * kDnSlots, s));
    LPA_CUDA(launch_init_labels(labels_out, p->labels_in, n, s));
    // pruning: act[0] = every vertex unprocessed before iteration 0; iteration l reads
    // act[l & 1] and marks act[(l + 1) & 1]
    uint8_t* act = (uint8_t*)(p->ws + p->lay.act);
    unsigned long long* scanned = prune ? (unsigned long long*)(p->ws + p->lay.scanned) : nullptr;
    unsigned long long* scan_total = (unsigned long long*)(p->ws + p->lay.scan_total);
    if (prune) {
      LPA_CUDA(launch_fill_u8(act, 1, n, s));
      LPA_CUDA(launch_fill_u64(scanned, 0ull, (int64_t)max_iter * kDnSlots, s));
    }
    int32_t* buf[2] = {labels_out, p->tmp};
    for (int l = 0; l < max_iter; ++l) {
      const int pick_less = (p->rho > 0 && l % p->rho == 0) ? 1 : 0;
      SweepArgs a = sweep_args(p, buf[l & 1], buf[(l + 1) & 1], pick_less,
                               p->dn + (int64_t)l * kDnSlots, &p->st->done);
      if (prune) {
        a.act_in = act + (int64_t)(l & 1) * n;
        a.act_out = act + (int64_t)((l + 1) & 1) * n;
        a.scanned = scanned + (int64_t)l * kDnSlots;
      }
      if (timing) LPA_CUDA(cudaEventRecord(p->events[2 + 2 * l], s));
      if (prune) LPA_CUDA(launch_fill_u8(a.act_out, 0, n, s));
      LPA_CUDA(launch_one_sweep(p, a));
      if (timing) LPA_CUDA(cudaEventRecord(p->events[3 + 2 * l], s));
      LPA_CUDA(launch_converge(p->st, p->dn, p->dn_total, scanned, scan_total, l, pick_less, tol,
                               n, s));
    }
    LPA_CUDA(launch_finalize(p->st, labels_out, p->tmp, n, s));
    if (want_q) {
      LPA_CUDA(launch_plan_modularity(p, labels_out));
      LPA_CUDA(cudaMemcpyAsync(p->host_q, p->ws + p->lay.out4, sizeof(double) * 4,
                               cudaMemcpyDeviceToHost, s));
    }
    LPA_CUDA(cudaMemcpyAsync(p->host_state, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    if (max_iter > 0)
      LPA_CUDA(cudaMemcpyAsync(p->host_dn, p->dn_total, sizeof(unsigned long long) * max_iter,
                               cudaMemcpyDeviceToHost, s));
    if (max_iter > 0 && prune)
      LPA_CUDA(cudaMemcpyAsync(p->host_scan, scan_total, sizeof(unsigned long long) * max_iter,
                               cudaMemcpyDeviceToHost, s));
    return LPA_OK;
  };
  const lpa_status es = (p->flags & LPA_GRAPH) ? run_recorded(p, labels_out, tol, max_iter, enqueue)
                                              : enqueue(s);
  if (es != LPA_OK) return es;
  LPA_CUDA(cudaStreamSynchronize(s));
  const int iters = p->host_state->iterations;
  if (iters < 0 || iters > max_iter) return fail(LPA_EINTERNAL, "device reported %d iterations", iters);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = iters;
    stats->converged = p->host_state->converged;
    for (int l = 0; l < iters; ++l) stats->changed[l] = (int64_t)p->host_dn[l];
    stats->edges_scanned = 0;
    for (int l = 0; l < iters; ++l) {
      stats->scanned_iter[l] = prune ? (int64_t)p->host_scan[l] : p->m;
      stats->edges_scanned += stats->scanned_iter[l];
    }
    stats->sweep_launches = iters;
    stats->device_bytes = p->ws_bytes + (p->own_tab ? (size_t)(2 * p->hub_edges) * 8 : 0);
    stats->chunks = (int32_t)p->nchunks;
    stats->hubs = (int32_t)p->nhubs;
    stats->setup_ms = p->setup_ms;
    stats->modularity = want_q ? p->host_q[3] : 0.0;
    if (timing) {
      double tot = 0.0;
      for (int l = 0; l < iters; ++l) {
        float ms = 0.f;
        LPA_CUDA(cudaEventElapsedTime(&ms, p->events[2 + 2 * l], p->events[3 + 2 * l]));
        tot += ms;
      }
      stats->sweep_ms = tot;
      for (int l = 0; l < iters; ++l) {
        float ms = 0.f;
        LPA_CUDA(cudaEventElapsedTime(&ms, p->events[2 + 2 * l], p->events[3 + 2 * l]));
        stats->sweep_ms_iter[l] = ms;
      }
    }
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return LPA_OK;
}

// The batched run on a plan over the packed block-diagonal graph: per-graph stop tests
// (batch_converge), the sweeps skipping stopped graphs, labels unpacked per graph.
struct BatchCtx {
  const BatchGraph* gs;  // device table
  int count;
  const int32_t* gid;
  int32_t *gdone, *giter, *gconv, *active;
  uint32_t* gdn;         // max_iter * count
  int32_t* labels;       // packed labels, n of the plan
};

lpa_status batch_run(lpa_plan_s* p, const BatchCtx& b, double tol, int32_t max_iter) {
  cudaStream_t s = p->stream;
  const int32_t n = p->n;
  LPA_CUDA(launch_fill_i32((int32_t*)p->st, 0, 4, s));
  LPA_CUDA(launch_batch_init(b.gs, b.count, b.gdone, b.giter, b.gconv, b.active, p->st, s));
  if (n == 0) return LPA_OK;
  LPA_CUDA(launch_fill_u64(p->dn, 0ull, (int64_t)max_iter * kDnSlots, s));
  LPA_CUDA(launch_fill_i32((int32_t*)b.gdn, 0, (int64_t)max_iter * b.count, s));
  LPA_CUDA(launch_init_labels(b.labels, nullptr, n, s));
  const bool prune = (p->flags & LPA_PRUNE) != 0;
  uint8_t* act = (uint8_t*)(p->ws + p->lay.act);
  unsigned long long* scanned = prune ? (unsigned long long*)(p->ws + p->lay.scanned) : nullptr;
  if (prune) {
    LPA_CUDA(launch_fill_u8(act, 1, n, s));
    LPA_CUDA(launch_fill_u64(scanned, 0ull, (int64_t)max_iter * kDnSlots, s));
  }
  int32_t* buf[2] = {b.labels, p->tmp};
  for (int l = 0; l < max_iter; ++l) {
    const int pick_less = (p->rho > 0 && l % p->rho == 0) ? 1 : 0;
    SweepArgs a = sweep_args(p, buf[l & 1], buf[(l + 1) & 1], pick_less,
                             p->dn + (int64_t)l * kDnSlots, &p->st->done);
    a.gid = b.gid;
    a.gdone = b.gdone;
    a.gdn = b.gdn + (int64_t)l * b.count;
    if (prune) {
      a.act_in = act + (int64_t)(l & 1) * n;
      a.act_out = act + (int64_t)((l + 1) & 1) * n;
      a.scanned = scanned + (int64_t)l * kDnSlots;
      LPA_CUDA(launch_fill_u8(a.act_out, 0, n, s));
    }
    LPA_CUDA(launch_one_sweep(p, a));
    LPA_CUDA(launch_batch_converge(b.gs, b.count, a.gdn, b.gdone, b.giter, b.gconv, b.active,
                                   p->st, l, pick_less, tol, s));
  }
  LPA_CUDA(launch_finalize(p->st, b.labels, p->tmp, n, s));
  LPA_CUDA(launch_unpack_labels(b.gs, b.gid, b.labels, n, s));
  return LPA_OK;
}

// ------------------------------------------------------------------ served form

// One request of a server: the caller's graph (device arrays that must stay valid until
// the request is reported done) and its progress.
struct ServeReq {
  uint64_t ticket = 0;
  lpa_graph g{};
  size_t foot = 0;
  int32_t state = 0;  // 0 waiting, 1 resident, 2 done
  int32_t iterations = 0, converged = 0;
  int64_t vb = -1;    // vertex base in the current packing while resident
};

// The resident graphs packed block-diagonally in an arena with room to grow: graphs are
// appended at the end of the used part (only their own CSR is copied, and the other
// graphs' labels stay in place); a graph that stops stays as a dead slot that the sweeps
// skip, until a compaction re-packs the live graphs into a fresh arena (labels carried
// over, shifted to their new base).  The plan covers the used part and is rebuilt
// whenever it changes.
struct Packing {
  char* dev = nullptr;
  int gcap = 0, count = 0;      // graph slots: capacity, used
  int64_t ncap = 0, mcap = 0;   // vertex and entry capacity
  int64_t N = 0, M = 0;         // used vertices and entries
  int64_t dead_n = 0;           // vertices of dead slots
  bool weighted = false;
  BatchGraph* tab = nullptr;
  int64_t *bases = nullptr, *off = nullptr, *old_vb = nullptr;  // bases: scratch for appends
  int32_t* idx = nullptr;
  float* w = nullptr;
  int32_t* gid = nullptr;
  int32_t *gdone = nullptr, *giter = nullptr, *gconv = nullptr, *gpl = nullptr, *gfin = nullptr;
  uint32_t* gdn = nullptr;
  int32_t* lab[2] = {nullptr, nullptr};
  int cur = 0;
  lpa_plan_s* plan = nullptr;
  bool plan_ok = false;   // the plan bins the used part as it is now
  int64_t binned_n = 0;   // vertices the plan's binning covers
};

// HBM a resident graph takes: packed CSR (8 B offset + 4 B index (+ 4 B weight) per entry),
// graph id and two labels per vertex, the plan's vertex and lane descriptors, and its
// sliced copy of the indices (and weights): 16 B per group of four, about one group per
// leaf more than the entries fill.
size_t serve_footprint(const lpa_graph& g, int e0) {
  const size_t n = (size_t)g.n, m = (size_t)g.m;
  const size_t lanes = n + m / (size_t)e0 + 32;
  return 8 * (n + 1) + 8 * m + 12 * n + 32 * n + 16 * lanes +
         (g.weights ? 2 : 1) * 16 * (m / 4 + lanes) + 1024;
}

}  // namespace

struct lpa_server_s {
  int mode = kMG, k = 8;
  lpa_tuning tune{};
  double tol = 0.05;
  int max_iter = 20;
  lpa_options opt{};
  cudaStream_t stream = nullptr;
  size_t budget = 0, used = 0;
  uint64_t next = 1;
  std::deque<ServeReq*> waiting;
  std::vector<ServeReq*> slots;  // per graph slot of the packing; nullptr = dead
  int live = 0;
  std::unordered_map<uint64_t, ServeReq*> reqs;
  std::vector<uint64_t> finished;  // tickets done since the last drain
  Packing pk;
  int32_t* d_err = nullptr;      // validation scratch
  int32_t* h_state = nullptr;    // page-locked: giter, gconv, gfin of the last step
  size_t h_state_cap = 0;
};

namespace {

void free_packing(Packing& P, cudaStream_t s) {
  if (P.plan) destroy_plan(P.plan);
  if (P.dev) cudaFreeAsync(P.dev, s);
  P = Packing{};
}

// A fresh arena with the given capacities (no graph yet).
lpa_status alloc_packing(Packing& P, int gcap, int64_t ncap, int64_t mcap, bool weighted,
                         cudaStream_t s) {
  P = Packing{};
  P.gcap = gcap;
  P.ncap = ncap;
  P.mcap = mcap;
  P.weighted = weighted;
  size_t at = 0;
  auto take = [&](size_t bytes) {
    const size_t r = at;
    at = align256(at + bytes);
    return r;
  };
  const size_t o_tab = take(sizeof(BatchGraph) * gcap), o_b = take(8 * 2 * (size_t)(gcap + 1)),
               o_ovb = take(8 * (size_t)gcap), o_off = take(8 * (size_t)(ncap + 1)),
               o_idx = take(4 * (size_t)mcap + 16), o_w = weighted ? take(4 * (size_t)mcap + 16) : 0,
               o_gid = take(4 * (size_t)ncap + 4), o_st = take(4 * 5 * (size_t)gcap),
               o_gdn = take(4 * (size_t)gcap), o_l0 = take(4 * (size_t)ncap + 4),
               o_l1 = take(4 * (size_t)ncap + 4);
  LPA_CUDA(lib_alloc((void**)&P.dev, at, s));
  P.tab = (BatchGraph*)(P.dev + o_tab);
  P.bases = (int64_t*)(P.dev + o_b);
  P.old_vb = (int64_t*)(P.dev + o_ovb);
  P.off = (int64_t*)(P.dev + o_off);
  P.idx = (int32_t*)(P.dev + o_idx);
  P.w = weighted ? (float*)(P.dev + o_w) : nullptr;
  P.gid = (int32_t*)(P.dev + o_gid);
  int32_t* st = (int32_t*)(P.dev + o_st);
  P.gdone = st;
  P.giter = st + gcap;
  P.gconv = st + 2 * (size_t)gcap;
  P.gpl = st + 3 * (size_t)gcap;
  P.gfin = st + 4 * (size_t)gcap;
  P.gdn = (uint32_t*)(P.dev + o_gdn);
  P.lab[0] = (int32_t*)(P.dev + o_l0);
  P.lab[1] = (int32_t*)(P.dev + o_l1);
  return LPA_OK;
}

// Append graphs rs at the end of P's used part (capacity checked by the caller).  Each
// graph's iteration count comes from its request; old_vb[g] >= 0 carries its labels
// from `from` (a compaction), else it starts from C[v] = v.
lpa_status append_graphs(Packing& P, const std::vector<ServeReq*>& rs, const int32_t* from,
                         int rho, cudaStream_t s) {
  const int c = (int)rs.size();
  if (c == 0) return LPA_OK;
  std::vector<BatchGraph> tab(c);
  std::vector<int64_t> bases(2 * (size_t)(c + 1), 0), old_vb(c);
  std::vector<int32_t> st(5 * (size_t)c, 0);
  int64_t nv = 0, ne = 0;
  bool carry = false;
  for (int g = 0; g < c; ++g) {
    ServeReq* r = rs[g];
    tab[g] = BatchGraph{r->g.offsets, r->g.indices, r->g.weights, r->g.labels_out, P.N + nv,
                        P.M + ne, r->g.m, r->g.n, 0};
    old_vb[g] = r->vb;
    carry = carry || r->vb >= 0;
    nv += r->g.n;
    ne += r->g.m;
    bases[g + 1] = nv;
    bases[(size_t)(c + 1) + g + 1] = ne;
    st[(size_t)c + g] = r->iterations;
    st[3 * (size_t)c + g] = (rho > 0 && r->iterations % rho == 0) ? 1 : 0;
  }
  const int g0 = P.count;
  const int64_t endM = P.M + ne;
  cudaError_t ce = cudaMemcpyAsync(P.tab + g0, tab.data(), sizeof(BatchGraph) * c,
                                   cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(P.bases, bases.data(), 8 * bases.size(), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(P.old_vb + g0, old_vb.data(), 8 * (size_t)c, cudaMemcpyHostToDevice, s);
  for (int q = 0; q < 5 && ce == cudaSuccess; ++q)  // gdone, giter, gconv, gpl, gfin
    ce = cudaMemcpyAsync(P.gdone + (size_t)q * P.gcap + g0, st.data() + (size_t)q * c,
                         4 * (size_t)c, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(P.off + P.N + nv, &endM, sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = launch_pack_batch(P.tab + g0, P.bases, P.bases + (c + 1), c, nv, ne, P.off + P.N,
                           P.idx + P.M, P.w ? P.w + P.M : nullptr, P.gid + P.N, g0, false,
                           nullptr, s);
  if (ce == cudaSuccess) {
    if (carry)
      ce = launch_carry_labels(P.tab, P.old_vb, P.gid + P.N, from, P.lab[P.cur] + P.N, P.N, nv, s);
    else
      ce = launch_iota_i32(P.lab[P.cur] + P.N, P.N, nv, s);
  }
  // the host vectors must outlive the copies from pageable memory
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return fail(LPA_ECUDA, "server append: %s", cudaGetErrorString(ce));
  for (int g = 0; g < c; ++g) rs[g]->vb = P.N + bases[g];
  P.count += c;
  P.N += nv;
  P.M = endM;
  return LPA_OK;
}

// The plan over the packing's used part (rebuilt after every change of it).
// The plan over the packing's used part.  After an append (keep) only the binning windows
// from the first appended vertex on, their lanes and slices, and the hubs are redone; after
// a compaction, everything.  A sketch-mode plan that can hold the arena is re-bound in
// place (its workspace, pinned blocks and streams are reused); otherwise a plan is created
// for the arena's capacity.
lpa_status replan(lpa_server_s* S, bool keep) {
  Packing& P = S->pk;
  if (P.N == 0) {
    P.plan_ok = false;
    P.binned_n = 0;
    return LPA_OK;
  }
  if (P.plan && S->mode != kExact && P.N <= P.plan->cap_n && P.M <= P.plan->cap_m &&
      (!P.w || P.plan->lay.sl_w)) {
    const int32_t keep_n = keep && P.plan_ok ? (int32_t)P.binned_n : 0;
    const lpa_status s = plan_rebind(P.plan, P.off, P.idx, P.w, (int32_t)P.N, P.M, keep_n);
    P.plan_ok = s == LPA_OK;
    P.binned_n = P.plan_ok ? P.N : 0;
    return s;
  }
  if (P.plan) {
    destroy_plan(P.plan);
    P.plan = nullptr;
  }
  P.plan_ok = false;
  lpa_options po = S->opt;
  po.flags &= ~(LPA_VALIDATE | LPA_TIMING | LPA_MODULARITY | LPA_PRUNE);
  po.workspace = nullptr;
  po.workspace_bytes = 0;
  po.labels_in = nullptr;
  const lpa_status s = plan_create(P.off, P.idx, P.w, (int32_t)P.N, P.M, (lpa_mode)S->mode, S->k,
                                   &po, &P.plan, P.ncap, P.mcap);
  P.plan_ok = s == LPA_OK;
  P.binned_n = P.plan_ok ? P.N : 0;
  return s;
}

// Admit fresh requests: append them if they fit the arena, else (or when dead slots hold
// more than half of it) compact the live graphs and the fresh ones into a new arena.
lpa_status serve_admit(lpa_server_s* S, std::vector<ServeReq*>& fresh, bool compact) {
  cudaStream_t s = S->stream;
  Packing& P = S->pk;
  int64_t nv = 0, ne = 0;
  bool w = false;
  for (ServeReq* r : fresh) {
    nv += r->g.n;
    ne += r->g.m;
    w = w || (r->g.weights && r->g.m > 0);
  }
  const bool fits = P.dev && P.count + (int)fresh.size() <= P.gcap && P.N + nv <= P.ncap &&
                    P.M + ne <= P.mcap && (!w || P.weighted) && !compact;
  if (fits) {
    lpa_status rs = append_graphs(P, fresh, nullptr, S->opt.pl_period, s);
    if (rs != LPA_OK) return rs;
    for (ServeReq* r : fresh) S->slots.push_back(r);
    return replan(S, true);
  } else {
    std::vector<ServeReq*> live;
    int64_t lv = 0, le = 0;
    bool lw = w;
    for (ServeReq* r : S->slots)
      if (r) {
        live.push_back(r);
        lv += r->g.n;
        le += r->g.m;
        lw = lw || (r->g.weights && r->g.m > 0);
      }
    const int gc = (int)(live.size() + fresh.size());
    if (lv + nv > 0x7ffffff0LL) return fail(LPA_EUNSUPPORTED, "resident vertices exceed int32 ids");
    Packing Q;
    lpa_status rs = alloc_packing(Q, std::max(64, 2 * gc), std::max<int64_t>(1 << 16, 2 * (lv + nv)),
                                  std::max<int64_t>(1 << 20, 2 * (le + ne)), lw, s);
    if (rs != LPA_OK) return rs;
    if (!live.empty()) {
      rs = append_graphs(Q, live, P.lab[P.cur], S->opt.pl_period, s);
      if (rs != LPA_OK) {
        free_packing(Q, s);
        return rs;
      }
    }
    for (ServeReq* r : fresh) r->vb = -1;
    rs = append_graphs(Q, fresh, nullptr, S->opt.pl_period, s);
    if (rs != LPA_OK) {
      free_packing(Q, s);
      return rs;
    }
    Q.plan = P.plan;  // the plan moves to the new arena (re-bound below)
    P.plan = nullptr;
    free_packing(P, s);
    S->pk = Q;
    S->slots = live;
    for (ServeReq* r : fresh) S->slots.push_back(r);
  }
  return replan(S, false);
}

lpa_status serve_step(lpa_server_s* S, int32_t* pending_out) {
  cudaStream_t s = S->stream;
  std::vector<ServeReq*> fresh;
  size_t used = S->used;
  while (!S->waiting.empty()) {  // admission by HBM footprint, first come first served
    ServeReq* r = S->waiting.front();
    if (S->budget && used + r->foot > S->budget && (S->live > 0 || !fresh.empty())) break;
    S->waiting.pop_front();
    r->state = 1;
    r->vb = -1;
    fresh.push_back(r);
    used += r->foot;
  }
  Packing& P0 = S->pk;
  const bool compact = P0.N > 0 && 2 * P0.dead_n > P0.N;
  if (!fresh.empty() || compact) {
    lpa_status rs = serve_admit(S, fresh, compact);
    // on a failure before the fresh requests were placed, they go back to the queue
    const bool placed =
        fresh.empty() || std::find(S->slots.begin(), S->slots.end(), fresh.front()) != S->slots.end();
    if (placed) {
      S->used = used;
      S->live += (int)fresh.size();
    } else {
      for (auto it = fresh.rbegin(); it != fresh.rend(); ++it) {
        (*it)->state = 0;
        S->waiting.push_front(*it);
      }
    }
    if (rs != LPA_OK) return rs;
  }
  if (S->live > 0 && !S->pk.plan_ok) {  // a previous re-plan failed: try again
    lpa_status rs = replan(S, false);
    if (rs != LPA_OK) return rs;
  }
  Packing& P = S->pk;
  if (S->live == 0 || !P.plan_ok) {
    if (pending_out) *pending_out = (int32_t)S->waiting.size();
    return LPA_OK;
  }
  LPA_CUDA(launch_fill_i32((int32_t*)P.gdn, 0, P.count, s));
  LPA_CUDA(launch_fill_i32(P.gfin, 0, P.count, s));
  SweepArgs a = sweep_args(P.plan, P.lab[P.cur], P.lab[1 - P.cur], 0, P.plan->dn, nullptr);
  a.gid = P.gid;
  a.gdone = P.gdone;
  a.gdn = P.gdn;
  a.gpl = P.gpl;
  LPA_CUDA(launch_one_sweep(P.plan, a));
  LPA_CUDA(launch_serve_converge(P.tab, P.count, P.gdn, P.gdone, P.giter, P.gconv, P.gpl, P.gfin,
                                 S->max_iter, S->opt.pl_period, S->tol, s));
  P.cur ^= 1;
  LPA_CUDA(launch_unpack_finished(P.tab, P.gid, P.gfin, P.lab[P.cur], P.N, s));
  if (S->h_state_cap < 3 * (size_t)P.gcap) {
    if (S->h_state) cudaFreeHost(S->h_state);
    S->h_state = nullptr;
    S->h_state_cap = 0;
    LPA_CUDA(cudaMallocHost((void**)&S->h_state, 4 * 3 * (size_t)P.gcap));
    S->h_state_cap = 3 * (size_t)P.gcap;
  }
  LPA_CUDA(cudaMemcpyAsync(S->h_state, P.giter, 4 * (size_t)P.count, cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaMemcpyAsync(S->h_state + P.count, P.gconv, 4 * (size_t)P.count,
                           cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaMemcpyAsync(S->h_state + 2 * (size_t)P.count, P.gfin, 4 * (size_t)P.count,
                           cudaMemcpyDeviceToHost, s));
  LPA_CUDA(cudaStreamSynchronize(s));
  for (int g = 0; g < P.count; ++g) {
    ServeReq* r = S->slots[g];
    if (!r) continue;
    r->iterations = S->h_state[g];
    if (S->h_state[2 * (size_t)P.count + g]) {
      r->state = 2;
      r->converged = S->h_state[P.count + g];
      r->vb = -1;
      S->used -= r->foot;
      S->slots[g] = nullptr;
      S->live -= 1;
      P.dead_n += r->g.n;
      S->finished.push_back(r->ticket);
    }
  }
  if (S->live == 0) {  // everything stopped: the arena is empty again (its plan is kept)
    P.plan_ok = false;
    P.binned_n = 0;
    P.count = 0;
    P.N = P.M = P.dead_n = 0;
    S->slots.clear();
  }
  if (pending_out) *pending_out = (int32_t)(S->live + S->waiting.size());
  return LPA_OK;
}

}  // namespace

int lpa::check_modularity_args(const int64_t* offsets, const int32_t* indices, int32_t n,
                               int64_t m, const int32_t* labels, const double* q_out) {
  lpa_status s = check_graph_args(offsets, indices, n, m);
  if (s != LPA_OK) return s;
  if (!q_out) return fail(LPA_EINVAL, "q_out is NULL");
  if (n > 0 && !labels) return fail(LPA_EINVAL, "labels is NULL");
  return LPA_OK;
}

extern "C" {

void lpa_options_init(lpa_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->pl_period = 8;
  opt->leaf_e0 = 64;
  opt->leaf_max = 256;
  opt->flags = LPA_VALIDATE;
}

size_t lpa_workspace_size(int32_t n, int64_t m, lpa_mode mode, int32_t k) {
  return lpa_workspace_size_ex(n, m, mode, k, nullptr);
}

size_t lpa_workspace_size_ex(int32_t n, int64_t m, lpa_mode mode, int32_t k,
                             const lpa_options* opt) {
  (void)k;
  if (n < 0 || m < 0) return 0;
  lpa_options o;
  lpa_options_init(&o);
  if (opt) o = *opt;
  if (o.leaf_e0 < 1) return 0;
  lpa_tuning t;
  if (resolve_tuning(o, &t) != LPA_OK) return 0;
  return layout(n, m, (int)mode, o.leaf_e0, t.window, true, mode == LPA_EXACT ? 2 * m : 0).total;
}

size_t lpa_modularity_workspace_size(int32_t n) {
  if (n < 0) return 0;
  return align256(sizeof(double) * (size_t)n) + align256(sizeof(double) * 3 * modularity_partials(n)) +
         align256(sizeof(double) * 4) + align256(sizeof(DevState));
}

lpa_status lpa_plan_create(const int64_t* offsets, const int32_t* indices, const float* weights,
                           int32_t n, int64_t m, lpa_mode mode, int32_t k, const lpa_options* opt,
                           lpa_plan* plan_out) {
  if (!plan_out) return fail(LPA_EINVAL, "plan_out is NULL");
  return plan_create(offsets, indices, weights, n, m, mode, k, opt, plan_out);
}

lpa_status lpa_plan_sweep(lpa_plan p, const int32_t* c_prev, int32_t* c_next, int32_t pick_less,
                          int64_t* dn_out) {
  if (!p) return fail(LPA_EINVAL, "plan is NULL");
  if (p->n == 0) {
    if (dn_out) *dn_out = 0;
    return LPA_OK;
  }
  if (!c_prev || !c_next) return fail(LPA_EINVAL, "c_prev/c_next is NULL");
  const char* a0 = (const char*)c_prev;
  const char* b0 = (const char*)c_next;
  const size_t bytes = sizeof(int32_t) * (size_t)p->n;
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(LPA_EINVAL, "c_prev and c_next overlap");
  LPA_CUDA(launch_fill_u64(p->dn, 0ull, kDnSlots, p->stream));
  const SweepArgs a = sweep_args(p, c_prev, c_next, pick_less ? 1 : 0, p->dn, nullptr);
  LPA_CUDA(launch_one_sweep(p, a));
  if (dn_out) {
    LPA_CUDA(launch_dn_sum(p->dn, p->dn_total, p->stream));
    LPA_CUDA(cudaMemcpyAsync(p->host_dn, p->dn_total, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, p->stream));
    LPA_CUDA(cudaStreamSynchronize(p->stream));
    *dn_out = (int64_t)p->host_dn[0];
  }
  return LPA_OK;
}

lpa_status lpa_plan_run(lpa_plan p, double tol, int32_t max_iter, int32_t* labels_out,
                        lpa_stats* stats) {
  if (!p) return fail(LPA_EINVAL, "plan is NULL");
  return plan_run(p, tol, max_iter, labels_out, stats);
}

lpa_status lpa_plan_destroy(lpa_plan p) {
  destroy_plan(p);
  return LPA_OK;
}

lpa_status lpa_detect_ex(const int64_t* offsets, const int32_t* indices, const float* weights,
                         int32_t n, int64_t m, lpa_mode mode, int32_t k, double tol,
                         int32_t max_iter, int32_t* labels_out, lpa_stats* stats,
                         const lpa_options* opt) {
  const auto t0 = std::chrono::steady_clock::now();
  if (max_iter < 0 || max_iter > LPA_MAX_ITER)
    return fail(LPA_EINVAL, "max_iter = %d outside [0, %d]", max_iter, LPA_MAX_ITER);
  lpa_plan_s* p = nullptr;
  lpa_status s = plan_create(offsets, indices, weights, n, m, mode, k, opt, &p);
  if (s != LPA_OK) return s;
  s = plan_run(p, tol, max_iter, labels_out, stats);
  destroy_plan(p);
  if (s == LPA_OK && stats)
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

lpa_status lpa_detect(const int64_t* offsets, const int32_t* indices, const float* weights,
                      int32_t n, int64_t m, lpa_mode mode, int32_t k, double tol, int32_t max_iter,
                      int32_t* labels_out, lpa_stats* stats) {
  return lpa_detect_ex(offsets, indices, weights, n, m, mode, k, tol, max_iter, labels_out, stats,
                       nullptr);
}

lpa_status lpa_detect_host(const int64_t* offsets, const int32_t* indices, const float* weights,
                           int32_t n, int64_t m, lpa_mode mode, int32_t k, double tol,
                           int32_t max_iter, int32_t* labels_out, lpa_stats* stats,
                           const lpa_options* opt) {
  const auto t0 = std::chrono::steady_clock::now();
  lpa_status s = check_graph_args(offsets, indices, n, m);
  if (s != LPA_OK) return s;
  if (n > 0 && !labels_out) return fail(LPA_EINVAL, "labels_out is NULL");
  lpa_options o;
  lpa_options_init(&o);
  if (opt) o = *opt;
  cudaStream_t st = (cudaStream_t)o.stream;
  char* dev = nullptr;
  const size_t b_off = align256(sizeof(int64_t) * ((size_t)n + 1));
  const size_t b_idx = align256(sizeof(int32_t) * (size_t)m);
  const size_t b_w = weights ? align256(sizeof(float) * (size_t)m) : 0;
  const size_t b_lab = align256(sizeof(int32_t) * (size_t)n);
  LPA_CUDA(lib_alloc((void**)&dev, b_off + b_idx + b_w + b_lab, st));
  int64_t* d_off = (int64_t*)dev;
  int32_t* d_idx = (int32_t*)(dev + b_off);
  float* d_w = weights ? (float*)(dev + b_off + b_idx) : nullptr;
  int32_t* d_lab = (int32_t*)(dev + b_off + b_idx + b_w);
  cudaError_t ce = cudaMemcpyAsync(d_off, offsets, sizeof(int64_t) * ((size_t)n + 1),
                                   cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && m > 0)
    ce = cudaMemcpyAsync(d_idx, indices, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && weights && m > 0)
    ce = cudaMemcpyAsync(d_w, weights, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, st);
  if (ce != cudaSuccess) {
    cudaFreeAsync(dev, st);
    return fail(LPA_ECUDA, "host-to-device copy: %s", cudaGetErrorString(ce));
  }
  s = lpa_detect_ex(d_off, d_idx, d_w, n, m, mode, k, tol, max_iter, d_lab, stats, &o);
  if (s == LPA_OK && n > 0) {
    ce = cudaMemcpyAsync(labels_out, d_lab, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) s = fail(LPA_ECUDA, "device-to-host copy: %s", cudaGetErrorString(ce));
  }
  cudaFreeAsync(dev, st);
  ce = cudaStreamSynchronize(st);
  if (s == LPA_OK && ce != cudaSuccess) s = fail(LPA_ECUDA, "sync: %s", cudaGetErrorString(ce));
  if (s == LPA_OK && stats)
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

lpa_status lpa_modularity_ex(const int64_t* offsets, const int32_t* indices, const float* weights,
                             int32_t n, int64_t m, const int32_t* labels, double* q_out,
                             const lpa_options* opt) {
  lpa_status s = (lpa_status)check_modularity_args(offsets, indices, n, m, labels, q_out);
  if (s != LPA_OK) return s;
  lpa_options o;
  lpa_options_init(&o);
  if (opt) o = *opt;
  cudaStream_t st = (cudaStream_t)o.stream;
  const int npart = modularity_partials(n);
  const size_t need = lpa_modularity_workspace_size(n);
  char* ws = (char*)o.workspace;
  bool own = false;
  if (ws) {
    if (o.workspace_bytes < need) return fail(LPA_ENOMEM, "workspace of %zu bytes, %zu needed", o.workspace_bytes, need);
    if (((uintptr_t)ws & 255) != 0) return fail(LPA_EINVAL, "workspace is not 256-byte aligned");
  } else {
    LPA_CUDA(lib_alloc((void**)&ws, need, st));
    own = true;
  }
  double* sigma_c = (double*)ws;
  double* partials = (double*)(ws + align256(sizeof(double) * (size_t)n));
  double* out3 = (double*)((char*)partials + align256(sizeof(double) * 3 * npart));
  DevState* dst = (DevState*)((char*)out3 + align256(sizeof(double) * 4));
  double host_out[4] = {0, 0, 0, 0};
  DevState host_st{};
  cudaError_t ce = cudaSuccess;
  if (o.flags & LPA_VALIDATE) {
    ce = launch_fill_i32((int32_t*)dst, 0, sizeof(DevState) / 4, st);
    if (ce == cudaSuccess) ce = launch_validate(offsets, indices, weights, n, m, labels, &dst->err, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&host_st, dst, sizeof(DevState), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess && host_st.err) {
      if (own) cudaFreeAsync(ws, st);
      cudaStreamSynchronize(st);
      return fail(LPA_EINVAL, "invalid input (error bits 0x%x)", host_st.err);
    }
  }
  if (ce == cudaSuccess) ce = launch_modularity(offsets, indices, weights, m, labels, n, sigma_c, partials, npart, out3, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(host_out, out3, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
  if (own) cudaFreeAsync(ws, st);
  cudaError_t ce2 = cudaStreamSynchronize(st);
  if (ce == cudaSuccess) ce = ce2;
  if (ce != cudaSuccess) return fail(LPA_ECUDA, "modularity: %s", cudaGetErrorString(ce));
  *q_out = host_out[3];
  return LPA_OK;
}

lpa_status lpa_modularity(const int64_t* offsets, const int32_t* indices, const float* weights,
                          int32_t n, int64_t m, const int32_t* labels, double* q_out) {
  return lpa_modularity_ex(offsets, indices, weights, n, m, labels, q_out, nullptr);
}

const char* lpa_status_string(lpa_status s) {
  switch (s) {
    case LPA_OK: return "ok";
    case LPA_EINVAL: return "invalid argument";
    case LPA_ENOMEM: return "out of device memory";
    case LPA_ECUDA: return "CUDA error";
    case LPA_ETIMEOUT: return "device wait timed out";
    case LPA_EUNSUPPORTED: return "unsupported";
    case LPA_EINTERNAL: return "internal error";
  }
  return "unknown status";
}

const char* lpa_last_error(void) { return g_err.c_str(); }

const char* lpa_version(void) { return "lpa-gb300 0.1 (sm_103a)"; }

uint64_t lpa_launch_count(void) { return (uint64_t)g_launches.load(); }


lpa_status lpa_batch_detect(const lpa_graph* graphs, int32_t count, lpa_mode mode, int32_t k,
                            double tol, int32_t max_iter, const lpa_options* opt,
                            lpa_graph_stats* stats, int64_t* changed_out) {
  if (count < 0) return fail(LPA_EINVAL, "count = %d is negative", count);
  if (count > 0 && !graphs) return fail(LPA_EINVAL, "graphs is NULL");
  if (max_iter < 0 || max_iter > LPA_MAX_ITER)
    return fail(LPA_EINVAL, "max_iter = %d outside [0, %d]", max_iter, LPA_MAX_ITER);
  if (!(tol == tol)) return fail(LPA_EINVAL, "tol is NaN");
  lpa_options o;
  lpa_options_init(&o);
  if (opt) o = *opt;
  if (o.labels_in) return fail(LPA_EINVAL, "labels_in is not supported by lpa_batch_detect");
  if (count == 0) return LPA_OK;
  // host: vertex and entry bases of the packed block-diagonal graph
  std::vector<int64_t> vb(count + 1), eb(count + 1);
  std::vector<BatchGraph> tab(count);
  bool weighted = false;
  for (int g = 0; g < count; ++g) {
    const lpa_graph& G = graphs[g];
    lpa_status cs = check_graph_args(G.offsets, G.indices, G.n, G.m);
    if (cs != LPA_OK) return fail(cs, "graph %d: %s", g, lpa_last_error());
    if (G.n > 0 && !G.labels_out) return fail(LPA_EINVAL, "graph %d: labels_out is NULL", g);
    tab[g] = BatchGraph{G.offsets, G.indices, G.weights, G.labels_out, vb[g], eb[g], G.m, G.n, 0};
    vb[g + 1] = vb[g] + G.n;
    eb[g + 1] = eb[g] + G.m;
    weighted = weighted || (G.weights != nullptr && G.m > 0);
  }
  const int64_t N = vb[count], M = eb[count];
  if (N > 0x7ffffff0LL) return fail(LPA_EUNSUPPORTED, "batch of %lld vertices exceeds int32 ids", (long long)N);
  cudaStream_t s = (cudaStream_t)o.stream;
  // one device block: table, bases, packed CSR, graph ids, per-graph state, packed labels
  size_t at = 0;
  auto take = [&](size_t bytes) {
    const size_t r = at;
    at = align256(at + bytes);
    return r;
  };
  const size_t o_tab = take(sizeof(BatchGraph) * count), o_vb = take(8 * (size_t)(count + 1)),
               o_eb = take(8 * (size_t)(count + 1)), o_off = take(8 * (size_t)(N + 1)),
               o_idx = take(4 * (size_t)M), o_w = weighted ? take(4 * (size_t)M) : 0,
               o_gid = take(4 * (size_t)N), o_state = take(4 * (3 * (size_t)count + 2)),
               o_gdn = take(4 * (size_t)max_iter * count + 4), o_lab = take(4 * (size_t)N + 4),
               o_q = take(8 * 3 * (size_t)count);  // per graph: 2m, intra weight, Q
  char* dev = nullptr;
  LPA_CUDA(lib_alloc((void**)&dev, at, s));
  auto cleanup = [&](lpa_status st) {
    cudaFreeAsync(dev, s);
    cudaStreamSynchronize(s);
    return st;
  };
  BatchGraph* d_tab = (BatchGraph*)(dev + o_tab);
  int64_t* d_off = (int64_t*)(dev + o_off);
  int32_t* d_idx = (int32_t*)(dev + o_idx);
  float* d_w = weighted ? (float*)(dev + o_w) : nullptr;
  int32_t* d_gid = (int32_t*)(dev + o_gid);
  int32_t* d_state = (int32_t*)(dev + o_state);  // gdone, giter, gconv, active, err
  BatchCtx b{d_tab, count, d_gid, d_state, d_state + count, d_state + 2 * count,
             d_state + 3 * count, (uint32_t*)(dev + o_gdn), (int32_t*)(dev + o_lab)};
  int32_t* d_err = d_state + 3 * count + 1;
  cudaError_t ce = cudaMemcpyAsync(d_tab, tab.data(), sizeof(BatchGraph) * count,
                                   cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(dev + o_vb, vb.data(), 8 * (size_t)(count + 1), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(dev + o_eb, eb.data(), 8 * (size_t)(count + 1), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d_off + N, &M, sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = launch_fill_i32(d_err, 0, 1, s);
  const bool validate = (o.flags & LPA_VALIDATE) != 0;
  if (ce == cudaSuccess)
    ce = launch_pack_batch(d_tab, (const int64_t*)(dev + o_vb), (const int64_t*)(dev + o_eb),
                           count, N, M, d_off, d_idx, d_w, d_gid, 0, validate, d_err, s);
  if (ce != cudaSuccess)
    return cleanup(fail(LPA_ECUDA, "batch packing: %s", cudaGetErrorString(ce)));
  if (validate) {
    int32_t err = 0;
    ce = cudaMemcpyAsync(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cleanup(fail(LPA_ECUDA, "batch validation: %s", cudaGetErrorString(ce)));
    if (err)
      return cleanup(fail(LPA_EINVAL, "invalid input in the batch:%s%s%s",
                          (err & kErrOffsets) ? " offsets" : "",
                          (err & kErrIndex) ? " index out of range" : "",
                          (err & kErrWeight) ? " negative/non-finite weight" : ""));
  }
  lpa_options po = o;
  po.flags &= ~(LPA_VALIDATE | LPA_TIMING | LPA_MODULARITY);
  po.workspace = nullptr;
  po.workspace_bytes = 0;
  lpa_plan_s* p = nullptr;
  lpa_status st = plan_create(d_off, d_idx, d_w, (int32_t)N, M, mode, k, &po, &p);
  if (st == LPA_OK && mode == LPA_EXACT && (o.flags & LPA_MODULARITY)) {
    destroy_plan(p);
    return cleanup(fail(LPA_EUNSUPPORTED, "LPA_MODULARITY in a batch needs a sketch mode"));
  }
  if (st != LPA_OK) return cleanup(st);
  st = (o.flags & LPA_GRAPH)
           ? run_recorded(p, b.labels, tol, max_iter,
                          [&](cudaStream_t) { return batch_run(p, b, tol, max_iter); })
           : batch_run(p, b, tol, max_iter);
  const bool want_q = (o.flags & LPA_MODULARITY) != 0;
  double* d_q = (double*)(dev + o_q);
  if (st == LPA_OK && want_q && N > 0) {  // Eq. 1 per graph on the packed final labels
    ce = cudaMemsetAsync(d_q, 0, 8 * 2 * (size_t)count, s);
    if (ce == cudaSuccess)
      ce = launch_modularity_plan(p->off, p->idx, p->w, p->m, b.labels, p->n, p->wp,
                                  (double*)(p->ws + p->lay.sigma), (double*)(p->ws + p->lay.partials),
                                  modularity_plan_partials(p->wp, p->n),
                                  (double*)(p->ws + p->lay.out4), s, d_gid, d_q, d_q + count);
    if (ce == cudaSuccess)
      ce = launch_batch_q(d_tab, count, (double*)(p->ws + p->lay.sigma), d_q, d_q + count,
                          d_q + 2 * (size_t)count, s);
    if (ce != cudaSuccess) st = fail(LPA_ECUDA, "batch modularity: %s", cudaGetErrorString(ce));
  }
  std::vector<int32_t> h_state(3 * (size_t)count);
  std::vector<double> h_q(want_q ? (size_t)count : 0);
  std::vector<uint32_t> h_gdn((size_t)max_iter * count);
  if (st == LPA_OK) {
    ce = cudaMemcpyAsync(h_state.data(), d_state, 4 * 3 * (size_t)count, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && changed_out && max_iter > 0)
      ce = cudaMemcpyAsync(h_gdn.data(), b.gdn, 4 * (size_t)max_iter * count,
                           cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && want_q && N > 0)
      ce = cudaMemcpyAsync(h_q.data(), d_q + 2 * (size_t)count, 8 * (size_t)count,
                           cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) st = fail(LPA_ECUDA, "batch results: %s", cudaGetErrorString(ce));
  }
  destroy_plan(p);
  if (st != LPA_OK) return cleanup(st);
  const bool prune = (o.flags & LPA_PRUNE) != 0;
  for (int g = 0; g < count; ++g) {
    const int32_t it = h_state[(size_t)count + g];
    if (stats) {
      stats[g].iterations = it;
      stats[g].converged = h_state[2 * (size_t)count + g];
      stats[g].edges_scanned = prune ? -1 : (int64_t)it * graphs[g].m;
      stats[g].modularity = (want_q && N > 0) ? h_q[g] : 0.0;
    }
    if (changed_out)
      for (int l = 0; l < max_iter; ++l)
        changed_out[(size_t)g * max_iter + l] = l < it ? (int64_t)h_gdn[(size_t)l * count + g] : 0;
  }
  return cleanup(LPA_OK);
}


lpa_status lpa_server_create(lpa_mode mode, int32_t k, double tol, int32_t max_iter,
                             size_t hbm_budget_bytes, const lpa_options* opt, lpa_server* out) {
  if (!out) return fail(LPA_EINVAL, "out is NULL");
  *out = nullptr;
  if (mode != LPA_EXACT && mode != LPA_MG && mode != LPA_BM)
    return fail(LPA_EINVAL, "unknown mode %d", (int)mode);
  if (mode == LPA_MG && !valid_k(k)) return fail(LPA_EUNSUPPORTED, "k = %d is not built", k);
  if (max_iter < 0 || max_iter > LPA_MAX_ITER)
    return fail(LPA_EINVAL, "max_iter = %d outside [0, %d]", max_iter, LPA_MAX_ITER);
  if (!(tol == tol)) return fail(LPA_EINVAL, "tol is NaN");
  lpa_options o;
  lpa_options_init(&o);
  if (opt) o = *opt;
  if (o.flags & LPA_PRUNE) return fail(LPA_EUNSUPPORTED, "LPA_PRUNE is not supported by the server");
  if (o.labels_in) return fail(LPA_EINVAL, "labels_in is not supported by the server");
  if (o.leaf_e0 < 1) return fail(LPA_EINVAL, "leaf_e0 = %d must be >= 1", o.leaf_e0);
  if ((o.flags & (LPA_MG_UNCLAMPED | LPA_RESCAN)) && mode != LPA_MG)
    return fail(LPA_EINVAL, "LPA_MG_UNCLAMPED and LPA_RESCAN apply to LPA_MG only");
  lpa_tuning tune;
  const lpa_status ts = resolve_tuning(o, &tune);
  if (ts != LPA_OK) return ts;
  lpa_server_s* S = new lpa_server_s();
  S->mode = (int)mode;
  S->k = mode == LPA_MG ? k : 1;
  S->tol = tol;
  S->max_iter = max_iter;
  S->tune = tune;  // a copy: the caller's struct need not outlive the call
  S->opt = o;
  S->opt.tuning = &S->tune;
  S->stream = (cudaStream_t)o.stream;
  S->budget = hbm_budget_bytes;
  cudaError_t ce = lib_alloc((void**)&S->d_err, 256, S->stream);
  if (ce != cudaSuccess) {
    delete S;
    return fail(LPA_ENOMEM, "server scratch: %s", cudaGetErrorString(ce));
  }
  *out = S;
  return LPA_OK;
}

lpa_status lpa_server_submit(lpa_server S, const lpa_graph* graph, uint64_t* ticket) {
  if (!S || !graph || !ticket) return fail(LPA_EINVAL, "NULL argument");
  const lpa_graph& g = *graph;
  lpa_status cs = check_graph_args(g.offsets, g.indices, g.n, g.m);
  if (cs != LPA_OK) return cs;
  if (g.n > 0 && !g.labels_out) return fail(LPA_EINVAL, "labels_out is NULL");
  const size_t foot = serve_footprint(g, S->opt.leaf_e0);
  if (S->budget && foot > S->budget)
    return fail(LPA_EINVAL, "graph needs %zu bytes, the server's budget is %zu", foot, S->budget);
  if ((S->opt.flags & LPA_VALIDATE) && g.n > 0) {
    int32_t err = 0;
    cudaError_t ce = launch_fill_i32(S->d_err, 0, 1, S->stream);
    if (ce == cudaSuccess)
      ce = launch_validate(g.offsets, g.indices, g.weights, g.n, g.m, nullptr, S->d_err, S->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&err, S->d_err, 4, cudaMemcpyDeviceToHost, S->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(S->stream);
    if (ce != cudaSuccess) return fail(LPA_ECUDA, "validation: %s", cudaGetErrorString(ce));
    if (err) return fail(LPA_EINVAL, "invalid graph (error bits %d)", err);
  }
  ServeReq* r = new ServeReq();
  r->ticket = S->next++;
  r->g = g;
  r->foot = foot;
  if (g.n == 0 || S->max_iter == 0) {  // nothing to sweep
    r->state = 2;
    r->converged = g.n == 0;
    if (g.n > 0) {  // max_iter = 0: the initial labels C[i] = i
      cudaError_t ce = launch_init_labels(g.labels_out, nullptr, g.n, S->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(S->stream);
      if (ce != cudaSuccess) {
        delete r;
        return fail(LPA_ECUDA, "init: %s", cudaGetErrorString(ce));
      }
    }
  } else {
    S->waiting.push_back(r);
  }
  S->reqs[r->ticket] = r;
  *ticket = r->ticket;
  return LPA_OK;
}

lpa_status lpa_server_step(lpa_server S, int32_t* pending_out) {
  if (!S) return fail(LPA_EINVAL, "server is NULL");
  return serve_step(S, pending_out);
}

lpa_status lpa_server_poll(lpa_server S, uint64_t ticket, int32_t* done, lpa_graph_stats* stats) {
  if (!S || !done) return fail(LPA_EINVAL, "NULL argument");
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(LPA_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  ServeReq* r = it->second;
  *done = r->state == 2;
  if (stats) {
    stats->iterations = r->iterations;
    stats->converged = r->converged;
    stats->edges_scanned = (int64_t)r->iterations * r->g.m;
    stats->modularity = 0.0;
  }
  if (r->state == 2) {
    S->reqs.erase(it);
    delete r;
  }
  return LPA_OK;
}

lpa_status lpa_server_drain(lpa_server S, uint64_t* tickets, int32_t cap, int32_t* count) {
  if (!S || !count || (cap > 0 && !tickets)) return fail(LPA_EINVAL, "NULL argument");
  const int32_t c = (int32_t)std::min<size_t>((size_t)std::max(cap, 0), S->finished.size());
  for (int32_t i = 0; i < c; ++i) tickets[i] = S->finished[i];
  S->finished.erase(S->finished.begin(), S->finished.begin() + c);
  *count = c;
  return LPA_OK;
}

lpa_status lpa_release_memory(void) {
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    for (char* b : g_host_free) cudaFreeHost(b);
    g_host_free.clear();
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (int d = 0; d < kMaxDevices; ++d)
    if (g_pools[d]) {
      cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
      if (e != cudaSuccess) return fail(LPA_ECUDA, "cudaMemPoolTrimTo: %s", cudaGetErrorString(e));
    }
  return LPA_OK;
}

lpa_status lpa_server_destroy(lpa_server S) {
  if (!S) return LPA_OK;
  free_packing(S->pk, S->stream);
  if (S->d_err) cudaFreeAsync(S->d_err, S->stream);
  cudaStreamSynchronize(S->stream);
  if (S->h_state) cudaFreeHost(S->h_state);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
  return LPA_OK;
}

}  // extern "C"
