// lpa_internal.cuh -- definitions shared by the library's translation units.
//
// Work decomposition of one sweep (the move step of Alg. 1):
//   * sketch modes (MG, BM): the window binning below.  Hubs take a CTA each (one leaf
//     per thread; leaves merge by shuffles within a warp and through shared memory
//     across warps); every other vertex takes L consecutive lanes of the lane kernel, one
//     leaf (partial sketch, Sec. 4.3) per lane, merged by warp shuffles.  Merges always
//     follow the stride-doubling order, so results never depend on the path.
//   * exact mode: "chunks", runs of consecutive vertices whose rows together fit one
//     CTA's shared-memory table (cost <= kChunkCapExact), and hubs with global tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace lpa {

constexpr int kThreads = 256;          // threads per CTA; also max leaves per chunk
constexpr int kLaneThreads = 128;      // threads per CTA of the lane sweep
constexpr int kChunkCap = 4096;        // sketch modes: max chunk cost (>= its edges)
constexpr int kChunkCapExact = 2048;   // exact mode: its smem table needs 2 slots/edge
constexpr int kMaxWarpLeaves = 32;     // vertices with more leaves become hubs
constexpr int kSegment = 2048;         // vertices per thread of the greedy binning
constexpr int kMaxLeaves = 256;        // largest leaf_max accepted

// Binning of the warp-per-row sweep (sketch modes).  Vertices are cut into windows of
// `win` consecutive ids (kWinVerts unless a tuning picks a smaller power of two).  Inside a window they are counting-sorted into hubs (rows
// longer than kHubDegree or with more than 32 leaves), then kMidClasses mid classes
// (2..32 leaves, by leaf count descending, then leaf-length quarter), then one-leaf (low)
// rows by degree, descending.  Mid and low vertices are packed onto consecutive lanes, L
// lanes for a vertex of L leaves: as L only decreases along the order and divides 32,
// each vertex's lanes start at a multiple of L and stay inside one warp.  Each window's
// lanes are padded to whole warps and the windows' lanes concatenated in id order, one
// 16-byte descriptor per lane, so a thread finds its work with one load and rows swept at
// the same time share neighbour-label ranges in L2.  The grid runs every hub first (a CTA
// each), then the lanes, kThreads to a CTA.
constexpr int kWinVerts = 16384;      // default window (lpa_tuning.window)
constexpr int kWinVertsMin = 2048;    // smallest window a tuning may choose
constexpr int kLowKeys = 1024;         // low-row sort keys (degree, capped)
constexpr int kMidSub = 4;             // leaf-length quarters per leaf count
constexpr int kMidClasses = 5 * kMidSub;
constexpr int kLaneGroups = kMidClasses + 1;  // mid classes, then the low rows
// Hubs are grouped by their CTA size, max(32, L) = 256 >> c for class c, so a hub of 64
// leaves runs in a 64-thread CTA instead of idling three quarters of a 256-thread one.
constexpr int kHubClasses = 4;
constexpr int kSortKeys = kHubClasses + kMidClasses + kLowKeys;
constexpr int kHubDegree = 4096;
// Per-window table (kWinTab int32): [0] hub count; [kTabLane + g] first lane of lane group
// g; [kTabLanes] lanes in use; [kTabVert + g] window slot of group g's first vertex;
// [kTabHub + c] window slot of hub class c's first hub.
constexpr int kTabLane = 1;
constexpr int kTabLanes = kTabLane + kLaneGroups;
constexpr int kTabVert = 24;
constexpr int kTabHub = kTabVert + kLaneGroups;
constexpr int kWinTab = 52;
static_assert(kTabLanes < kTabVert && kTabHub + kHubClasses <= kWinTab, "window table layout");
// Lane descriptor word w: leaf length (< 2^13, rows of a lane have <= kHubDegree
// positions), leaf index, log2 of the vertex's leaf count.
constexpr int kLaneLeafShift = 13;
constexpr int kLaneLgShift = 18;
static_assert(kHubDegree < (1 << kLaneLeafShift), "leaf length field");
constexpr int kDnSlots = 64;           // dN is spread over this many counters

enum Mode { kExact = 0, kMG = 1, kBM = 2 };

// Device-resident state of one run (lives at the start of the workspace).
struct DevState {
  int32_t done;        // set once the run has converged; later sweeps exit at once
  int32_t iterations;  // sweeps performed so far
  int32_t converged;
  int32_t err;         // validation error bits (kErr*)
  int64_t nchunks;     // binning totals
  int64_t nhubs;
  int64_t hub_edges;
  int64_t pad;
};

enum : int32_t {
  kErrOffsets = 1,   // offsets[0] != 0, offsets[n] != m or a decreasing step
  kErrIndex = 2,     // an index outside [0, n)
  kErrWeight = 4,    // a weight that is negative, infinite or NaN
  kErrLabels = 8,    // a labels_in value outside [0, n)
};

// Number of leaves of a row of d positions (the partition fixed in lpa.h).
__host__ __device__ __forceinline__ int leaf_count(int64_t d, int e0, int lmax) {
  if (d < 2 * (int64_t)e0) return 1;
  int64_t q = d / e0;  // >= 2
  int64_t p = 1;
#if defined(__CUDA_ARCH__)
  p = (int64_t)1 << (63 - __clzll(q));
#else
  while (2 * p <= q) p *= 2;
#endif
  return (int)(p < lmax ? p : lmax);
}

// Weight formats of the sliced copy: unit weights (no weight array) or fp32 weights in
// sl_w.
enum WFmt : int { kUnitW = 0, kSplitW = 1 };

// Sliced copy of the CSR (built once per plan).  A leaf's positions, in CSR order, are
// cut into ceil(len / 4) groups of four; each group is one 16-byte element of sl_idx and
// of sl_w, so the lanes of a warp read their groups side by side instead of 32 separate
// rows.  An index of -1 marks a position no vote comes from (a self-loop, a weight that
// is not positive, padding past the leaf's end, weight 0), so the sweep tests one sign.
//  * lane warps: column k of a warp holds group k of every lane that has one, in lane
//    order (a warp vote gives each lane its place), so a warp's slice has exactly the
//    groups of its lanes; lane_base[w] is its first element.
//  * hubs of L leaves: width W = min(32, L); group k of leaf t sits at
//    hub_base[h] + (t / 32) * W * G + k * W + t % 32, with G = ceil(ceil(d / L) / 4) the
//    groups of the longest leaf.
struct WarpPlan {
  const int4* hub_desc;   // per hub: {v, offset lo, offset hi, degree}, grouped by class
  const int4* lane_desc;  // per lane (see kLaneLeafShift); v = -1 on padding lanes
  const int4* sl_idx;     // sliced copy of the indices
  const float4* sl_w;     // sliced copy of the weights (null: unit weights)
  const int64_t* lane_base;  // first sliced element of each lane warp
  const int64_t* hub_base;   // first sliced element of each hub (in hub_desc order)
  int64_t nlanes;         // a multiple of 32
  int32_t nhubs;
  int32_t nctas;          // nhubs + ceil(nlanes / kThreads) (work units, for the stats)
  int32_t e0, lmax;       // the leaf partition the plan was binned with
  int32_t wfmt;           // WFmt of the sliced copy
  int32_t lane_threads;   // CTA size of the lane sweep (lpa_tuning)
  int32_t hub_start[kHubClasses + 1];  // first hub of each class; [kHubClasses] = nhubs
};

// Groups of four positions a hub leaf is padded to (the longest of its L leaves).
__host__ __device__ __forceinline__ int64_t hub_leaf_groups(int64_t d, int L) {
  return ((d + L - 1) / L + 3) / 4;
}

// Arguments of one sweep launch.
struct SweepArgs {
  const int64_t* off;
  const int32_t* idx;
  const float* w;  // may be null when the kernel is instantiated for unit weights
  const int32_t* c_prev;
  int32_t* c_next;
  const int32_t* chunk_v0;
  const int32_t* chunk_v1;
  const int32_t* hubs;
  const int64_t* hub_tab;  // exact mode: table offset of each hub
  int32_t* tab_keys;       // exact mode: hub tables (global)
  float* tab_vals;
  unsigned long long* dn;  // dN counters of this sweep (kDnSlots for the warp kernels)
  const int32_t* done;     // skip the sweep if *done (null: never)
  // Pruning (the unprocessed flags of Alg. 1), null when off: only vertices with
  // act_in[v] != 0 are swept (the rest keep their label); a vertex whose label changes
  // sets act_out[j] = 1 for every j in its row; scanned (kDnSlots counters) receives
  // the CSR positions of the swept rows.
  const uint8_t* act_in;
  uint8_t* act_out;
  unsigned long long* scanned;
  // Batched form, null otherwise: vertex v belongs to graph gid[v]; a graph with
  // gdone[g] != 0 has stopped (its vertices keep their labels); gdn[g] counts the
  // graph's changed labels of this sweep.
  const int32_t* gid;
  const int32_t* gdone;
  uint32_t* gdn;
  // Served form, null otherwise: graph g's own pick-less setting for this sweep
  // (graphs that joined at different sweeps are at different iterations).
  const int32_t* gpl;
  int32_t nchunks;
  int32_t nhubs;
  int32_t pick_less;
  int32_t e0;
  int32_t lmax;
  int64_t m;
};

// One graph of a batch (device table): its caller arrays, output, and its vertex and
// CSR-entry bases in the packed block-diagonal graph.
struct BatchGraph {
  const int64_t* off;
  const int32_t* idx;
  const float* w;   // null: unit weights
  int32_t* out;     // labels_out of the graph
  int64_t vb, eb;
  int64_t m;
  int32_t n;
  int32_t pad;
};

// Arguments of the degree binning.
struct BinArgs {
  const int64_t* off;
  int32_t n;
  int32_t cap;          // chunk cost capacity
  int32_t cost_floor;   // cap / kThreads: bounds vertices and leaves per chunk
  int32_t e0, lmax;
  int32_t leaves;       // 0 for exact mode (leaves do not apply)
  int64_t* seg_chunks;  // per segment counts, then exclusive prefix
  int64_t* seg_hubs;
  int64_t* seg_hub_edges;
  int32_t* chunk_v0;    // written by the second pass
  int32_t* chunk_v1;
  int32_t* hubs;
  int64_t* hub_tab;
};

// Host-side launchers (stream-ordered, no synchronisation).
// Sketch modes (MG, BM): hub and lane kernels over a WarpPlan (its weight format decides
// the instantiation).  The hub kernel goes to s_hub, the lane kernel to s.
cudaError_t launch_sweep_warp(int mode, int k, const SweepArgs& a, const WarpPlan& p,
                              cudaStream_t s, cudaStream_t s_hub);
cudaError_t launch_sweep_mg16(const SweepArgs& a, const WarpPlan& p, cudaStream_t s,
                              cudaStream_t s_hub);
cudaError_t launch_sweep_mg32(const SweepArgs& a, const WarpPlan& p, cudaStream_t s,
                              cudaStream_t s_hub);
// MG ablations (at least one of literal, rescan set): paper-literal accumulate and / or
// double scan, hub kernel on s_hub and lane kernel on s as launch_sweep_warp.
cudaError_t launch_sweep_mg_variant(int k, bool literal, bool rescan, const SweepArgs& a,
                                    const WarpPlan& p, cudaStream_t s, cudaStream_t s_hub);
cudaError_t launch_sweep_mg16_variant(bool literal, bool rescan, const SweepArgs& a,
                                      const WarpPlan& p, cudaStream_t s, cudaStream_t s_hub);
cudaError_t launch_sweep_mg32_variant(bool literal, bool rescan, const SweepArgs& a,
                                      const WarpPlan& p, cudaStream_t s, cudaStream_t s_hub);
// Weight profile: out[0] = 1 if every weight is integer-valued (AND), out[1] = largest
// weight's bits, out[2] = largest row length.  out must be zeroed except out[0] = 1.
cudaError_t launch_weight_profile(const int64_t* off, const float* w, int32_t n, int64_t m,
                                  unsigned long long* out, cudaStream_t s);
// Exact mode: chunk kernel over the chunk/hub binning.
cudaError_t launch_sweep_exact(bool weighted, const SweepArgs& a, cudaStream_t s);
size_t exact_smem_bytes(bool weighted);
// Binning for the warp-per-row kernels.  Per window: sort the vertices into groups, write
// their descriptors, the window table, the hub count of each class (class-major:
// hcnt[c * nwin + window]) and the padded lane count.
// Windows w_first .. ceil(n / win) - 1 only (the tables of earlier windows are kept);
// hub counts are class-major with stride hstride (>= the number of windows).
cudaError_t launch_window_sort(const int64_t* off, int32_t n, int e0, int lmax, int win,
                               int32_t w_first, int64_t hstride, int4* desc, int32_t* wtab,
                               int32_t* hcnt, int32_t* lcnt, cudaStream_t s);
// prefix[0, len] = exclusive prefix sums of cnt[0, len), prefix[len] the total.  With
// tiles (scan_tile_slots(len) int64 scratch) long arrays are scanned by many CTAs.
cudaError_t launch_scan_counts(const int32_t* cnt, int64_t len, int64_t* prefix, cudaStream_t s,
                               int64_t* tiles = nullptr);
inline int64_t scan_tile_slots(int64_t len) { return len / 8192 + 2; }
// Hub and lane descriptors of every window at their prefix offsets (hub_prefix over the
// class-major hub counts; capacities bound the writes).
// Every window's hubs; lanes of windows w_lanes .. nwin - 1 only.
cudaError_t launch_expand_lanes(const int4* desc, const int32_t* wtab, const int64_t* hub_prefix,
                                const int64_t* lane_prefix, int32_t nwin, int win, int64_t hstride,
                                int32_t w_lanes, int4* hub_desc, int64_t hub_cap, int4* lane_desc,
                                int64_t lane_cap, cudaStream_t s);
// Sliced copy of the CSR for a binned plan (lpa_setup.cu), for the lanes from lane_from
// on (a multiple of 32; the slices of the lanes before it are kept) and every hub.  Pass 1
// counts each lane warp's groups into lane_cnt and each hub's into hub_cnt, continues
// lane_base (lanes grow from element 0 up; lane_base[nlanes / 32] ends them) and fills
// hub_base (hubs fill the top of `cap` elements downwards; hub_pre[nhubs] is their total).
// Pass 2 (after the host has checked the totals against cap) copies the positions.
cudaError_t launch_slice_count(const WarpPlan& p, int e0, int lmax, int64_t lane_from,
                               int32_t* lane_cnt, int32_t* hub_cnt, int64_t* scan_tmp,
                               int64_t* tiles, int64_t* lane_base, int64_t* hub_pre,
                               int64_t* hub_base, int64_t cap, cudaStream_t s);
cudaError_t launch_slice_fill(const int32_t* idx, const float* w, int64_t m, const WarpPlan& p,
                              int e0, int lmax, int64_t lane_from, int4* sl_idx, float4* sl_w,
                              cudaStream_t s);
// Whether the sweeps are built with every lane CTA size of lpa_tuning (MG with k = 8 and
// BM; the other sketches and the MG ablations use the default).
inline bool full_tuning_sketch(int mode, int k) { return mode == kBM || (mode == kMG && k == 8); }
// Modularity over a WarpPlan: rows, then Sigma_c^2; out4 as launch_modularity.  With gid
// (a batch), each graph's 2m and intra-community weight also accumulate into g2m / gin
// (zeroed by the caller).
cudaError_t launch_modularity_plan(const int64_t* off, const int32_t* idx, const float* w,
                                   int64_t m, const int32_t* labels, int32_t n,
                                   const WarpPlan& p, double* sigma_c, double* partials,
                                   int64_t npart, double* out4, cudaStream_t s,
                                   const int32_t* gid = nullptr, double* g2m = nullptr,
                                   double* gin = nullptr);
int64_t modularity_plan_partials(const WarpPlan& p, int32_t n);

cudaError_t launch_dn_sum(const unsigned long long* slots, unsigned long long* out,
                          cudaStream_t s);
cudaError_t launch_validate(const int64_t* off, const int32_t* idx, const float* w,
                            int32_t n, int64_t m, const int32_t* labels_in, int32_t* err,
                            cudaStream_t s);
cudaError_t launch_bin(const BinArgs& b, DevState* st, cudaStream_t s, bool write_pass);
cudaError_t launch_init_labels(int32_t* c, const int32_t* labels_in, int32_t n,
                               cudaStream_t s);
// dn: kDnSlots counters per iteration; the test sums iteration l's slots into dn_total[l]
// (and, when scanned is not null, iteration l's scanned slots into scan_total[l]).
cudaError_t launch_converge(DevState* st, const unsigned long long* dn,
                            unsigned long long* dn_total, const unsigned long long* scanned,
                            unsigned long long* scan_total, int l, int pick_less, double tol,
                            int32_t n, cudaStream_t s);
cudaError_t launch_fill_u8(uint8_t* p, uint8_t value, int64_t count, cudaStream_t s);
cudaError_t launch_finalize(const DevState* st, int32_t* out, const int32_t* tmp,
                            int32_t n, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t* p, int32_t value, int64_t count, cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long* p, unsigned long long value, int64_t count,
                            cudaStream_t s);
// Modularity without a plan (lpa_modularity.cu): out4 receives {2m, sum of
// intra-community weight, sum_c Sigma_c^2, Q}.  sigma_c: n doubles; partials: 3 * npart
// doubles with npart = modularity_partials(n).  Neither needs clearing.
cudaError_t launch_modularity(const int64_t* off, const int32_t* idx, const float* w, int64_t m,
                              const int32_t* labels, int32_t n, double* sigma_c,
                              double* partials, int32_t npart, double* out4, cudaStream_t s);
int modularity_partials(int32_t n);

inline int64_t num_segments(int64_t n) { return (n + kSegment - 1) / kSegment; }

// Batched form (lpa_batch.cu).  vb / eb: count + 1 ascending vertex / entry bases.
// gs[0, count) are written from packed vertex / entry 0 of off / idx / w / gid (callers
// appending to a packing pass pointers past its used part); gid = g0 + g; vb / eb are
// count + 1 bases relative to those pointers, while gs[g].vb / eb are absolute.
cudaError_t launch_pack_batch(const BatchGraph* gs, const int64_t* vb, const int64_t* eb, int count,
                              int64_t nv, int64_t ne, int64_t* off, int32_t* idx, float* w,
                              int32_t* gid, int g0, bool validate, int32_t* err, cudaStream_t s);
cudaError_t launch_iota_i32(int32_t* p, int64_t start, int64_t count, cudaStream_t s);
cudaError_t launch_batch_init(const BatchGraph* gs, int count, int32_t* gdone, int32_t* giter,
                              int32_t* gconv, int32_t* active, DevState* st, cudaStream_t s);
cudaError_t launch_batch_converge(const BatchGraph* gs, int count, const uint32_t* gdn_l,
                                  int32_t* gdone, int32_t* giter, int32_t* gconv, int32_t* active,
                                  DevState* st, int l, int pick_less, double tol, cudaStream_t s);
cudaError_t launch_unpack_labels(const BatchGraph* gs, const int32_t* gid, const int32_t* c,
                                 int64_t nv, cudaStream_t s);
// Per-graph Q after launch_modularity_plan with gid (lpa_modularity.cu).
cudaError_t launch_batch_q(const BatchGraph* gs, int count, const double* sigma_c, const double* g2m,
                           const double* gin, double* gq, cudaStream_t s);

// Served form (lpa_batch.cu): per-graph stop test after a sweep, label carry-over into a
// new packing (old_vb[g] < 0 for a new graph; gid and c_new point at vertex v0), output
// of the graphs that stopped.
cudaError_t launch_serve_converge(const BatchGraph* gs, int count, const uint32_t* gdn,
                                  int32_t* gdone, int32_t* giter, int32_t* gconv, int32_t* gpl,
                                  int32_t* gfin, int max_iter, int rho, double tol,
                                  cudaStream_t s);
cudaError_t launch_carry_labels(const BatchGraph* gs, const int64_t* old_vb, const int32_t* gid,
                                const int32_t* c_old, int32_t* c_new, int64_t v0, int64_t nv,
                                cudaStream_t s);
cudaError_t launch_unpack_finished(const BatchGraph* gs, const int32_t* gid, const int32_t* gfin,
                                   const int32_t* c, int64_t nv, cudaStream_t s);

// Record the message returned by lpa_last_error() on this host thread; returns s.
int set_last_error(int s, const char* msg);
// Argument checks shared by the modularity entry points (a status of lpa.h; the message
// is recorded as by set_last_error).
int check_modularity_args(const int64_t* offsets, const int32_t* indices, int32_t n, int64_t m,
                          const int32_t* labels, const double* q_out);

// Kernels launched by the library (counted at every launch site).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace lpa
