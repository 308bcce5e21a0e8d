// lpa_internal.cuh -- definitions shared by the library's translation units.
//
// Work decomposition of one sweep (the move step of Alg. 1):
//   * "chunks": runs of consecutive vertices whose rows together fit one CTA's
//     shared-memory stage (cost <= kChunkCap, see binning below).  A CTA stages the
//     chunk's (neighbour label, weight) pairs edge-parallel, then every thread folds
//     one leaf (partial sketch, Sec. 4.3) from shared memory, and leaves of one vertex
//     merge by warp shuffles.
//   * "hubs": vertices whose row is longer than a chunk, or that have more than 32
//     leaves.  One CTA per hub; each thread folds one leaf straight from global
//     memory; leaves merge by shuffles within a warp and through shared memory across
//     warps, always in the stride-doubling order, so results never depend on the path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace lpa {

constexpr int kThreads = 256;          // threads per CTA; also max leaves per chunk
constexpr int kChunkCap = 4096;        // sketch modes: max chunk cost (>= its edges)
constexpr int kChunkCapExact = 2048;   // exact mode: its smem table needs 2 slots/edge
constexpr int kMaxWarpLeaves = 32;     // vertices with more leaves become hubs
constexpr int kSegment = 2048;         // vertices per thread of the greedy binning
constexpr int kMaxLeaves = 256;        // largest leaf_max accepted

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
  unsigned long long* dn;  // dN counter of this sweep
  const int32_t* done;     // skip the sweep if *done (null: never)
  int32_t nchunks;
  int32_t nhubs;
  int32_t pick_less;
  int32_t e0;
  int32_t lmax;
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
cudaError_t launch_sweep(int mode, int k, bool weighted, const SweepArgs& a,
                         cudaStream_t s);
size_t sweep_smem_bytes(int mode, bool weighted);
cudaError_t launch_validate(const int64_t* off, const int32_t* idx, const float* w,
                            int32_t n, int64_t m, const int32_t* labels_in, int32_t* err,
                            cudaStream_t s);
cudaError_t launch_bin(const BinArgs& b, DevState* st, cudaStream_t s, bool write_pass);
cudaError_t launch_init_labels(int32_t* c, const int32_t* labels_in, int32_t n,
                               cudaStream_t s);
cudaError_t launch_converge(DevState* st, const unsigned long long* dn, int l,
                            int pick_less, double tol, int32_t n, cudaStream_t s);
cudaError_t launch_finalize(const DevState* st, int32_t* out, const int32_t* tmp,
                            int32_t n, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t* p, int32_t value, int64_t count, cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long* p, unsigned long long value, int64_t count,
                            cudaStream_t s);
// Modularity: out4 receives {2m, sum of intra-community weight, sum_c Sigma_c^2, Q}.
cudaError_t launch_modularity(const int64_t* off, const int32_t* idx, const float* w,
                              const int32_t* labels, int32_t n, double* sigma_c,
                              double* partials, int32_t npart, double* out3,
                              cudaStream_t s);
int modularity_partials(int32_t n);

inline int64_t num_segments(int64_t n) { return (n + kSegment - 1) / kSegment; }

// Record the message returned by lpa_last_error() on this host thread; returns s.
int set_last_error(int s, const char* msg);

// Kernels launched by the library (counted at every launch site).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace lpa
