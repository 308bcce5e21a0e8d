// lpa_batch.cu -- the batched form: many independent graphs swept as one block-diagonal
// graph.  Graph g's vertices take ids [vb_g, vb_g + n_g) and its CSR entries positions
// [eb_g, eb_g + m_g) of the packed arrays; neighbour ids (and so labels) are shifted by
// vb_g.  The shift is monotone inside a graph, so every tie-break and pick-less test
// (Sec. 4.4, 4.5) decides as it would for the graph alone, and a graph's sweeps read only
// its own labels.  Each graph keeps its own dN, iteration count and stop test (Alg. 1);
// a stopped graph's vertices keep their labels while the others continue.
#include "lpa_internal.cuh"

namespace lpa {
namespace {

// Upper bound: the last g with base[g] <= x (base ascending, base[0] = 0).
__device__ __forceinline__ int find_graph(const int64_t* __restrict__ base, int count, int64_t x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Offsets and graph ids of the packed vertices; with validate, checks each graph's
// offsets (first 0, non-decreasing, last = m_g).
__global__ void pack_offsets_kernel(const BatchGraph* __restrict__ gs, const int64_t* __restrict__ vb,
                                    int count, int64_t nv, int64_t* off, int32_t* gid, int g0,
                                    int validate, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    // graphs with n_g = 0 share a base with the next one; find_graph takes the last
    const int g = find_graph(vb, count, v);
    const BatchGraph G = gs[g];
    const int64_t i = v - vb[g];
    const int64_t o0 = G.off[i], o1 = G.off[i + 1];
    off[v] = o0 + G.eb;
    gid[v] = g0 + g;
    if (validate && ((i == 0 && o0 != 0) || o1 < o0 || (i + 1 == G.n && o1 != G.m)))
      atomicOr(err, kErrOffsets);
  }
}

// Indices (shifted by the graph's vertex base) and weights (1 for unweighted graphs) of
// the packed entries; with validate, checks index range and weight values.
__global__ void pack_edges_kernel(const BatchGraph* __restrict__ gs, const int64_t* __restrict__ eb,
                                  int count, int64_t ne, int32_t* idx, float* w, int validate,
                                  int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    const int g = find_graph(eb, count, e);
    const BatchGraph G = gs[g];
    const int64_t q = e - eb[g];
    const int32_t j = G.idx[q];
    const float x = G.w ? G.w[q] : 1.f;
    if (validate) {
      if (j < 0 || j >= G.n) atomicOr(err, kErrIndex);
      if (!(x >= 0.f) || isinf(x)) atomicOr(err, kErrWeight);
    }
    idx[e] = (int32_t)(j + G.vb);
    if (w) w[e] = x;
  }
}

// Per-graph run state before iteration 0: empty graphs are converged with 0 iterations.
__global__ void batch_init_kernel(const BatchGraph* __restrict__ gs, int count, int32_t* gdone,
                                  int32_t* giter, int32_t* gconv, int32_t* active, DevState* st) {
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < count; g += blockDim.x) {
    const int empty = gs[g].n == 0;
    gdone[g] = empty;
    gconv[g] = empty;
    giter[g] = 0;
    if (!empty) atomicAdd(&s_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *active = s_active;
    st->done = s_active == 0;
    st->converged = s_active == 0;
    st->iterations = 0;
  }
}

// After sweep l: every running graph counts the sweep and applies the stop test of
// Alg. 1 to its own dN; the run stops once no graph is running.  One block, so the
// "did sweep l run" test reads the state before any graph of this launch stops.
__global__ void batch_converge_kernel(const BatchGraph* __restrict__ gs, int count,
                                      const uint32_t* __restrict__ gdn_l, int32_t* gdone,
                                      int32_t* giter, int32_t* gconv, int32_t* active, DevState* st,
                                      int l, int pick_less, double tol) {
  __shared__ int s_ran, s_stopped;
  if (threadIdx.x == 0) {
    s_ran = !st->done;
    s_stopped = 0;
  }
  __syncthreads();
  if (!s_ran) return;
  for (int g = threadIdx.x; g < count; g += blockDim.x) {
    if (gdone[g]) continue;
    giter[g] = l + 1;
    if (!pick_less && (double)gdn_l[g] / (double)gs[g].n < tol) {
      gdone[g] = 1;
      gconv[g] = 1;
      atomicAdd(&s_stopped, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->iterations = l + 1;
    *active -= s_stopped;
    if (*active == 0) {
      st->done = 1;
      st->converged = 1;
    }
  }
}

// Final labels back to each graph's own ids: out_g[v - vb_g] = C[v] - vb_g.
__global__ void unpack_labels_kernel(const BatchGraph* __restrict__ gs, const int32_t* __restrict__ gid,
                                     const int32_t* __restrict__ c, int64_t nv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    const BatchGraph G = gs[gid[v]];
    G.out[v - G.vb] = (int32_t)(c[v] - G.vb);
  }
}

// Served form, after one sweep of every resident graph: graph g counts its sweep, applies
// its own stop test (its own pick-less setting and iteration number, Alg. 1) or stops at
// max_iter, and sets its pick-less flag for its next sweep.  gfin marks the graphs that
// stopped in this sweep.
__global__ void serve_converge_kernel(const BatchGraph* __restrict__ gs, int count,
                                      const uint32_t* __restrict__ gdn, int32_t* gdone,
                                      int32_t* giter, int32_t* gconv, int32_t* gpl, int32_t* gfin,
                                      int max_iter, int rho, double tol) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count || gdone[g]) return;
  const int l = giter[g];  // sweeps done before this one
  giter[g] = l + 1;
  const bool stop = !gpl[g] && (double)gdn[g] / (double)gs[g].n < tol;
  if (stop || l + 1 >= max_iter) {
    gdone[g] = 1;
    gconv[g] = stop;
    gfin[g] = 1;
  }
  gpl[g] = (rho > 0 && (l + 1) % rho == 0) ? 1 : 0;
}

// Re-packed graphs: vertices [v0, v0 + nv) of the new packing (gid and c_new point at
// v0); a graph that was resident before (old_vb[g] >= 0) carries its labels over,
// shifted to its new base; a new graph starts from C[v] = v.
__global__ void carry_labels_kernel(const BatchGraph* __restrict__ gs,
                                    const int64_t* __restrict__ old_vb, const int32_t* __restrict__ gid,
                                    const int32_t* __restrict__ c_old, int32_t* c_new, int64_t v0,
                                    int64_t nv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const int g = gid[i];
    const int64_t v = v0 + i, ob = old_vb[g], nb = gs[g].vb;
    c_new[i] = ob < 0 ? (int32_t)v : (int32_t)(c_old[ob + (v - nb)] - ob + nb);
  }
}

// Labels of the graphs that stopped in this sweep back to their own outputs.
__global__ void unpack_finished_kernel(const BatchGraph* __restrict__ gs, const int32_t* __restrict__ gid,
                                       const int32_t* __restrict__ gfin, const int32_t* __restrict__ c,
                                       int64_t nv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    const int g = gid[v];
    if (!gfin[g]) continue;
    const BatchGraph G = gs[g];
    G.out[v - G.vb] = (int32_t)(c[v] - G.vb);
  }
}

// p[i] = start + i: the initial labels C[v] = v of vertices appended at base start.
__global__ void iota_i32_kernel(int32_t* p, int64_t start, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    p[i] = (int32_t)(start + i);
}

inline unsigned grid_of(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (unsigned)(g < 152 * 32 ? (g > 0 ? g : 1) : 152 * 32);
}

}  // namespace

cudaError_t launch_pack_batch(const BatchGraph* gs, const int64_t* vb, const int64_t* eb, int count,
                              int64_t nv, int64_t ne, int64_t* off, int32_t* idx, float* w,
                              int32_t* gid, int g0, bool validate, int32_t* err, cudaStream_t s) {
  if (nv > 0) {
    pack_offsets_kernel<<<grid_of(nv), 256, 0, s>>>(gs, vb, count, nv, off, gid, g0, validate, err);
    count_launch();
  }
  if (ne > 0) {
    pack_edges_kernel<<<grid_of(ne), 256, 0, s>>>(gs, eb, count, ne, idx, w, validate, err);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_init(const BatchGraph* gs, int count, int32_t* gdone, int32_t* giter,
                              int32_t* gconv, int32_t* active, DevState* st, cudaStream_t s) {
  batch_init_kernel<<<1, 1024, 0, s>>>(gs, count, gdone, giter, gconv, active, st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_converge(const BatchGraph* gs, int count, const uint32_t* gdn_l,
                                  int32_t* gdone, int32_t* giter, int32_t* gconv, int32_t* active,
                                  DevState* st, int l, int pick_less, double tol, cudaStream_t s) {
  batch_converge_kernel<<<1, 1024, 0, s>>>(gs, count, gdn_l, gdone, giter, gconv, active, st, l,
                                           pick_less, tol);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_unpack_labels(const BatchGraph* gs, const int32_t* gid, const int32_t* c,
                                 int64_t nv, cudaStream_t s) {
  if (nv == 0) return cudaSuccess;
  unpack_labels_kernel<<<grid_of(nv), 256, 0, s>>>(gs, gid, c, nv);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_iota_i32(int32_t* p, int64_t start, int64_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  iota_i32_kernel<<<grid_of(count), 256, 0, s>>>(p, start, count);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_serve_converge(const BatchGraph* gs, int count, const uint32_t* gdn,
                                  int32_t* gdone, int32_t* giter, int32_t* gconv, int32_t* gpl,
                                  int32_t* gfin, int max_iter, int rho, double tol,
                                  cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  serve_converge_kernel<<<(count + 255) / 256, 256, 0, s>>>(gs, count, gdn, gdone, giter, gconv,
                                                             gpl, gfin, max_iter, rho, tol);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_carry_labels(const BatchGraph* gs, const int64_t* old_vb, const int32_t* gid,
                                const int32_t* c_old, int32_t* c_new, int64_t v0, int64_t nv,
                                cudaStream_t s) {
  if (nv == 0) return cudaSuccess;
  carry_labels_kernel<<<grid_of(nv), 256, 0, s>>>(gs, old_vb, gid, c_old, c_new, v0, nv);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_unpack_finished(const BatchGraph* gs, const int32_t* gid, const int32_t* gfin,
                                   const int32_t* c, int64_t nv, cudaStream_t s) {
  if (nv == 0) return cudaSuccess;
  unpack_finished_kernel<<<grid_of(nv), 256, 0, s>>>(gs, gid, gfin, c, nv);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lpa
