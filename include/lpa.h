/*
 * lpa.h -- C ABI of the GB300 (sm_103a) label-propagation library.
 *
 * Community detection by label propagation (LPA, Sec. 3.3, Eq. 3) with the
 * memory-efficient label choice of arxiv 2411.19901: a k-slot weighted Misra-Gries
 * sketch per vertex (Sec. 4.1-4.4, Alg. 1-2), the weighted Boyer-Moore variant
 * (Sec. 4.7, Alg. 3) and an exact per-vertex table mode (the ν-LPA baseline, Sec. 4,
 * Fig. 1), plus modularity (Sec. 3.2, Eq. 1), pruning by unprocessed flags (Alg. 1),
 * the paper-literal sketch and double scan (ablations), and batched and served forms
 * for many graphs.
 *
 * Conventions for every entry point:
 *  - Graphs are CSR: offsets int64[n+1] (offsets[0] = 0, non-decreasing,
 *    offsets[n] = m), indices int32[m] in [0, n), weights fp32[m] finite and >= 0, or
 *    NULL for unit weights.  The graph must be symmetric (w_ij = w_ji, Sec. 3); this is
 *    not checked.  Self-loops are allowed: the sweep skips them (the scan of Alg. 1
 *    skips j = i), modularity counts them once as stored.  Edges of weight 0 carry no
 *    vote.  n < 2^31, m < 2^62.  indices and weights must start on a 16-byte boundary
 *    (the sweep reads them as 16-byte vectors; cudaMalloc and PyTorch allocations do),
 *    else LPA_EINVAL; lpa_graph entries of a batch or a server are exempt (copied).
 *  - Pointers are DEVICE memory owned by the caller unless marked "host".  The library
 *    frees nothing it did not allocate.
 *  - Calls are ordered on the caller's stream (lpa_options.stream; NULL = the legacy
 *    default stream) and return after the stream work they issued has finished.
 *  - Labels are int32 in [0, n): the initial label of vertex i is i (Alg. 1, `lpa`),
 *    or the caller's labels_in.
 *  - Results are deterministic: labels and per-iteration change counts do not depend
 *    on kernel shapes, launch order or the GPU's scheduling.  Iterations are
 *    synchronous: iteration l reads only the labels of iteration l-1.
 *  - Errors return a negative lpa_status, leave the outputs unspecified and set a
 *    thread-local message (lpa_last_error).  Without LPA_VALIDATE, an invalid graph
 *    (an index outside [0, n), offsets that are not monotone) is undefined behaviour.
 */
#ifndef LPA_H
#define LPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Label-choice rule.  LPA_EXACT: argmax of Eq. 3 (all neighbour labels).  LPA_MG: the
 * heaviest candidate of a k-slot weighted Misra-Gries sketch (Sec. 4.1, single scan of
 * Sec. 4.4).  LPA_BM: the weighted Boyer-Moore candidate (Sec. 4.7). */
typedef enum { LPA_EXACT = 0, LPA_MG = 1, LPA_BM = 2 } lpa_mode;

typedef enum {
  LPA_OK = 0,
  LPA_EINVAL = -1,        /* bad argument or (with LPA_VALIDATE) malformed graph */
  LPA_ENOMEM = -2,        /* device allocation failed or workspace too small */
  LPA_ECUDA = -3,         /* a CUDA runtime call failed (message in lpa_last_error) */
  LPA_ETIMEOUT = -4,      /* a bounded device wait gave up */
  LPA_EUNSUPPORTED = -5,  /* valid but not built (e.g. k not a power of two) */
  LPA_EINTERNAL = -6      /* internal consistency check failed */
} lpa_status;

/* Flags for lpa_options.flags. */
#define LPA_VALIDATE 0x1u /* check the CSR (and labels_in) on the device first */
#define LPA_TIMING 0x2u   /* time the sweep and binning kernels with CUDA events */
#define LPA_MODULARITY 0x4u /* also compute the modularity of the result (Eq. 1) */
/* Pruning by the unprocessed flags of Alg. 1, read synchronously: iteration 0 sweeps
 * every vertex; iteration l+1 sweeps only the vertices listed in the row of a vertex
 * whose label changed in iteration l, the others keep their label.  Fewer CSR
 * positions are read (lpa_stats.scanned_iter); with pick-less off the MG and exact
 * results equal the unpruned ones on symmetric graphs.  Runs only (lpa_detect*,
 * lpa_plan_run); lpa_plan_sweep ignores it. */
#define LPA_PRUNE 0x8u
/* MG ablations of the paper (LPA_MG only, else LPA_EINVAL).  LPA_MG_UNCLAMPED: the
 * accumulate exactly as printed in Alg. 2 for a private sketch -- a key match ignores
 * the slot's value, a full sketch subtracts w from every slot and drops the label, so
 * values may go negative; merges feed every slot of non-zero value; the choice is the
 * largest positive value.  LPA_RESCAN: the double scan of Sec. 4.4 -- after the
 * sketch, each candidate's exact K_{i->c} is summed (each leaf in CSR order, leaves
 * along the merge tree) and the heaviest, ties to the smallest label, is chosen. */
#define LPA_MG_UNCLAMPED 0x10u
#define LPA_RESCAN 0x20u
/* Record a run's launches as one CUDA graph and launch that (the driver loop of Alg. 1:
 * every sweep with its on-device stop test, the labels' final copy, the optional
 * modularity pass and the copies of the results to the host).  A plan keeps the
 * instantiated graph and replays it on the next lpa_plan_run with the same labels_out,
 * tol, max_iter and flags (a new combination records a new graph); lpa_detect*,
 * lpa_batch_detect (its sweeps and per-graph stop tests) record and launch a graph per
 * call.  Results are the same bits as without the flag.  The graph is recorded on a
 * stream of the library's own and launched on the caller's stream, so the legacy
 * default stream works too.  Not with LPA_TIMING (LPA_EINVAL): per-sweep events are not
 * timed inside a graph.  The server ignores the flag. */
#define LPA_GRAPH 0x40u

/* Largest max_iter accepted; lpa_stats.changed has this many entries. */
#define LPA_MAX_ITER 1024

/* Per-call statistics (HOST struct, filled on success). */
typedef struct {
  int32_t iterations;               /* sweeps performed */
  int32_t converged;                /* 1 if dN/N < tol stopped the run (Alg. 1) */
  int64_t changed[LPA_MAX_ITER];    /* dN of each performed sweep */
  int64_t edges_scanned;            /* CSR positions read by the sweeps */
  double seconds;                   /* host wall time of the call */
  double sweep_ms;                  /* device time of all sweeps (LPA_TIMING) */
  double setup_ms;                  /* device time of the degree binning (LPA_TIMING) */
  int64_t sweep_launches;           /* sweeps that did work (== iterations) */
  size_t device_bytes;              /* device workspace bytes used */
  int32_t chunks;                   /* CTA work units of the binned graph */
  int32_t hubs;                     /* vertices swept by a whole CTA */
  double modularity;                /* Q of the result (LPA_MODULARITY), else 0 */
  float sweep_ms_iter[LPA_MAX_ITER]; /* device time of each sweep (LPA_TIMING) */
  int64_t scanned_iter[LPA_MAX_ITER]; /* CSR positions swept by each sweep (m unless
                                         LPA_PRUNE) */
} lpa_stats;

/* Launch choices that never change a result: how the graph is binned and laid out for
 * the sketch-mode sweeps and how their kernels are launched.  An autotuner (the Python
 * binding's tune module) times candidates on a graph or batch and picks one; every
 * candidate gives the same labels and change counts bit for bit.  Zero in a field means
 * its default.  Exact mode ignores the struct. */
typedef struct {
  int32_t window;       /* vertices per binning window: a power of two in [2048, 16384];
                           0 = 16384 */
  int32_t lane_threads; /* threads per CTA of the lane sweep: 64, 128 or 256 (MG with k = 8
                           and BM; other sketches always use 128); 0 = 128 */
  int32_t serial_hubs;  /* 1: run the hub kernels on the caller's stream after the lane
                           kernel; 0 = on a second stream beside it */
} lpa_tuning;

/* Options.  Call lpa_options_init first; it sets the paper's defaults (Sec. 5.1.2). */
typedef struct {
  int32_t pl_period;        /* rho: pick-less every rho iterations from the first;
                               0 = never (Sec. 4.5).  Default 8. */
  int32_t leaf_e0;          /* e0: rows shorter than 2*e0 are one sequential sketch;
                               longer rows are split into L(d) partial sketches.
                               Default 64. */
  int32_t leaf_max;         /* Lmax: most partial sketches per row, power of two
                               <= 256.  Default 256. */
  uint32_t flags;           /* LPA_VALIDATE | LPA_TIMING | LPA_MODULARITY | LPA_PRUNE |
                               LPA_MG_UNCLAMPED | LPA_RESCAN | LPA_GRAPH.  Default
                               LPA_VALIDATE. */
  const int32_t* labels_in; /* device, n labels in [0, n) to start from; NULL = C[i]=i */
  void* stream;             /* cudaStream_t; NULL = legacy default stream */
  void* workspace;          /* device scratch of workspace_bytes bytes, 256-byte
                               aligned; NULL = allocated and freed by the call */
  size_t workspace_bytes;
  const lpa_tuning* tuning; /* host, read during the call (plans and servers keep a copy);
                               NULL = defaults */
} lpa_options;

/* Leaf partition used by the sketches (fixed, so the result never depends on launch
 * shapes): a row of d CSR positions has L(d) = 1 if d < 2*e0, else
 * min(Lmax, largest power of two p with p*e0 <= d) leaves; leaf l covers positions
 * [floor(l*d/L), floor((l+1)*d/L)) in CSR order and folds them into an empty sketch;
 * leaves merge by the stride-doubling tree S[l] <- merge(S[l], S[l+s]), s = 1, 2, ...,
 * where merge(A, B) accumulates B's occupied slots into A in slot order (partial
 * sketches merged into S[0], Sec. 4.3).  MG is clamped: when no slot matches and none
 * is free, all slots and the incoming weight drop by min(w, smallest slot) and a
 * remainder takes the lowest free slot (Sec. 4.1).  Ties go to the smallest label. */

void lpa_options_init(lpa_options* opt);

/* Run LPA to convergence (Alg. 1, `lpa`): at most max_iter (<= LPA_MAX_ITER)
 * synchronous sweeps; pick-less in iteration l iff rho > 0 and l mod rho == 0; stop
 * after a non-pick-less sweep with (double)dN / n < tol.  k: MG slots, one of 1, 2, 4,
 * 8, 16, 32 (ignored for EXACT and BM).  labels_out: device int32[n]; it may equal
 * labels_in.  stats: host, may be NULL.  Default options. */
lpa_status lpa_detect(const int64_t* offsets, const int32_t* indices, const float* weights,
                      int32_t n, int64_t m, lpa_mode mode, int32_t k, double tol,
                      int32_t max_iter, int32_t* labels_out, lpa_stats* stats);

/* lpa_detect with explicit options (opt may be NULL for the defaults). */
lpa_status lpa_detect_ex(const int64_t* offsets, const int32_t* indices,
                         const float* weights, int32_t n, int64_t m, lpa_mode mode,
                         int32_t k, double tol, int32_t max_iter, int32_t* labels_out,
                         lpa_stats* stats, const lpa_options* opt);

/* lpa_detect_ex for a graph held in HOST memory: offsets/indices/weights and
 * labels_out are host pointers (page-locked memory gives the fastest copies); the call
 * copies the graph to the device, runs, and copies the labels back.  opt->labels_in
 * and opt->workspace, if set, are device pointers as usual. */
lpa_status lpa_detect_host(const int64_t* offsets, const int32_t* indices,
                           const float* weights, int32_t n, int64_t m, lpa_mode mode,
                           int32_t k, double tol, int32_t max_iter, int32_t* labels_out,
                           lpa_stats* stats, const lpa_options* opt);

/* Modularity of labels (device int32[n], values in [0, n)), Eq. 1:
 * Q = sum_c [sigma_c / 2m - (Sigma_c / 2m)^2] with 2m the sum of all CSR weights,
 * sigma_c the weight of entries (i, j) with C_i = C_j = c and Sigma_c the summed
 * weighted degree of c's vertices; fp64 accumulation; Q = 0 when 2m = 0.
 * q_out: host. */
lpa_status lpa_modularity(const int64_t* offsets, const int32_t* indices,
                          const float* weights, int32_t n, int64_t m, const int32_t* labels,
                          double* q_out);

/* lpa_modularity with options (stream, workspace, LPA_VALIDATE; opt may be NULL). */
lpa_status lpa_modularity_ex(const int64_t* offsets, const int32_t* indices,
                             const float* weights, int32_t n, int64_t m,
                             const int32_t* labels, double* q_out, const lpa_options* opt);

/* Modularity for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is an interface convenience.  Some callers cannot, or must not,
 * allocate at the moment they ask for a result -- a host program whose own caching
 * allocator already holds nearly all device memory, or a latency-critical loop where
 * cudaMalloc / cudaFree would stall the GPU.  This call allocates nothing: its scratch
 * is a fixed device array inside the library (about 8 MB, held on every GPU that loads
 * the library until the process exits), so n must be <= LPA_NOALLOC_MAX_N; larger n
 * returns LPA_EINVAL.  Arguments and result are as for lpa_modularity_ex (opt may be
 * NULL: legacy default stream, LPA_VALIDATE on; workspace fields are ignored).
 * The first call on each device looks up the array's device address once (with that
 * device current); make that first call before any CUDA stream capture.  All calls
 * share the one array: calls that overlap on the GPU (other streams, other host
 * threads) race and give wrong results, so order them.  Each call clears what it needs,
 * so results never depend on an earlier call. */
#define LPA_NOALLOC_MAX_N (1 << 20)
lpa_status lpa_modularity_noalloc(const int64_t* offsets, const int32_t* indices,
                                  const float* weights, int32_t n, int64_t m,
                                  const int32_t* labels, double* q_out,
                                  const lpa_options* opt);

/* Device workspace an lpa_detect_ex call needs: an upper bound for any graph with these
 * sizes under the default options (leaf_e0 = 64, default tuning).  The sketch modes' lane
 * table grows as m / leaf_e0 and with smaller binning windows, so a call with other
 * options takes lpa_workspace_size_ex with them (opt == NULL: the defaults).  Both return
 * 0 for negative sizes, leaf_e0 < 1 or a tuning out of range.  The sketch modes' share is
 * about 40 B per vertex, 16 B per lane and the sliced copy of the graph (16 B per group
 * of four CSR positions for the indices, as much again for fp32 weights).
 * lpa_modularity_ex needs lpa_modularity_workspace_size(n). */
size_t lpa_workspace_size(int32_t n, int64_t m, lpa_mode mode, int32_t k);
size_t lpa_workspace_size_ex(int32_t n, int64_t m, lpa_mode mode, int32_t k,
                             const lpa_options* opt);
size_t lpa_modularity_workspace_size(int32_t n);

/* ---- Plans: bin a graph once, then run sweeps or whole runs on it. ---------------
 * A plan keeps device pointers to the caller's graph (which must outlive it) and its
 * own workspace.  lpa_plan_create performs the degree binning on the device. */
typedef struct lpa_plan_s* lpa_plan;

lpa_status lpa_plan_create(const int64_t* offsets, const int32_t* indices,
                           const float* weights, int32_t n, int64_t m, lpa_mode mode,
                           int32_t k, const lpa_options* opt, lpa_plan* plan_out);

/* One synchronous sweep (Alg. 1, `lpaMove`): c_next[i] = the label vertex i chooses
 * from c_prev, committed only if it differs and, when pick_less != 0, is smaller.
 * c_prev and c_next are device int32[n] and must not overlap.  dn_out (host, may be
 * NULL) receives dN; with dn_out == NULL the call does not wait for the sweep. */
lpa_status lpa_plan_sweep(lpa_plan plan, const int32_t* c_prev, int32_t* c_next,
                          int32_t pick_less, int64_t* dn_out);

/* A whole run on the plan's graph (as lpa_detect_ex after binning). */
lpa_status lpa_plan_run(lpa_plan plan, double tol, int32_t max_iter, int32_t* labels_out,
                        lpa_stats* stats);

lpa_status lpa_plan_destroy(lpa_plan plan);

/* ---- Batched form: many independent graphs in one call. ---------------------------
 * The graphs are packed into one block-diagonal graph on the device (graph g's vertex
 * ids shifted by the vertices of the graphs before it; the shift keeps every tie-break
 * and pick-less decision of the graph alone) and swept together; each graph keeps its
 * own dN, iteration count and stop test of Alg. 1, and a stopped graph's labels stay
 * fixed while the others continue.  Results equal one lpa_detect_ex call per graph.
 * Every pointer in lpa_graph is DEVICE memory owned by the caller; the array of
 * lpa_graph, stats and changed_out are HOST memory.  The call allocates its packed copy
 * of the graphs (about 12 B per CSR entry + 40 B per vertex) and frees it before
 * returning; opt->workspace and opt->labels_in are not used (labels_in must be NULL);
 * LPA_TIMING is ignored; LPA_VALIDATE checks every graph; LPA_MODULARITY fills each
 * graph's modularity (Eq. 1) in stats (sketch modes; with LPA_EXACT it is
 * LPA_EUNSUPPORTED). */
typedef struct {
  const int64_t* offsets;  /* device, n + 1 */
  const int32_t* indices;  /* device, m; 16-byte alignment not required here */
  const float* weights;    /* device, m, or NULL = unit weights */
  int32_t n;
  int64_t m;
  int32_t* labels_out;     /* device, n: the graph's labels in its own ids */
} lpa_graph;

typedef struct {
  int32_t iterations;      /* sweeps the graph took part in */
  int32_t converged;       /* 1 if its own dN/N < tol stopped it */
  int64_t edges_scanned;   /* iterations * m, or -1 with LPA_PRUNE (not tracked per graph) */
  double modularity;       /* Q of the graph's labels with LPA_MODULARITY, else 0 */
} lpa_graph_stats;

/* stats: count entries or NULL; changed_out: count * max_iter entries (graph-major: the
 * dN of graph g's sweep l at [g * max_iter + l], 0 after it stopped) or NULL.  The total
 * number of vertices must stay below 2^31 - 16. */
lpa_status lpa_batch_detect(const lpa_graph* graphs, int32_t count, lpa_mode mode, int32_t k,
                            double tol, int32_t max_iter, const lpa_options* opt,
                            lpa_graph_stats* stats, int64_t* changed_out);

/* ---- Served form: continuous batching of label-propagation requests. ---------------
 * A server owns a set of resident graphs, packed block-diagonally as in lpa_batch_detect.
 * lpa_server_submit queues a request (the graph's device arrays must stay valid, and
 * labels_out untouched, until lpa_server_poll reports it done); every lpa_server_step
 * first admits queued requests in arrival order while the resident graphs' HBM
 * footprint (packed CSR, labels and descriptors: about 8(n+1) + 8m + 44n + 16m/e0
 * bytes each) fits hbm_budget_bytes (0 = no limit; one request is always admitted when
 * none is resident), then runs one sweep of every resident graph -- each at its own
 * iteration, with its own pick-less setting and stop test (Alg. 1) -- and writes the
 * labels of the graphs that stopped.  Resident graphs live in an arena: a new graph is
 * appended (only its own CSR is copied), a stopped one leaves a slot the sweeps skip,
 * and the live graphs are re-packed when dead slots hold more than half of the arena or
 * a new graph does not fit.  A request's result equals lpa_detect_ex on its graph
 * alone, whatever else is resident.  One host thread drives a server; calls are
 * ordered on opt->stream and each step synchronises it once.  LPA_PRUNE and labels_in
 * are not supported; LPA_VALIDATE checks each graph at submission. */
typedef struct lpa_server_s* lpa_server;

lpa_status lpa_server_create(lpa_mode mode, int32_t k, double tol, int32_t max_iter,
                             size_t hbm_budget_bytes, const lpa_options* opt,
                             lpa_server* server_out);
/* graph: HOST struct of device pointers; ticket (host) identifies the request.  A graph
 * larger than the budget is refused (LPA_EINVAL). */
lpa_status lpa_server_submit(lpa_server server, const lpa_graph* graph, uint64_t* ticket);
/* pending_out (host, may be NULL): requests resident or queued after the step. */
lpa_status lpa_server_step(lpa_server server, int32_t* pending_out);
/* done (host) = 1 once the request's labels are written; stats (host, may be NULL) as in
 * lpa_batch_detect.  A ticket reported done is forgotten (later polls: LPA_EINVAL). */
lpa_status lpa_server_poll(lpa_server server, uint64_t ticket, int32_t* done,
                           lpa_graph_stats* stats);
/* Tickets of the requests that finished since the last drain (at most cap of them, in
 * finishing order; the rest stay for the next drain) into tickets (host), their number
 * into count_out.  Lets a caller poll only the finished requests. */
lpa_status lpa_server_drain(lpa_server server, uint64_t* tickets, int32_t cap, int32_t* count_out);
/* Frees the server; requests not yet done are dropped (their outputs unspecified). */
lpa_status lpa_server_destroy(lpa_server server);

/* ---- Memory. ------------------------------------------------------------------------
 * Device memory the library allocates (plan workspaces, lpa_detect_host staging, batch
 * and server arenas) comes from one stream-ordered pool per device that keeps freed
 * memory for later calls instead of returning it to the driver; the small page-locked
 * host blocks of plans are kept for reuse too.  lpa_release_memory returns every unused
 * byte of both (memory of live plans and servers stays). */
lpa_status lpa_release_memory(void);

const char* lpa_status_string(lpa_status s);
/* Message of the last failed call on this host thread ("" if none). */
const char* lpa_last_error(void);
/* Library version string. */
const char* lpa_version(void);
/* Number of CUDA kernels this library has launched in this process (diagnostics). */
uint64_t lpa_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LPA_H */
