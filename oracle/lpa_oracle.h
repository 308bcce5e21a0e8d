/*
 * lpa_oracle.h -- plain, slow CPU oracle for memory-efficient label propagation
 * (weighted Misra-Gries / weighted Boyer-Moore / exact label choice), arxiv 2411.19901.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library against the
 * paper.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load or call it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Semantics (each function cites the passage it follows):
 *   - Label update, Eq. 3 (Sec. 3.3); self-loops are skipped (Alg. 1 and Alg. 3 scans).
 *   - Driver: identity init, pick-less every rho iterations from the first, stop when
 *     dN/N < tau in a non-pick-less iteration (Alg. 1 `lpa`, Sec. 4.5).
 *   - Iterations are synchronous: every C_next[i] reads only C_prev (a stated
 *     departure from the paper's asynchronous in-place updates).
 *   - Weighted MG sketch with k slots (Sec. 4.1, Alg. 2), read as the clamped
 *     weighted Misra-Gries summary; partial sketches merged (Sec. 4.3) along a fixed
 *     leaf partition and stride-doubling tree; single scan (Sec. 4.4).
 *   - Weighted BM as printed (Sec. 4.7, Alg. 3); partial results combined by the pair
 *     max the paper's block reduce computes.
 *   - Modularity, Eq. 1 (Sec. 3.2), in fp64.
 * Precision: int32 labels, fp32 weights and sketch values (Sec. 5.1.2); fp64 for Q.
 */
#ifndef LPA_ORACLE_H
#define LPA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_EXACT = 0, ORACLE_MG = 1, ORACLE_BM = 2 };

/* Variant flags: pruning by unprocessed flags (R19), the paper-literal sketch (R20) and
 * the double scan (R21); the last two apply to MG only. */
enum { ORACLE_PRUNE = 1, ORACLE_UNCLAMPED = 2, ORACLE_RESCAN = 4 };

/* Number of leaves (partial sketches) for a row of d CSR positions. */
int32_t oracle_leaf_count(int64_t d, int32_t e0, int32_t lmax);

/* MG sketch of one sequence of (label, weight) pairs, folded leaf by leaf and merged
 * along the stride-doubling tree.  Entries with label < 0 or weight <= 0 are skipped
 * but still occupy their position.  keys/vals receive the k final slots (val 0 = empty,
 * key of an empty slot is -1).  Returns 0, or -1 for bad arguments. */
int oracle_mg_sketch(const int32_t* labels, const float* weights, int64_t d,
                     int32_t k, int32_t e0, int32_t lmax,
                     int32_t* keys_out, float* vals_out);

/* As oracle_mg_sketch with variant flags (ORACLE_UNCLAMPED); the raw slots are returned
 * (keys of empty slots as they stand). */
int oracle_mg_sketch_ex(const int32_t* labels, const float* weights, int64_t d,
                        int32_t k, int32_t e0, int32_t lmax, int32_t flags,
                        int32_t* keys_out, float* vals_out);

/* Weighted BM over one sequence, same leaf partition; (c#, w#) of the winning leaf. */
int oracle_bm_sketch(const int32_t* labels, const float* weights, int64_t d,
                     int32_t own_label, int32_t e0, int32_t lmax,
                     int32_t* c_out, float* w_out);

/* The label vertex i would choose from C_prev (before the pick-less test), or -1 if
 * it has no valid neighbour.  weights == NULL means unit weights. */
int32_t oracle_choose(int32_t i, const int64_t* offsets, const int32_t* indices,
                      const float* weights, const int32_t* c_prev,
                      int32_t mode, int32_t k, int32_t e0, int32_t lmax);

/* One synchronous sweep C_prev -> C_next.  Returns dN (number of changed labels). */
int64_t oracle_move(int32_t n, const int64_t* offsets, const int32_t* indices,
                    const float* weights, const int32_t* c_prev, int32_t* c_next,
                    int32_t mode, int32_t k, int32_t e0, int32_t lmax,
                    int32_t pick_less, int32_t threads);

/* One sweep over the vertices with active[i] != 0 (all when active is NULL); the others
 * keep their label.  scanned_out (may be NULL) receives the CSR entries of swept rows. */
int64_t oracle_move_ex(int32_t n, const int64_t* offsets, const int32_t* indices,
                       const float* weights, const int32_t* c_prev, int32_t* c_next,
                       const uint8_t* active, int32_t mode, int32_t k, int32_t e0,
                       int32_t lmax, int32_t pick_less, int32_t flags, int32_t threads,
                       int64_t* scanned_out);

/* Full driver with variant flags; scanned_out (may be NULL) has room for max_iter
 * entries and receives the CSR entries swept per iteration. */
int oracle_lpa_ex(int32_t n, const int64_t* offsets, const int32_t* indices,
                  const float* weights, int32_t mode, int32_t k, double tol,
                  int32_t max_iter, int32_t rho, int32_t e0, int32_t lmax, int32_t flags,
                  const int32_t* labels_in, int32_t* labels_out, int64_t* changed_out,
                  int64_t* scanned_out, int32_t* iterations_out, int32_t* converged_out,
                  int32_t threads);

/* Full driver.  changed_out has room for max_iter entries.  labels_in may be NULL
 * (identity init).  Returns 0, or -1 for bad arguments. */
int oracle_lpa(int32_t n, const int64_t* offsets, const int32_t* indices,
               const float* weights, int32_t mode, int32_t k, double tol,
               int32_t max_iter, int32_t rho, int32_t e0, int32_t lmax,
               const int32_t* labels_in, int32_t* labels_out, int64_t* changed_out,
               int32_t* iterations_out, int32_t* converged_out, int32_t threads);

/* Modularity Q of labels (values in [0, n)), Eq. 1 right-hand form, fp64. */
double oracle_modularity(int32_t n, const int64_t* offsets, const int32_t* indices,
                         const float* weights, const int32_t* labels);

#ifdef __cplusplus
}
#endif
#endif
