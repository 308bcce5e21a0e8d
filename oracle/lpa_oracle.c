/*
 * lpa_oracle.c -- plain, slow CPU oracle for memory-efficient label propagation
 * (arxiv 2411.19901).  TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA path.
 *
 * Written for a reader holding the paper: names follow its notation (S_k, S_v,
 * sketchClear, sketchAccumulate, sketchMaxKey, C, dN, rho, tau).  No blocking, fusion or
 * reordering beyond what the definitions below state.  Compiled with
 * -ffp-contract=off and without fast-math, so every float operation is the single
 * IEEE add/sub/compare written here.
 *
 * Readings of the paper that this file fixes (each also listed in the design notes):
 *  R1 synchronous sweeps: C_next[i] depends on C_prev only (the paper updates in place).
 *  R2 clamped weighted MG (Sec. 4.1, Alg. 2): when no slot matches and no slot is free,
 *     every slot and the incoming weight are reduced by delta = min(w, min_s S_v[s]);
 *     a remaining weight goes into the lowest free slot.  With unit weights and no
 *     merges this is exactly the paper's "decrement all by w".
 *  R3 a slot is empty iff S_v[s] == 0 (Sec. 4.1); a key only matches an occupied slot.
 *  R4 the free slot taken is the lowest-index one (find-first-set in Alg. 2).
 *  R5 partial sketches (Sec. 4.3) follow a fixed partition: a row of d positions has
 *     L(d) leaves, L(d) = 1 if d < 2*e0, else min(lmax, largest power of two p with
 *     p*e0 <= d); leaf l covers positions [floor(l*d/L), floor((l+1)*d/L)).  Leaves are
 *     merged by the stride-doubling tree; merge(A, B) feeds B's occupied slots into A
 *     in ascending slot order with sketchAccumulate (the merge loop of Alg. 1).
 *  R6 sketchMaxKey: the occupied slot of largest S_v, ties to the smallest label; an
 *     empty sketch means no move (the paper fixes no tie-break).
 *  R7 weighted BM (Sec. 4.7, Alg. 3) exactly as printed, including the replace branch
 *     when w# == w; partial results per leaf are combined by the pair max (largest w#,
 *     ties to the smallest label); a best w# of 0 means no move.
 *  R8 exact mode (Eq. 3): K_{i->c} summed over valid neighbours, argmax with ties to the
 *     smallest label; it uses a dense accumulator with a touched-label list (the
 *     collision-free table of GVE-LPA, Sec. 2).
 *  R9 edges with j == i or w <= 0 are skipped in every mode (the scans of Alg. 1 and
 *     Alg. 3 skip j == i; a non-positive weight carries no vote).
 *  R10 convergence: after iteration l (0-based), stop iff pick-less was off in l and
 *     (double)dN / (double)N < tau; pick-less is on iff rho > 0 and l mod rho == 0.
 *  R19 pruning (the unprocessed flags of Alg. 1), synchronous: iteration 0 sweeps every
 *     vertex; iteration l+1 sweeps exactly the vertices j that appear in the row of a
 *     vertex whose label changed in iteration l (every stored entry, self-loops and zero
 *     weights included).  A vertex not swept keeps its label.
 *  R20 the paper-literal sketch (ORACLE_UNCLAMPED; Alg. 2 without sharing): a slot whose
 *     key equals c takes += w whatever its value; otherwise the lowest slot with value
 *     exactly 0 takes (c, w); otherwise every slot takes -= w and c is dropped.  Values
 *     may go negative; merges feed every slot with a non-zero value; the choice is the
 *     largest positive value (R6).
 *  R21 double scan (ORACLE_RESCAN, Sec. 4.4): after the sketch, K_{i->c} of every
 *     occupied candidate c is summed over the row's valid entries, each leaf in CSR
 *     order and the leaves along the stride-doubling tree; the choice is the largest
 *     sum, ties to the smallest label.
 */
#include "lpa_oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_K 32
#define ORACLE_MAX_LMAX 4096

/* ------------------------------------------------------------------ MG sketch */

typedef struct {
  int32_t k;
  int32_t S_k[ORACLE_MAX_K]; /* candidate labels */
  float S_v[ORACLE_MAX_K];   /* sketch weights; 0 means the slot is empty */
} mg_sketch;

/* sketchClear (Alg. 1): every slot empty. */
static void sketchClear(mg_sketch* S, int32_t k) {
  S->k = k;
  for (int32_t s = 0; s < k; ++s) {
    S->S_k[s] = -1;
    S->S_v[s] = 0.0f;
  }
}

/* Lowest-index empty slot, or -1 (R4). */
static int32_t lowest_empty_slot(const mg_sketch* S) {
  for (int32_t s = 0; s < S->k; ++s)
    if (S->S_v[s] == 0.0f) return s;
  return -1;
}

/* sketchAccumulate(S, c, w) for one pair with w > 0 (Sec. 4.1, Alg. 2; readings R2-R4). */
static void sketchAccumulate(mg_sketch* S, int32_t c, float w) {
  /* 1. the label is already a candidate: add the edge weight to its slot */
  for (int32_t s = 0; s < S->k; ++s) {
    if (S->S_v[s] > 0.0f && S->S_k[s] == c) {
      S->S_v[s] = S->S_v[s] + w;
      return;
    }
  }
  /* 2. populate a free slot */
  int32_t sphi = lowest_empty_slot(S);
  if (sphi >= 0) {
    S->S_k[sphi] = c;
    S->S_v[sphi] = w;
    return;
  }
  /* 3. no free slot: decrement every slot and the weight by delta (clamped, R2) */
  float delta = w;
  for (int32_t s = 0; s < S->k; ++s)
    if (S->S_v[s] < delta) delta = S->S_v[s];
  for (int32_t s = 0; s < S->k; ++s) {
    S->S_v[s] = S->S_v[s] - delta;
    if (S->S_v[s] == 0.0f) S->S_k[s] = -1;
  }
  w = w - delta;
  if (w > 0.0f) {
    sphi = lowest_empty_slot(S); /* exists: the minimum slot just reached zero */
    S->S_k[sphi] = c;
    S->S_v[sphi] = w;
  }
}

/* sketchAccumulate as printed in Alg. 2 for a private sketch (R20): the key compare
 * ignores the value, and a full sketch loses w from every slot. */
static void sketchAccumulateLiteral(mg_sketch* S, int32_t c, float w) {
  int has = 0;
  for (int32_t s = 0; s < S->k; ++s) {
    if (S->S_k[s] == c) {
      S->S_v[s] = S->S_v[s] + w;
      has = 1;
    }
  }
  if (has) return;
  int32_t sphi = lowest_empty_slot(S);
  if (sphi >= 0) {
    S->S_k[sphi] = c;
    S->S_v[sphi] = w;
    return;
  }
  for (int32_t s = 0; s < S->k; ++s) S->S_v[s] = S->S_v[s] - w;
}

/* merge(A, B): B's occupied slots, ascending, accumulated into A (Sec. 4.3; R5).  The
 * literal variant feeds every slot of non-zero value (the merge loop of Alg. 1). */
static void sketchMerge(mg_sketch* A, const mg_sketch* B, int literal) {
  for (int32_t s = 0; s < B->k; ++s) {
    if (literal) {
      if (B->S_v[s] != 0.0f) sketchAccumulateLiteral(A, B->S_k[s], B->S_v[s]);
    } else if (B->S_v[s] > 0.0f) {
      sketchAccumulate(A, B->S_k[s], B->S_v[s]);
    }
  }
}

/* sketchMaxKey (Alg. 1, single scan Sec. 4.4; R6): -1 if the sketch is empty. */
static int32_t sketchMaxKey(const mg_sketch* S) {
  int32_t best = -1;
  float bestv = 0.0f;
  for (int32_t s = 0; s < S->k; ++s) {
    if (S->S_v[s] <= 0.0f) continue;
    if (best < 0 || S->S_v[s] > bestv || (S->S_v[s] == bestv && S->S_k[s] < best)) {
      best = S->S_k[s];
      bestv = S->S_v[s];
    }
  }
  return best;
}

/* -------------------------------------------------------------- leaf partition */

int32_t oracle_leaf_count(int64_t d, int32_t e0, int32_t lmax) {
  if (e0 < 1 || lmax < 1) return 1;
  if (d < 2 * (int64_t)e0) return 1;
  int64_t p = 1;
  while (2 * p <= lmax && 2 * p * (int64_t)e0 <= d) p *= 2;
  return (int32_t)p;
}

static int64_t leaf_begin(int64_t d, int32_t L, int32_t l) { return ((int64_t)l * d) / L; }

static int valid_params(int32_t k, int32_t e0, int32_t lmax) {
  if (k < 1 || k > ORACLE_MAX_K) return 0;
  if (e0 < 1) return 0;
  if (lmax < 1 || lmax > ORACLE_MAX_LMAX || (lmax & (lmax - 1)) != 0) return 0;
  return 1;
}

/* The MG sketch of a row given as a sequence of (label, weight); label < 0 marks a
 * position to skip (a self-loop at the caller), weight <= 0 is skipped as well (R9). */
static void mg_row(const int32_t* lab, const float* w, int64_t d, int32_t k, int32_t e0,
                   int32_t lmax, int literal, mg_sketch* out) {
  int32_t L = oracle_leaf_count(d, e0, lmax);
  mg_sketch* S = (mg_sketch*)malloc(sizeof(mg_sketch) * (size_t)L);
  /* each leaf folds its positions in ascending CSR order into an empty sketch */
  for (int32_t l = 0; l < L; ++l) {
    sketchClear(&S[l], k);
    for (int64_t p = leaf_begin(d, L, l); p < leaf_begin(d, L, l + 1); ++p) {
      float wp = w ? w[p] : 1.0f;
      if (lab[p] < 0 || !(wp > 0.0f)) continue;
      if (literal)
        sketchAccumulateLiteral(&S[l], lab[p], wp);
      else
        sketchAccumulate(&S[l], lab[p], wp);
    }
  }
  /* stride-doubling tree: S[l] <- merge(S[l], S[l+s]) for l = 0 mod 2s */
  for (int32_t s = 1; s < L; s *= 2)
    for (int32_t l = 0; l + s < L; l += 2 * s) sketchMerge(&S[l], &S[l + s], literal);
  *out = S[0];
  free(S);
}

/* Double scan (R21): the choice among the sketch's occupied candidates by their exact
 * linking weight K_{i->c}; per leaf a sequential sum in CSR order, then the leaves'
 * sums along the stride-doubling tree.  -1 when the sketch has no candidate. */
static int32_t rescan_choice(const mg_sketch* S, const int32_t* lab, const float* w,
                             int64_t d, int32_t e0, int32_t lmax) {
  int32_t L = oracle_leaf_count(d, e0, lmax);
  float* part = (float*)calloc((size_t)L * ORACLE_MAX_K, sizeof(float));
  for (int32_t l = 0; l < L; ++l)
    for (int64_t p = leaf_begin(d, L, l); p < leaf_begin(d, L, l + 1); ++p) {
      float wp = w ? w[p] : 1.0f;
      if (lab[p] < 0 || !(wp > 0.0f)) continue;
      for (int32_t s = 0; s < S->k; ++s)
        if (S->S_v[s] > 0.0f && S->S_k[s] == lab[p])
          part[(size_t)l * ORACLE_MAX_K + s] = part[(size_t)l * ORACLE_MAX_K + s] + wp;
    }
  for (int32_t st = 1; st < L; st *= 2)
    for (int32_t l = 0; l + st < L; l += 2 * st)
      for (int32_t s = 0; s < S->k; ++s)
        part[(size_t)l * ORACLE_MAX_K + s] =
            part[(size_t)l * ORACLE_MAX_K + s] + part[(size_t)(l + st) * ORACLE_MAX_K + s];
  int32_t best = -1;
  float bestK = 0.0f;
  for (int32_t s = 0; s < S->k; ++s) {
    if (!(S->S_v[s] > 0.0f)) continue;
    float K = part[s];
    if (best < 0 || K > bestK || (K == bestK && S->S_k[s] < best)) {
      best = S->S_k[s];
      bestK = K;
    }
  }
  free(part);
  return best;
}

int oracle_mg_sketch(const int32_t* labels, const float* weights, int64_t d, int32_t k,
                     int32_t e0, int32_t lmax, int32_t* keys_out, float* vals_out) {
  if (!valid_params(k, e0, lmax) || d < 0 || (d > 0 && !labels)) return -1;
  mg_sketch S;
  mg_row(labels, weights, d, k, e0, lmax, 0, &S);
  for (int32_t s = 0; s < k; ++s) {
    keys_out[s] = S.S_v[s] > 0.0f ? S.S_k[s] : -1;
    vals_out[s] = S.S_v[s];
  }
  return 0;
}

int oracle_mg_sketch_ex(const int32_t* labels, const float* weights, int64_t d, int32_t k,
                        int32_t e0, int32_t lmax, int32_t flags, int32_t* keys_out,
                        float* vals_out) {
  if (!valid_params(k, e0, lmax) || d < 0 || (d > 0 && !labels)) return -1;
  mg_sketch S;
  mg_row(labels, weights, d, k, e0, lmax, (flags & ORACLE_UNCLAMPED) != 0, &S);
  for (int32_t s = 0; s < k; ++s) {
    keys_out[s] = S.S_k[s];  /* raw slots: the literal sketch keeps stale keys */
    vals_out[s] = S.S_v[s];
  }
  return 0;
}

/* ------------------------------------------------------------------ weighted BM */

typedef struct {
  int32_t c; /* c#: majority weighted label */
  float w;   /* w#: its weight */
} bm_state;

/* One leaf of weighted BM, the rule of Sec. 4.7 / Alg. 3 as printed (R7). */
static bm_state bm_leaf(const int32_t* lab, const float* w, int64_t b, int64_t e,
                        int32_t own_label) {
  bm_state st = {own_label, 0.0f};
  for (int64_t p = b; p < e; ++p) {
    float wp = w ? w[p] : 1.0f;
    if (lab[p] < 0 || !(wp > 0.0f)) continue;
    if (lab[p] == st.c) {
      st.w = st.w + wp;
    } else if (st.w > wp) {
      st.w = st.w - wp;
    } else {
      st.c = lab[p];
      st.w = wp;
    }
  }
  return st;
}

static bm_state bm_row(const int32_t* lab, const float* w, int64_t d, int32_t own_label,
                       int32_t e0, int32_t lmax) {
  int32_t L = oracle_leaf_count(d, e0, lmax);
  bm_state best = {own_label, 0.0f};
  for (int32_t l = 0; l < L; ++l) {
    bm_state st = bm_leaf(lab, w, leaf_begin(d, L, l), leaf_begin(d, L, l + 1), own_label);
    /* pair max: larger w#, ties to the smaller label */
    if (st.w > best.w || (st.w == best.w && st.c < best.c)) best = st;
  }
  return best;
}

int oracle_bm_sketch(const int32_t* labels, const float* weights, int64_t d,
                     int32_t own_label, int32_t e0, int32_t lmax, int32_t* c_out,
                     float* w_out) {
  if (!valid_params(1, e0, lmax) || d < 0 || (d > 0 && !labels)) return -1;
  bm_state st = bm_row(labels, weights, d, own_label, e0, lmax);
  *c_out = st.c;
  *w_out = st.w;
  return 0;
}

/* ------------------------------------------------------------- per-vertex choice */

/* Exact label choice, Eq. 3 (R8).  dense[] has one zeroed float per label; touched[]
 * lists the labels written, so the accumulator can be reset in O(d). */
static int32_t exact_choice(int32_t i, const int64_t* off, const int32_t* idx,
                            const float* w, const int32_t* C, float* dense,
                            int32_t* touched) {
  int32_t ntouched = 0;
  for (int64_t p = off[i]; p < off[i + 1]; ++p) {
    int32_t j = idx[p];
    float wij = w ? w[p] : 1.0f;
    if (j == i || !(wij > 0.0f)) continue;
    int32_t c = C[j];
    if (dense[c] == 0.0f) touched[ntouched++] = c;
    dense[c] = dense[c] + wij; /* K_{i->c} */
  }
  int32_t best = -1;
  float bestK = 0.0f;
  for (int32_t t = 0; t < ntouched; ++t) {
    int32_t c = touched[t];
    if (best < 0 || dense[c] > bestK || (dense[c] == bestK && c < best)) {
      best = c;
      bestK = dense[c];
    }
  }
  for (int32_t t = 0; t < ntouched; ++t) dense[touched[t]] = 0.0f;
  return best;
}

/* Neighbour labels of row i, with -1 at self-loop positions. */
static int32_t* row_labels(int32_t i, const int64_t* off, const int32_t* idx,
                           const int32_t* C) {
  int64_t d = off[i + 1] - off[i];
  int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * (size_t)(d > 0 ? d : 1));
  for (int64_t p = 0; p < d; ++p) {
    int32_t j = idx[off[i] + p];
    lab[p] = (j == i) ? -1 : C[j];
  }
  return lab;
}

static int32_t choose_sketch(int32_t i, const int64_t* off, const int32_t* idx,
                             const float* w, const int32_t* C, int32_t mode, int32_t k,
                             int32_t e0, int32_t lmax, int32_t flags) {
  int64_t d = off[i + 1] - off[i];
  int32_t* lab = row_labels(i, off, idx, C);
  const float* wrow = w ? w + off[i] : NULL;
  int32_t choice;
  if (mode == ORACLE_MG) {
    mg_sketch S;
    mg_row(lab, wrow, d, k, e0, lmax, (flags & ORACLE_UNCLAMPED) != 0, &S);
    choice = (flags & ORACLE_RESCAN) ? rescan_choice(&S, lab, wrow, d, e0, lmax)
                                     : sketchMaxKey(&S);
  } else {
    bm_state st = bm_row(lab, wrow, d, C[i], e0, lmax);
    choice = st.w > 0.0f ? st.c : -1;
  }
  free(lab);
  return choice;
}

int32_t oracle_choose(int32_t i, const int64_t* offsets, const int32_t* indices,
                      const float* weights, const int32_t* c_prev, int32_t mode, int32_t k,
                      int32_t e0, int32_t lmax) {
  if (mode == ORACLE_EXACT) {
    /* labels lie in [0, n); n is not passed here, so size the accumulator by the
     * largest label seen in the row */
    int32_t cmax = 0;
    for (int64_t p = offsets[i]; p < offsets[i + 1]; ++p)
      if (c_prev[indices[p]] > cmax) cmax = c_prev[indices[p]];
    float* dense = (float*)calloc((size_t)cmax + 1, sizeof(float));
    int32_t* touched =
        (int32_t*)malloc(sizeof(int32_t) * (size_t)(offsets[i + 1] - offsets[i] + 1));
    int32_t c = exact_choice(i, offsets, indices, weights, c_prev, dense, touched);
    free(dense);
    free(touched);
    return c;
  }
  return choose_sketch(i, offsets, indices, weights, c_prev, mode, k, e0, lmax, 0);
}

/* ------------------------------------------------------------------- the sweep */

int64_t oracle_move_ex(int32_t n, const int64_t* off, const int32_t* idx, const float* w,
                       const int32_t* c_prev, int32_t* c_next, const uint8_t* active,
                       int32_t mode, int32_t k, int32_t e0, int32_t lmax, int32_t pick_less,
                       int32_t flags, int32_t threads, int64_t* scanned_out) {
  int64_t dN = 0, scanned = 0;
#ifdef _OPENMP
  if (threads < 1) threads = 1;
#pragma omp parallel num_threads(threads) reduction(+ : dN, scanned)
#endif
  {
    float* dense = NULL;
    int32_t* touched = NULL;
    if (mode == ORACLE_EXACT) {
      dense = (float*)calloc((size_t)n + 1, sizeof(float));
      touched = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1024)
#endif
    for (int32_t i = 0; i < n; ++i) {
      if (active && !active[i]) { /* not swept this iteration (R19) */
        c_next[i] = c_prev[i];
        continue;
      }
      scanned += off[i + 1] - off[i];
      int32_t c = (mode == ORACLE_EXACT)
                      ? exact_choice(i, off, idx, w, c_prev, dense, touched)
                      : choose_sketch(i, off, idx, w, c_prev, mode, k, e0, lmax, flags);
      /* commit (Alg. 1 move step): change only to a different label, and under
       * pick-less only to a smaller one (Sec. 4.5) */
      if (c >= 0 && c != c_prev[i] && (!pick_less || c < c_prev[i])) {
        c_next[i] = c;
        dN += 1;
      } else {
        c_next[i] = c_prev[i];
      }
    }
    free(dense);
    free(touched);
  }
  if (scanned_out) *scanned_out = scanned;
  return dN;
}

int64_t oracle_move(int32_t n, const int64_t* off, const int32_t* idx, const float* w,
                    const int32_t* c_prev, int32_t* c_next, int32_t mode, int32_t k,
                    int32_t e0, int32_t lmax, int32_t pick_less, int32_t threads) {
  return oracle_move_ex(n, off, idx, w, c_prev, c_next, NULL, mode, k, e0, lmax, pick_less, 0,
                        threads, NULL);
}

/* ------------------------------------------------------------------ the driver */

int oracle_lpa_ex(int32_t n, const int64_t* off, const int32_t* idx, const float* w,
                  int32_t mode, int32_t k, double tol, int32_t max_iter, int32_t rho,
                  int32_t e0, int32_t lmax, int32_t flags, const int32_t* labels_in,
                  int32_t* labels_out, int64_t* changed_out, int64_t* scanned_out,
                  int32_t* iterations_out, int32_t* converged_out, int32_t threads) {
  if (n < 0 || max_iter < 0 || rho < 0) return -1;
  if (mode != ORACLE_EXACT && mode != ORACLE_MG && mode != ORACLE_BM) return -1;
  if (mode == ORACLE_MG && !valid_params(k, e0, lmax)) return -1;
  if (mode == ORACLE_BM && !valid_params(1, e0, lmax)) return -1;
  if ((flags & (ORACLE_UNCLAMPED | ORACLE_RESCAN)) && mode != ORACLE_MG) return -1;
  *iterations_out = 0;
  *converged_out = 0;
  if (n == 0) {
    *converged_out = 1;
    return 0;
  }
  int32_t* C = labels_out;
  int32_t* C2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  uint8_t* active = NULL;
  if (flags & ORACLE_PRUNE) {
    active = (uint8_t*)malloc((size_t)n);
    memset(active, 1, (size_t)n); /* iteration 0 sweeps every vertex */
  }
  /* C <- [0 .. |V|), or the caller's warm start */
  for (int32_t i = 0; i < n; ++i) C[i] = labels_in ? labels_in[i] : i;
  for (int32_t l = 0; l < max_iter; ++l) {
    int32_t pick_less = (rho > 0 && l % rho == 0);
    int64_t scanned = 0;
    int64_t dN = oracle_move_ex(n, off, idx, w, C, C2, active, mode, k, e0, lmax, pick_less,
                                flags, threads, &scanned);
    if (active) {
      /* Alg. 1: a vertex that changed marks every vertex of its row unprocessed (R19) */
      memset(active, 0, (size_t)n);
      for (int32_t i = 0; i < n; ++i)
        if (C2[i] != C[i])
          for (int64_t p = off[i]; p < off[i + 1]; ++p) active[idx[p]] = 1;
    }
    memcpy(C, C2, sizeof(int32_t) * (size_t)n);
    changed_out[l] = dN;
    if (scanned_out) scanned_out[l] = scanned;
    *iterations_out = l + 1;
    if (!pick_less && (double)dN / (double)n < tol) {
      *converged_out = 1;
      break;
    }
  }
  free(active);
  free(C2);
  return 0;
}

int oracle_lpa(int32_t n, const int64_t* off, const int32_t* idx, const float* w,
               int32_t mode, int32_t k, double tol, int32_t max_iter, int32_t rho,
               int32_t e0, int32_t lmax, const int32_t* labels_in, int32_t* labels_out,
               int64_t* changed_out, int32_t* iterations_out, int32_t* converged_out,
               int32_t threads) {
  return oracle_lpa_ex(n, off, idx, w, mode, k, tol, max_iter, rho, e0, lmax, 0, labels_in,
                       labels_out, changed_out, NULL, iterations_out, converged_out, threads);
}

/* ------------------------------------------------------------------ modularity */

/* Eq. 1, right-hand form: Q = sum_c [ sigma_c / 2m - (Sigma_c / 2m)^2 ], where
 * 2m = sum of all CSR entry weights, sigma_c = weight of entries (i, j) with
 * C_i = C_j = c (both directions counted, a self-loop once as stored) and
 * Sigma_c = sum over i in c of K_i.  Returns 0 when 2m == 0. */
double oracle_modularity(int32_t n, const int64_t* off, const int32_t* idx, const float* w,
                         const int32_t* C) {
  double* sigma = (double*)calloc((size_t)n + 1, sizeof(double));
  double* Sigma = (double*)calloc((size_t)n + 1, sizeof(double));
  double two_m = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    double K_i = 0.0;
    for (int64_t p = off[i]; p < off[i + 1]; ++p) {
      double wij = w ? (double)w[p] : 1.0;
      K_i += wij;
      if (C[idx[p]] == C[i]) sigma[C[i]] += wij;
    }
    Sigma[C[i]] += K_i;
    two_m += K_i;
  }
  double Q = 0.0;
  if (two_m > 0.0) {
    for (int32_t c = 0; c < n; ++c) {
      double a = Sigma[c] / two_m;
      Q += sigma[c] / two_m - a * a;
    }
  }
  free(sigma);
  free(Sigma);
  return Q;
}
