/*
 * graphgen.c -- seeded synthetic graph generators (host C, OpenMP).
 *
 * These stand in for the paper's SuiteSparse web/social graphs (Sec. 5.1.3, Table 1),
 * which are not available here.  The module holds no part of label propagation: it
 * only produces symmetric CSR graphs (int64 offsets, int32 sorted neighbour ids, fp32
 * integer-valued weights) for the CUDA library and the oracle alike.
 *
 * Randomness: SplitMix64 and xoshiro256** (Blackman and Vigna), written from their
 * published definitions.  A "stream" (seed, tag, index) seeds a xoshiro256** state
 * with four SplitMix64 outputs, so every parallel item owns its own stream and the
 * result does not depend on the number of threads.  Uniform doubles are
 * (x >> 11) * 2^-53.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG */

static uint64_t splitmix64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t mix64(uint64_t x) {
  uint64_t s = x;
  return splitmix64_next(&s);
}

typedef struct {
  uint64_t s[4];
} rng_t;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return result;
}

static rng_t rng_stream(uint64_t seed, uint64_t tag, uint64_t index) {
  uint64_t sm = mix64(seed ^ mix64(tag * 0xD1B54A32D192ED03ULL ^ mix64(index)));
  rng_t r;
  for (int i = 0; i < 4; ++i) r.s[i] = splitmix64_next(&sm);
  return r;
}

static double rng_uniform(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, bound) (bound >= 1) by Lemire's multiply-shift; the tiny bias is
 * irrelevant for synthetic inputs */
static uint64_t rng_below(rng_t* r, uint64_t bound) {
  return (uint64_t)(((__uint128_t)rng_next(r) * (__uint128_t)bound) >> 64);
}

/* continuous power law with exponent gamma on [lo, hi), by inverse CDF */
static double powerlaw(double u, double gamma, double lo, double hi) {
  double a = pow(lo, 1.0 - gamma), b = pow(hi, 1.0 - gamma);
  return pow(a + u * (b - a), 1.0 / (1.0 - gamma));
}

/* ------------------------------------------------------------------ CSR result */

typedef struct {
  int64_t n;
  int64_t m;
  int64_t* offsets; /* n + 1 */
  int32_t* indices; /* m */
  float* weights;   /* m */
} gg_csr;

void gg_free(gg_csr* g) {
  if (!g) return;
  free(g->offsets);
  free(g->indices);
  free(g->weights);
  memset(g, 0, sizeof(*g));
}

static int nthreads_of(int threads) {
#ifdef _OPENMP
  if (threads < 1) threads = omp_get_max_threads();
  return threads;
#else
  (void)threads;
  return 1;
#endif
}

/* radix sort of uint64 keys on the high 32 bits (neighbour id), stable */
static void sort_hi32(uint64_t* a, uint64_t* tmp, int64_t len) {
  if (len < 48) {
    for (int64_t i = 1; i < len; ++i) {
      uint64_t x = a[i];
      int64_t j = i - 1;
      while (j >= 0 && (a[j] >> 32) > (x >> 32)) {
        a[j + 1] = a[j];
        --j;
      }
      a[j + 1] = x;
    }
    return;
  }
  uint64_t* src = a;
  uint64_t* dst = tmp;
  for (int pass = 0; pass < 4; ++pass) {
    int shift = 32 + 8 * pass;
    int64_t cnt[257];
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < len; ++i) cnt[((src[i] >> shift) & 255) + 1]++;
    for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
    for (int64_t i = 0; i < len; ++i) dst[cnt[(src[i] >> shift) & 255]++] = src[i];
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  /* four passes: the result is back in a */
}

/* Build a symmetric CSR from undirected pairs (u[e], v[e]).  Self-loops are dropped.
 * Both directions are stored.  Duplicates of a pair are merged: sum_dups != 0 sums
 * their weights, otherwise the first is kept (callers whose weight is a function of
 * the pair see no difference).  w == NULL gives every pair weight 1.  Rows come out
 * sorted by neighbour id; the result does not depend on the thread count. */
static int build_sym_csr(int64_t n, int64_t E, const int32_t* u, const int32_t* v,
                         const float* w, int sum_dups, int threads, gg_csr* out) {
  int T = nthreads_of(threads);
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -1;
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    if (u[e] == v[e]) continue;
#pragma omp atomic
    cnt[u[e]]++;
#pragma omp atomic
    cnt[v[e]]++;
  }
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  start[0] = 0;
  for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + cnt[i];
  int64_t total = start[n];
  uint64_t* ent = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(total > 0 ? total : 1));
  int64_t* cur = cnt; /* reuse as cursor */
  for (int64_t i = 0; i < n; ++i) cur[i] = start[i];
  if (!ent) {
    free(cnt);
    free(start);
    return -1;
  }
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    if (u[e] == v[e]) continue;
    float we = w ? w[e] : 1.0f;
    uint32_t wb;
    memcpy(&wb, &we, 4);
    int64_t pu, pv;
#pragma omp atomic capture
    pu = cur[u[e]]++;
#pragma omp atomic capture
    pv = cur[v[e]]++;
    ent[pu] = ((uint64_t)(uint32_t)v[e] << 32) | wb;
    ent[pv] = ((uint64_t)(uint32_t)u[e] << 32) | wb;
  }
  /* sort and merge each row in place; cnt[i] becomes the merged length */
#pragma omp parallel num_threads(T)
  {
    uint64_t* tmp = NULL;
    int64_t tmpcap = 0;
#pragma omp for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
      int64_t b = start[i], len = start[i + 1] - start[i];
      if (len > tmpcap) {
        free(tmp);
        tmpcap = len * 2;
        tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)tmpcap);
      }
      sort_hi32(ent + b, tmp, len);
      int64_t o = 0;
      for (int64_t p = 0; p < len; ++p) {
        if (o > 0 && (ent[b + o - 1] >> 32) == (ent[b + p] >> 32)) {
          if (sum_dups) {
            float a, c;
            uint32_t ab = (uint32_t)ent[b + o - 1], cb = (uint32_t)ent[b + p];
            memcpy(&a, &ab, 4);
            memcpy(&c, &cb, 4);
            a = a + c;
            memcpy(&ab, &a, 4);
            ent[b + o - 1] = (ent[b + o - 1] & 0xFFFFFFFF00000000ULL) | ab;
          }
          continue;
        }
        ent[b + o++] = ent[b + p];
      }
      cnt[i] = o;
    }
    free(tmp);
  }
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  off[0] = 0;
  for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + cnt[i];
  int64_t m = off[n];
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  float* wt = (float*)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1));
  if (!off || !idx || !wt) {
    free(cnt);
    free(start);
    free(ent);
    free(off);
    free(idx);
    free(wt);
    return -1;
  }
#pragma omp parallel for num_threads(T) schedule(dynamic, 4096)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t p = 0; p < cnt[i]; ++p) {
      uint64_t x = ent[start[i] + p];
      uint32_t wb = (uint32_t)x;
      idx[off[i] + p] = (int32_t)(x >> 32);
      memcpy(&wt[off[i] + p], &wb, 4);
    }
  }
  free(cnt);
  free(start);
  free(ent);
  out->n = n;
  out->m = m;
  out->offsets = off;
  out->indices = idx;
  out->weights = wt;
  return 0;
}

/* ------------------------------------------------- planted partition (small) */

/* n vertices, community of i = i / (n / ncomm) (last absorbs the rest); every pair
 * i < j in lexicographic order draws one uniform from a single stream and becomes an
 * edge if u < p_in (same community) or u < p_out (different).  Unit weights. */
int gg_planted_partition(int32_t n, int32_t ncomm, double p_in, double p_out,
                         uint64_t seed, gg_csr* out) {
  if (n < 0 || ncomm < 1) return -1;
  memset(out, 0, sizeof(*out));
  int32_t csize = ncomm > n ? 1 : n / ncomm;
  rng_t r = rng_stream(seed, 101, 0);
  int64_t cap = 1024, E = 0;
  int32_t* u = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  int32_t* v = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  for (int32_t i = 0; i < n; ++i) {
    int32_t ci = i / csize < ncomm ? i / csize : ncomm - 1;
    for (int32_t j = i + 1; j < n; ++j) {
      int32_t cj = j / csize < ncomm ? j / csize : ncomm - 1;
      double x = rng_uniform(&r);
      if (x < (ci == cj ? p_in : p_out)) {
        if (E == cap) {
          cap *= 2;
          u = (int32_t*)realloc(u, sizeof(int32_t) * (size_t)cap);
          v = (int32_t*)realloc(v, sizeof(int32_t) * (size_t)cap);
        }
        u[E] = i;
        v[E] = j;
        ++E;
      }
    }
  }
  int rc = build_sym_csr(n, E, u, v, NULL, 0, 1, out);
  free(u);
  free(v);
  return rc;
}

/* -------------------------------------------------------------------- RMAT */

/* R-MAT (Chakrabarti et al.): 2^scale vertices, edge_factor * 2^scale generated edges;
 * each edge descends `scale` levels choosing quadrant (a, b, c, d = 1-a-b-c) from its
 * own stream.  Vertex ids are then relabelled by a seeded Fisher-Yates permutation.
 * The graph is symmetrised, self-loops dropped, and duplicates merged with their unit
 * weights summed (integer-valued fp32). */
int gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c,
            uint64_t seed, int threads, gg_csr* out) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
  memset(out, 0, sizeof(*out));
  int T = nthreads_of(threads);
  int64_t n = (int64_t)1 << scale;
  int64_t E = (int64_t)edge_factor * n;
  int32_t* u = (int32_t*)malloc(sizeof(int32_t) * (size_t)E);
  int32_t* v = (int32_t*)malloc(sizeof(int32_t) * (size_t)E);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!u || !v || !perm) return -1;
  double ab = a + b, abc = a + b + c;
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    rng_t r = rng_stream(seed, 201, (uint64_t)e);
    int64_t s = 0, d = 0;
    for (int32_t l = 0; l < scale; ++l) {
      double x = rng_uniform(&r);
      int bs = 0, bd = 0;
      if (x < a) {
      } else if (x < ab) {
        bd = 1;
      } else if (x < abc) {
        bs = 1;
      } else {
        bs = 1;
        bd = 1;
      }
      s = 2 * s + bs;
      d = 2 * d + bd;
    }
    u[e] = (int32_t)s;
    v[e] = (int32_t)d;
  }
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  rng_t pr = rng_stream(seed, 202, 0);
  for (int64_t i = n - 1; i > 0; --i) {
    int64_t j = (int64_t)rng_below(&pr, (uint64_t)(i + 1));
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    u[e] = perm[u[e]];
    v[e] = perm[v[e]];
  }
  free(perm);
  int rc = build_sym_csr(n, E, u, v, NULL, 1, T, out);
  free(u);
  free(v);
  return rc;
}

/* ------------------------------------------------------------ random shuffles */

/* In-place uniform shuffle of a[0..len), deterministic for (seed, tag) and independent
 * of the thread count: elements are scattered to 2^12 buckets by a hash of their
 * position, buckets are laid out in order, and each bucket is Fisher-Yates shuffled
 * from its own stream.  Small arrays use one Fisher-Yates pass. */
static void shuffle_i32(int32_t* a, int64_t len, uint64_t seed, uint64_t tag, int T) {
  if (len < 2) return;
  if (len < (1 << 22)) {
    rng_t r = rng_stream(seed, tag, 0);
    for (int64_t i = len - 1; i > 0; --i) {
      int64_t j = (int64_t)rng_below(&r, (uint64_t)(i + 1));
      int32_t t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
    return;
  }
  const int B = 4096;
  const int64_t CH = 1 << 20;
  int64_t nch = (len + CH - 1) / CH;
  int64_t* cnt = (int64_t*)calloc((size_t)(nch * B), sizeof(int64_t));
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)len);
  uint64_t salt = mix64(seed ^ (tag * 0x9E3779B97F4A7C15ULL));
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t ch = 0; ch < nch; ++ch) {
    int64_t e = (ch + 1) * CH < len ? (ch + 1) * CH : len;
    for (int64_t i = ch * CH; i < e; ++i) cnt[ch * B + (int64_t)(mix64(salt ^ (uint64_t)i) % B)]++;
  }
  /* exclusive prefix in (bucket, chunk) order */
  int64_t* bstart = (int64_t*)malloc(sizeof(int64_t) * (B + 1));
  int64_t acc = 0;
  for (int b = 0; b < B; ++b) {
    bstart[b] = acc;
    for (int64_t ch = 0; ch < nch; ++ch) {
      int64_t c = cnt[ch * B + b];
      cnt[ch * B + b] = acc;
      acc += c;
    }
  }
  bstart[B] = acc;
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t ch = 0; ch < nch; ++ch) {
    int64_t e = (ch + 1) * CH < len ? (ch + 1) * CH : len;
    for (int64_t i = ch * CH; i < e; ++i)
      tmp[cnt[ch * B + (int64_t)(mix64(salt ^ (uint64_t)i) % B)]++] = a[i];
  }
#pragma omp parallel for num_threads(T) schedule(dynamic, 16)
  for (int b = 0; b < B; ++b) {
    rng_t r = rng_stream(seed, tag + 1, (uint64_t)b);
    int32_t* x = tmp + bstart[b];
    int64_t nb = bstart[b + 1] - bstart[b];
    for (int64_t i = nb - 1; i > 0; --i) {
      int64_t j = (int64_t)rng_below(&r, (uint64_t)(i + 1));
      int32_t t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  memcpy(a, tmp, sizeof(int32_t) * (size_t)len);
  free(tmp);
  free(cnt);
  free(bstart);
}

/* ------------------------------------------ LFR-style heavy-tailed planted partition */

/* Lancichinetti-Fortunato-Radicchi-style benchmark graph:
 *  - degrees: floor of a continuous power law (exponent gamma_d) on [dmin, dmax + 1);
 *  - community sizes: floor of a power law (exponent gamma_c) on [cmin, cmax + 1), drawn
 *    until their sum reaches n; the last one is trimmed to make the sum exactly n;
 *  - internal degree round((1 - mu) * d);
 *  - vertices, highest internal degree first, go to a random community with room whose
 *    size exceeds their internal degree (the LFR rule); if none has room, to any
 *    community with room, with the internal degree capped at its size - 1;
 *  - vertex ids are community-contiguous, communities in seeded random order, members
 *    in seeded random order (permute != 0: one more global random relabel);
 *  - internal stubs are paired at random inside each community, external stubs
 *    globally (configuration model); self-loops and repeated pairs are dropped;
 *  - weight of an undirected edge: uniform integer in 1..wmax from a hash of the pair.
 * comm_out (optional, n entries, caller-owned) receives each vertex's planted community. */
int gg_lfr(int64_t n, double gamma_d, int32_t dmin, int32_t dmax, double gamma_c,
           int32_t cmin, int32_t cmax, double mu, int32_t wmax, uint64_t seed,
           int permute, int threads, int32_t* comm_out, gg_csr* out) {
  if (n < 2 || n > 0x7FFFFFFF || dmin < 1 || dmax < dmin || cmin < 2 || cmax < cmin ||
      wmax < 1)
    return -1;
  memset(out, 0, sizeof(*out));
  int T = nthreads_of(threads);
  /* degrees and internal degrees */
  int32_t* deg = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* kin = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    rng_t r = rng_stream(seed, 301, (uint64_t)i);
    double x = powerlaw(rng_uniform(&r), gamma_d, (double)dmin, (double)dmax + 1.0);
    int32_t d = (int32_t)floor(x);
    if (d < dmin) d = dmin;
    if (d > dmax) d = dmax;
    deg[i] = d;
    kin[i] = (int32_t)lround((1.0 - mu) * (double)d);
  }
  /* community sizes */
  int64_t ncap = 1024, nc = 0, sum = 0;
  int64_t* csize = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncap);
  rng_t rc = rng_stream(seed, 302, 0);
  while (sum < n) {
    int64_t s = (int64_t)floor(powerlaw(rng_uniform(&rc), gamma_c, (double)cmin, (double)cmax + 1.0));
    if (s < cmin) s = cmin;
    if (s > cmax) s = cmax;
    if (sum + s > n) s = n - sum;
    if (nc == ncap) {
      ncap *= 2;
      csize = (int64_t*)realloc(csize, sizeof(int64_t) * (size_t)ncap);
    }
    csize[nc++] = s;
    sum += s;
  }
  /* communities sorted by size ascending (stable counting by index order) */
  int64_t* corder = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  {
    int64_t maxs = 0;
    for (int64_t c = 0; c < nc; ++c) maxs = csize[c] > maxs ? csize[c] : maxs;
    int64_t* h = (int64_t*)calloc((size_t)maxs + 2, sizeof(int64_t));
    for (int64_t c = 0; c < nc; ++c) h[csize[c] + 1]++;
    for (int64_t s = 0; s <= maxs; ++s) h[s + 1] += h[s];
    for (int64_t c = 0; c < nc; ++c) corder[h[csize[c]]++] = c;
    free(h);
  }
  /* vertices by internal degree descending (counting sort, stable) */
  int32_t* vorder = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  {
    int32_t maxk = 0;
    for (int64_t i = 0; i < n; ++i) maxk = kin[i] > maxk ? kin[i] : maxk;
    int64_t* h = (int64_t*)calloc((size_t)maxk + 2, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) h[(maxk - kin[i]) + 1]++;
    for (int32_t s = 0; s <= maxk; ++s) h[s + 1] += h[s];
    for (int64_t i = 0; i < n; ++i) vorder[h[maxk - kin[i]]++] = (int32_t)i;
    free(h);
  }
  /* placement: community of each (original) vertex.  Vertices come in descending
   * internal degree, so the set of communities large enough only grows; `open` holds
   * those with room, and a vertex picks one uniformly.  If none is left, it takes the
   * largest smaller community with room and its internal degree is capped. */
  int32_t* comm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* room = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  int64_t* open = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  for (int64_t c = 0; c < nc; ++c) room[c] = csize[c];
  rng_t rp = rng_stream(seed, 303, 0);
  int64_t nopen = 0, hi = nc, fb = nc - 1;
  for (int64_t t = 0; t < n; ++t) {
    int32_t v = vorder[t];
    while (hi > 0 && csize[corder[hi - 1]] > kin[v]) {
      --hi;
      if (room[corder[hi]] > 0) open[nopen++] = corder[hi];
    }
    int64_t chosen;
    if (nopen > 0) {
      int64_t q = (int64_t)rng_below(&rp, (uint64_t)nopen);
      chosen = open[q];
      if (room[chosen] == 1) open[q] = open[--nopen];
    } else {
      if (fb > hi - 1) fb = hi - 1;
      while (fb >= 0 && room[corder[fb]] == 0) --fb;
      chosen = corder[fb]; /* total room equals the vertices left, so one exists */
      if (kin[v] > csize[chosen] - 1) kin[v] = (int32_t)(csize[chosen] - 1);
    }
    room[chosen]--;
    comm[v] = (int32_t)chosen;
  }
  free(open);
  free(room);
  free(vorder);
  free(corder);
  /* id layout: communities in random order, members in random order */
  int32_t* cperm = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
  for (int64_t c = 0; c < nc; ++c) cperm[c] = (int32_t)c;
  shuffle_i32(cperm, nc, seed, 304, 1);
  int64_t* cstart = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nc + 1));
  {
    int64_t acc = 0;
    for (int64_t q = 0; q < nc; ++q) {
      cstart[cperm[q]] = acc;
      acc += csize[cperm[q]];
    }
    cstart[nc] = acc;
  }
  int32_t* members = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
    for (int64_t c = 0; c < nc; ++c) fill[c] = cstart[c];
    for (int64_t i = 0; i < n; ++i) members[fill[comm[i]]++] = (int32_t)i;
    free(fill);
  }
#pragma omp parallel for num_threads(T) schedule(dynamic, 64)
  for (int64_t c = 0; c < nc; ++c) {
    rng_t r = rng_stream(seed, 305, (uint64_t)c);
    int32_t* x = members + cstart[c];
    for (int64_t i = csize[c] - 1; i > 0; --i) {
      int64_t j = (int64_t)rng_below(&r, (uint64_t)(i + 1));
      int32_t t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  /* newid[original vertex] */
  int32_t* newid = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t p = 0; p < n; ++p) newid[members[p]] = (int32_t)p;
  if (permute) {
    int32_t* gp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) gp[i] = (int32_t)i;
    shuffle_i32(gp, n, seed, 306, T);
#pragma omp parallel for num_threads(T) schedule(static)
    for (int64_t i = 0; i < n; ++i) newid[i] = gp[newid[i]];
    free(gp);
  }
  if (comm_out) {
#pragma omp parallel for num_threads(T) schedule(static)
    for (int64_t i = 0; i < n; ++i) comm_out[newid[i]] = comm[i];
  }
  /* stubs: internal ones grouped by community (in member order), external ones global */
  /* community c's internal stubs occupy [ioff[c], ioff[c] + ilen[c]), in id order */
  int64_t* ioff = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nc + 1));
  int64_t* ilen = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nc + 1));
  int64_t next = 0, nin = 0;
  {
    for (int64_t q = 0; q < nc; ++q) {
      int64_t c = cperm[q];
      ioff[c] = nin;
      int64_t len = 0;
      for (int64_t p = cstart[c]; p < cstart[c] + csize[c]; ++p) len += kin[members[p]];
      ilen[c] = len;
      nin += len;
    }
    for (int64_t i = 0; i < n; ++i) next += deg[i] - kin[i];
  }
  int32_t* istub = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nin > 0 ? nin : 1));
  int32_t* estub = (int32_t*)malloc(sizeof(int32_t) * (size_t)(next > 0 ? next : 1));
#pragma omp parallel for num_threads(T) schedule(dynamic, 64)
  for (int64_t c = 0; c < nc; ++c) {
    int64_t o = ioff[c];
    for (int64_t p = cstart[c]; p < cstart[c] + csize[c]; ++p) {
      int32_t v = members[p];
      for (int32_t s = 0; s < kin[v]; ++s) istub[o++] = newid[v];
    }
  }
  {
    int64_t o = 0;
    for (int64_t p = 0; p < n; ++p) {
      int32_t v = members[p];
      for (int32_t s = kin[v]; s < deg[v]; ++s) estub[o++] = newid[v];
    }
  }
  free(members);
  free(newid);
  free(deg);
  free(kin);
  free(comm);
  /* pair stubs at random */
#pragma omp parallel for num_threads(T) schedule(dynamic, 1)
  for (int64_t c = 0; c < nc; ++c) {
    int64_t len = ilen[c];
    if (len >= (1 << 22)) continue; /* large ones below, in parallel */
    shuffle_i32(istub + ioff[c], len, seed ^ mix64((uint64_t)c), 307, 1);
  }
  for (int64_t c = 0; c < nc; ++c) {
    int64_t len = ilen[c];
    if (len >= (1 << 22)) shuffle_i32(istub + ioff[c], len, seed ^ mix64((uint64_t)c), 307, T);
  }
  shuffle_i32(estub, next, seed, 309, T);
  int64_t npairs = 0;
  for (int64_t c = 0; c < nc; ++c) npairs += ilen[c] / 2;
  npairs += next / 2;
  int32_t* u = (int32_t*)malloc(sizeof(int32_t) * (size_t)(npairs > 0 ? npairs : 1));
  int32_t* v = (int32_t*)malloc(sizeof(int32_t) * (size_t)(npairs > 0 ? npairs : 1));
  float* w = (float*)malloc(sizeof(float) * (size_t)(npairs > 0 ? npairs : 1));
  {
    int64_t o = 0;
    for (int64_t c = 0; c < nc; ++c) {
      int64_t len = ilen[c];
      for (int64_t t = 0; t + 1 < len; t += 2) {
        u[o] = istub[ioff[c] + t];
        v[o] = istub[ioff[c] + t + 1];
        ++o;
      }
    }
    for (int64_t t = 0; t + 1 < next; t += 2) {
      u[o] = estub[t];
      v[o] = estub[t + 1];
      ++o;
    }
  }
  free(istub);
  free(estub);
  free(ioff);
  free(ilen);
  free(cstart);
  free(cperm);
  free(csize);
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t e = 0; e < npairs; ++e) {
    uint64_t a = (uint64_t)(uint32_t)(u[e] < v[e] ? u[e] : v[e]);
    uint64_t b = (uint64_t)(uint32_t)(u[e] < v[e] ? v[e] : u[e]);
    uint64_t h = mix64(seed ^ mix64((a << 32) | b));
    w[e] = (float)(1 + (int32_t)(h % (uint64_t)wmax));
  }
  int rc2 = build_sym_csr(n, npairs, u, v, w, 0, T, out);
  free(u);
  free(v);
  free(w);
  return rc2;
}

/* --------------------------------------------- batch member (uneven SBM graphs) */

/* One graph of the batched workload.  Graph g draws from streams tagged by g:
 * n log-uniform in [nmin, nmax], average degree uniform in [dmin, dmax], community
 * count log-uniform in [cmin, cmax] capped at floor(n / 20) (at least 1), equal sizes
 * (community of i = i * nc / n).  round(n * davg / 2) edge draws: u uniform; with
 * probability p_in the partner is uniform inside u's community, else uniform outside
 * it.  Self-loops and repeats dropped, unit weights. */
int gg_sbm_member(uint64_t seed, int64_t g, int32_t nmin, int32_t nmax, double dmin,
                  double dmax, int32_t cmin, int32_t cmax, double p_in, gg_csr* out) {
  if (nmin < 2 || nmax < nmin) return -1;
  memset(out, 0, sizeof(*out));
  rng_t r = rng_stream(seed, 401, (uint64_t)g);
  int32_t n = (int32_t)floor(exp(log((double)nmin) +
                                 rng_uniform(&r) * (log((double)nmax + 1.0) - log((double)nmin))));
  if (n < nmin) n = nmin;
  if (n > nmax) n = nmax;
  double davg = dmin + rng_uniform(&r) * (dmax - dmin);
  int32_t nc = (int32_t)floor(exp(log((double)cmin) +
                                  rng_uniform(&r) * (log((double)cmax + 1.0) - log((double)cmin))));
  if (nc > cmax) nc = cmax;
  if (nc > n / 20) nc = n / 20;
  if (nc < 1) nc = 1;
  int64_t E = (int64_t)llround((double)n * davg / 2.0);
  int32_t* u = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  int32_t* v = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  for (int64_t e = 0; e < E; ++e) {
    int32_t a = (int32_t)rng_below(&r, (uint64_t)n);
    int32_t ca = (int32_t)(((int64_t)a * nc) / n);
    /* community ca covers [lo, hi) */
    int32_t lo = (int32_t)(((int64_t)ca * n + nc - 1) / nc);
    int32_t hi = (int32_t)(((int64_t)(ca + 1) * n + nc - 1) / nc);
    int32_t b;
    if (nc == 1 || rng_uniform(&r) < p_in) {
      b = lo + (int32_t)rng_below(&r, (uint64_t)(hi - lo));
    } else {
      int32_t t = (int32_t)rng_below(&r, (uint64_t)(n - (hi - lo)));
      b = t < lo ? t : t + (hi - lo);
    }
    u[e] = a;
    v[e] = b;
  }
  int rc = build_sym_csr(n, E, u, v, NULL, 0, 1, out);
  free(u);
  free(v);
  return rc;
}
