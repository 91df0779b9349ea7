/*
 * Seeded synthetic corpora for the n-gram counting workloads.
 *
 * This file generates INPUTS only. It contains none of the counting method:
 * no window enumeration, no counting, no selection. Both the CUDA path and the
 * CPU oracle consume what it writes.
 *
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), keyed per
 * sequence so that sequences can be generated in parallel and reproducibly.
 * Discrete draws use Vose's alias method (Vose 1991). Normal deviates use the
 * Box-Muller transform; Gamma deviates use Marsaglia & Tsang (2000), with the
 * U^(1/a) boost for shape a < 1.
 *
 * Byte models (stand-ins for the paper's datasets, which are not available):
 *   MARKOV  : order-1 Markov chain over 256 symbols. Row a puts Zipf(s) mass
 *             on a row-specific random permutation of the symbols. Optional
 *             zero blocks and planted motifs (a Zipf-drawn pool of substrings).
 *   UNIFORM : uniform random bytes, with optional planted motifs.
 *   DNA     : order-3 Markov chain over {A,C,G,T} = codes 0..3 with
 *             Dirichlet(alpha) rows, plus repeat segments copied from earlier
 *             in the same sequence with point mutations. Output is packed
 *             2 bits per base, most significant bits first within each byte,
 *             sequences concatenated at arbitrary base offsets.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox */

static void philox4x32_10(const uint32_t in_ctr[4], const uint32_t in_key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = in_ctr[0], c1 = in_ctr[1], c2 = in_ctr[2], c3 = in_ctr[3];
  uint32_t k0 = in_key[0], k1 = in_key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t buf[4];
  int idx;
} rng_t;

/* Stream `stream` of generator `seed`: key = (seed low, seed high ^ stream
 * mix), counter word 2 carries the stream id so distinct streams never share
 * a counter block. */
static void rng_init(rng_t* r, uint64_t seed, uint32_t stream, uint32_t purpose) {
  r->key[0] = (uint32_t)seed;
  r->key[1] = (uint32_t)(seed >> 32) ^ 0x5EED1234u;
  r->ctr[0] = 0; r->ctr[1] = 0; r->ctr[2] = stream; r->ctr[3] = purpose;
  r->idx = 4;
}

static inline uint32_t rng_u32(rng_t* r) {
  if (r->idx == 4) {
    philox4x32_10(r->ctr, r->key, r->buf);
    if (++r->ctr[0] == 0) ++r->ctr[1];
    r->idx = 0;
  }
  return r->buf[r->idx++];
}

/* uniform in (0, 1), 53-bit resolution */
static inline double rng_unif(rng_t* r) {
  uint64_t a = rng_u32(r) >> 5, b = rng_u32(r) >> 6;
  return ((double)((a << 26) | b) + 0.5) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, n) by the multiply-high method (n < 2^32) */
static inline uint32_t rng_below(rng_t* r, uint32_t n) {
  return (uint32_t)(((uint64_t)rng_u32(r) * n) >> 32);
}

static double rng_normal(rng_t* r) {
  double u1 = rng_unif(r), u2 = rng_unif(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static double rng_gamma(rng_t* r, double a) {
  if (a < 1.0) {
    double g = rng_gamma(r, a + 1.0);
    return g * pow(rng_unif(r), 1.0 / a);
  }
  double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  for (;;) {
    double x, v;
    do { x = rng_normal(r); v = 1.0 + c * x; } while (v <= 0.0);
    v = v * v * v;
    double u = rng_unif(r);
    if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
  }
}

/* ------------------------------------------------------------- alias table */

typedef struct {
  uint32_t n;
  uint32_t* thresh; /* accept index i when a 32-bit draw < thresh[i] */
  uint32_t* alias;
} alias_t;

static int alias_build(alias_t* t, const double* w, uint32_t n) {
  t->n = n;
  t->thresh = (uint32_t*)malloc(sizeof(uint32_t) * n);
  t->alias = (uint32_t*)malloc(sizeof(uint32_t) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  uint32_t* small = (uint32_t*)malloc(sizeof(uint32_t) * n);
  uint32_t* large = (uint32_t*)malloc(sizeof(uint32_t) * n);
  if (!t->thresh || !t->alias || !p || !small || !large) {
    free(p); free(small); free(large);
    return -1;
  }
  double sum = 0.0;
  for (uint32_t i = 0; i < n; ++i) sum += w[i];
  uint32_t ns = 0, nl = 0;
  for (uint32_t i = 0; i < n; ++i) {
    p[i] = w[i] * n / sum;
    if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns && nl) {
    uint32_t s = small[--ns], l = large[--nl];
    t->thresh[s] = (uint32_t)fmin(4294967295.0, floor(p[s] * 4294967296.0));
    t->alias[s] = l;
    p[l] = (p[l] + p[s]) - 1.0;
    if (p[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl) { uint32_t l = large[--nl]; t->thresh[l] = 0xFFFFFFFFu; t->alias[l] = l; }
  while (ns) { uint32_t s = small[--ns]; t->thresh[s] = 0xFFFFFFFFu; t->alias[s] = s; }
  free(p); free(small); free(large);
  return 0;
}

static inline uint32_t alias_draw(const alias_t* t, rng_t* r) {
  uint32_t i = rng_below(r, t->n);
  return (rng_u32(r) < t->thresh[i]) ? i : t->alias[i];
}

static void alias_free(alias_t* t) { free(t->thresh); free(t->alias); }

/* ------------------------------------------------------------------ models */

enum { SYNTH_MARKOV = 0, SYNTH_UNIFORM = 1, SYNTH_DNA = 2 };

typedef struct {
  uint32_t kind;
  double markov_zipf_s;     /* MARKOV: Zipf exponent of each transition row */
  double zero_block_frac;   /* MARKOV: fraction of blocks replaced by zeros */
  uint32_t block;           /* block size for zero runs and motif planting */
  uint32_t n_motifs;        /* motif pool size (0 = none) */
  uint32_t motif_len_lo, motif_len_hi;
  double motif_zipf_s;      /* Zipf exponent of motif popularity */
  double motif_rate;        /* probability of planting one motif per block */
  double dirichlet_alpha;   /* DNA: transition rows ~ Dirichlet(alpha) */
  double repeat_frac;       /* DNA: target fraction of bases inside repeats */
  uint32_t repeat_len_lo, repeat_len_hi;
  double mutation_rate;     /* DNA: per-base substitution rate in repeats */
} synth_spec;

typedef struct {
  synth_spec spec;
  uint64_t seed;
  uint8_t perm[256][256];   /* MARKOV: row a, rank r -> symbol */
  alias_t rank_alias;       /* MARKOV: Zipf over ranks 0..255 */
  alias_t motif_alias;      /* Zipf over motif pool indices */
  uint8_t* motif_bytes;
  uint64_t* motif_off;      /* n_motifs + 1 */
  uint32_t dna_thresh[64][3]; /* DNA: cumulative thresholds of each context row */
} synth_model;

void synth_model_free(synth_model* M) {
  if (!M) return;
  alias_free(&M->rank_alias);
  alias_free(&M->motif_alias);
  free(M->motif_bytes);
  free(M->motif_off);
  free(M);
}

synth_model* synth_model_new(const synth_spec* spec, uint64_t seed) {
  synth_model* M = (synth_model*)calloc(1, sizeof(synth_model));
  if (!M) return NULL;
  M->spec = *spec;
  M->seed = seed;
  rng_t r;
  rng_init(&r, seed, 0xFFFFFFF0u, 1);
  /* per-row random permutations (Fisher-Yates) */
  for (int a = 0; a < 256; ++a) {
    for (int i = 0; i < 256; ++i) M->perm[a][i] = (uint8_t)i;
    for (int i = 255; i > 0; --i) {
      uint32_t j = rng_below(&r, (uint32_t)i + 1);
      uint8_t t = M->perm[a][i]; M->perm[a][i] = M->perm[a][j]; M->perm[a][j] = t;
    }
  }
  double w[256];
  for (int i = 0; i < 256; ++i) w[i] = pow((double)(i + 1), -spec->markov_zipf_s);
  if (alias_build(&M->rank_alias, w, 256)) { synth_model_free(M); return NULL; }
  /* motif pool */
  uint32_t nm = spec->n_motifs;
  M->motif_off = (uint64_t*)calloc((size_t)nm + 1, sizeof(uint64_t));
  if (!M->motif_off) { synth_model_free(M); return NULL; }
  for (uint32_t i = 0; i < nm; ++i) {
    uint32_t span = spec->motif_len_hi - spec->motif_len_lo + 1;
    M->motif_off[i + 1] = M->motif_off[i] + spec->motif_len_lo + rng_below(&r, span);
  }
  M->motif_bytes = (uint8_t*)malloc(M->motif_off[nm] + 1);
  if (!M->motif_bytes) { synth_model_free(M); return NULL; }
  for (uint64_t i = 0; i < M->motif_off[nm]; ++i) M->motif_bytes[i] = (uint8_t)(rng_u32(&r) >> 24);
  if (nm) {
    double* mw = (double*)malloc(sizeof(double) * nm);
    if (!mw) { synth_model_free(M); return NULL; }
    for (uint32_t i = 0; i < nm; ++i) mw[i] = pow((double)(i + 1), -spec->motif_zipf_s);
    int rc = alias_build(&M->motif_alias, mw, nm);
    free(mw);
    if (rc) { synth_model_free(M); return NULL; }
  }
  /* DNA context rows */
  for (int c = 0; c < 64; ++c) {
    double g[4], s = 0.0;
    for (int b = 0; b < 4; ++b) { g[b] = rng_gamma(&r, spec->dirichlet_alpha > 0 ? spec->dirichlet_alpha : 0.5); s += g[b]; }
    double acc = 0.0;
    for (int b = 0; b < 3; ++b) {
      acc += g[b] / s;
      double t = floor(acc * 4294967296.0);
      M->dna_thresh[c][b] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
  }
  return M;
}

/* ----------------------------------------------------------------- lengths */

/* dist 0: uniform integer in [lo, hi]. dist 1: lognormal with the given
 * median and log-sd, rounded and clamped to [lo, hi]. */
void synth_lengths(uint32_t dist, double median, double sigma, uint64_t lo, uint64_t hi,
                   uint64_t seed, uint32_t m, uint64_t* out) {
  rng_t r;
  rng_init(&r, seed, 0xFFFFFFF1u, 2);
  for (uint32_t i = 0; i < m; ++i) {
    uint64_t L;
    if (dist == 0) {
      uint64_t span = hi - lo + 1;
      uint64_t u = ((uint64_t)rng_u32(&r) << 32) | rng_u32(&r);
      L = lo + u % span;
    } else {
      double x = exp(log(median) + sigma * rng_normal(&r));
      double v = floor(x + 0.5);
      if (v < (double)lo) v = (double)lo;
      if (v > (double)hi) v = (double)hi;
      L = (uint64_t)v;
    }
    out[i] = L;
  }
}

/* ------------------------------------------------------------ generation */

static void gen_bytes(const synth_model* M, uint32_t seq, uint8_t* dst, uint64_t L) {
  const synth_spec* S = &M->spec;
  rng_t r;
  rng_init(&r, M->seed, seq, 3);
  if (S->kind == SYNTH_MARKOV) {
    uint32_t prev = 0; /* the first symbol is drawn from row 0 */
    for (uint64_t p = 0; p < L; ++p) {
      uint32_t cur = M->perm[prev][alias_draw(&M->rank_alias, &r)];
      dst[p] = (uint8_t)cur;
      prev = cur;
    }
  } else {
    uint64_t p = 0;
    for (; p + 4 <= L; p += 4) {
      uint32_t u = rng_u32(&r);
      memcpy(dst + p, &u, 4);
    }
    for (; p < L; ++p) dst[p] = (uint8_t)(rng_u32(&r) >> 24);
  }
  /* zero blocks and planted motifs, block by block */
  uint32_t B = S->block ? S->block : 4096;
  rng_t q;
  rng_init(&q, M->seed, seq, 4);
  for (uint64_t b0 = 0; b0 < L; b0 += B) {
    uint64_t blen = (L - b0 < B) ? L - b0 : B;
    double u = rng_unif(&q);
    if (S->kind == SYNTH_MARKOV && u < S->zero_block_frac) {
      memset(dst + b0, 0, blen);
      continue;
    }
    if (S->n_motifs && rng_unif(&q) < S->motif_rate) {
      uint32_t mi = alias_draw(&M->motif_alias, &q);
      uint64_t mlen = M->motif_off[mi + 1] - M->motif_off[mi];
      if (mlen <= blen) {
        uint64_t off = rng_below(&q, (uint32_t)(blen - mlen + 1));
        memcpy(dst + b0 + off, M->motif_bytes + M->motif_off[mi], mlen);
      }
    }
  }
}

static void gen_dna(const synth_model* M, uint32_t seq, uint8_t* codes, uint64_t L) {
  const synth_spec* S = &M->spec;
  rng_t r;
  rng_init(&r, M->seed, seq, 5);
  uint32_t ctx = 0;
  for (uint64_t p = 0; p < L; ++p) {
    uint32_t b;
    if (p < 3) {
      b = rng_u32(&r) >> 30;
    } else {
      uint32_t u = rng_u32(&r);
      const uint32_t* t = M->dna_thresh[ctx];
      b = (u < t[0]) ? 0 : (u < t[1]) ? 1 : (u < t[2]) ? 2 : 3;
    }
    codes[p] = (uint8_t)b;
    ctx = ((ctx << 2) | b) & 63u;
  }
  if (S->repeat_frac <= 0.0) return;
  /* repeat segments: starts form a Bernoulli process whose rate gives the
   * target fraction of bases inside repeats */
  rng_t q;
  rng_init(&q, M->seed, seq, 6);
  double mean_len = 0.5 * (S->repeat_len_lo + S->repeat_len_hi);
  double rate = S->repeat_frac / (mean_len * (1.0 - S->repeat_frac));
  uint64_t p = S->repeat_len_hi;
  for (;;) {
    double gap = floor(log(rng_unif(&q)) / log(1.0 - rate));
    if (gap > (double)L) break;
    p += (uint64_t)gap;
    uint32_t len = S->repeat_len_lo + rng_below(&q, S->repeat_len_hi - S->repeat_len_lo + 1);
    if (p + len > L || p < len) break;
    uint64_t src = (uint64_t)rng_below(&q, (uint32_t)(p - len + 1));
    for (uint32_t t = 0; t < len; ++t) {
      uint8_t b = codes[src + t];
      if (rng_unif(&q) < S->mutation_rate) b = (uint8_t)((b + 1 + rng_below(&q, 3)) & 3u);
      codes[p + t] = b;
    }
    p += len;
  }
}

typedef struct {
  const synth_model* M;
  const uint64_t* offsets;
  uint8_t* out;
  uint32_t m;
  uint32_t next;           /* work counter (atomic) */
  uint64_t max_len;
} fill_job;

static void pack_dna(uint8_t* out, uint64_t start, const uint8_t* codes, uint64_t L) {
  uint64_t p = 0;
  /* leading partial byte shared with the previous sequence */
  while (p < L && ((start + p) & 3u)) {
    uint64_t g = start + p;
    uint8_t v = (uint8_t)(codes[p] << (6 - 2 * (g & 3u)));
    __atomic_fetch_or(out + (g >> 2), v, __ATOMIC_RELAXED);
    ++p;
  }
  for (; p + 4 <= L; p += 4) {
    uint64_t g = start + p;
    out[g >> 2] = (uint8_t)((codes[p] << 6) | (codes[p + 1] << 4) | (codes[p + 2] << 2) | codes[p + 3]);
  }
  for (; p < L; ++p) {
    uint64_t g = start + p;
    uint8_t v = (uint8_t)(codes[p] << (6 - 2 * (g & 3u)));
    __atomic_fetch_or(out + (g >> 2), v, __ATOMIC_RELAXED);
  }
}

static void* fill_worker(void* arg) {
  fill_job* J = (fill_job*)arg;
  uint8_t* codes = NULL;
  if (J->M->spec.kind == SYNTH_DNA) {
    codes = (uint8_t*)malloc(J->max_len ? J->max_len : 1);
    if (!codes) return (void*)1;
  }
  for (;;) {
    uint32_t i = __atomic_fetch_add(&J->next, 1u, __ATOMIC_RELAXED);
    if (i >= J->m) break;
    uint64_t a = J->offsets[i], L = J->offsets[i + 1] - a;
    if (J->M->spec.kind == SYNTH_DNA) {
      gen_dna(J->M, i, codes, L);
      pack_dna(J->out, a, codes, L);
    } else {
      gen_bytes(J->M, i, J->out + a, L);
    }
  }
  free(codes);
  return NULL;
}

/* Fill `out` with the m sequences delimited by offsets[0..m] (in symbols).
 * For DNA, `out` must hold ceil(offsets[m] / 4) bytes and is zeroed here.
 * Returns 0 on success. */
int synth_fill(const synth_model* M, uint32_t m, const uint64_t* offsets, uint8_t* out, int nthreads) {
  fill_job J;
  J.M = M; J.offsets = offsets; J.out = out; J.m = m; J.next = 0; J.max_len = 0;
  for (uint32_t i = 0; i < m; ++i) {
    uint64_t L = offsets[i + 1] - offsets[i];
    if (L > J.max_len) J.max_len = L;
  }
  if (M->spec.kind == SYNTH_DNA) memset(out, 0, (size_t)((offsets[m] + 3) / 4));
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0, rc = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, fill_worker, &J) == 0) ++started; else break;
  }
  if (fill_worker(&J)) rc = -1;
  for (int t = 1; t <= started; ++t) {
    void* ret = NULL;
    pthread_join(th[t], &ret);
    if (ret) rc = -1;
  }
  return rc;
}

/* Raw Philox output, exposed so tests can check the generator against the
 * published known-answer vectors. */
void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox4x32_10(ctr, key, out);
}
