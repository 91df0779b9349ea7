/*
 * CPU ORACLE for top-k n-gram counting (test infrastructure only).
 *
 * This file is the plain, slow reference the GPU path is checked against. It
 * is used only by the tests, by the package's smoke check and by the CPU
 * baseline leg of the benchmark; the product path never calls it. It shares
 * no code with the CUDA library.
 *
 * Everything is written directly from the paper's definitions, with qsort and
 * bsearch from the C library as the only primitives, and no blocking, fusion
 * or reordering beyond what the definitions state:
 *
 *   Problem statement (Sec. 2, Eq. 1 and Eq. 2): a sequence s_i contributes
 *   the windows s_i[p .. p+n), p = 0 .. |s_i|-n. Under Eq. 1 every window
 *   counts once ("count every occurrence"); under Eq. 2 an n-gram counts once
 *   per sequence that contains it ("count once per sequence", the paper's
 *   focus and the default here). The answer is the k-argmax of the counts.
 *
 *   Naive method (Sec. 3): gather all n-grams, count them, sort by count and
 *   keep the top k.  -> oracle_exhaustive
 *
 *   Intergrams (Sec. 7, Algorithm 3, with Algorithm 2 as its first pass):
 *   P^(b) = the top-Z b-grams of an exact count (b = base length, 3 in the
 *   paper); for j = b+1 .. n, count only the j-grams whose (j-1)-gram prefix
 *   is in P^(j-1); if j < n, P^(j) = the top-Z of those counts; finally
 *   return the top k of the last counts.  -> oracle_intergrams
 *
 * Readings where the paper is silent (each one is listed with the design):
 *   - ties are broken by count descending, then by the n-gram's symbols in
 *     ascending unsigned order, at every selection (intermediate and final);
 *   - only nonzero counts are ever selected, so fewer than Z (or k) results
 *     are returned when fewer distinct n-grams exist;
 *   - a sequence shorter than j contributes no j-grams; windows never cross
 *     sequence boundaries;
 *   - Z (the paper's zk) is given as an integer.
 *
 * Symbols: with symbol_bits = 8 each byte of `data` is one symbol (0..255);
 * with symbol_bits = 2 each byte holds four base codes (0..3), most
 * significant bits first, and sequence boundaries are given in bases. The
 * oracle unpacks to one code per byte before anything else. Output keys are
 * written one symbol code per byte (k_out rows of n bytes).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };

/* ------------------------------------------------------------- symbols */

static uint8_t* unpack_symbols(const uint8_t* data, uint64_t total, uint32_t symbol_bits) {
  uint8_t* s = (uint8_t*)malloc(total ? total : 1);
  if (!s) return NULL;
  if (symbol_bits == 8) {
    memcpy(s, data, total);
  } else {
    for (uint64_t g = 0; g < total; ++g) s[g] = (uint8_t)((data[g >> 2] >> (6 - 2 * (g & 3))) & 3u);
  }
  return s;
}

/* qsort has no context argument in ISO C; the oracle is single-threaded, so
 * the symbol array and window length being compared live in file scope. */
static const uint8_t* g_sym;
static uint32_t g_len;

static int cmp_window(const void* a, const void* b) {
  uint64_t pa = *(const uint64_t*)a, pb = *(const uint64_t*)b;
  return memcmp(g_sym + pa, g_sym + pb, g_len);
}

typedef struct {
  uint64_t pos;   /* position of one occurrence (the n-gram's symbols) */
  uint64_t count;
} gram_count;

/* count descending, then symbols ascending */
static int cmp_count_then_symbols(const void* a, const void* b) {
  const gram_count* x = (const gram_count*)a;
  const gram_count* y = (const gram_count*)b;
  if (x->count != y->count) return x->count > y->count ? -1 : 1;
  return memcmp(g_sym + x->pos, g_sym + y->pos, g_len);
}

/* ---------------------------------------------------- the counting step */

/* Membership of a (len)-symbol string in a sorted table of keys. */
typedef struct {
  uint8_t* keys;  /* nkeys rows of len symbols, ascending */
  uint64_t nkeys;
  uint32_t len;
} key_set;

static int cmp_key_row(const void* key, const void* row) {
  return memcmp(key, row, g_len);
}

static int in_set(const key_set* P, const uint8_t* s) {
  if (!P) return 1;
  uint32_t save = g_len;
  g_len = P->len;
  int hit = bsearch(s, P->keys, P->nkeys, P->len, cmp_key_row) != NULL;
  g_len = save;
  return hit;
}

/*
 * Count the j-grams of the corpus, keeping only windows whose (j-1)-prefix is
 * in `prefixes` (all windows when prefixes == NULL).
 *   Eq. 1 (count_mode 1): every kept window adds one.
 *   Eq. 2 (count_mode 0): each sequence adds one per distinct kept j-gram.
 * Returns the distinct j-grams with nonzero counts (one representative
 * position each) in *out, their number in *nout.
 */
static int count_grams(const uint8_t* sym, const uint64_t* offsets, uint32_t m, uint32_t j,
                       uint32_t count_mode, const key_set* prefixes,
                       gram_count** out, uint64_t* nout) {
  uint64_t nwin = 0;
  for (uint32_t i = 0; i < m; ++i) {
    uint64_t L = offsets[i + 1] - offsets[i];
    if (L >= j) nwin += L - j + 1;
  }
  uint64_t* pos = (uint64_t*)malloc(sizeof(uint64_t) * (nwin ? nwin : 1));
  if (!pos) return OR_ENOMEM;
  uint64_t np = 0;
  g_sym = sym;
  for (uint32_t i = 0; i < m; ++i) {
    uint64_t a = offsets[i], L = offsets[i + 1] - a;
    if (L < j) continue;
    uint64_t first = np;
    for (uint64_t p = a; p + j <= a + L; ++p) {
      if (prefixes && !in_set(prefixes, sym + p)) continue;
      pos[np++] = p;
    }
    if (count_mode == 0 && np > first) {
      /* Eq. 2: keep one window per distinct j-gram of this sequence */
      g_len = j;
      qsort(pos + first, np - first, sizeof(uint64_t), cmp_window);
      uint64_t w = first + 1;
      for (uint64_t r = first + 1; r < np; ++r)
        if (memcmp(sym + pos[r], sym + pos[w - 1], j) != 0) pos[w++] = pos[r];
      np = w;
    }
  }
  /* gather equal j-grams together and count them */
  g_len = j;
  qsort(pos, np, sizeof(uint64_t), cmp_window);
  gram_count* gc = (gram_count*)malloc(sizeof(gram_count) * (np ? np : 1));
  if (!gc) { free(pos); return OR_ENOMEM; }
  uint64_t nd = 0;
  for (uint64_t r = 0; r < np; ++r) {
    if (nd && memcmp(sym + pos[r], sym + gc[nd - 1].pos, j) == 0) {
      gc[nd - 1].count += 1;
    } else {
      gc[nd].pos = pos[r];
      gc[nd].count = 1;
      ++nd;
    }
  }
  free(pos);
  *out = gc;
  *nout = nd;
  return OR_OK;
}

/* Sort by (count desc, symbols asc) and keep the first `keep` entries. */
static uint64_t select_top(const uint8_t* sym, gram_count* gc, uint64_t nd, uint32_t j, uint64_t keep) {
  g_sym = sym;
  g_len = j;
  qsort(gc, nd, sizeof(gram_count), cmp_count_then_symbols);
  return nd < keep ? nd : keep;
}

static void write_top(const uint8_t* sym, const gram_count* gc, uint64_t nk, uint32_t j,
                      uint8_t* keys_out, uint64_t* counts_out) {
  for (uint64_t r = 0; r < nk; ++r) {
    if (keys_out) memcpy(keys_out + r * j, sym + gc[r].pos, j);
    if (counts_out) counts_out[r] = gc[r].count;
  }
}

static int valid_corpus(const uint64_t* offsets, uint32_t m, uint32_t symbol_bits) {
  if (symbol_bits != 8 && symbol_bits != 2) return 0;
  if (offsets[0] != 0) return 0;
  for (uint32_t i = 0; i < m; ++i)
    if (offsets[i + 1] < offsets[i]) return 0;
  return 1;
}

/* ------------------------------------------------------------ public API */

/*
 * Exhaustive top-k (Eq. 1 / Eq. 2 and the naive method of Sec. 3).
 * keys_out: k rows of n symbol codes; counts_out: k counts; *k_out: rows
 * written (= min(k, number of distinct n-grams)).
 */
int oracle_exhaustive(const uint8_t* data, const uint64_t* offsets, uint32_t m, uint32_t symbol_bits,
                      uint32_t n, uint32_t count_mode, uint64_t k,
                      uint8_t* keys_out, uint64_t* counts_out, uint64_t* k_out) {
  *k_out = 0;
  if (n == 0 || !valid_corpus(offsets, m, symbol_bits)) return OR_EINVAL;
  uint8_t* sym = unpack_symbols(data, offsets[m], symbol_bits);
  if (!sym) return OR_ENOMEM;
  gram_count* gc = NULL;
  uint64_t nd = 0;
  int rc = count_grams(sym, offsets, m, n, count_mode, NULL, &gc, &nd);
  if (rc == OR_OK) {
    uint64_t nk = select_top(sym, gc, nd, n, k);
    write_top(sym, gc, nk, n, keys_out, counts_out);
    *k_out = nk;
  }
  free(gc);
  free(sym);
  return rc;
}

/*
 * Intergrams (Algorithm 3 with Algorithm 2 generalised to a base length b):
 *   pass b     : exact counts of all b-grams; if b < n, P^(b) = top-Z;
 *   pass j > b : counts of the j-grams whose (j-1)-prefix is in P^(j-1);
 *                if j < n, P^(j) = top-Z of these counts;
 *   result     : top-k of the counts of the last pass run.
 * When n <= b the single exact pass over n-grams is the answer.
 * `stop_j` (b <= stop_j <= n, or 0 for n) ends the run after pass stop_j and
 * returns that pass's top-k; this equals the top-k a caller sees after that
 * pass of a run to n, because passes never look ahead.
 * `survivors_out` (optional): number of windows counted in the last pass
 * (their prefix was in the candidate set); used by the Lemma 1 test.
 */
int oracle_intergrams(const uint8_t* data, const uint64_t* offsets, uint32_t m, uint32_t symbol_bits,
                      uint32_t n, uint32_t base_n, uint64_t Z, uint32_t count_mode, uint64_t k,
                      uint32_t stop_j, uint8_t* keys_out, uint64_t* counts_out, uint64_t* k_out,
                      uint64_t* survivors_out) {
  *k_out = 0;
  if (n == 0 || base_n == 0 || Z == 0 || !valid_corpus(offsets, m, symbol_bits)) return OR_EINVAL;
  if (stop_j == 0) stop_j = n;
  uint32_t b = base_n < n ? base_n : n;
  if (stop_j < b || stop_j > n) return OR_EINVAL;
  uint8_t* sym = unpack_symbols(data, offsets[m], symbol_bits);
  if (!sym) return OR_ENOMEM;

  key_set P = {NULL, 0, 0};
  gram_count* gc = NULL;
  uint64_t nd = 0;
  int rc = OR_OK;
  for (uint32_t j = b; j <= stop_j; ++j) {
    free(gc);
    gc = NULL;
    if (survivors_out && j == stop_j) {
      /* count the windows kept in this pass, before any per-sequence dedupe */
      uint64_t kept = 0;
      for (uint32_t i = 0; i < m; ++i) {
        uint64_t a = offsets[i], L = offsets[i + 1] - a;
        for (uint64_t p = a; L >= j && p + j <= a + L; ++p)
          if (j == b || in_set(&P, sym + p)) ++kept;
      }
      *survivors_out = kept;
    }
    rc = count_grams(sym, offsets, m, j, count_mode, j == b ? NULL : &P, &gc, &nd);
    if (rc != OR_OK) break;
    if (j == stop_j) break;
    /* P^(j) = top-Z j-grams by (count desc, symbols asc), stored sorted by
     * symbols so that membership is a binary search */
    uint64_t nz = select_top(sym, gc, nd, j, Z);
    free(P.keys);
    P.keys = (uint8_t*)malloc((size_t)(nz ? nz : 1) * j);
    if (!P.keys) { rc = OR_ENOMEM; break; }
    for (uint64_t r = 0; r < nz; ++r) memcpy(P.keys + r * j, sym + gc[r].pos, j);
    P.nkeys = nz;
    P.len = j;
    g_len = j;
    qsort(P.keys, nz, j, cmp_key_row);
  }
  if (rc == OR_OK) {
    uint64_t nk = select_top(sym, gc, nd, stop_j, k);
    write_top(sym, gc, nk, stop_j, keys_out, counts_out);
    *k_out = nk;
  }
  free(gc);
  free(P.keys);
  free(sym);
  return rc;
}

/*
 * One counting step of Algorithm 3 on its own (Sec. 7): the j-grams of the
 * corpus whose (j-1)-prefix is one of `prefixes` (nprefix rows of j-1 symbol
 * codes in ascending order; every j-gram when use_prefixes is 0, the dense
 * pass of Algorithm 2), counted by Eq. 1 (count_mode 1) or Eq. 2 (count_mode
 * 0). Writes every distinct counted j-gram with its count, in ascending
 * symbol order: keys_out (capacity rows of j codes), counts_out. *nout is
 * always the number of distinct j-grams; OR_EINVAL when it exceeds capacity.
 *
 * Sequences are independent under both equations, so the counts of a corpus
 * split into groups of whole sequences are the sums of the groups' counts;
 * the test harness uses this to run the oracle on several cores.
 */
int oracle_count_pass(const uint8_t* data, const uint64_t* offsets, uint32_t m, uint32_t symbol_bits, uint32_t j,
                      uint32_t count_mode, const uint8_t* prefixes, uint64_t nprefix, uint32_t use_prefixes,
                      uint8_t* keys_out, uint64_t* counts_out, uint64_t capacity, uint64_t* nout) {
  *nout = 0;
  if (j == 0 || (use_prefixes && j < 2) || !valid_corpus(offsets, m, symbol_bits)) return OR_EINVAL;
  uint8_t* sym = unpack_symbols(data, offsets[m], symbol_bits);
  if (!sym) return OR_ENOMEM;
  key_set P = {(uint8_t*)prefixes, nprefix, j - 1};
  gram_count* gc = NULL;
  uint64_t nd = 0;
  int rc = count_grams(sym, offsets, m, j, count_mode, use_prefixes ? &P : NULL, &gc, &nd);
  if (rc == OR_OK) {
    *nout = nd;
    if (nd > capacity) {
      rc = OR_EINVAL;
    } else {
      /* count_grams leaves the distinct j-grams in ascending symbol order */
      write_top(sym, gc, nd, j, keys_out, counts_out);
    }
  }
  free(gc);
  free(sym);
  return rc;
}

/* ----------------------------------------------------- counting given keys */

static uint8_t symbol_at(const uint8_t* data, uint32_t symbol_bits, uint64_t g) {
  if (symbol_bits == 8) return data[g];
  return (uint8_t)((data[g >> 2] >> (6 - 2 * (g & 3))) & 3u);
}

/*
 * Exact frequency of each of `nkeys` given n-grams (rows of n symbol codes),
 * by the definitions of Eq. 1 (count_mode 1: every window equal to the key)
 * and Eq. 2 (count_mode 0: the number of sequences containing the key), over
 * every window of every sequence. Used to check single outputs of a run on a
 * corpus too large for the exhaustive count. Keys may repeat; counts_out[i]
 * is the count of keys[i]. The scan is one pass over the corpus; a bitmap of
 * the keys' first symbols (2 for bytes, 8 for bases) rejects most windows
 * before a binary search over the sorted keys.
 */
int oracle_count_keys(const uint8_t* data, const uint64_t* offsets, uint32_t m, uint32_t symbol_bits, uint32_t n,
                      uint32_t count_mode, const uint8_t* keys, uint64_t nkeys, uint64_t* counts_out) {
  if (n == 0 || !valid_corpus(offsets, m, symbol_bits)) return OR_EINVAL;
  const uint32_t head = symbol_bits == 8 ? (n < 2 ? n : 2) : (n < 8 ? n : 8);
  uint8_t* sorted = (uint8_t*)malloc((size_t)(nkeys ? nkeys : 1) * n);
  uint64_t* cnt = (uint64_t*)calloc(nkeys ? nkeys : 1, sizeof(uint64_t));
  int64_t* last = (int64_t*)malloc(sizeof(int64_t) * (nkeys ? nkeys : 1));
  uint8_t* bitmap = (uint8_t*)calloc(8192, 1);
  uint8_t* win = (uint8_t*)malloc(n);
  if (!sorted || !cnt || !last || !bitmap || !win) {
    free(sorted); free(cnt); free(last); free(bitmap); free(win);
    return OR_ENOMEM;
  }
  memcpy(sorted, keys, (size_t)nkeys * n);
  g_len = n;
  qsort(sorted, nkeys, n, cmp_key_row);
  for (uint64_t i = 0; i < nkeys; ++i) last[i] = -1;
  const uint32_t hb = symbol_bits == 8 ? 8 : 2;
  for (uint64_t i = 0; i < nkeys; ++i) {
    uint32_t code = 0;
    for (uint32_t t = 0; t < head; ++t) code = (code << hb) | sorted[i * n + t];
    bitmap[code >> 3] |= (uint8_t)(1u << (code & 7));
  }
  for (uint32_t s = 0; s < m; ++s) {
    const uint64_t a = offsets[s], L = offsets[s + 1] - a;
    if (L < n) continue;
    for (uint64_t p = a; p + n <= a + L; ++p) {
      uint32_t code = 0;
      for (uint32_t t = 0; t < head; ++t) code = (code << hb) | symbol_at(data, symbol_bits, p + t);
      if (!((bitmap[code >> 3] >> (code & 7)) & 1u)) continue;
      for (uint32_t t = 0; t < n; ++t) win[t] = symbol_at(data, symbol_bits, p + t);
      const uint8_t* hit = (const uint8_t*)bsearch(win, sorted, nkeys, n, cmp_key_row);
      if (!hit) continue;
      const uint64_t idx = (uint64_t)(hit - sorted) / n;
      if (count_mode == 1) {
        cnt[idx] += 1;
      } else if (last[idx] != (int64_t)s) {
        last[idx] = s;
        cnt[idx] += 1;
      }
    }
  }
  for (uint64_t i = 0; i < nkeys; ++i) {
    const uint8_t* hit = (const uint8_t*)bsearch(keys + i * n, sorted, nkeys, n, cmp_key_row);
    counts_out[i] = hit ? cnt[(uint64_t)(hit - sorted) / n] : 0;
  }
  free(sorted); free(cnt); free(last); free(bitmap); free(win);
  return OR_OK;
}

/*
 * The Boolean sequence x feature matrix that the top-k n-grams are chosen
 * for (Sec. 1, Fig. 1): entry (i, f) is 1 exactly when sequence i contains
 * the n-gram keys[f] (nkeys distinct rows of n symbol codes). Output in CSR
 * form: row_ptr[m + 1] and, when capacity allows, cols with the f of each
 * row in ascending order. *nnz_out is always set; OR_EINVAL if cols is too
 * small (cols then holds the first capacity entries).
 */
static const uint8_t* g_feat_rows;
static int cmp_feat_index(const void* a, const void* b) {
  const uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return memcmp(g_feat_rows + (size_t)x * g_len, g_feat_rows + (size_t)y * g_len, g_len);
}
static int cmp_u32(const void* a, const void* b) {
  const uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return x < y ? -1 : x > y;
}

int oracle_features(const uint8_t* data, const uint64_t* offsets, uint32_t m, uint32_t symbol_bits, uint32_t n,
                    const uint8_t* keys, uint32_t nkeys, uint64_t* row_ptr, uint32_t* cols, uint64_t capacity,
                    uint64_t* nnz_out) {
  *nnz_out = 0;
  if (n == 0 || !valid_corpus(offsets, m, symbol_bits)) return OR_EINVAL;
  const size_t nk = nkeys ? nkeys : 1;
  uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * nk);
  uint8_t* sorted = (uint8_t*)malloc(nk * n);
  uint8_t* present = (uint8_t*)calloc(nk, 1);
  uint32_t* touched = (uint32_t*)malloc(sizeof(uint32_t) * nk);
  uint8_t* win = (uint8_t*)malloc(n);
  if (!order || !sorted || !present || !touched || !win) {
    free(order); free(sorted); free(present); free(touched); free(win);
    return OR_ENOMEM;
  }
  for (uint32_t f = 0; f < nkeys; ++f) order[f] = f;
  g_len = n;
  g_feat_rows = keys;
  qsort(order, nkeys, sizeof(uint32_t), cmp_feat_index);
  for (uint32_t i = 0; i < nkeys; ++i) memcpy(sorted + (size_t)i * n, keys + (size_t)order[i] * n, n);
  uint64_t nnz = 0;
  row_ptr[0] = 0;
  for (uint32_t s = 0; s < m; ++s) {
    const uint64_t a = offsets[s], L = offsets[s + 1] - a;
    uint32_t nt = 0;
    for (uint64_t p = a; L >= n && p + n <= a + L; ++p) {
      for (uint32_t t = 0; t < n; ++t) win[t] = symbol_at(data, symbol_bits, p + t);
      const uint8_t* hit = (const uint8_t*)bsearch(win, sorted, nkeys, n, cmp_key_row);
      if (!hit) continue;
      const uint32_t f = order[(uint64_t)(hit - sorted) / n];
      if (!present[f]) {
        present[f] = 1;
        touched[nt++] = f;
      }
    }
    qsort(touched, nt, sizeof(uint32_t), cmp_u32);
    for (uint32_t t = 0; t < nt; ++t) {
      if (nnz < capacity) cols[nnz] = touched[t];
      ++nnz;
      present[touched[t]] = 0;
    }
    row_ptr[s + 1] = nnz;
  }
  free(order); free(sorted); free(present); free(touched); free(win);
  *nnz_out = nnz;
  return nnz <= capacity ? OR_OK : OR_EINVAL;
}
