/*
 * intergrams.h - C ABI of the GB300 (sm_103a) top-k n-gram library.
 *
 * Problem (paper Sec. 2, Eq. 1 and Eq. 2): given m sequences s_1..s_m over an
 * alphabet of sigma symbols, n and k, return the k most frequent n-grams
 * (contiguous length-n windows, never crossing a sequence boundary) with
 * their counts. Under Eq. 2 (the default) an n-gram counts once per sequence
 * that contains it; under Eq. 1 every occurrence counts. Ties are broken by
 * count descending, then by the n-gram's symbols in ascending order.
 *
 * Method (paper Sec. 6-7, Algorithm 2 and Algorithm 3): a dense first pass
 * counts every base_n-gram exactly (base_n = 3 in the paper); its top-Z form
 * the candidate set P^(base_n). Pass j = base_n+1 .. n counts only the
 * j-grams whose (j-1)-gram prefix is in P^(j-1), then keeps their top-Z as
 * P^(j). The answer is the top-k of the last pass. Z is the paper's zk.
 *
 * Conventions for every call:
 *   - No C++ exception crosses this boundary; every call returns ig_status.
 *     On an error the call also records a message for intergrams_last_error().
 *   - Work is ordered on the plan's CUDA stream. A plan is not thread-safe;
 *     distinct plans are independent and may be used from different threads.
 *   - All counts are exact integers. The GPU path is deterministic: the same
 *     inputs and parameters give byte-identical results regardless of the
 *     tuning choices.
 */
#ifndef INTERGRAMS_H
#define INTERGRAMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IG_OK = 0,
  IG_DONE = 1,            /* intergrams_pass: every pass has already run */
  IG_EINVAL = -1,         /* invalid argument or unsupported parameter combination */
  IG_ENOMEM = -2,         /* device or host allocation failed */
  IG_ETABLE_FULL = -3,    /* a device hash table ran out of room (internal limit) */
  IG_EOVERFLOW = -4,      /* a 32-bit device count overflowed (Eq. 1 on > 2^32-1 windows) */
  IG_ETIMEOUT = -5,       /* a bounded device-side wait gave up */
  IG_ECUDA = -6,          /* a CUDA runtime call failed; see intergrams_last_error() */
  IG_ESTATE = -7          /* call out of order (e.g. topk before any pass) */
} ig_status;

/* count_mode */
#define IG_COUNT_ONCE_PER_SEQUENCE 0u   /* Eq. 2 (paper's focus, default) */
#define IG_COUNT_EVERY_OCCURRENCE  1u   /* Eq. 1 */

/* flags */
#define IG_F_HOST_INPUT (1u << 0)  /* data/offsets are HOST pointers: the plan copies
                                      them to device memory it owns (stream-ordered) */
#define IG_F_GRAPH      (1u << 1)  /* capture each pass's launch sequence as a CUDA
                                      graph on first use and replay it afterwards */
#define IG_F_AUTOTUNE   (1u << 2)  /* let the autotuner pick the tuning knobs left at 0 */
#define IG_F_TIMING     (1u << 3)  /* record CUDA events around every scan kernel and pass
                                      (on the plan's stream) for intergrams_timings */
#define IG_F_OFFSETS_HOST (1u << 4) /* offsets is a HOST pointer (data stays on the device);
                                       the plan copies the offsets and needs no device read-back */
#define IG_F_ASYNC_ALLOC (1u << 5) /* allocate and free the plan's tables stream-ordered
                                      (cudaMallocAsync / cudaFreeAsync on the plan's stream) */
#define IG_F_DRY_RUN    (1u << 6)  /* size the plan without allocating or launching anything;
                                      only intergrams_plan_device_bytes and intergrams_free apply */
#define IG_F_SHARDED    (1u << 7)  /* this plan counts one shard of a corpus split across
                                      processes or GPUs (intergrams_pass_scan .. _select):
                                      32-bit counters, so every shard has the same layout */
#define IG_F_EXHAUSTIVE_CHECKS (1u << 8) /* after every scan, check on the device that no
                                      j-gram is counted above its (j-1)-prefix's count in the
                                      previous pass and, for counts the plan computed itself
                                      (not imported), that they sum to the registrations and
                                      that no Eq. 2 count exceeds m; a failed check ends the
                                      pass with IG_ESTATE */

typedef struct {
  uint32_t n;            /* target n-gram length in symbols: 1..64 */
  uint32_t k;            /* number of results wanted, >= 1 */
  uint32_t candidates;   /* Z: size of each intermediate candidate set P^(j); k <= Z < 2^24 */
  uint32_t base_n;       /* length of the dense first pass: 1..3 (bytes), 1..12 (2-bit);
                            the paper uses 3. Passes run for j = min(base_n, n) .. n */
  uint32_t symbol_bits;  /* 8: one symbol per byte; 2: bases A,C,G,T = 0..3 packed four per
                            byte, most significant bits first, sequences at any base offset */
  uint32_t count_mode;   /* IG_COUNT_ONCE_PER_SEQUENCE or IG_COUNT_EVERY_OCCURRENCE */
  uint32_t flags;        /* IG_F_* */
} ig_params;

/* Tuning knobs. A zero field means "default" (or "autotune" with IG_F_AUTOTUNE).
 * No knob changes any result; they only change speed and memory. */
typedef struct {
  uint32_t ctas_per_sm;      /* persistent scan CTAs per SM (1..4) */
  uint32_t threads;          /* threads per scan CTA (256, 512 or 1024) */
  uint32_t words_per_thread; /* 32-bit smem words of symbols each thread scans per tile (odd, 1..31) */
  uint32_t smem_set_log2;    /* log2 entries of the per-sequence shared-memory dedupe set (8..15) */
  uint32_t table_load_pct;   /* maximum load of the candidate probe table, percent (10..50) */
  uint32_t hot_log2;         /* log2 entries of the shared-memory cache of the most frequent
                                candidates in front of the probe table (6..13; default 11) */
  uint32_t chain_from;       /* first pass run from the previous pass's survivor lists instead of a
                                corpus scan (default: n - 1 for bytes when n >= base_n + 4, the
                                passes where few windows survive, else none; n + 1 = none); passes
                                whose (j-1)-gram exceeds 64 bits always run this way */
  uint32_t list_pct;         /* initial capacity of each survivor list, percent of the corpus
                                symbols (default: 100 when two full lists fit in 25% of the free
                                device memory, else 25). A pass that needs more makes
                                intergrams_run / intergrams_pass grow both lists to what was asked
                                for and run the job again; IG_ETABLE_FULL only when the device has
                                no memory for them (the plan then refuses further passes) */
  /* Registration log of the candidate passes: a count increment is appended to
     a log chunk of its counter range and the log is counted range by range
     after the scan, so the increments of any moment fall in one range of the
     counter array (results are identical; only speed and memory change). */
  uint32_t log_mode;         /* 0 = off (default), 1 = on */
  uint32_t log_pct;          /* log capacity in percent of the corpus symbols (default 60 under Eq. 2,
                                80 under Eq. 1, plus the chunks held open; at most a quarter of the
                                device memory). Registrations past it are counted at once */
  uint32_t log_chunk_log2;   /* log2 entries of a log chunk (14..20; default 18) */
  uint32_t log_range_log2;   /* log2 counters of one range (10..30; default 16 MiB of counters);
                                raised until there are at most 32 ranges */
  uint32_t dedupe_bitmap;    /* Eq. 2 dedupe of a pass by a per-CTA bit vector over its slots (the
                                paper's C_i, Sec. 6) instead of the shared-memory set with spill
                                lists: 0 = auto (when the scan CTAs' bit vectors take at most
                                48 MiB), 1 = never, 2 = whenever they fit in a quarter of the
                                device memory */
  uint32_t dense_prefix;     /* first candidate pass (j = base_n + 1), where every window is a
                                candidate: 0 = auto (when a dense map of the sigma^base_n prefixes
                                and the counter array take at most 112 MiB together, so both stay
                                in L2, each thread rolls the key over its own run of windows and
                                indexes the map; otherwise the queue path looks the prefix up by
                                rank/select in a bit vector of the candidate prefixes, 8 bytes per
                                32 prefixes), 1 = queue path with the hot cache and probe table,
                                2 = runs with the dense map, 3 = runs with the hot cache and probe
                                table, 4 = queue path with rank/select */
  uint32_t base_words_per_thread; /* the dense base pass's own words_per_thread and smem_set_log2 */
  uint32_t base_smem_set_log2;    /* (0 = the values above); it needs no queue or hot cache, so a */
                                  /* larger set fits beside a larger tile */
  uint32_t set_probes;       /* Eq. 2: positions a slot may take in the shared-memory set before it
                                goes to the spill list (1..8; default 1: fewest instructions per
                                window, measured fastest; skipping the set for long sequences
                                measured slower) */
  uint32_t tile_buffers;     /* corpus tiles staged by bulk copy into 2 shared-memory buffers (the
                                next tile's copy overlaps this tile's work) when both fit, else 1;
                                1 forces one buffer (0 = default 2) */
  uint32_t rs_depth;         /* with rank/select (dense_prefix 0 without the dense map, or 4): the
                                first rs_depth key-probe candidate passes (1..4; default 2) look
                                their prefix up level by level in bit vectors of the selected slots
                                instead of the hot cache and probe table */
  uint32_t tile_cache_hint;  /* L2 policy of the corpus tile copies: 1 = none, 2 = evict first (read
                                once per pass, so the counters, spill lists and tables keep L2);
                                0 = default (2) */
  uint32_t prefetch_tiles;   /* corpus tiles of a sequence prefetched into L2 ahead of their copies
                                to shared memory: value - 1 tiles (1 = none, up to 9); 0 = default
                                (none) */
  uint32_t spill_dedupe;     /* Eq. 2 dedupe of the slots a sequence spilled from its shared-memory
                                set: 2 = counting-sort into buckets by 32-slot word (interleaved),
                                then one bit vector per bucket in the set's shared memory; 1 = hash
                                partition (one or two levels) and a hash set per bucket; 0 = default
                                (2) */
  uint32_t spill_min_fill;   /* with spill_dedupe 2: a sequence's spills take the bit-vector path
                                when they fill each of its buckets with at least value - 1 entries
                                on average (fewer: the hash path); 0 = default (512) */
  uint32_t carry_slots;      /* rank/select passes after the first read each window's slot of the
                                previous pass from a per-symbol array (one lookup instead of one per
                                level; 4 bytes per corpus symbol): 2 = on, 1 or 0 (default) = off */
  uint32_t set_max_windows;  /* Eq. 2: a sequence with more windows than this sends every survivor
                                straight to its spill list, skipping the shared-memory set (0 =
                                default: never) */
  uint32_t scan_variants;    /* byte-corpus scans under Eq. 2 with the set and spill lists and 16-bit
                                counters (the base pass; candidate passes with rank/select prefixes
                                over one or two levels, or with the probe table) run compiled variants
                                with the other configurations' switches fixed at compile time: 2 = on,
                                1 = off (every scan runs the general kernel), 0 = default (on) */
} ig_tuning;

typedef struct ig_plan ig_plan;

/*
 * intergrams_plan - validate the inputs and build a plan for one corpus: the
 * problem of Sec. 2 - m sequences s_1..s_m over an alphabet, a length n and a
 * count k - with the frequency of Eq. 2 (count_mode 0: once per sequence
 * containing the n-gram) or Eq. 1 (count_mode 1: every occurrence), solved by
 * the passes of Algorithm 3 (Sec. 7) from a dense pass of Algorithm 2 (Sec. 6)
 * over base_n-grams; Z = candidates plays the paper's zk. The trailing
 * `tuning` argument is this library's own (the knobs only change speed and
 * memory, never the result).
 *   p        : parameters (copied).
 *   data     : the concatenated sequences (device pointer; host pointer with
 *              IG_F_HOST_INPUT). Bytes for symbol_bits 8; packed bases for 2.
 *              Caller-owned; must stay valid and unchanged until
 *              intergrams_free unless IG_F_HOST_INPUT is set.
 *   offsets  : uint64[m + 1] sequence boundaries in symbols; offsets[0] = 0,
 *              non-decreasing; offsets[m] = total symbols. Same ownership
 *              rules as data. Sequence i is symbols [offsets[i], offsets[i+1]).
 *   m        : number of sequences (0 is allowed: every result is empty).
 *   stream   : cudaStream_t the plan's work is ordered on (NULL = legacy default).
 *   tuning   : optional knobs (NULL = defaults).
 *   out      : receives the plan. The plan owns every table it allocates.
 * Reads offsets to the host once (one small D2H copy) to schedule work.
 * Errors: IG_EINVAL (bad parameters or offsets), IG_ENOMEM, IG_ECUDA.
 */
ig_status intergrams_plan(const ig_params* p, const void* data, const uint64_t* offsets,
                          uint32_t m, void* stream, const ig_tuning* tuning, ig_plan** out);

/*
 * intergrams_autotune - pick the tuning knobs for a job by timing a few
 * candidate settings on a prefix of the sequences of about sample_bytes
 * (0 = 256 MiB); every candidate must return byte-identical results (else
 * IG_ESTATE). Arguments as for intergrams_plan; out receives the fastest
 * knobs, best_ms (optional) their job time on the sample, or 0 when the
 * knobs came from the cache without timing anything. Choices are cached per
 * (device name and SM count, alphabet, n, base_n, candidate-count bucket,
 * count mode, corpus-size bucket) in the process and in a text file, so a
 * later process skips the sample runs: INTERGRAMS_TUNE_CACHE if set (empty
 * or "none": no file), else $XDG_CACHE_HOME/intergrams/autotune.txt or
 * $HOME/.cache/intergrams/autotune.txt (a file that cannot be read or
 * written is ignored). intergrams_plan with IG_F_AUTOTUNE calls this for
 * the knobs left at 0. Synchronises the stream.
 */
ig_status intergrams_autotune(const ig_params* p, const void* data, const uint64_t* offsets, uint32_t m,
                              void* stream, uint64_t sample_bytes, ig_tuning* out, float* best_ms);

/*
 * intergrams_pass - run the next pass (the dense base pass first, then the
 * candidate passes j = base_n+1 .. n, paper Algorithm 3) and its selection.
 *   j_done : receives the n-gram length j of the pass just run.
 * Returns IG_OK, or IG_DONE (nothing run) once pass n has completed.
 * Synchronises the plan's stream once to read the device status word.
 */
ig_status intergrams_pass(ig_plan* pl, uint32_t* j_done);

/*
 * intergrams_run - run every remaining pass (equivalent to calling
 * intergrams_pass until it returns IG_DONE, with one status read at the end).
 */
ig_status intergrams_run(ig_plan* pl);

/*
 * intergrams_rewind - return the plan to its state before the first pass so
 * the whole job can run again over the same corpus buffers (whose contents
 * may have changed, as long as the offsets did not). Tables are reused; with
 * IG_F_GRAPH a graph captured by intergrams_run is replayed. With
 * IG_F_HOST_INPUT the host data buffer given to intergrams_plan (which must
 * still be valid) is copied to the device again, so the rerun sees its
 * current contents. Stream-ordered, no synchronisation.
 */
ig_status intergrams_rewind(ig_plan* pl);

/*
 * intergrams_prefetch - with IG_F_HOST_INPUT: start copying the next run's
 * corpus (same offsets and size) from `host_data` (NULL = the buffer given to
 * intergrams_plan) into a second device buffer of the plan, on a copy stream
 * of its own, so the copy overlaps the passes still queued on the current
 * buffer (no counterpart in the paper: input pipelining for repeated jobs).
 * The next intergrams_rewind switches to that buffer, and the work queued
 * after it waits for the copy, instead of copying again. The copy first
 * waits for the work that read the buffer it overwrites. host_data must stay
 * valid and unchanged until that next run has finished. The second buffer
 * (the corpus size) is allocated at the first call and kept until
 * intergrams_free; with IG_F_GRAPH each buffer gets its own captured graph.
 * Errors: IG_EINVAL (NULL plan), IG_ESTATE (plan without IG_F_HOST_INPUT, or
 * a prefetch already pending), IG_ENOMEM, IG_ECUDA.
 */
ig_status intergrams_prefetch(ig_plan* pl, const void* host_data);

/* ---------------------------------------------------------------- sharding
 * A corpus split into groups of whole sequences - across processes, or one
 * group per GPU - is counted pass by pass as the sum of the groups' counts:
 * sequences are independent under Eq. 1 and Eq. 2 (Sec. 2; a window never
 * crosses a sequence boundary, and under Eq. 2 each sequence adds one per
 * distinct n-gram). Each shard makes its plan over its own sequences with
 * IG_F_SHARDED and the same params and layout knobs (dense_prefix, rs_depth,
 * chain_from), then, for every pass:
 *   intergrams_pass_scan     - the pass's corpus scan over this shard;
 *   intergrams_counts_export - this shard's counts into a caller buffer;
 *   (the caller sums the buffers over all shards: e.g. one all-reduce)
 *   intergrams_counts_import - the summed counts back into the plan;
 *   intergrams_pass_select   - the pass's selection (Algorithm 3's top-Z,
 *                              or the top-k after pass n) on the sums.
 * Every shard then holds the same P^(j) (the selection is deterministic), so
 * nothing else is exchanged; intergrams_topk gives the whole corpus's rows
 * on every shard. A survivor list that runs out of room in a sharded pass is
 * not grown and replayed (every shard would have to replay with it):
 * intergrams_pass_select returns IG_ETABLE_FULL; give such plans a list_pct
 * that holds the passes' candidates. Calls are stream-ordered on the plan's stream; the export
 * is complete once the stream has reached it, and the import must be
 * enqueued after the caller's reduction has written the buffer (synchronise
 * or order the streams). No counterpart in the paper, which runs on one
 * machine; the partition follows from its Eq. 1/Eq. 2.
 */

/*
 * intergrams_pass_scan - the corpus scan of the next pass, without its
 * selection. j_out receives the pass's j. IG_DONE when every pass has run.
 * Errors: IG_ESTATE (a scan is already pending; a plan made with IG_F_GRAPH
 * or IG_F_DRY_RUN).
 */
ig_status intergrams_pass_scan(ig_plan* pl, uint32_t* j_out);

/*
 * intergrams_counts_export - the pending pass's counts into d_counts (DEVICE
 * buffer of `capacity` uint32, stream-ordered): one count per slot of the
 * pass, in the plan's slot order (identical on every shard). n_out receives
 * the number of slots (also when the call fails for a small buffer).
 * Errors: IG_ESTATE (no scan pending), IG_EINVAL (NULL, capacity < slots).
 */
ig_status intergrams_counts_export(ig_plan* pl, uint32_t* d_counts, uint64_t capacity, uint64_t* n_out);

/*
 * intergrams_counts_import - replace the pending pass's counts with d_counts
 * (DEVICE, n uint32 = the pass's slots, e.g. the sum over the shards;
 * stream-ordered). Errors: IG_ESTATE (no scan pending), IG_EINVAL (NULL, n
 * differs from the pass's slots).
 */
ig_status intergrams_counts_import(ig_plan* pl, const uint32_t* d_counts, uint64_t n);

/*
 * intergrams_pass_select - the pending pass's selection on its current
 * counts (Algorithm 3: P^(j) = top-Z, or the final top-k after pass n).
 * j_done receives the pass's j. Synchronises once to read the device status
 * word (errors as intergrams_pass). Errors: IG_ESTATE (no scan pending).
 */
ig_status intergrams_pass_select(ig_plan* pl, uint32_t* j_done);

/*
 * intergrams_shard_assign - split m sequences (HOST offsets, m + 1 entries,
 * in symbols) into nshards groups of about equal total length, greedily by
 * bytes: longest sequence first, each to the group with the fewest symbols
 * so far (ties to the lower index). shard_of[i] receives sequence i's group;
 * shard_symbols (optional, nshards entries) each group's total. Host only.
 * Errors: IG_EINVAL (NULL, nshards == 0, decreasing offsets).
 */
ig_status intergrams_shard_assign(const uint64_t* offsets, uint32_t m, uint32_t nshards, uint32_t* shard_of,
                                  uint64_t* shard_symbols);

/*
 * intergrams_topk - the top-k j-grams of the latest completed pass j (paper
 * Algorithm 3, final k-argmax; after pass j < n this is the top-k of that
 * intermediate pass).
 *   keys_out   : HOST buffer of capacity * ceil(j * symbol_bits / 8) bytes; row r is
 *                the r-th n-gram, symbols in order, packed like the input
 *                (2-bit symbols most significant first, zero padded). May be NULL.
 *   counts_out : HOST buffer of capacity uint64 counts. May be NULL.
 *   capacity   : rows the buffers hold; min(k, capacity, #nonzero) rows are written.
 *   k_out      : receives the number of rows written.
 *   j_out      : optional; receives j (the length of each returned n-gram).
 * Rows are ordered by count descending, then symbols ascending.
 * Errors: IG_ESTATE if no pass has run yet.
 */
ig_status intergrams_topk(ig_plan* pl, uint8_t* keys_out, uint64_t* counts_out,
                          uint32_t capacity, uint32_t* k_out, uint32_t* j_out);

/*
 * intergrams_features - the Boolean sequence x feature matrix the top-k
 * n-grams are selected for (paper Sec. 1, Fig. 1): entry (i, f) is 1 exactly
 * when sequence i contains the n-gram of row f of intergrams_topk after the
 * last pass (Eq. 2 presence; the column sums are therefore the Eq. 2 counts
 * of the rows). Runs two more scans of the corpus (a counting scan, then a
 * writing scan) on the plan's stream and synchronises it.
 *   row_ptr  : HOST uint64[m + 1], CSR row starts (row_ptr[0] = 0), or NULL.
 *   cols     : HOST uint32[capacity], the feature ids of each row, ascending
 *              and distinct, or NULL.
 *   capacity : entries cols holds.
 *   nnz_out  : receives the number of nonzeros (set whenever the matrix was
 *              counted, also when capacity is too small).
 * With both buffers NULL only nnz is computed; the count is kept until
 * intergrams_rewind, so a second call with buffers sized nnz does not count
 * again. Requires every pass to have run (IG_ESTATE otherwise), n * symbol_bits
 * <= 64 and at most 2^20 rows (IG_EINVAL); capacity < nnz with cols given is
 * IG_EINVAL (nothing written). Device scratch is allocated by the call and
 * released by intergrams_free.
 */
ig_status intergrams_features(ig_plan* pl, uint64_t* row_ptr, uint32_t* cols, uint64_t capacity,
                              uint64_t* nnz_out);

/* Device bytes the plan allocated (or would allocate, for a plan made with IG_F_DRY_RUN). */
ig_status intergrams_plan_device_bytes(const ig_plan* pl, uint64_t* bytes);

/* Per-pass statistics of the latest pass (device counters, read on demand). */
typedef struct {
  uint32_t j;               /* n-gram length of the pass */
  uint64_t windows;         /* windows in the corpus for this j */
  uint64_t survivors;       /* windows whose (j-1)-prefix was a candidate (all, for the base pass) */
  uint64_t registrations;   /* count increments issued (Eq. 2: distinct (sequence, j-gram) pairs) */
  uint64_t nonzero_selected;/* size of the selected set (<= Z, or <= k at the last pass) */
  uint64_t scanned_bytes;   /* bytes of corpus streamed by the scan */
} ig_pass_stats;

ig_status intergrams_stats(ig_plan* pl, ig_pass_stats* out);

/*
 * intergrams_timings - device times of the latest run, from CUDA events
 * recorded on the plan's stream (requires IG_F_TIMING; synchronises).
 *   scan_ms / pass_ms : arrays of `cap` floats, or NULL: per pass, the scan
 *                       kernel's duration and the whole pass's duration
 *                       (reset, scan, selection, candidate build), in pass order.
 *   npasses           : receives the number of passes of the latest run.
 *   kernels           : optional; receives the number of kernels the latest
 *                       run launched (graph replays count their kernel nodes).
 */
ig_status intergrams_timings(ig_plan* pl, float* scan_ms, float* pass_ms, uint32_t cap,
                             uint32_t* npasses, uint32_t* kernels);

/*
 * intergrams_dense_topk_static - exact top-k n-grams of a short length n,
 * computed WITHOUT allocating anything (no counterpart in the paper).
 *
 * For callers that must not allocate device memory when they ask for an
 * answer: code inside a memory pool that owns the device budget, hot paths
 * with a no-allocation contract (allocation can synchronise the device or
 * fail under fragmentation), embedders that forbid cudaMalloc after start-up.
 * It runs the planned path's dense counting pass, selection and ordering
 * kernels with every table placed in one file-scope device array of 40 MiB
 * that the library holds on each GPU that loads it, until the process exits.
 *
 *   p            : n, k, symbol_bits and count_mode are used (candidates,
 *                  base_n and flags are ignored). Limits of the fixed scratch:
 *                  sigma^n <= 65536 (n <= 2 bytes or n <= 8 bases), k <= 65536,
 *                  m <= 2^20 sequences; anything larger returns IG_EINVAL.
 *   data, offsets: DEVICE inputs, as for intergrams_plan (offsets has m + 1
 *                  entries; total_symbols = offsets[m], given by the caller).
 *   stream       : cudaStream_t the work is ordered on (not synchronised).
 *   keys_out     : DEVICE buffer of k * ceil(n * symbol_bits / 8) bytes.
 *   counts_out   : DEVICE buffer of k uint64 counts.
 *   rows_out     : DEVICE uint32: number of rows written (min(k, #nonzero)),
 *                  0 when status_out reports a failure.
 *   status_out   : DEVICE int32, written stream-ordered at the end of the
 *                  call's work: IG_OK, or the failure the device reported -
 *                  IG_ETIMEOUT (a bounded wait for a corpus tile ran out;
 *                  the counts are incomplete) or IG_ETABLE_FULL (a dedupe
 *                  set filled up). On a failure rows_out is 0 and the
 *                  rows in keys_out/counts_out must be ignored. The return
 *                  value only covers what the host can see when the work is
 *                  queued (arguments, launch errors): read status_out after
 *                  the stream has reached it.
 * Rows are in the same order and format as intergrams_topk after a run with
 * n = base_n. Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors returned at once: IG_EINVAL (NULL pointer, sizes beyond the limits
 * above, Eq. 1 on 2^32 - 1 or more symbols, whose counts the 32-bit scratch
 * counters cannot hold), IG_ECUDA (a launch or runtime call failed).
 *
 * Every call looks up the scratch array's device address on the current
 * device (cudaGetSymbolAddress; the first lookup on a device loads the
 * library's module there): make the first call on each device before any
 * stream capture. Every call reuses the same array, which keeps the previous
 * call's contents (the call clears what must start at zero, and the dedupe
 * epochs carry over), so calls whose work overlaps on the GPU - from two
 * streams or two threads - race and give wrong results: serialise them.
 */
ig_status intergrams_dense_topk_static(const ig_params* p, const void* data, const uint64_t* offsets,
                                       uint32_t m, uint64_t total_symbols, void* stream,
                                       uint8_t* keys_out, uint64_t* counts_out, uint32_t* rows_out,
                                       int32_t* status_out);

/* ------------------------------------------------------------------ serving
 * A server runs many top-k jobs on one GPU with continuous batching: a
 * scheduler thread admits submitted jobs in arrival order whenever a slot is
 * free and the job's tables fit the device-memory budget, keeps each admitted
 * job's plan (its candidate and count tables) resident on its own stream, and
 * advances every active job one pass at a time, so jobs at different passes
 * have work on the GPU together. A job's result is the same as when it runs
 * alone (each job owns its tables; kernels are deterministic). max_active = 1
 * gives one job per launch, in order. No counterpart in the paper, which runs
 * one job at a time. */
typedef struct ig_server ig_server;
typedef struct {
  uint64_t mem_budget;   /* device bytes all active jobs' tables may use (0 = 80% of free memory) */
  uint32_t max_active;   /* jobs in flight at once (0 = 8) */
  uint32_t flags;        /* IG_SRV_* */
  uint64_t large_work;   /* IG_SRV_LARGE_ALONE: a job is large from this many bytes streamed over
                            all its passes (0 = 2e9, about 15 ms of scans on a GB300) */
} ig_server_config;
/* Server policy flags. Default (0): admit the pending job with the least
 * estimated work first (corpus bytes x passes plus its counter arrays; the
 * estimate halves for every 100 ms a job has waited, so none starves), on a
 * CUDA stream whose priority falls with the job's work (three classes:
 * below 1 GB, below 8 GB, more), so a small job's pass is started before a
 * large job's next pass. IG_SRV_FIFO: arrival order, default priority. */
#define IG_SRV_FIFO (1u << 0)
/* IG_SRV_OLDEST_FIRST: arrival order, and each job's stream one priority
 * level below the jobs already running when it was admitted, so the oldest
 * job's passes start first and younger jobs fill the gaps it leaves. */
#define IG_SRV_OLDEST_FIRST (1u << 1)
/* IG_SRV_LARGE_ALONE: a job whose estimated work is at least large_work
 * bytes streamed (default 2 GB) is admitted only when no other job is
 * running and runs with none beside it, so the largest jobs keep the whole
 * GPU (a scan holds its SMs for a whole pass and is not preempted); smaller
 * jobs still run together. Combines with the admission orders above. */
#define IG_SRV_LARGE_ALONE (1u << 2)
typedef struct {
  uint64_t submitted, completed, failed;
  uint32_t active, peak_active, pending;
  uint64_t mem_used, peak_mem, mem_budget;
} ig_server_stats;

/* Start a server on the current device (its scheduler thread uses that device). */
ig_status intergrams_server_create(const ig_server_config* cfg, ig_server** out);

/* Queue a job. data: DEVICE corpus (caller-owned, valid until the job is
 * waited for); offsets: HOST uint64[m + 1] (copied). The job's device bytes
 * are sized at once (a dry-run plan); IG_ENOMEM if they exceed the budget. */
ig_status intergrams_server_submit(ig_server* sv, const ig_params* p, const void* data, const uint64_t* offsets,
                                   uint32_t m, const ig_tuning* tuning, uint64_t* job_id);

/* Wait for a job (timeout_us < 0: no limit; IG_ETIMEOUT when it expires),
 * copy its top-k (format of intergrams_topk after the last pass) into HOST
 * buffers and release it. latency_s: submit-to-completion time. Returns the
 * job's status. */
ig_status intergrams_server_wait(ig_server* sv, uint64_t job_id, int64_t timeout_us, uint8_t* keys_out,
                                 uint64_t* counts_out, uint32_t capacity, uint32_t* k_out, double* latency_s);

ig_status intergrams_server_stats(ig_server* sv, ig_server_stats* out);

/* Finish every queued job, stop the scheduler and free the server. */
void intergrams_server_destroy(ig_server* sv);

/* Release every resource of the plan (stream-ordered frees). NULL is ignored.
 * No counterpart in the paper (resource management of this library). */
void intergrams_free(ig_plan* pl);

/* Message describing the last error on the calling thread ("" if none). No
 * counterpart in the paper (error reporting of this library: no exception
 * crosses the ABI, every call returns an ig_status). */
const char* intergrams_last_error(void);

/*
 * Test hooks: failures made on the host, for testing the error paths (no
 * counterpart in the paper; nothing here faults, traps or hangs a device).
 *
 * intergrams_test_fail_alloc - the nth device allocation the library makes
 * from now on (any plan, any thread) fails as if the device were out of
 * memory, so the call making it returns IG_ENOMEM; nth = 0 disarms.
 *   live_out : optional; receives the number of device allocations the
 *              library currently holds (all plans), so a test can check that
 *              a failed call released everything it had allocated.
 * Always returns IG_OK.
 */
ig_status intergrams_test_fail_alloc(uint32_t nth, uint64_t* live_out);

/*
 * intergrams_test_stall_tiles - every later corpus scan of `pl` waits for
 * shared-memory tiles whose copies are never issued: each scan CTA's bounded
 * wait (about one second) runs out, the CTA stops, and the pass returns
 * IG_ETIMEOUT (the scan's results are then incomplete; free the plan). The
 * device and other plans stay usable. Chain passes stage no tiles and are
 * unaffected. With pl = NULL the hook arms the next call of
 * intergrams_dense_topk_static instead (once): its scan stalls the same way
 * and the call reports IG_ETIMEOUT through its status_out word.
 * Errors: IG_ESTATE (plan made with IG_F_GRAPH, whose captured launches the
 * hook cannot reach).
 */
ig_status intergrams_test_stall_tiles(ig_plan* pl);

#ifdef __cplusplus
}
#endif

#endif /* INTERGRAMS_H */
