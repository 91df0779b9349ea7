// Internal declarations shared by the sm_103a translation units of the
// top-k n-gram library. Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "intergrams.h"

namespace ig {

constexpr uint32_t kEmpty32 = 0xFFFFFFFFu;
constexpr int kHistBins = 4096;      // bins of one threshold-search level
constexpr int kMaxLevels = 4;        // threshold-search levels (4096^k >= 2^32 at k = 3; one spare)
constexpr int kSortDigits = 256;     // 8-bit digits of the final stable sort
constexpr int kSortChunk = 1024;     // elements per one-warp block of the stable sort
constexpr uint32_t kRunChunk = 2048; // survivors are listed in runs of at most this many candidates
constexpr uint32_t kMaxRuns = 64;    // runs per tile (tile windows <= 65536 / ... / kRunChunk)
// registration log: a CTA holds one open chunk per counter range and, before
// a step that registers at most chunk / 8 slots, makes room for that many in
// each
constexpr uint32_t kLogMaxRanges = 32;
constexpr uint32_t kMaxRsLevels = 4;     // rank/select levels (candidate passes base + 1 .. base + 4)
constexpr uint32_t kNoChunk = 0xFFFFFFFEu;  // range has no open chunk yet (kEmpty32: pool exhausted)

// Sticky device status bits (PassCtl::status).
enum : uint32_t {
  kStSetFull = 1u << 0,        // a per-sequence dedupe set filled up
  kStTableFull = 1u << 1,      // the candidate probe table had no empty slot
  kStCountOverflow = 1u << 2,  // a 32-bit count wrapped (Eq. 1 only)
  kStQueue = 1u << 3,          // work queue inconsistency
  kStListFull = 1u << 4,       // a survivor list ran out of its capacity
  kStTimeout = 1u << 5,        // a bounded wait for a tile's bulk copy ran out
  kStCheck = 1u << 6,          // an exhaustive check failed (IG_F_EXHAUSTIVE_CHECKS)
};

// Device-side control block, one per plan. The pass fields are zeroed at the
// start of each pass by a kernel, so a captured graph can replay a pass.
struct PassCtl {
  uint32_t queue;                    // next sequence to scan
  uint32_t status;                   // sticky kStXxx bits (never cleared)
  unsigned long long survivors;      // windows whose prefix was a candidate
  unsigned long long registrations;  // count increments issued
  // selection state
  uint32_t target;                   // how many entries to keep (Z or k)
  uint32_t max_count;
  uint32_t nonzero;
  uint32_t lo, hi;                   // threshold search range (inclusive)
  uint32_t above;                    // entries with count > hi
  uint32_t done;                     // threshold found
  uint32_t thr;                      // selected: count > thr, plus the first need_eq with count == thr
  uint32_t need_eq;
  uint32_t nsel;                     // number selected
  uint32_t take_all;                 // nonzero <= target: keep every nonzero entry
  // Eq. 2 dedupe epochs: sequence s of the current pass uses epoch_base + s + 1
  uint32_t epoch_base;
  uint32_t epoch_next;
  uint32_t gset_clear;               // epochs wrapped: clear the dedupe sets before the scan
  uint32_t rlog_next;                // registration-log chunks handed out in this pass
  unsigned long long list_used;      // entries reserved in this pass's survivor list
  unsigned long long list_need;      // largest reservation end any pass asked for (sticky)
};

struct ScanArgs {
  const uint8_t* data;
  uint64_t data_bytes;
  const uint64_t* offsets;
  const uint32_t* order;       // sequences in scheduling order (longest first)
  uint32_t m;
  uint32_t j;                  // window length in symbols
  uint64_t key_mask;           // low j*symbol_bits bits
  const uint4* table;          // candidate probe table {key lo, key hi, id, 0}; null for the base pass
  uint32_t table_log2;
  uint32_t* counts;            // dense count table, indexed by slot
  unsigned long long* gset;    // per-CTA global dedupe sets, (epoch << 32 | slot); null = spill lists
  uint32_t gset_log2;          // log2 entries of each CTA's set
  uint32_t* spill;             // per-CTA spill list + partition buffer (2 * spill_cap words each)
  uint64_t spill_cap;          // >= windows of the longest sequence
  uint32_t spill_extra_log2;   // extra spill buckets (raised when a bucket overflowed)
  uint32_t count_mode;
  uint32_t words_per_thread;   // 32-bit smem words of symbols per thread per tile
  uint32_t sset_log2;          // log2 entries of the shared-memory dedupe set
  uint32_t tile_words;         // 32-bit words in the shared-memory tile buffer
  uint32_t queue_words;        // 32-bit words of the candidate queue (2 bytes per tile window) + survivor bits
  uint32_t check_overflow;     // Eq. 1 with >= 2^32 windows: detect count wrap
  uint32_t narrow;             // 16-bit counters (two per word): every count is known to be < 65536
  // survivor bitmasks (bit p: the window starting at corpus symbol p survived)
  const uint32_t* alive_in;    // previous pass's survivors; null = every window is a candidate
  uint32_t* alive_out;         // this pass's survivors; null = not needed
  // shared-memory cache of the most frequent candidates {key lo, key hi, id, count}
  const uint4* hot;
  uint32_t hot_log2;           // 0 = no cache
  // survivor lists (chain mode): tile g (tile_base[seq] + window / tile windows)
  // has runs_per_tile runs of entries (slot << 32 | window index in the
  // sequence); run r of tile g is at off[g * runs + r], cnt[g * runs + r] entries
  const uint32_t* tile_base;   // m + 1 entries
  uint32_t tile_windows;
  const unsigned long long* list_in;       // previous pass's list (chain passes)
  const unsigned long long* list_in_off;
  const uint32_t* list_in_cnt;
  unsigned long long* list_out;            // this pass's list (null = not written)
  unsigned long long* list_out_off;
  uint32_t* list_out_cnt;
  unsigned long long list_cap;
  uint32_t runs_per_tile;
  // registration log (counter arrays far larger than L2): a registered slot is
  // appended to the CTA's open chunk for its counter range (slot >> range_shift)
  // and counted later, one range at a time, by launch_log_count; null = count
  // at once. A CTA that finds the pool exhausted counts at once.
  uint32_t* rlog;              // rlog_chunks chunks of 2^rlog_chunk_log2 slots
  uint32_t* rlog_range;        // counter range of each handed-out chunk
  uint32_t* rlog_fill;         // slots in each handed-out chunk
  uint32_t rlog_chunks;
  uint32_t rlog_chunk_log2;
  uint32_t range_shift;
  uint32_t nranges;            // <= kLogMaxRanges
  // Eq. 2 dedupe by bit vector (small slot spaces): CTA b owns bits
  // [b * bitmap_words * 32, ...) of `bitmap`, one bit per slot, cleared at
  // the start of each of its sequences; null = shared-memory set + spills
  uint32_t* bitmap;
  uint32_t bitmap_words;
  // first candidate pass (j = base + 1, j * symbol_bits <= 32): counter row of
  // every base-length prefix, kEmpty32 = not a candidate; null = probe table
  const uint32_t* dmap;
  uint32_t first_runs;         // pass base + 1 in per-thread window runs (no queue; no survivor lists)
  // candidate passes base + 1 .. base + rs_depth by rank/select: level L is
  // the bit vector over pass base + L's slots of the selected ones, each
  // 32-bit word beside the number of selected slots in earlier words; a
  // prefix's byte-order id follows level by level (0 = the probe table)
  const uint2* rs[kMaxRsLevels];
  uint32_t rs_depth;
  // carried slots of rank/select passes: carry[p] = the slot the window
  // starting at corpus symbol p got in the previous pass (read when carry_in:
  // one lookup, at the last level, instead of rs_depth), and the slot it
  // gets in this pass (written for survivors when carry_out)
  uint32_t* carry;
  uint32_t carry_in, carry_out;
  uint32_t base_len;
  uint32_t set_probes;         // bounded probe length of the shared-memory dedupe set (1..8)
  uint32_t tile2;              // word offset of the second tile buffer in dynamic smem (0 = one buffer)
  uint32_t stall_tiles;        // test hook: tile barriers are never armed, so tile waits run out
  uint32_t tile_evict_first;   // corpus tile copies carry an L2 evict-first policy
  uint32_t prefetch_tiles;     // tiles of the sequence prefetched into L2 ahead of the copies (0 = none)
  uint64_t nslots;             // slots (counters) of this pass
  uint32_t range_dedupe;       // Eq. 2 spill dedupe by word bucket and bit vector (else hash partition + set)
  uint32_t range_min_fill;     // ... for sequences whose spills fill each bucket with at least this many
  uint32_t set_max_windows;    // Eq. 2: sequences with more windows skip the shared-memory set (0 = never)
  uint32_t general_only;       // never launch a configuration's compiled variant
  PassCtl* ctl;
};

// Launchers (ig_scan.cu)
void launch_scan(const ScanArgs& a, uint32_t symbol_bits, bool base_pass, int grid, int threads,
                 size_t smem, cudaStream_t s);
// candidate pass driven by the previous pass's survivor lists
void launch_chain(const ScanArgs& a, uint32_t symbol_bits, int grid, int threads, size_t smem, cudaStream_t s);
int scan_max_ctas_per_sm(uint32_t symbol_bits, bool base_pass, int threads, size_t smem);
cudaError_t scan_set_smem_limit(uint32_t symbol_bits, bool base_pass, size_t smem);
cudaError_t chain_set_smem_limit(uint32_t symbol_bits, size_t smem);
// Raise (never lower) the scan kernel's dynamic shared-memory limit to `smem`.
cudaError_t scan_raise_smem_limit(uint32_t symbol_bits, bool base_pass, size_t smem);
// Boolean sequence x feature matrix (ig_features.cu)
size_t feature_smem_bytes(uint32_t nfeat, uint32_t tile_words);
cudaError_t feature_set_smem(uint32_t sb, size_t smem);
void launch_features(const uint8_t* data, uint64_t data_bytes, const uint64_t* offsets, const uint32_t* order,
                     uint32_t m, uint32_t n, uint32_t sb, const uint8_t* rows, uint32_t nrows, uint32_t row_bytes,
                     unsigned long long* keys, uint4* table, uint32_t table_log2, uint32_t* queue, uint32_t* status,
                     uint32_t* row_nnz, uint64_t* row_ptr, uint32_t* cols, bool count, int grid,
                     uint32_t words_per_thread, uint32_t tile_words, size_t smem, cudaStream_t s);

// Test hook of the allocation-free entry point (ig_noalloc.cu): its next
// call's scan waits for tiles that are never sent.
void arm_static_stall();

// Count the registration log of the pass just scanned: one launch per counter
// range, so the counters being incremented at any time span one range.
void launch_log_count(const ScanArgs& a, cudaStream_t s);

// Launchers (ig_select.cu)
void launch_pass_reset(PassCtl* ctl, uint32_t m, unsigned long long* gset, uint64_t gset_entries, cudaStream_t s);
// rank: null for the dense base pass; otherwise the counter of slot id*sigma+sym is
// at rank[id]*sigma+sym (candidate passes count in rank space)
// narrow: the counters are 16-bit (counter s is the s-th uint16_t)
void launch_select(const uint32_t* counts, bool narrow, const uint32_t* rank, uint32_t sb, uint64_t ns,
                   uint32_t target, PassCtl* ctl, uint32_t* hist /* kMaxLevels*kHistBins */,
                   uint32_t* blk /* 2*G */, int G, uint32_t* sel_slot, uint32_t* sel_count, cudaStream_t s);
// rank[order[x]] = x for the nsel selected candidates, rank[i] = i beyond
void launch_rank(const uint32_t* order, const PassCtl* ctl, uint32_t* rank, uint32_t n, cudaStream_t s);
// stable LSD radix sort of the selected entries by count, descending; key_bits
// 16 when every count is < 65536 (two digit passes), else 32 (four)
void launch_sort_by_count(const uint32_t* sel_count, PassCtl* ctl, uint32_t cap, uint32_t key_bits,
                          uint32_t* idx_a, uint32_t* idx_b, uint32_t* key_a, uint32_t* key_b,
                          uint32_t* hist /* kSortDigits * (ceil(cap/kSortChunk) + 1) */, cudaStream_t s);

// Launchers (ig_table.cu)
// keys_next[r] = key of selected slot r; ids are in byte order
void launch_build_keys(const uint32_t* sel_slot, const PassCtl* ctl, const unsigned long long* keys_prev,
                       bool from_base, uint32_t symbol_bits, unsigned long long* keys_next, cudaStream_t s);
// probe table: key -> rank[r] (the counter row the next scan uses)
void launch_build_table(const unsigned long long* keys, const uint32_t* rank, const PassCtl* ctl, uint4* table,
                        uint32_t table_log2, cudaStream_t s);
// rank/select words after the base pass: bit s of word s / 32 set for every
// selected base gram s, .y = number of selected grams in earlier words
void launch_build_pbits(const uint32_t* sel_slot, const PassCtl* ctl, uint2* pbits, uint32_t words,
                        uint32_t* block_sums /* ceil(words / 1024) + 1 */, cudaStream_t s);
// dense prefix map after the base pass: dmap[sel_slot[i]] = rank[i], the rest kEmpty32
void launch_build_dmap(const uint32_t* sel_slot, const PassCtl* ctl, const uint32_t* rank, uint32_t* dmap,
                       uint64_t entries, cudaStream_t s);
void launch_build_hot(const unsigned long long* keys, const uint32_t* sel_count, const uint32_t* rank,
                      const PassCtl* ctl, uint4* hot, unsigned long long* hot_pick, uint32_t hot_log2,
                      cudaStream_t s);
// rows of the top-k of pass j: symbols rebuilt by walking back through every
// pass's selection (sel_hist[(jj - b) * Z + id] = byte-order slot of P^(jj))
void launch_write_topk(const uint32_t* sel_hist, uint64_t Z, uint32_t b, const uint32_t* sel_count,
                       const uint32_t* order, const PassCtl* ctl, uint32_t symbol_bits, uint32_t j,
                       uint32_t row_bytes, uint32_t cap, uint8_t* keys_out, unsigned long long* counts_out,
                       cudaStream_t s);
// chain keys of P^(j): the scan slot of each selected j-gram (rank space of pass j)
void launch_chain_keys(const uint32_t* sel_slot, const PassCtl* ctl, const uint32_t* rank_prev, bool from_base,
                       uint32_t symbol_bits, unsigned long long* keys_out, cudaStream_t s);

// ------------------------------------------------------------- helpers

__host__ __device__ inline uint32_t ceil_log2_u64(uint64_t x) {
  uint32_t l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

// Multiply-shift hashing (Dietzfelbinger, Hagerup, Katajainen, Penttonen,
// "A reliable randomized algorithm for the closest-pair problem", 1997):
// the top l bits of a*x mod 2^w for an odd multiplier a.
__device__ __forceinline__ uint32_t hash64_top(uint64_t x, uint32_t l) {
  return l == 0 ? 0u : (uint32_t)((x * 0x9E3779B97F4A7C15ull) >> (64 - l));
}
__device__ __forceinline__ uint32_t hash32_top(uint32_t x, uint32_t l) {
  return l == 0 ? 0u : (x * 0x9E3779B1u) >> (32 - l);
}

}  // namespace ig
