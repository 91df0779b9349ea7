// C ABI of the top-k n-gram library: plan / pass / run / topk / stats / free.
//
// A plan owns every device table of one job. Pass j (paper Algorithm 3):
//   reset queue + epochs -> zero the slot counters -> scan the corpus ->
//   select top-Z (top-k at the last pass) -> if j < n, build P^(j).
// All sizes the kernels need are kept on the device, so the launch sequence
// of a pass is fixed; with IG_F_GRAPH the whole remaining pass sequence is
// captured once as a CUDA graph and replayed by later runs of the same plan.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "ig_internal.cuh"
#include <nvtx3/nvToolsExt.h>

using namespace ig;

namespace {

thread_local std::string g_last_error;

// NVTX range around an API call (a no-op unless a profiler is attached), so
// a profile can be filtered by call and pass, e.g. `ncu --nvtx
// --nvtx-include "ig pass 4/"`.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

ig_status fail(ig_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

#define IG_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? IG_ENOMEM : IG_ECUDA,                      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    }                                                                                          \
  } while (0)

}  // namespace

namespace ig {
// Lets other translation units record a message for intergrams_last_error().
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ig

namespace {

// Every device allocation of the library goes through these two, so a test
// can make the n-th allocation fail (host-side fault injection) and check
// that nothing stays allocated after a failed call.
std::atomic<uint32_t> g_fail_alloc_in{0};  // the allocation this many from now fails (0 = none)
std::atomic<int64_t> g_live_allocs{0};

cudaError_t device_malloc(void** p, size_t bytes, bool async, cudaStream_t s) {
  *p = nullptr;
  uint32_t n = g_fail_alloc_in.load();
  while (n && !g_fail_alloc_in.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) return cudaErrorMemoryAllocation;
  const cudaError_t e = async ? cudaMallocAsync(p, bytes, s) : cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

void device_free(void* q, bool async, cudaStream_t s) {
  if (!q) return;
  if (async) cudaFreeAsync(q, s);
  else cudaFree(q);
  g_live_allocs.fetch_sub(1);
}

}  // namespace

struct ig_plan {
  ig_params p{};
  ig_tuning t{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;

  const uint8_t* data = nullptr;
  uint64_t data_bytes = 0;
  const uint64_t* offsets = nullptr;
  uint32_t m = 0;
  uint8_t* own_data = nullptr;
  uint64_t* own_offsets = nullptr;
  std::vector<uint64_t> h_offsets;
  uint64_t total_syms = 0, max_len = 0;

  uint32_t sigma = 256, sb = 8;
  uint32_t b = 3;          // length of the first (dense) pass
  uint32_t next_j = 0;     // next pass to run
  uint32_t last_j = 0;     // last completed pass (0 = none)
  uint32_t nsel_last = 0;  // size of the latest selection

  uint64_t nslots_base = 0, nslots_cand = 0;
  uint32_t* counts = nullptr;
  uint4* table = nullptr;
  uint32_t table_log2 = 0;
  unsigned long long* keys[2] = {nullptr, nullptr};
  int cur = 0;             // keys[cur] = keys of the latest candidate set
  uint32_t* sel_hist = nullptr;      // selection of every pass j (byte-order slots), Z per pass
  uint32_t* sel_count = nullptr;
  uint32_t* rank = nullptr;          // rank of each candidate id (counter row of the next scan)
  uint32_t* hist = nullptr;
  uint32_t* blk = nullptr;
  int G = 1024;
  uint32_t *sidx[2] = {nullptr, nullptr}, *skey[2] = {nullptr, nullptr}, *shist = nullptr;
  uint32_t sort_cap = 0;
  uint32_t* alive[2] = {nullptr, nullptr};  // survivor bitmasks, ping-pong by pass parity
  uint64_t alive_words = 0;
  uint4* hot = nullptr;                      // hot cache of the latest candidate set
  unsigned long long* hot_pick = nullptr;
  uint32_t hot_log2 = 0;
  uint32_t* spill = nullptr;         // Eq. 2: per scan CTA, spill list + partition buffer
  uint64_t spill_cap = 0;
  // chain mode: per-tile survivor lists, ping-pong by pass parity
  uint32_t chain_from = 0;           // first pass run from survivor lists
  uint32_t tile_windows = 0;
  uint32_t* d_tile_base = nullptr;   // m + 1
  uint32_t ntiles = 0;
  uint32_t runs_per_tile = 1;
  unsigned long long* lists[2] = {nullptr, nullptr};
  unsigned long long* list_off[2] = {nullptr, nullptr};
  uint32_t* list_cnt[2] = {nullptr, nullptr};
  uint64_t list_cap = 0;
  PassCtl* ctl = nullptr;
  PassCtl* h_ctl = nullptr;  // pinned mirror for status reads
  uint32_t* d_order = nullptr;

  int scan_grid = 0, scan_threads = 512;
  size_t scan_smem = 0;
  uint32_t tile_words = 0;
  // the dense base pass's own tile and set (no queue, no hot cache)
  uint32_t base_wpt = 0, base_sset_log2 = 0, base_tile_words = 0;
  size_t base_smem = 0;
  uint32_t tile2 = 0, base_tile2 = 0;  // word offsets of the second tile buffers (0 = one buffer)
  uint32_t queue_words = 0;

  uint8_t* out_keys = nullptr;
  unsigned long long* out_counts = nullptr;
  uint32_t out_cap = 0;

  const void* host_data = nullptr;   // IG_F_HOST_INPUT: re-read by intergrams_rewind
  // intergrams_prefetch: a second device copy of the corpus, filled on a copy
  // stream while the passes on the current one run; rewind switches to it
  uint8_t* own_data_alt = nullptr;
  uint32_t data_slot = 0;            // 0: own_data is current, 1: own_data_alt
  bool prefetched = false;           // a copy into the other slot is pending
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied = nullptr;   // the pending copy has landed
  cudaEvent_t ev_left[2] = {nullptr, nullptr};  // the work reading slot s was all queued before this
  cudaGraphExec_t graph_alt = nullptr;  // the job's graph over own_data_alt
  // IG_F_TIMING: events around each pass and its scan, indexed by j - b
  std::vector<cudaEvent_t> ev_pass0, ev_pass1, ev_scan0, ev_scan1;
  uint32_t kernels = 0;              // kernels launched since the last rewind
  uint32_t graph_kernels = 0;        // kernels in the captured graph
  uint64_t dev_bytes = 0;            // device bytes allocated (or that would be, with IG_F_DRY_RUN)
  bool dry_run = false, async_alloc = false;
  uint32_t test_stall_tiles = 0;  // test hook: scans wait for tiles that are never sent
  cudaGraphExec_t graph = nullptr;  // full job from the first pass (IG_F_GRAPH)
  cudaStream_t cap_stream = nullptr; // private stream the graph is captured on
  bool check_overflow = false;
  bool narrow = false;               // 16-bit counters (every count provably < 65536)
  uint32_t pending_j = 0;            // sharded pass: scan of pass pending_j done, selection not yet
  bool broken = false;               // the survivor lists could not grow: no further passes
  bool imported = false;             // the pending pass's counts were replaced by intergrams_counts_import
  // IG_F_EXHAUSTIVE_CHECKS: the previous pass's selected counts by counter
  // row of this pass, and the sum of this pass's counters
  uint32_t* prev_count = nullptr;
  unsigned long long* check_sum = nullptr;
  // registration log of the candidate passes (counter arrays far larger than L2)
  uint32_t* rlog = nullptr;
  uint32_t* rlog_range = nullptr;
  uint32_t* rlog_fill = nullptr;
  uint32_t rlog_chunks = 0, rlog_chunk_log2 = 0, range_shift = 0, nranges = 0;
  // Eq. 2 dedupe bit vectors (one per scan CTA) for passes with at most bitmap_bits slots
  uint32_t* bitmap = nullptr;
  uint64_t bitmap_bits = 0;
  // dense prefix map of the first candidate pass (sigma^b rows)
  uint32_t* dmap = nullptr;
  // rank/select levels: level L covers pass b + L's slots (sigma^b for L = 0,
  // sigma * Z above) and serves candidate passes b + L + 1 .. b + rs_levels
  uint2* rs[kMaxRsLevels] = {};
  uint32_t rs_words[kMaxRsLevels] = {};
  uint32_t* rs_sums = nullptr;
  uint32_t rs_levels = 0;
  uint32_t* carry = nullptr;         // carried slots between rank/select passes (one per corpus symbol)
  // feature matrix scratch (intergrams_features), kept until free; the count
  // stays valid until rewind
  unsigned long long* feat_keys = nullptr;
  uint4* feat_table = nullptr;
  uint32_t* feat_q = nullptr;  // two queue counters + status
  uint32_t* feat_nnz = nullptr;
  uint64_t* feat_rowptr = nullptr;
  uint32_t feat_table_log2 = 0, feat_rows = 0;
  bool feat_ready = false;
  uint64_t feat_total = 0;
};

namespace {

// The scan kernels' dynamic shared-memory limits belong to the kernels, so
// every plan of the process shares them: each plan sets them to the largest
// size any plan has needed (per alphabet width and kernel group), never
// lowering them under a live plan made with larger tiles or sets.
cudaError_t set_shared_limits(uint32_t sb, size_t base_smem, size_t scan_smem) {
  static std::mutex mu;
  static size_t most[2][2] = {{0, 0}, {0, 0}};  // [sb == 8][base pass, candidate and chain passes]
  std::lock_guard<std::mutex> lock(mu);
  size_t* m = most[sb == 8 ? 1 : 0];
  m[0] = std::max(m[0], base_smem);
  m[1] = std::max(m[1], scan_smem);
  cudaError_t e = scan_set_smem_limit(sb, true, m[0]);
  if (e == cudaSuccess) e = scan_set_smem_limit(sb, false, m[1]);
  if (e == cudaSuccess) e = chain_set_smem_limit(sb, m[1]);
  return e;
}

// Every device allocation of a plan goes through here: counted, skipped in a
// dry run, stream-ordered with IG_F_ASYNC_ALLOC.
template <class T>
cudaError_t dev_alloc(ig_plan* pl, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
  pl->dev_bytes += bytes;
  if (pl->dry_run) return cudaSuccess;
  return device_malloc(reinterpret_cast<void**>(p), bytes, pl->async_alloc, pl->stream);
}

uint32_t row_bytes_for(const ig_plan* pl, uint32_t j) { return (j * pl->sb + 7) / 8; }

uint64_t windows_for(const ig_plan* pl, uint32_t j) {
  uint64_t w = 0;
  for (uint32_t i = 0; i < pl->m; ++i) {
    uint64_t L = pl->h_offsets[i + 1] - pl->h_offsets[i];
    if (L >= j) w += L - j + 1;
  }
  return w;
}

void release(ig_plan* pl) {
  if (!pl) return;
  if (pl->graph) cudaGraphExecDestroy(pl->graph);
  if (pl->graph_alt) cudaGraphExecDestroy(pl->graph_alt);
  // a prefetch copy may still be landing in a buffer freed below
  if (pl->copy_stream) cudaStreamSynchronize(pl->copy_stream);
  for (cudaEvent_t e : {pl->ev_copied, pl->ev_left[0], pl->ev_left[1]})
    if (e) cudaEventDestroy(e);
  if (pl->copy_stream) cudaStreamDestroy(pl->copy_stream);
  for (auto* v : {&pl->ev_pass0, &pl->ev_pass1, &pl->ev_scan0, &pl->ev_scan1})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  void* ptrs[] = {pl->own_data, pl->own_data_alt, pl->own_offsets, pl->counts, pl->table, pl->keys[0], pl->keys[1],
                  pl->sel_hist, pl->sel_count, pl->d_tile_base, pl->lists[0], pl->lists[1], pl->list_off[0],
                  pl->list_off[1], pl->list_cnt[0], pl->list_cnt[1], pl->hist, pl->blk, pl->sidx[0], pl->sidx[1], pl->skey[0],
                  pl->skey[1], pl->shist, pl->spill, pl->ctl, pl->d_order, pl->out_keys, pl->out_counts,
                  pl->alive[0], pl->alive[1], pl->hot, pl->hot_pick, pl->rank, pl->prev_count, pl->check_sum,
                  pl->rlog, pl->rlog_range, pl->rlog_fill, pl->bitmap, pl->dmap, pl->rs[0], pl->rs[1], pl->rs[2], pl->rs[3], pl->rs_sums, pl->carry, pl->feat_keys,
                  pl->feat_table, pl->feat_q, pl->feat_nnz, pl->feat_rowptr};
  for (void* q : ptrs) device_free(q, pl->async_alloc, pl->stream);
  if (pl->h_ctl) cudaFreeHost(pl->h_ctl);
  delete pl;
}

// Enqueue pass j (no host synchronisation).
// How pass j runs: the dense base pass; a scan of the corpus that probes each
// window's (j-1)-gram by key (keys of up to 64 bits); or a chain pass driven
// by the survivor lists of pass j-1 (any key length; work proportional to the
// survivors). Chain mode is monotone in j.
enum PassMode : uint32_t { kModeBase = 0, kModeShort = 1, kModeChain = 2, kModeNone = 3 };

uint32_t mode_of(const ig_plan* pl, uint32_t j) {
  if (j > pl->p.n) return kModeNone;
  if (j == pl->b) return kModeBase;
  if (j == pl->b + 1) return kModeShort;
  if ((j - 1) * pl->sb > 64 || j >= pl->chain_from) return kModeChain;
  return kModeShort;
}

// Pass j is the first candidate pass run in per-thread window runs (it is
// not followed by a chain pass, which needs survivor lists); with a dense
// prefix map it looks prefixes up there.
bool runs_pass(const ig_plan* pl, uint32_t j) {
  return (pl->dmap || pl->t.dense_prefix == 3) && j == pl->b + 1 && mode_of(pl, j) == kModeShort &&
         mode_of(pl, j + 1) != kModeChain;
}
bool dense_pass(const ig_plan* pl, uint32_t j) { return pl->dmap && runs_pass(pl, j); }
// Pass j looks its prefix up by rank/select through levels 0 .. j - b - 1
// (and counts in byte-order ids).
bool rs_pass(const ig_plan* pl, uint32_t j) {
  return pl->rs_levels && j > pl->b && j <= pl->b + pl->rs_levels && mode_of(pl, j) == kModeShort;
}

// Kernels of one sort by count: init + (histogram, two scans, scatter) per 8-bit digit.
uint32_t sort_kernels(const ig_plan* pl) { return 1 + 4 * (pl->narrow ? 2u : 4u); }

// IG_F_EXHAUSTIVE_CHECKS. Every counter of the pass: the sum over all of
// them (must equal the registrations: each one increments one counter by
// one), Eq. 2 counts at most `limit` = m, and - with the previous pass's
// counts by row - no j-gram above its (j-1)-prefix (a window of the j-gram
// is a window of the prefix; the prefix's count was exact).
__global__ void check_counts_kernel(const uint32_t* counts, bool narrow, uint64_t ns, uint32_t row_shift,
                                    const uint32_t* prev_count, uint32_t limit, unsigned long long* sum,
                                    PassCtl* ctl) {
  unsigned long long local = 0;
  bool bad = false;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < ns; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = narrow ? (counts[i >> 1] >> ((i & 1u) << 4)) & 0xFFFFu : counts[i];
    local += c;
    if (c > limit) bad = true;
    if (prev_count && c > prev_count[i >> row_shift]) bad = true;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31u) == 0 && local) atomicAdd(sum, local);
  if (bad) atomicOr(&ctl->status, kStCheck);
}

__global__ void check_sum_kernel(const unsigned long long* sum, PassCtl* ctl) {
  if (threadIdx.x == 0 && *sum != ctl->registrations) atomicOr(&ctl->status, kStCheck);
}

// The selected counts by the next pass's counter row: byte-order id (a
// rank/select pass) or rank by count.
__global__ void prev_count_kernel(const uint32_t* sel_count, const uint32_t* rank, const PassCtl* ctl,
                                  uint32_t* prev_count) {
  const uint32_t n = ctl->nsel;
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
    prev_count[rank ? rank[x] : x] = sel_count[x];
}

// Counters of pass j: narrow (16-bit) <-> the 32-bit exchange format.
__global__ void widen_counts_kernel(const uint32_t* packed, uint64_t ns, uint32_t* out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < ns; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (packed[i >> 1] >> ((i & 1u) << 4)) & 0xFFFFu;
}
__global__ void narrow_counts_kernel(const uint32_t* in, uint64_t ns, uint32_t* packed, PassCtl* ctl) {
  const uint64_t words = (ns + 1) / 2;
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t lo = in[2 * w], hi = 2 * w + 1 < ns ? in[2 * w + 1] : 0u;
    if ((lo | hi) > 0xFFFFu) atomicOr(&ctl->status, kStCountOverflow);
    packed[w] = (lo & 0xFFFFu) | (hi << 16);
  }
}

// Enqueue the scan half of pass j (reset, counters cleared, corpus scan);
// returns the kernels launched.
uint32_t enqueue_scan(ig_plan* pl, uint32_t j, cudaStream_t s) {
  const uint32_t md = mode_of(pl, j), md_next = mode_of(pl, j + 1);
  const bool base = (md == kModeBase);
  const bool timing = (pl->p.flags & IG_F_TIMING) != 0;
  const uint32_t ti = j - pl->b;
  const uint64_t ns = base ? pl->nslots_base : pl->nslots_cand;
  uint32_t* sel = pl->sel_hist + (uint64_t)(j - pl->b) * pl->p.candidates;
  uint32_t kernels = 0;
  // inside a stream capture an event record must be an explicit graph node
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (timing) cudaStreamIsCapturing(s, &cs);
  const unsigned evf = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (timing) cudaEventRecordWithFlags(pl->ev_pass0[ti], s, evf);
  const bool seq_mode = pl->p.count_mode == IG_COUNT_ONCE_PER_SEQUENCE;
  launch_pass_reset(pl->ctl, pl->m, nullptr, 0, s);
  kernels += 1;
  cudaMemsetAsync(pl->counts, 0, pl->narrow ? ((ns + 1) / 2) * sizeof(uint32_t) : ns * sizeof(uint32_t), s);
  ScanArgs a{};
  a.data = pl->data;
  a.data_bytes = pl->data_bytes;
  a.offsets = pl->offsets;
  a.order = pl->d_order;
  a.m = pl->m;
  a.j = j;
  a.key_mask = (j * pl->sb >= 64) ? ~0ull : ((1ull << (j * pl->sb)) - 1ull);
  a.table = base ? nullptr : pl->table;
  a.table_log2 = pl->table_log2;
  a.counts = pl->counts;
  a.gset = nullptr;
  a.gset_log2 = 0;
  a.spill = seq_mode ? pl->spill : nullptr;
  a.spill_cap = pl->spill_cap;
  a.spill_extra_log2 = 0;
  a.count_mode = pl->p.count_mode;
  a.words_per_thread = pl->t.words_per_thread;
  a.sset_log2 = pl->t.smem_set_log2;
  a.tile_words = pl->tile_words;
  a.queue_words = pl->queue_words;
  a.check_overflow = pl->check_overflow ? 1u : 0u;
  a.narrow = pl->narrow ? 1u : 0u;
  a.set_probes = pl->t.set_probes ? pl->t.set_probes : 1u;
  a.tile2 = pl->tile2;
  a.stall_tiles = pl->test_stall_tiles;
  a.tile_evict_first = pl->t.tile_cache_hint != 1u;
  a.prefetch_tiles = pl->t.prefetch_tiles ? pl->t.prefetch_tiles - 1u : 0u;
  a.nslots = ns;
  a.range_dedupe = pl->t.spill_dedupe != 1u;
  a.range_min_fill = pl->t.spill_min_fill ? pl->t.spill_min_fill - 1u : 512u;
  a.set_max_windows = pl->t.set_max_windows;
  a.general_only = pl->t.scan_variants == 1;
  if (base) {  // the base pass's own tile and set; no queue
    a.words_per_thread = pl->base_wpt;
    a.sset_log2 = pl->base_sset_log2;
    a.tile_words = pl->base_tile_words;
    a.queue_words = 0;
    a.tile2 = pl->base_tile2;
  }
  a.tile_base = pl->d_tile_base;
  a.tile_windows = pl->tile_windows;
  a.runs_per_tile = pl->runs_per_tile;
  // survivor bitmasks link consecutive scans; survivor lists feed chain passes
  a.alive_in = (md == kModeShort && j >= pl->b + 2 && mode_of(pl, j - 1) == kModeShort)
                   ? pl->alive[(j - 1) & 1u] : nullptr;
  a.alive_out = (md == kModeShort && md_next == kModeShort) ? pl->alive[j & 1u] : nullptr;
  if (a.alive_out) cudaMemsetAsync(a.alive_out, 0, pl->alive_words * sizeof(uint32_t), s);
  if (md_next == kModeChain) {
    a.list_out = pl->lists[j & 1u];
    a.list_out_off = pl->list_off[j & 1u];
    a.list_out_cnt = pl->list_cnt[j & 1u];
    a.list_cap = pl->list_cap;
    cudaMemsetAsync(a.list_out_cnt, 0, (size_t)pl->ntiles * pl->runs_per_tile * sizeof(uint32_t), s);
  }
  if (md == kModeChain) {
    a.list_in = pl->lists[(j - 1) & 1u];
    a.list_in_off = pl->list_off[(j - 1) & 1u];
    a.list_in_cnt = pl->list_cnt[(j - 1) & 1u];
  }
  a.hot = pl->hot;
  a.hot_log2 = (md == kModeShort) ? pl->hot_log2 : 0u;
  if (runs_pass(pl, j)) a.first_runs = 1;
  if (rs_pass(pl, j)) {
    for (uint32_t L = 0; L < j - pl->b; ++L) a.rs[L] = pl->rs[L];
    a.rs_depth = j - pl->b;
    a.base_len = pl->b;
    a.hot_log2 = 0;
    if (pl->carry) {  // in place: a window reads its previous slot, then writes its new one
      a.carry = pl->carry;
      a.carry_in = j >= pl->b + 2;
      a.carry_out = rs_pass(pl, j + 1);
    }
  }
  if (dense_pass(pl, j)) {
    a.dmap = pl->dmap;
    a.hot_log2 = 0;
  }
  if (!base && pl->rlog) {
    a.rlog = pl->rlog;
    a.rlog_range = pl->rlog_range;
    a.rlog_fill = pl->rlog_fill;
    a.rlog_chunks = pl->rlog_chunks;
    a.rlog_chunk_log2 = pl->rlog_chunk_log2;
    a.range_shift = pl->range_shift;
    a.nranges = pl->nranges;
  }
  if (seq_mode && pl->bitmap && ns <= pl->bitmap_bits) {
    a.bitmap = pl->bitmap;
    a.bitmap_words = (uint32_t)((ns + 31) / 32);
  }
  a.ctl = pl->ctl;
  if (timing) cudaEventRecordWithFlags(pl->ev_scan0[ti], s, evf);
  if (pl->m > 0) {
    if (md == kModeChain) launch_chain(a, pl->sb, pl->scan_grid, pl->scan_threads, pl->scan_smem, s);
    else launch_scan(a, pl->sb, base, pl->scan_grid, pl->scan_threads, base ? pl->base_smem : pl->scan_smem, s);
    kernels += 1;
    if (a.rlog) {
      launch_log_count(a, s);
      kernels += a.nranges;
    }
  }
  if (timing) cudaEventRecordWithFlags(pl->ev_scan1[ti], s, evf);
  return kernels;
}

// Enqueue the selection half of pass j (its top-T and, before pass j + 1,
// the candidate set P^(j)) on the counts the scan left; returns the kernels
// launched.
uint32_t enqueue_select(ig_plan* pl, uint32_t j, cudaStream_t s) {
  const uint32_t md = mode_of(pl, j), md_next = mode_of(pl, j + 1);
  const bool base = (md == kModeBase);
  const bool timing = (pl->p.flags & IG_F_TIMING) != 0;
  const uint32_t ti = j - pl->b;
  const uint64_t ns = base ? pl->nslots_base : pl->nslots_cand;
  uint32_t* sel = pl->sel_hist + (uint64_t)(j - pl->b) * pl->p.candidates;
  uint32_t kernels = 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (timing) cudaStreamIsCapturing(s, &cs);
  const unsigned evf = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (pl->check_sum) {
    cudaMemsetAsync(pl->check_sum, 0, sizeof(unsigned long long), s);
    // counts imported from a sum over shards may reach the whole corpus's m:
    // only the prefix check applies to them
    const uint32_t limit =
        (pl->p.count_mode == IG_COUNT_ONCE_PER_SEQUENCE && !pl->imported) ? pl->m : 0xFFFFFFFFu;
    check_counts_kernel<<<4 * 152, 256, 0, s>>>(pl->counts, pl->narrow, ns, pl->sb, base ? nullptr : pl->prev_count,
                                                limit, pl->check_sum, pl->ctl);
    kernels += 1;
    if (!pl->imported) {
      check_sum_kernel<<<1, 32, 0, s>>>(pl->check_sum, pl->ctl);
      kernels += 1;
    }
  }
  const uint32_t target = (j < pl->p.n) ? pl->p.candidates : pl->p.k;
  // the scan of a candidate pass counted in rank space; selection reads the
  // counters back in byte order through the rank map
  // (a rank/select pass counts in byte-order ids: no rank map)
  launch_select(pl->counts, pl->narrow, (base || rs_pass(pl, j)) ? nullptr : pl->rank, pl->sb, ns, target, pl->ctl,
                pl->hist, pl->blk, pl->G, sel, pl->sel_count, s);
  kernels += 12;
  if (j < pl->p.n) {
    const int nxt = pl->cur ^ 1;
    // P^(j): the next scan's keys (byte-order keys for a key probe, scan
    // slots for a chain pass), then ranks by (count desc, id asc) for the
    // next counters, then the probe table (key -> rank) and hot cache
    if (md_next == kModeShort)
      launch_build_keys(sel, pl->ctl, pl->keys[pl->cur], base, pl->sb, pl->keys[nxt], s);
    else
      launch_chain_keys(sel, pl->ctl, pl->rank, base || rs_pass(pl, j), pl->sb, pl->keys[nxt], s);
    launch_sort_by_count(pl->sel_count, pl->ctl, pl->sort_cap, pl->narrow ? 16u : 32u, pl->sidx[0], pl->sidx[1], pl->skey[0], pl->skey[1],
                         pl->shist, s);
    launch_rank(pl->sidx[0], pl->ctl, pl->rank, pl->p.candidates, s);
    kernels += 1 + sort_kernels(pl) + 2;
    if (dense_pass(pl, j + 1)) {
      launch_build_dmap(sel, pl->ctl, pl->rank, pl->dmap, pl->nslots_base, s);
      kernels += 1;
    } else if (rs_pass(pl, j + 1)) {  // level j - b from this pass's selection
      launch_build_pbits(sel, pl->ctl, pl->rs[j - pl->b], pl->rs_words[j - pl->b], pl->rs_sums, s);
      kernels += 5;
    } else {
      launch_build_table(pl->keys[nxt], pl->rank, pl->ctl, pl->table, pl->table_log2, s);
      kernels += 2;
    }
    if (pl->hot_log2 && md_next == kModeShort && !dense_pass(pl, j + 1) && !rs_pass(pl, j + 1)) {
      launch_build_hot(pl->keys[nxt], pl->sel_count, pl->rank, pl->ctl, pl->hot, pl->hot_pick, pl->hot_log2, s);
      kernels += 3;
    }
    if (pl->prev_count) {  // rows without a candidate keep 0: any count there fails the check
      cudaMemsetAsync(pl->prev_count, 0, sizeof(uint32_t) * pl->p.candidates, s);
      prev_count_kernel<<<256, 256, 0, s>>>(pl->sel_count, rs_pass(pl, j + 1) ? nullptr : pl->rank, pl->ctl,
                                            pl->prev_count);
      kernels += 1;
    }
  }
  if (timing) cudaEventRecordWithFlags(pl->ev_pass1[ti], s, evf);
  return kernels;
}

// Enqueue pass j (no host synchronisation); returns the kernels launched.
uint32_t enqueue_pass(ig_plan* pl, uint32_t j, cudaStream_t s) {
  const uint32_t k = enqueue_scan(pl, j, s);
  return k + enqueue_select(pl, j, s);
}


// After pass j has been enqueued: bookkeeping on the host.
void finish_pass_host(ig_plan* pl, uint32_t j) {
  if (j < pl->p.n) pl->cur ^= 1;
  pl->last_j = j;
  pl->next_j = j + 1;
}

ig_status read_status(ig_plan* pl) {
  IG_CUDA(cudaMemcpyAsync(pl->h_ctl, pl->ctl, sizeof(PassCtl), cudaMemcpyDeviceToHost, pl->stream));
  IG_CUDA(cudaStreamSynchronize(pl->stream));
  IG_CUDA(cudaGetLastError());
  const uint32_t st = pl->h_ctl->status;
  pl->nsel_last = pl->h_ctl->nsel;
  if (st & kStCountOverflow) return fail(IG_EOVERFLOW, "a 32-bit count overflowed");
  if (st & kStListFull) return fail(IG_ETABLE_FULL, "a survivor list exceeded its capacity (raise list_pct)");
  if (st & kStTimeout) return fail(IG_ETIMEOUT, "a tile's bulk copy did not complete");
  if (st & (kStSetFull | kStTableFull)) return fail(IG_ETABLE_FULL, "a device hash table filled up");
  if (st & kStCheck)
    return fail(IG_ESTATE, "an exhaustive check failed: counters do not sum to the registrations, an Eq. 2 count "
                           "exceeds m, or a j-gram's count exceeds its prefix's");
  if (st) return fail(IG_ECUDA, "device status error");
  return IG_OK;
}

// Did the last status read report a survivor list out of room, and nothing else?
bool list_full_only(const ig_plan* pl) { return pl->h_ctl->status == kStListFull; }

// A survivor list ran out of room: grow both lists to the largest
// reservation any pass asked for (plus a quarter), drop the captured graphs
// (they name the old buffers) and clear the status, so the job can be run
// again. IG_ETABLE_FULL when the device has no memory for the larger lists.
ig_status grow_lists(ig_plan* pl) {
  const uint64_t need = pl->h_ctl->list_need;
  const uint64_t cap = std::max<uint64_t>(need + need / 4 + 1, 2 * pl->list_cap);
  IG_CUDA(cudaStreamSynchronize(pl->stream));
  const size_t old_bytes = (pl->list_cap * sizeof(unsigned long long) + 255) & ~size_t(255);
  for (int q = 0; q < 2; ++q) {
    device_free(pl->lists[q], pl->async_alloc, pl->stream);
    pl->lists[q] = nullptr;
    pl->dev_bytes -= old_bytes;
  }
  for (int q = 0; q < 2; ++q)
    if (dev_alloc(pl, &pl->lists[q], cap) != cudaSuccess) {
      cudaGetLastError();
      pl->list_cap = 0;
      pl->broken = true;
      return fail(IG_ETABLE_FULL, "a survivor list exceeded its capacity and the device has no memory to grow it");
    }
  pl->list_cap = cap;
  for (cudaGraphExec_t* g : {&pl->graph, &pl->graph_alt})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  IG_CUDA(cudaMemsetAsync(&pl->ctl->status, 0, sizeof(uint32_t), pl->stream));
  IG_CUDA(cudaMemsetAsync(&pl->ctl->list_need, 0, sizeof(unsigned long long), pl->stream));
  return IG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Asynchronous plan steps for the serving engine (same library): nothing here
// synchronises; completion is signalled by the event each step records.
namespace ig {

bool plan_passes_done(const ig_plan* pl) { return pl->next_j > pl->p.n; }

uint32_t plan_row_bytes(const ig_plan* pl) { return row_bytes_for(pl, pl->p.n); }

// Enqueue the next pass, the read-back of its status word, and `ev`.
ig_status plan_enqueue_next(ig_plan* pl, cudaEvent_t ev) {
  const uint32_t j = pl->next_j;
  pl->kernels += enqueue_pass(pl, j, pl->stream);
  finish_pass_host(pl, j);
  IG_CUDA(cudaMemcpyAsync(pl->h_ctl, pl->ctl, sizeof(PassCtl), cudaMemcpyDeviceToHost, pl->stream));
  IG_CUDA(cudaEventRecord(ev, pl->stream));
  IG_CUDA(cudaGetLastError());
  return IG_OK;
}

// Status of the last enqueued pass; call once its event has completed.
ig_status plan_last_status(ig_plan* pl) {
  const uint32_t st = pl->h_ctl->status;
  pl->nsel_last = pl->h_ctl->nsel;
  if (st & kStCountOverflow) return fail(IG_EOVERFLOW, "a 32-bit count overflowed");
  if (st & kStListFull) return fail(IG_ETABLE_FULL, "a survivor list exceeded its capacity (raise list_pct)");
  if (st & kStTimeout) return fail(IG_ETIMEOUT, "a tile's bulk copy did not complete");
  if (st & (kStSetFull | kStTableFull)) return fail(IG_ETABLE_FULL, "a device hash table filled up");
  if (st & kStCheck)
    return fail(IG_ESTATE, "an exhaustive check failed: counters do not sum to the registrations, an Eq. 2 count "
                           "exceeds m, or a j-gram's count exceeds its prefix's");
  if (st) return fail(IG_ECUDA, "device status error");
  return IG_OK;
}

// After plan_last_status reported a survivor list out of room (and nothing
// else): grow the lists and rewind, so the job runs again from its first
// pass. False when that was not the failure or the lists could not grow.
bool plan_regrow_and_restart(ig_plan* pl) {
  if (!list_full_only(pl)) return false;
  if (grow_lists(pl) != IG_OK) return false;
  return intergrams_rewind(pl) == IG_OK;
}

// Enqueue the final top-k into PINNED host buffers, and `ev`; *rows is known
// at once (from the last status).
ig_status plan_enqueue_topk(ig_plan* pl, uint8_t* keys_host, uint64_t* counts_host, uint32_t cap, uint32_t* rows,
                            cudaEvent_t ev) {
  const uint32_t j = pl->last_j;
  const uint32_t r = std::min(std::min(pl->p.k, cap), pl->nsel_last);
  *rows = r;
  cudaStream_t s = pl->stream;
  if (r) {
    launch_sort_by_count(pl->sel_count, pl->ctl, pl->sort_cap, pl->narrow ? 16u : 32u, pl->sidx[0], pl->sidx[1], pl->skey[0], pl->skey[1],
                         pl->shist, s);
    const uint32_t rb = row_bytes_for(pl, j);
    launch_write_topk(pl->sel_hist, pl->p.candidates, pl->b, pl->sel_count, pl->sidx[0], pl->ctl, pl->sb, j, rb, r,
                      pl->out_keys, pl->out_counts, s);
    pl->kernels += sort_kernels(pl) + 1;
    IG_CUDA(cudaMemcpyAsync(keys_host, pl->out_keys, (size_t)r * rb, cudaMemcpyDeviceToHost, s));
    IG_CUDA(cudaMemcpyAsync(counts_host, pl->out_counts, (size_t)r * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  }
  IG_CUDA(cudaEventRecord(ev, s));
  IG_CUDA(cudaGetLastError());
  return IG_OK;
}

}  // namespace ig

extern "C" {

const char* intergrams_last_error(void) { return g_last_error.c_str(); }

ig_status intergrams_plan(const ig_params* p, const void* data, const uint64_t* offsets, uint32_t m, void* stream,
                          const ig_tuning* tuning, ig_plan** out) {
  g_last_error.clear();
  if (!out) return fail(IG_EINVAL, "out is NULL");
  Range range("ig plan");
  *out = nullptr;
  if (!p) return fail(IG_EINVAL, "params is NULL");
  if (p->symbol_bits != 8 && p->symbol_bits != 2) return fail(IG_EINVAL, "symbol_bits must be 8 or 2");
  if (p->n < 1 || p->n > 64) return fail(IG_EINVAL, "n must be in 1..64");
  if (p->k < 1) return fail(IG_EINVAL, "k must be >= 1");
  if (p->candidates < p->k || p->candidates >= (1u << 24)) return fail(IG_EINVAL, "need k <= candidates < 2^24");
  const uint32_t max_base = p->symbol_bits == 8 ? 3u : 12u;
  if (p->base_n < 1 || p->base_n > max_base) return fail(IG_EINVAL, "base_n out of range");
  if (p->count_mode > 1) return fail(IG_EINVAL, "count_mode must be 0 or 1");
  if (!offsets) return fail(IG_EINVAL, "offsets is NULL");

  // IG_F_AUTOTUNE: knobs left at 0 come from the autotuner (timed on a sample)
  ig_tuning tuned{};
  if ((p->flags & IG_F_AUTOTUNE) && !(p->flags & IG_F_DRY_RUN)) {
    ig_params ap = *p;
    ap.flags &= ~(IG_F_AUTOTUNE | IG_F_GRAPH | IG_F_TIMING);
    ig_tuning best{};
    const ig_status ast = intergrams_autotune(&ap, data, offsets, m, stream, 0, &best, nullptr);
    if (ast != IG_OK) return ast;
    tuned = tuning ? *tuning : ig_tuning{};
    uint32_t* dst = &tuned.ctas_per_sm;
    const uint32_t* src = &best.ctas_per_sm;
    for (size_t i = 0; i < sizeof(ig_tuning) / sizeof(uint32_t); ++i)
      if (dst[i] == 0) dst[i] = src[i];
    tuning = &tuned;
  }
  ig_plan* pl = new (std::nothrow) ig_plan();
  if (!pl) return fail(IG_ENOMEM, "host allocation failed");
  pl->p = *p;
  pl->stream = reinterpret_cast<cudaStream_t>(stream);
  pl->m = m;
  pl->sb = p->symbol_bits;
  pl->sigma = 1u << pl->sb;
  pl->b = std::min(p->base_n, p->n);
  pl->next_j = pl->b;
  pl->dry_run = (p->flags & IG_F_DRY_RUN) != 0;
  pl->async_alloc = (p->flags & IG_F_ASYNC_ALLOC) != 0;

  auto bail = [&](ig_status st) {
    release(pl);
    return st;
  };
#define PLAN_CUDA(call)                                                                              \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return bail(fail(e_ == cudaErrorMemoryAllocation ? IG_ENOMEM : IG_ECUDA,                       \
                       std::string(#call) + ": " + cudaGetErrorString(e_)));                        \
  } while (0)

  PLAN_CUDA(cudaGetDevice(&pl->device));
  PLAN_CUDA(cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, pl->device));

  // offsets on the host
  pl->h_offsets.resize((size_t)m + 1);
  if (p->flags & (IG_F_HOST_INPUT | IG_F_OFFSETS_HOST)) {
    std::memcpy(pl->h_offsets.data(), offsets, sizeof(uint64_t) * ((size_t)m + 1));
  } else {
    PLAN_CUDA(cudaMemcpyAsync(pl->h_offsets.data(), offsets, sizeof(uint64_t) * ((size_t)m + 1),
                              cudaMemcpyDeviceToHost, pl->stream));
    PLAN_CUDA(cudaStreamSynchronize(pl->stream));
  }
  if (pl->h_offsets[0] != 0) return bail(fail(IG_EINVAL, "offsets[0] must be 0"));
  for (uint32_t i = 0; i < m; ++i) {
    if (pl->h_offsets[i + 1] < pl->h_offsets[i]) return bail(fail(IG_EINVAL, "offsets must be non-decreasing"));
    pl->max_len = std::max(pl->max_len, pl->h_offsets[i + 1] - pl->h_offsets[i]);
  }
  pl->total_syms = pl->h_offsets[m];
  pl->data_bytes = (pl->total_syms * pl->sb + 7) / 8;
  if (pl->data_bytes && !data) return bail(fail(IG_EINVAL, "data is NULL"));

  if (p->flags & (IG_F_HOST_INPUT | IG_F_OFFSETS_HOST)) {
    if (p->flags & IG_F_HOST_INPUT) {
      PLAN_CUDA(dev_alloc(pl, &pl->own_data, pl->data_bytes));
      if (pl->data_bytes && !pl->dry_run)
        PLAN_CUDA(cudaMemcpyAsync(pl->own_data, data, pl->data_bytes, cudaMemcpyHostToDevice, pl->stream));
      pl->data = pl->own_data;
      pl->host_data = data;
    } else {
      pl->data = reinterpret_cast<const uint8_t*>(data);
    }
    PLAN_CUDA(dev_alloc(pl, &pl->own_offsets, (size_t)m + 1));
    if (!pl->dry_run)
      PLAN_CUDA(cudaMemcpyAsync(pl->own_offsets, pl->h_offsets.data(), sizeof(uint64_t) * ((size_t)m + 1),
                                cudaMemcpyHostToDevice, pl->stream));
    pl->offsets = pl->own_offsets;
  } else {
    pl->data = reinterpret_cast<const uint8_t*>(data);
    pl->offsets = offsets;
  }

  // tuning (defaults; the autotuner in the binding may override)
  ig_tuning t{};
  if (tuning) t = *tuning;
  const bool auto_set = (t.smem_set_log2 == 0);
  if (!t.ctas_per_sm) t.ctas_per_sm = 1;
  if (!t.threads) t.threads = 1024;
  if (!t.words_per_thread) t.words_per_thread = p->symbol_bits == 8 ? 5 : 3;
  if (!t.smem_set_log2) t.smem_set_log2 = 15;
  if (!t.table_load_pct) t.table_load_pct = 25;
  if (!t.hot_log2) t.hot_log2 = 11;
  const bool auto_list = (t.list_pct == 0);
  if (!t.list_pct) t.list_pct = 25;
  if (t.ctas_per_sm > 4 || (t.threads != 256 && t.threads != 512 && t.threads != 1024) ||
      !(t.words_per_thread & 1u) || t.words_per_thread > 31 || t.smem_set_log2 < 8 || t.smem_set_log2 > 15 ||
      t.table_load_pct < 10 || t.table_load_pct > 50 || t.hot_log2 < 6 || t.hot_log2 > 13 || t.list_pct > 200 ||
      t.log_mode > 1 || t.dedupe_bitmap > 2 || t.tile_cache_hint > 2 || t.prefetch_tiles > 9 || t.spill_dedupe > 2 || t.carry_slots > 2 || t.scan_variants > 2 || t.set_probes > 8 || t.tile_buffers > 2 || t.dense_prefix > 4 || t.rs_depth > kMaxRsLevels || t.log_pct > 400 || (t.log_chunk_log2 && (t.log_chunk_log2 < 14 || t.log_chunk_log2 > 20)) ||
      (t.log_range_log2 && (t.log_range_log2 < 10 || t.log_range_log2 > 30)))
    return bail(fail(IG_EINVAL, "tuning knob out of range"));
  pl->t = t;

  // sizes
  uint64_t nb = 1;
  for (uint32_t i = 0; i < pl->b; ++i) nb *= pl->sigma;
  pl->nslots_base = nb;
  pl->nslots_cand = (pl->b < p->n) ? (uint64_t)pl->sigma * p->candidates : 0;
  const uint64_t nslots = std::max(pl->nslots_base, pl->nslots_cand);
  pl->table_log2 = ceil_log2_u64((uint64_t)p->candidates * 100 / t.table_load_pct + 1);
  if (pl->table_log2 < 4) pl->table_log2 = 4;
  pl->sort_cap = p->candidates;
  const uint32_t sortG = (pl->sort_cap + kSortChunk - 1) / kSortChunk;

  // Eq. 1 with 2^32 or more windows can overflow a 32-bit count
  pl->check_overflow = p->count_mode == IG_COUNT_EVERY_OCCURRENCE && pl->total_syms >= 0xFFFFFFFFull;
  // 16-bit counters when no count can reach 65536: Eq. 2 counts are at most m,
  // Eq. 1 counts at most the number of windows (halves the counter array, so
  // far more of it stays in L2)
  pl->narrow = (p->count_mode == IG_COUNT_ONCE_PER_SEQUENCE) ? (m < 65536u) : (pl->total_syms < 65536u);
  if (p->flags & IG_F_SHARDED) pl->narrow = false;  // shards agree on one counter layout

  // scan launch geometry: shared memory = dedupe set + hot cache + tile (with
  // halo and alignment slop) + candidate queue (2 bytes per tile window) +
  // the tile's survivor bits. Tiles are capped at 65536 windows (16-bit
  // queue entries).
  const uint32_t spw = 32 / pl->sb;
  if ((uint64_t)t.words_per_thread * spw * t.threads > 65536)
    return bail(fail(IG_EINVAL, "tile too large: threads * words_per_thread * symbols per word must be <= 65536"));
  pl->hot_log2 = (pl->b < p->n) ? t.hot_log2 : 0u;
  const uint64_t tile_windows = (uint64_t)t.words_per_thread * spw * t.threads;
  const uint64_t tile_syms = tile_windows + p->n + 2 * 16 * (8 / pl->sb);
  pl->tile_words = (uint32_t)((tile_syms * pl->sb + 31) / 32) + 8;
  pl->tile_words = (pl->tile_words + 3) & ~3u;
  pl->queue_words = (uint32_t)(((tile_windows + 1) / 2 + 3) & ~3ull);
  const uint32_t alive_tile_words = (uint32_t)((tile_windows + 31) / 32);
  auto smem_for = [&](uint32_t set_log2) {
    return ((size_t)4 << set_log2) + (size_t)12 * (pl->hot_log2 ? (1u << pl->hot_log2) : 0u) +
           (size_t)4 * (pl->tile_words + pl->queue_words + ((alive_tile_words + 3) & ~3u));
  };
  int max_optin = 0;
  PLAN_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device));
  while (auto_set && t.smem_set_log2 > 8 && smem_for(t.smem_set_log2) + 256 > (size_t)max_optin) --t.smem_set_log2;
  if (smem_for(t.smem_set_log2) + 256 > (size_t)max_optin)
    return bail(fail(IG_EINVAL, "tuning needs more shared memory than a CTA can have"));
  pl->t = t;
  pl->scan_threads = (int)t.threads;
  pl->scan_smem = smem_for(t.smem_set_log2);
  // the base pass: its own words per thread and set size; shared memory =
  // set + tile only
  pl->base_wpt = t.base_words_per_thread ? t.base_words_per_thread : t.words_per_thread;
  pl->base_sset_log2 = t.base_smem_set_log2 ? t.base_smem_set_log2 : t.smem_set_log2;
  if (!(pl->base_wpt & 1u) || pl->base_wpt > 31 || pl->base_sset_log2 < 8 || pl->base_sset_log2 > 15 ||
      (uint64_t)pl->base_wpt * spw * t.threads > 65536)
    return bail(fail(IG_EINVAL, "base-pass tuning knob out of range"));
  {
    const uint64_t bw = (uint64_t)pl->base_wpt * spw * t.threads;
    pl->base_tile_words = (uint32_t)((((bw + p->n + 2 * 16 * (8 / pl->sb)) * pl->sb + 31) / 32 + 8 + 3) & ~3ull);
    pl->base_smem = ((size_t)4 << pl->base_sset_log2) + (size_t)4 * pl->base_tile_words;
    if (pl->base_smem + 256 > (size_t)max_optin)
      return bail(fail(IG_EINVAL, "base-pass tuning needs more shared memory than a CTA can have"));
  }
  // second tile buffers, where they fit (with room for the kernels' static
  // shared memory)
  if (t.tile_buffers != 1) {
    if (pl->scan_smem + (size_t)4 * pl->tile_words + 2048 <= (size_t)max_optin) {
      pl->tile2 = (uint32_t)(pl->scan_smem / 4);
      pl->scan_smem += (size_t)4 * pl->tile_words;
    }
    if (pl->base_smem + (size_t)4 * pl->base_tile_words + 2048 <= (size_t)max_optin) {
      pl->base_tile2 = (uint32_t)(pl->base_smem / 4);
      pl->base_smem += (size_t)4 * pl->base_tile_words;
    }
  }
  PLAN_CUDA(set_shared_limits(pl->sb, pl->base_smem, pl->scan_smem));
  pl->tile_windows = (uint32_t)tile_windows;
  pl->runs_per_tile = (uint32_t)((tile_windows + kRunChunk - 1) / kRunChunk);
  int occ = std::min(scan_max_ctas_per_sm(pl->sb, false, pl->scan_threads, pl->scan_smem),
                     scan_max_ctas_per_sm(pl->sb, true, pl->scan_threads, pl->base_smem));
  if (occ < 1) return bail(fail(IG_EINVAL, "scan kernel does not fit on an SM with these tuning knobs"));
  pl->scan_grid = pl->sms * (int)std::min<uint32_t>(t.ctas_per_sm, (uint32_t)occ);

  // Eq. 2 spill buffers: per scan CTA a list and a partition buffer, each
  // holding every window of the longest sequence
  if (p->count_mode == IG_COUNT_ONCE_PER_SEQUENCE) pl->spill_cap = std::max<uint64_t>(pl->max_len, 1);

  // chain passes: from pass chain_from on (and whenever a (j-1)-gram key
  // exceeds 64 bits) a pass runs from the previous pass's survivor lists
  // default: the last two passes of a byte job with enough passes run from
  // survivor lists (few windows survive there: measured 24.1 -> 18.1 and
  // 15.9 -> 9.2 ms for passes 7 and 8 of the 8.8 GB malware-like job)
  pl->chain_from = t.chain_from ? t.chain_from
                                : ((pl->sb == 8 && p->n >= pl->b + 4) ? p->n - 1 : p->n + 1);
  bool any_chain = false;
  for (uint32_t j = pl->b; j <= p->n; ++j) any_chain = any_chain || mode_of(pl, j) == kModeChain;
  std::vector<uint32_t> tile_base((size_t)m + 1, 0);
  for (uint32_t i = 0; i < m; ++i) {
    const uint64_t L = pl->h_offsets[i + 1] - pl->h_offsets[i];
    const uint64_t nt = (L + tile_windows - 1) / tile_windows;
    if ((uint64_t)tile_base[i] + nt > 0xFFFFFFFFull) return bail(fail(IG_EINVAL, "too many tiles"));
    tile_base[i + 1] = tile_base[i] + (uint32_t)nt;
  }
  pl->ntiles = tile_base[m];

  PLAN_CUDA(dev_alloc(pl, &pl->counts, pl->narrow ? (nslots + 1) / 2 : nslots));
  pl->alive_words = (pl->total_syms + 31) / 32 + 1;
  if (p->n >= pl->b + 2) {
    PLAN_CUDA(dev_alloc(pl, &pl->alive[0], pl->alive_words));
    PLAN_CUDA(dev_alloc(pl, &pl->alive[1], pl->alive_words));
  }
  if (pl->hot_log2) {
    PLAN_CUDA(dev_alloc(pl, &pl->hot, (size_t)1 << pl->hot_log2));
    PLAN_CUDA(dev_alloc(pl, &pl->hot_pick, (size_t)1 << pl->hot_log2));
  }
  PLAN_CUDA(dev_alloc(pl, &pl->table, (size_t)1 << pl->table_log2));
  PLAN_CUDA(dev_alloc(pl, &pl->keys[0], p->candidates));
  PLAN_CUDA(dev_alloc(pl, &pl->keys[1], p->candidates));
  PLAN_CUDA(dev_alloc(pl, &pl->sel_hist, (size_t)(p->n - pl->b + 1) * p->candidates));
  PLAN_CUDA(dev_alloc(pl, &pl->sel_count, p->candidates));
  PLAN_CUDA(dev_alloc(pl, &pl->rank, p->candidates));
  if (p->flags & IG_F_EXHAUSTIVE_CHECKS) {
    PLAN_CUDA(dev_alloc(pl, &pl->prev_count, p->candidates));
    PLAN_CUDA(dev_alloc(pl, &pl->check_sum, 1));
  }
  PLAN_CUDA(dev_alloc(pl, &pl->hist, (size_t)kMaxLevels * kHistBins));
  PLAN_CUDA(dev_alloc(pl, &pl->blk, (size_t)2 * pl->G));
  PLAN_CUDA(dev_alloc(pl, &pl->sidx[0], pl->sort_cap));
  PLAN_CUDA(dev_alloc(pl, &pl->sidx[1], pl->sort_cap));
  PLAN_CUDA(dev_alloc(pl, &pl->skey[0], pl->sort_cap));
  PLAN_CUDA(dev_alloc(pl, &pl->skey[1], pl->sort_cap));
  PLAN_CUDA(dev_alloc(pl, &pl->shist, (size_t)kSortDigits * (sortG + 1)));
  if (pl->spill_cap) PLAN_CUDA(dev_alloc(pl, &pl->spill, (size_t)pl->scan_grid * 2 * pl->spill_cap));
  PLAN_CUDA(dev_alloc(pl, &pl->d_tile_base, (size_t)m + 1));
  if (!pl->dry_run)
    PLAN_CUDA(cudaMemcpyAsync(pl->d_tile_base, tile_base.data(), sizeof(uint32_t) * ((size_t)m + 1),
                              cudaMemcpyHostToDevice, pl->stream));
  if (any_chain) {
    // default capacity: every window when two such lists use at most 25% of the
    // free device memory, else list_pct (25%) of the windows
    uint64_t list_pct = t.list_pct;
    if (auto_list) {
      size_t free_b = 0, total_b = 0;
      PLAN_CUDA(cudaMemGetInfo(&free_b, &total_b));
      if ((long double)2 * 8 * pl->total_syms <= 0.25L * free_b) list_pct = 100;
    }
    pl->list_cap = std::max<uint64_t>(1u << 16, pl->total_syms * list_pct / 100);
    for (int q = 0; q < 2; ++q) {
      PLAN_CUDA(dev_alloc(pl, &pl->lists[q], pl->list_cap));
      PLAN_CUDA(dev_alloc(pl, &pl->list_off[q], std::max<size_t>((size_t)pl->ntiles * pl->runs_per_tile, 1)));
      PLAN_CUDA(dev_alloc(pl, &pl->list_cnt[q], std::max<size_t>((size_t)pl->ntiles * pl->runs_per_tile, 1)));
    }
  }
  // registration log: when the candidate passes' counter array is far larger
  // than L2, registrations are logged per counter range (16 MiB of counters)
  // and counted range by range after the scan, so the random increments hit
  // L2 instead of HBM. Capacity: log_pct of the corpus symbols (60% under
  // Eq. 2, 80% under Eq. 1), plus the room lost when chunks are closed early
  // and, by default, the chunks held open; at most a quarter of the device
  // memory. A pass that needs more counts the rest at once. Off by default:
  // it halves the scan's DRAM traffic on the 8.8 GB malware-like workload but
  // not its time (the scan is bound by instruction issue there).
  if (pl->nslots_cand && t.log_mode == 1) {
    const uint32_t cl = t.log_chunk_log2 ? t.log_chunk_log2 : 18u;
    uint32_t rl = t.log_range_log2 ? t.log_range_log2 : (pl->narrow ? 23u : 22u);
    while (((pl->nslots_cand + (1ull << rl) - 1) >> rl) > kLogMaxRanges) ++rl;
    const uint32_t nr = (uint32_t)((pl->nslots_cand + (1ull << rl) - 1) >> rl);
    const uint64_t open = (uint64_t)pl->scan_grid * nr;
    const uint64_t pct = t.log_pct ? t.log_pct : (p->count_mode == IG_COUNT_ONCE_PER_SEQUENCE ? 60u : 80u);
    const uint64_t est = pl->total_syms * pct / 100u;
    {
      size_t free_b = 0, total_b = 0;
      PLAN_CUDA(cudaMemGetInfo(&free_b, &total_b));
      uint64_t chunks = (est + est / 7 + (1ull << cl) - 1) >> cl;
      if (!t.log_pct) chunks += 2 * open;
      chunks = std::max<uint64_t>(chunks, 1);
      chunks = std::min<uint64_t>(chunks, std::max<uint64_t>(1, (uint64_t)total_b / 4 / (4ull << cl)));
      chunks = std::min<uint64_t>(chunks, 0xFFFFFF00ull);
      pl->range_shift = rl;
      pl->nranges = nr;
      pl->rlog_chunks = (uint32_t)chunks;
      pl->rlog_chunk_log2 = cl;
      PLAN_CUDA(dev_alloc(pl, &pl->rlog, chunks << cl));
      PLAN_CUDA(dev_alloc(pl, &pl->rlog_range, chunks));
      PLAN_CUDA(dev_alloc(pl, &pl->rlog_fill, chunks));
    }
  }
  // dense prefix map for pass b + 1 when it and the counter array fit in L2
  // together (else the probe table with its hot cache wins: measured)
  {
    const uint64_t cbytes = pl->nslots_cand * (pl->narrow ? 2u : 4u), mbytes = pl->nslots_base * 4u;
    const bool want = t.dense_prefix == 2 || (t.dense_prefix == 0 && cbytes + mbytes <= (112ull << 20));
    const bool first_ok = pl->b < p->n && mode_of(pl, pl->b + 1) == kModeShort && mode_of(pl, pl->b + 2) != kModeChain;
    if (want && first_ok) {
      PLAN_CUDA(dev_alloc(pl, &pl->dmap, pl->nslots_base));
    } else if ((t.dense_prefix == 0 || t.dense_prefix == 4) && pl->b < p->n && pl->nslots_base <= (1ull << 24) &&
               pl->nslots_cand <= (1ull << 35)) {
      // rank/select for the first rs_depth candidate passes that are key-probe passes
      const uint32_t want_levels = std::min<uint32_t>(t.rs_depth ? t.rs_depth : 2u, kMaxRsLevels);
      uint32_t lv = 0;
      while (lv < want_levels && pl->b + lv + 1 <= p->n && mode_of(pl, pl->b + lv + 1) == kModeShort) ++lv;
      pl->rs_levels = lv;
      uint32_t maxw = 1;
      for (uint32_t L = 0; L < lv; ++L) {
        pl->rs_words[L] = (uint32_t)(((L == 0 ? pl->nslots_base : pl->nslots_cand) + 31) / 32);
        maxw = std::max(maxw, pl->rs_words[L]);
        PLAN_CUDA(dev_alloc(pl, &pl->rs[L], pl->rs_words[L]));
      }
      if (lv) PLAN_CUDA(dev_alloc(pl, &pl->rs_sums, (maxw + 1023) / 1024 + 1));
      // carried slots (opt-in): with two or more rank/select passes, each one
      // after the first reads the window's slot from the pass before and
      // makes one lookup instead of one per level (4 bytes per corpus
      // symbol). Off by default: the rank/select words stay in L2, so the
      // saved lookups cost less than writing the array (malware-like 8.8 GB
      // job: pass 4 +5.2 ms, pass 5 -2.4 ms)
      if (lv >= 2 && t.carry_slots == 2) PLAN_CUDA(dev_alloc(pl, &pl->carry, std::max<uint64_t>(pl->total_syms, 1)));
    }
  }
  // Eq. 2 bit vectors: a pass whose slot space is small dedupes each sequence
  // with one bit per slot (atomicOr; the bit vectors of all scan CTAs stay
  // in L2) instead of the shared-memory set and its spill lists
  if (p->count_mode == IG_COUNT_ONCE_PER_SEQUENCE && t.dedupe_bitmap != 1) {
    size_t free_b = 0, total_b = 0;
    PLAN_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const uint64_t budget_bits = t.dedupe_bitmap == 2 ? (uint64_t)total_b / 4 * 8 : (48ull << 20) * 8;
    const uint64_t limit = std::min<uint64_t>(budget_bits / (uint64_t)pl->scan_grid, 0xFFFFFFFFull * 32);
    uint64_t bits = 0;
    for (uint64_t ns : {pl->nslots_base, pl->nslots_cand})
      if (ns && ns <= limit) bits = std::max(bits, ns);
    if (bits) {
      pl->bitmap_bits = bits;
      PLAN_CUDA(dev_alloc(pl, &pl->bitmap, (size_t)pl->scan_grid * ((bits + 31) / 32)));
    }
  }
  PLAN_CUDA(dev_alloc(pl, &pl->ctl, 1));
  if (pl->dry_run) {  // also count the result buffers and the schedule allocated below
    pl->dev_bytes += (((uint64_t)p->k * row_bytes_for(pl, p->n) + 8 + 255) & ~255ull) +
                     (((uint64_t)p->k * 8 + 255) & ~255ull) + (((uint64_t)m * 4 + 255) & ~255ull);
    *out = pl;
    return IG_OK;
  }
  PLAN_CUDA(cudaMemsetAsync(pl->ctl, 0, sizeof(PassCtl), pl->stream));
  PLAN_CUDA(cudaMallocHost(reinterpret_cast<void**>(&pl->h_ctl), sizeof(PassCtl)));
  if (p->flags & IG_F_TIMING) {
    const uint32_t np = p->n - pl->b + 1;
    for (auto* v : {&pl->ev_pass0, &pl->ev_pass1, &pl->ev_scan0, &pl->ev_scan1}) {
      v->assign(np, nullptr);
      for (auto& e : *v) PLAN_CUDA(cudaEventCreate(&e));
    }
  }
  pl->out_cap = p->k;
  PLAN_CUDA(dev_alloc(pl, &pl->out_keys, (size_t)pl->out_cap * row_bytes_for(pl, p->n) + 8));
  PLAN_CUDA(dev_alloc(pl, &pl->out_counts, pl->out_cap));

  // schedule: sequences longest first (ties by index)
  std::vector<uint32_t> order(m);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    return pl->h_offsets[x + 1] - pl->h_offsets[x] > pl->h_offsets[y + 1] - pl->h_offsets[y];
  });
  PLAN_CUDA(dev_alloc(pl, &pl->d_order, m));
  if (m) PLAN_CUDA(cudaMemcpyAsync(pl->d_order, order.data(), sizeof(uint32_t) * m, cudaMemcpyHostToDevice, pl->stream));
  // host staging above is pageable, so the copies have consumed it already;
  // the synchronisation only makes plan creation a clean point for callers
  if (!pl->async_alloc) PLAN_CUDA(cudaStreamSynchronize(pl->stream));
#undef PLAN_CUDA
  *out = pl;
  return IG_OK;
}

ig_status intergrams_pass(ig_plan* pl, uint32_t* j_done) {
  g_last_error.clear();
  if (!pl) return fail(IG_EINVAL, "plan is NULL");
  if (pl->pending_j) return fail(IG_ESTATE, "a sharded pass is waiting for intergrams_pass_select");
  if (pl->broken) return fail(IG_ESTATE, "the plan's survivor lists could not grow: free the plan");
  if (pl->next_j > pl->p.n) return IG_DONE;
  const uint32_t j = pl->next_j;
  char name[32];
  std::snprintf(name, sizeof(name), "ig pass %u", j);
  Range range(name);
  pl->kernels += enqueue_pass(pl, j, pl->stream);
  IG_CUDA(cudaGetLastError());
  finish_pass_host(pl, j);
  if (j_done) *j_done = j;
  ig_status st = read_status(pl);
  // a survivor list ran out of room: grow it and replay the job up to pass j
  for (int attempt = 0; st == IG_ETABLE_FULL && list_full_only(pl) && attempt < 8; ++attempt) {
    st = grow_lists(pl);
    if (st != IG_OK) return st;
    st = intergrams_rewind(pl);
    if (st != IG_OK) return st;
    g_last_error.clear();
    while (pl->next_j <= j) {
      const uint32_t jj = pl->next_j;
      pl->kernels += enqueue_pass(pl, jj, pl->stream);
      finish_pass_host(pl, jj);
    }
    IG_CUDA(cudaGetLastError());
    st = read_status(pl);
  }
  return st;
}

static ig_status run_remaining(ig_plan* pl);

ig_status intergrams_run(ig_plan* pl) {
  g_last_error.clear();
  if (!pl) return fail(IG_EINVAL, "plan is NULL");
  ig_status st = run_remaining(pl);
  // a survivor list ran out of room: grow it and run the whole job again
  for (int attempt = 0; st == IG_ETABLE_FULL && list_full_only(pl) && attempt < 8; ++attempt) {
    st = grow_lists(pl);
    if (st != IG_OK) return st;
    st = intergrams_rewind(pl);
    if (st != IG_OK) return st;
    g_last_error.clear();
    st = run_remaining(pl);
  }
  return st;
}

static ig_status run_remaining(ig_plan* pl) {
  g_last_error.clear();
  if (!pl) return fail(IG_EINVAL, "plan is NULL");
  if (pl->broken) return fail(IG_ESTATE, "the plan's survivor lists could not grow: free the plan");
  Range range("ig run");
  if (pl->pending_j) return fail(IG_ESTATE, "a sharded pass is waiting for intergrams_pass_select");
  if (pl->next_j > pl->p.n) return IG_OK;
  const bool from_start = pl->next_j == pl->b;
  if ((pl->p.flags & IG_F_GRAPH) && from_start) {
    // one graph per corpus buffer (the scans' arguments name the buffer)
    cudaGraphExec_t& graph = pl->data_slot ? pl->graph_alt : pl->graph;
    if (!graph) {
      // capture on a private stream (the legacy default stream cannot be
      // captured); the graph is then launched on the plan's stream
      cudaGraph_t g = nullptr;
      if (!pl->cap_stream) IG_CUDA(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
      IG_CUDA(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int cur0 = pl->cur;
      pl->graph_kernels = 0;
      for (uint32_t j = pl->b; j <= pl->p.n; ++j) {
        pl->graph_kernels += enqueue_pass(pl, j, pl->cap_stream);
        if (j < pl->p.n) pl->cur ^= 1;
      }
      pl->cur = cur0;
      cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
      if (e != cudaSuccess) return fail(IG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(IG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    IG_CUDA(cudaGraphLaunch(graph, pl->stream));
    pl->kernels += pl->graph_kernels;
    for (uint32_t j = pl->b; j <= pl->p.n; ++j) finish_pass_host(pl, j);
    return read_status(pl);
  }
  for (uint32_t j = pl->next_j; j <= pl->p.n; ++j) {
    pl->kernels += enqueue_pass(pl, j, pl->stream);
    finish_pass_host(pl, j);
  }
  IG_CUDA(cudaGetLastError());
  return read_status(pl);
}

ig_status intergrams_rewind(ig_plan* pl) {
  g_last_error.clear();
  if (!pl) return fail(IG_EINVAL, "plan is NULL");
  pl->cur = 0;  // the key buffers' parity at the start of a run (graphs are captured with it)
  pl->next_j = pl->b;
  pl->pending_j = 0;
  pl->last_j = 0;
  pl->nsel_last = 0;
  pl->kernels = 0;
  pl->feat_ready = false;
  if (pl->prefetched) {
    // switch to the prefetched buffer: everything queued so far read the old
    // one; what follows waits for the copy
    IG_CUDA(cudaEventRecord(pl->ev_left[pl->data_slot], pl->stream));
    pl->data_slot ^= 1u;
    pl->data = pl->data_slot ? pl->own_data_alt : pl->own_data;
    IG_CUDA(cudaStreamWaitEvent(pl->stream, pl->ev_copied, 0));
    pl->prefetched = false;
    return IG_OK;
  }
  if ((pl->p.flags & IG_F_HOST_INPUT) && pl->data_bytes)
    IG_CUDA(cudaMemcpyAsync(const_cast<uint8_t*>(pl->data), pl->host_data, pl->data_bytes, cudaMemcpyHostToDevice,
                            pl->stream));
  return IG_OK;
}

ig_status intergrams_prefetch(ig_plan* pl, const void* host_data) {
  g_last_error.clear();
  if (!pl) return fail(IG_EINVAL, "plan is NULL");
  if (!(pl->p.flags & IG_F_HOST_INPUT) || pl->dry_run) return fail(IG_ESTATE, "prefetch needs a plan made with IG_F_HOST_INPUT");
  if (pl->prefetched) return fail(IG_ESTATE, "a prefetch is already pending (rewind first)");
  if (!host_data) host_data = pl->host_data;
  if (!pl->data_bytes) {  // nothing to copy; the switch is a no-op
    pl->prefetched = false;
    return IG_OK;
  }
  if (!pl->copy_stream) IG_CUDA(cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&pl->ev_copied, &pl->ev_left[0], &pl->ev_left[1]})
    if (!*e) IG_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  if (!pl->own_data_alt) IG_CUDA(dev_alloc(pl, &pl->own_data_alt, pl->data_bytes));
  const uint32_t other = pl->data_slot ^ 1u;
  uint8_t* dst = other ? pl->own_data_alt : pl->own_data;
  // the other buffer may still be read by work queued before it was left
  IG_CUDA(cudaStreamWaitEvent(pl->copy_stream, pl->ev_left[other], 0));
  IG_CUDA(cudaMemcpyAsync(dst, host_data, pl->data_bytes, cudaMemcpyHostToDevice, pl->copy_stream));
  IG_CUDA(cudaEventRecord(pl->ev_copied, pl->copy_stream));
  pl->prefetched = true;
  return IG_OK;
}

// ---- sharded passes --------------------------------------------------------

ig_status intergrams_pass_scan(ig_plan* pl, uint32_t* j_out) {
  g_last_error.clear();
  if (!pl) return fail(IG_EINVAL, "plan is NULL");
  if (pl->dry_run) return fail(IG_ESTATE, "dry-run plan");
  if (pl->p.flags & IG_F_GRAPH) return fail(IG_ESTATE, "sharded passes are launched one by one (no IG_F_GRAPH)");
  if (pl->pending_j) return fail(IG_ESTATE, "the previous scan is waiting for intergrams_pass_select");
  if (pl->broken) return fail(IG_ESTATE, "the plan's survivor lists could not grow: free the plan");
  if (pl->next_j > pl->p.n) return IG_DONE;
  const uint32_t j = pl->next_j;
  char name[40];
  std::snprintf(name, sizeof(name), "ig pass %u scan", j);
  Range range(name);
  pl->kernels += enqueue_scan(pl, j, pl->stream);
  IG_CUDA(cudaGetLastError());
  pl->pending_j = j;
  pl->imported = false;
  if (j_out) *j_out = j;
  return IG_OK;
}

// Slots of the pending pass's counters.
static uint64_t pending_slots(const ig_plan* pl) {
  return mode_of(pl, pl->pending_j) == kModeBase ? pl->nslots_base : pl->nslots_cand;
}

ig_status intergrams_counts_export(ig_plan* pl, uint32_t* d_counts, uint64_t capacity, uint64_t* n_out) {
  g_last_error.clear();
  if (!pl || !n_out) return fail(IG_EINVAL, "plan or n_out is NULL");
  if (!pl->pending_j) return fail(IG_ESTATE, "no scan is pending (call intergrams_pass_scan first)");
  const uint64_t ns = pending_slots(pl);
  *n_out = ns;
  if (!d_counts || capacity < ns) return fail(IG_EINVAL, "counts buffer is NULL or smaller than the pass's slots");
  if (pl->narrow) {
    widen_counts_kernel<<<4 * 152, 256, 0, pl->stream>>>(pl->counts, ns, d_counts);
    pl->kernels += 1;
  } else {
    IG_CUDA(cudaMemcpyAsync(d_counts, pl->counts, ns * sizeof(uint32_t), cudaMemcpyDeviceToDevice, pl->stream));
  }
  IG_CUDA(cudaGetLastError());
  return IG_OK;
}

ig_status intergrams_counts_import(ig_plan* pl, const uint32_t* d_counts, uint64_t n) {
  g_last_error.clear();
  if (!pl || !d_counts) return fail(IG_EINVAL, "plan or counts is NULL");
  if (!pl->pending_j) return fail(IG_ESTATE, "no scan is pending (call intergrams_pass_scan first)");
  const uint64_t ns = pending_slots(pl);
  if (n != ns) return fail(IG_EINVAL, "count array length differs from the pass's slots");
  if (pl->narrow) {
    narrow_counts_kernel<<<4 * 152, 256, 0, pl->stream>>>(d_counts, ns, pl->counts, pl->ctl);
    pl->kernels += 1;
  } else {
    IG_CUDA(cudaMemcpyAsync(pl->counts, d_counts, ns * sizeof(uint32_t), cudaMemcpyDeviceToDevice, pl->stream));
  }
  IG_CUDA(cudaGetLastError());
  pl->imported = true;
  return IG_OK;
}

ig_status intergrams_pass_select(ig_plan* pl, uint32_t* j_done) {
  g_last_error.clear();
  if (!pl) return fail(IG_EINVAL, "plan is NULL");
  if (!pl->pending_j) return fail(IG_ESTATE, "no scan is pending (call intergrams_pass_scan first)");
  const uint32_t j = pl->pending_j;
  char name[40];
  std::snprintf(name, sizeof(name), "ig pass %u select", j);
  Range range(name);
  pl->kernels += enqueue_select(pl, j, pl->stream);
  IG_CUDA(cudaGetLastError());
  pl->pending_j = 0;
  pl->imported = false;
  finish_pass_host(pl, j);
  if (j_done) *j_done = j;
  return read_status(pl);
}

ig_status intergrams_shard_assign(const uint64_t* offsets, uint32_t m, uint32_t nshards, uint32_t* shard_of,
                                  uint64_t* shard_symbols) {
  g_last_error.clear();
  if (!offsets || (m && !shard_of) || nshards == 0) return fail(IG_EINVAL, "NULL argument or no shards");
  std::vector<uint32_t> order(m);
  for (uint32_t i = 0; i < m; ++i) {
    if (offsets[i + 1] < offsets[i]) return fail(IG_EINVAL, "offsets decrease");
    order[i] = i;
  }
  // longest sequence first (ties: lower index first), each to the shard
  // with the fewest symbols so far (ties: lower shard)
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
    return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
  });
  std::vector<uint64_t> load(nshards, 0);
  for (uint32_t i : order) {
    uint32_t best = 0;
    for (uint32_t g = 1; g < nshards; ++g)
      if (load[g] < load[best]) best = g;
    shard_of[i] = best;
    load[best] += offsets[i + 1] - offsets[i];
  }
  if (shard_symbols)
    for (uint32_t g = 0; g < nshards; ++g) shard_symbols[g] = load[g];
  return IG_OK;
}

ig_status intergrams_topk(ig_plan* pl, uint8_t* keys_out, uint64_t* counts_out, uint32_t capacity, uint32_t* k_out,
                          uint32_t* j_out) {
  g_last_error.clear();
  if (!pl || !k_out) return fail(IG_EINVAL, "plan or k_out is NULL");
  *k_out = 0;
  if (pl->last_j == 0) return fail(IG_ESTATE, "no pass has run yet");
  const uint32_t j = pl->last_j;
  if (j_out) *j_out = j;
  const uint32_t rows = std::min(std::min(pl->p.k, capacity), pl->nsel_last);
  if (rows == 0) return IG_OK;
  cudaStream_t s = pl->stream;
  launch_sort_by_count(pl->sel_count, pl->ctl, pl->sort_cap, pl->narrow ? 16u : 32u, pl->sidx[0], pl->sidx[1], pl->skey[0], pl->skey[1],
                       pl->shist, s);
  // symbols of each selected j-gram: walk back through every pass's selection
  const uint32_t rb = row_bytes_for(pl, j);
  launch_write_topk(pl->sel_hist, pl->p.candidates, pl->b, pl->sel_count, pl->sidx[0], pl->ctl, pl->sb, j, rb, rows,
                    pl->out_keys, pl->out_counts, s);
  pl->kernels += sort_kernels(pl) + 1;  // sort, then the row writer
  IG_CUDA(cudaGetLastError());
  if (keys_out) IG_CUDA(cudaMemcpyAsync(keys_out, pl->out_keys, (size_t)rows * rb, cudaMemcpyDeviceToHost, s));
  if (counts_out)
    IG_CUDA(cudaMemcpyAsync(counts_out, pl->out_counts, (size_t)rows * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  IG_CUDA(cudaStreamSynchronize(s));
  *k_out = rows;
  return IG_OK;
}

ig_status intergrams_features(ig_plan* pl, uint64_t* row_ptr, uint32_t* cols, uint64_t capacity, uint64_t* nnz_out) {
  g_last_error.clear();
  if (!pl || !nnz_out) return fail(IG_EINVAL, "plan or nnz_out is NULL");
  Range range("ig features");
  *nnz_out = 0;
  if (pl->dry_run) return fail(IG_ESTATE, "dry-run plan");
  if (pl->last_j != pl->p.n || pl->next_j <= pl->p.n) return fail(IG_ESTATE, "the job's passes have not all run");
  if (pl->p.n * pl->sb > 64) return fail(IG_EINVAL, "the feature matrix needs n * symbol_bits <= 64");
  const uint32_t rows = std::min(pl->p.k, pl->nsel_last);
  if (rows > (1u << 20)) return fail(IG_EINVAL, "the feature matrix takes at most 2^20 rows");
  cudaStream_t s = pl->stream;
  const uint32_t rb = row_bytes_for(pl, pl->p.n);
  // feature scans: 1024 threads, the plan's words per thread, tile + halo
  const uint32_t spw = 32 / pl->sb;
  const uint64_t fwin = (uint64_t)pl->t.words_per_thread * spw * 1024;
  const uint32_t ftile = (uint32_t)((((fwin + pl->p.n + 2 * 16 * (8 / pl->sb)) * pl->sb + 31) / 32 + 8 + 3) & ~3ull);
  const size_t fsmem = feature_smem_bytes(std::max(rows, 1u), ftile);
  int dev = 0, max_optin = 0;
  IG_CUDA(cudaGetDevice(&dev));
  IG_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (fsmem > (size_t)max_optin) return fail(IG_EINVAL, "feature bit vector and tile exceed shared memory");
  if (!pl->feat_ready) {
    if (rows) {  // the final rows on the device, as intergrams_topk writes them
      launch_sort_by_count(pl->sel_count, pl->ctl, pl->sort_cap, pl->narrow ? 16u : 32u, pl->sidx[0], pl->sidx[1],
                           pl->skey[0], pl->skey[1], pl->shist, s);
      launch_write_topk(pl->sel_hist, pl->p.candidates, pl->b, pl->sel_count, pl->sidx[0], pl->ctl, pl->sb, pl->p.n,
                        rb, rows, pl->out_keys, pl->out_counts, s);
    }
    if (!pl->feat_q) {
      uint32_t tl = 8;
      while ((1u << tl) < 4ull * std::max(pl->p.k, 1u)) ++tl;
      pl->feat_table_log2 = tl;
      // each buffer once: a failed call keeps what it got for the next one
      auto get = [&](auto** q, size_t bytes) {
        return *q ? cudaSuccess : device_malloc(reinterpret_cast<void**>(q), bytes, false, s);
      };
      IG_CUDA(get(&pl->feat_keys, sizeof(unsigned long long) * std::max(pl->p.k, 1u)));
      IG_CUDA(get(&pl->feat_table, sizeof(uint4) << tl));
      IG_CUDA(get(&pl->feat_nnz, sizeof(uint32_t) * std::max<uint32_t>(pl->m, 1)));
      IG_CUDA(get(&pl->feat_rowptr, sizeof(uint64_t) * ((size_t)pl->m + 1)));
      IG_CUDA(get(&pl->feat_q, 4 * sizeof(uint32_t)));
    }
    IG_CUDA(feature_set_smem(pl->sb, fsmem));
    IG_CUDA(cudaMemsetAsync(pl->feat_q, 0, 4 * sizeof(uint32_t), s));
    launch_features(pl->data, pl->data_bytes, pl->offsets, pl->d_order, pl->m, pl->p.n, pl->sb, pl->out_keys, rows, rb,
                    pl->feat_keys, pl->feat_table, pl->feat_table_log2, pl->feat_q, pl->feat_q + 2, pl->feat_nnz,
                    pl->feat_rowptr, nullptr, true, pl->sms, pl->t.words_per_thread, ftile, fsmem, s);
    uint32_t st = 0;
    IG_CUDA(cudaMemcpyAsync(&pl->feat_total, pl->feat_rowptr + pl->m, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    IG_CUDA(cudaMemcpyAsync(&st, pl->feat_q + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    IG_CUDA(cudaStreamSynchronize(s));
    IG_CUDA(cudaGetLastError());
    if (st) return fail(IG_ETABLE_FULL, "feature table full");
    pl->feat_rows = rows;
    pl->feat_ready = true;
  }
  *nnz_out = pl->feat_total;
  if (cols && capacity < pl->feat_total) return fail(IG_EINVAL, "cols capacity is below the number of nonzeros");
  if (cols && pl->feat_total) {
    uint32_t* d_cols = nullptr;
    IG_CUDA(device_malloc(reinterpret_cast<void**>(&d_cols), sizeof(uint32_t) * pl->feat_total, false, s));
    // the limit again: another plan's feature call since the counting scan may have changed it
    cudaError_t e = feature_set_smem(pl->sb, fsmem);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->feat_q + 1, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) {
      launch_features(pl->data, pl->data_bytes, pl->offsets, pl->d_order, pl->m, pl->p.n, pl->sb, pl->out_keys,
                      pl->feat_rows, rb, pl->feat_keys, pl->feat_table, pl->feat_table_log2, pl->feat_q, pl->feat_q + 2,
                      pl->feat_nnz, pl->feat_rowptr, d_cols, false, pl->sms, pl->t.words_per_thread, ftile, fsmem, s);
      e = cudaMemcpyAsync(cols, d_cols, sizeof(uint32_t) * pl->feat_total, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    device_free(d_cols, false, s);
    if (e != cudaSuccess) return fail(IG_ECUDA, cudaGetErrorString(e));
  }
  if (row_ptr) {
    IG_CUDA(cudaMemcpyAsync(row_ptr, pl->feat_rowptr, sizeof(uint64_t) * ((size_t)pl->m + 1), cudaMemcpyDeviceToHost, s));
    IG_CUDA(cudaStreamSynchronize(s));
  }
  return IG_OK;
}

ig_status intergrams_plan_device_bytes(const ig_plan* pl, uint64_t* bytes) {
  if (!pl || !bytes) return fail(IG_EINVAL, "plan or bytes is NULL");
  *bytes = pl->dev_bytes;
  return IG_OK;
}

ig_status intergrams_stats(ig_plan* pl, ig_pass_stats* out) {
  if (!pl || !out) return fail(IG_EINVAL, "plan or out is NULL");
  std::memset(out, 0, sizeof(*out));
  if (pl->last_j == 0) return fail(IG_ESTATE, "no pass has run yet");
  IG_CUDA(cudaMemcpyAsync(pl->h_ctl, pl->ctl, sizeof(PassCtl), cudaMemcpyDeviceToHost, pl->stream));
  IG_CUDA(cudaStreamSynchronize(pl->stream));
  out->j = pl->last_j;
  out->windows = windows_for(pl, pl->last_j);
  out->survivors = pl->h_ctl->survivors;
  out->registrations = pl->h_ctl->registrations;
  out->nonzero_selected = pl->h_ctl->nsel;
  out->scanned_bytes = pl->data_bytes;
  return IG_OK;
}

ig_status intergrams_timings(ig_plan* pl, float* scan_ms, float* pass_ms, uint32_t cap, uint32_t* npasses,
                             uint32_t* kernels) {
  g_last_error.clear();
  if (!pl || !npasses) return fail(IG_EINVAL, "plan or npasses is NULL");
  *npasses = 0;
  if (kernels) *kernels = pl->kernels;
  if (!(pl->p.flags & IG_F_TIMING)) return fail(IG_ESTATE, "plan was made without IG_F_TIMING");
  if (pl->last_j == 0) return IG_OK;
  IG_CUDA(cudaStreamSynchronize(pl->stream));
  const uint32_t np = pl->last_j - pl->b + 1;
  for (uint32_t i = 0; i < np && i < cap; ++i) {
    if (scan_ms) IG_CUDA(cudaEventElapsedTime(scan_ms + i, pl->ev_scan0[i], pl->ev_scan1[i]));
    if (pass_ms) IG_CUDA(cudaEventElapsedTime(pass_ms + i, pl->ev_pass0[i], pl->ev_pass1[i]));
  }
  *npasses = np;
  return IG_OK;
}

ig_status intergrams_test_fail_alloc(uint32_t nth, uint64_t* live_out) {
  g_fail_alloc_in.store(nth);
  if (live_out) *live_out = (uint64_t)std::max<int64_t>(0, g_live_allocs.load());
  return IG_OK;
}

ig_status intergrams_test_stall_tiles(ig_plan* pl) {
  g_last_error.clear();
  if (!pl) {
    arm_static_stall();
    return IG_OK;
  }
  if (pl->p.flags & IG_F_GRAPH) return fail(IG_ESTATE, "the stall hook needs pass-by-pass launches (no IG_F_GRAPH)");
  pl->test_stall_tiles = 1;
  return IG_OK;
}

void intergrams_free(ig_plan* pl) {
  if (!pl) return;
  if (!pl->dry_run) cudaStreamSynchronize(pl->stream);
  release(pl);
}

}  // extern "C"
