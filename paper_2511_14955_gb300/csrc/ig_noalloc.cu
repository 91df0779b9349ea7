// Allocation-free entry point: exact top-k of short n-grams using only a
// fixed scratch array compiled into the library.
//
// Some callers cannot allocate device memory at the time they need an answer:
// code running inside a memory pool or arena that owns the whole device
// budget, callers holding a strict no-allocation contract on a hot path (an
// allocator call can synchronise the device or fail under fragmentation),
// and embedders that forbid cudaMalloc/cudaFree after start-up. For them this
// call runs the same dense counting pass, selection and ordering kernels as
// the planned path, but every table those kernels need lives in one
// file-scope __device__ array of kScratchBytes bytes. The caller passes only
// its inputs and its output buffers.
//
// Nothing here is allocated: no cudaMalloc, cudaFree, host-pinned memory or
// allocating library routine. The scratch array occupies kScratchBytes on
// every GPU that loads the library, until the process exits.
#include <atomic>

#include "ig_internal.cuh"

namespace ig {
namespace {

constexpr size_t kScratchBytes = 40ull << 20;        // 40 MiB per device
constexpr uint32_t kMaxSlots = 1u << 16;             // sigma^n limit (bytes: n <= 2, bases: n <= 8)
constexpr uint32_t kMaxSeqs = 1u << 20;              // sequences per call
constexpr uint32_t kGrid = 32;                       // scan CTAs
constexpr uint32_t kThreads = 512, kWords = 9, kSsetLog2 = 15;
constexpr uint32_t kGsetLog2 = 17;                   // >= 2 * kMaxSlots entries per CTA set

// Host code must not take this array's address directly (the host-side name
// is only a stand-in); every call asks the runtime for the device address on
// the current device (cheap, allocates nothing) and passes that pointer to
// the kernels, so a context made again after a device reset is followed.
// The array starts zeroed when the module loads; the control block's dedupe
// epochs carry over from call to call, so the dedupe sets are cleared only
// when the 32-bit epochs wrap.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Layout {
  size_t ctl, counts, hist, blk, sel_slot, sel_count, idx0, idx1, key0, key1, shist, order, gset, end;
};

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout layout() {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  L.ctl = take(sizeof(PassCtl));
  L.counts = take(sizeof(uint32_t) * kMaxSlots);
  L.hist = take(sizeof(uint32_t) * kMaxLevels * kHistBins);
  L.blk = take(sizeof(uint32_t) * 2 * 1024);
  L.sel_slot = take(sizeof(uint32_t) * kMaxSlots);
  L.sel_count = take(sizeof(uint32_t) * kMaxSlots);
  L.idx0 = take(sizeof(uint32_t) * kMaxSlots);
  L.idx1 = take(sizeof(uint32_t) * kMaxSlots);
  L.key0 = take(sizeof(uint32_t) * kMaxSlots);
  L.key1 = take(sizeof(uint32_t) * kMaxSlots);
  L.shist = take(sizeof(uint32_t) * kSortDigits * (kMaxSlots / kSortChunk + 1));
  L.order = take(sizeof(uint32_t) * kMaxSeqs);
  L.gset = take(sizeof(unsigned long long) * ((size_t)kGrid << kGsetLog2));
  L.end = o;
  return L;
}

__global__ void iota_kernel(uint32_t* order, uint32_t m) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) order[i] = i;
}

// Start of a call: the sticky status bits of the previous call are dropped
// (the dedupe epochs are kept).
__global__ void clear_status_kernel(PassCtl* ctl) {
  if (threadIdx.x == 0) ctl->status = 0;
}

// End of a call: the row count, or 0 rows and the failure when the scan
// reported one (a tile wait that ran out, a full dedupe set).
__global__ void finish_kernel(const PassCtl* ctl, uint32_t k, uint32_t* rows, int32_t* status) {
  if (threadIdx.x != 0) return;
  const uint32_t st = ctl->status;
  int32_t code = IG_OK;
  if (st & kStTimeout) code = IG_ETIMEOUT;
  else if (st & kStCountOverflow) code = IG_EOVERFLOW;
  else if (st & (kStSetFull | kStTableFull | kStListFull | kStQueue)) code = IG_ETABLE_FULL;
  rows[0] = code != IG_OK ? 0u : (ctl->nsel < k ? ctl->nsel : k);
  status[0] = code;
}

std::atomic<uint32_t> g_stall_next{0};  // test hook: the next call's tile waits run out

}  // namespace

// Defined in ig_api.cu: records the message for intergrams_last_error().
void set_last_error(const std::string& msg);

}  // namespace ig

using namespace ig;

extern "C" ig_status intergrams_dense_topk_static(const ig_params* p, const void* data, const uint64_t* offsets,
                                                  uint32_t m, uint64_t total_symbols, void* stream,
                                                  uint8_t* keys_out, uint64_t* counts_out, uint32_t* rows_out,
                                                  int32_t* status_out) {
  auto bad = [&](ig_status st, const char* msg) {
    set_last_error(msg);
    return st;
  };
  set_last_error("");
  if (!p || !offsets || !keys_out || !counts_out || !rows_out || !status_out) return bad(IG_EINVAL, "NULL argument");
  if (p->symbol_bits != 8 && p->symbol_bits != 2) return bad(IG_EINVAL, "symbol_bits must be 8 or 2");
  if (p->count_mode > 1) return bad(IG_EINVAL, "count_mode must be 0 or 1");
  if (p->n < 1 || p->n * p->symbol_bits > 16)
    return bad(IG_EINVAL, "n too large for the static scratch: sigma^n must be <= 65536 (n <= 2 bytes or 8 bases)");
  if (p->k < 1 || p->k > kMaxSlots) return bad(IG_EINVAL, "k must be in 1..65536");
  if (m > kMaxSeqs) return bad(IG_EINVAL, "too many sequences for the static scratch (limit 2^20)");
  if (total_symbols && !data) return bad(IG_EINVAL, "data is NULL");
  if (p->count_mode == IG_COUNT_EVERY_OCCURRENCE && total_symbols >= 0xFFFFFFFFull)
    return bad(IG_EINVAL, "Eq. 1 counts of 2^32 - 1 or more windows do not fit the 32-bit counters of the static scratch");
  const Layout L = layout();
  if (L.end > kScratchBytes) return bad(IG_EINVAL, "internal: scratch layout exceeds its array");

  void* base = nullptr;
  if (cudaGetSymbolAddress(&base, g_scratch) != cudaSuccess || !base)
    return bad(IG_ECUDA, "cudaGetSymbolAddress(g_scratch) failed");
  unsigned char* S = static_cast<unsigned char*>(base);
  PassCtl* ctl = reinterpret_cast<PassCtl*>(S + L.ctl);
  uint32_t* counts = reinterpret_cast<uint32_t*>(S + L.counts);
  unsigned long long* gset = reinterpret_cast<unsigned long long*>(S + L.gset);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t sb = p->symbol_bits, n = p->n;
  const uint64_t nslots = 1ull << (n * sb);

  // smem of the scan: dedupe set + tile (+ halo, alignment slop)
  const uint32_t spw = 32 / sb;
  const uint64_t tile_syms = (uint64_t)kWords * spw * kThreads + n + 2 * 16 * (8 / sb);
  uint32_t tile_words = (uint32_t)((tile_syms * sb + 31) / 32) + 8;
  tile_words = (tile_words + 3) & ~3u;
  const size_t smem = ((size_t)4 << kSsetLog2) + (size_t)tile_words * 4;
  if (scan_raise_smem_limit(sb, true, smem) != cudaSuccess) return bad(IG_ECUDA, "cudaFuncSetAttribute failed");

  // the scratch keeps the previous call's contents: zero what must start at
  // 0 (status bits, counters); the dedupe sets are cleared when the epochs
  // carried over from earlier calls would wrap
  clear_status_kernel<<<1, 32, 0, s>>>(ctl);
  if (m) iota_kernel<<<256, 256, 0, s>>>(reinterpret_cast<uint32_t*>(S + L.order), m);
  launch_pass_reset(ctl, m, p->count_mode == IG_COUNT_ONCE_PER_SEQUENCE ? gset : nullptr,
                    (uint64_t)kGrid << kGsetLog2, s);
  if (cudaMemsetAsync(counts, 0, nslots * sizeof(uint32_t), s) != cudaSuccess)
    return bad(IG_ECUDA, "cudaMemsetAsync failed");
  ScanArgs a{};
  a.data = static_cast<const uint8_t*>(data);
  a.data_bytes = (total_symbols * sb + 7) / 8;
  a.offsets = offsets;
  a.order = reinterpret_cast<const uint32_t*>(S + L.order);
  a.m = m;
  a.j = n;
  a.key_mask = (1ull << (n * sb)) - 1ull;
  a.table = nullptr;
  a.table_log2 = 0;
  a.counts = counts;
  a.gset = gset;
  a.gset_log2 = kGsetLog2;
  a.count_mode = p->count_mode;
  a.words_per_thread = kWords;
  a.sset_log2 = kSsetLog2;
  a.tile_words = tile_words;
  a.check_overflow = 0;  // Eq. 1 inputs of 2^32 - 1 or more windows are rejected above
  a.stall_tiles = g_stall_next.exchange(0);
  a.ctl = ctl;
  if (m) launch_scan(a, sb, true, (int)kGrid, (int)kThreads, smem, s);
  launch_select(counts, false, nullptr, sb, nslots, p->k, ctl, reinterpret_cast<uint32_t*>(S + L.hist),
                reinterpret_cast<uint32_t*>(S + L.blk), 1024, reinterpret_cast<uint32_t*>(S + L.sel_slot),
                reinterpret_cast<uint32_t*>(S + L.sel_count), s);
  launch_sort_by_count(reinterpret_cast<uint32_t*>(S + L.sel_count), ctl, kMaxSlots, 32u,
                       reinterpret_cast<uint32_t*>(S + L.idx0), reinterpret_cast<uint32_t*>(S + L.idx1),
                       reinterpret_cast<uint32_t*>(S + L.key0), reinterpret_cast<uint32_t*>(S + L.key1),
                       reinterpret_cast<uint32_t*>(S + L.shist), s);
  launch_write_topk(reinterpret_cast<uint32_t*>(S + L.sel_slot), 0, n, reinterpret_cast<uint32_t*>(S + L.sel_count),
                    reinterpret_cast<uint32_t*>(S + L.idx0), ctl, sb, n, (n * sb + 7) / 8, p->k, keys_out,
                    reinterpret_cast<unsigned long long*>(counts_out), s);
  finish_kernel<<<1, 32, 0, s>>>(ctl, p->k, rows_out, status_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bad(IG_ECUDA, cudaGetErrorString(e));
  return IG_OK;
}

// Test hook behind intergrams_test_stall_tiles(NULL): the next call's scan
// waits for tiles that are never sent.
void ig::arm_static_stall() { g_stall_next.store(1); }
