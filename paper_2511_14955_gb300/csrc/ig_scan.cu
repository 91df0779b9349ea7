// Corpus scan of one pass (paper Algorithm 2 for the dense base pass,
// Algorithm 3's inner loop for the candidate passes).
//
// A persistent grid pulls whole sequences from a queue ordered longest
// first. A CTA owns its sequence: it streams it through shared memory in
// tiles (each tile carries a halo of j-1 symbols so windows that cross a
// tile edge are complete; tiles arrive by bulk copy, the next one in flight
// while the current one is processed), and
//   base pass      : each thread rolls a j-symbol key over its run of
//                    windows; slot = the j-gram itself (sigma^j counters);
//   candidate pass : windows alive in the previous pass's survivor bits are
//                    queued; a queued window's (j-1)-gram prefix is looked up
//                    (hot cache in shared memory, then the probe table of
//                    P^(j-1); in pass base+1 by rank/select over the
//                    candidate bit vector of base-length prefixes, or a dense
//                    map); a hit is a survivor with slot = row * sigma + last
//                    symbol, and it sets its survivor bit for the next pass.
// Under Eq. 2 a survivor is counted only the first time its slot appears in
// the sequence (the paper's per-sequence bit vector C_i): a per-CTA bit
// vector over the slots when the slot space is small, else a bounded-probe
// shared-memory set whose overflow goes to a CTA-private spill list that is
// hash-partitioned and deduplicated bucket by bucket at the sequence's end
// (the allocation-free entry point uses an epoch-stamped global set
// instead). Under Eq. 1 every survivor counts. Counting is an atomic
// increment of the dense slot counter (the paper's C).
//
// chain_kernel runs a pass from the previous pass's survivor lists instead
// of the corpus (keys longer than 64 bits).
#include <vector>

#include "ig_internal.cuh"

namespace ig {

namespace {

template <int SB>
struct Sym {
  static constexpr uint32_t kPerWord = 32 / SB;
  static constexpr uint32_t kMask = (1u << SB) - 1u;
};

__device__ __forceinline__ uint32_t bswap32(uint32_t w) { return __byte_perm(w, 0, 0x0123); }

// Candidate lookup: id of `prefix` in P^(j-1), or kEmpty32.
__device__ __forceinline__ uint32_t probe_table(const uint4* __restrict__ table, uint32_t log2,
                                                uint64_t prefix, PassCtl* ctl) {
  const uint32_t mask = (1u << log2) - 1u;
  uint32_t h = hash64_top(prefix, log2);
  const uint32_t lo = (uint32_t)prefix, hi = (uint32_t)(prefix >> 32);
  for (uint32_t it = 0; it <= mask; ++it) {
    uint4 e = __ldg(table + h);
    if (e.z == kEmpty32) return kEmpty32;
    if (e.x == lo && e.y == hi) return e.z;
    h = (h + 1) & mask;
  }
  atomicOr(&ctl->status, kStTableFull);
  return kEmpty32;
}

// The paper's per-sequence bit vector C_i: set bit `slot`; true if it was
// clear (first occurrence of the slot in the sequence).
__device__ __forceinline__ bool bitmap_first(uint32_t* bm, uint32_t slot) {
  const uint32_t bit = 1u << (slot & 31u);
  return (atomicOr(bm + (slot >> 5), bit) & bit) == 0u;
}

// probe_table with the entry at the prefix's home position already loaded.
__device__ __forceinline__ uint32_t probe_from(const uint4* __restrict__ table, uint32_t log2, uint64_t prefix,
                                               uint4 e, PassCtl* ctl) {
  const uint32_t mask = (1u << log2) - 1u;
  uint32_t h = hash64_top(prefix, log2);
  const uint32_t lo = (uint32_t)prefix, hi = (uint32_t)(prefix >> 32);
  for (uint32_t it = 0; it <= mask; ++it) {
    if (e.z == kEmpty32) return kEmpty32;
    if (e.x == lo && e.y == hi) return e.z;
    h = (h + 1) & mask;
    e = __ldg(table + h);
  }
  atomicOr(&ctl->status, kStTableFull);
  return kEmpty32;
}

// Insert into the CTA-private global set; true if `slot` is new for this
// (pass, sequence) epoch.
__device__ __forceinline__ bool gset_insert(unsigned long long* set, uint32_t log2, uint32_t epoch,
                                            uint32_t slot, PassCtl* ctl) {
  const uint32_t mask = (1u << log2) - 1u;
  uint32_t h = hash32_top(slot, log2);
  const unsigned long long want = ((unsigned long long)epoch << 32) | slot;
  uint32_t it = 0;
  unsigned long long cur = *((volatile unsigned long long*)(set + h));
  while (it <= mask) {
    if ((uint32_t)(cur >> 32) == epoch) {
      if ((uint32_t)cur == slot) return false;
      h = (h + 1) & mask;
      ++it;
      cur = *((volatile unsigned long long*)(set + h));
      continue;
    }
    unsigned long long old = atomicCAS(set + h, cur, want);
    if (old == cur) return true;
    cur = old;  // lost a race at this position: look at it again
  }
  atomicOr(&ctl->status, kStSetFull);
  return false;
}

// Insert into the shared-memory set of the current sequence; falls back to
// the global set when the bounded probe finds no room.
__device__ __forceinline__ bool seq_first_seen(uint32_t* sset, uint32_t slog, unsigned long long* gset,
                                               uint32_t glog, uint32_t epoch, uint32_t slot, PassCtl* ctl) {
  const uint32_t mask = (1u << slog) - 1u;
  uint32_t h = hash32_top(slot, slog);
  const uint32_t maxp = mask < 7u ? mask + 1u : 8u;
  for (uint32_t p = 0; p < maxp; ++p) {
    uint32_t cur = sset[h];
    if (cur == slot) return false;
    if (cur == kEmpty32) {
      uint32_t old = atomicCAS(sset + h, kEmpty32, slot);
      if (old == kEmpty32) return true;
      if (old == slot) return false;
    }
    h = (h + 1) & mask;
  }
  return gset_insert(gset, glog, epoch, slot, ctl);
}

// Key of the window whose first symbol is tile symbol `o` (j * SB <= 64 bits):
// 64 bits of the (big-endian) symbol stream starting at bit o * SB, shifted
// down to j symbols. Reads three words; the tile buffer has slack past its end.
template <int SB>
__device__ __forceinline__ uint64_t tile_key(const uint32_t* tile, uint32_t o, uint32_t j) {
  const uint32_t bit = o * SB, wi = bit >> 5, sh = bit & 31;
  const uint64_t hi = ((uint64_t)__byte_perm(tile[wi], 0, 0x0123) << 32) | __byte_perm(tile[wi + 1], 0, 0x0123);
  const uint32_t w2 = __byte_perm(tile[wi + 2], 0, 0x0123);
  const uint64_t v = sh ? ((hi << sh) | (w2 >> (32 - sh))) : hi;
  const uint32_t bits = j * SB;
  return bits >= 64 ? v : (v >> (64 - bits));
}

// ---- tile staging with the bulk-copy engine --------------------------------
// A tile's bytes [al, al + nbytes) (al 16-byte aligned, nbytes a multiple of
// 16) go to shared memory by one cp.async.bulk for the part inside the
// corpus' 16-byte aligned extent, completing on an mbarrier; the few 16-byte
// chunks outside it (only at the corpus' ends) are built with byte loads,
// zero past the corpus.
struct TileGeom {
  uint32_t nwin, sym_off, nbytes;
  uint64_t gsym;
  uintptr_t al;
};

template <int SB>
__device__ __forceinline__ TileGeom tile_geom(const ScanArgs& a, uint64_t s0, uint64_t W, uint64_t w0,
                                              uint32_t tile_windows, uint32_t j) {
  TileGeom g;
  g.nwin = (uint32_t)((W - w0) < tile_windows ? (W - w0) : tile_windows);
  g.gsym = s0 + w0;
  const uint64_t nsym = (uint64_t)g.nwin + j - 1;
  const uint64_t b_first = (g.gsym * SB) >> 3;
  const uint64_t b_end = ((g.gsym + nsym) * SB + 7) >> 3;
  const uintptr_t addr_first = reinterpret_cast<uintptr_t>(a.data) + b_first;
  g.al = addr_first & ~(uintptr_t)15;
  g.sym_off = (uint32_t)(addr_first - g.al) * (32 / SB) / 4u + (uint32_t)(g.gsym % (8u / SB));
  g.nbytes = (uint32_t)((reinterpret_cast<uintptr_t>(a.data) + b_end - g.al + 15) & ~(uintptr_t)15);
  return g;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for phase `parity` of `bar`: false if it did not complete
// within kTileWaitNs of global time (or 2^31 polls, whichever comes first).
constexpr uint64_t kTileWaitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_addr(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < (1u << 31); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 31u) == 0) {
      const uint64_t t = global_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > kTileWaitNs) return false;
    }
  }
  return false;
}

// Start staging tile `g` into `buf` (all threads call; thread 0 issues the
// bulk copy and arms the barrier, the others build the edge chunks).
__device__ __forceinline__ void stage_issue(const ScanArgs& a, const TileGeom& g, uint8_t* buf, uint64_t* bar) {
  const uintptr_t lo_ok = reinterpret_cast<uintptr_t>(a.data), hi_ok = lo_ok + a.data_bytes;
  const uintptr_t lo16 = (lo_ok + 15) & ~(uintptr_t)15, hi16 = hi_ok & ~(uintptr_t)15;
  const uintptr_t ia = g.al > lo16 ? g.al : lo16;
  const uintptr_t ie = (g.al + g.nbytes) < hi16 ? (g.al + g.nbytes) : hi16;
  const uint32_t bytes = ie > ia ? (uint32_t)(ie - ia) : 0u;
  if (threadIdx.x == 0 && !a.stall_tiles) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    if (bytes && a.tile_evict_first) {
      // the corpus is read once per pass: its lines go first, so the
      // counters, spill lists and tables stay in L2
      uint64_t pol;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
          "%4;" ::"r"(smem_addr(buf + (ia - g.al))),
          "l"(ia), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
          : "memory");
    } else if (bytes) {
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(buf + (ia - g.al))),
          "l"(ia), "r"(bytes), "r"(smem_addr(bar))
          : "memory");
    }
  }
  for (uint32_t x = threadIdx.x * 16u; x < g.nbytes; x += blockDim.x * 16u) {
    const uintptr_t p = g.al + x;
    if (bytes && p >= ia && p < ie) continue;  // part of the bulk copy
    uint32_t w[4] = {0, 0, 0, 0};
    for (int b = 0; b < 16; ++b) {
      const uintptr_t q = p + b;
      const uint32_t byte = (q >= lo_ok && q < hi_ok) ? *reinterpret_cast<const uint8_t*>(q) : 0u;
      w[b >> 2] |= byte << (8 * (b & 3));
    }
    *reinterpret_cast<uint4*>(buf + x) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Prefetch tile `g`'s bytes inside the corpus' 16-byte aligned extent into
// L2 (one bulk prefetch by thread 0; no shared memory, nothing to wait for),
// so that the tile's later bulk copy reads L2: with one copy in flight per
// CTA, a copy from HBM per tile left streaming passes latency-bound.
__device__ __forceinline__ void prefetch_tile(const ScanArgs& a, const TileGeom& g) {
  if (threadIdx.x != 0 || a.stall_tiles) return;
  const uintptr_t lo_ok = reinterpret_cast<uintptr_t>(a.data), hi_ok = lo_ok + a.data_bytes;
  const uintptr_t lo16 = (lo_ok + 15) & ~(uintptr_t)15, hi16 = hi_ok & ~(uintptr_t)15;
  const uintptr_t ia = g.al > lo16 ? g.al : lo16;
  const uintptr_t ie = (g.al + g.nbytes) < hi16 ? (g.al + g.nbytes) : hi16;
  if (ie > ia)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ia), "r"((uint32_t)(ie - ia)) : "memory");
}

// tile_key for keys of at most 32 bits (two words).
template <int SB>
__device__ __forceinline__ uint64_t tile_key32(const uint32_t* tile, uint32_t o, uint32_t j) {
  const uint32_t bit = o * SB, wi = bit >> 5, sh = bit & 31;
  const uint32_t v = __funnelshift_l(__byte_perm(tile[wi + 1], 0, 0x0123), __byte_perm(tile[wi], 0, 0x0123), sh);
  const uint32_t bits = j * SB;
  return bits >= 32 ? v : (v >> (32 - bits));
}

// Symbol `o` of the tile.
template <int SB>
__device__ __forceinline__ uint32_t tile_sym(const uint32_t* tile, uint32_t o) {
  const uint32_t bit = o * SB;
  const uint32_t w = __byte_perm(tile[bit >> 5], 0, 0x0123);
  return (w >> (32 - SB - (bit & 31))) & ((1u << SB) - 1u);
}

// Phase 1 of the spill dedupe: bounded probe of the shared-memory set of the
// current sequence. 0 = already present, 1 = inserted (first occurrence),
// 2 = no room on the probe path (the slot goes to the spill list). A slot that
// once found its path full finds it full forever (entries are never removed
// within a sequence), so the spilled slots and the slots in the set are
// disjoint.
__device__ __forceinline__ int sset_try_insert(uint32_t* sset, uint32_t slog, uint32_t slot, uint32_t probes) {
  const uint32_t mask = (1u << slog) - 1u;
  uint32_t h = hash32_top(slot, slog);
  const uint32_t maxp = mask < probes - 1u ? mask + 1u : probes;
  for (uint32_t p = 0; p < maxp; ++p) {
    uint32_t cur = sset[h];
    if (cur == slot) return 0;
    if (cur == kEmpty32) {
      uint32_t old = atomicCAS(sset + h, kEmpty32, slot);
      if (old == kEmpty32) return 1;
      if (old == slot) return 0;
    }
    h = (h + 1) & mask;
  }
  return 2;
}

// Unbounded (whole-table) probe: the caller guarantees room for every
// distinct slot it inserts; a full table is reported.
__device__ __forceinline__ bool sset_insert_full(uint32_t* sset, uint32_t slog, uint32_t slot, PassCtl* ctl) {
  const uint32_t mask = (1u << slog) - 1u;
  uint32_t h = hash32_top(slot, slog);
  for (uint32_t p = 0; p <= mask; ++p) {
    uint32_t cur = sset[h];
    if (cur == slot) return false;
    if (cur == kEmpty32) {
      uint32_t old = atomicCAS(sset + h, kEmpty32, slot);
      if (old == kEmpty32) return true;
      if (old == slot) return false;
    }
    h = (h + 1) & mask;
  }
  atomicOr(&ctl->status, kStSetFull);
  return false;
}

// Append `slot` to the spill list: one shared-memory atomic per warp among
// the lanes spilling together.
__device__ __forceinline__ void spill_push(uint32_t* list, uint32_t* n, uint32_t slot) {
  const uint32_t peers = __activemask();
  const uint32_t lane = threadIdx.x & 31u, leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(n, (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  list[base + __popc(peers & ((1u << lane) - 1u))] = slot;
}

// Bucket bits of a spilled slot: bits [shift, shift + kb) (from the top) of
// the murmur3 32-bit finaliser (Appleby), unrelated to the multiply-shift
// bits that index the shared-memory set.
__device__ __forceinline__ uint32_t spill_bucket(uint32_t x, uint32_t shift, uint32_t kb) {
  x ^= x >> 16; x *= 0x85ebca6bu; x ^= x >> 13; x *= 0xc2b2ae35u; x ^= x >> 16;
  return kb == 0 ? 0u : (x << shift) >> (32 - kb);
}

// FIX: 16-bit counters known at compile time.
template <bool FIX = false>
__device__ __forceinline__ void count_at_once(const ScanArgs& a, uint32_t slot) {
  if (FIX || a.narrow) {  // 16-bit counter slot of word slot / 2 (little-endian half); counts < 65536
    atomicAdd(a.counts + (slot >> 1), 1u << ((slot & 1u) << 4));
    return;
  }
  if (a.check_overflow) {
    if (atomicAdd(a.counts + slot, 1u) == 0xFFFFFFFFu) atomicOr(&a.ctl->status, kStCountOverflow);
  } else {
    atomicAdd(a.counts + slot, 1u);
  }
}

// The CTA's registration-log state in shared memory: open chunk and fill of
// each counter range.
struct LogState {
  uint32_t* chunk;
  uint32_t* fill;
};

__device__ __forceinline__ void log_init(const LogState& lg) {
  if (threadIdx.x < kLogMaxRanges) {
    lg.chunk[threadIdx.x] = kNoChunk;
    lg.fill[threadIdx.x] = 0;
  }
}

// Count `slot` (Eq. 1 / Eq. 2 increment of C): appended to the log when the
// pass keeps one, else counted at once. A chunk that is somehow full also
// falls back to counting at once, so the log never overflows.
template <bool FIX = false>
__device__ __forceinline__ void register_slot(const ScanArgs& a, const LogState& lg, uint32_t slot) {
  if (!FIX && a.rlog) {
    const uint32_t r = slot >> a.range_shift;
    const uint32_t c = lg.chunk[r];
    if (c < kNoChunk) {
      // one shared-memory atomic per range among the lanes registering now
      const uint32_t peers = __match_any_sync(__activemask(), r);
      const uint32_t lane = threadIdx.x & 31u, leader = __ffs(peers) - 1;
      uint32_t pos = 0;
      if (lane == leader) pos = atomicAdd(lg.fill + r, (uint32_t)__popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & ((1u << lane) - 1u));
      if (pos < (1u << a.rlog_chunk_log2)) {
        a.rlog[((uint64_t)c << a.rlog_chunk_log2) + pos] = slot;
        return;
      }
    }
  }
  count_at_once<FIX>(a, slot);
}

// Before a step that registers at most `need` slots (threads < nranges; the
// caller synchronises before the step and after it): every range's open
// chunk gets room for `need` more entries; a chunk without room is closed and
// a new one taken from the pool.
__device__ __forceinline__ void log_room(const ScanArgs& a, const LogState& lg, uint32_t need) {
  const uint32_t r = threadIdx.x;
  if (!a.rlog || r >= a.nranges) return;
  const uint32_t size = 1u << a.rlog_chunk_log2;
  uint32_t c = lg.chunk[r];
  if (c == kEmpty32) return;  // pool exhausted: this CTA counts at once
  if (c != kNoChunk) {
    if (lg.fill[r] + need <= size) return;
    a.rlog_fill[c] = lg.fill[r] < size ? lg.fill[r] : size;
  }
  c = atomicAdd(&a.ctl->rlog_next, 1u);
  if (c < a.rlog_chunks) {
    a.rlog_range[c] = r;
    lg.chunk[r] = c;
  } else {
    lg.chunk[r] = kEmpty32;
  }
  lg.fill[r] = 0;
}

// Kernel end (after a barrier): close the open chunks.
__device__ __forceinline__ void log_close(const ScanArgs& a, const LogState& lg) {
  const uint32_t r = threadIdx.x;
  if (!a.rlog || r >= a.nranges) return;
  const uint32_t c = lg.chunk[r], size = 1u << a.rlog_chunk_log2;
  if (c < kNoChunk) a.rlog_fill[c] = lg.fill[r] < size ? lg.fill[r] : size;
}

__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t* warp_tot, uint32_t& total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < nw ? warp_tot[lane] : 0u, ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= (uint32_t)o) ti += u;
    }
    if (lane < nw) warp_tot[lane] = ti - t;   // exclusive warp offsets
    if (lane == 31) warp_tot[32] = ti;        // block total
  }
  __syncthreads();
  total = warp_tot[32];
  return warp_tot[warp] + incl - v;
}

// Global-memory loops below take kBatch entries per thread per round, all
// loaded before any is used, so enough loads are in flight to cover memory
// latency with one CTA per SM.
constexpr uint32_t kBatch = 8;
constexpr uint32_t kProbeBatch = 4;
constexpr uint32_t kDead = 0xFFFFFFFDu;  // rank/select chain: a level's bit was clear

// Exact dedupe of src[lo, hi) in a cleared table at the front of the
// shared-memory set, sized to at least twice the entries (at most the whole
// set); each distinct slot is registered once. Fits whenever hi - lo <=
// capacity / 2.
template <bool FIX = false>
__device__ __forceinline__ void insert_range(const ScanArgs& a, const LogState& lg, const uint32_t* src, uint32_t lo, uint32_t hi,
                             uint32_t* sset, unsigned long long& my_regs) {
  const uint32_t tid = threadIdx.x, nthr = blockDim.x;
  uint32_t slog = ceil_log2_u64(2ull * (hi - lo));
  slog = slog < 8u ? 8u : slog;
  slog = slog > a.sset_log2 ? a.sset_log2 : slog;
  const uint32_t cap = 1u << slog;
  for (uint32_t i = tid; i < cap; i += nthr) sset[i] = kEmpty32;
  log_room(a, lg, hi - lo);
  __syncthreads();
  for (uint32_t i0 = lo + tid; i0 < hi; i0 += kBatch * nthr) {
    uint32_t v[kBatch];
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k) v[k] = i0 + k * nthr < hi ? src[i0 + k * nthr] : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k) {
      if (i0 + k * nthr < hi && sset_insert_full(sset, slog, v[k], a.ctl)) {
        ++my_regs;
        register_slot<FIX>(a, lg, v[k]);
      }
    }
  }
  __syncthreads();
}

// Counting-sort src[lo, hi) into dst[lo, hi) by bucket bits (shift, kb);
// bucket b ends up in dst[bnd[b], bnd[b + 1]).
__device__ void partition_range(const uint32_t* src, uint32_t* dst, uint32_t lo, uint32_t hi, uint32_t shift,
                                uint32_t kb, uint32_t* bnd, uint32_t* cur) {
  __shared__ uint32_t s_wt[33];
  const uint32_t tid = threadIdx.x, nthr = blockDim.x, K = 1u << kb;
  for (uint32_t b = tid; b < K; b += nthr) bnd[b] = 0;
  __syncthreads();
  for (uint32_t i0 = lo + tid; i0 < hi; i0 += kBatch * nthr) {
    uint32_t v[kBatch];
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k) v[k] = i0 + k * nthr < hi ? src[i0 + k * nthr] : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k)
      if (i0 + k * nthr < hi) atomicAdd(bnd + spill_bucket(v[k], shift, kb), 1u);
  }
  __syncthreads();
  // bucket starts: each thread scans a run of consecutive buckets
  const uint32_t per = (K + nthr - 1) / nthr, b0 = tid * per, b1 = b0 + per < K ? b0 + per : K;
  uint32_t mine = 0;
  for (uint32_t b = b0; b < b1; ++b) mine += bnd[b];
  uint32_t total = 0;
  uint32_t run = lo + block_excl_sum(mine, s_wt, total);
  __syncthreads();
  for (uint32_t b = b0; b < b1; ++b) {
    const uint32_t c = bnd[b];
    bnd[b] = run;
    cur[b] = run;
    run += c;
  }
  if (tid == 0) bnd[K] = hi;
  __syncthreads();
  for (uint32_t i0 = lo + tid; i0 < hi; i0 += kBatch * nthr) {
    uint32_t v[kBatch];
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k) v[k] = i0 + k * nthr < hi ? src[i0 + k * nthr] : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k)
      if (i0 + k * nthr < hi) dst[atomicAdd(cur + spill_bucket(v[k], shift, kb), 1u)] = v[k];
  }
  __syncthreads();
}

// smallest kb with 4n <= cap * 2^kb (expected distinct per bucket <= cap / 4)
__device__ __forceinline__ uint32_t bucket_bits(uint32_t n, uint32_t cap, uint32_t kbmax) {
  uint32_t kb = 0;
  while (kb < kbmax && ((uint64_t)n << 2) > ((uint64_t)cap << kb)) ++kb;
  return kb;
}

// Counting-sort src[lo, hi) into dst[lo, hi) by the low kb bits of the
// slot's 32-slot word: bucket b holds the slots whose word index is b mod
// 2^kb and ends up in dst[bnd[b], bnd[b + 1]). Interleaving the words over
// the buckets spreads slots that cluster in a few ranges (rank order puts
// the frequent prefixes first) evenly, so no bucket counter is hammered.
__device__ void partition_by_word(const uint32_t* src, uint32_t* dst, uint32_t lo, uint32_t hi, uint32_t kb,
                                  uint32_t* bnd, uint32_t* cur, const uint32_t* counts) {
  __shared__ uint32_t s_wt[33];
  const uint32_t tid = threadIdx.x, nthr = blockDim.x, K = 1u << kb, mask = K - 1u;
  for (uint32_t b = tid; b < K; b += nthr) bnd[b] = counts ? counts[b] : 0u;
  __syncthreads();
  if (!counts) {  // (counted already while the slots were spilled)
    for (uint32_t i0 = lo + tid; i0 < hi; i0 += kBatch * nthr) {
      uint32_t v[kBatch];
#pragma unroll
      for (uint32_t k = 0; k < kBatch; ++k) v[k] = i0 + k * nthr < hi ? src[i0 + k * nthr] : 0u;
#pragma unroll
      for (uint32_t k = 0; k < kBatch; ++k)
        if (i0 + k * nthr < hi) atomicAdd(bnd + ((v[k] >> 5) & mask), 1u);
    }
    __syncthreads();
  }
  const uint32_t per = (K + nthr - 1) / nthr, b0 = tid * per, b1 = b0 + per < K ? b0 + per : K;
  uint32_t mine = 0;
  for (uint32_t b = b0; b < b1; ++b) mine += bnd[b];
  uint32_t total = 0;
  uint32_t run = lo + block_excl_sum(mine, s_wt, total);
  __syncthreads();
  for (uint32_t b = b0; b < b1; ++b) {
    const uint32_t c = bnd[b];
    bnd[b] = run;
    cur[b] = run;
    run += c;
  }
  if (tid == 0) bnd[K] = hi;
  __syncthreads();
  for (uint32_t i0 = lo + tid; i0 < hi; i0 += kBatch * nthr) {
    uint32_t v[kBatch];
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k) v[k] = i0 + k * nthr < hi ? src[i0 + k * nthr] : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k)
      if (i0 + k * nthr < hi) dst[atomicAdd(cur + ((v[k] >> 5) & mask), 1u)] = v[k];
  }
  __syncthreads();
}

// Exact dedupe of src[lo, hi) (the slots of one bucket: word index = b mod
// 2^kb) with a bit vector in shared memory (the per-sequence set's words, all
// zero on entry and on exit): slot v is bit v mod 32 of word v >> (5 + kb);
// the thread that sets a slot's bit registers it. The bits are cleared again
// word by word after use, or all at once when the bucket holds more entries
// than the vector has words.
template <bool FIX = false>
__device__ __forceinline__ void bitmap_bucket(const ScanArgs& a, const LogState& lg, const uint32_t* src, uint32_t lo, uint32_t hi,
                              uint32_t kb, uint32_t* bm, uint32_t bm_words, unsigned long long& my_regs) {
  const uint32_t tid = threadIdx.x, nthr = blockDim.x, ws = 5u + kb;
  if (a.rlog) {
    log_room(a, lg, hi - lo);
    __syncthreads();
  }
  for (uint32_t i0 = lo + tid; i0 < hi; i0 += kBatch * nthr) {
    uint32_t v[kBatch];
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k) v[k] = i0 + k * nthr < hi ? src[i0 + k * nthr] : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kBatch; ++k) {
      if (i0 + k * nthr < hi) {
        const uint32_t bit = 1u << (v[k] & 31u);
        if (!(atomicOr(bm + (v[k] >> ws), bit) & bit)) {
          ++my_regs;
          register_slot<FIX>(a, lg, v[k]);
        }
      }
    }
  }
  __syncthreads();
  if (hi - lo >= bm_words) {
    for (uint32_t i = tid; i < bm_words; i += nthr) bm[i] = 0u;
  } else {
    for (uint32_t i = lo + tid; i < hi; i += nthr) bm[src[i] >> ws] = 0u;
  }
  __syncthreads();
}

// Phase 2 by bit vector: the spilled slots of one sequence (S entries,
// duplicates included, disjoint from the slots already in the set) are
// counting-sorted into K = 2^kb buckets by their 32-slot word index, K just
// large enough that a bucket's slots fit one bit vector in the set's shared
// memory, and each bucket is deduplicated with that bit vector. One
// partition level, no hashing, no probing.
template <bool FIX = false>
__device__ __forceinline__ void dedupe_spills_by_word(const ScanArgs& a, const LogState& lg, uint32_t S, uint32_t kb, uint32_t* sset,
                                      uint32_t* scratch, uint32_t* list, uint32_t* part, const uint32_t* counts,
                                      unsigned long long& my_regs) {
  const uint32_t words = 1u << a.sset_log2, K = 1u << kb;
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) sset[i] = 0u;  // the set becomes the bit vector
  partition_by_word(list, part, 0, S, kb, scratch, scratch + K + 1, counts);
  for (uint32_t b = 0; b < K; ++b) {
    const uint32_t lo = scratch[b], hi = scratch[b + 1];
    if (hi > lo) bitmap_bucket<FIX>(a, lg, part, lo, hi, kb, sset, words, my_regs);  // uniform across the CTA
  }
}

// Phase 2: the spilled slots of one sequence (S entries, duplicates
// included, disjoint from the slots already in the set) are hash-partitioned
// (at most two levels, bucket tables in the free tile buffer) into buckets of
// at most half the set's capacity, and each bucket is deduplicated exactly.
template <bool FIX = false>
__device__ __forceinline__ void dedupe_spills(const ScanArgs& a, const LogState& lg, uint32_t S, uint32_t* sset, uint32_t* scratch,
                              uint32_t scratch_words, uint32_t* list, uint32_t* part,
                              unsigned long long& my_regs, const uint32_t* bucket_counts = nullptr,
                              uint32_t counted_kb = 0xFFFFFFFFu) {
  const uint32_t cap = 1u << a.sset_log2, fit = cap / 2;
  if (S <= fit) {
    insert_range<FIX>(a, lg, list, 0, S, sset, my_regs);
    return;
  }
  if (a.range_dedupe && a.nslots) {
    // buckets: the fewest (a power of two) whose words fit the bit vector
    uint32_t kb = 0;
    while ((a.nslots + 31) / 32 > ((uint64_t)cap << kb)) ++kb;
    // worth its two barriers per bucket once the buckets are well filled
    if (2 * (1ull << kb) + 1 <= scratch_words && ((uint64_t)S >> kb) >= a.range_min_fill) {
      dedupe_spills_by_word<FIX>(a, lg, S, kb, sset, scratch, list, part, kb == counted_kb ? bucket_counts : nullptr,
                            my_regs);
      return;
    }
  }
  const uint32_t half = scratch_words / 2;
  uint32_t kbmax = 0;
  while (kbmax < 12 && (2u << (kbmax + 1)) + 1 <= half) ++kbmax;
  uint32_t* bnd1 = scratch;
  uint32_t* bnd2 = scratch + half;
  const uint32_t kb1 = bucket_bits(S, cap, kbmax) + a.spill_extra_log2 > kbmax
                           ? kbmax : bucket_bits(S, cap, kbmax) + a.spill_extra_log2;
  const uint32_t K1 = 1u << kb1;
  partition_range(list, part, 0, S, 0, kb1, bnd1, bnd1 + K1 + 1);
  for (uint32_t b1 = 0; b1 < K1; ++b1) {
    const uint32_t lo = bnd1[b1], hi = bnd1[b1 + 1];
    if (hi == lo) continue;  // uniform across the CTA
    if (hi - lo <= fit) {
      insert_range<FIX>(a, lg, part, lo, hi, sset, my_regs);
      continue;
    }
    const uint32_t kb2 = bucket_bits(hi - lo, cap, kbmax);
    const uint32_t K2 = 1u << kb2;
    partition_range(part, list, lo, hi, kb1, kb2, bnd2, bnd2 + K2 + 1);
    for (uint32_t b2 = 0; b2 < K2; ++b2) {
      const uint32_t l2 = bnd2[b2], h2 = bnd2[b2 + 1];
      if (h2 > l2) insert_range<FIX>(a, lg, list, l2, h2, sset, my_regs);
    }
  }
}

// V = 0: every switch of ScanArgs read at run time. V = 1..3: Eq. 2 with
// the set and spill lists and 16-bit counters, without carried slots, dense
// map, window runs, registration log, bit vectors or global sets, fixed at
// compile time; V = 1 or 2: prefix ids by V rank/select levels (no hot cache,
// survivors not listed); V = 3: the probe table (or the base pass).
template <int SB, bool BASE, uint32_t V>
__device__ __forceinline__ void scan_body(const ScanArgs& a) {
  constexpr bool kFix = V != 0, kRs = V == 1 || V == 2;
  const uint32_t rs_depth = kRs ? V : (V == 3 ? 0u : a.rs_depth);
  const uint32_t carry_in = kFix ? 0u : a.carry_in, carry_out = kFix ? 0u : a.carry_out;
  uint32_t* const carry = kFix ? nullptr : a.carry;
  const uint32_t hot_log2 = kRs ? 0u : a.hot_log2;
  const uint32_t* const dmap = kFix ? nullptr : a.dmap;
  const uint32_t first_runs = kFix ? 0u : a.first_runs;
  unsigned long long* const list_out = kRs ? nullptr : a.list_out;
  const bool seq_mode = kFix || a.count_mode == IG_COUNT_ONCE_PER_SEQUENCE;
  const uint32_t set_max_windows = kFix ? 0u : a.set_max_windows;
  const uint32_t prefetch_tiles = kFix ? 0u : a.prefetch_tiles;
  uint32_t* const rlog = kFix ? nullptr : a.rlog;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_item, s_nspill, s_qn;
  // spills per bit-vector bucket of the sequence, counted as they are
  // pushed (K = 2^kb buckets of 32-slot words; kb as the dedupe picks it)
  constexpr uint32_t kMaxCountedBuckets = 128;
  __shared__ uint32_t s_bcnt[kMaxCountedBuckets];
  uint32_t spill_kb = 0;
  while ((a.nslots + 31) / 32 > ((uint64_t)1 << (a.sset_log2 + spill_kb))) ++spill_kb;
  const bool count_buckets = a.range_dedupe && (1u << spill_kb) <= kMaxCountedBuckets;
  const uint32_t bmask = (1u << spill_kb) - 1u;
  __shared__ unsigned long long s_run_base[kMaxRuns];
  __shared__ uint32_t s_run_cnt[kMaxRuns];
  __shared__ unsigned long long s_surv, s_regs;
  __shared__ uint32_t s_log_chunk[kLogMaxRanges], s_log_fill[kLogMaxRanges];
  const LogState lg{s_log_chunk, s_log_fill};
  log_init(lg);

  using S = Sym<SB>;
  const uint32_t tid = threadIdx.x, nthr = blockDim.x;
  const uint32_t R = a.words_per_thread * S::kPerWord;  // windows per thread per tile
  const uint32_t tile_windows = R * nthr;
  const uint32_t H = (BASE || hot_log2 == 0) ? 0u : (1u << hot_log2);
  // shared memory: [dedupe set][hot keys][hot ids][tile]
  uint32_t* sset = smem;
  unsigned long long* hot_keys = reinterpret_cast<unsigned long long*>(smem + (1u << a.sset_log2));
  uint32_t* hot_ids = reinterpret_cast<uint32_t*>(hot_keys + H);
  uint32_t* tile0 = hot_ids + H;
  // candidate passes: queue of alive windows (tile-relative indices) and the
  // tile's survivor bits; a second tile buffer at word a.tile2 (0 = none)
  // lets the next tile's bulk copy run while this one is processed
  uint16_t* queue = reinterpret_cast<uint16_t*>(tile0 + a.tile_words);
  uint32_t* tile_alive = tile0 + a.tile_words + a.queue_words;
  uint32_t* const tile1 = a.tile2 ? smem + a.tile2 : tile0;
  __shared__ __align__(8) uint64_t s_bar[2];
  if (tid == 0) {
    mbar_init(&s_bar[0]);
    mbar_init(&s_bar[1]);
  }
  uint32_t bar_phases = 0;  // bit b: phase parity of barrier b
  const uint32_t alive_tile_words = (tile_windows + 31) / 32;
  unsigned long long* gset = (!kFix && a.gset) ? a.gset + ((unsigned long long)blockIdx.x << a.gset_log2) : nullptr;
  uint32_t* bm = (!kFix && a.bitmap) ? a.bitmap + (uint64_t)blockIdx.x * a.bitmap_words : nullptr;
  // CTA-private spill list and partition buffer (Eq. 2 without a global set)
  uint32_t* spill_list = a.spill ? a.spill + (uint64_t)blockIdx.x * 2 * a.spill_cap : nullptr;
  uint32_t* spill_part = spill_list ? spill_list + a.spill_cap : nullptr;
  const uint32_t j = a.j;
  const uint32_t epoch_base = a.ctl->epoch_base;

  // the most frequent candidates, cached in shared memory in front of the table
  for (uint32_t i = tid; i < H; i += nthr) {
    const uint4 e = a.hot[i];
    hot_keys[i] = ((unsigned long long)e.y << 32) | e.x;
    hot_ids[i] = e.z;
  }

  unsigned long long my_surv = 0, my_regs = 0;
  if (tid == 0) { s_surv = 0; s_regs = 0; }
  bool stopped = false;  // a tile wait ran out

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&a.ctl->queue, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= a.m) break;
    const uint32_t seq = a.order[item];
    const uint64_t s0 = a.offsets[seq];
    const uint64_t L = a.offsets[seq + 1] - s0;
    if (L < j) continue;
    const uint64_t W = L - j + 1;
    const uint32_t epoch = epoch_base + seq + 1;
    const uint32_t sprobes = a.set_probes;
    // a sequence this long sends every survivor straight to its spill list
    // (the set would only hold a small share of its slots)
    const bool no_set = set_max_windows && W > set_max_windows;
    uint32_t slog = 0, glog = 0;
    if (seq_mode) {
      uint32_t need = ceil_log2_u64(2 * W);
      slog = need < a.sset_log2 ? need : a.sset_log2;
      if (slog < 1) slog = 1;
      glog = need < a.gset_log2 ? need : a.gset_log2;
      if (glog < 1) glog = 1;
      if (bm) {
        for (uint32_t i = tid; i < a.bitmap_words; i += nthr) bm[i] = 0u;
      } else {
        for (uint32_t i = tid; i < (1u << slog); i += nthr) sset[i] = kEmpty32;
      }
    }
    if (tid == 0) s_nspill = 0;
    if (count_buckets && tid <= bmask) s_bcnt[tid] = 0;

    // tile t of the sequence is in buffer t & 1 (always buffer 0 without a
    // second buffer); tile 0 is issued here, tile t + 1 once tile t arrived
    __syncthreads();  // the previous sequence is done with both buffers
    stage_issue(a, tile_geom<SB>(a, s0, W, 0, tile_windows, j), reinterpret_cast<uint8_t*>(tile0), &s_bar[0]);
    for (uint32_t d = 1; d <= prefetch_tiles; ++d)
      if ((uint64_t)d * tile_windows < W) prefetch_tile(a, tile_geom<SB>(a, s0, W, (uint64_t)d * tile_windows, tile_windows, j));
    uint32_t tix = 0;
    for (uint64_t w0 = 0; w0 < W; w0 += tile_windows, ++tix) {
      const TileGeom g = tile_geom<SB>(a, s0, W, w0, tile_windows, j);
      const uint32_t nwin = g.nwin, sym_off = g.sym_off;
      const uint64_t gsym = g.gsym;
      const uint32_t bsel = a.tile2 ? (tix & 1u) : 0u;
      uint32_t* tile = bsel ? tile1 : tile0;
      const uint32_t parity = (bar_phases >> bsel) & 1u;
      const bool arrived = mbar_wait(s_bar + bsel, parity);
      bar_phases ^= 1u << bsel;
      // (the barrier also makes edge chunks written by other threads visible)
      if (__syncthreads_or(!arrived)) {
        // the tile did not arrive in time: report it, let a copy still in
        // flight land (bounded again) and stop this CTA
        if (tid == 0) {
          atomicOr(&a.ctl->status, kStTimeout);
          if (!a.stall_tiles) mbar_wait(s_bar + bsel, parity);
        }
        stopped = true;
        break;
      }
      if (a.tile2 && w0 + tile_windows < W)
        stage_issue(a, tile_geom<SB>(a, s0, W, w0 + tile_windows, tile_windows, j),
                    reinterpret_cast<uint8_t*>(bsel ? tile0 : tile1), s_bar + (bsel ^ 1u));
      if (prefetch_tiles && w0 + (uint64_t)(prefetch_tiles + 1) * tile_windows < W)
        prefetch_tile(a, tile_geom<SB>(a, s0, W, w0 + (uint64_t)(prefetch_tiles + 1) * tile_windows, tile_windows, j));

      const uint32_t wb = tid * R;
      if (BASE) {
        if (wb < nwin) {
          const uint32_t we = (wb + R) < nwin ? (wb + R) : nwin;
          uint32_t s = sym_off + wb;
          uint32_t widx = s / S::kPerWord, q = s % S::kPerWord;
          uint32_t word = bswap32(tile[widx]);
          uint64_t key = 0;
          const uint32_t total = (we - wb) + j - 1;
          for (uint32_t i = 0; i < total; ++i) {
            const uint32_t sym = (word >> (32 - SB * (q + 1))) & S::kMask;
            if (++q == S::kPerWord) {
              q = 0;
              ++widx;
              word = (widx < a.tile_words) ? bswap32(tile[widx]) : 0u;
            }
            key = ((key << SB) | sym) & a.key_mask;
            if (i + 1 < j) continue;
            const uint32_t slot = (uint32_t)key;
            ++my_surv;
            bool count_it = true;
            if (seq_mode) {
              if (bm) {
                count_it = bitmap_first(bm, slot);
              } else if (spill_list) {
                const int r = no_set ? 2 : sset_try_insert(sset, slog, slot, sprobes);
                count_it = (r == 1);
                if (r == 2) {
                  spill_push(spill_list, &s_nspill, slot);
                  if (count_buckets) atomicAdd(s_bcnt + ((slot >> 5) & bmask), 1u);
                }
              } else {
                count_it = seq_first_seen(sset, slog, gset, glog, epoch, slot, a.ctl);
              }
            }
            if (count_it) {
              ++my_regs;
              count_at_once<kFix>(a, slot);  // the dense base pass never keeps a log
            }
          }
        }
      } else if (first_runs) {
        // first candidate pass: every window is a candidate, so each thread
        // rolls the key over its own run of windows as in the base pass; the
        // (j-1)-gram prefix indexes the dense map, or goes to the hot cache
        // and then the probe table (kProbeBatch loads in flight per thread)
        if (a.alive_out)
          for (uint32_t i = tid; i < alive_tile_words; i += nthr) tile_alive[i] = 0;
        __syncthreads();
        if (wb < nwin) {
          const uint32_t we = (wb + R) < nwin ? (wb + R) : nwin;
          const uint32_t kmask = (uint32_t)a.key_mask;  // j * SB <= 32 here
          uint32_t s = sym_off + wb;
          uint32_t widx = s / S::kPerWord, q = s % S::kPerWord;
          uint32_t word = bswap32(tile[widx]);
          uint32_t key = 0;
#define IG_NEXT_SYM(dst)                                                   \
  do {                                                                     \
    (dst) = (word >> (32 - SB * (q + 1))) & S::kMask;                      \
    if (++q == S::kPerWord) {                                              \
      q = 0;                                                               \
      ++widx;                                                              \
      word = (widx < a.tile_words) ? bswap32(tile[widx]) : 0u;             \
    }                                                                      \
  } while (0)
          for (uint32_t i = 0; i + 1 < j; ++i) {
            uint32_t sym;
            IG_NEXT_SYM(sym);
            key = ((key << SB) | sym) & kmask;
          }
          for (uint32_t w = wb; w < we; w += kProbeBatch) {
            uint32_t kk[kProbeBatch], rk[kProbeBatch], pend = 0;
            uint4 e[kProbeBatch];
#pragma unroll
            for (uint32_t k = 0; k < kProbeBatch; ++k) {
              rk[k] = kEmpty32;
              kk[k] = 0;
              e[k] = make_uint4(0, 0, 0, 0);
              if (w + k < we) {
                uint32_t sym;
                IG_NEXT_SYM(sym);
                key = ((key << SB) | sym) & kmask;
                kk[k] = key;
                const uint32_t prefix = key >> SB;
                if (dmap) {
                  rk[k] = __ldg(dmap + prefix);
                } else {
                  if (H) {
                    const uint32_t h = hash64_top(prefix, hot_log2);
                    if (hot_keys[h] == prefix) rk[k] = hot_ids[h];
                  }
                  if (rk[k] == kEmpty32) {
                    e[k] = __ldg(a.table + hash64_top(prefix, a.table_log2));
                    pend |= 1u << k;
                  }
                }
              }
            }
#pragma unroll
            for (uint32_t k = 0; k < kProbeBatch; ++k) {
              if ((pend >> k) & 1u) rk[k] = probe_from(a.table, a.table_log2, kk[k] >> SB, e[k], a.ctl);
              if (rk[k] == kEmpty32) continue;
              const uint32_t slot = (rk[k] << SB) | (kk[k] & S::kMask);
              const uint32_t wt = w + k;
              if (a.alive_out) atomicOr(tile_alive + (wt >> 5), 1u << (wt & 31));
              ++my_surv;
              bool count_it = true;
              if (seq_mode) {
                if (bm) {
                  count_it = bitmap_first(bm, slot);
                } else if (spill_list) {
                  const int r = no_set ? 2 : sset_try_insert(sset, slog, slot, sprobes);
                  count_it = (r == 1);
                  if (r == 2) {
                  spill_push(spill_list, &s_nspill, slot);
                  if (count_buckets) atomicAdd(s_bcnt + ((slot >> 5) & bmask), 1u);
                }
                } else {
                  count_it = seq_first_seen(sset, slog, gset, glog, epoch, slot, a.ctl);
                }
              }
              if (count_it) {
                ++my_regs;
                register_slot<kFix>(a, lg, slot);
              }
            }
          }
#undef IG_NEXT_SYM
        }
        if (a.alive_out) {
          __syncthreads();
          // tile bit w is corpus bit gsym + w
          const uint32_t off = (uint32_t)(gsym & 31);
          const uint64_t g0 = gsym >> 5;
          const uint32_t nw = (nwin + off + 31) / 32;
          for (uint32_t k = tid; k < nw; k += nthr) {
            const uint32_t cur = k < alive_tile_words ? tile_alive[k] : 0u;
            const uint32_t prev = (k > 0 && off) ? tile_alive[k - 1] : 0u;
            const uint32_t v = off ? ((cur << off) | (prev >> (32 - off))) : cur;
            if (v) atomicOr(a.alive_out + g0 + k, v);
          }
        }
      } else {
        // phase A: every thread walks its run of windows; alive ones are
        // queued (warp-aggregated), so phase B can process them densely
        if (tid == 0) s_qn = 0;
        if (a.alive_out)
          for (uint32_t i = tid; i < alive_tile_words; i += nthr) tile_alive[i] = 0;
        __syncthreads();
        const uint32_t lane = tid & 31;
        if (a.alive_in) {
          // word-parallel: each thread takes whole 32-bit words of the
          // survivor mask (corpus bits gsym .. gsym + nwin - 1), a warp scan
          // places their set bits in the queue
          const uint64_t k0 = gsym >> 5;
          const uint32_t nwords = (uint32_t)(((gsym + nwin - 1) >> 5) - k0 + 1);
          for (uint32_t kb = 0; kb < nwords; kb += nthr) {
            const uint32_t k = kb + tid;
            uint32_t bits = 0;
            if (k < nwords) {
              bits = __ldg(a.alive_in + k0 + k);
              const uint64_t p0 = (k0 + k) << 5;  // corpus bit of bit 0
              if (p0 < gsym) bits &= ~0u << (uint32_t)(gsym - p0);
              const uint64_t end = gsym + nwin;  // first bit past the tile
              if (p0 + 32 > end) bits &= (end - p0 >= 32) ? ~0u : ((1u << (uint32_t)(end - p0)) - 1u);
            }
            const uint32_t c = __popc(bits);
            uint32_t incl = c;
            for (int o = 1; o < 32; o <<= 1) {
              const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= (uint32_t)o) incl += v;
            }
            uint32_t base = 0;
            const uint32_t wsum = __shfl_sync(0xffffffffu, incl, 31);
            if (lane == 31 && wsum) base = atomicAdd(&s_qn, wsum);
            base = __shfl_sync(0xffffffffu, base, 31) + incl - c;
            // tile window of bit b of word k: (k0 + k) * 32 + b - gsym
            const uint32_t wbase = (uint32_t)(((k0 + k) << 5) - gsym);
            while (bits) {
              const uint32_t b = __ffs(bits) - 1;
              bits &= bits - 1;
              queue[base++] = (uint16_t)(wbase + b);
            }
          }
        } else {
          // no survivor mask: every window of the tile is a candidate
          for (uint32_t w = tid; w < nwin; w += nthr) queue[w] = (uint16_t)w;
          if (tid == 0) s_qn = nwin;
        }
        __syncthreads();
        // survivor list for a chain pass next: run r of this tile takes queue
        // entries [r * kRunChunk, (r + 1) * kRunChunk); room is reserved for
        // every candidate up front, survivors are written at once
        const uint32_t qn = s_qn;
        const uint32_t tile_g = a.tile_base[seq] + (uint32_t)(w0 / a.tile_windows);
        const uint32_t nruns = (qn + kRunChunk - 1) / kRunChunk;
        if (list_out) {
          if (tid < nruns) {
            const uint32_t rn = (qn - tid * kRunChunk) < kRunChunk ? qn - tid * kRunChunk : kRunChunk;
            unsigned long long base = atomicAdd(&a.ctl->list_used, (unsigned long long)rn);
            atomicMax(&a.ctl->list_need, base + rn);
            if (base + rn > a.list_cap) {
              atomicOr(&a.ctl->status, kStListFull);
              base = ~0ull;
            }
            s_run_base[tid] = base;
            s_run_cnt[tid] = 0;
          }
          __syncthreads();
        }
        // phase B: probe, count, dedupe the queued windows (in steps of at
        // most chunk / 8 when registrations go to the log)
        const uint32_t step = rlog ? (1u << a.rlog_chunk_log2) >> 3 : (qn ? qn : 1u);
        for (uint32_t q0 = 0; q0 < qn; q0 += step) {
        const uint32_t q1 = qn - q0 < step ? qn : q0 + step;
        if (rlog) {
          log_room(a, lg, q1 - q0);
          __syncthreads();
        }
        // kProbeBatch queued windows per thread per round: the probe-table
        // loads of a round's hot-cache misses are all issued before any is used
        const bool short_key = (j - 1) * SB <= 32;
        for (uint32_t qb = q0 + tid; qb < q1; qb += kProbeBatch * nthr) {
          uint64_t prefix[kProbeBatch];
          uint32_t wl[kProbeBatch], id[kProbeBatch];
          uint4 e[kProbeBatch];
#pragma unroll
          for (uint32_t k = 0; k < kProbeBatch; ++k) {
            const uint32_t qi = qb + k * nthr;
            id[k] = kEmpty32;
            wl[k] = 0xFFFFFFFFu;  // not a window
            prefix[k] = 0;
            uint64_t hp = 0;  // one multiply-shift product for the hot cache and the table
            e[k] = make_uint4(0, 0, 0, 0);
            if (qi < q1) {
              const uint32_t w = queue[qi];
              wl[k] = (w << 8) | tile_sym<SB>(tile, sym_off + w + j - 1);
              if (rs_depth && carry_in) {  // the last level: the window's slot in the previous pass
                prefix[k] = carry[gsym + w];
                const uint2 pe = __ldg(a.rs[rs_depth - 1] + (prefix[k] >> 5));
                e[k] = make_uint4(pe.x, pe.y, 0, 0);
              } else if (rs_depth) {  // level 0: the base-length prefix; its word and the count before it
                prefix[k] = tile_key32<SB>(tile, sym_off + w, a.base_len);
                const uint2 pe = __ldg(a.rs[0] + (prefix[k] >> 5));
                e[k] = make_uint4(pe.x, pe.y, 0, 0);
              } else {
                prefix[k] = short_key ? tile_key32<SB>(tile, sym_off + w, j - 1) : tile_key<SB>(tile, sym_off + w, j - 1);
                hp = prefix[k] * 0x9E3779B97F4A7C15ull;
                if (H) {
                  const uint32_t h = (uint32_t)(hp >> (64 - hot_log2));
                  if (hot_keys[h] == prefix[k]) id[k] = hot_ids[h];
                }
                if (id[k] == kEmpty32) e[k] = __ldg(a.table + (uint32_t)(hp >> (64 - a.table_log2)));
              }
            }
          }
          if (rs_depth) {
            // rank/select chain: the byte-order id of the prefix's first
            // base_len + L symbols at level L is its position among the
            // selected slots of pass base + L (all levels' loads of a round
            // are issued together)
            const uint32_t L0 = carry_in ? rs_depth - 1 : 0;
#pragma unroll
            for (uint32_t L = 0; L < kMaxRsLevels; ++L) {  // levels L0 .. rs_depth - 1
              if (L < L0) continue;
#pragma unroll
              for (uint32_t k = 0; k < kProbeBatch; ++k) {
                if (wl[k] == 0xFFFFFFFFu || id[k] == kDead) continue;
                const uint32_t bit = (uint32_t)prefix[k] & 31u;
                id[k] = ((e[k].x >> bit) & 1u) ? e[k].y + __popc(e[k].x & ((1u << bit) - 1u)) : kDead;
              }
              if (L + 1 >= rs_depth) break;
#pragma unroll
              for (uint32_t k = 0; k < kProbeBatch; ++k) {
                if (wl[k] == 0xFFFFFFFFu || id[k] == kDead) continue;
                const uint32_t w = wl[k] >> 8;
                prefix[k] = ((uint64_t)id[k] << SB) | tile_sym<SB>(tile, sym_off + w + a.base_len + L);
                const uint2 pe = __ldg(a.rs[L + 1] + (prefix[k] >> 5));
                e[k] = make_uint4(pe.x, pe.y, 0, 0);
              }
            }
#pragma unroll
            for (uint32_t k = 0; k < kProbeBatch; ++k)
              if (id[k] == kDead) id[k] = kEmpty32;
          }
#pragma unroll
          for (uint32_t k = 0; k < kProbeBatch; ++k) {
            if (wl[k] == 0xFFFFFFFFu) continue;
            if (!rs_depth && id[k] == kEmpty32) id[k] = probe_from(a.table, a.table_log2, prefix[k], e[k], a.ctl);
            if (id[k] == kEmpty32) continue;
            const uint32_t qi = qb + k * nthr;
            const uint32_t w = wl[k] >> 8, last = wl[k] & 255u;
            const uint32_t slot = (id[k] << SB) | last;
            if (carry_out) carry[gsym + w] = slot;
            if (a.alive_out) atomicOr(tile_alive + (w >> 5), 1u << (w & 31));
            if (list_out) {
              const uint32_t r = qi / kRunChunk;
              if (s_run_base[r] != ~0ull)
                list_out[s_run_base[r] + atomicAdd(s_run_cnt + r, 1u)] =
                    ((unsigned long long)slot << 32) | (uint32_t)(w0 + w);
            }
            ++my_surv;
            bool count_it = true;
            if (seq_mode) {
              if (bm) {
                count_it = bitmap_first(bm, slot);
              } else if (spill_list) {
                const int r = no_set ? 2 : sset_try_insert(sset, slog, slot, sprobes);
                count_it = (r == 1);
                if (r == 2) {
                  spill_push(spill_list, &s_nspill, slot);
                  if (count_buckets) atomicAdd(s_bcnt + ((slot >> 5) & bmask), 1u);
                }
              } else {
                count_it = seq_first_seen(sset, slog, gset, glog, epoch, slot, a.ctl);
              }
            }
            if (count_it) {
              ++my_regs;
              register_slot<kFix>(a, lg, slot);
            }
          }
        }
        if (rlog) __syncthreads();
        }
        if (list_out) {
          __syncthreads();
          if (tid < nruns) {
            const uint32_t run = tile_g * a.runs_per_tile + tid;
            a.list_out_off[run] = s_run_base[tid];
            a.list_out_cnt[run] = s_run_base[tid] == ~0ull ? 0u : s_run_cnt[tid];
          }
        }
        if (a.alive_out) {
          __syncthreads();
          // tile bit w is corpus bit gsym + w
          const uint32_t off = (uint32_t)(gsym & 31);
          const uint64_t g0 = gsym >> 5;
          const uint32_t nw = (nwin + off + 31) / 32;
          for (uint32_t k = tid; k < nw; k += nthr) {
            const uint32_t cur = k < alive_tile_words ? tile_alive[k] : 0u;
            const uint32_t prev = (k > 0 && off) ? tile_alive[k - 1] : 0u;
            const uint32_t v = off ? ((cur << off) | (prev >> (32 - off))) : cur;
            if (v) atomicOr(a.alive_out + g0 + k, v);
          }
        }
      }
      __syncthreads();
      if (!a.tile2 && w0 + tile_windows < W)  // one buffer: stage the next tile now
        stage_issue(a, tile_geom<SB>(a, s0, W, w0 + tile_windows, tile_windows, j),
                    reinterpret_cast<uint8_t*>(tile0), &s_bar[0]);
    }
    if (stopped) break;  // uniform: every thread saw the same barrier result
    if (spill_list && seq_mode) {
      const uint32_t nsp = s_nspill;  // read after the tile loop's final barrier
      if (nsp)
        dedupe_spills<kFix>(a, lg, nsp, sset, tile0, a.tile_words + a.queue_words, spill_list, spill_part, my_regs,
                      count_buckets ? s_bcnt : nullptr, spill_kb);
      __syncthreads();
    }
  }
  // per-CTA statistics
  for (int o = 16; o > 0; o >>= 1) {
    my_surv += __shfl_down_sync(0xffffffffu, my_surv, o);
    my_regs += __shfl_down_sync(0xffffffffu, my_regs, o);
  }
  if ((tid & 31) == 0) {
    atomicAdd(&s_surv, my_surv);
    atomicAdd(&s_regs, my_regs);
  }
  __syncthreads();
  log_close(a, lg);
  if (tid == 0) {
    atomicAdd(&a.ctl->survivors, s_surv);
    atomicAdd(&a.ctl->registrations, s_regs);
  }
}


// Candidate pass j driven by survivor lists. An entry of pass j-1 says that
// window w of the sequence survived pass j-1 with scan slot s; the window's
// (j-1)-gram is in P^(j-1) exactly when s was selected, which the probe table
// (keyed by slot) answers with the counter row of pass j. The last symbol is
// read from the corpus. No tile is staged: work is proportional to the
// survivors of pass j-1, and keys of any length stay exact.
//
// A CTA owns a sequence. Its runs (the run-table entries of all its tiles)
// are taken in chunks: a block scan of the chunk's run sizes turns the runs
// into one index space, each thread takes entries of that space (a binary
// search finds an entry's run), and the chunk's survivors are written as one
// run at the chunk's first index (the others stay empty). Only a few
// barriers per chunk, however few survivors a tile has.
template <int SB, bool BASE>
__global__ void __launch_bounds__(1024) scan_kernel(const ScanArgs a) {
  scan_body<SB, BASE, 0>(a);
}

// Scans of byte corpora under Eq. 2 with the set and spill lists and 16-bit
// counters, with the switches of every other configuration fixed at compile
// time (the same code, fewer branches and live values): scan_rs_kernel<1|2>
// for candidate passes with prefix ids by one or two rank/select levels,
// scan_rs_kernel<3> for candidate passes with the probe table,
// scan_base_kernel for the base pass.
template <uint32_t V>
__global__ void __launch_bounds__(1024) scan_rs_kernel(const ScanArgs a) {
  scan_body<8, false, V>(a);
}
__global__ void __launch_bounds__(1024) scan_base_kernel(const ScanArgs a) {
  scan_body<8, true, 3>(a);
}

// The variant that stands in for scan_kernel with these arguments (0 =
// none: the general kernel runs; 1..3 as scan_body's V).
uint32_t scan_variant(const ScanArgs& a, uint32_t symbol_bits, bool base_pass) {
  if (a.general_only || symbol_bits != 8 || a.carry || a.dmap || a.first_runs || a.rlog || a.bitmap || a.gset ||
      !a.narrow || a.check_overflow || a.count_mode != IG_COUNT_ONCE_PER_SEQUENCE || !a.spill ||
      a.set_max_windows || a.prefetch_tiles)
    return 0;
  if (base_pass || a.rs_depth == 0) return 3;
  return (a.rs_depth <= 2 && !a.hot_log2 && !a.list_out) ? a.rs_depth : 0;
}

template <int SB>
__global__ void __launch_bounds__(1024) chain_kernel(const ScanArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_item, s_nspill, s_out_cnt;
  __shared__ unsigned long long s_surv, s_regs, s_out_base;
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_log_chunk[kLogMaxRanges], s_log_fill[kLogMaxRanges];
  const LogState lg{s_log_chunk, s_log_fill};
  log_init(lg);
  const uint32_t tid = threadIdx.x, nthr = blockDim.x;
  uint32_t* sset = smem;
  uint32_t* scratch = smem + (1u << a.sset_log2);
  const uint32_t scratch_words = a.tile_words + a.queue_words;
  // run chunk in the scratch area: offsets (u64) then exclusive prefix sums
  const uint32_t chunk_runs = (scratch_words - 2) / 3 < nthr ? (scratch_words - 2) / 3 : nthr;
  unsigned long long* c_off = reinterpret_cast<unsigned long long*>(scratch);
  uint32_t* c_pre = scratch + 2 * chunk_runs;
  uint32_t* spill_list = a.spill ? a.spill + (uint64_t)blockIdx.x * 2 * a.spill_cap : nullptr;
  uint32_t* spill_part = spill_list ? spill_list + a.spill_cap : nullptr;
  uint32_t* bm = a.bitmap ? a.bitmap + (uint64_t)blockIdx.x * a.bitmap_words : nullptr;
  const uint32_t j = a.j;
  const uint32_t step = a.rlog ? (1u << a.rlog_chunk_log2) >> 3 : 0xFFFFFFFFu;
  unsigned long long my_surv = 0, my_regs = 0;
  if (tid == 0) { s_surv = 0; s_regs = 0; }

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&a.ctl->queue, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= a.m) break;
    const uint32_t seq = a.order[item];
    const uint64_t s0 = a.offsets[seq];
    const uint64_t L = a.offsets[seq + 1] - s0;
    if (L < j) continue;
    const uint64_t W = L - j + 1;
    const uint32_t sprobes = a.set_probes;
    uint32_t slog = 0;
    if (a.count_mode == IG_COUNT_ONCE_PER_SEQUENCE) {
      const uint32_t need = ceil_log2_u64(2 * W);
      slog = need < a.sset_log2 ? need : a.sset_log2;
      if (slog < 1) slog = 1;
      if (bm) {
        for (uint32_t i = tid; i < a.bitmap_words; i += nthr) bm[i] = 0u;
      } else {
        for (uint32_t i = tid; i < (1u << slog); i += nthr) sset[i] = kEmpty32;
      }
    }
    if (tid == 0) s_nspill = 0;
    // every run-table entry of the sequence's tiles (a fixed range for all passes)
    const uint32_t x0 = a.tile_base[seq] * a.runs_per_tile, x1 = a.tile_base[seq + 1] * a.runs_per_tile;
    __syncthreads();
    for (uint32_t c0 = x0; c0 < x1; c0 += chunk_runs) {
      const uint32_t nr = (x1 - c0) < chunk_runs ? (x1 - c0) : chunk_runs;
      uint32_t cnt = 0;
      if (tid < nr) {
        cnt = a.list_in_cnt[c0 + tid];
        c_off[tid] = a.list_in_off[c0 + tid];
      }
      uint32_t total = 0;
      const uint32_t pre = block_excl_sum(cnt, s_warp, total);
      if (tid < nr) c_pre[tid] = pre;
      if (tid == 0 && a.list_out) {
        unsigned long long base = ~0ull;
        if (total) {
          base = atomicAdd(&a.ctl->list_used, (unsigned long long)total);
          atomicMax(&a.ctl->list_need, base + total);
          if (base + total > a.list_cap) {
            atomicOr(&a.ctl->status, kStListFull);
            base = ~0ull;
          }
        }
        s_out_base = base;
        s_out_cnt = 0;
      }
      __syncthreads();
      for (uint32_t e0 = 0; e0 < total; e0 += step) {
        const uint32_t e1 = total - e0 < step ? total : e0 + step;
        if (a.rlog) {
          log_room(a, lg, e1 - e0);
          __syncthreads();
        }
        // kProbeBatch entries per thread per round: entry, corpus and
        // probe-table loads of a round are issued before any result is used
        for (uint32_t eb = e0 + tid; eb < e1; eb += kProbeBatch * nthr) {
          unsigned long long ent[kProbeBatch];
#pragma unroll
          for (uint32_t k = 0; k < kProbeBatch; ++k) {
            const uint32_t e = eb + k * nthr;
            ent[k] = ~0ull;  // no entry
            if (e < e1) {
              // run of entry e: the last run whose prefix is <= e (it is not empty)
              uint32_t lo = 0, hi = nr;
              while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (c_pre[mid] <= e) lo = mid;
                else hi = mid;
              }
              ent[k] = a.list_in[c_off[lo] + (e - c_pre[lo])];
            }
          }
          uint32_t sym[kProbeBatch];
          uint4 t[kProbeBatch];
#pragma unroll
          for (uint32_t k = 0; k < kProbeBatch; ++k) {
            sym[k] = 0;
            t[k] = make_uint4(0, 0, kEmpty32, 0);
            const uint32_t w = (uint32_t)ent[k];
            if (ent[k] == ~0ull || w >= W) continue;  // the last window of pass j-1 has no j-gram
            const uint64_t pos = s0 + w + j - 1;
            if (SB == 8) {
              sym[k] = __ldg(a.data + pos);
            } else {
              sym[k] = (__ldg(a.data + (pos >> 2)) >> (6 - 2 * (pos & 3))) & 3u;
            }
            t[k] = __ldg(a.table + hash64_top(ent[k] >> 32, a.table_log2));
          }
#pragma unroll
          for (uint32_t k = 0; k < kProbeBatch; ++k) {
            const uint32_t w = (uint32_t)ent[k];
            if (ent[k] == ~0ull || w >= W) continue;
            const uint32_t id = probe_from(a.table, a.table_log2, ent[k] >> 32, t[k], a.ctl);
            if (id == kEmpty32) continue;
            const uint32_t slot = (id << SB) | sym[k];
            ++my_surv;
            if (a.list_out && s_out_base != ~0ull)
              a.list_out[s_out_base + atomicAdd(&s_out_cnt, 1u)] = ((unsigned long long)slot << 32) | w;
            bool count_it = true;
            if (a.count_mode == IG_COUNT_ONCE_PER_SEQUENCE) {
              if (bm) {
                count_it = bitmap_first(bm, slot);
              } else {
                const int rr = sset_try_insert(sset, slog, slot, sprobes);
                count_it = (rr == 1);
                if (rr == 2) spill_push(spill_list, &s_nspill, slot);
              }
            }
            if (count_it) {
              ++my_regs;
              register_slot(a, lg, slot);
            }
          }
        }
        if (a.rlog) __syncthreads();
      }
      __syncthreads();
      if (tid == 0 && a.list_out && total) {
        a.list_out_off[c0] = s_out_base;
        a.list_out_cnt[c0] = s_out_base == ~0ull ? 0u : s_out_cnt;
      }
    }
    if (spill_list && a.count_mode == IG_COUNT_ONCE_PER_SEQUENCE) {
      __syncthreads();
      const uint32_t nsp = s_nspill;
      if (nsp) dedupe_spills(a, lg, nsp, sset, scratch, scratch_words, spill_list, spill_part, my_regs);
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) {
    my_surv += __shfl_down_sync(0xffffffffu, my_surv, o);
    my_regs += __shfl_down_sync(0xffffffffu, my_regs, o);
  }
  if ((tid & 31) == 0) {
    atomicAdd(&s_surv, my_surv);
    atomicAdd(&s_regs, my_regs);
  }
  __syncthreads();
  log_close(a, lg);
  if (tid == 0) {
    atomicAdd(&a.ctl->survivors, s_surv);
    atomicAdd(&a.ctl->registrations, s_regs);
  }
}

// Counting of the registration log, range r: each block takes whole chunks
// of that range and increments their slots' counters (16-byte loads; chunks
// are at least 64 KiB and the pool is 256-byte aligned).
__global__ void __launch_bounds__(512) log_count_kernel(const ScanArgs a, uint32_t r) {
  const uint32_t used = a.ctl->rlog_next < a.rlog_chunks ? a.ctl->rlog_next : a.rlog_chunks;
  for (uint32_t c = blockIdx.x; c < used; c += gridDim.x) {
    if (a.rlog_range[c] != r) continue;  // uniform across the block
    const uint32_t n = a.rlog_fill[c];
    const uint4* e = reinterpret_cast<const uint4*>(a.rlog + ((uint64_t)c << a.rlog_chunk_log2));
    for (uint32_t i = threadIdx.x; 4 * i < n; i += blockDim.x) {
      const uint4 v = __ldcs(e + i);
      const uint32_t b = 4 * i;
      count_at_once(a, v.x);
      if (b + 1 < n) count_at_once(a, v.y);
      if (b + 2 < n) count_at_once(a, v.z);
      if (b + 3 < n) count_at_once(a, v.w);
    }
  }
}

template <int SB, bool BASE>
void* kernel_ptr() {
  return reinterpret_cast<void*>(scan_kernel<SB, BASE>);
}

void* pick(uint32_t symbol_bits, bool base_pass) {
  if (symbol_bits == 8) return base_pass ? kernel_ptr<8, true>() : kernel_ptr<8, false>();
  return base_pass ? kernel_ptr<2, true>() : kernel_ptr<2, false>();
}

}  // namespace

cudaError_t scan_set_smem_limit(uint32_t symbol_bits, bool base_pass, size_t smem) {
  if (symbol_bits == 8) {
    void* const rs[] = {reinterpret_cast<void*>(scan_rs_kernel<1>), reinterpret_cast<void*>(scan_rs_kernel<2>),
                        reinterpret_cast<void*>(scan_rs_kernel<3>)};
    void* const bs[] = {reinterpret_cast<void*>(scan_base_kernel)};
    for (void* f : base_pass ? std::vector<void*>(bs, bs + 1) : std::vector<void*>(rs, rs + 3)) {
      const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaFuncSetAttribute(pick(symbol_bits, base_pass), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

cudaError_t chain_set_smem_limit(uint32_t symbol_bits, size_t smem) {
  void* f = symbol_bits == 8 ? reinterpret_cast<void*>(chain_kernel<8>) : reinterpret_cast<void*>(chain_kernel<2>);
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

void launch_chain(const ScanArgs& a, uint32_t symbol_bits, int grid, int threads, size_t smem, cudaStream_t s) {
  if (symbol_bits == 8) chain_kernel<8><<<grid, threads, smem, s>>>(a);
  else chain_kernel<2><<<grid, threads, smem, s>>>(a);
}

cudaError_t scan_raise_smem_limit(uint32_t symbol_bits, bool base_pass, size_t smem) {
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, pick(symbol_bits, base_pass));
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return scan_set_smem_limit(symbol_bits, base_pass, smem);
}

int scan_max_ctas_per_sm(uint32_t symbol_bits, bool base_pass, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(symbol_bits, base_pass), threads, smem) !=
      cudaSuccess)
    return 0;
  return n;
}

void launch_log_count(const ScanArgs& a, cudaStream_t s) {
  for (uint32_t r = 0; r < a.nranges; ++r) log_count_kernel<<<8 * 152, 512, 0, s>>>(a, r);
}

void launch_scan(const ScanArgs& a, uint32_t symbol_bits, bool base_pass, int grid, int threads,
                 size_t smem, cudaStream_t s) {
  if (symbol_bits == 8) {
    const uint32_t v = scan_variant(a, symbol_bits, base_pass);
    if (v && base_pass) scan_base_kernel<<<grid, threads, smem, s>>>(a);
    else if (v == 1) scan_rs_kernel<1><<<grid, threads, smem, s>>>(a);
    else if (v == 2) scan_rs_kernel<2><<<grid, threads, smem, s>>>(a);
    else if (v == 3) scan_rs_kernel<3><<<grid, threads, smem, s>>>(a);
    else if (base_pass) scan_kernel<8, true><<<grid, threads, smem, s>>>(a);
    else scan_kernel<8, false><<<grid, threads, smem, s>>>(a);
  } else {
    if (base_pass) scan_kernel<2, true><<<grid, threads, smem, s>>>(a);
    else scan_kernel<2, false><<<grid, threads, smem, s>>>(a);
  }
}

}  // namespace ig
