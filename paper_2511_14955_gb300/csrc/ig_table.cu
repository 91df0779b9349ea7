// Candidate set P^(j) and result rows.
//
// After the selection of pass j the chosen slots are in slot order, which is
// the byte order of the j-grams; their rank r becomes the id of the j-gram in
// P^(j). Its key is rebuilt from the parent (j-1)-gram key and the last
// symbol: key_j = key_{j-1}[slot / sigma] * sigma + slot % sigma (for the
// dense base pass the slot is the j-gram itself). Keys are right-aligned
// integers of j * symbol_bits <= 64 bits, so integer order is byte order.
//
// The next scan counts in rank space (candidates renumbered by count, hottest
// first, so the counters it hits most are packed together): the probe table
// maps a key to its rank: open addressing with linear probing
// over 16-byte entries {key low, key high, id, 0}, multiply-shift hashed,
// kept at or below the configured load so that lookups (one per window in the
// next scan) touch about one 32-byte sector.
#include "ig_internal.cuh"

namespace ig {

namespace {

__global__ void table_clear_kernel(uint4* table, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    table[i] = make_uint4(0u, 0u, kEmpty32, 0u);
}

__device__ __forceinline__ unsigned long long key_of_slot(uint32_t slot, const unsigned long long* keys_prev,
                                                          bool from_base, uint32_t sb) {
  if (from_base) return slot;
  return (keys_prev[slot >> sb] << sb) | (slot & ((1u << sb) - 1u));
}

__global__ void keys_kernel(const uint32_t* sel_slot, const PassCtl* ctl, const unsigned long long* keys_prev,
                            bool from_base, uint32_t sb, unsigned long long* keys_next) {
  const uint32_t n = ctl->nsel;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    keys_next[r] = key_of_slot(sel_slot[r], keys_prev, from_base, sb);
}

__global__ void build_kernel(const unsigned long long* keys, const uint32_t* rank, const PassCtl* ctl, uint4* table,
                             uint32_t log2, PassCtl* ctl_w) {
  const uint32_t n = ctl->nsel, mask = (1u << log2) - 1u;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const unsigned long long key = keys[r];
    const uint32_t val = rank[r];
    uint32_t h = hash64_top(key, log2);
    bool placed = false;
    for (uint32_t it = 0; it <= mask; ++it) {
      uint32_t* idp = &table[h].z;
      if (atomicCAS(idp, kEmpty32, val) == kEmpty32) {
        table[h].x = (uint32_t)key;
        table[h].y = (uint32_t)(key >> 32);
        placed = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (!placed) atomicOr(&ctl_w->status, kStTableFull);
  }
}

// Row r of the top-k of pass j. The selection of every pass is kept in byte
// order (sel_hist), and slot = id * sigma + last symbol with id the parent's
// position in the previous selection, so the j symbols are recovered by
// walking back to the dense base pass, whose slot is the base_n-gram itself.
__global__ void write_topk_kernel(const uint32_t* sel_hist, uint64_t Z, uint32_t b, const uint32_t* sel_count,
                                  const uint32_t* order, const PassCtl* ctl, uint32_t sb, uint32_t j,
                                  uint32_t row_bytes, uint32_t cap, uint8_t* keys_out,
                                  unsigned long long* counts_out) {
  const uint32_t n = min(ctl->nsel, cap);
  const uint32_t mask = (1u << sb) - 1u;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const uint32_t e = order[r];
    counts_out[r] = sel_count[e];
    uint8_t* row = keys_out + (size_t)r * row_bytes;
    for (uint32_t x = 0; x < row_bytes; ++x) row[x] = 0;
    uint32_t slot = sel_hist[(uint64_t)(j - b) * Z + e];
    for (uint32_t jj = j; jj > b; --jj) {
      const uint32_t p = jj - 1, sym = slot & mask;   // symbol position p (0-based)
      if (sb == 8) row[p] = (uint8_t)sym;
      else row[p >> 2] |= (uint8_t)(sym << (6 - 2 * (p & 3)));
      slot = sel_hist[(uint64_t)(jj - 1 - b) * Z + (slot >> sb)];
    }
    for (uint32_t p = 0; p < b; ++p) {
      const uint32_t sym = (slot >> (sb * (b - 1 - p))) & mask;
      if (sb == 8) row[p] = (uint8_t)sym;
      else row[p >> 2] |= (uint8_t)(sym << (6 - 2 * (p & 3)));
    }
  }
}

// Chain keys of P^(j): the scan slot (rank space of pass j) of each selected
// j-gram, i.e. what pass j wrote into its survivor lists.
__global__ void chain_keys_kernel(const uint32_t* sel_slot, const PassCtl* ctl, const uint32_t* rank_prev,
                                  bool from_base, uint32_t sb, unsigned long long* keys_out) {
  const uint32_t n = ctl->nsel;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const uint32_t s = sel_slot[r];
    keys_out[r] = from_base ? s : (((uint64_t)rank_prev[s >> sb] << sb) | (s & ((1u << sb) - 1u)));
  }
}

// Hot cache of P^(j): a direct-mapped table in which each bucket keeps the
// candidate with the highest count (lowest id on ties) among those hashing
// to it. It only caches exact (key, id) pairs, so its content never changes
// a result.
__global__ void hot_clear_kernel(uint4* hot, unsigned long long* pick, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    hot[i] = make_uint4(0u, 0u, kEmpty32, 0u);
    pick[i] = 0ull;
  }
}

__global__ void hot_pick_kernel(const unsigned long long* keys, const uint32_t* sel_count, const PassCtl* ctl,
                                unsigned long long* pick, uint32_t log2) {
  const uint32_t n = ctl->nsel;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const uint32_t h = hash64_top(keys[r], log2);
    atomicMax(pick + h, ((unsigned long long)sel_count[r] << 32) | (0xFFFFFFFFu - r));
  }
}

__global__ void hot_fill_kernel(const unsigned long long* keys, const uint32_t* rank,
                                const unsigned long long* pick, uint4* hot, uint32_t n) {
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
    const unsigned long long v = pick[h];
    if (!v) continue;
    const uint32_t r = 0xFFFFFFFFu - (uint32_t)v;
    const unsigned long long key = keys[r];
    hot[h] = make_uint4((uint32_t)key, (uint32_t)(key >> 32), rank[r], (uint32_t)(v >> 32));
  }
}

}  // namespace

void launch_build_hot(const unsigned long long* keys, const uint32_t* sel_count, const uint32_t* rank,
                      const PassCtl* ctl, uint4* hot, unsigned long long* hot_pick, uint32_t hot_log2,
                      cudaStream_t s) {
  const uint32_t n = 1u << hot_log2;
  const int g = (int)((n + 255) / 256);
  hot_clear_kernel<<<g, 256, 0, s>>>(hot, hot_pick, n);
  hot_pick_kernel<<<512, 256, 0, s>>>(keys, sel_count, ctl, hot_pick, hot_log2);
  hot_fill_kernel<<<g, 256, 0, s>>>(keys, rank, hot_pick, hot, n);
}

void launch_build_keys(const uint32_t* sel_slot, const PassCtl* ctl, const unsigned long long* keys_prev,
                       bool from_base, uint32_t symbol_bits, unsigned long long* keys_next, cudaStream_t s) {
  keys_kernel<<<1024, 256, 0, s>>>(sel_slot, ctl, keys_prev, from_base, symbol_bits, keys_next);
}

void launch_build_table(const unsigned long long* keys, const uint32_t* rank, const PassCtl* ctl, uint4* table,
                        uint32_t table_log2, cudaStream_t s) {
  const uint32_t n = 1u << table_log2;
  table_clear_kernel<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(table, n);
  build_kernel<<<1024, 256, 0, s>>>(keys, rank, ctl, table, table_log2, const_cast<PassCtl*>(ctl));
}

void launch_write_topk(const uint32_t* sel_hist, uint64_t Z, uint32_t b, const uint32_t* sel_count,
                       const uint32_t* order, const PassCtl* ctl, uint32_t symbol_bits, uint32_t j,
                       uint32_t row_bytes, uint32_t cap, uint8_t* keys_out, unsigned long long* counts_out,
                       cudaStream_t s) {
  write_topk_kernel<<<256, 256, 0, s>>>(sel_hist, Z, b, sel_count, order, ctl, symbol_bits, j, row_bytes, cap,
                                        keys_out, counts_out);
}

void launch_chain_keys(const uint32_t* sel_slot, const PassCtl* ctl, const uint32_t* rank_prev, bool from_base,
                       uint32_t symbol_bits, unsigned long long* keys_out, cudaStream_t s) {
  chain_keys_kernel<<<1024, 256, 0, s>>>(sel_slot, ctl, rank_prev, from_base, symbol_bits, keys_out);
}

namespace {
__global__ void dmap_fill_kernel(const uint32_t* sel_slot, const PassCtl* ctl, const uint32_t* rank, uint32_t* dmap) {
  const uint32_t n = ctl->nsel;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dmap[sel_slot[i]] = rank[i];
}
}  // namespace

void launch_build_dmap(const uint32_t* sel_slot, const PassCtl* ctl, const uint32_t* rank, uint32_t* dmap,
                       uint64_t entries, cudaStream_t s) {
  cudaMemsetAsync(dmap, 0xFF, entries * sizeof(uint32_t), s);
  dmap_fill_kernel<<<1024, 256, 0, s>>>(sel_slot, ctl, rank, dmap);
}

namespace {
__global__ void pbits_clear_kernel(uint2* pbits, uint32_t words) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
    pbits[i] = make_uint2(0u, 0u);
}
__global__ void pbits_set_kernel(const uint32_t* sel_slot, const PassCtl* ctl, uint2* pbits) {
  const uint32_t n = ctl->nsel;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t s = sel_slot[i];
    atomicOr(&pbits[s >> 5].x, 1u << (s & 31));
  }
}
// block b of 1024 words: exclusive prefix of popcounts within the block into
// .y, the block's total to sums[b]
__global__ void pbits_scan_blocks_kernel(uint2* pbits, uint32_t words, uint32_t* sums) {
  __shared__ uint32_t sh[1024];
  const uint32_t i = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t v = i < words ? __popc(pbits[i].x) : 0u;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (uint32_t o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
    const uint32_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < words) pbits[i].y = sh[threadIdx.x] - v;
  if (threadIdx.x == 1023) sums[blockIdx.x] = sh[1023];
}
// one block: exclusive scan of the block totals, 1024 at a time with a carry
__global__ void pbits_scan_sums_kernel(uint32_t* sums, uint32_t nblocks) {
  __shared__ uint32_t sh[1024];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < nblocks; c0 += 1024) {
    const uint32_t i = c0 + threadIdx.x;
    const uint32_t v = i < nblocks ? sums[i] : 0u;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {
      const uint32_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nblocks) sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
}
__global__ void pbits_add_kernel(uint2* pbits, uint32_t words, const uint32_t* sums) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
    pbits[i].y += sums[i / 1024];
}
}  // namespace

void launch_build_pbits(const uint32_t* sel_slot, const PassCtl* ctl, uint2* pbits, uint32_t words,
                        uint32_t* block_sums, cudaStream_t s) {
  const uint32_t nb = (words + 1023) / 1024;
  pbits_clear_kernel<<<1024, 256, 0, s>>>(pbits, words);
  pbits_set_kernel<<<1024, 256, 0, s>>>(sel_slot, ctl, pbits);
  pbits_scan_blocks_kernel<<<nb, 1024, 0, s>>>(pbits, words, block_sums);
  pbits_scan_sums_kernel<<<1, 1024, 0, s>>>(block_sums, nb);
  pbits_add_kernel<<<1024, 256, 0, s>>>(pbits, words, block_sums);
}

}  // namespace ig
