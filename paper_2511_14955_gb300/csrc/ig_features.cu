// The Boolean sequence x feature matrix the paper builds its top-k n-grams
// for (Sec. 1, Fig. 1): entry (i, f) is 1 exactly when sequence i contains
// the f-th n-gram of the final top-k (rows in count-desc, bytes-asc order).
//
// One more pass over the corpus, run twice: a counting scan gives each
// sequence's number of distinct top-k n-grams, a block scan turns those into
// CSR row starts, and a writing scan emits every row's feature ids in
// ascending order. A CTA owns a sequence (longest first, as in the scan);
// the sequence's features are one bit each in a shared-memory bit vector
// (at most 2^20 features), so the ids of a row come out sorted and distinct
// without a sort. Windows are keyed by the same big-endian symbol encoding
// as the scan's and looked up in an open-addressing table of the top-k keys.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ig_internal.cuh"

namespace ig {

namespace {

struct FeatArgs {
  const uint8_t* data;
  uint64_t data_bytes;
  const uint64_t* offsets;
  const uint32_t* order;
  uint32_t m, n;
  uint64_t key_mask;
  const uint4* table;  // {key lo, key hi, feature id, 0}; id kEmpty32 = free
  uint32_t table_log2;
  uint32_t nfeat;
  uint32_t words_per_thread, tile_words;
  uint32_t* queue;          // next sequence (one counter)
  uint32_t* row_nnz;        // counting scan: distinct features of each sequence
  const uint64_t* row_ptr;  // writing scan: CSR row starts
  uint32_t* cols;           // writing scan: feature ids
  uint32_t* status;         // kStTableFull if the table is full (cannot happen at load <= 1/4)
};

__device__ __forceinline__ uint32_t feat_probe(const uint4* __restrict__ table, uint32_t log2, uint64_t key,
                                               uint4 e, uint32_t* status) {
  const uint32_t mask = (1u << log2) - 1u;
  uint32_t h = hash64_top(key, log2);
  const uint32_t lo = (uint32_t)key, hi = (uint32_t)(key >> 32);
  for (uint32_t it = 0; it <= mask; ++it) {
    if (e.z == kEmpty32) return kEmpty32;
    if (e.x == lo && e.y == hi) return e.z;
    h = (h + 1) & mask;
    e = __ldg(table + h);
  }
  atomicOr(status, kStTableFull);
  return kEmpty32;
}

__device__ __forceinline__ uint32_t bswap32f(uint32_t w) { return __byte_perm(w, 0, 0x0123); }

__device__ __forceinline__ uint32_t block_excl_sum32(uint32_t v, uint32_t* warp_tot, uint32_t& total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < nw ? warp_tot[lane] : 0u;
    uint32_t ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= (uint32_t)o) ti += u;
    }
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  total = warp_tot[32];
  const uint32_t r = warp_tot[warp] + incl - v;
  __syncthreads();
  return r;
}

template <int SB, bool WRITE>
__global__ void __launch_bounds__(1024) feature_scan_kernel(const FeatArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_item, s_warp[33];
  constexpr uint32_t kPerWord = 32 / SB, kMask = (1u << SB) - 1u, kBatch = 4;
  const uint32_t tid = threadIdx.x, nthr = blockDim.x;
  const uint32_t nwords = (a.nfeat + 31) / 32;
  uint32_t* bits = smem;                         // one bit per feature
  uint32_t* tile = smem + ((nwords + 3) & ~3u);  // 16-byte aligned
  uint8_t* tile_b = reinterpret_cast<uint8_t*>(tile);
  const uint32_t R = a.words_per_thread * kPerWord, tile_windows = R * nthr, n = a.n;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.queue, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= a.m) break;
    const uint32_t seq = a.order[item];
    const uint64_t s0 = a.offsets[seq];
    const uint64_t L = a.offsets[seq + 1] - s0;
    if (L < n) {
      if (!WRITE && tid == 0) a.row_nnz[seq] = 0;
      continue;
    }
    const uint64_t W = L - n + 1;
    for (uint32_t i = tid; i < nwords; i += nthr) bits[i] = 0u;
    for (uint64_t w0 = 0; w0 < W; w0 += tile_windows) {
      const uint32_t nwin = (uint32_t)((W - w0) < tile_windows ? (W - w0) : tile_windows);
      const uint64_t gsym = s0 + w0;
      const uint64_t nsym = (uint64_t)nwin + n - 1;
      const uint64_t b_first = (gsym * SB) >> 3;
      const uint64_t b_end = ((gsym + nsym) * SB + 7) >> 3;
      const uintptr_t addr_first = reinterpret_cast<uintptr_t>(a.data) + b_first;
      const uintptr_t al = addr_first & ~(uintptr_t)15;
      const uint32_t sym_off = (uint32_t)(addr_first - al) * kPerWord / 4u + (uint32_t)(gsym % (8u / SB));
      const uint32_t nbytes = (uint32_t)((reinterpret_cast<uintptr_t>(a.data) + b_end - al + 15) & ~(uintptr_t)15);
      const uintptr_t lo_ok = reinterpret_cast<uintptr_t>(a.data), hi_ok = lo_ok + a.data_bytes;
      __syncthreads();  // the previous tile's windows are done with the buffer
      for (uint32_t x = tid * 16u; x < nbytes; x += nthr * 16u) {
        const uintptr_t p = al + x;
        uint4 v;
        if (p >= lo_ok && p + 16 <= hi_ok) {
          v = __ldcs(reinterpret_cast<const uint4*>(p));
        } else {
          uint32_t w[4] = {0, 0, 0, 0};
          for (int b = 0; b < 16; ++b) {
            const uintptr_t q = p + b;
            const uint32_t byte = (q >= lo_ok && q < hi_ok) ? *reinterpret_cast<const uint8_t*>(q) : 0u;
            w[b >> 2] |= byte << (8 * (b & 3));
          }
          v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *reinterpret_cast<uint4*>(tile_b + x) = v;
      }
      __syncthreads();
      const uint32_t wb = tid * R;
      if (wb < nwin) {
        const uint32_t we = (wb + R) < nwin ? (wb + R) : nwin;
        const uint32_t s = sym_off + wb;
        uint32_t widx = s / kPerWord, q = s % kPerWord;
        uint32_t word = bswap32f(tile[widx]);
        uint64_t key = 0;
        auto next_sym = [&]() {
          const uint32_t sym = (word >> (32 - SB * (q + 1))) & kMask;
          if (++q == kPerWord) {
            q = 0;
            ++widx;
            word = (widx < a.tile_words) ? bswap32f(tile[widx]) : 0u;
          }
          return sym;
        };
        for (uint32_t i = 0; i + 1 < n; ++i) key = ((key << SB) | next_sym()) & a.key_mask;
        for (uint32_t w = wb; w < we; w += kBatch) {
          uint64_t kk[kBatch];
          uint4 e[kBatch];
#pragma unroll
          for (uint32_t k = 0; k < kBatch; ++k) {
            e[k] = make_uint4(0, 0, kEmpty32, 0);
            kk[k] = 0;
            if (w + k < we) {
              key = ((key << SB) | next_sym()) & a.key_mask;
              kk[k] = key;
              e[k] = __ldg(a.table + hash64_top(key, a.table_log2));
            }
          }
#pragma unroll
          for (uint32_t k = 0; k < kBatch; ++k) {
            if (w + k >= we) continue;
            const uint32_t f = feat_probe(a.table, a.table_log2, kk[k], e[k], a.status);
            if (f != kEmpty32) atomicOr(bits + (f >> 5), 1u << (f & 31));
          }
        }
      }
    }
    __syncthreads();
    // each thread takes a contiguous run of bit-vector words
    const uint32_t per = (nwords + nthr - 1) / nthr, x0 = tid * per, x1 = x0 + per < nwords ? x0 + per : nwords;
    uint32_t mine = 0;
    for (uint32_t x = x0; x < x1; ++x) mine += __popc(bits[x]);
    uint32_t total = 0;
    const uint32_t before = block_excl_sum32(mine, s_warp, total);
    if (!WRITE) {
      if (tid == 0) a.row_nnz[seq] = total;
    } else {
      uint64_t o = a.row_ptr[seq] + before;
      for (uint32_t x = x0; x < x1; ++x) {
        uint32_t v = bits[x];
        while (v) {
          const uint32_t b = __ffs(v) - 1;
          v &= v - 1;
          a.cols[o++] = x * 32 + b;
        }
      }
    }
    __syncthreads();
  }
}

// key of output row r: its first n symbols as one big-endian integer
__global__ void feature_keys_kernel(const uint8_t* rows, uint32_t nrows, uint32_t row_bytes, uint32_t key_bits,
                                    unsigned long long* keys) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    unsigned long long k = 0;
    for (uint32_t b = 0; b < row_bytes; ++b) k = (k << 8) | rows[(size_t)r * row_bytes + b];
    keys[r] = k >> (row_bytes * 8 - key_bits);
  }
}

__global__ void feature_table_kernel(const unsigned long long* keys, uint32_t nrows, uint4* table, uint32_t log2,
                                     uint32_t* status) {
  const uint32_t mask = (1u << log2) - 1u;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    const unsigned long long key = keys[r];
    uint32_t h = hash64_top(key, log2);
    bool placed = false;
    for (uint32_t it = 0; it <= mask && !placed; ++it) {
      if (atomicCAS(&table[h].z, kEmpty32, r) == kEmpty32) {
        table[h].x = (uint32_t)key;
        table[h].y = (uint32_t)(key >> 32);
        placed = true;
      }
      h = (h + 1) & mask;
    }
    if (!placed) atomicOr(status, kStTableFull);
  }
}

__global__ void feature_clear_kernel(uint4* table, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    table[i] = make_uint4(0u, 0u, kEmpty32, 0u);
}

// row_ptr[0] = 0, row_ptr[i + 1] = row_ptr[i] + row_nnz[i] (one block, chunks of blockDim)
__global__ void feature_rowptr_kernel(const uint32_t* row_nnz, uint32_t m, uint64_t* row_ptr) {
  __shared__ uint64_t s_part[1024];
  __shared__ uint64_t s_carry;
  if (threadIdx.x == 0) {
    s_carry = 0;
    row_ptr[0] = 0;
  }
  __syncthreads();
  for (uint32_t c0 = 0; c0 < m; c0 += blockDim.x) {
    const uint32_t i = c0 + threadIdx.x;
    s_part[threadIdx.x] = i < m ? row_nnz[i] : 0u;
    __syncthreads();
    for (uint32_t o = 1; o < blockDim.x; o <<= 1) {  // Hillis-Steele inclusive scan
      const uint64_t t = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0ull;
      __syncthreads();
      s_part[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < m) row_ptr[i + 1] = s_carry + s_part[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry += s_part[threadIdx.x];
    __syncthreads();
  }
}

template <bool WRITE>
void* feature_kernel_ptr(uint32_t sb) {
  return sb == 8 ? reinterpret_cast<void*>(feature_scan_kernel<8, WRITE>)
                 : reinterpret_cast<void*>(feature_scan_kernel<2, WRITE>);
}

}  // namespace

size_t feature_smem_bytes(uint32_t nfeat, uint32_t tile_words) {
  return (size_t)(((nfeat + 31) / 32 + 3) & ~3u) * 4 + (size_t)tile_words * 4;
}

cudaError_t feature_set_smem(uint32_t sb, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(feature_kernel_ptr<false>(sb), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(feature_kernel_ptr<true>(sb), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// The launch sequence of one feature matrix (see intergrams_features): keys
// and table of the `nrows` output rows, the counting scan, the row starts,
// and (when `cols` is set) the writing scan. `queue` is two counters.
void launch_features(const uint8_t* data, uint64_t data_bytes, const uint64_t* offsets, const uint32_t* order,
                     uint32_t m, uint32_t n, uint32_t sb, const uint8_t* rows, uint32_t nrows, uint32_t row_bytes,
                     unsigned long long* keys, uint4* table, uint32_t table_log2, uint32_t* queue, uint32_t* status,
                     uint32_t* row_nnz, uint64_t* row_ptr, uint32_t* cols, bool count, int grid,
                     uint32_t words_per_thread, uint32_t tile_words, size_t smem, cudaStream_t s) {
  FeatArgs a{};
  a.data = data;
  a.data_bytes = data_bytes;
  a.offsets = offsets;
  a.order = order;
  a.m = m;
  a.n = n;
  a.key_mask = (n * sb >= 64) ? ~0ull : ((1ull << (n * sb)) - 1ull);
  a.table = table;
  a.table_log2 = table_log2;
  a.nfeat = nrows;
  a.words_per_thread = words_per_thread;
  a.tile_words = tile_words;
  a.row_nnz = row_nnz;
  a.row_ptr = row_ptr;
  a.cols = cols;
  a.status = status;
  if (count) {
    feature_keys_kernel<<<256, 256, 0, s>>>(rows, nrows, row_bytes, n * sb, keys);
    const uint32_t tn = 1u << table_log2;
    feature_clear_kernel<<<(tn + 255) / 256 < 4096 ? (tn + 255) / 256 : 4096, 256, 0, s>>>(table, tn);
    feature_table_kernel<<<256, 256, 0, s>>>(keys, nrows, table, table_log2, status);
    a.queue = queue;
    if (m) {
      if (sb == 8) feature_scan_kernel<8, false><<<grid, 1024, smem, s>>>(a);
      else feature_scan_kernel<2, false><<<grid, 1024, smem, s>>>(a);
    }
    feature_rowptr_kernel<<<1, 1024, 0, s>>>(row_nnz, m, row_ptr);
  }
  if (cols && m) {
    a.queue = queue + 1;
    if (sb == 8) feature_scan_kernel<8, true><<<grid, 1024, smem, s>>>(a);
    else feature_scan_kernel<2, true><<<grid, 1024, smem, s>>>(a);
  }
}

}  // namespace ig
