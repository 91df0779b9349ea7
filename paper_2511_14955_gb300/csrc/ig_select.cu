// Deterministic top-T selection over the dense slot counters (paper
// Algorithm 3: "zk-argmax" after each pass and the final "k-argmax").
//
// Order: count descending, then slot ascending. Slot order is the byte order
// of the n-grams (ids of P^(j-1) are assigned in byte order and
// slot = id * sigma + symbol), so this is the count-then-bytes order.
//
//   1. max / nonzero pass over the counters;
//   2. threshold search: successive 4096-bin histograms over a shrinking
//      count range find t = the T-th largest count (each level is one pass;
//      levels beyond the first are skipped on the device once t is exact);
//   3. stable compaction in slot order of every counter with count > t plus
//      the first (T - #greater) counters with count == t.
// The selected entries therefore come out in slot order, which is exactly
// the id order the next pass needs. The final top-k is then put in rank
// order by a stable LSD radix sort on the count (descending).
//
// Every size is read from device memory, so the launch sequence is fixed and
// can be captured in a CUDA graph.
#include <algorithm>

#include "ig_internal.cuh"

namespace ig {

namespace {

constexpr int kThreads = 256;

// Start of a pass: empty the work queue and statistics and advance the
// dedupe epochs by m (one epoch per sequence). When the 32-bit epochs would
// wrap, the dedupe sets are cleared and the epochs restart.
__global__ void pass_reset_kernel(PassCtl* ctl, uint32_t m) {
  if (threadIdx.x == 0) {
    ctl->queue = 0;
    ctl->survivors = 0;
    ctl->registrations = 0;
    ctl->list_used = 0;
    ctl->rlog_next = 0;
    uint64_t e = ctl->epoch_next;
    if (e + m + 1 > 0xFFFFFFFFull) {
      ctl->gset_clear = 1;
      e = 0;
    }
    ctl->epoch_base = (uint32_t)e;
    ctl->epoch_next = (uint32_t)(e + m);
  }
}

__global__ void gset_clear_kernel(PassCtl* ctl, unsigned long long* gset, uint64_t n) {
  if (!ctl->gset_clear) return;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    gset[i] = 0ull;
}

__global__ void gset_clear_done_kernel(PassCtl* ctl) {
  if (threadIdx.x == 0) ctl->gset_clear = 0;
}

__global__ void sel_reset_kernel(PassCtl* ctl, uint32_t target, uint32_t* hist) {
  for (int i = threadIdx.x; i < kMaxLevels * kHistBins; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) {
    ctl->target = target;
    ctl->max_count = 0;
    ctl->nonzero = 0;
    ctl->lo = 1;
    ctl->hi = 0;
    ctl->above = 0;
    ctl->done = 0;
    ctl->thr = 0;
    ctl->need_eq = 0;
    ctl->nsel = 0;
    ctl->take_all = 0;
  }
}

// Counters are read in units of U consecutive byte-order slots with one
// vector load: U = 8, or 4 where a rank map splits an 8-slot group (sigma = 4).
// A unit starting at byte-order slot s0 (a multiple of U) lives at
// rank[s0 >> sb] * sigma + (s0 & (sigma - 1)) in rank space (at s0 without a
// rank map). Slots at or past ns read as 0.
__device__ __forceinline__ uint32_t unit_size(const uint32_t* rank, uint32_t sb) { return (rank && sb < 3) ? 4u : 8u; }

__device__ __forceinline__ void load_unit(const uint32_t* __restrict__ c, bool narrow,
                                          const uint32_t* __restrict__ rank, uint32_t sb, uint64_t ns,
                                          uint64_t s0, uint32_t U, uint32_t v[8]) {
  const uint64_t loc = rank ? (((uint64_t)__ldg(rank + (s0 >> sb)) << sb) | (s0 & ((1u << sb) - 1u))) : s0;
  uint32_t w[4];
  if (narrow) {
    const uint16_t* c16 = reinterpret_cast<const uint16_t*>(c) + loc;
    if (U == 8) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(c16));
      w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
    } else {
      const uint2 q = __ldcs(reinterpret_cast<const uint2*>(c16));
      w[0] = q.x; w[1] = q.y; w[2] = 0; w[3] = 0;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      v[2 * e] = w[e] & 0xFFFFu;
      v[2 * e + 1] = w[e] >> 16;
    }
  } else {
    const uint4 q = __ldcs(reinterpret_cast<const uint4*>(c + loc));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    if (U == 8) {
      const uint4 r = __ldcs(reinterpret_cast<const uint4*>(c + loc + 4));
      v[4] = r.x; v[5] = r.y; v[6] = r.z; v[7] = r.w;
    } else {
      v[4] = v[5] = v[6] = v[7] = 0;
    }
  }
#pragma unroll
  for (int e = 0; e < 8; ++e)
    if ((uint32_t)e >= U || s0 + e >= ns) v[e] = 0;
}

__global__ void max_nonzero_kernel(const uint32_t* __restrict__ c, bool narrow, const uint32_t* __restrict__ rank,
                                   uint32_t sb, uint64_t ns, PassCtl* ctl) {
  const uint32_t U = unit_size(rank, sb);
  const uint64_t nu = (ns + U - 1) / U;
  uint32_t mx = 0, nz = 0;
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < nu; u += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v[8];
    load_unit(c, narrow, rank, sb, ns, u * U, U, v);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      mx = v[e] > mx ? v[e] : mx;
      nz += v[e] != 0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    nz += __shfl_down_sync(0xffffffffu, nz, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (mx) atomicMax(&ctl->max_count, mx);
    if (nz) atomicAdd(&ctl->nonzero, nz);
  }
}

// Decide whether a threshold search is needed and set its first range.
__global__ void threshold_init_kernel(PassCtl* ctl) {
  if (threadIdx.x != 0) return;
  if (ctl->nonzero <= ctl->target) {
    ctl->take_all = 1;
    ctl->done = 1;
    ctl->thr = 0;      // every nonzero counter has count > 0
    ctl->need_eq = 0;
    ctl->nsel = ctl->nonzero;
    return;
  }
  ctl->lo = 1;
  ctl->hi = ctl->max_count;
  ctl->above = 0;
}

__device__ __forceinline__ uint32_t level_shift(uint32_t lo, uint32_t hi) {
  uint64_t span = (uint64_t)hi - lo + 1;
  uint32_t l = ceil_log2_u64(span);
  return l > 12 ? l - 12 : 0;
}

__global__ void level_hist_kernel(const uint32_t* __restrict__ c, bool narrow, const uint32_t* __restrict__ rank,
                                  uint32_t sb, uint64_t ns, PassCtl* ctl, uint32_t* hist) {
  __shared__ uint32_t sh[kHistBins];
  if (ctl->done) return;
  const uint32_t lo = ctl->lo, hi = ctl->hi, sh_bits = level_shift(lo, hi);
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t U = unit_size(rank, sb);
  const uint64_t nu = (ns + U - 1) / U;
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < nu; u += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v[8];
    load_unit(c, narrow, rank, sb, ns, u * U, U, v);
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (v[e] >= lo && v[e] <= hi) atomicAdd(sh + ((v[e] - lo) >> sh_bits), 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
    if (sh[i]) atomicAdd(hist + i, sh[i]);
}

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_tot, uint32_t& total) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = lane < nw ? warp_tot[lane] : 0;
    uint32_t s = t;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= (uint32_t)o) s += y;
    }
    if (lane < nw) warp_tot[lane] = s - t;   // exclusive warp offsets
    if (lane == 31) warp_tot[32] = s;        // block total
  }
  __syncthreads();
  uint32_t r = warp_tot[wid] + x - v;
  total = warp_tot[32];
  __syncthreads();
  return r;
}

// Find the bin holding the target-th largest count and narrow the range (one
// block of kHistBins / 4 threads, four bins each, bins counted from the top).
__global__ void level_pick_kernel(PassCtl* ctl, uint32_t* hist) {
  __shared__ uint32_t wt[33];
  if (ctl->done) return;
  const uint32_t lo = ctl->lo, hi = ctl->hi, sh_bits = level_shift(lo, hi);
  const uint32_t nb = (uint32_t)((((uint64_t)hi - lo) >> sh_bits) + 1);
  const uint32_t T = ctl->target;
  const uint64_t above = ctl->above;
  const uint32_t b0 = 4 * threadIdx.x;
  uint32_t h[4], mine = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    h[e] = b0 + e < nb ? hist[b0 + e] : 0u;
    mine += h[e];
  }
  uint32_t total = 0;
  const uint32_t before = block_excl_scan(mine, wt, total);
  uint64_t cum = above + (total - before - mine);  // counts in the bins above this thread's
  for (int e = 3; e >= 0; --e) {
    const uint32_t b = b0 + e;
    if (b < nb && cum < T && cum + h[e] >= T) {
      const uint64_t nlo = (uint64_t)lo + ((uint64_t)b << sh_bits);
      uint64_t nhi = nlo + (1ull << sh_bits) - 1;
      if (nhi > hi) nhi = hi;
      ctl->lo = (uint32_t)nlo;
      ctl->hi = (uint32_t)nhi;
      ctl->above = (uint32_t)cum;
      if (sh_bits == 0) {
        ctl->done = 1;
        ctl->thr = (uint32_t)nlo;
        ctl->need_eq = T - (uint32_t)cum;
        ctl->nsel = T;
      }
    }
    cum += h[e];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (b0 + e < nb) hist[b0 + e] = 0;  // ready for the next level
}

// Stable compaction, phase 1: per-block numbers of counters > thr and == thr;
// block b takes units [b * chunk, (b + 1) * chunk).
__global__ void compact_count_kernel(const uint32_t* __restrict__ c, bool narrow, const uint32_t* __restrict__ rank,
                                     uint32_t sb, uint64_t ns, const PassCtl* ctl, uint32_t* blk, uint64_t chunk) {
  const uint32_t thr = ctl->thr;
  const bool eq_used = !ctl->take_all;
  const uint32_t U = unit_size(rank, sb);
  const uint64_t nu = (ns + U - 1) / U;
  const uint64_t u0 = blockIdx.x * chunk, u1 = min(nu, u0 + chunk);
  uint32_t gt = 0, eq = 0;
  for (uint64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    uint32_t v[8];
    load_unit(c, narrow, rank, sb, ns, u * U, U, v);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      gt += v[e] > thr;
      eq += eq_used && v[e] == thr && v[e] != 0;
    }
  }
  __shared__ uint32_t s_gt, s_eq;
  if (threadIdx.x == 0) { s_gt = 0; s_eq = 0; }
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) {
    gt += __shfl_down_sync(0xffffffffu, gt, o);
    eq += __shfl_down_sync(0xffffffffu, eq, o);
  }
  if ((threadIdx.x & 31) == 0) { atomicAdd(&s_gt, gt); atomicAdd(&s_eq, eq); }
  __syncthreads();
  if (threadIdx.x == 0) {
    blk[2 * blockIdx.x] = s_gt;
    blk[2 * blockIdx.x + 1] = s_eq;
  }
}

// Phase 2: exclusive scan of the per-block numbers (one block).
__global__ void compact_scan_kernel(uint32_t* blk, int G) {
  __shared__ uint32_t s_gt[1024], s_eq[1024];
  // G <= 1024 * per; each thread owns a contiguous run of blocks
  const int per = (G + blockDim.x - 1) / blockDim.x;
  const int a = threadIdx.x * per, b = min(G, a + per);
  uint32_t gt = 0, eq = 0;
  for (int i = a; i < b; ++i) { gt += blk[2 * i]; eq += blk[2 * i + 1]; }
  s_gt[threadIdx.x] = gt;
  s_eq[threadIdx.x] = eq;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t rg = 0, re = 0;
    for (unsigned t = 0; t < blockDim.x; ++t) {
      uint32_t x = s_gt[t], y = s_eq[t];
      s_gt[t] = rg; s_eq[t] = re;
      rg += x; re += y;
    }
  }
  __syncthreads();
  uint32_t rg = s_gt[threadIdx.x], re = s_eq[threadIdx.x];
  for (int i = a; i < b; ++i) {
    uint32_t x = blk[2 * i], y = blk[2 * i + 1];
    blk[2 * i] = rg; blk[2 * i + 1] = re;
    rg += x; re += y;
  }
}

// Phase 3: write the selected (slot, count) pairs in slot order. A slot is
// taken if its count is > thr, or == thr and it is among the first need_eq
// such slots; its position is (taken slots before it).
__global__ void compact_write_kernel(const uint32_t* __restrict__ c, bool narrow, const uint32_t* __restrict__ rank,
                                     uint32_t sb, uint64_t ns, const PassCtl* ctl, const uint32_t* blk, uint64_t chunk,
                                     uint32_t* sel_slot, uint32_t* sel_count) {
  __shared__ uint32_t wt[33];
  const uint32_t thr = ctl->thr, need = ctl->need_eq;
  const bool eq_used = !ctl->take_all;
  const uint32_t U = unit_size(rank, sb);
  const uint64_t nu = (ns + U - 1) / U;
  const uint64_t u0 = blockIdx.x * chunk, u1 = min(nu, u0 + chunk);
  uint32_t base_gt = blk[2 * blockIdx.x], base_eq = blk[2 * blockIdx.x + 1];
  for (uint64_t t0 = u0; t0 < u1; t0 += blockDim.x) {
    const uint64_t u = t0 + threadIdx.x;
    uint32_t v[8];
    uint32_t ng = 0, ne = 0;
    if (u < u1) {
      load_unit(c, narrow, rank, sb, ns, u * U, U, v);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        ng += v[e] > thr;
        ne += eq_used && v[e] == thr && v[e] != 0;
      }
    }
    // at most 8 per thread and 8 * blockDim in all: both fit 16 bits
    uint32_t tot = 0;
    const uint32_t ex = block_excl_scan((ng << 16) | ne, wt, tot);
    if (ng | ne) {
      uint32_t lg = base_gt + (ex >> 16), le = base_eq + (ex & 0xFFFFu);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const bool g = v[e] > thr;
        const bool q = eq_used && v[e] == thr && v[e] != 0;
        if (g || (q && le < need)) {
          const uint32_t pos = lg + (le < need ? le : need);
          sel_slot[pos] = (uint32_t)(u * U + e);
          sel_count[pos] = v[e];
        }
        lg += g;
        le += q;
      }
    }
    base_gt += tot >> 16;
    base_eq += tot & 0xFFFFu;
  }
}

// ----------------------------------------------------- stable radix sort

// key = ~count (16-bit keys: 0xFFFF - count, counts < 65536), so ascending
// key order is descending count order
__global__ void sort_init_kernel(const uint32_t* sel_count, const PassCtl* ctl, uint32_t key_bits, uint32_t* key,
                                 uint32_t* idx) {
  const uint32_t n = ctl->nsel;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    key[i] = key_bits == 16 ? 0xFFFFu - sel_count[i] : ~sel_count[i];
    idx[i] = i;
  }
}

__global__ void sort_hist_kernel(const uint32_t* key, const PassCtl* ctl, uint32_t shift, uint32_t* hist, int G) {
  __shared__ uint32_t h[kSortDigits];
  const uint32_t n = ctl->nsel;
  for (int i = threadIdx.x; i < kSortDigits; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t a = blockIdx.x * kSortChunk, b = min(n, a + kSortChunk);
  for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x) atomicAdd(h + ((key[i] >> shift) & 255u), 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kSortDigits; d += blockDim.x) hist[d * G + blockIdx.x] = h[d];
}

// Exclusive scan of hist (digit-major: hist[d * G + g]) in two steps: block d
// scans row d in place and leaves the row total at hist[256 * G + d]; then the
// 256 totals are scanned in place into digit bases.
__global__ void sort_scan_rows_kernel(uint32_t* hist, int G) {
  __shared__ uint32_t wt[33];
  uint32_t* row = hist + (size_t)blockIdx.x * G;
  uint32_t run = 0;
  for (int g0 = 0; g0 < G; g0 += blockDim.x) {
    const int g = g0 + threadIdx.x;
    const uint32_t v = g < G ? row[g] : 0u;
    uint32_t tot = 0;
    const uint32_t ex = block_excl_scan(v, wt, tot);
    if (g < G) row[g] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) hist[(size_t)kSortDigits * G + blockIdx.x] = run;
}

__global__ void sort_scan_digits_kernel(uint32_t* hist, int G) {
  __shared__ uint32_t wt[33];
  uint32_t* tot = hist + (size_t)kSortDigits * G;
  const uint32_t v = tot[threadIdx.x];
  uint32_t all = 0;
  const uint32_t ex = block_excl_scan(v, wt, all);
  tot[threadIdx.x] = ex;
}

// one warp per block: walk the chunk in order, so equal digits keep their order
__global__ void sort_scatter_kernel(const uint32_t* key_in, const uint32_t* idx_in, uint32_t* key_out,
                                    uint32_t* idx_out, const PassCtl* ctl, uint32_t shift, const uint32_t* hist, int G) {
  __shared__ uint32_t run[kSortDigits];
  const uint32_t n = ctl->nsel, lane = threadIdx.x;
  for (int d = lane; d < kSortDigits; d += 32) run[d] = hist[d * G + blockIdx.x] + hist[(size_t)kSortDigits * G + d];
  __syncwarp();
  const uint32_t a = blockIdx.x * kSortChunk, b = min(n, a + kSortChunk);
  for (uint32_t t = a; t < b; t += 32) {
    const uint32_t i = t + lane;
    const bool ok = i < b;
    const uint32_t k = ok ? key_in[i] : 0u;
    const uint32_t d = ok ? ((k >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    uint32_t base = 0;
    if (ok) base = run[d];
    __syncwarp();
    if (ok) {
      key_out[base + rank] = k;
      idx_out[base + rank] = idx_in[i];
      if (rank == 0) run[d] = base + __popc(peers);
    }
    __syncwarp();
  }
}

// rank[id] = id: ids beyond the candidate set then map to counters that are
// never incremented (they read as zero).
__global__ void rank_init_kernel(uint32_t* rank, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) rank[i] = i;
}

// order[x] = id of the x-th candidate by (count desc, id asc)  ->  rank[id] = x
__global__ void rank_scatter_kernel(const uint32_t* order, const PassCtl* ctl, uint32_t* rank) {
  const uint32_t n = ctl->nsel;
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) rank[order[x]] = x;
}

}  // namespace

void launch_rank(const uint32_t* order, const PassCtl* ctl, uint32_t* rank, uint32_t n, cudaStream_t s) {
  rank_init_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(rank, n);
  rank_scatter_kernel<<<256, 256, 0, s>>>(order, ctl, rank);
}

void launch_pass_reset(PassCtl* ctl, uint32_t m, unsigned long long* gset, uint64_t gset_entries, cudaStream_t s) {
  pass_reset_kernel<<<1, 32, 0, s>>>(ctl, m);
  if (gset && gset_entries) {
    gset_clear_kernel<<<1024, 256, 0, s>>>(ctl, gset, gset_entries);
    gset_clear_done_kernel<<<1, 32, 0, s>>>(ctl);
  }
}

void launch_select(const uint32_t* counts, bool narrow, const uint32_t* rank, uint32_t sb, uint64_t ns,
                   uint32_t target, PassCtl* ctl, uint32_t* hist, uint32_t* blk, int G, uint32_t* sel_slot,
                   uint32_t* sel_count, cudaStream_t s) {
  sel_reset_kernel<<<1, 1024, 0, s>>>(ctl, target, hist);
  // counters are read in 8-slot units (4-slot with a rank map over sigma = 4)
  const uint64_t U = (rank && sb < 3) ? 4 : 8, nu = (ns + U - 1) / U;
  const uint64_t per_sm = (nu + 152 * 256 - 1) / (152 * 256);
  const int grid = (int)std::min<uint64_t>(8 * 152, std::max<uint64_t>(1, per_sm) * 152);
  max_nonzero_kernel<<<grid, kThreads, 0, s>>>(counts, narrow, rank, sb, ns, ctl);
  threshold_init_kernel<<<1, 32, 0, s>>>(ctl);
  for (int l = 0; l < 3; ++l) {
    level_hist_kernel<<<grid, 512, 0, s>>>(counts, narrow, rank, sb, ns, ctl, hist);
    level_pick_kernel<<<1, kHistBins / 4, 0, s>>>(ctl, hist);
  }
  uint64_t chunk = (nu + G - 1) / G;  // units per compaction block
  if (chunk == 0) chunk = 1;
  compact_count_kernel<<<G, kThreads, 0, s>>>(counts, narrow, rank, sb, ns, ctl, blk, chunk);
  compact_scan_kernel<<<1, 1024, 0, s>>>(blk, G);
  compact_write_kernel<<<G, kThreads, 0, s>>>(counts, narrow, rank, sb, ns, ctl, blk, chunk, sel_slot,
                                             sel_count);
}

void launch_sort_by_count(const uint32_t* sel_count, PassCtl* ctl, uint32_t cap, uint32_t key_bits,
                          uint32_t* idx_a, uint32_t* idx_b, uint32_t* key_a, uint32_t* key_b, uint32_t* hist,
                          cudaStream_t s) {
  const int G = (int)((cap + kSortChunk - 1) / kSortChunk);
  sort_init_kernel<<<256, 256, 0, s>>>(sel_count, ctl, key_bits, key_a, idx_a);
  uint32_t *ki = key_a, *ko = key_b, *ii = idx_a, *io = idx_b;
  for (uint32_t shift = 0; shift < key_bits; shift += 8) {
    sort_hist_kernel<<<G, 256, 0, s>>>(ki, ctl, shift, hist, G);
    sort_scan_rows_kernel<<<kSortDigits, 256, 0, s>>>(hist, G);
    sort_scan_digits_kernel<<<1, kSortDigits, 0, s>>>(hist, G);
    sort_scatter_kernel<<<G, 32, 0, s>>>(ki, ii, ko, io, ctl, shift, hist, G);
    uint32_t* t = ki; ki = ko; ko = t;
    t = ii; ii = io; io = t;
  }
  // an even number of passes: the result is back in (key_a, idx_a)
}

}  // namespace ig
