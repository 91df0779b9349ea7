// Autotuner: picks the scan's tuning knobs by timing a few candidates on a
// sample of the corpus.
//
// The sample is a prefix of the sequences (sequences are independent, so a
// prefix is a fair sample of an i.i.d. corpus) of about sample_bytes. Each
// candidate runs the whole job on the sample with per-pass CUDA-event timing;
// the candidate with the fastest candidate passes wins, and the dense base
// pass takes the tile and set size of the candidate (same CTA shape) with the
// fastest base pass. Every candidate must return byte-identical top-k
// rows and counts (the knobs only change speed and memory); a mismatch is
// reported as IG_ESTATE. Choices are cached in-process per (device, alphabet,
// n, base, candidate-count bucket, count mode, corpus-size bucket).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "ig_internal.cuh"

namespace ig {
void set_last_error(const std::string& msg);
}

namespace {

using Key = std::tuple<int, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;
std::mutex g_mu;
std::map<Key, ig_tuning> g_cache;

// knob sets tried: (ctas/SM, threads, words/thread, set log2, table load %, hot log2)
const ig_tuning kCandidates[] = {
    {1, 1024, 5, 15, 25, 11, 0, 0},
    {1, 1024, 3, 15, 25, 12, 0, 0},
    {1, 1024, 7, 14, 25, 10, 0, 0},
    {2, 512, 5, 14, 25, 10, 0, 0},
    {2, 512, 3, 13, 40, 11, 0, 0},
    {4, 256, 5, 13, 25, 9, 0, 0},
};

uint32_t log2_bucket(uint64_t x) {
  uint32_t l = 0;
  while ((1ull << l) < x && l < 63) ++l;
  return l;
}

}  // namespace

extern "C" ig_status intergrams_autotune(const ig_params* p, const void* data, const uint64_t* offsets, uint32_t m,
                                         void* stream, uint64_t sample_bytes, ig_tuning* out, float* best_ms) {
  ig::set_last_error("");
  if (!p || !offsets || !out) return IG_EINVAL;
  // offsets on the host (device input is read back once)
  std::vector<uint64_t> h((size_t)m + 1);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (p->flags & (IG_F_HOST_INPUT | IG_F_OFFSETS_HOST)) {
    std::memcpy(h.data(), offsets, sizeof(uint64_t) * h.size());
  } else {
    if (cudaMemcpyAsync(h.data(), offsets, sizeof(uint64_t) * h.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      ig::set_last_error("offsets read-back failed");
      return IG_ECUDA;
    }
  }
  if (sample_bytes == 0) sample_bytes = 256ull << 20;
  const uint64_t sym_bytes_num = p->symbol_bits;  // bytes = symbols * bits / 8
  uint32_t ms = 0;
  while (ms < m && (h[ms] * sym_bytes_num) / 8 < sample_bytes) ++ms;
  if (ms == 0) ms = std::min<uint32_t>(m, 1);
  int dev = 0;
  cudaGetDevice(&dev);
  const Key key{dev, p->symbol_bits, p->n, p->base_n, log2_bucket(p->candidates), p->count_mode,
                log2_bucket(h[m] + 1)};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second;
      if (best_ms) *best_ms = 0.f;
      return IG_OK;
    }
  }
  ig_params sp = *p;
  sp.flags = (p->flags & (IG_F_HOST_INPUT | IG_F_OFFSETS_HOST)) | IG_F_TIMING;
  sp.flags |= IG_F_OFFSETS_HOST;
  const void* sdata = data;
  std::vector<uint8_t> ref_keys, keys;
  std::vector<uint64_t> ref_counts, counts;
  const uint32_t rb = (p->n * p->symbol_bits + 7) / 8;
  float best = 1e30f;
  ig_tuning best_t = kCandidates[0];
  bool have_ref = false;
  std::vector<std::pair<ig_tuning, float>> base_times;  // base-pass ms of every candidate that ran
  for (const ig_tuning& cand : kCandidates) {
    ig_plan* pl = nullptr;
    ig_status st = intergrams_plan(&sp, sdata, h.data(), ms, stream, &cand, &pl);
    if (st == IG_EINVAL || st == IG_ENOMEM) continue;  // does not fit this device or corpus
    if (st != IG_OK) return st;
    float total = 0.f, base_ms = 0.f;
    for (int rep = 0; rep < 2 && st == IG_OK; ++rep) {  // first run warms caches and the pool
      intergrams_rewind(pl);
      st = intergrams_run(pl);
      if (st != IG_OK) break;
      std::vector<float> pass(p->n + 1, 0.f);
      uint32_t np = 0;
      st = intergrams_timings(pl, nullptr, pass.data(), (uint32_t)pass.size(), &np, nullptr);
      total = 0.f;
      base_ms = np ? pass[0] : 0.f;  // pass[0] is the dense base pass
      for (uint32_t i = 1; i < np; ++i) total += pass[i];
      if (np == 1) total = base_ms;  // n == base_n: the base pass is the whole job
    }
    if (st == IG_OK) {
      keys.assign((size_t)p->k * rb, 0);
      counts.assign(p->k, 0);
      uint32_t kout = 0;
      st = intergrams_topk(pl, keys.data(), counts.data(), p->k, &kout, nullptr);
      keys.resize((size_t)kout * rb);
      counts.resize(kout);
    }
    intergrams_free(pl);
    if (st == IG_ETABLE_FULL) continue;
    if (st != IG_OK) return st;
    if (!have_ref) {
      ref_keys = keys;
      ref_counts = counts;
      have_ref = true;
    } else if (keys != ref_keys || counts != ref_counts) {
      ig::set_last_error("autotune: tuning candidates disagree on the result");
      return IG_ESTATE;
    }
    base_times.emplace_back(cand, base_ms);
    if (total < best) {
      best = total;
      best_t = cand;
    }
  }
  {
    float bb = 1e30f;
    for (const auto& bt : base_times)
      if (bt.first.ctas_per_sm == best_t.ctas_per_sm && bt.first.threads == best_t.threads && bt.second < bb) {
        bb = bt.second;
        best_t.base_words_per_thread = bt.first.words_per_thread;
        best_t.base_smem_set_log2 = bt.first.smem_set_log2;
      }
  }
  if (!have_ref) {
    ig::set_last_error("autotune: no candidate could run");
    return IG_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = best_t;
  }
  *out = best_t;
  if (best_ms) *best_ms = best;
  return IG_OK;
}
