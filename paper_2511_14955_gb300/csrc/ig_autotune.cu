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
// reported as IG_ESTATE. Choices are cached per (device name and SM count,
// alphabet, n, base, candidate-count bucket, count mode, corpus-size bucket):
// in the process, and in a cache file so that later processes skip the
// sample runs. The file is INTERGRAMS_TUNE_CACHE if that is set (empty or
// "none": no file), else $XDG_CACHE_HOME/intergrams/autotune.txt or
// $HOME/.cache/intergrams/autotune.txt. One line per choice: the key, then
// the ig_tuning fields in header order, preceded by their number (a line
// whose field count differs from this build's is ignored). Lines are
// appended whole; the last line for a key wins.
#include <sys/stat.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "ig_internal.cuh"

namespace ig {
void set_last_error(const std::string& msg);
}

namespace {

using Key = std::tuple<std::string, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;
std::mutex g_mu;
std::map<Key, ig_tuning> g_cache;
bool g_file_loaded = false;
constexpr uint32_t kFields = sizeof(ig_tuning) / sizeof(uint32_t);

std::string cache_path() {
  const char* env = std::getenv("INTERGRAMS_TUNE_CACHE");
  if (env) return (env[0] == 0 || std::strcmp(env, "none") == 0) ? std::string() : std::string(env);
  std::string dir;
  if (const char* x = std::getenv("XDG_CACHE_HOME"); x && x[0]) dir = x;
  else if (const char* h = std::getenv("HOME"); h && h[0]) dir = std::string(h) + "/.cache";
  else return std::string();
  return dir + "/intergrams/autotune.txt";
}

// Device name with blanks replaced, so a key is whitespace-separated tokens.
std::string device_token(int dev, uint32_t* sms) {
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    *sms = 0;
    return "unknown";
  }
  *sms = (uint32_t)prop.multiProcessorCount;
  std::string n = prop.name;
  for (char& c : n)
    if (c == ' ' || c == '\t') c = '_';
  return n.empty() ? "unknown" : n;
}

std::string key_line(const Key& k) {
  std::ostringstream o;
  o << std::get<0>(k) << ' ' << std::get<1>(k) << ' ' << std::get<2>(k) << ' ' << std::get<3>(k) << ' '
    << std::get<4>(k) << ' ' << std::get<5>(k) << ' ' << std::get<6>(k) << ' ' << std::get<7>(k);
  return o.str();
}

// Read the cache file into g_cache (caller holds g_mu).
void load_file_locked() {
  g_file_loaded = true;
  const std::string path = cache_path();
  if (path.empty()) return;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return;
  char buf[1024];
  while (std::fgets(buf, sizeof(buf), f)) {
    std::istringstream in(buf);
    std::string name;
    uint32_t a[7], nf = 0;
    if (!(in >> name >> a[0] >> a[1] >> a[2] >> a[3] >> a[4] >> a[5] >> a[6] >> nf) || nf != kFields) continue;
    ig_tuning t{};
    uint32_t* dst = &t.ctas_per_sm;
    bool ok = true;
    for (uint32_t i = 0; i < kFields && ok; ++i) ok = static_cast<bool>(in >> dst[i]);
    if (ok) g_cache[Key{name, a[0], a[1], a[2], a[3], a[4], a[5], a[6]}] = t;
  }
  std::fclose(f);
}

// Append one choice to the cache file (caller holds g_mu); failures to
// write are ignored (the file is only a cache).
void append_file_locked(const Key& k, const ig_tuning& t) {
  const std::string path = cache_path();
  if (path.empty()) return;
  for (size_t i = 1; i < path.size(); ++i)
    if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
  std::ostringstream o;
  o << key_line(k) << ' ' << kFields;
  const uint32_t* src = &t.ctas_per_sm;
  for (uint32_t i = 0; i < kFields; ++i) o << ' ' << src[i];
  o << '\n';
  const std::string line = o.str();
  FILE* f = std::fopen(path.c_str(), "a");
  if (!f) return;
  std::fwrite(line.data(), 1, line.size(), f);
  std::fclose(f);
}

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
  uint32_t sms = 0;
  const std::string dname = device_token(dev, &sms);
  const Key key{dname, sms, p->symbol_bits, p->n, p->base_n, log2_bucket(p->candidates), p->count_mode,
                log2_bucket(h[m] + 1)};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_file_loaded) load_file_locked();
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
    append_file_locked(key, best_t);
  }
  *out = best_t;
  if (best_ms) *best_ms = best;
  return IG_OK;
}
