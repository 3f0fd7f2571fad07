// Autotuner: the schedule and tile size of one matrix chosen by timing every
// candidate on the caller's own data.  The paper fixes the choice by a size
// rule (Sec. 6.2, alpha = 500 rows or columns, beta = 10,000 nonzeros); that
// rule is kept as the prior -- its pick is timed first and wins ties -- and
// the measurement decides.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "lb_internal.h"

using namespace lbh;

namespace {

// splitmix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a bijective 64-bit mixer.
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Order-independent fingerprint of the tile set and of a sample of the column
// indices: XOR over entries of mix64(position, value).
__global__ void fingerprint_kernel(const int32_t* __restrict__ rp, int32_t R, const int32_t* __restrict__ ci,
                                   int64_t N, int64_t stride, int32_t samples, unsigned long long* out) {
  uint64_t h = 0;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= R; i += nthreads)
    h ^= mix64(((uint64_t)i << 32) ^ (uint32_t)rp[i]);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < samples; q += nthreads) {
    const int64_t k = q * stride;
    if (k < N) h ^= mix64(0x5bd1e995ULL * (uint64_t)(k + 1) ^ ((uint64_t)(uint32_t)ci[k] << 17));
  }
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0 && h) atomicXor(out, (unsigned long long)h);
}

struct Candidate {
  lb_schedule_t schedule;
  int ipt, group, variant;
  int units = 1;       // merge-path warp workers: work units per CTA
  int row_weight = 1;  // merge-path variant 0: weight of a row end in the shares
  int staged = 0;      // thread-mapped: atoms staged in shared memory
};

// Cache key: the GPU (name / SM count / compute capability, so that a cache
// file moves only between identical devices), sizes, fingerprint, candidate
// families and the cold-L2 flag.
using Key = std::tuple<std::string, int32_t, int32_t, int32_t, uint64_t, int32_t, int32_t>;
std::mutex g_cache_mu;
std::map<Key, lb_tune_result_t> g_cache;
bool g_env_loaded = false;  // LB_AUTOTUNE_CACHE read into g_cache (once per process)

std::string device_ident(int dev) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
  return std::string(pr.name) + "/" + std::to_string(pr.multiProcessorCount) + "/" + std::to_string(pr.major) + "." +
         std::to_string(pr.minor);
}

// Batch cache key: the GPU, number of matrices, total rows / columns / atoms,
// fingerprint of the concatenated row offsets and a column sample, passes
// timed and the cold-L2 flag.
using BKey = std::tuple<std::string, int32_t, int32_t, int32_t, int64_t, uint64_t, int32_t, int32_t>;
std::map<BKey, lb_batch_tune_result_t> g_bcache;

// ---- persisted cache: one JSON object per line, written and read only here --
//
// {"format":"lb_autotune_cache","version":V,"device":"NAME/SMS/CC","rows":R,"atoms":N,"cols":C,
//  "fingerprint":"0x...","families":F,"cold_l2":0|1,"best":b,"heuristic":h,"best_schedule":s,
//  "best_opts":[12 ints of lb_plan_opts_t],"candidates":[[schedule,ipt,group,variant,units,row_weight,
//  staged,status,reps,ms,gbps],...]}
constexpr int kOptsInts = (int)(sizeof(lb_plan_opts_t) / sizeof(int32_t));

std::string entry_line(const Key& k, const lb_tune_result_t& r) {
  std::string out;
  char buf[512];
  std::string dev = std::get<0>(k);
  for (char& ch : dev)
    if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
  std::snprintf(buf, sizeof(buf),
                "{\"format\":\"lb_autotune_cache\",\"version\":%d,\"device\":\"%s\",\"rows\":%d,\"atoms\":%d,"
                "\"cols\":%d,\"fingerprint\":\"0x%016llx\",\"families\":%d,\"cold_l2\":%d,\"best\":%d,"
                "\"heuristic\":%d,\"best_schedule\":%d,\"best_opts\":[",
                (int)lb_version(), dev.c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                (unsigned long long)std::get<4>(k), std::get<5>(k), std::get<6>(k), r.best, r.heuristic,
                r.best_schedule);
  out += buf;
  const int32_t* o = reinterpret_cast<const int32_t*>(&r.best_opts);
  for (int i = 0; i < kOptsInts; ++i) {
    std::snprintf(buf, sizeof(buf), "%s%d", i ? "," : "", o[i]);
    out += buf;
  }
  out += "],\"candidates\":[";
  for (int i = 0; i < r.num_candidates; ++i) {
    const lb_tune_candidate_t& c = r.candidates[i];
    std::snprintf(buf, sizeof(buf), "%s[%d,%d,%d,%d,%d,%d,%d,%d,%d,%.9g,%.9g]", i ? "," : "", c.schedule,
                  c.items_per_thread, c.group_size, c.mp_variant, c.units_per_cta, c.row_weight, c.staged, c.status,
                  c.reps, (double)c.ms, (double)c.gbps);
    out += buf;
  }
  out += "]}\n";
  return out;
}

// value after "key": in one line (nullptr if absent)
const char* field(const std::string& line, const char* key) {
  const std::string pat = std::string("\"") + key + "\":";
  const size_t at = line.find(pat);
  return at == std::string::npos ? nullptr : line.c_str() + at + pat.size();
}

bool field_ll(const std::string& line, const char* key, long long& v) {
  const char* p = field(line, key);
  if (!p) return false;
  char* end = nullptr;
  v = std::strtoll(p, &end, 10);
  return end != p;
}

bool field_str(const std::string& line, const char* key, std::string& v) {
  const char* p = field(line, key);
  if (!p || *p != '"') return false;
  const char* e = std::strchr(p + 1, '"');
  if (!e) return false;
  v.assign(p + 1, e);
  return true;
}

// every number inside the (possibly nested) array that follows "key":
bool field_nums(const std::string& line, const char* key, std::vector<double>& v) {
  const char* p = field(line, key);
  if (!p || *p != '[') return false;
  int depth = 0;
  v.clear();
  while (*p) {
    if (*p == '[') {
      ++depth;
      ++p;
    } else if (*p == ']') {
      if (--depth == 0) return true;
      ++p;
    } else if (*p == ',' || *p == ' ') {
      ++p;
    } else {
      char* end = nullptr;
      const double d = std::strtod(p, &end);
      if (end == p) return false;
      v.push_back(d);
      p = end;
    }
  }
  return false;
}

// one line -> (key, result); false if it is not a valid entry of this library version
bool parse_entry(const std::string& line, Key& k, lb_tune_result_t& r) {
  long long ver, rows, atoms, cols, fam, cold, best, heur, bs;
  std::string dev, fps, fmt;
  std::vector<double> opts, cands;
  if (!field_str(line, "format", fmt) || fmt != "lb_autotune_cache" || !field_ll(line, "version", ver) ||
      ver != lb_version() || !field_str(line, "device", dev) || !field_ll(line, "rows", rows) ||
      !field_ll(line, "atoms", atoms) || !field_ll(line, "cols", cols) || !field_str(line, "fingerprint", fps) ||
      !field_ll(line, "families", fam) || !field_ll(line, "cold_l2", cold) || !field_ll(line, "best", best) ||
      !field_ll(line, "heuristic", heur) || !field_ll(line, "best_schedule", bs) ||
      !field_nums(line, "best_opts", opts) || !field_nums(line, "candidates", cands))
    return false;
  constexpr size_t kStride = 11;
  if ((int)opts.size() != kOptsInts || cands.size() % kStride != 0 || cands.size() / kStride > LB_TUNE_MAX_CANDIDATES ||
      cands.empty() || best < 0 || best >= (long long)(cands.size() / kStride) ||
      heur >= (long long)(cands.size() / kStride))
    return false;
  std::memset(&r, 0, sizeof(r));
  r.num_candidates = (int32_t)(cands.size() / kStride);
  r.best = (int32_t)best;
  r.heuristic = (int32_t)heur;
  r.best_schedule = (int32_t)bs;
  int32_t* o = reinterpret_cast<int32_t*>(&r.best_opts);
  for (int i = 0; i < kOptsInts; ++i) o[i] = (int32_t)opts[i];
  for (int i = 0; i < r.num_candidates; ++i) {
    const double* c = cands.data() + kStride * i;
    lb_tune_candidate_t& t = r.candidates[i];
    t.schedule = (int32_t)c[0];
    t.items_per_thread = (int32_t)c[1];
    t.group_size = (int32_t)c[2];
    t.mp_variant = (int32_t)c[3];
    t.units_per_cta = (int32_t)c[4];
    t.row_weight = (int32_t)c[5];
    t.staged = (int32_t)c[6];
    t.status = (int32_t)c[7];
    t.reps = (int32_t)c[8];
    t.ms = (float)c[9];
    t.gbps = (float)c[10];
  }
  const uint64_t fp = std::strtoull(fps.c_str(), nullptr, 16);
  k = Key{dev, (int32_t)rows, (int32_t)atoms, (int32_t)cols, fp, (int32_t)fam, (int32_t)cold};
  return true;
}

// Batch entries: {"format":"lb_batch_autotune_cache","version":V,"device":"...","mats":M,"rows":R,
//  "cols":C,"atoms":N,"fingerprint":"0x...","passes":P,"cold_l2":0|1,"best":b,"best_opts":[12 ints],
//  "candidates":[[12 ints of options,status,reps,ms,gbps],...]}
std::string bentry_line(const BKey& k, const lb_batch_tune_result_t& r) {
  std::string out;
  char buf[512];
  std::string dev = std::get<0>(k);
  for (char& ch : dev)
    if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
  std::snprintf(buf, sizeof(buf),
                "{\"format\":\"lb_batch_autotune_cache\",\"version\":%d,\"device\":\"%s\",\"mats\":%d,"
                "\"rows\":%d,\"cols\":%d,\"atoms\":%lld,\"fingerprint\":\"0x%016llx\",\"passes\":%d,"
                "\"cold_l2\":%d,\"best\":%d,\"best_opts\":[",
                (int)lb_version(), dev.c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                (long long)std::get<4>(k), (unsigned long long)std::get<5>(k), std::get<6>(k), std::get<7>(k),
                r.best);
  out += buf;
  const int32_t* o = reinterpret_cast<const int32_t*>(&r.best_opts);
  for (int i = 0; i < kOptsInts; ++i) {
    std::snprintf(buf, sizeof(buf), "%s%d", i ? "," : "", o[i]);
    out += buf;
  }
  out += "],\"candidates\":[";
  for (int i = 0; i < r.num_candidates; ++i) {
    const lb_batch_tune_candidate_t& c = r.candidates[i];
    out += i ? ",[" : "[";
    const int32_t* co = reinterpret_cast<const int32_t*>(&c.opts);
    for (int q = 0; q < kOptsInts; ++q) {
      std::snprintf(buf, sizeof(buf), "%d,", co[q]);
      out += buf;
    }
    std::snprintf(buf, sizeof(buf), "%d,%d,%.9g,%.9g]", c.status, c.reps, (double)c.ms, (double)c.gbps);
    out += buf;
  }
  out += "]}\n";
  return out;
}

bool parse_bentry(const std::string& line, BKey& k, lb_batch_tune_result_t& r) {
  long long ver, mats, rows, cols, atoms, passes, cold, best;
  std::string dev, fps, fmt;
  std::vector<double> opts, cands;
  constexpr int kStride = kOptsInts + 4;
  if (!field_str(line, "format", fmt) || fmt != "lb_batch_autotune_cache" || !field_ll(line, "version", ver) ||
      ver != lb_version() || !field_str(line, "device", dev) || !field_ll(line, "mats", mats) ||
      !field_ll(line, "rows", rows) || !field_ll(line, "cols", cols) || !field_ll(line, "atoms", atoms) ||
      !field_str(line, "fingerprint", fps) || !field_ll(line, "passes", passes) ||
      !field_ll(line, "cold_l2", cold) || !field_ll(line, "best", best) || !field_nums(line, "best_opts", opts) ||
      !field_nums(line, "candidates", cands))
    return false;
  if ((int)opts.size() != kOptsInts || cands.empty() || cands.size() % kStride != 0 ||
      cands.size() / kStride > LB_TUNE_MAX_CANDIDATES || best < 0 || best >= (long long)(cands.size() / kStride))
    return false;
  std::memset(&r, 0, sizeof(r));
  r.num_candidates = (int32_t)(cands.size() / kStride);
  r.best = (int32_t)best;
  r.passes = (int32_t)passes;
  int32_t* o = reinterpret_cast<int32_t*>(&r.best_opts);
  for (int i = 0; i < kOptsInts; ++i) o[i] = (int32_t)opts[i];
  for (int i = 0; i < r.num_candidates; ++i) {
    const double* c = cands.data() + kStride * i;
    lb_batch_tune_candidate_t& t = r.candidates[i];
    int32_t* co = reinterpret_cast<int32_t*>(&t.opts);
    for (int q = 0; q < kOptsInts; ++q) co[q] = (int32_t)c[q];
    t.status = (int32_t)c[kOptsInts];
    t.reps = (int32_t)c[kOptsInts + 1];
    t.ms = (float)c[kOptsInts + 2];
    t.gbps = (float)c[kOptsInts + 3];
  }
  const uint64_t fp = std::strtoull(fps.c_str(), nullptr, 16);
  k = BKey{dev, (int32_t)mats, (int32_t)rows, (int32_t)cols, (int64_t)atoms, fp, (int32_t)passes, (int32_t)cold};
  return true;
}

// caller holds g_cache_mu
lb_status_t load_locked(const char* path, int32_t* loaded) {
  if (loaded) *loaded = 0;
  FILE* f = std::fopen(path, "r");
  if (!f) {
    set_error(std::string("autotune cache: cannot open ") + path);
    return LB_ERR_INVALID_ARG;
  }
  std::string line;
  char buf[4096];
  int32_t n = 0;
  while (std::fgets(buf, sizeof(buf), f)) {
    line += buf;
    if (line.empty() || line.back() != '\n') {
      if (!std::feof(f)) continue;  // a line longer than the buffer: keep reading
    }
    Key k;
    lb_tune_result_t r;
    BKey bk;
    lb_batch_tune_result_t br;
    if (parse_entry(line, k, r)) {
      g_cache[k] = r;
      ++n;
    } else if (parse_bentry(line, bk, br)) {
      g_bcache[bk] = br;
      ++n;
    }
    line.clear();
  }
  std::fclose(f);
  if (loaded) *loaded = n;
  return LB_OK;
}

// caller holds g_cache_mu; written to a temporary file first, then renamed over `path`
lb_status_t save_locked(const char* path) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) {
    set_error(std::string("autotune cache: cannot write ") + tmp);
    return LB_ERR_INVALID_ARG;
  }
  bool ok = true;
  for (const auto& kv : g_cache) {
    const std::string l = entry_line(kv.first, kv.second);
    ok = ok && std::fwrite(l.data(), 1, l.size(), f) == l.size();
  }
  for (const auto& kv : g_bcache) {
    const std::string l = bentry_line(kv.first, kv.second);
    ok = ok && std::fwrite(l.data(), 1, l.size(), f) == l.size();
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    set_error(std::string("autotune cache: cannot write ") + path);
    return LB_ERR_INVALID_ARG;
  }
  return LB_OK;
}

// the file named by LB_AUTOTUNE_CACHE, if any (caller holds g_cache_mu)
const char* env_cache_path() {
  const char* p = std::getenv("LB_AUTOTUNE_CACHE");
  return p && *p ? p : nullptr;
}

void env_load_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char* p = env_cache_path();
  if (!p) return;
  FILE* f = std::fopen(p, "r");
  if (!f) return;  // no file yet: the first tuning creates it
  std::fclose(f);
  load_locked(p, nullptr);
}

std::vector<Candidate> candidate_list(lb_schedule_t prior, int families, bool aligned) {
  std::vector<Candidate> v;
  // the heuristic's pick first, so that it wins ties
  if (prior == LB_THREAD_MAPPED && (families & LB_TUNE_THREAD)) v.push_back({LB_THREAD_MAPPED, 0, 0, 0});
  if (families & LB_TUNE_MP_WARP) {
    for (int ipt : {8, 4, 16}) v.push_back({LB_MERGE_PATH, ipt, 0, 0});
    for (int ipt : {4, 8}) v.push_back({LB_MERGE_PATH, ipt, 0, 0, 1, 2});
    for (int ipt : {8, 4}) v.push_back({LB_MERGE_PATH, ipt, 0, 3});
  }
  if (families & LB_TUNE_MP_CTA) {
    for (int ipt : {4, 8}) v.push_back({LB_MERGE_PATH, ipt, 0, 1});
    if (aligned)
      for (int ipt : {4, 8}) v.push_back({LB_MERGE_PATH, ipt, 0, 2});
  }
  if (prior != LB_THREAD_MAPPED && (families & LB_TUNE_THREAD)) v.push_back({LB_THREAD_MAPPED, 0, 0, 0});
  if (families & LB_TUNE_THREAD) v.push_back({LB_THREAD_MAPPED, 0, 0, 0, 1, 1, 1});
  if (families & LB_TUNE_GROUP) {
    for (int g : {4, 8, 16}) v.push_back({LB_GROUP_MAPPED, 0, g, 0});
    v.push_back({LB_WARP_MAPPED, 0, 32, 0});
    for (int g : {64, 128}) v.push_back({LB_GROUP_MAPPED, 0, g, 0});
    v.push_back({LB_BLOCK_MAPPED, 0, 256, 0});
  }
  return v;
}

lb_plan_opts_t opts_of(const Candidate& c, int32_t num_cols) {
  lb_plan_opts_t o{};
  o.num_cols = num_cols;
  o.items_per_thread = c.ipt ? c.ipt : 8;
  o.group_size = c.group;
  o.mp_variant = c.variant;
  o.units_per_cta = c.units;
  o.row_weight = c.row_weight;
  o.staged = c.staged;
  return o;
}

// Events and the optional cold-L2 scratch of one tuning call.
struct Timer {
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* flush = nullptr;
  size_t flush_bytes = 0;
  int flush_round = 0;
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (flush) cudaFree(flush);
  }
  lb_status_t init(bool cold_l2, int dev) {
    LB_CUDA_TRY(cudaEventCreate(&e0));
    LB_CUDA_TRY(cudaEventCreate(&e1));
    if (cold_l2) {
      int l2 = 0;
      LB_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
      flush_bytes = (size_t)std::max(l2, 1 << 20) * 2;
      LB_CUDA_TRY(cudaMalloc(&flush, flush_bytes));
    }
    return LB_OK;
  }
  // one launch of the plan, timed on the stream; the scratch is rewritten first
  lb_status_t once(lb_plan_t p, const int32_t* ci, const float* v, const float* x, float* y, float* ms) {
    if (flush) LB_CUDA_TRY(cudaMemsetAsync(flush, ++flush_round & 0xff, flush_bytes, s));
    LB_CUDA_TRY(cudaEventRecord(e0, s));
    LB_TRY(lb_spmv(p, ci, v, x, y, s));
    LB_CUDA_TRY(cudaEventRecord(e1, s));
    LB_CUDA_TRY(cudaEventSynchronize(e1));
    LB_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return LB_OK;
  }
};

lb_status_t run_candidate(const Candidate& c, const int32_t* rp, int32_t R, int32_t N, int32_t C,
                          const int32_t* ci, const float* v, const float* x, float* y, int reps, float prune_ms,
                          Timer& t, lb_tune_candidate_t* out) {
  const lb_plan_opts_t o = opts_of(c, C);
  lb_plan_t p = nullptr;
  LB_TRY(lb_plan_ex(&p, rp, R, N, c.schedule, &o, t.s));
  struct Guard {
    lb_plan_t p;
    ~Guard() { lb_plan_destroy(p); }
  } guard{p};
  LB_TRY(lb_spmv(p, ci, v, x, y, t.s));  // untimed: first-use costs (module load, cold TLB)
  float first = 0.f;
  LB_TRY(t.once(p, ci, v, x, y, &first));
  std::vector<float> ms{first};
  if (!(first > prune_ms)) {
    for (int r = 1; r < reps; ++r) {
      float m = 0.f;
      LB_TRY(t.once(p, ci, v, x, y, &m));
      ms.push_back(m);
    }
  }
  std::sort(ms.begin(), ms.end());
  out->ms = ms[ms.size() / 2];
  out->reps = (int32_t)ms.size();
  return LB_OK;
}

// Fingerprint of a tile set (its R + 1 offsets) and of 4096 evenly spaced
// column indices, on the device; synchronises s.
lb_status_t fingerprint(const int32_t* rp, int32_t R, const int32_t* ci, int64_t N, cudaStream_t s, uint64_t* out) {
  unsigned long long* d_fp = nullptr;
  LB_CUDA_TRY(cudaMalloc(&d_fp, sizeof(unsigned long long)));
  const int32_t samples = N > 0 ? (int32_t)std::min<int64_t>(4096, N) : 0;
  const int64_t stride = samples > 0 ? std::max<int64_t>(1, N / samples) : 1;
  const int64_t work = std::max<int64_t>((int64_t)R + 1, samples);
  const unsigned blocks = (unsigned)std::min<int64_t>((work + 255) / 256, 4096);
  cudaError_t e = cudaMemsetAsync(d_fp, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    fingerprint_kernel<<<blocks, 256, 0, s>>>(rp, R, ci, N, stride, samples, d_fp);
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_fp, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_fp);
  LB_CUDA_TRY(e);
  *out = h;
  return LB_OK;
}

// Batch candidates: the library's default batch plan first (it wins ties),
// then warp workers at items_per_thread 4, the look-back shares at 4 and 8
// (4 with two-tile shares), one wave for the whole batch, and dynamic units.
std::vector<lb_plan_opts_t> batch_candidates() {
  std::vector<lb_plan_opts_t> v;
  auto add = [&](int ipt, int variant, int tps, int units, int wave_items) {
    lb_plan_opts_t o{};
    o.items_per_thread = ipt;
    o.mp_variant = variant;
    o.tiles_per_share = tps;
    o.units_per_cta = units;
    o.wave_items = wave_items;
    v.push_back(o);
  };
  add(8, 0, 0, 0, 0);
  add(4, 0, 0, 0, 0);
  add(4, 3, 0, 0, 0);
  add(8, 3, 0, 0, 0);
  add(4, 3, 2, 0, 0);
  add(4, 0, 0, 4, 0);
  add(8, 0, 0, 0, 1 << 30);
  return v;
}

}  // namespace

extern "C" {

void lb_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  g_cache.clear();
  g_bcache.clear();
}

int32_t lb_autotune_cache_size(void) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  return (int32_t)(g_cache.size() + g_bcache.size());
}

lb_status_t lb_autotune_cache_save(const char* path) {
  if (!path || !*path) {
    set_error("lb_autotune_cache_save: path must not be empty");
    return LB_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_cache_mu);
  return save_locked(path);
}

lb_status_t lb_autotune_cache_load(const char* path, int32_t* loaded) {
  if (!path || !*path) {
    set_error("lb_autotune_cache_load: path must not be empty");
    return LB_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_cache_mu);
  return load_locked(path, loaded);
}

lb_status_t lb_autotune(const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms, const int32_t* col_idx,
                        const float* vals, const float* x, float* y, const lb_tune_opts_t* opts,
                        lb_tune_result_t* result, lb_plan_t* out_plan, void* stream) {
  if (out_plan) *out_plan = nullptr;
  if (!result || !opts) {
    set_error("lb_autotune: result and opts must not be NULL");
    return LB_ERR_INVALID_ARG;
  }
  std::memset(result, 0, sizeof(*result));
  const int32_t C = opts->num_cols;
  if (num_tiles < 0 || num_atoms < 0 || (num_tiles == 0 && num_atoms != 0) || (num_tiles > 0 && !tile_offsets) ||
      (num_tiles > 0 && !y) || (num_atoms > 0 && (!col_idx || !vals || !x || C < 1)) || C < 0 ||
      opts->reps < 0 || opts->prune_factor < 0.f) {
    set_error("lb_autotune: need num_tiles, num_atoms >= 0, buffers for nonzero sizes and num_cols >= 1");
    return LB_ERR_INVALID_ARG;
  }
  const int reps = opts->reps ? opts->reps : 5;
  const float prune = opts->prune_factor > 0.f ? opts->prune_factor : 3.f;
  const int families = opts->families ? opts->families : (LB_TUNE_MP_WARP | LB_TUNE_MP_CTA | LB_TUNE_THREAD |
                                                           LB_TUNE_GROUP);
  const lb_schedule_t prior = lb_heuristic_schedule(num_tiles, C > 0 ? C : num_tiles, num_atoms);
  const bool aligned = ((reinterpret_cast<uintptr_t>(col_idx) | reinterpret_cast<uintptr_t>(vals)) & 15u) == 0;
  const std::vector<Candidate> cands = candidate_list(prior, families, aligned);
  if (cands.empty()) {
    set_error("lb_autotune: no candidate family selected");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  LB_CUDA_TRY(cudaGetDevice(&dev));

  // fingerprint for the cache
  uint64_t fp = 0;
  const bool use_cache = !opts->no_cache && num_tiles > 0;
  if (use_cache) LB_TRY(fingerprint(tile_offsets, num_tiles, col_idx, num_atoms, s, &fp));
  const Key key{use_cache ? device_ident(dev) : std::string(), num_tiles, num_atoms, C, fp, families,
                opts->cold_l2 ? 1 : 0};
  bool hit = false;
  if (use_cache) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    env_load_locked();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *result = it->second;
      result->from_cache = 1;
      hit = true;
    }
  }

  if (!hit) {
    Timer t;
    t.s = s;
    LB_TRY(t.init(opts->cold_l2 != 0, dev));
    const double bytes = 8.0 * num_atoms + 4.0 * (num_tiles + 1) + 4.0 * C + 4.0 * num_tiles;
    float best_ms = -1.f;
    int best = -1, heur = -1;
    const int n = (int)std::min<size_t>(cands.size(), LB_TUNE_MAX_CANDIDATES);
    for (int i = 0; i < n; ++i) {
      const Candidate& c = cands[i];
      lb_tune_candidate_t& r = result->candidates[i];
      r.schedule = c.schedule;
      r.items_per_thread = c.ipt;
      r.group_size = c.group;
      r.mp_variant = c.variant;
      r.units_per_cta = c.units;
      r.row_weight = c.row_weight;
      r.staged = c.staged;
      if ((c.schedule == prior) && heur < 0 && !c.staged &&
          (c.schedule != LB_MERGE_PATH || (c.ipt == 8 && c.variant == 0 && c.units == 1 && c.row_weight == 1)))
        heur = i;
      if (num_tiles == 0) {
        r.status = LB_OK;
        if (best < 0) best = i;
        continue;
      }
      const float prune_ms = best_ms > 0.f ? prune * best_ms : 3.0e38f;
      r.status = run_candidate(c, tile_offsets, num_tiles, num_atoms, C, col_idx, vals, x, y, reps, prune_ms, t, &r);
      if (r.status != LB_OK) {
        // a candidate that cannot run here (e.g. out of memory for its tables) is skipped;
        // a sticky device error ends the tuning
        r.ms = 0.f;
        r.reps = 0;
        if (cudaPeekAtLastError() != cudaSuccess && cudaDeviceSynchronize() != cudaSuccess) return LB_ERR_CUDA;
        continue;
      }
      r.gbps = r.ms > 0.f ? (float)(bytes / (r.ms * 1e-3) / 1e9) : 0.f;
      if (best < 0 || r.ms < best_ms) {
        best = i;
        best_ms = r.ms;
      }
    }
    if (best < 0) {
      set_error("lb_autotune: no candidate ran");
      return LB_ERR_CUDA;
    }
    result->num_candidates = n;
    result->best = best;
    result->heuristic = heur;
    result->best_schedule = result->candidates[best].schedule;
    result->best_opts = opts_of(cands[best], C);
    if (use_cache) {
      std::lock_guard<std::mutex> lock(g_cache_mu);
      g_cache[key] = *result;
      // persist the new entry when LB_AUTOTUNE_CACHE names a file (a failed write is not an error of the tuning)
      if (const char* path = env_cache_path()) save_locked(path);
    }
  }

  // the winner's plan; y = A x by it
  lb_plan_t p = nullptr;
  LB_TRY(lb_plan_ex(&p, tile_offsets, num_tiles, num_atoms, (lb_schedule_t)result->best_schedule,
                    &result->best_opts, s));
  lb_status_t st = lb_spmv(p, col_idx, vals, x, y, s);
  if (st == LB_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("lb_autotune: final launch failed");
    st = LB_ERR_CUDA;
  }
  if (st != LB_OK || !out_plan) {
    lb_plan_destroy(p);
  } else {
    *out_plan = p;
  }
  return st;
}

lb_status_t lb_batch_autotune(int32_t num_mats, const int32_t* host_rows, const int32_t* host_cols,
                              const int64_t* host_nnz, const int32_t* rp_cat, const int32_t* col_cat,
                              const float* vals_cat, const float* x_cat, float* y_cat, const float* dy_cat,
                              float* dx_cat, float* dvals_cat, int32_t passes, const lb_tune_opts_t* opts,
                              lb_batch_tune_result_t* result, lb_plan_t* out_plan, void* stream) {
  if (out_plan) *out_plan = nullptr;
  if (!result || !opts || num_mats < 1 || !host_rows || !host_cols || !host_nnz || !rp_cat || passes < 1 ||
      passes > (LB_TUNE_PASS_FWD | LB_TUNE_PASS_DX | LB_TUNE_PASS_DVALS) || opts->reps < 0) {
    set_error("lb_batch_autotune: need result, opts, num_mats >= 1, the size arrays, rp_cat and passes in 1..7");
    return LB_ERR_INVALID_ARG;
  }
  std::memset(result, 0, sizeof(*result));
  int64_t R = 0, C = 0, N = 0;
  for (int m = 0; m < num_mats; ++m) {
    if (host_rows[m] < 0 || host_cols[m] < 0 || host_nnz[m] < 0) {
      set_error("lb_batch_autotune: negative size");
      return LB_ERR_INVALID_ARG;
    }
    R += host_rows[m];
    C += host_cols[m];
    N += host_nnz[m];
  }
  const bool fwd = passes & LB_TUNE_PASS_FWD, dx = passes & LB_TUNE_PASS_DX, dv = passes & LB_TUNE_PASS_DVALS;
  if ((fwd && !y_cat) || ((dx || dv) && !dy_cat) || (dx && !dx_cat) || (dv && !dvals_cat) ||
      (N > 0 && (!col_cat || !vals_cat || !x_cat))) {
    set_error("lb_batch_autotune: a buffer the timed passes need is NULL");
    return LB_ERR_INVALID_ARG;
  }
  if (R >= INT32_MAX || C >= INT32_MAX) {
    set_error("lb_batch_autotune: batch totals must stay below 2^31 rows and columns");
    return LB_ERR_UNSUPPORTED;
  }
  const int reps = opts->reps ? opts->reps : 5;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  LB_CUDA_TRY(cudaGetDevice(&dev));
  const bool use_cache = !opts->no_cache;
  uint64_t fp = 0;
  if (use_cache) LB_TRY(fingerprint(rp_cat, (int32_t)(R + num_mats - 1), col_cat, N, s, &fp));
  const BKey key{use_cache ? device_ident(dev) : std::string(), num_mats, (int32_t)R, (int32_t)C, N, fp, passes,
                 opts->cold_l2 ? 1 : 0};
  bool hit = false;
  if (use_cache) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    env_load_locked();
    auto it = g_bcache.find(key);
    if (it != g_bcache.end()) {
      *result = it->second;
      result->from_cache = 1;
      hit = true;
    }
  }
  // one step of the timed passes with plan p
  auto step = [&](lb_plan_t p) -> lb_status_t {
    if (fwd) LB_TRY(lb_batch_spmv(p, col_cat, vals_cat, x_cat, y_cat, s));
    if (dx || dv)
      LB_TRY(lb_batch_spmv_backward(p, col_cat, vals_cat, x_cat, dy_cat, dx ? dx_cat : nullptr,
                                    dv ? dvals_cat : nullptr, s));
    return LB_OK;
  };
  if (!hit) {
    Timer t;
    t.s = s;
    LB_TRY(t.init(opts->cold_l2 != 0, dev));
    double bytes = 0.0;
    if (fwd) bytes += 8.0 * N + 4.0 * (R + num_mats) + 4.0 * C + 4.0 * R;
    if (dx) bytes += 12.0 * N + 4.0 * (C + num_mats) + 4.0 * R + 4.0 * C;
    if (dv) bytes += 8.0 * N + 4.0 * (R + num_mats) + 4.0 * R + 4.0 * C;
    const std::vector<lb_plan_opts_t> cands = batch_candidates();
    const int n = (int)std::min<size_t>(cands.size(), LB_TUNE_MAX_CANDIDATES);
    int best = -1;
    float best_ms = 0.f;
    for (int i = 0; i < n; ++i) {
      lb_batch_tune_candidate_t& r = result->candidates[i];
      r.opts = cands[i];
      lb_plan_t p = nullptr;
      lb_status_t st = lb_batch_plan(&p, num_mats, host_rows, host_cols, host_nnz, rp_cat, &cands[i], s);
      if (st == LB_OK && (dx || dv) && N > 0) st = lb_batch_prepare_backward(p, col_cat, s);
      if (st == LB_OK) st = step(p);  // untimed: first-use costs
      std::vector<float> ms;
      for (int q = 0; st == LB_OK && q < reps; ++q) {
        if (t.flush) {
          if (cudaMemsetAsync(t.flush, ++t.flush_round & 0xff, t.flush_bytes, s) != cudaSuccess) st = LB_ERR_CUDA;
        }
        if (st == LB_OK && cudaEventRecord(t.e0, s) != cudaSuccess) st = LB_ERR_CUDA;
        if (st == LB_OK) st = step(p);
        if (st == LB_OK && (cudaEventRecord(t.e1, s) != cudaSuccess || cudaEventSynchronize(t.e1) != cudaSuccess))
          st = LB_ERR_CUDA;
        float m = 0.f;
        if (st == LB_OK && cudaEventElapsedTime(&m, t.e0, t.e1) != cudaSuccess) st = LB_ERR_CUDA;
        if (st == LB_OK) ms.push_back(m);
      }
      if (p) lb_plan_destroy(p);
      r.status = st;
      if (st != LB_OK) {
        if (cudaPeekAtLastError() != cudaSuccess && cudaDeviceSynchronize() != cudaSuccess) return LB_ERR_CUDA;
        continue;
      }
      std::sort(ms.begin(), ms.end());
      r.ms = ms[ms.size() / 2];
      r.reps = (int32_t)ms.size();
      r.gbps = r.ms > 0.f ? (float)(bytes / (r.ms * 1e-3) / 1e9) : 0.f;
      if (best < 0 || r.ms < best_ms) {
        best = i;
        best_ms = r.ms;
      }
    }
    if (best < 0) {
      set_error("lb_batch_autotune: no candidate ran");
      return LB_ERR_CUDA;
    }
    result->num_candidates = n;
    result->best = best;
    result->passes = passes;
    result->best_opts = cands[best];
    if (use_cache) {
      std::lock_guard<std::mutex> lock(g_cache_mu);
      g_bcache[key] = *result;
      if (const char* path = env_cache_path()) save_locked(path);
    }
  }
  // the winner's plan; the outputs of the timed passes by it
  lb_plan_t p = nullptr;
  LB_TRY(lb_batch_plan(&p, num_mats, host_rows, host_cols, host_nnz, rp_cat, &result->best_opts, s));
  lb_status_t st = ((dx || dv) && N > 0) ? lb_batch_prepare_backward(p, col_cat, s) : LB_OK;
  if (st == LB_OK) st = step(p);
  if (st == LB_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("lb_batch_autotune: final launch failed");
    st = LB_ERR_CUDA;
  }
  if (st != LB_OK || !out_plan) {
    lb_plan_destroy(p);
  } else {
    *out_plan = p;
  }
  return st;
}

}  // extern "C"
