// Autotuner of the plan partition (include/tho.h: tho_autotune, tho_tune_key,
// tho_tune_cache_get, tho_tune_cache_put).
//
// Two choices shape every plan without changing what Algorithm 1 computes: the
// TSQR leaf height P (the Householder QR of A'_2 runs over row panels of P/2 to
// P rows, then over a binary tree of their R factors) and the split-n factor
// (how many row chunks the streaming sweeps W^* A, the rank-k0 updates and
// W^* [0; Qbar] are cut into).  The tuner measures candidates through the
// public entry points (tho_plan_tuned, tho_orth, tho_orth_batched) on seeded
// synthetic operands of the requested shapes and remembers the winner in a
// JSON-lines cache keyed by device, dtype, precision, flags and shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tho.h"

namespace {

// floor(4 log2 n) for n >= 1: the octave from the bit length, the quarter from
// n / 2^e in [1, 2) against 2^(1/4), 2^(1/2), 2^(3/4) (exact scaling, so the
// bucket is the same on every host).
int n_bucket(int64_t n) {
  int e = 0;
  while (e < 62 && (int64_t(1) << (e + 1)) <= n) ++e;
  const double r = std::ldexp((double)n, -e);
  const int q = (r >= 1.189207115002721) + (r >= 1.4142135623730951) + (r >= 1.681792830507429);
  return 4 * e + q;
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

bool key_char_ok(char c) { return c != '"' && c != '\\' && (unsigned char)c >= 0x20; }

std::string make_key(const tho_desc_t* d, int32_t count, const char* device_name) {
  std::string dev;
  for (const char* c = device_name; *c; ++c) dev += (key_char_ok(*c) && *c != '|') ? *c : '_';
  static const char* const kDt[] = {"f64", "c128"};
  static const char* const kPr[] = {"fp64", "fp32bulk", "emu"};
  char head[64];
  std::snprintf(head, sizeof(head), "|%s|%s|f%x|", kDt[d[0].dtype == THO_C128 ? 1 : 0],
                kPr[(d[0].prec >= 0 && d[0].prec <= 2) ? d[0].prec : 0], (unsigned)d[0].flags);
  std::string list;
  for (int i = 0; i < count; ++i) {
    char b[64];
    std::snprintf(b, sizeof(b), "%sq%d:%lld:%lld", i ? "," : "", n_bucket(d[i].n), (long long)d[i].k0,
                  (long long)d[i].k);
    list += b;
  }
  if (count > 8) {
    char b[64];
    std::snprintf(b, sizeof(b), "batch%d:%016llx", count, (unsigned long long)fnv1a(list));
    list = b;
  }
  return dev + head + list;
}

// Value after `"name":` on a cache line, or false.
bool find_num(const char* line, const char* name, double* v) {
  char pat[40];
  std::snprintf(pat, sizeof(pat), "\"%s\":", name);
  const char* p = std::strstr(line, pat);
  if (!p) return false;
  p += std::strlen(pat);
  char* end = nullptr;
  *v = std::strtod(p, &end);
  return end != p && std::isfinite(*v);
}

bool parse_line(const char* line, std::string* key, tho_tuning_t* t, double* ms) {
  const char* p = std::strstr(line, "\"key\":");
  if (!p) return false;
  p = std::strchr(p + 6, '"');
  if (!p) return false;
  const char* q = std::strchr(p + 1, '"');
  if (!q) return false;
  key->assign(p + 1, q);
  double lr = 0, sc = 0, bl = 0, m = 0;
  if (!find_num(q, "leaf_rows", &lr) || !find_num(q, "split_chunks", &sc) || !find_num(q, "balance", &bl) ||
      !find_num(q, "ms", &m))
    return false;
  if (lr != std::floor(lr) || sc != std::floor(sc) || lr < 0 || sc < 0 || sc > THO_TUNE_MAX_SPLIT) return false;
  if (bl != 0.0 && bl != 1.0) return false;
  t->leaf_rows = (int32_t)lr;
  t->split_chunks = (int32_t)sc;
  t->balance = (int32_t)bl;
  *ms = m;
  return true;
}

// splitmix64 (Steele, Lea and Flood, 2014) of the element index: uniform
// values in [-scale, scale).
__global__ void k_tune_fill(double* x, int64_t count, uint64_t seed, double scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = ((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * scale;
  }
}

struct Operands {
  void* buf = nullptr;
  std::vector<tho_instance_t> inst;
  ~Operands() {
    if (buf) cudaFree(buf);
  }
};

tho_status_t make_operands(const tho_desc_t* d, int32_t count, cudaStream_t st, Operands* ops) {
  const size_t el = d[0].dtype == THO_C128 ? 16 : 8;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  std::vector<size_t> off(count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    const size_t n = (size_t)d[i].n, k0 = (size_t)d[i].k0, k = (size_t)d[i].k;
    off[i] = total;
    total += al(n * k0 * el) + 2 * al(n * k * el) + al(k * k * el) + al(std::max<size_t>(k0 * k, 1) * el);
  }
  if (cudaMalloc(&ops->buf, total) != cudaSuccess) {
    cudaGetLastError();
    ops->buf = nullptr;
    return THO_ERR_NOMEM;
  }
  ops->inst.resize(count);
  unsigned char* b = static_cast<unsigned char*>(ops->buf);
  for (int i = 0; i < count; ++i) {
    const size_t n = (size_t)d[i].n, k0 = (size_t)d[i].k0, k = (size_t)d[i].k;
    unsigned char* V = b + off[i];
    unsigned char* A = V + al(n * k0 * el);
    unsigned char* Q = A + al(n * k * el);
    unsigned char* R = Q + al(n * k * el);
    unsigned char* S = R + al(k * k * el);
    ops->inst[i] = tho_instance_t{k0 ? V : nullptr, A, Q, R, k0 ? S : nullptr, (int64_t)n, (int64_t)n, (int64_t)n};
    // V and A, entries of magnitude below 1/sqrt(n) (Q, R and S are outputs).
    const double scale = 1.0 / std::sqrt((double)n);
    auto fill = [&](void* x, size_t elems, uint64_t seed) {
      const int64_t cnt = (int64_t)(elems * (el / 8));
      if (cnt > 0)
        k_tune_fill<<<(int)std::min<int64_t>((cnt + 255) / 256, 4096), 256, 0, st>>>(
            reinterpret_cast<double*>(x), cnt, seed, scale);
    };
    fill(V, n * k0, 0x5600000000ull + 2 * (uint64_t)i);
    fill(A, n * k, 0x5600000001ull + 2 * (uint64_t)i);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return THO_ERR_CUDA;
  return THO_OK;
}

tho_status_t run_once(tho_plan_t p, int32_t count, const Operands& ops, cudaStream_t st) {
  if (count == 1) {
    const tho_instance_t& x = ops.inst[0];
    return tho_orth(p, x.V, x.ldv, x.A, x.lda, x.Q, x.ldq, x.R, x.S, st);
  }
  return tho_orth_batched(p, ops.inst.data(), count, st);
}

// Median time per call of one candidate (one warm-up call, then 3 to 9 timed
// calls, about 0.3 s in all), and in *eff the choices the plan resolved.  Plan
// errors (UNSUPPORTED, NOMEM) come back as the status.
tho_status_t time_candidate(const tho_desc_t* d, int32_t count, const tho_tuning_t& t, const Operands& ops,
                            cudaStream_t st, double* ms, tho_tuning_t* eff) {
  tho_plan_t p = nullptr;
  tho_status_t s = tho_plan_tuned(d, count, &t, &p);
  if (s != THO_OK) return s;
  tho_plan_tuning(p, eff);
  constexpr int kMaxReps = 9;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) s = THO_ERR_CUDA;
  auto cleanup = [&]() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    tho_plan_destroy(p);
  };
  if (s == THO_OK) s = run_once(p, count, ops, st);  // warm-up (instantiates the batch graph)
  float first = 0.f;
  if (s == THO_OK) {
    if (cudaEventRecord(ev[0], st) != cudaSuccess) s = THO_ERR_CUDA;
    if (s == THO_OK) s = run_once(p, count, ops, st);
    if (s == THO_OK && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                        cudaEventElapsedTime(&first, ev[0], ev[1]) != cudaSuccess))
      s = THO_ERR_CUDA;
  }
  if (s != THO_OK) {
    cleanup();
    return s;
  }
  const int reps = (int)std::min<double>(kMaxReps, std::max<double>(3.0, std::floor(300.0 / std::max(first, 1e-3f))));
  std::vector<float> t_ms;
  t_ms.push_back(first);
  for (int r = 1; r < reps && s == THO_OK; ++r) {
    if (cudaEventRecord(ev[0], st) != cudaSuccess) s = THO_ERR_CUDA;
    if (s == THO_OK) s = run_once(p, count, ops, st);
    float x = 0.f;
    if (s == THO_OK && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                        cudaEventElapsedTime(&x, ev[0], ev[1]) != cudaSuccess))
      s = THO_ERR_CUDA;
    t_ms.push_back(x);
  }
  cleanup();
  if (s != THO_OK) return s;
  std::sort(t_ms.begin(), t_ms.end());
  *ms = t_ms[t_ms.size() / 2];
  return THO_OK;
}

}  // namespace

extern "C" {

tho_status_t tho_tune_key(const tho_desc_t* descs, int32_t count, const char* device_name, char* buf,
                          size_t len) {
  if (!descs || count < 1 || !device_name || !buf) return THO_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (descs[i].n < 1) return THO_ERR_ARG;
  const std::string k = make_key(descs, count, device_name);
  if (k.size() + 1 > len) return THO_ERR_ARG;
  std::memcpy(buf, k.c_str(), k.size() + 1);
  return THO_OK;
}

tho_status_t tho_tune_cache_get(const char* path, const char* key, tho_tuning_t* out, double* ms,
                                int32_t* found) {
  if (!path || !key || !out || !found) return THO_ERR_ARG;
  *found = 0;
  FILE* f = std::fopen(path, "r");
  if (!f) return THO_OK;
  std::string line;
  int ch;
  auto consider = [&]() {
    std::string k;
    tho_tuning_t t{};
    double m = 0;
    if (parse_line(line.c_str(), &k, &t, &m) && k == key) {
      *out = t;
      if (ms) *ms = m;
      *found = 1;
    }
    line.clear();
  };
  while ((ch = std::fgetc(f)) != EOF) {
    if (ch == '\n')
      consider();
    else
      line.push_back((char)ch);
  }
  if (!line.empty()) consider();
  std::fclose(f);
  return THO_OK;
}

tho_status_t tho_tune_cache_put(const char* path, const char* key, const tho_tuning_t* t, double ms) {
  if (!path || !key || !t) return THO_ERR_ARG;
  for (const char* c = key; *c; ++c)
    if (!key_char_ok(*c)) return THO_ERR_ARG;
  char tail[160];
  std::snprintf(tail, sizeof(tail), "\", \"leaf_rows\": %d, \"split_chunks\": %d, \"balance\": %d, \"ms\": %.6f}\n",
                t->leaf_rows, t->split_chunks, t->balance, std::isfinite(ms) ? ms : 0.0);
  const std::string line = std::string("{\"key\": \"") + key + tail;
  FILE* f = std::fopen(path, "a");
  if (!f) return THO_ERR_ARG;
  // One write per entry, so that entries appended by concurrent processes stay whole lines.
  const bool ok = std::fwrite(line.data(), 1, line.size(), f) == line.size();
  return (std::fclose(f) == 0 && ok) ? THO_OK : THO_ERR_ARG;
}

tho_status_t tho_autotune(const tho_desc_t* descs, int32_t count, const char* cache_path, void* stream,
                          tho_tuning_t* out, double* ms) {
  if (!descs || count < 1 || !out) return THO_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return THO_ERR_CUDA;
  // The default plan validates the descriptors and gives the baseline.
  const char* path = cache_path ? cache_path : std::getenv("THO_TUNE_CACHE");
  if (path && !*path) path = nullptr;
  const std::string key = make_key(descs, count, prop.name);
  if (path) {
    tho_tuning_t t{};
    double m = 0;
    int32_t found = 0;
    if (tho_tune_cache_get(path, key.c_str(), &t, &m, &found) == THO_OK && found) {
      tho_plan_t p = nullptr;
      if (tho_plan_tuned(descs, count, &t, &p) == THO_OK) {
        tho_plan_destroy(p);
        *out = t;
        if (ms) *ms = m;
        return THO_OK;
      }
    }
  }
  Operands ops;
  tho_status_t s = THO_OK;
  {
    // Descriptor errors before any allocation.
    tho_plan_t p = nullptr;
    s = tho_plan_tuned(descs, count, nullptr, &p);
    if (s != THO_OK) return s;
    tho_plan_destroy(p);
  }
  s = make_operands(descs, count, st, &ops);
  if (s != THO_OK) return s;
  tho_tuning_t def{}, eff{};
  double def_ms = 0;
  s = time_candidate(descs, count, tho_tuning_t{0, 0, 0}, ops, st, &def_ms, &def);
  if (s != THO_OK) return s;
  tho_tuning_t best = def;
  double best_ms = def_ms;
  const char* lg = std::getenv("THO_LOG");
  const bool log = lg && *lg && std::strcmp(lg, "0") != 0;
  if (log)
    std::fprintf(stderr, "[tho] tune: default leaf_rows=%d split_chunks=%d -> %.3f ms\n", def.leaf_rows,
                 def.split_chunks, def_ms);
  auto consider = [&](const tho_tuning_t& t) -> tho_status_t {
    double m = 0;
    tho_status_t r = time_candidate(descs, count, t, ops, st, &m, &eff);
    if (log)
      std::fprintf(stderr, "[tho] tune: leaf_rows=%d split_chunks=%d balance=%d -> %s %.3f ms\n", t.leaf_rows,
                   t.split_chunks, t.balance, r == THO_OK ? "ok" : tho_status_string(r), r == THO_OK ? m : 0.0);
    if (r == THO_ERR_UNSUPPORTED || r == THO_ERR_NOMEM) return THO_OK;  // not a valid candidate here
    if (r != THO_OK) return r;
    if (m < best_ms) {
      best_ms = m;
      best = eff;
    }
    return THO_OK;
  };
  // Split-n factor at the default leaf height.
  std::vector<int> splits = {sms / 2, sms - 1, 2 * sms - 1, 4 * sms, 8 * sms, 16 * sms, 32 * sms, 64 * sms};
  std::sort(splits.begin(), splits.end());
  splits.erase(std::unique(splits.begin(), splits.end()), splits.end());
  for (int sp : splits) {
    if (sp < 1 || sp > THO_TUNE_MAX_SPLIT || sp == def.split_chunks) continue;
    if ((s = consider(tho_tuning_t{def.leaf_rows, sp, 0})) != THO_OK) return s;
  }
  // Leaf height at the best split.
  const int32_t split_best = best.split_chunks;
  for (int P : {64, 128, 256}) {
    if (P == def.leaf_rows) continue;
    if ((s = consider(tho_tuning_t{P, split_best, 0})) != THO_OK) return s;
  }
  // Batches: chunks shared by streaming work instead of rows.
  if (count > 1 && (s = consider(tho_tuning_t{best.leaf_rows, best.split_chunks, 1})) != THO_OK) return s;
  // Keep the default unless a candidate is clearly faster (timing noise).
  if (best_ms > 0.98 * def_ms) {
    best = def;
    best_ms = def_ms;
  }
  *out = best;
  if (ms) *ms = best_ms;
  if (log)
    std::fprintf(stderr, "[tho] tune: chose leaf_rows=%d split_chunks=%d balance=%d (%.3f ms)\n", best.leaf_rows,
                 best.split_chunks, best.balance, best_ms);
  if (path) tho_tune_cache_put(path, key.c_str(), &best, best_ms);
  return THO_OK;
}

}  // extern "C"
