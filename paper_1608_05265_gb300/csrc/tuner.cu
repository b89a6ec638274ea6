// Autotuner: times every legal configuration of a problem shape on the GPU
// (CUDA events, median of `reps` runs after one warm-up) and keeps the
// results in a per-handle cache keyed by shape, transposes and leading-
// dimension alignment.
//
// The paper fixes its micro-kernel sizes (m, n, KSUB, NSUB, CORES) at compile
// time (Section III-C, III-D); here the tile shape and path are chosen per
// shape at run time by measurement.
//
// Each configuration gets two numbers:
//   latency  time of one gbgemm_sgemm-style call of that configuration on
//            that problem alone (CUDA events around the launches);
//   cost     GPU time the problem takes inside a grouped batch: a grouped
//            plan of R copies of the problem (R sized so that the copies
//            fill every SM twice, at most 256) is captured and replayed,
//            and cost = replay time / R.  Launch latencies and partly idle
//            GPUs, which dominate the latency of small problems, vanish in a
//            batch, and so they do here.
// The single-problem path ranks by latency, grouped plans by cost.
// Timing runs on scratch buffers owned by the tuner, never on caller data
// (the copies share them; they write identical values).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "grouped.h"
#include "tuner.h"

namespace gbg {
namespace {

__global__ void fill_uniform_kernel(float* x, size_t n, uint32_t seed) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
    x[i] = (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
  }
}

int blocks_per_sm(int cfg) {
  switch (cfg) {
    case GBGEMM_CFG_SIMT_128x128: return 2;
    case GBGEMM_CFG_SIMT_64x64: return 4;
    case GBGEMM_CFG_SIMT_128x64: return 3;
    default: return 1;
  }
}

int64_t tiles_of(const gbgemm_problem& q, int cfg) {
  int bm = 128, bn = 128;
  if (cfg == GBGEMM_CFG_SIMT_64x64) { bm = 64; bn = 64; }
  else if (cfg == GBGEMM_CFG_SIMT_128x64) { bm = 128; bn = 64; }
  else if (cfg == GBGEMM_CFG_SPLIT_BN64) bn = 64;
  else if (cfg == GBGEMM_CFG_SPLIT_BN256) bn = 256;
  return ((q.m + bm - 1) / bm) * ((q.n + bn - 1) / bn);
}

int align_class(int64_t ld, const void* p) {
  return ((ld & 3) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) ? 1 : 0;
}

}  // namespace

std::string tune_key(const gbgemm_problem& q) {
  char buf[160];
  const int ta = (q.transa == 'N' || q.transa == 'n') ? 0 : 1;
  const int tb = (q.transb == 'N' || q.transb == 'n') ? 0 : 1;
  std::snprintf(buf, sizeof(buf), "%lld %lld %lld %d %d %d %d %d", (long long)q.m, (long long)q.n, (long long)q.k, ta,
                tb, align_class(q.lda, q.A), align_class(q.ldb, q.B), align_class(q.ldc, q.C));
  return std::string(buf);
}

Tuner::~Tuner() {
  if (cap_) cudaStreamDestroy(cap_);
  if (buf_) cudaFree(buf_);
  if (e0_) cudaEventDestroy(e0_);
  if (e1_) cudaEventDestroy(e1_);
}

int Tuner::ensure(size_t bytes) {
  if (!e0_ && (cudaEventCreate(&e0_) != cudaSuccess || cudaEventCreate(&e1_) != cudaSuccess)) return GBGEMM_ERR_CUDA;
  if (bytes <= buf_bytes_) return GBGEMM_OK;
  if (buf_) cudaFree(buf_);
  buf_ = nullptr;
  buf_bytes_ = 0;
  if (cudaMalloc(&buf_, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GBGEMM_ERR_ALLOC;
  }
  buf_bytes_ = bytes;
  fill_uniform_kernel<<<1024, 256, 0, stream_>>>(static_cast<float*>(buf_), bytes / 4, 0x9E3779B9u);
  return cudaGetLastError() == cudaSuccess ? GBGEMM_OK : GBGEMM_ERR_CUDA;
}

// Scratch operands with q0's shape, leading dimensions and 16-byte alignment
// classes, followed by ws_bytes of split workspace.
int Tuner::scratch(const gbgemm_problem& q0, size_t ws_bytes, gbgemm_problem* q, uint8_t** wsp) {
  const int ta = (q0.transa == 'N' || q0.transa == 'n') ? 0 : 1;
  const int tb = (q0.transb == 'N' || q0.transb == 'n') ? 0 : 1;
  // scratch layout: A | B | C | split workspace (panels, maxima); same leading dimensions as the problem
  const int64_t acols = ta ? q0.m : q0.k, bcols = tb ? q0.k : q0.n;
  const size_t a_bytes = (size_t)q0.lda * std::max<int64_t>(acols, 1) * 4 + 16;
  const size_t b_bytes = (size_t)q0.ldb * std::max<int64_t>(bcols, 1) * 4 + 16;
  const size_t c_bytes = (size_t)q0.ldc * std::max<int64_t>(q0.n, 1) * 4 + 16;
  auto r256 = [](size_t x) { return (x + 255) / 256 * 256; };
  int rc = ensure(r256(a_bytes) + r256(b_bytes) + r256(c_bytes) + ws_bytes);
  if (rc != GBGEMM_OK) return rc;
  uint8_t* base = static_cast<uint8_t*>(buf_);
  // keep the problem's 16-byte alignment class
  const size_t aoff = (reinterpret_cast<uintptr_t>(q0.A) & 15), boff = (reinterpret_cast<uintptr_t>(q0.B) & 15);
  const size_t coff = (reinterpret_cast<uintptr_t>(q0.C) & 15);
  *q = q0;
  q->A = reinterpret_cast<const float*>(base + aoff);
  q->B = reinterpret_cast<const float*>(base + r256(a_bytes) + boff);
  q->C = reinterpret_cast<float*>(base + r256(a_bytes) + r256(b_bytes) + coff);
  *wsp = base + r256(a_bytes) + r256(b_bytes) + r256(c_bytes);
  return GBGEMM_OK;
}

// Median of `reps` CUDA-event timings of run() after one warm-up, in us.
int Tuner::time_us(const std::function<cudaError_t()>& run, int reps, float* us) {
  if (run() != cudaSuccess) return GBGEMM_ERR_CUDA;  // warm-up
  std::vector<float> t;
  for (int r = 0; r < std::max(reps, 1); ++r) {
    if (cudaEventRecord(e0_, stream_) != cudaSuccess || run() != cudaSuccess || cudaEventRecord(e1_, stream_) != cudaSuccess ||
        cudaEventSynchronize(e1_) != cudaSuccess)
      return GBGEMM_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0_, e1_);
    t.push_back(ms * 1000.f);
  }
  std::sort(t.begin(), t.end());
  *us = t[t.size() / 2];
  return GBGEMM_OK;
}

int Tuner::measure_schedules(const gbgemm_problem& q0, int reps, std::vector<float>* out) {
  const std::string key = tune_key(q0);
  auto it = sched_cache.find(key);
  if (it != sched_cache.end()) {
    *out = it->second;
    return GBGEMM_OK;
  }
  const int ta = (q0.transa == 'N' || q0.transa == 'n') ? 0 : 1;
  const int tb = (q0.transb == 'N' || q0.transb == 'n') ? 0 : 1;
  size_t ws = 0;  // the largest split workspace of the legal schedules
  for (int sc = 0; sc < GBGEMM_NUM_SCHEDULES; ++sc) {
    Schedule d;
    if (schedule_resolve(sc, q0.m, q0.n, q0.k, q0.alpha, num_sms_, &d) && d.path == GBGEMM_PATH_SPLIT_BF16)
      ws = std::max(ws, split_layout(q0.m, q0.n, q0.k, 1, d.splitk, d.bn).total);
  }
  gbgemm_problem q;
  uint8_t* wsp = nullptr;
  int rc = scratch(q0, ws, &q, &wsp);
  if (rc != GBGEMM_OK) return rc;
  Problem p{ta, tb, q.m, q.n, q.k, 1.0f, 0.0f, q.A, q.lda, q.B, q.ldb, q.C, q.ldc};
  std::vector<float> lat((size_t)GBGEMM_NUM_SCHEDULES, -1.f);
  for (int sc = 0; sc < GBGEMM_NUM_SCHEDULES; ++sc) {
    Schedule d;
    if (!schedule_resolve(sc, q.m, q.n, q.k, q.alpha, num_sms_, &d)) continue;
    auto run = [&]() -> cudaError_t {
      if (d.path == GBGEMM_PATH_SIMT) return launch_simt(p, d.simt_cfg, stream_);
      SplitCall c;
      c.ta = ta; c.tb = tb; c.m = q.m; c.n = q.n; c.k = q.k; c.alpha = 1.0f; c.beta = 0.0f;
      c.A = q.A; c.lda = q.lda; c.B = q.B; c.ldb = q.ldb; c.C = q.C; c.ldc = q.ldc;
      c.bn = d.bn; c.raster = d.raster; c.splitk = d.splitk;
      c.ws = wsp; c.status = status_; c.num_sms = num_sms_;
      return launch_split_call(c, stream_);
    };
    rc = time_us(run, reps, &lat[(size_t)sc]);
    if (rc != GBGEMM_OK) return rc;
  }
  sched_cache[key] = lat;
  *out = lat;
  return GBGEMM_OK;
}

int Tuner::measure(const gbgemm_problem& q0, int reps, TuneResult* out) {
  const std::string key = tune_key(q0);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return GBGEMM_OK;
  }
  const int ta = (q0.transa == 'N' || q0.transa == 'n') ? 0 : 1;
  const int tb = (q0.transb == 'N' || q0.transb == 'n') ? 0 : 1;
  size_t ws = 0;  // the largest split workspace of the three tile widths
  for (int bn : {64, 128, 256}) ws = std::max(ws, split_layout(q0.m, q0.n, q0.k, 1, 1, bn).total);
  gbgemm_problem q;
  uint8_t* wsp = nullptr;
  int rc = scratch(q0, ws, &q, &wsp);
  if (rc != GBGEMM_OK) return rc;
  const float* A = q.A;
  const float* B = q.B;
  float* C = q.C;
  Problem p{ta, tb, q0.m, q0.n, q0.k, 1.0f, 0.0f, A, q0.lda, B, q0.ldb, C, q0.ldc};

  TuneResult res;
  for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c) { res.latency_us[c] = -1.f; res.cost_us[c] = -1.f; }
  for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c) {
    if (!config_legal(q, c)) continue;
    auto run = [&]() -> cudaError_t {
      if (c < GBGEMM_CFG_SPLIT_BN64) return launch_simt(p, c, stream_);
      SplitCall sc;
      sc.ta = ta; sc.tb = tb; sc.m = q.m; sc.n = q.n; sc.k = q.k; sc.alpha = 1.0f; sc.beta = 0.0f;
      sc.A = A; sc.lda = q.lda; sc.B = B; sc.ldb = q.ldb; sc.C = C; sc.ldc = q.ldc;
      sc.bn = c == GBGEMM_CFG_SPLIT_BN64 ? 64 : c == GBGEMM_CFG_SPLIT_BN128 ? 128 : 256;
      sc.raster = 16;
      sc.ws = wsp; sc.status = status_; sc.num_sms = num_sms_;
      return launch_split_call(sc, stream_);
    };
    rc = time_us(run, reps, &res.latency_us[c]);
    if (rc != GBGEMM_OK) return rc;
    // batch cost: replicas of the problem in one captured grouped plan
    const double slots = (double)num_sms_ * blocks_per_sm(c);
    const int64_t reps_in_batch =
        std::max<int64_t>(1, std::min<int64_t>(256, (int64_t)std::ceil(2.0 * slots / (double)tiles_of(q, c))));
    std::vector<gbgemm_problem> copies((size_t)reps_in_batch, q);
    std::vector<int> cfgs((size_t)reps_in_batch, c);
    GroupedPlan plan;
    plan.device = 0;
    cudaGetDevice(&plan.device);
    plan.num_sms = num_sms_;
    plan.status = status_;
    plan.count = reps_in_batch;
    if (build_grouped_plan(&plan, copies.data(), reps_in_batch, cfgs.data(), cap_stream()) != GBGEMM_OK)
      return GBGEMM_ERR_CUDA;
    if (cudaGraphLaunch(plan.exec, stream_) != cudaSuccess) return GBGEMM_ERR_CUDA;  // warm-up
    std::vector<float> tb;
    for (int r = 0; r < std::max(reps, 1); ++r) {
      if (cudaEventRecord(e0_, stream_) != cudaSuccess || cudaGraphLaunch(plan.exec, stream_) != cudaSuccess ||
          cudaEventRecord(e1_, stream_) != cudaSuccess || cudaEventSynchronize(e1_) != cudaSuccess)
        return GBGEMM_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0_, e1_);
      tb.push_back(ms * 1000.f / (float)reps_in_batch);
    }
    std::sort(tb.begin(), tb.end());
    res.cost_us[c] = tb[tb.size() / 2];
  }
  cache[key] = res;
  *out = res;
  return GBGEMM_OK;
}

cudaStream_t Tuner::cap_stream() {
  if (!cap_) cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking);
  return cap_;
}

int best_config(const TuneResult& r, bool by_cost) {
  int best = -1;
  for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c) {
    const float v = by_cost ? r.cost_us[c] : r.latency_us[c];
    if (v < 0.f) continue;
    const float b = best < 0 ? 0.f : (by_cost ? r.cost_us[best] : r.latency_us[best]);
    if (best < 0 || v < b) best = c;  // ties keep the lower index
  }
  return best;
}

int Tuner::save(const char* path) const {
  FILE* f = std::fopen(path, "w");
  if (!f) return GBGEMM_ERR_INVALID_VALUE;
  std::fprintf(f, "# gbgemm tuning cache v1: m n k ta tb alignA alignB alignC | latency_us x6 | cost_us x6\n");
  for (const auto& kv : cache) {
    std::fprintf(f, "%s |", kv.first.c_str());
    for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c) std::fprintf(f, " %.4f", kv.second.latency_us[c]);
    std::fprintf(f, " |");
    for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c) std::fprintf(f, " %.4f", kv.second.cost_us[c]);
    std::fprintf(f, "\n");
  }
  // schedule latencies: "S key | latency_us x GBGEMM_NUM_SCHEDULES"
  for (const auto& kv : sched_cache) {
    std::fprintf(f, "S %s |", kv.first.c_str());
    for (float v : kv.second) std::fprintf(f, " %.4f", v);
    std::fprintf(f, "\n");
  }
  std::fclose(f);
  return GBGEMM_OK;
}

int Tuner::load(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return GBGEMM_ERR_INVALID_VALUE;
  char line[1024];
  int rc = GBGEMM_OK;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    if (line[0] == 'S' && line[1] == ' ') {
      char* bar = std::strchr(line, '|');
      if (!bar) { rc = GBGEMM_ERR_INVALID_VALUE; break; }
      std::string key(line + 2, bar - line - 2);
      while (!key.empty() && key.back() == ' ') key.pop_back();
      std::vector<float> lat((size_t)GBGEMM_NUM_SCHEDULES);
      bool ok = true;
      char* sp = bar + 1;
      for (int c = 0; c < GBGEMM_NUM_SCHEDULES && ok; ++c) {
        char* end = nullptr;
        lat[(size_t)c] = std::strtof(sp, &end);
        ok = end != sp;
        sp = end;
      }
      if (!ok) { rc = GBGEMM_ERR_INVALID_VALUE; break; }
      sched_cache[key] = lat;
      continue;
    }
    char* bar = std::strchr(line, '|');
    char* bar2 = bar ? std::strchr(bar + 1, '|') : nullptr;
    if (!bar2) { rc = GBGEMM_ERR_INVALID_VALUE; break; }
    std::string key(line, bar - line);
    while (!key.empty() && key.back() == ' ') key.pop_back();
    TuneResult r;
    bool ok = true;
    char* s = bar + 1;
    for (int c = 0; c < GBGEMM_NUM_CONFIGS && ok; ++c) {
      char* end = nullptr;
      r.latency_us[c] = std::strtof(s, &end);
      ok = end != s;
      s = end;
    }
    s = bar2 + 1;
    for (int c = 0; c < GBGEMM_NUM_CONFIGS && ok; ++c) {
      char* end = nullptr;
      r.cost_us[c] = std::strtof(s, &end);
      ok = end != s;
      s = end;
    }
    if (!ok) { rc = GBGEMM_ERR_INVALID_VALUE; break; }
    cache[key] = r;
  }
  std::fclose(f);
  return rc;
}

}  // namespace gbg
