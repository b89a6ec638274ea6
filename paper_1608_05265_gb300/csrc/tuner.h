// Autotuner interface (tuner.cu).
#pragma once

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "internal.h"

namespace gbg {

struct TuneResult {
  float latency_us[GBGEMM_NUM_CONFIGS];  // -1 for an illegal configuration
  float cost_us[GBGEMM_NUM_CONFIGS];     // GPU time per problem inside a grouped batch
};

// Cache key of a problem: m n k, transposes, 16-byte alignment class of A, B, C.
std::string tune_key(const gbgemm_problem& q);
// Lowest-latency (by_cost = false) or lowest-cost configuration; -1 if none.
int best_config(const TuneResult& r, bool by_cost);

class Tuner {
 public:
  ~Tuner();
  void bind(cudaStream_t s, int* status, int num_sms) { stream_ = s; status_ = status; num_sms_ = num_sms; }
  // Time every legal configuration of q's shape (cached).  Synchronises the stream.
  int measure(const gbgemm_problem& q, int reps, TuneResult* out);
  // Latency of every legal single-call schedule of q's shape (GBGEMM_NUM_SCHEDULES
  // entries, -1 illegal; cached).  Synchronises the stream.
  int measure_schedules(const gbgemm_problem& q, int reps, std::vector<float>* out);
  int save(const char* path) const;
  int load(const char* path);
  std::map<std::string, TuneResult> cache;
  std::map<std::string, std::vector<float>> sched_cache;

 private:
  int ensure(size_t bytes);
  int scratch(const gbgemm_problem& q0, size_t ws_bytes, gbgemm_problem* q, uint8_t** wsp);
  int time_us(const std::function<cudaError_t()>& run, int reps, float* us);
  cudaStream_t cap_stream();
  cudaStream_t cap_ = nullptr;           // capture stream of the replica plans
  cudaStream_t stream_ = nullptr;
  int* status_ = nullptr;
  int num_sms_ = 148;
  void* buf_ = nullptr;
  size_t buf_bytes_ = 0;
  cudaEvent_t e0_ = nullptr, e1_ = nullptr;
};

}  // namespace gbg
