// Learned configuration predictor (mlp.cu).
#pragma once

#include "internal.h"

namespace gbg {

// Feature vector (8 floats) of a problem: log2 m/14, log2 n/14, log2 k/14,
// transa, transb, alignment classes of A, B, C.
void predictor_features(const gbgemm_problem& q, float* x);

class Predictor {
 public:
  // outputs: GBGEMM_NUM_CONFIGS (grouped configurations) or
  // GBGEMM_NUM_SCHEDULES (single-call schedules)
  explicit Predictor(int outputs = GBGEMM_NUM_CONFIGS);
  ~Predictor();
  Predictor(const Predictor&) = delete;
  Predictor& operator=(const Predictor&) = delete;
  bool ready() const { return ready_; }
  int outputs() const { return out_; }
  int params() const;  // parameter count
  int set(const float* host_params);
  int get(float* host_params) const;
  // Device arrays: dx[n][8]; dlegal[n][(outputs + 7) / 8], bit c % 8 of
  // byte c / 8 = output c allowed; dscores[n][outputs] (may be NULL);
  // dconfigs[n].  Asynchronous on s.
  int predict(const float* dx, const uint8_t* dlegal, int64_t n, float* dscores, int* dconfigs, cudaStream_t s) const;
  // Mean masked squared error of n <= 256 samples and its gradient (device dgrad).
  int loss_grad(const float* dx, const float* dy, const float* dmask, int64_t n, float* host_loss, float* dgrad,
                cudaStream_t s) const;
  // Adam on mini-batches; starts from He-uniform weights (seeded) when no
  // parameters are set.  Synchronises s.
  int train(const float* dx, const float* dy, const float* dmask, int64_t n, int epochs, int batch, float lr,
            uint64_t seed, float* host_loss, cudaStream_t s);

 private:
  int out_;
  float* dparams_ = nullptr;
  bool ready_ = false;
};

}  // namespace gbg
