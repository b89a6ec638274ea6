// Internal interface of the grouped sgemm plan (grouped.cu), used by the C
// ABI front end (api.cu) and the autotuner.
#pragma once

#include "internal.h"

namespace gbg {

struct GroupedPlan {
  int device = 0;
  int num_sms = 0;
  int* status = nullptr;          // device status word (the handle's)
  void* dmem = nullptr;           // one allocation: panels, maxima, descriptors, work lists
  size_t dbytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t count = 0;              // problems given
  int64_t n_split = 0, n_simt = 0;
  int64_t split_tiles = 0;
  int kernels_per_run = 0;
  double flops_split = 0.0, flops_simt = 0.0;
  int* configs = nullptr;         // host copy of the per-problem configuration (count entries)
  ~GroupedPlan();
};

// Argument check of one problem: 0, or minus the BLAS position of the first bad argument.
int validate_problem(const gbgemm_problem& q);
// Whether configuration `cfg` may run problem q (split configurations need k >= 16 and alpha != 0).
bool config_legal(const gbgemm_problem& q, int cfg);
// The heuristic configuration used when no tuner or predictor is asked for.
int default_config(const gbgemm_problem& q);
// Lay out device memory, upload descriptors and capture the graph on `capture_stream`.
int build_grouped_plan(GroupedPlan* P, const gbgemm_problem* probs, int64_t count, const int* configs,
                       cudaStream_t capture_stream);

}  // namespace gbg
