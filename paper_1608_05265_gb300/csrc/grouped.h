// Internal interface of the grouped sgemm plan (grouped.cu), used by the C
// ABI front end (api.cu) and the autotuner.
#pragma once

#include <vector>

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
  bool fused = true;              // packing inside the GEMM kernel (panel ring) or by a launch ahead of it
  size_t ring_bytes = 0;          // requested panel ring (0: kGroupedRingBytes)
  size_t ring_used = 0;           // ring bytes of the built plan
  ~GroupedPlan();
};

// Default size of a grouped plan's panel ring: well inside L2, so that
// panels are read back from L2 by the GEMM.
constexpr size_t kGroupedRingBytes = (size_t)64 << 20;

// Argument check of one problem: 0, or minus the BLAS position of the first bad argument.
int validate_problem(const gbgemm_problem& q);
// Whether configuration `cfg` may run problem q (split configurations need k >= 128 and alpha != 0).
bool config_legal(const gbgemm_problem& q, int cfg);
// The heuristic configuration used when no tuner or predictor is asked for.
int default_config(const gbgemm_problem& q);
// Panel ring layout: regions of `sizes` bytes (multiples of `granule`, none
// larger than `ring`) placed one after another in packing order, wrapping
// to offset 0 when the next one does not fit; wait list of region i: the
// distinct earlier regions that last wrote one of its granules (those must
// have been read before region i is rewritten).
void ring_layout(const std::vector<size_t>& sizes, size_t ring, size_t granule, std::vector<size_t>& off,
                 std::vector<int>& wait_begin, std::vector<int>& wait_count, std::vector<int>& wait_list);
// Lay out device memory, upload descriptors and capture the graph on `capture_stream`.
int build_grouped_plan(GroupedPlan* P, const gbgemm_problem* probs, int64_t count, const int* configs,
                       cudaStream_t capture_stream);

}  // namespace gbg
