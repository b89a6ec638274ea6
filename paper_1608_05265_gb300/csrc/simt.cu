// Plain FP32 SIMT sgemm (CUDA-core fused multiply-add), one launch per
// problem, and the C := beta*C kernel.  The tile computation is in
// simt_device.cuh.
#include "simt_device.cuh"

namespace gbg {
namespace {

// 256-thread tiles keep two blocks per SM (at most 128 registers a thread).
template <int BM, int BN, bool TA, bool TB, bool VEC>
__global__ void __launch_bounds__((BM / 8) * (BN / 8), 512 / ((BM / 8) * (BN / 8)))
sgemm_simt_kernel(Problem P) {
  __shared__ __align__(16) SimtSmem<BM, BN> sm;
  simt_tile<BM, BN, TA, TB, VEC>(P, (int64_t)blockIdx.x * BM, (int64_t)blockIdx.y * BN, sm.As, sm.Bs);
}

template <int BM, int BN>
cudaError_t launch_cfg(const Problem& p, cudaStream_t s) {
  const bool vec = ((p.lda & 3) == 0) && ((p.ldb & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(p.A) & 15) == 0) && ((reinterpret_cast<uintptr_t>(p.B) & 15) == 0);
  dim3 grid((unsigned)((p.m + BM - 1) / BM), (unsigned)((p.n + BN - 1) / BN));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  dim3 block((BM / 8) * (BN / 8));
#define GBG_SIMT_CASE(TA, TB, V)                                                      \
  if (p.ta == TA && p.tb == TB && vec == V) {                                          \
    sgemm_simt_kernel<BM, BN, TA, TB, V><<<grid, block, 0, s>>>(p);                    \
    return cudaGetLastError();                                                         \
  }
  GBG_SIMT_CASE(0, 0, true) GBG_SIMT_CASE(0, 1, true) GBG_SIMT_CASE(1, 0, true) GBG_SIMT_CASE(1, 1, true)
  GBG_SIMT_CASE(0, 0, false) GBG_SIMT_CASE(0, 1, false) GBG_SIMT_CASE(1, 0, false) GBG_SIMT_CASE(1, 1, false)
#undef GBG_SIMT_CASE
  return cudaErrorInvalidValue;
}

__global__ void scale_c_kernel(int64_t m, int64_t n, float beta, float* C, int64_t ldc) {
  const int64_t total = m * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % m, j = t / m;
    float* c = C + i + j * ldc;
    *c = (beta == 0.f) ? 0.f : beta * *c;
  }
}

}  // namespace

cudaError_t launch_simt(const Problem& p, int config, cudaStream_t s) {
  switch (config) {
    case SIMT_128x128: return launch_cfg<128, 128>(p, s);
    case SIMT_64x64: return launch_cfg<64, 64>(p, s);
    case SIMT_128x64: return launch_cfg<128, 64>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_scale_c(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const int64_t total = m * n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  scale_c_kernel<<<(unsigned)blocks, 256, 0, s>>>(m, n, beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace gbg
