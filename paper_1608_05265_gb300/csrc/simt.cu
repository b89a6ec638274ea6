// Plain FP32 SIMT sgemm (CUDA-core fused multiply-add), one launch per
// problem, and the C := beta*C kernel.  The tile computation is in
// simt_device.cuh.
#include "simt_device.cuh"

namespace gbg {
namespace {

// 256-thread tiles keep two blocks per SM (at most 128 registers a thread).
// blockIdx.z selects the problem of a strided batch (A + z*sa, B + z*sb,
// C + z*sc; all 0 for one problem).
template <int BM, int BN, bool TA, bool TB, bool VEC>
__global__ void __launch_bounds__((BM / 8) * (BN / 8), 512 / ((BM / 8) * (BN / 8)))
sgemm_simt_kernel(Problem P, int64_t sa, int64_t sb, int64_t sc) {
  __shared__ __align__(16) SimtSmem<BM, BN> sm;
  const int64_t z = blockIdx.z;
  if (z > 0) {
    if (P.A) P.A += z * sa;
    if (P.B) P.B += z * sb;
    P.C += z * sc;
  }
  simt_tile<BM, BN, TA, TB, VEC>(P, (int64_t)blockIdx.x * BM, (int64_t)blockIdx.y * BN, sm.As, sm.Bs);
}

template <int BM, int BN>
cudaError_t launch_cfg(const Problem& p, int64_t batch, int64_t sa, int64_t sb, int64_t sc, cudaStream_t s) {
  // vector loads need every problem's A and B 16-byte aligned: strides multiples of 4
  const bool vec = ((p.lda & 3) == 0) && ((p.ldb & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(p.A) & 15) == 0) && ((reinterpret_cast<uintptr_t>(p.B) & 15) == 0) &&
                   (batch == 1 || (((sa & 3) == 0) && ((sb & 3) == 0)));
  dim3 grid((unsigned)((p.m + BM - 1) / BM), (unsigned)((p.n + BN - 1) / BN), (unsigned)batch);
  if (grid.y > 65535u || batch > 65535 || batch < 1) return cudaErrorInvalidConfiguration;
  dim3 block((BM / 8) * (BN / 8));
#define GBG_SIMT_CASE(TA, TB, V)                                                      \
  if (p.ta == TA && p.tb == TB && vec == V) {                                          \
    sgemm_simt_kernel<BM, BN, TA, TB, V><<<grid, block, 0, s>>>(p, sa, sb, sc);        \
    return cudaGetLastError();                                                         \
  }
  GBG_SIMT_CASE(0, 0, true) GBG_SIMT_CASE(0, 1, true) GBG_SIMT_CASE(1, 0, true) GBG_SIMT_CASE(1, 1, true)
  GBG_SIMT_CASE(0, 0, false) GBG_SIMT_CASE(0, 1, false) GBG_SIMT_CASE(1, 0, false) GBG_SIMT_CASE(1, 1, false)
#undef GBG_SIMT_CASE
  return cudaErrorInvalidValue;
}

__global__ void scale_c_kernel(int64_t m, int64_t n, float beta, float* C, int64_t ldc, int64_t batch, int64_t sc) {
  const int64_t per = m * n, total = per * batch;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = t / per, r = t - z * per;
    const int64_t i = r % m, j = r / m;
    float* c = C + z * sc + i + j * ldc;
    *c = (beta == 0.f) ? 0.f : beta * *c;
  }
}

}  // namespace

cudaError_t launch_simt(const Problem& p, int config, cudaStream_t s) {
  return launch_simt_batched(p, config, 1, 0, 0, 0, s);
}

cudaError_t launch_simt_batched(const Problem& p, int config, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                cudaStream_t s) {
  switch (config) {
    case SIMT_128x128: return launch_cfg<128, 128>(p, batch, sa, sb, sc, s);
    case SIMT_64x64: return launch_cfg<64, 64>(p, batch, sa, sb, sc, s);
    case SIMT_128x64: return launch_cfg<128, 64>(p, batch, sa, sb, sc, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_scale_c(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t s) {
  return launch_scale_c_batched(m, n, beta, C, ldc, 1, 0, s);
}

cudaError_t launch_scale_c_batched(int64_t m, int64_t n, float beta, float* C, int64_t ldc, int64_t batch,
                                   int64_t sc, cudaStream_t s) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  const int64_t total = m * n * batch;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  scale_c_kernel<<<(unsigned)blocks, 256, 0, s>>>(m, n, beta, C, ldc, batch, sc);
  return cudaGetLastError();
}

}  // namespace gbg
