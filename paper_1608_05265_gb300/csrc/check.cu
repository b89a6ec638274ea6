// On-GPU FP64 error check of an sgemm result (test and benchmark tool; not
// part of the sgemm path, and the only FP64 arithmetic on the GPU).
//
// For every (i, j) of a block it recomputes the definition of the operation
// (Section III-A: C_out = alpha op(A) op(B) + beta C_in) with FP64 products
// and sums in p order, together with the acceptance bound
//     bound_ij = 2 max(k,1) 2^-24 (|alpha| sum_p |opA(i,p)||opB(p,j)| + |beta||C_in,ij|),
// and reduces max_ij |C_out,ij - C64_ij| / bound_ij (+inf when a zero bound is
// exceeded or the difference is NaN).
#include <cstring>

#include "internal.h"

namespace gbg {
namespace {

__device__ __forceinline__ void atomic_max_pos_double(unsigned long long* addr, double v) {
  // non-negative doubles (including +inf) order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void check_kernel(int ta, int tb, int64_t k, float alpha, const float* __restrict__ A, int64_t lda,
                             const float* __restrict__ B, int64_t ldb, float beta, const float* __restrict__ Cin,
                             const float* __restrict__ Cout, int64_t ldc, int64_t i0, int64_t i1, int64_t j0,
                             int64_t j1, unsigned long long* __restrict__ result) {
  const int64_t bm = i1 - i0;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= bm * (j1 - j0)) return;
  const int64_t i = i0 + idx % bm, j = j0 + idx / bm;
  const bool use_ab = (alpha != 0.f) && (k > 0);
  double s = 0.0, sabs = 0.0;
  if (use_ab) {
    for (int64_t p = 0; p < k; ++p) {
      const double a = (double)(ta ? A[p + i * lda] : A[i + p * lda]);
      const double b = (double)(tb ? B[j + p * ldb] : B[p + j * ldb]);
      s = fma(a, b, s);
      sabs = fma(fabs(a), fabs(b), sabs);
    }
  }
  const double c = (beta != 0.f) ? (double)Cin[i + j * ldc] : 0.0;
  const double ref = (use_ab ? (double)alpha * s : 0.0) + (beta != 0.f ? (double)beta * c : 0.0);
  const double bound = 2.0 * (double)(k > 1 ? k : 1) * 0x1p-24 *
                       ((use_ab ? fabs((double)alpha) * sabs : 0.0) + (beta != 0.f ? fabs((double)beta) * fabs(c) : 0.0));
  const double d = fabs((double)Cout[i + j * ldc] - ref);
  double r;
  if (d != d) r = __longlong_as_double(0x7FF0000000000000ll);        // NaN difference: +inf
  else if (bound == 0.0) r = (d == 0.0) ? 0.0 : __longlong_as_double(0x7FF0000000000000ll);
  else r = d / bound;
  atomic_max_pos_double(result, r);
}

}  // namespace
}  // namespace gbg

namespace gbg {

int run_error_check(cudaStream_t s, char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                    const float* A, int64_t lda, const float* B, int64_t ldb, float beta, const float* C_in,
                    const float* C_out, int64_t ldc, int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                    double* max_ratio) {
  auto tcode = [](char t) {
    switch (t) {
      case 'N': case 'n': return 0;
      case 'T': case 't': case 'C': case 'c': return 1;
      default: return -1;
    }
  };
  const int ta = tcode(transa), tb = tcode(transb);
  if (ta < 0 || tb < 0 || m < 0 || n < 0 || k < 0 || !max_ratio) return GBGEMM_ERR_INVALID_VALUE;
  if (i0 < 0 || j0 < 0 || i1 > m || j1 > n || i0 > i1 || j0 > j1) return GBGEMM_ERR_INVALID_VALUE;
  if (ldc < (m > 1 ? m : 1) || !C_out || (beta != 0.f && !C_in)) return GBGEMM_ERR_INVALID_VALUE;
  if (alpha != 0.f && k > 0 && (!A || !B)) return GBGEMM_ERR_INVALID_VALUE;
  *max_ratio = 0.0;
  const int64_t total = (i1 - i0) * (j1 - j0);
  if (total == 0) return GBGEMM_OK;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return GBGEMM_ERR_ALLOC;
  }
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    check_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ta, tb, k, alpha, A, lda, B, ldb, beta, C_in,
                                                                  C_out, ldc, i0, i1, j0, j1, d);
    e = cudaGetLastError();
  }
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return GBGEMM_ERR_CUDA;
  double r;
  memcpy(&r, &bits, sizeof(r));
  *max_ratio = r;
  return GBGEMM_OK;
}

}  // namespace gbg
