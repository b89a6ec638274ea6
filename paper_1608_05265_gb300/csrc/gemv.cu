// FP32 sgemv, y := alpha op(A) x + beta y (BLAS convention): the Level-2
// operation the paper names as the weak point of its HPL run (Section IV-C,
// V).  Memory-bound: every element of A is read once from HBM, in coalesced
// order, with several independent loads in flight per thread.
//
//   op(A) = A   ("N"): a thread owns one row i and runs over a slice of the
//               columns; x comes through shared memory.  y_i needs the whole
//               row, so when the rows alone give too few blocks the columns
//               are cut into slices whose partial sums a reduction adds in
//               slice order.
//   op(A) = A^T ("T"): a block owns four columns j and runs over a slice of
//               the rows (consecutive rows of a column are consecutive in
//               memory); each x_i is read once for the four columns, and the
//               block's threads are combined in a fixed order.
//
// Every sum is formed in the same order on every run (no atomics).
#include "internal.h"

namespace gbg {
namespace {

constexpr int kGemvThreads = 256;
constexpr int kXChunk = 1024;  // x values staged in shared memory at a time ("N")
constexpr int kTCols = 4;      // columns per block ("T")

// Element e of a BLAS vector of length len with increment inc (inc < 0: the
// vector runs backwards from the end of the storage).
__device__ __forceinline__ int64_t vec_index(int64_t e, int64_t len, int64_t inc) {
  return inc > 0 ? e * inc : (len - 1 - e) * (-inc);
}

// Partial (or final) y_i over columns [j0, j1): thread per row.
__global__ void __launch_bounds__(kGemvThreads) gemv_n_kernel(int64_t m, int64_t n, const float* __restrict__ A,
                                                              int64_t lda, const float* __restrict__ x, int64_t incx,
                                                              int64_t slice, float* __restrict__ partial,
                                                              float alpha, float beta, float* __restrict__ y,
                                                              int64_t incy) {
  __shared__ float xs[kXChunk];
  const int64_t i = (int64_t)blockIdx.x * kGemvThreads + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * slice;
  const int64_t j1 = (j0 + slice < n) ? j0 + slice : n;
  const bool row = i < m;
  const float* a = A + (row ? i : 0);
  float acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.f;
  for (int64_t jc = j0; jc < j1; jc += kXChunk) {
    const int nj = (int)((j1 - jc < kXChunk) ? j1 - jc : kXChunk);
    __syncthreads();  // the previous chunk is no longer read
    for (int t = threadIdx.x; t < nj; t += kGemvThreads) xs[t] = x[vec_index(jc + t, n, incx)];
    __syncthreads();
    if (row) {
      const float* col = a + jc * lda;
      int t = 0;
      for (; t + 8 <= nj; t += 8) {  // eight independent loads in flight
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fmaf(col[(int64_t)(t + u) * lda], xs[t + u], acc[u]);
      }
      for (; t < nj; ++t) acc[0] = fmaf(col[(int64_t)t * lda], xs[t], acc[0]);
    }
  }
  if (!row) return;
  const float s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  if (partial) {
    partial[(int64_t)blockIdx.y * m + i] = s;
  } else {
    float* yi = y + vec_index(i, m, incy);
    *yi = (beta != 0.f) ? fmaf(alpha, s, beta * *yi) : alpha * s;
  }
}

// Partial (or final) y_j for columns j .. j+3 over rows [i0, i1).
__global__ void __launch_bounds__(kGemvThreads) gemv_t_kernel(int64_t m, int64_t n, const float* __restrict__ A,
                                                              int64_t lda, const float* __restrict__ x, int64_t incx,
                                                              int64_t slice, float* __restrict__ partial,
                                                              float alpha, float beta, float* __restrict__ y,
                                                              int64_t incy) {
  __shared__ float red[kTCols][kGemvThreads / 32];
  const int64_t jb = (int64_t)blockIdx.x * kTCols;
  const int64_t i0 = (int64_t)blockIdx.y * slice;
  const int64_t i1 = (i0 + slice < m) ? i0 + slice : m;
  const int nc = (int)((n - jb < kTCols) ? n - jb : kTCols);
  float acc[kTCols][2];
#pragma unroll
  for (int c = 0; c < kTCols; ++c) acc[c][0] = acc[c][1] = 0.f;
  int64_t i = i0 + threadIdx.x;
  for (; i + kGemvThreads < i1; i += 2 * kGemvThreads) {  // two rows per step, eight loads in flight
    const float x0 = x[vec_index(i, m, incx)], x1 = x[vec_index(i + kGemvThreads, m, incx)];
#pragma unroll
    for (int c = 0; c < kTCols; ++c) {
      if (c < nc) {
        const float* col = A + (jb + c) * lda;
        acc[c][0] = fmaf(col[i], x0, acc[c][0]);
        acc[c][1] = fmaf(col[i + kGemvThreads], x1, acc[c][1]);
      }
    }
  }
  if (i < i1) {
    const float x0 = x[vec_index(i, m, incx)];
#pragma unroll
    for (int c = 0; c < kTCols; ++c)
      if (c < nc) acc[c][0] = fmaf(A[(jb + c) * lda + i], x0, acc[c][0]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kTCols; ++c) {
    float v = acc[c][0] + acc[c][1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[c][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    const int c = threadIdx.x;
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kGemvThreads / 32; ++w) s += red[c][w];
    const int64_t j = jb + c;
    if (partial) {
      partial[(int64_t)blockIdx.y * n + j] = s;
    } else {
      float* yj = y + vec_index(j, n, incy);
      *yj = (beta != 0.f) ? fmaf(alpha, s, beta * *yj) : alpha * s;
    }
  }
}

// y_t := alpha sum_s partial[s][t] + beta y_t, slices summed in order; with
// nslice 0, y_t := beta y_t (alpha == 0).
__global__ void gemv_finish_kernel(int64_t len, int nslice, const float* __restrict__ partial, float alpha,
                                   float beta, float* __restrict__ y, int64_t incy) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
    float* yt = y + vec_index(t, len, incy);
    if (nslice == 0) {
      *yt = (beta == 0.f) ? 0.f : beta * *yt;
      continue;
    }
    float s = 0.f;
    for (int k = 0; k < nslice; ++k) s += partial[(int64_t)k * len + t];
    *yt = (beta != 0.f) ? fmaf(alpha, s, beta * *yt) : alpha * s;
  }
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

int64_t gemv_slices(bool trans, int64_t m, int64_t n, int num_sms) {
  const int64_t want = 4 * (int64_t)num_sms;  // blocks to cover the SMs
  if (!trans) {
    const int64_t rb = ceil_div(m, kGemvThreads);
    int64_t s = ceil_div(want, rb);
    const int64_t cap = ceil_div(n, 32);  // at least 32 columns a slice
    if (s > cap) s = cap;
    if (s > 65535) s = 65535;
    return s < 1 ? 1 : s;
  }
  const int64_t cb = ceil_div(n, kTCols);
  int64_t s = ceil_div(want, cb);
  const int64_t cap = ceil_div(m, 2048);  // at least 2048 rows a slice
  if (s > cap) s = cap;
  if (s > 65535) s = 65535;
  return s < 1 ? 1 : s;
}

cudaError_t launch_gemv(bool trans, int64_t m, int64_t n, float alpha, const float* A, int64_t lda, const float* x,
                        int64_t incx, float beta, float* y, int64_t incy, int64_t slices, float* partial,
                        int num_sms, cudaStream_t s) {
  const int64_t len_y = trans ? n : m;
  if (len_y <= 0) return cudaSuccess;
  const int64_t fin_blocks = [&] {
    int64_t b = ceil_div(len_y, 256);
    const int64_t cap = (int64_t)(num_sms > 0 ? num_sms : 148) * 8;
    return b > cap ? cap : b;
  }();
  if (alpha == 0.f || (trans ? m : n) == 0) {
    gemv_finish_kernel<<<(unsigned)fin_blocks, 256, 0, s>>>(len_y, 0, nullptr, alpha, beta, y, incy);
    return cudaGetLastError();
  }
  if (slices > 1 && !partial) return cudaErrorInvalidValue;
  float* part = slices > 1 ? partial : nullptr;
  if (!trans) {
    const int64_t slice = ceil_div(n, slices);
    const dim3 grid((unsigned)ceil_div(m, kGemvThreads), (unsigned)ceil_div(n, slice));
    if (ceil_div(m, kGemvThreads) > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
    gemv_n_kernel<<<grid, kGemvThreads, 0, s>>>(m, n, A, lda, x, incx, slice, part, alpha, beta, y, incy);
    slices = grid.y;
  } else {
    const int64_t slice = ceil_div(m, slices);
    const dim3 grid((unsigned)ceil_div(n, kTCols), (unsigned)ceil_div(m, slice));
    if (ceil_div(n, kTCols) > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
    gemv_t_kernel<<<grid, kGemvThreads, 0, s>>>(m, n, A, lda, x, incx, slice, part, alpha, beta, y, incy);
    slices = grid.y;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !part) return e;
  gemv_finish_kernel<<<(unsigned)fin_blocks, 256, 0, s>>>(len_y, (int)slices, part, alpha, beta, y, incy);
  return cudaGetLastError();
}

}  // namespace gbg
