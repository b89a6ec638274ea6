// Plain FP32 SIMT sgemm (CUDA-core fused multiply-add) and the C := beta*C kernel.
//
// The kernel follows the paper's BLIS layering (Section III-A, III-C): the
// output is cut into BM x BN blocks, the k dimension into BK-deep slices, and
// a register-tiled micro-kernel accumulates each thread's 8 x 8 piece over
// all slices before alpha and beta are applied once (the "Accumulator" of
// Section III-C: clear once, accumulate, write the result once).  Slices are
// staged through shared memory in two buffers, the next slice's global loads
// in flight while the current one is multiplied (the double-buffered input
// staging of Section III-C, here within one thread block).
#include "internal.h"

namespace gbg {
namespace {

constexpr int BK = 16;

template <int BM, int BN, bool TA, bool TB, bool VEC>
struct SimtTile {
  static constexpr int NT = (BM / 8) * (BN / 8);
  static constexpr int LDS_A = BM + 4;
  static constexpr int LDS_B = BN + 4;
  static constexpr int A_VEC = BM * BK / 4 / NT;   // float4 loads per thread
  static constexpr int B_VEC = BN * BK / 4 / NT;
  static constexpr int A_SCL = BM * BK / NT;       // scalar loads per thread
  static constexpr int B_SCL = BN * BK / NT;
  static constexpr int A_REG = VEC ? A_VEC * 4 : A_SCL;
  static constexpr int B_REG = VEC ? B_VEC * 4 : B_SCL;
};

// Load one BM x BK slice of op(A) (or, with the roles swapped, one BK x BN
// slice of op(B)) into registers.  `rowcontig` means consecutive tile rows
// (the M or N index) are consecutive in memory; otherwise the k index is.
// Elements outside [0, rows) x [0, kdim) read as zero.
template <int ROWS, int NT, bool VEC, bool ROWCONTIG>
__device__ __forceinline__ void load_slice(float* reg, const float* __restrict__ X, int64_t ld,
                                           int64_t row0, int64_t rows, int64_t k0, int64_t kdim, int tid) {
  if constexpr (VEC) {
    constexpr int NV = ROWS * BK / 4 / NT;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int f = tid + v * NT;
      int64_t r, p;
      if constexpr (ROWCONTIG) { p = f / (ROWS / 4); r = (f % (ROWS / 4)) * 4; }
      else { r = f / (BK / 4); p = (f % (BK / 4)) * 4; }
      const int64_t gr = row0 + r, gp = k0 + p;
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (ROWCONTIG) {
        // Four consecutive rows of one k column.  gr % 4 == 0 and ld % 4 == 0
        // keep the vector inside column gp; rows >= `rows` only feed outputs
        // that are never stored.
        if (gr < rows && gp < kdim) val = *reinterpret_cast<const float4*>(X + gr + gp * ld);
      } else {
        // Four consecutive k of one row; k beyond kdim is zeroed.
        if (gr < rows && gp < kdim) {
          val = *reinterpret_cast<const float4*>(X + gp + gr * ld);
          if (gp + 1 >= kdim) val.y = 0.f;
          if (gp + 2 >= kdim) val.z = 0.f;
          if (gp + 3 >= kdim) val.w = 0.f;
        }
      }
      reg[4 * v + 0] = val.x; reg[4 * v + 1] = val.y; reg[4 * v + 2] = val.z; reg[4 * v + 3] = val.w;
    }
  } else {
    constexpr int NS = ROWS * BK / NT;
#pragma unroll
    for (int v = 0; v < NS; ++v) {
      const int f = tid + v * NT;
      int64_t r, p;
      if constexpr (ROWCONTIG) { p = f / ROWS; r = f % ROWS; }
      else { r = f / BK; p = f % BK; }
      const int64_t gr = row0 + r, gp = k0 + p;
      float val = 0.f;
      if (gr < rows && gp < kdim) val = ROWCONTIG ? X[gr + gp * ld] : X[gp + gr * ld];
      reg[v] = val;
    }
  }
}

// Store the registers of load_slice into the k-major shared tile S[p][r].
template <int ROWS, int NT, int LDS, bool VEC, bool ROWCONTIG>
__device__ __forceinline__ void store_slice(float* S, const float* reg, int tid) {
  if constexpr (VEC) {
    constexpr int NV = ROWS * BK / 4 / NT;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int f = tid + v * NT;
      if constexpr (ROWCONTIG) {
        const int p = f / (ROWS / 4), r = (f % (ROWS / 4)) * 4;
        *reinterpret_cast<float4*>(S + p * LDS + r) = make_float4(reg[4 * v], reg[4 * v + 1], reg[4 * v + 2], reg[4 * v + 3]);
      } else {
        const int r = f / (BK / 4), p = (f % (BK / 4)) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) S[(p + q) * LDS + r] = reg[4 * v + q];
      }
    }
  } else {
    constexpr int NS = ROWS * BK / NT;
#pragma unroll
    for (int v = 0; v < NS; ++v) {
      const int f = tid + v * NT;
      int r, p;
      if constexpr (ROWCONTIG) { p = f / ROWS; r = f % ROWS; }
      else { r = f / BK; p = f % BK; }
      S[p * LDS + r] = reg[v];
    }
  }
}

template <int BM, int BN, bool TA, bool TB, bool VEC>
__global__ void __launch_bounds__((BM / 8) * (BN / 8))
sgemm_simt_kernel(Problem P) {
  using T = SimtTile<BM, BN, TA, TB, VEC>;
  constexpr int NT = T::NT;
  __shared__ __align__(16) float As[2][BK * T::LDS_A];
  __shared__ __align__(16) float Bs[2][BK * T::LDS_B];

  const int tid = threadIdx.x;
  const int tx = tid % (BN / 8), ty = tid / (BN / 8);
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t nk = (P.k + BK - 1) / BK;

  // op(A): rows are M (contiguous when A is not transposed).
  // op(B): rows of the staged tile are N (contiguous when B is transposed).
  float ra[T::A_REG], rb[T::B_REG];
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  load_slice<BM, NT, VEC, !TA>(ra, P.A, P.lda, m0, P.m, 0, P.k, tid);
  load_slice<BN, NT, VEC, TB>(rb, P.B, P.ldb, n0, P.n, 0, P.k, tid);
  store_slice<BM, NT, T::LDS_A, VEC, !TA>(As[0], ra, tid);
  store_slice<BN, NT, T::LDS_B, VEC, TB>(Bs[0], rb, tid);
  __syncthreads();

  for (int64_t kt = 0; kt < nk; ++kt) {
    const int cur = (int)(kt & 1);
    if (kt + 1 < nk) {
      load_slice<BM, NT, VEC, !TA>(ra, P.A, P.lda, m0, P.m, (kt + 1) * BK, P.k, tid);
      load_slice<BN, NT, VEC, TB>(rb, P.B, P.ldb, n0, P.n, (kt + 1) * BK, P.k, tid);
    }
    const float* a_s = As[cur];
    const float* b_s = Bs[cur];
#pragma unroll
    for (int p = 0; p < BK; ++p) {
      const float4 a0 = *reinterpret_cast<const float4*>(a_s + p * T::LDS_A + ty * 4);
      const float4 a1 = *reinterpret_cast<const float4*>(a_s + p * T::LDS_A + BM / 2 + ty * 4);
      const float4 b0 = *reinterpret_cast<const float4*>(b_s + p * T::LDS_B + tx * 4);
      const float4 b1 = *reinterpret_cast<const float4*>(b_s + p * T::LDS_B + BN / 2 + tx * 4);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      store_slice<BM, NT, T::LDS_A, VEC, !TA>(As[cur ^ 1], ra, tid);
      store_slice<BN, NT, T::LDS_B, VEC, TB>(Bs[cur ^ 1], rb, tid);
    }
    __syncthreads();
  }

  // Epilogue: C = alpha*acc + beta*C, columns of C contiguous along M.
  const bool vec_c = ((P.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.C) & 15) == 0);
#pragma unroll
  for (int jh = 0; jh < 2; ++jh) {
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int64_t j = n0 + jh * (BN / 2) + tx * 4 + jj;
      if (j >= P.n) continue;
#pragma unroll
      for (int ih = 0; ih < 2; ++ih) {
        const int64_t i = m0 + ih * (BM / 2) + ty * 4;
        float* cp = P.C + i + j * P.ldc;
        // alpha*acc + beta*c with one rounding of beta*c and one of the sum
        // (fmaf), so that k = 1 stays within 2*2^-24 of the exact value.
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = acc[ih * 4 + q][jh * 4 + jj];
        if (vec_c && i + 3 < P.m) {
          if (P.beta != 0.f) {
            const float4 c = *reinterpret_cast<const float4*>(cp);
            v[0] = fmaf(P.alpha, v[0], P.beta * c.x); v[1] = fmaf(P.alpha, v[1], P.beta * c.y);
            v[2] = fmaf(P.alpha, v[2], P.beta * c.z); v[3] = fmaf(P.alpha, v[3], P.beta * c.w);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = P.alpha * v[q];
          }
          *reinterpret_cast<float4*>(cp) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (i + q < P.m) cp[q] = (P.beta != 0.f) ? fmaf(P.alpha, v[q], P.beta * cp[q]) : P.alpha * v[q];
          }
        }
      }
    }
  }
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
