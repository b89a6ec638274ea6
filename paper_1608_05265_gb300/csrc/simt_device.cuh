// Device side of the FP32 SIMT sgemm, shared by the single-problem kernel
// (simt.cu) and the grouped kernel (grouped.cu).
//
// The tile computation follows the paper's BLIS layering (Section III-A,
// III-C): the output is cut into BM x BN blocks, the k dimension into BK-deep
// slices, and a register-tiled micro-kernel accumulates each thread's 8 x 8
// piece over all slices before alpha and beta are applied once (the
// "Accumulator" of Section III-C: clear once, accumulate, write the result
// once).  Slices are staged through shared memory in two buffers, the next
// slice's global loads in flight while the current one is multiplied (the
// double-buffered input staging of Section III-C, within one thread block).
#pragma once

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

// One BM x BN tile of C = alpha*op(A)*op(B) + beta*C starting at (m0, n0),
// computed by the (BM/8)*(BN/8) threads of the calling block.  As and Bs are
// the block's two-buffer shared-memory slices (SimtSmem<BM, BN>).
template <int BM, int BN, bool TA, bool TB, bool VEC>
__device__ __forceinline__ void simt_tile(const Problem& P, int64_t m0, int64_t n0,
                                          float (*As)[BK * (BM + 4)], float (*Bs)[BK * (BN + 4)]) {
  using T = SimtTile<BM, BN, TA, TB, VEC>;
  constexpr int NT = T::NT;
  const int tid = threadIdx.x;
  // Consecutive lanes take consecutive row groups (ty), so an epilogue store
  // of one column by a warp covers contiguous rows of column-major C.
  const int ty = tid % (BM / 8), tx = tid / (BM / 8);
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
    // Unrolled by two, not sixteen: the fully unrolled slice (about 1100
    // instructions) missed the instruction cache (measured: short-k grouped
    // tiles stalled mostly on instruction fetch).
#pragma unroll 2
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
struct SimtSmem {
  float As[2][BK * (BM + 4)];
  float Bs[2][BK * (BN + 4)];
};

}  // namespace
}  // namespace gbg
