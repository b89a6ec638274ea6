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

// Loads of one operand's BK-deep slices into registers.  A thread's load v
// (v = 0 .. NL-1) of slice kt reads tile row r and k offset p with
//   rowcontig (consecutive tile rows consecutive in memory, element (r, p) at
//     X[r + p*ld]):  r = (tid % PER) W fixed,  p = tid / PER + v STRIDE;
//   otherwise (element (r, p) at X[p + r*ld]):  p = (tid % PER) W fixed,
//     r = tid / PER + v STRIDE,
// W floats per load (4 with VEC).  One coordinate is fixed for the whole
// tile and the other advances by a compile-time stride, so a base pointer
// and counts of in-range loads, set up once per tile, replace per-element
// index arithmetic and bounds checks.  Elements outside [0, rows) x [0, kdim)
// read as zero; a float4 of rows (rowcontig VEC) is read when its first row
// is in range (gr % 4 == 0 and ld % 4 == 0 keep it inside its column; rows
// >= rows only feed outputs that are never stored).
template <int ROWS, int NT, bool VEC, bool ROWCONTIG>
struct SliceLoader {
  static constexpr int W = VEC ? 4 : 1;
  static constexpr int PER = ROWCONTIG ? ROWS / W : BK / W;
  static constexpr int STRIDE = NT / PER;
  static constexpr int NL = ROWS * BK / W / NT;
  static_assert(NT % PER == 0 && (STRIDE & (STRIDE - 1)) == 0, "load mapping");
  static constexpr int KSHIFT = ROWCONTIG ? (STRIDE == 1 ? 4 : STRIDE == 2 ? 3 : STRIDE == 4 ? 2 : STRIDE == 8 ? 1 : 0) : 0;
  static_assert(!ROWCONTIG || (BK >> KSHIFT) == STRIDE, "slice step = BK / STRIDE load steps");
  const float* base;   // load v = 0 of slice 0
  int64_t vstep;       // elements between a thread's consecutive loads (STRIDE ld)
  int kfix;            // k offset of load v = 0 within a slice (rowcontig) or of every load (otherwise)
  int nrow;            // loads whose row is in range

  __device__ __forceinline__ SliceLoader(const float* X, int64_t ld, int64_t row0, int64_t rows, int tid) {
    const int fx = (tid % PER) * W, vr = tid / PER;
    vstep = (int64_t)STRIDE * ld;
    if constexpr (ROWCONTIG) {
      const int64_t r = row0 + fx;
      base = X + r + (int64_t)vr * ld;
      kfix = vr;
      nrow = r < rows ? NL : 0;
    } else {
      const int64_t r = row0 + vr;
      base = X + fx + r * ld;
      kfix = fx;
      const int64_t nv = r < rows ? (rows - r + STRIDE - 1) / STRIDE : 0;
      nrow = nv < NL ? (int)nv : NL;
    }
  }

  // Slice kt of an operand with kdim k indices into reg[0 .. NL*W - 1].
  __device__ __forceinline__ void load(float* reg, int64_t kt, int64_t kdim) const {
    // one slice is BK / STRIDE load steps (rowcontig) or BK elements along the row
    const float* p = ROWCONTIG ? base + ((kt * vstep) << KSHIFT) : base + kt * BK;
    const int64_t krem = kdim - kt * BK - kfix;  // in-range k offsets from this thread's first one
    int nv;
    if constexpr (ROWCONTIG) {
      const int64_t nk = krem <= 0 ? 0 : (krem + STRIDE - 1) / STRIDE;
      nv = nk < nrow ? (int)nk : nrow;
    } else {
      nv = krem > 0 ? nrow : 0;
    }
#pragma unroll
    for (int v = 0; v < NL; ++v) {
      if constexpr (VEC) {
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v < nv) {
          val = *reinterpret_cast<const float4*>(p);
          if constexpr (!ROWCONTIG) {
            // four consecutive k of one row; k beyond kdim is zeroed
            if (krem < 2) val.y = 0.f;
            if (krem < 3) val.z = 0.f;
            if (krem < 4) val.w = 0.f;
          }
        }
        reg[4 * v + 0] = val.x; reg[4 * v + 1] = val.y; reg[4 * v + 2] = val.z; reg[4 * v + 3] = val.w;
      } else {
        reg[v] = v < nv ? *p : 0.f;
      }
      p += vstep;
    }
  }
};

// Store the registers of SliceLoader::load into the k-major shared tile S[p][r].
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

  const SliceLoader<BM, NT, VEC, !TA> LA(P.A, P.lda, m0, P.m, tid);
  const SliceLoader<BN, NT, VEC, TB> LB(P.B, P.ldb, n0, P.n, tid);
  LA.load(ra, 0, P.k);
  LB.load(rb, 0, P.k);
  store_slice<BM, NT, T::LDS_A, VEC, !TA>(As[0], ra, tid);
  store_slice<BN, NT, T::LDS_B, VEC, TB>(Bs[0], rb, tid);
  __syncthreads();

  for (int64_t kt = 0; kt < nk; ++kt) {
    const int cur = (int)(kt & 1);
    if (kt + 1 < nk) {
      LA.load(ra, kt + 1, P.k);
      LB.load(rb, kt + 1, P.k);
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
