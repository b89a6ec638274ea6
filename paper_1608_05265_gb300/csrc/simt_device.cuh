// Device side of the FP32 SIMT sgemm, shared by the single-problem kernel
// (simt.cu) and the grouped kernel (grouped.cu).
//
// The tile computation follows the paper's BLIS layering (Section III-A,
// III-C): the output is cut into BM x BN blocks, the k dimension into BK-deep
// slices, and a register-tiled micro-kernel accumulates each thread's 8 x 8
// piece over all slices before alpha and beta are applied once (the
// "Accumulator" of Section III-C: clear once, accumulate, write the result
// once).  Slices are staged in shared memory in two buffers by asynchronous
// copies, the next slice's copies in flight while the current one is
// multiplied (the double-buffered input staging of Section III-C, within one
// thread block).
#pragma once

#include "internal.h"

namespace gbg {
namespace {

constexpr int BK = 16;

// Register-staged tiles (k-contiguous float4 operands) put row r of k row p
// at column r ^ 8((p / 4) mod 4): a warp's transposing stores (eight rows of
// k rows p, p + 4, p + 8, p + 12, same q) then fall in 32 different banks
// instead of two rows per bank, and groups of four consecutive rows stay
// together for the 16-byte reads of the multiply loop.
__device__ __forceinline__ int swz(int p, int r) { return r ^ (((p >> 2) & 3) << 3); }

template <int BM, int BN, bool TA, bool TB, bool VEC>
struct SimtTile {
  static constexpr int NT = (BM / 8) * (BN / 8);
  static constexpr int LDS_A = BM + 4;
  static constexpr int LDS_B = BN + 4;
};

__device__ __forceinline__ void cp_async4s(uint32_t dst, const float* src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Loads of one operand's BK-deep slices into shared memory.  A thread's load v
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

  // Register staging, used for the VEC k-contiguous case only (its float4 of
  // four k values lands in four rows of the k-major tile, which a 16-byte
  // asynchronous copy cannot do): slice kt into reg[0 .. 4 NL - 1] ...
  __device__ __forceinline__ void load(float* reg, int64_t kt, int64_t kdim) const {
    static_assert(VEC && !ROWCONTIG, "register staging serves the VEC k-contiguous case");
    const float* p = base + kt * BK;
    const int64_t krem = kdim - kt * BK - kfix;
    const int nv = krem > 0 ? nrow : 0;
#pragma unroll
    for (int v = 0; v < NL; ++v) {
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if (v < nv) {
        val = *reinterpret_cast<const float4*>(p);
        if (krem < 2) val.y = 0.f;  // k beyond kdim is zeroed
        if (krem < 3) val.z = 0.f;
        if (krem < 4) val.w = 0.f;
      }
      reg[4 * v + 0] = val.x; reg[4 * v + 1] = val.y; reg[4 * v + 2] = val.z; reg[4 * v + 3] = val.w;
      p += vstep;
    }
  }
  // ... and from the registers into the k-major shared tile S[p][r], row r
  // of k row p at S[p LDS + swz(p, r)] (see swz).
  template <int LDS>
  __device__ __forceinline__ void store(float* S, const float* reg, int tid) const {
    const int fx = (tid % PER) * W, vr = tid / PER;
#pragma unroll
    for (int v = 0; v < NL; ++v)
#pragma unroll
      for (int q = 0; q < 4; ++q) S[(fx + q) * LDS + swz(fx + q, vr + v * STRIDE)] = reg[4 * v + q];
  }

  // Copy slice kt of an operand with kdim k indices into the k-major shared
  // tile S[p][r] (row pitch LDS floats, at shared address s_addr) with
  // asynchronous copies: out-of-range elements are zero-filled without a
  // read (and with the source pointer kept at a valid address).
  template <int LDS>
  __device__ __forceinline__ void issue(uint32_t s_addr, int64_t kt, int64_t kdim, const float* X, int tid) const {
    const float* p = ROWCONTIG ? base + ((kt * vstep) << KSHIFT) : base + kt * BK;
    const int64_t krem = kdim - kt * BK - kfix;  // in-range k offsets from this thread's first one
    int nv;
    if constexpr (ROWCONTIG) {
      const int64_t nk = krem <= 0 ? 0 : (krem + STRIDE - 1) / STRIDE;
      nv = nk < nrow ? (int)nk : nrow;
    } else {
      nv = krem > 0 ? nrow : 0;
    }
    const int fx = (tid % PER) * W, vr = tid / PER;
#pragma unroll
    for (int v = 0; v < NL; ++v) {
      const bool ok = v < nv;
      const float* src = ok ? p : X;
      if constexpr (ROWCONTIG) {
        // tile row fx (.. fx + W - 1), k offset vr + v STRIDE
        const uint32_t dst = s_addr + (uint32_t)((vr + v * STRIDE) * LDS + fx) * 4u;
        if constexpr (VEC) cp_async16(dst, src, ok ? 16u : 0u);
        else cp_async4s(dst, src, ok ? 4u : 0u);
      } else {
        // k offset fx, tile row vr + v STRIDE (scalar: VEC goes through registers)
        static_assert(!VEC, "the VEC k-contiguous case uses load() and store()");
        cp_async4s(s_addr + (uint32_t)(fx * LDS + vr + v * STRIDE) * 4u, src, ok ? 4u : 0u);
      }
      p += vstep;
    }
  }
};

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
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  using LoadA = SliceLoader<BM, NT, VEC, !TA>;
  using LoadB = SliceLoader<BN, NT, VEC, TB>;
  constexpr bool REG_A = VEC && TA, REG_B = VEC && !TB;  // k-contiguous float4 operands stage through registers
  const LoadA LA(P.A, P.lda, m0, P.m, tid);
  const LoadB LB(P.B, P.ldb, n0, P.n, tid);
  float ra[REG_A ? LoadA::NL * 4 : 1], rb[REG_B ? LoadB::NL * 4 : 1];
  const uint32_t sA0 = (uint32_t)__cvta_generic_to_shared(As[0]), sA1 = (uint32_t)__cvta_generic_to_shared(As[1]);
  const uint32_t sB0 = (uint32_t)__cvta_generic_to_shared(Bs[0]), sB1 = (uint32_t)__cvta_generic_to_shared(Bs[1]);
  // slice kt into buffer b (register-staged operands: into registers only)
  auto fetch = [&](int64_t kt, int b) {
    if constexpr (REG_A) LA.load(ra, kt, P.k);
    else LA.template issue<T::LDS_A>(b ? sA1 : sA0, kt, P.k, P.A, tid);
    if constexpr (REG_B) LB.load(rb, kt, P.k);
    else LB.template issue<T::LDS_B>(b ? sB1 : sB0, kt, P.k, P.B, tid);
    cp_async_commit_all();
  };
  auto put = [&](int b) {  // register-staged operands into buffer b
    if constexpr (REG_A) LA.template store<T::LDS_A>(As[b], ra, tid);
    if constexpr (REG_B) LB.template store<T::LDS_B>(Bs[b], rb, tid);
  };
  if (nk > 0) {  // (k = 0: A and B are not read, and may be null)
    fetch(0, 0);
    put(0);
    cp_async_wait_all();
  }
  __syncthreads();

  for (int64_t kt = 0; kt < nk; ++kt) {
    const int cur = (int)(kt & 1);
    // the other buffer was last read before the previous barrier
    if (kt + 1 < nk) fetch(kt + 1, cur ^ 1);
    const float* a_s = As[cur];
    const float* b_s = Bs[cur];
    // Unrolled by two, not sixteen: the fully unrolled slice (about 1100
    // instructions) missed the instruction cache (measured: short-k grouped
    // tiles stalled mostly on instruction fetch).
#pragma unroll 2
    for (int p = 0; p < BK; ++p) {
      const int ca0 = REG_A ? swz(p, ty * 4) : ty * 4, ca1 = REG_A ? swz(p, BM / 2 + ty * 4) : BM / 2 + ty * 4;
      const int cb0 = REG_B ? swz(p, tx * 4) : tx * 4, cb1 = REG_B ? swz(p, BN / 2 + tx * 4) : BN / 2 + tx * 4;
      const float4 a0 = *reinterpret_cast<const float4*>(a_s + p * T::LDS_A + ca0);
      const float4 a1 = *reinterpret_cast<const float4*>(a_s + p * T::LDS_A + ca1);
      const float4 b0 = *reinterpret_cast<const float4*>(b_s + p * T::LDS_B + cb0);
      const float4 b1 = *reinterpret_cast<const float4*>(b_s + p * T::LDS_B + cb1);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < nk) put(cur ^ 1);
    cp_async_wait_all();  // the next slice's copies by this thread have landed
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
