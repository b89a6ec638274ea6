// Grouped split-BF16 GEMM with the split done on load ("fused"): no hi/lo
// panels in HBM.  Converter warps copy FP32 slices of op(A) and op(B) from
// the caller's matrices into shared memory with cp.async (4-byte copies: any
// leading dimension and alignment), split every value into BF16 hi and lo in
// the tensor cores' swizzled K-major layout, and hand each 32-deep k chunk to
// the MMA warp; the accumulator and epilogue work as in split_gemm_kernel.
//
// Scaling.  A tile reads the whole k extent of its 128 rows of op(A) and its
// BN columns of op(B), so by its last chunk it knows their exact max |x|.
// The split is done unscaled, which is the method's definition for
// well-scaled vectors (max |x| in [2^-48, 2^48)).  If any of the tile's
// vectors is badly scaled, the epilogue does not store the tile: it appends
// it to a fallback list that the grouped FP32 SIMT kernel finishes (the
// SIMT path meets the acceptance bound at any scale).
//
// Roles (one CTA per SM, 416 threads):
//   warps 0-7   converters.  Warp w owns k sub-chunk cc = w % 4 (8 values)
//               of the 32-row blocks w / 4 and w / 4 + 2 of op(A) and of
//               op(B): it copies exactly the values it converts, through a
//               private 3-stage cp.async ring, so the converter warps never
//               wait for one another; each signals the MMA warp per chunk;
//   warp 8      TMEM owner (256 columns: two 128 x 128 accumulators); lane 0
//               issues the MMAs and commits;
//   warps 9-12  epilogue: warp w reads TMEM lanes 32*(w%4) .. +31, all of
//               the tile's columns.
// Row maxima of a tile are combined across the converter warps with 64-bit
// shared-memory atomicMax on (tile epoch << 32 | max |x| bits), so a slot
// needs no reset between tiles: a newer epoch always wins.
#pragma once

#include "split_device.cuh"

namespace gbg {
namespace {

constexpr int kFusedConvWarps = 8;
constexpr int kFusedMmaWarp = kFusedConvWarps;
constexpr int kFusedEpiWarps = 4;
constexpr int kFusedThreads = 32 * kFusedConvWarps + 32 + 32 * kFusedEpiWarps;
constexpr int kFusedMaxBN = 128;
constexpr int kFusedStagesF = 3;                     // FP32 stages per converter warp
constexpr int kFusedAhead = kFusedStagesF - 1;       // chunks of copies in flight ahead of conversion
constexpr int kFusedStagesB = 3;                     // BF16 stages consumed by the MMA
constexpr int kMaxSlots = 4;                         // tile slots of row maxima
// One converter warp's FP32 stage: its 64 rows x 8 k of op(A) (2 KiB), then
// of op(B).  A k-contiguous operand is staged [row][8 k], the two 16-byte
// halves of a row swapped on rows with bit 2 set (so that 8 consecutive
// rows read the same half from 8 distinct bank groups); a row-contiguous
// operand is staged [k][64 rows].
constexpr uint32_t kWarpPart = 2048;
constexpr uint32_t kWarpStage = 2 * kWarpPart;
constexpr uint32_t kFusedStageB = 2u * (uint32_t)kBlockBytes;            // A block + B block (128 rows each)
constexpr uint32_t kFusedTmemCols = 2 * kFusedMaxBN;
constexpr uint32_t kOffF32 = kFusedStagesB * kFusedStageB;
constexpr uint32_t kOffSlots = kOffF32 + kFusedConvWarps * kFusedStagesF * kWarpStage;
constexpr uint32_t kOffBars = kOffSlots + kMaxSlots * 256 * 8;
constexpr int kFusedSmemBytes = (int)kOffBars + 256 + 1024;  // + barriers, TMEM holder; + 1024-byte alignment

// One problem of the batch on the fused path.
struct FusedGroup {
  const float* A; int64_t lda;
  const float* B; int64_t ldb;
  float* C; int64_t ldc;
  int64_t m, n, k;
  float alpha, beta;
  int a_kcontig, b_kcontig;   // element (r, p) at X[r*ld + p] when set, else X[r + p*ld]
  int bn, nkc;
  int simt_index;             // the problem's index in the SIMT descriptor array (fallback)
  int pad_;
};

struct FusedSched {
  const int4* items;          // (group, tile row, tile column, 0), costliest first
  const FusedGroup* groups;
  int n_items;
  int* fb_count;              // fallback list length (zeroed before every run)
  int4* fb_items;             // fallback list: (SIMT problem, 128-row tile, 64-column tile, 0)
};

// 4-byte asynchronous copy global -> shared; bytes = 0 writes a zero and
// reads nothing.
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void st_shared_zero(uint32_t dst) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(dst), "r"(0u) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Word index of (row ri, k kk) in a k-contiguous part.
__device__ __forceinline__ uint32_t kpart_word(int ri, int kk) {
  return (uint32_t)(ri * 8 + ((((kk >> 2) ^ (ri >> 2)) & 1) << 2) + (kk & 3));
}

// Stage a converter warp's part of one operand: k [pb, pb + 8) of the rows
// R + lane-row and R + 64 + lane-row (nb = 2), or only the first 32 (nb = 1).
// Rows past the matrix are clamped into it and copied as zeros (bytes 0);
// k past its end likewise.
//   row-contiguous (element (r, p) at X[r + p*ld]): lane l takes row R + l
//     (+ 64); one warp instruction reads 128 consecutive bytes;
//   k-contiguous (element (r, p) at X[r*ld + p]): lane l takes row
//     R + 4 j + l / 8, k pb + l % 8; one warp instruction reads 4 rows x 32
//     consecutive bytes.
__device__ __forceinline__ void stage_part(uint32_t dst, const float* X, int64_t ld, bool kcontig, int64_t rows,
                                           int64_t k, int64_t R, int64_t pb, int nb, int lane) {
  const bool full_k = pb + 8 <= k;
  if (!kcontig) {
    int64_t rc[2];
    uint32_t sz[2];
#pragma unroll
    for (int bi = 0; bi < 2; ++bi) {
      const int64_t r = R + 64 * bi + lane;
      const bool rv = r < rows;
      rc[bi] = rv ? r : rows - 1;
      sz[bi] = rv ? 4u : 0u;
    }
    const uint32_t d = dst + (uint32_t)lane * 4u;
    if (full_k) {
      // common case: one pointer walks the 8 columns
      const float* q = X + pb * ld + rc[0];
      const int64_t d1 = rc[1] - rc[0];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        cp_async4(d + kk * 256u, q, sz[0]);
        if (nb == 2) cp_async4(d + kk * 256u + 128u, q + d1, sz[1]);
        q += ld;
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int64_t p = pb + kk;
        if (p < k) {  // warp-uniform
          const float* col = X + p * ld;
          cp_async4(d + kk * 256u, col + rc[0], sz[0]);
          if (nb == 2) cp_async4(d + kk * 256u + 128u, col + rc[1], sz[1]);
        } else {
          st_shared_zero(d + kk * 256u);
          if (nb == 2) st_shared_zero(d + kk * 256u + 128u);
        }
      }
    }
  } else {
    const int rs = lane >> 3, kk = lane & 7;
    if (full_k && R + 64 * (nb - 1) + 32 <= rows) {
      // common case: every row of the part inside the matrix; one pointer
      // per 32-row block walks its rows 4 at a time
      const uint32_t w_even = kpart_word(rs, kk), w_odd = kpart_word(4 + rs, kk) - 32;
      const float* q = X + (R + rs) * ld + pb + kk;
      const int64_t s4 = 4 * ld;
#pragma unroll
      for (int bi = 0; bi < 2; ++bi) {
        if (bi < nb) {
          const float* qb = q + 64 * bi * ld;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t w = ((j & 1) ? w_odd : w_even) + (uint32_t)(bi * 32 + 4 * j) * 8u;
            cp_async4(dst + w * 4u, qb, 4u);
            qb += s4;
          }
        }
      }
    } else {
      const int64_t p = pb + kk;
      const bool pv = p < k;
      const float* src = X + (pv ? p : k - 1);
#pragma unroll
      for (int bi = 0; bi < 2; ++bi) {
        if (bi < nb) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int ri = bi * 32 + 4 * j + rs;
            const int64_t r = R + 64 * bi + 4 * j + rs;
            const bool rv = r < rows;
            cp_async4(dst + kpart_word(ri, kk) * 4u, src + (rv ? r : rows - 1) * ld, (rv && pv) ? 4u : 0u);
          }
        }
      }
    }
  }
}

// Split the 8 staged values of one (row, 8-wide k sub-chunk) item into the
// swizzled BF16 block (hi at hi_dst, lo at lo_dst); returns max(m, max |x|).
// Non-finite x gets lo = 0 (an infinity would otherwise give lo = NaN).
template <bool KCONTIG>
__device__ __forceinline__ float convert_item(const uint8_t* part, int ri, uint8_t* hi_dst, uint8_t* lo_dst, float m) {
  float x[8];
  if (KCONTIG) {
    const float* row = reinterpret_cast<const float*>(part) + ri * 8;
    const int sw = (ri >> 2) & 1;
    const float4 u = *reinterpret_cast<const float4*>(row + 4 * sw);         // k 0-3
    const float4 v = *reinterpret_cast<const float4*>(row + 4 * (sw ^ 1));   // k 4-7
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
    x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
  } else {
    const float* col = reinterpret_cast<const float*>(part) + ri;
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = col[q * 64];
  }
  float mx = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) mx = fmaxf(mx, fabsf(x[q]));
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    const uint32_t hb = *reinterpret_cast<const uint32_t*>(&h2);
    const float h0 = __uint_as_float(hb << 16), h1 = __uint_as_float(hb & 0xFFFF0000u);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(x[2 * q] - h0, x[2 * q + 1] - h1);
    hw[q] = hb;
    lw[q] = *reinterpret_cast<const uint32_t*>(&l2);
  }
  if (!(mx < __int_as_float(0x7F800000))) {  // rare: an infinity among the 8
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!isfinite(x[2 * q])) lw[q] &= 0xFFFF0000u;
      if (!isfinite(x[2 * q + 1])) lw[q] &= 0x0000FFFFu;
    }
  }
  *reinterpret_cast<uint4*>(hi_dst) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(lo_dst) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  return fmaxf(m, mx);
}

__global__ void __launch_bounds__(kFusedThreads, 1)
fused_gemm_kernel(const FusedSched S, int* status, uint64_t timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  uint8_t* const base_ptr = smem_raw + (base - raw_addr);
  const uint32_t sB16 = base;                       // kFusedStagesB x (A block | B block)
  const uint32_t sF32 = base + kOffF32;             // per converter warp: kFusedStagesF x (A part | B part)
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(base_ptr + kOffSlots);  // kMaxSlots x 256
  const uint32_t bar0 = base + kOffBars;
  auto bfull = [&](int s) { return bar0 + 8u * s; };
  auto bempty = [&](int s) { return bar0 + 8u * (kFusedStagesB + s); };
  auto accf = [&](int b) { return bar0 + 8u * (2 * kFusedStagesB + b); };
  auto acce = [&](int b) { return bar0 + 8u * (2 * kFusedStagesB + 2 + b); };
  auto mxfull = [&](int i) { return bar0 + 8u * (2 * kFusedStagesB + 4 + i); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kFusedStagesB + 4 + kMaxSlots);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(base_ptr + kOffBars + 8 * (2 * kFusedStagesB + 5 + kMaxSlots));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_items = S.n_items;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFusedStagesB; ++s) { mbar_init(bfull(s), kFusedConvWarps); mbar_init(bempty(s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf(b), 1); mbar_init(acce(b), kFusedEpiWarps); }
    for (int i = 0; i < kMaxSlots; ++i) mbar_init(mxfull(i), 32 * kFusedConvWarps);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kMaxSlots * 256; i += blockDim.x) slots[i] = 0ull;
  if (warp == kFusedMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_holder)), "r"(kFusedTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  // the item's problem, copied into registers (the cp.async asm statements
  // clobber memory, so a reference would be reloaded after each of them)
  auto group_of = [&](int t, int4& it) -> FusedGroup {
    it = S.items[t];
    return S.groups[it.x];
  };

  if (warp < kFusedConvWarps) {
    // ---------------- converters ----------------
    const int cc = warp & 3;         // k sub-chunk: k 8 cc .. 8 cc + 7 of every chunk
    const int b0 = warp >> 2;        // 32-row blocks b0 and b0 + 2 of op(A) and of op(B)
    const uint32_t my_f32 = sF32 + (uint32_t)warp * kFusedStagesF * kWarpStage;
    // issue cursor (item, k chunk) runs kFusedAhead chunks ahead of the convert cursor
    int it_i = blockIdx.x, kc_i = 0;
    int issued = 0;
    int4 iti = make_int4(0, 0, 0, 0);
    FusedGroup Gi{};
    if (it_i < num_items) Gi = group_of(it_i, iti);
    auto issue_next = [&]() {
      if (it_i < num_items) {
        const uint32_t st = my_f32 + (uint32_t)(issued % kFusedStagesF) * kWarpStage;
        const int64_t pb = (int64_t)kc_i * 32 + cc * 8;
        stage_part(st, Gi.A, Gi.lda, Gi.a_kcontig != 0, Gi.m, Gi.k, (int64_t)iti.y * 128 + 32 * b0, pb, 2, lane);
        stage_part(st + kWarpPart, Gi.B, Gi.ldb, Gi.b_kcontig != 0, Gi.n, Gi.k, (int64_t)iti.z * Gi.bn + 32 * b0, pb,
                   Gi.bn == 128 ? 2 : 1, lane);
        if (++kc_i == Gi.nkc) {
          kc_i = 0;
          it_i += gridDim.x;
          if (it_i < num_items) Gi = group_of(it_i, iti);
        }
      }
      cp_async_commit();  // an empty group keeps the group count in step
      ++issued;
    };
    for (int a = 0; a < kFusedAhead; ++a) issue_next();

    // This lane's conversion items: row ri = 32 bi + lane of the warp's part
    // (tile row 32 (b0 + 2 bi) + lane), bi = 0, 1 of op(A) and of op(B).
    uint32_t hi_off[4], lo_off[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int trow = 32 * (b0 + 2 * (i & 1)) + lane;  // row within the operand's tile
      const uint32_t rowb = (uint32_t)(i >> 1) * (uint32_t)kBlockBytes + (uint32_t)trow * 128u;
      hi_off[i] = rowb + ((uint32_t)(cc ^ (trow & 7)) << 4);
      lo_off[i] = rowb + ((uint32_t)((cc + 4) ^ (trow & 7)) << 4);
    }
    float my_max[4] = {0.f, 0.f, 0.f, 0.f};
    int g = 0, ordinal = 0;
    bool ok = true;
    for (int tt = blockIdx.x; tt < num_items && ok; tt += gridDim.x, ++ordinal) {
      int4 it;
      const FusedGroup G = group_of(tt, it);
      const bool a_k = G.a_kcontig != 0, b_k = G.b_kcontig != 0;
      const bool b_two = G.bn == 128;  // op(B) has row blocks b0 and b0 + 2
      for (int kc = 0; kc < G.nkc; ++kc, ++g) {
        issue_next();
        cp_async_wait<kFusedAhead>();  // chunk g's copies by this thread have landed
        __syncwarp();                  // ... and those of the other lanes
        const int sb = g % kFusedStagesB;
        int go = 1;
        if (lane == 0) {
          go = mbar_wait_hint(bempty(sb), (uint32_t)(((g / kFusedStagesB) & 1) ^ 1), abort_flag, timeout_ns, 1000u)
                   ? 1 : 0;
          if (!go) raise_status(status, abort_flag);
        }
        if (!__shfl_sync(0xFFFFFFFFu, go, 0)) { ok = false; break; }
        const uint8_t* stf = base_ptr + (my_f32 - base) + (uint32_t)(g % kFusedStagesF) * kWarpStage;
        uint8_t* stb = base_ptr + (sB16 - base) + (uint32_t)sb * kFusedStageB;
        if (a_k) {
          my_max[0] = convert_item<true>(stf, lane, stb + hi_off[0], stb + lo_off[0], my_max[0]);
          my_max[1] = convert_item<true>(stf, 32 + lane, stb + hi_off[1], stb + lo_off[1], my_max[1]);
        } else {
          my_max[0] = convert_item<false>(stf, lane, stb + hi_off[0], stb + lo_off[0], my_max[0]);
          my_max[1] = convert_item<false>(stf, 32 + lane, stb + hi_off[1], stb + lo_off[1], my_max[1]);
        }
        if (b_k) {
          my_max[2] = convert_item<true>(stf + kWarpPart, lane, stb + hi_off[2], stb + lo_off[2], my_max[2]);
          if (b_two)
            my_max[3] = convert_item<true>(stf + kWarpPart, 32 + lane, stb + hi_off[3], stb + lo_off[3], my_max[3]);
        } else {
          my_max[2] = convert_item<false>(stf + kWarpPart, lane, stb + hi_off[2], stb + lo_off[2], my_max[2]);
          if (b_two)
            my_max[3] = convert_item<false>(stf + kWarpPart, 32 + lane, stb + hi_off[3], stb + lo_off[3], my_max[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // BF16 writes -> tensor core reads
        __syncwarp();
        if (lane == 0) mbar_arrive(bfull(sb));
        if (kc == G.nkc - 1) {
          // tile complete: contribute this lane's row maxima to the tile's slot
          // (rows 0-127 op(A), 128-255 op(B)) and report to the epilogue
          const unsigned long long epoch = (unsigned long long)(ordinal + 1) << 32;
          unsigned long long* slot = slots + (ordinal % kMaxSlots) * 256;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (i < 3 || b_two) {
              const int srow = (i >> 1) * 128 + 32 * (b0 + 2 * (i & 1)) + lane;
              atomicMax(slot + srow, epoch | __float_as_uint(my_max[i]));
            }
            my_max[i] = 0.f;
          }
          mbar_arrive(mxfull(ordinal % kMaxSlots));
        }
      }
    }
    cp_async_wait<0>();
  } else if (warp == kFusedMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int g = 0, abuf = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int tt = blockIdx.x; tt < num_items && ok; tt += gridDim.x) {
        int4 it;
        const FusedGroup G = group_of(tt, it);
        const uint32_t idesc = make_idesc_bf16(128, G.bn);
        if (!mbar_wait_hint(acce(abuf), aphase ^ 1u, abort_flag, timeout_ns, 20000u)) {
          raise_status(status, abort_flag);
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * kFusedMaxBN);
        for (int kc = 0; kc < G.nkc; ++kc, ++g) {
          const int sb = g % kFusedStagesB;
          if (!mbar_wait_hint(bfull(sb), (uint32_t)((g / kFusedStagesB) & 1), abort_flag, timeout_ns, 1000u)) {
            raise_status(status, abort_flag);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = sB16 + (uint32_t)sb * kFusedStageB;
          const uint32_t b_addr = a_addr + kBlockBytes;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t ah = make_desc_sw128(a_addr + 32u * kk);
            const uint64_t al = make_desc_sw128(a_addr + 64u + 32u * kk);
            const uint64_t bh = make_desc_sw128(b_addr + 32u * kk);
            const uint64_t bl = make_desc_sw128(b_addr + 64u + 32u * kk);
            mma_bf16(d_tmem, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d_tmem, ah, bl, idesc, 1u);
            mma_bf16(d_tmem, al, bh, idesc, 1u);
          }
          mma_commit(bempty(sb));
        }
        if (!ok) break;
        mma_commit(accf(abuf));
        if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
      }
      mma_commit(drain_bar);
      volatile int never = 0;
      if (!mbar_wait(drain_bar, 0u, &never, timeout_ns)) raise_status(status, abort_flag);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    int abuf = 0, ordinal = 0;
    uint32_t aphase = 0;
    for (int tt = blockIdx.x; tt < num_items; tt += gridDim.x, ++ordinal) {
      int4 it;
      const FusedGroup G = group_of(tt, it);
      const int sl = ordinal % kMaxSlots;
      int ok = 1;
      if (lane == 0) ok = mbar_wait_hint(accf(abuf), aphase, abort_flag, timeout_ns, 20000u) ? 1 : 0;
      if (lane == 0 && ok)
        ok = mbar_wait_hint(mxfull(sl), (uint32_t)((ordinal / kMaxSlots) & 1), abort_flag, timeout_ns, 20000u);
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_status(status, abort_flag);
        break;
      }
      tc_fence_after();
      const int64_t m0 = (int64_t)it.y * 128, n0 = (int64_t)it.z * G.bn;
      // every epilogue warp reads the whole slot and reaches the same verdict
      const unsigned long long* slot = slots + sl * 256;
      const uint32_t epoch = (uint32_t)(ordinal + 1);
      int bad_l = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int srow = 32 * i + lane;
        const bool is_a = srow < 128;
        const int64_t r = is_a ? m0 + srow : n0 + (srow - 128);
        const bool used = is_a ? (r < G.m) : (srow - 128 < G.bn && r < G.n);
        if (used) {
          const unsigned long long v = slot[srow];
          if ((uint32_t)(v >> 32) != epoch || scale_exp_from_bits((uint32_t)v) != 0) bad_l = 1;
        }
      }
      const bool bad = __any_sync(0xFFFFFFFFu, bad_l) != 0;
      if (bad) {
        // leave C to the SIMT fallback: one 128 x 64 SIMT tile per 64 columns
        if (warp == kFusedMmaWarp + 1 && lane == 0) {
          for (int c = 0; c < G.bn && n0 + c < G.n; c += 64) {
            const int slot_i = atomicAdd(S.fb_count, 1);
            S.fb_items[slot_i] = make_int4(G.simt_index, it.y, (int)((n0 + c) / 64), 0);
          }
        }
      } else {
        const int64_t i = m0 + q * 32 + lane;
        const bool row_ok = i < G.m;
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * kFusedMaxBN);
        float* const crow = G.C + i;
        for (int c0 = 0; c0 < G.bn; c0 += 32) {
          if (n0 + c0 >= G.n) break;  // warp-uniform
          const int jmax = (G.n - (n0 + c0) < 32) ? (int)(G.n - (n0 + c0)) : 32;
          float* cp = crow + (n0 + c0) * G.ldc;
          float cv[32];
          if (G.beta != 0.f) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) cv[jj] = (row_ok && jj < jmax) ? __ldcs(cp + jj * G.ldc) : 0.f;
          }
          uint32_t r[32];
          tmem_ld32(taddr + (uint32_t)c0, r);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const float acc = __uint_as_float(r[jj]);
            const float out = (G.beta != 0.f) ? fmaf(G.alpha, acc, G.beta * cv[jj]) : G.alpha * acc;
            if (row_ok && jj < jmax) __stcs(cp + jj * G.ldc, out);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce(abuf));
      if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kFusedMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kFusedTmemCols) : "memory");
  }
}

}  // namespace
}  // namespace gbg
