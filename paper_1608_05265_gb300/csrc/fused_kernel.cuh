// Grouped split-BF16 GEMM with the split done on load ("fused"): no hi/lo
// panels in HBM.  Converter warps stream FP32 tiles of op(A) and op(B) from
// the caller's matrices into a shared-memory staging ring with cp.async
// (4-byte copies: any leading dimension and alignment), split every value
// into BF16 hi and lo in shared memory in the tensor cores' swizzled K-major
// layout, and hand each chunk to the MMA warp; the accumulator and epilogue
// work as in split_gemm_kernel.
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
//   warps 0-3   converters: cp.async copies kFusedAhead chunks ahead of the
//               chunk they convert; named barrier 1 among the 128 threads;
//   warp 4      TMEM owner (256 columns: two 128 x 128 accumulators); lane 0
//               issues the MMAs and commits;
//   warps 5-12  epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 for half of
//               the tile's columns.
#pragma once

#include "split_device.cuh"

namespace gbg {
namespace {

constexpr int kFusedConvThreads = 128;
constexpr int kFusedEpiWarps = 8;
constexpr int kFusedThreads = kFusedConvThreads + 32 + 32 * kFusedEpiWarps;
constexpr int kFusedMaxBN = 128;
constexpr int kFusedStagesF = 4;                     // FP32 staging stages
constexpr int kFusedAhead = kFusedStagesF - 1;       // chunks of copies in flight ahead of conversion
constexpr int kFusedStagesB = 2;                     // BF16 stages consumed by the MMA
constexpr int kStagePitch = 33;                      // floats per staged row (32 + 1 against bank conflicts)
constexpr uint32_t kFusedStageF = 2u * 128u * kStagePitch * 4u;          // A rows + B rows
constexpr uint32_t kFusedStageB = 2u * (uint32_t)kBlockBytes;            // A block + B block (128 rows each)
constexpr uint32_t kFusedTmemCols = 2 * kFusedMaxBN;
constexpr int kFusedSmemBytes = (int)(kFusedStagesB * kFusedStageB + kFusedStagesF * kFusedStageF) + 1024 + 2048;

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

__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void conv_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Stage the FP32 rows [r0, r0 + nrows) x k [p0, p0 + 32) of an operand (128
// threads, 32 copies each for 128 rows); out-of-range elements become zero.
__device__ __forceinline__ void stage_rows(uint32_t dst, const float* X, int64_t ld, bool kcontig, int64_t rows,
                                           int64_t k, int64_t r0, int64_t p0, int nrows, int t) {
  const int w = t >> 5, lane = t & 31;
  if (kcontig) {
    // one row per warp instruction: 32 consecutive k of row r
    for (int rr = w; rr < nrows; rr += 4) {
      const int64_t r = r0 + rr, p = p0 + lane;
      const bool ok = r < rows && p < k;
      cp_async4(dst + (uint32_t)(rr * kStagePitch + lane) * 4u, ok ? X + r * ld + p : X, ok);
    }
  } else {
    // 32 consecutive rows of one k per warp instruction
    for (int g = 0; g < nrows / 32; ++g) {
      const int rr = g * 32 + lane;
      const int64_t r = r0 + rr;
#pragma unroll 4
      for (int pp = w; pp < 32; pp += 4) {
        const int64_t p = p0 + pp;
        const bool ok = r < rows && p < k;
        cp_async4(dst + (uint32_t)(rr * kStagePitch + pp) * 4u, ok ? X + r + p * ld : X, ok);
      }
    }
  }
}

// Split 8 staged values of row rr (chunk cc) into the swizzled BF16 block;
// returns their max |x| bit pattern.
__device__ __forceinline__ uint32_t convert8(const float* srow, uint8_t* blk, int rr, int cc) {
  uint32_t hw[4], lw[4], mx = 0u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = srow[cc * 8 + 2 * q], x1 = srow[cc * 8 + 2 * q + 1];
    mx = max(mx, max(__float_as_uint(x0) & 0x7FFFFFFFu, __float_as_uint(x1) & 0x7FFFFFFFu));
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h2);
    __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    uint32_t lb = *reinterpret_cast<uint32_t*>(&l2);
    if (!isfinite(x0)) lb &= 0xFFFF0000u;  // non-finite x: lo = 0
    if (!isfinite(x1)) lb &= 0x0000FFFFu;
    hw[q] = *reinterpret_cast<const uint32_t*>(&h2);
    lw[q] = lb;
  }
  const int sw = rr & 7;
  *reinterpret_cast<uint4*>(blk + rr * 128 + ((cc ^ sw) << 4)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(blk + rr * 128 + (((cc + 4) ^ sw) << 4)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  return mx;
}

__global__ void __launch_bounds__(kFusedThreads, 1)
fused_gemm_kernel(const FusedSched S, int* status, uint64_t timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  uint8_t* const base_ptr = smem_raw + (base - raw_addr);
  const uint32_t sB16 = base;                                             // kFusedStagesB x (A block | B block)
  const uint32_t sF32 = base + kFusedStagesB * kFusedStageB;              // kFusedStagesF x (A rows | B rows)
  const uint32_t misc = sF32 + kFusedStagesF * kFusedStageF;              // maxima, flags, barriers
  uint32_t* rowmax = reinterpret_cast<uint32_t*>(base_ptr + (misc - base));   // 256 words
  int* flags = reinterpret_cast<int*>(rowmax + 256);                           // 4-entry ring
  int* tile_bad = flags + 4;
  volatile int* conv_go = flags + 5;  // thread 0's go/stop decision for the converters, read after a barrier
  const uint32_t bar0 = (misc + 256 * 4 + 64 + 7) & ~7u;
  auto bfull = [&](int s) { return bar0 + 8u * s; };
  auto bempty = [&](int s) { return bar0 + 8u * (kFusedStagesB + s); };
  auto accf = [&](int b) { return bar0 + 8u * (2 * kFusedStagesB + b); };
  auto acce = [&](int b) { return bar0 + 8u * (2 * kFusedStagesB + 2 + b); };
  auto flagbar = [&](int i) { return bar0 + 8u * (2 * kFusedStagesB + 4 + i); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kFusedStagesB + 8);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(base_ptr + (bar0 - base) + 8 * (2 * kFusedStagesB + 9));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_items = S.n_items;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFusedStagesB; ++s) { mbar_init(bfull(s), 1); mbar_init(bempty(s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf(b), 1); mbar_init(acce(b), kFusedEpiWarps); }
    for (int i = 0; i < 4; ++i) mbar_init(flagbar(i), 1);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (threadIdx.x < 256) rowmax[threadIdx.x] = 0u;
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_holder)), "r"(kFusedTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  auto group_of = [&](int t, int4& it) -> const FusedGroup& {
    it = S.items[t];
    return S.groups[it.x];
  };

  if (warp < 4) {
    // ---------------- converters ----------------
    const int t = threadIdx.x;
    // issue cursor (item, k chunk) runs kFusedAhead chunks ahead of the convert cursor
    int it_i = blockIdx.x, kc_i = 0;
    int issued = 0;
    auto issue_next = [&]() {
      if (it_i < num_items) {
        int4 it;
        const FusedGroup& G = group_of(it_i, it);
        const uint32_t st = sF32 + (uint32_t)(issued % kFusedStagesF) * kFusedStageF;
        const int64_t p0 = (int64_t)kc_i * 32;
        stage_rows(st, G.A, G.lda, G.a_kcontig != 0, G.m, G.k, (int64_t)it.y * 128, p0, 128, t);
        stage_rows(st + 128u * kStagePitch * 4u, G.B, G.ldb, G.b_kcontig != 0, G.n, G.k, (int64_t)it.z * G.bn, p0,
                   G.bn, t);
        if (++kc_i == G.nkc) { kc_i = 0; it_i += gridDim.x; }
      }
      cp_async_commit();  // an empty group keeps the group count in step
      ++issued;
    };
    for (int a = 0; a < kFusedAhead; ++a) issue_next();
    uint32_t my_max[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) my_max[i] = 0u;
    int g = 0, ordinal = 0;
    bool ok = true;
    for (int tt = blockIdx.x; tt < num_items && ok; tt += gridDim.x, ++ordinal) {
      int4 it;
      const FusedGroup& G = group_of(tt, it);
      const int items = (128 + G.bn) * 4;  // (row, 8-wide chunk) items: A rows then B rows
      for (int kc = 0; kc < G.nkc; ++kc, ++g) {
        issue_next();
        cp_async_wait<kFusedAhead>();  // chunk g's copies by this thread have landed
        const int sb = g % kFusedStagesB;
        if (t == 0) {
          const bool go = mbar_wait(bempty(sb), (uint32_t)(((g / kFusedStagesB) & 1) ^ 1), abort_flag, timeout_ns);
          if (!go) raise_status(status, abort_flag);
          *conv_go = (go && !*abort_flag) ? 1 : 0;
        }
        conv_bar();  // every converter's copies of chunk g are visible; the BF16 stage is free
        if (!*conv_go) { ok = false; break; }  // the same decision in all 128 threads
        const float* stf = reinterpret_cast<const float*>(base_ptr + (sF32 - base) + (uint32_t)(g % kFusedStagesF) * kFusedStageF);
        uint8_t* stb = base_ptr + (sB16 - base) + (uint32_t)sb * kFusedStageB;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int item = t + 128 * i;
          if (item < items) {
            const int row = item >> 2, cc = item & 3;  // rows 0-127: op(A); 128-: op(B)
            const uint32_t mx = convert8(stf + row * kStagePitch, stb, row, cc);
            my_max[i] = max(my_max[i], mx);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // BF16 writes -> tensor core reads
        if (kc == G.nkc - 1) {
          // tile complete: exact max |x| of its vectors; flag the tile if any is badly scaled
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int item = t + 128 * i;
            if (item < items && my_max[i] != 0u) atomicMax(&rowmax[item >> 2], my_max[i]);
            my_max[i] = 0u;
          }
          if (t == 0) *tile_bad = 0;
          conv_bar();
          const int64_t rA = (int64_t)it.y * 128 + t, rB = (int64_t)it.z * G.bn + t;
          int bad = 0;
          if (rA < G.m && scale_exp_from_bits(rowmax[t]) != 0) bad = 1;
          if (t < G.bn && rB < G.n && scale_exp_from_bits(rowmax[128 + t]) != 0) bad = 1;
          if (bad) atomicOr(tile_bad, 1);
          conv_bar();
          rowmax[t] = 0u;
          rowmax[128 + t] = 0u;
          if (t == 0) {
            flags[ordinal & 3] = *tile_bad;
            mbar_arrive(flagbar(ordinal & 3));
          }
        }
        conv_bar();  // all conversions of chunk g done: its FP32 stage may be refilled
        if (t == 0) mbar_arrive(bfull(sb));
      }
    }
    cp_async_wait<0>();
  } else if (warp == 4) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int g = 0, abuf = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int tt = blockIdx.x; tt < num_items && ok; tt += gridDim.x) {
        int4 it;
        const FusedGroup& G = group_of(tt, it);
        const uint32_t idesc = make_idesc_bf16(128, G.bn);
        if (!mbar_wait(acce(abuf), aphase ^ 1u, abort_flag, timeout_ns)) {
          raise_status(status, abort_flag);
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * kFusedMaxBN);
        for (int kc = 0; kc < G.nkc; ++kc, ++g) {
          const int sb = g % kFusedStagesB;
          if (!mbar_wait(bfull(sb), (uint32_t)((g / kFusedStagesB) & 1), abort_flag, timeout_ns)) {
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
    const int half = (warp - 5) >> 2;
    int abuf = 0, ordinal = 0;
    uint32_t aphase = 0;
    for (int tt = blockIdx.x; tt < num_items; tt += gridDim.x, ++ordinal) {
      int4 it;
      const FusedGroup& G = group_of(tt, it);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(accf(abuf), aphase, abort_flag, timeout_ns) ? 1 : 0;
      if (lane == 0 && ok) ok = mbar_wait(flagbar(ordinal & 3), (uint32_t)((ordinal >> 2) & 1), abort_flag, timeout_ns);
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_status(status, abort_flag);
        break;
      }
      tc_fence_after();
      const int bad = flags[ordinal & 3];
      const int64_t m0 = (int64_t)it.y * 128, n0 = (int64_t)it.z * G.bn;
      if (bad) {
        // leave C to the SIMT fallback: one 128 x 64 SIMT tile per 64 columns
        if (warp == 5 && lane == 0) {
          for (int c = 0; c < G.bn && n0 + c < G.n; c += 64) {
            const int slot = atomicAdd(S.fb_count, 1);
            S.fb_items[slot] = make_int4(G.simt_index, it.y, (int)((n0 + c) / 64), 0);
          }
        }
      } else {
        const int64_t i = m0 + q * 32 + lane;
        const bool row_ok = i < G.m;
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * kFusedMaxBN);
        float* const crow = G.C + i;
        const int c_begin = half * (G.bn >> 1), c_end = c_begin + (G.bn >> 1);
        for (int c0 = c_begin; c0 < c_end; c0 += 32) {
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
  if (warp == 4) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kFusedTmemCols) : "memory");
  }
}

}  // namespace
}  // namespace gbg
