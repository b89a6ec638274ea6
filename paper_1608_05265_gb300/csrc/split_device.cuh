// Device helpers of the split-BF16 path, shared by the single-problem
// launches (split.cu) and the grouped plans (grouped.cu): scaling and hi/lo
// splitting, panel-chunk stores, the re-pack of badly scaled rows, and the
// PTX wrappers for mbarriers, asynchronous copies, fences and tcgen05 (MMA,
// commit, TMEM loads).
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace gbg {
namespace {

// ---------------------------------------------------------------------------
// Shared helpers
// ---------------------------------------------------------------------------

// Scaling exponent of a K-vector from the bits of its max magnitude: 0 for
// 0, Inf, NaN and for well-scaled maxima in [2^-48, 2^48); otherwise the
// frexp exponent, which brings the max into [0.5, 1).
constexpr uint32_t kWellScaledLo = (127u - 48u) << 23;  // bits of 2^-48
constexpr uint32_t kWellScaledHi = (127u + 48u) << 23;  // bits of 2^48
__device__ __forceinline__ int scale_exp_from_bits(uint32_t b) {
  if (b == 0u || b >= 0x7F800000u) return 0;
  if (b >= kWellScaledLo && b < kWellScaledHi) return 0;
  const int E = (int)(b >> 23);
  if (E > 0) return E - 126;
  return (32 - __clz(b)) - 149;  // subnormal: value = b * 2^-149
}

// x * 2^-e with a single rounding (exact unless the product is subnormal).
__device__ __forceinline__ float scale_pow2(float x, int e) {
  const int s = -e;  // s in [-128, 148]
  if (s >= -126 && s <= 127) return x * __int_as_float((s + 127) << 23);
  if (s < -126) return x * __int_as_float(1 << (s + 149));  // 2^-127, 2^-128: subnormal powers of two
  // s > 127 only when the whole row is subnormal: both steps are exact.
  return (x * 0x1p127f) * __int_as_float((s - 127 + 127) << 23);
}

__device__ __forceinline__ void split_bf16(float xs, uint32_t& h, uint32_t& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(xs);
  h = (uint32_t)__bfloat16_as_ushort(hb);
  if (!isfinite(xs)) { l = 0u; return; }
  const float r = xs - __bfloat162float(hb);
  l = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(r));
}

// ---------------------------------------------------------------------------
// Split and pack.  One pass writes the hi/lo panel of the UNSCALED
// operand and the max |x| of every K-vector (bit patterns; NaN > Inf >
// finite as unsigned).  Well-scaled vectors (the large majority) are then
// final.  A second, usually empty pass re-packs the badly scaled ones with
// their scaling exponent.  For a well-scaled vector the two definitions
// give the same GEMM result: scaling by a power of two commutes with every
// FP32 rounding as long as nothing leaves the normal range.
//
// Thread work item: one row r of a 128-row x 32-k block and one 8-wide
// k-chunk cc (0..3) -> two 16-byte stores (hi chunk cc, lo chunk cc + 4) at
// chunk positions XOR (r mod 8).
// ---------------------------------------------------------------------------

// Two floats rounded to BF16 (RN-even) in one instruction: `a` into the
// low half, `b` into the high half.
__device__ __forceinline__ uint32_t cvt_bf16x2(float a, float b) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
  return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t d) { return __uint_as_float(d << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t d) { return __uint_as_float(d & 0xFFFF0000u); }

// True when none of the 8 values is Inf or NaN (the packed splits below
// apply; otherwise the element-wise ones, which give lo = 0 for them).
__device__ __forceinline__ bool all_finite8(const float (&x)[8]) {
  uint32_t e = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) e = max(e, __float_as_uint(x[q]) & 0x7F800000u);
  return e != 0x7F800000u;
}

// Split 8 values (already scaled) and store the hi and lo chunks of row rr.
__device__ __forceinline__ void store_split8(uint8_t* blk, int rr, int cc, const float (&x)[8]) {
  uint32_t hw[4], lw[4];
  if (all_finite8(x)) {
    // x - hi is exact in FP32, so the packed form equals the element-wise one
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hw[q] = cvt_bf16x2(x[2 * q], x[2 * q + 1]);
      lw[q] = cvt_bf16x2(x[2 * q] - bf16_lo(hw[q]), x[2 * q + 1] - bf16_hi(hw[q]));
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t h0, l0, h1, l1;
      split_bf16(x[2 * q], h0, l0);
      split_bf16(x[2 * q + 1], h1, l1);
      hw[q] = h0 | (h1 << 16);
      lw[q] = l0 | (l1 << 16);
    }
  }
  const int sw = rr & 7;
  *reinterpret_cast<uint4*>(blk + rr * 128 + ((cc ^ sw) << 4)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(blk + rr * 128 + (((cc + 4) ^ sw) << 4)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// Three-part split of 8 values: [hi | mid] into blk (as store_split8, mid =
// the two-part lo) into blk and lo3 = bf16((x - hi) - mid) into half `half` of the compact block blk2.
__device__ __forceinline__ void store_split8_3(uint8_t* blk, uint8_t* blk2, int half, int rr, int cc,
                                               const float (&x)[8]) {
  uint32_t hw[4], mw[4], lw[4];
  if (all_finite8(x)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hw[q] = cvt_bf16x2(x[2 * q], x[2 * q + 1]);
      const float r0 = x[2 * q] - bf16_lo(hw[q]), r1 = x[2 * q + 1] - bf16_hi(hw[q]);
      mw[q] = cvt_bf16x2(r0, r1);
      lw[q] = cvt_bf16x2(r0 - bf16_lo(mw[q]), r1 - bf16_hi(mw[q]));
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t hb[2], mb[2], lb[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float v = x[2 * q + u];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hb[u] = (uint32_t)__bfloat16_as_ushort(h);
        if (!isfinite(v)) { mb[u] = 0u; lb[u] = 0u; continue; }
        const float r1 = v - __bfloat162float(h);
        const __nv_bfloat16 mdl = __float2bfloat16_rn(r1);
        mb[u] = (uint32_t)__bfloat16_as_ushort(mdl);
        lb[u] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(mdl)));
      }
      hw[q] = hb[0] | (hb[1] << 16);
      mw[q] = mb[0] | (mb[1] << 16);
      lw[q] = lb[0] | (lb[1] << 16);
    }
  }
  const int sw = rr & 7;
  *reinterpret_cast<uint4*>(blk + rr * 128 + ((cc ^ sw) << 4)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(blk + rr * 128 + (((cc + 4) ^ sw) << 4)) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
  // lo3 of an even k chunk in logical chunks 0-3 of the compact block, of an
  // odd one in 4-7
  *reinterpret_cast<uint4*>(blk2 + rr * 128 + (((cc + 4 * half) ^ sw) << 4)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05, bulk copy, mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}

// As mbar_try, but a thread whose phase is not complete may be suspended for
// up to `hint_ns` (it resumes as soon as the phase completes): long waits
// then take no issue slots from the warps doing work.
__device__ __forceinline__ bool mbar_try_hint(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0u;
}

// Wait for the phase of parity `parity` to complete.  Gives up (returns
// false) once `timeout_ns` has passed or another role raised the abort flag.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint64_t timeout_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 31u) == 0u) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > timeout_ns) return false;
    }
  }
}

// mbar_wait with suspending polls (see mbar_try_hint); same limits.
__device__ __noinline__ bool mbar_wait_hint(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                            uint64_t timeout_ns, uint32_t hint_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_hint(bar, parity, hint_ns)) return true;
    if ((it & 7u) == 0u) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > timeout_ns) return false;
    }
  }
}

// Ask L2 for the 128-byte line holding `p`.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile whose rows are
// 128 bytes, 8-row groups 1024 bytes apart, 128-byte swizzle.
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4)   // start address
         | ((uint64_t)1 << 16)                 // leading byte offset (unused for swizzled K-major)
         | ((uint64_t)(1024 >> 4) << 32)       // stride byte offset: 8 rows x 128 B
         | ((uint64_t)1 << 46)                 // descriptor version
         | ((uint64_t)2 << 61);                // 128-byte swizzle
}

// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N) {
  return (1u << 4)                 // D format FP32
         | (1u << 7)               // A format BF16
         | (1u << 10)              // B format BF16
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Clusters of two CTAs (pair tiles): the CTA's rank in its cluster, the
// cluster index and count along x, a barrier over every thread of the
// cluster, and mbarrier operations across the pair.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t num_clusters_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The shared::cluster address of shared-memory offset `saddr` in CTA `rank`.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
// Arrive on an mbarrier of another CTA of the cluster.  The default
// (CTA-scope) release: a cluster-scope release would make the arriving
// thread wait for its own earlier global stores to complete, and nothing the
// other CTA reads after the arrival was written by this thread's generic
// stores (its operands land by bulk copies, and TMEM reads are ordered by
// tcgen05 fences).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// The MMA of a CTA pair (issued by the even CTA): M = 256 rows, 128 from
// each CTA's A block at the same shared-memory offset; the B operand's N
// rows are half in each CTA's shared memory (again at the same offset); each
// CTA's TMEM receives its own 128 rows of the accumulator.
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive on the mbarrier at offset `bar` of every CTA in `mask` once the
// pair MMAs issued so far have completed.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
               ::"r"(bar), "h"(mask) : "memory");
}

__device__ __forceinline__ void raise_status(int* status, volatile int* abort_flag) {
  *abort_flag = 1;
  atomicCAS(status, 0, (int)GBGEMM_ERR_DEVICE_TIMEOUT);
}

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group, int& tm, int& tn) {
  const int per_group = group * tiles_n;
  const int g = t / per_group;
  const int first_m = g * group;
  const int gm = min(group, tiles_m - first_m);
  const int r = t - g * per_group;
  tm = first_m + r % gm;
  tn = r / gm;
}

// Panels hold `rows_alloc` rows (a multiple of 8) per k chunk: row r of
// chunk kc is the 128 bytes at (kc*rows_alloc + r)*128.  Rows from `rows`
// up to rows_alloc are written as zeros, rows past rows_alloc not at all.
// With a second panel the three-part split is written ([hi | mid] into the
// panel, lo3 into the compact panel2: block kc / 2, half kc % 2).

// Re-pack the badly scaled K-vectors of one 128-row block over all k chunks
// with x' = x * 2^-e (one CTA of 256 threads).  A block without such rows
// returns at once.  The maxima are read through L2 (they were built by
// atomics of other CTAs).  se: 128 ints of shared memory.
__device__ __forceinline__ void rescale_block(int64_t rows, int64_t k, const float* __restrict__ X, int64_t ld,
                                              bool kcontig, const uint32_t* __restrict__ amax,
                                              uint8_t* __restrict__ panel, uint8_t* __restrict__ panel2,
                                              int64_t rows_alloc, int64_t nkc, int64_t rb, int* se) {
  const int64_t r0 = rb * 128;
  const int tid = threadIdx.x;
  int e = 0;
  if (tid < 128 && r0 + tid < rows) e = scale_exp_from_bits(__ldcg(&amax[r0 + tid]));
  if (tid < 128) se[tid] = e;
  if (!__syncthreads_or(e != 0)) return;
  for (int64_t kc = 0; kc < nkc; ++kc) {
    const size_t boff = ((size_t)kc * rows_alloc + r0) * 128;
    const size_t boff2 = ((size_t)(kc >> 1) * rows_alloc + r0) * 128;
    uint8_t* blk = panel + boff;
    for (int it = 0; it < 2; ++it) {
      const int idx = tid + 256 * it, rr = idx >> 2, cc = idx & 3;
      const int er = se[rr];
      if (er == 0 || r0 + rr >= rows_alloc) continue;
      const int64_t r = r0 + rr, p = kc * 32 + cc * 8;
      float x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float v = (r < rows && p + q < k) ? (kcontig ? X[r * ld + p + q] : X[r + (p + q) * ld]) : 0.f;
        x[q] = isfinite(v) ? scale_pow2(v, er) : v;
      }
      if (panel2) store_split8_3(blk, panel2 + boff2, (int)(kc & 1), rr, cc, x);
      else store_split8(blk, rr, cc, x);
    }
  }
}

}  // namespace
}  // namespace gbg
