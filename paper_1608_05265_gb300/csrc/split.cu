// Split-BF16 tensor-core sgemm for sm_103a: the scaling/packing kernels and
// the persistent tcgen05 GEMM.
//
// Method.  Every K-vector of the problem -- a row of op(A) or a column of
// op(B) -- is scaled by 2^-e, e being the frexp exponent of its largest
// magnitude, so its entries lie in (-1, 1).  Each scaled entry x' becomes
// hi = bf16_rn(x') and lo = bf16_rn(x' - hi) (x' - hi is exact in FP32).  The
// tensor cores accumulate hi_a*hi_b + hi_a*lo_b + lo_a*hi_b in FP32 and the
// epilogue multiplies by 2^(e_i + f_j), then applies alpha and beta once.
//
// Structure (after the paper's BLIS sgemm, Sections III-A and III-C):
//  * packing -- the BLIS packing of A and B panels becomes a pass that writes
//    hi/lo BF16 panels in exactly the byte order the tensor cores read from
//    shared memory (128-byte rows, 16-byte chunks XOR-swizzled by row mod 8);
//  * the micro-kernel's k loop -- the paper sends KSUB-deep blocks of a1 and
//    b1 into two alternating buffers with a `selector` while the coprocessor
//    works on the other (Section III-C).  Here a producer thread streams
//    32-deep blocks with bulk asynchronous copies into a ring of shared
//    memory stages guarded by full/empty mbarriers;
//  * the Accumulator -- the paper's `command` 0/1/2/3 protocol (clear on the
//    first block, accumulate, send the result on the last) becomes the
//    tcgen05.mma accumulate flag (off for the first MMA of a tile) and a
//    commit to an "accumulator full" barrier after the last block.  The
//    accumulator lives in tensor memory (TMEM), two buffers of 128 x BN FP32
//    so that the epilogue of one tile overlaps the main loop of the next;
//  * output ownership -- each CTA owns whole 128 x BN tiles of column-major
//    C, and the epilogue writes each column's 128 rows with one coalesced
//    warp store per 32 rows (Section III-D assigns each core whole column
//    blocks of the result for the same reason).
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
// K1: split and pack.  One pass writes the hi/lo panel of the UNSCALED
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

// Split 8 values (already scaled) and store the hi and lo chunks of row rr.
__device__ __forceinline__ void store_split8(uint8_t* blk, int rr, int cc, const float (&x)[8]) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t h0, l0, h1, l1;
    split_bf16(x[2 * q], h0, l0);
    split_bf16(x[2 * q + 1], h1, l1);
    hw[q] = h0 | (h1 << 16);
    lw[q] = l0 | (l1 << 16);
  }
  const int sw = rr & 7;
  *reinterpret_cast<uint4*>(blk + rr * 128 + ((cc ^ sw) << 4)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(blk + rr * 128 + (((cc + 4) ^ sw) << 4)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// Item mapping inside a 256-thread CTA, two items per thread.
// KCONTIG (element (r,p) at X[r*ld + p]): four lanes per row, eight rows per
//   warp, so a warp reads eight 128-byte row segments.
// !KCONTIG (element (r,p) at X[r + p*ld]): 32 consecutive rows per warp and
//   one chunk per warp, so every load instruction reads 128 contiguous bytes.
template <bool KCONTIG>
__device__ __forceinline__ void item_of(int tid, int it, int& rr, int& cc) {
  if (KCONTIG) {
    const int idx = tid + 256 * it;
    rr = idx >> 2;
    cc = idx & 3;
  } else {
    const int w = tid >> 5;
    cc = w & 3;
    rr = ((w >> 2) + 2 * it) * 32 + (tid & 31);
  }
}

template <bool KCONTIG>
__device__ __forceinline__ void load8(const float* __restrict__ X, int64_t ld, int64_t r, int64_t p, int64_t rows,
                                      int64_t k, bool vec, float (&x)[8]) {
  if (KCONTIG) {
    if (r < rows && vec && p + 8 <= k) {
      const float4 a = *reinterpret_cast<const float4*>(X + r * ld + p);
      const float4 b = *reinterpret_cast<const float4*>(X + r * ld + p + 4);
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = (r < rows && p + q < k) ? X[r * ld + p + q] : 0.f;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = (r < rows && p + q < k) ? X[r + (p + q) * ld] : 0.f;
  }
}

template <bool KCONTIG>
__global__ void __launch_bounds__(256) pack_kernel(int64_t rows, int64_t k, const float* __restrict__ X, int64_t ld,
                                                   uint32_t* __restrict__ amax, uint8_t* __restrict__ panel,
                                                   int64_t rb_count) {
  __shared__ uint32_t smax[128];
  const int64_t rb = blockIdx.x, kc = blockIdx.y;
  const int64_t r0 = rb * 128, p0 = kc * 32;
  const int tid = threadIdx.x;
  const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (tid < 128) smax[tid] = 0u;
  float x[2][8];
#pragma unroll
  for (int it = 0; it < 2; ++it) {  // all loads first: 16 (or 4 vector) loads in flight per thread
    int rr, cc;
    item_of<KCONTIG>(tid, it, rr, cc);
    load8<KCONTIG>(X, ld, r0 + rr, p0 + cc * 8, rows, k, vec, x[it]);
  }
  __syncthreads();
  uint8_t* blk = panel + (size_t)(kc * rb_count + rb) * kBlockBytes;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    int rr, cc;
    item_of<KCONTIG>(tid, it, rr, cc);
    uint32_t mx = 0u;
#pragma unroll
    for (int q = 0; q < 8; ++q) mx = max(mx, __float_as_uint(x[it][q]) & 0x7FFFFFFFu);
    store_split8(blk, rr, cc, x[it]);
    if (KCONTIG) {
      mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 1));
      mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 2));
      if (cc == 0 && mx != 0u) atomicMax(&smax[rr], mx);
    } else if (mx != 0u) {
      atomicMax(&smax[rr], mx);
    }
  }
  __syncthreads();
  if (tid < 128 && r0 + tid < rows && smax[tid] != 0u) atomicMax(&amax[r0 + tid], smax[tid]);
}

// Re-pack the badly scaled K-vectors of one 128-row block over all k chunks
// with x' = x * 2^-e.  A block without such rows returns at once.
__global__ void __launch_bounds__(256) rescale_kernel(int64_t rows, int64_t k, const float* __restrict__ X, int64_t ld,
                                                      bool kcontig, const uint32_t* __restrict__ amax,
                                                      uint8_t* __restrict__ panel, int64_t rb_count, int64_t nkc) {
  __shared__ int se[128];
  const int64_t rb = blockIdx.x, r0 = rb * 128;
  const int tid = threadIdx.x;
  int e = 0;
  if (tid < 128 && r0 + tid < rows) e = scale_exp_from_bits(amax[r0 + tid]);
  if (tid < 128) se[tid] = e;
  if (!__syncthreads_or(e != 0)) return;
  for (int64_t kc = 0; kc < nkc; ++kc) {
    uint8_t* blk = panel + (size_t)(kc * rb_count + rb) * kBlockBytes;
    for (int it = 0; it < 2; ++it) {
      const int idx = tid + 256 * it, rr = idx >> 2, cc = idx & 3;
      const int er = se[rr];
      if (er == 0) continue;
      const int64_t r = r0 + rr, p = kc * 32 + cc * 8;
      float x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float v = (r < rows && p + q < k) ? (kcontig ? X[r * ld + p + q] : X[r + (p + q) * ld]) : 0.f;
        x[q] = isfinite(v) ? scale_pow2(v, er) : v;
      }
      store_split8(blk, rr, cc, x);
    }
  }
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

// ---------------------------------------------------------------------------
// K3: persistent split-BF16 GEMM.
// Warp 0 lane 0: producer.  Warp 1: TMEM owner, lane 0 issues the MMAs.
// Warps 2-9: epilogue; warp w reads TMEM lanes 32*(w%4) .. +31 (the rows it
// owns) and columns [h*BN/2, (h+1)*BN/2) with h = (w-2)/4.
// ---------------------------------------------------------------------------
constexpr int kStages = 4;
constexpr int kEpiWarps = 8;                       // two per TMEM lane quadrant, each half of the columns
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue warps
constexpr uint64_t kTimeoutNs = 2000000000ull;

struct GemmParams {
  const uint8_t* panelA; const uint8_t* panelB;
  const uint32_t* amaxA; const uint32_t* amaxB;
  int64_t m, n;
  float alpha, beta;
  float* C; int64_t ldc;
  int* status;
  int tiles_m, tiles_n, nkc, raster;
  int64_t rbA, rbB;
  uint64_t timeout_ns;
};

template <int BN>
constexpr int gemm_smem_bytes() {
  return kStages * (kBlockBytes + BN * 128) + 1024 + 256;
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) split_gemm_kernel(const GemmParams P) {
  constexpr uint32_t A_BYTES = kBlockBytes;        // 128 rows x 128 B
  constexpr uint32_t B_BYTES = BN * 128;           // BN rows x 128 B
  constexpr uint32_t TMEM_COLS = 2 * BN;           // two accumulator buffers
  constexpr uint32_t IDESC = make_idesc_bf16(128, BN);

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  uint8_t* const base_ptr = smem_raw + (base - raw_addr);
  const uint32_t sA = base;                                   // kStages x A_BYTES
  const uint32_t sB = base + kStages * A_BYTES;               // kStages x B_BYTES
  const uint32_t bar0 = sB + kStages * B_BYTES;               // barriers
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * kStages + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 4);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(base_ptr + (bar0 - base) + 8 * (2 * kStages + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_tiles = P.tiles_m * P.tiles_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf_bar(b), 1); mbar_init(acce_bar(b), kEpiWarps); }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_holder)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued_phase[kStages];
      bool issued[kStages];
      for (int s = 0; s < kStages; ++s) { issued[s] = false; issued_phase[s] = 0; }
      bool ok = true;
      for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
        int tm, tn;
        tile_coords(t, P.tiles_m, P.tiles_n, P.raster, tm, tn);
        const uint8_t* a_src = P.panelA + (size_t)tm * A_BYTES;
        const uint8_t* b_src = P.panelB + (size_t)tn * (BN / 128) * kBlockBytes;
        for (int kc = 0; kc < P.nkc; ++kc) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, P.timeout_ns)) {
            raise_status(P.status, abort_flag);
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(stage), A_BYTES + B_BYTES);
          bulk_copy_g2s(sA + stage * A_BYTES, a_src + (size_t)kc * P.rbA * kBlockBytes, A_BYTES, full_bar(stage));
          bulk_copy_g2s(sB + stage * B_BYTES, b_src + (size_t)kc * P.rbB * kBlockBytes, B_BYTES, full_bar(stage));
          issued[stage] = true;
          issued_phase[stage] = (int)phase;
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
      // Let every copy this thread started land before the CTA can exit.
      volatile int never = 0;
      for (int s = 0; s < kStages; ++s)
        if (issued[s]) (void)mbar_wait(full_bar(s), (uint32_t)issued_phase[s], &never, P.timeout_ns);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int abuf = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
        if (!mbar_wait(acce_bar(abuf), aphase ^ 1u, abort_flag, P.timeout_ns)) {
          raise_status(P.status, abort_flag);
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * BN);
        for (int kc = 0; kc < P.nkc; ++kc) {
          if (!mbar_wait(full_bar(stage), phase, abort_flag, P.timeout_ns)) {
            raise_status(P.status, abort_flag);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = sA + stage * A_BYTES;
          const uint32_t b_addr = sB + stage * B_BYTES;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t ah = make_desc_sw128(a_addr + 32u * kk);
            const uint64_t al = make_desc_sw128(a_addr + 64u + 32u * kk);
            const uint64_t bh = make_desc_sw128(b_addr + 32u * kk);
            const uint64_t bl = make_desc_sw128(b_addr + 64u + 32u * kk);
            mma_bf16(d_tmem, ah, bh, IDESC, (kc > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d_tmem, ah, bl, IDESC, 1u);
            mma_bf16(d_tmem, al, bh, IDESC, 1u);
          }
          mma_commit(empty_bar(stage));  // frees the stage once these MMAs have read it
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(accf_bar(abuf));      // the tile's accumulator is complete
        if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
      }
      // Wait until every MMA issued here has finished before TMEM is released.
      mma_commit(drain_bar);
      volatile int never = 0;
      if (!mbar_wait(drain_bar, 0u, &never, P.timeout_ns)) raise_status(P.status, abort_flag);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const int c_begin = ((warp - 2) >> 2) * (BN / 2);
    int abuf = 0;
    uint32_t aphase = 0;
    for (int t = blockIdx.x; t < num_tiles; t += gridDim.x) {
      int tm, tn;
      tile_coords(t, P.tiles_m, P.tiles_n, P.raster, tm, tn);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(accf_bar(abuf), aphase, abort_flag, P.timeout_ns) ? 1 : 0;
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_status(P.status, abort_flag);
        break;
      }
      tc_fence_after();
      const int64_t i = (int64_t)tm * 128 + q * 32 + lane;
      const int64_t n0 = (int64_t)tn * BN;
      const bool row_ok = i < P.m;
      const int ea = row_ok ? scale_exp_from_bits(P.amaxA[i]) : 0;
      const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * BN);
      float* const crow = P.C + i;
      for (int c0 = c_begin; c0 < c_begin + BN / 2; c0 += 32) {
        if (n0 + c0 >= P.n) break;  // warp-uniform
        const int jmax = (P.n - (n0 + c0) < 32) ? (int)(P.n - (n0 + c0)) : 32;
        float* cp = crow + (n0 + c0) * P.ldc;
        // All loads of the chunk are issued before any result is formed, so
        // the 32 column reads of C overlap instead of queueing one by one.
        float cv[32];
        if (P.beta != 0.f) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) cv[jj] = (row_ok && jj < jmax) ? __ldcs(cp + jj * P.ldc) : 0.f;
        }
        const int64_t jl = n0 + c0 + lane;
        const int eb_l = (jl < P.n) ? scale_exp_from_bits(P.amaxB[jl]) : 0;
        uint32_t r[32];
        tmem_ld32(taddr + (uint32_t)c0, r);
        // Every lane runs every shuffle; only the stores are predicated.
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int s = ea + __shfl_sync(0xFFFFFFFFu, eb_l, jj);
          const float acc = __uint_as_float(r[jj]);
          // acc * 2^s: one multiply when 2^s is a normal float, else scalbnf.
          const float v = (s >= -126 && s <= 127) ? acc * __int_as_float((s + 127) << 23) : scalbnf(acc, s);
          const float out = (P.beta != 0.f) ? fmaf(P.alpha, v, P.beta * cv[jj]) : P.alpha * v;
          if (row_ok && jj < jmax) __stcs(cp + jj * P.ldc, out);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce_bar(abuf));
      if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

template <int BN>
cudaError_t launch_gemm_bn(const SplitGemmArgs& a, cudaStream_t s) {
  GemmParams P;
  P.panelA = static_cast<const uint8_t*>(a.panelA);
  P.panelB = static_cast<const uint8_t*>(a.panelB);
  P.amaxA = a.amaxA;
  P.amaxB = a.amaxB;
  P.m = a.m; P.n = a.n;
  P.alpha = a.alpha; P.beta = a.beta;
  P.C = a.C; P.ldc = a.ldc;
  P.status = a.status;
  const int64_t tm = (a.m + 127) / 128, tn = (a.n + BN - 1) / BN;
  if (tm * tn > (int64_t)0x7FFFFFFF || panel_k_chunks(a.k) > (int64_t)0x7FFFFFFF) return cudaErrorInvalidValue;
  P.tiles_m = (int)tm; P.tiles_n = (int)tn;
  P.nkc = (int)panel_k_chunks(a.k);
  P.raster = a.raster > 0 ? a.raster : 16;
  P.rbA = panel_row_blocks(a.m);
  P.rbB = panel_row_blocks(a.n);
  P.timeout_ns = kTimeoutNs;
  constexpr int smem = gemm_smem_bytes<BN>();
  // The shared-memory opt-in is a per-device function attribute: set it once
  // for every device this kernel instance is launched on.
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(split_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  const int64_t tiles = tm * tn;
  const int grid = (int)(tiles < (int64_t)(a.num_sms > 0 ? a.num_sms : 148) ? tiles : (int64_t)(a.num_sms > 0 ? a.num_sms : 148));
  split_gemm_kernel<BN><<<grid, kGemmThreads, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split_pack(int64_t rows, int64_t k, const float* X, int64_t ld, bool kcontig,
                              uint32_t* amax_bits, void* panel, cudaStream_t s) {
  if (rows <= 0 || k <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(amax_bits, 0, (size_t)rows * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const int64_t rbc = panel_row_blocks(rows);
  const int64_t nkc = panel_k_chunks(k);
  dim3 g((unsigned)rbc, (unsigned)nkc);
  if (g.y > 65535u) return cudaErrorInvalidConfiguration;
  uint8_t* pn = static_cast<uint8_t*>(panel);
  if (kcontig) pack_kernel<true><<<g, 256, 0, s>>>(rows, k, X, ld, amax_bits, pn, rbc);
  else pack_kernel<false><<<g, 256, 0, s>>>(rows, k, X, ld, amax_bits, pn, rbc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rescale_kernel<<<(unsigned)rbc, 256, 0, s>>>(rows, k, X, ld, kcontig, amax_bits, pn, rbc, nkc);
  return cudaGetLastError();
}

cudaError_t launch_split_gemm(const SplitGemmArgs& a, cudaStream_t s) {
  if (a.m <= 0 || a.n <= 0 || a.k <= 0) return cudaSuccess;
  if (a.bn == 128) return launch_gemm_bn<128>(a, s);
  return launch_gemm_bn<256>(a, s);
}

}  // namespace gbg
