// The persistent split-BF16 tcgen05 GEMM kernel, templated on its tile
// scheduler: SingleSched walks the tiles of one problem in a rasterised
// order, GroupedSched walks a cost-sorted list of (group, tile row, tile
// column) items over many problems.  The per-tile job carries everything a
// role needs, including the tile width BN (64, 128 or 256) as a run-time
// value: the MMA instruction descriptor, the B copy size and the epilogue
// width all follow it, and shared memory and TMEM are sized for 256.
//
// Roles (one CTA per SM, 576 threads):
//   warp 0, lane 0  producer: per 32-deep k chunk one bulk async copy of the
//                   128-row A block and one of the BN-row B rows into a
//                   4-stage ring, signalled on the stage's "full" mbarrier;
//   warp 1          owns TMEM (512 columns: two 128 x 256 FP32
//                   accumulators); lane 0 issues the MMAs (hi*hi, hi*lo,
//                   lo*hi for both 16-deep halves of a chunk), commits each
//                   stage to its "empty" barrier and each finished tile to an
//                   "accumulator full" barrier -- the paper's Accumulator
//                   (Section III-C): clear on the first k block, accumulate,
//                   send the result after the last;
//   warps 2-17      epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (the
//                   tile rows it owns) for a quarter of the tile's columns
//                   (at least 32; sixteen warps keep enough C loads in
//                   flight for the HBM-bound shapes with beta != 0),
//                   applies 2^(e_i + f_j), alpha and beta once and stores
//                   column-major C with one 128-byte store per warp and
//                   column (Section III-D: each core owns whole column
//                   blocks of the result so that stores stay contiguous).
// Every wait is bounded: on expiry the kernel records GBGEMM_ERR_DEVICE_TIMEOUT,
// raises a CTA-wide abort flag, drains its own copies and MMAs, frees TMEM
// and returns.
#pragma once

#include "split_device.cuh"

namespace gbg {
namespace {

constexpr int kStages = 4;                         // ring depth of the general (BN <= 256) kernel
constexpr int kMaxBN = 256;
constexpr int kEpiWarps = 16;                      // four per TMEM lane quadrant, each a quarter of the columns
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue warps
constexpr uint64_t kTimeoutNs = 2000000000ull;
// The final drain waits (the producer's copies landing, the MMAs finishing
// before TMEM is freed) take their own, longer bound, whatever limit the
// caller gave the work waits: the CTA must not exit with its own copies
// still in flight.
constexpr uint64_t kDrainTimeoutNs = 4000000000ull;
// Shared memory of a kernel instance: STAGES ring slots of one A block and
// MAXBN B rows, barriers, 1024-byte alignment.  With tiles of at most 128
// columns the same memory holds a six-slot ring (more copies in flight for
// the latency-bound grouped batches).
template <int STAGES, int MAXBN>
constexpr int gemm_smem_bytes() { return STAGES * (kBlockBytes + MAXBN * 128) + 1024 + 256; }
constexpr int kGemmSmemBytes = gemm_smem_bytes<kStages, kMaxBN>();
constexpr int kNarrowStages = 6;                   // ring depth of the BN <= 128 instance
constexpr int kNarrowBN = 128;

// Everything one tile needs.
struct TileJob {
  const uint8_t* a_src;     // A panel block of this tile row, k chunk 0
  const uint8_t* b_src;     // first B panel row of this tile column, k chunk 0
  size_t a_kstride;         // bytes between k chunks of the A panel
  size_t b_kstride;         // bytes between k chunks of the B panel
  int nkc;                  // k chunks
  int bn;                   // tile width: 64, 128 or 256
  int parts;                // 1: [hi | lo] panels, 3 products; 2: also compact lo3 panels, 6 products
  int64_t a_part, b_part;   // byte offsets from the [hi | mid] panels to the compact lo3 panels
  int64_t m0, n0;           // tile origin in C
  int64_t m, n;             // problem extents
  const uint32_t* amaxA;
  const uint32_t* amaxB;
  float* C;
  int64_t ldc;
  float alpha, beta;
  // split-K: when set, the epilogue stores the raw 128 x bn accumulator here
  // (element (row, col) at partial[col * 128 + row]) and a reduction kernel
  // finishes C
  float* partial;
};

// B rows [r0, r0 + bn) of a panel start inside 128-row block r0/128 at row
// r0 % 128; the 64-row case uses half a block.
__device__ __forceinline__ const uint8_t* panel_rows(const uint8_t* panel, int64_t r0) {
  return panel + (size_t)(r0 >> 7) * kBlockBytes + (size_t)(r0 & 127) * 128;
}

// One problem, or a strided batch of equal problems, tiles of 128 x BN in
// groups of `raster` tile rows; problem z has its panels at panelA/B + z*ps,
// its row maxima at amaxA/B + z*as and its result at C + z*cs.
struct SingleSched {
  const uint8_t* panelA; const uint8_t* panelB;
  const uint32_t* amaxA; const uint32_t* amaxB;
  int64_t m, n;
  float alpha, beta;
  float* C; int64_t ldc;
  int tiles_m, tiles_n, nkc, raster, bn, parts;
  int64_t rbA, rbB;
  int64_t a_part, b_part;
  int batch;
  int64_t ps, as, cs;
  // split-K (batch 1, two-part panels): item = (tile, slice), slice s covering
  // k chunks [s * slice_chunks, min(nkc, (s + 1) * slice_chunks)); partials
  // of slice s, tile (tm, tn) at partial + ((s * tiles_m + tm) * tiles_n + tn) * 128 * bn
  int splitk, slice_chunks;
  float* partial;
  __device__ __forceinline__ int num_items() const { return tiles_m * tiles_n * batch * splitk; }
  __device__ __forceinline__ TileJob job(int t) const {
    const int per = tiles_m * tiles_n;
    const int sl = t % splitk;
    t /= splitk;
    const int z = t / per;
    int tm, tn;
    tile_coords(t - z * per, tiles_m, tiles_n, raster, tm, tn);
    const int kc0 = sl * slice_chunks;
    TileJob j;
    j.a_kstride = (size_t)rbA * kBlockBytes;
    j.b_kstride = (size_t)rbB * kBlockBytes;
    j.a_src = panelA + (size_t)z * ps + (size_t)tm * kBlockBytes + (size_t)kc0 * j.a_kstride;
    j.b_src = panel_rows(panelB + (size_t)z * ps, (int64_t)tn * bn) + (size_t)kc0 * j.b_kstride;
    j.nkc = (nkc - kc0 < slice_chunks) ? nkc - kc0 : slice_chunks;
    j.bn = bn;
    j.partial = splitk > 1 ? partial + ((size_t)(sl * tiles_m + tm) * tiles_n + tn) * 128 * bn : nullptr;
    j.parts = parts; j.a_part = a_part; j.b_part = b_part;
    j.m0 = (int64_t)tm * 128; j.n0 = (int64_t)tn * bn;
    j.m = m; j.n = n;
    j.amaxA = amaxA + (size_t)z * as; j.amaxB = amaxB + (size_t)z * as;
    j.C = C + (size_t)z * cs; j.ldc = ldc; j.alpha = alpha; j.beta = beta;
    return j;
  }
};

// Device descriptor of one problem of a grouped batch on the split path.
struct GroupDev {
  const uint8_t* panelA; const uint8_t* panelB;
  const uint32_t* amaxA; const uint32_t* amaxB;
  float* C; int64_t ldc;
  int64_t m, n;
  int nkc, bn;
  int64_t rowsA, rowsB;     // panel rows per k chunk
  float alpha, beta;
  int parts, pad_;
  int64_t a_part, b_part;   // byte offsets to the compact lo3 panels (parts == 2)
};

// Many problems: item t = (group, tile row, tile column), items sorted by
// decreasing cost so that a static round robin balances the CTAs.
struct GroupedSched {
  const int4* items;
  const GroupDev* groups;
  int n_items;
  __device__ __forceinline__ int num_items() const { return n_items; }
  __device__ __forceinline__ TileJob job(int t) const {
    const int4 it = items[t];
    const GroupDev g = groups[it.x];
    TileJob j;
    j.a_src = g.panelA + (size_t)it.y * kBlockBytes;
    j.b_src = panel_rows(g.panelB, (int64_t)it.z * g.bn);
    j.a_kstride = (size_t)g.rowsA * 128;
    j.b_kstride = (size_t)g.rowsB * 128;
    j.nkc = g.nkc; j.bn = g.bn;
    j.parts = g.parts; j.a_part = g.a_part; j.b_part = g.b_part;
    j.m0 = (int64_t)it.y * 128; j.n0 = (int64_t)it.z * g.bn;
    j.m = g.m; j.n = g.n;
    j.amaxA = g.amaxA; j.amaxB = g.amaxB;
    j.C = g.C; j.ldc = g.ldc; j.alpha = g.alpha; j.beta = g.beta;
    j.partial = nullptr;
    return j;
  }
};

template <class Sched, int STAGES = kStages, int MAXBN = kMaxBN>
__global__ void __launch_bounds__(kGemmThreads, 1)
split_gemm_kernel(const Sched S, int* status, uint64_t timeout_ns) {
  constexpr uint32_t A_BYTES = kBlockBytes;        // 128 rows x 128 B
  constexpr uint32_t B_STAGE = MAXBN * 128;        // room for MAXBN rows x 128 B
  constexpr uint32_t kTmemCols = 2 * MAXBN;        // two accumulator buffers
  constexpr int kStages = STAGES;
  constexpr int kMaxBN = MAXBN;

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  uint8_t* const base_ptr = smem_raw + (base - raw_addr);
  const uint32_t sA = base;                                   // kStages x A_BYTES
  const uint32_t sB = base + kStages * A_BYTES;               // kStages x B_STAGE
  const uint32_t bar0 = sB + kStages * B_STAGE;               // barriers
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * kStages + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 4);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(base_ptr + (bar0 - base) + 8 * (2 * kStages + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_items = S.num_items();

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
                 ::"r"(smem_u32(tmem_holder)), "r"(kTmemCols) : "memory");
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
      for (int t = blockIdx.x; t < num_items && ok; t += gridDim.x) {
        const TileJob J = S.job(t);
        const uint32_t b_bytes = (uint32_t)J.bn * 128u;
        // one ring slot per k chunk, and with three parts one more per pair
        // of chunks (the compact [lo3 | lo3] block, loaded with the even chunk)
        for (int kc = 0; kc < J.nkc && ok; ++kc) {
          const int nparts = (J.parts == 2 && (kc & 1) == 0) ? 2 : 1;
          for (int part = 0; part < nparts; ++part) {
            if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, timeout_ns)) {
              raise_status(status, abort_flag);
              ok = false;
              break;
            }
            const uint8_t* a = part ? J.a_src + J.a_part + (size_t)(kc >> 1) * J.a_kstride
                                    : J.a_src + (size_t)kc * J.a_kstride;
            const uint8_t* b = part ? J.b_src + J.b_part + (size_t)(kc >> 1) * J.b_kstride
                                    : J.b_src + (size_t)kc * J.b_kstride;
            mbar_arrive_expect_tx(full_bar(stage), A_BYTES + b_bytes);
            bulk_copy_g2s(sA + stage * A_BYTES, a, A_BYTES, full_bar(stage));
            bulk_copy_g2s(sB + stage * B_STAGE, b, b_bytes, full_bar(stage));
            issued[stage] = true;
            issued_phase[stage] = (int)phase;
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
          }
        }
      }
      // Let every copy this thread started land before the CTA can exit.
      volatile int never = 0;
      for (int s = 0; s < kStages; ++s)
        if (issued[s]) (void)mbar_wait(full_bar(s), (uint32_t)issued_phase[s], &never, kDrainTimeoutNs);
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
      for (int t = blockIdx.x; t < num_items && ok; t += gridDim.x) {
        const TileJob J = S.job(t);
        const uint32_t idesc = make_idesc_bf16(128, J.bn);
        if (!mbar_wait(acce_bar(abuf), aphase ^ 1u, abort_flag, timeout_ns)) {
          raise_status(status, abort_flag);
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * kMaxBN);
        int s1 = 0;  // with three parts: the slot of the current [lo3 | lo3] block
        for (int kc = 0; kc < J.nkc; ++kc) {
          // the chunk's slot s0 holds [hi | lo] (or [hi | mid]); with three parts
          // an even chunk also brings the pair's [lo3 | lo3] slot
          const int s0 = stage;
          const uint32_t ph0 = phase;
          if (!mbar_wait(full_bar(s0), ph0, abort_flag, timeout_ns)) {
            raise_status(status, abort_flag);
            ok = false;
            break;
          }
          if (J.parts == 2 && (kc & 1) == 0) {
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
            s1 = stage;
            if (!mbar_wait(full_bar(s1), phase, abort_flag, timeout_ns)) {
              raise_status(status, abort_flag);
              ok = false;
              break;
            }
          }
          tc_fence_after();
          const uint32_t a_addr = sA + s0 * A_BYTES;
          const uint32_t b_addr = sB + s0 * B_STAGE;
          const uint32_t a3_addr = sA + s1 * A_BYTES + 64u * (uint32_t)(kc & 1);
          const uint32_t b3_addr = sB + s1 * B_STAGE + 64u * (uint32_t)(kc & 1);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t ah = make_desc_sw128(a_addr + 32u * kk);
            const uint64_t al = make_desc_sw128(a_addr + 64u + 32u * kk);
            const uint64_t bh = make_desc_sw128(b_addr + 32u * kk);
            const uint64_t bl = make_desc_sw128(b_addr + 64u + 32u * kk);
            mma_bf16(d_tmem, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d_tmem, ah, bl, idesc, 1u);
            mma_bf16(d_tmem, al, bh, idesc, 1u);
            if (J.parts == 2) {
              // with three parts: hi*lo3 + mid*mid + lo3*hi (al, bl above are mid)
              const uint64_t a3 = make_desc_sw128(a3_addr + 32u * kk);
              const uint64_t b3 = make_desc_sw128(b3_addr + 32u * kk);
              mma_bf16(d_tmem, ah, b3, idesc, 1u);
              mma_bf16(d_tmem, al, bl, idesc, 1u);
              mma_bf16(d_tmem, a3, bh, idesc, 1u);
            }
          }
          mma_commit(empty_bar(s0));  // frees the slot once these MMAs have read it
          if (J.parts == 2 && ((kc & 1) == 1 || kc == J.nkc - 1)) mma_commit(empty_bar(s1));
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(accf_bar(abuf));      // the tile's accumulator is complete
        if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
      }
      // Wait until every MMA issued here has finished before TMEM is released.
      mma_commit(drain_bar);
      volatile int never = 0;
      if (!mbar_wait(drain_bar, 0u, &never, kDrainTimeoutNs)) raise_status(status, abort_flag);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;  // column part: 0 .. kEpiWarps / 4 - 1
    int abuf = 0;
    uint32_t aphase = 0;
    for (int t = blockIdx.x; t < num_items; t += gridDim.x) {
      const TileJob J = S.job(t);
      int ok = 1;
      if (lane == 0) ok = mbar_wait_hint(accf_bar(abuf), aphase, abort_flag, timeout_ns, 2000u) ? 1 : 0;
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_status(status, abort_flag);
        break;
      }
      tc_fence_after();
      const int64_t i = J.m0 + q * 32 + lane;
      const bool row_ok = i < J.m;
      const int ea = row_ok ? scale_exp_from_bits(J.amaxA[i]) : 0;
      const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * kMaxBN);
      float* const crow = J.C + i;
      const int cols = (J.bn / (kEpiWarps / 4)) > 32 ? J.bn / (kEpiWarps / 4) : 32;
      const int c_begin = part * cols, c_end = (c_begin + cols < J.bn) ? c_begin + cols : J.bn;
      if (J.partial) {
        // split-K slice: the raw accumulator, whole tile, 32 consecutive rows per warp store
        float* pp = J.partial + q * 32 + lane;
        for (int c0 = c_begin; c0 < c_end; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(taddr + (uint32_t)c0, r);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) __stcg(pp + (size_t)(c0 + jj) * 128, __uint_as_float(r[jj]));
        }
      }
      for (int c0 = c_begin; c0 < c_end && !J.partial; c0 += 32) {
        if (J.n0 + c0 >= J.n) break;  // warp-uniform
        const int jmax = (J.n - (J.n0 + c0) < 32) ? (int)(J.n - (J.n0 + c0)) : 32;
        float* cp = crow + (J.n0 + c0) * J.ldc;
        // All loads of the chunk are issued before any result is formed, so
        // the 32 column reads of C overlap instead of queueing one by one.
        float cv[32];
        if (J.beta != 0.f) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) cv[jj] = (row_ok && jj < jmax) ? __ldcs(cp + jj * J.ldc) : 0.f;
        }
        const int64_t jl = J.n0 + c0 + lane;
        const int eb_l = (jl < J.n) ? scale_exp_from_bits(J.amaxB[jl]) : 0;
        uint32_t r[32];
        tmem_ld32(taddr + (uint32_t)c0, r);
        // Every lane runs every shuffle; only the stores are predicated.
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int s = ea + __shfl_sync(0xFFFFFFFFu, eb_l, jj);
          const float acc = __uint_as_float(r[jj]);
          // acc * 2^s: one multiply when 2^s is a normal float, else scalbnf.
          const float v = (s >= -126 && s <= 127) ? acc * __int_as_float((s + 127) << 23) : scalbnf(acc, s);
          const float out = (J.beta != 0.f) ? fmaf(J.alpha, v, J.beta * cv[jj]) : J.alpha * v;
          if (row_ok && jj < jmax) __stcs(cp + jj * J.ldc, out);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
  }
}

// The shared-memory opt-in is a per-device function attribute: set it once
// for every device a kernel instance is launched on.
template <class Sched, int STAGES = kStages, int MAXBN = kMaxBN>
cudaError_t ensure_gemm_smem_attr() {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(split_gemm_kernel<Sched, STAGES, MAXBN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             gemm_smem_bytes<STAGES, MAXBN>());
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace gbg
