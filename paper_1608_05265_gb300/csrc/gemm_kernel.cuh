// The persistent split-BF16 tcgen05 GEMM kernel and the packing kernel
// that runs ahead of it, templated on the scheduler: SingleSched walks the
// tiles of one problem (or a strided batch) in a rasterised order,
// GroupedSched walks the tiles of many problems, problem after problem.  The
// per-tile job carries everything a role needs, including the tile width BN
// (64, 128 or 256) as a run-time value: the MMA instruction descriptor, the
// B copy size and the epilogue width all follow it, and shared memory and
// TMEM are sized for MAXBN.
//
// Packing (BLIS packing, Section III-A): one CTA of 256 threads per packing
// task (4 x 32 k of one 128-row band of one operand), several per SM, the
// operand read straight into registers; each task counts itself on its
// band's counter, and the task that completes a band re-packs the band's
// badly scaled rows.  The GEMM launch follows on the same stream.
//
// GEMM roles (one CTA per SM, 608 threads):
//   warp 0, lane 0  producer: takes the next tile from a device-wide counter
//                   (dynamic scheduling, so the CTAs that run finish the
//                   work however many are resident), hands its index to the
//                   other roles through a four-slot queue in shared memory,
//                   and streams one bulk async copy of the 128-row A block
//                   and one of the BN B rows per 32-deep k chunk into the
//                   stage ring ("full" mbarriers);
//   warp 1          owns TMEM (two 128 x MAXBN FP32 accumulators); lane 0
//                   issues the MMAs (hi*hi, hi*lo, lo*hi for both 16-deep
//                   halves of a chunk, six products with the three-part
//                   split), commits each stage back to its "empty" barrier
//                   and each finished tile to an "accumulator full" barrier
//                   -- the paper's Accumulator (Section III-C): clear on the
//                   first k block, accumulate, send the result after the
//                   last;
//   warps 2-17      epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (the
//                   tile rows it owns) for a quarter of the tile's columns,
//                   applies 2^(e_i + f_j), alpha and beta once and stores
//                   column-major C with one 128-byte store per warp and
//                   column (Section III-D: each core owns whole column
//                   blocks of the result so that stores stay contiguous);
//   warp 18         with beta != 0 and k <= 512, asks L2 for each tile's C
//                   columns as soon as the tile is handed out, so that the
//                   epilogue's reads of C find them there.
// Every wait is bounded: on expiry the kernel records GBGEMM_ERR_DEVICE_TIMEOUT,
// raises a CTA-wide abort flag, drains its own copies and MMAs, frees TMEM
// and returns.  Waiting threads sleep (mbarrier try_wait with a suspend
// hint) instead of spinning.
#pragma once

#include "split_device.cuh"

namespace gbg {
namespace {

constexpr int kStages = 4;                         // ring depth of the general (BN <= 256) kernel
constexpr int kMaxBN = 256;
constexpr int kNarrowStages = 6;                   // ring depth of the BN <= 128 instance
constexpr int kNarrowBN = 128;
constexpr int kPairStages = 6;                     // ring depth of the pair-tile instance (half the B rows per CTA)
constexpr int kEpiWarps = 16;
constexpr int kCpfWarp = 2 + kEpiWarps;            // the C prefetch warp
constexpr int kGemmThreads = 32 * (kCpfWarp + 1);  // 19 warps, charged as 20: 96 registers per thread
constexpr int kTileQ = 4;                          // tile-index queue between the roles
constexpr int kPackChunks = 4;                     // k chunks per packing task
constexpr uint64_t kTimeoutNs = 2000000000ull;
// Suspend-time hint of the mbarrier waits: a waiting thread sleeps until the
// phase completes (or this long) instead of spinning.
constexpr uint32_t kHintNs = 20000u;
// The final drain waits (the producer's copies landing, the MMAs finishing
// before TMEM is freed) take their own, longer bound, whatever limit the
// caller gave the work waits: the CTA must not exit with its own copies
// still in flight.
constexpr uint64_t kDrainTimeoutNs = 4000000000ull;
// Shared memory of a kernel instance: STAGES ring slots of one A block and
// MAXBN B rows (MAXBN / 2 for pair tiles, whose CTAs hold half the B rows
// each), barriers and the tile queue, 1024-byte alignment.  With tiles of at
// most 128 columns the same memory holds a six-slot ring, and so it does for
// pair tiles.
template <int STAGES, int MAXBN, bool PAIR = false>
constexpr int gemm_smem_bytes() { return STAGES * (kBlockBytes + (PAIR ? MAXBN / 2 : MAXBN) * 128) + 1024 + 256; }
constexpr int kGemmSmemBytes = gemm_smem_bytes<kStages, kMaxBN>();

// The dependent launch of a kernel started with programmatic stream
// serialisation may begin before this grid finishes; it waits (below) for
// the grid's completion before it reads what the grid wrote.
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Wait until the grid this one depends on has completed and its memory is
// visible (returns at once without such a dependency).
__device__ __forceinline__ void wait_prerequisite_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Per-launch control words; zeroed before every launch together with the
// band counters and the row maxima.
struct WorkCtl {
  int tile_next;   // next work item
  int pad[63];
};
static_assert(sizeof(WorkCtl) == kSplitCtlBytes, "control block size");

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

// One packing task: chunks kc0 .. kc0 + chunks - 1 (those below nkc) of the
// 128-row band rb of one operand.
struct PackJob {
  const float* X;
  int64_t ld;
  uint32_t* amax;           // maxima of the operand's K-vectors (row 0)
  uint8_t* panel;           // the operand's panel (row 0, k chunk 0)
  uint8_t* panel2;          // its compact lo3 panel (three parts), else NULL
  int64_t rows, k;          // K-vectors and their length
  int64_t rows_alloc;       // panel rows per k chunk
  int64_t rb;
  int kc0, nkc;
  int chunks;               // k chunks per task of this operand (1, 2 or kPackChunks)
  int kcontig;
  int band, band_tasks;     // band counter and the tasks that fill it
};

// B rows [r0, r0 + bn) of a panel start inside 128-row block r0/128 at row
// r0 % 128; the 64-row case uses half a block.
__device__ __forceinline__ const uint8_t* panel_rows(const uint8_t* panel, int64_t r0) {
  return panel + (size_t)(r0 >> 7) * kBlockBytes + (size_t)(r0 & 127) * 128;
}

// Packing order of the bands of one problem: each band in the order of the
// first tile that reads it.  Tiles go in groups of `gm` tile rows (all
// tile columns of a group before the next group), so the order is the B
// bands of tile column 0, the A bands of the first group, the other B bands,
// then the remaining A bands.  Returns the band as (is_a, index).
__device__ __forceinline__ void band_at(int pos, int ra, int rb, int gm, int nb0, bool& is_a, int& idx) {
  if (pos < nb0) { is_a = false; idx = pos; return; }
  if (pos < nb0 + gm) { is_a = true; idx = pos - nb0; return; }
  if (pos < rb + gm) { is_a = false; idx = pos - gm; return; }
  is_a = true; idx = pos - rb;
}

// One problem, or a strided batch of equal problems, tiles of 128 x BN in
// groups of `raster` tile rows; problem z reads its operands at A + z*sa and
// B + z*sb, has its panels at panelA/B + z*ps, its row maxima at amaxA/B +
// z*as and its result at C + z*cs.  Band counters: problem z's A band a at
// band_cnt[z*(ra+rb) + a], its B band b at band_cnt[z*(ra+rb) + ra + b].
struct SingleSched {
  WorkCtl* ctl;
  int* band_cnt;
  const float* A; const float* B;
  int64_t lda, ldb, sa, sb;
  int ta, tb;
  const uint8_t* panelA; const uint8_t* panelB;
  uint32_t* amaxA; uint32_t* amaxB;
  int64_t m, n, k;
  float alpha, beta;
  float* C; int64_t ldc;
  int tiles_m, tiles_n, nkc, raster, bn, parts;
  int64_t rbA, rbB;          // panel row blocks (padded to even)
  int ra, rb;                // bands packed (ceil(m/128), ceil(n/128))
  int pchunks;               // k chunks per packing task
  int ngroups;               // packing tasks per band (ceil(nkc / pchunks))
  int64_t a_part, b_part;
  int batch;
  int64_t ps, as, cs;
  // split-K (batch 1, two-part panels): item = (tile, slice), slice s covering
  // k chunks [s * slice_chunks, min(nkc, (s + 1) * slice_chunks)); partials
  // of slice s, tile (tm, tn) at partial + ((s * tiles_m + tm) * tiles_n + tn) * 128 * bn
  int splitk, slice_chunks;
  float* partial;
  // pair tiles (clusters of two CTAs, bn = 256): item t is a 256 x 256 tile
  // (with split-K: one k slice of it), tile rows 2 tm2 and 2 tm2 + 1 of pair
  // row tm2
  int pair;
  __device__ __forceinline__ int num_items() const {
    return (pair ? ((tiles_m + 1) >> 1) : tiles_m) * tiles_n * batch * splitk;
  }
  __device__ __forceinline__ TileJob job(int t) const {
    const int per = tiles_m * tiles_n;
    const int sl = t % splitk;
    t /= splitk;
    const int z = t / per;
    int tm, tn;
    tile_coords(t - z * per, tiles_m, tiles_n, raster, tm, tn);
    return tile_job(z, tm, tn, sl, (int64_t)tn * bn);
  }
  // The half of pair item t that CTA `rank` of the pair computes: tile row
  // 2 tm2 + rank (the A panel has an even number of row blocks, so the odd
  // row of a last, half-empty pair reads the panel's padding block, which is
  // never written; its rows lie past m and its epilogue stores nothing),
  // B rows [n0 + 128 rank, n0 + 128 rank + 128) for its share of the B
  // operand, and the item's k slice.  Pair rows go in groups of
  // raster / 2, the same rows of C as the single-CTA groups of `raster` tile
  // rows.
  __device__ __forceinline__ TileJob job_pair(int t, int rank) const {
    const int tiles_m2 = (tiles_m + 1) >> 1;
    const int per = tiles_m2 * tiles_n;
    const int sl = t % splitk;
    t /= splitk;
    const int z = t / per;
    int tm2, tn;
    tile_coords(t - z * per, tiles_m2, tiles_n, raster > 1 ? raster >> 1 : 1, tm2, tn);
    return tile_job(z, 2 * tm2 + rank, tn, sl, (int64_t)tn * bn + 128 * rank);
  }
  __device__ __forceinline__ TileJob tile_job(int z, int tm, int tn, int sl, int64_t b_row0) const {
    const int kc0 = sl * slice_chunks;
    TileJob j;
    j.a_kstride = (size_t)rbA * kBlockBytes;
    j.b_kstride = (size_t)rbB * kBlockBytes;
    j.a_src = panelA + (size_t)z * ps + (size_t)tm * kBlockBytes + (size_t)kc0 * j.a_kstride;
    j.b_src = panel_rows(panelB + (size_t)z * ps, b_row0) + (size_t)kc0 * j.b_kstride;
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
  __device__ __forceinline__ int num_pack_tasks() const { return batch * (ra + rb) * ngroups; }
  __device__ __forceinline__ PackJob pack_job(int i) const {
    const int per = (ra + rb) * ngroups;
    const int z = i / per;
    const int r = i - z * per;
    const int pos = r / ngroups, g = r - pos * ngroups;
    const int gm = min(raster, tiles_m);
    const int nb0 = min(rb, max(1, bn >> 7));
    bool is_a;
    int idx;
    band_at(pos, ra, rb, gm, nb0, is_a, idx);
    PackJob P;
    P.X = is_a ? A + (size_t)z * sa : B + (size_t)z * sb;
    P.ld = is_a ? lda : ldb;
    P.kcontig = is_a ? (ta == 1) : (tb == 0);
    P.rows = is_a ? m : n;
    P.k = k;
    P.amax = (is_a ? amaxA : amaxB) + (size_t)z * as;
    P.panel = const_cast<uint8_t*>(is_a ? panelA : panelB) + (size_t)z * ps;
    P.panel2 = parts == 2 ? P.panel + (is_a ? a_part : b_part) : nullptr;
    P.rows_alloc = (is_a ? rbA : rbB) * 128;
    P.rb = idx;
    P.kc0 = g * pchunks;
    P.chunks = pchunks;
    P.nkc = nkc;
    P.band = z * (ra + rb) + (is_a ? 0 : ra) + idx;
    P.band_tasks = ngroups;
    return P;
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

// One 128-row band of one operand of a grouped problem, as the packers see it.
struct PackBand {
  const float* X;
  int64_t ld;
  uint32_t* amax;
  uint8_t* panel;
  uint8_t* panel2;
  int64_t rows, k, rows_alloc;
  int rb, nkc;
  int kcontig, ngroups;
  int first_task, cnt;      // the band's first packing task and its counter
};

// Many problems: item t = (group, tile row, tile column), the items of one
// problem together, problems in decreasing cost per tile, so that the cheap
// tiles come last and fill the gaps.
struct GroupedSched {
  WorkCtl* ctl;
  int* band_cnt;
  const int4* items;
  const GroupDev* groups;
  const PackBand* bands;
  const int* task_band;
  int n_items, n_tasks;
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
  __device__ __forceinline__ int num_pack_tasks() const { return n_tasks; }
  __device__ __forceinline__ PackJob pack_job(int i) const {
    const int b = task_band[i];
    const PackBand B = bands[b];
    PackJob P;
    P.X = B.X; P.ld = B.ld; P.amax = B.amax; P.panel = B.panel; P.panel2 = B.panel2;
    P.rows = B.rows; P.k = B.k; P.rows_alloc = B.rows_alloc; P.rb = B.rb;
    P.kc0 = (i - B.first_task) * kPackChunks;
    P.chunks = kPackChunks;
    P.nkc = B.nkc;
    P.kcontig = B.kcontig;
    P.band = B.cnt;
    P.band_tasks = B.ngroups;
    return P;
  }
};

// Item (rr, cc) of a chunk in a packing CTA: row rr (0..127) of the band and
// 8-wide k piece cc (0..3); item idx = tid + 256 * it, two per thread.
// KCONTIG (element (r,p) at X[r*ld + p]): four consecutive items per row, so
// a warp reads eight 128-byte row pieces.  !KCONTIG (X[r + p*ld]): 32
// consecutive rows per warp and one piece per warp, so every load
// instruction reads 128 contiguous bytes.
template <bool KCONTIG>
__device__ __forceinline__ void item_of(int tid, int it, int& rr, int& cc) {
  const int idx = tid + 256 * it;
  if (KCONTIG) {
    rr = idx >> 2;
    cc = idx & 3;
  } else {
    const int w = idx >> 5;
    cc = w & 3;
    rr = (w >> 2) * 32 + (idx & 31);
  }
}

__device__ __forceinline__ int task_chunks(const PackJob& P) {
  return (P.nkc - P.kc0 < P.chunks) ? P.nkc - P.kc0 : P.chunks;
}

// ---------------------------------------------------------------------------
// Packing ahead of the GEMM: one CTA of 256 threads per packing task of the
// scheduler, the operand read straight into registers (all loads of two
// chunks in flight before any is split), several CTAs per SM.  Counts the
// task on its band's counter; the task that completes a band re-packs the
// band's badly scaled rows.
// ---------------------------------------------------------------------------
template <bool KCONTIG>
__device__ __forceinline__ void load8(const PackJob& P, int64_t r, int64_t p, bool vec, float (&x)[8]) {
  if (KCONTIG) {
    if (r < P.rows && vec && p + 8 <= P.k) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(P.X + r * P.ld + p));
      const float4 b = __ldg(reinterpret_cast<const float4*>(P.X + r * P.ld + p + 4));
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = (r < P.rows && p + q < P.k) ? __ldg(P.X + r * P.ld + p + q) : 0.f;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = (r < P.rows && p + q < P.k) ? __ldg(P.X + r + (p + q) * P.ld) : 0.f;
  }
}

template <bool KCONTIG>
__device__ __forceinline__ void pack_task_regs(const PackJob& P, uint32_t* smax) {
  const int tid = threadIdx.x;
  const int64_t r0 = P.rb * 128;
  const bool vec = ((P.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.X) & 15) == 0);
  const int nch = task_chunks(P);
  if (tid < 128) smax[tid] = 0u;
  uint32_t mxr[2] = {0u, 0u};
  for (int c0 = 0; c0 < nch; c0 += 2) {
    float x[2][2][8];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        int rr, cc;
        item_of<KCONTIG>(tid, it, rr, cc);
        if (c0 + c < nch) load8<KCONTIG>(P, r0 + rr, (int64_t)(P.kc0 + c0 + c) * 32 + cc * 8, vec, x[c][it]);
      }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (c0 + c >= nch) break;
      const int64_t kc = P.kc0 + c0 + c;
      uint8_t* blk = P.panel + ((size_t)kc * P.rows_alloc + r0) * 128;
      uint8_t* blk2 = P.panel2 ? P.panel2 + ((size_t)(kc >> 1) * P.rows_alloc + r0) * 128 : nullptr;
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        int rr, cc;
        item_of<KCONTIG>(tid, it, rr, cc);
#pragma unroll
        for (int q = 0; q < 8; ++q) mxr[it] = max(mxr[it], __float_as_uint(x[c][it][q]) & 0x7FFFFFFFu);
        if (r0 + rr < P.rows_alloc) {
          if (blk2) store_split8_3(blk, blk2, (int)(kc & 1), rr, cc, x[c][it]);
          else store_split8(blk, rr, cc, x[c][it]);
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    int rr, cc;
    item_of<KCONTIG>(tid, it, rr, cc);
    if (mxr[it] != 0u) atomicMax(&smax[rr], mxr[it]);
  }
  __syncthreads();
  if (tid < 128 && r0 + tid < P.rows && smax[tid] != 0u) atomicMax(&P.amax[r0 + tid], smax[tid]);
}

// Four CTAs per SM (64 registers, no spills): 3.6% faster than the 80-register
// build on the uneven grouped batch, 5% at 1024^3.
template <class Sched>
__global__ void __launch_bounds__(256, 4) pack_tasks_kernel(const Sched S) {
  __shared__ uint32_t smax[128];
  __shared__ int finisher;
  launch_dependents();  // the GEMM may launch and set up while the packing runs
  const PackJob P = S.pack_job((int)blockIdx.x);
  if (P.kcontig) pack_task_regs<true>(P, smax);
  else pack_task_regs<false>(P, smax);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int old = atomicAdd(S.band_cnt + P.band, 1);
    __threadfence();  // the other tasks' maxima are visible from here on
    finisher = (old == P.band_tasks - 1) ? 1 : 0;
  }
  __syncthreads();
  if (finisher) {
    __threadfence();
    rescale_block(P.rows, P.k, P.X, P.ld, P.kcontig != 0, P.amax, P.panel, P.panel2, P.rows_alloc, P.nkc, P.rb,
                  reinterpret_cast<int*>(smax));
  }
}

// One CTA per SM.  Registers are handed out to whole groups of four warps,
// so the 19 warps are charged as 20: 96 registers per thread.
//
// PAIR: launched in clusters of two CTAs on two SMs, each pair computing
// 256 x 256 tiles (SingleSched pair items) with tcgen05 MMAs of
// cta_group::2.  Each CTA loads its own 128-row A block and half of the
// tile's 256 B rows, so per SM a k chunk brings 32 KiB instead of 48 KiB and
// the tensor cores read half as many B bytes from shared memory.  The even
// CTA (rank 0) issues the MMAs for both; the odd CTA's warp 1 relays each
// of its landed stages to rank 0's "full" barrier (which then counts two
// arrivals), its epilogue warps release the accumulator on rank 0's
// "accumulator empty" barrier (32 arrivals), and rank 0's commits arrive on
// both CTAs' "empty" and "accumulator full" barriers.  Pairs take items in a
// fixed order (cluster c: items c, c + clusters, ...), so both CTAs of a
// pair walk the same tiles without exchanging indices.
template <class Sched, int STAGES = kStages, int MAXBN = kMaxBN, bool PAIR = false, bool THREE = false>
__global__ void __launch_bounds__(kGemmThreads, 1)
split_gemm_kernel(const Sched S, int* status, uint64_t timeout_ns) {
  constexpr uint32_t A_BYTES = kBlockBytes;        // 128 rows x 128 B
  constexpr uint32_t B_STAGE = (PAIR ? MAXBN / 2 : MAXBN) * 128;  // room for the B rows of a stage
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
  auto tqf_bar = [&](int s) { return bar0 + 8u * (2 * kStages + 5 + s); };
  auto tqe_bar = [&](int s) { return bar0 + 8u * (2 * kStages + 5 + kTileQ + s); };
  uint8_t* const tail = base_ptr + (bar0 - base) + 8 * (2 * kStages + 5 + 2 * kTileQ);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tail);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tail + 4);
  volatile int* tile_q = reinterpret_cast<volatile int*>(tail + 16);          // kTileQ ints

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_items = S.num_items();
  // the CTA's rank in its pair (0: issues the MMAs), the pair's index and count
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;
  const int pair_id = PAIR ? (int)cluster_id_x() : 0;
  const int num_pairs = PAIR ? (int)num_clusters_x() : 1;
  auto job_of = [&](int t) -> TileJob {
    if constexpr (PAIR) return S.job_pair(t, (int)crank);
    else return S.job(t);
  };
  auto wait_bar = [&](uint32_t bar, uint32_t parity) -> bool {
    return mbar_wait_hint(bar, parity, abort_flag, timeout_ns, kHintNs);
  };

  if (threadIdx.x == 0) {
    const uint32_t full_count = (PAIR && crank == 0u) ? 2u : 1u;  // rank 0: its own copies + the relay
    for (int s = 0; s < kStages; ++s) { mbar_init(full_bar(s), full_count); mbar_init(empty_bar(s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(accf_bar(b), 1); mbar_init(acce_bar(b), (PAIR ? 2 : 1) * kEpiWarps); }
    mbar_init(drain_bar, 1);
    for (int s = 0; s < kTileQ; ++s) { mbar_init(tqf_bar(s), 1); mbar_init(tqe_bar(s), 2 + kEpiWarps); }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      // one warp of each CTA of the pair allocates, together, the same columns in both
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                   ::"r"(smem_u32(tmem_holder)), "r"(kTmemCols) : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                   ::"r"(smem_u32(tmem_holder)), "r"(kTmemCols) : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair's barriers are initialised on both sides before either side uses the other's
  if constexpr (PAIR) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const int first_item = PAIR ? pair_id : (int)blockIdx.x;
  if (warp == kCpfWarp && first_item < num_items) {
    // While the packing runs: ask L2 for the C of the tile this CTA most
    // likely takes first (CTA b usually draws item b), for short tiles with
    // beta != 0 as below.  C is not written by the packing; a wrong guess
    // only costs the prefetch.
    const TileJob J = job_of(first_item);
    if (J.beta != 0.f && !J.partial && J.nkc <= 16 && J.m0 < J.m) {
      const int64_t rows = (J.m - J.m0 < 128) ? J.m - J.m0 : 128;
      const int64_t ncols = (J.n - J.n0 < J.bn) ? J.n - J.n0 : J.bn;
      const float* c0 = J.C + J.m0 + J.n0 * J.ldc;
      for (int64_t j = lane; j < ncols; j += 32) {
        const char* col = reinterpret_cast<const char*>(c0 + j * J.ldc);
        for (int64_t off = 0; off < rows * 4; off += 128) prefetch_l2(col + off);
        prefetch_l2(col + rows * 4 - 4);
      }
    }
  }
  // everything above overlaps the packing launch; the panels and maxima it
  // writes are read only from here on
  wait_prerequisite_grid();
  launch_dependents();

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int tq = 0;
      uint32_t tqph = 0;
      int next_item = first_item;
      int issued_phase[kStages];
      bool issued[kStages];
      for (int s = 0; s < kStages; ++s) { issued[s] = false; issued_phase[s] = 0; }
      bool ok = true;
      while (ok) {
        if (!mbar_wait_hint(tqe_bar(tq), tqph ^ 1u, abort_flag, timeout_ns, kHintNs)) {
          raise_status(status, abort_flag);
          break;
        }
        int t;
        if constexpr (PAIR) {
          t = next_item;  // a fixed order, the same in both CTAs of the pair
          next_item += num_pairs;
        } else {
          t = atomicAdd(&S.ctl->tile_next, 1);
        }
        if (t >= num_items || *abort_flag) t = -1;
        tile_q[tq] = t;
        mbar_arrive(tqf_bar(tq));
        if (++tq == kTileQ) { tq = 0; tqph ^= 1u; }
        if (t < 0) break;
        const TileJob J = job_of(t);
        const uint32_t b_bytes = (uint32_t)(PAIR ? J.bn / 2 : J.bn) * 128u;
        // one ring slot per k chunk, and with three parts one more per pair
        // of chunks (the compact [lo3 | lo3] block, loaded with the even chunk)
        for (int kc = 0; kc < J.nkc && ok; ++kc) {
          const int nparts = (J.parts == 2 && (kc & 1) == 0) ? 2 : 1;
          for (int part = 0; part < nparts; ++part) {
            if (!wait_bar(empty_bar(stage), phase ^ 1u)) {
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
      // With pairs, rank 0's MMA commits release this CTA's slots by arriving
      // on its "empty" barriers: wait for the releases of the last fills, so
      // that no such arrival is still on its way when the CTA exits.
      if constexpr (PAIR) {
        for (int i = 0; i < kStages; ++i) {
          if (!wait_bar(empty_bar(stage), phase ^ 1u)) {
            raise_status(status, abort_flag);
            break;
          }
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
      }
    }
    __syncwarp();
  } else if (PAIR && warp == 1 && crank != 0u) {
    // ---------------- relay (odd CTA of a pair) ----------------
    // Tell rank 0's MMA issuer, stage by stage, that this CTA's share of the
    // stage has landed (rank 0's "full" barrier counts this arrival).
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int tq = 0;
      uint32_t tqph = 0;
      bool ok = true;
      while (ok) {
        if (!mbar_wait_hint(tqf_bar(tq), tqph, abort_flag, timeout_ns, kHintNs)) {
          raise_status(status, abort_flag);
          break;
        }
        const int t = tile_q[tq];
        mbar_arrive(tqe_bar(tq));
        if (++tq == kTileQ) { tq = 0; tqph ^= 1u; }
        if (t < 0) break;
        const TileJob J = job_of(t);
        if constexpr (THREE) {
          // every slot in the producer's fill order: one per k chunk and the
          // [lo3 | lo3] slot after each even chunk
          for (int kc = 0; kc < J.nkc && ok; ++kc) {
            const int nparts = (J.parts == 2 && (kc & 1) == 0) ? 2 : 1;
            for (int part = 0; part < nparts; ++part) {
              if (!wait_bar(full_bar(stage), phase)) {
                raise_status(status, abort_flag);
                ok = false;
                break;
              }
              mbar_arrive_remote(map_to_rank(full_bar(stage), 0u));
              if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
          }
        } else {
          for (int kc = 0; kc < J.nkc; ++kc) {
            if (!wait_bar(full_bar(stage), phase)) {
              raise_status(status, abort_flag);
              ok = false;
              break;
            }
            mbar_arrive_remote(map_to_rank(full_bar(stage), 0u));
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int abuf = 0;
      uint32_t aphase = 0;
      int tq = 0;
      uint32_t tqph = 0;
      bool ok = true;
      while (ok) {
        if (!mbar_wait_hint(tqf_bar(tq), tqph, abort_flag, timeout_ns, kHintNs)) {
          raise_status(status, abort_flag);
          break;
        }
        const int t = tile_q[tq];
        mbar_arrive(tqe_bar(tq));
        if (++tq == kTileQ) { tq = 0; tqph ^= 1u; }
        if (t < 0) break;
        const TileJob J = job_of(t);
        const uint32_t idesc = make_idesc_bf16(PAIR ? 256 : 128, J.bn);
        if (!wait_bar(acce_bar(abuf), aphase ^ 1u)) {
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
          if (!wait_bar(full_bar(s0), ph0)) {
            raise_status(status, abort_flag);
            ok = false;
            break;
          }
          if (J.parts == 2 && (kc & 1) == 0) {
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
            s1 = stage;
            if (!mbar_wait_hint(full_bar(s1), phase, abort_flag, timeout_ns, kHintNs)) {
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
            if constexpr (PAIR) {
              mma_bf16_pair(d_tmem, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
              mma_bf16_pair(d_tmem, ah, bl, idesc, 1u);
              mma_bf16_pair(d_tmem, al, bh, idesc, 1u);
              if constexpr (THREE) {
                // with three parts: hi*lo3 + mid*mid + lo3*hi (al, bl above are mid)
                const uint64_t a3 = make_desc_sw128(a3_addr + 32u * kk);
                const uint64_t b3 = make_desc_sw128(b3_addr + 32u * kk);
                mma_bf16_pair(d_tmem, ah, b3, idesc, 1u);
                mma_bf16_pair(d_tmem, al, bl, idesc, 1u);
                mma_bf16_pair(d_tmem, a3, bh, idesc, 1u);
              }
            } else {
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
          }
          if constexpr (PAIR) {
            mma_commit_pair(empty_bar(s0), 0x3);  // frees the slot in both CTAs once these MMAs have read it
            if constexpr (THREE) {
              if ((kc & 1) == 1 || kc == J.nkc - 1) mma_commit_pair(empty_bar(s1), 0x3);
            }
          } else {
            mma_commit(empty_bar(s0));  // frees the slot once these MMAs have read it
            if (J.parts == 2 && ((kc & 1) == 1 || kc == J.nkc - 1)) mma_commit(empty_bar(s1));
          }
          if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        // the tile's accumulator is complete (with pairs: in both CTAs' TMEM)
        if constexpr (PAIR) mma_commit_pair(accf_bar(abuf), 0x3);
        else mma_commit(accf_bar(abuf));
        if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
      }
      // Wait until every MMA issued here has finished before TMEM is released.
      if constexpr (PAIR) mma_commit_pair(drain_bar, 0x1);
      else mma_commit(drain_bar);
      volatile int never = 0;
      if (!mbar_wait(drain_bar, 0u, &never, kDrainTimeoutNs)) raise_status(status, abort_flag);
    }
    __syncwarp();
  } else if (warp < kCpfWarp) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;  // column quarter: 0 .. 3
    int abuf = 0;
    uint32_t aphase = 0;
    int tq = 0;
    uint32_t tqph = 0;
    for (;;) {
      int ok = 1, t = -1;
      if (lane == 0) {
        ok = mbar_wait_hint(tqf_bar(tq), tqph, abort_flag, timeout_ns, kHintNs) ? 1 : 0;
        if (ok) {
          t = tile_q[tq];
          mbar_arrive(tqe_bar(tq));
        }
      }
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      t = __shfl_sync(0xFFFFFFFFu, t, 0);
      if (++tq == kTileQ) { tq = 0; tqph ^= 1u; }
      if (!ok) {
        if (lane == 0) raise_status(status, abort_flag);
        break;
      }
      if (t < 0) break;
      const TileJob J = job_of(t);
      if (lane == 0) ok = wait_bar(accf_bar(abuf), aphase) ? 1 : 0;
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_status(status, abort_flag);
        break;
      }
      tc_fence_after();
      const int64_t i = J.m0 + q * 32 + lane;
      const bool row_ok = i < J.m;
      // maxima were built by other CTAs' atomics: read them through L2
      const int ea = row_ok ? scale_exp_from_bits(__ldcg(J.amaxA + i)) : 0;
      const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * kMaxBN);
      float* const crow = J.C + i;
      constexpr int EC = 32;
      const int cols = (J.bn / (kEpiWarps / 4)) > 32 ? J.bn / (kEpiWarps / 4) : 32;
      const int c_begin = part * cols, c_end = (c_begin + cols < J.bn) ? c_begin + cols : J.bn;
      if (J.partial && J.m0 < J.m) {
        // split-K slice: the raw accumulator, whole tile, 32 consecutive rows
        // per warp store (not for the empty odd half of a last pair, which
        // has no partial tile)
        float* pp = J.partial + q * 32 + lane;
        for (int c0 = c_begin; c0 < c_end; c0 += EC) {
          uint32_t r[EC];
          tmem_ld32(taddr + (uint32_t)c0, r);
#pragma unroll
          for (int jj = 0; jj < EC; ++jj) __stcg(pp + (size_t)(c0 + jj) * 128, __uint_as_float(r[jj]));
        }
      }
      for (int c0 = c_begin; c0 < c_end && !J.partial; c0 += EC) {
        if (J.n0 + c0 >= J.n) break;  // warp-uniform
        const int jmax = (J.n - (J.n0 + c0) < EC) ? (int)(J.n - (J.n0 + c0)) : EC;
        float* cp = crow + (J.n0 + c0) * J.ldc;
        // All loads of the chunk are issued before any result is formed, so
        // the column reads of C overlap instead of queueing one by one.
        float cv[EC];
        if (J.beta != 0.f) {
#pragma unroll
          for (int jj = 0; jj < EC; ++jj) cv[jj] = (row_ok && jj < jmax) ? __ldcs(cp + jj * J.ldc) : 0.f;
        }
        const int64_t jl = J.n0 + c0 + lane;
        const int eb_l = (lane < EC && jl < J.n) ? scale_exp_from_bits(__ldcg(J.amaxB + jl)) : 0;
        uint32_t r[EC];
        tmem_ld32(taddr + (uint32_t)c0, r);
        if (__all_sync(0xFFFFFFFFu, ea == 0 && eb_l == 0)) {
          // No badly scaled row or column in this 32 x 32 block (the usual
          // case): the scale factor is 1 and acc * 1 = acc exactly.
          if (__all_sync(0xFFFFFFFFu, row_ok) && jmax == EC) {
            if (J.beta != 0.f) {
#pragma unroll
              for (int jj = 0; jj < EC; ++jj) __stcs(cp + jj * J.ldc, fmaf(J.alpha, __uint_as_float(r[jj]), J.beta * cv[jj]));
            } else {
#pragma unroll
              for (int jj = 0; jj < EC; ++jj) __stcs(cp + jj * J.ldc, J.alpha * __uint_as_float(r[jj]));
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < EC; ++jj) {
              const float acc = __uint_as_float(r[jj]);
              const float out = (J.beta != 0.f) ? fmaf(J.alpha, acc, J.beta * cv[jj]) : J.alpha * acc;
              if (row_ok && jj < jmax) __stcs(cp + jj * J.ldc, out);
            }
          }
        } else {
          // Every lane runs every shuffle; only the stores are predicated.
#pragma unroll
          for (int jj = 0; jj < EC; ++jj) {
            const int s = ea + __shfl_sync(0xFFFFFFFFu, eb_l, jj);
            const float acc = __uint_as_float(r[jj]);
            // acc * 2^s: one multiply when 2^s is a normal float, else scalbnf.
            const float v = (s >= -126 && s <= 127) ? acc * __int_as_float((s + 127) << 23) : scalbnf(acc, s);
            const float out = (J.beta != 0.f) ? fmaf(J.alpha, v, J.beta * cv[jj]) : J.alpha * v;
            if (row_ok && jj < jmax) __stcs(cp + jj * J.ldc, out);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        // the accumulator buffer is free again: rank 0's MMA issuer waits for
        // both CTAs' epilogue warps of a pair
        if (PAIR && crank != 0u) mbar_arrive_remote(map_to_rank(acce_bar(abuf), 0u));
        else mbar_arrive(acce_bar(abuf));
      }
      if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
    }
  } else if (warp == kCpfWarp) {
    // ---------------- C prefetch ----------------
    // With beta != 0 the epilogue reads the tile's C: ask L2 for it as soon
    // as the tile is handed out, one to three tiles ahead of the epilogue.
    int tq = 0;
    uint32_t tqph = 0;
    for (;;) {
      int ok = 1, t = -1;
      if (lane == 0) {
        ok = mbar_wait_hint(tqf_bar(tq), tqph, abort_flag, timeout_ns, kHintNs) ? 1 : 0;
        if (ok) {
          t = tile_q[tq];
          mbar_arrive(tqe_bar(tq));
        }
      }
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      t = __shfl_sync(0xFFFFFFFFu, t, 0);
      if (++tq == kTileQ) { tq = 0; tqph ^= 1u; }
      if (!ok || t < 0) break;
      const TileJob J = job_of(t);
      // Only short tiles (k <= 512), whose epilogue rather than their MMAs
      // sets the pace, are prefetched: for long ones the C reads overlap the
      // next tile's MMAs anyway, and prefetching several 128 KB tiles ahead
      // would push the operand panels out of L2.
      if (J.beta == 0.f || J.partial || J.nkc > 16 || J.m0 >= J.m) continue;
      const int64_t rows = (J.m - J.m0 < 128) ? J.m - J.m0 : 128;
      const int64_t ncols = (J.n - J.n0 < J.bn) ? J.n - J.n0 : J.bn;
      const float* c0 = J.C + J.m0 + J.n0 * J.ldc;
      for (int64_t j = lane; j < ncols; j += 32) {
        const char* col = reinterpret_cast<const char*>(c0 + j * J.ldc);
        for (int64_t off = 0; off < rows * 4; off += 128) prefetch_l2(col + off);
        prefetch_l2(col + rows * 4 - 4);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // a pair's CTAs leave together: rank 0's MMAs (which read the odd CTA's
  // shared memory and write its TMEM) have completed, and no arrival on the
  // other CTA's barriers is still to come
  if constexpr (PAIR) cluster_sync_all();
  tc_fence_after();
  if (warp == 1) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
  }
}

// The shared-memory opt-in is a per-device function attribute: set it once
// for every device a kernel instance is launched on.
template <class Sched, int STAGES = kStages, int MAXBN = kMaxBN, bool PAIR = false, bool THREE = false>
cudaError_t ensure_gemm_smem_attr() {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(split_gemm_kernel<Sched, STAGES, MAXBN, PAIR, THREE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             gemm_smem_bytes<STAGES, MAXBN, PAIR>());
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  return cudaSuccess;
}

// Launch the GEMM on stream s; with `dependent` it may start while the
// kernel before it on the stream (the packing launch) still runs, and waits
// for that kernel's results after setting itself up.
template <class Sched, int STAGES = kStages, int MAXBN = kMaxBN>
cudaError_t launch_gemm_kernel(const Sched& S, int grid, int* status, cudaStream_t s, bool dependent) {
  cudaError_t e = ensure_gemm_smem_attr<Sched, STAGES, MAXBN>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kGemmThreads);
  cfg.dynamicSmemBytes = gemm_smem_bytes<STAGES, MAXBN>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, split_gemm_kernel<Sched, STAGES, MAXBN>, S, status, (uint64_t)kTimeoutNs);
}

// The pair-tile instances: clusters of two CTAs, THREE for three-part panels
// (k < 512).  How many pairs the GPU holds at once (one CTA per SM; a pair
// needs two SMs of one cluster-capable group) is asked once per device and
// instance; 0 when clusters of two cannot run.
template <class Sched, bool THREE = false>
int gemm_pair_capacity() {
  static int cap[64];
  static bool known[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!known[dev]) {
    int n = 0;
    if (ensure_gemm_smem_attr<Sched, kPairStages, kMaxBN, true, THREE>() == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2);
      cfg.blockDim = dim3(kGemmThreads);
      cfg.dynamicSmemBytes = gemm_smem_bytes<kPairStages, kMaxBN, true>();
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cudaOccupancyMaxActiveClusters(&n, split_gemm_kernel<Sched, kPairStages, kMaxBN, true, THREE>, &cfg) !=
          cudaSuccess)
        n = 0;
    }
    (void)cudaGetLastError();  // a failed query leaves the pair instance unused, not an error
    cap[dev] = n;
    known[dev] = true;
  }
  return cap[dev];
}

// Launch `pairs` clusters of two CTAs of a pair-tile instance (S.pair set).
template <class Sched, bool THREE = false>
cudaError_t launch_gemm_kernel_pair(const Sched& S, int pairs, int* status, cudaStream_t s, bool dependent) {
  cudaError_t e = ensure_gemm_smem_attr<Sched, kPairStages, kMaxBN, true, THREE>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  cfg.blockDim = dim3(kGemmThreads);
  cfg.dynamicSmemBytes = gemm_smem_bytes<kPairStages, kMaxBN, true>();
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, split_gemm_kernel<Sched, kPairStages, kMaxBN, true, THREE>, S, status,
                            (uint64_t)kTimeoutNs);
}

}  // namespace
}  // namespace gbg
