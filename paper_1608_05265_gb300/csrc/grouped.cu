// Grouped sgemm: thousands of independent problems in one captured CUDA
// graph.  This is the BLIS driver idea of Section III-A -- divide the work
// into small predefined multiplications for the micro-kernel -- applied
// across problems: every problem is cut into tiles, the tiles of all
// problems form one work list per kernel, and persistent CTAs drain it.
//
// Graph (one launch): [zero row maxima] -> grouped pack -> grouped re-pack
// of badly scaled vectors -> grouped tcgen05 GEMM over all split-path
// problems -> one grouped SIMT kernel per SIMT tile shape.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gemm_kernel.cuh"
#include "grouped.h"
#include "simt_device.cuh"

namespace gbg {
namespace {

// One operand of one split-path problem, as seen by the packing kernels.
struct PackTask {
  const float* X;
  int64_t ld;
  uint32_t* amax;
  uint8_t* panel;
  uint8_t* panel2;         // compact lo3 panel of a three-part split, else NULL
  int64_t rows, k;
  int64_t rb_count, nkc;   // 128-row blocks per k chunk, k chunks
  int64_t rows_alloc;      // panel rows per k chunk (rows rounded up to 8)
  int64_t block_begin;     // first pack-kernel block of this task
  int64_t rowblock_begin;  // first rescale-kernel block of this task
  int kcontig;
  int pad_;
};

// block_task[b]: the task of pack-kernel block b (and, for the re-pack
// kernel, of row block b), built on the host at plan creation.  A pack
// block splits kPackChunks consecutive k chunks of one 128-row block, with
// all their loads in flight at once.
constexpr int kPackChunks = 2;
__global__ void __launch_bounds__(256) grouped_pack_kernel(const PackTask* __restrict__ tasks,
                                                           const int* __restrict__ block_task) {
  __shared__ uint32_t smax[128];
  const PackTask T = tasks[block_task[blockIdx.x]];
  const int64_t local = (int64_t)blockIdx.x - T.block_begin;
  const int64_t rb = local % T.rb_count, kc0 = (local / T.rb_count) * kPackChunks;
  if (T.kcontig)
    pack_block<true, kPackChunks>(T.rows, T.k, T.X, T.ld, T.amax, T.panel, T.panel2, T.rows_alloc, rb, kc0, smax, T.nkc);
  else
    pack_block<false, kPackChunks>(T.rows, T.k, T.X, T.ld, T.amax, T.panel, T.panel2, T.rows_alloc, rb, kc0, smax, T.nkc);
}

__global__ void __launch_bounds__(256) grouped_rescale_kernel(const PackTask* __restrict__ tasks,
                                                              const int* __restrict__ rowblock_task) {
  __shared__ int se[128];
  const PackTask T = tasks[rowblock_task[blockIdx.x]];
  const int64_t rb = (int64_t)blockIdx.x - T.rowblock_begin;
  rescale_block(T.rows, T.k, T.X, T.ld, T.kcontig != 0, T.amax, T.panel, T.panel2, T.rows_alloc, T.nkc, rb, se);
}

// Items: x = problem index into `probs`, y = tile row, z = tile column.
// One launch per tile shape and (transpose, vector-load) variant, so each
// launch is a fully specialised tile loop.
template <int BM, int BN, bool TA, bool TB, bool VEC>
__global__ void __launch_bounds__((BM / 8) * (BN / 8), 512 / ((BM / 8) * (BN / 8)))
grouped_simt_kernel(const int4* __restrict__ items, int n_items, const Problem* __restrict__ probs) {
  __shared__ __align__(16) SimtSmem<BM, BN> sm;
  // The item's problem descriptor is staged in shared memory so that its
  // fields are re-read where used instead of held in registers.
  __shared__ Problem sp;
  __shared__ int4 sit;
  for (int t = blockIdx.x; t < n_items; t += gridDim.x) {
    if (threadIdx.x == 0) {
      sit = items[t];
      sp = probs[sit.x];
    }
    __syncthreads();
    simt_tile<BM, BN, TA, TB, VEC>(sp, (int64_t)sit.y * BM, (int64_t)sit.z * BN, sm.As, sm.Bs);
    __syncthreads();  // the next item reuses the shared-memory slices and descriptor
  }
}

template <int BM, int BN>
void launch_grouped_simt(int variant, int grid, cudaStream_t s, const int4* items, int n, const Problem* probs) {
  constexpr int NT = (BM / 8) * (BN / 8);
  switch (variant) {
    case 0: grouped_simt_kernel<BM, BN, false, false, false><<<grid, NT, 0, s>>>(items, n, probs); break;
    case 1: grouped_simt_kernel<BM, BN, true, false, false><<<grid, NT, 0, s>>>(items, n, probs); break;
    case 2: grouped_simt_kernel<BM, BN, false, true, false><<<grid, NT, 0, s>>>(items, n, probs); break;
    case 3: grouped_simt_kernel<BM, BN, true, true, false><<<grid, NT, 0, s>>>(items, n, probs); break;
    case 4: grouped_simt_kernel<BM, BN, false, false, true><<<grid, NT, 0, s>>>(items, n, probs); break;
    case 5: grouped_simt_kernel<BM, BN, true, false, true><<<grid, NT, 0, s>>>(items, n, probs); break;
    case 6: grouped_simt_kernel<BM, BN, false, true, true><<<grid, NT, 0, s>>>(items, n, probs); break;
    default: grouped_simt_kernel<BM, BN, true, true, true><<<grid, NT, 0, s>>>(items, n, probs); break;
  }
}

int trans_code_g(char t) {
  switch (t) {
    case 'N': case 'n': return 0;
    case 'T': case 't': case 'C': case 'c': return 1;
    default: return -1;
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------

int validate_problem(const gbgemm_problem& q) {
  const int ta = trans_code_g(q.transa), tb = trans_code_g(q.transb);
  if (ta < 0) return -1;
  if (tb < 0) return -2;
  if (q.m < 0) return -3;
  if (q.n < 0) return -4;
  if (q.k < 0) return -5;
  const int64_t arows = ta ? q.k : q.m, brows = tb ? q.n : q.k;
  if (q.lda < (arows > 1 ? arows : 1)) return -8;
  if (q.ldb < (brows > 1 ? brows : 1)) return -10;
  if (q.ldc < (q.m > 1 ? q.m : 1)) return -13;
  const bool use_ab = (q.alpha != 0.0f) && (q.k > 0);
  if (q.m > 0 && q.n > 0) {
    if (use_ab && !q.A) return -7;
    if (use_ab && !q.B) return -9;
    if (!q.C) return -12;
  }
  return 0;
}

bool config_legal(const gbgemm_problem& q, int cfg) {
  if (cfg < 0 || cfg >= GBGEMM_NUM_CONFIGS) return false;
  if (cfg >= GBGEMM_CFG_SPLIT_BN64) return q.k >= kSplitMinK && q.alpha != 0.0f;
  return true;
}

int default_config(const gbgemm_problem& q) {
  if (q.k >= kSplitMinK && q.alpha != 0.0f) return q.n <= 64 ? GBGEMM_CFG_SPLIT_BN64 : GBGEMM_CFG_SPLIT_BN128;
  // SIMT: the tile shape with the least padded area (ties to the larger tile)
  auto area = [&](int64_t bm, int64_t bn) { return ((q.m + bm - 1) / bm) * bm * (((q.n + bn - 1) / bn) * bn); };
  const int64_t a_big = area(128, 128), a_wide = area(128, 64), a_small = area(64, 64);
  if (a_big <= a_wide && a_big <= a_small) return GBGEMM_CFG_SIMT_128x128;
  return a_wide <= a_small ? GBGEMM_CFG_SIMT_128x64 : GBGEMM_CFG_SIMT_64x64;
}

int config_bn(int cfg) { return cfg == GBGEMM_CFG_SPLIT_BN64 ? 64 : cfg == GBGEMM_CFG_SPLIT_BN128 ? 128 : 256; }

void simt_tile_shape(int cfg, int& bm, int& bn) {
  switch (cfg) {
    case GBGEMM_CFG_SIMT_64x64: bm = 64; bn = 64; break;
    case GBGEMM_CFG_SIMT_128x64: bm = 128; bn = 64; break;
    default: bm = 128; bn = 128; break;
  }
}

GroupedPlan::~GroupedPlan() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (dmem) cudaFree(dmem);
}

int build_grouped_plan(GroupedPlan* P, const gbgemm_problem* probs, int64_t count, const int* configs,
                       cudaStream_t capture_stream) {
  // ---- classify and lay out device memory ----
  std::vector<PackTask> tasks;
  std::vector<GroupDev> gdev;
  std::vector<int64_t> split_of;           // problem index of each split group
  std::vector<Problem> sprobs;             // SIMT problems
  std::vector<int> simt_cfg;
  struct Region { size_t off, bytes; };
  size_t off = 0;
  auto take = [&](size_t bytes) { Region r{off, bytes}; off = align256(off + bytes); return r; };
  std::vector<Region> panelA_r, panelB_r, panelA2_r, panelB2_r;
  int64_t amax_words = 0;
  P->flops_split = P->flops_simt = 0.0;
  for (int64_t g = 0; g < count; ++g) {
    const gbgemm_problem& q = probs[g];
    const int cfg = configs[g];
    if (q.m == 0 || q.n == 0) continue;
    const bool use_ab = (q.alpha != 0.0f) && (q.k > 0);
    if (!use_ab && q.beta == 1.0f) continue;
    const int ta = trans_code_g(q.transa), tb = trans_code_g(q.transb);
    if (use_ab && cfg >= GBGEMM_CFG_SPLIT_BN64) {
      // Compact panels: rows rounded up to 8 per k chunk.  A tile copy may
      // run past the last row into the next chunk (or, for the last chunk,
      // into 32 KiB of slack): those rows feed only outputs that are never
      // stored.
      const int bn = config_bn(cfg);
      const int64_t rowsA = (q.m + 7) / 8 * 8, rowsB = (q.n + 7) / 8 * 8;
      const int64_t nkc = panel_k_chunks(q.k);
      const int parts = split_parts(q.k);
      panelA_r.push_back(take((size_t)rowsA * nkc * 128 + 32768));
      panelB_r.push_back(take((size_t)rowsB * nkc * 128 + 32768));
      // three parts: compact [lo3 | lo3] panels, one block per pair of k chunks
      panelA2_r.push_back(parts == 2 ? take((size_t)rowsA * ((nkc + 1) / 2) * 128 + 32768) : Region{0, 0});
      panelB2_r.push_back(parts == 2 ? take((size_t)rowsB * ((nkc + 1) / 2) * 128 + 32768) : Region{0, 0});
      split_of.push_back(g);
      GroupDev d{};
      d.m = q.m; d.n = q.n; d.nkc = (int)nkc; d.bn = bn; d.rowsA = rowsA; d.rowsB = rowsB;
      d.parts = parts;
      d.alpha = q.alpha; d.beta = q.beta; d.C = q.C; d.ldc = q.ldc;
      gdev.push_back(d);
      amax_words += q.m + q.n;
      P->flops_split += 2.0 * q.m * q.n * q.k;
    } else {
      Problem p{ta, tb, q.m, q.n, use_ab ? q.k : 0, use_ab ? q.alpha : 0.0f, q.beta, q.A, q.lda, q.B, q.ldb, q.C, q.ldc};
      sprobs.push_back(p);
      simt_cfg.push_back(cfg >= GBGEMM_CFG_SPLIT_BN64 ? default_config(q) : cfg);
      if (use_ab) P->flops_simt += 2.0 * q.m * q.n * q.k;
    }
  }
  const Region amax_r = take((size_t)amax_words * 4 + 4);
  // work lists
  std::vector<int4> split_items;
  for (size_t s = 0; s < gdev.size(); ++s) {
    const int64_t tm = (gdev[s].m + 127) / 128, tn = (gdev[s].n + gdev[s].bn - 1) / gdev[s].bn;
    for (int64_t i = 0; i < tm; ++i)
      for (int64_t j = 0; j < tn; ++j) split_items.push_back(make_int4((int)s, (int)i, (int)j, 0));
  }
  // Longest-processing-time order: costlier tiles first (k chunks x tile width).
  std::stable_sort(split_items.begin(), split_items.end(), [&](const int4& a, const int4& b) {
    return (int64_t)gdev[a.x].nkc * gdev[a.x].bn > (int64_t)gdev[b.x].nkc * gdev[b.x].bn;
  });
  std::vector<int4> simt_items[3 * 8];  // index: config * 8 + variant
  for (size_t s = 0; s < sprobs.size(); ++s) {
    int bm, bn;
    simt_tile_shape(simt_cfg[s], bm, bn);
    const Problem& p = sprobs[s];
    const bool vec = ((p.lda & 3) == 0) && ((p.ldb & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.A) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(p.B) & 15) == 0);
    const int flags = p.ta | (p.tb << 1) | ((vec && p.k > 0) ? 4 : 0);
    const int64_t tm = (p.m + bm - 1) / bm, tn = (p.n + bn - 1) / bn;
    for (int64_t i = 0; i < tm; ++i)
      for (int64_t j = 0; j < tn; ++j) simt_items[simt_cfg[s] * 8 + flags].push_back(make_int4((int)s, (int)i, (int)j, 0));
  }
  for (auto& v : simt_items)
    std::stable_sort(v.begin(), v.end(), [&](const int4& a, const int4& b) { return sprobs[a.x].k > sprobs[b.x].k; });
  const Region gdev_r = take(gdev.size() * sizeof(GroupDev) + 16);
  const Region sitems_r = take(split_items.size() * sizeof(int4) + 16);
  const Region sprob_r = take(sprobs.size() * sizeof(Problem) + 16);
  Region simt_items_r[24];
  for (int c = 0; c < 24; ++c) simt_items_r[c] = take(simt_items[c].size() * sizeof(int4) + 16);
  const Region tasks_r = take(2 * gdev.size() * sizeof(PackTask) + 16);
  // block -> task maps of the packing kernels (sized below, once the tasks are known)
  int64_t n_blocks = 0, n_rowblocks = 0;
  for (size_t s = 0; s < gdev.size(); ++s) {
    const gbgemm_problem& q = probs[split_of[s]];
    n_blocks += ((q.m + 127) / 128 + (q.n + 127) / 128) * ((gdev[s].nkc + kPackChunks - 1) / kPackChunks);
    n_rowblocks += (q.m + 127) / 128 + (q.n + 127) / 128;
  }
  if (n_blocks > 0x7FFFFFFF || n_rowblocks > 0x7FFFFFFF) return GBGEMM_ERR_INVALID_VALUE;
  const Region bmap_r = take((size_t)n_blocks * 4 + 16);
  const Region rmap_r = take((size_t)n_rowblocks * 4 + 16);

  if (off > 0 && cudaMalloc(&P->dmem, off) != cudaSuccess) {
    cudaGetLastError();
    P->dmem = nullptr;
    return GBGEMM_ERR_ALLOC;
  }
  P->dbytes = off;
  uint8_t* base = static_cast<uint8_t*>(P->dmem);
  // fill pointers
  int64_t aw = 0;
  uint32_t* amax_base = reinterpret_cast<uint32_t*>(base + amax_r.off);
  int64_t blocks = 0, rowblocks = 0;
  for (size_t s = 0; s < gdev.size(); ++s) {
    const gbgemm_problem& q = probs[split_of[s]];
    GroupDev& d = gdev[s];
    d.panelA = base + panelA_r[s].off;
    d.panelB = base + panelB_r[s].off;
    uint8_t* pA2 = d.parts == 2 ? base + panelA2_r[s].off : nullptr;
    uint8_t* pB2 = d.parts == 2 ? base + panelB2_r[s].off : nullptr;
    d.a_part = d.parts == 2 ? (int64_t)(pA2 - d.panelA) : 0;
    d.b_part = d.parts == 2 ? (int64_t)(pB2 - d.panelB) : 0;
    d.amaxA = amax_base + aw;
    d.amaxB = amax_base + aw + q.m;
    aw += q.m + q.n;
    const int ta = trans_code_g(q.transa), tb = trans_code_g(q.transb);
    const int64_t rbA = (q.m + 127) / 128, rbB = (q.n + 127) / 128;
    PackTask ta_{q.A, q.lda, const_cast<uint32_t*>(d.amaxA), const_cast<uint8_t*>(d.panelA), pA2, q.m, q.k,
                 rbA, d.nkc, d.rowsA, blocks, rowblocks, ta == 1, 0};
    blocks += rbA * ((d.nkc + kPackChunks - 1) / kPackChunks);
    rowblocks += rbA;
    PackTask tb_{q.B, q.ldb, const_cast<uint32_t*>(d.amaxB), const_cast<uint8_t*>(d.panelB), pB2, q.n, q.k,
                 rbB, d.nkc, d.rowsB, blocks, rowblocks, tb == 0, 0};
    blocks += rbB * ((d.nkc + kPackChunks - 1) / kPackChunks);
    rowblocks += rbB;
    tasks.push_back(ta_);
    tasks.push_back(tb_);
  }
  std::vector<int> bmap((size_t)blocks), rmap((size_t)rowblocks);
  for (size_t t = 0; t < tasks.size(); ++t) {
    const int64_t nb = tasks[t].rb_count * ((tasks[t].nkc + kPackChunks - 1) / kPackChunks);
    for (int64_t b = 0; b < nb; ++b) bmap[(size_t)(tasks[t].block_begin + b)] = (int)t;
    for (int64_t b = 0; b < tasks[t].rb_count; ++b) rmap[(size_t)(tasks[t].rowblock_begin + b)] = (int)t;
  }
  auto h2d = [&](const Region& r, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpy(base + r.off, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  bool ok = h2d(gdev_r, gdev.data(), gdev.size() * sizeof(GroupDev)) &&
            h2d(sitems_r, split_items.data(), split_items.size() * sizeof(int4)) &&
            h2d(sprob_r, sprobs.data(), sprobs.size() * sizeof(Problem)) &&
            h2d(tasks_r, tasks.data(), tasks.size() * sizeof(PackTask)) &&
            h2d(bmap_r, bmap.data(), bmap.size() * 4) && h2d(rmap_r, rmap.data(), rmap.size() * 4);
  for (int c = 0; c < 24; ++c) ok = ok && h2d(simt_items_r[c], simt_items[c].data(), simt_items[c].size() * sizeof(int4));
  if (!ok) return GBGEMM_ERR_CUDA;
  P->n_split = (int64_t)gdev.size();
  P->n_simt = (int64_t)sprobs.size();
  P->split_tiles = (int64_t)split_items.size();
  P->kernels_per_run = 0;

  // ---- capture the graph ----
  if (blocks > 0x7FFFFFFF || rowblocks > 0x7FFFFFFF) return GBGEMM_ERR_INVALID_VALUE;
  // Tiles of at most 128 columns everywhere: the six-slot ring instance.
  bool narrow = true;
  for (const GroupDev& gd : gdev) narrow = narrow && gd.bn <= kNarrowBN;
  if (!gdev.empty()) {
    const cudaError_t ea = narrow ? ensure_gemm_smem_attr<GroupedSched, kNarrowStages, kNarrowBN>()
                                  : ensure_gemm_smem_attr<GroupedSched>();
    if (ea != cudaSuccess) return GBGEMM_ERR_CUDA;
  }
  // Graph: the SIMT launches run on side branches, concurrently with the
  // split chain (packing, re-packing, tcgen05 GEMM) on the main branch; the
  // branches join at the end.  (Holding the GEMM back until the SIMT
  // branches finish, so that they overlap the memory-bound packing, measured
  // 1% slower.)
  constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, joins[kSide] = {};
  bool res_ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < kSide && res_ok; ++i)
    res_ok = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming) == cudaSuccess;
  auto release = [&]() {
    for (int i = 0; i < kSide; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (joins[i]) cudaEventDestroy(joins[i]);
    }
    if (fork) cudaEventDestroy(fork);
  };
  if (!res_ok) {
    cudaGetLastError();
    release();
    return GBGEMM_ERR_CUDA;
  }
  if (cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    release();
    return GBGEMM_ERR_CUDA;
  }
  cudaError_t e = cudaEventRecord(fork, capture_stream);
  for (int i = 0; i < kSide && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(side[i], fork, 0);
  const Problem* dprobs = reinterpret_cast<const Problem*>(base + sprob_r.off);
  int simt_launches = 0;
  for (int cv = 0; cv < 24 && e == cudaSuccess; ++cv) {
    const int n = (int)simt_items[cv].size();
    if (n == 0) continue;
    const int c = cv / 8, variant = cv % 8;
    const int4* di = reinterpret_cast<const int4*>(base + simt_items_r[cv].off);
    // resident CTAs per SM at the kernels' 512-thread bound: 2, 4 or 8
    const int per_sm = (c == GBGEMM_CFG_SIMT_128x128) ? 2 : (c == GBGEMM_CFG_SIMT_128x64) ? 4 : 8;
    const int grid = (int)std::min<int64_t>(n, (int64_t)P->num_sms * per_sm);
    cudaStream_t st = side[simt_launches % kSide];
    if (c == GBGEMM_CFG_SIMT_128x128) launch_grouped_simt<128, 128>(variant, grid, st, di, n, dprobs);
    else if (c == GBGEMM_CFG_SIMT_64x64) launch_grouped_simt<64, 64>(variant, grid, st, di, n, dprobs);
    else launch_grouped_simt<128, 64>(variant, grid, st, di, n, dprobs);
    ++simt_launches;
  }
  P->kernels_per_run += simt_launches;
  if (!gdev.empty() && e == cudaSuccess) {
    const PackTask* dt = reinterpret_cast<const PackTask*>(base + tasks_r.off);
    e = cudaMemsetAsync(amax_base, 0, (size_t)amax_words * 4, capture_stream);
    if (e == cudaSuccess) {
      const int* dbmap = reinterpret_cast<const int*>(base + bmap_r.off);
      const int* drmap = reinterpret_cast<const int*>(base + rmap_r.off);
      grouped_pack_kernel<<<(unsigned)blocks, 256, 0, capture_stream>>>(dt, dbmap);
      grouped_rescale_kernel<<<(unsigned)rowblocks, 256, 0, capture_stream>>>(dt, drmap);
      P->kernels_per_run += 2;
    }
  }
  if (!gdev.empty() && e == cudaSuccess) {
    GroupedSched S;
    S.items = reinterpret_cast<const int4*>(base + sitems_r.off);
    S.groups = reinterpret_cast<const GroupDev*>(base + gdev_r.off);
    S.n_items = (int)split_items.size();
    const int grid = (int)std::min<int64_t>((int64_t)split_items.size(), P->num_sms);
    if (narrow)
      split_gemm_kernel<GroupedSched, kNarrowStages, kNarrowBN>
          <<<grid, kGemmThreads, gemm_smem_bytes<kNarrowStages, kNarrowBN>(), capture_stream>>>(S, P->status,
                                                                                               kTimeoutNs);
    else
      split_gemm_kernel<GroupedSched><<<grid, kGemmThreads, kGemmSmemBytes, capture_stream>>>(S, P->status, kTimeoutNs);
    P->kernels_per_run += 1;
  }
  for (int i = 0; i < kSide && e == cudaSuccess; ++i) {
    e = cudaEventRecord(joins[i], side[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(capture_stream, joins[i], 0);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(capture_stream, &g);
  release();
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return GBGEMM_ERR_CUDA;
  }
  P->graph = g;
  if (cudaGraphInstantiate(&P->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    P->exec = nullptr;
    return GBGEMM_ERR_CUDA;
  }
  return GBGEMM_OK;
}

}  // namespace gbg
