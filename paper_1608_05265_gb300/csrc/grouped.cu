// Grouped sgemm: thousands of independent problems in one captured CUDA
// graph.  This is the BLIS driver idea of Section III-A -- divide the work
// into small predefined multiplications for the micro-kernel -- applied
// across problems: every problem is cut into tiles, the tiles of all
// problems form one work list per kernel, and persistent CTAs drain it.
//
// Graph (one launch): zero the counters and row maxima, pack every operand
// of the split-path problems (one CTA per 128-row band and four k chunks),
// then the persistent tcgen05 GEMM over all their tiles; the SIMT-configured
// problems run on side branches, one grouped SIMT kernel per tile shape and
// variant.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gemm_kernel.cuh"
#include "grouped.h"
#include "simt_device.cuh"

namespace gbg {
namespace {

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
  if (cfg >= GBGEMM_CFG_SPLIT_BN64) return q.k >= kSplitShortK && q.alpha != 0.0f;
  return true;
}

int default_config(const gbgemm_problem& q) {
  if (q.k >= kSplitShortK && q.alpha != 0.0f) return q.n <= 64 ? GBGEMM_CFG_SPLIT_BN64 : GBGEMM_CFG_SPLIT_BN128;
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
  // ---- classify ----
  struct SplitProb {
    int64_t g;             // index into probs
    int bn, nkc, parts, ra, rb, tiles;
    int64_t rowsA, rowsB;
    size_t offA, offB, offA2, offB2, size;  // panel layout inside the problem's region
    double cost;           // per tile: k chunks x width x products
  };
  std::vector<SplitProb> sp;
  std::vector<Problem> sprobs;             // SIMT problems
  std::vector<int> simt_cfg;
  P->flops_split = P->flops_simt = 0.0;
  for (int64_t g = 0; g < count; ++g) {
    const gbgemm_problem& q = probs[g];
    const int cfg = configs[g];
    if (q.m == 0 || q.n == 0) continue;
    const bool use_ab = (q.alpha != 0.0f) && (q.k > 0);
    if (!use_ab && q.beta == 1.0f) continue;
    const int ta = trans_code_g(q.transa), tb = trans_code_g(q.transb);
    if (use_ab && cfg >= GBGEMM_CFG_SPLIT_BN64) {
      SplitProb x{};
      x.g = g;
      x.bn = config_bn(cfg);
      x.nkc = (int)panel_k_chunks(q.k);
      x.parts = split_parts(q.k);
      x.ra = (int)((q.m + 127) / 128);
      x.rb = (int)((q.n + 127) / 128);
      x.tiles = x.ra * (int)((q.n + x.bn - 1) / x.bn);
      // compact panels: rows rounded up to 8 per k chunk
      x.rowsA = (q.m + 7) / 8 * 8;
      x.rowsB = (q.n + 7) / 8 * 8;
      x.cost = (double)x.nkc * x.bn * (x.parts == 2 ? 2.0 : 1.0);
      sp.push_back(x);
      P->flops_split += 2.0 * q.m * q.n * q.k;
    } else {
      Problem p{ta, tb, q.m, q.n, use_ab ? q.k : 0, use_ab ? q.alpha : 0.0f, q.beta, q.A, q.lda, q.B, q.ldb, q.C, q.ldc};
      sprobs.push_back(p);
      simt_cfg.push_back(cfg >= GBGEMM_CFG_SPLIT_BN64 ? default_config(q) : cfg);
      if (use_ab) P->flops_simt += 2.0 * q.m * q.n * q.k;
    }
  }
  // Packing and tile order: problem after problem, costlier tiles first, so
  // that the cheap tiles come last and even out the CTAs' finishing times.
  std::stable_sort(sp.begin(), sp.end(), [](const SplitProb& a, const SplitProb& b) { return a.cost > b.cost; });

  // ---- panels ----
  // Each problem's panels ([hi | lo] or [hi | mid] of op(A) and op(B), and
  // with three parts the compact lo3 panels) take one contiguous region.  A
  // tile copy may run up to 32 KiB past its panel's end: into the next
  // region, or into slack after the last; those rows only feed outputs that
  // are never stored.
  auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t total = 0;
  std::vector<size_t> prob_off(sp.size());
  for (size_t i = 0; i < sp.size(); ++i) {
    SplitProb& x = sp[i];
    const size_t a = a256((size_t)x.rowsA * x.nkc * 128), b = a256((size_t)x.rowsB * x.nkc * 128);
    const int pairs = (x.nkc + 1) / 2;
    const size_t a2 = x.parts == 2 ? a256((size_t)x.rowsA * pairs * 128) : 0;
    const size_t b2 = x.parts == 2 ? a256((size_t)x.rowsB * pairs * 128) : 0;
    x.offA = 0; x.offB = a; x.offA2 = a + b; x.offB2 = a + b + a2;
    x.size = a + b + a2 + b2;
    prob_off[i] = total;
    total += x.size;
  }

  // ---- bands, packing tasks, tiles ----
  std::vector<PackBand> bands;
  std::vector<int> band_prob, band_isa;  // host only: each band's problem and operand
  std::vector<int> task_band;
  std::vector<int4> split_items;
  std::vector<GroupDev> gdev(sp.size());
  int64_t amax_words = 0, n_cnt = 0;
  for (size_t i = 0; i < sp.size(); ++i) {
    amax_words += probs[sp[i].g].m + probs[sp[i].g].n;
    n_cnt += sp[i].ra + sp[i].rb;
  }
  if (n_cnt > 0x3FFFFFFF) return GBGEMM_ERR_INVALID_VALUE;
  struct Region { size_t off, bytes; };
  size_t off = 0;
  auto take = [&](size_t bytes) { Region r{off, bytes}; off = align256(off + bytes); return r; };
  const Region ctl_r = take(kSplitCtlBytes);
  const Region cnt_r = take((size_t)n_cnt * 4);
  const Region amax_r = take((size_t)amax_words * 4 + 4);
  const size_t head_bytes = off;
  int64_t cnt_base = 0, aw = 0;
  for (size_t i = 0; i < sp.size(); ++i) {
    const SplitProb& x = sp[i];
    const gbgemm_problem& q = probs[x.g];
    GroupDev& d = gdev[i];
    d.m = q.m; d.n = q.n; d.nkc = x.nkc; d.bn = x.bn; d.rowsA = x.rowsA; d.rowsB = x.rowsB;
    d.parts = x.parts;
    d.alpha = q.alpha; d.beta = q.beta; d.C = q.C; d.ldc = q.ldc;
    // bands in the order of the first tile that reads them (tiles go column
    // of tiles by column of tiles): op(B)'s bands of tile column 0, every
    // band of op(A), the remaining bands of op(B)
    const int nb0 = std::min(x.rb, std::max(1, x.bn >> 7));
    const int ngroups = (x.nkc + kPackChunks - 1) / kPackChunks;
    const int ta = trans_code_g(q.transa), tb = trans_code_g(q.transb);
    auto add_band = [&](bool is_a, int j) {
      PackBand b{};
      b.X = is_a ? q.A : q.B;
      b.ld = is_a ? q.lda : q.ldb;
      b.rows = is_a ? q.m : q.n;
      b.k = q.k;
      b.rows_alloc = is_a ? x.rowsA : x.rowsB;
      b.rb = j;
      b.nkc = x.nkc;
      b.kcontig = is_a ? (ta == 1) : (tb == 0);
      b.ngroups = ngroups;
      b.first_task = (int)task_band.size();
      b.cnt = (int)cnt_base + (is_a ? 0 : x.ra) + j;
      for (int t = 0; t < ngroups; ++t) task_band.push_back((int)bands.size());
      bands.push_back(b);
      band_prob.push_back((int)i);
      band_isa.push_back(is_a ? 1 : 0);
    };
    for (int j = 0; j < nb0; ++j) add_band(false, j);
    for (int j = 0; j < x.ra; ++j) add_band(true, j);
    for (int j = nb0; j < x.rb; ++j) add_band(false, j);
    const int tn = (int)((q.n + x.bn - 1) / x.bn);
    for (int c = 0; c < tn; ++c)
      for (int r = 0; r < x.ra; ++r) split_items.push_back(make_int4((int)i, r, c, 0));
    cnt_base += x.ra + x.rb;
    aw += q.m + q.n;
  }
  if (task_band.size() > 0x7FFFFFFF || split_items.size() > 0x7FFFFFFF) return GBGEMM_ERR_INVALID_VALUE;
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
  const Region bands_r = take(bands.size() * sizeof(PackBand) + 16);
  const Region tband_r = take(task_band.size() * 4 + 16);
  const Region sprob_r = take(sprobs.size() * sizeof(Problem) + 16);
  Region simt_items_r[24];
  for (int c = 0; c < 24; ++c) simt_items_r[c] = take(simt_items[c].size() * sizeof(int4) + 16);
  const Region panels_r = take(sp.empty() ? 16 : total + 32768);

  if (off > 0 && cudaMalloc(&P->dmem, off) != cudaSuccess) {
    cudaGetLastError();
    P->dmem = nullptr;
    return GBGEMM_ERR_ALLOC;
  }
  P->dbytes = off;
  uint8_t* base = static_cast<uint8_t*>(P->dmem);
  // device addresses of the panels and maxima
  uint32_t* amax_base = reinterpret_cast<uint32_t*>(base + amax_r.off);
  aw = 0;
  std::vector<uint8_t*> pa(sp.size()), pb(sp.size()), pa2(sp.size()), pb2(sp.size());
  for (size_t i = 0; i < sp.size(); ++i) {
    const SplitProb& x = sp[i];
    const gbgemm_problem& q = probs[x.g];
    uint8_t* r0 = base + panels_r.off + prob_off[i];
    pa[i] = r0 + x.offA;
    pb[i] = r0 + x.offB;
    pa2[i] = x.parts == 2 ? r0 + x.offA2 : nullptr;
    pb2[i] = x.parts == 2 ? r0 + x.offB2 : nullptr;
    GroupDev& d = gdev[i];
    d.panelA = pa[i];
    d.panelB = pb[i];
    d.a_part = x.parts == 2 ? (int64_t)(pa2[i] - pa[i]) : 0;
    d.b_part = x.parts == 2 ? (int64_t)(pb2[i] - pb[i]) : 0;
    d.amaxA = amax_base + aw;
    d.amaxB = amax_base + aw + q.m;
    aw += q.m + q.n;
  }
  for (size_t bi = 0; bi < bands.size(); ++bi) {
    PackBand& b = bands[bi];
    const int i = band_prob[bi];
    const bool is_a = band_isa[bi] != 0;
    b.amax = const_cast<uint32_t*>(is_a ? gdev[i].amaxA : gdev[i].amaxB);
    b.panel = is_a ? pa[i] : pb[i];
    b.panel2 = is_a ? pa2[i] : pb2[i];
  }
  auto h2d = [&](const Region& r, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpy(base + r.off, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  bool ok = h2d(gdev_r, gdev.data(), gdev.size() * sizeof(GroupDev)) &&
            h2d(sitems_r, split_items.data(), split_items.size() * sizeof(int4)) &&
            h2d(bands_r, bands.data(), bands.size() * sizeof(PackBand)) &&
            h2d(tband_r, task_band.data(), task_band.size() * 4) &&
            h2d(sprob_r, sprobs.data(), sprobs.size() * sizeof(Problem));
  for (int c = 0; c < 24; ++c) ok = ok && h2d(simt_items_r[c], simt_items[c].data(), simt_items[c].size() * sizeof(int4));
  if (!ok) return GBGEMM_ERR_CUDA;
  P->n_split = (int64_t)sp.size();
  P->n_simt = (int64_t)sprobs.size();
  P->split_tiles = (int64_t)split_items.size();
  P->kernels_per_run = 0;

  // ---- capture the graph ----
  // Tiles of at most 128 columns everywhere: the six-slot ring instance.
  bool narrow = true;
  for (const GroupDev& gd : gdev) narrow = narrow && gd.bn <= kNarrowBN;
  if (!gdev.empty()) {
    const cudaError_t ea = narrow ? ensure_gemm_smem_attr<GroupedSched, kNarrowStages, kNarrowBN>()
                                  : ensure_gemm_smem_attr<GroupedSched>();
    if (ea != cudaSuccess) return GBGEMM_ERR_CUDA;
  }
  // Graph: the SIMT launches run on side branches, concurrently with the
  // split kernel on the main branch; the branches join at the end.  The
  // split kernel hands out its tiles and packing tasks dynamically, so it
  // needs no SM to itself while the branches run.
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
    e = cudaMemsetAsync(base, 0, head_bytes, capture_stream);
    GroupedSched S;
    S.ctl = reinterpret_cast<WorkCtl*>(base + ctl_r.off);
    S.band_cnt = reinterpret_cast<int*>(base + cnt_r.off);
    S.items = reinterpret_cast<const int4*>(base + sitems_r.off);
    S.groups = reinterpret_cast<const GroupDev*>(base + gdev_r.off);
    S.bands = reinterpret_cast<const PackBand*>(base + bands_r.off);
    S.task_band = reinterpret_cast<const int*>(base + tband_r.off);
    S.n_items = (int)split_items.size();
    S.n_tasks = (int)task_band.size();
    if (e == cudaSuccess) {
      // every packing task as its own CTA, then the GEMM
      pack_tasks_kernel<GroupedSched><<<(unsigned)task_band.size(), 256, 0, capture_stream>>>(S);
      const int grid = (int)std::min<int64_t>((int64_t)split_items.size(), P->num_sms);
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = narrow ? launch_gemm_kernel<GroupedSched, kNarrowStages, kNarrowBN>(S, grid, P->status, capture_stream, true)
                   : launch_gemm_kernel<GroupedSched>(S, grid, P->status, capture_stream, true);
      P->kernels_per_run += 3;  // the memset, the packing and the GEMM
    }
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
