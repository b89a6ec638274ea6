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
#include "gemm_kernel.cuh"

namespace gbg {
namespace {

// Split-K reduction: a thread per four consecutive rows i .. i+3 of one
// column j of C (rows of a 128-row tile, so the partials are 16-byte
// vectors), the slices' raw accumulators summed in slice order
// (deterministic), then the epilogue of split_gemm_kernel: x 2^(e_i + f_j),
// alpha, and beta C with one rounding of beta C and one fused multiply-add.
// Every load of a thread is independent, so one pass over the grid keeps
// them all in flight.
__global__ void __launch_bounds__(256) splitk_reduce_kernel(int64_t m, int64_t n, int bn, int tiles_m, int tiles_n,
                                                            int splitk, const float* __restrict__ partial,
                                                            const uint32_t* __restrict__ amaxA,
                                                            const uint32_t* __restrict__ amaxB, float alpha,
                                                            float beta, float* __restrict__ C, int64_t ldc) {
  wait_prerequisite_grid();  // launched as a dependent of the GEMM
  const int64_t mq = (m + 3) / 4, total = mq * n;
  const size_t tile_elems = (size_t)128 * bn, slice_elems = (size_t)tiles_m * tiles_n * tile_elems;
  const bool c_vec = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = (t % mq) * 4, j = t / mq;
    const int64_t tm = i0 >> 7, tn = j / bn;
    const float4* p = reinterpret_cast<const float4*>(
        partial + (size_t)(tm * tiles_n + tn) * tile_elems + (size_t)(j - tn * bn) * 128 + (i0 & 127));
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s0 = 0; s0 < splitk; s0 += 8) {
      // eight slices' loads in flight, then summed in slice order
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < splitk) v[u] = __ldcs(p + (size_t)(s0 + u) * (slice_elems / 4));
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < splitk) { acc.x += v[u].x; acc.y += v[u].y; acc.z += v[u].z; acc.w += v[u].w; }
    }
    const int fj = scale_exp_from_bits(amaxB[j]);
    float* c = C + i0 + j * ldc;
    const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
    float o[4];
    if (c_vec && i0 + 3 < m) {
      const float4 cv = beta != 0.f ? *reinterpret_cast<const float4*>(c) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = scale_exp_from_bits(amaxA[i0 + q]) + fj;
        const float v = (e >= -126 && e <= 127) ? a4[q] * __int_as_float((e + 127) << 23) : scalbnf(a4[q], e);
        o[q] = (beta != 0.f) ? fmaf(alpha, v, beta * c4[q]) : alpha * v;
      }
      *reinterpret_cast<float4*>(c) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (i0 + q >= m) break;
        const int e = scale_exp_from_bits(amaxA[i0 + q]) + fj;
        const float v = (e >= -126 && e <= 127) ? a4[q] * __int_as_float((e + 127) << 23) : scalbnf(a4[q], e);
        c[q] = (beta != 0.f) ? fmaf(alpha, v, beta * c[q]) : alpha * v;
      }
    }
  }
}

// Failure-detection probe: one thread waits on an mbarrier that nothing
// arrives on and no copy is bound to, with the library's bounded wait; when
// the limit runs out it records GBGEMM_ERR_DEVICE_TIMEOUT in *status, as
// every kernel's waits do, and the CTA returns normally.
__global__ void __launch_bounds__(32) wait_probe_kernel(int* status, uint64_t timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0u, &abort_flag, timeout_ns))
    raise_status(status, &abort_flag);
  __syncwarp();
}

}  // namespace

cudaError_t launch_wait_probe(int* status, uint64_t timeout_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(status, timeout_ns);
  return cudaGetLastError();
}

int choose_splitk(int64_t tiles, int64_t k, int num_sms) {
  if (split_parts(k) != 1 || tiles <= 0 || tiles * 2 > num_sms) return 1;
  int64_t s = num_sms / tiles;                    // about one item per SM
  const int64_t max_by_k = panel_k_chunks(k) / 4; // at least 4 k chunks (128 deep) per slice
  if (s > max_by_k) s = max_by_k;
  if (s > 32) s = 32;
  if (s < 2) return 1;
  // every slice gets at least one chunk: ceil(nkc / ceil(nkc / s)) slices
  const int64_t nkc = panel_k_chunks(k), per = (nkc + s - 1) / s;
  s = (nkc + per - 1) / per;
  return s >= 2 ? (int)s : 1;
}

SplitLayout split_layout(int64_t m, int64_t n, int64_t k, int64_t batch, int splitk, int bn) {
  SplitLayout L{};
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const int64_t ra = (m + 127) / 128, rb = (n + 127) / 128;
  L.bands = (size_t)(ra + rb) * (size_t)batch;
  L.band_off = kSplitCtlBytes;
  L.amax_off = L.band_off + up(L.bands * 4);
  L.amax_stride = m + n;
  L.head = L.amax_off + up((size_t)batch * (size_t)(m + n) * 4);
  L.pa = up(panel_bytes(m, k));
  L.pb = up(panel_bytes(n, k));
  L.block = (size_t)split_parts(k) * (L.pa + L.pb);
  L.panel_off = L.head;
  L.partial_off = L.panel_off + L.block * (size_t)batch;
  const size_t tiles = (size_t)((m + 127) / 128) * (size_t)((n + bn - 1) / bn);
  L.total = L.partial_off + (splitk > 1 ? (size_t)splitk * tiles * 128 * (size_t)bn * 4 : 0);
  return L;
}

namespace {

// The scheduler of one call (or strided batch) over the workspace `ws`.
// pack_only: no tiles, only the packing of op(A)'s rows (panel inspection).
SingleSched make_single_sched(const SplitCall& c, const SplitLayout& L) {
  uint8_t* ws = static_cast<uint8_t*>(c.ws);
  SingleSched S;
  S.ctl = reinterpret_cast<WorkCtl*>(ws);
  S.band_cnt = reinterpret_cast<int*>(ws + L.band_off);
  S.A = c.A; S.B = c.B; S.lda = c.lda; S.ldb = c.ldb; S.sa = c.sa; S.sb = c.sb;
  S.ta = c.ta; S.tb = c.tb;
  S.panelA = ws + L.panel_off;
  S.panelB = ws + L.panel_off + L.pa;
  S.amaxA = reinterpret_cast<uint32_t*>(ws + L.amax_off);
  S.amaxB = S.amaxA + c.m;
  S.m = c.m; S.n = c.n; S.k = c.k;
  S.alpha = c.alpha; S.beta = c.beta;
  S.C = c.C; S.ldc = c.ldc;
  S.tiles_m = (int)((c.m + 127) / 128);
  S.tiles_n = (int)((c.n + c.bn - 1) / c.bn);
  S.nkc = (int)panel_k_chunks(c.k);
  S.raster = c.raster > 0 ? c.raster : 16;
  S.bn = c.bn;
  S.parts = split_parts(c.k);
  S.rbA = panel_row_blocks(c.m);
  S.rbB = panel_row_blocks(c.n);
  S.ra = (int)((c.m + 127) / 128);
  S.rb = (int)((c.n + 127) / 128);
  // Chunks per packing task: kPackChunks, halved (down to 1) while the
  // tasks would not give every SM three of them, so that small operands are
  // packed in one round of loads.
  const int64_t sms = c.num_sms > 0 ? c.num_sms : 148;
  S.pchunks = kPackChunks;
  while (S.pchunks > 1 && c.batch * (S.ra + S.rb) * ((S.nkc + S.pchunks - 1) / S.pchunks) < 3 * sms) S.pchunks >>= 1;
  S.ngroups = (S.nkc + S.pchunks - 1) / S.pchunks;
  // per problem [A | B | A2 | B2]: A2 - A = B2 - B = pa + pb
  S.a_part = S.parts == 2 ? (int64_t)(L.pa + L.pb) : 0;
  S.b_part = S.a_part;
  S.batch = (int)c.batch;
  S.ps = (int64_t)L.block;
  S.as = L.amax_stride;
  S.cs = c.sc;
  S.splitk = c.splitk > 1 ? c.splitk : 1;
  S.slice_chunks = (S.nkc + S.splitk - 1) / S.splitk;
  S.partial = c.splitk > 1 ? reinterpret_cast<float*>(ws + L.partial_off) : nullptr;
  S.pair = 0;
  return S;
}

}  // namespace

cudaError_t launch_split_call(const SplitCall& c, cudaStream_t s) {
  if (c.m <= 0 || c.k <= 0 || c.batch <= 0) return cudaSuccess;
  if (c.n < 0 || (c.n == 0 && !c.pack_only)) return cudaSuccess;
  if (c.bn != 64 && c.bn != 128 && c.bn != 256) return cudaErrorInvalidValue;
  if (c.batch > 65535 || !c.ws) return cudaErrorInvalidValue;
  const int splitk = c.splitk > 1 ? c.splitk : 1;
  if (splitk > 1 && (c.batch != 1 || split_parts(c.k) != 1)) return cudaErrorInvalidValue;
  const int64_t tm = (c.m + 127) / 128, tn = (c.n + c.bn - 1) / c.bn;
  const int64_t nkc = panel_k_chunks(c.k);
  const int64_t tasks = c.batch * (tm + (c.n + 127) / 128) * ((nkc + kPackChunks - 1) / kPackChunks);
  if (tm * tn * c.batch * splitk > (int64_t)0x7FFFFFFF || tasks > (int64_t)0x7FFFFFFF) return cudaErrorInvalidValue;
  const SplitLayout L = split_layout(c.m, c.n, c.k, c.batch, splitk, c.bn);
  SingleSched S = make_single_sched(c, L);
  // fewer chunks per task only below 3 tasks per SM: still far below 2^31
  const int64_t ptasks = c.batch * (int64_t)(S.ra + S.rb) * S.ngroups;
  if (c.pack_only) {
    S.tiles_n = 0;  // no tiles: the packers only
    if (c.panel_out) {
      S.panelA = static_cast<const uint8_t*>(c.panel_out);
      S.a_part = c.panel2_out ? static_cast<const uint8_t*>(c.panel2_out) - S.panelA : 0;
    }
    if (c.amax_out) S.amaxA = c.amax_out;
  }
  // no empty slice (an empty slice would store a stale accumulator)
  if ((int64_t)(S.splitk - 1) * S.slice_chunks >= S.nkc) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(c.ws, 0, L.head, s);
  if (e != cudaSuccess) return e;
  if (c.pack_only && c.amax_out) {
    e = cudaMemsetAsync(c.amax_out, 0, (size_t)c.m * 4, s);
    if (e != cudaSuccess) return e;
  }
  const int64_t items = tm * tn * c.batch * splitk;
  const int64_t sms = c.num_sms > 0 ? c.num_sms : 148;
  // packing tasks first, each its own CTA, then the GEMM
  if (ptasks > 0) pack_tasks_kernel<SingleSched><<<(unsigned)ptasks, 256, 0, s>>>(S);
  e = cudaGetLastError();
  if (e != cudaSuccess || items == 0) return e;
  const int grid = (int)(items < sms ? items : sms);
  const bool timed = c.gemm_begin && c.gemm_end;
  // Pair tiles (clusters of two CTAs, 256 x 256 tiles) for the widest tiles
  // of calls with at least two tile rows; with three-part panels (k < 512)
  // only from 8 k chunks: below that a tile's MMAs take less time than its
  // epilogue, and pairing two CTAs' epilogues (and the fixed tile order) cost
  // more than the halved operand loads gain (k = 128: 21% slower at 16384^2).
  const int64_t pair_items = (tm + 1) / 2 * tn * c.batch * splitk;
  const bool pair_ok = !c.pack_only && c.bn == 256 && tm >= 2 && (S.parts == 1 || S.nkc >= 8);
  const int pair_cap = !pair_ok ? 0
                       : S.parts == 2 ? gemm_pair_capacity<SingleSched, true>() : gemm_pair_capacity<SingleSched>();
  if (timed && (e = cudaEventRecord(c.gemm_begin, s)) != cudaSuccess) return e;
  if (pair_cap > 0) {
    S.pair = 1;
    const int pairs = (int)(pair_items < pair_cap ? pair_items : pair_cap);
    e = S.parts == 2 ? launch_gemm_kernel_pair<SingleSched, true>(S, pairs, c.status, s, ptasks > 0 && !timed)
                     : launch_gemm_kernel_pair<SingleSched>(S, pairs, c.status, s, ptasks > 0 && !timed);
  } else {
    e = launch_gemm_kernel<SingleSched>(S, grid, c.status, s, ptasks > 0 && !timed);
  }
  if (e != cudaSuccess) return e;
  if (timed && (e = cudaEventRecord(c.gemm_end, s)) != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess || splitk == 1 || c.pack_only) return e;
  SplitGemmArgs a;
  a.m = c.m; a.n = c.n; a.k = c.k; a.alpha = c.alpha; a.beta = c.beta; a.C = c.C; a.ldc = c.ldc;
  a.amaxA = S.amaxA; a.amaxB = S.amaxB; a.num_sms = c.num_sms; a.bn = c.bn; a.splitk = splitk;
  a.partial = S.partial;
  return launch_splitk_reduce(a, s);
}

cudaError_t launch_splitk_reduce(const SplitGemmArgs& a, cudaStream_t s) {
  if (a.m <= 0 || a.n <= 0 || a.splitk <= 1) return cudaSuccess;
  const int tm = (int)((a.m + 127) / 128), tn = (int)((a.n + a.bn - 1) / a.bn);
  const int64_t total = (a.m + 3) / 4 * a.n;  // a thread per four rows of a column
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)(a.num_sms > 0 ? a.num_sms : 148) * 16;
  if (blocks > cap) blocks = cap;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, splitk_reduce_kernel, a.m, a.n, a.bn, tm, tn, a.splitk, (const float*)a.partial,
                            a.amaxA, a.amaxB, a.alpha, a.beta, a.C, a.ldc);
}

}  // namespace gbg
