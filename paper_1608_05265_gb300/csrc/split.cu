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

// blockIdx.z selects the problem of a strided batch: its operand at
// X + z*xs, its row maxima at amax + z*as, its panels at panel(2) + z*ps.
template <bool KCONTIG>
__global__ void __launch_bounds__(256) pack_kernel(int64_t rows, int64_t k, const float* __restrict__ X, int64_t ld,
                                                   uint32_t* __restrict__ amax, uint8_t* __restrict__ panel,
                                                   uint8_t* __restrict__ panel2, int64_t rows_alloc, int64_t xs,
                                                   int64_t as, int64_t ps) {
  __shared__ uint32_t smax[128];
  const int64_t z = blockIdx.z;
  pack_block<KCONTIG>(rows, k, X + z * xs, ld, amax + z * as, panel + z * ps, panel2 ? panel2 + z * ps : nullptr,
                      rows_alloc, blockIdx.x, blockIdx.y, smax);
}

__global__ void __launch_bounds__(256) rescale_kernel(int64_t rows, int64_t k, const float* __restrict__ X, int64_t ld,
                                                      bool kcontig, const uint32_t* __restrict__ amax,
                                                      uint8_t* __restrict__ panel, uint8_t* __restrict__ panel2,
                                                      int64_t rows_alloc, int64_t nkc, int64_t xs, int64_t as,
                                                      int64_t ps) {
  __shared__ int se[128];
  const int64_t z = blockIdx.z;
  rescale_block(rows, k, X + z * xs, ld, kcontig, amax + z * as, panel + z * ps, panel2 ? panel2 + z * ps : nullptr,
                rows_alloc, nkc, blockIdx.x, se);
}

// Split-K reduction: thread per C element (i, j), the slices' raw
// accumulators summed in slice order (deterministic), then the epilogue of
// split_gemm_kernel: x 2^(e_i + f_j), alpha, and beta C with one rounding of
// beta C and one fused multiply-add.
__global__ void __launch_bounds__(256) splitk_reduce_kernel(int64_t m, int64_t n, int bn, int tiles_m, int tiles_n,
                                                            int splitk, const float* __restrict__ partial,
                                                            const uint32_t* __restrict__ amaxA,
                                                            const uint32_t* __restrict__ amaxB, float alpha,
                                                            float beta, float* __restrict__ C, int64_t ldc) {
  const int64_t total = m * n;
  const size_t tile_elems = (size_t)128 * bn, slice_elems = (size_t)tiles_m * tiles_n * tile_elems;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % m, j = t / m;
    const int64_t tm = i >> 7, tn = j / bn;
    const float* p = partial + (size_t)(tm * tiles_n + tn) * tile_elems + (size_t)(j - tn * bn) * 128 + (i & 127);
    float acc = 0.f;
    for (int s = 0; s < splitk; ++s) acc += p[(size_t)s * slice_elems];
    const int e = scale_exp_from_bits(amaxA[i]) + scale_exp_from_bits(amaxB[j]);
    const float v = (e >= -126 && e <= 127) ? acc * __int_as_float((e + 127) << 23) : scalbnf(acc, e);
    float* c = C + i + j * ldc;
    *c = (beta != 0.f) ? fmaf(alpha, v, beta * *c) : alpha * v;
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

cudaError_t launch_split_pack(int64_t rows, int64_t k, const float* X, int64_t ld, bool kcontig,
                              uint32_t* amax_bits, void* panel, void* panel2, cudaStream_t s) {
  return launch_split_pack_batched(rows, k, X, ld, kcontig, amax_bits, panel, panel2, 1, 0, 0, 0, s);
}

cudaError_t launch_split_pack_batched(int64_t rows, int64_t k, const float* X, int64_t ld, bool kcontig,
                                      uint32_t* amax_bits, void* panel, void* panel2, int64_t batch, int64_t xs,
                                      int64_t as, int64_t ps, cudaStream_t s) {
  if (rows <= 0 || k <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidConfiguration;
  if (batch > 1 && as < rows) return cudaErrorInvalidValue;
  // every problem's row maxima start at zero (they sit between its panels)
  cudaError_t e = batch == 1 ? cudaMemsetAsync(amax_bits, 0, (size_t)rows * sizeof(uint32_t), s)
                             : cudaMemset2DAsync(amax_bits, (size_t)as * sizeof(uint32_t), 0,
                                                 (size_t)rows * sizeof(uint32_t), (size_t)batch, s);
  if (e != cudaSuccess) return e;
  const int64_t rbc = panel_row_blocks(rows);
  const int64_t nkc = panel_k_chunks(k);
  dim3 g((unsigned)rbc, (unsigned)nkc, (unsigned)batch);
  if (g.y > 65535u) return cudaErrorInvalidConfiguration;
  uint8_t* pn = static_cast<uint8_t*>(panel);
  uint8_t* pn2 = split_parts(k) == 2 ? static_cast<uint8_t*>(panel2) : nullptr;
  if (split_parts(k) == 2 && !pn2) return cudaErrorInvalidValue;
  if (kcontig) pack_kernel<true><<<g, 256, 0, s>>>(rows, k, X, ld, amax_bits, pn, pn2, rbc * 128, xs, as, ps);
  else pack_kernel<false><<<g, 256, 0, s>>>(rows, k, X, ld, amax_bits, pn, pn2, rbc * 128, xs, as, ps);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rescale_kernel<<<dim3((unsigned)rbc, 1, (unsigned)batch), 256, 0, s>>>(rows, k, X, ld, kcontig, amax_bits, pn, pn2,
                                                                         rbc * 128, nkc, xs, as, ps);
  return cudaGetLastError();
}

cudaError_t launch_split_gemm(const SplitGemmArgs& a, cudaStream_t s) {
  if (a.m <= 0 || a.n <= 0 || a.k <= 0) return cudaSuccess;
  if (a.bn != 64 && a.bn != 128 && a.bn != 256) return cudaErrorInvalidValue;
  const int64_t tm = (a.m + 127) / 128, tn = (a.n + a.bn - 1) / a.bn;
  const int64_t batch = a.batch > 0 ? a.batch : 1;
  if (tm * tn * batch > (int64_t)0x7FFFFFFF || panel_k_chunks(a.k) > (int64_t)0x7FFFFFFF) return cudaErrorInvalidValue;
  SingleSched S;
  S.panelA = static_cast<const uint8_t*>(a.panelA);
  S.panelB = static_cast<const uint8_t*>(a.panelB);
  S.amaxA = a.amaxA; S.amaxB = a.amaxB;
  S.m = a.m; S.n = a.n;
  S.alpha = a.alpha; S.beta = a.beta;
  S.C = a.C; S.ldc = a.ldc;
  S.tiles_m = (int)tm; S.tiles_n = (int)tn;
  S.nkc = (int)panel_k_chunks(a.k);
  S.raster = a.raster > 0 ? a.raster : 16;
  S.bn = a.bn;
  S.rbA = panel_row_blocks(a.m);
  S.rbB = panel_row_blocks(a.n);
  S.parts = split_parts(a.k);
  if (S.parts == 2 && (!a.panelA2 || !a.panelB2)) return cudaErrorInvalidValue;
  S.a_part = S.parts == 2 ? (size_t)(static_cast<const uint8_t*>(a.panelA2) - S.panelA) : 0;
  S.b_part = S.parts == 2 ? (size_t)(static_cast<const uint8_t*>(a.panelB2) - S.panelB) : 0;
  S.batch = (int)batch;
  S.ps = a.panel_stride; S.as = a.amax_stride; S.cs = a.c_stride;
  S.splitk = a.splitk > 1 ? a.splitk : 1;
  if (S.splitk > 1 && (batch != 1 || S.parts != 1 || !a.partial)) return cudaErrorInvalidValue;
  S.slice_chunks = (S.nkc + S.splitk - 1) / S.splitk;
  // no empty slice (an empty slice would store a stale accumulator)
  if ((int64_t)(S.splitk - 1) * S.slice_chunks >= S.nkc) return cudaErrorInvalidValue;
  S.partial = a.partial;
  cudaError_t e = ensure_gemm_smem_attr<SingleSched>();
  if (e != cudaSuccess) return e;
  const int64_t tiles = tm * tn * batch * S.splitk;
  const int64_t sms = a.num_sms > 0 ? a.num_sms : 148;
  const int grid = (int)(tiles < sms ? tiles : sms);
  split_gemm_kernel<SingleSched><<<grid, kGemmThreads, kGemmSmemBytes, s>>>(S, a.status, kTimeoutNs);
  return cudaGetLastError();
}

cudaError_t launch_splitk_reduce(const SplitGemmArgs& a, cudaStream_t s) {
  if (a.m <= 0 || a.n <= 0 || a.splitk <= 1) return cudaSuccess;
  const int tm = (int)((a.m + 127) / 128), tn = (int)((a.n + a.bn - 1) / a.bn);
  const int64_t total = a.m * a.n;
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)(a.num_sms > 0 ? a.num_sms : 148) * 8;
  if (blocks > cap) blocks = cap;
  splitk_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(a.m, a.n, a.bn, tm, tn, a.splitk, a.partial, a.amaxA,
                                                         a.amaxB, a.alpha, a.beta, a.C, a.ldc);
  return cudaGetLastError();
}

}  // namespace gbg
