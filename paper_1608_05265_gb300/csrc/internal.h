// Internal declarations shared by the gbgemm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbgemm.h"

namespace gbg {

// Problem after argument checks; op letters reduced to 0 (N) / 1 (T).
struct Problem {
  int ta, tb;
  int64_t m, n, k;
  float alpha, beta;
  const float* A; int64_t lda;
  const float* B; int64_t ldb;
  float* C; int64_t ldc;
};

// ---- SIMT path (simt.cu) ----
// Tile configurations of the SIMT kernel, indexed by the autotuner.
enum SimtConfig { SIMT_128x128 = 0, SIMT_64x64 = 1, SIMT_128x64 = 2, SIMT_NUM_CONFIGS = 3 };
cudaError_t launch_simt(const Problem& p, int config, cudaStream_t s);
// A strided batch of equal problems (batch <= 65535): problem z reads
// A + z*sa, B + z*sb and writes C + z*sc.
cudaError_t launch_simt_batched(const Problem& p, int config, int64_t batch, int64_t sa, int64_t sb, int64_t sc,
                                cudaStream_t s);
// C := beta * C over m x n (beta == 0 writes zeros without reading C).
cudaError_t launch_scale_c(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t s);
// sgemv (gemv.cu): slices of the summed dimension for a launch (>= 1), and the
// launch (partial: slices x len(y) floats when slices > 1).
int64_t gemv_slices(bool trans, int64_t m, int64_t n, int num_sms);
cudaError_t launch_gemv(bool trans, int64_t m, int64_t n, float alpha, const float* A, int64_t lda, const float* x,
                        int64_t incx, float beta, float* y, int64_t incy, int64_t slices, float* partial,
                        int num_sms, cudaStream_t s);
cudaError_t launch_scale_c_batched(int64_t m, int64_t n, float beta, float* C, int64_t ldc, int64_t batch,
                                   int64_t sc, cudaStream_t s);

// ---- LU factorisation (lu.cu) ----
constexpr int kLuMaxNb = GBGEMM_SGETRF_MAX_NB;  // widest panel
constexpr int kLuSolveSmemN = 32768; // the row exchanges of the solve run in shared memory up to this n
constexpr int kLuPermInts = 1 + 3 * kLuMaxNb;  // a block's row permutation (the handle holds two)
constexpr int kLuPanelNb = 32;      // columns per panel inside a block
// Factor the panel rows [j0, n) x columns [j0, j0 + nbp) in place (a
// cluster of up to kLuPanelCluster blocks holding the panel in shared
// memory), writing ipiv[j0 ..) (1-based), the first zero pivot into *info
// (when *info is 0) and the panel's row permutation into perm; a wait between
// the cluster's blocks that runs out sets *status.  nbp must not
// exceed lu_panel_width(n - j0), the widest panel whose rows fit.
constexpr int kLuPanelCluster = 16;  // largest cluster (8 is the portable size)
constexpr int kLuPanelSlabBytes = 192 * 1024;
int lu_panel_width(int rows);
// With jp >= 0 the panel first applies the previous block [jp, j0) (nbq
// columns, its row permutation in perm_prev, its L factors final) to its own
// columns: the exchanges, U12 = L11^-1 A12 (written to rows [jp, j0)) and
// A22 -= L21 U12 for the panel rows.
cudaError_t launch_lu_panel(int n, float* A, int64_t lda, int j0, int nbp, int* ipiv, int* info, int* perm,
                            int* status, cudaStream_t s, int jp = -1, int nbq = 0, const int* perm_prev = nullptr);
// The permutation of pivot rows [j0, j0 + nbp), rebuilt from ipiv (for a
// block factored as several panels).
cudaError_t launch_lu_perm(int j0, int nbp, const int* ipiv, int* perm, cudaStream_t s);
// The permutation of pivot rows [j0, j0 + nbp) applied to columns [c_lo, j0)
// and [r_lo, c_hi) (r_lo < 0: j0 + nbp), then U12 = L11^-1 A12 for the latter.
cudaError_t launch_lu_swap_trsm(int n, float* A, int64_t lda, int j0, int nbp, const int* perm, int c_lo, int c_hi,
                                cudaStream_t s, int r_lo = -1);
// The solve with the packed factors: the row exchanges of ipiv on each of
// nrhs columns of B, then per diagonal block of kSolveBlock rows the
// triangular solve of that block (UPPER: back substitution with U, else
// forward with unit L); the off-diagonal updates are gemv/gemm calls.
constexpr int kSolveBlock = 256;
cudaError_t launch_lu_laswp_rhs(int n, int64_t nrhs, const int* ipiv, float* B, int64_t ldb, cudaStream_t s);
cudaError_t launch_lu_trsv_block(bool upper, const float* LU, int64_t lda, int j0, int w, int64_t nrhs, float* B,
                                 int64_t ldb, cudaStream_t s);
// One right-hand side: the whole forward (or back) substitution as one
// cooperative launch; flags: ceil(n / kSolveBlock) ints of scratch (zeroed
// here); a wait between CTAs that runs out sets *status.
cudaError_t launch_lu_trsv_sweep(bool upper, int n, const float* LU, int64_t lda, float* x, int* flags, int* status,
                                 int num_sms, cudaStream_t s);

// ---- split path (split.cu) ----
constexpr int kPanelRows = 128;     // rows per panel block
constexpr int kPanelK = 32;         // k per panel block (hi and lo: 64 BF16 = 128 bytes per row)
constexpr int kBlockBytes = kPanelRows * 128;  // 16 KiB
constexpr int kSplitCtlBytes = 256; // per-launch control words of the fused split GEMM
constexpr int kSplitMinK = 128;     // AUTO uses the split path from this k upwards
constexpr int kSplitShortK = 16;    // the split path holds the bound from this k (grouped configurations)
constexpr int kSplitTwoPartK = 512; // from this k two BF16 parts (3 products) meet the bound; below, three parts (6 products)

// Number of panel parts of the split path for a given k: 1 ([hi | lo]) or 2 ([hi | mid] and compact lo3).
inline int split_parts(int64_t k) { return k < kSplitTwoPartK ? 2 : 1; }

inline int64_t panel_row_blocks(int64_t rows) { return (rows + 255) / 256 * 2; }
inline int64_t panel_k_chunks(int64_t k) { return (k + kPanelK - 1) / kPanelK; }
inline size_t panel_bytes(int64_t rows, int64_t k) {
  return (size_t)panel_row_blocks(rows) * (size_t)panel_k_chunks(k) * (size_t)kBlockBytes;
}

// Workspace of one split-path call (or strided batch), in bytes from its
// start: [control words | band counters | row maxima | per problem: panel A,
// panel B (and with three parts the compact lo3 panels A2, B2) | split-K
// partials].  The head (control words, band counters, maxima) is zeroed
// before every launch.
struct SplitLayout {
  size_t bands;           // band counters
  size_t band_off, amax_off, head;
  int64_t amax_stride;    // words between problems' maxima (m + n; op(B)'s follow op(A)'s)
  size_t pa, pb, block;   // panel bytes of op(A), op(B), and per problem
  size_t panel_off, partial_off, total;
};
SplitLayout split_layout(int64_t m, int64_t n, int64_t k, int64_t batch, int splitk, int bn);


// One split-path call: the packing launch, then the persistent tcgen05 GEMM.
struct SplitCall {
  int ta = 0, tb = 0;
  int64_t m = 0, n = 0, k = 0;
  float alpha = 1.f, beta = 0.f;
  const float* A = nullptr; int64_t lda = 1;
  const float* B = nullptr; int64_t ldb = 1;
  float* C = nullptr; int64_t ldc = 1;
  int64_t batch = 1, sa = 0, sb = 0, sc = 0;  // strided batch: problem z at A + z*sa, B + z*sb, C + z*sc
  int bn = 256;          // tile width: 64, 128 or 256
  int raster = 16;       // tile rows per group of the tile order
  int splitk = 1;        // k slices (batch 1, k >= kSplitTwoPartK)
  void* ws = nullptr;    // split_layout(...).total bytes
  int* status = nullptr;
  int num_sms = 0;
  // panel inspection: pack op(A)'s rows only, into these caller buffers
  bool pack_only = false;
  void* panel_out = nullptr;
  void* panel2_out = nullptr;
  uint32_t* amax_out = nullptr;
  // profiling: when set, recorded on the stream around the GEMM launch alone
  // (the GEMM is then launched as a plain launch, not as a programmatic
  // dependent of the packing, so the pair brackets the GEMM only)
  cudaEvent_t gemm_begin = nullptr, gemm_end = nullptr;
};
// Zero the workspace head, pack both operands, run the GEMM (and the split-K
// reduction).
cudaError_t launch_split_call(const SplitCall& c, cudaStream_t s);

struct SplitGemmArgs {
  const uint32_t* amaxA; const uint32_t* amaxB;
  int64_t m, n, k;
  float alpha, beta;
  float* C; int64_t ldc;
  int num_sms;
  int bn;
  int splitk = 1;
  float* partial = nullptr;
};

// Number of k slices for a single split-path call with `tiles` output tiles
// (1 when the tiles already fill half of the SMs, or k is short).
int choose_splitk(int64_t tiles, int64_t k, int num_sms);
// C := alpha 2^(e_i + f_j) sum_s partial_s + beta C, slices summed in order.
cudaError_t launch_splitk_reduce(const SplitGemmArgs& a, cudaStream_t s);

// Failure-detection probe: a bounded mbarrier wait that nothing completes;
// sets *status to GBGEMM_ERR_DEVICE_TIMEOUT after timeout_ns.
cudaError_t launch_wait_probe(int* status, uint64_t timeout_ns, cudaStream_t s);

// FP64 error check of C_out against alpha op(A) op(B) + beta C_in over a
// block (check.cu); synchronises s.
int run_error_check(cudaStream_t s, char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                    const float* A, int64_t lda, const float* B, int64_t ldb, float beta, const float* C_in,
                    const float* C_out, int64_t ldc, int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                    double* max_ratio);


// ---- single-call schedules (gbgemm_schedule_info) ----
struct Schedule {
  int path;      // GBGEMM_PATH_SIMT or GBGEMM_PATH_SPLIT_BF16
  int simt_cfg;  // SimtConfig (SIMT path)
  int bn;        // tile columns (split path)
  int raster;    // tile rows per group of the tile order (split path)
  int level;     // k-slicing level 0..3 (split path): S = 1, F/4, F/2, F
  int splitk;    // k slices once resolved for a problem (schedule_resolve); 1 before
};
inline bool schedule_decode(int s, Schedule* o) {
  if (s < 0 || s >= GBGEMM_NUM_SCHEDULES) return false;
  if (s < SIMT_NUM_CONFIGS) {
    *o = Schedule{GBGEMM_PATH_SIMT, s, 0, 0, 0, 1};
    return true;
  }
  const int t = s - SIMT_NUM_CONFIGS, b = t / 12, r = (t / 4) % 3, q = t % 4;
  *o = Schedule{GBGEMM_PATH_SPLIT_BF16, -1, 64 << b, r == 0 ? 1 : (r == 1 ? 4 : 16), q, 1};
  return true;
}
inline int schedule_encode_split(int bn, int raster, int level) {
  const int b = bn == 64 ? 0 : (bn == 128 ? 1 : 2);
  const int r = raster == 1 ? 0 : (raster == 4 ? 1 : 2);
  return SIMT_NUM_CONFIGS + 12 * b + 4 * r + level;
}
// k slices of k-slicing level `level` for an m x n x k problem with tiles of
// 128 x bn: F = choose_splitk (the slices that give about one item per SM,
// 1 when the output already fills half the SMs or k is short), S = F >> (3 -
// level) rounded down to a count without an empty slice; 0 when the level
// gives fewer than 2 slices or the same count as the level below.
inline int schedule_slices(int64_t m, int64_t n, int64_t k, int bn, int level, int num_sms) {
  if (level <= 0) return 1;
  const int64_t tiles = ((m + 127) / 128) * ((n + bn - 1) / bn);
  const int F = choose_splitk(tiles, k, num_sms);
  int S = F >> (3 - level);
  if (F < 2 || S < 2) return 0;
  const int64_t nkc = panel_k_chunks(k), per = (nkc + S - 1) / S;
  S = (int)((nkc + per - 1) / per);
  if (S < 2) return 0;
  if (level > 1 && schedule_slices(m, n, k, bn, level - 1, num_sms) == S) return 0;
  return S;
}
// Legality of schedule s for one problem (m, n, k, alpha) on num_sms SMs.
inline bool schedule_legal(int64_t m, int64_t n, int64_t k, float alpha, int s, int num_sms) {
  Schedule d;
  if (!schedule_decode(s, &d)) return false;
  if (d.path == GBGEMM_PATH_SIMT) return true;
  if (k < kSplitShortK || alpha == 0.0f) return false;
  return d.level == 0 || schedule_slices(m, n, k, d.bn, d.level, num_sms) >= 2;
}
// Decode s and resolve its k slices for a problem (false when s is illegal for it).
inline bool schedule_resolve(int s, int64_t m, int64_t n, int64_t k, float alpha, int num_sms, Schedule* o) {
  if (!schedule_legal(m, n, k, alpha, s, num_sms) || !schedule_decode(s, o)) return false;
  if (o->path == GBGEMM_PATH_SPLIT_BF16) o->splitk = schedule_slices(m, n, k, o->bn, o->level, num_sms);
  return true;
}

}  // namespace gbg
