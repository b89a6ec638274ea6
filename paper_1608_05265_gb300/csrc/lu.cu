// FP32 LU factorisation with partial pivoting, and the solve that follows it:
// the HPL run of the paper (Section IV-C, Table VII) on one GPU, with the
// library's own sgemm doing the trailing updates (the Linpack-shaped
// C := C - A B of the benchmark).
//
// Right-looking, blocked by nb columns; each block is factored as panels of
// at most 32 columns:
//   panel    rows [j1, n) x the panel's columns, held in the shared memory
//            of a cluster of up to 16 blocks for the whole factorisation
//            (lu_panel_kernel): per column a block argmax, one exchange of
//            candidates between the blocks (remote stores completing on the
//            receivers' mbarriers), the pivot (first row of largest |a|)
//            chosen identically in every block, the exchange and the rank-1
//            update done locally.  The panel's exchanges are written out as
//            a permutation of the rows they touch.  When every block is one
//            panel, the kernel first applies the previous block to its own
//            columns (a prologue: exchanges, U12, update).
//   swap+U12 the other columns get that permutation (one gather per column:
//            all sources read before any row is written), and right of the
//            panel U12 = L11^-1 A12 is solved in shared memory
//            (lu_swap_trsm_kernel); the block columns right of a panel are
//            updated by the SIMT sgemm.
//   block    the block's exchanges, rebuilt as one permutation
//            (lu_perm_kernel), reach every column outside the block, U12 of
//            the block rows is solved, and the trailing matrix is updated by
//            the library's sgemm with k = nb; the next block is factored on
//            a second stream meanwhile (look-ahead).
// The result is LAPACK's packed P A = L U.  The solve (lu_laswp_rhs_kernel,
// lu_trsv_block_kernel) applies the exchanges, then forward and back
// substitution by 256-row diagonal blocks (each triangle staged in shared
// memory), the off-diagonal parts by the library's sgemv or sgemm.  Every
// sum is formed in a fixed order: runs are bit-identical.
#include <cfloat>
#include <climits>

#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace gbg {
namespace {

constexpr int kPanelThreads = 512;  // per block of the panel's cluster
constexpr int kPushLanes = 1 + 2 * (kLuPanelNb / 4);  // lanes sending to one block: candidate, its row, row q
static_assert(kPanelThreads == 32 * kLuPanelCluster && kPushLanes <= 30,
              "a warp per destination block; the last two threads (lanes 30, 31 of the last warp) never push");
constexpr int kTrsmCols = 64;     // columns per block of the swap + triangular solve kernel
constexpr int kSwapThreads = 256;  // its threads (the first kTrsmCols solve one column each)
constexpr int kXP = kTrsmCols + 1;
constexpr int kSweepThreads = 512;  // cooperative triangular solve: two thread groups per row block

struct MaxLoc {
  float v;
  int i;
};

__device__ __forceinline__ void maxloc_merge(float& v, int& i, float v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

// Largest v over the block (smallest i on ties), returned to every thread:
// each warp reduces its lanes, then every warp reduces the per-warp results
// itself (one barrier, no broadcast).  Callers alternate between two `red`
// buffers, so no closing barrier is needed.
__device__ __forceinline__ MaxLoc block_argmax(float v, int i, MaxLoc* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxloc_merge(v, i, __shfl_xor_sync(0xFFFFFFFFu, v, o), __shfl_xor_sync(0xFFFFFFFFu, i, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = MaxLoc{v, i};
  __syncthreads();
  MaxLoc m = lane < (int)(blockDim.x >> 5) ? red[lane] : MaxLoc{-1.f, INT_MAX};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    maxloc_merge(m.v, m.i, __shfl_xor_sync(0xFFFFFFFFu, m.v, o), __shfl_xor_sync(0xFFFFFFFFu, m.i, o));
  return m;
}

// The exchanges of pivot rows [j0, j0 + nbp) (row j0 + q with piv[q],
// 0-based, q ascending) as a permutation of the rows they touch: slot s holds
// row prow[s] and receives the original row pcont[s].  Slots 0 .. nbp-1 are
// rows j0 ..; rows below that an exchange touches get slots after them.  Run
// by one full warp, serial in q.  Writes perm = [extras, source row of row
// j0 + q (nbp), (row, source) per extra].
__device__ void build_perm(int j0, int nbp, const int* piv, int* prow, int* pcont, int* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  for (int s = lane; s < nbp; s += 32) prow[s] = pcont[s] = j0 + s;
  __syncwarp();
  int next = nbp;
  for (int q = 0; q < nbp; ++q) {
    const int p = piv[q];
    if (p == j0 + q) continue;
    int slot = -1;
    if (p < j0 + nbp) {
      slot = p - j0;
    } else {
      for (int base = nbp; base < next && slot < 0; base += 32) {
        const unsigned hit = __ballot_sync(0xFFFFFFFFu, base + lane < next && prow[base + lane] == p);
        if (hit) slot = base + __ffs(hit) - 1;
      }
      if (slot < 0) {
        slot = next++;
        if (lane == 0) prow[slot] = pcont[slot] = p;
      }
    }
    __syncwarp();
    if (lane == 0) {
      const int t = pcont[q];
      pcont[q] = pcont[slot];
      pcont[slot] = t;
    }
    __syncwarp();
  }
  for (int s = lane; s < nbp; s += 32) perm[1 + s] = pcont[s];
  for (int s = nbp + lane; s < next; s += 32) {
    perm[1 + nbp + 2 * (s - nbp)] = prow[s];
    perm[2 + nbp + 2 * (s - nbp)] = pcont[s];
  }
  if (lane == 0) perm[0] = next - nbp;
}

// The permutation of pivot rows [j0, j0 + nbp) from ipiv (one warp).
__global__ void lu_perm_kernel(int j0, int nbp, const int* __restrict__ ipiv, int* __restrict__ perm) {
  __shared__ int piv[kLuMaxNb];
  __shared__ int prow[2 * kLuMaxNb], pcont[2 * kLuMaxNb];
  for (int q = threadIdx.x; q < nbp; q += 32) piv[q] = ipiv[j0 + q] - 1;
  __syncwarp();
  build_perm(j0, nbp, piv, prow, pcont, perm);
}

// PTX helpers of the panel's exchange between the blocks of a cluster.
__device__ __forceinline__ uint32_t lu_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t lu_mapa(uint32_t a, int rank) {  // the same variable in block `rank`
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Remote store into block `rank`'s shared memory that completes its bytes on
// that block's mbarrier.
__device__ __forceinline__ void lu_push4(uint32_t raddr, float4 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               ::"r"(raddr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar) : "memory");
}
__device__ __forceinline__ void lu_push1(uint32_t raddr, float v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];"
               ::"r"(raddr), "f"(v), "r"(rbar) : "memory");
}
__device__ __forceinline__ void lu_push2(uint32_t raddr, uint32_t a, uint32_t b, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.u32 [%0], {%1, %2}, [%3];"
               ::"r"(raddr), "r"(a), "r"(b), "r"(rbar) : "memory");
}
__device__ __forceinline__ void lu_mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void lu_mbar_arm(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool lu_mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Wait for the phase of parity `parity`; false after 2 s of %globaltimer.
__device__ __noinline__ bool lu_mbar_wait(uint32_t bar, uint32_t parity) {
  if (lu_mbar_try(bar, parity)) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t it = 1;; ++it) {
    if (lu_mbar_try(bar, parity)) return true;
    if ((it & 63u) == 0u) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) return false;
    }
  }
}

// Panel rows [j0, n) x columns [j0, j0 + nbp) (nbp <= 32), resident in the
// shared memory of a cluster of C blocks for the whole factorisation: block c
// holds panel rows [c RS, c RS + RS) (counted from j0), row-major, row rr at
// Sp + rr * pitch (lu_slab_pitch: rows of 16-byte multiples whose quarter
// warps touch distinct banks).  Per column q:
//   every block finds its candidate (largest |a| in column q among its rows
//   below q, the first such row on ties; tracked during the previous
//   column's update) and pushes it, with the candidate's row and, from the
//   block holding it, row q, into every block's receive buffers with remote
//   stores that complete bytes on the receiver's mbarrier;
//   each block waits on its own mbarrier (no cluster-wide barrier), reduces
//   the C candidates in the same order to the pivot row p, and takes its
//   values from its buffers.  The block holding q writes the pivot row
//   there; the thread holding row p writes row q's values into it while it
//   updates it; every block scales its rows below q by the pivot's
//   reciprocal (as LAPACK's unblocked factorisation and HPL scale; by the
//   pivot itself when the reciprocal would overflow) and updates the rest of
//   them: a row's values are loaded as float4 before any is stored, and the
//   pivot row is held in registers.
// The receive buffers and their mbarriers alternate with the parity of q.  A
// buffer is refilled for column q + 2 only by a block that has received
// every block's column q + 1 values, which each block sends after it has
// finished column q: no buffer is overwritten before it has been read.  A
// wait that runs out (2 s) sets *status, and the block stops factoring but
// still reaches the final cluster barrier, so no block leaves while another
// may still write to it.
__global__ void __launch_bounds__(kPanelThreads, 1)
    lu_panel_kernel(int n, float* __restrict__ A, int64_t lda, int j0, int nbp, int RS, int pitch,
                    int* __restrict__ ipiv, int* __restrict__ info, int* __restrict__ perm, int* __restrict__ status,
                    int jp, int nbq, const int* __restrict__ perm_prev) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int c = (int)cl.block_rank();
  extern __shared__ float4 Sp4[];
  float* Sp = reinterpret_cast<float*>(Sp4);
  __shared__ MaxLoc red[2][33];
  __shared__ __align__(8) MaxLoc rx_cand[2][kLuPanelCluster];               // from each block
  // rows received: each block's candidate row, then (slot kLuPanelCluster) row q
  __shared__ __align__(16) float rx_row[2][kLuPanelCluster + 1][kLuPanelNb];
  __shared__ __align__(8) uint64_t rx_bar[2];
  __shared__ int piv_s[kLuPanelNb];
  __shared__ int prow_s[2 * kLuPanelNb], pcont_s[2 * kLuPanelNb];
  __shared__ __align__(16) float Ux[kLuPanelNb][kLuPanelNb];      // prologue: U12 of this panel's columns
  __shared__ float Lx[kLuPanelNb][kLuPanelNb + 1];                 // prologue: the previous block's L11
  const int tid = threadIdx.x;
  const int R = n - j0;
  const int rlo = c * RS;
  const int nr = max(0, min(R, rlo + RS) - rlo);  // rows of this block's slab
  const bool vec = nbp > 2;                       // rows in float4 groups
  const int groups = (nbp + 3) / 4;
  const int row_bytes = vec ? 16 * groups : 4 * nbp;
  // bytes other blocks push for column q: a candidate and its row from each,
  // and row q unless this block holds it (a block writes its own values
  // into its buffers with plain stores)
  auto rx_bytes = [&](int q) -> uint32_t {
    return (uint32_t)((C - 1) * (8 + row_bytes) + (q / RS == c ? 0 : row_bytes));
  };
  float* G = A + j0 + (int64_t)j0 * lda;
  if (tid == 0) {
    lu_mbar_init(lu_smem(&rx_bar[0]));
    lu_mbar_init(lu_smem(&rx_bar[1]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    lu_mbar_arm(lu_smem(&rx_bar[0]), rx_bytes(0));
    if (nbp > 1) lu_mbar_arm(lu_smem(&rx_bar[1]), rx_bytes(1));
  }
  for (int rr = tid; rr < nr; rr += kPanelThreads) {  // a row per thread: its loads all in flight, then stored
    float v[kLuPanelNb];
#pragma unroll
    for (int q = 0; q < kLuPanelNb; ++q)
      if (q < nbp) v[q] = G[(rlo + rr) + (int64_t)q * lda];
#pragma unroll
    for (int q = 0; q < kLuPanelNb; ++q)
      if (q < nbp) Sp[rr * pitch + q] = v[q];
  }
  if (jp >= 0) {
    // Prologue: the previous block [jp, j0) (nbq columns, its exchanges in
    // perm_prev) has not yet touched this panel's columns.  (a) Slab rows
    // that its exchanges replaced take their new values; (b) every block
    // solves U12 = L11^-1 (the block's rows, exchanged) for this panel's
    // columns; (c) the slab rows get A -= L21 U12.  Only original values of
    // A are read here; U12 is written back after the cluster barrier below.
    const int nx = perm_prev[0];
    const int* psrc = perm_prev + 1;
    const int* pext = perm_prev + 1 + nbq;
    __syncthreads();
    for (int e = tid; e < nx * nbp; e += kPanelThreads) {
      const int x = e / nbp, k = e % nbp;
      const int r = pext[2 * x] - j0 - rlo;
      if (r >= 0 && r < nr) Sp[r * pitch + k] = A[pext[2 * x + 1] + (int64_t)(j0 + k) * lda];
    }
    for (int e = tid; e < nbq * kLuPanelNb; e += kPanelThreads) {
      const int qq = e / kLuPanelNb, k = e % kLuPanelNb;
      Ux[qq][k] = k < nbp ? A[psrc[qq] + (int64_t)(j0 + k) * lda] : 0.f;
    }
    for (int e = tid; e < nbq * nbq; e += kPanelThreads) {
      const int i = e % nbq, p2 = e / nbq;
      Lx[i][p2] = A[(jp + i) + (int64_t)(jp + p2) * lda];
    }
    __syncthreads();
    if (tid < nbp)  // one thread per column, rows in order (unit lower L11)
      for (int i = 1; i < nbq; ++i) {
        float acc = Ux[i][tid];
        for (int p2 = 0; p2 < i; ++p2) acc = fmaf(-Lx[i][p2], Ux[p2][tid], acc);
        Ux[i][tid] = acc;
      }
    __syncthreads();
    for (int rr = tid; rr < nr; rr += kPanelThreads) {
      const float* lrow = A + (j0 + rlo + rr) + (int64_t)jp * lda;  // L21, row j0 + rlo + rr
      float l[kLuPanelNb];
#pragma unroll
      for (int qq = 0; qq < kLuPanelNb; ++qq) l[qq] = qq < nbq ? lrow[(int64_t)qq * lda] : 0.f;
      float* row = Sp + rr * pitch;
      if (vec) {
        for (int h = 0; h < 2; ++h) {  // two halves of the row's float4 groups (registers)
          float4 x[kLuPanelNb / 8];
#pragma unroll
          for (int j = 0; j < kLuPanelNb / 8; ++j)
            if (4 * h + j < groups) x[j] = reinterpret_cast<const float4*>(row)[4 * h + j];
#pragma unroll
          for (int qq = 0; qq < kLuPanelNb; ++qq) {
            if (qq < nbq) {
              const float lq = l[qq];
#pragma unroll
              for (int j = 0; j < kLuPanelNb / 8; ++j)
                if (4 * h + j < groups) {
                  const float4 u4 = reinterpret_cast<const float4*>(Ux[qq])[4 * h + j];
                  x[j].x = fmaf(-lq, u4.x, x[j].x);
                  x[j].y = fmaf(-lq, u4.y, x[j].y);
                  x[j].z = fmaf(-lq, u4.z, x[j].z);
                  x[j].w = fmaf(-lq, u4.w, x[j].w);
                }
            }
          }
#pragma unroll
          for (int j = 0; j < kLuPanelNb / 8; ++j)
            if (4 * h + j < groups) reinterpret_cast<float4*>(row)[4 * h + j] = x[j];
        }
      } else {
        for (int k = 0; k < nbp; ++k) {
          float acc = row[k];
#pragma unroll
          for (int qq = 0; qq < kLuPanelNb; ++qq)
            if (qq < nbq) acc = fmaf(-l[qq], Ux[qq][k], acc);
          row[k] = acc;
        }
      }
    }
    __syncthreads();
  }
  cl.sync();  // every block's mbarriers are initialised before any value is pushed; prologue reads done
  if (jp >= 0 && c == 0)  // U12 of this panel's columns, rows [jp, j0)
    for (int e = tid; e < nbq * nbp; e += kPanelThreads) {
      const int qq = e / nbp, k = e % nbp;
      A[(jp + qq) + (int64_t)(j0 + k) * lda] = Ux[qq][k];
    }
  float best = -1.f;
  int bi = INT_MAX;  // candidate as a panel row
  for (int rr = tid; rr < nr; rr += kPanelThreads) {
    const float v = fabsf(Sp[rr * pitch]);
    if (v > best) { best = v; bi = rlo + rr; }  // rows ascend: the first maximum stays
  }
  bool ok = true;
  for (int q = 0; q < nbp && ok; ++q) {
    const int par = q & 1;
    const MaxLoc m = block_argmax(best, bi, red[par]);
    const int oq = q / RS;  // the block holding row q
    // push: warp d sends to block d: lane 0 the candidate, the next lanes the
    // candidate's row, the following ones row q (from the block holding it)
    if ((tid >> 5) < C && (tid & 31) < kPushLanes) {
      const int d = tid >> 5, l = tid & 31;
      const bool self = d == c;
      const uint32_t rbar = self ? 0u : lu_mapa(lu_smem(&rx_bar[par]), d);
      const int nchunk = vec ? groups : nbp;
      if (l == 0) {
        if (self)
          rx_cand[par][c] = m;
        else
          lu_push2(lu_mapa(lu_smem(&rx_cand[par][c]), d), __float_as_uint(m.v), (uint32_t)m.i, rbar);
      } else if (l <= nchunk) {
        const int k = l - 1;
        const float* src = Sp + (m.i != INT_MAX ? (m.i - rlo) : 0) * pitch;  // any row when there is no candidate
        if (vec) {
          const float4 v = reinterpret_cast<const float4*>(src)[k];
          if (self)
            reinterpret_cast<float4*>(rx_row[par][c])[k] = v;
          else
            lu_push4(lu_mapa(lu_smem(&rx_row[par][c][4 * k]), d), v, rbar);
        } else {
          if (self)
            rx_row[par][c][k] = src[k];
          else
            lu_push1(lu_mapa(lu_smem(&rx_row[par][c][k]), d), src[k], rbar);
        }
      } else if (l <= 2 * nchunk && c == oq) {
        const int k = l - 1 - nchunk;
        const float* src = Sp + (q - rlo) * pitch;
        if (vec) {
          const float4 v = reinterpret_cast<const float4*>(src)[k];
          if (self)
            reinterpret_cast<float4*>(rx_row[par][kLuPanelCluster])[k] = v;
          else
            lu_push4(lu_mapa(lu_smem(&rx_row[par][kLuPanelCluster][4 * k]), d), v, rbar);
        } else {
          if (self)
            rx_row[par][kLuPanelCluster][k] = src[k];
          else
            lu_push1(lu_mapa(lu_smem(&rx_row[par][kLuPanelCluster][k]), d), src[k], rbar);
        }
      }
    }
    const bool got = lu_mbar_wait(lu_smem(&rx_bar[par]), (uint32_t)((q >> 1) & 1));
    ok = __syncthreads_and(got) != 0;  // the same decision in every thread; every thread has seen the phase ...
    if (!ok) {
      if (tid == 0) atomicCAS(status, 0, GBGEMM_ERR_DEVICE_TIMEOUT);
      break;
    }
    // ... before it is re-armed, by a thread with no global stores of its own
    // to wait for (the arrive releases the arriving thread's earlier writes)
    if (tid == kPanelThreads - 1 && q + 2 < nbp) lu_mbar_arm(lu_smem(&rx_bar[par]), rx_bytes(q + 2));
    // the pivot: every warp reduces the C candidates with shuffles (largest
    // |a|, smallest row on ties: the same choice in every block)
    MaxLoc w{-1.f, INT_MAX};
    int wr = -1;
    {
      const int lane = tid & 31;
      if (lane < C) {
        w = rx_cand[par][lane];
        wr = lane;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xFFFFFFFFu, w.v, o);
        const int i2 = __shfl_xor_sync(0xFFFFFFFFu, w.i, o);
        const int r2 = __shfl_xor_sync(0xFFFFFFFFu, wr, o);
        if (v2 > w.v || (v2 == w.v && i2 < w.i)) { w.v = v2; w.i = i2; wr = r2; }
      }
    }
    const int p = (w.i == INT_MAX) ? q : w.i;  // (a column of NaNs keeps its row)
    const int ps = (w.i == INT_MAX) ? kLuPanelCluster : wr;  // the pivot row's slot
    float* const qrow = rx_row[par][kLuPanelCluster];
    float* const prow = rx_row[par][ps];
    if (c == 0 && tid == kPanelThreads - 2) {
      ipiv[j0 + q] = j0 + p + 1;
      piv_s[q] = j0 + p;
    }
    // row q <- the pivot row (in the block holding q); row p <- row q (in the
    // update below, by the thread holding row p)
    if (p != q && c == oq && tid < nbp) Sp[(q - rlo) * pitch + tid] = prow[tid];
    const float d = prow[q];
    best = -1.f;
    bi = INT_MAX;
    const int rs = max(q + 1 - rlo, 0);  // this block's first row below q
    if (d == 0.f) {
      if (c == 0 && tid == 0 && *info == 0) *info = j0 + q + 1;  // the first exactly zero pivot, 1-based
      if (p != q && p >= rlo && p < rlo + nr && tid < nbp) Sp[(p - rlo) * pitch + tid] = qrow[tid];
      __syncthreads();
      if (q + 1 < nbp)
        for (int rr = rs + tid; rr < nr; rr += kPanelThreads) {
          const float v = fabsf(Sp[rr * pitch + q + 1]);
          if (v > best) { best = v; bi = rlo + rr; }
        }
    } else {
      const bool use_rcp = fabsf(d) >= FLT_MIN;  // 1 / d is finite
      const float rcp = __frcp_rn(d);            // correctly rounded, as 1.0f / d
      const float p1 = q + 1 < nbp ? prow[q + 1] : 0.f;
      const int jb = (q + 2) / 4;  // the first group holding a column beyond q + 1
      float4 u[kLuPanelNb / 4];    // the pivot row
      if (vec) {
#pragma unroll
        for (int j = 0; j < kLuPanelNb / 4; ++j)
          if (j < groups) u[j] = reinterpret_cast<const float4*>(prow)[j];
      }
      for (int rr = rs + tid; rr < nr; rr += kPanelThreads) {
        float* row = Sp + rr * pitch;
        if (rlo + rr != p) {
          const float a = row[q];
          const float l = use_rcp ? a * rcp : a / d;
          const float v1 = q + 1 < nbp ? fmaf(-l, p1, row[q + 1]) : 0.f;
          if (vec) {
            float4 x[kLuPanelNb / 4];  // every load issued before any store
#pragma unroll
            for (int j = 0; j < kLuPanelNb / 4; ++j)
              if (j >= jb && j < groups) x[j] = reinterpret_cast<const float4*>(row)[j];
#pragma unroll
            for (int j = 0; j < kLuPanelNb / 4; ++j) {
              if (j > jb && j < groups) {
                x[j].x = fmaf(-l, u[j].x, x[j].x);
                x[j].y = fmaf(-l, u[j].y, x[j].y);
                x[j].z = fmaf(-l, u[j].z, x[j].z);
                x[j].w = fmaf(-l, u[j].w, x[j].w);
                reinterpret_cast<float4*>(row)[j] = x[j];
              } else if (j == jb && j < groups) {  // columns <= q + 1 keep their values
                if (4 * j + 0 > q + 1) x[j].x = fmaf(-l, u[j].x, x[j].x);
                if (4 * j + 1 > q + 1) x[j].y = fmaf(-l, u[j].y, x[j].y);
                if (4 * j + 2 > q + 1) x[j].z = fmaf(-l, u[j].z, x[j].z);
                x[j].w = fmaf(-l, u[j].w, x[j].w);
                reinterpret_cast<float4*>(row)[j] = x[j];
              }
            }
          }
          row[q] = l;
          if (q + 1 < nbp) {  // the next column: its largest |a| is the next candidate
            row[q + 1] = v1;
            if (fabsf(v1) > best) { best = fabsf(v1); bi = rlo + rr; }
          }
        } else {  // row p: receives row q's values, updated beyond column q
          const float a = qrow[q];
          const float l = use_rcp ? a * rcp : a / d;
          float v1 = 0.f;
          if (vec) {
            float4 x[kLuPanelNb / 4];  // every load issued before any store
#pragma unroll
            for (int j = 0; j < kLuPanelNb / 4; ++j)
              if (j < groups) x[j] = reinterpret_cast<const float4*>(qrow)[j];
#pragma unroll
            for (int j = 0; j < kLuPanelNb / 4; ++j) {
              if (j < groups) {
                if (4 * j + 0 > q) x[j].x = fmaf(-l, u[j].x, x[j].x);
                if (4 * j + 1 > q) x[j].y = fmaf(-l, u[j].y, x[j].y);
                if (4 * j + 2 > q) x[j].z = fmaf(-l, u[j].z, x[j].z);
                if (4 * j + 3 > q) x[j].w = fmaf(-l, u[j].w, x[j].w);
                reinterpret_cast<float4*>(row)[j] = x[j];
              }
            }
            if (q + 1 < nbp) v1 = row[q + 1];
          } else {
            for (int k = 0; k < nbp; ++k) row[k] = k > q ? fmaf(-l, prow[k], qrow[k]) : qrow[k];
            if (q + 1 < nbp) v1 = row[q + 1];
          }
          row[q] = l;
          if (q + 1 < nbp && fabsf(v1) > best) { best = fabsf(v1); bi = rlo + rr; }
        }
      }
    }
  }
  __syncthreads();
  for (int q = 0; q < nbp; ++q)
    for (int rr = tid; rr < nr; rr += kPanelThreads) G[(rlo + rr) + (int64_t)q * lda] = Sp[rr * pitch + q];
  if (c == 0 && tid < 32) build_perm(j0, nbp, piv_s, prow_s, pcont_s, perm);
  cl.sync();  // no block leaves while another may still read its published values
}

// Columns [c_lo, j0) and [j0 + nbp, c_hi): apply the row permutation of
// pivot rows [j0, j0 + nbp) (all sources read before any row is written);
// right of them, then U12 = L11^-1 A12, one thread per column, L11 and the
// block's columns staged in shared memory.  Blocks [0, left_tiles) cover the
// left range.
__global__ void __launch_bounds__(kSwapThreads) lu_swap_trsm_kernel(int n, float* __restrict__ A, int64_t lda, int j0,
                                                                 int nbp, const int* __restrict__ perm, int c_lo,
                                                                 int r_lo, int c_hi, int left_tiles) {
  extern __shared__ float sm[];
  const int next = perm[0];
  const int* src = perm + 1;
  const int* ext = perm + 1 + nbp;
  float* V = sm;                   // permuted panel rows: V[q * kXP + col]
  float* W = V + nbp * kXP;        // extra rows: W[x * kXP + col]
  float* Ls = W + nbp * kXP;       // L11: Ls[i * (nbp + 1) + p]
  const bool left = (int)blockIdx.x < left_tiles;
  const int c0 = left ? c_lo + (int)blockIdx.x * kTrsmCols : r_lo + ((int)blockIdx.x - left_tiles) * kTrsmCols;
  const int cend = left ? min(c0 + kTrsmCols, j0) : min(c0 + kTrsmCols, c_hi);
  const int ncol = cend - c0;
  const int tid = threadIdx.x;
#pragma unroll 8
  for (int e = tid; e < nbp * ncol; e += kSwapThreads) {  // up to eight loads in flight per thread
    const int q = e % nbp, col = e / nbp;
    V[q * kXP + col] = A[src[q] + (int64_t)(c0 + col) * lda];
  }
#pragma unroll 8
  for (int e = tid; e < next * ncol; e += kSwapThreads) {
    const int x = e % next, col = e / next;
    W[x * kXP + col] = A[ext[2 * x + 1] + (int64_t)(c0 + col) * lda];
  }
  if (!left)
#pragma unroll 8
    for (int e = tid; e < nbp * nbp; e += kSwapThreads) {
      const int i = e % nbp, p = e / nbp;
      Ls[i * (nbp + 1) + p] = A[(j0 + i) + (int64_t)(j0 + p) * lda];
    }
  __syncthreads();
  for (int e = tid; e < next * ncol; e += kSwapThreads) {
    const int x = e % next, col = e / next;
    A[ext[2 * x] + (int64_t)(c0 + col) * lda] = W[x * kXP + col];
  }
  if (!left && tid < ncol) {  // two partial sums: half the dependent chain
    for (int i = 1; i < nbp; ++i) {
      const float* li = Ls + i * (nbp + 1);
      float s0 = V[i * kXP + tid], s1 = 0.f;
      int p = 0;
      for (; p + 1 < i; p += 2) {
        s0 = fmaf(-li[p], V[p * kXP + tid], s0);
        s1 = fmaf(-li[p + 1], V[(p + 1) * kXP + tid], s1);
      }
      if (p < i) s0 = fmaf(-li[p], V[p * kXP + tid], s0);
      V[i * kXP + tid] = s0 + s1;
    }
  }
  __syncthreads();
  for (int e = tid; e < nbp * ncol; e += kSwapThreads) {
    const int q = e % nbp, col = e / nbp;
    A[(j0 + q) + (int64_t)(c0 + col) * lda] = V[q * kXP + col];
  }
}

// The row exchanges of ipiv applied to one right-hand side per block, in
// order, the column staged in shared memory when SMEM.  An entry out of range
// is skipped, never followed.
template <bool SMEM>
__global__ void __launch_bounds__(256) lu_laswp_rhs_kernel(int n, const int* __restrict__ ipiv, float* __restrict__ B,
                                                           int64_t ldb) {
  extern __shared__ float ys[];
  __shared__ int pv[1024];  // a chunk of ipiv, loaded by every thread
  float* b = B + (int64_t)blockIdx.x * ldb;
  float* y = SMEM ? ys : b;
  if (SMEM) {
#pragma unroll 8
    for (int i = threadIdx.x; i < n; i += blockDim.x) ys[i] = b[i];
  }
  for (int j0 = 0; j0 < n; j0 += 1024) {
    const int cnt = min(1024, n - j0);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) pv[t] = ipiv[j0 + t];
    __syncthreads();
    if (threadIdx.x == 0)
      for (int j = 0; j < cnt; ++j) {
        const int p = pv[j] - 1, r = j0 + j;
        if (p != r && p >= 0 && p < n) {
          const float t = y[r];
          y[r] = y[p];
          y[p] = t;
        }
      }
    __syncthreads();
  }
  if (SMEM)
    for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = ys[i];
}

// Strip t of a diagonal block of w rows holds its columns [32t, 32t + 32)
// (fewer in the last strip), column-major, rows [32t, w) for the lower
// triangle or [0, 32t + 32) for the upper one: the entries a triangular
// solve reads, packed.
__device__ __forceinline__ int strip_rows(bool upper, int w, int t) {
  const int ws = min(32, w - 32 * t);
  return upper ? 32 * t + ws : w - 32 * t;
}

// Offsets of the packed strips of a diagonal block of w rows (one thread).
template <bool UPPER>
__device__ __forceinline__ void strip_offsets(int w, int* soff) {
  const int nsub = (w + 31) / 32;
  int o = 0;
  for (int t = 0; t < nsub; ++t) {
    soff[t] = o;
    o += min(32, w - 32 * t) * strip_rows(UPPER, w, t);
  }
  soff[nsub] = o;
}

// Issue the 4-byte asynchronous copies of the packed triangle of the
// diagonal block T (w rows) into tri (no wait; no alignment needed).
template <bool UPPER>
__device__ __forceinline__ void stage_triangle(const float* __restrict__ T, int64_t lda, int w, float* tri,
                                               const int* soff) {
  const int nsub = (w + 31) / 32;
  for (int t = 0; t < nsub; ++t) {
    const int h = strip_rows(UPPER, w, t), r0 = UPPER ? 0 : 32 * t;
    const int cnt = min(32, w - 32 * t) * h;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int col = e / h, r = e % h;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(tri + soff[t] + e);
      const float* src = T + (r0 + r) + (int64_t)(32 * t + col) * lda;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
    }
  }
}

// Solve the staged triangle in place on ys (w values), in steps of 32 rows:
// each 32 x 32 triangle by warp 0 from registers, the rest of the block by
// threads 0 .. w-1.  Every thread of the block calls it (it synchronises).
template <bool UPPER>
__device__ __forceinline__ void solve_triangle(const float* tri, const int* soff, int w, float* ys) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsub = (w + 31) / 32;
  for (int k = 0; k < nsub; ++k) {
    const int t = UPPER ? nsub - 1 - k : k;
    const int s0 = 32 * t;
    const int ws = min(32, w - s0);
    const int h = strip_rows(UPPER, w, t);
    const float* S = tri + soff[t];  // (i, s0 + q) at S[q * h + i - (UPPER ? 0 : s0)]
    const int ri = UPPER ? 0 : s0;
    if (warp == 0) {
      float M[32];
      float v = lane < ws ? ys[s0 + lane] : 0.f;
      if (!UPPER) {
#pragma unroll
        for (int q = 0; q < 32; ++q) M[q] = (q < lane && lane < ws) ? S[q * h + lane] : 0.f;
#pragma unroll
        for (int q = 0; q < 31; ++q) {
          const float yq = __shfl_sync(0xFFFFFFFFu, v, q);
          if (q < lane) v = fmaf(-M[q], yq, v);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) M[q] = (lane <= q && q < ws) ? S[q * h + s0 + lane] : 0.f;
        const float dmine = lane < ws ? S[lane * h + s0 + lane] : 1.f;  // this lane's diagonal entry
#pragma unroll
        for (int q = 31; q >= 0; --q) {
          if (q < ws) {  // every lane forms the same x_q = v_q / u_qq (no divergent division)
            const float xq = __shfl_sync(0xFFFFFFFFu, v, q) / __shfl_sync(0xFFFFFFFFu, dmine, q);
            if (lane == q) v = xq;
            if (lane < q) v = fmaf(-M[q], xq, v);
          }
        }
      }
      if (lane < ws) ys[s0 + lane] = v;
    }
    __syncthreads();
    // rows of the block beyond the 32 just solved (below for L, above for U)
    const int i = tid;
    if (UPPER ? i < s0 : (i >= s0 + 32 && i < w)) {
      float acc = ys[i];
#pragma unroll
      for (int q = 0; q < 32; ++q)
        if (q < ws) acc = fmaf(-S[q * h + i - ri], ys[s0 + q], acc);
      ys[i] = acc;
    }
    __syncthreads();
  }
}

// One diagonal block of the triangular solves, rows [j0, j0 + w) (w <= 256)
// of one right-hand side per block: forward substitution with the unit lower
// triangle (UPPER false) or back substitution with the upper one (UPPER true).
// The triangle is first copied into shared memory (4-byte asynchronous
// copies, all in flight at once, no alignment needed), then solved in steps
// of 32 rows.
template <bool UPPER>
__global__ void __launch_bounds__(kSolveBlock) lu_trsv_block_kernel(const float* __restrict__ LU, int64_t lda, int j0,
                                                                   int w, float* __restrict__ B, int64_t ldb) {
  extern __shared__ float tri[];  // the packed strips
  __shared__ float ys[kSolveBlock];
  __shared__ int soff[kSolveBlock / 32 + 1];
  float* b = B + (int64_t)blockIdx.x * ldb + j0;
  const float* T = LU + j0 + (int64_t)j0 * lda;  // the diagonal block: (i, q) at T[i + q * lda]
  const int tid = threadIdx.x;
  if (tid == 0) strip_offsets<UPPER>(w, soff);
  if (tid < w) ys[tid] = b[tid];
  __syncthreads();
  stage_triangle<UPPER>(T, lda, w, tri, soff);
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  solve_triangle<UPPER>(tri, soff, w, ys);
  if (tid < w) b[tid] = ys[tid];
}

// A whole triangular solve with one right-hand side in one cooperative
// launch (the blocked substitution without host-side steps): the rows are
// cut into blocks of 256, taken in the order of the solve (forward: first to
// last; back: last to first), block k of that order by CTA k mod the grid.
// A CTA takes the contribution of every earlier block c as soon as c's flag
// is set (y_b -= A_bc x_c, the 256 x 256 product split over two thread
// groups of 128 columns, added in a fixed order), then solves its diagonal
// triangle (staged in shared memory while it waits) and publishes x_b and
// its flag.  Every wait is on an earlier block of the order, so the chain
// always progresses; a wait is bounded (2 s) and sets *status.
template <bool UPPER>
__global__ void __launch_bounds__(kSweepThreads, 1)
    lu_trsv_sweep_kernel(int n, const float* __restrict__ LU, int64_t lda, float* __restrict__ x,
                         int* __restrict__ flags, int* __restrict__ status) {
  extern __shared__ float tri[];
  __shared__ float ys[kSolveBlock];
  __shared__ float xs[kSolveBlock];
  __shared__ float part[kSweepThreads / kSolveBlock][kSolveBlock];
  __shared__ int soff[kSolveBlock / 32 + 1];
  __shared__ int go;
  const int tid = threadIdx.x;
  const int nblk = (n + kSolveBlock - 1) / kSolveBlock;
  for (int k = blockIdx.x; k < nblk; k += gridDim.x) {
    const int b = UPPER ? nblk - 1 - k : k;
    const int r0 = kSolveBlock * b, w = min(kSolveBlock, n - r0);
    __syncthreads();  // the previous block's use of soff, tri, ys is over
    if (tid == 0) strip_offsets<UPPER>(w, soff);
    if (tid < w) ys[tid] = x[r0 + tid];
    __syncthreads();
    stage_triangle<UPPER>(LU + r0 + (int64_t)r0 * lda, lda, w, tri, soff);  // lands while the contributions run
    for (int kk = 0; kk < k; ++kk) {
      const int cb = UPPER ? nblk - 1 - kk : kk;
      const int c0 = kSolveBlock * cb, wc = min(kSolveBlock, n - c0);
      if (tid == 0) {
        int ok = 0;
        uint64_t t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (uint32_t it = 0;; ++it) {
          int f;
          asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(f) : "l"(flags + cb) : "memory");
          if (f) { ok = 1; break; }
          if ((it & 63u) == 63u) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 2000000000ull) break;
          }
        }
        if (!ok) atomicCAS(status, 0, GBGEMM_ERR_DEVICE_TIMEOUT);
        go = ok;
      }
      __syncthreads();
      if (!go) {  // uniform: every thread read go after the barrier
        asm volatile("cp.async.wait_all;" ::: "memory");  // no copy lands after the block has left
        return;
      }
      if (tid < wc) xs[tid] = __ldcg(x + c0 + tid);
      __syncthreads();
      {  // part[g][i] = sum over this group's columns of A(r0 + i, c0 + q) x_q
        const int i = tid % kSolveBlock, g = tid / kSolveBlock;
        constexpr int kq = kSolveBlock / (kSweepThreads / kSolveBlock);
        float acc = 0.f;
        if (i < w) {
          const float* a = LU + (r0 + i) + (int64_t)(c0 + g * kq) * lda;
          if (wc == kSolveBlock) {  // a full block of columns: 32 loads in flight, four partial sums
            float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 32
            for (int q = 0; q < kq; ++q) s4[q & 3] = fmaf(a[(int64_t)q * lda], xs[g * kq + q], s4[q & 3]);
            acc = (s4[0] + s4[1]) + (s4[2] + s4[3]);
          } else {
#pragma unroll 16
            for (int q = 0; q < kq; ++q)
              if (g * kq + q < wc) acc = fmaf(a[(int64_t)q * lda], xs[g * kq + q], acc);
          }
        }
        part[g][i] = acc;
      }
      __syncthreads();
      if (tid < w) {
        float v = ys[tid];
#pragma unroll
        for (int g = 0; g < kSweepThreads / kSolveBlock; ++g) v -= part[g][tid];
        ys[tid] = v;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    solve_triangle<UPPER>(tri, soff, w, ys);
    if (tid < w) x[r0 + tid] = ys[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flags + b), "r"(1) : "memory");
  }
}

bool g_attr_done[64][7];

cudaError_t set_smem_once(const void* fn, int which, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && g_attr_done[dev][which]) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_attr_done[dev][which] = true;
  return e;
}

}  // namespace

int lu_slab_pitch(int nbp) { return nbp <= 2 ? nbp : 4 * (((nbp + 3) / 4) | 1); }

int lu_panel_width(int rows) {
  for (int w = kLuPanelNb; w > 1; w /= 2)
    if ((int64_t)rows <= (int64_t)kLuPanelCluster * (kLuPanelSlabBytes / (4 * lu_slab_pitch(w)))) return w;
  return 1;
}

cudaError_t launch_lu_panel(int n, float* A, int64_t lda, int j0, int nbp, int* ipiv, int* info, int* perm,
                            int* status, cudaStream_t s, int jp, int nbq, const int* perm_prev) {
  if (jp >= 0 && (nbq <= 0 || nbq > kLuPanelNb || jp + nbq != j0 || !perm_prev)) return cudaErrorInvalidValue;
  if (nbp <= 0 || nbp > kLuPanelNb) return cudaErrorInvalidValue;
  const int R = n - j0;
  const int pitch = lu_slab_pitch(nbp);
  const int cap = kLuPanelSlabBytes / (4 * pitch);  // slab rows a block holds
  // one block up to 256 rows; 8 while a block's slab has at most 512 rows
  // (a row per thread), else 16 (a cluster size the GPU allows by opt-in)
  // (one block for more rows, two or three a thread, measured slower than the cluster's exchange)
  int C = R <= 256 ? 1 : ((R + 7) / 8 <= kPanelThreads ? 8 : kLuPanelCluster);
  cudaError_t e = set_smem_once((const void*)lu_panel_kernel, 0, kLuPanelSlabBytes);
  if (e != cudaSuccess) return e;
  static bool wide_set[64] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !wide_set[dev]) {
    e = cudaFuncSetAttribute((const void*)lu_panel_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    wide_set[dev] = true;
  }
  for (;;) {
    const int RS = (R + C - 1) / C;
    if (RS > cap) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kPanelThreads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)RS * pitch * sizeof(float);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, lu_panel_kernel, n, A, lda, j0, nbp, RS, pitch, ipiv, info, perm, status, jp, nbq,
                           perm_prev);
    if (e == cudaSuccess || C != kLuPanelCluster) return e;
    cudaGetLastError();  // a cluster of 16 could not be launched: 8, if the rows fit
    C = 8;
  }
}

cudaError_t launch_lu_perm(int j0, int nbp, const int* ipiv, int* perm, cudaStream_t s) {
  if (nbp <= 0 || nbp > kLuMaxNb) return cudaErrorInvalidValue;
  lu_perm_kernel<<<1, 32, 0, s>>>(j0, nbp, ipiv, perm);
  return cudaGetLastError();
}

cudaError_t launch_lu_swap_trsm(int n, float* A, int64_t lda, int j0, int nbp, const int* perm, int c_lo, int c_hi,
                                cudaStream_t s, int r_lo) {
  if (r_lo < 0) r_lo = j0 + nbp;
  if (nbp <= 0 || nbp > kLuMaxNb || c_lo < 0 || c_lo > j0 || r_lo < j0 + nbp || c_hi < r_lo || c_hi > n)
    return cudaErrorInvalidValue;
  const int left_tiles = (j0 - c_lo + kTrsmCols - 1) / kTrsmCols;
  const int right_tiles = (c_hi - r_lo + kTrsmCols - 1) / kTrsmCols;
  if (left_tiles + right_tiles == 0) return cudaSuccess;
  const size_t max_smem = ((size_t)2 * kLuMaxNb * kXP + (size_t)kLuMaxNb * (kLuMaxNb + 1)) * sizeof(float);
  cudaError_t e = set_smem_once((const void*)lu_swap_trsm_kernel, 1, max_smem);
  if (e != cudaSuccess) return e;
  const size_t smem = ((size_t)2 * nbp * kXP + (size_t)nbp * (nbp + 1)) * sizeof(float);
  lu_swap_trsm_kernel<<<left_tiles + right_tiles, kSwapThreads, smem, s>>>(n, A, lda, j0, nbp, perm, c_lo, r_lo,
                                                                           c_hi, left_tiles);
  return cudaGetLastError();
}

cudaError_t launch_lu_laswp_rhs(int n, int64_t nrhs, const int* ipiv, float* B, int64_t ldb, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
  if (n <= kLuSolveSmemN) {
    cudaError_t e = set_smem_once((const void*)lu_laswp_rhs_kernel<true>, 2, (size_t)kLuSolveSmemN * sizeof(float));
    if (e != cudaSuccess) return e;
    lu_laswp_rhs_kernel<true><<<(unsigned)nrhs, 256, (size_t)n * sizeof(float), s>>>(n, ipiv, B, ldb);
  } else {
    lu_laswp_rhs_kernel<false><<<(unsigned)nrhs, 256, 0, s>>>(n, ipiv, B, ldb);
  }
  return cudaGetLastError();
}

cudaError_t launch_lu_trsv_sweep(bool upper, int n, const float* LU, int64_t lda, float* x, int* flags, int* status,
                                 int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t tri_bytes = (size_t)kSolveBlock * (kSolveBlock + 32) / 2 * sizeof(float);
  const void* fn = upper ? (const void*)lu_trsv_sweep_kernel<true> : (const void*)lu_trsv_sweep_kernel<false>;
  cudaError_t e = set_smem_once(fn, upper ? 5 : 6, tri_bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSweepThreads, tri_bytes)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int nblk = (n + kSolveBlock - 1) / kSolveBlock;
  const int grid = nblk < per_sm * num_sms ? nblk : per_sm * num_sms;  // every CTA resident at once
  if ((e = cudaMemsetAsync(flags, 0, (size_t)nblk * sizeof(int), s)) != cudaSuccess) return e;
  void* args[] = {(void*)&n, (void*)&LU, (void*)&lda, (void*)&x, (void*)&flags, (void*)&status};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSweepThreads), args, tri_bytes, s);
}

cudaError_t launch_lu_trsv_block(bool upper, const float* LU, int64_t lda, int j0, int w, int64_t nrhs, float* B,
                                 int64_t ldb, cudaStream_t s) {
  if (w <= 0 || nrhs <= 0) return cudaSuccess;
  if (w > kSolveBlock || nrhs > 0x7FFFFFFF) return cudaErrorInvalidValue;
  // packed triangle: sum over strips of (columns x rows), at most 36864 floats for w = 256
  size_t floats = 0;
  for (int t = 0; 32 * t < w; ++t) {
    const int ws = w - 32 * t < 32 ? w - 32 * t : 32;
    floats += (size_t)ws * (upper ? 32 * t + ws : w - 32 * t);
  }
  const size_t max_bytes = (size_t)kSolveBlock * (kSolveBlock + 32) / 2 * sizeof(float);
  cudaError_t e = set_smem_once(upper ? (const void*)lu_trsv_block_kernel<true> : (const void*)lu_trsv_block_kernel<false>,
                                upper ? 3 : 4, max_bytes);
  if (e != cudaSuccess) return e;
  if (upper)
    lu_trsv_block_kernel<true><<<(unsigned)nrhs, kSolveBlock, floats * sizeof(float), s>>>(LU, lda, j0, w, B, ldb);
  else
    lu_trsv_block_kernel<false><<<(unsigned)nrhs, kSolveBlock, floats * sizeof(float), s>>>(LU, lda, j0, w, B, ldb);
  return cudaGetLastError();
}

}  // namespace gbg
