// C-ABI front end: argument checks in BLAS order, quick returns, path choice,
// workspace management and kernel dispatch (the BLIS driver layer of
// Section III-A, which hands fixed-shape pieces of the problem to the
// micro-kernel).  One handle holds the per-device state the paper keeps in
// its long-lived service process (Section III-B): device properties, the
// stream and a persistent workspace, set up once instead of on every call.
#include <climits>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <string>
#include <vector>

#include "grouped.h"
#include "internal.h"
#include "mlp.h"
#include "tuner.h"

struct gbgemm_grouped_plan : gbg::GroupedPlan {};

struct gbgemm_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  int path = GBGEMM_PATH_AUTO;
  int last_path = 0;
  int num_sms = 0;
  int cc_major = 0, cc_minor = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* d_status = nullptr;
  int* d_lu_perm = nullptr;  // row permutation of the current LU panel
  cudaStream_t lu_side = nullptr;  // LU look-ahead: the next block's factorisation
  cudaEvent_t lu_ev[2] = {nullptr, nullptr};
  // profiling
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;  // pairs (start, stop)
  size_t ev_used = 0;                // events recorded in this profiling window
  int64_t gemm_launches = 0;
  int64_t kernel_launches = 0;
  // tuning
  int tuning = 0;
  gbg::Tuner tuner;
  gbg::Predictor predictor{GBGEMM_NUM_CONFIGS};
  gbg::Predictor sched_predictor{GBGEMM_NUM_SCHEDULES};
  int pred_sel = 0;                          // network addressed by gbgemm_predictor_*
  std::map<std::string, int> sched_choice;   // tuning mode 2: predicted schedule per shape key
  void* pred_scratch = nullptr;              // device scratch of one schedule prediction
  int last_schedule = -1;
  int pinned_schedule = -1;                  // gbgemm_set_schedule
};

namespace {

int trans_code(char t) {
  switch (t) {
    case 'N': case 'n': return 0;
    case 'T': case 't': case 'C': case 'c': return 1;
    default: return -1;
  }
}

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

int ensure_workspace(gbgemm_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return GBGEMM_OK;
  // The old buffer may still be in use by queued work on the stream.
  if (h->ws) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GBGEMM_ERR_ALLOC;
  }
  h->ws = p;
  h->ws_bytes = bytes;
  return GBGEMM_OK;
}

bool split_supported(const gbgemm_handle* h) { return h->cc_major == 10 && h->cc_minor == 3; }

// The next pair of profiling events (both null when not profiling); the
// split launch records them again around its GEMM launch.
cudaError_t prof_pair(gbgemm_handle* h, cudaEvent_t* e0, cudaEvent_t* e1) {
  *e0 = *e1 = nullptr;
  if (!h->profiling) return cudaSuccess;
  while (h->ev_used + 2 > h->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    h->ev_pool.push_back(e);
  }
  *e0 = h->ev_pool[h->ev_used++];
  *e1 = h->ev_pool[h->ev_used++];
  // recorded once here so that a call that launches no GEMM counts 0 ms
  cudaError_t err = cudaEventRecord(*e0, h->stream);
  return err != cudaSuccess ? err : cudaEventRecord(*e1, h->stream);
}

}  // namespace

extern "C" {

size_t gbgemm_panel_bytes(int64_t rows, int64_t k) {
  if (rows <= 0 || k <= 0) return 0;
  return gbg::panel_bytes(rows, k);
}

size_t gbgemm_split_workspace_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return gbg::split_layout(m, n, k, 1, 1, 256).total;
}

int gbgemm_create(gbgemm_handle** out, int device) {
  if (!out) return GBGEMM_ERR_INVALID_VALUE;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return GBGEMM_ERR_CUDA;
  }
  gbgemm_handle* h = new (std::nothrow) gbgemm_handle();
  if (!h) return GBGEMM_ERR_ALLOC;
  h->device = device;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete h;
    return GBGEMM_ERR_CUDA;
  }
  h->num_sms = prop.multiProcessorCount;
  h->cc_major = prop.major;
  h->cc_minor = prop.minor;
  if (cudaMalloc(&h->d_status, 256) != cudaSuccess || cudaMemset(h->d_status, 0, 256) != cudaSuccess) {
    cudaGetLastError();
    if (h->d_status) cudaFree(h->d_status);
    delete h;
    return GBGEMM_ERR_ALLOC;
  }
  *out = h;
  return GBGEMM_OK;
}

int gbgemm_destroy(gbgemm_handle* h) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  DeviceGuard g(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->lu_side) cudaStreamSynchronize(h->lu_side);
  if (h->ws) cudaFree(h->ws);
  if (h->d_status) cudaFree(h->d_status);
  if (h->d_lu_perm) cudaFree(h->d_lu_perm);
  for (cudaEvent_t e : h->lu_ev)
    if (e) cudaEventDestroy(e);
  if (h->lu_side) cudaStreamDestroy(h->lu_side);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->pred_scratch) cudaFree(h->pred_scratch);
  delete h;
  return GBGEMM_OK;
}

int gbgemm_set_stream(gbgemm_handle* h, void* s) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  h->stream = static_cast<cudaStream_t>(s);
  return GBGEMM_OK;
}

int gbgemm_set_path(gbgemm_handle* h, int path) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (path != GBGEMM_PATH_AUTO && path != GBGEMM_PATH_SIMT && path != GBGEMM_PATH_SPLIT_BF16)
    return GBGEMM_ERR_INVALID_VALUE;
  if (path == GBGEMM_PATH_SPLIT_BF16 && !split_supported(h)) return GBGEMM_ERR_UNSUPPORTED_DEVICE;
  h->path = path;
  return GBGEMM_OK;
}

int gbgemm_last_path(gbgemm_handle* h, int* path) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!path) return GBGEMM_ERR_INVALID_VALUE;
  *path = h->last_path;
  return GBGEMM_OK;
}

int gbgemm_reserve_workspace(gbgemm_handle* h, size_t bytes) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  DeviceGuard g(h->device);
  return ensure_workspace(h, bytes);
}

namespace {

// The fixed heuristic's schedule of a call (tuning mode 0).  Path AUTO: split
// from k = 128 on a GPU that has the split path, SIMT below.  Split: the
// widest tile that still gives at least half of the SMs a tile (measured at
// 2048^3: 128 BN-256 tiles beat 256 BN-128 tiles, 208 against 150 TFLOP/s),
// tile rows in groups of 16, and for one problem with a long k and too few
// tiles the k range cut into slices (keeping the widest tile).  SIMT: 64 x 64
// for small outputs, else 128 x 128.
gbg::Schedule default_schedule(const gbgemm_handle* h, int path, int64_t m, int64_t n, int64_t k, int64_t batch) {
  if (path == GBGEMM_PATH_AUTO) path = (k >= gbg::kSplitMinK && split_supported(h)) ? GBGEMM_PATH_SPLIT_BF16 : GBGEMM_PATH_SIMT;
  gbg::Schedule d{};
  d.path = path;
  d.raster = 16;
  d.level = 0;
  d.splitk = 1;
  d.simt_cfg = (m * n <= (int64_t)512 * 512) ? gbg::SIMT_64x64 : gbg::SIMT_128x128;
  auto tiles = [&](int64_t bm, int64_t bn) { return ((m + bm - 1) / bm) * ((n + bn - 1) / bn) * batch; };
  const int64_t half_sms = h->num_sms / 2;
  d.bn = tiles(128, 256) >= half_sms ? 256 : tiles(128, 128) >= half_sms ? 128 : 64;
  if (batch == 1) {
    const int s = gbg::choose_splitk(tiles(128, 256), k, h->num_sms);
    if (s > 1) {  // k-slicing level 3 of the schedules: the slices that fill the SMs
      d.bn = 256;
      d.level = 3;
      d.splitk = s;
    }
  }
  return d;
}

bool in_training_range3(int64_t m, int64_t n, int64_t k) {
  auto ok = [](int64_t v) { return v >= 8 && v <= 16384; };
  return ok(m) && ok(n) && ok(k);
}

// Schedules a call may take on this handle: legal for the problem, on the
// handle's path (AUTO: either), the split path only where the GPU has it.
bool schedule_allowed(const gbgemm_handle* h, const gbgemm_problem& q, int s) {
  gbg::Schedule d;
  if (!gbg::schedule_decode(s, &d)) return false;
  if (h->path != GBGEMM_PATH_AUTO && d.path != h->path) return false;
  if (d.path == GBGEMM_PATH_SPLIT_BF16 && !split_supported(h)) return false;
  return gbg::schedule_legal(q.m, q.n, q.k, q.alpha, s, h->num_sms);
}

// Tuning modes 1 and 2: the tuner's fastest allowed schedule, or the schedule
// predictor's choice (cached per shape key; the tuner where the predictor
// has no parameters or the shape is outside its training range).  *best = -1
// when nothing is allowed.  Synchronises the stream on a shape's first call.
int choose_schedule(gbgemm_handle* h, const gbgemm_problem& q, int* best) {
  *best = -1;
  if (h->tuning == 2 && h->sched_predictor.ready() && in_training_range3(q.m, q.n, q.k)) {
    const std::string key = gbg::tune_key(q) + (h->path == GBGEMM_PATH_AUTO ? " a" : h->path == GBGEMM_PATH_SIMT ? " s" : " b");
    auto it = h->sched_choice.find(key);
    if (it != h->sched_choice.end()) {
      *best = it->second;
      return GBGEMM_OK;
    }
    constexpr int kLB = (GBGEMM_NUM_SCHEDULES + 7) / 8;
    float x[8];
    gbg::predictor_features(q, x);
    uint8_t legal[kLB] = {};
    for (int s = 0; s < GBGEMM_NUM_SCHEDULES; ++s)
      if (schedule_allowed(h, q, s)) legal[s >> 3] |= (uint8_t)(1u << (s & 7));
    if (!h->pred_scratch && cudaMalloc(&h->pred_scratch, 256) != cudaSuccess) {
      cudaGetLastError();
      h->pred_scratch = nullptr;
      return GBGEMM_ERR_ALLOC;
    }
    float* dx = static_cast<float*>(h->pred_scratch);
    uint8_t* dl = reinterpret_cast<uint8_t*>(static_cast<char*>(h->pred_scratch) + 64);
    int* dc = reinterpret_cast<int*>(static_cast<char*>(h->pred_scratch) + 128);
    int choice = -1;
    if (cudaMemcpyAsync(dx, x, sizeof(x), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(dl, legal, sizeof(legal), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return GBGEMM_ERR_CUDA;
    int rc = h->sched_predictor.predict(dx, dl, 1, nullptr, dc, h->stream);
    if (rc != GBGEMM_OK) return rc;
    if (cudaMemcpyAsync(&choice, dc, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return GBGEMM_ERR_CUDA;
    if (choice >= 0) {
      h->sched_choice[key] = choice;
      *best = choice;
      return GBGEMM_OK;
    }
  }
  std::vector<float> lat;
  h->tuner.bind(h->stream, h->d_status, h->num_sms);
  if (h->tuner.measure_schedules(q, 3, &lat) != GBGEMM_OK) return GBGEMM_ERR_CUDA;
  for (int s = 0; s < GBGEMM_NUM_SCHEDULES; ++s) {
    if (lat[(size_t)s] < 0.f || !schedule_allowed(h, q, s)) continue;
    if (*best < 0 || lat[(size_t)s] < lat[(size_t)*best]) *best = s;
  }
  return GBGEMM_OK;
}

}  // namespace

// The call after argument checks: one problem (batch 1) or a strided batch of
// equal problems, problem z at A + z*sa, B + z*sb, C + z*sc.
static int run_sgemm(gbgemm_handle* h, int ta, int tb, char transa, char transb, int64_t m, int64_t n, int64_t k,
                     float alpha, const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                     int64_t ldc, int64_t batch, int64_t sa, int64_t sb, int64_t sc) {
  const bool use_ab = (alpha != 0.0f) && (k > 0);
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  h->last_path = 0;
  if (m == 0 || n == 0) return GBGEMM_OK;
  if (!use_ab && beta == 1.0f) return GBGEMM_OK;
  DeviceGuard g(h->device);
  if (!use_ab) {
    if (gbg::launch_scale_c_batched(m, n, beta, C, ldc, batch, sc, h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
    h->kernel_launches += 1;
    return GBGEMM_OK;
  }
  gbg::Problem p{ta, tb, m, n, k, alpha, beta, A, lda, B, ldb, C, ldc};
  gbg::Schedule d = default_schedule(h, h->path, m, n, k, batch);
  const gbgemm_problem q1{transa, transb, m, n, k, alpha, beta, A, lda, B, ldb, C, ldc};
  if (batch == 1 && h->pinned_schedule >= 0 && schedule_allowed(h, q1, h->pinned_schedule)) {
    gbg::schedule_resolve(h->pinned_schedule, m, n, k, alpha, h->num_sms, &d);
  } else if (h->tuning >= 1 && batch == 1) {
    const gbgemm_problem q{transa, transb, m, n, k, alpha, beta, A, lda, B, ldb, C, ldc};
    int best = -1;
    const int rc = choose_schedule(h, q, &best);
    if (rc != GBGEMM_OK) return rc;
    if (best >= 0) gbg::schedule_resolve(best, m, n, k, alpha, h->num_sms, &d);
  }
  const int path = d.path;
  const int simt_cfg = d.simt_cfg, split_bn = d.bn;
  if (path == GBGEMM_PATH_SIMT) {
    const int cfg = simt_cfg;
    if (gbg::launch_simt_batched(p, cfg, batch, sa, sb, sc, h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
    h->kernel_launches += 1;
    h->last_path = GBGEMM_PATH_SIMT;
    h->last_schedule = cfg;
    return GBGEMM_OK;
  }
  if (!split_supported(h)) return GBGEMM_ERR_UNSUPPORTED_DEVICE;
  // Workspace (one problem or a strided batch): control words, band counters
  // and row maxima (zeroed per call), the packed panels, and with split-K
  // (one problem, long k, too few tiles for the SMs) splitk x tiles raw
  // 128 x bn accumulators, summed by a reduction.
  const int splitk = batch == 1 ? d.splitk : 1;
  const gbg::SplitLayout L = gbg::split_layout(m, n, k, batch, splitk, split_bn);
  if (L.block > ((size_t)1 << 62) / (size_t)batch) return GBGEMM_ERR_ALLOC;
  int rc = ensure_workspace(h, L.total);
  if (rc != GBGEMM_OK) return rc;
  gbg::SplitCall c;
  c.ta = ta; c.tb = tb; c.m = m; c.n = n; c.k = k; c.alpha = alpha; c.beta = beta;
  c.A = A; c.lda = lda; c.B = B; c.ldb = ldb; c.C = C; c.ldc = ldc;
  c.batch = batch; c.sa = sa; c.sb = sb; c.sc = sc;
  c.bn = split_bn; c.raster = d.raster; c.splitk = splitk;
  c.ws = h->ws; c.status = h->d_status; c.num_sms = h->num_sms;
  h->kernel_launches += 1;  // the packing launch (the memset of the workspace head is not a kernel of ours)
  if (prof_pair(h, &c.gemm_begin, &c.gemm_end) != cudaSuccess) return GBGEMM_ERR_CUDA;
  if (gbg::launch_split_call(c, h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
  h->kernel_launches += splitk > 1 ? 2 : 1;
  h->gemm_launches += 1;
  h->last_path = GBGEMM_PATH_SPLIT_BF16;
  h->last_schedule = gbg::schedule_encode_split(split_bn, d.raster, batch == 1 ? d.level : 0);
  return GBGEMM_OK;
}


int gbgemm_sgemm(gbgemm_handle* h, char transa, char transb, int64_t m, int64_t n, int64_t k,
                 float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                 float beta, float* C, int64_t ldc) {
  const int ta = trans_code(transa), tb = trans_code(transb);
  if (ta < 0) return -1;
  if (tb < 0) return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  const int64_t arows = ta ? k : m, brows = tb ? n : k;
  if (lda < (arows > 1 ? arows : 1)) return -8;
  if (ldb < (brows > 1 ? brows : 1)) return -10;
  if (ldc < (m > 1 ? m : 1)) return -13;
  const bool use_ab = (alpha != 0.0f) && (k > 0);
  if (m > 0 && n > 0) {
    if (use_ab && !A) return -7;
    if (use_ab && !B) return -9;
    if (!C) return -12;
  }
  return run_sgemm(h, ta, tb, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 1, 0, 0, 0);
}

int gbgemm_sgemm_strided_batched(gbgemm_handle* h, char transa, char transb, int64_t m, int64_t n, int64_t k,
                                 float alpha, const float* A, int64_t lda, int64_t stride_a, const float* B,
                                 int64_t ldb, int64_t stride_b, float beta, float* C, int64_t ldc, int64_t stride_c,
                                 int64_t batch) {
  const int ta = trans_code(transa), tb = trans_code(transb);
  if (ta < 0) return -1;
  if (tb < 0) return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  const int64_t arows = ta ? k : m, brows = tb ? n : k;
  if (lda < (arows > 1 ? arows : 1)) return -8;
  if (stride_a < 0) return -9;
  if (ldb < (brows > 1 ? brows : 1)) return -11;
  if (stride_b < 0) return -12;
  if (ldc < (m > 1 ? m : 1)) return -15;
  // results of different problems must not overlap
  if (stride_c < 0 || (batch > 1 && m > 0 && n > 0 && stride_c < ldc * (n - 1) + m)) return -16;
  if (batch < 0 || batch > 65535) return -17;
  const bool use_ab = (alpha != 0.0f) && (k > 0);
  if (m > 0 && n > 0 && batch > 0) {
    if (use_ab && !A) return -7;
    if (use_ab && !B) return -10;
    if (!C) return -14;
  }
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (batch == 0) {
    h->last_path = 0;
    return GBGEMM_OK;
  }
  return run_sgemm(h, ta, tb, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, batch, stride_a,
                   stride_b, stride_c);
}

int gbgemm_sgemv(gbgemm_handle* h, char trans, int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
                 const float* x, int64_t incx, float beta, float* y, int64_t incy) {
  const int t = trans_code(trans);
  if (t < 0) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -6;
  if (incx == 0) return -8;
  if (incy == 0) return -11;
  const int64_t len_x = t ? m : n, len_y = t ? n : m;
  const bool use_ax = (alpha != 0.0f) && (len_x > 0);
  if (len_y > 0) {
    if (use_ax && !A) return -5;
    if (use_ax && !x) return -7;
    if (!y) return -10;
  }
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (len_y == 0 || (!use_ax && beta == 1.0f)) return GBGEMM_OK;
  DeviceGuard g(h->device);
  const int64_t slices = use_ax ? gbg::gemv_slices(t == 1, m, n, h->num_sms) : 1;
  float* partial = nullptr;
  if (slices > 1) {
    const int rc = ensure_workspace(h, (size_t)slices * (size_t)len_y * sizeof(float));
    if (rc != GBGEMM_OK) return rc;
    partial = static_cast<float*>(h->ws);
  }
  if (gbg::launch_gemv(t == 1, m, n, use_ax ? alpha : 0.0f, A, lda, x, incx, beta, y, incy, slices, partial,
                       h->num_sms, h->stream) != cudaSuccess)
    return GBGEMM_ERR_CUDA;
  h->kernel_launches += slices > 1 ? 2 : 1;
  return GBGEMM_OK;
}

int gbgemm_sgetrf(gbgemm_handle* h, int64_t n, float* A, int64_t lda, int* ipiv, int* info, int nb) {
  if (n < 0 || n > INT_MAX) return -1;
  if (n > 0 && !A) return -2;
  if (lda < (n > 1 ? n : 1)) return -3;
  if (n > 0 && !ipiv) return -4;
  if (!info) return -5;
  if (nb < 0 || nb > gbg::kLuMaxNb) return -6;
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  DeviceGuard g(h->device);
  if (cudaMemsetAsync(info, 0, sizeof(int), h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
  h->last_path = 0;
  if (n == 0) return GBGEMM_OK;
  if (!h->d_lu_perm && cudaMalloc(&h->d_lu_perm, 2 * gbg::kLuPermInts * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    h->d_lu_perm = nullptr;
    return GBGEMM_ERR_ALLOC;
  }
  const int b = nb > 0 ? nb : (n < GBGEMM_SGETRF_WIDE_N ? GBGEMM_SGETRF_DEFAULT_NB : GBGEMM_SGETRF_MAX_NB);
  if (!h->lu_side) {  // look-ahead stream (highest priority) and its two events
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->lu_side, cudaStreamNonBlocking, greatest) != cudaSuccess) {
      h->lu_side = nullptr;
      return GBGEMM_ERR_CUDA;
    }
    for (cudaEvent_t& e : h->lu_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return GBGEMM_ERR_CUDA;
  }
  // The trailing updates run with the handle's path choice but never through
  // the per-call tuner (each update has a new shape).
  const int tuning = h->tuning;
  h->tuning = 0;
  int rc = GBGEMM_OK;
  auto update = [&](int64_t r, int64_t c, int64_t rows, int64_t cols, int64_t kc, int64_t k) {
    // A(r:r+rows, c:c+cols) -= A(r:r+rows, kc:kc+k) A(kc:kc+k, c:c+cols), on the handle's stream
    return run_sgemm(h, 0, 0, 'N', 'N', rows, cols, k, -1.0f, A + r + kc * lda, lda, A + kc + c * lda, lda, 1.0f,
                     A + r + c * lda, lda, 1, 0, 0, 0);
  };
  int* perm = h->d_lu_perm;
  // Factor the block [j0, j0 + nbo) on stream s: panels of pw columns, each
  // followed by its exchanges and triangular solve over the rest of the block
  // and the SIMT update of the block columns right of it (no workspace, so
  // the block can be factored while the handle's stream updates other
  // columns); then the block's exchanges as one permutation.
  auto factor_block = [&](int64_t j0, int nbo, cudaStream_t s) -> int {
    const int fit = gbg::lu_panel_width((int)(n - j0));
    const int pw = b < fit ? b : fit;
    for (int64_t j1 = j0; j1 < j0 + nbo; j1 += pw) {
      const int w = (int)(j0 + nbo - j1 < pw ? j0 + nbo - j1 : pw);
      if (gbg::launch_lu_panel((int)n, A, lda, (int)j1, w, ipiv, info, perm, h->d_status, s) != cudaSuccess)
        return GBGEMM_ERR_CUDA;
      h->kernel_launches += 1;
      if (w == nbo) return GBGEMM_OK;  // one panel: its permutation is the block's
      if (gbg::launch_lu_swap_trsm((int)n, A, lda, (int)j1, w, perm, (int)j0, (int)(j0 + nbo), s) != cudaSuccess)
        return GBGEMM_ERR_CUDA;
      h->kernel_launches += 1;
      const int64_t rows = n - j1 - w, cols = j0 + nbo - j1 - w;
      if (cols > 0) {
        const int64_t r = j1 + w, c = j1 + w;
        const gbg::Problem p{0, 0, rows, cols, w, -1.0f, 1.0f, A + r + j1 * lda, lda, A + j1 + c * lda, lda,
                             A + r + c * lda, lda};
        const int cfg = rows * cols <= (int64_t)512 * 512 ? gbg::SIMT_64x64 : gbg::SIMT_128x128;
        if (gbg::launch_simt(p, cfg, s) != cudaSuccess) return GBGEMM_ERR_CUDA;
        h->kernel_launches += 1;
      }
    }
    if (gbg::launch_lu_perm((int)j0, nbo, ipiv, perm, s) != cudaSuccess) return GBGEMM_ERR_CUDA;
    h->kernel_launches += 1;
    return GBGEMM_OK;
  };
  if (b <= gbg::kLuPanelNb && gbg::lu_panel_width((int)n) >= b) {
    // Every block is one panel.  Look-ahead with a fused prologue: the next
    // panel, on the side stream, applies block k's exchanges, U12 and update
    // to its own columns itself and factors them, while the handle's stream
    // applies block k to every other column (exchanges, U12, trailing
    // update).  The two touch disjoint columns; the two permutation buffers
    // alternate between the blocks.
    int* pbuf[2] = {h->d_lu_perm, h->d_lu_perm + gbg::kLuPermInts};
    int nbo = (int)(n < b ? n : b);
    if (gbg::launch_lu_panel((int)n, A, lda, 0, nbo, ipiv, info, pbuf[0], h->d_status, h->stream) != cudaSuccess)
      rc = GBGEMM_ERR_CUDA;
    h->kernel_launches += 1;
    int k = 0;
    for (int64_t j0 = 0; j0 < n && rc == GBGEMM_OK; j0 += nbo, ++k) {
      nbo = (int)(n - j0 < b ? n - j0 : b);
      int* pk = pbuf[k & 1];
      int* pn = pbuf[(k + 1) & 1];
      const int64_t jn = j0 + nbo;
      const int nbn = jn < n ? (int)(n - jn < b ? n - jn : b) : 0;
      if (nbn > 0) {
        if (cudaEventRecord(h->lu_ev[0], h->stream) != cudaSuccess ||
            cudaStreamWaitEvent(h->lu_side, h->lu_ev[0], 0) != cudaSuccess ||
            gbg::launch_lu_panel((int)n, A, lda, (int)jn, nbn, ipiv, info, pn, h->d_status, h->lu_side, (int)j0, nbo,
                                 pk) != cudaSuccess ||
            cudaEventRecord(h->lu_ev[1], h->lu_side) != cudaSuccess) {
          rc = GBGEMM_ERR_CUDA;
          break;
        }
        h->kernel_launches += 1;
      }
      if (j0 > 0 || jn + nbn < n) {
        if (gbg::launch_lu_swap_trsm((int)n, A, lda, (int)j0, nbo, pk, 0, (int)n, h->stream, (int)(jn + nbn)) !=
            cudaSuccess) {
          rc = GBGEMM_ERR_CUDA;
          break;
        }
        h->kernel_launches += 1;
      }
      const int64_t rest = n - jn - nbn;
      if (nbn > 0 && rest > 0) rc = update(jn, jn + nbn, n - jn, rest, j0, nbo);
      if (rc != GBGEMM_OK) break;
      if (nbn > 0 && cudaStreamWaitEvent(h->stream, h->lu_ev[1], 0) != cudaSuccess) rc = GBGEMM_ERR_CUDA;
    }
    if (rc != GBGEMM_OK && cudaEventRecord(h->lu_ev[1], h->lu_side) == cudaSuccess)
      cudaStreamWaitEvent(h->stream, h->lu_ev[1], 0);  // never leave work on the side stream unjoined
    h->tuning = tuning;
    return rc;
  }
  // Look-ahead: after block k's exchanges and U12, the next block's columns
  // are updated first; the next block is then factored on the side stream
  // while the handle's stream updates the remaining columns.  The two touch
  // disjoint columns; the handle's stream waits for the block before
  // applying its exchanges.
  int nbo = (int)(n < b ? n : b);
  rc = factor_block(0, nbo, h->stream);
  for (int64_t j0 = 0; j0 < n && rc == GBGEMM_OK; j0 += nbo) {
    nbo = (int)(n - j0 < b ? n - j0 : b);
    if (j0 > 0 || j0 + nbo < n) {
      if (gbg::launch_lu_swap_trsm((int)n, A, lda, (int)j0, nbo, perm, 0, (int)n, h->stream) != cudaSuccess) {
        rc = GBGEMM_ERR_CUDA;
        break;
      }
      h->kernel_launches += 1;
    }
    const int64_t jn = j0 + nbo;  // the next block
    if (jn >= n) break;
    const int nbn = (int)(n - jn < b ? n - jn : b);
    rc = update(jn, jn, n - jn, nbn, j0, nbo);
    if (rc != GBGEMM_OK) break;
    if (cudaEventRecord(h->lu_ev[0], h->stream) != cudaSuccess ||
        cudaStreamWaitEvent(h->lu_side, h->lu_ev[0], 0) != cudaSuccess) {
      rc = GBGEMM_ERR_CUDA;
      break;
    }
    rc = factor_block(jn, nbn, h->lu_side);
    if (rc != GBGEMM_OK) break;
    if (cudaEventRecord(h->lu_ev[1], h->lu_side) != cudaSuccess) {
      rc = GBGEMM_ERR_CUDA;
      break;
    }
    const int64_t rest = n - jn - nbn;
    if (rest > 0) rc = update(jn, jn + nbn, n - jn, rest, j0, nbo);
    if (rc != GBGEMM_OK) break;
    if (cudaStreamWaitEvent(h->stream, h->lu_ev[1], 0) != cudaSuccess) rc = GBGEMM_ERR_CUDA;
  }
  if (rc != GBGEMM_OK) {  // never leave work on the side stream unjoined
    if (cudaEventRecord(h->lu_ev[1], h->lu_side) == cudaSuccess) cudaStreamWaitEvent(h->stream, h->lu_ev[1], 0);
  }
  h->tuning = tuning;
  return rc;
}

int gbgemm_sgetrs(gbgemm_handle* h, int64_t n, int64_t nrhs, const float* LU, int64_t lda, const int* ipiv, float* B,
                  int64_t ldb) {
  if (n < 0 || n > INT_MAX) return -1;
  if (nrhs < 0 || nrhs > INT_MAX) return -2;
  if (n > 0 && !LU) return -3;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (n > 0 && !ipiv) return -5;
  if (n > 0 && nrhs > 0 && !B) return -6;
  if (ldb < (n > 1 ? n : 1)) return -7;
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (n == 0 || nrhs == 0) return GBGEMM_OK;
  DeviceGuard g(h->device);
  if (gbg::launch_lu_laswp_rhs((int)n, nrhs, ipiv, B, ldb, h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
  h->kernel_launches += 1;
  if (nrhs == 1) {  // each substitution as one cooperative launch (flags in the workspace)
    const int64_t nblk = (n + gbg::kSolveBlock - 1) / gbg::kSolveBlock;
    const int rc = ensure_workspace(h, (size_t)nblk * sizeof(int));
    if (rc != GBGEMM_OK) return rc;
    int* flags = static_cast<int*>(h->ws);
    if (gbg::launch_lu_trsv_sweep(false, (int)n, LU, lda, B, flags, h->d_status, h->num_sms, h->stream) !=
            cudaSuccess ||
        gbg::launch_lu_trsv_sweep(true, (int)n, LU, lda, B, flags, h->d_status, h->num_sms, h->stream) !=
            cudaSuccess)
      return GBGEMM_ERR_CUDA;
    h->kernel_launches += 2;
    return GBGEMM_OK;
  }
  // several right-hand sides: B(r:r+rows, :) -= LU(r:r+rows, c:c+w) B(c:c+w, :)
  // by the sgemm (never through the per-call tuner)
  const int tuning = h->tuning;
  h->tuning = 0;
  auto update = [&](int64_t r, int64_t rows, int64_t c, int64_t w) {
    return run_sgemm(h, 0, 0, 'N', 'N', rows, nrhs, w, -1.0f, LU + r + c * lda, lda, B + c, ldb, 1.0f, B + r, ldb,
                     1, 0, 0, 0);
  };
  const int nbs = gbg::kSolveBlock;
  int rc = GBGEMM_OK;
  for (int64_t j0 = 0; j0 < n && rc == GBGEMM_OK; j0 += nbs) {  // L y = P b, top down
    const int w = (int)(n - j0 < nbs ? n - j0 : nbs);
    if (gbg::launch_lu_trsv_block(false, LU, lda, (int)j0, w, nrhs, B, ldb, h->stream) != cudaSuccess) {
      rc = GBGEMM_ERR_CUDA;
      break;
    }
    h->kernel_launches += 1;
    if (j0 + w < n) rc = update(j0 + w, n - j0 - w, j0, w);
  }
  for (int64_t j0 = (n - 1) / nbs * nbs; j0 >= 0 && rc == GBGEMM_OK; j0 -= nbs) {  // U x = y, bottom up
    const int w = (int)(n - j0 < nbs ? n - j0 : nbs);
    if (gbg::launch_lu_trsv_block(true, LU, lda, (int)j0, w, nrhs, B, ldb, h->stream) != cudaSuccess) {
      rc = GBGEMM_ERR_CUDA;
      break;
    }
    h->kernel_launches += 1;
    if (j0 > 0) rc = update(0, j0, j0, w);
  }
  h->tuning = tuning;
  return rc;
}

int gbgemm_split_pack(gbgemm_handle* h, char which, char trans, int64_t rows, int64_t k,
                      const float* X, int64_t ldx, uint32_t* amax_bits, void* panel, void* panel2) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  const int t = trans_code(trans);
  if (t < 0 || (which != 'A' && which != 'B') || rows < 0 || k < 0) return GBGEMM_ERR_INVALID_VALUE;
  if (rows == 0 || k == 0) return GBGEMM_OK;
  if (!X || !amax_bits || !panel || (gbg::split_parts(k) == 2 && !panel2)) return GBGEMM_ERR_INVALID_VALUE;
  if (!split_supported(h)) return GBGEMM_ERR_UNSUPPORTED_DEVICE;
  // Stored rows of X: op(A) rows come from A (m x k or k x m); op(B) columns from B.
  const bool kcontig = (which == 'A') ? (t == 1) : (t == 0);
  const int64_t stored_rows = kcontig ? k : rows;
  if (ldx < (stored_rows > 1 ? stored_rows : 1)) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard g(h->device);
  // The packing launch alone (no tiles), on the K-vectors as rows of an "A"
  // operand; the panels are cleared first so that the padding rows of the
  // last (even) block read as zeros.
  const gbg::SplitLayout L = gbg::split_layout(rows, 0, k, 1, 1, 256);
  int rc = ensure_workspace(h, L.head);
  if (rc != GBGEMM_OK) return rc;
  const size_t pbytes = gbg::panel_bytes(rows, k);
  if (cudaMemsetAsync(panel, 0, pbytes, h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
  if (gbg::split_parts(k) == 2 && cudaMemsetAsync(panel2, 0, pbytes, h->stream) != cudaSuccess)
    return GBGEMM_ERR_CUDA;
  gbg::SplitCall c;
  c.ta = kcontig ? 1 : 0; c.m = rows; c.n = 0; c.k = k;
  c.A = X; c.lda = ldx;
  c.ws = h->ws; c.status = h->d_status; c.num_sms = h->num_sms;
  c.pack_only = true; c.panel_out = panel; c.panel2_out = gbg::split_parts(k) == 2 ? panel2 : nullptr;
  c.amax_out = amax_bits;
  return gbg::launch_split_call(c, h->stream) == cudaSuccess ? GBGEMM_OK : GBGEMM_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Grouped sgemm plans
// ---------------------------------------------------------------------------
namespace {

int create_plan(gbgemm_handle* h, const gbgemm_problem* probs, int64_t count, const int* configs,
                gbgemm_grouped_plan** out) {
  gbgemm_grouped_plan* P = new (std::nothrow) gbgemm_grouped_plan();
  if (!P) return GBGEMM_ERR_ALLOC;
  P->device = h->device;
  P->num_sms = h->num_sms;
  P->status = h->d_status;
  P->count = count;
  P->configs = new (std::nothrow) int[count > 0 ? count : 1];
  if (!P->configs) {
    delete P;
    return GBGEMM_ERR_ALLOC;
  }
  for (int64_t g = 0; g < count; ++g) {
    const gbgemm_problem& q = probs[g];
    const bool skip = q.m == 0 || q.n == 0 || (!((q.alpha != 0.0f) && (q.k > 0)) && q.beta == 1.0f);
    P->configs[g] = skip ? -1 : configs[g];
  }
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete[] P->configs;
    delete P;
    return GBGEMM_ERR_CUDA;
  }
  const int rc = gbg::build_grouped_plan(P, probs, count, configs, cs);
  cudaStreamDestroy(cs);
  if (rc != GBGEMM_OK) {
    delete[] P->configs;
    delete P;
    return rc;
  }
  *out = P;
  return GBGEMM_OK;
}

// Configuration of every problem: the default heuristic, the tuner's lowest
// cost, or the learned predictor (falling back to the tuner).
uint8_t legal_mask(const gbgemm_handle* h, const gbgemm_problem& q) {
  uint8_t m = 0;
  for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c)
    if (gbg::config_legal(q, c) && !(c >= GBGEMM_CFG_SPLIT_BN64 && !split_supported(h))) m |= (uint8_t)(1u << c);
  return m;
}

// Grouped plans keep the default rule's path for every problem (split from
// k = 128, SIMT below) and let the tuner or the predictor pick the tile shape
// within it: chosen per problem in isolation, moving problems between the
// paths made whole batches slower (per-problem batch costs do not add up
// across the graph's SIMT branches and split chain).
uint8_t family_mask(int cfg) { return cfg >= GBGEMM_CFG_SPLIT_BN64 ? 0x38u : 0x07u; }

bool in_training_range(const gbgemm_problem& q) {
  auto ok = [](int64_t v) { return v >= 8 && v <= 16384; };
  return ok(q.m) && ok(q.n) && ok(q.k);
}

// Predicted configurations of the problems flagged in `want` (-1 where the
// predictor is not used).
int predict_configs(gbgemm_handle* h, const gbgemm_problem* probs, int64_t count, std::vector<char>& want,
                    std::vector<int>& out) {
  std::vector<float> x;
  std::vector<uint8_t> legal;
  std::vector<int64_t> which;
  for (int64_t g = 0; g < count; ++g) {
    if (!want[g]) continue;
    float f[8];
    gbg::predictor_features(probs[g], f);
    x.insert(x.end(), f, f + 8);
    legal.push_back(legal_mask(h, probs[g]) & family_mask(gbg::default_config(probs[g])));
    which.push_back(g);
  }
  out.assign((size_t)count, -1);
  const int64_t n = (int64_t)which.size();
  if (n == 0) return GBGEMM_OK;
  void* d = nullptr;
  const size_t bx = (size_t)n * 8 * sizeof(float), bl = ((size_t)n + 255) / 256 * 256, bc = (size_t)n * sizeof(int);
  if (cudaMalloc(&d, bx + bl + bc) != cudaSuccess) {
    cudaGetLastError();
    return GBGEMM_ERR_ALLOC;
  }
  float* dx = static_cast<float*>(d);
  uint8_t* dl = reinterpret_cast<uint8_t*>(static_cast<char*>(d) + bx);
  int* dc = reinterpret_cast<int*>(static_cast<char*>(d) + bx + bl);
  std::vector<int> cfg((size_t)n);
  int rc = GBGEMM_ERR_CUDA;
  if (cudaMemcpy(dx, x.data(), bx, cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemcpy(dl, legal.data(), (size_t)n, cudaMemcpyHostToDevice) == cudaSuccess) {
    rc = h->predictor.predict(dx, dl, n, nullptr, dc, h->stream);
    if (rc == GBGEMM_OK && (cudaMemcpyAsync(cfg.data(), dc, bc, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
                            cudaStreamSynchronize(h->stream) != cudaSuccess))
      rc = GBGEMM_ERR_CUDA;
  }
  cudaFree(d);
  if (rc != GBGEMM_OK) return rc;
  for (int64_t i = 0; i < n; ++i) out[(size_t)which[i]] = cfg[(size_t)i];
  return GBGEMM_OK;
}

int choose_configs(gbgemm_handle* h, const gbgemm_problem* probs, int64_t count, int source, int* cfg) {
  std::vector<int> predicted;
  if (source == GBGEMM_CONFIG_PREDICTED && h->predictor.ready()) {
    std::vector<char> want((size_t)count, 0);
    for (int64_t g = 0; g < count; ++g) {
      const gbgemm_problem& q = probs[g];
      const bool skip = q.m == 0 || q.n == 0 || !((q.alpha != 0.0f) && (q.k > 0));
      want[g] = !skip && in_training_range(q);
    }
    const int rc = predict_configs(h, probs, count, want, predicted);
    if (rc != GBGEMM_OK) return rc;
  }
  for (int64_t g = 0; g < count; ++g) {
    const gbgemm_problem& q = probs[g];
    const bool skip = q.m == 0 || q.n == 0 || !((q.alpha != 0.0f) && (q.k > 0));
    cfg[g] = gbg::default_config(q);
    if (!skip && source == GBGEMM_CONFIG_PREDICTED && !predicted.empty() && predicted[g] >= 0) {
      cfg[g] = predicted[g];
    } else if (!skip && source != GBGEMM_CONFIG_DEFAULT) {
      gbg::TuneResult r;
      h->tuner.bind(h->stream, h->d_status, h->num_sms);
      const int rc = h->tuner.measure(q, 3, &r);
      if (rc != GBGEMM_OK) return rc;
      const uint8_t fam = family_mask(cfg[g]);
      int b = -1;
      for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c)
        if (((fam >> c) & 1u) && r.cost_us[c] >= 0.f && (b < 0 || r.cost_us[c] < r.cost_us[b])) b = c;
      if (b >= 0) cfg[g] = b;
    }
    if (cfg[g] >= GBGEMM_CFG_SPLIT_BN64 && !split_supported(h)) cfg[g] = GBGEMM_CFG_SIMT_128x128;
  }
  return GBGEMM_OK;
}

int check_problems(const gbgemm_problem* probs, int64_t count, const int* configs, int64_t* bad_index) {
  for (int64_t g = 0; g < count; ++g) {
    if (gbg::validate_problem(probs[g]) != 0 || (configs && !gbg::config_legal(probs[g], configs[g]))) {
      if (bad_index) *bad_index = g;
      return GBGEMM_ERR_BAD_PLAN;
    }
  }
  return GBGEMM_OK;
}

}  // namespace

int gbgemm_grouped_plan_create_with_configs(gbgemm_handle* h, const gbgemm_problem* probs, int64_t count,
                                            const int* configs, gbgemm_grouped_plan** plan, int64_t* bad_index) {
  if (bad_index) *bad_index = -1;
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!plan || count < 0 || (count > 0 && (!probs || !configs))) return GBGEMM_ERR_INVALID_VALUE;
  *plan = nullptr;
  int rc = check_problems(probs, count, configs, bad_index);
  if (rc != GBGEMM_OK) return rc;
  for (int64_t g = 0; g < count; ++g)
    if (configs[g] >= GBGEMM_CFG_SPLIT_BN64 && !split_supported(h)) return GBGEMM_ERR_UNSUPPORTED_DEVICE;
  DeviceGuard dg(h->device);
  return create_plan(h, probs, count, configs, plan);
}

int gbgemm_grouped_plan_create(gbgemm_handle* h, const gbgemm_problem* probs, int64_t count, int config_source,
                               gbgemm_grouped_plan** plan, int64_t* bad_index) {
  if (bad_index) *bad_index = -1;
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!plan || count < 0 || (count > 0 && !probs)) return GBGEMM_ERR_INVALID_VALUE;
  if (config_source != GBGEMM_CONFIG_DEFAULT && config_source != GBGEMM_CONFIG_TUNED &&
      config_source != GBGEMM_CONFIG_PREDICTED)
    return GBGEMM_ERR_INVALID_VALUE;
  *plan = nullptr;
  int rc = check_problems(probs, count, nullptr, bad_index);
  if (rc != GBGEMM_OK) return rc;
  DeviceGuard dg(h->device);
  std::vector<int> cfg((size_t)(count > 0 ? count : 1));
  rc = choose_configs(h, probs, count, config_source, cfg.data());
  if (rc != GBGEMM_OK) return rc;
  return create_plan(h, probs, count, cfg.data(), plan);
}

int gbgemm_grouped_plan_run(gbgemm_grouped_plan* plan, void* cuda_stream) {
  if (!plan) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!plan->exec) return GBGEMM_ERR_BAD_PLAN;
  DeviceGuard dg(plan->device);
  return cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? GBGEMM_OK
                                                                                            : GBGEMM_ERR_CUDA;
}

int gbgemm_grouped_plan_configs(const gbgemm_grouped_plan* plan, int* configs) {
  if (!plan) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!configs && plan->count > 0) return GBGEMM_ERR_INVALID_VALUE;
  for (int64_t g = 0; g < plan->count; ++g) configs[g] = plan->configs[g];
  return GBGEMM_OK;
}

int gbgemm_grouped_plan_stats(const gbgemm_grouped_plan* plan, int64_t* n_split, int64_t* n_simt, double* flops_split,
                              double* flops_simt, int* kernels_per_run, size_t* device_bytes) {
  if (!plan) return GBGEMM_ERR_NOT_INITIALIZED;
  if (n_split) *n_split = plan->n_split;
  if (n_simt) *n_simt = plan->n_simt;
  if (flops_split) *flops_split = plan->flops_split;
  if (flops_simt) *flops_simt = plan->flops_simt;
  if (kernels_per_run) *kernels_per_run = plan->kernels_per_run;
  if (device_bytes) *device_bytes = plan->dbytes;
  return GBGEMM_OK;
}

int gbgemm_grouped_plan_destroy(gbgemm_grouped_plan* plan) {
  if (!plan) return GBGEMM_ERR_NOT_INITIALIZED;
  DeviceGuard dg(plan->device);
  cudaDeviceSynchronize();
  delete[] plan->configs;
  delete plan;
  return GBGEMM_OK;
}

int gbgemm_autotune(gbgemm_handle* h, const gbgemm_problem* prob, int reps, float* latency_us, float* cost_us,
                    int* best_by_latency, int* best_by_cost) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!prob || reps < 1) return GBGEMM_ERR_INVALID_VALUE;
  if (gbg::validate_problem(*prob) != 0 || prob->m == 0 || prob->n == 0) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard dg(h->device);
  gbg::TuneResult r;
  h->tuner.bind(h->stream, h->d_status, h->num_sms);
  const int rc = h->tuner.measure(*prob, reps, &r);
  if (rc != GBGEMM_OK) return rc;
  for (int c = 0; c < GBGEMM_NUM_CONFIGS; ++c) {
    const bool usable = !(c >= GBGEMM_CFG_SPLIT_BN64 && !split_supported(h));
    if (latency_us) latency_us[c] = usable ? r.latency_us[c] : -1.f;
    if (cost_us) cost_us[c] = usable ? r.cost_us[c] : -1.f;
  }
  if (best_by_latency) *best_by_latency = gbg::best_config(r, false);
  if (best_by_cost) *best_by_cost = gbg::best_config(r, true);
  return GBGEMM_OK;
}

int gbgemm_predictor_set(gbgemm_handle* h, const float* params) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!params) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard dg(h->device);
  if (h->pred_sel == 1) h->sched_choice.clear();
  return (h->pred_sel == 1 ? h->sched_predictor : h->predictor).set(params);
}

int gbgemm_predictor_select(gbgemm_handle* h, int which) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (which != 0 && which != 1) return GBGEMM_ERR_INVALID_VALUE;
  h->pred_sel = which;
  return GBGEMM_OK;
}

int gbgemm_predictor_get(gbgemm_handle* h, float* params) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!params) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard dg(h->device);
  return (h->pred_sel == 1 ? h->sched_predictor : h->predictor).get(params);
}

int gbgemm_predictor_features(const gbgemm_problem* prob, float* x) {
  if (!prob || !x) return GBGEMM_ERR_INVALID_VALUE;
  gbg::predictor_features(*prob, x);
  return GBGEMM_OK;
}

int gbgemm_predictor_predict(gbgemm_handle* h, const float* x, const uint8_t* legal, int64_t n, float* scores,
                             int* configs) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (n < 0 || (n > 0 && !x)) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard dg(h->device);
  return (h->pred_sel == 1 ? h->sched_predictor : h->predictor).predict(x, legal, n, scores, configs, h->stream);
}

int gbgemm_predictor_loss_grad(gbgemm_handle* h, const float* x, const float* y, const float* mask, int64_t n,
                               float* loss, float* grad) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!x || !y || !mask || !grad) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard dg(h->device);
  return (h->pred_sel == 1 ? h->sched_predictor : h->predictor).loss_grad(x, y, mask, n, loss, grad, h->stream);
}

int gbgemm_predictor_train(gbgemm_handle* h, const float* x, const float* y, const float* mask, int64_t n, int epochs,
                           int batch, float lr, uint64_t seed, float* final_loss) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!x || !y || !mask) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard dg(h->device);
  if (h->pred_sel == 1) h->sched_choice.clear();
  return (h->pred_sel == 1 ? h->sched_predictor : h->predictor)
      .train(x, y, mask, n, epochs, batch, lr, seed, final_loss, h->stream);
}

int gbgemm_tuning_save(gbgemm_handle* h, const char* path) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!path) return GBGEMM_ERR_INVALID_VALUE;
  return h->tuner.save(path);
}

int gbgemm_tuning_load(gbgemm_handle* h, const char* path) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!path) return GBGEMM_ERR_INVALID_VALUE;
  return h->tuner.load(path);
}

int gbgemm_tuning_clear(gbgemm_handle* h) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  h->tuner.cache.clear();
  h->tuner.sched_cache.clear();
  h->sched_choice.clear();
  return GBGEMM_OK;
}

int gbgemm_set_tuning(gbgemm_handle* h, int mode) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (mode != 0 && mode != 1 && mode != 2) return GBGEMM_ERR_INVALID_VALUE;
  h->tuning = mode;
  return GBGEMM_OK;
}

int gbgemm_schedule_info(int s, int* path, int* tile_m, int* tile_n, int* raster, int* kslice_level) {
  gbg::Schedule d;
  if (!gbg::schedule_decode(s, &d)) return GBGEMM_ERR_INVALID_VALUE;
  const bool simt = d.path == GBGEMM_PATH_SIMT;
  if (path) *path = d.path;
  if (tile_m) *tile_m = simt ? (d.simt_cfg == gbg::SIMT_64x64 ? 64 : 128) : 128;
  if (tile_n) *tile_n = simt ? (d.simt_cfg == gbg::SIMT_128x128 ? 128 : 64) : d.bn;
  if (raster) *raster = simt ? 1 : d.raster;
  if (kslice_level) *kslice_level = simt ? 0 : d.level;
  return GBGEMM_OK;
}

int gbgemm_schedule_legal(gbgemm_handle* h, const gbgemm_problem* prob, int s, int* legal) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!prob || !legal || s < 0 || s >= GBGEMM_NUM_SCHEDULES) return GBGEMM_ERR_INVALID_VALUE;
  gbg::Schedule d;
  gbg::schedule_decode(s, &d);
  *legal = gbg::schedule_legal(prob->m, prob->n, prob->k, prob->alpha, s, h->num_sms) &&
           !(d.path == GBGEMM_PATH_SPLIT_BF16 && !split_supported(h));
  return GBGEMM_OK;
}

int gbgemm_schedule_default(gbgemm_handle* h, const gbgemm_problem* prob, int* s) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!prob || !s) return GBGEMM_ERR_INVALID_VALUE;
  const gbg::Schedule d = default_schedule(h, GBGEMM_PATH_AUTO, prob->m, prob->n, prob->k, 1);
  *s = d.path == GBGEMM_PATH_SIMT ? d.simt_cfg : gbg::schedule_encode_split(d.bn, d.raster, d.level);
  return GBGEMM_OK;
}

int gbgemm_autotune_schedules(gbgemm_handle* h, const gbgemm_problem* prob, int reps, float* latency_us, int* best) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!prob || reps < 1) return GBGEMM_ERR_INVALID_VALUE;
  if (gbg::validate_problem(*prob) != 0 || prob->m == 0 || prob->n == 0 || prob->k == 0) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard dg(h->device);
  std::vector<float> lat;
  h->tuner.bind(h->stream, h->d_status, h->num_sms);
  const int rc = h->tuner.measure_schedules(*prob, reps, &lat);
  if (rc != GBGEMM_OK) return rc;
  int b = -1;
  for (int s = 0; s < GBGEMM_NUM_SCHEDULES; ++s) {
    gbg::Schedule d;
    gbg::schedule_decode(s, &d);
    if (d.path == GBGEMM_PATH_SPLIT_BF16 && !split_supported(h)) lat[(size_t)s] = -1.f;
    if (lat[(size_t)s] >= 0.f && (b < 0 || lat[(size_t)s] < lat[(size_t)b])) b = s;
  }
  if (latency_us) std::memcpy(latency_us, lat.data(), sizeof(float) * GBGEMM_NUM_SCHEDULES);
  if (best) *best = b;
  return GBGEMM_OK;
}

int gbgemm_last_schedule(gbgemm_handle* h, int* s) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!s) return GBGEMM_ERR_INVALID_VALUE;
  *s = h->last_schedule;
  return GBGEMM_OK;
}

int gbgemm_set_schedule(gbgemm_handle* h, int s) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (s < -1 || s >= GBGEMM_NUM_SCHEDULES) return GBGEMM_ERR_INVALID_VALUE;
  h->pinned_schedule = s;
  return GBGEMM_OK;
}

int gbgemm_check_error(gbgemm_handle* h, char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                       const float* A, int64_t lda, const float* B, int64_t ldb, float beta, const float* C_in,
                       const float* C_out, int64_t ldc, int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                       double* max_ratio) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  DeviceGuard dg(h->device);
  return gbg::run_error_check(h->stream, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C_in, C_out, ldc, i0,
                              i1, j0, j1, max_ratio);
}

int gbgemm_get_device_status(gbgemm_handle* h, int* status) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (!status) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard g(h->device);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GBGEMM_ERR_CUDA;
  if (v != 0 && cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) return GBGEMM_ERR_CUDA;
  *status = v;
  return GBGEMM_OK;
}

int gbgemm_debug_expire_wait(gbgemm_handle* h, uint64_t timeout_ns) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  if (timeout_ns == 0 || timeout_ns > GBGEMM_DEBUG_MAX_WAIT_NS) return GBGEMM_ERR_INVALID_VALUE;
  DeviceGuard g(h->device);
  if (gbg::launch_wait_probe(h->d_status, timeout_ns, h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
  h->kernel_launches += 1;
  return GBGEMM_OK;
}

int gbgemm_profile_begin(gbgemm_handle* h) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  h->profiling = true;
  h->ev_used = 0;
  h->gemm_launches = 0;
  h->kernel_launches = 0;
  return GBGEMM_OK;
}

int gbgemm_profile_end(gbgemm_handle* h, double* gemm_ms, int64_t* gemm_launches, int64_t* kernel_launches) {
  if (!h) return GBGEMM_ERR_NOT_INITIALIZED;
  DeviceGuard g(h->device);
  h->profiling = false;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return GBGEMM_ERR_CUDA;
  double total = 0.0;
  for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]) != cudaSuccess) return GBGEMM_ERR_CUDA;
    total += ms;
  }
  if (gemm_ms) *gemm_ms = total;
  if (gemm_launches) *gemm_launches = h->gemm_launches;
  if (kernel_launches) *kernel_launches = h->kernel_launches;
  h->ev_used = 0;
  return GBGEMM_OK;
}

const char* gbgemm_status_string(int s) {
  if (s > -100 && s < 0) return "GBGEMM_ERR_ARGUMENT (minus the 1-based position of the bad argument)";
  switch (s) {
    case GBGEMM_OK: return "GBGEMM_OK";
    case GBGEMM_ERR_NOT_INITIALIZED: return "GBGEMM_ERR_NOT_INITIALIZED";
    case GBGEMM_ERR_ALLOC: return "GBGEMM_ERR_ALLOC";
    case GBGEMM_ERR_CUDA: return "GBGEMM_ERR_CUDA";
    case GBGEMM_ERR_UNSUPPORTED_DEVICE: return "GBGEMM_ERR_UNSUPPORTED_DEVICE";
    case GBGEMM_ERR_DEVICE_TIMEOUT: return "GBGEMM_ERR_DEVICE_TIMEOUT";
    case GBGEMM_ERR_BAD_PLAN: return "GBGEMM_ERR_BAD_PLAN";
    case GBGEMM_ERR_INVALID_VALUE: return "GBGEMM_ERR_INVALID_VALUE";
    case GBGEMM_ERR_SCRATCH_LIMIT: return "GBGEMM_ERR_SCRATCH_LIMIT";
    default: return "GBGEMM_UNKNOWN_STATUS";
  }
}

}  // extern "C"
