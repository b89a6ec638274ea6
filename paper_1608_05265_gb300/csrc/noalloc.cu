// gbgemm_sgemm_split_noalloc: the split-BF16 sgemm without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code that runs where allocating device memory is not
// allowed or not possible at call time -- inside a region being captured
// into a CUDA graph by someone else's stream capture, inside a custom
// allocator or memory-pool callback that must not re-enter the allocator,
// in a real-time loop whose latency budget forbids the implicit device
// synchronisation of cudaMalloc/cudaFree, or in a process whose device
// memory is fully reserved up front by another framework.  Such callers
// pass inputs and outputs as usual; the scratch (hi/lo panels, row maxima
// and a status word) comes from a fixed array in this library's device
// memory instead of a handle's workspace.
//
// The scratch is one file-scope __device__ array of GBGEMM_NOALLOC_SCRATCH_BYTES.
// Every GPU that loads this library holds it until the process exits.  In
// host code the array's name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress once per device (with that
// device current) and cached; the first call on each device does this.
#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GBGEMM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr size_t kStatusBytes = 256;  // the status word's slot at the start of the array

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};
bool g_split_ok[kMaxDevices] = {};

int trans_code_na(char t) {
  switch (t) {
    case 'N': case 'n': return 0;
    case 'T': case 't': case 'C': case 'c': return 1;
    default: return -1;
  }
}

// Per-device set-up: the device address of the scratch array, the SM count
// and whether the split kernels run here.  Called with `dev` current.
int setup_device(int dev, void** scratch, int* num_sms, bool* split_ok) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return GBGEMM_ERR_CUDA;
    }
    int sms = 0, major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
      cudaGetLastError();
      return GBGEMM_ERR_CUDA;
    }
    g_num_sms[dev] = sms;
    g_split_ok[dev] = (major == 10 && minor == 3);
    g_scratch_ptr[dev] = p;
  }
  *scratch = g_scratch_ptr[dev];
  *num_sms = g_num_sms[dev];
  *split_ok = g_split_ok[dev];
  return GBGEMM_OK;
}

// Scratch bytes one call needs: the status slot plus gbgemm_split_workspace_bytes(m, n, k).
size_t noalloc_scratch_bytes(int64_t m, int64_t n, int64_t k) {
  return kStatusBytes + gbg::split_layout(m, n, k, 1, 1, 256).total;
}

}  // namespace

extern "C" {

int gbgemm_sgemm_split_noalloc(void* cuda_stream, char transa, char transb, int64_t m, int64_t n, int64_t k,
                               float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                               float beta, float* C, int64_t ldc, int* status) {
  const int ta = trans_code_na(transa), tb = trans_code_na(transb);
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
  if (m == 0 || n == 0) return GBGEMM_OK;
  if (!use_ab && beta == 1.0f) return GBGEMM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (!use_ab) return gbg::launch_scale_c(m, n, beta, C, ldc, s) == cudaSuccess ? GBGEMM_OK : GBGEMM_ERR_CUDA;
  const size_t need = noalloc_scratch_bytes(m, n, k);
  if (need > (size_t)GBGEMM_NOALLOC_SCRATCH_BYTES) return GBGEMM_ERR_SCRATCH_LIMIT;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GBGEMM_ERR_CUDA;
  }
  void* scratch = nullptr;
  int num_sms = 0;
  bool split_ok = false;
  const int rc = setup_device(dev, &scratch, &num_sms, &split_ok);
  if (rc != GBGEMM_OK) return rc;
  if (!split_ok) return GBGEMM_ERR_UNSUPPORTED_DEVICE;

  // Carve the array: [status | the call's workspace: control words, band
  // counters and row maxima (zeroed by launch_split_call before the kernel
  // runs), then the panels, which the kernel's packers rewrite in full before
  // any tile reads them], so stale contents of earlier calls do not leak
  // into this one.
  unsigned char* base = static_cast<unsigned char*>(scratch);
  int* dstatus = status ? status : reinterpret_cast<int*>(base);
  if (!status && cudaMemsetAsync(dstatus, 0, sizeof(int), s) != cudaSuccess) return GBGEMM_ERR_CUDA;
  gbg::SplitCall c;
  c.ta = ta; c.tb = tb; c.m = m; c.n = n; c.k = k; c.alpha = alpha; c.beta = beta;
  c.A = A; c.lda = lda; c.B = B; c.ldb = ldb; c.C = C; c.ldc = ldc;
  c.bn = 256; c.raster = 16; c.splitk = 1;
  c.ws = base + kStatusBytes; c.status = dstatus; c.num_sms = num_sms;
  return gbg::launch_split_call(c, s) == cudaSuccess ? GBGEMM_OK : GBGEMM_ERR_CUDA;
}

}  // extern "C"
