// noalloc_sum.cu -- gmq_tree_sum_noalloc: the pairwise-tree sum of
// gmq_tree_sum with its working memory in a fixed static device array, for
// callers that must not allocate device memory (see gmq.h).
//
// The per-tile partial sums and the last-block ticket live in
// g_noalloc_scratch below.  Host code cannot use the array's name as a
// device address (in host code it names a host-side stand-in), so the first
// call on each device looks the address up with cudaGetSymbolAddress while
// that device is current and caches it; every later call on that device
// reuses the cached pointer.
#include <mutex>

#include "gmq_common.cuh"
#include "sweep_kernels.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr int64_t kMaxTiles = GMQ_NOALLOC_MAX_N / gmq::kTile;
constexpr size_t kStatusBytes = 256;  // DevStatus, padded to the array's alignment
constexpr size_t kScratchBytes = kStatusBytes + sizeof(double) * (size_t)kMaxTiles;

static_assert(GMQ_NOALLOC_MAX_N % gmq::kTile == 0, "whole tiles");
static_assert(sizeof(gmq::DevStatus) <= kStatusBytes, "status fits its slot");

// Scratch of the allocation-free tree sum: [DevStatus | partial sums].
// Every call on a device shares it; it lives until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (the caller has made it
// current); looked up once per device.
cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = (unsigned char*)g_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" gmq_status gmq_tree_sum_noalloc(int32_t device, int64_t n, const double* d_v,
                                           double* d_sum, void* cuda_stream) {
  if (n < 0 || !d_sum || (n > 0 && !d_v)) return GMQ_ERR_INVALID;
  if (n > GMQ_NOALLOC_MAX_N) return GMQ_ERR_TOO_LARGE;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return GMQ_ERR_CUDA;
  }
  if (device < 0 || device >= ndev || device >= kMaxDevices) return GMQ_ERR_INVALID;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return GMQ_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return GMQ_ERR_CUDA;
  gmq_status status = GMQ_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned char* base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) {
    status = GMQ_ERR_CUDA;
  } else if (n == 0) {
    if (cudaMemsetAsync(d_sum, 0, sizeof(double), s) != cudaSuccess) status = GMQ_ERR_CUDA;
  } else {
    gmq::DevStatus* st = (gmq::DevStatus*)base;
    double* partials = (double*)(base + kStatusBytes);
    // the ticket must start at zero; clear it on the caller's stream
    if (cudaMemsetAsync(st, 0, sizeof(gmq::DevStatus), s) != cudaSuccess ||
        gmq::launch_tree_sum(d_v, n, partials, st, d_sum, s) != cudaSuccess)
      status = GMQ_ERR_CUDA;
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return status;
}
