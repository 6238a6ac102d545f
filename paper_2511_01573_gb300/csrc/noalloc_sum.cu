// noalloc_sum.cu -- gmq_tree_sum_noalloc: the pairwise-tree sum of
// gmq_tree_sum with its working memory in a fixed static device array, for
// callers that must not allocate device memory (see gmq.h).
//
// The per-tile partial sums and the last-block ticket live in
// g_noalloc_scratch below.  Host code cannot use the array's name as a
// device address (in host code it names a host-side stand-in), so every
// call looks the address up with cudaGetSymbolAddress while the caller's
// device is current.  The lookup allocates nothing; doing it per call (not
// once per device) keeps the address right after the device's context has
// been torn down and re-created (cudaDeviceReset).
#include "gmq_common.cuh"
#include "sweep_kernels.cuh"

namespace {

constexpr int64_t kMaxTiles = GMQ_NOALLOC_MAX_N / gmq::kTile;
constexpr size_t kStatusBytes = 256;  // DevStatus, padded to the array's alignment
constexpr size_t kScratchBytes = kStatusBytes + sizeof(double) * (size_t)kMaxTiles;

static_assert(GMQ_NOALLOC_MAX_N % gmq::kTile == 0, "whole tiles");
static_assert(sizeof(gmq::DevStatus) <= kStatusBytes, "status fits its slot");

// Scratch of the allocation-free tree sum: [DevStatus | partial sums].
// Every call on a device shares it; it lives until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// A CUDA failure is returned as GMQ_ERR_CUDA with the error cleared, so a
// later, unrelated CUDA call does not report it as its own.
gmq_status fail_cuda() {
  cudaGetLastError();
  return GMQ_ERR_CUDA;
}

// True if p is device (or managed) memory of `device`.
bool on_device(const void* p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
         at.device == device;
}

}  // namespace

extern "C" gmq_status gmq_tree_sum_noalloc(int32_t device, int64_t n, const double* d_v,
                                           double* d_sum, void* cuda_stream) {
  if (n < 0 || !d_sum || (n > 0 && !d_v)) return GMQ_ERR_INVALID;
  if (n > GMQ_NOALLOC_MAX_N) return GMQ_ERR_TOO_LARGE;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return fail_cuda();
  if (device < 0 || device >= ndev) return GMQ_ERR_INVALID;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return fail_cuda();
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return fail_cuda();
  gmq_status status = GMQ_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  if (!on_device(d_sum, device) || (n > 0 && !on_device(d_v, device))) {
    status = GMQ_ERR_INVALID;  // memory of another device, or host memory
  } else if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess) {
    status = fail_cuda();
  } else if (n == 0) {
    if (cudaMemsetAsync(d_sum, 0, sizeof(double), s) != cudaSuccess) status = fail_cuda();
  } else {
    gmq::DevStatus* st = (gmq::DevStatus*)base;
    double* partials = (double*)((unsigned char*)base + kStatusBytes);
    // the ticket must start at zero; clear it on the caller's stream
    if (cudaMemsetAsync(st, 0, sizeof(gmq::DevStatus), s) != cudaSuccess ||
        gmq::launch_tree_sum(d_v, n, partials, st, d_sum, s) != cudaSuccess)
      status = fail_cuda();
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return status;
}
