// fma_probe.cu -- floating-point issue-rate probe: the measured peak that
// the rule kernels' rooflines are reported against (a measurement aid; the
// paper has no counterpart).
//
// Every thread runs kChains independent chains of one operation for `iters`
// iterations: x <- x * a + b (fused multiply-add), x <- x + b or x <- x * a;
// a and b are kernel arguments, so nothing folds, and every chain's result
// is stored, so nothing is dead.  With 16 chains per thread and up to 64
// warps per SM there are far more independent operations in flight than the
// pipe's latency needs: the launch measures the pipe's issue rate alone.
#include "sweep_kernels.cuh"

namespace gmq {
namespace {

constexpr int kChains = 16;

template <class T, int OP>
__global__ void __launch_bounds__(kProbeBlock) k_fma_probe(int64_t iters, T a, T b, T* sink) {
  T x[kChains];
  const T seed = (T)(threadIdx.x + 1) * (T)1e-3;
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed + (T)i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if constexpr (OP == 0)
        x[i] = fma(x[i], a, b);
      else if constexpr (OP == 1)
        x[i] = x[i] + b;
      else
        x[i] = x[i] * a;
    }
  }
  T s = x[0];
#pragma unroll
  for (int i = 1; i < kChains; ++i) s += x[i];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

template <class T>
void launch_probe_t(int op, int blocks, int64_t iters, T a, T b, T* sink, cudaStream_t s) {
  if (op == 0)
    k_fma_probe<T, 0><<<blocks, kProbeBlock, 0, s>>>(iters, a, b, sink);
  else if (op == 1)
    k_fma_probe<T, 1><<<blocks, kProbeBlock, 0, s>>>(iters, a, b, sink);
  else
    k_fma_probe<T, 2><<<blocks, kProbeBlock, 0, s>>>(iters, a, b, sink);
}

cudaError_t launch_fma_probe(int fp64, int op, int blocks, int64_t iters, void* sink,
                             cudaStream_t s) {
  if (op < 0 || op > 2) return cudaErrorInvalidValue;
  if (fp64)
    launch_probe_t<double>(op, blocks, iters, 0.999999999, 1e-9, (double*)sink, s);
  else
    launch_probe_t<float>(op, blocks, iters, 0.9999999f, 1e-7f, (float*)sink, s);
  return cudaGetLastError();
}

int64_t fma_probe_lane_fmas(int blocks, int64_t iters) {
  return (int64_t)blocks * kProbeBlock * iters * kChains;
}

}  // namespace gmq
