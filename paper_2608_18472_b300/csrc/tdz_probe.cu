// Device arithmetic rates that decide the mixed-precision design: the FP32 and binary64 fused
// multiply-add throughput of the current device, measured with eight independent FMA chains per thread
// over a grid of a few blocks per SM (CUDA events, best of three). On sm_103a binary64 runs at a small
// fraction of the FP32 rate, which is why the mixed path forms its binary64-class residuals in
// double-float (a pair of FP32 values) instead of in binary64.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "tdz_internal.h"

namespace tdz {
namespace {

constexpr int kChains = 8;

template <class T>
__global__ void k_fma_rate(T* out, T a, T b, int iters) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = v[c] * a + b;  // contracted to one FMA
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

template <class T>
double rate(int sms, int iters, int* err) {
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * 4096) != cudaSuccess) {
    *err = 1;
    return 0.0;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    k_fma_rate<T><<<blocks, threads>>>(out, (T)0.999999, (T)1e-7, iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      *err = 1;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3));  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return best;
}

}  // namespace
}  // namespace tdz

extern "C" int tdz_device_rates(double* fp32_flops, double* fp64_flops) {
  if (!fp32_flops || !fp64_flops) return TDZ_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    tdz::set_error("tdz_device_rates: no CUDA device");
    return TDZ_ECUDA;
  }
  int err = 0;
  *fp32_flops = tdz::rate<float>(sms, 4096, &err);   // ~40 ms per launch on B300
  *fp64_flops = tdz::rate<double>(sms, 256, &err);   // ~0.2 s per launch on B300
  if (err) {
    tdz::set_error(std::string("tdz_device_rates: ") + cudaGetErrorString(cudaGetLastError()));
    return TDZ_ECUDA;
  }
  return TDZ_OK;
}
