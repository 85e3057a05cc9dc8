// Arithmetic-peak probe: the FP64 or FP32 fused multiply-add rate of the
// current device, measured with a loop of independent FMA chains. The
// transport passes in FP64 are bound by this rate (their arithmetic intensity
// is far above the FP64 ridge), so the probe gives their roofline denominator
// a measured counterpart to the one derived from unit counts and clocks.
#include <algorithm>

#include <cuda_runtime.h>

#include "ts_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads)
k_fma_probe(T* out, T a, T b, int iters) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + 1) * (T)(c + 1) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
ts_status probe(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ts::cuda_status(cudaGetLastError(), "ts_probe_fma_rate: device query");
  const int blocks = sms * kBlocksPerSM;
  const int iters = sizeof(T) == 8 ? 4096 : 131072;  // about 10 ms at the nominal rates
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * kProbeThreads);
  if (e != cudaSuccess) return ts::cuda_status(e, "ts_probe_fma_rate: cudaMalloc");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  const T a = (T)0.999999, b = (T)1e-6;  // contracting map: values stay near b / (1 - a)
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // rep 0 warms up
    e = cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, kProbeThreads, 0, st>>>(out, a, b, iters);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return ts::cuda_status(e, "ts_probe_fma_rate");
  const double flops = 2.0 * kChains * (double)iters * blocks * kProbeThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return TS_OK;
}

__global__ void k_widen_probe(const float* __restrict__ in, double* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = ts::widen_f32(in[i]);
}

}  // namespace

extern "C" ts_status ts_probe_widen(const float* in, double* out, size_t n, void* stream) {
  if ((!in || !out) && n) return ts::fail_status(TS_ERR_ARG, "ts_probe_widen: null pointer");
  if (n == 0) return TS_OK;
  const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
  k_widen_probe<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, out, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TS_OK : ts::cuda_status(e, "ts_probe_widen");
}

extern "C" ts_status ts_probe_fma_rate(int precision, double* tflops, void* stream) {
  if (!tflops) return ts::fail_status(TS_ERR_ARG, "ts_probe_fma_rate: null output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == TS_FP64) return probe<double>(tflops, st);
  if (precision == TS_FP32) return probe<float>(tflops, st);
  return ts::fail_status(TS_ERR_UNSUPPORTED, "ts_probe_fma_rate: precision must be TS_FP64 or TS_FP32");
}
