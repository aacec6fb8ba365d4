// Peak-rate probe for the rooflines of the FP64 and FP32 kernels: a bounded loop of independent
// fused multiply-adds on every SM, timed with CUDA events. The paper has no counterpart; the
// measured rates are the denominators the benchmark reports its "alu" rooflines against.
#include "kkt_internal.cuh"

namespace kkt {
namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (hides the pipe latency)

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* __restrict__ sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = static_cast<T>(threadIdx.x + c) * static_cast<T>(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot drop, taken by no thread for these inputs
  if (s == static_cast<T>(-1.2345)) sink[blockIdx.x] = s;
}

template <typename T>
int run_probe(int iters, double* flops_per_s, cudaStream_t st) {
  int dev = 0, sms = 0;
  KKT_CUDA_TRY(cudaGetDevice(&dev));
  KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KKT_CUDA_TRY(cudaMalloc(&sink, blocks * sizeof(T)));
  KKT_CUDA_TRY(cudaEventCreate(&e0));
  KKT_CUDA_TRY(cudaEventCreate(&e1));
  const T a = static_cast<T>(0.999999), b = static_cast<T>(1e-7);
  fma_probe_kernel<T><<<blocks, threads, 0, st>>>(sink, iters / 8, a, b);   // warm-up
  float best = 0.f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0, st);
    fma_probe_kernel<T><<<blocks, threads, 0, st>>>(sink, iters, a, b);
    cudaEventRecord(e1, st);
    const cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0 || ms < best) best = ms;
  }
  const cudaError_t le = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  KKT_CUDA_TRY(le);
  const double fmas = static_cast<double>(blocks) * threads * iters * kChains;
  *flops_per_s = best > 0.f ? 2.0 * fmas / (best * 1e-3) : 0.0;
  return KKT_OK;
}

}  // namespace
}  // namespace kkt

using namespace kkt;

extern "C" int kkt_probe_fma_rate(int precision, double* flops_per_s, void* stream) {
  if (!flops_per_s || (precision != 0 && precision != 1))
    return set_error(KKT_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (FP32), flops_per_s non-null");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // about 20 ms per timed launch at this part's rates: 2^12 (FP64) or 2^18 (FP32) iterations
  return precision == 0 ? run_probe<double>(1 << 12, flops_per_s, st) : run_probe<float>(1 << 18, flops_per_s, st);
}
