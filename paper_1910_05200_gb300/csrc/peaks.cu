// Roofline denominators measured on the running GPU: FP32 FMA throughput of
// the CUDA cores and streaming read bandwidth of the L2 cache.  The render
// and its gradient are bound by FP32 ALU work on data that stays in L2, so
// these two numbers, not the HBM copy rate, are the roofs its kernels are
// judged against.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/facert.h"

namespace {

constexpr int FMA_CHAINS = 8;      // independent FMA chains per thread
constexpr int FMA_THREADS = 256;
constexpr int FMA_BLOCKS_PER_SM = 8;

// Each thread advances FMA_CHAINS independent chains v <- v * a + b; a and b
// are runtime values, so nothing folds.  The sum is stored only when it hits
// a value it never takes, which keeps the chains live.
__global__ void __launch_bounds__(FMA_THREADS) k_fma_probe(int iters, float a, float b, float* __restrict__ sink) {
  float v[FMA_CHAINS];
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) v[k] = (float)threadIdx.x * 1e-3f + (float)k;
#pragma unroll 8
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) v[k] = fmaf(v[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) s += v[k];
  if (s == -1.0f) sink[blockIdx.x] = s;
}

// Grid-stride read of n4 float4 through L2 only (ld.global.cg), reps times.
__global__ void k_l2_probe(const float4* __restrict__ buf, long long n4, int reps, float* __restrict__ sink) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  float acc = 0.0f;
  for (int r = 0; r < reps; ++r)
    for (long long i = tid; i < n4; i += stride) {
      float4 q = __ldcg(buf + i);
      acc += q.x + q.y + q.z + q.w;
    }
  if (acc == -1.0f) sink[blockIdx.x] = acc;
}

}  // namespace

extern "C" int fr_probe_peaks(int32_t device, double* fp32_tflops, double* l2_read_gbs, int32_t* sm_count) {
  if (!fp32_tflops || !l2_read_gbs) return FR_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FR_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return FR_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return FR_ERR_CUDA;
  const int sms = prop.multiProcessorCount;
  if (sm_count) *sm_count = sms;
  const long long n4 = (32ll << 20) / 16;   // 32 MiB: resident in L2
  const int l2_blocks = sms * 8, l2_reps = 20;
  float4* buf = nullptr;
  float* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FR_OK;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == FR_OK) rc = (e == cudaErrorMemoryAllocation) ? FR_ERR_OOM : FR_ERR_CUDA;
    return rc == FR_OK;
  };
  if (ok(cudaMalloc(&buf, n4 * sizeof(float4))) && ok(cudaMalloc(&sink, sizeof(float) * std::max(l2_blocks,
                                                                   sms * FMA_BLOCKS_PER_SM))) &&
      ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) && ok(cudaEventCreate(&e0)) &&
      ok(cudaEventCreate(&e1)) && ok(cudaMemsetAsync(buf, 0, n4 * sizeof(float4), s))) {
    const int iters = 1 << 15;
    const int fma_blocks = sms * FMA_BLOCKS_PER_SM;
    double best = 0.0;
    for (int t = 0; t < 6 && rc == FR_OK; ++t) {      // the first run warms up the clocks
      ok(cudaEventRecord(e0, s));
      k_fma_probe<<<fma_blocks, FMA_THREADS, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
      ok(cudaGetLastError());
      ok(cudaEventRecord(e1, s));
      float ms = 0.0f;
      if (ok(cudaEventSynchronize(e1)) && ok(cudaEventElapsedTime(&ms, e0, e1)) && ms > 0.0f) {
        double flop = 2.0 * FMA_CHAINS * (double)iters * fma_blocks * FMA_THREADS;
        if (t > 0) best = std::max(best, flop / (ms * 1e-3) / 1e12);
      }
    }
    *fp32_tflops = best;
    double best_l2 = 0.0;
    for (int t = 0; t < 6 && rc == FR_OK; ++t) {
      ok(cudaEventRecord(e0, s));
      k_l2_probe<<<l2_blocks, 256, 0, s>>>(buf, n4, l2_reps, sink);
      ok(cudaGetLastError());
      ok(cudaEventRecord(e1, s));
      float ms = 0.0f;
      if (ok(cudaEventSynchronize(e1)) && ok(cudaEventElapsedTime(&ms, e0, e1)) && ms > 0.0f) {
        double bytes = (double)n4 * 16.0 * l2_reps;
        if (t > 0) best_l2 = std::max(best_l2, bytes / (ms * 1e-3) / 1e9);
      }
    }
    *l2_read_gbs = best_l2;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  return rc;
}
