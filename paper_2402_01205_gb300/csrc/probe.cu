// Arithmetic-pipe probe used to state roofline fractions against measured
// peaks (declared in include/tpcfit_probe.h).
#include <cuda_runtime.h>

#include "tpcfit.h"
#include "tpcfit_probe.h"

namespace {

constexpr int kIters = 2048;

__global__ void k_dfma_chain(double *out, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int i = 0; i < kIters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_ffma_chain(float *out, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
        x7 = x0 + 7;
  for (int i = 0; i < 16 * kIters; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

extern "C" int tpcfit_probe_fma_rates(int device, double *fp64, double *fp32, int *clk) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return TPCFIT_E_NODEV;
  }
  if (cudaSetDevice(device) != cudaSuccess) return TPCFIT_E_CUDA;
  int sms = 0, khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
  const int threads = 256, blocks = sms * 8;
  const size_t n = (size_t)threads * blocks;
  void *buf = nullptr;
  if (cudaMalloc(&buf, n * sizeof(double)) != cudaSuccess) return TPCFIT_E_NOMEM;
  cudaStream_t s;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms64 = 0.f, ms32 = 0.f;
  for (int rep = 0; rep < 2; ++rep) {  // the first round warms up clocks and caches
    cudaEventRecord(e0, s);
    k_dfma_chain<<<blocks, threads, 0, s>>>((double *)buf, 0.999, 1e-3);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms64, e0, e1);
    cudaEventRecord(e0, s);
    k_ffma_chain<<<blocks, threads, 0, s>>>((float *)buf, 0.999f, 1e-3f);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms32, e0, e1);
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(buf);
  if (err != cudaSuccess) return TPCFIT_E_CUDA;
  if (fp64) *fp64 = (double)n * kIters * 8 / (ms64 * 1e-3);
  if (fp32) *fp32 = (double)n * 16 * kIters * 8 / (ms32 * 1e-3);
  if (clk) *clk = khz;
  return TPCFIT_OK;
}
