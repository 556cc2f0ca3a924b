// FMA-pipe probe for the roofline of the Krylov items kernel: independent FMA
// chains in FP32 and FP64, with all 32 lanes of every warp active and with one
// lane active. Prints one JSON line (TFLOP/s counted as 2 flops per FMA lane).
#include <cstdio>

#include <cuda_runtime.h>

template <typename T, int ACTIVE>
__global__ void fma_chains(T *out, int iters, T a, T b) {
  const int lane = threadIdx.x & 31;
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
    x7 = x0 + 7;
  if (lane < ACTIVE) {
    for (int i = 0; i < iters; ++i) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T, int ACTIVE>
double run_ms(int blocks, int threads, int iters) {
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T, ACTIVE><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);  // warm-up
  cudaEventRecord(e0);
  fma_chains<T, ACTIVE><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return ms;
}

int main() {
  int sms = 0, clk_khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  const int blocks = sms * 4, threads = 512;
  const int it32 = 4096, it64 = 512;
  const double lanes = (double)blocks * threads * 8;  // FMA chains
  const double t32 = run_ms<float, 32>(blocks, threads, it32), t32one = run_ms<float, 1>(blocks, threads, it32);
  const double t64 = run_ms<double, 32>(blocks, threads, it64), t64one = run_ms<double, 1>(blocks, threads, it64);
  const cudaError_t e = cudaGetLastError();
  printf("{\"sms\": %d, \"clock_mhz\": %.0f, \"fp32_tflops\": %.3f, \"fp64_tflops\": %.4f, "
         "\"fp32_ms_all_lanes\": %.4f, \"fp32_ms_one_lane\": %.4f, \"fp64_ms_all_lanes\": %.4f, "
         "\"fp64_ms_one_lane\": %.4f, \"status\": \"%s\"}\n",
         sms, clk_khz / 1e3, 2.0 * lanes * it32 / (t32 * 1e-3) / 1e12, 2.0 * lanes * it64 / (t64 * 1e-3) / 1e12, t32,
         t32one, t64, t64one, cudaGetErrorString(e));
  return e != cudaSuccess;
}
