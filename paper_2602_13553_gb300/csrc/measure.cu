// measure.cu -- the FP64 FMA throughput of the device, measured with CUDA
// events: the peak against which the FP64 kernels' arithmetic is reported.
#include <cuda_runtime.h>

#include "pimd.h"
#include "runtime.h"

namespace pimd {

// Eight independent FMA chains per thread (enough to cover the pipe's
// latency); x <- x m + c converges to c / (1 - m), so nothing overflows and
// the final store keeps the chains live.
__global__ void __launch_bounds__(256) k_fma64(int iters, double m, double c, double *out) {
  double a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = (double)(threadIdx.x + q);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace pimd

using namespace pimd;

extern "C" pimd_status pimd_fp64_fma_rate(int32_t iters, double *tflops) {
  if (!tflops || iters < 1) return fail(PIMD_EINVAL, "pimd_fp64_fma_rate: need iters >= 1 and an output");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(PIMD_ECUDA, "pimd_fp64_fma_rate: %s", cudaGetErrorString(e));
  const int blocks = 4 * nsm, threads = 256;
  double *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaMalloc(&out, sizeof(double) * blocks * threads)) != cudaSuccess)
    return fail(PIMD_ENOMEM, "pimd_fp64_fma_rate: %s", cudaGetErrorString(e));
  float ms = 0.f;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fma64<<<blocks, threads>>>(iters, 0.999999, 1e-6, out);   // warm-up
    cudaEventRecord(e0);
    k_fma64<<<blocks, threads>>>(iters, 0.999999, 1e-6, out);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return fail(PIMD_ECUDA, "pimd_fp64_fma_rate: %s", cudaGetErrorString(e));
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return PIMD_OK;
}
