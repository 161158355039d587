// noise.cu -- the PILE_L noise of App. D exactly as the FP64 step kernels
// draw it, exposed for checking: the Philox-4x32-10 words and the three
// Box-Muller deviates of every (mode, atom) of one (seed, stream, step).
#include <cuda_runtime.h>

#include "common.cuh"
#include "pimd.h"
#include "runtime.h"

namespace pimd {

__global__ void k_noise_sample(uint64_t seed, uint32_t stream, uint64_t step, int N, int K, uint32_t *words,
                               double *eta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * K) return;
  const int k = t / N, i = t - k * N;
  if (words) {
    const uint4 w = philox4x32_10(
        make_uint4((uint32_t)i, ((uint32_t)k & 0xffffu) | (stream << 16), (uint32_t)step, (uint32_t)(step >> 32)),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    words[4 * (size_t)t + 0] = w.x;
    words[4 * (size_t)t + 1] = w.y;
    words[4 * (size_t)t + 2] = w.z;
    words[4 * (size_t)t + 3] = w.w;
  }
  if (eta) {
    double e0, e1, e2;
    gauss3(seed, (uint32_t)i, (uint32_t)k, stream, step, e0, e1, e2);
    eta[3 * (size_t)t + 0] = e0;
    eta[3 * (size_t)t + 1] = e1;
    eta[3 * (size_t)t + 2] = e2;
  }
}

}  // namespace pimd

using namespace pimd;

extern "C" pimd_status pimd_noise_sample(uint64_t seed, uint32_t stream, uint64_t step, int32_t n_atoms,
                                         int32_t n_modes, uint32_t *words, double *eta) {
  if (n_atoms < 1 || n_modes < 1 || n_modes > 65536 || (int64_t)n_atoms * n_modes > (1 << 24) || stream > 0xffffu)
    return fail(PIMD_EINVAL, "pimd_noise_sample: need 1 <= n_atoms, 1 <= n_modes <= 65536, "
                             "n_atoms * n_modes <= 2^24, stream < 65536");
  const size_t n = (size_t)n_atoms * n_modes;
  uint32_t *dw = nullptr;
  double *de = nullptr;
  cudaError_t e = cudaSuccess;
  if (words) e = cudaMalloc(&dw, n * 4 * sizeof(uint32_t));
  if (e == cudaSuccess && eta) e = cudaMalloc(&de, n * 3 * sizeof(double));
  if (e == cudaSuccess) {
    k_noise_sample<<<(unsigned)((n + 255) / 256), 256>>>(seed, stream, step, n_atoms, n_modes, dw, de);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && words) e = cudaMemcpy(words, dw, n * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && eta) e = cudaMemcpy(eta, de, n * 3 * sizeof(double), cudaMemcpyDeviceToHost);
  if (dw) cudaFree(dw);
  if (de) cudaFree(de);
  if (e != cudaSuccess) return fail(PIMD_ECUDA, "pimd_noise_sample: %s", cudaGetErrorString(e));
  return PIMD_OK;
}
