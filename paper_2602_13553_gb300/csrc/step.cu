// step.cu -- the fused normal-mode integrator step of the PIMD method
// (Sec. IV.A; App. B normal modes; App. D PILE_L), FP64.
//
// One thread block owns a tile of A atoms with all P beads of every one of
// them staged in shared memory, so the three normal-mode transforms of a step
// (forces, positions forward; positions back) never leave the SM: the
// inter-bead communication of the paper's MPI design becomes shared-memory
// traffic.  Per step and atom tile the kernel reads x, v~, F once and writes
// x, v~ once, coalesced (every atom's P beads are contiguous per component).
//
// Tasks: thread (mode k, atom a) computes the three components of
//   F~_k = sum_j M[k][j] F_j and q~_k = sum_j M[k][j] x_j        (Eq. A1)
// applies B / A / O / A (BAOAB) or the pending B O of the previous step then
// O B A (OBABO) in registers, and stores v~; after a barrier, thread
// (bead j, atom a) forms x_j = sum_k M[k][j] q~_k (Eq. A3).
#include "common.cuh"

namespace pimd {

__device__ __forceinline__ void rotate(double &q, double &v, double c, double s_over_w, double w_s) {
  // exact flow of a free-ring-polymer mode for time tA:
  //   q' = cos q + sin/w v,  v' = -w sin q + cos v   (k = 0: q' = q + tA v)
  const double qn = fma(c, q, s_over_w * v);
  const double vn = fma(-w_s, q, c * v);
  q = qn;
  v = vn;
}

__global__ void __launch_bounds__(256) k_step_f64(StepArgs a) {
  extern __shared__ double sm[];
  const int P = a.P;
  const int tileLen = a.A * 3 * P;
  double *sX = sm;
  double *sV = sX + tileLen;
  double *sF = sV + tileLen;
  double *sQ = sF + tileLen;
  const int tile0 = blockIdx.x * a.A;
  const int na = min(a.A, a.N - tile0);
  const int len = na * 3 * P;
  const size_t base = (size_t)tile0 * 3 * P;
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    sX[t] = a.x[base + t];
    sV[t] = a.v[base + t];
    sF[t] = a.F[base + t];
  }
  __syncthreads();
  const uint64_t step = (uint64_t)(*a.step + a.step_off);
  const double *__restrict__ Mt = a.mt.Mt;
  for (int task = threadIdx.x; task < na * P; task += blockDim.x) {
    const int k = task % P;
    const int al = task / P;
    const int i = tile0 + al;
    const double *fx = sF + al * 3 * P;
    const double *xx = sX + al * 3 * P;
    double f0 = 0.0, f1 = 0.0, f2 = 0.0, q0 = 0.0, q1 = 0.0, q2 = 0.0;
    for (int j = 0; j < P; ++j) {
      const double m = __ldg(Mt + j * P + k);
      f0 = fma(m, fx[j], f0);
      f1 = fma(m, fx[P + j], f1);
      f2 = fma(m, fx[2 * P + j], f2);
      q0 = fma(m, xx[j], q0);
      q1 = fma(m, xx[P + j], q1);
      q2 = fma(m, xx[2 * P + j], q2);
    }
    const double *vv = sV + al * 3 * P;
    double v0 = vv[k], v1 = vv[P + k], v2 = vv[2 * P + k];
    const double im = __ldg(a.inv_mm + i);
    const double cA = __ldg(a.mt.cA + k), sA = __ldg(a.mt.sA + k), wsA = __ldg(a.mt.wsA + k);
    const double c1 = __ldg(a.mt.c1 + k), c2s = __ldg(a.mt.c2 + k) * __ldg(a.sigv + i);
    if (a.integrator == 0) {
      // B(h/2) of this step, merged with the final B(h/2) of the previous one
      const double kb = a.kick * im;
      v0 = fma(kb, f0, v0);
      v1 = fma(kb, f1, v1);
      v2 = fma(kb, f2, v2);
      rotate(q0, v0, cA, sA, wsA);
      rotate(q1, v1, cA, sA, wsA);
      rotate(q2, v2, cA, sA, wsA);
      if (a.thermo) {
        double e0, e1, e2;
        gauss3(a.seed, (uint32_t)i, (uint32_t)k, kStreamO1, step, e0, e1, e2);
        v0 = fma(c1, v0, c2s * e0);
        v1 = fma(c1, v1, c2s * e1);
        v2 = fma(c1, v2, c2s * e2);
      }
      rotate(q0, v0, cA, sA, wsA);
      rotate(q1, v1, cA, sA, wsA);
      rotate(q2, v2, cA, sA, wsA);
    } else {
      const double kb = a.half * im;
      if (!a.first) {
        // the previous step's closing B(h/2) O(h/2)
        v0 = fma(kb, f0, v0);
        v1 = fma(kb, f1, v1);
        v2 = fma(kb, f2, v2);
        if (a.thermo) {
          double e0, e1, e2;
          gauss3(a.seed, (uint32_t)i, (uint32_t)k, kStreamO2, step - 1, e0, e1, e2);
          v0 = fma(c1, v0, c2s * e0);
          v1 = fma(c1, v1, c2s * e1);
          v2 = fma(c1, v2, c2s * e2);
        }
      }
      if (a.thermo) {
        double e0, e1, e2;
        gauss3(a.seed, (uint32_t)i, (uint32_t)k, kStreamO1, step, e0, e1, e2);
        v0 = fma(c1, v0, c2s * e0);
        v1 = fma(c1, v1, c2s * e1);
        v2 = fma(c1, v2, c2s * e2);
      }
      v0 = fma(kb, f0, v0);
      v1 = fma(kb, f1, v1);
      v2 = fma(kb, f2, v2);
      rotate(q0, v0, cA, sA, wsA);
      rotate(q1, v1, cA, sA, wsA);
      rotate(q2, v2, cA, sA, wsA);
    }
    double *qq = sQ + al * 3 * P;
    qq[k] = q0;
    qq[P + k] = q1;
    qq[2 * P + k] = q2;
    double *vg = a.v + base + (size_t)al * 3 * P;
    vg[k] = v0;
    vg[P + k] = v1;
    vg[2 * P + k] = v2;
  }
  __syncthreads();
  const double *__restrict__ M = a.mt.M;
  for (int task = threadIdx.x; task < na * P; task += blockDim.x) {
    const int j = task % P;
    const int al = task / P;
    const double *qq = sQ + al * 3 * P;
    double x0 = 0.0, x1 = 0.0, x2 = 0.0;
    for (int k = 0; k < P; ++k) {
      const double m = __ldg(M + k * P + j);
      x0 = fma(m, qq[k], x0);
      x1 = fma(m, qq[P + k], x1);
      x2 = fma(m, qq[2 * P + k], x2);
    }
    double *xg = a.x + base + (size_t)al * 3 * P;
    xg[j] = x0;
    xg[P + j] = x1;
    xg[2 * P + j] = x2;
  }
}

// Closing kick of the last step of a call: B(h/2) (and, for OBABO, the final
// O(h/2) of that step), leaving v~ at integer time.
__global__ void __launch_bounds__(256) k_close_f64(StepArgs a) {
  extern __shared__ double sm[];
  const int P = a.P;
  double *sF = sm;
  const int tile0 = blockIdx.x * a.A;
  const int na = min(a.A, a.N - tile0);
  const int len = na * 3 * P;
  const size_t base = (size_t)tile0 * 3 * P;
  for (int t = threadIdx.x; t < len; t += blockDim.x) sF[t] = a.F[base + t];
  __syncthreads();
  const uint64_t step = (uint64_t)(*a.step + a.step_off);
  const double *__restrict__ Mt = a.mt.Mt;
  for (int task = threadIdx.x; task < na * P; task += blockDim.x) {
    const int k = task % P;
    const int al = task / P;
    const int i = tile0 + al;
    const double *fx = sF + al * 3 * P;
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    for (int j = 0; j < P; ++j) {
      const double m = __ldg(Mt + j * P + k);
      f0 = fma(m, fx[j], f0);
      f1 = fma(m, fx[P + j], f1);
      f2 = fma(m, fx[2 * P + j], f2);
    }
    double *vg = a.v + base + (size_t)al * 3 * P;
    const double kb = a.half * __ldg(a.inv_mm + i);
    double v0 = fma(kb, f0, vg[k]);
    double v1 = fma(kb, f1, vg[P + k]);
    double v2 = fma(kb, f2, vg[2 * P + k]);
    if (a.integrator == 1 && a.thermo) {
      const double c1 = __ldg(a.mt.c1 + k), c2s = __ldg(a.mt.c2 + k) * __ldg(a.sigv + i);
      double e0, e1, e2;
      gauss3(a.seed, (uint32_t)i, (uint32_t)k, kStreamO2, step, e0, e1, e2);
      v0 = fma(c1, v0, c2s * e0);
      v1 = fma(c1, v1, c2s * e1);
      v2 = fma(c1, v2, c2s * e2);
    }
    vg[k] = v0;
    vg[P + k] = v1;
    vg[2 * P + k] = v2;
  }
}

__global__ void k_advance(int64_t *step, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += n;
}

// Initial normal-mode velocities ~ N(0, P kB T / (m mvv2e)), noise stream 2.
__global__ void k_thermal_v(double *v, const double *sigv, uint64_t seed, int N, int P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * P) return;
  const int i = t / P, k = t % P;
  double e0, e1, e2;
  gauss3(seed, (uint32_t)i, (uint32_t)k, kStreamInit, 0ull, e0, e1, e2);
  const double s = sigv[i];
  v[((size_t)i * 3 + 0) * P + k] = s * e0;
  v[((size_t)i * 3 + 1) * P + k] = s * e1;
  v[((size_t)i * 3 + 2) * P + k] = s * e2;
}

// Layout changes between the host order [P][N][3] and the device order [N][3][P].
__global__ void k_pna_to_nap(const double *src, double *dst, int N, int P) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)N * 3 * P;
  if (t >= total) return;
  const int k = (int)(t % P);
  const size_t ia = t / P;
  const int a = (int)(ia % 3);
  const size_t i = ia / 3;
  dst[t] = src[((size_t)k * N + i) * 3 + a];
}

__global__ void k_nap_to_pna(const double *src, double *dst, int N, int P) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)N * 3 * P;
  if (t >= total) return;
  const int a = (int)(t % 3);
  const size_t ki = t / 3;
  const size_t i = ki % N;
  const int k = (int)(ki / N);
  dst[t] = src[(i * 3 + a) * P + k];
}

// --- host launchers --------------------------------------------------------
size_t step_smem_bytes(int A, int P) { return (size_t)4 * A * 3 * P * sizeof(double); }
size_t close_smem_bytes(int A, int P) { return (size_t)A * 3 * P * sizeof(double); }

cudaError_t launch_step(const StepArgs &a, int threads, cudaStream_t s) {
  const int grid = (a.N + a.A - 1) / a.A;
  k_step_f64<<<grid, threads, step_smem_bytes(a.A, a.P), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_close(const StepArgs &a, int threads, cudaStream_t s) {
  const int grid = (a.N + a.A - 1) / a.A;
  k_close_f64<<<grid, threads, close_smem_bytes(a.A, a.P), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *step, int n, cudaStream_t s) {
  k_advance<<<1, 32, 0, s>>>(step, n);
  return cudaGetLastError();
}

cudaError_t launch_thermal_v(double *v, const double *sigv, uint64_t seed, int N, int P,
                             cudaStream_t s) {
  const int total = N * P;
  k_thermal_v<<<(total + 255) / 256, 256, 0, s>>>(v, sigv, seed, N, P);
  return cudaGetLastError();
}

cudaError_t launch_pna_to_nap(const double *src, double *dst, int N, int P, cudaStream_t s) {
  const size_t total = (size_t)N * 3 * P;
  k_pna_to_nap<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(src, dst, N, P);
  return cudaGetLastError();
}

cudaError_t launch_nap_to_pna(const double *src, double *dst, int N, int P, cudaStream_t s) {
  const size_t total = (size_t)N * 3 * P;
  k_nap_to_pna<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(src, dst, N, P);
  return cudaGetLastError();
}

}  // namespace pimd
