// estimators.cu -- App. A outputs 1-10 reduced on the device, FP64.
//
// Pass 1 (k_est_f64): atom tiles with all P beads in shared memory, as in the
// step kernel.  Thread (k, a) forms q~_k = (M x)_k and adds
//   1/2 m |v~_k|^2            -> K^(k)   (output 1)
//   1/2 m w_n^2 lam_k |q~_k|^2 -> S^(k)   (output 2; sum_k S^(k) is the
//                                          ring's spring energy)
// and, as bead j = k, r^j . F^j and (r^j - r_c) . F^j (r_c = bead average).
// Per-mode sums over the tile's atoms are taken in a fixed order in shared
// memory, the scalars through a fixed shuffle tree, all compensated (CSum).
// One row of partials per block.
// Pass 2 (k_est_final): one block sums the rows in block order with
// Neumaier compensation, adds the per-bead U^(k) and Tr Xi^(k) rows of the
// force kernel and assembles the outputs; a NaN/Inf sets the error word.
#include "common.cuh"

namespace pimd {

__global__ void __launch_bounds__(256) k_est_f64(EstArgs a) {
  extern __shared__ double sm[];
  const int P = a.P;
  const int tileLen = a.A * 3 * P;
  double *sX = sm;
  double *sV = sX + tileLen;
  double *sF = sV + tileLen;
  double *sK = sF + tileLen;          // [A*P]
  double *sS = sK + a.A * P;          // [A*P]
  double *sC = sS + a.A * P;          // [A*3] centroids
  __shared__ CSum sred[3][8];
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
  for (int t = threadIdx.x; t < na * 3; t += blockDim.x) {
    const double *row = sX + t * P;
    double s = 0.0;
    for (int j = 0; j < P; ++j) s += row[j];
    sC[t] = s / P;
  }
  __syncthreads();
  CSum rF{0.0, 0.0}, rcF{0.0, 0.0}, mv0{0.0, 0.0};
  const double *__restrict__ Mt = a.mt.Mt;
  for (int task = threadIdx.x; task < a.A * P; task += blockDim.x) {
    const int k = task % P;
    const int al = task / P;
    double kk = 0.0, ss = 0.0;
    if (al < na) {
      const int i = tile0 + al;
      const double *xx = sX + al * 3 * P;
      const double *vv = sV + al * 3 * P;
      const double *ff = sF + al * 3 * P;
      double q0 = 0.0, q1 = 0.0, q2 = 0.0;
      for (int j = 0; j < P; ++j) {
        const double m = __ldg(Mt + j * P + k);
        q0 = fma(m, xx[j], q0);
        q1 = fma(m, xx[P + j], q1);
        q2 = fma(m, xx[2 * P + j], q2);
      }
      const double mm = __ldg(a.mass_mm + i);
      const double v0 = vv[k], v1 = vv[P + k], v2 = vv[2 * P + k];
      const double v2s = v0 * v0 + v1 * v1 + v2 * v2;
      kk = 0.5 * mm * __ldg(a.mt.mu + k) * v2s;   // fictitious mass m^(k)
      if (a.method == 0) {
        ss = 0.5 * mm * a.wn2 * __ldg(a.mt.lam + k) * (q0 * q0 + q1 * q1 + q2 * q2);
        if (k == 0) mv0.add(mm * __ldg(a.mt.mu) * v2s);
      } else {
        // Cartesian bead form of output 2, and v~^(0) = sum_k v^(k) / sqrt(P)
        const int km = k == 0 ? P - 1 : k - 1, kp = k == P - 1 ? 0 : k + 1;
        double s2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double *xr = xx + d * P;
          const double dm = xr[k] - xr[km], dp = xr[k] - xr[kp];
          s2 += dm * dm + dp * dp;
        }
        ss = 0.25 * mm * a.wn2 * s2;
        if (k == 0) {
          double w2 = 0.0;
          for (int d = 0; d < 3; ++d) {
            double sv = 0.0;
            for (int j = 0; j < P; ++j) sv += vv[d * P + j];
            w2 += sv * sv;
          }
          mv0.add(mm * __ldg(a.mt.mu) * w2 / P);
        }
      }
      // bead j = k
      const double x0 = xx[k], x1 = xx[P + k], x2 = xx[2 * P + k];
      const double f0 = ff[k], f1 = ff[P + k], f2 = ff[2 * P + k];
      rF.add(x0 * f0);
      rF.add(x1 * f1);
      rF.add(x2 * f2);
      rcF.add((x0 - sC[al * 3]) * f0);
      rcF.add((x1 - sC[al * 3 + 1]) * f1);
      rcF.add((x2 - sC[al * 3 + 2]) * f2);
    }
    sK[task] = kk;
    sS[task] = ss;
  }
  rF = warp_csum(rF);
  rcF = warp_csum(rcF);
  mv0 = warp_csum(mv0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sred[0][warp] = rF;
    sred[1][warp] = rcF;
    sred[2][warp] = mv0;
  }
  __syncthreads();
  const int W = 2 * P + 4;
  double *out = a.part + (size_t)blockIdx.x * W;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    CSum sk{0.0, 0.0}, sss{0.0, 0.0};
    for (int al = 0; al < na; ++al) {
      sk.add(sK[al * P + k]);
      sss.add(sS[al * P + k]);
    }
    out[k] = sk.value();
    out[P + k] = sss.value();
  }
  if (threadIdx.x < 3) {
    const int nw = (blockDim.x + 31) / 32;
    CSum s{0.0, 0.0};
    for (int w = 0; w < nw; ++w) s.add(sred[threadIdx.x][w]);
    out[2 * P + threadIdx.x] = s.value();
  }
  if (threadIdx.x == 3) out[2 * P + 3] = 0.0;
}

// Neumaier-compensated sum of a strided column.
__device__ double comp_sum(const double *p, int n, size_t stride) {
  double s = 0.0, c = 0.0;
  for (int b = 0; b < n; ++b) {
    const double x = p[(size_t)b * stride];
    const double t = s + x;
    if (fabs(s) >= fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  return s + c;
}

__global__ void k_est_final(EstFinalArgs a) {
  __shared__ double tot[2 * kMaxBeads + 4];
  __shared__ double U[kMaxBeads], Wv[kMaxBeads];
  const int P = a.P;
  const int W = 2 * P + 4;
  for (int s = threadIdx.x; s < W; s += blockDim.x) tot[s] = comp_sum(a.part + s, a.nblk_est, W);
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    U[k] = comp_sum(a.Upart + k, a.nblk_force, P);
    Wv[k] = comp_sum(a.Wpart + k, a.nblk_force, P);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double *o = a.out;
  double Ktot = 0.0, Stot = 0.0, Utot = 0.0, Wtot = 0.0;
  for (int k = 0; k < P; ++k) {
    o[k] = tot[k];
    o[P + k] = tot[P + k];
    o[2 * P + k] = U[k];
    Ktot += tot[k];
    Stot += tot[P + k];
    Utot += U[k];
    Wtot += Wv[k];
  }
  const double rF = tot[2 * P], rcF = tot[2 * P + 1], mv0 = tot[2 * P + 2];
  const double N = (double)a.N, Pd = (double)P, kT = a.kT;
  const double V = a.dbox ? a.dbox[0] * a.dbox[1] * a.dbox[2] : a.volume;
  const double spring = 2.0 * Stot;   // sum_k sum_i m w_n^2 |r^k - r^(k+1)|^2
  double *g = o + 3 * P;
  g[0] = Ktot + Stot + Utot;                                    // H
  g[1] = 1.5 * Pd * N * kT - 0.5 * spring / Pd;                 // K_PR
  g[2] = -rF / (2.0 * Pd);                                      // K_VR
  g[3] = 1.5 * N * kT - rcF / (2.0 * Pd);                       // K_CV
  if (V > 0.0) {
    g[4] = (3.0 * Pd * N * kT - spring / Pd + Wtot / Pd) / (3.0 * V);  // P_PR
    g[5] = (2.0 * Ktot + Wtot) / (3.0 * V);                            // P_MD
    g[6] = (mv0 - rcF + Wtot) / (3.0 * Pd * V);                        // P_CV
  } else {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    g[4] = g[5] = g[6] = nan;
  }
  g[7] = 2.0 * Ktot / (3.0 * N * Pd * a.kB);                   // T_ring
  g[8] = V;
  g[9] = Wtot;
  bool finite = isfinite(g[0]) && isfinite(g[1]) && isfinite(g[2]) && isfinite(g[3]);
  if (!finite) atomicOr(a.err, kErrNonFinite);
}

size_t est_smem_bytes(int A, int P) {
  return (size_t)(3 * A * 3 * P + 2 * A * P + 3 * A) * sizeof(double);
}

cudaError_t launch_est(const EstArgs &a, int threads, cudaStream_t s) {
  const int grid = (a.N + a.A - 1) / a.A;
  k_est_f64<<<grid, threads, est_smem_bytes(a.A, a.P), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_est_final(const EstFinalArgs &a, cudaStream_t s) {
  k_est_final<<<1, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pimd
