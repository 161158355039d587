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
// Tasks: thread (mode k, component d, atom a) forms
//   F~_k = sum_j M[k][j] F_j and q~_k = sum_j M[k][j] x_j        (Eq. A1)
// applies B / A / O / A (BAOAB) or the pending B O of the previous step then
// O B A (OBABO) in registers, and stores v~; after a barrier, thread
// (bead j, component d, atom a) forms x_j = sum_k M[k][j] q~_k (Eq. A3).
// For water-like systems the same kernel also measures, per oxygen, the
// centroid drift since the last neighbour-list build and the bead spread.
#include "common.cuh"

#include <algorithm>

namespace pimd {

__device__ __forceinline__ void rotate(double &q, double &v, double c, double s_over_w, double w_s) {
  // exact flow of a free-ring-polymer mode for time tA:
  //   q' = cos q + sin/w v,  v' = -w sin q + cos v   (k = 0: q' = q + tA v)
  const double qn = fma(c, q, s_over_w * v);
  const double vn = fma(-w_s, q, c * v);
  q = qn;
  v = vn;
}

// Centroid mode under the barostat for time tA at v_W (App. E):
//   q~0 <- e^a q~0 + (e^a - e^-a) / (2 v_W) v~0,  v~0 <- e^-a v~0,  a = tA v_W
__device__ __forceinline__ void baro_drift(double &q, double &v, double vW, double tA) {
  const double a = tA * vW;
  const double ea = exp(a), ema = exp(-a);
  const double sh = fabs(a) < 1e-8 ? tA * (1.0 + a * a / 6.0) : (ea - ema) / (2.0 * vW);
  q = ea * q + sh * v;
  v = ema * v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Thread task t = (al * 3 + d) * P + k: atom al of the tile, component d,
// mode k (forward) or bead j = k (inverse).  This is also the offset of the
// element in the tile, so loads, stores and shared memory share one index.
// The transforms use the parity of the rows of M (Eq. A1) under j -> P - j:
// modes k <= H = floor(P/2) (constant, cosine and alternating rows) are even,
// the sine rows k > H odd.  Staging each row folded -- u_j = x_j + x_{P-j}
// and u_{P-j} = x_j - x_{P-j} for 0 < j < P - j, x_0 and x_{P/2} kept --
// makes every forward output a sum over one half of the row (Tf), and every
// inverse pair x_j, x_{P-j} = C_j +- S_j of an even-mode sum C_j and an
// odd-mode sum S_j (Ti): about P/2 FMAs per output instead of P.
__global__ void __launch_bounds__(256) k_step_f64(StepArgs a) {
  extern __shared__ double sm[];
  const int P = a.P;
  const int tileLen = a.A * 3 * P;
  double *sX = sm;
  double *sV = sX + tileLen;
  double *sF = sV + tileLen;
  double *sQ = sF + tileLen;
  double *sE = sQ + tileLen;     // PILE_L deviates of this step, stream O1, per element
  double *sE2 = sE + tileLen;    // OBABO: stream O2 of the previous step
  __shared__ float sred[2][8];
  const int tile0 = blockIdx.x * a.A;
  const int na = min(a.A, a.N - tile0);
  const int len = na * 3 * P;
  const size_t base = (size_t)tile0 * 3 * P;
  const int H = P >> 1;
  // stage the tile's x, F and v~ once each (16-byte loads where the tile
  // starts on an even element: it is contiguous in [N][3][P])
  if ((base & 1) == 0) {
    const double2 *__restrict__ x2 = reinterpret_cast<const double2 *>(a.x + base);
    const double2 *__restrict__ f2 = reinterpret_cast<const double2 *>(a.F + base);
    const double2 *__restrict__ v2 = reinterpret_cast<const double2 *>(a.v + base);
    for (int t = threadIdx.x; t < (len >> 1); t += blockDim.x) {
      const double2 xv = x2[t], fv = f2[t], vv = v2[t];
      sX[2 * t] = xv.x;
      sX[2 * t + 1] = xv.y;
      sF[2 * t] = fv.x;
      sF[2 * t + 1] = fv.y;
      sV[2 * t] = vv.x;
      sV[2 * t + 1] = vv.y;
    }
    if ((len & 1) && threadIdx.x == 0) {
      sX[len - 1] = a.x[base + len - 1];
      sF[len - 1] = a.F[base + len - 1];
      sV[len - 1] = a.v[base + len - 1];
    }
  } else {
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
      sX[t] = a.x[base + t];
      sF[t] = a.F[base + t];
      sV[t] = a.v[base + t];
    }
  }
  __syncthreads();
  // fold each staged row in place: (x_j, x_{P-j}) -> (x_j + x_{P-j}, x_j - x_{P-j})
  // for 0 < j < P - j, one thread per pair
  {
    const int hp = (P - 1) >> 1;   // pairs per row
    for (int t = threadIdx.x; t < na * 3 * hp; t += blockDim.x) {
      const int r = t / hp, j = t - r * hp + 1;
      double *xr = sX + r * P, *fr = sF + r * P;
      const double xa = xr[j], xb = xr[P - j], fa = fr[j], fb = fr[P - j];
      xr[j] = xa + xb;
      xr[P - j] = xa - xb;
      fr[j] = fa + fb;
      fr[P - j] = fa - fb;
    }
  }
  const uint64_t step = (uint64_t)(*a.step + a.step_off);
  // Large grids: one Philox draw and Box-Muller per (atom, mode) serve the
  // three components (throughput).  Small grids (noise_pre = 0): each element
  // draws its own component inline, in parallel with the others (latency).
  if (a.thermo && a.noise_pre && a.phase != 2) {
    const bool o2 = a.integrator == 1 && !a.first;
    for (int t = threadIdx.x; t < na * P; t += blockDim.x) {
      const int al = t / P, k = t - al * P;
      const int e = al * 3 * P + k;
      gauss3(a.seed, (uint32_t)(tile0 + al), (uint32_t)k, kStreamO1, step, sE[e], sE[e + P], sE[e + 2 * P]);
      if (o2)
        gauss3(a.seed, (uint32_t)(tile0 + al), (uint32_t)k, kStreamO2, step - 1, sE2[e], sE2[e + P],
               sE2[e + 2 * P]);
    }
  }
  __syncthreads();
  const double *__restrict__ Tf = a.mt.Tf;
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int k = task % P;
    const int r = task / P;
    const int i = tile0 + r / 3;
    auto noise = [&](uint32_t stream, uint64_t st, const double *pre) {
      return a.noise_pre ? pre[task] : gauss1(a.seed, (uint32_t)i, (uint32_t)k, stream, st, r % 3);
    };
    // F~_k = (M F)_k and q~_k = (M x)_k over the even (k <= H) or odd half
    // of the folded row, two independent chains each
    const bool even = k <= H;
    const int n = even ? H + 1 : P - H - 1;
    const double *fx = sF + r * P + (even ? 0 : H + 1);
    const double *xx = sX + r * P + (even ? 0 : H + 1);
    const double *tf = Tf + k;
    double fa = 0.0, fb = 0.0, qa = 0.0, qb = 0.0;
    int j = 0;
    for (; j + 1 < n; j += 2) {
      const double m0 = __ldg(tf + j * P), m1 = __ldg(tf + (j + 1) * P);
      fa = fma(m0, fx[j], fa);
      fb = fma(m1, fx[j + 1], fb);
      qa = fma(m0, xx[j], qa);
      qb = fma(m1, xx[j + 1], qb);
    }
    if (j < n) {
      const double m0 = __ldg(tf + j * P);
      fa = fma(m0, fx[j], fa);
      qa = fma(m0, xx[j], qa);
    }
    const double f = fa + fb;
    double q = qa + qb;
    double v = sV[task];
    const double im = __ldg(a.inv_mm + i) * __ldg(a.mt.imu + k);   // 1 / (m^(k) mvv2e)
    const double cA = __ldg(a.mt.cA + k), sA = __ldg(a.mt.sA + k), wsA = __ldg(a.mt.wsA + k);
    const double c1 = __ldg(a.mt.c1 + k), c2s = __ldg(a.mt.c2 + k) * __ldg(a.sigv + i);
    if (a.integrator == 0) {
      // B(h/2) of this step, merged with the final B(h/2) of the previous one
      v = fma(a.kick * im, f, v);
      if (k == 0 && a.baro) {   // the centroid rides on the barostat
        baro_drift(q, v, a.baro[kBaroVA1 + r % 3], a.half);
        if (a.thermo) v = fma(c1, v, c2s * noise(kStreamO1, step, sE));
        baro_drift(q, v, a.baro[kBaroVA2 + r % 3], a.half);
      } else {
        rotate(q, v, cA, sA, wsA);
        if (a.thermo) v = fma(c1, v, c2s * noise(kStreamO1, step, sE));
        rotate(q, v, cA, sA, wsA);
      }
    } else {
      const double kb = a.half * im;
      if (a.phase != 2) {
        if (!a.first) {
          // the previous step's closing B(h/2) O(h/2)
          v = fma(kb, f, v);
          if (a.thermo) v = fma(c1, v, c2s * noise(kStreamO2, step - 1, sE2));
        }
        if (a.thermo) v = fma(c1, v, c2s * noise(kStreamO1, step, sE));
      }
      if (a.phase != 1) {
        v = fma(kb, f, v);
        if (k == 0 && a.baro)   // A(h) of the centroid under the barostat
          baro_drift(q, v, a.baro[kBaroVA1 + r % 3], 2.0 * a.half);
        else
          rotate(q, v, cA, sA, wsA);
      }
    }
    sQ[task] = q;
    a.v[base + task] = v;
  }
  if (a.phase == 1) return;   // velocities only: the barostat's B_W reads them next
  __syncthreads();
  // inverse, first half: C_j (bead j <= H, even modes) or S_{P-j} (bead
  // j > H, odd modes) into sF, which the forward pass no longer needs
  const double *__restrict__ Ti = a.mt.Ti;
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int j = task % P;
    const bool even = j <= H;
    const int n = even ? H + 1 : P - H - 1;
    const double *qq = sQ + (task - j) + (even ? 0 : H + 1);
    const double *ti = Ti + j;
    double xa = 0.0, xb = 0.0;
    int k = 0;
    for (; k + 1 < n; k += 2) {
      xa = fma(__ldg(ti + k * P), qq[k], xa);
      xb = fma(__ldg(ti + (k + 1) * P), qq[k + 1], xb);
    }
    if (k < n) xa = fma(__ldg(ti + k * P), qq[k], xa);
    sF[task] = xa + xb;
  }
  __syncthreads();
  // second half: x_j = C_j + S_j (j <= H), x_{P-j} = C_j - S_j
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int j = task % P, pj = j == 0 ? 0 : P - j;
    const int row0 = task - j;
    const double xn = j <= H ? sF[task] + (pj > H ? sF[row0 + pj] : 0.0) : sF[row0 + pj] - sF[task];
    a.x[base + task] = xn;
    if (a.x32) a.x32[base + task] = (float)xn;
    sX[task] = xn;
  }
  if (!a.blkmax) return;
  // Neighbour-list skin check for the oxygens of this tile: centroid
  // c = q~_0 / sqrt(P), its drift since the last build and the bead spread.
  // Tiles without an oxygen report zero at once.  The differences are taken
  // in FP64, their squares and the maxima in FP32 (the FP64 pipe is the
  // scarce unit; a relative margin keeps the reported bound conservative).
  if ((tile0 + 2) / 3 * 3 >= tile0 + na) {
    if (threadIdx.x < 2) a.blkmax[2 * blockIdx.x + threadIdx.x] = 0.0;
    return;
  }
  __syncthreads();
  float vdisp = 0.f, vdev = 0.f;
  const double rsp = rsqrt((double)P);
  for (int t = threadIdx.x; t < na * P; t += blockDim.x) {
    const int al = t / P, k = t % P;
    const int i = tile0 + al;
    if (i % 3) continue;
    const double *xq = sQ + al * 3 * P;
    const double c0 = xq[0] * rsp, c1 = xq[P] * rsp, c2 = xq[2 * P] * rsp;
    const double *xs = sX + al * 3 * P;
    const float e0 = (float)(xs[k] - c0), e1 = (float)(xs[P + k] - c1), e2 = (float)(xs[2 * P + k] - c2);
    vdev = fmaxf(vdev, e0 * e0 + e1 * e1 + e2 * e2);
    if (k == 0) {
      const int m = i / 3;
      const float g0 = (float)(c0 - a.cref[3 * m]), g1 = (float)(c1 - a.cref[3 * m + 1]);
      const float g2 = (float)(c2 - a.cref[3 * m + 2]);
      vdisp = fmaxf(vdisp, g0 * g0 + g1 * g1 + g2 * g2);
      a.ccur[3 * m] = c0;
      a.ccur[3 * m + 1] = c1;
      a.ccur[3 * m + 2] = c2;
    }
  }
  // NaN positions force a rebuild (and fail later at a synchronising call)
  if (vdisp != vdisp) vdisp = __int_as_float(0x7f800000);
  if (vdev != vdev) vdev = __int_as_float(0x7f800000);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vdisp = fmaxf(vdisp, __shfl_down_sync(0xffffffffu, vdisp, o));
    vdev = fmaxf(vdev, __shfl_down_sync(0xffffffffu, vdev, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sred[0][threadIdx.x >> 5] = vdisp;
    sred[1][threadIdx.x >> 5] = vdev;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float mx = 0.f;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) mx = fmaxf(mx, sred[threadIdx.x][w]);
    a.blkmax[2 * blockIdx.x + threadIdx.x] = mx <= 3.0e38f ? sqrt((double)mx) * (1.0 + 1e-6) : 1e300;
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
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int k = task % P;
    const int r = task / P;
    const int d = r % 3;
    const int i = tile0 + r / 3;
    const double *fx = sF + r * P;
    double fa = 0.0, fb = 0.0;
    int j = 0;
    for (; j + 1 < P; j += 2) {
      fa = fma(__ldg(Mt + j * P + k), fx[j], fa);
      fb = fma(__ldg(Mt + (j + 1) * P + k), fx[j + 1], fb);
    }
    if (j < P) fa = fma(__ldg(Mt + j * P + k), fx[j], fa);
    double v = fma(a.half * (__ldg(a.inv_mm + i) * __ldg(a.mt.imu + k)), fa + fb, a.v[base + task]);
    if (a.integrator == 1 && a.thermo) {
      const double c1 = __ldg(a.mt.c1 + k), c2s = __ldg(a.mt.c2 + k) * __ldg(a.sigv + i);
      v = fma(c1, v, c2s * gauss1(a.seed, (uint32_t)i, (uint32_t)k, kStreamO2, step, d));
    }
    a.v[base + task] = v;
  }
}

// ---- Cartesian method (Sec. III.C "method pimd") ---------------------------
// Bead velocities v; the springs of Eq. (1) enter the kicks as forces
// F_s^(k) = -m w_n^2 (2 x^k - x^(k-1) - x^(k+1)) (cyclic); A is the free drift
// x += tA v; O (App. D) acts on every bead with one friction.  Thread task
// t = (al * 3 + d) * P + k as in the normal-mode kernel.
__device__ __forceinline__ double spring_force(const double *row, int k, int P, double mmw2) {
  const double xm = row[k == 0 ? P - 1 : k - 1], xp = row[k == P - 1 ? 0 : k + 1];
  return -mmw2 * (2.0 * row[k] - xm - xp);
}

__global__ void __launch_bounds__(256) k_step_cart_f64(StepArgs a) {
  extern __shared__ double sm[];
  const int P = a.P;
  const int tileLen = a.A * 3 * P;
  double *sX = sm;               // positions at the start of the step
  double *sN = sX + tileLen;     // new positions
  double *sE = sN + tileLen;     // PILE_L deviates, stream O1, per element
  double *sE2 = sE + tileLen;    // OBABO: stream O2 of the previous step
  double *sC = sE2 + tileLen;    // [A][3] new centroids (water skin check)
  __shared__ double sred[2][8];
  const int tile0 = blockIdx.x * a.A;
  const int na = min(a.A, a.N - tile0);
  const int len = na * 3 * P;
  const size_t base = (size_t)tile0 * 3 * P;
  for (int t = threadIdx.x; t < len; t += blockDim.x) sX[t] = a.x[base + t];
  const uint64_t step = (uint64_t)(*a.step + a.step_off);
  if (a.thermo && a.noise_pre) {   // one Philox draw per (atom, bead) serves the three components
    const bool o2 = a.integrator == 1 && !a.first;
    for (int t = threadIdx.x; t < na * P; t += blockDim.x) {
      const int al = t / P, k = t - al * P;
      const int e = al * 3 * P + k;
      gauss3(a.seed, (uint32_t)(tile0 + al), (uint32_t)k, kStreamO1, step, sE[e], sE[e + P], sE[e + 2 * P]);
      if (o2)
        gauss3(a.seed, (uint32_t)(tile0 + al), (uint32_t)k, kStreamO2, step - 1, sE2[e], sE2[e + P],
               sE2[e + 2 * P]);
    }
  }
  __syncthreads();
  const double c1 = __ldg(a.mt.c1), c2 = __ldg(a.mt.c2);
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int k = task % P;
    const int r = task / P;
    const int i = tile0 + r / 3;
    auto noise = [&](uint32_t stream, uint64_t st, const double *pre) {
      return a.noise_pre ? pre[task] : gauss1(a.seed, (uint32_t)i, (uint32_t)k, stream, st, r % 3);
    };
    const double f = a.F[base + task] + spring_force(sX + r * P, k, P, __ldg(a.mass_mm + i) * a.wn2);
    const double im = __ldg(a.inv_mm + i) * a.ifmass;
    const double c2s = c2 * __ldg(a.sigv + i);
    double v = a.v[base + task];
    double x = sX[task];
    if (a.integrator == 0) {
      v = fma(a.kick * im, f, v);
      x = fma(a.half, v, x);
      if (a.thermo) v = fma(c1, v, c2s * noise(kStreamO1, step, sE));
      x = fma(a.half, v, x);
    } else {
      const double kb = a.half * im;
      if (!a.first) {
        v = fma(kb, f, v);
        if (a.thermo) v = fma(c1, v, c2s * noise(kStreamO2, step - 1, sE2));
      }
      if (a.thermo) v = fma(c1, v, c2s * noise(kStreamO1, step, sE));
      v = fma(kb, f, v);
      x = fma(2.0 * a.half, v, x);
    }
    a.v[base + task] = v;
    a.x[base + task] = x;
    if (a.x32) a.x32[base + task] = (float)x;
    sN[task] = x;
  }
  if (!a.blkmax) return;
  // neighbour-list skin check of the oxygens: centroid = bead mean
  __syncthreads();
  for (int t = threadIdx.x; t < na * 3; t += blockDim.x) {
    const double *row = sN + t * P;
    double sum = 0.0;
    for (int j = 0; j < P; ++j) sum += row[j];
    sC[t] = sum / P;
  }
  __syncthreads();
  double vdisp = 0.0, vdev = 0.0;
  for (int t = threadIdx.x; t < na * P; t += blockDim.x) {
    const int al = t / P, k = t % P;
    const int i = tile0 + al;
    if (i % 3) continue;
    const double c0 = sC[al * 3], cc1 = sC[al * 3 + 1], cc2 = sC[al * 3 + 2];
    const double *xs = sN + al * 3 * P;
    const double e0 = xs[k] - c0, e1 = xs[P + k] - cc1, e2 = xs[2 * P + k] - cc2;
    vdev = fmax(vdev, e0 * e0 + e1 * e1 + e2 * e2);
    if (k == 0) {
      const int m = i / 3;
      const double g0 = c0 - a.cref[3 * m], g1 = cc1 - a.cref[3 * m + 1], g2 = cc2 - a.cref[3 * m + 2];
      vdisp = fmax(vdisp, g0 * g0 + g1 * g1 + g2 * g2);
      a.ccur[3 * m] = c0;
      a.ccur[3 * m + 1] = cc1;
      a.ccur[3 * m + 2] = cc2;
    }
  }
  vdisp = warp_max(vdisp);
  vdev = warp_max(vdev);
  if ((threadIdx.x & 31) == 0) {
    sred[0][threadIdx.x >> 5] = vdisp;
    sred[1][threadIdx.x >> 5] = vdev;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double mx = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) mx = fmax(mx, sred[threadIdx.x][w]);
    a.blkmax[2 * blockIdx.x + threadIdx.x] = (mx == mx) ? sqrt(mx) : 1e300;
  }
}

// Closing kick of a call, Cartesian: B(h/2) with the springs (and the final
// O(h/2) of OBABO).
__global__ void __launch_bounds__(256) k_close_cart_f64(StepArgs a) {
  const int P = a.P;
  const size_t total = (size_t)a.N * 3 * P;
  const uint64_t step = (uint64_t)(*a.step + a.step_off);
  const double c1 = __ldg(a.mt.c1), c2 = __ldg(a.mt.c2);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % P);
    const size_t r = t / P;
    const int d = (int)(r % 3);
    const int i = (int)(r / 3);
    const double f = a.F[t] + spring_force(a.x + r * P, k, P, __ldg(a.mass_mm + i) * a.wn2);
    double v = fma(a.half * (__ldg(a.inv_mm + i) * a.ifmass), f, a.v[t]);
    if (a.integrator == 1 && a.thermo)
      v = fma(c1, v, c2 * __ldg(a.sigv + i) * gauss1(a.seed, (uint32_t)i, (uint32_t)k, kStreamO2, step, d));
    a.v[t] = v;
  }
}

// fixcom: one block; deterministic sums (fixed per-thread strides, then a
// fixed tree) of m v, F and (Cartesian) m x per (bead or centroid mode,
// component), then v -= u on every atom.
__device__ double block_sum(double v, double *red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_fixcom_f64(FixcomArgs a) {
  __shared__ double red[256];
  __shared__ double sp[3 * kMaxBeads], sf[3 * kMaxBeads], sx[3 * kMaxBeads], u[3 * kMaxBeads];
  const int P = a.P, N = a.N;
  const int nb = a.method == 0 ? 1 : P;
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) m += a.mass_mm[i];
  const double msum = block_sum(m, red);
  for (int kc = 0; kc < 3 * nb; ++kc) {
    const int k = kc / 3, c = kc % 3;
    double pv = 0.0, pf = 0.0, px = 0.0, pn = 0.0;
    const uint64_t s = (uint64_t)(*a.step - 1);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const size_t row = ((size_t)i * 3 + c) * P;
      const double mm = a.mass_mm[i];
      pv = fma(mm, a.v[row + k], pv);
      if (a.obabo_thermo)
        pn = fma(mm * a.sigv[i], gauss1(a.seed, (uint32_t)i, (uint32_t)k, kStreamO2, s, c), pn);
      if (a.method == 0) {
        double fs = 0.0;   // sqrt(P) F~_0 = sum over beads
        for (int j = 0; j < P; ++j) fs += a.F[row + j];
        pf += fs;
      } else {
        pf += a.F[row + k];
        px = fma(mm, a.x[row + k], px);
      }
    }
    pv = block_sum(pv, red);
    pf = block_sum(pf, red);
    px = block_sum(px, red);
    pn = block_sum(pn, red);
    if (threadIdx.x == 0) {
      // the closing O(h/2) scales by c1 and adds c2 sigv eta: remove its mean too
      sp[kc] = a.obabo_thermo ? pv + a.c2[k] * pn / a.c1[k] : pv;
      sf[kc] = a.method == 0 ? pf / sqrt((double)P) : pf;
      sx[kc] = px;
    }
  }
  __syncthreads();
  for (int kc = threadIdx.x; kc < 3 * nb; kc += blockDim.x) {
    const int k = kc / 3, c = kc % 3;
    double f = sf[kc];
    if (a.method == 1) {
      const int km = k == 0 ? P - 1 : k - 1, kp = k == P - 1 ? 0 : k + 1;
      f -= a.wn2 * (2.0 * sx[kc] - sx[3 * km + c] - sx[3 * kp + c]);
    }
    u[kc] = fma(a.half * a.imu0, f, sp[kc]) / msum;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N * 3 * nb; t += blockDim.x) {
    const int k = t % nb;
    const int ic = t / nb;
    a.v[(size_t)ic * P + k] -= u[3 * k + ic % 3];
  }
}

// B_W of the BZP barostat (App. E) over [t0, t0 + tB] of the kick that the
// next kernel applies to the current velocities, with n = P.  Isotropic:
//   v_W += (3 tB / W)[n V P_CV - n V P_ext + n kB T] + (tB^2 / W) sum F~0.v~0
//          + (tB^3 / 3W) sum |F~0|^2 / m~0,
//   3 n V P_CV = sum m~0 |v~0|^2 - sum (r - r_c).F + sum_k Tr Xi^(k);
// anisotropic, for each edge a in the mask, the same with the a components
// alone, W the per-edge mass and 3 n V P_CV -> n V P_CV^aa (the Xi_aa rows).
// Then, if a step follows, its v_W at the first A, after O_W (PILE_L: each
// edge its own deviate) and the box after both A sub-steps.  One block;
// fixed-order sums.
__global__ void __launch_bounds__(256) k_baro_kick(BaroArgs a) {
  __shared__ double red[256];
  const int P = a.P;
  double mv2[3] = {0.0, 0.0, 0.0}, fv[3] = {0.0, 0.0, 0.0}, f2m[3] = {0.0, 0.0, 0.0};
  double rcf[3] = {0.0, 0.0, 0.0}, vir[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < a.N; i += blockDim.x) {
    const double mm = a.mass_mm[i] * a.mu0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t row = ((size_t)i * 3 + c) * P;
      double f0 = 0.0, xm = 0.0;
      for (int j = 0; j < P; ++j) {
        f0 = fma(a.Mt[j * P], a.F[row + j], f0);   // F~0 = (M F)_0
        xm += a.x[row + j];
      }
      xm /= P;
      for (int j = 0; j < P; ++j) rcf[c] = fma(a.x[row + j] - xm, a.F[row + j], rcf[c]);
      const double v0 = fma(a.t0, f0 / mm, a.v[row]);   // at t0 into the kick
      mv2[c] = fma(mm * v0, v0, mv2[c]);
      fv[c] = fma(f0, v0, fv[c]);
      f2m[c] += f0 * f0 / mm;
    }
  }
  if (a.axes) {
    for (int t = threadIdx.x; t < a.nmol * P; t += blockDim.x)
#pragma unroll
      for (int c = 0; c < 3; ++c) vir[c] += a.W3part[(size_t)t * 3 + c];
  } else {
    for (int t = threadIdx.x; t < a.nmol * P; t += blockDim.x) vir[0] += a.Wpart[t];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    mv2[c] = block_sum(mv2[c], red);
    fv[c] = block_sum(fv[c], red);
    f2m[c] = block_sum(f2m[c], red);
    rcf[c] = block_sum(rcf[c], red);
    vir[c] = block_sum(vir[c], red);
  }
  if (threadIdx.x != 0) return;
  double *b = a.baro;
  const double V = b[kBaroL] * b[kBaroL + 1] * b[kBaroL + 2];
  const double tB = a.tB;
  // O_W: v_W <- c1 v_W + sigW eta, eta from Philox atom 0xffffffff, stream 3,
  // the given mode; each edge its own deviate, the isotropic v_W the first
  auto langevin = [&](double *w, uint32_t mode, uint64_t st) {
    double e[3];
    gauss3(a.seed, 0xffffffffu, mode, 3u, st, e[0], e[1], e[2]);
    if (a.axes) {
      for (int c = 0; c < 3; ++c)
        if (a.axes >> c & 1) w[c] = a.c1W * w[c] + a.sigW * e[c];
    } else {
      w[0] = w[1] = w[2] = a.c1W * w[0] + a.sigW * e[0];
    }
  };
  const uint64_t step = (uint64_t)*a.step;
  double vW[3] = {b[kBaroV], b[kBaroV + 1], b[kBaroV + 2]};
  if (a.obabo && a.step_follows && a.thermo) langevin(vW, 0u, step);   // this step's first O(h/2)
  if (a.axes) {
    for (int c = 0; c < 3; ++c)
      vW[c] = (a.axes >> c & 1)
                  ? vW[c] + tB / a.W * (mv2[c] - rcf[c] + vir[c] - V * a.npext + a.nkT) +
                        tB * tB / a.W * fv[c] + tB * tB * tB / (3.0 * a.W) * f2m[c]
                  : 0.0;
  } else {
    const double smv2 = mv2[0] + mv2[1] + mv2[2], srcf = rcf[0] + rcf[1] + rcf[2];
    const double sfv = fv[0] + fv[1] + fv[2], sf2m = f2m[0] + f2m[1] + f2m[2];
    const double w = vW[0] + 3.0 * tB / a.W * ((smv2 - srcf + vir[0]) / 3.0 - V * a.npext + a.nkT) +
                     tB * tB / a.W * sfv + tB * tB * tB / (3.0 * a.W) * sf2m;
    vW[0] = vW[1] = vW[2] = w;
  }
  if (!a.step_follows) {
    // OBABO: the closing O(h/2) of the step just completed (the counter has
    // already been advanced past it)
    if (a.obabo && a.thermo) langevin(vW, 1u, step - 1);
    for (int c = 0; c < 3; ++c) b[kBaroV + c] = vW[c];
    return;
  }
  double vO[3] = {vW[0], vW[1], vW[2]};
  if (a.thermo && !a.obabo) langevin(vO, 0u, step);
  for (int c = 0; c < 3; ++c) {
    b[kBaroVA1 + c] = vW[c];
    b[kBaroVA2 + c] = vO[c];
    b[kBaroV + c] = vO[c];
    // BAOAB: A(h/2) at v_W, O_W, A(h/2) at v_O; OBABO: one A(h) at v_W
    const double L = a.obabo ? b[kBaroL + c] * exp(a.tA * vW[c])
                             : b[kBaroL + c] * exp(a.tA * vW[c]) * exp(a.tA * vO[c]);
    b[kBaroL + c] = L;
    b[kBaroInvL + c] = 1.0 / L;
    if (!(L > a.Lmin)) atomicOr(a.err, kErrBoxSmall);
  }
}

__global__ void k_to_f32(const double *src, float *dst, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (float)src[t];
}

__global__ void k_advance(int64_t *step, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += n;
}

// Initial velocities of mode (or bead) k ~ N(0, P kB T / (mu_k m mvv2e)),
// noise stream 2.
__global__ void k_thermal_v(double *v, const double *sigv, const double *imu, uint64_t seed, int N, int P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * P) return;
  const int i = t / P, k = t % P;
  double e0, e1, e2;
  gauss3(seed, (uint32_t)i, (uint32_t)k, kStreamInit, 0ull, e0, e1, e2);
  const double s = imu ? sigv[i] * sqrt(imu[k]) : sigv[i];
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
size_t step_smem_bytes(int A, int P) { return ((size_t)6 * A * 3 * P + 3 * A) * sizeof(double); }
size_t close_smem_bytes(int A, int P) { return (size_t)A * 3 * P * sizeof(double); }

cudaError_t launch_step(const StepArgs &a0, int threads, cudaStream_t s) {
  const int grid = (a0.N + a0.A - 1) / a0.A;
  StepArgs a = a0;
  static int nsm = 0;   // SM count of the device (one GPU per process)
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 152;
  }
  a.noise_pre = grid >= 4 * nsm ? 1 : 0;
  if (a.method == 1) {
    k_step_cart_f64<<<grid, threads, step_smem_bytes(a.A, a.P), s>>>(a);
    return cudaGetLastError();
  }
  k_step_f64<<<grid, threads, step_smem_bytes(a.A, a.P), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_close(const StepArgs &a, int threads, cudaStream_t s) {
  if (a.method == 1) {
    const size_t total = (size_t)a.N * 3 * a.P;
    k_close_cart_f64<<<(unsigned)std::min<size_t>((total + 255) / 256, 4096), 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  const int grid = (a.N + a.A - 1) / a.A;
  k_close_f64<<<grid, threads, close_smem_bytes(a.A, a.P), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_baro_kick(const BaroArgs &a, cudaStream_t s) {
  k_baro_kick<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fixcom(const FixcomArgs &a, cudaStream_t s) {
  k_fixcom_f64<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double *src, float *dst, size_t n, cudaStream_t s) {
  k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *step, int n, cudaStream_t s) {
  k_advance<<<1, 32, 0, s>>>(step, n);
  return cudaGetLastError();
}

cudaError_t launch_thermal_v(double *v, const double *sigv, const double *imu, uint64_t seed, int N, int P,
                             cudaStream_t s) {
  const int total = N * P;
  k_thermal_v<<<(total + 255) / 256, 256, 0, s>>>(v, sigv, imu, seed, N, P);
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
