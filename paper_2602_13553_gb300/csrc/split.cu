// split.cu -- the split-precision form of the PIMD step and forces.
//
// State: the ring-polymer centroid of every atom in FP64 (position xc and
// centroid-mode velocity v~_0), the beads as FP32 deviations d^j = x^j - xc
// and the internal-mode velocities v~_k (k >= 1) in FP32, forces in FP32.
// Because rows k >= 1 of the normal-mode matrix (Eq. A1) are orthogonal to
// the constant row, q~_k = (M x)_k = (M d)_k for k >= 1: the internal modes
// are transformed from the small deviations alone, so FP32 rounding acts on
// ~0.1 A quantities instead of on absolute coordinates.  FP64 is kept for
// the centroid's position/momentum accumulation (A and O of mode 0 and its
// kick) and, in the estimators, for the compensated sums.
//
// HBM per bead-atom and step: step kernel reads F, d, v~ (36 B) and writes
// d, v~ (24 B), plus 96 B per atom for xc, v~_0; force kernel reads d (12 B)
// and writes F (12 B).
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace pimd {

// FP32 deviate of the same Philox words as gauss1 (component d = 0, 1, 2):
// u = (w >> 8 + 1/2) 2^-24, Box-Muller in FP32.
__device__ __forceinline__ float gauss1f(uint64_t seed, uint32_t atom, uint32_t mode, uint32_t stream,
                                         uint64_t step, int d) {
  const uint4 w = philox4x32_10(
      make_uint4(atom, (mode & 0xffffu) | (stream << 16), (uint32_t)step, (uint32_t)(step >> 32)),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint32_t wa = d < 2 ? w.x : w.z;
  const uint32_t wb = d < 2 ? w.y : w.w;
  const float s = 5.9604644775390625e-8f;  // 2^-24
  const float r = sqrtf(-2.0f * __logf(((float)(wa >> 8) + 0.5f) * s));
  const float ang = 2.0f * (((float)(wb >> 8) + 0.5f) * s);
  float sn, cs;
  sincospif(ang, &sn, &cs);
  return r * (d == 1 ? sn : cs);
}

// The three deviates of gauss1f for d = 0, 1, 2 from one Philox draw (the
// same words and the same FP32 arithmetic, so the same values).
__device__ __forceinline__ void gauss3f(uint64_t seed, uint32_t atom, uint32_t mode, uint32_t stream,
                                        uint64_t step, float &e0, float &e1, float &e2) {
  const uint4 w = philox4x32_10(
      make_uint4(atom, (mode & 0xffffu) | (stream << 16), (uint32_t)step, (uint32_t)(step >> 32)),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float s = 5.9604644775390625e-8f;  // 2^-24
  const float r0 = sqrtf(-2.0f * __logf(((float)(w.x >> 8) + 0.5f) * s));
  const float r1 = sqrtf(-2.0f * __logf(((float)(w.z >> 8) + 0.5f) * s));
  float sn, cs, sn2, cs2;
  sincospif(2.0f * (((float)(w.y >> 8) + 0.5f) * s), &sn, &cs);
  sincospif(2.0f * (((float)(w.w >> 8) + 0.5f) * s), &sn2, &cs2);
  e0 = r0 * cs;
  e1 = r0 * sn;
  e2 = r1 * cs2;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void rotatef(float &q, float &v, float c, float s_over_w, float w_s) {
  const float qn = fmaf(c, q, s_over_w * v);
  const float vn = fmaf(-w_s, q, c * v);
  q = qn;
  v = vn;
}


__device__ __forceinline__ float wrapf(double x, double L, double invL) {
  return L > 0.0 ? (float)(x - L * floor(x * invL)) : (float)x;
}

// Tasks as in the FP64 step: t = (al * 3 + c) * P + k.  Phase 1 (every
// task, FP32): F~_k, q~_k (k >= 1) and the internal-mode update; the k = 0
// slot keeps F~_0 for phase 2.  Phase 2: centroid tasks (al, c) in FP64 --
// kick, drift, O with an FP32 deviate, drift -- packed one per lane; and
// the inverse transform of the internal modes into new deviations.
// PT > 0 fixes the bead count at compile time (the index arithmetic of every
// element -- divisions by P and by 3 -- then reduces to shifts and multiplies,
// which matter in this issue-bound kernel); PT = 0 reads it from the arguments.
template <int PT>
__global__ void __launch_bounds__(256) k_step_split(SplitStepArgs a) {
  extern __shared__ float smf[];
  const int P = PT > 0 ? PT : a.P;
  const int tileLen = a.A * 3 * P;
  float *sD = smf;
  float *sV = sD + tileLen;
  float *sF = sV + tileLen;
  float *sQ = sF + tileLen;
  float *sE = sQ + tileLen;      // PILE_L deviates of this step (stream O1), per element
  float *sE2 = sE + tileLen;     // OBABO: stream O2 of the previous step
  __shared__ float sred[2][8];
  const int tile0 = blockIdx.x * a.A;
  const int na = min(a.A, a.N - tile0);
  const int len = na * 3 * P;
  const size_t base = (size_t)tile0 * 3 * P;
  // d and F staged folded (u_j = x_j + x_{P-j}, u_{P-j} = x_j - x_{P-j}):
  // the forward transforms then sum one half of a row (rows of M are even
  // for modes k <= H = P/2, odd above), as in the FP64 step kernel
  const int H = P >> 1;
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    const int j = t % P, pj = j == 0 ? 0 : P - j;
    const size_t g = base + t, gp = g - j + pj;
    const float da = a.d[g], fa = a.F[g];
    float du = da, fu = fa;
    if (pj != j) {
      const float db = a.d[gp], fb = a.F[gp];
      du = j < pj ? da + db : db - da;
      fu = j < pj ? fa + fb : fb - fa;
    }
    sD[t] = du;
    sV[t] = a.vk[g];
    sF[t] = fu;
  }
  const uint64_t step = (uint64_t)(*a.step + a.step_off);
  // one Philox draw per (atom, mode) serves the three components
  const bool o2 = a.integrator == 1 && !a.first;
  if (a.thermo) {
    for (int t = threadIdx.x; t < na * P; t += blockDim.x) {
      const int al = t / P, k = t - al * P;
      const int e = al * 3 * P + k;
      gauss3f(a.seed, (uint32_t)(tile0 + al), (uint32_t)k, kStreamO1, step, sE[e], sE[e + P], sE[e + 2 * P]);
      if (o2)
        gauss3f(a.seed, (uint32_t)(tile0 + al), (uint32_t)k, kStreamO2, step - 1, sE2[e], sE2[e + P],
                sE2[e + 2 * P]);
    }
  }
  __syncthreads();
  const float *__restrict__ Tf = a.Tff;
  const float kick = (float)a.kick, half = (float)a.half;
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int k = task % P;
    const int r = task / P;
    const int c = r % 3;
    const int i = tile0 + r / 3;
    const bool even = k <= H;
    const int n = even ? H + 1 : P - H - 1;
    const float *fx = sF + r * P + (even ? 0 : H + 1);
    const float *xx = sD + r * P + (even ? 0 : H + 1);
    const float *tf = Tf + k;
    float fa = 0.f, fb = 0.f, qa = 0.f, qb = 0.f;
    int j = 0;
    for (; j + 1 < n; j += 2) {
      const float m0 = __ldg(tf + j * P), m1 = __ldg(tf + (j + 1) * P);
      fa = fmaf(m0, fx[j], fa);
      fb = fmaf(m1, fx[j + 1], fb);
      qa = fmaf(m0, xx[j], qa);
      qb = fmaf(m1, xx[j + 1], qb);
    }
    if (j < n) {
      const float m0 = __ldg(tf + j * P);
      fa = fmaf(m0, fx[j], fa);
      qa = fmaf(m0, xx[j], qa);
    }
    const float f = fa + fb;
    if (k == 0) {
      sQ[task] = f;      // F~_0, consumed by the centroid task below
      continue;
    }
    float q = qa + qb;
    float v = sV[task];
    const float im = (float)__ldg(a.inv_mm + i);
    const float cA = __ldg(a.cAf + k), sA = __ldg(a.sAf + k), wsA = __ldg(a.wsAf + k);
    const float c1 = __ldg(a.c1f + k), c2s = __ldg(a.c2f + k) * (float)__ldg(a.sigv + i);
    if (a.integrator == 0) {
      v = fmaf(kick * im, f, v);
      rotatef(q, v, cA, sA, wsA);
      if (a.thermo) v = fmaf(c1, v, c2s * sE[task]);
      rotatef(q, v, cA, sA, wsA);
    } else {
      const float kb = half * im;
      if (!a.first) {
        v = fmaf(kb, f, v);
        if (a.thermo) v = fmaf(c1, v, c2s * sE2[task]);
      }
      if (a.thermo) v = fmaf(c1, v, c2s * sE[task]);
      v = fmaf(kb, f, v);
      rotatef(q, v, cA, sA, wsA);
    }
    sQ[task] = q;
    a.vk[base + task] = v;
  }
  __syncthreads();
  // centroid tasks, FP64: q~_0 = sqrt(P) xc, so drift is xc += tA v~_0 / sqrt(P)
  const double rsp = rsqrt((double)P);
  for (int t = threadIdx.x; t < na * 3; t += blockDim.x) {
    const int al = t / 3, c = t % 3;
    const int i = tile0 + al;
    const size_t ic = (size_t)i * 3 + c;
    const double f0 = (double)sQ[t * P];
    double x = a.xc[ic], v = a.v0[ic];
    const double im = __ldg(a.inv_mm + i);
    const double dr = a.tA * rsp;
    if (a.integrator == 0) {
      v = fma(a.kick * im, f0, v);
      x = fma(dr, v, x);
      if (a.thermo) v = fma(a.c1_0, v, a.c2_0 * __ldg(a.sigv + i) * (double)sE[t * P]);
      x = fma(dr, v, x);
    } else {
      const double kb = a.half * im;
      if (!a.first) {
        v = fma(kb, f0, v);
        if (a.thermo) v = fma(a.c1_0, v, a.c2_0 * __ldg(a.sigv + i) * (double)sE2[t * P]);
      }
      if (a.thermo) v = fma(a.c1_0, v, a.c2_0 * __ldg(a.sigv + i) * (double)sE[t * P]);
      v = fma(kb, f0, v);
      x = fma(dr, v, x);
    }
    a.xc[ic] = x;
    a.v0[ic] = v;
    if (a.xcw) a.xcw[ic] = wrapf(x, a.box[c], a.invbox[c]);
    sQ[t * P] = 0.f;   // the deviations carry no centroid mode
  }
  __syncthreads();
  // inverse, first half: C_j (bead j <= H, even modes) or S_{P-j} (bead
  // j > H, odd modes) into sF, free since the forward pass
  const float *__restrict__ Ti = a.Tif;
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int j = task % P;
    const bool even = j <= H;
    const int n = even ? H + 1 : P - H - 1;
    const float *qq = sQ + (task - j) + (even ? 0 : H + 1);
    const float *ti = Ti + j;
    float xa = 0.f, xb = 0.f;
    int k = 0;
    for (; k + 1 < n; k += 2) {
      xa = fmaf(__ldg(ti + k * P), qq[k], xa);
      xb = fmaf(__ldg(ti + (k + 1) * P), qq[k + 1], xb);
    }
    if (k < n) xa = fmaf(__ldg(ti + k * P), qq[k], xa);
    sF[task] = xa + xb;
  }
  __syncthreads();
  // second half: d'_j = C_j + S_j (j <= H), d'_{P-j} = C_j - S_j
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int j = task % P, pj = j == 0 ? 0 : P - j;
    const int row0 = task - j;
    const float dn = j <= H ? sF[task] + (pj > H ? sF[row0 + pj] : 0.f) : sF[row0 + pj] - sF[task];
    a.d[base + task] = dn;
    sD[task] = dn;
  }
  if (!a.blkmax) return;
  __syncthreads();
  // neighbour-list skin check of the oxygens: bead spread |d^k| and centroid
  // drift, squared and reduced in FP32 (the FP64 pipe is the scarce one; a
  // relative margin below keeps the bound conservative)
  float vdisp = 0.f, vdev = 0.f;
  for (int t = threadIdx.x; t < na * P; t += blockDim.x) {
    const int al = t / P, k = t % P;
    const int i = tile0 + al;
    if (i % 3) continue;
    const float *ds = sD + al * 3 * P;
    const float e0 = ds[k], e1 = ds[P + k], e2 = ds[2 * P + k];
    vdev = fmaxf(vdev, e0 * e0 + e1 * e1 + e2 * e2);
    if (k == 0) {
      const int m = i / 3;
      const double c0 = a.xc[3 * (size_t)i], c1 = a.xc[3 * (size_t)i + 1], c2 = a.xc[3 * (size_t)i + 2];
      const float g0 = (float)(c0 - a.cref[3 * m]), g1 = (float)(c1 - a.cref[3 * m + 1]);
      const float g2 = (float)(c2 - a.cref[3 * m + 2]);
      vdisp = fmaxf(vdisp, g0 * g0 + g1 * g1 + g2 * g2);
      a.ccur[3 * m] = c0;
      a.ccur[3 * m + 1] = c1;
      a.ccur[3 * m + 2] = c2;
    }
  }
  // NaN positions force a rebuild
  if (vdisp != vdisp) vdisp = __int_as_float(0x7f800000);
  if (vdev != vdev) vdev = __int_as_float(0x7f800000);
  vdisp = warp_maxf(vdisp);
  vdev = warp_maxf(vdev);
  if ((threadIdx.x & 31) == 0) {
    sred[0][threadIdx.x >> 5] = vdisp;
    sred[1][threadIdx.x >> 5] = vdev;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float mx = 0.f;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) mx = fmaxf(mx, sred[threadIdx.x][w]);
    // margins for FP32 rounding of the deviations and of the squares
    a.blkmax[2 * blockIdx.x + threadIdx.x] = mx <= 3.0e38f ? sqrt((double)mx) * (1.0 + 1e-6) + 1e-4 : 1e300;
  }
}

// Closing B(h/2) (and O(h/2) for OBABO) of a call's last step.
__global__ void __launch_bounds__(256) k_close_split(SplitStepArgs a) {
  extern __shared__ float smf[];
  const int P = a.P;
  float *sF = smf;
  const int tile0 = blockIdx.x * a.A;
  const int na = min(a.A, a.N - tile0);
  const int len = na * 3 * P;
  const size_t base = (size_t)tile0 * 3 * P;
  for (int t = threadIdx.x; t < len; t += blockDim.x) sF[t] = a.F[base + t];
  __syncthreads();
  const uint64_t step = (uint64_t)(*a.step + a.step_off);
  const float *__restrict__ Mt = a.Mtf;
  for (int task = threadIdx.x; task < len; task += blockDim.x) {
    const int k = task % P;
    const int r = task / P;
    const int c = r % 3;
    const int i = tile0 + r / 3;
    const float *fx = sF + r * P;
    float fa = 0.f, fb = 0.f;
    int j = 0;
    for (; j + 1 < P; j += 2) {
      fa = fmaf(__ldg(Mt + j * P + k), fx[j], fa);
      fb = fmaf(__ldg(Mt + (j + 1) * P + k), fx[j + 1], fb);
    }
    if (j < P) fa = fmaf(__ldg(Mt + j * P + k), fx[j], fa);
    const float f = fa + fb;
    if (k == 0) {
      const size_t ic = (size_t)i * 3 + c;
      double v = fma(a.half * __ldg(a.inv_mm + i), (double)f, a.v0[ic]);
      if (a.integrator == 1 && a.thermo)
        v = fma(a.c1_0, v, a.c2_0 * __ldg(a.sigv + i) *
                               (double)gauss1f(a.seed, (uint32_t)i, 0u, kStreamO2, step, c));
      a.v0[ic] = v;
      continue;
    }
    float v = fmaf((float)a.half * (float)__ldg(a.inv_mm + i), f, a.vk[base + task]);
    if (a.integrator == 1 && a.thermo) {
      const float c1 = __ldg(a.c1f + k), c2s = __ldg(a.c2f + k) * (float)__ldg(a.sigv + i);
      v = fmaf(c1, v, c2s * gauss1f(a.seed, (uint32_t)i, (uint32_t)k, kStreamO2, step, c));
    }
    a.vk[base + task] = v;
  }
}

// --- forces -----------------------------------------------------------------

__global__ void __launch_bounds__(256) k_force_harmonic_split(SplitForceArgs a) {
  __shared__ double sU[256], sW[256];
  const int P = a.P;
  const int per = blockDim.x / P;
  const int i = blockIdx.x * per + threadIdx.x / P;
  const int k = threadIdx.x % P;
  float u = 0.f, w = 0.f;
  if (threadIdx.x < per * P && i < a.N) {
    const float ks = (float)__ldg(a.kspring + i);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t id = ((size_t)i * 3 + c) * P + k;
      const float x = (float)a.xc[(size_t)i * 3 + c] + a.d[id];
      const float f = -ks * x;
      a.F[id] = f;
      u = fmaf(0.5f * ks * x, x, u);
      w = fmaf(x, f, w);
    }
  }
  sU[threadIdx.x] = u;
  sW[threadIdx.x] = w;
  __syncthreads();
  const int groups = min(per, a.N - blockIdx.x * per);
  for (int kk = threadIdx.x; kk < P; kk += blockDim.x) {
    double su = 0.0, sw = 0.0;
    for (int g = 0; g < groups; ++g) {
      su += sU[g * P + kk];
      sw += sW[g * P + kk];
    }
    a.Upart[(size_t)blockIdx.x * P + kk] = su;
    a.Wpart[(size_t)blockIdx.x * P + kk] = sw;
  }
  if (a.step_inc && blockIdx.x == 0 && threadIdx.x == 0) *a.step_inc += 1;
}

__device__ __forceinline__ float micf(float d, float L, float invL) { return fmaf(-rintf(d * invL), L, d); }

// Water-like model in FP32, same decomposition as the FP64 kernel: a
// kForceBlocks-block cluster per (molecule, bead chunk), warps 0 ..
// kLJWarps - 1 own buckets of the O-O neighbour list, warp kLJWarps the
// bonds, warp kLJWarps + 1 the angle; partials are
// reduced through distributed shared memory in rank order.  A pair vector is
// the minimum-image difference of the wrapped FP32 centroids plus the
// difference of the FP32 deviations.
__global__ void __cluster_dims__(kForceBlocks, 1, 1) __launch_bounds__(128) k_force_water_split(SplitForceArgs a) {
  __shared__ float sacc[9][128];
  __shared__ double saccd[2][128];
  __shared__ float red[9][32];
  __shared__ double redd[2][32];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int P = a.P;
  const int Bk = P < 32 ? P : 32;
  const int G = a.nbr_groups;
  const int NS = kLJWarps * G;
  const int nchunk = (P + Bk - 1) / Bk;
  const int cid = blockIdx.x / kForceBlocks;
  const int m = cid / nchunk, chunk = cid % nchunk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = rank * 4 + warp;
  const int u = lane / Bk, kl = lane % Bk;
  const int k = chunk * Bk + kl;
  float acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.f;
  double ue = 0.0, we = 0.0;
  if (u < G && k < P && m < a.nmol) {
    const int o = 3 * m;
    const float L0 = (float)a.box[0], L1 = (float)a.box[1], L2 = (float)a.box[2];
    const float i0 = (float)a.invbox[0], i1 = (float)a.invbox[1], i2 = (float)a.invbox[2];
    const size_t so = (size_t)o * 3 * P + k;
    const float co0 = a.xcw[3 * o], co1 = a.xcw[3 * o + 1], co2 = a.xcw[3 * o + 2];
    const float do0 = a.d[so], do1 = a.d[so + P], do2 = a.d[so + 2 * P];
    if (s >= kLJWarps) {
      if (u == 0) {
        float dv[2][3], r[2], ir[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int hh = o + 1 + h;
          const size_t sh = (size_t)hh * 3 * P + k;
          dv[h][0] = micf(a.xcw[3 * hh] - co0, L0, i0) + (a.d[sh] - do0);
          dv[h][1] = micf(a.xcw[3 * hh + 1] - co1, L1, i1) + (a.d[sh + P] - do1);
          dv[h][2] = micf(a.xcw[3 * hh + 2] - co2, L2, i2) + (a.d[sh + 2 * P] - do2);
          r[h] = sqrtf(dv[h][0] * dv[h][0] + dv[h][1] * dv[h][1] + dv[h][2] * dv[h][2]);
          ir[h] = 1.f / r[h];
        }
        float uu = 0.f, w = 0.f;
        if (s == kLJWarps) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float dr = r[h] - (float)a.r0;
            uu = fmaf(0.5f * (float)a.kb * dr, dr, uu);
            const float g = -(float)a.kb * dr * ir[h];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float fc = g * dv[h][c];
              acc[3 + 3 * h + c] = fc;
              acc[c] -= fc;
              w = fmaf(dv[h][c], fc, w);
            }
          }
        } else {
          const float ir01 = ir[0] * ir[1];
          const float dot = dv[0][0] * dv[1][0] + dv[0][1] * dv[1][1] + dv[0][2] * dv[1][2];
          const float cth = fminf(1.f, fmaxf(-1.f, dot * ir01));
          const float th = acosf(cth);
          const float dth = th - (float)a.th0;
          const float pref = (float)a.kth * dth / sinf(th);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int g = 1 - h;
            const float ch = cth * ir[h] * ir[h];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float fa = pref * fmaf(dv[g][c], ir01, -ch * dv[h][c]);
              acc[3 + 3 * h + c] = fa;
              acc[c] -= fa;
              w = fmaf(dv[h][c], fa, w);
            }
          }
          uu = 0.5f * (float)a.kth * dth * dth;
        }
        ue = uu;
        we = w;
      }
    } else {
      const int b = s * G + u;
      const int *off = a.nbr_off + (size_t)m * (NS + 1);
      const int q0 = __ldg(off + b), q1 = __ldg(off + b + 1);
      const int *nl = a.nbr + (size_t)m * kMaxNeighbours;
      const float rc2 = (float)(a.rc * a.rc);
      const float sig2 = (float)(a.sig * a.sig);
      const float e4 = (float)(4.0 * a.eps), e24 = (float)(24.0 * a.eps);
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, ulj = 0.f, wlj = 0.f;
      for (int q = q0; q < q1; ++q) {
        const int j = __ldg(nl + q);
        const size_t sj = (size_t)(3 * j) * 3 * P + k;
        const float d0 = micf(__ldg(a.xcw + 9 * j) - co0, L0, i0) + (__ldg(a.d + sj) - do0);
        const float d1 = micf(__ldg(a.xcw + 9 * j + 1) - co1, L1, i1) + (__ldg(a.d + sj + P) - do1);
        const float d2 = micf(__ldg(a.xcw + 9 * j + 2) - co2, L2, i2) + (__ldg(a.d + sj + 2 * P) - do2);
        const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 < rc2) {
          const float inv = 1.f / r2;
          const float s2 = sig2 * inv;
          const float s6 = s2 * s2 * s2;
          ulj = fmaf(e4, fmaf(s6, s6, -s6), ulj);
          const float fr = e24 * fmaf(2.f * s6, s6, -s6) * inv;
          f0 = fmaf(-fr, d0, f0);
          f1 = fmaf(-fr, d1, f1);
          f2 = fmaf(-fr, d2, f2);
          wlj = fmaf(fr, r2, wlj);
        }
      }
      acc[0] = f0;
      acc[1] = f1;
      acc[2] = f2;
      ue = 0.5 * (double)ulj;
      we = 0.5 * (double)wlj;
    }
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) sacc[c][threadIdx.x] = acc[c];
  saccd[0][threadIdx.x] = ue;
  saccd[1][threadIdx.x] = we;
  __syncthreads();
  for (int t = threadIdx.x; t < 11 * Bk; t += blockDim.x) {
    const int comp = t / Bk, kk = t % Bk;
    if (comp < 9) {
      float sum = 0.f;
      for (int w = 0; w < 4; ++w)
        for (int g = 0; g < G; ++g) sum += sacc[comp][w * 32 + g * Bk + kk];
      red[comp][kk] = sum;
    } else {
      double sum = 0.0;
      for (int w = 0; w < 4; ++w)
        for (int g = 0; g < G; ++g) sum += saccd[comp - 9][w * 32 + g * Bk + kk];
      redd[comp - 9][kk] = sum;
    }
  }
  cluster.sync();
  if (rank == 0 && m < a.nmol) {
    for (int t = threadIdx.x; t < 11 * Bk; t += blockDim.x) {
      const int comp = t / Bk, kk = t % Bk;
      const int k2 = chunk * Bk + kk;
      if (k2 >= P) continue;
      if (comp < 9) {
        float sum = 0.f;
        for (int r = 0; r < kForceBlocks; ++r) sum += cluster.map_shared_rank(&red[0][0], r)[comp * 32 + kk];
        a.F[(size_t)(3 * m + comp / 3) * 3 * P + (comp % 3) * P + k2] = sum;
      } else {
        double sum = 0.0;
        for (int r = 0; r < kForceBlocks; ++r) sum += cluster.map_shared_rank(&redd[0][0], r)[(comp - 9) * 32 + kk];
        if (comp == 9)
          a.Upart[(size_t)m * P + k2] = sum;
        else
          a.Wpart[(size_t)m * P + k2] = sum;
      }
    }
    if (a.step_inc && blockIdx.x == 0 && threadIdx.x == 0) *a.step_inc += 1;
  }
  cluster.sync();
}

// --- conversions between the split state and FP64 [N][3][P] arrays ----------

// x = xc + d, v~ (mode 0 from v~_0), F -> FP64
__global__ void k_expand_split(SplitStepArgs a, const float *F, double *x, double *v, double *Fd) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)a.N * 3 * a.P;
  if (t >= total) return;
  const int k = (int)(t % a.P);
  const size_t ic = t / a.P;
  x[t] = a.xc[ic] + (double)a.d[t];
  v[t] = k == 0 ? a.v0[ic] : (double)a.vk[t];
  if (Fd) Fd[t] = (double)F[t];
}

// xc = bead average, d = x - xc, v~_0 and v~_k from FP64 [N][3][P] arrays
__global__ void k_compress_split(SplitStepArgs a, const double *x, const double *v) {
  const size_t ic = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ic >= (size_t)a.N * 3) return;
  const int P = a.P;
  const int c = (int)(ic % 3);
  double s = 0.0;
  for (int k = 0; k < P; ++k) s += x[ic * P + k];
  const double xc = s / P;
  a.xc[ic] = xc;
  a.v0[ic] = v[ic * P];
  if (a.xcw) a.xcw[ic] = wrapf(xc, a.box[c], a.invbox[c]);
  for (int k = 0; k < P; ++k) {
    a.d[ic * P + k] = (float)(x[ic * P + k] - xc);
    a.vk[ic * P + k] = k == 0 ? 0.f : (float)v[ic * P + k];
  }
}

// --- host launchers ----------------------------------------------------------
size_t split_step_smem_bytes(int A, int P) { return (size_t)6 * A * 3 * P * sizeof(float); }

cudaError_t launch_step_split(const SplitStepArgs &a, int threads, cudaStream_t s) {
  const int grid = (a.N + a.A - 1) / a.A;
  const size_t smem = split_step_smem_bytes(a.A, a.P);
  switch (a.P) {
    case 8: k_step_split<8><<<grid, threads, smem, s>>>(a); break;
    case 16: k_step_split<16><<<grid, threads, smem, s>>>(a); break;
    case 32: k_step_split<32><<<grid, threads, smem, s>>>(a); break;
    case 64: k_step_split<64><<<grid, threads, smem, s>>>(a); break;
    case 128: k_step_split<128><<<grid, threads, smem, s>>>(a); break;
    default: k_step_split<0><<<grid, threads, smem, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_close_split(const SplitStepArgs &a, int threads, cudaStream_t s) {
  const int grid = (a.N + a.A - 1) / a.A;
  k_close_split<<<grid, threads, (size_t)a.A * 3 * a.P * sizeof(float), s>>>(a);
  return cudaGetLastError();
}

int force_blocks(int n_groups, int P);
int force_block_threads(int P);
int water_force_blocks(int nmol, int P);

cudaError_t launch_force_split(const SplitForceArgs &a, bool water, cudaStream_t s) {
  if (water)
    k_force_water_split<<<water_force_blocks(a.nmol, a.P), 128, 0, s>>>(a);
  else
    k_force_harmonic_split<<<force_blocks(a.N, a.P), force_block_threads(a.P), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_expand_split(const SplitStepArgs &a, const float *F, double *x, double *v, double *Fd,
                                cudaStream_t s) {
  const size_t total = (size_t)a.N * 3 * a.P;
  k_expand_split<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a, F, x, v, Fd);
  return cudaGetLastError();
}

cudaError_t launch_compress_split(const SplitStepArgs &a, const double *x, const double *v,
                                  cudaStream_t s) {
  const size_t n = (size_t)a.N * 3;
  k_compress_split<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a, x, v);
  return cudaGetLastError();
}

}  // namespace pimd
