// noalloc.cu -- pimd_estimators_noalloc: the App. A estimator reduction for
// state held in the caller's own device buffers, with every intermediate in
// one file-scope device array, so the call allocates no memory at all.
//
// This serves callers that cannot let a library allocate device memory: a
// host application that owns a fixed device pool reserved at start-up, or a
// time-stepping loop in which a cudaMalloc / cudaFree would synchronise the
// device and stall its other streams.  They pass their inputs and the output
// struct; the reduction runs entirely in this file's static scratch.
//
// The scratch (kStaticScratchDoubles doubles, 1 MiB) exists once per GPU
// that loads the library and stays resident until the process exits.  Every
// call on a device reuses it, so two calls whose kernels overlap on that GPU
// race; serialise them (one stream, or events).  Nothing in it needs to
// start at zero: each call rewrites every entry it reads.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "pimd.h"

namespace pimd {

constexpr int kStaticScratchDoubles = 1 << 17;   // 1 MiB
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) double g_est_scratch[kStaticScratchDoubles];

namespace {

// Per device: the device address of g_est_scratch (host code may not use the
// symbol itself; it names a host-side stand-in).
std::mutex g_mu;
double *g_scratch_ptr[kStaticMaxDevices] = {nullptr};

// Eq. (A1), Eq. (A2) and the fictitious-mass factors mu_k (m^(k) = mu_k m,
// Sec. III.C keywords fmmode and fmass; lambda_0 = 0 keeps the centroid at
// fmass m) evaluated on the device into the scratch.
__global__ void k_nm_tables_static(int P, int normal_masses, double fmass, double *M, double *lam, double *mu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < P * P) {
    const int i = t / P, j = t % P;
    const double rp = 1.0 / sqrt((double)P);
    double val;
    if (i == 0)
      val = rp;
    else if (P % 2 == 0 && 2 * i == P)
      val = (j & 1) ? -rp : rp;
    else if (2 * i < P)
      val = sqrt(2.0 / P) * cospi(2.0 * (double)((long long)i * j % P) / P);
    else
      val = sqrt(2.0 / P) * sinpi(2.0 * (double)((long long)i * j % P) / P);
    M[t] = val;
  }
  if (t < P) {
    const double s = sinpi((double)t / P);
    lam[t] = 4.0 * s * s;
    mu[t] = (normal_masses && t > 0) ? fmass * lam[t] : fmass;
  }
}

// Pass 1: persistent blocks walk atom tiles (stride gridDim.x); thread task
// (atom al, mode k) adds 1/2 m^(k) |v~_k|^2 to K^(k) and the ring's spring
// energy of mode k (normal modes: 1/2 m w_n^2 lambda_k |q~_k|^2 with q~ = M x;
// Cartesian beads: 1/4 m w_n^2 (|r^k - r^(k-1)|^2 + |r^k - r^(k+1)|^2)) to
// S^(k), and, as bead j = k, r^j.F^j and (r^j - r_c).F^j; the centroid-mode
// term m^(0) |v~_0|^2 of P_CV (Cartesian: v~_0 = sum_k v^(k) / sqrt(P)).
// Every sum is compensated; the block writes one row of partials.  Inputs use
// the public [P][N][3] layout.
__global__ void __launch_bounds__(256) k_est_static(int N, int P, int A, int cart, const double *__restrict__ x,
                                                   const double *__restrict__ v,
                                                   const double *__restrict__ F,
                                                   const double *__restrict__ mass, double wn2,
                                                   const double *__restrict__ M,
                                                   const double *__restrict__ lam,
                                                   const double *__restrict__ mu, double *part) {
  extern __shared__ double sm[];
  const int tileLen = A * 3 * P;
  double *sX = sm, *sV = sX + tileLen, *sF = sV + tileLen, *sC = sF + tileLen;
  CSum *sK = reinterpret_cast<CSum *>(sC + 3 * A), *sS = sK + A * P;
  __shared__ CSum sred[3][8];
  for (int t = threadIdx.x; t < A * P; t += blockDim.x) {
    sK[t] = CSum{0.0, 0.0};
    sS[t] = CSum{0.0, 0.0};
  }
  CSum rF{0.0, 0.0}, rcF{0.0, 0.0}, mv0{0.0, 0.0};
  const int ntiles = (N + A - 1) / A;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = tile * A;
    const int na = min(A, N - i0);
    __syncthreads();
    for (int t = threadIdx.x; t < P * na * 3; t += blockDim.x) {
      const int k = t / (na * 3), r = t % (na * 3);
      const int a = r / 3, d = r % 3;
      const size_t g = ((size_t)k * N + i0) * 3 + r;
      const int s = (a * 3 + d) * P + k;
      sX[s] = x[g];
      sV[s] = v[g];
      sF[s] = F[g];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < na * 3; t += blockDim.x) {
      CSum s{0.0, 0.0};
      for (int j = 0; j < P; ++j) s.add(sX[t * P + j]);
      sC[t] = s.value() / P;
    }
    __syncthreads();
    for (int task = threadIdx.x; task < na * P; task += blockDim.x) {
      const int k = task % P, al = task / P, i = i0 + al;
      const double *xx = sX + al * 3 * P, *vv = sV + al * 3 * P, *ff = sF + al * 3 * P;
      const double mm = mass[i] * kMvv2e;
      const double v2s = vv[k] * vv[k] + vv[P + k] * vv[P + k] + vv[2 * P + k] * vv[2 * P + k];
      sK[task].add(0.5 * mm * mu[k] * v2s);
      if (!cart) {
        double q0 = 0.0, q1 = 0.0, q2 = 0.0;
        for (int j = 0; j < P; ++j) {
          const double m = M[k * P + j];
          q0 = fma(m, xx[j], q0);
          q1 = fma(m, xx[P + j], q1);
          q2 = fma(m, xx[2 * P + j], q2);
        }
        sS[task].add(0.5 * mm * wn2 * lam[k] * (q0 * q0 + q1 * q1 + q2 * q2));
        if (k == 0) mv0.add(mm * mu[0] * v2s);
      } else {
        const int km = k == 0 ? P - 1 : k - 1, kp = k == P - 1 ? 0 : k + 1;
        double s2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double *xr = xx + d * P;
          const double dm = xr[k] - xr[km], dp = xr[k] - xr[kp];
          s2 += dm * dm + dp * dp;
        }
        sS[task].add(0.25 * mm * wn2 * s2);
        if (k == 0) {
          double w2 = 0.0;
          for (int d = 0; d < 3; ++d) {
            CSum sv{0.0, 0.0};
            for (int j = 0; j < P; ++j) sv.add(vv[d * P + j]);
            w2 += sv.value() * sv.value();
          }
          mv0.add(mm * mu[0] * w2 / P);
        }
      }
      const double x0 = xx[k], x1 = xx[P + k], x2 = xx[2 * P + k];
      const double f0 = ff[k], f1 = ff[P + k], f2 = ff[2 * P + k];
      rF.add(x0 * f0);
      rF.add(x1 * f1);
      rF.add(x2 * f2);
      rcF.add((x0 - sC[al * 3]) * f0);
      rcF.add((x1 - sC[al * 3 + 1]) * f1);
      rcF.add((x2 - sC[al * 3 + 2]) * f2);
    }
  }
  rF = warp_csum(rF);
  rcF = warp_csum(rcF);
  mv0 = warp_csum(mv0);
  if ((threadIdx.x & 31) == 0) {
    sred[0][threadIdx.x >> 5] = rF;
    sred[1][threadIdx.x >> 5] = rcF;
    sred[2][threadIdx.x >> 5] = mv0;
  }
  __syncthreads();
  const int W = 2 * P + 4;
  double *out = part + (size_t)blockIdx.x * W;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    CSum a{0.0, 0.0}, b{0.0, 0.0};
    for (int al = 0; al < A; ++al) {
      a.add(sK[al * P + k]);
      b.add(sS[al * P + k]);
    }
    out[k] = a.value();
    out[P + k] = b.value();
  }
  if (threadIdx.x < 3) {
    CSum s{0.0, 0.0};
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) s.add(sred[threadIdx.x][w]);
    out[2 * P + threadIdx.x] = s.value();
  }
  if (threadIdx.x == 3) out[2 * P + 3] = 0.0;
}

__device__ double neumaier(const double *p, int n, int stride) {
  CSum s{0.0, 0.0};
  for (int b = 0; b < n; ++b) s.add(p[(size_t)b * stride]);
  return s.value();
}

// Pass 2: one block; output laid out exactly like pimd_estimates from K_mode
// on (K_mode[128], S_mode[128], U_bead[128], H, K_PR, K_VR, K_CV, P_PR, P_MD,
// P_CV, T_ring, volume, vir_sum).
__global__ void k_est_static_final(int N, int P, int G, const double *part, const double *U_bead,
                                   double vir, double kT, double V, double *out) {
  __shared__ double tot[2 * kMaxBeads + 4];
  const int W = 2 * P + 4;
  for (int s = threadIdx.x; s < W; s += blockDim.x) tot[s] = neumaier(part + s, G, W);
  for (int k = threadIdx.x; k < 3 * kMaxBeads; k += blockDim.x) out[k] = 0.0;
  __syncthreads();
  if (threadIdx.x != 0) return;
  CSum Kt{0.0, 0.0}, St{0.0, 0.0}, Ut{0.0, 0.0};
  for (int k = 0; k < P; ++k) {
    out[k] = tot[k];
    out[kMaxBeads + k] = tot[P + k];
    out[2 * kMaxBeads + k] = U_bead[k];
    Kt.add(tot[k]);
    St.add(tot[P + k]);
    Ut.add(U_bead[k]);
  }
  const double rF = tot[2 * P], rcF = tot[2 * P + 1], mv0 = tot[2 * P + 2];
  const double Nd = N, Pd = P, spring = 2.0 * St.value(), K = Kt.value();
  double *g = out + 3 * kMaxBeads;
  g[0] = K + St.value() + Ut.value();
  g[1] = 1.5 * Pd * Nd * kT - 0.5 * spring / Pd;
  g[2] = -rF / (2.0 * Pd);
  g[3] = 1.5 * Nd * kT - rcF / (2.0 * Pd);
  if (V > 0.0) {
    g[4] = (3.0 * Pd * Nd * kT - spring / Pd + vir / Pd) / (3.0 * V);
    g[5] = (2.0 * K + vir) / (3.0 * V);
    g[6] = (mv0 - rcF + vir) / (3.0 * Pd * V);
  } else {
    g[4] = g[5] = g[6] = __longlong_as_double(0x7ff8000000000000ll);
  }
  g[7] = 2.0 * K / (3.0 * Nd * Pd * kBoltzmann);
  g[8] = V;
  g[9] = vir;
}

}  // namespace

// message for pimd_last_error() (defined with the rest of the C ABI)
void set_last_error(const char *msg);

}  // namespace pimd

static pimd_status noalloc_fail(pimd_status s, const char *fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  pimd::set_last_error(buf);
  return s;
}

extern "C" pimd_status pimd_estimators_noalloc(int32_t N, int32_t P, double T, double volume,
                                               const double *x, const double *v_nm, const double *F,
                                               const double *mass, const double *U_bead, double vir_sum,
                                               const pimd_params *params, void *stream, pimd_estimates *out) {
  using namespace pimd;
  if (!x || !v_nm || !F || !mass || !U_bead || !out)
    return noalloc_fail(PIMD_EINVAL, "NULL argument");
  if (P < 1 || P > PIMD_MAX_BEADS) return noalloc_fail(PIMD_EINVAL, "P = %d outside 1..128", P);
  if (N < 1 || (long long)N * 3 * P > 0x7fffffffll)
    return noalloc_fail(PIMD_EINVAL, "N = %d outside 1..2^31/(3P)", N);
  if (!(T > 0.0) || !(volume >= 0.0)) return noalloc_fail(PIMD_EINVAL, "T > 0 and volume >= 0 required");
  // the keywords the estimators depend on (defaults without params)
  double sp = 1.0, fmass = 1.0;
  int method = PIMD_METHOD_NMPIMD, fmmode = PIMD_FMMODE_PHYSICAL;
  if (params) {
    sp = params->sp;
    fmass = params->fmass;
    method = params->method;
    fmmode = params->fmmode;
  }
  if (!(sp > 0.0) || !(fmass > 0.0)) return noalloc_fail(PIMD_EINVAL, "sp > 0 and fmass > 0 required");
  if (method != PIMD_METHOD_NMPIMD && method != PIMD_METHOD_PIMD)
    return noalloc_fail(PIMD_EINVAL, "unknown method %d", method);
  if (fmmode != PIMD_FMMODE_PHYSICAL && fmmode != PIMD_FMMODE_NORMAL)
    return noalloc_fail(PIMD_EINVAL, "unknown fmmode %d", fmmode);
  if (method == PIMD_METHOD_PIMD && fmmode == PIMD_FMMODE_NORMAL)
    return noalloc_fail(PIMD_EINVAL, "fmmode normal needs method nmpimd");
  const int A = 256 / P > 0 ? 256 / P : 1;
  const int W = 2 * P + 4;
  const int fixed = P * P + 2 * P + 3 * kMaxBeads + 10;
  const int Gmax = (kStaticScratchDoubles - fixed) / W;
  const int ntiles = (N + A - 1) / A;
  const int G = ntiles < Gmax ? ntiles : Gmax;
  if (G < 1) return noalloc_fail(PIMD_EINVAL, "static scratch too small for P = %d", P);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(PIMD_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kStaticMaxDevices) return noalloc_fail(PIMD_EINVAL, "device %d out of range", dev);
  double *base = nullptr;
  {
    // one-time set-up per device, with that device current: the device
    // address of the scratch array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_est_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(PIMD_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_scratch_ptr[dev] = (double *)p;
    }
    base = g_scratch_ptr[dev];
  }
  double *M = base;
  double *lam = M + P * P;
  double *mu = lam + P;
  double *res = mu + P;                     // 3*128 + 10 doubles, pimd_estimates layout
  double *part = res + 3 * kMaxBeads + 10;  // G rows of W
  cudaStream_t s = (cudaStream_t)stream;
  const double hbar = sp * kPlanck / (2.0 * kPi);
  const double wn = P * kBoltzmann * T / hbar;
  const int cart = method == PIMD_METHOD_PIMD;
  k_nm_tables_static<<<(P * P + 127) / 128, 128, 0, s>>>(P, fmmode == PIMD_FMMODE_NORMAL && !cart, fmass, M, lam,
                                                         mu);
  const int threads = ((A * P + 31) / 32) * 32 < 256 ? ((A * P + 31) / 32) * 32 : 256;
  const size_t smem = (size_t)(3 * A * 3 * P + 3 * A + 4 * A * P) * sizeof(double);
  k_est_static<<<G, threads, smem, s>>>(N, P, A, cart, x, v_nm, F, mass, wn * wn, M, lam, mu, part);
  k_est_static_final<<<1, 128, 0, s>>>(N, P, G, part, U_bead, vir_sum, kBoltzmann * T, volume, res);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(PIMD_ECUDA, "launch: %s", cudaGetErrorString(e));
  e = cudaMemcpyAsync(out->K_mode, res, sizeof(double) * (3 * kMaxBeads + 10), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(PIMD_ECUDA, "copy back: %s", cudaGetErrorString(e));
  out->step = 0;
  out->P = P;
  out->N = N;
  // no barostat state and no box edges reach this call: outputs 11-15, the
  // box and v_Wa are zero, as pimd_estimators reports them without a barostat
  out->vW = out->K_W = out->U_W = out->J_W = out->enthalpy = 0.0;
  for (int d = 0; d < 3; ++d) out->box[d] = out->vWa[d] = 0.0;
  if (!std::isfinite(out->H)) return noalloc_fail(PIMD_ENONFINITE, "non-finite estimator sum");
  return PIMD_OK;
}
