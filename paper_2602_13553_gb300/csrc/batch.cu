// batch.cu -- many independent ring-polymer systems ("replicas") of uneven
// size advanced together in split precision, and the serving layer on top.
//
// Every replica's state lives in its own device arena and is described by a
// RepDesc in a device table.  Each MD step is a sequence of launches over all
// replicas -- control; the step, one kernel per class of bead count present
// (warp items of 64 beads; of 8, 16 or 32; of 128; block items of any other
// count), the classes side by side on two streams; rebuild decision;
// rebuilds; forces -- each a persistent grid of fixed size that walks a
// device-resident work list (step tiles, force clusters, neighbour blocks)
// whose length it reads from device memory.  Because neither grid sizes nor
// pointers change when replicas join or leave, one CUDA graph of G steps is
// captured once per batch and replayed for the batch's lifetime: continuous
// batching without re-capture (a graph is captured again only when the set
// of classes present changes, a work list outgrows its array, or the
// autotuner changes a grid).  Per-replica
// step counters, step budgets and the "at integer time" flag live on the
// device, so every replica runs exactly its own number of steps.
//
// A replica's arithmetic never depends on the other replicas or on the tile
// size: the fused step is per (atom, component, mode) task, the force sums
// depend only on the replica's interacting pairs (neighbour buckets keyed by
// index), so a replica's trajectory is bitwise the same alone and in any mix.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "pimd.h"
#include "runtime.h"

namespace cg = cooperative_groups;

namespace pimd {

cudaError_t launch_pna_to_nap(const double *src, double *dst, int N, int P, cudaStream_t s);
cudaError_t launch_nap_to_pna(const double *src, double *dst, int N, int P, cudaStream_t s);
cudaError_t launch_thermal_v(double *v, const double *sigv, const double *imu, uint64_t seed, int N, int P,
                             cudaStream_t s);
cudaError_t launch_compress_split(const SplitStepArgs &a, const double *x, const double *v, cudaStream_t s);
cudaError_t launch_expand_split(const SplitStepArgs &a, const float *F, double *x, double *v, double *Fd,
                                cudaStream_t s);
cudaError_t launch_centroids(const NbrArgs &a, double *ccur, cudaStream_t s);
int water_lane_groups(int P);

constexpr int kTileMax = 3 * 512;   // largest A * 3 * P of a step tile (A P <= 512)
constexpr int kMmaRowsMax = 192;    // padded rows 8 NT of the tensor-core path (A P <= 512)
constexpr int kMmaTile = 2304;      // max padded rows x (P + 4) over P % 8 == 0
constexpr int kStepSmem = 3 * kMmaTile;   // floats; >= 4 * kTileMax
constexpr int kBatchMaxMol = 4096;   // molecules per replica (centroids staged in shared memory)
constexpr int kNbrMolPerItem = 8;    // molecules per neighbour-list work item
constexpr int kNbrThreads = 32 * kNbrMolPerItem;   // one warp per molecule
constexpr size_t kNbrSmem = 3 * kBatchMaxMol * sizeof(float);
constexpr int kOutStride = 3 * kMaxBeads + 10;  // pimd_estimates layout from K_mode on
constexpr int kEstItems = 64;        // estimator work items (e-blocks) per replica, at most
// Per-replica control words.  kCtlSkin holds two 32-bit maxima of this step
// (bit patterns of non-negative floats, merged by atomicMax): the squared
// centroid drift of the oxygens since the last rebuild and their squared bead
// spread about the centroid.
enum {
  kCtlStep = 0, kCtlLeft = 1, kCtlFirst = 2, kCtlActive = 3, kCtlClose = 4, kCtlRebuilds = 5, kCtlSkin = 6,
  kCtlWords = 8
};

// Merge a step item's squared drift (which 0) or spread (which 1) maximum.
__device__ __forceinline__ void skin_max(long long *ctl, int which, float v2) {
  atomicMax(reinterpret_cast<unsigned int *>(ctl + kCtlSkin) + which, __float_as_uint(v2));
}

struct RepDesc {
  int live, N, P, nmol, A, G, integrator, thermo;
  int nstep_items, ne;
  int ffma;                   // 1: block-item step with FP32 FMA transforms (comparison path)
  int pad1;
  uint64_t seed;
  double dt, tA, c1_0, c2_0, kT, volume, wn2;
  double dr0;                 // tA / sqrt(P): centroid drift per unit v~_0
  double box[3], invbox[3];
  double kb, r0, kth, th0, eps, sig, rc, rlist, skin;
  // FP32 copies for the force kernel: box, 1/box, kb, r0, kth, th0, rc^2,
  // sigma^2, 4 eps, 24 eps
  float boxf[3], invboxf[3], kbf, r0f, kthf, th0f, rc2f, sig2f, e4f, e24f;
  long long *ctl;
  double *xc, *v0;
  float *d, *vk, *F, *xcw;
  float *pO;                  // [nmol][3][P] oxygen bead positions xcw + d (FP32), for the pair loop
  const double *inv_mm, *sigv, *mass_mm;
  const float *inv_mmf, *sigvf;   // FP32 copies for the FP32 mode updates
  const float *Mf, *Mtf, *cAf, *sAf, *wsAf, *c1f, *c2f;
  const double *Mt64, *lam;
  // tensor-core path (P % 8 == 0): M (forward) and M^T (inverse) as TF32
  // hi/lo halves in m16n8k8 A-fragment order [mode tile][k step][lane][4]
  const float4 *mfa_hi, *mfa_lo, *mia_hi, *mia_lo;
  double *cref, *ccur;
  int *nbr, *nbr_off;
  double *Upart, *Wpart, *epart;
  const int *mperm;           // [nmol] molecules in space-filling-curve order (force work order)
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Per-replica control, one thread per slot.
//   mode 0 (begin step): apply the previous step's advance, then mark the
//                        replica active for this step if it has steps left
//   mode 1 (finalize):   apply the last advance; a replica that stepped since
//                        its last closing kick needs one now
//   mode 2 (after close): the closed replicas are at integer time again
// Mode 0 also resets the item counter of the warp-item step kernel and the
// rebuild list.
__global__ void k_bctl(const RepDesc *reps, int nslots, int mode, int *wnext) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (mode == 0 && r == 0 && wnext) {
    wnext[0] = 0;   // warp-item counter of the step kernel
    wnext[1] = 0;   // length of this step's rebuild list
    wnext[3] = 0;   // warp-item counter of the 128-bead step kernel
    wnext[5] = 0;   // warp-item counter of the 8-, 16-, 32-bead step kernel
  }
  if (r >= nslots || !reps[r].live) return;
  long long *c = reps[r].ctl;
  if (mode < 2 && c[kCtlActive]) {
    c[kCtlStep] += 1;
    c[kCtlLeft] -= 1;
    c[kCtlFirst] = 0;
    c[kCtlActive] = 0;
  }
  if (mode == 0) {
    c[kCtlActive] = c[kCtlLeft] > 0;
    c[kCtlSkin] = 0;
  }
  if (mode == 1) c[kCtlClose] = c[kCtlFirst] == 0;
  if (mode == 2 && c[kCtlClose]) {
    c[kCtlFirst] = 1;
    c[kCtlClose] = 0;
  }
}

// FP32 Box-Muller on the 24 high bits of Philox words: u = (w >> 8 + 1/2) 2^-24
// in (0, 1), radius sqrt(-2 ln u) and angle 2 pi u' from hardware
// approximations (errors near 1e-6 of the deviate).  sin and cos of 2 pi u'
// are taken as -sin, -cos of pi (2 u' - 1), whose argument lies in (-pi, pi).
__device__ __forceinline__ float bm_radius(uint32_t w) {
  const float u = fmaf((float)(w >> 8), 5.9604644775390625e-8f, 2.98023223876953125e-8f);
  const float x = fmaxf(-2.0f * __logf(u), 1e-30f);
  return x * rsqrtf(x);
}
__device__ __forceinline__ float bm_angle(uint32_t w) {   // pi (2 u - 1)
  const float u = fmaf((float)(w >> 8), 5.9604644775390625e-8f, 2.98023223876953125e-8f);
  return 3.14159265358979f * fmaf(2.0f, u, -1.0f);
}

__device__ __forceinline__ float gauss1f_b(uint64_t seed, uint32_t atom, uint32_t mode, uint32_t stream,
                                           uint64_t step, int d) {
  const uint4 w = philox4x32_10(
      make_uint4(atom, (mode & 0xffffu) | (stream << 16), (uint32_t)step, (uint32_t)(step >> 32)),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float r = bm_radius(d < 2 ? w.x : w.z);
  const float b = bm_angle(d < 2 ? w.y : w.w);
  return -r * (d == 1 ? __sinf(b) : __cosf(b));
}

__device__ __forceinline__ void rotb(float &q, float &v, float c, float s_over_w, float w_s) {
  const float qn = fmaf(c, q, s_over_w * v);
  const float vn = fmaf(-w_s, q, c * v);
  q = qn;
  v = vn;
}

__device__ __forceinline__ float wrapb(double x, double L, double invL) {
  return (float)(x - L * floor(x * invL));
}

__device__ __forceinline__ float micb(float d, float L, float invL) { return fmaf(-rintf(d * invL), L, d); }

// Three standard normal deviates of (atom, mode, stream, step) in FP32 from
// one Philox call (the same words and mapping as gauss1f_b per component).
__device__ __forceinline__ void gauss3f_b(uint64_t seed, uint32_t atom, uint32_t mode, uint32_t stream,
                                          uint64_t step, float &e0, float &e1, float &e2) {
  const uint4 w = philox4x32_10(
      make_uint4(atom, (mode & 0xffffu) | (stream << 16), (uint32_t)step, (uint32_t)(step >> 32)),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float r0 = bm_radius(w.x), r1 = bm_radius(w.z);
  float sn, cs;
  __sincosf(bm_angle(w.y), &sn, &cs);
  e0 = -r0 * cs;
  e1 = -r0 * sn;
  e2 = -r1 * __cosf(bm_angle(w.w));
}

// ---- tensor-core mode transforms (P % 8 == 0) -------------------------------
// The forward transforms F~ = M F and q~ = M d and the inverse d' = M^T q~' of
// a tile are GEMMs with K = P: A = the P x P matrix (rows padded to 16),
// B = the tile's rows (one column per atom-component row, padded to 8).
// mma.sync m16n8k8 in TF32 with the 3xTF32 split (a = a_hi + a_lo in TF32;
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi) keeps FP32-level accuracy.

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kMmaPairsMax = 6;   // (mode tile, row tile) pairs per warp

// acc[p][0..3] = (A B1) tile, acc[p][4..7] = (A B2) tile for the warp's pairs
// p = warp, warp + 4, ...; B1, B2 are [row][k] arrays with row stride PS.
__device__ __forceinline__ void mma_gemm2(const float4 *__restrict__ ahi, const float4 *__restrict__ alo, int KS,
                                          int MT, int NT, const float *B1, const float *B2, int PS,
                                          float (&acc)[kMmaPairsMax][8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int p = 0; p < kMmaPairsMax; ++p) {
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;
    const int pair = warp + 4 * p;
    if (pair >= MT * NT) continue;
    const int mt = pair / NT, nt = pair - mt * NT;
    const float *b1 = B1 + (8 * nt + g) * PS + t;
    const float *b2 = B2 ? B2 + (8 * nt + g) * PS + t : nullptr;
    for (int ks = 0; ks < KS; ++ks) {
      const float4 h = __ldg(ahi + ((size_t)mt * KS + ks) * 32 + lane);
      const float4 l = __ldg(alo + ((size_t)mt * KS + ks) * 32 + lane);
      const uint32_t ah[4] = {__float_as_uint(h.x), __float_as_uint(h.y), __float_as_uint(h.z), __float_as_uint(h.w)};
      const uint32_t al[4] = {__float_as_uint(l.x), __float_as_uint(l.y), __float_as_uint(l.z), __float_as_uint(l.w)};
      {
        const float x0 = b1[8 * ks], x1 = b1[8 * ks + 4];
        const uint32_t h0 = tf32_rna(x0), h1 = tf32_rna(x1);
        const uint32_t l0 = tf32_rna(x0 - __uint_as_float(h0)), l1 = tf32_rna(x1 - __uint_as_float(h1));
        float (&c)[4] = *reinterpret_cast<float(*)[4]>(&acc[p][0]);
        mma_tf32(c, al, h0, h1);
        mma_tf32(c, ah, l0, l1);
        mma_tf32(c, ah, h0, h1);
      }
      if (b2) {
        const float x0 = b2[8 * ks], x1 = b2[8 * ks + 4];
        const uint32_t h0 = tf32_rna(x0), h1 = tf32_rna(x1);
        const uint32_t l0 = tf32_rna(x0 - __uint_as_float(h0)), l1 = tf32_rna(x1 - __uint_as_float(h1));
        float (&c)[4] = *reinterpret_cast<float(*)[4]>(&acc[p][4]);
        mma_tf32(c, al, h0, h1);
        mma_tf32(c, ah, l0, l1);
        mma_tf32(c, ah, h0, h1);
      }
    }
  }
}

// Writes a GEMM result tile pair back as [row][col] with row stride PS:
// D[col = 16 mt + g (+8)][row = 8 nt + 2 t (+1)] from the C fragment.
__device__ __forceinline__ void mma_store(const float (&acc)[kMmaPairsMax][8], int half, int MT, int NT, int P,
                                          int rows, float *dst, int PS) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int p = 0; p < kMmaPairsMax; ++p) {
    const int pair = warp + 4 * p;
    if (pair >= MT * NT) continue;
    const int mt = pair / NT, nt = pair - mt * NT;
    const int c0 = 16 * mt + g, r0 = 8 * nt + 2 * t;
    const float *c = &acc[p][4 * half];
    if (c0 < P) {
      if (r0 < rows) dst[r0 * PS + c0] = c[0];
      if (r0 + 1 < rows) dst[(r0 + 1) * PS + c0] = c[1];
    }
    if (c0 + 8 < P) {
      if (r0 < rows) dst[r0 * PS + c0 + 8] = c[2];
      if (r0 + 1 < rows) dst[(r0 + 1) * PS + c0 + 8] = c[3];
    }
  }
}

// The batched step of one tile on tensor cores.  sF, sX, sV: [row][P] tiles
// with row stride PS = P + 4 (bank-conflict-free B fragments).
__device__ __forceinline__ void bstep_mma(const RepDesc *__restrict__ Rp, int P, int tile0, int na, size_t base,
                                          float *sF, float *sX, float *sV, uint64_t step, int first) {
  const int PS = P + 4;
  const int rows = na * 3;
  const int NT = (rows + 7) >> 3;
  const int MT = (P + 15) >> 4;
  const int KS = P >> 3;
  float acc[kMmaPairsMax][8];
  mma_gemm2(Rp->mfa_hi, Rp->mfa_lo, KS, MT, NT, sF, sX, PS, acc);
  __syncthreads();
  mma_store(acc, 0, MT, NT, P, rows, sF, PS);   // F~ [row][mode]
  mma_store(acc, 1, MT, NT, P, rows, sX, PS);   // q~ [row][mode]
  __syncthreads();
  // per-mode update: thread (atom al, modes 4 g4 .. 4 g4 + 3), all components
  const int NG = P >> 2;
  const float *__restrict__ cAf = Rp->cAf;
  const float *__restrict__ sAf = Rp->sAf;
  const float *__restrict__ wsAf = Rp->wsAf;
  const float *__restrict__ c1f = Rp->c1f;
  const float *__restrict__ c2f = Rp->c2f;
  const double *__restrict__ inv_mm = Rp->inv_mm;
  const double *__restrict__ sigv = Rp->sigv;
  float *__restrict__ vkg = Rp->vk;
  double *__restrict__ xcg = Rp->xc;
  double *__restrict__ v0g = Rp->v0;
  float *__restrict__ xcw = Rp->xcw;
  const int integ = Rp->integrator, thermo = Rp->thermo;
  const uint64_t seed = Rp->seed;
  const double dt = Rp->dt;
  const float hd = (float)dt, half = 0.5f * hd;
  const float kick = first ? half : hd;
  const float *__restrict__ inv_mmf = Rp->inv_mmf;
  const float *__restrict__ sigvf = Rp->sigvf;
  for (int task = threadIdx.x; task < na * NG; task += blockDim.x) {
    const int al = task / NG, g4 = task - al * NG;
    const int i = tile0 + al;
    const float im = __ldg(inv_mmf + i);
    const float sg = __ldg(sigvf + i);
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
      const int k = 4 * g4 + tt;
      if (k == 0) continue;   // the centroid mode: packed FP64 phase below
      const float cA = __ldg(cAf + k), sA = __ldg(sAf + k), wsA = __ldg(wsAf + k);
      const float c1 = __ldg(c1f + k), c2s = __ldg(c2f + k) * sg;
      float e[3] = {0.f, 0.f, 0.f}, e2[3] = {0.f, 0.f, 0.f};
      if (thermo) gauss3f_b(seed, (uint32_t)i, (uint32_t)k, kStreamO1, step, e[0], e[1], e[2]);
      if (thermo && integ == 1 && !first)
        gauss3f_b(seed, (uint32_t)i, (uint32_t)k, kStreamO2, step - 1, e2[0], e2[1], e2[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int sidx = (al * 3 + c) * PS + k;
        float v = sV[sidx];
        float qq = sX[sidx];
        const float ff = sF[sidx];
        if (integ == 0) {
          v = fmaf(kick * im, ff, v);
          rotb(qq, v, cA, sA, wsA);
          if (thermo) v = fmaf(c1, v, c2s * e[c]);
          rotb(qq, v, cA, sA, wsA);
        } else {
          const float kb = half * im;
          if (!first) {
            v = fmaf(kb, ff, v);
            if (thermo) v = fmaf(c1, v, c2s * e2[c]);
          }
          if (thermo) v = fmaf(c1, v, c2s * e[c]);
          v = fmaf(kb, ff, v);
          rotb(qq, v, cA, sA, wsA);
        }
        sX[sidx] = qq;
        vkg[base + (size_t)(al * 3 + c) * P + k] = v;
      }
    }
  }
  // centroid mode, FP64, one (atom, component) per lane: q~_0 = sqrt(P) xc
  {
    const double dr = Rp->dr0, c1_0 = Rp->c1_0;
    const double kfac = (integ == 0 ? (first ? 0.5 : 1.0) : 0.5) * dt;
    for (int t = threadIdx.x; t < na * 3; t += blockDim.x) {
      const int al = t / 3, c = t - 3 * al;
      const int i = tile0 + al;
      const size_t ic = (size_t)i * 3 + c;
      // one Philox draw serves the three components; components are lanes here
      float e = 0.f, e2 = 0.f;
      if (thermo) {
        float a0, a1, a2;
        gauss3f_b(seed, (uint32_t)i, 0u, kStreamO1, step, a0, a1, a2);
        e = c == 0 ? a0 : (c == 1 ? a1 : a2);
        if (integ == 1 && !first) {
          gauss3f_b(seed, (uint32_t)i, 0u, kStreamO2, step - 1, a0, a1, a2);
          e2 = c == 0 ? a0 : (c == 1 ? a1 : a2);
        }
      }
      const double kb = kfac * __ldg(inv_mm + i);
      const double c2s = Rp->c2_0 * __ldg(sigv + i);
      const double f0 = (double)sF[t * PS];
      double x = xcg[ic], v = v0g[ic];
      if (integ == 0) {
        v = fma(kb, f0, v);
        x = fma(dr, v, x);
        if (thermo) v = fma(c1_0, v, c2s * (double)e);
        x = fma(dr, v, x);
      } else {
        if (!first) {
          v = fma(kb, f0, v);
          if (thermo) v = fma(c1_0, v, c2s * (double)e2);
        }
        if (thermo) v = fma(c1_0, v, c2s * (double)e);
        v = fma(kb, f0, v);
        x = fma(dr, v, x);
      }
      xcg[ic] = x;
      v0g[ic] = v;
      xcw[ic] = wrapb(x, Rp->box[c], Rp->invbox[c]);
      sX[t * PS] = 0.f;   // the deviations carry no centroid mode
    }
  }
  __syncthreads();
  // inverse: d' = M^T q~' (mode 0 zeroed above)
  mma_gemm2(Rp->mia_hi, Rp->mia_lo, KS, MT, NT, sX, nullptr, PS, acc);
  mma_store(acc, 0, MT, NT, P, rows, sF, PS);   // new deviations [row][bead] into sF
  __syncthreads();
  float *__restrict__ dg = Rp->d + base;
  for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5)
    for (int j = threadIdx.x & 31; j < P; j += 32) dg[r * P + j] = sF[r * PS + j];
}

// ---- warp-item step on tensor cores: P in {8, 16, 32, 64} --------------------
// One warp advances a tile of 8 atoms x 3 components x P beads with no block
// barrier, so the warps of an SM overlap one another's memory waits.  Per
// component c the forward transforms are GEMMs C[mode][atom] = M[mode][bead]
// X_c[bead][atom] whose B operand (8 atoms = one n-tile) is the staged tile;
// the C fragment of lane (g, t) then holds modes {16 mt + g, 16 mt + g + 8} of
// atoms {2t, 2t + 1} for all three components, so one Philox draw per
// (atom, mode) serves the three components in registers, and the mode update
// runs on the accumulators.  The inverse d'_c[bead][atom] = M^T q~'_c reads
// q~' back from shared memory as its B operand.  3xTF32 throughout.
constexpr int kWAtoms = 8;      // atoms per warp item
constexpr int kWWarps = 4;      // warps per block
constexpr int kWMaxP = 64;
__host__ __device__ constexpr int wslot_floats(int P) { return 48 * (P + 4) + 128; }
__host__ __device__ constexpr bool warp_class(int P) { return P == 8 || P == 16 || P == 32 || P == 64; }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void split_tf32(float x, uint32_t &h, uint32_t &l) {
  h = tf32_rna(x);
  l = tf32_rna(x - __uint_as_float(h));
}

// c += A B with the 3xTF32 split, small terms first
__device__ __forceinline__ void mma3(float (&c)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  mma_tf32(c, al, bh0, bh1);
  mma_tf32(c, ah, bl0, bl1);
  mma_tf32(c, ah, bh0, bh1);
}

// A fragment of a mode-matrix table, kept in L1 in preference to streamed data
__device__ __forceinline__ float4 ld_frag(const float4 *p) {
  float4 v;
  asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}

__device__ __forceinline__ void frag_u32(const float4 &v, uint32_t (&a)[4]) {
  a[0] = __float_as_uint(v.x);
  a[1] = __float_as_uint(v.y);
  a[2] = __float_as_uint(v.z);
  a[3] = __float_as_uint(v.w);
}

// C_c[mode][atom] = M[mode][bead] S_c[bead][atom] for the three components of
// a staged tile S ([c*8 + atom][bead], row stride P + 4), all mode tiles.
template <int P>
__device__ __forceinline__ void fwd_tile(const float4 *__restrict__ thi, const float4 *__restrict__ tlo,
                                         const float *__restrict__ S, float (&C)[(P + 15) / 16][3][4]) {
  constexpr int PS = P + 4, MT = (P + 15) / 16, KS = P / 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) C[mt][c][q] = 0.f;
#pragma unroll 2
  for (int ks = 0; ks < KS; ++ks) {
    uint32_t bh[3][2], bl[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int so = (c * 8 + g) * PS + 8 * ks + t;
      split_tf32(S[so], bh[c][0], bl[c][0]);
      split_tf32(S[so + 4], bh[c][1], bl[c][1]);
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      uint32_t ah[4], al[4];
      const int o = (mt * KS + ks) * 32 + lane;
      frag_u32(ld_frag(thi + o), ah);
      frag_u32(ld_frag(tlo + o), al);
#pragma unroll
      for (int c = 0; c < 3; ++c) mma3(C[mt][c], ah, al, bh[c][0], bh[c][1], bl[c][0], bl[c][1]);
    }
  }
}

// Shared-memory slot of one warp (floats): staged forces [c*8 + atom][bead]
// and deviations (the latter reused as q~' [c][mode][atom]), row stride P + 4
// (conflict-free B fragments); then F~_0, the centroid-mode noise of both
// streams per (atom, component) and the new FP64 centroids.
template <int P>
__device__ void bstep_warp(const RepDesc *__restrict__ Rp, int tile, float *__restrict__ slot, uint64_t step,
                           int first) {
  constexpr int PS = P + 4, MT = (P + 15) / 16, KS = P / 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int tile0 = tile * kWAtoms;
  const int na = min(kWAtoms, Rp->N - tile0);
  const size_t base = (size_t)tile0 * 3 * P;
  float *sF = slot;
  float *sX = slot + 24 * PS;
  float *__restrict__ sf0 = slot + 48 * PS;
  float *__restrict__ se = sf0 + 24;
  float *__restrict__ se2 = se + 24;
  double *__restrict__ sxc = reinterpret_cast<double *>(se2 + 24);
  {
    constexpr int CPR = P / 4;   // 16-byte chunks per (atom, component) row
    const float *__restrict__ gF = Rp->F + base;
    const float *__restrict__ gX = Rp->d + base;
    const int nchunk = na * 3 * CPR;
    for (int q = lane; q < nchunk; q += 32) {
      const int row = q / CPR, col = (q - row * CPR) * 4;
      const int a = row / 3, c = row - 3 * a;
      const int so = (c * 8 + a) * PS + col;
      cp_async16(sF + so, gF + (size_t)row * P + col);
      cp_async16(sX + so, gX + (size_t)row * P + col);
    }
    cp_async_commit();
    for (int q = lane; q < (kWAtoms - na) * 3 * P; q += 32) {   // rows of missing atoms
      const int r = q / P, j = q - r * P;
      const int a = na + r / 3, c = r - 3 * (r / 3);
      sF[(c * 8 + a) * PS + j] = 0.f;
      sX[(c * 8 + a) * PS + j] = 0.f;
    }
  }
  const int integ = Rp->integrator, thermo = Rp->thermo;
  const uint64_t seed = Rp->seed;
  const double dt = Rp->dt;
  const float hd = (float)dt, half = 0.5f * hd;
  const float kick = first ? half : hd;
  const float *__restrict__ cAf = Rp->cAf;
  const float *__restrict__ sAf = Rp->sAf;
  const float *__restrict__ wsAf = Rp->wsAf;
  const float *__restrict__ c1f = Rp->c1f;
  const float *__restrict__ c2f = Rp->c2f;
  float *__restrict__ vkg = Rp->vk + base;
  // per-lane atom constants (atoms 2t, 2t + 1) and the centroid prefetch
  float imv[2], sgv[2];
#pragma unroll
  for (int aa = 0; aa < 2; ++aa) {
    const int a = min(2 * t + aa, na - 1);
    imv[aa] = __ldg(Rp->inv_mmf + tile0 + a);
    sgv[aa] = __ldg(Rp->sigvf + tile0 + a);
  }
  cp_async_wait_all();
  __syncwarp();

  // v~ of update iteration j (modes 16 (j/2) + g + 8 (j%2), atoms 2t, 2t + 1),
  // loaded one iteration ahead; the centroid mode and padding rows read none
  auto load_v = [&](int j, float (&vv)[2][3]) {
    const int k = 16 * (j >> 1) + g + 8 * (j & 1);
    const bool on = k < P && k != 0;
#pragma unroll
    for (int aa = 0; aa < 2; ++aa) {
      const int a = min(2 * t + aa, na - 1);
#pragma unroll
      for (int c = 0; c < 3; ++c) vv[aa][c] = on ? __ldcs(vkg + (a * 3 + c) * P + k) : 0.f;
    }
  };
  float vv[2][3], vn[2][3];
  const float4 *__restrict__ fhi = Rp->mfa_hi;
  const float4 *__restrict__ flo = Rp->mfa_lo;
  float *sQ = sX;   // q~ [c][mode][atom] once the deviations are transformed
  float C[MT][3][4];
  // forward transform of the deviations: q~_c = M d_c
  fwd_tile<P>(fhi, flo, sX, C);
  __syncwarp();   // every lane is done with the staged deviations
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int k = 16 * mt + g;
      *reinterpret_cast<float2 *>(sQ + (c * P + k) * 8 + 2 * t) = make_float2(C[mt][c][0], C[mt][c][1]);
      if (k + 8 < P)
        *reinterpret_cast<float2 *>(sQ + (c * P + k + 8) * 8 + 2 * t) = make_float2(C[mt][c][2], C[mt][c][3]);
    }
  // forward transform of the forces: F~_c = M F_c, then F~ [c][mode][atom]
  // over the staged forces
  fwd_tile<P>(fhi, flo, sF, C);
  __syncwarp();   // every lane is done with the staged forces
  float *sG = sF;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int k = 16 * mt + g;
      *reinterpret_cast<float2 *>(sG + (c * P + k) * 8 + 2 * t) = make_float2(C[mt][c][0], C[mt][c][1]);
      if (k + 8 < P)
        *reinterpret_cast<float2 *>(sG + (c * P + k + 8) * 8 + 2 * t) = make_float2(C[mt][c][2], C[mt][c][3]);
    }
  // mode update: lane (g, t) owns modes {16 mt + g, 16 mt + g + 8} of atoms
  // {2t, 2t + 1}, the same (mode, atom) slots it wrote; q~' replaces q~
  load_v(0, vv);
  double xpre = 0.0, vpre = 0.0;   // this lane's centroid entry, used after the update
  if (lane < 3 * na) {
    xpre = Rp->xc[(size_t)tile0 * 3 + lane];
    vpre = Rp->v0[(size_t)tile0 * 3 + lane];
  }
#pragma unroll 1
  for (int j = 0; j < 2 * MT; ++j) {
    if (j + 1 < 2 * MT) load_v(j + 1, vn);
    const int k = 16 * (j >> 1) + g + 8 * (j & 1);
    if (k >= P) {
#pragma unroll
      for (int aa = 0; aa < 2; ++aa)
#pragma unroll
        for (int c = 0; c < 3; ++c) vv[aa][c] = vn[aa][c];
      continue;
    }
    const float cA = __ldg(cAf + k), sA = __ldg(sAf + k), wsA = __ldg(wsAf + k);
    const float c1 = __ldg(c1f + k), c2 = __ldg(c2f + k);
    float2 qv[3], fv[3];
    float e[2][3], e2[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      qv[c] = *reinterpret_cast<const float2 *>(sQ + (c * P + k) * 8 + 2 * t);
      fv[c] = *reinterpret_cast<const float2 *>(sG + (c * P + k) * 8 + 2 * t);
    }
#pragma unroll
    for (int aa = 0; aa < 2; ++aa) {
      const int a = min(2 * t + aa, na - 1);
#pragma unroll
      for (int c = 0; c < 3; ++c) e[aa][c] = e2[aa][c] = 0.f;
      if (thermo) gauss3f_b(seed, (uint32_t)(tile0 + a), (uint32_t)k, kStreamO1, step, e[aa][0], e[aa][1], e[aa][2]);
      if (thermo && integ == 1 && !first)
        gauss3f_b(seed, (uint32_t)(tile0 + a), (uint32_t)k, kStreamO2, step - 1, e2[aa][0], e2[aa][1], e2[aa][2]);
    }
    if (k == 0) {   // the centroid mode: FP64 phase below
#pragma unroll
      for (int aa = 0; aa < 2; ++aa) {
        const int a = 2 * t + aa;
        if (a >= na) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sf0[a * 3 + c] = aa == 0 ? fv[c].x : fv[c].y;
          se[a * 3 + c] = e[aa][c];
          se2[a * 3 + c] = e2[aa][c];
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) qv[c] = make_float2(0.f, 0.f);   // the deviations carry no centroid mode
    } else {
#pragma unroll
      for (int aa = 0; aa < 2; ++aa) {
        const int a = 2 * t + aa;
        if (a >= na) continue;
        const float im = imv[aa], c2s = c2 * sgv[aa];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float v = vv[aa][c], qq = aa == 0 ? qv[c].x : qv[c].y;
          const float ff = aa == 0 ? fv[c].x : fv[c].y;
          if (integ == 0) {
            v = fmaf(kick * im, ff, v);
            rotb(qq, v, cA, sA, wsA);
            if (thermo) v = fmaf(c1, v, c2s * e[aa][c]);
            rotb(qq, v, cA, sA, wsA);
          } else {
            const float kb = half * im;
            if (!first) {
              v = fmaf(kb, ff, v);
              if (thermo) v = fmaf(c1, v, c2s * e2[aa][c]);
            }
            if (thermo) v = fmaf(c1, v, c2s * e[aa][c]);
            v = fmaf(kb, ff, v);
            rotb(qq, v, cA, sA, wsA);
          }
          if (aa == 0) qv[c].x = qq; else qv[c].y = qq;
          __stcs(vkg + (a * 3 + c) * P + k, v);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) *reinterpret_cast<float2 *>(sQ + (c * P + k) * 8 + 2 * t) = qv[c];
#pragma unroll
    for (int aa = 0; aa < 2; ++aa)
#pragma unroll
      for (int c = 0; c < 3; ++c) vv[aa][c] = vn[aa][c];
  }
  __syncwarp();
  // centroid mode in FP64, one (atom, component) per lane: q~_0 = sqrt(P) xc
  if (lane < 3 * na) {
    const int a = lane / 3, c = lane - 3 * a;
    const int i = tile0 + a;
    const size_t ic = (size_t)tile0 * 3 + lane;
    // the increments (kick, noise) are products of FP32 quantities, formed
    // in FP32; the velocity and position accumulate them in FP64
    const double dr = Rp->dr0, c1_0 = Rp->c1_0;
    const float kbf = (integ == 0 ? kick : half) * __ldg(Rp->inv_mmf + i);
    const float c2sf = __ldg(c2f) * __ldg(Rp->sigvf + i);
    const float f0 = sf0[lane];
    const float e = se[lane], e2 = se2[lane];
    double x = xpre, v = vpre;
    if (integ == 0) {
      v += (double)(kbf * f0);
      x = fma(dr, v, x);
      if (thermo) v = fma(c1_0, v, (double)(c2sf * e));
      x = fma(dr, v, x);
    } else {
      if (!first) {
        v += (double)(kbf * f0);
        if (thermo) v = fma(c1_0, v, (double)(c2sf * e2));
      }
      if (thermo) v = fma(c1_0, v, (double)(c2sf * e));
      v += (double)(kbf * f0);
      x = fma(dr, v, x);
    }
    Rp->xc[ic] = x;
    Rp->v0[ic] = v;
    const float xw = wrapb(x, Rp->box[c], Rp->invbox[c]);
    Rp->xcw[ic] = xw;
    sxc[lane] = x;
    sf0[lane] = xw;   // this lane's own entry, read above
  }
  // inverse: d'_c = M^T q~'_c, bead tiles of 16 as the M dimension
  const float4 *__restrict__ ihi = Rp->mia_hi;
  const float4 *__restrict__ ilo = Rp->mia_lo;
  float D[MT][3][4];
#pragma unroll
  for (int bt = 0; bt < MT; ++bt)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) D[bt][c][q] = 0.f;
#pragma unroll 2
  for (int ks = 0; ks < KS; ++ks) {
    uint32_t bh[3][2], bl[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float *qp = sQ + (c * P + 8 * ks + t) * 8 + g;
      split_tf32(qp[0], bh[c][0], bl[c][0]);
      split_tf32(qp[32], bh[c][1], bl[c][1]);
    }
#pragma unroll
    for (int bt = 0; bt < MT; ++bt) {
      uint32_t ah[4], al[4];
      const int o = (bt * KS + ks) * 32 + lane;
      frag_u32(ld_frag(ihi + o), ah);
      frag_u32(ld_frag(ilo + o), al);
#pragma unroll
      for (int c = 0; c < 3; ++c) mma3(D[bt][c], ah, al, bh[c][0], bh[c][1], bl[c][0], bl[c][1]);
    }
  }
  __syncwarp();   // the centroids in sxc are visible to every lane
  // new deviations, and the skin criterion: bead spread of the oxygens
  // (water-like systems, which carry reference centroids)
  const bool water = Rp->cref != nullptr;
  float *__restrict__ dg = Rp->d + base;
  float vdev = 0.f;
#pragma unroll
  for (int bt = 0; bt < MT; ++bt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int bead = 16 * bt + g + 8 * (q >> 1);
      const int a = 2 * t + (q & 1);
      if (bead < P && a < na) {
#pragma unroll
        for (int c = 0; c < 3; ++c) __stcs(dg + (a * 3 + c) * P + bead, D[bt][c][q]);
        if (water && (tile0 + a) % 3 == 0) {
          if (Rp->pO) {
            float *po = Rp->pO + (size_t)(tile0 + a) * P + bead;   // molecule (tile0 + a) / 3, row 3 m + c
#pragma unroll
            for (int c = 0; c < 3; ++c) po[c * P] = sf0[a * 3 + c] + D[bt][c][q];
          }
          const float s2 = D[bt][0][q] * D[bt][0][q] + D[bt][1][q] * D[bt][1][q] + D[bt][2][q] * D[bt][2][q];
          vdev = fmaxf(vdev, s2 == s2 ? s2 : __int_as_float(0x7f800000));   // NaN forces a rebuild
        }
      }
    }
  // centroid drift of the oxygens since the last rebuild
  float vdisp = 0.f;
  if (water && lane < na && (tile0 + lane) % 3 == 0) {
    const int m = (tile0 + lane) / 3;
    double s2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = sxc[lane * 3 + c];
      const double gd = x - Rp->cref[3 * m + c];
      s2 = fma(gd, gd, s2);
      Rp->ccur[3 * m + c] = x;
    }
    vdisp = s2 == s2 ? (float)s2 : __int_as_float(0x7f800000);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vdisp = fmaxf(vdisp, __shfl_xor_sync(0xffffffffu, vdisp, o));
    vdev = fmaxf(vdev, __shfl_xor_sync(0xffffffffu, vdev, o));
  }
  if (water && lane < 2) skin_max(Rp->ctl, lane, lane == 0 ? vdisp : vdev);
  __syncwarp();   // the slot is free for the next item
}

// Warp items (replica, 8-atom tile) of the bead counts in {8, 16, 32, 64}:
// the 64-bead items are the range [0, counts[9]) of the step list, claimed
// from *next; the 8-, 16- and 32-bead items the range [counts[9], counts[4]),
// run by the kSmall instance, whose smaller accumulator tiles fit four blocks
// per SM (128 registers, 7.4 KB warp slots) where the 64-bead instance fits
// three.  Lane 0 of each warp claims the next item (counters reset by k_bctl).
template <bool kSmall>
__global__ void __launch_bounds__(kWWarps * 32, kSmall ? 4 : 3) k_bstep_w(const RepDesc *__restrict__ reps,
                                                                         const int2 *__restrict__ items,
                                                                         const int *__restrict__ counts, int *next,
                                                                         int slot_floats) {
  extern __shared__ __align__(16) float wsm[];
  float *slot = wsm + (threadIdx.x >> 5) * slot_floats;
  const int lo = kSmall ? counts[9] : 0, hi = kSmall ? counts[4] : counts[9];
  const int lane = threadIdx.x & 31;
  for (;;) {
    int it = 0;
    if (lane == 0) it = lo + atomicAdd(next, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= hi) break;
    const int2 w = items[it];
    const RepDesc *__restrict__ Rp = reps + w.x;
    const long long *ctl = Rp->ctl;
    if (!ctl[kCtlActive]) continue;
    const uint64_t step = (uint64_t)ctl[kCtlStep];
    const int first = (int)ctl[kCtlFirst];
    if (kSmall) {
      switch (Rp->P) {
        case 8: bstep_warp<8>(Rp, w.y, slot, step, first); break;
        case 16: bstep_warp<16>(Rp, w.y, slot, step, first); break;
        case 32: bstep_warp<32>(Rp, w.y, slot, step, first); break;
        default: break;
      }
    } else if (Rp->P == 64) {
      bstep_warp<64>(Rp, w.y, slot, step, first);
    }
  }
}

// Warp items of bead count 128, the range [counts[4], counts[7]) of the step
// list: the same per-item arithmetic as k_bstep_w in a kernel of its own,
// whose larger accumulator tiles (eight mode tiles) and 26 KB warp slots
// would otherwise set the register and shared-memory budget of the smaller
// bead counts; claimed from the counter *next (reset by k_bctl).
__global__ void __launch_bounds__(kWWarps * 32, 1) k_bstep_w128(const RepDesc *__restrict__ reps,
                                                               const int2 *__restrict__ items,
                                                               const int *__restrict__ counts, int *next) {
  extern __shared__ __align__(16) float wsm[];
  float *slot = wsm + (threadIdx.x >> 5) * wslot_floats(128);
  const int lo = counts[4], hi = counts[7];
  const int lane = threadIdx.x & 31;
  for (;;) {
    int it = 0;
    if (lane == 0) it = lo + atomicAdd(next, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= hi) break;
    const int2 w = items[it];
    const RepDesc *__restrict__ Rp = reps + w.x;
    const long long *ctl = Rp->ctl;
    if (!ctl[kCtlActive] || Rp->P != 128) continue;
    bstep_warp<128>(Rp, w.y, slot, (uint64_t)ctl[kCtlStep], (int)ctl[kCtlFirst]);
  }
}

// The warp-item step of one system (a single-system handle in split
// precision, bead counts 8, 16, 32, 64, 128): the same per-item arithmetic as
// k_bstep_w, with the step index read from the handle's counter.  Warps take
// the 8-atom tiles in turn.  For water-like systems the last warp to finish
// turns the step's skin maxima (squared FP32 bit patterns in ctl) into the
// one conservative (drift, spread) pair that the neighbour-list check reads,
// and clears them for the next step (threadfence-and-count, no waiting).
// kClass: 0 the 32-bead instance (128 registers, four blocks per SM), 1 the
// 64-bead one (three blocks), 2 the 128-bead one (eight mode tiles, one
// block's share of registers), 3 the 8- and 16-bead one (one mode tile, six
// blocks: its short items leave the memory waits exposed unless more warps
// share an SM; 8 and 16 beads step 15% and 10% faster than at four blocks).
template <int kClass>
__global__ void __launch_bounds__(kWWarps * 32, kClass == 3 ? 6 : (kClass == 0 ? 4 : (kClass == 1 ? 3 : 1)))
    k_sstep_w(const RepDesc *__restrict__ Rp, const int64_t *__restrict__ stepp, int step_off, int first,
              int slot_floats, double *blkmax, unsigned *done) {
  extern __shared__ __align__(16) float wsm[];
  float *slot = wsm + (threadIdx.x >> 5) * slot_floats;
  const int lane = threadIdx.x & 31;
  const int ntiles = (Rp->N + kWAtoms - 1) / kWAtoms;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const uint64_t step = (uint64_t)(*stepp + step_off);
  for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles; tile += nw) {
    if (kClass == 3) {
      if (Rp->P == 8)
        bstep_warp<8>(Rp, tile, slot, step, first);
      else if (Rp->P == 16)
        bstep_warp<16>(Rp, tile, slot, step, first);
    } else if (kClass == 2) {
      if (Rp->P == 128) bstep_warp<128>(Rp, tile, slot, step, first);
    } else if (kClass == 1) {
      if (Rp->P == 64) bstep_warp<64>(Rp, tile, slot, step, first);
    } else if (Rp->P == 32) {
      bstep_warp<32>(Rp, tile, slot, step, first);
    }
  }
  if (!blkmax) return;
  __threadfence();
  if (lane == 0) {
    const unsigned t = atomicAdd(done, 1u);
    if (t == (unsigned)nw - 1) {
      __threadfence();
      const unsigned *w = reinterpret_cast<const unsigned *>(Rp->ctl + kCtlSkin);
      const float d2 = __uint_as_float(atomicOr(const_cast<unsigned *>(w), 0u));
      const float s2 = __uint_as_float(atomicOr(const_cast<unsigned *>(w) + 1, 0u));
      blkmax[0] = d2 <= 3.0e38f ? sqrt((double)d2) * (1.0 + 1e-6) : 1e300;
      blkmax[1] = s2 <= 3.0e38f ? sqrt((double)s2) * (1.0 + 1e-6) : 1e300;
      atomicExch(reinterpret_cast<unsigned long long *>(Rp->ctl + kCtlSkin), 0ull);
      atomicExch(done, 0u);
    }
  }
}

// The split-precision fused step (same arithmetic as the single-system split
// kernel) over the block items (replica, tile) of the bead counts outside the
// warp-item classes: the suffix [counts[7], counts[0]) of the step list.
// Every descriptor field an item
// needs is read once into registers (restrict-qualified), and the task index
// split (mode, row) uses shifts when P is a power of two.
__global__ void __launch_bounds__(128, 4) k_bstep(const RepDesc *__restrict__ reps, const int2 *__restrict__ items,
                                               const int *__restrict__ counts) {
  __shared__ __align__(16) float sbuf[kStepSmem];
  float *sD = sbuf, *sV = sbuf + kTileMax, *sF = sbuf + 2 * kTileMax, *sQ = sbuf + 3 * kTileMax;
  __shared__ double sred[2][4];
  const int n = counts[0];
  for (int it = counts[7] + blockIdx.x; it < n; it += gridDim.x) {
    const int2 w = items[it];
    const RepDesc *__restrict__ Rp = reps + w.x;
    long long *__restrict__ ctl = Rp->ctl;
    if (!ctl[kCtlActive]) continue;
    if ((Rp->P & 7) == 0 && !Rp->ffma) {
      // tensor-core path: tiles with padded rows in sF (forces), sX
      // (deviations), sV (velocities)
      const int P = Rp->P, A = Rp->A, N = Rp->N, PS = P + 4;
      const int tile0 = w.y * A;
      const int na = min(A, N - tile0);
      const int len = na * 3 * P;
      const size_t base = (size_t)tile0 * 3 * P;
      float *mF = sbuf, *mX = sbuf + kMmaTile, *mV = sbuf + 2 * kMmaTile;
      {
        // rows over warps, beads over lanes (coalesced, no division)
        const float *__restrict__ gF = Rp->F + base;
        const float *__restrict__ gX = Rp->d + base;
        const float *__restrict__ gV = Rp->vk + base;
        const int rows = na * 3;
        for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5)
          for (int j = threadIdx.x & 31; j < P; j += 32) {
            mF[r * PS + j] = __ldg(gF + r * P + j);
            mX[r * PS + j] = __ldg(gX + r * P + j);
            mV[r * PS + j] = __ldg(gV + r * P + j);
          }
      }
      __syncthreads();
      bstep_mma(Rp, P, tile0, na, base, mF, mX, mV, (uint64_t)ctl[kCtlStep], (int)ctl[kCtlFirst]);
      // skin check on the new deviations (mF) and the new centroids
      double vdisp = 0.0;
      float vdevf = 0.f;
      // oxygens only: atoms i = 3 m of the tile, warps over atoms, lanes over beads
      for (int al = (3 - tile0 % 3) % 3 + (threadIdx.x >> 5) * 3; al < na; al += 3 * (blockDim.x >> 5))
        for (int k = threadIdx.x & 31; k < P; k += 32) {
        const int i = tile0 + al;
        const float *ds = mF + al * 3 * PS;
        const float e0 = ds[k], e1 = ds[PS + k], e2 = ds[2 * PS + k];
        vdevf = fmaxf(vdevf, e0 * e0 + e1 * e1 + e2 * e2);
        {
          float *po = Rp->pO + (size_t)i * P + k;
          po[0] = Rp->xcw[3 * (size_t)i] + e0;
          po[P] = Rp->xcw[3 * (size_t)i + 1] + e1;
          po[2 * P] = Rp->xcw[3 * (size_t)i + 2] + e2;
        }
        if (k == 0) {
          const int m = i / 3;
          const double c0 = Rp->xc[3 * (size_t)i], c1 = Rp->xc[3 * (size_t)i + 1], c2 = Rp->xc[3 * (size_t)i + 2];
          const double g0 = c0 - Rp->cref[3 * m], g1 = c1 - Rp->cref[3 * m + 1], g2 = c2 - Rp->cref[3 * m + 2];
          vdisp = fmax(vdisp, g0 * g0 + g1 * g1 + g2 * g2);
          Rp->ccur[3 * m] = c0;
          Rp->ccur[3 * m + 1] = c1;
          Rp->ccur[3 * m + 2] = c2;
        }
      }
      float vdispf = (float)vdisp;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        vdispf = fmaxf(vdispf, __shfl_down_sync(0xffffffffu, vdispf, o));
        vdevf = fmaxf(vdevf, __shfl_down_sync(0xffffffffu, vdevf, o));
      }
      if ((threadIdx.x & 31) == 0) {
        sred[0][threadIdx.x >> 5] = vdispf;
        sred[1][threadIdx.x >> 5] = vdevf;
      }
      __syncthreads();
      if (threadIdx.x < 2) {
        float mx = 0.f;
        bool nan = false;
        for (int ww = 0; ww < (int)((blockDim.x + 31) / 32); ++ww) {
          mx = fmaxf(mx, (float)sred[threadIdx.x][ww]);
          nan |= sred[threadIdx.x][ww] != sred[threadIdx.x][ww];
        }
        skin_max(Rp->ctl, threadIdx.x, nan ? __int_as_float(0x7fc00000) : mx);
      }
      __syncthreads();
      continue;
    }
    const int P = Rp->P, A = Rp->A, N = Rp->N, integ = Rp->integrator, thermo = Rp->thermo;
    const int lg = (P & (P - 1)) == 0 ? __ffs(P) - 1 : -1;
    const uint64_t seed = Rp->seed;
    const float *__restrict__ Mtf = Rp->Mtf;
    const float *__restrict__ Mf = Rp->Mf;
    const float *__restrict__ cAf = Rp->cAf;
    const float *__restrict__ sAf = Rp->sAf;
    const float *__restrict__ wsAf = Rp->wsAf;
    const float *__restrict__ c1f = Rp->c1f;
    const float *__restrict__ c2f = Rp->c2f;
    const double *__restrict__ inv_mm = Rp->inv_mm;
    const double *__restrict__ sigv = Rp->sigv;
    float *__restrict__ dg = Rp->d;
    float *__restrict__ vkg = Rp->vk;
    const float *__restrict__ Fg = Rp->F;
    double *__restrict__ xcg = Rp->xc;
    double *__restrict__ v0g = Rp->v0;
    float *__restrict__ xcw = Rp->xcw;
    const double dt = Rp->dt, tA = Rp->tA, c1_0 = Rp->c1_0, c2_0 = Rp->c2_0;
    const int tile0 = w.y * A;
    const int na = min(A, N - tile0);
    const int len = na * 3 * P;
    const size_t base = (size_t)tile0 * 3 * P;
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
      sD[t] = dg[base + t];
      sV[t] = vkg[base + t];
      sF[t] = Fg[base + t];
    }
    __syncthreads();
    const uint64_t step = (uint64_t)ctl[kCtlStep];
    const int first = (int)ctl[kCtlFirst];
    const float hd = (float)dt, half = 0.5f * hd;
    const float kick = first ? half : hd;
    {
    for (int task = threadIdx.x; task < len; task += blockDim.x) {
      const int k = lg >= 0 ? (task & (P - 1)) : task % P;
      const int r = lg >= 0 ? (task >> lg) : task / P;
      const int c = r % 3;
      const int i = tile0 + r / 3;
      const float *fx = sF + r * P;
      const float *xx = sD + r * P;
      float fa = 0.f, fb = 0.f, qa = 0.f, qb = 0.f;
      const float *mcol = Mtf + k;
      int j = 0;
#pragma unroll 4
      for (; j + 1 < P; j += 2) {
        const float m0 = __ldg(mcol + j * P), m1 = __ldg(mcol + (j + 1) * P);
        fa = fmaf(m0, fx[j], fa);
        fb = fmaf(m1, fx[j + 1], fb);
        qa = fmaf(m0, xx[j], qa);
        qb = fmaf(m1, xx[j + 1], qb);
      }
      if (j < P) {
        const float m0 = __ldg(mcol + j * P);
        fa = fmaf(m0, fx[j], fa);
        qa = fmaf(m0, xx[j], qa);
      }
      const float f = fa + fb;
      if (k == 0) {
        sQ[task] = f;
        continue;
      }
      float q = qa + qb;
      float v = sV[task];
      const float im = (float)__ldg(inv_mm + i);
      const float cA = __ldg(cAf + k), sA = __ldg(sAf + k), wsA = __ldg(wsAf + k);
      const float c1 = __ldg(c1f + k), c2s = __ldg(c2f + k) * (float)__ldg(sigv + i);
      if (integ == 0) {
        v = fmaf(kick * im, f, v);
        rotb(q, v, cA, sA, wsA);
        if (thermo) v = fmaf(c1, v, c2s * gauss1f_b(seed, (uint32_t)i, (uint32_t)k, kStreamO1, step, c));
        rotb(q, v, cA, sA, wsA);
      } else {
        const float kb = half * im;
        if (!first) {
          v = fmaf(kb, f, v);
          if (thermo) v = fmaf(c1, v, c2s * gauss1f_b(seed, (uint32_t)i, (uint32_t)k, kStreamO2, step - 1, c));
        }
        if (thermo) v = fmaf(c1, v, c2s * gauss1f_b(seed, (uint32_t)i, (uint32_t)k, kStreamO1, step, c));
        v = fmaf(kb, f, v);
        rotb(q, v, cA, sA, wsA);
      }
      sQ[task] = q;
      vkg[base + task] = v;
    }
    __syncthreads();
    const double rsp = rsqrt((double)P);
    for (int t = threadIdx.x; t < na * 3; t += blockDim.x) {
      const int al = t / 3, c = t % 3;
      const int i = tile0 + al;
      const size_t ic = (size_t)i * 3 + c;
      const double f0 = (double)sQ[t * P];
      double x = xcg[ic], v = v0g[ic];
      const double im = __ldg(inv_mm + i);
      const double dr = tA * rsp;
      const double c2s = c2_0 * __ldg(sigv + i);
      if (integ == 0) {
        v = fma((first ? 0.5 : 1.0) * dt * im, f0, v);
        x = fma(dr, v, x);
        if (thermo) v = fma(c1_0, v, c2s * (double)gauss1f_b(seed, (uint32_t)i, 0u, kStreamO1, step, c));
        x = fma(dr, v, x);
      } else {
        const double kb = 0.5 * dt * im;
        if (!first) {
          v = fma(kb, f0, v);
          if (thermo) v = fma(c1_0, v, c2s * (double)gauss1f_b(seed, (uint32_t)i, 0u, kStreamO2, step - 1, c));
        }
        if (thermo) v = fma(c1_0, v, c2s * (double)gauss1f_b(seed, (uint32_t)i, 0u, kStreamO1, step, c));
        v = fma(kb, f0, v);
        x = fma(dr, v, x);
      }
      xcg[ic] = x;
      v0g[ic] = v;
      xcw[ic] = wrapb(x, Rp->box[c], Rp->invbox[c]);
      sQ[t * P] = 0.f;
    }
    __syncthreads();
    for (int task = threadIdx.x; task < len; task += blockDim.x) {
      const int jj = lg >= 0 ? (task & (P - 1)) : task % P;
      const int row = lg >= 0 ? (task >> lg) : task / P;
      const float *qq = sQ + row * P;
      const float *mrow = Mf + jj;
      float xa = 0.f, xb = 0.f;
      int k = 1;
#pragma unroll 4
      for (; k + 1 < P; k += 2) {
        xa = fmaf(__ldg(mrow + k * P), qq[k], xa);
        xb = fmaf(__ldg(mrow + (k + 1) * P), qq[k + 1], xb);
      }
      if (k < P) xa = fmaf(__ldg(mrow + k * P), qq[k], xa);
      const float dn = xa + xb;
      dg[base + task] = dn;
      sD[task] = dn;
    }
    }  // generic P
    __syncthreads();
    double vdisp = 0.0;
    float vdevf = 0.f;
    const double *__restrict__ cref = Rp->cref;
    double *__restrict__ ccur = Rp->ccur;
    for (int t = threadIdx.x; t < na * P; t += blockDim.x) {
      const int al = lg >= 0 ? (t >> lg) : t / P;
      const int k = lg >= 0 ? (t & (P - 1)) : t % P;
      const int i = tile0 + al;
      if (i % 3) continue;
      const float *ds = sD + al * 3 * P;
      const float e0 = ds[k], e1 = ds[P + k], e2 = ds[2 * P + k];
      vdevf = fmaxf(vdevf, e0 * e0 + e1 * e1 + e2 * e2);
      {
        float *po = Rp->pO + (size_t)i * P + k;
        po[0] = xcw[3 * (size_t)i] + e0;
        po[P] = xcw[3 * (size_t)i + 1] + e1;
        po[2 * P] = xcw[3 * (size_t)i + 2] + e2;
      }
      if (k == 0) {
        const int m = i / 3;
        const double c0 = xcg[3 * (size_t)i], c1 = xcg[3 * (size_t)i + 1], c2 = xcg[3 * (size_t)i + 2];
        const double g0 = c0 - cref[3 * m], g1 = c1 - cref[3 * m + 1], g2 = c2 - cref[3 * m + 2];
        vdisp = fmax(vdisp, g0 * g0 + g1 * g1 + g2 * g2);
        ccur[3 * m] = c0;
        ccur[3 * m + 1] = c1;
        ccur[3 * m + 2] = c2;
      }
    }
    float vdispf = (float)vdisp;   // squared drifts: FP32 is ample for a rebuild criterion
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vdispf = fmaxf(vdispf, __shfl_down_sync(0xffffffffu, vdispf, o));
      vdevf = fmaxf(vdevf, __shfl_down_sync(0xffffffffu, vdevf, o));
    }
    if ((threadIdx.x & 31) == 0) {
      sred[0][threadIdx.x >> 5] = vdispf;
      sred[1][threadIdx.x >> 5] = vdevf;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      float mx = 0.f;
      bool nan = false;
      for (int ww = 0; ww < (int)((blockDim.x + 31) / 32); ++ww) {
        mx = fmaxf(mx, (float)sred[threadIdx.x][ww]);
        nan |= sred[threadIdx.x][ww] != sred[threadIdx.x][ww];
      }
      skin_max(Rp->ctl, threadIdx.x, nan ? __int_as_float(0x7fc00000) : mx);
    }
    __syncthreads();
  }
}

// Closing B(h/2) (O(h/2) for OBABO) of the replicas that stepped since their
// last closing kick, over step items.
__global__ void __launch_bounds__(128) k_bclose(const RepDesc *reps, const int2 *items, const int *count) {
  __shared__ float sF[kTileMax];
  const int n = *count;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int2 w = items[it];
    const RepDesc &R = reps[w.x];
    if (!R.ctl[kCtlClose]) continue;
    const int P = R.P, A = R.A;
    const int item0 = w.y * A;
    const int nitem = min(A, R.N - item0);
    // the item's atoms in sub-tiles that fit the shared tile (a 128-bead
    // warp item spans twice kTileMax)
    const int sub = max(1, kTileMax / (3 * P));
    for (int a0 = 0; a0 < nitem; a0 += sub) {
    const int tile0 = item0 + a0;
    const int na = min(sub, nitem - a0);
    const int len = na * 3 * P;
    const size_t base = (size_t)tile0 * 3 * P;
    for (int t = threadIdx.x; t < len; t += blockDim.x) sF[t] = R.F[base + t];
    __syncthreads();
    const uint64_t step = (uint64_t)R.ctl[kCtlStep] - 1;
    for (int task = threadIdx.x; task < len; task += blockDim.x) {
      const int k = task % P;
      const int r = task / P;
      const int c = r % 3;
      const int i = tile0 + r / 3;
      const float *fx = sF + r * P;
      float fa = 0.f, fb = 0.f;
      int j = 0;
      for (; j + 1 < P; j += 2) {
        fa = fmaf(__ldg(R.Mtf + j * P + k), fx[j], fa);
        fb = fmaf(__ldg(R.Mtf + (j + 1) * P + k), fx[j + 1], fb);
      }
      if (j < P) fa = fmaf(__ldg(R.Mtf + j * P + k), fx[j], fa);
      const float f = fa + fb;
      if (k == 0) {
        const size_t ic = (size_t)i * 3 + c;
        double v = fma(0.5 * R.dt * __ldg(R.inv_mm + i), (double)f, R.v0[ic]);
        if (R.integrator == 1 && R.thermo)
          v = fma(R.c1_0, v, R.c2_0 * __ldg(R.sigv + i) *
                                 (double)gauss1f_b(R.seed, (uint32_t)i, 0u, kStreamO2, step, c));
        R.v0[ic] = v;
        continue;
      }
      float v = fmaf(0.5f * (float)R.dt * (float)__ldg(R.inv_mm + i), f, R.vk[base + task]);
      if (R.integrator == 1 && R.thermo) {
        const float c1 = __ldg(R.c1f + k), c2s = __ldg(R.c2f + k) * (float)__ldg(R.sigv + i);
        v = fmaf(c1, v, c2s * gauss1f_b(R.seed, (uint32_t)i, (uint32_t)k, kStreamO2, step, c));
      }
      R.vk[base + task] = v;
    }
    __syncthreads();
    }
  }
}

// Rebuild decision of this step, one thread per neighbour item (replica,
// block of kNbrMolPerItem molecules): the replica's skin maxima of the step,
// with margins for FP32 rounding of the deviations and squared drifts (NaN or
// infinity forces a rebuild), against the skin; the items of the replicas
// that rebuild are appended to the list go (order immaterial: an item's list
// does not depend on who builds it).
__global__ void k_bdecide(const RepDesc *reps, const int2 *items, const int *count, int2 *go, int *ngo) {
  const int n = *count;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
    const int2 w = items[it];
    const RepDesc &R = reps[w.x];
    if (!R.ctl[kCtlActive]) continue;
    const unsigned *sk = reinterpret_cast<const unsigned *>(R.ctl + kCtlSkin);
    double lim[2];
    for (int q = 0; q < 2; ++q) {
      const float v2 = __uint_as_float(sk[q]);
      lim[q] = (v2 == v2 && v2 <= 3.0e38f) ? sqrt((double)v2) * (1.0 + 1e-6) + 1e-4 : 1e300;
    }
    if (2.0 * lim[0] + 2.0 * lim[1] > R.skin) go[atomicAdd(ngo, 1)] = w;
  }
}

// Neighbour lists of the listed items (replica, block of kNbrMolPerItem
// molecules), rebuilt unconditionally: the items of the replicas k_bdecide
// chose, or every item of a new replica.
__global__ void k_bnbr(const RepDesc *reps, const int2 *items, const int *count) {
  const int n = *count;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int2 w = items[it];
    const RepDesc &R = reps[w.x];
    if (threadIdx.x == 0 && w.y == 0) R.ctl[kCtlRebuilds] += 1;
    {
      // the replica's oxygen centroids (wrapped, FP32) into shared memory
      extern __shared__ float s_cw[];
#pragma unroll 4
      for (int t = threadIdx.x; t < 3 * R.nmol; t += blockDim.x) s_cw[t] = R.xcw[9 * (t / 3) + t % 3];
      __syncthreads();
      // One warp per molecule of this item's 8: the warp walks the buckets
      // b = 0..NS-1 (neighbours j = b mod NS, increasing j), 32 candidates per
      // ballot, and compacts the hits in order.  Candidates are tested in FP32
      // on the wrapped centroids within rc + skin + 1e-3 A (FP32 rounding of
      // the centroids is ~1e-5 A); extra far candidates add nothing to any
      // force.
      const int NS = kLJWarps * R.G;
      const float *cw = s_cw;
      const float L0 = (float)R.box[0], L1 = (float)R.box[1], L2 = (float)R.box[2];
      const float i0 = (float)R.invbox[0], i1 = (float)R.invbox[1], i2 = (float)R.invbox[2];
      const float rl = (float)(R.rlist + 1e-3);
      const float rl2 = rl * rl;
      const int lane = threadIdx.x & 31;
      const int nmol = R.nmol;
      for (int mm = threadIdx.x >> 5; mm < kNbrMolPerItem; mm += blockDim.x >> 5) {
        const int m = w.y * kNbrMolPerItem + mm;
        if (m >= nmol) break;
        const float c0 = cw[3 * m], c1 = cw[3 * m + 1], c2 = cw[3 * m + 2];
        int *off = R.nbr_off + (size_t)m * (NS + 1);
        int *nl = R.nbr + (size_t)m * kMaxNeighbours;
        int total = 0;
        auto near = [&](int j) {
          const float d0 = micb(cw[3 * j] - c0, L0, i0);
          const float d1 = micb(cw[3 * j + 1] - c1, L1, i1);
          const float d2 = micb(cw[3 * j + 2] - c2, L2, i2);
          return d0 * d0 + d1 * d1 + d2 * d2 < rl2;
        };
        const int n0 = (nmol + NS - 1) / NS;   // candidates of bucket 0, the longest
        if (n0 <= 16) {
          // short buckets: 32 / seg consecutive buckets per ballot, seg lanes
          // each in bucket order, so the lane prefix count is the list order
          int seg = 1;
          while (seg < n0) seg <<= 1;
          const int kb = 32 / seg;
          const int sg = lane / seg, tl = lane - sg * seg;
          for (int b = 0; b < NS; b += kb) {
            const int bb = b + sg, j = bb + tl * NS;
            const bool hit = bb < NS && j < nmol && j != m && near(j);
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            const int pos = total + __popc(mask & ((1u << lane) - 1u));
            if (tl == 0 && bb < NS) off[bb] = pos;
            if (hit && pos < kMaxNeighbours) nl[pos] = j;
            total += __popc(mask);
          }
        } else {
          for (int b = 0; b < NS; ++b) {
            if (lane == 0) off[b] = total;
            for (int j0 = b; j0 < nmol; j0 += 32 * NS) {
              const int j = j0 + lane * NS;
              const bool hit = j < nmol && j != m && near(j);
              const unsigned mask = __ballot_sync(0xffffffffu, hit);
              const int pos = total + __popc(mask & ((1u << lane) - 1u));
              if (hit && pos < kMaxNeighbours) nl[pos] = j;
              total += __popc(mask);
            }
          }
        }
        if (lane == 0) {
          if (total > kMaxNeighbours) {
            // leave an empty list and report: the forces are incomplete
            atomicOr((unsigned long long *)&R.ctl[kCtlWords - 1], (unsigned long long)kErrNbrOverflow);
            for (int b = 0; b <= NS; ++b) off[b] = 0;
          } else {
            off[NS] = total;
            R.cref[3 * m] = R.ccur[3 * m];
            R.cref[3 * m + 1] = R.ccur[3 * m + 1];
            R.cref[3 * m + 2] = R.ccur[3 * m + 2];
          }
        }
      }
    }
    __syncthreads();
  }
}

// Water-like forces in FP32, one warp per work item (replica, first
// molecule, bead chunk): lane = (group u, bead kl) with Bk = min(P, 32) beads
// per group and G = 32 / Bk molecules per warp (m = first + u), so every
// lane is busy whatever P is.  Each lane evaluates its molecule-bead's two
// bonds, the angle and the O-O Lennard-Jones sum over the whole neighbour
// list, and writes the three atoms' forces and its U / Tr Xi row entries:
// no cross-lane reduction.  The list is grouped by j mod NS and index-ordered
// within a group, so the summation order depends only on the interacting
// pairs (far candidates add nothing): alone-vs-mix and rebuild invariant.
// One work item of k_bforce; PT > 0 fixes the bead count at compile time
// (constant strides and lane split), PT = 0 reads it from the descriptor.
template <int PT>
__device__ __forceinline__ void bforce_item(const RepDesc &R, const int4 w, int lane) {
  {
    const int P = PT > 0 ? PT : R.P;
    const float *__restrict__ dg = R.d;
    const float *__restrict__ xcw = R.xcw;
    const int Bk = P < 32 ? P : 32;
    const int G = 32 / Bk;
    const int u = lane / Bk, kl = lane % Bk;
    const int pos = w.y + u;
    const int k = w.z * Bk + kl;
    if (u >= G || pos >= R.nmol || k >= P) return;
    const int m = __ldg(R.mperm + pos);
    const int o = 3 * m;
    const float L0 = R.boxf[0], L1 = R.boxf[1], L2 = R.boxf[2];
    const float i0 = R.invboxf[0], i1 = R.invboxf[1], i2 = R.invboxf[2];
    const size_t so = (size_t)o * 3 * P + k;
    const float co0 = R.xcw[3 * o], co1 = R.xcw[3 * o + 1], co2 = R.xcw[3 * o + 2];
    const float do0 = R.d[so], do1 = R.d[so + P], do2 = R.d[so + 2 * P];
    float fO[3] = {0.f, 0.f, 0.f}, fH[2][3];
    float dv[2][3], r[2], ir[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int hh = o + 1 + h;
      const size_t sh = (size_t)hh * 3 * P + k;
      dv[h][0] = micb(R.xcw[3 * hh] - co0, L0, i0) + (R.d[sh] - do0);
      dv[h][1] = micb(R.xcw[3 * hh + 1] - co1, L1, i1) + (R.d[sh + P] - do1);
      dv[h][2] = micb(R.xcw[3 * hh + 2] - co2, L2, i2) + (R.d[sh + 2 * P] - do2);
      r[h] = sqrtf(dv[h][0] * dv[h][0] + dv[h][1] * dv[h][1] + dv[h][2] * dv[h][2]);
      ir[h] = 1.f / r[h];
    }
    // bonds: U = 1/2 kb (r - r0)^2
    float ub = 0.f, wb = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float dr = r[h] - R.r0f;
      ub = fmaf(0.5f * R.kbf * dr, dr, ub);
      const float g = -R.kbf * dr * ir[h];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fH[h][c] = g * dv[h][c];
        wb = fmaf(dv[h][c], fH[h][c], wb);
      }
    }
    // angle: U = 1/2 kth (theta - th0)^2
    {
      const float ir01 = ir[0] * ir[1];
      const float dot = dv[0][0] * dv[1][0] + dv[0][1] * dv[1][1] + dv[0][2] * dv[1][2];
      const float cth = fminf(1.f, fmaxf(-1.f, dot * ir01));
      const float th = acosf(cth);
      const float dth = th - R.th0f;
      const float pref = R.kthf * dth / sinf(th);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int g = 1 - h;
        const float ch = cth * ir[h] * ir[h];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float fa = pref * fmaf(dv[g][c], ir01, -ch * dv[h][c]);
          fH[h][c] += fa;
          wb = fmaf(dv[h][c], fa, wb);
        }
      }
      ub = fmaf(0.5f * R.kthf * dth, dth, ub);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) fO[c] = -(fH[0][c] + fH[1][c]);
    // O-O Lennard-Jones over the whole list
    const int NS = kLJWarps * R.G;
    const int *off = R.nbr_off + (size_t)m * (NS + 1);
    const int q1 = __ldg(off + NS);
    const int *__restrict__ nl = R.nbr + (size_t)m * kMaxNeighbours;
    const float rc2 = R.rc2f, sig2 = R.sig2f, e4 = R.e4f, e24 = R.e24f, e48 = 2.0f * R.e24f;
    const float *__restrict__ pO = R.pO;
    const size_t sm = (size_t)m * 3 * P + k;
    const float po0 = pO[sm], po1 = pO[sm + P], po2 = pO[sm + 2 * P];
    float ulj = 0.f, wlj = 0.f;
    // per-bead minimum image of the oxygen bead positions
#pragma unroll 4
    for (int q = __ldg(off); q < q1; ++q) {
      const int j = __ldg(nl + q);
      const size_t sj = (size_t)j * 3 * P + k;
      const float d0 = micb(__ldg(pO + sj) - po0, L0, i0);
      const float d1 = micb(__ldg(pO + sj + P) - po1, L1, i1);
      const float d2 = micb(__ldg(pO + sj + 2 * P) - po2, L2, i2);
      const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (r2 < rc2) {
        // 4 eps (s^12 - s^6) = s6 (e4 s6 - e4); f r = 24 eps (2 s^12 - s^6) / r^2 = s6 (e48 s6 - e24) / r^2
        const float inv = __fdividef(1.0f, r2);
        const float s2 = sig2 * inv;
        const float s6 = s2 * s2 * s2;
        ulj = fmaf(s6, fmaf(e4, s6, -e4), ulj);
        const float fr = fmaf(e48, s6, -e24) * s6 * inv;
        fO[0] = fmaf(-fr, d0, fO[0]);
        fO[1] = fmaf(-fr, d1, fO[1]);
        fO[2] = fmaf(-fr, d2, fO[2]);
        wlj = fmaf(fr, r2, wlj);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R.F[so + c * P] = fO[c];
      R.F[so + 3 * P + c * P] = fH[0][c];
      R.F[so + 6 * P + c * P] = fH[1][c];
    }
    R.Upart[(size_t)m * P + k] = (double)fmaf(0.5f, ulj, ub);
    R.Wpart[(size_t)m * P + k] = (double)fmaf(0.5f, wlj, wb);
  }
}

// Bonded terms (two O-H bonds, the H-O-H angle) of molecule m at bead k:
// forces on O and the two H, and the bead's bonded energy and virial.  Same
// arithmetic as the scalar item above.
__device__ __forceinline__ void bonded_bead(const RepDesc &R, int P, int m, int k, float (&fO)[3],
                                            float (&fH)[2][3], float &ub, float &wb) {
  const int o = 3 * m;
  const float L0 = R.boxf[0], L1 = R.boxf[1], L2 = R.boxf[2];
  const float i0 = R.invboxf[0], i1 = R.invboxf[1], i2 = R.invboxf[2];
  const size_t so = (size_t)o * 3 * P + k;
  const float co0 = R.xcw[3 * o], co1 = R.xcw[3 * o + 1], co2 = R.xcw[3 * o + 2];
  const float do0 = R.d[so], do1 = R.d[so + P], do2 = R.d[so + 2 * P];
  float dv[2][3], r[2], ir[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int hh = o + 1 + h;
    const size_t sh = (size_t)hh * 3 * P + k;
    dv[h][0] = micb(R.xcw[3 * hh] - co0, L0, i0) + (R.d[sh] - do0);
    dv[h][1] = micb(R.xcw[3 * hh + 1] - co1, L1, i1) + (R.d[sh + P] - do1);
    dv[h][2] = micb(R.xcw[3 * hh + 2] - co2, L2, i2) + (R.d[sh + 2 * P] - do2);
    r[h] = sqrtf(dv[h][0] * dv[h][0] + dv[h][1] * dv[h][1] + dv[h][2] * dv[h][2]);
    ir[h] = 1.f / r[h];
  }
  ub = 0.f;
  wb = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float dr = r[h] - R.r0f;
    ub = fmaf(0.5f * R.kbf * dr, dr, ub);
    const float g = -R.kbf * dr * ir[h];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fH[h][c] = g * dv[h][c];
      wb = fmaf(dv[h][c], fH[h][c], wb);
    }
  }
  {
    const float ir01 = ir[0] * ir[1];
    const float dot = dv[0][0] * dv[1][0] + dv[0][1] * dv[1][1] + dv[0][2] * dv[1][2];
    const float cth = fminf(1.f, fmaxf(-1.f, dot * ir01));
    const float th = acosf(cth);
    const float dth = th - R.th0f;
    const float pref = R.kthf * dth / sinf(th);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 1 - h;
      const float ch = cth * ir[h] * ir[h];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float fa = pref * fmaf(dv[g][c], ir01, -ch * dv[h][c]);
        fH[h][c] += fa;
        wb = fmaf(dv[h][c], fa, wb);
      }
    }
    ub = fmaf(0.5f * R.kthf * dth, dth, ub);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) fO[c] = -(fH[0][c] + fH[1][c]);
}

__device__ __forceinline__ float2 ldg2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }

// Minimum image of a pair of components: d - L rint(d / L), elementwise.
__device__ __forceinline__ float2 micb2(float2 d, float2 invL, float2 nL) {
  float2 t = __fmul2_rn(d, invL);
  t.x = rintf(t.x);
  t.y = rintf(t.y);
  return __ffma2_rn(t, nL, d);
}

// The work item of k_bforce for an even bead count, two adjacent beads
// (k, k + 1) per lane: lane = (group u, bead pair kl) with Bk = min(P, 64)
// beads per group and G = 32 / (Bk / 2) molecules per warp.  The pair loop
// runs on packed FP32 pairs (Blackwell's two-wide FP32 add, multiply and
// fused multiply-add), each element rounded exactly as the scalar item
// rounds it, so the forces, energies and virials are the scalar item's; a
// bead of the pair outside the cutoff adds exact zeros.  The neighbour
// index and the list bounds serve both beads.
template <int PT>
__device__ __forceinline__ void bforce_item2(const RepDesc &R, const int4 w, int lane) {
  const int P = PT > 0 ? PT : R.P;
  const int Bk = P < 64 ? P : 64;
  const int Lg = Bk >> 1;
  const int G = 32 / Lg;
  const int u = lane / Lg, kl = lane - u * Lg;
  const int pos = w.y + u;
  const int k = w.z * Bk + 2 * kl;
  if (u >= G || pos >= R.nmol || k >= P) return;
  const int m = __ldg(R.mperm + pos);
  float fO[2][3], fH[2][2][3], ub[2], wb[2];
  bonded_bead(R, P, m, k, fO[0], fH[0], ub[0], wb[0]);
  bonded_bead(R, P, m, k + 1, fO[1], fH[1], ub[1], wb[1]);
  const float2 iL0 = make_float2(R.invboxf[0], R.invboxf[0]), nL0 = make_float2(-R.boxf[0], -R.boxf[0]);
  const float2 iL1 = make_float2(R.invboxf[1], R.invboxf[1]), nL1 = make_float2(-R.boxf[1], -R.boxf[1]);
  const float2 iL2 = make_float2(R.invboxf[2], R.invboxf[2]), nL2 = make_float2(-R.boxf[2], -R.boxf[2]);
  const int NS = kLJWarps * R.G;
  const int *off = R.nbr_off + (size_t)m * (NS + 1);
  const int q1 = __ldg(off + NS);
  const int *__restrict__ nl = R.nbr + (size_t)m * kMaxNeighbours;
  const float rc2 = R.rc2f;
  const float2 sig2 = make_float2(R.sig2f, R.sig2f), e4 = make_float2(R.e4f, R.e4f);
  const float2 ne4 = make_float2(-R.e4f, -R.e4f), ne24 = make_float2(-R.e24f, -R.e24f);
  const float2 e48 = make_float2(2.0f * R.e24f, 2.0f * R.e24f);
  const float *__restrict__ pO = R.pO;
  const float *__restrict__ pm = pO + (size_t)m * 3 * P + k;
  const float2 p0 = ldg2(pm), p1 = ldg2(pm + P), p2 = ldg2(pm + 2 * P);
  const float2 np0 = make_float2(-p0.x, -p0.y), np1 = make_float2(-p1.x, -p1.y), np2 = make_float2(-p2.x, -p2.y);
  float2 f0 = make_float2(fO[0][0], fO[1][0]), f1 = make_float2(fO[0][1], fO[1][1]);
  float2 f2 = make_float2(fO[0][2], fO[1][2]);
  float2 ulj = make_float2(0.f, 0.f), wlj = make_float2(0.f, 0.f);
  // one candidate: the pair's minimum-image separation for both beads and,
  // inside the cutoff, the Lennard-Jones force, energy and virial
  auto pair = [&](float2 a0, float2 a1, float2 a2) {
    const float2 d0 = micb2(__fadd2_rn(a0, np0), iL0, nL0);
    const float2 d1 = micb2(__fadd2_rn(a1, np1), iL1, nL1);
    const float2 d2 = micb2(__fadd2_rn(a2, np2), iL2, nL2);
    const float2 r2 = __ffma2_rn(d2, d2, __ffma2_rn(d1, d1, __fmul2_rn(d0, d0)));
    const bool in0 = r2.x < rc2, in1 = r2.y < rc2;
    if (in0 || in1) {
      // a bead outside the cutoff gets 1/r^2 = 0: every term it adds is an exact zero
      const float2 inv = make_float2(in0 ? __fdividef(1.0f, r2.x) : 0.f, in1 ? __fdividef(1.0f, r2.y) : 0.f);
      const float2 s2 = __fmul2_rn(sig2, inv);
      const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
      ulj = __ffma2_rn(s6, __ffma2_rn(e4, s6, ne4), ulj);
      const float2 fr = __fmul2_rn(__fmul2_rn(__ffma2_rn(e48, s6, ne24), s6), inv);
      const float2 nfr = make_float2(-fr.x, -fr.y);
      f0 = __ffma2_rn(nfr, d0, f0);
      f1 = __ffma2_rn(nfr, d1, f1);
      f2 = __ffma2_rn(nfr, d2, f2);
      wlj = __ffma2_rn(fr, r2, wlj);
    }
  };
  // four candidates per round: their indices, then their twelve rows, are
  // requested before any arithmetic, so the gathers overlap; the candidates
  // are then summed in list order
  int q = __ldg(off);
  for (; q + 4 <= q1; q += 4) {
    int jj[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) jj[v] = __ldg(nl + q + v);
    float2 a[4][3];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float *__restrict__ pj = pO + (size_t)jj[v] * 3 * P + k;
      a[v][0] = ldg2(pj);
      a[v][1] = ldg2(pj + P);
      a[v][2] = ldg2(pj + 2 * P);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) pair(a[v][0], a[v][1], a[v][2]);
  }
  for (; q < q1; ++q) {
    const float *__restrict__ pj = pO + (size_t)__ldg(nl + q) * 3 * P + k;
    pair(ldg2(pj), ldg2(pj + P), ldg2(pj + 2 * P));
  }
  const size_t so = (size_t)(3 * m) * 3 * P + k;
  float *__restrict__ F = R.F;
  const float2 fo[3] = {f0, f1, f2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    *reinterpret_cast<float2 *>(F + so + c * P) = fo[c];
    *reinterpret_cast<float2 *>(F + so + 3 * P + c * P) = make_float2(fH[0][0][c], fH[1][0][c]);
    *reinterpret_cast<float2 *>(F + so + 6 * P + c * P) = make_float2(fH[0][1][c], fH[1][1][c]);
  }
  double *up = R.Upart + (size_t)m * P + k, *wp = R.Wpart + (size_t)m * P + k;
  up[0] = (double)fmaf(0.5f, ulj.x, ub[0]);
  up[1] = (double)fmaf(0.5f, ulj.y, ub[1]);
  wp[0] = (double)fmaf(0.5f, wlj.x, wb[0]);
  wp[1] = (double)fmaf(0.5f, wlj.y, wb[1]);
}

__global__ void __launch_bounds__(128, 6) k_bforce(const RepDesc *__restrict__ reps, const int4 *__restrict__ items,
                                                const int *__restrict__ count, int force_all) {
  const int n = *count;
  const int lane = threadIdx.x & 31;
  // the warps of a block take consecutive items (molecules in
  // space-filling-curve order, so they share neighbour rows in L1)
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int it = gw; it < n; it += nw) {
    const int4 w = items[it];
    const RepDesc *__restrict__ Rp = reps + w.x;
    if (!force_all && !Rp->ctl[kCtlActive]) continue;
    switch (Rp->P) {
      case 8: bforce_item2<8>(*Rp, w, lane); break;
      case 16: bforce_item2<16>(*Rp, w, lane); break;
      case 32: bforce_item2<32>(*Rp, w, lane); break;
      case 64: bforce_item2<64>(*Rp, w, lane); break;
      default:
        if (Rp->P & 1)
          bforce_item<0>(*Rp, w, lane);
        else
          bforce_item2<0>(*Rp, w, lane);
        break;
    }
  }
}

// Estimators, pass 1: work items (replica, e-block); e-block b walks the
// replica's tiles b, b + ne, ... (x = xc + d in FP64; q~_k = (M d)_k and the
// bead mean of d in FP32 from the FP32 deviations, relative error ~P 2^-24;
// r - r_c = d - mean_j d_j); products and sums in FP64.
__global__ void __launch_bounds__(128) k_best(const RepDesc *reps, const int2 *items, const int *count) {
  __shared__ CSum sK[128], sS[128];
  __shared__ CSum sred[3][4];
  __shared__ float sDv[3 * 128];   // the tile's deviation rows (A atoms x 3 x P <= 384)
  const int n = *count;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int2 w = items[it];
    const RepDesc &R = reps[w.x];
    const int P = R.P, N = R.N;
    const int A = P >= 128 ? 1 : 128 / P;       // estimator tile: A P <= 128 tasks
    const int ntiles = (N + A - 1) / A;
    const int ntask = A * P;
    // per thread a handful of tiles (plain FP64 sums: a few tens of terms);
    // every combination across threads and blocks below is compensated
    double kk = 0.0, ss = 0.0, rF = 0.0, rcF = 0.0, mv0 = 0.0;
    for (int tile = w.y; tile < ntiles; tile += R.ne) {
      const int tile0 = tile * A;
      // stage the tile's deviations (contiguous in [N][3][P]) once: every
      // mode's transform reads the whole row
      const int nrow = min(A, N - tile0) * 3 * P;
      __syncthreads();
      for (int t = threadIdx.x; t < nrow; t += blockDim.x) sDv[t] = R.d[(size_t)tile0 * 3 * P + t];
      __syncthreads();
      for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        const int k = task % P, al = task / P;
        const int i = tile0 + al;
        if (i >= N) continue;
        // the FP64 pipe is the scarce unit: products of FP32 quantities stay
        // in FP32 and are converted once per task; only terms with an FP64
        // factor (the centroid x_c, the centroid-mode velocity, the masses)
        // are formed in FP64.  x.F = x_c.F + d.F, (x - x_c).F = (d - <d>).F.
        const double mm = __ldg(R.mass_mm + i);
        double v2 = 0.0, xcF = 0.0;
        float v2f = 0.f, q2f = 0.f, dF = 0.f, dcF = 0.f;
        const float invP = 1.0f / (float)P;
        for (int c = 0; c < 3; ++c) {
          const size_t row = ((size_t)i * 3 + c) * P;
          if (k == 0) {
            const double v = R.v0[(size_t)i * 3 + c];
            v2 = fma(v, v, v2);
          } else {
            const float v = R.vk[row + k];
            v2f = fmaf(v, v, v2f);
          }
          float qa = 0.f, qb = 0.f, dma = 0.f, dmb = 0.f;
          const float *__restrict__ dr = sDv + (al * 3 + c) * P;
          const float *__restrict__ mc = R.Mtf + k;
          int j = 0;
          for (; j + 1 < P; j += 2) {
            const float d0 = dr[j], d1 = dr[j + 1];
            qa = fmaf(__ldg(mc + j * P), d0, qa);
            qb = fmaf(__ldg(mc + (j + 1) * P), d1, qb);
            dma += d0;
            dmb += d1;
          }
          if (j < P) {
            qa = fmaf(__ldg(mc + j * P), dr[j], qa);
            dma += dr[j];
          }
          const float q = qa + qb;
          if (k > 0) q2f = fmaf(q, q, q2f);
          const float dk = dr[k];
          const float fk = R.F[row + k];
          xcF = fma(R.xc[(size_t)i * 3 + c], (double)fk, xcF);
          dF = fmaf(dk, fk, dF);
          dcF = fmaf(dk - (dma + dmb) * invP, fk, dcF);
        }
        v2 += (double)v2f;
        rF += xcF + (double)dF;
        rcF += (double)dcF;
        kk = fma(0.5 * mm, v2, kk);
        ss = fma(0.5 * mm * R.wn2 * __ldg(R.lam + k), (double)q2f, ss);
        if (k == 0) mv0 = fma(mm, v2, mv0);
      }
    }
    // per-mode sums: tile tasks never exceed the 128 threads, so thread t
    // always held task t, i.e. mode t mod P; sum over atoms in order
    double *out = R.epart + (size_t)w.y * (2 * P + 4);
    sK[threadIdx.x] = CSum{kk, 0.0};
    sS[threadIdx.x] = CSum{ss, 0.0};
    __syncthreads();
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
      CSum a{0.0, 0.0}, b2{0.0, 0.0};
      for (int t = k; t < ntask; t += P) {
        a.add(sK[t]);
        b2.add(sS[t]);
      }
      out[k] = a.value();
      out[P + k] = b2.value();
    }
    const CSum crF = warp_csum(CSum{rF, 0.0}), crcF = warp_csum(CSum{rcF, 0.0}), cmv0 = warp_csum(CSum{mv0, 0.0});
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      sred[0][threadIdx.x >> 5] = crF;
      sred[1][threadIdx.x >> 5] = crcF;
      sred[2][threadIdx.x >> 5] = cmv0;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      CSum sum{0.0, 0.0};
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) sum.add(sred[threadIdx.x][ww]);
      out[2 * P + threadIdx.x] = sum.value();
    }
    if (threadIdx.x == 3) out[2 * P + 3] = 0.0;
    __syncthreads();
  }
}

// Oxygen bead positions pO = xcw + d of one replica (after its state is set).
__global__ void k_bpos(const RepDesc *reps, int slot) {
  const RepDesc &R = reps[slot];
  const int P = R.P;
  const int n = R.nmol * 3 * P;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int row = e / P, k = e - row * P;   // row = 3 m + c
    const int m = row / 3, c = row - 3 * m;
    R.pO[e] = R.xcw[9 * (size_t)m + c] + R.d[((size_t)9 * m + c) * P + k];
  }
}

// Control words of every slot gathered into one array (one copy to the host).
__global__ void k_bgather_ctl(const RepDesc *reps, int nslots, long long *out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nslots) return;
  for (int w = 0; w < kCtlWords; ++w) out[(size_t)r * kCtlWords + w] = reps[r].live ? reps[r].ctl[w] : -1;
}

__device__ double neumaier_b(const double *p, int n, size_t stride) {
  double s = 0.0, c = 0.0;
  for (int b = 0; b < n; ++b) {
    const double x = p[(size_t)b * stride];
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  return s + c;
}

// Estimators, pass 2: one block per replica; output in the pimd_estimates
// layout from K_mode on.
__global__ void k_best_final(const RepDesc *reps, int nslots, double *eout) {
  __shared__ double tot[2 * kMaxBeads + 4];
  __shared__ double U[kMaxBeads], Wv[kMaxBeads];
  __shared__ CSum cu[128], cw[128];
  const int r = blockIdx.x;
  if (r >= nslots) return;
  const RepDesc &R = reps[r];
  if (!R.live) return;
  const int P = R.P;
  const int W = 2 * P + 4;
  for (int s = threadIdx.x; s < W; s += blockDim.x) tot[s] = neumaier_b(R.epart + s, R.ne, W);
  // the bead sums of U and Tr Xi over the molecules: thread t sums bead
  // t mod P over the molecule rows of chunk t / P (compensated), then the
  // chunks are added in order -- a fixed decomposition for a given P
  const int nch = P >= 128 ? 1 : 128 / P;
  const int per = (R.nmol + nch - 1) / nch;
  if (threadIdx.x < nch * P) {
    const int k = threadIdx.x % P, ch = threadIdx.x / P;
    CSum su{0.0, 0.0}, sw{0.0, 0.0};
    const int m1 = min(R.nmol, (ch + 1) * per);
    for (int m = ch * per; m < m1; ++m) {
      su.add(R.Upart[(size_t)m * P + k]);
      sw.add(R.Wpart[(size_t)m * P + k]);
    }
    cu[threadIdx.x] = su;
    cw[threadIdx.x] = sw;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    CSum su{0.0, 0.0}, sw{0.0, 0.0};
    for (int ch = 0; ch < nch; ++ch) {
      su.add(cu[ch * P + k]);
      sw.add(cw[ch * P + k]);
    }
    U[k] = su.value();
    Wv[k] = sw.value();
  }
  double *o = eout + (size_t)r * kOutStride;
  for (int k = threadIdx.x; k < 3 * kMaxBeads; k += blockDim.x) o[k] = 0.0;
  __syncthreads();
  if (threadIdx.x) return;
  double Kt = 0.0, St = 0.0, Ut = 0.0, Wt = 0.0;
  for (int k = 0; k < P; ++k) {
    o[k] = tot[k];
    o[kMaxBeads + k] = tot[P + k];
    o[2 * kMaxBeads + k] = U[k];
    Kt += tot[k];
    St += tot[P + k];
    Ut += U[k];
    Wt += Wv[k];
  }
  const double rF = tot[2 * P], rcF = tot[2 * P + 1], mv0 = tot[2 * P + 2];
  const double Nd = R.N, Pd = P, kT = R.kT, V = R.volume, spring = 2.0 * St;
  double *g = o + 3 * kMaxBeads;
  g[0] = Kt + St + Ut;
  g[1] = 1.5 * Pd * Nd * kT - 0.5 * spring / Pd;
  g[2] = -rF / (2.0 * Pd);
  g[3] = 1.5 * Nd * kT - rcF / (2.0 * Pd);
  g[4] = (3.0 * Pd * Nd * kT - spring / Pd + Wt / Pd) / (3.0 * V);
  g[5] = (2.0 * Kt + Wt) / (3.0 * V);
  g[6] = (mv0 - rcF + Wt) / (3.0 * Pd * V);
  g[7] = 2.0 * Kt / (3.0 * Nd * Pd * kBoltzmann);
  g[8] = V;
  g[9] = Wt;
}

}  // namespace pimd

// ===========================================================================
// host side: the batch engine
// ===========================================================================
namespace pimd {

namespace {

struct Replica {
  bool live = false;
  int N = 0, P = 0, nmol = 0, A = 1, G = 1, ntiles = 0, ne = 0;
  size_t bytes = 0;
  void *arena = nullptr;
  RepDesc desc{};
  std::vector<int2> items_step, items_nbr, items_est;
  std::vector<int4> items_clu;
  int2 *d_items_step = nullptr, *d_items_nbr = nullptr;
  int4 *d_items_clu = nullptr;
  int *d_counts = nullptr;   // [4] own item counts: step, cluster, nbr, est
};

template <typename T>
T *carve_ptr(char *base, size_t &off, size_t count) {
  off = (off + 255) & ~(size_t)255;
  T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
  off += count * sizeof(T);
  return p;
}

// Lay out (base == nullptr: size) a replica arena and fill the descriptor
// pointers.  Step tiles may use any A >= 1, so per-tile arrays are sized for
// A = 1 (one tile per atom).
size_t layout_replica(Replica &r, char *base) {
  const size_t N = r.N, P = r.P, len = N * 3 * P, nmol = r.nmol;
  const int NS = kLJWarps * r.G;
  RepDesc &d = r.desc;
  size_t off = 0;
  d.ctl = carve_ptr<long long>(base, off, kCtlWords);
  d.xc = carve_ptr<double>(base, off, N * 3);
  d.v0 = carve_ptr<double>(base, off, N * 3);
  d.d = carve_ptr<float>(base, off, len);
  d.vk = carve_ptr<float>(base, off, len);
  d.F = carve_ptr<float>(base, off, len);
  d.xcw = carve_ptr<float>(base, off, N * 3);
  d.pO = carve_ptr<float>(base, off, nmol * 3 * P);
  d.inv_mm = carve_ptr<double>(base, off, N);
  d.sigv = carve_ptr<double>(base, off, N);
  d.mass_mm = carve_ptr<double>(base, off, N);
  d.inv_mmf = carve_ptr<float>(base, off, N);
  d.sigvf = carve_ptr<float>(base, off, N);
  d.cAf = carve_ptr<float>(base, off, P);
  d.sAf = carve_ptr<float>(base, off, P);
  d.wsAf = carve_ptr<float>(base, off, P);
  d.c1f = carve_ptr<float>(base, off, P);
  d.c2f = carve_ptr<float>(base, off, P);
  d.Mt64 = carve_ptr<double>(base, off, P * P);
  d.lam = carve_ptr<double>(base, off, P);
  d.cref = carve_ptr<double>(base, off, nmol * 3);
  d.ccur = carve_ptr<double>(base, off, nmol * 3);
  d.nbr = carve_ptr<int>(base, off, nmol * kMaxNeighbours);
  d.nbr_off = carve_ptr<int>(base, off, nmol * (NS + 1));
  d.Upart = carve_ptr<double>(base, off, nmol * P);
  d.Wpart = carve_ptr<double>(base, off, nmol * P);
  d.epart = carve_ptr<double>(base, off, kEstItems * (2 * P + 4));
  d.mperm = carve_ptr<int>(base, off, nmol);
  r.d_items_step = carve_ptr<int2>(base, off, N);
  r.d_items_nbr = carve_ptr<int2>(base, off, (nmol + kNbrMolPerItem - 1) / kNbrMolPerItem);
  r.d_items_clu = carve_ptr<int4>(base, off, nmol * ((P + 31) / 32));
  r.d_counts = carve_ptr<int>(base, off, 4);
  return off + 256;
}

// step tile (atoms per item): A P <= 512 for the tensor-core path (P a
// multiple of 8), A 3 P <= 256 otherwise
int default_tile(int P) { return (P % 8 == 0) ? std::max(1, 512 / P) : std::max(1, 256 / (3 * P)); }

}  // namespace
}  // namespace pimd

using namespace pimd;

struct pimd_batch {
  int capacity = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // a second stream and two events: the step kernels of the bead classes run
  // side by side (a fork and a join inside every step, captured into the graph)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  DevAllocator alloc;
  std::vector<Replica> reps;
  RepDesc *d_reps = nullptr;
  // [8]: step, cluster, nbr, est items (all replicas); [4] warp-item prefix
  // of the step list; [5] the warp-item counter; [6] the rebuild-list length
  int *d_counts = nullptr;
  int2 *d_step = nullptr, *d_nbr = nullptr, *d_est = nullptr;
  int2 *d_nbr_go = nullptr;                // this step's rebuild list
  size_t cap_nbr_go = 0;
  int4 *d_clu = nullptr;
  size_t cap_step = 0, cap_clu = 0, cap_nbr = 0, cap_est = 0;
  double *d_eout = nullptr, *h_eout = nullptr;
  long long *d_ctl = nullptr, *h_ctl = nullptr;   // gathered per-replica control words
  double *stg_x = nullptr, *stg_v = nullptr, *stg_t = nullptr;
  size_t stg_len = 0;
  int grid_step = 0, grid_clu = 0, grid_nbr = 0, grid_est = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 8;
  bool dirty = true;
  int64_t launches = 0;
  int tileA[PIMD_MAX_BEADS + 1] = {0};     // autotuned step tile per P (0 = default)
  // one FP32 copy of M and M^T per bead count, shared by all replicas with
  // that P (the normal-mode matrix depends on P only): small, L1-resident
  float *ptab[PIMD_MAX_BEADS + 1] = {nullptr};
  // tensor-core fragment tables per bead count (P % 8 == 0): forward hi, lo,
  // inverse hi, lo, each [mode tile][k step][lane] float4
  float4 *mtab[PIMD_MAX_BEADS + 1] = {nullptr};
  std::vector<int2> h_step, h_nbr, h_est;
  std::vector<int4> h_clu;
  // [0] step items, [1] force, [2] nbr, [3] est, [4] end of the warp items,
  // [5] claim counter of the 64-bead warp items, [6] rebuild-list length,
  // [7] end of the 128-bead warp items, [8] their claim counter, [9] end of
  // the 64-bead warp items, [10] claim counter of the smaller warp items
  int h_counts[16] = {0};
  int wslot = wslot_floats(64);   // floats of shared memory per warp of the 64-bead warp-item kernel
  int grid_w = 0;         // its blocks (persistent grid)
  int grid_ws = 0;        // blocks of the 8-, 16-, 32-bead warp-item kernel
  bool w64_items = false, wsmall_items = false;   // which warp-item kernels have items
  int grid_w128 = 0;      // blocks of the 128-bead warp-item kernel
  bool block_items = true;   // some replica has a bead count outside the warp-item classes
  bool w128_items = false;   // some replica has 128 beads
  bool ffma = false;         // every step on the block-item kernel with FP32 FMA transforms
  int wblocks_sm = 0;     // blocks per SM in use
  int wtuned = 0;         // blocks per SM chosen by the autotuner (0: the occupancy limit)
  int nsm = 152;
};

namespace hostside {

#define BK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(PIMD_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                 \
  } while (0)

template <typename T>
pimd_status grow(pimd_batch *b, T **ptr, size_t *cap, size_t need) {
  if (need <= *cap && *ptr) return PIMD_OK;
  size_t nc = std::max<size_t>(need, std::max<size_t>(1024, 2 * *cap));
  BK(cudaStreamSynchronize(b->stream));
  dev_free(b->alloc, *ptr, b->stream);
  *ptr = (T *)dev_alloc(b->alloc, nc * sizeof(T), b->stream);
  if (!*ptr) return fail(PIMD_ENOMEM, "batch work-list allocation failed");
  *cap = nc;
  if (b->graph) {   // the captured kernels point at the old array
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return PIMD_OK;
}

void replica_items(pimd_batch *b, int slot, Replica &r) {
  if (b->ffma)
    r.A = b->tileA[r.P] > 0 ? b->tileA[r.P] : std::max(1, 256 / (3 * r.P));
  else
    r.A = (warp_class(r.P) || r.P == 128) ? kWAtoms : (b->tileA[r.P] > 0 ? b->tileA[r.P] : default_tile(r.P));
  r.desc.ffma = b->ffma ? 1 : 0;
  r.ntiles = (r.N + r.A - 1) / r.A;
  r.ne = std::min(r.ntiles, kEstItems);
  r.items_step.clear();
  for (int t = 0; t < r.ntiles; ++t) r.items_step.push_back(make_int2(slot, t));
  r.items_nbr.clear();
  for (int mb = 0; mb < (r.nmol + kNbrMolPerItem - 1) / kNbrMolPerItem; ++mb)
    r.items_nbr.push_back(make_int2(slot, mb));
  r.items_clu.clear();
  // force items (molecules per warp, bead chunks): even bead counts take two
  // beads per lane in chunks of 64, odd ones one bead per lane in chunks of 32
  const int cb = r.P % 2 == 0 ? 64 : 32;
  const int nchunk = (r.P + cb - 1) / cb;
  const int per = r.P < cb ? 32 / ((r.P % 2 == 0) ? r.P / 2 : r.P) : 1;   // molecules per warp
  for (int m = 0; m < r.nmol; m += per)
    for (int c = 0; c < nchunk; ++c) r.items_clu.push_back(make_int4(slot, m, c, 0));
  r.items_est.clear();
  const int Ae = r.P >= 128 ? 1 : 128 / r.P;
  r.ne = std::min((r.N + Ae - 1) / Ae, kEstItems);
  for (int e = 0; e < r.ne; ++e) r.items_est.push_back(make_int2(slot, e));
  r.desc.A = r.A;
  r.desc.nstep_items = r.ntiles;
  r.desc.ne = r.ne;
}

// Upload the descriptor table and the concatenated work lists (stream-ordered
// after every earlier launch that reads them).
pimd_status upload(pimd_batch *b) {
  b->h_step.clear();
  b->h_clu.clear();
  b->h_nbr.clear();
  b->h_est.clear();
  std::vector<RepDesc> descs(b->capacity);
  // warp items first, largest bead count first (the costliest items are
  // claimed first), then the block items of the other bead counts
  int n64 = 0;
  for (int P : {64, 32, 16, 8}) {
    for (int s = 0; s < b->capacity && !b->ffma; ++s) {
      Replica &r = b->reps[s];
      if (r.live && r.P == P) b->h_step.insert(b->h_step.end(), r.items_step.begin(), r.items_step.end());
    }
    if (P == 64) n64 = (int)b->h_step.size();
  }
  const int nw = (int)b->h_step.size();
  for (int s = 0; s < b->capacity && !b->ffma; ++s) {   // then the 128-bead warp items
    Replica &r = b->reps[s];
    if (r.live && r.P == 128) b->h_step.insert(b->h_step.end(), r.items_step.begin(), r.items_step.end());
  }
  const int nw128 = (int)b->h_step.size();
  for (int s = 0; s < b->capacity; ++s) {   // block items: the other bead counts (all with FFMA transforms)
    Replica &r = b->reps[s];
    if (r.live && (b->ffma || (!warp_class(r.P) && r.P != 128)))
      b->h_step.insert(b->h_step.end(), r.items_step.begin(), r.items_step.end());
  }
  for (int s = 0; s < b->capacity; ++s) {
    Replica &r = b->reps[s];
    if (r.live) {
      b->h_clu.insert(b->h_clu.end(), r.items_clu.begin(), r.items_clu.end());
      b->h_nbr.insert(b->h_nbr.end(), r.items_nbr.begin(), r.items_nbr.end());
      b->h_est.insert(b->h_est.end(), r.items_est.begin(), r.items_est.end());
      descs[s] = r.desc;
    } else {
      std::memset(&descs[s], 0, sizeof(RepDesc));
    }
  }
  pimd_status st;
  if ((st = grow(b, &b->d_step, &b->cap_step, b->h_step.size() + 1)) ||
      (st = grow(b, &b->d_clu, &b->cap_clu, b->h_clu.size() + 1)) ||
      (st = grow(b, &b->d_nbr, &b->cap_nbr, b->h_nbr.size() + 1)) ||
      (st = grow(b, &b->d_nbr_go, &b->cap_nbr_go, b->h_nbr.size() + 1)) ||
      (st = grow(b, &b->d_est, &b->cap_est, b->h_est.size() + 1)))
    return st;
  b->h_counts[0] = (int)b->h_step.size();
  b->h_counts[1] = (int)b->h_clu.size();
  b->h_counts[2] = (int)b->h_nbr.size();
  b->h_counts[3] = (int)b->h_est.size();
  b->h_counts[4] = nw;
  b->h_counts[5] = 0;
  b->h_counts[6] = 0;
  b->h_counts[7] = nw128;
  b->h_counts[8] = 0;
  b->h_counts[9] = n64;
  b->h_counts[10] = 0;
  const bool blk = b->h_counts[0] > nw128, w128 = nw128 > nw, w64 = n64 > 0, wsm = nw > n64;
  if (blk != b->block_items || w128 != b->w128_items || w64 != b->w64_items || wsm != b->wsmall_items) {
    b->block_items = blk;
    b->w128_items = w128;
    b->w64_items = w64;
    b->wsmall_items = wsm;
    if (b->graph) {   // the captured step launches another set of step kernels
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  if (!b->h_step.empty())
    BK(cudaMemcpyAsync(b->d_step, b->h_step.data(), b->h_step.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  if (!b->h_clu.empty())
    BK(cudaMemcpyAsync(b->d_clu, b->h_clu.data(), b->h_clu.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
  if (!b->h_nbr.empty())
    BK(cudaMemcpyAsync(b->d_nbr, b->h_nbr.data(), b->h_nbr.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  if (!b->h_est.empty())
    BK(cudaMemcpyAsync(b->d_est, b->h_est.data(), b->h_est.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  BK(cudaMemcpyAsync(b->d_counts, b->h_counts, sizeof(b->h_counts), cudaMemcpyHostToDevice, b->stream));
  BK(cudaMemcpyAsync(b->d_reps, descs.data(), sizeof(RepDesc) * b->capacity, cudaMemcpyHostToDevice, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  b->dirty = false;
  return PIMD_OK;
}

// The two step kernels: warp items, then block items.
// The classes' step kernels touch disjoint replicas, so the 8-32-bead and
// block-item kernels run on the side stream beside the 64- and 128-bead ones
// (fork after the control kernel, join before the rebuild decision): one
// kernel's tail fills with the other's work.
void launch_step_kernels(pimd_batch *b) {
  const bool fork = (b->w64_items || b->w128_items) && (b->wsmall_items || b->block_items);
  cudaStream_t s2 = fork ? b->side : b->stream;
  if (fork) {
    cudaEventRecord(b->fork_ev, b->stream);
    cudaStreamWaitEvent(b->side, b->fork_ev, 0);
  }
  if (b->w64_items)
    k_bstep_w<false><<<b->grid_w, kWWarps * 32, (size_t)kWWarps * b->wslot * sizeof(float), b->stream>>>(
        b->d_reps, b->d_step, b->d_counts, b->d_counts + 5, b->wslot);
  if (b->wsmall_items)
    k_bstep_w<true><<<b->grid_ws, kWWarps * 32, (size_t)kWWarps * wslot_floats(32) * sizeof(float), s2>>>(
        b->d_reps, b->d_step, b->d_counts, b->d_counts + 10, wslot_floats(32));
  if (b->w128_items)
    k_bstep_w128<<<b->grid_w128, kWWarps * 32, (size_t)kWWarps * wslot_floats(128) * sizeof(float), b->stream>>>(
        b->d_reps, b->d_step, b->d_counts, b->d_counts + 8);
  if (b->block_items) k_bstep<<<b->grid_step, 128, 0, s2>>>(b->d_reps, b->d_step, b->d_counts);
  if (fork) {
    cudaEventRecord(b->join_ev, b->side);
    cudaStreamWaitEvent(b->stream, b->join_ev, 0);
  }
}

// The rebuild decision over all neighbour items, then the rebuilds listed.
void launch_nbr_kernels(pimd_batch *b) {
  k_bdecide<<<b->nsm, 256, 0, b->stream>>>(b->d_reps, b->d_nbr, b->d_counts + 2, b->d_nbr_go, b->d_counts + 6);
  k_bnbr<<<b->grid_nbr, kNbrThreads, kNbrSmem, b->stream>>>(b->d_reps, b->d_nbr_go, b->d_counts + 6);
}

// Kernels launched per MD step: control, warp-item step, 128-bead warp-item
// step and block-item step (each when some replica needs it), rebuild
// decision, rebuilds, forces.
int step_launches(const pimd_batch *b) {
  return 4 + (b->w64_items ? 1 : 0) + (b->wsmall_items ? 1 : 0) + (b->block_items ? 1 : 0) + (b->w128_items ? 1 : 0);
}

// One MD step of every active replica.
cudaError_t launch_one_step(pimd_batch *b, cudaEvent_t e0, cudaEvent_t e1) {
  k_bctl<<<(b->capacity + 127) / 128, 128, 0, b->stream>>>(b->d_reps, b->capacity, 0, b->d_counts + 5);
  if (e0) cudaEventRecord(e0, b->stream);
  launch_step_kernels(b);
  if (e1) cudaEventRecord(e1, b->stream);
  launch_nbr_kernels(b);
  k_bforce<<<b->grid_clu, 128, 0, b->stream>>>(b->d_reps, b->d_clu, b->d_counts + 1, 0);
  return cudaGetLastError();
}

pimd_status capture(pimd_batch *b) {
  cudaGraph_t g = nullptr;
  BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < b->graph_steps && e == cudaSuccess; ++s) e = launch_one_step(b, nullptr, nullptr);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(PIMD_ECUDA, "batch graph capture failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return fail(PIMD_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
  }
  return PIMD_OK;
}

pimd_status ensure_staging(pimd_batch *b, size_t len) {
  if (len <= b->stg_len && b->stg_x) return PIMD_OK;
  BK(cudaStreamSynchronize(b->stream));
  dev_free(b->alloc, b->stg_x, b->stream);
  b->stg_x = (double *)dev_alloc(b->alloc, 3 * len * sizeof(double), b->stream);
  if (!b->stg_x) {
    b->stg_len = 0;
    return fail(PIMD_ENOMEM, "batch staging allocation failed");
  }
  b->stg_v = b->stg_x + len;
  b->stg_t = b->stg_v + len;
  b->stg_len = len;
  return PIMD_OK;
}

// TF32 rounding as cvt.rna (to nearest, ties away from zero): 10 mantissa bits.
float tf32_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x1000u;
    u &= 0xffffe000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// m16n8k8 A fragments of a P x P matrix A (row-major, rows padded to 16 with
// zeros) as [mode tile mt][k step ks][lane] float4 = (a0, a1, a2, a3):
// a0 = A[16 mt + g][8 ks + t], a1 = A[16 mt + g + 8][8 ks + t],
// a2 = A[16 mt + g][8 ks + t + 4], a3 = A[16 mt + g + 8][8 ks + t + 4],
// g = lane / 4, t = lane % 4; hi = tf32(a), lo = tf32(a - hi).
void fragment_tables(const std::vector<double> &A, int P, std::vector<float> &hi, std::vector<float> &lo) {
  const int MT = (P + 15) / 16, KS = P / 8;
  hi.assign((size_t)MT * KS * 32 * 4, 0.f);
  lo.assign(hi.size(), 0.f);
  auto at = [&](int r, int c) -> float { return r < P ? (float)A[(size_t)r * P + c] : 0.f; };
  for (int mt = 0; mt < MT; ++mt)
    for (int ks = 0; ks < KS; ++ks)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane / 4, t = lane % 4;
        const float v[4] = {at(16 * mt + g, 8 * ks + t), at(16 * mt + g + 8, 8 * ks + t),
                            at(16 * mt + g, 8 * ks + t + 4), at(16 * mt + g + 8, 8 * ks + t + 4)};
        for (int q = 0; q < 4; ++q) {
          const size_t o = (((size_t)mt * KS + ks) * 32 + lane) * 4 + q;
          hi[o] = tf32_round(v[q]);
          lo[o] = tf32_round(v[q] - hi[o]);
        }
      }
}

SplitStepArgs replica_split_args(const Replica &r) {
  SplitStepArgs a{};
  std::memset(&a, 0, sizeof(a));
  a.N = r.N;
  a.P = r.P;
  a.A = r.A;
  a.xc = r.desc.xc;
  a.v0 = r.desc.v0;
  a.d = r.desc.d;
  a.vk = r.desc.vk;
  a.F = r.desc.F;
  a.xcw = r.desc.xcw;
  for (int c = 0; c < 3; ++c) {
    a.box[c] = r.desc.box[c];
    a.invbox[c] = r.desc.invbox[c];
  }
  return a;
}

}  // namespace hostside
using namespace hostside;

namespace pimd {

// ---- the warp-item step for a single-system handle (split precision) ------
size_t split_warp_desc_bytes() { return sizeof(RepDesc); }
size_t split_warp_frag_float4(int P) { return 4 * (size_t)((P + 15) / 16) * (P / 8) * 32; }
bool split_warp_class(int P) { return warp_class(P) || P == 128; }

// Fill a descriptor for the handle's own arrays and upload it with the FP32
// per-atom constants and the TF32 fragment tables of M and M^T into the
// device buffers the handle carved for them.
namespace {
int g_sw_nsm = 0;   // SM count of the device, read at set-up (one GPU per process)

cudaError_t split_warp_prepare() {
  if (g_sw_nsm) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_sstep_w<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kWWarps * wslot_floats(32) * sizeof(float)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_sstep_w<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kWWarps * wslot_floats(64) * sizeof(float)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_sstep_w<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kWWarps * wslot_floats(128) * sizeof(float)));
  if (e == cudaSuccess) g_sw_nsm = nsm > 0 ? nsm : 152;
  return e;
}
}  // namespace

cudaError_t split_warp_setup(const SplitWarpSetup &w, cudaStream_t st) {
  const cudaError_t pe = split_warp_prepare();   // outside any stream capture
  if (pe != cudaSuccess) return pe;
  const int N = w.N, P = w.P;
  RepDesc d;
  std::memset(&d, 0, sizeof(d));
  d.live = 1;
  d.N = N;
  d.P = P;
  d.nmol = w.cref ? N / 3 : 0;
  d.integrator = w.integrator;
  d.thermo = w.thermo;
  d.seed = w.seed;
  d.dt = w.dt;
  d.tA = w.tA;
  d.dr0 = w.tA / std::sqrt((double)P);
  d.c1_0 = w.c1_0;
  d.c2_0 = w.c2_0;
  for (int c = 0; c < 3; ++c) {
    d.box[c] = w.box[c];
    d.invbox[c] = w.box[c] > 0 ? 1.0 / w.box[c] : 0.0;
  }
  d.ctl = w.ctl;
  d.xc = w.xc;
  d.v0 = w.v0;
  d.d = w.d;
  d.vk = w.vk;
  d.F = w.F;
  d.xcw = w.xcw;
  d.pO = nullptr;
  d.inv_mm = w.inv_mm;
  d.sigv = w.sigv;
  d.inv_mmf = w.inv_mmf;
  d.sigvf = w.sigvf;
  d.cAf = w.cAf;
  d.sAf = w.sAf;
  d.wsAf = w.wsAf;
  d.c1f = w.c1f;
  d.c2f = w.c2f;
  d.cref = w.cref;
  d.ccur = w.ccur;
  const size_t one = split_warp_frag_float4(P) / 4;
  d.mfa_hi = w.frag;
  d.mfa_lo = w.frag + one;
  d.mia_hi = w.frag + 2 * one;
  d.mia_lo = w.frag + 3 * one;
  std::vector<double> Mt((size_t)P * P);
  std::vector<double> M(w.M_host, w.M_host + (size_t)P * P);
  for (int k = 0; k < P; ++k)
    for (int j = 0; j < P; ++j) Mt[(size_t)j * P + k] = M[(size_t)k * P + j];
  std::vector<float> fh, fl, ih, il;
  fragment_tables(M, P, fh, fl);
  fragment_tables(Mt, P, ih, il);
  std::vector<float> imf(N), sgf(N);
  for (int i = 0; i < N; ++i) {
    imf[i] = (float)w.inv_mm_host[i];
    sgf[i] = (float)w.sigv_host[i];
  }
  long long ctl[kCtlWords] = {0};
  const struct {
    void *dst;
    const void *src;
    size_t bytes;
  } ups[] = {
      {w.desc, &d, sizeof(RepDesc)},
      {w.frag, fh.data(), one * sizeof(float4)},
      {w.frag + one, fl.data(), one * sizeof(float4)},
      {w.frag + 2 * one, ih.data(), one * sizeof(float4)},
      {w.frag + 3 * one, il.data(), one * sizeof(float4)},
      {w.inv_mmf, imf.data(), N * sizeof(float)},
      {w.sigvf, sgf.data(), N * sizeof(float)},
      {w.ctl, ctl, sizeof(ctl)},
  };
  for (const auto &u : ups) {
    // pageable sources: the copy completes before the call returns
    const cudaError_t e = cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = cudaMemsetAsync(w.done, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t launch_step_split_warp(const void *desc, int N, int P, const int64_t *step, int step_off, int first,
                                   double *blkmax, unsigned *done, cudaStream_t s) {
  const cudaError_t pe = split_warp_prepare();
  if (pe != cudaSuccess) return pe;
  const int nsm = g_sw_nsm;
  const int cls = P == 128 ? 2 : (P == 64 ? 1 : (P == 32 ? 0 : 3));
  const int slot = wslot_floats(P);
  // resident blocks per SM (registers, shared memory)
  const int per_sm = cls == 2 ? 2 : (cls == 1 ? 3 : (cls == 0 ? 4 : 6));
  const int smem = (int)(kWWarps * slot * sizeof(float));
  const int ntiles = (N + kWAtoms - 1) / kWAtoms;
  const int warps = std::min(ntiles, nsm * per_sm * kWWarps);
  const int grid = std::max(1, (warps + kWWarps - 1) / kWWarps);
  const RepDesc *d = reinterpret_cast<const RepDesc *>(desc);
  if (cls == 3)
    k_sstep_w<3><<<grid, kWWarps * 32, smem, s>>>(d, step, step_off, first, slot, blkmax, done);
  else if (cls == 2)
    k_sstep_w<2><<<grid, kWWarps * 32, smem, s>>>(d, step, step_off, first, slot, blkmax, done);
  else if (cls == 1)
    k_sstep_w<1><<<grid, kWWarps * 32, smem, s>>>(d, step, step_off, first, slot, blkmax, done);
  else
    k_sstep_w<0><<<grid, kWWarps * 32, smem, s>>>(d, step, step_off, first, slot, blkmax, done);
  return cudaGetLastError();
}

}  // namespace pimd

size_t batch_replica_bytes(int N, int P) {
  Replica r;
  r.N = N;
  r.P = P;
  r.nmol = N / 3;
  r.G = water_lane_groups(P);
  return layout_replica(r, nullptr);
}

extern "C" size_t pimd_batch_replica_bytes(int32_t n_atoms, int32_t P) {
  if (n_atoms <= 0 || P < 1 || P > PIMD_MAX_BEADS) return 0;
  return batch_replica_bytes(n_atoms, P);
}

extern "C" pimd_status pimd_batch_create(int32_t max_replicas, void *stream, pimd_batch **out) {
  if (!out) return fail(PIMD_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_replicas < 1 || max_replicas > 65536) return fail(PIMD_EINVAL, "max_replicas outside 1..65536");
  pimd_batch *b = new pimd_batch();
  b->capacity = max_replicas;
  b->reps.resize(max_replicas);
  b->alloc = current_allocator();
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(PIMD_ECUDA, "cudaStreamCreate failed");
    }
    b->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    pimd_batch_destroy(b);
    return fail(PIMD_ECUDA, "cannot create the batch's side stream");
  }
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // the rebuild stages up to kBatchMaxMol centroids in dynamic shared memory
  if (cudaFuncSetAttribute((const void *)k_bnbr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNbrSmem) !=
      cudaSuccess) {
    cudaGetLastError();
    pimd_batch_destroy(b);
    return fail(PIMD_ECUDA, "cannot enable %zu bytes of shared memory for the neighbour kernel", kNbrSmem);
  }
  const int wsmem = (int)(kWWarps * wslot_floats(kWMaxP) * sizeof(float));
  const int wsmem128 = (int)(kWWarps * wslot_floats(128) * sizeof(float));
  if (cudaFuncSetAttribute((const void *)k_bstep_w<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute((const void *)k_bstep_w<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kWWarps * wslot_floats(32) * sizeof(float))) != cudaSuccess ||
      cudaFuncSetAttribute((const void *)k_bstep_w128, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem128) !=
          cudaSuccess) {
    cudaGetLastError();
    pimd_batch_destroy(b);
    return fail(PIMD_ECUDA, "cannot enable %d bytes of shared memory for the step kernels", wsmem128);
  }
  b->nsm = nsm;
  // persistent grids: every SM filled to the kernel's occupancy limit
  auto occ = [&](const void *fn, size_t smem = 0, int threads = 128) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess || n < 1) n = 2;
    return nsm * n;
  };
  b->grid_step = occ((const void *)k_bstep);
  b->grid_w128 = occ((const void *)k_bstep_w128, (size_t)kWWarps * wslot_floats(128) * sizeof(float));
  b->grid_ws = occ((const void *)k_bstep_w<true>, (size_t)kWWarps * wslot_floats(32) * sizeof(float));
  b->wblocks_sm = 0;
  {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)k_bstep_w<false>, kWWarps * 32,
                                                      (size_t)kWWarps * b->wslot * sizeof(float)) != cudaSuccess ||
        nb < 1)
      nb = 1;
    b->wblocks_sm = nb;
    b->grid_w = nsm * nb;
  }
  b->grid_clu = occ((const void *)k_bforce);
  b->grid_nbr = occ((const void *)k_bnbr, kNbrSmem, kNbrThreads);
  b->grid_est = 8 * nsm;
  auto fail_free = [&](pimd_status st) {
    pimd_batch_destroy(b);
    return st;
  };
  b->d_reps = (RepDesc *)dev_alloc(b->alloc, sizeof(RepDesc) * max_replicas, b->stream);
  b->d_counts = (int *)dev_alloc(b->alloc, sizeof(b->h_counts), b->stream);
  b->d_eout = (double *)dev_alloc(b->alloc, sizeof(double) * kOutStride * max_replicas, b->stream);
  b->d_ctl = (long long *)dev_alloc(b->alloc, sizeof(long long) * kCtlWords * max_replicas, b->stream);
  if (!b->d_reps || !b->d_counts || !b->d_eout || !b->d_ctl)
    return fail_free(fail(PIMD_ENOMEM, "batch allocation failed"));
  if (cudaMallocHost(&b->h_eout, sizeof(double) * kOutStride * max_replicas) != cudaSuccess ||
      cudaMallocHost(&b->h_ctl, sizeof(long long) * kCtlWords * max_replicas) != cudaSuccess)
    return fail_free(fail(PIMD_ENOMEM, "pinned allocation failed"));
  pimd_status st = upload(b);
  if (st != PIMD_OK) return fail_free(st);
  *out = b;
  return PIMD_OK;
}

extern "C" void pimd_batch_destroy(pimd_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto &r : b->reps)
    if (r.arena) dev_free(b->alloc, r.arena, b->stream);
  dev_free(b->alloc, b->d_reps, b->stream);
  dev_free(b->alloc, b->d_counts, b->stream);
  dev_free(b->alloc, b->d_eout, b->stream);
  dev_free(b->alloc, b->d_ctl, b->stream);
  dev_free(b->alloc, b->d_step, b->stream);
  dev_free(b->alloc, b->d_clu, b->stream);
  dev_free(b->alloc, b->d_nbr, b->stream);
  dev_free(b->alloc, b->d_nbr_go, b->stream);
  dev_free(b->alloc, b->d_est, b->stream);
  dev_free(b->alloc, b->stg_x, b->stream);
  for (auto p : b->ptab) dev_free(b->alloc, p, b->stream);
  for (auto p : b->mtab) dev_free(b->alloc, p, b->stream);
  if (b->h_eout) cudaFreeHost(b->h_eout);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->join_ev) cudaEventDestroy(b->join_ev);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

extern "C" pimd_status pimd_batch_add(pimd_batch *b, const pimd_system *sys, int32_t P, double T, double dt,
                                      double gamma0, const pimd_params *params, int64_t nsteps,
                                      int32_t *slot_out) {
  if (!b || !slot_out) return fail(PIMD_EINVAL, "NULL argument");
  pimd_params prm;
  pimd_status st = validate_create(sys, P, T, dt, gamma0, params, &prm);
  if (st != PIMD_OK) return st;
  if ((st = require_default_keywords(prm, "the batch engine")) != PIMD_OK) return st;
  if (sys->potential != PIMD_POT_WATERLIKE)
    return fail(PIMD_EINVAL, "the batch engine runs water-like systems");
  if (sys->n_atoms / 3 > kBatchMaxMol)
    return fail(PIMD_EINVAL, "batch replicas hold at most %d molecules", kBatchMaxMol);
  if (nsteps < 0) return fail(PIMD_EINVAL, "nsteps must be >= 0");
  // no batch kernel may be in flight while a new descriptor goes live
  BK(cudaStreamSynchronize(b->stream));
  int slot = -1;
  for (int s = 0; s < b->capacity; ++s)
    if (!b->reps[s].live) {
      slot = s;
      break;
    }
  if (slot < 0) return fail(PIMD_EBUDGET, "batch is full (%d replicas)", b->capacity);
  Replica r;
  r.N = sys->n_atoms;
  r.P = P;
  r.nmol = r.N / 3;
  r.G = water_lane_groups(P);
  r.bytes = layout_replica(r, nullptr);
  r.arena = dev_alloc(b->alloc, r.bytes, b->stream);
  if (!r.arena) return fail(PIMD_ENOMEM, "replica allocation of %zu bytes failed", r.bytes);
  layout_replica(r, (char *)r.arena);
  replica_items(b, slot, r);
  RepDesc &d = r.desc;
  HostTables tb;
  build_tables(P, T, dt, prm, tb);
  d.live = 1;
  d.N = r.N;
  d.P = P;
  d.nmol = r.nmol;
  d.G = r.G;
  d.integrator = prm.integrator;
  d.thermo = prm.thermostat == PIMD_THERMO_PILE_L;
  d.seed = prm.seed;
  d.dt = dt;
  d.tA = tb.tA;
  d.dr0 = tb.tA / std::sqrt((double)P);
  d.c1_0 = tb.c1[0];
  d.c2_0 = tb.c2[0];
  d.kT = kBoltzmann * T;
  d.volume = sys->box[0] * sys->box[1] * sys->box[2];
  d.wn2 = tb.wn * tb.wn;
  for (int c = 0; c < 3; ++c) {
    d.box[c] = sys->box[c];
    d.invbox[c] = 1.0 / sys->box[c];
  }
  d.kb = sys->ff[0];
  d.r0 = sys->ff[1];
  d.kth = sys->ff[2];
  d.th0 = sys->ff[3];
  d.eps = sys->ff[4];
  d.sig = sys->ff[5];
  d.rc = sys->ff[6];
  // Verlet skin of the replica's O-O list (A): a thinner skin than the
  // single-system 1.5 A trades more frequent rebuilds for fewer list
  // candidates in the force kernel (the 256-replica mix: 1.5 A 0.289, 1.0 A
  // 0.276, 0.85 A 0.273, 0.7 A 0.270 ms per MD step; rebuilds on 1.6, 2.7,
  // 3.4, 4.7% of replica-steps).  0.85 A keeps every replica of 100-400 K
  // well clear of rebuilding every step (the oxygens' bead spread alone
  // uses up to ~0.5 A of the budget at 100 K).  Rebuild timing changes no
  // force: the list is complete whenever it is used and its sums are
  // ordered by neighbour index.
  d.skin = 0.85;
  d.rlist = d.rc + d.skin;
  for (int c = 0; c < 3; ++c) {
    d.boxf[c] = (float)d.box[c];
    d.invboxf[c] = (float)d.invbox[c];
  }
  d.kbf = (float)d.kb;
  d.r0f = (float)d.r0;
  d.kthf = (float)d.kth;
  d.th0f = (float)d.th0;
  d.rc2f = (float)(d.rc * d.rc);
  d.sig2f = (float)(d.sig * d.sig);
  d.e4f = (float)(4.0 * d.eps);
  d.e24f = (float)(24.0 * d.eps);
  auto cleanup = [&](pimd_status s2) {
    cudaStreamSynchronize(b->stream);
    dev_free(b->alloc, r.arena, b->stream);
    return s2;
  };
  // tables and per-atom constants
  const int N = r.N;
  std::vector<double> inv_mm(N), sigv(N), mass_mm(N);
  std::vector<float> inv_mmf(N), sigvf(N);
  for (int i = 0; i < N; ++i) {
    const double mm = sys->mass[i] * kMvv2e;
    mass_mm[i] = mm;
    inv_mm[i] = 1.0 / mm;
    sigv[i] = std::sqrt(P * kBoltzmann * T / mm);
    inv_mmf[i] = (float)inv_mm[i];
    sigvf[i] = (float)sigv[i];
  }
  // force work order: molecules sorted along a Morton curve of their initial
  // oxygen bead-mean positions (wrapped into the box, 10 bits per axis), so
  // consecutive items are near each other in space and share neighbours
  const int nmol = N / 3;
  std::vector<int> mperm(nmol);
  {
    std::vector<std::pair<uint64_t, int>> key(nmol);
    auto spread = [](uint64_t v) {   // bits of v at every third position
      uint64_t x = v & 0x3ff;
      x = (x | (x << 16)) & 0x30000ff;
      x = (x | (x << 8)) & 0x300f00f;
      x = (x | (x << 4)) & 0x30c30c3;
      x = (x | (x << 2)) & 0x9249249;
      return x;
    };
    for (int m = 0; m < nmol; ++m) {
      uint64_t code = 0;
      for (int c = 0; c < 3; ++c) {
        double a = 0.0;
        for (int k = 0; k < P; ++k) a += sys->pos[((size_t)k * N + 3 * m) * 3 + c];
        a /= P;
        const double L = sys->box[c];
        double f = a / L - std::floor(a / L);
        if (!(f >= 0.0 && f < 1.0)) f = 0.0;
        code |= spread((uint64_t)(f * 1024.0)) << c;
      }
      key[m] = {code, m};
    }
    std::sort(key.begin(), key.end());
    for (int m = 0; m < nmol; ++m) mperm[m] = key[m].second;
  }
  std::vector<float> Mf(tb.M.begin(), tb.M.end()), Mtf(tb.Mt.begin(), tb.Mt.end());
  if (!b->ptab[P]) {
    float *t = (float *)dev_alloc(b->alloc, 2 * (size_t)P * P * sizeof(float), b->stream);
    if (!t) return cleanup(fail(PIMD_ENOMEM, "mode-table allocation failed"));
    if (cudaMemcpy(t, Mf.data(), Mf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t + (size_t)P * P, Mtf.data(), Mtf.size() * sizeof(float), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      dev_free(b->alloc, t, b->stream);
      return cleanup(fail(PIMD_ECUDA, "mode-table upload failed"));
    }
    b->ptab[P] = t;
  }
  d.Mf = b->ptab[P];
  d.Mtf = b->ptab[P] + (size_t)P * P;
  d.mfa_hi = d.mfa_lo = d.mia_hi = d.mia_lo = nullptr;
  if (P % 8 == 0) {
    const size_t one = (size_t)((P + 15) / 16) * (P / 8) * 32;   // float4 per table
    if (!b->mtab[P]) {
      std::vector<float> fh, fl, ih, il;
      fragment_tables(tb.M, P, fh, fl);
      fragment_tables(tb.Mt, P, ih, il);
      float4 *t = (float4 *)dev_alloc(b->alloc, 4 * one * sizeof(float4), b->stream);
      if (!t) return cleanup(fail(PIMD_ENOMEM, "mode-table allocation failed"));
      const std::vector<float> *parts[4] = {&fh, &fl, &ih, &il};
      for (int q = 0; q < 4; ++q)
        if (cudaMemcpy(t + q * one, parts[q]->data(), one * sizeof(float4), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
          dev_free(b->alloc, t, b->stream);
          return cleanup(fail(PIMD_ECUDA, "mode-table upload failed"));
        }
      b->mtab[P] = t;
    }
    d.mfa_hi = b->mtab[P];
    d.mfa_lo = b->mtab[P] + one;
    d.mia_hi = b->mtab[P] + 2 * one;
    d.mia_lo = b->mtab[P] + 3 * one;
  }
  std::vector<float> cAf(tb.cA.begin(), tb.cA.end()), sAf(tb.sA.begin(), tb.sA.end());
  std::vector<float> wsAf(tb.wsA.begin(), tb.wsA.end()), c1f(tb.c1.begin(), tb.c1.end());
  std::vector<float> c2f(tb.c2.begin(), tb.c2.end());
  long long ctl[kCtlWords] = {0, (long long)nsteps, 1, 0, 0, 0, 0, 0};
  int counts[4] = {(int)r.items_step.size(), (int)r.items_clu.size(), (int)r.items_nbr.size(),
                   (int)r.items_est.size()};
  const struct {
    void *dst;
    const void *src;
    size_t bytes;
  } ups[] = {
      {d.ctl, ctl, sizeof(ctl)},
      {(void *)d.inv_mm, inv_mm.data(), N * sizeof(double)},
      {(void *)d.sigv, sigv.data(), N * sizeof(double)},
      {(void *)d.mass_mm, mass_mm.data(), N * sizeof(double)},
      {(void *)d.inv_mmf, inv_mmf.data(), N * sizeof(float)},
      {(void *)d.sigvf, sigvf.data(), N * sizeof(float)},
      {(void *)d.cAf, cAf.data(), P * sizeof(float)},
      {(void *)d.sAf, sAf.data(), P * sizeof(float)},
      {(void *)d.wsAf, wsAf.data(), P * sizeof(float)},
      {(void *)d.c1f, c1f.data(), P * sizeof(float)},
      {(void *)d.c2f, c2f.data(), P * sizeof(float)},
      {(void *)d.Mt64, tb.Mt.data(), (size_t)P * P * sizeof(double)},
      {(void *)d.lam, tb.lam.data(), P * sizeof(double)},
      {r.d_items_step, r.items_step.data(), r.items_step.size() * sizeof(int2)},
      {r.d_items_nbr, r.items_nbr.data(), r.items_nbr.size() * sizeof(int2)},
      {r.d_items_clu, r.items_clu.data(), r.items_clu.size() * sizeof(int4)},
      {(void *)d.mperm, mperm.data(), nmol * sizeof(int)},
      {r.d_counts, counts, sizeof(counts)},
      {b->d_reps + slot, &d, sizeof(RepDesc)},
  };
  for (const auto &u : ups)
    if (u.bytes && cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return cleanup(fail(PIMD_ECUDA, "replica upload failed"));
  const size_t len = (size_t)N * 3 * P;
  if ((st = ensure_staging(b, len)) != PIMD_OK) return cleanup(st);
  cudaError_t e = cudaMemcpyAsync(b->stg_t, sys->pos, len * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = launch_pna_to_nap(b->stg_t, b->stg_x, N, P, b->stream);
  if (e == cudaSuccess) {
    if (sys->vel) {
      e = cudaMemcpyAsync(b->stg_t, sys->vel, len * sizeof(double), cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = launch_pna_to_nap(b->stg_t, b->stg_v, N, P, b->stream);
    } else {
      e = launch_thermal_v(b->stg_v, d.sigv, nullptr, d.seed, N, P, b->stream);
    }
  }
  if (e == cudaSuccess) e = launch_compress_split(replica_split_args(r), b->stg_x, b->stg_v, b->stream);
  if (e == cudaSuccess) {
    NbrArgs na{};
    std::memset(&na, 0, sizeof(na));
    na.nmol = r.nmol;
    na.P = P;
    na.x = b->stg_x;
    e = launch_centroids(na, d.ccur, b->stream);
  }
  // initial neighbour list and forces of this replica only
  if (e == cudaSuccess) {
    k_bpos<<<std::min(1024, (r.nmol * 3 * P + 255) / 256), 256, 0, b->stream>>>(b->d_reps, slot);
    k_bnbr<<<std::max(1, (int)r.items_nbr.size()), kNbrThreads, kNbrSmem, b->stream>>>(b->d_reps, r.d_items_nbr,
                                                                        r.d_counts + 2);
    k_bforce<<<std::max(1, (int)std::min<size_t>((r.items_clu.size() + 3) / 4, b->grid_clu)), 128, 0,
               b->stream>>>(b->d_reps, r.d_items_clu, r.d_counts + 1, 1);
    b->launches += 3;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    // the slot's descriptor was uploaded: mark it dead again
    RepDesc z;
    std::memset(&z, 0, sizeof(z));
    cudaMemcpyAsync(b->d_reps + slot, &z, sizeof(z), cudaMemcpyHostToDevice, b->stream);
    return cleanup(fail(PIMD_ECUDA, "replica initialisation failed: %s", cudaGetErrorString(e)));
  }
  r.live = true;
  b->reps[slot] = r;
  b->dirty = true;
  *slot_out = slot;
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_remove(pimd_batch *b, int32_t slot) {
  if (!b || slot < 0 || slot >= b->capacity || !b->reps[slot].live)
    return fail(PIMD_ENOTFOUND, "no replica in slot %d", slot);
  BK(cudaStreamSynchronize(b->stream));
  Replica &r = b->reps[slot];
  RepDesc z;
  std::memset(&z, 0, sizeof(z));
  BK(cudaMemcpyAsync(b->d_reps + slot, &z, sizeof(z), cudaMemcpyHostToDevice, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  dev_free(b->alloc, r.arena, b->stream);
  r = Replica();
  b->dirty = true;
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_run(pimd_batch *b, int64_t nsteps) {
  if (!b || nsteps < 0) return fail(PIMD_EINVAL, "invalid argument");
  pimd_status st;
  if (b->dirty && (st = upload(b)) != PIMD_OK) return st;
  if (nsteps == 0) return PIMD_OK;
  int64_t left = nsteps;
  if (left >= b->graph_steps) {
    if (!b->graph && (st = capture(b)) != PIMD_OK) return st;
    while (left >= b->graph_steps) {
      BK(cudaGraphLaunch(b->graph, b->stream));
      b->launches += (int64_t)step_launches(b) * b->graph_steps;
      left -= b->graph_steps;
    }
  }
  for (; left > 0; --left) {
    BK(launch_one_step(b, nullptr, nullptr));
    b->launches += step_launches(b);
  }
  const int cg = (b->capacity + 127) / 128;
  k_bctl<<<cg, 128, 0, b->stream>>>(b->d_reps, b->capacity, 1, nullptr);
  k_bclose<<<b->grid_step, 128, 0, b->stream>>>(b->d_reps, b->d_step, b->d_counts + 0);
  k_bctl<<<cg, 128, 0, b->stream>>>(b->d_reps, b->capacity, 2, nullptr);
  b->launches += 3;
  BK(cudaGetLastError());
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_sync(pimd_batch *b) {
  if (!b) return fail(PIMD_EINVAL, "batch is NULL");
  BK(cudaStreamSynchronize(b->stream));
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_status(pimd_batch *b, int64_t *step, int64_t *steps_left, int64_t *rebuilds) {
  if (!b) return fail(PIMD_EINVAL, "batch is NULL");
  pimd_status st;
  if (b->dirty && (st = upload(b)) != PIMD_OK) return st;
  k_bgather_ctl<<<(b->capacity + 127) / 128, 128, 0, b->stream>>>(b->d_reps, b->capacity, b->d_ctl);
  BK(cudaGetLastError());
  BK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(long long) * kCtlWords * b->capacity, cudaMemcpyDeviceToHost,
                     b->stream));
  BK(cudaStreamSynchronize(b->stream));
  for (int s = 0; s < b->capacity; ++s) {
    const long long *c = b->h_ctl + (size_t)s * kCtlWords;
    if (step) step[s] = b->reps[s].live ? c[kCtlStep] : -1;
    if (steps_left) steps_left[s] = b->reps[s].live ? c[kCtlLeft] : -1;
    if (rebuilds) rebuilds[s] = b->reps[s].live ? c[kCtlRebuilds] : -1;
    if (b->reps[s].live && (c[kCtlWords - 1] & kErrNbrOverflow))
      return fail(PIMD_EOVERFLOW, "replica %d: neighbour list overflow", s);
  }
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_estimators(pimd_batch *b, pimd_estimates *out) {
  if (!b || !out) return fail(PIMD_EINVAL, "NULL argument");
  pimd_status st;
  if (b->dirty && (st = upload(b)) != PIMD_OK) return st;
  if (b->h_counts[3] > 0) {
    k_best<<<std::min(b->grid_est, b->h_counts[3]), 128, 0, b->stream>>>(b->d_reps, b->d_est, b->d_counts + 3);
    k_best_final<<<b->capacity, 128, 0, b->stream>>>(b->d_reps, b->capacity, b->d_eout);
    b->launches += 2;
    BK(cudaGetLastError());
  }
  // the control words (steps, error bits) and the outputs, one synchronisation
  k_bgather_ctl<<<(b->capacity + 127) / 128, 128, 0, b->stream>>>(b->d_reps, b->capacity, b->d_ctl);
  b->launches += 1;
  BK(cudaGetLastError());
  BK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(long long) * kCtlWords * b->capacity, cudaMemcpyDeviceToHost,
                     b->stream));
  BK(cudaMemcpyAsync(b->h_eout, b->d_eout, sizeof(double) * kOutStride * b->capacity, cudaMemcpyDeviceToHost,
                     b->stream));
  BK(cudaStreamSynchronize(b->stream));
  for (int s = 0; s < b->capacity; ++s)
    if (b->reps[s].live && (b->h_ctl[(size_t)s * kCtlWords + kCtlWords - 1] & kErrNbrOverflow))
      return fail(PIMD_EOVERFLOW, "replica %d: neighbour list overflow", s);
  for (int s = 0; s < b->capacity; ++s) {
    pimd_estimates &e = out[s];
    std::memset(&e, 0, sizeof(e));
    if (!b->reps[s].live) {
      e.step = -1;
      continue;
    }
    std::memcpy(e.K_mode, b->h_eout + (size_t)s * kOutStride, sizeof(double) * kOutStride);
    e.step = b->h_ctl[(size_t)s * kCtlWords + kCtlStep];
    e.P = b->reps[s].P;
    e.N = b->reps[s].N;
    if (!std::isfinite(e.H)) return fail(PIMD_ENONFINITE, "replica %d: non-finite estimator sum", s);
  }
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_get_state(pimd_batch *b, int32_t slot, double *x, double *v_nm,
                                            int64_t *step) {
  if (!b || slot < 0 || slot >= b->capacity || !b->reps[slot].live)
    return fail(PIMD_ENOTFOUND, "no replica in slot %d", slot);
  const Replica &r = b->reps[slot];
  const size_t len = (size_t)r.N * 3 * r.P;
  pimd_status st = ensure_staging(b, len);
  if (st != PIMD_OK) return st;
  BK(launch_expand_split(replica_split_args(r), r.desc.F, b->stg_x, b->stg_v, nullptr, b->stream));
  if (x) {
    BK(launch_nap_to_pna(b->stg_x, b->stg_t, r.N, r.P, b->stream));
    BK(cudaMemcpyAsync(x, b->stg_t, len * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  if (v_nm) {
    BK(launch_nap_to_pna(b->stg_v, b->stg_t, r.N, r.P, b->stream));
    BK(cudaMemcpyAsync(v_nm, b->stg_t, len * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  long long c[kCtlWords];
  BK(cudaMemcpyAsync(c, r.desc.ctl, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  if (step) *step = c[kCtlStep];
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_set_transforms(pimd_batch *b, int32_t kind) {
  if (!b || (kind != PIMD_TRANSFORMS_TENSOR && kind != PIMD_TRANSFORMS_FFMA))
    return fail(PIMD_EINVAL, "pimd_batch_set_transforms: unknown kind");
  pimd_status st = pimd_batch_sync(b);
  if (st != PIMD_OK) return st;
  const bool f = kind == PIMD_TRANSFORMS_FFMA;
  if (f == b->ffma) return PIMD_OK;
  b->ffma = f;
  for (int P = 0; P <= PIMD_MAX_BEADS; ++P) b->tileA[P] = 0;   // the tiles of the other path no longer apply
  for (int s = 0; s < b->capacity; ++s)
    if (b->reps[s].live) replica_items(b, s, b->reps[s]);
  b->dirty = true;
  return PIMD_OK;
}

extern "C" int64_t pimd_batch_kernel_launches(const pimd_batch *b) { return b ? b->launches : -1; }

// nsteps steps launched one kernel at a time with CUDA events around each of
// the four kernels of a step; ms[4] receives the summed device milliseconds
// of control, step, neighbour and force kernels.  The steps are real steps.
extern "C" pimd_status pimd_batch_time_kernels(pimd_batch *b, int32_t nsteps, double *ms) {
  if (!b || !ms || nsteps < 1) return fail(PIMD_EINVAL, "invalid argument");
  pimd_status st;
  if (b->dirty && (st = upload(b)) != PIMD_OK) return st;
  cudaEvent_t ev[5];
  for (auto &e : ev) BK(cudaEventCreate(&e));
  double acc[4] = {0, 0, 0, 0};
  for (int s = 0; s < nsteps; ++s) {
    cudaEventRecord(ev[0], b->stream);
    k_bctl<<<(b->capacity + 127) / 128, 128, 0, b->stream>>>(b->d_reps, b->capacity, 0, b->d_counts + 5);
    cudaEventRecord(ev[1], b->stream);
    launch_step_kernels(b);
    cudaEventRecord(ev[2], b->stream);
    launch_nbr_kernels(b);
    cudaEventRecord(ev[3], b->stream);
    k_bforce<<<b->grid_clu, 128, 0, b->stream>>>(b->d_reps, b->d_clu, b->d_counts + 1, 0);
    cudaEventRecord(ev[4], b->stream);
    BK(cudaEventSynchronize(ev[4]));
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      BK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      acc[k] += t;
    }
    b->launches += step_launches(b);
  }
  for (auto &e : ev) cudaEventDestroy(e);
  for (int k = 0; k < 4; ++k) ms[k] = acc[k];
  return pimd_batch_run(b, 0) == PIMD_OK ? PIMD_OK : fail(PIMD_ECUDA, "timing close failed");
}

// Autotuner of the step kernels, timed with CUDA events while the replicas
// keep stepping: for the warp-item kernel (P in {8, 16, 32, 64}, 8-atom
// tiles) the number of resident blocks per SM, which trades warps in flight
// against L1 left for the mode-matrix fragments; for every other bead count
// present the block tile A = Amax, Amax/2, ..., 1 (A atoms x 3 components x P
// modes per block).  Neither changes a replica's arithmetic, so tuning
// changes no trajectory; the tuning steps count toward the step budgets.
extern "C" pimd_status pimd_batch_autotune(pimd_batch *b, int32_t steps_per_trial, int32_t *tiles_out) {
  if (!b) return fail(PIMD_EINVAL, "batch is NULL");
  if (steps_per_trial < 1) steps_per_trial = 2;
  std::vector<int> classes;
  for (auto &r : b->reps)
    if (r.live && std::find(classes.begin(), classes.end(), r.P) == classes.end()) classes.push_back(r.P);
  std::sort(classes.begin(), classes.end());
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  auto time_step = [&](float *ms_out) -> pimd_status {
    pimd_status st;
    if (b->dirty && (st = upload(b)) != PIMD_OK) return st;
    float total = 0.f;
    for (int s = 0; s < steps_per_trial; ++s) {
      BK(launch_one_step(b, e0, e1));
      BK(cudaEventSynchronize(e1));
      float ms = 0.f;
      BK(cudaEventElapsedTime(&ms, e0, e1));
      total += ms;
    }
    b->launches += (int64_t)step_launches(b) * steps_per_trial;
    *ms_out = total;
    return PIMD_OK;
  };
  pimd_status st = PIMD_OK;
  if (!b->ffma && std::find(classes.begin(), classes.end(), 64) != classes.end()) {
    if (b->dirty && (st = upload(b)) != PIMD_OK) return st;
    int nbmax = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbmax, (const void *)k_bstep_w<false>, kWWarps * 32,
                                                      (size_t)kWWarps * b->wslot * sizeof(float)) != cudaSuccess ||
        nbmax < 1)
      nbmax = 1;
    // each candidate: one untimed step (caches and clocks settle), then the
    // faster of two timed trials; a smaller grid than the occupancy limit must
    // win by more than 3% (the timings are a few milliseconds and noisy)
    std::vector<float> tms(nbmax + 1, 1e30f);
    for (int nb = nbmax; nb >= 1 && st == PIMD_OK; --nb) {
      b->wblocks_sm = nb;
      b->grid_w = b->nsm * nb;
      if (launch_one_step(b, nullptr, nullptr) != cudaSuccess) return fail(PIMD_ECUDA, "autotune step failed");
      b->launches += step_launches(b);
      for (int rep = 0; rep < 2 && st == PIMD_OK; ++rep) {
        float ms = 0.f;
        st = time_step(&ms);
        if (st == PIMD_OK) tms[nb] = std::min(tms[nb], ms);
      }
    }
    int best = nbmax;
    for (int nb = nbmax - 1; nb >= 1; --nb)
      if (tms[nb] < 0.97f * tms[best]) best = nb;
    b->wblocks_sm = best;
    b->wtuned = best;
    b->grid_w = b->nsm * best;
    if (b->graph) {   // captured with another grid
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  for (int P : classes) {
    if (st != PIMD_OK) break;
    if (!b->ffma && (warp_class(P) || P == 128)) {   // warp items: fixed 8-atom tiles
      b->tileA[P] = kWAtoms;
      continue;
    }
    const int amax = b->ffma ? std::max(1, 256 / (3 * P)) : default_tile(P);
    int best = amax;
    float best_ms = 1e30f;
    for (int A = amax; A >= 1; A = (A == 1) ? 0 : std::max(1, A / 2)) {
      b->tileA[P] = A;
      for (int s = 0; s < b->capacity; ++s)
        if (b->reps[s].live && b->reps[s].P == P) replica_items(b, s, b->reps[s]);
      b->dirty = true;
      float ms = 0.f;
      if ((st = time_step(&ms)) != PIMD_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = A;
      }
    }
    if (st != PIMD_OK) break;
    b->tileA[P] = best;
    for (int s = 0; s < b->capacity; ++s)
      if (b->reps[s].live && b->reps[s].P == P) replica_items(b, s, b->reps[s]);
    b->dirty = true;
  }
  // finish the tuning steps: closing kick, back at integer time
  if (st == PIMD_OK) st = pimd_batch_run(b, 0);
  if (st == PIMD_OK) {
    const int cg = (b->capacity + 127) / 128;
    k_bctl<<<cg, 128, 0, b->stream>>>(b->d_reps, b->capacity, 1, nullptr);
    k_bclose<<<b->grid_step, 128, 0, b->stream>>>(b->d_reps, b->d_step, b->d_counts + 0);
    k_bctl<<<cg, 128, 0, b->stream>>>(b->d_reps, b->capacity, 2, nullptr);
    b->launches += 3;
    if (cudaGetLastError() != cudaSuccess) st = fail(PIMD_ECUDA, "autotune close failed");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tiles_out) {
    for (int P = 0; P <= PIMD_MAX_BEADS; ++P) tiles_out[P] = b->tileA[P];
    tiles_out[0] = b->wblocks_sm;   // blocks per SM of the warp-item step kernel
  }
  return st;
}

// ===========================================================================
// serving: FIFO admission by HBM budget, continuous batching, worker thread
// ===========================================================================
namespace pimd {
namespace serving {

enum JobState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

struct Job {
  uint64_t id = 0;
  int state = kQueued;
  pimd_status status = PIMD_OK;
  // copies of the submitted arrays
  int32_t n_atoms = 0, potential = 0, P = 0;
  std::vector<double> mass, pos, vel;
  double box[3] = {0, 0, 0}, ff[8] = {0};
  double T = 0, dt = 0, gamma0 = 0;
  pimd_params params{};
  int64_t nsteps = 0;
  size_t bytes = 0;
  int slot = -1;
  bool cancel = false;
  int64_t steps_seen = 0;
  pimd_estimates result{};
  double t_submit = -1, t_start = -1, t_end = -1;
  int bypassed = 0;                 // admissions of later jobs while this one waited at the head
  std::vector<double> final_x, final_v;   // kept final state (pimd_server_keep_state)
  int64_t final_step = -1;
};

// A job at the head of the queue that does not fit lets later jobs that fit
// go first, at most this many times; then admission waits for it.
constexpr int kMaxBypass = 32;

}  // namespace serving
}  // namespace pimd

struct pimd_server {
  pimd_batch *batch = nullptr;
  size_t budget = 0, used = 0;
  int64_t chunk = 100;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, pimd::serving::Job> jobs;
  uint64_t next_id = 1;
  std::thread worker;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;
  pimd_server_stats stats{};
  std::vector<int64_t> st_step, st_left;
  std::vector<pimd_estimates> est;
  bool keep_state = false;
};

namespace {

double now_s(pimd_server *s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Admit queued jobs while one fits the budget and a slot is free.  The queue
// is scanned in FIFO order and the first job that fits is admitted (a head
// job that does not fit can be passed kMaxBypass times).  Called with the
// lock held; the lock is released around pimd_batch_add, which computes the
// job's initial forces on the GPU, so submissions and polls never wait for
// device work.
void admit(pimd_server *s, std::unique_lock<std::mutex> &lk) {
  using namespace pimd::serving;
  for (;;) {
    uint64_t id = 0;
    bool found = false, head = true, head_blocked = false;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      Job &q = s->jobs[*it];
      if (q.cancel) {
        q.state = kCancelled;
        it = s->queue.erase(it);
        continue;
      }
      if (s->used + q.bytes <= s->budget) {
        id = *it;
        s->queue.erase(it);
        found = true;
        break;
      }
      if (head) {
        if (q.bypassed >= kMaxBypass) break;   // the head waits for memory; nothing passes it
        head_blocked = true;
      }
      head = false;
      ++it;
    }
    if (!found) return;
    if (head_blocked) s->jobs[s->queue.front()].bypassed++;
    Job &j = s->jobs[id];
    s->used += j.bytes;   // reserved while the job is added
    pimd_system sys;
    sys.n_atoms = j.n_atoms;
    sys.potential = j.potential;
    sys.mass = j.mass.data();
    sys.pos = j.pos.data();
    sys.vel = j.vel.empty() ? nullptr : j.vel.data();
    std::memcpy(sys.box, j.box, sizeof(sys.box));
    std::memcpy(sys.ff, j.ff, sizeof(sys.ff));
    const int32_t P = j.P;
    const double T = j.T, dt = j.dt, gamma0 = j.gamma0;
    const pimd_params prm = j.params;
    const int64_t nsteps = j.nsteps;
    int32_t slot = -1;
    lk.unlock();   // the job's arrays are only read by this thread meanwhile
    const pimd_status st = pimd_batch_add(s->batch, &sys, P, T, dt, gamma0, &prm, nsteps, &slot);
    lk.lock();
    if (st == PIMD_EBUDGET) {   // no free slot: back to the head, wait for a job to leave
      s->used -= j.bytes;
      s->queue.push_front(id);
      return;
    }
    if (st != PIMD_OK) {
      s->used -= j.bytes;
      j.state = kFailed;
      j.status = st;
      j.t_end = now_s(s);
      s->stats.failed++;
      continue;
    }
    j.state = kRunning;
    j.slot = slot;
    j.t_start = now_s(s);
  }
}

void server_loop(pimd_server *s) {
  using namespace pimd::serving;
  struct Leaving {
    uint64_t id;
    int slot;
    bool keep;
    std::vector<double> x, v;
    int64_t step;
  };
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    admit(s, lk);
    int running = 0;
    for (auto &kv : s->jobs)
      if (kv.second.state == kRunning) ++running;
    s->stats.running = running;
    s->stats.queued = (int64_t)s->queue.size();
    s->stats.bytes_in_use = s->used;
    if (!running) {
      s->cv.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    // one chunk outside the lock: submissions and polls proceed meanwhile
    lk.unlock();
    const double t_run = now_s(s);
    pimd_status st = pimd_batch_run(s->batch, s->chunk);
    if (st == PIMD_OK) st = pimd_batch_status(s->batch, s->st_step.data(), s->st_left.data(), nullptr);
    bool any_done = false;
    if (st == PIMD_OK)
      for (int k = 0; k < (int)s->st_left.size(); ++k) any_done |= (s->st_left[k] == 0);
    if (st == PIMD_OK && any_done) st = pimd_batch_estimators(s->batch, s->est.data());
    const double t_after = now_s(s);
    lk.lock();
    s->stats.chunks++;
    s->stats.gpu_busy_s += t_after - t_run;
    std::vector<Leaving> leaving;
    const bool keep = s->keep_state;
    for (auto &kv : s->jobs) {
      Job &j = kv.second;
      if (j.state != kRunning) continue;
      if (st == PIMD_OK) {
        const int64_t done = s->st_step[j.slot];
        s->stats.bead_atom_steps += (double)j.n_atoms * j.P * (double)(done - j.steps_seen);
        j.steps_seen = done;
      }
      const bool finished = st == PIMD_OK && s->st_left[j.slot] == 0;
      if (st != PIMD_OK || finished || j.cancel) {
        Leaving l;
        l.id = kv.first;
        l.slot = j.slot;
        l.keep = keep && st == PIMD_OK && finished && !j.cancel;
        l.step = -1;
        if (l.keep) {
          l.x.resize((size_t)j.P * j.n_atoms * 3);
          l.v.resize(l.x.size());
        }
        if (st != PIMD_OK) {
          j.state = kFailed;
          j.status = st;
          s->stats.failed++;
          j.t_end = t_after;
        } else if (j.cancel) {
          j.state = kCancelled;
          j.t_end = t_after;
        } else {
          j.result = s->est[j.slot];   // marked done once its memory is released
        }
        leaving.push_back(std::move(l));
      }
    }
    if (leaving.empty()) continue;
    // copies of kept states and removals outside the lock
    lk.unlock();
    for (Leaving &l : leaving) {
      if (l.keep && pimd_batch_get_state(s->batch, l.slot, l.x.data(), l.v.data(), &l.step) != PIMD_OK) {
        l.x.clear();
        l.v.clear();
        l.step = -1;
      }
      pimd_batch_remove(s->batch, l.slot);
    }
    const double t_left = now_s(s);
    lk.lock();
    for (Leaving &l : leaving) {
      Job &j = s->jobs[l.id];
      s->used -= j.bytes;
      j.slot = -1;
      if (j.state == kRunning) {
        j.state = kDone;
        j.t_end = t_left;
        s->stats.completed++;
        if (l.keep) {
          j.final_x = std::move(l.x);
          j.final_v = std::move(l.v);
          j.final_step = l.step;
        }
      }
    }
  }
}

}  // namespace

extern "C" pimd_status pimd_server_create(size_t hbm_budget_bytes, int32_t max_replicas, int64_t chunk_steps,
                                          void *stream, pimd_server **out) {
  if (!out) return fail(PIMD_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0 || chunk_steps < 1) return fail(PIMD_EINVAL, "budget and chunk must be > 0");
  pimd_server *s = new pimd_server();
  pimd_status st = pimd_batch_create(max_replicas, stream, &s->batch);
  if (st != PIMD_OK) {
    delete s;
    return st;
  }
  s->budget = hbm_budget_bytes;
  s->chunk = chunk_steps;
  s->t0 = std::chrono::steady_clock::now();
  s->st_step.assign(max_replicas, -1);
  s->st_left.assign(max_replicas, -1);
  s->est.resize(max_replicas);
  s->worker = std::thread(server_loop, s);
  *out = s;
  return PIMD_OK;
}

extern "C" void pimd_server_destroy(pimd_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  pimd_batch_destroy(s->batch);
  delete s;
}

extern "C" pimd_status pimd_batch_submit(pimd_server *s, const pimd_system *sys, int32_t P, double T, double dt,
                                         double gamma0, const pimd_params *params, int64_t nsteps,
                                         uint64_t *job) {
  using namespace pimd::serving;
  if (!s || !job) return fail(PIMD_EINVAL, "NULL argument");
  pimd_params prm;
  pimd_status st = validate_create(sys, P, T, dt, gamma0, params, &prm);
  if (st != PIMD_OK) return st;
  if ((st = require_default_keywords(prm, "the server")) != PIMD_OK) return st;
  if (sys->potential != PIMD_POT_WATERLIKE) return fail(PIMD_EINVAL, "the server runs water-like systems");
  if (nsteps < 0) return fail(PIMD_EINVAL, "nsteps must be >= 0");
  const size_t bytes = pimd_batch_replica_bytes(sys->n_atoms, P);
  if (bytes > s->budget) return fail(PIMD_EBUDGET, "job needs %zu bytes, budget is %zu", bytes, s->budget);
  Job j;
  j.n_atoms = sys->n_atoms;
  j.potential = sys->potential;
  j.P = P;
  const size_t len = (size_t)P * sys->n_atoms * 3;
  j.mass.assign(sys->mass, sys->mass + sys->n_atoms);
  j.pos.assign(sys->pos, sys->pos + len);
  if (sys->vel) j.vel.assign(sys->vel, sys->vel + len);
  std::memcpy(j.box, sys->box, sizeof(j.box));
  std::memcpy(j.ff, sys->ff, sizeof(j.ff));
  j.T = T;
  j.dt = dt;
  j.gamma0 = 0.0;
  j.params = prm;            // tau already reflects gamma0
  j.nsteps = nsteps;
  j.bytes = bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    j.id = s->next_id++;
    j.t_submit = now_s(s);
    s->jobs[j.id] = std::move(j);
    s->queue.push_back(s->next_id - 1);
    s->stats.submitted++;
    *job = s->next_id - 1;
  }
  s->cv.notify_all();
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_poll(pimd_server *s, uint64_t job, pimd_estimates *out) {
  using namespace pimd::serving;
  if (!s) return fail(PIMD_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end() || it->second.state == kCancelled) return fail(PIMD_ENOTFOUND, "unknown job %llu", (unsigned long long)job);
  const Job &j = it->second;
  if (j.state == kQueued || j.state == kRunning) return PIMD_EPENDING;
  if (j.state == kFailed) return fail(j.status, "job %llu failed", (unsigned long long)job);
  if (out) *out = j.result;
  return PIMD_OK;
}

extern "C" pimd_status pimd_batch_cancel(pimd_server *s, uint64_t job) {
  if (!s) return fail(PIMD_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return fail(PIMD_ENOTFOUND, "unknown job %llu", (unsigned long long)job);
  it->second.cancel = true;
  return PIMD_OK;
}

extern "C" pimd_status pimd_server_job_times(pimd_server *s, uint64_t job, double *submitted, double *started,
                                             double *finished) {
  if (!s) return fail(PIMD_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end()) return fail(PIMD_ENOTFOUND, "unknown job %llu", (unsigned long long)job);
  if (submitted) *submitted = it->second.t_submit;
  if (started) *started = it->second.t_start;
  if (finished) *finished = it->second.t_end;
  return PIMD_OK;
}

extern "C" pimd_status pimd_server_stats_get(pimd_server *s, pimd_server_stats *out) {
  if (!s || !out) return fail(PIMD_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return PIMD_OK;
}

extern "C" pimd_status pimd_server_keep_state(pimd_server *s, int enable) {
  if (!s) return fail(PIMD_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->keep_state = enable != 0;
  return PIMD_OK;
}

extern "C" pimd_status pimd_server_get_state(pimd_server *s, uint64_t job, double *x, double *v_nm,
                                             int64_t *step) {
  using namespace pimd::serving;
  if (!s) return fail(PIMD_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job);
  if (it == s->jobs.end() || it->second.state == kCancelled)
    return fail(PIMD_ENOTFOUND, "unknown job %llu", (unsigned long long)job);
  Job &j = it->second;
  if (j.state == kQueued || j.state == kRunning) return PIMD_EPENDING;
  if (j.state == kFailed) return fail(j.status, "job %llu failed", (unsigned long long)job);
  if (j.final_step < 0) return fail(PIMD_ENOTFOUND, "no final state kept for job %llu", (unsigned long long)job);
  const size_t n = (size_t)j.P * j.n_atoms * 3;
  if (x) std::memcpy(x, j.final_x.data(), n * sizeof(double));
  if (v_nm) std::memcpy(v_nm, j.final_v.data(), n * sizeof(double));
  if (step) *step = j.final_step;
  std::vector<double>().swap(j.final_x);
  std::vector<double>().swap(j.final_v);
  j.final_step = -1;
  return PIMD_OK;
}
