// force.cu -- bead-batched forces U(r^(k)) of every bead k in one grid
// (Eq. 1: each bead feels the physical potential of its own copy of the
// system), FP64, plus the per-bead energy U^(k) and virial Tr Xi^(k) that the
// estimators of App. A need.
//
// Harmonic well: thread (atom i, bead k), F = -m mvv2e w^2 x.
// Water-like model: one block per (molecule, chunk of beads); the beads of the
// chunk sit in adjacent lanes, so each lane's gather of a neighbour's bead is
// a contiguous segment of that neighbour's bead row.  O-O Lennard-Jones runs
// over a centroid neighbour list (cutoff + skin) shared by all beads.  Each
// molecule sums its full neighbour list (no atomics), so forces are
// deterministic and independent of what else is on the GPU.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace pimd {

// Per-block bead sums of U and W in a fixed order: the block holds `groups`
// groups of P lanes (one atom or molecule per group).
__device__ __forceinline__ void block_bead_sums(double u, double w, int P, int groups,
                                                double *Upart, double *Wpart) {
  __shared__ double sU[256];
  __shared__ double sW[256];
  sU[threadIdx.x] = u;
  sW[threadIdx.x] = w;
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    double su = 0.0, sw = 0.0;
    for (int g = 0; g < groups; ++g) {
      su += sU[g * P + k];
      sw += sW[g * P + k];
    }
    Upart[(size_t)blockIdx.x * P + k] = su;
    Wpart[(size_t)blockIdx.x * P + k] = sw;
  }
}

__global__ void __launch_bounds__(256) k_force_harmonic_f64(ForceArgs a) {
  const int P = a.P;
  const int per = blockDim.x / P;                  // atoms per block
  const int i = blockIdx.x * per + threadIdx.x / P;
  const int k = threadIdx.x % P;
  double u = 0.0, w = 0.0;
  if (threadIdx.x < per * P && i < a.N) {
    const double ks = __ldg(a.kspring + i);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const size_t id = ((size_t)i * 3 + d) * P + k;
      const double x = a.x[id];
      const double f = -ks * x;
      a.F[id] = f;
      u = fma(0.5 * ks * x, x, u);
      w = fma(x, f, w);
    }
  }
  const int groups = min(per, a.N - blockIdx.x * per);
  block_bead_sums(u, w, P, groups, a.Upart, a.Wpart);
  if (a.step_inc && blockIdx.x == 0 && threadIdx.x == 0) *a.step_inc += 1;
}

// Water-like model, FP64.  A cluster of kForceBlocks (4) blocks x 4 warps
// serves one (molecule m, chunk of Bk = min(P, 32) beads).  Lane = (group u,
// bead kl): beads of the chunk in adjacent lanes (coalesced gathers of a
// neighbour's bead row), G = 32 / Bk groups when P < 32.  Warps s = 0 ..
// kLJWarps - 1 split the molecule's O-O neighbour list: warp s, group u owns
// bucket b = s G + u, the neighbours j with j mod (kLJWarps G) = b, in index
// order -- every lane of a warp runs the same loop (no divergent filtering),
// and because a pair's bucket depends on j alone, every sum depends only on
// the set of interacting pairs: a rebuilt list cannot change a bit.  Warp
// kLJWarps evaluates the two O-H bonds, warp kLJWarps + 1 the H-O-H angle.
// A neighbour is first tested in FP32 against (rc + 0.05 A)^2 -- a
// conservative bound, FP32 rounding of a <100 A coordinate being ~1e-5 A --
// and only survivors are evaluated in FP64 with the exact r < rc test, so the
// FP64 result is that of an all-FP64 loop; the FP32 image shift is exact for
// every pair that can be inside rc (their |d| is well below L/2).
// Reduction: warps and groups in shared memory, then the blocks of the
// cluster through distributed shared memory in rank order -- deterministic,
// no atomics, no global scratch.
// kDiag (anisotropic barostat) also accumulates the diagonal of the virial
// tensor, Xi_aa = sum d_a f_a, into W3part.
template <bool kDiag>
__global__ void __cluster_dims__(kForceBlocks, 1, 1) __launch_bounds__(128) k_force_water_f64(ForceArgs a) {
  constexpr int NC = kDiag ? 14 : 11;   // F (9), U, Tr Xi, then Xi_xx, Xi_yy, Xi_zz
  __shared__ double sacc[NC][128];
  __shared__ double gath[kForceBlocks][NC][32];   // rank 0: every block's partial sums
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
  const int s = rank * 4 + warp;     // 0..kLJWarps-1: LJ buckets; then bonds, angle
  const int u = lane / Bk, kl = lane % Bk;
  const int k = chunk * Bk + kl;
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  // the neighbour list of molecule m: the stored one, or rebuilt here when
  // this step's skin test fails (every block takes the same decision from the
  // same maxima and builds the same list into its own shared memory; the
  // cluster of chunk 0 also stores it and the new reference centroid)
  __shared__ int s_nl[kMaxNeighbours];
  __shared__ int s_off[kMaxBuckets + 1];
  __shared__ int s_go;
  __shared__ double s_mx[4][2];
  if (a.check_nbr) {
    // the step kernel's per-block maxima: every thread loads its share (one
    // 16-byte pair per block entry, all loads in flight at once), then warp
    // and block maxima
    double md = 0.0, me = 0.0;
    const double2 *bm = reinterpret_cast<const double2 *>(a.blkmax);
    int b = threadIdx.x;
    for (; b + (int)blockDim.x < a.nblk_check; b += 2 * blockDim.x) {   // two entries in flight
      const double2 e = bm[b], f = bm[b + blockDim.x];
      md = fmax(md, fmax(e.x, f.x));
      me = fmax(me, fmax(e.y, f.y));
    }
    if (b < a.nblk_check) {
      const double2 e = bm[b];
      md = fmax(md, e.x);
      me = fmax(me, e.y);
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o2));
      me = fmax(me, __shfl_xor_sync(0xffffffffu, me, o2));
    }
    if (lane == 0) {
      s_mx[warp][0] = md;
      s_mx[warp][1] = me;
    }
    __syncthreads();
    if (warp == 0) {
      md = fmax(fmax(s_mx[0][0], s_mx[1][0]), fmax(s_mx[2][0], s_mx[3][0]));
      me = fmax(fmax(s_mx[0][1], s_mx[1][1]), fmax(s_mx[2][1], s_mx[3][1]));
      int go = 2.0 * md + 2.0 * me > a.skin;
      if (go && m < a.nmol) {
        // bucket b holds the neighbours j = b mod NS in increasing j
        const bool db0 = a.dbox != nullptr;
        const double B0 = db0 ? a.dbox[0] : a.box[0], B1 = db0 ? a.dbox[1] : a.box[1], B2 = db0 ? a.dbox[2] : a.box[2];
        const double I0 = db0 ? a.dbox[3] : a.invbox[0], I1 = db0 ? a.dbox[4] : a.invbox[1];
        const double I2 = db0 ? a.dbox[5] : a.invbox[2];
        const double c0 = a.ccur[3 * m], c1 = a.ccur[3 * m + 1], c2 = a.ccur[3 * m + 2];
        const double rl2 = a.rlist * a.rlist;
        int total = 0;
        for (int b = 0; b < NS; ++b) {
          if (lane == 0) s_off[b] = total;
          for (int j0 = b; j0 < a.nmol; j0 += 32 * NS) {
            const int j = j0 + lane * NS;
            bool hit = false;
            if (j < a.nmol && j != m) {
              const double d0 = mic(a.ccur[3 * j] - c0, B0, I0);
              const double d1 = mic(a.ccur[3 * j + 1] - c1, B1, I1);
              const double d2 = mic(a.ccur[3 * j + 2] - c2, B2, I2);
              hit = d0 * d0 + d1 * d1 + d2 * d2 < rl2;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            const int pos = total + __popc(mask & ((1u << lane) - 1u));
            if (hit && pos < kMaxNeighbours) s_nl[pos] = j;
            total += __popc(mask);
          }
        }
        if (total > kMaxNeighbours) {   // report, and use an empty list
          if (lane == 0 && rank == 0 && chunk == 0) atomicOr(a.err, kErrNbrOverflow);
          for (int b = lane; b <= NS; b += 32) s_off[b] = 0;
          total = 0;
        }
        if (lane == 0) s_off[NS] = total;
        __syncwarp();
        if (rank == 0 && chunk == 0) {   // keep it for the following steps
          for (int q = lane; q < total; q += 32) a.nbr[(size_t)m * kMaxNeighbours + q] = s_nl[q];
          for (int b = lane; b <= NS; b += 32) a.nbr_off[(size_t)m * (NS + 1) + b] = s_off[b];
          if (lane < 3 && total <= kMaxNeighbours) a.cref[3 * m + lane] = a.ccur[3 * m + lane];
        }
      }
      if (lane == 0) s_go = go;
    }
    __syncthreads();
  }
  if (u < G && k < P && m < a.nmol) {
    const int o = 3 * m;
    const bool db = a.dbox != nullptr;
    const double L0 = db ? a.dbox[0] : a.box[0], L1 = db ? a.dbox[1] : a.box[1], L2 = db ? a.dbox[2] : a.box[2];
    const double i0 = db ? a.dbox[3] : a.invbox[0], i1 = db ? a.dbox[4] : a.invbox[1];
    const double i2 = db ? a.dbox[5] : a.invbox[2];
    const size_t so = (size_t)o * 3 * P + k;
    const double xo0 = a.x[so], xo1 = a.x[so + P], xo2 = a.x[so + 2 * P];
    if (s >= kLJWarps) {
      // warp kLJWarps: the two O-H bonds; warp kLJWarps + 1: the H-O-H angle
      if (u == 0) {
        double dv[2][3], r[2], ir[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const size_t sh = (size_t)(o + 1 + h) * 3 * P + k;
          dv[h][0] = mic(a.x[sh] - xo0, L0, i0);
          dv[h][1] = mic(a.x[sh + P] - xo1, L1, i1);
          dv[h][2] = mic(a.x[sh + 2 * P] - xo2, L2, i2);
          r[h] = sqrt(dv[h][0] * dv[h][0] + dv[h][1] * dv[h][1] + dv[h][2] * dv[h][2]);
          ir[h] = 1.0 / r[h];
        }
        if (s == kLJWarps) {
          // U = 1/2 kb (r - r0)^2 per bond, force on H = -kb (r - r0) d / r
          double uu = 0.0, w = 0.0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const double dr = r[h] - a.r0;
            uu = fma(0.5 * a.kb * dr, dr, uu);
            const double g = -a.kb * dr * ir[h];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const double fc = g * dv[h][c];
              acc[3 + 3 * h + c] = fc;
              acc[c] -= fc;
              w = fma(dv[h][c], fc, w);
              if (kDiag) acc[11 + c] = fma(dv[h][c], fc, acc[11 + c]);
            }
          }
          acc[9] = uu;
          acc[10] = w;
        } else {
          // U = 1/2 kth (theta - th0)^2; F_h = kth (theta - th0)/sin(theta) d cos(theta)/d r_h
          const double ir01 = ir[0] * ir[1];
          const double dot = dv[0][0] * dv[1][0] + dv[0][1] * dv[1][1] + dv[0][2] * dv[1][2];
          const double cth = fmin(1.0, fmax(-1.0, dot * ir01));
          const double th = acos(cth);
          const double dth = th - a.th0;
          // sin(acos c) = sqrt(1 - c^2): one square root on the FP64 pipe
          // in place of a sine (the H-O-H angle stays far from 0 and pi)
          const double pref = a.kth * dth / sqrt(fma(-cth, cth, 1.0));
          double w = 0.0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int g = 1 - h;
            const double ch = cth * ir[h] * ir[h];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const double fa = pref * fma(dv[g][c], ir01, -ch * dv[h][c]);
              acc[3 + 3 * h + c] = fa;
              acc[c] -= fa;
              w = fma(dv[h][c], fa, w);
              if (kDiag) acc[11 + c] = fma(dv[h][c], fa, acc[11 + c]);
            }
          }
          acc[9] = 0.5 * a.kth * dth * dth;
          acc[10] = w;
        }
      }
    } else {
    // O-O Lennard-Jones over bucket b of the neighbour list
    const int b = s * G + u;          // neighbours j with j mod (kLJWarps G) = b
    const bool own = a.check_nbr && s_go;   // rebuilt in this block's shared memory
    const int *off = own ? s_off : a.nbr_off + (size_t)m * (NS + 1);
    const int q0 = off[b], q1 = off[b + 1];
    const int *nl = own ? s_nl : a.nbr + (size_t)m * kMaxNeighbours;
    const float xf0 = a.x32[so], xf1 = a.x32[so + P], xf2 = a.x32[so + 2 * P];
    const float Lf0 = (float)L0, Lf1 = (float)L1, Lf2 = (float)L2;
    const float if0 = (float)i0, if1 = (float)i1, if2 = (float)i2;
    const float rpre = (float)(a.rc + 0.05);
    const float rpre2 = rpre * rpre;
    const double rc2 = a.rc * a.rc;
    const double sig2 = a.sig * a.sig;
    const double e4 = 4.0 * a.eps, e24 = 24.0 * a.eps;
    double f0 = 0.0, f1 = 0.0, f2 = 0.0, ulj = 0.0, wlj = 0.0;
    double wx = 0.0, wy = 0.0, wz = 0.0;
    // one candidate j from its FP32 and FP64 bead positions: the FP32
    // prefilter, then the exact FP64 cutoff test and the pair terms
    auto pair = [&](const float (&pf)[3], const double (&pd)[3]) {
      float d0f = pf[0] - xf0, d1f = pf[1] - xf1, d2f = pf[2] - xf2;
      const float n0 = rintf(d0f * if0), n1 = rintf(d1f * if1), n2 = rintf(d2f * if2);
      d0f = fmaf(-n0, Lf0, d0f);
      d1f = fmaf(-n1, Lf1, d1f);
      d2f = fmaf(-n2, Lf2, d2f);
      if (d0f * d0f + d1f * d1f + d2f * d2f >= rpre2) return;
      const double d0 = fma(-(double)n0, L0, pd[0] - xo0);
      const double d1 = fma(-(double)n1, L1, pd[1] - xo1);
      const double d2 = fma(-(double)n2, L2, pd[2] - xo2);
      const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (r2 < rc2) {
        // 1 / r2 by Newton's iteration x <- x (2 - r2 x) from the FP32
        // reciprocal: each step squares the relative error (2^-23 -> 2^-46
        // -> below FP64 rounding), two FMAs each on the FP64 pipe
        double inv = (double)__frcp_rn((float)r2);
        inv = fma(inv, fma(-r2, inv, 1.0), inv);
        inv = fma(inv, fma(-r2, inv, 1.0), inv);
        const double s2 = sig2 * inv;
        const double s6 = s2 * s2 * s2;
        ulj = fma(e4, fma(s6, s6, -s6), ulj);
        const double fr = e24 * fma(2.0 * s6, s6, -s6) * inv;   // force on j = fr * d
        f0 = fma(-fr, d0, f0);
        f1 = fma(-fr, d1, f1);
        f2 = fma(-fr, d2, f2);
        wlj = fma(fr, r2, wlj);
        if (kDiag) {
          wx = fma(fr * d0, d0, wx);
          wy = fma(fr * d1, d1, wy);
          wz = fma(fr * d2, d2, wz);
        }
      }
    };
    // four candidates per round: their indices, then their bead rows (FP32
    // and FP64), are requested before any arithmetic, so the gathers of a
    // round overlap; the candidates are then summed in list order
    int q = q0;
    for (; q + 4 <= q1; q += 4) {
      int jj[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) jj[v] = nl[q + v];
      float pf[4][3];
      double pd[4][3];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const size_t sj = (size_t)(3 * jj[v]) * 3 * P + k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pf[v][c] = __ldg(a.x32 + sj + c * P);
          pd[v][c] = a.x[sj + c * P];
        }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) pair(pf[v], pd[v]);
    }
    for (; q < q1; ++q) {
      const size_t sj = (size_t)(3 * nl[q]) * 3 * P + k;
      float pf[3];
      double pd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pf[c] = __ldg(a.x32 + sj + c * P);
        pd[c] = a.x[sj + c * P];
      }
      pair(pf, pd);
    }
    // each molecule takes half of every pair's energy and virial
    acc[0] = f0;
    acc[1] = f1;
    acc[2] = f2;
    acc[9] = 0.5 * ulj;
    acc[10] = 0.5 * wlj;
    if (kDiag) {
      acc[11] = 0.5 * wx;
      acc[12] = 0.5 * wy;
      acc[13] = 0.5 * wz;
    }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) sacc[c][threadIdx.x] = acc[c];
  __syncthreads();
  // each block's partial sums go straight into rank 0's shared memory
  // (distributed shared memory stores), so after one cluster barrier rank 0
  // sums them locally in rank order and the other blocks may exit
  for (int t = threadIdx.x; t < NC * Bk; t += blockDim.x) {
    const int comp = t / Bk, kk = t % Bk;
    double sum = 0.0;
    for (int w = 0; w < 4; ++w)
      for (int g = 0; g < G; ++g) sum += sacc[comp][w * 32 + g * Bk + kk];
    *cluster.map_shared_rank(&gath[rank][comp][kk], 0) = sum;
  }
  cluster.sync();
  if (rank == 0 && m < a.nmol) {
    for (int t = threadIdx.x; t < NC * Bk; t += blockDim.x) {
      const int comp = t / Bk, kk = t % Bk;
      const int k2 = chunk * Bk + kk;
      if (k2 >= P) continue;
      double sum = 0.0;
      for (int r = 0; r < kForceBlocks; ++r) sum += gath[r][comp][kk];
      if (comp < 9)
        a.F[(size_t)(3 * m + comp / 3) * 3 * P + (comp % 3) * P + k2] = sum;
      else if (comp == 9)
        a.Upart[(size_t)m * P + k2] = sum;
      else if (comp == 10)
        a.Wpart[(size_t)m * P + k2] = sum;
      else
        a.W3part[((size_t)m * P + k2) * 3 + (comp - 11)] = sum;
    }
    if (a.step_inc && blockIdx.x == 0 && threadIdx.x == 0) *a.step_inc += 1;
  }
}

// --- O-O neighbour list on ring-polymer centroids ---------------------------
// A pair (m, j) can interact at some bead only if its centroid distance at
// the last build was below rc + skin, as long as
//   2 max_m |c_m - c_m(build)| + 2 max_{m,k} |x_O^k - c_m| <= skin
// (triangle inequality on the minimum-image metric: a pair's bead distance
// is at least its build-time centroid distance minus both centroid drifts
// and both bead deviations).  The step kernel writes per-block maxima of the
// two terms and the current centroids; this kernel rebuilds when the bound
// exceeds the skin (or when forced), listing neighbours in index order.
__global__ void k_nbr_build(NbrArgs a, const double *ccur) {
  __shared__ double sd[128], se[128];
  __shared__ int s_go;
  double md = 0.0, me = 0.0;
  for (int b = threadIdx.x; b < a.nblk_check; b += blockDim.x) {
    md = fmax(md, a.blkmax[2 * b]);
    me = fmax(me, a.blkmax[2 * b + 1]);
  }
  sd[threadIdx.x] = md;
  se[threadIdx.x] = me;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + st]);
      se[threadIdx.x] = fmax(se[threadIdx.x], se[threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) s_go = a.force || (2.0 * sd[0] + 2.0 * se[0] > a.skin);
  __syncthreads();
  if (!s_go) return;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.nmol) return;
  const int NS = kLJWarps * a.nbr_groups;
  const double c0 = ccur[3 * m], c1 = ccur[3 * m + 1], c2 = ccur[3 * m + 2];
  const double rl2 = a.rlist * a.rlist;
  const bool db = a.dbox != nullptr;
  const double L0 = db ? a.dbox[0] : a.box[0], L1 = db ? a.dbox[1] : a.box[1], L2 = db ? a.dbox[2] : a.box[2];
  const double i0 = db ? a.dbox[3] : a.invbox[0], i1 = db ? a.dbox[4] : a.invbox[1];
  const double i2 = db ? a.dbox[5] : a.invbox[2];
  int cnt[kMaxBuckets];
  for (int b = 0; b < NS; ++b) cnt[b] = 0;
  int n = 0;
  for (int j = 0; j < a.nmol; ++j) {
    if (j == m) continue;
    const double d0 = mic(ccur[3 * j] - c0, L0, i0);
    const double d1 = mic(ccur[3 * j + 1] - c1, L1, i1);
    const double d2 = mic(ccur[3 * j + 2] - c2, L2, i2);
    if (d0 * d0 + d1 * d1 + d2 * d2 < rl2) {
      ++cnt[j % NS];
      ++n;
    }
  }
  int *off = a.nbr_off + (size_t)m * (NS + 1);
  if (n > kMaxNeighbours) {
    // leave an empty list and report: the forces of this step are incomplete
    atomicOr(a.err, kErrNbrOverflow);
    for (int b = 0; b <= NS; ++b) off[b] = 0;
    return;
  }
  int acc = 0;
  for (int b = 0; b < NS; ++b) {
    off[b] = acc;
    acc += cnt[b];
    cnt[b] = 0;
  }
  off[NS] = acc;
  int *nl = a.nbr + (size_t)m * kMaxNeighbours;
  for (int j = 0; j < a.nmol; ++j) {
    if (j == m) continue;
    const double d0 = mic(ccur[3 * j] - c0, L0, i0);
    const double d1 = mic(ccur[3 * j + 1] - c1, L1, i1);
    const double d2 = mic(ccur[3 * j + 2] - c2, L2, i2);
    if (d0 * d0 + d1 * d1 + d2 * d2 < rl2) {
      const int b = j % NS;
      nl[off[b] + cnt[b]++] = j;
    }
  }
  a.cref[3 * m] = c0;
  a.cref[3 * m + 1] = c1;
  a.cref[3 * m + 2] = c2;
}

// Centroids of the oxygens from the positions (used when the positions were
// set from outside the step kernel: create, set_state), and a forced build.
__global__ void k_centroids(NbrArgs a, double *ccur) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.nmol) return;
  const int P = a.P;
  const size_t so = (size_t)(3 * m) * 3 * P;
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int k = 0; k < P; ++k) s += a.x[so + d * P + k];
    ccur[3 * m + d] = s / P;
  }
}

// --- host launchers --------------------------------------------------------
int force_block_threads(int P) {
  // a whole number of bead groups per block, at least one warp
  int per = 128 / P;
  if (per < 1) per = 1;
  int t = per * P;
  if (t < 32) t = 32;
  return t;
}

int force_blocks(int n_groups, int P) {
  const int per = force_block_threads(P) / P;
  return (n_groups + per - 1) / per;
}

int water_force_blocks(int nmol, int P) {
  const int Bk = P < 32 ? P : 32;
  return kForceBlocks * nmol * ((P + Bk - 1) / Bk);
}

// lane groups per warp of the water force kernel: the largest power of two
// <= min(8, 32 / min(P, 32))
int water_lane_groups(int P) {
  const int Bk = P < 32 ? P : 32;
  int g = 1;
  while (2 * g <= 8 && 2 * g * Bk <= 32) g *= 2;
  return g;
}

cudaError_t launch_force_harmonic(const ForceArgs &a, cudaStream_t s) {
  k_force_harmonic_f64<<<force_blocks(a.N, a.P), force_block_threads(a.P), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_force_water(const ForceArgs &a, cudaStream_t s) {
  if (a.W3part)
    k_force_water_f64<true><<<water_force_blocks(a.nmol, a.P), 128, 0, s>>>(a);
  else
    k_force_water_f64<false><<<water_force_blocks(a.nmol, a.P), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nbr_build(const NbrArgs &a, const double *ccur, cudaStream_t s) {
  k_nbr_build<<<(a.nmol + 127) / 128, 128, 0, s>>>(a, ccur);
  return cudaGetLastError();
}

cudaError_t launch_centroids(const NbrArgs &a, double *ccur, cudaStream_t s) {
  k_centroids<<<(a.nmol + 127) / 128, 128, 0, s>>>(a, ccur);
  return cudaGetLastError();
}

}  // namespace pimd
