// force.cu -- bead-batched forces U(r^(k)) of every bead k in one grid
// (Eq. 1: each bead feels the physical potential of its own copy of the
// system), FP64, plus the per-bead energy U^(k) and virial Tr Xi^(k) that the
// estimators of App. A need.
//
// Harmonic well: thread (atom i, bead k), F = -m mvv2e w^2 x.
// Water-like model: thread (molecule m, bead k); the P beads of one molecule
// sit in adjacent lanes, so each lane's gather of a neighbour's bead is a
// contiguous segment of that neighbour's bead row.  Bonds and the angle of the
// molecule are evaluated in place; O-O Lennard-Jones runs over a centroid
// neighbour list (cutoff + skin) shared by all beads.  Each molecule sums its
// full neighbour list in index order (no atomics), so forces are
// deterministic and independent of what else is on the GPU.
#include "common.cuh"

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
}

__global__ void __launch_bounds__(256) k_force_water_f64(ForceArgs a) {
  const int P = a.P;
  const int per = blockDim.x / P;                  // molecules per block
  const int m = blockIdx.x * per + threadIdx.x / P;
  const int k = threadIdx.x % P;
  double u = 0.0, w = 0.0;
  if (threadIdx.x < per * P && m < a.nmol) {
    const int o = 3 * m;
    const double L0 = a.box[0], L1 = a.box[1], L2 = a.box[2];
    const double i0 = a.invbox[0], i1 = a.invbox[1], i2 = a.invbox[2];
    const size_t so = (size_t)o * 3 * P + k;     // O, component 0, bead k
    const double xo0 = a.x[so], xo1 = a.x[so + P], xo2 = a.x[so + 2 * P];
    double dv[2][3], r[2];
    double fo0 = 0.0, fo1 = 0.0, fo2 = 0.0;
    double fh[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t sh = (size_t)(o + 1 + h) * 3 * P + k;
      dv[h][0] = mic(a.x[sh] - xo0, L0, i0);
      dv[h][1] = mic(a.x[sh + P] - xo1, L1, i1);
      dv[h][2] = mic(a.x[sh + 2 * P] - xo2, L2, i2);
      r[h] = sqrt(dv[h][0] * dv[h][0] + dv[h][1] * dv[h][1] + dv[h][2] * dv[h][2]);
      // O-H bond, U = 1/2 kb (r - r0)^2
      const double dr = r[h] - a.r0;
      u = fma(0.5 * a.kb * dr, dr, u);
      const double g = -a.kb * dr / r[h];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fh[h][c] = g * dv[h][c];
        w = fma(dv[h][c], fh[h][c], w);
      }
    }
    // H-O-H angle, U = 1/2 kth (theta - th0)^2
    const double r01 = r[0] * r[1];
    const double dot = dv[0][0] * dv[1][0] + dv[0][1] * dv[1][1] + dv[0][2] * dv[1][2];
    double cth = dot / r01;
    cth = fmin(1.0, fmax(-1.0, cth));
    const double th = acos(cth);
    const double dth = th - a.th0;
    u = fma(0.5 * a.kth * dth, dth, u);
    const double pref = a.kth * dth / sin(th);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 1 - h;
      const double inv_rh2 = 1.0 / (r[h] * r[h]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double dcos = dv[g][c] / r01 - cth * dv[h][c] * inv_rh2;
        const double fa = pref * dcos;
        fh[h][c] += fa;
        w = fma(dv[h][c], fa, w);
      }
    }
    fo0 = -(fh[0][0] + fh[1][0]);
    fo1 = -(fh[0][1] + fh[1][1]);
    fo2 = -(fh[0][2] + fh[1][2]);
    // O-O Lennard-Jones over the centroid neighbour list; each molecule takes
    // half of every pair's energy and virial.
    const double rc2 = a.rc * a.rc;
    const double sig2 = a.sig * a.sig;
    const double e4 = 4.0 * a.eps, e24 = 24.0 * a.eps;
    const int nn = a.nnbr[m];
    const int *nl = a.nbr + (size_t)m * kMaxNeighbours;
    double ulj = 0.0, wlj = 0.0;
    for (int q = 0; q < nn; ++q) {
      const int j = __ldg(nl + q);
      const size_t sj = (size_t)(3 * j) * 3 * P + k;
      const double d0 = mic(a.x[sj] - xo0, L0, i0);
      const double d1 = mic(a.x[sj + P] - xo1, L1, i1);
      const double d2 = mic(a.x[sj + 2 * P] - xo2, L2, i2);
      const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (r2 < rc2) {
        const double s2 = sig2 / r2;
        const double s6 = s2 * s2 * s2;
        ulj = fma(e4, s6 * s6 - s6, ulj);
        const double fr = e24 * (2.0 * s6 * s6 - s6) / r2;   // force on j = fr * d
        fo0 = fma(-fr, d0, fo0);
        fo1 = fma(-fr, d1, fo1);
        fo2 = fma(-fr, d2, fo2);
        wlj = fma(fr, r2, wlj);
      }
    }
    u = fma(0.5, ulj, u);
    w = fma(0.5, wlj, w);
    a.F[so] = fo0;
    a.F[so + P] = fo1;
    a.F[so + 2 * P] = fo2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t sh = (size_t)(o + 1 + h) * 3 * P + k;
      a.F[sh] = fh[h][0];
      a.F[sh + P] = fh[h][1];
      a.F[sh + 2 * P] = fh[h][2];
    }
  }
  const int groups = min(per, a.nmol - blockIdx.x * per);
  block_bead_sums(u, w, P, groups, a.Upart, a.Wpart);
}

// --- O-O neighbour list on ring-polymer centroids ---------------------------
// A pair (m, j) can interact at some bead only if its centroid distance at
// the last build was below rc + skin, as long as
//   2 max_m |c_m - c_m(build)| + 2 max_{m,k} |x_O^k - c_m| <= skin
// (triangle inequality on the minimum-image metric).  The check kernel
// evaluates the left side every step; the build kernel rebuilds when it
// exceeds the skin.

__global__ void k_nbr_check(NbrArgs a, double *ccur) {
  __shared__ double smax[256];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double val = 0.0;
  if (m < a.nmol) {
    const int P = a.P;
    const size_t so = (size_t)(3 * m) * 3 * P;
    double c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
      for (int k = 0; k < P; ++k) s += a.x[so + d * P + k];
      c[d] = s / P;
      ccur[3 * m + d] = c[d];
    }
    double dmax2 = 0.0;
    for (int k = 0; k < P; ++k) {
      const double e0 = a.x[so + k] - c[0], e1 = a.x[so + P + k] - c[1], e2 = a.x[so + 2 * P + k] - c[2];
      dmax2 = fmax(dmax2, e0 * e0 + e1 * e1 + e2 * e2);
    }
    const double g0 = c[0] - a.cref[3 * m], g1 = c[1] - a.cref[3 * m + 1], g2 = c[2] - a.cref[3 * m + 2];
    val = 2.0 * sqrt(g0 * g0 + g1 * g1 + g2 * g2) + 2.0 * sqrt(dmax2);
    if (!(val == val)) val = 1e300;   // NaN positions force a rebuild (and fail later)
  }
  smax[threadIdx.x] = val;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) a.blkmax[blockIdx.x] = smax[0];
}

__global__ void k_nbr_build(NbrArgs a, const double *ccur) {
  __shared__ int s_go;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int b = 0; b < a.nblk_check; ++b) mx = fmax(mx, a.blkmax[b]);
    s_go = a.force || (mx > a.skin);
  }
  __syncthreads();
  if (!s_go) return;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.nmol) return;
  const double c0 = ccur[3 * m], c1 = ccur[3 * m + 1], c2 = ccur[3 * m + 2];
  const double rl2 = a.rlist * a.rlist;
  int n = 0;
  int *nl = a.nbr + (size_t)m * kMaxNeighbours;
  for (int j = 0; j < a.nmol; ++j) {
    if (j == m) continue;
    const double d0 = mic(ccur[3 * j] - c0, a.box[0], a.invbox[0]);
    const double d1 = mic(ccur[3 * j + 1] - c1, a.box[1], a.invbox[1]);
    const double d2 = mic(ccur[3 * j + 2] - c2, a.box[2], a.invbox[2]);
    if (d0 * d0 + d1 * d1 + d2 * d2 < rl2) {
      if (n < kMaxNeighbours) nl[n] = j;
      ++n;
    }
  }
  if (n > kMaxNeighbours) {
    atomicOr(a.err, kErrNbrOverflow);
    n = kMaxNeighbours;
  }
  a.nnbr[m] = n;
  a.cref[3 * m] = c0;
  a.cref[3 * m + 1] = c1;
  a.cref[3 * m + 2] = c2;
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

cudaError_t launch_force_harmonic(const ForceArgs &a, cudaStream_t s) {
  k_force_harmonic_f64<<<force_blocks(a.N, a.P), force_block_threads(a.P), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_force_water(const ForceArgs &a, cudaStream_t s) {
  k_force_water_f64<<<force_blocks(a.nmol, a.P), force_block_threads(a.P), 0, s>>>(a);
  return cudaGetLastError();
}

int nbr_check_blocks(int nmol) { return (nmol + 127) / 128; }

cudaError_t launch_nbr(const NbrArgs &a, double *ccur, cudaStream_t s) {
  const int nb = nbr_check_blocks(a.nmol);
  k_nbr_check<<<nb, 128, 0, s>>>(a, ccur);
  k_nbr_build<<<nb, 128, 0, s>>>(a, ccur);
  return cudaGetLastError();
}

}  // namespace pimd
