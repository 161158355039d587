// common.cuh -- device-side building blocks shared by the PIMD kernels:
// metal-unit constants, the Philox-4x32-10 generator, the Gaussian noise of
// the PILE_L O step, and the argument structs of every kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pimd {

// Metal units (A, ps, eV, amu, K).  h and mvv2e are the values printed in
// App. C of the paper; Boltzmann's constant (not printed) is CODATA 2018.
constexpr double kBoltzmann = 8.617333262e-5;   // eV / K
constexpr double kPlanck = 4.135667403e-3;      // eV ps
constexpr double kMvv2e = 1.0364269e-4;         // eV per amu A^2 / ps^2
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxBeads = 128;
constexpr int kMaxNeighbours = 192;     // per molecule, O-O list with skin
// The single-system water force kernels run one cluster of kForceBlocks
// blocks x 4 warps per (molecule, bead chunk): kLJWarps warps share the
// molecule's O-O neighbour list, one takes the two bonds, one the angle.
// (Two blocks per cluster -- one block per SM for a 64-molecule box, six
// list warps -- measured slower: 25.1 against 21.5 us per FP64 launch.)
constexpr int kForceBlocks = 4;
constexpr int kLJWarps = 4 * kForceBlocks - 2;   // warps sharing one molecule's O-O neighbour list
constexpr int kMaxBuckets = kLJWarps * 8;        // kLJWarps * max lane groups (8)

// Bits of the device error word (read back at synchronising calls).
enum : unsigned { kErrNbrOverflow = 1u, kErrNonFinite = 2u, kErrBoxSmall = 4u };

// Device barostat state (App. E), [kBaroWords] doubles, one v_W per box edge
// (the isotropic barostat keeps the three equal):
//   [0..2] v_W after the last completed sub-step
//   [3..5] v_W of this step's first A (after its B_W), [6..8] after its O
//   [9..11] box edges L, [12..14] 1 / L (the layout of ForceArgs::dbox)
enum { kBaroV = 0, kBaroVA1 = 3, kBaroVA2 = 6, kBaroL = 9, kBaroInvL = 12, kBaroWords = 16 };

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
//   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Noise streams of the counter's second word (bits 16..31).
enum : uint32_t { kStreamO1 = 0u, kStreamO2 = 1u, kStreamInit = 2u };

// Three standard normal deviates for (atom, normal mode, stream, step):
// counter = (atom, mode | stream << 16, step lo, step hi), key = seed;
// u = (w + 1/2) 2^-32; Box-Muller: (eta_x, eta_y) = r0 (cos, sin)(2 pi u1),
// eta_z = r1 cos(2 pi u3), r = sqrt(-2 ln u).
__device__ __forceinline__ void gauss3(uint64_t seed, uint32_t atom, uint32_t mode, uint32_t stream,
                                       uint64_t step, double &e0, double &e1, double &e2) {
  const uint4 w = philox4x32_10(
      make_uint4(atom, (mode & 0xffffu) | (stream << 16), (uint32_t)step, (uint32_t)(step >> 32)),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double s = 2.3283064365386962890625e-10;  // 2^-32
  const double u0 = ((double)w.x + 0.5) * s;
  const double u1 = ((double)w.y + 0.5) * s;
  const double u2 = ((double)w.z + 0.5) * s;
  const double u3 = ((double)w.w + 0.5) * s;
  const double r0 = sqrt(-2.0 * log(u0));
  const double r1 = sqrt(-2.0 * log(u2));
  double sn, cs;
  sincospi(2.0 * u1, &sn, &cs);
  e0 = r0 * cs;
  e1 = r0 * sn;
  e2 = r1 * cospi(2.0 * u3);
}

// One standard normal deviate of the triple above (component d = 0, 1, 2),
// computed on its own so that one thread per component needs no exchange.
__device__ __forceinline__ double gauss1(uint64_t seed, uint32_t atom, uint32_t mode, uint32_t stream,
                                         uint64_t step, int d) {
  const uint4 w = philox4x32_10(
      make_uint4(atom, (mode & 0xffffu) | (stream << 16), (uint32_t)step, (uint32_t)(step >> 32)),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double s = 2.3283064365386962890625e-10;  // 2^-32
  const uint32_t wa = d < 2 ? w.x : w.z;
  const uint32_t wb = d < 2 ? w.y : w.w;
  const double r = sqrt(-2.0 * log(((double)wa + 0.5) * s));
  const double ang = 2.0 * (((double)wb + 0.5) * s);
  return r * (d == 1 ? sinpi(ang) : cospi(ang));
}

// Compensated running sum: (s, c) holds s + c, every addition keeping its
// rounding error in c (Neumaier's variant of Kahan summation), so a sum of
// many terms carries about one rounding of the total.  Plain aggregate
// (usable in shared memory); start from CSum{0.0, 0.0}.
struct CSum {
  double s, c;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ void add(const CSum &o) {
    add(o.s);
    c += o.c;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

// Warp-wide compensated sum (fixed shuffle tree); lane 0 holds the total.
__device__ __forceinline__ CSum warp_csum(CSum v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    CSum w{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
    v.add(w);
  }
  return v;
}

// Minimum-image component (box edge L > 0; round half to even like rint).
__device__ __forceinline__ double mic(double d, double L, double invL) {
  return d - L * rint(d * invL);
}

// ---------------------------------------------------------------------------
// Kernel arguments.  Device layout of x, v, F: [N][3][P] (atom, component,
// bead/mode), i.e. every atom's P beads are contiguous per component.
// ---------------------------------------------------------------------------
struct ModeTables {
  const double *M;     // [P][P]  M[k][j]  (mode k, bead j), Eq. (A1)
  const double *Mt;    // [P][P]  Mt[j][k] = M[k][j]
  const double *cA;    // [P] cos(w_k tA)
  const double *sA;    // [P] sin(w_k tA)/w_k   (tA for k = 0)
  const double *wsA;   // [P] w_k sin(w_k tA)   (0 for k = 0)
  const double *c1;    // [P] exp(-tO / tau_k)
  const double *c2;    // [P] sqrt(1 - c1^2) / sqrt(mu_k)  (noise of mode k)
  const double *lam;   // [P] lambda_k (Eq. A2)
  const double *mu;    // [P] fictitious-mass factor mu_k: m^(k) = mu_k m (fmmode, fmass)
  const double *imu;   // [P] 1 / mu_k
  // folded transforms (H = floor(P/2)), [H + 1][P] each:
  //   Tf[i][k]: k <= H: M[k][i]; k > H: M[k][P - (H + 1 + i)] (0 past the row)
  //   Ti[i][j]: j <= H: M[i][j]; j > H: M[H + 1 + i][P - j] (0 past the modes)
  const double *Tf;
  const double *Ti;
};

struct StepArgs {
  int N, P, A;                 // atoms, beads, atoms per tile
  ModeTables mt;
  const double *inv_mm;        // [N] 1 / (m mvv2e)
  const double *sigv;          // [N] sqrt(P kB T / (m mvv2e))
  double *x;                   // [N][3][P] Cartesian positions
  double *v;                   // [N][3][P] normal-mode velocities
  const double *F;             // [N][3][P] Cartesian forces
  const int64_t *step;         // device step counter (step index of this step = *step + step_off)
  int step_off;
  float *x32;                  // [N][3][P] FP32 copy of x for the force kernel's cutoff prefilter, or null
  // water-like systems: neighbour-list skin check of the oxygens (atoms 3m)
  const double *cref;          // [nmol][3] centroids at the last list build, or null
  double *ccur;                // [nmol][3] current centroids (written)
  double *blkmax;              // [gridDim.x][2] per-block max |c - cref| and max_k |x^k - c|
  double kick;                 // B before A: h/2 (first step of a call) or h (two merged halves)
  double half;                 // h/2
  int integrator;              // 0 BAOAB, 1 OBABO
  int first;                   // OBABO: 1 if no B+O of a previous step is pending
  int thermo;                  // 1 PILE_L
  uint64_t seed;
  // Cartesian method (v holds bead velocities): springs -m w_n^2 (2 x_k -
  // x_{k-1} - x_{k+1}) join the forces, bead masses fmass m; mt.c1/c2 hold
  // the one bead friction (tau = scale / (2 w_n)) and its noise factor
  int method;                  // 0 nmpimd, 1 pimd (Cartesian)
  double ifmass;               // 1 / fmass
  double wn2;                  // omega_n^2
  const double *mass_mm;       // [N] m mvv2e
  const double *baro;          // barostat state (centroid propagation under v_W), or null
  // OBABO with the barostat runs a step in two launches around the B_W that
  // needs the velocities after the O(h/2) sub-steps: phase 1 = the previous
  // step's closing B O and this step's O (velocities only), phase 2 = B(h/2)
  // A(h) and the new positions; phase 0 = the whole step in one launch
  int phase;
  int noise_pre;               // 1: PILE_L deviates drawn once per (atom, mode) into shared memory
};

// B_W of the barostat (App. E) over a kick of length tB that starts from the
// current velocities, and, when a step follows, that step's v_W at its two A
// sub-steps (O_W in between) and the box they leave.
struct BaroArgs {
  int N, P, nmol;
  const double *x, *v, *F;     // [N][3][P]
  const double *Mt;            // [P][P]
  const double *mass_mm;       // [N] m mvv2e
  const double *Wpart;         // [nmol][P] Tr Xi rows of the force kernel
  const double *W3part;        // [nmol][P][3] diagonal Xi_aa rows (anisotropic), or null
  int axes;                    // 0: isotropic; else the mask of edges with their own v_W
  double *baro;
  double t0, tB, tA;            // the B_W covers [t0, t0 + tB] of the kick that the next kernel applies
  int step_follows;
  // OBABO: the start-of-step call first applies the opening O_W (mode 0) and
  // scales the box once by exp(tA v_W), tA = h; the end-of-step call applies
  // the closing O_W (mode 1, keyed on the step just completed) after its B_W
  int obabo;
  double W, nkT, npext, mu0;   // W (3 n N kB T taup^2, or n N kB T taup^2 per edge); n kB T; n P_ext; mu_0
  int thermo;
  double c1W, sigW;            // exp(-h / tau_0); c2 sqrt(n kB T / W)
  uint64_t seed;
  const int64_t *step;
  double Lmin;                 // smallest allowed box edge (2 rc)
  unsigned *err;
};

// fixcom: remove the centre-of-mass velocity of the centroid mode (normal
// modes) or of every bead (Cartesian) as it will stand after the closing
// B(h/2) that the next kernel applies (the removal belongs at the end of the
// step; subtracting its predicted value first is the same linear operation).
struct FixcomArgs {
  int N, P, method;
  const double *mass_mm;       // [N] m mvv2e
  const double *x, *F;         // [N][3][P]
  double *v;                   // [N][3][P]
  double half;                 // h/2
  double imu0;                 // 1 / mu_0 (normal modes) or 1 / fmass (Cartesian)
  double wn2;                  // omega_n^2 (Cartesian springs)
  // OBABO with PILE_L: the closing O(h/2) follows the kick, v <- c1 v + c2 sigv eta
  int obabo_thermo;
  uint64_t seed;
  const int64_t *step;         // device counter, already advanced past this step
  const double *c1, *c2;       // [P] O tables (c2 includes 1 / sqrt(mu_k))
  const double *sigv;          // [N] sqrt(P kB T / (m mvv2e))
};

struct ForceArgs {
  int N, P, nmol;
  const double *dbox;          // device box (barostat state at kBaroL), overriding box/invbox, or null
  const double *x;             // [N][3][P]
  const float *x32;            // [N][3][P] FP32 copy of x (water prefilter)
  int64_t *step_inc;           // if not null, block 0 advances the step counter by one
  double *F;                   // [N][3][P]
  double *Upart, *Wpart;       // [rows][P] bead sums of U and Tr Xi (rows: blocks or molecules)
  double *W3part;              // water: [nmol][P][3] diagonal Xi_aa as well, or null
  const double *kspring;       // harmonic: [N] m mvv2e omega^2
  double box[3], invbox[3];
  double kb, r0, kth, th0, eps, sig, rc;
  int *nbr;                    // [nmol][kMaxNeighbours] neighbours grouped by bucket j mod NS
  int *nbr_off;                // [nmol][NS + 1] bucket offsets into the molecule's row
  int nbr_groups;              // G: lane groups per warp; NS = kLJWarps * G buckets
  // check_nbr: the force kernel itself takes the step's rebuild decision
  // (the skin test of k_nbr_build on the step kernel's per-block maxima) and,
  // when it rebuilds, lists its molecule's neighbours before the pair loop
  int check_nbr;
  const double *blkmax;        // [nblk_check][2]
  int nblk_check;
  double skin, rlist;
  const double *ccur;          // [nmol][3] current centroids of the oxygens
  double *cref;                // [nmol][3] centroids at the last build (written on rebuild)
  unsigned *err;
};

struct NbrArgs {
  int nmol, P;
  const double *x;             // [N][3][P]
  double *cref;                // [nmol][3] centroids of the oxygens at the last build
  const double *blkmax;        // [nblk_check][2] per-block max |c - cref|, max_k |x^k - c|
  int nblk_check;
  int *nbr, *nbr_off;
  int nbr_groups;
  unsigned *err;
  double box[3], invbox[3];
  const double *dbox;          // device box (barostat state at kBaroL), overriding box/invbox, or null
  double rlist;                // rc + skin
  double skin;
  int force;                   // rebuild unconditionally
};

// Split precision (split.cu): FP64 centroid xc, v~_0 [N][3]; FP32 deviations
// d = x - xc and internal-mode velocities v~_k (k >= 1) [N][3][P]; FP32 forces.
struct SplitStepArgs {
  int N, P, A;
  const float *Mf, *Mtf;       // [P][P] FP32 copies of M and M^T
  const float *Tff, *Tif;      // [P/2 + 1][P] FP32 folded forward / inverse tables (as ModeTables::Tf, Ti)
  const float *cAf, *sAf, *wsAf, *c1f, *c2f;   // FP32 mode coefficients (k >= 1)
  double tA, c1_0, c2_0;       // centroid: drift time of one A, O coefficients
  const double *inv_mm, *sigv; // [N]
  double *xc, *v0;             // [N][3]
  float *d, *vk;               // [N][3][P]
  const float *F;              // [N][3][P]
  float *xcw;                  // [N][3] centroids wrapped into the box, FP32 (water), or null
  double box[3], invbox[3];
  const int64_t *step;
  int step_off;
  const double *cref;          // water: [nmol][3] centroids at the last list build, or null
  double *ccur;
  double *blkmax;
  double kick, half;
  int integrator, first, thermo;
  uint64_t seed;
};

struct SplitForceArgs {
  int N, P, nmol;
  const double *xc;            // [N][3]
  const float *xcw;            // [N][3] wrapped FP32 centroids (water)
  const float *d;              // [N][3][P]
  float *F;                    // [N][3][P]
  double *Upart, *Wpart;
  int64_t *step_inc;
  const double *kspring;
  double box[3], invbox[3];
  double kb, r0, kth, th0, eps, sig, rc;
  const int *nbr, *nbr_off;
  int nbr_groups;
};

struct EstArgs {
  int N, P, A;
  int method;                  // 0 nmpimd, 1 pimd (Cartesian: v holds bead velocities)
  ModeTables mt;
  const double *mass_mm;       // [N] m mvv2e
  const double *x, *v, *F;
  double wn2;                  // omega_n^2
  double *part;                // [nblk][2P + 4]
};

struct EstFinalArgs {
  int N, P, nblk_est, nblk_force;
  const double *part;          // [nblk_est][2P + 4]
  const double *Upart, *Wpart; // [nblk_force][P]
  double kT, volume, kB;
  const double *dbox;          // device box edges (barostat): volume = L0 L1 L2, or null
  double *out;                 // [3P + 12]
  unsigned *err;
};

}  // namespace pimd
