/*
 * pimd_oracle.c -- plain, slow, FP64 CPU oracle of the ring-polymer PIMD step
 * of "fix pimd/langevin" (arXiv 2602.13553).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * import this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the one thing both sides have in common is
 * the published definition of the Philox-4x32-10 generator (Salmon, Moraes,
 * Dror, Shaw, SC'11) and of the Box-Muller transform, each written here
 * independently.
 *
 * Everything is written in the paper's order and notation, with no blocking,
 * fusion or reordering: the normal-mode matrix is built as a dense P x P
 * matrix from Eq. (A1); forces are brute force over all pairs with the
 * minimum-image convention; the BAOAB / OBABO splittings of Sec. III.C are
 * applied one sub-step at a time; estimators follow App. A term by term.
 * Compiled with -ffp-contract=off so every multiply and add is a separate
 * IEEE operation.
 *
 * Units are LAMMPS "metal": Angstrom, ps, eV, amu, K.
 *
 * Array layouts (plain, C order):
 *   x, v, F  : [P][N][3]   bead (or mode) k, atom i, Cartesian component a
 *   M        : [P][P]      row = normal mode, column = bead
 *
 * Readings of the paper taken here (each is pinned by a CPU test):
 *   - Eq. (1) and App. A print "m omega_n" in the spring terms; read m omega_n^2.
 *   - K_PR (App. A) carries an extra 1/P on the spring sum; P_PR carries the 1/P
 *     and the virial term sum_k Tr Xi^(k) / P that the printed line lacks.
 *   - Eq. (A1): cos rows are 1 <= i <= floor((P-1)/2); row P/2 (P even) is the
 *     alternating row; sin rows are i > P/2, signs as printed.
 *   - The A step (Sec. IV.A defers to i-PI) is the exact harmonic flow of each
 *     free-ring-polymer mode for half a step; the centroid drifts.
 *   - App. D: c1 = exp(-dt_O / tau_k) with dt_O = h for BAOAB and h/2 for each
 *     O of OBABO; tau_0 = tau, tau_k = scale / (2 omega_k).
 *   - Boltzmann's constant is not printed; CODATA 2018 8.617333262e-5 eV/K.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Constants (metal units).  h and mvv2e are the values printed in App. C.   */
/* ------------------------------------------------------------------------ */
static const double OR_KB = 8.617333262e-5;      /* eV / K (CODATA 2018)      */
static const double OR_H = 4.135667403e-3;       /* eV ps, App. C             */
static const double OR_MVV2E = 1.0364269e-4;     /* eV / (amu A^2 ps^-2), App. C */
static const double OR_PI = 3.14159265358979323846;

void or_constants(double out[4]) {
  out[0] = OR_KB;
  out[1] = OR_H;
  out[2] = OR_H / (2.0 * OR_PI); /* hbar */
  out[3] = OR_MVV2E;
}

void or_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* App. C: de Boer quantumness  Lambda* = h / (sigma sqrt(m eps)), with the
 * mass converted to eV ps^2 / A^2 through mvv2e. */
double or_de_boer(double m_amu, double eps_ev, double sigma_a) {
  return OR_H / (sigma_a * sqrt(m_amu * OR_MVV2E * eps_ev));
}

/* ------------------------------------------------------------------------ */
/* Normal modes, App. B                                                     */
/* ------------------------------------------------------------------------ */

/* Eq. (A1): M[i][j], i = mode, j = bead. */
void or_nm_matrix(int P, double *M) {
  for (int i = 0; i < P; ++i) {
    for (int j = 0; j < P; ++j) {
      double val;
      if (i == 0) {
        val = 1.0 / sqrt((double)P);
      } else if ((P % 2 == 0) && (i == P / 2)) {
        val = ((j % 2) ? -1.0 : 1.0) / sqrt((double)P);
      } else if (i <= P / 2) {
        val = sqrt(2.0 / P) * cos(2.0 * OR_PI * i * j / P);
      } else {
        val = sqrt(2.0 / P) * sin(2.0 * OR_PI * i * j / P);
      }
      M[i * P + j] = val;
    }
  }
}

/* Eq. (A2): lambda_k = 4 sin^2(k pi / P). */
void or_mode_lambda(int P, double *lam) {
  for (int k = 0; k < P; ++k) {
    double s = sin(k * OR_PI / P);
    lam[k] = 4.0 * s * s;
  }
}

/* Eq. (2): omega_n = P / (beta hbar), beta = 1/(kB T); hbar scaled by sp
 * (the "sp" keyword of Sec. III.C). */
double or_omega_n(int P, double T, double sp) {
  double hbar = sp * OR_H / (2.0 * OR_PI);
  return P * OR_KB * T / hbar;
}

/* App. D: omega_k = sqrt(lambda_k) omega_n. */
void or_mode_omega(int P, double T, double sp, double *omega) {
  double wn = or_omega_n(P, T, sp);
  double lam[1024];
  or_mode_lambda(P, lam);
  for (int k = 0; k < P; ++k) omega[k] = sqrt(lam[k]) * wn;
}

/* ------------------------------------------------------------------------ */
/* Philox counter-based generator (Salmon et al., SC'11), written from the  */
/* published round function for word size 32 or 64:                        */
/*   (hi0,lo0) = mulhilo(M0, c0); (hi1,lo1) = mulhilo(M1, c2)               */
/*   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)                          */
/* and the key is bumped by the Weyl constants (W0, W1) between rounds.      */
/* ------------------------------------------------------------------------ */
static void or_mulhilo(int wbits, uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  if (wbits == 32) {
    uint64_t p = (a & 0xffffffffull) * (b & 0xffffffffull);
    *hi = p >> 32;
    *lo = p & 0xffffffffull;
  } else {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
  }
}

/* Generic Philox-4xW: wbits 32 or 64; ctr/key/out hold one word per element. */
void or_philox4(int wbits, int rounds, const uint64_t ctr[4], const uint64_t key[2],
                uint64_t out[4]) {
  uint64_t M0, M1, W0, W1, mask;
  if (wbits == 32) {
    M0 = 0xD2511F53ull; M1 = 0xCD9E8D57ull;
    W0 = 0x9E3779B9ull; W1 = 0xBB67AE85ull;
    mask = 0xffffffffull;
  } else {
    M0 = 0xD2E7470EE14C6C93ull; M1 = 0xCA5A826395121157ull;
    W0 = 0x9E3779B97F4A7C15ull; W1 = 0xBB67AE8584CAA73Bull;
    mask = ~0ull;
  }
  uint64_t c0 = ctr[0] & mask, c1 = ctr[1] & mask, c2 = ctr[2] & mask, c3 = ctr[3] & mask;
  uint64_t k0 = key[0] & mask, k1 = key[1] & mask;
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) { k0 = (k0 + W0) & mask; k1 = (k1 + W1) & mask; }
    uint64_t hi0, lo0, hi1, lo1;
    or_mulhilo(wbits, M0, c0, &hi0, &lo0);
    or_mulhilo(wbits, M1, c2, &hi1, &lo1);
    uint64_t n0 = (hi1 ^ c1 ^ k0) & mask;
    uint64_t n1 = lo1;
    uint64_t n2 = (hi0 ^ c3 ^ k1) & mask;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Noise keying used by the method (one Philox-4x32-10 call per draw):
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (atom, (mode & 0xffff) | (stream << 16), step low 32, step high 32)
 * The four 32-bit words w0..w3 become uniforms u = (w + 1/2) 2^-32 in (0,1);
 * Box-Muller on (u0,u1) gives (eta_x, eta_y) = r (cos, sin)(2 pi u1) with
 * r = sqrt(-2 ln u0), and on (u2,u3) eta_z = r' cos(2 pi u3).
 * Streams: 0 = O step (BAOAB, or first O of OBABO), 1 = second O of OBABO,
 *          2 = initial normal-mode velocities. */
void or_philox_words(uint64_t seed, uint32_t atom, uint32_t word1, uint64_t step,
                     uint32_t w[4]) {
  uint64_t ctr[4] = {atom, word1, step & 0xffffffffull, step >> 32};
  uint64_t key[2] = {seed & 0xffffffffull, seed >> 32};
  uint64_t out[4];
  or_philox4(32, 10, ctr, key, out);
  for (int q = 0; q < 4; ++q) w[q] = (uint32_t)out[q];
}

void or_gauss3(uint64_t seed, uint32_t atom, uint32_t mode, uint32_t stream, uint64_t step,
               double eta[3]) {
  uint32_t w[4];
  or_philox_words(seed, atom, (mode & 0xffffu) | (stream << 16), step, w);
  double u[4];
  for (int q = 0; q < 4; ++q) u[q] = ((double)w[q] + 0.5) * (1.0 / 4294967296.0);
  double r0 = sqrt(-2.0 * log(u[0]));
  double r1 = sqrt(-2.0 * log(u[2]));
  eta[0] = r0 * cos(2.0 * OR_PI * u[1]);
  eta[1] = r0 * sin(2.0 * OR_PI * u[1]);
  eta[2] = r1 * cos(2.0 * OR_PI * u[3]);
}

/* ------------------------------------------------------------------------ */
/* Forces                                                                   */
/* ------------------------------------------------------------------------ */

/* Minimum-image component: d - L * rint(d / L) (round half to even); a box
 * edge of 0 means that dimension is not periodic. */
static double or_mic(double d, double L) {
  if (L > 0.0) return d - L * nearbyint(d / L);
  return d;
}

/* Harmonic external potential U = 1/2 m omega^2 |r|^2 per atom (metal units:
 * the energy carries mvv2e).  x, F: [N][3].  *U = energy, *vir = sum r.F. */
void or_force_harmonic(int N, const double *mass, double omega, const double *x, double *F,
                       double *U, double *vir) {
  double u = 0.0, w = 0.0;
  for (int i = 0; i < N; ++i) {
    double kspring = mass[i] * OR_MVV2E * omega * omega;
    for (int a = 0; a < 3; ++a) {
      double xi = x[3 * i + a];
      F[3 * i + a] = -kspring * xi;
      u += 0.5 * kspring * xi * xi;
      w += xi * F[3 * i + a];
    }
  }
  *U = u;
  *vir = w;
}

/* Water-like flexible 3-site model (synthetic workload):
 *   atoms 3m, 3m+1, 3m+2 = O, H, H of molecule m;
 *   U = sum_bonds 1/2 kb (r - r0)^2 + sum_angles 1/2 kth (theta - th0)^2
 *     + sum_{O-O pairs, r < rc} 4 eps [(sig/r)^12 - (sig/r)^6]   (no shift)
 * ff = {kb, r0, kth, th0 (rad), eps, sig, rc}.  All pair vectors are minimum
 * image.  *vir = Tr Xi = sum over interaction terms of r_rel . f (App. A,
 * virial of the bead); vir3 (or NULL) receives the diagonal Xi_aa, summed per
 * component a (App. E, the anisotropic barostat).  x, F: [3*nmol][3]. */
void or_force_water_v(int nmol, const double box[3], const double ff[7], const double *x,
                      double *F, double *U, double *vir, double *vir3) {
  const double kb = ff[0], r0 = ff[1], kth = ff[2], th0 = ff[3];
  const double eps = ff[4], sig = ff[5], rc = ff[6];
  int N = 3 * nmol;
  for (int i = 0; i < 3 * N; ++i) F[i] = 0.0;
  double u = 0.0, w = 0.0, w3[3] = {0.0, 0.0, 0.0};
  for (int m = 0; m < nmol; ++m) {
    int o = 3 * m;
    double dv[2][3], r[2];
    for (int h = 0; h < 2; ++h) {
      int hh = o + 1 + h;
      for (int a = 0; a < 3; ++a) dv[h][a] = or_mic(x[3 * hh + a] - x[3 * o + a], box[a]);
      r[h] = sqrt(dv[h][0] * dv[h][0] + dv[h][1] * dv[h][1] + dv[h][2] * dv[h][2]);
      /* bond O-H */
      double dr = r[h] - r0;
      u += 0.5 * kb * dr * dr;
      for (int a = 0; a < 3; ++a) {
        double fa = -kb * dr * dv[h][a] / r[h]; /* force on H */
        F[3 * hh + a] += fa;
        F[3 * o + a] -= fa;
        w += dv[h][a] * fa;
        w3[a] += dv[h][a] * fa;
      }
    }
    /* angle H1-O-H2 */
    double dot = dv[0][0] * dv[1][0] + dv[0][1] * dv[1][1] + dv[0][2] * dv[1][2];
    double cth = dot / (r[0] * r[1]);
    if (cth > 1.0) cth = 1.0;
    if (cth < -1.0) cth = -1.0;
    double th = acos(cth);
    double sth = sin(th);
    double dth = th - th0;
    u += 0.5 * kth * dth * dth;
    double pref = kth * dth / sth; /* F_h = pref * d(cos theta)/d(r_h) */
    for (int h = 0; h < 2; ++h) {
      int hh = o + 1 + h;
      int g = 1 - h;
      for (int a = 0; a < 3; ++a) {
        double dcos = dv[g][a] / (r[0] * r[1]) - cth * dv[h][a] / (r[h] * r[h]);
        double fa = pref * dcos;
        F[3 * hh + a] += fa;
        F[3 * o + a] -= fa;
        w += dv[h][a] * fa;
        w3[a] += dv[h][a] * fa;
      }
    }
  }
  /* Lennard-Jones between oxygens, every pair once */
  for (int mi = 0; mi < nmol; ++mi) {
    for (int mj = mi + 1; mj < nmol; ++mj) {
      int oi = 3 * mi, oj = 3 * mj;
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = or_mic(x[3 * oj + a] - x[3 * oi + a], box[a]);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 < rc * rc) {
        double s2 = sig * sig / r2;
        double s6 = s2 * s2 * s2;
        u += 4.0 * eps * (s6 * s6 - s6);
        double fr = 24.0 * eps * (2.0 * s6 * s6 - s6) / r2; /* f_j = fr * d */
        for (int a = 0; a < 3; ++a) {
          F[3 * oj + a] += fr * d[a];
          F[3 * oi + a] -= fr * d[a];
          w += d[a] * fr * d[a];
          w3[a] += d[a] * fr * d[a];
        }
      }
    }
  }
  *U = u;
  *vir = w;
  if (vir3)
    for (int a = 0; a < 3; ++a) vir3[a] = w3[a];
}

void or_force_water(int nmol, const double box[3], const double ff[7], const double *x,
                    double *F, double *U, double *vir) {
  or_force_water_v(nmol, box, ff, x, F, U, vir, NULL);
}

/* ------------------------------------------------------------------------ */
/* The simulation state and one PIMD step (Sec. III.C keywords, Sec. IV.A)  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t N, P;
  int32_t potential;   /* 0 harmonic, 1 water-like */
  int32_t thermostat;  /* 0 none (NVE), 1 PILE_L */
  int32_t integrator;  /* 0 BAOAB, 1 OBABO */
  int32_t method;      /* 0 nmpimd (normal modes), 1 pimd (Cartesian), Sec. III.C */
  double T, dt, tau, scale, sp;
  uint64_t seed;
  double box[3];
  double ff[8];
  const double *mass;        /* [N] physical masses */
  double *x, *v, *F;         /* [P][N][3]; v: normal-mode (nmpimd) or bead (pimd) velocities */
  double *U, *vir;           /* [P] */
  int64_t step;
  int32_t fmmode;      /* 0 physical, 1 normal (Sec. III.C) */
  int32_t fixcom;      /* remove the centre-of-mass velocity every step */
  double fmass;        /* factor on the fictitious masses (Sec. III.C) */
  int32_t barostat;    /* 0 none, 1 BZP isotropic (App. E); box[] then changes */
  int32_t pad1;
  double pext;         /* target pressure (eV/A^3) */
  double taup;         /* barostat time (ps): W = 3 P N kB T taup^2 (App. A output 12) */
  double vW;           /* barostat velocity (1/ps) */
  int32_t baro_axes;   /* barostat 2 (anisotropic): axes that move, bits x = 1, y = 2, z = 4 */
  int32_t pad2;
  double vWa[3];       /* barostat 2: velocity of each axis (1/ps) */
  double vir3[3 * 128]; /* [P][3] diagonal virial Xi_aa of every bead */
} or_sim;

/* Fictitious-mass factor of mode k (nmpimd), Sec. III.C keywords fmmode and
 * fmass: m^(k) = fmass * mu_k * m with mu_k = 1 (physical) or lambda_k
 * (normal, k >= 1); the centroid keeps mu_0 = 1 since lambda_0 = 0.  The
 * Cartesian method uses fmass * m for every bead. */
static double or_mode_mu(const or_sim *s, int k) {
  if (s->method == 0 && s->fmmode == 1 && k > 0) {
    double sn = sin(OR_PI * k / s->P);
    return s->fmass * 4.0 * sn * sn;
  }
  return s->fmass;
}

/* Forces on every bead k from its own coordinates (Eq. (1): U(r^(k))). */
void or_compute_forces(or_sim *s) {
  int N = s->N, P = s->P;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < P; ++k) {
    const double *xk = s->x + (size_t)k * N * 3;
    double *Fk = s->F + (size_t)k * N * 3;
    if (s->potential == 0)
      or_force_harmonic(N, s->mass, s->ff[0], xk, Fk, &s->U[k], &s->vir[k]);
    else
      or_force_water_v(N / 3, s->box, s->ff, xk, Fk, &s->U[k], &s->vir[k], &s->vir3[3 * k]);
  }
}

/* Cartesian -> normal mode (Eq. (A1)): q[i][n][a] = sum_j M[i][j] x[j][n][a]. */
void or_to_nm(int P, int N, const double *M, const double *x, double *q) {
#pragma omp parallel for schedule(static)
  for (int n = 0; n < N; ++n)
    for (int i = 0; i < P; ++i)
      for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int j = 0; j < P; ++j) acc += M[i * P + j] * x[((size_t)j * N + n) * 3 + a];
        q[((size_t)i * N + n) * 3 + a] = acc;
      }
}

/* Normal mode -> Cartesian (Eq. (A3), M^-1 = M^T): x[j] = sum_i M[i][j] q[i]. */
void or_from_nm(int P, int N, const double *M, const double *q, double *x) {
#pragma omp parallel for schedule(static)
  for (int n = 0; n < N; ++n)
    for (int j = 0; j < P; ++j)
      for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int i = 0; i < P; ++i) acc += M[i * P + j] * q[((size_t)i * N + n) * 3 + a];
        x[((size_t)j * N + n) * 3 + a] = acc;
      }
}

/* B: v~ += tau * F~ / (m mvv2e), F~ = M F (Sec. IV.A: forces are transformed
 * to normal modes after the force evaluation). */
static void or_B(or_sim *s, const double *M, double *Ft, double tau) {
  int N = s->N, P = s->P;
  or_to_nm(P, N, M, s->F, Ft);
  for (int k = 0; k < P; ++k) {
    double mu = or_mode_mu(s, k);
    for (int n = 0; n < N; ++n)
      for (int a = 0; a < 3; ++a) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        s->v[id] += tau * Ft[id] / (s->mass[n] * mu * OR_MVV2E);
      }
  }
}

/* A: exact flow of the free ring polymer H_k = 1/2 m^(k) v~^2 + 1/2 m w_k^2 q~^2
 * for time tau, mode by mode (i-PI's equations of motion, Sec. IV.A): the
 * mode oscillates at omega[k] = w_k / sqrt(m^(k) / m) (the caller's table).
 * The centroid (w_0 = 0) drifts. */
static void or_A(or_sim *s, const double *omega, double *q, double tau) {
  int N = s->N, P = s->P;
  for (int k = 0; k < P; ++k) {
    double wk = omega[k];
    for (int n = 0; n < N; ++n)
      for (int a = 0; a < 3; ++a) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        double qq = q[id], vv = s->v[id];
        if (k == 0 && s->barostat) {
          continue;   /* or_A_baro_centroid */
        } else if (k == 0 || wk == 0.0) {
          q[id] = qq + tau * vv;
        } else {
          double c = cos(wk * tau), sn = sin(wk * tau);
          q[id] = c * qq + sn / wk * vv;
          s->v[id] = -wk * sn * qq + c * vv;
        }
      }
  }
}

/* O: PILE_L, App. D:  v~ <- c1 v~ + c2 sqrt(P kB T / (m^(k) mvv2e)) eta, with
 * tau_k = scale / (2 omega_k) for the mode's own frequency omega[k]. */
static void or_O(or_sim *s, const double *omega, double dtO, uint32_t stream) {
  int N = s->N, P = s->P;
  for (int k = 0; k < P; ++k) {
    double tauk = (k == 0) ? s->tau : s->scale / (2.0 * omega[k]);
    double c1 = exp(-dtO / tauk);
    double c2 = sqrt(1.0 - c1 * c1);
    double mu = or_mode_mu(s, k);
    for (int n = 0; n < N; ++n) {
      double eta[3];
      or_gauss3(s->seed, (uint32_t)n, (uint32_t)k, stream, (uint64_t)s->step, eta);
      double sig = sqrt(P * OR_KB * s->T / (s->mass[n] * mu * OR_MVV2E));
      for (int a = 0; a < 3; ++a) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        s->v[id] = c1 * s->v[id] + c2 * sig * eta[a];
      }
    }
  }
}

/* Draw v~ for every mode (or v for every bead, Cartesian) from
 * N(0, P kB T / (m^(k) mvv2e)) with noise stream 2 at step 0 (the ring
 * polymer is thermostatted at P T, Sec. IV.A). */
void or_thermal_velocities(or_sim *s) {
  int N = s->N, P = s->P;
  for (int k = 0; k < P; ++k)
    for (int n = 0; n < N; ++n) {
      double eta[3];
      or_gauss3(s->seed, (uint32_t)n, (uint32_t)k, 2u, 0u, eta);
      double sig = sqrt(P * OR_KB * s->T / (s->mass[n] * or_mode_mu(s, k) * OR_MVV2E));
      for (int a = 0; a < 3; ++a) s->v[((size_t)k * N + n) * 3 + a] = sig * eta[a];
    }
}

/* fixcom (Sec. III.C): subtract the mass-weighted mean velocity of the
 * centroid mode (nmpimd) or of every bead separately (pimd), once per step at
 * its end (after the closing B, and after the closing O of OBABO). */
static void or_fixcom(or_sim *s) {
  int N = s->N, P = s->P;
  int nb = s->method == 0 ? 1 : P;
  double mt = 0.0;
  for (int n = 0; n < N; ++n) mt += s->mass[n];
  for (int k = 0; k < nb; ++k) {
    double pc[3] = {0.0, 0.0, 0.0};
    for (int n = 0; n < N; ++n)
      for (int a = 0; a < 3; ++a) pc[a] += s->mass[n] * s->v[((size_t)k * N + n) * 3 + a];
    for (int n = 0; n < N; ++n)
      for (int a = 0; a < 3; ++a) s->v[((size_t)k * N + n) * 3 + a] -= pc[a] / mt;
  }
}

/* Cartesian method (Sec. III.C "method pimd"): bead velocities v, the ring
 * springs of Eq. (1) as forces, F_s^(k) = -m omega_n^2 (2 r^k - r^(k-1) -
 * r^(k+1)) (cyclic), and the bead masses fmass * m. */
static void or_B_cart(or_sim *s, double wn, double tau) {
  int N = s->N, P = s->P;
  for (int k = 0; k < P; ++k) {
    int km = (k + P - 1) % P, kp = (k + 1) % P;
    for (int n = 0; n < N; ++n) {
      double mm = s->mass[n] * OR_MVV2E;
      for (int a = 0; a < 3; ++a) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        double xk = s->x[id];
        double fs = -mm * wn * wn *
                    (2.0 * xk - s->x[((size_t)km * N + n) * 3 + a] - s->x[((size_t)kp * N + n) * 3 + a]);
        s->v[id] += tau * (s->F[id] + fs) / (mm * s->fmass);
      }
    }
  }
}

/* Cartesian A: free drift r += tau v. */
static void or_A_cart(or_sim *s, double tau) {
  size_t len = (size_t)s->P * s->N * 3;
  for (size_t id = 0; id < len; ++id) s->x[id] += tau * s->v[id];
}

/* Cartesian O (App. D): every bead with tau = scale / (2 omega_n),
 * v <- c1 v + c2 sqrt(P kB T / (fmass m mvv2e)) eta; the noise of bead k is
 * keyed like mode k of the normal-mode method. */
static void or_O_cart(or_sim *s, double wn, double dtO, uint32_t stream) {
  int N = s->N, P = s->P;
  double c1 = exp(-dtO / (s->scale / (2.0 * wn)));
  double c2 = sqrt(1.0 - c1 * c1);
  for (int k = 0; k < P; ++k)
    for (int n = 0; n < N; ++n) {
      double eta[3];
      or_gauss3(s->seed, (uint32_t)n, (uint32_t)k, stream, (uint64_t)s->step, eta);
      double sig = sqrt(P * OR_KB * s->T / (s->mass[n] * s->fmass * OR_MVV2E));
      for (int a = 0; a < 3; ++a) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        s->v[id] = c1 * s->v[id] + c2 * sig * eta[a];
      }
    }
}

/* ------------------------------------------------------------------------ */
/* BZP barostat, isotropic (App. E), acting on the centroid mode.            */
/* ------------------------------------------------------------------------ */
static double or_baro_W(const or_sim *s) {
  return 3.0 * s->P * s->N * OR_KB * s->T * s->taup * s->taup;
}

/* Sum over beads and atoms of (r - r_c) . F, r_c the bead average. */
static double or_rcF(const or_sim *s) {
  int N = s->N, P = s->P;
  double rcF = 0.0;
  for (int n = 0; n < N; ++n)
    for (int a = 0; a < 3; ++a) {
      double rc = 0.0;
      for (int k = 0; k < P; ++k) rc += s->x[((size_t)k * N + n) * 3 + a];
      rc /= P;
      for (int k = 0; k < P; ++k) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        rcF += (s->x[id] - rc) * s->F[id];
      }
    }
  return rcF;
}

/* B_W over a kick of length tB that starts from the current velocities:
 *   v_W += (3 tB / W) [n V (P_CV - P_ext) + n kB T] + (tB^2 / W) sum F~0 . v~0
 *          + (tB^3 / (3 W)) sum |F~0|^2 / m,
 * n V P_CV = (sum m |v~0|^2 - sum (r - r_c).F + sum_k Tr Xi^(k)) / 3 (output
 * 10); the tB^2 and tB^3 terms integrate the centroid kinetic pressure along
 * the kick exactly.  The printed "1/(n kB T)" is read as n kB T (an energy,
 * the volume Jacobian of J_W = -n kB T ln V). */
static void or_B_baro(or_sim *s, const double *M, double *Ft, double tB) {
  int N = s->N, P = s->P;
  or_to_nm(P, N, M, s->F, Ft);
  double mv2 = 0.0, Fv = 0.0, F2m = 0.0, vir = 0.0;
  for (int n = 0; n < N; ++n) {
    double mm = s->mass[n] * or_mode_mu(s, 0) * OR_MVV2E;
    for (int a = 0; a < 3; ++a) {
      double v0 = s->v[(size_t)n * 3 + a], f0 = Ft[(size_t)n * 3 + a];
      mv2 += mm * v0 * v0;
      Fv += f0 * v0;
      F2m += f0 * f0 / mm;
    }
  }
  for (int k = 0; k < P; ++k) vir += s->vir[k];
  double V = s->box[0] * s->box[1] * s->box[2];
  double W = or_baro_W(s);
  double nVPcv = (mv2 - or_rcF(s) + vir) / 3.0;
  s->vW += 3.0 * tB / W * (nVPcv - P * V * s->pext + P * OR_KB * s->T) + tB * tB / W * Fv +
           tB * tB * tB / (3.0 * W) * F2m;
}

/* A for the centroid under the barostat (App. E): q~0 <- e^a q~0 +
 * (e^a - e^-a) / (2 v_W) v~0, v~0 <- e^-a v~0, box <- e^a box, a = tA v_W. */
static void or_A_baro_centroid(or_sim *s, double *q, double tA) {
  int N = s->N;
  double a = tA * s->vW;
  double ea = exp(a), ema = exp(-a);
  double sh = fabs(a) < 1e-8 ? tA * (1.0 + a * a / 6.0) : (ea - ema) / (2.0 * s->vW);
  for (int n = 0; n < N; ++n)
    for (int c = 0; c < 3; ++c) {
      size_t id = (size_t)n * 3 + c;
      q[id] = ea * q[id] + sh * s->v[id];
      s->v[id] = ema * s->v[id];
    }
  for (int c = 0; c < 3; ++c) s->box[c] *= ea;
}

/* Langevin on the barostat velocity (App. E, NpT): v_W <- c1 v_W +
 * c2 sqrt(n kB T / W) eta with c1 = exp(-dtO / tau_0) (the centroid damping
 * time; the printed "m_i" under the root is read as W), eta the first
 * deviate of Philox atom 0xffffffff, stream 3, mode 0 (the O of BAOAB, the
 * first O(h/2) of OBABO) or 1 (the second O(h/2) of OBABO). */
static void or_O_baro(or_sim *s, double dtO, uint32_t mode) {
  double c1 = exp(-dtO / s->tau), c2 = sqrt(1.0 - c1 * c1);
  double eta[3];
  or_gauss3(s->seed, 0xffffffffu, mode, 3u, (uint64_t)s->step, eta);
  s->vW = c1 * s->vW + c2 * sqrt(s->P * OR_KB * s->T / or_baro_W(s)) * eta[0];
}

/* ---- anisotropic BZP barostat (App. E, "aniso" / "x" "y" "z") ---------- */
/* Each axis a in baro_axes has its own v_Wa with W = n N kB T taup^2:
 *   v_Wa += (tB / W)[n V (P_CV^aa - P_ext) + n kB T] + (tB^2 / W) sum F~0a v~0a
 *           + (tB^3 / 3W) sum F~0a^2 / m,
 *   n V P_CV^aa = sum m v~0a^2 - sum (r - r_c)_a F_a + sum_k Xi^(k)_aa,
 * the A steps scale component a of the centroid mode and L_a by
 * exp(tA v_Wa), and O draws each v_Wa from component a of the barostat's
 * deviates.  The printed 1/(n kB T) is read as n kB T, as for "iso". */
static double or_baro_Wa(const or_sim *s) {
  return s->P * s->N * OR_KB * s->T * s->taup * s->taup;
}

static void or_B_baro_aniso(or_sim *s, const double *M, double *Ft, double tB) {
  int N = s->N, P = s->P;
  or_to_nm(P, N, M, s->F, Ft);
  double W = or_baro_Wa(s), V = s->box[0] * s->box[1] * s->box[2];
  for (int a = 0; a < 3; ++a) {
    if (!(s->baro_axes >> a & 1)) continue;
    double mv2 = 0.0, Fv = 0.0, F2m = 0.0, vir = 0.0, rcF = 0.0;
    for (int n = 0; n < N; ++n) {
      double mm = s->mass[n] * or_mode_mu(s, 0) * OR_MVV2E;
      double v0 = s->v[(size_t)n * 3 + a], f0 = Ft[(size_t)n * 3 + a];
      mv2 += mm * v0 * v0;
      Fv += f0 * v0;
      F2m += f0 * f0 / mm;
      double rc = 0.0;
      for (int k = 0; k < P; ++k) rc += s->x[((size_t)k * N + n) * 3 + a];
      rc /= P;
      for (int k = 0; k < P; ++k) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        rcF += (s->x[id] - rc) * s->F[id];
      }
    }
    for (int k = 0; k < P; ++k) vir += s->vir3[3 * k + a];
    s->vWa[a] += tB / W * (mv2 - rcF + vir - P * V * s->pext + P * OR_KB * s->T) + tB * tB / W * Fv +
                 tB * tB * tB / (3.0 * W) * F2m;
  }
}

static void or_A_baro_centroid_aniso(or_sim *s, double *q, double tA) {
  int N = s->N;
  for (int c = 0; c < 3; ++c) {
    double vw = s->vWa[c];
    double a = tA * vw;
    double ea = exp(a), ema = exp(-a);
    double sh = fabs(a) < 1e-8 ? tA * (1.0 + a * a / 6.0) : (ea - ema) / (2.0 * vw);
    for (int n = 0; n < N; ++n) {
      size_t id = (size_t)n * 3 + c;
      q[id] = ea * q[id] + sh * s->v[id];
      s->v[id] = ema * s->v[id];
    }
    s->box[c] *= ea;
  }
}

static void or_O_baro_aniso(or_sim *s, double dtO, uint32_t mode) {
  double c1 = exp(-dtO / s->tau), c2 = sqrt(1.0 - c1 * c1);
  double eta[3];
  or_gauss3(s->seed, 0xffffffffu, mode, 3u, (uint64_t)s->step, eta);
  double sig = sqrt(s->P * OR_KB * s->T / or_baro_Wa(s));
  for (int a = 0; a < 3; ++a)
    if (s->baro_axes >> a & 1) s->vWa[a] = c1 * s->vWa[a] + c2 * sig * eta[a];
}

/* n steps.  BAOAB: B(h/2) A(h/2) O(h) A(h/2) [forces] B(h/2).
 *           OBABO: O(h/2) B(h/2) A(h) [forces] B(h/2) O(h/2).
 * The O sub-steps are skipped when thermostat == 0 (NVE); with fixcom the
 * centre-of-mass velocity is removed at the end of every step.  Requires F, U, vir to
 * hold the forces at x on entry (call or_compute_forces once first). */
void or_run(or_sim *s, int64_t nsteps) {
  int N = s->N, P = s->P;
  size_t len = (size_t)P * N * 3;
  double *M = (double *)malloc(sizeof(double) * P * P);
  double *omega = (double *)malloc(sizeof(double) * P);
  double *q = (double *)malloc(sizeof(double) * len);
  double *Ft = (double *)malloc(sizeof(double) * len);
  or_nm_matrix(P, M);
  or_mode_omega(P, s->T, s->sp, omega);
  for (int k = 0; k < P; ++k) omega[k] /= sqrt(or_mode_mu(s, k));   /* the mode's own frequency */
  double wn = or_omega_n(P, s->T, s->sp);
  double h = s->dt;
  for (int64_t it = 0; it < nsteps; ++it) {
    if (s->method == 1) {
      if (s->integrator == 0) {
        or_B_cart(s, wn, 0.5 * h);
        or_A_cart(s, 0.5 * h);
        if (s->thermostat) or_O_cart(s, wn, h, 0u);
        or_A_cart(s, 0.5 * h);
        or_compute_forces(s);
        or_B_cart(s, wn, 0.5 * h);
      } else {
        if (s->thermostat) or_O_cart(s, wn, 0.5 * h, 0u);
        or_B_cart(s, wn, 0.5 * h);
        or_A_cart(s, h);
        or_compute_forces(s);
        or_B_cart(s, wn, 0.5 * h);
        if (s->thermostat) or_O_cart(s, wn, 0.5 * h, 1u);
      }
    } else if (s->integrator == 0) {
      int iso = s->barostat == 1, ani = s->barostat == 2;
      if (iso) or_B_baro(s, M, Ft, 0.5 * h);
      if (ani) or_B_baro_aniso(s, M, Ft, 0.5 * h);
      or_B(s, M, Ft, 0.5 * h);
      or_to_nm(P, N, M, s->x, q);
      or_A(s, omega, q, 0.5 * h);
      if (iso) or_A_baro_centroid(s, q, 0.5 * h);
      if (ani) or_A_baro_centroid_aniso(s, q, 0.5 * h);
      if (s->thermostat) or_O(s, omega, h, 0u);
      if (s->thermostat && iso) or_O_baro(s, h, 0u);
      if (s->thermostat && ani) or_O_baro_aniso(s, h, 0u);
      or_A(s, omega, q, 0.5 * h);
      if (iso) or_A_baro_centroid(s, q, 0.5 * h);
      if (ani) or_A_baro_centroid_aniso(s, q, 0.5 * h);
      or_from_nm(P, N, M, q, s->x);
      or_compute_forces(s);
      if (iso) or_B_baro(s, M, Ft, 0.5 * h);
      if (ani) or_B_baro_aniso(s, M, Ft, 0.5 * h);
      or_B(s, M, Ft, 0.5 * h);
    } else {
      /* OBABO; with the barostat each O(h/2) also thermostats v_W, each
       * B(h/2) carries its B_W and A(h) drives the centroid and the box */
      int iso = s->barostat == 1, ani = s->barostat == 2;
      if (s->thermostat) or_O(s, omega, 0.5 * h, 0u);
      if (s->thermostat && iso) or_O_baro(s, 0.5 * h, 0u);
      if (s->thermostat && ani) or_O_baro_aniso(s, 0.5 * h, 0u);
      if (iso) or_B_baro(s, M, Ft, 0.5 * h);
      if (ani) or_B_baro_aniso(s, M, Ft, 0.5 * h);
      or_B(s, M, Ft, 0.5 * h);
      or_to_nm(P, N, M, s->x, q);
      or_A(s, omega, q, h);
      if (iso) or_A_baro_centroid(s, q, h);
      if (ani) or_A_baro_centroid_aniso(s, q, h);
      or_from_nm(P, N, M, q, s->x);
      or_compute_forces(s);
      if (iso) or_B_baro(s, M, Ft, 0.5 * h);
      if (ani) or_B_baro_aniso(s, M, Ft, 0.5 * h);
      or_B(s, M, Ft, 0.5 * h);
      if (s->thermostat) or_O(s, omega, 0.5 * h, 1u);
      if (s->thermostat && iso) or_O_baro(s, 0.5 * h, 1u);
      if (s->thermostat && ani) or_O_baro_aniso(s, 0.5 * h, 1u);
    }
    if (s->fixcom) or_fixcom(s);
    s->step += 1;
  }
  free(M); free(omega); free(q); free(Ft);
}

/* ------------------------------------------------------------------------ */
/* Estimators, App. A (outputs 1-10), at integer time                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t step;
  int32_t P, N;
  double K_mode[128], S_mode[128], U_bead[128];
  double H, K_PR, K_VR, K_CV, P_PR, P_MD, P_CV, T_ring;
  double volume, vir_sum;
  double vW, K_W, U_W, J_W, enthalpy;   /* App. A outputs 11-15 (barostat) */
  double vWa[3];                        /* output 11, anisotropic barostat */
} or_estimates;

void or_estimators(const or_sim *s, or_estimates *e) {
  int N = s->N, P = s->P;
  size_t len = (size_t)P * N * 3;
  double *M = (double *)malloc(sizeof(double) * P * P);
  double *lam = (double *)malloc(sizeof(double) * P);
  double *q = (double *)malloc(sizeof(double) * len);
  or_nm_matrix(P, M);
  or_mode_lambda(P, lam);
  or_to_nm(P, N, M, s->x, q);
  double wn = or_omega_n(P, s->T, s->sp);
  double kT = OR_KB * s->T;
  memset(e, 0, sizeof(*e));
  e->step = s->step;
  e->P = P;
  e->N = N;
  double V = s->box[0] * s->box[1] * s->box[2];
  e->volume = V;
  double Ktot = 0.0, Stot = 0.0, Utot = 0.0, virtot = 0.0;
  for (int k = 0; k < P; ++k) {
    double K = 0.0, S = 0.0;
    double mu = or_mode_mu(s, k);
    int km = (k + P - 1) % P, kp = (k + 1) % P;
    for (int n = 0; n < N; ++n) {
      double mm = s->mass[n] * OR_MVV2E;
      for (int a = 0; a < 3; ++a) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        K += 0.5 * mm * mu * s->v[id] * s->v[id];              /* output 1 */
        if (s->method == 0) {
          S += 0.5 * mm * wn * wn * lam[k] * q[id] * q[id];    /* output 2 */
        } else {                                                /* output 2, Cartesian form */
          double dm = s->x[id] - s->x[((size_t)km * N + n) * 3 + a];
          double dp = s->x[id] - s->x[((size_t)kp * N + n) * 3 + a];
          S += 0.25 * mm * wn * wn * (dm * dm + dp * dp);
        }
      }
    }
    e->K_mode[k] = K;
    e->S_mode[k] = S;
    e->U_bead[k] = s->U[k];                                     /* output 3 */
    Ktot += K;
    Stot += S;
    Utot += s->U[k];
    virtot += s->vir[k];
  }
  e->H = Ktot + Stot + Utot;                                     /* output 4 */
  /* Cartesian spring sum  sum_k sum_i m wn^2 |r^k - r^{k+1}|^2 (r^P = r^0) */
  double spring = 0.0, rF = 0.0, rcF = 0.0;
  for (int k = 0; k < P; ++k) {
    int kp = (k + 1) % P;
    for (int n = 0; n < N; ++n) {
      double mm = s->mass[n] * OR_MVV2E;
      for (int a = 0; a < 3; ++a) {
        double d = s->x[((size_t)k * N + n) * 3 + a] - s->x[((size_t)kp * N + n) * 3 + a];
        spring += mm * wn * wn * d * d;
      }
    }
  }
  for (int n = 0; n < N; ++n)
    for (int a = 0; a < 3; ++a) {
      double rc = 0.0;
      for (int k = 0; k < P; ++k) rc += s->x[((size_t)k * N + n) * 3 + a];
      rc /= P;                                                   /* centroid r^(c) */
      for (int k = 0; k < P; ++k) {
        size_t id = ((size_t)k * N + n) * 3 + a;
        rF += s->x[id] * s->F[id];
        rcF += (s->x[id] - rc) * s->F[id];
      }
    }
  /* m^(0) |v~^(0)|^2; Cartesian: v~^(0) = (1/sqrt(P)) sum_k v^(k) */
  double mv0 = 0.0, mvall = 0.0;
  double mu0 = or_mode_mu(s, 0);
  for (int n = 0; n < N; ++n) {
    double mm = s->mass[n] * OR_MVV2E * mu0;
    for (int a = 0; a < 3; ++a) {
      double v0 = 0.0;
      if (s->method == 0) {
        v0 = s->v[(size_t)n * 3 + a];
      } else {
        for (int k = 0; k < P; ++k) v0 += s->v[((size_t)k * N + n) * 3 + a];
        v0 /= sqrt((double)P);
      }
      mv0 += mm * v0 * v0;
    }
  }
  mvall = 2.0 * Ktot;
  e->K_PR = 1.5 * P * N * kT - 0.5 * spring / P;                 /* output 5 */
  e->K_VR = -rF / (2.0 * P);                                     /* output 6 */
  e->K_CV = 1.5 * N * kT - rcF / (2.0 * P);                      /* output 7 */
  if (V > 0.0) {
    e->P_PR = (3.0 * P * N * kT - spring / P + virtot / P) / (3.0 * V);   /* output 8 */
    e->P_MD = (mvall + virtot) / (3.0 * V);                                /* output 9 */
    e->P_CV = (mv0 - rcF + virtot) / (3.0 * P * V);                        /* output 10 */
  } else {
    e->P_PR = e->P_MD = e->P_CV = NAN;
  }
  e->T_ring = 2.0 * Ktot / (3.0 * N * P * OR_KB);
  e->vir_sum = virtot;
  if (s->barostat) {                                             /* outputs 11-15 */
    e->vW = s->vW;
    e->K_W = 0.5 * or_baro_W(s) * s->vW * s->vW;
    if (s->barostat == 2) {
      e->vW = 0.0;
      e->K_W = 0.0;
      for (int a = 0; a < 3; ++a) {
        e->vWa[a] = s->vWa[a];
        e->K_W += 0.5 * or_baro_Wa(s) * s->vWa[a] * s->vWa[a];
      }
    }
    e->U_W = P * s->pext * V;
    e->J_W = -P * kT * log(V);
    if (s->barostat == 2) {           /* one ln L_a per barostat axis */
      e->J_W = 0.0;
      for (int a = 0; a < 3; ++a)
        if (s->baro_axes >> a & 1) e->J_W -= P * kT * log(s->box[a]);
    }
    e->enthalpy = e->H + e->K_W + e->U_W + e->J_W;
  }
  free(M); free(lam); free(q);
}
