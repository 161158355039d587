/*
 * pimd.h -- C ABI of libpimd: ring-polymer path-integral molecular dynamics
 * (the "fix pimd/langevin" method of arXiv 2602.13553) on one NVIDIA GB300.
 *
 * The library advances N atoms x P beads with the PILE_L-thermostatted
 * normal-mode integrator of Sec. IV.A (BAOAB or OBABO splitting, Sec. III.C
 * keyword "integrator"), evaluates bead-batched forces (a harmonic external
 * well or a flexible water-like model with O-O Lennard-Jones), and reduces
 * the estimators of App. A.  Every step of that path runs in this library's
 * CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every entry point
 *   Units       LAMMPS "metal": Angstrom, ps, eV, amu, K (Sec. III.A example).
 *   Layouts     host arrays are C order [P][N][3] (bead or mode k, atom i,
 *               component a).  Positions are Cartesian and unwrapped
 *               (Sec. IV.B: every bead of an atom carries the same image);
 *               velocities are normal-mode velocities (Sec. III.A: the
 *               per-bead velocities the method reports are in the normal-mode
 *               representation).
 *   Ownership   caller buffers are read or written only during the call;
 *               device state belongs to the handle and is freed by
 *               pimd_destroy.
 *   Errors      every call returns a pimd_status and never aborts the
 *               process.  Asynchronous failures of pimd_step (a CUDA error, a
 *               neighbour-list overflow, a non-finite sum) are latched in the
 *               handle and returned by the next synchronising call
 *               (pimd_estimators, pimd_get_state, pimd_sync).
 *               pimd_last_error() gives a human-readable message for the
 *               calling thread's most recent failure.
 *   Threads     one host thread per handle at a time.  The serving entry
 *               points are internally synchronised.
 */
#ifndef PIMD_H
#define PIMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIMD_MAX_BEADS 128

typedef enum {
  PIMD_OK = 0,
  PIMD_EINVAL = 1,      /* an argument is out of range (message in pimd_last_error) */
  PIMD_ENOMEM = 2,      /* a device or host allocation failed */
  PIMD_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  PIMD_ENONFINITE = 4,  /* an estimator sum became NaN or Inf */
  PIMD_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
  PIMD_EPENDING = 6,    /* serving: the job has not finished yet */
  PIMD_ENOTFOUND = 7,   /* serving: unknown job id */
  PIMD_EBUDGET = 8,     /* serving: the job can never fit the HBM budget */
  PIMD_EOVERFLOW = 9    /* a fixed-capacity device table (neighbour list) overflowed */
} pimd_status;

/* potential energy surface U(r^(k)) of one bead (Eq. 1) */
enum { PIMD_POT_HARMONIC = 0, PIMD_POT_WATERLIKE = 1 };
/* Sec. III.C keyword "thermostat": none (NVE) or PILE_L (App. D) */
enum { PIMD_THERMO_NONE = 0, PIMD_THERMO_PILE_L = 1 };
/* Sec. III.C keyword "integrator" */
enum { PIMD_BAOAB = 0, PIMD_OBABO = 1 };
/* Sec. III.C keyword "method": nmpimd integrates in normal modes (App. B);
 * pimd integrates bead by bead in Cartesian coordinates with the ring
 * springs of Eq. (1) as forces (velocity-Verlet B and A, PILE_L O on every
 * bead with tau = scale / (2 omega_n), App. D) */
enum { PIMD_METHOD_NMPIMD = 0, PIMD_METHOD_PIMD = 1 };
/* Sec. III.C keyword "fmmode": fictitious masses of the normal modes,
 * m^(k) = m (physical) or lambda_k m (normal, k >= 1; the centroid keeps m
 * because lambda_0 = 0).  Every internal mode then oscillates at omega_n. */
enum { PIMD_FMMODE_PHYSICAL = 0, PIMD_FMMODE_NORMAL = 1 };
/* Sec. III.C keywords "barostat" / "iso" / "aniso" / "x" "y" "z", App. E:
 * none (NVE/NVT), the isotropic Bussi-Zykova-Parrinello barostat on the
 * centroid mode, or the anisotropic one (one v_W per box edge in baro_axes);
 * NpH without a thermostat, NpT with PILE_L, which also thermostats v_W. */
enum { PIMD_BARO_NONE = 0, PIMD_BARO_BZP_ISO = 1, PIMD_BARO_BZP_ANISO = 2 };
/* bits of pimd_params.baro_axes (anisotropic barostat only) */
enum { PIMD_AXIS_X = 1, PIMD_AXIS_Y = 2, PIMD_AXIS_Z = 4 };
/* arithmetic of the step and force kernels:
 *   FP64   every quantity in FP64.
 *   SPLIT  the ring-polymer centroid (position and centroid-mode velocity) in
 *          FP64; bead deviations from the centroid, internal-mode velocities,
 *          forces and the normal-mode transforms in FP32; estimator sums in
 *          FP64.  Values returned by pimd_get_state are the FP64
 *          reconstructions x = centroid + deviation. */
enum { PIMD_PREC_FP64 = 0, PIMD_PREC_SPLIT = 1 };

typedef struct pimd_handle pimd_handle;

/* The physical system.  Copied at pimd_create; the pointers are host memory.
 *   mass      [n_atoms] physical masses (amu).
 *   pos       [P][n_atoms][3] bead positions (A), unwrapped.
 *   vel       [P][n_atoms][3] velocities (A/ps) at integer time: normal-mode
 *             velocities (method nmpimd) or bead velocities (method pimd),
 *             or NULL: every mode (bead) k is then drawn from
 *             N(0, P kB T/(m^(k) mvv2e)) (the ring polymer is thermostatted
 *             at P T, Sec. IV.A) with noise stream 2 of the Philox keying
 *             described at pimd_create.
 *   potential PIMD_POT_HARMONIC: U = 1/2 m omega^2 |r|^2 per atom,
 *               ff[0] = omega (1/ps); box ignored (no pressure estimators).
 *             PIMD_POT_WATERLIKE: atoms 3m, 3m+1, 3m+2 are the O, H, H of
 *               molecule m (n_atoms a multiple of 3); ff = {kb (eV/A^2),
 *               r0 (A), kth (eV/rad^2), th0 (rad), eps (eV), sigma (A),
 *               rc (A)}; U = sum 1/2 kb (r - r0)^2 over the two O-H bonds +
 *               1/2 kth (theta - th0)^2 over H-O-H + 4 eps[(s/r)^12-(s/r)^6]
 *               over O-O pairs closer than rc (no shift), minimum image in a
 *               periodic orthorhombic box with every edge > 2 rc. */
typedef struct {
  int32_t n_atoms;
  int32_t potential;
  const double *mass;
  const double *pos;
  const double *vel;
  double box[3];
  double ff[8];
} pimd_system;

/* Method keywords (Sec. III.C).  Defaults from pimd_params_default:
 * thermostat PILE_L, integrator BAOAB, method nmpimd, seed 1, tau 1 ps,
 * scale 1, sp 1, fixcom 0 (the paper's default is "yes"; it couples
 * otherwise independent systems, so this library defaults to "no", as the
 * paper's own example input does), fmmode physical, fmass 1, precision FP64.
 *   tau     damping time of the centroid mode (ps), App. D.
 *   scale   tau_k = scale / (2 Omega_k) for k >= 1 with Omega_k the mode's own
 *           frequency omega_k / sqrt(m^(k) / m) (App. D); Cartesian method:
 *           tau = scale / (2 omega_n) for every bead.
 *   sp      hbar -> sp * hbar; only omega_n changes (Eq. 2).  Must be > 0.
 *   fixcom  1: subtract the mass-weighted mean velocity of the centroid mode
 *           (nmpimd) or of every bead (pimd) at the end of every step.
 *   fmmode  PIMD_FMMODE_PHYSICAL or PIMD_FMMODE_NORMAL (nmpimd only).
 *   fmass   > 0, multiplies every fictitious mass (m^(k) = fmass mu_k m).
 *   barostat PIMD_BARO_NONE or PIMD_BARO_BZP_ISO (App. E): every step
 *           B_W: v_W += (3 tB / W)[n V (P_CV - P_ext) + n kB T]
 *                      + (tB^2 / W) sum F~0.v~0 + (tB^3 / 3W) sum |F~0|^2 / m
 *           beside each B(tB) (exact along the kick; the printed 1/(n kB T)
 *           read as n kB T), the A steps scale the centroid mode and the box
 *           by exp(tA v_W), and with PILE_L the O step also draws
 *           v_W <- c1 v_W + c2 sqrt(n kB T / W) eta (c1 = exp(-h / tau),
 *           Philox atom 0xffffffff, mode 0, stream 3).  n = P, W = 3 P N kB T
 *           taup^2.  OBABO: each O(h/2) draws v_W with c1 = exp(-h / 2tau)
 *           (mode 0 the first, mode 1 the second), one A(h) scales by
 *           exp(h v_W).  Water-like periodic systems, method nmpimd, FP64.
 *           PIMD_BARO_BZP_ANISO: each edge a in baro_axes has its own
 *           v_Wa with W = P N kB T taup^2 and
 *             v_Wa += (tB / W)[n V (P_CV^aa - P_ext) + n kB T]
 *                     + (tB^2 / W) sum F~0a v~0a + (tB^3 / 3W) sum F~0a^2 / m,
 *           n V P_CV^aa = sum m v~0a^2 - sum (r - r_c)_a F_a + sum_k Xi^(k)_aa;
 *           the A steps scale component a of the centroid mode and L_a by
 *           exp(tA v_Wa), the O step draws v_Wa from component a of the
 *           same deviates; the other edges stay fixed.
 *   baro_axes  PIMD_AXIS_* mask, nonzero (anisotropic barostat; ignored
 *           otherwise; default all three).
 *   pext    target pressure (eV/A^3) of the barostat.
 *   taup    barostat time (ps) > 0.
 * method pimd, fmmode normal, fmass != 1, fixcom and the barostat run in FP64
 * on a single handle (EINVAL with PIMD_PREC_SPLIT and in the batch engine and
 * server). */
typedef struct {
  int32_t thermostat;
  int32_t integrator;
  int32_t method;
  int32_t precision;
  uint64_t seed;
  double tau;
  double scale;
  double sp;
  int32_t fixcom;
  int32_t fmmode;
  double fmass;
  int32_t barostat;
  int32_t baro_axes;
  double pext;
  double taup;
} pimd_params;

/* App. A outputs 1-10 at integer time, plus bookkeeping.
 *   K_mode[k]  output 1: 1/2 sum_i m^(k)_i |v~_i^(k)|^2 (eV), k < P (method
 *              pimd: 1/2 sum_i fmass m_i |v_i^(k)|^2 of bead k)
 *   S_mode[k]  output 2: 1/2 sum_i m_i omega_n^2 lambda_k |q~_i^(k)|^2 (eV),
 *              reading the printed "m omega_n" as m omega_n^2 (method pimd:
 *              the bead form 1/4 sum_i m_i omega_n^2 (|r^k - r^(k-1)|^2 +
 *              |r^k - r^(k+1)|^2))
 *   U_bead[k]  output 3: potential energy of bead k (eV)
 *   H          output 4: sum_k (K + S + U)
 *   K_PR       output 5: 3 P N kB T / 2 - (1/P) sum 1/2 m omega_n^2 |r^k - r^(k+1)|^2
 *   K_VR       output 6: -(1/2P) sum r.F
 *   K_CV       output 7: 3 N kB T / 2 - (1/2P) sum (r - r_c).F
 *   P_PR       output 8: [3 P N kB T - (1/P) sum m omega_n^2 |dr|^2 + (1/P) sum_k Tr Xi^(k)] / 3V
 *   P_MD       output 9: sum_k [sum_i m |v~^(k)|^2 + Tr Xi^(k)] / 3V
 *   P_CV       output 10: [sum_i m^(0) |v~^(0)|^2 - sum (r - r_c).F + sum_k Tr Xi^(k)] / 3PV
 *              (method pimd: v~^(0) = sum_k v^(k) / sqrt(P))
 *   T_ring     2 sum_k K^(k) / (3 N P kB): equals P T in equilibrium (Sec. IV.A)
 *   vW, K_W, U_W, J_W, enthalpy   outputs 11-15 with the barostat (zero
 *              without): v_W (1/ps), 1/2 W v_W^2, n P_ext V, -n kB T ln V and
 *              H + K_W + U_W + J_W, conserved in NpH (eV).  Anisotropic: vW
 *              is 0, K_W = sum_a 1/2 W v_Wa^2 and J_W = -n kB T sum_a ln L_a
 *              over the barostat axes
 *   box        the current box edges (A)
 *   vWa        the anisotropic barostat's v_Wa per edge (1/ps; zero otherwise)
 * Pressures are eV/A^3 (NaN without a periodic box); volume in A^3;
 * vir_sum = sum_k Tr Xi^(k) (eV). */
typedef struct {
  int64_t step;
  int32_t P;
  int32_t N;
  double K_mode[PIMD_MAX_BEADS];
  double S_mode[PIMD_MAX_BEADS];
  double U_bead[PIMD_MAX_BEADS];
  double H, K_PR, K_VR, K_CV, P_PR, P_MD, P_CV, T_ring;
  double volume, vir_sum;
  double vW, K_W, U_W, J_W, enthalpy;
  double box[3];
  double vWa[3];
} pimd_estimates;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes usable on `stream`,
 * or NULL on failure; free releases it.  With no allocator set the library
 * uses cudaMalloc / cudaFree.  Affects handles created afterwards. */
typedef void *(*pimd_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*pimd_free_fn)(void *ptr, void *stream, void *ctx);
void pimd_set_allocator(pimd_alloc_fn alloc, pimd_free_fn release, void *ctx);

void pimd_params_default(pimd_params *out);
const char *pimd_status_string(pimd_status s);
const char *pimd_last_error(void);

/* Create a handle for one ring-polymer system (Sec. III.C: "fix ... pimd/langevin").
 *   P       number of beads, 1..PIMD_MAX_BEADS.
 *   T       temperature (K) > 0; omega_n = P kB T / (sp hbar) (Eq. 2).
 *   dt      time step (ps) > 0.
 *   gamma0  centroid friction (1/ps); if > 0 it sets tau = 1/gamma0, and a
 *           params->tau that disagrees by more than 1e-12 relative is EINVAL.
 *           Pass 0 to use params->tau.
 *   params  NULL for pimd_params_default().
 *   stream  a cudaStream_t on which every kernel of this handle runs (NULL
 *           for the legacy default stream).
 * The PILE_L noise is Philox-4x32-10 (Salmon et al., SC'11) with key =
 * (seed low 32, seed high 32) and counter = (atom, (mode & 0xffff) |
 * (stream << 16), step low 32, step high 32); its four words w become
 * u = (w + 1/2) 2^-32 and Box-Muller gives (eta_x, eta_y) from (u0, u1) and
 * eta_z from (u2, u3).  Streams: 0 = O step of BAOAB and first O of OBABO,
 * 1 = second O of OBABO, 2 = initial velocities.
 * Validation (EINVAL): P outside 1..128, T <= 0, dt <= 0, n_atoms <= 0, NULL
 * mass/pos, non-positive mass, unknown potential/thermostat/integrator/
 * method/precision/fmmode, tau <= 0 or scale <= 0 with PILE_L, sp <= 0,
 * fmass <= 0, fixcom not 0 or 1, fmmode normal with method pimd, method pimd /
 * fmmode normal / fmass != 1 / fixcom with PIMD_PREC_SPLIT, water-like
 * n_atoms not a multiple of 3 or a box edge <= 2 rc.
 * Computes the forces of the initial positions before returning. */
pimd_status pimd_create(const pimd_system *sys, int32_t P, double T, double dt, double gamma0,
                        const pimd_params *params, void *stream, pimd_handle **out);

/* Advance n >= 0 time steps (asynchronous on the handle's stream).  Each
 * step is the splitting chosen at create: BAOAB = B(h/2) A(h/2) O(h) A(h/2)
 * [forces] B(h/2); OBABO = O(h/2) B(h/2) A(h) [forces] B(h/2) O(h/2), where
 * B kicks v~ with the normal-mode forces M F (Sec. IV.A), A is the exact
 * harmonic flow of each free-ring-polymer mode (i-PI's equations of motion)
 * and O is PILE_L (App. D); method pimd: B kicks the bead velocities with the
 * forces plus the ring springs, A is the free drift.  With fixcom the
 * centre-of-mass velocity is removed at the end of every step.  On return of
 * the queued work the state is at integer time. */
pimd_status pimd_step(pimd_handle *h, int64_t n);

/* Wait for the handle's queued work; returns any latched error. */
pimd_status pimd_sync(pimd_handle *h);

/* Reduce the App. A estimators of the current state on the device (one
 * fixed-order, compensated pass) and copy them to *out (host).  Synchronises
 * the handle's stream. */
pimd_status pimd_estimators(pimd_handle *h, pimd_estimates *out);

/* Copy the state to host arrays: x [P][N][3] Cartesian positions (A), v_nm
 * [P][N][3] normal-mode velocities (A/ps; bead velocities with method pimd),
 * *step the step counter.  Any of
 * the three pointers may be NULL.  Synchronises the handle's stream. */
pimd_status pimd_get_state(pimd_handle *h, double *x, double *v_nm, int64_t *step);

/* Replace the state from host arrays (layouts as pimd_get_state; both x and
 * v_nm are required) and recompute the forces.  Together with
 * pimd_get_state this is checkpoint / resume: the noise is keyed on the step
 * counter, so a resumed run continues bit for bit. */
pimd_status pimd_set_state(pimd_handle *h, const double *x, const double *v_nm, int64_t step);

/* The barostat state (App. E) for checkpoints: vW (1/ps) and box[3] (A).
 * vW points to one double (isotropic) or three, x y z (anisotropic; edges
 * outside baro_axes hold 0 and set requires 0 there).  get: either pointer
 * may be NULL; set: EINVAL without a barostat or with a box edge <= 2 rc; the
 * forces are recomputed for the new box.  Both wait for the handle's queued
 * work. */
pimd_status pimd_get_barostat(pimd_handle *h, double *vW, double *box);
pimd_status pimd_set_barostat(pimd_handle *h, const double *vW, const double *box);

/* Release the handle and its device memory (waits for its queued work). */
void pimd_destroy(pimd_handle *h);

/* ---- measurement ---------------------------------------------------------
 * Kernel kinds of one step: the fused normal-mode step, the bead-batched
 * force kernel, the neighbour-list check+build pair, the closing half-kick,
 * the two estimator passes, and bookkeeping (step counter). */
enum {
  PIMD_KIND_STEP = 0,
  PIMD_KIND_FORCE = 1,
  PIMD_KIND_NBR = 2,
  PIMD_KIND_CLOSE = 3,
  PIMD_KIND_EST = 4,
  PIMD_KIND_OTHER = 5,
  PIMD_NKINDS = 6
};

/* Enable (1) or disable (0) per-launch timing and reset its accumulators.
 * While enabled, pimd_step launches every kernel individually (no graph
 * replay) and brackets each launch with CUDA events on the handle's stream,
 * so the results are per-kernel device durations. */
pimd_status pimd_set_kernel_timing(pimd_handle *h, int enable);

/* Accumulated milliseconds and launch counts per kind (arrays of
 * PIMD_NKINDS, either may be NULL) since the last pimd_set_kernel_timing.
 * Synchronises the handle's stream. */
pimd_status pimd_kernel_times(pimd_handle *h, double *ms, int64_t *launches);

/* Number of this library's kernels the handle has enqueued so far (nodes of
 * replayed CUDA graphs included); -1 for a NULL handle. */
int64_t pimd_kernel_launches(const pimd_handle *h);

/* The PILE_L noise of App. D (eta ~ N(0, 1), independent per mode, atom and
 * step) exactly as the FP64 step kernels draw it, for checking a trajectory's
 * noise: for mode k < n_modes and atom i < n_atoms, the four Philox-4x32-10
 * words of counter (i, (k & 0xffff) | (stream << 16), step low 32, step high
 * 32) under key (seed low 32, seed high 32), and the three Box-Muller
 * deviates made from them (the keying and map described at pimd_create).
 *   words  host [n_modes][n_atoms][4] uint32, or NULL
 *   eta    host [n_modes][n_atoms][3] double, or NULL
 * EINVAL unless 1 <= n_atoms, 1 <= n_modes <= 65536, n_atoms n_modes <= 2^24
 * and stream < 65536.  Allocates and frees its own device buffers and
 * synchronises the device. */
pimd_status pimd_noise_sample(uint64_t seed, uint32_t stream, uint64_t step, int32_t n_atoms, int32_t n_modes,
                              uint32_t *words, double *eta);

/* FP64 fused multiply-add throughput of the current device in TFLOP/s (2
 * flops per FMA), measured with CUDA events over one launch of 4 blocks of
 * 256 threads per SM, each thread running eight independent chains of iters
 * FMAs (after one untimed launch): the FP64 peak the step and force kernels'
 * arithmetic is compared with.  Allocates a small device buffer and
 * synchronises the device.  EINVAL for iters < 1 or a NULL output. */
pimd_status pimd_fp64_fma_rate(int32_t iters, double *tflops);

/* ---- batches of independent systems --------------------------------------
 * A batch advances many independent water-like ring-polymer systems
 * ("replicas": their own N, P, T, masses, seed and step count) together in
 * split precision (PIMD_PREC_SPLIT arithmetic).  Each MD step of the batch
 * is a sequence of kernel launches covering every replica -- control; the
 * fused step, as one launch per class of bead count present (warp items of
 * 64 beads; of 8, 16 or 32 beads; of 128 beads; block items of any other
 * count); rebuild decision; neighbour-list rebuilds; forces -- captured once
 * in a CUDA graph and replayed; replicas can be added and removed between
 * calls, and the graph is captured again only when the set of classes
 * present changes.  Each replica stops after its own step count;
 * a replica's trajectory does not depend on which other replicas share the
 * batch.  Same units, layouts and error rules as the single-system calls. */
typedef struct pimd_batch pimd_batch;

/* Device bytes one replica of n_atoms x P occupies (0 for invalid sizes). */
size_t pimd_batch_replica_bytes(int32_t n_atoms, int32_t P);

/* Empty batch with room for max_replicas (1..65536) on `stream` (NULL: a
 * private stream). */
pimd_status pimd_batch_create(int32_t max_replicas, void *stream, pimd_batch **out);

/* Add one replica: arguments as pimd_create (water-like potential only; the
 * precision field is ignored, the batch computes in split precision), plus
 * nsteps >= 0, the number of steps it will run.  Computes its initial
 * forces; *slot receives its index.  EBUDGET when the batch is full,
 * ENOMEM when its memory cannot be allocated. */
pimd_status pimd_batch_add(pimd_batch *b, const pimd_system *sys, int32_t P, double T, double dt,
                           double gamma0, const pimd_params *params, int64_t nsteps, int32_t *slot);

/* Remove a replica and free its memory (synchronises). */
pimd_status pimd_batch_remove(pimd_batch *b, int32_t slot);

/* Advance every replica with steps left by up to nsteps steps (asynchronous);
 * afterwards every replica is at integer time. */
pimd_status pimd_batch_run(pimd_batch *b, int64_t nsteps);
pimd_status pimd_batch_sync(pimd_batch *b);

/* step[s], steps_left[s] and rebuilds[s] (neighbour-list builds so far) for
 * every slot s < max_replicas (-1 for empty slots); any array may be NULL.
 * Synchronises. */
pimd_status pimd_batch_status(pimd_batch *b, int64_t *step, int64_t *steps_left, int64_t *rebuilds);

/* App. A estimators of every slot into out[0..max_replicas) (empty slots get
 * step = -1).  Synchronises. */
pimd_status pimd_batch_estimators(pimd_batch *b, pimd_estimates *out);

/* State of one replica, as pimd_get_state. */
pimd_status pimd_batch_get_state(pimd_batch *b, int32_t slot, double *x, double *v_nm, int64_t *step);

/* Pick the step-kernel tile (atoms per block) for every bead count in the
 * batch by timing candidates with CUDA events while the replicas step
 * (steps_per_trial steps per candidate; they count toward the replicas'
 * budgets; trajectories do not depend on the tile), and the blocks per SM of
 * the 64-bead warp-item step kernel.  tiles_out, if not NULL, receives
 * PIMD_MAX_BEADS + 1 entries: [0] the 64-bead warp-item blocks per SM, [P]
 * the tile for bead count P (0 = unused; 8 for the warp-item counts). */
pimd_status pimd_batch_autotune(pimd_batch *b, int32_t steps_per_trial, int32_t *tiles_out);

/* Normal-mode transforms of the batch's step: PIMD_TRANSFORMS_TENSOR (the
 * default) runs bead counts 8, 16, 32, 64 and 128 as warp items whose
 * transforms are 3xTF32 tensor-core products; PIMD_TRANSFORMS_FFMA runs every
 * replica on the block-item kernel with FP32 fused-multiply-add transforms,
 * the comparison path for that choice.  Both compute the same split-precision
 * step (FP32-level transforms); trajectories differ by FP32 rounding.
 * Waits for queued work; step tiles return to their defaults (run
 * pimd_batch_autotune again to tune them).  EINVAL for another kind. */
enum { PIMD_TRANSFORMS_TENSOR = 0, PIMD_TRANSFORMS_FFMA = 1 };
pimd_status pimd_batch_set_transforms(pimd_batch *b, int32_t kind);

/* Kernel accounting: kernels enqueued so far (graph nodes included), and
 * nsteps real steps launched one kernel at a time with CUDA events around
 * four groups of the step's kernels: ms[0..3] receive the summed device
 * milliseconds of the control kernel, the fused-step kernels (warp items and,
 * when launched, block items), the neighbour-list kernels (rebuild decision
 * and rebuilds) and the force kernel.
 * The timed steps leave the replicas at integer time, like pimd_batch_run. */
int64_t pimd_batch_kernel_launches(const pimd_batch *b);
pimd_status pimd_batch_time_kernels(pimd_batch *b, int32_t nsteps, double *ms);
void pimd_batch_destroy(pimd_batch *b);

/* ---- serving -----------------------------------------------------------------
 * A server owns one batch and a worker thread.  Submitted jobs wait in a
 * queue; between chunks of chunk_steps MD steps the worker admits queued jobs
 * while their device memory (pimd_batch_replica_bytes) fits the HBM budget
 * and a slot is free, so jobs that arrive while others run join the running
 * batch (continuous batching); finished jobs leave it and free their memory.
 * Admission scans the queue in submission order and admits the first job
 * that fits; a job at the head that does not fit can be passed by at most 32
 * later jobs, after which admission waits until it fits.  The worker never
 * holds the server's lock during device work, so submit, poll and cancel do
 * not wait for the GPU.  All server calls are thread-safe. */
typedef struct pimd_server pimd_server;

pimd_status pimd_server_create(size_t hbm_budget_bytes, int32_t max_replicas, int64_t chunk_steps,
                               void *stream, pimd_server **out);

/* Queue a job (arguments as pimd_batch_add; the arrays are copied).  EBUDGET
 * if the job alone exceeds the budget; EINVAL for invalid arguments. */
pimd_status pimd_batch_submit(pimd_server *s, const pimd_system *sys, int32_t P, double T, double dt,
                              double gamma0, const pimd_params *params, int64_t nsteps, uint64_t *job);

/* EPENDING while the job is queued or running; PIMD_OK once done (out, if not
 * NULL, receives its final estimators); the job's own error otherwise
 * (ENOMEM, ECUDA, ...); ENOTFOUND for unknown or cancelled jobs. */
pimd_status pimd_batch_poll(pimd_server *s, uint64_t job, pimd_estimates *out);

/* Cancel a queued or running job (its memory is freed at the next chunk
 * boundary). */
pimd_status pimd_batch_cancel(pimd_server *s, uint64_t job);

/* Host wall-clock seconds (since the server was created) at which the job
 * was submitted, admitted to the GPU and finished (-1 if not yet). */
pimd_status pimd_server_job_times(pimd_server *s, uint64_t job, double *submitted, double *started,
                                  double *finished);

typedef struct {
  int64_t submitted, completed, failed, running, queued;
  size_t bytes_in_use;
  int64_t chunks;
  double bead_atom_steps;   /* total over completed chunks */
  double gpu_busy_s;        /* wall time the worker spent running chunks */
} pimd_server_stats;
pimd_status pimd_server_stats_get(pimd_server *s, pimd_server_stats *out);

/* Keep (enable = 1) or stop keeping (0) a host copy of every job's final
 * state as it finishes, for pimd_server_get_state.  Off by default: a copy
 * costs 48 P N bytes of host memory until it is fetched. */
pimd_status pimd_server_keep_state(pimd_server *s, int enable);

/* The final state of a finished job, as pimd_batch_get_state: x [P][N][3]
 * (A), v_nm [P][N][3] (A/ps), *step; any pointer may be NULL.  The copy is
 * released once fetched.  EPENDING while the job is queued or running;
 * ENOTFOUND for unknown or cancelled jobs and for jobs that finished while
 * keeping was off (or whose copy was already fetched). */
pimd_status pimd_server_get_state(pimd_server *s, uint64_t job, double *x, double *v_nm, int64_t *step);

/* Stop the worker (queued and running jobs are dropped) and free everything. */
void pimd_server_destroy(pimd_server *s);

/* ---- estimators without any allocation -----------------------------------
 * The paper has no counterpart to this entry point.  It computes the
 * estimators that pimd_estimators reports (K_mode through vir_sum), but for a
 * state held in the caller's own device buffers, and it allocates no memory
 * at all: no cudaMalloc, no cudaFree, no pinned or host heap allocation.  It
 * exists for callers that cannot let a library allocate: a host application
 * that owns a fixed device pool reserved at start-up, or a time-stepping loop
 * in which an allocation would synchronise the device and stall its other
 * streams.  Every intermediate lives in one statically sized device array of
 * 1 MiB inside this library; every GPU that loads the library holds it until
 * the process exits.
 *   x, v_nm, F  device arrays [P][N][3]: Cartesian positions (A), velocities
 *               at integer time (A/ps; normal-mode velocities for method
 *               nmpimd, bead velocities for method pimd), Cartesian forces
 *               (eV/A)
 *   mass        device [N] (amu);  U_bead device [P] (eV), bead energies
 *   vir_sum     sum_k Tr Xi^(k) (eV);  volume in A^3, 0 for no box (NaN
 *               pressures);  T (K) as at pimd_create
 *   params      the keywords the estimators depend on -- sp, method, fmmode,
 *               fmass, read as pimd_create reads them -- or NULL for the
 *               defaults (sp 1, nmpimd, fmmode physical, fmass 1); the
 *               other fields are ignored
 *   stream      cudaStream_t the kernels run on; the call waits for it
 *   out         host struct; step is set to 0; outputs 11-15, box and vWa
 *               are set to 0 (no barostat or box edges reach this call)
 * Limits: 1 <= P <= 128 and 1 <= N with 3 N P < 2^31; other sizes are
 * EINVAL, as are T <= 0, volume < 0, sp <= 0, fmass <= 0 and fmmode normal
 * with method pimd.  The call synchronises the stream and copies the result
 * into *out before it returns, so it cannot be captured into a CUDA graph.
 * The array is shared by every call on a
 * device and keeps the last call's contents; each call rewrites all it
 * reads, but calls whose kernels overlap on one GPU race and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current),
 * which loads the library's device code there if nothing has yet; make that
 * first call while no other stream of the device is capturing a graph. */
pimd_status pimd_estimators_noalloc(int32_t N, int32_t P, double T, double volume, const double *x,
                                    const double *v_nm, const double *F, const double *mass,
                                    const double *U_bead, double vir_sum, const pimd_params *params,
                                    void *stream, pimd_estimates *out);

#ifdef __cplusplus
}
#endif
#endif /* PIMD_H */
