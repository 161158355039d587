// capi.cu -- host runtime behind the C ABI of include/pimd.h: validation,
// the precomputed mode tables (App. B, App. D), device memory, the launch
// sequence of a step, CUDA-graph replay of steady-state steps, and the
// estimator / state transfers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "pimd.h"
#include "runtime.h"

namespace pimd {
size_t step_smem_bytes(int A, int P);
size_t close_smem_bytes(int A, int P);
size_t est_smem_bytes(int A, int P);
cudaError_t launch_step(const StepArgs &a, int threads, cudaStream_t s);
cudaError_t launch_close(const StepArgs &a, int threads, cudaStream_t s);
cudaError_t launch_advance(int64_t *step, int n, cudaStream_t s);
cudaError_t launch_to_f32(const double *src, float *dst, size_t n, cudaStream_t s);
cudaError_t launch_thermal_v(double *v, const double *sigv, const double *imu, uint64_t seed, int N, int P,
                             cudaStream_t s);
cudaError_t launch_fixcom(const FixcomArgs &a, cudaStream_t s);
cudaError_t launch_baro_kick(const BaroArgs &a, cudaStream_t s);
cudaError_t launch_pna_to_nap(const double *src, double *dst, int N, int P, cudaStream_t s);
cudaError_t launch_nap_to_pna(const double *src, double *dst, int N, int P, cudaStream_t s);
cudaError_t launch_force_harmonic(const ForceArgs &a, cudaStream_t s);
cudaError_t launch_force_water(const ForceArgs &a, cudaStream_t s);
cudaError_t launch_nbr_build(const NbrArgs &a, const double *ccur, cudaStream_t s);
cudaError_t launch_centroids(const NbrArgs &a, double *ccur, cudaStream_t s);
cudaError_t launch_est(const EstArgs &a, int threads, cudaStream_t s);
cudaError_t launch_est_final(const EstFinalArgs &a, cudaStream_t s);
int force_blocks(int n_groups, int P);
int water_lane_groups(int P);
cudaError_t launch_step_split(const SplitStepArgs &a, int threads, cudaStream_t s);
cudaError_t launch_close_split(const SplitStepArgs &a, int threads, cudaStream_t s);
cudaError_t launch_force_split(const SplitForceArgs &a, bool water, cudaStream_t s);
cudaError_t launch_expand_split(const SplitStepArgs &a, const float *F, double *x, double *v, double *Fd,
                                cudaStream_t s);
cudaError_t launch_compress_split(const SplitStepArgs &a, const double *x, const double *v,
                                  cudaStream_t s);
}  // namespace pimd

using namespace pimd;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

namespace pimd {
pimd_status fail(pimd_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}
}  // namespace pimd

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(PIMD_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                               \
  } while (0)

extern "C" const char *pimd_last_error(void) { return g_err; }

namespace pimd {
void set_last_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace pimd

extern "C" const char *pimd_status_string(pimd_status s) {
  switch (s) {
    case PIMD_OK: return "ok";
    case PIMD_EINVAL: return "invalid argument";
    case PIMD_ENOMEM: return "out of memory";
    case PIMD_ECUDA: return "CUDA error";
    case PIMD_ENONFINITE: return "non-finite estimator";
    case PIMD_ETIMEOUT: return "device wait timed out";
    case PIMD_EPENDING: return "pending";
    case PIMD_ENOTFOUND: return "not found";
    case PIMD_EBUDGET: return "exceeds memory budget";
    case PIMD_EOVERFLOW: return "device table overflow";
  }
  return "unknown status";
}

// ---------------------------------------------------------------------------
// device allocator (optional external callbacks, e.g. a caching allocator)
// ---------------------------------------------------------------------------
static std::mutex g_alloc_mu;
static DevAllocator g_alloc;

namespace pimd {
DevAllocator current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc;
}
}  // namespace pimd

extern "C" void pimd_set_allocator(pimd_alloc_fn alloc, pimd_free_fn release, void *ctx) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.release = release;
  g_alloc.ctx = ctx;
}

extern "C" void pimd_params_default(pimd_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->thermostat = PIMD_THERMO_PILE_L;
  p->integrator = PIMD_BAOAB;
  p->method = PIMD_METHOD_NMPIMD;
  p->precision = PIMD_PREC_FP64;
  p->seed = 1;
  p->tau = 1.0;
  p->scale = 1.0;
  p->sp = 1.0;
  p->fixcom = 0;
  p->fmmode = PIMD_FMMODE_PHYSICAL;
  p->fmass = 1.0;
  p->barostat = PIMD_BARO_NONE;
  p->baro_axes = PIMD_AXIS_X | PIMD_AXIS_Y | PIMD_AXIS_Z;
  p->pext = 0.0;
  p->taup = 1.0;
}

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------
struct pimd_handle {
  int N = 0, P = 0, potential = 0, nmol = 0, integrator = 0, thermostat = 0, precision = 0;
  int method = 0, fixcom = 0, barostat = 0;
  int baro_axes = 0;          // anisotropic barostat: mask of edges with their own v_W (0: isotropic)
  double *W3part = nullptr;   // anisotropic barostat: [nmol][P][3] diagonal virial rows
  double T = 0, dt = 0, tau = 0, scale = 0, sp = 0, fmass = 1.0, pext = 0, taup = 0;
  double *baro = nullptr;     // device barostat state (kBaroWords), or null
  double h_baro[kBaroWords] = {0};
  uint64_t seed = 0;
  double box[3] = {0, 0, 0};
  double ff[8] = {0};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevAllocator alloc;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  // device state, layout [N][3][P]
  double *x = nullptr, *v = nullptr, *F = nullptr, *tmp = nullptr;
  float *x32 = nullptr;   // FP32 copy of x (water-like: the force kernel's cutoff prefilter)
  // split precision: FP64 centroids, FP32 deviations / internal modes / forces
  // (x, v, F above then only serve as FP64 staging for estimators and state copies)
  double *xc = nullptr, *v0 = nullptr;
  float *dev = nullptr, *vk = nullptr, *F32 = nullptr, *xcw = nullptr;
  float *Mf = nullptr, *Mtf = nullptr, *cAf = nullptr, *sAf = nullptr, *wsAf = nullptr;
  float *Tff = nullptr, *Tif = nullptr;   // split: FP32 folded transforms
  float *c1f = nullptr, *c2f = nullptr;
  double tA = 0.0, c1_0 = 0.0, c2_0 = 0.0;
  // split precision with 8, 16, 32, 64 or 128 beads: the warp-item step kernel
  // (tensor-core transforms) and its descriptor, tables and control words
  bool split_warp = false;
  char *sw_desc = nullptr;
  float4 *sw_frag = nullptr;
  float *sw_imf = nullptr, *sw_sgf = nullptr;
  long long *sw_ctl = nullptr;
  unsigned *sw_done = nullptr;
  double *inv_mm = nullptr, *sigv = nullptr, *mass_mm = nullptr, *kspring = nullptr;
  double *M = nullptr, *Mt = nullptr, *cA = nullptr, *sA = nullptr, *wsA = nullptr;
  double *c1 = nullptr, *c2 = nullptr, *lam = nullptr, *mu = nullptr, *imu = nullptr;
  double *Tf = nullptr, *Ti = nullptr;   // folded transforms, [P/2 + 1][P]
  double *Upart = nullptr, *Wpart = nullptr;
  int nblk_force = 0;
  double *cref = nullptr, *ccur = nullptr, *blkmax = nullptr;
  int *nbr = nullptr, *nbr_off = nullptr;
  int nbr_groups = 1;
  double *est_part = nullptr, *est_out = nullptr;
  int nblk_est = 0;
  int64_t *d_step = nullptr;
  unsigned *d_err = nullptr;
  // pinned host mirrors
  double *h_est = nullptr;
  unsigned *h_err = nullptr;
  // launch shapes
  int A_step = 1, threads_step = 32, A_est = 1, threads_est = 32;
  double wn = 0;
  double skin = 1.5, rlist = 0;
  int64_t step = 0;
  pimd_status latched = PIMD_OK;
  char latched_msg[256] = "";
  // steady-state step graph (kick = h, no pending first step)
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  int64_t graph_kernels = 0;
  bool use_graph = true;
  bool capturing = false;
  // accounting: kernels enqueued (graph nodes included) and, when enabled,
  // CUDA-event timing of every launch by kind
  int64_t launches = 0;
  bool timing = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double t_ms[PIMD_NKINDS] = {0};
  int64_t t_n[PIMD_NKINDS] = {0};
};

static pimd_status flush_timing(pimd_handle *h) {
  if (h->pending.empty()) return PIMD_OK;
  CK(cudaStreamSynchronize(h->stream));
  for (auto &p : h->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p.second.first, p.second.second));
    h->t_ms[p.first] += ms;
    h->t_n[p.first] += 1;
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  h->pending.clear();
  return PIMD_OK;
}

// Enqueue `nk` kernels of one kind through `fn`, counting them and, in timing
// mode, bracketing them with events on the handle's stream.
template <class Fn>
static pimd_status enqueue(pimd_handle *h, int kind, int nk, Fn &&fn) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool t = h->timing && !h->capturing;
  if (t) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, h->stream));
  }
  CK(fn());
  if (t) {
    CK(cudaEventRecord(e1, h->stream));
    h->pending.push_back({kind, {e0, e1}});
    if (h->pending.size() >= 4096) {
      pimd_status st = flush_timing(h);
      if (st != PIMD_OK) return st;
    }
  }
  h->launches += nk;
  return PIMD_OK;
}

namespace pimd {
void *dev_alloc(const DevAllocator &a, size_t bytes, cudaStream_t s) {
  if (a.alloc) return a.alloc(bytes, (void *)s, a.ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(const DevAllocator &a, void *p, cudaStream_t s) {
  if (!p) return;
  if (a.release)
    a.release(p, (void *)s, a.ctx);
  else
    cudaFree(p);
}
}  // namespace pimd

// Eq. (A1), with cos rows 1 <= i <= floor((P-1)/2), the alternating row at
// i = P/2 for even P, and sin rows i > P/2.
static void build_nm_matrix(int P, std::vector<double> &M) {
  M.assign((size_t)P * P, 0.0);
  const double rp = 1.0 / std::sqrt((double)P), r2p = std::sqrt(2.0 / P);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double val;
      if (i == 0)
        val = rp;
      else if (P % 2 == 0 && 2 * i == P)
        val = (j & 1) ? -rp : rp;
      else if (2 * i < P)
        val = r2p * std::cos(2.0 * kPi * (double)i * j / P);
      else
        val = r2p * std::sin(2.0 * kPi * (double)i * j / P);
      M[(size_t)i * P + j] = val;
    }
}

// Step-kernel tiles: one thread per (atom, component, mode) task, up to 256
// tasks per block; small systems use small tiles so that the grid still
// covers the 152 SMs twice where the atom count allows.
static int tile_atoms(int N, int P) {
  const int amax = std::max(1, 256 / (3 * P));
  const int want = (N + 303) / 304;
  return std::min(amax, std::max(1, want));
}

static int tile_threads(int A, int P) {
  int t = ((3 * A * P + 31) / 32) * 32;
  return std::min(256, std::max(32, t));
}

static int est_threads(int A, int P) {
  int t = ((A * P + 31) / 32) * 32;
  return std::min(256, std::max(32, t));
}

static StepArgs step_args(pimd_handle *h) {
  StepArgs a{};
  a.N = h->N;
  a.P = h->P;
  a.A = h->A_step;
  a.mt = ModeTables{h->M, h->Mt, h->cA, h->sA, h->wsA, h->c1, h->c2, h->lam, h->mu, h->imu, h->Tf, h->Ti};
  a.inv_mm = h->inv_mm;
  a.sigv = h->sigv;
  a.x = h->x;
  a.v = h->v;
  a.F = h->F;
  a.method = h->method;
  a.ifmass = 1.0 / h->fmass;
  a.wn2 = h->wn * h->wn;
  a.mass_mm = h->mass_mm;
  a.baro = h->baro;
  a.phase = 0;
  a.step = h->d_step;
  a.step_off = 0;
  const bool water = h->potential == PIMD_POT_WATERLIKE;
  a.x32 = water ? h->x32 : nullptr;
  a.cref = water ? h->cref : nullptr;
  a.ccur = water ? h->ccur : nullptr;
  a.blkmax = water ? h->blkmax : nullptr;
  a.kick = h->dt;
  a.half = 0.5 * h->dt;
  a.integrator = h->integrator;
  a.first = 0;
  a.thermo = h->thermostat == PIMD_THERMO_PILE_L;
  a.seed = h->seed;
  return a;
}

static ForceArgs force_args(pimd_handle *h) {
  ForceArgs a{};
  a.dbox = h->baro ? h->baro + kBaroL : nullptr;
  a.N = h->N;
  a.P = h->P;
  a.nmol = h->nmol;
  a.x = h->x;
  a.x32 = h->x32;
  a.step_inc = nullptr;
  a.F = h->F;
  a.Upart = h->Upart;
  a.Wpart = h->Wpart;
  a.W3part = h->W3part;
  a.kspring = h->kspring;
  for (int d = 0; d < 3; ++d) {
    a.box[d] = h->box[d];
    a.invbox[d] = h->box[d] > 0 ? 1.0 / h->box[d] : 0.0;
  }
  a.kb = h->ff[0];
  a.r0 = h->ff[1];
  a.kth = h->ff[2];
  a.th0 = h->ff[3];
  a.eps = h->ff[4];
  a.sig = h->ff[5];
  a.rc = h->ff[6];
  a.nbr = h->nbr;
  a.nbr_off = h->nbr_off;
  a.nbr_groups = h->nbr_groups;
  a.check_nbr = 0;
  a.blkmax = h->blkmax;
  // the warp-item split step reports one (drift, spread) pair for the system
  a.nblk_check = h->split_warp ? 1 : (h->N + h->A_step - 1) / h->A_step;
  a.skin = h->skin;
  a.rlist = h->rlist;
  a.ccur = h->ccur;
  a.cref = h->cref;
  a.err = h->d_err;
  return a;
}

static NbrArgs nbr_args(pimd_handle *h, bool force) {
  NbrArgs a;
  a.nmol = h->nmol;
  a.P = h->P;
  a.x = h->x;
  a.cref = h->cref;
  a.blkmax = h->blkmax;
  // the warp-item split step reports one (drift, spread) pair for the system
  a.nblk_check = h->split_warp ? 1 : (h->N + h->A_step - 1) / h->A_step;
  a.nbr = h->nbr;
  a.nbr_off = h->nbr_off;
  a.nbr_groups = h->nbr_groups;
  a.err = h->d_err;
  for (int d = 0; d < 3; ++d) {
    a.box[d] = h->box[d];
    a.invbox[d] = 1.0 / h->box[d];
  }
  a.dbox = h->baro ? h->baro + kBaroL : nullptr;
  a.rlist = h->rlist;
  a.skin = h->skin;
  a.force = force ? 1 : 0;
  return a;
}

// Forces of the current positions (and the neighbour list they need).
// from_outside: the positions were not written by the step kernel (create,
// set_state), so the centroids are recomputed and the list rebuilt.
// advance: the force kernel also advances the device step counter.
static SplitStepArgs split_args(pimd_handle *h) {
  SplitStepArgs a{};
  a.N = h->N;
  a.P = h->P;
  a.A = h->A_step;
  a.Mf = h->Mf;
  a.Mtf = h->Mtf;
  a.Tff = h->Tff;
  a.Tif = h->Tif;
  a.cAf = h->cAf;
  a.sAf = h->sAf;
  a.wsAf = h->wsAf;
  a.c1f = h->c1f;
  a.c2f = h->c2f;
  a.tA = h->tA;
  a.c1_0 = h->c1_0;
  a.c2_0 = h->c2_0;
  a.inv_mm = h->inv_mm;
  a.sigv = h->sigv;
  a.xc = h->xc;
  a.v0 = h->v0;
  a.d = h->dev;
  a.vk = h->vk;
  a.F = h->F32;
  const bool water = h->potential == PIMD_POT_WATERLIKE;
  a.xcw = water ? h->xcw : nullptr;
  for (int d = 0; d < 3; ++d) {
    a.box[d] = h->box[d];
    a.invbox[d] = h->box[d] > 0 ? 1.0 / h->box[d] : 0.0;
  }
  a.step = h->d_step;
  a.step_off = 0;
  a.cref = water ? h->cref : nullptr;
  a.ccur = water ? h->ccur : nullptr;
  a.blkmax = water ? h->blkmax : nullptr;
  a.kick = h->dt;
  a.half = 0.5 * h->dt;
  a.integrator = h->integrator;
  a.first = 0;
  a.thermo = h->thermostat == PIMD_THERMO_PILE_L;
  a.seed = h->seed;
  return a;
}

static SplitForceArgs split_force_args(pimd_handle *h) {
  const ForceArgs f = force_args(h);
  SplitForceArgs a{};
  a.N = h->N;
  a.P = h->P;
  a.nmol = h->nmol;
  a.xc = h->xc;
  a.xcw = h->xcw;
  a.d = h->dev;
  a.F = h->F32;
  a.Upart = h->Upart;
  a.Wpart = h->Wpart;
  a.step_inc = nullptr;
  a.kspring = h->kspring;
  for (int d = 0; d < 3; ++d) {
    a.box[d] = f.box[d];
    a.invbox[d] = f.invbox[d];
  }
  a.kb = f.kb;
  a.r0 = f.r0;
  a.kth = f.kth;
  a.th0 = f.th0;
  a.eps = f.eps;
  a.sig = f.sig;
  a.rc = f.rc;
  a.nbr = h->nbr;
  a.nbr_off = h->nbr_off;
  a.nbr_groups = h->nbr_groups;
  return a;
}

// Split precision: FP64 staging arrays x, v (and F) from the split state.
static pimd_status expand_split(pimd_handle *h, bool with_forces) {
  return enqueue(h, PIMD_KIND_OTHER, 1, [&] {
    return launch_expand_split(split_args(h), h->F32, h->x, h->v, with_forces ? h->F : nullptr,
                               h->stream);
  });
}

static pimd_status enqueue_forces(pimd_handle *h, bool from_outside, bool advance) {
  if (h->precision == PIMD_PREC_SPLIT) {
    const bool water = h->potential == PIMD_POT_WATERLIKE;
    SplitForceArgs sa = split_force_args(h);
    sa.step_inc = advance ? h->d_step : nullptr;
    pimd_status st;
    if (water) {
      if (from_outside) {
        st = enqueue(h, PIMD_KIND_OTHER, 1, [&] {
          return launch_centroids(nbr_args(h, true), h->ccur, h->stream);
        });
        if (st != PIMD_OK) return st;
      }
      st = enqueue(h, PIMD_KIND_NBR, 1, [&] {
        return launch_nbr_build(nbr_args(h, from_outside), h->ccur, h->stream);
      });
      if (st != PIMD_OK) return st;
    }
    return enqueue(h, PIMD_KIND_FORCE, 1, [&] { return launch_force_split(sa, water, h->stream); });
  }
  ForceArgs fa = force_args(h);
  fa.step_inc = advance ? h->d_step : nullptr;
  if (h->potential == PIMD_POT_WATERLIKE) {
    pimd_status st;
    if (from_outside) {
      st = enqueue(h, PIMD_KIND_OTHER, 2, [&] {
        cudaError_t e = launch_to_f32(h->x, h->x32, (size_t)h->N * 3 * h->P, h->stream);
        if (e != cudaSuccess) return e;
        return launch_centroids(nbr_args(h, true), h->ccur, h->stream);
      });
      if (st != PIMD_OK) return st;
    }
    if (from_outside) {
      st = enqueue(h, PIMD_KIND_NBR, 1, [&] {
        return launch_nbr_build(nbr_args(h, true), h->ccur, h->stream);
      });
      if (st != PIMD_OK) return st;
    } else {
      fa.check_nbr = 1;   // the skin test and any rebuild run inside the force kernel
    }
    return enqueue(h, PIMD_KIND_FORCE, 1, [&] { return launch_force_water(fa, h->stream); });
  }
  return enqueue(h, PIMD_KIND_FORCE, 1, [&] { return launch_force_harmonic(fa, h->stream); });
}

// B_W of the barostat over [t0, t0 + tB] of the kick the next kernel
// applies (App. E); with step_follows also that step's O_W and box.
static pimd_status enqueue_baro(pimd_handle *h, double t0, double tB, bool step_follows) {
  BaroArgs b{};
  b.obabo = h->integrator == PIMD_OBABO;
  b.N = h->N;
  b.P = h->P;
  b.nmol = h->nmol;
  b.x = h->x;
  b.v = h->v;
  b.F = h->F;
  b.Mt = h->Mt;
  b.mass_mm = h->mass_mm;
  b.Wpart = h->Wpart;
  b.W3part = h->W3part;
  b.axes = h->baro_axes;
  b.baro = h->baro;
  b.t0 = t0;
  b.tB = tB;
  b.tA = b.obabo ? h->dt : 0.5 * h->dt;
  b.step_follows = step_follows ? 1 : 0;
  const double kT = kBoltzmann * h->T;
  b.W = (h->baro_axes ? 1.0 : 3.0) * h->P * h->N * kT * h->taup * h->taup;
  b.nkT = h->P * kT;
  b.npext = h->P * h->pext;
  b.mu0 = h->fmass;
  b.thermo = h->thermostat == PIMD_THERMO_PILE_L;
  b.c1W = std::exp(-(b.obabo ? 0.5 * h->dt : h->dt) / h->tau);   // the O_W's own duration
  b.sigW = std::sqrt(1.0 - b.c1W * b.c1W) * std::sqrt(b.nkT / b.W);
  b.seed = h->seed;
  b.step = h->d_step;
  b.Lmin = 2.0 * h->ff[6];
  b.err = h->d_err;
  return enqueue(h, PIMD_KIND_OTHER, 1, [&] { return launch_baro_kick(b, h->stream); });
}

// One full step: the fused integrator kernel, the forces of the new
// positions, and the step counter.
static pimd_status enqueue_step(pimd_handle *h, bool first) {
  if (h->precision == PIMD_PREC_SPLIT) {
    pimd_status st;
    if (h->split_warp) {
      const bool water = h->potential == PIMD_POT_WATERLIKE;
      st = enqueue(h, PIMD_KIND_STEP, 1, [&] {
        return launch_step_split_warp(h->sw_desc, h->N, h->P, h->d_step, 0, first ? 1 : 0,
                                      water ? h->blkmax : nullptr, h->sw_done, h->stream);
      });
    } else {
      SplitStepArgs a = split_args(h);
      a.first = first ? 1 : 0;
      a.kick = first ? 0.5 * h->dt : h->dt;
      st = enqueue(h, PIMD_KIND_STEP, 1, [&] { return launch_step_split(a, h->threads_step, h->stream); });
    }
    if (st != PIMD_OK) return st;
    return enqueue_forces(h, false, true);
  }
  StepArgs a = step_args(h);
  a.first = first ? 1 : 0;
  a.kick = first ? 0.5 * h->dt : h->dt;
  pimd_status st;
  if (h->baro && h->integrator == PIMD_OBABO) {
    // OBABO: the opening B_W needs the velocities after both O(h/2), so the
    // step runs as [closing B O + opening O] -> O_W, B_W, box -> [B, A(h)]
    StepArgs a1 = a, a2 = a;
    a1.phase = 1;
    a2.phase = 2;
    st = enqueue(h, PIMD_KIND_STEP, 1, [&] { return launch_step(a1, h->threads_step, h->stream); });
    if (st != PIMD_OK) return st;
    if ((st = enqueue_baro(h, 0.0, 0.5 * h->dt, true)) != PIMD_OK) return st;
    st = enqueue(h, PIMD_KIND_STEP, 1, [&] { return launch_step(a2, h->threads_step, h->stream); });
    if (st != PIMD_OK) return st;
  } else {
    // the B_W beside this step's opening B(h/2), which follows the previous
    // step's closing B(h/2) inside a merged kick
    if (h->baro && (st = enqueue_baro(h, first ? 0.0 : 0.5 * h->dt, 0.5 * h->dt, true)) != PIMD_OK)
      return st;
    st = enqueue(h, PIMD_KIND_STEP, 1, [&] { return launch_step(a, h->threads_step, h->stream); });
    if (st != PIMD_OK) return st;
  }
  st = enqueue_forces(h, false, true);
  if (st != PIMD_OK) return st;
  // the B_W beside this step's closing B(h/2) (applied by the next kernel)
  if (h->baro && (st = enqueue_baro(h, 0.0, 0.5 * h->dt, false)) != PIMD_OK) return st;
  if (!h->fixcom) return st;
  // fixcom at the end of this step: the next kernel (step or close) applies
  // this step's closing B(h/2) (and O(h/2)); remove the momentum it will leave
  FixcomArgs f{};
  f.N = h->N;
  f.P = h->P;
  f.method = h->method;
  f.mass_mm = h->mass_mm;
  f.x = h->x;
  f.F = h->F;
  f.v = h->v;
  f.half = 0.5 * h->dt;
  f.imu0 = 1.0 / h->fmass;   // mu_0 = fmass in both methods
  f.wn2 = h->wn * h->wn;
  f.obabo_thermo = h->integrator == PIMD_OBABO && h->thermostat == PIMD_THERMO_PILE_L;
  f.seed = h->seed;
  f.step = h->d_step;
  f.c1 = h->c1;
  f.c2 = h->c2;
  f.sigv = h->sigv;
  return enqueue(h, PIMD_KIND_OTHER, 1, [&] { return launch_fixcom(f, h->stream); });
}

static pimd_status enqueue_close(pimd_handle *h) {
  if (h->precision == PIMD_PREC_SPLIT) {
    SplitStepArgs a = split_args(h);
    a.step_off = -1;
    return enqueue(h, PIMD_KIND_CLOSE, 1, [&] { return launch_close_split(a, h->threads_step, h->stream); });
  }
  StepArgs a = step_args(h);
  a.step_off = -1;
  return enqueue(h, PIMD_KIND_CLOSE, 1, [&] { return launch_close(a, h->threads_step, h->stream); });
}

static pimd_status build_graph(pimd_handle *h, int nsteps) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  const int64_t before = h->launches;
  pimd_status st = PIMD_OK;
  for (int s = 0; s < nsteps && st == PIMD_OK; ++s) st = enqueue_step(h, false);
  h->capturing = false;
  h->graph_kernels = h->launches - before;
  h->launches = before;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (st != PIMD_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(PIMD_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return fail(PIMD_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  h->graph_steps = nsteps;
  return PIMD_OK;
}

static pimd_status check_device_errors(pimd_handle *h) {
  CK(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (*h->h_err & kErrNbrOverflow) {
    h->latched = PIMD_EOVERFLOW;
    snprintf(h->latched_msg, sizeof(h->latched_msg),
             "neighbour list overflow (more than %d O-O neighbours within rc + skin)",
             kMaxNeighbours);
  } else if (*h->h_err & kErrNonFinite) {
    h->latched = PIMD_ENONFINITE;
    snprintf(h->latched_msg, sizeof(h->latched_msg), "non-finite estimator sum");
  } else if (*h->h_err & kErrBoxSmall) {
    h->latched = PIMD_EINVAL;
    snprintf(h->latched_msg, sizeof(h->latched_msg), "the barostat shrank a box edge below 2 rc");
  }
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  return PIMD_OK;
}

static void release(pimd_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto &p : h->pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  if (h->graph) cudaGraphExecDestroy(h->graph);
  dev_free(h->alloc, h->arena, h->stream);
  if (h->h_est) cudaFreeHost(h->h_est);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

extern "C" void pimd_destroy(pimd_handle *h) { release(h); }

struct Carver {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

static void carve(pimd_handle *h, Carver &c) {
  const size_t len = (size_t)h->N * 3 * h->P;
  const int P = h->P, N = h->N;
  h->x = c.take<double>(len);
  h->v = c.take<double>(len);
  h->F = c.take<double>(len);
  h->tmp = c.take<double>(len);
  if (h->potential == PIMD_POT_WATERLIKE) h->x32 = c.take<float>(len);
  h->inv_mm = c.take<double>(N);
  h->sigv = c.take<double>(N);
  h->mass_mm = c.take<double>(N);
  h->kspring = c.take<double>(N);
  h->M = c.take<double>((size_t)P * P);
  h->Mt = c.take<double>((size_t)P * P);
  h->cA = c.take<double>(P);
  h->sA = c.take<double>(P);
  h->wsA = c.take<double>(P);
  h->c1 = c.take<double>(P);
  h->c2 = c.take<double>(P);
  h->lam = c.take<double>(P);
  h->mu = c.take<double>(P);
  h->imu = c.take<double>(P);
  h->Tf = c.take<double>((size_t)(P / 2 + 1) * P);
  h->Ti = c.take<double>((size_t)(P / 2 + 1) * P);
  // rows of per-bead U / Tr Xi sums: one per molecule (water) or per block
  h->nblk_force = h->potential == PIMD_POT_WATERLIKE ? h->nmol : force_blocks(h->N, P);
  h->Upart = c.take<double>((size_t)h->nblk_force * P);
  h->Wpart = c.take<double>((size_t)h->nblk_force * P);
  if (h->potential == PIMD_POT_WATERLIKE) {
    h->cref = c.take<double>((size_t)h->nmol * 3);
    h->ccur = c.take<double>((size_t)h->nmol * 3);
    h->blkmax = c.take<double>(2 * ((N + h->A_step - 1) / h->A_step));
    h->nbr = c.take<int>((size_t)h->nmol * kMaxNeighbours);
    h->nbr_groups = water_lane_groups(P);
    h->nbr_off = c.take<int>((size_t)h->nmol * (kLJWarps * h->nbr_groups + 1));
  }
  h->nblk_est = (N + h->A_est - 1) / h->A_est;
  h->est_part = c.take<double>((size_t)h->nblk_est * (2 * P + 4));
  h->est_out = c.take<double>(3 * P + 12);
  h->d_step = c.take<int64_t>(1);
  h->d_err = c.take<unsigned>(4);
  if (h->barostat) h->baro = c.take<double>(kBaroWords);
  if (h->baro_axes) h->W3part = c.take<double>((size_t)h->nmol * P * 3);
  if (h->precision == PIMD_PREC_SPLIT) {
    h->xc = c.take<double>((size_t)N * 3);
    h->v0 = c.take<double>((size_t)N * 3);
    h->dev = c.take<float>(len);
    h->vk = c.take<float>(len);
    h->F32 = c.take<float>(len);
    h->xcw = c.take<float>((size_t)N * 3);
    h->Mf = c.take<float>((size_t)P * P);
    h->Mtf = c.take<float>((size_t)P * P);
    h->Tff = c.take<float>((size_t)(P / 2 + 1) * P);
    h->Tif = c.take<float>((size_t)(P / 2 + 1) * P);
    h->cAf = c.take<float>(P);
    h->sAf = c.take<float>(P);
    h->wsAf = c.take<float>(P);
    h->c1f = c.take<float>(P);
    h->c2f = c.take<float>(P);
    if (h->split_warp) {
      h->sw_desc = c.take<char>(split_warp_desc_bytes());
      h->sw_frag = c.take<float4>(split_warp_frag_float4(P));
      h->sw_imf = c.take<float>(N);
      h->sw_sgf = c.take<float>(N);
      h->sw_ctl = c.take<long long>(8);
      h->sw_done = c.take<unsigned>(1);
    }
  }
}

static pimd_status upload_state(pimd_handle *h, const double *x, const double *v) {
  const size_t bytes = (size_t)h->N * 3 * h->P * sizeof(double);
  CK(cudaMemcpyAsync(h->tmp, x, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(launch_pna_to_nap(h->tmp, h->x, h->N, h->P, h->stream));
  if (v) {
    CK(cudaMemcpyAsync(h->tmp, v, bytes, cudaMemcpyHostToDevice, h->stream));
    CK(launch_pna_to_nap(h->tmp, h->v, h->N, h->P, h->stream));
  } else {
    CK(launch_thermal_v(h->v, h->sigv, h->imu, h->seed, h->N, h->P, h->stream));
  }
  if (h->precision == PIMD_PREC_SPLIT) CK(launch_compress_split(split_args(h), h->x, h->v, h->stream));
  return PIMD_OK;
}

namespace pimd {
pimd_status validate_create(const pimd_system *sys, int32_t P, double T, double dt, double gamma0,
                            const pimd_params *params, pimd_params *out) {
  if (!sys) return fail(PIMD_EINVAL, "sys is NULL");
  pimd_params prm;
  if (params)
    prm = *params;
  else
    pimd_params_default(&prm);
  if (P < 1 || P > PIMD_MAX_BEADS) return fail(PIMD_EINVAL, "P = %d outside 1..%d", P, PIMD_MAX_BEADS);
  if (!(T > 0.0)) return fail(PIMD_EINVAL, "T must be > 0");
  if (!(dt > 0.0)) return fail(PIMD_EINVAL, "dt must be > 0");
  if (sys->n_atoms <= 0) return fail(PIMD_EINVAL, "n_atoms must be > 0");
  if (!sys->mass || !sys->pos) return fail(PIMD_EINVAL, "mass and pos are required");
  if (sys->potential != PIMD_POT_HARMONIC && sys->potential != PIMD_POT_WATERLIKE)
    return fail(PIMD_EINVAL, "unknown potential %d", sys->potential);
  if (prm.thermostat != PIMD_THERMO_NONE && prm.thermostat != PIMD_THERMO_PILE_L)
    return fail(PIMD_EINVAL, "unknown thermostat %d", prm.thermostat);
  if (prm.integrator != PIMD_BAOAB && prm.integrator != PIMD_OBABO)
    return fail(PIMD_EINVAL, "unknown integrator %d", prm.integrator);
  if (prm.method != PIMD_METHOD_NMPIMD && prm.method != PIMD_METHOD_PIMD)
    return fail(PIMD_EINVAL, "unknown method %d", prm.method);
  if (prm.precision != PIMD_PREC_FP64 && prm.precision != PIMD_PREC_SPLIT)
    return fail(PIMD_EINVAL, "unknown precision %d", prm.precision);
  if (prm.fixcom != 0 && prm.fixcom != 1) return fail(PIMD_EINVAL, "fixcom must be 0 or 1");
  if (prm.fmmode != PIMD_FMMODE_PHYSICAL && prm.fmmode != PIMD_FMMODE_NORMAL)
    return fail(PIMD_EINVAL, "unknown fmmode %d", prm.fmmode);
  if (prm.fmmode == PIMD_FMMODE_NORMAL && prm.method == PIMD_METHOD_PIMD)
    return fail(PIMD_EINVAL, "fmmode normal applies to normal modes (method nmpimd)");
  if (!(prm.fmass > 0.0) || !std::isfinite(prm.fmass)) return fail(PIMD_EINVAL, "fmass must be > 0");
  if (!(prm.sp > 0.0)) return fail(PIMD_EINVAL, "sp must be > 0");
  if (prm.barostat != PIMD_BARO_NONE && prm.barostat != PIMD_BARO_BZP_ISO &&
      prm.barostat != PIMD_BARO_BZP_ANISO)
    return fail(PIMD_EINVAL, "unknown barostat %d", prm.barostat);
  if (prm.barostat == PIMD_BARO_BZP_ANISO && (prm.baro_axes < 1 || prm.baro_axes > 7))
    return fail(PIMD_EINVAL, "baro_axes must be a nonzero mask of PIMD_AXIS_X/Y/Z");
  if (prm.barostat != PIMD_BARO_NONE) {
    if (sys->potential != PIMD_POT_WATERLIKE)
      return fail(PIMD_EINVAL, "the barostat needs a periodic (water-like) system");
    if (prm.method != PIMD_METHOD_NMPIMD) return fail(PIMD_EINVAL, "the barostat acts on normal modes (nmpimd)");
    if (!(prm.taup > 0.0) || !std::isfinite(prm.taup)) return fail(PIMD_EINVAL, "taup must be > 0");
    if (!std::isfinite(prm.pext)) return fail(PIMD_EINVAL, "pext must be finite");
  }
  if (prm.precision == PIMD_PREC_SPLIT) {
    pimd_status ks = require_default_keywords(prm, "split precision");
    if (ks != PIMD_OK) return ks;
  }
  if (gamma0 > 0.0) {
    const double tau = 1.0 / gamma0;
    if (params && std::fabs(params->tau - tau) > 1e-12 * tau)
      return fail(PIMD_EINVAL, "gamma0 and params->tau disagree");
    prm.tau = tau;
  } else if (gamma0 < 0.0) {
    return fail(PIMD_EINVAL, "gamma0 must be >= 0");
  }
  if (prm.thermostat == PIMD_THERMO_PILE_L && (!(prm.tau > 0.0) || !(prm.scale > 0.0)))
    return fail(PIMD_EINVAL, "PILE_L needs tau > 0 and scale > 0");
  const int N = sys->n_atoms;
  for (int i = 0; i < N; ++i)
    if (!(sys->mass[i] > 0.0)) return fail(PIMD_EINVAL, "mass[%d] must be > 0", i);
  if (sys->potential == PIMD_POT_WATERLIKE) {
    if (N % 3) return fail(PIMD_EINVAL, "water-like systems need 3 atoms per molecule");
    const double rc = sys->ff[6];
    if (!(rc > 0.0)) return fail(PIMD_EINVAL, "cutoff must be > 0");
    for (int d = 0; d < 3; ++d)
      if (!(sys->box[d] > 2.0 * rc))
        return fail(PIMD_EINVAL, "box edge %d (%g) must exceed 2 rc (%g)", d, sys->box[d], 2 * rc);
    if (!(sys->ff[0] >= 0 && sys->ff[1] > 0 && sys->ff[2] >= 0 && sys->ff[4] >= 0 && sys->ff[5] > 0))
      return fail(PIMD_EINVAL, "invalid water-like force-field parameters");
  }

  *out = prm;
  return PIMD_OK;
}

pimd_status require_default_keywords(const pimd_params &prm, const char *where) {
  if (prm.method != PIMD_METHOD_NMPIMD || prm.fmmode != PIMD_FMMODE_PHYSICAL || prm.fmass != 1.0 ||
      prm.fixcom != 0 || prm.barostat != PIMD_BARO_NONE)
    return fail(PIMD_EINVAL, "%s implements method nmpimd, fmmode physical, fmass 1, fixcom 0 and no barostat",
                where);
  return PIMD_OK;
}

void build_tables(int P, double T, double dt, const pimd_params &prm, HostTables &t) {
  build_nm_matrix(P, t.M);
  t.Mt.assign((size_t)P * P, 0.0);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) t.Mt[(size_t)j * P + i] = t.M[(size_t)i * P + j];
  // folded transforms: rows k <= H of M are even under j -> P - j, rows k > H
  // odd, so each output needs one half of a folded row
  const int H = P / 2;
  t.Tf.assign((size_t)(H + 1) * P, 0.0);
  t.Ti.assign((size_t)(H + 1) * P, 0.0);
  for (int i = 0; i <= H; ++i)
    for (int k = 0; k < P; ++k) {
      const int pos = H + 1 + i;   // odd rows: folded position, holding x_{P-pos} - x_pos
      t.Tf[(size_t)i * P + k] = k <= H ? t.M[(size_t)k * P + i] : (pos < P ? t.M[(size_t)k * P + (P - pos)] : 0.0);
      const int kodd = H + 1 + i;  // inverse of bead k > H: odd mode kodd at bead P - k
      t.Ti[(size_t)i * P + k] = k <= H ? t.M[(size_t)i * P + k] : (kodd < P ? t.M[(size_t)kodd * P + (P - k)] : 0.0);
    }
  const double hbar = prm.sp * kPlanck / (2.0 * kPi);
  t.wn = P * kBoltzmann * T / hbar;                      // Eq. (2)
  t.tA = prm.integrator == PIMD_BAOAB ? 0.5 * dt : dt;
  t.tO = prm.integrator == PIMD_BAOAB ? dt : 0.5 * dt;
  t.cA.resize(P);
  t.sA.resize(P);
  t.wsA.resize(P);
  t.c1.resize(P);
  t.c2.resize(P);
  t.lam.resize(P);
  t.mu.resize(P);
  t.imu.resize(P);
  const bool cart = prm.method == PIMD_METHOD_PIMD;
  for (int k = 0; k < P; ++k) {
    const double s = std::sin(kPi * k / P);
    t.lam[k] = 4.0 * s * s;                               // Eq. (A2)
    // fictitious mass m^(k) = mu_k m (Sec. III.C fmmode, fmass; lambda_0 = 0
    // leaves the centroid at fmass m)
    t.mu[k] = (!cart && prm.fmmode == PIMD_FMMODE_NORMAL && k > 0) ? prm.fmass * t.lam[k] : prm.fmass;
    t.imu[k] = 1.0 / t.mu[k];
    // the mode's own frequency in the free ring polymer: w_k / sqrt(mu_k)
    const double wk = 2.0 * t.wn * std::fabs(s) / std::sqrt(t.mu[k]);
    if (k == 0 || wk == 0.0) {
      t.cA[k] = 1.0;
      t.sA[k] = t.tA;
      t.wsA[k] = 0.0;
    } else {
      t.cA[k] = std::cos(wk * t.tA);
      t.sA[k] = std::sin(wk * t.tA) / wk;
      t.wsA[k] = wk * std::sin(wk * t.tA);
    }
    // App. D: tau_0 = tau, tau_k = scale / (2 w_k); Cartesian: scale / (2 w_n) for every bead
    const double tauk = cart ? prm.scale / (2.0 * t.wn) : ((k == 0) ? prm.tau : prm.scale / (2.0 * wk));
    t.c1[k] = std::exp(-t.tO / tauk);
    t.c2[k] = std::sqrt(1.0 - t.c1[k] * t.c1[k]) / std::sqrt(t.mu[k]);   // noise of sqrt(P kB T / (m^(k) mvv2e))
  }
}
}  // namespace pimd

extern "C" pimd_status pimd_create(const pimd_system *sys, int32_t P, double T, double dt,
                                   double gamma0, const pimd_params *params, void *stream,
                                   pimd_handle **out) {
  if (!out) return fail(PIMD_EINVAL, "out is NULL");
  *out = nullptr;
  pimd_params prm;
  {
    pimd_status vs = validate_create(sys, P, T, dt, gamma0, params, &prm);
    if (vs != PIMD_OK) return vs;
  }
  const int N = sys->n_atoms;
  pimd_handle *h = new pimd_handle();
  h->N = N;
  h->P = P;
  h->potential = sys->potential;
  h->nmol = sys->potential == PIMD_POT_WATERLIKE ? N / 3 : 0;
  h->integrator = prm.integrator;
  h->thermostat = prm.thermostat;
  h->precision = prm.precision;
  h->method = prm.method;
  h->fixcom = prm.fixcom;
  h->fmass = prm.fmass;
  h->barostat = prm.barostat;
  h->baro_axes = prm.barostat == PIMD_BARO_BZP_ANISO ? prm.baro_axes : 0;
  h->pext = prm.pext;
  h->taup = prm.taup;
  h->T = T;
  h->dt = dt;
  h->tau = prm.tau;
  h->scale = prm.scale;
  h->sp = prm.sp;
  h->seed = prm.seed;
  for (int d = 0; d < 3; ++d) h->box[d] = sys->box[d];
  for (int q = 0; q < 8; ++q) h->ff[q] = sys->ff[q];
  h->rlist = h->ff[6] + h->skin;
  h->alloc = current_allocator();
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return fail(PIMD_ECUDA, "cudaStreamCreate failed");
    }
    h->own_stream = true;
  }
  h->A_step = tile_atoms(N, P);
  h->threads_step = tile_threads(h->A_step, P);
  h->split_warp = prm.precision == PIMD_PREC_SPLIT && split_warp_class(P);
  h->A_est = std::max(1, 256 / P);
  h->threads_est = est_threads(h->A_est, P);
  const char *ng = getenv("PIMD_NO_GRAPH");
  h->use_graph = !(ng && ng[0] == '1');

  Carver c0{nullptr};
  carve(h, c0);
  h->arena_bytes = c0.off + 256;
  h->arena = dev_alloc(h->alloc, h->arena_bytes, h->stream);
  if (!h->arena) {
    release(h);
    return fail(PIMD_ENOMEM, "device allocation of %zu bytes failed", h->arena_bytes);
  }
  Carver c1{(char *)h->arena};
  carve(h, c1);
  if (cudaMallocHost(&h->h_est, sizeof(double) * (3 * P + 12)) != cudaSuccess ||
      cudaMallocHost(&h->h_err, sizeof(unsigned) * 4) != cudaSuccess) {
    release(h);
    return fail(PIMD_ENOMEM, "pinned host allocation failed");
  }

  // ---- host tables (App. B, App. D), FP64 ----
  HostTables tb;
  build_tables(P, T, dt, prm, tb);
  h->wn = tb.wn;
  const std::vector<double> &M = tb.M, &Mt = tb.Mt, &cA = tb.cA, &sA = tb.sA, &wsA = tb.wsA;
  const std::vector<double> &c1v = tb.c1, &c2v = tb.c2, &lam = tb.lam;
  const double tA = tb.tA;
  std::vector<double> inv_mm(N), sigv(N), mass_mm(N), ksp(N);
  for (int i = 0; i < N; ++i) {
    const double mm = sys->mass[i] * kMvv2e;
    mass_mm[i] = mm;
    inv_mm[i] = 1.0 / mm;
    sigv[i] = std::sqrt(P * kBoltzmann * T / mm);
    ksp[i] = mm * sys->ff[0] * sys->ff[0];
  }
  pimd_status st = PIMD_OK;
  auto up = [&](double *dst, const std::vector<double> &src) -> pimd_status {
    CK(cudaMemcpy(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice));
    return PIMD_OK;
  };
  if ((st = up(h->M, M)) || (st = up(h->Mt, Mt)) || (st = up(h->cA, cA)) || (st = up(h->sA, sA)) ||
      (st = up(h->wsA, wsA)) || (st = up(h->c1, c1v)) || (st = up(h->c2, c2v)) ||
      (st = up(h->lam, lam)) || (st = up(h->mu, tb.mu)) || (st = up(h->imu, tb.imu)) ||
      (st = up(h->Tf, tb.Tf)) || (st = up(h->Ti, tb.Ti)) ||
      (st = up(h->inv_mm, inv_mm)) || (st = up(h->sigv, sigv)) ||
      (st = up(h->mass_mm, mass_mm)) || (st = up(h->kspring, ksp))) {
    release(h);
    return st;
  }
  if (h->precision == PIMD_PREC_SPLIT) {
    auto upf = [&](float *dst, const std::vector<double> &src) -> pimd_status {
      std::vector<float> f(src.begin(), src.end());
      CK(cudaMemcpy(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
      return PIMD_OK;
    };
    if ((st = upf(h->Mf, M)) || (st = upf(h->Mtf, Mt)) || (st = upf(h->Tff, tb.Tf)) ||
        (st = upf(h->Tif, tb.Ti)) || (st = upf(h->cAf, cA)) ||
        (st = upf(h->sAf, sA)) || (st = upf(h->wsAf, wsA)) || (st = upf(h->c1f, c1v)) ||
        (st = upf(h->c2f, c2v))) {
      release(h);
      return st;
    }
    h->tA = tA;
    h->c1_0 = c1v[0];
    h->c2_0 = c2v[0];
    if (h->split_warp) {
      SplitWarpSetup w{};
      w.N = N;
      w.P = P;
      w.integrator = h->integrator;
      w.thermo = h->thermostat == PIMD_THERMO_PILE_L;
      w.seed = h->seed;
      w.dt = h->dt;
      w.tA = tA;
      w.c1_0 = c1v[0];
      w.c2_0 = c2v[0];
      for (int c = 0; c < 3; ++c) w.box[c] = h->potential == PIMD_POT_WATERLIKE ? h->box[c] : 0.0;
      w.xc = h->xc;
      w.v0 = h->v0;
      w.d = h->dev;
      w.vk = h->vk;
      w.F = h->F32;
      w.xcw = h->xcw;
      w.inv_mm = h->inv_mm;
      w.sigv = h->sigv;
      w.cAf = h->cAf;
      w.sAf = h->sAf;
      w.wsAf = h->wsAf;
      w.c1f = h->c1f;
      w.c2f = h->c2f;
      const bool water = h->potential == PIMD_POT_WATERLIKE;
      w.cref = water ? h->cref : nullptr;
      w.ccur = water ? h->ccur : nullptr;
      w.M_host = M.data();
      w.inv_mm_host = inv_mm.data();
      w.sigv_host = sigv.data();
      w.desc = h->sw_desc;
      w.frag = h->sw_frag;
      w.inv_mmf = h->sw_imf;
      w.sigvf = h->sw_sgf;
      w.ctl = h->sw_ctl;
      w.done = h->sw_done;
      const cudaError_t e = split_warp_setup(w, h->stream);
      if (e != cudaSuccess) {
        release(h);
        return fail(PIMD_ECUDA, "split step set-up failed: %s", cudaGetErrorString(e));
      }
    }
  }
  auto init = [&]() -> pimd_status {
    CK(cudaMemsetAsync(h->d_step, 0, sizeof(int64_t), h->stream));
    CK(cudaMemsetAsync(h->d_err, 0, 4 * sizeof(unsigned), h->stream));
    if (h->baro) {
      for (int c = 0; c < 3; ++c) {
        h->h_baro[kBaroL + c] = h->box[c];
        h->h_baro[kBaroInvL + c] = 1.0 / h->box[c];
      }
      CK(cudaMemcpyAsync(h->baro, h->h_baro, sizeof(h->h_baro), cudaMemcpyHostToDevice, h->stream));
    }
    if (h->potential == PIMD_POT_WATERLIKE) {
      CK(cudaMemsetAsync(h->cref, 0, sizeof(double) * 3 * h->nmol, h->stream));
      CK(cudaMemsetAsync(h->nbr_off, 0,
                         sizeof(int) * h->nmol * (kLJWarps * h->nbr_groups + 1), h->stream));
    }
    pimd_status s2 = upload_state(h, sys->pos, sys->vel);
    if (s2 != PIMD_OK) return s2;
    s2 = enqueue_forces(h, true, false);
    if (s2 != PIMD_OK) return s2;
    return check_device_errors(h);
  };
  if ((st = init()) != PIMD_OK) {
    release(h);
    return st;
  }
  *out = h;
  return PIMD_OK;
}

extern "C" pimd_status pimd_step(pimd_handle *h, int64_t n) {
  if (!h) return fail(PIMD_EINVAL, "handle is NULL");
  if (n < 0) return fail(PIMD_EINVAL, "n must be >= 0");
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  if (n == 0) return PIMD_OK;
  pimd_status st = enqueue_step(h, true);
  if (st != PIMD_OK) return st;
  int64_t left = n - 1;
  // steps per graph replay (8: 31.1, 32: 30.8 us per MD step on 64 x 32 water)
  const int G = 32;
  if (h->use_graph && !h->timing && left >= G) {
    if (!h->graph) {
      st = build_graph(h, G);
      if (st != PIMD_OK) return st;
    }
    while (left >= h->graph_steps) {
      CK(cudaGraphLaunch(h->graph, h->stream));
      h->launches += h->graph_kernels;
      left -= h->graph_steps;
    }
  }
  for (; left > 0; --left) {
    st = enqueue_step(h, false);
    if (st != PIMD_OK) return st;
  }
  st = enqueue_close(h);
  if (st != PIMD_OK) return st;
  h->step += n;
  return PIMD_OK;
}

extern "C" pimd_status pimd_sync(pimd_handle *h) {
  if (!h) return fail(PIMD_EINVAL, "handle is NULL");
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  return check_device_errors(h);
}

extern "C" pimd_status pimd_estimators(pimd_handle *h, pimd_estimates *out) {
  if (!h || !out) return fail(PIMD_EINVAL, "NULL argument");
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  const int P = h->P;
  if (h->precision == PIMD_PREC_SPLIT) {
    pimd_status se = expand_split(h, true);
    if (se != PIMD_OK) return se;
  }
  EstArgs a{};
  a.N = h->N;
  a.P = P;
  a.A = h->A_est;
  a.method = h->method;
  a.mt = ModeTables{h->M, h->Mt, h->cA, h->sA, h->wsA, h->c1, h->c2, h->lam, h->mu, h->imu, h->Tf, h->Ti};
  a.mass_mm = h->mass_mm;
  a.x = h->x;
  a.v = h->v;
  a.F = h->F;
  a.wn2 = h->wn * h->wn;
  a.part = h->est_part;
  pimd_status st0 = enqueue(h, PIMD_KIND_EST, 1, [&] { return launch_est(a, h->threads_est, h->stream); });
  if (st0 != PIMD_OK) return st0;
  EstFinalArgs f{};
  f.N = h->N;
  f.P = P;
  f.nblk_est = h->nblk_est;
  f.nblk_force = h->nblk_force;
  f.part = h->est_part;
  f.Upart = h->Upart;
  f.Wpart = h->Wpart;
  f.kT = kBoltzmann * h->T;
  f.kB = kBoltzmann;
  f.volume = (h->potential == PIMD_POT_WATERLIKE) ? h->box[0] * h->box[1] * h->box[2] : 0.0;
  f.dbox = h->baro ? h->baro + kBaroL : nullptr;
  f.out = h->est_out;
  f.err = h->d_err;
  st0 = enqueue(h, PIMD_KIND_EST, 1, [&] { return launch_est_final(f, h->stream); });
  if (st0 != PIMD_OK) return st0;
  CK(cudaMemcpyAsync(h->h_est, h->est_out, sizeof(double) * (3 * P + 12), cudaMemcpyDeviceToHost,
                     h->stream));
  if (h->baro)
    CK(cudaMemcpyAsync(h->h_baro, h->baro, sizeof(h->h_baro), cudaMemcpyDeviceToHost, h->stream));
  pimd_status st = check_device_errors(h);
  if (st != PIMD_OK) return st;
  std::memset(out, 0, sizeof(*out));
  out->step = h->step;
  out->P = P;
  out->N = h->N;
  const double *e = h->h_est;
  for (int k = 0; k < P; ++k) {
    out->K_mode[k] = e[k];
    out->S_mode[k] = e[P + k];
    out->U_bead[k] = e[2 * P + k];
  }
  const double *g = e + 3 * P;
  out->H = g[0];
  out->K_PR = g[1];
  out->K_VR = g[2];
  out->K_CV = g[3];
  out->P_PR = g[4];
  out->P_MD = g[5];
  out->P_CV = g[6];
  out->T_ring = g[7];
  out->volume = g[8];
  out->vir_sum = g[9];
  for (int c = 0; c < 3; ++c) out->box[c] = h->baro ? h->h_baro[kBaroL + c] : h->box[c];
  if (h->baro) {   // outputs 11-15
    const double kT = kBoltzmann * h->T, n = P;
    const double V = out->box[0] * out->box[1] * out->box[2];
    if (h->baro_axes) {   // one barostat per edge in baro_axes, W = n N kB T taup^2 each
      const double W = n * h->N * kT * h->taup * h->taup;
      out->vW = 0.0;
      out->K_W = 0.0;
      out->J_W = 0.0;
      for (int c = 0; c < 3; ++c) {
        out->vWa[c] = h->h_baro[kBaroV + c];
        out->K_W += 0.5 * W * out->vWa[c] * out->vWa[c];
        if (h->baro_axes >> c & 1) out->J_W -= n * kT * std::log(out->box[c]);
      }
    } else {
      const double W = 3.0 * n * h->N * kT * h->taup * h->taup;
      out->vW = h->h_baro[kBaroV];
      out->K_W = 0.5 * W * out->vW * out->vW;
      out->J_W = -n * kT * std::log(V);
    }
    out->U_W = n * h->pext * V;
    out->enthalpy = out->H + out->K_W + out->U_W + out->J_W;
  }
  return PIMD_OK;
}

extern "C" pimd_status pimd_get_barostat(pimd_handle *h, double *vW, double *box) {
  if (!h) return fail(PIMD_EINVAL, "handle is NULL");
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  if (h->baro) CK(cudaMemcpyAsync(h->h_baro, h->baro, sizeof(h->h_baro), cudaMemcpyDeviceToHost, h->stream));
  pimd_status st = check_device_errors(h);
  if (st != PIMD_OK) return st;
  if (vW) {
    if (h->baro_axes)
      for (int c = 0; c < 3; ++c) vW[c] = h->h_baro[kBaroV + c];
    else
      *vW = h->baro ? h->h_baro[kBaroV] : 0.0;
  }
  if (box)
    for (int c = 0; c < 3; ++c) box[c] = h->baro ? h->h_baro[kBaroL + c] : h->box[c];
  return PIMD_OK;
}

extern "C" pimd_status pimd_set_barostat(pimd_handle *h, const double *vW, const double *box) {
  if (!h || !box) return fail(PIMD_EINVAL, "NULL argument");
  if (!h->baro) return fail(PIMD_EINVAL, "the handle has no barostat");
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  if (!vW) return fail(PIMD_EINVAL, "NULL argument");
  double vw3[3];
  for (int c = 0; c < 3; ++c) {
    vw3[c] = h->baro_axes ? vW[c] : vW[0];
    if (!std::isfinite(vw3[c])) return fail(PIMD_EINVAL, "vW must be finite");
    if (h->baro_axes && !(h->baro_axes >> c & 1) && vw3[c] != 0.0)
      return fail(PIMD_EINVAL, "vW of edge %d (outside baro_axes) must be 0", c);
  }
  for (int c = 0; c < 3; ++c)
    if (!(box[c] > 2.0 * h->ff[6])) return fail(PIMD_EINVAL, "box edge %d must exceed 2 rc", c);
  CK(cudaStreamSynchronize(h->stream));
  std::memset(h->h_baro, 0, sizeof(h->h_baro));
  for (int c = 0; c < 3; ++c) h->h_baro[kBaroV + c] = vw3[c];
  for (int c = 0; c < 3; ++c) {
    h->h_baro[kBaroL + c] = box[c];
    h->h_baro[kBaroInvL + c] = 1.0 / box[c];
  }
  CK(cudaMemcpyAsync(h->baro, h->h_baro, sizeof(h->h_baro), cudaMemcpyHostToDevice, h->stream));
  pimd_status st = enqueue_forces(h, true, false);
  if (st != PIMD_OK) return st;
  return check_device_errors(h);
}

extern "C" pimd_status pimd_get_state(pimd_handle *h, double *x, double *v_nm, int64_t *step) {
  if (!h) return fail(PIMD_EINVAL, "handle is NULL");
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  const size_t bytes = (size_t)h->N * 3 * h->P * sizeof(double);
  if (h->precision == PIMD_PREC_SPLIT && (x || v_nm)) {
    pimd_status se = expand_split(h, false);
    if (se != PIMD_OK) return se;
  }
  if (x) {
    CK(launch_nap_to_pna(h->x, h->tmp, h->N, h->P, h->stream));
    CK(cudaMemcpyAsync(x, h->tmp, bytes, cudaMemcpyDeviceToHost, h->stream));
  }
  if (v_nm) {
    CK(launch_nap_to_pna(h->v, h->tmp, h->N, h->P, h->stream));
    CK(cudaMemcpyAsync(v_nm, h->tmp, bytes, cudaMemcpyDeviceToHost, h->stream));
  }
  if (step) *step = h->step;
  return check_device_errors(h);
}

extern "C" pimd_status pimd_set_state(pimd_handle *h, const double *x, const double *v_nm,
                                      int64_t step) {
  if (!h || !x || !v_nm) return fail(PIMD_EINVAL, "NULL argument");
  if (step < 0) return fail(PIMD_EINVAL, "step must be >= 0");
  if (h->latched != PIMD_OK) return fail(h->latched, "%s", h->latched_msg);
  pimd_status st = upload_state(h, x, v_nm);
  if (st != PIMD_OK) return st;
  h->step = step;
  CK(cudaMemcpyAsync(h->d_step, &h->step, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  st = enqueue_forces(h, true, false);
  if (st != PIMD_OK) return st;
  return check_device_errors(h);
}

extern "C" pimd_status pimd_set_kernel_timing(pimd_handle *h, int enable) {
  if (!h) return fail(PIMD_EINVAL, "handle is NULL");
  pimd_status st = flush_timing(h);
  if (st != PIMD_OK) return st;
  for (int k = 0; k < PIMD_NKINDS; ++k) {
    h->t_ms[k] = 0.0;
    h->t_n[k] = 0;
  }
  h->timing = enable != 0;
  return PIMD_OK;
}

extern "C" pimd_status pimd_kernel_times(pimd_handle *h, double *ms, int64_t *launches) {
  if (!h) return fail(PIMD_EINVAL, "handle is NULL");
  pimd_status st = flush_timing(h);
  if (st != PIMD_OK) return st;
  for (int k = 0; k < PIMD_NKINDS; ++k) {
    if (ms) ms[k] = h->t_ms[k];
    if (launches) launches[k] = h->t_n[k];
  }
  return PIMD_OK;
}

extern "C" int64_t pimd_kernel_launches(const pimd_handle *h) { return h ? h->launches : -1; }
