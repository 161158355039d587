// runtime.h -- host-side pieces shared by the single-system handle (capi.cu)
// and the multi-replica batch / server (batch.cu): argument validation, the
// precomputed mode tables, and error reporting.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "pimd.h"

namespace pimd {

// Per-mode tables of App. B / App. D for one (P, T, dt, params), FP64.
struct HostTables {
  std::vector<double> M, Mt;            // [P][P] Eq. (A1) and its transpose
  std::vector<double> Tf, Ti;           // [P/2 + 1][P] folded forward / inverse (ModeTables)
  std::vector<double> cA, sA, wsA;      // exact A step of length tA
  std::vector<double> c1, c2;           // O step of length tO
  std::vector<double> lam;              // Eq. (A2)
  std::vector<double> mu, imu;          // fictitious-mass factors m^(k) / m and their inverses
  double wn = 0.0, tA = 0.0, tO = 0.0;  // Eq. (2), A and O durations
};

void build_tables(int P, double T, double dt, const pimd_params &prm, HostTables &t);

// Checks of pimd_create (shared by pimd_create and the batch/server);
// fills *prm with the effective parameters (defaults, gamma0 -> tau).
pimd_status validate_create(const pimd_system *sys, int32_t P, double T, double dt, double gamma0,
                            const pimd_params *params, pimd_params *prm);

// EINVAL unless the keywords are the ones the split-precision, batch and
// server paths implement (method nmpimd, fmmode physical, fmass 1, fixcom 0).
pimd_status require_default_keywords(const pimd_params &prm, const char *where);

// Device memory through the optional pimd_set_allocator hooks (else cudaMalloc).
struct DevAllocator {
  pimd_alloc_fn alloc = nullptr;
  pimd_free_fn release = nullptr;
  void *ctx = nullptr;
};
DevAllocator current_allocator();
void *dev_alloc(const DevAllocator &a, size_t bytes, cudaStream_t s);
void dev_free(const DevAllocator &a, void *p, cudaStream_t s);

// The warp-item split-precision step for a single-system handle (bead
// counts 8, 16, 32, 64, 128): the handle's device arrays and the device buffers
// it carved for the step's descriptor, FP32 constants, TF32 fragment tables
// (split_warp_frag_float4 float4s), control words and completion counter.
struct SplitWarpSetup {
  int N, P, integrator, thermo;
  uint64_t seed;
  double dt, tA, c1_0, c2_0, box[3];
  double *xc, *v0;
  float *d, *vk, *F, *xcw;
  const double *inv_mm, *sigv;                  // device [N]
  const float *cAf, *sAf, *wsAf, *c1f, *c2f;    // device [P]
  double *cref, *ccur;                          // water-like: skin test, else null
  const double *M_host, *inv_mm_host, *sigv_host;
  void *desc;
  float4 *frag;
  float *inv_mmf, *sigvf;
  long long *ctl;
  unsigned *done;
};
size_t split_warp_desc_bytes();
size_t split_warp_frag_float4(int P);
bool split_warp_class(int P);
cudaError_t split_warp_setup(const SplitWarpSetup &w, cudaStream_t st);
cudaError_t launch_step_split_warp(const void *desc, int N, int P, const int64_t *step, int step_off, int first,
                                   double *blkmax, unsigned *done, cudaStream_t s);

pimd_status fail(pimd_status s, const char *fmt, ...);
void set_last_error(const char *msg);

}  // namespace pimd
