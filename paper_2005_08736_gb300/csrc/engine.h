// Internal interface between the host runtime (hgks_api.cu) and the kernel
// translation units (kernels_f32.cu, kernels_f64.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hgks.h"

namespace hgks {

struct GridDev;

// Device buffers and derived launch data of one context.
struct Engine {
  hgks_config cfg;
  cudaStream_t stream = nullptr;
  int n[3];
  int p[3];
  long long P = 0;  // padded cells per variable
  long long N = 0;  // interior cells
  // The two padded state buffers swap roles every step: q holds Q^n, the
  // step writes Q* and then Q^{n+1} into qs, and the host swaps q and qs
  // (with comp and comp2) after enqueuing the step, so that Q^n survives a
  // step whose result is non-physical.
  void* q = nullptr;     // padded state Q^n (deviation), 5 * P
  void* qs = nullptr;    // padded state Q*, then Q^{n+1}, 5 * P
  void* qx = nullptr;    // padded state with x slowest, [5][x][z][y], read by the x sweep
                         // (null: the x sweep reads q with pair loads along x)
  void* inc = nullptr;   // stage-1 increment, 5 * N
  void* comp = nullptr;  // FP32 compensation of Q^n, 5 * N (null for FP64)
  void* comp2 = nullptr; // FP32 compensation of Q^{n+1}, 5 * N (null for FP64)
  bool guard = true;     // the step's writes stop once the non-physical flag is set
  void* fd[3] = {nullptr, nullptr, nullptr};  // face fluxes per direction, 10 * faces
  void* w[3] = {nullptr, nullptr, nullptr};   // cell widths incl. ghosts, n + 6
  double* scal = nullptr;                      // [0] dt, [1] t, [2] step
  unsigned long long* dtmin = nullptr;
  int* flag = nullptr;
  double* part = nullptr;      // diagnostic partials
  double* diag_out = nullptr;  // 8 doubles
  double* io = nullptr;        // FP64 staging buffer, 5 * N
  void* adj_acc = nullptr;  // adjoint: padded cotangent accumulator, 5 * P
  void* adj_mu = nullptr;   // adjoint: cotangent of Q*, 5 * N
  void* adj_wL = nullptr;   // adjoint: cotangents of L and dL/dt, 5 * N each
  void* adj_wdL = nullptr;
  double* turb_part = nullptr;  // turbulence statistics: per-block partials
  double* turb_out = nullptr;   // and the final sums (allocated on first use)
  double* chan_out = nullptr;   // channel statistics: kChanSums sums per y row (first use)
  double* kin_w = nullptr;      // kinetic-energy functional: FP64 interior widths x, y, z (first use)
  // Statistics history (hgks_history_start): when hist_every > 0 the step
  // appends a record [t, step, kTurbSums sums] of the new state every
  // hist_every steps, while fewer than hist_cap records are stored.
  int hist_every = 0;
  int hist_cap = 0;
  double* hist = nullptr;
  int* hist_count = nullptr;
  int diag_blocks = 0;
  int cfl_blocks = 0;
  int sms = 152;  // multiprocessors of the device
  // Sweep launch choices (set by hgks_autotune): tile variant (0: the default
  // tile; 1, 2: wider tiles of the linear-weight smooth FP32 sweep; 3: the
  // 32x8 tile in packed FP32 pairs) and the number of face layers each CTA
  // marches through (0: automatic).
  int sweep_variant = 0;
  int sweep_chunk = 0;
};

// Turbulence statistics (turbulence.cuh): raw sums, each the sum over cells
// of the quantity times the cell volume.
enum TurbSum {
  TS_VOL = 0,      // volume
  TS_KE,           // 1/2 rho |U|^2
  TS_ENS,          // 1/2 rho |omega|^2
  TS_MU_SDSD,      // mu S^d : S^d
  TS_MUB_TH2,      // mu_b theta^2
  TS_P_TH,         // p theta
  TS_DRHO,         // rho - rho_ref
  TS_DRHO2,        // (rho - rho_ref)^2
  TS_Q2,           // |U|^2
  TS_MU_W2,        // mu |omega|^2
  TS_MU_TH2,       // mu theta^2
  TS_TH2,          // theta^2
  TS_W2,           // |omega|^2
  TS_DU2,          // (d_i U_i)^2, i = x, y, z (3 entries)
  TS_DU3 = TS_DU2 + 3,
  TS_DU4 = TS_DU3 + 3,
  kTurbSums = TS_DU4 + 3
};

// A history record: time, step count, then the kTurbSums sums.
constexpr int kHistStride = kTurbSums + 2;

// Channel statistics (turbulence.cuh, k_channel_rows): plane sums per y row
// of rho, rho U, U, V, W, U V, U U, T.
constexpr int kChanSums = 8;

// Kernel classes timed by hgks_profile_step (order of its output array).
enum KernelClass {
  KC_CFL = 0,        // CFL reduction and dt
  KC_GHOST = 1,      // ghost-cell fills
  KC_FACE = 2,       // unused (face fields are fused into the sweep)
  KC_FLUX1 = 3,      // sweep kernels of stage 1 (face fields, reconstruction, flux)
  KC_FLUX2 = 4,      // sweep kernels of stage 2
  KC_UPDATE = 5,     // divergence + S2O4 update
  KC_COUNT = 6
};

// Optional CUDA-event probe around kernel launches (profiling only; null in
// the captured step).
struct Probe {
  static constexpr int kMax = 64;
  cudaEvent_t start[kMax], stop[kMax];
  int cls[kMax];
  int n = 0;
  void begin(cudaStream_t s, int c) {
    if (n >= kMax) return;
    cls[n] = c;
    cudaEventRecord(start[n], s);
  }
  void end(cudaStream_t s) {
    if (n >= kMax) return;
    cudaEventRecord(stop[n], s);
    ++n;
  }
};

// Kernel sequences, implemented per floating type in kernels_f32.cu / kernels_f64.cu.
template <class T> cudaError_t enqueue_ghosts(const Engine& e, void* qbuf, Probe* probe = nullptr);
template <class T> cudaError_t enqueue_turbulence(const Engine& e);
// Append a history record of the state in qbuf (gated: only if the step
// count is a multiple of e.hist_every and the non-physical flag is clear).
template <class T> cudaError_t enqueue_history_record(const Engine& e, const void* qbuf, bool gated);
template <class T> cudaError_t enqueue_channel_rows(const Engine& e);
template <class T> cudaError_t enqueue_rhs_and_update(const Engine& e, int stage, Probe* probe = nullptr);
template <class T> cudaError_t enqueue_cfl(const Engine& e, const void* qbuf);
// The stage-1 sweep of direction d on e.q alone (tuning).
template <class T> cudaError_t enqueue_sweep_only(const Engine& e, int d);
template <class T> cudaError_t enqueue_diag(const Engine& e);
template <class T> cudaError_t enqueue_from_fp64(const Engine& e, const double* src, int conservative);
template <class T> cudaError_t enqueue_to_fp64(const Engine& e, double* dst);
// Adjoint of one S2O4 step at the state e.q with the step dt already in
// e.scal[0]: adj_out = (dQ^{n+1}/dQ^n)^T adj_in (FP64 device arrays, [5][N]).
// Number of tile variants of the sweep kernel for the context's configuration.
int sweep_variant_count(const Engine& e);
template <class T> cudaError_t enqueue_adjoint_step(const Engine& e, const double* adj_in,
                                                    double* adj_out);
// One S2O4 step of every member with one batched launch per phase (the
// members share precision, reconstruction, flux and tile variant and have
// no mass-flux force and no statistics history); Q^{n+1} of each ends in its
// qs.  On stream s.
template <class T> cudaError_t enqueue_batched_step(const std::vector<Engine*>& members, double dt_fixed,
                                                    cudaStream_t s);
cudaError_t enqueue_reset_scalars(const Engine& e);
// Swap the roles of the two state buffers (and the compensation buffers)
// after a step has been enqueued: Q^{n+1} is in qs.
inline void swap_state_buffers(Engine& e) {
  void* t = e.q;
  e.q = e.qs;
  e.qs = t;
  t = e.comp;
  e.comp = e.comp2;
  e.comp2 = t;
}
cudaError_t enqueue_set_dt(const Engine& e, double dt_fixed);
cudaError_t enqueue_advance_time(const Engine& e);

// Empty string if cfg is a valid problem statement, else the reason.
std::string validate_config(const hgks_config& cfg);

// Sizes (in elements) of the per-direction face buffers.
long long face_flux_elems(const Engine& e, int d);

}  // namespace hgks
