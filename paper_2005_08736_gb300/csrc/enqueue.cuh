// Kernel sequences of one S2O4 stage and of the reductions, per floating
// type.  Included once by kernels_f32.cu and once by kernels_f64.cu.
#pragma once

#include "engine.h"
#include "kernels.cuh"
#include "sweep.cuh"
#include "adjoint.cuh"
#include "turbulence.cuh"
#include "batch.cuh"

#include <algorithm>
#include <type_traits>
#include <vector>

namespace hgks {

inline GridDev grid_of(const Engine& e) {
  GridDev g;
  for (int c = 0; c < 3; ++c) {
    g.n[c] = e.n[c];
    g.p[c] = e.p[c];
  }
  g.P = e.P;
  g.N = e.N;
  return g;
}

template <class T>
Gas<T> gas_of(const hgks_config& c) {
  Gas<T> g;
  g.gamma = T(c.gamma);
  g.gm1 = T(c.gamma - 1.0);
  g.K = T((5.0 - 3.0 * c.gamma) / (c.gamma - 1.0));
  g.pr_fix = T(1.0 / c.prandtl - 1.0);
  g.visc_law = c.visc;
  g.mu_ref = T(c.mu_ref);
  g.T_ref_inv = T(1.0 / c.T_ref);
  g.visc_exp = T(c.visc_exp);
  g.tau_num_C = c.flux == HGKS_FLUX_FULL ? T(c.tau_num_C) : T(0);
  g.rho_r = T(c.rho_ref);
  g.p_r = T(c.p_ref);
  g.h_r = T(c.gamma / (c.gamma - 1.0) * c.p_ref);
  return g;
}

// Kernel MODE of a configuration: the reconstruction, + 2 for WENO in
// characteristic variables (with linear weights the projection changes
// nothing, so it is skipped).
inline int sweep_mode(const hgks_config& c) {
  return c.recon + (c.recon_vars == 1 && c.recon != HGKS_RECON_LINEAR ? 2 : 0);
}

inline unsigned blocks_for(long long n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

template <class T>
cudaError_t enqueue_ghosts(const Engine& e, void* qbuf, Probe* probe) {
  T* q = static_cast<T*>(qbuf);
  const GridDev g = grid_of(e);
  const int th = 256;
  if (probe) probe->begin(e.stream, KC_GHOST);
  k_ghost_x<T><<<blocks_for(6LL * g.n[1] * g.n[2], th), th, 0, e.stream>>>(q, g);
  k_ghost_y<T><<<blocks_for(6LL * g.p[0] * g.n[2], th), th, 0, e.stream>>>(
      q, g, e.cfg.bc_y == HGKS_BC_WALL_ISOTHERMAL, gas_of<T>(e.cfg), T(e.cfg.T_wall));
  k_ghost_z<T><<<blocks_for(6LL * g.p[0] * g.p[1], th), th, 0, e.stream>>>(q, g);
  if (probe) probe->end(e.stream);
  return cudaGetLastError();
}

// Tile of the sweep kernel per precision and flux: TP x TS faces, sized so
// that the shared-memory staging fits and every tile gives 1, 2 or 4 threads
// per face.
// NL face layers share one face-field pass (phase 1).
template <class T, int FLUX> struct SweepTile { static constexpr int TP = 16, TS = 8, NL = 4; };
template <> struct SweepTile<float, FLUX_FULL> { static constexpr int TP = 16, TS = 8, NL = 2; };
template <> struct SweepTile<double, FLUX_SMOOTH> { static constexpr int TP = 16, TS = 8, NL = 2; };
template <> struct SweepTile<double, FLUX_FULL> { static constexpr int TP = 8, TS = 8, NL = 2; };

// Arguments and grid (gx, gy, gz) of the sweep of direction d on the padded
// state q with a TP x TS tile and NL layers per face-field pass.
template <class T, int TP, int TS, int NL>
SweepArgs<T> sweep_args(const Engine& e, const T* q, int d, int& gx, int& gy, int& gz) {
  const GridDev g = grid_of(e);
  SweepArgs<T> a;
  // The x sweep reads the copy of the state with x slowest (k_transpose_x).
  const bool xt = d == 0 && e.qx != nullptr;
  a.q = xt ? static_cast<const T*>(e.qx) : q;
  a.xt = xt ? 1 : 0;
  a.fd = static_cast<T*>(e.fd[d]);
  a.wn = static_cast<const T*>(e.w[d]);
  a.wt1 = static_cast<const T*>(e.w[(d + 1) % 3]);
  a.wt2 = static_cast<const T*>(e.w[(d + 2) % 3]);
  a.scal = e.scal;
  a.g = g;
  a.d = d;
  a.gas = gas_of<T>(e.cfg);
  const int P = d == 0 ? 1 : 0, S = d == 2 ? 1 : 2;
  gx = (g.n[P] + TP - 1) / TP;
  gy = (g.n[S] + TS - 1) / TS;
  // Chunk the march along d so that the grid holds several waves of CTAs.
  const int layers = g.n[d] + 1;
  int chunk = e.sweep_chunk;
  if (chunk <= 0) {
    const int want_chunks = (4 * e.sms + gx * gy - 1) / (gx * gy);
    chunk = (layers + want_chunks - 1) / want_chunks;
    if (chunk < 2 * NL) chunk = 2 * NL;
  }
  chunk = (chunk + NL - 1) / NL * NL;
  a.chunk = chunk;
  gz = (layers + chunk - 1) / chunk;
  return a;
}

template <class T, int MODE, int FLUX, int STAGE, int TP, int TS, int NL, bool PK = false>
cudaError_t launch_sweep_tile(const Engine& e, const T* q, int d) {
  const GridDev g = grid_of(e);
  if (d == 0 && e.qx != nullptr) {
    const dim3 tgrid((g.p[0] + 31) / 32, (g.p[1] + 31) / 32, g.p[2]);
    k_transpose_x<T><<<tgrid, 256, 0, e.stream>>>(q, static_cast<T*>(e.qx), g);
  }
  int gx, gy, gz;
  const SweepArgs<T> a = sweep_args<T, TP, TS, NL>(e, q, d, gx, gy, gz);
  constexpr size_t smem = sweep_smem_bytes<T, MODE, FLUX, TP, TS, NL>();
  auto kern = k_sweep<T, MODE, FLUX, STAGE, TP, TS, NL, PK>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<dim3(gx, gy, gz), sweep_threads(TP, TS), smem, e.stream>>>(a);
  return cudaGetLastError();
}

// Tile variants: 0 is SweepTile; the linear-weight smooth FP32 sweep also has
// 32x8 and 16x16 tiles with two layers per face-field pass (1, 2) and the
// 32x8 tile with the packed FP32-pair last phase (3).
template <class T, int MODE, int FLUX, int STAGE>
cudaError_t launch_sweep(const Engine& e, const T* q, int d) {
  if constexpr (std::is_same<T, float>::value && MODE == RECON_LINEAR && FLUX == FLUX_SMOOTH) {
    if (e.sweep_variant == 1) return launch_sweep_tile<T, MODE, FLUX, STAGE, 32, 8, 2>(e, q, d);
    if (e.sweep_variant == 2) return launch_sweep_tile<T, MODE, FLUX, STAGE, 16, 16, 2>(e, q, d);
    if (e.sweep_variant == 3) return launch_sweep_tile<T, MODE, FLUX, STAGE, 32, 8, 2, true>(e, q, d);

  }
  return launch_sweep_tile<T, MODE, FLUX, STAGE, SweepTile<T, FLUX>::TP, SweepTile<T, FLUX>::TS,
                           SweepTile<T, FLUX>::NL>(e, q, d);
}

template <class T, int MODE, int FLUX>
cudaError_t launch_all_directions(const Engine& e, const T* q, int stage, Probe* probe) {
  for (int d = 0; d < 3; ++d) {
    if (probe) probe->begin(e.stream, stage == 1 ? KC_FLUX1 : KC_FLUX2);
    const cudaError_t err = stage == 1 ? launch_sweep<T, MODE, FLUX, 1>(e, q, d)
                                       : launch_sweep<T, MODE, FLUX, 2>(e, q, d);
    if (probe) probe->end(e.stream);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Arguments of the update kernel on the context's current buffers.
template <class T>
UpdateArgs<T> update_args(const Engine& e) {
  UpdateArgs<T> ua;
  ua.q = static_cast<T*>(e.q);
  ua.qs = static_cast<T*>(e.qs);
  ua.inc = static_cast<T*>(e.inc);
  ua.comp = static_cast<T*>(e.comp);
  ua.comp_out = static_cast<T*>(e.comp2);
  ua.flag = e.guard ? e.flag : nullptr;
  ua.fx = static_cast<const T*>(e.fd[0]);
  ua.fy = static_cast<const T*>(e.fd[1]);
  ua.fz = static_cast<const T*>(e.fd[2]);
  ua.wx = static_cast<const T*>(e.w[0]);
  ua.wy = static_cast<const T*>(e.w[1]);
  ua.wz = static_cast<const T*>(e.w[2]);
  ua.scal = e.scal;
  ua.g = grid_of(e);
  const bool mass_flux = e.cfg.force_mode == HGKS_FORCE_MASS_FLUX;
  ua.force_x = mass_flux ? T(0) : T(e.cfg.force_x);
  ua.rho_r = T(e.cfg.rho_ref);
  return ua;
}

template <class T>
cudaError_t enqueue_rhs_and_update(const Engine& e, int stage, Probe* probe) {
  T* qin = static_cast<T*>(stage == 1 ? e.q : e.qs);
  cudaError_t err = enqueue_ghosts<T>(e, qin, probe);
  if (err != cudaSuccess) return err;
  const int mode = sweep_mode(e.cfg), flux = e.cfg.flux;
#define HGKS_DISPATCH(M, F) \
  if (mode == M && flux == F) err = launch_all_directions<T, M, F>(e, qin, stage, probe);
  HGKS_DISPATCH(0, 0) HGKS_DISPATCH(1, 0) HGKS_DISPATCH(2, 0) HGKS_DISPATCH(3, 0) HGKS_DISPATCH(4, 0)
  HGKS_DISPATCH(0, 1) HGKS_DISPATCH(1, 1) HGKS_DISPATCH(2, 1) HGKS_DISPATCH(3, 1) HGKS_DISPATCH(4, 1)
#undef HGKS_DISPATCH
  if (err != cudaSuccess) return err;
  const UpdateArgs<T> ua = update_args<T>(e);
  const bool mass_flux = e.cfg.force_mode == HGKS_FORCE_MASS_FLUX;
  if (probe) probe->begin(e.stream, KC_UPDATE);
  const dim3 ugrid((e.n[0] + kUpdTX - 1) / kUpdTX, (e.n[1] + kUpdTY - 1) / kUpdTY, e.n[2]);
  if (stage == 1)
    k_update<T, 1><<<ugrid, kUpdTX * kUpdTY, 0, e.stream>>>(ua);
  else
    k_update<T, 2><<<ugrid, kUpdTX * kUpdTY, 0, e.stream>>>(ua);
  if (mass_flux && stage == 2) {
    // Sec. 3.3: the force that keeps the volume integral of rho U at its
    // target, on Q~^{n+1} (in qs, compensation in comp2), with rho^n and
    // (rho U)^n read from Q^n (q).
    const GridDev g = grid_of(e);
    k_massflux_sums<T><<<e.diag_blocks, 256, 0, e.stream>>>(
        ua.qs, ua.q, ua.comp_out, g, ua.wx, ua.wy, ua.wz, e.cfg.rho_ref, e.part, ua.flag);
    k_massflux_force<<<1, 256, 0, e.stream>>>(e.part, e.diag_blocks, e.cfg.mass_flux, e.scal, ua.flag);
    k_force_apply<T><<<blocks_for(e.N, 256), 256, 0, e.stream>>>(ua.qs, ua.q, ua.comp_out, g,
                                                                 e.cfg.rho_ref, e.scal, ua.flag);
  }
  if (probe) probe->end(e.stream);
  return cudaGetLastError();
}

template <class T>
cudaError_t enqueue_sweep_only(const Engine& e, int d) {
  const T* q = static_cast<const T*>(e.q);
  const int mode = sweep_mode(e.cfg), flux = e.cfg.flux;
#define HGKS_SW(M, F) \
  if (mode == M && flux == F) return launch_sweep<T, M, F, 1>(e, q, d);
  HGKS_SW(0, 0) HGKS_SW(1, 0) HGKS_SW(2, 0) HGKS_SW(3, 0) HGKS_SW(4, 0)
  HGKS_SW(0, 1) HGKS_SW(1, 1) HGKS_SW(2, 1) HGKS_SW(3, 1) HGKS_SW(4, 1)
#undef HGKS_SW
  return cudaErrorInvalidValue;
}

template <class T>
cudaError_t enqueue_cfl(const Engine& e, const void* qbuf) {
  k_cfl<T><<<e.cfl_blocks, 256, 0, e.stream>>>(
      static_cast<const T*>(qbuf), grid_of(e), static_cast<const T*>(e.w[0]),
      static_cast<const T*>(e.w[1]), static_cast<const T*>(e.w[2]), e.cfg.rho_ref, e.cfg.p_ref,
      e.cfg.gamma, e.dtmin, e.flag);
  return cudaGetLastError();
}

template <class T>
cudaError_t enqueue_diag(const Engine& e) {
  k_diag<T><<<e.diag_blocks, 256, 0, e.stream>>>(
      static_cast<const T*>(e.q), grid_of(e), static_cast<const T*>(e.w[0]),
      static_cast<const T*>(e.w[1]), static_cast<const T*>(e.w[2]), e.cfg.rho_ref, e.cfg.p_ref,
      e.cfg.gamma, e.part);
  k_diag_final<<<1, 256, 0, e.stream>>>(e.part, e.diag_blocks, e.diag_out);
  return cudaGetLastError();
}

inline TurbArgs turb_args(const hgks_config& c, const int n[3]) {
  TurbArgs a;
  const double L[3] = {c.lx, c.ly, c.lz};
  double vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    const double h = L[d] / n[d];
    a.inv60h[d] = 1.0 / (60.0 * h);
    vol *= h;
  }
  a.vol = vol;
  a.rho_r = c.rho_ref;
  a.E_r = c.p_ref / (c.gamma - 1.0);
  a.gm1 = c.gamma - 1.0;
  a.visc_law = c.visc;
  a.mu_ref = c.mu_ref;
  a.T_ref_inv = 1.0 / c.T_ref;
  a.visc_exp = c.visc_exp;
  const double K = (5.0 - 3.0 * c.gamma) / (c.gamma - 1.0);
  a.mub_ratio = 2.0 * K / (3.0 * (K + 3.0));
  return a;
}

// Turbulence statistics of Q^n: per-block FP64 sums, final sum into
// e.turb_out (kTurbSums doubles).
template <class T>
cudaError_t enqueue_turbulence(const Engine& e) {
  const HistGate gate{e.scal, nullptr, 0};
  k_turb<T><<<e.diag_blocks, 256, 0, e.stream>>>(static_cast<const T*>(e.q), grid_of(e),
                                                 turb_args(e.cfg, e.n), e.turb_part, gate);
  const TurbSink sink{e.turb_out, nullptr, nullptr, 0};
  k_turb_final<<<1, 256, 0, e.stream>>>(e.turb_part, e.diag_blocks, sink, gate);
  return cudaGetLastError();
}

// A record of the statistics history from the state in qbuf.
template <class T>
cudaError_t enqueue_history_record(const Engine& e, const void* qbuf, bool gated) {
  const HistGate gate{e.scal, e.flag, gated ? e.hist_every : 0};
  k_turb<T><<<e.diag_blocks, 256, 0, e.stream>>>(static_cast<const T*>(qbuf), grid_of(e),
                                                 turb_args(e.cfg, e.n), e.turb_part, gate);
  const TurbSink sink{nullptr, e.hist, e.hist_count, e.hist_cap};
  k_turb_final<<<1, 256, 0, e.stream>>>(e.turb_part, e.diag_blocks, sink, gate);
  return cudaGetLastError();
}

// Channel plane averages: kChanSums FP64 sums per y row into e.chan_out.
template <class T>
cudaError_t enqueue_channel_rows(const Engine& e) {
  const hgks_config& c = e.cfg;
  k_channel_rows<T><<<e.n[1], 256, 0, e.stream>>>(static_cast<const T*>(e.q), grid_of(e), c.rho_ref,
                                                  c.p_ref, c.gamma - 1.0, e.chan_out);
  return cudaGetLastError();
}

template <class T>
cudaError_t enqueue_from_fp64(const Engine& e, const double* src, int conservative) {
  const GridDev g = grid_of(e);
  const dim3 grid((g.n[0] + 255) / 256, g.n[1], g.n[2]);
  const double inv_gm1 = 1.0 / (e.cfg.gamma - 1.0);
  k_from_prim<T><<<grid, 256, 0, e.stream>>>(src, static_cast<T*>(e.q), g, e.cfg.rho_ref,
                                              e.cfg.p_ref / (e.cfg.gamma - 1.0), inv_gm1, conservative);
  return cudaGetLastError();
}

template <class T>
cudaError_t enqueue_to_fp64(const Engine& e, double* dst) {
  const GridDev g = grid_of(e);
  const dim3 grid((g.n[0] + 255) / 256, g.n[1], g.n[2]);
  k_to_cons<T><<<grid, 256, 0, e.stream>>>(static_cast<const T*>(e.q), dst, g, e.cfg.rho_ref,
                                            e.cfg.p_ref / (e.cfg.gamma - 1.0));
  return cudaGetLastError();
}

// Tiles of the adjoint sweep: four shared-memory planes (face fields, t1 pass
// and their cotangents) must fit one CTA.
template <class T, int FLUX> struct AdjTile { static constexpr int TP = 16, TS = 8, NT = 256; };
template <> struct AdjTile<float, FLUX_FULL> { static constexpr int TP = 8, TS = 8, NT = 256; };
template <> struct AdjTile<double, FLUX_FULL> { static constexpr int TP = 8, TS = 4, NT = 128; };

template <class T, int MODE, int FLUX>
cudaError_t launch_adjoint_sweeps(const Engine& e, const T* q, const T* wL, const T* wdL) {
  constexpr int TP = AdjTile<T, FLUX>::TP, TS = AdjTile<T, FLUX>::TS, NT = AdjTile<T, FLUX>::NT;
  const GridDev g = grid_of(e);
  constexpr size_t smem = adj_smem_bytes<T, FLUX, TP, TS>();
  auto kern = k_sweep_adj<T, MODE, FLUX, TP, TS, NT>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  for (int d = 0; d < 3; ++d) {
    AdjArgs<T> a;
    a.q = q;
    a.wL = wL;
    a.wdL = wdL;
    a.acc = static_cast<T*>(e.adj_acc);
    a.wn = static_cast<const T*>(e.w[d]);
    a.wt1 = static_cast<const T*>(e.w[(d + 1) % 3]);
    a.wt2 = static_cast<const T*>(e.w[(d + 2) % 3]);
    a.scal = e.scal;
    a.g = g;
    a.d = d;
    a.gas = gas_of<T>(e.cfg);
    const int P = d == 0 ? 1 : 0, S = d == 2 ? 1 : 2;
    const int gx = (g.n[P] + TP - 1) / TP, gy = (g.n[S] + TS - 1) / TS;
    const int layers = g.n[d] + 1;
    const int want_chunks = (4 * e.sms + gx * gy - 1) / (gx * gy);
    int chunk = (layers + want_chunks - 1) / want_chunks;
    if (chunk < 1) chunk = 1;
    a.chunk = chunk;
    const int gz = (layers + chunk - 1) / chunk;
    kern<<<dim3(gx, gy, gz), NT, smem, e.stream>>>(a);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  T* acc = static_cast<T*>(e.adj_acc);
  k_fold_ghosts_z<T><<<blocks_for(6LL * g.p[0] * g.p[1], 256), 256, 0, e.stream>>>(acc, g);
  k_fold_ghosts_y<T><<<blocks_for(6LL * g.p[0] * g.n[2], 256), 256, 0, e.stream>>>(acc, g);
  k_fold_ghosts_x<T><<<blocks_for(6LL * g.n[1] * g.n[2], 256), 256, 0, e.stream>>>(acc, g);
  return cudaGetLastError();
}

template <class T>
cudaError_t dispatch_adjoint_sweeps(const Engine& e, const T* q, const T* wL, const T* wdL) {
  const int mode = e.cfg.recon, flux = e.cfg.flux;
#define HGKS_ADJ(M, F) \
  if (mode == M && flux == F) return launch_adjoint_sweeps<T, M, F>(e, q, wL, wdL);
  HGKS_ADJ(0, 0) HGKS_ADJ(1, 0) HGKS_ADJ(2, 0)
  HGKS_ADJ(0, 1) HGKS_ADJ(1, 1) HGKS_ADJ(2, 1)
#undef HGKS_ADJ
  return cudaErrorInvalidValue;
}

template <class T>
cudaError_t enqueue_adjoint_step(const Engine& e, const double* adj_in, double* adj_out) {
  const GridDev g = grid_of(e);
  T* acc = static_cast<T*>(e.adj_acc);
  T* mu = static_cast<T*>(e.adj_mu);
  T* wL = static_cast<T*>(e.adj_wL);
  T* wdL = static_cast<T*>(e.adj_wdL);
  const size_t accb = 5 * (size_t)e.P * sizeof(T);
  // Q* = Q^n + dt/2 L + dt^2/8 dL (also fills the ghost cells of Q^n); the
  // step's non-physical guard does not apply here.
  Engine ea = e;
  ea.guard = false;
  cudaError_t err = enqueue_rhs_and_update<T>(ea, 1);
  if (err != cudaSuccess) return err;
  err = enqueue_ghosts<T>(e, e.qs);
  if (err != cudaSuccess) return err;
  // mu* = (d dL(Q*)/dQ*)^T (dt^2/3 lam).
  err = cudaMemsetAsync(acc, 0, accb, e.stream);
  if (err != cudaSuccess) return err;
  k_adj_combine<T><<<blocks_for(e.N, 256), 256, 0, e.stream>>>(0, adj_in, acc, mu, wL, wdL, nullptr,
                                                               e.scal, g);
  err = dispatch_adjoint_sweeps<T>(e, static_cast<const T*>(e.qs), nullptr, wdL);
  if (err != cudaSuccess) return err;
  // Cotangents of L(Q^n) and dL(Q^n), then their VJP at Q^n.
  k_adj_combine<T><<<blocks_for(e.N, 256), 256, 0, e.stream>>>(1, adj_in, acc, mu, wL, wdL, nullptr,
                                                               e.scal, g);
  err = cudaMemsetAsync(acc, 0, accb, e.stream);
  if (err != cudaSuccess) return err;
  err = dispatch_adjoint_sweeps<T>(e, static_cast<const T*>(e.q), wL, wdL);
  if (err != cudaSuccess) return err;
  k_adj_combine<T><<<blocks_for(e.N, 256), 256, 0, e.stream>>>(2, adj_in, acc, mu, wL, wdL, adj_out,
                                                               e.scal, g);
  return cudaGetLastError();
}

// ---------------------------------------------------------- batched step ---
// One S2O4 step of every member (same precision, reconstruction, flux, tile
// variant; constant or no body force) with one batched launch per phase
// (batch.cuh) on stream s.  Each member's arguments are those of its own
// launches: its buffers, grid, chunking and non-physical guard.

// Launch Job over the members (in groups of kBatchMax): job i runs blocks[i] blocks.
template <class Job>
cudaError_t launch_batched(const std::vector<Job>& jobs, const std::vector<int>& blocks, size_t smem,
                           cudaStream_t s) {
  auto kern = k_batched<Job>;
  if (smem > 0) {
    const cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  for (size_t i0 = 0; i0 < jobs.size(); i0 += kBatchMax) {
    BatchTable<Job> t;
    t.n = (int)std::min<size_t>(kBatchMax, jobs.size() - i0);
    int acc = 0;
    for (int m = 0; m < t.n; ++m) {
      t.start[m] = acc;
      t.job[m] = jobs[i0 + m];
      acc += blocks[i0 + m];
    }
    t.start[t.n] = acc;
    if (acc == 0) continue;
    kern<<<acc, Job::kThreads, smem, s>>>(t);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <class T, int MODE, int FLUX, int STAGE, int TP, int TS, int NL, bool PK>
cudaError_t batched_sweeps(const std::vector<Engine*>& ms, int stage, cudaStream_t s) {
  for (int d = 0; d < 3; ++d) {
    if (d == 0) {
      std::vector<TransposeJob<T>> tj;
      std::vector<int> tb;
      for (Engine* e : ms) {
        if (!e->qx) continue;
        const GridDev g = grid_of(*e);
        const int gx = (g.p[0] + 31) / 32, gy = (g.p[1] + 31) / 32;
        tj.push_back({static_cast<const T*>(stage == 1 ? e->q : e->qs), static_cast<T*>(e->qx), g, gx, gy});
        tb.push_back(gx * gy * g.p[2]);
      }
      const cudaError_t err = launch_batched(tj, tb, 0, s);
      if (err != cudaSuccess) return err;
    }
    using Job = SweepJob<T, MODE, FLUX, STAGE, TP, TS, NL, PK>;
    std::vector<Job> jobs;
    std::vector<int> blocks;
    for (Engine* e : ms) {
      int gx, gy, gz;
      Job j;
      j.a = sweep_args<T, TP, TS, NL>(*e, static_cast<const T*>(stage == 1 ? e->q : e->qs), d, gx, gy, gz);
      j.gx = gx;
      j.gy = gy;
      jobs.push_back(j);
      blocks.push_back(gx * gy * gz);
    }
    const cudaError_t err = launch_batched(jobs, blocks, sweep_smem_bytes<T, MODE, FLUX, TP, TS, NL>(), s);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <class T, int MODE, int FLUX, int STAGE>
cudaError_t batched_sweeps_variant(const std::vector<Engine*>& ms, int stage, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value && MODE == RECON_LINEAR && FLUX == FLUX_SMOOTH) {
    const int v = ms[0]->sweep_variant;
    if (v == 1) return batched_sweeps<T, MODE, FLUX, STAGE, 32, 8, 2, false>(ms, stage, s);
    if (v == 2) return batched_sweeps<T, MODE, FLUX, STAGE, 16, 16, 2, false>(ms, stage, s);
    if (v == 3) return batched_sweeps<T, MODE, FLUX, STAGE, 32, 8, 2, true>(ms, stage, s);
  }
  return batched_sweeps<T, MODE, FLUX, STAGE, SweepTile<T, FLUX>::TP, SweepTile<T, FLUX>::TS,
                        SweepTile<T, FLUX>::NL, false>(ms, stage, s);
}

template <class T>
cudaError_t enqueue_batched_step(const std::vector<Engine*>& ms, double dt_fixed, cudaStream_t s) {
  cudaError_t err;
  {
    std::vector<CflJob<T>> jobs;
    std::vector<int> blocks;
    for (Engine* e : ms) {
      jobs.push_back({static_cast<const T*>(e->q), grid_of(*e), static_cast<const T*>(e->w[0]),
                      static_cast<const T*>(e->w[1]), static_cast<const T*>(e->w[2]), e->cfg.rho_ref,
                      e->cfg.p_ref, e->cfg.gamma, e->dtmin, e->flag, e->cfl_blocks});
      blocks.push_back(e->cfl_blocks);
    }
    if ((err = launch_batched(jobs, blocks, 0, s)) != cudaSuccess) return err;
  }
  {
    std::vector<SetDtJob> jobs;
    std::vector<int> blocks;
    for (Engine* e : ms) {
      jobs.push_back({e->scal, e->dtmin, e->cfg.cfl, dt_fixed, e->guard ? e->flag : nullptr});
      blocks.push_back(1);
    }
    if ((err = launch_batched(jobs, blocks, 0, s)) != cudaSuccess) return err;
  }
  const int mode = sweep_mode(ms[0]->cfg), flux = ms[0]->cfg.flux;
  for (int stage = 1; stage <= 2; ++stage) {
    std::vector<GhostXJob<T>> gxj;
    std::vector<GhostYJob<T>> gyj;
    std::vector<GhostZJob<T>> gzj;
    std::vector<int> bx, by, bz;
    for (Engine* e : ms) {
      T* q = static_cast<T*>(stage == 1 ? e->q : e->qs);
      const GridDev g = grid_of(*e);
      gxj.push_back({q, g});
      bx.push_back(blocks_for(6LL * g.n[1] * g.n[2], 256));
      gyj.push_back({q, g, e->cfg.bc_y == HGKS_BC_WALL_ISOTHERMAL ? 1 : 0, gas_of<T>(e->cfg), T(e->cfg.T_wall)});
      by.push_back(blocks_for(6LL * g.p[0] * g.n[2], 256));
      gzj.push_back({q, g});
      bz.push_back(blocks_for(6LL * g.p[0] * g.p[1], 256));
    }
    if ((err = launch_batched(gxj, bx, 0, s)) != cudaSuccess) return err;
    if ((err = launch_batched(gyj, by, 0, s)) != cudaSuccess) return err;
    if ((err = launch_batched(gzj, bz, 0, s)) != cudaSuccess) return err;
    err = cudaErrorInvalidValue;
#define HGKS_BSW(M, F)                                                                           \
    if (mode == M && flux == F)                                                                  \
      err = stage == 1 ? batched_sweeps_variant<T, M, F, 1>(ms, stage, s)                        \
                       : batched_sweeps_variant<T, M, F, 2>(ms, stage, s);
    HGKS_BSW(0, 0) HGKS_BSW(1, 0) HGKS_BSW(2, 0) HGKS_BSW(3, 0) HGKS_BSW(4, 0)
    HGKS_BSW(0, 1) HGKS_BSW(1, 1) HGKS_BSW(2, 1) HGKS_BSW(3, 1) HGKS_BSW(4, 1)
#undef HGKS_BSW
    if (err != cudaSuccess) return err;
    std::vector<int> ub;
    if (stage == 1) {
      std::vector<UpdateJob<T, 1>> uj;
      for (Engine* e : ms) {
        const int gx = (e->n[0] + kUpdTX - 1) / kUpdTX, gy = (e->n[1] + kUpdTY - 1) / kUpdTY;
        uj.push_back({update_args<T>(*e), gx, gy});
        ub.push_back(gx * gy * e->n[2]);
      }
      err = launch_batched(uj, ub, 0, s);
    } else {
      std::vector<UpdateJob<T, 2>> uj;
      for (Engine* e : ms) {
        const int gx = (e->n[0] + kUpdTX - 1) / kUpdTX, gy = (e->n[1] + kUpdTY - 1) / kUpdTY;
        uj.push_back({update_args<T>(*e), gx, gy});
        ub.push_back(gx * gy * e->n[2]);
      }
      err = launch_batched(uj, ub, 0, s);
    }
    if (err != cudaSuccess) return err;
  }
  std::vector<AdvanceJob> aj;
  std::vector<int> ab;
  for (Engine* e : ms) {
    aj.push_back({e->scal, e->guard ? e->flag : nullptr});
    ab.push_back(1);
  }
  return launch_batched(aj, ab, 0, s);
}

#define HGKS_INSTANTIATE(T)                                                  \
  template cudaError_t enqueue_ghosts<T>(const Engine&, void*, Probe*);      \
  template cudaError_t enqueue_rhs_and_update<T>(const Engine&, int, Probe*); \
  template cudaError_t enqueue_cfl<T>(const Engine&, const void*);           \
  template cudaError_t enqueue_sweep_only<T>(const Engine&, int);            \
  template cudaError_t enqueue_diag<T>(const Engine&);                       \
  template cudaError_t enqueue_turbulence<T>(const Engine&);                 \
  template cudaError_t enqueue_history_record<T>(const Engine&, const void*, bool); \
  template cudaError_t enqueue_channel_rows<T>(const Engine&);               \
  template cudaError_t enqueue_from_fp64<T>(const Engine&, const double*, int); \
  template cudaError_t enqueue_to_fp64<T>(const Engine&, double*);           \
  template cudaError_t enqueue_adjoint_step<T>(const Engine&, const double*, double*); \
  template cudaError_t enqueue_batched_step<T>(const std::vector<Engine*>&, double, cudaStream_t);

}  // namespace hgks
