// Kernels of one S2O4 step of the high-order gas-kinetic scheme (Cao, Pan &
// Xu, arXiv:2005.08736), templated on the storage/arithmetic type T.
//
// State layout in HBM: structure of arrays, 5 planes (rho, rho U, rho V,
// rho W, rho E) of (nx+6)(ny+6)(nz+6) cells, x fastest, 3 ghost layers on
// every side, holding deviations from the reference state at rest.
//
// Per stage, the fused sweep kernel (sweep.cuh) writes the face fluxes of
// each direction; k_update then forms L = -(1/|Omega|) sum F (Eq. (4)) and
// the S2O4 stage (Eq. (6)).  Ghost fills, the CFL and diagnostic reductions
// and the state conversions are here too.
#pragma once

#include <cstdint>

#include "recon.cuh"

namespace hgks {

constexpr int kGhost = 3;

struct GridDev {
  int n[3];       // interior cells
  int p[3];       // padded extents n + 6
  long long P;    // padded cells per variable
  long long N;    // interior cells
};

__host__ __device__ __forceinline__ long long pad_index(const GridDev& g, int x, int y, int z) {
  return ((long long)(z + kGhost) * g.p[1] + (y + kGhost)) * g.p[0] + (x + kGhost);
}

// Extents and offsets of the face-field box of direction d: faces 0..n_d
// along d, tangential rows -2..n+1 along the two other axes.
struct FaceBox {
  int r[3], o[3];
  long long size;
};
__host__ __device__ __forceinline__ FaceBox face_box(const GridDev& g, int d, int tang_halo) {
  FaceBox b;
  for (int c = 0; c < 3; ++c) {
    if (c == d) {
      b.r[c] = g.n[c] + 1;
      b.o[c] = 0;
    } else {
      b.r[c] = g.n[c] + 2 * tang_halo;
      b.o[c] = -tang_halo;
    }
  }
  b.size = (long long)b.r[0] * b.r[1] * b.r[2];
  return b;
}

// ------------------------------------------------------------- ghost cells ---

// The ghost fills and the CFL reduction are bodies over explicit block
// coordinates (device functions) with thin __global__ wrappers; the update,
// the transposed copy and the sweep keep their bodies in the kernels, as
// included texts (update_body.inc, transpose_body.inc, sweep_body.inc).  The
// ensemble's batched launches (batch.cuh) run the same bodies for many
// instances in one grid.

// x ghosts (periodic) for interior y, z; tid indexes the ghost cells.
template <class T>
__device__ __forceinline__ void ghost_x_cells(T* __restrict__ q, const GridDev& g, long long tid) {
  const long long total = 6LL * g.n[1] * g.n[2];
  if (tid >= total) return;
  const int m = int(tid % 6);
  const long long r = tid / 6;
  const int y = int(r % g.n[1]), z = int(r / g.n[1]);
  const int x = m < 3 ? -1 - m : g.n[0] + (m - 3);
  const int src = m < 3 ? g.n[0] - 1 - m : m - 3;
  const long long dst = pad_index(g, x, y, z), s = pad_index(g, src, y, z);
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v * g.P + dst] = q[v * g.P + s];
}
template <class T>
__global__ void k_ghost_x(T* __restrict__ q, GridDev g) {
  ghost_x_cells(q, g, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// y ghosts for all x (ghosts included) and interior z: periodic, or the
// isothermal no-slip wall (Sec. 3.3): the ghost mirrors interior cell m with
// velocity negated, equal pressure and T_g = 2 T_w - T_m (floored at T_w/2).
template <class T>
__device__ __forceinline__ void ghost_y_cells(T* __restrict__ q, const GridDev& g, int wall,
                                              const Gas<T>& gas, T T_wall, long long tid) {
  const long long total = 6LL * g.p[0] * g.n[2];
  if (tid >= total) return;
  const int x = int(tid % g.p[0]) - kGhost;
  const long long r = tid / g.p[0];
  const int m = int(r % 6), z = int(r / 6);
  const int y = m < 3 ? -1 - m : g.n[1] + (m - 3);
  const long long dst = pad_index(g, x, y, z);
  if (!wall) {
    const int src = m < 3 ? g.n[1] - 1 - m : m - 3;
    const long long s = pad_index(g, x, src, z);
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v * g.P + dst] = q[v * g.P + s];
    return;
  }
  const int src = m < 3 ? m : g.n[1] - 1 - (m - 3);
  const long long s = pad_index(g, x, src, z);
  T dq[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) dq[v] = q[v * g.P + s];
  const Prim<T> st = prim_of(dq, gas);
  T Tg = T(2) * T_wall - st.theta;
  if (Tg < T(0.5) * T_wall) Tg = T(0.5) * T_wall;
  const T rg = st.p / Tg;
  const T ke = T(0.5) * rg * (st.U * st.U + st.V * st.V + st.W * st.W);
  q[0 * g.P + dst] = rg - gas.rho_r;
  q[1 * g.P + dst] = -rg * st.U;
  q[2 * g.P + dst] = -rg * st.V;
  q[3 * g.P + dst] = -rg * st.W;
  q[4 * g.P + dst] = st.dp / gas.gm1 + ke;
}
template <class T>
__global__ void k_ghost_y(T* __restrict__ q, GridDev g, int wall, Gas<T> gas, T T_wall) {
  ghost_y_cells(q, g, wall, gas, T_wall, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// z ghosts (periodic) for all x, y including ghosts.
template <class T>
__device__ __forceinline__ void ghost_z_cells(T* __restrict__ q, const GridDev& g, long long tid) {
  const long long plane = (long long)g.p[0] * g.p[1];
  const long long total = 6LL * plane;
  if (tid >= total) return;
  const long long xy = tid % plane;
  const int m = int(tid / plane);
  const int z = m < 3 ? -1 - m : g.n[2] + (m - 3);
  const int src = m < 3 ? g.n[2] - 1 - m : m - 3;
  const long long dst = (long long)(z + kGhost) * plane + xy;
  const long long s = (long long)(src + kGhost) * plane + xy;
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v * g.P + dst] = q[v * g.P + s];
}
template <class T>
__global__ void k_ghost_z(T* __restrict__ q, GridDev g) {
  ghost_z_cells(q, g, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Copy of the padded state with x slowest, qx[v][x][z][y] = q[v][z][y][x]
// (padded coordinates, ghosts included), so that the x sweep reads its cells
// like the y and z sweeps read q: consecutive threads along y, the normal
// axis strided.  One CTA per 32 x 32 tile of an x-y plane, all five
// variables through shared memory (the 20 loads of a thread are in flight
// together); grid (ceil(p0/32), ceil(p1/32), p2), 256 threads.
template <class T>
__global__ void __launch_bounds__(256) k_transpose_x(const T* __restrict__ q, T* __restrict__ qx,
                                                     GridDev g) {
#define HGKS_TR_BX blockIdx.x
#define HGKS_TR_BY blockIdx.y
#define HGKS_TR_BZ blockIdx.z
#include "transpose_body.inc"
#undef HGKS_TR_BX
#undef HGKS_TR_BY
#undef HGKS_TR_BZ
}

// Global conservative-variable index of local-frame component i for sweep
// direction d (local frame: normal momentum first, then t1, t2).
__host__ __device__ __forceinline__ int global_var(int d, int i) {
  if (i == 0 || i == 4) return i;
  return 1 + (d + i - 1) % 3;
}

// ------------------------------------------------------------------ update ---

template <class T>
struct UpdateArgs {
  T* __restrict__ q;          // Q^n (padded); read only
  T* __restrict__ qs;         // Q* (padded), written in stage 1; Q^{n+1} written here in
                              // stage 2 (Q* is dead by then), so that Q^n stays intact
  T* __restrict__ inc;        // dt L(Q^n) + dt^2/6 dL(Q^n), interior
  T* __restrict__ comp;       // compensation of the FP32 accumulation of Q^n (or null)
  T* __restrict__ comp_out;   // stage 2: compensation of Q^{n+1} (or null)
  const int* __restrict__ flag;  // non-physical flag: nothing is written once it is set
                                 // (null: no guard)
  const T* __restrict__ fx;
  const T* __restrict__ fy;
  const T* __restrict__ fz;
  const T* __restrict__ wx;
  const T* __restrict__ wy;
  const T* __restrict__ wz;
  const double* __restrict__ scal;
  GridDev g;
  T force_x;
  T rho_r;
};

// Stage 1: L, dL of Q^n; Q* = Q^n + dt/2 L + dt^2/8 dL; inc = dt L + dt^2/6 dL.
// Stage 2: dL of Q*; Q^{n+1} = Q^n + inc + dt^2/3 dL(Q*), then the body force,
// into the buffer of Q* (qs).  With the non-physical flag set (by the CFL
// kernel of this step, on Q^n) the kernel writes nothing.
// One CTA per 32 x 8 cells of an x-y plane.  The x-face fluxes are stored y
// fastest ([z][x][y]); the CTA stages its 33 x 8 x-faces through shared
// memory so that both their loads and the per-cell reads are contiguous.
// The kernel waits on memory; in FP32 its registers are held to 32 so that
// eight CTAs (all 64 warps) fit an SM.
constexpr int kUpdTX = 32, kUpdTY = 8;
template <class T, int STAGE>
__global__ void __launch_bounds__(kUpdTX * kUpdTY, sizeof(T) == 4 ? 8 : 1) k_update(UpdateArgs<T> a) {
  __shared__ T sfx[STAGE == 1 ? 10 : 5][kUpdTX + 1][kUpdTY];
#define HGKS_UPD_BX blockIdx.x
#define HGKS_UPD_BY blockIdx.y
#define HGKS_UPD_BZ blockIdx.z
#include "update_body.inc"
#undef HGKS_UPD_BX
#undef HGKS_UPD_BY
#undef HGKS_UPD_BZ
}

// -------------------------------------------------------------- reductions ---

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CFL time-step bound min over cells and directions of width/(|u_d| + c),
// with a flag for non-physical states (rho <= 0, p <= 0, NaN).  The per-cell
// arithmetic runs in T; the minimum is combined in FP64: positive doubles
// order like their bit patterns, so block minima meet in a 64-bit atomicMin.
template <class T>
__device__ __forceinline__ void cfl_block(const T* __restrict__ q, const GridDev& g,
                                          const T* __restrict__ wx, const T* __restrict__ wy,
                                          const T* __restrict__ wz, double rho_r, double p_r,
                                          double gamma, unsigned long long* __restrict__ dtmin,
                                          int* __restrict__ flag, int block, int nblocks) {
  T best = T(1e30);
  int bad = 0;
  const int nx = g.n[0], ny = g.n[1];
  const T tr = T(rho_r), tp = T(p_r), tg = T(gamma), tg1 = T(gamma - 1.0);
  // Rows (y, z) of the interior, four per block and pass, x over the threads
  // (coalesced, no 64-bit division per cell); the loads of the four rows are
  // issued before any of them is used.
  const int rows = ny * g.n[2];
  auto cell = [&](T rho, T mx, T my, T mz, T E, int x, int y, int z) {
    const T inv = T(1) / rho;
    const T ke = T(0.5) * (mx * mx + my * my + mz * mz) * inv;
    const T p = tp + tg1 * (E - ke);
    const bool ok = rho > T(0) && p > T(0);  // false for NaN too
    bad |= !ok;
    const T cs = tsqrt(ok ? tg * p * inv : T(1));
    T b = fmin(wx[x + kGhost] / (tabs(mx * inv) + cs), wy[y + kGhost] / (tabs(my * inv) + cs));
    b = fmin(b, wz[z + kGhost] / (tabs(mz * inv) + cs));
    if (ok) best = fmin(best, b);
  };
  for (int row0 = 4 * block; row0 < rows; row0 += 4 * nblocks) {
    for (int x0 = 0; x0 < nx; x0 += blockDim.x) {
      const int x = x0 + threadIdx.x;
      T v[4][5];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int row = row0 + k;
        if (row < rows && x < nx) {
          const long long pi = pad_index(g, x, row % ny, row / ny);
#pragma unroll
          for (int c = 0; c < 5; ++c) v[k][c] = q[c * g.P + pi];
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int row = row0 + k;
        if (row < rows && x < nx)
          cell(tr + v[k][0], v[k][1], v[k][2], v[k][3], v[k][4], x, row % ny, row / ny);
      }
    }
  }
  double bd = warp_min(double(best));
  __shared__ double sm[32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  if (bad) atomicOr(&sbad, 1);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = bd;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 1e300;
    v = warp_min(v);
    if (threadIdx.x == 0) {
      atomicMin(dtmin, (unsigned long long)__double_as_longlong(v));
      if (sbad) atomicOr(flag, 1);
    }
  }
}
template <class T>
__global__ void __launch_bounds__(256) k_cfl(const T* __restrict__ q, GridDev g,
                                             const T* __restrict__ wx, const T* __restrict__ wy,
                                             const T* __restrict__ wz, double rho_r, double p_r,
                                             double gamma, unsigned long long* __restrict__ dtmin,
                                             int* __restrict__ flag) {
  cfl_block(q, g, wx, wy, wz, rho_r, p_r, gamma, dtmin, flag, blockIdx.x, gridDim.x);
}

// Scalars: [0] dt, [1] t, [2] steps taken.  dt_fixed > 0 overrides the CFL step.
// With the non-physical flag set (flag may be null: no guard) the step's
// scalars are left as they are.
static __global__ void k_set_dt(double* scal, unsigned long long* dtmin, double cfl, double dt_fixed,
                                const int* flag) {
  if (threadIdx.x != 0) return;
  if (flag && *flag) return;
  scal[0] = dt_fixed > 0.0 ? dt_fixed : cfl * __longlong_as_double((long long)*dtmin);
  *dtmin = (unsigned long long)__double_as_longlong(1e300);
}
static __global__ void k_advance_time(double* scal, const int* flag) {
  if (threadIdx.x != 0) return;
  if (flag && *flag) return;
  scal[1] += scal[0];
  scal[2] += 1.0;
}

// FP64 partial sums per block: mass, momentum (3), energy, kinetic energy,
// and minima of rho and p; cell volume weights from the widths.
template <class T>
__global__ void __launch_bounds__(256) k_diag(const T* __restrict__ q, GridDev g,
                                              const T* __restrict__ wx, const T* __restrict__ wy,
                                              const T* __restrict__ wz, double rho_r, double p_r,
                                              double gamma, double* __restrict__ part) {
  double s[6] = {0, 0, 0, 0, 0, 0};
  double rmin = 1e300, pmin = 1e300;
  const int nx = g.n[0], ny = g.n[1];
  const double E_r = p_r / (gamma - 1.0);
  // Rows (y, z) of the interior spread over the blocks, x over the threads
  // (coalesced, no 64-bit division per cell).
  const int rows = ny * g.n[2];
  for (int row = blockIdx.x; row < rows; row += gridDim.x)
#pragma unroll 2
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    const int y = row % ny, z = row / ny;
    const long long pi = pad_index(g, x, y, z);
    const double vol = double(wx[x + kGhost]) * double(wy[y + kGhost]) * double(wz[z + kGhost]);
    const double rho = rho_r + double(q[pi]);
    const double mx = q[g.P + pi], my = q[2 * g.P + pi], mz = q[3 * g.P + pi];
    const double E = E_r + double(q[4 * g.P + pi]);
    const double ke = 0.5 * (mx * mx + my * my + mz * mz) / rho;
    s[0] += rho * vol;
    s[1] += mx * vol;
    s[2] += my * vol;
    s[3] += mz * vol;
    s[4] += E * vol;
    s[5] += ke * vol;
    rmin = fmin(rmin, rho);
    pmin = fmin(pmin, (gamma - 1.0) * (E - ke));
  }
  __shared__ double sm[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double v = warp_sum(s[k]);
    if (lane == 0) sm[k][wid] = v;
  }
  rmin = warp_min(rmin);
  pmin = warp_min(pmin);
  if (lane == 0) {
    sm[6][wid] = rmin;
    sm[7][wid] = pmin;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double v = lane < nw ? sm[k][lane] : (k < 6 ? 0.0 : 1e300);
      v = k < 6 ? warp_sum(v) : warp_min(v);
      if (lane == 0) part[blockIdx.x * 8 + k] = v;
    }
  }
}

// Deterministic final reduction of the per-block partials (one block).
static __global__ void k_diag_final(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  __shared__ double sm[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double s[8] = {0, 0, 0, 0, 0, 0, 1e300, 1e300};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] += part[b * 8 + k];
    s[6] = fmin(s[6], part[b * 8 + 6]);
    s[7] = fmin(s[7], part[b * 8 + 7]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double v = k < 6 ? warp_sum(s[k]) : warp_min(s[k]);
    if (lane == 0) sm[k][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double v = lane < nw ? sm[k][lane] : (k < 6 ? 0.0 : 1e300);
      v = k < 6 ? warp_sum(v) : warp_min(v);
      if (lane == 0) out[k] = v;
    }
  }
}

// ------------------------------------------------- constant mass flux force ---
// Sec. 3.3: after the two S2O4 stages (state Q~^{n+1} in q; rho^n and
// (rho U)^n in planes 0 and 1 of `stash`, the buffer of Q^n, which the step
// leaves intact), per-block FP64 sums of the cell volume, of (rho U)~ and of
// (rho^n + rho~)/2, each times the cell volume, into part[3 b + k].  comp
// (FP32 compensation) may be null.
template <class T>
__global__ void __launch_bounds__(256) k_massflux_sums(const T* __restrict__ q, const T* __restrict__ stash,
                                                       const T* __restrict__ comp,
                                                       GridDev g, const T* __restrict__ wx,
                                                       const T* __restrict__ wy, const T* __restrict__ wz,
                                                       double rho_r, double* __restrict__ part,
                                                       const int* __restrict__ flag) {
  if (flag && *flag) return;
  double s[3] = {0.0, 0.0, 0.0};
  const int nx = g.n[0], ny = g.n[1];
  // Rows (y, z) of the interior spread over the blocks, x over the threads
  // (coalesced, no 64-bit division per cell).
  const int rows = ny * g.n[2];
  for (int row = blockIdx.x; row < rows; row += gridDim.x)
#pragma unroll 2
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    const int y = row % ny, z = row / ny;
    const long long pi = pad_index(g, x, y, z);
    const long long c = ((long long)z * ny + y) * nx + x;  // interior index
    const double vol = double(wx[x + kGhost]) * double(wy[y + kGhost]) * double(wz[z + kGhost]);
    // FP32: the stored value minus its compensation is the accumulated sum.
    const double c0 = comp ? double(comp[c]) : 0.0, c1 = comp ? double(comp[g.N + c]) : 0.0;
    s[0] += vol;
    s[1] += (double(q[g.P + pi]) - c1) * vol;
    s[2] += (rho_r + 0.5 * (double(q[pi]) - c0 + double(stash[pi]))) * vol;
  }
  __shared__ double sm[3][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum(s[k]);
    if (lane == 0) sm[k][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v = lane < nw ? sm[k][lane] : 0.0;
      v = warp_sum(v);
      if (lane == 0) part[blockIdx.x * 3 + k] = v;
    }
  }
}

// f_x = (mass_flux * volume - int (rho U)~) / (dt * int (rho^n + rho~)/2)
// into scal[3] (one block of 256; deterministic order).
static __global__ void __launch_bounds__(256) k_massflux_force(const double* __restrict__ part, int nblocks,
                                                               double mass_flux, double* __restrict__ scal,
                                                               const int* __restrict__ flag) {
  __shared__ double sm[3][8];
  if (flag && *flag) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] += part[b * 3 + k];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum(s[k]);
    if (lane == 0) sm[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[3] = {0.0, 0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int k = 0; k < 3; ++k) t[k] += sm[k][w];
    scal[3] = (mass_flux * t[0] - t[1]) / (scal[0] * t[2]);
  }
}

// (rho U)^{n+1} = (rho U)~ + dt/2 (rho~ + rho^n) f_x;
// (rho E)^{n+1} = (rho E)~ + dt/2 ((rho U)^{n+1} + (rho U)^n) f_x, with the
// FP32 compensation continued (comp may be null for FP64).
template <class T>
__global__ void __launch_bounds__(256) k_force_apply(T* __restrict__ q, const T* __restrict__ stash,
                                                     T* __restrict__ comp, GridDev g, double rho_r,
                                                     const double* __restrict__ scal,
                                                     const int* __restrict__ flag) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  if (flag && *flag) return;
  const int nx = g.n[0], ny = g.n[1];
  const int x = int(c % nx);
  const long long r = c / nx;
  const int y = int(r % ny), z = int(r / ny);
  const long long pi = pad_index(g, x, y, z);
  const T f = T(scal[3]), hdt = T(0.5 * scal[0]);
  const T rho_t = T(rho_r) + q[pi], rho_n = T(rho_r) + stash[pi];
  const T m_t = q[g.P + pi], m_n = stash[g.P + pi];
  const T dm = hdt * (rho_t + rho_n) * f;
  const T dE = hdt * (m_t + dm + m_n) * f;
  const T inc[2] = {dm, dE};
  const int var[2] = {1, 4};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const long long qi = var[k] * g.P + pi;
    if (comp) {
      const long long ci = var[k] * g.N + c;
      const T yv = inc[k] - comp[ci];
      const T t = q[qi] + yv;
      comp[ci] = (t - q[qi]) - yv;
      q[qi] = t;
    } else {
      q[qi] += inc[k];
    }
  }
}

// ----------------------------------------------------------- state in/out ---

// FP64 primitive (rho, u, v, w, p) [5][N] -> deviation conservative (padded interior).
// FP64 state in / out, one thread per cell of an x row: grid (ceil(nx /
// 256), ny, nz), so that the cell's coordinates come without integer
// division; inv_gm1 = 1 / (gamma - 1) and E_r = p_r / (gamma - 1) are formed
// on the host.
template <class T>
__global__ void k_from_prim(const double* __restrict__ prim, T* __restrict__ q, GridDev g,
                            double rho_r, double E_r, double inv_gm1, int conservative) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.n[0]) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long c = ((long long)z * g.n[1] + y) * g.n[0] + x;
  const long long pi = pad_index(g, x, y, z);
  double Q[5];
  if (conservative) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Q[v] = prim[v * g.N + c];
  } else {
    const double rho = prim[c], u = prim[g.N + c], v = prim[2 * g.N + c], w = prim[3 * g.N + c],
                 p = prim[4 * g.N + c];
    Q[0] = rho;
    Q[1] = rho * u;
    Q[2] = rho * v;
    Q[3] = rho * w;
    Q[4] = p * inv_gm1 + 0.5 * rho * (u * u + v * v + w * w);
  }
  q[pi] = T(Q[0] - rho_r);
  q[g.P + pi] = T(Q[1]);
  q[2 * g.P + pi] = T(Q[2]);
  q[3 * g.P + pi] = T(Q[3]);
  q[4 * g.P + pi] = T(Q[4] - E_r);
}

template <class T>
__global__ void k_to_cons(const T* __restrict__ q, double* __restrict__ out, GridDev g, double rho_r,
                          double E_r) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.n[0]) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long c = ((long long)z * g.n[1] + y) * g.n[0] + x;
  const long long pi = pad_index(g, x, y, z);
  out[c] = rho_r + double(q[pi]);
  out[g.N + c] = double(q[g.P + pi]);
  out[2 * g.N + c] = double(q[2 * g.P + pi]);
  out[3 * g.N + c] = double(q[3 * g.P + pi]);
  out[4 * g.N + c] = E_r + double(q[4 * g.P + pi]);
}

}  // namespace hgks
