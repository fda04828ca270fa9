// Turbulence statistics of the current state (Sec. 3.1 and Sec. 3.4):
// kinetic energy, enstrophy, the three Navier-Stokes dissipation
// contributions eps1..eps3, rho_rms, K, the skewness / flatness moments of
// the velocity slopes, the solenoidal and dilatational dissipation rates and
// the pressure dilatation.  Velocity gradients use the sixth-order central
// difference (Sec. 3.1) on the periodic, uniform grid, the neighbours taken
// by periodic wrap of the interior indices (no ghost fill needed).  Every
// sum is FP64; the per-cell arithmetic is FP64 whatever the storage type.
// Output: kTurbSums raw volume-weighted sums, composed into the ABI's
// statistics on the host -- on demand, or appended to the statistics
// history by the step itself (gated on the step count).
#pragma once

#include "engine.h"
#include "kernels.cuh"

namespace hgks {

struct TurbArgs {
  double inv60h[3];  // 1 / (60 h_d) of the uniform spacing per axis
  double rho_r, E_r, gm1;
  int visc_law;
  double mu_ref, T_ref_inv, visc_exp;
  double mub_ratio;  // mu_b / mu = 2N / (3(N + 3))
  double vol;        // cell volume
};

template <class T>
__device__ __forceinline__ void velocity_at(const T* __restrict__ q, long long P, long long i,
                                            double rho_r, double u[3]) {
  const double inv = 1.0 / (rho_r + double(q[i]));
  u[0] = double(q[P + i]) * inv;
  u[1] = double(q[2 * P + i]) * inv;
  u[2] = double(q[3 * P + i]) * inv;
}

// Gate of the history record: with every > 0 the kernels run only when the
// step count scal[2] is a multiple of every and the non-physical flag is
// clear; every = 0 always runs.
struct HistGate {
  const double* scal;
  const int* flag;
  int every;
  __device__ __forceinline__ bool skip() const {
    return every > 0 && ((flag && *flag) || ((long long)scal[2]) % every != 0);
  }
};

template <class T>
__global__ void __launch_bounds__(256) k_turb(const T* __restrict__ q, GridDev g, TurbArgs a,
                                              double* __restrict__ part, HistGate gate) {
  if (gate.skip()) return;
  double s[kTurbSums];
#pragma unroll
  for (int k = 0; k < kTurbSums; ++k) s[k] = 0.0;
  const int nx = g.n[0], ny = g.n[1];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = int(c % nx);
    const long long r = c / nx;
    const int y = int(r % ny), z = int(r / ny);
    const int cc[3] = {x, y, z};
    const long long pi = pad_index(g, x, y, z);
    const double drho = double(q[pi]);
    const double rho = a.rho_r + drho;
    double U[3];
    velocity_at(q, g.P, pi, a.rho_r, U);
    const double q2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    const double p = a.gm1 * (a.E_r + double(q[4 * g.P + pi]) - 0.5 * rho * q2);
    const double mu = a.visc_law == 1 ? a.mu_ref * pow(p / rho * a.T_ref_inv, a.visc_exp) : a.mu_ref;
    // G[i][j] = dU_i/dx_j: sixth-order central differences along each axis.
    double G[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 1; k <= 3; ++k) {
        const double ck = k == 1 ? 45.0 : (k == 2 ? -9.0 : 1.0);
        int cp[3] = {cc[0], cc[1], cc[2]}, cm[3] = {cc[0], cc[1], cc[2]};
        cp[j] = cc[j] + k < g.n[j] ? cc[j] + k : cc[j] + k - g.n[j];  // periodic wrap
        cm[j] = cc[j] - k >= 0 ? cc[j] - k : cc[j] - k + g.n[j];
        double up[3], um[3];
        velocity_at(q, g.P, pad_index(g, cp[0], cp[1], cp[2]), a.rho_r, up);
        velocity_at(q, g.P, pad_index(g, cm[0], cm[1], cm[2]), a.rho_r, um);
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i] += ck * (up[i] - um[i]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) G[i][j] = acc[i] * a.inv60h[j];
    }
    const double th = G[0][0] + G[1][1] + G[2][2];
    const double w0 = G[2][1] - G[1][2], w1 = G[0][2] - G[2][0], w2 = G[1][0] - G[0][1];
    const double om2 = w0 * w0 + w1 * w1 + w2 * w2;
    double sdsd = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double d = G[i][i] - th * (1.0 / 3.0);
      sdsd += d * d;
#pragma unroll
      for (int j = i + 1; j < 3; ++j) {
        const double o = 0.5 * (G[i][j] + G[j][i]);
        sdsd += 2.0 * o * o;
      }
    }
    const double v = a.vol;
    s[TS_VOL] += v;
    s[TS_KE] += 0.5 * rho * q2 * v;
    s[TS_ENS] += 0.5 * rho * om2 * v;
    s[TS_MU_SDSD] += mu * sdsd * v;
    s[TS_MUB_TH2] += a.mub_ratio * mu * th * th * v;
    s[TS_P_TH] += p * th * v;
    s[TS_DRHO] += drho * v;
    s[TS_DRHO2] += drho * drho * v;
    s[TS_Q2] += q2 * v;
    s[TS_MU_W2] += mu * om2 * v;
    s[TS_MU_TH2] += mu * th * th * v;
    s[TS_TH2] += th * th * v;
    s[TS_W2] += om2 * v;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double d2 = G[i][i] * G[i][i];
      s[TS_DU2 + i] += d2 * v;
      s[TS_DU3 + i] += d2 * G[i][i] * v;
      s[TS_DU4 + i] += d2 * d2 * v;
    }
  }
  // Block sum: warp shuffles, then one warp over the warps' partials.
  __shared__ double sm[kTurbSums][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kTurbSums; ++k) {
    const double t = warp_sum(s[k]);
    if (lane == 0) sm[k][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < kTurbSums; ++k) {
      double t = lane < nw ? sm[k][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) part[(long long)blockIdx.x * kTurbSums + k] = t;
    }
  }
}

// Where the final sums go: out (on demand), or the next record of the
// history (hist != null): [t, step, sums], then the count is advanced;
// records beyond cap are dropped.
struct TurbSink {
  double* out;
  double* hist;
  int* count;
  int cap;
};

// Deterministic final sum of the per-block partials (one block of 256).
static __global__ void __launch_bounds__(256) k_turb_final(const double* __restrict__ part, int nblocks,
                                                           TurbSink sink, HistGate gate) {
  __shared__ double sm[kTurbSums][8];
  if (gate.skip()) return;
  double* out = sink.out;
  if (sink.hist) {
    const int idx = *sink.count;  // one block: read before any thread advances it
    if (idx >= sink.cap) return;
    out = sink.hist + (long long)idx * kHistStride + 2;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < kTurbSums; ++k) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) t += part[(long long)b * kTurbSums + k];
    t = warp_sum(t);
    if (lane == 0) sm[k][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < kTurbSums; ++k) {
      double t = lane < nw ? sm[k][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) out[k] = t;
    }
    if (sink.hist && lane == 0) {
      out[-2] = gate.scal[1];
      out[-1] = gate.scal[2];
      __threadfence();
      *sink.count = *sink.count + 1;
    }
  }
}

// Plane averages of a wall-bounded channel (Sec. 3.3): one block per y row,
// FP64 sums over the x-z plane of rho, rho U, U, V, W, U V, U U and
// T = p / rho (interior cells; x and z are uniform and periodic, so the
// plane mean is the plain mean).  out[k * ny + y] = sum k of row y.
template <class T>
__global__ void __launch_bounds__(256) k_channel_rows(const T* __restrict__ q, GridDev g, double rho_r,
                                                      double p_r, double gm1, double* __restrict__ out) {
  const int y = blockIdx.x;
  const int nx = g.n[0], nz = g.n[2];
  double s[kChanSums];
#pragma unroll
  for (int k = 0; k < kChanSums; ++k) s[k] = 0.0;
  for (int c = threadIdx.x; c < nx * nz; c += blockDim.x) {
    const long long pi = pad_index(g, c % nx, y, c / nx);
    const double rho = rho_r + double(q[pi]);
    const double mx = double(q[g.P + pi]), my = double(q[2 * g.P + pi]), mz = double(q[3 * g.P + pi]);
    const double inv = 1.0 / rho;
    const double U = mx * inv, V = my * inv, W = mz * inv;
    // p - p_r = (gamma - 1)(dE - |m|^2 / (2 rho)); the reference is at rest.
    const double p = p_r + gm1 * (double(q[4 * g.P + pi]) - 0.5 * (mx * U + my * V + mz * W));
    s[0] += rho;
    s[1] += mx;
    s[2] += U;
    s[3] += V;
    s[4] += W;
    s[5] += U * V;
    s[6] += U * U;
    s[7] += p * inv;
  }
  __shared__ double sm[kChanSums][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kChanSums; ++k) {
    const double t = warp_sum(s[k]);
    if (lane == 0) sm[k][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kChanSums; ++k) {
      double t = lane < nw ? sm[k][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) out[k * g.n[1] + y] = t;
    }
  }
}

}  // namespace hgks
