// Batched launches of an ensemble step: ONE grid per phase of the S2O4 step
// (CFL reduction, dt, ghost fills, transposed copy, the three sweeps and the
// update of each stage, time) covering every instance of the ensemble.  The
// instance table is a kernel parameter (__grid_constant__: it stays in the
// constant bank, no copy): instance m owns the blocks [start[m], start[m+1])
// of the grid, and each block runs the same body as the single-instance
// kernel (kernels.cuh, sweep.cuh) on its instance's arguments and its local
// block coordinates.  No block waits on another: the phases are ordered by
// the stream (and the captured graph) only.
#pragma once

#include "kernels.cuh"
#include "sweep.cuh"

namespace hgks {

constexpr int kBatchMax = 32;  // instances per batched launch

template <class Job>
struct BatchTable {
  int n;                      // instances
  int start[kBatchMax + 1];   // first block of each instance; start[n] = grid size
  Job job[kBatchMax];
};

// The instance that owns block b: the last m with start[m] <= b.
template <class Job>
__device__ __forceinline__ int batch_instance(const BatchTable<Job>& t, int b) {
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class Job>
__global__ void __launch_bounds__(Job::kThreads, Job::kMinBlocks)
    k_batched(const __grid_constant__ BatchTable<Job> t) {
  const int b = blockIdx.x;
  const int m = batch_instance(t, b);
  t.job[m].run(b - t.start[m]);
}

// ------------------------------------------------------------------ jobs ---

template <class T>
struct CflJob {
  static constexpr int kThreads = 256, kMinBlocks = 1;
  const T* q;
  GridDev g;
  const T *wx, *wy, *wz;
  double rho_r, p_r, gamma;
  unsigned long long* dtmin;
  int* flag;
  int nblocks;
  __device__ __forceinline__ void run(int b) const {
    cfl_block(q, g, wx, wy, wz, rho_r, p_r, gamma, dtmin, flag, b, nblocks);
  }
};

struct SetDtJob {
  static constexpr int kThreads = 32, kMinBlocks = 1;
  double* scal;
  unsigned long long* dtmin;
  double cfl, dt_fixed;
  const int* flag;
  __device__ __forceinline__ void run(int) const {
    if (threadIdx.x != 0) return;
    if (flag && *flag) return;
    scal[0] = dt_fixed > 0.0 ? dt_fixed : cfl * __longlong_as_double((long long)*dtmin);
    *dtmin = (unsigned long long)__double_as_longlong(1e300);
  }
};

struct AdvanceJob {
  static constexpr int kThreads = 32, kMinBlocks = 1;
  double* scal;
  const int* flag;
  __device__ __forceinline__ void run(int) const {
    if (threadIdx.x != 0) return;
    if (flag && *flag) return;
    scal[1] += scal[0];
    scal[2] += 1.0;
  }
};

template <class T>
struct GhostXJob {
  static constexpr int kThreads = 256, kMinBlocks = 1;
  T* q;
  GridDev g;
  __device__ __forceinline__ void run(int b) const {
    ghost_x_cells(q, g, b * (long long)kThreads + threadIdx.x);
  }
};

template <class T>
struct GhostYJob {
  static constexpr int kThreads = 256, kMinBlocks = 1;
  T* q;
  GridDev g;
  int wall;
  Gas<T> gas;
  T T_wall;
  __device__ __forceinline__ void run(int b) const {
    ghost_y_cells(q, g, wall, gas, T_wall, b * (long long)kThreads + threadIdx.x);
  }
};

template <class T>
struct GhostZJob {
  static constexpr int kThreads = 256, kMinBlocks = 1;
  T* q;
  GridDev g;
  __device__ __forceinline__ void run(int b) const {
    ghost_z_cells(q, g, b * (long long)kThreads + threadIdx.x);
  }
};

template <class T>
struct TransposeJob {
  static constexpr int kThreads = 256, kMinBlocks = 1;
  const T* q;
  T* qx;
  GridDev g;
  int gx, gy;
  __device__ __forceinline__ void run(int b) const {
#define HGKS_TR_BX (b % gx)
#define HGKS_TR_BY ((b / gx) % gy)
#define HGKS_TR_BZ (b / (gx * gy))
#include "transpose_body.inc"
#undef HGKS_TR_BX
#undef HGKS_TR_BY
#undef HGKS_TR_BZ
  }
};

template <class T, int MODE, int FLUX, int STAGE, int TP, int TS, int NL, bool PK>
struct SweepJob {
  static constexpr int kThreads = sweep_threads(TP, TS);
  static constexpr int kMinBlocks = PK ? 2 : sweep_min_blocks<T, MODE, FLUX, TP, TS>();
  SweepArgs<T> a;
  int gx, gy;
  __device__ __forceinline__ void run(int b) const {
#define HGKS_SW_BX (b % gx)
#define HGKS_SW_BY ((b / gx) % gy)
#define HGKS_SW_BZ (b / (gx * gy))
#include "sweep_body.inc"
#undef HGKS_SW_BX
#undef HGKS_SW_BY
#undef HGKS_SW_BZ
  }
};

template <class T, int STAGE>
struct UpdateJob {
  static constexpr int kThreads = kUpdTX * kUpdTY, kMinBlocks = sizeof(T) == 4 ? 8 : 1;
  UpdateArgs<T> a;
  int gx, gy;
  __device__ __forceinline__ void run(int b) const {
    __shared__ T sfx[STAGE == 1 ? 10 : 5][kUpdTX + 1][kUpdTY];
#define HGKS_UPD_BX (b % gx)
#define HGKS_UPD_BY ((b / gx) % gy)
#define HGKS_UPD_BZ (b / (gx * gy))
#include "update_body.inc"
#undef HGKS_UPD_BX
#undef HGKS_UPD_BY
#undef HGKS_UPD_BZ
  }
};

}  // namespace hgks
