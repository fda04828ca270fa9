// hgks_step_noalloc: the S2O4 step for callers that cannot allocate device
// memory.  Some callers run where cudaMalloc is unavailable or forbidden --
// inside a host framework that owns every device allocation, from a context
// that must not grow its memory footprint, or in code paths that must not
// synchronise the device the way an allocation can.  This entry point takes
// the caller's state buffer and does all its work in one scratch array that
// is part of the library image: a file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cstring>
#include <mutex>

#include "engine.h"
#include "kernels.cuh"

namespace {

constexpr int kMaxN = 32;                 // cells per axis at most
constexpr int kMaxP = kMaxN + 6;          // padded extent
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
// Scratch layout for the largest grid, in FP64 (FP32 uses the same offsets).
constexpr size_t kQBytes = align_up(5ull * kMaxP * kMaxP * kMaxP * 8);
constexpr size_t kIncBytes = align_up(5ull * kMaxN * kMaxN * kMaxN * 8);
constexpr size_t kFdBytes = align_up(10ull * (kMaxN + 1) * kMaxN * kMaxN * 8);
constexpr size_t kWBytes = align_up(kMaxP * 8);
constexpr size_t kScalBytes = align_up(4 * 8 + 8 + 4);
constexpr size_t kScratchBytes =
    2 * kQBytes + 3 * kIncBytes + 3 * kFdBytes + 3 * kWBytes + kScalBytes;  // ~16 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once with that device current.
std::mutex g_mu;
void* g_addr[64] = {nullptr};

// Cell widths (with 3 ghost cells per side) of axis d, as in hgks_create.
template <class T>
__global__ void k_fill_widths(T* w, int n, double L, int stretched, double b, double ly) {
  const int i = threadIdx.x;
  if (i >= n + 6) return;
  double v = L / n;
  if (stretched) {
    // Sec. 3.3 mapping, faces j and j+1 of the interior cell j; ghost cells
    // take the widths of their mirror images across the walls.
    int j = i - 3;
    if (j < 0) j = -1 - j;
    if (j >= n) j = 2 * n - 1 - j;
    const double pi = 3.14159265358979323846;
    const double e0 = 3.0 * pi * j / n, e1 = 3.0 * pi * (j + 1) / n;
    const double y0 = 0.5 * ly * (1.0 + tanh(b * (e0 / (1.5 * pi) - 1.0)) / tanh(b));
    const double y1 = 0.5 * ly * (1.0 + tanh(b * (e1 / (1.5 * pi) - 1.0)) / tanh(b));
    v = y1 - y0;
  }
  w[i] = T(v);
}

}  // namespace

extern "C" hgks_status hgks_step_noalloc(const hgks_config* cfg, double* cons_inout, int nsteps,
                                         double dt, void* stream) {
  if (!cfg || !cons_inout || nsteps < 0) return HGKS_E_INVAL;
  if (!hgks::validate_config(*cfg).empty()) return HGKS_E_INVAL;
  if (cfg->nx > kMaxN || cfg->ny > kMaxN || cfg->nz > kMaxN) return HGKS_E_UNSUPPORTED;
  if (cfg->force_mode != HGKS_FORCE_CONSTANT) return HGKS_E_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HGKS_E_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HGKS_E_CUDA;
      g_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_addr[dev]);
  }
  hgks::Engine e;
  e.cfg = *cfg;
  e.stream = static_cast<cudaStream_t>(stream);
  e.n[0] = cfg->nx;
  e.n[1] = cfg->ny;
  e.n[2] = cfg->nz;
  for (int d = 0; d < 3; ++d) e.p[d] = e.n[d] + 6;
  e.P = (long long)e.p[0] * e.p[1] * e.p[2];
  e.N = (long long)e.n[0] * e.n[1] * e.n[2];
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e.sms = sms > 0 ? sms : 152;
  e.cfl_blocks = e.sms;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    void* p = base + off;
    off += bytes;
    return p;
  };
  e.q = take(kQBytes);
  e.qs = take(kQBytes);
  e.inc = take(kIncBytes);
  void* comp = take(kIncBytes);
  void* comp2 = take(kIncBytes);
  e.comp = cfg->prec == HGKS_FP32 ? comp : nullptr;
  e.comp2 = cfg->prec == HGKS_FP32 ? comp2 : nullptr;
  // No non-physical check here: the steps run to the end whatever the state.
  e.guard = false;
  for (int d = 0; d < 3; ++d) e.fd[d] = take(kFdBytes);
  for (int d = 0; d < 3; ++d) e.w[d] = take(kWBytes);
  unsigned char* sc = static_cast<unsigned char*>(take(kScalBytes));
  e.scal = reinterpret_cast<double*>(sc);
  e.dtmin = reinterpret_cast<unsigned long long*>(sc + 32);
  e.flag = reinterpret_cast<int*>(sc + 40);
  const bool f32 = cfg->prec == HGKS_FP32;
  const size_t es = f32 ? 4 : 8;
  // The array keeps the previous call's contents: clear what must start at
  // zero (padded states, so that unused ghost corners are finite; the FP32
  // compensation; the scalars).
  cudaError_t err = cudaMemsetAsync(e.q, 0, 5 * e.P * es, e.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(e.qs, 0, 5 * e.P * es, e.stream);
  if (err == cudaSuccess && e.comp) err = cudaMemsetAsync(e.comp, 0, 5 * e.N * es, e.stream);
  const double L[3] = {cfg->lx, cfg->ly, cfg->lz};
  for (int d = 0; d < 3 && err == cudaSuccess; ++d) {
    const int st = d == 1 && cfg->y_stretch;
    if (f32)
      k_fill_widths<float><<<1, kMaxP, 0, e.stream>>>(static_cast<float*>(e.w[d]), e.n[d], L[d], st,
                                                     cfg->stretch_b, cfg->ly);
    else
      k_fill_widths<double><<<1, kMaxP, 0, e.stream>>>(static_cast<double*>(e.w[d]), e.n[d], L[d],
                                                      st, cfg->stretch_b, cfg->ly);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = hgks::enqueue_reset_scalars(e);
  if (err == cudaSuccess)
    err = f32 ? hgks::enqueue_from_fp64<float>(e, cons_inout, 1)
              : hgks::enqueue_from_fp64<double>(e, cons_inout, 1);
  const double dt_fixed = dt > 0.0 ? dt : 0.0;
  for (int n = 0; n < nsteps && err == cudaSuccess; ++n) {
    err = f32 ? hgks::enqueue_cfl<float>(e, e.q) : hgks::enqueue_cfl<double>(e, e.q);
    if (err == cudaSuccess) err = hgks::enqueue_set_dt(e, dt_fixed);
    for (int stage = 1; stage <= 2 && err == cudaSuccess; ++stage)
      err = f32 ? hgks::enqueue_rhs_and_update<float>(e, stage)
                : hgks::enqueue_rhs_and_update<double>(e, stage);
    if (err == cudaSuccess) err = hgks::enqueue_advance_time(e);
    hgks::swap_state_buffers(e);  // Q^{n+1} was written into qs
  }
  if (err == cudaSuccess)
    err = f32 ? hgks::enqueue_to_fp64<float>(e, cons_inout) : hgks::enqueue_to_fp64<double>(e, cons_inout);
  return err == cudaSuccess ? HGKS_OK : HGKS_E_CUDA;
}
