// Host runtime behind include/hgks.h: validation, device buffers, the grid
// metrics, and the captured CUDA graph of one S2O4 step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "kernels.cuh"

struct hgks_ctx {
  hgks::Engine e;
  bool own_stream = false;
  std::string err;
  // The captured step, one graph per assignment of the two state buffers
  // (graph[0]: q is buf0; graph[1]: q is buf1); the host swaps the
  // assignment after every step.
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  double graph_dt[2] = {0.0, 0.0};
  void* buf0 = nullptr;  // the state buffer allocated first
  int device = 0;
  // Host mirror of the device step counter: steps enqueued since the state
  // was set (init_steps: the counter when it was set).  Used to find the last
  // good state after a non-physical one.
  long long steps_host = 0, init_steps = 0;
};

namespace {

thread_local std::string g_create_error;

hgks_status fail(hgks_ctx* c, hgks_status s, const std::string& msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return s;
}

hgks_status cuda_fail(hgks_ctx* c, cudaError_t e, const char* where) {
  const hgks_status s = (e == cudaErrorMemoryAllocation) ? HGKS_E_NOMEM : HGKS_E_CUDA;
  return fail(c, s, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HGKS_CHECK(c, expr)                                        \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return cuda_fail((c), _e, #expr);       \
  } while (0)

size_t elem_size(const hgks_config& c) { return c.prec == HGKS_FP32 ? 4 : 8; }

}  // namespace

std::string hgks::validate_config(const hgks_config& c) {
  if (c.nx < 6 || c.ny < 6 || c.nz < 6) return "every axis needs at least 6 cells";
  // Kernels launch one grid row per padded y and z index (grid dimensions <= 65535).
  if (c.nx > 65529 || c.ny > 65529 || c.nz > 65529) return "every axis has at most 65529 cells";
  if (!(c.gamma > 1.0)) return "gamma must exceed 1";
  if (!(c.prandtl > 0.0)) return "Prandtl number must be positive";
  if (!(c.cfl > 0.0)) return "cfl must be positive";
  if (!(c.lx > 0.0) || !(c.ly > 0.0) || !(c.lz > 0.0)) return "box extents must be positive";
  if (!(c.rho_ref > 0.0) || !(c.p_ref > 0.0)) return "reference density and pressure must be positive";
  if (!(c.mu_ref >= 0.0)) return "mu_ref must be non-negative";
  if (c.visc != HGKS_VISC_CONST && c.visc != HGKS_VISC_POWER) return "unknown viscosity law";
  if (c.visc == HGKS_VISC_POWER && !(c.T_ref > 0.0)) return "T_ref must be positive";
  if (c.recon < 0 || c.recon > 2) return "unknown reconstruction";
  if (c.flux < 0 || c.flux > 1) return "unknown flux";
  if (c.prec < 0 || c.prec > 1) return "unknown precision";
  if (c.bc_y != HGKS_BC_PERIODIC && c.bc_y != HGKS_BC_WALL_ISOTHERMAL) return "unknown y boundary";
  if (c.bc_y == HGKS_BC_WALL_ISOTHERMAL && !(c.T_wall > 0.0)) return "wall temperature must be positive";
  if (c.y_stretch && c.bc_y != HGKS_BC_WALL_ISOTHERMAL) return "the tanh mapping needs wall boundaries";
  if (c.y_stretch && !(c.stretch_b > 0.0)) return "stretch_b must be positive";
  if (c.y_stretch && std::fabs(c.ly - 2.0) > 1e-12)
    return "the tanh mapping spans the channel height ly = 2";
  if (!(c.tau_num_C >= 0.0)) return "tau_num_C must be non-negative";
  if (c.force_mode != HGKS_FORCE_CONSTANT && c.force_mode != HGKS_FORCE_MASS_FLUX)
    return "unknown force mode";
  if (c.recon_vars != 0 && c.recon_vars != 1) return "recon_vars must be 0 or 1";
  return "";
}

namespace {

// Cell widths along each axis including 3 ghost cells per side: uniform, or
// the y mapping of Sec. 3.3 with ghost widths mirrored across the walls.
std::vector<double> widths(const hgks_config& c, int d) {
  const int n = d == 0 ? c.nx : (d == 1 ? c.ny : c.nz);
  const double L = d == 0 ? c.lx : (d == 1 ? c.ly : c.lz);
  std::vector<double> w(n + 6, L / n);
  if (d == 1 && c.y_stretch) {
    const double pi = 3.14159265358979323846;
    std::vector<double> yf(n + 1);
    for (int j = 0; j <= n; ++j) {
      const double eta = 3.0 * pi * j / n;
      yf[j] = c.y0 + 0.5 * c.ly * (1.0 + std::tanh(c.stretch_b * (eta / (1.5 * pi) - 1.0)) /
                                             std::tanh(c.stretch_b));
    }
    for (int j = 0; j < n; ++j) w[j + 3] = yf[j + 1] - yf[j];
    for (int m = 0; m < 3; ++m) {
      w[2 - m] = w[3 + m];
      w[3 + n + m] = w[3 + n - 1 - m];
    }
  }
  return w;
}

template <class T>
cudaError_t upload_widths(hgks::Engine& e, int d, const std::vector<double>& w) {
  std::vector<T> tw(w.begin(), w.end());
  return cudaMemcpyAsync(e.w[d], tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice, e.stream);
}

void free_all(hgks::Engine& e) {
  void* ptrs[] = {e.q, e.qs, e.qx, e.inc, e.comp, e.comp2, e.fd[0], e.fd[1], e.fd[2], e.w[0], e.w[1],
                  e.w[2], e.scal, e.dtmin, e.flag, e.part, e.diag_out, e.io,
                  e.adj_acc, e.adj_mu, e.adj_wL, e.adj_wdL, e.turb_part, e.turb_out,
                  e.chan_out, e.kin_w, e.hist, e.hist_count};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// One S2O4 step on the context's current buffers; Q^{n+1} ends in e.qs (the
// caller swaps the buffers after enqueuing).
cudaError_t enqueue_stage_pair(hgks::Engine& e, double dt_fixed, hgks::Probe* probe = nullptr) {
  cudaError_t err;
  const bool f32 = e.cfg.prec == HGKS_FP32;
  if (probe) probe->begin(e.stream, hgks::KC_CFL);
  err = f32 ? hgks::enqueue_cfl<float>(e, e.q) : hgks::enqueue_cfl<double>(e, e.q);
  if (err != cudaSuccess) return err;
  err = hgks::enqueue_set_dt(e, dt_fixed);
  if (probe) probe->end(e.stream);
  if (err != cudaSuccess) return err;
  for (int stage = 1; stage <= 2; ++stage) {
    err = f32 ? hgks::enqueue_rhs_and_update<float>(e, stage, probe)
              : hgks::enqueue_rhs_and_update<double>(e, stage, probe);
    if (err != cudaSuccess) return err;
  }
  err = hgks::enqueue_advance_time(e);
  if (err != cudaSuccess || e.hist_every <= 0) return err;
  // Statistics history: a record of Q^{n+1} (in qs) every hist_every steps.
  return f32 ? hgks::enqueue_history_record<float>(e, e.qs, true)
             : hgks::enqueue_history_record<double>(e, e.qs, true);
}

void drop_graphs(hgks_ctx* c) {
  for (int k = 0; k < 2; ++k)
    if (c->graph[k]) {
      cudaGraphExecDestroy(c->graph[k]);
      c->graph[k] = nullptr;
    }
}

// Capture the step for the current buffer assignment (graph[k]).
hgks_status capture_step(hgks_ctx* c, int k, double dt_fixed) {
  hgks::Engine& e = c->e;
  if (c->graph[k]) {
    cudaGraphExecDestroy(c->graph[k]);
    c->graph[k] = nullptr;
  }
  cudaGraph_t g = nullptr;
  HGKS_CHECK(c, cudaStreamBeginCapture(e.stream, cudaStreamCaptureModeThreadLocal));
  const cudaError_t err = enqueue_stage_pair(e, dt_fixed);
  const cudaError_t end = cudaStreamEndCapture(e.stream, &g);
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(c, err, "capturing the step");
  }
  HGKS_CHECK(c, end);
  const cudaError_t inst = cudaGraphInstantiate(&c->graph[k], g, 0);
  cudaGraphDestroy(g);
  HGKS_CHECK(c, inst);
  c->graph_dt[k] = dt_fixed;
  return HGKS_OK;
}

}  // namespace

namespace hgks {

static __global__ void k_reset_scalars(double* scal, unsigned long long* dtmin, int* flag) {
  if (threadIdx.x != 0) return;
  scal[0] = 0.0;
  scal[1] = 0.0;
  scal[2] = 0.0;
  scal[3] = 0.0;
  *dtmin = (unsigned long long)__double_as_longlong(1e300);
  *flag = 0;
}

static __global__ void k_reset_flag(unsigned long long* dtmin, int* flag) {
  if (threadIdx.x != 0) return;
  *dtmin = (unsigned long long)__double_as_longlong(1e300);
  *flag = 0;
}

static __global__ void k_set_time(double* scal, double t, double step) {
  if (threadIdx.x != 0) return;
  scal[1] = t;
  scal[2] = step;
}

// Kinetic-energy functional of an FP64 conservative array [5][nz][ny][nx]:
// per-block FP64 partial sums of |m|^2 / (2 rho) |Omega_c| over rows of the
// grid (x over the threads), and, if grad is not null, the gradient
// d/dQ of scale * |m|^2 / (2 rho) |Omega_c| per cell (zero for rho E).
static __global__ void __launch_bounds__(256) k_kinetic(const double* __restrict__ cons, GridDev g,
                                                        const double* __restrict__ w, double scale,
                                                        double* __restrict__ grad,
                                                        double* __restrict__ part) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const double* wx = w;
  const double* wy = w + nx;
  const double* wz = w + nx + ny;
  double s = 0.0;
  const int rows = ny * nz;
  for (int row = blockIdx.x; row < rows; row += gridDim.x)
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const int y = row % ny, z = row / ny;
      const long long c = (long long)row * nx + x;
      const double vol = wx[x] * wy[y] * wz[z];
      const double rho = cons[c], mx = cons[g.N + c], my = cons[2 * g.N + c], mz = cons[3 * g.N + c];
      const double inv = 1.0 / rho;
      const double ke = 0.5 * (mx * mx + my * my + mz * mz) * inv;
      s += ke * vol;
      if (grad) {
        const double f = scale * vol;
        grad[c] = -ke * inv * f;
        grad[g.N + c] = mx * inv * f;
        grad[2 * g.N + c] = my * inv * f;
        grad[3 * g.N + c] = mz * inv * f;
        grad[4 * g.N + c] = 0.0;
      }
    }
  __shared__ double sm[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// Deterministic sum of the block partials (one block) times scale into *out.
static __global__ void __launch_bounds__(256) k_kinetic_final(const double* __restrict__ part, int nblocks,
                                                              double scale, double* __restrict__ out) {
  __shared__ double sm[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v * scale;
  }
}

cudaError_t enqueue_reset_scalars(const Engine& e) {
  k_reset_scalars<<<1, 32, 0, e.stream>>>(e.scal, e.dtmin, e.flag);
  return cudaGetLastError();
}

cudaError_t enqueue_set_dt(const Engine& e, double dt_fixed) {
  k_set_dt<<<1, 32, 0, e.stream>>>(e.scal, e.dtmin, e.cfg.cfl, dt_fixed, e.guard ? e.flag : nullptr);
  return cudaGetLastError();
}
cudaError_t enqueue_advance_time(const Engine& e) {
  k_advance_time<<<1, 32, 0, e.stream>>>(e.scal, e.guard ? e.flag : nullptr);
  return cudaGetLastError();
}

}  // namespace hgks

extern "C" {

hgks_status hgks_default_config(hgks_config* cfg, int n) {
  if (!cfg) return HGKS_E_INVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  const double pi = 3.14159265358979323846;
  cfg->nx = cfg->ny = cfg->nz = n;
  cfg->lx = cfg->ly = cfg->lz = 2.0 * pi;
  cfg->stretch_b = 2.0;
  cfg->bc_y = HGKS_BC_PERIODIC;
  cfg->gamma = 1.4;
  cfg->prandtl = 0.72;
  cfg->visc = HGKS_VISC_CONST;
  cfg->mu_ref = 1.0 / 1600.0;
  cfg->T_ref = 1.0;
  cfg->visc_exp = 0.76;
  cfg->T_wall = 1.0;
  cfg->recon = HGKS_RECON_LINEAR;
  cfg->flux = HGKS_FLUX_SMOOTH;
  cfg->tau_num_C = 0.0;
  cfg->cfl = 0.5;
  cfg->prec = HGKS_FP32;
  cfg->rho_ref = 1.0;
  cfg->p_ref = 100.0 / 1.4;  // rho0 c0^2 / gamma with c0 = V0 / Ma = 10
  return n >= 6 ? HGKS_OK : HGKS_E_INVAL;
}

hgks_status hgks_create(const hgks_config* cfg, void* stream, hgks_ctx** out) {
  if (!cfg || !out) return fail(nullptr, HGKS_E_INVAL, "null argument");
  *out = nullptr;
  const std::string why = hgks::validate_config(*cfg);
  if (!why.empty()) return fail(nullptr, HGKS_E_INVAL, why);
  hgks_ctx* c = new hgks_ctx();
  hgks::Engine& e = c->e;
  e.cfg = *cfg;
  e.stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&c->device);
  if (!e.stream) {
    // The legacy default stream cannot be captured into a graph: use a stream
    // of the context's own.
    const cudaError_t se = cudaStreamCreateWithFlags(&e.stream, cudaStreamNonBlocking);
    if (se != cudaSuccess) {
      delete c;
      return cuda_fail(nullptr, se, "cudaStreamCreateWithFlags");
    }
    c->own_stream = true;
  }
  e.n[0] = cfg->nx;
  e.n[1] = cfg->ny;
  e.n[2] = cfg->nz;
  for (int d = 0; d < 3; ++d) e.p[d] = e.n[d] + 6;
  e.P = (long long)e.p[0] * e.p[1] * e.p[2];
  e.N = (long long)e.n[0] * e.n[1] * e.n[2];
  const size_t es = elem_size(*cfg);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if (sms <= 0) sms = 152;
  e.sms = sms;
  e.cfl_blocks = sms * 4;
  e.diag_blocks = sms * 4;
  auto alloc = [&](void** p, size_t bytes) -> cudaError_t { return cudaMalloc(p, bytes); };
  cudaError_t err = cudaSuccess;
  if (err == cudaSuccess) err = alloc(&e.q, 5 * e.P * es);
  if (err == cudaSuccess) err = alloc(&e.qs, 5 * e.P * es);
  if (err == cudaSuccess) err = alloc(&e.qx, 5 * e.P * es);
  if (err == cudaSuccess) err = alloc(&e.inc, 5 * e.N * es);
  if (err == cudaSuccess && cfg->prec == HGKS_FP32) err = alloc(&e.comp, 5 * e.N * es);
  if (err == cudaSuccess && cfg->prec == HGKS_FP32) err = alloc(&e.comp2, 5 * e.N * es);
  for (int d = 0; d < 3 && err == cudaSuccess; ++d) err = alloc(&e.fd[d], hgks::face_flux_elems(e, d) * es);
  for (int d = 0; d < 3 && err == cudaSuccess; ++d) err = alloc(&e.w[d], (e.n[d] + 6) * es);
  if (err == cudaSuccess) err = alloc((void**)&e.scal, 4 * sizeof(double));
  if (err == cudaSuccess) err = alloc((void**)&e.dtmin, sizeof(unsigned long long));
  if (err == cudaSuccess) err = alloc((void**)&e.flag, sizeof(int));
  if (err == cudaSuccess) err = alloc((void**)&e.part, 8 * sizeof(double) * e.diag_blocks);
  if (err == cudaSuccess) err = alloc((void**)&e.diag_out, 8 * sizeof(double));
  if (err == cudaSuccess) err = alloc((void**)&e.io, 5 * e.N * sizeof(double));
  if (err != cudaSuccess) {
    const hgks_status s = cuda_fail(nullptr, err, "hgks_create allocation");
    free_all(e);
    if (c->own_stream) cudaStreamDestroy(e.stream);
    delete c;
    return s;
  }
  // Zero the padded buffers once so that unused ghost corners stay finite.
  err = cudaMemsetAsync(e.q, 0, 5 * e.P * es, e.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(e.qs, 0, 5 * e.P * es, e.stream);
  if (err == cudaSuccess && e.comp) err = cudaMemsetAsync(e.comp, 0, 5 * e.N * es, e.stream);
  if (err == cudaSuccess && e.comp2) err = cudaMemsetAsync(e.comp2, 0, 5 * e.N * es, e.stream);
  for (int d = 0; d < 3 && err == cudaSuccess; ++d) {
    const std::vector<double> w = widths(*cfg, d);
    err = cfg->prec == HGKS_FP32 ? upload_widths<float>(e, d, w) : upload_widths<double>(e, d, w);
  }
  if (err == cudaSuccess) {
    hgks::k_reset_scalars<<<1, 32, 0, e.stream>>>(e.scal, e.dtmin, e.flag);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(e.stream);
  if (err != cudaSuccess) {
    const hgks_status s = cuda_fail(nullptr, err, "hgks_create initialisation");
    free_all(e);
    if (c->own_stream) cudaStreamDestroy(e.stream);
    delete c;
    return s;
  }
  c->buf0 = e.q;
  *out = c;
  return HGKS_OK;
}

hgks_status hgks_destroy(hgks_ctx* c) {
  if (!c) return HGKS_OK;
  cudaStreamSynchronize(c->e.stream);
  drop_graphs(c);
  free_all(c->e);
  if (c->own_stream) cudaStreamDestroy(c->e.stream);
  delete c;
  return HGKS_OK;
}

static hgks_status init_common(hgks_ctx* c, const double* src, int is_host, int conservative) {
  if (!c || !src) return fail(c, HGKS_E_INVAL, "null argument");
  hgks::Engine& e = c->e;
  const double* dsrc = src;
  if (is_host) {
    HGKS_CHECK(c, cudaMemcpyAsync(e.io, src, 5 * e.N * sizeof(double), cudaMemcpyHostToDevice, e.stream));
    dsrc = e.io;
  }
  const bool f32 = e.cfg.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_from_fp64<float>(e, dsrc, conservative)
                    : hgks::enqueue_from_fp64<double>(e, dsrc, conservative));
  if (e.comp) HGKS_CHECK(c, cudaMemsetAsync(e.comp, 0, 5 * e.N * sizeof(float), e.stream));
  hgks::k_reset_scalars<<<1, 32, 0, e.stream>>>(e.scal, e.dtmin, e.flag);
  HGKS_CHECK(c, cudaGetLastError());
  c->steps_host = c->init_steps = 0;
  if (is_host) HGKS_CHECK(c, cudaStreamSynchronize(e.stream));  // the host buffer is borrowed
  return HGKS_OK;
}

hgks_status hgks_init_state(hgks_ctx* c, const double* prim, int is_host) {
  return init_common(c, prim, is_host, 0);
}
hgks_status hgks_init_conservative(hgks_ctx* c, const double* cons, int is_host) {
  return init_common(c, cons, is_host, 1);
}

hgks_status hgks_set_time(hgks_ctx* c, double t, long long step) {
  if (!c || step < 0) return fail(c, HGKS_E_INVAL, "null context or negative step");
  hgks::k_set_time<<<1, 32, 0, c->e.stream>>>(c->e.scal, t, double(step));
  HGKS_CHECK(c, cudaGetLastError());
  c->steps_host = c->init_steps = step;
  return HGKS_OK;
}

hgks_status hgks_get_state(hgks_ctx* c, double* out, int is_host) {
  if (!c || !out) return fail(c, HGKS_E_INVAL, "null argument");
  hgks::Engine& e = c->e;
  double* dst = is_host ? e.io : out;
  const bool f32 = e.cfg.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_to_fp64<float>(e, dst) : hgks::enqueue_to_fp64<double>(e, dst));
  if (is_host) {
    HGKS_CHECK(c, cudaMemcpyAsync(out, e.io, 5 * e.N * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
    HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  }
  return HGKS_OK;
}

hgks_status hgks_step(hgks_ctx* c, int nsteps, double dt, int sync, double* t_out) {
  if (!c) return fail(c, HGKS_E_INVAL, "null context");
  if (nsteps < 0) return fail(c, HGKS_E_INVAL, "nsteps must be non-negative");
  hgks::Engine& e = c->e;
  const double dt_fixed = dt > 0.0 ? dt : 0.0;
  for (int n = 0; n < nsteps; ++n) {
    const int k = e.q == c->buf0 ? 0 : 1;
    if (!c->graph[k] || c->graph_dt[k] != dt_fixed) {
      const hgks_status s = capture_step(c, k, dt_fixed);
      if (s != HGKS_OK) return s;
    }
    HGKS_CHECK(c, cudaGraphLaunch(c->graph[k], e.stream));
    hgks::swap_state_buffers(e);
    ++c->steps_host;
  }
  if (!sync) return HGKS_OK;
  // Check the state reached: the CFL kernel flags rho <= 0, p <= 0 and NaN.
  // The flag raised by the CFL kernel of a step stopped that step and every
  // later one from writing, so the state before the first non-physical one
  // is still in one of the two buffers.
  const bool f32 = e.cfg.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_cfl<float>(e, e.q) : hgks::enqueue_cfl<double>(e, e.q));
  double scal[3];
  int flag = 0;
  HGKS_CHECK(c, cudaMemcpyAsync(scal, e.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaMemcpyAsync(&flag, e.flag, sizeof(int), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  if (!flag) {
    if (t_out) *t_out = scal[1];
    return HGKS_OK;
  }
  // scal[2] steps completed, the last of them non-physical (or, if none was
  // completed since the state was set, the state set was non-physical).
  const long long done = (long long)scal[2];
  // The last good state: after done - 1 steps, or, if no step completed since
  // the state was set (the state set was non-physical), that state.  The
  // state after s steps is in q if steps_host - s is even, else in qs.
  const bool rolled = done > c->init_steps;
  const long long target = rolled ? done - 1 : done;
  if (((c->steps_host - target) & 1LL) != 0) hgks::swap_state_buffers(e);
  c->steps_host = target;
  char buf[160];
  if (rolled) {
    const double t_good = scal[1] - scal[0];
    hgks::k_set_time<<<1, 32, 0, e.stream>>>(e.scal, t_good, double(target));
    HGKS_CHECK(c, cudaGetLastError());
    if (t_out) *t_out = t_good;
    std::snprintf(buf, sizeof buf,
                  "non-physical state (rho <= 0, p <= 0 or NaN) after step %lld; the state is left "
                  "at step %lld",
                  done, target);
  } else {
    if (t_out) *t_out = scal[1];
    std::snprintf(buf, sizeof buf,
                  "non-physical state (rho <= 0, p <= 0 or NaN) at step %lld, the state set by the "
                  "caller; no step was taken",
                  done);
  }
  // Clear the flag (and the CFL minimum) so that the caller may continue,
  // e.g. with a smaller fixed dt.
  hgks::k_reset_flag<<<1, 32, 0, e.stream>>>(e.dtmin, e.flag);
  HGKS_CHECK(c, cudaGetLastError());
  HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  return fail(c, HGKS_E_NONPHYSICAL, buf);
}

hgks_status hgks_diagnostics(hgks_ctx* c, hgks_diag* out) {
  if (!c || !out) return fail(c, HGKS_E_INVAL, "null argument");
  hgks::Engine& e = c->e;
  const bool f32 = e.cfg.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_diag<float>(e) : hgks::enqueue_diag<double>(e));
  double r[8], scal[4];
  HGKS_CHECK(c, cudaMemcpyAsync(r, e.diag_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaMemcpyAsync(scal, e.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  const double vol = e.cfg.lx * e.cfg.ly * e.cfg.lz;
  out->t = scal[1];
  out->dt = scal[0];
  out->step = (long long)scal[2];
  out->mass = r[0];
  out->mom[0] = r[1];
  out->mom[1] = r[2];
  out->mom[2] = r[3];
  out->energy = r[4];
  out->Ek = r[5] / (e.cfg.rho_ref * vol);
  out->rho_min = r[6];
  out->p_min = r[7];
  out->force_x = e.cfg.force_mode == HGKS_FORCE_MASS_FLUX ? scal[3] : e.cfg.force_x;
  return HGKS_OK;
}

// Linear solve of a small dense system by Gaussian elimination with partial
// pivoting (n <= 4): the cell-average fits of the channel statistics.
static void solve_small(int n, double* A, double* b) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
    for (int k = 0; k < n; ++k) std::swap(A[col * n + k], A[piv * n + k]);
    std::swap(b[col], b[piv]);
    for (int r = col + 1; r < n; ++r) {
      const double f = A[r * n + col] / A[col * n + col];
      for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double t = b[r];
    for (int k = r + 1; k < n; ++k) t -= A[r * n + k] * b[k];
    b[r] = t / A[r * n + r];
  }
}

// Mean over [a, b] of s^p.
static double mean_pow(double a, double b, int p) {
  return (std::pow(b, p + 1) - std::pow(a, p + 1)) / ((p + 1) * (b - a));
}

// d<U>/ds at a wall (s = distance from it) from the averages U1, U2 of the
// first two cells, [0, w1] and [w1, w1 + w2]: the quadratic a s + b s^2 with
// U = 0 at the wall whose cell averages are U1 and U2; returns a.
static double wall_gradient(double w1, double w2, double U1, double U2) {
  double A[4] = {mean_pow(0, w1, 1), mean_pow(0, w1, 2), mean_pow(w1, w1 + w2, 1), mean_pow(w1, w1 + w2, 2)};
  double r[2] = {U1, U2};
  solve_small(2, A, r);
  return r[0];
}

hgks_status hgks_channel_compose(const hgks_config* cfp, const double* means, double* profiles,
                                 hgks_channel* out) {
  if (!cfp || !means || !out) return fail(nullptr, HGKS_E_INVAL, "null argument");
  const hgks_config& cf = *cfp;
  const std::string why = hgks::validate_config(cf);
  if (!why.empty()) return fail(nullptr, HGKS_E_INVAL, why);
  if (cf.bc_y != HGKS_BC_WALL_ISOTHERMAL)
    return fail(nullptr, HGKS_E_UNSUPPORTED, "channel statistics need the isothermal walls in y");
  const int ny = cf.ny, NS = hgks::kChanSums;
  const double* m = means;
  const std::vector<double> w = widths(cf, 1);  // includes 3 ghosts per side
  auto wy = [&](int j) { return w[j + 3]; };
  const double* rho = &m[0];
  const double* U = &m[2 * ny];
  const double* V = &m[3 * ny];
  const double* UV = &m[5 * ny];
  // Wall shear stress (Sec. 3.3): tau_w = mu(T_wall) d<U>/dn at each wall.
  const double a_lo = wall_gradient(wy(0), wy(1), U[0], U[1]);
  const double a_hi = wall_gradient(wy(ny - 1), wy(ny - 2), U[ny - 1], U[ny - 2]);
  const double mu_w = cf.visc == HGKS_VISC_POWER ? cf.mu_ref * std::pow(cf.T_wall / cf.T_ref, cf.visc_exp)
                                                 : cf.mu_ref;
  out->t = 0.0;
  out->tau_w_lower = mu_w * a_lo;
  out->tau_w_upper = mu_w * a_hi;
  out->tau_w = 0.5 * (out->tau_w_lower + out->tau_w_upper);
  out->mu_w = mu_w;
  out->rho_w = 0.5 * (rho[0] + rho[ny - 1]);
  out->u_tau = std::sqrt(std::fmax(out->tau_w, 0.0) / out->rho_w);
  const double H = 0.5 * cf.ly;
  out->Re_tau = out->rho_w * out->u_tau * H / mu_w;
  // Bulk means over the height.
  double ub = 0.0, rb = 0.0;
  for (int j = 0; j < ny; ++j) {
    ub += U[j] * wy(j);
    rb += rho[j] * wy(j);
  }
  out->U_b = ub / cf.ly;
  out->rho_b = rb / cf.ly;
  // Centreline <U>: the cubic whose averages over the four cells nearest the
  // mid-plane equal theirs, at the mid-plane.
  std::vector<double> yf(ny + 1);
  yf[0] = cf.y0;
  for (int j = 0; j < ny; ++j) yf[j + 1] = yf[j] + wy(j);
  const double yc = cf.y0 + H;
  int j0 = 0;
  double best = 1e300;
  for (int j = 0; j + 3 < ny; ++j) {  // the window of four cells centred best on yc
    const double d = std::fabs(0.5 * (yf[j] + yf[j + 4]) - yc);
    if (d < best) {
      best = d;
      j0 = j;
    }
  }
  if (ny >= 4) {
    double A[16], r[4];
    for (int k = 0; k < 4; ++k) {
      for (int pw = 0; pw < 4; ++pw) A[k * 4 + pw] = mean_pow(yf[j0 + k] - yc, yf[j0 + k + 1] - yc, pw);
      r[k] = U[j0 + k];
    }
    solve_small(4, A, r);
    out->U_c = r[0];
  } else {
    out->U_c = U[ny / 2];
  }
  const double nu = mu_w / out->rho_b;
  out->Re_c = out->U_c * H / nu;
  out->Re_b = out->U_b * 2.0 * H / nu;
  out->C_f = out->tau_w / (0.5 * out->rho_b * out->U_b * out->U_b);
  if (!profiles) return HGKS_OK;
  // Plane means, then the wall-unit profiles of each row j (cell centre y_j):
  // y+ = rho_w u_tau d_j / mu_w with d_j the distance to the nearer wall,
  // U+ = <U>/u_tau, <u'v'>+ = (<UV> - <U><V>)/u_tau^2, dU+/dY+ =
  // mu_w d<U>/dy / (rho_w u_tau^2) (d<U>/dy by the second-order difference
  // of the row means on the non-uniform centres, one-sided at the first and
  // last rows), and the total-stress residual of the stationary channel,
  // dU+/dY+ - <u'v'>+ - (1 - Y+/Re_tau) (Sec. 3.3).
  std::memcpy(profiles, m, sizeof(double) * NS * ny);
  double* y = profiles + NS * ny;
  double* yp = y + ny;
  double* Up = yp + ny;
  double* uvp = Up + ny;
  double* dUp = uvp + ny;
  double* res = dUp + ny;
  const double ut = out->u_tau, ut2 = ut * ut;
  for (int j = 0; j < ny; ++j) {
    y[j] = 0.5 * (yf[j] + yf[j + 1]);
    const double dist = std::fmin(y[j] - cf.y0, cf.y0 + cf.ly - y[j]);
    yp[j] = out->rho_w * ut * dist / mu_w;
    Up[j] = U[j] / ut;
    uvp[j] = (UV[j] - U[j] * V[j]) / ut2;
  }
  for (int j = 0; j < ny; ++j) {
    double g;
    if (j == 0) {
      g = (U[1] - U[0]) / (y[1] - y[0]);
    } else if (j == ny - 1) {
      g = (U[ny - 1] - U[ny - 2]) / (y[ny - 1] - y[ny - 2]);
    } else {
      const double hs = y[j] - y[j - 1], hd = y[j + 1] - y[j];
      g = (hs * hs * U[j + 1] + (hd * hd - hs * hs) * U[j] - hd * hd * U[j - 1]) / (hs * hd * (hd + hs));
    }
    dUp[j] = mu_w * g / (out->rho_w * ut2);
    res[j] = dUp[j] - uvp[j] - (1.0 - yp[j] / out->Re_tau);
  }
  return HGKS_OK;
}

hgks_status hgks_channel_stats(hgks_ctx* c, double* profiles, hgks_channel* out) {
  if (!c || !out) return fail(c, HGKS_E_INVAL, "null argument");
  hgks::Engine& e = c->e;
  const hgks_config& cf = e.cfg;
  if (cf.bc_y != HGKS_BC_WALL_ISOTHERMAL)
    return fail(c, HGKS_E_UNSUPPORTED, "channel statistics need the isothermal walls in y");
  const int ny = e.n[1], NS = hgks::kChanSums;
  if (!e.chan_out) HGKS_CHECK(c, cudaMalloc((void**)&e.chan_out, sizeof(double) * NS * ny));
  const bool f32 = cf.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_channel_rows<float>(e) : hgks::enqueue_channel_rows<double>(e));
  std::vector<double> m(size_t(NS) * ny);
  double scal[3];
  HGKS_CHECK(c, cudaMemcpyAsync(m.data(), e.chan_out, m.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                e.stream));
  HGKS_CHECK(c, cudaMemcpyAsync(scal, e.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  const double cells = double(e.n[0]) * e.n[2];
  for (double& v : m) v /= cells;  // plane means
  const hgks_status st = hgks_channel_compose(&cf, m.data(), profiles, out);
  if (st != HGKS_OK) return fail(c, st, g_create_error);
  out->t = scal[1];
  return HGKS_OK;
}

hgks_status hgks_kinetic_energy(hgks_ctx* c, const double* cons, double* grad, double* ek_out) {
  if (!c || !cons || !ek_out) return fail(c, HGKS_E_INVAL, "null argument");
  hgks::Engine& e = c->e;
  if (!e.kin_w) {
    std::vector<double> w;
    for (int d = 0; d < 3; ++d) {
      const std::vector<double> wd = widths(e.cfg, d);
      w.insert(w.end(), wd.begin() + 3, wd.end() - 3);
    }
    HGKS_CHECK(c, cudaMalloc((void**)&e.kin_w, w.size() * sizeof(double)));
    HGKS_CHECK(c, cudaMemcpyAsync(e.kin_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  e.stream));
    HGKS_CHECK(c, cudaStreamSynchronize(e.stream));  // w is a host temporary
  }
  hgks::GridDev g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = e.n[d];
    g.p[d] = e.p[d];
  }
  g.P = e.P;
  g.N = e.N;
  const double scale = 1.0 / (e.cfg.rho_ref * e.cfg.lx * e.cfg.ly * e.cfg.lz);
  hgks::k_kinetic<<<e.diag_blocks, 256, 0, e.stream>>>(cons, g, e.kin_w, scale, grad, e.part);
  HGKS_CHECK(c, cudaGetLastError());
  hgks::k_kinetic_final<<<1, 256, 0, e.stream>>>(e.part, e.diag_blocks, scale, e.diag_out);
  HGKS_CHECK(c, cudaGetLastError());
  HGKS_CHECK(c, cudaMemcpyAsync(ek_out, e.diag_out, sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  return HGKS_OK;
}

hgks_status hgks_cell_widths(const hgks_config* cfg, int axis, double* out) {
  if (!cfg || !out || axis < 0 || axis > 2) return fail(nullptr, HGKS_E_INVAL, "bad argument");
  const std::string why = hgks::validate_config(*cfg);
  if (!why.empty()) return fail(nullptr, HGKS_E_INVAL, why);
  const std::vector<double> w = widths(*cfg, axis);
  const int n = axis == 0 ? cfg->nx : (axis == 1 ? cfg->ny : cfg->nz);
  for (int j = 0; j < n; ++j) out[j] = w[j + 3];
  return HGKS_OK;
}

// The statistics of include/hgks.h from the kTurbSums raw sums r.
static void turb_from_sums(const hgks_config& cf, const double* r, double t, hgks_turbulence* out) {
  using namespace hgks;
  const double V = r[TS_VOL], rho0 = cf.rho_ref;
  auto avg = [&](int k) { return r[k] / V; };
  out->t = t;
  out->K = avg(TS_KE);
  out->Ek = out->K / rho0;
  out->zeta = avg(TS_ENS) / rho0;
  out->eps1 = 2.0 * avg(TS_MU_SDSD) / rho0;
  out->eps2 = avg(TS_MUB_TH2) / rho0;
  out->eps3 = -avg(TS_P_TH) / rho0;
  const double dm = avg(TS_DRHO);
  out->rho_mean = rho0 + dm;
  out->rho_rms = std::sqrt(std::fmax(avg(TS_DRHO2) - dm * dm, 0.0));
  out->u_rms = std::sqrt(avg(TS_Q2) / 3.0);
  double su = 0.0, fu = 0.0;
  int live = 0;
  for (int i = 0; i < 3; ++i) {
    const double m2 = avg(TS_DU2 + i), m3 = avg(TS_DU3 + i), m4 = avg(TS_DU4 + i);
    out->du2[i] = m2;
    out->du3[i] = m3;
    out->du4[i] = m4;
    if (m2 > 0.0) {
      su += m3 / (m2 * std::sqrt(m2));
      fu += m4 / (m2 * m2);
      ++live;
    }
  }
  out->Su = live ? su / live : 0.0;
  out->Fu = live ? fu / live : 0.0;
  out->eps_s = avg(TS_MU_W2);
  out->eps_d = 4.0 / 3.0 * avg(TS_MU_TH2);
  out->p_theta = avg(TS_P_TH);
  out->theta_rms = std::sqrt(avg(TS_TH2));
  out->omega_rms = std::sqrt(avg(TS_W2));
  // Sec. 3.1: eps(zeta) = 2 mu zeta / rho0 with the reference viscosity mu_ref.
  out->eps_zeta = 2.0 * cf.mu_ref * out->zeta / rho0;
}

static bool periodic_uniform(const hgks_config& cf) {
  return cf.bc_y == HGKS_BC_PERIODIC && !cf.y_stretch;
}

hgks_status hgks_turbulence_stats(hgks_ctx* c, hgks_turbulence* out) {
  if (!c || !out) return fail(c, HGKS_E_INVAL, "null argument");
  hgks::Engine& e = c->e;
  if (!periodic_uniform(e.cfg))
    return fail(c, HGKS_E_UNSUPPORTED, "turbulence statistics need a periodic uniform grid");
  constexpr int NS = hgks::kTurbSums;
  if (!e.turb_part) {
    HGKS_CHECK(c, cudaMalloc((void**)&e.turb_part, sizeof(double) * NS * e.diag_blocks));
    HGKS_CHECK(c, cudaMalloc((void**)&e.turb_out, sizeof(double) * NS));
  }
  const bool f32 = e.cfg.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_turbulence<float>(e) : hgks::enqueue_turbulence<double>(e));
  double r[NS], scal[3];
  HGKS_CHECK(c, cudaMemcpyAsync(r, e.turb_out, NS * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaMemcpyAsync(scal, e.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
  HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  turb_from_sums(e.cfg, r, scal[1], out);
  return HGKS_OK;
}

hgks_status hgks_history_start(hgks_ctx* c, int every, int capacity) {
  if (!c || every <= 0 || capacity <= 0) return fail(c, HGKS_E_INVAL, "bad history arguments");
  hgks::Engine& e = c->e;
  if (!periodic_uniform(e.cfg))
    return fail(c, HGKS_E_UNSUPPORTED, "the statistics history needs a periodic uniform grid");
  if (!e.turb_part) {
    HGKS_CHECK(c, cudaMalloc((void**)&e.turb_part, sizeof(double) * hgks::kTurbSums * e.diag_blocks));
    HGKS_CHECK(c, cudaMalloc((void**)&e.turb_out, sizeof(double) * hgks::kTurbSums));
  }
  if (e.hist_cap < capacity) {
    if (e.hist) cudaFree(e.hist);
    e.hist = nullptr;
    e.hist_cap = 0;
    HGKS_CHECK(c, cudaMalloc((void**)&e.hist, sizeof(double) * hgks::kHistStride * capacity));
    e.hist_cap = capacity;
  }
  e.hist_cap = capacity;
  if (!e.hist_count) HGKS_CHECK(c, cudaMalloc((void**)&e.hist_count, sizeof(int)));
  HGKS_CHECK(c, cudaMemsetAsync(e.hist_count, 0, sizeof(int), e.stream));
  e.hist_every = every;
  drop_graphs(c);  // the captured steps gain the record
  // The first record: the current state.
  const bool f32 = e.cfg.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_history_record<float>(e, e.q, false)
                    : hgks::enqueue_history_record<double>(e, e.q, false));
  return HGKS_OK;
}

hgks_status hgks_history_stop(hgks_ctx* c) {
  if (!c) return fail(c, HGKS_E_INVAL, "null context");
  if (c->e.hist_every != 0) {
    c->e.hist_every = 0;
    drop_graphs(c);
  }
  return HGKS_OK;
}

hgks_status hgks_history_read(hgks_ctx* c, hgks_history_rec* out, int capacity, int* count) {
  if (!c || !count || capacity < 0 || (capacity > 0 && !out)) return fail(c, HGKS_E_INVAL, "bad argument");
  hgks::Engine& e = c->e;
  int n = 0;
  if (e.hist_count) {
    HGKS_CHECK(c, cudaMemcpyAsync(&n, e.hist_count, sizeof(int), cudaMemcpyDeviceToHost, e.stream));
    HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  }
  *count = n;
  const int m = std::min(n, capacity);
  if (m == 0) return HGKS_OK;
  std::vector<double> raw(size_t(hgks::kHistStride) * n);
  HGKS_CHECK(c, cudaMemcpyAsync(raw.data(), e.hist, raw.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                e.stream));
  HGKS_CHECK(c, cudaStreamSynchronize(e.stream));
  std::vector<double> t(n), ek(n);
  std::vector<hgks_history_rec> rec(n);
  for (int i = 0; i < n; ++i) {
    const double* r = &raw[size_t(hgks::kHistStride) * i];
    turb_from_sums(e.cfg, r + 2, r[0], &rec[i].s);
    rec[i].step = (long long)r[1];
    t[i] = r[0];
    ek[i] = rec[i].s.Ek;
  }
  // eps(E_k) = -dE_k/dt (Sec. 3.1) by second-order differences of the
  // recorded history on its (possibly non-uniform) times: the central
  // formula inside, the one-sided three-point formula at both ends; two
  // records give the one difference, one record none (NaN).
  for (int i = 0; i < n; ++i) {
    double d = std::nan("");
    if (n >= 3) {
      if (i == 0 || i == n - 1) {
        const int a = i == 0 ? 0 : n - 1, s1 = i == 0 ? 1 : -1;
        const double h1 = t[a + s1] - t[a], h2 = t[a + 2 * s1] - t[a + s1];
        d = -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * ek[a] + (h1 + h2) / (h1 * h2) * ek[a + s1] -
            h1 / (h2 * (h1 + h2)) * ek[a + 2 * s1];
      } else {
        const double hl = t[i] - t[i - 1], hr = t[i + 1] - t[i];
        d = (hl * hl * ek[i + 1] + (hr * hr - hl * hl) * ek[i] - hr * hr * ek[i - 1]) / (hl * hr * (hl + hr));
      }
    } else if (n == 2) {
      d = (ek[1] - ek[0]) / (t[1] - t[0]);
    }
    rec[i].eps_Ek = -d;
    // Sec. 3.1: the numerical dissipation eps(E_k) - (eps1 + eps2 + eps3).
    rec[i].eps_num = rec[i].eps_Ek - (rec[i].s.eps1 + rec[i].s.eps2 + rec[i].s.eps3);
  }
  std::memcpy(out, rec.data(), sizeof(hgks_history_rec) * m);
  return HGKS_OK;
}

hgks_status hgks_adjoint_step(hgks_ctx* c, double dt, const double* adj_in, double* adj_out) {
  if (!c || !adj_in || !adj_out) return fail(c, HGKS_E_INVAL, "null argument");
  if (!(dt > 0.0)) return fail(c, HGKS_E_INVAL, "the adjoint needs the forward step dt > 0");
  hgks::Engine& e = c->e;
  if (e.cfg.bc_y != HGKS_BC_PERIODIC)
    return fail(c, HGKS_E_UNSUPPORTED, "the adjoint supports periodic boundaries only");
  if (e.cfg.force_x != 0.0 || e.cfg.force_mode != HGKS_FORCE_CONSTANT)
    return fail(c, HGKS_E_UNSUPPORTED, "the adjoint has no body force");
  if (e.cfg.recon_vars != 0 && e.cfg.recon != HGKS_RECON_LINEAR)
    return fail(c, HGKS_E_UNSUPPORTED, "the adjoint reconstructs conservative variables only");
  const size_t es = elem_size(e.cfg);
  if (!e.adj_acc) {
    HGKS_CHECK(c, cudaMalloc(&e.adj_acc, 5 * e.P * es));
    HGKS_CHECK(c, cudaMalloc(&e.adj_mu, 5 * e.N * es));
    HGKS_CHECK(c, cudaMalloc(&e.adj_wL, 5 * e.N * es));
    HGKS_CHECK(c, cudaMalloc(&e.adj_wdL, 5 * e.N * es));
  }
  HGKS_CHECK(c, hgks::enqueue_set_dt(e, dt));
  const bool f32 = e.cfg.prec == HGKS_FP32;
  HGKS_CHECK(c, f32 ? hgks::enqueue_adjoint_step<float>(e, adj_in, adj_out)
                    : hgks::enqueue_adjoint_step<double>(e, adj_in, adj_out));
  return HGKS_OK;
}

struct hgks_ensemble {
  std::vector<hgks_ctx*> members;
  cudaStream_t stream = nullptr;  // the first member's stream: fork and join point
  std::vector<cudaEvent_t> events;
  // Captured batch steps, each for the members' state-buffer assignment at
  // capture (the members' q pointers); the assignment alternates every step,
  // so two slots serve a run.
  struct Slot {
    cudaGraphExec_t graph = nullptr;
    double dt = -1.0;
    std::vector<void*> q;
  } slot[2];
  int next_slot = 0;
  bool batched = false;  // one batched launch per phase (else graph branches)
  std::string err;
};

// Whether the members can share batched launches: same precision,
// reconstruction (and variables), flux and sweep tile variant, no mass-flux
// force and no statistics history.
static bool ensemble_batchable(const hgks_ensemble* en) {
  const hgks::Engine& a = en->members[0]->e;
  for (hgks_ctx* c : en->members) {
    const hgks::Engine& e = c->e;
    if (e.cfg.prec != a.cfg.prec || e.cfg.recon != a.cfg.recon || e.cfg.flux != a.cfg.flux ||
        e.cfg.recon_vars != a.cfg.recon_vars || e.sweep_variant != a.sweep_variant ||
        e.cfg.force_mode != HGKS_FORCE_CONSTANT || e.hist_every != 0)
      return false;
  }
  return true;
}

hgks_status hgks_ensemble_create(hgks_ctx** ctxs, int n, hgks_ensemble** out) {
  if (!ctxs || n <= 0 || !out) return fail(nullptr, HGKS_E_INVAL, "bad ensemble arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(nullptr, HGKS_E_INVAL, "null member");
    if (ctxs[i]->device != ctxs[0]->device) return fail(nullptr, HGKS_E_INVAL, "members on different devices");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || ctxs[j]->e.stream == ctxs[i]->e.stream)
        return fail(nullptr, HGKS_E_INVAL, "members must be distinct contexts on distinct streams");
  }
  hgks_ensemble* en = new hgks_ensemble();
  en->members.assign(ctxs, ctxs + n);
  en->stream = ctxs[0]->e.stream;
  en->events.resize(n + 1, nullptr);
  for (auto& ev : en->events) {
    const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (auto& x : en->events)
        if (x) cudaEventDestroy(x);
      delete en;
      return cuda_fail(nullptr, e, "cudaEventCreateWithFlags");
    }
  }
  en->batched = ensemble_batchable(en);
  *out = en;
  return HGKS_OK;
}

hgks_status hgks_ensemble_set_batched(hgks_ensemble* en, int batched) {
  if (!en) return HGKS_E_INVAL;
  if (batched && !ensemble_batchable(en)) {
    en->err = "batched launches need members of one precision, scheme and tile variant, without the "
              "mass-flux force or a statistics history";
    return HGKS_E_UNSUPPORTED;
  }
  if (en->batched != (batched != 0)) {
    en->batched = batched != 0;
    for (auto& sl : en->slot)
      if (sl.graph) {
        cudaGraphExecDestroy(sl.graph);
        sl.graph = nullptr;
      }
  }
  return HGKS_OK;
}

hgks_status hgks_ensemble_destroy(hgks_ensemble* en) {
  if (!en) return HGKS_OK;
  cudaStreamSynchronize(en->stream);
  for (auto& sl : en->slot)
    if (sl.graph) cudaGraphExecDestroy(sl.graph);
  for (auto& ev : en->events)
    if (ev) cudaEventDestroy(ev);
  delete en;
  return HGKS_OK;
}

// One graph holding every member's step as a parallel branch: fork from the
// first member's stream, each member's kernels on its own stream, join back.
static hgks_status capture_ensemble(hgks_ensemble* en, hgks_ensemble::Slot& sl, double dt_fixed) {
  if (sl.graph) {
    cudaGraphExecDestroy(sl.graph);
    sl.graph = nullptr;
  }
  cudaStream_t s0 = en->stream;
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) {
    en->err = std::string("capture: ") + cudaGetErrorString(err);
    return HGKS_E_CUDA;
  }
  const int n = (int)en->members.size();
  if (en->batched) {
    // One launch per phase over all members, on the first member's stream.
    std::vector<hgks::Engine*> ms;
    for (hgks_ctx* c : en->members) ms.push_back(&c->e);
    err = en->members[0]->e.cfg.prec == HGKS_FP32 ? hgks::enqueue_batched_step<float>(ms, dt_fixed, s0)
                                                   : hgks::enqueue_batched_step<double>(ms, dt_fixed, s0);
  } else {
    err = cudaEventRecord(en->events[0], s0);
  }
  for (int i = 0; i < n && err == cudaSuccess && !en->batched; ++i) {
    hgks::Engine& e = en->members[i]->e;
    if (e.stream != s0) err = cudaStreamWaitEvent(e.stream, en->events[0], 0);
    if (err == cudaSuccess) err = enqueue_stage_pair(e, dt_fixed);
    if (err == cudaSuccess && e.stream != s0) {
      err = cudaEventRecord(en->events[i + 1], e.stream);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(s0, en->events[i + 1], 0);
    }
  }
  const cudaError_t end = cudaStreamEndCapture(s0, &g);
  if (err == cudaSuccess) err = end;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&sl.graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (err != cudaSuccess) {
    en->err = std::string("ensemble capture: ") + cudaGetErrorString(err);
    return err == cudaErrorMemoryAllocation ? HGKS_E_NOMEM : HGKS_E_CUDA;
  }
  sl.dt = dt_fixed;
  sl.q.clear();
  for (hgks_ctx* c : en->members) sl.q.push_back(c->e.q);
  return HGKS_OK;
}

hgks_status hgks_ensemble_step(hgks_ensemble* en, int nsteps, double dt, int sync) {
  if (!en || nsteps < 0) return HGKS_E_INVAL;
  const double dt_fixed = dt > 0.0 ? dt : 0.0;
  const int nm = (int)en->members.size();
  // The batch runs on the first member's stream: it waits for the work
  // already enqueued on the other members' streams, and they wait for it.
  if (nsteps > 0) {
    for (int i = 1; i < nm; ++i) {
      cudaError_t e = cudaEventRecord(en->events[i + 1], en->members[i]->e.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(en->stream, en->events[i + 1], 0);
      if (e != cudaSuccess) {
        en->err = std::string("ordering the member streams: ") + cudaGetErrorString(e);
        return HGKS_E_CUDA;
      }
    }
  }
  for (int n = 0; n < nsteps; ++n) {
    // The slot captured for the members' current buffer assignment, or a new capture.
    hgks_ensemble::Slot* sl = nullptr;
    for (auto& cand : en->slot) {
      bool same = cand.graph && cand.dt == dt_fixed && cand.q.size() == en->members.size();
      for (size_t i = 0; same && i < en->members.size(); ++i) same = cand.q[i] == en->members[i]->e.q;
      if (same) sl = &cand;
    }
    if (!sl) {
      sl = &en->slot[en->next_slot];
      en->next_slot ^= 1;
      const hgks_status s = capture_ensemble(en, *sl, dt_fixed);
      if (s != HGKS_OK) return s;
    }
    const cudaError_t e = cudaGraphLaunch(sl->graph, en->stream);
    if (e != cudaSuccess) {
      en->err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
      return HGKS_E_CUDA;
    }
    for (hgks_ctx* c : en->members) {
      hgks::swap_state_buffers(c->e);
      ++c->steps_host;
    }
  }
  if (nsteps > 0) {
    cudaError_t e = cudaEventRecord(en->events[0], en->stream);
    for (int i = 1; i < nm && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(en->members[i]->e.stream, en->events[0], 0);
    if (e != cudaSuccess) {
      en->err = std::string("ordering the member streams: ") + cudaGetErrorString(e);
      return HGKS_E_CUDA;
    }
  }
  if (!sync) return HGKS_OK;
  // Per-member state check, as in hgks_step.
  for (hgks_ctx* c : en->members) {
    const hgks_status s = hgks_step(c, 0, dt, 1, nullptr);
    if (s != HGKS_OK) {
      en->err = c->err;
      return s;
    }
  }
  return HGKS_OK;
}

const char* hgks_ensemble_last_error(const hgks_ensemble* en) { return en ? en->err.c_str() : ""; }

hgks_status hgks_autotune(hgks_ctx* c, int* variant_out, int* chunk_out, double* ms_out) {
  if (!c) return fail(c, HGKS_E_INVAL, "null context");
  hgks::Engine& e = c->e;
  const bool f32 = e.cfg.prec == HGKS_FP32;
  // The state is not changed: only the stage-1 ghost fill and sweeps run (they
  // write the ghost layers and the face-flux buffers).
  HGKS_CHECK(c, f32 ? hgks::enqueue_ghosts<float>(e, e.q) : hgks::enqueue_ghosts<double>(e, e.q));
  HGKS_CHECK(c, hgks::enqueue_set_dt(e, 1e-3));
  cudaEvent_t t0, t1;
  HGKS_CHECK(c, cudaEventCreate(&t0));
  HGKS_CHECK(c, cudaEventCreate(&t1));
  const int nmax = std::max(e.n[0], std::max(e.n[1], e.n[2])) + 1;
  const int chunks[] = {0, 8, 16, 32, 64, 128};
  float best = 1e30f;
  int best_v = 0, best_c = 0;
  cudaError_t err = cudaSuccess;
  for (int v = 0; v < hgks::sweep_variant_count(e) && err == cudaSuccess; ++v) {
    for (int ci = 0; ci < 6 && err == cudaSuccess; ++ci) {
      if (chunks[ci] > 2 * nmax) continue;
      e.sweep_variant = v;
      e.sweep_chunk = chunks[ci];
      float ms = 0.f;
      for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {  // rep 0 warms up
        if (rep == 1) err = cudaEventRecord(t0, e.stream);
        for (int d = 0; d < 3 && err == cudaSuccess; ++d)
          err = f32 ? hgks::enqueue_sweep_only<float>(e, d) : hgks::enqueue_sweep_only<double>(e, d);
      }
      if (err == cudaSuccess) err = cudaEventRecord(t1, e.stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(t1);
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t0, t1);
      if (err == cudaSuccess && ms < best) {
        best = ms;
        best_v = v;
        best_c = chunks[ci];
      }
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  HGKS_CHECK(c, err);
  e.sweep_variant = best_v;
  e.sweep_chunk = best_c;
  drop_graphs(c);  // the captured steps hold the old launch shapes
  if (variant_out) *variant_out = best_v;
  if (chunk_out) *chunk_out = best_c;
  if (ms_out) *ms_out = best / 2.0;
  return HGKS_OK;
}

hgks_status hgks_set_sweep_shape(hgks_ctx* c, int variant, int chunk) {
  if (!c) return fail(c, HGKS_E_INVAL, "null context");
  if (variant < 0 || variant >= hgks::sweep_variant_count(c->e) || chunk < 0)
    return fail(c, HGKS_E_INVAL, "no such sweep variant");
  c->e.sweep_variant = variant;
  c->e.sweep_chunk = chunk;
  drop_graphs(c);
  return HGKS_OK;
}

hgks_status hgks_profile_step(hgks_ctx* c, double dt, double* ms_out, int nclass) {
  if (!c || !ms_out || nclass < hgks::KC_COUNT) return fail(c, HGKS_E_INVAL, "bad argument");
  hgks::Engine& e = c->e;
  hgks::Probe probe;
  for (int i = 0; i < hgks::Probe::kMax; ++i) {
    HGKS_CHECK(c, cudaEventCreate(&probe.start[i]));
    HGKS_CHECK(c, cudaEventCreate(&probe.stop[i]));
  }
  const cudaError_t err = enqueue_stage_pair(e, dt > 0.0 ? dt : 0.0, &probe);
  if (err == cudaSuccess) {
    hgks::swap_state_buffers(e);
    ++c->steps_host;
  }
  cudaError_t sync = cudaStreamSynchronize(e.stream);
  for (int k = 0; k < nclass; ++k) ms_out[k] = 0.0;
  for (int i = 0; i < probe.n && sync == cudaSuccess; ++i) {
    float ms = 0.f;
    sync = cudaEventElapsedTime(&ms, probe.start[i], probe.stop[i]);
    ms_out[probe.cls[i]] += ms;
  }
  for (int i = 0; i < hgks::Probe::kMax; ++i) {
    cudaEventDestroy(probe.start[i]);
    cudaEventDestroy(probe.stop[i]);
  }
  HGKS_CHECK(c, err);
  HGKS_CHECK(c, sync);
  return HGKS_OK;
}

const char* hgks_last_error(const hgks_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

namespace hgks {

int sweep_variant_count(const Engine& e) {
  return (e.cfg.prec == HGKS_FP32 && e.cfg.recon == HGKS_RECON_LINEAR &&
          e.cfg.flux == HGKS_FLUX_SMOOTH) ? 4 : 1;
}

long long face_flux_elems(const Engine& e, int d) {
  long long s = 1;
  for (int c = 0; c < 3; ++c) s *= (c == d) ? e.n[c] + 1 : e.n[c];
  return s * 10;
}

}  // namespace hgks
