// qcl_api.cu -- host implementation of the C ABI declared in include/qcl.h:
// argument validation, buffer sizing, model constants, and the launch
// sequences of the FP64 comparator and the FP32-bulk persistent path.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "model.h"

using namespace qcl;


namespace {

thread_local std::string g_err;
int64_t g_opt_grid_cap = 0;
bool g_opt_timing = false;
int g_opt_modes_mem = 0;
std::mutex g_tmu;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_events[2];

// Event pair around one launch of kernel class `which` when timing is on.
struct TimedLaunch {
  int which;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedLaunch(int w, cudaStream_t st) : which(w), s(st) {
    if (!g_opt_timing) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  ~TimedLaunch() {
    if (!a) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_tmu);
    g_events[which].push_back({a, b});
  }
};

qcl_status fail(qcl_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

qcl_status ok() {
  g_err.clear();
  return QCL_OK;
}

#define CUDA_TRY(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(QCL_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

qcl_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCL_ERR_CUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
  return QCL_OK;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

bool symmetric(const double* A, int ns) {
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < i; ++j) {
      const double x = A[i * ns + j], y = A[j * ns + i];
      if (std::fabs(x - y) > 1e-12 * (1.0 + std::fabs(x) + std::fabs(y))) return false;
    }
  return true;
}

qcl_status check_ens(const qcl_model* m, const qcl_ensemble_desc* e) {
  if (!m) return fail(QCL_ERR_INVALID_ARG, "model is NULL");
  if (!e) return fail(QCL_ERR_INVALID_ARG, "ensemble descriptor is NULL");
  if (e->n_traj < 1) return fail(QCL_ERR_INVALID_ARG, "n_traj must be >= 1 (got %lld)", (long long)e->n_traj);
  if (e->n_traj > (int64_t)1 << 40) return fail(QCL_ERR_INVALID_ARG, "n_traj too large");
  if (e->precision != QCL_PREC_FP64 && e->precision != QCL_PREC_FP32_BULK)
    return fail(QCL_ERR_INVALID_ARG, "unknown precision %d", e->precision);
  return QCL_OK;
}

}  // namespace

namespace qcl {
qcl_status set_error(qcl_status st, const char* msg) {
  g_err = msg ? msg : "";
  return st;
}
qcl_status check_ensemble(const qcl_model* m, const qcl_ensemble_desc* e) { return check_ens(m, e); }
int64_t option_grid_cap() { return g_opt_grid_cap; }
int option_modes_in_memory() { return g_opt_modes_mem; }
}  // namespace qcl

extern "C" {

const char* qcl_last_error(void) { return g_err.c_str(); }

const char* qcl_version(void) { return "qcl-gb300 0.1 (sm_103a)"; }

qcl_status qcl_set_option(int32_t key, int64_t value) {
  if (key == QCL_OPT_GRID_CAP) {
    if (value < 0) return fail(QCL_ERR_INVALID_ARG, "grid cap must be >= 0");
    g_opt_grid_cap = value;
    return ok();
  }
  if (key == QCL_OPT_TIMING) {
    g_opt_timing = value != 0;
    return ok();
  }
  if (key == QCL_OPT_MODES_IN_MEMORY) {
    if (value < 0 || value > 2) return fail(QCL_ERR_INVALID_ARG, "modes-in-memory option takes 0, 1 or 2");
    g_opt_modes_mem = (int)value;
    return ok();
  }
  return fail(QCL_ERR_INVALID_ARG, "unknown option %d", key);
}

qcl_status qcl_launch_count(int64_t* count, int32_t reset) {
  if (!count) return fail(QCL_ERR_INVALID_ARG, "count is NULL");
  *count = launches_read(reset != 0);
  return ok();
}

qcl_status qcl_kernel_time(int32_t which, double* total_ms, int64_t* launches) {
  if (which < 0 || which > 1) return fail(QCL_ERR_INVALID_ARG, "unknown kernel class %d", which);
  if (!total_ms || !launches) return fail(QCL_ERR_INVALID_ARG, "NULL output");
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    ev.swap(g_events[which]);
  }
  double tot = 0.0;
  qcl_status st = QCL_OK;
  for (auto& p : ev) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(p.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.first, p.second);
    if (e != cudaSuccess && st == QCL_OK) st = fail(QCL_ERR_CUDA, "event timing failed: %s", cudaGetErrorString(e));
    tot += ms;
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  *total_ms = tot;
  *launches = (int64_t)ev.size();
  return st ? st : ok();
}

qcl_status qcl_ensemble_layout(const qcl_model* model, const qcl_ensemble_desc* ens, size_t offsets[11]) {
  if (!offsets) return fail(QCL_ERR_INVALID_ARG, "offsets is NULL");
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  const EnsLayout L = EnsLayout::make(ens->n_traj, model->ns, model->n, ens->precision);
  offsets[0] = L.off_R;
  offsets[1] = L.off_P;
  offsets[2] = L.off_m;
  offsets[3] = L.off_mlo;
  offsets[4] = L.off_phi;
  offsets[5] = L.off_philo;
  offsets[6] = L.off_ab;
  offsets[7] = L.total;
  offsets[8] = L.off_mexp;
  offsets[9] = L.off_U;
  offsets[10] = L.off_E;
  return ok();
}

qcl_status qcl_ensemble_restore(const qcl_model* model, const qcl_ensemble_desc* ens, void* ens_buf,
                                size_t ens_bytes, int64_t step, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!ens_buf) return fail(QCL_ERR_INVALID_ARG, "ens_buf is NULL");
  if (((uintptr_t)ens_buf & 255) != 0) return fail(QCL_ERR_INVALID_ARG, "ens_buf must be 256-byte aligned");
  if (step < 0) return fail(QCL_ERR_INVALID_ARG, "step must be >= 0 (got %lld)", (long long)step);
  const EnsLayout L = EnsLayout::make(ens->n_traj, model->ns, model->n, ens->precision);
  if (ens_bytes < L.total) return fail(QCL_ERR_OUT_OF_MEMORY, "ens_buf holds %zu bytes, needs %zu", ens_bytes, L.total);
  EnsHeader h{};
  h.magic = kEnsMagic;
  h.n_traj = ens->n_traj;
  h.precision = ens->precision;
  h.ns = model->ns;
  h.n = model->n;
  h.step = step;
  launch_header_set(ens_buf, h, (cudaStream_t)stream);
  CUDA_TRY(cudaGetLastError());
  return ok();
}

qcl_status qcl_create_model(const qcl_model_desc* d, qcl_model** out) {
  if (!out) return fail(QCL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(QCL_ERR_INVALID_ARG, "model descriptor is NULL");
  const int ns = d->n_states, n = d->n_modes;
  if (ns < 2 || ns > QCL_MAX_STATES) return fail(ns < 2 ? QCL_ERR_INVALID_ARG : QCL_ERR_UNSUPPORTED, "n_states = %d outside [2, %d]", ns, QCL_MAX_STATES);
  if (n < 1 || n > QCL_MAX_MODES) return fail(n < 1 ? QCL_ERR_INVALID_ARG : QCL_ERR_UNSUPPORTED, "n_modes = %d outside [1, %d]", n, QCL_MAX_MODES);
  if (!d->mass || !d->omega || !d->E || !d->K) return fail(QCL_ERR_INVALID_ARG, "a model array is NULL");
  if (!(d->hbar > 0.0) || !std::isfinite(d->hbar)) return fail(QCL_ERR_INVALID_ARG, "hbar must be positive");
  const double hop = d->hop_scale == 0.0 ? 1.0 : d->hop_scale;
  const double pmax = d->p_max == 0.0 ? 0.5 : d->p_max;
  // (bounds that keep one step's weight factor within [2^-16, 2^17] wherever
  // it follows from the model: the FP32-bulk steps check the weight's range
  // only every fourth step)
  if (!(hop >= 0x1p-16 && hop <= 0x1p16)) return fail(QCL_ERR_INVALID_ARG, "hop_scale = %g outside [2^-16, 2^16]", hop);
  if (!(pmax > 0.0 && pmax <= 1.0 - 0x1p-16)) return fail(QCL_ERR_INVALID_ARG, "p_max = %g outside (0, 1 - 2^-16]", pmax);
  if (d->repr != QCL_REPR_ADIABATIC && d->repr != QCL_REPR_DIABATIC) return fail(QCL_ERR_INVALID_ARG, "repr = %d is neither adiabatic (0) nor diabatic (1)", d->repr);
  if (d->reserved != 0) return fail(QCL_ERR_INVALID_ARG, "reserved must be 0");
  for (int j = 0; j < n; ++j) {
    if (!(d->mass[j] > 0.0) || !std::isfinite(d->mass[j])) return fail(QCL_ERR_INVALID_ARG, "mass[%d] must be positive", j);
    if (!(d->omega[j] > 0.0) || !std::isfinite(d->omega[j])) return fail(QCL_ERR_INVALID_ARG, "omega[%d] must be positive", j);
  }
  const size_t nn = (size_t)ns * ns;
  if (!finite_all(d->E, nn) || !finite_all(d->K, nn * n)) return fail(QCL_ERR_INVALID_ARG, "E or K has a non-finite entry");
  if (!symmetric(d->E, ns)) return fail(QCL_ERR_INVALID_ARG, "E is not symmetric");
  for (int j = 0; j < n; ++j)
    if (!symmetric(d->K + nn * j, ns)) return fail(QCL_ERR_INVALID_ARG, "K[%d] is not symmetric", j);

  qcl_model* m = new (std::nothrow) qcl_model();
  if (!m) return fail(QCL_ERR_OUT_OF_MEMORY, "host allocation failed");
  m->ns = ns;
  m->n = n;
  m->hbar = d->hbar;
  m->hop_scale = hop;
  m->p_max = pmax;
  m->mass.assign(d->mass, d->mass + n);
  m->omega.assign(d->omega, d->omega + n);
  m->E.assign(d->E, d->E + nn);
  m->K.assign(d->K, d->K + nn * n);
  DevModel& h = m->host;
  h.ns = ns;
  h.n = n;
  h.hbar = d->hbar;
  h.hop_scale = hop;
  h.p_max = pmax;
  bool general = false;
  if (ns == 2) {
    // W = s 1 + a sigma_z + b sigma_x,  a = (W00 - W11)/2, b = W01, s = (W00 + W11)/2
    h.a0 = 0.5 * (d->E[0] - d->E[3]);
    h.b0 = d->E[1];
    h.s0 = 0.5 * (d->E[0] + d->E[3]);
  }
  for (int j = 0; j < n; ++j) {
    h.mass[j] = d->mass[j];
    h.omega[j] = d->omega[j];
    h.k[j] = d->mass[j] * d->omega[j] * d->omega[j];
    if (ns == 2) {
      const double* Kj = d->K + 4 * j;
      h.a[j] = 0.5 * (Kj[0] - Kj[3]);
      h.b[j] = Kj[1];
      h.s[j] = 0.5 * (Kj[0] + Kj[3]);
      if (h.b[j] != 0.0 || h.s[j] != 0.0) general = true;
    }
  }
  for (size_t k = 0; k < nn; ++k) h.E[k] = d->E[k];
  h.kind = general ? 1 : 0;
  h.repr = d->repr;
  int dev = 0;
  cudaGetDevice(&dev);
  m->device = dev;
  char* blk = nullptr;
  const size_t bytes = sizeof(DevModel) + sizeof(double) * nn * n;
  cudaError_t e = cudaMalloc((void**)&blk, bytes);
  if (e != cudaSuccess) {
    delete m;
    return fail(e == cudaErrorMemoryAllocation ? QCL_ERR_OUT_OF_MEMORY : QCL_ERR_CUDA, "cudaMalloc of the model block failed: %s", cudaGetErrorString(e));
  }
  h.K = (const double*)(blk + sizeof(DevModel));
  e = cudaMemcpy(blk, &h, sizeof(DevModel), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(blk + sizeof(DevModel), d->K, sizeof(double) * nn * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(blk);
    delete m;
    return fail(QCL_ERR_CUDA, "copy of the model block failed: %s", cudaGetErrorString(e));
  }
  m->dev = (DevModel*)blk;
  *out = m;
  return ok();
}

qcl_status qcl_destroy_model(qcl_model* model) {
  if (!model) return ok();
  if (model->dev) cudaFree(model->dev);
  delete model;
  return ok();
}

qcl_status qcl_ensemble_bytes(const qcl_model* model, const qcl_ensemble_desc* ens, size_t* bytes) {
  if (!bytes) return fail(QCL_ERR_INVALID_ARG, "bytes is NULL");
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  *bytes = EnsLayout::make(ens->n_traj, model->ns, model->n, ens->precision).total;
  return ok();
}

qcl_status qcl_obs_bytes(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t n_out, size_t* bytes) {
  if (!bytes) return fail(QCL_ERR_INVALID_ARG, "bytes is NULL");
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (n_out < 1) return fail(QCL_ERR_INVALID_ARG, "n_out must be >= 1");
  *bytes = ObsLayout::make(ens->n_traj, model->ns, n_out, tile_walkers(ens->precision, model->n, model->ns)).total;
  return ok();
}

}  // extern "C"

namespace {
// FP32 per-mode coefficients of a two-state model for time step dt.
void fill_coef2(const qcl_model* model, double dt, Coef2* cf) {
  const DevModel& h = model->host;
  for (int j = 0; j < model->n; ++j) {
    cf->hk[j] = (float)(0.5 * dt * h.k[j]);
    cf->hs[j] = (float)(0.5 * dt * h.s[j]);
    cf->dtm[j] = (float)(dt / h.mass[j]);
    cf->a[j] = (float)h.a[j];
    cf->b[j] = (float)h.b[j];
    cf->am[j] = (float)(h.a[j] / h.mass[j]);
    cf->bm[j] = (float)(h.b[j] / h.mass[j]);
  }
}

// FP32 per-mode coefficients of an N_s-state model for one time step dt
// (upper triangles of E and of each K_j; the per-mode arrays hold the first 32
// modes, the kernels that keep the modes in memory build the whole table on
// the device from the model pointer and dt stored here).
void fill_coefN(const qcl_model* model, double dt, CoefN& cn) {
  const DevModel& h = model->host;
  const int ns = model->ns;
  auto tri = [ns](int a, int b) { return a * ns - a * (a - 1) / 2 + (b - a); };
  for (int a = 0; a < ns; ++a)
    for (int b = a; b < ns; ++b) cn.E[tri(a, b)] = (float)model->E[a * ns + b];
  const int n_reg = model->n < 32 ? model->n : 32;
  for (int j = 0; j < n_reg; ++j) {
    cn.hk[j] = (float)(0.5 * dt * h.k[j]);
    cn.dtm[j] = (float)(dt / h.mass[j]);
    cn.minv[j] = (float)(1.0 / h.mass[j]);
    for (int a = 0; a < ns; ++a)
      for (int b = a; b < ns; ++b) cn.K[j][tri(a, b)] = (float)model->K[(size_t)j * ns * ns + a * ns + b];
  }
  coef_set_model(cn, model->dev, dt);
  cn.modes_in_memory = g_opt_modes_mem;
}

void make_sampleN32(const qcl_model* model, const SampleParams& sp, SampleN32& s) {
  const int ns = model->ns, n = model->n;
  s.n_traj = sp.n_traj;
  s.traj_offset = sp.traj_offset;
  s.seed = sp.seed;
  s.n = n;
  s.ns = ns;
  s.wigner = sp.wigner;
  s.repr = model->host.repr;
  for (int j = 0; j < kMaxN; ++j) {
    const bool on = j < n;
    s.R0[j] = on ? (float)sp.R0[j] : 0.0f;
    s.P0[j] = on ? (float)sp.P0[j] : 0.0f;
    s.sR[j] = on ? (float)sp.sR[j] : 0.0f;
    s.sP[j] = on ? (float)sp.sP[j] : 0.0f;
  }
  for (int k = 0; k < kMaxNS * kMaxNS; ++k) {
    s.E[k] = k < ns * ns ? (float)model->E[k] : 0.0f;
    s.rho[k] = k < ns * ns ? (float)sp.rho[k] : 0.0f;
  }
  const size_t nk = (size_t)n * ns * ns;
  for (size_t k = 0; k < (size_t)kSampleNK; ++k) s.K[k] = k < nk ? (float)model->K[k] : 0.0f;
  s.Kd = model->host.K;
}

// Validates an initial condition and builds the sampling parameters.
qcl_status prepare_sample(const qcl_model* model, const qcl_ensemble_desc* ens, const qcl_init_desc* init,
                          SampleParams** out) {
  *out = nullptr;
  if (!init || !init->rho_el0 || !init->R0 || !init->P0) return fail(QCL_ERR_INVALID_ARG, "init descriptor or one of its arrays is NULL");
  const int ns = model->ns, n = model->n;
  if (!finite_all(init->rho_el0, (size_t)ns * ns) || !symmetric(init->rho_el0, ns)) return fail(QCL_ERR_INVALID_ARG, "rho_el0 must be finite and symmetric");
  bool nz = false;
  for (int k = 0; k < ns * ns; ++k) nz |= init->rho_el0[k] != 0.0;
  if (!nz) return fail(QCL_ERR_INVALID_ARG, "rho_el0 is zero");
  if (!finite_all(init->R0, n) || !finite_all(init->P0, n)) return fail(QCL_ERR_INVALID_ARG, "R0 or P0 has a non-finite entry");
  if (init->wigner && !(init->beta > 0.0)) return fail(QCL_ERR_INVALID_ARG, "beta must be positive (INFINITY for the ground state)");
  SampleParams* sp = new (std::nothrow) SampleParams();
  if (!sp) return fail(QCL_ERR_OUT_OF_MEMORY, "host allocation failed");
  sp->n_traj = ens->n_traj;
  sp->traj_offset = ens->traj_id_offset;
  sp->seed = ens->seed;
  sp->n = n;
  sp->ns = ns;
  sp->wigner = init->wigner ? 1 : 0;
  for (int j = 0; j < n; ++j) {
    const double M = model->mass[j], w = model->omega[j], hb = model->hbar;
    const double cth = std::isinf(init->beta) ? 1.0 : 1.0 / std::tanh(0.5 * init->beta * hb * w);
    sp->R0[j] = init->R0[j];
    sp->P0[j] = init->P0[j];
    sp->sR[j] = std::sqrt(hb / (2.0 * M * w) * cth);
    sp->sP[j] = std::sqrt(0.5 * hb * M * w * cth);
  }
  for (int k = 0; k < ns * ns; ++k) sp->rho[k] = init->rho_el0[k];
  *out = sp;
  return QCL_OK;
}
}  // namespace

extern "C" {

qcl_status qcl_sample_initial(const qcl_model* model, const qcl_ensemble_desc* ens, const qcl_init_desc* init,
                              void* ens_buf, size_t ens_bytes, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!ens_buf) return fail(QCL_ERR_INVALID_ARG, "ens_buf is NULL");
  if (((uintptr_t)ens_buf & 255) != 0) return fail(QCL_ERR_INVALID_ARG, "ens_buf must be 256-byte aligned");
  const size_t need = EnsLayout::make(ens->n_traj, model->ns, model->n, ens->precision).total;
  if (ens_bytes < need) return fail(QCL_ERR_OUT_OF_MEMORY, "ens_buf has %zu bytes, needs %zu", ens_bytes, need);
  SampleParams* sp = nullptr;
  st = prepare_sample(model, ens, init, &sp);
  if (st) return st;
  const int ns = model->ns;
  cudaStream_t s = (cudaStream_t)stream;
  if (ns > 2) {
    SampleN32* s32 = nullptr;
    if (ens->precision == QCL_PREC_FP32_BULK) {
      s32 = new (std::nothrow) SampleN32();
      if (!s32) {
        delete sp;
        return fail(QCL_ERR_OUT_OF_MEMORY, "host allocation failed");
      }
      make_sampleN32(model, *sp, *s32);
    }
    launch_sampleN(model->dev, *sp, s32, ens_buf, ens->precision, s);
    delete s32;
  }
  else if (ens->precision == QCL_PREC_FP64)
    launch_sample_f64(model->dev, *sp, ens_buf, s);
  else
    launch_sample_f32(model->host, *sp, ens_buf, s);
  delete sp;
  st = check_launch("sample");
  return st ? st : ok();
}

qcl_status qcl_propagate(const qcl_model* model, const qcl_ensemble_desc* ens, void* ens_buf, size_t ens_bytes,
                         int64_t step0, int64_t n_steps, double dt, int32_t out_stride, void* obs_buf,
                         size_t obs_bytes, int64_t n_out, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!ens_buf || !obs_buf) return fail(QCL_ERR_INVALID_ARG, "ens_buf or obs_buf is NULL");
  if (((uintptr_t)ens_buf & 255) != 0 || ((uintptr_t)obs_buf & 255) != 0) return fail(QCL_ERR_INVALID_ARG, "buffers must be 256-byte aligned");
  if (step0 < 0 || n_steps < 0) return fail(QCL_ERR_INVALID_ARG, "step0 and n_steps must be >= 0");
  if (step0 + n_steps >= ((int64_t)1 << 34)) return fail(QCL_ERR_INVALID_ARG, "absolute step beyond 2^34");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(QCL_ERR_INVALID_ARG, "dt must be positive");
  if (out_stride < 1) return fail(QCL_ERR_INVALID_ARG, "out_stride must be >= 1");
  if (n_out < 1) return fail(QCL_ERR_INVALID_ARG, "n_out must be >= 1");
  const int64_t k_last = (step0 + n_steps) / out_stride;
  if (k_last >= n_out) return fail(QCL_ERR_INVALID_ARG, "output row %lld beyond n_out = %lld", (long long)k_last, (long long)n_out);
  const EnsLayout EL = EnsLayout::make(ens->n_traj, model->ns, model->n, ens->precision);
  if (ens_bytes < EL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "ens_buf has %zu bytes, needs %zu", ens_bytes, EL.total);
  const ObsLayout OL = ObsLayout::make(ens->n_traj, model->ns, n_out, tile_walkers(ens->precision, model->n, model->ns));
  if (obs_bytes < OL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "obs_buf has %zu bytes, needs %zu", obs_bytes, OL.total);
  cudaStream_t s = (cudaStream_t)stream;
  char* ob = (char*)obs_buf;
  double* rows = (double*)(ob + OL.off_rows);
  double* part = (double*)(ob + OL.off_part);
  double* fold = (double*)(ob + OL.off_fold);
  const int q2 = OL.q2;
  const int64_t nt = ens->n_traj;
  // per-chunk sums of output row k (only kept when there is more than one chunk)
  auto chunk_row = [&](int64_t k) -> double* {
    return OL.n_fold_blocks > 1 ? (double*)(ob + OL.off_chunk) + (size_t)k * OL.n_fold_blocks * q2 : nullptr;
  };

  if (ens->precision == QCL_PREC_FP64) {
    const int ns = model->ns;
    auto observe = [&](int64_t k) {
      if (ns == 2)
        launch_observe_f64(model->dev, ens_buf, nt, model->n, part, s);
      else
        launch_observeN_f64(model->dev, ns, ens_buf, nt, model->n, part, s);
      launch_fold(part, rows + (size_t)k * q2, fold, OL.n_tiles, q2, 1, s, chunk_row(k));
    };
    if (step0 == 0) observe(0);
    for (int64_t t = step0; t < step0 + n_steps; ++t) {
      {
        TimedLaunch tl(1, s);
        if (ns == 2)
          launch_step_f64(model->dev, model->host.repr, ens_buf, nt, model->n, step0, t, dt, ens->seed, ens->traj_id_offset, s);
        else
          launch_stepN_f64(model->dev, model->host.repr, ns, ens_buf, nt, model->n, step0, t, dt, ens->seed, ens->traj_id_offset, s);
      }
      if ((t + 1) % out_stride == 0) observe((t + 1) / out_stride);
    }
    st = check_launch("FP64 step");
    if (st) return st;
  } else {
    Coef2* cf = new (std::nothrow) Coef2();
    if (!cf) return fail(QCL_ERR_OUT_OF_MEMORY, "host allocation failed");
    const DevModel& h = model->host;
    fill_coef2(model, dt, cf);
    BulkParams bp{};
    bp.n_traj = nt;
    bp.n_tiles = OL.n_tiles;
    bp.traj_offset = ens->traj_id_offset;
    bp.seed = ens->seed;
    bp.step0 = step0;
    bp.stride = out_stride;
    bp.n = model->n;
    bulk_model_scalars(bp, h, dt);
    CoefN* cn = nullptr;
    if (model->ns > 2) {
      cn = new (std::nothrow) CoefN();
      if (!cn) {
        delete cf;
        return fail(QCL_ERR_OUT_OF_MEMORY, "host allocation failed");
      }
      fill_coefN(model, dt, *cn);
    }
    // chunks of at most outs (the launch shape's outputs per launch) output times
    const int outs = model->shape_outs > 0 ? model->shape_outs : kChunkOut;
    int64_t cs = step0;
    bool first = (step0 == 0);
    const int64_t end = step0 + n_steps;
    do {
      int64_t k_first = first ? 0 : cs / out_stride + 1;
      int n_slots = first ? 1 : 0;
      int64_t ce = cs;
      // extend to the (outs - n_slots)-th output step after cs, or to end
      const int64_t next_out = (cs / out_stride + 1) * out_stride;
      const int64_t room = outs - n_slots;
      int64_t last_out = next_out + (room - 1) * out_stride;
      if (last_out <= end) {
        ce = last_out;
        n_slots += (int)room;
      } else {
        ce = end;
        if (end >= next_out) n_slots += (int)((end - next_out) / out_stride + 1);
      }
      if (!first && n_slots > 0) k_first = next_out / out_stride;
      if (ce - cs > ((int64_t)1 << 30)) {  // keep the in-kernel step count in 32 bits
        ce = cs + ((int64_t)1 << 30);
        const int64_t k_last_out = ce / out_stride;
        n_slots = (first ? 1 : 0) + (int)(k_last_out >= next_out / out_stride ? k_last_out - next_out / out_stride + 1 : 0);
      }
      bp.cs = cs;
      bp.ce = ce;
      bp.k_first = k_first;
      bp.obs_first = first ? 1 : 0;
      bp.len = (int32_t)(ce - cs);
      bp.to_out0 = (int32_t)(out_stride - (cs % out_stride));
      bp.blk0 = (uint32_t)(cs >> 2);
      bp.widx0 = (int32_t)(cs & 3);
      int grid = 0;
      {
        TimedLaunch tl(0, s);
        LaunchShape ls;
        ls.wpt = model->shape_wpt;
        ls.blocks_per_sm = model->shape_bps;
        ls.grid_cap = (int)g_opt_grid_cap;
        grid = cn ? launch_bulkN(model->ns, bp, *cn, ens_buf, part, ls, s)
                  : launch_bulk2(bp, *cf, ens_buf, part, ls, s);
      }
      if (grid == 0) {
        delete cf;
        delete cn;
        return fail(QCL_ERR_UNSUPPORTED, "no FP32-bulk kernel for n_modes = %d", model->n);
      }
      if (n_slots > 0)
        launch_fold(part, rows + (size_t)k_first * q2, fold, OL.n_tiles, q2, n_slots, s, chunk_row(k_first));
      first = false;
      cs = ce;
    } while (cs < end);
    delete cf;
    delete cn;
    st = check_launch("FP32-bulk propagate");
    if (st) return st;
  }
  launch_header_finish(ens_buf, step0, step0 + n_steps, s);
  st = check_launch("header");
  return st ? st : ok();
}

qcl_status qcl_reduce_observables(const qcl_model* model, const qcl_ensemble_desc* ens, const void* obs_buf,
                                  size_t obs_bytes, int64_t n_out, int64_t k0, int64_t n_rows, double* host_out,
                                  size_t host_len, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!obs_buf || !host_out) return fail(QCL_ERR_INVALID_ARG, "obs_buf or host_out is NULL");
  if (n_out < 1 || k0 < 0 || n_rows < 0 || k0 + n_rows > n_out) return fail(QCL_ERR_INVALID_ARG, "rows [%lld, %lld) outside [0, %lld)", (long long)k0, (long long)(k0 + n_rows), (long long)n_out);
  const ObsLayout OL = ObsLayout::make(ens->n_traj, model->ns, n_out, tile_walkers(ens->precision, model->n, model->ns));
  if (obs_bytes < OL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "obs_buf has %zu bytes, needs %zu", obs_bytes, OL.total);
  const int nq = OL.q2 / 2;
  const size_t per = (size_t)(2 * nq + 3);
  if (host_len < per * (size_t)n_rows) return fail(QCL_ERR_INVALID_ARG, "host_out holds %zu doubles, needs %zu", host_len, per * (size_t)n_rows);
  if (n_rows == 0) return ok();
  cudaStream_t s = (cudaStream_t)stream;
  const char* ob = (const char*)obs_buf;
  double* fin = (double*)(ob + OL.off_fin);
  launch_finalize((const double*)(ob + OL.off_rows), fin, nq, k0, n_rows, ens->n_traj, model->ns, s);
  st = check_launch("finalize");
  if (st) return st;
  CUDA_TRY(cudaMemcpyAsync(host_out, fin, sizeof(double) * per * n_rows, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return ok();
}

qcl_status qcl_finalize_observables(const qcl_model* model, const qcl_ensemble_desc* ens, const void* obs_buf,
                                    size_t obs_bytes, int64_t n_out, int64_t k0, int64_t n_rows, double* dev_out,
                                    size_t dev_len, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!obs_buf || !dev_out) return fail(QCL_ERR_INVALID_ARG, "obs_buf or dev_out is NULL");
  if (n_out < 1 || k0 < 0 || n_rows < 0 || k0 + n_rows > n_out) return fail(QCL_ERR_INVALID_ARG, "rows [%lld, %lld) outside [0, %lld)", (long long)k0, (long long)(k0 + n_rows), (long long)n_out);
  const ObsLayout OL = ObsLayout::make(ens->n_traj, model->ns, n_out, tile_walkers(ens->precision, model->n, model->ns));
  if (obs_bytes < OL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "obs_buf has %zu bytes, needs %zu", obs_bytes, OL.total);
  const int nq = OL.q2 / 2;
  const size_t per = (size_t)(2 * nq + 3);
  if (dev_len < per * (size_t)n_rows) return fail(QCL_ERR_INVALID_ARG, "dev_out holds %zu doubles, needs %zu", dev_len, per * (size_t)n_rows);
  if (n_rows == 0) return ok();
  launch_finalize((const double*)((const char*)obs_buf + OL.off_rows), dev_out, nq, k0, n_rows, ens->n_traj,
                  model->ns, (cudaStream_t)stream);
  st = check_launch("finalize");
  return st ? st : ok();
}

qcl_status qcl_read_chunk_sums(const qcl_model* model, const qcl_ensemble_desc* ens, const void* obs_buf,
                               size_t obs_bytes, int64_t n_out, int64_t k0, int64_t n_rows, double* host_out,
                               size_t host_len, int64_t* n_chunks, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!obs_buf || !n_chunks) return fail(QCL_ERR_INVALID_ARG, "obs_buf or n_chunks is NULL");
  if (n_out < 1 || k0 < 0 || n_rows < 0 || k0 + n_rows > n_out) return fail(QCL_ERR_INVALID_ARG, "rows outside [0, n_out)");
  const ObsLayout OL = ObsLayout::make(ens->n_traj, model->ns, n_out, tile_walkers(ens->precision, model->n, model->ns));
  if (obs_bytes < OL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "obs_buf has %zu bytes, needs %zu", obs_bytes, OL.total);
  *n_chunks = OL.n_fold_blocks;
  if (!host_out) return ok();  // size query
  const size_t per_row = (size_t)OL.n_fold_blocks * OL.q2;
  if (host_len < per_row * n_rows) return fail(QCL_ERR_INVALID_ARG, "host_out holds %zu doubles, needs %zu", host_len, per_row * n_rows);
  if (n_rows == 0) return ok();
  cudaStream_t s = (cudaStream_t)stream;
  // one chunk: its sums are the rows themselves
  const size_t off = OL.n_fold_blocks > 1 ? OL.off_chunk : OL.off_rows;
  const double* src = (const double*)((const char*)obs_buf + off) + (size_t)k0 * per_row;
  CUDA_TRY(cudaMemcpyAsync(host_out, src, sizeof(double) * per_row * n_rows, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return ok();
}

qcl_status qcl_read_sums(const qcl_model* model, const qcl_ensemble_desc* ens, const void* obs_buf, size_t obs_bytes,
                         int64_t n_out, int64_t k0, int64_t n_rows, double* host_out, size_t host_len, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!obs_buf || !host_out) return fail(QCL_ERR_INVALID_ARG, "obs_buf or host_out is NULL");
  if (n_out < 1 || k0 < 0 || n_rows < 0 || k0 + n_rows > n_out) return fail(QCL_ERR_INVALID_ARG, "rows outside [0, n_out)");
  const ObsLayout OL = ObsLayout::make(ens->n_traj, model->ns, n_out, tile_walkers(ens->precision, model->n, model->ns));
  if (obs_bytes < OL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "obs_buf has %zu bytes, needs %zu", obs_bytes, OL.total);
  if (host_len < (size_t)OL.q2 * n_rows) return fail(QCL_ERR_INVALID_ARG, "host_out too small");
  if (n_rows == 0) return ok();
  cudaStream_t s = (cudaStream_t)stream;
  const double* rows = (const double*)((const char*)obs_buf + OL.off_rows);
  CUDA_TRY(cudaMemcpyAsync(host_out, rows + (size_t)k0 * OL.q2, sizeof(double) * OL.q2 * n_rows, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return ok();
}

qcl_status qcl_ensemble_status(const qcl_model* model, const qcl_ensemble_desc* ens, const void* ens_buf,
                               size_t ens_bytes, qcl_ens_status* out, void* stream) {
  qcl_status st = check_ens(model, ens);
  if (st) return st;
  if (!ens_buf || !out) return fail(QCL_ERR_INVALID_ARG, "ens_buf or out is NULL");
  if (ens_bytes < sizeof(EnsHeader)) return fail(QCL_ERR_OUT_OF_MEMORY, "ens_buf too small");
  EnsHeader h;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(&h, ens_buf, sizeof(h), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h.magic != kEnsMagic) return fail(QCL_ERR_INVALID_ARG, "ens_buf holds no sampled ensemble");
  out->step = h.step;
  out->flags = h.flags;
  out->reserved = 0;
  out->n_degenerate = h.n_degenerate;
  out->n_nonfinite = h.n_nonfinite;
  return ok();
}

// ------------------------------------------------------------ launch shape --
qcl_status qcl_set_launch_shape(qcl_model* model, const qcl_launch_shape* shape) {
  if (!model || !shape) return fail(QCL_ERR_INVALID_ARG, "model or shape is NULL");
  if (shape->walkers_per_thread < 0 || shape->walkers_per_thread > 2)
    return fail(QCL_ERR_INVALID_ARG, "walkers_per_thread must be 0, 1 or 2");
  if (shape->blocks_per_sm < 0) return fail(QCL_ERR_INVALID_ARG, "blocks_per_sm must be >= 0");
  if (shape->outputs_per_launch < 0 || shape->outputs_per_launch > kChunkOut)
    return fail(QCL_ERR_INVALID_ARG, "outputs_per_launch must be in [0, %d]", kChunkOut);
  model->shape_wpt = shape->walkers_per_thread;
  model->shape_bps = shape->blocks_per_sm;
  model->shape_outs = shape->outputs_per_launch;
  model->shape_rate = shape->walker_steps_per_s;
  return ok();
}

qcl_status qcl_get_launch_shape(const qcl_model* model, qcl_launch_shape* shape) {
  if (!model || !shape) return fail(QCL_ERR_INVALID_ARG, "model or shape is NULL");
  shape->walkers_per_thread = model->shape_wpt;
  shape->blocks_per_sm = model->shape_bps;
  shape->walker_steps_per_s = model->shape_rate;
  shape->outputs_per_launch = model->shape_outs;
  shape->reserved = 0;
  return ok();
}

}  // extern "C"

namespace {
struct ProbeSizes {
  qcl_ensemble_desc ens;
  int64_t n_out;
  size_t ens_bytes, obs_bytes, total;
};
// Steps of the outputs-per-launch probe: enough output times for two launches
// of the largest candidate.
int64_t outs_probe_steps(int64_t n_steps, int32_t out_stride) {
  return std::max<int64_t>(n_steps, 2 * (int64_t)kChunkOut * out_stride);
}

ProbeSizes probe_sizes(const qcl_model* model, int64_t probe_walkers, int64_t n_steps, int32_t out_stride) {
  ProbeSizes p{};
  p.ens = qcl_ensemble_desc{probe_walkers, 0x5EEDull, 0, QCL_PREC_FP32_BULK, 0};
  p.n_out = outs_probe_steps(n_steps, out_stride) / out_stride + 1;
  p.ens_bytes = align256(EnsLayout::make(probe_walkers, model->ns, model->n, QCL_PREC_FP32_BULK).total);
  p.obs_bytes = ObsLayout::make(probe_walkers, model->ns, p.n_out,
                                tile_walkers(QCL_PREC_FP32_BULK, model->n, model->ns)).total;
  p.total = p.ens_bytes + p.obs_bytes;
  return p;
}
}  // namespace

extern "C" {

qcl_status qcl_autotune_bytes(const qcl_model* model, int64_t probe_walkers, int64_t n_steps, int32_t out_stride,
                              size_t* bytes) {
  if (!model || !bytes) return fail(QCL_ERR_INVALID_ARG, "model or bytes is NULL");
  if (probe_walkers < 1 || n_steps < 1 || out_stride < 1)
    return fail(QCL_ERR_INVALID_ARG, "probe_walkers, n_steps and out_stride must be >= 1");
  *bytes = probe_sizes(model, probe_walkers, n_steps, out_stride).total;
  return ok();
}

qcl_status qcl_autotune(qcl_model* model, int64_t probe_walkers, int64_t n_steps, double dt, int32_t out_stride,
                        void* scratch, size_t scratch_bytes, qcl_launch_shape* best, void* stream) {
  if (!model || !scratch || !best) return fail(QCL_ERR_INVALID_ARG, "model, scratch or best is NULL");
  if (probe_walkers < 1 || n_steps < 1 || out_stride < 1)
    return fail(QCL_ERR_INVALID_ARG, "probe_walkers, n_steps and out_stride must be >= 1");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(QCL_ERR_INVALID_ARG, "dt must be positive");
  const ProbeSizes ps = probe_sizes(model, probe_walkers, n_steps, out_stride);
  if (scratch_bytes < ps.total) return fail(QCL_ERR_OUT_OF_MEMORY, "scratch has %zu bytes, needs %zu", scratch_bytes, ps.total);
  qcl_status st = check_ens(model, &ps.ens);
  if (st) return st;
  const int ns = model->ns, n = model->n;
  std::vector<double> rho((size_t)ns * ns, 0.0), zero((size_t)n, 0.0);
  rho[0] = 1.0;
  const qcl_init_desc init{rho.data(), zero.data(), zero.data(), INFINITY, 1, 0};
  // candidates: walkers per thread, then blocks per SM up to the occupancy limit
  const bool dia = model->host.repr == QCL_REPR_DIABATIC;
  const bool two_state_reg = ns == 2 && (dia ? n <= 256 : (n <= 8 || (n > 32 && n <= 256)));
  const int wmax = (ns == 2 && max_wpt(n) == 2) ? 2 : 1;
  const int keep_wpt = model->shape_wpt, keep_bps = model->shape_bps, keep_outs = model->shape_outs;
  const double keep_rate = model->shape_rate;
  cudaStream_t s = (cudaStream_t)stream;
  char* ens_buf = (char*)scratch;
  char* obs_buf = ens_buf + ps.ens_bytes;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = -1.0f;
  int best_wpt = 1, best_bps = 0, best_outs = 0;
  // one warm-up run and one timed run of the probe with the model's current shape
  auto time_probe = [&](int64_t steps, float* ms) -> qcl_status {
    qcl_status r = QCL_OK;
    for (int rep = 0; rep < 2 && !r; ++rep) {
      r = qcl_sample_initial(model, &ps.ens, &init, ens_buf, ps.ens_bytes, stream);
      if (!r) cudaEventRecord(e0, s);
      if (!r) r = qcl_propagate(model, &ps.ens, ens_buf, ps.ens_bytes, 0, steps, dt, out_stride, obs_buf,
                                ps.obs_bytes, ps.n_out, stream);
      if (!r) cudaEventRecord(e1, s);
      if (!r && cudaEventSynchronize(e1) != cudaSuccess) r = fail(QCL_ERR_CUDA, "autotune: event wait failed");
      if (!r) cudaEventElapsedTime(ms, e0, e1);
    }
    return r;
  };
  model->shape_outs = 0;
  for (int wpt = 1; wpt <= wmax; ++wpt) {
    int limit = two_state_reg ? bulk2_blocks_per_sm(n, bulk_kind(model->host), model->host.repr, wpt) : 4;
    if (limit < 1) limit = 1;
    for (int bps = 1; bps <= limit; ++bps) {
      model->shape_wpt = wpt;
      model->shape_bps = bps;
      float ms = 0.0f;
      st = time_probe(n_steps, &ms);
      if (st) break;
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best_wpt = wpt;
        best_bps = bps;
      }
    }
    if (st) break;
  }
  // output times per launch, with the fastest walkers per thread and blocks per SM
  const int64_t steps2 = outs_probe_steps(n_steps, out_stride);
  float best2 = -1.0f;
  for (int outs : {8, 16, 32}) {
    if (st) break;
    model->shape_wpt = best_wpt;
    model->shape_bps = best_bps;
    model->shape_outs = outs;
    float ms = 0.0f;
    st = time_probe(steps2, &ms);
    if (!st && (best2 < 0.0f || ms < best2)) {
      best2 = ms;
      best_outs = outs;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    model->shape_wpt = keep_wpt;
    model->shape_bps = keep_bps;
    model->shape_outs = keep_outs;
    model->shape_rate = keep_rate;
    return st;
  }
  model->shape_wpt = best_wpt;
  model->shape_bps = best_bps;
  model->shape_outs = best_outs;
  model->shape_rate = best2 > 0.0f ? (double)probe_walkers * (double)steps2 / (best2 * 1e-3) : 0.0;
  best->walkers_per_thread = best_wpt;
  best->blocks_per_sm = best_bps;
  best->outputs_per_launch = best_outs;
  best->reserved = 0;
  best->walker_steps_per_s = model->shape_rate;
  return ok();
}

// ------------------------------------------------------------- spawning --
}  // extern "C"

namespace {
qcl_status check_spawn(const qcl_model* m, const qcl_ensemble_desc* e, int64_t capacity) {
  qcl_status st = check_ens(m, e);
  if (st) return st;
  if (e->n_traj >= ((int64_t)1 << 31)) return fail(QCL_ERR_INVALID_ARG, "n_traj must be below 2^31 for a spawning ensemble");
  if (capacity < e->n_traj || capacity > ((int64_t)1 << 36))
    return fail(QCL_ERR_INVALID_ARG, "capacity %lld outside [n_traj, 2^36]", (long long)capacity);
  return QCL_OK;
}
}  // namespace

extern "C" {

qcl_status qcl_spawn_bytes(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t capacity, size_t* bytes) {
  if (!bytes) return fail(QCL_ERR_INVALID_ARG, "bytes is NULL");
  qcl_status st = check_spawn(model, ens, capacity);
  if (st) return st;
  *bytes = SpawnLayout::make(capacity, model->n, ens->n_traj, ens->precision, model->ns).total;
  return ok();
}

qcl_status qcl_spawn_layout(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t capacity, int32_t set,
                            size_t offsets[12]) {
  if (!offsets) return fail(QCL_ERR_INVALID_ARG, "offsets is NULL");
  qcl_status st = check_spawn(model, ens, capacity);
  if (st) return st;
  if (set != 0 && set != 1) return fail(QCL_ERR_INVALID_ARG, "set must be 0 or 1");
  const SpawnLayout L = SpawnLayout::make(capacity, model->n, ens->n_traj, ens->precision, model->ns);
  const size_t b = L.set_off[set];
  const bool f32 = ens->precision == QCL_PREC_FP32_BULK;
  offsets[0] = b + L.R;
  offsets[1] = b + L.P;
  offsets[2] = b + L.m;
  offsets[3] = b + L.phi;
  offsets[4] = b + L.ab;
  offsets[5] = b + L.id;
  offsets[6] = b + L.fam;
  offsets[7] = L.total;
  offsets[8] = f32 ? b + L.mlo : 0;
  offsets[9] = f32 ? b + L.mexp : 0;
  offsets[10] = f32 ? b + L.philo : 0;
  offsets[11] = model->ns > 2 ? b + L.U : 0;
  return ok();
}

qcl_status qcl_spawn_sample(const qcl_model* model, const qcl_ensemble_desc* ens, const qcl_init_desc* init,
                            int64_t capacity, void* buf, size_t bytes, void* stream) {
  qcl_status st = check_spawn(model, ens, capacity);
  if (st) return st;
  if (!buf) return fail(QCL_ERR_INVALID_ARG, "buf is NULL");
  if (((uintptr_t)buf & 255) != 0) return fail(QCL_ERR_INVALID_ARG, "buf must be 256-byte aligned");
  const size_t need = SpawnLayout::make(capacity, model->n, ens->n_traj, ens->precision, model->ns).total;
  if (bytes < need) return fail(QCL_ERR_OUT_OF_MEMORY, "buf has %zu bytes, needs %zu", bytes, need);
  SampleParams* sp = nullptr;
  st = prepare_sample(model, ens, init, &sp);
  if (st) return st;
  if (model->ns > 2 && ens->precision == QCL_PREC_FP32_BULK) {
    SampleN32* s32 = new (std::nothrow) SampleN32();
    if (!s32) {
      delete sp;
      return fail(QCL_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    make_sampleN32(model, *sp, *s32);
    launch_spawnN_sample32(model->ns, *s32, capacity, buf, (cudaStream_t)stream);
    delete s32;
  } else if (model->ns > 2)
    launch_spawnN_sample(model->dev, model->ns, *sp, capacity, buf, (cudaStream_t)stream);
  else if (ens->precision == QCL_PREC_FP32_BULK)
    launch_spawn_sample32(model->host, *sp, capacity, buf, (cudaStream_t)stream);
  else
    launch_spawn_sample(model->dev, *sp, capacity, buf, (cudaStream_t)stream);
  delete sp;
  st = check_launch("spawn sample");
  return st ? st : ok();
}

qcl_status qcl_spawn_propagate(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t capacity, void* buf,
                               size_t bytes, int64_t step0, int64_t n_steps, double dt, int32_t out_stride,
                               void* obs_buf, size_t obs_bytes, int64_t n_out, void* stream) {
  qcl_status st = check_spawn(model, ens, capacity);
  if (st) return st;
  if (!buf || !obs_buf) return fail(QCL_ERR_INVALID_ARG, "buf or obs_buf is NULL");
  if (((uintptr_t)buf & 255) != 0 || ((uintptr_t)obs_buf & 255) != 0) return fail(QCL_ERR_INVALID_ARG, "buffers must be 256-byte aligned");
  if (step0 < 0 || n_steps < 0) return fail(QCL_ERR_INVALID_ARG, "step0 and n_steps must be >= 0");
  if (step0 + n_steps >= ((int64_t)1 << 32)) return fail(QCL_ERR_INVALID_ARG, "absolute step beyond 2^32");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(QCL_ERR_INVALID_ARG, "dt must be positive");
  if (out_stride < 1) return fail(QCL_ERR_INVALID_ARG, "out_stride must be >= 1");
  if (n_out < 1) return fail(QCL_ERR_INVALID_ARG, "n_out must be >= 1");
  const int64_t k_last = (step0 + n_steps) / out_stride;
  if (k_last >= n_out) return fail(QCL_ERR_INVALID_ARG, "output row %lld beyond n_out = %lld", (long long)k_last, (long long)n_out);
  const SpawnLayout SL = SpawnLayout::make(capacity, model->n, ens->n_traj, ens->precision, model->ns);
  if (bytes < SL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "buf has %zu bytes, needs %zu", bytes, SL.total);
  // tiles of families as the ensemble's own tiles: 256 (two states, <= 32 modes in
  // FP32), 128 for FP32 N_s-state models
  const ObsLayout OL = ObsLayout::make(ens->n_traj, model->ns, n_out, tile_walkers(ens->precision, model->n, model->ns));
  if (obs_bytes < OL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "obs_buf has %zu bytes, needs %zu", obs_bytes, OL.total);
  cudaStream_t s = (cudaStream_t)stream;
  char* ob = (char*)obs_buf;
  double* rows = (double*)(ob + OL.off_rows);
  double* part = (double*)(ob + OL.off_part);
  double* fold = (double*)(ob + OL.off_fold);
  const int q2 = OL.q2;
  const int64_t n0 = ens->n_traj;
  const bool f32 = ens->precision == QCL_PREC_FP32_BULK;
  const bool f32n = f32 && model->ns > 2;
  Coef2* cf = nullptr;
  CoefN* cn = nullptr;
  BulkParams bp{};
  if (f32) {
    cf = new (std::nothrow) Coef2();
    if (f32n) cn = new (std::nothrow) CoefN();
    if (!cf || (f32n && !cn)) {
      delete cf;
      delete cn;
      return fail(QCL_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    fill_coef2(model, dt, cf);
    if (f32n) fill_coefN(model, dt, *cn);
    bp.n_traj = n0;
    bp.seed = ens->seed;
    bp.step0 = step0;
    bp.stride = out_stride;
    bp.n = model->n;
    bulk_model_scalars(bp, model->host, dt);
  }
  auto observe = [&](double* row, int64_t step) {
    if (f32n)
      launch_spawnN_observe32(model->ns, bp, *cn, buf, capacity, n0, (int)(step & 1), part, s);
    else if (f32)
      launch_spawn_observe32(bp, *cf, buf, capacity, n0, (int)(step & 1), part, s);
    else if (model->ns > 2)
      launch_spawnN_observe(model->dev, model->ns, buf, capacity, model->n, n0, (int)(step & 1), part, s);
    else
      launch_spawn_observe(model->dev, buf, capacity, model->n, n0, (int)(step & 1), part, s);
    launch_fold(part, row, fold, OL.n_tiles, q2, 1, s);
  };
  if (step0 == 0) observe(rows, 0);
  for (int64_t t = step0; t < step0 + n_steps; ++t) {
    {
      TimedLaunch tl(1, s);
      if (f32n)
        launch_spawnN_step32(model->ns, bp, *cn, buf, capacity, n0, step0, t, s);
      else if (f32)
        launch_spawn_step32(bp, *cf, buf, capacity, n0, step0, t, s);
      else if (model->ns > 2)
        launch_spawnN_step(model->dev, model->ns, buf, capacity, model->n, n0, step0, t, dt, ens->seed, s);
      else
        launch_spawn_step(model->dev, model->host.repr, buf, capacity, model->n, n0, step0, t, dt, ens->seed, s);
    }
    if ((t + 1) % out_stride == 0) observe(rows + (size_t)((t + 1) / out_stride) * q2, t + 1);
  }
  delete cf;
  delete cn;
  st = check_launch("spawn step");
  if (st) return st;
  launch_header_finish(buf, step0, step0 + n_steps, s);
  st = check_launch("header");
  return st ? st : ok();
}

qcl_status qcl_spawn_live(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t capacity, const void* buf,
                          int64_t* n_live, void* stream) {
  qcl_status st = check_spawn(model, ens, capacity);
  if (st) return st;
  if (!buf || !n_live) return fail(QCL_ERR_INVALID_ARG, "buf or n_live is NULL");
  struct {
    EnsHeader h;
    SpawnHeader s;
  } hs;
  static_assert(offsetof(decltype(hs), s) == kSpawnHeaderOff, "spawn header offset");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(&hs, buf, sizeof(hs), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hs.h.magic != kEnsMagic) return fail(QCL_ERR_INVALID_ARG, "buf holds no sampled ensemble");
  *n_live = hs.s.n_live[hs.h.step & 1];
  return ok();
}

qcl_status qcl_shard_tile_walkers(const qcl_model* model, int32_t precision, int64_t* walkers) {
  if (!model || !walkers) return fail(QCL_ERR_INVALID_ARG, "NULL argument");
  if (precision != QCL_PREC_FP64 && precision != QCL_PREC_FP32_BULK) return fail(QCL_ERR_INVALID_ARG, "unknown precision");
  *walkers = tile_walkers(precision, model->n, model->ns);
  return ok();
}

qcl_status qcl_shard_chunk_walkers(const qcl_model* model, int32_t precision, int64_t* walkers) {
  if (!model || !walkers) return fail(QCL_ERR_INVALID_ARG, "NULL argument");
  if (precision != QCL_PREC_FP64 && precision != QCL_PREC_FP32_BULK) return fail(QCL_ERR_INVALID_ARG, "unknown precision");
  *walkers = (int64_t)kFoldBlock * tile_walkers(precision, model->n, model->ns);
  return ok();
}

qcl_status qcl_combine_shards(const double* shard_sums, int32_t n_shards, int64_t n_elems, double* out) {
  if (!shard_sums || !out || n_shards < 1 || n_elems < 0) return fail(QCL_ERR_INVALID_ARG, "bad arguments");
  int32_t p2 = 1;
  while (p2 < n_shards) p2 <<= 1;
  std::vector<double> level((size_t)p2);
  for (int64_t i = 0; i < n_elems; ++i) {
    for (int32_t s = 0; s < p2; ++s) level[s] = (s < n_shards) ? shard_sums[(size_t)s * n_elems + i] : 0.0;
    for (int32_t w = p2; w > 1; w >>= 1)
      for (int32_t s = 0; s < w / 2; ++s) level[s] = level[2 * s] + level[2 * s + 1];
    out[i] = level[0];
  }
  return ok();
}

}  // extern "C"
