// noalloc.cu -- qcl_propagate_noalloc: the FP32-bulk propagation for callers
// that cannot allocate device memory at the time they propagate (for example a
// service that sized all device memory at start-up and must not call
// cudaMalloc/cudaFree afterwards, since those calls can block on the whole
// device, or code that is handed fixed buffers by a host application).  The
// only scratch memory the persistent kernel needs -- the per-tile FP64 partial
// sums of each output time and the fold scratch -- lives in a file-scope static
// device array instead of the caller's observation buffer.  Nothing here
// allocates: no cudaMalloc, no cudaFree, no host heap.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "kernels.h"
#include "model.h"

namespace {

constexpr size_t kScratchBytes = QCL_NOALLOC_SCRATCH_BYTES;
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

qcl_status fail(qcl_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return qcl::set_error(st, buf);
}

// The array's name is only a host-side stand-in; its device address is looked
// up once per device (with that device current) and cached.  The cache
// belongs to the device's primary context: after cudaDeviceReset, or under a
// context the caller created with the driver API, the module is loaded anew
// and the cached address would be stale (both are documented preconditions).
qcl_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(QCL_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(QCL_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(QCL_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return QCL_OK;
}

}  // namespace

extern "C" qcl_status qcl_propagate_noalloc(const qcl_model* model, const qcl_ensemble_desc* ens,
                                            void* ens_buf, size_t ens_bytes, int64_t step0,
                                            int64_t n_steps, double dt, int32_t out_stride,
                                            double* rows, size_t rows_bytes, int64_t n_out,
                                            void* stream) {
  using namespace qcl;
  // the checks of qcl_propagate first, in its order, so that the same bad
  // input gets the same code from both calls
  qcl_status st = check_ensemble(model, ens);
  if (st) return st;
  if (!ens_buf || !rows) return fail(QCL_ERR_INVALID_ARG, "ens_buf or rows is NULL");
  if (((uintptr_t)ens_buf & 255) != 0 || ((uintptr_t)rows & 7) != 0)
    return fail(QCL_ERR_INVALID_ARG, "ens_buf must be 256-byte aligned and rows 8-byte aligned");
  if (step0 < 0 || n_steps < 0) return fail(QCL_ERR_INVALID_ARG, "step0 and n_steps must be >= 0");
  if (step0 + n_steps >= ((int64_t)1 << 34)) return fail(QCL_ERR_INVALID_ARG, "absolute step beyond 2^34");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(QCL_ERR_INVALID_ARG, "dt must be positive");
  if (out_stride < 1 || n_out < 1) return fail(QCL_ERR_INVALID_ARG, "out_stride and n_out must be >= 1");
  if ((step0 + n_steps) / out_stride >= n_out) return fail(QCL_ERR_INVALID_ARG, "last output row beyond n_out");
  const int q2 = 8 * model->ns * model->ns;
  const EnsLayout EL = EnsLayout::make(ens->n_traj, model->ns, model->n, ens->precision);
  if (ens_bytes < EL.total) return fail(QCL_ERR_OUT_OF_MEMORY, "ens_buf has %zu bytes, needs %zu", ens_bytes, EL.total);
  if (rows_bytes < sizeof(double) * (size_t)n_out * q2)
    return fail(QCL_ERR_OUT_OF_MEMORY, "rows has %zu bytes, needs %zu", rows_bytes, sizeof(double) * (size_t)n_out * q2);
  // what only this call rejects: other precisions, more states, and walker
  // counts whose scratch does not fit the static array
  if (ens->precision != QCL_PREC_FP32_BULK)
    return fail(QCL_ERR_UNSUPPORTED, "qcl_propagate_noalloc runs FP32-bulk ensembles only");
  if (model->ns != 2)
    return fail(QCL_ERR_UNSUPPORTED, "qcl_propagate_noalloc supports two-state models");
  // static-scratch capacity: per output time n_tiles x q2 partials plus fold scratch
  const int tile = tile_walkers(ens->precision, model->n);
  const int64_t n_tiles = (ens->n_traj + tile - 1) / tile;
  const int64_t nb1 = (n_tiles + kFoldBlock - 1) / kFoldBlock;
  const int64_t per_slot = n_tiles * q2 + (nb1 + (nb1 + kFoldBlock - 1) / kFoldBlock + 1) * q2;
  int64_t slots = (int64_t)kScratchDoubles / per_slot;
  if (slots < 1)
    return fail(QCL_ERR_UNSUPPORTED,
                "n_traj = %lld needs %lld bytes of scratch per output time; the static scratch holds "
                "%zu bytes (at most about %lld walkers for this model's %d-walker tiles)",
                (long long)ens->n_traj, (long long)(per_slot * 8), kScratchBytes,
                (long long)((int64_t)kScratchDoubles / (q2 + 1) * tile * 99 / 100), tile);
  const int outs = model->shape_outs > 0 ? model->shape_outs : kChunkOut;
  if (slots > outs) slots = outs;

  double* scratch = nullptr;
  st = scratch_address(&scratch);
  if (st) return st;
  double* part = scratch;
  double* fold = scratch + (size_t)slots * n_tiles * q2;
  cudaStream_t s = (cudaStream_t)stream;

  Coef2 cf;  // on the stack: no heap allocation
  const DevModel& h = model->host;
  for (int j = 0; j < kMaxN; ++j) {
    const bool on = j < model->n;
    cf.hk[j] = on ? (float)(0.5 * dt * h.k[j]) : 0.0f;
    cf.hs[j] = on ? (float)(0.5 * dt * h.s[j]) : 0.0f;
    cf.dtm[j] = on ? (float)(dt / h.mass[j]) : 0.0f;
    cf.a[j] = on ? (float)h.a[j] : 0.0f;
    cf.b[j] = on ? (float)h.b[j] : 0.0f;
    cf.am[j] = on ? (float)(h.a[j] / h.mass[j]) : 0.0f;
    cf.bm[j] = on ? (float)(h.b[j] / h.mass[j]) : 0.0f;
  }
  BulkParams bp{};
  bp.n_traj = ens->n_traj;
  bp.n_tiles = n_tiles;
  bp.traj_offset = ens->traj_id_offset;
  bp.seed = ens->seed;
  bp.step0 = step0;
  bp.stride = out_stride;
  bp.n = model->n;
  bulk_model_scalars(bp, h, dt);

  // chunks of at most `slots` output times (the reduction tree does not depend
  // on the chunking, so the rows equal those of qcl_propagate bit for bit)
  const int64_t end = step0 + n_steps;
  int64_t cs = step0;
  bool first = (step0 == 0);
  while (first || cs < end) {
    int n_slots = first ? 1 : 0;
    const int64_t next_out = (cs / out_stride + 1) * out_stride;
    const int64_t room = slots - n_slots;
    int64_t ce;
    if (room <= 0) {
      ce = cs;
    } else if (next_out + (room - 1) * out_stride <= end) {
      ce = next_out + (room - 1) * out_stride;
      n_slots += (int)room;
    } else {
      ce = end;
      if (end >= next_out) n_slots += (int)((end - next_out) / out_stride + 1);
    }
    if (ce - cs > ((int64_t)1 << 30)) {
      ce = cs + ((int64_t)1 << 30);
      const int64_t kl = ce / out_stride, kn = next_out / out_stride;
      n_slots = (first ? 1 : 0) + (int)(kl >= kn ? kl - kn + 1 : 0);
    }
    const int64_t k_first = first ? 0 : next_out / out_stride;
    bp.cs = cs;
    bp.ce = ce;
    bp.k_first = k_first;
    bp.obs_first = first ? 1 : 0;
    bp.len = (int32_t)(ce - cs);
    bp.to_out0 = (int32_t)(out_stride - (cs % out_stride));
    bp.blk0 = (uint32_t)(cs >> 2);
    bp.widx0 = (int32_t)(cs & 3);
    LaunchShape ls;
    ls.wpt = model->shape_wpt;
    ls.blocks_per_sm = model->shape_bps;
    ls.grid_cap = (int)option_grid_cap();
    if (launch_bulk2(bp, cf, ens_buf, part, ls, s) == 0)
      return fail(QCL_ERR_UNSUPPORTED, "no FP32-bulk kernel for n_modes = %d", model->n);
    if (n_slots > 0) launch_fold(part, rows + (size_t)k_first * q2, fold, n_tiles, q2, n_slots, s);
    first = false;
    cs = ce;
  }
  launch_header_finish(ens_buf, step0, step0 + n_steps, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCL_ERR_CUDA, "qcl_propagate_noalloc launch failed: %s", cudaGetErrorString(e));
  return qcl::set_error(QCL_OK, "");
}
