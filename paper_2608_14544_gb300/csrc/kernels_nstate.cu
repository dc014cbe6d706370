// kernels_nstate.cu -- dispatch of the N_s-state launchers (N_s = 3..8) to
// their per-N_s translation units (kernels_nstate_*.cu, kernels_nstate64_*.cu).
#include "kernels.h"

namespace qcl {

#define QCL_NS_DECL(k)                                                                        \
  void nstate_sample64_##k(const DevModel*, const SampleParams&, void*, cudaStream_t);        \
  void nstate_sample32_##k(const SampleN32&, void*, cudaStream_t);                           \
  void nstate_step64_##k(const DevModel*, int, void*, int64_t, int, int64_t, int64_t, double, \
                         uint64_t, uint64_t, cudaStream_t);                                   \
  void nstate_observe64_##k(const DevModel*, const void*, int64_t, int, double*, cudaStream_t); \
  int nstate_bulk_##k(const BulkParams&, const CoefN&, void*, double*, int, int, cudaStream_t); \
  void nstate_spawn_sample64_##k(const DevModel*, const SampleParams&, int64_t, void*,        \
                                 cudaStream_t);                                               \
  void nstate_spawn_step64_##k(const DevModel*, void*, int64_t, int, int64_t, int64_t, int64_t, \
                               double, uint64_t, cudaStream_t);                               \
  void nstate_spawn_observe64_##k(const DevModel*, const void*, int64_t, int, int64_t, int,   \
                                  double*, cudaStream_t);                                     \
  void nstate_spawn_sample32_##k(const SampleN32&, int64_t, void*, cudaStream_t);            \
  int nstate_spawn_step32_##k(const BulkParams&, const CoefN&, void*, int64_t, int64_t,       \
                              int64_t, int64_t, cudaStream_t);                                \
  void nstate_spawn_observe32_##k(const BulkParams&, const CoefN&, const void*, int64_t,      \
                                  int64_t, int, double*, cudaStream_t);
QCL_NS_DECL(3)
QCL_NS_DECL(4)
QCL_NS_DECL(5)
QCL_NS_DECL(6)
QCL_NS_DECL(7)
QCL_NS_DECL(8)

#define QCL_NS_SWITCH(ns, F, ...)          \
  switch (ns) {                            \
    case 3: F##_3(__VA_ARGS__); break;     \
    case 4: F##_4(__VA_ARGS__); break;     \
    case 5: F##_5(__VA_ARGS__); break;     \
    case 6: F##_6(__VA_ARGS__); break;     \
    case 7: F##_7(__VA_ARGS__); break;     \
    case 8: F##_8(__VA_ARGS__); break;     \
    default: break;                        \
  }

void launch_sampleN(const DevModel* dm, const SampleParams& sp, const SampleN32* s32, void* buf,
                    int precision, cudaStream_t st) {
  if (precision == QCL_PREC_FP64) {
    QCL_NS_SWITCH(sp.ns, nstate_sample64, dm, sp, buf, st);
  } else {
    QCL_NS_SWITCH(sp.ns, nstate_sample32, *s32, buf, st);
  }
  launches_add(1);
}

void launch_stepN_f64(const DevModel* dm, int repr, int ns, void* buf, int64_t nt, int n,
                      int64_t step0, int64_t step, double dt, uint64_t seed, uint64_t traj_off,
                      cudaStream_t st) {
  QCL_NS_SWITCH(ns, nstate_step64, dm, repr, buf, nt, n, step0, step, dt, seed, traj_off, st);
  launches_add(1);
}

void launch_observeN_f64(const DevModel* dm, int ns, const void* buf, int64_t nt, int n,
                         double* part, cudaStream_t st) {
  QCL_NS_SWITCH(ns, nstate_observe64, dm, buf, nt, n, part, st);
  launches_add(1);
}

void launch_spawnN_sample(const DevModel* dm, int ns, const SampleParams& sp, int64_t capacity,
                          void* buf, cudaStream_t st) {
  QCL_NS_SWITCH(ns, nstate_spawn_sample64, dm, sp, capacity, buf, st);
}

void launch_spawnN_step(const DevModel* dm, int ns, void* buf, int64_t capacity, int n, int64_t n0,
                        int64_t step0, int64_t step, double dt, uint64_t seed, cudaStream_t st) {
  QCL_NS_SWITCH(ns, nstate_spawn_step64, dm, buf, capacity, n, n0, step0, step, dt, seed, st);
}

void launch_spawnN_observe(const DevModel* dm, int ns, const void* buf, int64_t capacity, int n,
                           int64_t n0, int set, double* part, cudaStream_t st) {
  QCL_NS_SWITCH(ns, nstate_spawn_observe64, dm, buf, capacity, n, n0, set, part, st);
}

void launch_spawnN_sample32(int ns, const SampleN32& sp, int64_t capacity, void* buf,
                            cudaStream_t st) {
  QCL_NS_SWITCH(ns, nstate_spawn_sample32, sp, capacity, buf, st);
}

int launch_spawnN_step32(int ns, const BulkParams& bp, const CoefN& cf, void* buf,
                         int64_t capacity, int64_t n0, int64_t step0, int64_t step,
                         cudaStream_t st) {
  switch (ns) {
    case 3: return nstate_spawn_step32_3(bp, cf, buf, capacity, n0, step0, step, st);
    case 4: return nstate_spawn_step32_4(bp, cf, buf, capacity, n0, step0, step, st);
    case 5: return nstate_spawn_step32_5(bp, cf, buf, capacity, n0, step0, step, st);
    case 6: return nstate_spawn_step32_6(bp, cf, buf, capacity, n0, step0, step, st);
    case 7: return nstate_spawn_step32_7(bp, cf, buf, capacity, n0, step0, step, st);
    case 8: return nstate_spawn_step32_8(bp, cf, buf, capacity, n0, step0, step, st);
    default: return 0;
  }
}

void launch_spawnN_observe32(int ns, const BulkParams& bp, const CoefN& cf, const void* buf,
                             int64_t capacity, int64_t n0, int set, double* part,
                             cudaStream_t st) {
  QCL_NS_SWITCH(ns, nstate_spawn_observe32, bp, cf, buf, capacity, n0, set, part, st);
}

int launch_bulkN(int ns, const BulkParams& bp, const CoefN& cf, void* buf, double* part,
                 const LaunchShape& ls, cudaStream_t st) {
  // blocks per SM become a cap on the grid (one walker per thread here)
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  }
  int grid_cap = ls.grid_cap;
  if (ls.blocks_per_sm > 0 && (grid_cap == 0 || ls.blocks_per_sm * n_sm < grid_cap))
    grid_cap = ls.blocks_per_sm * n_sm;
  int g = 0;
  switch (ns) {
    case 3: g = nstate_bulk_3(bp, cf, buf, part, grid_cap, ls.wpt, st); break;
    case 4: g = nstate_bulk_4(bp, cf, buf, part, grid_cap, ls.wpt, st); break;
    case 5: g = nstate_bulk_5(bp, cf, buf, part, grid_cap, ls.wpt, st); break;
    case 6: g = nstate_bulk_6(bp, cf, buf, part, grid_cap, ls.wpt, st); break;
    case 7: g = nstate_bulk_7(bp, cf, buf, part, grid_cap, ls.wpt, st); break;
    case 8: g = nstate_bulk_8(bp, cf, buf, part, grid_cap, ls.wpt, st); break;
    default: break;
  }
  if (g) launches_add(1);
  return g;
}

}  // namespace qcl
