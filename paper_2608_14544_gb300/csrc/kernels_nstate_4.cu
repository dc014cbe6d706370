// kernels_nstate_4.cu -- the FP32-bulk and FP64-observation N_s-state kernels
// instantiated for N_s = 4.
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample32_4(const SampleN32& sp, void* buf, cudaStream_t st) {
  NStateOps<4>::sample32(sp, buf, st);
}
void nstate_observe64_4(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                         cudaStream_t st) {
  NStateOps<4>::observe64(dm, buf, nt, n, part, st);
}
int nstate_bulk_4(const BulkParams& bp, const CoefN& cf, void* buf, double* part, int grid_cap,
                  int wpt, cudaStream_t st) {
  return NStateOps<4>::bulk(bp, cf, buf, part, grid_cap, wpt, st);
}
void nstate_spawn_sample32_4(const SampleN32& sp, int64_t cap, void* buf, cudaStream_t st) {
  NStateOps<4>::spawn_sample32(sp, cap, buf, st);
}
int nstate_spawn_step32_4(const BulkParams& bp, const CoefN& cf, void* buf, int64_t cap,
                          int64_t n0, int64_t step0, int64_t step, cudaStream_t st) {
  return NStateOps<4>::spawn_step32(bp, cf, buf, cap, n0, step0, step, st);
}
void nstate_spawn_observe32_4(const BulkParams& bp, const CoefN& cf, const void* buf, int64_t cap,
                              int64_t n0, int set, double* part, cudaStream_t st) {
  NStateOps<4>::spawn_observe32(bp, cf, buf, cap, n0, set, part, st);
}
}  // namespace qcl
