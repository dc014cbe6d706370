// kernels_nstate_8.cu -- the FP32-bulk and FP64-observation N_s-state kernels
// instantiated for N_s = 8.
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample32_8(const SampleN32& sp, void* buf, cudaStream_t st) {
  NStateOps<8>::sample32(sp, buf, st);
}
void nstate_observe64_8(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                         cudaStream_t st) {
  NStateOps<8>::observe64(dm, buf, nt, n, part, st);
}
int nstate_bulk_8(const BulkParams& bp, const CoefN& cf, void* buf, double* part, int grid_cap,
                  int wpt, cudaStream_t st) {
  return NStateOps<8>::bulk(bp, cf, buf, part, grid_cap, wpt, st);
}
void nstate_spawn_sample32_8(const SampleN32& sp, int64_t cap, void* buf, cudaStream_t st) {
  NStateOps<8>::spawn_sample32(sp, cap, buf, st);
}
int nstate_spawn_step32_8(const BulkParams& bp, const CoefN& cf, void* buf, int64_t cap,
                          int64_t n0, int64_t step0, int64_t step, cudaStream_t st) {
  return NStateOps<8>::spawn_step32(bp, cf, buf, cap, n0, step0, step, st);
}
void nstate_spawn_observe32_8(const BulkParams& bp, const CoefN& cf, const void* buf, int64_t cap,
                              int64_t n0, int set, double* part, cudaStream_t st) {
  NStateOps<8>::spawn_observe32(bp, cf, buf, cap, n0, set, part, st);
}
}  // namespace qcl
