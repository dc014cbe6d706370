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
}  // namespace qcl
