// kernels_nstate_3.cu -- the FP32-bulk and FP64-observation N_s-state kernels
// instantiated for N_s = 3.
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample32_3(const SampleN32& sp, void* buf, cudaStream_t st) {
  NStateOps<3>::sample32(sp, buf, st);
}
void nstate_observe64_3(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                         cudaStream_t st) {
  NStateOps<3>::observe64(dm, buf, nt, n, part, st);
}
int nstate_bulk_3(const BulkParams& bp, const CoefN& cf, void* buf, double* part, int grid_cap,
                  int wpt, cudaStream_t st) {
  return NStateOps<3>::bulk(bp, cf, buf, part, grid_cap, wpt, st);
}
}  // namespace qcl
