// kernels_nstate_7.cu -- the FP32-bulk and FP64-observation N_s-state kernels
// instantiated for N_s = 7.
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample32_7(const SampleN32& sp, void* buf, cudaStream_t st) {
  NStateOps<7>::sample32(sp, buf, st);
}
void nstate_observe64_7(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                         cudaStream_t st) {
  NStateOps<7>::observe64(dm, buf, nt, n, part, st);
}
int nstate_bulk_7(const BulkParams& bp, const CoefN& cf, void* buf, double* part, int grid_cap,
                  int wpt, cudaStream_t st) {
  return NStateOps<7>::bulk(bp, cf, buf, part, grid_cap, wpt, st);
}
}  // namespace qcl
