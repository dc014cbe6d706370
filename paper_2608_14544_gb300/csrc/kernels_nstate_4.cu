// kernels_nstate_4.cu -- the N_s-state kernels instantiated for N_s = 4.
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample_4(const DevModel* dm, const SampleParams& sp, void* buf, int precision,
                     cudaStream_t st) {
  NStateOps<4>::sample(dm, sp, buf, precision, st);
}
void nstate_step64_4(const DevModel* dm, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st) {
  NStateOps<4>::step64(dm, buf, nt, n, step0, step, dt, seed, traj_off, st);
}
void nstate_observe64_4(const void* buf, int64_t nt, int n, double* part, cudaStream_t st) {
  NStateOps<4>::observe64(buf, nt, n, part, st);
}
int nstate_bulk_4(const BulkParams& bp, const CoefN& cf, void* buf, double* part, int grid_cap,
                  cudaStream_t st) {
  return NStateOps<4>::bulk(bp, cf, buf, part, grid_cap, st);
}
}  // namespace qcl
