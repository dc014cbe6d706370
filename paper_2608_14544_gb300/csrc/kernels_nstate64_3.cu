// kernels_nstate64_3.cu -- the FP64 N_s-state sampling and step kernels for
// N_s = 3 (compiled without multiply-add contraction).
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample64_3(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st) {
  NStateOps<3>::sample64(dm, sp, buf, st);
}
void nstate_step64_3(const DevModel* dm, int repr, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st) {
  NStateOps<3>::step64(dm, repr, buf, nt, n, step0, step, dt, seed, traj_off, st);
}
}  // namespace qcl
