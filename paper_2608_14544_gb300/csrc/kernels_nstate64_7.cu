// kernels_nstate64_7.cu -- the FP64 N_s-state sampling and step kernels for
// N_s = 7 (compiled without multiply-add contraction).
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample64_7(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st) {
  NStateOps<7>::sample64(dm, sp, buf, st);
}
void nstate_step64_7(const DevModel* dm, int repr, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st) {
  NStateOps<7>::step64(dm, repr, buf, nt, n, step0, step, dt, seed, traj_off, st);
}
}  // namespace qcl
