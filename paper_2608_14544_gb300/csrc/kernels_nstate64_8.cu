// kernels_nstate64_8.cu -- the FP64 N_s-state sampling and step kernels for
// N_s = 8 (compiled without multiply-add contraction).
#include "nstate_kernels.cuh"

namespace qcl {
void nstate_sample64_8(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st) {
  NStateOps<8>::sample64(dm, sp, buf, st);
}
void nstate_step64_8(const DevModel* dm, int repr, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st) {
  NStateOps<8>::step64(dm, repr, buf, nt, n, step0, step, dt, seed, traj_off, st);
}
void nstate_spawn_sample64_8(const DevModel* dm, const SampleParams& sp, int64_t cap, void* buf,
                             cudaStream_t st) {
  NStateOps<8>::spawn_sample64(dm, sp, cap, buf, st);
}
void nstate_spawn_step64_8(const DevModel* dm, void* buf, int64_t cap, int n, int64_t n0,
                           int64_t step0, int64_t step, double dt, uint64_t seed, cudaStream_t st) {
  NStateOps<8>::spawn_step64(dm, buf, cap, n, n0, step0, step, dt, seed, st);
}
void nstate_spawn_observe64_8(const DevModel* dm, const void* buf, int64_t cap, int n, int64_t n0,
                              int set, double* part, cudaStream_t st) {
  NStateOps<8>::spawn_observe64(dm, buf, cap, n, n0, set, part, st);
}
}  // namespace qcl
