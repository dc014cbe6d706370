// kernels_dia.cu -- FP32-bulk persistent kernel of the diabatic representation
// (two states, one thread per walker, up to 32 modes): the same tile body as
// the adiabatic kernel with the diagonal mean force, the diabatic phase and
// the quarter-turn transitions (bulk2.cuh, DIA = true).
#include "bulk2.cuh"

namespace qcl {

template <int NPL, int KIND>
__global__ void __launch_bounds__(256, 3)
    k_bulk2_dia(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
  __shared__ double red[2][8][32];
  __shared__ __align__(16) float obs_rows[256 * kObsRow];
  W32 ws = view32(buf, bp.n_traj, 2, bp.n);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  unsigned int n_deg = 0;  // no degeneracy test in this representation
  int rb = 0;
  for (int64_t tile = blockIdx.x; tile < bp.n_tiles; tile += gridDim.x)
    bulk2_tile<NPL, KIND, Coef2, (NPL > 12), true>(bp, cf, ws, part, tile, rb, n_deg, red,
                                                   obs_rows);
}

namespace {
template <int NPL, int KIND>
int run_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part, int grid_cap,
            cudaStream_t st) {
  static int per_sm = -1, n_sm = 0;
  return run_bulk_kernel(k_bulk2_dia<NPL, KIND>, per_sm, n_sm, bp, cf, buf, part, grid_cap, st);
}

template <int KIND>
int dispatch_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part, int cap,
                 cudaStream_t st) {
  const int n = bp.n;
  if (n <= 1) return run_dia<1, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 2) return run_dia<2, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 3) return run_dia<3, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 4) return run_dia<4, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 8) return run_dia<8, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 16) return run_dia<16, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 32) return run_dia<32, KIND>(bp, cf, buf, part, cap, st);
  return 0;
}
}  // namespace

int launch_bulk2_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part, int grid_cap,
                     cudaStream_t st) {
  return bp.kind == 0 ? dispatch_dia<0>(bp, cf, buf, part, grid_cap, st)
                      : dispatch_dia<1>(bp, cf, buf, part, grid_cap, st);
}

}  // namespace qcl
