// kernels_dia.cu -- FP32-bulk persistent kernel of the diabatic representation
// (two states, one thread per walker, up to 32 modes): the same tile body as
// the adiabatic kernel with the diagonal mean force, the diabatic phase and
// the quarter-turn transitions (bulk2.cuh, DIA = true).  Models of 33..256
// modes run the split form (kernels_split.cu).
#include "bulk2.cuh"

namespace qcl {

// (kernels_split.cu)
int launch_bulk2_split_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                           const LaunchShape& ls, cudaStream_t st);
BulkFn bulk2_split_dia_fn(int n, int kind, int wpt);

template <int NPL, int KIND, int WPT>
__global__ void __launch_bounds__(256, (WPT == 1 || NPL <= 4) ? 3 : 2)
    k_bulk2_dia(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
  __shared__ double red[2 * WPT][8][32];
  __shared__ __align__(16) float obs_rows[256 * kObsRow];
  W32 ws = view32(buf, bp.n_traj, 2, bp.n);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  unsigned int n_deg = 0;  // no degeneracy test in this representation
  int rb = 0;
  for (int64_t tile = (int64_t)blockIdx.x * WPT; tile < bp.n_tiles; tile += (int64_t)gridDim.x * WPT)
    bulk2_tile<NPL, KIND, Coef2, (NPL > 12), true, WPT>(bp, cf, ws, part, tile, rb, n_deg, red,
                                                        obs_rows);
}

namespace {
template <int NPL, int KIND, int WPT>
BulkFn dia_fn() {
  if constexpr (WPT == 2 && NPL <= 8) return k_bulk2_dia<NPL, KIND, 2>;
  else return k_bulk2_dia<NPL, KIND, 1>;
}

template <int NPL, int KIND>
int run_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part, const LaunchShape& ls,
            cudaStream_t st) {
  static int per_sm[2] = {-1, -1}, n_sm[2] = {0, 0};
  int wpt = (ls.wpt > 0 ? ls.wpt : default_wpt(NPL)) >= 2 && NPL <= 8 ? 2 : 1;
  if (wpt == 2) wpt = bulk_wpt(dia_fn<NPL, KIND, 2>(), per_sm[1], n_sm[1], bp.n_tiles, ls);
  if (wpt == 2)
    return run_bulk_kernel(dia_fn<NPL, KIND, 2>(), per_sm[1], n_sm[1], bp, cf, buf, part, ls, 2, st);
  return run_bulk_kernel(dia_fn<NPL, KIND, 1>(), per_sm[0], n_sm[0], bp, cf, buf, part, ls, 1, st);
}

template <int KIND>
int dispatch_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                 const LaunchShape& ls, cudaStream_t st) {
  const int n = bp.n;
  if (n <= 1) return run_dia<1, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 2) return run_dia<2, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 3) return run_dia<3, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 4) return run_dia<4, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 8) return run_dia<8, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 16) return run_dia<16, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 32) return run_dia<32, KIND>(bp, cf, buf, part, ls, st);
  return launch_bulk2_split_dia(bp, cf, buf, part, ls, st);
}

template <int KIND, int WPT>
BulkFn dia_fn_n(int n) {
  if (n <= 1) return dia_fn<1, KIND, WPT>();
  if (n <= 2) return dia_fn<2, KIND, WPT>();
  if (n <= 3) return dia_fn<3, KIND, WPT>();
  if (n <= 4) return dia_fn<4, KIND, WPT>();
  if (n <= 8) return dia_fn<8, KIND, WPT>();
  if (n <= 16) return dia_fn<16, KIND, 1>();
  if (n <= 32) return dia_fn<32, KIND, 1>();
  return nullptr;
}
}  // namespace

BulkFn bulk2_dia_fn(int n, int kind, int wpt) {
  if (n > 32) return bulk2_split_dia_fn(n, kind, wpt);
  const bool two = wpt == 2 && n <= 8;
  return kind == 0 ? (two ? dia_fn_n<0, 2>(n) : dia_fn_n<0, 1>(n))
                   : (two ? dia_fn_n<1, 2>(n) : dia_fn_n<1, 1>(n));
}

int launch_bulk2_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                     const LaunchShape& ls, cudaStream_t st) {
  return bp.kind == 0 ? dispatch_dia<0>(bp, cf, buf, part, ls, st)
                      : dispatch_dia<1>(bp, cf, buf, part, ls, st);
}

}  // namespace qcl
