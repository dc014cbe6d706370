// kernels_f32.cu -- FP32-bulk path: a persistent kernel in which each thread
// owns one walker for a whole chunk of steps with its state in registers.
// Verlet, forces and couplings run in FP32; the phase and the weight are
// carried as compensated FP32 pairs (about 46 significant bits) so that no
// FP64 instruction sits in the step loop; observations are reduced per tile in
// FP64.  Random numbers: one Philox4x32-10 call per four steps.
#include <atomic>
#include <cstdio>

#include "bulk2.cuh"

namespace qcl {

// ---------------------------------------------------------------- sampling --
// FP32 initial sample from the same Philox words as the FP64 path.
__global__ void __launch_bounds__(256) k_sample_f32(const Sample32 sp, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = sp.n_traj;
  const int n = sp.n;
  W32 w = view32(buf, nt, 2, n);
  if (i == 0) {
    w.hdr->magic = kEnsMagic;
    w.hdr->n_traj = nt;
    w.hdr->precision = QCL_PREC_FP32_BULK;
    w.hdr->ns = 2;
    w.hdr->n = n;
    w.hdr->step = 0;
    w.hdr->flags = 0;
    w.hdr->n_degenerate = 0;
    w.hdr->n_nonfinite = 0;
  }
  if (i >= nt) return;
  float mh;
  uint16_t ab;
  sample_walker_f32(sp, sp.traj_offset + (uint64_t)i, w.R + i, w.P + i, nt, mh, ab);
  w.mh[i] = mh;
  w.ml[i] = 0.0f;
  w.me[i] = 0;
  w.ph[i] = 0.0f;
  w.pl[i] = 0.0f;
  w.ab[i] = ab;
}

// One thread per walker, all modes in registers, coefficients as constant-bank
// operands.  Tile = the block's 256 walkers.
template <int NPL, int KIND, int WPT = 1>
__global__ void __launch_bounds__(256, (WPT == 1 || NPL <= 4) ? 3 : 2)
    k_bulk2(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
  __shared__ double red[2 * WPT][8][32];  // per-warp partials, two sets of WPT
  __shared__ __align__(16) float obs_rows[256 * kObsRow];  // per-walker contributions
  W32 ws = view32(buf, bp.n_traj, 2, bp.n);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  unsigned int n_deg = 0;
  int rb = 0;
  for (int64_t tile = (int64_t)blockIdx.x * WPT; tile < bp.n_tiles; tile += (int64_t)gridDim.x * WPT)
    bulk2_tile<NPL, KIND, Coef2, (NPL > 12), false, WPT>(bp, cf, ws, part, tile, rb, n_deg, red,
                                                        obs_rows);
  if (n_deg) {
    atomicAdd(&ws.hdr->n_degenerate, (unsigned long long)n_deg);
    atomicOr(&ws.hdr->flags, QCL_FLAG_DEGENERATE);
  }
}

// ------------------------------------------------------------------ launch --
namespace {
std::atomic<int64_t> g_launches{0};
}
void launches_add(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_read(bool reset) {
  return reset ? g_launches.exchange(0) : g_launches.load();
}

void launch_sample_f32(const DevModel& host, const SampleParams& sp, void* buf, cudaStream_t st) {
  const int64_t nb = (sp.n_traj + 255) / 256;
  Sample32 s32;
  make_sample32(host, sp, s32);
  k_sample_f32<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, st>>>(s32, buf);
  launches_add(1);
}

namespace {
void occupancy(BulkFn fn, int& per_sm, int& n_sm) {
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
}
}  // namespace

int bulk_wpt(BulkFn fn2, int& per_sm, int& n_sm, int64_t n_tiles, const LaunchShape& ls) {
  occupancy(fn2, per_sm, n_sm);
  const int bps = (ls.blocks_per_sm > 0 && ls.blocks_per_sm < per_sm) ? ls.blocks_per_sm : per_sm;
  int64_t slots = (int64_t)bps * n_sm;
  if (ls.grid_cap > 0 && slots > ls.grid_cap) slots = ls.grid_cap;
  return n_tiles > slots ? 2 : 1;
}

int run_bulk_kernel(BulkFn fn, int& per_sm, int& n_sm, const BulkParams& bp, const Coef2& cf,
                    void* buf, double* part, const LaunchShape& ls, int wpt, cudaStream_t st) {
  occupancy(fn, per_sm, n_sm);
  const int bps = (ls.blocks_per_sm > 0 && ls.blocks_per_sm < per_sm) ? ls.blocks_per_sm : per_sm;
  int64_t grid = (int64_t)bps * n_sm;
  if (ls.grid_cap > 0 && grid > ls.grid_cap) grid = ls.grid_cap;
  const int64_t units = (bp.n_tiles + wpt - 1) / wpt;
  if (grid > units) grid = units;
  if (grid < 1) grid = 1;
  fn<<<(unsigned)grid, 256, 0, st>>>(bp, cf, buf, part);
  launches_add(1);
  return (int)grid;
}

namespace {
int run_kernel(BulkFn fn, int& per_sm, int& n_sm, const BulkParams& bp, const Coef2& cf, void* buf,
               double* part, const LaunchShape& ls, cudaStream_t st) {
  return run_bulk_kernel(fn, per_sm, n_sm, bp, cf, buf, part, ls, 1, st);
}

template <int NPL, int KIND, int WPT>
BulkFn bulk_fn() {
  if constexpr (WPT == 2 && NPL <= 8) return k_bulk2<NPL, KIND, 2>;
  else return k_bulk2<NPL, KIND, 1>;
}

template <int NPL, int KIND>
int run_bulk(const BulkParams& bp, const Coef2& cf, void* buf, double* part, const LaunchShape& ls,
             cudaStream_t st) {
  static int per_sm[2] = {-1, -1}, n_sm[2] = {0, 0};
  int wpt = (ls.wpt > 0 ? ls.wpt : default_wpt(NPL)) >= 2 && NPL <= 8 ? 2 : 1;
  if (wpt == 2) wpt = bulk_wpt(bulk_fn<NPL, KIND, 2>(), per_sm[1], n_sm[1], bp.n_tiles, ls);
  if (wpt == 2)
    return run_bulk_kernel(bulk_fn<NPL, KIND, 2>(), per_sm[1], n_sm[1], bp, cf, buf, part, ls, 2, st);
  return run_bulk_kernel(bulk_fn<NPL, KIND, 1>(), per_sm[0], n_sm[0], bp, cf, buf, part, ls, 1, st);
}

template <int KIND>
int dispatch_n(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
               const LaunchShape& cap, cudaStream_t st) {
  const int n = bp.n;
  if (n <= 1) return run_bulk<1, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 2) return run_bulk<2, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 3) return run_bulk<3, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 4) return run_bulk<4, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 6) return run_bulk<6, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 8) return run_bulk<8, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 12) return run_bulk<12, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 16) return run_bulk<16, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 24) return run_bulk<24, KIND>(bp, cf, buf, part, cap, st);
  if (n <= 32) return run_bulk<32, KIND>(bp, cf, buf, part, cap, st);
  return launch_bulk2_split(bp, cf, buf, part, cap, st);
}
}  // namespace

int launch_bulk2(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                 const LaunchShape& ls, cudaStream_t st) {
  if (bp.repr == QCL_REPR_DIABATIC) return launch_bulk2_dia(bp, cf, buf, part, ls, st);
  return bp.kind == 0 ? dispatch_n<0>(bp, cf, buf, part, ls, st)
                      : dispatch_n<1>(bp, cf, buf, part, ls, st);
}

namespace {
template <int KIND, int WPT>
BulkFn adiabatic_fn(int n) {
  if (n <= 1) return bulk_fn<1, KIND, WPT>();
  if (n <= 2) return bulk_fn<2, KIND, WPT>();
  if (n <= 3) return bulk_fn<3, KIND, WPT>();
  if (n <= 4) return bulk_fn<4, KIND, WPT>();
  if (n <= 6) return bulk_fn<6, KIND, WPT>();
  if (n <= 8) return bulk_fn<8, KIND, WPT>();
  return nullptr;
}
}  // namespace

BulkFn bulk2_dia_fn(int n, int kind, int wpt);

int bulk2_blocks_per_sm(int n, int kind, int repr, int wpt) {
  BulkFn fn = nullptr;
  if (repr == QCL_REPR_DIABATIC) {
    fn = bulk2_dia_fn(n, kind, wpt);
  } else if (n > 32) {
    fn = bulk2_split_fn(n, kind, wpt);
  } else if (n <= 8) {
    fn = kind == 0 ? (wpt == 2 ? adiabatic_fn<0, 2>(n) : adiabatic_fn<0, 1>(n))
                   : (wpt == 2 ? adiabatic_fn<1, 2>(n) : adiabatic_fn<1, 1>(n));
  }
  if (!fn) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess) return 0;
  return per_sm;
}

const char* bulk2_variant(int n, int kind) {
  (void)kind;
  switch (bulk_lanes(n)) {
    case 1: return "k_bulk2: one thread per walker, all modes in registers";
    case 2: return "k_bulk2_split2: two warps per 32 walkers";
    default:
      return n <= 100 ? "k_bulk2_split2: four warps per 32 walker slots, two walkers per thread"
                      : "k_bulk2_split2: four warps per 32 walkers";
  }
}

__global__ void k_header_finish(EnsHeader* h, int64_t step0, int64_t step1) {
  if (h->step == step0) h->step = step1;
}

void launch_header_finish(void* buf, int64_t step0, int64_t step1, cudaStream_t st) {
  k_header_finish<<<1, 1, 0, st>>>((EnsHeader*)buf, step0, step1);
  launches_add(1);
}

__global__ void k_header_set(EnsHeader* h, const EnsHeader v) { *h = v; }

void launch_header_set(void* buf, const EnsHeader& v, cudaStream_t st) {
  k_header_set<<<1, 1, 0, st>>>((EnsHeader*)buf, v);
  launches_add(1);
}

}  // namespace qcl
