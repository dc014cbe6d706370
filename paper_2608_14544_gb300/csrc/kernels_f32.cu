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

// Many-mode models: a walker's modes are split over L warps (warp role r holds
// modes r NPL .. r NPL + NPL - 1 of the same 32 walkers), so every coefficient
// index stays warp-uniform and compile-time (a constant-bank operand, no
// loads).  The two collective sums of a step are exchanged through shared
// memory under a named barrier of the L warps, and added in role order, so all
// L warps hold the same bits of the scalar state.  The role-0 warp observes
// exactly as the one-thread-per-walker kernel does.  Tile = the block's 256 / L
// walkers (8 / L groups of 32).
__device__ __forceinline__ void group_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int NPL, int L, int KIND, int ROLE>
__device__ __forceinline__ void split_tiles(const BulkParams& bp, const Coef2& cf, W32& ws,
                                            double* __restrict__ part, float (*x0)[256 / L][2],
                                            float (*xa)[256 / L][2], float (*xv)[256 / L][2],
                                            double (*red)[8][32], float* obs_rows,
                                            unsigned int& n_deg) {
  constexpr int BW = 256 / L;  // walkers per tile
  constexpr int G = BW / 32;   // groups (of 32 walkers) per tile
  constexpr int OFF = ROLE * NPL;
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp % G;             // this warp's walker group in the tile
  const int wslot = grp * 32 + lane;    // walker slot within the tile
  const int bar_id = 1 + grp;           // named barrier of the group's L warps
  int rb = 0;
  for (int64_t tile = blockIdx.x; tile < bp.n_tiles; tile += gridDim.x) {
    // every warp of the group has finished the previous tile's exchanges
    group_barrier(bar_id, 32 * L);
    const int64_t i = tile * BW + wslot;
    const bool active = i < nt;
    const int64_t ii = active ? i : 0;
    Walker<NPL> w;
#pragma unroll
    for (int t = 0; t < NPL; ++t) {
      const bool on = active && OFF + t < bp.n;
      w.R[t] = on ? ws.R[(int64_t)(OFF + t) * nt + ii] : 0.0f;
      w.P[t] = on ? ws.P[(int64_t)(OFF + t) * nt + ii] : 0.0f;
    }
    Scal z;
    z.m = {active ? ws.mh[ii] : 0.0f, active ? ws.ml[ii] : 0.0f};
    z.mexp = active ? ws.me[ii] : 0;
    z.ph = {active ? ws.ph[ii] : 0.0f, active ? ws.pl[ii] : 0.0f};
    const uint32_t ab = active ? ws.ab[ii] : 0u;
    z.sa = sgn(ab & 0xf);
    z.sb = sgn((ab >> 8) & 0xf);
    z.q = 0;
    const uint64_t traj = bp.traj_offset + (uint64_t)ii;
    unsigned int deg = 0;

    // sum over the L roles of per-role partials, in role order
    auto exchange = [&](float (*x)[BW][2], float pa, float pb, float& A, float& B) {
      x[ROLE][wslot][0] = pa;
      if (KIND == 1) x[ROLE][wslot][1] = pb;
      group_barrier(bar_id, 32 * L);
      float sa_ = x[0][wslot][0], sb_ = (KIND == 1) ? x[0][wslot][1] : 0.0f;
#pragma unroll
      for (int r = 1; r < L; ++r) {
        sa_ += x[r][wslot][0];
        if (KIND == 1) sb_ += x[r][wslot][1];
      }
      A = sa_;
      B = sb_;
    };

    {
      float pa = 0.0f, pb = 0.0f;
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        pa = __fmaf_rn(cf.a[OFF + t], w.R[t], pa);
        if (KIND == 1) pb = __fmaf_rn(cf.b[OFF + t], w.R[t], pb);
      }
      float A, B;
      exchange(x0, pa, pb, A, B);  // own buffer: the first step writes xa next
      z.A = bp.a0 + A;
      z.B = bp.b0 + B;
    }
    closed_form(z);

    auto observe = [&](int slot) {
      if (ROLE == 0) {
        observe_warp<false, false>(z, active, obs_rows, wslot, grp * 32, lane, red[rb][grp]);
      } else {  // the same phase bookkeeping on every role
        phase_wrap(z);
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        const int q = threadIdx.x;
        double t0;
        if (G == 1) t0 = red[rb][0][q];
        else if (G == 2) t0 = red[rb][0][q] + red[rb][G - 1][q];
        else t0 = (red[rb][0][q] + red[rb][1 % G][q]) + (red[rb][2 % G][q] + red[rb][3 % G][q]);
        part[((int64_t)slot * bp.n_tiles + tile) * 32 + q] = t0;
      }
      rb ^= 1;
    };

    int slot = bp.obs_first;
    if (bp.obs_first) observe(0);
    int to_out = bp.to_out0;
    uint32_t blk = bp.blk0;
    int widx = bp.widx0;
    const PhiloxStream rng(bp.seed, traj, kPurposeHop);
    u4 wd = rng.draw(blk);
    for (int it = 0; it < bp.len; ++it) {
      const uint32_t word = pick_word(wd, widx);
      const float hsab = bp.hdt * 0.5f * (z.sa + z.sb);
      const float hu = hsab * z.c2, hv = hsab * z.s2;
      float pa = 0.0f, pb = 0.0f;
#pragma unroll
      for (int t = 0; t < NPL; ++t) {  // first half kick at R_n, drift, partial sums at R_{n+1}
        float p = __fmaf_rn(-cf.hk[OFF + t], w.R[t], w.P[t]);
        if (KIND == 1) p -= cf.hs[OFF + t];
        p = __fmaf_rn(-hu, cf.a[OFF + t], p);
        if (KIND == 1) p = __fmaf_rn(-hv, cf.b[OFF + t], p);
        w.P[t] = p;
        w.R[t] = __fmaf_rn(cf.dtm[OFF + t], p, w.R[t]);
        pa = __fmaf_rn(cf.a[OFF + t], w.R[t], pa);
        if (KIND == 1) pb = __fmaf_rn(cf.b[OFF + t], w.R[t], pb);
      }
      const float r_old = z.r;
      {
        float A, B;
        exchange(xa, pa, pb, A, B);
        z.A = bp.a0 + A;
        z.B = bp.b0 + B;
      }
      closed_form<KIND == 1>(z);
      const float hu2 = hsab * z.c2, hv2 = hsab * z.s2;
      float av = 0.0f, bv = 0.0f;
#pragma unroll
      for (int t = 0; t < NPL; ++t) {  // second half kick at R_{n+1}, partial coupling sums
        float p = __fmaf_rn(-cf.hk[OFF + t], w.R[t], w.P[t]);
        if (KIND == 1) p -= cf.hs[OFF + t];
        p = __fmaf_rn(-hu2, cf.a[OFF + t], p);
        if (KIND == 1) p = __fmaf_rn(-hv2, cf.b[OFF + t], p);
        w.P[t] = p;
        av = __fmaf_rn(cf.am[OFF + t], p, av);
        if (KIND == 1) bv = __fmaf_rn(cf.bm[OFF + t], p, bv);
      }
      float Av, Bv;
      exchange(xv, av, bv, Av, Bv);
      phase_and_transition<KIND>(z, r_old, Av, Bv, word, bp, deg);
      if (++widx == 4) {  // pairs renormalised at the end of every Philox block
        widx = 0;
        block_end(z);
        ++blk;
        if (it + 1 < bp.len) wd = rng.draw(blk);
      }
      if (--to_out == 0) {
        observe(slot++);
        to_out = bp.stride;
      }
    }
    if (active) {
      n_deg += deg;
#pragma unroll
      for (int t = 0; t < NPL; ++t)
        if (OFF + t < bp.n) {
          ws.R[(int64_t)(OFF + t) * nt + i] = w.R[t];
          ws.P[(int64_t)(OFF + t) * nt + i] = w.P[t];
        }
      if (ROLE == 0) {
        ws.mh[i] = z.m.hi;
        ws.ml[i] = z.m.lo;
        ws.me[i] = z.mexp;
        ws.ph[i] = z.ph.hi;
        ws.pl[i] = z.ph.lo;
        ws.ab[i] = (uint16_t)((z.sa > 0.0f ? 1 : 0) | ((z.sb > 0.0f ? 1 : 0) << 8));
        if (!isfinite(z.m.hi) || !isfinite(z.ph.hi)) {
          atomicAdd(&ws.hdr->n_nonfinite, 1ull);
          atomicOr(&ws.hdr->flags, QCL_FLAG_NONFINITE);
        }
      }
    }
  }
}

template <int NPL, int L, int KIND, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_bulk2_split(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
  constexpr int BW = 256 / L;
  // per role and walker: partial sums a(R), b(R) at tile start (x0) and in the
  // step (xa), partial coupling sums (xv); three buffers so that no warp
  // overwrites a value its partners have not read yet
  __shared__ float x0[L][BW][2];
  __shared__ float xa[L][BW][2];
  __shared__ float xv[L][BW][2];
  __shared__ double red[2][8][32];
  __shared__ __align__(16) float obs_rows[BW * kObsRow];
  W32 ws = view32(buf, bp.n_traj, 2, bp.n);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  unsigned int n_deg = 0;
  const int role = (threadIdx.x >> 5) / (BW / 32);
  if (role == 0) split_tiles<NPL, L, KIND, 0>(bp, cf, ws, part, x0, xa, xv, red, obs_rows, n_deg);
  else if (role == 1) split_tiles<NPL, L, KIND, 1 % L>(bp, cf, ws, part, x0, xa, xv, red, obs_rows, n_deg);
  else if (role == 2) split_tiles<NPL, L, KIND, 2 % L>(bp, cf, ws, part, x0, xa, xv, red, obs_rows, n_deg);
  else split_tiles<NPL, L, KIND, 3 % L>(bp, cf, ws, part, x0, xa, xv, red, obs_rows, n_deg);
  if (n_deg && role == 0) {  // every role counted the same walkers
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

template <int NPL, int L, int KIND, int MINB>
int run_wide(const BulkParams& bp, const Coef2& cf, void* buf, double* part, const LaunchShape& cap,
             cudaStream_t st) {
  static int per_sm = -1, n_sm = 0;
  return run_kernel(k_bulk2_split<NPL, L, KIND, MINB>, per_sm, n_sm, bp, cf, buf, part, cap, st);
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
  // warps per walker must agree with bulk_lanes(n)
  constexpr int MB = KIND == 0 ? 2 : 1;
  if (n <= 64) return run_wide<32, 2, KIND, MB>(bp, cf, buf, part, cap, st);
  if (n <= 100) return launch_bulk2_split2(bp, cf, buf, part, cap, st);
  if (n <= 128) return run_wide<32, 4, KIND, MB>(bp, cf, buf, part, cap, st);
  if (n <= 256) return run_wide<64, 4, KIND, 1>(bp, cf, buf, part, cap, st);
  return 0;
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
  } else if (n > 64 && n <= 100) {
    fn = bulk2_split2_fn(kind, wpt);
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
    case 2: return "k_bulk2_split: two warps per 32 walkers";
    default:
      return n <= 100 ? "k_bulk2_split2: four warps per 32 walker slots, two walkers per thread"
                      : "k_bulk2_split: four warps per 32 walkers";
  }
}

__global__ void k_header_finish(EnsHeader* h, int64_t step0, int64_t step1) {
  if (h->step == step0) h->step = step1;
}

void launch_header_finish(void* buf, int64_t step0, int64_t step1, cudaStream_t st) {
  k_header_finish<<<1, 1, 0, st>>>((EnsHeader*)buf, step0, step1);
  launches_add(1);
}

}  // namespace qcl
