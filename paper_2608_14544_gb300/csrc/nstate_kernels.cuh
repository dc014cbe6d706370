// nstate_kernels.cuh -- models with N_s = 3..8 electronic states: the per-N_s
// launchers over the FP64 path (nstate_f64.cuh), the FP32-bulk kernels
// (nstate_bulk.cuh) and FP32 spawning (nstate_spawn32.cuh).
#pragma once
#include <mutex>

#include "nstate_f64.cuh"
#include "nstate_spawn32.cuh"

namespace qcl {

// ------------------------------------------------------- per-N_s launchers --
// Instantiated one N_s per translation unit; the FP64 sampling and step
// kernels in their own units (kernels_nstate64_*.cu, compiled without FMA
// contraction so that their arithmetic is the oracle's).
template <int NS>
struct NStateOps {
  static void sample64(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_sampleN_f64<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(dm, sp, buf);
  }
  static void sample32(const SampleN32& sp, void* buf, cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_sampleN_f32<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(sp, buf);
  }
  static void step64(const DevModel* dm, int repr, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st) {
    const unsigned nb = (unsigned)((nt + 127) / 128);
    if (repr == QCL_REPR_DIABATIC)
      k_stepN_dia_f64<NS><<<nb, 128, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
    else
      k_stepN_f64<NS><<<nb, 128, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
  }
  static void observe64(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                        cudaStream_t st) {
    k_observeN_f64<NS><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(dm, buf, nt, n, part);
  }
  static void spawn_sample64(const DevModel* dm, const SampleParams& sp, int64_t cap, void* buf,
                             cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_spawnN_sample<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(dm, sp, cap, buf);
    launches_add(1);
  }
  // one spawning step: step kernel, scan, scatter (set step & 1 -> the other)
  static void spawn_step64(const DevModel* dm, void* buf, int64_t cap, int n, int64_t n0,
                           int64_t step0, int64_t step, double dt, uint64_t seed,
                           cudaStream_t st) {
    const unsigned nb = spawn_grid(cap);
    k_spawnN_step<NS><<<nb, 256, 0, st>>>(dm, buf, cap, n, n0, step0, step, dt, seed);
    launch_spawn_scan(buf, cap, n, n0, QCL_PREC_FP64, NS, step0, step, st);
    k_spawnN_scatter<NS><<<nb, 256, 0, st>>>(buf, cap, n, n0, step0, step, seed);
    launches_add(2);
  }
  static void spawn_sample32(const SampleN32& sp, int64_t cap, void* buf, cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_spawnN_sample32<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(sp, cap, buf);
    launches_add(1);
  }
  template <int NPL>
  static void spawn_step32_npl(const BulkParams& bp, const CoefN& cf, void* buf, int64_t cap,
                               int64_t n0, int64_t step, cudaStream_t st) {
    // (NPL = 0: the mode table in dynamic shared memory)
    size_t dyn = 0;
    if constexpr (NPL == 0) {
      dyn = ModeRow<NS>::bytes(bp.n);
      static std::mutex mu;
      static size_t dyn_set = 0;
      std::lock_guard<std::mutex> lock(mu);
      if (dyn > dyn_set) {
        cudaFuncSetAttribute(k_spawnN_step32<NS, NPL>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        dyn_set = dyn;
      }
    }
    k_spawnN_step32<NS, NPL><<<spawn_grid(cap), 256, dyn, st>>>(bp, cf, buf, cap, n0, step);
  }
  // one FP32 spawning step (step kernel, scan, scatter): up to 8 modes in
  // registers, beyond (or under the modes-in-memory option) in memory
  static int spawn_step32(const BulkParams& bp, const CoefN& cf, void* buf, int64_t cap,
                          int64_t n0, int64_t step0, int64_t step, cudaStream_t st) {
    if (cf.modes_in_memory == 1 || bp.n > 8) spawn_step32_npl<0>(bp, cf, buf, cap, n0, step, st);
    else if (bp.n <= 4) spawn_step32_npl<4>(bp, cf, buf, cap, n0, step, st);
    else spawn_step32_npl<8>(bp, cf, buf, cap, n0, step, st);
    launch_spawn_scan(buf, cap, bp.n, n0, QCL_PREC_FP32_BULK, NS, step0, step, st);
    k_spawnN_scatter32<NS><<<spawn_grid(cap), 256, 0, st>>>(buf, cap, bp.n, n0, step0, step,
                                                            bp.seed);
    launches_add(2);
    return 1;
  }
  static void spawn_observe32(const BulkParams& bp, const CoefN& cf, const void* buf, int64_t cap,
                              int64_t n0, int set, double* part, cudaStream_t st) {
    launch_spawn_fstart(buf, cap, bp.n, n0, QCL_PREC_FP32_BULK, NS, set, st);
    k_spawnN_observe32<NS><<<(unsigned)((n0 + 127) / 128), 128, 0, st>>>(bp, cf, buf, cap, n0,
                                                                         set, part);
    launches_add(1);
  }
  static void spawn_observe64(const DevModel* dm, const void* buf, int64_t cap, int n,
                              int64_t n0, int set, double* part, cudaStream_t st) {
    launch_spawn_fstart(buf, cap, n, n0, QCL_PREC_FP64, NS, set, st);
    k_spawnN_observe<NS><<<(unsigned)((n0 + 255) / 256), 256, 0, st>>>(dm, buf, cap, n, n0, set,
                                                                       part);
    launches_add(1);
  }
  template <int NPL, int WPT = 1>
  static int bulk_npl(const BulkParams& bp, const CoefN& cf, void* buf, double* part,
                      int grid_cap, cudaStream_t st) {
    // (occupancy cached per kernel and table size: [0] adiabatic, [1] diabatic;
    // NPL = 0: the mode table in dynamic shared memory)
    static int per_sm[2] = {-1, -1}, n_sm[2] = {0, 0};
    static size_t dyn_at[2] = {0, 0};
    const size_t dyn = NPL == 0 ? ModeRow<NS>::bytes(bp.n) : 0;
    if (bp.repr == QCL_REPR_DIABATIC)
      return launch_persistent(k_bulkN_dia<NS, NPL>, per_sm[1], n_sm[1], dyn_at[1], bp, cf, buf,
                               part, grid_cap, 1, dyn, st);
    return launch_persistent(k_bulkN<NS, NPL, WPT>, per_sm[0], n_sm[0], dyn_at[0], bp, cf, buf,
                             part, grid_cap, WPT, dyn, st);
  }
  // one persistent grid: the occupancy limit of resident blocks on every SM
  // (capped), at most one block per WPT tiles
  // (dyn > 0, the modes-in-memory kernels: the shared-memory limit only grows
  // and the occupancy is computed for this call's table, under a lock, so
  // that threads launching models of different mode counts do not race)
  template <typename Fn>
  static int launch_persistent(Fn fn, int& per_sm, int& n_sm, size_t& dyn_at, const BulkParams& bp,
                               const CoefN& cf, void* buf, double* part, int grid_cap, int WPT,
                               size_t dyn, cudaStream_t st) {
    int blocks = per_sm;
    if (dyn > 0) {
      static std::mutex mu;
      std::lock_guard<std::mutex> lock(mu);
      if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      }
      if (dyn > dyn_at) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        dyn_at = dyn;
      }
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 128, dyn) != cudaSuccess ||
          blocks < 1)
        blocks = 1;
    } else if (per_sm < 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 128, 0) != cudaSuccess ||
          blocks < 1)
        blocks = 1;
      per_sm = blocks;
    }
    int64_t grid = (int64_t)blocks * n_sm;
    if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
    const int64_t units = (bp.n_tiles + WPT - 1) / WPT;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    fn<<<(unsigned)grid, 128, dyn, st>>>(bp, cf, buf, part);
    return (int)grid;
  }
  // wpt: walkers per thread asked for.  The kernel takes one or two, but only
  // one is instantiated: two walkers per thread (packed lanes, 205-245
  // registers, 8 resident warps per SM) measured 10 % slower on a four-state
  // six-mode model than one (114 registers, 16 warps), with the same bits.
  static int bulk(const BulkParams& bp, const CoefN& cf, void* buf, double* part, int grid_cap,
                  int wpt, cudaStream_t st) {
    (void)wpt;
    // Register forms exist up to 8 modes for any N_s and up to 32 modes for
    // N_s <= 4 (larger N_s x modes would not fit a walker in registers); the
    // modes-in-memory form takes any mode count with the same bits.  The
    // automatic choice follows measured solve rates on GB300 (1e6 walkers,
    // 200 steps, random LVC models): registers for N_s = 3 (except adiabatic
    // models of 9-16 modes, where the 32-mode register form is 10-30 % slower)
    // and for N_s = 4 up to 8 modes (20-30 % faster); the memory form beyond
    // (N_s = 4 with 12-32 modes: 1.3-2.6x faster) and for N_s >= 5 at every
    // mode count (1.0-2.2x, the register forms there run one or two blocks per
    // SM).  Models of at most 4 or 6 modes get their own instantiations,
    // which skip the padding modes' arithmetic (padding modes have zero
    // coefficients and stay at zero).
    const int reg_max = NS <= 4 ? 32 : 8;
    bool mem;
    if (cf.modes_in_memory == 1) mem = true;
    else if (cf.modes_in_memory == 2) mem = bp.n > reg_max;
    else if (NS == 3) mem = bp.n > 32 || (bp.repr != QCL_REPR_DIABATIC && bp.n > 8 && bp.n <= 16);
    else if (NS == 4) mem = bp.n > 8;
    else mem = true;
    if (mem) return bulk_npl<0>(bp, cf, buf, part, grid_cap, st);
    if constexpr (NS <= 5) {
      if (bp.n <= 4) return bulk_npl<4>(bp, cf, buf, part, grid_cap, st);
      if (bp.n <= 6) return bulk_npl<6>(bp, cf, buf, part, grid_cap, st);
    }
    if (bp.n <= 8) return bulk_npl<8>(bp, cf, buf, part, grid_cap, st);
    if (NS <= 4 && bp.n <= 32) return bulk_npl<(NS <= 4 ? 32 : 8)>(bp, cf, buf, part, grid_cap, st);
    return 0;
  }
};

}  // namespace qcl
