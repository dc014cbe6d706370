// kernels.h -- host-side declarations of the kernel launchers and their
// parameter blocks (passed by value as kernel parameters).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "qcl_common.cuh"

namespace qcl {

struct SampleParams {
  int64_t n_traj;
  uint64_t traj_offset;
  uint64_t seed;
  int32_t n, ns;
  int32_t wigner;
  int32_t pad;
  double R0[kMaxN], P0[kMaxN], sR[kMaxN], sP[kMaxN];
  double rho[kMaxNS * kMaxNS];
};

// The two-state FP32 sampler's inputs, converted to FP32 once on the host
// (make_sample32), so that the sampler does no FP64 arithmetic.
struct Sample32 {
  int64_t n_traj;
  uint64_t traj_offset;
  uint64_t seed;
  int32_t n, wigner, repr, pad;
  float a0, b0;
  float rho[4];
  float R0[kMaxN], P0[kMaxN], sR[kMaxN], sP[kMaxN], a[kMaxN], b[kMaxN];
};

inline void make_sample32(const DevModel& h, const SampleParams& sp, Sample32& s) {
  s.n_traj = sp.n_traj;
  s.traj_offset = sp.traj_offset;
  s.seed = sp.seed;
  s.n = sp.n;
  s.wigner = sp.wigner;
  s.repr = h.repr;
  s.pad = 0;
  s.a0 = (float)h.a0;
  s.b0 = (float)h.b0;
  for (int k = 0; k < 4; ++k) s.rho[k] = (float)sp.rho[k];
  for (int j = 0; j < kMaxN; ++j) {
    const bool on = j < sp.n;
    s.R0[j] = on ? (float)sp.R0[j] : 0.0f;
    s.P0[j] = on ? (float)sp.P0[j] : 0.0f;
    s.sR[j] = on ? (float)sp.sR[j] : 0.0f;
    s.sP[j] = on ? (float)sp.sP[j] : 0.0f;
    s.a[j] = on ? (float)h.a[j] : 0.0f;
    s.b[j] = on ? (float)h.b[j] : 0.0f;
  }
}

// The N_s-state FP32 sampler's inputs, converted to FP32 once on the host:
// E (N_s x N_s), K_j (N_s x N_s each, j < n, when n N_s^2 <= kSampleNK; larger
// models are read from the model's FP64 K on the device and rounded to FP32
// there, the same values) and the initial density.
constexpr int kSampleNK = 512;
struct SampleN32 {
  int64_t n_traj;
  uint64_t traj_offset;
  uint64_t seed;
  int32_t n, ns, wigner, repr;
  float R0[kMaxN], P0[kMaxN], sR[kMaxN], sP[kMaxN];
  float E[kMaxNS * kMaxNS];
  float rho[kMaxNS * kMaxNS];
  float K[kSampleNK];
  const double* Kd;  // the model's K on the device, [n][N_s][N_s]
};

// FP32 per-mode coefficients of a two-state model for one time step dt.
struct Coef2 {
  float hk[kMaxN];   // dt/2 * k_j
  float hs[kMaxN];   // dt/2 * s_j
  float dtm[kMaxN];  // dt / M_j
  float a[kMaxN];    // d a / d R_j
  float b[kMaxN];    // d b / d R_j
  float am[kMaxN];   // a_j / M_j
  float bm[kMaxN];   // b_j / M_j
};

struct BulkParams {
  int64_t n_traj;
  int64_t n_tiles;
  uint64_t traj_offset;
  uint64_t seed;
  int64_t step0;       // ensemble step expected at the start of the call
  int64_t cs, ce;      // absolute steps [cs, ce) advanced by this launch
  int64_t k_first;     // absolute output index of slot 0
  int32_t stride;      // output stride
  int32_t obs_first;   // observe at cs before stepping (only at s = 0)
  int32_t len;         // ce - cs
  int32_t to_out0;     // steps from cs until the first output
  uint32_t blk0;       // Philox block of step cs (cs >> 2)
  int32_t widx0;       // word of step cs in its block (cs & 3)
  int32_t n;           // modes
  int32_t kind;        // 0: a_j only (spin-boson form), 1: general two-state
  int32_t repr;        // QCL_REPR_ADIABATIC or QCL_REPR_DIABATIC
  float a0, b0;
  float dt, hdt;       // dt, dt/2
  float hdt_hbar;      // dt / (2 hbar)
  float amp;           // amplitude per unit coupling: |A_e| = amp |g| (adiabatic,
                       // amp = dt) or amp |V_01| (diabatic, amp = dt / hbar)
  float kamp;          // hop_scale * amp
  float p_max;
  uint32_t tmax;       // floor(p_max 2^24)
  float kappa;         // hop_scale
  // sum_j a_j a_j / M_j, sum_j a_j b_j / M_j, sum_j b_j b_j / M_j over the
  // FP32 coefficients (the split kernel's one-exchange coupling sums)
  float caa, cab, cbb;
};

// FP32 degeneracy test of the adiabatic two-state kernels: the coupling is set
// to zero where r^2 < kDegR2_32 (2r = e_b - e_a below kDegTol32).
constexpr float kDegTol32 = 1e-6f;
constexpr float kDegR2_32 = 0.25f * kDegTol32 * kDegTol32;

// Kernel form of a two-state model in the FP32-bulk kernels: 0 (only a(R)
// depends on R, b = b0) or 1 (general).  In the adiabatic representation the
// spin-boson form is used only when b0^2 alone keeps r^2 = a^2 + b0^2 at or
// above the degeneracy threshold, so that its kernels need no degeneracy
// test; a spin-boson model with |b0| that small runs the general form.
inline int bulk_kind(const DevModel& h) {
  if (h.kind != 0 || h.repr == QCL_REPR_DIABATIC) return h.kind;
  const float b0 = (float)h.b0;
  return b0 * b0 >= kDegR2_32 ? 0 : 1;
}

// The model-dependent scalars of a bulk launch for time step dt (every caller
// fills them here, so the single-request, packed and no-allocation routes see
// the same values).
inline void bulk_model_scalars(BulkParams& bp, const DevModel& h, double dt) {
  bp.kind = bulk_kind(h);
  bp.repr = h.repr;
  bp.a0 = (float)h.a0;
  bp.b0 = (float)h.b0;
  bp.dt = (float)dt;
  bp.hdt = (float)(0.5 * dt);
  bp.hdt_hbar = (float)(0.5 * dt / h.hbar);
  const double amp = (h.repr == QCL_REPR_DIABATIC) ? dt / h.hbar : dt;
  bp.amp = (float)amp;
  bp.kamp = (float)(h.hop_scale * amp);
  bp.p_max = (float)h.p_max;
  bp.tmax = (uint32_t)std::floor(h.p_max * kP24);
  bp.kappa = (float)h.hop_scale;
  double caa = 0.0, cab = 0.0, cbb = 0.0;
  for (int j = 0; j < h.n; ++j) {
    const double a = (float)h.a[j], b = (float)h.b[j];
    const double am = (float)(h.a[j] / h.mass[j]), bm = (float)(h.b[j] / h.mass[j]);
    caa += am * a;
    cab += am * b;
    cbb += bm * b;
  }
  bp.caa = (float)caa;
  bp.cab = (float)cab;
  bp.cbb = (float)cbb;
}

// FP32 coefficients of an N_s-state model (N_s <= 8): upper triangles
// (row-major a <= b) of E and of each K_j, the per-mode ones for the first 32
// modes.  The kernels that keep the modes in memory build their per-mode table
// on the device from the model (dm) and dt, with the same roundings.
struct CoefN {
  float hk[32];    // dt/2 * k_j
  float dtm[32];   // dt / M_j
  float minv[32];  // 1 / M_j
  float K[32][36];
  float E[36];
  // the model on the device and dt, as 32-bit words (the struct keeps 4-byte
  // alignment, so the kernels' parameter layout stays as it was)
  uint32_t dm_w[2];
  uint32_t dt_w[2];
  int32_t modes_in_memory;  // 0: measured choice, 1: modes in memory, 2: in registers where a form exists
  int32_t pad;
};
inline void coef_set_model(CoefN& c, const DevModel* dm, double dt) {
  uint64_t a, d;
  std::memcpy(&a, &dm, sizeof a);
  std::memcpy(&d, &dt, sizeof d);
  c.dm_w[0] = (uint32_t)a;
  c.dm_w[1] = (uint32_t)(a >> 32);
  c.dt_w[0] = (uint32_t)d;
  c.dt_w[1] = (uint32_t)(d >> 32);
}
__device__ __forceinline__ const DevModel* coef_dm(const CoefN& c) {
  return reinterpret_cast<const DevModel*>(((uint64_t)c.dm_w[1] << 32) | c.dm_w[0]);
}
__device__ __forceinline__ double coef_dt(const CoefN& c) {
  return __hiloint2double((int)c.dt_w[1], (int)c.dt_w[0]);
}

// One request of a packed launch: a two-state model with at most 8 modes
// advancing over its own steps [cs, ce) (device table entry).
constexpr int kMaxPacked = 256;
struct PackedReq {
  BulkParams bp;
  void* ens;          // the request's ensemble buffer
  double* part;       // its per-tile partials
  int64_t work0;      // first global work item (tile) of this request
  float hk[8], hs[8], dtm[8], a[8], b[8], am[8], bm[8];
};
struct PackedTable {
  int64_t n_work;     // total tiles of all requests
  int32_t n_req;
  int32_t pad;
  PackedReq req[kMaxPacked];
};
// Mode-count buckets of the packed kernel (a request with n modes runs in the
// smallest bucket >= n); returns the bucket index or -1 if n > 8.
inline int packed_bucket(int n) {
  return n <= 1 ? 0 : n <= 2 ? 1 : n <= 3 ? 2 : n <= 4 ? 3 : n <= 6 ? 4 : n <= 8 ? 5 : -1;
}
constexpr int kPackedBuckets = 6;
// Launches the packed kernel of (bucket, kind) over the device table; returns
// the grid size.
int launch_packed(int bucket, int kind, const PackedTable* dtab, cudaStream_t st);

// ------------------------------------------------------------- spawning --
// Buffer of a spawning ensemble (any precision and N_s): the common header (its
// n_traj = the n0 initial walkers = families) with SpawnHeader after it, then
// two walker sets of `capacity` slots (the current set alternates with the
// absolute step: set = step & 1), per-parent staging of the children of a
// step, per-block spawn counts and offsets, and the family start indices.
struct SpawnHeader {
  int64_t capacity;
  int64_t n0;
  int64_t n_live[2];  // live walkers of set 0 and set 1
  int32_t drop;       // set by the scan when a step's children do not fit
  int32_t pad;
};
constexpr size_t kSpawnHeaderOff = 64;  // after EnsHeader, inside the first 256 bytes

struct SpawnLayout {
  // walker set: R[n][cap], P[n][cap], m, phi, ab (uint16), id (uint64),
  // fam (uint32); FP32 sets add m_lo, m_exp (int32) and phi_lo (compensated
  // pairs with a carried exponent, as in the bulk kernels); sets of N_s > 2
  // states add the carried eigenvectors U[ns * ns][cap] and, in FP32, the
  // eigenvalues E[ns][cap] (the warm start of the next decomposition)
  size_t set_off[2];
  size_t R, P, m, mlo, mexp, phi, philo, ab, id, fam, U, E, set_bytes;
  // staging of a step's children, per parent: weight (FP32: hi, lo, exp), pair
  size_t cm, cmlo, cmexp, cab, flag, bsum, boff, fstart, total;
  int64_t n_blocks;  // capacity / 256, rounded up
  __host__ __device__ static SpawnLayout make(int64_t cap, int n, int64_t n0, int precision,
                                              int ns = 2) {
    SpawnLayout L{};
    const size_t c = (size_t)cap;
    const bool f32 = precision == QCL_PREC_FP32_BULK;
    const size_t w = f32 ? 4 : 8;
    size_t o = 0;
    L.R = o;
    o = align256(o + w * c * (size_t)n);
    L.P = o;
    o = align256(o + w * c * (size_t)n);
    L.m = o;
    o = align256(o + w * c);
    L.mlo = o;
    if (f32) o = align256(o + 4 * c);
    L.mexp = o;
    if (f32) o = align256(o + 4 * c);
    L.phi = o;
    o = align256(o + w * c);
    L.philo = o;
    if (f32) o = align256(o + 4 * c);
    L.ab = o;
    o = align256(o + 2 * c);
    L.id = o;
    o = align256(o + 8 * c);
    L.fam = o;
    o = align256(o + 4 * c);
    L.U = o;
    if (ns > 2) o = align256(o + w * c * (size_t)(ns * ns));
    L.E = o;
    if (ns > 2 && f32) o = align256(o + 4 * c * (size_t)ns);
    L.set_bytes = o;
    L.set_off[0] = 256;
    L.set_off[1] = 256 + L.set_bytes;
    o = 256 + 2 * L.set_bytes;
    L.cm = o;
    o = align256(o + w * c);
    L.cmlo = o;
    if (f32) o = align256(o + 4 * c);
    L.cmexp = o;
    if (f32) o = align256(o + 4 * c);
    L.cab = o;
    o = align256(o + 2 * c);
    L.flag = o;
    o = align256(o + c);
    L.n_blocks = (cap + 255) / 256;
    L.bsum = o;
    o = align256(o + 4 * (size_t)L.n_blocks);
    L.boff = o;
    o = align256(o + 8 * (size_t)L.n_blocks);
    L.fstart = o;
    o = align256(o + 8 * ((size_t)n0 + 1));
    L.total = o;
    return L;
  }
};

void launch_spawn_sample(const DevModel* dm, const SampleParams& sp, int64_t capacity, void* buf,
                         cudaStream_t st);
// One spawning step (step kernel, scan, scatter) from set step & 1 to the other.
void launch_spawn_step(const DevModel* dm, int repr, void* buf, int64_t capacity, int n,
                       int64_t n0, int64_t step0, int64_t step, double dt, uint64_t seed,
                       cudaStream_t st);
// Family sums of the current set (set) into per-tile partials (tiles of 256
// families).
void launch_spawn_observe(const DevModel* dm, const void* buf, int64_t capacity, int n, int64_t n0,
                          int set, double* part, cudaStream_t st);
// Grid of the spawning kernels: a few blocks per SM, each walking groups of 256
// walkers up to the live count (which the host does not know).
unsigned spawn_grid(int64_t capacity);
// The block-count scan and the family starts, for either precision's layout.
void launch_spawn_scan(void* buf, int64_t capacity, int n, int64_t n0, int precision, int ns, int64_t step0,
                       int64_t step, cudaStream_t st);
void launch_spawn_fstart(const void* buf, int64_t capacity, int n, int64_t n0, int precision, int ns, int set,
                         cudaStream_t st);
// FP64 spawning for N_s = 3..8 states (either representation): sample, one
// step (step kernel, scan, scatter), observation (family starts, family sums).
void launch_spawnN_sample(const DevModel* dm, int ns, const SampleParams& sp, int64_t capacity,
                          void* buf, cudaStream_t st);
void launch_spawnN_step(const DevModel* dm, int ns, void* buf, int64_t capacity, int n, int64_t n0,
                        int64_t step0, int64_t step, double dt, uint64_t seed, cudaStream_t st);
void launch_spawnN_observe(const DevModel* dm, int ns, const void* buf, int64_t capacity, int n,
                           int64_t n0, int set, double* part, cudaStream_t st);
// FP32-bulk spawning for N_s = 3..8 states (either representation, any mode
// count; kernels in nstate_spawn32.cuh): sample, one step, observation.
void launch_spawnN_sample32(int ns, const SampleN32& sp, int64_t capacity, void* buf,
                            cudaStream_t st);
int launch_spawnN_step32(int ns, const BulkParams& bp, const CoefN& cf, void* buf,
                         int64_t capacity, int64_t n0, int64_t step0, int64_t step,
                         cudaStream_t st);
void launch_spawnN_observe32(int ns, const BulkParams& bp, const CoefN& cf, const void* buf,
                             int64_t capacity, int64_t n0, int set, double* part,
                             cudaStream_t st);
// FP32-bulk spawning (two states, n <= 32 modes): sample, one step (step
// kernel, scan, scatter), family observation.
void launch_spawn_sample32(const DevModel& host, const SampleParams& sp, int64_t capacity, void* buf,
                           cudaStream_t st);
int launch_spawn_step32(const BulkParams& bp, const Coef2& cf, void* buf, int64_t capacity,
                        int64_t n0, int64_t step0, int64_t step, cudaStream_t st);
void launch_spawn_observe32(const BulkParams& bp, const Coef2& cf, const void* buf, int64_t capacity,
                            int64_t n0, int set, double* part, cudaStream_t st);

// Kernel launches issued by the library (instrumentation).
void launches_add(int64_t k);
int64_t launches_read(bool reset);

void launch_sample_f64(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st);
void launch_step_f64(const DevModel* dm, int repr, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st);
void launch_observe_f64(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                        cudaStream_t st);

// Launch shape of a persistent bulk launch; the results do not depend on it.
struct LaunchShape {
  int wpt = 0;            // walkers per thread, 1 or 2 (0: the default for the mode count)
  int blocks_per_sm = 0;  // resident blocks per SM (0: the occupancy maximum)
  int grid_cap = 0;       // total blocks at most (0: no cap)
};
// Walkers per thread a two-state kernel of n modes can take (1 or 2), and the
// default when none is set.
// (n = 65..100 modes: the split kernel with two walkers per thread.)
inline int max_wpt(int n) { return (n <= 8 || (n > 64 && n <= 100)) ? 2 : 1; }
inline int default_wpt(int n) { return (n <= 4 || (n > 64 && n <= 100)) ? 2 : 1; }

void launch_sample_f32(const DevModel& host, const SampleParams& sp, void* buf, cudaStream_t st);
// Returns the persistent grid size used (0 on launch failure).
int launch_bulk2(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                 const LaunchShape& ls, cudaStream_t st);
// The split kernels (two states, 33..256 modes, a walker's modes over 2 or 4
// warps; two walkers per thread for 65..100 modes).
int launch_bulk2_split(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                       const LaunchShape& ls, cudaStream_t st);
// The diabatic-representation bulk kernel (two states, n <= 32 modes).
int launch_bulk2_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                     const LaunchShape& ls, cudaStream_t st);
// Launches a persistent bulk kernel whose blocks take `wpt` tiles at a time:
// one wave of ls.blocks_per_sm (at most the occupancy limit) blocks per SM,
// capped by ls.grid_cap and by the tile count; per_sm / n_sm cache the
// occupancy query.
using BulkFn = void (*)(const BulkParams, const Coef2, void*, double*);
// The split kernel a launch of (n modes, kind, walkers per thread) uses.
BulkFn bulk2_split_fn(int n, int kind, int wpt);
// Walkers per thread actually launched when two are asked for: 2 only if the
// tiles outnumber the resident block slots of the two-walker kernel fn2 (at
// ls.blocks_per_sm and ls.grid_cap); a smaller ensemble runs one walker per
// thread so that every slot gets a tile.  Results do not depend on it.
int bulk_wpt(BulkFn fn2, int& per_sm, int& n_sm, int64_t n_tiles, const LaunchShape& ls);
int run_bulk_kernel(BulkFn fn, int& per_sm, int& n_sm, const BulkParams& bp, const Coef2& cf,
                    void* buf, double* part, const LaunchShape& ls, int wpt, cudaStream_t st);
// Occupancy limit (resident blocks per SM) of the two-state bulk kernel that
// a launch of (n, kind, repr, wpt) would use; 0 if there is none.
int bulk2_blocks_per_sm(int n, int kind, int repr, int wpt);
// Kernel-selection description of the bulk kernel chosen for (n, kind).
const char* bulk2_variant(int n, int kind);

// N_s-state initial sample: FP64 (dm, sp) or FP32 bulk (s32).
void launch_sampleN(const DevModel* dm, const SampleParams& sp, const SampleN32* s32, void* buf,
                    int precision, cudaStream_t st);
void launch_stepN_f64(const DevModel* dm, int repr, int ns, void* buf, int64_t nt, int n,
                      int64_t step0, int64_t step, double dt, uint64_t seed, uint64_t traj_off,
                      cudaStream_t st);
void launch_observeN_f64(const DevModel* dm, int ns, const void* buf, int64_t nt, int n,
                         double* part, cudaStream_t st);
int launch_bulkN(int ns, const BulkParams& bp, const CoefN& cf, void* buf, double* part,
                 const LaunchShape& ls, cudaStream_t st);

// Folds n_slots output times of per-tile partials into rows; with chunk_out
// (rows of [n_slots][ceil(n_tiles / 1024)][q2]) the first level's 1024-tile
// block sums are kept there when there is more than one block.
void launch_fold(const double* part, double* rows_out, double* scratch, int64_t n_tiles,
                 int q2, int n_slots, cudaStream_t st, double* chunk_out = nullptr);
void launch_finalize(const double* rows, double* fin, int nq, int64_t k0, int64_t nrows,
                     int64_t n_traj, int ns, cudaStream_t st);
void launch_header_finish(void* buf, int64_t step0, int64_t step1, cudaStream_t st);
// Writes a whole ensemble header (checkpoint restore).
void launch_header_set(void* buf, const EnsHeader& v, cudaStream_t st);

}  // namespace qcl
