// spawn.cu -- trajectory spawning on the GPU (FP64, two states; N_s > 2 in
// nstate_f64.cuh, and the scan and family starts here serve both): the scheme of
// the CPU code that the paper's GPU version replaces (Sec. II B).  Every step a
// walker whose transition test fires keeps its pair and weight and spawns a
// child at the event's target pair with weight m A_e / p_hat_e (no stay
// factor).  Children are inserted right after their parents by a
// deterministic count / scan / scatter, so the walker order -- and with it
// every result -- is reproducible bit for bit, and each initial walker's
// descendants (its family) stay contiguous.  Observables sum each family
// before squaring, so standard errors count independent families.
#include "f64_2state.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace qcl {

namespace {

struct Set64 {
  double* R;
  double* P;
  double* m;
  double* phi;
  uint16_t* ab;
  uint64_t* id;
  uint32_t* fam;
};

__device__ __forceinline__ Set64 spawn_set(void* buf, const SpawnLayout& L, int set) {
  char* b = (char*)buf + L.set_off[set];
  return {(double*)(b + L.R),    (double*)(b + L.P),    (double*)(b + L.m),
          (double*)(b + L.phi),  (uint16_t*)(b + L.ab), (uint64_t*)(b + L.id),
          (uint32_t*)(b + L.fam)};
}

__device__ __forceinline__ SpawnHeader* spawn_header(void* buf) {
  return (SpawnHeader*)((char*)buf + kSpawnHeaderOff);
}

// Random-stream id of the child spawned at `step` by the walker with id
// `parent`: words 0 and 1 of Philox block (c0 = step, parent, purpose SPAWN),
// bit 63 set (initial walkers have ids below 2^63).
constexpr uint32_t kPurposeSpawn = 3u;
__device__ __forceinline__ uint64_t child_id(uint64_t seed, int64_t step, uint64_t parent) {
  const u4 w = philox_draw(seed, (uint32_t)step, parent, kPurposeSpawn);
  return (((uint64_t)w.y << 32) | w.x) | (1ull << 63);
}

__global__ void __launch_bounds__(256) k_spawn_sample(const DevModel* __restrict__ M,
                                                      SampleParams sp, int64_t cap, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n0 = sp.n_traj;
  const SpawnLayout L = SpawnLayout::make(cap, sp.n, n0, QCL_PREC_FP64);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = spawn_header(buf);
  if (i == 0) {
    hdr->magic = kEnsMagic;
    hdr->n_traj = n0;
    hdr->precision = QCL_PREC_FP64;
    hdr->ns = 2;
    hdr->n = sp.n;
    hdr->step = 0;
    hdr->flags = 0;
    hdr->n_degenerate = 0;
    hdr->n_nonfinite = 0;
    sh->capacity = cap;
    sh->n0 = n0;
    sh->n_live[0] = n0;
    sh->n_live[1] = 0;
    sh->drop = 0;
  }
  if (i >= n0) return;
  const Set64 w = spawn_set(buf, L, 0);
  const uint64_t traj = sp.traj_offset + (uint64_t)i;
  uint16_t ab;
  sample_walker_f64(M, sp, traj, w.R + i, w.P + i, cap, w.m[i], ab);
  w.phi[i] = 0.0;
  w.ab[i] = ab;
  w.id[i] = traj;
  w.fam[i] = (uint32_t)i;
}

// Step of every live walker of set `src` (in place); the children's weights
// and pair words go to the per-parent staging arrays, each block's child count
// to bsum.
template <int NP, bool DIA>
__global__ void __launch_bounds__(256) k_spawn_step(const DevModel* __restrict__ M, void* buf,
                                                    int64_t cap, int n, int64_t n0, int64_t step0,
                                                    int64_t step, double dt, uint64_t seed) {
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP64);
  EnsHeader* hdr = (EnsHeader*)buf;
  const int src = (int)(step & 1);
  const int64_t n_live = spawn_header(buf)->n_live[src];
  const bool ok = hdr->step == step0;
  if (!ok) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  // a grid of a few blocks per SM walks the live walkers in groups of 256
  const int64_t nvb = (n_live + 255) / 256;
  for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const int64_t i = vb * 256 + threadIdx.x;
    int flag = 0;
    if (i < n_live) {
      const Set64 w = spawn_set(buf, L, src);
      const uint16_t ab = w.ab[i];
      const int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
      double phi = w.phi[i];
      const double m = w.m[i];
      const Step64 o = walker_step_f64<NP, DIA>(M, w.R + i, w.P + i, cap, n, al, be, phi, dt,
                                                seed, w.id[i], step);
      w.phi[i] = phi;
      flag = o.ev > 0;
      double* cm = (double*)((char*)buf + L.cm);
      uint16_t* cab = (uint16_t*)((char*)buf + L.cab);
      uint8_t* fl = (uint8_t*)((char*)buf + L.flag);
      fl[i] = (uint8_t)flag;
      if (flag) {
        const double mc = m * o.num / o.den;
        cm[i] = mc;
        cab[i] = (uint16_t)((al ^ (o.ev == 1)) | (((q + o.dq) & 3) << 4) | ((be ^ (o.ev == 2)) << 8));
        if (!isfinite(mc)) {
          atomicAdd(&hdr->n_nonfinite, 1ull);
          atomicOr(&hdr->flags, QCL_FLAG_NONFINITE);
        }
      }
      if (o.deg) {
        atomicAdd(&hdr->n_degenerate, 1ull);
        atomicOr(&hdr->flags, QCL_FLAG_DEGENERATE);
      }
      if (!isfinite(phi)) {
        atomicAdd(&hdr->n_nonfinite, 1ull);
        atomicOr(&hdr->flags, QCL_FLAG_NONFINITE);
      }
    }
    const int cnt = __syncthreads_count(flag);
    if (threadIdx.x == 0) ((int32_t*)((char*)buf + L.bsum))[vb] = cnt;
  }
}

// Exclusive scan of the block counts of the live blocks (one block of 1024
// threads, each over a contiguous run of blocks), the destination set's live
// count, and the overflow test.
__global__ void __launch_bounds__(1024) k_spawn_scan(void* buf, int64_t cap, int n, int64_t n0,
                                                     int prec, int ns, int64_t step0,
                                                     int64_t step) {
  __shared__ int64_t wsum[32];
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, prec, ns);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = spawn_header(buf);
  if (hdr->step != step0) return;
  const int src = (int)(step & 1);
  const int64_t n_live = sh->n_live[src];
  const int64_t nb = (n_live + 255) / 256;
  const int32_t* bsum = (const int32_t*)((char*)buf + L.bsum);
  int64_t* boff = (int64_t*)((char*)buf + L.boff);
  const int t = threadIdx.x;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b0 = (int64_t)t * per, b1 = min(b0 + per, nb);
  int64_t local = 0;
  for (int64_t b = b0; b < b1; ++b) local += bsum[b];
  // block-wide exclusive scan of the 1024 thread totals
  const int lane = t & 31, wid = t >> 5;
  int64_t x = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t z = wsum[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, z, off);
      if (lane >= off) z += y;
    }
    wsum[lane] = z;  // inclusive over warps
  }
  __syncthreads();
  int64_t run = x - local + (wid > 0 ? wsum[wid - 1] : 0);  // exclusive start of this thread
  for (int64_t b = b0; b < b1; ++b) {
    boff[b] = run;
    run += bsum[b];
  }
  if (t == 1023) {
    const int64_t total = wsum[31];
    const int drop = n_live + total > cap;
    sh->drop = drop;
    sh->n_live[src ^ 1] = drop ? n_live : n_live + total;
    if (drop) atomicOr(&hdr->flags, QCL_FLAG_SPAWN_OVERFLOW);
  }
}

// Moves every live walker of set src to its place in the other set (after the
// children of the walkers before it) and writes each child right after its
// parent.
__global__ void __launch_bounds__(256) k_spawn_scatter(void* buf, int64_t cap, int n, int64_t n0,
                                                       int64_t step0, int64_t step,
                                                       uint64_t seed) {
  __shared__ int wcnt[8];
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP64);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = spawn_header(buf);
  if (hdr->step != step0) return;  // uniform over the grid
  const int src = (int)(step & 1);
  const int64_t n_live = sh->n_live[src];
  const bool drop = sh->drop != 0;
  const uint8_t* fl = (const uint8_t*)((char*)buf + L.flag);
  const int64_t nvb = (n_live + 255) / 256;
  for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const int64_t i = vb * 256 + threadIdx.x;
    const bool live = i < n_live;
    const int flag = (live && !drop) ? fl[i] : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    int before = __popc(bal & ((1u << lane) - 1u));
    for (int k = 0; k < wid; ++k) before += wcnt[k];
    if (live) {
      const int64_t boff = drop ? 0 : ((const int64_t*)((char*)buf + L.boff))[vb];
      const int64_t pos = i + boff + before;
      const Set64 s = spawn_set(buf, L, src);
      const Set64 d = spawn_set(buf, L, src ^ 1);
      for (int j = 0; j < n; ++j) {
        const double r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
        d.R[(int64_t)j * cap + pos] = r;
        d.P[(int64_t)j * cap + pos] = p;
        if (flag) {
          d.R[(int64_t)j * cap + pos + 1] = r;
          d.P[(int64_t)j * cap + pos + 1] = p;
        }
      }
      const double phi = s.phi[i];
      const uint64_t id = s.id[i];
      const uint32_t fam = s.fam[i];
      d.m[pos] = s.m[i];
      d.phi[pos] = phi;
      d.ab[pos] = s.ab[i];
      d.id[pos] = id;
      d.fam[pos] = fam;
      if (flag) {
        d.m[pos + 1] = ((const double*)((char*)buf + L.cm))[i];
        d.phi[pos + 1] = phi;
        d.ab[pos + 1] = ((const uint16_t*)((char*)buf + L.cab))[i];
        d.id[pos + 1] = child_id(seed, step, id);
        d.fam[pos + 1] = fam;
      }
    }
    __syncthreads();  // wcnt is rewritten by the next group
  }
}

// Family start indices of set `set`: fstart[k] = index of family k's first
// walker, fstart[n0] = the live count.
__global__ void __launch_bounds__(256) k_spawn_fstart(const void* buf, int64_t cap, int n,
                                                      int64_t n0, int prec, int ns, int set) {
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, prec, ns);
  const int64_t n_live = spawn_header((void*)buf)->n_live[set];
  const uint32_t* fam = (const uint32_t*)((const char*)buf + L.set_off[set] + L.fam);
  int64_t* fstart = (int64_t*)((char*)buf + L.fstart);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_live;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t f = fam[i];
    if (i == 0 || fam[i - 1] != f) fstart[f] = i;
    if (i == n_live - 1) fstart[n0] = n_live;
  }
}

// One thread per family: the family sum X of the walkers' contributions (in
// walker order), then X and X^2 reduced over the tile's 256 families by the
// fixed tree of the observation kernel.
__global__ void __launch_bounds__(256) k_spawn_observe(const DevModel* __restrict__ M,
                                                       const void* buf, int64_t cap, int n,
                                                       int64_t n0, int set,
                                                       double* __restrict__ part) {
  __shared__ double red[8][32];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP64);
  const Set64 s = spawn_set((void*)buf, L, set);
  const int64_t* fstart = (const int64_t*)((const char*)buf + L.fstart);
  double v[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = 0.0;
  if (k < n0) {
    const int64_t j0 = fstart[k], j1 = fstart[k + 1];
    for (int64_t j = j0; j < j1; ++j) {
      double c[32];
      contrib_f64(M, s.R + j, cap, n, s.m[j], s.phi[j], s.ab[j], c);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] += c[q];
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) v[16 + q] = v[q] * v[q];
  }
  const double x = warp_transpose_sum<double>(v);
  red[threadIdx.x >> 5][threadIdx.x & 31] = x;
  __syncthreads();
  if (threadIdx.x < 32)
    part[(int64_t)blockIdx.x * 32 + threadIdx.x] = tile_tree8(&red[0][0], 32, threadIdx.x);
}

}  // namespace

unsigned spawn_grid(int64_t capacity) {
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm < 1) n_sm = 1;
  }
  const int64_t groups = (capacity + 255) / 256;
  const int64_t g = (int64_t)8 * n_sm;
  return (unsigned)(groups < g ? (groups > 0 ? groups : 1) : g);
}

void launch_spawn_sample(const DevModel* dm, const SampleParams& sp, int64_t capacity, void* buf,
                         cudaStream_t st) {
  const int64_t nb = (sp.n_traj + 255) / 256;
  k_spawn_sample<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, st>>>(dm, sp, capacity, buf);
  launches_add(1);
}

void launch_spawn_step(const DevModel* dm, int repr, void* buf, int64_t capacity, int n,
                       int64_t n0, int64_t step0, int64_t step, double dt, uint64_t seed,
                       cudaStream_t st) {
  const unsigned nb = spawn_grid(capacity);
  const bool dia = repr == QCL_REPR_DIABATIC;
#define QCL_SPAWN_STEP(NP)                                                                   \
  (dia ? k_spawn_step<NP, true><<<nb, 256, 0, st>>>(dm, buf, capacity, n, n0, step0, step, dt, seed) \
       : k_spawn_step<NP, false><<<nb, 256, 0, st>>>(dm, buf, capacity, n, n0, step0, step, dt, seed))
  if (n <= 1)
    QCL_SPAWN_STEP(1);
  else if (n <= 4)
    QCL_SPAWN_STEP(4);
  else if (n <= 16)
    QCL_SPAWN_STEP(16);
  else
    QCL_SPAWN_STEP(0);
#undef QCL_SPAWN_STEP
  k_spawn_scan<<<1, 1024, 0, st>>>(buf, capacity, n, n0, QCL_PREC_FP64, 2, step0, step);
  k_spawn_scatter<<<nb, 256, 0, st>>>(buf, capacity, n, n0, step0, step, seed);
  launches_add(3);
}

void launch_spawn_observe(const DevModel* dm, const void* buf, int64_t capacity, int n, int64_t n0,
                          int set, double* part, cudaStream_t st) {
  const unsigned nf = (unsigned)((n0 + 255) / 256);
  k_spawn_fstart<<<spawn_grid(capacity), 256, 0, st>>>(buf, capacity, n, n0, QCL_PREC_FP64, 2, set);
  k_spawn_observe<<<nf, 256, 0, st>>>(dm, buf, capacity, n, n0, set, part);
  launches_add(2);
}

void launch_spawn_scan(void* buf, int64_t capacity, int n, int64_t n0, int precision, int ns,
                       int64_t step0, int64_t step, cudaStream_t st) {
  k_spawn_scan<<<1, 1024, 0, st>>>(buf, capacity, n, n0, precision, ns, step0, step);
  launches_add(1);
}

void launch_spawn_fstart(const void* buf, int64_t capacity, int n, int64_t n0, int precision, int ns,
                         int set, cudaStream_t st) {
  k_spawn_fstart<<<spawn_grid(capacity), 256, 0, st>>>(buf, capacity, n, n0, precision, ns, set);
  launches_add(1);
}

}  // namespace qcl
