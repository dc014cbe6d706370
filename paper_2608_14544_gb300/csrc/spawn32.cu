// spawn32.cu -- trajectory spawning in FP32 bulk precision (two states, any
// mode count, either representation).  The same scheme and walker order as the
// FP64 spawning kernels (spawn.cu): one step per launch, a child inserted right
// after its parent by the deterministic count / scan / scatter; the walker's
// arithmetic is that of the FP32-bulk kernels (compensated phase and weight
// pairs with a carried exponent), with the state read from and written to HBM
// every step.  Family observation in FP64 from the walkers' FP32 contributions.
#include "bulk2.cuh"
#include "model.h"
#include "reduce.cuh"

namespace qcl {

namespace {

struct Set32 {
  float* R;
  float* P;
  float* mh;
  float* ml;
  int32_t* me;
  float* ph;
  float* pl;
  uint16_t* ab;
  uint64_t* id;
  uint32_t* fam;
};

__device__ __forceinline__ Set32 set32(void* buf, const SpawnLayout& L, int set) {
  char* b = (char*)buf + L.set_off[set];
  return {(float*)(b + L.R),     (float*)(b + L.P),    (float*)(b + L.m),
          (float*)(b + L.mlo),   (int32_t*)(b + L.mexp), (float*)(b + L.phi),
          (float*)(b + L.philo), (uint16_t*)(b + L.ab), (uint64_t*)(b + L.id),
          (uint32_t*)(b + L.fam)};
}

__device__ __forceinline__ SpawnHeader* hdr_spawn(void* buf) {
  return (SpawnHeader*)((char*)buf + kSpawnHeaderOff);
}

// the child's random-stream id (the definition used by the FP64 kernels)
__device__ __forceinline__ uint64_t child_id32(uint64_t seed, int64_t step, uint64_t parent) {
  const u4 w = philox_draw(seed, (uint32_t)step, parent, 3u);
  return (((uint64_t)w.y << 32) | w.x) | (1ull << 63);
}

__global__ void __launch_bounds__(256) k_spawn_sample32(const Sample32 sp, int64_t cap, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n0 = sp.n_traj;
  const SpawnLayout L = SpawnLayout::make(cap, sp.n, n0, QCL_PREC_FP32_BULK);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = hdr_spawn(buf);
  if (i == 0) {
    hdr->magic = kEnsMagic;
    hdr->n_traj = n0;
    hdr->precision = QCL_PREC_FP32_BULK;
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
  const Set32 w = set32(buf, L, 0);
  const uint64_t traj = sp.traj_offset + (uint64_t)i;
  float mh;
  uint16_t ab;
  sample_walker_f32(sp, traj, w.R + i, w.P + i, cap, mh, ab);
  w.mh[i] = mh;
  w.ml[i] = 0.0f;
  w.me[i] = 0;
  w.ph[i] = 0.0f;
  w.pl[i] = 0.0f;
  w.ab[i] = ab;
  w.id[i] = traj;
  w.fam[i] = (uint32_t)i;
}

// One step of every live walker of set `src` (in place); children to the
// per-parent staging, each block's child count to bsum.
// NPL = 0: the modes stay in memory (any mode count), read and written back
// mode by mode with the register form's operations in its order (the same
// bits): one pass for the diabatic step, three for the adiabatic one (a(R_n),
// b(R_n); first half kick, drift, a and b at R_{n+1}; second half kick and the
// coupling sums).
template <int NPL, int KIND, bool DIA>
__global__ void __launch_bounds__(256) k_spawn_step32(const BulkParams bp, const Coef2 cf,
                                                      void* buf, int64_t cap, int64_t n0,
                                                      int64_t step) {
  constexpr bool MEM = NPL == 0;
  constexpr int NR = MEM ? 1 : NPL;
  const SpawnLayout L = SpawnLayout::make(cap, bp.n, n0, QCL_PREC_FP32_BULK);
  EnsHeader* hdr = (EnsHeader*)buf;
  const int src = (int)(step & 1);
  const int64_t n_live = hdr_spawn(buf)->n_live[src];
  const bool ok = hdr->step == bp.step0;
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
      const Set32 s = set32(buf, L, src);
      Walker<NR> w;
  #pragma unroll
      for (int j = 0; j < NPL; ++j) {
        const bool on = j < bp.n;
        w.R[j] = on ? s.R[(int64_t)j * cap + i] : 0.0f;
        w.P[j] = on ? s.P[(int64_t)j * cap + i] : 0.0f;
      }
      Scal z;
      z.m = {s.mh[i], s.ml[i]};
      z.mexp = s.me[i];
      z.ph = {s.ph[i], s.pl[i]};
      const uint32_t ab = s.ab[i];
      z.sa = sgn(ab & 0xf);
      z.sb = sgn((ab >> 8) & 0xf);
      z.q = DIA ? (int)((ab >> 4) & 3u) : 0;
      z.A = bp.a0;
      z.B = bp.b0;
      if constexpr (MEM) {
        for (int j = 0; j < bp.n; ++j) {
          const float r = s.R[(int64_t)j * cap + i];
          z.A = __fmaf_rn(cf.a[j], r, z.A);
          if (KIND == 1) z.B = __fmaf_rn(cf.b[j], r, z.B);
        }
      }
  #pragma unroll
      for (int j = 0; j < NPL; ++j) {
        z.A = __fmaf_rn(cf.a[j], w.R[j], z.A);
        if (KIND == 1) z.B = __fmaf_rn(cf.b[j], w.R[j], z.B);
      }
      closed_form(z);
      const u4 wd = philox_draw(bp.seed, (uint32_t)(step >> 2), s.id[i], kPurposeHop);
      const uint32_t word = word_of(wd, (int)(step & 3));
      unsigned int deg = 0;
      Scal child;
      bool hop;
      const float hsab = bp.hdt * 0.5f * (z.sa + z.sb);
      if constexpr (MEM) {
        // P += dt/2 F with the pair's force (kick / kick_dia of one mode)
        auto kick1 = [&](int j, float r, float p, float hu, float hv) {
          p = __fmaf_rn(-cf.hk[j], r, p);
          if (KIND == 1) p = __fadd_rn(p, -cf.hs[j]);
          if (DIA) return __fmaf_rn(hsab, cf.a[j], p);
          p = __fmaf_rn(hu, -cf.a[j], p);
          if (KIND == 1) p = __fmaf_rn(hv, -cf.b[j], p);
          return p;
        };
        if (DIA) {
          const float a_old = z.A;
          z.A = bp.a0;
          if (KIND == 1) z.B = bp.b0;
          for (int j = 0; j < bp.n; ++j) {
            float r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
            p = kick1(j, r, p, 0.0f, 0.0f);
            r = __fmaf_rn(cf.dtm[j], p, r);
            z.A = __fmaf_rn(cf.a[j], r, z.A);
            if (KIND == 1) z.B = __fmaf_rn(cf.b[j], r, z.B);
            s.R[(int64_t)j * cap + i] = r;
            s.P[(int64_t)j * cap + i] = kick1(j, r, p, 0.0f, 0.0f);
          }
          hop = spawn_transition<KIND, true>(z, a_old, 0.0f, z.B, word, bp, deg, child);
        } else {
          const float hu = hsab * z.c2, hv = hsab * z.s2;
          const float r_old = z.r;
          z.A = bp.a0;
          z.B = bp.b0;
          for (int j = 0; j < bp.n; ++j) {
            float r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
            p = kick1(j, r, p, hu, hv);
            r = __fmaf_rn(cf.dtm[j], p, r);
            z.A = __fmaf_rn(cf.a[j], r, z.A);
            if (KIND == 1) z.B = __fmaf_rn(cf.b[j], r, z.B);
            s.R[(int64_t)j * cap + i] = r;
            s.P[(int64_t)j * cap + i] = p;
          }
          closed_form(z);
          const float hu2 = hsab * z.c2, hv2 = hsab * z.s2;
          float Av = 0.0f, Bv = 0.0f;
          for (int j = 0; j < bp.n; ++j) {
            const float r = s.R[(int64_t)j * cap + i];
            const float p = kick1(j, r, s.P[(int64_t)j * cap + i], hu2, hv2);
            Av = __fmaf_rn(cf.am[j], p, Av);
            if (KIND == 1) Bv = __fmaf_rn(cf.bm[j], p, Bv);
            s.P[(int64_t)j * cap + i] = p;
          }
          hop = spawn_transition<KIND, false>(z, r_old, Av, Bv, word, bp, deg, child);
        }
      } else if (DIA) {
        kick_dia<NPL, KIND, Coef2>(w, cf, hsab);
  #pragma unroll
        for (int j = 0; j < NPL; ++j) w.R[j] = __fmaf_rn(cf.dtm[j], w.P[j], w.R[j]);
        const float a_old = z.A;
        z.A = bp.a0;
        if (KIND == 1) z.B = bp.b0;
  #pragma unroll
        for (int j = 0; j < NPL; ++j) {
          z.A = __fmaf_rn(cf.a[j], w.R[j], z.A);
          if (KIND == 1) z.B = __fmaf_rn(cf.b[j], w.R[j], z.B);
        }
        kick_dia<NPL, KIND, Coef2>(w, cf, hsab);
        hop = spawn_transition<KIND, true>(z, a_old, 0.0f, z.B, word, bp, deg, child);
      } else {
        kick<NPL, KIND, Coef2>(w, cf, hsab * z.c2, hsab * z.s2);
  #pragma unroll
        for (int j = 0; j < NPL; ++j) w.R[j] = __fmaf_rn(cf.dtm[j], w.P[j], w.R[j]);
        const float r_old = z.r;
        z.A = bp.a0;
        z.B = bp.b0;
  #pragma unroll
        for (int j = 0; j < NPL; ++j) {
          z.A = __fmaf_rn(cf.a[j], w.R[j], z.A);
          if (KIND == 1) z.B = __fmaf_rn(cf.b[j], w.R[j], z.B);
        }
        closed_form(z);
        kick<NPL, KIND, Coef2>(w, cf, hsab * z.c2, hsab * z.s2);
        float Av = 0.0f, Bv = 0.0f;
  #pragma unroll
        for (int j = 0; j < NPL; ++j) {
          Av = __fmaf_rn(cf.am[j], w.P[j], Av);
          if (KIND == 1) Bv = __fmaf_rn(cf.bm[j], w.P[j], Bv);
        }
        hop = spawn_transition<KIND, false>(z, r_old, Av, Bv, word, bp, deg, child);
      }
      // the phase pair is renormalised, and wrapped past 2^10 rad, at the end of
      // every Philox block (absolute steps 4k + 3)
      if ((step & 3) == 3) {
        z.ph = two_sum(z.ph.hi, z.ph.lo);
        phase_wrap(z);
      }
  #pragma unroll
      for (int j = 0; j < NPL; ++j)
        if (j < bp.n) {
          s.R[(int64_t)j * cap + i] = w.R[j];
          s.P[(int64_t)j * cap + i] = w.P[j];
        }
      s.ph[i] = z.ph.hi;
      s.pl[i] = z.ph.lo;
      flag = hop ? 1 : 0;
      uint8_t* fl = (uint8_t*)((char*)buf + L.flag);
      fl[i] = (uint8_t)flag;
      if (hop) {
        renorm(child.m, child.mexp);
        ((float*)((char*)buf + L.cm))[i] = child.m.hi;
        ((float*)((char*)buf + L.cmlo))[i] = child.m.lo;
        ((int32_t*)((char*)buf + L.cmexp))[i] = child.mexp;
        ((uint16_t*)((char*)buf + L.cab))[i] =
            (uint16_t)((child.sa > 0.0f ? 1 : 0) | (child.q << 4) | ((child.sb > 0.0f ? 1 : 0) << 8));
        if (!isfinite(child.m.hi)) {
          atomicAdd(&hdr->n_nonfinite, 1ull);
          atomicOr(&hdr->flags, QCL_FLAG_NONFINITE);
        }
      }
      if (deg) {
        atomicAdd(&hdr->n_degenerate, 1ull);
        atomicOr(&hdr->flags, QCL_FLAG_DEGENERATE);
      }
      if (!isfinite(z.ph.hi)) {
        atomicAdd(&hdr->n_nonfinite, 1ull);
        atomicOr(&hdr->flags, QCL_FLAG_NONFINITE);
      }
    }
    const int cnt = __syncthreads_count(flag);
    if (threadIdx.x == 0) ((int32_t*)((char*)buf + L.bsum))[vb] = cnt;
  }
}

// Moves every live walker of set src to its place in the other set and writes
// each child right after its parent.
__global__ void __launch_bounds__(256) k_spawn_scatter32(void* buf, int64_t cap, int n, int64_t n0,
                                                         int64_t step0, int64_t step,
                                                         uint64_t seed) {
  __shared__ int wcnt[8];
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP32_BULK);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = hdr_spawn(buf);
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
      const Set32 s = set32(buf, L, src);
      const Set32 d = set32(buf, L, src ^ 1);
      for (int j = 0; j < n; ++j) {
        const float r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
        d.R[(int64_t)j * cap + pos] = r;
        d.P[(int64_t)j * cap + pos] = p;
        if (flag) {
          d.R[(int64_t)j * cap + pos + 1] = r;
          d.P[(int64_t)j * cap + pos + 1] = p;
        }
      }
      const float ph = s.ph[i], pl = s.pl[i];
      const uint64_t id = s.id[i];
      const uint32_t fam = s.fam[i];
      d.mh[pos] = s.mh[i];
      d.ml[pos] = s.ml[i];
      d.me[pos] = s.me[i];
      d.ph[pos] = ph;
      d.pl[pos] = pl;
      d.ab[pos] = s.ab[i];
      d.id[pos] = id;
      d.fam[pos] = fam;
      if (flag) {
        d.mh[pos + 1] = ((const float*)((char*)buf + L.cm))[i];
        d.ml[pos + 1] = ((const float*)((char*)buf + L.cmlo))[i];
        d.me[pos + 1] = ((const int32_t*)((char*)buf + L.cmexp))[i];
        d.ph[pos + 1] = ph;
        d.pl[pos + 1] = pl;
        d.ab[pos + 1] = ((const uint16_t*)((char*)buf + L.cab))[i];
        d.id[pos + 1] = child_id32(seed, step, id);
        d.fam[pos + 1] = fam;
      }
    }
    __syncthreads();  // wcnt is rewritten by the next group
  }
}

// Family observation: for each family the sum X of its walkers' contributions
// and X^2.  A warp takes 32 families, one at a time: lane l takes the family's
// walkers l, l + 32, ... (coalesced loads; no lane idles on a small family while
// another walks a large one).  The family shares one power of two (its largest
// weight exponent), so each walker's contribution is an FP32 value, summed as a
// compensated FP32 pair per lane and then over the lanes by a reduce-scatter of
// pairs, which leaves lanes 2q and 2q + 1 with quantity q; X is rebuilt in FP64
// from the pair and the exponent exactly, and the even lane accumulates X, the
// odd lane X^2, over the warp's families in order.  (Accumulating every walker
// in FP64 kept the FP64 pipe 84 % busy: FP64 is slow on this part.)  The tile's
// 8 warps are then folded by the fixed tree of the observation kernels.
template <int KIND, bool DIA>
__global__ void __launch_bounds__(256) k_spawn_observe32(const BulkParams bp, const Coef2 cf,
                                                         const void* buf, int64_t cap, int64_t n0,
                                                         int set, double* __restrict__ part) {
  __shared__ double red[8][32];
  const SpawnLayout L = SpawnLayout::make(cap, bp.n, n0, QCL_PREC_FP32_BULK);
  const Set32 s = set32((void*)buf, L, set);
  const int64_t* fstart = (const int64_t*)((const char*)buf + L.fstart);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double T = 0.0;
  const int64_t f0 = (int64_t)blockIdx.x * 256 + warp * 32;
#pragma unroll 1
  for (int f = 0; f < 32; ++f) {
    const int64_t k = f0 + f;
    if (k >= n0) break;  // (warp-uniform)
    const int64_t j0 = fstart[k], j1 = fstart[k + 1];
    int em = -(1 << 28);
    for (int64_t j = j0 + lane; j < j1; j += 32)
      if (s.mh[j] != 0.0f) em = max(em, s.me[j]);
    em = __reduce_max_sync(0xffffffffu, em);
    f2 acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = {0.0f, 0.0f};
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      Scal z;
      z.A = bp.a0;
      z.B = bp.b0;
      for (int m = 0; m < bp.n; ++m) {
        const float r = s.R[(int64_t)m * cap + j];
        z.A = __fmaf_rn(cf.a[m], r, z.A);
        if (KIND == 1) z.B = __fmaf_rn(cf.b[m], r, z.B);
      }
      closed_form(z);
      const uint32_t ab = s.ab[j];
      z.sa = sgn(ab & 0xf);
      z.sb = sgn((ab >> 8) & 0xf);
      z.q = DIA ? (int)((ab >> 4) & 3u) : 0;
      z.ph = {s.ph[j], s.pl[j]};
      const float mh = s.mh[j];
      const float mm = mh == 0.0f ? 0.0f : (mh + s.ml[j]) * pow2i(s.me[j] - em);
      float c[16];
      contributions<DIA>(z, mm, c);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const f2 t = two_sum(acc[q].hi, c[q]);
        acc[q] = {t.hi, acc[q].lo + t.lo};
      }
    }
    // reduce-scatter of the pairs: at the step with offset `off`, the lane with
    // that bit set keeps the upper half of its values
#pragma unroll
    for (int lev = 0; lev < 4; ++lev) {
      const int half = 8 >> lev, off = 16 >> lev;
      const bool upper = (lane & off) != 0;
#pragma unroll
      for (int i2 = 0; i2 < half; ++i2) {
        const f2 snd = upper ? acc[i2] : acc[half + i2];
        const f2 kp = upper ? acc[half + i2] : acc[i2];
        const float rh = __shfl_xor_sync(0xffffffffu, snd.hi, off);
        const float rl = __shfl_xor_sync(0xffffffffu, snd.lo, off);
        const f2 t = two_sum(kp.hi, rh);
        acc[i2] = {t.hi, t.lo + (kp.lo + rl)};
      }
    }
    const float rh = __shfl_xor_sync(0xffffffffu, acc[0].hi, 1);
    const float rl = __shfl_xor_sync(0xffffffffu, acc[0].lo, 1);
    const f2 t = two_sum(acc[0].hi, rh);
    const int ex = (em < -(1 << 27)) ? 0 : em;
    const double X = scaled_double(t.hi, ex) + scaled_double(t.lo + (acc[0].lo + rl), ex);
    T = (lane & 1) ? fma(X, X, T) : T + X;
  }
  red[warp][(lane & 1) ? 16 + (lane >> 1) : (lane >> 1)] = T;
  __syncthreads();
  if (threadIdx.x < 32)
    part[(int64_t)blockIdx.x * 32 + threadIdx.x] = tile_tree8(&red[0][0], 32, threadIdx.x);
}

template <int NPL, int KIND, bool DIA>
void run_step32(const BulkParams& bp, const Coef2& cf, void* buf, int64_t cap, int64_t n0,
                int64_t step, cudaStream_t st) {
  k_spawn_step32<NPL, KIND, DIA><<<spawn_grid(cap), 256, 0, st>>>(bp, cf, buf, cap, n0, step);
}

// in registers up to 32 modes, beyond that (or under QCL_OPT_MODES_IN_MEMORY = 1)
// in memory
template <int KIND, bool DIA>
int dispatch_step32(const BulkParams& bp, const Coef2& cf, void* buf, int64_t cap, int64_t n0,
                    int64_t step, cudaStream_t st) {
  const int n = bp.n;
  if (n > 32 || option_modes_in_memory() == 1) run_step32<0, KIND, DIA>(bp, cf, buf, cap, n0, step, st);
  else if (n <= 1) run_step32<1, KIND, DIA>(bp, cf, buf, cap, n0, step, st);
  else if (n <= 2) run_step32<2, KIND, DIA>(bp, cf, buf, cap, n0, step, st);
  else if (n <= 4) run_step32<4, KIND, DIA>(bp, cf, buf, cap, n0, step, st);
  else if (n <= 8) run_step32<8, KIND, DIA>(bp, cf, buf, cap, n0, step, st);
  else if (n <= 16) run_step32<16, KIND, DIA>(bp, cf, buf, cap, n0, step, st);
  else run_step32<32, KIND, DIA>(bp, cf, buf, cap, n0, step, st);
  return 1;
}

}  // namespace

void launch_spawn_sample32(const DevModel& host, const SampleParams& sp, int64_t capacity, void* buf,
                           cudaStream_t st) {
  const int64_t nb = (sp.n_traj + 255) / 256;
  Sample32 s32;
  make_sample32(host, sp, s32);
  k_spawn_sample32<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, st>>>(s32, capacity, buf);
  launches_add(1);
}

int launch_spawn_step32(const BulkParams& bp, const Coef2& cf, void* buf, int64_t capacity,
                        int64_t n0, int64_t step0, int64_t step, cudaStream_t st) {
  const bool dia = bp.repr == QCL_REPR_DIABATIC;
  const int ok = dia ? (bp.kind == 0 ? dispatch_step32<0, true>(bp, cf, buf, capacity, n0, step, st)
                                     : dispatch_step32<1, true>(bp, cf, buf, capacity, n0, step, st))
                     : (bp.kind == 0 ? dispatch_step32<0, false>(bp, cf, buf, capacity, n0, step, st)
                                     : dispatch_step32<1, false>(bp, cf, buf, capacity, n0, step, st));
  if (!ok) return 0;
  launch_spawn_scan(buf, capacity, bp.n, n0, QCL_PREC_FP32_BULK, 2, step0, step, st);
  k_spawn_scatter32<<<spawn_grid(capacity), 256, 0, st>>>(buf, capacity, bp.n, n0, step0, step, bp.seed);
  launches_add(2);
  return 1;
}

void launch_spawn_observe32(const BulkParams& bp, const Coef2& cf, const void* buf, int64_t capacity,
                            int64_t n0, int set, double* part, cudaStream_t st) {
  launch_spawn_fstart(buf, capacity, bp.n, n0, QCL_PREC_FP32_BULK, 2, set, st);
  const unsigned nf = (unsigned)((n0 + 255) / 256);
  const bool dia = bp.repr == QCL_REPR_DIABATIC;
  if (dia)
    (bp.kind == 0 ? k_spawn_observe32<0, true> : k_spawn_observe32<1, true>)
        <<<nf, 256, 0, st>>>(bp, cf, buf, capacity, n0, set, part);
  else
    (bp.kind == 0 ? k_spawn_observe32<0, false> : k_spawn_observe32<1, false>)
        <<<nf, 256, 0, st>>>(bp, cf, buf, capacity, n0, set, part);
  launches_add(1);
}

}  // namespace qcl
