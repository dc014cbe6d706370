// kernels_f32.cu -- FP32-bulk path: a persistent kernel in which each thread
// owns one walker for a whole chunk of steps with its state in registers.
// Verlet, forces and couplings run in FP32; the phase and the weight are
// carried as compensated FP32 pairs (about 46 significant bits) so that no
// FP64 instruction sits in the step loop; observations are reduced per tile in
// FP64.  Random numbers: one Philox4x32-10 call per four steps.
#include <atomic>
#include <cstdio>

#include "kernels.h"
#include "reduce.cuh"

namespace qcl {

namespace {

// 2 pi = C1 + C2 + C3 with C1, C2 of 14 significant bits (k * C exact for |k| < 2^10)
constexpr float kTwoPi1 = 6.283203125f;
constexpr float kTwoPi2 = -1.7818063497543335e-05f;
constexpr float kTwoPi3 = 2.430840251310684e-10f;
constexpr float kInvTwoPi = 0.15915494309189535f;
constexpr float kDegTol32 = 1e-6f;  // |e_b - e_a| below this: coupling set to 0

struct W32 {
  float* R;
  float* P;
  float* mh;
  float* ml;
  int32_t* me;
  float* ph;
  float* pl;
  uint16_t* ab;
  EnsHeader* hdr;
};

__device__ __forceinline__ W32 view32(void* buf, int64_t nt, int ns, int n) {
  const EnsLayout L = EnsLayout::make(nt, ns, n, QCL_PREC_FP32_BULK);
  char* b = (char*)buf;
  return {(float*)(b + L.off_R),    (float*)(b + L.off_P),     (float*)(b + L.off_m),
          (float*)(b + L.off_mlo),  (int32_t*)(b + L.off_mexp), (float*)(b + L.off_phi),
          (float*)(b + L.off_philo), (uint16_t*)(b + L.off_ab),  (EnsHeader*)b};
}

__device__ __forceinline__ float sgn(int idx) { return idx ? 1.0f : -1.0f; }

// Unbiased exponent of a float (normal numbers), -127 for zero/denormals.
__device__ __forceinline__ int fexp(float x) {
  return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127;
}

// 2^d for -126 <= d <= 127 (0 below)
__device__ __forceinline__ float pow2i(int d) {
  return d < -126 ? 0.0f : __uint_as_float((uint32_t)(127 + d) << 23);
}

// The weight is carried as (hi + lo) * 2^e: move hi's exponent into e so that
// hi stays in [1, 2) and the FP32 range never limits the weight.
__device__ __forceinline__ void renorm(f2& m, int& e) {
  if (m.hi == 0.0f) return;
  const int k = fexp(m.hi);
  const float sc = (k == -127) ? 0x1p+126f : (k >= 127 ? 0x1p-127f : pow2i(-k));
  m.hi *= sc;
  m.lo *= sc;
  e += (k == -127) ? -126 : k;
}

}  // namespace

// ---------------------------------------------------------------- sampling --
// FP32 initial sample from the same Philox words as the FP64 path.
__global__ void __launch_bounds__(256) k_sample_f32(const DevModel* __restrict__ M,
                                                    SampleParams sp, void* buf) {
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
  const uint64_t traj = sp.traj_offset + (uint64_t)i;
  float a = (float)M->a0, b = (float)M->b0;
  for (int j = 0; j < n; ++j) {
    float R = (float)sp.R0[j], P = (float)sp.P0[j];
    if (sp.wigner) {
      const u4 wd = philox_draw(sp.seed, (uint32_t)j, traj, kPurposeInit);
      const float u0 = __fmaf_rn(__uint2float_rn(wd.x), 0x1p-32f, 0x1p-33f);
      const float u1 = __fmaf_rn(__uint2float_rn(wd.y), 0x1p-32f, 0x1p-33f);
      const float rad = sqrtf(-2.0f * logf(u0));
      float sn, cs;
      sincospif(2.0f * u1, &sn, &cs);
      R = __fmaf_rn((float)sp.sR[j] * rad, cs, R);
      P = __fmaf_rn((float)sp.sP[j] * rad, sn, P);
    }
    w.R[(int64_t)j * nt + i] = R;
    w.P[(int64_t)j * nt + i] = P;
    a = __fmaf_rn((float)M->a[j], R, a);
    b = __fmaf_rn((float)M->b[j], R, b);
  }
  const float r2 = a * a + b * b;
  float c = 1.0f, s = 0.0f;
  if (r2 > 0.0f) {
    const float ir = rsqrtf(r2);
    const float c2 = a * ir, s2 = b * ir;
    if (a >= 0.0f) {
      c = sqrtf(0.5f + 0.5f * c2);
      s = 0.5f * s2 / c;
    } else {
      s = copysignf(sqrtf(0.5f - 0.5f * c2), b);
      c = 0.5f * s2 / s;
    }
  }
  const float U[4] = {-s, c, c, s};
  double rho_ad[4];
  double tot = 0.0;
  for (int al = 0; al < 2; ++al)
    for (int be = 0; be < 2; ++be) {
      float acc = 0.0f;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l)
          acc = __fmaf_rn(U[k * 2 + al] * (float)sp.rho[k * 2 + l], U[l * 2 + be], acc);
      rho_ad[al * 2 + be] = acc;
      tot += fabsf(acc);
    }
  // index pair from |rho_ad| with 2^-24 quantised probabilities (remainder to the
  // last nonzero pair), m0 = rho_ad / p_hat
  uint32_t Tk[4];
  uint32_t sumT = 0;
  int last = 0;
  for (int k = 0; k < 4; ++k) {
    Tk[k] = (uint32_t)floorf((float)(fabs(rho_ad[k]) / tot) * kP24f);
    sumT += Tk[k];
    if (rho_ad[k] != 0.0) last = k;
  }
  Tk[last] += 16777216u - sumT;
  const u4 wd = philox_draw(sp.seed, (uint32_t)n, traj, kPurposeInit);
  const uint32_t y = wd.x >> 8;
  uint32_t cum = 0;
  int pick = last;
  for (int k = 0; k < 4; ++k) {
    cum += Tk[k];
    if (y < cum) {
      pick = k;
      break;
    }
  }
  w.mh[i] = (float)rho_ad[pick] * (kP24f / (float)Tk[pick]);
  w.ml[i] = 0.0f;
  w.me[i] = 0;
  w.ph[i] = 0.0f;
  w.pl[i] = 0.0f;
  w.ab[i] = (uint16_t)((pick >> 1) | ((pick & 1) << 8));
}

// ------------------------------------------------------- persistent step --
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Sum of 32 floats at stride 33 (one column of a warp's rows) by a fixed
// pairwise tree: ((x0 + x1) + (x2 + x3)) + ...
__device__ __forceinline__ float column_sum32(const float* col) {
  float l1[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) l1[t] = col[(2 * t) * 33] + col[(2 * t + 1) * 33];
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int t = 0; t < w; ++t) l1[t] = l1[2 * t] + l1[2 * t + 1];
  return l1[0];
}

// 2^e as a double, -1022 <= e <= 1023
__device__ __forceinline__ double pow2d(int e) { return __hiloint2double((e + 1023) << 20, 0); }

// Shared-memory float4 load that the compiler may not hoist out of the step
// loop (hoisting the per-mode coefficients would hold them all in registers).
__device__ __forceinline__ float4 lds4(const float4* p) {
  float4 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}

// Scalar state of one walker that every lane holding a part of it keeps
// identical: weight (compensated pair and exponent), phase (compensated pair),
// the pair's sigmas, and the closed-form decomposition at the current R.
struct Scal {
  f2 m;
  int mexp;
  f2 ph;
  float sa, sb;          // sigma of the index pair: -1 lower, +1 upper adiabatic state
  float A, B;            // a(R), b(R)
  float r2, ir, r;       // r^2, 1/r, r
  float c2, s2;          // cos 2theta, sin 2theta (theta = 0 at r = 0)
};

__device__ __forceinline__ void closed_form(Scal& z) {
  z.r2 = __fmaf_rn(z.A, z.A, z.B * z.B);
  z.ir = rsqrtf(z.r2);
  z.r = z.r2 * z.ir;
  z.c2 = z.r2 > 0.0f ? z.A * z.ir : 1.0f;
  z.s2 = z.r2 > 0.0f ? z.B * z.ir : 0.0f;
}

// Phase (trapezoid) and transition of one step, given the decomposition at
// R_{n+1} (in z), r at R_n, and the coupling sums Av = sum a_j P_j/M_j,
// Bv = sum b_j P_j/M_j at P_{n+1}.
__device__ __forceinline__ void phase_and_transition(Scal& z, float r_old, float Av, float Bv,
                                                     uint32_t word, const BulkParams& bp,
                                                     bool active, unsigned int& n_deg) {
  // phase: dt/2 (w_ab(R_n) + w_ab(R_{n+1})), hbar w_ab = (sig_a - sig_b) r
  z.ph = df_add(z.ph, bp.hdt_hbar * (z.sa - z.sb) * (r_old + z.r));
  // coupling contracted with P/M: g = (a Bv - b Av) / (2 r^2)
  const bool degen = 2.0f * z.r < kDegTol32;
  n_deg += (degen && active) ? 1u : 0u;
  const float g = degen ? 0.0f : (z.A * Bv - z.B * Av) * (0.5f * z.ir * z.ir);
  // both events have |A_e| = dt |g|: p = min(kappa dt |g|, p_max) quantised to
  // 24-bit thresholds, scaled down together in integers when 2T > Tmax
  uint32_t T = min(__float2uint_rz(fminf(bp.kdt * fabsf(g) * kP24f, 33554432.0f)), bp.tmax);
  if (2u * T > bp.tmax) T = bp.tmax >> 1;
  const uint32_t y = word >> 8;
  const bool hop1 = y < T;
  const bool hop2 = !hop1 && (y < 2u * T);
  // weight factor: A_e / p_hat on a hop (A_1 = -sig_a dt g, A_2 = -sig_b dt g),
  // 1 / (1 - sum p_hat) otherwise; num / den as a compensated quotient
  const float dtg = bp.dt * g * kP24f;
  const float num = hop1 ? -z.sa * dtg : (hop2 ? -z.sb * dtg : kP24f);
  const float den = __uint2float_rn((hop1 || hop2) ? T : 16777216u - 2u * T);
  const float rd = rcp_approx(den);
  const float q0 = num * rd;
  const float q1 = __fmaf_rn(-q0, den, num) * rd;
  z.m = df_mul(z.m, q0, q1);
  if (!(fabsf(z.m.hi) <= 0x1p32f && fabsf(z.m.hi) >= 0x1p-32f)) renorm(z.m, z.mexp);
  z.sa = hop1 ? -z.sa : z.sa;
  z.sb = hop2 ? -z.sb : z.sb;
}

// The walker's 16 observable contributions (diabatic rho_ij and adiabatic
// rho_ab, real and imaginary) with weight mantissa `mm`; reduces the phase
// into [-pi, pi] as a side effect.
__device__ __forceinline__ void contributions(Scal& z, float mm, float (&v)[16]) {
  const float kq = rintf(z.ph.hi * kInvTwoPi);
  z.ph = df_add(z.ph, -kq * kTwoPi1);
  z.ph = df_add(z.ph, -kq * kTwoPi2);
  z.ph = df_add(z.ph, -kq * kTwoPi3);
  float sh, chh;
  __sincosf(z.ph.hi, &sh, &chh);
  const float cphi = __fmaf_rn(-z.ph.lo, sh, chh);
  const float sphi = __fmaf_rn(z.ph.lo, chh, sh);
  // eigenvector angle theta from (cos 2theta, sin 2theta), half-angle form
  // without cancellation: the larger of cos/sin is sqrt((1 + |cos2t|)/2)
  const float t = __fmaf_rn(0.5f, fabsf(z.c2), 0.5f);
  const float rt = rsqrtf(t);
  const float big = t * rt, small = 0.5f * fabsf(z.s2) * rt;
  const bool cpos = z.c2 >= 0.0f;
  const float c = cpos ? big : small;
  const float s = copysignf(cpos ? small : big, z.s2);
  const bool al = z.sa > 0.0f, be = z.sb > 0.0f;
  const float ua0 = al ? c : -s, ua1 = al ? s : c;  // column alpha of U
  const float ub0 = be ? c : -s, ub1 = be ? s : c;  // column beta of U
  const float zr = mm * cphi, zi = -mm * sphi;
  const float f00 = ua0 * ub0, f01 = ua0 * ub1, f10 = ua1 * ub0, f11 = ua1 * ub1;
  v[0] = zr * f00;
  v[1] = zi * f00;
  v[2] = zr * f01;
  v[3] = zi * f01;
  v[4] = zr * f10;
  v[5] = zi * f10;
  v[6] = zr * f11;
  v[7] = zi * f11;
  const int k = (al ? 2 : 0) + (be ? 1 : 0);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    v[8 + 2 * kk] = (kk == k) ? zr : 0.0f;
    v[9 + 2 * kk] = (kk == k) ? zi : 0.0f;
  }
}

__device__ __forceinline__ uint32_t pick_word(const u4& wd, int widx) {
  return (widx & 2) ? ((widx & 1) ? wd.w : wd.z) : ((widx & 1) ? wd.y : wd.x);
}

template <int NPL>
struct Walker {
  float R[NPL], P[NPL];
};

// P += dt/2 F_ab(R),  F_j = -k_j R_j - s_j - sab (a_j cos2t + b_j sin2t);
// hu = dt/2 sab cos2t, hv = dt/2 sab sin2t
template <int NPL, int KIND>
__device__ __forceinline__ void kick(Walker<NPL>& w, const Coef2& cf, float hu, float hv) {
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    float p = __fmaf_rn(-cf.hk[j], w.R[j], w.P[j]);
    if (KIND == 1) p -= cf.hs[j];
    p = __fmaf_rn(-hu, cf.a[j], p);
    if (KIND == 1) p = __fmaf_rn(-hv, cf.b[j], p);
    w.P[j] = p;
  }
}

// One thread per walker, all modes in registers, coefficients as constant-bank
// operands.  Tile = the block's 256 walkers.
template <int NPL, int KIND>
__global__ void __launch_bounds__(256, 3)
    k_bulk2(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
  __shared__ double red[2][8][32];      // double-buffered group partials
  __shared__ float obs_rows[256 * 33];  // per-walker contributions, padded rows
  W32 ws = view32(buf, bp.n_traj, 2, bp.n);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int n_deg = 0;
  int rb = 0;

  for (int64_t tile = blockIdx.x; tile < bp.n_tiles; tile += gridDim.x) {
    const int64_t i = tile * kTile + threadIdx.x;
    const bool active = i < nt;
    const int64_t ii = active ? i : 0;
    Walker<NPL> w;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const bool on = active && j < bp.n;
      w.R[j] = on ? ws.R[(int64_t)j * nt + ii] : 0.0f;
      w.P[j] = on ? ws.P[(int64_t)j * nt + ii] : 0.0f;
    }
    Scal z;
    z.m = {active ? ws.mh[ii] : 0.0f, active ? ws.ml[ii] : 0.0f};
    z.mexp = active ? ws.me[ii] : 0;
    z.ph = {active ? ws.ph[ii] : 0.0f, active ? ws.pl[ii] : 0.0f};
    const uint32_t ab = active ? ws.ab[ii] : 0u;
    z.sa = sgn(ab & 0xff);
    z.sb = sgn((ab >> 8) & 0xff);
    const uint64_t traj = bp.traj_offset + (uint64_t)ii;
    z.A = bp.a0;
    z.B = bp.b0;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      z.A = __fmaf_rn(cf.a[j], w.R[j], z.A);
      if (KIND == 1) z.B = __fmaf_rn(cf.b[j], w.R[j], z.B);
    }
    closed_form(z);

    // observation into slot `slot` of the tile partials: the warp's 32 walkers
    // share one power of two (FP32 sums of scaled weights, the exponent restored
    // exactly in FP64); each walker's 16 contributions and their squares go to
    // its padded row of shared memory and lane q sums column q of its warp's 32
    // rows by a fixed pairwise tree (conflict-free: row stride 33 words)
    auto observe = [&](int slot) {
      renorm(z.m, z.mexp);
      const bool live = active && z.m.hi != 0.0f;
      int ew = live ? z.mexp : -(1 << 28);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ew = max(ew, __shfl_xor_sync(0xffffffffu, ew, off));
      float v[16];
      contributions(z, live ? z.m.hi * pow2i(z.mexp - ew) : 0.0f, v);
      float* row = &obs_rows[threadIdx.x * 33];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        row[q] = v[q];
        row[16 + q] = v[q] * v[q];
      }
      __syncwarp();
      const float x = column_sum32(&obs_rows[(warp * 32) * 33 + lane]);
      __syncwarp();
      const int ex = (ew < -(1 << 27)) ? 0 : ((lane < 16) ? ew : 2 * ew);
      const double xd = (double)x;
      red[rb][warp][lane] = (ex >= -1022 && ex <= 1023) ? xd * pow2d(ex) : ldexp(xd, ex);
      __syncthreads();
      if (threadIdx.x < 32)
        part[((int64_t)slot * bp.n_tiles + tile) * 32 + threadIdx.x] =
            tile_tree8(&red[rb][0][0], 32, threadIdx.x);
      rb ^= 1;
    };

    int slot = bp.obs_first;
    if (bp.obs_first) observe(0);
    int to_out = bp.to_out0;
    uint32_t blk = bp.blk0;
    int widx = bp.widx0;
    u4 wd = philox_draw(bp.seed, blk, traj, kPurposeHop);
    for (int it = 0; it < bp.len; ++it) {
      const uint32_t word = pick_word(wd, widx);
      const float hsab = bp.hdt * 0.5f * (z.sa + z.sb);  // dt/2 (sig_a + sig_b)/2
      kick<NPL, KIND>(w, cf, hsab * z.c2, hsab * z.s2);  // first half kick at R_n
#pragma unroll
      for (int j = 0; j < NPL; ++j) w.R[j] = __fmaf_rn(cf.dtm[j], w.P[j], w.R[j]);  // drift
      const float r_old = z.r;
      z.A = bp.a0;
      z.B = bp.b0;
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        z.A = __fmaf_rn(cf.a[j], w.R[j], z.A);
        if (KIND == 1) z.B = __fmaf_rn(cf.b[j], w.R[j], z.B);
      }
      closed_form(z);
      kick<NPL, KIND>(w, cf, hsab * z.c2, hsab * z.s2);  // second half kick at R_{n+1}
      float Av = 0.0f, Bv = 0.0f;
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        Av = __fmaf_rn(cf.am[j], w.P[j], Av);
        if (KIND == 1) Bv = __fmaf_rn(cf.bm[j], w.P[j], Bv);
      }
      phase_and_transition(z, r_old, Av, Bv, word, bp, active, n_deg);
      if (++widx == 4) {
        widx = 0;
        ++blk;
        if (it + 1 < bp.len) wd = philox_draw(bp.seed, blk, traj, kPurposeHop);
      }
      if (--to_out == 0) {
        observe(slot++);
        to_out = bp.stride;
      }
    }
    if (active) {
#pragma unroll
      for (int j = 0; j < NPL; ++j)
        if (j < bp.n) {
          ws.R[(int64_t)j * nt + i] = w.R[j];
          ws.P[(int64_t)j * nt + i] = w.P[j];
        }
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
    z.sa = sgn(ab & 0xff);
    z.sb = sgn((ab >> 8) & 0xff);
    const uint64_t traj = bp.traj_offset + (uint64_t)ii;

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
      renorm(z.m, z.mexp);
      if (ROLE == 0) {
        const bool live = active && z.m.hi != 0.0f;
        int ew = live ? z.mexp : -(1 << 28);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ew = max(ew, __shfl_xor_sync(0xffffffffu, ew, off));
        float v[16];
        contributions(z, live ? z.m.hi * pow2i(z.mexp - ew) : 0.0f, v);
        float* row = &obs_rows[wslot * 33];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          row[q] = v[q];
          row[16 + q] = v[q] * v[q];
        }
        __syncwarp();
        const float x = column_sum32(&obs_rows[(grp * 32) * 33 + lane]);
        __syncwarp();
        const int ex = (ew < -(1 << 27)) ? 0 : ((lane < 16) ? ew : 2 * ew);
        const double xd = (double)x;
        red[rb][grp][lane] = (ex >= -1022 && ex <= 1023) ? xd * pow2d(ex) : ldexp(xd, ex);
      } else {
        float v[16];
        contributions(z, 0.0f, v);  // keeps the phase reduction identical on every role
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
    u4 wd = philox_draw(bp.seed, blk, traj, kPurposeHop);
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
      closed_form(z);
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
      phase_and_transition(z, r_old, Av, Bv, word, bp, active, n_deg);
      if (++widx == 4) {
        widx = 0;
        ++blk;
        if (it + 1 < bp.len) wd = philox_draw(bp.seed, blk, traj, kPurposeHop);
      }
      if (--to_out == 0) {
        observe(slot++);
        to_out = bp.stride;
      }
    }
    if (active) {
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
  __shared__ float obs_rows[BW * 33];
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

void launch_sample_f32(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st) {
  const int64_t nb = (sp.n_traj + 255) / 256;
  k_sample_f32<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, st>>>(dm, sp, buf);
  launches_add(1);
}

namespace {
using BulkFn = void (*)(const BulkParams, const Coef2, void*, double*);

int run_kernel(BulkFn fn, int& per_sm, int& n_sm, const BulkParams& bp, const Coef2& cf, void* buf,
               double* part, int grid_cap, cudaStream_t st) {
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  int64_t grid = (int64_t)per_sm * n_sm;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid > bp.n_tiles) grid = bp.n_tiles;
  if (grid < 1) grid = 1;
  fn<<<(unsigned)grid, 256, 0, st>>>(bp, cf, buf, part);
  launches_add(1);
  return (int)grid;
}

template <int NPL, int KIND>
int run_bulk(const BulkParams& bp, const Coef2& cf, void* buf, double* part, int grid_cap,
             cudaStream_t st) {
  static int per_sm = -1, n_sm = 0;
  return run_kernel(k_bulk2<NPL, KIND>, per_sm, n_sm, bp, cf, buf, part, grid_cap, st);
}

template <int NPL, int L, int KIND, int MINB>
int run_wide(const BulkParams& bp, const Coef2& cf, void* buf, double* part, int grid_cap,
             cudaStream_t st) {
  static int per_sm = -1, n_sm = 0;
  return run_kernel(k_bulk2_split<NPL, L, KIND, MINB>, per_sm, n_sm, bp, cf, buf, part, grid_cap,
                    st);
}

template <int KIND>
int dispatch_n(const BulkParams& bp, const Coef2& cf, void* buf, double* part, int cap,
               cudaStream_t st) {
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
  if (n <= 100) return run_wide<50, 2, KIND, 1>(bp, cf, buf, part, cap, st);
  if (n <= 128) return run_wide<32, 4, KIND, MB>(bp, cf, buf, part, cap, st);
  if (n <= 256) return run_wide<64, 4, KIND, 1>(bp, cf, buf, part, cap, st);
  return 0;
}
}  // namespace

int launch_bulk2(const BulkParams& bp, const Coef2& cf, void* buf, double* part, int grid_cap,
                 cudaStream_t st) {
  return bp.kind == 0 ? dispatch_n<0>(bp, cf, buf, part, grid_cap, st)
                      : dispatch_n<1>(bp, cf, buf, part, grid_cap, st);
}

const char* bulk2_variant(int n, int kind) {
  (void)kind;
  switch (bulk_lanes(n)) {
    case 1: return "k_bulk2: one thread per walker, all modes in registers";
    case 2: return "k_bulk2_split: two warps per 32 walkers";
    default: return "k_bulk2_split: four warps per 32 walkers";
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
