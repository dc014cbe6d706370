// bulk2.cuh -- device code of the two-state FP32-bulk walker kernels shared by
// the single-request persistent kernel (kernels_f32.cu) and the packed
// multi-request kernel of the server (packed.cu): walker views, compensated
// weight/phase helpers, the per-step scalar algebra and the tile body.
#pragma once
#include <type_traits>

#include "kernels.h"
#include "lanes.cuh"
#include "reduce.cuh"

namespace qcl {


namespace b2 {

// 2 pi = C1 + C2 + C3 with C1, C2 of 14 significant bits (k * C exact for |k| < 2^10)
constexpr float kTwoPi1 = 6.283203125f;
constexpr float kTwoPi2 = -1.7818063497543335e-05f;
constexpr float kTwoPi3 = 2.430840251310684e-10f;
constexpr float kInvTwoPi = 0.15915494309189535f;

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

}  // namespace b2
using namespace b2;

// ------------------------------------------------------- persistent step --
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Row stride (floats) of the observation rows in shared memory: 16-byte
// aligned rows that a warp writes with 128-bit stores (the 8 threads of a
// quarter warp start 4 banks apart) and reads with 128-bit loads (a quarter
// warp reads 32 consecutive floats of one row), both without bank conflicts.
constexpr int kObsRow = 36;

// State of one walker (V = float) or two (V = float2) that every holder of a
// walker keeps identical: weight (compensated pair and exponent), phase
// (compensated pair), the pair's sigmas, and the closed-form decomposition at
// the current R.
template <typename V>
struct ScalV {
  PairV<V> m;
  typename Lanes<V>::I mexp;
  typename Lanes<V>::I q;  // quarter turns of the weight (diabatic representation)
  PairV<V> ph;
  V sa, sb;                // sigma of the index pair: -1 lower, +1 upper adiabatic state
  V A, B;                  // a(R), b(R)
  V r2, ir, r;             // r^2, 1/r, r
  V c2, s2;                // cos 2theta, sin 2theta (theta = 0 at r = 0)
};
using Scal = ScalV<float>;

// Walker l of a two-walker state as a one-walker state, and back.
__device__ __forceinline__ Scal lane_of(const ScalV<float2>& z, int l) {
  Scal o;
  o.m = {ln(z.m.hi, l), ln(z.m.lo, l)};
  o.mexp = ln(z.mexp, l);
  o.q = ln(z.q, l);
  o.ph = {ln(z.ph.hi, l), ln(z.ph.lo, l)};
  o.sa = ln(z.sa, l);
  o.sb = ln(z.sb, l);
  o.A = ln(z.A, l);
  o.B = ln(z.B, l);
  o.r2 = ln(z.r2, l);
  o.ir = ln(z.ir, l);
  o.r = ln(z.r, l);
  o.c2 = ln(z.c2, l);
  o.s2 = ln(z.s2, l);
  return o;
}
__device__ __forceinline__ void set_lane(ScalV<float2>& z, int l, const Scal& o) {
  ln(z.m.hi, l) = o.m.hi;
  ln(z.m.lo, l) = o.m.lo;
  ln(z.mexp, l) = o.mexp;
  ln(z.q, l) = o.q;
  ln(z.ph.hi, l) = o.ph.hi;
  ln(z.ph.lo, l) = o.ph.lo;
  ln(z.sa, l) = o.sa;
  ln(z.sb, l) = o.sb;
  ln(z.A, l) = o.A;
  ln(z.B, l) = o.B;
  ln(z.r2, l) = o.r2;
  ln(z.ir, l) = o.ir;
  ln(z.r, l) = o.r;
  ln(z.c2, l) = o.c2;
  ln(z.s2, l) = o.s2;
}
__device__ __forceinline__ Scal lane_of(const Scal& z, int) { return z; }
__device__ __forceinline__ void set_lane(Scal& z, int, const Scal& o) { z = o; }

// cos 2theta = a / r, sin 2theta = b / r.  r^2 is floored at the smallest
// normal float, so at an exact degeneracy (a = b = 0 in FP32, where the angle
// is undefined and the coupling is set to zero) both come out 0 -- the mean of
// the two branches -- instead of a division by zero.
// S2 = false leaves s2 stale (the spin-boson step needs no sin 2theta; the
// observation recomputes it).
template <bool S2 = true, typename V>
__device__ __forceinline__ void closed_form(ScalV<V>& z) {
  z.r2 = vfma(z.A, z.A, vmul(z.B, z.B));
#pragma unroll
  for (int l = 0; l < Lanes<V>::W; ++l) ln(z.ir, l) = rsqrtf(fmaxf(ln(z.r2, l), 0x1p-126f));
  z.r = vmul(z.r2, z.ir);
  z.c2 = vmul(z.A, z.ir);
  if (S2) z.s2 = vmul(z.B, z.ir);
}

// Lane l's weight: moves hi's exponent into mexp when hi has left
// [2^-32, 2^32].
template <typename V>
__device__ __forceinline__ void weight_range(ScalV<V>& z, int l) {
  const float h = ln(z.m.hi, l);
  if (!(fabsf(h) <= 0x1p32f && fabsf(h) >= 0x1p-32f)) {
    f2 m = {h, ln(z.m.lo, l)};
    int ex = ln(z.mexp, l);
    renorm(m, ex);
    ln(z.m.hi, l) = m.hi;
    ln(z.m.lo, l) = m.lo;
    ln(z.mexp, l) = ex;
  }
}

// m *= num / den (den an integer below 2^25, so exact in FP32) as a
// compensated quotient: rcp.approx, one exact FMA residual, and the product
// with the error terms collected in lo, then (CHECK) the range check.  The
// persistent two-state kernels pass CHECK = false and check the range where the
// pairs are renormalised (block_end, every fourth absolute step) and before
// each observation.  Model creation bounds the parameter-fixed factors to
// [2^-16, 2^17] (stay 1/(1 - sum p), uncapped hop in [1/kappa, 2/kappa)), so
// four of them take a mantissa in [2^-32, 2^32] to [2^-96, 2^100]: hi and lo
// stay normal FP32 numbers and moving the exponent later is exact, so the
// values and observables are those of a per-step check.  Only capped hops,
// |A_e| / p_e ~ 2 |A_e| / p_max, grow with the data; four of them beyond 2^23
// overflow hi, which the store flags as non-finite.
template <bool CHECK = true, typename V>
__device__ __forceinline__ void weight_factor(ScalV<V>& z, V num, const typename Lanes<V>::U& iden) {
  V den, rd;
#pragma unroll
  for (int l = 0; l < Lanes<V>::W; ++l) {
    ln(den, l) = __uint2float_rn(ln(iden, l));
    ln(rd, l) = rcp_approx(ln(den, l));
  }
  const V q0 = vmul(num, rd);
  // num - q0 den = fma(q0, -den, num), exactly as fma(-q0, den, num)
  const V q1 = vmul(vfma(q0, vmul(den, splat<V>(-1.0f)), num), rd);
  const V p = vmul(z.m.hi, q0);
  V e = vfma(z.m.hi, q0, vmul(p, splat<V>(-1.0f)));
  e = vfma(z.m.hi, q1, e);
  z.m = {p, vfma(z.m.lo, q0, e)};
  if (CHECK) {
#pragma unroll
    for (int l = 0; l < Lanes<V>::W; ++l) weight_range(z, l);
  }
}

// Phase (trapezoid) and transition of one step, given the decomposition at
// R_{n+1} (in z), r at R_n, and the coupling sums Av = sum a_j P_j/M_j,
// Bv = sum b_j P_j/M_j at P_{n+1} (Bv = 0 when only a(R) depends on R).
// `deg` counts steps whose coupling was set to zero at a degeneracy.  The
// weight and phase pairs are left unnormalised (|lo| may grow past ulp(hi)/2
// by about an ulp per step); the step loop renormalises both at every fourth
// step (block_end).  WEIGHT = false skips the phase and the weight (for holders
// of a walker that need only its index pair: the split kernels' other roles).
template <int KIND, bool WEIGHT = true, bool CHECK = true, bool LANE_PHASE = false, typename V>
__device__ __forceinline__ void phase_and_transition(ScalV<V>& z, V r_old, V Av, V Bv,
                                                     const typename Lanes<V>::U& word,
                                                     const BulkParams& bp,
                                                     typename Lanes<V>::U& deg) {
  constexpr int W = Lanes<V>::W;
  // phase: dt/2 (w_ab(R_n) + w_ab(R_{n+1})), hbar w_ab = (sig_a - sig_b) r, added
  // to the low word of the pair (at most four increments and their rounding
  // errors until block_end folds it into hi)
  // LANE_PHASE: per lane with the scalar round-to-nearest operations.  Measured
  // on GB300: in the branch-free step (CHECK = false) the packed form of this one
  // update gave results one ulp apart between one and two walkers per thread,
  // while the per-lane form keeps both bit for bit (and equal to the packed form
  // in the step with the range check).
  if (WEIGHT && LANE_PHASE) {
#pragma unroll
    for (int l = 0; l < W; ++l)
      ln(z.ph.lo, l) = __fmaf_rn(__fmul_rn(bp.hdt_hbar, __fsub_rn(ln(z.sa, l), ln(z.sb, l))),
                                 __fadd_rn(ln(r_old, l), ln(z.r, l)), ln(z.ph.lo, l));
  } else if (WEIGHT) {
    z.ph.lo = vfma(vmul(splat<V>(bp.hdt_hbar), vsub(z.sa, z.sb)), vadd(r_old, z.r), z.ph.lo);
  }
  // coupling contracted with P/M: g = (a Bv - b Av) / (2 r^2)
  // (2 r < tol, compared as r^2 < tol^2 / 4); the spin-boson form has b = b0,
  // so -b/2 is a per-launch constant
  const V gn = (KIND == 1) ? vmul(splat<V>(0.5f), vsub(vmul(z.A, Bv), vmul(z.B, Av)))
                           : vmul(splat<V>(-0.5f * bp.b0), Av);
  V g = vmul(gn, vmul(z.ir, z.ir));
  // both events have |A_e| = dt |g|: p = min(kappa dt |g|, p_max) quantised to
  // 24-bit thresholds T = floor(p 2^24); when 2T exceeds Tmax = floor(p_max 2^24)
  // the integer rescale floor(T Tmax / 2T) gives floor(Tmax / 2), so
  // T = min(floor(kappa dt |g| 2^24), floor(Tmax / 2)) (the conversion saturates)
  typename Lanes<V>::U T, iden;
  bool hop1[W], hop2[W], hop[W];
  if (KIND == 1) {  // (the spin-boson form runs only where r^2 >= b0^2 excludes degeneracy)
#pragma unroll
    for (int l = 0; l < W; ++l) {
      const bool degen = ln(z.r2, l) < kDegR2_32;
      ln(deg, l) += degen ? 1u : 0u;
      ln(g, l) = degen ? 0.0f : ln(g, l);
    }
  }
  const V t = vmul(splat<V>(bp.kamp * kP24f), g);
  // weight factor: A_e / p_hat on a hop (A_1 = -sig_a dt g, A_2 = -sig_b dt g),
  // 1 / (1 - sum p_hat) otherwise
  const V dtgn = vmul(splat<V>(-(bp.amp * kP24f)), g);
  V sel;
#pragma unroll
  for (int l = 0; l < W; ++l) {
    ln(T, l) = min(__float2uint_rz(fabsf(ln(t, l))), bp.tmax >> 1);
    const uint32_t y = ln(word, l) >> 8;
    hop1[l] = y < ln(T, l);
    hop[l] = y < 2u * ln(T, l);
    hop2[l] = hop[l] && !hop1[l];
    ln(sel, l) = hop1[l] ? ln(z.sa, l) : ln(z.sb, l);
    ln(iden, l) = hop[l] ? ln(T, l) : 16777216u - 2u * ln(T, l);
  }
  V num = vmul(sel, dtgn);
  const V nsa = vmul(z.sa, splat<V>(-1.0f)), nsb = vmul(z.sb, splat<V>(-1.0f));
#pragma unroll
  for (int l = 0; l < W; ++l) {
    ln(num, l) = hop[l] ? ln(num, l) : kP24f;
    ln(z.sa, l) = hop1[l] ? ln(nsa, l) : ln(z.sa, l);
    ln(z.sb, l) = hop2[l] ? ln(nsb, l) : ln(z.sb, l);
  }
  // (sigmas flipped after the weight factor has taken the pre-hop sigma in sel)
  if (WEIGHT) weight_factor<CHECK>(z, num, iden);
}

// Diabatic representation: phase with hbar w_ab = V_aa - V_bb = -(sig_a - sig_b)
// a(R) (sig = -1 for diabatic state 0, whose energy is s + a), a_old = a(R_n),
// z.A = a(R_{n+1}); the transitions a -> 1-a (amplitude -i c) and b -> 1-b
// (+i c) with c = V_01 dt / hbar = b(R_{n+1}) dt / hbar = amp * Bc.  Both have
// |A_e| = |c|, so the thresholds follow the adiabatic rule; a hop adds three or
// one quarter turns.
template <bool CHECK = true, typename V>
__device__ __forceinline__ void dia_phase_and_transition(ScalV<V>& z, V a_old, V Bc,
                                                         const typename Lanes<V>::U& word,
                                                         const BulkParams& bp) {
  constexpr int W = Lanes<V>::W;
#pragma unroll
  for (int l = 0; l < W; ++l)  // (per lane, as in phase_and_transition)
    ln(z.ph.lo, l) = __fmaf_rn(__fmul_rn(bp.hdt_hbar, __fsub_rn(ln(z.sb, l), ln(z.sa, l))),
                               __fadd_rn(ln(a_old, l), ln(z.A, l)), ln(z.ph.lo, l));
  const V t = vmul(splat<V>(bp.kamp * kP24f), Bc);
  V num = vmul(splat<V>(bp.amp * kP24f), Bc);
  typename Lanes<V>::U iden;
  bool hop1[W], hop2[W], hop[W];
#pragma unroll
  for (int l = 0; l < W; ++l) {
    const uint32_t T = min(__float2uint_rz(fabsf(ln(t, l))), bp.tmax >> 1);
    const uint32_t y = ln(word, l) >> 8;
    hop1[l] = y < T;
    hop[l] = y < 2u * T;
    hop2[l] = hop[l] && !hop1[l];
    ln(num, l) = hop[l] ? ln(num, l) : kP24f;
    ln(iden, l) = hop[l] ? T : 16777216u - 2u * T;
  }
  weight_factor<CHECK>(z, num, iden);
  const V nsa = vmul(z.sa, splat<V>(-1.0f)), nsb = vmul(z.sb, splat<V>(-1.0f));
#pragma unroll
  for (int l = 0; l < W; ++l) {
    ln(z.q, l) = (ln(z.q, l) + (hop1[l] ? 3 : (hop2[l] ? 1 : 0))) & 3;
    ln(z.sa, l) = hop1[l] ? ln(nsa, l) : ln(z.sa, l);
    ln(z.sb, l) = hop2[l] ? ln(nsb, l) : ln(z.sb, l);
  }
}

// Renormalises the weight and phase pairs and (CHECK) checks the weight's
// range; called at the end of every Philox block (absolute steps 4k + 3),
// whatever the chunking.  Kernels whose steps check the range themselves pass
// CHECK = false.
template <bool CHECK = true, typename V>
__device__ __forceinline__ void block_end(ScalV<V>& z) {
  z.m = fast_two_sum_v(z.m.hi, z.m.lo);
  z.ph = two_sum_v(z.ph.hi, z.ph.lo);
  if (CHECK) {
#pragma unroll
    for (int l = 0; l < Lanes<V>::W; ++l) weight_range(z, l);
  }
}

// FP32 initial sample of one walker with random-stream id `traj` from the same
// Philox words as the FP64 path: (R, P) at Rg[j * stride], Pg[j * stride], the
// weight mantissa mh (low part, exponent and phase start at 0) and the index
// pair word ab.  All arithmetic in FP32 (inputs converted on the host).
__device__ __forceinline__ void sample_walker_f32(const Sample32& sp, uint64_t traj, float* Rg,
                                                  float* Pg, int64_t stride, float& mh,
                                                  uint16_t& ab) {
  const int n = sp.n;
  float a = sp.a0, b = sp.b0;
  for (int j = 0; j < n; ++j) {
    float R = sp.R0[j], P = sp.P0[j];
    if (sp.wigner) {
      const u4 wd = philox_draw(sp.seed, (uint32_t)j, traj, kPurposeInit);
      const float u0 = __fmaf_rn(__uint2float_rn(wd.x), 0x1p-32f, 0x1p-33f);
      const float u1 = __fmaf_rn(__uint2float_rn(wd.y), 0x1p-32f, 0x1p-33f);
      const float rad = sqrtf(-2.0f * logf(u0));
      float sn, cs;
      sincospif(2.0f * u1, &sn, &cs);
      R = __fmaf_rn(sp.sR[j] * rad, cs, R);
      P = __fmaf_rn(sp.sP[j] * rad, sn, P);
    }
    Rg[(int64_t)j * stride] = R;
    Pg[(int64_t)j * stride] = P;
    a = __fmaf_rn(sp.a[j], R, a);
    b = __fmaf_rn(sp.b[j], R, b);
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
  float rho_ad[4];  // the density in the walkers' representation
  float tot = 0.0f;
  for (int al = 0; al < 2; ++al)
    for (int be = 0; be < 2; ++be) {
      float acc = 0.0f;
      if (sp.repr == QCL_REPR_DIABATIC) {
        acc = sp.rho[al * 2 + be];
      } else {
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l)
            acc = __fmaf_rn(U[k * 2 + al] * sp.rho[k * 2 + l], U[l * 2 + be], acc);
      }
      rho_ad[al * 2 + be] = acc;
      tot += fabsf(acc);
    }
  // index pair from |rho_ad| with 2^-24 quantised probabilities (remainder to the
  // last nonzero pair), m0 = rho_ad / p_hat.  FP32 rounding of the quotients can
  // make the floors sum past 2^24 by a few units; the excess then comes off the
  // largest threshold.
  uint32_t Tk[4];
  uint32_t sumT = 0;
  int last = 0, big = 0;
  for (int k = 0; k < 4; ++k) {
    Tk[k] = (uint32_t)floorf(__fdiv_rn(fabsf(rho_ad[k]), tot) * kP24f);
    sumT += Tk[k];
    if (rho_ad[k] != 0.0f) last = k;
    if (Tk[k] > Tk[big]) big = k;
  }
  if (sumT <= 16777216u) Tk[last] += 16777216u - sumT;
  else Tk[big] -= sumT - 16777216u;
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
  mh = rho_ad[pick] * (kP24f / (float)Tk[pick]);
  ab = (uint16_t)((pick >> 1) | ((pick & 1) << 8));
}

// Transition test of a spawning walker (the scheme that starts a new walker
// whenever the test fires): the phase as in phase_and_transition (DIA: as in
// dia_phase_and_transition, w_old = a(R_n), Bv = b(R_{n+1})); when the test
// fires for event e, `child` becomes a copy of the walker with its weight times
// A_e / p_hat_e, the flipped index and (DIA) the event's quarter turns, and the
// walker keeps its pair and weight (no stay factor).  Returns whether it fired.
template <int KIND, bool DIA>
__device__ __forceinline__ bool spawn_transition(Scal& z, float w_old, float Av, float Bv,
                                                 uint32_t word, const BulkParams& bp,
                                                 unsigned int& deg, Scal& child) {
  uint32_t T;
  float fac;  // A_e 2^24 of the first-index event (DIA: both events)
  if (DIA) {
    z.ph.lo = __fmaf_rn(bp.hdt_hbar * (z.sb - z.sa), w_old + z.A, z.ph.lo);
    T = min(__float2uint_rz((bp.kamp * kP24f) * fabsf(Bv)), bp.tmax >> 1);
    fac = (bp.amp * kP24f) * Bv;
  } else {
    z.ph.lo = __fmaf_rn(bp.hdt_hbar * (z.sa - z.sb), w_old + z.r, z.ph.lo);
    const bool degen = z.r2 < kDegR2_32;
    deg += degen ? 1u : 0u;
    const float gn = (KIND == 1) ? 0.5f * (z.A * Bv - z.B * Av) : (-0.5f * bp.b0) * Av;
    const float g = degen ? 0.0f : gn * (z.ir * z.ir);
    T = min(__float2uint_rz((bp.kamp * kP24f) * fabsf(g)), bp.tmax >> 1);
    fac = (bp.amp * kP24f) * g;
  }
  const uint32_t y = word >> 8;
  const bool hop1 = y < T;
  const bool hop = y < 2u * T;
  if (!hop) return false;
  child = z;
  // adiabatic: A_1 = -sig_a dt g, A_2 = -sig_b dt g; diabatic: both c = b dt / hbar
  const float num = DIA ? fac : -(hop1 ? z.sa : z.sb) * fac;
  weight_factor(child, num, T);
  child.m = fast_two_sum(child.m.hi, child.m.lo);
  if (hop1) child.sa = -child.sa;
  else child.sb = -child.sb;
  if (DIA) child.q = (child.q + (hop1 ? 3 : 1)) & 3;
  return true;
}

// Keeps the stored phase within about 2^10 rad, where the three-part
// reduction below is exact; every holder of a walker calls it at the same
// steps (the observations).
__device__ __forceinline__ void phase_wrap(Scal& z) {
  if (fabsf(z.ph.hi) > 1024.0f) {
    const float kq = rintf(z.ph.hi * kInvTwoPi);
    z.ph = df_add(z.ph, -kq * kTwoPi1);
    z.ph = df_add(z.ph, -kq * kTwoPi2);
    z.ph = df_add(z.ph, -kq * kTwoPi3);
  }
}

// The walker's observable factors: z = mm exp(-i phi) (times i^q for a
// diabatic walker), which goes to the walker's own pair k = 2 alpha + beta in
// its own representation, and the products f_kl = U_{alpha k} U_{beta l} that
// carry it to every element of the other (U is symmetric: the same products
// serve both directions).
struct Contrib {
  float zr, zi;
  float f00, f01, f10, f11;
  int k;
};

template <bool DIA>
__device__ __forceinline__ Contrib contrib_factors(const Scal& z, float mm) {
  // phase reduced into [-pi, pi]: ph_hi - k C1 is exact (|k| < 2^10), the
  // small terms are added once
  const float kq = rintf(z.ph.hi * kInvTwoPi);
  const float x = __fmaf_rn(-kq, kTwoPi1, z.ph.hi) + __fmaf_rn(-kq, kTwoPi2, z.ph.lo);
  float sphi, cphi;
  __sincosf(x, &sphi, &cphi);
  // eigenvector angle theta from (cos 2theta, sin 2theta), half-angle form
  // without cancellation: the larger of cos/sin is sqrt((1 + |cos2t|)/2); at an
  // exact degeneracy (both 0) theta = 0
  const float c2 = (z.c2 == 0.0f && z.s2 == 0.0f) ? 1.0f : z.c2;
  const float t = __fmaf_rn(0.5f, fabsf(c2), 0.5f);
  const float rt = rsqrtf(t);
  const float big = t * rt, small = 0.5f * fabsf(z.s2) * rt;
  const bool cpos = c2 >= 0.0f;
  const float c = cpos ? big : small;
  const float s = copysignf(cpos ? small : big, z.s2);
  const bool al = z.sa > 0.0f, be = z.sb > 0.0f;
  const float ua0 = al ? c : -s, ua1 = al ? s : c;  // column alpha of U
  const float ub0 = be ? c : -s, ub1 = be ? s : c;  // column beta of U
  Contrib o;
  o.zr = mm * cphi;
  o.zi = -mm * sphi;
  if (DIA) {  // times i^q
    const float xr = o.zr, xi = o.zi;
    o.zr = (z.q & 1) ? -xi : xr;
    o.zi = (z.q & 1) ? xr : xi;
    o.zr = (z.q & 2) ? -o.zr : o.zr;
    o.zi = (z.q & 2) ? -o.zi : o.zi;
  }
  o.f00 = ua0 * ub0;
  o.f01 = ua0 * ub1;
  o.f10 = ua1 * ub0;
  o.f11 = ua1 * ub1;
  o.k = (al ? 2 : 0) + (be ? 1 : 0);
  return o;
}

// The walker's 16 observable contributions (diabatic rho_ij and adiabatic
// rho_ab, real and imaginary) with weight mantissa `mm`.
template <bool DIA>
__device__ __forceinline__ void contributions(const Scal& z, float mm, float (&v)[16]) {
  const Contrib c = contrib_factors<DIA>(z, mm);
  constexpr int other = DIA ? 8 : 0, own = DIA ? 0 : 8;
  v[other + 0] = c.zr * c.f00;
  v[other + 1] = c.zi * c.f00;
  v[other + 2] = c.zr * c.f01;
  v[other + 3] = c.zi * c.f01;
  v[other + 4] = c.zr * c.f10;
  v[other + 5] = c.zi * c.f10;
  v[other + 6] = c.zr * c.f11;
  v[other + 7] = c.zi * c.f11;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    v[own + 2 * kk] = (kk == c.k) ? c.zr : 0.0f;
    v[own + 1 + 2 * kk] = (kk == c.k) ? c.zi : 0.0f;
  }
}

// x 2^ex as a double, exactly (built from the bits for normal x and results in
// the normal double range; zero, subnormal, non-finite or out-of-range values
// go through ldexp).
__device__ __forceinline__ double scaled_double(float x, int ex) {
  const uint32_t u = __float_as_uint(x);
  const int e8 = (int)((u >> 23) & 0xffu);
  const int e11 = e8 + (1023 - 127) + ex;
  if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (e8 != 0 && e8 != 255 && e11 > 0 && e11 < 2047)
    return __hiloint2double((int)((u & 0x80000000u) | ((uint32_t)e11 << 20) | ((u & 0x7fffffu) >> 3)),
                            (int)(u << 29));
  return ldexp((double)x, ex);
}

// The same value on the FP64 pipe (a conversion and one multiply), which the
// two-state bulk kernels leave idle: their observations take it, sparing the
// issue slots of the bit construction above.
__device__ __forceinline__ double scaled_double_fp64(float x, int ex) {
  return (ex >= -1022 && ex <= 1023) ? (double)x * __hiloint2double((ex + 1023) << 20, 0)
                                     : ldexp((double)x, ex);
}

__device__ __forceinline__ float4 sq4(float4 a) {
  return make_float4(a.x * a.x, a.y * a.y, a.z * a.z, a.w * a.w);
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Observation by one warp of 32 walkers.  The warp shares one power of two
// (FP32 sums of scaled weights, the exponent restored exactly in FP64).  Each
// walker writes its 16 contributions and their squares to its row `row` of
// shared memory (the four slots of its own representation as zeros, then its
// own pair's slot).  The warp's 32 rows (from row0) are summed column by
// column with a fixed pairwise tree ((x0 + x1) + (x2 + x3)) + ...: lane
// L = 8 g + c reads rows 8g .. 8g+7 of columns 4c .. 4c+3 with 128-bit loads
// and sums them, and two butterfly exchanges with lanes L ^ 8 and L ^ 16 join
// the four row groups, leaving lane L with the total of column
// 4c + 2 (g & 1) + (g >> 1), which it writes, scaled, to red_row[column].
// WIDE = false sums the same tree with lane q reading column q by 32-bit loads
// (for kernels short of registers).
template <bool DIA, bool WIDE = true>
__device__ __forceinline__ void observe_warp(Scal& z, bool active, float* obs_rows, int row,
                                             int row0, int lane, double* red_row) {
  // (no renormalisation of the weight here: the step keeps its mantissa within
  // [2^-32, 2^32], so scaled contributions and squares stay far inside FP32)
  phase_wrap(z);
  if (DIA) closed_form(z);  // the rotation to the adiabatic basis at the walker's R
  else z.s2 = z.B * z.ir;   // (the same value closed_form gives)
  const bool live = active && z.m.hi != 0.0f;
  const int ew = __reduce_max_sync(0xffffffffu, live ? z.mexp : -(1 << 28));
  const Contrib c =
      contrib_factors<DIA>(z, live ? (z.m.hi + z.m.lo) * pow2i(z.mexp - ew) : 0.0f);
  constexpr int other = DIA ? 8 : 0, own = DIA ? 0 : 8;
  float* r = &obs_rows[row * kObsRow];
  const float4 o0 = make_float4(c.zr * c.f00, c.zi * c.f00, c.zr * c.f01, c.zi * c.f01);
  const float4 o1 = make_float4(c.zr * c.f10, c.zi * c.f10, c.zr * c.f11, c.zi * c.f11);
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  *reinterpret_cast<float4*>(r + other) = o0;
  *reinterpret_cast<float4*>(r + other + 4) = o1;
  *reinterpret_cast<float4*>(r + 16 + other) = sq4(o0);
  *reinterpret_cast<float4*>(r + 16 + other + 4) = sq4(o1);
  *reinterpret_cast<float4*>(r + own) = zero;
  *reinterpret_cast<float4*>(r + own + 4) = zero;
  *reinterpret_cast<float4*>(r + 16 + own) = zero;
  *reinterpret_cast<float4*>(r + 16 + own + 4) = zero;
  *reinterpret_cast<float2*>(r + own + 2 * c.k) = make_float2(c.zr, c.zi);
  *reinterpret_cast<float2*>(r + 16 + own + 2 * c.k) = make_float2(c.zr * c.zr, c.zi * c.zi);
  __syncwarp();
  float x;
  int col;
  if (WIDE) {
    const int g = lane >> 3, c4 = lane & 7;
    const float* base = &obs_rows[(row0 + 8 * g) * kObsRow + 4 * c4];
    float4 s[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = *reinterpret_cast<const float4*>(base + i * kObsRow);
    __syncwarp();
    const float4 S = add4(add4(add4(s[0], s[1]), add4(s[2], s[3])),
                          add4(add4(s[4], s[5]), add4(s[6], s[7])));
    const bool odd = g & 1, hi = g >> 1;
    const float t0 = (odd ? S.z : S.x) + __shfl_xor_sync(0xffffffffu, odd ? S.x : S.z, 8);
    const float t1 = (odd ? S.w : S.y) + __shfl_xor_sync(0xffffffffu, odd ? S.y : S.w, 8);
    x = (hi ? t1 : t0) + __shfl_xor_sync(0xffffffffu, hi ? t0 : t1, 16);
    col = 4 * c4 + 2 * (g & 1) + (g >> 1);
  } else {  // the same tree, one column per lane with 32-bit loads (fewer live registers)
    const float* cl = &obs_rows[row0 * kObsRow + lane];
    float l1[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) l1[t] = cl[(2 * t) * kObsRow] + cl[(2 * t + 1) * kObsRow];
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
      for (int t = 0; t < w; ++t) l1[t] = l1[2 * t] + l1[2 * t + 1];
    __syncwarp();
    x = l1[0];
    col = lane;
  }
  const int ex = (ew < -(1 << 27)) ? 0 : ((col < 16) ? ew : 2 * ew);
  red_row[col] = scaled_double(x, ex);
}

__device__ __forceinline__ uint32_t pick_word(const u4& wd, int widx) {
  return (widx & 2) ? ((widx & 1) ? wd.w : wd.z) : ((widx & 1) ? wd.y : wd.x);
}

// The hop stream through the whole Philox function (fewer live registers
// than PhiloxStream, the same words).
struct PlainStream {
  uint64_t seed, traj;
  PlainStream() = default;
  __device__ __forceinline__ PlainStream(uint64_t s, uint64_t t, uint32_t) : seed(s), traj(t) {}
  __device__ __forceinline__ u4 draw(uint32_t n) const {
    return philox_draw(seed, n, traj, kPurposeHop);
  }
};

template <int NPL, typename V = float>
struct WalkerV {
  V R[NPL], P[NPL];
};
template <int NPL>
using Walker = WalkerV<NPL, float>;

// P += dt/2 F_ab(R),  F_j = -k_j R_j - s_j - sab (a_j cos2t + b_j sin2t);
// hu = dt/2 sab cos2t, hv = dt/2 sab sin2t
template <int NPL, int KIND, typename CF, typename V>
__device__ __forceinline__ void kick(WalkerV<NPL, V>& w, const CF& cf, V hu, V hv) {
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    V p = vfma(splat<V>(-cf.hk[j]), w.R[j], w.P[j]);
    if (KIND == 1) p = vadd(p, splat<V>(-cf.hs[j]));
    p = vfma(hu, splat<V>(-cf.a[j]), p);
    if (KIND == 1) p = vfma(hv, splat<V>(-cf.b[j]), p);
    w.P[j] = p;
  }
}

// Diabatic kick: P += dt/2 F_ab(R), F_j = -k_j R_j - s_j + sab a_j (the
// adiabatic kick's force with cos 2theta = -1, sin 2theta = 0), hsab = dt/2 sab.
template <int NPL, int KIND, typename CF, typename V>
__device__ __forceinline__ void kick_dia(WalkerV<NPL, V>& w, const CF& cf, V hsab) {
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    V p = vfma(splat<V>(-cf.hk[j]), w.R[j], w.P[j]);
    if (KIND == 1) p = vadd(p, splat<V>(-cf.hs[j]));
    w.P[j] = vfma(hsab, splat<V>(cf.a[j]), p);
  }
}

// Per-mode coefficients of a packed request, held in registers.
template <int NPL>
struct CoefLocal {
  float hk[NPL], hs[NPL], dtm[NPL], a[NPL], b[NPL], am[NPL], bm[NPL];
};

// WPT (1 or 2) consecutive 256-walker tiles (tile0, tile0 + 1) of the
// one-thread-per-walker kernel, thread t owning walker t of each: load the
// walkers, advance them over steps [cs, ce) with their observations, store
// them.  With WPT = 2 the thread's two walkers are the two lanes of float2
// values and step together through the packed FP32x2 instructions; each
// walker's arithmetic and each tile's reduction are exactly those of WPT = 1,
// so the results do not depend on WPT.  `cf` holds the per-mode coefficients
// (kernel parameters, or registers in the packed kernel); all threads of the
// block call it together.  LEAN selects the register-lean form for kernels
// short of registers (many modes, coefficients in registers): steps one at a
// time and the whole Philox function per draw, instead of the unrolled
// four-step blocks below and the precomputed stream.  Both forms give the same
// bits.
template <int NPL, int KIND, typename CF, bool LEAN, bool DIA = false, int WPT = 1>
__device__ __forceinline__ void bulk2_tile(const BulkParams& bp, const CF& cf, W32& ws,
                                           double* __restrict__ part, int64_t tile0, int& rb,
                                           unsigned int& n_deg, double (*red)[8][32],
                                           float* obs_rows) {
  static_assert(WPT == 1 || WPT == 2, "one or two walkers per thread");
  using V = std::conditional_t<WPT == 2, float2, float>;
  using U = typename Lanes<V>::U;
  using Stream = std::conditional_t<LEAN, PlainStream, PhiloxStream>;
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WalkerV<NPL, V> w;
  ScalV<V> z;
  bool active[WPT];
  U deg;
#pragma unroll
  for (int k = 0; k < WPT; ++k) {
    const int64_t i = (tile0 + k) * kTile + threadIdx.x;
    active[k] = i < nt;
    const int64_t ii = active[k] ? i : 0;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const bool on = active[k] && j < bp.n;
      ln(w.R[j], k) = on ? ws.R[(int64_t)j * nt + ii] : 0.0f;
      ln(w.P[j], k) = on ? ws.P[(int64_t)j * nt + ii] : 0.0f;
    }
    ln(z.m.hi, k) = active[k] ? ws.mh[ii] : 0.0f;
    ln(z.m.lo, k) = active[k] ? ws.ml[ii] : 0.0f;
    ln(z.mexp, k) = active[k] ? ws.me[ii] : 0;
    ln(z.ph.hi, k) = active[k] ? ws.ph[ii] : 0.0f;
    ln(z.ph.lo, k) = active[k] ? ws.pl[ii] : 0.0f;
    const uint32_t ab = active[k] ? ws.ab[ii] : 0u;  // alpha | q << 4 | beta << 8
    ln(z.sa, k) = sgn(ab & 0xf);
    ln(z.sb, k) = sgn((ab >> 8) & 0xf);
    ln(z.q, k) = DIA ? (int)((ab >> 4) & 3u) : 0;
    ln(deg, k) = 0u;
  }
  z.A = splat<V>(bp.a0);
  z.B = splat<V>(bp.b0);
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    z.A = vfma(splat<V>(cf.a[j]), w.R[j], z.A);
    if (KIND == 1) z.B = vfma(splat<V>(cf.b[j]), w.R[j], z.B);
  }
  closed_form(z);

  // observation into slot `slot` of the tiles' partials: each warp's column
  // sums of walker k go to red[WPT rb + k], then (one barrier for all k) warp k
  // folds tile k's 8 warp rows by the fixed FP64 tree.  red holds 2 WPT
  // buffers: consecutive observations alternate between two sets, so a set is
  // rewritten only after the barrier that follows the warps' reads of it.
  auto observe_all = [&](int slot) {
#pragma unroll
    for (int k = 0; k < WPT; ++k) weight_range(z, k);
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      Scal zk = lane_of(z, k);
      observe_warp<DIA>(zk, active[k], obs_rows, threadIdx.x, warp * 32, lane,
                        red[WPT * rb + k][warp]);
      set_lane(z, k, zk);
    }
    __syncthreads();
    if (warp < WPT && tile0 + warp < bp.n_tiles)
      part[((int64_t)slot * bp.n_tiles + tile0 + warp) * 32 + lane] =
          tile_tree8(&red[WPT * rb + warp][0][0], 32, lane);
    rb ^= 1;
  };

  // one velocity-Verlet step of the walkers with their phase and transition
  // (hop words `word`)
  auto step = [&](const U& word) {
    const V hsab = vmul(splat<V>(bp.hdt * 0.5f), vadd(z.sa, z.sb));  // dt/2 (sig_a + sig_b)/2
    if constexpr (DIA) {
      kick_dia<NPL, KIND, CF>(w, cf, hsab);
#pragma unroll
      for (int j = 0; j < NPL; ++j) w.R[j] = vfma(splat<V>(cf.dtm[j]), w.P[j], w.R[j]);
      const V a_old = z.A;
      z.A = splat<V>(bp.a0);
      if (KIND == 1) z.B = splat<V>(bp.b0);
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        z.A = vfma(splat<V>(cf.a[j]), w.R[j], z.A);
        if (KIND == 1) z.B = vfma(splat<V>(cf.b[j]), w.R[j], z.B);
      }
      kick_dia<NPL, KIND, CF>(w, cf, hsab);
      dia_phase_and_transition<false>(z, a_old, z.B, word, bp);
      return;
    }
    kick<NPL, KIND, CF>(w, cf, vmul(hsab, z.c2), vmul(hsab, z.s2));  // first half kick at R_n
#pragma unroll
    for (int j = 0; j < NPL; ++j) w.R[j] = vfma(splat<V>(cf.dtm[j]), w.P[j], w.R[j]);  // drift
    const V r_old = z.r;
    z.A = splat<V>(bp.a0);
    z.B = splat<V>(bp.b0);
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      z.A = vfma(splat<V>(cf.a[j]), w.R[j], z.A);
      if (KIND == 1) z.B = vfma(splat<V>(cf.b[j]), w.R[j], z.B);
    }
    closed_form<KIND == 1>(z);
    kick<NPL, KIND, CF>(w, cf, vmul(hsab, z.c2), vmul(hsab, z.s2));  // second half kick at R_{n+1}
    V Av = splat<V>(0.0f), Bv = splat<V>(0.0f);
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      Av = vfma(splat<V>(cf.am[j]), w.P[j], Av);
      if (KIND == 1) Bv = vfma(splat<V>(cf.bm[j]), w.P[j], Bv);
    }
    phase_and_transition<KIND, true, false, true>(z, r_old, Av, Bv, word, bp, deg);
  };

  // Steps are grouped by Philox block (four steps share one draw).  A whole
  // block with no output before its last step runs unrolled with its words in
  // fixed registers; other steps (a chunk's ragged ends, blocks with an output
  // inside) run one at a time.  The weight and phase pairs are renormalised at
  // the end of every block, i.e. at the same absolute steps on both routes.
  int slot = bp.obs_first;
  if (bp.obs_first) observe_all(0);
  int to_out = bp.to_out0;
  uint32_t blk = bp.blk0;
  int widx = bp.widx0;
  Stream rng[WPT] = {};
  u4 wd[WPT];
#pragma unroll
  for (int k = 0; k < WPT; ++k) {
    const int64_t ii = active[k] ? (tile0 + k) * kTile + threadIdx.x : 0;
    rng[k] = Stream(bp.seed, bp.traj_offset + (uint64_t)ii, kPurposeHop);
    wd[k] = rng[k].draw(blk);
  }
  auto words = [&](int q) {
    U u;
#pragma unroll
    for (int k = 0; k < WPT; ++k) ln(u, k) = pick_word(wd[k], q);
    return u;
  };
  int it = 0;
  while (it < bp.len) {
    if (!LEAN && widx == 0 && bp.len - it >= 4 && to_out >= 4) {
      step(words(0));
      step(words(1));
      step(words(2));
      step(words(3));
      block_end(z);
      it += 4;
      to_out -= 4;
      ++blk;
      if (it < bp.len) {
#pragma unroll
        for (int k = 0; k < WPT; ++k) wd[k] = rng[k].draw(blk);
      }
    } else {
      step(words(widx));
      ++it;
      --to_out;
      if (++widx == 4) {
        widx = 0;
        block_end(z);
        ++blk;
        if (it < bp.len) {
#pragma unroll
          for (int k = 0; k < WPT; ++k) wd[k] = rng[k].draw(blk);
        }
      }
    }
    if (to_out == 0) {
      observe_all(slot++);
      to_out = bp.stride;
    }
  }
#pragma unroll
  for (int k = 0; k < WPT; ++k) {
    if (!active[k]) continue;
    const int64_t i = (tile0 + k) * kTile + threadIdx.x;
    n_deg += ln(deg, k);
#pragma unroll
    for (int j = 0; j < NPL; ++j)
      if (j < bp.n) {
        ws.R[(int64_t)j * nt + i] = ln(w.R[j], k);
        ws.P[(int64_t)j * nt + i] = ln(w.P[j], k);
      }
    const float mh = ln(z.m.hi, k), ph = ln(z.ph.hi, k);
    ws.mh[i] = mh;
    ws.ml[i] = ln(z.m.lo, k);
    ws.me[i] = ln(z.mexp, k);
    ws.ph[i] = ph;
    ws.pl[i] = ln(z.ph.lo, k);
    ws.ab[i] = (uint16_t)((ln(z.sa, k) > 0.0f ? 1 : 0) | (ln(z.q, k) << 4) |
                          ((ln(z.sb, k) > 0.0f ? 1 : 0) << 8));
    if (!isfinite(mh) || !isfinite(ph)) {
      atomicAdd(&ws.hdr->n_nonfinite, 1ull);
      atomicOr(&ws.hdr->flags, QCL_FLAG_NONFINITE);
    }
  }
}

}  // namespace qcl
