// kernels_split.cu -- many-mode two-state models (33..256 modes) on the FP32
// bulk path, in either representation.  A walker's modes are split over L warps (warp role r holds modes
// r NPL .. r NPL + NPL - 1 of the same 32 walker slots); a tile is 256 / L
// walkers.  Coefficient indices are warp-uniform: compile-time constant-bank
// operands with one copy of the unrolled code per role, or, where those copies
// would not fit the instruction cache, one copy for all roles reading the
// role's coefficients from shared memory (split_shared below).  For 65..100
// modes (four roles of 25 modes) each thread carries the walker in its slot of
// two consecutive tiles as the two lanes of packed FP32x2 values: every mode
// FMA of a step (half kicks, drift, collective sums) is one FFMA2 for both
// walkers, with the model coefficients as broadcast operands.  With one walker
// per thread (small ensembles, or more modes per warp) the same code runs on
// scalar lanes and gives the same bits.
//
// One exchange per step.  The coupling sums need the momentum after the second
// half kick, P'' = q - hu2 a - hv2 b with q = P' - (dt/2)(k R' + s) and
// hu2, hv2 known only once a(R'), b(R') are summed over all modes.  So each
// role sums a_j R'_j, b_j R'_j and the coupling sums over q,
// sum_j (a_j / M_j) q_j, sum_j (b_j / M_j) q_j, in its mode loop; the L roles'
// partials are exchanged together through shared memory under one named
// barrier of the group's warps and added in role order (every role then holds
// the same bits of the scalar state), and the second half kick's terms enter
// the coupling sums through the model constants
// sum_j a_j a_j / M_j, sum_j a_j b_j / M_j, sum_j b_j b_j / M_j:
//   Av = Xa - hu2 caa - hv2 cab,  Bv = Xb - hu2 cab - hv2 cbb.
// The momenta themselves are updated exactly as in the two-exchange form.
#include "bulk2.cuh"

namespace qcl {

namespace {

__device__ __forceinline__ void group_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Exchange buffer: per role and walker slot, the NV partial sums of a step
// (a R', a/M q; with KIND 1 also b R', b/M q), contiguous per thread.
template <typename V, int NV>
struct alignas(16) XVec {
  V v[NV];
};
template <typename V, int L, int BW, int NV>
struct XBuf {
  XVec<V, NV> x[L][BW];
};

// Warp-to-role mapping.  false: role = warp / G, so a walker group's L role
// warps sit on two of the four schedulers; true: role = warp % L, one role per
// scheduler (each scheduler then fetches one role's unrolled code).  Measured
// at 40-200 modes, both forms: the first is as fast or faster everywhere but
// on the 200-mode spin-boson model (7 %).
template <int NPL, int L, int KIND, int WPT>
constexpr bool split_rps() {
  return false;
}

// Where the coefficients come from.  false: constant-bank operands at
// compile-time offsets, one copy of the unrolled code per role; true: one
// copy of the code for all roles (the role is a runtime value), the role's
// coefficients loaded from shared memory (two broadcast loads per mode and
// kick).  The unrolled code of all roles has to fit the SM's instruction
// cache: four roles of the general form, or of 64 modes, do not (measured,
// 1e6 walkers: 100-mode general model 8.9e9 -> 1.35e10 walker-steps/s with one
// copy, 128 modes 3.3e9 -> 9.4e9, 200 modes 1.2e9 -> 5.5e9, 200-mode
// spin-boson 2.6e9 -> 7.5e9), while the spin-boson form of at most 32 modes
// per warp, and the general form on two roles, run faster with constant
// operands (100-mode spin-boson 2.83e10 against 2.06e10).
template <int NPL, int L, int KIND, int WPT>
constexpr bool split_shared() {
  return (KIND == 1 && L == 4) || NPL >= 64;
}

// One mode's coefficients: c0 = (dt/2 k, dt/M, a/M, b/M), c1 = (a, b, dt/2 s, 0).
struct ModeCoef {
  float hk, dtm, am, bm, a, b, hs;
};

template <int NPL, int L, int KIND, int ROLE, int WPT, bool SH>
__device__ __forceinline__ void split_tiles_v(const BulkParams& bp, const Coef2& cf, W32& ws,
                                              double* __restrict__ part, void* xbuf,
                                              double (*red)[8][32], float* obs_rows,
                                              unsigned int& n_deg, const float4* scoef,
                                              int role_rt) {
  using V = std::conditional_t<WPT == 2, float2, float>;
  using U = typename Lanes<V>::U;
  constexpr int BW = 256 / L;  // walkers per tile
  constexpr int G = BW / 32;   // groups (of 32 walkers) per tile
  const int role = SH ? role_rt : ROLE;
  const int OFF = role * NPL;
  // mode t's coefficients (all of them, or only a and b for the second kick)
  auto coef = [&](int t) {
    ModeCoef c;
    if constexpr (SH) {
      const float4 c0 = scoef[2 * (OFF + t)], c1 = scoef[2 * (OFF + t) + 1];
      c = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z};
    } else {
      c = {cf.hk[ROLE * NPL + t], cf.dtm[ROLE * NPL + t], cf.am[ROLE * NPL + t],
           cf.bm[ROLE * NPL + t], cf.a[ROLE * NPL + t],  cf.b[ROLE * NPL + t],
           cf.hs[ROLE * NPL + t]};
    }
    return c;
  };
  auto coef_ab = [&](int t) {
    if constexpr (SH) {
      const float2 ab = *reinterpret_cast<const float2*>(&scoef[2 * (OFF + t) + 1]);
      return ab;
    } else {
      return make_float2(cf.a[ROLE * NPL + t], cf.b[ROLE * NPL + t]);
    }
  };
  constexpr int NV = KIND == 1 ? 4 : 2;
  using X = XBuf<V, L, BW, NV>;
  using XV = XVec<V, NV>;
  // x[0]: sums at tile start; x[1], x[2]: the steps' sums, alternating (a warp
  // can run at most one barrier ahead of its partners, so the buffer it writes
  // is never the one they may still be reading)
  X* const x = reinterpret_cast<X*>(xbuf);
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = split_rps<NPL, L, KIND, WPT>() ? warp / L : warp % G;  // walker group in the tile
  const int wslot = grp * 32 + lane;  // walker slot within the tile
  const int bar_id = 1 + grp;         // named barrier of the group's L warps
  int rb = 0;
  for (int64_t tile0 = (int64_t)blockIdx.x * WPT; tile0 < bp.n_tiles;
       tile0 += (int64_t)gridDim.x * WPT) {
    // every warp of the group has finished the previous tiles' exchanges
    group_sync(bar_id, 32 * L);
    WalkerV<NPL, V> w;
    ScalV<V> z;
    bool active[WPT];
    U deg;
    PhiloxStream rng[WPT];
    u4 wd[WPT];
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      const int64_t i = (tile0 + k) * BW + wslot;
      active[k] = i < nt;
      const int64_t ii = active[k] ? i : 0;
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        const bool on = active[k] && OFF + t < bp.n;
        ln(w.R[t], k) = on ? ws.R[(int64_t)(OFF + t) * nt + ii] : 0.0f;
        ln(w.P[t], k) = on ? ws.P[(int64_t)(OFF + t) * nt + ii] : 0.0f;
      }
      ln(z.m.hi, k) = active[k] ? ws.mh[ii] : 0.0f;
      ln(z.m.lo, k) = active[k] ? ws.ml[ii] : 0.0f;
      ln(z.mexp, k) = active[k] ? ws.me[ii] : 0;
      ln(z.ph.hi, k) = active[k] ? ws.ph[ii] : 0.0f;
      ln(z.ph.lo, k) = active[k] ? ws.pl[ii] : 0.0f;
      const uint32_t ab = active[k] ? ws.ab[ii] : 0u;
      ln(z.sa, k) = sgn(ab & 0xf);
      ln(z.sb, k) = sgn((ab >> 8) & 0xf);
      ln(z.q, k) = 0;
      ln(deg, k) = 0u;
      rng[k] = PhiloxStream(bp.seed, bp.traj_offset + (uint64_t)ii, kPurposeHop);
    }

    // sums over the L roles of per-role partials, in role order
    auto exchange = [&](X& xb, XV& v) {
      xb.x[role][wslot] = v;
      group_sync(bar_id, 32 * L);
      v = xb.x[0][wslot];
#pragma unroll
      for (int r = 1; r < L; ++r) {
        const XV o = xb.x[r][wslot];
#pragma unroll
        for (int c = 0; c < NV; ++c) v.v[c] = vadd(v.v[c], o.v[c]);
      }
    };

    {
      XV v;
#pragma unroll
      for (int c = 0; c < NV; ++c) v.v[c] = splat<V>(0.0f);
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        const float2 ab = coef_ab(t);
        v.v[0] = vfma(splat<V>(ab.x), w.R[t], v.v[0]);
        if (KIND == 1) v.v[2] = vfma(splat<V>(ab.y), w.R[t], v.v[2]);
      }
      exchange(x[0], v);
      z.A = vadd(splat<V>(bp.a0), v.v[0]);
      z.B = vadd(splat<V>(bp.b0), (KIND == 1) ? v.v[2] : splat<V>(0.0f));
    }
    closed_form(z);

    // observation by the role-0 warps, lane by lane, then the tiles' trees
    auto observe = [&](int slot) {
      if (role == 0) {
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
          Scal zk = lane_of(z, k);
          observe_warp<false, false>(zk, active[k], obs_rows, wslot, grp * 32, lane,
                                     red[WPT * rb + k][grp]);
          set_lane(z, k, zk);
        }
      }
      __syncthreads();
      if (warp < WPT && tile0 + warp < bp.n_tiles) {
        const double* r = &red[WPT * rb + warp][0][0];
        double t0;
        if (G == 1) t0 = r[lane];
        else if (G == 2) t0 = r[lane] + r[32 + lane];
        else t0 = (r[lane] + r[32 + lane]) + (r[64 + lane] + r[96 + lane]);
        part[((int64_t)slot * bp.n_tiles + tile0 + warp) * 32 + lane] = t0;
      }
      rb ^= 1;
    };

    int slot = bp.obs_first;
    if (bp.obs_first) observe(0);
    int to_out = bp.to_out0;
    uint32_t blk = bp.blk0;
    int widx = bp.widx0;
    int xsel = 0;
#pragma unroll
    for (int k = 0; k < WPT; ++k) wd[k] = rng[k].draw(blk);
    for (int it = 0; it < bp.len; ++it) {
      U word;
#pragma unroll
      for (int k = 0; k < WPT; ++k) ln(word, k) = pick_word(wd[k], widx);
      const V hsab = vmul(splat<V>(bp.hdt * 0.5f), vadd(z.sa, z.sb));
      const V hu = vmul(hsab, z.c2), hv = vmul(hsab, z.s2);
      XV v;  // a R', a/M q (, b R', b/M q)
#pragma unroll
      for (int c = 0; c < NV; ++c) v.v[c] = splat<V>(0.0f);
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        // first half kick at R_n, drift, then the R_{n+1} terms of the second
        // half kick (q); its coupling terms wait for the exchange
        const ModeCoef c = coef(t);
        V p = vfma(splat<V>(-c.hk), w.R[t], w.P[t]);
        if (KIND == 1) p = vadd(p, splat<V>(-c.hs));
        p = vfma(hu, splat<V>(-c.a), p);
        if (KIND == 1) p = vfma(hv, splat<V>(-c.b), p);
        const V r = vfma(splat<V>(c.dtm), p, w.R[t]);
        w.R[t] = r;
        v.v[0] = vfma(splat<V>(c.a), r, v.v[0]);
        if (KIND == 1) v.v[2] = vfma(splat<V>(c.b), r, v.v[2]);
        V qm = vfma(splat<V>(-c.hk), r, p);
        if (KIND == 1) qm = vadd(qm, splat<V>(-c.hs));
        w.P[t] = qm;
        v.v[1] = vfma(splat<V>(c.am), qm, v.v[1]);
        if (KIND == 1) v.v[3] = vfma(splat<V>(c.bm), qm, v.v[3]);
      }
      const V r_old = z.r;
      exchange(x[1 + xsel], v);
      xsel ^= 1;
      z.A = vadd(splat<V>(bp.a0), v.v[0]);
      z.B = vadd(splat<V>(bp.b0), (KIND == 1) ? v.v[2] : splat<V>(0.0f));
      closed_form<KIND == 1>(z);
      const V hu2 = vmul(hsab, z.c2), hv2 = vmul(hsab, z.s2);
#pragma unroll
      for (int t = 0; t < NPL; ++t) {  // coupling terms of the second half kick at R_{n+1}
        const float2 ab = coef_ab(t);
        V p = vfma(hu2, splat<V>(-ab.x), w.P[t]);
        if (KIND == 1) p = vfma(hv2, splat<V>(-ab.y), p);
        w.P[t] = p;
      }
      // coupling sums at P_{n+1}: the q sums less the kick's coupling terms
      V Av = vfma(hu2, splat<V>(-bp.caa), v.v[1]), Bv = splat<V>(0.0f);
      if (KIND == 1) {
        Av = vfma(hv2, splat<V>(-bp.cab), Av);
        Bv = vfma(hu2, splat<V>(-bp.cab), v.v[3]);
        Bv = vfma(hv2, splat<V>(-bp.cbb), Bv);
      }
      // only role 0 keeps the weight and phase (it observes and stores them);
      // the other roles need the index pair alone
      // (the split kernel keeps the per-step range check and the packed phase
      // update: measured faster here than the branch-free form)
      if (role == 0) phase_and_transition<KIND, true>(z, r_old, Av, Bv, word, bp, deg);
      else phase_and_transition<KIND, false>(z, r_old, Av, Bv, word, bp, deg);
      if (++widx == 4) {  // pairs renormalised at the end of every Philox block
        widx = 0;
        if (role == 0) block_end<false>(z);
        ++blk;
        if (it + 1 < bp.len) {
#pragma unroll
          for (int k = 0; k < WPT; ++k) wd[k] = rng[k].draw(blk);
        }
      }
      if (--to_out == 0) {
        observe(slot++);
        to_out = bp.stride;
      }
    }
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      if (!active[k]) continue;
      const int64_t i = (tile0 + k) * BW + wslot;
      n_deg += ln(deg, k);
#pragma unroll
      for (int t = 0; t < NPL; ++t)
        if (OFF + t < bp.n) {
          ws.R[(int64_t)(OFF + t) * nt + i] = ln(w.R[t], k);
          ws.P[(int64_t)(OFF + t) * nt + i] = ln(w.P[t], k);
        }
      if (role == 0) {
        const float mh = ln(z.m.hi, k), ph = ln(z.ph.hi, k);
        ws.mh[i] = mh;
        ws.ml[i] = ln(z.m.lo, k);
        ws.me[i] = ln(z.mexp, k);
        ws.ph[i] = ph;
        ws.pl[i] = ln(z.ph.lo, k);
        ws.ab[i] = (uint16_t)((ln(z.sa, k) > 0.0f ? 1 : 0) | ((ln(z.sb, k) > 0.0f ? 1 : 0) << 8));
        if (!isfinite(mh) || !isfinite(ph)) {
          atomicAdd(&ws.hdr->n_nonfinite, 1ull);
          atomicOr(&ws.hdr->flags, QCL_FLAG_NONFINITE);
        }
      }
    }
  }
}

// The diabatic representation (two states, 33..256 modes) on the same split:
// the diagonal mean force is a constant of the pair, so both half kicks and
// the drift run in one mode loop, and the transition (a -> 1 - a, b -> 1 - b
// with amplitude -/+ i b(R_{n+1}) dt / hbar) needs only a(R_{n+1}) and
// b(R_{n+1}): one exchange of those sums per step, no momentum sums.  The
// scalar step is the one-thread-per-walker kernel's (dia_phase_and_transition);
// role 0 keeps the weight's range checked every step (as in the adiabatic split
// kernel) and observes.
template <int NPL, int L, int KIND, int ROLE, int WPT, bool SH>
__device__ __forceinline__ void split_tiles_dia(const BulkParams& bp, const Coef2& cf, W32& ws,
                                                double* __restrict__ part, void* xbuf,
                                                double (*red)[8][32], float* obs_rows,
                                                const float4* scoef, int role_rt) {
  using V = std::conditional_t<WPT == 2, float2, float>;
  using U = typename Lanes<V>::U;
  constexpr int BW = 256 / L;
  constexpr int G = BW / 32;
  const int role = SH ? role_rt : ROLE;
  const int OFF = role * NPL;
  auto coef = [&](int t) {
    ModeCoef c;
    if constexpr (SH) {
      const float4 c0 = scoef[2 * (OFF + t)], c1 = scoef[2 * (OFF + t) + 1];
      c = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z};
    } else {
      c = {cf.hk[ROLE * NPL + t], cf.dtm[ROLE * NPL + t], cf.am[ROLE * NPL + t],
           cf.bm[ROLE * NPL + t], cf.a[ROLE * NPL + t],  cf.b[ROLE * NPL + t],
           cf.hs[ROLE * NPL + t]};
    }
    return c;
  };
  constexpr int NV = KIND == 1 ? 2 : 1;  // a R (, b R)
  using X = XBuf<V, L, BW, NV>;
  using XV = XVec<V, NV>;
  X* const x = reinterpret_cast<X*>(xbuf);
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp % G;
  const int wslot = grp * 32 + lane;
  const int bar_id = 1 + grp;
  int rb = 0;
  for (int64_t tile0 = (int64_t)blockIdx.x * WPT; tile0 < bp.n_tiles;
       tile0 += (int64_t)gridDim.x * WPT) {
    group_sync(bar_id, 32 * L);
    WalkerV<NPL, V> w;
    ScalV<V> z;
    bool active[WPT];
    PhiloxStream rng[WPT];
    u4 wd[WPT];
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      const int64_t i = (tile0 + k) * BW + wslot;
      active[k] = i < nt;
      const int64_t ii = active[k] ? i : 0;
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        const bool on = active[k] && OFF + t < bp.n;
        ln(w.R[t], k) = on ? ws.R[(int64_t)(OFF + t) * nt + ii] : 0.0f;
        ln(w.P[t], k) = on ? ws.P[(int64_t)(OFF + t) * nt + ii] : 0.0f;
      }
      ln(z.m.hi, k) = active[k] ? ws.mh[ii] : 0.0f;
      ln(z.m.lo, k) = active[k] ? ws.ml[ii] : 0.0f;
      ln(z.mexp, k) = active[k] ? ws.me[ii] : 0;
      ln(z.ph.hi, k) = active[k] ? ws.ph[ii] : 0.0f;
      ln(z.ph.lo, k) = active[k] ? ws.pl[ii] : 0.0f;
      const uint32_t ab = active[k] ? ws.ab[ii] : 0u;  // alpha | q << 4 | beta << 8
      ln(z.sa, k) = sgn(ab & 0xf);
      ln(z.sb, k) = sgn((ab >> 8) & 0xf);
      ln(z.q, k) = (int)((ab >> 4) & 3u);
      rng[k] = PhiloxStream(bp.seed, bp.traj_offset + (uint64_t)ii, kPurposeHop);
    }
    auto exchange = [&](X& xb, XV& v) {
      xb.x[role][wslot] = v;
      group_sync(bar_id, 32 * L);
      v = xb.x[0][wslot];
#pragma unroll
      for (int r = 1; r < L; ++r) {
        const XV o = xb.x[r][wslot];
#pragma unroll
        for (int c = 0; c < NV; ++c) v.v[c] = vadd(v.v[c], o.v[c]);
      }
    };
    // a(R), b(R): b0 + b R stays b0 for the spin-boson form
    auto sums = [&](X& xb, XV& v) {
      exchange(xb, v);
      z.A = vadd(splat<V>(bp.a0), v.v[0]);
      z.B = (KIND == 1) ? vadd(splat<V>(bp.b0), v.v[NV - 1]) : splat<V>(bp.b0);
    };
    {
      XV v;
#pragma unroll
      for (int c = 0; c < NV; ++c) v.v[c] = splat<V>(0.0f);
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        const ModeCoef c = coef(t);
        v.v[0] = vfma(splat<V>(c.a), w.R[t], v.v[0]);
        if (KIND == 1) v.v[NV - 1] = vfma(splat<V>(c.b), w.R[t], v.v[NV - 1]);
      }
      sums(x[0], v);
    }
    auto observe = [&](int slot) {
      if (role == 0) {
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
          Scal zk = lane_of(z, k);
          observe_warp<true, false>(zk, active[k], obs_rows, wslot, grp * 32, lane,
                                    red[WPT * rb + k][grp]);
          set_lane(z, k, zk);
        }
      }
      __syncthreads();
      if (warp < WPT && tile0 + warp < bp.n_tiles) {
        const double* r = &red[WPT * rb + warp][0][0];
        double t0;
        if (G == 1) t0 = r[lane];
        else if (G == 2) t0 = r[lane] + r[32 + lane];
        else t0 = (r[lane] + r[32 + lane]) + (r[64 + lane] + r[96 + lane]);
        part[((int64_t)slot * bp.n_tiles + tile0 + warp) * 32 + lane] = t0;
      }
      rb ^= 1;
    };

    int slot = bp.obs_first;
    if (bp.obs_first) observe(0);
    int to_out = bp.to_out0;
    uint32_t blk = bp.blk0;
    int widx = bp.widx0;
    int xsel = 0;
#pragma unroll
    for (int k = 0; k < WPT; ++k) wd[k] = rng[k].draw(blk);
    for (int it = 0; it < bp.len; ++it) {
      U word;
#pragma unroll
      for (int k = 0; k < WPT; ++k) ln(word, k) = pick_word(wd[k], widx);
      const V hsab = vmul(splat<V>(bp.hdt * 0.5f), vadd(z.sa, z.sb));
      XV v;
#pragma unroll
      for (int c = 0; c < NV; ++c) v.v[c] = splat<V>(0.0f);
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        // half kick with the pair's diagonal force, drift, a and b at
        // R_{n+1}, the second half kick (the same force)
        const ModeCoef c = coef(t);
        V p = vfma(splat<V>(-c.hk), w.R[t], w.P[t]);
        if (KIND == 1) p = vadd(p, splat<V>(-c.hs));
        p = vfma(hsab, splat<V>(c.a), p);
        const V r = vfma(splat<V>(c.dtm), p, w.R[t]);
        w.R[t] = r;
        v.v[0] = vfma(splat<V>(c.a), r, v.v[0]);
        if (KIND == 1) v.v[NV - 1] = vfma(splat<V>(c.b), r, v.v[NV - 1]);
        p = vfma(splat<V>(-c.hk), r, p);
        if (KIND == 1) p = vadd(p, splat<V>(-c.hs));
        w.P[t] = vfma(hsab, splat<V>(c.a), p);
      }
      const V a_old = z.A;
      sums(x[1 + xsel], v);
      xsel ^= 1;
      if (role == 0) dia_phase_and_transition<true>(z, a_old, z.B, word, bp);
      else dia_phase_and_transition<false>(z, a_old, z.B, word, bp);
      if (++widx == 4) {
        widx = 0;
        if (role == 0) block_end<false>(z);
        ++blk;
        if (it + 1 < bp.len) {
#pragma unroll
          for (int k = 0; k < WPT; ++k) wd[k] = rng[k].draw(blk);
        }
      }
      if (--to_out == 0) {
        observe(slot++);
        to_out = bp.stride;
      }
    }
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
      if (!active[k]) continue;
      const int64_t i = (tile0 + k) * BW + wslot;
#pragma unroll
      for (int t = 0; t < NPL; ++t)
        if (OFF + t < bp.n) {
          ws.R[(int64_t)(OFF + t) * nt + i] = ln(w.R[t], k);
          ws.P[(int64_t)(OFF + t) * nt + i] = ln(w.P[t], k);
        }
      if (role == 0) {
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
  }
}

}  // namespace

template <int NPL, int L, int KIND, int WPT, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_bulk2_split2(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
  static_assert(L == 2 || L == 4, "two or four roles");
  using V = std::conditional_t<WPT == 2, float2, float>;
  constexpr int BW = 256 / L;
  // exchange buffers: the sums at tile start and two alternating for the steps
  __shared__ __align__(16) XBuf<V, L, BW, KIND == 1 ? 4 : 2> xbuf[3];
  __shared__ double red[2 * WPT][8][32];
  __shared__ __align__(16) float obs_rows[BW * kObsRow];
  W32 ws = view32(buf, bp.n_traj, 2, bp.n);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  unsigned int n_deg = 0;
  // (the warp-to-role mapping: split_rps above)
  const int warp = threadIdx.x >> 5;
  const int role = split_rps<NPL, L, KIND, WPT>() ? warp % L : warp / (BW / 32);
  if constexpr (split_shared<NPL, L, KIND, WPT>()) {
    __shared__ float4 scoef[2 * L * NPL];
    for (int i = threadIdx.x; i < L * NPL; i += blockDim.x) {
      scoef[2 * i] = make_float4(cf.hk[i], cf.dtm[i], cf.am[i], cf.bm[i]);
      scoef[2 * i + 1] = make_float4(cf.a[i], cf.b[i], cf.hs[i], 0.0f);
    }
    __syncthreads();
    split_tiles_v<NPL, L, KIND, 0, WPT, true>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg, scoef,
                                              role);
  } else {
    if (role == 0)
      split_tiles_v<NPL, L, KIND, 0, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg,
                                                 nullptr, 0);
    else if (role == 1)
      split_tiles_v<NPL, L, KIND, 1, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg,
                                                 nullptr, 1);
    else if (role == 2)
      split_tiles_v<NPL, L, KIND, 2 % L, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg,
                                                     nullptr, 2);
    else
      split_tiles_v<NPL, L, KIND, 3 % L, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg,
                                                     nullptr, 3);
  }
  if (n_deg && role == 0) {  // every role counted the same walkers
    atomicAdd(&ws.hdr->n_degenerate, (unsigned long long)n_deg);
    atomicOr(&ws.hdr->flags, QCL_FLAG_DEGENERATE);
  }
}

namespace {
// Resident blocks per SM the launch bounds ask for: two for the spin-boson
// form with at most 32 modes per warp and one walker per thread (the state fits
// 128 registers), else one.
template <int NPL, int KIND, int WPT>
constexpr int split_minb() {
  return (KIND == 0 && NPL <= 32 && WPT == 1) ? 2 : 1;
}

template <int NPL, int L, int KIND, int WPT>
BulkFn split_fn() {
  return k_bulk2_split2<NPL, L, KIND, WPT, split_minb<NPL, KIND, WPT>()>;
}

// Two walkers per thread where a warp holds at most 25 modes (twice its modes'
// R and P must fit the registers); otherwise one.
template <int NPL, int L, int KIND>
int run_split(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
              const LaunchShape& ls, cudaStream_t st) {
  static int per_sm[2] = {-1, -1}, n_sm[2] = {0, 0};
  if constexpr (NPL <= 25) {
    int wpt = (ls.wpt > 0 ? ls.wpt : 2) >= 2 ? 2 : 1;
    if (wpt == 2) wpt = bulk_wpt(split_fn<NPL, L, KIND, 2>(), per_sm[1], n_sm[1], bp.n_tiles, ls);
    if (wpt == 2)
      return run_bulk_kernel(split_fn<NPL, L, KIND, 2>(), per_sm[1], n_sm[1], bp, cf, buf, part,
                             ls, 2, st);
  }
  return run_bulk_kernel(split_fn<NPL, L, KIND, 1>(), per_sm[0], n_sm[0], bp, cf, buf, part, ls,
                         1, st);
}

// warps per walker must agree with bulk_lanes(n)
template <int KIND>
int dispatch_split(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                   const LaunchShape& ls, cudaStream_t st) {
  const int n = bp.n;
  if (n <= 64) return run_split<32, 2, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 100) return run_split<25, 4, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 128) return run_split<32, 4, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 256) return run_split<64, 4, KIND>(bp, cf, buf, part, ls, st);
  return 0;
}
}  // namespace

int launch_bulk2_split(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                       const LaunchShape& ls, cudaStream_t st) {
  return bp.kind == 0 ? dispatch_split<0>(bp, cf, buf, part, ls, st)
                      : dispatch_split<1>(bp, cf, buf, part, ls, st);
}

BulkFn bulk2_split_fn(int n, int kind, int wpt) {
  const bool two = wpt == 2 && n > 64 && n <= 100;
  if (n <= 64) return kind == 0 ? split_fn<32, 2, 0, 1>() : split_fn<32, 2, 1, 1>();
  if (n <= 100) {
    if (kind == 0) return two ? split_fn<25, 4, 0, 2>() : split_fn<25, 4, 0, 1>();
    return two ? split_fn<25, 4, 1, 2>() : split_fn<25, 4, 1, 1>();
  }
  if (n <= 128) return kind == 0 ? split_fn<32, 4, 0, 1>() : split_fn<32, 4, 1, 1>();
  if (n <= 256) return kind == 0 ? split_fn<64, 4, 0, 1>() : split_fn<64, 4, 1, 1>();
  return nullptr;
}

// The diabatic split kernel (two states, 33..256 modes): split_tiles_dia over
// the same roles, tiles and exchange buffers as k_bulk2_split2.
template <int NPL, int L, int KIND, int WPT, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_bulk2_split_dia(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
  static_assert(L == 2 || L == 4, "two or four roles");
  using V = std::conditional_t<WPT == 2, float2, float>;
  constexpr int BW = 256 / L;
  __shared__ __align__(16) XBuf<V, L, BW, KIND == 1 ? 2 : 1> xbuf[3];
  __shared__ double red[2 * WPT][8][32];
  __shared__ __align__(16) float obs_rows[BW * kObsRow];
  W32 ws = view32(buf, bp.n_traj, 2, bp.n);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  const int role = (threadIdx.x >> 5) / (BW / 32);
  if constexpr (split_shared<NPL, L, KIND, WPT>()) {
    __shared__ float4 scoef[2 * L * NPL];
    for (int i = threadIdx.x; i < L * NPL; i += blockDim.x) {
      scoef[2 * i] = make_float4(cf.hk[i], cf.dtm[i], cf.am[i], cf.bm[i]);
      scoef[2 * i + 1] = make_float4(cf.a[i], cf.b[i], cf.hs[i], 0.0f);
    }
    __syncthreads();
    split_tiles_dia<NPL, L, KIND, 0, WPT, true>(bp, cf, ws, part, xbuf, red, obs_rows, scoef,
                                                role);
  } else {
    if (role == 0)
      split_tiles_dia<NPL, L, KIND, 0, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows,
                                                   nullptr, 0);
    else if (role == 1)
      split_tiles_dia<NPL, L, KIND, 1, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows,
                                                   nullptr, 1);
    else if (role == 2)
      split_tiles_dia<NPL, L, KIND, 2 % L, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows,
                                                       nullptr, 2);
    else
      split_tiles_dia<NPL, L, KIND, 3 % L, WPT, false>(bp, cf, ws, part, xbuf, red, obs_rows,
                                                       nullptr, 3);
  }
}

namespace {
// (two resident blocks per SM for the spin-boson form with at most 32 modes
// per warp and one walker per thread, as in the adiabatic split kernel: the
// general form would spill at the 128 registers that takes)
template <int NPL, int L, int KIND, int WPT>
BulkFn split_dia_fn() {
  return k_bulk2_split_dia<NPL, L, KIND, WPT, split_minb<NPL, KIND, WPT>()>;
}

// Two walkers per thread (packed FP32x2 lanes) where a warp holds at most 25
// modes, as in the adiabatic split kernel; otherwise one.
template <int NPL, int L, int KIND>
int run_split_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                  const LaunchShape& ls, cudaStream_t st) {
  static int per_sm[2] = {-1, -1}, n_sm[2] = {0, 0};
  if constexpr (NPL <= 25) {
    int wpt = (ls.wpt > 0 ? ls.wpt : 2) >= 2 ? 2 : 1;
    if (wpt == 2)
      wpt = bulk_wpt(split_dia_fn<NPL, L, KIND, 2>(), per_sm[1], n_sm[1], bp.n_tiles, ls);
    if (wpt == 2)
      return run_bulk_kernel(split_dia_fn<NPL, L, KIND, 2>(), per_sm[1], n_sm[1], bp, cf, buf,
                             part, ls, 2, st);
  }
  return run_bulk_kernel(split_dia_fn<NPL, L, KIND, 1>(), per_sm[0], n_sm[0], bp, cf, buf, part,
                         ls, 1, st);
}

// warps per walker must agree with bulk_lanes(n)
template <int KIND>
int dispatch_split_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                       const LaunchShape& ls, cudaStream_t st) {
  const int n = bp.n;
  if (n <= 64) return run_split_dia<32, 2, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 100) return run_split_dia<25, 4, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 128) return run_split_dia<32, 4, KIND>(bp, cf, buf, part, ls, st);
  if (n <= 256) return run_split_dia<64, 4, KIND>(bp, cf, buf, part, ls, st);
  return 0;
}
}  // namespace

int launch_bulk2_split_dia(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                           const LaunchShape& ls, cudaStream_t st) {
  return bp.kind == 0 ? dispatch_split_dia<0>(bp, cf, buf, part, ls, st)
                      : dispatch_split_dia<1>(bp, cf, buf, part, ls, st);
}

BulkFn bulk2_split_dia_fn(int n, int kind, int wpt) {
  const bool two = wpt == 2 && n > 64 && n <= 100;
  if (n <= 64) return kind == 0 ? split_dia_fn<32, 2, 0, 1>() : split_dia_fn<32, 2, 1, 1>();
  if (n <= 100) {
    if (kind == 0) return two ? split_dia_fn<25, 4, 0, 2>() : split_dia_fn<25, 4, 0, 1>();
    return two ? split_dia_fn<25, 4, 1, 2>() : split_dia_fn<25, 4, 1, 1>();
  }
  if (n <= 128) return kind == 0 ? split_dia_fn<32, 4, 0, 1>() : split_dia_fn<32, 4, 1, 1>();
  if (n <= 256) return kind == 0 ? split_dia_fn<64, 4, 0, 1>() : split_dia_fn<64, 4, 1, 1>();
  return nullptr;
}

}  // namespace qcl
