// kernels_split.cu -- many-mode two-state models (65..100 modes) on the FP32
// bulk path with two walkers per thread.  A walker's modes are split over four
// warps (warp role r holds modes r NPL .. r NPL + NPL - 1 of the same 32 walker
// slots), and each thread carries the walker in that slot of two consecutive
// 64-walker tiles as the two lanes of packed FP32x2 values: every mode FMA of a
// step (half kicks, drift, collective sums) is one FFMA2 for both walkers, with
// the model coefficients as broadcast constant-bank operands.  With one walker
// per thread (small ensembles) the same code runs on scalar lanes and gives the
// same bits.
//
// One exchange per step.  The coupling sums need the momentum after the second
// half kick, P'' = q - hu2 a - hv2 b with q = P' - (dt/2)(k R' + s) and
// hu2, hv2 known only once a(R'), b(R') are summed over all modes.  So each
// role sums a_j R'_j, b_j R'_j and the coupling sums over q,
// sum_j (a_j / M_j) q_j, sum_j (b_j / M_j) q_j, in its mode loop; the four
// partials of the four roles are exchanged together through shared memory under
// one named barrier of the group's warps and added in role order (every role
// then holds the same bits of the scalar state), and the second half kick's
// terms enter the coupling sums through the model constants
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

template <int NPL, int L, int KIND, int ROLE, int WPT>
__device__ __forceinline__ void split_tiles_v(const BulkParams& bp, const Coef2& cf, W32& ws,
                                              double* __restrict__ part, void* xbuf,
                                              double (*red)[8][32], float* obs_rows,
                                              unsigned int& n_deg) {
  using V = std::conditional_t<WPT == 2, float2, float>;
  using U = typename Lanes<V>::U;
  constexpr int BW = 256 / L;  // walkers per tile
  constexpr int G = BW / 32;   // groups (of 32 walkers) per tile
  constexpr int OFF = ROLE * NPL;
  constexpr int NV = KIND == 1 ? 4 : 2;
  using X = XBuf<V, L, BW, NV>;
  using XV = XVec<V, NV>;
  // x[0]: sums at tile start; x[1], x[2]: the steps' sums, alternating (a warp
  // can run at most one barrier ahead of its partners, so the buffer it writes
  // is never the one they may still be reading)
  X* const x = reinterpret_cast<X*>(xbuf);
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp % G;           // this warp's walker group in the tile
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
      xb.x[ROLE][wslot] = v;
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
        v.v[0] = vfma(splat<V>(cf.a[OFF + t]), w.R[t], v.v[0]);
        if (KIND == 1) v.v[2] = vfma(splat<V>(cf.b[OFF + t]), w.R[t], v.v[2]);
      }
      exchange(x[0], v);
      z.A = vadd(splat<V>(bp.a0), v.v[0]);
      z.B = vadd(splat<V>(bp.b0), (KIND == 1) ? v.v[2] : splat<V>(0.0f));
    }
    closed_form(z);

    // observation by the role-0 warps, lane by lane, then the tiles' trees
    auto observe = [&](int slot) {
      if (ROLE == 0) {
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
        V p = vfma(splat<V>(-cf.hk[OFF + t]), w.R[t], w.P[t]);
        if (KIND == 1) p = vadd(p, splat<V>(-cf.hs[OFF + t]));
        p = vfma(hu, splat<V>(-cf.a[OFF + t]), p);
        if (KIND == 1) p = vfma(hv, splat<V>(-cf.b[OFF + t]), p);
        const V r = vfma(splat<V>(cf.dtm[OFF + t]), p, w.R[t]);
        w.R[t] = r;
        v.v[0] = vfma(splat<V>(cf.a[OFF + t]), r, v.v[0]);
        if (KIND == 1) v.v[2] = vfma(splat<V>(cf.b[OFF + t]), r, v.v[2]);
        V qm = vfma(splat<V>(-cf.hk[OFF + t]), r, p);
        if (KIND == 1) qm = vadd(qm, splat<V>(-cf.hs[OFF + t]));
        w.P[t] = qm;
        v.v[1] = vfma(splat<V>(cf.am[OFF + t]), qm, v.v[1]);
        if (KIND == 1) v.v[3] = vfma(splat<V>(cf.bm[OFF + t]), qm, v.v[3]);
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
        V p = vfma(hu2, splat<V>(-cf.a[OFF + t]), w.P[t]);
        if (KIND == 1) p = vfma(hv2, splat<V>(-cf.b[OFF + t]), p);
        w.P[t] = p;
      }
      // coupling sums at P_{n+1}: the q sums less the kick's coupling terms
      V Av = vfma(hu2, splat<V>(-bp.caa), v.v[1]), Bv = splat<V>(0.0f);
      if (KIND == 1) {
        Av = vfma(hv2, splat<V>(-bp.cab), Av);
        Bv = vfma(hu2, splat<V>(-bp.cab), v.v[3]);
        Bv = vfma(hv2, splat<V>(-bp.cbb), Bv);
      }
      phase_and_transition<KIND>(z, r_old, Av, Bv, word, bp, deg);
      if (++widx == 4) {  // pairs renormalised at the end of every Philox block
        widx = 0;
        block_end(z);
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
      if (ROLE == 0) {
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

}  // namespace

template <int NPL, int L, int KIND, int WPT>
__global__ void __launch_bounds__(256, 1)
    k_bulk2_split2(const BulkParams bp, const Coef2 cf, void* buf, double* __restrict__ part) {
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
  static_assert(L == 4, "four roles");
  unsigned int n_deg = 0;
  // role = warp / G.  (Measured: role = warp % L, which puts one role's warps
  // on each scheduler, is 6 % slower with two walkers per thread -- longer
  // barrier waits -- though 11 % faster with one.)
  const int role = (threadIdx.x >> 5) / (BW / 32);
  if (role == 0)
    split_tiles_v<NPL, L, KIND, 0, WPT>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg);
  else if (role == 1)
    split_tiles_v<NPL, L, KIND, 1, WPT>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg);
  else if (role == 2)
    split_tiles_v<NPL, L, KIND, 2, WPT>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg);
  else
    split_tiles_v<NPL, L, KIND, 3, WPT>(bp, cf, ws, part, xbuf, red, obs_rows, n_deg);
  if (n_deg && role == 0) {  // every role counted the same walkers
    atomicAdd(&ws.hdr->n_degenerate, (unsigned long long)n_deg);
    atomicOr(&ws.hdr->flags, QCL_FLAG_DEGENERATE);
  }
}

namespace {
template <int KIND>
int run_split2(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
               const LaunchShape& ls, cudaStream_t st) {
  constexpr int NPL = 25, L = 4;
  static int per_sm[2] = {-1, -1}, n_sm[2] = {0, 0};
  int wpt = (ls.wpt > 0 ? ls.wpt : default_wpt(65)) >= 2 ? 2 : 1;
  if (wpt == 2) wpt = bulk_wpt(k_bulk2_split2<NPL, L, KIND, 2>, per_sm[1], n_sm[1], bp.n_tiles, ls);
  if (wpt == 2)
    return run_bulk_kernel(k_bulk2_split2<NPL, L, KIND, 2>, per_sm[1], n_sm[1], bp, cf, buf, part,
                           ls, 2, st);
  return run_bulk_kernel(k_bulk2_split2<NPL, L, KIND, 1>, per_sm[0], n_sm[0], bp, cf, buf, part,
                         ls, 1, st);
}
}  // namespace

int launch_bulk2_split2(const BulkParams& bp, const Coef2& cf, void* buf, double* part,
                        const LaunchShape& ls, cudaStream_t st) {
  return bp.kind == 0 ? run_split2<0>(bp, cf, buf, part, ls, st)
                      : run_split2<1>(bp, cf, buf, part, ls, st);
}

BulkFn bulk2_split2_fn(int kind, int wpt) {
  constexpr int NPL = 25, L = 4;
  if (kind == 0) return wpt == 2 ? k_bulk2_split2<NPL, L, 0, 2> : k_bulk2_split2<NPL, L, 0, 1>;
  return wpt == 2 ? k_bulk2_split2<NPL, L, 1, 2> : k_bulk2_split2<NPL, L, 1, 1>;
}

}  // namespace qcl
