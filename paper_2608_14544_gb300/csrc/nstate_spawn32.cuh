// nstate_spawn32.cuh -- trajectory spawning of N_s-state models in FP32 bulk
// precision (the FP32 walker arithmetic of nstate_bulk.cuh, one step per
// launch).
#pragma once
#include "nstate_bulk.cuh"

namespace qcl {

// ------------------------------------------------------ FP32 spawning, N_s --
// Trajectory spawning for N_s-state models in FP32 bulk precision (either
// representation, any mode count: up to 8 modes in registers, beyond that in
// memory): one step per launch with the walker state in HBM, the walker
// arithmetic of the FP32 N_s-state kernels (the carried eigenvectors and
// eigenvalues warm-start each decomposition; the diabatic step needs none),
// compensated FP32 weight and phase pairs with a carried exponent.  A fired test stages a child (weight m A_e / p_hat_e, the event's
// quarter turns) and leaves the walker in place; the count / scan / scatter is
// the FP64 scheme's.  Family observation accumulated in FP64.
struct SetN32 {
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
  float* U;  // [NS * NS][cap]
  float* E;  // [NS][cap]
};

__device__ __forceinline__ SetN32 spawn_setN32(void* buf, const SpawnLayout& L, int set) {
  char* b = (char*)buf + L.set_off[set];
  return {(float*)(b + L.R),     (float*)(b + L.P),      (float*)(b + L.m),
          (float*)(b + L.mlo),   (int32_t*)(b + L.mexp), (float*)(b + L.phi),
          (float*)(b + L.philo), (uint16_t*)(b + L.ab),  (uint64_t*)(b + L.id),
          (uint32_t*)(b + L.fam), (float*)(b + L.U),     (float*)(b + L.E)};
}

template <int NS>
__global__ void __launch_bounds__(128) k_spawnN_sample32(const SampleN32 sp, int64_t cap, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n0 = sp.n_traj;
  const SpawnLayout L = SpawnLayout::make(cap, sp.n, n0, QCL_PREC_FP32_BULK, NS);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = (SpawnHeader*)((char*)buf + kSpawnHeaderOff);
  if (i == 0) {
    hdr->magic = kEnsMagic;
    hdr->n_traj = n0;
    hdr->precision = QCL_PREC_FP32_BULK;
    hdr->ns = NS;
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
  const SetN32 w = spawn_setN32(buf, L, 0);
  const uint64_t traj = sp.traj_offset + (uint64_t)i;
  float e[NS], U[NS][NS], m0;
  uint16_t ab;
  sample_walkerN_f32<NS>(sp, traj, w.R + i, w.P + i, cap, m0, ab, e, U);
  w.mh[i] = m0;
  w.ml[i] = 0.0f;
  w.me[i] = 0;
  w.ph[i] = 0.0f;
  w.pl[i] = 0.0f;
  w.ab[i] = ab;
  w.id[i] = traj;
  w.fam[i] = (uint32_t)i;
#pragma unroll
  for (int a = 0; a < NS; ++a) {
#pragma unroll
    for (int b = 0; b < NS; ++b) w.U[(int64_t)(a * NS + b) * cap + i] = U[a][b];
    w.E[(int64_t)a * cap + i] = e[a];
  }
}

// Step of every live walker of set `src` in place (groups of 256 walkers, as
// the scan expects), the children staged per parent.
template <int NS, int NPL>
__global__ void __launch_bounds__(256) k_spawnN_step32(const BulkParams bp, const CoefN cf,
                                                       void* buf, int64_t cap, int64_t n0,
                                                       int64_t step) {
  constexpr int NTRI = NS * (NS + 1) / 2, NC = 2 * NS;
  // NPL = 0: the modes stay in memory (any mode count)
  constexpr bool MEM = NPL == 0;
  constexpr int NR = MEM ? 1 : NPL;
  using MR = ModeRow<NS>;
  extern __shared__ float4 mode_tab4[];
  float* const mtab = reinterpret_cast<float*>(mode_tab4);
  const SpawnLayout L = SpawnLayout::make(cap, bp.n, n0, QCL_PREC_FP32_BULK, NS);
  EnsHeader* hdr = (EnsHeader*)buf;
  const int src = (int)(step & 1);
  const int64_t n_live = ((SpawnHeader*)((char*)buf + kSpawnHeaderOff))->n_live[src];
  if (hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  if constexpr (MEM) fill_mode_table<NS>(mtab, coef_dm(cf), coef_dt(cf), bp.n);
  const bool dia = bp.repr == QCL_REPR_DIABATIC;
  const float tmaxf = (float)bp.tmax;
  const int64_t nvb = (n_live + 255) / 256;
  for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    // every lane runs the walker update (the decomposition takes warp-wide
    // votes), lanes past the live count on walker 0's state, storing nothing
    const int64_t i0 = vb * 256 + threadIdx.x;
    const bool live = i0 < n_live;
    const int64_t i = live ? i0 : 0;
    int flag = 0;
    {
      const SetN32 s = spawn_setN32(buf, L, src);
      float R[NR], P[NR];
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        const bool on = j < bp.n;
        R[j] = on ? s.R[(int64_t)j * cap + i] : 0.0f;
        P[j] = on ? s.P[(int64_t)j * cap + i] : 0.0f;
      }
      const uint16_t ab = s.ab[i];
      const int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
      f2 ph = {s.ph[i], s.pl[i]};
      const u4 wd = philox_draw(bp.seed, (uint32_t)(step >> 2), s.id[i], kPurposeHop);
      const uint32_t y = word_of(wd, (int)(step & 3)) >> 8;
      auto build_w = [&](float (&t)[NTRI]) {
#pragma unroll
        for (int k = 0; k < NTRI; ++k) t[k] = cf.E[k];
#pragma unroll
        for (int j = 0; j < NPL; ++j)
#pragma unroll
          for (int k = 0; k < NTRI; ++k) t[k] = __fmaf_rn(R[j], cf.K[j][k], t[k]);
      };
      float A[NC];  // event amplitudes (0 for the slots that are not events)
      bool deg = false;
      if (dia) {
        // diagonal force constants of the pair, W_aa - W_bb at R_n and R_{n+1}
        float hkd[NR];
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
          float ka = cf.K[j][tri<NS>(0, 0)], kb = ka;
#pragma unroll
          for (int c = 1; c < NS; ++c) {
            const float d = cf.K[j][tri<NS>(c, c)];
            ka = (c == al) ? d : ka;
            kb = (c == be) ? d : kb;
          }
          hkd[j] = __fmul_rn(0.5f * bp.hdt, __fadd_rn(ka, kb));
        }
        auto gap = [&](const float (&t)[NTRI]) {
          float va = t[tri<NS>(0, 0)], vb = va;
#pragma unroll
          for (int c = 1; c < NS; ++c) {
            const float d = t[tri<NS>(c, c)];
            va = (c == al) ? d : va;
            vb = (c == be) ? d : vb;
          }
          return __fsub_rn(va, vb);
        };
        float t[NTRI];
        float w0;
        if constexpr (MEM) {
          // one pass: W(R_n), both half kicks, the drift and W(R_{n+1}) mode
          // by mode (the register form's operations in its order)
          const float hh = 0.5f * bp.hdt;
          const int da = tri<NS>(al, al), db = tri<NS>(be, be);
          float t0[NTRI];
#pragma unroll
          for (int k = 0; k < NTRI; ++k) t0[k] = t[k] = cf.E[k];
#pragma unroll 2
          for (int j = 0; j < bp.n; ++j) {
            const float* row = mtab + j * MR::CS;
            float kr[MR::CS];
            mode_row<NS>(mtab, j, kr);
            float r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
            const float hd = __fmul_rn(hh, __fadd_rn(row[da], row[db]));
#pragma unroll
            for (int k = 0; k < NTRI; ++k) t0[k] = __fmaf_rn(r, kr[k], t0[k]);
            p = __fsub_rn(__fmaf_rn(-kr[MR::HK], r, p), hd);
            r = __fmaf_rn(kr[MR::DTM], p, r);
#pragma unroll
            for (int k = 0; k < NTRI; ++k) t[k] = __fmaf_rn(r, kr[k], t[k]);
            p = __fsub_rn(__fmaf_rn(-kr[MR::HK], r, p), hd);
            if (live) {
              s.R[(int64_t)j * cap + i] = r;
              s.P[(int64_t)j * cap + i] = p;
            }
          }
          w0 = gap(t0);
        } else {
          build_w(t);
          w0 = gap(t);
#pragma unroll
          for (int j = 0; j < NPL; ++j) P[j] = __fsub_rn(__fmaf_rn(-cf.hk[j], R[j], P[j]), hkd[j]);
#pragma unroll
          for (int j = 0; j < NPL; ++j) R[j] = __fmaf_rn(cf.dtm[j], P[j], R[j]);
          build_w(t);
#pragma unroll
          for (int j = 0; j < NPL; ++j) P[j] = __fsub_rn(__fmaf_rn(-cf.hk[j], R[j], P[j]), hkd[j]);
        }
        ph = df_add(ph, __fmul_rn(bp.hdt_hbar, __fadd_rn(w0, gap(t))));
#pragma unroll
        for (int g = 0; g < NS; ++g) {
          float wga = t[tri<NS>(g, 0)], wbg = wga;
#pragma unroll
          for (int h = 1; h < NS; ++h) {
            const float x = t[tri<NS>(g, h)];
            wga = (h == al) ? x : wga;
            wbg = (h == be) ? x : wbg;
          }
          A[g] = (g == al) ? 0.0f : __fmul_rn(bp.amp, wga);
          A[NS + g] = (g == be) ? 0.0f : __fmul_rn(bp.amp, wbg);
        }
      } else {
        float U[NS][NS], e[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) {
#pragma unroll
          for (int b = 0; b < NS; ++b) U[a][b] = s.U[(int64_t)(a * NS + b) * cap + i];
          e[a] = s.E[(int64_t)a * cap + i];
        }
        // P += dt/2 F_ab with the pair's columns ua, ub (the persistent
        // kernel's force term)
        auto make_q = [&](const float (&Uc)[NS][NS], float (&Q)[NTRI]) {
          float ua[NS], ub[NS];
          column<float, NS>(Uc, al, ua);
          column<float, NS>(Uc, be, ub);
#pragma unroll
          for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int b = a; b < NS; ++b)
              Q[tri<NS>(a, b)] = __fmul_rn((a == b ? 0.5f : 1.0f) * bp.hdt,
                                           __fmaf_rn(ua[a], ua[b], __fmul_rn(ub[a], ub[b])));
        };
        auto kick = [&](const float (&Uc)[NS][NS]) {
          float Q[NTRI];
          make_q(Uc, Q);
#pragma unroll
          for (int j = 0; j < NPL; ++j) {
            float gj = 0.0f;
#pragma unroll
            for (int k = 0; k < NTRI; ++k) gj = __fmaf_rn(cf.K[j][k], Q[k], gj);
            P[j] = __fsub_rn(__fmaf_rn(-cf.hk[j], R[j], P[j]), gj);
          }
        };
        const float de0 = __fsub_rn(pick<float, NS>(e, al), pick<float, NS>(e, be));
        float W[NS][NS], U1[NS][NS];
        float G[NTRI];
#pragma unroll
        for (int k = 0; k < NTRI; ++k) G[k] = 0.0f;
        if constexpr (MEM) {
          // pass A: first half kick, drift, W(R_{n+1}); pass B: second half
          // kick and G (the register form's operations in its order)
          float Q[NTRI], t[NTRI];
          make_q(U, Q);
#pragma unroll
          for (int k = 0; k < NTRI; ++k) t[k] = cf.E[k];
#pragma unroll 2
          for (int j = 0; j < bp.n; ++j) {
            float kr[MR::CS];
            mode_row<NS>(mtab, j, kr);
            float r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
            float g = 0.0f;
#pragma unroll
            for (int k = 0; k < NTRI; ++k) g = __fmaf_rn(kr[k], Q[k], g);
            p = __fsub_rn(__fmaf_rn(-kr[MR::HK], r, p), g);
            r = __fmaf_rn(kr[MR::DTM], p, r);
#pragma unroll
            for (int k = 0; k < NTRI; ++k) t[k] = __fmaf_rn(r, kr[k], t[k]);
            if (live) {
              s.R[(int64_t)j * cap + i] = r;
              s.P[(int64_t)j * cap + i] = p;
            }
          }
#pragma unroll
          for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int b = 0; b < NS; ++b) W[a][b] = t[tri<NS>(a, b)];
          eigh_warm_fast<NS, float>(W, U, e, U1);
          make_q(U1, Q);
#pragma unroll 2
          for (int j = 0; j < bp.n; ++j) {
            float kr[MR::CS];
            mode_row<NS>(mtab, j, kr);
            const float r = s.R[(int64_t)j * cap + i];
            float p = s.P[(int64_t)j * cap + i];
            float g = 0.0f;
#pragma unroll
            for (int k = 0; k < NTRI; ++k) g = __fmaf_rn(kr[k], Q[k], g);
            p = __fsub_rn(__fmaf_rn(-kr[MR::HK], r, p), g);
            const float v = __fmul_rn(p, kr[MR::MINV]);
#pragma unroll
            for (int k = 0; k < NTRI; ++k) G[k] = __fmaf_rn(v, kr[k], G[k]);
            if (live) s.P[(int64_t)j * cap + i] = p;
          }
        } else {
          kick(U);
#pragma unroll
          for (int j = 0; j < NPL; ++j) R[j] = __fmaf_rn(cf.dtm[j], P[j], R[j]);
          {
            float t[NTRI];
            build_w(t);
#pragma unroll
            for (int a = 0; a < NS; ++a)
#pragma unroll
              for (int b = 0; b < NS; ++b) W[a][b] = t[tri<NS>(a, b)];
          }
          eigh_warm_fast<NS, float>(W, U, e, U1);
          kick(U1);
#pragma unroll
          for (int j = 0; j < NPL; ++j) {
            const float v = __fmul_rn(P[j], cf.minv[j]);
#pragma unroll
            for (int k = 0; k < NTRI; ++k) G[k] = __fmaf_rn(v, cf.K[j][k], G[k]);
          }
        }
        const float ea = pick<float, NS>(e, al), eb = pick<float, NS>(e, be);
        ph = df_add(ph, __fmul_rn(bp.hdt_hbar, __fadd_rn(de0, __fsub_rn(ea, eb))));
        // event amplitudes: slots 0..NS-1 a -> nu with A = -dt (v.d)_{nu a},
        // slots NS..2NS-1 b -> nu with A = +dt (v.d)_{b nu}
        float ua[NS], ub[NS], Gua[NS], Gub[NS];
        column<float, NS>(U1, al, ua);
        column<float, NS>(U1, be, ub);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
          for (int c = 0; c < NS; ++c) {
            s0 = __fmaf_rn(G[tri<NS>(k, c)], ua[c], s0);
            s1 = __fmaf_rn(G[tri<NS>(k, c)], ub[c], s1);
          }
          Gua[k] = s0;
          Gub[k] = s1;
        }
#pragma unroll
        for (int sl = 0; sl < 2; ++sl)
#pragma unroll
          for (int nu = 0; nu < NS; ++nu) {
            float h = 0.0f;
#pragma unroll
            for (int k = 0; k < NS; ++k) h = __fmaf_rn(U1[k][nu], sl == 0 ? Gua[k] : Gub[k], h);
            const float gp = (sl == 0) ? __fsub_rn(ea, e[nu]) : __fsub_rn(e[nu], eb);
            const bool evl = (sl == 0) ? (nu != al) : (nu != be);
            const bool dg = evl && fabsf(gp) < kDegTolF;
            deg |= dg;
            const float qd = __fdividef(h, gp);
            A[sl * NS + nu] = __fmul_rn(sl == 0 ? -bp.dt : bp.dt, (!evl || dg) ? 0.0f : qd);
          }
        if (live) {
#pragma unroll
          for (int a = 0; a < NS; ++a) {
#pragma unroll
            for (int b = 0; b < NS; ++b) s.U[(int64_t)(a * NS + b) * cap + i] = U1[a][b];
            s.E[(int64_t)a * cap + i] = e[a];
          }
        }
      }
      // thresholds and the draw, as in the persistent kernels
      uint32_t T[NC], sumT = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        T[k] = __float2uint_rz(fminf(fabsf(__fmul_rn(bp.kappa, A[k])) * kP24f, tmaxf));
        sumT += T[k];
      }
      if (sumT > bp.tmax) {
        const float sc = (float)bp.tmax / (float)sumT;
#pragma unroll
        for (int k = 0; k < NC; ++k) T[k] = min(__float2uint_rz((float)T[k] * sc), T[k]);
      }
      uint32_t cum = 0;
      int cnt = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        cum += T[k];
        cnt += (y >= cum) ? 1 : 0;
      }
      const int hit = cnt < NC ? cnt : -1;
      // the phase pair is renormalised, and wrapped past 2^10 rad, at the end
      // of every Philox block (absolute steps 4k + 3)
      if ((step & 3) == 3) {
        ph = two_sum(ph.hi, ph.lo);
        if (fabsf(ph.hi) > 1024.0f) {
          const float kq = rintf(ph.hi * kInvTwoPiN);
          ph = df_add(ph, -kq * kTwoPi1N);
          ph = df_add(ph, -kq * kTwoPi2N);
          ph = df_add(ph, -kq * kTwoPi3N);
        }
      }
      if (live) {
#pragma unroll
        for (int j = 0; j < NPL; ++j)
          if (j < bp.n) {
            s.R[(int64_t)j * cap + i] = R[j];
            s.P[(int64_t)j * cap + i] = P[j];
          }
        s.ph[i] = ph.hi;
        s.pl[i] = ph.lo;
        ((uint8_t*)((char*)buf + L.flag))[i] = (uint8_t)(hit >= 0);
      }
      flag = live && hit >= 0;
      if (flag) {
        float Ah = A[0];
        uint32_t Th = T[0];
#pragma unroll
        for (int k = 1; k < NC; ++k) {
          Ah = (k == hit) ? A[k] : Ah;
          Th = (k == hit) ? T[k] : Th;
        }
        const float num = Ah * kP24f, den = __uint2float_rn(Th);
        const float rd = __frcp_rn(den);
        const float q0 = __fmul_rn(num, rd);
        const float q1 = __fmul_rn(__fmaf_rn(-q0, den, num), rd);
        f2 cm = df_mul({s.mh[i], s.ml[i]}, q0, q1);
        int cexp = s.me[i];
        renormN(cm, cexp);
        const bool first = hit < NS;
        const int ca = first ? hit : al, cb = first ? be : hit - NS;
        const int cq = dia ? ((q + (first ? 3 : 1)) & 3) : q;
        ((float*)((char*)buf + L.cm))[i] = cm.hi;
        ((float*)((char*)buf + L.cmlo))[i] = cm.lo;
        ((int32_t*)((char*)buf + L.cmexp))[i] = cexp;
        ((uint16_t*)((char*)buf + L.cab))[i] = (uint16_t)(ca | (cq << 4) | (cb << 8));
        if (!isfinite(cm.hi)) {
          atomicAdd(&hdr->n_nonfinite, 1ull);
          atomicOr(&hdr->flags, QCL_FLAG_NONFINITE);
        }
      }
      if (live && deg) {
        atomicAdd(&hdr->n_degenerate, 1ull);
        atomicOr(&hdr->flags, QCL_FLAG_DEGENERATE);
      }
      if (live && !isfinite(ph.hi)) {
        atomicAdd(&hdr->n_nonfinite, 1ull);
        atomicOr(&hdr->flags, QCL_FLAG_NONFINITE);
      }
    }
    const int cnt = __syncthreads_count(flag);
    if (threadIdx.x == 0) ((int32_t*)((char*)buf + L.bsum))[vb] = cnt;
  }
}

// Moves every live walker of set src (eigenvectors and eigenvalues too) to its
// place in the other set and writes each child right after its parent.
template <int NS>
__global__ void __launch_bounds__(256) k_spawnN_scatter32(void* buf, int64_t cap, int n,
                                                          int64_t n0, int64_t step0,
                                                          int64_t step, uint64_t seed) {
  __shared__ int wcnt[8];
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP32_BULK, NS);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = (SpawnHeader*)((char*)buf + kSpawnHeaderOff);
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
      const SetN32 s = spawn_setN32(buf, L, src);
      const SetN32 d = spawn_setN32(buf, L, src ^ 1);
      for (int j = 0; j < n; ++j) {
        const float r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
        d.R[(int64_t)j * cap + pos] = r;
        d.P[(int64_t)j * cap + pos] = p;
        if (flag) {
          d.R[(int64_t)j * cap + pos + 1] = r;
          d.P[(int64_t)j * cap + pos + 1] = p;
        }
      }
#pragma unroll
      for (int k = 0; k < NS * NS; ++k) {
        const float u = s.U[(int64_t)k * cap + i];
        d.U[(int64_t)k * cap + pos] = u;
        if (flag) d.U[(int64_t)k * cap + pos + 1] = u;
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const float x = s.E[(int64_t)k * cap + i];
        d.E[(int64_t)k * cap + pos] = x;
        if (flag) d.E[(int64_t)k * cap + pos + 1] = x;
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
        d.id[pos + 1] = spawn_child_id(seed, step, id);
        d.fam[pos + 1] = fam;
      }
    }
    __syncthreads();  // wcnt is rewritten by the next group
  }
}

// One thread per family: the family sum X of its walkers' 4 N_s^2
// contributions accumulated in FP64 (each walker's FP32 contributions scaled
// by its weight exponent), then X and X^2 over the tile's 128 families (the
// FP32 N_s-state tile) by the fixed tree, in passes of 16.  Adiabatic walkers
// use their carried eigenvectors, diabatic ones those of W(R) decomposed
// afresh.
template <int NS>
__global__ void __launch_bounds__(128) k_spawnN_observe32(const BulkParams bp, const CoefN cf,
                                                          const void* buf, int64_t cap, int64_t n0,
                                                          int set, double* __restrict__ part) {
  __shared__ double red[4][32];
  constexpr int NN = NS * NS, NQ = 4 * NN, NP = (NQ + 15) / 16;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const SpawnLayout L = SpawnLayout::make(cap, bp.n, n0, QCL_PREC_FP32_BULK, NS);
  const SetN32 s = spawn_setN32((void*)buf, L, set);
  const int64_t* fstart = (const int64_t*)((const char*)buf + L.fstart);
  const bool dia = bp.repr == QCL_REPR_DIABATIC;
  double X[NQ];
  for (int t = 0; t < NQ; ++t) X[t] = 0.0;
  if (k < n0) {
    const int64_t j0 = fstart[k], j1 = fstart[k + 1];
    for (int64_t j = j0; j < j1; ++j) {
      float U[NS][NS];
      if (dia) {
        float W[NS][NS], e[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) W[a][b] = cf.E[tri<NS>(a, b)];
        // (modes past the 32 of cf from the model's FP64 K, rounded alike)
        for (int m = 0; m < bp.n; ++m) {
          const float r = s.R[(int64_t)m * cap + j];
          const double* Km = coef_dm(cf)->K + (size_t)m * NS * NS;
#pragma unroll
          for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int b = 0; b < NS; ++b) {
              const float kv = m < 32 ? cf.K[m][tri<NS>(a, b)]
                                      : (float)Km[a <= b ? a * NS + b : b * NS + a];
              W[a][b] = __fmaf_rn(r, kv, W[a][b]);
            }
        }
        eigh_ns<float, NS>(W, nullptr, e, U, 12, 1e-13f);
      } else {
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) U[a][b] = s.U[(int64_t)(a * NS + b) * cap + j];
      }
      const uint16_t ab = s.ab[j];
      const int al = ab & 0xf, be = (ab >> 8) & 0xf, qt = (ab >> 4) & 3;
      f2 ph = {s.ph[j], s.pl[j]};
      const float kq = rintf(ph.hi * kInvTwoPiN);
      ph = df_add(ph, -kq * kTwoPi1N);
      ph = df_add(ph, -kq * kTwoPi2N);
      ph = df_add(ph, -kq * kTwoPi3N);
      float sh, chh;
      __sincosf(ph.hi, &sh, &chh);
      const float mm = s.mh[j] + s.ml[j];
      const float xr = mm * __fmaf_rn(-ph.lo, sh, chh), xi = -mm * __fmaf_rn(ph.lo, chh, sh);
      const float zr = qt == 0 ? xr : (qt == 1 ? -xi : (qt == 2 ? -xr : xi));
      const float zi = qt == 0 ? xi : (qt == 1 ? xr : (qt == 2 ? -xi : -xr));
      const int me = s.me[j];
      const double sc = (me >= -1022 && me <= 1023) ? pow2dN(me) : ldexp(1.0, me);
      for (int p = 0; p < NP; ++p) {
        float v16[16];
        if (dia) contrib_values_dia<float, NS>(U, al, be, zr, zi, p, v16);
        else contrib_values<float, NS>(U, al, be, zr, zi, p, v16);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (16 * p + t < NQ) X[16 * p + t] += (double)v16[t] * sc;
      }
    }
  }
  for (int p = 0; p < NP; ++p) {
    double v[32];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const double x = (16 * p + t < NQ) ? X[16 * p + t] : 0.0;
      v[t] = x;
      v[16 + t] = x * x;
    }
    const double x = warp_transpose_sum<double>(v);
    red[threadIdx.x >> 5][threadIdx.x & 31] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const int qq = (lane < 16) ? 16 * p + lane : NQ + 16 * p + (lane - 16);
      if (16 * p + (lane & 15) < NQ)
        part[(int64_t)blockIdx.x * 8 * NN + qq] =
            (red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane]);
    }
    __syncthreads();
  }
}

}  // namespace qcl
