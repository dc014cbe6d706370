// nstate_bulk.cuh -- the FP32-bulk path of N_s-state models: sampling and the
// persistent kernels of both representations, with the walker's modes in
// registers or, for any mode count, in the ensemble buffer.
#pragma once
#include "nstate_common.cuh"

namespace qcl {

// ------------------------------------------------------------ FP32 sampling --
// One initial walker in FP32 (inputs converted on the host): Wigner (R, P) at
// Rg[j * stride], Pg[j * stride], the decomposition (e, U) at R_0 (Jacobi to
// FP32 convergence, eigenvalues ascending, each eigenvector's
// largest-magnitude component positive: the FP64 sampler's conventions), and
// the pair drawn from |rho| (U^T rho_el0 U, or rho_el0 itself in the diabatic
// representation) with m_0 = rho / p_hat.
template <int NS>
__device__ __forceinline__ void sample_walkerN_f32(const SampleN32& sp, uint64_t traj, float* Rg,
                                                   float* Pg, int64_t stride, float& m0,
                                                   uint16_t& ab, float (&e)[NS],
                                                   float (&U)[NS][NS]) {
  const int n = sp.n;
  const bool k_dev = n * NS * NS > kSampleNK;  // K past the parameter copy: from the model
  float W[NS][NS];
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) W[a][b] = sp.E[a * NS + b];
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
    const float* Kj = sp.K + j * NS * NS;
    const double* Kdj = sp.Kd + (size_t)j * NS * NS;
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
      for (int b = 0; b < NS; ++b) {
        const float kv = k_dev ? (float)Kdj[a * NS + b] : Kj[a * NS + b];
        W[a][b] = __fmaf_rn(R, kv, W[a][b]);
      }
  }
  eigh_ns<float, NS>(W, nullptr, e, U, 12, 1e-13f);
  // the pair's density: U^T rho U in the adiabatic basis, rho itself in the
  // diabatic one
  const bool dia = sp.repr == QCL_REPR_DIABATIC;
  float rho_ad[NS * NS];
  float tot = 0.0f;
#pragma unroll
  for (int al = 0; al < NS; ++al)
#pragma unroll
    for (int be = 0; be < NS; ++be) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int l = 0; l < NS; ++l) acc = __fmaf_rn(U[k][al] * sp.rho[k * NS + l], U[l][be], acc);
      acc = dia ? sp.rho[al * NS + be] : acc;
      rho_ad[al * NS + be] = acc;
      tot += fabsf(acc);
    }
  // thresholds as in the two-state FP32 sampler: remainder to the last nonzero
  // pair, an excess from FP32 rounding off the largest threshold
  uint32_t Tk[NS * NS];
  uint32_t sumT = 0;
  int last = 0, big = 0;
  for (int k = 0; k < NS * NS; ++k) {
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
  int pickk = last;
  for (int k = 0; k < NS * NS; ++k) {
    cum += Tk[k];
    if (y < cum) {
      pickk = k;
      break;
    }
  }
  m0 = rho_ad[pickk] * (kP24f / (float)Tk[pickk]);
  ab = (uint16_t)((pickk / NS) | ((pickk % NS) << 8));
}

template <int NS>
__global__ void __launch_bounds__(128) k_sampleN_f32(const SampleN32 sp, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = sp.n_traj;
  const int n = sp.n;
  WN<float> w = viewN<float>(buf, nt, NS, n, QCL_PREC_FP32_BULK);
  if (i == 0) {
    w.hdr->magic = kEnsMagic;
    w.hdr->n_traj = nt;
    w.hdr->precision = QCL_PREC_FP32_BULK;
    w.hdr->ns = NS;
    w.hdr->n = n;
    w.hdr->step = 0;
    w.hdr->flags = 0;
    w.hdr->n_degenerate = 0;
    w.hdr->n_nonfinite = 0;
  }
  if (i >= nt) return;
  float e[NS], U[NS][NS], m0;
  uint16_t ab;
  sample_walkerN_f32<NS>(sp, sp.traj_offset + (uint64_t)i, w.R + i, w.P + i, nt, m0, ab, e, U);
  w.m[i] = m0;
  w.mlo[i] = 0.0f;
  w.mexp[i] = 0;
  w.phi[i] = 0.0f;
  w.philo[i] = 0.0f;
  w.ab[i] = ab;
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) w.U[(int64_t)(a * NS + b) * nt + i] = U[a][b];
#pragma unroll
  for (int a = 0; a < NS; ++a) w.E[(int64_t)a * nt + i] = e[a];
}

// ------------------------------------------------------- FP32-bulk kernel --
__device__ __forceinline__ int fexpN(float x) {
  return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127;
}
__device__ __forceinline__ float pow2iN(int d) {
  return d < -126 ? 0.0f : __uint_as_float((uint32_t)(127 + d) << 23);
}
__device__ __forceinline__ void renormN(f2& m, int& e) {
  if (m.hi == 0.0f) return;
  const int k = fexpN(m.hi);
  const float sc = (k == -127) ? 0x1p+126f : (k >= 127 ? 0x1p-127f : pow2iN(-k));
  m.hi *= sc;
  m.lo *= sc;
  e += (k == -127) ? -126 : k;
}
__device__ __forceinline__ double pow2dN(int e) { return __hiloint2double((e + 1023) << 20, 0); }

constexpr float kTwoPi1N = 6.283203125f;
constexpr float kTwoPi2N = -1.7818063497543335e-05f;
constexpr float kTwoPi3N = 2.430840251310684e-10f;
constexpr float kInvTwoPiN = 0.15915494309189535f;

// W's upper triangle index
template <int NS>
__host__ __device__ constexpr int tri(int a, int b) {
  return a <= b ? a * NS - a * (a - 1) / 2 + (b - a) : b * NS - b * (b - 1) / 2 + (a - b);
}

// ---------------------------------------------------------- modes in memory --
// The FP32 kernels' form for any mode count: R and P stay in the ensemble
// buffer and are read (and written back) mode by mode in each pass of a step;
// the per-mode coefficients come from a table in shared memory, row j = the
// upper triangle of K_j, dt/2 k_j, dt/M_j and 1/M_j (padded to whole float4s),
// built from the FP64 model with the host's roundings (the CoefN values).
template <int NS>
struct ModeRow {
  static constexpr int NTRI = NS * (NS + 1) / 2;
  static constexpr int HK = NTRI, DTM = NTRI + 1, MINV = NTRI + 2;
  static constexpr int CS = (NTRI + 3 + 3) / 4 * 4;
  static size_t bytes(int n) { return (size_t)n * CS * sizeof(float); }
};

template <int NS>
__device__ void fill_mode_table(float* mt, const DevModel* dm, double dt, int n) {
  using MR = ModeRow<NS>;
  for (int idx = threadIdx.x; idx < n * MR::CS; idx += blockDim.x) {
    const int j = idx / MR::CS, c = idx - j * MR::CS;
    float v = 0.0f;
    if (c < MR::NTRI) {
      int a = 0, rem = c;  // row a, column a + rem of the upper triangle
      while (rem >= NS - a) {
        rem -= NS - a;
        ++a;
      }
      v = (float)dm->K[(size_t)j * NS * NS + a * NS + a + rem];
    } else if (c == MR::HK) {
      v = (float)(0.5 * dt * dm->k[j]);
    } else if (c == MR::DTM) {
      v = (float)(dt / dm->mass[j]);
    } else if (c == MR::MINV) {
      v = (float)(1.0 / dm->mass[j]);
    }
    mt[idx] = v;
  }
  __syncthreads();
}

template <int NS>
__device__ __forceinline__ void mode_row(const float* mt, int j, float (&r)[ModeRow<NS>::CS]) {
  const float4* p = reinterpret_cast<const float4*>(mt + j * ModeRow<NS>::CS);
#pragma unroll
  for (int q = 0; q < ModeRow<NS>::CS / 4; ++q) {
    const float4 v = p[q];
    r[4 * q] = v.x;
    r[4 * q + 1] = v.y;
    r[4 * q + 2] = v.z;
    r[4 * q + 3] = v.w;
  }
}

// WPT (1 or 2) tiles of 128 walkers per block, thread t holding walker t of
// each: with WPT = 2 the two walkers are the lanes of float2 values and their
// FP32 arithmetic runs as packed FP32x2 instructions (explicit round-to-nearest
// operations throughout, so each walker's bits do not depend on WPT); event
// selection, divisions, square roots and the observation run per lane.
template <int NS, int NPL, int WPT>
struct BulkNMinBlocks {
  static constexpr int value =
      NPL > 8 ? 1 : (WPT == 1 ? (NS <= 4 ? 4 : (NS == 5 ? 3 : 1)) : (NS <= 4 ? 2 : 1));
};

template <int NS, int NPL, int WPT>
__global__ void __launch_bounds__(128, (BulkNMinBlocks<NS, NPL, WPT>::value))
    k_bulkN(const BulkParams bp, const CoefN cf, void* buf, double* __restrict__ part) {
  static_assert(WPT == 1 || WPT == 2, "one or two walkers per thread");
  // NPL = 0: the modes stay in memory (any mode count, one walker per thread)
  constexpr bool MEM = NPL == 0;
  constexpr int NR = MEM ? 1 : NPL;
  static_assert(!MEM || WPT == 1, "modes in memory: one walker per thread");
  using MR = ModeRow<NS>;
  constexpr int MU = NS <= 4 ? 4 : 2;  // mode-loop unrolling (loads in flight; registers)
  using V = std::conditional_t<WPT == 2, float2, float>;
  constexpr int NN = NS * NS, NTRI = NS * (NS + 1) / 2;
  constexpr int NP = (4 * NN + 15) / 16;  // observation passes of 32 quantities
  constexpr int TW = 128;                 // walkers per tile
  __shared__ double red[2][4][32];
  __shared__ float obs_rows[TW * 33];
  extern __shared__ float4 mode_tab4[];
  float* const mtab = reinterpret_cast<float*>(mode_tab4);
  WN<float> ws = viewN<float>(buf, bp.n_traj, NS, bp.n, QCL_PREC_FP32_BULK);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  if constexpr (MEM) fill_mode_table<NS>(mtab, coef_dm(cf), coef_dt(cf), bp.n);
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int n_deg = 0;
  int rb = 0;
  for (int64_t tile0 = (int64_t)blockIdx.x * WPT; tile0 < bp.n_tiles;
       tile0 += (int64_t)gridDim.x * WPT) {
    bool active[WPT];
    int64_t iw[WPT];
    V R[NR], P[NR], U[NS][NS], e[NS];
    PairV<V> m, ph;
    int mexp[WPT], al[WPT], be[WPT];
    uint64_t traj[WPT];
#pragma unroll
    for (int l = 0; l < WPT; ++l) {
      const int64_t i = (tile0 + l) * TW + threadIdx.x;
      active[l] = i < nt;
      const int64_t ii = active[l] ? i : 0;
      iw[l] = i;
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        const bool on = active[l] && j < bp.n;
        ln(R[j], l) = on ? ws.R[(int64_t)j * nt + ii] : 0.0f;
        ln(P[j], l) = on ? ws.P[(int64_t)j * nt + ii] : 0.0f;
      }
#pragma unroll
      for (int a = 0; a < NS; ++a) {
#pragma unroll
        for (int b = 0; b < NS; ++b)
          ln(U[a][b], l) = active[l] ? ws.U[(int64_t)(a * NS + b) * nt + ii] : (a == b ? 1.f : 0.f);
        // decomposition at R_n as left by the previous step (stored exactly, so
        // a chunk boundary changes no bit)
        ln(e[a], l) = active[l] ? ws.E[(int64_t)a * nt + ii] : (float)a;
      }
      ln(m.hi, l) = active[l] ? ws.m[ii] : 0.0f;
      ln(m.lo, l) = active[l] ? ws.mlo[ii] : 0.0f;
      mexp[l] = active[l] ? ws.mexp[ii] : 0;
      ln(ph.hi, l) = active[l] ? ws.phi[ii] : 0.0f;
      ln(ph.lo, l) = active[l] ? ws.philo[ii] : 0.0f;
      const uint32_t ab0 = active[l] ? ws.ab[ii] : 0u;
      al[l] = ab0 & 0xff;
      be[l] = (ab0 >> 8) & 0xff;
      traj[l] = bp.traj_offset + (uint64_t)ii;
    }

    auto build_w = [&](V (&W)[NS][NS]) {
      V t[NTRI];
#pragma unroll
      for (int k = 0; k < NTRI; ++k) t[k] = splat<V>(cf.E[k]);
#pragma unroll
      for (int j = 0; j < NPL; ++j)
#pragma unroll
        for (int k = 0; k < NTRI; ++k) t[k] = vfma(R[j], splat<V>(cf.K[j][k]), t[k]);
#pragma unroll
      for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int b = 0; b < NS; ++b) W[a][b] = t[tri<NS>(a, b)];
    };
    // columns al, be of U (per lane)
    auto columns = [&](V (&ua)[NS], V (&ub)[NS]) {
#pragma unroll
      for (int l = 0; l < WPT; ++l)
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          float va = ln(U[i][0], l), vb = va;
#pragma unroll
          for (int c = 1; c < NS; ++c) {
            const float uc = ln(U[i][c], l);  // (a value, not a reference, in the selects)
            va = (c == al[l]) ? uc : va;
            vb = (c == be[l]) ? uc : vb;
          }
          ln(ua[i], l) = va;
          ln(ub[i], l) = vb;
        }
    };
    // e_al, e_be (per lane picks) and their difference
    auto gap_ab = [&](V& ea, V& eb) {
#pragma unroll
      for (int l = 0; l < WPT; ++l) {
        float va = ln(e[0], l), vb = va;
#pragma unroll
        for (int c = 1; c < NS; ++c) {
          const float ec = ln(e[c], l);
          va = (c == al[l]) ? ec : va;
          vb = (c == be[l]) ? ec : vb;
        }
        ln(ea, l) = va;
        ln(eb, l) = vb;
      }
      return vsub(ea, eb);
    };
    // the coupling part of dt/2 F_ab: g_j = sum_k K_jk Q_k with
    // Q = dt/2 * (1/2)(u_a u_a^T + u_b u_b^T) folded with the off-diagonal
    // factor 2 (ua, ub: columns al, be of U)
    auto make_q = [&](const V (&ua)[NS], const V (&ub)[NS], V (&Q)[NTRI]) {
#pragma unroll
      for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int b = a; b < NS; ++b)
          Q[tri<NS>(a, b)] = vmul(splat<V>((a == b ? 0.5f : 1.0f) * bp.hdt),
                                  vfma(ua[a], ua[b], vmul(ub[a], ub[b])));
    };
    auto force = [&](const V (&ua)[NS], const V (&ub)[NS], V (&g)[NR]) {
      V Q[NTRI];
      make_q(ua, ub, Q);
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        V gj = splat<V>(0.0f);
#pragma unroll
        for (int k = 0; k < NTRI; ++k) gj = vfma(splat<V>(cf.K[j][k]), Q[k], gj);
        g[j] = gj;
      }
    };
    // P += dt/2 F_ab(R) = P - dt/2 k R - g
    auto kick = [&](const V (&g)[NR]) {
#pragma unroll
      for (int j = 0; j < NPL; ++j) P[j] = vsub(vfma(splat<V>(-cf.hk[j]), R[j], P[j]), g[j]);
    };
    // Modes in memory, mode by mode with the register form's operations in its
    // order.  Pass A: the first half kick with the force term of Q, the drift
    // and the upper triangle of W(R_{n+1}); pass B: the second half kick with
    // the force term of Q and the sum G = sum_j (P_j/M_j) K_j.
    // Each pass loads R and P of MU modes before computing them and stores them
    // after, so that a batch's loads are not ordered behind the previous
    // mode's stores (lanes past the ensemble load walker 0's values, take
    // zeros as the register form does, and store nothing).
    auto mode_a = [&](int jj, const V (&Q)[NTRI], V (&t)[NTRI], V& r, V& p) {
      float kr[MR::CS];
      mode_row<NS>(mtab, jj, kr);
      V g = splat<V>(0.0f);
#pragma unroll
      for (int k = 0; k < NTRI; ++k) g = vfma(splat<V>(kr[k]), Q[k], g);
      p = vsub(vfma(splat<V>(-kr[MR::HK]), r, p), g);
      r = vfma(splat<V>(kr[MR::DTM]), p, r);
#pragma unroll
      for (int k = 0; k < NTRI; ++k) t[k] = vfma(r, splat<V>(kr[k]), t[k]);
    };
    auto mode_b = [&](int jj, const V (&Q)[NTRI], V (&t)[NTRI], V r, V& p) {
      float kr[MR::CS];
      mode_row<NS>(mtab, jj, kr);
      V g = splat<V>(0.0f);
#pragma unroll
      for (int k = 0; k < NTRI; ++k) g = vfma(splat<V>(kr[k]), Q[k], g);
      p = vsub(vfma(splat<V>(-kr[MR::HK]), r, p), g);
      const V v = vmul(p, splat<V>(kr[MR::MINV]));
#pragma unroll
      for (int k = 0; k < NTRI; ++k) t[k] = vfma(v, splat<V>(kr[k]), t[k]);
    };
    auto pass_a = [&](const V (&Q)[NTRI], V (&W)[NS][NS]) {
      V t[NTRI];
#pragma unroll
      for (int k = 0; k < NTRI; ++k) t[k] = splat<V>(cf.E[k]);
      float* R0 = ws.R + (active[0] ? iw[0] : 0);
      float* P0 = ws.P + (active[0] ? iw[0] : 0);
      int j = 0;
      for (; j + MU <= bp.n; j += MU, R0 += MU * nt, P0 += MU * nt) {
        V rb[MU], pb[MU];
#pragma unroll
        for (int u = 0; u < MU; ++u) {
          ln(rb[u], 0) = active[0] ? R0[u * nt] : 0.0f;
          ln(pb[u], 0) = active[0] ? P0[u * nt] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < MU; ++u) mode_a(j + u, Q, t, rb[u], pb[u]);
        if (active[0]) {
#pragma unroll
          for (int u = 0; u < MU; ++u) {
            R0[u * nt] = ln(rb[u], 0);
            P0[u * nt] = ln(pb[u], 0);
          }
        }
      }
      for (; j < bp.n; ++j, R0 += nt, P0 += nt) {
        V r, p;
        ln(r, 0) = active[0] ? *R0 : 0.0f;
        ln(p, 0) = active[0] ? *P0 : 0.0f;
        mode_a(j, Q, t, r, p);
        if (active[0]) {
          *R0 = ln(r, 0);
          *P0 = ln(p, 0);
        }
      }
#pragma unroll
      for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int b = 0; b < NS; ++b) W[a][b] = t[tri<NS>(a, b)];
    };
    auto pass_b = [&](const V (&Q)[NTRI], V (&t)[NTRI]) {
#pragma unroll
      for (int k = 0; k < NTRI; ++k) t[k] = splat<V>(0.0f);
      const float* R0 = ws.R + (active[0] ? iw[0] : 0);
      float* P0 = ws.P + (active[0] ? iw[0] : 0);
      int j = 0;
      for (; j + MU <= bp.n; j += MU, R0 += MU * nt, P0 += MU * nt) {
        V rb[MU], pb[MU];
#pragma unroll
        for (int u = 0; u < MU; ++u) {
          ln(rb[u], 0) = active[0] ? R0[u * nt] : 0.0f;
          ln(pb[u], 0) = active[0] ? P0[u * nt] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < MU; ++u) mode_b(j + u, Q, t, rb[u], pb[u]);
        if (active[0]) {
#pragma unroll
          for (int u = 0; u < MU; ++u) P0[u * nt] = ln(pb[u], 0);
        }
      }
      for (; j < bp.n; ++j, R0 += nt, P0 += nt) {
        V r, p;
        ln(r, 0) = active[0] ? *R0 : 0.0f;
        ln(p, 0) = active[0] ? *P0 : 0.0f;
        mode_b(j, Q, t, r, p);
        if (active[0]) *P0 = ln(p, 0);
      }
    };
    // observation of walker lane l into slot `slot` of tile tile0 + l
    auto observe_lane = [&](int l, int slot) {
      f2 ml = {ln(m.hi, l), ln(m.lo, l)};
      f2 pl = {ln(ph.hi, l), ln(ph.lo, l)};
      int me = mexp[l];
      renormN(ml, me);
      const bool live = active[l] && ml.hi != 0.0f;
      int ew = live ? me : -(1 << 28);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ew = max(ew, __shfl_xor_sync(0xffffffffu, ew, off));
      const float kq = rintf(pl.hi * kInvTwoPiN);
      pl = df_add(pl, -kq * kTwoPi1N);
      pl = df_add(pl, -kq * kTwoPi2N);
      pl = df_add(pl, -kq * kTwoPi3N);
      ln(m.hi, l) = ml.hi;
      ln(m.lo, l) = ml.lo;
      mexp[l] = me;
      ln(ph.hi, l) = pl.hi;
      ln(ph.lo, l) = pl.lo;
      float sh, chh;
      __sincosf(pl.hi, &sh, &chh);
      const float mm = live ? ml.hi * pow2iN(me - ew) : 0.0f;
      const float zr = mm * __fmaf_rn(-pl.lo, sh, chh), zi = -mm * __fmaf_rn(pl.lo, chh, sh);
      const int ex = (ew < -(1 << 27)) ? 0 : ((lane < 16) ? ew : 2 * ew);
      float Ul[NS][NS];
#pragma unroll
      for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int b = 0; b < NS; ++b) Ul[a][b] = ln(U[a][b], l);
      float* row = &obs_rows[threadIdx.x * 33];
      // passes unrolled for N_s <= 4 (their quantity indices are then
      // compile-time: no local-memory arrays), rolled for larger N_s
      constexpr int kPassUnroll = NP <= 4 ? NP : 1;
#pragma unroll kPassUnroll
      for (int p = 0; p < NP; ++p) {
        float v[16];
        contrib_values<float, NS>(Ul, al[l], be[l], zr, zi, p, v);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          row[t] = v[t];
          row[16 + t] = v[t] * v[t];
        }
        __syncwarp();
        float l1[16];
        const float* col = &obs_rows[(warp * 32) * 33 + lane];
#pragma unroll
        for (int t = 0; t < 16; ++t) l1[t] = col[(2 * t) * 33] + col[(2 * t + 1) * 33];
#pragma unroll
        for (int wdt = 8; wdt >= 1; wdt >>= 1)
#pragma unroll
          for (int t = 0; t < wdt; ++t) l1[t] = l1[2 * t] + l1[2 * t + 1];
        __syncwarp();
        const double xd = (double)l1[0];
        red[rb][warp][lane] = (ex >= -1022 && ex <= 1023) ? xd * pow2dN(ex) : ldexp(xd, ex);
        __syncthreads();
        if (threadIdx.x < 32 && tile0 + l < bp.n_tiles) {
          const int q = (lane < 16) ? 16 * p + lane : 4 * NN + 16 * p + (lane - 16);
          if (16 * p + (lane & 15) < 4 * NN)
            part[((int64_t)slot * bp.n_tiles + tile0 + l) * 8 * NN + q] =
                (red[rb][0][lane] + red[rb][1][lane]) + (red[rb][2][lane] + red[rb][3][lane]);
        }
        rb ^= 1;
      }
    };
    auto observe = [&](int slot) {
#pragma unroll
      for (int l = 0; l < WPT; ++l) observe_lane(l, slot);
    };

    int slot = bp.obs_first;
    if (bp.obs_first) observe(0);
    int to_out = bp.to_out0;
    uint32_t blk = bp.blk0;
    int widx = bp.widx0;
    u4 wd[WPT];
#pragma unroll
    for (int l = 0; l < WPT; ++l) wd[l] = philox_draw(bp.seed, blk, traj[l], kPurposeHop);
    // Carried from one step to the next while no walker of the thread hops:
    // the pair's columns ua, ub and energies ea, eb at R_{n+1}, their gap and the
    // force term g (its Q with the modes in memory), which the next step's
    // first half kick (the same R, U and pair) would compute again bit for
    // bit.  A hop, and the first step of a launch, compute them afresh.
    V ua[NS], ub[NS], gk[NR], Qc[NTRI], ea, eb, de0;
    bool cached = false;
    for (int it = 0; it < bp.len; ++it) {
      if (!cached) {
        de0 = gap_ab(ea, eb);
        columns(ua, ub);
        if constexpr (MEM) make_q(ua, ub, Qc);
        else force(ua, ub, gk);
      }
      V Gt[NTRI];  // (modes in memory: G's upper triangle from pass B)
      if constexpr (MEM) {
        V W[NS][NS], Uref[NS][NS];
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) Uref[a][b] = U[a][b];
        pass_a(Qc, W);  // first half kick at R_n, drift, W(R_{n+1})
        eigh_warm_fast<NS, V>(W, Uref, e, U);
        columns(ua, ub);
        make_q(ua, ub, Qc);
        pass_b(Qc, Gt);  // second half kick at R_{n+1}, G
      } else {
        kick(gk);  // first half kick at R_n
#pragma unroll
        for (int j = 0; j < NPL; ++j) R[j] = vfma(splat<V>(cf.dtm[j]), P[j], R[j]);
        {
          V W[NS][NS], Uref[NS][NS];
#pragma unroll
          for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int b = 0; b < NS; ++b) Uref[a][b] = U[a][b];
          build_w(W);
          eigh_warm_fast<NS, V>(W, Uref, e, U);
        }
        columns(ua, ub);  // (the new decomposition's columns)
        force(ua, ub, gk);
        kick(gk);  // second half kick at R_{n+1}
      }
      const V de1 = gap_ab(ea, eb);
      ph = df_add_v(ph, vmul(splat<V>(bp.hdt_hbar), vadd(de0, de1)));
      de0 = de1;
      // G = sum_j (P_j/M_j) K_j
      V G[NS][NS];
      if constexpr (MEM) {
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) G[a][b] = Gt[tri<NS>(a, b)];
      } else {
        V t[NTRI];
#pragma unroll
        for (int k = 0; k < NTRI; ++k) t[k] = splat<V>(0.0f);
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
          const V v = vmul(P[j], splat<V>(cf.minv[j]));
#pragma unroll
          for (int k = 0; k < NTRI; ++k) t[k] = vfma(v, splat<V>(cf.K[j][k]), t[k]);
        }
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) G[a][b] = t[tri<NS>(a, b)];
      }
      // event amplitudes of the coupling term of Eq. 1 (as event_amplitudes):
      // slots 0..NS-1 move the first index a -> nu with A = -dt (v.d)_{nu a},
      // slots NS..2NS-1 the second index b -> nu with A = +dt (v.d)_{b nu}
      constexpr int NC = 2 * NS;
      V A[NC];  // (0 for the two slots that would leave the pair unchanged)
      {
        V Gua[NS], Gub[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          V s0 = splat<V>(0.0f), s1 = splat<V>(0.0f);
#pragma unroll
          for (int c = 0; c < NS; ++c) {
            s0 = vfma(G[k][c], ua[c], s0);
            s1 = vfma(G[k][c], ub[c], s1);
          }
          Gua[k] = s0;
          Gub[k] = s1;
        }
        bool dgl[WPT];
#pragma unroll
        for (int l = 0; l < WPT; ++l) dgl[l] = false;
#pragma unroll
        for (int sl = 0; sl < 2; ++sl)
#pragma unroll
          for (int nu = 0; nu < NS; ++nu) {
            V h = splat<V>(0.0f);
#pragma unroll
            for (int k = 0; k < NS; ++k) h = vfma(U[k][nu], sl == 0 ? Gua[k] : Gub[k], h);
            const V gap = (sl == 0) ? vsub(ea, e[nu]) : vsub(e[nu], eb);
            V vd;
#pragma unroll
            for (int l = 0; l < WPT; ++l) {
              const bool evl = (sl == 0) ? (nu != al[l]) : (nu != be[l]);
              const bool dg = evl && fabsf(ln(gap, l)) < kDegTolF;
              dgl[l] |= dg;
              // approximate division (the amplitude enters a probability and a
              // weight factor, both far above its 2-ulp error), taken on every
              // slot and discarded by the select (no branch around it)
              const float qd = __fdividef(ln(h, l), ln(gap, l));
              ln(vd, l) = (!evl || dg) ? 0.0f : qd;
            }
            A[sl * NS + nu] = vmul(splat<V>(sl == 0 ? -bp.dt : bp.dt), vd);
          }
#pragma unroll
        for (int l = 0; l < WPT; ++l) n_deg += (dgl[l] && active[l]) ? 1u : 0u;
      }
      // thresholds, event choice and the weight factor (per lane), the
      // compensated weight product (lanes)
      V num, den, rd;
      int hitl[WPT];
#pragma unroll
      for (int l = 0; l < WPT; ++l) {
        const uint32_t word = (widx & 2) ? ((widx & 1) ? wd[l].w : wd[l].z)
                                         : ((widx & 1) ? wd[l].y : wd[l].x);
        // T = min(floor(kappa |A| 2^24), Tmax), the clamp taken in FP32 (Tmax < 2^24
        // is exact there); the excluded slots have A = 0, so T = 0
        const float tmaxf = (float)bp.tmax;
        uint32_t T[NC], sumT = 0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const float ka = fabsf(ln(vmul(splat<V>(bp.kappa), A[k]), l));
          T[k] = __float2uint_rz(fminf(ka * kP24f, tmaxf));
          sumT += T[k];
        }
        if (sumT > bp.tmax) {
          const float sc = (float)bp.tmax / (float)sumT;
          uint32_t s2 = 0;
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            T[k] = min(__float2uint_rz((float)T[k] * sc), T[k]);
            s2 += T[k];
          }
          sumT = s2;
        }
        // the event whose interval [cum_{k-1}, cum_k) holds y: the number of
        // cumulative thresholds at or below y (NC: none, no transition)
        const uint32_t y = word >> 8;
        uint32_t cum = 0;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          cum += T[k];
          cnt += (y >= cum) ? 1 : 0;
        }
        const int hit = cnt < NC ? cnt : -1;
        float Ah = ln(A[0], l);
        uint32_t Th = T[0];
#pragma unroll
        for (int k = 1; k < NC; ++k) {
          const float Ak = ln(A[k], l);
          Ah = (k == hit) ? Ak : Ah;
          Th = (k == hit) ? T[k] : Th;
        }
        const bool hop = hit >= 0;
        ln(num, l) = hop ? Ah * kP24f : kP24f;
        ln(den, l) = __uint2float_rn(hop ? Th : 16777216u - sumT);
        ln(rd, l) = __frcp_rn(ln(den, l));
        hitl[l] = hit;
      }
      const V q0 = vmul(num, rd);
      const V q1 = vmul(vfma(q0, vmul(den, splat<V>(-1.0f)), num), rd);
      m = df_mul_v(m, q0, q1);
#pragma unroll
      for (int l = 0; l < WPT; ++l) {
        const float h = ln(m.hi, l);
        if (!(fabsf(h) <= 0x1p32f && fabsf(h) >= 0x1p-32f)) {
          f2 ml = {h, ln(m.lo, l)};
          renormN(ml, mexp[l]);
          ln(m.hi, l) = ml.hi;
          ln(m.lo, l) = ml.lo;
        }
        const int hit = hitl[l];
        if (hit >= 0) {
          if (hit < NS) al[l] = hit;
          else be[l] = hit - NS;
        }
      }
      cached = true;
#pragma unroll
      for (int l = 0; l < WPT; ++l) cached = cached && hitl[l] < 0;
      if (++widx == 4) {
        widx = 0;
        ++blk;
        if (it + 1 < bp.len) {
#pragma unroll
          for (int l = 0; l < WPT; ++l) wd[l] = philox_draw(bp.seed, blk, traj[l], kPurposeHop);
        }
      }
      if (--to_out == 0) {
        observe(slot++);
        to_out = bp.stride;
      }
    }
#pragma unroll
    for (int l = 0; l < WPT; ++l) {
      if (!active[l]) continue;
      const int64_t i = iw[l];
#pragma unroll
      for (int j = 0; j < NPL; ++j)
        if (j < bp.n) {
          ws.R[(int64_t)j * nt + i] = ln(R[j], l);
          ws.P[(int64_t)j * nt + i] = ln(P[j], l);
        }
#pragma unroll
      for (int a = 0; a < NS; ++a) {
#pragma unroll
        for (int b = 0; b < NS; ++b) ws.U[(int64_t)(a * NS + b) * nt + i] = ln(U[a][b], l);
        ws.E[(int64_t)a * nt + i] = ln(e[a], l);
      }
      const float mh = ln(m.hi, l), phh = ln(ph.hi, l);
      ws.m[i] = mh;
      ws.mlo[i] = ln(m.lo, l);
      ws.mexp[i] = mexp[l];
      ws.phi[i] = phh;
      ws.philo[i] = ln(ph.lo, l);
      ws.ab[i] = (uint16_t)(al[l] | (be[l] << 8));
      if (!isfinite(mh) || !isfinite(phh)) {
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

// ----------------------------------------- FP32-bulk kernel, diabatic pairs --
// The diabatic representation of N_s-state models on the FP32-bulk path: one
// walker per thread, 128-walker tiles, persistent over tiles.  No
// decomposition is carried or needed for the step: the mean force is the
// diagonal one (its coupling part (dt/2) 1/2 (K_j,aa + K_j,bb) is a constant of
// the pair, taken again after a hop), the phase comes from W's diagonal and
// the events from its columns a and b at R_{n+1} (the FP64 step's order of
// events, quarter turns and 24-bit thresholds).  The observation diagonalises
// W(R) afresh at output times (Jacobi, the sampler's conventions) for the
// adiabatic block.
template <int NS, int NPL>
__global__ void __launch_bounds__(128, (NPL > 8 || NS > 5) ? 2 : 4)
    k_bulkN_dia(const BulkParams bp, const CoefN cf, void* buf, double* __restrict__ part) {
  constexpr int NN = NS * NS, NTRI = NS * (NS + 1) / 2;
  constexpr int NP = (4 * NN + 15) / 16;
  constexpr int TW = 128;
  constexpr int NC = 2 * NS;
  // NPL = 0: the modes stay in memory (any mode count)
  constexpr bool MEM = NPL == 0;
  constexpr int NR = MEM ? 1 : NPL;
  using MR = ModeRow<NS>;
  constexpr int MU = NS <= 4 ? 4 : 2;  // mode-loop unrolling (loads in flight; registers)
  __shared__ double red[2][4][32];
  __shared__ float obs_rows[TW * 33];
  extern __shared__ float4 mode_tab4[];
  float* const mtab = reinterpret_cast<float*>(mode_tab4);
  WN<float> ws = viewN<float>(buf, bp.n_traj, NS, bp.n, QCL_PREC_FP32_BULK);
  if (ws.hdr->step != bp.step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  if constexpr (MEM) fill_mode_table<NS>(mtab, coef_dm(cf), coef_dt(cf), bp.n);
  const int64_t nt = bp.n_traj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int rb = 0;
  for (int64_t tile0 = blockIdx.x; tile0 < bp.n_tiles; tile0 += gridDim.x) {
    const int64_t i = tile0 * TW + threadIdx.x;
    const bool active = i < nt;
    const int64_t ii = active ? i : 0;
    float R[NR], P[NR];
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const bool on = active && j < bp.n;
      R[j] = on ? ws.R[(int64_t)j * nt + ii] : 0.0f;
      P[j] = on ? ws.P[(int64_t)j * nt + ii] : 0.0f;
    }
    f2 m = {active ? ws.m[ii] : 0.0f, active ? ws.mlo[ii] : 0.0f};
    int mexp = active ? ws.mexp[ii] : 0;
    f2 ph = {active ? ws.phi[ii] : 0.0f, active ? ws.philo[ii] : 0.0f};
    const uint32_t ab0 = active ? ws.ab[ii] : 0u;
    int al = ab0 & 0xf, be = (ab0 >> 8) & 0xf, q = (ab0 >> 4) & 3;
    const uint64_t traj = bp.traj_offset + (uint64_t)ii;

    // W(R) (upper triangle) at the walker's R
    auto build_w = [&](float (&t)[NTRI]) {
#pragma unroll
      for (int k = 0; k < NTRI; ++k) t[k] = cf.E[k];
#pragma unroll
      for (int j = 0; j < NPL; ++j)
#pragma unroll
        for (int k = 0; k < NTRI; ++k) t[k] = __fmaf_rn(R[j], cf.K[j][k], t[k]);
    };
    // W_aa - W_bb
    auto diag_gap = [&](const float (&t)[NTRI]) {
      float va = t[tri<NS>(0, 0)], vb = va;
#pragma unroll
      for (int c = 1; c < NS; ++c) {
        const float d = t[tri<NS>(c, c)];
        va = (c == al) ? d : va;
        vb = (c == be) ? d : vb;
      }
      return __fsub_rn(va, vb);
    };
    // the pair's force constants: hkd_j = dt/2 * 1/2 (K_j,aa + K_j,bb)
    float hkd[NR];
    auto pair_force = [&]() {
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
    };
    auto kick = [&]() {
#pragma unroll
      for (int j = 0; j < NPL; ++j)
        P[j] = __fsub_rn(__fmaf_rn(-cf.hk[j], R[j], P[j]), hkd[j]);
    };
    // Modes in memory: one pass per step, mode by mode with the register
    // form's operations in its order.  The second half kick of a step is
    // taken at the start of the next step's pass (the transition does not
    // depend on the momenta here), with the pair it was due with (pa, pb),
    // then the first half kick of the current pair, the drift and the upper
    // triangle of W(R_{n+1}); a last pass ends the launch with the pending kick.
    const float hh = 0.5f * bp.hdt;
    auto pass_dia = [&](float (&t)[NTRI], bool pend, int pa, int pb, bool step) {
#pragma unroll
      for (int k = 0; k < NTRI; ++k) t[k] = cf.E[k];
      const int dpa = tri<NS>(pa, pa), dpb = tri<NS>(pb, pb);
      const int da = tri<NS>(al, al), db = tri<NS>(be, be);
      auto mode = [&](int jj, float& r, float& p) {
        const float* row = mtab + jj * MR::CS;
        float kr[MR::CS];
        mode_row<NS>(mtab, jj, kr);
        if (pend) p = __fsub_rn(__fmaf_rn(-kr[MR::HK], r, p), __fmul_rn(hh, __fadd_rn(row[dpa], row[dpb])));
        if (step) {
          p = __fsub_rn(__fmaf_rn(-kr[MR::HK], r, p), __fmul_rn(hh, __fadd_rn(row[da], row[db])));
          r = __fmaf_rn(kr[MR::DTM], p, r);
        }
#pragma unroll
        for (int k = 0; k < NTRI; ++k) t[k] = __fmaf_rn(r, kr[k], t[k]);
      };
      // batches of MU modes: loads before the batch's arithmetic, stores after
      // (lanes past the ensemble take zeros, as in the register form)
      const bool store = active && (pend || step);
      float* R0 = ws.R + (active ? i : 0);
      float* P0 = ws.P + (active ? i : 0);
      int j = 0;
      for (; j + MU <= bp.n; j += MU, R0 += MU * nt, P0 += MU * nt) {
        float rb[MU], pb[MU];
#pragma unroll
        for (int u = 0; u < MU; ++u) {
          rb[u] = active ? R0[u * nt] : 0.0f;
          pb[u] = active ? P0[u * nt] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < MU; ++u) mode(j + u, rb[u], pb[u]);
        if (store) {
#pragma unroll
          for (int u = 0; u < MU; ++u) {
            R0[u * nt] = rb[u];
            P0[u * nt] = pb[u];
          }
        }
      }
      for (; j < bp.n; ++j, R0 += nt, P0 += nt) {
        float r = active ? *R0 : 0.0f, p = active ? *P0 : 0.0f;
        mode(j, r, p);
        if (store) {
          *R0 = r;
          *P0 = p;
        }
      }
    };
    float t[NTRI];
    bool pend = false;
    int pa = al, pb = be;
    if constexpr (MEM) pass_dia(t, false, al, be, false);
    else build_w(t);
    pair_force();
    float w0 = diag_gap(t);  // hbar w_ab at R_n (times 1/hbar in hdt_hbar)

    // observation of the walker into slot `slot` (W(R) in t)
    auto observe = [&](int slot) {
      renormN(m, mexp);
      const bool live = active && m.hi != 0.0f;
      int ew = live ? mexp : -(1 << 28);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ew = max(ew, __shfl_xor_sync(0xffffffffu, ew, off));
      const float kq = rintf(ph.hi * kInvTwoPiN);
      ph = df_add(ph, -kq * kTwoPi1N);
      ph = df_add(ph, -kq * kTwoPi2N);
      ph = df_add(ph, -kq * kTwoPi3N);
      float sh, chh;
      __sincosf(ph.hi, &sh, &chh);
      const float mm = live ? m.hi * pow2iN(mexp - ew) : 0.0f;
      const float xr = mm * __fmaf_rn(-ph.lo, sh, chh), xi = -mm * __fmaf_rn(ph.lo, chh, sh);
      const float zr = q == 0 ? xr : (q == 1 ? -xi : (q == 2 ? -xr : xi));
      const float zi = q == 0 ? xi : (q == 1 ? xr : (q == 2 ? -xi : -xr));
      const int ex = (ew < -(1 << 27)) ? 0 : ((lane < 16) ? ew : 2 * ew);
      float W[NS][NS], e[NS], U[NS][NS];
#pragma unroll
      for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int b = 0; b < NS; ++b) W[a][b] = t[tri<NS>(a, b)];
      eigh_cold_fast<NS>(W, e, U);  // (every lane: warp votes)
      float* row = &obs_rows[threadIdx.x * 33];
      constexpr int kPassUnroll = NP <= 4 ? NP : 1;
#pragma unroll kPassUnroll
      for (int p = 0; p < NP; ++p) {
        float v[16];
        contrib_values_dia<float, NS>(U, al, be, zr, zi, p, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          row[k] = v[k];
          row[16 + k] = v[k] * v[k];
        }
        __syncwarp();
        float l1[16];
        const float* col = &obs_rows[(warp * 32) * 33 + lane];
#pragma unroll
        for (int k = 0; k < 16; ++k) l1[k] = col[(2 * k) * 33] + col[(2 * k + 1) * 33];
#pragma unroll
        for (int wdt = 8; wdt >= 1; wdt >>= 1)
#pragma unroll
          for (int k = 0; k < wdt; ++k) l1[k] = l1[2 * k] + l1[2 * k + 1];
        __syncwarp();
        const double xd = (double)l1[0];
        red[rb][warp][lane] = (ex >= -1022 && ex <= 1023) ? xd * pow2dN(ex) : ldexp(xd, ex);
        __syncthreads();
        if (threadIdx.x < 32) {
          const int qq = (lane < 16) ? 16 * p + lane : 4 * NN + 16 * p + (lane - 16);
          if (16 * p + (lane & 15) < 4 * NN)
            part[((int64_t)slot * bp.n_tiles + tile0) * 8 * NN + qq] =
                (red[rb][0][lane] + red[rb][1][lane]) + (red[rb][2][lane] + red[rb][3][lane]);
        }
        rb ^= 1;
      }
    };

    int slot = bp.obs_first;
    if (bp.obs_first) observe(0);
    int to_out = bp.to_out0;
    uint32_t blk = bp.blk0;
    int widx = bp.widx0;
    u4 wd = philox_draw(bp.seed, blk, traj, kPurposeHop);
    const float tmaxf = (float)bp.tmax;
    for (int it = 0; it < bp.len; ++it) {
      if constexpr (MEM) {
        pass_dia(t, pend, pa, pb, true);
        pend = true;  // the second half kick at R_{n+1}, with this pair
        pa = al;
        pb = be;
      } else {
        kick();  // first half kick at R_n
#pragma unroll
        for (int j = 0; j < NPL; ++j) R[j] = __fmaf_rn(cf.dtm[j], P[j], R[j]);
        build_w(t);
        kick();  // second half kick at R_{n+1} (the diagonal force's coupling part is a constant)
      }
      const float w1 = diag_gap(t);
      ph = df_add(ph, __fmul_rn(bp.hdt_hbar, __fadd_rn(w0, w1)));
      // events at R_{n+1}: slots 0..NS-1 a -> g with c = W_ga dt / hbar (three
      // quarter turns), slots NS..2NS-1 b -> g with c = W_bg dt / hbar (one);
      // the slots g = a and g = b are not events (c = 0)
      float c[NC];
#pragma unroll
      for (int g = 0; g < NS; ++g) {
        float wga = t[tri<NS>(g, 0)], wbg = wga;
#pragma unroll
        for (int h = 1; h < NS; ++h) {
          const float x = t[tri<NS>(g, h)];
          wga = (h == al) ? x : wga;
          wbg = (h == be) ? x : wbg;
        }
        c[g] = (g == al) ? 0.0f : __fmul_rn(bp.amp, wga);
        c[NS + g] = (g == be) ? 0.0f : __fmul_rn(bp.amp, wbg);
      }
      const uint32_t word = (widx & 2) ? ((widx & 1) ? wd.w : wd.z) : ((widx & 1) ? wd.y : wd.x);
      uint32_t T[NC], sumT = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const float ka = fabsf(__fmul_rn(bp.kappa, c[k]));
        T[k] = __float2uint_rz(fminf(ka * kP24f, tmaxf));
        sumT += T[k];
      }
      if (sumT > bp.tmax) {
        const float sc = (float)bp.tmax / (float)sumT;
        uint32_t s2 = 0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          T[k] = min(__float2uint_rz((float)T[k] * sc), T[k]);
          s2 += T[k];
        }
        sumT = s2;
      }
      const uint32_t y = word >> 8;
      uint32_t cum = 0;
      int cnt = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        cum += T[k];
        cnt += (y >= cum) ? 1 : 0;
      }
      const int hit = cnt < NC ? cnt : -1;
      float ch = c[0];
      uint32_t Th = T[0];
#pragma unroll
      for (int k = 1; k < NC; ++k) {
        ch = (k == hit) ? c[k] : ch;
        Th = (k == hit) ? T[k] : Th;
      }
      const bool hop = hit >= 0;
      const float num = hop ? ch * kP24f : kP24f;
      const float den = __uint2float_rn(hop ? Th : 16777216u - sumT);
      const float rd = __frcp_rn(den);
      const float q0 = __fmul_rn(num, rd);
      const float q1 = __fmul_rn(__fmaf_rn(-q0, den, num), rd);
      m = df_mul(m, q0, q1);
      if (!(fabsf(m.hi) <= 0x1p32f && fabsf(m.hi) >= 0x1p-32f)) renormN(m, mexp);
      w0 = w1;
      if (hop) {
        if (hit < NS) {
          al = hit;
          q = (q + 3) & 3;
        } else {
          be = hit - NS;
          q = (q + 1) & 3;
        }
        pair_force();
        w0 = diag_gap(t);  // the new pair's gap at R_{n+1}
      }
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
    if constexpr (MEM) {
      if (pend) pass_dia(t, true, pa, pb, false);
    }
    if (active) {
#pragma unroll
      for (int j = 0; j < NPL; ++j)
        if (j < bp.n) {
          ws.R[(int64_t)j * nt + i] = R[j];
          ws.P[(int64_t)j * nt + i] = P[j];
        }
      ws.m[i] = m.hi;
      ws.mlo[i] = m.lo;
      ws.mexp[i] = mexp;
      ws.phi[i] = ph.hi;
      ws.philo[i] = ph.lo;
      ws.ab[i] = (uint16_t)(al | (q << 4) | (be << 8));
      if (!isfinite(m.hi) || !isfinite(ph.hi)) {
        atomicAdd(&ws.hdr->n_nonfinite, 1ull);
        atomicOr(&ws.hdr->flags, QCL_FLAG_NONFINITE);
      }
    }
  }
}

}  // namespace qcl
