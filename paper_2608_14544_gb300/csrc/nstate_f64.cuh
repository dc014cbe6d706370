// nstate_f64.cuh -- the FP64 path of N_s-state models: sampling, one launch
// per step (adiabatic and diabatic), observation and trajectory spawning, in
// the oracle's operation order (its units are compiled without multiply-add
// contraction).
#pragma once
#include "nstate_common.cuh"

namespace qcl {

// ----------------------------------------------------------- FP64 sampling --
// One initial walker (FP64): Wigner (R, P) at Rg[j * stride], Pg[j * stride],
// the decomposition U at R_0, and the pair drawn from |rho| (U^T rho_el0 U in
// the adiabatic basis, rho_el0 itself in the diabatic one) with m_0 = rho /
// p_hat.
template <int NS>
__device__ __forceinline__ void sample_walkerN_f64(const DevModel* __restrict__ M,
                                                   const SampleParams& sp, uint64_t traj,
                                                   double* Rg, double* Pg, int64_t stride,
                                                   double& m0, uint16_t& ab,
                                                   double (&U)[NS][NS]) {
  const int n = sp.n;
  for (int j = 0; j < n; ++j) {
    double R = sp.R0[j], P = sp.P0[j];
    if (sp.wigner) {
      const u4 wd = philox_draw(sp.seed, (uint32_t)j, traj, kPurposeInit);
      const double u0 = ((double)wd.x + 0.5) * 0x1p-32;
      const double u1 = ((double)wd.y + 0.5) * 0x1p-32;
      const double rad = sqrt(-2.0 * log(u0));
      double sn, cs;
      sincospi(2.0 * u1, &sn, &cs);
      R += sp.sR[j] * rad * cs;
      P += sp.sP[j] * rad * sn;
    }
    Rg[(int64_t)j * stride] = R;
    Pg[(int64_t)j * stride] = P;
  }
  double W[NS][NS], e[NS];
  elec_g<NS>(M, Rg, stride, n, W);
  eigh_ns<double, NS>(W, nullptr, e, U, 100, 1e-34);
  // the pair's density: U^T rho U in the adiabatic basis, rho itself in the
  // diabatic one
  const bool dia = M->repr == QCL_REPR_DIABATIC;
  double rho_ad[NS * NS];
#pragma unroll
  for (int al = 0; al < NS; ++al)
#pragma unroll
    for (int be = 0; be < NS; ++be) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int l = 0; l < NS; ++l) acc += U[k][al] * sp.rho[k * NS + l] * U[l][be];
      rho_ad[al * NS + be] = dia ? sp.rho[al * NS + be] : acc;
    }
  double tot = 0.0;
  for (int k = 0; k < NS * NS; ++k) tot += fabs(rho_ad[k]);
  uint32_t Tk[NS * NS];
  uint64_t sumT = 0;
  int last = 0;
  for (int k = 0; k < NS * NS; ++k) {
    Tk[k] = (uint32_t)floor(fabs(rho_ad[k]) / tot * kP24);
    sumT += Tk[k];
    if (rho_ad[k] != 0.0) last = k;
  }
  Tk[last] += (uint32_t)(16777216ull - sumT);
  const u4 wd = philox_draw(sp.seed, (uint32_t)n, traj, kPurposeInit);
  const uint32_t y = wd.x >> 8;
  uint64_t cum = 0;
  int pickk = last;
  for (int k = 0; k < NS * NS; ++k) {
    cum += Tk[k];
    if ((uint64_t)y < cum) {
      pickk = k;
      break;
    }
  }
  m0 = rho_ad[pickk] / ((double)Tk[pickk] / kP24);
  ab = (uint16_t)((pickk / NS) | ((pickk % NS) << 8));
}

template <int NS>
__global__ void __launch_bounds__(128) k_sampleN_f64(const DevModel* __restrict__ M,
                                                     SampleParams sp, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = sp.n_traj;
  const int n = sp.n;
  WN<double> w = viewN<double>(buf, nt, NS, n, QCL_PREC_FP64);
  if (i == 0) {
    w.hdr->magic = kEnsMagic;
    w.hdr->n_traj = nt;
    w.hdr->precision = QCL_PREC_FP64;
    w.hdr->ns = NS;
    w.hdr->n = n;
    w.hdr->step = 0;
    w.hdr->flags = 0;
    w.hdr->n_degenerate = 0;
    w.hdr->n_nonfinite = 0;
  }
  if (i >= nt) return;
  double U[NS][NS];
  double m0;
  uint16_t ab;
  sample_walkerN_f64<NS>(M, sp, sp.traj_offset + (uint64_t)i, w.R + i, w.P + i, nt, m0, ab, U);
  w.m[i] = m0;
  w.phi[i] = 0.0;
  w.ab[i] = ab;
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) w.U[(int64_t)(a * NS + b) * nt + i] = U[a][b];
}

// --------------------------------------------------------------- FP64 step --
// Outcome of one walker's FP64 N_s-state step (either representation): the
// event slot drawn (-1: none), its amplitude and threshold, the sum of all
// thresholds (for the stay factor) and whether a gap was degenerate.  The
// caller applies it: a moving walker takes the hop or the stay factor, a
// spawning walker stages a child and keeps its own pair and weight.
struct StepN {
  int hit;
  double A;
  uint64_t T, sumT;
  bool deg;
};

// The draw of `step` for the walker with random stream `traj` among the
// slots' thresholds, in slot order.
template <int NC>
__device__ __forceinline__ StepN draw_event(const double (&A)[NC], const uint64_t (&T)[NC],
                                            uint64_t sumT, bool deg, uint64_t seed, uint64_t traj,
                                            int64_t step) {
  const u4 wd = philox_draw(seed, (uint32_t)(step >> 2), traj, kPurposeHop);
  const uint64_t y = word_of(wd, (int)(step & 3)) >> 8;
  uint64_t cum = 0;
  int hit = -1;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    cum += T[k];
    if (hit < 0 && y < cum) hit = k;
  }
  double Ah = A[0];
  uint64_t Th = T[0];
#pragma unroll
  for (int k = 1; k < NC; ++k) {
    Ah = (k == hit) ? A[k] : Ah;
    Th = (k == hit) ? T[k] : Th;
  }
  return {hit, Ah, Th, sumT, deg};
}

// Adiabatic pairs: velocity Verlet on the pair's mean force with the
// decompositions at R_n and R_{n+1} (gauge following the carried eigenvectors
// Uc; U1 receives those at R_{n+1}), the trapezoid phase, the 2 N_s event
// slots' amplitudes and thresholds, and the draw.  R and P at R[j * nt].
template <int NS>
__device__ __forceinline__ StepN walker_stepN_f64(const DevModel* __restrict__ M, double* R,
                                                  double* P, int64_t nt, int n, int al, int be,
                                                  double& phi, const double (&Uc)[NS][NS],
                                                  double (&U1)[NS][NS], double dt, uint64_t seed,
                                                  uint64_t traj, int64_t step) {
  double W[NS][NS], e0[NS], U0[NS][NS], e1[NS];
  // decomposition at R_n, gauge following the carried eigenvectors
  elec_g<NS>(M, R, nt, n, W);
  eigh_ns<double, NS>(W, Uc, e0, U0, 100, 1e-34, false);
  half_kick_g<NS>(M, R, P, nt, n, U0, al, be, dt);
  for (int j = 0; j < n; ++j) R[(int64_t)j * nt] += dt * P[(int64_t)j * nt] / M->mass[j];
  elec_g<NS>(M, R, nt, n, W);
  eigh_ns<double, NS>(W, U0, e1, U1, 100, 1e-34, false);
  half_kick_g<NS>(M, R, P, nt, n, U1, al, be, dt);
  const double w0 = (pick<double, NS>(e0, al) - pick<double, NS>(e0, be)) / M->hbar;
  const double w1 = (pick<double, NS>(e1, al) - pick<double, NS>(e1, be)) / M->hbar;
  phi += 0.5 * dt * (w0 + w1);
  bool deg = false;
#pragma unroll
  for (int a = 0; a + 1 < NS; ++a) deg |= (e0[a + 1] - e0[a] < kDegTolD) || (e1[a + 1] - e1[a] < kDegTolD);
  // event amplitudes, accumulated mode by mode as sum_j (P_j/M_j) d_j with the
  // Hellmann-Feynman couplings d_j = (U^T K_j U)_{mu nu} / (e_nu - e_mu)
  constexpr int NC = 2 * NS;
  double A[NC];
  bool ev[NC];
  {
    double ua[NS], ub[NS];
    column<double, NS>(U1, al, ua);
    column<double, NS>(U1, be, ub);
    const double ea = pick<double, NS>(e1, al), eb = pick<double, NS>(e1, be);
    double acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.0;
#pragma unroll
    for (int nu = 0; nu < NS; ++nu) {
      ev[nu] = nu != al;
      ev[NS + nu] = nu != be;
      deg |= (ev[nu] && fabs(ea - e1[nu]) < kDegTolD) || (ev[NS + nu] && fabs(e1[nu] - eb) < kDegTolD);
    }
    for (int j = 0; j < n; ++j) {
      const double v = P[(int64_t)j * nt] / M->mass[j];
      const double* Kj = M->K + (size_t)j * NS * NS;
#pragma unroll
      for (int nu = 0; nu < NS; ++nu) {
        double r0 = 0.0, r1 = 0.0;  // (U^T K_j U)_{nu a} and (U^T K_j U)_{b nu}
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
          for (int l = 0; l < NS; ++l) {
            r0 += U1[k][nu] * Kj[k * NS + l] * ua[l];
            r1 += ub[k] * Kj[k * NS + l] * U1[l][nu];
          }
        const double g0 = ea - e1[nu], g1 = e1[nu] - eb;
        const double d0 = (!ev[nu] || fabs(g0) < kDegTolD) ? 0.0 : r0 / g0;
        const double d1 = (!ev[NS + nu] || fabs(g1) < kDegTolD) ? 0.0 : r1 / g1;
        acc[nu] += v * d0;
        acc[NS + nu] += v * d1;
      }
    }
#pragma unroll
    for (int nu = 0; nu < NS; ++nu) {
      A[nu] = -dt * acc[nu];
      A[NS + nu] = dt * acc[NS + nu];
    }
  }
  // thresholds: min(kappa |A|, p_max) quantised to 2^-24, scaled down together in
  // exact integers when their sum exceeds Tmax = floor(p_max 2^24)
  uint64_t T[NC], sumT = 0;
  const uint64_t Tmax = (uint64_t)floor(M->p_max * kP24);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const double p = fmin(M->hop_scale * fabs(A[k]), M->p_max);
    T[k] = ev[k] ? (uint64_t)floor(p * kP24) : 0;
    sumT += T[k];
  }
  if (sumT > Tmax) {
    const uint64_t s = sumT;
    sumT = 0;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      T[k] = T[k] * Tmax / s;
      sumT += T[k];
    }
  }
  return draw_event<NC>(A, T, sumT, deg, seed, traj, step);
}

template <int NS>
__global__ void __launch_bounds__(128) k_stepN_f64(const DevModel* __restrict__ M, void* buf,
                                                   int64_t nt, int n, int64_t step0, int64_t step,
                                                   double dt, uint64_t seed, uint64_t traj_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  WN<double> w = viewN<double>(buf, nt, NS, n, QCL_PREC_FP64);
  if (i >= nt) return;
  if (w.hdr->step != step0) {
    if (i == 0) atomicOr(&w.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  const uint16_t ab = w.ab[i];
  int al = ab & 0xf, be = (ab >> 8) & 0xf;
  double m = w.m[i], phi = w.phi[i];
  double Uc[NS][NS], U1[NS][NS];
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) Uc[a][b] = w.U[(int64_t)(a * NS + b) * nt + i];
  const StepN o = walker_stepN_f64<NS>(M, w.R + i, w.P + i, nt, n, al, be, phi, Uc, U1, dt, seed,
                                       traj_off + (uint64_t)i, step);
  if (o.hit < 0) {
    m = m / (1.0 - (double)o.sumT / kP24);
  } else {
    m = m * o.A / ((double)o.T / kP24);
    if (o.hit < NS) al = o.hit;
    else be = o.hit - NS;
  }
  w.m[i] = m;
  w.phi[i] = phi;
  w.ab[i] = (uint16_t)(al | (be << 8));
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) w.U[(int64_t)(a * NS + b) * nt + i] = U1[a][b];
  if (o.deg) {
    atomicAdd(&w.hdr->n_degenerate, 1ull);
    atomicOr(&w.hdr->flags, QCL_FLAG_DEGENERATE);
  }
  if (!isfinite(m) || !isfinite(phi)) {
    atomicAdd(&w.hdr->n_nonfinite, 1ull);
    atomicOr(&w.hdr->flags, QCL_FLAG_NONFINITE);
  }
}

// --------------------------------------------------------- FP64 diabatic step --
// The diabatic representation (pairs of the R-independent basis of W, weights
// carried with a quarter-turn count q in bits 4-5 of the pair word): velocity
// Verlet on the diagonal mean force F_j = -k_j R_j - 1/2 (K_j,aa + K_j,bb), the
// trapezoid phase with hbar w_ab = W_aa - W_bb, and one transition among the
// coupling term's 2 (N_s - 1) events at R_{n+1}: the first index a -> g with
// amplitude -i c, c = W_ga dt / hbar (three quarter turns), or the second
// b -> g with +i c, c = W_bg dt / hbar (one quarter turn); probabilities
// min(kappa |c|, p_max) quantised and scaled as in the adiabatic step.
template <int NS>
__device__ __forceinline__ void dia_kick_g(const DevModel* M, double* R, double* P, int64_t nt,
                                           int n, int al, int be, double dt) {
  for (int j = 0; j < n; ++j) {
    const double* Kj = M->K + (size_t)j * NS * NS;
    double kaa = Kj[0], kbb = Kj[0];
#pragma unroll
    for (int c = 1; c < NS; ++c) {
      kaa = (c == al) ? Kj[c * NS + c] : kaa;
      kbb = (c == be) ? Kj[c * NS + c] : kbb;
    }
    const int64_t o = (int64_t)j * nt;
    const double F = -M->k[j] * R[o] - 0.5 * (kaa + kbb);
    P[o] += 0.5 * dt * F;
  }
}

template <int NS>
__device__ __forceinline__ double diag_pick(const double (&W)[NS][NS], int a) {
  double v = W[0][0];
#pragma unroll
  for (int c = 1; c < NS; ++c) v = (c == a) ? W[c][c] : v;
  return v;
}

// Diabatic pairs: the deterministic part and the draw (A = c, the real factor
// of the event's amplitude; slot < NS takes three quarter turns, the others one).
template <int NS>
__device__ __forceinline__ StepN walker_stepN_dia_f64(const DevModel* __restrict__ M, double* R,
                                                      double* P, int64_t nt, int n, int al, int be,
                                                      double& phi, double dt, uint64_t seed,
                                                      uint64_t traj, int64_t step) {
  double W0[NS][NS], W1[NS][NS];
  elec_g<NS>(M, R, nt, n, W0);
  dia_kick_g<NS>(M, R, P, nt, n, al, be, dt);
  for (int j = 0; j < n; ++j) R[(int64_t)j * nt] += dt * P[(int64_t)j * nt] / M->mass[j];
  elec_g<NS>(M, R, nt, n, W1);
  dia_kick_g<NS>(M, R, P, nt, n, al, be, dt);
  const double w0 = (diag_pick<NS>(W0, al) - diag_pick<NS>(W0, be)) / M->hbar;
  const double w1 = (diag_pick<NS>(W1, al) - diag_pick<NS>(W1, be)) / M->hbar;
  phi += 0.5 * dt * (w0 + w1);
  // slots 0..NS-1: a -> g with c = W_ga dt / hbar; slots NS..2NS-1: b -> g with
  // c = W_bg dt / hbar; the slots g = a and g = b are not events (T = 0)
  constexpr int NC = 2 * NS;
  double c[NC];
  bool ev[NC];
#pragma unroll
  for (int g = 0; g < NS; ++g) {
    double wga = W1[g][0], wbg = W1[0][g];
#pragma unroll
    for (int h = 1; h < NS; ++h) {
      wga = (h == al) ? W1[g][h] : wga;
      wbg = (h == be) ? W1[h][g] : wbg;
    }
    c[g] = wga * dt / M->hbar;
    c[NS + g] = wbg * dt / M->hbar;
    ev[g] = g != al;
    ev[NS + g] = g != be;
  }
  uint64_t T[NC], sumT = 0;
  const uint64_t Tmax = (uint64_t)floor(M->p_max * kP24);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const double p = fmin(M->hop_scale * fabs(c[k]), M->p_max);
    T[k] = ev[k] ? (uint64_t)floor(p * kP24) : 0;
    sumT += T[k];
  }
  if (sumT > Tmax) {
    const uint64_t s = sumT;
    sumT = 0;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      T[k] = T[k] * Tmax / s;
      sumT += T[k];
    }
  }
  return draw_event<NC>(c, T, sumT, false, seed, traj, step);
}

template <int NS>
__global__ void __launch_bounds__(128) k_stepN_dia_f64(const DevModel* __restrict__ M, void* buf,
                                                       int64_t nt, int n, int64_t step0,
                                                       int64_t step, double dt, uint64_t seed,
                                                       uint64_t traj_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  WN<double> w = viewN<double>(buf, nt, NS, n, QCL_PREC_FP64);
  if (i >= nt) return;
  if (w.hdr->step != step0) {
    if (i == 0) atomicOr(&w.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  const uint16_t ab = w.ab[i];
  int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
  double m = w.m[i], phi = w.phi[i];
  const StepN o = walker_stepN_dia_f64<NS>(M, w.R + i, w.P + i, nt, n, al, be, phi, dt, seed,
                                           traj_off + (uint64_t)i, step);
  if (o.hit < 0) {
    m = m / (1.0 - (double)o.sumT / kP24);
  } else {
    m = m * o.A / ((double)o.T / kP24);
    if (o.hit < NS) {
      al = o.hit;
      q = (q + 3) & 3;
    } else {
      be = o.hit - NS;
      q = (q + 1) & 3;
    }
  }
  w.m[i] = m;
  w.phi[i] = phi;
  w.ab[i] = (uint16_t)(al | (q << 4) | (be << 8));
  if (!isfinite(m) || !isfinite(phi)) {
    atomicAdd(&w.hdr->n_nonfinite, 1ull);
    atomicOr(&w.hdr->flags, QCL_FLAG_NONFINITE);
  }
}

// --------------------------------------------------------- FP64 observation --
// Contributions in passes of 32 quantities: pass p holds values 16p..16p+15
// (lanes 0-15 of the reduce-scatter) and their squares (lanes 16-31).
template <typename T, int NS>
__device__ __forceinline__ void contrib_values(const T (&U)[NS][NS], int al, int be, T zr, T zi,
                                               int p, T (&v)[16]) {
  T ua[NS], ub[NS];
  column<T, NS>(U, al, ua);
  column<T, NS>(U, be, ub);
  constexpr int NN = NS * NS;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int q = 16 * p + t;  // quantity index in [0, 4 NN)
    T val = T(0);
    if (q < 2 * NN) {  // diabatic rho_ij, q = 2 (i NS + j) + c
      const int ij = q >> 1, ii = ij / NS, jj = ij % NS;
      const T f = ua[ii] * ub[jj];
      val = (q & 1) ? zi * f : zr * f;
    } else if (q < 4 * NN) {  // adiabatic rho_ab at the walker's pair
      const int ab = (q - 2 * NN) >> 1;
      const bool hit = ab == al * NS + be;
      val = hit ? ((q & 1) ? zi : zr) : T(0);
    }
    v[t] = val;
  }
}

// A diabatic walker's contributions: z at its own pair in the diabatic block,
// z U_ai U_bj (rows a, b of the eigenvectors at its R) in the adiabatic one.
template <typename T, int NS>
__device__ __forceinline__ void contrib_values_dia(const T (&U)[NS][NS], int al, int be, T zr,
                                                   T zi, int p, T (&v)[16]) {
  T ra[NS], rb[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    T x = U[0][k], y = U[0][k];
#pragma unroll
    for (int c = 1; c < NS; ++c) {
      x = (c == al) ? U[c][k] : x;
      y = (c == be) ? U[c][k] : y;
    }
    ra[k] = x;
    rb[k] = y;
  }
  constexpr int NN = NS * NS;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int q = 16 * p + t;
    T val = T(0);
    if (q < 2 * NN) {  // diabatic rho_ij at the walker's pair
      const int ij = q >> 1;
      const bool hit = ij == al * NS + be;
      val = hit ? ((q & 1) ? zi : zr) : T(0);
    } else if (q < 4 * NN) {  // adiabatic rho_kl, q = 2 NN + 2 (k NS + l) + c
      const int kl = (q - 2 * NN) >> 1, kk = kl / NS, ll = kl % NS;
      const T f = ra[kk] * rb[ll];
      val = (q & 1) ? zi * f : zr * f;
    }
    v[t] = val;
  }
}

template <int NS>
__global__ void __launch_bounds__(256) k_observeN_f64(const DevModel* __restrict__ M,
                                                      const void* buf, int64_t nt, int n,
                                                      double* __restrict__ part) {
  __shared__ double red[8][32];
  constexpr int NN = NS * NS, NP = (4 * NN + 15) / 16;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  WN<double> w = viewN<double>((void*)buf, nt, NS, n, QCL_PREC_FP64);
  const bool dia = M->repr == QCL_REPR_DIABATIC;
  double U[NS][NS];
  double zr = 0.0, zi = 0.0;
  int al = 0, be = 0;
  if (i < nt) {
    if (dia) {  // the eigenvectors at the walker's R, decomposed afresh
      double W[NS][NS], e[NS];
      elec_g<NS>(M, w.R + i, nt, n, W);
      eigh_ns<double, NS>(W, nullptr, e, U, 100, 1e-34);
    } else {
#pragma unroll
      for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int b = 0; b < NS; ++b) U[a][b] = w.U[(int64_t)(a * NS + b) * nt + i];
    }
    const uint16_t ab = w.ab[i];
    al = ab & 0xf;
    be = (ab >> 8) & 0xf;
    const int qt = (ab >> 4) & 3;  // quarter turns (diabatic walkers): z = m exp(-i phi) i^q
    double sn, cs;
    sincos(w.phi[i], &sn, &cs);
    const double xr = w.m[i] * cs, xi = -w.m[i] * sn;
    zr = qt == 0 ? xr : (qt == 1 ? -xi : (qt == 2 ? -xr : xi));
    zi = qt == 0 ? xi : (qt == 1 ? xr : (qt == 2 ? -xi : -xr));
  } else {
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
      for (int b = 0; b < NS; ++b) U[a][b] = 0.0;
  }
  for (int p = 0; p < NP; ++p) {
    double v16[16];
    if (dia) contrib_values_dia<double, NS>(U, al, be, zr, zi, p, v16);
    else contrib_values<double, NS>(U, al, be, zr, zi, p, v16);
    double v[32];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      v[t] = v16[t];
      v[16 + t] = v16[t] * v16[t];
    }
    const double x = warp_transpose_sum<double>(v);
    red[threadIdx.x >> 5][threadIdx.x & 31] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const int q = (lane < 16) ? 16 * p + lane : 4 * NN + 16 * p + (lane - 16);
      if (16 * p + (lane & 15) < 4 * NN)
        part[(int64_t)blockIdx.x * 8 * NN + q] = tile_tree8(&red[0][0], 32, lane);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------ FP64 spawning, N_s --
// Trajectory spawning for N_s-state models (FP64, either representation): the
// two-state scheme with the N_s-state step.  Every step a walker whose
// transition test fires keeps its pair, eigenvectors and weight and spawns a
// child at the event's target pair with weight m A_e / p_hat_e (the diabatic
// one with the event's quarter turns); children follow their parents by the
// same count / scan / scatter, so the walker order is reproducible bit for
// bit and each family stays contiguous.
struct SetN {
  double* R;
  double* P;
  double* m;
  double* phi;
  uint16_t* ab;
  uint64_t* id;
  uint32_t* fam;
  double* U;  // [NS * NS][cap]
};

__device__ __forceinline__ SetN spawn_setN(void* buf, const SpawnLayout& L, int set) {
  char* b = (char*)buf + L.set_off[set];
  return {(double*)(b + L.R),   (double*)(b + L.P),    (double*)(b + L.m),
          (double*)(b + L.phi), (uint16_t*)(b + L.ab), (uint64_t*)(b + L.id),
          (uint32_t*)(b + L.fam), (double*)(b + L.U)};
}

// Random-stream id of the child spawned at `step` by the walker `parent`
// (the two-state spawning's: words 0 and 1 of Philox block (step, parent,
// purpose 3), bit 63 set).
__device__ __forceinline__ uint64_t spawn_child_id(uint64_t seed, int64_t step, uint64_t parent) {
  const u4 w = philox_draw(seed, (uint32_t)step, parent, 3u);
  return (((uint64_t)w.y << 32) | w.x) | (1ull << 63);
}

template <int NS>
__global__ void __launch_bounds__(128) k_spawnN_sample(const DevModel* __restrict__ M,
                                                       SampleParams sp, int64_t cap, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n0 = sp.n_traj;
  const SpawnLayout L = SpawnLayout::make(cap, sp.n, n0, QCL_PREC_FP64, NS);
  EnsHeader* hdr = (EnsHeader*)buf;
  SpawnHeader* sh = (SpawnHeader*)((char*)buf + kSpawnHeaderOff);
  if (i == 0) {
    hdr->magic = kEnsMagic;
    hdr->n_traj = n0;
    hdr->precision = QCL_PREC_FP64;
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
  const SetN w = spawn_setN(buf, L, 0);
  const uint64_t traj = sp.traj_offset + (uint64_t)i;
  double U[NS][NS];
  double m0;
  uint16_t ab;
  sample_walkerN_f64<NS>(M, sp, traj, w.R + i, w.P + i, cap, m0, ab, U);
  w.m[i] = m0;
  w.phi[i] = 0.0;
  w.ab[i] = ab;
  w.id[i] = traj;
  w.fam[i] = (uint32_t)i;
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) w.U[(int64_t)(a * NS + b) * cap + i] = U[a][b];
}

// Step of every live walker of set `src` in place; the children's weights and
// pair words go to the per-parent staging arrays, each group's child count to
// bsum (groups of 256 walkers, as the scan expects).
template <int NS>
__global__ void __launch_bounds__(256) k_spawnN_step(const DevModel* __restrict__ M, void* buf,
                                                     int64_t cap, int n, int64_t n0, int64_t step0,
                                                     int64_t step, double dt, uint64_t seed) {
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP64, NS);
  EnsHeader* hdr = (EnsHeader*)buf;
  const int src = (int)(step & 1);
  const int64_t n_live = ((SpawnHeader*)((char*)buf + kSpawnHeaderOff))->n_live[src];
  if (hdr->step != step0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  const bool dia = M->repr == QCL_REPR_DIABATIC;
  const int64_t nvb = (n_live + 255) / 256;
  for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const int64_t i = vb * 256 + threadIdx.x;
    int flag = 0;
    if (i < n_live) {
      const SetN w = spawn_setN(buf, L, src);
      const uint16_t ab = w.ab[i];
      const int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
      double phi = w.phi[i];
      const double m = w.m[i];
      StepN o;
      if (dia) {
        o = walker_stepN_dia_f64<NS>(M, w.R + i, w.P + i, cap, n, al, be, phi, dt, seed, w.id[i],
                                     step);
      } else {
        double Uc[NS][NS], U1[NS][NS];
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) Uc[a][b] = w.U[(int64_t)(a * NS + b) * cap + i];
        o = walker_stepN_f64<NS>(M, w.R + i, w.P + i, cap, n, al, be, phi, Uc, U1, dt, seed,
                                 w.id[i], step);
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) w.U[(int64_t)(a * NS + b) * cap + i] = U1[a][b];
      }
      w.phi[i] = phi;
      flag = o.hit >= 0;
      uint8_t* fl = (uint8_t*)((char*)buf + L.flag);
      fl[i] = (uint8_t)flag;
      if (flag) {
        const double mc = m * o.A / ((double)o.T / kP24);
        const bool first = o.hit < NS;
        const int ca = first ? o.hit : al, cb = first ? be : o.hit - NS;
        const int cq = dia ? ((q + (first ? 3 : 1)) & 3) : q;
        ((double*)((char*)buf + L.cm))[i] = mc;
        ((uint16_t*)((char*)buf + L.cab))[i] = (uint16_t)(ca | (cq << 4) | (cb << 8));
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

// Moves every live walker of set src (eigenvectors too) to its place in the
// other set, after the children of the walkers before it, and writes each
// child right after its parent.
template <int NS>
__global__ void __launch_bounds__(256) k_spawnN_scatter(void* buf, int64_t cap, int n, int64_t n0,
                                                        int64_t step0, int64_t step,
                                                        uint64_t seed) {
  __shared__ int wcnt[8];
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP64, NS);
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
      const SetN s = spawn_setN(buf, L, src);
      const SetN d = spawn_setN(buf, L, src ^ 1);
      for (int j = 0; j < n; ++j) {
        const double r = s.R[(int64_t)j * cap + i], p = s.P[(int64_t)j * cap + i];
        d.R[(int64_t)j * cap + pos] = r;
        d.P[(int64_t)j * cap + pos] = p;
        if (flag) {
          d.R[(int64_t)j * cap + pos + 1] = r;
          d.P[(int64_t)j * cap + pos + 1] = p;
        }
      }
#pragma unroll
      for (int k = 0; k < NS * NS; ++k) {
        const double u = s.U[(int64_t)k * cap + i];
        d.U[(int64_t)k * cap + pos] = u;
        if (flag) d.U[(int64_t)k * cap + pos + 1] = u;
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
        d.id[pos + 1] = spawn_child_id(seed, step, id);
        d.fam[pos + 1] = fam;
      }
    }
    __syncthreads();  // wcnt is rewritten by the next group
  }
}

// One thread per family: the family sum X of its walkers' 4 N_s^2
// contributions (in walker order), then X and X^2 reduced over the tile's 256
// families by the fixed tree of the observation kernel, in passes of 16.
template <int NS>
__global__ void __launch_bounds__(256) k_spawnN_observe(const DevModel* __restrict__ M,
                                                        const void* buf, int64_t cap, int n,
                                                        int64_t n0, int set,
                                                        double* __restrict__ part) {
  __shared__ double red[8][32];
  constexpr int NN = NS * NS, NQ = 4 * NN, NP = (NQ + 15) / 16;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const SpawnLayout L = SpawnLayout::make(cap, n, n0, QCL_PREC_FP64, NS);
  const SetN s = spawn_setN((void*)buf, L, set);
  const int64_t* fstart = (const int64_t*)((const char*)buf + L.fstart);
  const bool dia = M->repr == QCL_REPR_DIABATIC;
  double X[NQ];
  for (int t = 0; t < NQ; ++t) X[t] = 0.0;
  if (k < n0) {
    const int64_t j0 = fstart[k], j1 = fstart[k + 1];
    for (int64_t j = j0; j < j1; ++j) {
      double U[NS][NS];
      if (dia) {
        double W[NS][NS], e[NS];
        elec_g<NS>(M, s.R + j, cap, n, W);
        eigh_ns<double, NS>(W, nullptr, e, U, 100, 1e-34);
      } else {
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) U[a][b] = s.U[(int64_t)(a * NS + b) * cap + j];
      }
      const uint16_t ab = s.ab[j];
      const int al = ab & 0xf, be = (ab >> 8) & 0xf, qt = (ab >> 4) & 3;
      double sn, cs;
      sincos(s.phi[j], &sn, &cs);
      const double xr = s.m[j] * cs, xi = -s.m[j] * sn;
      const double zr = qt == 0 ? xr : (qt == 1 ? -xi : (qt == 2 ? -xr : xi));
      const double zi = qt == 0 ? xi : (qt == 1 ? xr : (qt == 2 ? -xi : -xr));
      for (int p = 0; p < NP; ++p) {
        double v16[16];
        if (dia) contrib_values_dia<double, NS>(U, al, be, zr, zi, p, v16);
        else contrib_values<double, NS>(U, al, be, zr, zi, p, v16);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (16 * p + t < NQ) X[16 * p + t] += v16[t];
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
        part[(int64_t)blockIdx.x * 8 * NN + qq] = tile_tree8(&red[0][0], 32, lane);
    }
    __syncthreads();
  }
}

}  // namespace qcl
