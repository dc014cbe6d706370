// nstate_kernels.cuh -- models with N_s = 3..8 electronic states: sampling,
// the FP64 one-launch-per-step path, the FP32-bulk persistent kernels (the
// walker's modes in registers, or for any mode count in the ensemble buffer)
// and trajectory spawning in both precisions.
// The per-step algorithm is the two-state one with the closed form replaced by
// a Jacobi decomposition carried along the trajectory (nstate.cuh):
// velocity Verlet on the mean force -1/2 (F_a + F_b), trapezoid phase
// (e_a - e_b)/hbar, and one transition among the 2 (N_s - 1) events of the
// coupling term of Eq. 1.
#pragma once
#include <mutex>
#include <type_traits>

#include "kernels.h"
#include "nstate.cuh"
#include "reduce.cuh"

namespace qcl {

namespace nsd {

constexpr double kDegTolD = 1e-12;
constexpr float kDegTolF = 1e-6f;

template <typename T>
struct WN {
  T* R;
  T* P;
  T* m;
  T* mlo;
  int32_t* mexp;
  T* phi;
  T* philo;
  uint16_t* ab;
  T* U;  // [NS*NS][n_traj]
  T* E;  // [NS][n_traj] eigenvalues (FP32 bulk)
  EnsHeader* hdr;
};

template <typename T>
__device__ __forceinline__ WN<T> viewN(void* buf, int64_t nt, int ns, int n, int prec) {
  const EnsLayout L = EnsLayout::make(nt, ns, n, prec);
  char* b = (char*)buf;
  return {(T*)(b + L.off_R),    (T*)(b + L.off_P),       (T*)(b + L.off_m),
          (T*)(b + L.off_mlo),  (int32_t*)(b + L.off_mexp), (T*)(b + L.off_phi),
          (T*)(b + L.off_philo), (uint16_t*)(b + L.off_ab), (T*)(b + L.off_U),
          (T*)(b + L.off_E),     (EnsHeader*)b};
}

// column a of U (runtime a) without indexing a register array at run time
template <typename T, int NS>
__device__ __forceinline__ void column(const T (&U)[NS][NS], int a, T (&u)[NS]) {
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    T v = U[i][0];
#pragma unroll
    for (int c = 1; c < NS; ++c) v = (c == a) ? U[i][c] : v;
    u[i] = v;
  }
}

template <typename T, int NS>
__device__ __forceinline__ T pick(const T (&e)[NS], int a) {
  T v = e[0];
#pragma unroll
  for (int c = 1; c < NS; ++c) v = (c == a) ? e[c] : v;
  return v;
}

// W(R) = E + sum_j R_j K_j from the device model (FP64 path, R in global memory)
template <int NS>
__device__ __forceinline__ void elec_g(const DevModel* M, const double* R, int64_t nt, int n,
                                       double (&W)[NS][NS]) {
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) W[a][b] = M->E[a * NS + b];
  for (int j = 0; j < n; ++j) {
    const double x = R[(int64_t)j * nt];
    const double* Kj = M->K + (size_t)j * NS * NS;
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
      for (int b = 0; b < NS; ++b) W[a][b] += x * Kj[a * NS + b];
  }
}

// P += dt/2 F_ab, F_j = -k_j R_j - 1/2 ((U^T K_j U)_aa + (U^T K_j U)_bb)  (FP64 path;
// the Hellmann-Feynman elements accumulated in the same order as the oracle)
template <int NS>
__device__ __forceinline__ void half_kick_g(const DevModel* M, double* R, double* P, int64_t nt,
                                            int n, const double (&U)[NS][NS], int al, int be,
                                            double dt) {
  double ua[NS], ub[NS];
  column<double, NS>(U, al, ua);
  column<double, NS>(U, be, ub);
  for (int j = 0; j < n; ++j) {
    const double* Kj = M->K + (size_t)j * NS * NS;
    double ga = 0.0, gb = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int l = 0; l < NS; ++l) {
        ga += ua[k] * Kj[k * NS + l] * ua[l];
        gb += ub[k] * Kj[k * NS + l] * ub[l];
      }
    const int64_t o = (int64_t)j * nt;
    const double F = -M->k[j] * R[o] - 0.5 * (ga + gb);
    P[o] += 0.5 * dt * F;
  }
}

// Event amplitudes of the coupling term of Eq. 1 at (R, P) with decomposition
// (e, U), one slot per candidate in the fixed event order: slots 0..NS-1 move
// the first index a -> nu with A = -dt (v.d)_{nu a}, slots NS..2NS-1 move the
// second index b -> nu with A = +dt (v.d)_{b nu}; (v.d)_{mu nu} =
// u_mu^T G u_nu / (e_nu - e_mu), G = sum_j (P_j/M_j) K_j.  The slots nu = a and
// nu = b are not events (amplitude 0, never drawn), so walking the slots in
// order walks the 2 (NS - 1) events in their order.  Returns true if a needed
// gap was degenerate.
template <typename T>
__device__ __forceinline__ T quot(T a, T b) {
  return a / b;
}
template <>
__device__ __forceinline__ float quot<float>(float a, float b) {
  return __fdividef(a, b);
}

// (with columns al, be of U already extracted into ua, ub)
template <typename T, int NS>
__device__ __forceinline__ bool event_amplitudes_cols(const T (&G)[NS][NS], const T (&U)[NS][NS],
                                                      const T (&ua)[NS], const T (&ub)[NS],
                                                      const T (&e)[NS], int al, int be, T dt,
                                                      T tol, T (&A)[2 * NS],
                                                      bool (&is_event)[2 * NS]) {
  T Gua[NS], Gub[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int l = 0; l < NS; ++l) {
      s0 += G[k][l] * ua[l];
      s1 += G[k][l] * ub[l];
    }
    Gua[k] = s0;
    Gub[k] = s1;
  }
  const T ea = pick<T, NS>(e, al), eb = pick<T, NS>(e, be);
  bool deg = false;
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
#pragma unroll
    for (int nu = 0; nu < NS; ++nu) {
      T h = T(0);
#pragma unroll
      for (int k = 0; k < NS; ++k) h += U[k][nu] * (slot == 0 ? Gua[k] : Gub[k]);
      const T gap = (slot == 0) ? (ea - e[nu]) : (e[nu] - eb);
      const bool ev = (slot == 0) ? (nu != al) : (nu != be);
      const bool dg = ev && fabs(gap) < tol;
      deg |= dg;
      // FP32: approximate division (the amplitude enters a probability and a
      // weight factor, both far above its 2-ulp error)
      const T vd = (!ev || dg) ? T(0) : quot<T>(h, gap);
      A[slot * NS + nu] = (slot == 0) ? -dt * vd : dt * vd;
      is_event[slot * NS + nu] = ev;
    }
  }
  return deg;
}

template <typename T, int NS>
__device__ __forceinline__ bool event_amplitudes(const T (&G)[NS][NS], const T (&U)[NS][NS],
                                                 const T (&e)[NS], int al, int be, T dt, T tol,
                                                 T (&A)[2 * NS], bool (&is_event)[2 * NS]) {
  T ua[NS], ub[NS];
  column<T, NS>(U, al, ua);
  column<T, NS>(U, be, ub);
  return event_amplitudes_cols<T, NS>(G, U, ua, ub, e, al, be, dt, tol, A, is_event);
}

}  // namespace nsd
using namespace nsd;

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

// ------------------------------------------------------ FP32 spawning, N_s --
// Trajectory spawning for N_s-state models in FP32 bulk precision (either
// representation, any mode count: up to 8 modes in registers, beyond that in
// memory): one step per launch with the walker state in HBM, the walker arithmetic of the FP32 N_s-state kernels (the carried
// eigenvectors and eigenvalues warm-start each decomposition; the diabatic
// step needs none), compensated FP32 weight and phase pairs with a carried
// exponent.  A fired test stages a child (weight m A_e / p_hat_e, the event's
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

// ------------------------------------------------------- per-N_s launchers --
// Instantiated one N_s per translation unit; the FP64 sampling and step
// kernels in their own units (kernels_nstate64_*.cu, compiled without FMA
// contraction so that their arithmetic is the oracle's).
template <int NS>
struct NStateOps {
  static void sample64(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_sampleN_f64<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(dm, sp, buf);
  }
  static void sample32(const SampleN32& sp, void* buf, cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_sampleN_f32<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(sp, buf);
  }
  static void step64(const DevModel* dm, int repr, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st) {
    const unsigned nb = (unsigned)((nt + 127) / 128);
    if (repr == QCL_REPR_DIABATIC)
      k_stepN_dia_f64<NS><<<nb, 128, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
    else
      k_stepN_f64<NS><<<nb, 128, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
  }
  static void observe64(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                        cudaStream_t st) {
    k_observeN_f64<NS><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(dm, buf, nt, n, part);
  }
  static void spawn_sample64(const DevModel* dm, const SampleParams& sp, int64_t cap, void* buf,
                             cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_spawnN_sample<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(dm, sp, cap, buf);
    launches_add(1);
  }
  // one spawning step: step kernel, scan, scatter (set step & 1 -> the other)
  static void spawn_step64(const DevModel* dm, void* buf, int64_t cap, int n, int64_t n0,
                           int64_t step0, int64_t step, double dt, uint64_t seed,
                           cudaStream_t st) {
    const unsigned nb = spawn_grid(cap);
    k_spawnN_step<NS><<<nb, 256, 0, st>>>(dm, buf, cap, n, n0, step0, step, dt, seed);
    launch_spawn_scan(buf, cap, n, n0, QCL_PREC_FP64, NS, step0, step, st);
    k_spawnN_scatter<NS><<<nb, 256, 0, st>>>(buf, cap, n, n0, step0, step, seed);
    launches_add(2);
  }
  static void spawn_sample32(const SampleN32& sp, int64_t cap, void* buf, cudaStream_t st) {
    const int64_t nb = (sp.n_traj + 127) / 128;
    k_spawnN_sample32<NS><<<(unsigned)(nb > 0 ? nb : 1), 128, 0, st>>>(sp, cap, buf);
    launches_add(1);
  }
  template <int NPL>
  static void spawn_step32_npl(const BulkParams& bp, const CoefN& cf, void* buf, int64_t cap,
                               int64_t n0, int64_t step, cudaStream_t st) {
    // (NPL = 0: the mode table in dynamic shared memory)
    size_t dyn = 0;
    if constexpr (NPL == 0) {
      dyn = ModeRow<NS>::bytes(bp.n);
      static std::mutex mu;
      static size_t dyn_set = 0;
      std::lock_guard<std::mutex> lock(mu);
      if (dyn > dyn_set) {
        cudaFuncSetAttribute(k_spawnN_step32<NS, NPL>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        dyn_set = dyn;
      }
    }
    k_spawnN_step32<NS, NPL><<<spawn_grid(cap), 256, dyn, st>>>(bp, cf, buf, cap, n0, step);
  }
  // one FP32 spawning step (step kernel, scan, scatter): up to 8 modes in
  // registers, beyond (or under the modes-in-memory option) in memory
  static int spawn_step32(const BulkParams& bp, const CoefN& cf, void* buf, int64_t cap,
                          int64_t n0, int64_t step0, int64_t step, cudaStream_t st) {
    if (cf.modes_in_memory == 1 || bp.n > 8) spawn_step32_npl<0>(bp, cf, buf, cap, n0, step, st);
    else if (bp.n <= 4) spawn_step32_npl<4>(bp, cf, buf, cap, n0, step, st);
    else spawn_step32_npl<8>(bp, cf, buf, cap, n0, step, st);
    launch_spawn_scan(buf, cap, bp.n, n0, QCL_PREC_FP32_BULK, NS, step0, step, st);
    k_spawnN_scatter32<NS><<<spawn_grid(cap), 256, 0, st>>>(buf, cap, bp.n, n0, step0, step,
                                                            bp.seed);
    launches_add(2);
    return 1;
  }
  static void spawn_observe32(const BulkParams& bp, const CoefN& cf, const void* buf, int64_t cap,
                              int64_t n0, int set, double* part, cudaStream_t st) {
    launch_spawn_fstart(buf, cap, bp.n, n0, QCL_PREC_FP32_BULK, NS, set, st);
    k_spawnN_observe32<NS><<<(unsigned)((n0 + 127) / 128), 128, 0, st>>>(bp, cf, buf, cap, n0,
                                                                         set, part);
    launches_add(1);
  }
  static void spawn_observe64(const DevModel* dm, const void* buf, int64_t cap, int n,
                              int64_t n0, int set, double* part, cudaStream_t st) {
    launch_spawn_fstart(buf, cap, n, n0, QCL_PREC_FP64, NS, set, st);
    k_spawnN_observe<NS><<<(unsigned)((n0 + 255) / 256), 256, 0, st>>>(dm, buf, cap, n, n0, set,
                                                                       part);
    launches_add(1);
  }
  template <int NPL, int WPT = 1>
  static int bulk_npl(const BulkParams& bp, const CoefN& cf, void* buf, double* part,
                      int grid_cap, cudaStream_t st) {
    // (occupancy cached per kernel and table size: [0] adiabatic, [1] diabatic;
    // NPL = 0: the mode table in dynamic shared memory)
    static int per_sm[2] = {-1, -1}, n_sm[2] = {0, 0};
    static size_t dyn_at[2] = {0, 0};
    const size_t dyn = NPL == 0 ? ModeRow<NS>::bytes(bp.n) : 0;
    if (bp.repr == QCL_REPR_DIABATIC)
      return launch_persistent(k_bulkN_dia<NS, NPL>, per_sm[1], n_sm[1], dyn_at[1], bp, cf, buf,
                               part, grid_cap, 1, dyn, st);
    return launch_persistent(k_bulkN<NS, NPL, WPT>, per_sm[0], n_sm[0], dyn_at[0], bp, cf, buf,
                             part, grid_cap, WPT, dyn, st);
  }
  // one persistent grid: the occupancy limit of resident blocks on every SM
  // (capped), at most one block per WPT tiles
  // (dyn > 0, the modes-in-memory kernels: the shared-memory limit only grows
  // and the occupancy is computed for this call's table, under a lock, so
  // that threads launching models of different mode counts do not race)
  template <typename Fn>
  static int launch_persistent(Fn fn, int& per_sm, int& n_sm, size_t& dyn_at, const BulkParams& bp,
                               const CoefN& cf, void* buf, double* part, int grid_cap, int WPT,
                               size_t dyn, cudaStream_t st) {
    int blocks = per_sm;
    if (dyn > 0) {
      static std::mutex mu;
      std::lock_guard<std::mutex> lock(mu);
      if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      }
      if (dyn > dyn_at) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        dyn_at = dyn;
      }
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 128, dyn) != cudaSuccess ||
          blocks < 1)
        blocks = 1;
    } else if (per_sm < 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 128, 0) != cudaSuccess ||
          blocks < 1)
        blocks = 1;
      per_sm = blocks;
    }
    int64_t grid = (int64_t)blocks * n_sm;
    if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
    const int64_t units = (bp.n_tiles + WPT - 1) / WPT;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    fn<<<(unsigned)grid, 128, dyn, st>>>(bp, cf, buf, part);
    return (int)grid;
  }
  // wpt: walkers per thread asked for.  The kernel takes one or two, but only
  // one is instantiated: two walkers per thread (packed lanes, 205-245
  // registers, 8 resident warps per SM) measured 10 % slower on a four-state
  // six-mode model than one (114 registers, 16 warps), with the same bits.
  static int bulk(const BulkParams& bp, const CoefN& cf, void* buf, double* part, int grid_cap,
                  int wpt, cudaStream_t st) {
    (void)wpt;
    // Register forms exist up to 8 modes for any N_s and up to 32 modes for
    // N_s <= 4 (larger N_s x modes would not fit a walker in registers); the
    // modes-in-memory form takes any mode count with the same bits.  The
    // automatic choice follows measured solve rates on GB300 (1e6 walkers,
    // 200 steps, random LVC models): registers for N_s = 3 (except adiabatic
    // models of 9-16 modes, where the 32-mode register form is 10-30 % slower)
    // and for N_s = 4 up to 8 modes (20-30 % faster); the memory form beyond
    // (N_s = 4 with 12-32 modes: 1.3-2.6x faster) and for N_s >= 5 at every
    // mode count (1.0-2.2x, the register forms there run one or two blocks per
    // SM).  Models of at most 4 or 6 modes get their own instantiations,
    // which skip the padding modes' arithmetic (padding modes have zero
    // coefficients and stay at zero).
    const int reg_max = NS <= 4 ? 32 : 8;
    bool mem;
    if (cf.modes_in_memory == 1) mem = true;
    else if (cf.modes_in_memory == 2) mem = bp.n > reg_max;
    else if (NS == 3) mem = bp.n > 32 || (bp.repr != QCL_REPR_DIABATIC && bp.n > 8 && bp.n <= 16);
    else if (NS == 4) mem = bp.n > 8;
    else mem = true;
    if (mem) return bulk_npl<0>(bp, cf, buf, part, grid_cap, st);
    if constexpr (NS <= 5) {
      if (bp.n <= 4) return bulk_npl<4>(bp, cf, buf, part, grid_cap, st);
      if (bp.n <= 6) return bulk_npl<6>(bp, cf, buf, part, grid_cap, st);
    }
    if (bp.n <= 8) return bulk_npl<8>(bp, cf, buf, part, grid_cap, st);
    if (NS <= 4 && bp.n <= 32) return bulk_npl<(NS <= 4 ? 32 : 8)>(bp, cf, buf, part, grid_cap, st);
    return 0;
  }
};

}  // namespace qcl
