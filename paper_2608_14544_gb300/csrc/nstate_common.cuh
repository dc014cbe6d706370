// nstate_common.cuh -- models with N_s = 3..8 electronic states: the walker
// views of the ensemble buffer and the small helpers that the FP64 and FP32
// N_s-state kernels share (nstate_f64.cuh, nstate_bulk.cuh, nstate_spawn32.cuh).
// The per-step algorithm is the two-state one with the closed form replaced by
// a Jacobi decomposition carried along the trajectory (nstate.cuh):
// velocity Verlet on the mean force -1/2 (F_a + F_b), trapezoid phase
// (e_a - e_b)/hbar, and one transition among the 2 (N_s - 1) events of the
// coupling term of Eq. 1.
#pragma once
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

}  // namespace qcl
