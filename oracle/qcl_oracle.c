/*
 * qcl_oracle.c -- plain FP64 CPU oracle for momentum-jump-free QCL dynamics.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product path.  Plain, slow,
 * one walker at a time, every step written in the order the method states it.
 * Compile with -ffp-contract=off so that the results do not depend on whether
 * the host compiler fuses multiply-adds.
 *
 * Readings where the paper is silent (the paper defers the algorithm to its
 * Refs. Santer 2001 and Ando 2003, which are not reproduced in it):
 *  - integrator: velocity Verlet on the pair-averaged force of Eq. 1's last
 *    term, -1/2 (F_a + F_b) d/dP, with the momentum left unchanged at a
 *    transition (Sec. II A: no momentum jump);
 *  - phase: trapezoid rule for the -i w_ab rho_ab term;
 *  - transitions: the coupling term of Eq. 1 realised by one importance-sampled
 *    branch per step with weight correction (Sec. II B: fixed walker count);
 *  - random numbers: Philox4x32-10 keyed by (seed) with counter
 *    (c0, traj_lo, traj_hi, purpose).
 */
#include "qcl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define DEG_TOL 1e-12       /* |e_b - e_a| below this: coupling set to 0, counted */
#define P24 16777216.0      /* 2^24: probability quantum for branch decisions */

/* ---------------------------------------------------------------- Philox -- */
/* Philox4x32-10, Salmon et al., SC'11: ten rounds of two 32x32->64 products
 * with the Weyl key schedule between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

static void draw(uint64_t seed, uint32_t c0, uint64_t traj, uint32_t purpose, uint32_t w[4]) {
  uint32_t ctr[4] = {c0, (uint32_t)traj, (uint32_t)(traj >> 32), purpose};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, w);
}

/* Uniform on (0, 1) from one 32-bit word. */
static double u01(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

/* --------------------------------------------------------- linear algebra -- */
void orc_jacobi_eigh(int32_t n, const double* Ain, double* w, double* V) {
  double A[ORC_MAX_NS * ORC_MAX_NS];
  memcpy(A, Ain, sizeof(double) * (size_t)(n * n));
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) V[i * n + k] = (i == k) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off <= 1e-34 * fro) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        /* Golub & Van Loan, symmetric Schur decomposition of the (p,q) block */
        double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        for (int k = 0; k < n; ++k) { /* A <- A J */
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* A <- J^T A */
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) { /* V <- V J */
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  /* ascending order, stable insertion sort of (w, columns of V) */
  for (int i = 1; i < n; ++i) {
    for (int j = i; j > 0 && w[j] < w[j - 1]; --j) {
      double tw = w[j];
      w[j] = w[j - 1];
      w[j - 1] = tw;
      for (int k = 0; k < n; ++k) {
        double tv = V[k * n + j];
        V[k * n + j] = V[k * n + j - 1];
        V[k * n + j - 1] = tv;
      }
    }
  }
}

/* W(R) = E + sum_j R_j K_j: the state-dependent part of the potential. */
static void elec_matrix(const orc_model* md, const double* R, double* W) {
  int ns = md->n_states, nn = ns * ns;
  for (int k = 0; k < nn; ++k) W[k] = md->E[k];
  for (int j = 0; j < md->n_modes; ++j)
    for (int k = 0; k < nn; ++k) W[k] += R[j] * md->K[(size_t)j * nn + k];
}

int32_t orc_adiabatic(const orc_model* md, const double* R, const double* U_ref, double* e,
                      double* U) {
  int ns = md->n_states;
  double W[ORC_MAX_NS * ORC_MAX_NS];
  elec_matrix(md, R, W);
  if (ns == 2) {
    /* W = s 1 + a sigma_z + b sigma_x,  e = s -/+ r,  theta = atan2(b, a)/2,
     * lower u0 = (-sin, cos), upper u1 = (cos, sin). */
    double s = 0.5 * (W[0] + W[3]), a = 0.5 * (W[0] - W[3]), b = W[1];
    double r = sqrt(a * a + b * b);
    double th = 0.5 * atan2(b, a);
    double c = cos(th), sn = sin(th);
    e[0] = s - r;
    e[1] = s + r;
    U[0] = -sn; /* U[i*2 + alpha] = (u_alpha)_i */
    U[2] = c;
    U[1] = c;
    U[3] = sn;
    return (2.0 * r < DEG_TOL) ? 1 : 0;
  }
  orc_jacobi_eigh(ns, W, e, U);
  for (int al = 0; al < ns; ++al) {
    double sgn;
    if (U_ref) {
      double dot = 0.0;
      for (int i = 0; i < ns; ++i) dot += U[i * ns + al] * U_ref[i * ns + al];
      sgn = (dot < 0.0) ? -1.0 : 1.0;
    } else {
      int imax = 0;
      for (int i = 1; i < ns; ++i)
        if (fabs(U[i * ns + al]) > fabs(U[imax * ns + al])) imax = i;
      sgn = (U[imax * ns + al] < 0.0) ? -1.0 : 1.0;
    }
    if (sgn < 0.0)
      for (int i = 0; i < ns; ++i) U[i * ns + al] = -U[i * ns + al];
  }
  int deg = 0;
  for (int al = 0; al + 1 < ns; ++al)
    if (e[al + 1] - e[al] < DEG_TOL) deg = 1;
  return deg;
}

/* (U^T K_j U)[mu][nu] */
static double rotated(const orc_model* md, int j, const double* U, int mu, int nu) {
  int ns = md->n_states;
  const double* Kj = md->K + (size_t)j * ns * ns;
  double acc = 0.0;
  for (int k = 0; k < ns; ++k)
    for (int l = 0; l < ns; ++l) acc += U[k * ns + mu] * Kj[k * ns + l] * U[l * ns + nu];
  return acc;
}

/* d_{mu nu, j} = <mu| dW/dR_j |nu> / (e_nu - e_mu)  (Hellmann-Feynman form of the
 * first-order nonadiabatic coupling of Eq. 1); dW/dR_j = K_j for this model. */
static double nac1(const orc_model* md, const double* e, const double* U, int mu, int nu, int j,
                   int* deg) {
  if (mu == nu) return 0.0;
  double gap = e[nu] - e[mu];
  if (fabs(gap) < DEG_TOL) {
    if (deg) *deg = 1;
    return 0.0;
  }
  return rotated(md, j, U, mu, nu) / gap;
}

void orc_nac(const orc_model* md, const double* e, const double* U, double* d) {
  int ns = md->n_states, n = md->n_modes;
  for (int mu = 0; mu < ns; ++mu)
    for (int nu = 0; nu < ns; ++nu)
      for (int j = 0; j < n; ++j) d[((size_t)mu * ns + nu) * n + j] = nac1(md, e, U, mu, nu, j, 0);
}

void orc_mean_force(const orc_model* md, const double* R, const double* U, int32_t a, int32_t b,
                    double* F) {
  for (int j = 0; j < md->n_modes; ++j) {
    double k = md->mass[j] * md->omega[j] * md->omega[j];
    /* Hellmann-Feynman: dE_a/dR_j = (U^T K_j U)_aa */
    F[j] = -k * R[j] - 0.5 * (rotated(md, j, U, a, a) + rotated(md, j, U, b, b));
  }
}

/* Events of the coupling term of Eq. 1, in the fixed order (first index,
 * target ascending), then (second index, target ascending):
 *   rho_ab receives -(P/M) d_{a g} rho_gb  => walker (g,b) -> (a',b) with
 *     amplitude A = -dt sum_j (P_j/M_j) d_{a' g, j}
 *   rho_ab receives +(P/M) rho_ag d_{g b}  => walker (a,g) -> (a,b') with
 *     amplitude A = +dt sum_j (P_j/M_j) d_{g b', j}
 * Probabilities p_e = min(kappa |A_e|, p_max) are quantised to 24-bit integer
 * thresholds T_e = floor(p_e 2^24); when their sum exceeds Tmax = floor(p_max
 * 2^24) they are scaled down together, T_e <- floor(T_e Tmax / sum T). */
static int32_t events_impl(const orc_model* md, const double* P, const double* e, const double* U,
                           int32_t a, int32_t b, double dt, int32_t* ta, int32_t* tb, double* A,
                           uint32_t* T, int* deg) {
  int ns = md->n_states, n = md->n_modes, ne = 0;
  double p[2 * ORC_MAX_NS];
  for (int slot = 0; slot < 2; ++slot) {
    for (int nu = 0; nu < ns; ++nu) {
      if (slot == 0 && nu == a) continue;
      if (slot == 1 && nu == b) continue;
      double acc = 0.0;
      for (int j = 0; j < n; ++j) {
        double dj = (slot == 0) ? nac1(md, e, U, nu, a, j, deg) : nac1(md, e, U, b, nu, j, deg);
        acc += (P[j] / md->mass[j]) * dj;
      }
      A[ne] = (slot == 0) ? -dt * acc : dt * acc;
      ta[ne] = (slot == 0) ? nu : a;
      tb[ne] = (slot == 0) ? b : nu;
      ++ne;
    }
  }
  /* quantise first, then scale the integer thresholds down proportionally:
   * floor(T_e Tmax / sum T) is exact, so equal events stay exactly equal */
  uint64_t sumT = 0;
  const uint64_t Tmax = (uint64_t)floor(md->p_max * P24);
  for (int k = 0; k < ne; ++k) {
    p[k] = md->hop_scale * fabs(A[k]);
    if (p[k] > md->p_max) p[k] = md->p_max;
    T[k] = (uint32_t)floor(p[k] * P24);
    sumT += T[k];
  }
  if (sumT > Tmax)
    for (int k = 0; k < ne; ++k) T[k] = (uint32_t)(((uint64_t)T[k] * Tmax) / sumT);
  return ne;
}

int32_t orc_events(const orc_model* md, const double* P, const double* e, const double* U,
                   int32_t a, int32_t b, double dt, int32_t* tgt_a, int32_t* tgt_b, double* A,
                   uint32_t* T) {
  return events_impl(md, P, e, U, a, b, dt, tgt_a, tgt_b, A, T, 0);
}

/* ----------------------------------------------------------- propagation -- */
/* Velocity Verlet on the mean force of pair (a,b) (characteristics of the last
 * two terms of Eq. 1) and the trapezoid rule for the phase term -i w_ab rho_ab,
 * hbar w_ab = e_a - e_b.  Decomposition at the end point is left in (e1, U1). */
static int det_step(const orc_model* md, double* R, double* P, double* phi, int a, int b,
                    const double* Uin, double dt, double* e1, double* U1) {
  int n = md->n_modes, ns = md->n_states;
  double e0[ORC_MAX_NS], U0[ORC_MAX_NS * ORC_MAX_NS], F[ORC_MAX_N];
  int deg = orc_adiabatic(md, R, (ns > 2) ? Uin : 0, e0, U0);
  orc_mean_force(md, R, U0, a, b, F);
  for (int j = 0; j < n; ++j) P[j] += 0.5 * dt * F[j];
  for (int j = 0; j < n; ++j) R[j] += dt * P[j] / md->mass[j];
  deg |= orc_adiabatic(md, R, (ns > 2) ? U0 : 0, e1, U1);
  orc_mean_force(md, R, U1, a, b, F);
  for (int j = 0; j < n; ++j) P[j] += 0.5 * dt * F[j];
  double w0 = (e0[a] - e0[b]) / md->hbar;
  double w1 = (e1[a] - e1[b]) / md->hbar;
  *phi += 0.5 * dt * (w0 + w1);
  return deg;
}

/* Diabatic representation: mean force of pair (a, b) from the diagonal of W,
 * F_j = -k_j R_j - 1/2 (K_j,aa + K_j,bb). */
static void dia_force(const orc_model* md, const double* R, int a, int b, double* F) {
  int ns = md->n_states, nn = ns * ns;
  for (int j = 0; j < md->n_modes; ++j) {
    double k = md->mass[j] * md->omega[j] * md->omega[j];
    const double* Kj = md->K + (size_t)j * nn;
    F[j] = -k * R[j] - 0.5 * (Kj[a * ns + a] + Kj[b * ns + b]);
  }
}

/* Diabatic deterministic step: velocity Verlet on the diagonal mean force and
 * the trapezoid rule for the phase term, hbar w_ab = V_aa(R) - V_bb(R). */
static void det_step_dia(const orc_model* md, double* R, double* P, double* phi, int a, int b,
                         double dt) {
  int n = md->n_modes, ns = md->n_states;
  double W0[ORC_MAX_NS * ORC_MAX_NS], W1[ORC_MAX_NS * ORC_MAX_NS], F[ORC_MAX_N];
  elec_matrix(md, R, W0);
  dia_force(md, R, a, b, F);
  for (int j = 0; j < n; ++j) P[j] += 0.5 * dt * F[j];
  for (int j = 0; j < n; ++j) R[j] += dt * P[j] / md->mass[j];
  elec_matrix(md, R, W1);
  dia_force(md, R, a, b, F);
  for (int j = 0; j < n; ++j) P[j] += 0.5 * dt * F[j];
  double w0 = (W0[a * ns + a] - W0[b * ns + b]) / md->hbar;
  double w1 = (W1[a * ns + a] - W1[b * ns + b]) / md->hbar;
  *phi += 0.5 * dt * (w0 + w1);
}

void orc_step_deterministic(const orc_model* md, double* R, double* P, double* phi, int32_t a,
                            int32_t b, double* U, double dt) {
  int ns = md->n_states;
  if (md->repr == ORC_REPR_DIABATIC) {
    det_step_dia(md, R, P, phi, a, b, dt);
    return;
  }
  double e1[ORC_MAX_NS], U1[ORC_MAX_NS * ORC_MAX_NS];
  det_step(md, R, P, phi, a, b, U, dt, e1, U1);
  if (ns > 2 && U) memcpy(U, U1, sizeof(double) * (size_t)(ns * ns));
}

/* Diabatic events (the coupling terms of the diabatic equation above):
 *   rho_gb receives -(i/hbar) V_ga rho_ab  => walker (a,b) -> (g,b), amplitude
 *     -i c with c = V_ga dt/hbar (three quarter turns)
 *   rho_ag receives +(i/hbar) rho_ab V_bg  => walker (a,b) -> (a,g), amplitude
 *     +i c with c = V_bg dt/hbar (one quarter turn)
 * with W at the end point R_{n+1}; |A_e| = |c_e|, and the probabilities are
 * quantised and scaled exactly as in the adiabatic representation. */
int32_t orc_events_dia(const orc_model* md, const double* R, int32_t a, int32_t b, double dt,
                       int32_t* ta, int32_t* tb, double* c, int32_t* dq, uint32_t* T) {
  int ns = md->n_states, ne = 0;
  double W[ORC_MAX_NS * ORC_MAX_NS];
  elec_matrix(md, R, W);
  for (int slot = 0; slot < 2; ++slot) {
    for (int g = 0; g < ns; ++g) {
      if (slot == 0 && g == a) continue;
      if (slot == 1 && g == b) continue;
      c[ne] = ((slot == 0) ? W[g * ns + a] : W[b * ns + g]) * dt / md->hbar;
      dq[ne] = (slot == 0) ? 3 : 1;
      ta[ne] = (slot == 0) ? g : a;
      tb[ne] = (slot == 0) ? b : g;
      ++ne;
    }
  }
  uint64_t sumT = 0;
  const uint64_t Tmax = (uint64_t)floor(md->p_max * P24);
  for (int k = 0; k < ne; ++k) {
    double p = md->hop_scale * fabs(c[k]);
    if (p > md->p_max) p = md->p_max;
    T[k] = (uint32_t)floor(p * P24);
    sumT += T[k];
  }
  if (sumT > Tmax)
    for (int k = 0; k < ne; ++k) T[k] = (uint32_t)(((uint64_t)T[k] * Tmax) / sumT);
  return ne;
}

/* One full step n -> n+1 of one walker: deterministic part, then one
 * stochastic transition decided by Philox word (n & 3) of block n >> 2.  The
 * walker hops to event e with weight m A_e / p_hat_e, or stays with weight
 * m / (1 - sum p_hat); the momentum is never changed by a hop. */
static void full_step_dia(const orc_model* md, uint64_t seed, uint64_t traj, double* R,
                          double* P, double* m, double* phi, int32_t* a, int32_t* b, int32_t* q,
                          int64_t step, double dt) {
  det_step_dia(md, R, P, phi, *a, *b, dt);
  int32_t ta[2 * ORC_MAX_NS], tb[2 * ORC_MAX_NS], dq[2 * ORC_MAX_NS];
  double c[2 * ORC_MAX_NS];
  uint32_t T[2 * ORC_MAX_NS];
  int ne = orc_events_dia(md, R, *a, *b, dt, ta, tb, c, dq, T);
  uint32_t w[4];
  draw(seed, (uint32_t)(step >> 2), traj, ORC_PURPOSE_HOP, w);
  uint32_t y = w[step & 3] >> 8;
  uint64_t cum = 0, tot = 0;
  for (int k = 0; k < ne; ++k) tot += T[k];
  for (int k = 0; k < ne; ++k) {
    cum += T[k];
    if ((uint64_t)y < cum) {
      double phat = (double)T[k] / P24;
      *m = *m * c[k] / phat;
      *q = (*q + dq[k]) & 3;
      *a = ta[k];
      *b = tb[k];
      return;
    }
  }
  *m = *m / (1.0 - (double)tot / P24);
}

static void full_step(const orc_model* md, uint64_t seed, uint64_t traj, double* R, double* P,
                      double* m, double* phi, int32_t* a, int32_t* b, double* U, int32_t* q,
                      int64_t step, double dt, int64_t* n_deg) {
  int ns = md->n_states;
  if (md->repr == ORC_REPR_DIABATIC) {
    full_step_dia(md, seed, traj, R, P, m, phi, a, b, q, step, dt);
    return;
  }
  double e1[ORC_MAX_NS], U1[ORC_MAX_NS * ORC_MAX_NS];
  int deg = det_step(md, R, P, phi, *a, *b, U, dt, e1, U1);
  if (ns > 2 && U) memcpy(U, U1, sizeof(double) * (size_t)(ns * ns));
  int32_t ta[2 * ORC_MAX_NS], tb[2 * ORC_MAX_NS];
  double A[2 * ORC_MAX_NS];
  uint32_t T[2 * ORC_MAX_NS];
  int edeg = 0;
  int ne = events_impl(md, P, e1, U1, *a, *b, dt, ta, tb, A, T, &edeg);
  if ((deg || edeg) && n_deg) *n_deg += 1;
  uint32_t w[4];
  draw(seed, (uint32_t)(step >> 2), traj, ORC_PURPOSE_HOP, w);
  uint32_t y = w[step & 3] >> 8;
  uint64_t cum = 0, tot = 0;
  for (int k = 0; k < ne; ++k) tot += T[k];
  for (int k = 0; k < ne; ++k) {
    cum += T[k];
    if ((uint64_t)y < cum) {
      double phat = (double)T[k] / P24;
      *m = *m * A[k] / phat;
      *a = ta[k];
      *b = tb[k];
      return;
    }
  }
  *m = *m / (1.0 - (double)tot / P24);
}

int32_t orc_advance(const orc_model* md, uint64_t seed, uint64_t traj_offset, int64_t n_traj,
                    double* R, double* P, double* m, double* phi, int32_t* alpha, int32_t* beta,
                    double* U, int32_t* qturn, int64_t step0, int64_t n_steps, double dt,
                    int64_t* n_deg) {
  int n = md->n_modes, nn = md->n_states * md->n_states;
  if (md->repr == ORC_REPR_DIABATIC && !qturn) return -1;
  for (int64_t i = 0; i < n_traj; ++i) {
    double* Ui = (md->n_states > 2) ? U + (size_t)i * nn : 0;
    int32_t* qi = qturn ? qturn + i : 0;
    for (int64_t s = step0; s < step0 + n_steps; ++s)
      full_step(md, seed, traj_offset + (uint64_t)i, R + (size_t)i * n, P + (size_t)i * n, m + i,
                phi + i, alpha + i, beta + i, Ui, qi, s, dt, n_deg);
  }
  return 0;
}

/* -------------------------------------------------------------- sampling -- */
/* Initial walkers.  (R, P): independent Gaussians per harmonic mode, the Wigner
 * function of the thermal (or ground) state,
 *   var R = hbar/(2 M w) coth(beta hbar w / 2),  var P = hbar M w/2 coth(...),
 * drawn by Box-Muller from Philox block (c0 = j, purpose INIT).  Index pair:
 * rho_ad = U^T rho_el0 U at the walker's own R; the pair (a,b) is drawn from
 * |rho_ad_ab| / sum |rho_ad| (row-major walk, probabilities quantised to 2^-24,
 * the remainder given to the last nonzero pair) with word 0 of block
 * (c0 = N, purpose INIT), and m0 = rho_ad_ab / p_hat_ab, phi0 = 0.  In the
 * diabatic representation the pair is drawn the same way from rho_el0 itself,
 * and q0 = 0. */
int32_t orc_sample(const orc_model* md, const orc_init* in, uint64_t seed, uint64_t traj_offset,
                   int64_t n_traj, double* R, double* P, double* m, double* phi, int32_t* alpha,
                   int32_t* beta, double* U, int32_t* qturn) {
  int n = md->n_modes, ns = md->n_states, nn = ns * ns;
  for (int64_t i = 0; i < n_traj; ++i) {
    uint64_t traj = traj_offset + (uint64_t)i;
    double* Ri = R + (size_t)i * n;
    double* Pi = P + (size_t)i * n;
    for (int j = 0; j < n; ++j) {
      if (!in->wigner) {
        Ri[j] = in->R0[j];
        Pi[j] = in->P0[j];
        continue;
      }
      double M = md->mass[j], w = md->omega[j], hb = md->hbar;
      double cth = isinf(in->beta) ? 1.0 : 1.0 / tanh(0.5 * in->beta * hb * w);
      double sR = sqrt(hb / (2.0 * M * w) * cth);
      double sP = sqrt(0.5 * hb * M * w * cth);
      uint32_t wd[4];
      draw(seed, (uint32_t)j, traj, ORC_PURPOSE_INIT, wd);
      double rad = sqrt(-2.0 * log(u01(wd[0])));
      double ang = 2.0 * M_PI * u01(wd[1]);
      Ri[j] = in->R0[j] + sR * rad * cos(ang);
      Pi[j] = in->P0[j] + sP * rad * sin(ang);
    }
    double e[ORC_MAX_NS], Ua[ORC_MAX_NS * ORC_MAX_NS], rad_[ORC_MAX_NS * ORC_MAX_NS];
    orc_adiabatic(md, Ri, 0, e, Ua);
    double tot = 0.0;
    for (int al = 0; al < ns; ++al)
      for (int be = 0; be < ns; ++be) {
        double acc = 0.0;
        if (md->repr == ORC_REPR_DIABATIC) {
          acc = in->rho_el0[al * ns + be]; /* pairs of the diabatic basis itself */
        } else {
          for (int k = 0; k < ns; ++k)
            for (int l = 0; l < ns; ++l)
              acc += Ua[k * ns + al] * in->rho_el0[k * ns + l] * Ua[l * ns + be];
        }
        rad_[al * ns + be] = acc;
        tot += fabs(acc);
      }
    if (!(tot > 0.0)) return -1;
    uint32_t T[ORC_MAX_NS * ORC_MAX_NS];
    uint64_t sumT = 0;
    int last = -1;
    for (int k = 0; k < nn; ++k) {
      T[k] = (uint32_t)floor(fabs(rad_[k]) / tot * P24);
      sumT += T[k];
      if (rad_[k] != 0.0) last = k;
    }
    T[last] += (uint32_t)(16777216u - sumT);
    uint32_t wd[4];
    draw(seed, (uint32_t)n, traj, ORC_PURPOSE_INIT, wd);
    uint32_t y = wd[0] >> 8;
    uint64_t cum = 0;
    int pick = last;
    for (int k = 0; k < nn; ++k) {
      cum += T[k];
      if ((uint64_t)y < cum) {
        pick = k;
        break;
      }
    }
    alpha[i] = pick / ns;
    beta[i] = pick % ns;
    m[i] = rad_[pick] / ((double)T[pick] / P24);
    phi[i] = 0.0;
    if (qturn) qturn[i] = 0;
    if (ns > 2) memcpy(U + (size_t)i * nn, Ua, sizeof(double) * (size_t)nn);
  }
  return 0;
}

/* ----------------------------------------------------------- observables -- */
/* Walker contribution to the diabatic density matrix
 *   rho_ij = (1/N) sum m exp(-i phi) U_ia(R) U_jb(R)
 * and to the adiabatic one, rho_ab = (1/N) sum m exp(-i phi) [walker at (a,b)];
 * the adiabatic excited-state population P_ad of Figs. 1-4 is its top diagonal
 * element. */
void orc_contrib(const orc_model* md, int64_t n_traj, const double* R, const double* m,
                 const double* phi, const int32_t* alpha, const int32_t* beta, const double* U,
                 const int32_t* qturn, double* q) {
  int ns = md->n_states, nn = ns * ns, n = md->n_modes, nq = 4 * nn;
  int dia = md->repr == ORC_REPR_DIABATIC;
  for (int64_t i = 0; i < n_traj; ++i) {
    double e[ORC_MAX_NS], Uw[ORC_MAX_NS * ORC_MAX_NS];
    const double* Ui;
    if (ns > 2 && !dia) {
      Ui = U + (size_t)i * nn;
    } else {
      orc_adiabatic(md, R + (size_t)i * n, 0, e, Uw);
      Ui = Uw;
    }
    /* z = m exp(-i phi) i^q */
    double xr = m[i] * cos(phi[i]);
    double xi = -m[i] * sin(phi[i]);
    int qq = qturn ? (qturn[i] & 3) : 0;
    double zr = (qq == 0) ? xr : (qq == 1) ? -xi : (qq == 2) ? -xr : xi;
    double zi = (qq == 0) ? xi : (qq == 1) ? xr : (qq == 2) ? -xi : -xr;
    double* qi = q + (size_t)i * nq;
    for (int k = 0; k < nq; ++k) qi[k] = 0.0;
    int a = alpha[i], b = beta[i];
    /* "own" block: the representation the pair lives in; "other": rotated */
    int own = dia ? 0 : 2 * nn, other = dia ? 2 * nn : 0;
    for (int ii = 0; ii < ns; ++ii)
      for (int jj = 0; jj < ns; ++jj) {
        /* adiabatic pair: U_ia U_jb; diabatic pair: U_ai U_bj */
        double f = dia ? Ui[a * ns + ii] * Ui[b * ns + jj] : Ui[ii * ns + a] * Ui[jj * ns + b];
        qi[other + 2 * (ii * ns + jj)] = zr * f;
        qi[other + 2 * (ii * ns + jj) + 1] = zi * f;
      }
    qi[own + 2 * (a * ns + b)] = zr;
    qi[own + 2 * (a * ns + b) + 1] = zi;
  }
}

/* Pairwise summation over a power-of-two tree (zero-padded). */
static double pairwise(const double* x, int64_t stride, int64_t lo, int64_t size, int64_t n,
                       int square) {
  if (lo >= n) return 0.0;
  if (size == 1) {
    double v = x[lo * stride];
    return square ? v * v : v;
  }
  int64_t h = size / 2;
  return pairwise(x, stride, lo, h, n, square) + pairwise(x, stride, lo + h, h, n, square);
}

void orc_observe(const orc_model* md, int64_t n_traj, const double* R, const double* m,
                 const double* phi, const int32_t* alpha, const int32_t* beta, const double* U,
                 const int32_t* qturn, double* row) {
  int nq = 4 * md->n_states * md->n_states;
  double* q = (double*)malloc(sizeof(double) * (size_t)(n_traj > 0 ? n_traj : 1) * nq);
  orc_contrib(md, n_traj, R, m, phi, alpha, beta, U, qturn, q);
  int64_t size = 1;
  while (size < n_traj) size *= 2;
  for (int k = 0; k < nq; ++k) {
    row[k] = (n_traj > 0) ? pairwise(q + k, nq, 0, size, n_traj, 0) : 0.0;
    row[nq + k] = (n_traj > 0) ? pairwise(q + k, nq, 0, size, n_traj, 1) : 0.0;
  }
  free(q);
}

int32_t orc_run(const orc_model* md, const orc_init* in, uint64_t seed, uint64_t traj_offset,
                int64_t n_traj, double dt, int64_t n_steps, int64_t out_stride, double* rows,
                int64_t* n_deg) {
  int n = md->n_modes, ns = md->n_states, nn = ns * ns, nrow = 8 * nn;
  size_t nt = (size_t)(n_traj > 0 ? n_traj : 1);
  double* R = (double*)malloc(sizeof(double) * nt * n);
  double* P = (double*)malloc(sizeof(double) * nt * n);
  double* m = (double*)malloc(sizeof(double) * nt);
  double* phi = (double*)malloc(sizeof(double) * nt);
  int32_t* al = (int32_t*)malloc(sizeof(int32_t) * nt);
  int32_t* be = (int32_t*)malloc(sizeof(int32_t) * nt);
  double* U = (double*)malloc(sizeof(double) * nt * nn);
  int32_t* qt = (int32_t*)malloc(sizeof(int32_t) * nt);
  int32_t rc = orc_sample(md, in, seed, traj_offset, n_traj, R, P, m, phi, al, be, U, qt);
  if (rc == 0) {
    orc_observe(md, n_traj, R, m, phi, al, be, U, qt, rows);
    for (int64_t s = 0; s < n_steps; ++s) {
      for (int64_t i = 0; i < n_traj; ++i)
        full_step(md, seed, traj_offset + (uint64_t)i, R + (size_t)i * n, P + (size_t)i * n,
                  m + i, phi + i, al + i, be + i, (ns > 2) ? U + (size_t)i * nn : 0, qt + i, s,
                  dt, n_deg);
      if ((s + 1) % out_stride == 0)
        orc_observe(md, n_traj, R, m, phi, al, be, U, qt,
                    rows + (size_t)((s + 1) / out_stride) * nrow);
    }
  }
  free(R);
  free(P);
  free(m);
  free(phi);
  free(al);
  free(be);
  free(U);
  free(qt);
  return rc;
}

/* ------------------------------------------------------------- spawning -- */
static uint64_t child_id(uint64_t seed, int64_t step, uint64_t parent) {
  uint32_t w[4];
  draw(seed, (uint32_t)step, parent, ORC_PURPOSE_SPAWN, w);
  return (((uint64_t)w[1] << 32) | w[0]) | (1ull << 63);
}

int32_t orc_spawn_sample(const orc_model* md, const orc_init* in, uint64_t seed,
                         uint64_t traj_offset, int64_t n0, double* R, double* P, double* m,
                         double* phi, int32_t* alpha, int32_t* beta, double* U, int32_t* qturn,
                         uint64_t* id, int64_t* family) {
  int32_t rc = orc_sample(md, in, seed, traj_offset, n0, R, P, m, phi, alpha, beta, U, qturn);
  for (int64_t i = 0; i < n0; ++i) {
    id[i] = traj_offset + (uint64_t)i;
    family[i] = i;
  }
  return rc;
}

/* One walker's step under spawning: the deterministic part, then the same
 * transition test as full_step.  Returns 1 and fills the child's pair, weight
 * and quarter turns when the test fires. */
static int spawn_walker_step(const orc_model* md, uint64_t seed, uint64_t traj, double* R,
                             double* P, double* m, double* phi, int32_t a, int32_t b, double* U,
                             int32_t q, int64_t step, double dt, int32_t* ca, int32_t* cb,
                             double* cm, int32_t* cq) {
  int ns = md->n_states;
  int32_t ta[2 * ORC_MAX_NS], tb[2 * ORC_MAX_NS], dq[2 * ORC_MAX_NS];
  double A[2 * ORC_MAX_NS];
  uint32_t T[2 * ORC_MAX_NS];
  int ne;
  if (md->repr == ORC_REPR_DIABATIC) {
    det_step_dia(md, R, P, phi, a, b, dt);
    ne = orc_events_dia(md, R, a, b, dt, ta, tb, A, dq, T);
  } else {
    double e1[ORC_MAX_NS], U1[ORC_MAX_NS * ORC_MAX_NS];
    det_step(md, R, P, phi, a, b, U, dt, e1, U1);
    if (ns > 2 && U) memcpy(U, U1, sizeof(double) * (size_t)(ns * ns));
    ne = events_impl(md, P, e1, U1, a, b, dt, ta, tb, A, T, 0);
    for (int k = 0; k < ne; ++k) dq[k] = 0;
  }
  uint32_t w[4];
  draw(seed, (uint32_t)(step >> 2), traj, ORC_PURPOSE_HOP, w);
  uint32_t y = w[step & 3] >> 8;
  uint64_t cum = 0;
  for (int k = 0; k < ne; ++k) {
    cum += T[k];
    if ((uint64_t)y < cum) {
      *ca = ta[k];
      *cb = tb[k];
      *cm = *m * A[k] / ((double)T[k] / P24);
      *cq = (q + dq[k]) & 3;
      return 1;
    }
  }
  return 0;
}

int32_t orc_spawn_advance(const orc_model* md, uint64_t seed, int64_t capacity, int64_t* n_live,
                          double* R, double* P, double* m, double* phi, int32_t* alpha,
                          int32_t* beta, double* U, int32_t* qturn, uint64_t* id,
                          int64_t* family, int64_t step0, int64_t n_steps, double dt) {
  int n = md->n_modes, ns = md->n_states, nn = ns * ns;
  for (int64_t s = step0; s < step0 + n_steps; ++s) {
    int64_t nl = *n_live;
    /* step every live walker; children go to scratch, in parent order */
    int32_t* hit = (int32_t*)calloc((size_t)(nl > 0 ? nl : 1), sizeof(int32_t));
    int32_t* ca = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    int32_t* cb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    int32_t* cq = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    double* cm = (double*)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    /* keep the pre-step ensemble in case the step overflows */
    double* keep = (double*)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1) * (2 * n + 2 + nn));
    int64_t n_child = 0;
    for (int64_t i = 0; i < nl; ++i) {
      double* k = keep + (size_t)i * (2 * n + 2 + nn);
      memcpy(k, R + (size_t)i * n, sizeof(double) * n);
      memcpy(k + n, P + (size_t)i * n, sizeof(double) * n);
      k[2 * n] = m[i];
      k[2 * n + 1] = phi[i];
      memcpy(k + 2 * n + 2, U + (size_t)i * nn, sizeof(double) * nn);
      hit[i] = spawn_walker_step(md, seed, id[i], R + (size_t)i * n, P + (size_t)i * n, m + i,
                                 phi + i, alpha[i], beta[i], (ns > 2) ? U + (size_t)i * nn : 0,
                                 qturn[i], s, dt, ca + i, cb + i, cm + i, cq + i);
      n_child += hit[i];
    }
    if (nl + n_child > capacity) {
      for (int64_t i = 0; i < nl; ++i) {
        double* k = keep + (size_t)i * (2 * n + 2 + nn);
        memcpy(R + (size_t)i * n, k, sizeof(double) * n);
        memcpy(P + (size_t)i * n, k + n, sizeof(double) * n);
        m[i] = k[2 * n];
        phi[i] = k[2 * n + 1];
        memcpy(U + (size_t)i * nn, k + 2 * n + 2, sizeof(double) * nn);
      }
      free(hit); free(ca); free(cb); free(cq); free(cm); free(keep);
      return -2;
    }
    /* insert each child right after its parent: walk from the end so that
     * every walker moves to its final place before its old slot is reused */
    int64_t dst = nl + n_child;
    for (int64_t i = nl - 1; i >= 0; --i) {
      if (hit[i]) {
        --dst;
        memcpy(R + (size_t)dst * n, R + (size_t)i * n, sizeof(double) * n);
        memcpy(P + (size_t)dst * n, P + (size_t)i * n, sizeof(double) * n);
        memcpy(U + (size_t)dst * nn, U + (size_t)i * nn, sizeof(double) * nn);
        m[dst] = cm[i];
        phi[dst] = phi[i];
        alpha[dst] = ca[i];
        beta[dst] = cb[i];
        qturn[dst] = cq[i];
        id[dst] = child_id(seed, s, id[i]);
        family[dst] = family[i];
      }
      --dst;
      if (dst != i) {
        memcpy(R + (size_t)dst * n, R + (size_t)i * n, sizeof(double) * n);
        memcpy(P + (size_t)dst * n, P + (size_t)i * n, sizeof(double) * n);
        memcpy(U + (size_t)dst * nn, U + (size_t)i * nn, sizeof(double) * nn);
        m[dst] = m[i];
        phi[dst] = phi[i];
        alpha[dst] = alpha[i];
        beta[dst] = beta[i];
        qturn[dst] = qturn[i];
        id[dst] = id[i];
        family[dst] = family[i];
      }
    }
    *n_live = nl + n_child;
    free(hit); free(ca); free(cb); free(cq); free(cm); free(keep);
  }
  return 0;
}

void orc_spawn_observe(const orc_model* md, int64_t n0, int64_t n_live, const double* R,
                       const double* m, const double* phi, const int32_t* alpha,
                       const int32_t* beta, const double* U, const int32_t* qturn,
                       const int64_t* family, double* row) {
  int ns = md->n_states, nq = 4 * ns * ns;
  double* q = (double*)malloc(sizeof(double) * (size_t)(n_live > 0 ? n_live : 1) * nq);
  double* X = (double*)calloc((size_t)(n0 > 0 ? n0 : 1) * nq, sizeof(double));
  orc_contrib(md, n_live, R, m, phi, alpha, beta, U, qturn, q);
  for (int64_t i = 0; i < n_live; ++i) /* in walker order within each family */
    for (int k = 0; k < nq; ++k) X[(size_t)family[i] * nq + k] += q[(size_t)i * nq + k];
  int64_t size = 1;
  while (size < n0) size *= 2;
  for (int k = 0; k < nq; ++k) {
    row[k] = (n0 > 0) ? pairwise(X + k, nq, 0, size, n0, 0) : 0.0;
    row[nq + k] = (n0 > 0) ? pairwise(X + k, nq, 0, size, n0, 1) : 0.0;
  }
  free(q);
  free(X);
}

int32_t orc_run_spawn(const orc_model* md, const orc_init* in, uint64_t seed, uint64_t traj_offset,
                      int64_t n0, int64_t capacity, double dt, int64_t n_steps, int64_t out_stride,
                      double* rows, int64_t* n_live_out) {
  int n = md->n_modes, ns = md->n_states, nn = ns * ns, nrow = 8 * nn;
  if (capacity < n0) return -2;
  size_t c = (size_t)(capacity > 0 ? capacity : 1);
  double* R = (double*)malloc(sizeof(double) * c * n);
  double* P = (double*)malloc(sizeof(double) * c * n);
  double* m = (double*)malloc(sizeof(double) * c);
  double* phi = (double*)malloc(sizeof(double) * c);
  int32_t* al = (int32_t*)malloc(sizeof(int32_t) * c);
  int32_t* be = (int32_t*)malloc(sizeof(int32_t) * c);
  double* U = (double*)calloc(c * nn, sizeof(double));
  int32_t* qt = (int32_t*)malloc(sizeof(int32_t) * c);
  uint64_t* id = (uint64_t*)malloc(sizeof(uint64_t) * c);
  int64_t* fam = (int64_t*)malloc(sizeof(int64_t) * c);
  int64_t nl = n0;
  int32_t rc = orc_spawn_sample(md, in, seed, traj_offset, n0, R, P, m, phi, al, be, U, qt, id, fam);
  if (rc == 0) {
    orc_spawn_observe(md, n0, nl, R, m, phi, al, be, U, qt, fam, rows);
    if (n_live_out) n_live_out[0] = nl;
    for (int64_t s = 0; s < n_steps && rc == 0; ++s) {
      rc = orc_spawn_advance(md, seed, capacity, &nl, R, P, m, phi, al, be, U, qt, id, fam, s, 1, dt);
      if (rc == 0 && (s + 1) % out_stride == 0) {
        orc_spawn_observe(md, n0, nl, R, m, phi, al, be, U, qt, fam,
                          rows + (size_t)((s + 1) / out_stride) * nrow);
        if (n_live_out) n_live_out[(s + 1) / out_stride] = nl;
      }
    }
  }
  free(R); free(P); free(m); free(phi); free(al); free(be); free(U); free(qt); free(id); free(fam);
  return rc;
}
