/*
 * qcl_oracle.h -- plain FP64 CPU oracle for momentum-jump-free mixed
 * quantum-classical Liouville (QCL) dynamics.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library: everything here (the Philox generator included) is written
 * out again from its published definition.
 *
 * Method (paper, Sec. II A, Eq. 1): the partially Wigner-transformed density
 * matrix element rho_ab(R,P) obeys
 *   d/dt rho_ab = -i w_ab rho_ab - (P/M) sum_g (d_ag rho_gb - rho_ag d_gb)
 *                 - (P/M) d rho_ab/dR - 1/2 (F_a + F_b) d rho_ab/dP .
 * It is estimated by a fixed ensemble of walkers (Sec. II B: no spawning, the
 * walker count is fixed).  Each walker carries (R, P), an index pair (a, b) and
 * a complex weight m exp(-i phi).  The walker layout in this oracle is
 * walker-major: R[i*N + j].
 */
#ifndef QCL_ORACLE_H
#define QCL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_NS 8
#define ORC_MAX_N 256

/* Philox counter word 3 ("purpose") values.  They are part of the random
 * stream definition that the GPU library follows too. */
#define ORC_PURPOSE_INIT 1u
#define ORC_PURPOSE_HOP 2u
#define ORC_PURPOSE_SPAWN 3u

/* Electronic basis of the walkers' index pairs (orc_model.repr).
 *
 * ADIABATIC (Eq. 1 as printed): pairs of eigenstates of W(R); phase from
 * e_a - e_b, mean force from the Hellmann-Feynman diagonal, transitions from
 * the nonadiabatic coupling d_ab contracted with P/M.
 *
 * DIABATIC (the same equation written in the R-independent basis of W, in
 * which d = 0 and the electronic coupling is the off-diagonal potential):
 *   d/dt rho_ab = -(i/hbar)(V_aa - V_bb) rho_ab
 *                 - (i/hbar) sum_{g != a} V_ag rho_gb + (i/hbar) sum_{g != b} rho_ag V_gb
 *                 - (P/M) d rho_ab/dR - 1/2 (F_a + F_b) d rho_ab/dP,
 * F_a = -dV_aa/dR (the diagonal diabatic force; off-diagonal force terms are
 * dropped as in Eq. 1).  The transition amplitudes are imaginary, -i c or +i c
 * with real c = V dt/hbar, so a walker carries its weight as
 * m exp(-i phi) i^q with an integer count q (mod 4) of quarter turns. */
#define ORC_REPR_ADIABATIC 0
#define ORC_REPR_DIABATIC 1

/* Linear vibronic-coupling model: V(R) = 1/2 sum_j k_j R_j^2 + W(R),
 * W(R) = E + sum_j R_j K_j, with k_j = M_j w_j^2 and E, K_j real symmetric
 * n_states x n_states (row-major).  K is [n_modes][n_states*n_states]. */
typedef struct {
  int32_t n_states;
  int32_t n_modes;
  double hbar;
  const double* mass;
  const double* omega;
  const double* E;
  const double* K;
  double hop_scale; /* kappa: p_e = min(kappa |A_e|, p_max) */
  double p_max;
  int32_t repr;     /* ORC_REPR_ADIABATIC (0) or ORC_REPR_DIABATIC (1) */
  int32_t reserved;
} orc_model;

/* Initial condition: diabatic electronic density rho_el0 (real symmetric),
 * Wigner distribution of harmonic modes centred at (R0, P0) at inverse
 * temperature beta (INFINITY = ground state).  wigner = 0 puts every walker
 * exactly at (R0, P0). */
typedef struct {
  const double* rho_el0;
  const double* R0;
  const double* P0;
  double beta;
  int32_t wigner;
} orc_init;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Symmetric eigen-decomposition by cyclic Jacobi rotations, eigenvalues
 * ascending, eigenvectors in the columns of V (row-major n x n). */
void orc_jacobi_eigh(int32_t n, const double* A, double* w, double* V);

/* Adiabatic energies e[a] (ascending) and eigenvectors U[i*NS + a] of W(R).
 * Two states: closed form theta = atan2(b, a)/2.  More states: Jacobi, with
 * each eigenvector's sign aligned to U_ref (parallel transport) when U_ref is
 * given, else its largest-magnitude component made positive.  Returns 1 if two
 * energies are closer than the degeneracy threshold, else 0. */
int32_t orc_adiabatic(const orc_model* md, const double* R, const double* U_ref, double* e,
                      double* U);

/* Nonadiabatic coupling d[(mu*NS + nu)*N + j] = <mu|d_j nu> (Hellmann-Feynman
 * form) at R, from the decomposition (e, U).  Degenerate pairs give 0. */
void orc_nac(const orc_model* md, const double* e, const double* U, double* d);

/* Mean force of pair (a, b): F_j = -k_j R_j - 1/2 (dE_a/dR_j + dE_b/dR_j). */
void orc_mean_force(const orc_model* md, const double* R, const double* U, int32_t a, int32_t b,
                    double* F);

/* Transition events of walker (a, b) at (R, P) with decomposition (e, U):
 * writes, in the fixed event order, the target pair, amplitude A_e and the
 * quantised probability threshold T_e (p_hat = T_e 2^-24).  Returns the event
 * count 2 (NS - 1). */
int32_t orc_events(const orc_model* md, const double* P, const double* e, const double* U,
                   int32_t a, int32_t b, double dt, int32_t* tgt_a, int32_t* tgt_b, double* A,
                   uint32_t* T);

/* Diabatic transition events of walker (a, b) at R, in the fixed order (first
 * index, target ascending), then (second index, target ascending): target pair,
 * real amplitude factor c_e (V_{g a} dt/hbar, then V_{b g} dt/hbar), quarter
 * turns dq_e of the amplitude (3 for -i, 1 for +i) and the quantised threshold
 * T_e.  Returns the event count 2 (NS - 1). */
int32_t orc_events_dia(const orc_model* md, const double* R, int32_t a, int32_t b, double dt,
                       int32_t* tgt_a, int32_t* tgt_b, double* c, int32_t* dq, uint32_t* T);

/* Deterministic part of one step (velocity Verlet on the pair's mean force and
 * trapezoid phase); U (NS > 2 only, adiabatic only) carries the gauge in and
 * out. */
void orc_step_deterministic(const orc_model* md, double* R, double* P, double* phi, int32_t a,
                            int32_t b, double* U, double dt);

/* Sample n_traj walkers with global ids traj_offset + i.  qturn (may be NULL
 * in the adiabatic representation) receives the quarter-turn counts. */
int32_t orc_sample(const orc_model* md, const orc_init* in, uint64_t seed, uint64_t traj_offset,
                   int64_t n_traj, double* R, double* P, double* m, double* phi, int32_t* alpha,
                   int32_t* beta, double* U, int32_t* qturn);

/* Advance n_traj walkers from absolute step step0 by n_steps.  n_deg (may be
 * NULL) accumulates the count of degenerate-gap events. */
int32_t orc_advance(const orc_model* md, uint64_t seed, uint64_t traj_offset, int64_t n_traj,
                    double* R, double* P, double* m, double* phi, int32_t* alpha, int32_t* beta,
                    double* U, int32_t* qturn, int64_t step0, int64_t n_steps, double dt,
                    int64_t* n_deg);

/* Per-walker observable contributions q[i*4NS^2 + k]:
 *   k = 2(i*NS+j)+c          diabatic rho_ij,  c = 0 real, 1 imaginary
 *   k = 2NS^2 + 2(a*NS+b)+c  adiabatic rho_ab
 * With z = m exp(-i phi) i^q: an adiabatic pair (a, b) adds z U_ia U_jb to
 * rho_ij and z to rho_ab; a diabatic pair (a, b) adds z to rho_ab (diabatic)
 * and z U_ak U_bl to the adiabatic rho_kl, U the eigenvectors at the walker's R
 * (closed form for two states, else Jacobi with the largest-magnitude component
 * of each eigenvector positive). */
void orc_contrib(const orc_model* md, int64_t n_traj, const double* R, const double* m,
                 const double* phi, const int32_t* alpha, const int32_t* beta, const double* U,
                 const int32_t* qturn, double* q);

/* Sum over walkers (pairwise) of each contribution and of its square:
 * row[k] = sum q_k, row[4NS^2 + k] = sum q_k^2. */
void orc_observe(const orc_model* md, int64_t n_traj, const double* R, const double* m,
                 const double* phi, const int32_t* alpha, const int32_t* beta, const double* U,
                 const int32_t* qturn, double* row);

/* Whole run: sample, then n_steps steps with an observation row at every
 * absolute step s = k * out_stride (k = 0 .. n_steps / out_stride). */
int32_t orc_run(const orc_model* md, const orc_init* in, uint64_t seed, uint64_t traj_offset,
                int64_t n_traj, double dt, int64_t n_steps, int64_t out_stride, double* rows,
                int64_t* n_deg);

/* ------------------------------------------------------------- spawning --
 * Trajectory spawning, the scheme of the CPU code that the paper's GPU version
 * replaces (Sec. II B): the transition test of a step (the same Philox word and
 * thresholds as without spawning) does not move the walker; when it fires for
 * event e the walker spawns a child at e's target pair with weight
 * m A_e / p_hat_e (diabatic: m c_e / p_hat_e and q + dq_e) and the same (R, P,
 * phi, U), and the parent keeps its pair and weight -- no 1/(1 - sum p_hat)
 * factor.  The expectation of parent plus child is (1 + dt L) m, as without
 * spawning, but no weight grows by the stay factor; the walker count grows
 * instead.
 *
 * Walker order: each child is inserted right after its parent, so the walkers
 * descending from one initial walker (a family) stay contiguous; family[i] is
 * that initial walker's index.  A child's random stream is keyed by the id
 * made of words 0 and 1 of Philox block (c0 = step, parent id, purpose SPAWN)
 * with bit 63 set (initial walkers: traj_offset + index).  Observables are the
 * sums over families of the family sums X_k and of X_k^2, so the standard error
 * counts the n0 independent families, not the correlated walkers. */

/* Initial spawning ensemble of n0 walkers (arrays of capacity >= n0 walkers). */
int32_t orc_spawn_sample(const orc_model* md, const orc_init* in, uint64_t seed,
                         uint64_t traj_offset, int64_t n0, double* R, double* P, double* m,
                         double* phi, int32_t* alpha, int32_t* beta, double* U, int32_t* qturn,
                         uint64_t* id, int64_t* family);

/* Advances the *n_live walkers by n_steps from absolute step step0.  Returns
 * 0, or -2 if a step would exceed capacity (the ensemble is left at the end of
 * the previous step and *n_live unchanged by that step). */
int32_t orc_spawn_advance(const orc_model* md, uint64_t seed, int64_t capacity, int64_t* n_live,
                          double* R, double* P, double* m, double* phi, int32_t* alpha,
                          int32_t* beta, double* U, int32_t* qturn, uint64_t* id,
                          int64_t* family, int64_t step0, int64_t n_steps, double dt);

/* row[k] = sum over families of X_k, row[4NS^2 + k] = sum of X_k^2 (pairwise
 * over the n0 families), X_k = the family's sum of the contributions of
 * orc_contrib. */
void orc_spawn_observe(const orc_model* md, int64_t n0, int64_t n_live, const double* R,
                       const double* m, const double* phi, const int32_t* alpha,
                       const int32_t* beta, const double* U, const int32_t* qturn,
                       const int64_t* family, double* row);

/* Whole spawning run: rows as orc_run, n_live_out[k] = live walkers at output k.
 * Returns -2 on capacity overflow. */
int32_t orc_run_spawn(const orc_model* md, const orc_init* in, uint64_t seed, uint64_t traj_offset,
                      int64_t n0, int64_t capacity, double dt, int64_t n_steps, int64_t out_stride,
                      double* rows, int64_t* n_live_out);

#ifdef __cplusplus
}
#endif
#endif
