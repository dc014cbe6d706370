// nstate.cuh -- adiabatic decomposition and couplings of N_s-state linear
// vibronic-coupling models (N_s = 3..8) for the FP64 and FP32-bulk kernels.
//
// W(R) = E + sum_j R_j K_j is diagonalised by cyclic Jacobi rotations.  Along a
// trajectory the previous eigenvectors U_ref are the starting basis (the
// rotated matrix U_ref^T W U_ref is nearly diagonal), the eigenvalues are
// sorted ascending and each eigenvector's sign is aligned with its reference
// (parallel transport), which makes the couplings d_ab and the products
// U_ia U_jb continuous along the path.  Without a reference (initial sample)
// the largest-magnitude component of each eigenvector is made positive.
#pragma once
#include "lanes.cuh"
#include "qcl_common.cuh"

namespace qcl {

template <typename T>
__device__ __forceinline__ T q_sqrt(T x) {
  return sqrt(x);
}
template <>
__device__ __forceinline__ float q_sqrt<float>(float x) {
  return sqrtf(x);
}

// One Jacobi rotation annihilating A[p][q] of the symmetric matrix A and
// accumulating it into the columns of V (Golub & Van Loan, symmetric Schur).
// A zero A[p][q] gives the identity rotation (c = 1, s = 0 exactly, so every
// update reproduces its input); it is selected rather than branched to, which
// keeps the warp's walkers on one path.
template <typename T, int NS>
__device__ __forceinline__ void jacobi_rotate(T (&A)[NS][NS], T (&V)[NS][NS], int p, int q) {
  const T apq = A[p][q];
  const bool zero = apq == T(0);
  const T tau = (A[q][q] - A[p][p]) / (T(2) * (zero ? T(1) : apq));
  const T tr = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + q_sqrt<T>(T(1) + tau * tau));
  const T t = zero ? T(0) : tr;
  const T c = zero ? T(1) : T(1) / q_sqrt<T>(T(1) + t * t);
  const T s = t * c;
#pragma unroll
  for (int k = 0; k < NS; ++k) {  // A <- A J (columns p, q)
    const T akp = A[k][p], akq = A[k][q];
    A[k][p] = c * akp - s * akq;
    A[k][q] = s * akp + c * akq;
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) {  // A <- J^T A (rows p, q)
    const T apk = A[p][k], aqk = A[q][k];
    A[p][k] = c * apk - s * aqk;
    A[q][k] = s * apk + c * aqk;
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) {  // V <- V J
    const T vkp = V[k][p], vkq = V[k][q];
    V[k][p] = c * vkp - s * vkq;
    V[k][q] = s * vkp + c * vkq;
  }
}

template <typename T, int NS>
__device__ __forceinline__ T offdiag2(const T (&A)[NS][NS]) {
  T off = T(0);
#pragma unroll
  for (int p = 0; p < NS; ++p)
#pragma unroll
    for (int q = p + 1; q < NS; ++q) off += A[p][q] * A[p][q];
  return off;
}

// Diagonalises W into ascending e and eigenvectors U[i][a]; with `ref` the
// signs follow ref, and with `warm` the rotations also start from ref's basis
// (otherwise from W itself).  Sweeps: at most max_sweeps, stopping when the
// off-diagonal mass is below tol2 times the matrix norm (a fixed sweep count
// when tol2 < 0).
template <typename T, int NS>
__device__ __forceinline__ void eigh_ns(const T (&W)[NS][NS], const T (*ref)[NS], T (&e)[NS],
                                        T (&U)[NS][NS], int max_sweeps, T tol2,
                                        bool warm = true) {
  T A[NS][NS], V[NS][NS];
  if (ref && warm) {
    // A = ref^T W ref
    T Wr[NS][NS];
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int b = 0; b < NS; ++b) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NS; ++k) acc += W[i][k] * ref[k][b];
        Wr[i][b] = acc;
      }
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
      for (int b = 0; b < NS; ++b) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NS; ++k) acc += ref[k][a] * Wr[k][b];
        A[a][b] = acc;
      }
    // symmetrise the rotated matrix (rounding)
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
      for (int b = a + 1; b < NS; ++b) {
        const T m = T(0.5) * (A[a][b] + A[b][a]);
        A[a][b] = m;
        A[b][a] = m;
      }
  } else {
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
      for (int b = 0; b < NS; ++b) A[a][b] = W[a][b];
  }
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) V[a][b] = (a == b) ? T(1) : T(0);
  T fro = T(0);
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) fro += A[a][b] * A[a][b];
#pragma unroll 1
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tol2 >= T(0) && offdiag2<T, NS>(A) <= tol2 * fro) break;
#pragma unroll
    for (int p = 0; p < NS; ++p)
#pragma unroll
      for (int q = p + 1; q < NS; ++q) jacobi_rotate<T, NS>(A, V, p, q);
  }
  // eigenvectors in the original basis
  if (ref && warm) {
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int b = 0; b < NS; ++b) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NS; ++k) acc += ref[i][k] * V[k][b];
        U[i][b] = acc;
      }
  } else {
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int b = 0; b < NS; ++b) U[i][b] = V[i][b];
  }
#pragma unroll
  for (int a = 0; a < NS; ++a) e[a] = A[a][a];
  // ascending order (stable insertion sort; fixed compare pattern)
#pragma unroll
  for (int i = 1; i < NS; ++i)
#pragma unroll
    for (int j = i; j > 0; --j) {
      const bool sw = e[j] < e[j - 1];
      const T t0 = e[j], t1 = e[j - 1];
      e[j] = sw ? t1 : t0;
      e[j - 1] = sw ? t0 : t1;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const T u0 = U[k][j], u1 = U[k][j - 1];
        U[k][j] = sw ? u1 : u0;
        U[k][j - 1] = sw ? u0 : u1;
      }
    }
  // gauge: follow the reference, else largest-magnitude component positive
#pragma unroll
  for (int a = 0; a < NS; ++a) {
    bool flip;
    if (ref) {
      T dot = T(0);
#pragma unroll
      for (int i = 0; i < NS; ++i) dot += U[i][a] * ref[i][a];
      flip = dot < T(0);
    } else {
      int imax = 0;
      T vmax = fabs(U[0][a]);
#pragma unroll
      for (int i = 1; i < NS; ++i) {
        const bool g = fabs(U[i][a]) > vmax;
        vmax = g ? fabs(U[i][a]) : vmax;
        imax = g ? i : imax;
      }
      T v = U[0][a];
#pragma unroll
      for (int i = 1; i < NS; ++i) v = (i == imax) ? U[i][a] : v;
      flip = v < T(0);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) U[i][a] = flip ? -U[i][a] : U[i][a];
  }
}

// Warm-started decomposition for the FP32-bulk kernels.  A = ref^T W ref (its
// upper triangle) is nearly diagonal: the previous step's eigenvectors ref
// almost diagonalise W(R_{n+1}).  Two cyclic Jacobi sweeps annihilate the
// off-diagonal elements with the symmetric update (a_pp -= t a_pq,
// a_qq += t a_pq, a_pq = 0, rows r != p, q rotated), and each rotation is
// applied to the columns of U, which starts as ref, so U = ref J_1 J_2 ...
// directly.  Sweep 1 computes t = 2 a_pq / (d + sgn(d) sqrt(d^2 + 4 a_pq^2)),
// d = a_qq - a_pp, c = 1 / sqrt(1 + t^2), s = t c.  After it the angles are
// small: where every walker of the warp has |a_pq| <= 2^-12 |d| for every
// pair, sweep 2 takes the small-angle form t = a_pq / d, c = 1, s = t, which
// equals the full rotation in FP32 (t^2 / 2 <= 2^-25 rounds c to 1, and t
// differs from a_pq / d by a relative t^2); otherwise (a walker near a
// crossing) sweep 2 is a full sweep too.  Then the eigenvalues are sorted
// ascending and each column of U is aligned in sign with its reference column
// (parallel transport).
// (tm: the largest |t| of the sweep's rotations so far, per lane)
template <int NS, bool SMALL, typename V>
__device__ __forceinline__ void jacobi_sweep_warm(V (&A)[NS][NS], V (&U)[NS][NS], V& tm) {
  constexpr bool small = SMALL;
  constexpr int L = Lanes<V>::W;
  auto at = [&](int i, int j) -> V& { return i < j ? A[i][j] : A[j][i]; };
#pragma unroll
  for (int p = 0; p < NS; ++p)
#pragma unroll
    for (int q = p + 1; q < NS; ++q) {
      const V apq = A[p][q];
      const V d = vsub(A[q][q], A[p][p]);
      V t, c, sn;
      if (small) {
#pragma unroll
        for (int l = 0; l < L; ++l) {  // (a zero a_pq gives t = 0, also where d = 0)
          const float q = __fdividef(ln(apq, l), ln(d, l));
          ln(t, l) = ln(apq, l) == 0.0f ? 0.0f : q;
        }
        sn = t;
      } else {
        const V twoa = vmul(splat<V>(2.0f), apq);
        const V r2 = vfma(d, d, vmul(twoa, twoa));
#pragma unroll
        for (int l = 0; l < L; ++l) {
          // d + sgn(d) sqrt(d^2 + 4 a_pq^2) is never 0 unless a_pq = 0 (then t = 0)
          const float rl = ln(r2, l);
          const float den = ln(d, l) + copysignf(rl * rsqrtf(rl), ln(d, l));
          const float q = __fdividef(ln(twoa, l), den);
          ln(t, l) = ln(apq, l) == 0.0f ? 0.0f : q;
        }
        const V tt1 = vfma(t, t, splat<V>(1.0f));
#pragma unroll
        for (int l = 0; l < L; ++l) ln(c, l) = rsqrtf(ln(tt1, l));
        sn = vmul(t, c);
      }
#pragma unroll
      for (int l = 0; l < L; ++l) ln(tm, l) = fmaxf(ln(tm, l), fabsf(ln(t, l)));
      const V nsn = vmul(sn, splat<V>(-1.0f));
      A[p][p] = vfma(t, vmul(apq, splat<V>(-1.0f)), A[p][p]);  // a_pp - t a_pq
      A[q][q] = vfma(t, apq, A[q][q]);
      A[p][q] = splat<V>(0.0f);
#pragma unroll
      for (int r = 0; r < NS; ++r) {
        if (r == p || r == q) continue;
        const V arp = at(r, p), arq = at(r, q);
        if (small) {
          at(r, p) = vfma(nsn, arq, arp);
          at(r, q) = vfma(sn, arp, arq);
        } else {
          at(r, p) = vfma(c, arp, vmul(nsn, arq));
          at(r, q) = vfma(sn, arp, vmul(c, arq));
        }
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const V ukp = U[k][p], ukq = U[k][q];
        if (small) {
          U[k][p] = vfma(nsn, ukq, ukp);
          U[k][q] = vfma(sn, ukp, ukq);
        } else {
          U[k][p] = vfma(c, ukp, vmul(nsn, ukq));
          U[k][q] = vfma(sn, ukp, vmul(c, ukq));
        }
      }
    }
}

template <int NS, typename V>
__device__ __forceinline__ void eigh_warm_fast(const V (&W)[NS][NS], const V (&ref)[NS][NS],
                                               V (&e)[NS], V (&U)[NS][NS]) {
  // V = float (one walker) or float2 (two walkers, one per lane): the FP32
  // arithmetic is the packed lane arithmetic of lanes.cuh (explicit
  // round-to-nearest, so each lane's bits do not depend on the lane count);
  // divisions, square roots, compares and selects run per lane.
  constexpr int L = Lanes<V>::W;
  V A[NS][NS];
  {
    V Wr[NS][NS];
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int b = 0; b < NS; ++b) {
        V acc = splat<V>(0.0f);
#pragma unroll
        for (int k = 0; k < NS; ++k) acc = vfma(W[i][k], ref[k][b], acc);
        Wr[i][b] = acc;
      }
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
      for (int b = a; b < NS; ++b) {
        V acc = splat<V>(0.0f);
#pragma unroll
        for (int k = 0; k < NS; ++k) acc = vfma(ref[k][a], Wr[k][b], acc);
        A[a][b] = acc;  // upper triangle only
      }
  }
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) U[a][b] = ref[a][b];
  // full sweeps (one copy of the code): the first always, the second where
  // some walker of the warp still has a large angle; else the small-angle sweep
  V tm = splat<V>(0.0f);
#pragma unroll 1
  for (int sweep = 0; sweep < 2; ++sweep) {
    if (sweep == 1) {
      bool large = false;
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int p = 0; p < NS; ++p)
#pragma unroll
          for (int q = p + 1; q < NS; ++q)
            large |= !(fabsf(ln(A[p][q], l)) * 4096.0f <= fabsf(ln(A[q][q], l) - ln(A[p][p], l)));
      if (!__any_sync(0xffffffffu, large)) {
        jacobi_sweep_warm<NS, true, V>(A, U, tm);
        break;
      }
    }
    jacobi_sweep_warm<NS, false, V>(A, U, tm);
  }
#pragma unroll
  for (int a = 0; a < NS; ++a) e[a] = A[a][a];
  // ascending order of (e, columns of U) by a fixed compare network.  The warm
  // start keeps the reference's ascending order except where eigenvalues pass
  // each other, and on sorted input the network swaps nothing, so it runs only
  // when some walker of the warp is out of order (the same result either way).
  bool unsorted = false;
#pragma unroll
  for (int l = 0; l < L; ++l)
#pragma unroll
    for (int j = 1; j < NS; ++j) unsorted |= ln(e[j], l) < ln(e[j - 1], l);
  const bool swapped = __any_sync(0xffffffffu, unsorted);
  if (swapped) {
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int i = 1; i < NS; ++i)
#pragma unroll
        for (int j = i; j > 0; --j) {
          const bool sw = ln(e[j], l) < ln(e[j - 1], l);
          const float t0 = ln(e[j], l), t1 = ln(e[j - 1], l);
          ln(e[j], l) = sw ? t1 : t0;
          ln(e[j - 1], l) = sw ? t0 : t1;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            const float u0 = ln(U[k][j], l), u1 = ln(U[k][j - 1], l);
            ln(U[k][j], l) = sw ? u1 : u0;
            ln(U[k][j - 1], l) = sw ? u0 : u1;
          }
        }
  }
  // eigenvector b follows reference column b.  Without a swap in the sort,
  // column b is reference column b turned by the rotations (p, q) with b in
  // {p, q}: at most 2 (N_s - 1) of them, each by |theta| = atan |t|.  While every
  // |t| <= 1/4 that is at most 6 atan(1/4) = 1.47 < pi/2 for N_s <= 4, so the
  // dot product is positive and the signs below would all be +1: the warp skips
  // them.
  bool far = swapped || NS > 4;
#pragma unroll
  for (int l = 0; l < L; ++l) far |= ln(tm, l) > 0.25f;
  if (!__any_sync(0xffffffffu, far)) return;
#pragma unroll
  for (int b = 0; b < NS; ++b) {
    V dot = splat<V>(0.0f);
#pragma unroll
    for (int i = 0; i < NS; ++i) dot = vfma(U[i][b], ref[i][b], dot);
    V sg;
#pragma unroll
    for (int l = 0; l < L; ++l) ln(sg, l) = ln(dot, l) < 0.0f ? -1.0f : 1.0f;
#pragma unroll
    for (int i = 0; i < NS; ++i) U[i][b] = vmul(U[i][b], sg);
  }
}

// Decomposition from the identity for the FP32 observation of diabatic walkers
// (the adiabatic block at the walker's R): the warm kernel's sweeps on W's
// upper triangle with U starting as the identity.  Full sweeps until every
// walker of the warp has |a_pq| <= 2^-12 |d| for every pair (at most eight),
// then one small-angle sweep; eigenvalues ascending, each eigenvector's
// largest-magnitude component positive (the convention of eigh_ns without a
// reference).  Takes warp-wide votes: every lane of the warp calls it.
template <int NS>
__device__ __forceinline__ void eigh_cold_fast(const float (&W)[NS][NS], float (&e)[NS],
                                               float (&U)[NS][NS]) {
  float A[NS][NS];
#pragma unroll
  for (int a = 0; a < NS; ++a)
#pragma unroll
    for (int b = 0; b < NS; ++b) {
      A[a][b] = W[a][b];
      U[a][b] = a == b ? 1.0f : 0.0f;
    }
  float tm = 0.0f;
#pragma unroll 1
  for (int sweep = 0; sweep < 9; ++sweep) {
    bool large = false;
#pragma unroll
    for (int p = 0; p < NS; ++p)
#pragma unroll
      for (int q = p + 1; q < NS; ++q)
        large |= !(fabsf(A[p][q]) * 4096.0f <= fabsf(A[q][q] - A[p][p]));
    if (!__any_sync(0xffffffffu, large)) {
      jacobi_sweep_warm<NS, true, float>(A, U, tm);
      break;
    }
    if (sweep == 8) break;
    jacobi_sweep_warm<NS, false, float>(A, U, tm);
  }
#pragma unroll
  for (int a = 0; a < NS; ++a) e[a] = A[a][a];
#pragma unroll
  for (int i = 1; i < NS; ++i)
#pragma unroll
    for (int j = i; j > 0; --j) {
      const bool sw = e[j] < e[j - 1];
      const float t0 = e[j], t1 = e[j - 1];
      e[j] = sw ? t1 : t0;
      e[j - 1] = sw ? t0 : t1;
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const float u0 = U[k][j], u1 = U[k][j - 1];
        U[k][j] = sw ? u1 : u0;
        U[k][j - 1] = sw ? u0 : u1;
      }
    }
#pragma unroll
  for (int a = 0; a < NS; ++a) {
    float vmax = fabsf(U[0][a]), v = U[0][a];
#pragma unroll
    for (int i = 1; i < NS; ++i) {
      const bool g = fabsf(U[i][a]) > vmax;
      vmax = g ? fabsf(U[i][a]) : vmax;
      v = g ? U[i][a] : v;
    }
    const float sg = v < 0.0f ? -1.0f : 1.0f;
#pragma unroll
    for (int i = 0; i < NS; ++i) U[i][a] *= sg;
  }
}

}  // namespace qcl
