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

// Warm-started decomposition for the FP32-bulk kernels: A = ref^T W ref (its
// upper triangle), two cyclic Jacobi sweeps with the symmetric update
// (a_pp -= t a_pq, a_qq += t a_pq, a_pq = 0, and the rows r != p, q rotated),
// then U = ref V, eigenvalues ascending and each eigenvector's sign aligned with
// its reference column.  The same rotations as eigh_ns in exact arithmetic, with
// about a third fewer operations per rotation (no update of the elements the
// rotation annihilates or leaves symmetric).
template <int NS, typename V>
__device__ __forceinline__ void eigh_warm_sym(const V (&W)[NS][NS], const V (&ref)[NS][NS],
                                              V (&e)[NS], V (&U)[NS][NS]) {
  // V = float (one walker) or float2 (two walkers, one per lane): the FP32
  // arithmetic is the packed lane arithmetic of lanes.cuh (explicit
  // round-to-nearest, so each lane's bits do not depend on the lane count);
  // divisions, square roots, compares and selects run per lane.
  constexpr int L = Lanes<V>::W;
  V A[NS][NS], Vm[NS][NS];
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
    for (int b = 0; b < NS; ++b) Vm[a][b] = splat<V>(a == b ? 1.0f : 0.0f);
  // upper-triangle element (i, j) of A for any order of i, j
  auto at = [&](int i, int j) -> V& { return i < j ? A[i][j] : A[j][i]; };
#pragma unroll 1
  for (int sweep = 0; sweep < 2; ++sweep) {
#pragma unroll
    for (int p = 0; p < NS; ++p)
#pragma unroll
      for (int q = p + 1; q < NS; ++q) {
        const V apq = A[p][q];
        // t = sgn(tau) / (|tau| + sqrt(1 + tau^2)) with approximate division and
        // square root (c and s follow from the same t, so the rotation stays
        // orthogonal to rounding); |tau| is capped at 1e18, where t < 1e-18; a
        // zero a_pq selects the identity rotation
        const V d = vsub(A[q][q], A[p][p]);
        const V twoa = vmul(splat<V>(2.0f), apq);
        V tau, t, c;
        bool zero[L];
#pragma unroll
        for (int l = 0; l < L; ++l) {
          zero[l] = ln(apq, l) == 0.0f;
          ln(tau, l) = fminf(fmaxf(__fdividef(ln(d, l), zero[l] ? 2.0f : ln(twoa, l)), -1e18f), 1e18f);
        }
        const V w2 = vfma(tau, tau, splat<V>(1.0f));
#pragma unroll
        for (int l = 0; l < L; ++l) {
          const float tl = ln(tau, l), wl = ln(w2, l);
          const float tr = __fdividef(tl >= 0.0f ? 1.0f : -1.0f, __fmaf_rn(wl, rsqrtf(wl), fabsf(tl)));
          ln(t, l) = zero[l] ? 0.0f : tr;
        }
        const V tt1 = vfma(t, t, splat<V>(1.0f));
#pragma unroll
        for (int l = 0; l < L; ++l) ln(c, l) = zero[l] ? 1.0f : rsqrtf(ln(tt1, l));
        const V sn = vmul(t, c), nsn = vmul(sn, splat<V>(-1.0f));
        A[p][p] = vfma(t, vmul(apq, splat<V>(-1.0f)), A[p][p]);  // a_pp - t a_pq
        A[q][q] = vfma(t, apq, A[q][q]);
        A[p][q] = splat<V>(0.0f);
#pragma unroll
        for (int r = 0; r < NS; ++r) {
          if (r == p || r == q) continue;
          const V arp = at(r, p), arq = at(r, q);
          at(r, p) = vfma(c, arp, vmul(nsn, arq));
          at(r, q) = vfma(sn, arp, vmul(c, arq));
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const V vkp = Vm[k][p], vkq = Vm[k][q];
          Vm[k][p] = vfma(c, vkp, vmul(nsn, vkq));
          Vm[k][q] = vfma(sn, vkp, vmul(c, vkq));
        }
      }
  }
#pragma unroll
  for (int a = 0; a < NS; ++a) e[a] = A[a][a];
  // ascending order of (e, columns of Vm) by a fixed compare network.  The warm
  // start keeps the reference's ascending order except where eigenvalues pass
  // each other, and on sorted input the network swaps nothing, so it runs only
  // when some walker of the warp is out of order (the same result either way).
  bool unsorted = false;
#pragma unroll
  for (int l = 0; l < L; ++l)
#pragma unroll
    for (int j = 1; j < NS; ++j) unsorted |= ln(e[j], l) < ln(e[j - 1], l);
  if (__any_sync(0xffffffffu, unsorted)) {
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
            const float u0 = ln(Vm[k][j], l), u1 = ln(Vm[k][j - 1], l);
            ln(Vm[k][j], l) = sw ? u1 : u0;
            ln(Vm[k][j - 1], l) = sw ? u0 : u1;
          }
        }
  }
  // U = ref Vm; eigenvector b follows reference column b: <U_b, ref_b> = Vm[b][b]
  V sg[NS];
#pragma unroll
  for (int b = 0; b < NS; ++b)
#pragma unroll
    for (int l = 0; l < L; ++l) ln(sg[b], l) = ln(Vm[b][b], l) < 0.0f ? -1.0f : 1.0f;
#pragma unroll
  for (int i = 0; i < NS; ++i)
#pragma unroll
    for (int b = 0; b < NS; ++b) {
      V acc = splat<V>(0.0f);
#pragma unroll
      for (int k = 0; k < NS; ++k) acc = vfma(ref[i][k], Vm[k][b], acc);
      U[i][b] = vmul(acc, sg[b]);
    }
}

}  // namespace qcl
