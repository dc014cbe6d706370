// f64_2state.cuh -- device code of the FP64 two-state walker shared by the
// one-launch-per-step kernels (kernels_f64.cu) and the spawning kernels
// (spawn.cu): SoA views, the closed-form decomposition, the half kicks, one
// whole step of one walker (Verlet, phase, transition test) and the walker's
// observable contributions.
#pragma once
#include "kernels.h"

namespace qcl {

constexpr double kDegTol = 1e-12;  // |e_b - e_a| below this: coupling set to 0

struct W64 {
  double* R;
  double* P;
  double* m;
  double* phi;
  uint16_t* ab;
  EnsHeader* hdr;
};

__device__ __forceinline__ W64 view64(void* buf, int64_t nt, int ns, int n) {
  const EnsLayout L = EnsLayout::make(nt, ns, n, QCL_PREC_FP64);
  char* b = (char*)buf;
  return {(double*)(b + L.off_R), (double*)(b + L.off_P), (double*)(b + L.off_m),
          (double*)(b + L.off_phi), (uint16_t*)(b + L.off_ab), (EnsHeader*)b};
}

// Closed-form two-state decomposition at R: W = s + a sigma_z + b sigma_x,
// r = |(a, b)|, cos 2theta = a/r, sin 2theta = b/r (theta = atan2(b, a)/2, with
// theta = 0 at r = 0); the eigenvector angle (c, s) = (cos theta, sin theta) by
// the cancellation-free half-angle formulas.
struct Ad2 {
  double a, b, r, c2, s2;
};

template <int NP>
__device__ __forceinline__ Ad2 decomp(const DevModel* M, const double* R, int n) {
  double a = M->a0, b = M->b0;
#pragma unroll
  for (int j = 0; j < NP; ++j)
    if (j < n) {
      a += M->a[j] * R[j];
      b += M->b[j] * R[j];
    }
  Ad2 d;
  d.a = a;
  d.b = b;
  d.r = sqrt(a * a + b * b);
  if (d.r > 0.0) {
    d.c2 = a / d.r;
    d.s2 = b / d.r;
  } else {
    d.c2 = 1.0;
    d.s2 = 0.0;
  }
  return d;
}

__device__ __forceinline__ void half_angle(const Ad2& d, double& c, double& s) {
  if (d.r == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  if (d.a >= 0.0) {
    c = sqrt((d.r + d.a) / (2.0 * d.r));
    s = d.b / (2.0 * d.r * c);
  } else {
    s = copysign(sqrt((d.r - d.a) / (2.0 * d.r)), d.b);
    c = d.b / (2.0 * d.r * s);
  }
}

__device__ __forceinline__ double sigma(int idx) { return idx ? 1.0 : -1.0; }

// P += dt/2 F_ab(R), F_j = -k_j R_j - s_j - 1/2 (sig_a + sig_b)(a_j cos2t + b_j sin2t)
template <int NP>
__device__ __forceinline__ void half_kick(const DevModel* M, const double* R, double* P, int n,
                                          const Ad2& d, int al, int be, double dt) {
  const double sab = 0.5 * (sigma(al) + sigma(be));
#pragma unroll
  for (int j = 0; j < NP; ++j)
    if (j < n) {
      const double F =
          -M->k[j] * R[j] - (M->s[j] + sab * (M->a[j] * d.c2 + M->b[j] * d.s2));
      P[j] += 0.5 * dt * F;
    }
}

// Global-memory variant for large mode counts: the same arithmetic reading
// R, P from the SoA arrays (stride nt).
__device__ __forceinline__ Ad2 decomp_g(const DevModel* M, const double* R, int64_t nt, int n) {
  double a = M->a0, b = M->b0;
  for (int j = 0; j < n; ++j) {
    const double x = R[(int64_t)j * nt];
    a += M->a[j] * x;
    b += M->b[j] * x;
  }
  Ad2 d;
  d.a = a;
  d.b = b;
  d.r = sqrt(a * a + b * b);
  if (d.r > 0.0) {
    d.c2 = a / d.r;
    d.s2 = b / d.r;
  } else {
    d.c2 = 1.0;
    d.s2 = 0.0;
  }
  return d;
}


template <typename T>
__device__ __forceinline__ void pick_pair(const double* rho_ad, int ns, uint32_t word,
                                          int& al, int& be, double& m0) {
  double tot = 0.0;
  for (int k = 0; k < ns * ns; ++k) tot += fabs(rho_ad[k]);
  uint32_t Tk[kMaxNS * kMaxNS];
  uint64_t sumT = 0;
  int last = -1;
  for (int k = 0; k < ns * ns; ++k) {
    Tk[k] = (uint32_t)floor(fabs(rho_ad[k]) / tot * kP24);
    sumT += Tk[k];
    if (rho_ad[k] != 0.0) last = k;
  }
  Tk[last] += (uint32_t)(16777216ull - sumT);
  const uint32_t y = word >> 8;
  uint64_t cum = 0;
  int pick = last;
  for (int k = 0; k < ns * ns; ++k) {
    cum += Tk[k];
    if ((uint64_t)y < cum) {
      pick = k;
      break;
    }
  }
  al = pick / ns;
  be = pick % ns;
  m0 = rho_ad[pick] / ((double)Tk[pick] / kP24);
}

// Initial sample of one walker with random-stream id `traj`: (R, P) from the
// harmonic Wigner distribution (Box-Muller pair of Philox block (c0 = j,
// purpose INIT) per mode), then the index pair drawn from |rho| in the
// walkers' representation (adiabatic: U^T rho_el0 U at the walker's R;
// diabatic: rho_el0) with word 0 of block (c0 = n, purpose INIT), m0 = rho_ab /
// p_hat.  R, P written at Rg[j * stride], Pg[j * stride].
__device__ __forceinline__ void sample_walker_f64(const DevModel* __restrict__ M,
                                                  const SampleParams& sp, uint64_t traj,
                                                  double* Rg, double* Pg, int64_t stride,
                                                  double& m0, uint16_t& ab) {
  const int n = sp.n;
  double a = M->a0, b = M->b0;
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
    a += M->a[j] * R;
    b += M->b[j] * R;
  }
  Ad2 d;
  d.a = a;
  d.b = b;
  d.r = sqrt(a * a + b * b);
  double c, s;
  half_angle(d, c, s);
  const double U[4] = {-s, c, c, s};  // U[i*2 + alpha]
  double rho_ad[4];  // the density in the walkers' representation
  for (int al = 0; al < 2; ++al)
    for (int be = 0; be < 2; ++be) {
      double acc = 0.0;
      if (M->repr == QCL_REPR_DIABATIC) {
        acc = sp.rho[al * 2 + be];
      } else {
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l) acc += U[k * 2 + al] * sp.rho[k * 2 + l] * U[l * 2 + be];
      }
      rho_ad[al * 2 + be] = acc;
    }
  const u4 wd = philox_draw(sp.seed, (uint32_t)n, traj, kPurposeInit);
  int al, be;
  pick_pair<double>(rho_ad, 2, wd.x, al, be, m0);
  ab = (uint16_t)(al | (be << 8));
}

// Outcome of one step's transition test: event 0 (none), 1 (first index) or
// 2 (second index); the weight factor num / den that the event carries
// (m <- m * num / den: A_e / p_hat_e for an event, 1 / (1 - sum p_hat) for
// none), the event's quarter turns, and whether a degenerate gap was met.
struct Step64 {
  int ev;
  double num, den;
  int dq;
  bool deg;
};

// One step n -> n+1 of one two-state walker in FP64: velocity Verlet on the
// pair's mean force (adiabatic: Hellmann-Feynman diagonal; diabatic: the
// diagonal of W), the trapezoid phase, and the transition test with the
// walker's hop stream `stream` (Philox word n & 3 of block n >> 2).  R and P
// are read and written at Rg[j * stride], Pg[j * stride].
template <int NP, bool DIA>
__device__ __forceinline__ Step64 walker_step_f64(const DevModel* __restrict__ M, double* Rg,
                                                  double* Pg, int64_t stride, int n, int al,
                                                  int be, double& phi, double dt, uint64_t seed,
                                                  uint64_t stream, int64_t step) {
  Ad2 d0, d1;
  double Av = 0.0, Bv = 0.0;
  if constexpr (NP > 0) {
    double R[NP], P[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) {
        R[j] = Rg[(int64_t)j * stride];
        P[j] = Pg[(int64_t)j * stride];
      }
    d0 = decomp<NP>(M, R, n);
    if (DIA) {  // the diagonal force is the kick's with cos 2theta = -1, sin 2theta = 0
      d0.c2 = -1.0;
      d0.s2 = 0.0;
    }
    half_kick<NP>(M, R, P, n, d0, al, be, dt);
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) R[j] += dt * P[j] / M->mass[j];
    d1 = decomp<NP>(M, R, n);
    if (DIA) {
      d1.c2 = -1.0;
      d1.s2 = 0.0;
    }
    half_kick<NP>(M, R, P, n, d1, al, be, dt);
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) {
        if (!DIA) {
          Av += M->a[j] * (P[j] / M->mass[j]);
          Bv += M->b[j] * (P[j] / M->mass[j]);
        }
        Rg[(int64_t)j * stride] = R[j];
        Pg[(int64_t)j * stride] = P[j];
      }
  } else {
    // large mode counts: several passes over the SoA arrays
    d0 = decomp_g(M, Rg, stride, n);
    const double sab = 0.5 * (sigma(al) + sigma(be));
    const double c0 = DIA ? -1.0 : d0.c2, s0 = DIA ? 0.0 : d0.s2;
    for (int j = 0; j < n; ++j) {
      const int64_t o = (int64_t)j * stride;
      const double x = Rg[o];
      double p = Pg[o];
      p += 0.5 * dt * (-M->k[j] * x - (M->s[j] + sab * (M->a[j] * c0 + M->b[j] * s0)));
      Pg[o] = p;
      Rg[o] = x + dt * p / M->mass[j];
    }
    d1 = decomp_g(M, Rg, stride, n);
    const double c1 = DIA ? -1.0 : d1.c2, s1 = DIA ? 0.0 : d1.s2;
    for (int j = 0; j < n; ++j) {
      const int64_t o = (int64_t)j * stride;
      const double x = Rg[o];
      double p = Pg[o];
      p += 0.5 * dt * (-M->k[j] * x - (M->s[j] + sab * (M->a[j] * c1 + M->b[j] * s1)));
      Pg[o] = p;
      if (!DIA) {
        Av += M->a[j] * (p / M->mass[j]);
        Bv += M->b[j] * (p / M->mass[j]);
      }
    }
  }
  Step64 o;
  o.deg = false;
  double A1, A2;
  if (DIA) {
    // phase: V_aa - V_bb = (d_a - d_b) a = -(sig_a - sig_b) a
    const double w0 = -(sigma(al) - sigma(be)) * d0.a / M->hbar;
    const double w1 = -(sigma(al) - sigma(be)) * d1.a / M->hbar;
    phi += 0.5 * dt * (w0 + w1);
    // both events have the real factor c = V_01 dt / hbar = b(R_{n+1}) dt / hbar
    A1 = d1.b * dt / M->hbar;
    A2 = A1;
  } else {
    if (2.0 * d0.r < kDegTol || 2.0 * d1.r < kDegTol) o.deg = true;
    // phase: hbar w_ab = e_a - e_b = (sig_a - sig_b) r
    const double w0 = (sigma(al) - sigma(be)) * d0.r / M->hbar;
    const double w1 = (sigma(al) - sigma(be)) * d1.r / M->hbar;
    phi += 0.5 * dt * (w0 + w1);
    // coupling contracted with P/M: g = sum_j (P_j/M_j) d_01,j, d_01,j = (a b_j - b a_j)/(2 r^2)
    double g = 0.0;
    if (2.0 * d1.r >= kDegTol) g = (d1.a * Bv - d1.b * Av) / (2.0 * d1.r * d1.r);
    // events: (first index flips) then (second index flips)
    A1 = (al == 0) ? dt * g : -(dt * g);
    A2 = (be == 0) ? dt * g : -(dt * g);
  }
  // probabilities min(kappa |A_e|, p_max) quantised to 24-bit thresholds, then
  // scaled down together in exact integer arithmetic when their sum exceeds Tmax
  const double p1 = fmin(M->hop_scale * fabs(A1), M->p_max);
  const double p2 = fmin(M->hop_scale * fabs(A2), M->p_max);
  uint64_t T1 = (uint64_t)floor(p1 * kP24), T2 = (uint64_t)floor(p2 * kP24);
  const uint64_t Tmax = (uint64_t)floor(M->p_max * kP24);
  if (T1 + T2 > Tmax) {
    const uint64_t sT = T1 + T2;
    T1 = T1 * Tmax / sT;
    T2 = T2 * Tmax / sT;
  }
  const u4 wd = philox_draw(seed, (uint32_t)(step >> 2), stream, kPurposeHop);
  const uint32_t y = word_of(wd, (int)(step & 3)) >> 8;
  if ((uint64_t)y < T1) {  // diabatic: amplitude -i c
    o.ev = 1;
    o.num = A1;
    o.den = (double)T1 / kP24;
    o.dq = 3;
  } else if ((uint64_t)y < T1 + T2) {  // diabatic: amplitude +i c
    o.ev = 2;
    o.num = A2;
    o.den = (double)T2 / kP24;
    o.dq = 1;
  } else {
    o.ev = 0;
    o.num = 1.0;
    o.den = 1.0 - (double)(T1 + T2) / kP24;
    o.dq = 0;
  }
  if (!DIA) o.dq = 0;
  return o;
}

// The 16 observable contributions of one walker and their squares (v[16..31]):
// z = m exp(-i phi) i^q at the walker's own pair in its own representation,
// z U_ia U_jb (U symmetric) at every element of the other.  R at Rg[j * stride].
__device__ __forceinline__ void contrib_f64(const DevModel* __restrict__ M, const double* Rg,
                                            int64_t stride, int n, double m, double phi,
                                            uint16_t ab, double (&v)[32]) {
  const Ad2 d = decomp_g(M, Rg, stride, n);
  double c, s;
  half_angle(d, c, s);
  const double U[4] = {-s, c, c, s};
  const int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
  double sn, cs;
  sincos(phi, &sn, &cs);
  const double xr = m * cs, xi = -m * sn;
  const double zr = q == 0 ? xr : (q == 1 ? -xi : (q == 2 ? -xr : xi));
  const double zi = q == 0 ? xi : (q == 1 ? xr : (q == 2 ? -xi : -xr));
  const bool dia = M->repr == QCL_REPR_DIABATIC;
  const int own = dia ? 0 : 8, other = dia ? 8 : 0;
#pragma unroll
  for (int ii = 0; ii < 2; ++ii)
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const double f = U[ii * 2 + al] * U[jj * 2 + be];
      v[other + 2 * (ii * 2 + jj)] = zr * f;
      v[other + 2 * (ii * 2 + jj) + 1] = zi * f;
    }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool hit = (k == al * 2 + be);
    v[own + 2 * k] = hit ? zr : 0.0;
    v[own + 2 * k + 1] = hit ? zi : 0.0;
  }
#pragma unroll
  for (int q2 = 0; q2 < 16; ++q2) v[16 + q2] = v[q2] * v[q2];
}

}  // namespace qcl
