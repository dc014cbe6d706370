// kernels_f64.cu -- FP64 path: the plain comparator with the paper's structure
// (Sec. II B: walker state in contiguous GPU arrays, one kernel launch per time
// step, 256 threads per block, ceil-div grid), in double precision.  It is
// also the per-trajectory parity path against the CPU oracle.
#include "kernels.h"
#include "reduce.cuh"

namespace qcl {

namespace {

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

}  // namespace

// ---------------------------------------------------------------- sampling --
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

__global__ void __launch_bounds__(256) k_sample_f64(const DevModel* __restrict__ M,
                                                    SampleParams sp, void* buf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = sp.n_traj;
  const int n = sp.n, ns = sp.ns;
  W64 w = view64(buf, nt, ns, n);
  if (i == 0) {
    w.hdr->magic = kEnsMagic;
    w.hdr->n_traj = nt;
    w.hdr->precision = QCL_PREC_FP64;
    w.hdr->ns = ns;
    w.hdr->n = n;
    w.hdr->step = 0;
    w.hdr->flags = 0;
    w.hdr->n_degenerate = 0;
    w.hdr->n_nonfinite = 0;
  }
  if (i >= nt) return;
  const uint64_t traj = sp.traj_offset + (uint64_t)i;
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
    w.R[(int64_t)j * nt + i] = R;
    w.P[(int64_t)j * nt + i] = P;
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
  double m0;
  pick_pair<double>(rho_ad, 2, wd.x, al, be, m0);
  w.m[i] = m0;
  w.phi[i] = 0.0;
  w.ab[i] = (uint16_t)(al | (be << 8));
}

// -------------------------------------------------------------------- step --
// One full step n -> n+1 of one walker (velocity Verlet on the pair's mean
// force, trapezoid phase, one transition from the coupling term of Eq. 1).
template <int NP>
__global__ void __launch_bounds__(256) k_step_f64(const DevModel* __restrict__ M, void* buf,
                                                  int64_t nt, int n, int64_t step0, int64_t step,
                                                  double dt, uint64_t seed, uint64_t traj_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  W64 w = view64(buf, nt, 2, n);
  if (i >= nt) return;
  if (w.hdr->step != step0) {
    if (i == 0) atomicOr(&w.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  double R[NP > 0 ? NP : 1], P[NP > 0 ? NP : 1];
  const uint16_t ab = w.ab[i];
  int al = ab & 0xff, be = ab >> 8;
  double m = w.m[i], phi = w.phi[i];
  bool deg = false;
  Ad2 d0, d1;
  double Av = 0.0, Bv = 0.0;
  if constexpr (NP > 0) {
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) {
        R[j] = w.R[(int64_t)j * nt + i];
        P[j] = w.P[(int64_t)j * nt + i];
      }
    d0 = decomp<NP>(M, R, n);
    half_kick<NP>(M, R, P, n, d0, al, be, dt);
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) R[j] += dt * P[j] / M->mass[j];
    d1 = decomp<NP>(M, R, n);
    half_kick<NP>(M, R, P, n, d1, al, be, dt);
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) {
        Av += M->a[j] * (P[j] / M->mass[j]);
        Bv += M->b[j] * (P[j] / M->mass[j]);
        w.R[(int64_t)j * nt + i] = R[j];
        w.P[(int64_t)j * nt + i] = P[j];
      }
  } else {
    // large mode counts: several passes over the SoA arrays
    double* Rg = w.R + i;
    double* Pg = w.P + i;
    d0 = decomp_g(M, Rg, nt, n);
    const double sab = 0.5 * (sigma(al) + sigma(be));
    for (int j = 0; j < n; ++j) {
      const int64_t o = (int64_t)j * nt;
      const double x = Rg[o];
      double p = Pg[o];
      p += 0.5 * dt * (-M->k[j] * x - (M->s[j] + sab * (M->a[j] * d0.c2 + M->b[j] * d0.s2)));
      Pg[o] = p;
      Rg[o] = x + dt * p / M->mass[j];
    }
    d1 = decomp_g(M, Rg, nt, n);
    for (int j = 0; j < n; ++j) {
      const int64_t o = (int64_t)j * nt;
      const double x = Rg[o];
      double p = Pg[o];
      p += 0.5 * dt * (-M->k[j] * x - (M->s[j] + sab * (M->a[j] * d1.c2 + M->b[j] * d1.s2)));
      Pg[o] = p;
      Av += M->a[j] * (p / M->mass[j]);
      Bv += M->b[j] * (p / M->mass[j]);
    }
  }
  if (2.0 * d0.r < kDegTol || 2.0 * d1.r < kDegTol) deg = true;
  // phase: hbar w_ab = e_a - e_b = (sig_a - sig_b) r
  const double w0 = (sigma(al) - sigma(be)) * d0.r / M->hbar;
  const double w1 = (sigma(al) - sigma(be)) * d1.r / M->hbar;
  phi += 0.5 * dt * (w0 + w1);
  // coupling contracted with P/M: g = sum_j (P_j/M_j) d_01,j, d_01,j = (a b_j - b a_j)/(2 r^2)
  double g = 0.0;
  if (2.0 * d1.r >= kDegTol) g = (d1.a * Bv - d1.b * Av) / (2.0 * d1.r * d1.r);
  // events: (first index flips) then (second index flips)
  const double A1 = (al == 0) ? dt * g : -(dt * g);
  const double A2 = (be == 0) ? dt * g : -(dt * g);
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
  const u4 wd = philox_draw(seed, (uint32_t)(step >> 2), traj_off + (uint64_t)i, kPurposeHop);
  const uint32_t y = word_of(wd, (int)(step & 3)) >> 8;
  if ((uint64_t)y < T1) {
    m = m * A1 / ((double)T1 / kP24);
    al ^= 1;
  } else if ((uint64_t)y < T1 + T2) {
    m = m * A2 / ((double)T2 / kP24);
    be ^= 1;
  } else {
    m = m / (1.0 - (double)(T1 + T2) / kP24);
  }
  w.m[i] = m;
  w.phi[i] = phi;
  w.ab[i] = (uint16_t)(al | (be << 8));
  if (deg) {
    atomicAdd(&w.hdr->n_degenerate, 1ull);
    atomicOr(&w.hdr->flags, QCL_FLAG_DEGENERATE);
  }
  if (!isfinite(m) || !isfinite(phi)) {
    atomicAdd(&w.hdr->n_nonfinite, 1ull);
    atomicOr(&w.hdr->flags, QCL_FLAG_NONFINITE);
  }
}

// One full step of a diabatic walker: velocity Verlet on the diagonal mean
// force F_j = -k_j R_j - s_j - 1/2 (d_a + d_b) a_j (d = +1 for state 0, -1 for
// state 1), trapezoid phase with hbar w_ab = V_aa - V_bb = (d_a - d_b) a(R),
// and one transition: a -> 1-a with amplitude -i b(R) dt/hbar, b -> 1-b with
// +i b(R) dt/hbar (R at the end of the step).  The index pair word carries the
// quarter-turn count in bits 4-5.
template <int NP>
__global__ void __launch_bounds__(256) k_step_dia_f64(const DevModel* __restrict__ M, void* buf,
                                                      int64_t nt, int n, int64_t step0,
                                                      int64_t step, double dt, uint64_t seed,
                                                      uint64_t traj_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  W64 w = view64(buf, nt, 2, n);
  if (i >= nt) return;
  if (w.hdr->step != step0) {
    if (i == 0) atomicOr(&w.hdr->flags, QCL_FLAG_STEP_MISMATCH);
    return;
  }
  const uint16_t ab = w.ab[i];
  int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
  double m = w.m[i], phi = w.phi[i];
  // the diagonal force is the adiabatic kick's with cos 2theta = -1, sin 2theta = 0
  Ad2 d0, d1;
  if constexpr (NP > 0) {
    double R[NP], P[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) {
        R[j] = w.R[(int64_t)j * nt + i];
        P[j] = w.P[(int64_t)j * nt + i];
      }
    d0 = decomp<NP>(M, R, n);
    d0.c2 = -1.0;
    d0.s2 = 0.0;
    half_kick<NP>(M, R, P, n, d0, al, be, dt);
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) R[j] += dt * P[j] / M->mass[j];
    d1 = decomp<NP>(M, R, n);
    d1.c2 = -1.0;
    d1.s2 = 0.0;
    half_kick<NP>(M, R, P, n, d1, al, be, dt);
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) {
        w.R[(int64_t)j * nt + i] = R[j];
        w.P[(int64_t)j * nt + i] = P[j];
      }
  } else {
    double* Rg = w.R + i;
    double* Pg = w.P + i;
    d0 = decomp_g(M, Rg, nt, n);
    const double sab = 0.5 * (sigma(al) + sigma(be));
    for (int j = 0; j < n; ++j) {
      const int64_t o = (int64_t)j * nt;
      const double x = Rg[o];
      double p = Pg[o];
      p += 0.5 * dt * (-M->k[j] * x - (M->s[j] + sab * (M->a[j] * -1.0 + M->b[j] * 0.0)));
      Pg[o] = p;
      Rg[o] = x + dt * p / M->mass[j];
    }
    d1 = decomp_g(M, Rg, nt, n);
    for (int j = 0; j < n; ++j) {
      const int64_t o = (int64_t)j * nt;
      const double x = Rg[o];
      double p = Pg[o];
      p += 0.5 * dt * (-M->k[j] * x - (M->s[j] + sab * (M->a[j] * -1.0 + M->b[j] * 0.0)));
      Pg[o] = p;
    }
  }
  // phase: V_aa - V_bb = (d_a - d_b) a = -(sig_a - sig_b) a
  const double w0 = -(sigma(al) - sigma(be)) * d0.a / M->hbar;
  const double w1 = -(sigma(al) - sigma(be)) * d1.a / M->hbar;
  phi += 0.5 * dt * (w0 + w1);
  // both events have the real factor c = V_01 dt / hbar = b(R_{n+1}) dt / hbar
  const double cfac = d1.b * dt / M->hbar;
  const double p1 = fmin(M->hop_scale * fabs(cfac), M->p_max);
  uint64_t T1 = (uint64_t)floor(p1 * kP24), T2 = T1;
  const uint64_t Tmax = (uint64_t)floor(M->p_max * kP24);
  if (T1 + T2 > Tmax) {
    const uint64_t sT = T1 + T2;
    T1 = T1 * Tmax / sT;
    T2 = T2 * Tmax / sT;
  }
  const u4 wd = philox_draw(seed, (uint32_t)(step >> 2), traj_off + (uint64_t)i, kPurposeHop);
  const uint32_t y = word_of(wd, (int)(step & 3)) >> 8;
  if ((uint64_t)y < T1) {  // a -> 1 - a, amplitude -i c
    m = m * cfac / ((double)T1 / kP24);
    q = (q + 3) & 3;
    al ^= 1;
  } else if ((uint64_t)y < T1 + T2) {  // b -> 1 - b, amplitude +i c
    m = m * cfac / ((double)T2 / kP24);
    q = (q + 1) & 3;
    be ^= 1;
  } else {
    m = m / (1.0 - (double)(T1 + T2) / kP24);
  }
  w.m[i] = m;
  w.phi[i] = phi;
  w.ab[i] = (uint16_t)(al | (q << 4) | (be << 8));
  if (!isfinite(m) || !isfinite(phi)) {
    atomicAdd(&w.hdr->n_nonfinite, 1ull);
    atomicOr(&w.hdr->flags, QCL_FLAG_NONFINITE);
  }
}

// ------------------------------------------------------------- observation --
// Walker contributions m exp(-i phi) U_ia U_jb (diabatic) and m exp(-i phi) at
// (a, b) (adiabatic), and their squares, summed per 256-walker tile.
__global__ void __launch_bounds__(256) k_observe_f64(const DevModel* __restrict__ M,
                                                     const void* buf, int64_t nt, int n,
                                                     double* __restrict__ part) {
  __shared__ double red[8][32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  W64 w = view64((void*)buf, nt, 2, n);
  double v[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = 0.0;
  if (i < nt) {
    const Ad2 d = decomp_g(M, w.R + i, nt, n);
    double c, s;
    half_angle(d, c, s);
    const double U[4] = {-s, c, c, s};
    const uint16_t ab = w.ab[i];
    const int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
    double sn, cs;
    sincos(w.phi[i], &sn, &cs);
    // z = m exp(-i phi) i^q
    const double xr = w.m[i] * cs, xi = -w.m[i] * sn;
    const double zr = q == 0 ? xr : (q == 1 ? -xi : (q == 2 ? -xr : xi));
    const double zi = q == 0 ? xi : (q == 1 ? xr : (q == 2 ? -xi : -xr));
    // the walker's own representation gets z at its pair, the other one the
    // rotated products (U is symmetric, so U_ia U_jb and U_ai U_bj coincide)
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
    for (int q = 0; q < 16; ++q) v[16 + q] = v[q] * v[q];
  }
  const double x = warp_transpose_sum<double>(v);
  red[threadIdx.x >> 5][threadIdx.x & 31] = x;
  __syncthreads();
  if (threadIdx.x < 32) part[(int64_t)blockIdx.x * 32 + threadIdx.x] =
      tile_tree8(&red[0][0], 32, threadIdx.x);
}

// ------------------------------------------------------------------ launch --
void launch_sample_f64(const DevModel* dm, const SampleParams& sp, void* buf, cudaStream_t st) {
  const int64_t nb = (sp.n_traj + 255) / 256;
  k_sample_f64<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, st>>>(dm, sp, buf);
  launches_add(1);
}

void launch_step_f64(const DevModel* dm, int repr, void* buf, int64_t nt, int n, int64_t step0,
                     int64_t step, double dt, uint64_t seed, uint64_t traj_off, cudaStream_t st) {
  const unsigned nb = (unsigned)((nt + 255) / 256);
  if (repr == QCL_REPR_DIABATIC) {
    if (n <= 1)
      k_step_dia_f64<1><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
    else if (n <= 4)
      k_step_dia_f64<4><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
    else if (n <= 16)
      k_step_dia_f64<16><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
    else
      k_step_dia_f64<0><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
    launches_add(1);
    return;
  }
  if (n <= 1)
    k_step_f64<1><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
  else if (n <= 4)
    k_step_f64<4><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
  else if (n <= 16)
    k_step_f64<16><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
  else
    k_step_f64<0><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off);
  launches_add(1);
}

void launch_observe_f64(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                        cudaStream_t st) {
  const unsigned nb = (unsigned)((nt + 255) / 256);
  k_observe_f64<<<nb, 256, 0, st>>>(dm, buf, nt, n, part);
  launches_add(1);
}

}  // namespace qcl
