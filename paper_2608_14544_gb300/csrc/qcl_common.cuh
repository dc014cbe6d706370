// qcl_common.cuh -- device-side building blocks shared by the kernels:
// Philox4x32-10, compensated FP32 arithmetic, buffer layouts and the device
// model block.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qcl.h"

namespace qcl {

constexpr int kTile = 256;       // walkers per reduction tile
constexpr int kGroup = 32;       // walkers per shuffle group
constexpr int kMaxNS = QCL_MAX_STATES;
constexpr int kMaxN = QCL_MAX_MODES;
constexpr uint32_t kPurposeInit = 1u;
constexpr uint32_t kPurposeHop = 2u;
constexpr float kP24f = 16777216.0f;
constexpr double kP24 = 16777216.0;

// ------------------------------------------------------------------ Philox --
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, each two 32x32->64 bit
// products mixed with the other counter words and the round key; Weyl key
// schedule between rounds.
struct u4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return {c0, c1, c2, c3};
}

__device__ __forceinline__ u4 philox_draw(uint64_t seed, uint32_t c0, uint64_t traj,
                                          uint32_t purpose) {
  return philox(c0, (uint32_t)traj, (uint32_t)(traj >> 32), purpose, (uint32_t)seed,
                (uint32_t)(seed >> 32));
}

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// The Philox4x32-10 stream of one walker and purpose: counter (n, traj_lo,
// traj_hi, purpose) with only the block number n varying between draws.  The
// terms of the first two rounds that involve the fixed counter words alone are
// computed once; with n the same on every thread (a block-uniform step), what
// is left of those two rounds is uniform work and two XORs per walker.
// draw(n) returns the same words as philox(n, traj_lo, traj_hi, purpose, key).
struct PhiloxStream {
  uint32_t e, f, d;  // per-walker words entering round 2 (see draw)
  uint32_t g;        // purpose ^ k1
  uint32_t k0, k1;

  PhiloxStream() = default;
  __host__ __device__ __forceinline__ PhiloxStream(uint64_t seed, uint64_t traj, uint32_t purpose) {
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
    const uint32_t tl = (uint32_t)traj, th = (uint32_t)(traj >> 32);
    // round 0, the product of the fixed word traj_hi
    const uint32_t a = mulhi32(0xCD9E8D57u, th) ^ tl ^ k0;  // new word 0
    const uint32_t b = 0xCD9E8D57u * th;                    // new word 1
    // round 1, the product of word 0 (fixed)
    e = b ^ (k0 + 0x9E3779B9u);
    f = mulhi32(0xD2511F53u, a) ^ (k1 + 0xBB67AE85u);
    d = 0xD2511F53u * a;
    g = purpose ^ k1;
  }

  __host__ __device__ __forceinline__ u4 draw(uint32_t n) const {
    // round 0: the product of the block number
    const uint32_t s2 = mulhi32(0xD2511F53u, n) ^ g;
    const uint32_t s3 = 0xD2511F53u * n;
    // round 1: the product of word 2
    uint32_t c0 = mulhi32(0xCD9E8D57u, s2) ^ e;
    uint32_t c1 = 0xCD9E8D57u * s2;
    uint32_t c2 = s3 ^ f;
    uint32_t c3 = d;
    uint32_t q0 = k0 + 2u * 0x9E3779B9u, q1 = k1 + 2u * 0xBB67AE85u;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
      const uint32_t hi0 = mulhi32(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
      const uint32_t hi1 = mulhi32(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
      c0 = hi1 ^ c1 ^ q0;
      c1 = lo1;
      c2 = hi0 ^ c3 ^ q1;
      c3 = lo0;
      q0 += 0x9E3779B9u;
      q1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
  }
};

__device__ __forceinline__ uint32_t word_of(const u4& w, int i) {
  return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

// ------------------------------------------------ compensated FP32 pairs --
// (hi, lo) with |lo| <= ulp(hi)/2 represents hi + lo to about 2^-46.  V is
// float, or float2 for the same pair of two walkers held in one register pair.
template <typename V>
struct PairV {
  V hi, lo;
};
using f2 = PairV<float>;

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float err = (a - (s - bb)) + (b - bb);
  return {s, err};
}

__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

// (hi, lo) += b
__device__ __forceinline__ f2 df_add(f2 a, float b) {
  const f2 s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, s.lo + a.lo);
}

// (hi, lo) *= (q0 + q1)
__device__ __forceinline__ f2 df_mul(f2 a, float q0, float q1) {
  const float p = a.hi * q0;
  float e = __fmaf_rn(a.hi, q0, -p);
  e = __fmaf_rn(a.hi, q1, e);
  e = __fmaf_rn(a.lo, q0, e);
  return fast_two_sum(p, e);
}

// c / d as an unevaluated pair q0 + q1 (d exact, c exact)
__device__ __forceinline__ void df_div(float c, float d, float& q0, float& q1) {
  const float r = __frcp_rn(d);
  q0 = c * r;
  const float res = __fmaf_rn(-q0, d, c);
  q1 = res * r;
}

// ------------------------------------------------------------ device model --
// Constants derived on the host by qcl_create_model.  Two-state models use the
// closed form W = s 1 + a sigma_z + b sigma_x with a = a0 + sum a_j R_j,
// b = b0 + sum b_j R_j; s only enters through its constant gradient s_j.
struct DevModel {
  int32_t ns, n;
  int32_t kind;       // 0: only a_j nonzero (spin-boson form), 1: general two-state
  int32_t repr;       // QCL_REPR_ADIABATIC or QCL_REPR_DIABATIC
  double hbar, hop_scale, p_max;
  double a0, b0, s0;
  // per-mode arrays [n]
  double mass[kMaxN], omega[kMaxN], k[kMaxN];
  double a[kMaxN], b[kMaxN], s[kMaxN];
  double E[kMaxNS * kMaxNS];
  // K[j][ns*ns] follows in a separate allocation (pointer below)
  const double* K;
};

// ------------------------------------------------------------------ layouts --
constexpr uint64_t kEnsMagic = 0x31454C4351ull;  // "QCLE1"

struct EnsHeader {
  uint64_t magic;
  int64_t n_traj;
  int32_t precision, ns, n, pad0;
  int64_t step;
  uint32_t flags;
  uint32_t pad1;
  unsigned long long n_degenerate;
  unsigned long long n_nonfinite;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// SoA ensemble layout.  Every array starts on a 256-byte boundary.
struct EnsLayout {
  size_t off_R, off_P, off_m, off_mlo, off_mexp, off_phi, off_philo, off_ab, off_U, off_E, total;
  __host__ __device__ static EnsLayout make(int64_t n_traj, int ns, int n, int precision) {
    EnsLayout L{};
    const size_t nt = (size_t)n_traj;
    const size_t w = (precision == QCL_PREC_FP64) ? 8 : 4;
    size_t o = align256(sizeof(EnsHeader));
    L.off_R = o;
    o = align256(o + w * nt * (size_t)n);
    L.off_P = o;
    o = align256(o + w * nt * (size_t)n);
    L.off_m = o;
    o = align256(o + w * nt);
    L.off_mlo = o;
    o = align256(o + w * nt);
    L.off_mexp = o;
    o = align256(o + 4 * nt);
    L.off_phi = o;
    o = align256(o + w * nt);
    L.off_philo = o;
    o = align256(o + w * nt);
    L.off_ab = o;
    o = align256(o + 2 * nt);
    L.off_U = o;
    if (ns > 2) o = align256(o + w * nt * (size_t)(ns * ns));
    L.off_E = o;
    if (ns > 2) o = align256(o + w * nt * (size_t)ns);
    L.total = o;
    return L;
  }
};

// Observation buffer: [rows n_out][2Q] FP64 sums, then per-tile partials
// [chunk][n_tiles][2Q] FP64, then finalised rows [n_out][2Q+3], then fold
// scratch for block partials.
constexpr int kChunkOut = 32;      // output times per persistent launch
constexpr int kFoldBlock = 1024;   // tiles per first-level fold block (power of two)

// Threads per walker of the FP32-bulk kernel for a model of n modes: up to 32
// modes a thread holds a whole walker in registers; beyond that the walker's
// modes are split over 2 or 4 warps (one thread of each).  A tile (the unit of
// the fixed reduction tree) is one block of 256 threads: 256 / that walkers.
__host__ __device__ inline int bulk_lanes(int n) { return n <= 32 ? 1 : (n <= 64 ? 2 : 4); }
__host__ __device__ inline int tile_walkers(int precision, int n, int ns = 2) {
  if (precision == QCL_PREC_FP64) return kTile;
  return ns > 2 ? 128 : kTile / bulk_lanes(n);
}

// The per-chunk sums (chunks of kFoldBlock tiles, the first level of the tile
// fold: aligned subtrees of the reduction tree) are kept for every output row
// when there is more than one chunk, for combining shards.
struct ObsLayout {
  size_t off_rows, off_part, off_fin, off_fold, off_chunk, total;
  int64_t n_tiles, n_fold_blocks;
  int q2;
  __host__ __device__ static ObsLayout make(int64_t n_traj, int ns, int64_t n_out,
                                            int tile = kTile) {
    ObsLayout L{};
    L.q2 = 8 * ns * ns;
    L.n_tiles = (n_traj + tile - 1) / tile;
    L.n_fold_blocks = (L.n_tiles + kFoldBlock - 1) / kFoldBlock;
    size_t o = 0;
    L.off_rows = o;
    o = align256(o + sizeof(double) * (size_t)n_out * L.q2);
    L.off_part = o;
    o = align256(o + sizeof(double) * (size_t)kChunkOut * (size_t)L.n_tiles * L.q2);
    L.off_fin = o;
    o = align256(o + sizeof(double) * (size_t)n_out * (L.q2 + 3));
    L.off_fold = o;
    const int64_t fold_rows = L.n_fold_blocks + (L.n_fold_blocks + kFoldBlock - 1) / kFoldBlock + 1;
    o = align256(o + sizeof(double) * (size_t)kChunkOut * (size_t)fold_rows * L.q2);
    L.off_chunk = o;
    if (L.n_fold_blocks > 1) o = align256(o + sizeof(double) * (size_t)n_out * (size_t)L.n_fold_blocks * L.q2);
    L.total = o;
    return L;
  }
};

}  // namespace qcl
