// kernels_f64.cu -- FP64 path: the plain comparator with the paper's structure
// (Sec. II B: walker state in contiguous GPU arrays, one kernel launch per time
// step, 256 threads per block, ceil-div grid), in double precision.  It is
// also the per-trajectory parity path against the CPU oracle.
#include "f64_2state.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace qcl {


// ---------------------------------------------------------------- sampling --
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
  uint16_t ab;
  sample_walker_f64(M, sp, sp.traj_offset + (uint64_t)i, w.R + i, w.P + i, nt, w.m[i], ab);
  w.phi[i] = 0.0;
  w.ab[i] = ab;
}

// -------------------------------------------------------------------- step --
// One full step n -> n+1 of one walker (velocity Verlet on the pair's mean
// force, trapezoid phase, one transition from the coupling term of Eq. 1, or
// of its diabatic form when DIA), one launch per step.  The index-pair word
// carries the quarter-turn count of a diabatic walker in bits 4-5.
template <int NP, bool DIA>
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
  const uint16_t ab = w.ab[i];
  int al = ab & 0xf, be = (ab >> 8) & 0xf, q = (ab >> 4) & 3;
  double m = w.m[i], phi = w.phi[i];
  const Step64 o = walker_step_f64<NP, DIA>(M, w.R + i, w.P + i, nt, n, al, be, phi, dt, seed,
                                            traj_off + (uint64_t)i, step);
  m = m * o.num / o.den;
  if (o.ev == 1) al ^= 1;
  if (o.ev == 2) be ^= 1;
  q = (q + o.dq) & 3;
  w.m[i] = m;
  w.phi[i] = phi;
  w.ab[i] = (uint16_t)(al | (q << 4) | (be << 8));
  if (o.deg) {
    atomicAdd(&w.hdr->n_degenerate, 1ull);
    atomicOr(&w.hdr->flags, QCL_FLAG_DEGENERATE);
  }
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
  if (i < nt) contrib_f64(M, w.R + i, nt, n, w.m[i], w.phi[i], w.ab[i], v);
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
  const bool dia = repr == QCL_REPR_DIABATIC;
#define QCL_STEP64(NP)                                                                       \
  (dia ? k_step_f64<NP, true><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off) \
       : k_step_f64<NP, false><<<nb, 256, 0, st>>>(dm, buf, nt, n, step0, step, dt, seed, traj_off))
  if (n <= 1)
    QCL_STEP64(1);
  else if (n <= 4)
    QCL_STEP64(4);
  else if (n <= 16)
    QCL_STEP64(16);
  else
    QCL_STEP64(0);
#undef QCL_STEP64
  launches_add(1);
}

void launch_observe_f64(const DevModel* dm, const void* buf, int64_t nt, int n, double* part,
                        cudaStream_t st) {
  const unsigned nb = (unsigned)((nt + 255) / 256);
  k_observe_f64<<<nb, 256, 0, st>>>(dm, buf, nt, n, part);
  launches_add(1);
}

}  // namespace qcl
