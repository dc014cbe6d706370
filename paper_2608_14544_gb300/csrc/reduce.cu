// reduce.cu -- tile fold and finalisation kernels of the fixed-order ensemble
// reduction (see reduce.cuh for the tree).
#include "kernels.h"
#include "reduce.cuh"

namespace qcl {

// One level of the tile fold: in[row][n][nq] -> out[row][ceil(n/1024)][nq],
// each output the perfect binary tree over its 1024 inputs in natural order
// (zero past n).  Grid (ceil(n/1024), ceil(nq/32), rows), 256 threads: lane c
// of warp w takes column q0 + c and the tiles [128 w, 128 w + 128) of the
// block, as four 32-leaf trees in registers (a warp's load is 32 consecutive
// columns of one tile row, 256 contiguous bytes); the eight warp results are
// paired in shared memory.  The tree is the same for every launch shape.
__global__ void __launch_bounds__(256) k_fold_level(const double* __restrict__ in,
                                                    double* __restrict__ out, int64_t n, int nq,
                                                    int64_t in_row_stride,
                                                    int64_t out_row_stride) {
  __shared__ double c8[8][32];
  const int64_t blk = blockIdx.x;
  const int q = blockIdx.y * 32 + (threadIdx.x & 31);
  const int w = threadIdx.x >> 5;
  const int row = blockIdx.z;
  const bool col = q < nq;
  const double* src = in + (int64_t)row * in_row_stride + (col ? q : 0);
  double g[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t base = blk * 1024 + (int64_t)(w * 4 + k) * 32;
    double v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int64_t t = base + i;
      v[i] = (col && t < n) ? src[t * nq] : 0.0;
    }
#pragma unroll
    for (int s = 1; s < 32; s *= 2) {
#pragma unroll
      for (int i = 0; i < 32; i += 2 * s) v[i] += v[i + s];
    }
    g[k] = v[0];
  }
  c8[w][threadIdx.x & 31] = (g[0] + g[1]) + (g[2] + g[3]);
  __syncthreads();
  if (w == 0 && col) {
    const int c = threadIdx.x;
    const double x = ((c8[0][c] + c8[1][c]) + (c8[2][c] + c8[3][c])) +
                     ((c8[4][c] + c8[5][c]) + (c8[6][c] + c8[7][c]));
    out[(int64_t)row * out_row_stride + blk * nq + q] = x;
  }
}

// Means and standard errors of rows [k0, k0 + nrows) of sums (divide by N).
__global__ void k_finalize(const double* __restrict__ rows, double* __restrict__ fin, int nq,
                           int64_t k0, int64_t nrows, int64_t n_traj, int ns) {
  const int64_t r = blockIdx.x;
  if (r >= nrows) return;
  const double* s = rows + (k0 + r) * 2 * nq;
  double* o = fin + r * (2 * nq + 3);
  const double N = (double)n_traj;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const double S = s[q], S2 = s[nq + q];
    o[q] = S / N;
    const double var = fmax(S2 - S * S / N, 0.0) / fmax(N - 1.0, 1.0);
    o[nq + q] = sqrt(var / N);
  }
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int i = 0; i < ns; ++i) {
      tr += s[2 * (i * ns + i)];
      ti += s[2 * (i * ns + i) + 1];
    }
    o[2 * nq] = tr / N;
    o[2 * nq + 1] = ti / N;
    o[2 * nq + 2] = N;
  }
}

// ------------------------------------------------------------ fold/finalize --
void launch_fold(const double* part, double* rows_out, double* scratch, int64_t n_tiles, int q2,
                 int n_slots, cudaStream_t st, double* chunk_out) {
  // level 1: tiles -> 1024-tile blocks (kept in chunk_out when it is given and
  // there is more than one block); repeat until one value per row
  const double* in = part;
  int64_t n = n_tiles;
  int64_t in_stride = n_tiles * q2;
  double* bufs[2] = {scratch, scratch + (size_t)n_slots * ((n_tiles + 1023) / 1024) * q2};
  int which = 0;
  bool first = true;
  while (true) {
    const int64_t nb = (n + 1023) / 1024;
    double* out = (nb == 1) ? rows_out : ((first && chunk_out) ? chunk_out : bufs[which]);
    first = false;
    const int64_t out_stride = (nb == 1) ? q2 : nb * q2;
    dim3 grid((unsigned)nb, (unsigned)((q2 + 31) / 32), (unsigned)n_slots);
    k_fold_level<<<grid, 256, 0, st>>>(in, out, n, q2, in_stride, out_stride);
    launches_add(1);
    if (nb == 1) break;
    in = out;
    in_stride = out_stride;
    n = nb;
    which ^= 1;
  }
}

void launch_finalize(const double* rows, double* fin, int nq, int64_t k0, int64_t nrows,
                     int64_t n_traj, int ns, cudaStream_t st) {
  if (nrows <= 0) return;
  k_finalize<<<(unsigned)nrows, 64, 0, st>>>(rows, fin, nq, k0, nrows, n_traj, ns);
  launches_add(1);
}

}  // namespace qcl
