// reduce.cuh -- fixed-order ensemble reduction.
//
// The sum of every observable over the walkers follows one tree that does not
// depend on the launch shape (the paper's Sec. II B reduces with a
// deterministic-order mapreduce rather than atomics, for reproducibility):
//   1. 32-walker group: reduce-scatter butterfly across the warp (lane l ends
//      with quantity l); FP32 in the bulk path, FP64 in the FP64 path;
//   2. 256-walker tile: FP64 binary tree over the 8 groups, written to a
//      per-tile partial (no atomics);
//   3. tiles: FP64 binary tree in tile-index order, zero-padded to a power of
//      two, computed as 1024-tile blocks (power-of-two aligned subtrees).
#pragma once
#include "qcl_common.cuh"

namespace qcl {

// Reduce-scatter butterfly: on entry lane l holds v[0..31] for its walker; on
// exit v[0] of lane l is the sum over the 32 lanes of quantity l.  Pairing at
// level k is (lane, lane ^ (16 >> k)); a + b == b + a keeps both partners'
// results identical.
template <typename T>
__device__ __forceinline__ T warp_transpose_sum(T (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int lev = 0; lev < 5; ++lev) {
    const int half = 16 >> lev;
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const T send = upper ? v[i] : v[half + i];
      const T keep = upper ? v[half + i] : v[i];
      const T recv = __shfl_xor_sync(0xffffffffu, send, half);
      v[i] = keep + recv;
    }
  }
  return v[0];
}

// Binary tree over the 8 group partials of a tile held in smem red[8][nq];
// thread q (< nq) writes the tile partial of quantity q.
__device__ __forceinline__ double tile_tree8(const double* red, int nq, int q) {
  const double a = red[0 * nq + q] + red[1 * nq + q];
  const double b = red[2 * nq + q] + red[3 * nq + q];
  const double c = red[4 * nq + q] + red[5 * nq + q];
  const double d = red[6 * nq + q] + red[7 * nq + q];
  return (a + b) + (c + d);
}

}  // namespace qcl
