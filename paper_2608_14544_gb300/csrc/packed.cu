// packed.cu -- the server's packed persistent kernel: one launch advances the
// tiles of many two-state requests (each with its own model, walkers, steps
// and output slots), read from a device table of (request, tile) work items.
// Every request runs the same tile body as the single-request kernel, so its
// results do not depend on what else is packed with it.
#include "bulk2.cuh"

namespace qcl {

template <int NPL, int KIND>
__global__ void __launch_bounds__(256, 3) k_bulk2_packed(const PackedTable* __restrict__ tab) {
  __shared__ double red[2][8][32];
  __shared__ __align__(16) float obs_rows[256 * kObsRow];
  const int64_t n_work = tab->n_work;
  const int n_req = tab->n_req;
  int rb = 0;
  for (int64_t w = blockIdx.x; w < n_work; w += gridDim.x) {
    int lo = 0, hi = n_req - 1;  // the request owning work item w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab->req[mid].work0 <= w) lo = mid;
      else hi = mid - 1;
    }
    const PackedReq& R = tab->req[lo];
    const BulkParams bp = R.bp;
    CoefLocal<NPL> c;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      c.hk[j] = R.hk[j];
      c.hs[j] = R.hs[j];
      c.dtm[j] = R.dtm[j];
      c.a[j] = R.a[j];
      c.b[j] = R.b[j];
      c.am[j] = R.am[j];
      c.bm[j] = R.bm[j];
    }
    W32 ws = view32(R.ens, bp.n_traj, 2, bp.n);
    const int64_t tile = w - R.work0;
    if (ws.hdr->step != bp.step0) {
      if (tile == 0 && threadIdx.x == 0) atomicOr(&ws.hdr->flags, QCL_FLAG_STEP_MISMATCH);
      continue;
    }
    unsigned int n_deg = 0;
    bulk2_tile<NPL, KIND, CoefLocal<NPL>, true>(bp, c, ws, R.part, tile, rb, n_deg, red, obs_rows);
    if (n_deg) {
      atomicAdd(&ws.hdr->n_degenerate, (unsigned long long)n_deg);
      atomicOr(&ws.hdr->flags, QCL_FLAG_DEGENERATE);
    }
  }
}

namespace {
template <int NPL, int KIND>
int run_packed(const PackedTable* dtab, cudaStream_t st) {
  static int per_sm = -1, n_sm = 0;
  auto fn = k_bulk2_packed<NPL, KIND>;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  const int grid = per_sm * n_sm;
  fn<<<grid, 256, 0, st>>>(dtab);
  return grid;
}
template <int KIND>
int packed_kind(int bucket, const PackedTable* dtab, cudaStream_t st) {
  switch (bucket) {
    case 0: return run_packed<1, KIND>(dtab, st);
    case 1: return run_packed<2, KIND>(dtab, st);
    case 2: return run_packed<3, KIND>(dtab, st);
    case 3: return run_packed<4, KIND>(dtab, st);
    case 4: return run_packed<6, KIND>(dtab, st);
    case 5: return run_packed<8, KIND>(dtab, st);
    default: return 0;
  }
}
}  // namespace

int launch_packed(int bucket, int kind, const PackedTable* dtab, cudaStream_t st) {
  const int g = kind == 0 ? packed_kind<0>(bucket, dtab, st) : packed_kind<1>(bucket, dtab, st);
  if (g) launches_add(1);
  return g;
}

}  // namespace qcl
