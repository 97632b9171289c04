// col_batched.cu — one launch of a column pass over every patch of a batch.
//
// The launch is a grid of thread-block clusters of kBatchCluster CTAs (256 threads,
// 4096 complex values each, the same shared memory for every azimuth length), one
// cluster per work item.  An item is a group of tiles of one patch: the length-N_a
// column transform of a tile takes P_e(N_a) CTAs (the plan's column configuration for
// that length: 1 CTA up to 1024 rows, 2 at 2048, 4 at 4096), so a cluster holds
// kBatchCluster / P_e tiles side by side, each on its own CTAs, with its own exchange
// mbarriers and peers (cluster ranks rank0 .. rank0 + P_e - 1).  The statements per CTA
// are those of the per-patch kernel (col_body.inc); a CTA past the patch's last tile
// leaves at once.
#include "col_pass.cuh"

namespace csar {

constexpr int kBatchCluster = 4;
constexpr int kBatchE = 4096;

// CTAs per tile in a batch, by azimuth length (0: not served by the batched passes).
__host__ __device__ constexpr int batch_col_p(int na) {
  return na == 512 || na == 1024 ? 1 : (na == 2048 ? 2 : (na == 4096 ? 4 : 0));
}

template <int N, int MODE>
__device__ __forceinline__ void col_item(const ColArgs& a, int unit, int rank) {
  constexpr int P = batch_col_p(N);
  constexpr int W = ColCfg<N, P, kBatchE>::W;
  const int sub = rank / P, c = rank % P;
  const int tile = unit * (kBatchCluster / P) + sub;
  if (tile >= a.nr / W) return;   // uniform per tile group
  col_body<N, P, kBatchE, MODE>(a, ColOfItem{c, tile, rank - c, tile * P + c});
}

template <int MODE>
__global__ void __launch_bounds__(ColCfg<1024, 1, kBatchE>::NT, col_ctas_per_sm(kBatchE))
    k_col_batched(const ColArgs* __restrict__ args, const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x / kBatchCluster];
  const int rank = (int)(blockIdx.x % kBatchCluster);
  const ColArgs& a = args[it.patch];
  switch (it.n) {
#define CSAR_CASE(N) \
  case N: col_item<N, MODE>(a, it.unit, rank); break;
    CSAR_BATCH_COL_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: break;
  }
}

template <int MODE>
static size_t col_batched_smem() {
  size_t m = 0;
#define CSAR_CASE(N)                                                                       \
  m = col_smem<N, batch_col_p(N), kBatchE>(MODE) > m ? col_smem<N, batch_col_p(N), kBatchE>(MODE) : m;
  CSAR_BATCH_COL_SIZES(CSAR_CASE)
#undef CSAR_CASE
  return m;
}

template <int MODE>
static cudaError_t col_batched_attr() {
  return cudaFuncSetAttribute(k_col_batched<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)col_batched_smem<MODE>());
}

template <int MODE>
static cudaError_t col_batched_launch(const ColArgs* args, const BatchItem* items, int n_items,
                                      cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_items * kBatchCluster);
  cfg.blockDim = dim3(ColCfg<1024, 1, kBatchE>::NT);
  cfg.dynamicSmemBytes = col_batched_smem<MODE>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBatchCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_col_batched<MODE>, args, items);
}

int batch_col_cluster(int na) { return batch_col_p(na); }
bool batch_member_ok(int na, int nr) {
  bool row = false;
#define CSAR_CASE(N) row = row || nr == N;
  CSAR_BATCH_ROW_SIZES(CSAR_CASE)
#undef CSAR_CASE
  return row && batch_col_p(na) > 0;
}
int batch_col_tiles_per_item(int na) { return batch_col_p(na) ? kBatchCluster / batch_col_p(na) : 0; }

cudaError_t col_batched_set_attributes() {
  cudaError_t e = col_batched_attr<COL_SPARSE_FWD>();
  if (e == cudaSuccess) e = col_batched_attr<COL_RESID>();
  if (e == cudaSuccess) e = col_batched_attr<COL_SELECT>();
  if (e == cudaSuccess) e = col_batched_attr<COL_REPASS>();
  return e;
}

cudaError_t launch_col_batched(ColMode mode, const ColArgs* args, const BatchItem* items, int n_items,
                               cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  switch (mode) {
    case COL_SPARSE_FWD: return col_batched_launch<COL_SPARSE_FWD>(args, items, n_items, s);
    case COL_RESID: return col_batched_launch<COL_RESID>(args, items, n_items, s);
    case COL_SELECT: return col_batched_launch<COL_SELECT>(args, items, n_items, s);
    case COL_REPASS: return col_batched_launch<COL_REPASS>(args, items, n_items, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace csar
