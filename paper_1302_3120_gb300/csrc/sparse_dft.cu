// sparse_dft.cu — azimuth DFT of the K-sparse iterate by direct summation.
//
// The first column pass of G(X) transforms X^(i), which has at most K nonzeros
// (K = 20000 on 8192 x 8192: ~2.4 per column).  For a group of 16 columns holding
// few entries, X[k, col] = sum_e x_e W_N^(k row_e) is cheaper than an N-point FFT:
// the group's entries are bucketed by column in shared memory, one warp per column
// accumulates its own entries for 8 output rows per lane (the twiddle advances by
// W_N^(32 row_e) per row step from an exact table start), and a 256 x 16 block is
// staged in shared memory and written as 128-byte row segments.
// Groups with more entries are left to the FFT path (k_col, COL_SPARSE_FWD).
#include "fft.cuh"
#include "internal.h"

namespace csar {

constexpr int kSdThreads = 512;               // 16 warps = 16 columns
constexpr int kSdRows = kDirectRows;          // output rows per chunk (8 per lane)

template <int N>
__global__ void __launch_bounds__(kSdThreads) k_sparse_dft(ColArgs a, int col_tile, int chunks_per_cta) {
  __shared__ float2 tw[kTwLo + kTwHi];
  __shared__ uint32_t e_key[kDirectMaxEntries];   // flat index, then (column, row) order key
  __shared__ uint32_t e_row[kDirectMaxEntries];
  __shared__ float2 e_val[kDirectMaxEntries];
  __shared__ int col_beg[kDirectCols + 1];
  __shared__ float2 blk[kSdRows][kDirectCols + 1];
  if (a.gate && *a.gate != a.gate_val) return;
  const int grp = blockIdx.x;
  const int bpg = kDirectCols / col_tile > 0 ? kDirectCols / col_tile : 1;
  const int n_buckets = a.nr / col_tile;
  const int b1 = (grp + 1) * bpg < n_buckets ? (grp + 1) * bpg : n_buckets;
  const uint32_t e0 = a.xs_off[grp * bpg], e1 = a.xs_off[b1];
  const int ne = (int)(e1 - e0);
  if (ne > kDirectMaxEntries) return;         // FFT path
  const int tid = threadIdx.x;
  load_twiddles(tw, a.tw);
  const int col0 = grp * kDirectCols;
  // Entries ordered by (column, row): each warp then walks only its own column, and
  // the order (hence the summation order) does not depend on the list order, which
  // comes from atomics: the pass is deterministic.
  uint32_t key = 0u;
  float2 val = make_float2(0.f, 0.f);
  if (tid < ne) {
    const uint32_t idx = a.xs_idx[e0 + tid];
    const uint32_t row = idx / (uint32_t)a.nr;
    uint32_t cl = idx % (uint32_t)a.nr - (uint32_t)col0;
    val = a.xs_val[e0 + tid];
    if (!CSAR_CHECK(cl, kDirectCols, a.ctl) || !CSAR_CHECK(row, N, a.ctl)) {
      cl = 0u;
      val = make_float2(0.f, 0.f);
    }
    key = (cl << 16) | row;                     // row < 2^13, column < 16
    e_key[tid] = key;
  }
  __syncthreads();
  if (tid < ne) {
    int rank = 0;
    for (int j = 0; j < ne; ++j) rank += e_key[j] < key;
    e_row[rank] = key & 0xffffu;
    e_val[rank] = val;
  }
  if (tid <= kDirectCols) {
    int cnt = 0;
    for (int j = 0; j < ne; ++j) cnt += (int)(e_key[j] >> 16) < tid;
    col_beg[tid] = cnt;
  }
  __syncthreads();
  const int w = tid >> 5, lane = tid & 31;
  const int i0 = col_beg[w], i1 = col_beg[w + 1];
  constexpr int kScale = kTwN / N;            // W_N^m = W_8192^(m * kScale)
  for (int ch = 0; ch < chunks_per_cta; ++ch) {
    const int k0 = (blockIdx.y * chunks_per_cta + ch) * kSdRows;
    float2 acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int i = i0; i < i1; ++i) {           // uniform per warp
      const uint32_t row = e_row[i];
      const float2 x = e_val[i];
      float2 e = cmul(x, twiddle_tab<false>(tw, (int)(((uint32_t)(k0 + lane) * row) % N) * kScale));
      const float2 st = twiddle_tab<false>(tw, (int)((32u * row) % N) * kScale);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[j] = cadd(acc[j], e);
        e = cmul(e, st);
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j) blk[lane + 32 * j][w] = acc[j];
    __syncthreads();
    // 256 rows x 16 columns: each half-warp writes one 128-byte row segment
    for (int i = tid; i < kSdRows * kDirectCols; i += kSdThreads) {
      const int r = i / kDirectCols, c = i % kDirectCols;
      const size_t gi = (size_t)(k0 + r) * a.nr + col0 + c;
      if (CSAR_CHECK(gi, (size_t)N * a.nr, a.ctl)) __stcs(&a.out[gi], blk[r][c]);
    }
  }
}

cudaError_t launch_sparse_dft(int na, const ColArgs& a, int col_tile, cudaStream_t s) {
  if (a.nr < kDirectCols || na < kSdRows) return cudaSuccess;   // small grids: FFT path only
  const int chunks = na / kSdRows;
  const int split = chunks >= 8 ? chunks / 8 : 1;
  const dim3 grid(a.nr / kDirectCols, split);
  const int per = chunks / split;
  switch (na) {
    case 256: k_sparse_dft<256><<<grid, kSdThreads, 0, s>>>(a, col_tile, per); break;
    case 512: k_sparse_dft<512><<<grid, kSdThreads, 0, s>>>(a, col_tile, per); break;
    case 1024: k_sparse_dft<1024><<<grid, kSdThreads, 0, s>>>(a, col_tile, per); break;
    case 2048: k_sparse_dft<2048><<<grid, kSdThreads, 0, s>>>(a, col_tile, per); break;
    case 4096: k_sparse_dft<4096><<<grid, kSdThreads, 0, s>>>(a, col_tile, per); break;
    case 8192: k_sparse_dft<8192><<<grid, kSdThreads, 0, s>>>(a, col_tile, per); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace csar
