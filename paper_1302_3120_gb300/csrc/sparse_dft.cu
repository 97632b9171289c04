// sparse_dft.cu — azimuth DFT of the K-sparse iterate by direct summation.
//
// The first column pass of G(X) transforms X^(i), which has at most K nonzeros
// (K = 20000 on 8192 x 8192: ~2.4 per column).  For a group of 16 columns holding
// few entries, X[k, col] = sum_e x_e W_N^(k row_e) is cheaper than an N-point FFT:
// the group's entries are bucketed by column in shared memory and a warp accumulates a
// column's entries for 8 output rows per lane (the twiddle advances by W_N^(32 row_e) per
// row step from an exact table start).  Entry counts per column vary (Poisson, mean ~2.4),
// so two chunks of rows are in flight, one per group of 8 warps, and a warp takes a
// heaviest-with-lightest pair of columns of its chunk.  Each 256 x 16 block is
// staged in shared memory and written to global memory by one tensor copy
// (cp.async.bulk.tensor, 128-byte rows, 128-byte swizzle so that the column-wise
// staging writes spread over the banks), one staging block per chunk in flight; the
// copies of a chunk pair overlap the lightest columns' sums of the next pair, and the
// pass issues no per-element store instructions.
// Groups with more entries are left to the FFT path (k_col, COL_SPARSE_FWD).
#include <cuda.h>

#include "fft.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace csar {

constexpr int kSdThreads = 512;               // 16 warps = 16 columns
constexpr int kSdRows = kDirectRows;          // output rows per chunk (8 per lane)
constexpr int kSdBlkBytes = kSdRows * kDirectCols * (int)sizeof(float2);   // 32 KiB staging block
// dynamic shared memory: two staging blocks (1024-byte aligned for the swizzle), then the
// twiddles and the entry lists
constexpr size_t kSdSmem = 1024 + 2 * kSdBlkBytes + (kTwLo + kTwHi) * sizeof(float2) +
                           kDirectMaxEntries * (2 * sizeof(uint32_t) + sizeof(float2)) +
                           (2 * kDirectCols + 1) * sizeof(int);

// Byte offset of element (r, c) of a staging block: rows of 128 bytes whose 16-byte
// chunks are permuted by XOR with r mod 8 (the tensor map's 128-byte swizzle).
__device__ __forceinline__ uint32_t blk_off(int r, int c) {
  return (uint32_t)(r * 128 + (((c >> 1) ^ (r & 7)) << 4) + ((c & 1) << 3));
}

template <int N>
__global__ void __launch_bounds__(kSdThreads) k_sparse_dft(const __grid_constant__ CUtensorMap omap, ColArgs a,
                                                           int col_tile, int chunks_per_cta) {
  extern __shared__ unsigned char sd_smem[];
  const uint32_t sbase = (smem_addr(sd_smem) + 1023u) & ~1023u;
  unsigned char* const blk = sd_smem + (sbase - smem_addr(sd_smem));
  float2* tw = reinterpret_cast<float2*>(blk + 2 * kSdBlkBytes);
  uint32_t* e_key = reinterpret_cast<uint32_t*>(tw + kTwLo + kTwHi);   // flat index, then (column, row) key
  uint32_t* e_row = e_key + kDirectMaxEntries;
  float2* e_val = reinterpret_cast<float2*>(e_row + kDirectMaxEntries);
  int* col_beg = reinterpret_cast<int*>(e_val + kDirectMaxEntries);
  int* col_order = col_beg + kDirectCols + 1;   // columns by entry count, heaviest first
  if (a.gate && *a.gate != a.gate_val) return;
  const int grp = blockIdx.x;
  const int bpg = kDirectCols / col_tile > 0 ? kDirectCols / col_tile : 1;
  const int n_buckets = a.nr / col_tile;
  const int b1 = (grp + 1) * bpg < n_buckets ? (grp + 1) * bpg : n_buckets;
  const uint32_t e0 = a.xs_off[grp * bpg], e1 = a.xs_off[b1];
  const int ne = (int)(e1 - e0);
  if (ne > kDirectMaxEntries) {               // FFT path
    if (threadIdx.x == 0 && a.h_dense) cudaGraphSetConditional(a.h_dense, 1u);
    return;
  }
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
  if (tid < kDirectCols) {
    // position of column tid in the order by entry count (descending; ties by column)
    const int mine = col_beg[tid + 1] - col_beg[tid];
    int pos = 0;
    for (int cc = 0; cc < kDirectCols; ++cc) {
      const int n = col_beg[cc + 1] - col_beg[cc];
      pos += (n > mine) || (n == mine && cc < tid);
    }
    col_order[pos] = tid;
  }
  __syncthreads();
  // Two chunks in flight, one per group of 8 warps; warp w sums the (w % 8)-th heaviest
  // and the (w % 8)-th lightest column of its group's chunk (8 rows per lane each), so a
  // chunk pair waits for the heaviest column pair instead of one chunk for the heaviest
  // column.
  const int w = tid >> 5, lane = tid & 31;
  const int g = w >> 3;
  const int c_light = col_order[kDirectCols - 1 - (w & 7)], c_heavy = col_order[w & 7];
  constexpr int kScale = kTwN / N;            // W_N^m = W_8192^(m * kScale)
  const bool in_range = CSAR_CHECK((size_t)col0 + kDirectCols - 1, (size_t)a.nr, a.ctl);
  auto column_sum = [&](int cl, int k0, float2 (&acc)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
    const int i1 = col_beg[cl + 1];
    for (int i = col_beg[cl]; i < i1; ++i) {   // uniform per warp
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
  };
  for (int ch0 = 0; ch0 < chunks_per_cta; ch0 += 2) {
    const int ch = ch0 + g;
    const bool act = ch < chunks_per_cta;
    const int k0 = (blockIdx.y * chunks_per_cta + ch) * kSdRows;
    unsigned char* const bk = blk + g * kSdBlkBytes;
    float2 acc[8];
    if (act) column_sum(c_light, k0, acc);
    // both staging blocks are free once the copies of the previous chunk pair have read them
    if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();
    if (act) {
#pragma unroll
      for (int j = 0; j < 8; ++j) *reinterpret_cast<float2*>(bk + blk_off(lane + 32 * j, c_light)) = acc[j];
      column_sum(c_heavy, k0, acc);
#pragma unroll
      for (int j = 0; j < 8; ++j) *reinterpret_cast<float2*>(bk + blk_off(lane + 32 * j, c_heavy)) = acc[j];
    }
    // the staging writes become visible to the tensor copies (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && in_range) {
      for (int gg = 0; gg < 2 && ch0 + gg < chunks_per_cta; ++gg) {
        const int kk = (blockIdx.y * chunks_per_cta + ch0 + gg) * kSdRows;
        if (!CSAR_CHECK((size_t)kk + kSdRows - 1, (size_t)N, a.ctl)) continue;
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     ::"l"(&omap), "r"(col0), "r"(kk), "r"(sbase + (uint32_t)(gg * kSdBlkBytes))
                     : "memory");
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  // the copies complete (their writes performed) before the CTA's shared memory is released
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <int N>
static cudaError_t sd_attrs() {
  return cudaFuncSetAttribute(k_sparse_dft<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSdSmem);
}

cudaError_t sparse_dft_set_attributes(int na) {
  switch (na) {
    case 256: return sd_attrs<256>();
    case 512: return sd_attrs<512>();
    case 1024: return sd_attrs<1024>();
    case 2048: return sd_attrs<2048>();
    case 4096: return sd_attrs<4096>();
    case 8192: return sd_attrs<8192>();
    default: return cudaSuccess;
  }
}

bool sparse_dft_applies(int na, int nr) { return nr >= kDirectCols && na >= kSdRows; }

cudaError_t launch_sparse_dft(int na, const ColArgs& a, int col_tile, cudaStream_t s) {
  if (!sparse_dft_applies(na, a.nr)) return cudaSuccess;   // small grids: FFT path only
  CUtensorMap omap;
  if (cudaError_t e = encode_map(&omap, a.out, na, a.nr, kDirectCols, kSdRows, true)) return e;
  const int chunks = na / kSdRows;
  const int split = chunks >= 8 ? chunks / 8 : 1;
  const dim3 grid(a.nr / kDirectCols, split);
  const int per = chunks / split;
  switch (na) {
#define CSAR_SD(NA) \
  case NA: k_sparse_dft<NA><<<grid, kSdThreads, kSdSmem, s>>>(omap, a, col_tile, per); break;
    CSAR_SD(256) CSAR_SD(512) CSAR_SD(1024) CSAR_SD(2048) CSAR_SD(4096) CSAR_SD(8192)
#undef CSAR_SD
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace csar
