// row_pass.cu — range (row, contiguous-axis) passes with the chirp-scaling phases.
//
// One CTA owns row_w(N) whole rows of the range-Doppler array (azimuth-frequency
// rows).  Per row, in registers:
//
//   x exp(j 2 pi phi_pro(j'))  ->  range FFT  ->  x exp(j 2 pi phi_mid(m))
//       ->  range IFFT  ->  x exp(j 2 pi phi_epi(j')) / N_r
//
// With (pro, mid, epi) = (H1, H2, H3) this is the middle of the focusing operator M;
// with the conjugates (H3*, H2*, H1*) it is the middle of G (Section III-C/D).
// In the ITA's range pass of M the pass first forms its input F_a r = F_a(S.Y) -
// F_a(S.G(X)) from the echo's azimuth transform and the residue column pass's output,
// with the partial sums of |F_a r|^2; at N_r = 8192 the CTA's row of F_a(S.Y) arrives
// by one bulk asynchronous copy into the (still unused) exchange buffer while the
// threads load the other operand, so the two reads overlap.
// j' = j - N_r/2 is the signed range-time bin, m the signed range-frequency bin;
// each phase is evaluated on the fly from per-row FP64-derived coefficients
// (phase.cuh), so the pass reads and writes each element exactly once.
#include "fft.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace csar {

// Rows of at least 1024 bins apply each phase as chains along the thread's elements
// (phase_chain, with per-row Gamma tables in shared memory); shorter rows, with many
// rows per CTA, keep the re-anchored recurrence (phase_ap).
template <int N>
constexpr bool kRowChains = N >= 1024;

// The residue form takes F_a(S.Y) by one bulk asynchronous copy at N_r = 8192 (one row
// per CTA); shorter rows load it in groups of 8 per thread, which keeps their register
// allocation free of spills.
template <int N>
constexpr bool kBulkY = N == 8192;

// Threads of a CTA with R values per thread.
__host__ __device__ constexpr int row_threads_r(int n, int r) { return n * row_w(n) / r; }

// RESID: the residue form (a.yf set), a separate instance so that the plain pass
// carries none of its code.  R: values per thread, which sets the radix schedule of the
// transforms (R = 32: 8192 = 8 x 32 x 32, two exchanges; R = 16: 2 x 16 x 16 x 16, three
// exchanges and twice the threads per row); the plan chooses (autotuner, CSAR_ROW_REGS).
// Block index of a CTA: the grid's own (read from the special register where it is
// used, which keeps it out of the register file) or a batch item's.
struct BlkOfGrid {
  __device__ __forceinline__ int operator()() const { return (int)blockIdx.x; }
};
struct BlkOfItem {
  int b;
  __device__ __forceinline__ int operator()() const { return b; }
};

template <int N, bool RESID, int R, class BLK>
__device__ __forceinline__ void row_body(const RowArgs& a, BLK blk) {
#include "row_body.inc"
}

// The per-pass kernel carries the statements itself (see col_pass.cuh): the hot passes
// keep their register allocation.
template <int N, bool RESID, int R = regs_for(N)>
__global__ void __launch_bounds__(row_threads_r(N, R), 2) k_row(RowArgs a) {
  const BlkOfGrid blk{};
#include "row_body.inc"
}

// Range passes of a batch of patches in one launch: CTA i runs row block items[i].unit of
// patch items[i].patch (row length items[i].n) with that patch's arguments.  Every row
// length runs 256 threads on 8192 values, so one launch serves every patch size.
template <bool RESID>
__global__ void __launch_bounds__(256, 2) k_row_batched(const RowArgs* __restrict__ args,
                                                        const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const RowArgs a = args[it.patch];
  switch (it.n) {
#define CSAR_CASE(N) \
  case N: row_body<N, RESID, regs_for(N)>(a, BlkOfItem{it.unit}); break;
    CSAR_BATCH_ROW_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: break;
  }
}

template <int N, int R = regs_for(N)>
static size_t row_smem() {
  using L = Layout<N, row_w(N), false>;
  return (size_t)L::kSmemElems * sizeof(float2) + (kTwLo + kTwHi) * sizeof(float2) +
         32 * sizeof(float) + 2 * sizeof(float2) +
         (kRowChains<N> ? (size_t)row_w(N) * 3 * R * sizeof(float2) : 0);
}

// The radix-16 schedule (16 values per thread) is built for rows of 1024 bins and more.
template <int N>
constexpr bool kRow16 = N >= 1024;

template <int N, int R>
static cudaError_t row_attrs_r() {
  cudaError_t e = cudaFuncSetAttribute(k_row<N, false, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)row_smem<N, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_row<N, true, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)row_smem<N, R>());
  return e;
}

template <int N, int R>
static cudaError_t row_launch_r(const RowArgs& a, cudaStream_t s) {
  const int grid = (a.n_rows + row_w(N) - 1) / row_w(N);
  if (a.yf) k_row<N, true, R><<<grid, row_threads_r(N, R), row_smem<N, R>(), s>>>(a);
  else k_row<N, false, R><<<grid, row_threads_r(N, R), row_smem<N, R>(), s>>>(a);
  return cudaGetLastError();
}

#define CSAR_ROW_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

cudaError_t row_set_attributes(int nr) {
  switch (nr) {
#define CSAR_CASE(N)                                                   \
  case N: {                                                            \
    cudaError_t e = row_attrs_r<N, regs_for(N)>();                     \
    if constexpr (kRow16<N>)                                           \
      if (e == cudaSuccess) e = row_attrs_r<N, (kRow16<N> ? 16 : regs_for(N))>(); \
    return e;                                                          \
  }
    CSAR_ROW_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

static size_t row_batched_smem() {
  size_t m = 0;
#define CSAR_CASE(N) m = row_smem<N, regs_for(N)>() > m ? row_smem<N, regs_for(N)>() : m;
  CSAR_BATCH_ROW_SIZES(CSAR_CASE)
#undef CSAR_CASE
  return m;
}

cudaError_t row_batched_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_row_batched<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)row_batched_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_row_batched<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)row_batched_smem());
  return e;
}

cudaError_t launch_row_batched(bool resid, const RowArgs* args, const BatchItem* items, int n_items,
                               cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  if (resid) k_row_batched<true><<<n_items, 256, row_batched_smem(), s>>>(args, items);
  else k_row_batched<false><<<n_items, 256, row_batched_smem(), s>>>(args, items);
  return cudaGetLastError();
}

cudaError_t launch_row(int nr, const RowArgs& a, cudaStream_t s) {
  switch (nr) {
#define CSAR_CASE(N)                                                                       \
  case N:                                                                                  \
    if constexpr (kRow16<N>)                                                               \
      if (a.regs == 16) return row_launch_r<N, (kRow16<N> ? 16 : regs_for(N))>(a, s);     \
    return row_launch_r<N, regs_for(N)>(a, s);
    CSAR_ROW_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace csar
