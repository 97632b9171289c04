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
template <int N, bool RESID, int R = regs_for(N)>
__global__ void __launch_bounds__(row_threads_r(N, R), 2) k_row(RowArgs a) {
  constexpr int WR = row_w(N);
  constexpr int QR = N / R;
  constexpr int NTR = row_threads_r(N, R);
  using L = Layout<N, WR, false>;
  extern __shared__ float2 smem[];
  if (a.gate && *a.gate != a.gate_val) return;
  float2* sm = smem;
  float2* tw = smem + L::kSmemElems;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tw + kTwLo + kTwHi + 16);   // after 32 floats of reduction scratch
  float2* gam = tw + kTwLo + kTwHi + 18;
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * WR;
  if (RESID && kBulkY<N> && tid == 0) {
    // rows row0 .. row0 + live_rows - 1 of F_a(S.Y) into the exchange buffer, plain order
    const int live_rows = a.n_rows - row0 < WR ? a.n_rows - row0 : WR;
    const uint32_t mb = smem_addr(mbar);
    mbar_init(mb, 1u);
    bulk_load_armed(smem_addr(sm), a.yf + (size_t)row0 * N, (uint32_t)(live_rows * N * sizeof(float2)), mb);
  }
  load_twiddles(tw, a.tw);
  const int w = tid / QR, t = tid % QR;
  const int row = row0 + w;
  const bool live = row < a.n_rows;
  const RowCoef* cp = a.coef + (live ? row : 0);
  float2* rp = a.data + (size_t)(live ? row : 0) * N;
  const float2* sp = a.src ? a.src + (size_t)(live ? row : 0) * N : rp;
  float2 v[R];
  const bool ok_row = !live || CSAR_CHECK((size_t)row * N + (N - 1), (size_t)a.n_rows * N, a.ctl);
#pragma unroll
  for (int s = 0; s < R; ++s) v[s] = live && ok_row ? __ldcs(&sp[t + s * QR]) : make_float2(0.f, 0.f);
  if constexpr (kRowChains<N>) {
    // Gamma tables of this CTA's rows for the three phases: gam[(row*3 + phase)*R + u]
    for (int i = tid; i < WR * 3 * R; i += NTR) {
      const int rw = blockIdx.x * WR + i / (3 * R);
      const RowCoef& rc = a.coef[rw < a.n_rows ? rw : 0];
      const int ph = (i / R) % 3;
      gam[i] = phase_gamma(ph == 0 ? rc.pro : (ph == 1 ? rc.mid : rc.epi), QR, i % R);
    }
    __syncthreads();
  }
  const float2* gw = gam + w * 3 * R;
  if constexpr (RESID) {
    // residue form: v = F_a(S.Y) - v, its squared norm and a finiteness check
    float acc = 0.f;
    bool bad = false;
    if constexpr (kBulkY<N>) {
      const uint32_t mb = smem_addr(mbar);   // initialised before the Gamma-table barrier
      bool landed = mbar_wait_for(mb, 0u, 1000000000ull);
      if (!landed) {
        // the copy did not land within a second: report it, and give it one more second
        atomicOr(&a.ctl->err, kErrTimeout);
        landed = mbar_wait_for(mb, 0u, 1000000000ull);
      }
      // if any thread still saw no completion, the whole CTA leaves without touching the
      // buffer again (the latched error marks the result invalid)
      if (__syncthreads_or(!landed)) return;
      const float2* ys = sm + w * N;
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const float2 y = live ? ys[t + s * QR] : make_float2(0.f, 0.f);
        v[s] = csub(y, v[s]);
        acc += cabs2(v[s]);
        bad |= !(isfinite(v[s].x) && isfinite(v[s].y));
      }
    } else {
      const float2* yp = a.yf + (size_t)(live ? row : 0) * N;
      constexpr int kG = R >= 8 ? 8 : R;   // loads in flight per group (register pressure)
#pragma unroll
      for (int g0 = 0; g0 < R; g0 += kG) {
        float2 y[kG];
#pragma unroll
        for (int j = 0; j < kG; ++j) y[j] = live ? __ldcs(&yp[t + (g0 + j) * QR]) : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kG; ++j) {
          v[g0 + j] = csub(y[j], v[g0 + j]);
          acc += cabs2(v[g0 + j]);
          bad |= !(isfinite(v[g0 + j].x) && isfinite(v[g0 + j].y));
        }
      }
    }
    if (bad) atomicOr(&a.ctl->err, kErrNonfinite);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    float* red = reinterpret_cast<float*>(tw + kTwLo + kTwHi);
    constexpr int kWarps = NTR / 32;
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      float tot = 0.f;
#pragma unroll
      for (int i = 0; i < kWarps; ++i) tot += red[i];
      a.partial[blockIdx.x] = tot * a.resid_scale;
    }
  }
  if constexpr (kRowChains<N>) {
    phase_chain<R, 0, R>(v, cp->pro, t - N / 2, QR, 1.f, gw);
  } else {
    const PhaseCoef c = cp->pro;
    phase_ap<R, 0, R>(v, c, t - N / 2, QR, 1.f, phase_second_diff(c, QR));
  }
  // The range IFFT runs as the forward FFT of the conjugate (unnormalised IFFT(u) =
  // conj(FFT(conj(u))); conjugation commutes exactly with every rounded operation, so
  // the result is the same), which lets one copy of the FFT code serve both transforms
  // in a rolled loop: half the instruction footprint of two unrolled transforms.
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    fft<N, false, L, false, R>(v, sm, tw, t, w);
    if (pass == 1) break;
    // range-frequency bin of v[s]: t + s*QR for s < R/2, t + (s - R)*QR above
    if constexpr (kRowChains<N>) {
      phase_chain<R, 0, R / 2>(v, cp->mid, t, QR, 1.f, gw + R);
      phase_chain<R, R / 2, R>(v, cp->mid, t - (R / 2) * QR, QR, 1.f, gw + R);
    } else {
      const PhaseCoef c = cp->mid;
      const float2 dd = phase_second_diff(c, QR);
      phase_ap<R, 0, R / 2>(v, c, t, QR, 1.f, dd);
      phase_ap<R, R / 2, R>(v, c, t - (R / 2) * QR, QR, 1.f, dd);
    }
#pragma unroll
    for (int s = 0; s < R; ++s) v[s].y = -v[s].y;
  }
#pragma unroll
  for (int s = 0; s < R; ++s) v[s].y = -v[s].y;
  if constexpr (kRowChains<N>) {
    phase_chain<R, 0, R>(v, cp->epi, t - N / 2, QR, a.scale, gw + 2 * R);
  } else {
    const PhaseCoef c = cp->epi;
    phase_ap<R, 0, R>(v, c, t - N / 2, QR, a.scale, phase_second_diff(c, QR));
  }
  if (live && ok_row) {
#pragma unroll
    for (int s = 0; s < R; ++s) __stcs(&rp[t + s * QR], v[s]);
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
