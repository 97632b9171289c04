// rda_pass.cu — the range pass of the range-Doppler operator pair (Section III-C,
// Eqs. (14)-(18), (22)): range compression, RCMC and the azimuth matched filter in one
// pass over the range-Doppler rows.
//
// Range compression acts along range with the same filter on every row, so it commutes
// with the azimuth transforms:
//   M = F_a^-1 P_eta C F_a F_r^-1 P_tau F_r = F_a^-1 [P_eta C F_r^-1 P_tau F_r] F_a,
//   G = M^H                                 = F_a^-1 [F_r^-1 P_tau^* F_r D P_eta^*] F_a,
// and each operator is a column FFT, this row pass, a column IFFT (three passes, like
// the chirp-scaling pair).  In the ITA the pass of M also takes the residue form of
// the chirp-scaling range pass (F_a r = F_a(S.Y) - input, with the partial sums of
// |F_a r|^2; F_a(S.Y) by a bulk asynchronous copy overlapping the other load).
// Per azimuth-frequency row, in registers and shared memory:
//   M:  range FFT, x P_tau, range IFFT / N_r, row staged in shared memory, every bin
//       tau interpolated from bins b..b+7 (b = floor(tau + dr) - 3, mod N_r) with
//       weights sinc(b + t - tau - dr), x P_eta(tau);
//   G:  x conj(P_eta), each bin added with the same weights onto the bins it is read
//       from in M (D = C^T), range FFT, x conj(P_tau), range IFFT / N_r.
// The transpose scatters without atomics: the first tap b(tau) rises by one per bin up
// to a rounding step (slope 1 + alpha, alpha >= 0), so bins 9 or more apart start
// 8-bin spans at least 8 apart, which are disjoint.
// Thread t holds the bins 16 t + c + j N_r / 2 (c < 16); the rounds (c, j) each
// update, in plain read-add-writes, one bin per thread; threads may drift up to 7
// rounds apart (a barrier every 8 rounds) without their spans meeting, and within a
// half row the spans cannot wrap onto each other while alpha < 1 - 18/N_r.
// Every accumulator therefore sums its terms in the fixed order of the rounds and G is
// deterministic.
// The migration dr = alpha (c0 + j') (alpha = 1/D - 1, c0 = 2 R_ref fs / c,
// j' = tau - N_r/2) is evaluated in double-float from FP64 per-row coefficients, so its
// fraction, which sets the weights, is accurate to ~1e-7 samples.
#include "fft.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace csar {

// First tap b of output bin tau and the fraction f: tau + dr = b + 3 + f, f in [0, 1).
__device__ __forceinline__ int rcmc_tap(const RcmcCoef& k, int tau, int nr, float* f) {
  const float fj = (float)(tau - nr / 2);
  const float p = k.al_hi * fj;
  const float e = fmaf(k.al_hi, fj, -p);              // exact error of the product
  const float n1 = rintf(k.a0_hi), n2 = rintf(p);
  const float fr = (k.a0_hi - n1) + (p - n2) + (k.a0_lo + e + k.al_lo * fj);
  const float fl = floorf(fr);
  const float fc = fr - fl;
  // a fraction a few 1e-8 under 1 (fr just below an integer) rounds to 1: that is the
  // next tap with fraction 0
  const bool up = fc >= 1.f;
  *f = up ? 0.f : fc;
  return tau + (int)n1 + (int)n2 + (int)fl - 3 + (up ? 1 : 0);
}

// Weights w[t] = sinc(m - f), m = t - 3, from one sinpi (sin(pi (m - f)) =
// -(-1)^m sin(pi f)) and one division: the eight reciprocals 1/(m - f) come from the
// reciprocal of their product (batch inversion: prefix products forward, the inverse
// carried back), a few ulp each.
__device__ __forceinline__ void rcmc_weights(float f, float (&w)[8]) {
  if (!(f > 1e-20f)) {      // f = 0 (and fractions too small to matter): the tap itself
#pragma unroll
    for (int t = 0; t < 8; ++t) w[t] = t == 3 ? 1.f : 0.f;
    return;
  }
  float d[8], pre[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) d[t] = (float)(t - 3) - f;
  pre[0] = d[0];
#pragma unroll
  for (int t = 1; t < 8; ++t) pre[t] = pre[t - 1] * d[t];
  float inv = sinpif(f) * 0.31830988618379067f / pre[7];   // (sin(pi f) / pi) / prod d
#pragma unroll
  for (int t = 7; t > 0; --t) {
    const float r = inv * pre[t - 1];                      // (sin(pi f) / pi) / d[t]
    w[t] = (t & 1) ? -r : r;                               // m = t - 3 odd <=> t even
    inv *= d[t];
  }
  w[0] = inv;
}

// Rows of at least 1024 bins apply the range filter as chains with per-row Gamma tables
// in shared memory; shorter rows use the re-anchored recurrence.
template <int N>
constexpr bool kRdaChains = N >= 1024;

template <int N>
constexpr int rda_gamma_elems() { return kRdaChains<N> ? row_w(N) * regs_for(N) : 0; }

// Accumulator of the transpose: one pad slot per 16 bins, so the bins of a round (16
// apart) fall on different banks.
__device__ __forceinline__ int rda_pad(int i) { return i + (i >> 4); }

// acc[pad(b + u mod N)] += w[u] x, u < 8.  Away from the row's end the 8 slots are
// pad(b) + u, plus one from the first tap that crosses a pad slot on.  The 8 slots are
// distinct: all are read before any is written, so the reads overlap.
template <int N>
__device__ __forceinline__ void rda_scatter8(float2* acc, int b, float2 x, const float (&wt)[8]) {
  const int bm = b & (N - 1);
  int ad[8];
  if (bm <= N - 8) {
    const int base = rda_pad(bm);
    const int uc = 16 - (bm & 15);
#pragma unroll
    for (int u = 0; u < 8; ++u) ad[u] = base + u + (u >= uc ? 1 : 0);
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) ad[u] = rda_pad((b + u) & (N - 1));
  }
  float2 y[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) y[u] = acc[ad[u]];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    y[u].x = fmaf(x.x, wt[u], y[u].x);
    y[u].y = fmaf(x.y, wt[u], y[u].y);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[ad[u]] = y[u];
}

// sum_u w[u] row[b + u mod N], u < 8 (plain row).
template <int N>
__device__ __forceinline__ float2 rda_gather8(const float2* row, int b, const float (&wt)[8]) {
  const int bm = b & (N - 1);
  float2 y = make_float2(0.f, 0.f);
  if (bm <= N - 8) {
    const float2* p = row + bm;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float2 x = p[u];
      y.x = fmaf(x.x, wt[u], y.x);
      y.y = fmaf(x.y, wt[u], y.y);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float2 x = row[(b + u) & (N - 1)];
      y.x = fmaf(x.x, wt[u], y.x);
      y.y = fmaf(x.y, wt[u], y.y);
    }
  }
  return y;
}

template <int N, int MODE>
__global__ void __launch_bounds__(row_threads(N), 2) k_row_rda(RdaArgs a) {
  constexpr int WR = row_w(N);
  constexpr int R = regs_for(N);
  constexpr int QR = N / R;
  constexpr int NT = row_threads(N);
  using L = Layout<N, WR, false>;
  static_assert(WR * (N + N / 16) <= L::kSmemElems, "accumulator rows exceed the exchange buffer");
  extern __shared__ float2 smem[];
  if (a.gate && *a.gate != a.gate_val) return;
  float2* sm = smem;                         // transform exchanges, and the staged rows
  float2* tw = smem + L::kSmemElems;
  float* red = reinterpret_cast<float*>(tw + kTwLo + kTwHi);   // 32 floats
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tw + kTwLo + kTwHi + 16);
  float2* gam = tw + kTwLo + kTwHi + 18;      // Gamma tables of the range filter, per row
  const int tid = threadIdx.x;
  if (MODE == 0 && a.yf && tid == 0) {
    // residue form: this CTA's rows of F_a(S.Y) by one bulk asynchronous copy into the
    // still unused exchange buffer, while the threads load the other operand
    const int row0 = blockIdx.x * WR;
    const int live_rows = a.n_rows - row0 < WR ? a.n_rows - row0 : WR;
    const uint32_t mb = smem_addr(mbar);
    mbar_init(mb, 1u);
    bulk_load_armed(smem_addr(sm), a.yf + (size_t)row0 * N, (uint32_t)(live_rows * N * sizeof(float2)), mb);
  }
  load_twiddles(tw, a.tw);
  const int w = tid / QR, t = tid % QR;
  const int row = blockIdx.x * WR + w;
  const bool live = row < a.n_rows;
  const int rw = live ? row : 0;
  float2* rp = a.data + (size_t)rw * N;
  const RcmcCoef k = a.rc[rw];
  const PhaseCoef mid = a.rg[rw].mid;
  if constexpr (kRdaChains<N>) {
    for (int i = tid; i < WR * R; i += NT) {
      const int r2 = blockIdx.x * WR + i / R;
      gam[i] = phase_gamma(a.rg[r2 < a.n_rows ? r2 : 0].mid, QR, i % R);
    }
  }
  const float2* gw = gam + w * R;
  float2 v[R];
  if constexpr (MODE == 1) {
    // G: thread t takes bins 16 t + c + j N/2 (c < 16) one per round, reading each from
    // global memory as it goes (the row's lines stay in L1 across the 16 rounds), times
    // conj(P_eta) (coefficients of G's rows) as chains of 16 from two exact evaluations
    constexpr int NJ = R / 16;
    float2* acc = sm + w * (N + N / 16);
    for (int i = t; i < N + N / 16; i += QR) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int j = 0; j < NJ; ++j) {
      const int tau0 = 16 * t + j * (N / 2);
      float2 p = phase_eval(k.az, tau0 - N / 2, 1.f);
      const float2 e1 = phase_eval(k.az, tau0 + 1 - N / 2, 1.f);
      const float2 lam = make_float2(fmaf(e1.x, p.x, e1.y * p.y), fmaf(e1.y, p.x, -e1.x * p.y));
#pragma unroll 1
      for (int c = 0; c < 16; ++c) {
        // threads t < t' at rounds c, c' with |c - c'| <= 7 hold bins at least 9 apart,
        // whose first taps differ by at least 8: disjoint spans.  A barrier every 8
        // rounds keeps every thread within 7 rounds of the others.
        if ((c & 7) == 0) __syncthreads();
        const int tau = tau0 + c;
        if (c == 1) p = e1;
        else if (c > 1) p = cmul(p, lam);
        const float2 x = live ? cmul(__ldg(&rp[tau]), p) : make_float2(0.f, 0.f);
        float f;
        const int b = rcmc_tap(k, tau, N, &f);
        float wt[8];
        rcmc_weights(f, wt);
        rda_scatter8<N>(acc, b, x, wt);
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = acc[rda_pad(t + s * QR)];
  } else {
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = live ? __ldcs(&rp[t + s * QR]) : make_float2(0.f, 0.f);
    if (a.yf) {
      // residue form: v = F_a(S.Y) - v, its squared norm and a finiteness check
      __syncthreads();   // the mbarrier is initialised
      const uint32_t mb = smem_addr(mbar);
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
      float sq = 0.f;
      bool bad = false;
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const float2 y = live ? ys[t + s * QR] : make_float2(0.f, 0.f);
        v[s] = csub(y, v[s]);
        sq += cabs2(v[s]);
        bad |= !(isfinite(v[s].x) && isfinite(v[s].y));
      }
      if (bad) atomicOr(&a.ctl->err, kErrNonfinite);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if ((tid & 31) == 0) red[tid >> 5] = sq;
      __syncthreads();
      if (tid == 0) {
        float tot = 0.f;
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) tot += red[i];
        a.partial[blockIdx.x] = tot * a.resid_scale;
      }
    }
    __syncthreads();   // twiddles and Gamma tables
  }
  // range compression: FFT, x P_tau (or conj), IFFT / N_r; range-frequency bin of v[s]
  // is t + s QR for s < R/2 and t + (s - R) QR above
  fft<N, false, L, false>(v, sm, tw, t, w);
  if (a.rtab) {
    // a recorded pulse (Section III-D): the filter is a table over the range-frequency
    // bins, FFT order, so v[s] (bin t + s QR modulo N) takes entry t + s QR
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = cmul(v[s], __ldg(&a.rtab[t + s * QR]));
  } else if constexpr (kRdaChains<N>) {
    phase_chain<R, 0, R / 2>(v, mid, t, QR, 1.f, gw);
    phase_chain<R, R / 2, R>(v, mid, t - (R / 2) * QR, QR, 1.f, gw);
  } else {
    const float2 dd = phase_second_diff(mid, QR);
    phase_ap<R, 0, R / 2>(v, mid, t, QR, 1.f, dd);
    phase_ap<R, R / 2, R>(v, mid, t - (R / 2) * QR, QR, 1.f, dd);
  }
  fft<N, true, L, false>(v, sm, tw, t, w);
  if constexpr (MODE == 0) {
    // M: C then P_eta on the staged row, one bin per step, stored as it is formed
    // (P_eta, a linear phase, as chains of 16 from two exact evaluations each)
    float2* rs = sm + w * N;
    __syncthreads();
#pragma unroll
    for (int s = 0; s < R; ++s) rs[t + s * QR] = cscale(v[s], a.scale);
    __syncthreads();
    float2 p = make_float2(1.f, 0.f), e1 = p, lam = p;
#pragma unroll 4
    for (int s = 0; s < R; ++s) {
      const int tau = t + s * QR;
      if ((s & 15) == 0) {
        p = phase_eval(k.az, tau - N / 2, 1.f);
        e1 = phase_eval(k.az, tau + QR - N / 2, 1.f);
        lam = make_float2(fmaf(e1.x, p.x, e1.y * p.y), fmaf(e1.y, p.x, -e1.x * p.y));
      } else {
        p = (s & 15) == 1 ? e1 : cmul(p, lam);
      }
      float f;
      const int b = rcmc_tap(k, tau, N, &f);
      float wt[8];
      rcmc_weights(f, wt);
      const float2 y = rda_gather8<N>(rs, b, wt);
      if (live) __stcs(&rp[tau], cmul(y, p));
    }
  } else {
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = cscale(v[s], a.scale);
    if (live) {
#pragma unroll
      for (int s = 0; s < R; ++s) __stcs(&rp[t + s * QR], v[s]);
    }
  }
}

template <int N>
static size_t rda_smem() {
  using L = Layout<N, row_w(N), false>;
  return (size_t)L::kSmemElems * sizeof(float2) + (kTwLo + kTwHi + 18) * sizeof(float2) +
         (size_t)rda_gamma_elems<N>() * sizeof(float2);
}

#define CSAR_RDA_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

cudaError_t rda_set_attributes(int nr) {
  switch (nr) {
#define CSAR_CASE(N)                                                                             \
  case N: {                                                                                      \
    cudaError_t e = cudaFuncSetAttribute(k_row_rda<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)rda_smem<N>());                                   \
    if (e == cudaSuccess)                                                                        \
      e = cudaFuncSetAttribute(k_row_rda<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                               (int)rda_smem<N>());                                             \
    return e;                                                                                    \
  }
    CSAR_RDA_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_row_rda(int nr, const RdaArgs& a, bool is_g, cudaStream_t s) {
  switch (nr) {
#define CSAR_CASE(N)                                                                 \
  case N: {                                                                          \
    const int grid = (a.n_rows + row_w(N) - 1) / row_w(N);                           \
    if (is_g) k_row_rda<N, 1><<<grid, row_threads(N), rda_smem<N>(), s>>>(a);        \
    else k_row_rda<N, 0><<<grid, row_threads(N), rda_smem<N>(), s>>>(a);             \
    return cudaGetLastError();                                                       \
  }
    CSAR_RDA_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace csar
