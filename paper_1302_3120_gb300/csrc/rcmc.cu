// rcmc.cu — range cell migration correction of the range-Doppler operator pair
// (Section III-C, Eq. (16); its transpose, Eqs. (17), (22)), with the azimuth matched
// filter.
//
// In the range-Doppler domain (one azimuth-frequency row per CTA) the RDA focusing
// operator interpolates every range bin tau from the 8 bins b..b+7 around tau + dr
// (b = floor(tau + dr) - 3, indices mod N_r) with truncated-sinc weights
// sinc(b + t - tau - dr), then multiplies by the azimuth matched filter
// P_eta = exp(j 2 pi (A + B j')) (j' = tau - N_r/2).  The approximated observation
// applies conj(P_eta) and the transpose: every input bin adds its value, with the same
// weights, to the 8 bins it would have been read from (shared-memory atomics; the
// order of the 8-term sums is not fixed, so this direction is reproducible to rounding
// only).  The migration dr = alpha (c0 + j') (alpha = 1/D - 1, c0 = 2 R_ref fs / c) is
// evaluated in double-float from FP64 per-row coefficients, so its fraction, which
// sets the weights, is accurate to ~1e-7 samples.
#include "fft.cuh"
#include "internal.h"

namespace csar {

constexpr int kRcmcThreads = 256;

// First tap b and fractional offset f of output bin tau: tau + dr = b + 3 + f, f in [0, 1).
__device__ __forceinline__ int rcmc_tap(const RcmcCoef& k, int tau, int nr, float* f) {
  const int jp = tau - nr / 2;
  const float fj = (float)jp;
  const float p = k.al_hi * fj;
  const float e = fmaf(k.al_hi, fj, -p);              // exact error of the product
  const float n1 = rintf(k.a0_hi), n2 = rintf(p);
  const float fr = (k.a0_hi - n1) + (p - n2) + (k.a0_lo + e + k.al_lo * fj);
  const float fl = floorf(fr);
  *f = fr - fl;
  return tau + (int)n1 + (int)n2 + (int)fl - 3;
}

// Weights sinc(m - f), m = -3..4, from one sinpi: sin(pi (m - f)) = -(-1)^m sin(pi f).
__device__ __forceinline__ void rcmc_weights(float f, float (&w)[8]) {
  if (f <= 0.f) {
#pragma unroll
    for (int t = 0; t < 8; ++t) w[t] = t == 3 ? 1.f : 0.f;
    return;
  }
  const float s = sinpif(f) * 0.31830988618379067f;     // sin(pi f) / pi
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int m = t - 3;
    const float sg = (m & 1) ? s : -s;                  // -(-1)^m sin(pi f) / pi
    w[t] = sg / ((float)m - f);
  }
}

__device__ __forceinline__ float2 az_phase(const PhaseCoef& c, int jp, bool conj) {
  float2 p = phase_eval(c, jp, 1.f);
  if (conj) p.y = -p.y;
  return p;
}

// mode 0: data <- P_eta . C(data) (focusing);  mode 1: data <- D(conj(P_eta) . data).
__global__ void __launch_bounds__(kRcmcThreads) k_rcmc(RcmcArgs a) {
  extern __shared__ float2 row_sm[];
  const int row = blockIdx.x;
  const int nr = a.nr;
  float2* rp = a.data + (size_t)row * nr;
  const RcmcCoef k = a.coef[row];
  if (a.mode == 0) {
    for (int i = threadIdx.x; i < nr; i += blockDim.x) row_sm[i] = rp[i];
    __syncthreads();
    for (int tau = threadIdx.x; tau < nr; tau += blockDim.x) {
      float f;
      const int b = rcmc_tap(k, tau, nr, &f);
      float w[8];
      rcmc_weights(f, w);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float2 v = row_sm[(b + t) & (nr - 1)];
        acc.x = fmaf(v.x, w[t], acc.x);
        acc.y = fmaf(v.y, w[t], acc.y);
      }
      rp[tau] = cmul(acc, az_phase(k.az, tau - nr / 2, false));
    }
  } else {
    for (int i = threadIdx.x; i < nr; i += blockDim.x) row_sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    float* acc = reinterpret_cast<float*>(row_sm);
    for (int tau = threadIdx.x; tau < nr; tau += blockDim.x) {
      const float2 v = cmul(rp[tau], az_phase(k.az, tau - nr / 2, true));
      float f;
      const int b = rcmc_tap(k, tau, nr, &f);
      float w[8];
      rcmc_weights(f, w);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int j = (b + t) & (nr - 1);
        atomicAdd(&acc[2 * j], v.x * w[t]);
        atomicAdd(&acc[2 * j + 1], v.y * w[t]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr; i += blockDim.x) rp[i] = row_sm[i];
  }
}

cudaError_t rcmc_set_attributes() {
  return cudaFuncSetAttribute(k_rcmc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(8192 * sizeof(float2)));
}

cudaError_t launch_rcmc(const RcmcArgs& a, cudaStream_t s) {
  k_rcmc<<<a.n_rows, kRcmcThreads, (size_t)a.nr * sizeof(float2), s>>>(a);
  return cudaGetLastError();
}

}  // namespace csar
