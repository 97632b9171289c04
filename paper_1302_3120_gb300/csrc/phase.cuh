// phase.cuh — on-the-fly evaluation of the chirp-scaling phase functions.
//
// Every phase the operators multiply by (H1, H2, H3 of the chirp-scaling
// algorithm, and their conjugates for G) is, for a fixed azimuth-frequency row, a
// quadratic polynomial in an exact integer index i (signed range bin or signed
// range-frequency bin):
//
//     phi(i) = A + B*i + C*i^2   [cycles],      H = exp(j 2 pi phi(i)).
//
// The host computes A (reduced mod 1), B and C per row in FP64 and splits each into
// an fp32 (hi, lo) pair.  The device evaluates the products of hi parts exactly
// (Dekker's product via fma: p = fl(h*x), e = fma(h, x, -p) is the exact error),
// removes the integer part of each large product exactly (|p| < 2^23, so p - rint(p)
// is exact), sums the small remaining terms in fp32, reduces once more and calls
// sincospif.  With |B i|, |C i^2| < 2^22 the phase error is a few 1e-7 cycles,
// against tens of millions of cycles in the raw argument of H3.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

namespace csar {

struct PhaseCoef {
  float a_hi, a_lo, b_hi, b_lo, c_hi, c_lo;
};

struct RowCoef {
  PhaseCoef pro, mid, epi;   // prologue (range time), middle (range freq), epilogue (range time)
};

// exp(j 2 pi (A + B i + C i^2)) * scale.  |i| <= 4096 so i^2 is exact in fp32.
__device__ __forceinline__ float2 phase_eval(const PhaseCoef& c, int i, float scale) {
  const float fi = (float)i;
  const float s = fi * fi;
  const float pb = c.b_hi * fi;
  const float eb = fmaf(c.b_hi, fi, -pb);
  const float pc = c.c_hi * s;
  const float ec = fmaf(c.c_hi, s, -pc);
  const float rb = pb - rintf(pb);
  const float rc = pc - rintf(pc);
  const float small = eb + ec + fmaf(c.b_lo, fi, fmaf(c.c_lo, s, c.a_lo));
  float t = (c.a_hi + rb) + (rc + small);
  t -= rintf(t);
  float sn, cs;
  sincospif(2.0f * t, &sn, &cs);
  return make_float2(cs * scale, sn * scale);
}

// exp(j 2 pi * 2 C d^2): ratio of consecutive first differences of phi along an
// arithmetic progression of step d (d a power of two, so 2 d^2 scales exactly).
__device__ __forceinline__ float2 phase_second_diff(const PhaseCoef& c, int d) {
  const float x = 2.0f * (float)d * (float)d;
  const float p = c.c_hi * x;
  float t = (p - rintf(p)) + c.c_lo * x;
  t -= rintf(t);
  float sn, cs;
  sincospif(2.0f * t, &sn, &cs);
  return make_float2(cs, sn);
}

// v[s] *= scale * exp(j 2 pi phi(i0 + (s - S0) d)) for s in [S0, S1), S1 - S0 a
// multiple of 8.  In each block of 8 consecutive s the first two factors are
// evaluated exactly (phase_eval) and the rest follow from the second-order
// recurrence  r_{u+1} = r_u q_u,  q_{u+1} = q_u exp(j 2 pi 2 C d^2)  (phi is
// quadratic), i.e. 2 complex products per element instead of a full evaluation;
// re-anchoring every 8 elements bounds the accumulated rounding to a few 1e-7.
template <int R, int S0, int S1>
__device__ __forceinline__ void phase_ap(float2 (&v)[R], const PhaseCoef& c, int i0, int d,
                                         float scale, float2 dd) {
#pragma unroll
  for (int blk = S0; blk < S1; blk += 8) {
    const int ib = i0 + (blk - S0) * d;
    const float2 e0 = phase_eval(c, ib, 1.f);
    const float2 e1 = phase_eval(c, ib + d, 1.f);
    float2 q = make_float2(fmaf(e1.x, e0.x, e1.y * e0.y), fmaf(e1.y, e0.x, -e1.x * e0.y));  // e1 conj(e0)
    float2 r = make_float2(e1.x * scale, e1.y * scale);
    v[blk] = cmul(v[blk], make_float2(e0.x * scale, e0.y * scale));
    v[blk + 1] = cmul(v[blk + 1], r);
#pragma unroll
    for (int u = 2; u < 8; ++u) {
      q = cmul(q, dd);
      r = cmul(r, q);
      v[blk + u] = cmul(v[blk + u], r);
    }
  }
}

// Gamma[u] = exp(j 2 pi gamma u^2), gamma = C d^2: the quadratic part of phi along an
// arithmetic progression of step d (d a power of two, so the scaling is exact).
__device__ __forceinline__ float2 phase_gamma(const PhaseCoef& c, int d, int u) {
  const float dd = (float)d * (float)d;
  PhaseCoef g;
  g.a_hi = g.a_lo = g.b_hi = g.b_lo = 0.f;
  g.c_hi = c.c_hi * dd;
  g.c_lo = c.c_lo * dd;
  return phase_eval(g, u, 1.f);
}

// v[s] *= scale * exp(j 2 pi phi(i0 + (s - S0) d)) for s in [S0, S1), as one chain:
//   phi(i0 + u d) = phi(i0) + u kappa + u^2 gamma,   kappa = d (B + 2 C i0),
// so the factor is E Lambda^u Gamma[u] with E = exp(j 2 pi phi(i0)), Lambda =
// exp(j 2 pi kappa) = exp(j 2 pi (phi(i0 + d) - phi(i0))) conj(Gamma[1]) and Gamma the
// per-row table of phase_gamma.  Two exact evaluations per chain and three complex
// products per element; the quadratic part comes exact from the table.  The powers
// Lambda^u run as four interleaved recurrences (u = 4m + j: E Lambda^j times
// (Lambda^4)^m), which gives the scheduler four independent dependency chains instead
// of one and accumulates at most S1/4 + 3 roundings per power (a few 1e-7).
template <int R, int S0, int S1>
__device__ __forceinline__ void phase_chain(float2 (&v)[R], const PhaseCoef& c, int i0, int d,
                                            float scale, const float2* gam) {
  const float2 e0 = phase_eval(c, i0, 1.f);
  const float2 e1 = phase_eval(c, i0 + d, 1.f);
  const float2 q = make_float2(fmaf(e1.x, e0.x, e1.y * e0.y), fmaf(e1.y, e0.x, -e1.x * e0.y));  // e1 conj(e0)
  const float2 g1 = gam[1];
  const float2 lam = make_float2(fmaf(q.x, g1.x, q.y * g1.y), fmaf(q.y, g1.x, -q.x * g1.y));  // q conj(g1)
  const float2 p0 = make_float2(e0.x * scale, e0.y * scale);
#pragma unroll
  for (int s = S0 + 1; s < S1; ++s) v[s] = cmul(v[s], gam[s - S0]);
  const float2 lam2 = cmul(lam, lam), lam4 = cmul(lam2, lam2);
  float2 p[4];
  p[0] = p0;
  p[1] = cmul(p0, lam);
  p[2] = cmul(p0, lam2);
  p[3] = cmul(p[1], lam2);
#pragma unroll
  for (int s = S0; s < S1; ++s) {
    v[s] = cmul(v[s], p[(s - S0) & 3]);
    p[(s - S0) & 3] = cmul(p[(s - S0) & 3], lam4);
  }
}

}  // namespace csar
