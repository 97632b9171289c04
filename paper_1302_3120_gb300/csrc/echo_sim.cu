// echo_sim.cu — raw stripmap echoes of point targets from the exact observation model
// (Section V-A: echoes generated in the time domain from the exact slant range), on the
// GPU in FP64.
//
// A target on image pixel (row, col) sits at azimuth time eta_t = (row - N_a/2)/PRF and
// closest range R_t = c tau_col / 2, tau_j = 2 R_ref/c + (j - N_r/2)/fs.  Its echo at
// pulse i, range bin j is
//     a rect(delay / T_p) rect((eta_i - eta_t) / T_a) exp(-j 4 pi f0 R / c + j pi K_r delay^2),
//     R = sqrt(R_t^2 + V^2 (eta_i - eta_t)^2),  delay = tau_j - 2 R / c,
// with the synthetic aperture T_a = 0.886 lambda R_t / (La V) and f0 = c / lambda,
// K_r = B / T_p (up-chirp), windows closed at their edges.
//
// One CTA owns a tile of kSimRows pulses x kSimCols range bins, one thread per range bin
// and its kSimRows pulses in registers.  The targets arrive sorted by row; a CTA scans
// the rows within the largest half-aperture of its tile (binary search) and keeps, in
// shared memory, those whose aperture and delay windows meet the tile; then every thread
// adds each kept target's contribution to its elements.  Geometry (slant range, delay,
// phase in cycles reduced mod 1) is FP64; the final sincospi and the sums are fp32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/csar.h"
#include "internal.h"

namespace csar {
namespace {

constexpr int kSimRows = 16;
constexpr int kSimCols = 256;
constexpr int kSimBatch = 256;   // targets staged per round

struct SimTarget {
  double eta_t;     // azimuth time of closest approach
  double r_t;       // closest range
  double half_ta;   // T_a / 2
  float2 amp;
  int row, col;
  int r_lo, r_hi;   // pulses the aperture can reach (conservative)
  int c_lo, c_hi;   // range bins the delay window can reach (conservative)
};

struct SimGeom {
  int na, nr;
  double prf, fs, c, two_r0_c, v, v2, half_tp, two_over_lambda, half_kr;
};

__global__ void __launch_bounds__(kSimCols) k_echo_points(SimGeom g, const SimTarget* tg, int n_tg,
                                                          int max_half_rows, float2* out, int accumulate) {
  __shared__ SimTarget st[kSimBatch];
  __shared__ int st_count;
  const int r0 = blockIdx.y * kSimRows;
  const int j = blockIdx.x * kSimCols + threadIdx.x;
  const int c0 = blockIdx.x * kSimCols;
  const int c1 = min(c0 + kSimCols, g.nr) - 1;
  const int r1 = min(r0 + kSimRows, g.na) - 1;
  // targets whose row lies within max_half_rows of the tile, by binary search on rows
  int lo = 0, hi = n_tg;
  const int want_lo = r0 - max_half_rows;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (tg[m].row < want_lo) lo = m + 1; else hi = m;
  }
  int end = lo, hi2 = n_tg;
  const int want_hi = r1 + max_half_rows;
  while (end < hi2) {
    const int m = (end + hi2) >> 1;
    if (tg[m].row <= want_hi) end = m + 1; else hi2 = m;
  }
  float2 acc[kSimRows];
#pragma unroll
  for (int r = 0; r < kSimRows; ++r) acc[r] = make_float2(0.f, 0.f);
  const double tau = g.two_r0_c + (double)(j - g.nr / 2) / g.fs;
  for (int base = lo; base < end; base += kSimBatch) {
    if (threadIdx.x == 0) st_count = 0;
    __syncthreads();
    const int i = base + threadIdx.x;
    if (i < end) {
      const SimTarget& t = tg[i];
      if (t.r_hi >= r0 && t.r_lo <= r1 && t.c_hi >= c0 && t.c_lo <= c1) st[atomicAdd(&st_count, 1)] = t;
    }
    __syncthreads();
    const int cnt = st_count;
    if (j < g.nr) {
      for (int k = 0; k < cnt; ++k) {
        const SimTarget& t = st[k];
#pragma unroll
        for (int r = 0; r < kSimRows; ++r) {
          const int row = r0 + r;
          const double eta = (double)(row - g.na / 2) / g.prf;
          const double de = eta - t.eta_t;
          if (row >= g.na || !(fabs(de) <= t.half_ta)) continue;
          // same operations, in the same order and without contraction, as the FP64
          // reference model, so that both take the window decisions alike
          const double vd = __dmul_rn(g.v, de);
          const double rng = __dsqrt_rn(__dadd_rn(__dmul_rn(t.r_t, t.r_t), __dmul_rn(vd, vd)));
          const double delay = __dsub_rn(tau, __ddiv_rn(__dmul_rn(2.0, rng), g.c));
          if (!(fabs(delay) <= g.half_tp)) continue;
          double cyc = -g.two_over_lambda * rng + g.half_kr * delay * delay;
          cyc -= rint(cyc);
          float sn, cs;
          sincospif(2.0f * (float)cyc, &sn, &cs);
          acc[r].x += t.amp.x * cs - t.amp.y * sn;
          acc[r].y += t.amp.x * sn + t.amp.y * cs;
        }
      }
    }
    __syncthreads();
  }
  if (j >= g.nr) return;
#pragma unroll
  for (int r = 0; r < kSimRows; ++r) {
    const int row = r0 + r;
    if (row >= g.na) break;
    float2* p = out + (size_t)row * g.nr + j;
    if (accumulate) {
      const float2 o = *p;
      *p = make_float2(o.x + acc[r].x, o.y + acc[r].y);
    } else {
      *p = acc[r];
    }
  }
}

csar_status sim_fail(csar_status st, const char* what, long long k) {
  char buf[160];
  std::snprintf(buf, sizeof buf, "csar_echo_points: target %lld %s", k, what);
  return set_error(st, buf);
}

}  // namespace
}  // namespace csar

using namespace csar;

extern "C" csar_status csar_echo_points(const csar_params* params, const int32_t* rows, const int32_t* cols,
                                        const float* amp, int64_t count, void* echo_dev, int32_t accumulate,
                                        void* stream) {
  if (csar_status st = validate_params(params)) return st;
  if (!(params->antenna_len > 0.0) || !std::isfinite(params->antenna_len))
    return set_error(CSAR_E_INVALID, "csar_echo_points: antenna_len must be finite and > 0");
  if (!echo_dev) return set_error(CSAR_E_INVALID, "csar_echo_points: echo is NULL");
  if (count < 0 || count > (int64_t)1 << 24)
    return set_error(CSAR_E_INVALID, "csar_echo_points: count must be in [0, 2^24]");
  if (count > 0 && (!rows || !cols || !amp))
    return set_error(CSAR_E_INVALID, "csar_echo_points: null target array");
  const csar_params& p = *params;
  const int na = p.n_az, nr = p.n_rg;
  const double c = p.c > 0.0 ? p.c : 299792458.0;
  SimGeom g{};
  g.na = na;
  g.nr = nr;
  g.prf = p.prf;
  g.fs = p.fs;
  g.c = c;
  g.two_r0_c = 2.0 * p.r0 / c;
  g.v = p.velocity;
  g.v2 = p.velocity * p.velocity;
  g.half_tp = p.pulse_len / 2.0;
  g.two_over_lambda = 2.0 / p.wavelength;
  g.half_kr = 0.5 * p.bandwidth / p.pulse_len;
  std::vector<SimTarget> tg((size_t)count);
  int max_half_rows = 0;
  for (int64_t k = 0; k < count; ++k) {
    const int row = rows[k], col = cols[k];
    if (row < 0 || row >= na || col < 0 || col >= nr)
      return sim_fail(CSAR_E_INVALID, "is off the grid", (long long)k);
    SimTarget& t = tg[(size_t)k];
    t.row = row;
    t.col = col;
    t.eta_t = (double)(row - na / 2) / p.prf;
    t.r_t = c * (g.two_r0_c + (double)(col - nr / 2) / p.fs) / 2.0;
    if (!(t.r_t > 0.0)) return sim_fail(CSAR_E_INVALID, "is at a non-positive range", (long long)k);
    t.half_ta = 0.886 * p.wavelength * t.r_t / (p.antenna_len * p.velocity) / 2.0;
    t.amp = make_float2(amp[2 * k], amp[2 * k + 1]);
    const double hr = t.half_ta * p.prf + 1.0;
    if (hr > 1e9) return set_error(CSAR_E_UNSUPPORTED, "csar_echo_points: aperture too long");
    const int h = (int)std::ceil(hr);
    t.r_lo = row - h;
    t.r_hi = row + h;
    max_half_rows = std::max(max_half_rows, h);
    const double r_max = std::sqrt(t.r_t * t.r_t + g.v2 * t.half_ta * t.half_ta);
    const double lead = g.half_tp * p.fs + 1.0;
    const double lag = (2.0 * (r_max - t.r_t) / c + g.half_tp) * p.fs + 1.0;
    if (lead > 1e9 || lag > 1e9) return set_error(CSAR_E_UNSUPPORTED, "csar_echo_points: pulse too long");
    t.c_lo = col - (int)std::ceil(lead);
    t.c_hi = col + (int)std::ceil(lag);
  }
  std::stable_sort(tg.begin(), tg.end(), [](const SimTarget& a, const SimTarget& b) { return a.row < b.row; });
  cudaStream_t s = (cudaStream_t)stream;
  SimTarget* d_tg = nullptr;
  cudaError_t e = cudaSuccess;
  if (count > 0) {
    e = cudaMallocAsync((void**)&d_tg, tg.size() * sizeof(SimTarget), s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_tg, tg.data(), tg.size() * sizeof(SimTarget), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) {
    const dim3 grid((nr + kSimCols - 1) / kSimCols, (na + kSimRows - 1) / kSimRows);
    k_echo_points<<<grid, kSimCols, 0, s>>>(g, d_tg, (int)count, max_half_rows, (float2*)echo_dev, accumulate);
    e = cudaGetLastError();
  }
  if (d_tg) {
    const cudaError_t f = cudaFreeAsync(d_tg, s);
    if (e == cudaSuccess) e = f;
  }
  // a copy from pageable memory returns once the data is staged, so tg may go now
  if (e != cudaSuccess) return set_error(CSAR_E_CUDA, cudaGetErrorString(e));
  return CSAR_OK;
}
