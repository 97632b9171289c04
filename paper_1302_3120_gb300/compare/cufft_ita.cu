// cufft_ita.cu — a cuFFT-based comparison build of the ITA iteration, timed by the
// benchmark beside the library; it is never part of libcsar's path.
//
// It runs the same schedule as the library (Algorithm 1, Eq. (25), chirp-scaling pair)
// in its plain dense form, one library call or kernel per step:
//   G(X) = F_a^-1 conj(H1) F_r^-1 conj(H2) F_r conj(H3) F_a X
//   r = S . (Y - G(X)),   Delta X = M(r) = F_a^-1 H3 F_r^-1 H2 F_r H1 F_a r
//   B = X + mu Delta X,   sigma = |B|_(K+1),   X <- soft(B, sigma)
// Every transform is a cuFFT C2C plan (batched along the strided azimuth axis or the
// contiguous range axis); the phase multiplies evaluate each chirp-scaling phase exactly
// per element from the library's FP64-derived row coefficients; sigma comes from a
// three-round radix select (11 + 12 + 8 key bits) over all n keys bits(|b|^2).  The
// whole iteration is captured once into a CUDA graph.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../csrc/internal.h"

namespace {

using namespace csar;

thread_local std::string g_err;

int fail(const char* where, const char* what) {
  g_err = std::string(where) + ": " + what;
  return 1;
}

struct SelState {
  uint32_t prefix;      // key bits fixed so far
  uint32_t rank;        // 1-based rank of the wanted key among keys with that prefix
  uint32_t sigma2_key;  // result (0: fewer than K+1 nonzero keys)
  uint32_t done;
};

constexpr uint32_t kMinKeyC = 1u << 23;   // |b|^2 below the smallest normal fp32 counts as 0
constexpr int kT = 256;

__device__ __forceinline__ uint32_t key_of_c(float2 b) {
  return __float_as_uint(fmaf(b.x, b.x, b.y * b.y)) & 0x7fffffffu;
}

// z[i] *= exp(j 2 pi phi_row(idx)) * scale; which: 0 prologue (range time j - N_r/2),
// 1 middle (signed range frequency), 2 epilogue (range time).  Two elements per thread.
__global__ void k_phase(float2* __restrict__ z, const RowCoef* __restrict__ coef, int which,
                        float scale, int log2_nr, long long n) {
  const int nr = 1 << log2_nr;
  for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 2; p < n;
       p += (long long)gridDim.x * blockDim.x * 2) {
    float4 v = *reinterpret_cast<const float4*>(z + p);
    const int row = (int)(p >> log2_nr);
    const int j = (int)(p & (nr - 1));
    const RowCoef& rc = coef[row];
    const PhaseCoef& pc = which == 0 ? rc.pro : (which == 1 ? rc.mid : rc.epi);
    const int i0 = which == 1 ? (j < nr / 2 ? j : j - nr) : j - nr / 2;
    const int i1 = which == 1 ? (j + 1 < nr / 2 ? j + 1 : j + 1 - nr) : j + 1 - nr / 2;
    const float2 a = cmul(make_float2(v.x, v.y), phase_eval(pc, i0, scale));
    const float2 b = cmul(make_float2(v.z, v.w), phase_eval(pc, i1, scale));
    *reinterpret_cast<float4*>(z + p) = make_float4(a.x, a.y, b.x, b.y);
  }
}

// z = S . (Y - z / N_a)
__global__ void k_resid(float2* __restrict__ z, const float2* __restrict__ y,
                        const uint32_t* __restrict__ mask, float inv_na, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool s = (mask[i >> 5] >> (i & 31)) & 1u;
    const float2 g = z[i];
    const float2 yy = y[i];
    z[i] = s ? make_float2(yy.x - g.x * inv_na, yy.y - g.y * inv_na) : make_float2(0.f, 0.f);
  }
}

// z = X + mu z / N_a (= B), with the first-round histogram of key >> 20 (2048 bins)
__global__ void k_step_hist(const float2* __restrict__ x, float2* __restrict__ z, float mu_na,
                            uint32_t* __restrict__ hist, long long n) {
  __shared__ uint32_t h[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 xx = x[i], d = z[i];
    const float2 b = make_float2(fmaf(mu_na, d.x, xx.x), fmaf(mu_na, d.y, xx.y));
    z[i] = b;
    const uint32_t k = key_of_c(b);
    if (k >= kMinKeyC) atomicAdd(&h[k >> 20], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// later rounds: level 1 counts (key >> 8) & 4095 among keys with key >> 20 == prefix,
// level 2 counts key & 255 among keys with key >> 8 == prefix
__global__ void k_hist(const float2* __restrict__ b, int level, const SelState* __restrict__ st,
                       uint32_t* __restrict__ hist, long long n) {
  __shared__ uint32_t h[4096];
  if (st->done) return;
  const int nb = level == 1 ? 4096 : 256;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t prefix = st->prefix;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint32_t k = key_of_c(b[i]);
    if (k < kMinKeyC) continue;
    if (level == 1) {
      if ((k >> 20) == prefix) atomicAdd(&h[(k >> 8) & 4095u], 1u);
    } else if ((k >> 8) == prefix) {
      atomicAdd(&h[k & 255u], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One CTA of 1024 threads: the bin holding the rank-th largest key (rank K+1 at level 0),
// then the histogram is cleared for the next round.
__global__ void __launch_bounds__(1024) k_pick(uint32_t* __restrict__ hist, int level, int64_t K,
                                               SelState* __restrict__ st) {
  __shared__ unsigned long long sh[1024];
  __shared__ int res;
  __shared__ unsigned long long res_above;
  const int nb = level == 0 ? 2048 : (level == 1 ? 4096 : 256);
  const int per = nb >= 1024 ? nb / 1024 : 1;
  const int tid = threadIdx.x;
  const bool skip = level > 0 && st->done;
  const unsigned long long target = level == 0 ? (unsigned long long)K + 1 : st->rank;
  unsigned long long cs = 0;
  const int lo = tid * per;
  if (lo < nb)
    for (int i = 0; i < per; ++i) cs += hist[lo + i];
  sh[tid] = cs;
  if (tid == 0) { res = -1; res_above = 0; }
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {   // inclusive suffix sums
    const unsigned long long add = tid + off < 1024 ? sh[tid + off] : 0ull;
    __syncthreads();
    sh[tid] += add;
    __syncthreads();
  }
  const unsigned long long suf = sh[tid];
  const unsigned long long nxt = tid + 1 < 1024 ? sh[tid + 1] : 0ull;
  if (!skip && lo < nb && suf >= target && nxt < target) {
    unsigned long long acc = nxt;
    for (int i = per - 1; i >= 0; --i) {
      const unsigned long long s2 = acc + hist[lo + i];
      if (s2 >= target) { res = lo + i; res_above = acc; break; }
      acc = s2;
    }
  }
  __syncthreads();
  if (tid == 0 && level == 0) {   // a fresh state every iteration
    *st = res < 0 ? SelState{0u, 0u, 0u, 1u}
                  : SelState{(uint32_t)res, (uint32_t)(target - res_above), 0u, 0u};
  } else if (tid == 0 && !skip) {
    if (res < 0) {
      st->done = 1u;
      st->sigma2_key = 0u;
    } else {
      st->rank = (uint32_t)(target - res_above);
      if (level == 1) st->prefix = (st->prefix << 12) | (uint32_t)res;
      else { st->sigma2_key = (st->prefix << 8) | (uint32_t)res; st->done = 1u; }
    }
  }
  for (int i = tid; i < nb; i += 1024) hist[i] = 0u;
}

// X = soft(B, sigma) with sigma^2 = the selected key; strict |b| > sigma
__global__ void k_thresh(const float2* __restrict__ b, float2* __restrict__ x,
                         SelState* __restrict__ st, long long n) {
  const uint32_t s2 = st->sigma2_key;
  const float sigma = sqrtf(__uint_as_float(s2));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 v = b[i];
    const uint32_t k = key_of_c(v);
    float2 o = make_float2(0.f, 0.f);
    if (k > s2 && k >= kMinKeyC) {
      const float f = 1.f - sigma / sqrtf(__uint_as_float(k));
      o = make_float2(v.x * f, v.y * f);
    }
    x[i] = o;
  }
}

struct Handle {
  int na = 0, nr = 0, log2_nr = 0;
  long long n = 0;
  RowCoef* coef_g = nullptr;
  RowCoef* coef_m = nullptr;
  float2* z = nullptr;
  uint32_t* hist = nullptr;
  SelState* st = nullptr;
  cufftHandle col = 0, row = 0;
  bool col_ok = false, row_ok = false;
  cudaGraphExec_t exec = nullptr;
  const void* key_y = nullptr;
  const void* key_m = nullptr;
  const void* key_x = nullptr;
  int64_t key_k = -1;
  float key_mu = 0.f;
  int grid = 0;
};

int log2_int(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

cudaError_t fft_err(cufftResult r) { return r == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown; }

// One iteration on stream s (X in/out).
cudaError_t enqueue(Handle* h, const float2* y, const uint32_t* mask, float2* x, int64_t K, float mu,
                    cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const int g = h->grid;
  if (fft_err(cufftSetStream(h->col, s)) || fft_err(cufftSetStream(h->row, s))) return cudaErrorUnknown;
  cufftComplex* z = reinterpret_cast<cufftComplex*>(h->z);
  // G(X)
  if (cudaMemcpyAsync(h->z, x, h->n * sizeof(float2), cudaMemcpyDeviceToDevice, s)) return cudaErrorUnknown;
  if (cufftExecC2C(h->col, z, z, CUFFT_FORWARD) != CUFFT_SUCCESS) return cudaErrorUnknown;
  k_phase<<<g, kT, 0, s>>>(h->z, h->coef_g, 0, 1.f, h->log2_nr, h->n);
  if (cufftExecC2C(h->row, z, z, CUFFT_FORWARD) != CUFFT_SUCCESS) return cudaErrorUnknown;
  k_phase<<<g, kT, 0, s>>>(h->z, h->coef_g, 1, 1.f, h->log2_nr, h->n);
  if (cufftExecC2C(h->row, z, z, CUFFT_INVERSE) != CUFFT_SUCCESS) return cudaErrorUnknown;
  k_phase<<<g, kT, 0, s>>>(h->z, h->coef_g, 2, 1.f / (float)h->nr, h->log2_nr, h->n);
  if (cufftExecC2C(h->col, z, z, CUFFT_INVERSE) != CUFFT_SUCCESS) return cudaErrorUnknown;
  // r = S . (Y - G X)
  k_resid<<<g, kT, 0, s>>>(h->z, y, mask, 1.f / (float)h->na, h->n);
  // Delta X = M(r)
  if (cufftExecC2C(h->col, z, z, CUFFT_FORWARD) != CUFFT_SUCCESS) return cudaErrorUnknown;
  k_phase<<<g, kT, 0, s>>>(h->z, h->coef_m, 0, 1.f, h->log2_nr, h->n);
  if (cufftExecC2C(h->row, z, z, CUFFT_FORWARD) != CUFFT_SUCCESS) return cudaErrorUnknown;
  k_phase<<<g, kT, 0, s>>>(h->z, h->coef_m, 1, 1.f, h->log2_nr, h->n);
  if (cufftExecC2C(h->row, z, z, CUFFT_INVERSE) != CUFFT_SUCCESS) return cudaErrorUnknown;
  k_phase<<<g, kT, 0, s>>>(h->z, h->coef_m, 2, 1.f / (float)h->nr, h->log2_nr, h->n);
  if (cufftExecC2C(h->col, z, z, CUFFT_INVERSE) != CUFFT_SUCCESS) return cudaErrorUnknown;
  // B, sigma, threshold
  k_step_hist<<<g, kT, 0, s>>>(x, h->z, mu / (float)h->na, h->hist, h->n);
  k_pick<<<1, 1024, 0, s>>>(h->hist, 0, K, h->st);
  k_hist<<<g, kT, 0, s>>>(h->z, 1, h->st, h->hist, h->n);
  k_pick<<<1, 1024, 0, s>>>(h->hist, 1, K, h->st);
  k_hist<<<g, kT, 0, s>>>(h->z, 2, h->st, h->hist, h->n);
  k_pick<<<1, 1024, 0, s>>>(h->hist, 2, K, h->st);
  k_thresh<<<g, kT, 0, s>>>(h->z, x, h->st, h->n);
  e = cudaGetLastError();
  return e;
}

}  // namespace

extern "C" {

const char* csar_cufft_last_error(void) { return g_err.c_str(); }

int csar_cufft_destroy(void* hv) {
  Handle* h = static_cast<Handle*>(hv);
  if (!h) return 0;
  cudaDeviceSynchronize();
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->col_ok) cufftDestroy(h->col);
  if (h->row_ok) cufftDestroy(h->row);
  void* p[] = {h->coef_g, h->coef_m, h->z, h->hist, h->st};
  for (void* q : p)
    if (q) cudaFree(q);
  delete h;
  return 0;
}

int csar_cufft_create(const csar_params* params, void** out) {
  if (!out) return fail("csar_cufft_create", "out is NULL");
  *out = nullptr;
  if (validate_params(params) != CSAR_OK) return fail("csar_cufft_create", "invalid parameters");
  Handle* h = new Handle();
  h->na = params->n_az;
  h->nr = params->n_rg;
  h->log2_nr = log2_int(h->nr);
  h->n = (long long)h->na * h->nr;
  h->grid = 152 * 8;
  std::vector<RowCoef> cg(h->na), cm(h->na);
  if (build_coefs_into(*params, cg.data(), cm.data()) != CSAR_OK) {
    csar_cufft_destroy(h);
    return fail("csar_cufft_create", "phase coefficients");
  }
  cudaError_t e = cudaMalloc(&h->coef_g, h->na * sizeof(RowCoef));
  if (!e) e = cudaMalloc(&h->coef_m, h->na * sizeof(RowCoef));
  if (!e) e = cudaMalloc(&h->z, h->n * sizeof(float2));
  if (!e) e = cudaMalloc(&h->hist, 4096 * sizeof(uint32_t));
  if (!e) e = cudaMalloc(&h->st, sizeof(SelState));
  if (!e) e = cudaMemcpy(h->coef_g, cg.data(), h->na * sizeof(RowCoef), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(h->coef_m, cm.data(), h->na * sizeof(RowCoef), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemset(h->hist, 0, 4096 * sizeof(uint32_t));
  if (!e) e = cudaMemset(h->st, 0, sizeof(SelState));
  if (e) {
    csar_cufft_destroy(h);
    return fail("csar_cufft_create", cudaGetErrorString(e));
  }
  // columns: N_r transforms of length N_a with stride N_r; rows: N_a contiguous transforms
  int n_a = h->na, n_r = h->nr;
  if (cufftPlanMany(&h->col, 1, &n_a, &n_a, h->nr, 1, &n_a, h->nr, 1, CUFFT_C2C, h->nr) != CUFFT_SUCCESS) {
    csar_cufft_destroy(h);
    return fail("csar_cufft_create", "cufftPlanMany (azimuth)");
  }
  h->col_ok = true;
  if (cufftPlanMany(&h->row, 1, &n_r, &n_r, 1, h->nr, &n_r, 1, h->nr, CUFFT_C2C, h->na) != CUFFT_SUCCESS) {
    csar_cufft_destroy(h);
    return fail("csar_cufft_create", "cufftPlanMany (range)");
  }
  h->row_ok = true;
  *out = h;
  return 0;
}

// iters iterations of the dense ITA from X = 0 (soft threshold, fixed step mu).
// Y_dev: n complex64 (zero-filled echo), mask_dev: n/32 words, X_dev: n complex64 out.
int csar_cufft_solve(void* hv, const void* Y_dev, const uint32_t* mask_dev, void* X_dev, int64_t K,
                     int32_t iters, float mu, void* stream) {
  Handle* h = static_cast<Handle*>(hv);
  if (!h || !Y_dev || !mask_dev || !X_dev || iters < 0 || K < 0) return fail("csar_cufft_solve", "invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  float2* x = static_cast<float2*>(X_dev);
  if (cudaMemsetAsync(x, 0, h->n * sizeof(float2), s)) return fail("csar_cufft_solve", "memset");
  if (!h->exec || h->key_y != Y_dev || h->key_m != mask_dev || h->key_x != X_dev || h->key_k != K ||
      h->key_mu != mu) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) return fail("csar_cufft_solve", "stream");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaError_t e1 = e ? e : enqueue(h, (const float2*)Y_dev, mask_dev, x, K, mu, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (e || e1 || e2) {
      if (g) cudaGraphDestroy(g);
      return fail("csar_cufft_solve", "graph capture");
    }
    e = cudaGraphInstantiate(&h->exec, g, 0);
    cudaGraphDestroy(g);
    if (e) return fail("csar_cufft_solve", cudaGetErrorString(e));
    h->key_y = Y_dev;
    h->key_m = mask_dev;
    h->key_x = X_dev;
    h->key_k = K;
    h->key_mu = mu;
  }
  for (int i = 0; i < iters; ++i)
    if (cudaGraphLaunch(h->exec, s)) return fail("csar_cufft_solve", "graph launch");
  return 0;
}

}  // extern "C"
