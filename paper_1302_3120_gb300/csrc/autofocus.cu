// autofocus.cu — kernels of the differentiable autofocus path.
//
// Observation with a per-pulse phase error theta: A_theta X = S . (exp(j theta_eta) G X).
// The ITA for it runs on the de-rotated echo Y_theta = exp(-j theta_eta) Y, and
//   L = ||S . (Y_theta - G X)||^2,  grad_X L = -2 M(r),  dL/dtheta_eta = 2 sum Im(conj(r) Y_theta)
// with r = S . (Y_theta - G X) (complex gradients in the dL = Re<grad, dz> convention).
// Backward through one soft-threshold iteration (sigma = |b|_(K+1) at element j*):
//   bbar = (1 - sigma/|b|) xbar + (sigma/|b|) Re(conj(u) xbar) u on kept entries,
//   bbar_{j*} += -sum_kept Re(conj(u) xbar) u_{j*},
//   Xbar = bbar - mu M(S . G bbar),   thetabar_eta += mu sum Im(conj(S . G bbar) Y_theta).
// Row reductions use one CTA per row (deterministic, no atomics).
#include "fft.cuh"
#include "internal.h"

namespace csar {

constexpr int kAfThreads = 256;

template <typename T>
__device__ __forceinline__ T block_reduce_sum(T v, T* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (tid < off) sh[tid] += sh[tid + off];
    __syncthreads();
  }
  const T r = sh[0];
  __syncthreads();
  return r;
}

// Yt = exp(-j theta_row) Y
__global__ void k_rotate_rows(const float2* __restrict__ y, const float* __restrict__ theta,
                              float2* __restrict__ yt, int nr) {
  const int row = blockIdx.x;
  float sn, cs;
  sincosf(theta[row], &sn, &cs);
  const float2 e = make_float2(cs, -sn);
  const float2* yr = y + (size_t)row * nr;
  float2* outr = yt + (size_t)row * nr;
  for (int j = threadIdx.x; j < nr; j += blockDim.x) outr[j] = cmul(yr[j], e);
}

// r = S.(Yt - g) (written over g), per row: sum |r|^2 and 2 sum Im(conj(r) Yt)
__global__ void k_af_resid_rows(float2* __restrict__ g, const float2* __restrict__ yt,
                                const uint32_t* __restrict__ mask, int nr, double* __restrict__ row_loss,
                                float* __restrict__ grad_theta) {
  __shared__ double sh[kAfThreads];
  const int row = blockIdx.x;
  double l = 0.0, th = 0.0;
  for (int j = threadIdx.x; j < nr; j += blockDim.x) {
    const size_t i = (size_t)row * nr + j;
    const bool on = (mask[i >> 5] >> (i & 31)) & 1u;
    const float2 yv = yt[i];
    const float2 r = on ? csub(yv, g[i]) : make_float2(0.f, 0.f);
    g[i] = r;
    l += (double)cabs2(r);
    th += (double)(r.x * yv.y - r.y * yv.x);   // Im(conj(r) y)
  }
  l = block_reduce_sum(l, sh);
  th = block_reduce_sum(th, sh);
  if (threadIdx.x == 0) {
    row_loss[row] = l;
    if (grad_theta) grad_theta[row] = (float)(2.0 * th);
  }
}

__global__ void k_sum_rows(const double* __restrict__ row_loss, int na, double* __restrict__ out) {
  __shared__ double sh[kAfThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < na; i += blockDim.x) s += row_loss[i];
  s = block_reduce_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// out = alpha * in (dense)
__global__ void k_scale(const float2* __restrict__ in, float2* __restrict__ out, float alpha, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = cscale(in[i], alpha);
}

// Threshold VJP on the kept entries of checkpoint (idx, val, count) with threshold sigma:
// writes bbar at those entries of the (zeroed) dense bbar.
__global__ void k_af_tvjp(const uint32_t* __restrict__ idx, const float2* __restrict__ val,
                          const CkptMeta* __restrict__ meta, const float2* __restrict__ xbar,
                          float2* __restrict__ bbar) {
  const uint32_t n = meta->count;
  const float sigma = meta->sigma;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const uint32_t i = idx[e];
    const float2 x = val[e];
    const float xm = sqrtf(cabs2(x));
    const float2 u = make_float2(x.x / xm, x.y / xm);
    const float bm = xm + sigma;
    const float2 xb = xbar[i];
    const float proj = u.x * xb.x + u.y * xb.y;   // Re(conj(u) xbar)
    const float a = 1.f - sigma / bm, c = sigma / bm * proj;
    bbar[i] = make_float2(a * xb.x + c * u.x, a * xb.y + c * u.y);
  }
}

// sigmabar = -sum_kept Re(conj(u) xbar) routed to the (K+1)-th element j*
__global__ void k_af_tvjp_sigma(const uint32_t* __restrict__ idx, const float2* __restrict__ val,
                                const CkptMeta* __restrict__ meta, const float2* __restrict__ xbar,
                                float2* __restrict__ bbar) {
  __shared__ double sh[kAfThreads];
  const uint32_t n = meta->count;
  double s = 0.0;
  for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
    const float2 x = val[e];
    const float xm = sqrtf(cabs2(x));
    const float2 xb = xbar[idx[e]];
    s += (double)((x.x * xb.x + x.y * xb.y) / xm);
  }
  s = block_reduce_sum(s, sh);
  if (threadIdx.x == 0 && meta->jstar != 0xffffffffu && meta->sigma > 0.f) {
    const float2 bj = meta->b_jstar;
    const float bm = sqrtf(cabs2(bj));
    const float sb = (float)(-s);
    float2 v = bbar[meta->jstar];
    v.x += sb * bj.x / bm;
    v.y += sb * bj.y / bm;
    bbar[meta->jstar] = v;
  }
}

// g <- S.g (in place); thetabar_row += mu sum Im(conj(S.g) Yt)
__global__ void k_af_mask_theta(float2* __restrict__ g, const float2* __restrict__ yt,
                                const uint32_t* __restrict__ mask, int nr, float mu,
                                float* __restrict__ theta_bar) {
  __shared__ double sh[kAfThreads];
  const int row = blockIdx.x;
  double th = 0.0;
  for (int j = threadIdx.x; j < nr; j += blockDim.x) {
    const size_t i = (size_t)row * nr + j;
    const bool on = (mask[i >> 5] >> (i & 31)) & 1u;
    const float2 gv = on ? g[i] : make_float2(0.f, 0.f);
    g[i] = gv;
    const float2 yv = yt[i];
    th += (double)(gv.x * yv.y - gv.y * yv.x);
  }
  th = block_reduce_sum(th, sh);
  if (threadIdx.x == 0) theta_bar[row] += (float)(mu * th);
}

// xbar = bbar - mu h
__global__ void k_af_axpy(const float2* __restrict__ bbar, const float2* __restrict__ h, float mu,
                          float2* __restrict__ xbar, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 b = bbar[i], hv = h[i];
    xbar[i] = make_float2(fmaf(-mu, hv.x, b.x), fmaf(-mu, hv.y, b.y));
  }
}

// Checkpoint of the iterate just written (list nxt, count ctl->nnz) into slot ctl->iter.
__global__ void k_ckpt_copy(const Ctl* __restrict__ ctl, const uint32_t* __restrict__ idx,
                            const float2* __restrict__ val, uint32_t* __restrict__ ck_idx,
                            float2* __restrict__ ck_val, CkptMeta* __restrict__ ck_meta, uint32_t cap) {
  const uint32_t it = ctl->iter;
  const uint32_t n = ctl->nnz < cap ? ctl->nnz : cap;
  uint32_t* di = ck_idx + (size_t)it * cap;
  float2* dv = ck_val + (size_t)it * cap;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    di[e] = idx[e];
    dv[e] = val[e];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CkptMeta m;
    m.count = n;
    m.sigma = ctl->sigma;
    m.jstar = ctl->jstar;
    m.b_jstar = ctl->b_jstar;
    ck_meta[it] = m;
  }
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

cudaError_t launch_rotate_rows(const float2* y, const float* theta, float2* yt, int na, int nr,
                               cudaStream_t s) {
  k_rotate_rows<<<na, kAfThreads, 0, s>>>(y, theta, yt, nr);
  return cudaGetLastError();
}
cudaError_t launch_af_resid(float2* g, const float2* yt, const uint32_t* mask, int na, int nr,
                            double* row_loss, float* grad_theta, double* loss, cudaStream_t s) {
  k_af_resid_rows<<<na, kAfThreads, 0, s>>>(g, yt, mask, nr, row_loss, grad_theta);
  k_sum_rows<<<1, kAfThreads, 0, s>>>(row_loss, na, loss);
  return cudaGetLastError();
}
cudaError_t launch_scale(const float2* in, float2* out, float alpha, long long n, cudaStream_t s) {
  k_scale<<<grid_for(n), 256, 0, s>>>(in, out, alpha, n);
  return cudaGetLastError();
}
cudaError_t launch_af_tvjp(const uint32_t* idx, const float2* val, const CkptMeta* meta,
                           const float2* xbar, float2* bbar, uint32_t cap, cudaStream_t s) {
  k_af_tvjp<<<grid_for(cap), 256, 0, s>>>(idx, val, meta, xbar, bbar);
  k_af_tvjp_sigma<<<1, kAfThreads, 0, s>>>(idx, val, meta, xbar, bbar);
  return cudaGetLastError();
}
cudaError_t launch_af_mask_theta(float2* g, const float2* yt, const uint32_t* mask, int na, int nr,
                                 float mu, float* theta_bar, cudaStream_t s) {
  k_af_mask_theta<<<na, kAfThreads, 0, s>>>(g, yt, mask, nr, mu, theta_bar);
  return cudaGetLastError();
}
cudaError_t launch_af_axpy(const float2* bbar, const float2* h, float mu, float2* xbar, long long n,
                           cudaStream_t s) {
  k_af_axpy<<<grid_for(n), 256, 0, s>>>(bbar, h, mu, xbar, n);
  return cudaGetLastError();
}
cudaError_t launch_ckpt_copy(const Ctl* ctl, const uint32_t* idx, const float2* val, uint32_t* ck_idx,
                             float2* ck_val, CkptMeta* ck_meta, uint32_t cap, cudaStream_t s) {
  k_ckpt_copy<<<grid_for(cap), 256, 0, s>>>(ctl, idx, val, ck_idx, ck_val, ck_meta, cap);
  return cudaGetLastError();
}

}  // namespace csar
