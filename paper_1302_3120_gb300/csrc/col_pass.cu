// col_pass.cu — azimuth (column, strided-axis) passes.
//
// One CTA owns a tile of W adjacent columns over all N_a rows (W*N_a = 16K
// complex64 = 128 KiB in shared memory).  Each warp reads/writes W*8-byte row
// segments of 32/W rows per instruction, straight into / out of the canonical
// register order of the length-N_a Stockham FFT (fft.cuh), so HBM is touched once
// per element per pass.  The passes carry the fused work of the ITA iteration:
//
//   COL_FWD / COL_INV      plain azimuth FFT / IFFT (operators G and M)
//   COL_SPARSE_FWD         the K-sparse iterate scattered into a zero tile, then FFT
//   COL_RESID              IFFT -> G(X); r = S.(Y - G(X)); FFT -> input of M   (Eq. (25))
//   COL_SELECT / REPASS    IFFT -> Delta X = M(r); Delta X at the support; histogram
//                          of |Delta X|^2 keys and compaction of the candidates for
//                          the (K+1)-th magnitude (Section IV-B)
//   COL_NORM               IFFT -> G(Delta X_Gamma); sum of S.|.|^2 (NIHT step)
#include "fft.cuh"
#include "internal.h"

namespace csar {

template <int NT>
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if constexpr (NT <= 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float s = 0.f;
    if (wid == 0) {
      s = lane < NT / 32 ? red[lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
  }
}

template <int N, int MODE>
__global__ void __launch_bounds__(col_threads(N), 1) k_col(ColArgs a) {
  constexpr int W = col_w(N);
  constexpr int NT = col_threads(N);
  constexpr int R = regs_for(N);
  constexpr int QR = N / R;
  using L = Layout<N, W, true>;
  extern __shared__ float2 smem[];
  float2* sm = smem;
  float2* tw = smem + L::kSmemElems;
  float* red = reinterpret_cast<float*>(tw + kTwLo + kTwHi);   // 32 floats
  uint32_t* hist = reinterpret_cast<uint32_t*>(red + 32);      // kHistBins (SELECT)

  if constexpr (MODE == COL_REPASS) {
    if (a.ctl->need_repass == 0) return;   // uniform for the whole grid
  }
  if (a.gate && *a.gate != a.gate_val) return;
  load_twiddles(tw, a.tw);
  const int tid = threadIdx.x;
  const int w = tid % W, t = tid / W;
  const int tile = blockIdx.x;
  const int col = tile * W + w;
  const size_t nr = (size_t)a.nr;
  float2 v[R];

  // ------------------------------------------------------------------ input
  if constexpr (MODE == COL_SPARSE_FWD) {
    for (int i = tid; i < L::kSmemElems; i += NT) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const uint32_t e0 = a.xs_off[tile], e1 = a.xs_off[tile + 1];
    for (uint32_t e = e0 + tid; e < e1; e += NT) {
      const uint32_t idx = a.xs_idx[e];
      const int row = (int)(idx / (uint32_t)a.nr);
      const int ww = (int)(idx % (uint32_t)a.nr) - tile * W;
      sm[L::template at<4>(ww, row)] = a.xs_val[e];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = sm[L::template at<4>(w, t + s * QR)];
  } else {
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = __ldcs(&a.in[(size_t)(t + s * QR) * nr + col]);
  }

  // ------------------------------------------------------------------ transforms
  if constexpr (MODE == COL_FWD || MODE == COL_SPARSE_FWD) {
    fft<N, false, L, true>(v, sm, tw, t, w);
#pragma unroll
    for (int s = 0; s < R; ++s) __stcs(&a.out[(size_t)(t + s * QR) * nr + col], v[s]);
  } else if constexpr (MODE == COL_INV) {
    fft<N, true, L, true>(v, sm, tw, t, w);
#pragma unroll
    for (int s = 0; s < R; ++s)
      __stcs(&a.out[(size_t)(t + s * QR) * nr + col], cscale(v[s], a.scale));
  } else if constexpr (MODE == COL_RESID) {
    fft<N, true, L, true>(v, sm, tw, t, w);
    // sampling bits of this thread's R rows, pre-transposed: bit s <-> row t + s*QR
    const uint32_t mbits = __ldg(&a.mask[(size_t)col * QR + t]);
    float acc = 0.f;
    bool bad = false;
    // the echo is read in halves so that at most R/2 loads are in flight per thread
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 yv[R / 2];
#pragma unroll
      for (int u = 0; u < R / 2; ++u)
        yv[u] = __ldcs(&a.y[(size_t)(t + (h * (R / 2) + u) * QR) * nr + col]);
#pragma unroll
      for (int u = 0; u < R / 2; ++u) {
        const int s = h * (R / 2) + u;
        const float2 g = cscale(v[s], a.scale);
        const float2 r = ((mbits >> s) & 1u) ? csub(yv[u], g) : make_float2(0.f, 0.f);
        bad |= !(isfinite(r.x) && isfinite(r.y));
        acc += cabs2(r);
        v[s] = r;
      }
      asm volatile("" ::: "memory");
    }
    if (bad) atomicOr(&a.ctl->err, kErrNonfinite);
    fft<N, false, L, true>(v, sm, tw, t, w);
#pragma unroll
    for (int s = 0; s < R; ++s) __stcs(&a.out[(size_t)(t + s * QR) * nr + col], v[s]);
    const float tot = block_sum<NT>(acc, red);
    if (tid == 0) a.partial[tile] = tot;
  } else if constexpr (MODE == COL_NORM) {
    fft<N, true, L, true>(v, sm, tw, t, w);
    const uint32_t mbits = __ldg(&a.mask[(size_t)col * QR + t]);
    float acc = 0.f;
#pragma unroll
    for (int s = 0; s < R; ++s) acc += ((mbits >> s) & 1u) ? cabs2(cscale(v[s], a.scale)) : 0.f;
    const float tot = block_sum<NT>(acc, red);
    if (tid == 0) a.partial[tile] = tot;
  } else {  // COL_SELECT / COL_REPASS
    constexpr bool HIST = (MODE == COL_SELECT);
    if constexpr (HIST) {
      for (int i = tid; i < (int)kHistBins; i += NT) hist[i] = 0u;
    }
    fft<N, true, L, true>(v, sm, tw, t, w);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < R; ++s) sm[L::template at<4>(w, t + s * QR)] = cscale(v[s], a.scale);
    __syncthreads();
    // support of the current iterate: record Delta X there, exclude from candidates
    const uint32_t e0 = a.xs_off[tile], e1 = a.xs_off[tile + 1];
    for (uint32_t e = e0 + tid; e < e1; e += NT) {
      const uint32_t idx = a.xs_idx[e];
      const int row = (int)(idx / (uint32_t)a.nr);
      const int ww = (int)(idx % (uint32_t)a.nr) - tile * W;
      const int p = L::template at<4>(ww, row);
      if constexpr (HIST) a.xs_dx[e] = sm[p];
      sm[p] = make_float2(__int_as_float(0x7fffffff), 0.f);
    }
    __syncthreads();
    const uint32_t cut = a.ctl->cut_key;
    constexpr uint32_t full = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
    const int lane = tid & 31;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const int row = t + s * QR;
      const float2 d = sm[L::template at<4>(w, row)];
      const bool on_support = isnan(d.x);
      const uint32_t key = __float_as_uint(cabs2(d)) & 0x7fffffffu;
      if constexpr (HIST) {
        if (!on_support) atomicAdd(&hist[key >> kHistShift], 1u);
      }
      const bool take = !on_support && key >= cut && key >= kMinKey;
      const uint32_t bal = __ballot_sync(full, take);
      if (bal) {
        const int leader = __ffs(bal) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&a.ctl->cand_count, (uint32_t)__popc(bal));
        base = __shfl_sync(full, base, leader);
        if (take) {
          const uint32_t pos = base + __popc(bal & ((1u << lane) - 1u));
          if (pos < a.cand_cap) {
            a.cand_idx[pos] = (uint32_t)((size_t)row * nr + col);
            a.cand_val[pos] = d;
          }
        }
      }
    }
    if constexpr (HIST) {
      __syncthreads();
      for (int i = tid; i < (int)kHistBins; i += NT) {
        const uint32_t h = hist[i];
        if (h) atomicAdd(&a.hist[i], h);
      }
    }
  }
}

// Sampling mask in the column passes' register order: word (col, t) holds the bits
// of rows t + s*(N/R), s = 0..R-1 (bit s), so a thread reads one word per pass.
template <int N>
__global__ void k_mask_transpose(const uint32_t* __restrict__ mask, uint32_t* __restrict__ mask_t,
                                 int nr) {
  constexpr int R = regs_for(N);
  constexpr int QR = N / R;
  const size_t total = (size_t)nr * QR;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(i / QR), t = (int)(i % QR);
    uint32_t wbits = 0u;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const size_t idx = (size_t)(t + s * QR) * nr + col;
      wbits |= ((__ldg(&mask[idx >> 5]) >> (idx & 31)) & 1u) << s;
    }
    mask_t[i] = wbits;
  }
}

template <int N>
static size_t col_smem(int mode) {
  using L = Layout<N, col_w(N), true>;
  size_t b = (size_t)L::kSmemElems * sizeof(float2) + (kTwLo + kTwHi) * sizeof(float2) +
             32 * sizeof(float);
  if (mode == COL_SELECT) b += kHistBins * sizeof(uint32_t);
  return b;
}

template <int N>
static cudaError_t col_attrs() {
  cudaError_t e = cudaSuccess;
#define CSAR_ATTR(M)                                                                  \
  if (e == cudaSuccess)                                                               \
    e = cudaFuncSetAttribute(k_col<N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)col_smem<N>(M));
  CSAR_ATTR(COL_FWD)
  CSAR_ATTR(COL_INV)
  CSAR_ATTR(COL_SPARSE_FWD)
  CSAR_ATTR(COL_RESID)
  CSAR_ATTR(COL_SELECT)
  CSAR_ATTR(COL_REPASS)
  CSAR_ATTR(COL_NORM)
#undef CSAR_ATTR
  return e;
}

template <int N>
static cudaError_t col_launch(ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s) {
  const dim3 grid(n_tiles), block(col_threads(N));
  const size_t sm = col_smem<N>(mode);
  switch (mode) {
    case COL_FWD: k_col<N, COL_FWD><<<grid, block, sm, s>>>(a); break;
    case COL_INV: k_col<N, COL_INV><<<grid, block, sm, s>>>(a); break;
    case COL_SPARSE_FWD: k_col<N, COL_SPARSE_FWD><<<grid, block, sm, s>>>(a); break;
    case COL_RESID: k_col<N, COL_RESID><<<grid, block, sm, s>>>(a); break;
    case COL_SELECT: k_col<N, COL_SELECT><<<grid, block, sm, s>>>(a); break;
    case COL_REPASS: k_col<N, COL_REPASS><<<grid, block, sm, s>>>(a); break;
    case COL_NORM: k_col<N, COL_NORM><<<grid, block, sm, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#define CSAR_COL_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

cudaError_t col_set_attributes(int na) {
  switch (na) {
#define CSAR_CASE(N) \
  case N: return col_attrs<N>();
    CSAR_COL_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mask_transpose(int na, int nr, const uint32_t* mask, uint32_t* mask_t,
                                  cudaStream_t s) {
  switch (na) {
#define CSAR_CASE(N)                                                          \
  case N:                                                                     \
    k_mask_transpose<N><<<1024, 256, 0, s>>>(mask, mask_t, nr);               \
    return cudaGetLastError();
    CSAR_COL_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col(int na, ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s) {
  switch (na) {
#define CSAR_CASE(N) \
  case N: return col_launch<N>(mode, a, n_tiles, s);
    CSAR_COL_SIZES(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace csar
