// col_pass.cuh — azimuth (column, strided-axis) passes.
//
// A column transform of length N_a is split over a thread-block cluster of P CTAs
// (P = 4 at N_a = 8192, 2 at 4096, else 1 by default), that together own a tile of
// W >= 4 adjacent columns (32-byte row segments, full DRAM sectors).  With N_a = P * Q,
// each CTA keeps E = Q*W complex64 values in registers: 8192 (64 KiB, two CTAs per SM,
// so one CTA's loads overlap the other's arithmetic), 4096 (four per SM) or 16384 (one
// per SM, 8- or 16-column tiles).
//
// Forward/inverse transform "BS" (blocked rows in, strided rows out):
//   CTA c loads rows Q*n1 + n2 for its block of n2 (all n1), does the length-P DFT
//   over n1 and the twiddle W_N^(n2 k1) in registers, and pushes output k1 into the
//   shared memory of CTA k1 (distributed shared memory); after a cluster barrier
//   every CTA runs the length-Q Stockham FFT (fft.cuh) and holds rows k1 + P*k2.
// Forward transform "SB" (strided rows in, blocked rows out), used after the
// residue so no extra exchange is needed: the local length-Q FFT first, twiddle
// W_N^(c k2), push to the CTA owning k2, cluster barrier, length-P DFT.
//
// Modes (the fused work of one ITA iteration, Algorithm 1 / Eq. (25)):
//   COL_FWD / COL_INV      plain azimuth FFT / IFFT (operators G and M)
//   COL_SPARSE_FWD         the K-sparse iterate scattered into a zero tile, then FFT
//   COL_RESID              IFFT -> G(X); mask S; FFT -> F_a(S.G(X)) (the next range
//                          pass subtracts it from F_a(S.Y): F_a of the residue)
//   COL_SELECT / REPASS    IFFT -> Delta X = M(r); Delta X at the support; histogram
//                          of |Delta X|^2 keys and compaction of the candidates for
//                          the (K+1)-th magnitude (Section IV-B)
//   COL_NORM               IFFT -> G(Delta X_Gamma); sum of S.|.|^2 (NIHT step)
#pragma once
#include <cooperative_groups.h>


#include "fft.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace cg = cooperative_groups;

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

template <int N, int P_, int E_ = kColCtaElems>
struct ColCfg {
  static constexpr int P = P_;
  static constexpr int E = E_;
  static constexpr int Q = N / P;
  static constexpr int W = col_w(N, P, E);
  static constexpr int R = col_regs(Q);
  static constexpr int QR = Q / R;
  static constexpr int NT = QR * W;
  static constexpr int RP = R / P;   // n2 values per thread in the cross-CTA step
};

// Cluster barrier (all CTAs of the cluster; release/acquire on shared memory).
template <int P>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (P > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------- cluster exchanges
// The cross-CTA steps move data with plain remote stores into the peers' shared memory
// and signal with single-use mbarriers (one per exchange, P arrivals each) instead of
// full cluster barriers: after a CTA-wide __syncthreads, thread k alone performs a
// release arrive (cluster scope) on the mbarrier of CTA k, and every thread waits on its
// own mbarrier with acquire semantics.  Only P threads per CTA execute a cluster-scope
// release, and loads issued before the wait are not held back by it.
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float2 x) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x.x), "f"(x.y) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t remote) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}
// Signal on mbarrier `mb` (local address; the same offset in every CTA) of all P CTAs
// that this CTA's prior shared-memory work (remote stores, or reads of its own buffer)
// is complete.
template <int P>
__device__ __forceinline__ void xch_signal(uint32_t mb, int rank0) {
  __syncthreads();
  if (threadIdx.x < P) mbar_arrive_cluster(cluster_map(mb, rank0 + (int)threadIdx.x));
}

// Mbarriers of the column pass (single use, phase 0, P arrivals each).
enum : int { kMbBs = 0, kMbFree = 1, kMbSb = 2, kMbCount = 4 };

// Cross-CTA step of the blocked-in transform: v holds, per i < RP, the P values
// n1 = 0..P-1 of n2 = c*Q/P + t + QR*i; their length-P DFT (times W_N^(n2 k1)) is
// pushed to element n2 of CTA k1.  Then the canonical input of the local FFT is read.
// The twiddles W_N^(n2 k1) are W^(n2 k1) = w1^k1 (w1 = W^n2 from the table) within
// each group of four k1, re-anchored from the table at every multiple of four.
template <int N, int P, int E, bool INV>
__device__ __forceinline__ void bs_cross(float2 (&v)[ColCfg<N, P, E>::R], float2* sm, const float2* tw,
                                         int c, int t, int w, const uint32_t (&peer)[P],
                                         uint32_t mb, Ctl* ctl, int rank0) {
  using C = ColCfg<N, P, E>;
  using L = Layout<C::Q, C::W, true>;
  if constexpr (C::P > 1) {
#pragma unroll
    for (int i = 0; i < C::RP; ++i) {
      const int n2 = c * (C::Q / C::P) + t + C::QR * i;
      float2 a[C::P];
#pragma unroll
      for (int n1 = 0; n1 < C::P; ++n1) a[n1] = v[i * C::P + n1];
      Dft<C::P, INV>::run(a);
      const float2 w1 = twiddle_tab<INV>(tw, n2 * (kTwN / N));
      float2 wp[4];
      wp[0] = make_float2(1.f, 0.f);
      wp[1] = w1;
      wp[2] = cmul(w1, w1);
      wp[3] = cmul(wp[2], w1);
      const uint32_t off = 8u * (uint32_t)L::template at<4>(w, n2);
      float2 anc = wp[0];
#pragma unroll
      for (int k1 = 0; k1 < C::P; ++k1) {
        if (k1 >= 4 && k1 % 4 == 0) anc = twiddle_tab<INV>(tw, n2 * k1 * (kTwN / N));
        const float2 tk = (k1 % 4 == 0) ? anc : (k1 < 4 ? wp[k1] : cmul(anc, wp[k1 % 4]));
        st_cluster(peer[k1] + off, k1 ? cmul(a[k1], tk) : a[k1]);
      }
    }
    xch_signal<C::P>(mb, rank0);
    mbar_wait(mb, 0u, ctl);
#pragma unroll
    for (int s = 0; s < C::R; ++s) v[s] = sm[L::template at<4>(w, t + s * C::QR)];
  }
}

// Global row of v-slot s before the cross step (blocked input) for CTA c.
template <int N, int P, int E>
__device__ __forceinline__ int bs_in_row(int c, int t, int s) {
  using C = ColCfg<N, P, E>;
  if constexpr (C::P == 1) {
    return t + s * C::QR;
  } else {
    const int i = s / C::P, n1 = s % C::P;
    return C::Q * n1 + c * (C::Q / C::P) + t + C::QR * i;
  }
}

// Global row of canonical slot s after the local FFT (strided output) for CTA c.
template <int N, int P, int E>
__device__ __forceinline__ int strided_row(int c, int t, int s) {
  using C = ColCfg<N, P, E>;
  return c + C::P * (t + s * C::QR);
}

// Place of a CTA in its pass: rank c in the group of P CTAs that transforms one tile, the
// tile, the cluster rank of the group's first CTA (peers are rank0 + k) and the CTA's
// index in the pass (its slot in per-CTA partial sums).  For a pass launched alone the
// group is the hardware cluster and all four come from the block index, read where used.
template <int P>
struct ColOfGrid {
  __device__ __forceinline__ int c() const { return (int)(blockIdx.x % P); }
  __device__ __forceinline__ int tile() const { return (int)(blockIdx.x / P); }
  __device__ __forceinline__ int rank0() const { return 0; }
  __device__ __forceinline__ int cta() const { return (int)blockIdx.x; }
};
struct ColOfItem {
  int c_, tile_, rank0_, cta_;
  __device__ __forceinline__ int c() const { return c_; }
  __device__ __forceinline__ int tile() const { return tile_; }
  __device__ __forceinline__ int rank0() const { return rank0_; }
  __device__ __forceinline__ int cta() const { return cta_; }
};

template <int N, int P, int E, int MODE, class WH>
__device__ __forceinline__ void col_body(const ColArgs& a, WH wh) {
#include "col_body.inc"
}

// The per-pass kernel carries the statements itself (not a call of col_body), which keeps
// the kernel parameter in the parameter space and the register allocation of the hot
// passes unchanged.
template <int N, int P, int E, int MODE>
__global__ void __launch_bounds__(ColCfg<N, P, E>::NT, col_ctas_per_sm(E)) k_col(ColArgs a) {
  const ColOfGrid<P> wh{};
#include "col_body.inc"
}

// Sampling mask in the residual pass's register order: word ((col*P + c)*QR + t) holds
// the bits of rows c + P*(t + s*QR), s = 0..R-1 (bit s).
template <int N, int P>
__global__ void k_mask_transpose(const uint32_t* __restrict__ mask, uint32_t* __restrict__ mask_t,
                                 int nr) {
  using C = ColCfg<N, P>;
  const size_t total = (size_t)nr * C::P * C::QR;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(i % C::QR);
    const int c = (int)((i / C::QR) % C::P);
    const int col = (int)(i / ((size_t)C::QR * C::P));
    uint32_t wbits = 0u;
#pragma unroll
    for (int s = 0; s < C::R; ++s) {
      const size_t idx = (size_t)(c + C::P * (t + s * C::QR)) * nr + col;
      wbits |= ((__ldg(&mask[idx >> 5]) >> (idx & 31)) & 1u) << s;
    }
    mask_t[i] = wbits;
  }
}

template <int N, int P, int E>
static size_t col_smem(int mode) {
  using C = ColCfg<N, P, E>;
  using L = Layout<C::Q, C::W, true>;
  size_t b = (size_t)L::kSmemElems * sizeof(float2) + (kTwLo + kTwHi) * sizeof(float2) +
             32 * sizeof(float) + kMbCount * sizeof(uint64_t);
  if (mode == COL_SELECT || mode == COL_REPASS) b += (kHistBins + C::NT) * sizeof(uint32_t);
  return b;
}

template <int N, int P, int E, int MODE>
static cudaError_t col_launch_mode(const ColArgs& a, int n_tiles, cudaStream_t s) {
  using C = ColCfg<N, P, E>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_tiles * C::P);
  cfg.blockDim = dim3(C::NT);
  cfg.dynamicSmemBytes = col_smem<N, P, E>(MODE);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C::P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_col<N, P, E, MODE>, a);
}

template <int N, int P, int E>
static cudaError_t col_attrs() {
  cudaError_t e = cudaSuccess;
#define CSAR_ATTR(M)                                                                          \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(k_col<N, P, E, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             (int)col_smem<N, P, E>(M));                                      \
  if (e == cudaSuccess && P > 8)                                                              \
    e = cudaFuncSetAttribute(k_col<N, P, E, M>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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

template <int N, int P, int E>
static cudaError_t col_launch(ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s) {
  switch (mode) {
    case COL_FWD: return col_launch_mode<N, P, E, COL_FWD>(a, n_tiles, s);
    case COL_INV: return col_launch_mode<N, P, E, COL_INV>(a, n_tiles, s);
    case COL_SPARSE_FWD: return col_launch_mode<N, P, E, COL_SPARSE_FWD>(a, n_tiles, s);
    case COL_RESID: return col_launch_mode<N, P, E, COL_RESID>(a, n_tiles, s);
    case COL_SELECT: return col_launch_mode<N, P, E, COL_SELECT>(a, n_tiles, s);
    case COL_REPASS: return col_launch_mode<N, P, E, COL_REPASS>(a, n_tiles, s);
    case COL_NORM: return col_launch_mode<N, P, E, COL_NORM>(a, n_tiles, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, int P>
static cudaError_t mask_transpose(int nr, const uint32_t* mask, uint32_t* mask_t, cudaStream_t s) {
  k_mask_transpose<N, P><<<1024, 256, 0, s>>>(mask, mask_t, nr);
  return cudaGetLastError();
}

// Entry points of one (N, P, E) instantiation, used by the dispatcher in col_dispatch.cu.
// The column-order sampling mask depends on (N, P) only.
#define CSAR_COL_INSTANTIATE(N, P, E)                                                              \
  cudaError_t col_attrs_##N##_##P##_##E() { return col_attrs<N, P, E>(); }                         \
  cudaError_t col_launch_##N##_##P##_##E(ColMode m, const ColArgs& a, int nt, cudaStream_t s) {    \
    return col_launch<N, P, E>(m, a, nt, s);                                                       \
  }
#define CSAR_COL_MASK_INSTANTIATE(N, P)                                                            \
  cudaError_t col_mask_##N##_##P(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s) {       \
    return mask_transpose<N, P>(nr, mk, mt, s);                                                    \
  }

}  // namespace csar
