// colp_pass.cuh — persistent azimuth (column) passes fed by tensor-memory-access copies.
//
// Same transforms and fused work as k_col (col_pass.cuh) for the modes COL_FWD, COL_INV,
// COL_RESID and COL_SELECT, but each cluster of P CTAs stays resident and walks the
// column tiles tile = cluster, cluster + clusters, ...  While a tile is transformed, the
// CTA's block of the next tile is already on its way into a landing buffer: P (or
// 2P) two-dimensional bulk tensor copies (cp.async.bulk.tensor, boxes of W columns x up
// to 256 rows of this GPU's own memory, no multicast) that complete on an mbarrier.  So
// the loads of a tile overlap the arithmetic of the previous one, the CTA issues a few
// copy instructions instead of one load per element, and the twiddle table and the
// mbarriers are set up once per CTA instead of once per tile.
//
// Shared memory per CTA: the landing buffer (E values), the exchange buffer of the
// cross-CTA steps and the local FFT (as in k_col), twiddles, the mbarriers and the
// selection's support words.  The selection histogram lives in the exchange buffer once
// a tile's transform is done and is flushed (non-zero bins only) per tile.
//
// Per tile, with k the CTA's tile count (every mbarrier completes once per tile, so it
// is waited on with parity k & 1):
//   full      the tile's landing copies have arrived (1 arrival + transaction bytes)
//   ready_bs  every peer has pushed its blocked-input DFT outputs into this CTA
//   free_b    (COL_RESID) every CTA of the cluster has finished its local FFTs
//   ready_sb  (COL_RESID) every peer has pushed its strided-input outputs
//   free_a    every CTA has finished reading its exchange buffer for the tile, so the
//             next tile's pushes may start (waited on before the next push, and once
//             more before the CTA exits, so no remote arrive is still on its way)
// Every wait is bounded (one second), latches CSAR_E_TIMEOUT in the control block and
// goes on; a CTA that finds the timeout latched leaves at its next tile boundary, so a
// failed cluster ends within a few bounded waits.
#pragma once
#include <cuda.h>

#include "col_pass.cuh"

namespace csar {

// mbarrier slots of the persistent column pass
enum : int { kPbFull = 0, kPbReadyBs = 1, kPbReadySb = 2, kPbFreeA = 3, kPbFreeB = 4, kPbCount = 6 };

__device__ __forceinline__ void mbar_expect_tx(uint32_t mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}

// Tiled 2-D bulk tensor copy of the box at (x, y) = (column, row) of `map` into this
// CTA's shared memory at `dst`, completing `mb`'s transaction count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mb)
      : "memory");
}

template <int N, int P, int E>
struct ColpCfg {
  using C = ColCfg<N, P, E>;
  static constexpr int QB = C::Q / P;                 // rows per n1 block of the blocked input
  static constexpr int BR = QB < 256 ? QB : 256;      // rows per tensor box
  static constexpr int NB = QB / BR;                  // boxes per block
  static constexpr int kLandElems = E;                // = P * QB * W
};

template <int N, int P, int E>
__host__ __device__ constexpr size_t colp_smem() {
  using C = ColCfg<N, P, E>;
  using L = Layout<C::Q, C::W, true>;
  return (size_t)E * sizeof(float2) + (size_t)L::kSmemElems * sizeof(float2) +
         (kTwLo + kTwHi) * sizeof(float2) + 32 * sizeof(float) + kPbCount * sizeof(uint64_t) +
         (size_t)C::NT * sizeof(uint32_t);
}

// One thread: expect the tile's bytes on `full` and start its P * NB box copies (block
// n1 = rows Q n1 + c QB .. + QB of columns tile W .. + W) into the landing buffer.
template <int N, int P, int E>
__device__ __forceinline__ void colp_issue(const CUtensorMap* map, uint32_t land, uint32_t full, int tile, int c) {
  using C = ColCfg<N, P, E>;
  using PC = ColpCfg<N, P, E>;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(full, (uint32_t)(E * sizeof(float2)));
#pragma unroll
  for (int n1 = 0; n1 < P; ++n1)
#pragma unroll
    for (int b = 0; b < PC::NB; ++b)
      tma_load_2d(land + (uint32_t)((n1 * PC::QB + b * PC::BR) * C::W * sizeof(float2)), map, tile * C::W,
                  n1 * C::Q + c * PC::QB + b * PC::BR, full);
}

// Signal mbarrier `mb` of every CTA of the cluster (thread k arrives on CTA k) after a
// CTA-wide barrier: this CTA's prior shared-memory work for the exchange is complete.
template <int P>
__device__ __forceinline__ void colp_signal(uint32_t mb) {
  __syncthreads();
  if (threadIdx.x < P) mbar_arrive_cluster(cluster_map(mb, (int)threadIdx.x));
}

// resident CTAs per SM the register allocation is sized for (shared memory: ~69 KB per
// CTA of 4096 values, ~137 KB per CTA of 8192)
__host__ __device__ constexpr int colp_ctas_per_sm(int e) { return e <= 4096 ? 3 : 1; }

template <int N, int P, int E, int MODE>
__global__ void __launch_bounds__(ColCfg<N, P, E>::NT, colp_ctas_per_sm(E))
    k_colp(const __grid_constant__ CUtensorMap tin, ColArgs a, int n_tiles) {
  static_assert(MODE == COL_FWD || MODE == COL_INV || MODE == COL_RESID || MODE == COL_SELECT, "mode");
  using C = ColCfg<N, P, E>;
  using PC = ColpCfg<N, P, E>;
  constexpr int W = C::W, R = C::R, QR = C::QR, NT = C::NT, Q = C::Q, RP = C::RP, QB = PC::QB;
  constexpr bool INV = MODE != COL_FWD;
  using L = Layout<Q, W, true>;
  extern __shared__ __align__(128) float2 smem[];
  float2* land = smem;
  float2* sm = smem + E;
  float2* tw = sm + L::kSmemElems;
  float* red = reinterpret_cast<float*>(tw + kTwLo + kTwHi);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(red + 32);
  uint32_t* msk = reinterpret_cast<uint32_t*>(mbar + kPbCount);
  (void)red;

  if (a.gate && *a.gate != a.gate_val) return;   // uniform for the grid
  const int c = (P > 1) ? (int)(blockIdx.x % P) : 0;
  const int cl = (int)(blockIdx.x / P), n_cl = (int)(gridDim.x / P);
  const int tid = threadIdx.x;
  const int w = tid % W, t = tid / W;
  const size_t nr = (size_t)a.nr;
  const uint32_t mb0 = smem_addr(mbar);
  const uint32_t mb_full = mb0 + 8u * kPbFull, mb_rbs = mb0 + 8u * kPbReadyBs,
                 mb_rsb = mb0 + 8u * kPbReadySb, mb_fa = mb0 + 8u * kPbFreeA, mb_fb = mb0 + 8u * kPbFreeB;
  const uint32_t land_a = smem_addr(land);
  if (tid == 0) {
    mbar_init(mb_full, 1u);
#pragma unroll
    for (int j = 1; j < 5; ++j) mbar_init(mb0 + 8u * j, (uint32_t)P);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tin)) : "memory");
  }
  uint32_t peer[P];
#pragma unroll
  for (int k = 0; k < P; ++k) peer[k] = P > 1 ? cluster_map(smem_addr(sm), k) : smem_addr(sm);
  load_twiddles(tw, a.tw);
  // every CTA of the cluster has initialised its mbarriers before any remote arrive
  if constexpr (P > 1) {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
  } else {
    __syncthreads();
  }
  if (tid == 0 && cl < n_tiles) colp_issue<N, P, E>(&tin, land_a, mb_full, cl, c);
  const uint32_t sel_cut = (MODE == COL_SELECT) ? a.ctl->cut_key : 0u;

  uint32_t k = 0;
  for (int tile = cl; tile < n_tiles; tile += n_cl, ++k) {
    const uint32_t ph = k & 1u;
    const int col = tile * W + w;
    // a latched timeout (this CTA or any other) ends the pass at a tile boundary, once
    // the copies already issued for this tile have landed (bounded wait)
    if (__syncthreads_or(tid == 0 && a.ctl && (*(volatile uint32_t*)&a.ctl->err & kErrTimeout))) {
      mbar_wait_for(mb_full, ph, 1000000000ull);
      break;
    }
    uint32_t mbits = 0u;
    if constexpr (MODE == COL_RESID) mbits = __ldg(&a.mask[((size_t)col * P + c) * QR + t]);
    uint32_t sel_e0 = 0u, sel_e1 = 0u, sel_idx = 0u;
    if constexpr (MODE == COL_SELECT) {
      sel_e0 = a.xs_off[tile];
      sel_e1 = a.xs_off[tile + 1];
      if (sel_e0 + tid < sel_e1) sel_idx = a.xs_idx[sel_e0 + tid];
      msk[tid] = 0u;
    }
    // ---------------------------------------------------------------- the tile's block
    mbar_wait(mb_full, ph, a.ctl);
    float2 v[R];
#pragma unroll
    for (int i = 0; i < RP; ++i)
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) v[i * P + n1] = land[(n1 * QB + t + QR * i) * W + w];
    __syncthreads();   // the landing buffer is free: start the next tile's copies
    if (tid == 0 && tile + n_cl < n_tiles) colp_issue<N, P, E>(&tin, land_a, mb_full, tile + n_cl, c);

    // ---------------------------------------------------------------- cross step (BS)
    if constexpr (P > 1) {
      // length-P DFT over n1 and twiddle W_N^(n2 k1) in place: v[i P + k1] goes to CTA k1
#pragma unroll
      for (int i = 0; i < RP; ++i) {
        const int n2 = c * QB + t + QR * i;
        float2 d[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) d[n1] = v[i * P + n1];
        Dft<P, INV>::run(d);
        const float2 w1 = twiddle_tab<INV>(tw, n2 * (kTwN / N));
        float2 wp[4];
        wp[0] = make_float2(1.f, 0.f);
        wp[1] = w1;
        wp[2] = cmul(w1, w1);
        wp[3] = cmul(wp[2], w1);
        float2 anc = wp[0];
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
          if (k1 >= 4 && k1 % 4 == 0) anc = twiddle_tab<INV>(tw, n2 * k1 * (kTwN / N));
          const float2 tk = (k1 % 4 == 0) ? anc : (k1 < 4 ? wp[k1] : cmul(anc, wp[k1 % 4]));
          v[i * P + k1] = k1 ? cmul(d[k1], tk) : d[k1];
        }
      }
      // the peers' exchange buffers are free once every CTA has finished the last tile
      if (k > 0) mbar_wait(mb_fa, (k - 1u) & 1u, a.ctl);
#pragma unroll
      for (int i = 0; i < RP; ++i) {
        const int n2 = c * QB + t + QR * i;
        const uint32_t off = 8u * (uint32_t)L::template at<4>(w, n2);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) st_cluster(peer[k1] + off, v[i * P + k1]);
      }
      colp_signal<P>(mb_rbs);
      mbar_wait(mb_rbs, ph, a.ctl);
#pragma unroll
      for (int s = 0; s < R; ++s) v[s] = sm[L::template at<4>(w, t + s * QR)];
    }

    // ---------------------------------------------------------------- transform + epilogue
    if constexpr (MODE == COL_FWD || MODE == COL_INV) {
      fft<Q, INV, L, true, R>(v, sm, tw, t, w);
#pragma unroll
      for (int s = 0; s < R; ++s)
        __stcs(&a.out[(size_t)strided_row<N, P, E>(c, t, s) * nr + col], INV ? cscale(v[s], a.scale) : v[s]);
      if constexpr (P > 1) colp_signal<P>(mb_fa);
    } else if constexpr (MODE == COL_RESID) {
      fft<Q, true, L, true, R>(v, sm, tw, t, w);
#pragma unroll
      for (int s = 0; s < R; ++s)
        v[s] = ((mbits >> s) & 1u) ? cscale(v[s], a.scale) : make_float2(0.f, 0.f);
      fft<Q, false, L, true, R>(v, sm, tw, t, w);
      if constexpr (P == 1) {
#pragma unroll
        for (int s = 0; s < R; ++s) __stcs(&a.out[(size_t)(t + s * QR) * nr + col], v[s]);
      } else {
        // SB step as in k_col: twiddle W_N^(c k2), push k2 to CTA s / RP, once every CTA
        // of the cluster has finished its local transforms
        colp_signal<P>(mb_fb);
        mbar_wait(mb_fb, ph, a.ctl);
        {
          float2 stp[4];
          stp[0] = make_float2(1.f, 0.f);
          stp[1] = twiddle_tab<false>(tw, c * QR * (kTwN / N));
          stp[2] = cmul(stp[1], stp[1]);
          stp[3] = cmul(stp[2], stp[1]);
          float2 anc = stp[0];
#pragma unroll
          for (int s = 0; s < R; ++s) {
            if (s % 4 == 0) anc = twiddle_tab<false>(tw, c * (t + s * QR) * (kTwN / N));
            const float2 x = c ? cmul(v[s], (s % 4 == 0) ? anc : cmul(anc, stp[s % 4])) : v[s];
            const int dst = s / RP, k2l = t + QR * (s % RP);
            st_cluster(peer[dst] + 8u * (uint32_t)L::template at<4>(w, c * QB + k2l), x);
          }
        }
        colp_signal<P>(mb_rsb);
        mbar_wait(mb_rsb, ph, a.ctl);
        float2* oc = a.out + (size_t)(c * QB + t) * nr + col;
        const size_t di = (size_t)QR * nr, dk = (size_t)Q * nr;
#pragma unroll
        for (int i = 0; i < RP; ++i) {
          const int k2l = t + QR * i;
          float2 b[P];
#pragma unroll
          for (int n1 = 0; n1 < P; ++n1) b[n1] = sm[L::template at<4>(w, n1 * QB + k2l)];
          Dft<P, false>::run(b);
#pragma unroll
          for (int k1 = 0; k1 < P; ++k1) __stcs(oc + i * di + k1 * dk, b[k1]);
        }
        colp_signal<P>(mb_fa);
      }
    } else {  // COL_SELECT
      fft<Q, true, L, true, R>(v, sm, tw, t, w);
      // support of the current iterate (bit m / QR of word (m % QR) W + w for local row m)
      const uint32_t first_idx = sel_idx;
      for (uint32_t e = sel_e0 + tid; e < sel_e1; e += NT) {
        const uint32_t idx = sel_idx;
        if (e + NT < sel_e1) sel_idx = a.xs_idx[e + NT];
        const int row = (int)(idx / (uint32_t)a.nr);
        if (P > 1 && row % P != c) continue;
        const int ww = (int)(idx % (uint32_t)a.nr) - tile * W;
        const int m = row / P;
        atomicOr(&msk[(m % QR) * W + ww], 1u << (m / QR));
      }
      __syncthreads();
      const uint32_t sup = msk[tid];
      // Delta X at the support: through the exchange buffer to the entry's thread
      if (sup) {
#pragma unroll
        for (int s = 0; s < R; ++s)
          if ((sup >> s) & 1u) sm[L::template at<4>(w, t + s * QR)] = cscale(v[s], a.scale);
      }
      __syncthreads();
      for (uint32_t e = sel_e0 + tid; e < sel_e1; e += NT) {
        const uint32_t idx = e == sel_e0 + tid ? first_idx : a.xs_idx[e];
        const int row = (int)(idx / (uint32_t)a.nr);
        if (P > 1 && row % P != c) continue;
        const int ww = (int)(idx % (uint32_t)a.nr) - tile * W;
        a.xs_dx[e] = sm[L::template at<4>(ww, row / P)];
      }
      __syncthreads();
      // histogram of off-support keys >= hist_floor(cut) (windowed as in k_col), in the
      // exchange buffer; candidates >= cut compacted by warp ballot
      uint32_t* hist = reinterpret_cast<uint32_t*>(sm);
      const uint32_t floor_key = hist_floor(sel_cut);
      const int hb0 = (int)(floor_key >> kHistShift);
      const int nbins = floor_key == 0u ? (int)kHistBins
                                        : ((int)kHistBins - hb0 < kHistWindow ? (int)kHistBins - hb0 : kHistWindow);
      for (int i = tid; i < nbins; i += NT) hist[i] = 0u;
      __syncthreads();
      constexpr uint32_t full = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
      const int lane = tid & 31;
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const int m = t + s * QR;
        const float2 d = cscale(v[s], a.scale);
        const bool on_support = (sup >> s) & 1u;
        const uint32_t key = __float_as_uint(cabs2(d)) & 0x7fffffffu;
        if (!on_support && key >= floor_key) {
          const int hb = (int)(key >> kHistShift) - hb0;
          atomicAdd(&hist[hb < nbins ? hb : nbins - 1], 1u);
        }
        const bool take = !on_support && key >= sel_cut && key >= kMinKey;
        const uint32_t bal = __ballot_sync(full, take);
        if (bal) {
          const int leader = __ffs(bal) - 1;
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(&a.ctl->cand_count, (uint32_t)__popc(bal));
          base = __shfl_sync(full, base, leader);
          if (take) {
            const uint32_t pos = base + __popc(bal & ((1u << lane) - 1u));
            if (pos < a.cand_cap) {
              a.cand_idx[pos] = (uint32_t)((size_t)(c + P * m) * nr + col);
              a.cand_val[pos] = d;
            }
          }
        }
      }
      __syncthreads();
      for (int i = tid; i < nbins; i += NT) {
        const uint32_t h = hist[i];
        if (h) atomicAdd(&a.hist[hb0 + i], h);
      }
      if constexpr (P > 1) colp_signal<P>(mb_fa);
      else __syncthreads();   // the histogram is read before the next tile's FFT writes
    }
  }
  // no CTA leaves while a peer may still arrive on its mbarriers: the last free_a phase
  // completes only after every peer's last remote operation into this CTA
  if constexpr (P > 1) {
    if (k > 0) mbar_wait(mb_fa, (k - 1u) & 1u, a.ctl);
  }
}

// ---------------------------------------------------------------- host side
template <int N, int P, int E, int MODE>
static cudaError_t colp_attrs_mode() {
  cudaError_t e = cudaFuncSetAttribute(k_colp<N, P, E, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)colp_smem<N, P, E>());
  if (e == cudaSuccess && P > 8)
    e = cudaFuncSetAttribute(k_colp<N, P, E, MODE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <int N, int P, int E>
static cudaError_t colp_attrs() {
  cudaError_t e = colp_attrs_mode<N, P, E, COL_FWD>();
  if (e == cudaSuccess) e = colp_attrs_mode<N, P, E, COL_INV>();
  if (e == cudaSuccess) e = colp_attrs_mode<N, P, E, COL_RESID>();
  if (e == cudaSuccess) e = colp_attrs_mode<N, P, E, COL_SELECT>();
  return e;
}

// Launch with as many clusters as can be resident at once (queried once per
// instantiation), each walking its share of the n_tiles column tiles.
template <int N, int P, int E, int MODE>
static cudaError_t colp_launch_mode(const CUtensorMap& map, const ColArgs& a, int n_tiles, cudaStream_t s) {
  using C = ColCfg<N, P, E>;
  static int resident = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(C::NT);
  cfg.dynamicSmemBytes = colp_smem<N, P, E>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (resident <= 0) {
    cfg.gridDim = dim3(P);
    int nc = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, k_colp<N, P, E, MODE>, &cfg);
    if (e != cudaSuccess) return e;
    if (nc <= 0) return cudaErrorInvalidConfiguration;
    resident = nc;
  }
  const int clusters = n_tiles < resident ? n_tiles : resident;
  cfg.gridDim = dim3((unsigned)(clusters * P));
  return cudaLaunchKernelEx(&cfg, k_colp<N, P, E, MODE>, map, a, n_tiles);
}

template <int N, int P, int E>
static cudaError_t colp_launch(ColMode mode, const CUtensorMap& map, const ColArgs& a, int n_tiles,
                               cudaStream_t s) {
  switch (mode) {
    case COL_FWD: return colp_launch_mode<N, P, E, COL_FWD>(map, a, n_tiles, s);
    case COL_INV: return colp_launch_mode<N, P, E, COL_INV>(map, a, n_tiles, s);
    case COL_RESID: return colp_launch_mode<N, P, E, COL_RESID>(map, a, n_tiles, s);
    case COL_SELECT: return colp_launch_mode<N, P, E, COL_SELECT>(map, a, n_tiles, s);
    default: return cudaErrorInvalidValue;
  }
}

// Box of the landing copies of one (N, P, E) instantiation: W columns x BR rows.
template <int N, int P, int E>
static void colp_box(int* cols, int* rows) {
  *cols = ColCfg<N, P, E>::W;
  *rows = ColpCfg<N, P, E>::BR;
}

#define CSAR_COLP_INSTANTIATE(N, P, E)                                                               \
  cudaError_t colp_attrs_##N##_##P##_##E() { return colp_attrs<N, P, E>(); }                         \
  cudaError_t colp_launch_##N##_##P##_##E(ColMode m, const CUtensorMap& map, const ColArgs& a, int nt, \
                                          cudaStream_t s) {                                          \
    return colp_launch<N, P, E>(m, map, a, nt, s);                                                   \
  }                                                                                                  \
  void colp_box_##N##_##P##_##E(int* c, int* r) { colp_box<N, P, E>(c, r); }

}  // namespace csar
