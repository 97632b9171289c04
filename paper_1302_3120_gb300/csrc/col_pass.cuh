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
__device__ __forceinline__ void xch_signal(uint32_t mb) {
  __syncthreads();
  if (threadIdx.x < P) mbar_arrive_cluster(cluster_map(mb, (int)threadIdx.x));
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
                                         uint32_t mb, Ctl* ctl) {
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
    xch_signal<C::P>(mb);
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

template <int N, int P, int E, int MODE>
__global__ void __launch_bounds__(ColCfg<N, P, E>::NT, col_ctas_per_sm(E)) k_col(ColArgs a) {
  static_assert(ColCfg<N, P, E>::NT <= 1024, "block too large");
  using C = ColCfg<N, P, E>;
  constexpr int W = C::W, R = C::R, QR = C::QR, NT = C::NT, Q = C::Q;
  using L = Layout<Q, W, true>;
  extern __shared__ float2 smem[];
  float2* sm = smem;
  float2* tw = smem + L::kSmemElems;
  float* red = reinterpret_cast<float*>(tw + kTwLo + kTwHi);   // 32 floats
  uint64_t* mbar = reinterpret_cast<uint64_t*>(red + 32);      // kMbCount mbarriers
  uint32_t* hist = reinterpret_cast<uint32_t*>(mbar + kMbCount);  // kHistBins (SELECT, REPASS)
  uint32_t* msk = hist + kHistBins;                                // NT words (SELECT, REPASS)

  uint32_t rstate = kRepassNone;
  if constexpr (MODE == COL_REPASS) {
    // uniform for the whole grid: the first re-pass launch (gate_val kRepassCut) runs in
    // states kRepassCut and kRepassHist, the second (kRepassCut2) in state kRepassCut2
    rstate = a.ctl->need_repass;
    const bool run = a.gate_val == kRepassCut2 ? rstate == kRepassCut2
                                               : (rstate == kRepassCut || rstate == kRepassHist);
    if (!run) return;
  }
  if (a.gate && *a.gate != a.gate_val) return;
  const int c = (P > 1) ? (int)(blockIdx.x % P) : 0;      // rank in the cluster
  const int tile = blockIdx.x / P;
  if constexpr (MODE == COL_SPARSE_FWD) {
    // groups of kDirectCols columns with few entries are transformed by k_sparse_dft;
    // the test is uniform per cluster (one tile), so whole clusters leave together
    const int bpg = kDirectCols / W > 0 ? kDirectCols / W : 1;
    const int grp = (tile * W) / kDirectCols;
    const uint32_t ge = a.xs_off[(grp + 1) * bpg < a.nr / W ? (grp + 1) * bpg : a.nr / W] -
                        a.xs_off[grp * bpg];
    if (N >= kDirectRows && ge <= (uint32_t)kDirectMaxEntries) return;
  }
  load_twiddles(tw, a.tw);
  const int tid = threadIdx.x;
  const int w = tid % W, t = tid / W;
  const int col = tile * W + w;
  const size_t nr = (size_t)a.nr;
  float2 v[R];
  // sampling bits of this thread's R rows (pre-transposed: bit s <-> strided row s),
  // fetched first so the load is long complete when the mask is applied
  uint32_t mbits = 0u;
  if constexpr (MODE == COL_RESID || MODE == COL_NORM) {
    const size_t mi = ((size_t)col * P + c) * QR + t;
    if (CSAR_CHECK(mi, (size_t)a.nr * (N / R), a.ctl)) mbits = __ldg(&a.mask[mi]);
  }
  // exchange mbarriers, then every CTA of the cluster is running (and its mbarriers are
  // initialised) before any remote store or arrive
  const uint32_t mb0 = smem_addr(mbar);
  uint32_t peer[P];
  if constexpr (P > 1) {
    if (tid == 0) {
#pragma unroll
      for (int j = 0; j < 3; ++j) mbar_init(mb0 + 8u * j, (uint32_t)P);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
#pragma unroll
    for (int k = 0; k < P; ++k) peer[k] = cluster_map(smem_addr(sm), k);
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
  } else {
    peer[0] = smem_addr(sm);
  }

  // ------------------------------------------------------------------ input
  if constexpr (MODE == COL_SPARSE_FWD) {
    // zero tile; entries whose row belongs to this CTA's blocked input set
    for (int i = tid; i < L::kSmemElems; i += NT) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const uint32_t e0 = a.xs_off[tile], e1 = a.xs_off[tile + 1];
    for (uint32_t e = e0 + tid; e < e1; e += NT) {
      const uint32_t idx = a.xs_idx[e];
      const int row = (int)(idx / (uint32_t)a.nr);
      const int ww = (int)(idx % (uint32_t)a.nr) - tile * W;
      const int n1 = row / Q, n2 = row % Q;
      if (P == 1 || n2 / (Q / P) == c) {
        // slot s = i*P + n1 of thread tt, with n2 = c*Q/P + tt + QR*i
        const int loc = (P == 1) ? row : (n2 - c * (Q / P));
        const int tt = loc % QR, i = loc / QR;
        const int s = (P == 1) ? i : i * P + n1;
        if (CSAR_CHECK(ww, W, a.ctl)) sm[L::template at<4>(ww, tt + QR * s)] = a.xs_val[e];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = sm[L::template at<4>(w, t + QR * s)];
    // the buffer is reused by the cross step: peers push into it only after every CTA of
    // the cluster has read its staged input
    if constexpr (P > 1) {
      xch_signal<P>(mb0 + 8u * kMbFree);
      mbar_wait(mb0 + 8u * kMbFree, 0u, a.ctl);
    } else {
      __syncthreads();
    }
  } else {
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const size_t gi = (size_t)bs_in_row<N, P, E>(c, t, s) * nr + col;
      v[s] = CSAR_CHECK(gi, (size_t)N * nr, a.ctl) ? __ldcs(&a.in[gi]) : make_float2(0.f, 0.f);
    }
  }
  // selection passes: the support range of this tile, its first entry per thread and the
  // candidate cut are fetched while the column loads are in flight
  uint32_t sel_e0 = 0u, sel_e1 = 0u, sel_idx = 0u, sel_cut = 0u;
  if constexpr (MODE == COL_SELECT || MODE == COL_REPASS) {
    sel_e0 = a.xs_off[tile];
    sel_e1 = a.xs_off[tile + 1];
    sel_cut = a.ctl->cut_key;
    if (sel_e0 + tid < sel_e1) sel_idx = a.xs_idx[sel_e0 + tid];
  }

  // ------------------------------------------------------------------ transforms
  if constexpr (MODE == COL_FWD || MODE == COL_SPARSE_FWD) {
    bs_cross<N, P, E, false>(v, sm, tw, c, t, w, peer, mb0 + 8u * kMbBs, a.ctl);
    fft<Q, false, L, true, R>(v, sm, tw, t, w);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const size_t gi = (size_t)strided_row<N, P, E>(c, t, s) * nr + col;
      if (CSAR_CHECK(gi, (size_t)N * nr, a.ctl)) __stcs(&a.out[gi], v[s]);
    }
  } else if constexpr (MODE == COL_INV) {
    bs_cross<N, P, E, true>(v, sm, tw, c, t, w, peer, mb0 + 8u * kMbBs, a.ctl);
    fft<Q, true, L, true, R>(v, sm, tw, t, w);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const size_t gi = (size_t)strided_row<N, P, E>(c, t, s) * nr + col;
      if (CSAR_CHECK(gi, (size_t)N * nr, a.ctl)) __stcs(&a.out[gi], cscale(v[s], a.scale));
    }
  } else if constexpr (MODE == COL_RESID) {
    // F_a(S.g): the residue F_a r = F_a(S.Y) - F_a(S.g) is formed by the next range pass
    // as it loads its rows (contiguous reads there, where the pass hides their latency)
    bs_cross<N, P, E, true>(v, sm, tw, c, t, w, peer, mb0 + 8u * kMbBs, a.ctl);
    // the local inverse transform runs as the forward one of the conjugate (unnormalised
    // IFFT(u) = conj(FFT(conj(u))), exact), so one copy of the FFT code serves both
    // transforms in a rolled loop
#pragma unroll
    for (int s = 0; s < R; ++s) v[s].y = -v[s].y;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      fft<Q, false, L, true, R>(v, sm, tw, t, w);
      if (pass == 1) break;
#pragma unroll
      for (int s = 0; s < R; ++s)
        v[s] = ((mbits >> s) & 1u) ? make_float2(v[s].x * a.scale, -v[s].y * a.scale) : make_float2(0.f, 0.f);
    }
    if constexpr (P == 1) {
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const size_t gi = (size_t)(t + s * QR) * nr + col;
        if (CSAR_CHECK(gi, (size_t)N * nr, a.ctl)) __stcs(&a.out[gi], v[s]);
      }
    } else {
      // SB step: twiddle W_N^(c k2) (k2 = t + s QR) and push k2 to CTA s / RP at element
      // c*Q/P + k2l (source-major, so pushes and the final reads are conflict-free), once
      // every CTA has finished reading its own buffer.  Twiddles: table anchors at every
      // fourth s, steps W^(c QR u) in between.
      xch_signal<P>(mb0 + 8u * kMbFree);
      mbar_wait(mb0 + 8u * kMbFree, 0u, a.ctl);
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
          const int dst = s / C::RP, k2l = t + QR * (s % C::RP);
          st_cluster(peer[dst] + 8u * (uint32_t)L::template at<4>(w, c * (Q / P) + k2l), x);
        }
      }
      xch_signal<P>(mb0 + 8u * kMbSb);
      mbar_wait(mb0 + 8u * kMbSb, 0u, a.ctl);
      float2* oc = a.out + (size_t)(c * (Q / P) + t) * nr + col;
      const size_t di = (size_t)QR * nr, dk = (size_t)Q * nr;
#pragma unroll
      for (int i = 0; i < C::RP; ++i) {
        const int k2l = t + QR * i;
        float2 b[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) b[n1] = sm[L::template at<4>(w, n1 * (Q / P) + k2l)];
        Dft<P, false>::run(b);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
          const size_t gi = (size_t)(c * (Q / P) + t) * nr + col + i * di + k1 * dk;
          if (CSAR_CHECK(gi, (size_t)N * nr, a.ctl)) __stcs(oc + i * di + k1 * dk, b[k1]);
        }
      }
    }
  } else if constexpr (MODE == COL_NORM) {
    bs_cross<N, P, E, true>(v, sm, tw, c, t, w, peer, mb0 + 8u * kMbBs, a.ctl);
    fft<Q, true, L, true, R>(v, sm, tw, t, w);
    float acc = 0.f;
#pragma unroll
    for (int s = 0; s < R; ++s) acc += ((mbits >> s) & 1u) ? cabs2(cscale(v[s], a.scale)) : 0.f;
    const float tot = block_sum<NT>(acc, red);
    if (tid == 0) a.partial[blockIdx.x] = tot;
  } else {  // COL_SELECT / COL_REPASS
    // COL_SELECT: histogram of off-support keys >= hist_floor(cut), candidates >= cut,
    // Delta X at the support.  COL_REPASS: full histogram and no candidates in state
    // kRepassHist, candidates only otherwise.
    const bool hist_on = (MODE == COL_SELECT) || rstate == kRepassHist;
    const uint32_t floor_key = (MODE == COL_SELECT) ? hist_floor(sel_cut) : 0u;
    const uint32_t cut = (MODE == COL_REPASS && rstate == kRepassHist) ? kNoCandidates : sel_cut;
    // histogram bins: all kHistBins without a floor, else a window of kHistWindow bins
    // from the floor's bin whose last bin also takes every larger key (so the global
    // bin found for the (K+1)-th key is still a valid lower bound)
    const int hb0 = (int)(floor_key >> kHistShift);
    const int nbins = floor_key == 0u ? (int)kHistBins
                                      : ((int)kHistBins - hb0 < kHistWindow ? (int)kHistBins - hb0 : kHistWindow);
    if (hist_on) {
      for (int i = tid; i < nbins; i += NT) hist[i] = 0u;
    }
    msk[tid] = 0u;
    bs_cross<N, P, E, true>(v, sm, tw, c, t, w, peer, mb0 + 8u * kMbBs, a.ctl);
    fft<Q, true, L, true, R>(v, sm, tw, t, w);
    __syncthreads();
    // support of the current iterate: local element m (global row c + P*m) of column w
    // is v[m / QR] of thread (m % QR)*W + w, which gets bit m / QR in its support word
    const uint32_t first_idx = sel_idx;
    for (uint32_t e = sel_e0 + tid; e < sel_e1; e += NT) {
      const uint32_t idx = sel_idx;
      if (e + NT < sel_e1) sel_idx = a.xs_idx[e + NT];
      const int row = (int)(idx / (uint32_t)a.nr);
      if (P > 1 && row % P != c) continue;
      const int ww = (int)(idx % (uint32_t)a.nr) - tile * W;
      const int m = row / P;
      if (!CSAR_CHECK(ww, W, a.ctl)) continue;
      atomicOr(&msk[(m % QR) * W + ww], 1u << (m / QR));
    }
    __syncthreads();
    const uint32_t sup = msk[tid];
    if constexpr (MODE == COL_SELECT) {
      // Delta X at the support goes through shared memory to the entry's thread
      if (sup) {
#pragma unroll
        for (int s = 0; s < R; ++s)
          if ((sup >> s) & 1u) sm[L::template at<4>(w, t + s * QR)] = cscale(v[s], a.scale);
      }
    }
    constexpr uint32_t full = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
    const int lane = tid & 31;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const int m = t + s * QR;
      const float2 d = cscale(v[s], a.scale);
      const bool on_support = (sup >> s) & 1u;
      const uint32_t key = __float_as_uint(cabs2(d)) & 0x7fffffffu;
      if (hist_on && !on_support && key >= floor_key) {
        const int hb = (int)(key >> kHistShift) - hb0;
        atomicAdd(&hist[hb < nbins ? hb : nbins - 1], 1u);
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
            a.cand_idx[pos] = (uint32_t)((size_t)(c + P * m) * nr + col);
            a.cand_val[pos] = d;
          }
        }
      }
    }
    if (MODE == COL_SELECT || hist_on) __syncthreads();
    if constexpr (MODE == COL_SELECT) {
      for (uint32_t e = sel_e0 + tid; e < sel_e1; e += NT) {
        const uint32_t idx = e == sel_e0 + tid ? first_idx : a.xs_idx[e];
        const int row = (int)(idx / (uint32_t)a.nr);
        if (P > 1 && row % P != c) continue;
        const int ww = (int)(idx % (uint32_t)a.nr) - tile * W;
        if (CSAR_CHECK(ww, W, a.ctl) && CSAR_CHECK(e, (size_t)N * nr, a.ctl))
          a.xs_dx[e] = sm[L::template at<4>(ww, row / P)];
      }
    }
    if (hist_on) {
      for (int i = tid; i < nbins; i += NT) {
        const uint32_t h = hist[i];
        if (h) atomicAdd(&a.hist[hb0 + i], h);
      }
    }
  }
  // no CTA may exit while a peer could still address its shared memory: every remote
  // store or arrive into this CTA precedes a completed wait of this CTA on an exchange
  // mbarrier, so none is outstanding here
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
