// select.cu — the threshold of Section IV-B: sigma = |b|_(K+1), the (K+1)-th largest
// magnitude of b = X + mu Delta X, and the complex soft / half / hard shrinkage of b.
//
// The column pass COL_SELECT has already (a) recorded Delta X on the support of the
// current K-sparse iterate and (b) histogrammed |Delta X|^2 of every off-support
// element (4096 bins on the float bit pattern) and compacted those above a cut.
// Off-support b = mu Delta X orders like |Delta X|, so:
//
//   sel_check   finds the histogram bin holding the (K+1)-th largest off-support
//               |Delta X|^2; if the cut was above that bin's lower edge (or the
//               candidate buffer overflowed) it asks for one exact re-pass.  The
//               column pass counts only keys at or above a floor under the cut; if
//               the (K+1)-th key lies below it, a full-histogram re-pass and a
//               second check (sel_check2) come first.
//   sel_round/  three rounds of radix select (12 + 12 + 8 key bits) over the union
//   sel_pick    {support} u {candidates} give the exact key of |b|_(K+1)^2.
//   thr_count/  strict |b| > sigma entries are counted per column tile, scanned,
//   thr_scan/   shrunk and scattered into the next bucketed iterate (at most K
//   thr_scatter entries).
//   sel_finish  statistics, next cut guess, counters reset.
//
// No kernel waits on another CTA: every dependency is a kernel boundary.
#include <cfloat>

#include "fft.cuh"
#include "internal.h"

namespace csar {

constexpr int kSelThreads = 1024;   // single-CTA kernels
constexpr int kGridThreads = 512;   // grid-stride kernels

__device__ __forceinline__ uint32_t key_of(float2 b) { return __float_as_uint(cabs2(b)) & 0x7fffffffu; }

// Column tile of flat index idx = row * n_rg + col (shifts: both sizes are powers of two).
__device__ __forceinline__ uint32_t tile_of(const SelArgs& a, uint32_t idx) {
  return (idx & (uint32_t)(a.nr - 1)) >> a.tile_shift;
}

// b of union element e: on-support entries first (X + mu dX), then candidates (mu dX).
__device__ __forceinline__ float2 union_b(const SelArgs& a, uint32_t e, uint32_t nx, float mu,
                                          uint32_t* idx) {
  if (e < nx) {
    *idx = a.xs_idx[e];
    const float2 x = a.xs_val[e];
    const float2 d = a.xs_dx[e];
    return make_float2(fmaf(mu, d.x, x.x), fmaf(mu, d.y, x.y));
  }
  const uint32_t c = e - nx;
  *idx = a.cand_idx[c];
  const float2 d = a.cand_val[c];
  return make_float2(mu * d.x, mu * d.y);
}

__device__ __forceinline__ uint32_t union_size(const Ctl* c, uint32_t cap) {
  const uint32_t nc = c->cand_count < cap ? c->cand_count : cap;
  return c->nx + nc;
}

// Shrinkage of b at threshold sigma (|b| > sigma is guaranteed by the caller).
//   soft (Eq. (9), complex sgn):  b (1 - sigma/|b|)
//   half (q = 1/2, the L_1/2 thresholding of [Xu2010]) with lambda mu chosen so that
//   the jump point equals sigma: b (2/3)(1 + cos(2pi/3 - (2/3) acos(c (3 sigma/|b|)^1.5))),
//   c = sqrt(96)/72.
//   hard (q = 0): b unchanged.
__device__ __forceinline__ float2 shrink(float2 b, float sigma, int kind) {
  if (kind == 2) return b;
  const float m = sqrtf(cabs2(b));
  float f;
  if (kind == 0) {
    f = 1.f - sigma / m;
  } else {
    const float u = 3.f * sigma / m;
    const float arg = fminf(0.13608276348795434f * u * sqrtf(u), 1.f);
    const float phi = acosf(arg);
    f = (2.f / 3.f) * (1.f + cosf(2.0943951023931957f - (2.f / 3.f) * phi));
  }
  return make_float2(b.x * f, b.y * f);
}

// Inclusive scan of one value per thread over the kSelThreads threads of the block
// (prefix: the sum over threads <= tid; suffix: over threads >= tid): a shuffle scan in
// each warp, then one over the 32 warp totals.  ws: 64 shared words; two barriers; every
// thread must call it.  Integer sums, so the result does not depend on the order.
template <bool SUFFIX>
__device__ __forceinline__ unsigned long long block_scan(unsigned long long v, unsigned long long* ws) {
  static_assert(kSelThreads == 1024, "32 warps");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long n = SUFFIX ? __shfl_down_sync(0xffffffffu, v, o) : __shfl_up_sync(0xffffffffu, v, o);
    if (SUFFIX ? lane + o < 32 : lane >= o) v += n;
  }
  if (lane == (SUFFIX ? 0 : 31)) ws[wid] = v;   // the warp's total
  __syncthreads();
  if (wid == 0) {
    unsigned long long t = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long n = SUFFIX ? __shfl_down_sync(0xffffffffu, t, o) : __shfl_up_sync(0xffffffffu, t, o);
      if (SUFFIX ? lane + o < 32 : lane >= o) t += n;
    }
    ws[32 + lane] = t;
  }
  __syncthreads();
  if (SUFFIX) return v + (wid + 1 < 32 ? ws[32 + wid + 1] : 0ull);
  return v + (wid > 0 ? ws[32 + wid - 1] : 0ull);
}

// Whole-block search, h[0..nb) with nb a multiple of 1024 or nb <= 1024:
// largest bin b with S(b) = sum_{i >= b} h[i] >= target; *above = S(b+1).
// Returns -1 if S(0) < target.  Uses sh (>= 1024 u64).  All threads get the result.
__device__ int find_bin(const uint32_t* h, int nb, uint64_t target, uint64_t* above,
                        unsigned long long* sh) {
  __shared__ int res_b;
  __shared__ unsigned long long res_above;
  const int tid = threadIdx.x;
  const int per = nb >= kSelThreads ? nb / kSelThreads : 1;
  const int lo = tid * per;
  unsigned long long cs = 0;
  if (lo < nb)
    for (int i = 0; i < per; ++i) cs += h[lo + i];
  if (tid == 0) { res_b = -1; res_above = 0; }
  const unsigned long long suf = block_scan<true>(cs, sh);   // S(lo)
  const unsigned long long nxt = suf - cs;                   // S(lo+per)
  if (lo < nb && suf >= target && nxt < target) {
    unsigned long long acc = nxt;
    for (int i = per - 1; i >= 0; --i) {
      const unsigned long long s2 = acc + h[lo + i];
      if (s2 >= target) { res_b = lo + i; res_above = acc; break; }
      acc = s2;
    }
  }
  __syncthreads();
  *above = res_above;
  return res_b;
}

// ------------------------------------------------------------------ selection record
// Every union element's index, b and key exactly as the ranking kernels form them
// (union_b, key_of), plus the union size and the control block (sigma2_key, mu, sigma).
__global__ void __launch_bounds__(kGridThreads) k_sel_dump(SelArgs a, SelDump d) {
  const Ctl* c = a.ctl;
  const uint32_t nu = union_size(c, a.cand_cap), nx = c->nx;
  const float mu = c->mu;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *d.count = nu;
    *d.ctl = *c;
  }
  const uint32_t lim = nu < d.cap ? nu : d.cap;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < lim; e += gridDim.x * blockDim.x) {
    uint32_t i;
    const float2 b = union_b(a, e, nx, mu, &i);
    d.idx[e] = i;
    d.b[e] = b;
    d.key[e] = key_of(b);
  }
}

cudaError_t launch_sel_dump(const SelArgs& a, const SelDump& d, cudaStream_t s) {
  k_sel_dump<<<256, kGridThreads, 0, s>>>(a, d);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ check / repass
// Capacity check of a re-pass with cut bin lb: off-support keys at or above it.
__device__ void check_capacity(const SelArgs& a, int lb) {
  unsigned long long cnt = 0;
  for (int i = lb; i < (int)kHistBins; ++i) cnt += a.hist[i];
  if (cnt > a.cand_cap) atomicOr(&a.ctl->err, kErrCapacity);
}

// Fixed step: does the union of the support and the candidates (off-support |Delta X|^2
// >= cut) already hold the K+1 largest |b|?  Every element left out has |b|^2 < mu^2 cut
// (up to a few ulp), so it does when at least K+1 union elements have |b|^2 >= T =
// mu^2 cut (1 + 2^-16): the support counted exactly, the candidates from the histogram
// bins above that of cut (1 + 2^-14) (a lower bound).  Then the selection on the union is
// exact whatever the (K+1)-th off-support key, and the candidate cut can sit just under
// the expected threshold instead of under the (K+1)-th off-support magnitude.
__device__ bool union_suffices(const SelArgs& a, unsigned long long* sh) {
  const Ctl* c = a.ctl;
  const uint32_t cut = c->cut_key;
  if (a.mu_mode != 0 || cut == kNoCandidates || c->cand_count > a.cand_cap) return false;
  const float mu = a.mu_fixed;
  const uint32_t t_key = __float_as_uint(mu * mu * __uint_as_float(cut) * (1.f + 1.f / 65536.f));
  const uint32_t cut_hi = __float_as_uint(__uint_as_float(cut) * (1.f + 1.f / 16384.f));
  const int tid = threadIdx.x;
  unsigned long long cnt = 0;
  const uint32_t nx = c->nx;
  for (uint32_t e = tid; e < nx; e += kSelThreads) {
    uint32_t idx;
    if (key_of(union_b(a, e, nx, mu, &idx)) >= t_key) ++cnt;
  }
  for (int i = (int)(cut_hi >> kHistShift) + 1 + tid; i < (int)kHistBins; i += kSelThreads) cnt += a.hist[i];
  __syncthreads();
  block_scan<false>(cnt, sh);
  const bool ok = sh[63] >= (unsigned long long)a.K + 1;   // the block's total
  __syncthreads();
  return ok;
}

__device__ __forceinline__ void sel_check_body(const SelArgs& a) {
  __shared__ unsigned long long sh[kSelThreads];
  __shared__ uint32_t state;
  Ctl* c = a.ctl;
  const uint64_t target = (uint64_t)a.K + 1;
  const bool suffices = union_suffices(a, sh);
  uint64_t above = 0;
  const int b = find_bin(a.hist, kHistBins, target, &above, sh);
  if (threadIdx.x == 0) {
    // the selection pass counted only keys >= hist_floor(cut): if fewer than K+1 lie
    // there, the (K+1)-th off-support key is below the floor and its bin is unknown
    const bool truncated = hist_floor(c->cut_key) > 0u;
    if (suffices) {
      c->need_repass = kRepassNone;
    } else if (b < 0 && truncated) {
      c->need_repass = kRepassHist;
      c->cut_key = kNoCandidates;
      c->cand_count = 0u;
    } else {
      uint32_t low = b > 0 ? ((uint32_t)b << kHistShift) : 0u;
      if (low < kMinKey) low = kMinKey;
      const bool ok = c->cut_key <= low && c->cand_count <= a.cand_cap;
      c->need_repass = ok ? kRepassNone : kRepassCut;
      if (!ok) {
        c->cut_key = low;
        c->cand_count = 0u;
      }
    }
    // NIHT with an empty support (first iteration): select on Delta X (mu = 1),
    // then the step is computed on that top-K support and applied afterwards
    c->niht_first = (a.mu_mode == 1 && c->nx == 0u) ? 1u : 0u;
    if (a.mu_mode == 0 || c->nx == 0u) c->mu = a.mu_mode == 0 ? a.mu_fixed : 1.f;
    state = c->need_repass;
    if (a.h_repass && (state == kRepassCut || state == kRepassHist)) cudaGraphSetConditional(a.h_repass, 1u);
    if (a.h_repass2 && state == kRepassHist) cudaGraphSetConditional(a.h_repass2, 1u);
    // the one-CTA selection when no re-pass changes the union and it fits
    const bool fused = a.fused_ok && a.mu_mode == 0 && state == kRepassNone &&
                       union_size(c, a.cand_cap) <= (uint32_t)kFusedMaxUnion && a.n_tiles <= kFusedMaxTiles;
    c->sel_fused = fused ? 1u : 0u;
    if (fused && a.h_fused) cudaGraphSetConditional(a.h_fused, 1u);
    if (!fused && a.h_multi) cudaGraphSetConditional(a.h_multi, 1u);
  }
  __syncthreads();
  if (state == kRepassHist) {
    // the full-histogram re-pass counts into a cleared histogram
    for (int i = threadIdx.x; i < (int)kHistBins; i += blockDim.x) a.hist_mut[i] = 0u;
  } else if (state == kRepassCut && threadIdx.x == 0) {
    check_capacity(a, b > 0 ? b : (int)(kMinKey >> kHistShift));
  }
}
__global__ void __launch_bounds__(kSelThreads) k_sel_check(SelArgs a) { sel_check_body(a); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kSelThreads) k_sel_check_b(const SelArgs* __restrict__ as) {
  sel_check_body(as[blockIdx.y]);
}

// After a full-histogram re-pass: the exact cut, and the second (candidate) re-pass.
__device__ __forceinline__ void sel_check2_body(const SelArgs& a) {
  __shared__ unsigned long long sh[kSelThreads];
  Ctl* c = a.ctl;
  if (c->need_repass != kRepassHist) return;   // uniform
  uint64_t above = 0;
  const int b = find_bin(a.hist, kHistBins, (uint64_t)a.K + 1, &above, sh);
  if (threadIdx.x == 0) {
    uint32_t low = b > 0 ? ((uint32_t)b << kHistShift) : 0u;
    if (low < kMinKey) low = kMinKey;
    c->cut_key = low;
    c->cand_count = 0u;
    c->need_repass = kRepassCut2;
    check_capacity(a, b > 0 ? b : (int)(kMinKey >> kHistShift));
  }
}
__global__ void __launch_bounds__(kSelThreads) k_sel_check2(SelArgs a) { sel_check2_body(a); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kSelThreads) k_sel_check2_b(const SelArgs* __restrict__ as) {
  sel_check2_body(as[blockIdx.y]);
}

// ------------------------------------------------------------------ radix select
__device__ __forceinline__ void sel_round_body(const SelArgs& a, int level) {
  __shared__ uint32_t h[kHistBins];
  const Ctl* c = a.ctl;
  if (c->sel_fused || c->sel_prefix == 0xffffffffu) return;   // fused path, or decided
  for (int i = threadIdx.x; i < (int)kHistBins; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const uint32_t nx = c->nx;
  const uint32_t nu = union_size(c, a.cand_cap);
  const float mu = c->mu;
  const uint32_t prefix = c->sel_prefix;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nu; e += gridDim.x * blockDim.x) {
    uint32_t idx;
    const uint32_t key = key_of(union_b(a, e, nx, mu, &idx));
    if (key < kMinKey) continue;
    if (level == 0) {
      atomicAdd(&h[key >> 20], 1u);
    } else if (level == 1) {
      if ((key >> 20) == prefix) atomicAdd(&h[(key >> 8) & 4095u], 1u);
    } else {
      if ((key >> 8) == prefix) atomicAdd(&h[key & 255u], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (int)kHistBins; i += blockDim.x)
    if (h[i]) atomicAdd(&a.hist2[i], h[i]);
}
__global__ void __launch_bounds__(kGridThreads) k_sel_round(SelArgs a, int level) { sel_round_body(a, level); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kGridThreads) k_sel_round_b(const SelArgs* __restrict__ as, int level) {
  sel_round_body(as[blockIdx.y], level);
}

__device__ __forceinline__ void sel_pick_body(const SelArgs& a, int level) {
  __shared__ unsigned long long sh[kSelThreads];
  Ctl* c = a.ctl;
  if (c->sel_fused) return;                   // uniform: the one-CTA kernel selects
  const bool done = c->sel_prefix == 0xffffffffu && level > 0;
  if (!done) {
    const uint64_t target = level == 0 ? (uint64_t)a.K + 1 : (uint64_t)c->sel_rank;
    const int nb = level == 2 ? 256 : (int)kHistBins;
    uint64_t above = 0;
    const int b = find_bin(a.hist2, nb, target, &above, sh);
    if (threadIdx.x == 0) {
      if (b < 0) {
        // fewer than K+1 nonzero magnitudes: keep every nonzero element
        c->sel_prefix = 0xffffffffu;
        c->sigma2_key = 0u;
        c->sigma = 0.f;
      } else {
        c->sel_rank = (uint32_t)(target - above);
        if (level == 0) {
          c->sel_prefix = (uint32_t)b;
        } else if (level == 1) {
          c->sel_prefix = (c->sel_prefix << 12) | (uint32_t)b;
        } else {
          const uint32_t key = (c->sel_prefix << 8) | (uint32_t)b;
          c->sigma2_key = key;
          c->sigma = sqrtf(__uint_as_float(key));
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (int)kHistBins; i += blockDim.x) a.hist2[i] = 0u;
}
__global__ void __launch_bounds__(kSelThreads) k_sel_pick(SelArgs a, int level) { sel_pick_body(a, level); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kSelThreads) k_sel_pick_b(const SelArgs* __restrict__ as, int level) {
  sel_pick_body(as[blockIdx.y], level);
}

// ------------------------------------------------------------------ threshold
__device__ __forceinline__ bool kept(uint32_t key, uint32_t s2) { return key > s2 && key >= kMinKey; }

__device__ __forceinline__ void thr_count_body(const SelArgs& a) {
  Ctl* c = a.ctl;
  if (c->sel_fused) return;
  const uint32_t nx = c->nx, nu = union_size(c, a.cand_cap), s2 = c->sigma2_key;
  const float mu = c->mu;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nu; e += gridDim.x * blockDim.x) {
    uint32_t idx;
    const uint32_t key = key_of(union_b(a, e, nx, mu, &idx));
    if (kept(key, s2)) atomicAdd(&a.tile_cnt[tile_of(a, idx)], 1u);
    else if (key == s2 && s2 >= kMinKey) atomicMin(&c->jstar, idx);   // the (K+1)-th element
  }
}
__global__ void __launch_bounds__(kGridThreads) k_thr_count(SelArgs a) { thr_count_body(a); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kGridThreads) k_thr_count_b(const SelArgs* __restrict__ as) {
  thr_count_body(as[blockIdx.y]);
}

// Exclusive scan of the per-tile counts into the next iterate's offsets.
__device__ __forceinline__ void thr_scan_body(const SelArgs& a) {
  __shared__ unsigned long long sh[kSelThreads];
  if (a.ctl->sel_fused) return;
  const int tid = threadIdx.x;
  const int per = (a.n_tiles + kSelThreads - 1) / kSelThreads;
  const int lo = tid * per;
  unsigned long long s = 0;
  for (int i = 0; i < per; ++i)
    if (lo + i < a.n_tiles) s += a.tile_cnt[lo + i];
  const unsigned long long incl = block_scan<false>(s, sh);
  unsigned long long run = incl - s;
  for (int i = 0; i < per; ++i) {
    const int k = lo + i;
    if (k < a.n_tiles) {
      a.xo_off[k] = (uint32_t)run;
      a.tile_cur[k] = (uint32_t)run;
      run += a.tile_cnt[k];
      a.tile_cnt[k] = 0u;
    }
  }
  if (tid == kSelThreads - 1) {
    a.xo_off[a.n_tiles] = (uint32_t)incl;
    a.ctl->nnz = (uint32_t)incl;
  }
}
__global__ void __launch_bounds__(kSelThreads) k_thr_scan(SelArgs a) { thr_scan_body(a); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kSelThreads) k_thr_scan_b(const SelArgs* __restrict__ as) {
  thr_scan_body(as[blockIdx.y]);
}

// raw != 0: store b itself (the NIHT support list of the first iteration).
__device__ __forceinline__ void thr_scatter_body(const SelArgs& a, int raw) {
  Ctl* c = a.ctl;
  if (c->sel_fused) return;
  raw = raw && c->niht_first;
  const uint32_t nx = c->nx, nu = union_size(c, a.cand_cap), s2 = c->sigma2_key;
  const float mu = c->mu, sigma = c->sigma;
  const uint32_t jstar = c->jstar;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nu; e += gridDim.x * blockDim.x) {
    uint32_t idx;
    const float2 b = union_b(a, e, nx, mu, &idx);
    if (idx == jstar) c->b_jstar = b;
    if (!kept(key_of(b), s2)) continue;
    const uint32_t tile = tile_of(a, idx);
    const uint32_t pos = atomicAdd(&a.tile_cur[tile], 1u);
    if (!CSAR_CHECK(pos, a.n, c) || !CSAR_CHECK(idx, a.n, c)) continue;
    a.xo_idx[pos] = idx;
    a.xo_val[pos] = raw ? b : shrink(b, sigma, a.thresh);
  }
}
__global__ void __launch_bounds__(kGridThreads) k_thr_scatter(SelArgs a, int raw) { thr_scatter_body(a, raw); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kGridThreads) k_thr_scatter_b(const SelArgs* __restrict__ as, int raw) {
  thr_scatter_body(as[blockIdx.y], raw);
}

// ------------------------------------------------------------------ one-CTA selection
// The radix select, the per-tile count, its scan and the scatter of k_sel_round /
// k_sel_pick / k_thr_count / k_thr_scan / k_thr_scatter in one CTA, with the union's
// keys held in shared memory: one launch instead of nine when the union (support and
// candidates) has at most kFusedMaxUnion elements, the step is fixed and no re-pass ran.
constexpr size_t kFusedSmem = (size_t)(kFusedMaxUnion + kHistBins + kFusedMaxTiles) * sizeof(uint32_t);

__device__ __forceinline__ void sel_fused_body(const SelArgs& a) {
  extern __shared__ uint32_t fsm[];
  uint32_t* key = fsm;                        // union keys
  uint32_t* h = key + kFusedMaxUnion;         // radix histogram
  uint32_t* tcnt = h + kHistBins;             // per-tile counts, then cursors
  __shared__ unsigned long long sh[kSelThreads];
  __shared__ uint32_t s_jstar;
  Ctl* c = a.ctl;
  if (!c->sel_fused) return;                  // uniform
  const int tid = threadIdx.x;
  const uint32_t nx = c->nx, nu = union_size(c, a.cand_cap);
  const float mu = c->mu;
  // one CTA has few threads for the latency of these loads: each thread keeps kU
  // elements' loads in flight at a time
  constexpr int kU = 8;
  // keys into shared memory, with the first radix round's histogram (12 high key bits)
  for (int i = tid; i < (int)kHistBins; i += kSelThreads) h[i] = 0u;
  __syncthreads();
  for (uint32_t e0 = tid; e0 < nu; e0 += kU * kSelThreads) {
    float2 bv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t e = e0 + u * kSelThreads;
      uint32_t idx;
      bv[u] = e < nu ? union_b(a, e, nx, mu, &idx) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t e = e0 + u * kSelThreads;
      if (e < nu) {
        const uint32_t k = key_of(bv[u]);
        key[e] = k;
        if (k >= kMinKey) atomicAdd(&h[k >> 20], 1u);
      }
    }
  }
  // three radix rounds (12 + 12 + 8 key bits) on the keys in shared memory
  uint64_t target = (uint64_t)a.K + 1;
  uint32_t prefix = 0u, s2 = 0u;
  bool all = false;
  for (int level = 0; level < 3; ++level) {
    const int nb = level == 2 ? 256 : (int)kHistBins;
    if (level > 0) {
      for (int i = tid; i < nb; i += kSelThreads) h[i] = 0u;
      __syncthreads();
      for (uint32_t e = tid; e < nu; e += kSelThreads) {
        const uint32_t k = key[e];
        if (k < kMinKey) continue;
        if (level == 1) { if ((k >> 20) == prefix) atomicAdd(&h[(k >> 8) & 4095u], 1u); }
        else if ((k >> 8) == prefix) atomicAdd(&h[k & 255u], 1u);
      }
    }
    __syncthreads();
    uint64_t above = 0;
    const int b = find_bin(h, nb, target, &above, sh);
    if (b < 0) {                              // fewer than K+1 nonzero magnitudes: keep all
      all = true;
      break;
    }
    target -= above;
    prefix = level == 0 ? (uint32_t)b : (level == 1 ? ((prefix << 12) | (uint32_t)b) : prefix);
    if (level == 2) s2 = (prefix << 8) | (uint32_t)b;
  }
  if (all) s2 = 0u;
  const float sigma = all ? 0.f : sqrtf(__uint_as_float(s2));
  // strict |b| > sigma per column tile, and the (K+1)-th element (smallest index at s2)
  const int nt = a.n_tiles;
  for (int i = tid; i < nt; i += kSelThreads) tcnt[i] = 0u;
  if (tid == 0) s_jstar = 0xffffffffu;
  __syncthreads();
  for (uint32_t e0 = tid; e0 < nu; e0 += kU * kSelThreads) {
    uint32_t ix[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t e = e0 + u * kSelThreads;
      const uint32_t k = e < nu ? key[e] : 0u;
      const bool need = e < nu && (kept(k, s2) || (k == s2 && s2 >= kMinKey));
      ix[u] = need ? (e < nx ? a.xs_idx[e] : a.cand_idx[e - nx]) : 0xffffffffu;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (ix[u] == 0xffffffffu) continue;
      const uint32_t e = e0 + u * kSelThreads;
      if (kept(key[e], s2)) atomicAdd(&tcnt[tile_of(a, ix[u])], 1u);
      else atomicMin(&s_jstar, ix[u]);
    }
  }
  __syncthreads();
  // exclusive scan of the tile counts (per-thread runs of nt/1024) into offsets
  const int per = (nt + kSelThreads - 1) / kSelThreads;
  const int lo = tid * per;
  unsigned long long run = 0;
  for (int i = 0; i < per; ++i)
    if (lo + i < nt) run += tcnt[lo + i];
  const unsigned long long incl = block_scan<false>(run, sh);
  const uint32_t total = (uint32_t)sh[63];   // the last warp's inclusive prefix
  run = incl - run;
  for (int i = 0; i < per; ++i) {
    const int k = lo + i;
    if (k < nt) {
      const uint32_t cnt = tcnt[k];
      a.xo_off[k] = (uint32_t)run;
      tcnt[k] = (uint32_t)run;                // cursor
      run += cnt;
    }
  }
  if (tid == 0) a.xo_off[nt] = total;
  __syncthreads();
  const uint32_t jstar = s_jstar;
  for (uint32_t e0 = tid; e0 < nu; e0 += kU * kSelThreads) {
    uint32_t ix[kU];
    float2 bv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t e = e0 + u * kSelThreads;
      const uint32_t k = e < nu ? key[e] : 0u;
      const bool need = e < nu && (kept(k, s2) || (k == s2 && s2 >= kMinKey));
      ix[u] = 0xffffffffu;
      bv[u] = make_float2(0.f, 0.f);
      if (need) bv[u] = union_b(a, e, nx, mu, &ix[u]);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (ix[u] == 0xffffffffu) continue;
      const uint32_t e = e0 + u * kSelThreads;
      if (ix[u] == jstar) c->b_jstar = bv[u];
      if (!kept(key[e], s2)) continue;
      const uint32_t pos = atomicAdd(&tcnt[tile_of(a, ix[u])], 1u);
      if (!CSAR_CHECK(pos, a.n, c) || !CSAR_CHECK(ix[u], a.n, c)) continue;
      a.xo_idx[pos] = ix[u];
      a.xo_val[pos] = shrink(bv[u], sigma, a.thresh);
    }
  }
  if (tid == 0) {
    c->sigma2_key = s2;
    c->sigma = sigma;
    c->jstar = jstar;
    c->nnz = total;
  }
}
__global__ void __launch_bounds__(kSelThreads) k_sel_fused(SelArgs a) { sel_fused_body(a); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kSelThreads) k_sel_fused_b(const SelArgs* __restrict__ as) {
  sel_fused_body(as[blockIdx.y]);
}

// NIHT: mu = ||Delta X_Gamma||^2 / ||S . G(Delta X_Gamma)||^2 (den from the column
// pass partials).  first != 0: Gamma is the new list (values = Delta X, first
// iteration); the list values are then replaced by their shrinkage at mu*sigma.
__global__ void __launch_bounds__(kSelThreads) k_niht_mu(SelArgs a, int first) {
  __shared__ double sd[kSelThreads];
  __shared__ double sn[kSelThreads];
  __shared__ float mu_s;
  Ctl* c = a.ctl;
  if (c->niht_first != (uint32_t)first) return;
  const int tid = threadIdx.x;
  double den = 0.0, num = 0.0;
  for (int i = tid; i < a.n_partial; i += kSelThreads) den += (double)a.partial_norm[i];
  const uint32_t n_g = first ? c->nnz : c->nx;
  const float2* vals = first ? a.xo_val : a.xs_dx;
  for (uint32_t e = tid; e < n_g; e += kSelThreads) num += (double)cabs2(vals[e]);
  sd[tid] = den;
  sn[tid] = num;
  __syncthreads();
  for (int off = kSelThreads / 2; off > 0; off >>= 1) {
    if (tid < off) { sd[tid] += sd[tid + off]; sn[tid] += sn[tid + off]; }
    __syncthreads();
  }
  if (tid == 0) {
    const double d = sd[0], nm = sn[0];
    const float mu = (nm > 0.0 && d > 0.0) ? (float)(nm / d) : 1.f;
    c->niht_num = nm;
    c->niht_den = d;
    c->mu = mu;
    if (first) c->sigma = c->sigma * mu;
    mu_s = mu;
  }
  __syncthreads();
  if (first) {
    const float mu = mu_s, sigma = c->sigma;
    for (uint32_t e = tid; e < n_g; e += kSelThreads) {
      const float2 d = a.xo_val[e];
      a.xo_val[e] = shrink(make_float2(mu * d.x, mu * d.y), sigma, a.thresh);
    }
  }
}

// Statistics, next cut guess and counter resets (after the scatter).
__device__ __forceinline__ void sel_finish_body(const SelArgs& a) {
  __shared__ double sd[kSelThreads];
  Ctl* c = a.ctl;
  const int tid = threadIdx.x;
  double r = 0.0;
  for (int i = tid; i < a.n_partial_resid; i += kSelThreads) r += (double)a.partial[i];
  sd[tid] = r;
  __syncthreads();
  for (int off = kSelThreads / 2; off > 0; off >>= 1) {
    if (tid < off) sd[tid] += sd[tid + off];
    __syncthreads();
  }
  for (int i = tid; i < (int)kHistBins; i += kSelThreads) a.hist_mut[i] = 0u;
  if (tid == 0) {
    IterStat st;
    st.resid_sq = sd[0];
    st.mu = c->mu;
    st.sigma = c->sigma;
    st.nnz = c->nnz;
    st.pad = 0;
    if (a.stats) a.stats[c->iter] = st;
    c->iter += 1u;
    // next cut on |Delta X|^2 (checked, and re-done exactly if wrong, by the next
    // sel_check): with a fixed step, (rho sigma / mu)^2 with rho = 0.95 times the last
    // ratio sigma_i / sigma_(i-1) when that falls below 1 (the threshold of the next
    // iteration is expected near sigma r), 0.7 before a ratio is known; with the NIHT
    // step (mu changes between iterations) half of (sigma/mu)^2
    const float mu = c->mu > 0.f ? c->mu : 1.f;
    const float s = c->sigma / mu;
    float rho2 = 0.5f;
    if (a.mu_mode == 0 && c->sigma_prev > 0.f) {
      const float r = fminf(1.f, c->sigma / c->sigma_prev);
      rho2 = (0.95f * r) * (0.95f * r);
    }
    c->sigma_prev = c->sigma;
    float g = rho2 * s * s;
    uint32_t cut = __float_as_uint(g);
    if (!(g > 0.f) || !isfinite(g)) cut = kNoCandidates;
    if (cut < kMinKey) cut = kMinKey;
    c->cut_key = cut;
    c->cand_count = 0u;
    c->nx = c->nnz;
    c->sel_prefix = 0u;
    c->jstar = 0xffffffffu;
  }
}
__global__ void __launch_bounds__(kSelThreads) k_sel_finish(SelArgs a) { sel_finish_body(a); }
// batched: patch blockIdx.y
__global__ void __launch_bounds__(kSelThreads) k_sel_finish_b(const SelArgs* __restrict__ as) {
  sel_finish_body(as[blockIdx.y]);
}

// ------------------------------------------------------------------ masked echo
// out = S . Y (row-major bit mask)
__global__ void k_mask_apply(const float2* __restrict__ y, const uint32_t* __restrict__ bits,
                             float2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool on = (__ldg(&bits[i >> 5]) >> (i & 31)) & 1u;
    out[i] = on ? y[i] : make_float2(0.f, 0.f);
  }
}

// ------------------------------------------------------------------ list <-> dense
__global__ void k_list_to_dense(const uint32_t* off, const uint32_t* idx, const float2* val,
                                int n_tiles, float2* dense) {
  const uint32_t n = off[n_tiles];
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    dense[idx[e]] = val[e];
}

__global__ void k_dense_count(const float2* dense, int na, int nr, int col_tile, uint32_t* cnt) {
  const size_t n = (size_t)na * nr;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = dense[i];
    if (v.x != 0.f || v.y != 0.f) atomicAdd(&cnt[(i % nr) / col_tile], 1u);
  }
}

__global__ void k_dense_scatter(const float2* dense, int na, int nr, int col_tile, uint32_t* cur,
                                uint32_t* idx, float2* val) {
  const size_t n = (size_t)na * nr;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = dense[i];
    if (v.x != 0.f || v.y != 0.f) {
      const uint32_t p = atomicAdd(&cur[(i % nr) / col_tile], 1u);
      idx[p] = (uint32_t)i;
      val[p] = v;
    }
  }
}

__global__ void __launch_bounds__(kSelThreads) k_dense_scan(uint32_t* cnt, uint32_t* cur, uint32_t* off,
                                                            int n_tiles, Ctl* ctl) {
  __shared__ unsigned long long sh[kSelThreads];
  const int tid = threadIdx.x;
  const int per = (n_tiles + kSelThreads - 1) / kSelThreads;
  const int lo = tid * per;
  unsigned long long s = 0;
  for (int i = 0; i < per; ++i)
    if (lo + i < n_tiles) s += cnt[lo + i];
  sh[tid] = s;
  __syncthreads();
  for (int o = 1; o < kSelThreads; o <<= 1) {
    const unsigned long long add = tid >= o ? sh[tid - o] : 0ull;
    __syncthreads();
    sh[tid] += add;
    __syncthreads();
  }
  unsigned long long run = tid ? sh[tid - 1] : 0ull;
  for (int i = 0; i < per; ++i) {
    const int k = lo + i;
    if (k < n_tiles) {
      off[k] = (uint32_t)run;
      cur[k] = (uint32_t)run;
      run += cnt[k];
      cnt[k] = 0u;
    }
  }
  if (tid == kSelThreads - 1) {
    off[n_tiles] = (uint32_t)sh[kSelThreads - 1];
    if (ctl) ctl->nx = (uint32_t)sh[kSelThreads - 1];
  }
}

// ------------------------------------------------------------------ launchers
static int g_grid_ctas = 0;
static int grid_ctas() {
  if (!g_grid_ctas) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_grid_ctas = 2 * (sms > 0 ? sms : 1);
  }
  return g_grid_ctas;
}

cudaError_t launch_sel_check(const SelArgs& a, cudaStream_t s) {
  k_sel_check<<<1, kSelThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_sel_check2(const SelArgs& a, cudaStream_t s) {
  k_sel_check2<<<1, kSelThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_sel_round(const SelArgs& a, int level, cudaStream_t s) {
  k_sel_round<<<grid_ctas(), kGridThreads, 0, s>>>(a, level);
  return cudaGetLastError();
}
cudaError_t launch_sel_pick(const SelArgs& a, int level, cudaStream_t s) {
  k_sel_pick<<<1, kSelThreads, 0, s>>>(a, level);
  return cudaGetLastError();
}
cudaError_t launch_thr_count(const SelArgs& a, cudaStream_t s) {
  k_thr_count<<<grid_ctas(), kGridThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_thr_scan(const SelArgs& a, cudaStream_t s) {
  k_thr_scan<<<1, kSelThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_thr_scatter_mode(const SelArgs& a, int raw, cudaStream_t s) {
  k_thr_scatter<<<grid_ctas(), kGridThreads, 0, s>>>(a, raw);
  return cudaGetLastError();
}
cudaError_t launch_thr_scatter(const SelArgs& a, cudaStream_t s) { return launch_thr_scatter_mode(a, 0, s); }
cudaError_t launch_niht_mu_mode(const SelArgs& a, int first, cudaStream_t s) {
  k_niht_mu<<<1, kSelThreads, 0, s>>>(a, first);
  return cudaGetLastError();
}
cudaError_t launch_niht_mu(const SelArgs& a, cudaStream_t s) { return launch_niht_mu_mode(a, 0, s); }
cudaError_t sel_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_sel_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sel_fused_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem);
  return e;
}

// One launch of selection kernel k for every patch of a batch: as[p] are patch p's
// arguments (device memory); single-CTA kernels get one CTA per patch, grid-stride
// kernels a share of the grid per patch (blockIdx.y = patch).  arg: level or raw.
cudaError_t launch_sel_batched(SelKernel k, const SelArgs* as, int np, int arg, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  const dim3 one(1, np);
  const int gx0 = (grid_ctas() + np - 1) / np;
  const dim3 grid(gx0 < 2 ? 2 : gx0, np);
  switch (k) {
    case SelKernel::kCheck: k_sel_check_b<<<one, kSelThreads, 0, s>>>(as); break;
    case SelKernel::kCheck2: k_sel_check2_b<<<one, kSelThreads, 0, s>>>(as); break;
    case SelKernel::kRound: k_sel_round_b<<<grid, kGridThreads, 0, s>>>(as, arg); break;
    case SelKernel::kPick: k_sel_pick_b<<<one, kSelThreads, 0, s>>>(as, arg); break;
    case SelKernel::kCount: k_thr_count_b<<<grid, kGridThreads, 0, s>>>(as); break;
    case SelKernel::kScan: k_thr_scan_b<<<one, kSelThreads, 0, s>>>(as); break;
    case SelKernel::kScatter: k_thr_scatter_b<<<grid, kGridThreads, 0, s>>>(as, arg); break;
    case SelKernel::kFused: k_sel_fused_b<<<one, kSelThreads, kFusedSmem, s>>>(as); break;
    case SelKernel::kFinish: k_sel_finish_b<<<one, kSelThreads, 0, s>>>(as); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
cudaError_t launch_sel_fused(const SelArgs& a, cudaStream_t s) {
  k_sel_fused<<<1, kSelThreads, kFusedSmem, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_sel_finish(const SelArgs& a, cudaStream_t s) {
  k_sel_finish<<<1, kSelThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mask_apply(const float2* y, const uint32_t* mask_bits, float2* out, long long n,
                              cudaStream_t s) {
  k_mask_apply<<<grid_ctas() * 4, kGridThreads, 0, s>>>(y, mask_bits, out, n);
  return cudaGetLastError();
}

cudaError_t launch_list_to_dense(const uint32_t* off, const uint32_t* idx, const float2* val,
                                 int n_tiles, float2* dense, cudaStream_t s) {
  k_list_to_dense<<<grid_ctas(), kGridThreads, 0, s>>>(off, idx, val, n_tiles, dense);
  return cudaGetLastError();
}
cudaError_t launch_dense_count(const float2* dense, int na, int nr, int col_tile, uint32_t* cnt,
                               cudaStream_t s) {
  k_dense_count<<<grid_ctas() * 2, kGridThreads, 0, s>>>(dense, na, nr, col_tile, cnt);
  return cudaGetLastError();
}
cudaError_t launch_dense_scan(uint32_t* cnt, uint32_t* cur, uint32_t* off, int n_tiles, Ctl* ctl,
                              cudaStream_t s) {
  k_dense_scan<<<1, kSelThreads, 0, s>>>(cnt, cur, off, n_tiles, ctl);
  return cudaGetLastError();
}
cudaError_t launch_dense_scatter(const float2* dense, int na, int nr, int col_tile, uint32_t* cur,
                                 uint32_t* idx, float2* val, cudaStream_t s) {
  k_dense_scatter<<<grid_ctas() * 2, kGridThreads, 0, s>>>(dense, na, nr, col_tile, cur, idx, val);
  return cudaGetLastError();
}

}  // namespace csar
