// internal.h — types shared by the host driver and the kernels of libcsar.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/csar.h"
#include "fft.cuh"
#include "phase.cuh"

namespace csar {

// ---------------------------------------------------------------- selection constants
// Keys are the IEEE bit patterns of |b|^2 (non-negative floats order like uint32).
constexpr uint32_t kHistBins = 4096;     // column-pass histogram: key >> 19 (bits 30..19)
constexpr int kHistShift = 19;
constexpr uint32_t kMinKey = 1u << 23;   // keys below this are 0 or subnormal |b|^2
constexpr uint32_t kNoCandidates = 0xffffffffu;
// The selection column pass histograms only keys at or above a floor 16 bins (two
// octaves of |Delta X|^2) under the bin of the candidate cut; with no cut yet (the
// first iteration) the floor is 0 and the histogram is complete.
constexpr uint32_t kFloorBins = 16;
constexpr int kHistWindow = 512;         // bins counted from the floor (64 octaves)
__host__ __device__ constexpr uint32_t hist_floor(uint32_t cut) {
  return cut == kNoCandidates ? 0u
         : ((cut >> kHistShift) > kFloorBins ? (((cut >> kHistShift) - kFloorBins) << kHistShift) : 0u);
}
// Re-pass states (Ctl::need_repass), set by the check kernels.
enum : uint32_t {
  kRepassNone = 0,   // the candidates of the selection pass are complete
  kRepassCut = 1,    // re-pass with the exact cut (first re-pass)
  kRepassHist = 2,   // the (K+1)-th key lies under the floor: full-histogram re-pass first
  kRepassCut2 = 3,   // then the exact cut from that histogram (second re-pass)
};

// Device-latched error bits (reported by csar_plan_check).
enum : uint32_t { kErrNonfinite = 1u, kErrCapacity = 2u, kErrTimeout = 4u, kErrIndex = 8u };

// Checked build (compiled with -DCSAR_CHECKED): the global indexes of the pass kernels'
// dense arrays and output lists are compared with the arrays' extents; an index out of
// range latches kErrIndex (reported as CSAR_E_INTERNAL) and the access is skipped (a
// skipped load reads zero).  In the normal build the test is constant true.
struct Ctl;
#ifdef CSAR_CHECKED
__device__ __forceinline__ bool csar_in_range(size_t i, size_t n, Ctl* ctl);
#define CSAR_CHECK(i, n, ctl) ::csar::csar_in_range((size_t)(i), (size_t)(n), (ctl))
#else
#define CSAR_CHECK(i, n, ctl) true
#endif

// Column-pass modes.
enum ColMode : int {
  COL_FWD = 0,        // out = F_a in
  COL_INV = 1,        // out = F_a^-1 in
  COL_SPARSE_FWD = 2, // out = F_a (list scattered into a zero tile)
  COL_RESID = 3,      // g = F_a^-1 in; out = F_a(S.g) (the range pass forms F_a r)
  COL_SELECT = 4,     // dx = F_a^-1 in; Delta X at the support; histogram; candidates
  COL_REPASS = 5,     // re-pass of COL_SELECT: gate_val 1 runs in states kRepassCut
                      // (candidates) and kRepassHist (full histogram), gate_val 3 in
                      // state kRepassCut2 (candidates)
  COL_NORM = 6,       // g = F_a^-1 in; partial sum of S.|g|^2 (no store)
};

// Control block of one plan's iteration pipeline (device memory).
struct Ctl {
  uint32_t cut_key;      // candidate threshold on |Delta X|^2 bits
  uint32_t cand_count;   // candidates appended (may exceed the capacity)
  uint32_t need_repass;  // set by the check kernel
  uint32_t err;          // latched error bits
  uint32_t sel_prefix;   // radix select: key bits fixed so far
  uint32_t sel_rank;     // radix select: rank (0-based, descending) within the prefix
  uint32_t sigma2_key;   // key of the (K+1)-th largest |b|^2 (0: keep every nonzero)
  uint32_t union_n;      // elements in the selection union
  uint32_t nx;           // current sparse-iterate length
  uint32_t nnz;          // new sparse-iterate length
  uint32_t iter;         // iteration index (stats slot)
  uint32_t niht_first;   // NIHT with an empty support: Gamma = top K of |Delta X|
  float mu;              // step of the current iteration
  float sigma;           // threshold of the current iteration
  uint32_t jstar;        // flat index of the (K+1)-th largest |b| (0xffffffff: none)
  float sigma_prev;      // threshold of the previous iteration (0: none yet)
  float2 b_jstar;        // b at jstar
  double niht_num;       // ||Delta X_Gamma||^2
  double niht_den;       // ||S . G(Delta X_Gamma)||^2
  uint32_t sel_fused;    // 1: this iteration's selection runs in the one-CTA kernel
  uint32_t pad2;
};

#ifdef CSAR_CHECKED
__device__ __forceinline__ bool csar_in_range(size_t i, size_t n, Ctl* ctl) {
  if (i < n) return true;
  if (ctl) atomicOr(&ctl->err, kErrIndex);
  return false;
}
#endif

// One-CTA selection (k_sel_fused): used when the union of support and candidates fits
// in its shared memory and the step is fixed.
constexpr int kFusedMaxUnion = 40960;
constexpr int kFusedMaxTiles = 4096;

// Per-iteration checkpoint of the ITA unroll (autofocus backward).
struct CkptMeta {
  uint32_t count;        // entries of X^(i+1)
  float sigma;           // sigma_i
  uint32_t jstar;        // index of the (K+1)-th largest |b| (0xffffffff: none)
  uint32_t pad;
  float2 b_jstar;
};

// Per-iteration statistics (device).
struct IterStat {
  double resid_sq;
  float mu;
  float sigma;
  uint32_t nnz;
  uint32_t pad;
};

struct ColArgs {
  const float2* in;
  float2* out;
  const float2* y;          // COL_RESID: F_a(S.Y), the azimuth-transformed masked echo
  const uint32_t* mask;     // COL_RESID / COL_NORM: sampling mask in column-pass order
                            // (launch_mask_transpose)
  const uint32_t* xs_off;   // sparse iterate bucketed by column tile: offsets [tiles+1]
  const uint32_t* xs_idx;   // flat indices row*nr+col
  const float2* xs_val;     // values (COL_SPARSE_FWD reads these)
  float2* xs_dx;            // COL_SELECT: Delta X at the support entries
  uint32_t* hist;           // COL_SELECT: global histogram [kHistBins]
  uint32_t* cand_idx;       // candidates (off-support, |Delta X|^2 >= cut)
  float2* cand_val;
  uint32_t cand_cap;
  Ctl* ctl;
  float* partial;           // COL_RESID / COL_NORM: one float per CTA
  const float2* tw;         // twiddle table (global)
  const uint32_t* gate;     // if non-null, the pass runs only when *gate == gate_val
  uint32_t gate_val;
  int nr;                   // row length N_r
  float scale;              // 1/N_a for inverse transforms
  // k_sparse_dft: conditional handle (captured graphs) set to 1 when a column group is
  // left to the FFT path, whose launch is then the body of an IF node (0: not captured)
  cudaGraphConditionalHandle h_dense;
  // COL_SPARSE_FWD: transform every tile, also those the direct DFT would take (batches)
  int no_direct;
};

// One unit of work of a batched pass: row block or column-tile group `unit` of patch
// `patch`, whose transform length along the pass is n.
struct BatchItem {
  int patch;
  int unit;
  int n;
  int pad;
};
// Row lengths and azimuth lengths the batched passes serve (other patch sizes take the
// per-patch graph branches).
#define CSAR_BATCH_ROW_SIZES(X) X(512) X(1024) X(2048) X(4096)
#define CSAR_BATCH_COL_SIZES(X) X(512) X(1024) X(2048) X(4096)

struct RowArgs {
  float2* data;             // output (and input unless src is set), [n_rows][N_r]
  const float2* src;        // if non-null, the rows are read from here instead of data
  const RowCoef* coef;      // one per row
  const float2* tw;
  const uint32_t* gate;     // if non-null, the pass runs only when *gate == gate_val
  uint32_t gate_val;
  int n_rows;
  float scale;              // 1/N_r of the range IFFT
  // residue form (range pass of M in the ITA): if yf is non-null the pass transforms
  // yf - data (F_a(S.Y) - F_a(S.G X) = F_a r), writes one partial sum of |F_a r|^2 *
  // resid_scale per CTA into partial[blockIdx.x] (||r||^2 by Parseval with 1/N_a) and
  // latches kErrNonfinite in ctl->err for non-finite values
  const float2* yf;
  float* partial;
  Ctl* ctl;
  float resid_scale;
  int regs;                 // values per thread of the range transforms: 32 (default) or 16
};

// Range-Doppler operator pair (rda_pass.cu): per azimuth-frequency row, the migration
// dr(tau) = alpha (c0 + j') in range samples (alpha = 1/D - 1, c0 = 2 R_ref fs / c,
// j' = tau - N_r/2) as fp32 (hi, lo) pairs, and the azimuth matched filter's phase.
struct RcmcCoef {
  float al_hi, al_lo;    // alpha
  float a0_hi, a0_lo;    // alpha * c0
  PhaseCoef az;          // P_eta = exp(j 2 pi (A + B j'))
};

// Range pass of the range-Doppler pair, in place on [n_rows][N_r] range-Doppler rows:
// M: P_eta . C(F_r^-1 P_tau F_r data);  G: F_r^-1 P_tau^* F_r D(conj(P_eta) . data).
// gate and the residue form (M only) act as in RowArgs.
struct RdaArgs {
  float2* data;
  const RcmcCoef* rc;    // migration and azimuth filter, one per row
  const RowCoef* rg;     // range filter P_tau (or its conjugate) as the middle phase
  const float2* rtab;    // if non-null: the range filter as a table over the N_r range-
                         // frequency bins in FFT order (non-chirp pulse), instead of rg
  const float2* tw;
  const uint32_t* gate;
  uint32_t gate_val;
  int n_rows;
  float scale;           // 1/N_r of the range IFFT
  const float2* yf;
  float* partial;
  Ctl* ctl;
  float resid_scale;
};

// Column passes: a cluster of P CTAs owns col_w(N, P, E) adjacent columns; each CTA
// holds E = N*W/P complex64 values (E = 8192: 64 KiB and two CTAs per SM; E = 4096:
// 32 KiB and four CTAs per SM; E = 16384: 128 KiB and one CTA of 1024 threads per SM).  A column configuration (P, E) is a plan choice among
// col_conf_ok(N, conf) (see col_dispatch.cu).
constexpr int kColCtaElems = 8192;   // default complex64 values per column-pass CTA
struct ColConf {
  int p = 1;                 // CTAs per cluster
  int e = kColCtaElems;      // complex64 values per CTA
  bool persist = false;      // persistent clusters fed by tensor copies (colp_pass.cuh) for
                             // the forward, inverse, residue and selection passes
};
__host__ __device__ constexpr int col_w(int n, int p, int e = kColCtaElems) {
  return e * p / n > 16 ? 16 : (e * p / n < 1 ? 1 : e * p / n);
}
__host__ __device__ constexpr int col_ctas_per_sm(int e) { return 2 * kColCtaElems / e; }
// Words of the column-order sampling mask (one per thread and column of a pass).
__host__ __device__ constexpr long long col_mask_words(int na, int nr, int p) {
  return (long long)nr * (na / col_regs(na / p));
}
__host__ __device__ constexpr int row_w(int n) { return n >= 8192 ? 1 : 8192 / n; }
__host__ __device__ constexpr int row_threads(int n) { return n * row_w(n) / regs_for(n); }
__host__ __device__ constexpr int row_ctas(int na, int nr) { return (na + row_w(nr) - 1) / row_w(nr); }

// Direct DFT of the K-sparse iterate (k_sparse_dft): groups of kDirectCols columns
// holding at most kDirectMaxEntries entries skip the FFT.
constexpr int kDirectCols = 16;
constexpr int kDirectMaxEntries = 128;
constexpr int kDirectRows = 256;   // smallest N_a the direct DFT handles

// ---------------------------------------------------------------- host helpers (csar_plan.cu)
csar_status validate_params(const csar_params* p);
csar_status build_coefs_into(const csar_params& p, RowCoef* g, RowCoef* m);
void build_twiddles(float2* tw);
csar_status set_error(csar_status st, const char* msg);

// ---------------------------------------------------------------- launchers
bool col_conf_ok(int na, ColConf c);
ColConf col_conf_default(int na);
ColConf col_conf_default_res(int na);   // residue / NIHT-norm passes (same W as the default)
ColConf col_conf_persist(int na);       // persistent passes: clusters of N_a/1024 CTAs of 4096 values
cudaError_t launch_col(int na, ColConf conf, ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s);
cudaError_t launch_row(int nr, const RowArgs& a, cudaStream_t s);
cudaError_t launch_sparse_dft(int na, const ColArgs& a, int col_tile, cudaStream_t s);
cudaError_t row_batched_set_attributes();
// Batched column passes (col_batched.cu): CTAs per tile for azimuth length na (0: na is
// not served), tiles per work item, attributes, one launch over all work items.
int batch_col_cluster(int na);
bool batch_member_ok(int na, int nr);
int batch_col_tiles_per_item(int na);
cudaError_t col_batched_set_attributes();
cudaError_t launch_col_batched(ColMode mode, const ColArgs* args, const BatchItem* items, int n_items,
                               cudaStream_t s);
cudaError_t launch_row_batched(bool resid, const RowArgs* args, const BatchItem* items, int n_items,
                               cudaStream_t s);
bool sparse_dft_applies(int na, int nr);
cudaError_t sparse_dft_set_attributes(int na);
// Tensor map (cuTensorMapEncodeTiled) of an [na][nr] complex64 array with boxes of
// box_cols x box_rows (col_dispatch.cu); the map is named by its struct tag so that this
// header needs no driver API header.
cudaError_t encode_map(struct CUtensorMap_st* map, const void* base, int na, int nr, int box_cols,
                       int box_rows, bool swizzle128);
cudaError_t launch_mask_apply(const float2* y, const uint32_t* mask_bits, float2* out, long long n,
                              cudaStream_t s);
cudaError_t col_set_attributes(int na, ColConf conf);
cudaError_t launch_mask_transpose(int na, int p, int nr, const uint32_t* mask, uint32_t* mask_t,
                                  cudaStream_t s);
cudaError_t row_set_attributes(int nr);

struct SelArgs {
  Ctl* ctl;
  const uint32_t* hist;       // column-pass histogram (zeroed by sel_finish)
  uint32_t* hist_mut;
  uint32_t* hist2;            // radix-select histogram [4096]
  const uint32_t* xs_idx;     // current iterate
  const float2* xs_val;
  const float2* xs_dx;
  const uint32_t* cand_idx;
  const float2* cand_val;
  uint32_t cand_cap;
  uint32_t* tile_cnt;         // [n_tiles]
  uint32_t* tile_cur;         // [n_tiles]
  uint32_t* xo_off;           // next iterate (bucketed)
  uint32_t* xo_idx;
  float2* xo_val;
  const float* partial;       // residual partials of the range pass of M (one per CTA)
  int n_partial_resid;
  const float* partial_norm;  // NIHT denominator partials (COL_NORM)
  int n_partial;
  IterStat* stats;
  int64_t K;
  int64_t n;
  int nr;
  int col_tile;               // columns per column-pass tile
  int tile_shift;             // log2(col_tile) (n_rg and col_tile are powers of two)
  int n_tiles;
  int thresh;                 // 0 soft, 1 half, 2 hard
  int mu_mode;                // 0 fixed, 1 NIHT
  float mu_fixed;
  // conditional graph nodes of the re-passes (0 when not captured): sel_check sets
  // h_repass in states kRepassCut / kRepassHist and h_repass2 in state kRepassHist
  cudaGraphConditionalHandle h_repass;
  cudaGraphConditionalHandle h_repass2;
  // selection path (0 when not captured): sel_check sets exactly one of them
  cudaGraphConditionalHandle h_fused;
  cudaGraphConditionalHandle h_multi;
  int fused_ok;               // 0: always the grid-wide path (CSAR_SEL_FUSED=0)
};

// Record of the union the selection ranked (tests of the exact lambda rule): each
// element's flat index, b and key, as the selection kernels formed them, the union size
// and the control block right after the threshold.
struct SelDump {
  uint32_t* idx = nullptr;
  float2* b = nullptr;
  uint32_t* key = nullptr;
  uint32_t* count = nullptr;
  Ctl* ctl = nullptr;
  uint32_t cap = 0;
};
cudaError_t launch_sel_dump(const SelArgs& a, const SelDump& d, cudaStream_t s);

cudaError_t launch_sel_check(const SelArgs& a, cudaStream_t s);
cudaError_t launch_sel_check2(const SelArgs& a, cudaStream_t s);
cudaError_t launch_sel_round(const SelArgs& a, int level, cudaStream_t s);
cudaError_t launch_sel_pick(const SelArgs& a, int level, cudaStream_t s);
cudaError_t launch_thr_count(const SelArgs& a, cudaStream_t s);
cudaError_t launch_thr_scan(const SelArgs& a, cudaStream_t s);
cudaError_t launch_thr_scatter(const SelArgs& a, cudaStream_t s);
cudaError_t launch_thr_scatter_mode(const SelArgs& a, int raw, cudaStream_t s);
cudaError_t launch_niht_mu(const SelArgs& a, cudaStream_t s);
cudaError_t launch_niht_mu_mode(const SelArgs& a, int first, cudaStream_t s);
cudaError_t launch_sel_finish(const SelArgs& a, cudaStream_t s);
enum class SelKernel { kCheck, kCheck2, kRound, kPick, kCount, kScan, kScatter, kFused, kFinish };
cudaError_t launch_sel_batched(SelKernel k, const SelArgs* as, int np, int arg, cudaStream_t s);
cudaError_t launch_sel_fused(const SelArgs& a, cudaStream_t s);
cudaError_t launch_row_rda(int nr, const RdaArgs& a, bool is_g, cudaStream_t s);
cudaError_t rda_set_attributes(int nr);
cudaError_t sel_set_attributes();

// autofocus (autofocus.cu)
cudaError_t launch_rotate_rows(const float2* y, const float* theta, float2* yt, int na, int nr,
                               cudaStream_t s);
cudaError_t launch_af_resid(float2* g, const float2* yt, const uint32_t* mask, int na, int nr,
                            double* row_loss, float* grad_theta, double* loss, cudaStream_t s);
cudaError_t launch_scale(const float2* in, float2* out, float alpha, long long n, cudaStream_t s);
cudaError_t launch_af_tvjp(const uint32_t* idx, const float2* val, const CkptMeta* meta,
                           const float2* xbar, float2* bbar, uint32_t cap, cudaStream_t s);
cudaError_t launch_af_mask_theta(float2* g, const float2* yt, const uint32_t* mask, int na, int nr,
                                 float mu, float* theta_bar, cudaStream_t s);
cudaError_t launch_af_axpy(const float2* bbar, const float2* h, float mu, float2* xbar, long long n,
                           cudaStream_t s);
cudaError_t launch_ckpt_copy(const Ctl* ctl, const uint32_t* idx, const float2* val, uint32_t* ck_idx,
                             float2* ck_val, CkptMeta* ck_meta, uint32_t cap, cudaStream_t s);

// list <-> dense
cudaError_t launch_list_to_dense(const uint32_t* off, const uint32_t* idx, const float2* val,
                                 int n_tiles, float2* dense, cudaStream_t s);
cudaError_t launch_dense_count(const float2* dense, int na, int nr, int col_tile,
                               uint32_t* tile_cnt, cudaStream_t s);
cudaError_t launch_dense_scan(uint32_t* tile_cnt, uint32_t* tile_cur, uint32_t* off, int n_tiles,
                              Ctl* ctl, cudaStream_t s);
cudaError_t launch_dense_scatter(const float2* dense, int na, int nr, int col_tile,
                                 uint32_t* tile_cur, uint32_t* idx, float2* val, cudaStream_t s);

}  // namespace csar
