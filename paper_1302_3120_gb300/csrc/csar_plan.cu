// csar_plan.cu — host side of libcsar: the C ABI declared in include/csar.h.
//
// Plan creation evaluates the chirp-scaling phase functions' coefficients in FP64
// (one quadratic polynomial per azimuth-frequency row and phase, Section III-D with
// the textbook CSA functions), the FFT twiddles, and allocates the workspace.  The
// ITA iteration (Algorithm 1) is a fixed sequence of kernels (column pass, row
// pass, column pass, row pass, column pass, selection, threshold) captured once per
// ping-pong parity into a CUDA graph; data-dependent choices (the exact re-pass of
// the selection, the NIHT branch) are taken on the device by kernels that return
// early, so one graph serves every iteration.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/csar.h"
#include "fft.cuh"
#include "internal.h"

using namespace csar;

namespace {

thread_local std::string g_last_error;

csar_status fail(csar_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

csar_status cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? CSAR_E_OOM : CSAR_E_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

void split(double v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (double)*hi);
}

PhaseCoef make_coef(double a, double b, double c, double sign) {
  PhaseCoef p;
  a *= sign;
  b *= sign;
  c *= sign;
  a -= std::nearbyint(a);
  split(a, &p.a_hi, &p.a_lo);
  split(b, &p.b_hi, &p.b_lo);
  split(c, &p.c_hi, &p.c_lo);
  return p;
}

csar_status validate(const csar_params* p) {
  if (!p) return fail(CSAR_E_INVALID, "params is NULL");
  if (!pow2_in(p->n_az, 16, 8192) || !pow2_in(p->n_rg, 16, 8192))
    return fail(CSAR_E_INVALID, "n_az=%d n_rg=%d: each must be a power of two in [16, 8192]",
                p->n_az, p->n_rg);
  const double vals[] = {p->wavelength, p->velocity, p->r0, p->prf, p->bandwidth, p->pulse_len, p->fs};
  const char* names[] = {"wavelength", "velocity", "r0", "prf", "bandwidth", "pulse_len", "fs"};
  for (int i = 0; i < 7; ++i)
    if (!(vals[i] > 0.0) || !std::isfinite(vals[i]))
      return fail(CSAR_E_INVALID, "%s must be finite and > 0", names[i]);
  if (p->c < 0.0 || !std::isfinite(p->c)) return fail(CSAR_E_INVALID, "c must be >= 0");
  return CSAR_OK;
}

struct Buffers {
  float2* z = nullptr;             // n: pass-to-pass array
  uint32_t* off[2] = {nullptr, nullptr};
  uint32_t* idx[2] = {nullptr, nullptr};
  float2* val[2] = {nullptr, nullptr};
  float2* dx = nullptr;            // Delta X on the support
  uint32_t* cand_idx = nullptr;
  float2* cand_val = nullptr;
  uint32_t cand_cap = 0;
  uint32_t* hist = nullptr;
  uint32_t* hist2 = nullptr;
  uint32_t* tile_cnt = nullptr;
  uint32_t* tile_cur = nullptr;
  float* partial = nullptr;
  float* partial_norm = nullptr;
  uint32_t* mask_t = nullptr;      // sampling mask in column-pass order
  float2* yf = nullptr;            // F_a(S . Y): azimuth-transformed masked echo
  Ctl* ctl = nullptr;
  IterStat* stats = nullptr;
  int stats_cap = 0;
  // autofocus
  float2* yt = nullptr;            // exp(-j theta) . Y
  float2* af_xbar = nullptr;
  float2* af_bbar = nullptr;
  float2* af_h = nullptr;
  double* row_loss = nullptr;
  uint32_t* ck_idx = nullptr;      // checkpoints: [iters][ck_cap]
  float2* ck_val = nullptr;
  CkptMeta* ck_meta = nullptr;
  uint32_t ck_cap = 0;
  int ck_iters_cap = 0;
  int ck_iters = 0;                // iterations checkpointed by the last autofocus solve
  bool ck_active = false;          // the iteration graphs copy checkpoints
  float ck_mu = 1.f;
  // host-buffer entry point
  float2* hY = nullptr;
  uint32_t* hMask = nullptr;
  float2* hX = nullptr;
};

struct GraphKey {
  const void* y = nullptr;
  const void* mask = nullptr;
  int64_t K = -1;
  int mu_mode = -1, thresh = -1;
  float mu = 0.f;
  uint32_t cand_cap = 0;
  IterStat* stats = nullptr;
  const void* ck = nullptr;
  const void* dump = nullptr;
  bool operator==(const GraphKey& o) const {
    return y == o.y && mask == o.mask && K == o.K && mu_mode == o.mu_mode && thresh == o.thresh &&
           mu == o.mu && cand_cap == o.cand_cap && stats == o.stats && ck == o.ck && dump == o.dump;
  }
};

}  // namespace

namespace csar {
// Per-row coefficients (cycles) of the three chirp-scaling phases; see phase.cuh.
//   H1 = exp{j pi K_m (1/D - 1)(tau - 2 R_ref/(c D))^2},      tau - 2R_ref/c = j'/fs
//   H2 = exp{j pi (D/K_m) f_tau^2} exp{j 4 pi f_tau R_ref (1/D - 1)/c},  f_tau = m fs/N_r
//   H3 = exp{j 4 pi R0 f0 D/c} exp{-j 4 pi (K_m/c^2)(1 - D)((R0 - R_ref)/D)^2},
//        R0 = R_ref + j' c/(2 fs)
csar_status build_coefs_into(const csar_params& p, RowCoef* g, RowCoef* m) {
  const double c = p.c > 0.0 ? p.c : 299792458.0;
  const double f0 = c / p.wavelength;
  const double kr = p.bandwidth / p.pulse_len;
  const double rref = p.r0;
  const double fs = p.fs;
  const int na = p.n_az, nr = p.n_rg;
  const double jmax = nr / 2.0;  // |j'|, |m| <= N_r/2
  const double lim = 4194304.0;  // 2^22
  for (int k = 0; k < na; ++k) {
    const int ks = k < na / 2 ? k : k - na;
    const double fe = ks * p.prf / na;
    const double x = c * fe / (2.0 * p.velocity * f0);
    if (!(x * x < 1.0))
      return fail(CSAR_E_UNSUPPORTED, "Doppler frequency %.6g Hz exceeds 2V/lambda", fe);
    const double d = std::sqrt(1.0 - x * x);
    const double km = kr / (1.0 - kr * c * rref * fe * fe / (2.0 * p.velocity * p.velocity * f0 * f0 * f0 * d * d * d));
    // H1
    const double a1 = 0.5 * km * (1.0 / d - 1.0);
    const double del = (2.0 * rref / c) * (1.0 / d - 1.0);
    const double h1c = a1 / (fs * fs), h1b = -2.0 * a1 * del / fs, h1a = a1 * del * del;
    // H2
    const double df = fs / nr;
    const double h2c = 0.5 * (d / km) * df * df, h2b = 2.0 * df * rref * (1.0 / d - 1.0) / c, h2a = 0.0;
    // H3
    const double h3a = 2.0 * f0 * d * rref / c, h3b = f0 * d / fs;
    const double h3c = -km * (1.0 - d) / (2.0 * d * d * fs * fs);
    const double bs[] = {h1b, h2b, h3b}, cs[] = {h1c, h2c, h3c};
    for (int i = 0; i < 3; ++i)
      if (std::fabs(bs[i]) * jmax >= lim || std::fabs(cs[i]) * jmax * jmax >= lim || !std::isfinite(bs[i]) ||
          !std::isfinite(cs[i]))
        return fail(CSAR_E_UNSUPPORTED,
                    "phase polynomial too large for on-the-fly evaluation (row %d, phase H%d)", k, i + 1);
    m[k].pro = make_coef(h1a, h1b, h1c, 1.0);
    m[k].mid = make_coef(h2a, h2b, h2c, 1.0);
    m[k].epi = make_coef(h3a, h3b, h3c, 1.0);
    g[k].pro = make_coef(h3a, h3b, h3c, -1.0);
    g[k].mid = make_coef(h2a, h2b, h2c, -1.0);
    g[k].epi = make_coef(h1a, h1b, h1c, -1.0);
  }
  return CSAR_OK;
}


// Coefficients of the range-Doppler operator pair (Section III-C, Eqs. (14)-(18)):
//   range filter P_tau = exp(j pi f_tau^2 / K_r): phase m^2 df^2 / (2 K_r) cycles per
//     signed range-frequency bin m (the middle phase of a range pass; no outer phases);
//   migration dr = (1/D - 1)(2 R_ref fs / c + j') range samples, j' = tau - N_r/2;
//   azimuth filter P_eta = exp(j 4 pi R0 f0 D / c) = exp(j 2 pi (2 R_ref f0 D / c + j' f0 D / fs)).
// rc holds 2 N_a rows: those of M, then those of G (azimuth filter conjugated).  The
// range pass of G scatters without atomics, which needs the migration slope alpha below
// 1/2 sample per sample (D >= 2/3; far beyond the beams the range-Doppler method serves).
csar_status build_rda_coefs(const csar_params& p, RowCoef* rg_g, RowCoef* rg_m, RcmcCoef* rc) {
  const double c = p.c > 0.0 ? p.c : 299792458.0;
  const double f0 = c / p.wavelength;
  const double kr = p.bandwidth / p.pulse_len;
  const double df = p.fs / p.n_rg;
  const double lim = 4194304.0;  // 2^22
  const double cq = 0.5 * df * df / kr;
  if (cq * (p.n_rg / 2.0) * (p.n_rg / 2.0) >= lim)
    return fail(CSAR_E_UNSUPPORTED, "range filter phase too large for on-the-fly evaluation");
  const PhaseCoef zero = make_coef(0.0, 0.0, 0.0, 1.0);
  const double c0 = 2.0 * p.r0 * p.fs / c;
  for (int k = 0; k < p.n_az; ++k) {
    rg_m[k].pro = zero;
    rg_m[k].mid = make_coef(0.0, 0.0, cq, 1.0);
    rg_m[k].epi = zero;
    rg_g[k].pro = zero;
    rg_g[k].mid = make_coef(0.0, 0.0, cq, -1.0);
    rg_g[k].epi = zero;
    const int ks = k < p.n_az / 2 ? k : k - p.n_az;
    const double fe = ks * p.prf / p.n_az;
    const double x = c * fe / (2.0 * p.velocity * f0);
    if (!(x * x < 1.0)) return fail(CSAR_E_UNSUPPORTED, "Doppler frequency %.6g Hz exceeds 2V/lambda", fe);
    const double d = std::sqrt(1.0 - x * x);
    const double alpha = 1.0 / d - 1.0;
    if (!(alpha <= 0.5))
      return fail(CSAR_E_UNSUPPORTED, "range migration slope %.3g > 0.5 (row %d)", alpha, k);
    split(alpha, &rc[k].al_hi, &rc[k].al_lo);
    split(alpha * c0, &rc[k].a0_hi, &rc[k].a0_lo);
    const double az_b = f0 * d / p.fs;
    if (std::fabs(az_b) * (p.n_rg / 2.0) >= lim || std::fabs(alpha * c0) >= lim)
      return fail(CSAR_E_UNSUPPORTED, "azimuth filter / migration too large (row %d)", k);
    rc[k].az = make_coef(2.0 * p.r0 * f0 * d / c, az_b, 0.0, 1.0);
    rc[p.n_az + k] = rc[k];
    rc[p.n_az + k].az = make_coef(2.0 * p.r0 * f0 * d / c, az_b, 0.0, -1.0);
  }
  return CSAR_OK;
}

// Twiddle table W_8192^m, two levels (kTwLo + kTwHi entries), FP64 then rounded once.
void build_twiddles(float2* tw) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < kTwLo; ++m) {
    const double a = two_pi * m / kTwN;
    tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  for (int h = 0; h < kTwHi; ++h) {
    const double a = two_pi * (double)(h * kTwLo) / kTwN;
    tw[kTwLo + h] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
}

csar_status validate_params(const csar_params* p) { return validate(p); }
csar_status set_error(csar_status st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace csar

// Column-pass cluster size chosen by csar_autotune, per (N_a, N_r), for plans created
// afterwards in this process (optionally persisted in the file named by CSAR_TUNE_FILE).
namespace {
std::mutex g_tune_mu;
std::map<std::pair<int, int>, std::pair<ColConf, ColConf>> g_tune;   // (main, residue)
std::map<std::pair<int, int>, int> g_tune_row;   // values per thread of the range passes
bool g_tune_loaded = false;

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = std::getenv("CSAR_TUNE_FILE");
  if (!f) return;
  FILE* fp = std::fopen(f, "r");
  if (!fp) return;
  // one line per (n_az, n_rg): main and residue column configurations, then (optional)
  // the range passes' values per thread
  char line[256];
  while (std::fgets(line, sizeof line, fp)) {
    int na, nr, p, e, pr, er, rr = 0;
    const int got = std::sscanf(line, "%d %d %d %d %d %d %d", &na, &nr, &p, &e, &pr, &er, &rr);
    if (got < 6) continue;
    ColConf c, r;
    c.p = p;
    c.e = e;
    r.p = pr;
    r.e = er;
    if (col_conf_ok(na, c) && col_conf_ok(na, r) && col_w(na, p, e) == col_w(na, pr, er))
      g_tune[{na, nr}] = {c, r};
    if (got == 7 && (rr == 16 || rr == 32)) g_tune_row[{na, nr}] = rr;
  }
  std::fclose(fp);
}

void tune_save_locked() {
  const char* f = std::getenv("CSAR_TUNE_FILE");
  if (!f) return;
  FILE* fp = std::fopen(f, "w");
  if (!fp) return;
  for (const auto& kv : g_tune) {
    const auto rr = g_tune_row.find(kv.first);
    std::fprintf(fp, "%d %d %d %d %d %d %d\n", kv.first.first, kv.first.second, kv.second.first.p,
                 kv.second.first.e, kv.second.second.p, kv.second.second.e,
                 rr == g_tune_row.end() ? 32 : rr->second);
  }
  std::fclose(fp);
}

bool tuned_conf(int na, int nr, ColConf* c, ColConf* r) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find({na, nr});
  if (it == g_tune.end()) return false;
  *c = it->second.first;
  *r = it->second.second;
  return true;
}

// Values per thread of the range passes chosen by the autotuner (0: none, the default).
int tuned_row_regs(int na, int nr) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  auto it = g_tune_row.find({na, nr});
  return it == g_tune_row.end() || it->second == 32 ? 0 : it->second;
}
}  // namespace

struct csar_plan_s {
  csar_params p{};
  int dev = 0;
  int na = 0, nr = 0;
  int64_t n = 0;
  ColConf col;                    // column-pass configuration (cluster size, values per CTA)
  ColConf col_res;                // configuration of the residue and NIHT-norm passes (same W)
  int sel_fused_ok = 1;           // one-CTA selection allowed (CSAR_SEL_FUSED=0 disables it)
  int row_regs = 0;               // values per thread of the range passes (0: default 32; 16)
  bool no_direct = false;         // batch member: the clustered FFT for every tile of C1
  int buf_gen = 0;                // bumped whenever ensure_capacity reallocates
  int col_tile = 0, n_tiles = 0;
  RowCoef* coef_g = nullptr;
  RowCoef* coef_m = nullptr;
  // range-Doppler operator pair (CSAR_PLAN_RDA): range-filter rows and RCMC rows
  bool rda = false;
  RowCoef* rda_rg_g = nullptr;
  RowCoef* rda_rg_m = nullptr;
  float2* rda_pulse_g = nullptr;  // recorded pulse spectrum S (G) and conj(S) (M), if set
  float2* rda_pulse_m = nullptr;
  RcmcCoef* rda_rcmc = nullptr;
  float2* tw = nullptr;
  Buffers b;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cond_stream = nullptr;   // captures the bodies of conditional graph nodes
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  GraphKey key[2];
  bool use_graphs = true;
  SelDump dump;                   // selection record (csar_debug_selection_*), off when idx is null
};

// A batch of independent patches: one plan per patch; each ITA iteration of the whole
// batch is one CUDA graph.  When every patch is a batch member (sizes the batched
// kernels serve) and the step is fixed, the graph holds one launch per pass over a work
// table of all patches' row blocks or tile groups (the patches' arguments in device
// arrays); otherwise its parallel branches are the patches' own kernel sequences.
struct csar_batch_s {
  std::vector<csar_plan> plans;
  bool single = false;                       // one launch per pass
  BatchItem* d_row_items = nullptr;          // row blocks of every patch
  BatchItem* d_col_items = nullptr;          // tile groups of every patch
  int n_row_items = 0, n_col_items = 0;
  RowArgs* d_r1 = nullptr;                   // per patch: range pass of G, of M
  RowArgs* d_r2 = nullptr;
  ColArgs* d_c[2][4] = {};                   // per parity: C1, C2 / C3, re-pass 1, re-pass 2
  SelArgs* d_sel[2] = {};                    // per parity
  std::vector<int> key_gen;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<const void*> key_y;
  std::vector<int64_t> key_k;
  csar_opts key_o{};
  int dev = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Allocation-failure injection (csar_debug_fail_alloc): the n-th device allocation
// after the call reports cudaErrorMemoryAllocation without allocating.
std::atomic<long> g_fail_alloc_at{0};
std::atomic<long> g_alloc_count{0};

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  const long at = g_fail_alloc_at.load();
  if (at > 0 && g_alloc_count.fetch_add(1) + 1 == at) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc((void**)p, count * sizeof(T) > 0 ? count * sizeof(T) : 1);
}

// NVTX ranges around the entry points and, outside graph capture, around each pass of
// an iteration (no cost without an attached tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void free_buffers(Buffers& b) {
  void* ptrs[] = {b.z, b.off[0], b.off[1], b.idx[0], b.idx[1], b.val[0], b.val[1], b.dx, b.cand_idx,
                  b.cand_val, b.hist, b.hist2, b.tile_cnt, b.tile_cur, b.partial, b.partial_norm, b.mask_t, b.yf, b.ctl,
                  b.stats, b.hY, b.hMask, b.hX, b.yt, b.af_xbar, b.af_bbar, b.af_h, b.row_loss,
                  b.ck_idx, b.ck_val, b.ck_meta};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  b = Buffers();
}

void drop_graphs(csar_plan plan) {
  for (int i = 0; i < 2; ++i) {
    if (plan->exec[i]) cudaGraphExecDestroy(plan->exec[i]);
    plan->exec[i] = nullptr;
    plan->key[i] = GraphKey();
  }
}

// Candidate capacity for sparsity K (grown on demand, never during capture).
csar_status ensure_capacity(csar_plan plan, int64_t K, int iters) {
  Buffers& b = plan->b;
  const int64_t want64 = std::min<int64_t>(plan->n, std::max<int64_t>(int64_t(1) << 20, 8 * (K + 1)));
  const uint32_t want = (uint32_t)want64;
  if (b.cand_cap < want) {
    drop_graphs(plan);
    ++plan->buf_gen;
    if (b.cand_idx) cudaFree(b.cand_idx);
    if (b.cand_val) cudaFree(b.cand_val);
    b.cand_idx = nullptr;
    b.cand_val = nullptr;
    b.cand_cap = 0;
    CK(dalloc(&b.cand_idx, want));
    CK(dalloc(&b.cand_val, want));
    b.cand_cap = want;
  }
  if (b.stats_cap < iters) {
    drop_graphs(plan);
    ++plan->buf_gen;
    if (b.stats) cudaFree(b.stats);
    b.stats = nullptr;
    b.stats_cap = 0;
    const int cap = std::max(iters, 256);
    CK(dalloc(&b.stats, cap));
    b.stats_cap = cap;
  }
  return CSAR_OK;
}

ColArgs col_args(csar_plan plan) {
  ColArgs a{};
  a.no_direct = plan->no_direct ? 1 : 0;
  a.tw = plan->tw;
  a.nr = plan->nr;
  a.ctl = plan->b.ctl;
  a.hist = plan->b.hist;
  a.cand_idx = plan->b.cand_idx;
  a.cand_val = plan->b.cand_val;
  a.cand_cap = plan->b.cand_cap;
  a.partial = plan->b.partial;
  a.xs_dx = plan->b.dx;
  a.scale = 1.0f / (float)plan->na;
  return a;
}

RowArgs row_args(csar_plan plan, float2* data, const RowCoef* coef) {
  RowArgs r{};
  r.data = data;
  r.coef = coef;
  r.tw = plan->tw;
  r.n_rows = plan->na;
  r.scale = 1.0f / (float)plan->nr;
  r.regs = plan->row_regs;
  return r;
}

// Range pass of G (is_g) or M over r.data, with r's gate and residue form: the
// chirp-scaling phases, or, on a range-Doppler plan, range compression, RCMC and the
// azimuth filter.
cudaError_t range_pass(csar_plan plan, const RowArgs& r, bool is_g, cudaStream_t s) {
  if (!plan->rda) return launch_row(plan->nr, r, s);
  if (r.src || (is_g && r.yf)) return cudaErrorInvalidValue;
  RdaArgs a{};
  a.data = r.data;
  a.rc = plan->rda_rcmc + (is_g ? plan->na : 0);
  a.rg = is_g ? plan->rda_rg_g : plan->rda_rg_m;
  a.rtab = is_g ? plan->rda_pulse_g : plan->rda_pulse_m;
  a.tw = r.tw;
  a.gate = r.gate;
  a.gate_val = r.gate_val;
  a.n_rows = r.n_rows;
  a.scale = r.scale;
  a.yf = r.yf;
  a.partial = r.partial;
  a.ctl = r.ctl;
  a.resid_scale = r.resid_scale;
  return launch_row_rda(plan->nr, a, is_g, s);
}

SelArgs sel_args(csar_plan plan, int cur, const csar_opts& o) {
  const Buffers& b = plan->b;
  const int nxt = 1 - cur;
  SelArgs s{};
  s.ctl = b.ctl;
  s.hist = b.hist;
  s.hist_mut = b.hist;
  s.hist2 = b.hist2;
  s.xs_idx = b.idx[cur];
  s.xs_val = b.val[cur];
  s.xs_dx = b.dx;
  s.cand_idx = b.cand_idx;
  s.cand_val = b.cand_val;
  s.cand_cap = b.cand_cap;
  s.tile_cnt = b.tile_cnt;
  s.tile_cur = b.tile_cur;
  s.xo_off = b.off[nxt];
  s.xo_idx = b.idx[nxt];
  s.xo_val = b.val[nxt];
  s.partial = b.partial;
  s.n_partial_resid = row_ctas(plan->na, plan->nr);
  s.partial_norm = b.partial_norm;
  s.n_partial = plan->n_tiles * plan->col_res.p;
  s.stats = b.stats;
  s.K = o.K;
  s.n = plan->n;
  s.nr = plan->nr;
  s.col_tile = plan->col_tile;
  s.tile_shift = 0;
  while ((1 << s.tile_shift) < plan->col_tile) ++s.tile_shift;
  s.n_tiles = plan->n_tiles;
  s.thresh = o.thresh;
  s.mu_mode = o.mu_mode;
  s.mu_fixed = o.mu;
  s.fused_ok = plan->sel_fused_ok;
  return s;
}

#define LK(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

// True while `s` is being captured into a graph.
bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive;
}

// A conditional handle of the graph being captured on `s` (reset to 0 at every launch).
cudaError_t capture_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  LK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
  return cudaGraphConditionalHandleCreate(h, g, 0u, cudaGraphCondAssignDefault);
}

// While capturing `s`: append an IF node on handle `h` whose body is what `body`
// enqueues (captured through `aux`), so work that is rarely needed costs no launch when
// a kernel upstream leaves the handle at 0.  Not capturing: `body` runs on `s` directly
// (its kernels then test the same condition on the device and return early).
template <class F>
cudaError_t enqueue_if(cudaStream_t s, cudaStream_t aux, cudaGraphConditionalHandle h, F&& body) {
  if (!h) return body(s);
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  LK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  LK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  LK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  LK(cudaStreamBeginCaptureToGraph(aux, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed));
  const cudaError_t e = body(aux);
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(aux, &out);
  return e != cudaSuccess ? e : e2;
}

// F_a of a sparse iterate into a.out: the direct DFT of the column groups with few
// entries, then the clustered FFT of the others.  When captured, the FFT launch is the
// body of an IF node that the direct DFT sets only if some group needs it (in the
// steady state none does: the launch of ~2000 early-exiting clusters is skipped).
cudaError_t sparse_forward(csar_plan plan, ColArgs a, cudaStream_t s) {
  const int na = plan->na;
  if (plan->no_direct) return launch_col(na, plan->col, COL_SPARSE_FWD, a, plan->n_tiles, s);
  if (capturing(s) && sparse_dft_applies(na, plan->nr)) LK(capture_handle(s, &a.h_dense));
  LK(launch_sparse_dft(na, a, plan->col_tile, s));
  const cudaGraphConditionalHandle h = a.h_dense;
  a.h_dense = 0;
  return enqueue_if(s, plan->cond_stream, h,
                    [&](cudaStream_t q) { return launch_col(na, plan->col, COL_SPARSE_FWD, a, plan->n_tiles, q); });
}

// One ITA iteration reading the sparse iterate in list `cur` and writing list 1-cur.
// Optional per-pass events (profiling): ev[0..kPasses].
constexpr int kPasses = 6;  // C1, R1, C2, R2, C3, selection+threshold
cudaError_t enqueue_iteration(csar_plan plan, const float2* y, int cur, const csar_opts& o,
                              cudaStream_t s, cudaEvent_t* ev) {
  Buffers& b = plan->b;
  const uint32_t* mask = b.mask_t;
  const int na = plan->na, nr = plan->nr, nt = plan->n_tiles;
  const int nxt = 1 - cur;
  // per-pass NVTX ranges (host enqueue; outside capture only)
  static const char* const kPassNames[kPasses] = {"C1 sparse azimuth FFT", "R1 range pass of G", "C2 residue",
                                                  "R2 range pass of M", "C3 selection pass", "selection"};
  struct PassRange {
    bool on, open = false;
    ~PassRange() {
      if (open) nvtxRangePop();
    }
  } nvtx{!capturing(s)};
  auto mark = [&](int i) -> cudaError_t {
    if (nvtx.on) {
      if (nvtx.open) nvtxRangePop();
      nvtx.open = i < kPasses;
      if (nvtx.open) nvtxRangePushA(kPassNames[i]);
    }
    return ev ? cudaEventRecord(ev[i], s) : cudaSuccess;
  };
  ColArgs c = col_args(plan);
  c.xs_off = b.off[cur];
  c.xs_idx = b.idx[cur];
  c.xs_val = b.val[cur];
  LK(mark(0));
  // G(X): F_a of the sparse iterate, range pass with conj(H3), conj(H2), conj(H1)
  c.out = b.z;
  LK(sparse_forward(plan, c, s));
  LK(mark(1));
  LK(range_pass(plan, row_args(plan, b.z, plan->coef_g), true, s));
  LK(mark(2));
  // residue r = S.(Y - G(X)), produced as F_a r = F_a(S.Y) - F_a(S.G(X)): this column
  // pass forms F_a(S.G(X)), the next range pass subtracts it from F_a(S.Y)
  c.in = b.z;
  c.out = b.z;
  (void)y;
  c.mask = mask;
  LK(launch_col(na, plan->col_res, COL_RESID, c, nt, s));
  LK(mark(3));
  // M(r): range pass with H1, H2, H3 on F_a r = F_a(S.Y) - F_a(S.G(X))
  RowArgs rm = row_args(plan, b.z, plan->coef_m);
  rm.yf = b.yf;
  rm.partial = b.partial;
  rm.ctl = b.ctl;
  rm.resid_scale = 1.0f / (float)na;
  LK(range_pass(plan, rm, false, s));
  LK(mark(4));
  // Delta X = F_a^-1: support values, histogram, candidates
  LK(launch_col(na, plan->col, COL_SELECT, c, nt, s));
  LK(mark(5));
  SelArgs sa = sel_args(plan, cur, o);
  // the re-passes are conditional graph nodes when captured (set by the check kernels)
  const bool cap = capturing(s);
  if (cap) {
    LK(capture_handle(s, &sa.h_repass));
    LK(capture_handle(s, &sa.h_repass2));
    if (o.mu_mode == CSAR_MU_FIXED) {
      LK(capture_handle(s, &sa.h_fused));
      LK(capture_handle(s, &sa.h_multi));
    }
  }
  LK(launch_sel_check(sa, s));
  LK(enqueue_if(s, plan->cond_stream, sa.h_repass, [&](cudaStream_t q) {
    ColArgs r = c;
    r.gate_val = kRepassCut;
    return launch_col(na, plan->col, COL_REPASS, r, nt, q);
  }));
  LK(enqueue_if(s, plan->cond_stream, sa.h_repass2, [&](cudaStream_t q) {
    LK(launch_sel_check2(sa, q));
    ColArgs r = c;
    r.gate_val = kRepassCut2;
    return launch_col(na, plan->col, COL_REPASS, r, nt, q);
  }));
  if (o.mu_mode == CSAR_MU_NIHT) {
    // NIHT step on Gamma = supp X^(i) (skipped on the device when the support is empty)
    ColArgs g = col_args(plan);
    g.gate = &b.ctl->niht_first;
    g.gate_val = 0u;
    g.xs_off = b.off[cur];
    g.xs_idx = b.idx[cur];
    g.xs_val = b.dx;
    g.out = b.z;
    LK(sparse_forward(plan, g, s));
    RowArgs r = row_args(plan, b.z, plan->coef_g);
    r.gate = g.gate;
    r.gate_val = 0u;
    LK(range_pass(plan, r, true, s));
    g.in = b.z;
    g.mask = mask;
    g.partial = b.partial_norm;
    LK(launch_col(na, plan->col_res, COL_NORM, g, nt, s));
    LK(launch_niht_mu_mode(sa, 0, s));
  }
  // selection and threshold: one CTA when the union fits (fixed step), else the
  // grid-wide radix select; the check kernel decides (conditional nodes when captured,
  // early exits otherwise)
  auto multi = [&](cudaStream_t q) -> cudaError_t {
    for (int lev = 0; lev < 3; ++lev) {
      LK(launch_sel_round(sa, lev, q));
      LK(launch_sel_pick(sa, lev, q));
    }
    LK(launch_thr_count(sa, q));
    LK(launch_thr_scan(sa, q));
    return launch_thr_scatter_mode(sa, o.mu_mode == CSAR_MU_NIHT ? 1 : 0, q);
  };
  if (o.mu_mode == CSAR_MU_FIXED) {
    LK(enqueue_if(s, plan->cond_stream, sa.h_fused, [&](cudaStream_t q) { return launch_sel_fused(sa, q); }));
    LK(enqueue_if(s, plan->cond_stream, sa.h_multi, multi));
  } else {
    LK(multi(s));
  }
  if (plan->dump.idx) LK(launch_sel_dump(sa, plan->dump, s));
  if (o.mu_mode == CSAR_MU_NIHT) {
    // first iteration: Gamma = the top-K list just written (raw Delta X values)
    ColArgs g = col_args(plan);
    g.gate = &b.ctl->niht_first;
    g.gate_val = 1u;
    g.xs_off = b.off[nxt];
    g.xs_idx = b.idx[nxt];
    g.xs_val = b.val[nxt];
    g.out = b.z;
    LK(sparse_forward(plan, g, s));
    RowArgs r = row_args(plan, b.z, plan->coef_g);
    r.gate = g.gate;
    r.gate_val = 1u;
    LK(range_pass(plan, r, true, s));
    g.in = b.z;
    g.mask = mask;
    g.partial = b.partial_norm;
    LK(launch_col(na, plan->col_res, COL_NORM, g, nt, s));
    LK(launch_niht_mu_mode(sa, 1, s));
  }
  if (b.ck_active)
    LK(launch_ckpt_copy(b.ctl, b.idx[nxt], b.val[nxt], b.ck_idx, b.ck_val, b.ck_meta, b.ck_cap, s));
  LK(launch_sel_finish(sa, s));
  LK(mark(6));
  return cudaSuccess;
}

__global__ void k_ctl_init(Ctl* c, uint32_t nx_from_list, const uint32_t* off0, int n_tiles) {
  Ctl z{};
  z.cut_key = kNoCandidates;
  z.jstar = 0xffffffffu;
  z.nx = nx_from_list ? off0[n_tiles] : 0u;
  *c = z;
}

// Deterministic synthetic echo and 50% mask for the autotuner (hash of the index).
__global__ void k_fill_synthetic(float2* y, uint32_t* mask, long long n, uint32_t seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    y[i] = make_float2((float)(h & 0xffff) / 65536.f - 0.5f, (float)(h >> 16) / 65536.f - 0.5f);
    if ((i & 31) == 0) mask[i >> 5] = h * 3266489917u;
  }
}

csar_status check_opts(csar_plan plan, const csar_opts* o, bool need_iters) {
  if (!o) return fail(CSAR_E_INVALID, "opts is NULL");
  if (o->K < 0) return fail(CSAR_E_INVALID, "K must be >= 0");
  if (need_iters && o->iters < 0) return fail(CSAR_E_INVALID, "iters must be >= 0");
  if (o->mu_mode != CSAR_MU_FIXED && o->mu_mode != CSAR_MU_NIHT)
    return fail(CSAR_E_INVALID, "mu_mode must be CSAR_MU_FIXED or CSAR_MU_NIHT");
  if (o->mu_mode == CSAR_MU_FIXED && !(o->mu > 0.f && std::isfinite(o->mu)))
    return fail(CSAR_E_INVALID, "mu must be finite and > 0");
  if (o->thresh != CSAR_THRESH_SOFT && o->thresh != CSAR_THRESH_HALF && o->thresh != CSAR_THRESH_HARD)
    return fail(CSAR_E_INVALID, "thresh must be CSAR_THRESH_SOFT, CSAR_THRESH_HALF or CSAR_THRESH_HARD");
  return CSAR_OK;
}

// Dense operator on device arrays: out = G(in) or M(in) (in may equal out).
cudaError_t dense_op(csar_plan plan, const float2* in, float2* out, bool is_g, cudaStream_t s) {
  ColArgs c = col_args(plan);
  c.in = in;
  c.out = out;
  LK(launch_col(plan->na, plan->col, COL_FWD, c, plan->n_tiles, s));
  LK(range_pass(plan, row_args(plan, out, is_g ? plan->coef_g : plan->coef_m), is_g, s));
  c.in = out;
  return launch_col(plan->na, plan->col, COL_INV, c, plan->n_tiles, s);
}

csar_status run_op(csar_plan plan, const void* in, void* out, bool is_g, void* stream) {
  NvtxRange nvtx_(is_g ? "csar_G" : "csar_M");
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (!in || !out) return fail(CSAR_E_INVALID, "null data pointer");
  const size_t bytes = (size_t)plan->n * sizeof(float2);
  const char* ib = (const char*)in;
  const char* ob = (const char*)out;
  if (ib != ob && ib < ob + bytes && ob < ib + bytes)
    return fail(CSAR_E_INVALID, "input and output overlap without being identical");
  DeviceGuard dg(plan->dev);
  cudaStream_t s = (cudaStream_t)stream;
  ColArgs c = col_args(plan);
  c.in = (const float2*)in;
  c.out = (float2*)out;
  cudaError_t e = launch_col(plan->na, plan->col, COL_FWD, c, plan->n_tiles, s);
  if (e == cudaSuccess)
    e = range_pass(plan, row_args(plan, (float2*)out, is_g ? plan->coef_g : plan->coef_m), is_g, s);
  c.in = (const float2*)out;
  if (e == cudaSuccess) e = launch_col(plan->na, plan->col, COL_INV, c, plan->n_tiles, s);
  if (e != cudaSuccess) return cuda_fail(e, is_g ? "csar_G" : "csar_M");
  return CSAR_OK;
}

// Per-solve preparation of the inputs: the sampling mask in column-pass order and
// F_a(S . Y) (uses the pass-to-pass buffer as scratch).
cudaError_t prepare_inputs(csar_plan plan, const float2* y, const uint32_t* mask, cudaStream_t s) {
  Buffers& b = plan->b;
  LK(launch_mask_transpose(plan->na, plan->col_res.p, plan->nr, mask, b.mask_t, s));
  LK(launch_mask_apply(y, mask, b.z, plan->n, s));
  ColArgs c = col_args(plan);
  c.in = b.z;
  c.out = b.yf;
  return launch_col(plan->na, plan->col, COL_FWD, c, plan->n_tiles, s);
}

csar_status latched(csar_plan plan) {
  Ctl c;
  CK(cudaMemcpy(&c, plan->b.ctl, sizeof c, cudaMemcpyDeviceToHost));
  if (c.err) {
    const uint32_t zero = 0;
    CK(cudaMemcpy(&plan->b.ctl->err, &zero, sizeof zero, cudaMemcpyHostToDevice));
    if (c.err & kErrNonfinite) return fail(CSAR_E_NONFINITE, "non-finite value in the echo or iterate");
    if (c.err & kErrCapacity)
      return fail(CSAR_E_INTERNAL, "selection candidate capacity exceeded (degenerate magnitudes)");
    if (c.err & kErrTimeout)
      return fail(CSAR_E_TIMEOUT, "a column-pass cluster exchange timed out (a peer CTA never signalled)");
    if (c.err & kErrIndex)
      return fail(CSAR_E_INTERNAL, "an index out of range was caught and skipped (checked build)");
    return fail(CSAR_E_INTERNAL, "device error bits 0x%x", c.err);
  }
  return CSAR_OK;
}

// Run `iters` iterations starting from list 0 (already initialised); returns the
// parity holding the result.
csar_status run_iterations(csar_plan plan, const float2* y, const uint32_t* mask, const csar_opts& o,
                           int iters, cudaStream_t s, int* result_parity) {
  int cur = 0;
  for (int i = 0; i < iters; ++i) {
    if (plan->use_graphs) {
      GraphKey k;
      k.y = y;
      k.mask = mask;
      k.K = o.K;
      k.mu_mode = o.mu_mode;
      k.thresh = o.thresh;
      k.mu = o.mu;
      k.cand_cap = plan->b.cand_cap;
      k.stats = plan->b.stats;
      k.ck = plan->b.ck_active ? (const void*)plan->b.ck_idx : nullptr;
      k.dump = plan->dump.idx;
      if (!plan->exec[cur] || !(plan->key[cur] == k)) {
        if (plan->exec[cur]) cudaGraphExecDestroy(plan->exec[cur]);
        plan->exec[cur] = nullptr;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_iteration(plan, y, cur, o, plan->cap_stream, nullptr);
        cudaError_t e2 = cudaStreamEndCapture(plan->cap_stream, &g);
        if (e != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          return cuda_fail(e, "capture of the ITA iteration");
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        cudaError_t e3 = cudaGraphInstantiate(&plan->exec[cur], g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) return cuda_fail(e3, "cudaGraphInstantiate");
        plan->key[cur] = k;
      }
      CK(cudaGraphLaunch(plan->exec[cur], s));
    } else {
      cudaError_t e = enqueue_iteration(plan, y, cur, o, s, nullptr);
      if (e != cudaSuccess) return cuda_fail(e, "ITA iteration");
    }
    cur = 1 - cur;
  }
  *result_parity = cur;
  return CSAR_OK;
}

csar_status solve_impl(csar_plan plan, const void* Y, const uint32_t* mask, void* X, const csar_opts* o,
                       const csar_stats* stats, cudaStream_t s) {
  if (csar_status st = check_opts(plan, o, true)) return st;
  if (!Y || !mask || !X) return fail(CSAR_E_INVALID, "null data pointer");
  if (csar_status st = ensure_capacity(plan, o->K, o->iters)) return st;
  Buffers& b = plan->b;
  CK(prepare_inputs(plan, (const float2*)Y, mask, s));
  // X^(0) = 0: empty list 0, fresh control block
  CK(cudaMemsetAsync(b.off[0], 0, (plan->n_tiles + 1) * sizeof(uint32_t), s));
  k_ctl_init<<<1, 1, 0, s>>>(b.ctl, 0u, b.off[0], plan->n_tiles);
  CK(cudaGetLastError());
  int par = 0;
  if (csar_status st = run_iterations(plan, (const float2*)Y, mask, *o, o->iters, s, &par)) return st;
  CK(cudaMemsetAsync(X, 0, (size_t)plan->n * sizeof(float2), s));
  CK(launch_list_to_dense(b.off[par], b.idx[par], b.val[par], plan->n_tiles, (float2*)X, s));
  if (stats && o->iters > 0) {
    std::vector<IterStat> h(o->iters);
    CK(cudaMemcpyAsync(h.data(), b.stats, o->iters * sizeof(IterStat), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < o->iters; ++i) {
      if (stats->resid_sq) stats->resid_sq[i] = h[i].resid_sq;
      if (stats->mu) stats->mu[i] = h[i].mu;
      if (stats->sigma) stats->sigma[i] = h[i].sigma;
      if (stats->nnz) stats->nnz[i] = h[i].nnz;
    }
    return latched(plan);
  }
  return CSAR_OK;
}


csar_status ensure_af(csar_plan plan, int64_t K, int iters) {
  Buffers& b = plan->b;
  const size_t n = (size_t)plan->n;
  if (!b.yt || !b.af_xbar || !b.af_bbar || !b.af_h || !b.row_loss) {
    // all or none: a failed allocation leaves none behind
    cudaError_t e = b.yt ? cudaSuccess : dalloc(&b.yt, n);
    if (e == cudaSuccess && !b.af_xbar) e = dalloc(&b.af_xbar, n);
    if (e == cudaSuccess && !b.af_bbar) e = dalloc(&b.af_bbar, n);
    if (e == cudaSuccess && !b.af_h) e = dalloc(&b.af_h, n);
    if (e == cudaSuccess && !b.row_loss) e = dalloc(&b.row_loss, plan->na);
    if (e != cudaSuccess) {
      for (void* q : {(void*)b.yt, (void*)b.af_xbar, (void*)b.af_bbar, (void*)b.af_h, (void*)b.row_loss})
        if (q) cudaFree(q);
      b.yt = nullptr;
      b.af_xbar = nullptr;
      b.af_bbar = nullptr;
      b.af_h = nullptr;
      b.row_loss = nullptr;
      return cuda_fail(e, "autofocus workspace");
    }
  }
  const uint32_t cap = (uint32_t)std::min<int64_t>(plan->n, std::max<int64_t>(K, 1));
  if (iters > 0 && (b.ck_cap < cap || b.ck_iters_cap < iters)) {
    drop_graphs(plan);
    if (b.ck_idx) cudaFree(b.ck_idx);
    if (b.ck_val) cudaFree(b.ck_val);
    if (b.ck_meta) cudaFree(b.ck_meta);
    b.ck_idx = nullptr;
    b.ck_val = nullptr;
    b.ck_meta = nullptr;
    b.ck_cap = 0;
    b.ck_iters_cap = 0;
    CK(dalloc(&b.ck_idx, (size_t)cap * iters));
    CK(dalloc(&b.ck_val, (size_t)cap * iters));
    CK(dalloc(&b.ck_meta, (size_t)iters));
    b.ck_cap = cap;
    b.ck_iters_cap = iters;
  }
  return CSAR_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

const char* csar_last_error(void) { return g_last_error.c_str(); }

int32_t csar_version(void) { return 10000; }

csar_status csar_plan_create(const csar_params* params, uint32_t flags, csar_plan* out) {
  NvtxRange nvtx_("csar_plan_create");
  if (!out) return fail(CSAR_E_INVALID, "out is NULL");
  *out = nullptr;
  if (flags & ~(0xff00u | CSAR_PLAN_COL_HALF_TILE | CSAR_PLAN_COL_WIDE_TILE | CSAR_PLAN_RDA |
                CSAR_PLAN_COL_PERSIST | CSAR_PLAN_COL_NO_PERSIST | CSAR_PLAN_BATCH_MEMBER))
    return fail(CSAR_E_INVALID, "unknown plan flags 0x%x", flags);
  const bool member = (flags & CSAR_PLAN_BATCH_MEMBER) != 0;
  if (member) {
    if (flags & (0xff00u | CSAR_PLAN_COL_HALF_TILE | CSAR_PLAN_COL_WIDE_TILE | CSAR_PLAN_COL_PERSIST |
                 CSAR_PLAN_COL_NO_PERSIST | CSAR_PLAN_RDA))
      return fail(CSAR_E_INVALID, "CSAR_PLAN_BATCH_MEMBER with other column or operator flags");
    if (!params) return fail(CSAR_E_INVALID, "params is NULL");
    if (!batch_member_ok(params->n_az, params->n_rg))
      return fail(CSAR_E_UNSUPPORTED, "batch member plans need n_az, n_rg in {512, 1024, 2048, 4096}");
    flags |= CSAR_PLAN_COL_CLUSTER(batch_col_cluster(params->n_az)) | CSAR_PLAN_COL_HALF_TILE |
             CSAR_PLAN_COL_NO_PERSIST;
  }
  if ((flags & CSAR_PLAN_COL_PERSIST) && (flags & CSAR_PLAN_COL_NO_PERSIST))
    return fail(CSAR_E_INVALID, "CSAR_PLAN_COL_PERSIST with CSAR_PLAN_COL_NO_PERSIST");
  const uint32_t tile_flags = flags & (CSAR_PLAN_COL_HALF_TILE | CSAR_PLAN_COL_WIDE_TILE);
  if (tile_flags == (CSAR_PLAN_COL_HALF_TILE | CSAR_PLAN_COL_WIDE_TILE))
    return fail(CSAR_E_UNSUPPORTED, "half and wide column tiles together");
  const int forced_p = (int)((flags >> 8) & 0xffu);
  ColConf forced;
  forced.p = forced_p;
  forced.e = (flags & CSAR_PLAN_COL_HALF_TILE) ? kColCtaElems / 2
                                               : ((flags & CSAR_PLAN_COL_WIDE_TILE) ? 2 * kColCtaElems : kColCtaElems);
  const bool persist = (flags & CSAR_PLAN_COL_PERSIST) != 0;
  if ((forced_p || tile_flags) && params) {
    if (!forced_p) forced.p = col_conf_default(params->n_az).p;
    forced.persist = persist;
    if (!col_conf_ok(params->n_az, forced))
      return fail(CSAR_E_UNSUPPORTED, "column configuration (cluster %d, %d values per CTA%s) not available "
                  "for n_az=%d", forced.p, forced.e, persist ? ", persistent" : "", params->n_az);
  } else if (persist && params) {
    forced = col_conf_persist(params->n_az);
    if (!col_conf_ok(params->n_az, forced))
      return fail(CSAR_E_UNSUPPORTED, "persistent column passes not available for n_az=%d", params->n_az);
  }
  if (csar_status st = validate(params)) return st;
  std::vector<RowCoef> cg(params->n_az), cm(params->n_az);
  if (csar_status st = build_coefs_into(*params, cg.data(), cm.data())) return st;
  // range-Doppler tables, also checked on the host before any CUDA call
  std::vector<RowCoef> rg, rm;
  std::vector<RcmcCoef> rc;
  if (flags & CSAR_PLAN_RDA) {
    rg.resize(params->n_az);
    rm.resize(params->n_az);
    rc.resize(2 * (size_t)params->n_az);
    if (csar_status st = build_rda_coefs(*params, rg.data(), rm.data(), rc.data())) return st;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  csar_plan plan = new csar_plan_s();
  plan->p = *params;
  plan->dev = dev;
  plan->na = params->n_az;
  plan->nr = params->n_rg;
  plan->n = (int64_t)plan->na * plan->nr;
  if (forced_p || tile_flags || persist) {
    plan->col = plan->col_res = forced;
  } else if (!tuned_conf(plan->na, plan->nr, &plan->col, &plan->col_res)) {
    plan->col = col_conf_default(plan->na);
    plan->col_res = col_conf_default_res(plan->na);
  }
  if (flags & CSAR_PLAN_COL_NO_PERSIST) plan->col.persist = plan->col_res.persist = false;
  // both configurations bucket the sparse iterate by the same tile width
  if (col_w(plan->na, plan->col_res.p, plan->col_res.e) != col_w(plan->na, plan->col.p, plan->col.e))
    plan->col_res = plan->col;
  plan->col_tile = col_w(plan->na, plan->col.p, plan->col.e);
  plan->n_tiles = plan->nr / plan->col_tile;
  if (const char* sf = std::getenv("CSAR_SEL_FUSED")) plan->sel_fused_ok = sf[0] != '0';
  plan->row_regs = tuned_row_regs(plan->na, plan->nr);
  if (const char* rr = std::getenv("CSAR_ROW_REGS")) plan->row_regs = std::atoi(rr) == 16 ? 16 : 0;
  if (member) {
    plan->row_regs = 0;
    plan->no_direct = true;
  }
  const char* ng = std::getenv("CSAR_NO_GRAPH");
  plan->use_graphs = !(ng && ng[0] == '1');
  auto bail = [&](csar_status st) {
    csar_plan_destroy(plan);
    return st;
  };
  cudaError_t e;
#define PK(call)                                      \
  if ((e = (call)) != cudaSuccess) {                  \
    csar_status st_ = cuda_fail(e, #call);            \
    return bail(st_);                                 \
  }
  PK(sel_set_attributes());
  PK(col_set_attributes(plan->na, plan->col));
  PK(col_set_attributes(plan->na, plan->col_res));
  PK(row_set_attributes(plan->nr));
  PK(sparse_dft_set_attributes(plan->na));
  PK(dalloc(&plan->coef_g, plan->na));
  PK(dalloc(&plan->coef_m, plan->na));
  PK(cudaMemcpy(plan->coef_g, cg.data(), cg.size() * sizeof(RowCoef), cudaMemcpyHostToDevice));
  PK(cudaMemcpy(plan->coef_m, cm.data(), cm.size() * sizeof(RowCoef), cudaMemcpyHostToDevice));
  if (flags & CSAR_PLAN_RDA) {
    PK(rda_set_attributes(plan->nr));
    PK(dalloc(&plan->rda_rg_g, plan->na));
    PK(dalloc(&plan->rda_rg_m, plan->na));
    PK(dalloc(&plan->rda_rcmc, 2 * (size_t)plan->na));
    PK(cudaMemcpy(plan->rda_rg_g, rg.data(), rg.size() * sizeof(RowCoef), cudaMemcpyHostToDevice));
    PK(cudaMemcpy(plan->rda_rg_m, rm.data(), rm.size() * sizeof(RowCoef), cudaMemcpyHostToDevice));
    PK(cudaMemcpy(plan->rda_rcmc, rc.data(), rc.size() * sizeof(RcmcCoef), cudaMemcpyHostToDevice));
    plan->rda = true;
  }
  {
    std::vector<float2> tw(kTwLo + kTwHi);
    build_twiddles(tw.data());
    PK(dalloc(&plan->tw, tw.size()));
    PK(cudaMemcpy(plan->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  Buffers& b = plan->b;
  const size_t n = (size_t)plan->n;
  const int nt = plan->n_tiles;
  PK(dalloc(&b.z, n));
  for (int i = 0; i < 2; ++i) {
    PK(dalloc(&b.off[i], nt + 1));
    PK(dalloc(&b.idx[i], n));
    PK(dalloc(&b.val[i], n));
    PK(cudaMemset(b.off[i], 0, (nt + 1) * sizeof(uint32_t)));
  }
  PK(dalloc(&b.dx, n));
  PK(dalloc(&b.yf, n));
  PK(dalloc(&b.hist, kHistBins));
  PK(dalloc(&b.hist2, kHistBins));
  PK(dalloc(&b.tile_cnt, nt));
  PK(dalloc(&b.tile_cur, nt));
  PK(dalloc(&b.partial, (size_t)std::max(nt * plan->col_res.p, row_ctas(plan->na, plan->nr))));
  PK(dalloc(&b.partial_norm, (size_t)nt * plan->col_res.p));
  PK(dalloc(&b.mask_t, (size_t)col_mask_words(plan->na, plan->nr, plan->col_res.p)));
  PK(dalloc(&b.ctl, 1));
  PK(cudaMemset(b.hist, 0, kHistBins * sizeof(uint32_t)));
  PK(cudaMemset(b.hist2, 0, kHistBins * sizeof(uint32_t)));
  PK(cudaMemset(b.tile_cnt, 0, nt * sizeof(uint32_t)));
  PK(cudaMemset(b.ctl, 0, sizeof(Ctl)));
  PK(cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking));
  PK(cudaStreamCreateWithFlags(&plan->cond_stream, cudaStreamNonBlocking));
#undef PK
  *out = plan;
  return CSAR_OK;
}

csar_status csar_plan_destroy(csar_plan plan) {
  if (!plan) return CSAR_OK;
  DeviceGuard dg(plan->dev);
  cudaDeviceSynchronize();
  drop_graphs(plan);
  if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
  if (plan->cond_stream) cudaStreamDestroy(plan->cond_stream);
  free_buffers(plan->b);
  void* dump[] = {plan->dump.idx, plan->dump.b, plan->dump.key, plan->dump.count, plan->dump.ctl};
  for (void* q : dump)
    if (q) cudaFree(q);
  if (plan->coef_g) cudaFree(plan->coef_g);
  if (plan->coef_m) cudaFree(plan->coef_m);
  if (plan->rda_rg_g) cudaFree(plan->rda_rg_g);
  if (plan->rda_rg_m) cudaFree(plan->rda_rg_m);
  if (plan->rda_pulse_g) cudaFree(plan->rda_pulse_g);
  if (plan->rda_pulse_m) cudaFree(plan->rda_pulse_m);
  if (plan->rda_rcmc) cudaFree(plan->rda_rcmc);
  if (plan->tw) cudaFree(plan->tw);
  delete plan;
  return CSAR_OK;
}

csar_status csar_G(csar_plan plan, const void* x_dev, void* y_dev, void* stream) {
  return run_op(plan, x_dev, y_dev, true, stream);
}

csar_status csar_M(csar_plan plan, const void* y_dev, void* x_dev, void* stream) {
  return run_op(plan, y_dev, x_dev, false, stream);
}

csar_status csar_ita_step(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev, void* X_dev,
                          const csar_opts* opts, float* sigma_dev, void* stream) {
  NvtxRange nvtx_("csar_ita_step");
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (csar_status st = check_opts(plan, opts, false)) return st;
  if (!Y_dev || !mask_dev || !X_dev) return fail(CSAR_E_INVALID, "null data pointer");
  DeviceGuard dg(plan->dev);
  if (csar_status st = ensure_capacity(plan, opts->K, 1)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Buffers& b = plan->b;
  const float2* X = (const float2*)X_dev;
  // dense X -> bucketed list 0
  CK(launch_dense_count(X, plan->na, plan->nr, plan->col_tile, b.tile_cnt, s));
  CK(launch_dense_scan(b.tile_cnt, b.tile_cur, b.off[0], plan->n_tiles, nullptr, s));
  CK(launch_dense_scatter(X, plan->na, plan->nr, plan->col_tile, b.tile_cur, b.idx[0], b.val[0], s));
  k_ctl_init<<<1, 1, 0, s>>>(b.ctl, 1u, b.off[0], plan->n_tiles);
  CK(cudaGetLastError());
  CK(prepare_inputs(plan, (const float2*)Y_dev, mask_dev, s));
  cudaError_t e = enqueue_iteration(plan, (const float2*)Y_dev, 0, *opts, s, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "csar_ita_step");
  CK(cudaMemsetAsync(X_dev, 0, (size_t)plan->n * sizeof(float2), s));
  CK(launch_list_to_dense(b.off[1], b.idx[1], b.val[1], plan->n_tiles, (float2*)X_dev, s));
  if (sigma_dev)
    CK(cudaMemcpyAsync(sigma_dev, &b.ctl->sigma, sizeof(float), cudaMemcpyDeviceToDevice, s));
  return CSAR_OK;
}

csar_status csar_solve(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev, void* X_dev,
                       const csar_opts* opts, const csar_stats* stats, void* stream) {
  NvtxRange nvtx_("csar_solve");
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  DeviceGuard dg(plan->dev);
  return solve_impl(plan, Y_dev, mask_dev, X_dev, opts, stats, (cudaStream_t)stream);
}

csar_status csar_solve_host(csar_plan plan, const void* Y_host, const uint32_t* mask_host, void* X_host,
                            const csar_opts* opts, const csar_stats* stats, void* stream) {
  NvtxRange nvtx_("csar_solve_host");
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (!Y_host || !mask_host || !X_host) return fail(CSAR_E_INVALID, "null data pointer");
  DeviceGuard dg(plan->dev);
  Buffers& b = plan->b;
  const size_t n = (size_t)plan->n;
  if (!b.hY || !b.hMask || !b.hX) {
    // all three or none: a failed allocation leaves none behind
    cudaError_t e = b.hY ? cudaSuccess : dalloc(&b.hY, n);
    if (e == cudaSuccess && !b.hMask) e = dalloc(&b.hMask, n / 32);
    if (e == cudaSuccess && !b.hX) e = dalloc(&b.hX, n);
    if (e != cudaSuccess) {
      for (void* q : {(void*)b.hY, (void*)b.hMask, (void*)b.hX})
        if (q) cudaFree(q);
      b.hY = nullptr;
      b.hMask = nullptr;
      b.hX = nullptr;
      return cuda_fail(e, "host-buffer staging");
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(b.hY, Y_host, n * sizeof(float2), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b.hMask, mask_host, n / 32 * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  if (csar_status st = solve_impl(plan, b.hY, b.hMask, b.hX, opts, stats, s)) return st;
  CK(cudaMemcpyAsync(X_host, b.hX, n * sizeof(float2), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return latched(plan);
}

csar_status csar_plan_check(csar_plan plan) {
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  DeviceGuard dg(plan->dev);
  CK(cudaDeviceSynchronize());
  return latched(plan);
}

csar_status csar_plan_set_pulse(csar_plan plan, const float* spectrum_host) {
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (!plan->rda)
    return fail(CSAR_E_UNSUPPORTED, "a recorded pulse replaces the range filter of the range-Doppler "
                "pair; chirp scaling assumes a linear FM pulse");
  const int nr = plan->nr;
  std::vector<float2> sg, sm;
  if (spectrum_host) {
    sg.resize(nr);
    sm.resize(nr);
    for (int j = 0; j < nr; ++j) {
      const float re = spectrum_host[2 * j], im = spectrum_host[2 * j + 1];
      if (!std::isfinite(re) || !std::isfinite(im)) return fail(CSAR_E_INVALID, "pulse spectrum bin %d is not finite", j);
      sg[j] = make_float2(re, im);
      sm[j] = make_float2(re, -im);
    }
  }
  DeviceGuard dg(plan->dev);
  CK(cudaDeviceSynchronize());
  drop_graphs(plan);
  if (!spectrum_host) {
    if (plan->rda_pulse_g) cudaFree(plan->rda_pulse_g);
    if (plan->rda_pulse_m) cudaFree(plan->rda_pulse_m);
    plan->rda_pulse_g = plan->rda_pulse_m = nullptr;
    return CSAR_OK;
  }
  if (!plan->rda_pulse_g) {
    float2* g = nullptr;
    float2* m = nullptr;
    cudaError_t e = dalloc(&g, (size_t)nr);
    if (e == cudaSuccess) e = dalloc(&m, (size_t)nr);
    if (e != cudaSuccess) {
      if (g) cudaFree(g);
      if (m) cudaFree(m);
      return fail(CSAR_E_OOM, "pulse spectrum: %s", cudaGetErrorString(e));
    }
    plan->rda_pulse_g = g;
    plan->rda_pulse_m = m;
  }
  CK(cudaMemcpy(plan->rda_pulse_g, sg.data(), nr * sizeof(float2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(plan->rda_pulse_m, sm.data(), nr * sizeof(float2), cudaMemcpyHostToDevice));
  return CSAR_OK;
}

csar_status csar_debug_selection_enable(csar_plan plan, int64_t capacity) {
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (capacity < 0 || capacity > plan->n + (int64_t)plan->b.cand_cap + (int64_t(1) << 24))
    return fail(CSAR_E_INVALID, "capacity out of range");
  DeviceGuard dg(plan->dev);
  CK(cudaDeviceSynchronize());
  drop_graphs(plan);
  SelDump& d = plan->dump;
  void* old[] = {d.idx, d.b, d.key, d.count, d.ctl};
  for (void* q : old)
    if (q) cudaFree(q);
  d = SelDump();
  if (capacity == 0) return CSAR_OK;
  SelDump n;
  cudaError_t e = dalloc(&n.idx, (size_t)capacity);
  if (e == cudaSuccess) e = dalloc(&n.b, (size_t)capacity);
  if (e == cudaSuccess) e = dalloc(&n.key, (size_t)capacity);
  if (e == cudaSuccess) e = dalloc(&n.count, 1);
  if (e == cudaSuccess) e = dalloc(&n.ctl, 1);
  if (e != cudaSuccess) {
    void* part[] = {n.idx, n.b, n.key, n.count, n.ctl};
    for (void* q : part)
      if (q) cudaFree(q);
    return fail(CSAR_E_OOM, "selection record: %s", cudaGetErrorString(e));
  }
  n.cap = (uint32_t)capacity;
  d = n;
  return CSAR_OK;
}

csar_status csar_debug_selection_read(csar_plan plan, uint32_t* idx_host, float* b_host, uint32_t* key_host,
                                      int64_t capacity, int64_t* count, uint32_t* sigma2_key, float* mu,
                                      float* sigma) {
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (!plan->dump.idx) return fail(CSAR_E_INVALID, "selection record not enabled");
  if (!count || !sigma2_key || !mu || !sigma) return fail(CSAR_E_INVALID, "null output pointer");
  DeviceGuard dg(plan->dev);
  CK(cudaDeviceSynchronize());
  uint32_t nu = 0;
  Ctl c;
  CK(cudaMemcpy(&nu, plan->dump.count, sizeof nu, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&c, plan->dump.ctl, sizeof c, cudaMemcpyDeviceToHost));
  *count = nu;
  *sigma2_key = c.sigma2_key;
  *mu = c.mu;
  *sigma = c.sigma;
  const int64_t m = std::min<int64_t>({(int64_t)nu, (int64_t)plan->dump.cap, capacity});
  if (m > 0 && idx_host) CK(cudaMemcpy(idx_host, plan->dump.idx, m * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (m > 0 && b_host) CK(cudaMemcpy(b_host, plan->dump.b, m * sizeof(float2), cudaMemcpyDeviceToHost));
  if (m > 0 && key_host) CK(cudaMemcpy(key_host, plan->dump.key, m * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if ((int64_t)nu > (int64_t)plan->dump.cap) return fail(CSAR_E_INTERNAL, "union larger than the record's capacity");
  return latched(plan);
}

csar_status csar_debug_fail_alloc(int32_t n) {
  if (n < 0) return fail(CSAR_E_INVALID, "n must be >= 0");
  g_alloc_count.store(0);
  g_fail_alloc_at.store(n);
  return CSAR_OK;
}

csar_status csar_solve_profile(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev, void* X_dev,
                               const csar_opts* opts, float* pass_ms, int32_t n_pass, void* stream) {
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (csar_status st = check_opts(plan, opts, true)) return st;
  if (!Y_dev || !mask_dev || !X_dev || !pass_ms || n_pass < kPasses)
    return fail(CSAR_E_INVALID, "null pointer or n_pass < %d", kPasses);
  DeviceGuard dg(plan->dev);
  if (csar_status st = ensure_capacity(plan, opts->K, opts->iters)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Buffers& b = plan->b;
  const int iters = opts->iters;
  std::vector<cudaEvent_t> ev((size_t)(kPasses + 1) * std::max(iters, 1));
  for (auto& x : ev) CK(cudaEventCreate(&x));
  CK(prepare_inputs(plan, (const float2*)Y_dev, mask_dev, s));
  CK(cudaMemsetAsync(b.off[0], 0, (plan->n_tiles + 1) * sizeof(uint32_t), s));
  k_ctl_init<<<1, 1, 0, s>>>(b.ctl, 0u, b.off[0], plan->n_tiles);
  int cur = 0;
  for (int i = 0; i < iters; ++i) {
    cudaError_t e = enqueue_iteration(plan, (const float2*)Y_dev, cur, *opts, s,
                                      &ev[(size_t)i * (kPasses + 1)]);
    if (e != cudaSuccess) return cuda_fail(e, "csar_solve_profile");
    cur = 1 - cur;
  }
  CK(cudaMemsetAsync(X_dev, 0, (size_t)plan->n * sizeof(float2), s));
  CK(launch_list_to_dense(b.off[cur], b.idx[cur], b.val[cur], plan->n_tiles, (float2*)X_dev, s));
  CK(cudaStreamSynchronize(s));
  for (int p = 0; p < kPasses; ++p) pass_ms[p] = 0.f;
  for (int i = 0; i < iters; ++i)
    for (int p = 0; p < kPasses; ++p) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[(size_t)i * (kPasses + 1) + p], ev[(size_t)i * (kPasses + 1) + p + 1]));
      pass_ms[p] += ms;
    }
  for (auto& x : ev) cudaEventDestroy(x);
  return latched(plan);
}

csar_status csar_af_solve(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev, const float* theta_dev,
                          void* X_dev, const csar_opts* opts, int32_t checkpoint, void* stream) {
  NvtxRange nvtx_("csar_af_solve");
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (!theta_dev) return fail(CSAR_E_INVALID, "theta is NULL");
  if (plan->rda) return fail(CSAR_E_UNSUPPORTED, "autofocus uses the chirp-scaling operator pair");
  if (csar_status st = check_opts(plan, opts, true)) return st;
  if (checkpoint && (opts->thresh != CSAR_THRESH_SOFT || opts->mu_mode != CSAR_MU_FIXED))
    return fail(CSAR_E_UNSUPPORTED, "the autofocus backward covers soft thresholding with a fixed step");
  if (!Y_dev || !mask_dev || !X_dev) return fail(CSAR_E_INVALID, "null data pointer");
  DeviceGuard dg(plan->dev);
  if (csar_status st = ensure_af(plan, opts->K, checkpoint ? opts->iters : 0)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Buffers& b = plan->b;
  CK(launch_rotate_rows((const float2*)Y_dev, theta_dev, b.yt, plan->na, plan->nr, s));
  b.ck_active = checkpoint != 0;
  csar_status st = solve_impl(plan, b.yt, mask_dev, X_dev, opts, nullptr, s);
  b.ck_active = false;
  b.ck_iters = checkpoint ? opts->iters : 0;
  b.ck_mu = opts->mu;
  return st;
}

csar_status csar_af_loss(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev, const float* theta_dev,
                         const void* X_dev, double* loss_dev, void* grad_X_dev, float* grad_theta_dev,
                         void* stream) {
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (plan->rda) return fail(CSAR_E_UNSUPPORTED, "autofocus uses the chirp-scaling operator pair");
  if (!Y_dev || !mask_dev || !theta_dev || !X_dev || !loss_dev)
    return fail(CSAR_E_INVALID, "null data pointer");
  DeviceGuard dg(plan->dev);
  if (csar_status st = ensure_af(plan, 1, 0)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Buffers& b = plan->b;
  CK(launch_rotate_rows((const float2*)Y_dev, theta_dev, b.yt, plan->na, plan->nr, s));
  CK(dense_op(plan, (const float2*)X_dev, b.af_h, true, s));
  CK(launch_af_resid(b.af_h, b.yt, mask_dev, plan->na, plan->nr, b.row_loss, grad_theta_dev, loss_dev, s));
  if (grad_X_dev) {
    CK(dense_op(plan, b.af_h, b.af_h, false, s));
    CK(launch_scale(b.af_h, (float2*)grad_X_dev, -2.f, plan->n, s));
  }
  return CSAR_OK;
}

csar_status csar_af_backward(csar_plan plan, const void* Y_dev, const uint32_t* mask_dev, const float* theta_dev,
                             const void* Xbar_dev, float* theta_bar_dev, void* X0bar_dev, void* stream) {
  NvtxRange nvtx_("csar_af_backward");
  if (!plan) return fail(CSAR_E_INVALID, "plan is NULL");
  if (plan->rda) return fail(CSAR_E_UNSUPPORTED, "autofocus uses the chirp-scaling operator pair");
  if (!Y_dev || !mask_dev || !theta_dev || !Xbar_dev || !theta_bar_dev)
    return fail(CSAR_E_INVALID, "null data pointer");
  if (plan->b.ck_iters <= 0)
    return fail(CSAR_E_INVALID, "no checkpointed csar_af_solve on this plan");
  DeviceGuard dg(plan->dev);
  cudaStream_t s = (cudaStream_t)stream;
  Buffers& b = plan->b;
  const size_t n = (size_t)plan->n;
  const float mu = b.ck_mu;
  CK(launch_rotate_rows((const float2*)Y_dev, theta_dev, b.yt, plan->na, plan->nr, s));
  CK(cudaMemcpyAsync(b.af_xbar, Xbar_dev, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  for (int i = b.ck_iters - 1; i >= 0; --i) {
    CK(cudaMemsetAsync(b.af_bbar, 0, n * sizeof(float2), s));
    CK(launch_af_tvjp(b.ck_idx + (size_t)i * b.ck_cap, b.ck_val + (size_t)i * b.ck_cap, b.ck_meta + i,
                      b.af_xbar, b.af_bbar, b.ck_cap, s));
    CK(dense_op(plan, b.af_bbar, b.af_h, true, s));                       // G(bbar)
    CK(launch_af_mask_theta(b.af_h, b.yt, mask_dev, plan->na, plan->nr, mu, theta_bar_dev, s));
    CK(dense_op(plan, b.af_h, b.af_h, false, s));                         // M(S.G(bbar))
    CK(launch_af_axpy(b.af_bbar, b.af_h, mu, b.af_xbar, plan->n, s));
  }
  if (X0bar_dev) CK(cudaMemcpyAsync(X0bar_dev, b.af_xbar, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  return CSAR_OK;
}

// ---------------------------------------------------------------- batches
csar_status csar_batch_destroy(csar_batch b);

namespace {

// Work tables of the one-launch-per-pass batch: every patch's row blocks (8192 values
// each) and tile groups (one cluster each), patch by patch.
csar_status batch_build_tables(csar_batch b) {
  std::vector<BatchItem> ri, ci;
  for (int i = 0; i < (int)b->plans.size(); ++i) {
    const csar_plan p = b->plans[i];
    const int blocks = p->na / row_w(p->nr);
    for (int k = 0; k < blocks; ++k) ri.push_back(BatchItem{i, k, p->nr, 0});
    const int per = batch_col_tiles_per_item(p->na);
    const int units = (p->n_tiles + per - 1) / per;
    for (int u = 0; u < units; ++u) ci.push_back(BatchItem{i, u, p->na, 0});
  }
  const size_t np = b->plans.size();
  CK(dalloc(&b->d_row_items, ri.size()));
  CK(dalloc(&b->d_col_items, ci.size()));
  CK(cudaMemcpy(b->d_row_items, ri.data(), ri.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->d_col_items, ci.data(), ci.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  b->n_row_items = (int)ri.size();
  b->n_col_items = (int)ci.size();
  CK(dalloc(&b->d_r1, np));
  CK(dalloc(&b->d_r2, np));
  for (int par = 0; par < 2; ++par) {
    for (int k = 0; k < 4; ++k) CK(dalloc(&b->d_c[par][k], np));
    CK(dalloc(&b->d_sel[par], np));
  }
  CK(row_batched_set_attributes());
  CK(col_batched_set_attributes());
  return CSAR_OK;
}

// The patches' pass arguments for this solve (buffers, step, threshold, K_p), as the
// per-patch iteration forms them, into the batch's device arrays.
csar_status batch_upload_args(csar_batch b, const int64_t* K, const csar_opts& o) {
  const int np = (int)b->plans.size();
  std::vector<RowArgs> r1(np), r2(np);
  std::vector<ColArgs> c[2][4];
  std::vector<SelArgs> sa[2];
  for (int par = 0; par < 2; ++par) {
    for (int k = 0; k < 4; ++k) c[par][k].resize(np);
    sa[par].resize(np);
  }
  for (int i = 0; i < np; ++i) {
    const csar_plan p = b->plans[i];
    const Buffers& bb = p->b;
    r1[i] = row_args(p, bb.z, p->coef_g);
    r2[i] = row_args(p, bb.z, p->coef_m);
    r2[i].yf = bb.yf;
    r2[i].partial = bb.partial;
    r2[i].ctl = bb.ctl;
    r2[i].resid_scale = 1.0f / (float)p->na;
    csar_opts oi = o;
    oi.K = K[i];
    for (int par = 0; par < 2; ++par) {
      ColArgs a = col_args(p);
      a.xs_off = bb.off[par];
      a.xs_idx = bb.idx[par];
      a.xs_val = bb.val[par];
      a.out = bb.z;
      c[par][0][i] = a;
      a.in = bb.z;
      a.mask = bb.mask_t;
      c[par][1][i] = a;
      a.gate_val = kRepassCut;
      c[par][2][i] = a;
      a.gate_val = kRepassCut2;
      c[par][3][i] = a;
      sa[par][i] = sel_args(p, par, oi);
    }
  }
  CK(cudaMemcpy(b->d_r1, r1.data(), np * sizeof(RowArgs), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->d_r2, r2.data(), np * sizeof(RowArgs), cudaMemcpyHostToDevice));
  for (int par = 0; par < 2; ++par) {
    for (int k = 0; k < 4; ++k)
      CK(cudaMemcpy(b->d_c[par][k], c[par][k].data(), np * sizeof(ColArgs), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_sel[par], sa[par].data(), np * sizeof(SelArgs), cudaMemcpyHostToDevice));
  }
  return CSAR_OK;
}

// One ITA iteration of every patch (fixed step), reading list `par` of each: one launch
// per pass and per selection kernel, whatever the number of patches.  The re-passes and
// the two selection paths are decided per patch on the device (early exits), as in the
// per-patch iteration outside a graph.
cudaError_t enqueue_batched_iteration(csar_batch b, int par, cudaStream_t s) {
  const int np = (int)b->plans.size();
  const BatchItem* ci = b->d_col_items;
  const int nci = b->n_col_items;
  LK(launch_col_batched(COL_SPARSE_FWD, b->d_c[par][0], ci, nci, s));   // C1: F_a X
  LK(launch_row_batched(false, b->d_r1, b->d_row_items, b->n_row_items, s));   // R1
  LK(launch_col_batched(COL_RESID, b->d_c[par][1], ci, nci, s));        // C2: F_a(S.G X)
  LK(launch_row_batched(true, b->d_r2, b->d_row_items, b->n_row_items, s));    // R2: M(r)
  LK(launch_col_batched(COL_SELECT, b->d_c[par][1], ci, nci, s));       // C3: Delta X, histogram
  const SelArgs* sa = b->d_sel[par];
  LK(launch_sel_batched(SelKernel::kCheck, sa, np, 0, s));
  LK(launch_col_batched(COL_REPASS, b->d_c[par][2], ci, nci, s));
  LK(launch_sel_batched(SelKernel::kCheck2, sa, np, 0, s));
  LK(launch_col_batched(COL_REPASS, b->d_c[par][3], ci, nci, s));
  LK(launch_sel_batched(SelKernel::kFused, sa, np, 0, s));
  for (int lev = 0; lev < 3; ++lev) {
    LK(launch_sel_batched(SelKernel::kRound, sa, np, lev, s));
    LK(launch_sel_batched(SelKernel::kPick, sa, np, lev, s));
  }
  LK(launch_sel_batched(SelKernel::kCount, sa, np, 0, s));
  LK(launch_sel_batched(SelKernel::kScan, sa, np, 0, s));
  LK(launch_sel_batched(SelKernel::kScatter, sa, np, 0, s));
  return launch_sel_batched(SelKernel::kFinish, sa, np, 0, s);
}

}  // namespace

csar_status csar_batch_create(const csar_params* params, int32_t n_patches, uint32_t flags, csar_batch* out) {
  if (!out) return fail(CSAR_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!params || n_patches <= 0) return fail(CSAR_E_INVALID, "need n_patches > 0 parameter sets");
  if (flags & CSAR_PLAN_RDA) return fail(CSAR_E_UNSUPPORTED, "batches use the chirp-scaling operator pair");
  // every patch a batch member (the sizes the batched kernels serve, no column flags):
  // one launch per pass
  bool single = !(flags & (0xff00u | CSAR_PLAN_COL_HALF_TILE | CSAR_PLAN_COL_WIDE_TILE | CSAR_PLAN_COL_PERSIST |
                           CSAR_PLAN_COL_NO_PERSIST | CSAR_PLAN_BATCH_MEMBER));
  for (int i = 0; single && i < n_patches; ++i) single = batch_member_ok(params[i].n_az, params[i].n_rg);
  const uint32_t pflags = single ? (flags | CSAR_PLAN_BATCH_MEMBER) : flags;
  csar_batch b = new csar_batch_s();
  CK(cudaGetDevice(&b->dev));
  for (int i = 0; i < n_patches; ++i) {
    csar_plan p = nullptr;
    if (csar_status st = csar_plan_create(&params[i], pflags, &p)) {
      csar_batch_destroy(b);
      return st;
    }
    b->plans.push_back(p);
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      csar_batch_destroy(b);
      return cuda_fail(ce, "csar_batch_create");
    }
    b->streams.push_back(s);
    b->join.push_back(e);
  }
  cudaError_t ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    csar_batch_destroy(b);
    return cuda_fail(ce, "csar_batch_create");
  }
  if (single) {
    if (csar_status st = batch_build_tables(b)) {
      csar_batch_destroy(b);
      return st;
    }
    b->single = true;
  }
  *out = b;
  return CSAR_OK;
}

csar_status csar_batch_destroy(csar_batch b) {
  if (!b) return CSAR_OK;
  DeviceGuard dg(b->dev);
  cudaDeviceSynchronize();
  for (int i = 0; i < 2; ++i)
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_row_items);
  cudaFree(b->d_col_items);
  cudaFree(b->d_r1);
  cudaFree(b->d_r2);
  for (int par = 0; par < 2; ++par) {
    for (int k = 0; k < 4; ++k) cudaFree(b->d_c[par][k]);
    cudaFree(b->d_sel[par]);
  }
  for (auto p : b->plans) csar_plan_destroy(p);
  delete b;
  return CSAR_OK;
}

csar_status csar_solve_batched(csar_batch b, const void* const* Y_dev, const uint32_t* const* mask_dev,
                               void* const* X_dev, const int64_t* K, const csar_opts* opts, void* stream) {
  NvtxRange nvtx_("csar_solve_batched");
  if (!b) return fail(CSAR_E_INVALID, "batch is NULL");
  if (!Y_dev || !mask_dev || !X_dev || !K || !opts) return fail(CSAR_E_INVALID, "null argument");
  const int np = (int)b->plans.size();
  DeviceGuard dg(b->dev);
  cudaStream_t s = (cudaStream_t)stream;
  csar_opts o = *opts;
  for (int i = 0; i < np; ++i) {
    o.K = K[i];
    if (csar_status st = check_opts(b->plans[i], &o, true)) return st;
    if (!Y_dev[i] || !mask_dev[i] || !X_dev[i]) return fail(CSAR_E_INVALID, "null data pointer (patch %d)", i);
    if (csar_status st = ensure_capacity(b->plans[i], K[i], o.iters)) return st;
  }
  // per-solve set-up of every patch
  for (int i = 0; i < np; ++i) {
    csar_plan p = b->plans[i];
    CK(prepare_inputs(p, (const float2*)Y_dev[i], mask_dev[i], s));
    CK(cudaMemsetAsync(p->b.off[0], 0, (p->n_tiles + 1) * sizeof(uint32_t), s));
    k_ctl_init<<<1, 1, 0, s>>>(p->b.ctl, 0u, p->b.off[0], p->n_tiles);
    CK(cudaGetLastError());
  }
  // one graph per parity: one launch per pass over all patches (batch members, fixed
  // step), or a fork to the patches' streams with one branch per patch and a join
  const bool single = b->single && o.mu_mode == CSAR_MU_FIXED;
  bool same = (int)b->key_y.size() == np && b->key_o.mu_mode == o.mu_mode && b->key_o.mu == o.mu &&
              b->key_o.thresh == o.thresh && (int)b->key_gen.size() == np;
  for (int i = 0; same && i < np; ++i)
    same = b->key_y[i] == Y_dev[i] && b->key_k[i] == K[i] && b->key_gen[i] == b->plans[i]->buf_gen;
  if (!same) {
    for (int par = 0; par < 2; ++par) {
      if (b->exec[par]) cudaGraphExecDestroy(b->exec[par]);
      b->exec[par] = nullptr;
    }
    if (single)
      if (csar_status st = batch_upload_args(b, K, o)) return st;
  }
  for (int par = 0; par < 2 && o.iters > 0; ++par) {
    if (b->exec[par]) continue;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, b->cap);
    if (single && e == cudaSuccess) e = enqueue_batched_iteration(b, par, b->cap);
    for (int i = 0; !single && i < np && e == cudaSuccess; ++i) {
      csar_opts oi = o;
      oi.K = K[i];
      e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
      if (e == cudaSuccess) e = enqueue_iteration(b->plans[i], (const float2*)Y_dev[i], par, oi, b->streams[i], nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(b->join[i], b->streams[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e != cudaSuccess ? e : e2, "capture of the batched iteration");
    }
    cudaError_t e3 = cudaGraphInstantiate(&b->exec[par], g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaGraphInstantiate (batch)");
  }
  b->key_y.assign(Y_dev, Y_dev + np);
  b->key_k.assign(K, K + np);
  b->key_o = o;
  b->key_gen.resize(np);
  for (int i = 0; i < np; ++i) b->key_gen[i] = b->plans[i]->buf_gen;
  int cur = 0;
  for (int it = 0; it < o.iters; ++it) {
    CK(cudaGraphLaunch(b->exec[cur], s));
    cur = 1 - cur;
  }
  for (int i = 0; i < np; ++i) {
    csar_plan p = b->plans[i];
    CK(cudaMemsetAsync(X_dev[i], 0, (size_t)p->n * sizeof(float2), s));
    CK(launch_list_to_dense(p->b.off[cur], p->b.idx[cur], p->b.val[cur], p->n_tiles, (float2*)X_dev[i], s));
  }
  return CSAR_OK;
}

csar_status csar_batch_check(csar_batch b) {
  if (!b) return fail(CSAR_E_INVALID, "batch is NULL");
  for (auto p : b->plans)
    if (csar_status st = csar_plan_check(p)) return st;
  return CSAR_OK;
}

// ---------------------------------------------------------------- autotuner
csar_status csar_autotune(const csar_params* params, int32_t iters, int32_t* chosen_cluster) {
  if (csar_status st = validate(params)) return st;
  if (iters <= 0) return fail(CSAR_E_INVALID, "iters must be > 0");
  const int na = params->n_az, nr = params->n_rg;
  const size_t n = (size_t)na * nr;
  float2* y = nullptr;
  float2* x = nullptr;
  uint32_t* m = nullptr;
  CK(dalloc(&y, n));
  CK(dalloc(&x, n));
  CK(dalloc(&m, n / 32));
  k_fill_synthetic<<<1024, 256, 0, 0>>>(y, m, (long long)n, 12345u);
  CK(cudaGetLastError());
  csar_opts o{};
  o.K = std::max<int64_t>(1, (int64_t)(0.01 * (double)n));
  o.iters = iters;
  o.mu_mode = CSAR_MU_FIXED;
  o.mu = 1.f;
  o.thresh = CSAR_THRESH_SOFT;
  // every configuration times the passes it serves (one profiled solve after a warm-up
  // solve); per tile width the fastest for the main passes (sparse-input FFT, selection)
  // and for the residue pass are combined, and the fastest width wins
  struct Trial {
    ColConf c;
    int w;
    float main_ms, res_ms;
  };
  std::vector<Trial> trials;
  for (int size = 0; size < 3; ++size) {   // half, full and wide tiles
    for (int p = 1; p <= 16; p <<= 1) {
      ColConf c;
      c.p = p;
      c.e = size == 0 ? kColCtaElems / 2 : (size == 1 ? kColCtaElems : 2 * kColCtaElems);
      if (!col_conf_ok(na, c)) continue;
      csar_plan plan = nullptr;
      const uint32_t fl = CSAR_PLAN_COL_CLUSTER(p) |
                          (size == 0 ? CSAR_PLAN_COL_HALF_TILE : (size == 2 ? CSAR_PLAN_COL_WIDE_TILE : 0u));
      if (csar_plan_create(params, fl, &plan) != CSAR_OK) continue;
      float pass[kPasses] = {};
      const bool ok = csar_solve(plan, y, m, x, &o, nullptr, nullptr) == CSAR_OK &&
                      csar_solve_profile(plan, y, m, x, &o, pass, kPasses, nullptr) == CSAR_OK;
      csar_plan_destroy(plan);
      if (ok) trials.push_back({c, col_w(na, c.p, c.e), pass[0] + pass[4] + pass[5], pass[2]});
    }
  }
  // radix schedule of the range passes (values per thread, 32 or 16 for rows of 1024
  // bins and more): the summed time of the two range passes decides
  int best_regs = 32;
  if (nr >= 1024) {
    float best_row = -1.f;
    for (int regs : {32, 16}) {
      csar_plan plan = nullptr;
      if (csar_plan_create(params, 0u, &plan) != CSAR_OK) continue;
      plan->row_regs = regs == 16 ? 16 : 0;
      float pass[kPasses] = {};
      const bool ok = csar_solve(plan, y, m, x, &o, nullptr, nullptr) == CSAR_OK &&
                      csar_solve_profile(plan, y, m, x, &o, pass, kPasses, nullptr) == CSAR_OK;
      csar_plan_destroy(plan);
      if (ok && (best_row < 0.f || pass[1] + pass[3] < best_row)) {
        best_row = pass[1] + pass[3];
        best_regs = regs;
      }
    }
  }
  cudaFree(y);
  cudaFree(x);
  cudaFree(m);
  if (trials.empty()) return fail(CSAR_E_INTERNAL, "autotune: no column configuration ran");
  ColConf best, best_res;
  float best_ms = -1.f;
  for (const Trial& a : trials) {
    for (const Trial& r : trials) {
      if (r.w != a.w) continue;
      const float t = a.main_ms + r.res_ms;
      if (best_ms < 0.f || t < best_ms) {
        best_ms = t;
        best = a.c;
        best_res = r.c;
      }
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    g_tune[{na, nr}] = {best, best_res};
    g_tune_row[{na, nr}] = best_regs;
    tune_save_locked();
  }
  if (chosen_cluster) *chosen_cluster = best.p;
  return CSAR_OK;
}

}  // extern "C"
