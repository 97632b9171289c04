// noalloc.cu — the approximated observation G for callers that cannot allocate
// device memory.
//
// csar_G needs per-row phase coefficients and FFT twiddles in device memory; a plan
// allocates them.  Some callers cannot call cudaMalloc at all: code running where
// the allocator is owned by someone else (a host framework that hands out only its
// own buffers), or embedded/real-time callers that must not allocate after start-up.
// csar_G_noalloc keeps those tables in one file-scope
// static device array instead, so it allocates nothing: the caller passes only its
// input and output buffers.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/csar.h"
#include "internal.h"

namespace csar {
namespace {

// Largest azimuth size the static array holds (one coefficient row per azimuth bin).
constexpr int kNoAllocMaxRows = 8192;
constexpr size_t kNoAllocCoefBytes = (size_t)kNoAllocMaxRows * sizeof(RowCoef);
constexpr size_t kNoAllocBytes = kNoAllocCoefBytes + (kTwLo + kTwHi) * sizeof(float2);

// Device scratch of every GPU that loads the library (~580 KiB, held until exit).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
  bool ready = false;
  unsigned char* ptr = nullptr;   // device address of g_noalloc_scratch on this device
  bool col_done[14][5][2] = {};   // kernel attributes set for (log2 N_a, log2 P, half tile)
  bool row_done[14] = {};         // ... and for log2 N_r
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_mu;                  // one call at a time (shared host staging below)
RowCoef g_coef_g[kNoAllocMaxRows];
RowCoef g_coef_m[kNoAllocMaxRows];
float2 g_tw[kTwLo + kTwHi];

int log2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace
}  // namespace csar

using namespace csar;

extern "C" csar_status csar_G_noalloc(const csar_params* params, const void* x_dev, void* y_dev,
                                      void* stream) {
  if (csar_status st = validate_params(params)) return st;
  if (params->n_az > kNoAllocMaxRows)
    return set_error(CSAR_E_UNSUPPORTED, "csar_G_noalloc: n_az exceeds the static table (8192 rows)");
  if (!x_dev || !y_dev) return set_error(CSAR_E_INVALID, "csar_G_noalloc: null data pointer");
  const int na = params->n_az, nr = params->n_rg;
  const size_t bytes = (size_t)na * nr * sizeof(float2);
  const char* xb = (const char*)x_dev;
  const char* yb = (const char*)y_dev;
  if (xb != yb && xb < yb + bytes && yb < xb + bytes)
    return set_error(CSAR_E_INVALID, "csar_G_noalloc: input and output overlap without being identical");
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error(CSAR_E_CUDA, "csar_G_noalloc: no usable current device");
  DeviceSetup& su = g_setup[dev];
  if (!su.ready) {
    // first call on this device: the host-side address of the static array is only a
    // stand-in; the device address comes from the runtime
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return set_error(CSAR_E_CUDA, cudaGetErrorString(e));
    su.ptr = (unsigned char*)p;
    su.ready = true;
  }
  ColConf conf = col_conf_default(na);
  conf.persist = false;   // the per-tile column kernels: no tensor maps, no occupancy queries
  bool& cd = su.col_done[log2i(na)][log2i(conf.p)][conf.e == kColCtaElems ? 0 : 1];
  if (!cd) {
    if (col_set_attributes(na, conf) != cudaSuccess)
      return set_error(CSAR_E_CUDA, "csar_G_noalloc: column kernel attributes");
    cd = true;
  }
  bool& rd = su.row_done[log2i(nr)];
  if (!rd) {
    if (row_set_attributes(nr) != cudaSuccess)
      return set_error(CSAR_E_CUDA, "csar_G_noalloc: row kernel attributes");
    rd = true;
  }
  // tables: every byte the passes read is rewritten here, nothing needs clearing
  if (csar_status st = build_coefs_into(*params, g_coef_g, g_coef_m)) return st;
  build_twiddles(g_tw);
  cudaStream_t s = (cudaStream_t)stream;
  RowCoef* coef_d = reinterpret_cast<RowCoef*>(su.ptr);
  float2* tw_d = reinterpret_cast<float2*>(su.ptr + kNoAllocCoefBytes);
  cudaError_t e = cudaMemcpyAsync(coef_d, g_coef_g, (size_t)na * sizeof(RowCoef), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tw_d, g_tw, sizeof(g_tw), cudaMemcpyHostToDevice, s);
  ColArgs c{};
  c.tw = tw_d;
  c.nr = nr;
  c.in = (const float2*)x_dev;
  c.out = (float2*)y_dev;
  c.scale = 1.0f / (float)na;
  const int n_tiles = nr / col_w(na, conf.p, conf.e);
  if (e == cudaSuccess) e = launch_col(na, conf, COL_FWD, c, n_tiles, s);
  RowArgs r{};
  r.data = (float2*)y_dev;
  r.coef = coef_d;
  r.tw = tw_d;
  r.n_rows = na;
  r.scale = 1.0f / (float)nr;
  if (e == cudaSuccess) e = launch_row(nr, r, s);
  c.in = (const float2*)y_dev;
  if (e == cudaSuccess) e = launch_col(na, conf, COL_INV, c, n_tiles, s);
  if (e != cudaSuccess) return set_error(CSAR_E_CUDA, cudaGetErrorString(e));
  return CSAR_OK;
}
