// col_dispatch.cu — run-time selection of the column-pass instantiation (N_a, P, E).
//
// P (CTAs per cluster) and E (complex64 values per CTA) set the tile width
// W = E P / N_a columns (row segments of 8 W bytes) and the CTAs per SM (two for
// E = 8192, four for E = 4096).  The default per N_a comes from measurements on GB300;
// the environment variables CSAR_COL_CLUSTER and CSAR_COL_ELEMS override it when the
// configuration is instantiated.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "internal.h"

namespace csar {

// Every instantiated configuration (N, P, E), and every (N, P) of the column-order mask.
#define CSAR_COL_CONFIGS(X)                                                                   \
  X(8192, 1, 8192) X(8192, 2, 8192) X(8192, 4, 8192) X(8192, 8, 8192) X(8192, 16, 8192)       \
  X(8192, 2, 4096) X(8192, 4, 4096) X(8192, 8, 4096) X(8192, 16, 4096)                         \
  X(8192, 4, 16384) X(8192, 8, 16384)                                                          \
  X(4096, 1, 8192) X(4096, 2, 8192) X(4096, 4, 8192) X(4096, 8, 8192)                          \
  X(4096, 1, 4096) X(4096, 2, 4096) X(4096, 4, 4096) X(4096, 8, 4096)                          \
  X(2048, 1, 8192) X(2048, 2, 8192) X(2048, 4, 8192)                                           \
  X(2048, 1, 4096) X(2048, 2, 4096) X(2048, 4, 4096)                                           \
  X(1024, 1, 8192) X(1024, 1, 4096) X(512, 1, 8192) X(512, 1, 4096) X(256, 1, 8192) X(128, 1, 8192)            \
  X(64, 1, 8192) X(32, 1, 8192) X(16, 1, 8192)
#define CSAR_MASK_CONFIGS(X)                                                                  \
  X(8192, 1) X(8192, 2) X(8192, 4) X(8192, 8) X(8192, 16) X(4096, 1) X(4096, 2) X(4096, 4)     \
  X(4096, 8) X(2048, 1) X(2048, 2) X(2048, 4) X(1024, 1) X(512, 1) X(256, 1) X(128, 1)         \
  X(64, 1) X(32, 1) X(16, 1)

#define CSAR_DECL(N, P, E)                                                                    \
  cudaError_t col_attrs_##N##_##P##_##E();                                                   \
  cudaError_t col_launch_##N##_##P##_##E(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
CSAR_COL_CONFIGS(CSAR_DECL)
#undef CSAR_DECL
#define CSAR_DECL(N, P) \
  cudaError_t col_mask_##N##_##P(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
CSAR_MASK_CONFIGS(CSAR_DECL)
#undef CSAR_DECL

// Persistent, tensor-copy-fed instantiations (colp_pass.cuh); each is also a k_col
// configuration, which serves the modes the persistent kernel does not cover.
#define CSAR_COLP_CONFIGS(X) \
  X(8192, 8, 4096) X(8192, 16, 4096) X(4096, 4, 4096) X(2048, 2, 4096) X(1024, 1, 4096)
#define CSAR_DECL(N, P, E)                                                                      \
  cudaError_t colp_attrs_##N##_##P##_##E();                                                    \
  cudaError_t colp_launch_##N##_##P##_##E(ColMode m, const CUtensorMap& map, const ColArgs& a, int nt, \
                                          cudaStream_t s);                                     \
  void colp_box_##N##_##P##_##E(int* c, int* r);
CSAR_COLP_CONFIGS(CSAR_DECL)
#undef CSAR_DECL

static constexpr long long conf_key(int n, int p, int e) { return (long long)n * 100000 + p * 10000 + e; }

static bool colp_conf_ok(int na, ColConf c) {
  switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) case conf_key(N, P, E):
    CSAR_COLP_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
      return true;
    default:
      return false;
  }
}

bool col_conf_ok(int na, ColConf c) {
  if (c.persist && !colp_conf_ok(na, c)) return false;
  switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) case conf_key(N, P, E):
    CSAR_COL_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
      return true;
    default:
      return false;
  }
}

static ColConf env_override(int na, ColConf c) {
  ColConf f = c;
  if (const char* s = std::getenv("CSAR_COL_CLUSTER")) f.p = std::atoi(s);
  if (const char* s = std::getenv("CSAR_COL_ELEMS")) f.e = std::atoi(s);
  if (const char* s = std::getenv("CSAR_COL_PERSIST")) f.persist = std::atoi(s) != 0;
  return col_conf_ok(na, f) ? f : c;
}

// Measured on GB300 (8192^2 spaceborne ITA): the selection and sparse-input passes are
// fastest with clusters of 4 full-size CTAs, the residue pass (two transforms per CTA)
// with clusters of 8 half-size CTAs (four per SM); both give tiles of 4 columns.
ColConf col_conf_default(int na) {
  ColConf c;
  c.p = na == 8192 ? 4 : (na == 4096 ? 2 : 1);
  c.e = kColCtaElems;
  return env_override(na, c);
}

ColConf col_conf_default_res(int na) {
  ColConf c;
  c.p = na == 8192 ? 8 : (na == 4096 ? 4 : (na == 2048 ? 2 : 1));
  c.e = na >= 2048 ? kColCtaElems / 2 : kColCtaElems;
  if (!col_conf_ok(na, c)) c = col_conf_default(na);
  return env_override(na, c);
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to the driver
// library).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of an [na][nr] complex64 array (8-byte elements) with boxes of
// box_cols x box_rows; the base must be 16-byte aligned.  swizzle128: the box's rows of
// 128 bytes are stored in shared memory with their 16-byte chunks XOR-permuted by the
// row index mod 8 (box_cols must then be 16).
cudaError_t encode_map(CUtensorMap* map, const void* base, int na, int nr, int box_cols, int box_rows,
                       bool swizzle128) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn || ((uintptr_t)base & 15u)) return cudaErrorInvalidValue;
  const cuuint64_t dim[2] = {(cuuint64_t)nr, (cuuint64_t)na};
  const cuuint64_t stride[1] = {(cuuint64_t)nr * 8u};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  static const int promo = [] {
    const char* s = std::getenv("CSAR_TMA_L2_PROMOTION");
    return s ? std::atoi(s) : 0;
  }();
  const CUtensorMapL2promotion l2 = promo >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                                    : promo >= 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                    : promo >= 64  ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
                                                   : CU_TENSOR_MAP_L2_PROMOTION_NONE;
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dim, stride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, l2,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static bool colp_mode(ColMode m) { return m == COL_FWD || m == COL_INV || m == COL_RESID || m == COL_SELECT; }

static cudaError_t launch_colp(int na, ColConf c, ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s) {
  int bc = 0, br = 0;
  switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) \
  case conf_key(N, P, E): colp_box_##N##_##P##_##E(&bc, &br); break;
    CSAR_COLP_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
  CUtensorMap map;
  if (cudaError_t e = encode_map(&map, a.in, na, a.nr, bc, br, false)) return e;
  switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) \
  case conf_key(N, P, E): return colp_launch_##N##_##P##_##E(mode, map, a, n_tiles, s);
    CSAR_COLP_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

ColConf col_conf_persist(int na) {
  ColConf c;
  c.p = na >= 1024 ? na / 1024 : 1;
  c.e = kColCtaElems / 2;
  c.persist = true;
  return c;
}

cudaError_t col_set_attributes(int na, ColConf c) {
  if (c.persist) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) \
  case conf_key(N, P, E): e = colp_attrs_##N##_##P##_##E(); break;
      CSAR_COLP_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
      default: break;
    }
    if (e != cudaSuccess) return e;
  }
  switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) \
  case conf_key(N, P, E): return col_attrs_##N##_##P##_##E();
    CSAR_COL_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col(int na, ColConf c, ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s) {
  if (c.persist && colp_mode(mode) && ((uintptr_t)a.in & 15u) == 0) return launch_colp(na, c, mode, a, n_tiles, s);
  switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) \
  case conf_key(N, P, E): return col_launch_##N##_##P##_##E(mode, a, n_tiles, s);
    CSAR_COL_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mask_transpose(int na, int p, int nr, const uint32_t* mask, uint32_t* mask_t,
                                  cudaStream_t s) {
  switch (conf_key(na, p, 0)) {
#define CSAR_CASE(N, P) \
  case conf_key(N, P, 0): return col_mask_##N##_##P(nr, mask, mask_t, s);
    CSAR_MASK_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace csar
