// col_dispatch.cu — run-time selection of the column-pass instantiation (N_a, P, E).
//
// P (CTAs per cluster) and E (complex64 values per CTA) set the tile width
// W = E P / N_a columns (row segments of 8 W bytes) and the CTAs per SM (two for
// E = 8192, four for E = 4096).  The default per N_a comes from measurements on GB300;
// the environment variables CSAR_COL_CLUSTER and CSAR_COL_ELEMS override it when the
// configuration is instantiated.
#include <cstdlib>

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
  X(1024, 1, 8192) X(1024, 1, 4096) X(512, 1, 8192) X(256, 1, 8192) X(128, 1, 8192)            \
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

static constexpr long long conf_key(int n, int p, int e) { return (long long)n * 100000 + p * 10000 + e; }

bool col_conf_ok(int na, ColConf c) {
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

cudaError_t col_set_attributes(int na, ColConf c) {
  switch (conf_key(na, c.p, c.e)) {
#define CSAR_CASE(N, P, E) \
  case conf_key(N, P, E): return col_attrs_##N##_##P##_##E();
    CSAR_COL_CONFIGS(CSAR_CASE)
#undef CSAR_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col(int na, ColConf c, ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s) {
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
