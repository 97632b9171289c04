// col_dispatch.cu — run-time selection of the column-pass instantiation (N_a, P).
//
// P (CTAs per cluster) trades DSMEM exchange against the width of the row segments
// each CTA reads: W = 8192 P / N_a columns (P = 4: 32 B, 8: 64 B, 16: 128 B at
// N_a = 8192).  The default per N_a comes from measurements on GB300; the
// environment variable CSAR_COL_CLUSTER overrides it when the pair is instantiated.
#include <cstdlib>

#include "internal.h"

namespace csar {

cudaError_t col_attrs_8192_1();
cudaError_t col_launch_8192_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_8192_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_8192_2();
cudaError_t col_launch_8192_2(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_8192_2(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_8192_4();
cudaError_t col_launch_8192_4(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_8192_4(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_8192_8();
cudaError_t col_launch_8192_8(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_8192_8(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_8192_16();
cudaError_t col_launch_8192_16(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_8192_16(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_4096_1();
cudaError_t col_launch_4096_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_4096_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_4096_2();
cudaError_t col_launch_4096_2(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_4096_2(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_4096_4();
cudaError_t col_launch_4096_4(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_4096_4(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_4096_8();
cudaError_t col_launch_4096_8(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_4096_8(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_2048_1();
cudaError_t col_launch_2048_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_2048_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_2048_2();
cudaError_t col_launch_2048_2(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_2048_2(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_2048_4();
cudaError_t col_launch_2048_4(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_2048_4(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_1024_1();
cudaError_t col_launch_1024_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_1024_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_512_1();
cudaError_t col_launch_512_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_512_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_256_1();
cudaError_t col_launch_256_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_256_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_128_1();
cudaError_t col_launch_128_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_128_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_64_1();
cudaError_t col_launch_64_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_64_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_32_1();
cudaError_t col_launch_32_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_32_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);
cudaError_t col_attrs_16_1();
cudaError_t col_launch_16_1(ColMode m, const ColArgs& a, int nt, cudaStream_t s);
cudaError_t col_mask_16_1(int nr, const uint32_t* mk, uint32_t* mt, cudaStream_t s);

bool col_cluster_ok(int na, int p) {
  switch (na * 100 + p) {
    case 819201:
    case 819202:
    case 819204:
    case 819208:
    case 819216:
    case 409601:
    case 409602:
    case 409604:
    case 409608:
    case 204801:
    case 204802:
    case 204804:
    case 102401:
    case 51201:
    case 25601:
    case 12801:
    case 6401:
    case 3201:
    case 1601:
      return true;
    default:
      return false;
  }
}

int col_cluster_default(int na) {
  int p = na == 8192 ? 4 : (na == 4096 ? 2 : 1);
  if (const char* e = std::getenv("CSAR_COL_CLUSTER")) {
    const int q = std::atoi(e);
    if (col_cluster_ok(na, q)) p = q;
  }
  return p;
}

cudaError_t col_set_attributes(int na, int p) {
  switch (na * 100 + p) {
    case 819201: return col_attrs_8192_1();
    case 819202: return col_attrs_8192_2();
    case 819204: return col_attrs_8192_4();
    case 819208: return col_attrs_8192_8();
    case 819216: return col_attrs_8192_16();
    case 409601: return col_attrs_4096_1();
    case 409602: return col_attrs_4096_2();
    case 409604: return col_attrs_4096_4();
    case 409608: return col_attrs_4096_8();
    case 204801: return col_attrs_2048_1();
    case 204802: return col_attrs_2048_2();
    case 204804: return col_attrs_2048_4();
    case 102401: return col_attrs_1024_1();
    case 51201: return col_attrs_512_1();
    case 25601: return col_attrs_256_1();
    case 12801: return col_attrs_128_1();
    case 6401: return col_attrs_64_1();
    case 3201: return col_attrs_32_1();
    case 1601: return col_attrs_16_1();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col(int na, int p, ColMode mode, const ColArgs& a, int n_tiles, cudaStream_t s) {
  switch (na * 100 + p) {
    case 819201: return col_launch_8192_1(mode, a, n_tiles, s);
    case 819202: return col_launch_8192_2(mode, a, n_tiles, s);
    case 819204: return col_launch_8192_4(mode, a, n_tiles, s);
    case 819208: return col_launch_8192_8(mode, a, n_tiles, s);
    case 819216: return col_launch_8192_16(mode, a, n_tiles, s);
    case 409601: return col_launch_4096_1(mode, a, n_tiles, s);
    case 409602: return col_launch_4096_2(mode, a, n_tiles, s);
    case 409604: return col_launch_4096_4(mode, a, n_tiles, s);
    case 409608: return col_launch_4096_8(mode, a, n_tiles, s);
    case 204801: return col_launch_2048_1(mode, a, n_tiles, s);
    case 204802: return col_launch_2048_2(mode, a, n_tiles, s);
    case 204804: return col_launch_2048_4(mode, a, n_tiles, s);
    case 102401: return col_launch_1024_1(mode, a, n_tiles, s);
    case 51201: return col_launch_512_1(mode, a, n_tiles, s);
    case 25601: return col_launch_256_1(mode, a, n_tiles, s);
    case 12801: return col_launch_128_1(mode, a, n_tiles, s);
    case 6401: return col_launch_64_1(mode, a, n_tiles, s);
    case 3201: return col_launch_32_1(mode, a, n_tiles, s);
    case 1601: return col_launch_16_1(mode, a, n_tiles, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mask_transpose(int na, int p, int nr, const uint32_t* mask, uint32_t* mask_t,
                                  cudaStream_t s) {
  switch (na * 100 + p) {
    case 819201: return col_mask_8192_1(nr, mask, mask_t, s);
    case 819202: return col_mask_8192_2(nr, mask, mask_t, s);
    case 819204: return col_mask_8192_4(nr, mask, mask_t, s);
    case 819208: return col_mask_8192_8(nr, mask, mask_t, s);
    case 819216: return col_mask_8192_16(nr, mask, mask_t, s);
    case 409601: return col_mask_4096_1(nr, mask, mask_t, s);
    case 409602: return col_mask_4096_2(nr, mask, mask_t, s);
    case 409604: return col_mask_4096_4(nr, mask, mask_t, s);
    case 409608: return col_mask_4096_8(nr, mask, mask_t, s);
    case 204801: return col_mask_2048_1(nr, mask, mask_t, s);
    case 204802: return col_mask_2048_2(nr, mask, mask_t, s);
    case 204804: return col_mask_2048_4(nr, mask, mask_t, s);
    case 102401: return col_mask_1024_1(nr, mask, mask_t, s);
    case 51201: return col_mask_512_1(nr, mask, mask_t, s);
    case 25601: return col_mask_256_1(nr, mask, mask_t, s);
    case 12801: return col_mask_128_1(nr, mask, mask_t, s);
    case 6401: return col_mask_64_1(nr, mask, mask_t, s);
    case 3201: return col_mask_32_1(nr, mask, mask_t, s);
    case 1601: return col_mask_16_1(nr, mask, mask_t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace csar
