// colp_8192.cu — persistent column-pass instantiations (see colp_pass.cuh).
#include "colp_pass.cuh"

namespace csar {
CSAR_COLP_INSTANTIATE(8192, 8, 4096)
CSAR_COLP_INSTANTIATE(8192, 16, 4096)
}  // namespace csar
