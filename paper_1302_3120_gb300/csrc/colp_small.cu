// colp_small.cu — persistent column-pass instantiations for 1024..4096 rows (see
// colp_pass.cuh).
#include "colp_pass.cuh"

namespace csar {
CSAR_COLP_INSTANTIATE(4096, 4, 4096)
CSAR_COLP_INSTANTIATE(2048, 2, 4096)
CSAR_COLP_INSTANTIATE(1024, 1, 4096)
}  // namespace csar
