// col_small.cu — column-pass instantiations (see col_pass.cuh).
#include "col_pass.cuh"

namespace csar {
CSAR_COL_INSTANTIATE(1024, 1)
CSAR_COL_INSTANTIATE(512, 1)
CSAR_COL_INSTANTIATE(256, 1)
CSAR_COL_INSTANTIATE(128, 1)
CSAR_COL_INSTANTIATE(64, 1)
CSAR_COL_INSTANTIATE(32, 1)
CSAR_COL_INSTANTIATE(16, 1)
}  // namespace csar
