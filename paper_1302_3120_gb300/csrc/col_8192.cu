// col_8192.cu — column-pass instantiations (see col_pass.cuh).
#include "col_pass.cuh"

namespace csar {
CSAR_COL_INSTANTIATE(8192, 1)
CSAR_COL_INSTANTIATE(8192, 2)
CSAR_COL_INSTANTIATE(8192, 4)
CSAR_COL_INSTANTIATE(8192, 8)
CSAR_COL_INSTANTIATE(8192, 16)
}  // namespace csar
