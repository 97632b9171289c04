// col_2048.cu — column-pass instantiations (see col_pass.cuh).
#include "col_pass.cuh"

namespace csar {
CSAR_COL_INSTANTIATE(2048, 1)
CSAR_COL_INSTANTIATE(2048, 2)
CSAR_COL_INSTANTIATE(2048, 4)
}  // namespace csar
