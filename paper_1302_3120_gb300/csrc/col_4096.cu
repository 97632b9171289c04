// col_4096.cu — column-pass instantiations (see col_pass.cuh).
#include "col_pass.cuh"

namespace csar {
CSAR_COL_INSTANTIATE(4096, 1)
CSAR_COL_INSTANTIATE(4096, 2)
CSAR_COL_INSTANTIATE(4096, 4)
CSAR_COL_INSTANTIATE(4096, 8)
}  // namespace csar
