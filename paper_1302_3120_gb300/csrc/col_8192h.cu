// col_8192h.cu — column-pass instantiations with 4096-value CTAs (see col_pass.cuh).
#include "col_pass.cuh"

namespace csar {
CSAR_COL_INSTANTIATE(8192, 2, 4096)
CSAR_COL_INSTANTIATE(8192, 4, 4096)
CSAR_COL_INSTANTIATE(8192, 8, 4096)
CSAR_COL_INSTANTIATE(8192, 16, 4096)
}  // namespace csar
