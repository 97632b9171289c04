// col_4096h.cu — column-pass instantiations with 4096-value CTAs (see col_pass.cuh).
#include "col_pass.cuh"

namespace csar {
CSAR_COL_INSTANTIATE(4096, 1, 4096)
CSAR_COL_INSTANTIATE(4096, 2, 4096)
CSAR_COL_INSTANTIATE(4096, 4, 4096)
CSAR_COL_INSTANTIATE(4096, 8, 4096)
}  // namespace csar
