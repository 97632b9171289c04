// col_8192w.cu — column-pass instantiations with CTAs of 16384 values (one per SM,
// 1024 threads): tiles of 8 (P = 4) or 16 (P = 8) columns, i.e. 64- or 128-byte row
// segments (see col_pass.cuh).
#include "col_pass.cuh"

namespace csar {
CSAR_COL_INSTANTIATE(8192, 4, 16384)
CSAR_COL_INSTANTIATE(8192, 8, 16384)
}  // namespace csar
