// Instances of the matrix pass: row-scaled BF16 storage.
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_bf16() {
  reg_shapes<8, 2, 2, FMT_BF16, true, false>();
  reg_shapes<8, 2, 2, FMT_BF16, true, true>();
  reg_shapes<8, 1, 2, FMT_BF16, false, false>();
  reg_sigs<8, 2, 2, FMT_BF16, true, false>();
  reg_sigs<8, 2, 2, FMT_BF16, true, true>();
  // packed chunks, more rows in flight
  reg_lowp_sigs<8, 1, 8, FMT_BF16, true, false>();
  reg_lowp_sigs<8, 1, 4, FMT_BF16, true, false>();
  reg_lowp_sigs<8, 2, 4, FMT_BF16, true, false>();
  // unaligned rows: GEMVER pass 1 with a low-precision output (element-interleaved loads)
  reg<8, 1, 2, 3, 1, 0, FMT_BF16, false, false, SIG_GEMVER1>();
}
}  // namespace mp
}  // namespace kf
