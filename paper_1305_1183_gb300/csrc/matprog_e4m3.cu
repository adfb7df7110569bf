// Instances of the matrix pass: row-scaled FP8-E4M3 storage.
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_e4m3() {
  reg_shapes<8, 1, 2, FMT_E4M3, true, false>();
  reg_shapes<8, 1, 2, FMT_E4M3, true, true>();
  reg_shapes<8, 1, 2, FMT_E4M3, false, false>();
  reg_sigs<8, 1, 2, FMT_E4M3, true, false>();
  reg_sigs<8, 1, 2, FMT_E4M3, true, true>();
  // packed chunks, more rows in flight
  reg_lowp_sigs<8, 1, 8, FMT_E4M3, true, false>();
  reg_lowp_sigs<8, 1, 4, FMT_E4M3, true, false>();
  // unaligned rows: GEMVER pass 1 with a low-precision output (element-interleaved loads)
  reg<8, 1, 2, 3, 1, 0, FMT_E4M3, false, false, SIG_GEMVER1>();
}
}  // namespace mp
}  // namespace kf
