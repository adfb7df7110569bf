// Instances of the matrix pass: row-scaled BF16 and FP8-E4M3 storage.
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_lowp() {
  reg_shapes<8, 2, 2, FMT_BF16, true>();
  reg_shapes<8, 1, 2, FMT_BF16, true>();
  reg_shapes<8, 1, 2, FMT_E4M3, true>();
  reg_shapes<8, 1, 4, FMT_E4M3, true>();
  reg<8, 1, 2, 1, 1, FMT_BF16, false, false>();
  reg<8, 1, 2, 2, 1, FMT_BF16, false, false>();
  reg<8, 1, 2, 4, 1, FMT_BF16, false, false>();
  reg<8, 1, 2, 1, 1, FMT_E4M3, false, false>();
  reg<8, 1, 2, 2, 1, FMT_E4M3, false, false>();
  reg<8, 1, 2, 4, 1, FMT_E4M3, false, false>();
}
}  // namespace mp
}  // namespace kf
