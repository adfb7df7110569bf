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
}
}  // namespace mp
}  // namespace kf
