// Instances of the matrix pass: FP32 storage, direct 16-byte loads.
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_f32_plain() {
  reg_shapes<8, 1, 4, FMT_F32, true, false>();
  reg_shapes<8, 2, 2, FMT_F32, true, false>();
  reg_shapes<4, 1, 4, FMT_F32, true, false>();
}
}  // namespace mp
}  // namespace kf
