// Instances of the matrix pass: FP32 storage, direct 16-byte loads and the
// element-wise form for unaligned rows.
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_f32_plain() {
  reg_shapes<8, 2, 4, FMT_F32, false>();
  reg_shapes<8, 4, 2, FMT_F32, false>();
  reg<8, 1, 2, 1, 1, FMT_F32, false, false>();
  reg<8, 1, 2, 2, 1, FMT_F32, false, false>();
  reg<8, 1, 2, 4, 1, FMT_F32, false, false>();
  reg<8, 1, 2, 2, 2, FMT_F32, false, false>();
  reg<8, 1, 2, 4, 2, FMT_F32, false, false>();
}
}  // namespace mp
}  // namespace kf
