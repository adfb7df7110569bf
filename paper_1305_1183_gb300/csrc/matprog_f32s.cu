// Instances of the matrix pass: FP32 storage, bulk-copy staged.
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_f32_staged() {
  reg_shapes<8, 1, 4, FMT_F32, true, true>();
  reg_shapes<8, 2, 2, FMT_F32, true, true>();
  reg_shapes<4, 1, 4, FMT_F32, true, true>();
}
}  // namespace mp
}  // namespace kf
