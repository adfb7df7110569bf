// Instances of the matrix pass: FP32 storage, element-wise loads (unaligned rows).
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_f32_elem() {
  reg_shapes<8, 1, 2, FMT_F32, false, false>();
}
}  // namespace mp
}  // namespace kf
