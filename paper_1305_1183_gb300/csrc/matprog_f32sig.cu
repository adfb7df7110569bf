// Instances of the matrix pass: FP32 storage, op signatures of the named
// sequences specialised at compile time (direct loads and staged).
#include "matprog_impl.cuh"

namespace kf {
namespace mp {
void register_f32_sigs() {
  reg_sigs<8, 2, 2, FMT_F32, true, false>();
  reg_sigs<8, 1, 4, FMT_F32, true, false>();
  reg_sigs<8, 4, 2, FMT_F32, true, false>();
  reg_sigs<8, 2, 2, FMT_F32, true, true>();
  reg_sigs<8, 2, 4, FMT_F32, true, true>();
  // eight rows in flight per warp, three blocks per SM
  reg_lowp_sigs<8, 1, 8, FMT_F32, true, false>();
  // GESUMMV with eight rows of each matrix in flight
  reg<8, 1, 8, 2, 2, 2, FMT_F32, true, false, SIG_GESUMMV>();
}
}  // namespace mp
}  // namespace kf
