// Path kernels instantiated for float, state dimension 8, control dimension 4.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f32_d8_u4 = make_ops<float, 8, 4>();
}  // namespace jd
