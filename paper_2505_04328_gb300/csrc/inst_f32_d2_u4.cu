// Path kernels instantiated for float, state dimension 2, control dimension 4.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f32_d2_u4 = make_ops<float, 2, 4>();
}  // namespace jd
