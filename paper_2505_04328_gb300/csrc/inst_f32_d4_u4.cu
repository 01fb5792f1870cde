// Path kernels instantiated for float, state dimension 4, control dimension 4.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f32_d4_u4 = make_ops<float, 4, 4>();
}  // namespace jd
