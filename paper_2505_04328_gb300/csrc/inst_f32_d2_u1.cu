// Path kernels instantiated for float, state dimension 2, control dimension 1.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f32_d2_u1 = make_ops<float, 2, 1>();
}  // namespace jd
