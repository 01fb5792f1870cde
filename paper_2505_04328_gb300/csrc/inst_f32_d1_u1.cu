// Path kernels instantiated for float, state dimension 1, control dimension 1.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f32_d1_u1 = make_ops<float, 1, 1>();
}  // namespace jd
