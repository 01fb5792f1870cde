// Path kernels instantiated for double, state dimension 8, control dimension 4.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f64_d8_u4 = make_ops<double, 8, 4>();
}  // namespace jd
