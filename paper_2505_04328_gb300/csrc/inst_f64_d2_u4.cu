// Path kernels instantiated for double, state dimension 2, control dimension 4.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f64_d2_u4 = make_ops<double, 2, 4>();
}  // namespace jd
