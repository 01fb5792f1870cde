// Path kernels instantiated for double, state dimension 4, control dimension 4.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f64_d4_u4 = make_ops<double, 4, 4>();
}  // namespace jd
