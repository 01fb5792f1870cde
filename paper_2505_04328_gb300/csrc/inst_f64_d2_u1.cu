// Path kernels instantiated for double, state dimension 2, control dimension 1.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f64_d2_u1 = make_ops<double, 2, 1>();
}  // namespace jd
