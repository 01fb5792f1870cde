// Path kernels instantiated for double, state dimension 1, control dimension 1.
#include "jd_kernels.cuh"

namespace jd {
extern const PathOps ops_f64_d1_u1 = make_ops<double, 1, 1>();
}  // namespace jd
