// Feedback-control kernels, FP64 path arithmetic, padded 4x4, 10x10 and 16x16 weights.
#include "jd_feedback.cuh"

namespace jd {

extern const FbOps fb_ops_f64[3] = {fb_make_ops<double, 4, 4>(), fb_make_ops<double, 10, 10>(),
                                    fb_make_ops<double, 16, 16>()};

}  // namespace jd
