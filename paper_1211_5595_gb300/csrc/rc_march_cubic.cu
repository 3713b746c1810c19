// Forward march with cubic B-spline reconstruction: the compositing march in
// every sample form (shaded or not, 1-D or 2-D table) and the other ray
// functions.
#include "rc_march.cuh"

namespace rc {

cudaError_t launch_march_cubic(const MarchArgs &a, int nviews, cudaStream_t s) {
    if (a.p.func != RC_FUNC_COMPOSITE) return launch_function<true>(a, nviews, s);
    const int f = (a.p.shade ? kShade : 0) | (a.tf.M >= 2 ? kTF2 : 0);
    switch (f) {
        case 0: return launch_composite<kCubic>(a, nviews, s);
        case kShade: return launch_composite<kCubic | kShade>(a, nviews, s);
        case kTF2: return launch_composite<kCubic | kTF2>(a, nviews, s);
        default: return launch_composite<kCubic | kTF2 | kShade>(a, nviews, s);
    }
}

}  // namespace rc
