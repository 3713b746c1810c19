// Forward march with the 2-D (value x gradient magnitude) table and trilinear
// reconstruction, shaded or not.
#include "rc_march.cuh"

namespace rc {

cudaError_t launch_march_tf2(const MarchArgs &a, int nviews, cudaStream_t s) {
    return a.p.shade ? launch_composite<kTF2 | kShade>(a, nviews, s) : launch_composite<kTF2>(a, nviews, s);
}

}  // namespace rc
