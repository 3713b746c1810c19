// Forward march, trilinear reconstruction with the 1-D table: the kernel
// instances of the plain and shaded compositing march and of the other ray
// functions, and the dispatch over every form.
#include "rc_march.cuh"

namespace rc {

// a.cam gives the image size of every view; with a.cams, grid.z = nviews.
cudaError_t launch_march(const MarchArgs &a, int nviews, cudaStream_t s) {
    if (a.p.filter == RC_FILTER_BSPLINE) return launch_march_cubic(a, nviews, s);
    if (a.p.func != RC_FUNC_COMPOSITE) return launch_function<false>(a, nviews, s);
    if (a.tf.M >= 2) return launch_march_tf2(a, nviews, s);
    return a.p.shade ? launch_composite<kShade>(a, nviews, s) : launch_composite<0>(a, nviews, s);
}

}  // namespace rc
