// Read-bandwidth probe for the roofline of the gather kernels: one launch
// reads a device buffer `reps` times with 16-byte loads that bypass L1
// (ld.global.cg), so a buffer smaller than L2 measures the L2 read rate.
#include "rc_internal.h"

namespace rc {

__global__ void __launch_bounds__(256) read_probe_kernel(const float4 *__restrict__ p, long long n4, int reps,
                                                         float *sink) {
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; r++)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(p + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    if (acc == -1.0f) *sink = acc;   // never true for the probe's data; keeps the loads
}

cudaError_t launch_read_probe(const void *buf, size_t bytes, int reps, float *sink, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    read_probe_kernel<<<sms * 8, 256, 0, s>>>(reinterpret_cast<const float4 *>(buf), (long long)(bytes / 16), reps,
                                              sink);
    return cudaGetLastError();
}

}  // namespace rc
