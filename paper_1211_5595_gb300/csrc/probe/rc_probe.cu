// Read-bandwidth probes for the rooflines of the gather kernels (declared in
// include/rc_probe.h). The loads are volatile inline PTX, so the compiler keeps
// every pass over the buffer; their sum goes to a sink that is never written
// for the probe's data.
#include <cuda_runtime.h>

#include "rc_probe.h"

namespace {

constexpr int kL1Ctas = 4, kL1Threads = 256, kL2Ctas = 8, kL2Threads = 256;
constexpr size_t kL1MaxBytes = 64 * 1024;

__device__ float g_probe_sink;

__device__ __forceinline__ float4 ld_cg(const float4 *p) {
    float4 v;
    asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ float4 ld_nc(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// The grid strides over the buffer: every 16-byte element read once per pass.
__global__ void __launch_bounds__(kL2Threads) read_l2_kernel(const float4 *__restrict__ p, long long n4, int reps) {
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; r++)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = ld_cg(p + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    if (acc == -1.0f) g_probe_sink = acc;
}

// Every CTA reads the whole (small) buffer on every pass.
__global__ void __launch_bounds__(kL1Threads) read_l1_kernel(const float4 *__restrict__ p, int n4, int reps) {
    float acc = 0.0f;
    for (int r = 0; r < reps; r++)
        for (int i = threadIdx.x; i < n4; i += blockDim.x) {
            const float4 v = ld_nc(p + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    if (acc == -1.0f) g_probe_sink = acc;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

bool valid(const void *buf, size_t bytes, int reps) {
    return buf && bytes >= 16 && bytes % 16 == 0 && (reinterpret_cast<size_t>(buf) & 15) == 0 && reps >= 1;
}

}  // namespace

extern "C" {

int rc_probe_read_l2(const void *buf, size_t bytes, int reps, void *cuda_stream) {
    if (!valid(buf, bytes, reps)) return (int)cudaErrorInvalidValue;
    const int sms = sm_count();
    if (sms < 1) return (int)cudaErrorInvalidDevice;
    read_l2_kernel<<<sms * kL2Ctas, kL2Threads, 0, (cudaStream_t)cuda_stream>>>(
        reinterpret_cast<const float4 *>(buf), (long long)(bytes / 16), reps);
    return (int)cudaGetLastError();
}

int rc_probe_read_l1(const void *buf, size_t bytes, int reps, void *cuda_stream) {
    if (!valid(buf, bytes, reps) || bytes > kL1MaxBytes) return (int)cudaErrorInvalidValue;
    const int sms = sm_count();
    if (sms < 1) return (int)cudaErrorInvalidDevice;
    read_l1_kernel<<<sms * kL1Ctas, kL1Threads, 0, (cudaStream_t)cuda_stream>>>(
        reinterpret_cast<const float4 *>(buf), (int)(bytes / 16), reps);
    return (int)cudaGetLastError();
}

size_t rc_probe_l1_bytes(size_t bytes, int reps) {
    const int sms = sm_count();
    return sms < 1 ? 0 : (size_t)sms * kL1Ctas * (size_t)reps * bytes;
}

}  // extern "C"
