// Volume preparation: re-layout of the uint16 codes into 16^3 bricks in the
// chosen storage, the cell-brick min/max grid and the occupancy mask of the
// current transfer function (Sec. 2.1 volume data, Sec. 2.6 classification).
#include "rc_device.cuh"

namespace rc {

// One thread per element of the padded bricked array; reads the linear
// staging copy (x fastest) and converts: F32 keeps the code, F16 stores
// fp16(code / vmax) (FP32 quotient, then round-to-nearest-even), U16 keeps the
// code. Codes above vmax clamp; padding outside the volume is 0.
template <int ST>
__global__ void relayout_kernel(const uint16_t *__restrict__ stage, int nx, int ny, int nz, int vmax,
                                int nbv0, int nbv1, void *dst, long long total) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int local = (int)(e & 4095);
    long long brick = e >> 12;
    int bx = (int)(brick % nbv0);
    long long r = brick / nbv0;
    int by = (int)(r % nbv1);
    int bz = (int)(r / nbv1);
    int x = bx * 16 + (local & 15), y = by * 16 + ((local >> 4) & 15), z = bz * 16 + (local >> 8);
    int code = 0;
    if (x < nx && y < ny && z < nz) code = min((int)stage[((size_t)z * ny + y) * nx + x], vmax);
    if (ST == RC_STORE_F32) ((float *)dst)[e] = (float)code;
    else if (ST == RC_STORE_F16) ((__half *)dst)[e] = __float2half_rn(__fdiv_rn((float)code, (float)vmax));
    else ((uint16_t *)dst)[e] = (uint16_t)code;
}

cudaError_t launch_relayout(const uint16_t *stage, VolDev v, void *dst, int nbv0, int nbv1, int nbv2,
                            cudaStream_t s) {
    long long total = (long long)nbv0 * nbv1 * nbv2 * kBrickVox;
    unsigned blocks = (unsigned)((total + 255) / 256);
    switch (v.storage) {
        case RC_STORE_F32:
            relayout_kernel<RC_STORE_F32><<<blocks, 256, 0, s>>>(stage, v.n[0], v.n[1], v.n[2], v.vmax, nbv0, nbv1, dst, total);
            break;
        case RC_STORE_F16:
            relayout_kernel<RC_STORE_F16><<<blocks, 256, 0, s>>>(stage, v.n[0], v.n[1], v.n[2], v.vmax, nbv0, nbv1, dst, total);
            break;
        default:
            relayout_kernel<RC_STORE_U16><<<blocks, 256, 0, s>>>(stage, v.n[0], v.n[1], v.n[2], v.vmax, nbv0, nbv1, dst, total);
    }
    return cudaGetLastError();
}

// One block per cell-brick: min and max of the (clamped) codes over the
// footprint voxels 16b .. min(16b + 16, N - 1) per axis.
__global__ void __launch_bounds__(256) minmax_kernel(const uint16_t *__restrict__ stage, int nx, int ny,
                                                     int nz, int cb0, int cb1, int vmax, uint16_t *mn,
                                                     uint16_t *mx) {
    const int b = blockIdx.x;
    const int bx = b % cb0, by = (b / cb0) % cb1, bz = b / (cb0 * cb1);
    const int x0 = bx * 16, y0 = by * 16, z0 = bz * 16;
    const int ex = min(x0 + 16, nx - 1) - x0 + 1;
    const int ey = min(y0 + 16, ny - 1) - y0 + 1;
    const int ez = min(z0 + 16, nz - 1) - z0 + 1;
    const int cnt = ex * ey * ez;
    int lo = 65535, hi = 0;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int lx = t % ex, r = t / ex, ly = r % ey, lz = r / ey;
        int v = min((int)stage[((size_t)(z0 + lz) * ny + (y0 + ly)) * nx + (x0 + lx)], vmax);
        lo = min(lo, v);
        hi = max(hi, v);
    }
    lo = __reduce_min_sync(0xffffffffu, (unsigned)lo);
    hi = __reduce_max_sync(0xffffffffu, (unsigned)hi);
    __shared__ int s_lo[8], s_hi[8];
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
        }
        mn[b] = (uint16_t)lo;
        mx[b] = (uint16_t)hi;
    }
}

cudaError_t launch_minmax(const uint16_t *stage, const int n[3], const int cb[3], int vmax, uint16_t *mn,
                          uint16_t *mx, cudaStream_t s) {
    int nb = cb[0] * cb[1] * cb[2];
    minmax_kernel<<<nb, 256, 0, s>>>(stage, n[0], n[1], n[2], cb[0], cb[1], vmax, mn, mx);
    return cudaGetLastError();
}

// A cell-brick is occupied unless every entry lo..hi its samples can touch has
// zero opacity: raw codes u(v) = v (K-1) / vmax floored in integers; FP16
// storage u(v) = fp16(v / vmax) (K-1), exact in FP32.
__global__ void occupancy_kernel(const uint16_t *mn, const uint16_t *mx, int nbricks, int vmax, int f16_values,
                                 TFDev tf, uint8_t *occ) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbricks) return;
    const int K = tf.K;
    int lo, hi;
    if (f16_values) {
        float hmn = __half2float(__float2half_rn(__fdiv_rn((float)mn[b], (float)vmax)));
        float hmx = __half2float(__float2half_rn(__fdiv_rn((float)mx[b], (float)vmax)));
        lo = (int)floorf(hmn * (float)(K - 1));
        hi = (int)floorf(hmx * (float)(K - 1)) + 1;
    } else {
        lo = (int)(((long long)mn[b] * (K - 1)) / vmax);
        hi = (int)(((long long)mx[b] * (K - 1)) / vmax) + 1;
    }
    hi = min(hi, K - 1);
    lo = min(lo, K - 1);
    uint8_t any = 0;
    for (int i = lo; i <= hi && !any; i++) {
        float a = tf.fp16 ? half4_to_float4(tf.f16[i]).w : tf.f32[i].w;
        any = a != 0.0f;
    }
    occ[b] = any;
}

cudaError_t launch_occupancy(const uint16_t *mn, const uint16_t *mx, int nbricks, int vmax, int f16_values,
                             TFDev tf, uint8_t *occ, cudaStream_t s) {
    occupancy_kernel<<<(nbricks + 127) / 128, 128, 0, s>>>(mn, mx, nbricks, vmax, f16_values, tf, occ);
    return cudaGetLastError();
}

}  // namespace rc
