// Volume preparation: re-layout of the uint16 codes into apron bricks (19^3
// voxels per 16^3-cell brick) in the chosen storage, the cell-brick min/max
// grid and the occupancy mask of the current transfer function (Sec. 2.1
// volume data, Sec. 2.6 classification).
#include "rc_device.cuh"

namespace rc {

// One thread per element of the apron-bricked array: cell-brick (bx, by, bz)
// stores voxels 16b-1 .. 16b+17 per axis, clamped to the volume (border voxels
// replicated). Reads the linear staging copy (x fastest) and converts: F32
// keeps the code, F16 stores fp16(code / vmax) (FP32 quotient, then
// round-to-nearest-even), U16 keeps the code. Codes above vmax clamp.
template <int ST>
__global__ void relayout_kernel(const uint16_t *__restrict__ stage, int nx, int ny, int nz, int vmax, int cb0,
                                int cb1, void *dst, long long total) {
    // 32-bit indices: a volume has fewer than 2^31 stored voxels (checked
    // at creation), and the divisions by constants become multiply-shifts
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    if ((long long)e >= total) return;
    const unsigned local = e % (unsigned)kApronVox, brick = e / (unsigned)kApronVox;
    const int bx = (int)(brick % (unsigned)cb0);
    const unsigned r = brick / (unsigned)cb0;
    const int by = (int)(r % (unsigned)cb1);
    const int bz = (int)(r / (unsigned)cb1);
    const int lx = (int)(local % kApron), ly = (int)((local / kApron) % kApron), lz = (int)(local / (kApron * kApron));
    const int x = min(max(bx * kBrick + lx - 1, 0), nx - 1);
    const int y = min(max(by * kBrick + ly - 1, 0), ny - 1);
    const int z = min(max(bz * kBrick + lz - 1, 0), nz - 1);
    const int code = min((int)stage[((size_t)z * ny + y) * nx + x], vmax);
    if (ST == RC_STORE_F32) ((float *)dst)[e] = (float)code;
    else if (ST == RC_STORE_F16) ((__half *)dst)[e] = __float2half_rn(__fdiv_rn((float)code, (float)vmax));
    else ((uint16_t *)dst)[e] = (uint16_t)code;
}

cudaError_t launch_relayout(const uint16_t *stage, VolDev v, void *dst, cudaStream_t s) {
    const long long total = (long long)v.cb[0] * v.cb[1] * v.cb[2] * kApronVox;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    switch (v.storage) {
        case RC_STORE_F32:
            relayout_kernel<RC_STORE_F32><<<blocks, 256, 0, s>>>(stage, v.n[0], v.n[1], v.n[2], v.vmax, v.cb[0], v.cb[1], dst, total);
            break;
        case RC_STORE_F16:
            relayout_kernel<RC_STORE_F16><<<blocks, 256, 0, s>>>(stage, v.n[0], v.n[1], v.n[2], v.vmax, v.cb[0], v.cb[1], dst, total);
            break;
        default:
            relayout_kernel<RC_STORE_U16><<<blocks, 256, 0, s>>>(stage, v.n[0], v.n[1], v.n[2], v.vmax, v.cb[0], v.cb[1], dst, total);
    }
    return cudaGetLastError();
}

// One thread per element of the value+gradient bricks (FP32 storage): brick b
// holds voxels 16b .. 16b+16 per axis (clamped to the volume) as
// (V, V(x+1) - V(x-1), V(y+1) - V(y-1), V(z+1) - V(z-1)), neighbour
// indices clamped to the volume, codes clamped to vmax; exact in FP32.
__global__ void gradvol_kernel(const uint16_t *__restrict__ stage, int nx, int ny, int nz, int vmax, int cb0, int cb1,
                               float4 *dst, long long total) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;     // fewer than 2^31 entries
    if ((long long)e >= total) return;
    const unsigned local = e % (unsigned)kGradVox, brick = e / (unsigned)kGradVox;
    const int bx = (int)(brick % (unsigned)cb0);
    const unsigned r = brick / (unsigned)cb0;
    const int by = (int)(r % (unsigned)cb1);
    const int bz = (int)(r / (unsigned)cb1);
    const int lx = (int)(local % kGradEdge), ly = (int)((local / kGradEdge) % kGradEdge),
              lz = (int)(local / (kGradEdge * kGradEdge));
    const int x = min(bx * kBrick + lx, nx - 1), y = min(by * kBrick + ly, ny - 1), z = min(bz * kBrick + lz, nz - 1);
    auto code = [&](int xx, int yy, int zz) {
        return (float)min((int)stage[((size_t)zz * ny + yy) * nx + xx], vmax);
    };
    float4 o;
    o.x = code(x, y, z);
    o.y = code(min(x + 1, nx - 1), y, z) - code(max(x - 1, 0), y, z);
    o.z = code(x, min(y + 1, ny - 1), z) - code(x, max(y - 1, 0), z);
    o.w = code(x, y, min(z + 1, nz - 1)) - code(x, y, max(z - 1, 0));
    dst[e] = o;
}

cudaError_t launch_gradvol(const uint16_t *stage, VolDev v, float4 *dst, cudaStream_t s) {
    const long long total = (long long)v.cb[0] * v.cb[1] * v.cb[2] * kGradVox;
    gradvol_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(stage, v.n[0], v.n[1], v.n[2], v.vmax, v.cb[0],
                                                                     v.cb[1], dst, total);
    return cudaGetLastError();
}

// One thread per entry of the pair bricks: entry (lz, ly, e) of brick b is
// the apron elements e and e + 1 of row (ly, lz), copied bit for bit (so the
// pairs hold exactly the stored values of every storage type).
template <typename T>
__global__ void pairs_kernel(const T *__restrict__ apron, T *__restrict__ dst, long long total) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;     // fewer than 2^31 entries
    if ((long long)e >= total) return;
    const unsigned local = e % (unsigned)kPairVox, brick = e / (unsigned)kPairVox;
    const unsigned ex = local % kPairRow, row = local / kPairRow;     // row = lz * 19 + ly
    const T *src = apron + (size_t)brick * kApronVox + row * kApron + ex;
    dst[2 * e] = src[0];
    dst[2 * e + 1] = src[1];
}

cudaError_t launch_pairs(VolDev v, void *dst, cudaStream_t s) {
    const long long total = (long long)v.cb[0] * v.cb[1] * v.cb[2] * kPairVox;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (v.storage == RC_STORE_F32)
        pairs_kernel<float><<<blocks, 256, 0, s>>>((const float *)v.data, (float *)dst, total);
    else
        pairs_kernel<uint16_t><<<blocks, 256, 0, s>>>((const uint16_t *)v.data, (uint16_t *)dst, total);
    return cudaGetLastError();
}

// One block per cell-brick: min and max of the (clamped) codes over the
// footprint voxels max(16b - before, 0) .. min(16b + after, N - 1) per axis:
// (0, 16) for trilinear samples, (1, 17) for cubic B-spline samples.
__global__ void __launch_bounds__(256) minmax_kernel(const uint16_t *__restrict__ stage, int nx, int ny,
                                                     int nz, int cb0, int cb1, int vmax, int before, int after,
                                                     uint16_t *mn, uint16_t *mx) {
    const int b = blockIdx.x;
    const int bx = b % cb0, by = (b / cb0) % cb1, bz = b / (cb0 * cb1);
    const int x0 = max(bx * 16 - before, 0), y0 = max(by * 16 - before, 0), z0 = max(bz * 16 - before, 0);
    const int ex = min(bx * 16 + after, nx - 1) - x0 + 1;
    const int ey = min(by * 16 + after, ny - 1) - y0 + 1;
    const int ez = min(bz * 16 + after, nz - 1) - z0 + 1;
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

cudaError_t launch_minmax(const uint16_t *stage, const int n[3], const int cb[3], int vmax, int filter,
                          uint16_t *mn, uint16_t *mx, cudaStream_t s) {
    int nb = cb[0] * cb[1] * cb[2];
    const int before = filter == RC_FILTER_BSPLINE ? 1 : 0, after = filter == RC_FILTER_BSPLINE ? 17 : 16;
    minmax_kernel<<<nb, 256, 0, s>>>(stage, n[0], n[1], n[2], cb[0], cb[1], vmax, before, after, mn, mx);
    return cudaGetLastError();
}

// One thread per 4^3 sub-block: min and max of the (clamped) codes over its
// footprint voxels max(4j - before, 0) .. min(4j + after, N - 1) per axis,
// (0, 4) for trilinear samples and (1, 5) for cubic B-spline samples;
// ceil((N-1)/4) sub-blocks per axis.
__global__ void minmax4_kernel(const uint16_t *__restrict__ stage, int nx, int ny, int nz, int vmax, int c0,
                               int c1, int c2, int before, int after, uint16_t *mn, uint16_t *mx) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c0 * c1 * c2) return;
    const int jx = j % c0, jy = (j / c0) % c1, jz = j / (c0 * c1);
    int lo = 65535, hi = 0;
    for (int z = max(4 * jz - before, 0); z <= min(4 * jz + after, nz - 1); z++)
        for (int y = max(4 * jy - before, 0); y <= min(4 * jy + after, ny - 1); y++)
            for (int x = max(4 * jx - before, 0); x <= min(4 * jx + after, nx - 1); x++) {
                const int v = min((int)stage[((size_t)z * ny + y) * nx + x], vmax);
                lo = min(lo, v);
                hi = max(hi, v);
            }
    mn[j] = (uint16_t)lo;
    mx[j] = (uint16_t)hi;
}

cudaError_t launch_minmax4(const uint16_t *stage, const int n[3], int vmax, int filter, uint16_t *mn, uint16_t *mx,
                           cudaStream_t s) {
    const int c0 = (n[0] - 1 + 3) / 4, c1 = (n[1] - 1 + 3) / 4, c2 = (n[2] - 1 + 3) / 4;
    const int total = c0 * c1 * c2;
    const int before = filter == RC_FILTER_BSPLINE ? 1 : 0, after = filter == RC_FILTER_BSPLINE ? 5 : 4;
    minmax4_kernel<<<(total + 127) / 128, 128, 0, s>>>(stage, n[0], n[1], n[2], vmax, c0, c1, c2, before, after, mn,
                                                       mx);
    return cudaGetLastError();
}

// Whether any table entry a value in [vmn, vmx] can touch has non-zero
// opacity, with the march's coordinate u(v) = fl(v * ucoef).
__device__ __forceinline__ bool range_visible(float vmn, float vmx, int vmax, int f16_values, const TFDev &tf) {
    const int K = tf.K;
    if (f16_values) {
        vmn = __half2float(__float2half_rn(__fdiv_rn(vmn, (float)vmax)));
        vmx = __half2float(__float2half_rn(__fdiv_rn(vmx, (float)vmax)));
    }
    const int lo = min((int)floorf(__fmul_rn(vmn, tf.ucoef)), K - 1);
    const int hi = min((int)floorf(__fmul_rn(vmx, tf.ucoef)) + 1, K - 1);
    for (int i = lo; i <= hi; i++) {
        const float a = tf.M >= 2 ? tf.amax[i] : (tf.fp16 ? half4_to_float4(tf.f16[i]).w : tf.f32[i].w);
        if (a != 0.0f) return true;
    }
    return false;
}

// One thread per sub-block, 64 per cell-brick: bit t = sz*16 + sy*4 + sx of
// the brick's mask is set when sub-block (4*bx + sx, 4*by + sy, 4*bz + sz)
// exists and may hold non-zero opacity; each warp's ballot is one 32-bit half.
__global__ void __launch_bounds__(128) finemask_kernel(const uint16_t *mn4, const uint16_t *mx4, int c0, int c1,
                                                       int c2, int cb0, int cb1, int nbricks, int vmax,
                                                       int f16_values, TFDev tf, uint32_t *fine) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e >> 6), t = (int)(e & 63);
    bool vis = false;
    if (b < nbricks) {
        const int bx = b % cb0, by = (b / cb0) % cb1, bz = b / (cb0 * cb1);
        const int jx = 4 * bx + (t & 3), jy = 4 * by + ((t >> 2) & 3), jz = 4 * bz + (t >> 4);
        if (jx < c0 && jy < c1 && jz < c2) {
            const int j = (jz * c1 + jy) * c0 + jx;
            vis = range_visible((float)mn4[j], (float)mx4[j], vmax, f16_values, tf);
        }
    }
    const unsigned bits = __ballot_sync(0xffffffffu, vis);
    if ((threadIdx.x & 31) == 0 && b < nbricks) fine[2 * b + (t >> 5)] = bits;
}

cudaError_t launch_finemask(const uint16_t *mn4, const uint16_t *mx4, const int n[3], const int cb[3], int vmax,
                            int f16_values, TFDev tf, unsigned long long *fine, cudaStream_t s) {
    const int c0 = (n[0] - 1 + 3) / 4, c1 = (n[1] - 1 + 3) / 4, c2 = (n[2] - 1 + 3) / 4;
    const int nb = cb[0] * cb[1] * cb[2];
    const long long threads = (long long)nb * 64;
    finemask_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(mn4, mx4, c0, c1, c2, cb[0], cb[1], nb, vmax,
                                                                      f16_values, tf,
                                                                      reinterpret_cast<uint32_t *>(fine));
    return cudaGetLastError();
}

// A cell-brick is occupied unless every entry lo..hi its samples can touch has
// zero opacity, with the march's own coordinate u(v) = fl(v * ucoef): raw codes
// v = min, max; FP16 storage v = fp16(min / vmax), fp16(max / vmax). With a
// 2-D table an entry's opacity is its largest over the gradient rows.
__global__ void occupancy_kernel(const uint16_t *mn, const uint16_t *mx, int nbricks, int vmax, int f16_values,
                                 TFDev tf, uint8_t *occ) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbricks) return;
    const int K = tf.K;
    int lo, hi;
    float vmn = (float)mn[b], vmx = (float)mx[b];
    if (f16_values) {
        vmn = __half2float(__float2half_rn(__fdiv_rn(vmn, (float)vmax)));
        vmx = __half2float(__float2half_rn(__fdiv_rn(vmx, (float)vmax)));
    }
    lo = (int)floorf(__fmul_rn(vmn, tf.ucoef));
    hi = (int)floorf(__fmul_rn(vmx, tf.ucoef)) + 1;
    hi = min(hi, K - 1);
    lo = min(lo, K - 1);
    uint8_t any = 0;
    for (int i = lo; i <= hi && !any; i++) {
        float a = tf.M >= 2 ? tf.amax[i] : (tf.fp16 ? half4_to_float4(tf.f16[i]).w : tf.f32[i].w);
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
