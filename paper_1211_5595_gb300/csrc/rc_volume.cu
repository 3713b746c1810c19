// Volume preparation: re-layout of the uint16 codes into apron bricks (19^3
// voxels per 16^3-cell brick) in the chosen storage, value+gradient and pair
// bricks, the min/max grids and the occupancy masks of the current transfer
// function (Sec. 2.1 volume data, Sec. 2.6 classification).
#include "rc_device.cuh"

namespace rc {

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

// The whole preparation of one cell-brick from one staged copy of its
// footprint (one block of 256 threads per cell-brick): the codes of the
// brick's 19^3 apron box (voxels 16b-1 .. 16b+17 per axis, clamped to the
// volume so border voxels are replicated; codes clamped to vmax) are read once
// into shared memory and written out as
//   - the apron brick in the storage type: F32 keeps the code, F16 stores
//     h = fp16((code - o) / o) with the volume's offset o (a power of two with
//     2o >= vmax, so |code - o| <= 2048 is an FP16 integer for 12-bit data and
//     h is exact), U16 the code;
//   - the 17^3 value+gradient entries of voxels 16b .. 16b+16 (clamped) as
//     (V, V(x+1) - V(x-1), V(y+1) - V(y-1), V(z+1) - V(z-1)) of the codes,
//     neighbour indices clamped to the volume: exact in FP32 (float4) for
//     FP32 storage; for uint16 as 16-bit fields with the differences offset
//     by 32768 (uint2: V | Dx << 16, Dy | Dz << 16); for FP16 the same with
//     the bits of the stored FP16 value h in place of V (the differences of
//     stored values are the code differences / o, exactly, when o <= 2048);
//   - the trilinear cell-brick min / max over voxels max(16b, 0) .. min(16b+16, N-1);
//   - the trilinear min / max of the brick's 4^3 sub-blocks j over voxels
//     4j .. min(4j+4, N-1) (ceil((N-1)/4) sub-blocks per axis).
// minmax_kernel and minmax4_kernel compute the same grids for the B-spline
// footprints, on first use.
struct PrepArgs {
    const uint16_t *stage;
    int n[3], cb[3], c4[3];
    int vmax;
    int f16o;                    // FP16 storage: the offset o
    void *apron;
    void *vg;                    // float4 (FP32 storage), uint2 (uint16, FP16 storage) or null
    uint16_t *mn, *mx, *mn4, *mx4;
};

template <int ST>
__global__ void __launch_bounds__(256) prep_kernel(const PrepArgs A) {
    __shared__ uint16_t s_code[kApronVox];
    __shared__ int s_lo[8], s_hi[8];
    const unsigned b = blockIdx.x;
    const int bx = (int)(b % (unsigned)A.cb[0]), by = (int)((b / (unsigned)A.cb[0]) % (unsigned)A.cb[1]),
              bz = (int)(b / ((unsigned)A.cb[0] * (unsigned)A.cb[1]));
    const int x0 = bx * kBrick - 1, y0 = by * kBrick - 1, z0 = bz * kBrick - 1;     // box origin
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    // box codes, and the apron brick from them
    for (unsigned e = threadIdx.x; e < (unsigned)kApronVox; e += blockDim.x) {
        const int lx = (int)(e % kApron), ly = (int)((e / kApron) % kApron), lz = (int)(e / (kApron * kApron));
        const int x = min(max(x0 + lx, 0), nx - 1), y = min(max(y0 + ly, 0), ny - 1), z = min(max(z0 + lz, 0), nz - 1);
        const int code = min((int)A.stage[((size_t)z * ny + y) * nx + x], A.vmax);
        s_code[e] = (uint16_t)code;
        const size_t o = (size_t)b * kApronVox + e;
        if (ST == RC_STORE_F32) ((float *)A.apron)[o] = (float)code;
        else if (ST == RC_STORE_F16)
            ((__half *)A.apron)[o] = __float2half_rn(__fdiv_rn((float)(code - A.f16o), (float)A.f16o));
        else ((uint16_t *)A.apron)[o] = (uint16_t)code;
    }
    __syncthreads();
    // the code at volume coordinate (x, y, z) inside the box
    auto at = [&](int x, int y, int z) {
        return (int)s_code[((z - z0) * kApron + (y - y0)) * kApron + (x - x0)];
    };
    if (A.vg != nullptr) {
        for (unsigned e = threadIdx.x; e < (unsigned)kGradVox; e += blockDim.x) {
            const int lx = (int)(e % kGradEdge), ly = (int)((e / kGradEdge) % kGradEdge),
                      lz = (int)(e / (kGradEdge * kGradEdge));
            const int x = min(bx * kBrick + lx, nx - 1), y = min(by * kBrick + ly, ny - 1),
                      z = min(bz * kBrick + lz, nz - 1);
            const int V = at(x, y, z);
            const int dx = at(min(x + 1, nx - 1), y, z) - at(max(x - 1, 0), y, z);
            const int dy = at(x, min(y + 1, ny - 1), z) - at(x, max(y - 1, 0), z);
            const int dz = at(x, y, min(z + 1, nz - 1)) - at(x, y, max(z - 1, 0));
            if (ST == RC_STORE_F32) {
                reinterpret_cast<float4 *>(A.vg)[(size_t)b * kGradVox + e] =
                    make_float4((float)V, (float)dx, (float)dy, (float)dz);
            } else if (ST == RC_STORE_F16) {
                // the apron brick's value of this voxel, h = fp16((V - o) / o)
                const __half h = __float2half_rn(__fdiv_rn((float)(V - A.f16o), (float)A.f16o));
                reinterpret_cast<uint2 *>(A.vg)[(size_t)b * kGradVox + e] =
                    make_uint2((unsigned)__half_as_ushort(h) | ((unsigned)(dx + 32768) << 16),
                               (unsigned)(dy + 32768) | ((unsigned)(dz + 32768) << 16));
            } else {
                // codes <= 65535 and differences in (-32768, 32768): 16-bit fields
                reinterpret_cast<uint2 *>(A.vg)[(size_t)b * kGradVox + e] =
                    make_uint2((unsigned)V | ((unsigned)(dx + 32768) << 16),
                               (unsigned)(dy + 32768) | ((unsigned)(dz + 32768) << 16));
            }
        }
    }
    // cell-brick min / max over voxels max(16b, 0) .. min(16b + 16, N - 1)
    {
        const int xa = bx * kBrick, ya = by * kBrick, za = bz * kBrick;
        const int ex = min(xa + 16, nx - 1) - xa + 1, ey = min(ya + 16, ny - 1) - ya + 1,
                  ez = min(za + 16, nz - 1) - za + 1;
        int lo = 65535, hi = 0;
        for (int row = threadIdx.x; row < ey * ez; row += blockDim.x) {      // rows (y, z), then along x
            const int y = ya + row % ey, z = za + row / ey;
            for (int x = xa; x < xa + ex; x++) {
                const int v = at(x, y, z);
                lo = min(lo, v);
                hi = max(hi, v);
            }
        }
        lo = (int)__reduce_min_sync(0xffffffffu, (unsigned)lo);
        hi = (int)__reduce_max_sync(0xffffffffu, (unsigned)hi);
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
            A.mn[b] = (uint16_t)lo;
            A.mx[b] = (uint16_t)hi;
        }
    }
    // the 4^3 sub-blocks j = 4b + s of the brick, four threads each, over
    // voxels 4j .. min(4j + 4, N - 1)
    {
        const int sb = threadIdx.x >> 2, q = threadIdx.x & 3;               // sub-block 0..63, quarter
        const int sx = sb & 3, sy = (sb >> 2) & 3, sz = sb >> 4;
        const int jx = 4 * bx + sx, jy = 4 * by + sy, jz = 4 * bz + sz;
        const bool exists = jx < A.c4[0] && jy < A.c4[1] && jz < A.c4[2];
        int lo = 65535, hi = 0;
        if (exists) {
            const int xa = 4 * jx, ya = 4 * jy, za = 4 * jz;
            const int ex = min(xa + 4, nx - 1) - xa + 1, ey = min(ya + 4, ny - 1) - ya + 1,
                      ez = min(za + 4, nz - 1) - za + 1;
            for (int row = q; row < ey * ez; row += 4) {                      // rows (y, z), then along x
                const int y = ya + row % ey, z = za + row / ey;
                for (int x = xa; x < xa + ex; x++) {
                    const int v = at(x, y, z);
                    lo = min(lo, v);
                    hi = max(hi, v);
                }
            }
        }
        // the four threads of a sub-block are lanes 4k .. 4k+3 of one warp
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, 1));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, 1));
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, 2));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, 2));
        if (exists && q == 0) {
            const size_t j = ((size_t)jz * A.c4[1] + jy) * A.c4[0] + jx;
            A.mn4[j] = (uint16_t)lo;
            A.mx4[j] = (uint16_t)hi;
        }
    }
}

cudaError_t launch_prep(const uint16_t *stage, VolDev v, void *apron, void *vg, uint16_t *mn, uint16_t *mx,
                        uint16_t *mn4, uint16_t *mx4, cudaStream_t s) {
    PrepArgs a;
    a.stage = stage;
    for (int i = 0; i < 3; i++) {
        a.n[i] = v.n[i];
        a.cb[i] = v.cb[i];
        a.c4[i] = (v.n[i] - 1 + 3) / 4;
    }
    a.vmax = v.vmax;
    a.f16o = (int)v.f16o;
    a.apron = apron;
    a.vg = vg;
    a.mn = mn;
    a.mx = mx;
    a.mn4 = mn4;
    a.mx4 = mx4;
    const unsigned nb = (unsigned)(v.cb[0] * v.cb[1] * v.cb[2]);
    switch (v.storage) {
        case RC_STORE_F32: prep_kernel<RC_STORE_F32><<<nb, 256, 0, s>>>(a); break;
        case RC_STORE_F16: prep_kernel<RC_STORE_F16><<<nb, 256, 0, s>>>(a); break;
        default: prep_kernel<RC_STORE_U16><<<nb, 256, 0, s>>>(a);
    }
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

// The march's table coordinate of a code as the volume stores it: raw codes
// u = fl(v * ucoef); FP16 storage (f16o = o > 0) h = fp16((v - o) / o) and
// u = fl((h + 1) * ucoef), as tf_coord computes them.
__device__ __forceinline__ float code_coord(float v, int f16o, float ucoef) {
    if (f16o) {
        const float h = __half2float(__float2half_rn(__fdiv_rn(v - (float)f16o, (float)f16o)));
        return __fmaf_rn(h, ucoef, ucoef);
    }
    return __fmul_rn(v, ucoef);
}

// Whether any table entry a value in [vmn, vmx] can touch has non-zero
// opacity, with the march's coordinate u.
__device__ __forceinline__ bool range_visible(float vmn, float vmx, int f16o, const TFDev &tf) {
    const int K = tf.K;
    const int lo = min((int)floorf(code_coord(vmn, f16o, tf.ucoef)), K - 1);
    const int hi = min((int)floorf(code_coord(vmx, f16o, tf.ucoef)) + 1, K - 1);
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
                                                       int c2, int cb0, int cb1, int nbricks, int f16o,
                                                       TFDev tf, uint32_t *fine) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e >> 6), t = (int)(e & 63);
    bool vis = false;
    if (b < nbricks) {
        const int bx = b % cb0, by = (b / cb0) % cb1, bz = b / (cb0 * cb1);
        const int jx = 4 * bx + (t & 3), jy = 4 * by + ((t >> 2) & 3), jz = 4 * bz + (t >> 4);
        if (jx < c0 && jy < c1 && jz < c2) {
            const int j = (jz * c1 + jy) * c0 + jx;
            vis = range_visible((float)mn4[j], (float)mx4[j], f16o, tf);
        }
    }
    const unsigned bits = __ballot_sync(0xffffffffu, vis);
    if ((threadIdx.x & 31) == 0 && b < nbricks) fine[2 * b + (t >> 5)] = bits;
}

cudaError_t launch_finemask(const uint16_t *mn4, const uint16_t *mx4, const int n[3], const int cb[3], int vmax,
                            int f16o, TFDev tf, unsigned long long *fine, cudaStream_t s) {
    const int c0 = (n[0] - 1 + 3) / 4, c1 = (n[1] - 1 + 3) / 4, c2 = (n[2] - 1 + 3) / 4;
    const int nb = cb[0] * cb[1] * cb[2];
    const long long threads = (long long)nb * 64;
    (void)vmax;
    finemask_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(mn4, mx4, c0, c1, c2, cb[0], cb[1], nb, f16o,
                                                                      tf, reinterpret_cast<uint32_t *>(fine));
    return cudaGetLastError();
}

// A cell-brick is occupied unless every entry lo..hi its samples can touch has
// zero opacity, with the march's own coordinate u of the brick's min and max
// as stored (code_coord). With a 2-D table an entry's opacity is its largest
// over the gradient rows.
__global__ void occupancy_kernel(const uint16_t *mn, const uint16_t *mx, int nbricks, int f16o, TFDev tf,
                                 uint8_t *occ) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbricks) return;
    const int K = tf.K;
    int lo, hi;
    lo = (int)floorf(code_coord((float)mn[b], f16o, tf.ucoef));
    hi = (int)floorf(code_coord((float)mx[b], f16o, tf.ucoef)) + 1;
    hi = min(hi, K - 1);
    lo = min(lo, K - 1);
    uint8_t any = 0;
    for (int i = lo; i <= hi && !any; i++) {
        float a = tf.M >= 2 ? tf.amax[i] : (tf.fp16 ? half4_to_float4(tf.f16[i]).w : tf.f32[i].w);
        any = a != 0.0f;
    }
    occ[b] = any;
}

cudaError_t launch_occupancy(const uint16_t *mn, const uint16_t *mx, int nbricks, int vmax, int f16o,
                             TFDev tf, uint8_t *occ, cudaStream_t s) {
    (void)vmax;
    occupancy_kernel<<<(nbricks + 127) / 128, 128, 0, s>>>(mn, mx, nbricks, f16o, tf, occ);
    return cudaGetLastError();
}

}  // namespace rc
