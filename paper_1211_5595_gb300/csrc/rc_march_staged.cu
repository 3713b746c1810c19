// Brick-staged variant of the shaded FP32 compositing march: each CTA copies
// the 17^3 value+gradient brick its rays need next into shared memory with
// one bulk (TMA) copy, the rays whose next sample lies in that brick march
// through it reading shared memory, and the CTA moves on to the next brick
// (the smallest brick index any of its rays needs) until every ray is done.
// The per-sample arithmetic is composite_kernel's (the same loads' values,
// the same operations), so the images are identical. It is an alternative
// kept for measurement: the staging of a whole 78.6 KB brick serves only the
// thin pencil of it that a 16 x 8 pixel tile's rays cross, so it moves far
// more bytes than the cached gathers of composite_kernel.
#include "rc_march.cuh"
#include "rc_tcgen05.cuh"

namespace rc {

constexpr unsigned kStagedBytes = (unsigned)kGradVox * 16u;     // 78,608 B: one value+gradient brick

// value_grad_vg on a brick in shared memory (same loads' values, same order).
__device__ __forceinline__ float value_grad_staged(const ulonglong2 *brick, const VolDev &v, const Cell &c,
                                                   float g[3]) {
    const unsigned idx = (unsigned)(((c.i[2] & 15) * kGradEdge + (c.i[1] & 15)) * kGradEdge + (c.i[0] & 15));
    const ulonglong2 *p = brick + idx;
    constexpr int DY = kGradEdge, DZ = kGradEdge * kGradEdge;
    const unsigned long long wx = pack2(c.w[0], c.w[0]), wy = pack2(c.w[1], c.w[1]), wz = pack2(c.w[2], c.w[2]);
    const ulonglong2 c00 = lerp4p(p[0], p[1], wx);
    const ulonglong2 c10 = lerp4p(p[DY], p[DY + 1], wx);
    const ulonglong2 c01 = lerp4p(p[DZ], p[DZ + 1], wx);
    const ulonglong2 c11 = lerp4p(p[DZ + DY], p[DZ + DY + 1], wx);
    const float4 r = unpack4(lerp4p(lerp4p(c00, c10, wy), lerp4p(c01, c11, wy), wz));
    g[0] = r.y * v.inv2s[0];
    g[1] = r.z * v.inv2s[1];
    g[2] = r.w * v.inv2s[2];
    return r.x;
}

template <int RM>
__global__ void __launch_bounds__(kMarchThreads) staged_kernel(const MarchArgs a, int *err, long long budget) {
    extern __shared__ __align__(128) uint8_t smem[];
    const ulonglong2 *s_vg = reinterpret_cast<const ulonglong2 *>(smem);
    float4 *s_tf = reinterpret_cast<float4 *>(smem + kStagedBytes);
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned s_min[kWarpsX * kWarpsY];
    load_tf(a.tf, s_tf);
    const uint32_t bar_a = tc::smem_addr(&bar);
    if (threadIdx.x == 0) tc::bar_init(bar_a, 1);
    __syncthreads();
    const VolDev &vol = a.vol;
    const CamRec cam = a.cams ? a.cams[blockIdx.z] : a.cam;
    float4 *out = a.out + (size_t)blockIdx.z * cam.W * cam.H;
    int x, y;
    pixel_of_thread(x, y);
    const bool inimg = x < cam.W && y < cam.H;
    Ray R;
    const bool hit = inimg && setup_ray(cam, vol, a.p.step_vox, x, y, R);
    const int nsamp = hit ? R.nsamp : 0;
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
    int k = 0;
    unsigned evald = 0;
    bool active = nsamp > 0;
    unsigned staged = 0xffffffffu, phase = 0;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        // through empty space (the masks only) to the next sample that needs data
        unsigned mine = 0xffffffffu;
        Cell c;
        while (active) {
            float p[3];
            position_at(R, sample_t(R, k), p);
            cell_of(vol, p, c);
            const int b = brick_of(vol, c);
            const int s = a.fine ? empty_block(__ldg(a.fine + b), c) : (__ldg(a.occ + b) ? -1 : 4);
            if (s >= 0) {
                k = jump_block(R, vol, c, k, s);
                active = k < nsamp;
                continue;
            }
            mine = (unsigned)b;
            break;
        }
        // the CTA's next brick: the smallest any ray needs
        const unsigned wmin = __reduce_min_sync(kFull, mine);
        if (lane == 0) s_min[warp] = wmin;
        __syncthreads();
        unsigned bmin = s_min[0];
#pragma unroll
        for (int w = 1; w < kWarpsX * kWarpsY; w++) bmin = min(bmin, s_min[w]);
        if (bmin == 0xffffffffu) break;
        if (bmin != staged) {
            if (threadIdx.x == 0) {
                tc::fence_async_smem();
                tc::bulk_g2s(tc::smem_addr(smem), reinterpret_cast<const float4 *>(vol.vg) + (size_t)bmin * kGradVox,
                             kStagedBytes, bar_a);
            }
            const bool ok = __syncthreads_and(tc::bar_wait(bar_a, phase, budget));
            if (!ok) {
                // the copy did not complete in time: report it, wait (bounded)
                // for the copy in flight and stop; the image is invalid
                if (threadIdx.x == 0) atomicOr(err, 1);
                tc::bar_wait(bar_a, phase, budget);
                break;
            }
            phase ^= 1u;
            staged = bmin;
        }
        if (active && mine == bmin) {
            for (;;) {
                float g[3];
                const float val = value_grad_staged(s_vg, vol, c, g);
                float4 e = classify(s_tf, a.tf.K, tf_coord<RC_STORE_F32>(val, a.tf.ucoef), nullptr, nullptr,
                                    RC_DBG_ERR(vol));
                const float ap = correct_alpha<RM>(e.w, a.p.rmode, a.p.ratio);
                float sf, spec;
                shade_factor(a.p, vol, g, R.dir, sf, spec);
                e.x = fminf(1.0f, __fmaf_rn(e.x, sf, spec));
                e.y = fminf(1.0f, __fmaf_rn(e.y, sf, spec));
                e.z = fminf(1.0f, __fmaf_rn(e.z, sf, spec));
                e.w = ap;
                composite_add(e, C0, C1, C2, T);
                evald++;
                k++;
                active = k < nsamp && (1.0f - T) < a.p.term;
                if (!active) break;
                float p[3];
                position_at(R, sample_t(R, k), p);
                cell_of(vol, p, c);
                const int b = brick_of(vol, c);
                if ((unsigned)b != bmin) break;
                if ((a.fine ? empty_block(__ldg(a.fine + b), c) : (__ldg(a.occ + b) ? -1 : 4)) >= 0) break;
            }
        }
        __syncthreads();      // the brick and s_min are read before the next stage replaces them
    }
    if (inimg) out[(size_t)y * cam.W + x] = make_float4(C0, C1, C2, 1.0f - T);
    if (a.stats) add_stats(a.stats, (unsigned)min(k, nsamp), evald, hit ? 1u : 0u, inimg ? 1u : 0u);
}

// The staged march for FP32 storage, shaded, trilinear, 1-D table, compositing;
// false when the form is another (the caller then runs composite_kernel).
bool staged_eligible(const MarchArgs &a) {
    return a.vol.storage == RC_STORE_F32 && a.vol.vg != nullptr && a.p.shade && a.p.skip &&
           a.p.func == RC_FUNC_COMPOSITE && a.p.filter == RC_FILTER_TRILINEAR && a.tf.M < 2 && a.batch == nullptr;
}

cudaError_t launch_march_staged(const MarchArgs &a, int nviews, int *err, long long budget, cudaStream_t s) {
    const size_t smem = kStagedBytes + (size_t)a.tf.K * sizeof(float4);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((a.cam.W + kTileW - 1) / kTileW, (a.cam.H + kTileH - 1) / kTileH, nviews);
        kern<<<grid, kMarchThreads, smem, s>>>(a, err, budget);
        return cudaGetLastError();
    };
    switch (a.p.rmode) {
        case 0: return go(staged_kernel<0>);
        case 1: return go(staged_kernel<1>);
        case 2: return go(staged_kernel<2>);
        default: return go(staged_kernel<3>);
    }
}

}  // namespace rc
