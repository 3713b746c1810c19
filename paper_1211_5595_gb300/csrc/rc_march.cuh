// Forward march kernels (Sec. 4.1-4.2): one thread per ray, warps on 8 x 4
// pixel tiles, bricked volume gathers through the read-only path, transfer
// function in shared memory (1-D) or global memory (2-D), exact empty-space
// skipping over the cell-brick occupancy mask and warp-vote early ray
// termination. The instances are spread over several translation units
// (rc_march.cu, rc_march_cubic.cu, rc_march_tf2.cu) so they compile in parallel.
#pragma once

#include "rc_device.cuh"

namespace rc {

constexpr unsigned kFull = 0xffffffffu;

// A CTA renders a tile of kTileW x kTileH pixels, each warp an 8 x 4 block
// of it.
constexpr int kWarpsX = 2, kWarpsY = 2;
constexpr int kTileW = 8 * kWarpsX, kTileH = 4 * kWarpsY, kMarchThreads = 32 * kWarpsX * kWarpsY;

__device__ __forceinline__ void pixel_of_thread(int &x, int &y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = blockIdx.x * kTileW + (warp % kWarpsX) * 8 + (lane & 7);
    y = blockIdx.y * kTileH + (warp / kWarpsX) * 4 + (lane >> 3);
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, unsigned dense, unsigned evald,
                                          unsigned hit, unsigned inimg) {
    dense = __reduce_add_sync(kFull, dense);
    evald = __reduce_add_sync(kFull, evald);
    hit = __reduce_add_sync(kFull, hit);
    inimg = __reduce_add_sync(kFull, inimg);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(stats + 0, (unsigned long long)dense);
        atomicAdd(stats + 1, (unsigned long long)evald);
        atomicAdd(stats + 2, (unsigned long long)hit);
        atomicAdd(stats + 3, (unsigned long long)inimg);
    }
}

// Compositing ray function (Sec. 4.2, Eq. 4): C += T a' c, T *= (1 - a'),
// front to back from the eye; stop after the sample where 1 - T >= term.
// F selects the sample form (kShade, kCubic, kTF2).
template <int ST, int F, int RM>
__global__ void __launch_bounds__(kMarchThreads) composite_kernel(const MarchArgs a) {
    extern __shared__ float4 s_tf[];
    if (!(F & kTF2)) {
        load_tf(a.tf, s_tf);
        __syncthreads();
    }
    // a batch of volumes: the volume's own data and masks, the shared record
    VolDev vol = a.vol;
    const uint8_t *occ = a.occ;
    const unsigned long long *fine = a.fine;
    int view = blockIdx.z;
    if (a.batch) {
        const int vi = blockIdx.z / a.views;
        view = blockIdx.z - vi * a.views;
        const BatchVol bv = a.batch[vi];
        vol.data = bv.data;
        vol.vg = bv.vg;
        vol.pairs = bv.pairs;
        occ = bv.occ;
        fine = bv.fine;
    }
    const CamRec cam = a.cams ? a.cams[view] : a.cam;
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
    while (__any_sync(kFull, active)) {
        if (!active) continue;
        float p[3];
        position_at(R, sample_t(R, k), p);
        Cell c;
        cell_of(vol, p, c);
        if (a.p.skip) {
            // the largest empty block around the sample: with the fine mask
            // the cell-brick, its octant or its 4^3 sub-block; else the brick
            const int b = brick_of(vol, c);
            const int s = fine ? empty_block(__ldg(fine + b), c) : (__ldg(occ + b) ? -1 : 4);
            if (s >= 0) {
                k = jump_block(R, vol, c, k, s);
                active = k < nsamp;
                continue;
            }
        }
        float4 e = eval_sample_x<ST, F, RM>(vol, a.p, s_tf, a.tf, R.dir, c, a.p.rmode, a.p.ratio);
        composite_add(e, C0, C1, C2, T);
        evald++;
        k++;
        active = k < nsamp && (1.0f - T) < a.p.term;
    }
    if (inimg) out[(size_t)y * cam.W + x] = make_float4(C0, C1, C2, 1.0f - T);
    if (a.stats) add_stats(a.stats, (unsigned)min(k, nsamp), evald, hit ? 1u : 0u, inimg ? 1u : 0u);
}

// The other ray functions of Sec. 4.1 (MIP, average, x-ray, isosurface,
// threshold); output channels as documented in rc.h. CUBIC: B-spline values
// and analytic gradient instead of trilinear values and central differences.
template <int ST, bool CUBIC>
__global__ void __launch_bounds__(kMarchThreads) function_kernel(const MarchArgs a) {
    extern __shared__ float4 s_tf[];
    if (a.p.func == RC_FUNC_THRESHOLD) {   // the only one that classifies (1-D table)
        load_tf(a.tf, s_tf);
        __syncthreads();
    }
    const CamRec cam = a.cams ? a.cams[blockIdx.z] : a.cam;
    float4 *outp = a.out + (size_t)blockIdx.z * cam.W * cam.H;
    int x, y;
    pixel_of_thread(x, y);
    const bool inimg = x < cam.W && y < cam.H;
    Ray R;
    const bool hit = inimg && setup_ray(cam, a.vol, a.p.step_vox, x, y, R);
    const int nsamp = hit ? R.nsamp : 0;
    const int func = a.p.func;
    float4 out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float acc = 0.0f, prev_v = 0.0f, prev_t = 0.0f;
    int k = 0;
    bool found = false;
    for (; k < nsamp; k++) {
        float t = sample_t(R, k), p[3];
        position_at(R, t, p);
        Cell c;
        cell_of(a.vol, p, c);
        float v = CUBIC ? bspline<ST>(a.vol, c) : trilinear<ST>(a.vol, c);
        if (func == RC_FUNC_MIP) {
            acc = k == 0 ? v : fmaxf(acc, v);
        } else if (func == RC_FUNC_AVERAGE || func == RC_FUNC_XRAY) {
            acc += v;
        } else if (v >= a.p.iso) {
            found = true;
            if (func == RC_FUNC_THRESHOLD) {
                float4 e = classify(s_tf, a.tf.K, tf_coord<ST>(v, a.tf.ucoef), nullptr, nullptr, RC_DBG_ERR(a.vol));
                out = make_float4(e.x, e.y, e.z, 1.0f);
            } else {
                float ts = k > 0 ? prev_t + (t - prev_t) * ((a.p.iso - prev_v) / (v - prev_v)) : t;
                float g[3], sf, spec;
                if (CUBIC) bspline_grad<ST>(a.vol, c, g);
                else value_grad<ST>(a.vol, c, g);
                shade_factor(a.p, a.vol, g, R.dir, sf, spec);
                out = make_float4(ts, fminf(1.0f, sf + spec), (float)k, 1.0f);
            }
            k++;
            break;
        }
        prev_v = v;
        prev_t = t;
    }
    if (!found && nsamp > 0) {
        // over full scale; FP16 values h = (code - o) / o are shifted by 1 first
        // (code / vmax = (h + 1) / vscale)
        float m = 0.0f;
        bool have = true;
        if (ST == RC_STORE_F16) {
            if (func == RC_FUNC_MIP) m = (acc + 1.0f) / a.vol.vscale;
            else if (func == RC_FUNC_AVERAGE) m = (acc / (float)nsamp + 1.0f) / a.vol.vscale;
            else if (func == RC_FUNC_XRAY) m = (acc + (float)nsamp) * R.ds / a.vol.vscale;
            else have = false;
        } else {
            if (func == RC_FUNC_MIP) m = acc / a.vol.vscale;
            else if (func == RC_FUNC_AVERAGE) m = acc / (float)nsamp / a.vol.vscale;
            else if (func == RC_FUNC_XRAY) m = acc * R.ds / a.vol.vscale;
            else have = false;
        }
        if (have) out = make_float4(m, m, m, 1.0f);
    }
    if (inimg) outp[(size_t)y * cam.W + x] = out;
    if (a.stats) add_stats(a.stats, (unsigned)k, (unsigned)k, hit ? 1u : 0u, inimg ? 1u : 0u);
}

template <typename K>
static cudaError_t launch_kernel(K kern, const MarchArgs &a, int nviews, bool table_in_smem, cudaStream_t s) {
    size_t smem = table_in_smem ? (size_t)a.tf.K * sizeof(float4) : 0;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.cam.W + kTileW - 1) / kTileW, (a.cam.H + kTileH - 1) / kTileH, nviews);
    kern<<<grid, kMarchThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Composite march with sample form F and opacity-correction mode RM for the
// volume's storage type.
template <int F, int RM>
static cudaError_t launch_composite_rm(const MarchArgs &a, int nviews, cudaStream_t s) {
    const bool smem = !(F & kTF2);
    switch (a.vol.storage) {
        case RC_STORE_F32: return launch_kernel(composite_kernel<RC_STORE_F32, F, RM>, a, nviews, smem, s);
        case RC_STORE_F16: return launch_kernel(composite_kernel<RC_STORE_F16, F, RM>, a, nviews, smem, s);
        default: return launch_kernel(composite_kernel<RC_STORE_U16, F, RM>, a, nviews, smem, s);
    }
}

// The step ratios of the fixed modes (1, 1/2, 1/4) get their own instances.
template <int F>
static cudaError_t launch_composite(const MarchArgs &a, int nviews, cudaStream_t s) {
    switch (a.p.rmode) {
        case 0: return launch_composite_rm<F, 0>(a, nviews, s);
        case 1: return launch_composite_rm<F, 1>(a, nviews, s);
        case 2: return launch_composite_rm<F, 2>(a, nviews, s);
        default: return launch_composite_rm<F, 3>(a, nviews, s);
    }
}

template <bool CUBIC>
static cudaError_t launch_function(const MarchArgs &a, int nviews, cudaStream_t s) {
    const bool smem = a.p.func == RC_FUNC_THRESHOLD;
    switch (a.vol.storage) {
        case RC_STORE_F32: return launch_kernel(function_kernel<RC_STORE_F32, CUBIC>, a, nviews, smem, s);
        case RC_STORE_F16: return launch_kernel(function_kernel<RC_STORE_F16, CUBIC>, a, nviews, smem, s);
        default: return launch_kernel(function_kernel<RC_STORE_U16, CUBIC>, a, nviews, smem, s);
    }
}

}  // namespace rc
