// Learned sampling proposal: opacity profiles of the plain march (training
// targets), the per-ray feature encoder, a 112-64-64-64-40 BF16 network on the
// tensor cores (mma.sync m16n8k16, FP32 accumulation, activations chained in
// registers), its SIMT training kernels (deterministic gradient reduction,
// Adam), and the importance-sampled march with fallback to the plain march.
//
// The paper has no learned part: the proposal replaces the evenly spaced
// samples of Sec. 4.1 by 64 samples drawn where the network expects opacity,
// and keeps the compositing of Sec. 4.2 (Eq. 3-4) with each sample's opacity
// corrected to the length of the segment it stands for.
#include <cuda_bf16.h>

#include "rc_device.cuh"

namespace rc {

constexpr int kFeatStride = 120;   // BF16 per feature row in shared memory (conflict-free fragments)
constexpr int kResStride = 33;     // floats per network-output row in shared memory

__device__ __forceinline__ void tile_pixel(int &x, int &y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    y = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
}

// ---------------------------------------------------------------------------
// opacity profiles: 512 samples at the centres of 512 equal segments of the
// chord, no termination; weights T_k a'_k summed 16 per bin; T at the end
// ---------------------------------------------------------------------------
template <int ST>
__global__ void __launch_bounds__(128) profiles_kernel(const MarchArgs a, float *out) {
    extern __shared__ float4 s_tf[];
    load_tf(a.tf, s_tf);
    __syncthreads();
    int x, y;
    tile_pixel(x, y);
    if (x >= a.cam.W || y >= a.cam.H) return;
    Ray R;
    const bool hit = setup_ray(a.cam, a.vol, a.p.step_vox, x, y, R);
    float *o = out + ((size_t)y * a.cam.W + x) * kOutUsed;
    if (!hit) {
        for (int b = 0; b < kBins; b++) o[b] = 0.0f;
        o[kBins] = 1.0f;
        return;
    }
    const float delta = __fdiv_rn(__fsub_rn(R.tf, R.tn), (float)kProfSamples);
    const float ratio = __fdiv_rn(delta, a.vol.smin);
    float T = 1.0f;
    for (int b = 0; b < kBins; b++) {
        float acc = 0.0f;
        for (int kk = 0; kk < kProfSamples / kBins; kk++) {
            const int k = b * (kProfSamples / kBins) + kk;
            float p[3];
            position_at(R, __fmaf_rn((float)k + 0.5f, delta, R.tn), p);
            Cell c;
            cell_of(a.vol, p, c);
            if (a.p.skip && !__ldg(a.occ + brick_of(a.vol, c))) continue;   // opacity exactly 0
            float4 e = eval_sample<ST, false>(a.vol, a.p, s_tf, a.tf.K, a.tf.ucoef, R.dir, c, 3, ratio);
            acc = __fmaf_rn(T, e.w, acc);
            T = T * (1.0f - e.w);
        }
        o[b] = acc;
    }
    o[kBins] = T;
}

// ---------------------------------------------------------------------------
// features: entry point (normalised to the box) and world direction, their
// sin/cos encodings at 6 octaves, 32 occupancy bits along the chord, 2 zeros
// ---------------------------------------------------------------------------
template <typename Put>
__device__ __forceinline__ void ray_features(const VolDev &v, const uint8_t *occ, const Ray &R, bool hit, Put put) {
    if (!hit) {
        for (int i = 0; i < kFeat; i++) put(i, 0.0f);
        return;
    }
    float xs[6];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        xs[c] = __fdiv_rn(__fmaf_rn(R.tn, R.d[c], R.o[c]), (float)(v.n[c] - 1));
        xs[3 + c] = R.dir[c];
    }
#pragma unroll
    for (int c = 0; c < 6; c++) put(c, xs[c]);
#pragma unroll
    for (int c = 0; c < 6; c++) {
#pragma unroll
        for (int j = 0; j < 6; j++) {
            float s, co;
            sincospif(ldexpf(xs[c], j), &s, &co);
            put(6 + 12 * c + 2 * j, s);
            put(7 + 12 * c + 2 * j, co);
        }
    }
    const float bw = __fdiv_rn(__fsub_rn(R.tf, R.tn), (float)kBins);
    for (int b = 0; b < kBins; b++) {
        float p[3];
        position_at(R, __fmaf_rn((float)b + 0.5f, bw, R.tn), p);
        Cell c;
        cell_of(v, p, c);
        put(78 + b, __ldg(occ + brick_of(v, c)) ? 1.0f : 0.0f);
    }
    put(110, 0.0f);
    put(111, 0.0f);
}

__global__ void __launch_bounds__(128) features_kernel(const MarchArgs a, float *out) {
    int x, y;
    tile_pixel(x, y);
    if (x >= a.cam.W || y >= a.cam.H) return;
    Ray R;
    const bool hit = setup_ray(a.cam, a.vol, a.p.step_vox, x, y, R);
    float *o = out + ((size_t)y * a.cam.W + x) * kFeat;
    ray_features(a.vol, a.occ, R, hit, [&](int i, float v) { o[i] = v; });
}

// ---------------------------------------------------------------------------
// the network on the tensor cores, one warp per 32 rays
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// c[m][j] = bias + sum over k-tiles of A[m][i] * B[i][j] for two 16-row m-tiles.
template <int KT, int NT>
__device__ __forceinline__ void dense_layer(const uint32_t (&a)[2][KT][4], const uint2 *__restrict__ frag,
                                            const float *__restrict__ bias, float (&c)[2][NT][4]) {
    const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
    for (int j = 0; j < NT; j++) {
        const float b0 = __ldg(bias + 8 * j + 2 * t), b1 = __ldg(bias + 8 * j + 2 * t + 1);
#pragma unroll
        for (int m = 0; m < 2; m++) {
            c[m][j][0] = b0;
            c[m][j][1] = b1;
            c[m][j][2] = b0;
            c[m][j][3] = b1;
        }
    }
#pragma unroll
    for (int i = 0; i < KT; i++) {
#pragma unroll
        for (int j = 0; j < NT; j++) {
            const uint2 b = __ldg(frag + (i * NT + j) * 32 + lane);
            mma_bf16_16816(c[0][j], a[0][i], b);
            mma_bf16_16816(c[1][j], a[1][i], b);
        }
    }
}

// ReLU, round to BF16 and re-pack: the accumulators of n-tiles 2i, 2i+1 are
// exactly the A fragment of k-tile i of the next layer.
template <int NT>
__device__ __forceinline__ void relu_pack(const float (&c)[2][NT][4], uint32_t (&a)[2][NT / 2][4]) {
#pragma unroll
    for (int m = 0; m < 2; m++) {
#pragma unroll
        for (int i = 0; i < NT / 2; i++) {
            a[m][i][0] = pack_bf16x2(fmaxf(c[m][2 * i][0], 0.0f), fmaxf(c[m][2 * i][1], 0.0f));
            a[m][i][1] = pack_bf16x2(fmaxf(c[m][2 * i][2], 0.0f), fmaxf(c[m][2 * i][3], 0.0f));
            a[m][i][2] = pack_bf16x2(fmaxf(c[m][2 * i + 1][0], 0.0f), fmaxf(c[m][2 * i + 1][1], 0.0f));
            a[m][i][3] = pack_bf16x2(fmaxf(c[m][2 * i + 1][2], 0.0f), fmaxf(c[m][2 * i + 1][3], 0.0f));
        }
    }
}

// feat: 32 rows (rays) of kFeatStride BF16; res: 32 rows of kResStride floats
// receiving the 32-bin PDF (softmax) and T^ (sigmoid). All 32 lanes must call.
__device__ __forceinline__ void warp_network(const NetDev &net, const __nv_bfloat16 *feat, float *res) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t a1[2][kFeat / 16][4];
#pragma unroll
    for (int m = 0; m < 2; m++) {
#pragma unroll
        for (int i = 0; i < kFeat / 16; i++) {
            const __nv_bfloat16 *r0 = feat + (16 * m + g) * kFeatStride + 16 * i + 2 * t;
            const __nv_bfloat16 *r1 = r0 + 8 * kFeatStride;
            a1[m][i][0] = *reinterpret_cast<const uint32_t *>(r0);
            a1[m][i][1] = *reinterpret_cast<const uint32_t *>(r1);
            a1[m][i][2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
            a1[m][i][3] = *reinterpret_cast<const uint32_t *>(r1 + 8);
        }
    }
    float c1[2][kHid / 8][4];
    dense_layer<kFeat / 16, kHid / 8>(a1, net.frag + kFragL1, net.params + kOffB1, c1);
    uint32_t a2[2][kHid / 16][4];
    relu_pack<kHid / 8>(c1, a2);
    float c2[2][kHid / 8][4];
    dense_layer<kHid / 16, kHid / 8>(a2, net.frag + kFragL2, net.params + kOffB2, c2);
    uint32_t a3[2][kHid / 16][4];
    relu_pack<kHid / 8>(c2, a3);
    float c3[2][kHid / 8][4];
    dense_layer<kHid / 16, kHid / 8>(a3, net.frag + kFragL3, net.params + kOffB3, c3);
    uint32_t a4[2][kHid / 16][4];
    relu_pack<kHid / 8>(c3, a4);
    float c4[2][kOut / 8][4];
    dense_layer<kHid / 16, kOut / 8>(a4, net.frag + kFragL4, net.params + kOffB4, c4);
#pragma unroll
    for (int m = 0; m < 2; m++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            float mx = -INFINITY;
#pragma unroll
            for (int j = 0; j < kBins / 8; j++) mx = fmaxf(mx, fmaxf(c4[m][j][2 * h], c4[m][j][2 * h + 1]));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
            float e[kBins / 8][2], sum = 0.0f;
#pragma unroll
            for (int j = 0; j < kBins / 8; j++) {
                e[j][0] = expf(c4[m][j][2 * h] - mx);
                e[j][1] = expf(c4[m][j][2 * h + 1] - mx);
                sum += e[j][0] + e[j][1];
            }
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            const float inv = 1.0f / sum;
            float *row = res + (16 * m + g + 8 * h) * kResStride;
#pragma unroll
            for (int j = 0; j < kBins / 8; j++) {
                row[8 * j + 2 * t] = e[j][0] * inv;
                row[8 * j + 2 * t + 1] = e[j][1] * inv;
            }
            if (t == 0) row[kBins] = 1.0f / (1.0f + expf(-c4[m][kBins / 8][2 * h]));
        }
    }
}

__global__ void __launch_bounds__(128) net_forward_kernel(const NetDev net, const float *__restrict__ feat,
                                                          long long n, float *__restrict__ out) {
    __shared__ __align__(16) __nv_bfloat16 s_feat[4][32 * kFeatStride];
    __shared__ float s_res[4][32 * kResStride];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = ((long long)blockIdx.x * 4 + warp) * 32;
    for (int e = lane; e < 32 * kFeat; e += 32) {
        const int r = e / kFeat, k = e % kFeat;
        const float v = base + r < n ? feat[(base + r) * kFeat + k] : 0.0f;
        s_feat[warp][r * kFeatStride + k] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    warp_network(net, s_feat[warp], s_res[warp]);
    __syncwarp();
    for (int e = lane; e < 32 * kOutUsed; e += 32) {
        const int r = e / kOutUsed, k = e % kOutUsed;
        if (base + r < n) out[(base + r) * kOutUsed + k] = s_res[warp][r * kResStride + k];
    }
}

// ---------------------------------------------------------------------------
// importance-sampled march, with the plain march as fallback
// ---------------------------------------------------------------------------
// The plain march of one ray (the same arithmetic as composite_kernel).
template <int ST, bool SHADE>
__device__ __forceinline__ void plain_ray(const MarchArgs &a, const float4 *s_tf, const Ray &R, float &C0, float &C1,
                                          float &C2, float &T, unsigned &evald) {
    C0 = C1 = C2 = 0.0f;
    T = 1.0f;
    int k = 0;
    while (k < R.nsamp) {
        float p[3];
        position_at(R, sample_t(R, k), p);
        Cell c;
        cell_of(a.vol, p, c);
        if (a.p.skip && !__ldg(a.occ + brick_of(a.vol, c))) {
            k = jump_empty(R, a.vol, c, k);
            continue;
        }
        float4 e = eval_sample<ST, SHADE>(a.vol, a.p, s_tf, a.tf.K, a.tf.ucoef, R.dir, c, a.p.rmode, a.p.ratio);
        composite_add(e, C0, C1, C2, T);
        evald++;
        k++;
        if ((1.0f - T) >= a.p.term) break;
    }
}

__device__ __forceinline__ bool occupied_at(const VolDev &v, const uint8_t *occ, const Ray &R, float t) {
    float p[3];
    position_at(R, t, p);
    Cell c;
    cell_of(v, p, c);
    return __ldg(occ + brick_of(v, c)) != 0;
}

// The PDF marks where the ray's contribution ends: b_end is one bin past the
// first bin >= b_start where its running sum reaches 1 - 1/64 (a margin for
// early predictions; at most 31, and 31 if never); b_start is the
// first bin whose start, centre or end lies in an occupied cell-brick (the
// whole chord when none does). nimp samples at the centres of nimp equal
// segments of [t_a, t_b] (start of bin b_start to end of bin b_end), each with
// its opacity corrected to the segment. FP32 operations as written.
template <int ST, bool SHADE>
__device__ __forceinline__ void importance_ray(const ImportanceArgs &A, const float4 *s_tf, const Ray &R,
                                               const float *pdf, float &C0, float &C1, float &C2, float &T,
                                               unsigned &evald) {
    const MarchArgs &a = A.m;
    const float bw = __fdiv_rn(__fsub_rn(R.tf, R.tn), (float)kBins);
    int b0 = -1, b1 = kBins - 1;
    for (int b = 0; b < kBins && b0 < 0; b++)
        if (occupied_at(a.vol, a.occ, R, __fmaf_rn((float)b, bw, R.tn)) ||
            occupied_at(a.vol, a.occ, R, __fmaf_rn((float)b + 0.5f, bw, R.tn)) ||
            occupied_at(a.vol, a.occ, R, __fmaf_rn((float)b + 1.0f, bw, R.tn)))
            b0 = b;
    if (b0 < 0) {
        b0 = 0;
    } else {
        float P = 0.0f;
        for (int b = 0; b < kBins; b++) {
            P = __fadd_rn(P, pdf[b]);
            if (b >= b0 && P >= 1.0f - 1.0f / 64.0f) {
                b1 = min(b + 1, kBins - 1);
                break;
            }
        }
    }
    const float ta = b0 == 0 ? R.tn : __fmaf_rn((float)b0, bw, R.tn);
    const float tb = b1 == kBins - 1 ? R.tf : __fmaf_rn((float)(b1 + 1), bw, R.tn);
    const float seg = __fdiv_rn(__fsub_rn(tb, ta), (float)A.nimp);
    const float ratio = __fdiv_rn(seg, a.vol.smin);
    C0 = C1 = C2 = 0.0f;
    T = 1.0f;
    for (int j = 0; j < A.nimp; j++) {
        float p[3];
        position_at(R, __fmaf_rn((float)j + 0.5f, seg, ta), p);
        Cell c;
        cell_of(a.vol, p, c);
        if (a.p.skip && !__ldg(a.occ + brick_of(a.vol, c))) continue;   // opacity exactly 0
        float4 e = eval_sample<ST, SHADE>(a.vol, a.p, s_tf, a.tf.K, a.tf.ucoef, R.dir, c, 3, ratio);
        composite_add(e, C0, C1, C2, T);
        evald++;
        if ((1.0f - T) >= a.p.term) break;
    }
}

template <int ST, bool SHADE, bool FUSED>
__global__ void __launch_bounds__(128) importance_kernel(const ImportanceArgs A) {
    const MarchArgs &a = A.m;
    extern __shared__ float4 smem[];
    float4 *s_tf = smem;
    float *s_res = reinterpret_cast<float *>(smem + a.tf.K);                   // 128 x 33
    __nv_bfloat16 *s_feat = reinterpret_cast<__nv_bfloat16 *>(s_res + 128 * kResStride);   // 4 x 32 x 120
    load_tf(a.tf, s_tf);
    int x, y;
    tile_pixel(x, y);
    const bool inimg = x < a.cam.W && y < a.cam.H;
    Ray R;
    const bool hit = inimg && setup_ray(a.cam, a.vol, a.p.step_vox, x, y, R);
    const size_t pix = (size_t)y * a.cam.W + x;
    float *mine = s_res + threadIdx.x * kResStride;
    if (FUSED) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __nv_bfloat16 *row = s_feat + (warp * 32 + lane) * kFeatStride;
        ray_features(a.vol, a.occ, R, hit, [&](int i, float v) { row[i] = __float2bfloat16_rn(v); });
        __syncwarp();
        warp_network(A.net, s_feat + warp * 32 * kFeatStride, s_res + warp * 32 * kResStride);
        __syncwarp();
    } else if (hit) {
        for (int b = 0; b < kBins; b++) mine[b] = A.pdf[pix * kBins + b];
        mine[kBins] = A.that[pix];
    }
    __syncthreads();
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
    unsigned evald = 0, fb = 0;
    if (hit) {
        importance_ray<ST, SHADE>(A, s_tf, R, mine, C0, C1, C2, T, evald);
        if (fabsf(T - mine[kBins]) > A.eps) {
            fb = 1;
            plain_ray<ST, SHADE>(a, s_tf, R, C0, C1, C2, T, evald);
        }
    }
    if (inimg) {
        a.out[pix] = make_float4(C0, C1, C2, 1.0f - T);
        if (A.fallback) A.fallback[pix] = (uint8_t)fb;
    }
    if (a.stats) {
        unsigned e = __reduce_add_sync(0xffffffffu, evald), f = __reduce_add_sync(0xffffffffu, fb);
        unsigned h = __reduce_add_sync(0xffffffffu, hit ? 1u : 0u), n = __reduce_add_sync(0xffffffffu, inimg ? 1u : 0u);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(a.stats + 0, (unsigned long long)f);     // fallback rays in the dense slot
            atomicAdd(a.stats + 1, (unsigned long long)e);
            atomicAdd(a.stats + 2, (unsigned long long)h);
            atomicAdd(a.stats + 3, (unsigned long long)n);
        }
    }
}

// ---------------------------------------------------------------------------
// training (SIMT FP32 with the inference's BF16 rounding points)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

constexpr int kTileRays = 32;
constexpr int kTrainThreads = 128;
constexpr int kTrainSmemFloats = kParams + kTileRays * (kFeat + 3 * kHid + kOut + 2 * kHid) + kTileRays;

// out[r][j] = act(bias[j] + sum_k in[r][k] * bf16(W[k][j])), rays r < 32.
template <int K, int N, bool RELU>
__device__ __forceinline__ void train_dense(const float *in, const float *__restrict__ W, const float *__restrict__ bias,
                                            float *out) {
    for (int o = threadIdx.x; o < kTileRays * N; o += kTrainThreads) {
        const int r = o / N, j = o % N;
        float acc = __ldg(bias + j);
        for (int k = 0; k < K; k++) acc = __fmaf_rn(in[r * K + k], bf16r(__ldg(W + k * N + j)), acc);
        out[r * N + j] = RELU ? bf16r(fmaxf(acc, 0.0f)) : acc;
    }
}

// g[W] += in^T dz, g[b] += sum_r dz (rays in order: deterministic)
template <int K, int N>
__device__ __forceinline__ void train_wgrad(const float *in, const float *dz, float *gW, float *gb) {
    for (int o = threadIdx.x; o < K * N; o += kTrainThreads) {
        const int k = o / N, j = o % N;
        float acc = 0.0f;
        for (int r = 0; r < kTileRays; r++) acc = __fmaf_rn(in[r * K + k], dz[r * N + j], acc);
        gW[o] += acc;
    }
    for (int j = threadIdx.x; j < N; j += kTrainThreads) {
        float acc = 0.0f;
        for (int r = 0; r < kTileRays; r++) acc += dz[r * N + j];
        gb[j] += acc;
    }
}

// dx[r][k] = (sum_j dz[r][j] bf16(W[k][j])) * [x[r][k] > 0]
template <int K, int N>
__device__ __forceinline__ void train_dgrad(const float *dz, const float *__restrict__ W, const float *x, float *dx) {
    for (int o = threadIdx.x; o < kTileRays * K; o += kTrainThreads) {
        const int r = o / K, k = o % K;
        float acc = 0.0f;
        for (int j = 0; j < N; j++) acc = __fmaf_rn(dz[r * N + j], bf16r(__ldg(W + k * N + j)), acc);
        dx[o] = x[o] > 0.0f ? acc : 0.0f;
    }
}

// Loss per ray: w KL(q || p) + (T^ - T)^2 with q = bins / sum(bins), w = sum(bins).
__global__ void __launch_bounds__(kTrainThreads) train_grad_kernel(const TrainArgs A) {
    extern __shared__ float sm[];
    float *g = sm;
    float *x = g + kParams;
    float *h1 = x + kTileRays * kFeat;
    float *h2 = h1 + kTileRays * kHid;
    float *h3 = h2 + kTileRays * kHid;
    float *z4 = h3 + kTileRays * kHid;
    float *dA = z4 + kTileRays * kOut;
    float *dB = dA + kTileRays * kHid;
    float *lossr = dB + kTileRays * kHid;
    const float *P = A.params;
    for (int i = threadIdx.x; i < kParams; i += kTrainThreads) g[i] = 0.0f;
    float block_loss = 0.0f;
    for (long long tile = blockIdx.x; tile * kTileRays < A.n; tile += gridDim.x) {
        const long long r0 = tile * kTileRays;
        __syncthreads();
        for (int e = threadIdx.x; e < kTileRays * kFeat; e += kTrainThreads) {
            const int r = e / kFeat;
            x[e] = r0 + r < A.n ? bf16r(A.feat[r0 * kFeat + e]) : 0.0f;
        }
        __syncthreads();
        train_dense<kFeat, kHid, true>(x, P + kOffW1, P + kOffB1, h1);
        __syncthreads();
        train_dense<kHid, kHid, true>(h1, P + kOffW2, P + kOffB2, h2);
        __syncthreads();
        train_dense<kHid, kHid, true>(h2, P + kOffW3, P + kOffB3, h3);
        __syncthreads();
        train_dense<kHid, kOut, false>(h3, P + kOffW4, P + kOffB4, z4);
        __syncthreads();
        if (threadIdx.x < kTileRays) {
            const int r = threadIdx.x;
            float *z = z4 + r * kOut;
            float loss = 0.0f;
            if (r0 + r < A.n) {
                const float *y = A.target + (r0 + r) * kOutUsed;
                float mx = -INFINITY, S = 0.0f;
                for (int b = 0; b < kBins; b++) {
                    mx = fmaxf(mx, z[b]);
                    S += y[b];
                }
                float se = 0.0f;
                for (int b = 0; b < kBins; b++) se += expf(z[b] - mx);
                const float lse = mx + logf(se);
                for (int b = 0; b < kBins; b++) {
                    const float p = expf(z[b] - lse);
                    float d = 0.0f;
                    if (S > 0.0f) {
                        const float q = y[b] / S;
                        d = S * (p - q);
                        if (q > 0.0f) loss += S * q * (logf(q) - (z[b] - lse));
                    }
                    z[b] = d * A.inv_n;
                }
                const float th = 1.0f / (1.0f + expf(-z[kBins]));
                const float dt = th - y[kBins];
                loss += dt * dt;
                z[kBins] = 2.0f * dt * th * (1.0f - th) * A.inv_n;
            } else {
                for (int b = 0; b <= kBins; b++) z[b] = 0.0f;
            }
            for (int b = kOutUsed; b < kOut; b++) z[b] = 0.0f;
            lossr[r] = loss;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int r = 0; r < kTileRays; r++) block_loss += lossr[r];
        // backward: z4 now holds dL/dz4
        train_wgrad<kHid, kOut>(h3, z4, g + kOffW4, g + kOffB4);
        train_dgrad<kHid, kOut>(z4, P + kOffW4, h3, dA);
        __syncthreads();
        train_wgrad<kHid, kHid>(h2, dA, g + kOffW3, g + kOffB3);
        train_dgrad<kHid, kHid>(dA, P + kOffW3, h2, dB);
        __syncthreads();
        train_wgrad<kHid, kHid>(h1, dB, g + kOffW2, g + kOffB2);
        train_dgrad<kHid, kHid>(dB, P + kOffW2, h1, dA);
        __syncthreads();
        train_wgrad<kFeat, kHid>(x, dA, g + kOffW1, g + kOffB1);
    }
    __syncthreads();
    float *part = A.partial + (size_t)blockIdx.x * kParams;
    for (int i = threadIdx.x; i < kParams; i += kTrainThreads) part[i] = g[i];
    if (threadIdx.x == 0) A.loss_partial[blockIdx.x] = block_loss;
}

__global__ void reduce_grad_kernel(const float *partial, const float *loss_partial, int nblocks, float inv_n,
                                   float *grad, float *loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kParams) {
        float s = 0.0f;
        for (int b = 0; b < nblocks; b++) s += partial[(size_t)b * kParams + i];
        grad[i] = s;
    }
    if (i == 0 && loss) {
        float s = 0.0f;
        for (int b = 0; b < nblocks; b++) s += loss_partial[b];
        *loss = s * inv_n;
    }
}

cudaError_t launch_train_grad(const TrainArgs &a, int grid, float *grad, float *loss, cudaStream_t s) {
    const size_t smem = (size_t)kTrainSmemFloats * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(train_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    train_grad_kernel<<<grid, kTrainThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_grad_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(a.partial, a.loss_partial, grid, a.inv_n, grad, loss);
    return cudaGetLastError();
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master parameters.
__global__ void adam_kernel(float *p, float *m, float *v, const float *g, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

cudaError_t launch_adam(float *params, float *m, float *v, const float *grad, long long step, float lr,
                        cudaStream_t s) {
    const float c1 = (float)(1.0 - pow(0.9, (double)step));
    const float c2 = (float)(1.0 - pow(0.999, (double)step));
    adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(params, m, v, grad, lr, c1, c2);
    return cudaGetLastError();
}

// BF16 B fragments: for k-tile i, n-tile j, lane (g, t): (W[16i+2t][8j+g],
// W[16i+2t+1][8j+g]) and (W[16i+2t+8][8j+g], W[16i+2t+9][8j+g]).
__global__ void pack_kernel(const float *params, uint2 *frag) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kFragTotal) return;
    int off, N, base;
    if (idx < kFragL2) { off = kOffW1; N = kHid; base = kFragL1; }
    else if (idx < kFragL3) { off = kOffW2; N = kHid; base = kFragL2; }
    else if (idx < kFragL4) { off = kOffW3; N = kHid; base = kFragL3; }
    else { off = kOffW4; N = kOut; base = kFragL4; }
    const int r = idx - base, lane = r & 31, tile = r >> 5, NT = N / 8;
    const int i = tile / NT, j = tile % NT, g = lane >> 2, t = lane & 3;
    const float *W = params + off;
    const int n = 8 * j + g, k0 = 16 * i + 2 * t;
    uint2 o;
    o.x = pack_bf16x2(W[k0 * N + n], W[(k0 + 1) * N + n]);
    o.y = pack_bf16x2(W[(k0 + 8) * N + n], W[(k0 + 9) * N + n]);
    frag[idx] = o;
}

cudaError_t launch_pack(const float *params, uint2 *frag, cudaStream_t s) {
    pack_kernel<<<(kFragTotal + 255) / 256, 256, 0, s>>>(params, frag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static dim3 image_grid(const CamRec &c) { return dim3((c.W + 15) / 16, (c.H + 7) / 8); }

cudaError_t launch_profiles(const MarchArgs &a, float *out, cudaStream_t s) {
    const size_t smem = (size_t)a.tf.K * sizeof(float4);
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<image_grid(a.cam), 128, smem, s>>>(a, out);
        return cudaGetLastError();
    };
    switch (a.vol.storage) {
        case RC_STORE_F32: return go(profiles_kernel<RC_STORE_F32>);
        case RC_STORE_F16: return go(profiles_kernel<RC_STORE_F16>);
        default: return go(profiles_kernel<RC_STORE_U16>);
    }
}

cudaError_t launch_features(const MarchArgs &a, float *out, cudaStream_t s) {
    features_kernel<<<image_grid(a.cam), 128, 0, s>>>(a, out);
    return cudaGetLastError();
}

cudaError_t launch_net_forward(const NetDev &net, const float *feat, long long n, float *out, cudaStream_t s) {
    const long long blocks = (n + 127) / 128;
    net_forward_kernel<<<(unsigned)blocks, 128, 0, s>>>(net, feat, n, out);
    return cudaGetLastError();
}

template <int ST, bool SHADE>
static cudaError_t launch_imp_st(const ImportanceArgs &a, cudaStream_t s) {
    const bool fused = a.pdf == nullptr;
    size_t smem = (size_t)a.m.tf.K * sizeof(float4) + 128 * kResStride * sizeof(float);
    if (fused) smem += 128 * kFeatStride * sizeof(__nv_bfloat16);
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<image_grid(a.m.cam), 128, smem, s>>>(a);
        return cudaGetLastError();
    };
    return fused ? go(importance_kernel<ST, SHADE, true>) : go(importance_kernel<ST, SHADE, false>);
}

cudaError_t launch_importance(const ImportanceArgs &a, cudaStream_t s) {
    switch (a.m.vol.storage * 2 + (a.m.p.shade ? 1 : 0)) {
        case RC_STORE_F32 * 2: return launch_imp_st<RC_STORE_F32, false>(a, s);
        case RC_STORE_F32 * 2 + 1: return launch_imp_st<RC_STORE_F32, true>(a, s);
        case RC_STORE_F16 * 2: return launch_imp_st<RC_STORE_F16, false>(a, s);
        case RC_STORE_F16 * 2 + 1: return launch_imp_st<RC_STORE_F16, true>(a, s);
        case RC_STORE_U16 * 2: return launch_imp_st<RC_STORE_U16, false>(a, s);
        default: return launch_imp_st<RC_STORE_U16, true>(a, s);
    }
}

}  // namespace rc
