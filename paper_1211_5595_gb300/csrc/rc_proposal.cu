// Learned sampling proposal: opacity profiles of the plain march (training
// targets), the per-ray feature encoder, a 112-64-64-64-40 BF16 network on the
// fifth-generation tensor cores (tcgen05 MMA, FP32 accumulators in tensor
// memory, one M = 128 tile of rays per CTA), its SIMT training kernels
// (deterministic gradient reduction, Adam), and the importance-sampled march
// with fallback to the plain march.
//
// The paper has no learned part: the proposal replaces the evenly spaced
// samples of Sec. 4.1 by 64 samples drawn where the network expects opacity,
// and keeps the compositing of Sec. 4.2 (Eq. 3-4) with each sample's opacity
// corrected to the length of the segment it stands for.
#include <cuda_bf16.h>

#include "rc_device.cuh"
#include "rc_tcgen05.cuh"

namespace rc {


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
            if (a.p.skip) {                                                   // opacity exactly 0
            const int b = brick_of(a.vol, c);
            if (a.fine ? empty_block(__ldg(a.fine + b), c) >= 0 : !__ldg(a.occ + b)) continue;
        }
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
// Emits the 112 features in 14 chunks of 8 (emit(chunk, v) in chunk order) and
// returns the occupancy bits at the bin centres as a mask (bit b = bin b).
// Feature order: 0-5 entry point and direction; 6 + 12c + 2j and 7 + 12c + 2j
// sin and cos of pi 2^j x_c; 78 + b occupancy of bin b's centre; 110-111 zero.
template <typename Emit>
__device__ __forceinline__ uint32_t ray_features(const VolDev &v, const uint8_t *occ, const Ray &R, bool hit,
                                                 Emit emit) {
    float buf[8];
    int fill = 0, chunk = 0;
    auto put = [&](float x) {
        buf[fill++] = x;
        if (fill == 8) {
            emit(chunk++, buf);
            fill = 0;
        }
    };
    if (!hit) {
#pragma unroll
        for (int i = 0; i < kFeat; i++) put(0.0f);
        return 0u;
    }
    float xs[6];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        xs[c] = __fdiv_rn(__fmaf_rn(R.tn, R.d[c], R.o[c]), (float)(v.n[c] - 1));
        xs[3 + c] = R.dir[c];
    }
#pragma unroll
    for (int c = 0; c < 6; c++) put(xs[c]);
    // sin and cos of pi 2^j x for j = 0 and 3 directly; j = 1, 2 and 4, 5 by
    // angle doubling, sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)(cos a + sin a)
    // (two doublings keep the error below 1e-6)
#pragma unroll
    for (int c = 0; c < 6; c++) {
        float s, co;
#pragma unroll
        for (int j = 0; j < 6; j++) {
            if (j == 0 || j == 3) {
                sincospif(ldexpf(xs[c], j), &s, &co);
            } else {
                const float s2 = 2.0f * s * co;
                co = (co - s) * (co + s);
                s = s2;
            }
            put(s);
            put(co);
        }
    }
    const float bw = __fdiv_rn(__fsub_rn(R.tf, R.tn), (float)kBins);
    uint32_t mask = 0;
#pragma unroll
    for (int b = 0; b < kBins; b++) {
        float p[3];
        position_at(R, __fmaf_rn((float)b + 0.5f, bw, R.tn), p);
        Cell c;
        cell_of(v, p, c);
        const bool o = __ldg(occ + brick_of(v, c)) != 0;
        mask |= (uint32_t)o << b;
        put(o ? 1.0f : 0.0f);
    }
    put(0.0f);
    put(0.0f);
    return mask;
}

__global__ void __launch_bounds__(128) features_kernel(const MarchArgs a, float *out) {
    int x, y;
    tile_pixel(x, y);
    if (x >= a.cam.W || y >= a.cam.H) return;
    Ray R;
    const bool hit = setup_ray(a.cam, a.vol, a.p.step_vox, x, y, R);
    float *o = out + ((size_t)y * a.cam.W + x) * kFeat;
    ray_features(a.vol, a.occ, R, hit, [&](int chunk, const float (&v)[8]) {
#pragma unroll
        for (int i = 0; i < 8; i++) o[8 * chunk + i] = v[i];
    });
}

// ---------------------------------------------------------------------------
// the network on the tensor cores: one M = 128 tile of rays per MMA
// ---------------------------------------------------------------------------
// A network CTA runs G independent groups of 128 threads, each on its own
// tiles of 128 rays with its own A operand, MMA barrier and 64 TMEM columns
// (TMEM lane = ray); the weights and biases are shared. The A operand holds a
// tile's features (128 x 112 BF16) and then, layer by layer, its hidden
// activations (128 x 64): every layer's MMA has completed before its output
// overwrites the operand it read. The camera-ray kernel runs one CTA of
// kCamGroups groups per SM (one copy of the weights, 209 KB of shared memory,
// 80 registers per thread; measured per 1024^2 view: 2 x 2 groups 0.146 ms,
// one CTA of 4 groups 0.149, of 5 groups 0.129, of 6 groups 0.121); the
// feature-matrix kernel two CTAs of kFeatGroups groups (its wide TMEM loads
// need more registers).
constexpr int kCamGroups = 6;
constexpr int kFeatGroups = 2;
constexpr int kGroupThreads = 128;
// TMEM columns of a CTA: 64 per group, allocated as a power of two
constexpr int tmem_cols(int groups) { return groups * 64 <= 128 ? 128 : groups * 64 <= 256 ? 256 : 512; }

template <int G>
struct NetSmem {
    uint8_t w[kUmmaBytes];                 // B operands of the four layers
    uint8_t a[G][128 * kFeat * 2];         // A operands
    float bias[3 * kHid + kN4];
    unsigned long long bar_w, bar_mma[G];
    uint32_t tmem;
};

struct NetLayer {
    unsigned b_off;                        // B operand offset in NetSmem::w
    int K, N;
};
__device__ __forceinline__ NetLayer net_layer(int l) {
    switch (l) {
        case 0: return NetLayer{kUmmaL1, kFeat, kHid};
        case 1: return NetLayer{kUmmaL2, kHid, kHid};
        case 2: return NetLayer{kUmmaL3, kHid, kHid};
        default: return NetLayer{kUmmaL4, kHid, kN4};
    }
}

// Barrier of one group (named barrier 1 + g, 128 threads); returns the AND of
// every thread's `ok`.
__device__ __forceinline__ bool group_sync_and(int g, bool ok) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)ok), "r"(1 + g), "r"(kGroupThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGroupThreads) : "memory");
}

// One layer, issued by one thread: D[128 x N] = A[128 x K] * W^T, K / 16 MMAs,
// then a commit that arrives on the group's MMA barrier when they are done.
template <int G>
__device__ __forceinline__ void issue_layer(const NetSmem<G> &S, int g, int l, uint32_t tmem_d, uint32_t bar) {
    const NetLayer L = net_layer(l);
    const uint32_t a0 = tc::smem_addr(S.a[g]), b0 = tc::smem_addr(S.w) + L.b_off;
    const uint32_t lbo_a = (128 / 8) * 128, lbo_b = (uint32_t)(L.N / 8) * 128;
    const uint32_t idesc = tc::idesc_bf16_f32(128, L.N);
    for (int ks = 0; ks < L.K / 16; ks++)
        tc::mma_bf16(tmem_d, tc::smem_desc(a0 + ks * 2 * lbo_a, lbo_a, 128),
                     tc::smem_desc(b0 + ks * 2 * lbo_b, lbo_b, 128), idesc, ks > 0);
    tc::commit(bar);
}

// Bias, ReLU and BF16 rounding of this thread's 64 hidden values, written as
// row `row` of the next layer's A operand (K = 64). Pairs of values: FP32x2
// bias add, one rounding to a BF16 pair, ReLU on the pair (max with +0 after
// rounding gives the same values as rounding after the ReLU).
__device__ __forceinline__ uint32_t bias_relu_bf16x2(float lo, float hi, float2 b) {
    uint64_t x, y, z;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(lo), "f"(hi));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    float zl, zh;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(zl), "=f"(zh) : "l"(z));
    uint32_t p, r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p) : "f"(zh), "f"(zl));
    asm("max.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(p), "r"(0u));
    return r;
}

// Bias, ReLU and BF16 rounding of 16 hidden values (columns c .. c + 15),
// stored as two 16-byte chunks of row `row` of the next A operand.
__device__ __forceinline__ void store_hidden16(uint8_t *A, const float *v, const float2 *b2, int c, int row) {
#pragma unroll
    for (int j = 0; j < 16; j += 8) {
        uint4 q;
        uint32_t *w = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
        for (int h = 0; h < 4; h++) w[h] = bias_relu_bf16x2(v[j + 2 * h], v[j + 2 * h + 1], b2[(c + j) / 2 + h]);
        *reinterpret_cast<uint4 *>(A + tc::core_offset(row, c + j, 128)) = q;
    }
}

// WIDE: the whole row in one TMEM load and wait (faster where the 64 live
// registers fit: the feature-matrix network and the training kernel); else
// four 16-column loads, each consumed before the next (the camera-ray
// network, at its register limit).
template <bool WIDE>
__device__ __forceinline__ void store_hidden(uint8_t *A, uint32_t taddr, const float *bias, int row) {
    const float2 *b2 = reinterpret_cast<const float2 *>(bias);
    if (WIDE) {
        float v[kHid];
        tc::tmem_ld64(taddr, v);
#pragma unroll
        for (int c = 0; c < kHid; c += 16) store_hidden16(A, v + c, b2, c, row);
    } else {
#pragma unroll
        for (int c = 0; c < kHid; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + c, v);
            store_hidden16(A, v, b2, c, row);
        }
    }
}

// Eight values as BF16 at (row, 8 * chunk .. 8 * chunk + 7) of an A operand:
// one 16-byte store (a warp's 32 rows fill 512 contiguous bytes).
__device__ __forceinline__ void store_chunk(uint8_t *A, int row, int chunk, const float (&v)[8]) {
    uint4 q;
    uint32_t *w = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
    for (int h = 0; h < 4; h++) {
        __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
        w[h] = *reinterpret_cast<uint32_t *>(&b2);
    }
    *reinterpret_cast<uint4 *>(A + tc::core_offset(row, 8 * chunk, 128)) = q;
}

// Network head: 32 logits -> PDF (softmax), logit 32 -> T^ (sigmoid).
template <bool WIDE>
__device__ __forceinline__ void net_head(uint32_t taddr, const float *bias, float (&pdf)[kBins], float &that) {
    // the head uses 33 of its 48 accumulator columns
    float z[kN4];
    if (WIDE) {
        float v[kHid];
        tc::tmem_ld64(taddr, v);
#pragma unroll
        for (int j = 0; j < kN4; j++) z[j] = v[j] + bias[j];
    } else {
#pragma unroll
        for (int c = 0; c < kN4; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + c, v);
#pragma unroll
            for (int j = 0; j < 16; j++) z[c + j] = v[j] + bias[c + j];
        }
    }
    float mx = z[0];
#pragma unroll
    for (int b = 1; b < kBins; b++) mx = fmaxf(mx, z[b]);
    // exponentials on the special-function unit (relative error ~2^-21,
    // far below the network's BF16 rounding)
    float sum = 0.0f;
#pragma unroll
    for (int b = 0; b < kBins; b++) {
        pdf[b] = __expf(z[b] - mx);
        sum += pdf[b];
    }
    const float inv = 1.0f / sum;
#pragma unroll
    for (int b = 0; b < kBins; b++) pdf[b] *= inv;
    that = 1.0f / (1.0f + __expf(-z[kBins]));
}

// Runs the four layers of group g on its A operand (the group's 128 threads
// call; thread t of the group is TMEM lane t). Returns false when a wait gave
// up; the caller then stops.
template <bool WIDE, int G>
__device__ __forceinline__ bool run_network(const TcNetArgs &A, NetSmem<G> &S, int g, uint32_t tmem, uint32_t bar,
                                            uint32_t &phase, float (&pdf)[kBins], float &that) {
    const int t = threadIdx.x - g * kGroupThreads;
    const uint32_t tmem_d = tmem + 64u * (uint32_t)g;
    const uint32_t taddr = tmem_d + ((uint32_t)(t & ~31) << 16);    // this warp's 32 lanes
#pragma unroll 1
    for (int l = 0; l < 4; l++) {
        tc::fence_async_smem();           // A written by ordinary stores -> visible to the MMA
        tc::fence_before();
        group_sync(g);
        tc::fence_after();
        if (t == 0 && A.issue_mma) issue_layer(S, g, l, tmem_d, bar);
        const bool ok = group_sync_and(g, tc::bar_wait(bar, phase, A.budget));
        if (!ok) return false;
        phase ^= 1u;
        tc::fence_after();
        if (l < 3) store_hidden<WIDE>(S.a[g], taddr, S.bias + l * kHid, t);
        else net_head<WIDE>(taddr, S.bias + 3 * kHid, pdf, that);
    }
    return true;
}

__device__ __forceinline__ void range_of(const MarchArgs &a, const Ray &R, const float (&pdf)[kBins], uint32_t centre,
                                         bool have_centre, int &b0, int &b1);

// FEAT: rays are rows of a feature matrix (outputs: the 33 network outputs);
// otherwise rays are the pixels of the cameras' views (outputs: the range
// record of each ray for the importance march).
template <bool FEAT, int G>
__global__ void __launch_bounds__(G * kGroupThreads) tc_net_kernel(const TcNetArgs A) {
    constexpr int kTmemCols = tmem_cols(G);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    NetSmem<G> &S = *reinterpret_cast<NetSmem<G> *>(smem_raw);
    const int tid = threadIdx.x, g = tid / kGroupThreads, t = tid % kGroupThreads;
    const int warp = t >> 5, lane = t & 31;
    const uint32_t bar_w = tc::smem_addr(&S.bar_w), bar_m = tc::smem_addr(&S.bar_mma[g]);
    if (tid < 32) tc::tmem_alloc<kTmemCols>(tc::smem_addr(&S.tmem));
    if (tid == 0) {
        tc::bar_init(bar_w, 1);
        for (int i = 0; i < G; i++) tc::bar_init(tc::smem_addr(&S.bar_mma[i]), 1);
    }
    for (int i = tid; i < 3 * kHid + kN4; i += blockDim.x) {
        const int l = i / kHid, j = i % kHid;
        float b = 0.0f;
        if (l < 3) b = A.net.params[(l == 0 ? kOffB1 : l == 1 ? kOffB2 : kOffB3) + j];
        else if (j < kOut) b = A.net.params[kOffB4 + j];
        S.bias[i] = b;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    if (tid == 0) tc::bulk_g2s(tc::smem_addr(S.w), A.net.umma, kUmmaBytes, bar_w);
    bool ok = __syncthreads_and(tc::bar_wait(bar_w, 0, A.budget));
    if (!ok) tc::bar_wait(bar_w, 0, A.budget);      // the weight copy may still be in flight
    uint32_t phase = 0;
    bool mma_waited_out = false;
    uint8_t *Ag = S.a[g];
    const long long stride = (long long)gridDim.x * G;
#pragma unroll 1
    for (long long tile = (long long)blockIdx.x * G + g; ok && tile < A.ntiles; tile += stride) {
        Ray R;
        bool hit = false;
        long long out_idx = -1;
        uint32_t centre = 0;
        if (FEAT) {
            // the tile's rows are one contiguous block of 128 x 112 floats:
            // coalesced float4 loads, each 4 features of one row -> 8 bytes
            // of BF16 in the A operand
            const long long r0 = tile * 128;
            const long long valid = min((long long)128, A.n - r0);
            const float4 *src = reinterpret_cast<const float4 *>(A.feat + r0 * kFeat);
#pragma unroll 7
            for (int i = 0; i < 128 * kFeat / 4 / kGroupThreads; i++) {
                const int e = i * kGroupThreads + t;          // float4 index within the tile
                const int row = e / (kFeat / 4), k = (e % (kFeat / 4)) * 4;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (row < valid) v = __ldg(src + e);
                __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
                uint2 q;
                q.x = *reinterpret_cast<uint32_t *>(&lo);
                q.y = *reinterpret_cast<uint32_t *>(&hi);
                *reinterpret_cast<uint2 *>(Ag + tc::core_offset(row, k, 128)) = q;
            }
        } else {
            const int per_view = A.tiles_x * A.tiles_y;
            const int view = (int)(tile / per_view), tl = (int)(tile % per_view);
            const CamRec &cam = A.m.cams[view];
            const int x = (tl % A.tiles_x) * 16 + (warp & 1) * 8 + (lane & 7);
            const int y = (tl / A.tiles_x) * 8 + (warp >> 1) * 4 + (lane >> 3);
            if (x < cam.W && y < cam.H) {
                hit = setup_ray(cam, A.m.vol, A.m.p.step_vox, x, y, R);
                out_idx = ((long long)view * cam.H + y) * cam.W + x;
            }
            // a tile none of whose rays meets the volume needs no network: the
            // importance march reads the records of rays that hit only (the
            // background around the volume: 61% of the tiles on a 1024^2 orbit
            // of the 256x256x180 phantom)
            if (group_sync_and(g, !hit)) continue;
            centre = ray_features(A.m.vol, A.m.occ, R, hit,
                                  [&](int chunk, const float (&v)[8]) { store_chunk(Ag, t, chunk, v); });
        }
        float pdf[kBins], that;
        ok = run_network<FEAT>(A, S, g, tmem, bar_m, phase, pdf, that);
        if (!ok) {
            mma_waited_out = true;
            break;
        }
        if (FEAT) {
            // stage the tile's 128 x 33 outputs in the A operand (its last
            // reader, the head layer's MMA, has completed), then store the
            // contiguous block with coalesced writes
            float *stage = reinterpret_cast<float *>(Ag);
#pragma unroll
            for (int b = 0; b < kBins; b++) stage[t * kOutUsed + b] = pdf[b];
            stage[t * kOutUsed + kBins] = that;
            group_sync(g);
            const long long r0 = tile * 128;
            const int valid = (int)min((long long)128, A.n - r0);
            float *o = A.net_out + r0 * kOutUsed;
            for (int e = t; e < valid * kOutUsed; e += kGroupThreads) o[e] = stage[e];
            group_sync(g);                  // before the next tile's features overwrite the stage
        } else if (out_idx >= 0) {
            if (A.pdf_out) {
                // the ray's PDF and T^ for the inverse-CDF march (32 + 1 floats)
                float4 *o = reinterpret_cast<float4 *>(A.pdf_out + out_idx * kBins);
#pragma unroll
                for (int b = 0; b < kBins; b += 4) o[b / 4] = make_float4(pdf[b], pdf[b + 1], pdf[b + 2], pdf[b + 3]);
                A.that_out[out_idx] = that;
            } else {
                int b0 = 0, b1 = kBins - 1;
                if (hit) range_of(A.m, R, pdf, centre, true, b0, b1);
                A.range[out_idx] = make_uint2((unsigned)b0 | ((unsigned)b1 << 8), __float_as_uint(that));
            }
        }
    }
    if (!ok) {
        if (t == 0) atomicOr(A.err, 1);
        if (mma_waited_out && A.issue_mma) tc::bar_wait(bar_m, phase, A.budget);   // MMAs may still be in flight
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_free<kTmemCols>(tmem);
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
        if (a.p.skip) {
            const int b = brick_of(a.vol, c);
            const int s = a.fine ? empty_block(__ldg(a.fine + b), c) : (__ldg(a.occ + b) ? -1 : 4);
            if (s >= 0) {
                k = jump_block(R, a.vol, c, k, s);
                continue;
            }
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
// whole chord when none does). FP32 operations as written.
__device__ __forceinline__ void range_of(const MarchArgs &a, const Ray &R, const float (&pdf)[kBins], uint32_t centre,
                                         bool have_centre, int &b0, int &b1) {
    const float bw = __fdiv_rn(__fsub_rn(R.tf, R.tn), (float)kBins);
    // bin b's start is boundary b, its end boundary b + 1 (both at
    // fma(k, bw, t_near)); its centre bit comes from the features when known
    b0 = -1;
    b1 = kBins - 1;
    bool start = occupied_at(a.vol, a.occ, R, R.tn);
    for (int b = 0; b < kBins && b0 < 0; b++) {
        const bool mid = have_centre ? ((centre >> b) & 1u) != 0
                                     : occupied_at(a.vol, a.occ, R, __fmaf_rn((float)b + 0.5f, bw, R.tn));
        if (start || mid) {
            b0 = b;
            break;
        }
        const bool end = occupied_at(a.vol, a.occ, R, __fmaf_rn((float)(b + 1), bw, R.tn));
        if (end) b0 = b;
        start = end;
    }
    if (b0 < 0) {
        b0 = 0;
        return;
    }
    float P = 0.0f;
    bool found = false;
#pragma unroll
    for (int b = 0; b < kBins; b++) {
        P = __fadd_rn(P, pdf[b]);
        if (!found && b >= b0 && P >= 1.0f - 1.0f / 64.0f) {
            b1 = min(b + 1, kBins - 1);
            found = true;
        }
    }
}

// nimp samples at the centres of nimp equal segments of [t_a, t_b] (start of
// bin b0 to end of bin b1), each with its opacity corrected to the segment.
// jump_block on the evenly spaced grid t_j = ta + (j + 0.5) seg, j < n, of a
// range march: the first sample index that may lie outside the empty block
// of 2^s cells around cell c (sample j is in it). The sample m just before
// the computed exit is verified to be in the same block, with its position
// computed exactly as the march computes it; positions are monotone in j
// along each axis, so every sample between j and m is in the block too.
// Falls back to j + 1 when the check fails.
__device__ __forceinline__ int jump_block_grid(const Ray &R, const VolDev &v, const Cell &c, int j, int s, float ta,
                                               float seg, int n) {
    const float INF = __int_as_float(0x7f800000);
    float texit = INF;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int lo = (c.i[a] >> s) << s, hi = lo + (1 << s);
        if (R.d[a] > 0.0f && hi <= v.n[a] - 2)
            texit = fminf(texit, __fdiv_rn((float)hi - R.o[a], R.d[a]));
        else if (R.d[a] < 0.0f && lo > 0)
            texit = fminf(texit, __fdiv_rn((float)lo - R.o[a], R.d[a]));
    }
    if (texit == INF) return n;
    const float fm = floorf(__fsub_rn(__fdiv_rn(texit - ta, seg), 0.5f));
    int m = fm >= (float)n ? n - 1 : (int)fm;
    if (m <= j) return j + 1;
#pragma unroll 1
    for (int tries = 0; tries < 2 && m > j; tries++, m--) {
        float p[3];
        position_at(R, __fmaf_rn((float)m + 0.5f, seg, ta), p);
        Cell cm;
        cell_of(v, p, cm);
        if (((cm.i[0] ^ c.i[0]) >> s) == 0 && ((cm.i[1] ^ c.i[1]) >> s) == 0 && ((cm.i[2] ^ c.i[2]) >> s) == 0)
            return m + 1;
    }
    return j + 1;
}

// JUMP: past an empty block in one step (jump_block_grid) instead of sample by
// sample; pays where a block spans several samples (measured on the bench
// orbit, ms per frame: 64 samples per ray 0.1735 -> 0.169, 128 samples
// 0.254 -> 0.228; 16 and 32 samples 3-4% slower, so chosen from 48 samples up)
template <int ST, bool SHADE, bool JUMP>
__device__ __forceinline__ void march_range(const ImportanceArgs &A, const float4 *s_tf, const Ray &R, int b0, int b1,
                                            float &C0, float &C1, float &C2, float &T, unsigned &evald) {
    const MarchArgs &a = A.m;
    const float bw = __fdiv_rn(__fsub_rn(R.tf, R.tn), (float)kBins);
    const float ta = b0 == 0 ? R.tn : __fmaf_rn((float)b0, bw, R.tn);
    const float tb = b1 == kBins - 1 ? R.tf : __fmaf_rn((float)(b1 + 1), bw, R.tn);
    const float seg = __fdiv_rn(__fsub_rn(tb, ta), (float)A.nimp);
    const float ratio = __fdiv_rn(seg, a.vol.smin);
    C0 = C1 = C2 = 0.0f;
    T = 1.0f;
    for (int j = 0; j < A.nimp;) {
        float p[3];
        position_at(R, __fmaf_rn((float)j + 0.5f, seg, ta), p);
        Cell c;
        cell_of(a.vol, p, c);
        if (a.p.skip) {          // opacity exactly 0: past the largest empty block around the sample
            const int b = brick_of(a.vol, c);
            const int s = a.fine ? empty_block(__ldg(a.fine + b), c) : (__ldg(a.occ + b) ? -1 : 4);
            if (s >= 0) {
                j = JUMP ? jump_block_grid(R, a.vol, c, j, s, ta, seg, A.nimp) : j + 1;
                continue;
            }
        }
        float4 e = eval_sample<ST, SHADE>(a.vol, a.p, s_tf, a.tf.K, a.tf.ucoef, R.dir, c, 3, ratio);
        composite_add(e, C0, C1, C2, T);
        evald++;
        j++;
        if ((1.0f - T) >= a.p.term) break;
    }
}

// Stratified inverse-CDF samples of the mixture q_b = (1 - lambda) pdf_b +
// lambda / 32 over the bins of the chord: sample j where the mixture's CDF
// reaches (j + 0.5) / nimp of its total, standing for the stretch between the
// midpoints to its neighbours (t_near and t_far at the ends), with its
// opacity corrected to that length. FP32 operations as written (the bin
// search continues from the previous sample's bin: the targets increase).
// pdf: the ray's 32 bins, or null for the uniform density (lambda = 1).
template <int ST, bool SHADE>
__device__ __forceinline__ void march_invcdf(const ImportanceArgs &A, const float4 *s_tf, const Ray &R,
                                             const float *pdf, float &C0, float &C1, float &C2, float &T,
                                             unsigned &evald) {
    const MarchArgs &a = A.m;
    const float bw = __fdiv_rn(__fsub_rn(R.tf, R.tn), (float)kBins);
    const float wp = __fsub_rn(1.0f, A.lambda), wu = __fdiv_rn(A.lambda, (float)kBins);
    auto qb = [&](int b) { return __fmaf_rn(wp, pdf ? __ldg(pdf + b) : 0.0f, wu); };
    float total = 0.0f;
#pragma unroll 8
    for (int b = 0; b < kBins; b++) total = __fadd_rn(total, qb(b));
    int b = 0;
    float Qb = 0.0f, q = qb(0);
    float Qn = __fadd_rn(Qb, q);
    auto position = [&](int j) {
        const float y = __fmul_rn(__fdiv_rn((float)j + 0.5f, (float)A.nimp), total);
        while (b < kBins - 1 && !(Qn > y)) {
            b++;
            Qb = Qn;
            q = qb(b);
            Qn = __fadd_rn(Qb, q);
        }
        float f = 0.0f;
        if (q > 0.0f) f = fminf(fmaxf(__fdiv_rn(__fsub_rn(y, Qb), q), 0.0f), 1.0f);
        return __fmaf_rn(__fadd_rn((float)b, f), bw, R.tn);
    };
    C0 = C1 = C2 = 0.0f;
    T = 1.0f;
    float tj = position(0), m = R.tn;
    for (int j = 0; j < A.nimp; j++) {
        const bool last = j + 1 == A.nimp;
        const float tn1 = last ? R.tf : position(j + 1);
        const float mn = last ? R.tf : __fmul_rn(__fadd_rn(tj, tn1), 0.5f);
        const float len = __fsub_rn(mn, m);
        float p[3];
        position_at(R, tj, p);
        Cell c;
        cell_of(a.vol, p, c);
        bool empty = false;
        if (a.p.skip) {                                                   // opacity exactly 0
            const int bb = brick_of(a.vol, c);
            empty = a.fine ? empty_block(__ldg(a.fine + bb), c) >= 0 : !__ldg(a.occ + bb);
        }
        if (!empty) {
            const float ratio = __fdiv_rn(len, a.vol.smin);
            float4 e = eval_sample<ST, SHADE>(a.vol, a.p, s_tf, a.tf.K, a.tf.ucoef, R.dir, c, 3, ratio);
            composite_add(e, C0, C1, C2, T);
            evald++;
            if ((1.0f - T) >= a.p.term) break;
        }
        m = mn;
        tj = tn1;
    }
}

__device__ __forceinline__ void importance_stats(const MarchArgs &a, unsigned evald, unsigned fb, bool hit,
                                                 bool inimg) {
    unsigned e = __reduce_add_sync(0xffffffffu, evald), f = __reduce_add_sync(0xffffffffu, fb);
    unsigned h = __reduce_add_sync(0xffffffffu, hit ? 1u : 0u), n = __reduce_add_sync(0xffffffffu, inimg ? 1u : 0u);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.stats + 0, (unsigned long long)f);     // fallback rays in the dense slot
        atomicAdd(a.stats + 1, (unsigned long long)e);
        atomicAdd(a.stats + 2, (unsigned long long)h);
        atomicAdd(a.stats + 3, (unsigned long long)n);
    }
}

// SRC = kSrcRecords: the sample range and T^ of each ray come from the
// network kernel's range records; kSrcRange: the range from the given per-ray
// PDF; kSrcInvCdf: inverse-CDF samples of the given PDF (or of the uniform
// density when A.pdf is null). Several views, grid.z = view, inputs
// view-major. Rays with |T_nimp - T^| > eps are re-marched by the plain march
// (never without a T^).
enum { kSrcRecords = 0, kSrcRange = 1, kSrcInvCdf = 2 };

template <int ST, bool SHADE, int SRC, bool JUMP = false>
__global__ void __launch_bounds__(128) importance_kernel(const ImportanceArgs A) {
    const MarchArgs &a = A.m;
    extern __shared__ float4 s_tf[];
    load_tf(a.tf, s_tf);
    __syncthreads();
    const CamRec cam = a.cams ? a.cams[blockIdx.z] : a.cam;
    const size_t view_off = (size_t)blockIdx.z * cam.W * cam.H;
    int x, y;
    tile_pixel(x, y);
    const bool inimg = x < cam.W && y < cam.H;
    Ray R;
    const bool hit = inimg && setup_ray(cam, a.vol, a.p.step_vox, x, y, R);
    const size_t pix = view_off + (size_t)y * cam.W + x;
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
    unsigned evald = 0, fb = 0;
    if (hit) {
        float that;
        bool check = true;
        if (SRC == kSrcInvCdf) {
            march_invcdf<ST, SHADE>(A, s_tf, R, A.pdf ? A.pdf + pix * kBins : nullptr, C0, C1, C2, T, evald);
            check = A.that != nullptr;
            that = check ? A.that[pix] : 0.0f;
        } else {
            int b0, b1;
            if (SRC == kSrcRecords) {
                const uint2 rec = A.range[pix];
                b0 = min((int)(rec.x & 255u), kBins - 1);
                b1 = min(max((int)((rec.x >> 8) & 255u), b0), kBins - 1);
                that = __uint_as_float(rec.y);
            } else {
                float pdf[kBins];
#pragma unroll
                for (int b = 0; b < kBins; b++) pdf[b] = A.pdf[pix * kBins + b];
                that = A.that[pix];
                range_of(a, R, pdf, 0u, false, b0, b1);
            }
            march_range<ST, SHADE, JUMP>(A, s_tf, R, b0, b1, C0, C1, C2, T, evald);
        }
        if (check && fabsf(T - that) > A.eps) {
            fb = 1;
            plain_ray<ST, SHADE>(a, s_tf, R, C0, C1, C2, T, evald);
        }
    }
    if (inimg) {
        a.out[pix] = make_float4(C0, C1, C2, 1.0f - T);
        if (A.fallback) A.fallback[pix] = (uint8_t)fb;
    }
    if (a.stats) importance_stats(a, evald, fb, hit, inimg);
}

// ---------------------------------------------------------------------------
// training on the tensor cores: forward as the inference, then per layer the
// weight gradient (rays as K, accumulated in TMEM over the CTA's tiles) and
// the input gradient (rays as M)
// ---------------------------------------------------------------------------
// Weight gradient of layer l: dW_l = H_{l-1}^T dZ_l over the tile's 128 rays,
// an M = 128, K = 128 MMA that reads both operands MN-major: A = H^T from H
// itself (rays x inputs, the forward's K-major operand, whose ones column
// gives the D row of the bias gradient sum_rays dZ, zero columns after it)
// and B = dZ^T from dZ (rays x outputs): no transposed copies. Input gradient:
// dH_{l-1} = dZ_l W_l^T, A = dZ (rays x outputs, K-major), B = W_l (inputs x
// outputs). All operands BF16 (dZ rounded once), FP32 accumulation. (Writing
// H^T and dZ^T as separate transposed operands took 1.062 ms per 1 M rays
// against 0.764 with the MN-major reads; the gradients are identical bit for
// bit.)
struct TrainSmem {
    uint8_t w[kUmmaAllBytes];              // forward and backward B operands
    uint8_t x[128 * 128 * 2];              // features (rays x 112), ones column 112, zero columns after it
    uint8_t h[3][128 * 128 * 2];           // H1..H3 (rays x 64), ones column 64, zero columns after it
    uint8_t adz[128 * kHid * 2];           // dZ (rays x outputs)
    float bias[3 * kHid + kN4];
    float wloss[4];
    unsigned long long bar_w, bar_m;
    uint32_t tmem;
};
constexpr int kTrainCols = 512;            // D (64) | dW4 (48) | dW3 | dW2 | dW1 (64 each)
constexpr uint32_t kColD = 0, kColW4 = 64, kColW3 = 128, kColW2 = 192, kColW1 = 256;

// D (+)= A B^T over K / 16 MMAs, A with `rows_a` rows, B with n rows.
__device__ __forceinline__ void issue_mma(uint32_t a0, int rows_a, uint32_t b0, int n, int K, uint32_t tmem_d,
                                          bool accumulate) {
    const uint32_t lbo_a = (uint32_t)(rows_a / 8) * 128, lbo_b = (uint32_t)(n / 8) * 128;
    const uint32_t idesc = tc::idesc_bf16_f32(128, n);
    for (int ks = 0; ks < K / 16; ks++)
        tc::mma_bf16(tmem_d, tc::smem_desc(a0 + ks * 2 * lbo_a, lbo_a, 128), tc::smem_desc(b0 + ks * 2 * lbo_b, lbo_b, 128),
                     idesc, accumulate || ks > 0);
}

// D (+)= A B^T over K = 128 rays with A and B read MN-major from operands
// stored rays x M and rays x N (core matrices of 8 rays x 8 elements; the
// K-adjacent cores 128 bytes apart, the M- or N-adjacent ones 2048): the
// weight gradient straight from the forward's operands.
__device__ __forceinline__ void issue_mma_mn(uint32_t a0, uint32_t b0, int n, uint32_t tmem_d, bool accumulate) {
    const uint32_t idesc = tc::idesc_bf16_f32(128, n) | tc::kIdescMnMajorA | tc::kIdescMnMajorB;
    for (int ks = 0; ks < 8; ks++)
        tc::mma_bf16(tmem_d, tc::smem_desc(a0 + ks * 256, 128, 2048), tc::smem_desc(b0 + ks * 256, 128, 2048), idesc,
                     accumulate || ks > 0);
}

// A bounded wait for the CTA's committed MMAs (all 128 threads).
__device__ __forceinline__ bool train_sync_mma(const TrainArgs &A, uint32_t bar, uint32_t &phase) {
    const bool ok = __syncthreads_and(tc::bar_wait(bar, phase, A.budget));
    if (ok) phase ^= 1u;
    tc::fence_after();
    return ok;
}

__device__ __forceinline__ void operands_ready() {
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// One BF16 value at (row, k) of a K-major operand with `rows` rows.
__device__ __forceinline__ void put_bf16(uint8_t *M, int row, int k, int rows, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(M + tc::core_offset(row, k, rows)) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ float get_bf16(const uint8_t *M, int row, int k, int rows) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(M + tc::core_offset(row, k, rows)));
}

// dZ of this thread's ray (n values, zeros up to k_pad) as row t of the dZ
// operand, 8 values per 16-byte store.
__device__ __forceinline__ void put_dz(TrainSmem &S, const float (&dz)[kHid], int n, int k_pad, int t) {
#pragma unroll
    for (int j0 = 0; j0 < kHid; j0 += 8) {
        if (j0 >= k_pad) break;
        uint4 q;
        uint32_t *w = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const float lo = j0 + 2 * h < n ? dz[j0 + 2 * h] : 0.0f, hi = j0 + 2 * h + 1 < n ? dz[j0 + 2 * h + 1] : 0.0f;
            __nv_bfloat162 b2 = __floats2bfloat162_rn(lo, hi);
            w[h] = *reinterpret_cast<uint32_t *>(&b2);
        }
        *reinterpret_cast<uint4 *>(S.adz + tc::core_offset(t, j0, 128)) = q;
    }
}

__global__ void __launch_bounds__(128) tc_train_kernel(const TrainArgs A) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t bar_w = tc::smem_addr(&S.bar_w), bar_m = tc::smem_addr(&S.bar_m);
    if (warp == 0) tc::tmem_alloc<kTrainCols>(tc::smem_addr(&S.tmem));
    if (t == 0) {
        tc::bar_init(bar_w, 1);
        tc::bar_init(bar_m, 1);
    }
    for (int i = t; i < 3 * kHid + kN4; i += blockDim.x) {
        const int l = i / kHid, j = i % kHid;
        float b = 0.0f;
        if (l < 3) b = A.params[(l == 0 ? kOffB1 : l == 1 ? kOffB2 : kOffB3) + j];
        else if (j < kOut) b = A.params[kOffB4 + j];
        S.bias[i] = b;
    }
    // features and hidden layers all zero, then their ones columns (constant:
    // the tiles rewrite the value columns only)
    for (int i = t; i < 4 * 128 * 128 * 2 / 16; i += blockDim.x) reinterpret_cast<uint4 *>(S.x)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    put_bf16(S.x, t, kFeat, 128, 1.0f);
    for (int l = 0; l < 3; l++) put_bf16(S.h[l], t, kHid, 128, 1.0f);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    if (t == 0) tc::bulk_g2s(tc::smem_addr(S.w), A.umma, kUmmaAllBytes, bar_w);
    bool ok = __syncthreads_and(tc::bar_wait(bar_w, 0, A.budget));
    if (!ok) tc::bar_wait(bar_w, 0, A.budget);
    uint32_t phase = 0;
    bool mma_waited_out = false, first = true;
    float loss_sum = 0.0f;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);      // this warp's lanes
    const long long ntiles = (A.n + 127) / 128;
#pragma unroll 1
    for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const long long r0 = tile * 128, r = r0 + t;
        const bool valid = r < A.n;
        // the CTA's next tile (features and targets) into L2
        const long long nt = tile + gridDim.x;
        if (t == 0 && nt < ntiles) {
            const long long nrows = min((long long)128, A.n - nt * 128);
            tc::prefetch_l2(A.feat + nt * 128 * kFeat, (uint32_t)(nrows * kFeat * sizeof(float)));
            tc::prefetch_l2(A.target + nt * 128 * kOutUsed, (uint32_t)((nrows * kOutUsed * sizeof(float)) & ~15ull));
        }
        // features: coalesced float4 loads of the contiguous tile -> BF16
        {
            const float4 *src = reinterpret_cast<const float4 *>(A.feat + r0 * kFeat);
            const long long nvalid = min((long long)128, A.n - r0);
#pragma unroll 7
            for (int i = 0; i < 128 * kFeat / 4 / 128; i++) {
                const int e = i * 128 + t, row = e / (kFeat / 4), k = (e % (kFeat / 4)) * 4;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (row < nvalid) v = __ldg(src + e);
                __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
                uint2 q;
                q.x = *reinterpret_cast<uint32_t *>(&lo);
                q.y = *reinterpret_cast<uint32_t *>(&hi);
                *reinterpret_cast<uint2 *>(S.x + tc::core_offset(row, k, 128)) = q;
            }
        }
        // forward: layers 1-3 into H1..H3, layer 4 -> logits
        float z[kN4];
#pragma unroll 1
        for (int l = 0; l < 4 && ok; l++) {
            operands_ready();
            const NetLayer L = net_layer(l);
            const uint8_t *Ain = l == 0 ? S.x : S.h[l - 1];
            if (t == 0 && A.issue_mma) {
                issue_mma(tc::smem_addr(Ain), 128, tc::smem_addr(S.w) + L.b_off, L.N, L.K, tmem + kColD, false);
                tc::commit(bar_m);
            }
            ok = train_sync_mma(A, bar_m, phase);
            if (!ok) {
                mma_waited_out = true;
                break;
            }
            if (l < 3) {
                store_hidden<true>(S.h[l], taddr + kColD, S.bias + l * kHid, t);
            } else {
                float v[64];
                tc::tmem_ld64(taddr + kColD, v);       // the 48 used of the 64 D columns, one round trip
#pragma unroll
                for (int j = 0; j < kN4; j++) z[j] = v[j] + S.bias[3 * kHid + j];
            }
        }
        if (!ok) break;
        // loss per ray: w KL(q || p) + (T^ - T)^2, q = bins / w, w = sum(bins);
        // dZ4 = dL/dz scaled by 1/n
        float dz[kHid];
        float loss = 0.0f;
#pragma unroll
        for (int j = 0; j < kN4; j++) dz[j] = 0.0f;
        if (valid) {
            const float *y = A.target + r * kOutUsed;
            float mx = z[0], W = 0.0f;
#pragma unroll
            for (int b = 0; b < kBins; b++) {
                mx = fmaxf(mx, z[b]);
                W += y[b];
            }
            float se = 0.0f;
#pragma unroll
            for (int b = 0; b < kBins; b++) se += expf(z[b] - mx);
            const float lse = mx + logf(se);
#pragma unroll
            for (int b = 0; b < kBins; b++) {
                const float p = expf(z[b] - lse);
                if (W > 0.0f) {
                    const float q = y[b] / W;
                    dz[b] = W * (p - q) * A.inv_n;
                    if (q > 0.0f) loss += W * q * (logf(q) - (z[b] - lse));
                }
            }
            const float th = 1.0f / (1.0f + expf(-z[kBins]));
            const float dt = th - y[kBins];
            loss += dt * dt;
            dz[kBins] = 2.0f * dt * th * (1.0f - th) * A.inv_n;
        }
        loss_sum += loss;
        // backward, layer 4 .. 1
#pragma unroll 1
        for (int l = 3; l >= 0 && ok; l--) {
            const int n_out = l == 3 ? kN4 : kHid;
            put_dz(S, dz, l == 3 ? kOut : kHid, n_out, t);
            operands_ready();
            const uint32_t wcol = l == 3 ? kColW4 : l == 2 ? kColW3 : l == 1 ? kColW2 : kColW1;
            if (t == 0 && A.issue_mma) {
                issue_mma_mn(tc::smem_addr(l == 0 ? S.x : S.h[l - 1]), tc::smem_addr(S.adz), n_out, tmem + wcol, !first);
                if (l > 0) {
                    const uint32_t bb = l == 3 ? kUmmaB4 : l == 2 ? kUmmaB3 : kUmmaB2;
                    issue_mma(tc::smem_addr(S.adz), 128, tc::smem_addr(S.w) + bb, kHid, n_out, tmem + kColD, false);
                }
                tc::commit(bar_m);
            }
            ok = train_sync_mma(A, bar_m, phase);
            if (!ok) {
                mma_waited_out = true;
                break;
            }
            if (l > 0) {
                // dZ_{l-1} = dH * [H_{l-1} > 0]
                float v[kHid];
                tc::tmem_ld64(taddr + kColD, v);
#pragma unroll
                for (int j = 0; j < kHid; j++) dz[j] = get_bf16(S.h[l - 1], t, j, 128) > 0.0f ? v[j] : 0.0f;
            }
        }
        first = false;
    }
    if (!ok) {
        if (t == 0) atomicOr(A.err, 1);
        if (mma_waited_out && A.issue_mma) tc::bar_wait(bar_m, phase, A.budget);
    }
    // the CTA's gradient: lane = input row (or the bias at row n_in), column = output
    float *part = A.partial + (size_t)blockIdx.x * kParams;
    const int row = warp * 32 + lane;
#pragma unroll 1
    for (int l = 0; l < 4; l++) {
        const int n_in = l == 0 ? kFeat : kHid, n_out = l == 3 ? kOut : kHid, n_cols = l == 3 ? kN4 : kHid;
        const uint32_t wcol = l == 3 ? kColW4 : l == 2 ? kColW3 : l == 1 ? kColW2 : kColW1;
        const int offW = l == 0 ? kOffW1 : l == 1 ? kOffW2 : l == 2 ? kOffW3 : kOffW4;
        const int offB = l == 0 ? kOffB1 : l == 1 ? kOffB2 : l == 2 ? kOffB3 : kOffB4;
        for (int c = 0; c < n_cols; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + wcol + c, v);
            for (int j = 0; j < 16 && c + j < n_out; j++) {
                const float g = (first || !ok) ? 0.0f : v[j];
                if (row < n_in) part[offW + row * n_out + c + j] = g;
                else if (row == n_in) part[offB + c + j] = g;
            }
        }
    }
    // loss: per-warp sums in a fixed order, then the CTA's
    for (int o = 16; o > 0; o >>= 1) loss_sum += __shfl_xor_sync(0xffffffffu, loss_sum, o);
    if (lane == 0) S.wloss[warp] = loss_sum;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (t == 0) A.loss_partial[blockIdx.x] = ((S.wloss[0] + S.wloss[1]) + S.wloss[2]) + S.wloss[3];
    if (warp == 0) tc::tmem_free<kTrainCols>(tmem);
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

int train_grid(long long n) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (n + 127) / 128;
    return (int)max(1ll, min((long long)sms, tiles));
}

cudaError_t launch_train_grad(const TrainArgs &a, int grid, float *grad, float *loss, cudaStream_t s) {
    const int smem = (int)sizeof(TrainSmem);
    cudaError_t e = cudaFuncSetAttribute(tc_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc_train_kernel<<<grid, 128, smem, s>>>(a);
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

// B operands of the four layers in the core-matrix layout: element (n, k) of
// layer l is bf16(W_l[k][n]) (0 for the padding rows n >= 40 of layer 4).
__global__ void pack_umma_kernel(const float *params, uint8_t *umma) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int n1 = kHid * kFeat, n2 = kHid * kHid, n4 = kN4 * kHid;
    if (idx >= n1 + 2 * n2 + n4) return;
    int r, K, N, nw, woff;
    unsigned boff;
    if (idx < n1) { r = idx; K = kFeat; N = kHid; nw = kHid; woff = kOffW1; boff = kUmmaL1; }
    else if (idx < n1 + n2) { r = idx - n1; K = kHid; N = kHid; nw = kHid; woff = kOffW2; boff = kUmmaL2; }
    else if (idx < n1 + 2 * n2) { r = idx - n1 - n2; K = kHid; N = kHid; nw = kHid; woff = kOffW3; boff = kUmmaL3; }
    else { r = idx - n1 - 2 * n2; K = kHid; N = kN4; nw = kOut; woff = kOffW4; boff = kUmmaL4; }
    const int n = r / K, k = r % K;
    const float w = n < nw ? params[woff + k * nw + n] : 0.0f;
    *reinterpret_cast<__nv_bfloat16 *>(umma + boff + tc::core_offset(n, k, N)) = __float2bfloat16_rn(w);
}

// B operands of the training backward: element (n, k) of layer l is
// bf16(W_l[n][k]) (inputs x outputs, as stored; 0 for the padding outputs
// k >= 40 of layer 4).
__global__ void pack_umma_back_kernel(const float *params, uint8_t *umma) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int n4 = kHid * kN4, n3 = kHid * kHid;
    if (idx >= n4 + 2 * n3) return;
    int r, K, nw, woff;
    unsigned boff;
    if (idx < n4) { r = idx; K = kN4; nw = kOut; woff = kOffW4; boff = kUmmaB4; }
    else if (idx < n4 + n3) { r = idx - n4; K = kHid; nw = kHid; woff = kOffW3; boff = kUmmaB3; }
    else { r = idx - n4 - n3; K = kHid; nw = kHid; woff = kOffW2; boff = kUmmaB2; }
    const int n = r / K, k = r % K;
    const float w = k < nw ? params[woff + n * nw + k] : 0.0f;
    *reinterpret_cast<__nv_bfloat16 *>(umma + boff + tc::core_offset(n, k, kHid)) = __float2bfloat16_rn(w);
}

cudaError_t launch_pack(const float *params, uint8_t *umma, cudaStream_t s) {
    constexpr int total = kHid * kFeat + 2 * kHid * kHid + kN4 * kHid;
    pack_umma_kernel<<<(total + 255) / 256, 256, 0, s>>>(params, umma);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr int back = kHid * kN4 + 2 * kHid * kHid;
    pack_umma_back_kernel<<<(back + 255) / 256, 256, 0, s>>>(params, umma);
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

// Persistent network CTAs: as many as fit on the device at once (shared
// memory, registers and the SM's 512 TMEM columns), at most one per G tiles.
template <bool FEAT, int G>
static cudaError_t launch_tc(const TcNetArgs &a, cudaStream_t s) {
    constexpr int kTmemCols = tmem_cols(G);
    auto kern = tc_net_kernel<FEAT, G>;
    const int smem = (int)sizeof(NetSmem<G>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
    // CTAs per SM from the SM's shared memory and registers (the occupancy
    // query does not see the carveout preference and answers 1), at most as
    // many as the 512 TMEM columns hold
    int dev = 0, sms = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    const int threads = G * kGroupThreads;
    const int by_smem = smem_sm / (smem + smem_rsv);
    const int by_regs = regs_sm / max(1, fa.numRegs * threads);
    const int per_sm = max(1, min(min(by_smem, by_regs), 512 / kTmemCols));
    const long long grid = min((long long)sms * per_sm, (a.ntiles + G - 1) / G);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc_net(const TcNetArgs &a, cudaStream_t s) {
    return a.feat ? launch_tc<true, kFeatGroups>(a, s) : launch_tc<false, kCamGroups>(a, s);
}

template <int ST, bool SHADE>
static cudaError_t launch_imp_st(const ImportanceArgs &a, int nviews, cudaStream_t s) {
    const size_t smem = (size_t)a.m.tf.K * sizeof(float4);
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        dim3 grid = image_grid(a.m.cam);
        grid.z = nviews;
        kern<<<grid, 128, smem, s>>>(a);
        return cudaGetLastError();
    };
    // the range marches jump empty blocks from 48 samples per ray up
    const bool jump = a.nimp >= 48;
    if (a.range)
        return jump ? go(importance_kernel<ST, SHADE, kSrcRecords, true>) : go(importance_kernel<ST, SHADE, kSrcRecords>);
    if (a.sampling == RC_SAMPLING_INVCDF) return go(importance_kernel<ST, SHADE, kSrcInvCdf>);
    return jump ? go(importance_kernel<ST, SHADE, kSrcRange, true>) : go(importance_kernel<ST, SHADE, kSrcRange>);
}

cudaError_t launch_importance(const ImportanceArgs &a, int nviews, cudaStream_t s) {
    switch (a.m.vol.storage * 2 + (a.m.p.shade ? 1 : 0)) {
        case RC_STORE_F32 * 2: return launch_imp_st<RC_STORE_F32, false>(a, nviews, s);
        case RC_STORE_F32 * 2 + 1: return launch_imp_st<RC_STORE_F32, true>(a, nviews, s);
        case RC_STORE_F16 * 2: return launch_imp_st<RC_STORE_F16, false>(a, nviews, s);
        case RC_STORE_F16 * 2 + 1: return launch_imp_st<RC_STORE_F16, true>(a, nviews, s);
        case RC_STORE_U16 * 2: return launch_imp_st<RC_STORE_U16, false>(a, nviews, s);
        default: return launch_imp_st<RC_STORE_U16, true>(a, nviews, s);
    }
}

}  // namespace rc
