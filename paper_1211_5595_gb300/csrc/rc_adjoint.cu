// Adjoint of the compositing ray function with respect to the transfer-function
// table (Eq. 4-5 are differentiable in the table entries).
//
// Per ray, pass 1 recomputes the forward march (with exact empty-space
// skipping) to get C_final, T_final and the number n of samples up to
// termination; when the caller gives the forward images, C_final and T_final
// are read from them instead and pass 2 stops at the termination sample by
// itself (it rebuilds T sample by sample, and the skipped samples of the
// forward have zero opacity, so its stop decisions are the forward's). Pass 2
// marches again front to back, rebuilding T_k and the prefix C_{<=k}, so that
// the suffix S_k = C_final - C_{<=k} is known without storing samples or
// dividing transmittance backwards:
//   dI_c/da'_k = T_k col_kc - S_kc / (1 - a'_k),  dI_a/da'_k = T_k - (T_{k+1} - T_n) / (1 - a'_k)
//   dI_c/dcol_kc = T_k a'_k,  da'/da = r (1 - min(a, 1 - 1e-6))^(r - 1)
// and the two table entries of the sample's lerp receive weights (1 - w, w).
// Lanes of a warp that hit the same entries are summed first (a fixed tree
// order). A 1-D table of at most kWarpAccK entries then keeps one FP32 copy
// per warp in shared memory, which only that warp's group leaders update, in
// its own program order; at the end each CTA adds its warps' copies in warp
// order and converts the sums to 64-bit fixed point (scale 2^32 / max|dL/dI|)
// for the global sums. Larger tables add each group's sums as 64-bit fixed
// point to the CTA's shared accumulators directly. Integer sums do not depend
// on the order of the atomics, and no other sum depends on thread scheduling,
// so the result is deterministic.
#include "rc_device.cuh"

namespace rc {

__global__ void absmax_kernel(const float *__restrict__ x, long long n, unsigned *out) {
    float m = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    unsigned u = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if ((threadIdx.x & 31) == 0) atomicMax(out, u);
}

cudaError_t launch_absmax(const float *x, long long n, float *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    absmax_kernel<<<1216, 256, 0, s>>>(x, n, (unsigned *)out);
    return cudaGetLastError();
}

__device__ __forceinline__ float fixed_scale(const float *absmax) {
    return 4294967296.0f / fmaxf(*absmax, 1e-30f);
}

__device__ __forceinline__ void acc_add(unsigned long long *acc, int idx, float v, float scale) {
    long long q = __float2ll_rn(v * scale);
    if (q != 0) atomicAdd(acc + idx, (unsigned long long)q);
}

// 1-D tables of up to this many entries take the per-warp FP32 accumulators
// (16 B per entry and warp; with the FP32 table 80 B per entry and CTA: 40 KB
// at 512 entries). Measured on the 128x128x96 workload (256 entries, 8 views
// at 512^2, ms per view given the forward images): 0.231 with the CTA's 64-bit
// fixed-point atomics, 0.151 per warp: no conversion and no atomic per group.
constexpr int kWarpAccK = 512;
constexpr int kAdjWarps = 4;                     // warps of a 1-D table's CTA

// Whether a 1-D table's gradient takes the per-warp accumulators: up to
// kWarpAccK entries, except with the cubic B-spline when the forward is
// recomputed: that march's 64-voxel gathers need the L1 capacity the larger
// shared-memory footprint takes (same workload, B-spline, ms per view:
// recomputing 0.529 with the CTA's accumulators, 0.575 per warp; given the
// forward images 0.340 and 0.315).
__host__ __device__ constexpr bool warp_acc(int K, bool tf2, bool cubic, bool given) {
    return !tf2 && K <= kWarpAccK && (!cubic || given);
}

// 2-D table accumulators: the table's M x K x 4 fixed-point sums live in
// global memory (they do not fit in shared memory), fronted per CTA by a
// direct-mapped cache of kSlots entries in shared memory (72 KB). A slot is
// claimed by the first entry that maps to it (compare-and-swap on its tag)
// and keeps it for the CTA's lifetime; an entry whose slot another entry
// holds adds to global memory directly. The cache absorbs the repeated adds of
// the CTA's hot entries (air, homogeneous tissue) that would otherwise
// serialise on a few global addresses. Integer sums: the result depends
// neither on which path an add takes nor on the order. (Measured on the
// 128x128x96 workload with a 32 x 256 table, ms per view: no cache 6.1; with
// 4-warp CTAs 1024 slots 1.50, 2048 slots 1.41, 4096 slots 3.34 as one CTA
// per SM is left, linear probing over 2-8 slots slower than one; 2048 slots
// shared by 8 warps 1.05, by 16 warps 1.03.)
constexpr int kSlotBits = 11;
constexpr int kSlots = 1 << kSlotBits;
// CTA of a 2-D table's instance: kWarps2D warps (16 x 2 kWarps2D pixels)
// share the one slot cache, so that the 72 KB per CTA leave room for more
// resident warps.
constexpr int kWarps2D = 8;

__device__ __forceinline__ void cache_add4(unsigned long long *s_val, int *s_tag, unsigned long long *g_acc, int e,
                                           const float *v, float scale) {
    const int slot = (int)(((unsigned)e * 2654435761u) >> (32 - kSlotBits));
    int t = *reinterpret_cast<volatile int *>(s_tag + slot);
    if (t == -1) {
        t = atomicCAS(s_tag + slot, -1, e);
        if (t == -1) t = e;                    // claimed here
    }
    // two explicit paths, so that each add is a shared- or a global-memory
    // atomic rather than a generic one
    if (t == e) {
#pragma unroll
        for (int c = 0; c < 4; c++) acc_add(s_val, 4 * slot + c, v[c], scale);
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++) acc_add(g_acc + 4 * (size_t)e, c, v[c], scale);
    }
}

// Sum of v (N values) over the lanes of this lane's group (lanes with the same key), in a
// fixed pairwise-tree order over the group's lanes sorted by lane id; the sum
// ends in the group's lowest lane (rank 0). Deterministic for a given key set.
template <int N>
__device__ __forceinline__ void group_sum(unsigned peers, float (&v)[N]) {
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(peers);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    // the lane of rank + s, by pointer jumping: first the next member above
    // this lane (or this lane itself when there is none)
    const unsigned above = peers & ~((2u << lane) - 1u);
    int nxt = above ? __ffs(above) - 1 : lane;
#pragma unroll 1
    for (int s = 1; __any_sync(0xffffffffu, s < cnt); s <<= 1) {
        const bool take = (rank % (2 * s)) == 0 && rank + s < cnt;
        const int src = take ? nxt : lane;
#pragma unroll
        for (int c = 0; c < N; c++) {
            const float o = __shfl_sync(0xffffffffu, v[c], src);
            if (take) v[c] += o;
        }
        nxt = __shfl_sync(0xffffffffu, nxt, nxt);          // rank + 2s
    }
}

// d a' / d a = r (1 - a)^(r - 1) for the step ratio r of mode RM, with
// x = 1 - a >= 1e-6: r = 1/2 and 1/4 as reciprocal square roots, else
// through log2 / exp2.
template <int RM>
__device__ __forceinline__ float dalpha_factor(float x, float ratio, int rmode) {
    const int m = RM >= 0 ? RM : rmode;
    if (m == 1) return 0.5f * rsqrtf(x);
    if (m == 2) {
        const float q = rsqrtf(x);
        return 0.25f * q * sqrtf(q);
    }
    return ratio * exp2f((ratio - 1.0f) * __log2f(x));
}

// CUBIC: cubic B-spline reconstruction (value and analytic gradient) instead
// of trilinear values and central differences; the table scatter is the same.
// TF2: a 2-D table over (value, gradient magnitude) in global memory; each
// sample scatters into the four entries of its bilinear cell, and the group
// leaders add through the CTA's slot cache to the global fixed-point
// accumulators (the M x K table's accumulators do not fit in shared memory).
template <int ST, bool SHADE, int RM, bool CUBIC, bool TF2>
__global__ void __launch_bounds__(TF2 ? 32 * kWarps2D : 32 * kAdjWarps) adjoint_kernel(const AdjointArgs A, const float *absmax) {
    const MarchArgs &a = A.m;
    const int K = a.tf.K;
    constexpr bool GRAD = SHADE || TF2;
    constexpr int NV = TF2 ? 16 : 8;                  // contributions per sample
    const bool wacc = warp_acc(K, TF2, CUBIC, A.fimg != nullptr);   // per-warp FP32 accumulators
    extern __shared__ float4 smem[];
    float4 *s_tf = smem;
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(smem + (TF2 ? 0 : K));
    float4 *s_wacc = smem + K;                        // [warp][entry], 1-D tables of <= kWarpAccK entries
    int *s_tag = reinterpret_cast<int *>(s_acc + 4 * kSlots);          // 2-D table only
    if (!TF2) {
        load_tf(a.tf, s_tf);
        if (wacc) {
            for (int e = threadIdx.x; e < kAdjWarps * K; e += blockDim.x) s_wacc[e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else {
            for (int e = threadIdx.x; e < 4 * K; e += blockDim.x) s_acc[e] = 0ull;
        }
    } else {
        for (int e = threadIdx.x; e < 4 * kSlots; e += blockDim.x) s_acc[e] = 0ull;
        for (int e = threadIdx.x; e < kSlots; e += blockDim.x) s_tag[e] = -1;
    }
    __syncthreads();
    const float scale = fixed_scale(absmax);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const CamRec cam = a.cams ? a.cams[blockIdx.z] : a.cam;
    const int x = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int y = blockIdx.y * (TF2 ? 2 * kWarps2D : 8) + (warp >> 1) * 4 + (lane >> 3);
    const bool inimg = x < cam.W && y < cam.H;
    Ray R;
    bool hit = inimg && setup_ray(cam, a.vol, a.p.step_vox, x, y, R);
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (hit) g = A.dimg[((size_t)blockIdx.z * cam.H + y) * cam.W + x];
    const bool has_g = hit && (g.x != 0.0f || g.y != 0.0f || g.z != 0.0f || g.w != 0.0f);
    // pass 1: the forward march, with exact empty-space skipping over empty
    // bricks, octants and 4^3 sub-blocks (identical result), for C_final,
    // T_final and the sample count n up to termination
    float Cf0 = 0.0f, Cf1 = 0.0f, Cf2 = 0.0f, Tf = 1.0f;
    int n = 0;
    const bool given = A.fimg != nullptr;
    if (given) {
        if (has_g) {
            const float4 f = A.fimg[((size_t)blockIdx.z * cam.H + y) * cam.W + x];
            Cf0 = f.x;
            Cf1 = f.y;
            Cf2 = f.z;
            Tf = 1.0f - f.w;
            n = R.nsamp;
        }
    } else if (has_g) {
        int k = 0;
        while (k < R.nsamp) {
            float p[3];
            position_at(R, sample_t(R, k), p);
            Cell c;
            cell_of(a.vol, p, c);
            const int b = brick_of(a.vol, c);
            const int s = a.fine ? empty_block(__ldg(a.fine + b), c) : (__ldg(a.occ + b) ? -1 : 4);
            if (s >= 0) {
                k = jump_block(R, a.vol, c, k, s);
                continue;
            }
            float4 e = eval_sample_x<ST, (SHADE ? kShade : 0) | (CUBIC ? kCubic : 0) | (TF2 ? kTF2 : 0), RM>(
                a.vol, a.p, s_tf, a.tf,
                                                                                          R.dir, c, a.p.rmode,
                                                               a.p.ratio);
            composite_add(e, Cf0, Cf1, Cf2, Tf);
            k++;
            if ((1.0f - Tf) >= a.p.term) break;
        }
        n = min(k, R.nsamp);
    }
    // pass 2: every sample again (an empty brick still has a gradient), the
    // prefix C_{<=k} rebuilt, one gradient contribution per sample; lanes that
    // hit the same table entries are summed first, then the group's leader
    // adds the sums to its warp's FP32 copy (or, for a large table, one 64-bit
    // fixed-point atomic per entry and channel)
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
    for (int k = 0; __any_sync(0xffffffffu, k < n); k++) {
        const bool active = k < n;
        int i = -1;
        float v[NV];
#pragma unroll
        for (int c = 0; c < NV; c++) v[c] = 0.0f;
        if (active) {
            float p[3], gr[3], val;
            position_at(R, sample_t(R, k), p);
            Cell c;
            cell_of(a.vol, p, c);
            if (CUBIC) val = GRAD ? bspline_grad<ST>(a.vol, c, gr) : bspline<ST>(a.vol, c);
            else val = GRAD ? value_grad<ST>(a.vol, c, gr) : trilinear<ST>(a.vol, c);
            float w, wb = 0.0f;
            float4 e;
            if (TF2) {
                int j;
                e = classify2_at(a.tf, tf_coord<ST>(val, a.tf.ucoef), tf2_row_coord(a.tf, gr), i, j, w, wb,
                                 RC_DBG_ERR(a.vol));
                i += j * K;                           // entry (i, j) of the M x K table
            } else {
                e = classify(s_tf, K, tf_coord<ST>(val, a.tf.ucoef), &i, &w, RC_DBG_ERR(a.vol));
            }
            float ap = correct_alpha<RM>(e.w, a.p.rmode, a.p.ratio);
            float r = e.x, gg = e.y, b = e.z;
            float d0 = 1.0f, d1 = 1.0f, d2 = 1.0f;
            if (SHADE) {
                float sf, spec;
                shade_factor(a.p, a.vol, gr, R.dir, sf, spec);
                float u0 = __fmaf_rn(r, sf, spec), u1 = __fmaf_rn(gg, sf, spec), u2 = __fmaf_rn(b, sf, spec);
                d0 = u0 < 1.0f ? sf : 0.0f;
                d1 = u1 < 1.0f ? sf : 0.0f;
                d2 = u2 < 1.0f ? sf : 0.0f;
                r = fminf(1.0f, u0);
                gg = fminf(1.0f, u1);
                b = fminf(1.0f, u2);
            }
            const float Tk = T;
            float ta = T * ap;
            C0 = __fmaf_rn(ta, r, C0);
            C1 = __fmaf_rn(ta, gg, C1);
            C2 = __fmaf_rn(ta, b, C2);
            T = T * (1.0f - ap);
            if (given && (1.0f - T) >= a.p.term) n = k + 1;        // the forward stopped after this sample
            const float om = 1.0f - ap;
            const float inv = om > 0.0f ? 1.0f / om : 0.0f;
            float dap = g.x * (Tk * r - (Cf0 - C0) * inv) + g.y * (Tk * gg - (Cf1 - C1) * inv) +
                        g.z * (Tk * b - (Cf2 - C2) * inv) + g.w * (Tk - (T - Tf) * inv);
            float ac = fminf(e.w, 1.0f - 1e-6f);
            const int m = RM >= 0 ? RM : a.p.rmode;
            const float dal = m == 0 ? dap : dap * dalpha_factor<RM>(1.0f - ac, a.p.ratio, m);
            float dr = g.x * ta * d0, dg = g.y * ta * d1, db = g.z * ta * d2;
            // bilinear weights of the cell's entries: (i, j), (i + 1, j), then
            // the next row (i, j + 1), (i + 1, j + 1) for a 2-D table
            const float w0 = 1.0f - w;
            const float wr[4] = {w0 * (1.0f - wb), w * (1.0f - wb), w0 * wb, w * wb};
#pragma unroll
            for (int q = 0; q < NV / 4; q++) {
                v[4 * q + 0] = wr[q] * dr;
                v[4 * q + 1] = wr[q] * dg;
                v[4 * q + 2] = wr[q] * db;
                v[4 * q + 3] = wr[q] * dal;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, active ? i : -1 - lane);
        group_sum<NV>(peers, v);
        const bool leader = active && (peers & ((1u << lane) - 1u)) == 0u;
        if (wacc) {
            // the leaders hold distinct entries i, but the i + 1 of one group
            // may be the i of another: entry i first, then (after the warp
            // barrier) entry i + 1, each a plain read-modify-write of a slot
            // no other leader touches in that phase. The barrier before the
            // first phase orders it after the previous sample's second phase.
            float4 *wa = s_wacc + warp * K;
            __syncwarp();
            if (leader) {
                float4 q = wa[i];
                q.x += v[0]; q.y += v[1]; q.z += v[2]; q.w += v[3];
                wa[i] = q;
            }
            __syncwarp();
            if (leader) {
                float4 q = wa[i + 1];
                q.x += v[4]; q.y += v[5]; q.z += v[6]; q.w += v[7];
                wa[i + 1] = q;
            }
        } else if (leader) {
            if constexpr (TF2) {
                unsigned long long *g_acc = reinterpret_cast<unsigned long long *>(A.acc);
                cache_add4(s_acc, s_tag, g_acc, i, v, scale);
                cache_add4(s_acc, s_tag, g_acc, i + 1, v + 4, scale);
                cache_add4(s_acc, s_tag, g_acc, i + K, v + 8, scale);
                cache_add4(s_acc, s_tag, g_acc, i + K + 1, v + 12, scale);
            } else {
#pragma unroll
                for (int c = 0; c < 8; c++) acc_add(s_acc, 4 * i + c, v[c], scale);
            }
        }
    }
    __syncthreads();
    unsigned long long *g_acc = reinterpret_cast<unsigned long long *>(A.acc);
    if (wacc) {
        // the warps' copies summed in warp order, then one fixed-point add
        const float *w = reinterpret_cast<const float *>(s_wacc);
        for (int e = threadIdx.x; e < 4 * K; e += blockDim.x) {
            float sum = w[e];
#pragma unroll
            for (int wi = 1; wi < kAdjWarps; wi++) sum += w[wi * 4 * K + e];
            const long long q = __float2ll_rn(sum * scale);
            if (q != 0) atomicAdd(g_acc + e, (unsigned long long)q);
        }
    } else if (!TF2) {
        for (int e = threadIdx.x; e < 4 * K; e += blockDim.x) {
            unsigned long long v = s_acc[e];
            if (v != 0ull) atomicAdd(g_acc + e, v);
        }
    } else {
        for (int e = threadIdx.x; e < 4 * kSlots; e += blockDim.x) {
            const int t = s_tag[e >> 2];
            unsigned long long v = s_acc[e];
            if (t >= 0 && v != 0ull) atomicAdd(g_acc + 4 * (size_t)t + (e & 3), v);
        }
    }
}

__global__ void finalize_kernel(const long long *acc, int n, const float *absmax, float *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = (double)fixed_scale(absmax);
    out[i] = (float)((double)acc[i] / scale);
}

template <bool CUBIC, typename Kern>
static cudaError_t launch_adj(Kern kern, const AdjointArgs &a, int nviews, const float *absmax, cudaStream_t s) {
    // the 1-D table and its accumulators in shared memory (per warp in FP32
    // where warp_acc says so, else per CTA in 64-bit fixed point); for a 2-D
    // table the slot cache (values and tags)
    const int K = a.m.tf.K;
    const bool wacc = warp_acc(K, a.m.tf.M >= 2, CUBIC, a.fimg != nullptr);
    size_t smem = a.m.tf.M >= 2 ? (size_t)kSlots * (4 * sizeof(long long) + sizeof(int))
                  : wacc         ? (size_t)K * (1 + kAdjWarps) * sizeof(float4)
                                 : (size_t)K * (sizeof(float4) + 4 * sizeof(long long));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int rows = a.m.tf.M >= 2 ? 2 * kWarps2D : 8;         // pixel rows per CTA
    dim3 grid((a.m.cam.W + 15) / 16, (a.m.cam.H + rows - 1) / rows, nviews);
    kern<<<grid, a.m.tf.M >= 2 ? 32 * kWarps2D : 32 * kAdjWarps, smem, s>>>(a, absmax);
    return cudaGetLastError();
}

// The instance for the volume's storage, shading, opacity-correction mode RM
// (RM = -1: read at run time) and reconstruction filter.
template <int RM, bool CUBIC, bool TF2>
static cudaError_t launch_adj_rm(const AdjointArgs &a, int nviews, const float *absmax, cudaStream_t s) {
    switch (a.m.vol.storage * 2 + (a.m.p.shade ? 1 : 0)) {
        case RC_STORE_F32 * 2:
            return launch_adj<CUBIC>(adjoint_kernel<RC_STORE_F32, false, RM, CUBIC, TF2>, a, nviews, absmax, s);
        case RC_STORE_F32 * 2 + 1:
            return launch_adj<CUBIC>(adjoint_kernel<RC_STORE_F32, true, RM, CUBIC, TF2>, a, nviews, absmax, s);
        case RC_STORE_F16 * 2:
            return launch_adj<CUBIC>(adjoint_kernel<RC_STORE_F16, false, RM, CUBIC, TF2>, a, nviews, absmax, s);
        case RC_STORE_F16 * 2 + 1:
            return launch_adj<CUBIC>(adjoint_kernel<RC_STORE_F16, true, RM, CUBIC, TF2>, a, nviews, absmax, s);
        case RC_STORE_U16 * 2:
            return launch_adj<CUBIC>(adjoint_kernel<RC_STORE_U16, false, RM, CUBIC, TF2>, a, nviews, absmax, s);
        default: return launch_adj<CUBIC>(adjoint_kernel<RC_STORE_U16, true, RM, CUBIC, TF2>, a, nviews, absmax, s);
    }
}

// 1-D tables: one instance per opacity-correction mode; 2-D tables: the mode
// read at run time (the table lookup and the global atomics dominate there).
template <bool CUBIC>
static cudaError_t launch_adj_filter(const AdjointArgs &a, int nviews, const float *absmax, cudaStream_t s) {
    if (a.m.tf.M >= 2) return launch_adj_rm<-1, CUBIC, true>(a, nviews, absmax, s);
    switch (a.m.p.rmode) {
        case 0: return launch_adj_rm<0, CUBIC, false>(a, nviews, absmax, s);
        case 1: return launch_adj_rm<1, CUBIC, false>(a, nviews, absmax, s);
        case 2: return launch_adj_rm<2, CUBIC, false>(a, nviews, absmax, s);
        default: return launch_adj_rm<3, CUBIC, false>(a, nviews, absmax, s);
    }
}

// acc must hold 4 K max(M, 1) long longs (one per table entry and channel)
// followed by one float (the |dL/dI| maximum). With a.m.cams, nviews views
// (grid.z), dimg view-major; the gradient is the sum over the views.
cudaError_t launch_adjoint(const AdjointArgs &a, int nviews, float *dL_dtf, cudaStream_t s) {
    const int nent = a.m.tf.K * (a.m.tf.M >= 2 ? a.m.tf.M : 1);
    float *absmax = reinterpret_cast<float *>(a.acc + 4 * (size_t)nent);
    cudaError_t e = launch_absmax(reinterpret_cast<const float *>(a.dimg),
                                  (long long)nviews * a.m.cam.W * a.m.cam.H * 4, absmax, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.acc, 0, sizeof(long long) * 4 * (size_t)nent, s);
    if (e != cudaSuccess) return e;
    e = a.m.p.filter == RC_FILTER_BSPLINE ? launch_adj_filter<true>(a, nviews, absmax, s)
                                          : launch_adj_filter<false>(a, nviews, absmax, s);
    if (e != cudaSuccess) return e;
    finalize_kernel<<<(4 * nent + 255) / 256, 256, 0, s>>>(a.acc, 4 * nent, absmax, dL_dtf);
    return cudaGetLastError();
}

}  // namespace rc
