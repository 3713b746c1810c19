// Device building blocks of the march: the FP32 ray specification, bricked
// voxel addressing, trilinear resampling with central-difference gradients,
// transfer-function classification, opacity correction and shading.
#pragma once

#include "rc_internal.h"

namespace rc {

// Debug builds (-DRC_DEBUG, librc_debug.so) check every brick index and every
// table entry index against its extent before it is used: one out of range
// sets bit 1 of the context's error word, and bit 8 + site, and is replaced
// by 0 (an element inside the buffer), so that no access leaves its buffer
// and nothing traps; the next rc_context_sync (or statistics read) returns
// RC_ERR_CUDA. Release builds compile none of it. The brick index feeds every
// voxel, value+gradient and pair gather and every mask lookup; the table
// index feeds the classification and the adjoint's accumulators.
#ifdef RC_DEBUG
enum { kSiteBrick = 0, kSiteTable = 1, kSiteTable2 = 2 };
__device__ __forceinline__ int dbg_index(int idx, int bound, int *err, int site) {
    if ((unsigned)idx < (unsigned)bound) return idx;
    if (err) atomicOr(err, 2 | (256 << site));
    return 0;
}
#define RC_DBG_ERR(v) ((v).dbg_err)
#else
#define RC_DBG_ERR(v) nullptr
#endif

struct Ray {
    float o[3], d[3], dir[3];
    float tn, tf, ds;
    int nsamp;
};

// Sec. 4.1 step 1, the path of the ray. Every operation is an explicitly
// rounded FP32 intrinsic (never contracted), so sample positions are the
// exact values of the written specification:
//   a = (x + 0.5) / W;  ndc_x = (a*2 - 1) * tx;  b = (y + 0.5) / H;
//   ndc_y = (1 - b*2) * ty;  v = (f + ndc_x r) + ndc_y u;
//   len = sqrt((v0^2 + v1^2) + v2^2);  dir = v / len;  d = dir / s;
//   slab against [0, N-1] per axis (axes with d == 0 test o against the box);
//   t_near = max(0, max_a min(t0, t1)), t_far = min_a max(t0, t1);
//   ds = step * smin;  nsamp = floor((t_far - t_near) / ds) + 1.
__device__ __forceinline__ bool setup_ray(const CamRec &c, const VolDev &v, float step_vox,
                                          int x, int y, Ray &R) {
    float a = __fdiv_rn(__fadd_rn((float)x, 0.5f), (float)c.W);
    float ndcx = __fmul_rn(__fsub_rn(__fmul_rn(a, 2.0f), 1.0f), c.tx);
    float b = __fdiv_rn(__fadd_rn((float)y, 0.5f), (float)c.H);
    float ndcy = __fmul_rn(__fsub_rn(1.0f, __fmul_rn(b, 2.0f)), c.ty);
    float vv[3];
#pragma unroll
    for (int i = 0; i < 3; i++)
        vv[i] = __fadd_rn(__fadd_rn(c.f[i], __fmul_rn(ndcx, c.r[i])), __fmul_rn(ndcy, c.u[i]));
    float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(vv[0], vv[0]), __fmul_rn(vv[1], vv[1])),
                                     __fmul_rn(vv[2], vv[2])));
    float tn = 0.0f, tf = __int_as_float(0x7f800000);
    bool hit = true;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R.dir[i] = __fdiv_rn(vv[i], len);
        R.d[i] = __fdiv_rn(R.dir[i], v.s[i]);
        R.o[i] = c.o[i];
        float hi = (float)(v.n[i] - 1);
        if (R.d[i] == 0.0f) {
            if (R.o[i] < 0.0f || R.o[i] > hi) hit = false;
        } else {
            float t0 = __fdiv_rn(__fsub_rn(0.0f, R.o[i]), R.d[i]);
            float t1 = __fdiv_rn(__fsub_rn(hi, R.o[i]), R.d[i]);
            tn = fmaxf(tn, fminf(t0, t1));
            tf = fminf(tf, fmaxf(t0, t1));
        }
    }
    if (!hit || !(tf >= tn)) {
        R.nsamp = 0;
        return false;
    }
    R.tn = tn;
    R.tf = tf;
    R.ds = __fmul_rn(step_vox, v.smin);
    // at most 2^24 samples per ray (the API bounds step_vox, so this only
    // guards the int conversion)
    R.nsamp = (int)fminf(floorf(__fdiv_rn(__fsub_rn(tf, tn), R.ds)), 16777215.0f) + 1;
    return true;
}

// Evenly spaced sample k (Sec. 4.1): t_k = fma(k, ds, t_near), p = fma(t_k, d, o).
__device__ __forceinline__ float sample_t(const Ray &R, int k) {
    return __fmaf_rn((float)k, R.ds, R.tn);
}

__device__ __forceinline__ void position_at(const Ray &R, float t, float p[3]) {
#pragma unroll
    for (int i = 0; i < 3; i++) p[i] = __fmaf_rn(t, R.d[i], R.o[i]);
}

// Trilinear cell of a position: p clamped to [0, N-1], base = min(floor, N-2),
// weight = p - base (exact in FP32).
struct Cell {
    int i[3];
    float w[3];
};

__device__ __forceinline__ void cell_of(const VolDev &v, const float p[3], Cell &c) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float q = fminf(fmaxf(p[a], 0.0f), (float)(v.n[a] - 1));
        int b = min((int)q, v.n[a] - 2);   // q >= 0: truncation is floor
        c.i[a] = b;
        c.w[a] = __fsub_rn(q, (float)b);
    }
}

__device__ __forceinline__ int brick_of(const VolDev &v, const Cell &c) {
    const int b = ((c.i[2] >> 4) * v.cb[1] + (c.i[1] >> 4)) * v.cb[0] + (c.i[0] >> 4);
#ifdef RC_DEBUG
    return dbg_index(b + v.dbg_poison, v.cb[0] * v.cb[1] * v.cb[2], v.dbg_err, kSiteBrick);
#else
    return b;
#endif
}

// Apron bricks: cell-brick b stores the voxels 16b-1 .. 16b+17 of each axis
// (clamped to the volume, so border voxels are replicated), 19^3 values. The
// whole 4x4x4 neighbourhood of a cell is then one base address plus constant
// offsets. Local coordinates of cell base i: (i & 15) + 1.
constexpr unsigned kDX = 1, kDY = kApron, kDZ = kApron * kApron;

__device__ __forceinline__ unsigned cell_address(const VolDev &v, const Cell &c) {
    const unsigned b = (unsigned)brick_of(v, c);
    const unsigned lx = (unsigned)(c.i[0] & 15) + 1, ly = (unsigned)(c.i[1] & 15) + 1,
                   lz = (unsigned)(c.i[2] & 15) + 1;
    return b * (unsigned)kApronVox + (lz * kApron + ly) * kApron + lx;
}

// Element type of each storage.
template <int ST> struct Voxel;
template <> struct Voxel<RC_STORE_F32> { using T = float; };
template <> struct Voxel<RC_STORE_F16> { using T = __half; };
template <> struct Voxel<RC_STORE_U16> { using T = unsigned short; };

// Pointer to voxel (i, j, k) of the cell's apron brick. Neighbours are read
// as p[dx + dy + dz] with compile-time offsets (dx in -1..2, dy in
// -19..38, dz in -361..722), which stay inside the apron brick and become
// immediate offsets of one 64-bit address.
template <int ST>
__device__ __forceinline__ const typename Voxel<ST>::T *cell_ptr(const VolDev &v, const Cell &c) {
    return reinterpret_cast<const typename Voxel<ST>::T *>(v.data) + cell_address(v, c);
}

template <int ST>
__device__ __forceinline__ float ldv(const typename Voxel<ST>::T *p) {
    if (ST == RC_STORE_F32) return __ldg(reinterpret_cast<const float *>(p));
    if (ST == RC_STORE_F16) return __half2float(__ldg(reinterpret_cast<const __half *>(p)));
    return (float)__ldg(reinterpret_cast<const unsigned short *>(p));
}

// a + w (b - a): one rounding, stays inside [min(a,b), max(a,b)] when b - a is
// exact (true for integer codes and for FP16 values in [0, 1]).
__device__ __forceinline__ float lerp(float a, float b, float w) { return __fmaf_rn(w, b - a, a); }

// Packed FP32 pairs of the sm_100 family (sub / fma .rn.f32x2): each lane
// rounds exactly as the scalar operation, so lerp2 on a pair equals lerp on
// each element bit for bit, in half the instructions. A pair is a 64-bit
// register holding (lo, hi).
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float2 unpack2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ unsigned long long lerp2(unsigned long long a, unsigned long long b,
                                                    unsigned long long w) {
    unsigned long long d, r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(b), "l"(a));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(w), "l"(d), "l"(a));
    return r;
}

// Four channels as two pairs: (x, y) in .x, (z, w) in .y.
__device__ __forceinline__ ulonglong2 lerp4p(const ulonglong2 &a, const ulonglong2 &b, unsigned long long w) {
    return make_ulonglong2(lerp2(a.x, b.x, w), lerp2(a.y, b.y, w));
}

__device__ __forceinline__ float4 unpack4(const ulonglong2 &v) {
    const float2 lo = unpack2(v.x), hi = unpack2(v.y);
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

__device__ __forceinline__ float4 lerp4(const float4 &a, const float4 &b, float w) {
    const unsigned long long W = pack2(w, w);
    return unpack4(lerp4p(make_ulonglong2(pack2(a.x, a.y), pack2(a.z, a.w)),
                          make_ulonglong2(pack2(b.x, b.y), pack2(b.z, b.w)), W));
}

template <int ST>
__device__ __forceinline__ float trilinear(const VolDev &v, const Cell &c) {
    const auto *p = cell_ptr<ST>(v, c);
    constexpr int DX = (int)kDX, DY = (int)kDY, DZ = (int)kDZ;
    float wx = c.w[0], wy = c.w[1], wz = c.w[2];
    float c00 = lerp(ldv<ST>(p), ldv<ST>(p + DX), wx);
    float c10 = lerp(ldv<ST>(p + DY), ldv<ST>(p + DY + DX), wx);
    float c01 = lerp(ldv<ST>(p + DZ), ldv<ST>(p + DZ + DX), wx);
    float c11 = lerp(ldv<ST>(p + DZ + DY), ldv<ST>(p + DZ + DY + DX), wx);
    return lerp(lerp(c00, c10, wy), lerp(c01, c11, wy), wz);
}

// Pair entries by storage: two stored elements, aligned to their size.
template <int ST> struct Pair;
template <> struct Pair<RC_STORE_F32> { using T = float2; };
template <> struct Pair<RC_STORE_F16> { using T = __half2; };
template <> struct Pair<RC_STORE_U16> { using T = ushort2; };

// Pointer to the pair entry of voxels (i-1, i) in the footprint row
// (j-1, k-1) of the cell: rows (oy, oz) and pairs starting at x = i-1+ox are
// the compile-time offsets (oz * 19 + oy) * 18 + ox from it.
template <int ST>
__device__ __forceinline__ const typename Pair<ST>::T *pair_ptr(const VolDev &v, const Cell &c) {
    return reinterpret_cast<const typename Pair<ST>::T *>(v.pairs) +
           ((unsigned)brick_of(v, c) * (unsigned)kPairVox +
            (unsigned)((((c.i[2] & 15) * kApron + (c.i[1] & 15)) * kPairRow) + (c.i[0] & 15)));
}

// The two voxels of a pair entry as FP32 (the stored values converted as ldv does).
template <int ST>
__device__ __forceinline__ float2 ld_pair(const typename Pair<ST>::T *q) {
    if constexpr (ST == RC_STORE_F32) return __ldg(q);
    else if constexpr (ST == RC_STORE_F16) return __half22float2(__ldg(q));
    else {
        const ushort2 u = __ldg(q);
        return make_float2((float)u.x, (float)u.y);
    }
}

template <int OY, int OZ, int OX>
constexpr int pair_off() { return (OZ * kApron + OY) * kPairRow + OX; }

// Value and world-space gradient from the value+gradient bricks (FP32
// storage): each voxel holds (V, D_x, D_y, D_z) with D_a = V(+1 along a) -
// V(-1 along a), neighbour indices clamped to the volume, all exact integers.
// Central differences of the trilinear field are linear in the voxels, so
// (f(p + e_a) - f(p - e_a)) / 2 equals the trilinear interpolation of D_a / 2
// at p, the clamped border included; 8 four-wide loads replace 32 scalar
// loads. The value is interpolated in the same order as trilinear().
__device__ __forceinline__ float value_grad_vg(const VolDev &v, const Cell &c, float g[3]) {
    // 32-bit index: a volume has fewer than 2^31 apron voxels (19^3 per
    // brick), so fewer value+gradient entries (17^3 per brick)
    const unsigned idx = (unsigned)brick_of(v, c) * (unsigned)kGradVox +
                         (unsigned)(((c.i[2] & 15) * kGradEdge + (c.i[1] & 15)) * kGradEdge + (c.i[0] & 15));
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(v.vg) + idx;
    constexpr int DY = kGradEdge, DZ = kGradEdge * kGradEdge;
    const unsigned long long wx = pack2(c.w[0], c.w[0]), wy = pack2(c.w[1], c.w[1]), wz = pack2(c.w[2], c.w[2]);
    const ulonglong2 c00 = lerp4p(__ldg(p), __ldg(p + 1), wx);
    const ulonglong2 c10 = lerp4p(__ldg(p + DY), __ldg(p + DY + 1), wx);
    const ulonglong2 c01 = lerp4p(__ldg(p + DZ), __ldg(p + DZ + 1), wx);
    const ulonglong2 c11 = lerp4p(__ldg(p + DZ + DY), __ldg(p + DZ + DY + 1), wx);
    const float4 r = unpack4(lerp4p(lerp4p(c00, c10, wy), lerp4p(c01, c11, wy), wz));
    g[0] = r.y * v.inv2s[0];
    g[1] = r.z * v.inv2s[1];
    g[2] = r.w * v.inv2s[2];
    return r.x;
}

// A uint16 value+gradient entry as biased FP32 pairs (V + m0, D_x + m1) and
// (D_y + m1, D_z + m1), exactly: a byte permute places each 16-bit field in
// the mantissa of 2^23, so m0 = 2^23 for the value and m1 = 2^23 + 32768 for
// the offset differences.
__device__ __forceinline__ ulonglong2 vg16_biased(uint2 q) {
    unsigned long long a, b;
    asm("mov.b64 %0, {%1, %2};"
        : "=l"(a)
        : "r"(__byte_perm(q.x, 0x4B000000u, 0x7610)), "r"(__byte_perm(q.x, 0x4B000000u, 0x7632)));
    asm("mov.b64 %0, {%1, %2};"
        : "=l"(b)
        : "r"(__byte_perm(q.y, 0x4B000000u, 0x7610)), "r"(__byte_perm(q.y, 0x4B000000u, 0x7632)));
    return make_ulonglong2(a, b);
}

// lerp4p of two uint16 entries a and b along x. With a' = a + m and
// b' = b + m (biased, exact integers below 2^24), b' - a' = b - a exactly,
// so fma(w, b' - a', a' - m) is lerp4p of the decoded entries bit for bit,
// with the bias removed from the first entry only.
__device__ __forceinline__ ulonglong2 vg16_lerp(uint2 qa, uint2 qb, unsigned long long w) {
    const ulonglong2 a = vg16_biased(qa), b = vg16_biased(qb);
    unsigned long long d0, d1, s0, s1, r0, r1;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(b.x), "l"(a.x));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(b.y), "l"(a.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(s0) : "l"(a.x), "l"(pack2(8388608.0f, 8421376.0f)));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(s1) : "l"(a.y), "l"(pack2(8421376.0f, 8421376.0f)));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r0) : "l"(w), "l"(d0), "l"(s0));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r1) : "l"(w), "l"(d1), "l"(s1));
    return make_ulonglong2(r0, r1);
}

// value_grad_vg for uint16 storage: the same integers from 8-byte entries
// (half the bytes of the float4 entries), so the same operations give the
// FP32 storage's result bit for bit.
__device__ __forceinline__ float value_grad_vg16(const VolDev &v, const Cell &c, float g[3]) {
    const unsigned idx = (unsigned)brick_of(v, c) * (unsigned)kGradVox +
                         (unsigned)(((c.i[2] & 15) * kGradEdge + (c.i[1] & 15)) * kGradEdge + (c.i[0] & 15));
    const uint2 *p = reinterpret_cast<const uint2 *>(v.vg) + idx;
    constexpr int DY = kGradEdge, DZ = kGradEdge * kGradEdge;
    const unsigned long long wx = pack2(c.w[0], c.w[0]), wy = pack2(c.w[1], c.w[1]), wz = pack2(c.w[2], c.w[2]);
    const ulonglong2 c00 = vg16_lerp(__ldg(p), __ldg(p + 1), wx);
    const ulonglong2 c10 = vg16_lerp(__ldg(p + DY), __ldg(p + DY + 1), wx);
    const ulonglong2 c01 = vg16_lerp(__ldg(p + DZ), __ldg(p + DZ + 1), wx);
    const ulonglong2 c11 = vg16_lerp(__ldg(p + DZ + DY), __ldg(p + DZ + DY + 1), wx);
    const float4 r = unpack4(lerp4p(lerp4p(c00, c10, wy), lerp4p(c01, c11, wy), wz));
    g[0] = r.y * v.inv2s[0];
    g[1] = r.z * v.inv2s[1];
    g[2] = r.w * v.inv2s[2];
    return r.x;
}

// value_grad_vg for FP16 storage (8-byte entries: the stored FP16 value h and
// the code differences offset by 32768): the value is interpolated from the
// h as the FP16 storage's other paths do (lerp(a, b, w) = fma(w, b - a, a),
// x, then y, then z), the differences as integers, and the gradient of h is
// the code gradient / o (o a power of two: exact scaling).
__device__ __forceinline__ float value_grad_vg16h(const VolDev &v, const Cell &c, float g[3]) {
    const unsigned idx = (unsigned)brick_of(v, c) * (unsigned)kGradVox +
                         (unsigned)(((c.i[2] & 15) * kGradEdge + (c.i[1] & 15)) * kGradEdge + (c.i[0] & 15));
    const uint2 *p = reinterpret_cast<const uint2 *>(v.vg) + idx;
    constexpr int DY = kGradEdge, DZ = kGradEdge * kGradEdge;
    const unsigned long long wx = pack2(c.w[0], c.w[0]), wy = pack2(c.w[1], c.w[1]), wz = pack2(c.w[2], c.w[2]);
    // (h, D_x + m) and (D_y + m, D_z + m) with m = 2^23 + 32768 (as vg16_biased);
    // along x the bias leaves the first entry only, and h is not biased
    auto lerp_x = [&](uint2 qa, uint2 qb) {
        const ulonglong2 a = vg16_biased(qa), b = vg16_biased(qb);
        const float ha = __half2float(__ushort_as_half((unsigned short)(qa.x & 0xFFFFu)));
        const float hb = __half2float(__ushort_as_half((unsigned short)(qb.x & 0xFFFFu)));
        const unsigned long long a0 = pack2(ha, unpack2(a.x).y), b0 = pack2(hb, unpack2(b.x).y);
        unsigned long long d0, d1, s0, s1, r0, r1;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(b0), "l"(a0));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(b.y), "l"(a.y));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(s0) : "l"(a0), "l"(pack2(0.0f, 8421376.0f)));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(s1) : "l"(a.y), "l"(pack2(8421376.0f, 8421376.0f)));
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r0) : "l"(wx), "l"(d0), "l"(s0));
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r1) : "l"(wx), "l"(d1), "l"(s1));
        return make_ulonglong2(r0, r1);
    };
    const ulonglong2 c00 = lerp_x(__ldg(p), __ldg(p + 1));
    const ulonglong2 c10 = lerp_x(__ldg(p + DY), __ldg(p + DY + 1));
    const ulonglong2 c01 = lerp_x(__ldg(p + DZ), __ldg(p + DZ + 1));
    const ulonglong2 c11 = lerp_x(__ldg(p + DZ + DY), __ldg(p + DZ + DY + 1));
    const float4 r = unpack4(lerp4p(lerp4p(c00, c10, wy), lerp4p(c01, c11, wy), wz));
    const float inv_o = 1.0f / (float)v.f16o;
    g[0] = r.y * v.inv2s[0] * inv_o;
    g[1] = r.z * v.inv2s[1] * inv_o;
    g[2] = r.w * v.inv2s[2] * inv_o;
    return r.x;
}

// Value and world-space central-difference gradient of the trilinear field,
// one index unit per axis, from the 32 distinct voxels around the cell.
// The samples at p -/+ e_a use the cells with base coordinates
// {max(i-1, 0), i} and {i+1, min(i+2, N-1)} and the same weight, which equals
// resampling the clamped positions p -/+ 1; the apron's replicated border
// voxels give the clamped coordinates.
template <int ST, bool PAIRS>
__device__ __forceinline__ float value_grad_x(const VolDev &v, const Cell &c, float g[3]) {
    const float wx = c.w[0], wy = c.w[1], wz = c.w[2];
    // rows along x at (y, z) = (j-1+oy, k-1+oz): L the centre cell's x edge,
    // M and P those of the -x and +x cells
    float L11, L21, L12, L22, M11, M21, M12, M22, P11, P21, P12, P22, L01, L02, L31, L32, L10, L20, L13, L23;
    if (PAIRS) {
        // pairs (i-1, i) and (i+1, i+2) of the 4 centre rows, (i, i+1) of the
        // 8 side rows: 16 loads
        const auto *pp = pair_ptr<ST>(v, c);
        auto row4 = [&](int off, float &M, float &L, float &P) {
            const float2 a = ld_pair<ST>(pp + off), b = ld_pair<ST>(pp + off + 2);
            M = lerp(a.x, a.y, wx);
            L = lerp(a.y, b.x, wx);
            P = lerp(b.x, b.y, wx);
        };
        auto row2 = [&](int off) {
            const float2 a = ld_pair<ST>(pp + off + 1);
            return lerp(a.x, a.y, wx);
        };
        row4(pair_off<1, 1, 0>(), M11, L11, P11);
        row4(pair_off<2, 1, 0>(), M21, L21, P21);
        row4(pair_off<1, 2, 0>(), M12, L12, P12);
        row4(pair_off<2, 2, 0>(), M22, L22, P22);
        L01 = row2(pair_off<0, 1, 0>());
        L02 = row2(pair_off<0, 2, 0>());
        L31 = row2(pair_off<3, 1, 0>());
        L32 = row2(pair_off<3, 2, 0>());
        L10 = row2(pair_off<1, 0, 0>());
        L20 = row2(pair_off<2, 0, 0>());
        L13 = row2(pair_off<1, 3, 0>());
        L23 = row2(pair_off<2, 3, 0>());
    } else {
        const auto *p = cell_ptr<ST>(v, c);
        constexpr int X0 = -(int)kDX, X1 = 0, X2 = (int)kDX, X3 = 2 * (int)kDX;
        constexpr int Y0 = -(int)kDY, Y1 = 0, Y2 = (int)kDY, Y3 = 2 * (int)kDY;
        constexpr int Z0 = -(int)kDZ, Z1 = 0, Z2 = (int)kDZ, Z3 = 2 * (int)kDZ;
#define RC_F(X, Y, Z) ldv<ST>(p + ((X) + (Y) + (Z)))
#define RC_LX(XA, XB, Y, Z) lerp(RC_F(XA, Y, Z), RC_F(XB, Y, Z), wx)
        L11 = RC_LX(X1, X2, Y1, Z1); L21 = RC_LX(X1, X2, Y2, Z1);
        L12 = RC_LX(X1, X2, Y1, Z2); L22 = RC_LX(X1, X2, Y2, Z2);
        M11 = RC_LX(X0, X1, Y1, Z1); M21 = RC_LX(X0, X1, Y2, Z1);
        M12 = RC_LX(X0, X1, Y1, Z2); M22 = RC_LX(X0, X1, Y2, Z2);
        P11 = RC_LX(X2, X3, Y1, Z1); P21 = RC_LX(X2, X3, Y2, Z1);
        P12 = RC_LX(X2, X3, Y1, Z2); P22 = RC_LX(X2, X3, Y2, Z2);
        L01 = RC_LX(X1, X2, Y0, Z1); L02 = RC_LX(X1, X2, Y0, Z2);
        L31 = RC_LX(X1, X2, Y3, Z1); L32 = RC_LX(X1, X2, Y3, Z2);
        L10 = RC_LX(X1, X2, Y1, Z0); L20 = RC_LX(X1, X2, Y2, Z0);
        L13 = RC_LX(X1, X2, Y1, Z3); L23 = RC_LX(X1, X2, Y2, Z3);
#undef RC_LX
#undef RC_F
    }
    float a1 = lerp(L11, L21, wy), a2 = lerp(L12, L22, wy);
    float val = lerp(a1, a2, wz);
    float xm = lerp(lerp(M11, M21, wy), lerp(M12, M22, wy), wz);
    float xp = lerp(lerp(P11, P21, wy), lerp(P12, P22, wy), wz);
    float ym = lerp(lerp(L01, L11, wy), lerp(L02, L12, wy), wz);
    float yp = lerp(lerp(L21, L31, wy), lerp(L22, L32, wy), wz);
    float a0 = lerp(L10, L20, wy), a3 = lerp(L13, L23, wy);
    float zm = lerp(a0, a1, wz);
    float zp = lerp(a2, a3, wz);
    g[0] = (xp - xm) * v.inv2s[0];
    g[1] = (yp - ym) * v.inv2s[1];
    g[2] = (zp - zm) * v.inv2s[2];
    return val;
}

// Value and gradient of the trilinear field: FP32 storage from the
// value+gradient bricks, uint16 from its 8-byte value+gradient bricks when
// the volume has them (vmax < 32768); FP16 from the pair bricks when the
// volume has them (one uniform branch per sample), else from the apron brick.
template <int ST>
__device__ __forceinline__ float value_grad(const VolDev &v, const Cell &c, float g[3]) {
    if (ST == RC_STORE_F32) return value_grad_vg(v, c, g);
    if (ST == RC_STORE_U16 && v.vg != nullptr) return value_grad_vg16(v, c, g);
    if (ST == RC_STORE_F16 && v.vg != nullptr) return value_grad_vg16h(v, c, g);
    if (ST == RC_STORE_F16 && v.pairs != nullptr) return value_grad_x<ST, true>(v, c, g);
    return value_grad_x<ST, false>(v, c, g);
}

// Uniform cubic B-spline reconstruction (Sec. 3.2's higher-order filter):
// f(p) = sum of the 4 x 4 x 4 voxels i-1 .. i+2 around cell base i, each
// weighted by the product of the B-spline kernel at its per-axis distance.
// With t the cell fraction, the four weights of an axis are
//   (1-t)^3/6,  t^3/2 - t^2 + 2/3,  -t^3/2 + t^2/2 + t/2 + 1/6,  t^3/6
// and their derivatives -(1-t)^2/2, 3t^2/2 - 2t, -3t^2/2 + t + 1/2, t^2/2.
// The apron brick holds exactly this footprint (its replicated border voxels
// are the clamped indices), so the 64 voxels are one base address plus
// constant offsets; with FP32 storage they come from the pair bricks, two
// 8-byte loads per row.
__device__ __forceinline__ void bspline_weights(float t, float w[4]) {
    const float s = 1.0f - t, t2 = t * t;
    w[0] = s * s * s * (1.0f / 6.0f);
    w[1] = __fmaf_rn(t2, __fmaf_rn(0.5f, t, -1.0f), 2.0f / 3.0f);
    w[2] = __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(-0.5f, t, 0.5f), 0.5f), 1.0f / 6.0f);
    w[3] = t2 * t * (1.0f / 6.0f);
}

__device__ __forceinline__ void bspline_dweights(float t, float d[4]) {
    const float s = 1.0f - t;
    d[0] = -0.5f * s * s;
    d[1] = t * __fmaf_rn(1.5f, t, -2.0f);
    d[2] = __fmaf_rn(t, __fmaf_rn(-1.5f, t, 1.0f), 0.5f);
    d[3] = 0.5f * t * t;
}



// The four voxels x = i-1 .. i+2 of footprint row (oy, oz): PAIRS, two pair
// loads; else four scalar loads from the apron brick.
template <int ST, bool PAIRS>
__device__ __forceinline__ void bspline_row(const typename Voxel<ST>::T *a, const typename Pair<ST>::T *pp, int oz,
                                            int oy, float &v0, float &v1, float &v2, float &v3) {
    if (PAIRS) {
        const auto *q = pp + (oz * kApron + oy) * kPairRow;
        const float2 p0 = ld_pair<ST>(q), p1 = ld_pair<ST>(q + 2);
        v0 = p0.x;
        v1 = p0.y;
        v2 = p1.x;
        v3 = p1.y;
    } else {
        const auto *r = a + (oz * (int)kDZ + oy * (int)kDY);
        v0 = ldv<ST>(r);
        v1 = ldv<ST>(r + 1);
        v2 = ldv<ST>(r + 2);
        v3 = ldv<ST>(r + 3);
    }
}

template <int ST, bool PAIRS>
__device__ __forceinline__ float bspline_x(const VolDev &v, const Cell &c) {
    const auto *a = cell_ptr<ST>(v, c) - (int)(kDX + kDY + kDZ);     // voxel (i-1, j-1, k-1)
    const typename Pair<ST>::T *pp = PAIRS ? pair_ptr<ST>(v, c) : nullptr;
    float wx[4], wy[4], wz[4];
    bspline_weights(c.w[0], wx);
    bspline_weights(c.w[1], wy);
    bspline_weights(c.w[2], wz);
    float f = 0.0f;
#pragma unroll
    for (int oz = 0; oz < 4; oz++) {
        float fz = 0.0f;
#pragma unroll
        for (int oy = 0; oy < 4; oy++) {
            float v0, v1, v2, v3;
            bspline_row<ST, PAIRS>(a, pp, oz, oy, v0, v1, v2, v3);
            float fx = v0 * wx[0];
            fx = __fmaf_rn(v1, wx[1], fx);
            fx = __fmaf_rn(v2, wx[2], fx);
            fx = __fmaf_rn(v3, wx[3], fx);
            fz = __fmaf_rn(fx, wy[oy], fz);
        }
        f = __fmaf_rn(fz, wz[oz], f);
    }
    return f;
}

// Value and analytic world-space gradient (value units per mm) of the
// B-spline field: d/dx sums the same voxels with the x weights replaced by
// their derivatives; 1/s = 2 * (0.5/s) exactly.
template <int ST, bool PAIRS>
__device__ __forceinline__ float bspline_grad_x(const VolDev &v, const Cell &c, float g[3]) {
    const auto *a = cell_ptr<ST>(v, c) - (int)(kDX + kDY + kDZ);     // voxel (i-1, j-1, k-1)
    const typename Pair<ST>::T *pp = PAIRS ? pair_ptr<ST>(v, c) : nullptr;
    float wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
    bspline_weights(c.w[0], wx);
    bspline_weights(c.w[1], wy);
    bspline_weights(c.w[2], wz);
    bspline_dweights(c.w[0], dx);
    bspline_dweights(c.w[1], dy);
    bspline_dweights(c.w[2], dz);
    float f = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int oz = 0; oz < 4; oz++) {
        float fz = 0.0f, gxz = 0.0f, gyz = 0.0f;
#pragma unroll
        for (int oy = 0; oy < 4; oy++) {
            float v0, v1, v2, v3;
            bspline_row<ST, PAIRS>(a, pp, oz, oy, v0, v1, v2, v3);
            float fx = v0 * wx[0], ex = v0 * dx[0];
            fx = __fmaf_rn(v1, wx[1], fx);
            ex = __fmaf_rn(v1, dx[1], ex);
            fx = __fmaf_rn(v2, wx[2], fx);
            ex = __fmaf_rn(v2, dx[2], ex);
            fx = __fmaf_rn(v3, wx[3], fx);
            ex = __fmaf_rn(v3, dx[3], ex);
            fz = __fmaf_rn(fx, wy[oy], fz);
            gxz = __fmaf_rn(ex, wy[oy], gxz);
            gyz = __fmaf_rn(fx, dy[oy], gyz);
        }
        f = __fmaf_rn(fz, wz[oz], f);
        gx = __fmaf_rn(gxz, wz[oz], gx);
        gy = __fmaf_rn(gyz, wz[oz], gy);
        gz = __fmaf_rn(fz, dz[oz], gz);
    }
    g[0] = gx * (2.0f * v.inv2s[0]);
    g[1] = gy * (2.0f * v.inv2s[1]);
    g[2] = gz * (2.0f * v.inv2s[2]);
    return f;
}

// The B-spline value (and gradient) with the footprint from the pair bricks
// when the volume has them (FP32 and FP16 storage; one uniform branch per
// sample), else from the apron brick; both read the same stored values.
template <int ST>
__device__ __forceinline__ float bspline(const VolDev &v, const Cell &c) {
    if (ST != RC_STORE_U16 && v.pairs != nullptr) return bspline_x<ST, true>(v, c);
    return bspline_x<ST, false>(v, c);
}

template <int ST>
__device__ __forceinline__ float bspline_grad(const VolDev &v, const Cell &c, float g[3]) {
    if (ST != RC_STORE_U16 && v.pairs != nullptr) return bspline_grad_x<ST, true>(v, c, g);
    return bspline_grad_x<ST, false>(v, c, g);
}

// Table coordinate of a stored value, one rounding, monotone in the value:
// raw codes v give u = fl(v * ucoef); FP16 values h = (code - o) / o give
// u = fl((h + 1) * ucoef) as one fused multiply-add (ucoef = fl(o (K-1) / vmax)).
// The occupancy mask floors the same function at a brick's min and max, which
// makes skipping exact.
template <int ST>
__device__ __forceinline__ float tf_coord(float val, float ucoef) {
    if (ST == RC_STORE_F16) return __fmaf_rn(val, ucoef, ucoef);
    return __fmul_rn(val, ucoef);
}

// Sec. 2.6: linear interpolation of the two neighbouring table entries.
__device__ __forceinline__ float4 classify(const float4 *tab, int K, float u, int *i0 = nullptr,
                                           float *w0 = nullptr, int *err = nullptr) {
    float q = fminf(fmaxf(u, 0.0f), (float)(K - 1));
    int i = min((int)q, K - 2);
    float w = q - (float)i;
#ifdef RC_DEBUG
    i = dbg_index(i, K - 1, err, kSiteTable);
#else
    (void)err;
#endif
    const ulonglong2 *t2 = reinterpret_cast<const ulonglong2 *>(tab);
    if (i0) *i0 = i;
    if (w0) *w0 = w;
    return unpack4(lerp4p(t2[i], t2[i + 1], pack2(w, w)));
}

// Two-dimensional classification over (value, gradient magnitude), the
// scalar / gradient-magnitude transfer functions of Sec. 3.1: u the value
// coordinate, w = fl(|grad| * wcoef) the gradient coordinate, each clamped to
// its axis; bilinear over the four entries (value direction first). The
// table stays in global memory (read-only path; at most a few MB).
// The bilinear cell (i, j) and weights (a, b) are returned for the gradient.
__device__ __forceinline__ float4 classify2_at(const TFDev &tf, float u, float w, int &i, int &j, float &a,
                                               float &b, int *err = nullptr) {
    const int K = tf.K, M = tf.M;
    const float qu = fminf(fmaxf(u, 0.0f), (float)(K - 1));
    const float qw = fminf(fmaxf(w, 0.0f), (float)(M - 1));
    i = min((int)qu, K - 2);
    j = min((int)qw, M - 2);
    a = qu - (float)i;
    b = qw - (float)j;
#ifdef RC_DEBUG
    i = dbg_index(i, K - 1, err, kSiteTable2);
    j = dbg_index(j, M - 1, err, kSiteTable2);
#else
    (void)err;
#endif
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(tf.tab2) + (size_t)j * K + i;
    const unsigned long long A = pack2(a, a);
    const ulonglong2 r0 = lerp4p(__ldg(p), __ldg(p + 1), A);
    const ulonglong2 r1 = lerp4p(__ldg(p + K), __ldg(p + K + 1), A);
    return unpack4(lerp4p(r0, r1, pack2(b, b)));
}

__device__ __forceinline__ float4 classify2(const TFDev &tf, float u, float w, int *err = nullptr) {
    int i, j;
    float a, b;
    return classify2_at(tf, u, w, i, j, a, b, err);
}

// The gradient-magnitude coordinate of a 2-D table: fl(|g| * wcoef).
__device__ __forceinline__ float tf2_row_coord(const TFDev &tf, const float g[3]) {
    const float gm = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    return __fmul_rn(gm, tf.wcoef);
}

// Eq. 3 for a segment of length ds: alpha' = 1 - (1 - alpha)^(ds/ds_ref).
// A general ratio (per-ray segments of the importance and profile marches)
// uses t^r = 2^(r log2 t) on the special-function unit: relative error about
// r * 2^-21 (below 1e-5 for segments up to 8 reference steps), with the end
// points exact (alpha 0 -> 0, alpha 1 -> 1).
// RM >= 0 fixes the mode at compile time (the march instances per mode);
// RM = -1 takes the runtime rmode.
template <int RM = -1>
__device__ __forceinline__ float correct_alpha(float a, int rmode, float ratio) {
    const int m = RM >= 0 ? RM : rmode;
    float t = 1.0f - a;
    if (m == 0) return a;
    if (m == 1) return 1.0f - sqrtf(t);
    if (m == 2) return 1.0f - sqrtf(sqrtf(t));
    if (t >= 1.0f) return 0.0f;
    if (t <= 0.0f) return 1.0f;
    return 1.0f - exp2f(ratio * __log2f(t));
}

// Headlight Blinn-Phong with a two-sided diffuse term: light and view along
// -dir, half vector = light vector; colour = min(1, rgb (ka + kd n.l) + ks (n.l)^16).
// Below gmin the normal is undefined and the colour is min(1, rgb (ka + kd)).
__device__ __forceinline__ void shade_factor(const MarchParams &P, const VolDev &v, const float g[3],
                                             const float dir[3], float &sf, float &spec) {
    float g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const bool flat = g2 < v.gmin * v.gmin;
    // selects instead of a branch; for g2 = 0 the product is NaN and fminf
    // returns 1, a value the select then discards
    float ndl = fabsf(g[0] * dir[0] + g[1] * dir[1] + g[2] * dir[2]) * rsqrtf(g2);
    ndl = fminf(ndl, 1.0f);
    float n2 = ndl * ndl, n4 = n2 * n2, n8 = n4 * n4;
    sf = flat ? P.ka + P.kd : P.ka + P.kd * ndl;
    spec = flat ? 0.0f : P.ks * (n8 * n8);
}

__device__ __forceinline__ float4 half4_to_float4(uint2 h) {
    __half2 lo = *reinterpret_cast<__half2 *>(&h.x);
    __half2 hi = *reinterpret_cast<__half2 *>(&h.y);
    float2 a = __half22float2(lo), b = __half22float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Copies the table into shared memory as FP32 (FP16 entries converted exactly).
__device__ __forceinline__ void load_tf(const TFDev &tf, float4 *s_tf) {
    for (int e = threadIdx.x; e < tf.K; e += blockDim.x)
        s_tf[e] = tf.fp16 ? half4_to_float4(tf.f16[e]) : tf.f32[e];
}

// One compositing sample (Sec. 4.1 step 2-3): resample at cell c, classify,
// correct the opacity to the segment, shade. Returns straight colour and
// corrected opacity; the caller composites. Shared by every march so that the
// plain, fallback and importance marches evaluate a sample identically.
// F: kShade, kCubic (B-spline instead of trilinear), kTF2 (2-D table from
// tf.tab2, else the 1-D table s_tf); the gradient is computed when shading or
// the 2-D table needs it.
template <int ST, int F, int RM = -1>
__device__ __forceinline__ float4 eval_sample_x(const VolDev &vol, const MarchParams &P, const float4 *s_tf,
                                                const TFDev &tf, const float dir[3], const Cell &c, int rmode,
                                                float ratio) {
    constexpr bool SHADE = (F & kShade) != 0, CUBIC = (F & kCubic) != 0, TF2 = (F & kTF2) != 0;
    constexpr bool GRAD = SHADE || TF2;
    float val, g[3];
    if (CUBIC) {
        if (GRAD) val = bspline_grad<ST>(vol, c, g);
        else val = bspline<ST>(vol, c);
    } else {
        if (GRAD) val = value_grad<ST>(vol, c, g);
        else val = trilinear<ST>(vol, c);
    }
    float4 e;
    if (TF2) {
        e = classify2(tf, tf_coord<ST>(val, tf.ucoef), tf2_row_coord(tf, g), RC_DBG_ERR(vol));
    } else {
        e = classify(s_tf, tf.K, tf_coord<ST>(val, tf.ucoef), nullptr, nullptr, RC_DBG_ERR(vol));
    }
    float ap = correct_alpha<RM>(e.w, rmode, ratio);
    if (SHADE) {
        float sf, spec;
        shade_factor(P, vol, g, dir, sf, spec);
        e.x = fminf(1.0f, __fmaf_rn(e.x, sf, spec));
        e.y = fminf(1.0f, __fmaf_rn(e.y, sf, spec));
        e.z = fminf(1.0f, __fmaf_rn(e.z, sf, spec));
    }
    e.w = ap;
    return e;
}

// The trilinear, 1-D-table sample of the marches that support only that form.
template <int ST, bool SHADE>
__device__ __forceinline__ float4 eval_sample(const VolDev &vol, const MarchParams &P, const float4 *s_tf, int K,
                                              float ucoef, const float dir[3], const Cell &c, int rmode,
                                              float ratio) {
    TFDev tf{};
    tf.K = K;
    tf.ucoef = ucoef;
    return eval_sample_x<ST, SHADE ? kShade : 0>(vol, P, s_tf, tf, dir, c, rmode, ratio);
}

// Front-to-back compositing of one sample (Eq. 4): C += T a' c, T *= 1 - a'.
__device__ __forceinline__ void composite_add(const float4 &e, float &C0, float &C1, float &C2, float &T) {
    float ta = T * e.w;
    C0 = __fmaf_rn(ta, e.x, C0);
    C1 = __fmaf_rn(ta, e.y, C1);
    C2 = __fmaf_rn(ta, e.z, C2);
    T = T * (1.0f - e.w);
}

// Jump over an empty axis-aligned block of 2^s cells per axis containing
// cell c (s = 4: the cell-brick; 3 and 2: its octants and 4^3 sub-blocks).
// Returns the index of the first sample that may lie outside the block: the
// sample m just before the computed exit distance is verified to be in the
// same block (cell bases agree above bit s on every axis); since each
// coordinate of the computed positions is monotone in k, every sample between
// k and m is then inside too. Falls back to k + 1 when the check fails, so
// the exit estimate needs no exact rounding.
__device__ __forceinline__ int jump_block(const Ray &R, const VolDev &v, const Cell &c, int k, int s) {
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
    if (texit == INF) return R.nsamp;
    float fm = floorf(__fdiv_rn(texit - R.tn, R.ds));
    int m = fm >= (float)R.nsamp ? R.nsamp - 1 : (int)fm;
    if (m <= k) return k + 1;
#pragma unroll 1
    for (int tries = 0; tries < 2 && m > k; tries++, m--) {
        float p[3];
        position_at(R, sample_t(R, m), p);
        Cell cm;
        cell_of(v, p, cm);
        if (((cm.i[0] ^ c.i[0]) >> s) == 0 && ((cm.i[1] ^ c.i[1]) >> s) == 0 && ((cm.i[2] ^ c.i[2]) >> s) == 0)
            return m + 1;
    }
    return k + 1;
}

// The empty block around cell c by the fine mask of its cell-brick (one bit
// per 4^3 sub-block, bit sz*16 + sy*4 + sx): 4 when the whole brick is empty,
// 3 when its octant is, 2 when the sub-block is, -1 when the sample may have
// non-zero opacity.
// The sub-block's own bit is tested first: most evaluated samples lie in an
// occupied sub-block and need nothing else.
__device__ __forceinline__ int empty_block(unsigned long long m, const Cell &c) {
    const int bit = ((c.i[0] >> 2) & 3) | (c.i[1] & 12) | ((c.i[2] & 12) << 2);   // sz*16 + sy*4 + sx
    const unsigned half = (bit & 32) ? (unsigned)(m >> 32) : (unsigned)m;
    if ((half >> (bit & 31)) & 1u) return -1;
    if (m == 0ull) return 4;
    const int oct = bit & 0x2A;                                          // bit of the octant's first sub-block
    if (((m >> oct) & 0x330033ull) == 0ull) return 3;                   // sub-blocks {0,1} x {0,1} x {0,1} of it
    return 2;
}

}  // namespace rc
