// Host side of the C ABI declared in include/rc.h: validation, object
// lifetimes, camera records, lazy occupancy rebuilds and kernel dispatch.
#include <algorithm>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "rc_internal.h"

namespace rc {
// the brick-staged march variant (rc_march_staged.cu)
bool staged_eligible(const MarchArgs &a);
cudaError_t launch_march_staged(const MarchArgs &a, int nviews, int *err, long long budget, cudaStream_t s);
}  // namespace rc

using namespace rc;

struct rc_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    char err[512] = {0};
    // transfer function
    float4 *d_tf32 = nullptr;
    uint2 *d_tf16 = nullptr;
    int tf_cap = 0;
    int K = 0;
    int tf_fp16 = 0;
    uint64_t tf_version = 0;
    // 2-D table (M >= 2 while it is the current table; M = 0: 1-D)
    float4 *d_tf2 = nullptr;
    float *d_amax = nullptr;
    long long tf2_cap = 0;
    int M = 0;
    float gmax = 0.0f;
    // camera
    bool cam_set = false;
    rc_camera cam{};
    // statistics counters (slots 0-4) and the device error word (slot 5:
    // bit 0 = a bounded wait of a kernel gave up)
    unsigned long long *d_stats = nullptr;
    unsigned long long *h_stats = nullptr;   // pinned
    void *h_tfstage = nullptr;               // pinned staging of host tables (rc_tf_set, rc_tf2d_set)
    size_t tfstage_cap = 0;
    cudaEvent_t ev_tfstage = nullptr;        // after the last copy out of the staging buffer
    bool tfstage_pending = false;
    // camera records of a multi-view render
    CamRec *d_cams = nullptr;
    int cams_cap = 0;
    // per-volume pointers of a batch render
    BatchVol *d_batch = nullptr;
    int batch_cap = 0;
    // scratch of the adjoint: 4K fixed-point accumulators + |dL/dI| maximum
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    int nvolumes = 0;
    // learned proposal: FP32 master parameters, Adam moments, packed BF16
    // fragments, gradient and per-block partials
    bool net_loaded = false;
    float *d_param = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
    uint8_t *d_umma = nullptr;               // BF16 B operands of the tcgen05 network
    uint2 *d_range = nullptr;                // range records of the proposal render
    long long range_cap = 0;
    float *d_netpdf = nullptr;               // inverse-CDF proposal render: per ray 32 PDF bins, then T^ per ray
    long long netpdf_cap = 0;
    float *d_partial = nullptr, *d_loss_partial = nullptr;
    int partial_blocks = 0;
    long long adam_step = 0;
    // host delivery of multi-view renders: a stream for the device-to-host
    // copies, two image buffers (pixels each) and their events
    cudaStream_t copy_stream = nullptr;
    cudaStream_t aux_stream = nullptr;       // renders every other group
    float4 *d_img[2] = {nullptr, nullptr};
    size_t img_cap = 0;
    cudaEvent_t ev_rendered[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr;
    cudaEvent_t ev_stats[2] = {nullptr, nullptr};   // around a call that returns statistics
};

struct rc_volume {
    rc_context *ctx = nullptr;
    int n[3] = {0, 0, 0};
    float s[3] = {0, 0, 0};
    int vmax = 0;
    rc_storage storage = RC_STORE_F32;
    int cb[3] = {0, 0, 0};       // cell-bricks per axis (each stored as a 19^3 apron brick)
    int nbricks = 0;             // cell-bricks
    void *d_data = nullptr;
    void *d_vg = nullptr;        // value+gradient bricks (FP32; uint16 with vmax < 32768; FP16 with vmax <= 4096)
    void *d_pairs = nullptr;     // pair bricks (storage type), built on the first render that reads them
    uint64_t pairs_data_version = ~0ull;
    uint16_t *d_stage = nullptr;
    // min/max grid and occupancy mask per reconstruction filter (index rc_filter)
    uint16_t *d_mn[2] = {nullptr, nullptr}, *d_mx[2] = {nullptr, nullptr};
    uint8_t *d_occ[2] = {nullptr, nullptr};
    // 4^3 sub-block min/max grid and the fine mask of the trilinear compositing march
    uint16_t *d_mn4[2] = {nullptr, nullptr}, *d_mx4[2] = {nullptr, nullptr};
    unsigned long long *d_fine[2] = {nullptr, nullptr};
    bool uploaded = false;
    uint64_t data_version = 0;
    uint64_t grid_data_version[2] = {~0ull, ~0ull};
    uint64_t occ_tf_version[2] = {~0ull, ~0ull};
    uint64_t occ_data_version[2] = {~0ull, ~0ull};
};

static thread_local char g_err[512];

// Host-side fault injection for tests: with RC_FAULT_ALLOC=n in the
// environment, the n-th device allocation after the variable's text last
// changed fails with cudaErrorMemoryAllocation (the allocation is not
// attempted); "1", "01", "001" each re-arm for the first allocation. Off when
// unset or empty.
static std::mutex g_fault_mu;
static char g_fault_env[32] = "";
static long g_fault_left = -1;

template <typename T>
static cudaError_t dev_alloc(T **p, size_t bytes) {
    {
        std::lock_guard<std::mutex> lock(g_fault_mu);
        const char *e = getenv("RC_FAULT_ALLOC");
        if (!e) e = "";
        if (strncmp(e, g_fault_env, sizeof g_fault_env) != 0) {
            snprintf(g_fault_env, sizeof g_fault_env, "%s", e);
            g_fault_left = e[0] ? atol(e) : -1;
        }
        if (g_fault_left > 0 && --g_fault_left == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

static rc_status fail(rc_context *ctx, rc_status s, const char *fmt, ...) {
    char *buf = ctx ? ctx->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return s;
}

#define RC_CUDA(ctx, call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? RC_ERR_OOM : RC_ERR_CUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                         \
    } while (0)

// Makes ctx's device current for the scope of one call.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

constexpr int kStatSlots = 6;       // dense, evaluated, hit, total, (spare), error word

static int *error_word(rc_context *ctx) { return reinterpret_cast<int *>(ctx->d_stats + 5); }

// Clock budget of the tensor-core kernels' waits (about 1 s at 2 GHz). With
// RC_FAULT_MMA_WAIT set (tests only) the network kernel issues no MMA and
// waits 1 ms for a completion that never comes, so the timeout path runs.
static long long wait_budget(int *issue_mma) {
    const char *e = getenv("RC_FAULT_MMA_WAIT");
    const bool fault = e && *e;
    *issue_mma = fault ? 0 : 1;
    return fault ? 2000000ll : 2000000000ll;
}

// Reads and clears the device error word (synchronises the stream): bit 0,
// a bounded wait of a tensor-core kernel gave up (RC_ERR_TIMEOUT); bit 1, an
// index check of a debug build failed, with the sites in bits 8 and up
// (RC_ERR_CUDA).
static rc_status check_device_errors(rc_context *ctx, const char *who) {
    RC_CUDA(ctx, cudaMemcpyAsync(ctx->h_stats + 5, ctx->d_stats + 5, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const unsigned long long word = ctx->h_stats[5];
    if (word != 0) {
        RC_CUDA(ctx, cudaMemsetAsync(ctx->d_stats + 5, 0, sizeof(unsigned long long), ctx->stream));
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (word & 2)
            return fail(ctx, RC_ERR_CUDA,
                        "%s: a device index check failed (debug build; sites 0x%llx: 1 brick, 2 table, 4 2-D table); "
                        "the outputs of the launches since the last check are invalid",
                        who, (word >> 8) & 0xffull);
        return fail(ctx, RC_ERR_TIMEOUT, "%s: a tensor-core wait gave up (outputs of that launch are invalid)", who);
    }
    return RC_OK;
}

extern "C" {

const char *rc_status_string(rc_status s) {
    switch (s) {
        case RC_OK: return "ok";
        case RC_ERR_INVALID_ARG: return "invalid argument";
        case RC_ERR_OOM: return "out of memory";
        case RC_ERR_CUDA: return "CUDA error";
        case RC_ERR_STATE: return "invalid state";
        case RC_ERR_TIMEOUT: return "device wait timed out";
        case RC_ERR_UNSUPPORTED: return "unsupported";
        case RC_ERR_FORMAT: return "malformed data";
    }
    return "unknown status";
}

const char *rc_last_error(const rc_context *ctx) { return ctx ? ctx->err : g_err; }

rc_status rc_context_create(int device, void *cuda_stream, rc_context **out) {
    if (!out) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_context_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(nullptr, RC_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev)
        return fail(nullptr, RC_ERR_INVALID_ARG, "rc_context_create: device %d of %d", device, ndev);
    DeviceScope ds(device);
    if (!ds.ok) return fail(nullptr, RC_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    rc_context *ctx = new (std::nothrow) rc_context();
    if (!ctx) return fail(nullptr, RC_ERR_OOM, "rc_context_create: host allocation");
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (dev_alloc(&ctx->d_stats, kStatSlots * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_stats, kStatSlots * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->d_stats, 0, kStatSlots * sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(ctx->d_stats);
        cudaFreeHost(ctx->h_stats);
        delete ctx;
        return fail(nullptr, RC_ERR_OOM, "rc_context_create: statistics buffers");
    }
    *out = ctx;
    return RC_OK;
}

rc_status rc_context_set_stream(rc_context *ctx, void *cuda_stream) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_context_set_stream: ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return RC_OK;
}

rc_status rc_context_destroy(rc_context *ctx) {
    if (!ctx) return RC_OK;
    if (ctx->nvolumes > 0) return fail(ctx, RC_ERR_STATE, "rc_context_destroy: %d volumes still alive", ctx->nvolumes);
    DeviceScope ds(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_tf32);
    cudaFree(ctx->d_tf16);
    cudaFree(ctx->d_tf2);
    cudaFree(ctx->d_amax);
    cudaFree(ctx->d_stats);
    cudaFree(ctx->d_cams);
    cudaFree(ctx->d_batch);
    cudaFreeHost(ctx->h_stats);
    cudaFreeHost(ctx->h_tfstage);
    if (ctx->ev_tfstage) cudaEventDestroy(ctx->ev_tfstage);
    cudaFree(ctx->d_scratch);
    cudaFree(ctx->d_param);
    cudaFree(ctx->d_m);
    cudaFree(ctx->d_v);
    cudaFree(ctx->d_grad);
    cudaFree(ctx->d_umma);
    cudaFree(ctx->d_range);
    cudaFree(ctx->d_netpdf);
    cudaFree(ctx->d_partial);
    cudaFree(ctx->d_loss_partial);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    if (ctx->aux_stream) cudaStreamSynchronize(ctx->aux_stream);
    for (int b = 0; b < 2; b++) {
        cudaFree(ctx->d_img[b]);
        if (ctx->ev_rendered[b]) cudaEventDestroy(ctx->ev_rendered[b]);
        if (ctx->ev_copied[b]) cudaEventDestroy(ctx->ev_copied[b]);
    }
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    for (int i = 0; i < 2; i++)
        if (ctx->ev_stats[i]) cudaEventDestroy(ctx->ev_stats[i]);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    delete ctx;
    return RC_OK;
}

// ---------------------------------------------------------------------------
// volumes
// ---------------------------------------------------------------------------
static void volume_free(rc_volume *v) {
    cudaFree(v->d_data);
    cudaFree(v->d_vg);
    cudaFree(v->d_pairs);
    cudaFree(v->d_stage);
    for (int f = 0; f < 2; f++) {
        cudaFree(v->d_mn[f]);
        cudaFree(v->d_mx[f]);
        cudaFree(v->d_occ[f]);
    }
    for (int f = 0; f < 2; f++) {
        cudaFree(v->d_mn4[f]);
        cudaFree(v->d_mx4[f]);
        cudaFree(v->d_fine[f]);
    }
}

rc_status rc_volume_create(rc_context *ctx, int nx, int ny, int nz, float sx, float sy, float sz, uint16_t vmax,
                           rc_storage storage, rc_volume **out) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_volume_create: ctx is NULL");
    if (!out) return fail(ctx, RC_ERR_INVALID_ARG, "rc_volume_create: out is NULL");
    *out = nullptr;
    if (nx < 2 || ny < 2 || nz < 2)
        return fail(ctx, RC_ERR_INVALID_ARG, "rc_volume_create: dims %d x %d x %d (each must be >= 2)", nx, ny, nz);
    if (!(sx > 0.0f && sy > 0.0f && sz > 0.0f) || !isfinite(sx) || !isfinite(sy) || !isfinite(sz))
        return fail(ctx, RC_ERR_INVALID_ARG, "rc_volume_create: spacing must be finite and > 0");
    if (vmax < 1) return fail(ctx, RC_ERR_INVALID_ARG, "rc_volume_create: vmax must be >= 1");
    if (storage != RC_STORE_F32 && storage != RC_STORE_F16 && storage != RC_STORE_U16)
        return fail(ctx, RC_ERR_INVALID_ARG, "rc_volume_create: storage %d", (int)storage);
    const int cbx = (nx - 1 + 15) / 16, cby = (ny - 1 + 15) / 16, cbz = (nz - 1 + 15) / 16;
    long long padded = (long long)cbx * cby * cbz * kApronVox;
    if (padded >= (1ll << 31))
        return fail(ctx, RC_ERR_UNSUPPORTED, "rc_volume_create: %lld stored voxels (limit 2^31)", padded);
    DeviceScope ds(ctx->device);
    rc_volume *v = new (std::nothrow) rc_volume();
    if (!v) return fail(ctx, RC_ERR_OOM, "rc_volume_create: host allocation");
    v->ctx = ctx;
    v->n[0] = nx; v->n[1] = ny; v->n[2] = nz;
    v->s[0] = sx; v->s[1] = sy; v->s[2] = sz;
    v->vmax = vmax;
    v->storage = storage;
    for (int a = 0; a < 3; a++) v->cb[a] = (v->n[a] - 1 + 15) / 16;
    v->nbricks = v->cb[0] * v->cb[1] * v->cb[2];
    size_t esz = storage == RC_STORE_F32 ? 4 : 2;
    size_t nvox = (size_t)nx * ny * nz;
    // value+gradient bricks: FP32 storage; uint16 storage while the central
    // differences fit 16 bits (vmax < 32768); FP16 storage while every stored
    // value is exact (vmax <= 4096: offset o <= 2048), so that the differences
    // of stored values are integer code differences / o
    const size_t vg_bytes = storage == RC_STORE_F32 ? (size_t)v->nbricks * kGradVox * sizeof(float4)
                            : (storage == RC_STORE_U16 && vmax < 32768) || (storage == RC_STORE_F16 && vmax <= 4096)
                                ? (size_t)v->nbricks * kGradVox * sizeof(uint2)
                                : 0;
    const size_t n4 = (size_t)((nx - 1 + 3) / 4) * ((ny - 1 + 3) / 4) * ((nz - 1 + 3) / 4);
    if (dev_alloc(&v->d_data, (size_t)padded * esz) != cudaSuccess ||
        (vg_bytes && dev_alloc(&v->d_vg, vg_bytes) != cudaSuccess) ||
        dev_alloc(&v->d_stage, nvox * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_mn[0], v->nbricks * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_mx[0], v->nbricks * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_occ[0], v->nbricks) != cudaSuccess ||
        dev_alloc(&v->d_mn[1], v->nbricks * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_mx[1], v->nbricks * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_occ[1], v->nbricks) != cudaSuccess ||
        dev_alloc(&v->d_mn4[0], n4 * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_mx4[0], n4 * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_fine[0], v->nbricks * sizeof(unsigned long long)) != cudaSuccess ||
        dev_alloc(&v->d_mn4[1], n4 * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_mx4[1], n4 * sizeof(uint16_t)) != cudaSuccess ||
        dev_alloc(&v->d_fine[1], v->nbricks * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        volume_free(v);
        delete v;
        return fail(ctx, RC_ERR_OOM, "rc_volume_create: device allocation (%lld voxels)", padded);
    }
    ctx->nvolumes++;
    *out = v;
    return RC_OK;
}

// FP16 storage holds h = (code - o) / o with o the smallest power of two
// (>= 1) for which 2o >= vmax: every code 0 .. min(vmax, 4096) then has
// |code - o| <= 2048, an integer FP16 represents exactly, so h is exact.
static int f16_offset(int vmax) {
    int o = 1;
    while (2 * o < vmax) o *= 2;
    return o;
}

// Full scale of the stored values: vmax for raw codes, vmax / o for FP16.
static float full_scale(const rc_volume *v) {
    return v->storage == RC_STORE_F16 ? (float)v->vmax / (float)f16_offset(v->vmax) : (float)v->vmax;
}

static VolDev vol_dev(const rc_volume *v) {
    VolDev d;
    d.data = v->d_data;
    d.vg = v->d_vg;
    d.pairs = v->pairs_data_version == v->data_version ? v->d_pairs : nullptr;
    d.storage = (int)v->storage;
    float smin = fminf(fminf(v->s[0], v->s[1]), v->s[2]);
    for (int a = 0; a < 3; a++) {
        d.n[a] = v->n[a];
        d.cb[a] = v->cb[a];
        d.s[a] = v->s[a];
        d.inv2s[a] = 0.5f / v->s[a];
    }
    d.smin = smin;
    d.vmax = v->vmax;
    d.vscale = full_scale(v);
    d.f16o = v->storage == RC_STORE_F16 ? (float)f16_offset(v->vmax) : 0.0f;
    d.gmin = 1e-6f * d.vscale;
#ifdef RC_DEBUG
    // debug builds: the kernels' index checks report to the context's error
    // word; RC_DEBUG_POISON (tests) moves every brick index out of range, so
    // that every check fires and replaces the index by 0
    d.dbg_err = error_word(v->ctx);
    const char *poison = getenv("RC_DEBUG_POISON");
    d.dbg_poison = poison && *poison ? v->nbricks : 0;
#endif
    return d;
}

rc_status rc_volume_upload(rc_volume *v, const uint16_t *src, size_t n_voxels, int src_is_device) {
    if (!v) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_volume_upload: vol is NULL");
    rc_context *ctx = v->ctx;
    if (!src) return fail(ctx, RC_ERR_INVALID_ARG, "rc_volume_upload: src is NULL");
    size_t nvox = (size_t)v->n[0] * v->n[1] * v->n[2];
    if (n_voxels != nvox)
        return fail(ctx, RC_ERR_INVALID_ARG, "rc_volume_upload: %zu voxels given, volume has %zu", n_voxels, nvox);
    DeviceScope ds(ctx->device);
    RC_CUDA(ctx, cudaMemcpyAsync(v->d_stage, src, nvox * sizeof(uint16_t),
                                 src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    // apron bricks, value+gradient bricks and the trilinear grids in one pass
    // over the staged codes (one block per cell-brick)
    RC_CUDA(ctx, launch_prep(v->d_stage, vol_dev(v), v->d_data, v->d_vg, v->d_mn[0], v->d_mx[0], v->d_mn4[0],
                             v->d_mx4[0], ctx->stream));
    v->uploaded = true;
    v->data_version++;
    v->grid_data_version[RC_FILTER_TRILINEAR] = v->data_version;   // the B-spline grid is built on first use
    return RC_OK;
}

rc_status rc_volume_destroy(rc_volume *v) {
    if (!v) return RC_OK;
    rc_context *ctx = v->ctx;
    DeviceScope ds(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    volume_free(v);
    ctx->nvolumes--;
    delete v;
    return RC_OK;
}

rc_status rc_volume_brick_dims(const rc_volume *v, int dims[3]) {
    if (!v || !dims) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_volume_brick_dims: NULL argument");
    for (int a = 0; a < 3; a++) dims[a] = v->cb[a];
    return RC_OK;
}

// ---------------------------------------------------------------------------
// transfer function and camera
// ---------------------------------------------------------------------------
static rc_status tf_reserve(rc_context *ctx, int K) {
    if (K <= ctx->tf_cap) return RC_OK;
    float4 *a = nullptr;
    uint2 *b = nullptr;
    if (dev_alloc(&a, (size_t)K * sizeof(float4)) != cudaSuccess ||
        dev_alloc(&b, (size_t)K * sizeof(uint2)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(a);
        return fail(ctx, RC_ERR_OOM, "rc_tf_set: device allocation");
    }
    // the old tables may still be read by queued kernels
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_tf32);
    cudaFree(ctx->d_tf16);
    ctx->d_tf32 = a;
    ctx->d_tf16 = b;
    ctx->tf_cap = K;
    return RC_OK;
}

__global__ void tf_to_half_kernel(const float4 *src, uint2 *dst, int K) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    float4 v = src[i];
    __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
    uint2 o;
    o.x = *reinterpret_cast<unsigned *>(&lo);
    o.y = *reinterpret_cast<unsigned *>(&hi);
    dst[i] = o;
}

// Copies a host table to device memory on the context's stream without
// waiting for the work queued before it: through a page-locked staging
// buffer owned by the context (the caller's memory may be reused as soon as
// the call returns). The buffer is reused once its previous copy has run,
// which in a frame loop happened before the previous frame's render.
static rc_status stage_table(rc_context *ctx, void *dst, const void *src, size_t bytes) {
    if (ctx->tfstage_pending) {
        RC_CUDA(ctx, cudaEventSynchronize(ctx->ev_tfstage));
        ctx->tfstage_pending = false;
    }
    if (!ctx->ev_tfstage) RC_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_tfstage, cudaEventDisableTiming));
    if (bytes > ctx->tfstage_cap) {
        void *nb = nullptr;
        RC_CUDA(ctx, cudaMallocHost(&nb, bytes));
        cudaFreeHost(ctx->h_tfstage);
        ctx->h_tfstage = nb;
        ctx->tfstage_cap = bytes;
    }
    memcpy(ctx->h_tfstage, src, bytes);
    RC_CUDA(ctx, cudaMemcpyAsync(dst, ctx->h_tfstage, bytes, cudaMemcpyHostToDevice, ctx->stream));
    RC_CUDA(ctx, cudaEventRecord(ctx->ev_tfstage, ctx->stream));
    ctx->tfstage_pending = true;
    return RC_OK;
}

static rc_status tf_common(rc_context *ctx, const float *rgba, int K, int fp16, bool dev) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_tf_set: ctx is NULL");
    if (!rgba) return fail(ctx, RC_ERR_INVALID_ARG, "rc_tf_set: rgba is NULL");
    if (K < 2 || K > 4096) return fail(ctx, RC_ERR_INVALID_ARG, "rc_tf_set: %d entries (2..4096)", K);
    if (!dev) {
        for (int i = 0; i < 4 * K; i++)
            if (!(rgba[i] >= 0.0f && rgba[i] <= 1.0f))
                return fail(ctx, RC_ERR_INVALID_ARG, "rc_tf_set: entry %d channel %d = %g outside [0, 1]", i / 4,
                            i % 4, (double)rgba[i]);
    }
    DeviceScope ds(ctx->device);
    rc_status st = tf_reserve(ctx, K);
    if (st != RC_OK) return st;
    if (dev) {
        RC_CUDA(ctx, cudaMemcpyAsync(ctx->d_tf32, rgba, (size_t)K * sizeof(float4), cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    } else {
        st = stage_table(ctx, ctx->d_tf32, rgba, (size_t)K * sizeof(float4));
        if (st != RC_OK) return st;
    }
    tf_to_half_kernel<<<(K + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_tf32, ctx->d_tf16, K);
    RC_CUDA(ctx, cudaGetLastError());
    ctx->K = K;
    ctx->M = 0;
    ctx->tf_fp16 = fp16 ? 1 : 0;
    ctx->tf_version++;
    return RC_OK;
}

// 2-D table: FP16 rounding of the entries in place (the FP16 table holds
// exactly these values), and per value entry the largest opacity over the rows.
__global__ void tf2_round_half_kernel(float4 *t, long long n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float4 v = t[e];
    v.x = __half2float(__float2half_rn(v.x));
    v.y = __half2float(__float2half_rn(v.y));
    v.z = __half2float(__float2half_rn(v.z));
    v.w = __half2float(__float2half_rn(v.w));
    t[e] = v;
}

__global__ void tf2_amax_kernel(const float4 *t, int K, int M, float *amax) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    float m = 0.0f;
    for (int j = 0; j < M; j++) m = fmaxf(m, t[(size_t)j * K + i].w);
    amax[i] = m;
}

rc_status rc_tf_set(rc_context *ctx, const float *rgba, int n_entries, int fp16) {
    return tf_common(ctx, rgba, n_entries, fp16, false);
}

rc_status rc_tf_set_device(rc_context *ctx, const float *rgba_dev, int n_entries, int fp16) {
    return tf_common(ctx, rgba_dev, n_entries, fp16, true);
}

static rc_status tf2_common(rc_context *ctx, const float *rgba, int K, int M, float gmax, int fp16, bool dev) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_tf2d_set: ctx is NULL");
    if (!rgba) return fail(ctx, RC_ERR_INVALID_ARG, "rc_tf2d_set: rgba is NULL");
    if (K < 2 || K > 4096 || M < 2 || M > 4096 || (long long)K * M > (1ll << 20))
        return fail(ctx, RC_ERR_INVALID_ARG, "rc_tf2d_set: %d x %d entries (2..4096 each, at most 2^20)", K, M);
    if (!(gmax > 0.0f) || !isfinite(gmax)) return fail(ctx, RC_ERR_INVALID_ARG, "rc_tf2d_set: gmax %g", (double)gmax);
    const long long n = (long long)K * M;
    if (!dev) {
        for (long long i = 0; i < 4 * n; i++)
            if (!(rgba[i] >= 0.0f && rgba[i] <= 1.0f))
                return fail(ctx, RC_ERR_INVALID_ARG, "rc_tf2d_set: entry %lld channel %lld = %g outside [0, 1]",
                            i / 4, i % 4, (double)rgba[i]);
    }
    DeviceScope ds(ctx->device);
    if (n > ctx->tf2_cap) {
        float4 *t = nullptr;
        float *am = nullptr;
        const long long cap = n;   // > K: also holds the K opacity maxima
        if (dev_alloc(&t, (size_t)cap * sizeof(float4)) != cudaSuccess ||
            dev_alloc(&am, (size_t)cap * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(t);
            return fail(ctx, RC_ERR_OOM, "rc_tf2d_set: device allocation");
        }
        cudaStreamSynchronize(ctx->stream);   // queued kernels may still read the old table
        cudaFree(ctx->d_tf2);
        cudaFree(ctx->d_amax);
        ctx->d_tf2 = t;
        ctx->d_amax = am;
        ctx->tf2_cap = cap;
    }
    if (dev) {
        RC_CUDA(ctx, cudaMemcpyAsync(ctx->d_tf2, rgba, (size_t)n * sizeof(float4), cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    } else {
        rc_status st = stage_table(ctx, ctx->d_tf2, rgba, (size_t)n * sizeof(float4));
        if (st != RC_OK) return st;
    }
    if (fp16) {
        tf2_round_half_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->d_tf2, n);
        RC_CUDA(ctx, cudaGetLastError());
    }
    tf2_amax_kernel<<<(K + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_tf2, K, M, ctx->d_amax);
    RC_CUDA(ctx, cudaGetLastError());
    ctx->K = K;
    ctx->M = M;
    ctx->gmax = gmax;
    ctx->tf_fp16 = fp16 ? 1 : 0;
    ctx->tf_version++;
    return RC_OK;
}

rc_status rc_tf2d_set(rc_context *ctx, const float *rgba, int K, int M, float gmax, int fp16) {
    return tf2_common(ctx, rgba, K, M, gmax, fp16, false);
}

rc_status rc_tf2d_set_device(rc_context *ctx, const float *rgba_dev, int K, int M, float gmax, int fp16) {
    return tf2_common(ctx, rgba_dev, K, M, gmax, fp16, true);
}

static rc_status check_camera(rc_context *ctx, const rc_camera *cam, const char *who) {
    if (cam->width < 1 || cam->height < 1 || (long long)cam->width * cam->height > (1ll << 28))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: image %d x %d", who, cam->width, cam->height);
    if (!(cam->fovy_deg > 0.0f && cam->fovy_deg < 180.0f))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: fovy %g", who, (double)cam->fovy_deg);
    double f[3], up[3], c[3];
    for (int a = 0; a < 3; a++) {
        if (!isfinite(cam->eye[a]) || !isfinite(cam->target[a]) || !isfinite(cam->up[a]))
            return fail(ctx, RC_ERR_INVALID_ARG, "%s: non-finite vector", who);
        f[a] = (double)cam->target[a] - (double)cam->eye[a];
        up[a] = cam->up[a];
    }
    c[0] = f[1] * up[2] - f[2] * up[1];
    c[1] = f[2] * up[0] - f[0] * up[2];
    c[2] = f[0] * up[1] - f[1] * up[0];
    if (f[0] * f[0] + f[1] * f[1] + f[2] * f[2] == 0.0 || c[0] * c[0] + c[1] * c[1] + c[2] * c[2] == 0.0)
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: eye == target or up parallel to the view", who);
    return RC_OK;
}

rc_status rc_camera_set(rc_context *ctx, const rc_camera *cam) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_camera_set: ctx is NULL");
    if (!cam) return fail(ctx, RC_ERR_INVALID_ARG, "rc_camera_set: cam is NULL");
    rc_status st = check_camera(ctx, cam, "rc_camera_set");
    if (st != RC_OK) return st;
    ctx->cam = *cam;
    ctx->cam_set = true;
    return RC_OK;
}

// Camera record: look-at basis in FP64 (f = normalize(target - eye),
// r = normalize(f x up), u = r x f), rounded once to FP32; eye in index space.
static CamRec camera_record(const rc_camera &cam, const float s[3]) {
    double f[3], up[3], r[3], u[3];
    for (int a = 0; a < 3; a++) {
        f[a] = (double)cam.target[a] - (double)cam.eye[a];
        up[a] = (double)cam.up[a];
    }
    double n = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int a = 0; a < 3; a++) f[a] /= n;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    n = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; a++) r[a] /= n;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    double th = tan((double)cam.fovy_deg * 3.14159265358979323846 / 360.0);
    double tx = th * (double)cam.width / (double)cam.height;
    CamRec c;
    for (int a = 0; a < 3; a++) {
        c.f[a] = (float)f[a];
        c.r[a] = (float)r[a];
        c.u[a] = (float)u[a];
        c.o[a] = (float)((double)cam.eye[a] / (double)s[a]);
    }
    c.tx = (float)tx;
    c.ty = (float)th;
    c.W = cam.width;
    c.H = cam.height;
    return c;
}

// ---------------------------------------------------------------------------
// rendering
// ---------------------------------------------------------------------------
static rc_status check_render(rc_context *ctx, const rc_volume *v, const rc_render_params *p, const void *out,
                              const char *who) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    if (!v || !p || !out) return fail(ctx, RC_ERR_INVALID_ARG, "%s: NULL argument", who);
    if (v->ctx != ctx) return fail(ctx, RC_ERR_INVALID_ARG, "%s: volume belongs to another context", who);
    if (!(p->step_vox >= 1e-3f) || !isfinite(p->step_vox))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: step_vox %g", who, (double)p->step_vox);
    if (!(p->term > 0.0f && p->term <= 1.0f)) return fail(ctx, RC_ERR_INVALID_ARG, "%s: term %g", who, (double)p->term);
    if (p->shade != 0 && p->shade != 1) return fail(ctx, RC_ERR_INVALID_ARG, "%s: shade %d", who, p->shade);
    if (p->skip != 0 && p->skip != 1) return fail(ctx, RC_ERR_INVALID_ARG, "%s: skip %d", who, p->skip);
    if (p->func < RC_FUNC_COMPOSITE || p->func > RC_FUNC_THRESHOLD)
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: func %d", who, p->func);
    if (p->filter != RC_FILTER_TRILINEAR && p->filter != RC_FILTER_BSPLINE)
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: filter %d", who, p->filter);
    if (!isfinite(p->ka) || !isfinite(p->kd) || !isfinite(p->ks) || p->ka < 0 || p->kd < 0 || p->ks < 0 ||
        !isfinite(p->iso))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: shading weights / iso", who);
    if (!v->uploaded) return fail(ctx, RC_ERR_STATE, "%s: volume has no data (call rc_volume_upload)", who);
    if (ctx->K < 2) return fail(ctx, RC_ERR_STATE, "%s: no transfer function (call rc_tf_set)", who);
    if (!ctx->cam_set) return fail(ctx, RC_ERR_STATE, "%s: no camera (call rc_camera_set)", who);
    if (v->storage != RC_STORE_F16 && (long long)(ctx->K - 1) * v->vmax >= (1ll << 24))
        return fail(ctx, RC_ERR_UNSUPPORTED, "%s: (entries - 1) * vmax must stay below 2^24", who);
    if (ctx->M >= 2 && p->func == RC_FUNC_THRESHOLD)
        return fail(ctx, RC_ERR_UNSUPPORTED, "%s: thresholding classifies with a 1-D table only", who);
    return RC_OK;
}

// A set of views: 1..65535 valid cameras of one image size, at most 2^31
// pixels in all.
static rc_status check_views(rc_context *ctx, const rc_camera *cams, int nviews, const char *who) {
    if (!cams || nviews < 1 || nviews > 65535)
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: %d cameras", who, cams ? nviews : 0);
    for (int i = 0; i < nviews; i++) {
        rc_status st = check_camera(ctx, &cams[i], who);
        if (st != RC_OK) return st;
        if (cams[i].width != cams[0].width || cams[i].height != cams[0].height)
            return fail(ctx, RC_ERR_INVALID_ARG, "%s: camera %d has another image size", who, i);
    }
    if ((long long)nviews * cams[0].width * cams[0].height > (1ll << 31))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: %d views of %d x %d pixels", who, nviews, cams[0].width,
                    cams[0].height);
    return RC_OK;
}

// Copies the views' camera records (for volume v) to the context's device
// array, growing it when needed; *first receives record 0.
static rc_status upload_views(rc_context *ctx, const rc_volume *v, const rc_camera *cams, int nviews, CamRec *first,
                              const char *who) {
    if (ctx->cams_cap < nviews) {
        CamRec *buf = nullptr;
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // queued kernels may still read the old records
        RC_CUDA(ctx, dev_alloc(&buf, (size_t)nviews * sizeof(CamRec)));
        cudaFree(ctx->d_cams);
        ctx->d_cams = buf;
        ctx->cams_cap = nviews;
    }
    CamRec *recs = new (std::nothrow) CamRec[nviews];
    if (!recs) return fail(ctx, RC_ERR_OOM, "%s: host allocation", who);
    for (int i = 0; i < nviews; i++) recs[i] = camera_record(cams[i], v->s);
    // pageable source: the copy is staged before the call returns
    cudaError_t ce = cudaMemcpyAsync(ctx->d_cams, recs, (size_t)nviews * sizeof(CamRec), cudaMemcpyHostToDevice,
                                     ctx->stream);
    *first = recs[0];
    delete[] recs;
    RC_CUDA(ctx, ce);
    return RC_OK;
}

// The render checks with cams[0] standing in for the context's camera.
static rc_status check_render_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                    const rc_camera *cams, const void *out, const char *who) {
    const bool had = ctx->cam_set;
    const rc_camera keep = ctx->cam;
    ctx->cam = cams[0];
    ctx->cam_set = true;
    rc_status st = check_render(ctx, vol, p, out, who);
    ctx->cam = keep;
    ctx->cam_set = had;
    return st;
}

// Entries of the current table: K for a 1-D table, M x K for a 2-D one.
static size_t tf_entries(const rc_context *ctx) {
    return (size_t)ctx->K * (ctx->M >= 2 ? ctx->M : 1);
}

// The table gradient's scratch: 4 fixed-point accumulators per table entry
// and the |dL/dI| maximum, grown (never shrunk) after the stream drains.
static rc_status ensure_grad_scratch(rc_context *ctx) {
    const size_t need = 4 * tf_entries(ctx) * sizeof(long long) + 16;
    if (ctx->scratch_bytes < need) {
        void *buf = nullptr;
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        RC_CUDA(ctx, dev_alloc(&buf, need));
        cudaFree(ctx->d_scratch);
        ctx->d_scratch = buf;
        ctx->scratch_bytes = need;
    }
    return RC_OK;
}

// The learned proposal marches trilinear samples classified by a 1-D table.
static rc_status check_plain_form(rc_context *ctx, const rc_render_params *p, const char *who) {
    if (p->filter != RC_FILTER_TRILINEAR)
        return fail(ctx, RC_ERR_UNSUPPORTED, "%s: trilinear reconstruction only", who);
    if (ctx->M >= 2) return fail(ctx, RC_ERR_UNSUPPORTED, "%s: 1-D transfer function only", who);
    return RC_OK;
}

// The table with its coordinate coefficients for volume v: ucoef = fl((K-1) / vscale)
// (u = fl(v ucoef) for raw codes, fl((h + 1) ucoef) for FP16 values), and for
// a 2-D table w = fl(|g| * fl((M-1) * vmax / (vscale * gmax))), vscale the
// full scale in stored units.
static TFDev tf_dev(const rc_context *ctx, const rc_volume *v) {
    const float vscale = full_scale(v);
    TFDev t{};
    t.K = ctx->K;
    t.fp16 = ctx->tf_fp16;
    t.ucoef = (float)(ctx->K - 1) / vscale;
    if (ctx->M >= 2) {
        t.tab2 = ctx->d_tf2;
        t.amax = ctx->d_amax;
        t.M = ctx->M;
        t.wcoef = (float)((double)(ctx->M - 1) * (double)v->vmax / ((double)vscale * (double)ctx->gmax));
    } else {
        t.f32 = ctx->d_tf32;
        t.f16 = ctx->d_tf16;
    }
    return t;
}

// The min/max grid of filter f, built from the staging copy of the codes when
// the data changed since it was last built.
static rc_status ensure_grid(rc_context *ctx, rc_volume *v, int f) {
    if (v->grid_data_version[f] == v->data_version) return RC_OK;
    RC_CUDA(ctx, launch_minmax(v->d_stage, v->n, v->cb, v->vmax, f, v->d_mn[f], v->d_mx[f], ctx->stream));
    RC_CUDA(ctx, launch_minmax4(v->d_stage, v->n, v->vmax, f, v->d_mn4[f], v->d_mx4[f], ctx->stream));
    v->grid_data_version[f] = v->data_version;
    return RC_OK;
}

// The pair bricks of FP32 and FP16 volumes, allocated on the first render
// that reads them and rebuilt after new data: B-spline renders, and
// trilinear renders of FP16 volumes that need the gradient footprint
// (shading, a 2-D table, the isosurface's shading). FP32 trilinear renders
// read the value+gradient bricks; uint16 volumes read the apron bricks
// (widening 16-bit integer pairs cost more than the loads they save).
static rc_status prepare_filter(rc_context *ctx, rc_volume *v, const rc_render_params *p) {
    const bool grad = p->shade || ctx->M >= 2 || p->func == RC_FUNC_ISO;
    const bool need = v->storage != RC_STORE_U16 &&
                      (p->filter == RC_FILTER_BSPLINE || (v->storage == RC_STORE_F16 && grad));
    if (!need || v->pairs_data_version == v->data_version) return RC_OK;
    const size_t esz = v->storage == RC_STORE_F32 ? 4 : 2;
    if (!v->d_pairs) RC_CUDA(ctx, dev_alloc(&v->d_pairs, (size_t)v->nbricks * kPairVox * 2 * esz));
    RC_CUDA(ctx, launch_pairs(vol_dev(v), v->d_pairs, ctx->stream));
    v->pairs_data_version = v->data_version;
    return RC_OK;
}

// The occupancy mask of filter f under the current table, rebuilt when the
// table or the data changed since it was last built.
static rc_status ensure_occupancy(rc_context *ctx, rc_volume *v, int f) {
    if (v->occ_tf_version[f] == ctx->tf_version && v->occ_data_version[f] == v->data_version) return RC_OK;
    rc_status st = ensure_grid(ctx, v, f);
    if (st != RC_OK) return st;
    TFDev tf = tf_dev(ctx, v);
    const int f16o = v->storage == RC_STORE_F16 ? f16_offset(v->vmax) : 0;
    RC_CUDA(ctx, launch_occupancy(v->d_mn[f], v->d_mx[f], v->nbricks, v->vmax, f16o, tf, v->d_occ[f], ctx->stream));
    RC_CUDA(ctx, launch_finemask(v->d_mn4[f], v->d_mx4[f], v->n, v->cb, v->vmax, f16o, tf, v->d_fine[f],
                                 ctx->stream));
    v->occ_tf_version[f] = ctx->tf_version;
    v->occ_data_version[f] = v->data_version;
    return RC_OK;
}

// Copies the device counters into *stats (synchronises the stream). The
// importance kernels count fallback rays in the first slot.
// Zeroes the statistics counters and marks the start of a call's device work
// on the context's stream (read_stats marks its end).
static cudaError_t stats_begin(rc_context *ctx) {
    cudaError_t e = cudaMemsetAsync(ctx->d_stats, 0, 5 * sizeof(unsigned long long), ctx->stream);
    for (int i = 0; i < 2 && e == cudaSuccess; i++)
        if (!ctx->ev_stats[i]) e = cudaEventCreate(&ctx->ev_stats[i]);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_stats[0], ctx->stream);
    return e;
}

static rc_status read_stats(rc_context *ctx, rc_stats *stats, bool importance) {
    RC_CUDA(ctx, cudaEventRecord(ctx->ev_stats[1], ctx->stream));
    RC_CUDA(ctx, cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    rc_status st = check_device_errors(ctx, "statistics");
    if (st != RC_OK) return st;
    float ms = 0.0f;
    RC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_stats[0], ctx->ev_stats[1]));
    stats->device_ms = ms;
    stats->dense_samples = importance ? 0 : ctx->h_stats[0];
    stats->evaluated_samples = ctx->h_stats[1];
    stats->rays_hit = ctx->h_stats[2];
    stats->rays_total = ctx->h_stats[3];
    stats->fallback_rays = importance ? ctx->h_stats[0] : 0;
    return RC_OK;
}

// The march of rc_render and rc_render_views. RC_MARCH_STAGED=1 in the
// environment selects, for the forms it covers (FP32 storage, shaded,
// trilinear, 1-D table, skipping on), the brick-staged variant
// (rc_march_staged.cu): the same images, kept to measure shared-memory
// staging against the cached gathers. A bulk copy that does not complete
// within its bounded wait is reported as RC_ERR_TIMEOUT at the next sync.
static cudaError_t launch_march_any(rc_context *ctx, const MarchArgs &a, int nviews) {
    const char *e = getenv("RC_MARCH_STAGED");
    if (e && e[0] == '1' && e[1] == 0 && staged_eligible(a))
        return launch_march_staged(a, nviews, error_word(ctx), 2000000000ll, ctx->stream);
    return launch_march(a, nviews, ctx->stream);
}

static MarchArgs march_args(rc_context *ctx, const rc_volume *v, const rc_render_params *p, float *out) {
    MarchArgs a;
    a.vol = vol_dev(v);
    a.cam = camera_record(ctx->cam, v->s);
    a.tf = tf_dev(ctx, v);
    a.p.step_vox = p->step_vox;
    a.p.term = p->term;
    a.p.shade = p->shade;
    a.p.ka = p->ka;
    a.p.kd = p->kd;
    a.p.ks = p->ks;
    a.p.func = p->func;
    // the iso-value in stored units: (iso - o) / o for FP16 values
    const float o = (float)f16_offset(v->vmax);
    a.p.iso = p->func == RC_FUNC_ISO || p->func == RC_FUNC_THRESHOLD
                  ? (v->storage == RC_STORE_F16 ? (p->iso - o) / o : p->iso)
                  : p->iso;
    a.p.skip = p->skip;
    // ds / ds_ref, with ds = step * smin rounded in FP32 as on the device
    float ds = p->step_vox * a.vol.smin;
    a.p.ratio = ds / a.vol.smin;
    a.p.rmode = a.p.ratio == 1.0f ? 0 : a.p.ratio == 0.5f ? 1 : a.p.ratio == 0.25f ? 2 : 3;
    a.p.filter = p->filter;
    a.occ = v->d_occ[p->filter];
    a.fine = v->d_fine[p->filter];
    a.out = reinterpret_cast<float4 *>(out);
    a.stats = nullptr;
    a.cams = nullptr;
    a.batch = nullptr;
    a.views = 1;
    return a;
}

rc_status rc_render(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, float *out_rgba,
                    rc_stats *stats) {
    rc_status st = check_render(ctx, vol, p, out_rgba, "rc_render");
    if (st != RC_OK) return st;
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    if (p->skip && p->func == RC_FUNC_COMPOSITE) {
        st = ensure_occupancy(ctx, v, p->filter);
        if (st != RC_OK) return st;
    }
    st = prepare_filter(ctx, v, p);
    if (st != RC_OK) return st;
    MarchArgs a = march_args(ctx, v, p, out_rgba);
    if (stats) {
        RC_CUDA(ctx, stats_begin(ctx));
        a.stats = ctx->d_stats;
    }
    RC_CUDA(ctx, launch_march_any(ctx, a, 1));
    if (stats) return read_stats(ctx, stats, false);
    return RC_OK;
}

rc_status rc_render_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, const rc_camera *cams,
                          int nviews, float *out_rgba, rc_stats *stats) {
    const char *who = "rc_render_views";
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    rc_status st = check_views(ctx, cams, nviews, who);
    if (st == RC_OK) st = check_render_views(ctx, vol, p, cams, out_rgba, who);
    if (st != RC_OK) return st;
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    if (p->skip && p->func == RC_FUNC_COMPOSITE) {
        st = ensure_occupancy(ctx, v, p->filter);
        if (st != RC_OK) return st;
    }
    st = prepare_filter(ctx, v, p);
    if (st != RC_OK) return st;
    CamRec first;
    st = upload_views(ctx, v, cams, nviews, &first, who);
    if (st != RC_OK) return st;
    MarchArgs a = march_args(ctx, v, p, out_rgba);
    a.cam = first;
    a.cams = ctx->d_cams;
    if (stats) {
        RC_CUDA(ctx, stats_begin(ctx));
        a.stats = ctx->d_stats;
    }
    RC_CUDA(ctx, launch_march_any(ctx, a, nviews));
    if (stats) return read_stats(ctx, stats, false);
    return RC_OK;
}

// The copy and second render streams, events and two image buffers of
// `pixels` each.
static rc_status ensure_host_path(rc_context *ctx, size_t pixels) {
    if (!ctx->copy_stream) RC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    if (!ctx->aux_stream) RC_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
    if (!ctx->ev_start) RC_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
    for (int b = 0; b < 2; b++) {
        if (!ctx->ev_rendered[b]) RC_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_rendered[b], cudaEventDisableTiming));
        if (!ctx->ev_copied[b]) RC_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming));
    }
    if (ctx->img_cap < pixels) {
        // earlier copies may still read the old buffers
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->copy_stream));
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->aux_stream));
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int b = 0; b < 2; b++) {
            cudaFree(ctx->d_img[b]);
            ctx->d_img[b] = nullptr;
        }
        ctx->img_cap = 0;
        for (int b = 0; b < 2; b++) RC_CUDA(ctx, dev_alloc(&ctx->d_img[b], pixels * sizeof(float4)));
        ctx->img_cap = pixels;
    }
    return RC_OK;
}

constexpr long long kHostGroupPixels = 1ll << 21;

// Groups of g views alternate between the context's stream and the second
// render stream (each with its own image buffer), so a group starts while the
// previous one drains; each group is copied to the host on the copy stream.
// The context's stream continues after the last copy.
static rc_status render_groups_to_host(rc_context *ctx, MarchArgs a, int nviews, int g, long long px,
                                       float *host_rgba) {
    // the second stream starts after the work queued so far
    RC_CUDA(ctx, cudaEventRecord(ctx->ev_start, ctx->stream));
    RC_CUDA(ctx, cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_start, 0));
    const int ngroups = (nviews + g - 1) / g;
    for (int j = 0; j < ngroups; j++) {
        const int b = j & 1, v0 = j * g, nv = std::min(g, nviews - v0);
        cudaStream_t rs = b ? ctx->aux_stream : ctx->stream;
        // buffer b is free once the copy of group j - 2 is done
        if (j >= 2) RC_CUDA(ctx, cudaStreamWaitEvent(rs, ctx->ev_copied[b], 0));
        a.cams = ctx->d_cams + v0;
        a.out = ctx->d_img[b];
        RC_CUDA(ctx, launch_march(a, nv, rs));
        RC_CUDA(ctx, cudaEventRecord(ctx->ev_rendered[b], rs));
        RC_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_rendered[b], 0));
        RC_CUDA(ctx, cudaMemcpyAsync(host_rgba + (size_t)v0 * px * 4, ctx->d_img[b], (size_t)nv * px * sizeof(float4),
                                     cudaMemcpyDeviceToHost, ctx->copy_stream));
        RC_CUDA(ctx, cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
    }
    // copies complete in order, each after its group's render
    RC_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_copied[(ngroups - 1) & 1], 0));
    return RC_OK;
}

rc_status rc_render_views_host(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, const rc_camera *cams,
                               int nviews, int group, float *host_rgba, rc_stats *stats) {
    const char *who = "rc_render_views_host";
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    rc_status st = check_views(ctx, cams, nviews, who);
    if (st == RC_OK) st = check_render_views(ctx, vol, p, cams, host_rgba, who);
    if (st != RC_OK) return st;
    if (group < 0) return fail(ctx, RC_ERR_INVALID_ARG, "%s: group %d", who, group);
    DeviceScope ds(ctx->device);
    {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, host_rgba) != cudaSuccess) cudaGetLastError();
        else if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged)
            return fail(ctx, RC_ERR_INVALID_ARG, "%s: host_rgba is device memory (use rc_render_views)", who);
    }
    rc_volume *v = const_cast<rc_volume *>(vol);
    if (p->skip && p->func == RC_FUNC_COMPOSITE) {
        st = ensure_occupancy(ctx, v, p->filter);
        if (st != RC_OK) return st;
    }
    st = prepare_filter(ctx, v, p);
    if (st != RC_OK) return st;
    CamRec first;
    st = upload_views(ctx, v, cams, nviews, &first, who);
    if (st != RC_OK) return st;
    const long long px = (long long)cams[0].width * cams[0].height;
    const int g = group > 0 ? std::min(group, nviews)
                            : (int)std::min<long long>(nviews, std::max<long long>(1, (kHostGroupPixels + px - 1) / px));
    st = ensure_host_path(ctx, (size_t)g * px);
    if (st != RC_OK) return st;
    MarchArgs a = march_args(ctx, v, p, nullptr);
    a.cam = first;
    if (stats) {
        RC_CUDA(ctx, stats_begin(ctx));
        a.stats = ctx->d_stats;
    }
    st = render_groups_to_host(ctx, a, nviews, g, px, host_rgba);
    if (st != RC_OK) {
        // no copy into the caller's memory may outlive the call
        cudaStreamSynchronize(ctx->stream);
        cudaStreamSynchronize(ctx->aux_stream);
        cudaStreamSynchronize(ctx->copy_stream);
        return st;
    }
    if (stats) return read_stats(ctx, stats, false);
    return check_device_errors(ctx, who);
}

rc_status rc_render_batch(rc_context *ctx, const rc_volume *const *vols, int nvols, const rc_render_params *p,
                          const rc_camera *cams, int nviews, float *out_rgba, rc_stats *stats) {
    const char *who = "rc_render_batch";
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    if (!vols || nvols < 1) return fail(ctx, RC_ERR_INVALID_ARG, "%s: %d volumes", who, vols ? nvols : 0);
    rc_status st = check_views(ctx, cams, nviews, who);
    if (st != RC_OK) return st;
    if ((long long)nvols * nviews > 65535)
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: %d volumes x %d views (at most 65535)", who, nvols, nviews);
    if ((long long)nvols * nviews * cams[0].width * cams[0].height > (1ll << 31))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: more than 2^31 pixels", who);
    for (int i = 0; i < nvols; i++) {
        st = check_render_views(ctx, vols[i], p, cams, out_rgba, who);
        if (st != RC_OK) return st;
        const rc_volume *v = vols[i], *v0 = vols[0];
        if (v->storage != v0->storage || v->vmax != v0->vmax || v->n[0] != v0->n[0] || v->n[1] != v0->n[1] ||
            v->n[2] != v0->n[2] || v->s[0] != v0->s[0] || v->s[1] != v0->s[1] || v->s[2] != v0->s[2])
            return fail(ctx, RC_ERR_INVALID_ARG, "%s: volume %d differs from volume 0 in shape, spacing, vmax or "
                        "storage", who, i);
    }
    if (p->func != RC_FUNC_COMPOSITE) return fail(ctx, RC_ERR_UNSUPPORTED, "%s: compositing function only", who);
    DeviceScope ds(ctx->device);
    for (int i = 0; i < nvols; i++) {
        st = ensure_occupancy(ctx, const_cast<rc_volume *>(vols[i]), p->filter);
        if (st == RC_OK) st = prepare_filter(ctx, const_cast<rc_volume *>(vols[i]), p);
        if (st != RC_OK) return st;
    }
    CamRec first;
    st = upload_views(ctx, vols[0], cams, nviews, &first, who);
    if (st != RC_OK) return st;
    if (ctx->batch_cap < nvols) {
        BatchVol *buf = nullptr;
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // queued kernels may still read the old records
        RC_CUDA(ctx, dev_alloc(&buf, (size_t)nvols * sizeof(BatchVol)));
        cudaFree(ctx->d_batch);
        ctx->d_batch = buf;
        ctx->batch_cap = nvols;
    }
    BatchVol *recs = new (std::nothrow) BatchVol[nvols];
    if (!recs) return fail(ctx, RC_ERR_OOM, "%s: host allocation", who);
    for (int i = 0; i < nvols; i++)
        recs[i] = BatchVol{vols[i]->d_data, vols[i]->d_vg, vol_dev(vols[i]).pairs, vols[i]->d_occ[p->filter],
                           vols[i]->d_fine[p->filter]};
    cudaError_t ce = cudaMemcpyAsync(ctx->d_batch, recs, (size_t)nvols * sizeof(BatchVol), cudaMemcpyHostToDevice,
                                     ctx->stream);
    delete[] recs;
    RC_CUDA(ctx, ce);
    MarchArgs a = march_args(ctx, vols[0], p, out_rgba);
    a.cam = first;
    a.cams = ctx->d_cams;
    a.batch = ctx->d_batch;
    a.views = nviews;
    if (stats) {
        RC_CUDA(ctx, stats_begin(ctx));
        a.stats = ctx->d_stats;
    }
    RC_CUDA(ctx, launch_march(a, nvols * nviews, ctx->stream));
    if (stats) return read_stats(ctx, stats, false);
    return RC_OK;
}

rc_status rc_render_backward(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                             const float *dL_dimage, float *dL_dtf) {
    rc_status st = check_render(ctx, vol, p, dL_dtf, "rc_render_backward");
    if (st != RC_OK) return st;
    if (!dL_dimage) return fail(ctx, RC_ERR_INVALID_ARG, "rc_render_backward: dL_dimage is NULL");
    if (p->func != RC_FUNC_COMPOSITE)
        return fail(ctx, RC_ERR_UNSUPPORTED, "rc_render_backward: compositing function only");
    DeviceScope ds(ctx->device);
    st = ensure_grad_scratch(ctx);
    if (st != RC_OK) return st;
    st = ensure_occupancy(ctx, const_cast<rc_volume *>(vol), p->filter);
    if (st == RC_OK) st = prepare_filter(ctx, const_cast<rc_volume *>(vol), p);
    if (st != RC_OK) return st;
    AdjointArgs a;
    a.m = march_args(ctx, vol, p, nullptr);
    a.m.p.skip = 0;
    a.dimg = reinterpret_cast<const float4 *>(dL_dimage);
    a.acc = reinterpret_cast<long long *>(ctx->d_scratch);
    a.acc_scale = 0.0f;
    a.fimg = nullptr;
    RC_CUDA(ctx, launch_adjoint(a, 1, dL_dtf, ctx->stream));
    return RC_OK;
}

static rc_status backward_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                const rc_camera *cams, int nviews, const float *images, const float *dL_dimages,
                                float *dL_dtf, const char *who);

rc_status rc_render_backward_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                   const rc_camera *cams, int nviews, const float *dL_dimages, float *dL_dtf) {
    return backward_views(ctx, vol, p, cams, nviews, nullptr, dL_dimages, dL_dtf, "rc_render_backward_views");
}

rc_status rc_render_backward_views_with_forward(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                                const rc_camera *cams, int nviews, const float *images,
                                                const float *dL_dimages, float *dL_dtf) {
    const char *who = "rc_render_backward_views_with_forward";
    if (ctx && !images) return fail(ctx, RC_ERR_INVALID_ARG, "%s: images is NULL", who);
    return backward_views(ctx, vol, p, cams, nviews, images, dL_dimages, dL_dtf, who);
}

}  // extern "C"

static rc_status backward_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                const rc_camera *cams, int nviews, const float *images, const float *dL_dimages,
                                float *dL_dtf, const char *who) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    rc_status st = check_views(ctx, cams, nviews, who);
    if (st == RC_OK) st = check_render_views(ctx, vol, p, cams, dL_dtf, who);
    if (st != RC_OK) return st;
    if (!dL_dimages) return fail(ctx, RC_ERR_INVALID_ARG, "%s: dL_dimages is NULL", who);
    if (p->func != RC_FUNC_COMPOSITE) return fail(ctx, RC_ERR_UNSUPPORTED, "%s: compositing function only", who);
    DeviceScope ds(ctx->device);
    st = ensure_grad_scratch(ctx);
    if (st != RC_OK) return st;
    rc_volume *v = const_cast<rc_volume *>(vol);
    st = ensure_occupancy(ctx, v, p->filter);
    if (st == RC_OK) st = prepare_filter(ctx, v, p);
    if (st != RC_OK) return st;
    CamRec first;
    st = upload_views(ctx, v, cams, nviews, &first, who);
    if (st != RC_OK) return st;
    AdjointArgs a;
    a.m = march_args(ctx, v, p, nullptr);
    a.m.p.skip = 0;
    a.m.cam = first;
    a.m.cams = ctx->d_cams;
    a.dimg = reinterpret_cast<const float4 *>(dL_dimages);
    a.acc = reinterpret_cast<long long *>(ctx->d_scratch);
    a.acc_scale = 0.0f;
    a.fimg = reinterpret_cast<const float4 *>(images);
    RC_CUDA(ctx, launch_adjoint(a, nviews, dL_dtf, ctx->stream));
    return RC_OK;
}

extern "C" {

}  // extern "C"

// ---------------------------------------------------------------------------
// transfer-function gradient without device allocation
// ---------------------------------------------------------------------------
// Scratch of rc_render_backward_noalloc: the 4 per entry fixed-point accumulators and
// the |dL/dI| maximum for tables of at most kNoAllocMaxEntries entries. It is a
// file-scope device array, so every GPU that loads this library holds it
// (32 KB + 256 B) until the process exits. Host code must not use the symbol
// itself as an address: it is a host-side stand-in. The device address is
// looked up once per device with that device current.
constexpr int kNoAllocMaxEntries = 1024;
static __device__ __align__(256) long long g_tf_grad_scratch[4 * kNoAllocMaxEntries + 32];

constexpr int kNoAllocMaxDevices = 64;
static void *g_tf_grad_scratch_addr[kNoAllocMaxDevices];
static std::mutex g_tf_grad_scratch_mu;

static rc_status noalloc_scratch(rc_context *ctx, long long **out) {
    if (ctx->device >= kNoAllocMaxDevices)
        return fail(ctx, RC_ERR_UNSUPPORTED, "rc_render_backward_noalloc: device index %d >= %d", ctx->device,
                    kNoAllocMaxDevices);
    std::lock_guard<std::mutex> lock(g_tf_grad_scratch_mu);
    if (!g_tf_grad_scratch_addr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_tf_grad_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, RC_ERR_CUDA, "rc_render_backward_noalloc: cudaGetSymbolAddress: %s",
                        cudaGetErrorString(e));
        g_tf_grad_scratch_addr[ctx->device] = p;
    }
    *out = reinterpret_cast<long long *>(g_tf_grad_scratch_addr[ctx->device]);
    return RC_OK;
}

extern "C" {

rc_status rc_render_backward_noalloc(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                     const float *dL_dimage, float *dL_dtf) {
    rc_status st = check_render(ctx, vol, p, dL_dtf, "rc_render_backward_noalloc");
    if (st != RC_OK) return st;
    if (!dL_dimage) return fail(ctx, RC_ERR_INVALID_ARG, "rc_render_backward_noalloc: dL_dimage is NULL");
    if (p->func != RC_FUNC_COMPOSITE)
        return fail(ctx, RC_ERR_UNSUPPORTED, "rc_render_backward_noalloc: compositing function only");
    if (tf_entries(ctx) > (size_t)kNoAllocMaxEntries)
        return fail(ctx, RC_ERR_UNSUPPORTED,
                    "rc_render_backward_noalloc: table of %zu entries exceeds the static scratch (at most %d)",
                    tf_entries(ctx), kNoAllocMaxEntries);
    DeviceScope ds(ctx->device);
    long long *scratch = nullptr;
    st = noalloc_scratch(ctx, &scratch);
    if (st != RC_OK) return st;
    rc_volume *v = const_cast<rc_volume *>(vol);
    st = ensure_occupancy(ctx, v, p->filter);   // no allocation: the grids and masks exist from creation
    // pair bricks that an earlier render allocated are rebuilt in place when
    // stale (a copy kernel, no allocation); a volume that never had them reads
    // the apron bricks (the same stored values)
    if (st == RC_OK && v->d_pairs) st = prepare_filter(ctx, v, p);
    if (st != RC_OK) return st;
    AdjointArgs a;
    a.m = march_args(ctx, vol, p, nullptr);
    a.m.p.skip = 0;
    a.dimg = reinterpret_cast<const float4 *>(dL_dimage);
    a.acc = scratch;            // cleared on the stream before the kernel runs
    a.acc_scale = 0.0f;
    a.fimg = nullptr;
    RC_CUDA(ctx, launch_adjoint(a, 1, dL_dtf, ctx->stream));
    return RC_OK;
}

rc_status rc_brick_grid_get_filter(rc_context *ctx, const rc_volume *v, int filter, uint16_t *mn, uint16_t *mx) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_brick_grid_get: ctx is NULL");
    if (!v || !mn || !mx) return fail(ctx, RC_ERR_INVALID_ARG, "rc_brick_grid_get: NULL argument");
    if (filter != RC_FILTER_TRILINEAR && filter != RC_FILTER_BSPLINE)
        return fail(ctx, RC_ERR_INVALID_ARG, "rc_brick_grid_get: filter %d", filter);
    if (!v->uploaded) return fail(ctx, RC_ERR_STATE, "rc_brick_grid_get: volume has no data");
    DeviceScope ds(ctx->device);
    rc_status st = ensure_grid(ctx, const_cast<rc_volume *>(v), filter);
    if (st != RC_OK) return st;
    RC_CUDA(ctx, cudaMemcpyAsync(mn, v->d_mn[filter], v->nbricks * sizeof(uint16_t), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    RC_CUDA(ctx, cudaMemcpyAsync(mx, v->d_mx[filter], v->nbricks * sizeof(uint16_t), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    return RC_OK;
}

rc_status rc_brick_grid_get(rc_context *ctx, const rc_volume *v, uint16_t *mn, uint16_t *mx) {
    return rc_brick_grid_get_filter(ctx, v, RC_FILTER_TRILINEAR, mn, mx);
}

rc_status rc_skip_mask_get_filter(rc_context *ctx, const rc_volume *vol, int filter, uint8_t *occ) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_skip_mask_get: ctx is NULL");
    if (!vol || !occ) return fail(ctx, RC_ERR_INVALID_ARG, "rc_skip_mask_get: NULL argument");
    if (filter != RC_FILTER_TRILINEAR && filter != RC_FILTER_BSPLINE)
        return fail(ctx, RC_ERR_INVALID_ARG, "rc_skip_mask_get: filter %d", filter);
    if (!vol->uploaded) return fail(ctx, RC_ERR_STATE, "rc_skip_mask_get: volume has no data");
    if (ctx->K < 2) return fail(ctx, RC_ERR_STATE, "rc_skip_mask_get: no transfer function");
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    rc_status st = ensure_occupancy(ctx, v, filter);
    if (st != RC_OK) return st;
    RC_CUDA(ctx, cudaMemcpyAsync(occ, v->d_occ[filter], v->nbricks, cudaMemcpyDeviceToDevice, ctx->stream));
    return RC_OK;
}

rc_status rc_skip_mask_get(rc_context *ctx, const rc_volume *vol, uint8_t *occ) {
    return rc_skip_mask_get_filter(ctx, vol, RC_FILTER_TRILINEAR, occ);
}

// ---------------------------------------------------------------------------
// learned proposal
// ---------------------------------------------------------------------------
struct BlobHeader {
    char magic[8];
    uint32_t version, n_feat, n_hidden, n_layers, n_out, n_out_used, n_params, has_adam;
    uint64_t adam_step;
};
static_assert(sizeof(BlobHeader) == 48, "blob header layout");

static rc_status net_alloc(rc_context *ctx) {
    if (ctx->d_param) return RC_OK;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    uint8_t *f = nullptr;
    if (dev_alloc(&p, kParams * sizeof(float)) != cudaSuccess || dev_alloc(&m, kParams * sizeof(float)) != cudaSuccess ||
        dev_alloc(&v, kParams * sizeof(float)) != cudaSuccess || dev_alloc(&g, kParams * sizeof(float)) != cudaSuccess ||
        dev_alloc(&f, kUmmaAllBytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        cudaFree(m);
        cudaFree(v);
        cudaFree(g);
        cudaFree(f);
        return fail(ctx, RC_ERR_OOM, "proposal: device allocation");
    }
    ctx->d_param = p;
    ctx->d_m = m;
    ctx->d_v = v;
    ctx->d_grad = g;
    ctx->d_umma = f;
    return RC_OK;
}

rc_status rc_proposal_load(rc_context *ctx, const void *blob, size_t bytes) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_proposal_load: ctx is NULL");
    if (!blob) return fail(ctx, RC_ERR_INVALID_ARG, "rc_proposal_load: blob is NULL");
    if (bytes < sizeof(BlobHeader)) return fail(ctx, RC_ERR_FORMAT, "rc_proposal_load: %zu bytes, header is 48", bytes);
    BlobHeader h;
    memcpy(&h, blob, sizeof h);
    if (memcmp(h.magic, "RCPROP01", 8) != 0 || h.version != 1)
        return fail(ctx, RC_ERR_FORMAT, "rc_proposal_load: bad magic or version");
    if (h.n_feat != (uint32_t)kFeat || h.n_hidden != (uint32_t)kHid || h.n_layers != 3 || h.n_out != (uint32_t)kOut ||
        h.n_out_used != (uint32_t)kOutUsed || h.n_params != (uint32_t)kParams || h.has_adam > 1)
        return fail(ctx, RC_ERR_FORMAT, "rc_proposal_load: dimensions do not match this library");
    size_t need = sizeof h + (size_t)kParams * sizeof(float) * (h.has_adam ? 3 : 1);
    if (bytes != need) return fail(ctx, RC_ERR_FORMAT, "rc_proposal_load: %zu bytes, expected %zu", bytes, need);
    const float *vals = reinterpret_cast<const float *>(reinterpret_cast<const char *>(blob) + sizeof h);
    for (size_t i = 0; i < (size_t)kParams * (h.has_adam ? 3 : 1); i++)
        if (!isfinite(vals[i])) return fail(ctx, RC_ERR_FORMAT, "rc_proposal_load: non-finite value at %zu", i);
    DeviceScope ds(ctx->device);
    rc_status st = net_alloc(ctx);
    if (st != RC_OK) return st;
    RC_CUDA(ctx, cudaMemcpyAsync(ctx->d_param, vals, kParams * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    if (h.has_adam) {
        RC_CUDA(ctx, cudaMemcpyAsync(ctx->d_m, vals + kParams, kParams * sizeof(float), cudaMemcpyHostToDevice,
                                     ctx->stream));
        RC_CUDA(ctx, cudaMemcpyAsync(ctx->d_v, vals + 2 * kParams, kParams * sizeof(float), cudaMemcpyHostToDevice,
                                     ctx->stream));
    } else {
        RC_CUDA(ctx, cudaMemsetAsync(ctx->d_m, 0, kParams * sizeof(float), ctx->stream));
        RC_CUDA(ctx, cudaMemsetAsync(ctx->d_v, 0, kParams * sizeof(float), ctx->stream));
    }
    RC_CUDA(ctx, launch_pack(ctx->d_param, ctx->d_umma, ctx->stream));
    RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // the host blob may be freed at once
    ctx->adam_step = h.has_adam ? (long long)h.adam_step : 0;
    ctx->net_loaded = true;
    return RC_OK;
}

rc_status rc_proposal_save(rc_context *ctx, void *blob, size_t capacity, size_t *bytes_out) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_proposal_save: ctx is NULL");
    const size_t need = sizeof(BlobHeader) + (size_t)kParams * sizeof(float) * 3;
    if (bytes_out) *bytes_out = need;
    if (!blob) return RC_OK;
    if (!ctx->net_loaded) return fail(ctx, RC_ERR_STATE, "rc_proposal_save: no network loaded");
    if (capacity < need) return fail(ctx, RC_ERR_INVALID_ARG, "rc_proposal_save: capacity %zu < %zu", capacity, need);
    BlobHeader h;
    memcpy(h.magic, "RCPROP01", 8);
    h.version = 1;
    h.n_feat = kFeat;
    h.n_hidden = kHid;
    h.n_layers = 3;
    h.n_out = kOut;
    h.n_out_used = kOutUsed;
    h.n_params = kParams;
    h.has_adam = 1;
    h.adam_step = (uint64_t)ctx->adam_step;
    DeviceScope ds(ctx->device);
    char *out = reinterpret_cast<char *>(blob);
    memcpy(out, &h, sizeof h);
    float *vals = reinterpret_cast<float *>(out + sizeof h);
    RC_CUDA(ctx, cudaMemcpyAsync(vals, ctx->d_param, kParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    RC_CUDA(ctx, cudaMemcpyAsync(vals + kParams, ctx->d_m, kParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    RC_CUDA(ctx, cudaMemcpyAsync(vals + 2 * kParams, ctx->d_v, kParams * sizeof(float), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RC_OK;
}

rc_status rc_profiles_generate(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, float *out) {
    rc_status st = check_render(ctx, vol, p, out, "rc_profiles_generate");
    if (st == RC_OK) st = check_plain_form(ctx, p, "rc_profiles_generate");
    if (st != RC_OK) return st;
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    if (p->skip) {
        st = ensure_occupancy(ctx, v, RC_FILTER_TRILINEAR);
        if (st != RC_OK) return st;
    }
    MarchArgs a = march_args(ctx, v, p, nullptr);
    RC_CUDA(ctx, launch_profiles(a, out, ctx->stream));
    return RC_OK;
}

rc_status rc_proposal_features(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, float *out) {
    rc_status st = check_render(ctx, vol, p, out, "rc_proposal_features");
    if (st == RC_OK) st = check_plain_form(ctx, p, "rc_proposal_features");
    if (st != RC_OK) return st;
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    st = ensure_occupancy(ctx, v, RC_FILTER_TRILINEAR);
    if (st != RC_OK) return st;
    MarchArgs a = march_args(ctx, v, p, nullptr);
    RC_CUDA(ctx, launch_features(a, out, ctx->stream));
    return RC_OK;
}

static rc_status check_net(rc_context *ctx, const void *a, const void *b, int64_t n, const char *who) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    if (!a || !b) return fail(ctx, RC_ERR_INVALID_ARG, "%s: NULL buffer", who);
    if (n < 1 || n > (1ll << 31)) return fail(ctx, RC_ERR_INVALID_ARG, "%s: n = %lld", who, (long long)n);
    if (!ctx->net_loaded) return fail(ctx, RC_ERR_STATE, "%s: no network (call rc_proposal_load)", who);
    return RC_OK;
}

rc_status rc_proposal_forward(rc_context *ctx, const float *features, int64_t n, float *out) {
    rc_status st = check_net(ctx, features, out, n, "rc_proposal_forward");
    if (st != RC_OK) return st;
    DeviceScope ds(ctx->device);
    TcNetArgs a{};
    a.net = NetDev{ctx->d_umma, ctx->d_param};
    a.feat = features;
    a.net_out = out;
    a.n = n;
    a.ntiles = (n + 127) / 128;
    a.budget = wait_budget(&a.issue_mma);
    a.err = error_word(ctx);
    RC_CUDA(ctx, launch_tc_net(a, ctx->stream));
    return RC_OK;
}

static rc_status net_grad(rc_context *ctx, const float *features, const float *targets, int64_t n, float *grad,
                          float *loss) {
    const int grid = train_grid(n);
    if (ctx->partial_blocks < grid) {
        float *pp = nullptr, *lp = nullptr;
        RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (dev_alloc(&pp, (size_t)grid * kParams * sizeof(float)) != cudaSuccess ||
            dev_alloc(&lp, grid * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(pp);
            return fail(ctx, RC_ERR_OOM, "proposal: gradient partials");
        }
        cudaFree(ctx->d_partial);
        cudaFree(ctx->d_loss_partial);
        ctx->d_partial = pp;
        ctx->d_loss_partial = lp;
        ctx->partial_blocks = grid;
    }
    TrainArgs a;
    a.feat = features;
    a.target = targets;
    a.n = n;
    a.params = ctx->d_param;
    a.umma = ctx->d_umma;
    a.partial = ctx->d_partial;
    a.loss_partial = ctx->d_loss_partial;
    a.inv_n = (float)(1.0 / (double)n);
    a.budget = wait_budget(&a.issue_mma);
    a.err = error_word(ctx);
    RC_CUDA(ctx, launch_train_grad(a, grid, grad, loss, ctx->stream));
    return RC_OK;
}

rc_status rc_proposal_grad(rc_context *ctx, const float *features, const float *targets, int64_t n, float *grad,
                           float *loss) {
    rc_status st = check_net(ctx, features, targets, n, "rc_proposal_grad");
    if (st != RC_OK) return st;
    if (!grad) return fail(ctx, RC_ERR_INVALID_ARG, "rc_proposal_grad: grad is NULL");
    DeviceScope ds(ctx->device);
    return net_grad(ctx, features, targets, n, grad, loss);
}

rc_status rc_proposal_train_step(rc_context *ctx, const float *features, const float *targets, int64_t n, float lr,
                                 float *loss) {
    rc_status st = check_net(ctx, features, targets, n, "rc_proposal_train_step");
    if (st != RC_OK) return st;
    if (!(lr > 0.0f) || !isfinite(lr)) return fail(ctx, RC_ERR_INVALID_ARG, "rc_proposal_train_step: lr %g", (double)lr);
    DeviceScope ds(ctx->device);
    st = net_grad(ctx, features, targets, n, ctx->d_grad, loss);
    if (st != RC_OK) return st;
    ctx->adam_step++;
    RC_CUDA(ctx, launch_adam(ctx->d_param, ctx->d_m, ctx->d_v, ctx->d_grad, ctx->adam_step, lr, ctx->stream));
    RC_CUDA(ctx, launch_pack(ctx->d_param, ctx->d_umma, ctx->stream));
    return RC_OK;
}

// Shared checks of the importance-sampled renders.
static rc_status check_importance(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, float *out,
                                  int nimp, float eps, const char *who) {
    rc_status st = check_render(ctx, vol, p, out, who);
    if (st == RC_OK) st = check_plain_form(ctx, p, who);
    if (st != RC_OK) return st;
    if (p->func != RC_FUNC_COMPOSITE) return fail(ctx, RC_ERR_UNSUPPORTED, "%s: compositing function only", who);
    if (nimp < 1 || nimp > 4096) return fail(ctx, RC_ERR_INVALID_ARG, "%s: nimp %d", who, nimp);
    if (!(eps >= 0.0f)) return fail(ctx, RC_ERR_INVALID_ARG, "%s: eps %g", who, (double)eps);
    return RC_OK;
}

static ImportanceArgs importance_args(rc_context *ctx, rc_volume *v, const rc_render_params *p, int nimp, float eps,
                                      float *out, uint8_t *fallback) {
    ImportanceArgs a;
    a.m = march_args(ctx, v, p, out);
    a.pdf = nullptr;
    a.that = nullptr;
    a.range = nullptr;
    a.sampling = RC_SAMPLING_RANGE;
    a.lambda = 0.0f;
    a.nimp = nimp;
    a.eps = eps;
    a.fallback = fallback;
    return a;
}

rc_status rc_render_importance(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, const float *pdf,
                               const float *that, int nimp, float eps, float *out_rgba, uint8_t *fallback,
                               rc_stats *stats) {
    const char *who = "rc_render_importance";
    if (ctx && (!pdf || !that)) return fail(ctx, RC_ERR_INVALID_ARG, "%s: pdf / that is NULL", who);
    rc_status st = check_importance(ctx, vol, p, out_rgba, nimp, eps, who);
    if (st != RC_OK) return st;
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    st = ensure_occupancy(ctx, v, RC_FILTER_TRILINEAR);
    if (st != RC_OK) return st;
    ImportanceArgs a = importance_args(ctx, v, p, nimp, eps, out_rgba, fallback);
    a.pdf = pdf;
    a.that = that;
    if (stats) {
        RC_CUDA(ctx, stats_begin(ctx));
        a.m.stats = ctx->d_stats;
    }
    RC_CUDA(ctx, launch_importance(a, 1, ctx->stream));
    if (stats) return read_stats(ctx, stats, true);
    return RC_OK;
}

}  // extern "C"

// The importance checks for views cams[0..nviews) (cams[0] standing in for
// the context's camera).
static rc_status check_importance_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, float *out,
                                        const rc_camera *cams, int nviews, int nimp, float eps, int sampling,
                                        float lambda, const char *who) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    rc_status st = check_views(ctx, cams, nviews, who);
    if (st != RC_OK) return st;
    if (sampling != RC_SAMPLING_RANGE && sampling != RC_SAMPLING_INVCDF)
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: sampling %d", who, sampling);
    if (sampling == RC_SAMPLING_INVCDF && !(lambda >= 0.0f && lambda <= 1.0f))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: lambda %g (must be in [0, 1])", who, (double)lambda);
    const bool had = ctx->cam_set;
    const rc_camera keep = ctx->cam;
    ctx->cam = cams[0];
    ctx->cam_set = true;
    st = check_importance(ctx, vol, p, out, nimp, eps, who);
    ctx->cam = keep;
    ctx->cam_set = had;
    return st;
}

// Grows a context-owned device buffer (after the stream drains: queued
// kernels may still use the old one).
template <typename T>
static rc_status grow_buffer(rc_context *ctx, T **buf, long long *cap, long long need) {
    if (*cap >= need) return RC_OK;
    T *nb = nullptr;
    RC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RC_CUDA(ctx, dev_alloc(&nb, (size_t)need * sizeof(T)));
    cudaFree(*buf);
    *buf = nb;
    *cap = need;
    return RC_OK;
}

extern "C" {

rc_status rc_render_importance_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                                const rc_camera *cams, int nviews, int sampling, float lambda,
                                                const float *pdf, const float *that, int nimp, float eps,
                                                float *out_rgba, uint8_t *fallback, rc_stats *stats) {
    const char *who = "rc_render_importance_views";
    rc_status st = check_importance_views(ctx, vol, p, out_rgba, cams, nviews, nimp, eps, sampling, lambda, who);
    if (st != RC_OK) return st;
    if (sampling == RC_SAMPLING_RANGE && (!pdf || !that))
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: pdf / that is NULL (the range reading needs both)", who);
    if (sampling == RC_SAMPLING_INVCDF && !pdf && lambda != 1.0f)
        return fail(ctx, RC_ERR_INVALID_ARG, "%s: pdf is NULL (allowed only for lambda = 1)", who);
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    st = ensure_occupancy(ctx, v, RC_FILTER_TRILINEAR);
    if (st != RC_OK) return st;
    CamRec first;
    st = upload_views(ctx, v, cams, nviews, &first, who);
    if (st != RC_OK) return st;
    ImportanceArgs a = importance_args(ctx, v, p, nimp, eps, out_rgba, fallback);
    a.m.cam = first;
    a.m.cams = ctx->d_cams;
    a.pdf = pdf;
    a.that = that;
    a.sampling = sampling;
    a.lambda = lambda;
    if (stats) {
        RC_CUDA(ctx, stats_begin(ctx));
        a.m.stats = ctx->d_stats;
    }
    RC_CUDA(ctx, launch_importance(a, nviews, ctx->stream));
    if (stats) return read_stats(ctx, stats, true);
    return RC_OK;
}

}  // extern "C"

// RANGE: the network kernel writes each ray's sample range and T^ (8 bytes
// per ray), then the importance march renders every view from those records.
// INVCDF: the network kernel writes each ray's PDF and T^, then the
// inverse-CDF march.
static rc_status proposal_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, const rc_camera *cams,
                                int nviews, int sampling, float lambda, int nimp, float eps, float *out,
                                uint8_t *fallback, rc_stats *stats, const char *who) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "%s: ctx is NULL", who);
    if (!ctx->net_loaded) return fail(ctx, RC_ERR_STATE, "%s: no network loaded", who);
    rc_status st = check_importance_views(ctx, vol, p, out, cams, nviews, nimp, eps, sampling, lambda, who);
    if (st != RC_OK) return st;
    const long long nrays = (long long)nviews * cams[0].width * cams[0].height;
    DeviceScope ds(ctx->device);
    rc_volume *v = const_cast<rc_volume *>(vol);
    st = ensure_occupancy(ctx, v, RC_FILTER_TRILINEAR);
    if (st != RC_OK) return st;
    const bool invcdf = sampling == RC_SAMPLING_INVCDF;
    st = invcdf ? grow_buffer(ctx, &ctx->d_netpdf, &ctx->netpdf_cap, nrays * (kBins + 1))
                : grow_buffer(ctx, &ctx->d_range, &ctx->range_cap, nrays);
    if (st != RC_OK) return st;
    CamRec first;
    st = upload_views(ctx, v, cams, nviews, &first, who);
    if (st != RC_OK) return st;
    TcNetArgs n{};
    n.m = march_args(ctx, v, p, nullptr);
    n.m.cam = first;
    n.m.cams = ctx->d_cams;
    n.net = NetDev{ctx->d_umma, ctx->d_param};
    if (invcdf) {
        n.pdf_out = ctx->d_netpdf;
        n.that_out = ctx->d_netpdf + nrays * kBins;
    } else {
        n.range = ctx->d_range;
    }
    n.tiles_x = (first.W + 15) / 16;
    n.tiles_y = (first.H + 7) / 8;
    n.ntiles = (long long)n.tiles_x * n.tiles_y * nviews;
    n.budget = wait_budget(&n.issue_mma);
    n.err = error_word(ctx);
    if (stats) RC_CUDA(ctx, stats_begin(ctx));       // the network kernel is part of the call's time
    RC_CUDA(ctx, launch_tc_net(n, ctx->stream));
    ImportanceArgs a = importance_args(ctx, v, p, nimp, eps, out, fallback);
    a.m.cam = first;
    a.m.cams = ctx->d_cams;
    if (invcdf) {
        a.pdf = ctx->d_netpdf;
        a.that = ctx->d_netpdf + nrays * kBins;
        a.sampling = RC_SAMPLING_INVCDF;
        a.lambda = lambda;
    } else {
        a.range = ctx->d_range;
    }
    if (stats) a.m.stats = ctx->d_stats;
    RC_CUDA(ctx, launch_importance(a, nviews, ctx->stream));
    if (stats) return read_stats(ctx, stats, true);
    return RC_OK;
}

extern "C" {

rc_status rc_render_proposal(rc_context *ctx, const rc_volume *vol, const rc_render_params *p, int nimp, float eps,
                             float *out_rgba, uint8_t *fallback, rc_stats *stats) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_render_proposal: ctx is NULL");
    if (!ctx->cam_set) return fail(ctx, RC_ERR_STATE, "rc_render_proposal: no camera (call rc_camera_set)");
    const rc_camera cam = ctx->cam;
    return proposal_views(ctx, vol, p, &cam, 1, RC_SAMPLING_RANGE, 0.0f, nimp, eps, out_rgba, fallback, stats,
                          "rc_render_proposal");
}

rc_status rc_render_proposal_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                   const rc_camera *cams, int nviews, int nimp, float eps, float *out_rgba,
                                   uint8_t *fallback, rc_stats *stats) {
    return proposal_views(ctx, vol, p, cams, nviews, RC_SAMPLING_RANGE, 0.0f, nimp, eps, out_rgba, fallback, stats,
                          "rc_render_proposal_views");
}

rc_status rc_render_proposal_sampled(rc_context *ctx, const rc_volume *vol, const rc_render_params *p,
                                     const rc_camera *cams, int nviews, int sampling, float lambda, int nimp,
                                     float eps, float *out_rgba, uint8_t *fallback, rc_stats *stats) {
    return proposal_views(ctx, vol, p, cams, nviews, sampling, lambda, nimp, eps, out_rgba, fallback, stats,
                          "rc_render_proposal_sampled");
}


rc_status rc_context_sync(rc_context *ctx) {
    if (!ctx) return fail(nullptr, RC_ERR_INVALID_ARG, "rc_context_sync: ctx is NULL");
    DeviceScope ds(ctx->device);
    return check_device_errors(ctx, "rc_context_sync");
}

}  // extern "C"
