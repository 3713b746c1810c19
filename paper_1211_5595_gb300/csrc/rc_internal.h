// Internal records shared by the host API (rc_api.cu) and the kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rc.h"

namespace rc {

constexpr int kBrick = 16;          // cell-brick edge (trilinear cells)
constexpr int kApron = 19;          // stored brick edge: cells 16b-1 .. 16b+17 (edges replicated)
constexpr int kApronVox = kApron * kApron * kApron;   // 6859
constexpr int kGradEdge = 17;       // value+gradient brick edge: voxels 16b .. 16b+16 (the trilinear footprint)
constexpr int kGradVox = kGradEdge * kGradEdge * kGradEdge;   // 4913
// Pair bricks: per cell-brick the apron rows (lz, ly in 0..18) as 18
// entries (V[16b-1+e], V[16b+e]), e = 0..17, in the storage type (two
// elements, aligned to their size), so two x-adjacent voxels of any footprint
// row arrive in one load.
constexpr int kPairRow = 18;
constexpr int kPairVox = kApron * kApron * kPairRow;          // 6498

// Camera record: FP64 look-at basis rounded once to FP32, eye in index space.
struct CamRec {
    float f[3], r[3], u[3];
    float tx, ty;          // tan(fovy/2) * W/H, tan(fovy/2)
    float o[3];            // eye / spacing
    int W, H;
};

// Device view of a bricked volume.
struct VolDev {
    const void *data;      // [bz][by][bx][19][19][19] apron bricks, storage type
    const void *pairs;     // pair bricks (storage type) once a render needed them, else null
    // value+gradient bricks [bz][by][bx][17][17][17] of (value, central
    // differences x2): F32 storage float4 entries, U16 storage uint2 entries
    // (value | (D_x + 32768) << 16, (D_y + 32768) | (D_z + 32768) << 16); F16: null
    const void *vg;
    int storage;           // rc_storage
    int n[3];              // voxels per axis
    int cb[3];             // cell-bricks per axis: ceil((n-1)/16)
    float s[3];            // spacing (mm)
    float inv2s[3];        // 0.5 / spacing
    float smin;            // reference step: finest spacing
    float vscale;          // full scale in stored units: vmax (raw codes) or vmax / o (FP16, see f16o)
    float f16o;            // FP16 storage: the offset o, a power of two; a stored value h is
                           // (code - o) / o, so code = (h + 1) o (exact for codes 0 .. 2o <= 4096). 0 for raw codes
    float gmin;            // shading falls back to ambient+diffuse below this |gradient|
    int vmax;
#ifdef RC_DEBUG
    int *dbg_err;          // debug builds: the context's error word (bit 1: an index check failed)
    int dbg_poison;        // debug builds, test hook: added to every brick index (0 unless set)
#endif
};

// Transfer function: K entries of straight RGBA, FP32 or FP16 in device memory
// (1-D), or M rows of K entries over (gradient magnitude, value) (2-D).
struct TFDev {
    const float4 *f32;
    const uint2 *f16;      // 4 halves per entry
    int K;
    int fp16;
    float ucoef;           // table coordinate per stored unit: fl((K-1) / vscale); u = fl(v ucoef) for
                           // raw codes, fl((h + 1) ucoef) for FP16 values h
    // 2-D table (M >= 2; M = 0 for a 1-D table)
    const float4 *tab2;    // [M][K] FP32 (entries already FP16-rounded for an FP16 table)
    const float *amax;     // K: largest opacity of each value entry over the M rows
    int M;
    float wcoef;           // gradient coordinate per unit of |grad| (stored value units per mm)
};

// Sample evaluation variants of the compositing march.
enum : int {
    kShade = 1,            // headlight Blinn-Phong
    kCubic = 2,            // cubic B-spline reconstruction (else trilinear)
    kTF2 = 4               // 2-D table over (value, gradient magnitude)
};

struct MarchParams {
    float step_vox, term;
    int shade;
    float ka, kd, ks;
    int func;
    float iso;
    int skip;
    float ratio;           // ds / ds_ref
    int rmode;             // opacity correction: 0 identity, 1 sqrt, 2 sqrt(sqrt), 3 powf
    int filter;            // rc_filter
};

// Per-volume pointers of a batch of volumes with one shape, spacing and
// storage (the rest of the volume record is shared).
struct BatchVol {
    const void *data;
    const void *vg;
    const void *pairs;
    const uint8_t *occ;
    const unsigned long long *fine;
};

struct MarchArgs {
    CamRec cam;
    VolDev vol;
    TFDev tf;
    MarchParams p;
    const uint8_t *occ;            // cell-brick occupancy (1 = may be non-empty)
    const unsigned long long *fine;   // compositing: per cell-brick, one bit per 4^3 sub-block (or null)
    float4 *out;                   // H x W RGBA (view-major for several views)
    unsigned long long *stats;     // dense, evaluated, hit, total (or null)
    const CamRec *cams;            // one record per view (blockIdx.z), or null: cam
    const BatchVol *batch;         // compositing: blockIdx.z = volume * views + view (or null)
    int views;                     // views per volume of a batch
};

// Adjoint arguments (compositing function only).
struct AdjointArgs {
    MarchArgs m;
    const float4 *dimg;            // H x W dL/dI
    const float4 *fimg;            // the forward images (C, 1 - T) of the same views, or null: recomputed
    long long *acc;                // K x 4 fixed-point accumulators (scratch)
    float acc_scale;               // fixed-point units per unit of gradient
};

// ---- learned proposal ----------------------------------------------------
constexpr int kBins = 32;                 // opacity PDF bins over [t_near, t_far]
constexpr int kProfSamples = 512;         // samples of the profile march (16 per bin)
constexpr int kFeat = 112;                // 6 raw + 72 encoded + 32 occupancy + 2 padding
constexpr int kHid = 64;
constexpr int kOut = 40;                  // 32 PDF logits + 1 transmittance logit + 7 padding
constexpr int kOutUsed = 33;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kFeat * kHid;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kHid * kOut;
constexpr int kParams = kOffB4 + kOut;    // 18152
// BF16 B operands of the four layers for the tcgen05 MMA (N x K, K-major,
// core-matrix layout): W1^T 64 x 112, W2^T 64 x 64, W3^T 64 x 64 and W4^T with
// its 40 outputs padded to 48 rows (N of an M = 128 MMA is a multiple of 16).
constexpr int kN4 = 48;
constexpr unsigned kUmmaL1 = 0;
constexpr unsigned kUmmaL2 = kUmmaL1 + kHid * kFeat * 2;
constexpr unsigned kUmmaL3 = kUmmaL2 + kHid * kHid * 2;
constexpr unsigned kUmmaL4 = kUmmaL3 + kHid * kHid * 2;
constexpr unsigned kUmmaBytes = kUmmaL4 + kN4 * kHid * 2;   // 36864
// B operands of the training backward's input gradients (dH = dZ W^T): W4 as
// 64 x 48 (outputs padded), W3 and W2 as 64 x 64, N = the layer's inputs,
// K = its outputs; stored after the forward operands.
constexpr unsigned kUmmaB4 = kUmmaBytes;
constexpr unsigned kUmmaB3 = kUmmaB4 + kHid * kN4 * 2;
constexpr unsigned kUmmaB2 = kUmmaB3 + kHid * kHid * 2;
constexpr unsigned kUmmaAllBytes = kUmmaB2 + kHid * kHid * 2;   // 59392

struct NetDev {
    const uint8_t *umma;      // packed BF16 B operands (kUmmaBytes, 16-byte aligned)
    const float *params;      // FP32 master parameters (biases read from here)
};

// The network kernel: 128 rays per tile (one M = 128 MMA tile, TMEM lane =
// ray), persistent CTAs. Rays from cameras (range records for the importance
// march) or from a feature matrix (network outputs).
struct TcNetArgs {
    MarchArgs m;              // rays: cameras (m.cams, grid of views), volume, occupancy
    NetDev net;
    const float *feat;        // feature-matrix form: n x 112 FP32 (else null)
    float *net_out;           // feature-matrix form: n x 33
    uint2 *range;             // camera form: per ray (b_start | b_end << 8, T^ bits), view-major; this and
                              // pdf_out are not written for tiles none of whose rays meets the volume
    float *pdf_out;           // camera form writing PDFs instead (else null): per ray 32 floats, view-major
    float *that_out;          // with pdf_out: per ray T^
    long long n;              // feature-matrix form: rays
    long long ntiles;         // tiles of 128 rays
    int tiles_x, tiles_y;     // camera form: 16 x 8 pixel tiles per view
    long long budget;         // clock cycles a wait may take before it gives up
    int *err;                 // bit 0: a wait gave up (the call reports RC_ERR_TIMEOUT)
    int issue_mma;            // 0 only in the timeout test: nothing is issued, the wait runs out
};

struct ImportanceArgs {
    MarchArgs m;
    const float *pdf;         // given-PDF form: H*W*32 per view, view-major (null: uniform, INVCDF with lambda 1)
    const float *that;        // given-PDF form: H*W per view (null: no fallback)
    const uint2 *range;       // range form: records of the network kernel (view-major)
    int sampling;             // given-PDF form: RC_SAMPLING_RANGE or RC_SAMPLING_INVCDF
    float lambda;             // INVCDF: weight of the uniform density in the mixture
    int nimp;                 // importance samples per ray
    float eps;                // fallback when |T_nimp - T^| > eps
    uint8_t *fallback;        // per pixel flag (or null), view-major
};

struct TrainArgs {
    const float *feat;        // n x 112
    const float *target;      // n x 33: 32 profile bins + final transmittance
    long long n;
    const float *params;      // FP32 master parameters (biases)
    const uint8_t *umma;      // packed BF16 B operands, forward and backward (kUmmaAllBytes)
    float *partial;           // gridDim x kParams gradient partials
    float *loss_partial;      // gridDim
    float inv_n;
    long long budget;         // clock cycles a wait may take before it gives up
    int *err;                 // bit 0: a wait gave up
    int issue_mma;            // 0 only in the timeout test
};

// ---- launchers (return the launch error) --------------------------------
cudaError_t launch_pairs(VolDev v, void *dst, cudaStream_t s);
cudaError_t launch_prep(const uint16_t *stage, VolDev v, void *apron, void *vg, uint16_t *mn, uint16_t *mx,
                        uint16_t *mn4, uint16_t *mx4, cudaStream_t s);
cudaError_t launch_minmax(const uint16_t *stage, const int n[3], const int cb[3], int vmax, int filter,
                          uint16_t *mn, uint16_t *mx, cudaStream_t s);
// f16o: 0 for raw codes; for FP16 storage the offset o of its values.
cudaError_t launch_occupancy(const uint16_t *mn, const uint16_t *mx, int nbricks, int vmax,
                             int f16o, TFDev tf, uint8_t *occ, cudaStream_t s);
// 4^3 sub-block min/max grid of a filter (cells 4j..4j+3; footprint voxels
// 4j..4j+4, or 4j-1..4j+5 for the B-spline, clamped) and the fine mask built
// from it: per cell-brick one bit per sub-block.
cudaError_t launch_minmax4(const uint16_t *stage, const int n[3], int vmax, int filter, uint16_t *mn, uint16_t *mx,
                           cudaStream_t s);
cudaError_t launch_finemask(const uint16_t *mn4, const uint16_t *mx4, const int n[3], const int cb[3], int vmax,
                            int f16o, TFDev tf, unsigned long long *fine, cudaStream_t s);
cudaError_t launch_march(const MarchArgs &a, int nviews, cudaStream_t s);
cudaError_t launch_march_cubic(const MarchArgs &a, int nviews, cudaStream_t s);   // filter = B-spline
cudaError_t launch_march_tf2(const MarchArgs &a, int nviews, cudaStream_t s);     // trilinear, 2-D table
cudaError_t launch_adjoint(const AdjointArgs &a, int nviews, float *dL_dtf, cudaStream_t s);
cudaError_t launch_absmax(const float *x, long long n, float *out, cudaStream_t s);
cudaError_t launch_profiles(const MarchArgs &a, float *out, cudaStream_t s);
cudaError_t launch_features(const MarchArgs &a, float *out, cudaStream_t s);
cudaError_t launch_tc_net(const TcNetArgs &a, cudaStream_t s);                  // feat != null: outputs, else ranges
cudaError_t launch_importance(const ImportanceArgs &a, int nviews, cudaStream_t s); // pdf != null: given PDFs, else ranges
cudaError_t launch_train_grad(const TrainArgs &a, int grid, float *grad, float *loss, cudaStream_t s);
int train_grid(long long n);      // CTAs of the training kernel for n rays (one per SM at most)
cudaError_t launch_adam(float *params, float *m, float *v, const float *grad, long long step, float lr,
                        cudaStream_t s);
cudaError_t launch_pack(const float *params, uint8_t *umma, cudaStream_t s);

}  // namespace rc
