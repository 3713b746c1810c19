// Internal records shared by the host API (rc_api.cu) and the kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rc.h"

namespace rc {

constexpr int kBrick = 16;          // brick edge (voxels / cells)
constexpr int kBrickVox = 4096;     // 16^3

// Camera record: FP64 look-at basis rounded once to FP32, eye in index space.
struct CamRec {
    float f[3], r[3], u[3];
    float tx, ty;          // tan(fovy/2) * W/H, tan(fovy/2)
    float o[3];            // eye / spacing
    int W, H;
};

// Device view of a bricked volume.
struct VolDev {
    const void *data;      // bricked [bz][by][bx][16][16][16], storage type
    int storage;           // rc_storage
    int n[3];              // voxels per axis
    int cb[3];             // cell-bricks per axis: ceil((n-1)/16)
    unsigned sy, sz;       // element strides of one brick step in y and z
    float s[3];            // spacing (mm)
    float inv2s[3];        // 0.5 / spacing
    float smin;            // reference step: finest spacing
    float vscale;          // FP32 code scale of the table coordinate: vmax (raw) or 1
    float gmin;            // shading falls back to ambient+diffuse below this |gradient|
    int vmax;
};

// Transfer function: K entries of straight RGBA, FP32 or FP16 in device memory.
struct TFDev {
    const float4 *f32;
    const uint2 *f16;      // 4 halves per entry
    int K;
    int fp16;
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
};

struct MarchArgs {
    CamRec cam;
    VolDev vol;
    TFDev tf;
    MarchParams p;
    const uint8_t *occ;            // cell-brick occupancy (1 = may be non-empty)
    float4 *out;                   // H x W RGBA
    unsigned long long *stats;     // dense, evaluated, hit, total (or null)
};

// Adjoint arguments (compositing function only).
struct AdjointArgs {
    MarchArgs m;
    const float4 *dimg;            // H x W dL/dI
    long long *acc;                // K x 4 fixed-point accumulators (scratch)
    float acc_scale;               // fixed-point units per unit of gradient
};

// ---- launchers (return the launch error) --------------------------------
cudaError_t launch_relayout(const uint16_t *stage, VolDev v, void *dst, int nbv0, int nbv1,
                            int nbv2, cudaStream_t s);
cudaError_t launch_minmax(const uint16_t *stage, const int n[3], const int cb[3], int vmax,
                          uint16_t *mn, uint16_t *mx, cudaStream_t s);
cudaError_t launch_occupancy(const uint16_t *mn, const uint16_t *mx, int nbricks, int vmax,
                             int f16_values, TFDev tf, uint8_t *occ, cudaStream_t s);
cudaError_t launch_march(const MarchArgs &a, cudaStream_t s);
cudaError_t launch_adjoint(const AdjointArgs &a, float *dL_dtf, cudaStream_t s);
cudaError_t launch_absmax(const float *x, long long n, float *out, cudaStream_t s);

}  // namespace rc
