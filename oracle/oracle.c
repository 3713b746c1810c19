/*
 * oracle.c -- plain, slow FP64 reference of the raycasting method.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the oracle against which the CUDA
 * library is checked. Only the test suite, the package smoke check and the
 * bench's CPU-baseline leg may load it. It shares no code, header, table or
 * helper with the CUDA library, and it never reads anything the library wrote.
 *
 * What it computes (Adeshina et al., "Hardware-Accelerated Raycasting: Towards
 * an Effective Brain MRI Visualization", Sec. 4.1-4.2):
 *   - one viewing ray per pixel, from the eye through the pixel centre into the
 *     volume (Sec. 4.1, step 1: the path of the ray);
 *   - evenly spaced samples S_k along the ray inside the volume, each the
 *     trilinear resample of the voxel grid (Sec. 4.1 step 2; Sec. 3.2 names
 *     trilinear filtering as the resampling filter);
 *   - classification of each sample by the transfer function into colour and
 *     opacity (Sec. 2.6, Sec. 4.2);
 *   - the compositing ray function (Sec. 4.1 step 3, Sec. 4.2): the intensity
 *     reaching the eye is the sum of the sample emissions I(S_k), each
 *     attenuated by e^{-tau(S_k, S_eye)} (Eq. 3-4), the discrete form of the
 *     integral of Eq. 5. Over one sample segment e^{-tau} is that segment's
 *     transparency (1 - alpha'), so the attenuation from S_k to the eye is the
 *     product of the transparencies of the samples in front of S_k;
 *   - the other ray functions the paper lists (Sec. 2.4 item ii, Sec. 4.1):
 *     maximum intensity projection, average intensity projection, x-ray sum,
 *     isosurface (first crossing) and thresholding (first sample above).
 *
 * Readings where the paper is silent (each one is a written specification that
 * the CUDA library implements on its own):
 *   - index space has voxel centres at integers; world x = i * spacing;
 *   - the camera basis is computed in FP64 from (eye, target, up) and rounded
 *     to FP32; ray directions and sample positions use the FP32 operations
 *     written out in ray_setup_f32, sample_t and position_at_t, each correctly
 *     rounded;
 *     every step after the sample position is FP64;
 *   - opacity is given per reference step (the finest voxel spacing) and is
 *     corrected to the step used: alpha' = 1 - (1 - alpha)^(ds / ds_ref), which
 *     is Eq. 3's e^{-tau} for a segment of length ds;
 *   - early termination after the first sample whose accumulated opacity is
 *     >= term; the first decision inside +-tie_band of term is reported and the
 *     result of the other branch is returned beside the primary one;
 *   - headlight Blinn-Phong shading with central-difference gradients (the
 *     paper's "simulated light effect", Sec. 2.4).
 *
 * Build: gcc -O2 -std=gnu11 -ffp-contract=off -fPIC -shared -pthread
 * (no contraction: each FP32 operation of the ray specification rounds once).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__FLT_EVAL_METHOD__) && __FLT_EVAL_METHOD__ != 0
#error "the FP32 ray specification needs FLT_EVAL_METHOD == 0"
#endif

/* ------------------------------------------------------------------------ */
/* public records (mirrored by oracle/__init__.py)                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint16_t *data;   /* x fastest, then y, then z */
    int32_t nx, ny, nz;
    float sx, sy, sz;       /* voxel spacing, mm */
    int32_t vmax;           /* largest valid code; larger codes clamp to it */
    int32_t value_mode;     /* 0: raw codes; 1: the code as FP16 storage holds it,
                               h = fp16((code - o) / o) with the offset o of
                               f16_offset, read back as (h + 1) o */
} orc_volume;

typedef struct {
    const float *rgba;      /* straight colour + opacity per reference step: K x 4
                               (1-D), or M rows of K entries x 4 (2-D; value index
                               fastest, row j = gradient-magnitude index) */
    int32_t K;
    int32_t fp16;           /* 1: use the FP16 rounding of each entry */
    int32_t M;              /* rows of a 2-D table; 0 or 1: 1-D table */
    float gmax;             /* 2-D: gradient magnitude (codes per mm) of the last row */
} orc_tf;

typedef struct {
    float eye[3], target[3], up[3];
    float fovy_deg;
    int32_t width, height;
} orc_camera;

enum { ORC_COMPOSITE = 0, ORC_MIP = 1, ORC_AVERAGE = 2, ORC_XRAY = 3, ORC_ISO = 4, ORC_THRESHOLD = 5 };

typedef struct {
    float step_vox;     /* sample spacing in units of the finest voxel spacing */
    float term;         /* early termination at accumulated opacity >= term */
    int32_t shade;      /* 1: headlight Blinn-Phong */
    float ka, kd, ks;   /* ambient, diffuse, specular weights; exponent 16 */
    int32_t func;       /* ray function, ORC_* */
    float iso;          /* iso-value / threshold in volume value units */
    int32_t fp64_rays;  /* 1: ray setup in FP64 (information only) */
    float tie_band;     /* half width of the termination tie band */
    int32_t filter;     /* 0: trilinear; 1: uniform cubic B-spline */
} orc_params;

enum { ORC_TRILINEAR = 0, ORC_BSPLINE = 1 };

/* ------------------------------------------------------------------------ */
/* internal state                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint16_t *v;
    int n[3];
    float s[3];
    double vrange;          /* value of full scale (vmax; every value is in code units) */
    double *lut;            /* value of each code, after the vmax clamp */
    double *tf;             /* M x K x 4 */
    int K;
    int M;                  /* 1 for a 1-D table */
    double gcoef;           /* 2-D: (M-1) / gmax in units of the stored values */
    float f[3], r[3], u[3], tx, ty, o[3];   /* FP32 camera record */
    double fd[3], rd[3], ud[3], txd, tyd, od[3];
    int W, H;
    orc_params P;
    float smin;             /* reference step ds_ref = finest spacing */
} scene;

typedef struct {
    int hit;
    float o[3], d[3], dir[3], tn, tf, ds;
    double od[3], dd[3], dird[3], tnd, tfd, dsd;
    int fp64;
    int nsamp;
} ray;

static double half_round(float x) { return (double)(_Float16)x; }

/* The offset of the FP16 storage form: the smallest power of two o >= 1 with
 * 2o >= vmax. A code c is held as h = fp16((c - o) / o); for vmax <= 4096 the
 * integer c - o lies in [-2048, 2048], where FP16 represents every integer, so
 * the stored value is exact (the representation reading of the precision
 * form; an FP16 of c / vmax keeps codes above 2048 only to +-1). */
static int f16_offset(int vmax) {
    int o = 1;
    while (2 * o < vmax) o *= 2;
    return o;
}

/* FP16 value of code c (value_mode 1), as a float. */
static float f16_value(int c, int vmax) {
    int o = f16_offset(vmax);
    return (float)half_round((float)(c - o) / (float)o);
}

static void normalize3(double v[3]) {
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n; v[1] /= n; v[2] /= n;
}

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static int scene_init(scene *S, const orc_volume *vol, const orc_tf *tf,
                      const orc_camera *cam, const orc_params *prm) {
    memset(S, 0, sizeof *S);
    if (vol->nx < 2 || vol->ny < 2 || vol->nz < 2 || vol->vmax < 1) return 1;
    if (!(vol->sx > 0 && vol->sy > 0 && vol->sz > 0)) return 1;
    if (tf->K < 2 || cam->width < 1 || cam->height < 1) return 1;
    if (tf->M >= 2 && !(tf->gmax > 0.0f)) return 1;
    if (prm->filter != ORC_TRILINEAR && prm->filter != ORC_BSPLINE) return 1;
    if (tf->M >= 2 && prm->func == ORC_THRESHOLD) return 3;   /* thresholding: 1-D tables only */
    S->v = vol->data;
    S->n[0] = vol->nx; S->n[1] = vol->ny; S->n[2] = vol->nz;
    S->s[0] = vol->sx; S->s[1] = vol->sy; S->s[2] = vol->sz;
    S->lut = (double *)malloc(65536 * sizeof(double));
    S->M = tf->M >= 2 ? tf->M : 1;
    S->tf = (double *)malloc((size_t)tf->K * S->M * 4 * sizeof(double));
    if (!S->lut || !S->tf) return 2;
    for (int code = 0; code < 65536; code++) {
        int c = code > vol->vmax ? vol->vmax : code;
        /* value_mode 1: the code recovered from its FP16 form, (h + 1) o */
        S->lut[code] = vol->value_mode ? ((double)f16_value(c, vol->vmax) + 1.0) * (double)f16_offset(vol->vmax)
                                       : (double)c;
    }
    S->vrange = (double)vol->vmax;
    S->K = tf->K;
    for (size_t i = 0; i < (size_t)4 * tf->K * S->M; i++)
        S->tf[i] = tf->fp16 ? half_round(tf->rgba[i]) : (double)tf->rgba[i];
    /* the gradient coordinate is defined on code units */
    S->gcoef = S->M >= 2 ? (double)(S->M - 1) / (double)tf->gmax : 0.0;
    S->P = *prm;
    S->W = cam->width; S->H = cam->height;
    S->smin = fminf(fminf(vol->sx, vol->sy), vol->sz);

    /* camera basis in FP64 (look-at), rounded once to FP32 */
    double f[3], up[3], r[3], u[3];
    for (int c = 0; c < 3; c++) {
        f[c] = (double)cam->target[c] - (double)cam->eye[c];
        up[c] = (double)cam->up[c];
    }
    normalize3(f);
    cross3(f, up, r);
    normalize3(r);
    cross3(r, f, u);
    double th = tan((double)cam->fovy_deg * 3.14159265358979323846 / 360.0);
    double tx = th * (double)cam->width / (double)cam->height;
    for (int c = 0; c < 3; c++) {
        S->fd[c] = f[c]; S->rd[c] = r[c]; S->ud[c] = u[c];
        S->f[c] = (float)f[c]; S->r[c] = (float)r[c]; S->u[c] = (float)u[c];
        S->od[c] = (double)cam->eye[c] / (double)S->s[c];
        S->o[c] = (float)S->od[c];
    }
    S->txd = tx; S->tyd = th;
    S->tx = (float)tx; S->ty = (float)th;
    return 0;
}

static void scene_free(scene *S) {
    free(S->lut);
    free(S->tf);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 step 1: the path of the ray                                       */
/* ------------------------------------------------------------------------ */
/* FP32 ray specification; each operation rounds once (no contraction). */
static void ray_setup_f32(const scene *S, float step_vox, int x, int y, ray *R) {
    float a = ((float)x + 0.5f) / (float)S->W;
    float ndcx = (a * 2.0f - 1.0f) * S->tx;
    float b = ((float)y + 0.5f) / (float)S->H;
    float ndcy = (1.0f - b * 2.0f) * S->ty;
    float v[3];
    for (int c = 0; c < 3; c++) v[c] = (S->f[c] + ndcx * S->r[c]) + ndcy * S->u[c];
    float len = sqrtf((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    for (int c = 0; c < 3; c++) {
        R->dir[c] = v[c] / len;
        R->d[c] = R->dir[c] / S->s[c];
        R->o[c] = S->o[c];
    }
    R->fp64 = 0;
    R->hit = 0;
    R->nsamp = 0;
    /* slab test against the box [0, N-1] in index space; t is world distance */
    float tn = 0.0f, tf = INFINITY;
    for (int c = 0; c < 3; c++) {
        float hi = (float)(S->n[c] - 1);
        if (R->d[c] == 0.0f) {
            if (R->o[c] < 0.0f || R->o[c] > hi) return;
            continue;
        }
        float t0 = (0.0f - R->o[c]) / R->d[c];
        float t1 = (hi - R->o[c]) / R->d[c];
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    if (!(tf >= tn)) return;
    R->tn = tn;
    R->tf = tf;
    R->ds = step_vox * S->smin;
    R->nsamp = (int)floorf((tf - tn) / R->ds) + 1;
    R->hit = 1;
}

/* The same construction in FP64 (information only: not the parity target). */
static void ray_setup_f64(const scene *S, float step_vox, int x, int y, ray *R) {
    double a = ((double)x + 0.5) / (double)S->W;
    double ndcx = (a * 2.0 - 1.0) * S->txd;
    double b = ((double)y + 0.5) / (double)S->H;
    double ndcy = (1.0 - b * 2.0) * S->tyd;
    double v[3];
    for (int c = 0; c < 3; c++) v[c] = (S->fd[c] + ndcx * S->rd[c]) + ndcy * S->ud[c];
    double len = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    for (int c = 0; c < 3; c++) {
        R->dird[c] = v[c] / len;
        R->dd[c] = R->dird[c] / (double)S->s[c];
        R->od[c] = S->od[c];
    }
    R->fp64 = 1;
    R->hit = 0;
    R->nsamp = 0;
    double tn = 0.0, tf = INFINITY;
    for (int c = 0; c < 3; c++) {
        double hi = (double)(S->n[c] - 1);
        if (R->dd[c] == 0.0) {
            if (R->od[c] < 0.0 || R->od[c] > hi) return;
            continue;
        }
        double t0 = (0.0 - R->od[c]) / R->dd[c];
        double t1 = (hi - R->od[c]) / R->dd[c];
        tn = fmax(tn, fmin(t0, t1));
        tf = fmin(tf, fmax(t0, t1));
    }
    if (!(tf >= tn)) return;
    R->tnd = tn;
    R->tfd = tf;
    R->dsd = (double)step_vox * (double)S->smin;
    R->nsamp = (int)floor((tf - tn) / R->dsd) + 1;
    R->hit = 1;
}

static void ray_setup(const scene *S, int x, int y, ray *R) {
    if (S->P.fp64_rays) ray_setup_f64(S, S->P.step_vox, x, y, R);
    else ray_setup_f32(S, S->P.step_vox, x, y, R);
}

/* world distance and index-space position of evenly spaced sample k */
static double sample_t(const ray *R, int k) {
    if (R->fp64) return R->tnd + (double)k * R->dsd;
    return (double)fmaf((float)k, R->ds, R->tn);
}

static void position_at_t(const ray *R, double t, double p[3]) {
    for (int c = 0; c < 3; c++) {
        if (R->fp64) p[c] = R->od[c] + t * R->dd[c];
        else p[c] = (double)fmaf((float)t, R->d[c], R->o[c]);
    }
}

static double step_len(const ray *R) { return R->fp64 ? R->dsd : (double)R->ds; }

static void world_dir(const ray *R, double dir[3]) {
    for (int c = 0; c < 3; c++) dir[c] = R->fp64 ? R->dird[c] : (double)R->dir[c];
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 step 2: the values along the ray (trilinear resampling)           */
/* ------------------------------------------------------------------------ */
static double voxel(const scene *S, int x, int y, int z) {
    return S->lut[S->v[((size_t)z * S->n[1] + y) * S->n[0] + x]];
}

/* cell base index and weight along one axis; p is clamped to [0, n-1] */
static void cell(double p, int n, int *i, double *w) {
    double q = p < 0.0 ? 0.0 : (p > (double)(n - 1) ? (double)(n - 1) : p);
    int b = (int)floor(q);
    if (b > n - 2) b = n - 2;
    *i = b;
    *w = q - (double)b;
}

static double trilinear(const scene *S, const double p[3]) {
    int i, j, k;
    double wx, wy, wz;
    cell(p[0], S->n[0], &i, &wx);
    cell(p[1], S->n[1], &j, &wy);
    cell(p[2], S->n[2], &k, &wz);
    double c00 = voxel(S, i, j, k) * (1 - wx) + voxel(S, i + 1, j, k) * wx;
    double c10 = voxel(S, i, j + 1, k) * (1 - wx) + voxel(S, i + 1, j + 1, k) * wx;
    double c01 = voxel(S, i, j, k + 1) * (1 - wx) + voxel(S, i + 1, j, k + 1) * wx;
    double c11 = voxel(S, i, j + 1, k + 1) * (1 - wx) + voxel(S, i + 1, j + 1, k + 1) * wx;
    double c0 = c00 * (1 - wy) + c10 * wy;
    double c1 = c01 * (1 - wy) + c11 * wy;
    return c0 * (1 - wz) + c1 * wz;
}

/* central differences of the trilinear field, one index unit per axis,
 * divided by the spacing: a world-space gradient (value units per mm) */
static void gradient(const scene *S, const double p[3], double g[3]) {
    for (int a = 0; a < 3; a++) {
        double q[3] = {p[0], p[1], p[2]};
        q[a] = p[a] + 1.0;
        double fp = trilinear(S, q);
        q[a] = p[a] - 1.0;
        double fm = trilinear(S, q);
        g[a] = (fp - fm) / 2.0 / (double)S->s[a];
    }
}

/* Uniform cubic B-spline reconstruction, the higher-order alternative to the
 * trilinear filter (Sec. 3.2: quadratic or cubic filters for higher image
 * quality). The textbook kernel
 *   beta(x) = (4 - 6 x^2 + 3 |x|^3) / 6   for |x| < 1,
 *             (2 - |x|)^3 / 6             for 1 <= |x| < 2,   0 beyond,
 * is applied to the voxel values directly (no interpolating prefilter):
 * f(p) = sum over voxels v of V(v) beta(p_x - v_x) beta(p_y - v_y) beta(p_z - v_z),
 * with p clamped to the box and voxel indices outside it clamped to the
 * nearest border voxel. Only the four voxels base-1 .. base+2 per axis around
 * the trilinear cell base can have beta != 0. */
static double bspline_beta(double x) {
    double a = fabs(x);
    if (a < 1.0) return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}

/* d beta / dx */
static double bspline_dbeta(double x) {
    double a = fabs(x), sg = x < 0.0 ? -1.0 : 1.0;
    if (a < 1.0) return sg * (-12.0 * a + 9.0 * a * a) / 6.0;
    if (a < 2.0) return -sg * (2.0 - a) * (2.0 - a) / 2.0;
    return 0.0;
}

static int clampi(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

/* value and, when g != NULL, the analytic world-space gradient (value units
 * per mm) of the B-spline field */
static double bspline(const scene *S, const double p[3], double g[3]) {
    double q[3], wb[3][4], wd[3][4];
    int base[3];
    for (int a = 0; a < 3; a++) {
        double w;
        cell(p[a], S->n[a], &base[a], &w);
        q[a] = (double)base[a] + w;               /* the clamped position */
        for (int o = 0; o < 4; o++) {
            double x = q[a] - (double)(base[a] - 1 + o);
            wb[a][o] = bspline_beta(x);
            wd[a][o] = bspline_dbeta(x);
        }
    }
    double f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int oz = 0; oz < 4; oz++)
        for (int oy = 0; oy < 4; oy++)
            for (int ox = 0; ox < 4; ox++) {
                double v = voxel(S, clampi(base[0] - 1 + ox, S->n[0]), clampi(base[1] - 1 + oy, S->n[1]),
                                 clampi(base[2] - 1 + oz, S->n[2]));
                f += v * wb[0][ox] * wb[1][oy] * wb[2][oz];
                gx += v * wd[0][ox] * wb[1][oy] * wb[2][oz];
                gy += v * wb[0][ox] * wd[1][oy] * wb[2][oz];
                gz += v * wb[0][ox] * wb[1][oy] * wd[2][oz];
            }
    if (g) {
        g[0] = gx / (double)S->s[0];
        g[1] = gy / (double)S->s[1];
        g[2] = gz / (double)S->s[2];
    }
    return f;
}

/* the reconstructed field at p under the selected filter */
static double field(const scene *S, const double p[3]) {
    return S->P.filter == ORC_BSPLINE ? bspline(S, p, NULL) : trilinear(S, p);
}

/* its world-space gradient: central differences of the trilinear field, the
 * analytic derivative of the B-spline field */
static void field_gradient(const scene *S, const double p[3], double g[3]) {
    if (S->P.filter == ORC_BSPLINE) bspline(S, p, g);
    else gradient(S, p, g);
}

/* ------------------------------------------------------------------------ */
/* classification (Sec. 2.6) and shading                                      */
/* ------------------------------------------------------------------------ */
/* table coordinate of a value: u = v (K-1) / full scale */
static double tf_coord(const scene *S, double v) { return v * (double)(S->K - 1) / S->vrange; }

static void classify(const scene *S, double u, double rgba[4], int *i0, double *w0) {
    double q = u < 0.0 ? 0.0 : (u > (double)(S->K - 1) ? (double)(S->K - 1) : u);
    int i = (int)floor(q);
    if (i > S->K - 2) i = S->K - 2;
    double w = q - (double)i;
    for (int c = 0; c < 4; c++) rgba[c] = S->tf[4 * i + c] * (1 - w) + S->tf[4 * (i + 1) + c] * w;
    if (i0) *i0 = i;
    if (w0) *w0 = w;
}

/* Two-dimensional classification over (value, gradient magnitude), the
 * boundary-emphasising transfer functions of Sec. 3.1: u is the value
 * coordinate, w = |grad f| (M-1) / gmax the gradient-magnitude coordinate; each
 * is clamped to its table axis and the four surrounding entries are blended
 * bilinearly (value direction first, then gradient direction). */
static void classify2(const scene *S, double u, double w, double rgba[4], int *i0, int *j0, double *a0,
                      double *b0) {
    int K = S->K, M = S->M;
    double qu = u < 0.0 ? 0.0 : (u > (double)(K - 1) ? (double)(K - 1) : u);
    double qw = w < 0.0 ? 0.0 : (w > (double)(M - 1) ? (double)(M - 1) : w);
    int i = (int)floor(qu), j = (int)floor(qw);
    if (i > K - 2) i = K - 2;
    if (j > M - 2) j = M - 2;
    double a = qu - (double)i, b = qw - (double)j;
    *i0 = i;
    *j0 = j;
    *a0 = a;
    *b0 = b;
    for (int c = 0; c < 4; c++) {
        double t00 = S->tf[4 * ((size_t)j * K + i) + c], t10 = S->tf[4 * ((size_t)j * K + i + 1) + c];
        double t01 = S->tf[4 * ((size_t)(j + 1) * K + i) + c], t11 = S->tf[4 * ((size_t)(j + 1) * K + i + 1) + c];
        double r0 = t00 * (1 - a) + t10 * a, r1 = t01 * (1 - a) + t11 * a;
        rgba[c] = r0 * (1 - b) + r1 * b;
    }
}

/* headlight Blinn-Phong: light and view both along -dir, so the half vector is
 * the light vector; two-sided |n.L|. dcol[c] = d colour / d rgb[c]. */
static void shade(const scene *S, const double rgb[3], const double g[3], const double dir[3],
                  double col[3], double dcol[3]) {
    const orc_params *P = &S->P;
    double gl = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double sf, spec;
    if (gl < 1e-6 * S->vrange) {
        sf = (double)P->ka + (double)P->kd;
        spec = 0.0;
    } else {
        double ndl = fabs(g[0] * dir[0] + g[1] * dir[1] + g[2] * dir[2]) / gl;
        double n2 = ndl * ndl, n4 = n2 * n2, n8 = n4 * n4, n16 = n8 * n8;
        sf = (double)P->ka + (double)P->kd * ndl;
        spec = (double)P->ks * n16;
    }
    for (int c = 0; c < 3; c++) {
        double x = rgb[c] * sf + spec;
        col[c] = x < 1.0 ? x : 1.0;
        dcol[c] = x < 1.0 ? sf : 0.0;
    }
}

/* opacity per reference step -> opacity of a segment of length ds (Eq. 3) */
static double correct_alpha(double a, double ratio) { return 1.0 - pow(1.0 - a, ratio); }

/* all quantities of one sample */
typedef struct {
    double t, p[3], v, u, rgba[4], a, col[3], dcol[3], w;
    double gm, gw;      /* |grad f| (value units per mm) and its table coordinate (2-D) */
    double wb;          /* 2-D table: weight along the gradient axis (entry rows j, j + 1) */
    int i, j;           /* table cell: value index i (and gradient row j for a 2-D table) */
} sample;

static void eval_sample(const scene *S, const ray *R, double t, double ratio, sample *s) {
    s->t = t;
    position_at_t(R, t, s->p);
    s->v = field(S, s->p);
    s->u = tf_coord(S, s->v);
    double g[3] = {0, 0, 0};
    s->gm = 0.0;
    s->gw = 0.0;
    if (S->P.shade || S->M >= 2) {
        field_gradient(S, s->p, g);
        s->gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    }
    if (S->M >= 2) {
        s->gw = s->gm * S->gcoef;
        classify2(S, s->u, s->gw, s->rgba, &s->i, &s->j, &s->w, &s->wb);
    } else {
        classify(S, s->u, s->rgba, &s->i, &s->w);
        s->j = 0;
        s->wb = 0.0;
    }
    s->a = correct_alpha(s->rgba[3], ratio);
    if (S->P.shade) {
        double dir[3];
        world_dir(R, dir);
        shade(S, s->rgba, g, dir, s->col, s->dcol);
    } else {
        for (int c = 0; c < 3; c++) { s->col[c] = s->rgba[c]; s->dcol[c] = 1.0; }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 step 3: the ray functions                                          */
/* ------------------------------------------------------------------------ */
/* Compositing (Sec. 4.2, Eq. 4): I = sum_k T_k alpha'_k c_k with
 * T_k = prod_{j<k} (1 - alpha'_j), evaluated from the eye backwards into the
 * volume, stopped after the first sample whose opacity 1 - T reaches term.
 * flip_k >= 0 inverts the stop decision at that sample (tie alternative). */
static void composite(const scene *S, const ray *R, int flip_k, double out[4], int *nsamp,
                      int *tie_k) {
    double C[3] = {0, 0, 0}, T = 1.0;
    double ratio = step_len(R) / (double)S->smin;
    int k = 0;
    if (tie_k) *tie_k = -1;
    for (; k < R->nsamp; k++) {
        sample s;
        eval_sample(S, R, sample_t(R, k), ratio, &s);
        for (int c = 0; c < 3; c++) C[c] += T * s.a * s.col[c];
        T *= (1.0 - s.a);
        double opacity = 1.0 - T;
        int stop = opacity >= (double)S->P.term;
        if (tie_k && *tie_k < 0 && fabs(opacity - (double)S->P.term) < (double)S->P.tie_band)
            *tie_k = k;
        if (k == flip_k) stop = !stop;
        if (stop) { k++; break; }
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
    *nsamp = k;
}

/* MIP, average, x-ray, isosurface and threshold (Sec. 2.4 ii, Sec. 4.1).
 * Output channels: MIP/average: (m, m, m, 1) with m the max / mean value over
 * full scale; x-ray: (x, x, x, 1) with x = sum_k v_k ds / full scale (mm);
 * isosurface: (t*, shaded intensity at the crossing sample, k*, 1) with t* the
 * linearly interpolated crossing distance between the two bracketing samples;
 * threshold: (TF colour of the first sample >= iso, 1). 0 when nothing is
 * found or the ray misses. */
static void other_function(const scene *S, const ray *R, double out[4], int *nsamp) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    int func = S->P.func;
    double acc = 0.0, prev_v = 0.0, prev_t = 0.0;
    *nsamp = R->nsamp;
    if (R->nsamp <= 0) return;
    for (int k = 0; k < R->nsamp; k++) {
        double p[3], t = sample_t(R, k);
        position_at_t(R, t, p);
        double v = field(S, p);
        if (func == ORC_MIP) {
            if (k == 0 || v > acc) acc = v;
        } else if (func == ORC_AVERAGE || func == ORC_XRAY) {
            acc += v;
        } else if (v >= (double)S->P.iso) {
            *nsamp = k + 1;
            if (func == ORC_THRESHOLD) {
                double rgba[4];
                classify(S, tf_coord(S, v), rgba, NULL, NULL);
                out[0] = rgba[0]; out[1] = rgba[1]; out[2] = rgba[2]; out[3] = 1.0;
            } else {
                double ts = t;
                if (k > 0) ts = prev_t + (t - prev_t) * ((double)S->P.iso - prev_v) / (v - prev_v);
                double g[3], dir[3], white[3] = {1, 1, 1}, col[3], dcol[3];
                field_gradient(S, p, g);
                world_dir(R, dir);
                shade(S, white, g, dir, col, dcol);
                out[0] = ts; out[1] = col[0]; out[2] = (double)k; out[3] = 1.0;
            }
            return;
        }
        prev_v = v;
        prev_t = t;
    }
    if (func == ORC_MIP) acc = acc / S->vrange;
    else if (func == ORC_AVERAGE) acc = acc / (double)R->nsamp / S->vrange;
    else if (func == ORC_XRAY) acc = acc * step_len(R) / S->vrange;
    else return;
    out[0] = out[1] = out[2] = acc;
    out[3] = 1.0;
}

/* ------------------------------------------------------------------------ */
/* threading over pixels                                                      */
/* ------------------------------------------------------------------------ */
typedef struct job job;
typedef void (*pixel_fn)(job *J, int64_t idx, int tid);
struct job {
    const scene *S;
    const int32_t *pix;
    int64_t npix;
    int64_t next;
    pixel_fn fn;
    int nthreads;
    /* outputs / extra inputs */
    double *rgba, *rgba_alt, *aux, *aux2;
    uint8_t *tie;
    int32_t *nsamp, *nsamp_alt;
    const double *dimg;
    double *dtf_thread;     /* nthreads x K x 4 */
    const float *pdf;
    const uint8_t *occ;
    int nimp;
    int sampling;           /* importance march: ORC_SAMPLING_* */
    float lambda;           /* importance march, INVCDF: uniform weight */
    float **fbuf;           /* per thread: 2 nimp floats */
    sample **scratch;       /* per thread */
    int *cap;               /* per thread: samples the scratch holds */
};

typedef struct { job *J; int tid; } worker_arg;

#define CHUNK 32

static void *worker(void *arg) {
    worker_arg *A = (worker_arg *)arg;
    job *J = A->J;
    for (;;) {
        int64_t start = __atomic_fetch_add(&J->next, CHUNK, __ATOMIC_RELAXED);
        if (start >= J->npix) break;
        int64_t end = start + CHUNK < J->npix ? start + CHUNK : J->npix;
        for (int64_t i = start; i < end; i++) J->fn(J, i, A->tid);
    }
    return NULL;
}

/* static round-robin chunks: results independent of thread timing */
static void *worker_static(void *arg) {
    worker_arg *A = (worker_arg *)arg;
    job *J = A->J;
    for (int64_t start = (int64_t)A->tid * CHUNK; start < J->npix;
         start += (int64_t)J->nthreads * CHUNK) {
        int64_t end = start + CHUNK < J->npix ? start + CHUNK : J->npix;
        for (int64_t i = start; i < end; i++) J->fn(J, i, A->tid);
    }
    return NULL;
}

static void run_job(job *J, int nthreads, int deterministic) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    J->nthreads = nthreads;
    J->next = 0;
    pthread_t th[256];
    worker_arg args[256];
    for (int t = 0; t < nthreads; t++) {
        args[t].J = J;
        args[t].tid = t;
    }
    void *(*fn)(void *) = deterministic ? worker_static : worker;
    int started = 0;
    for (int t = 1; t < nthreads; t++) {
        if (pthread_create(&th[t], NULL, fn, &args[t]) != 0) break;
        started = t;
    }
    fn(&args[0]);
    for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
    /* threads that failed to start leave their static chunks: run them here */
    if (deterministic)
        for (int t = started + 1; t < nthreads; t++) fn(&args[t]);
}

static void pixel_xy(const job *J, int64_t idx, int *x, int *y) {
    int64_t lin = J->pix ? (int64_t)J->pix[idx] : idx;
    *x = (int)(lin % J->S->W);
    *y = (int)(lin / J->S->W);
}

/* ------------------------------------------------------------------------ */
/* rendering                                                                  */
/* ------------------------------------------------------------------------ */
static void render_pixel(job *J, int64_t idx, int tid) {
    (void)tid;
    const scene *S = J->S;
    int x, y;
    pixel_xy(J, idx, &x, &y);
    ray R;
    ray_setup(S, x, y, &R);
    double out[4] = {0, 0, 0, 0}, alt[4] = {0, 0, 0, 0};
    int ns = 0, ns2 = 0, tie_k = -1;
    if (R.hit) {
        if (S->P.func == ORC_COMPOSITE) {
            composite(S, &R, -1, out, &ns, &tie_k);
            if (tie_k >= 0) {
                composite(S, &R, tie_k, alt, &ns2, NULL);
            } else {
                memcpy(alt, out, sizeof out);
                ns2 = ns;
            }
        } else {
            other_function(S, &R, out, &ns);
            memcpy(alt, out, sizeof out);
            ns2 = ns;
        }
    }
    for (int c = 0; c < 4; c++) {
        J->rgba[4 * idx + c] = out[c];
        if (J->rgba_alt) J->rgba_alt[4 * idx + c] = alt[c];
    }
    if (J->tie) J->tie[idx] = (uint8_t)(tie_k >= 0);
    if (J->nsamp) J->nsamp[idx] = ns;
    if (J->nsamp_alt) J->nsamp_alt[idx] = ns2;
}

int orc_render(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
               const orc_params *prm, const int32_t *pix, int64_t npix, double *rgba,
               double *rgba_alt, uint8_t *tie, int32_t *nsamp, int32_t *nsamp_alt,
               int nthreads) {
    scene S;
    int rc = scene_init(&S, vol, tf, cam, prm);
    if (rc) { scene_free(&S); return rc; }
    job J;
    memset(&J, 0, sizeof J);
    J.S = &S;
    J.pix = pix;
    J.npix = pix ? npix : (int64_t)cam->width * cam->height;
    J.fn = render_pixel;
    J.rgba = rgba;
    J.rgba_alt = rgba_alt;
    J.tie = tie;
    J.nsamp = nsamp;
    J.nsamp_alt = nsamp_alt;
    run_job(&J, nthreads, 0);
    scene_free(&S);
    return 0;
}

/* every sample of one ray, no termination; record of 16 doubles per sample:
 * t, px, py, pz, v, u, r, g, b, a, a', col r, col g, col b, |grad f|, w
 * (|grad f| and its table coordinate w are 0 unless shading or a 2-D table
 * needs the gradient) */
int orc_ray_samples(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
                    const orc_params *prm, int x, int y, int max_samples, double *out,
                    int32_t *nsamp_total) {
    scene S;
    int rc = scene_init(&S, vol, tf, cam, prm);
    if (rc) { scene_free(&S); return rc; }
    ray R;
    ray_setup(&S, x, y, &R);
    *nsamp_total = R.hit ? R.nsamp : 0;
    double ratio = R.hit ? step_len(&R) / (double)S.smin : 1.0;
    for (int k = 0; R.hit && k < R.nsamp && k < max_samples; k++) {
        sample s;
        eval_sample(&S, &R, sample_t(&R, k), ratio, &s);
        double *o = out + 16 * (size_t)k;
        o[0] = s.t; o[1] = s.p[0]; o[2] = s.p[1]; o[3] = s.p[2]; o[4] = s.v; o[5] = s.u;
        for (int c = 0; c < 4; c++) o[6 + c] = s.rgba[c];
        o[10] = s.a;
        for (int c = 0; c < 3; c++) o[11 + c] = s.col[c];
        o[14] = s.gm;
        o[15] = s.gw;
    }
    scene_free(&S);
    return 0;
}

/* ray geometry for tests: (hit, tn, tf, ds, nsamp, o[3], d[3], dir[3]) */
int orc_ray_geometry(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
                     const orc_params *prm, int x, int y, double *out) {
    scene S;
    int rc = scene_init(&S, vol, tf, cam, prm);
    if (rc) { scene_free(&S); return rc; }
    ray R;
    ray_setup(&S, x, y, &R);
    out[0] = R.hit;
    out[1] = R.fp64 ? R.tnd : R.tn;
    out[2] = R.fp64 ? R.tfd : R.tf;
    out[3] = step_len(&R);
    out[4] = R.nsamp;
    for (int c = 0; c < 3; c++) {
        out[5 + c] = R.fp64 ? R.od[c] : R.o[c];
        out[8 + c] = R.fp64 ? R.dd[c] : R.d[c];
        out[11 + c] = R.fp64 ? R.dird[c] : R.dir[c];
    }
    scene_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* transfer-function gradient of the compositing function                     */
/* ------------------------------------------------------------------------ */
/* For one ray with samples k = 0..n-1 (n up to termination) the image is
 * I_c = sum_k T_k a'_k col_kc (c = r, g, b) and I_a = 1 - T_n, with
 * T_{k+1} = T_k (1 - a'_k). Plain reverse-mode differentiation over the stored
 * samples: with G_{k} = dL/dT_k, G_n = -dL/dI_a and
 *   dL/da'_k  = T_k (g . col_k) - G_{k+1} T_k
 *   dL/dcol_kc = g_c T_k a'_k
 *   G_k       = a'_k (g . col_k) + G_{k+1} (1 - a'_k).
 * Then da'/da = r (1 - min(a, 1 - 1e-6))^(r - 1) and the table entries i, i+1
 * receive the lerp weights (1 - w, w). */
static void grad_pixel(job *J, int64_t idx, int tid) {
    const scene *S = J->S;
    int x, y;
    pixel_xy(J, idx, &x, &y);
    ray R;
    ray_setup(S, x, y, &R);
    double out[4] = {0, 0, 0, 0};
    double *dtf = J->dtf_thread + (size_t)tid * S->K * (S->M >= 2 ? S->M : 1) * 4;
    if (!R.hit) {
        if (J->rgba) for (int c = 0; c < 4; c++) J->rgba[4 * idx + c] = 0.0;
        return;
    }
    if (J->cap[tid] < R.nsamp) {
        free(J->scratch[tid]);
        J->scratch[tid] = (sample *)malloc((size_t)R.nsamp * sizeof(sample) +
                                           ((size_t)R.nsamp + 1) * sizeof(double));
        J->cap[tid] = J->scratch[tid] ? R.nsamp : 0;
        if (!J->scratch[tid]) abort();
    }
    sample *sm = J->scratch[tid];
    double *T = (double *)(sm + R.nsamp);
    double ratio = step_len(&R) / (double)S->smin;
    int n = 0;
    T[0] = 1.0;
    double C[3] = {0, 0, 0};
    for (int k = 0; k < R.nsamp; k++) {
        eval_sample(S, &R, sample_t(&R, k), ratio, &sm[k]);
        for (int c = 0; c < 3; c++) C[c] += T[k] * sm[k].a * sm[k].col[c];
        T[k + 1] = T[k] * (1.0 - sm[k].a);
        n = k + 1;
        if (1.0 - T[k + 1] >= (double)S->P.term) break;
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T[n];
    if (J->rgba) for (int c = 0; c < 4; c++) J->rgba[4 * idx + c] = out[c];
    const double *g = J->dimg + 4 * idx;
    double G = -g[3];
    for (int k = n - 1; k >= 0; k--) {
        const sample *s = &sm[k];
        double gc = g[0] * s->col[0] + g[1] * s->col[1] + g[2] * s->col[2];
        double dA = T[k] * gc - G * T[k];
        G = s->a * gc + G * (1.0 - s->a);
        double ac = s->rgba[3] < 1.0 - 1e-6 ? s->rgba[3] : 1.0 - 1e-6;
        double dalpha = dA * ratio * pow(1.0 - ac, ratio - 1.0);
        double d[4];
        for (int c = 0; c < 3; c++) d[c] = g[c] * T[k] * s->a * s->dcol[c];
        d[3] = dalpha;
        /* the entries the sample interpolated, with their lerp weights:
         * i, i + 1 of a 1-D table; (i, j) .. (i + 1, j + 1) of a 2-D one */
        if (S->M >= 2) {
            const size_t e00 = (size_t)s->j * S->K + s->i, e01 = e00 + S->K;
            const double w00 = (1.0 - s->w) * (1.0 - s->wb), w10 = s->w * (1.0 - s->wb);
            const double w01 = (1.0 - s->w) * s->wb, w11 = s->w * s->wb;
            for (int c = 0; c < 4; c++) {
                dtf[4 * e00 + c] += w00 * d[c];
                dtf[4 * (e00 + 1) + c] += w10 * d[c];
                dtf[4 * e01 + c] += w01 * d[c];
                dtf[4 * (e01 + 1) + c] += w11 * d[c];
            }
        } else {
            for (int c = 0; c < 4; c++) {
                dtf[4 * s->i + c] += (1.0 - s->w) * d[c];
                dtf[4 * (s->i + 1) + c] += s->w * d[c];
            }
        }
    }
}

int orc_render_grad(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
                    const orc_params *prm, const int32_t *pix, int64_t npix,
                    const double *dimg, double *dtf, double *rgba, int nthreads) {
    scene S;
    int rc = scene_init(&S, vol, tf, cam, prm);
    if (rc) { scene_free(&S); return rc; }
    const size_t nent = (size_t)S.K * (S.M >= 2 ? S.M : 1);     /* table entries */
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    job J;
    memset(&J, 0, sizeof J);
    J.S = &S;
    J.pix = pix;
    J.npix = pix ? npix : (int64_t)cam->width * cam->height;
    J.fn = grad_pixel;
    J.dimg = dimg;
    J.rgba = rgba;
    J.dtf_thread = (double *)calloc((size_t)nthreads * nent * 4, sizeof(double));
    J.scratch = (sample **)calloc((size_t)nthreads, sizeof(sample *));
    J.cap = (int *)calloc((size_t)nthreads, sizeof(int));
    int ok = J.dtf_thread && J.scratch && J.cap;
    if (ok) {
        run_job(&J, nthreads, 1);
        memset(dtf, 0, nent * 4 * sizeof(double));
        for (int t = 0; t < nthreads; t++)
            for (size_t i = 0; i < nent * 4; i++) dtf[i] += J.dtf_thread[(size_t)t * nent * 4 + i];
    }
    for (int t = 0; J.scratch && t < nthreads; t++) free(J.scratch[t]);
    free(J.scratch);
    free(J.cap);
    free(J.dtf_thread);
    scene_free(&S);
    return ok ? 0 : 2;
}

/* ------------------------------------------------------------------------ */
/* opacity profiles along the ray (training targets of the learned proposal)  */
/* ------------------------------------------------------------------------ */
/* 512 samples at the centres of 512 equal segments of [t_near, t_far]
 * (t_k = fmaf(k + 0.5, L / 512, t_near) in FP32), composited without early
 * termination; the weights T_k a'_k are summed 16 at a time into 32 bins.
 * aux = 32 bins per pixel, aux2 = final transmittance. */
#define PROF_SAMPLES 512
#define PROF_BINS 32

static void profile_pixel(job *J, int64_t idx, int tid) {
    (void)tid;
    const scene *S = J->S;
    int x, y;
    pixel_xy(J, idx, &x, &y);
    ray R;
    ray_setup_f32(S, S->P.step_vox, x, y, &R);
    double *bins = J->aux + (size_t)PROF_BINS * idx;
    for (int b = 0; b < PROF_BINS; b++) bins[b] = 0.0;
    double T = 1.0;
    if (R.hit) {
        float delta = (R.tf - R.tn) / (float)PROF_SAMPLES;
        double ratio = (double)delta / (double)S->smin;
        for (int k = 0; k < PROF_SAMPLES; k++) {
            float t = fmaf((float)k + 0.5f, delta, R.tn);
            sample s;
            eval_sample(S, &R, (double)t, ratio, &s);
            bins[k / (PROF_SAMPLES / PROF_BINS)] += T * s.a;
            T *= (1.0 - s.a);
        }
    }
    J->aux2[idx] = T;
}

int orc_profiles(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
                 const orc_params *prm, const int32_t *pix, int64_t npix, double *bins,
                 double *tfinal, int nthreads) {
    scene S;
    int rc = scene_init(&S, vol, tf, cam, prm);
    if (rc) { scene_free(&S); return rc; }
    job J;
    memset(&J, 0, sizeof J);
    J.S = &S;
    J.pix = pix;
    J.npix = pix ? npix : (int64_t)cam->width * cam->height;
    J.fn = profile_pixel;
    J.aux = bins;
    J.aux2 = tfinal;
    run_job(&J, nthreads, 0);
    scene_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* importance-sampled compositing from a per-ray opacity PDF                  */
/* ------------------------------------------------------------------------ */
/* The proposal's 32-bin PDF over the chord [t_near, t_far] (bin width
 * bw = (t_far - t_near) / 32) chooses nimp samples that replace the evenly
 * spaced march of Sec. 4.1; each sample stands for a segment of the ray and
 * its opacity is corrected to that segment's length (Eq. 3). Two readings of
 * how the samples follow the PDF:
 *
 * RANGE: the PDF marks where the ray's contribution ends. b_end is one bin
 * past the first bin >= b_start where its running sum reaches 1 - 1/64 (a
 * margin for early predictions; 31 at most, and 31 if the sum never gets
 * there). b_start is the first bin whose start, centre or end point lies in
 * an occupied cell-brick (exact knowledge of where the opacity is zero; with
 * no occupied point the range is the whole chord). The samples sit at the
 * centres of nimp equal segments of [t_a, t_b] (the start of bin b_start to
 * the end of bin b_end), each standing for its segment. FP32 specification
 * (each operation rounds once):
 *   point b: fmaf(b, bw, t_near), fmaf(b + 0.5, bw, t_near),
 *   fmaf(b + 1, bw, t_near); P_{b+1} = P_b + pdf_b;
 *   t_a = b_start == 0 ? t_near : fmaf(b_start, bw, t_near);
 *   t_b = b_end == 31 ? t_far : fmaf(b_end + 1, bw, t_near);
 *   seg = (t_b - t_a) / nimp; t_j = fmaf(j + 0.5, seg, t_a); len_j = seg.
 *
 * INVCDF: stratified inverse-CDF sampling of the PDF mixed with a uniform
 * density, q_b = (1 - lambda) pdf_b + lambda / 32 (piecewise constant over
 * the bins): sample j sits where the mixture's CDF reaches
 * u_j = (j + 0.5) / nimp of its total, and stands for the stretch between the
 * midpoints to its neighbours (the first from t_near, the last to t_far), so
 * the segments tile the chord. lambda = 1 gives nimp samples at the centres of
 * nimp equal segments of the whole chord (the uniform march the method
 * replaces). FP32 specification:
 *   q_b = fmaf(1 - lambda, pdf_b, lambda / 32); Q_0 = 0, Q_{b+1} = Q_b + q_b;
 *   y_j = ((j + 0.5) / nimp) * Q_32; b = the first bin with Q_{b+1} > y_j
 *   (31 if none); f = q_b > 0 ? min(max((y_j - Q_b) / q_b, 0), 1) : 0;
 *   t_j = fmaf(b + f, bw, t_near);
 *   m_0 = t_near, m_j = (t_{j-1} + t_j) * 0.5, m_nimp = t_far;
 *   len_j = m_{j+1} - m_j.
 *
 * Compositing and early termination as in composite(), with the same
 * termination tie report and alternative branch. */
enum { ORC_SAMPLING_RANGE = 0, ORC_SAMPLING_INVCDF = 1 };

static int occupied_at(const scene *S, const ray *R, const uint8_t *occ, float t) {
    int nb[3];
    for (int a = 0; a < 3; a++) nb[a] = (S->n[a] - 1 + 15) / 16;
    double p[3];
    for (int c = 0; c < 3; c++) p[c] = (double)fmaf(t, R->d[c], R->o[c]);
    int idx[3];
    for (int a = 0; a < 3; a++) {
        int i;
        double w;
        cell(p[a], S->n[a], &i, &w);
        idx[a] = i / 16;
    }
    return occ[(idx[2] * nb[1] + idx[1]) * nb[0] + idx[0]] != 0;
}

/* Positions t[j] and segment lengths len[j] of the nimp samples of ray R. */
static void importance_positions(const scene *S, const ray *R, const float *pdf, const uint8_t *occ, int nimp,
                                 int sampling, float lambda, float *t, float *len) {
    float bw = (R->tf - R->tn) / (float)PROF_BINS;
    if (sampling == ORC_SAMPLING_INVCDF) {
        float Q[PROF_BINS + 1], q[PROF_BINS];
        float wp = 1.0f - lambda, wu = lambda / (float)PROF_BINS;
        Q[0] = 0.0f;
        for (int b = 0; b < PROF_BINS; b++) {
            q[b] = fmaf(wp, pdf ? pdf[b] : 0.0f, wu);
            Q[b + 1] = Q[b] + q[b];
        }
        for (int j = 0; j < nimp; j++) {
            float y = (((float)j + 0.5f) / (float)nimp) * Q[PROF_BINS];
            int b = 0;
            while (b < PROF_BINS - 1 && !(Q[b + 1] > y)) b++;
            float f = 0.0f;
            if (q[b] > 0.0f) {
                f = (y - Q[b]) / q[b];
                f = f < 0.0f ? 0.0f : (f > 1.0f ? 1.0f : f);
            }
            t[j] = fmaf((float)b + f, bw, R->tn);
        }
        float m = R->tn;
        for (int j = 0; j < nimp; j++) {
            float next = j + 1 < nimp ? (t[j] + t[j + 1]) * 0.5f : R->tf;
            len[j] = next - m;
            m = next;
        }
        return;
    }
    int b0 = -1, b1 = PROF_BINS - 1;
    for (int b = 0; b < PROF_BINS && b0 < 0; b++)
        if (occupied_at(S, R, occ, fmaf((float)b, bw, R->tn)) ||
            occupied_at(S, R, occ, fmaf((float)b + 0.5f, bw, R->tn)) ||
            occupied_at(S, R, occ, fmaf((float)b + 1.0f, bw, R->tn)))
            b0 = b;
    if (b0 < 0) {
        b0 = 0;
    } else {
        float P = 0.0f;
        for (int b = 0; b < PROF_BINS; b++) {
            P = P + pdf[b];
            if (b >= b0 && P >= 1.0f - 1.0f / 64.0f) {
                b1 = b + 1 < PROF_BINS - 1 ? b + 1 : PROF_BINS - 1;
                break;
            }
        }
    }
    float ta = b0 == 0 ? R->tn : fmaf((float)b0, bw, R->tn);
    float tb = b1 == PROF_BINS - 1 ? R->tf : fmaf((float)(b1 + 1), bw, R->tn);
    float seg = (tb - ta) / (float)nimp;
    for (int j = 0; j < nimp; j++) {
        t[j] = fmaf((float)j + 0.5f, seg, ta);
        len[j] = seg;
    }
}

/* Eq. 4 over the given samples, front to back, stopped after the first sample
 * whose opacity reaches term; flip_k >= 0 inverts the stop decision at that
 * sample, and *tie_k (when given) receives the first decision within the tie
 * band, as in composite(). */
static void importance_composite(const scene *S, const ray *R, const float *t, const float *len, int nimp,
                                 int flip_k, double out[4], double *Tend, int *nsamp, int *tie_k) {
    double C[3] = {0, 0, 0}, T = 1.0;
    int k = 0;
    if (tie_k) *tie_k = -1;
    for (; k < nimp; k++) {
        sample s;
        eval_sample(S, R, (double)t[k], (double)len[k] / (double)S->smin, &s);
        for (int c = 0; c < 3; c++) C[c] += T * s.a * s.col[c];
        T *= (1.0 - s.a);
        double opacity = 1.0 - T;
        int stop = opacity >= (double)S->P.term;
        if (tie_k && *tie_k < 0 && fabs(opacity - (double)S->P.term) < (double)S->P.tie_band) *tie_k = k;
        if (k == flip_k) stop = !stop;
        if (stop) { k++; break; }
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
    *Tend = T;
    *nsamp = k;
}

static void importance_pixel(job *J, int64_t idx, int tid) {
    const scene *S = J->S;
    int x, y;
    pixel_xy(J, idx, &x, &y);
    ray R;
    ray_setup_f32(S, S->P.step_vox, x, y, &R);
    double out[4] = {0, 0, 0, 0}, alt[4] = {0, 0, 0, 0};
    double T = 1.0, T2;
    int ns = 0, ns2, tie_k = -1;
    if (R.hit && J->nimp > 0) {
        float *t = J->fbuf[tid], *len = J->fbuf[tid] + J->nimp;
        importance_positions(S, &R, J->pdf ? J->pdf + (size_t)PROF_BINS * idx : NULL, J->occ, J->nimp, J->sampling,
                             J->lambda, t, len);
        importance_composite(S, &R, t, len, J->nimp, -1, out, &T, &ns, &tie_k);
        if (tie_k >= 0) importance_composite(S, &R, t, len, J->nimp, tie_k, alt, &T2, &ns2, NULL);
        else memcpy(alt, out, sizeof out);
    }
    for (int c = 0; c < 4; c++) {
        J->rgba[4 * idx + c] = out[c];
        if (J->rgba_alt) J->rgba_alt[4 * idx + c] = alt[c];
    }
    if (J->tie) J->tie[idx] = (uint8_t)(tie_k >= 0);
    J->aux2[idx] = T;
    if (J->nsamp) J->nsamp[idx] = ns;
}

/* pdf: npix x 32 (may be NULL for INVCDF with lambda = 1); occ: cell-brick
 * occupancy (RANGE). Returns 0, or 1 for invalid arguments. */
int orc_importance(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
                   const orc_params *prm, const int32_t *pix, int64_t npix, const float *pdf,
                   const uint8_t *occ, int nimp, int sampling, float lambda, double *rgba, double *rgba_alt,
                   uint8_t *tie, double *tfinal, int32_t *nsamp, int nthreads) {
    if (nimp < 1 || (sampling != ORC_SAMPLING_RANGE && sampling != ORC_SAMPLING_INVCDF)) return 1;
    if (sampling == ORC_SAMPLING_RANGE && (!pdf || !occ)) return 1;
    if (sampling == ORC_SAMPLING_INVCDF && (!(lambda >= 0.0f && lambda <= 1.0f) || (!pdf && lambda != 1.0f)))
        return 1;
    scene S;
    int rc = scene_init(&S, vol, tf, cam, prm);
    if (rc) { scene_free(&S); return rc; }
    job J;
    memset(&J, 0, sizeof J);
    J.S = &S;
    J.pix = pix;
    J.npix = pix ? npix : (int64_t)cam->width * cam->height;
    J.fn = importance_pixel;
    J.pdf = pdf;
    J.occ = occ;
    J.nimp = nimp;
    J.sampling = sampling;
    J.lambda = lambda;
    J.rgba = rgba;
    J.rgba_alt = rgba_alt;
    J.tie = tie;
    J.aux2 = tfinal;
    J.nsamp = nsamp;
    int nt = nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads);
    J.fbuf = (float **)calloc((size_t)nt, sizeof(float *));
    int ok = J.fbuf != NULL;
    for (int i = 0; ok && i < nt; i++) ok = (J.fbuf[i] = (float *)malloc(2 * (size_t)nimp * sizeof(float))) != NULL;
    if (ok) run_job(&J, nt, 0);
    for (int i = 0; J.fbuf && i < nt; i++) free(J.fbuf[i]);
    free(J.fbuf);
    scene_free(&S);
    return ok ? 0 : 2;
}

/* The positions and segment lengths of one pixel's importance samples (the
 * sampling step alone, for the tests of the sampling rules). Returns the
 * number of samples written (nimp; 0 for a ray that misses), or -1. */
int orc_importance_positions(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
                             const orc_params *prm, int x, int y, const float *pdf, const uint8_t *occ, int nimp,
                             int sampling, float lambda, float *t, float *len) {
    if (nimp < 1) return -1;
    scene S;
    if (scene_init(&S, vol, tf, cam, prm)) { scene_free(&S); return -1; }
    ray R;
    ray_setup_f32(&S, S.P.step_vox, x, y, &R);
    int n = 0;
    if (R.hit) {
        importance_positions(&S, &R, pdf, occ, nimp, sampling, lambda, t, len);
        n = nimp;
    }
    scene_free(&S);
    return n;
}

/* ------------------------------------------------------------------------ */
/* inputs of the learned proposal                                            */
/* ------------------------------------------------------------------------ */
/* Per ray 112 features: the entry point e = fma(t_near, d, o) / (N - 1) (FP32,
 * as the ray specification) and the world direction, x = (e, dir); for each x_c
 * and j = 0..5, sin(2^j pi x_c) and cos(2^j pi x_c) in FP64; for b = 0..31 the
 * occupancy bit of the cell-brick holding the point at
 * t = fma(b + 0.5, (t_far - t_near) / 32, t_near); two zeros. occ is the
 * cell-brick occupancy (x fastest). Rays that miss give zeros. */
static int brick_of_point(const scene *S, const double p[3], const int nb[3]) {
    int idx[3];
    for (int a = 0; a < 3; a++) {
        int i;
        double w;
        cell(p[a], S->n[a], &i, &w);
        idx[a] = i / 16;
    }
    return (idx[2] * nb[1] + idx[1]) * nb[0] + idx[0];
}

int orc_proposal_features(const orc_volume *vol, const orc_tf *tf, const orc_camera *cam,
                          const orc_params *prm, const int32_t *pix, int64_t npix,
                          const uint8_t *occ, double *feat) {
    scene S;
    int rc = scene_init(&S, vol, tf, cam, prm);
    if (rc) { scene_free(&S); return rc; }
    int nb[3];
    for (int a = 0; a < 3; a++) nb[a] = (S.n[a] - 1 + 15) / 16;
    int64_t n = pix ? npix : (int64_t)cam->width * cam->height;
    for (int64_t r = 0; r < n; r++) {
        int64_t lin = pix ? (int64_t)pix[r] : r;
        int x = (int)(lin % S.W), y = (int)(lin / S.W);
        double *f = feat + 112 * r;
        for (int i = 0; i < 112; i++) f[i] = 0.0;
        ray R;
        ray_setup_f32(&S, S.P.step_vox, x, y, &R);
        if (!R.hit) continue;
        float xs[6];
        for (int c = 0; c < 3; c++) {
            xs[c] = fmaf(R.tn, R.d[c], R.o[c]) / (float)(S.n[c] - 1);
            xs[3 + c] = R.dir[c];
        }
        for (int c = 0; c < 6; c++) f[c] = (double)xs[c];
        for (int c = 0; c < 6; c++)
            for (int j = 0; j < 6; j++) {
                double arg = 3.14159265358979323846 * ldexp((double)xs[c], j);
                f[6 + 12 * c + 2 * j] = sin(arg);
                f[7 + 12 * c + 2 * j] = cos(arg);
            }
        float bw = (R.tf - R.tn) / 32.0f;
        for (int b = 0; b < 32; b++) {
            float t = fmaf((float)b + 0.5f, bw, R.tn);
            double p[3];
            for (int c = 0; c < 3; c++) p[c] = (double)fmaf(t, R.d[c], R.o[c]);
            f[78 + b] = occ[brick_of_point(&S, p, nb)] ? 1.0 : 0.0;
        }
    }
    scene_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* empty-space structures                                                     */
/* ------------------------------------------------------------------------ */
/* Cell-brick b along an axis holds the cells whose base index lies in
 * 16b..16b+15. A trilinear sample reads the voxels base..base+1, so the
 * brick's footprint is the voxels 16b..min(16b+16, n-1); a B-spline sample
 * reads base-1..base+2 (clamped), so its footprint is
 * max(16b-1, 0)..min(16b+17, n-1). There are ceil((n-1)/16) cell-bricks per
 * axis, x fastest. Values clamp to vmax. */
void orc_brick_minmax_filter(const orc_volume *vol, int filter, uint16_t *mn, uint16_t *mx) {
    int n[3] = {vol->nx, vol->ny, vol->nz};
    int nb[3];
    int before = filter == ORC_BSPLINE ? 1 : 0, after = filter == ORC_BSPLINE ? 17 : 16;
    for (int a = 0; a < 3; a++) nb[a] = (n[a] - 1 + 15) / 16;
    for (int bz = 0; bz < nb[2]; bz++)
        for (int by = 0; by < nb[1]; by++)
            for (int bx = 0; bx < nb[0]; bx++) {
                int lo = 65535, hi = 0;
                int z0 = 16 * bz - before > 0 ? 16 * bz - before : 0;
                int y0 = 16 * by - before > 0 ? 16 * by - before : 0;
                int x0 = 16 * bx - before > 0 ? 16 * bx - before : 0;
                int z1 = 16 * bz + after < n[2] - 1 ? 16 * bz + after : n[2] - 1;
                int y1 = 16 * by + after < n[1] - 1 ? 16 * by + after : n[1] - 1;
                int x1 = 16 * bx + after < n[0] - 1 ? 16 * bx + after : n[0] - 1;
                for (int z = z0; z <= z1; z++)
                    for (int y = y0; y <= y1; y++)
                        for (int x = x0; x <= x1; x++) {
                            int v = vol->data[((size_t)z * n[1] + y) * n[0] + x];
                            if (v > vol->vmax) v = vol->vmax;
                            if (v < lo) lo = v;
                            if (v > hi) hi = v;
                        }
                size_t b = ((size_t)bz * nb[1] + by) * nb[0] + bx;
                mn[b] = (uint16_t)lo;
                mx[b] = (uint16_t)hi;
            }
}

void orc_brick_minmax(const orc_volume *vol, uint16_t *mn, uint16_t *mx) {
    orc_brick_minmax_filter(vol, ORC_TRILINEAR, mn, mx);
}

/* A brick is occupied unless every table entry a sample inside it can touch
 * has zero opacity. For values in [mn, mx] the lerp touches entries
 * lo = floor(u(mn)) .. hi = min(floor(u(mx)) + 1, K - 1), with the table
 * coordinate of the written FP32 specification: raw codes v give
 * u(v) = fl(v * c) with c = fl((K - 1) / vmax); FP16 storage (value_mode 1)
 * holds h = fp16((code - o) / o) and gives u(h) = fl((h + 1) * c) with
 * c = fl((K - 1) / fl(vmax / o)) (h + 1 is exact in FP32). u is monotone in
 * the stored value, so every sample inside the brick has its coordinate in
 * [u(mn), u(mx)]. With a 2-D table the
 * gradient coordinate of a sample is not bounded by the grid, so every row of
 * those entries must have zero opacity. */
void orc_occupancy(const orc_volume *vol, const orc_tf *tf, const uint16_t *mn,
                   const uint16_t *mx, uint8_t *occ) {
    int nb = ((vol->nx - 1 + 15) / 16) * ((vol->ny - 1 + 15) / 16) * ((vol->nz - 1 + 15) / 16);
    int K = tf->K;
    float full = vol->value_mode ? (float)vol->vmax / (float)f16_offset(vol->vmax) : (float)vol->vmax;
    float c = (float)(K - 1) / full;
    for (int b = 0; b < nb; b++) {
        long lo, hi;
        float vmn = (float)mn[b], vmx = (float)mx[b];
        if (vol->value_mode) {
            vmn = f16_value(mn[b], vol->vmax) + 1.0f;
            vmx = f16_value(mx[b], vol->vmax) + 1.0f;
        }
        lo = (long)floorf(vmn * c);
        hi = (long)floorf(vmx * c) + 1;
        if (hi > K - 1) hi = K - 1;
        if (lo > K - 1) lo = K - 1;
        int any = 0;
        int rows = tf->M >= 2 ? tf->M : 1;
        for (int j = 0; j < rows; j++)
            for (long i = lo; i <= hi; i++) {
                size_t e = 4 * ((size_t)j * K + (size_t)i) + 3;
                double a = tf->fp16 ? half_round(tf->rgba[e]) : (double)tf->rgba[e];
                if (a != 0.0) any = 1;
            }
        occ[b] = (uint8_t)any;
    }
}
