"""Seeded synthetic inputs for the raycaster: MRI-like head phantoms, transfer-
function tables, orbit cameras and pixel samples.

This module is shared by the CUDA path's tests and bench and by the FP64 oracle.
It holds none of the rendering method's arithmetic (no ray setup, sampling,
classification, shading or compositing): it only draws inputs. The paper's own
data (50-100 brain MRI volumes, Sec. 4.4) is not available, so these phantoms stand
in for it: nested ellipsoids with the intensity classes of skull, CSF, grey and
white matter, one tumor sphere and Rician noise.

Random numbers come from one counter-based generator: output ``i`` of SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014)
seeded with ``mix64(seed)``, i.e. ``mix64(mix64(seed) + (i + 1) * GAMMA)``.
Normals use the Box-Muller transform on two such uniforms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

VMAX = 4095  # 12-bit MRI intensities

# Intensity classes of the head phantom (value units 0..4095).
SKULL, CSF, GREY, WHITE, TUMOR = 3000, 400, 1400, 1800, 2600
# Nested ellipsoid shells: (outer normalised radius, value), outermost first.
LAYERS = ((0.92, SKULL), (0.80, CSF), (0.74, GREY), (0.58, WHITE))


# --------------------------------------------------------------------------
# counter-based random numbers
# --------------------------------------------------------------------------
def mix64(z):
    """SplitMix64 output finaliser on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed: int, idx) -> np.ndarray:
    """Output ``idx`` (0-based) of SplitMix64 seeded with ``mix64(seed)``."""
    key = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + (idx + np.uint64(1)) * GAMMA)


def uniform01(seed: int, idx) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1): top 53 bits, centred."""
    u = counter_u64(seed, idx) >> np.uint64(11)
    return (u.astype(np.float64) + 0.5) * (2.0 ** -53)


def normal_pair(seed: int, idx):
    """Two independent standard normals per index (Box-Muller)."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = uniform01(seed, idx * np.uint64(2))
    u2 = uniform01(seed, idx * np.uint64(2) + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


# --------------------------------------------------------------------------
# head phantom
# --------------------------------------------------------------------------
@dataclass
class Phantom:
    vol: np.ndarray            # uint16, shape (nz, ny, nx): x fastest
    dims: tuple                # (nx, ny, nz)
    spacing: tuple             # (sx, sy, sz) mm
    tumor_center_mm: tuple
    tumor_radius_mm: float
    seed: int
    sigma: float
    meta: dict = field(default_factory=dict)


def _extent(dims, spacing):
    return np.array([(n - 1) * s for n, s in zip(dims, spacing)], dtype=np.float64)


def _draw_tumor(seed, dims, spacing, radius_vox):
    """Seeded tumor centre uniformly inside the white-matter ellipsoid, far
    enough in that the sphere stays inside it; radius in units of min spacing."""
    E = _extent(dims, spacing)
    half = E / 2.0
    r_mm = radius_vox * min(spacing)
    r_norm = r_mm / half.min()
    limit = max(LAYERS[-1][0] - r_norm, 0.05)
    for a in range(10000):
        u = uniform01(seed ^ 0x5475_6D6F72, np.arange(3 * a, 3 * a + 3))
        q = 2.0 * u - 1.0                      # uniform in the unit ball by rejection
        if float(np.sqrt((q * q).sum())) <= 1.0:
            return tuple(float(v) for v in half + limit * q * half), r_mm
    raise RuntimeError("tumor placement failed")


def head_phantom(dims, spacing, seed, sigma=40.0, tumor_radius_vox=6.0,
                 tumor_center_mm=None, vmax=VMAX, chunk_slices=16) -> Phantom:
    """Nested-ellipsoid head phantom, x fastest, values 0..vmax (uint16).

    The ellipsoids are centred at E/2 with semi-axes (fraction * E/2), E = (N-1)*s,
    so anisotropic spacing keeps the shape. Voxel i sits at world i*s. Rician
    noise: v = round(sqrt((v0 + sigma*n1)^2 + (sigma*n2)^2)), clamped to 0..vmax,
    with (n1, n2) drawn per voxel from the counter generator keyed by the voxel's
    linear index.
    """
    nx, ny, nz = (int(d) for d in dims)
    sp = tuple(float(s) for s in spacing)
    E = _extent((nx, ny, nz), sp)
    half = E / 2.0
    if tumor_center_mm is None:
        tc, r_mm = _draw_tumor(seed, (nx, ny, nz), sp, tumor_radius_vox)
    else:
        tc, r_mm = tuple(float(v) for v in tumor_center_mm), tumor_radius_vox * min(sp)
    out = np.empty((nz, ny, nx), dtype=np.uint16)
    xs = (np.arange(nx) * sp[0] - half[0]) / half[0]
    ys = (np.arange(ny) * sp[1] - half[1]) / half[1]
    xw = np.arange(nx) * sp[0]
    yw = np.arange(ny) * sp[1]
    noise_seed = seed ^ 0x4E6F697365
    for z0 in range(0, nz, chunk_slices):
        z1 = min(nz, z0 + chunk_slices)
        zs = (np.arange(z0, z1) * sp[2] - half[2]) / half[2]
        rho = np.sqrt(zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2)
        v0 = np.zeros(rho.shape, dtype=np.float64)
        for radius, value in LAYERS:
            v0[rho <= radius] = value
        zw = np.arange(z0, z1) * sp[2]
        d2 = ((zw[:, None, None] - tc[2]) ** 2 + (yw[None, :, None] - tc[1]) ** 2
              + (xw[None, None, :] - tc[0]) ** 2)
        v0[d2 <= r_mm * r_mm] = TUMOR
        if sigma > 0:
            lin = np.arange(z0 * nx * ny, z1 * nx * ny, dtype=np.uint64).reshape(v0.shape)
            n1, n2 = normal_pair(noise_seed, lin)
            v = np.rint(np.sqrt((v0 + sigma * n1) ** 2 + (sigma * n2) ** 2))
        else:
            v = v0
        out[z0:z1] = np.clip(v, 0, vmax).astype(np.uint16)
    return Phantom(out, (nx, ny, nz), sp, tc, r_mm, seed, sigma)


def symmetric_phantom(n_xy, n_z, spacing_xy=1.0, spacing_z=1.0, tumor_radius_vox=4.0):
    """Noise-free phantom with the tumor at the centre: invariant under 90-degree
    rotations about z and under x or y mirroring (equal x/y dims and spacing)."""
    dims = (n_xy, n_xy, n_z)
    sp = (spacing_xy, spacing_xy, spacing_z)
    c = tuple(float(v) for v in _extent(dims, sp) / 2.0)
    return head_phantom(dims, sp, seed=0, sigma=0.0, tumor_radius_vox=tumor_radius_vox,
                        tumor_center_mm=c)


# --------------------------------------------------------------------------
# transfer functions
# --------------------------------------------------------------------------
# Piecewise-linear control points (value, r, g, b, alpha): straight colour and
# opacity per reference step. Zero opacity below 300 keeps the Rician background
# (sigma 40) empty; every ramp spans >= 8 entries of a 256-entry table.
DEFAULT_TF_POINTS = (
    (0.0, 0.0, 0.0, 0.0, 0.0),
    (300.0, 0.0, 0.0, 0.0, 0.0),
    (400.0, 0.25, 0.45, 1.0, 0.02),    # CSF, blue
    (900.0, 0.6, 0.55, 0.7, 0.02),
    (1400.0, 0.9, 0.7, 0.6, 0.04),     # grey matter
    (1800.0, 1.0, 0.92, 0.82, 0.06),   # white matter
    (2400.0, 1.0, 0.8, 0.7, 0.06),
    (2600.0, 1.0, 0.12, 0.1, 0.8),     # tumor, red
    (2800.0, 1.0, 0.9, 0.9, 0.1),
    (3000.0, 1.0, 1.0, 1.0, 0.1),      # skull, white
    (4095.0, 1.0, 1.0, 1.0, 0.1),
)


def tf_table(K=256, points=DEFAULT_TF_POINTS, vmax=VMAX) -> np.ndarray:
    """Rasterise control points to a K x 4 float32 RGBA table; entry i holds the
    value i*vmax/(K-1) (the colour and opacity transfer functions of Sec. 2.6
    merged into one table)."""
    pts = np.asarray(points, dtype=np.float64)
    xs = np.arange(K, dtype=np.float64) * (vmax / (K - 1))
    tab = np.stack([np.interp(xs, pts[:, 0], pts[:, c]) for c in range(1, 5)], axis=1)
    return np.clip(tab, 0.0, 1.0).astype(np.float32)


def tf2d_table(K=256, M=32, gmax=1200.0, points=DEFAULT_TF_POINTS, vmax=VMAX, floor=0.3) -> np.ndarray:
    """Two-dimensional table over (gradient magnitude, value): M rows of K
    entries, float32 (M, K, 4); row j holds |grad f| = j*gmax/(M-1) codes per
    mm, entry i the value i*vmax/(K-1). Colour is the 1-D table's; opacity is
    the 1-D opacity times a boundary weight that rises from `floor` at
    |grad f| = 0 to 1 at gmax/2 (smoothstep), so that tissue interfaces stand
    out over homogeneous interiors. Rows are tinted slightly warmer with
    gradient so the gradient axis changes colour as well as opacity."""
    base = tf_table(K, points, vmax).astype(np.float64)
    g = np.arange(M, dtype=np.float64) / (M - 1)
    x = np.clip(g / 0.5, 0.0, 1.0)
    wgt = floor + (1.0 - floor) * x * x * (3.0 - 2.0 * x)
    tab = np.repeat(base[None], M, axis=0)
    tab[..., 3] *= wgt[:, None]
    tab[..., 0] = np.minimum(1.0, tab[..., 0] * (1.0 + 0.15 * g[:, None]))
    tab[..., 2] *= (1.0 - 0.3 * g[:, None])
    return np.clip(tab, 0.0, 1.0).astype(np.float32)


def random_tf(K, seed, alpha_max=0.1, n_points=12, vmax=VMAX) -> np.ndarray:
    """Seeded smooth random table: n_points random control points over
    300..vmax (opacity 0 below 300), colours in [0,1], opacity in [0, alpha_max]."""
    u = uniform01(seed, np.arange(5 * n_points)).reshape(n_points, 5)
    xs = np.linspace(300.0, vmax, n_points)
    pts = [(0.0, 0, 0, 0, 0.0), (300.0, 0, 0, 0, 0.0)]
    for j in range(n_points):
        pts.append((xs[j], u[j, 0], u[j, 1], u[j, 2], alpha_max * u[j, 3]))
    return tf_table(K, pts, vmax)


def noise_tf(K, seed, alpha_max=0.1) -> np.ndarray:
    """Seeded i.i.d. noise table: colours in [0,1], opacity in [0, alpha_max]."""
    u = uniform01(seed, np.arange(4 * K)).reshape(K, 4)
    tab = u.copy()
    tab[:, 3] *= alpha_max
    return tab.astype(np.float32)


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------
def _cos_sin_deg(deg):
    """Exact values at multiples of 90 degrees (rotation tests need them)."""
    d = float(deg) % 360.0
    exact = {0.0: (1.0, 0.0), 90.0: (0.0, 1.0), 180.0: (-1.0, 0.0), 270.0: (0.0, -1.0)}
    if d in exact:
        return exact[d]
    r = math.radians(d)
    return math.cos(r), math.sin(r)


def f32(x):
    return float(np.float32(x))


def orbit_camera(dims, spacing, azimuth_deg, elevation_deg=20.0, fovy_deg=30.0,
                 width=256, height=256, distance_scale=1.1) -> dict:
    """Perspective camera on an orbit about the z axis through the volume centre.

    Distance D = distance_scale * R / sin(fovy/2) with R the half diagonal of the
    volume box, so the bounding sphere fits the view. Returns FP32-rounded eye,
    target and up (up = +z) plus fovy and image size.
    """
    E = _extent(dims, spacing)
    c = E / 2.0
    R = float(np.sqrt((E * E).sum())) / 2.0
    D = distance_scale * R / math.sin(math.radians(fovy_deg / 2.0))
    ca, sa = _cos_sin_deg(azimuth_deg)
    ce, se = _cos_sin_deg(elevation_deg)
    # offsets on a 2^-10 mm grid: centre + offset is then exact in FP32, so
    # cameras at azimuths theta and theta + 90k are exact rotations of each other
    off = [round(D * ce * ca * 1024.0) / 1024.0, round(D * ce * sa * 1024.0) / 1024.0,
           round(D * se * 1024.0) / 1024.0]
    eye = (c[0] + off[0], c[1] + off[1], c[2] + off[2])
    return dict(eye=tuple(f32(v) for v in eye), target=tuple(f32(v) for v in c),
                up=(0.0, 0.0, 1.0), fovy_deg=f32(fovy_deg), width=int(width), height=int(height))


def sample_pixels(width, height, n, seed) -> np.ndarray:
    """n distinct pixel indices (y*width + x), ranked by the counter generator."""
    npx = width * height
    n = min(n, npx)
    keys = counter_u64(seed, np.arange(npx, dtype=np.uint64))
    sel = np.argpartition(keys, n - 1)[:n]
    return np.sort(sel).astype(np.int32)


# --------------------------------------------------------------------------
# workloads (shapes of the paper's brain-MRI use case; synthetic)
# --------------------------------------------------------------------------
WORKLOADS = {
    "plain_64x64x32": dict(dims=(64, 64, 32), spacing=(1.0, 1.0, 3.0), seed=1, K=256,
                           width=256, height=256, step=0.5, shade=False, term=0.99,
                           azimuths=(0.0, 120.0, 240.0), tumor_radius_vox=6.0),
    "shaded_256x256x180": dict(dims=(256, 256, 180), spacing=(1.0, 1.0, 1.0), seed=2, K=256,
                               width=1024, height=1024, step=0.5, shade=True, term=0.99,
                               azimuths=tuple(10.0 * i for i in range(36)), tumor_radius_vox=6.0),
    "precision_512x512x256": dict(dims=(512, 512, 256), spacing=(1.0, 1.0, 1.0), seed=3, K=1024,
                                  width=2048, height=2048, step=0.25, shade=True, term=0.99,
                                  azimuths=(0.0,), tumor_radius_vox=6.0, ray_seed=3003,
                                  n_rays=4096, small_width=512),
    "diff_128x128x96": dict(dims=(128, 128, 96), spacing=(1.0, 1.0, 1.0), seed=4, K=256,
                            width=512, height=512, step=0.5, shade=False, term=0.99,
                            azimuths=tuple(45.0 * i for i in range(8)), tumor_radius_vox=6.0,
                            hidden_tf_seed=104, init_tf_seed=204),
    "proposal_256x256x180": dict(dims=(256, 256, 180), spacing=(1.0, 1.0, 1.0), K=256,
                                 width=1024, height=1024, step=0.5, shade=True, term=0.99,
                                 train_seeds=tuple(range(1000, 1032)),
                                 eval_seeds=tuple(range(1032, 1040)),
                                 azimuths=tuple(10.0 * i for i in range(36))),
}


def proposal_phantom(seed, dims=(256, 256, 180), spacing=(1.0, 1.0, 1.0)):
    """Phantom with seeded tumor radius in [3, 15] voxels and seeded position."""
    r = 3.0 + 12.0 * float(uniform01(seed ^ 0x52616469, np.arange(1))[0])
    return head_phantom(dims, spacing, seed, tumor_radius_vox=r)


def workload_phantom(name, **over):
    w = dict(WORKLOADS[name])
    w.update(over)
    return head_phantom(w["dims"], w["spacing"], w["seed"], tumor_radius_vox=w["tumor_radius_vox"])


# --------------------------------------------------------------------------
# initial parameters of the proposal network (seeded input)
# --------------------------------------------------------------------------
PROPOSAL_LAYERS = ((112, 64), (64, 64), (64, 64), (64, 40))
PROPOSAL_PARAMS = 18152


def proposal_init_params(seed, n_feat_used=110, n_out_used=33) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)) and zero biases, in the
    parameter order W1, b1, W2, b2, W3, b3, W4, b4 (weights input-major).
    Padding inputs (features 110, 111) and padding outputs (33..39) get zero
    weights."""
    out = []
    off = 0
    for li, (k, n) in enumerate(PROPOSAL_LAYERS):
        fan_in = n_feat_used if li == 0 else k
        u = uniform01(seed + 7919 * li, np.arange(k * n)).reshape(k, n)
        w = (2.0 * u - 1.0) * np.sqrt(6.0 / fan_in)
        if li == 0:
            w[n_feat_used:, :] = 0.0
        if li == len(PROPOSAL_LAYERS) - 1:
            w[:, n_out_used:] = 0.0
        out.append(w.reshape(-1))
        out.append(np.zeros(n))
        off += k * n + n
    p = np.concatenate(out).astype(np.float32)
    assert p.size == PROPOSAL_PARAMS
    return p


def proposal_batch(seed, n):
    """Seeded feature rows and profile targets with the value ranges of real
    rays (6 coordinates in [0, 1] or [-1, 1], 72 encodings in [-1, 1], 32 0/1
    occupancy bits, 2 zeros) for unit tests of the network."""
    u = uniform01(seed, np.arange(n * 78)).reshape(n, 78)
    f = np.zeros((n, 112))
    f[:, :3] = u[:, :3]
    f[:, 3:78] = 2.0 * u[:, 3:78] - 1.0
    bits = uniform01(seed + 1, np.arange(n * 32)).reshape(n, 32) < 0.6
    f[:, 78:110] = bits
    w = uniform01(seed + 2, np.arange(n * 32)).reshape(n, 32) ** 4
    tot = uniform01(seed + 3, np.arange(n))
    bins = w / w.sum(axis=1, keepdims=True) * tot[:, None]
    bins[: max(1, n // 16)] = 0.0                          # some rays without opacity
    tgt = np.concatenate([bins, (1.0 - bins.sum(axis=1))[:, None]], axis=1)
    return f.astype(np.float32), tgt.astype(np.float32)


def _proposal_vol(seed):
    return proposal_phantom(seed).vol


def proposal_phantoms(seeds, workers=None):
    """proposal_phantom(seed).vol for every seed, generated in a pool of
    spawned processes (safe to call after CUDA has been initialised)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    seeds = list(seeds)
    workers = workers or max(1, min(len(seeds), (os.cpu_count() or 2) - 1, 16))
    if workers == 1 or len(seeds) == 1:
        return [_proposal_vol(s) for s in seeds]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_proposal_vol, seeds))
