"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-worked
closed forms (tests/golden), exact reproduction of affine fields by trilinear
resampling, symmetries of the ray geometry, the order independence of
compositing (Eq. 4 summed front-to-back or back-to-front), convergence to the
continuous emission-absorption integral (Eq. 5), and finite differences.
"""
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def axis_camera(nx, yc, zc, back=50.0):
    """Single-pixel camera on the +x side looking down -x along the line
    (y, z) = (yc, zc) mm: the one ray has direction exactly (-1, 0, 0)."""
    return dict(eye=(float(nx - 1 + back), float(yc), float(zc)), target=(0.0, float(yc), float(zc)),
                up=(0.0, 0.0, 1.0), fovy_deg=30.0, width=1, height=1)


def identity_tf(rows=None):
    """K = 4096 entries so the table coordinate of value v is v itself."""
    tf = np.zeros((4096, 4), dtype=np.float32)
    for v, rgba in (rows or {}).items():
        for w in (v - 1, v, v + 1):
            tf[w] = rgba
    return tf


# --------------------------------------------------------------------------
# geometry of the ray (Sec. 4.1 step 1)
# --------------------------------------------------------------------------
def test_axis_ray_geometry(orc):
    vol = np.zeros((8, 8, 40), dtype=np.uint16)
    sc = orc.Scene(vol, (1, 1, 1), identity_tf(), axis_camera(40, 3.0, 4.0), step=0.5)
    g = orc.ray_geometry(sc, 0, 0)
    assert g["hit"]
    assert np.array_equal(g["dir"], [-1.0, 0.0, 0.0])
    assert g["tn"] == 50.0 and g["tf"] == 89.0          # eye at x = 89, box x in [0, 39]
    assert g["nsamp"] == 2 * 39 + 1                      # floor(39 / 0.5) + 1


def test_axis_ray_hits_voxel_centres(orc):
    """Samples at integer positions return the voxel value; half-way samples
    return the mean of the two neighbours (hand-computed trilinear)."""
    rng = np.random.default_rng(5)
    vol = rng.integers(0, 4096, size=(6, 7, 30)).astype(np.uint16)
    yc, zc = 2.0, 3.0
    sc = orc.Scene(vol, (1, 1, 1), identity_tf(), axis_camera(30, yc, zc), step=0.5, term=1.0)
    s = orc.ray_samples(sc, 0, 0)
    assert len(s["v"]) == 59
    row = vol[int(zc), int(yc), :].astype(np.float64)
    for k in range(59):
        x = 29 - 0.5 * k
        assert s["px"][k] == x
        expect = row[int(x)] if k % 2 == 0 else 0.5 * (row[int(x)] + row[int(x) + 1])
        assert s["v"][k] == pytest.approx(expect, abs=1e-9)


def test_anisotropic_spacing_geometry(orc):
    """World distance t maps to index space through the spacing: along z with
    3 mm slices the ray crosses (nz-1) slices over (nz-1)*3 mm."""
    vol = np.zeros((20, 8, 8), dtype=np.uint16)
    cam = dict(eye=(3.0, 4.0, 19 * 3.0 + 30.0), target=(3.0, 4.0, 0.0), up=(0.0, 1.0, 0.0),
               fovy_deg=30.0, width=1, height=1)
    sc = orc.Scene(vol, (1, 1, 3), identity_tf(), cam, step=0.5)
    g = orc.ray_geometry(sc, 0, 0)
    assert g["hit"] and g["tn"] == 30.0 and g["tf"] == 30.0 + 57.0
    assert g["ds"] == 0.5                                 # half the finest spacing
    assert np.array_equal(g["d"], [0.0, 0.0, -1.0 / 3.0]) or abs(g["d"][2] + 1 / 3) < 1e-7
    assert g["nsamp"] == 115


def test_miss_gives_zero(orc):
    vol = np.full((8, 8, 8), 3000, dtype=np.uint16)
    cam = dict(eye=(100.0, 100.0, 100.0), target=(200.0, 200.0, 200.0), up=(0.0, 0.0, 1.0),
               fovy_deg=30.0, width=8, height=8)
    r = orc.render(orc.Scene(vol, (1, 1, 1), synth.tf_table(256), cam))
    assert np.all(r["rgba"] == 0) and np.all(r["nsamp"] == 0)


# --------------------------------------------------------------------------
# trilinear resampling (Sec. 3.2): affine fields are reproduced exactly
# --------------------------------------------------------------------------
def ramp_volume(dims, a, b, c, d):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = a * x + b * y + c * z + d
    assert v.min() >= 0 and v.max() <= 4095
    return v.astype(np.uint16)


def test_trilinear_reproduces_affine_ramp(orc):
    dims = (40, 30, 20)
    a, b, c, d = 7, 11, 13, 100
    vol = ramp_volume(dims, a, b, c, d)
    cam = synth.orbit_camera(dims, (1, 1, 1), 37.0, width=24, height=24)
    sc = orc.Scene(vol, (1, 1, 1), synth.tf_table(256), cam, term=1.0)
    checked = 0
    for (x, y) in [(12, 12), (5, 17), (20, 3), (9, 9)]:
        s = orc.ray_samples(sc, x, y)
        if len(s["v"]) == 0:
            continue
        px = np.clip(s["px"], 0, dims[0] - 1)
        py = np.clip(s["py"], 0, dims[1] - 1)
        pz = np.clip(s["pz"], 0, dims[2] - 1)
        np.testing.assert_allclose(s["v"], a * px + b * py + c * pz + d, rtol=0, atol=1e-9)
        checked += len(s["v"])
    assert checked > 100


# --------------------------------------------------------------------------
# compositing (Sec. 4.2, Eq. 3-5)
# --------------------------------------------------------------------------
def read_golden_slab():
    rows = []
    with open(os.path.join(GOLDEN, "constant_slab.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                a, r, n, op = line.split()
                rows.append((float(a), float(r), int(n), float(op)))
    return rows


@pytest.mark.parametrize("row", read_golden_slab())
def test_constant_slab_closed_form(orc, row):
    a, r, n_stop, op = row
    V0 = 2000
    colour = (0.25, 0.5, 1.0)
    vol = np.full((8, 8, 300), V0, dtype=np.uint16)
    tf = identity_tf({V0: (*colour, a)})
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(300, 3.5, 4.25), step=r, term=0.99)
    out = orc.render(sc)
    assert out["nsamp"][0, 0] == n_stop
    af = float(np.float32(a))
    expect = 1.0 - (1.0 - af) ** (r * n_stop)
    assert out["rgba"][0, 0, 3] == pytest.approx(expect, abs=1e-12)
    assert out["rgba"][0, 0, 3] == pytest.approx(op, abs=2e-8)
    np.testing.assert_allclose(out["rgba"][0, 0, :3], np.float32(colour) * expect, atol=1e-12)


def test_constant_slab_without_termination(orc):
    """term = 1: all floor(L/ds)+1 samples are composited."""
    V0, a = 1000, 0.01
    vol = np.full((8, 8, 100), V0, dtype=np.uint16)
    tf = identity_tf({V0: (1.0, 1.0, 1.0, a)})
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(100, 3.0, 3.0), step=0.5, term=1.0)
    out = orc.render(sc)
    n = 199
    assert out["nsamp"][0, 0] == n
    expect = 1.0 - (1.0 - float(np.float32(a))) ** (0.5 * n)
    assert out["rgba"][0, 0, 3] == pytest.approx(expect, abs=1e-12)


def test_front_to_back_equals_back_to_front(orc):
    """Eq. 4 is a sum; evaluated from the back (Eq. 5's S = 0 end) with
    C <- a'c + (1 - a') C it must give the oracle's front-to-back result."""
    ph = synth.head_phantom((48, 48, 40), (1, 1, 1), seed=9, tumor_radius_vox=5)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 30.0, width=32, height=32)
    sc = orc.Scene(ph.vol, ph.spacing, synth.tf_table(256), cam, term=1.0, shade=True)
    img = orc.render(sc)["rgba"]
    tested = 0
    for (x, y) in [(16, 16), (10, 20), (22, 13), (16, 5)]:
        s = orc.ray_samples(sc, x, y)
        if len(s["v"]) == 0:
            continue
        C = np.zeros(3)
        A = 0.0
        for k in range(len(s["v"]) - 1, -1, -1):
            ak = s["a_corr"][k]
            col = np.array([s["col_r"][k], s["col_g"][k], s["col_b"][k]])
            C = ak * col + (1 - ak) * C
            A = ak + (1 - ak) * A
        np.testing.assert_allclose(img[y, x, :3], C, rtol=0, atol=1e-12)
        assert img[y, x, 3] == pytest.approx(A, abs=1e-12)
        tested += 1
    assert tested >= 3


def test_converges_to_emission_absorption_integral(orc):
    """Constant extinction kappa along a chord of length L: Eq. 5 gives opacity
    1 - exp(-kappa L) and colour c (1 - exp(-kappa L)). With the per-step
    opacity correction the march composites floor(L/ds)+1 segments of length
    ds, so its error is below kappa ds and shrinks with ds."""
    V0 = 1500
    a_ref = 0.02                       # opacity per reference step (1 mm)
    kappa = -math.log(1.0 - float(np.float32(a_ref)))
    vol = np.full((8, 8, 120), V0, dtype=np.uint16)
    tf = identity_tf({V0: (1.0, 0.5, 0.25, a_ref)})
    errs = []
    for step in (1.0, 0.5, 0.25, 0.125):
        sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(120, 3.0, 3.0, back=10.3), step=step,
                       term=1.0)
        g = orc.ray_geometry(sc, 0, 0)
        L = g["tf"] - g["tn"]
        out = orc.render(sc)["rgba"][0, 0]
        exact = 1.0 - math.exp(-kappa * L)
        err = abs(out[3] - exact)
        assert err <= kappa * step + 1e-12
        assert out[1] == pytest.approx(0.5 * out[3], abs=1e-12)
        errs.append(err)
    assert errs[-1] < errs[0] / 4


# --------------------------------------------------------------------------
# symmetry of the whole pipeline
# --------------------------------------------------------------------------
def test_rotation_by_90_degrees(orc):
    """A phantom invariant under 90-degree rotations about z renders the same
    image from azimuths theta and theta + 90 (FP64 ray mode: exact up to
    rounding; FP32 ray specification: up to FP32 position rounding)."""
    ph = synth.symmetric_phantom(40, 30)
    assert np.array_equal(ph.vol, np.rot90(ph.vol, 1, axes=(1, 2)))
    tf = synth.tf_table(256)
    imgs = {}
    for fp64 in (True, False):
        for az in (0.0, 90.0, 180.0, 270.0):
            cam = synth.orbit_camera(ph.dims, ph.spacing, az, width=48, height=48)
            sc = orc.Scene(ph.vol, ph.spacing, tf, cam, shade=True, fp64_rays=fp64, term=1.0)
            imgs[fp64, az] = orc.render(sc)["rgba"]
    assert imgs[True, 0.0][..., 3].max() > 0.5
    for az in (90.0, 180.0, 270.0):
        np.testing.assert_allclose(imgs[True, az], imgs[True, 0.0], atol=1e-9)
        diff = np.abs(imgs[False, az] - imgs[False, 0.0])
        assert np.quantile(diff, 0.99) < 1e-4 and diff.max() < 5e-2


def test_mirror_in_x(orc):
    """Mirroring the volume in x mirrors the image left-right for a camera in
    the mirror plane's normal direction (azimuth 90: camera on +y)."""
    ph = synth.head_phantom((40, 40, 30), (1, 1, 1), seed=12, tumor_radius_vox=4)
    tf = synth.tf_table(256)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 90.0, width=40, height=40)
    a = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, fp64_rays=True, shade=True,
                             term=1.0))["rgba"]
    b = orc.render(orc.Scene(ph.vol[:, :, ::-1], ph.spacing, tf, cam, fp64_rays=True,
                             shade=True, term=1.0))["rgba"]
    assert a[..., 3].max() > 0.3
    np.testing.assert_allclose(b, a[:, ::-1], atol=1e-9)


def test_fp32_rays_close_to_fp64_rays(orc):
    ph = synth.head_phantom((48, 48, 32), (1, 1, 2), seed=1, tumor_radius_vox=5)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 45.0, width=40, height=40)
    tf = synth.tf_table(256)
    a = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, fp64_rays=True, term=1.0))["rgba"]
    b = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, term=1.0))["rgba"]
    assert np.abs(a - b).max() < 2e-2 and np.abs(a - b).mean() < 1e-4


# --------------------------------------------------------------------------
# shading: closed forms for affine fields
# --------------------------------------------------------------------------
@pytest.mark.parametrize("axis_grad,expect_ndl", [((9, 0, 0), 1.0), ((0, 9, 0), 0.0), ((0, 0, 9), 0.0)])
def test_shading_closed_form(orc, axis_grad, expect_ndl):
    """For a ramp v = 9*x + d and a ray along -x the gradient is parallel to
    the view direction (n.L = 1): colour = min(1, rgb (ka + kd) + ks). Ramps
    along y or z are perpendicular (n.L = 0): colour = rgb ka."""
    dims = (30, 20, 20)
    vol = ramp_volume(dims, *axis_grad, 1000)
    tf = np.zeros((256, 4), dtype=np.float32)
    tf[:, :] = (0.5, 0.25, 1.0, 0.01)
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(30, 9.5, 9.5), shade=True, term=1.0,
                   ka=0.1, kd=0.7, ks=0.2)
    s = orc.ray_samples(sc, 0, 0)
    inner = (s["px"] >= 1) & (s["px"] <= 28)        # central differences inside the box
    rgb = np.array([0.5, 0.25, 1.0])
    if expect_ndl == 1.0:
        expect = np.minimum(1.0, rgb * (0.1 + 0.7) + 0.2)
    else:
        expect = rgb * 0.1
    for c, name in enumerate(("col_r", "col_g", "col_b")):
        np.testing.assert_allclose(s[name][inner], expect[c], atol=1e-12)


# --------------------------------------------------------------------------
# other ray functions (Sec. 2.4 ii, Sec. 4.1): closed forms on one ray
# --------------------------------------------------------------------------
def test_mip_average_xray_on_axis_ray(orc):
    rng = np.random.default_rng(3)
    vol = rng.integers(0, 4000, size=(6, 6, 25)).astype(np.uint16)
    row = vol[2, 3, :].astype(np.float64)
    base = dict(step=0.5, term=1.0)
    cam = axis_camera(25, 3.0, 2.0)
    # samples: voxel values at even k, neighbour means at odd k
    samples = []
    for k in range(49):
        x = 24 - 0.5 * k
        samples.append(row[int(x)] if k % 2 == 0 else 0.5 * (row[int(x)] + row[int(x) + 1]))
    samples = np.array(samples)
    mip = orc.render(orc.Scene(vol, (1, 1, 1), identity_tf(), cam, func=orc.MIP, **base))["rgba"][0, 0]
    assert mip[0] == pytest.approx(row.max() / 4095, abs=1e-12) and mip[3] == 1.0
    avg = orc.render(orc.Scene(vol, (1, 1, 1), identity_tf(), cam, func=orc.AVERAGE, **base))["rgba"][0, 0]
    assert avg[0] == pytest.approx(samples.mean() / 4095, abs=1e-12)
    xr = orc.render(orc.Scene(vol, (1, 1, 1), identity_tf(), cam, func=orc.XRAY, **base))["rgba"][0, 0]
    assert xr[0] == pytest.approx(samples.sum() * 0.5 / 4095, abs=1e-12)


def test_isosurface_and_threshold_on_ramp(orc):
    """v = 100 x + 50 along -x: the iso-value 1234 is crossed at x* = 11.84,
    i.e. at t* = tn + (29 - x*) (linear interpolation of an affine field is
    exact). Threshold returns the table colour of the first sample >= 1234."""
    dims = (30, 4, 4)
    vol = ramp_volume(dims, 100, 0, 0, 50)
    cam = axis_camera(30, 1.5, 1.5)
    tf = identity_tf()
    tf[:, 0] = np.arange(4096) / 4095.0
    tf[:, 3] = 0.5
    # the ray enters at x = 29 (v = 2950 >= iso already); look the other way
    cam = dict(eye=(-20.0, 1.5, 1.5), target=(100.0, 1.5, 1.5), up=(0.0, 0.0, 1.0),
               fovy_deg=30.0, width=1, height=1)
    iso = orc.render(orc.Scene(vol, (1, 1, 1), tf, cam, func=orc.ISO, iso=1234.0,
                               term=1.0))["rgba"][0, 0]
    x_star = (1234.0 - 50.0) / 100.0
    assert iso[0] == pytest.approx(20.0 + x_star, abs=1e-9)
    assert iso[2] == math.ceil(x_star / 0.5) and iso[3] == 1.0
    thr = orc.render(orc.Scene(vol, (1, 1, 1), tf, cam, func=orc.THRESHOLD, iso=1234.0,
                               term=1.0))["rgba"][0, 0]
    v_first = 100.0 * (math.ceil(x_star / 0.5) * 0.5) + 50.0
    assert thr[0] == pytest.approx(float(tf[int(v_first), 0]), abs=1e-12) and thr[3] == 1.0


# --------------------------------------------------------------------------
# empty-space structures
# --------------------------------------------------------------------------
def test_brick_minmax_hand_cases(orc):
    vol = np.zeros((20, 40, 35), dtype=np.uint16)     # nz=20, ny=40, nx=35
    vol[5, 5, 16] = 1000       # x = 16 is shared by cell-bricks 0 and 1
    vol[19, 39, 34] = 4095     # last voxel: in the last brick of every axis
    vol[0, 0, 0] = 7
    mn, mx = orc.brick_minmax(vol)
    assert mn.shape == (2, 3, 3)                        # ceil(19/16), ceil(39/16), ceil(34/16)
    assert mx[0, 0, 0] == 1000 and mx[0, 0, 1] == 1000
    assert mx[1, 2, 2] == 4095 and mn[0, 0, 0] == 0
    others = np.ones_like(mx, dtype=bool)
    others[0, 0, 0] = others[0, 0, 1] = others[1, 2, 2] = False
    assert np.all(mx[others] == 0)
    vol2 = np.full((20, 40, 35), 5000, dtype=np.uint16)
    mn2, mx2 = orc.brick_minmax(vol2, vmax=4095)       # codes above vmax clamp
    assert np.all(mn2 == 4095) and np.all(mx2 == 4095)


def test_brick_minmax_brute_force(orc):
    rng = np.random.default_rng(8)
    vol = rng.integers(0, 4096, size=(18, 33, 37)).astype(np.uint16)
    mn, mx = orc.brick_minmax(vol)
    nz, ny, nx = vol.shape
    for bz in range(mn.shape[0]):
        for by in range(mn.shape[1]):
            for bx in range(mn.shape[2]):
                blk = vol[16 * bz:min(16 * bz + 17, nz), 16 * by:min(16 * by + 17, ny),
                          16 * bx:min(16 * bx + 17, nx)]
                assert mn[bz, by, bx] == blk.min() and mx[bz, by, bx] == blk.max()


def test_occupancy_is_conservative(orc):
    """Every sample whose cell lies in an unoccupied brick has opacity exactly
    0, so skipping those bricks cannot change the image."""
    ph = synth.head_phantom((128, 128, 64), (1, 1, 1), seed=21, tumor_radius_vox=5)
    tf = synth.tf_table(256)
    mn, mx = orc.brick_minmax(ph.vol)
    occ = orc.occupancy(ph.dims, tf, mn, mx)
    assert 0 < occ.sum() < occ.size
    cam = synth.orbit_camera(ph.dims, ph.spacing, 20.0, width=32, height=32)
    sc = orc.Scene(ph.vol, ph.spacing, tf, cam, term=1.0)
    skipped = 0
    for (x, y) in [(16, 16), (4, 16), (16, 4), (27, 27), (8, 24), (2, 2), (6, 6), (25, 7)]:
        s = orc.ray_samples(sc, x, y)
        for k in range(len(s["v"])):
            idx = []
            for p, n in ((s["pz"][k], 64), (s["py"][k], 128), (s["px"][k], 128)):
                i = min(int(math.floor(min(max(p, 0), n - 1))), n - 2)
                idx.append(i // 16)
            if not occ[tuple(idx)]:
                assert s["a"][k] == 0.0
                skipped += 1
    assert skipped > 20


def test_occupancy_hand_case(orc):
    """Opacity non-zero only on table entries 100..110 (K = 256): a brick is
    occupied exactly when its [floor(u(min)), floor(u(max)) + 1] overlaps."""
    tf = np.zeros((256, 4), dtype=np.float32)
    tf[100:111, 3] = 0.5
    vmax = 4095                    # u(v) = v * 255 / 4095
    mn = np.array([[[0, 1600, 1780, 1620, 1800, 1500]]], dtype=np.uint16)
    mx = np.array([[[1589, 1700, 4095, 1621, 4095, 1590]]], dtype=np.uint16)
    occ = orc.occupancy((97, 2, 2), tf, mn, mx, vmax=vmax)   # 6 x 1 x 1 bricks
    # u(1589) = 98.95: entries 0..99, all zero -> empty; [1600, 1700] -> 99..106;
    # u(1780) = 110.84 -> from 110 (non-zero); u(1620) = 100.88; u(1800) = 112.09
    # -> 112..255, all zero -> empty; u(1590) = 99.01 -> up to entry 100 -> hit
    assert occ.ravel().tolist() == [0, 1, 1, 1, 0, 1]


# --------------------------------------------------------------------------
# transfer-function gradient: reverse mode against central differences
# --------------------------------------------------------------------------
@pytest.mark.parametrize("bspline", [False, True])
def test_tf_gradient_matches_finite_differences(orc, bspline):
    """Reverse mode against central differences, with trilinear and with
    cubic B-spline reconstruction (the table gradient does not depend on
    how the sample value was reconstructed)."""
    filt = orc.BSPLINE if bspline else orc.TRILINEAR
    ph = synth.head_phantom((32, 32, 24), (1, 1, 1), seed=31, tumor_radius_vox=4)
    # every entry strictly inside (0, 1) so +-h stays a valid table
    tf = synth.noise_tf(256, 7, alpha_max=0.2)
    tf[:, :3] = 0.1 + 0.8 * tf[:, :3]
    tf[:, 3] += 0.02
    cam = synth.orbit_camera(ph.dims, ph.spacing, 30.0, width=16, height=16)
    rng = np.random.default_rng(2)
    dimg = rng.normal(size=(16 * 16, 4))

    def loss(t):
        sc = orc.Scene(ph.vol, ph.spacing, t, cam, term=1.0, shade=True, filter=filt)
        img = orc.render(sc)["rgba"].reshape(-1, 4)
        return float((img * dimg).sum())

    sc = orc.Scene(ph.vol, ph.spacing, tf, cam, term=1.0, shade=True, filter=filt)
    dtf, _ = orc.render_grad(sc, dimg)
    # table entries actually used by the rays, plus unused ones (gradient 0)
    used = np.argsort(-np.abs(dtf).sum(axis=1))[:6]
    h = 1e-3
    checked = 0
    for i in list(used) + [0, 255]:
        for c in range(4):
            # tf is float32; finite differences on an FP64 copy would be
            # rounded back, so perturb by an exactly representable step
            tp = tf.astype(np.float64).copy(); tp[i, c] += h
            tm = tf.astype(np.float64).copy(); tm[i, c] -= h
            if tp[i, c] > 1 or tm[i, c] < 0:
                continue
            fd = (loss(tp.astype(np.float32)) - loss(tm.astype(np.float32))) / (
                float(np.float32(tp[i, c])) - float(np.float32(tm[i, c])))
            assert dtf[i, c] == pytest.approx(fd, rel=2e-3, abs=1e-6)
            checked += 1
    assert checked >= 20


@pytest.mark.parametrize("tf2", [False, True])
def test_tf_gradient_constant_medium_closed_form(orc, tf2):
    """A ray along -x through a volume that varies only in y meets the same
    value (1105) and gradient (30 codes/mm along y) at every sample, so each
    of its n samples is classified alike (alpha, c) and the pixel is
    C = c (1 - (1 - a')^n), A = 1 - (1 - a')^n with a' = 1 - (1 - alpha)^r.
    The table gradient is the chain rule of that closed form, spread over the
    two lerp entries (1-D table) or the four bilinear entries of the cell
    (2-D table: row coordinate 30 (M-1) / gmax = 1.2)."""
    nx, K, M, gmax, r = 60, 256, 5, 100.0, 0.5
    vol = np.broadcast_to((1000 + 30 * np.arange(8))[None, :, None], (8, 8, nx)).astype(np.uint16)
    rng = np.random.default_rng(11)
    shape = (M, K, 4) if tf2 else (K, 4)
    tab = rng.uniform(0.05, 0.95, size=shape).astype(np.float32)
    tab[..., 3] = rng.uniform(0.02, 0.2, size=shape[:-1]).astype(np.float32)
    sc = orc.Scene(vol, (1, 1, 1), tab, axis_camera(nx, 3.5, 4.25), step=r, term=1.0,
                   gmax=gmax if tf2 else None)
    g = np.array([[0.3, -0.7, 0.5, 1.1]])
    dtf, rgba = orc.render_grad(sc, g)
    n = int(orc.render(sc)["nsamp"][0, 0])
    assert n == 119                                    # floor(59 / 0.5) + 1
    u = 1105.0 * (K - 1) / 4095.0
    i = int(np.floor(u)); a = u - i
    t = tab.astype(np.float64)
    if tf2:
        w = 30.0 * (M - 1) / gmax
        j = int(np.floor(w)); b = w - j
        cells = [((j, i), (1 - a) * (1 - b)), ((j, i + 1), a * (1 - b)),
                 ((j + 1, i), (1 - a) * b), ((j + 1, i + 1), a * b)]
    else:
        cells = [((i,), 1 - a), ((i + 1,), a)]
    e = sum(q * t[idx] for idx, q in cells)
    alpha, c = e[3], e[:3]
    ap = 1.0 - (1.0 - alpha) ** r
    Tn = (1.0 - ap) ** n
    np.testing.assert_allclose(rgba[0, :3], c * (1.0 - Tn), rtol=1e-12)
    assert rgba[0, 3] == pytest.approx(1.0 - Tn, rel=1e-12)
    dc = g[0, :3] * (1.0 - Tn)
    dalpha = (g[0, :3] @ c + g[0, 3]) * n * (1.0 - ap) ** (n - 1) * r * (1.0 - alpha) ** (r - 1.0)
    expect = np.zeros_like(dtf)
    for idx, q in cells:
        expect[idx + (slice(0, 3),)] += q * dc
        expect[idx + (3,)] += q * dalpha
    np.testing.assert_allclose(dtf, expect, rtol=1e-9, atol=1e-14)
    assert np.count_nonzero(np.abs(dtf).sum(axis=-1)) == len(cells)


# --------------------------------------------------------------------------
# opacity profiles and importance-sampled compositing
# --------------------------------------------------------------------------
def test_profiles_constant_volume(orc):
    """512 equal segments of a constant medium: weight k = (1-a')^k a', so bin b
    (16 samples) holds (1-a')^(16 b) (1 - (1-a')^16); the bins sum to 1 - T."""
    V0, a = 2000, 0.05
    vol = np.full((8, 8, 60), V0, dtype=np.uint16)
    tf = identity_tf({V0: (1.0, 1.0, 1.0, a)})
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=1.0)
    bins, tfin = orc.profiles(sc)
    g = orc.ray_geometry(sc, 0, 0)
    delta = float(np.float32(g["tf"] - g["tn"]) / np.float32(512))
    ap = 1.0 - (1.0 - float(np.float32(a))) ** delta
    expect = np.array([(1 - ap) ** (16 * b) * (1 - (1 - ap) ** 16) for b in range(32)])
    np.testing.assert_allclose(bins[0], expect, rtol=1e-9)
    assert bins[0].sum() == pytest.approx(1.0 - tfin[0], abs=1e-12)


@pytest.mark.parametrize("pdf_kind", ["uniform", "one_bin", "two_bins"])
@pytest.mark.parametrize("nimp", [64, 100, 7])
def test_importance_constant_volume_closed_form(orc, pdf_kind, nimp):
    """In a constant medium (every brick occupied: the range starts at t_near)
    the nimp equal segments tile [t_near, t_b], so the composite is
    1 - (1 - a)^((t_b - t_near) / ds_ref) for any nimp (Eq. 3); the range ends
    one bin past saturation. Uniform PDF: the running sum reaches 1 - 1/64 only
    at bin 31, t_b = t_far. All mass on bin 7: t_b is the end of bin 8 (9 L/32).
    Mass 0.3 on bin 3, 0.7 on bin 20: 22 L/32."""
    V0, a = 2000, 0.03
    vol = np.full((8, 8, 60), V0, dtype=np.uint16)
    tf = identity_tf({V0: (0.2, 0.4, 0.8, a)})
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=1.0)
    g = orc.ray_geometry(sc, 0, 0)
    L = g["tf"] - g["tn"]
    pdf = np.zeros(32)
    if pdf_kind == "uniform":
        pdf[:], cover = 1 / 32, L
    elif pdf_kind == "one_bin":
        pdf[7], cover = 1.0, 9 * L / 32
    else:
        pdf[3], pdf[20], cover = 0.3, 0.7, 22 * L / 32
    r = orc.importance(sc, pdf[None, :], nimp=nimp)
    rgba, ns = r["rgba"], r["nsamp"]
    expect = 1.0 - (1.0 - float(np.float32(a))) ** cover
    assert ns[0] == nimp
    assert rgba[0, 3] == pytest.approx(expect, abs=2e-6)
    np.testing.assert_allclose(rgba[0, :3], np.float32([0.2, 0.4, 0.8]) * rgba[0, 3], atol=1e-12)


def test_importance_range_starts_at_first_occupied_bin(orc):
    """Tissue in two slabs along the ray; a PDF that saturates early ends the
    range right after the near slab, so the far slab is not sampled: removing
    it changes nothing. A PDF that saturates only at the end samples both. The
    empty stretch before the near slab is never sampled."""
    vol = np.zeros((8, 8, 64), dtype=np.uint16)
    vol[:, :, 40:48] = 2000                                  # near slab (the ray runs from x = 63 down)
    vol[:, :, :8] = 2000                                     # far slab
    near_only = vol.copy()
    near_only[:, :, :8] = 0
    tf = identity_tf({2000: (1.0, 1.0, 1.0, 0.1)})
    cam = axis_camera(64, 3.0, 3.0)
    early = np.zeros(32); early[11] = 1.0                   # range ends after bin 12 (x about 38)
    late = np.full(32, 1 / 32)
    a = orc.importance(orc.Scene(vol, (1, 1, 1), tf, cam, term=1.0), early[None, :])["rgba"]
    b = orc.importance(orc.Scene(near_only, (1, 1, 1), tf, cam, term=1.0), early[None, :])["rgba"]
    c = orc.importance(orc.Scene(vol, (1, 1, 1), tf, cam, term=1.0), late[None, :])["rgba"]
    assert a[0, 3] > 0.3 and a[0, 3] == b[0, 3]
    assert c[0, 3] > a[0, 3] + 0.1
    # 8 voxels of opacity 0.1 per voxel: the composite approaches 1 - 0.9^8
    assert a[0, 3] == pytest.approx(1 - 0.9 ** 8, abs=0.06)


def test_importance_uniform_pdf_is_midpoint_march(orc):
    """In a medium with every brick occupied, a uniform PDF puts sample j at
    the centre of the j-th of nimp equal segments of the chord: the same
    samples as the 512-segment profile march."""
    rng = np.random.default_rng(9)
    vol = rng.integers(1000, 3200, size=(30, 40, 40)).astype(np.uint16)
    tf = synth.tf_table(256)
    cam = synth.orbit_camera((40, 40, 30), (1, 1, 1), 0.0, width=8, height=8)
    sc = orc.Scene(vol, (1, 1, 1), tf, cam, term=1.0)
    pdf = np.full((64, 32), 1 / 32)
    r = orc.importance(sc, pdf, nimp=512)
    rgba, tfin, ns = r["rgba"], r["tfinal"], r["nsamp"]
    bins, tprof = orc.profiles(sc)
    hit = ns > 0
    assert hit.sum() > 10
    np.testing.assert_allclose(tfin, tprof, atol=1e-12)
    np.testing.assert_allclose(rgba[:, 3], bins.sum(axis=1), atol=1e-12)


# --------------------------------------------------------------------------
# the inverse-CDF reading of the importance samples
# --------------------------------------------------------------------------
def mixture_cdf(pdf, lam, s):
    """CDF at s in [0, 32] (bin units) of the piecewise-constant density
    (1 - lam) pdf + lam / 32, normalised to 1 (FP64)."""
    q = (1 - lam) * np.asarray(pdf, np.float64) + lam / 32
    Q = np.concatenate([[0.0], np.cumsum(q)])
    b = np.minimum(np.floor(s).astype(int), 31)
    return (Q[b] + (s - b) * q[b]) / Q[-1]


@pytest.mark.parametrize("lam", [0.0, 0.05, 0.5])
def test_invcdf_samples_are_stratified(orc, lam):
    """Sample j sits where the mixture's CDF reaches (j + 0.5) / nimp (one
    sample per stratum), and the segments between the midpoints of
    neighbouring samples tile the chord [t_near, t_far]."""
    vol = np.full((8, 8, 60), 2000, dtype=np.uint16)
    tf = identity_tf({2000: (1.0, 1.0, 1.0, 0.05)})
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=1.0)
    g = orc.ray_geometry(sc, 0, 0)
    L = g["tf"] - g["tn"]
    rng = np.random.default_rng(4)
    pdf = rng.random(32) ** 4
    pdf[[2, 9, 10, 30]] = 0.0
    pdf /= pdf.sum()
    for nimp in (1, 7, 64):
        t, ln = orc.importance_positions(sc, 0, 0, pdf, nimp=nimp, sampling="invcdf", lam=lam)
        s = (t - g["tn"]) / (L / 32)
        np.testing.assert_allclose(mixture_cdf(pdf, lam, s), (np.arange(nimp) + 0.5) / nimp, atol=2e-6)
        assert np.all(np.diff(t) >= 0)
        mid = np.concatenate([[g["tn"]], (t[1:] + t[:-1]) / 2, [g["tf"]]])
        np.testing.assert_allclose(ln, np.diff(mid), atol=2e-5)     # FP32 rounding at t ~ 60 mm
        assert ln.sum() == pytest.approx(L, abs=1e-4)


def test_invcdf_hand_worked_positions(orc):
    """lambda = 0, mass 0.3 in bin 3 and 0.7 in bin 20, 10 samples: u = 0.05,
    0.15, 0.25 fall in bin 3 at fractions 1/6, 1/2, 5/6; u = 0.35 .. 0.95 in
    bin 20 at fractions (u - 0.3) / 0.7. lambda = 1 puts sample j at the centre
    of the j-th of nimp equal segments of the chord."""
    vol = np.full((8, 8, 60), 2000, dtype=np.uint16)
    tf = identity_tf({2000: (1.0, 1.0, 1.0, 0.05)})
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=1.0)
    g = orc.ray_geometry(sc, 0, 0)
    bw = (g["tf"] - g["tn"]) / 32
    pdf = np.zeros(32)
    pdf[3], pdf[20] = 0.3, 0.7
    t, _ = orc.importance_positions(sc, 0, 0, pdf, nimp=10, sampling="invcdf", lam=0.0)
    u = (np.arange(10) + 0.5) / 10
    pos = np.where(u < 0.3, 3 + u / 0.3, 20 + (u - 0.3) / 0.7)
    np.testing.assert_allclose(t, g["tn"] + pos * bw, atol=2e-5)
    t1, ln1 = orc.importance_positions(sc, 0, 0, None, nimp=5, sampling="invcdf", lam=1.0)
    L = g["tf"] - g["tn"]
    np.testing.assert_allclose(t1, g["tn"] + (np.arange(5) + 0.5) * L / 5, atol=2e-5)
    np.testing.assert_allclose(ln1, L / 5, atol=2e-5)


@pytest.mark.parametrize("lam", [0.05, 1.0])
@pytest.mark.parametrize("nimp", [64, 9])
def test_invcdf_constant_volume_closed_form(orc, lam, nimp):
    """In a constant medium the midpoint segments tile the whole chord, so for
    any PDF the composite is 1 - (1 - a)^(L / ds_ref) with L = t_far - t_near
    (Eq. 3 per segment, the segment lengths summing to L)."""
    V0, a = 2000, 0.03
    vol = np.full((8, 8, 60), V0, dtype=np.uint16)
    tf = identity_tf({V0: (0.2, 0.4, 0.8, a)})
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=1.0)
    g = orc.ray_geometry(sc, 0, 0)
    pdf = np.zeros(32)
    pdf[3], pdf[20] = 0.3, 0.7
    r = orc.importance(sc, pdf[None, :], nimp=nimp, sampling="invcdf", lam=lam)
    expect = 1.0 - (1.0 - float(np.float32(a))) ** (g["tf"] - g["tn"])
    assert r["nsamp"][0] == nimp
    assert r["rgba"][0, 3] == pytest.approx(expect, abs=2e-5)
    np.testing.assert_allclose(r["rgba"][0, :3], np.float32([0.2, 0.4, 0.8]) * r["rgba"][0, 3], atol=1e-12)


@pytest.mark.parametrize("sampling", ["range", "invcdf"])
def test_importance_termination_tie_gives_both_branches(orc, sampling):
    """With term set to the opacity the march reaches at its m-th sample, the
    stop decision there is a tie: the oracle flags it and returns both
    branches, the composites of m and m + 1 samples of the constant medium
    (Eq. 4 stopped either side of the threshold)."""
    V0, a = 2000, 0.03
    vol = np.full((8, 8, 60), V0, dtype=np.uint16)
    tf = identity_tf({V0: (0.2, 0.4, 0.8, a)})
    pdf = np.full((1, 32), 1 / 32)
    base = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=1.0)
    nimp, m = 64, 23
    t, ln = orc.importance_positions(base, 0, 0, pdf, nimp=nimp, sampling=sampling, lam=1.0)
    ap = 1.0 - (1.0 - float(np.float32(a))) ** (ln / 1.0)
    T = np.cumprod(1.0 - ap)
    term = float(np.float32(1.0 - T[m - 1]))
    sc = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=term)
    r = orc.importance(sc, pdf, nimp=nimp, sampling=sampling, lam=1.0)
    assert r["tie"][0]
    got = sorted([r["rgba"][0, 3], r["alt"][0, 3]])
    np.testing.assert_allclose(got, [1.0 - T[m - 1], 1.0 - T[m]], atol=1e-9)
    far = orc.Scene(vol, (1, 1, 1), tf, axis_camera(60, 3.0, 3.0), term=0.5 * term)
    assert not orc.importance(far, pdf, nimp=nimp, sampling=sampling, lam=1.0)["tie"][0]
