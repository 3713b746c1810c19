"""Pins of the oracle's cubic B-spline reconstruction and two-dimensional
(value x gradient magnitude) classification against closed forms.

The cubic B-spline (the higher-order filter of Sec. 3.2) reproduces
polynomials up to degree one exactly and shifts higher moments by known
amounts: sum_i i^2 beta(x - i) = x^2 + 1/3 and sum_i i^3 beta(x - i) = x^3 + x.
Border voxels are replicated, which gives a closed form on the first cell.
The 2-D table (the scalar / gradient-magnitude classification of Sec. 3.1) is
pinned by a table that is affine in (i, j), which bilinear interpolation
reproduces exactly, on ramp volumes whose gradient is known.
"""
import numpy as np
import pytest

import synth


def ramp_volume(dims, coef, d0):
    """V(x, y, z) = a x + b y + c z + d0 (integer codes)."""
    nx, ny, nz = dims
    a, b, c = coef
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = a * x + b * y + c * z + d0
    assert v.min() >= 0 and v.max() <= 4095
    return v.astype(np.uint16)


def samples_of(orc, sc, pixels):
    out = []
    for (x, y) in pixels:
        s = orc.ray_samples(sc, x, y)
        if len(s["v"]):
            out.append(s)
    assert out, "no ray hit the volume"
    return {k: np.concatenate([s[k] for s in out]) for k in out[0]}


def interior(s, dims, lo, hi_off):
    """Samples whose position lies in [lo, n - hi_off) on every axis."""
    m = np.ones(len(s["v"]), dtype=bool)
    for a, key in enumerate(("px", "py", "pz")):
        m &= (s[key] >= lo) & (s[key] < dims[a] - hi_off)
    return m


PIXELS = [(x, y) for x in (5, 11, 16, 20, 26) for y in (6, 13, 19, 25)]
GRID = [(x, y) for x in range(1, 32, 3) for y in range(1, 32, 3)]


# --------------------------------------------------------------------------
# cubic B-spline reconstruction
# --------------------------------------------------------------------------
def test_bspline_partition_of_unity(orc):
    vol = np.full((20, 24, 28), 1234, dtype=np.uint16)
    cam = synth.orbit_camera((28, 24, 20), (1.0, 1.5, 2.0), 35.0, width=32, height=32)
    sc = orc.Scene(vol, (1.0, 1.5, 2.0), synth.tf_table(256), cam, shade=True, filter=orc.BSPLINE)
    s = samples_of(orc, sc, PIXELS)
    np.testing.assert_allclose(s["v"], 1234.0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(s["gm"], 0.0, rtol=0, atol=1e-9)


@pytest.mark.parametrize("spacing", [(1.0, 1.0, 1.0), (0.8, 1.1, 2.5)])
def test_bspline_reproduces_affine_fields(orc, spacing):
    """Value a x + b y + c z + d and world gradient (a/sx, b/sy, c/sz) wherever
    the 4^3 footprint stays inside the volume (1 <= p < n - 2 per axis)."""
    dims = (30, 26, 22)
    coef = (37, -21, 53)
    d0 = 21 * 25 + 50
    vol = ramp_volume(dims, coef, d0)
    cam = synth.orbit_camera(dims, spacing, 25.0, width=32, height=32)
    sc = orc.Scene(vol, spacing, synth.tf_table(256), cam, shade=True, filter=orc.BSPLINE, term=1.0)
    s = samples_of(orc, sc, PIXELS)
    m = interior(s, dims, 1.0, 2.0)
    assert m.sum() > 100
    expect = coef[0] * s["px"] + coef[1] * s["py"] + coef[2] * s["pz"] + d0
    np.testing.assert_allclose(s["v"][m], expect[m], rtol=0, atol=1e-9)
    G = np.sqrt(sum((c / float(np.float32(sp))) ** 2 for c, sp in zip(coef, spacing)))   # spacing is FP32
    np.testing.assert_allclose(s["gm"][m], G, rtol=1e-12)


def axis_ray_camera(nx, yc, zc):
    return dict(eye=(float(nx - 1 + 40.0), float(yc), float(zc)), target=(0.0, float(yc), float(zc)),
                up=(0.0, 0.0, 1.0), fovy_deg=30.0, width=1, height=1)


@pytest.mark.parametrize("power,nx,closed,dclosed", [
    (2, 48, lambda x: x ** 2 + 1.0 / 3.0, lambda x: 2 * x),
    (3, 16, lambda x: x ** 3 + x, lambda x: 3 * x ** 2 + 1.0),
])
def test_bspline_moments(orc, power, nx, closed, dclosed):
    """V = x^2 and V = x^3 along one axis: the B-spline gives x^2 + 1/3 and
    x^3 + x (its second moment is 1/3, its odd moments vanish), with the
    analytic derivatives 2x and 3x^2 + 1 (per mm: divided by sx)."""
    sx = 1.25
    vol = np.zeros((6, 6, nx), dtype=np.uint16)
    vol[:] = (np.arange(nx) ** power).astype(np.uint16)
    sc = orc.Scene(vol, (sx, 1.0, 1.0), synth.tf_table(256), axis_ray_camera(nx * sx, 2.0, 3.0),
                   step=0.3, shade=True, filter=orc.BSPLINE, term=1.0)
    s = orc.ray_samples(sc, 0, 0)
    m = (s["px"] >= 1.0) & (s["px"] < nx - 2.0)
    assert m.sum() > 20
    x = s["px"][m]
    np.testing.assert_allclose(s["v"][m], closed(x), rtol=1e-13, atol=1e-10)
    np.testing.assert_allclose(s["gm"][m], np.abs(dclosed(x)) / sx, rtol=1e-12, atol=1e-10)


def test_bspline_border_replication(orc):
    """V = x: on the first cell the voxel at x = -1 is replaced by the border
    voxel (value 0 instead of -1), so f(x) = x + beta(x + 1) = x + (1 - x)^3/6;
    at the far end the voxel n stands in for value n - 1, so on the last cell
    f(x) = x - beta(x - n) = x - (1 - t)^3/6 with t = n - 1 - x."""
    nx = 24
    vol = np.zeros((5, 5, nx), dtype=np.uint16)
    vol[:] = np.arange(nx, dtype=np.uint16)
    sc = orc.Scene(vol, (1, 1, 1), synth.tf_table(256), axis_ray_camera(nx, 2.0, 2.0), step=0.1,
                   filter=orc.BSPLINE, term=1.0)
    s = orc.ray_samples(sc, 0, 0)
    x = s["px"]
    lo = x < 1.0
    hi = x > nx - 2.0
    assert lo.sum() > 3 and hi.sum() > 3
    np.testing.assert_allclose(s["v"][lo], x[lo] + (1 - x[lo]) ** 3 / 6, rtol=0, atol=1e-10)
    t = (nx - 1) - x[hi]
    np.testing.assert_allclose(s["v"][hi], x[hi] - (1 - t) ** 3 / 6, rtol=0, atol=1e-10)


def test_bspline_grid_and_skipping_are_sound(orc):
    """Every B-spline sample lies in [min, max] of its cell-brick's 19^3 apron
    footprint (the value is a convex combination of those voxels), samples in
    bricks the mask marks empty have opacity exactly 0, and the apron grid
    contains the 17^3 trilinear grid."""
    ph = synth.head_phantom((70, 52, 40), (1.0, 1.0, 1.4), seed=11, tumor_radius_vox=5)
    mn0, mx0 = orc.brick_minmax(ph.vol, filter=orc.TRILINEAR)
    mn1, mx1 = orc.brick_minmax(ph.vol, filter=orc.BSPLINE)
    assert (mn1 <= mn0).all() and (mx1 >= mx0).all() and ((mn1 < mn0) | (mx1 > mx0)).any()
    tf = synth.tf_table(256)
    occ = orc.occupancy(ph.dims, tf, mn1, mx1)
    assert 0 < occ.sum() < occ.size
    cam = synth.orbit_camera(ph.dims, ph.spacing, 70.0, width=32, height=32)
    sc = orc.Scene(ph.vol, ph.spacing, tf, cam, filter=orc.BSPLINE, term=1.0)
    s = samples_of(orc, sc, GRID)
    p = np.stack([s["px"], s["py"], s["pz"]], 1)
    dims = np.array(ph.dims)
    base = np.minimum(np.floor(np.clip(p, 0, dims - 1)), dims - 2).astype(int)
    b = base // 16
    bmn = mn1[b[:, 2], b[:, 1], b[:, 0]].astype(float)
    bmx = mx1[b[:, 2], b[:, 1], b[:, 0]].astype(float)
    assert (s["v"] >= bmn - 1e-9).all() and (s["v"] <= bmx + 1e-9).all()
    empty = occ[b[:, 2], b[:, 1], b[:, 0]] == 0
    assert empty.sum() > 50
    assert (s["a"][empty] == 0.0).all()


# --------------------------------------------------------------------------
# two-dimensional classification
# --------------------------------------------------------------------------
def affine_table(K, M, coef):
    """T(i, j)[c] = c0 + c1 i/(K-1) + c2 j/(M-1) per channel."""
    i = np.arange(K)[None, :] / (K - 1)
    j = np.arange(M)[:, None] / (M - 1)
    tab = np.zeros((M, K, 4))
    for c, (c0, c1, c2) in enumerate(coef):
        tab[..., c] = c0 + c1 * i + c2 * j
    assert tab.min() >= 0 and tab.max() <= 1
    return tab.astype(np.float32)


def table_value(tab_f32, K, M, v_over_vmax, g_over_gmax):
    """The affine table's function at (u, w), from its float32 corner entries:
    exact bilinear reproduction, so evaluate the plane through the corners."""
    t = tab_f32.astype(np.float64)
    c0 = t[0, 0]
    c1 = t[0, K - 1] - t[0, 0]
    c2 = t[M - 1, 0] - t[0, 0]
    return c0[None] + np.outer(v_over_vmax, c1) + np.outer(g_over_gmax, c2)


COEF = ((0.1, 0.5, 0.3), (0.05, 0.2, 0.7), (0.9, -0.6, -0.2), (0.01, 0.3, 0.15))


@pytest.mark.parametrize("gscale", [2.7, 0.4])
def test_tf2d_affine_table_on_a_ramp(orc, gscale):
    """Ramp volume, table affine in (i, j) with K != M: every interior sample's
    straight RGBA is the plane at (v/vmax, min(|g|/gmax, 1)). A transposed
    table, a swapped axis, a missing spacing or a wrong gradient scale moves
    the result off the plane. gscale < 1 clamps w to the last row."""
    dims = (30, 26, 22)
    spacing = (0.9, 1.2, 1.7)
    coef = (41, -17, 29)
    vol = ramp_volume(dims, coef, 17 * 25 + 100)
    K, M = 64, 8
    tab = affine_table(K, M, COEF)
    G = np.sqrt(sum((c / float(np.float32(sp))) ** 2 for c, sp in zip(coef, spacing)))   # spacing is FP32
    gmax = float(np.float32(gscale * G))
    cam = synth.orbit_camera(dims, spacing, 15.0, width=32, height=32)
    sc = orc.Scene(vol, spacing, tab, cam, term=1.0, gmax=gmax)
    s = samples_of(orc, sc, PIXELS)
    m = interior(s, dims, 1.0, 2.0)       # central differences stay inside
    assert m.sum() > 100
    np.testing.assert_allclose(s["gm"][m], G, rtol=1e-12)
    np.testing.assert_allclose(s["gw"][m], G * (M - 1) / gmax, rtol=1e-12)
    want = table_value(tab, K, M, s["v"][m] / 4095.0, np.full(m.sum(), min(G / gmax, 1.0)))
    got = np.stack([s["r"], s["g"], s["b"], s["a"]], 1)[m]
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-7)   # table entries are float32


def test_tf2d_equal_rows_equals_1d(orc):
    """A 2-D table whose rows are all the 1-D table renders exactly the 1-D image."""
    ph = synth.head_phantom((48, 40, 32), (1.0, 1.0, 1.5), seed=21, tumor_radius_vox=4)
    tf1 = synth.tf_table(256)
    tf2 = np.repeat(tf1[None], 5, axis=0)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 50.0, width=24, height=20)
    for shade in (False, True):
        for filt in (orc.TRILINEAR, orc.BSPLINE):
            a = orc.render(orc.Scene(ph.vol, ph.spacing, tf1, cam, shade=shade, filter=filt))["rgba"]
            b = orc.render(orc.Scene(ph.vol, ph.spacing, tf2, cam, shade=shade, filter=filt,
                                     gmax=500.0))["rgba"]
            np.testing.assert_allclose(b, a, rtol=0, atol=1e-13)


def test_tf2d_normalised_values_use_code_units(orc):
    """FP16 storage (values (code - o) / o, o = 2048 for vmax 4096) classifies
    with the gradient in code units: every code up to 4096 is exact in that
    form, so every sample (odd codes included) matches the raw-code scene."""
    dims = (30, 26, 22)
    vol = ramp_volume(dims, (40, -16, 28), 16 * 25 + 101)
    assert (vol & 1).any()
    tab = affine_table(64, 8, COEF)
    cam = synth.orbit_camera(dims, (1, 1, 1), 15.0, width=32, height=32)
    raw = orc.Scene(vol, (1, 1, 1), tab, cam, term=1.0, gmax=60.0, vmax=4096)
    nrm = orc.Scene(vol, (1, 1, 1), tab, cam, term=1.0, gmax=60.0, vmax=4096, value_mode=1)
    sr = samples_of(orc, raw, PIXELS)
    sn = samples_of(orc, nrm, PIXELS)
    np.testing.assert_array_equal(sn["v"], sr["v"])
    np.testing.assert_array_equal(sn["gw"], sr["gw"])
    np.testing.assert_array_equal(sn["a"], sr["a"])


def test_fp16_offset_form_is_exact_for_12_bit_codes(orc):
    """The FP16 storage form holds every 12-bit code exactly: (c - 2048) / 2048
    is an integer of magnitude <= 2048 over a power of two, and numpy's own
    FP16 rounding round-trips it for all 4096 codes (an FP16 of c / 4095 does
    not: codes above 2048 keep only 11 significant bits). So the oracle's
    diagnostic FP16 scene renders the raw-code image exactly, on a shaded
    phantom with a 12-bit table, and the occupancy mask of the stored form
    equals the raw one."""
    c = np.arange(4096, dtype=np.float64)
    h = ((c - 2048.0) / 2048.0).astype(np.float16)
    np.testing.assert_array_equal((h.astype(np.float64) + 1.0) * 2048.0, c)
    old = (c / 4095.0).astype(np.float16).astype(np.float64) * 4095.0
    assert np.abs(old - c).max() > 0.4
    ph = synth.head_phantom((40, 36, 30), (1.0, 1.1, 1.3), seed=17, tumor_radius_vox=4)
    tf = synth.tf_table(1024)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 35.0, width=40, height=36)
    a = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.25, shade=True))
    b = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.25, shade=True, value_mode=1))
    assert a["rgba"][..., 3].max() > 0.3
    np.testing.assert_array_equal(a["rgba"], b["rgba"])
    mn, mx = orc.brick_minmax(ph.vol)
    np.testing.assert_array_equal(orc.occupancy(ph.dims, tf, mn, mx, value_mode=1),
                                  orc.occupancy(ph.dims, tf, mn, mx))


def test_tf2d_occupancy_is_sound(orc):
    """With a 2-D table a brick is empty only when every row of its value
    entries has zero opacity: a table whose low-gradient row is transparent
    below 3500 (but whose other rows are not) must mark more bricks occupied
    than that row alone, and every sample in an empty brick has opacity 0."""
    ph = synth.head_phantom((70, 52, 40), (1.0, 1.0, 1.4), seed=12, tumor_radius_vox=5)
    tab = synth.tf2d_table(256, 16)
    lowrow = tab[0].copy()
    lowrow[: int(3500 / 4095 * 255), 3] = 0.0
    tab[0] = lowrow
    mn, mx = orc.brick_minmax(ph.vol)
    occ2 = orc.occupancy(ph.dims, tab, mn, mx)
    occ_row = orc.occupancy(ph.dims, lowrow, mn, mx)
    assert (occ2 >= occ_row).all() and (occ2 > occ_row).any()
    assert 0 < occ2.sum() < occ2.size
    cam = synth.orbit_camera(ph.dims, ph.spacing, 110.0, width=32, height=32)
    sc = orc.Scene(ph.vol, ph.spacing, tab, cam, term=1.0, gmax=1200.0)
    s = samples_of(orc, sc, GRID)
    p = np.stack([s["px"], s["py"], s["pz"]], 1)
    dims = np.array(ph.dims)
    b = np.minimum(np.floor(np.clip(p, 0, dims - 1)), dims - 2).astype(int) // 16
    empty = occ2[b[:, 2], b[:, 1], b[:, 0]] == 0
    assert empty.sum() > 50
    assert (s["a"][empty] == 0.0).all()
    assert (s["a"][~empty] > 0).any()


def test_tf2d_rejected_where_undefined(orc):
    """Thresholding is defined for 1-D tables only."""
    vol = np.full((8, 8, 8), 1000, dtype=np.uint16)
    cam = synth.orbit_camera((8, 8, 8), (1, 1, 1), 0.0, width=4, height=4)
    sc = orc.Scene(vol, (1, 1, 1), synth.tf2d_table(16, 4), cam, func=orc.THRESHOLD, iso=500, gmax=100.0)
    with pytest.raises(ValueError):
        orc.render(sc)


@pytest.mark.parametrize("shade", [False, True])
def test_tf2d_gradient_matches_finite_differences(orc, shade):
    """The table gradient of a 2-D table (each sample scatters into the four
    entries of its bilinear cell) against central differences of the render,
    on the entries the rays use most and on unused ones (gradient 0)."""
    ph = synth.head_phantom((30, 28, 22), (1, 1, 1.2), seed=37, tumor_radius_vox=4)
    tab = synth.tf2d_table(64, 8, 1200.0)
    tab = (0.05 + 0.9 * tab).astype(np.float32)           # entries strictly inside (0, 1)
    tab[..., 3] *= 0.3
    cam = synth.orbit_camera(ph.dims, ph.spacing, 40.0, width=14, height=12)
    dimg = np.random.default_rng(5).normal(size=(14 * 12, 4))

    def loss(t):
        sc = orc.Scene(ph.vol, ph.spacing, t, cam, term=1.0, shade=shade, gmax=1200.0)
        return float((orc.render(sc)["rgba"].reshape(-1, 4) * dimg).sum())

    sc = orc.Scene(ph.vol, ph.spacing, tab, cam, term=1.0, shade=shade, gmax=1200.0)
    dtf, _ = orc.render_grad(sc, dimg)
    assert dtf.shape == (8, 64, 4)
    flat = np.abs(dtf).sum(axis=2).ravel()
    used = [divmod(int(e), 64) for e in np.argsort(-flat)[:5]]
    unused = [divmod(int(e), 64) for e in np.nonzero(flat == 0)[0][:2]]
    assert len(unused) == 2
    h = 1e-3
    checked = 0
    for (j, i) in used + unused:
        for c in range(4):
            tp = tab.astype(np.float64).copy(); tp[j, i, c] += h
            tm = tab.astype(np.float64).copy(); tm[j, i, c] -= h
            fd = (loss(tp.astype(np.float32)) - loss(tm.astype(np.float32))) / (
                float(np.float32(tp[j, i, c])) - float(np.float32(tm[j, i, c])))
            assert dtf[j, i, c] == pytest.approx(fd, rel=2e-3, abs=1e-6)
            checked += 1
    assert checked == 28
