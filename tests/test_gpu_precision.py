"""Precision form: the 512x512x256 phantom stored as FP16 (offset-normalised,
(code - 2048) / 2048, exact for 12-bit codes) and as raw uint16, a 1024-entry
FP16 table, FP32 compositing, step 0.25, shaded, 2048^2 image. Checked against
the FP64 oracle on the original uint16 codes and the FP32 table (total error,
tolerance 4e-3) on 4096 seeded rays of the 2048^2 frame and on every pixel of
the full frame rendered at 512^2, and against the diagnostic oracle that uses
the same FP16-rounded volume and table (arithmetic error only, tolerance
2e-4)."""
import numpy as np
import pytest

import synth
from gpu_helpers import TOL_FP32, TOL_REDUCED, GPURenderer, compare

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["precision_512x512x256"]


@pytest.fixture(scope="module")
def rc():
    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc
    return rc


@pytest.fixture(scope="module")
def c3():
    ph = synth.workload_phantom("precision_512x512x256")
    return ph, synth.tf_table(W["K"])


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


@pytest.mark.parametrize("storage", ["F16", "U16"])
def test_precision_form(rc, orc, c3, storage):
    ph, tf = c3
    st = getattr(rc, "RC_STORE_" + storage)
    r = GPURenderer(rc, ph.vol, ph.spacing, storage=st)
    try:
        r.set_tf(tf, fp16=True)
        kw = dict(step=W["step"], term=W["term"], shade=True)
        # 4096 seeded rays of the 2048^2 frame
        cam = synth.orbit_camera(ph.dims, ph.spacing, 0.0, width=W["width"], height=W["height"])
        img = r.render(cam, step_vox=W["step"], term=W["term"], shade=True, skip=True)
        pix = synth.sample_pixels(W["width"], W["height"], W["n_rays"], seed=W["ray_seed"])
        total = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, **kw), pixels=pix)
        err_total, _ = compare(img, total, TOL_REDUCED, pixels=pix)
        diag = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, value_mode=int(storage == "F16"),
                                    tf_fp16=True, **kw), pixels=pix)
        err_diag, _ = compare(img, diag, TOL_FP32, pixels=pix)
        assert (total["nsamp"] > 0).sum() > 1000
        # the full frame at 512^2
        cs = synth.orbit_camera(ph.dims, ph.spacing, 0.0, width=W["small_width"], height=W["small_width"])
        small = r.render(cs, step_vox=W["step"], term=W["term"], shade=True, skip=True)
        diag_s = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cs, value_mode=int(storage == "F16"),
                                      tf_fp16=True, **kw))
        compare(small, diag_s, TOL_FP32)
        tot_s = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cs, **kw))
        # every pixel of the frame within the reduced-precision tolerance of the
        # FP64 oracle on the original codes and the FP32 table
        err_s, _ = compare(small, tot_s, TOL_REDUCED)
        print(f"{storage}: 4096 rays max-abs {err_total:.2e} (diagnostic {err_diag:.2e}); 512^2 max-abs "
              f"{err_s:.2e}, PSNR {psnr(small, tot_s['rgba']):.1f} dB")
    finally:
        r.close()


def test_fp32_storage_with_fp16_table_matches_diagnostic(rc, orc):
    """FP32 storage with the FP16 table: the only rounding is the table's."""
    ph = synth.head_phantom((128, 128, 96), (1, 1, 1), seed=3, tumor_radius_vox=6)
    tf = synth.tf_table(1024)
    r = GPURenderer(rc, ph.vol, ph.spacing)
    try:
        r.set_tf(tf, fp16=True)
        cam = synth.orbit_camera(ph.dims, ph.spacing, 60.0, width=160, height=128)
        img = r.render(cam, step_vox=0.25, term=0.99, shade=True, skip=True)
        o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.25, term=0.99, shade=True, tf_fp16=True))
        compare(img, o, TOL_FP32)
    finally:
        r.close()


@pytest.mark.parametrize("vmax,scale", [(4096, 1), (12000, 3)])
def test_f16_value_gradient_bricks_and_pairs(rc, orc, vmax, scale):
    """FP16 storage with vmax <= 4096 (offset o <= 2048, every stored value
    exact) reads shaded samples from its 8-byte value+gradient bricks (the
    stored FP16 value and the code differences); above, from pair bricks of
    the stored values (o = 8192 for vmax 12000: values rounded to FP16). Both
    match the FP64 oracle on the same stored values (diagnostic oracle, FP16
    table), shaded with a 1-D and a 2-D table and as isosurface, within 2e-4."""
    ph = synth.head_phantom((70, 58, 41), (1.0, 0.9, 1.3), seed=36, tumor_radius_vox=4)
    data = np.minimum(ph.vol.astype(np.int64) * scale, vmax).astype(np.uint16)
    # a table over the code range of this vmax: the default table's shape
    tf = synth.tf_table(256)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 140.0, width=75, height=53)
    r = GPURenderer(rc, data, ph.spacing, storage=rc.RC_STORE_F16, vmax=vmax)
    try:
        r.set_tf(tf, fp16=True)
        P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
        img = r.render(cam, **P)
        o = orc.render(orc.Scene(data, ph.spacing, tf, cam, step=0.5, term=0.99, shade=True, vmax=vmax,
                                 value_mode=1, tf_fp16=True))
        compare(img, o, TOL_FP32)
        assert o["rgba"][..., 3].max() > 0.3
        # isosurface: the hit sample (FP32 and FP64 may disagree on one within
        # rounding of the iso-value), its distance and its shading
        iso = float(0.4 * vmax)
        img = r.render(cam, step_vox=0.5, term=0.99, shade=True, skip=True, func=rc.RC_FUNC_ISO, iso=iso)
        o = orc.render(orc.Scene(data, ph.spacing, tf, cam, step=0.5, term=0.99, shade=True, vmax=vmax,
                                 value_mode=1, tf_fp16=True, func=orc.ISO, iso=iso))
        g, a = img.reshape(-1, 4).astype(np.float64), o["rgba"].reshape(-1, 4)
        same = (g[:, 3] == a[:, 3]) & (g[:, 2] == a[:, 2])
        assert same.mean() > 0.99 and a[:, 3].sum() > 100
        np.testing.assert_allclose(g[same][:, 0], a[same][:, 0], rtol=1e-5, atol=1e-4)
        np.testing.assert_allclose(g[same][:, 1], a[same][:, 1], atol=2e-4)
        gmax = 1200.0 * scale
        tab = synth.tf2d_table(256, 16, gmax)
        rc.rc_tf2d_set(r.ctx, tab, gmax, True)
        img = r.render(cam, **P)
        o = orc.render(orc.Scene(data, ph.spacing, tab, cam, step=0.5, term=0.99, shade=True, vmax=vmax,
                                 value_mode=1, tf_fp16=True, gmax=gmax))
        compare(img, o, TOL_FP32)
    finally:
        r.close()


def test_u16_value_gradient_bricks_equal_fp32_storage(rc, orc):
    """uint16 storage with vmax < 32768 reads the gradient from 8-byte
    value+gradient bricks holding the same integers as the FP32 storage's
    float4 bricks: shaded images (1-D and 2-D tables, isosurface) equal the
    FP32 storage's bit for bit. With vmax >= 32768 the differences do not fit
    16 bits and the apron path is used: it still matches the oracle."""
    ph = synth.head_phantom((70, 58, 41), (1.0, 0.9, 1.3), seed=35, tumor_radius_vox=4)
    tf = synth.tf_table(256)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 200.0, width=75, height=53)
    a = GPURenderer(rc, ph.vol, ph.spacing)
    b = GPURenderer(rc, ph.vol, ph.spacing, storage=rc.RC_STORE_U16)
    try:
        for r in (a, b):
            r.set_tf(tf)
        P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
        assert np.array_equal(a.render(cam, **P), b.render(cam, **P))
        # isosurface: the same hit sample and shading; the hit distance is a
        # division the compiler may schedule differently per storage instance
        iso = dict(step_vox=0.5, term=0.99, shade=True, skip=True, func=rc.RC_FUNC_ISO, iso=1500.0)
        ia, ib = a.render(cam, **iso), b.render(cam, **iso)
        assert np.array_equal(ia[..., 2:], ib[..., 2:])
        np.testing.assert_allclose(ib[..., :2], ia[..., :2], rtol=1e-6, atol=1e-6)
        tab = synth.tf2d_table(256, 16, 1200.0)
        for r in (a, b):
            rc.rc_tf2d_set(r.ctx, tab, 1200.0)
        P2 = dict(step_vox=0.5, term=0.99, shade=False, skip=True)
        assert np.array_equal(a.render(cam, **P2), b.render(cam, **P2))
    finally:
        a.close()
        b.close()
    # codes scaled to a 16-bit range: vmax 40000
    big = np.minimum((ph.vol.astype(np.int64) * 9), 40000).astype(np.uint16)
    c = GPURenderer(rc, big, ph.spacing, storage=rc.RC_STORE_U16, vmax=40000)
    try:
        c.set_tf(tf)
        img = c.render(cam, step_vox=0.5, term=0.99, shade=True, skip=True)
        o = orc.render(orc.Scene(big, ph.spacing, tf, cam, step=0.5, term=0.99, shade=True, vmax=40000))
        compare(img, o, TOL_FP32)
        assert o["rgba"][..., 3].max() > 0.3
    finally:
        c.close()
