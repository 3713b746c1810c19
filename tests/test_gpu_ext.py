"""GPU parity of the cubic B-spline reconstruction and the 2-D (value x
gradient magnitude) transfer function against the FP64 oracle.

Brick grids and occupancy masks: bit-exact. Images: max-abs <= 2e-4 per RGBA
channel element by element (ragged tiles, anisotropic spacing), skipping on
and off bit-identical, several views in one launch identical to single
renders, sampled pixels at the full 1024^2 / 256x256x180 workload, and the
forms the library does not support return RC_ERR_UNSUPPORTED.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import TOL_FP32, GPURenderer, compare

pytestmark = pytest.mark.gpu

GMAX = 1200.0


@pytest.fixture(scope="module")
def rc():
    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc
    return rc


def grid_filter(rc, r, filt):
    import torch
    bd = rc.rc_volume_brick_dims(r.vol)
    n = bd[0] * bd[1] * bd[2]
    mn = torch.empty(n, dtype=torch.int16, device="cuda")
    mx = torch.empty(n, dtype=torch.int16, device="cuda")
    rc.rc_brick_grid_get_filter(r.ctx, r.vol, filt, mn, mx)
    occ = torch.empty(n, dtype=torch.uint8, device="cuda")
    rc.rc_skip_mask_get_filter(r.ctx, r.vol, filt, occ)
    torch.cuda.synchronize()
    shp = (bd[2], bd[1], bd[0])
    return (mn.cpu().numpy().view(np.uint16).reshape(shp), mx.cpu().numpy().view(np.uint16).reshape(shp),
            occ.cpu().numpy().reshape(shp))


@pytest.fixture(scope="module")
def small(rc):
    ph = synth.head_phantom((90, 76, 52), (1.0, 1.0, 1.5), seed=31, tumor_radius_vox=5)
    r = GPURenderer(rc, ph.vol, ph.spacing)
    yield ph, r
    r.close()


# --------------------------------------------------------------------------
# grids and masks: bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(64, 64, 32), (37, 20, 19), (2, 2, 2), (17, 33, 49), (18, 18, 18)])
def test_bspline_grid_bit_exact(rc, orc, dims):
    ph = synth.head_phantom(dims, (1, 1, 1), seed=13, tumor_radius_vox=3)
    vol = ph.vol.copy()
    vol.flat[::89] = 4500          # codes above vmax clamp
    r = GPURenderer(rc, vol, (1, 1, 1))
    try:
        r.set_tf(synth.tf_table(256))
        for filt in (rc.RC_FILTER_TRILINEAR, rc.RC_FILTER_BSPLINE):
            mn, mx, occ = grid_filter(rc, r, filt)
            omn, omx = orc.brick_minmax(vol, vmax=4095, filter=filt)
            assert np.array_equal(mn, omn) and np.array_equal(mx, omx)
            assert np.array_equal(occ, orc.occupancy(ph.dims, synth.tf_table(256), omn, omx))
    finally:
        r.close()


@pytest.mark.parametrize("storage,fp16", [(0, False), (1, True), (2, False), (2, True)])
def test_tf2d_occupancy_bit_exact(rc, orc, storage, fp16):
    ph = synth.head_phantom((96, 80, 64), (1, 1, 1), seed=14, tumor_radius_vox=4)
    r = GPURenderer(rc, ph.vol, ph.spacing, storage=storage)
    try:
        tab = synth.tf2d_table(256, 16, GMAX)
        tab[0, : int(3500 / 4095 * 255), 3] = 0.0       # transparent low-gradient row
        tab[3, 128:131, 3] = 1e-9                        # FP16 rounds these to zero
        rc.rc_tf2d_set(r.ctx, tab, GMAX, fp16)
        for filt in (rc.RC_FILTER_TRILINEAR, rc.RC_FILTER_BSPLINE):
            _, _, occ = grid_filter(rc, r, filt)
            omn, omx = orc.brick_minmax(ph.vol, filter=filt)
            oocc = orc.occupancy(ph.dims, tab, omn, omx, value_mode=int(storage == 1), tf_fp16=fp16)
            assert np.array_equal(occ, oocc)
            assert 0 < occ.sum() < occ.size
    finally:
        r.close()


# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------
def test_bspline_after_new_data(rc, orc):
    """FP32 volumes read the B-spline footprint from pair bricks built on the
    first B-spline render; new data must rebuild them (against the oracle
    before and after the re-upload, F16 storage from the apron bricks alike)."""
    dims, sp = (50, 46, 34), (1.0, 1.1, 1.4)
    tf = synth.tf_table(256)
    cam = synth.orbit_camera(dims, sp, 61.0, width=45, height=39)
    P = dict(step_vox=0.5, term=0.99, shade=True, filter=rc.RC_FILTER_BSPLINE)
    for storage in (rc.RC_STORE_F32, rc.RC_STORE_F16):
        a = synth.head_phantom(dims, sp, seed=51, tumor_radius_vox=4)
        b = synth.head_phantom(dims, sp, seed=52, tumor_radius_vox=7)
        r = GPURenderer(rc, a.vol, sp, storage=storage)
        try:
            r.set_tf(tf)
            vm = int(storage == rc.RC_STORE_F16)
            for ph in (a, b):
                if ph is b:
                    rc.rc_volume_upload(r.ctx, r.vol, b.vol)
                img = r.render(cam, skip=True, **P)
                o = orc.render(orc.Scene(ph.vol, sp, tf, cam, step=0.5, term=0.99, shade=True,
                                         filter=orc.BSPLINE, value_mode=vm))
                compare(img, o, TOL_FP32)
                assert np.array_equal(img, r.render(cam, skip=False, **P))
        finally:
            r.close()


@pytest.mark.parametrize("shade", [False, True])
def test_bspline_parity(rc, orc, small, shade):
    ph, r = small
    tf = synth.tf_table(256)
    r.set_tf(tf)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 37.0, width=77, height=53)
    P = dict(step_vox=0.5, term=0.99, shade=shade, filter=rc.RC_FILTER_BSPLINE)
    img, st = r.render(cam, stats=True, skip=True, **P)
    assert np.array_equal(img, r.render(cam, skip=False, **P))
    assert st["evaluated_samples"] < st["dense_samples"]
    o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=0.99, shade=shade,
                             filter=orc.BSPLINE))
    compare(img, o, TOL_FP32)
    assert o["rgba"][..., 3].max() > 0.5
    # the filter changes the image (it smooths): not the trilinear result
    tri = r.render(cam, skip=True, step_vox=0.5, term=0.99, shade=shade)
    assert np.abs(tri - img).max() > 1e-2


@pytest.mark.parametrize("shade,filt", [(False, 0), (True, 0), (False, 1), (True, 1)])
def test_tf2d_parity(rc, orc, small, shade, filt):
    ph, r = small
    tab = synth.tf2d_table(256, 32, GMAX)
    rc.rc_tf2d_set(r.ctx, tab, GMAX)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 123.0, width=83, height=61)
    P = dict(step_vox=0.5, term=0.99, shade=shade, filter=filt)
    img = r.render(cam, skip=True, **P)
    assert np.array_equal(img, r.render(cam, skip=False, **P))
    o = orc.render(orc.Scene(ph.vol, ph.spacing, tab, cam, step=0.5, term=0.99, shade=shade, filter=filt,
                             gmax=GMAX))
    compare(img, o, TOL_FP32)
    assert o["rgba"][..., 3].max() > 0.3
    # equal rows give the 1-D image exactly
    rc.rc_tf2d_set(r.ctx, np.repeat(synth.tf_table(256)[None], 4, axis=0), GMAX)
    img_rows = r.render(cam, skip=True, **P)
    r.set_tf(synth.tf_table(256))
    img_1d = r.render(cam, skip=True, **P)
    np.testing.assert_allclose(img_rows, img_1d, rtol=0, atol=2e-6)


@pytest.mark.parametrize("storage,fp16", [(1, True), (2, True), (2, False)])
def test_reduced_storage_forms(rc, orc, storage, fp16):
    """F16 / U16 storage with the B-spline and the 2-D table, against the
    oracle on the same stored values (FP16-normalised for F16) and table."""
    ph = synth.head_phantom((70, 64, 48), (1.0, 1.0, 1.25), seed=32, tumor_radius_vox=4)
    r = GPURenderer(rc, ph.vol, ph.spacing, storage=storage)
    try:
        cam = synth.orbit_camera(ph.dims, ph.spacing, 250.0, width=64, height=48)
        tab = synth.tf2d_table(256, 16, GMAX)
        rc.rc_tf2d_set(r.ctx, tab, GMAX, fp16)
        for filt in (0, 1):
            img = r.render(cam, skip=True, step_vox=0.5, term=0.99, shade=True, filter=filt)
            o = orc.render(orc.Scene(ph.vol, ph.spacing, tab, cam, step=0.5, term=0.99, shade=True,
                                     filter=filt, gmax=GMAX, value_mode=int(storage == 1), tf_fp16=fp16))
            compare(img, o, TOL_FP32)
        tf = synth.tf_table(256)
        r.set_tf(tf, fp16)
        img = r.render(cam, skip=True, step_vox=0.5, term=0.99, shade=True, filter=1)
        o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=0.99, shade=True, filter=1,
                                 value_mode=int(storage == 1), tf_fp16=fp16))
        compare(img, o, TOL_FP32)
    finally:
        r.close()


@pytest.mark.parametrize("storage,fp16,filt", [(1, True, 0), (2, True, 1), (2, False, 0)])
def test_reduced_storage_gradients(rc, orc, storage, fp16, filt):
    """The table gradient (2-D and 1-D tables) on F16 / U16 storage against
    the oracle's reverse mode on the same stored values and table, within
    2e-4 of the largest entry, on a ragged 66 x 45 image (partial tiles in
    both directions); pixels whose termination is a tie are left out."""
    import torch
    ph = synth.head_phantom((70, 64, 48), (1.0, 1.0, 1.25), seed=33, tumor_radius_vox=4)
    r = GPURenderer(rc, ph.vol, ph.spacing, storage=storage)
    try:
        cam = synth.orbit_camera(ph.dims, ph.spacing, 70.0, width=66, height=45)
        rc.rc_camera_set(r.ctx, cam)
        for tab in (synth.tf2d_table(256, 16, GMAX), synth.tf_table(256)):
            if tab.ndim == 3:
                rc.rc_tf2d_set(r.ctx, tab, GMAX, fp16)
            else:
                r.set_tf(tab, fp16)
            sc = orc.Scene(ph.vol, ph.spacing, tab, cam, step=0.5, term=0.99, shade=True, filter=filt,
                           gmax=GMAX, value_mode=int(storage == 1), tf_fp16=fp16)
            fwd = orc.render(sc)
            keep = np.nonzero(~fwd["tie"].reshape(-1))[0]
            g = np.zeros((45 * 66, 4))
            g[keep] = np.random.default_rng(34).normal(size=(len(keep), 4))
            og, _ = orc.render_grad(sc, g[keep], pixels=keep)
            dtf = torch.empty(tab.shape, device="cuda")
            rc.rc_render_backward(r.ctx, r.vol, dict(step_vox=0.5, term=0.99, shade=True, filter=filt),
                                  torch.from_numpy(g.astype(np.float32)).cuda(), dtf)
            torch.cuda.synchronize()
            got = dtf.cpu().numpy().astype(np.float64)
            scale = np.abs(og).max()
            assert scale > 0
            assert np.abs(got - og).max() / scale < 2e-4
    finally:
        r.close()


@pytest.mark.parametrize("func", ["MIP", "AVERAGE", "XRAY", "ISO", "THRESHOLD"])
def test_bspline_ray_functions(rc, orc, small, func):
    ph, r = small
    tf = synth.tf_table(256)
    r.set_tf(tf)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 300.0, width=96, height=72)
    f = getattr(rc, "RC_FUNC_" + func)
    img = r.render(cam, step_vox=0.5, term=0.99, func=f, iso=2500.0, skip=True, filter=1)
    o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=0.99, func=f, iso=2500.0,
                             filter=orc.BSPLINE))
    g = img.reshape(-1, 4).astype(np.float64)
    a = o["rgba"].reshape(-1, 4)
    if func in ("MIP", "AVERAGE"):
        np.testing.assert_allclose(g, a, atol=1e-5)
    elif func == "XRAY":
        np.testing.assert_allclose(g, a, rtol=2e-5, atol=1e-5)
    else:
        same = g[:, 3] == a[:, 3]
        if func == "ISO":
            same &= g[:, 2] == a[:, 2]
        assert same.mean() > 0.999
        if func == "ISO":
            np.testing.assert_allclose(g[same][:, 0], a[same][:, 0], rtol=1e-5, atol=1e-4)
            np.testing.assert_allclose(g[same][:, 1], a[same][:, 1], atol=2e-4)
        else:
            np.testing.assert_allclose(g[same], a[same], atol=2e-4)
        assert a[:, 3].sum() > 100


def test_views_equal_single_renders(rc, small):
    import torch
    ph, r = small
    rc.rc_tf2d_set(r.ctx, synth.tf2d_table(256, 32, GMAX), GMAX)
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=64, height=40) for az in (5.0, 95.0, 222.0)]
    for filt in (0, 1):
        P = dict(step_vox=0.5, term=0.99, shade=True, skip=True, filter=filt)
        out = torch.empty((3, 40, 64, 4), device="cuda")
        rc.rc_render_views(r.ctx, r.vol, P, cams, out)
        torch.cuda.synchronize()
        for v, cam in enumerate(cams):
            assert np.array_equal(out[v].cpu().numpy(), r.render(cam, **P))


def test_full_workload_sampled(rc, orc):
    """256x256x180 at 1024^2, B-spline + 2-D table, shaded: seeded pixels of
    the multi-view launch against the oracle."""
    import torch
    ph = synth.workload_phantom("shaded_256x256x180")
    r = GPURenderer(rc, ph.vol, ph.spacing)
    try:
        tab = synth.tf2d_table(256, 32, GMAX)
        rc.rc_tf2d_set(r.ctx, tab, GMAX)
        cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=1024, height=1024) for az in (10.0, 200.0)]
        P = dict(step_vox=0.5, term=0.99, shade=True, skip=True, filter=1)
        out = torch.empty((2, 1024, 1024, 4), device="cuda")
        rc.rc_render_views(r.ctx, r.vol, P, cams, out)
        torch.cuda.synchronize()
        img = out.cpu().numpy()
        for v, cam in enumerate(cams):
            pix = synth.sample_pixels(1024, 1024, 2048, seed=4100 + v)
            o = orc.render(orc.Scene(ph.vol, ph.spacing, tab, cam, step=0.5, term=0.99, shade=True,
                                     filter=orc.BSPLINE, gmax=GMAX), pixels=pix)
            compare(img[v], o, TOL_FP32, pixels=pix)
    finally:
        r.close()


def test_unsupported_forms(rc, small):
    """The learned proposal takes trilinear samples and 1-D tables;
    thresholding takes 1-D tables; the non-allocating table gradient takes
    at most 1024 entries (here 8 x 256)."""
    import torch
    ph, r = small
    cam = synth.orbit_camera(ph.dims, ph.spacing, 0.0, width=32, height=24)
    rc.rc_camera_set(r.ctx, cam)
    out = torch.empty((24, 32, 4), device="cuda")
    g = torch.ones((24, 32, 4), device="cuda")
    dtf = torch.empty((256, 4), device="cuda")
    r.set_tf(synth.tf_table(256))
    feat = torch.empty((24 * 32, 112), device="cuda")
    with pytest.raises(rc.RCError) as ei:
        rc.rc_proposal_features(r.ctx, r.vol, dict(filter=1), feat)
    assert ei.value.status == rc.RC_ERR_UNSUPPORTED
    rc.rc_tf2d_set(r.ctx, synth.tf2d_table(256, 8, GMAX), GMAX)
    dtf2 = torch.empty((8, 256, 4), device="cuda")
    for call in (lambda: rc.rc_render_backward_noalloc(r.ctx, r.vol, dict(), g, dtf2),
                 lambda: rc.rc_render(r.ctx, r.vol, dict(func=rc.RC_FUNC_THRESHOLD, iso=100.0), out),
                 lambda: rc.rc_proposal_features(r.ctx, r.vol, dict(), feat)):
        with pytest.raises(rc.RCError) as ei:
            call()
        assert ei.value.status == rc.RC_ERR_UNSUPPORTED
    with pytest.raises(rc.RCError) as ei:
        rc.rc_render(r.ctx, r.vol, dict(filter=2), out)
    assert ei.value.status == rc.RC_ERR_INVALID_ARG
    for bad in ((np.full((4, 8, 4), 0.5, np.float32), 0.0), (np.full((1, 8, 4), 0.5, np.float32), 10.0),
                (np.full((4, 8, 4), 1.5, np.float32), 10.0)):
        with pytest.raises(rc.RCError) as ei:
            rc.rc_tf2d_set(r.ctx, bad[0], bad[1])
        assert ei.value.status == rc.RC_ERR_INVALID_ARG
    # a rejected table leaves the current one in place
    rc.rc_render(r.ctx, r.vol, dict(), out)
    torch.cuda.synchronize()
    assert out[..., 3].max() > 0.1


def gapped_tf(K, seed):
    """Opacity in narrow bands separated by transparent gaps, so that many
    4^3 sub-blocks, octants and bricks are empty next to occupied ones."""
    tab = synth.noise_tf(K, seed, alpha_max=0.2)
    u = np.random.default_rng(seed).random(K)
    tab[u < 0.7, 3] = 0.0          # 70% of the entries transparent
    tab[: K // 10, 3] = 0.0         # background transparent
    return tab


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_hierarchical_skip_exact_on_adversarial_data(rc, storage):
    """Skipping over empty bricks, octants and 4^3 sub-blocks is exact: with
    a noise volume (values change at every voxel) and a table of narrow
    opaque bands, every form renders the same image with skipping on and
    off, and skips part of the samples."""
    rng = np.random.default_rng(7 + storage)
    dims = (70, 61, 45)
    vol = rng.integers(0, 4096, size=dims[::-1]).astype(np.uint16)
    vol[:, :, :30] //= 16                    # a low-valued (transparent) half
    r = GPURenderer(rc, vol, (1.0, 1.2, 0.9), storage=storage)
    try:
        cam = synth.orbit_camera(dims, (1.0, 1.2, 0.9), 33.0, width=64, height=56)
        for K, seed in ((256, 3), (1024, 4)):
            r.set_tf(gapped_tf(K, seed), fp16=storage == 1)
            for shade in (False, True):
                for filt in (0, 1):
                    P = dict(step_vox=0.37, term=0.995, shade=shade, filter=filt)
                    on, st = r.render(cam, stats=True, skip=True, **P)
                    off = r.render(cam, skip=False, **P)
                    assert np.array_equal(on, off), (K, shade, filt)
                    assert st["evaluated_samples"] < st["dense_samples"]
    finally:
        r.close()
