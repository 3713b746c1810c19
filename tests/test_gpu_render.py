"""GPU parity of the forward path (FP32 storage) against the FP64 oracle.

Brick grid and occupancy mask: bit-exact. Images: max-abs <= 2e-4 per RGBA
channel, element by element on small cases (several tiles and a ragged tail)
and on seeded sampled pixels at the full 1024^2 / 256x256x180 workload, in the
launch configuration the bench times.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import TOL_FP32, GPURenderer, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc
    return rc


@pytest.fixture(scope="module")
def c1(rc):
    w = synth.WORKLOADS["plain_64x64x32"]
    ph = synth.workload_phantom("plain_64x64x32")
    r = GPURenderer(rc, ph.vol, ph.spacing)
    tf = synth.tf_table(w["K"])
    r.set_tf(tf)
    yield ph, tf, w, r
    r.close()


@pytest.fixture(scope="module")
def c2(rc):
    w = synth.WORKLOADS["shaded_256x256x180"]
    ph = synth.workload_phantom("shaded_256x256x180")
    r = GPURenderer(rc, ph.vol, ph.spacing)
    tf = synth.tf_table(w["K"])
    r.set_tf(tf)
    yield ph, tf, w, r
    r.close()


# --------------------------------------------------------------------------
# brick grid and occupancy: bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims,spacing", [((64, 64, 32), (1, 1, 3)), ((37, 20, 19), (1, 2, 1)),
                                          ((2, 2, 2), (1, 1, 1)), ((17, 33, 49), (0.5, 1, 1)),
                                          ((256, 256, 180), (1, 1, 1))])
def test_brick_grid_bit_exact(rc, orc, dims, spacing):
    ph = synth.head_phantom(dims, spacing, seed=11, tumor_radius_vox=3)
    vol = ph.vol.copy()
    vol.flat[::97] = 5000           # codes above vmax clamp
    r = GPURenderer(rc, vol, spacing)
    try:
        mn, mx = r.grid()
        omn, omx = orc.brick_minmax(vol, vmax=4095)
        assert np.array_equal(mn, omn) and np.array_equal(mx, omx)
    finally:
        r.close()


@pytest.mark.parametrize("storage,tf_fp16,K", [(0, False, 256), (2, False, 1024), (1, True, 1024),
                                              (1, False, 256), (2, True, 256)])
def test_occupancy_bit_exact(rc, orc, storage, tf_fp16, K):
    ph = synth.head_phantom((96, 80, 64), (1, 1, 1), seed=12, tumor_radius_vox=4)
    r = GPURenderer(rc, ph.vol, ph.spacing, storage=storage)
    try:
        for tf in (synth.tf_table(K), synth.random_tf(K, 5, alpha_max=0.2)):
            tf = tf.copy()
            tf[K // 2:K // 2 + 3, 3] = 1e-9      # FP16 rounds these to zero
            r.set_tf(tf, fp16=tf_fp16)
            occ = r.occupancy()
            omn, omx = orc.brick_minmax(ph.vol)
            oocc = orc.occupancy(ph.dims, tf, omn, omx, value_mode=int(storage == 1), tf_fp16=tf_fp16)
            assert np.array_equal(occ, oocc)
            assert 0 < occ.sum() < occ.size
    finally:
        r.close()


# --------------------------------------------------------------------------
# the plain raycast of a 64x64x32 phantom (1 x 1 x 3 mm), 256^2, 3 views
# --------------------------------------------------------------------------
@pytest.mark.parametrize("az", [0.0, 120.0, 240.0])
def test_plain_64x64x32_parity(c1, orc, az):
    ph, tf, w, r = c1
    cam = synth.orbit_camera(ph.dims, ph.spacing, az, width=w["width"], height=w["height"])
    img = r.render(cam, step_vox=w["step"], term=w["term"], shade=False, skip=True)
    o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=w["step"], term=w["term"]))
    err, ties = compare(img, o, TOL_FP32)
    assert o["rgba"][..., 3].max() > 0.9


def test_dense_sample_counts_exact(c1, orc):
    ph, tf, w, r = c1
    cam = synth.orbit_camera(ph.dims, ph.spacing, 30.0, width=200, height=150)
    img, st = r.render(cam, stats=True, step_vox=0.5, term=1.0, skip=True)
    o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=1.0))
    # with term = 1, FP32 1 - T reaches 1.0 once T < 2^-25: those rays are
    # termination ties (either branch is correct); every other ray is exact
    lo = int(np.minimum(o["nsamp"], o["nsamp_alt"]).sum())
    hi = int(np.maximum(o["nsamp"], o["nsamp_alt"]).sum())
    assert lo <= st["dense_samples"] <= hi
    assert hi - lo < 0.01 * lo
    assert st["rays_hit"] == int((o["nsamp"] > 0).sum())
    assert st["rays_total"] == 200 * 150
    assert st["evaluated_samples"] <= st["dense_samples"]   # every brick of this head is occupied
    compare(img, o, TOL_FP32)


def test_stats_report_device_time(c1):
    """rc_stats.device_ms: the device time of the call's work from CUDA events
    on the context's stream: positive, within the call's wall time, and
    longer for a 1024^2 image than for a 64^2 one."""
    import time
    ph, tf, w, r = c1
    times = []
    for size in (64, 1024):
        cam = synth.orbit_camera(ph.dims, ph.spacing, 30.0, width=size, height=size)
        r.render(cam, stats=True, step_vox=0.25, term=0.99, shade=True, skip=True)      # warm
        t0 = time.perf_counter()
        _, st = r.render(cam, stats=True, step_vox=0.25, term=0.99, shade=True, skip=True)
        wall_ms = 1e3 * (time.perf_counter() - t0)
        assert 0.0 < st["device_ms"] <= wall_ms
        times.append(st["device_ms"])
    assert times[1] > times[0]


@pytest.mark.parametrize("shade", [False, True])
def test_skip_on_off_bit_identical(c1, shade):
    ph, tf, w, r = c1
    for az in (0.0, 77.0, 200.0):
        cam = synth.orbit_camera(ph.dims, ph.spacing, az, width=128, height=96)
        a = r.render(cam, step_vox=0.5, term=0.99, shade=shade, skip=True)
        b = r.render(cam, step_vox=0.5, term=0.99, shade=shade, skip=False)
        assert np.array_equal(a, b)


def test_ragged_and_anisotropic(rc, orc):
    ph = synth.head_phantom((45, 38, 23), (0.9, 1.1, 2.5), seed=17, tumor_radius_vox=3)
    tf = synth.tf_table(256)
    r = GPURenderer(rc, ph.vol, ph.spacing)
    try:
        r.set_tf(tf)
        for shade, step in ((False, 0.5), (True, 0.37)):
            cam = synth.orbit_camera(ph.dims, ph.spacing, 33.0, elevation_deg=-25.0, width=131, height=77)
            img = r.render(cam, step_vox=step, term=0.95, shade=shade, skip=True)
            o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=step, term=0.95, shade=shade))
            compare(img, o, TOL_FP32)
    finally:
        r.close()


def test_tiny_volume_and_single_pixel(rc, orc):
    vol = np.array([[[0, 4095], [2000, 1000]], [[3000, 2600], [500, 100]]], dtype=np.uint16)
    tf = synth.tf_table(256)
    r = GPURenderer(rc, vol, (1, 1, 1))
    try:
        r.set_tf(tf)
        for cam in (synth.orbit_camera((2, 2, 2), (1, 1, 1), 15.0, width=1, height=1),
                    synth.orbit_camera((2, 2, 2), (1, 1, 1), 95.0, width=33, height=17)):
            img = r.render(cam, step_vox=0.25, term=0.99, shade=True, skip=True)
            o = orc.render(orc.Scene(vol, (1, 1, 1), tf, cam, step=0.25, term=0.99, shade=True))
            compare(img, o, TOL_FP32)
    finally:
        r.close()


def test_eye_inside_and_axis_aligned_rays(rc, orc):
    """The eye at the volume centre (t_near clamps to 0, the first sample is
    inside the box) and cameras whose middle pixel's ray is parallel to an
    axis (zero direction components in the slab test), shaded and unshaded."""
    ph = synth.head_phantom((40, 36, 28), (1.0, 1.2, 1.5), seed=23, tumor_radius_vox=4)
    tf = synth.tf_table(256)
    E = (np.array(ph.dims) - 1) * np.array(ph.spacing)
    c = [float(np.float32(v / 2)) for v in E]
    cams = [dict(eye=tuple(c), target=(c[0] + 10.0, c[1], c[2]), up=(0.0, 0.0, 1.0), fovy_deg=60.0,
                 width=33, height=17),
            dict(eye=(c[0], c[1], c[2] + 100.0), target=tuple(c), up=(0.0, 1.0, 0.0), fovy_deg=30.0,
                 width=31, height=25)]
    r = GPURenderer(rc, ph.vol, ph.spacing)
    try:
        r.set_tf(tf)
        for cam in cams:
            for shade in (False, True):
                img = r.render(cam, step_vox=0.5, term=0.99, shade=shade, skip=True)
                o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=0.99, shade=shade))
                compare(img, o, TOL_FP32)
                assert np.array_equal(img, r.render(cam, step_vox=0.5, term=0.99, shade=shade, skip=False))
                assert img[..., 3].max() > 0.5
    finally:
        r.close()


@pytest.mark.parametrize("K", [2, 4096])
def test_table_size_limits(rc, orc, K):
    """The smallest table (2 entries: one linear ramp over the code range) and
    the largest (4096 entries, 64 KB of shared memory per block, above the
    default 48 KB): images against the oracle, skip on = off, occupancy
    bit-exact."""
    ph = synth.head_phantom((48, 44, 30), (1.0, 1.0, 1.5), seed=29, tumor_radius_vox=4)
    if K == 2:
        tf = np.array([[0.0, 0.0, 0.0, 0.0], [1.0, 0.7, 0.4, 0.05]], np.float32)
    else:
        tf = synth.tf_table(K)
    r = GPURenderer(rc, ph.vol, ph.spacing)
    try:
        r.set_tf(tf)
        cam = synth.orbit_camera(ph.dims, ph.spacing, 40.0, width=57, height=43)
        for shade in (False, True):
            img = r.render(cam, step_vox=0.5, term=0.99, shade=shade, skip=True)
            o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=0.99, shade=shade))
            compare(img, o, TOL_FP32)
            assert np.array_equal(img, r.render(cam, step_vox=0.5, term=0.99, shade=shade, skip=False))
            assert img[..., 3].max() > 0.3
        omn, omx = orc.brick_minmax(ph.vol)
        assert np.array_equal(r.occupancy(), orc.occupancy(ph.dims, tf, omn, omx))
    finally:
        r.close()


def test_tf_set_copies_the_host_table_and_keeps_order(rc, c1):
    """rc_tf_set from host memory copies the table during the call (the
    caller's array is overwritten right after each call here) without waiting
    for the queued renders, and stays ordered with them: renders queued with
    tables A, B, A (1-D) and then a 2-D table, without synchronising between
    them, each equal the same render done alone."""
    import torch
    ph, tf, w, r = c1
    cam = synth.orbit_camera(ph.dims, ph.spacing, 30.0, width=80, height=72)
    tab_b = synth.noise_tf(256, 77, alpha_max=0.3)
    tab2 = np.repeat(tab_b[None], 4, axis=0)
    tab2[..., 3] *= np.linspace(0.3, 1.0, 4, dtype=np.float32)[:, None]
    P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
    try:
        refs = []
        for t in (tf, tab_b, tf):
            r.set_tf(t)
            refs.append(r.render(cam, **P))
        rc.rc_tf2d_set(r.ctx, tab2, 900.0)
        refs.append(r.render(cam, **P))
        rc.rc_camera_set(r.ctx, cam)
        outs = [torch.empty((72, 80, 4), device="cuda") for _ in range(4)]
        buf = np.empty((256, 4), np.float32)
        buf2 = np.empty_like(tab2)
        for o, src in zip(outs[:3], (tf, tab_b, tf)):
            buf[:] = src
            rc.rc_tf_set(r.ctx, buf)
            buf[:] = 0.5                                 # the call has taken its copy
            rc.rc_render(r.ctx, r.vol, P, o)
        buf2[:] = tab2
        rc.rc_tf2d_set(r.ctx, buf2, 900.0)
        buf2[:] = 0.5
        rc.rc_render(r.ctx, r.vol, P, outs[3])
        torch.cuda.synchronize()
        for o, ref in zip(outs, refs):
            assert np.array_equal(o.cpu().numpy(), ref)
        assert not np.array_equal(refs[0], refs[1]) and not np.array_equal(refs[1], refs[3])
    finally:
        r.set_tf(tf)


def test_empty_transfer_function_renders_black(c1):
    ph, tf, w, r = c1
    try:
        r.set_tf(np.zeros((256, 4), np.float32))
        cam = synth.orbit_camera(ph.dims, ph.spacing, 10.0, width=64, height=64)
        img, st = r.render(cam, stats=True, step_vox=0.5, term=0.99, skip=True)
        assert np.all(img == 0) and st["evaluated_samples"] == 0 and st["dense_samples"] > 0
    finally:
        r.set_tf(tf)


# --------------------------------------------------------------------------
# the shaded raycast of a 256x256x180 phantom at 1024^2 (bench workload)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("az", [0.0, 10.0, 90.0, 250.0])
def test_shaded_256x256x180_sampled_parity(c2, orc, az):
    ph, tf, w, r = c2
    cam = synth.orbit_camera(ph.dims, ph.spacing, az, width=w["width"], height=w["height"])
    img = r.render(cam, step_vox=w["step"], term=w["term"], shade=True, skip=True)
    pix = synth.sample_pixels(w["width"], w["height"], 4096, seed=7000 + int(az))
    o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=w["step"], term=w["term"], shade=True),
                   pixels=pix)
    compare(img, o, TOL_FP32, pixels=pix)
    assert (o["nsamp"] > 0).sum() > 500


def test_shaded_small_full_image(rc, orc):
    ph = synth.head_phantom((96, 96, 72), (1, 1, 1), seed=2, tumor_radius_vox=6)
    tf = synth.tf_table(256)
    r = GPURenderer(rc, ph.vol, ph.spacing)
    try:
        r.set_tf(tf)
        cam = synth.orbit_camera(ph.dims, ph.spacing, 10.0, width=192, height=160)
        img = r.render(cam, step_vox=0.5, term=0.99, shade=True, skip=True)
        o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=0.99, shade=True))
        compare(img, o, TOL_FP32)
    finally:
        r.close()


# --------------------------------------------------------------------------
# the other ray functions of Sec. 4.1
# --------------------------------------------------------------------------
@pytest.mark.parametrize("func", ["MIP", "AVERAGE", "XRAY", "THRESHOLD", "ISO"])
def test_ray_functions(rc, orc, c1, func):
    ph, tf, w, r = c1
    cam = synth.orbit_camera(ph.dims, ph.spacing, 40.0, width=160, height=120)
    f = getattr(rc, "RC_FUNC_" + func)
    img = r.render(cam, step_vox=0.5, term=0.99, shade=False, func=f, iso=2500.0, skip=True)
    o = orc.render(orc.Scene(ph.vol, ph.spacing, tf, cam, step=0.5, term=0.99, func=f, iso=2500.0))
    g = img.reshape(-1, 4).astype(np.float64)
    a = o["rgba"].reshape(-1, 4)
    if func in ("MIP", "AVERAGE"):
        np.testing.assert_allclose(g, a, atol=2e-6)
    elif func == "XRAY":
        np.testing.assert_allclose(g, a, rtol=2e-5, atol=1e-6)
    else:
        # the first sample at or above iso: FP32 and FP64 may disagree on a
        # sample that lies within rounding of the iso-value; compare the rest
        same = (g[:, 3] == a[:, 3])
        if func == "ISO":
            same &= g[:, 2] == a[:, 2]
        assert same.mean() > 0.999
        if func == "ISO":
            np.testing.assert_allclose(g[same][:, 0], a[same][:, 0], rtol=1e-5, atol=1e-4)
            np.testing.assert_allclose(g[same][:, 1], a[same][:, 1], atol=2e-4)
        else:
            np.testing.assert_allclose(g[same], a[same], atol=2e-4)
        assert a[:, 3].sum() > 100


# --------------------------------------------------------------------------
# several views in one launch
# --------------------------------------------------------------------------
def test_render_views_equals_single_renders(rc, c1):
    import torch
    ph, tf, w, r = c1
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=96, height=72) for az in (0.0, 33.0, 200.0, 310.0)]
    P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
    out = torch.empty((4, 72, 96, 4), device="cuda")
    st = rc.rc_render_views(r.ctx, r.vol, P, cams, out, stats=True)
    torch.cuda.synchronize()
    dense = 0
    for v, cam in enumerate(cams):
        img, s1 = r.render(cam, stats=True, **P)
        assert np.array_equal(out[v].cpu().numpy(), img)
        dense += s1["dense_samples"]
    assert st["dense_samples"] == dense and st["rays_total"] == 4 * 96 * 72
    bad = [cams[0], synth.orbit_camera(ph.dims, ph.spacing, 10.0, width=95, height=72)]
    with pytest.raises(rc.RCError) as ei:
        rc.rc_render_views(r.ctx, r.vol, P, bad, out)
    assert ei.value.status == rc.RC_ERR_INVALID_ARG


@pytest.mark.parametrize("step", [0.5, 1.0, 0.37])
def test_brick_staged_march_equals_cached_march(rc, c2, monkeypatch, step):
    """The brick-staged variant of the shaded FP32 march (RC_MARCH_STAGED=1:
    each CTA copies the value+gradient brick its rays need next into shared
    memory with one bulk copy) renders the cached-gather march's images bit for
    bit, with the same sample counts, on ragged tiles of the full-size phantom
    and a small ragged volume, for each opacity-correction instance."""
    import torch
    ph, tf, w, r = c2
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=203, height=141) for az in (10.0, 130.0, 250.0)]
    P = dict(step_vox=step, term=0.99, shade=True, skip=True)
    a = torch.empty((3, 141, 203, 4), device="cuda")
    b = torch.empty_like(a)
    sa = rc.rc_render_views(r.ctx, r.vol, P, cams, a, stats=True)
    monkeypatch.setenv("RC_MARCH_STAGED", "1")
    sb = rc.rc_render_views(r.ctx, r.vol, P, cams, b, stats=True)
    rc.rc_context_sync(r.ctx)
    monkeypatch.delenv("RC_MARCH_STAGED")
    assert torch.equal(a, b)
    ta, tb = sa.pop("device_ms"), sb.pop("device_ms")
    assert sa == sb and sa["evaluated_samples"] > 0
    assert tb > ta > 0.0                                 # the staged march is the slower one
    small = synth.head_phantom((37, 29, 21), (1.0, 1.2, 0.9), seed=8, tumor_radius_vox=3)
    g = GPURenderer(rc, small.vol, small.spacing)
    try:
        g.set_tf(tf)
        cam = synth.orbit_camera(small.dims, small.spacing, 75.0, width=45, height=39)
        ref = g.render(cam, **P)
        monkeypatch.setenv("RC_MARCH_STAGED", "1")
        got = g.render(cam, **P)
        rc.rc_context_sync(g.ctx)
        monkeypatch.delenv("RC_MARCH_STAGED")
        assert np.array_equal(ref, got)
    finally:
        g.close()


def test_render_views_host_equals_device_render(rc, c1):
    """Host delivery: groups rendered into two device buffers in turn and
    copied on a second stream give the device render's images bit for bit,
    for page-locked and pageable host memory, one group, one view per group
    and a ragged last group; the statistics equal the one-launch render's."""
    import torch
    ph, tf, w, r = c1
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=96, height=72)
            for az in (0.0, 33.0, 120.0, 200.0, 310.0)]
    P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
    dev = torch.empty((5, 72, 96, 4), device="cuda")
    st = rc.rc_render_views(r.ctx, r.vol, P, cams, dev, stats=True)
    ref = dev.cpu()
    for pinned in (True, False):
        for group in (0, 1, 3, 7):
            host = torch.full((5, 72, 96, 4), -1.0)
            if pinned:
                host = host.pin_memory()
            sh = rc.rc_render_views_host(r.ctx, r.vol, P, cams, host, group=group, stats=group == 3)
            assert torch.equal(host, ref), (pinned, group)
            if group == 3:
                ms = sh.pop("device_ms")
                assert sh == {k: v for k, v in st.items() if k != "device_ms"}
                assert 0.0 < ms < 1e4
    # the device render is unchanged after the host path used the context
    rc.rc_render_views(r.ctx, r.vol, P, cams, dev)
    assert torch.equal(dev.cpu(), ref)
    with pytest.raises(rc.RCError) as ei:
        rc.rc_render_views_host(r.ctx, r.vol, P, cams, torch.empty((5, 72, 96, 4)), group=-1)
    assert ei.value.status == rc.RC_ERR_INVALID_ARG
    with pytest.raises(rc.RCError) as ei:                 # device memory is not a host buffer
        rc.rc_render_views_host(r.ctx, r.vol, P, cams, dev)
    assert ei.value.status == rc.RC_ERR_INVALID_ARG


@pytest.mark.parametrize("form", ["bspline", "mip", "tf2d"])
def test_render_views_host_other_forms(rc, form):
    """Host delivery with the other marches (B-spline filter, a non-composite
    ray function, the 2-D table): images equal the device render's."""
    import torch
    ctx = rc.rc_context_create(0)
    vol = None
    try:
        dims, sp = (60, 52, 40), (1.0, 1.0, 1.5)
        ph = synth.head_phantom(dims, sp, seed=41, tumor_radius_vox=4)
        vol = rc.rc_volume_create(ctx, dims, sp, 4095, rc.RC_STORE_F32)
        rc.rc_volume_upload(ctx, vol, ph.vol)
        P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
        if form == "tf2d":
            rc.rc_tf2d_set(ctx, synth.tf2d_table(256, 16, 1200.0), 1200.0)
        else:
            rc.rc_tf_set(ctx, synth.tf_table(256))
        if form == "bspline":
            P["filter"] = rc.RC_FILTER_BSPLINE
        if form == "mip":
            P["func"] = rc.RC_FUNC_MIP
        cams = [synth.orbit_camera(dims, sp, az, width=40, height=36) for az in (5.0, 95.0, 185.0)]
        dev = torch.empty((3, 36, 40, 4), device="cuda")
        rc.rc_render_views(ctx, vol, P, cams, dev)
        host = torch.full((3, 36, 40, 4), -1.0).pin_memory()
        rc.rc_render_views_host(ctx, vol, P, cams, host, group=2)
        assert torch.equal(host, dev.cpu())
        assert float(host[..., 3].max()) > 0.0
    finally:
        torch.cuda.synchronize()
        if vol is not None:
            rc.rc_volume_destroy(ctx, vol)
        rc.rc_context_destroy(ctx)


def test_render_batch_equals_views(rc):
    """Several volumes x several views in one launch: every image equals the
    multi-view render of its volume; mismatched volumes are refused."""
    import torch
    ctx = rc.rc_context_create(0)
    vols = []
    try:
        rc.rc_tf_set(ctx, synth.tf_table(256))
        dims, sp = (72, 60, 44), (1.0, 1.0, 1.5)
        for seed in (31, 32, 33):
            ph = synth.head_phantom(dims, sp, seed=seed, tumor_radius_vox=3 + seed % 4)
            v = rc.rc_volume_create(ctx, dims, sp, 4095, rc.RC_STORE_F32)
            rc.rc_volume_upload(ctx, v, ph.vol)
            vols.append(v)
        cams = [synth.orbit_camera(dims, sp, az, width=64, height=48) for az in (10.0, 100.0, 250.0, 333.0)]
        P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
        out = torch.empty((3, 4, 48, 64, 4), device="cuda")
        st = rc.rc_render_batch(ctx, vols, P, cams, out, stats=True)
        one = torch.empty((4, 48, 64, 4), device="cuda")
        dense = 0
        for i, v in enumerate(vols):
            s1 = rc.rc_render_views(ctx, v, P, cams, one, stats=True)
            torch.cuda.synchronize()
            assert torch.equal(out[i], one)
            dense += s1["dense_samples"]
        assert st["dense_samples"] == dense and st["rays_total"] == 3 * 4 * 48 * 64
        other = rc.rc_volume_create(ctx, (72, 60, 45), sp, 4095, rc.RC_STORE_F32)
        vols.append(other)
        rc.rc_volume_upload(ctx, other, np.zeros(72 * 60 * 45, np.uint16))
        with pytest.raises(rc.RCError) as ei:
            rc.rc_render_batch(ctx, vols, P, cams, torch.empty((4, 4, 48, 64, 4), device="cuda"))
        assert ei.value.status == rc.RC_ERR_INVALID_ARG
        with pytest.raises(rc.RCError) as ei:
            rc.rc_render_batch(ctx, vols[:3], dict(P, func=rc.RC_FUNC_MIP), cams, out)
        assert ei.value.status == rc.RC_ERR_UNSUPPORTED
    finally:
        torch.cuda.synchronize()
        for v in vols:
            rc.rc_volume_destroy(ctx, v)
        rc.rc_context_destroy(ctx)
