"""Differentiable form: the hand-written transfer-function adjoint on a
128x128x96 phantom, 8 views at 512^2, checked against the FP64 oracle gradient
and against central finite differences (h = 1e-3, FP64 oracle) on 32 table
entries; the gradient of a 2-D table; determinism; the autograd wrapper; and a
table fit that lowers the L2 loss against images rendered with a hidden seeded
table."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["diff_128x128x96"]


@pytest.fixture(scope="module")
def rc():
    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc
    return rc


@pytest.fixture(scope="module")
def c4(rc):
    import torch
    ph = synth.workload_phantom("diff_128x128x96")
    ctx = rc.rc_context_create(0)
    vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, rc.RC_STORE_F32)
    rc.rc_volume_upload(ctx, vol, ph.vol)
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=W["width"], height=W["height"])
            for az in W["azimuths"]]
    yield ph, ctx, vol, cams
    torch.cuda.synchronize()
    rc.rc_volume_destroy(ctx, vol)
    rc.rc_context_destroy(ctx)


def init_tf():
    return synth.noise_tf(W["K"], W["init_tf_seed"], alpha_max=0.1)


def hidden_tf():
    return synth.random_tf(W["K"], W["hidden_tf_seed"], alpha_max=0.1)


def gpu_grad(rc, ctx, vol, cam, tf, g, term, shade=False, filt=0, noalloc=False):
    import torch
    rc.rc_tf_set(ctx, tf)
    rc.rc_camera_set(ctx, cam)
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    dtf = torch.empty((tf.shape[0], 4), device="cuda", dtype=torch.float32)
    p = rc.RenderParams(step_vox=W["step"], term=term, shade=shade, skip=False, filter=filt)
    (rc.rc_render_backward_noalloc if noalloc else rc.rc_render_backward)(ctx, vol, p, gd, dtf)
    torch.cuda.synchronize()
    return dtf.cpu().numpy().astype(np.float64)


def seeded_upstream(seed, pixels, shape):
    """dL/dI non-zero only on the seeded pixels (so the oracle can follow)."""
    g = np.zeros((shape[0] * shape[1], 4))
    g[pixels] = np.random.default_rng(seed).normal(size=(len(pixels), 4))
    return g


@pytest.mark.parametrize("shade,term,bspline", [(False, 0.99, False), (False, 1.0, False), (True, 0.99, False),
                                                (False, 0.99, True), (True, 0.99, True)])
def test_gradient_matches_oracle(rc, orc, c4, shade, term, bspline):
    """Against the FP64 oracle's reverse mode, with trilinear or cubic
    B-spline reconstruction (the B-spline also through the entry point that
    allocates nothing; here the pair bricks exist, so both entry points read
    them; the apron path of a volume without pairs is covered in
    test_zz_no_alloc.py)."""
    ph, ctx, vol, cams = c4
    tf = init_tf()
    filt = rc.RC_FILTER_BSPLINE if bspline else rc.RC_FILTER_TRILINEAR
    total_g = np.zeros((W["K"], 4))
    total_o = np.zeros((W["K"], 4))
    for v, cam in enumerate(cams):
        pix = synth.sample_pixels(W["width"], W["height"], 4096, seed=400 + v)
        sc = orc.Scene(ph.vol, ph.spacing, tf, cam, step=W["step"], term=term, shade=shade,
                       filter=orc.BSPLINE if bspline else orc.TRILINEAR)
        fwd = orc.render(sc, pixels=pix)
        keep = pix[~fwd["tie"]]                    # termination ties: either branch is right
        g = seeded_upstream(50 + v, keep, (W["height"], W["width"]))
        total_g += gpu_grad(rc, ctx, vol, cam, tf, g, term, shade, filt, noalloc=bspline and v % 2 == 1)
        og, _ = orc.render_grad(sc, g[keep], pixels=keep)
        total_o += og
    scale = np.abs(total_o).max()
    err = np.abs(total_g - total_o).max() / scale
    assert err < 2e-4, f"relative gradient error {err:.2e}"
    assert np.abs(total_o).sum() > 0


@pytest.mark.parametrize("K", [2, 512, 513, 4096])
def test_gradient_table_sizes(rc, orc, c4, K):
    """Both accumulator forms of a 1-D table against the FP64 oracle at their
    edges: per-warp FP32 copies up to 512 entries (2: every sample lerps
    entries 0 and 1; 512: the largest), the CTA's 64-bit fixed-point sums
    above (513: the smallest; 4096: the largest table), one 4-view launch and
    repeated bit for bit."""
    import torch
    ph, ctx, vol, cams = c4
    cams = cams[:4]
    tf = synth.noise_tf(K, 300 + K, alpha_max=0.1)
    term = 0.99
    total_o = np.zeros((K, 4))
    gs = []
    for v, cam in enumerate(cams):
        pix = synth.sample_pixels(W["width"], W["height"], 1024, seed=1300 + v)
        sc = orc.Scene(ph.vol, ph.spacing, tf, cam, step=W["step"], term=term)
        keep = pix[~orc.render(sc, pixels=pix)["tie"]]
        g = seeded_upstream(1350 + v, keep, (W["height"], W["width"]))
        gs.append(g)
        og, _ = orc.render_grad(sc, g[keep], pixels=keep)
        total_o += og
    rc.rc_tf_set(ctx, tf)
    G = torch.from_numpy(np.stack(gs).astype(np.float32).reshape(len(cams), W["height"], W["width"], 4)).cuda()
    dtf = torch.empty((K, 4), device="cuda", dtype=torch.float32)
    p = rc.RenderParams(step_vox=W["step"], term=term, shade=False, skip=False)
    rc.rc_render_backward_views(ctx, vol, p, cams, G, dtf)
    torch.cuda.synchronize()
    got = dtf.cpu().numpy().astype(np.float64)
    scale = np.abs(total_o).max()
    assert scale > 0
    assert np.abs(got - total_o).max() / scale < 2e-4, np.abs(got - total_o).max() / scale
    rc.rc_render_backward_views(ctx, vol, p, cams, G, dtf)
    torch.cuda.synchronize()
    assert np.array_equal(dtf.cpu().numpy().astype(np.float64), got)


@pytest.mark.parametrize("K,tf2d", [(256, False), (1024, False), (256, True)])
def test_gradient_ragged_image_every_pixel(rc, orc, c4, K, tf2d):
    """An image of 45 x 27 pixels, neither side a multiple of the block's
    16 x 8 (or, 2-D table, 16 x 16) pixels: the lanes outside the image take
    part in every warp barrier of the scatter and add nothing. Every pixel's
    upstream gradient is non-zero (except termination ties); two views in one
    launch, recomputing the forward and given the forward images, against the
    FP64 oracle; 256 entries take the per-warp accumulators, 1024 the block's
    fixed-point ones."""
    import torch
    ph, ctx, vol, _ = c4
    H, Wd = 27, 45
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=Wd, height=H) for az in (20.0, 200.0)]
    if tf2d:
        M = 8
        tab = np.repeat(synth.noise_tf(K, 1400, alpha_max=0.1)[None], M, axis=0)
        tab[..., 3] *= np.linspace(0.4, 1.0, M, dtype=np.float32)[:, None]
        rc.rc_tf2d_set(ctx, tab, GMAX)
        shape = tab.shape
    else:
        tab = synth.noise_tf(K, 1400 + K, alpha_max=0.1)
        rc.rc_tf_set(ctx, tab)
        shape = (K, 4)
    term = 0.99
    total_o = np.zeros(shape)
    gs = []
    for v, cam in enumerate(cams):
        sc = orc.Scene(ph.vol, ph.spacing, tab, cam, step=W["step"], term=term, gmax=GMAX if tf2d else None)
        fwd = orc.render(sc)
        keep = np.flatnonzero(~fwd["tie"].reshape(-1))
        assert len(keep) > 0.9 * H * Wd
        g = seeded_upstream(1450 + v, keep, (H, Wd))
        gs.append(g)
        total_o += orc.render_grad(sc, g[keep], pixels=keep)[0]
    G = torch.from_numpy(np.stack(gs).astype(np.float32).reshape(len(cams), H, Wd, 4)).cuda()
    p = rc.RenderParams(step_vox=W["step"], term=term, shade=False, skip=False)
    imgs = torch.empty((len(cams), H, Wd, 4), device="cuda")
    rc.rc_render_views(ctx, vol, p, cams, imgs)
    a = torch.empty(shape, device="cuda")
    b = torch.empty(shape, device="cuda")
    rc.rc_render_backward_views(ctx, vol, p, cams, G, a)
    rc.rc_render_backward_views_with_forward(ctx, vol, p, cams, imgs, G, b)
    torch.cuda.synchronize()
    scale = np.abs(total_o).max()
    assert scale > 0
    for got in (a, b):
        err = np.abs(got.cpu().numpy().astype(np.float64) - total_o).max() / scale
        assert err < 2e-4, err


def test_views_gradient_matches_oracle_and_single_views(rc, orc, c4):
    """One launch over all 8 views: the summed gradient equals the oracle's
    sum over the views, and the sum of the per-view gradients (to the
    fixed-point resolution: the views call has one scale for all views)."""
    import torch
    ph, ctx, vol, cams = c4
    tf = init_tf()
    term = 0.99
    gs, total_o, total_1 = [], np.zeros((W["K"], 4)), np.zeros((W["K"], 4))
    for v, cam in enumerate(cams):
        pix = synth.sample_pixels(W["width"], W["height"], 2048, seed=900 + v)
        sc = orc.Scene(ph.vol, ph.spacing, tf, cam, step=W["step"], term=term)
        keep = pix[~orc.render(sc, pixels=pix)["tie"]]
        g = seeded_upstream(950 + v, keep, (W["height"], W["width"]))
        gs.append(g)
        og, _ = orc.render_grad(sc, g[keep], pixels=keep)
        total_o += og
        total_1 += gpu_grad(rc, ctx, vol, cam, tf, g, term)
    rc.rc_tf_set(ctx, tf)
    G = torch.from_numpy(np.stack(gs).astype(np.float32).reshape(len(cams), W["height"], W["width"], 4)).cuda()
    dtf = torch.empty((W["K"], 4), device="cuda", dtype=torch.float32)
    p = rc.RenderParams(step_vox=W["step"], term=term, shade=False, skip=False)
    rc.rc_render_backward_views(ctx, vol, p, cams, G, dtf)
    torch.cuda.synchronize()
    got = dtf.cpu().numpy().astype(np.float64)
    scale = np.abs(total_o).max()
    assert np.abs(got - total_o).max() / scale < 2e-4
    assert np.abs(got - total_1).max() / scale < 1e-5
    # deterministic
    rc.rc_render_backward_views(ctx, vol, p, cams, G, dtf)
    torch.cuda.synchronize()
    assert np.array_equal(dtf.cpu().numpy().astype(np.float64), got)


@pytest.mark.parametrize("form", ["plain", "plain_term1", "shaded", "bspline", "tf2d"])
def test_gradient_with_forward_images(rc, orc, c4, form):
    """The gradient given the forward images (one march per ray, the final
    colour and transmittance read from the images, termination found by the
    gradient march itself) equals the gradient that recomputes the forward,
    for every form the gradient takes, over four views in one launch; the
    plain form also against the oracle."""
    import torch
    ph, ctx, vol, cams = c4
    cams = cams[:4]
    term = 1.0 if form == "plain_term1" else 0.99
    shade = form in ("shaded", "bspline")
    filt = rc.RC_FILTER_BSPLINE if form == "bspline" else rc.RC_FILTER_TRILINEAR
    if form == "tf2d":
        tab = init_tf2d(8)
        rc.rc_tf2d_set(ctx, tab, GMAX)
        shape = tab.shape
    else:
        rc.rc_tf_set(ctx, init_tf())
        shape = (W["K"], 4)
    p = rc.RenderParams(step_vox=W["step"], term=term, shade=shade, skip=True, filter=filt)
    H, Wd = W["height"], W["width"]
    imgs = torch.empty((len(cams), H, Wd, 4), device="cuda")
    rc.rc_render_views(ctx, vol, p, cams, imgs)
    G = torch.randn(imgs.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(77))
    a = torch.empty(shape, device="cuda")
    b = torch.empty(shape, device="cuda")
    rc.rc_render_backward_views(ctx, vol, p, cams, G, a)
    rc.rc_render_backward_views_with_forward(ctx, vol, p, cams, imgs, G, b)
    torch.cuda.synchronize()
    A, B = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    scale = np.abs(A).max()
    assert scale > 0 and np.abs(A - B).max() <= 2e-5 * scale, np.abs(A - B).max() / scale
    rc.rc_render_backward_views_with_forward(ctx, vol, p, cams, imgs, G, a)
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy().astype(np.float64), B)            # deterministic
    if form == "plain":
        tf = init_tf()
        total_o = np.zeros((W["K"], 4))
        gs = []
        for v, cam in enumerate(cams):
            pix = synth.sample_pixels(W["width"], W["height"], 2048, seed=960 + v)
            sc = orc.Scene(ph.vol, ph.spacing, tf, cam, step=W["step"], term=term)
            keep = pix[~orc.render(sc, pixels=pix)["tie"]]
            g = seeded_upstream(970 + v, keep, (H, Wd))
            gs.append(g)
            total_o += orc.render_grad(sc, g[keep], pixels=keep)[0]
        G2 = torch.from_numpy(np.stack(gs).astype(np.float32).reshape(len(cams), H, Wd, 4)).cuda()
        rc.rc_render_backward_views_with_forward(ctx, vol, p, cams, imgs, G2, b)
        torch.cuda.synchronize()
        got = b.cpu().numpy().astype(np.float64)
        assert np.abs(got - total_o).max() / np.abs(total_o).max() < 2e-4
    with pytest.raises(rc.RCError) as ei:
        rc.rc_render_backward_views_with_forward(ctx, vol, p, cams, None, G, b)
    assert ei.value.status == rc.RC_ERR_INVALID_ARG
    rc.rc_tf_set(ctx, init_tf())


GMAX = 1200.0


def init_tf2d(M):
    """The seeded noise table repeated over M gradient-magnitude rows, its
    opacity rising and its blue falling with the row, so that every row
    carries a different gradient."""
    g = np.arange(M, dtype=np.float64)[:, None] / (M - 1)
    tab = np.repeat(init_tf().astype(np.float64)[None], M, axis=0)
    tab[..., 3] *= 0.4 + 0.6 * g
    tab[..., 2] *= 1.0 - 0.4 * g
    return np.clip(tab, 0.0, 1.0).astype(np.float32)


@pytest.mark.parametrize("shade,bspline,M", [(False, False, 8), (True, False, 8), (True, True, 8),
                                             (False, False, 4)])
def test_tf2d_gradient_matches_oracle(rc, orc, c4, shade, bspline, M):
    """The gradient of a 2-D (value x gradient magnitude) table against the
    FP64 oracle's reverse mode, summed over four views; M = 4 (1024 entries,
    the largest table the non-allocating entry point takes) goes through
    that entry point."""
    import torch
    ph, ctx, vol, cams = c4
    tab = init_tf2d(M)
    term = 0.99
    filt = rc.RC_FILTER_BSPLINE if bspline else rc.RC_FILTER_TRILINEAR
    noalloc = M * W["K"] <= 1024
    total_g = np.zeros((M, W["K"], 4))
    total_o = np.zeros((M, W["K"], 4))
    rc.rc_tf2d_set(ctx, tab, GMAX)
    for v, cam in enumerate(cams[:4]):
        pix = synth.sample_pixels(W["width"], W["height"], 4096, seed=1400 + v)
        sc = orc.Scene(ph.vol, ph.spacing, tab, cam, step=W["step"], term=term, shade=shade,
                       filter=orc.BSPLINE if bspline else orc.TRILINEAR, gmax=GMAX)
        keep = pix[~orc.render(sc, pixels=pix)["tie"]]
        g = seeded_upstream(1450 + v, keep, (W["height"], W["width"]))
        og, _ = orc.render_grad(sc, g[keep], pixels=keep)
        assert og.shape == (M, W["K"], 4)
        total_o += og
        rc.rc_camera_set(ctx, cam)
        gd = torch.from_numpy(g.astype(np.float32)).cuda()
        dtf = torch.empty((M, W["K"], 4), device="cuda", dtype=torch.float32)
        p = rc.RenderParams(step_vox=W["step"], term=term, shade=shade, skip=False, filter=filt)
        (rc.rc_render_backward_noalloc if noalloc else rc.rc_render_backward)(ctx, vol, p, gd, dtf)
        torch.cuda.synchronize()
        total_g += dtf.cpu().numpy().astype(np.float64)
    scale = np.abs(total_o).max()
    err = np.abs(total_g - total_o).max() / scale
    assert err < 2e-4, f"relative gradient error {err:.2e}"
    # the gradient reaches several rows of the table
    assert (np.abs(total_o).sum(axis=(1, 2)) > 1e-3 * scale).sum() >= 3


def test_tf2d_views_gradient_is_the_sum_and_deterministic(rc, c4):
    """One launch over the views of a 2-D table equals the sum of the
    single-view gradients (to the fixed-point resolution) and repeats bit for bit."""
    import torch
    ph, ctx, vol, cams = c4
    tab = init_tf2d(8)
    rc.rc_tf2d_set(ctx, tab, GMAX)
    rng = np.random.default_rng(12)
    gs = [rng.normal(size=(W["height"], W["width"], 4)).astype(np.float32) for _ in cams[:3]]
    p = rc.RenderParams(step_vox=W["step"], term=0.99, shade=True, skip=False)
    total = np.zeros((8, W["K"], 4))
    dtf = torch.empty((8, W["K"], 4), device="cuda", dtype=torch.float32)
    for cam, g in zip(cams, gs):
        rc.rc_camera_set(ctx, cam)
        rc.rc_render_backward(ctx, vol, p, torch.from_numpy(g).cuda(), dtf)
        torch.cuda.synchronize()
        total += dtf.cpu().numpy()
    G = torch.from_numpy(np.stack(gs)).cuda()
    rc.rc_render_backward_views(ctx, vol, p, cams[:3], G, dtf)
    torch.cuda.synchronize()
    got = dtf.cpu().numpy().astype(np.float64)
    assert np.abs(got - total).max() / np.abs(total).max() < 1e-5
    rc.rc_render_backward_views(ctx, vol, p, cams[:3], G, dtf)
    torch.cuda.synchronize()
    assert np.array_equal(dtf.cpu().numpy().astype(np.float64), got)


def test_gradient_matches_central_differences(rc, orc, c4):
    """Central differences (h = 1e-3) of <I(tf), G> with the FP64 oracle,
    termination off so that h cannot flip a stop decision, on the 32 entries
    with the largest gradient."""
    ph, ctx, vol, cams = c4
    tf = init_tf()
    cam = cams[1]
    pix = synth.sample_pixels(W["width"], W["height"], 2048, seed=77)
    g = seeded_upstream(78, pix, (W["height"], W["width"]))
    grad = gpu_grad(rc, ctx, vol, cam, tf, g, 1.0)

    def loss(t):
        sc = orc.Scene(ph.vol, ph.spacing, t, cam, step=W["step"], term=1.0)
        return float((orc.render(sc, pixels=pix)["rgba"] * g[pix]).sum())

    flat = np.argsort(-np.abs(grad).ravel())[:32]
    h = 1e-3
    for f in flat:
        i, c = divmod(int(f), 4)
        tp = tf.copy(); tm = tf.copy()
        tp[i, c] = min(1.0, tf[i, c] + h)
        tm[i, c] = max(0.0, tf[i, c] - h)
        fd = (loss(tp) - loss(tm)) / (float(tp[i, c]) - float(tm[i, c]))
        assert grad[i, c] == pytest.approx(fd, rel=2e-3, abs=1e-3 * np.abs(grad).max())


def test_gradient_is_deterministic(rc, c4):
    ph, ctx, vol, cams = c4
    tf = init_tf()
    g = np.random.default_rng(1).normal(size=(W["height"] * W["width"], 4))
    a = gpu_grad(rc, ctx, vol, cams[2], tf, g, 0.99)
    b = gpu_grad(rc, ctx, vol, cams[2], tf, g, 0.99)
    assert np.array_equal(a, b)


def test_autograd_and_tf_fit(rc, c4):
    """Fit the learnable table (seeded noise) to 8 target views rendered with
    the hidden table: the L2 loss must fall by more than half."""
    import torch
    from paper_1211_5595_gb300.autograd import render_tf
    ph, ctx, vol, cams = c4
    params = rc.RenderParams(step_vox=W["step"], term=W["term"], shade=False, skip=True)
    hid = torch.from_numpy(hidden_tf()).cuda()
    with torch.no_grad():
        targets = [render_tf(hid, ctx, vol, params, cam).clone() for cam in cams]
    tf = torch.from_numpy(init_tf()).cuda().requires_grad_(True)
    # autograd gradient equals the direct adjoint call
    img = render_tf(tf, ctx, vol, params, cams[0])
    loss = ((img - targets[0]) ** 2).mean()
    loss.backward()
    direct = torch.empty_like(tf)
    rc.rc_tf_set_device(ctx, tf.detach())
    rc.rc_camera_set(ctx, cams[0])
    rc.rc_render_backward(ctx, vol, params, (2 * (img - targets[0]) / img.numel()).detach().contiguous(), direct)
    torch.cuda.synchronize()
    assert torch.allclose(tf.grad, direct, rtol=1e-5, atol=1e-9)
    opt = torch.optim.Adam([tf], lr=0.01)
    losses = []
    for it in range(60):
        opt.zero_grad()
        loss = sum(((render_tf(tf, ctx, vol, params, cam) - t) ** 2).mean() for cam, t in zip(cams, targets))
        loss.backward()
        opt.step()
        with torch.no_grad():
            tf.clamp_(0.0, 1.0)
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.5 * losses[0], losses[::10]


def test_autograd_tf2d_and_fit(rc, c4):
    """The autograd wrapper with a 2-D table (set from device memory): its
    gradient equals the direct adjoint call, and fitting the table to 4
    target views rendered with a hidden 2-D table lowers the L2 loss by more
    than half."""
    import torch
    from paper_1211_5595_gb300.autograd import render_tf
    ph, ctx, vol, cams = c4
    M = 8
    g = np.arange(M, dtype=np.float64)[:, None] / (M - 1)
    hid = np.repeat(hidden_tf().astype(np.float64)[None], M, axis=0)
    hid[..., 3] *= 0.3 + 0.7 * g
    params = rc.RenderParams(step_vox=W["step"], term=W["term"], shade=False, skip=True)
    views = cams[::2]
    with torch.no_grad():
        hid_t = torch.from_numpy(hid.astype(np.float32)).cuda()
        targets = [render_tf(hid_t, ctx, vol, params, cam, GMAX).clone() for cam in views]
    tf = torch.from_numpy(init_tf2d(M)).cuda().requires_grad_(True)
    img = render_tf(tf, ctx, vol, params, views[0], GMAX)
    loss = ((img - targets[0]) ** 2).mean()
    loss.backward()
    direct = torch.empty_like(tf)
    rc.rc_tf2d_set_device(ctx, tf.detach(), GMAX)
    rc.rc_camera_set(ctx, views[0])
    rc.rc_render_backward(ctx, vol, params, (2 * (img - targets[0]) / img.numel()).detach().contiguous(), direct)
    torch.cuda.synchronize()
    assert torch.allclose(tf.grad, direct, rtol=1e-5, atol=1e-9)
    # the device setter gives the same image as the host one
    rc.rc_tf2d_set(ctx, tf.detach().cpu().numpy(), GMAX)
    ref = torch.empty_like(img)
    rc.rc_render(ctx, vol, params, ref)
    torch.cuda.synchronize()
    assert torch.equal(ref, img.detach())
    opt = torch.optim.Adam([tf], lr=0.01)
    losses = []
    for it in range(40):
        opt.zero_grad()
        loss = sum(((render_tf(tf, ctx, vol, params, cam, GMAX) - t) ** 2).mean() for cam, t in zip(views, targets))
        loss.backward()
        opt.step()
        with torch.no_grad():
            tf.clamp_(0.0, 1.0)
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.5 * losses[0], losses[::10]
