"""Learned sampling proposal on the GPU: features, network, gradient, Adam,
blob save/resume, 512-sample profiles and the importance march checked against
the oracle; then the network trained on 32 seeded phantoms and evaluated on 8
held-out ones against the plain march, with the gain over the same march
without the network (uniform or occupancy-only sample densities)."""
import numpy as np
import pytest

import synth
from gpu_helpers import TOL_FP32, GPURenderer, compare

pytestmark = pytest.mark.gpu

W5 = synth.WORKLOADS["proposal_256x256x180"]


@pytest.fixture(scope="module")
def rc():
    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc
    return rc


@pytest.fixture(scope="module")
def mlp():
    import oracle.mlp as m
    return m


@pytest.fixture(scope="module")
def small(rc):
    ph = synth.head_phantom((128, 128, 96), (1, 1, 1), seed=1005, tumor_radius_vox=7)
    r = GPURenderer(rc, ph.vol, ph.spacing)
    tf = synth.tf_table(256)
    r.set_tf(tf)
    yield ph, tf, r
    r.close()


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def params_for(**kw):
    base = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
    base.update(kw)
    return base


# --------------------------------------------------------------------------
# features, network, gradient, optimiser
# --------------------------------------------------------------------------
def test_features_parity(rc, orc, small):
    import torch
    ph, tf, r = small
    cam = synth.orbit_camera(ph.dims, ph.spacing, 25.0, width=96, height=80)
    rc.rc_camera_set(r.ctx, cam)
    F = torch.empty((96 * 80, 112), device="cuda")
    rc.rc_proposal_features(r.ctx, r.vol, params_for(), F)
    torch.cuda.synchronize()
    g = F.cpu().numpy().astype(np.float64)
    mn, mx = orc.brick_minmax(ph.vol)
    occ = orc.occupancy(ph.dims, tf, mn, mx)
    o = orc.proposal_features(orc.Scene(ph.vol, ph.spacing, tf, cam), occ)
    np.testing.assert_allclose(g[:, :78], o[:, :78], atol=2e-6)
    assert np.array_equal(g[:, 78:], o[:, 78:])
    assert (o[:, 78:110].sum(axis=1) > 0).sum() > 1000


def test_network_forward_parity(rc, mlp):
    import torch
    ctx = rc.rc_context_create(0)
    try:
        p = synth.proposal_init_params(21)
        rc.rc_proposal_load(ctx, rc.pack_proposal_blob(p))
        f, _ = synth.proposal_batch(22, 1000)          # not a multiple of 32: ragged tail
        out = torch.empty((1000, 33), device="cuda")
        rc.rc_proposal_forward(ctx, cuda(f), 1000, out)
        torch.cuda.synchronize()
        g = out.cpu().numpy().astype(np.float64)
        o = mlp.forward(p, f)
        d_pdf = np.abs(g[:, :32] - o["pdf"])
        d_t = np.abs(g[:, 32] - o["that"])
        assert np.allclose(g[:, :32].sum(axis=1), 1.0, atol=1e-5)
        # FP32 accumulation order can move a hidden activation across a BF16
        # rounding boundary (1 ulp = 2^-8 relative); most rows agree to 1e-6
        assert np.median(d_pdf) < 1e-6 and d_pdf.max() < 2e-3
        assert np.median(d_t) < 1e-6 and d_t.max() < 2e-3
    finally:
        rc.rc_context_destroy(ctx)


def test_gradient_parity_and_adam(rc, mlp):
    import torch
    ctx = rc.rc_context_create(0)
    try:
        p = synth.proposal_init_params(31).astype(np.float32)
        p[:] += (0.01 * np.random.default_rng(3).normal(size=p.size) * (p != 0)).astype(np.float32)
        rc.rc_proposal_load(ctx, rc.pack_proposal_blob(p))
        f, t = synth.proposal_batch(32, 777)
        grad = torch.empty(rc.RC_PROPOSAL_PARAMS, device="cuda")
        loss = torch.empty(1, device="cuda")
        rc.rc_proposal_grad(ctx, cuda(f), cuda(t), 777, grad, loss)
        torch.cuda.synchronize()
        g = grad.cpu().numpy().astype(np.float64)
        ol, og = mlp.loss_and_grad(p, f, t)
        assert float(loss.item()) == pytest.approx(ol, rel=1e-3)
        assert np.abs(g - og).max() <= 1e-2 * np.abs(og).max()
        # one Adam step from zero moments: each weight moves by -lr sign(g)
        g2 = torch.empty_like(grad)
        rc.rc_proposal_grad(ctx, cuda(f), cuda(t), 777, g2)
        assert torch.equal(grad, g2)                     # deterministic reduction
        rc.rc_proposal_train_step(ctx, cuda(f), cuda(t), 777, 1e-3)
        after = rc.unpack_proposal_blob(rc.rc_proposal_save(ctx))
        step = after["params"].astype(np.float64) - p
        big = np.abs(og) > 1e-3 * np.abs(og).max()
        np.testing.assert_allclose(step[big], -1e-3 * np.sign(og[big]), rtol=2e-3, atol=1e-7)
        assert after["adam_step"] == 1
    finally:
        rc.rc_context_destroy(ctx)


def test_blob_resume_reproduces_training(rc):
    import torch
    ctx = rc.rc_context_create(0)
    try:
        rc.rc_proposal_load(ctx, rc.pack_proposal_blob(synth.proposal_init_params(41)))
        f, t = synth.proposal_batch(42, 512)
        F, T = cuda(f), cuda(t)
        loss = torch.empty(1, device="cuda")
        for _ in range(3):
            rc.rc_proposal_train_step(ctx, F, T, 512, 2e-3, loss)
        blob = rc.rc_proposal_save(ctx)
        curve_a = []
        for _ in range(4):
            rc.rc_proposal_train_step(ctx, F, T, 512, 2e-3, loss)
            curve_a.append(float(loss.item()))
        a = rc.rc_proposal_save(ctx)
        rc.rc_proposal_load(ctx, blob)
        curve_b = []
        for _ in range(4):
            rc.rc_proposal_train_step(ctx, F, T, 512, 2e-3, loss)
            curve_b.append(float(loss.item()))
        b = rc.rc_proposal_save(ctx)
        assert curve_a == curve_b and a == b
        with pytest.raises(rc.RCError) as ei:
            rc.rc_proposal_load(ctx, blob[:-4])
        assert ei.value.status == rc.RC_ERR_FORMAT
        bad = bytearray(blob)
        bad[0:8] = b"XXXXXXXX"
        with pytest.raises(rc.RCError):
            rc.rc_proposal_load(ctx, bytes(bad))
        assert rc.rc_proposal_save(ctx) == b                # the failed loads changed nothing
    finally:
        rc.rc_context_destroy(ctx)


# --------------------------------------------------------------------------
# profiles and the importance march
# --------------------------------------------------------------------------
def test_profiles_parity(rc, orc, small):
    import torch
    ph, tf, r = small
    cam = synth.orbit_camera(ph.dims, ph.spacing, 70.0, width=128, height=112)
    rc.rc_camera_set(r.ctx, cam)
    Y = torch.empty((128 * 112, 33), device="cuda")
    rc.rc_profiles_generate(r.ctx, r.vol, params_for(), Y)
    torch.cuda.synchronize()
    g = Y.cpu().numpy().astype(np.float64)
    pix = synth.sample_pixels(128, 112, 3000, seed=5)
    bins, tfin = orc.profiles(orc.Scene(ph.vol, ph.spacing, tf, cam), pixels=pix)
    np.testing.assert_allclose(g[pix, :32], bins, atol=2e-4)
    np.testing.assert_allclose(g[pix, 32], tfin, atol=2e-4)
    assert (tfin < 0.5).sum() > 100


def seeded_pdfs(n, seed):
    u = synth.uniform01(seed, np.arange(n * 32)).reshape(n, 32) ** 3
    return (u / u.sum(axis=1, keepdims=True)).astype(np.float32)


@pytest.mark.parametrize("term,nimp", [(1.0, 64), (1.0, 17), (0.99, 64), (0.99, 17)])
def test_importance_parity(rc, orc, small, term, nimp):
    """The range reading against the oracle, every pixel within 2e-4 (a ray
    whose stop decision lies within the tie band of term matches either
    branch)."""
    import torch
    ph, tf, r = small
    cam = synth.orbit_camera(ph.dims, ph.spacing, 140.0, width=80, height=72)
    rc.rc_camera_set(r.ctx, cam)
    n = 80 * 72
    pdf = seeded_pdfs(n, 77)
    that = np.full(n, 0.5, dtype=np.float32)
    out = torch.empty((72, 80, 4), device="cuda")
    fb = torch.empty(n, dtype=torch.uint8, device="cuda")
    rc.rc_render_importance(r.ctx, r.vol, params_for(term=term), cuda(pdf), cuda(that), nimp, 2.0, out, fb)
    torch.cuda.synchronize()
    o = orc.importance(orc.Scene(ph.vol, ph.spacing, tf, cam, term=term, shade=True), pdf, nimp=nimp)
    assert fb.sum().item() == 0
    err, ties = compare(out.cpu().numpy(), o, TOL_FP32)
    assert o["rgba"][:, 3].max() > 0.5
    print(f"importance range nimp {nimp} term {term}: max-abs {err:.2e}, {int(o['tie'].sum())} tie rays")


@pytest.mark.parametrize("lam,nimp,term,sparse", [(0.05, 64, 1.0, False), (0.05, 17, 0.99, False),
                                                  (0.0, 64, 0.99, False), (1.0, 64, 0.99, False),
                                                  (1.0, 128, 1.0, False), (0.05, 1, 0.99, False),
                                                  (0.0, 33, 0.99, True), (0.0, 1, 1.0, True)])
def test_importance_invcdf_parity(rc, orc, small, lam, nimp, term, sparse):
    """The inverse-CDF reading (stratified samples of the lambda-mixture,
    midpoint segments) over two views in one launch against the oracle, every
    pixel within 2e-4 (either branch of a termination tie); lambda = 1 without
    a PDF (the uniform march over the chord) and without T^ (no fallback); a
    single sample per ray (it stands for the whole chord); lambda = 0 with
    PDFs whose bins are mostly empty (the bin search steps over zero-width
    bins)."""
    import torch
    ph, tf, r = small
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=72, height=64) for az in (40.0, 230.0)]
    n = 72 * 64
    pdf = np.stack([seeded_pdfs(n, 81), seeded_pdfs(n, 82)])
    if sparse:
        keep = synth.uniform01(83, np.arange(2 * n * 32)).reshape(2, n, 32) < 0.15
        keep[..., 5] = True                                  # at least one bin per ray
        pdf = np.where(keep, pdf, 0.0)
        pdf = (pdf / pdf.sum(axis=-1, keepdims=True)).astype(np.float32)
    out = torch.empty((2, 64, 72, 4), device="cuda")
    fb = torch.empty((2, n), dtype=torch.uint8, device="cuda")
    uniform = lam == 1.0
    rc.rc_render_importance_views(r.ctx, r.vol, params_for(term=term), cams, rc.RC_SAMPLING_INVCDF, lam,
                                  None if uniform else cuda(pdf), None if uniform else cuda(np.full((2, n), 0.5)),
                                  nimp, 2.0, out, fb)
    torch.cuda.synchronize()
    assert fb.sum().item() == 0
    for v, cam in enumerate(cams):
        o = orc.importance(orc.Scene(ph.vol, ph.spacing, tf, cam, term=term, shade=True),
                           None if uniform else pdf[v], nimp=nimp, sampling="invcdf", lam=lam)
        err, _ = compare(out[v].cpu().numpy(), o, TOL_FP32)
        assert o["rgba"][:, 3].max() > 0.5


def test_importance_views_range_equals_single_views(rc, small):
    """The range reading through the several-view entry point gives each
    view's rc_render_importance image and fallback flags exactly."""
    import torch
    ph, tf, r = small
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=56, height=48) for az in (10.0, 100.0, 300.0)]
    n = 56 * 48
    pdf = cuda(np.stack([seeded_pdfs(n, 90 + v) for v in range(3)]))
    that = cuda(np.full((3, n), 0.4))
    out = torch.empty((3, 48, 56, 4), device="cuda")
    fb = torch.empty((3, n), dtype=torch.uint8, device="cuda")
    st = rc.rc_render_importance_views(r.ctx, r.vol, params_for(), cams, rc.RC_SAMPLING_RANGE, 0.0, pdf, that,
                                       64, 0.05, out, fb, stats=True)
    one = torch.empty((48, 56, 4), device="cuda")
    f1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    fb_total = 0
    for v, cam in enumerate(cams):
        rc.rc_camera_set(r.ctx, cam)
        s1 = rc.rc_render_importance(r.ctx, r.vol, params_for(), pdf[v].contiguous(), that[v].contiguous(), 64,
                                     0.05, one, f1, stats=True)
        torch.cuda.synchronize()
        assert torch.equal(out[v], one) and torch.equal(fb[v], f1)
        fb_total += s1["fallback_rays"]
    assert st["fallback_rays"] == fb_total > 0
    with pytest.raises(rc.RCError) as ei:
        rc.rc_render_importance_views(r.ctx, r.vol, params_for(), cams, rc.RC_SAMPLING_INVCDF, 1.5, None, None, 64,
                                      0.05, out)
    assert ei.value.status == rc.RC_ERR_INVALID_ARG
    with pytest.raises(rc.RCError) as ei:
        rc.rc_render_importance_views(r.ctx, r.vol, params_for(), cams, rc.RC_SAMPLING_INVCDF, 0.5, None, None, 64,
                                      0.05, out)
    assert ei.value.status == rc.RC_ERR_INVALID_ARG


def test_fallback_rays_equal_the_plain_march(rc, small):
    import torch
    ph, tf, r = small
    cam = synth.orbit_camera(ph.dims, ph.spacing, 200.0, width=96, height=96)
    rc.rc_camera_set(r.ctx, cam)
    n = 96 * 96
    plain = torch.empty((96, 96, 4), device="cuda")
    rc.rc_render(r.ctx, r.vol, params_for(), plain)
    out = torch.empty_like(plain)
    fb = torch.empty(n, dtype=torch.uint8, device="cuda")
    st = rc.rc_render_importance(r.ctx, r.vol, params_for(), cuda(seeded_pdfs(n, 3)),
                                 cuda(np.full(n, 2.0, np.float32)), 64, 0.0, out, fb, stats=True)
    torch.cuda.synchronize()
    m = fb.view(96, 96).bool()
    assert st["fallback_rays"] == int(m.sum()) and st["fallback_rays"] > 1000
    assert torch.equal(out[m], plain[m])


def test_invcdf_proposal_render_matches_network_pdfs(rc, small):
    """The inverse-CDF proposal render (network kernel writing every ray's
    PDF and T^, then the inverse-CDF march) equals the inverse-CDF march fed
    with the network's outputs for the same rays, fallback flags included."""
    import torch
    ph, tf, r = small
    rc.rc_proposal_load(r.ctx, rc.pack_proposal_blob(synth.proposal_init_params(54)))
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=80, height=64) for az in (75.0, 190.0)]
    n = 80 * 64
    net = torch.empty((2, n, 33), device="cuda")
    hit = []
    for v, cam in enumerate(cams):
        rc.rc_camera_set(r.ctx, cam)
        F = torch.empty((n, 112), device="cuda")
        rc.rc_proposal_features(r.ctx, r.vol, params_for(), F)
        rc.rc_proposal_forward(r.ctx, F, n, net[v])
        hit.append(F[:, 3:6].abs().sum(dim=1) > 0)
    a = torch.empty((2, 64, 80, 4), device="cuda")
    b = torch.empty_like(a)
    fa = torch.empty((2, n), dtype=torch.uint8, device="cuda")
    fbb = torch.empty_like(fa)
    rc.rc_render_importance_views(r.ctx, r.vol, params_for(), cams, rc.RC_SAMPLING_INVCDF, 0.05,
                                  net[:, :, :32].contiguous(), net[:, :, 32].contiguous(), 64, 0.02, a, fa)
    st = rc.rc_render_proposal_sampled(r.ctx, r.vol, params_for(), cams, rc.RC_SAMPLING_INVCDF, 0.05, 64, 0.02,
                                       b, fbb, stats=True)
    torch.cuda.synchronize()
    for v in range(2):
        h = hit[v]
        assert torch.equal(fa[v][h], fbb[v][h])
        assert torch.equal(a[v].view(-1, 4)[h], b[v].view(-1, 4)[h])
    assert st["rays_total"] == 2 * n


def test_fused_render_matches_network_pdfs(rc, small):
    """The proposal render (tensor-core network kernel writing each ray's
    range record, then the importance march) equals the importance march fed
    with the network's PDFs for the same rays."""
    import torch
    ph, tf, r = small
    rc.rc_proposal_load(r.ctx, rc.pack_proposal_blob(synth.proposal_init_params(51)))
    cam = synth.orbit_camera(ph.dims, ph.spacing, 300.0, width=112, height=96)
    rc.rc_camera_set(r.ctx, cam)
    n = 112 * 96
    F = torch.empty((n, 112), device="cuda")
    rc.rc_proposal_features(r.ctx, r.vol, params_for(), F)
    net = torch.empty((n, 33), device="cuda")
    rc.rc_proposal_forward(r.ctx, F, n, net)
    a = torch.empty((96, 112, 4), device="cuda")
    b = torch.empty_like(a)
    fa = torch.empty(n, dtype=torch.uint8, device="cuda")
    fbb = torch.empty_like(fa)
    rc.rc_render_importance(r.ctx, r.vol, params_for(), net[:, :32].contiguous(), net[:, 32].contiguous(), 64,
                            0.02, a, fa)
    rc.rc_render_proposal(r.ctx, r.vol, params_for(), 64, 0.02, b, fbb)
    torch.cuda.synchronize()
    hit = F[:, 3:6].abs().sum(dim=1) > 0
    assert torch.equal(fa, fbb)
    assert torch.equal(a.view(-1, 4)[hit], b.view(-1, 4)[hit])


@pytest.mark.parametrize("sampling", ["range", "invcdf"])
def test_proposal_render_with_empty_tiles(rc, small, sampling):
    """A distant camera: the volume covers a small part of a ragged image, so
    most 128-ray tiles have no ray that meets it and the network kernel skips
    them. The proposal render still equals the importance march fed with the
    network's outputs on every pixel (rays that miss are black), in both
    readings, over three views in one launch pair."""
    import torch
    ph, tf, r = small
    rc.rc_proposal_load(r.ctx, rc.pack_proposal_blob(synth.proposal_init_params(57)))
    W, H = 150, 131
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=W, height=H, distance_scale=4.0)
            for az in (20.0, 140.0, 260.0)]
    n = W * H
    net = torch.empty((3, n, 33), device="cuda")
    hits = []
    for v, cam in enumerate(cams):
        rc.rc_camera_set(r.ctx, cam)
        F = torch.empty((n, 112), device="cuda")
        rc.rc_proposal_features(r.ctx, r.vol, params_for(), F)
        rc.rc_proposal_forward(r.ctx, F, n, net[v])
        hits.append(F[:, 3:6].abs().sum(dim=1) > 0)
    hit = torch.stack(hits).view(3, H, W)
    # most 16 x 8 tiles see no hit ray
    tiles = torch.zeros((3, (H + 7) // 8 * 8, (W + 15) // 16 * 16), dtype=torch.bool, device="cuda")
    tiles[:, :H, :W] = hit
    any_hit = tiles.view(3, (H + 7) // 8, 8, (W + 15) // 16, 16).any(dim=4).any(dim=2)
    assert 0 < int(any_hit.sum()) < 0.5 * any_hit.numel()
    mode = rc.RC_SAMPLING_RANGE if sampling == "range" else rc.RC_SAMPLING_INVCDF
    a = torch.full((3, H, W, 4), -1.0, device="cuda")
    b = torch.full((3, H, W, 4), -1.0, device="cuda")
    fa = torch.empty((3, n), dtype=torch.uint8, device="cuda")
    fbb = torch.empty_like(fa)
    rc.rc_render_importance_views(r.ctx, r.vol, params_for(), cams, mode, 0.05, net[:, :, :32].contiguous(),
                                  net[:, :, 32].contiguous(), 64, 0.02, a, fa)
    rc.rc_render_proposal_sampled(r.ctx, r.vol, params_for(), cams, mode, 0.05, 64, 0.02, b, fbb)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(fa, fbb)
    assert float(b[hit].abs().max()) > 0 and float(b[~hit].abs().max()) == 0.0


# --------------------------------------------------------------------------
# trained on 32 phantoms, evaluated on 8 held out
# --------------------------------------------------------------------------
def psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


def test_trained_proposal_gain(rc):
    import torch
    from paper_1211_5595_gb300 import proposal
    train_vols = synth.proposal_phantoms(W5["train_seeds"])
    eval_vols = synth.proposal_phantoms(W5["eval_seeds"])
    dims, sp = W5["dims"], W5["spacing"]
    tf = synth.tf_table(W5["K"])
    ctx = rc.rc_context_create(0)
    vol = rc.rc_volume_create(ctx, dims, sp, 4095, rc.RC_STORE_F32)
    try:
        rc.rc_tf_set(ctx, tf)
        rc.rc_proposal_load(ctx, rc.pack_proposal_blob(synth.proposal_init_params(61)))
        P = params_for()
        train_cams = [synth.orbit_camera(dims, sp, az, width=512, height=512) for az in W5["azimuths"][::3]]
        feats, tgts = [], []
        for i, v in enumerate(train_vols):
            rc.rc_volume_upload(ctx, vol, v)
            f, t = proposal.collect_rays(ctx, vol, train_cams, P, 4096, seed=i)
            feats.append(f)
            tgts.append(t)
        F, T = torch.cat(feats), torch.cat(tgts)
        curve = proposal.train(ctx, F, T, epochs=30, batch=8192, lr=3e-3, seed=0)
        assert curve[-1] < 0.7 * curve[0], curve
        res = {k: [] for k in ("learned", "occupancy", "profile", "learned_fb", "uniform_chord", "learned_invcdf",
                               "profile_invcdf")}
        fb_rate = []
        for j, v in enumerate(eval_vols):
            rc.rc_volume_upload(ctx, vol, v)
            cam = synth.orbit_camera(dims, sp, 5.0 + 45.0 * j, width=W5["width"], height=W5["height"])
            rc.rc_camera_set(ctx, cam)
            n = cam["width"] * cam["height"]
            plain = torch.empty((cam["height"], cam["width"], 4), device="cuda")
            rc.rc_render(ctx, vol, P, plain)
            never = torch.full((n,), 2.0, device="cuda")
            img = torch.empty_like(plain)
            # 64 samples per ray over: the range the network predicts; the
            # occupancy range alone (a PDF that saturates only at the end: the
            # method without the network); the range of the ray's own 512-sample
            # profile (what a perfect network would predict)
            rc.rc_render_proposal(ctx, vol, P, 64, 2.0, img)
            res["learned"].append(psnr(img, plain))
            rc.rc_render_importance(ctx, vol, P, torch.full((n, 32), 1 / 32, device="cuda"), never, 64, 2.0, img)
            res["occupancy"].append(psnr(img, plain))
            Y = torch.empty((n, 33), device="cuda")
            rc.rc_profiles_generate(ctx, vol, P, Y)
            S = Y[:, :32].sum(dim=1, keepdim=True)
            prof = torch.where(S > 0, Y[:, :32] / S.clamp_min(1e-30), torch.full_like(Y[:, :32], 1 / 32)).contiguous()
            rc.rc_render_importance(ctx, vol, P, prof, never, 64, 2.0, img)
            res["profile"].append(psnr(img, plain))
            st = rc.rc_render_proposal(ctx, vol, P, 64, 0.02, img, stats=True)
            res["learned_fb"].append(psnr(img, plain))
            fb_rate.append(st["fallback_rays"] / max(1, st["rays_hit"]))
            # the same 64 samples placed by other rules: evenly over the whole
            # chord (no PDF, no occupancy: the uniform march the proposal
            # replaces), and by the inverse CDF of the network's PDF or of the
            # ray's own profile mixed with 5% uniform
            img4 = img.view(1, *img.shape)
            rc.rc_render_importance_views(ctx, vol, P, [cam], rc.RC_SAMPLING_INVCDF, 1.0, None, None, 64, 2.0, img4)
            res["uniform_chord"].append(psnr(img, plain))
            rc.rc_render_proposal_sampled(ctx, vol, P, [cam], rc.RC_SAMPLING_INVCDF, 0.05, 64, 2.0, img4)
            res["learned_invcdf"].append(psnr(img, plain))
            rc.rc_render_importance_views(ctx, vol, P, [cam], rc.RC_SAMPLING_INVCDF, 0.05, prof, None, 64, 2.0, img4)
            res["profile_invcdf"].append(psnr(img, plain))
        mean = {k: float(np.mean(v)) for k, v in res.items()}
        print("PSNR vs plain march (dB):", mean, "fallback rate", float(np.mean(fb_rate)), "loss", curve[0], curve[-1])
        assert mean["learned"] > mean["occupancy"] + 1.0
        assert mean["learned"] > mean["uniform_chord"] + 1.0
        assert mean["profile"] >= mean["learned"] - 0.5
        assert mean["learned_fb"] >= mean["learned"]
    finally:
        torch.cuda.synchronize()
        rc.rc_volume_destroy(ctx, vol)
        rc.rc_context_destroy(ctx)


def test_proposal_views_equal_single_views(rc, small):
    """Several views in two launches give the per-view renders exactly."""
    import torch
    ph, tf, r = small
    rc.rc_proposal_load(r.ctx, rc.pack_proposal_blob(synth.proposal_init_params(52)))
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=72, height=56) for az in (15.0, 140.0, 255.0)]
    out = torch.empty((3, 56, 72, 4), device="cuda")
    fb = torch.empty((3, 56 * 72), dtype=torch.uint8, device="cuda")
    st = rc.rc_render_proposal_views(r.ctx, r.vol, params_for(), cams, 64, 0.02, out, fb, stats=True)
    one = torch.empty((56, 72, 4), device="cuda")
    fb1 = torch.empty(56 * 72, dtype=torch.uint8, device="cuda")
    total_fb = 0
    for v, cam in enumerate(cams):
        rc.rc_camera_set(r.ctx, cam)
        s1 = rc.rc_render_proposal(r.ctx, r.vol, params_for(), 64, 0.02, one, fb1, stats=True)
        torch.cuda.synchronize()
        assert torch.equal(out[v], one) and torch.equal(fb[v], fb1)
        total_fb += s1["fallback_rays"]
    assert st["fallback_rays"] == total_fb
    assert st["rays_total"] == 3 * 56 * 72


def test_network_wait_timeout_is_reported(rc, small, monkeypatch):
    """A network launch whose MMA completion never arrives (the test hook
    issues no MMA) gives up after its bounded wait, frees its tensor memory
    and reports RC_ERR_TIMEOUT at the next sync; the context stays usable."""
    import torch
    ph, tf, r = small
    rc.rc_proposal_load(r.ctx, rc.pack_proposal_blob(synth.proposal_init_params(53)))
    cam = synth.orbit_camera(ph.dims, ph.spacing, 60.0, width=64, height=48)
    rc.rc_camera_set(r.ctx, cam)
    out = torch.empty((48, 64, 4), device="cuda")
    monkeypatch.setenv("RC_FAULT_MMA_WAIT", "1")
    rc.rc_render_proposal(r.ctx, r.vol, params_for(), 64, 0.02, out)
    with pytest.raises(rc.RCError) as ei:
        rc.rc_context_sync(r.ctx)
    assert ei.value.status == rc.RC_ERR_TIMEOUT
    monkeypatch.delenv("RC_FAULT_MMA_WAIT")
    rc.rc_context_sync(r.ctx)                       # the flag was cleared
    ref = torch.empty_like(out)
    st = rc.rc_render_proposal(r.ctx, r.vol, params_for(), 64, 0.02, out, stats=True)
    F = torch.empty((64 * 48, 112), device="cuda")
    rc.rc_proposal_features(r.ctx, r.vol, params_for(), F)
    net = torch.empty((64 * 48, 33), device="cuda")
    rc.rc_proposal_forward(r.ctx, F, 64 * 48, net)
    rc.rc_render_importance(r.ctx, r.vol, params_for(), net[:, :32].contiguous(), net[:, 32].contiguous(), 64,
                            0.02, ref)
    rc.rc_context_sync(r.ctx)
    hit = F[:, 3:6].abs().sum(dim=1) > 0
    assert torch.equal(out.view(-1, 4)[hit], ref.view(-1, 4)[hit])
    assert st["rays_total"] == 64 * 48
