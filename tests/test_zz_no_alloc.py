"""rc_render_backward_noalloc: the transfer-function gradient for callers that
cannot allocate device memory while they run (an application whose device
memory is all handed out up front by its own allocator, or a frame loop that
must not stall on a cudaMalloc). Its scratch is a fixed file-scope device array,
so it must give the same gradient as rc_render_backward, call after call, with
the array cleared between calls.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_gradient_matches_allocating_entry_point():
    import torch

    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc

    ph = synth.head_phantom((96, 80, 64), (1.0, 1.0, 1.5), seed=41, tumor_radius_vox=5)
    tf = synth.noise_tf(256, 8, alpha_max=0.1)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 35.0, width=160, height=120)
    params = rc.RenderParams(step_vox=0.5, term=0.99, shade=True, skip=False)
    ctx = rc.rc_context_create(0)
    vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, rc.RC_STORE_F32)
    try:
        rc.rc_volume_upload(ctx, vol, ph.vol)
        rc.rc_tf_set(ctx, tf)
        rc.rc_camera_set(ctx, cam)
        gen = torch.Generator("cuda").manual_seed(123)
        ups = [torch.randn((120, 160, 4), device="cuda", generator=gen) for _ in range(2)]
        refs = []
        for g in ups:
            ref = torch.empty((256, 4), device="cuda")
            rc.rc_render_backward(ctx, vol, params, g, ref)
            refs.append(ref)
        torch.cuda.synchronize()
        # two calls in a row, different upstream gradients: the shared scratch
        # keeps the last call's contents, so each call must clear it
        for g, ref in zip(ups, refs):
            out = torch.full((256, 4), float("nan"), device="cuda")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            rc.rc_render_backward_noalloc(ctx, vol, params, g, out)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0      # nothing allocated
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.isfinite(a).all()
            # the relative tolerance of the other gradient tests; the fixed-point
            # sums make the two entry points agree bit for bit in practice
            assert np.abs(a - b).max() <= 2e-4 * np.abs(b).max()
            assert np.abs(b).max() > 0
        # the largest table the static scratch holds: 1024 entries (its
        # |dL/dI| maximum sits right after the 4 x 1024 accumulators)
        tf_big = synth.noise_tf(1024, 9, alpha_max=0.1)
        rc.rc_tf_set(ctx, tf_big)
        for g in ups:
            ref = torch.empty((1024, 4), device="cuda")
            rc.rc_render_backward(ctx, vol, params, g, ref)
            out = torch.full((1024, 4), float("nan"), device="cuda")
            rc.rc_render_backward_noalloc(ctx, vol, params, g, out)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.isfinite(a).all() and np.abs(b).max() > 0
            assert np.abs(a - b).max() <= 2e-4 * np.abs(b).max()
        # tables beyond the static scratch are refused with a clear error,
        # from the first entry past the limit
        for n in (1025, 2048):
            rc.rc_tf_set(ctx, synth.tf_table(n))
            with pytest.raises(rc.RCError) as ei:
                rc.rc_render_backward_noalloc(ctx, vol, params, ups[0], torch.empty((n, 4), device="cuda"))
            assert ei.value.status == rc.RC_ERR_UNSUPPORTED and "1024" in str(ei.value)
    finally:
        torch.cuda.synchronize()
        rc.rc_volume_destroy(ctx, vol)
        rc.rc_context_destroy(ctx)


@pytest.mark.parametrize("storage,shade,bspline", [("F32", False, True), ("F32", True, True),
                                                   ("F16", True, False), ("F16", False, True)])
def test_noalloc_gradient_on_a_fresh_volume(orc, storage, shade, bspline):
    """A volume whose pair bricks were never built (no render has run on it)
    is read from its apron bricks by the entry point that allocates nothing:
    the gradient matches the FP64 oracle's and the allocating entry point's
    (which builds the pairs). After new data the stale pairs are rebuilt in
    place, again without allocating, and the three still agree."""
    import torch

    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc

    ph = synth.head_phantom((58, 50, 40), (1.0, 1.1, 1.4), seed=43, tumor_radius_vox=4)
    ph2 = synth.head_phantom((58, 50, 40), (1.0, 1.1, 1.4), seed=44, tumor_radius_vox=5)
    tf = synth.noise_tf(256, 11, alpha_max=0.1)
    H, Wd = 40, 48
    cam = synth.orbit_camera(ph.dims, ph.spacing, 70.0, width=Wd, height=H)
    filt = rc.RC_FILTER_BSPLINE if bspline else rc.RC_FILTER_TRILINEAR
    params = rc.RenderParams(step_vox=0.5, term=0.99, shade=shade, skip=False, filter=filt)
    st = getattr(rc, "RC_STORE_" + storage)
    ctx = rc.rc_context_create(0)
    # a second volume runs the same gradient through the allocating entry point
    # first, so that the kernels' device code is loaded (lazy module loading
    # may take device memory) before the allocation check below
    warm = rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, st)
    vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, st)
    try:
        rc.rc_tf_set(ctx, tf)
        rc.rc_camera_set(ctx, cam)
        rc.rc_volume_upload(ctx, warm, ph.vol)
        rc.rc_render_backward(ctx, warm, params, torch.ones((H, Wd, 4), device="cuda"),
                              torch.empty((256, 4), device="cuda"))
        for data in (ph.vol, ph2.vol):
            rc.rc_volume_upload(ctx, vol, data)
            sc = orc.Scene(data, ph.spacing, tf, cam, step=0.5, term=0.99, shade=shade,
                           filter=orc.BSPLINE if bspline else orc.TRILINEAR, value_mode=int(storage == "F16"))
            fwd = orc.render(sc)
            keep = np.flatnonzero(~fwd["tie"].reshape(-1))
            g = np.zeros((H * Wd, 4))
            g[keep] = np.random.default_rng(7).normal(size=(len(keep), 4))
            og, _ = orc.render_grad(sc, g[keep], pixels=keep)
            gd = torch.from_numpy(g.astype(np.float32)).cuda()
            # first the entry point that allocates nothing: on the first data the
            # volume has no pair bricks; on the second they are stale
            out = torch.full((256, 4), float("nan"), device="cuda")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            rc.rc_render_backward_noalloc(ctx, vol, params, gd, out)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            ref = torch.empty((256, 4), device="cuda")
            rc.rc_render_backward(ctx, vol, params, gd, ref)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
            scale = np.abs(og).max()
            assert scale > 0 and np.isfinite(a).all()
            assert np.abs(a - og).max() <= 2e-4 * scale, np.abs(a - og).max() / scale
            assert np.abs(b - og).max() <= 2e-4 * scale
            assert np.abs(a - b).max() <= 2e-4 * scale
    finally:
        torch.cuda.synchronize()
        rc.rc_volume_destroy(ctx, vol)
        rc.rc_volume_destroy(ctx, warm)
        rc.rc_context_destroy(ctx)
