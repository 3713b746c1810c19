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
        # tables beyond the static scratch are refused with a clear error
        rc.rc_tf_set(ctx, synth.tf_table(2048))
        with pytest.raises(rc.RCError) as ei:
            rc.rc_render_backward_noalloc(ctx, vol, params, ups[0], torch.empty((2048, 4), device="cuda"))
        assert ei.value.status == rc.RC_ERR_UNSUPPORTED and "1024" in str(ei.value)
    finally:
        torch.cuda.synchronize()
        rc.rc_volume_destroy(ctx, vol)
        rc.rc_context_destroy(ctx)
