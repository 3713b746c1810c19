"""Small renders of every kernel family through the C-ABI, for comparing the
release library with the debug build (RC_DEBUG=1 in the environment selects
librc_debug.so, whose kernels check every brick and table index).

    python tests/debug_scenarios.py OUT.npz [--poison]

Writes one array per scenario to OUT.npz. Every call is followed by
rc_context_sync, so a failed device index check raises there. --poison sets
the debug build's test hook (every brick index moved out of range: each check
fires and replaces the index by an in-range one) and expects RC_ERR_CUDA from
the first synchronising call, then checks that the context still renders
correctly once the hook is cleared.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402


def main(out_path, poison):
    import torch

    import paper_1211_5595_gb300 as rc

    ph = synth.head_phantom((70, 58, 41), (1.0, 0.9, 1.3), seed=35, tumor_radius_vox=4)
    tf = synth.tf_table(256)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 200.0, width=75, height=53)
    H, W = cam["height"], cam["width"]
    ctx = rc.rc_context_create(0)
    vols = {}
    res = {}
    try:
        for name, st in (("f32", rc.RC_STORE_F32), ("f16", rc.RC_STORE_F16), ("u16", rc.RC_STORE_U16)):
            vols[name] = rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, st)
            rc.rc_volume_upload(ctx, vols[name], ph.vol)
        rc.rc_tf_set(ctx, tf)
        rc.rc_camera_set(ctx, cam)
        img = torch.empty((H, W, 4), device="cuda")
        P = dict(step_vox=0.5, term=0.99, shade=True, skip=True)
        if poison:
            os.environ["RC_DEBUG_POISON"] = "1"
            rc.rc_render(ctx, vols["f32"], P, img)
            try:
                rc.rc_context_sync(ctx)
            except rc.RCError as e:
                assert e.status == rc.RC_ERR_CUDA and "index check" in str(e), str(e)
                res["poison_caught"] = np.array(1)
            else:
                raise AssertionError("the poisoned render reported no index failure")
            del os.environ["RC_DEBUG_POISON"]
            rc.rc_context_sync(ctx)                 # the error word was cleared
        # the compositing march in every storage and form
        for name in ("f32", "f16", "u16"):
            rc.rc_tf_set(ctx, tf, name != "f32")
            for form, kw in (("shaded", {}), ("plain", {"shade": False}), ("bspline", {"filter": 1})):
                rc.rc_render(ctx, vols[name], {**P, **kw}, img)
                rc.rc_context_sync(ctx)
                res[f"{name}_{form}"] = img.cpu().numpy()
        rc.rc_tf_set(ctx, tf)
        # the other ray functions
        for fname, f in (("mip", rc.RC_FUNC_MIP), ("iso", rc.RC_FUNC_ISO), ("threshold", rc.RC_FUNC_THRESHOLD)):
            rc.rc_render(ctx, vols["f32"], {**P, "func": f, "iso": 1500.0}, img)
            rc.rc_context_sync(ctx)
            res[fname] = img.cpu().numpy()
        # the table gradient, 1-D and 2-D
        g = torch.randn((H, W, 4), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
        dtf = torch.empty((256, 4), device="cuda")
        Pg = dict(step_vox=0.5, term=0.99, shade=True, skip=False)
        rc.rc_render_backward(ctx, vols["f32"], Pg, g, dtf)
        rc.rc_context_sync(ctx)
        res["grad_1d"] = dtf.cpu().numpy()
        tab2 = synth.tf2d_table(256, 16, 1200.0)
        rc.rc_tf2d_set(ctx, tab2, 1200.0)
        rc.rc_render(ctx, vols["f32"], P, img)
        rc.rc_context_sync(ctx)
        res["tf2d"] = img.cpu().numpy()
        dtf2 = torch.empty((16, 256, 4), device="cuda")
        rc.rc_render_backward(ctx, vols["f32"], Pg, g, dtf2)
        rc.rc_context_sync(ctx)
        res["grad_2d"] = dtf2.cpu().numpy()
        rc.rc_tf_set(ctx, tf)
        # the learned proposal: features, network, both importance readings
        rc.rc_proposal_load(ctx, rc.pack_proposal_blob(synth.proposal_init_params(5)))
        F = torch.empty((H * W, 112), device="cuda")
        rc.rc_proposal_features(ctx, vols["f32"], P, F)
        rc.rc_context_sync(ctx)
        res["features"] = F.cpu().numpy()
        rc.rc_render_proposal(ctx, vols["f32"], P, 64, 0.02, img)
        rc.rc_context_sync(ctx)
        res["proposal_range"] = img.cpu().numpy()
        img1 = img.view(1, H, W, 4)
        rc.rc_render_proposal_sampled(ctx, vols["f32"], P, [cam], rc.RC_SAMPLING_INVCDF, 0.05, 64, 0.02, img1)
        rc.rc_context_sync(ctx)
        res["proposal_invcdf"] = img.cpu().numpy()
    finally:
        torch.cuda.synchronize()
        for v in vols.values():
            rc.rc_volume_destroy(ctx, v)
        rc.rc_context_destroy(ctx)
    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1], "--poison" in sys.argv[2:])
