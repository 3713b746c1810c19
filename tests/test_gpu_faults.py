"""Failure handling of the C-ABI, injected on the host (no GPU fault): every
device allocation the library makes can be made to fail through
RC_FAULT_ALLOC=n (the n-th allocation after the variable's text last changed;
"1", "01", "001" each re-arm the first one); the calls must
return RC_ERR_OOM, leave earlier state usable, and leak nothing that breaks
later calls. Argument and state errors are status codes too."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    from paper_1211_5595_gb300 import build
    build.build()
    import paper_1211_5595_gb300 as rc
    return rc


def render(rc, ctx, vol, cam):
    import torch
    rc.rc_camera_set(ctx, cam)
    out = torch.empty((cam["height"], cam["width"], 4), device="cuda")
    rc.rc_render(ctx, vol, dict(step_vox=0.5, term=0.99, shade=True, skip=True), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_allocation_failures_are_clean(rc, monkeypatch):
    import torch
    ph = synth.head_phantom((48, 40, 32), (1, 1, 1), seed=3, tumor_radius_vox=4)
    tf = synth.tf_table(256)
    cam = synth.orbit_camera(ph.dims, ph.spacing, 20.0, width=64, height=48)
    ctx = rc.rc_context_create(0)
    try:
        rc.rc_tf_set(ctx, tf)
        # each of the fifteen device allocations of an FP32 rc_volume_create
        # fails in turn (apron bricks, value+gradient bricks, staging copy, and
        # per filter the min, max and mask arrays, the 4^3 min/max grid and the
        # fine mask)
        for n in range(1, 16):
            monkeypatch.setenv("RC_FAULT_ALLOC", str(n))
            with pytest.raises(rc.RCError) as ei:
                rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, rc.RC_STORE_F32)
            assert ei.value.status == rc.RC_ERR_OOM
        # uint16 storage with vmax < 32768 has the same fifteen (its
        # value+gradient bricks hold 8-byte entries)
        for n in range(1, 16):
            monkeypatch.setenv("RC_FAULT_ALLOC", "0" * (n % 2) + str(n))
            with pytest.raises(rc.RCError) as ei:
                rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, rc.RC_STORE_U16)
            assert ei.value.status == rc.RC_ERR_OOM
        monkeypatch.delenv("RC_FAULT_ALLOC")
        vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, 4095, rc.RC_STORE_F32)
        rc.rc_volume_upload(ctx, vol, ph.vol)
        ref = render(rc, ctx, vol, cam)
        assert ref[..., 3].max() > 0.5
        # a larger table whose buffers cannot be allocated keeps the old table
        monkeypatch.setenv("RC_FAULT_ALLOC", "01")
        with pytest.raises(rc.RCError) as ei:
            rc.rc_tf_set(ctx, synth.tf_table(1024))
        assert ei.value.status == rc.RC_ERR_OOM
        monkeypatch.delenv("RC_FAULT_ALLOC")
        assert np.array_equal(render(rc, ctx, vol, cam), ref)
        # the gradient's scratch
        g = torch.ones((48, 64, 4), device="cuda")
        dtf = torch.empty((256, 4), device="cuda")
        P = dict(step_vox=0.5, term=0.99, shade=False, skip=False)
        monkeypatch.setenv("RC_FAULT_ALLOC", "001")
        with pytest.raises(rc.RCError) as ei:
            rc.rc_render_backward(ctx, vol, P, g, dtf)
        assert ei.value.status == rc.RC_ERR_OOM
        monkeypatch.delenv("RC_FAULT_ALLOC")
        rc.rc_render_backward(ctx, vol, P, g, dtf)
        torch.cuda.synchronize()
        assert torch.isfinite(dtf).all() and dtf.abs().sum() > 0
        # the network: a failed load leaves no network behind
        monkeypatch.setenv("RC_FAULT_ALLOC", "0002")
        with pytest.raises(rc.RCError) as ei:
            rc.rc_proposal_load(ctx, rc.pack_proposal_blob(synth.proposal_init_params(1)))
        assert ei.value.status == rc.RC_ERR_OOM
        monkeypatch.delenv("RC_FAULT_ALLOC")
        out = torch.empty((48, 64, 4), device="cuda")
        with pytest.raises(rc.RCError) as ei:
            rc.rc_render_proposal(ctx, vol, P, 64, 0.02, out)
        assert ei.value.status == rc.RC_ERR_STATE
        assert np.array_equal(render(rc, ctx, vol, cam), ref)
        # the pair bricks, allocated by the first B-spline render: a failure
        # refuses that render and the next one allocates them
        Pb = dict(step_vox=0.5, term=0.99, shade=True, skip=True, filter=rc.RC_FILTER_BSPLINE)
        monkeypatch.setenv("RC_FAULT_ALLOC", "00001")
        with pytest.raises(rc.RCError) as ei:
            rc.rc_render(ctx, vol, Pb, out)
        assert ei.value.status == rc.RC_ERR_OOM
        monkeypatch.delenv("RC_FAULT_ALLOC")
        rc.rc_render(ctx, vol, Pb, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all() and float(out[..., 3].max()) > 0.5
        assert np.array_equal(render(rc, ctx, vol, cam), ref)
        rc.rc_volume_destroy(ctx, vol)
    finally:
        monkeypatch.delenv("RC_FAULT_ALLOC", raising=False)
        torch.cuda.synchronize()
        rc.rc_context_destroy(ctx)


def test_argument_and_state_errors(rc):
    import torch
    ctx = rc.rc_context_create(0)
    try:
        for dims, sp in (((1, 8, 8), (1, 1, 1)), ((8, 8, 8), (0, 1, 1)), ((8, 8, 8), (1, float("nan"), 1))):
            with pytest.raises(rc.RCError) as ei:
                rc.rc_volume_create(ctx, dims, sp)
            assert ei.value.status == rc.RC_ERR_INVALID_ARG
        vol = rc.rc_volume_create(ctx, (8, 8, 8), (1, 1, 1))
        out = torch.empty((4, 4, 4), device="cuda")
        P = dict(step_vox=0.5, term=0.99)
        with pytest.raises(rc.RCError) as ei:
            rc.rc_render(ctx, vol, P, out)            # no data, no table, no camera
        assert ei.value.status == rc.RC_ERR_STATE
        with pytest.raises(rc.RCError) as ei:
            rc.rc_volume_upload(ctx, vol, np.zeros(7, np.uint16))
        assert ei.value.status == rc.RC_ERR_INVALID_ARG and "voxels" in str(ei.value)
        rc.rc_volume_upload(ctx, vol, np.full(512, 3000, np.uint16))
        with pytest.raises(rc.RCError) as ei:
            rc.rc_tf_set(ctx, np.full((4, 4), 1.5, np.float32))
        assert ei.value.status == rc.RC_ERR_INVALID_ARG
        rc.rc_tf_set(ctx, synth.tf_table(256))
        with pytest.raises(rc.RCError):
            rc.rc_camera_set(ctx, dict(eye=(0, 0, 0), target=(0, 0, 0), up=(0, 0, 1), fovy_deg=30,
                                       width=4, height=4))
        rc.rc_camera_set(ctx, synth.orbit_camera((8, 8, 8), (1, 1, 1), 0.0, width=4, height=4))
        for bad in (dict(step_vox=0.0), dict(term=1.5), dict(func=9), dict(step_vox=float("inf"))):
            with pytest.raises(rc.RCError) as ei:
                rc.rc_render(ctx, vol, dict(P, **bad), out)
            assert ei.value.status == rc.RC_ERR_INVALID_ARG
        rc.rc_render(ctx, vol, P, out)
        torch.cuda.synchronize()
        assert out[..., 3].max() > 0.5
        with pytest.raises(rc.RCError) as ei:
            rc.rc_context_destroy(ctx)                 # a volume is still alive
        assert ei.value.status == rc.RC_ERR_STATE
        rc.rc_volume_destroy(ctx, vol)
    finally:
        torch.cuda.synchronize()
        rc.rc_context_destroy(ctx)


def test_read_probes(rc):
    """The read-bandwidth probes of librc_probe.so (include/rc_probe.h) run on
    the given stream, report launch errors as cudaError_t values and check
    their arguments before any launch; the L1 probe's byte count is CTAs x
    reps x buffer bytes and its rate is far above the L2 probe's."""
    import ctypes as C

    import torch
    from paper_1211_5595_gb300 import build
    L = C.CDLL(build.build_probe())
    for f in ("rc_probe_read_l1", "rc_probe_read_l2"):
        getattr(L, f).argtypes = [C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]
        getattr(L, f).restype = C.c_int
    L.rc_probe_l1_bytes.argtypes = [C.c_size_t, C.c_int]
    L.rc_probe_l1_bytes.restype = C.c_size_t
    s = torch.cuda.current_stream()
    small = torch.ones(8 << 10, device="cuda")                 # 32 KB
    big = torch.ones(24 << 20, device="cuda")                  # 96 MB
    rates = {}
    for name, buf, reps in (("l1", small, 200), ("l2", big, 4)):
        fn = getattr(L, "rc_probe_read_" + name)
        nbytes = buf.numel() * 4
        assert fn(buf.data_ptr(), nbytes, reps, s.cuda_stream) == 0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(s)
        assert fn(buf.data_ptr(), nbytes, reps, s.cuda_stream) == 0
        ev[1].record(s)
        torch.cuda.synchronize()
        moved = L.rc_probe_l1_bytes(nbytes, reps) if name == "l1" else nbytes * reps
        rates[name] = moved / (ev[0].elapsed_time(ev[1]) / 1e3)
        assert fn(buf.data_ptr() + 4, nbytes - 16, reps, s.cuda_stream) == 1      # not 16-byte aligned
        assert fn(buf.data_ptr(), nbytes, 0, s.cuda_stream) == 1
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert L.rc_probe_l1_bytes(32 << 10, 3) == sms * 4 * 3 * (32 << 10)
    assert L.rc_probe_read_l1(big.data_ptr(), 1 << 20, 1, s.cuda_stream) == 1    # above the 64 KB limit
    assert rates["l1"] > 2 * rates["l2"] > 0
