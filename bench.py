"""Throughput of the shaded raycast of a 256x256x180 uint16 head phantom at
1024 x 1024 over a 36-view orbit (FP32 storage, step 0.5 voxel, Blinn-Phong,
16^3 min/max brick grid for empty-space skipping, early termination at 0.99).

One step = one pass of the whole hot path over the resident phantom: re-layout
into apron bricks and value+gradient bricks and the min/max grid from the
device copy of the codes, occupancy mask for the transfer function, then the
36 views rendered in one launch. Metric: dense-equivalent
Gsamples/s (samples of the plain march up to termination, skipped ones
included) and ms/frame.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own orbit on its own GPU (weak scaling,
no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "shaded_256x256x180"
METRIC = "Gsamples/s (dense-equivalent), 1024^2 of 256x256x180 u16, shaded, 36-view orbit"
BYTES_PER_SAMPLE = 128          # 32 distinct FP32 voxels per shaded sample (8 value+gradient float4)
TF2_GMAX = 1200.0               # gradient magnitude (codes per mm) of the 2-D table's last row
L2_FLUSH_BYTES = 256 << 20      # > 129 MB L2


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the files composite_kernel<F32, shaded> is compiled from
# the files compiled into the march kernel (the public header only declares
# the C API around it; its constants reach the kernel through rc_internal.h)
MARCH_SOURCES = ("paper_1211_5595_gb300/csrc/rc_internal.h", "paper_1211_5595_gb300/csrc/rc_device.cuh",
                 "paper_1211_5595_gb300/csrc/rc_march.cuh", "paper_1211_5595_gb300/csrc/rc_march.cu")


def strip_comments(src):
    """C/C++ source without comments and blank lines (string literals kept)."""
    src = re.sub(r"//[^\n]*|/\*.*?\*/", "", src, flags=re.S)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_sources_hash():
    """Hash of the march kernel's code: comment edits do not change it."""
    h = hashlib.sha256()
    for f in MARCH_SOURCES:
        h.update(strip_comments(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


def profiled_counters():
    """Per-launch counters of the march from the committed ncu summary
    (DRAM bytes, L2-to-L1 bytes, warp instructions, L1 data-pipe use), if it
    was captured on the current kernel sources (else an empty dict)."""
    path = os.path.join(ROOT, "profiles", "march_shaded_256x256x180.md")
    try:
        kv = {}
        for line in open(path):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                kv[k.strip()] = (v.split() or [""])[0]
        if kv.get("sources_sha256_16") != kernel_sources_hash():
            return {}
        return {k: float(kv[k]) for k in ("dram_bytes_per_launch", "l2_to_l1_bytes_per_launch",
                                          "warp_instructions_per_launch", "l1_data_pipe_pct") if k in kv}
    except Exception:
        return {}


def profiled_traffic():
    return profiled_counters().get("dram_bytes_per_launch")


def probe_lib():
    """librc_probe.so (include/rc_probe.h): the read-bandwidth probes."""
    import ctypes as C
    from paper_1211_5595_gb300 import build
    L = C.CDLL(build.build_probe())
    for f in ("rc_probe_read_l1", "rc_probe_read_l2"):
        getattr(L, f).argtypes = [C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]
        getattr(L, f).restype = C.c_int
    L.rc_probe_l1_bytes.argtypes = [C.c_size_t, C.c_int]
    L.rc_probe_l1_bytes.restype = C.c_size_t
    return L


def _probe_best_ms(fn, stream, tries=5):
    import torch
    for _ in range(2):
        assert fn() == 0
    best = float("inf")
    for _ in range(tries):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        assert fn() == 0
        ev[1].record(stream)
        torch.cuda.synchronize()
        best = min(best, ev[0].elapsed_time(ev[1]))
    return best


def l2_read_peak(stream, reps=40):
    """L2 read bandwidth: the probe reads a 96 MB buffer (below the 129 MB L2)
    reps times in one launch with loads that bypass L1; best of 5, CUDA
    events; bytes read / time (GB/s)."""
    import torch
    L = probe_lib()
    buf = torch.ones(24 << 20, device="cuda", dtype=torch.float32)
    nbytes = buf.numel() * 4
    ms = _probe_best_ms(lambda: L.rc_probe_read_l2(buf.data_ptr(), nbytes, reps, stream.cuda_stream), stream)
    return reps * nbytes / (ms / 1e3) / 1e9


def l1_read_peak(stream, reps=2000, nbytes=32 << 10):
    """L1 load bandwidth of the whole GPU: every CTA (4 per SM) reads the same
    32 KB buffer reps times with 16-byte read-only loads (the march's load
    form), coalesced 512 bytes per warp; best of 5, CUDA events; GB/s."""
    import torch
    L = probe_lib()
    buf = torch.ones(nbytes // 4, device="cuda", dtype=torch.float32)
    ms = _probe_best_ms(lambda: L.rc_probe_read_l1(buf.data_ptr(), nbytes, reps, stream.cuda_stream), stream)
    return L.rc_probe_l1_bytes(nbytes, reps) / (ms / 1e3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, first=0, last=None):
        """Median SM clock, the largest maximum clock and the throttle reasons
        seen in samples[first:last]."""
        samples = self.samples[first:last]
        if not samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in samples for i in range(4) if s[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(samples)}


def max_over_ranks(value, world, device):
    """The largest value over all ranks (every rank gets it)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank_step, steps, max_total_ms):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank_step * steps / (max_total_ms / 1e3)


def setup_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def params(w, skip=True):
    import paper_1211_5595_gb300 as rc
    return rc.RenderParams(step_vox=w["step"], term=w["term"], shade=w["shade"], skip=skip)


def cameras(ph, w):
    return [synth.orbit_camera(ph.dims, ph.spacing, az, width=w["width"], height=w["height"])
            for az in w["azimuths"]]


def cpu_oracle_sample(ph, tf, w, cams, budget_s, pixels_per_view=None):
    """Times the FP64 oracle on host cores over whole views (or seeded pixel
    subsets) until budget_s of work is done. Returns (Gsamples/s, cores, desc)."""
    import oracle
    oracle.build()
    cores = oracle.default_threads()
    samples = 0
    views = 0
    t0 = time.perf_counter()
    for i, cam in enumerate(cams):
        sc = oracle.Scene(ph.vol, ph.spacing, tf, cam, step=w["step"], term=w["term"], shade=w["shade"])
        pix = None
        if pixels_per_view:
            pix = synth.sample_pixels(w["width"], w["height"], pixels_per_view, seed=9000 + i)
        r = oracle.render(sc, pixels=pix, nthreads=cores)
        samples += int(r["nsamp"].sum())
        views += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    what = f"{pixels_per_view} seeded pixels of each of" if pixels_per_view else "full 1024^2 frames of"
    return samples / dt / 1e9, cores, f"{what} {views} view(s), {samples} samples, {dt:.1f} s"


def cpu_model():
    """The host CPU's name from /proc/cpuinfo (x86 'model name', else the Arm
    implementer / part codes), or the machine type."""
    import platform
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model Name"):
        m = re.search(rf"^{key}\s*:\s*(.+)$", info, re.M)
        if m:
            return m.group(1).strip()
    imp = re.search(r"^CPU implementer\s*:\s*(\S+)", info, re.M)
    part = re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
    if imp and part:
        return f"{platform.machine()} (implementer {imp.group(1)}, part {part.group(1)})"
    return platform.machine()


def cpu_oracle_one_core(ph, tf, w, cam, budget_s=3.0, npix=4096):
    """The oracle on one host thread: seeded pixel sets of one view until
    budget_s of work is done. Returns (Gsamples/s, desc)."""
    import oracle
    sc = oracle.Scene(ph.vol, ph.spacing, tf, cam, step=w["step"], term=w["term"], shade=w["shade"])
    samples, sets = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        pix = synth.sample_pixels(w["width"], w["height"], npix, seed=9500 + sets)
        samples += int(oracle.render(sc, pixels=pix, nthreads=1)["nsamp"].sum())
        sets += 1
    dt = time.perf_counter() - t0
    return samples / dt / 1e9, f"{sets} x {npix} seeded pixels of one view, {samples} samples, {dt:.1f} s"


def filter_forms(rc, ctx, vol, w, P, cam_structs, outs, ref_imgs, flush, stream, hbm_peak):
    """The reconstruction / classification variants on the FP32 volume, every
    view in one launch: cubic B-spline (64 distinct FP32 voxels = 256 B per
    evaluated sample, value and analytic gradient from the same footprint),
    the 2-D value x gradient-magnitude table (trilinear, 128 B per sample plus
    four table entries from L1/L2), and both. Each form's own dense and
    evaluated counts; PSNR against the trilinear 1-D images is a difference
    by design (another filter, another table), reported for context."""
    import torch
    tab2 = synth.tf2d_table(w["K"], 32, TF2_GMAX)
    out = {}
    for name, filt, two_d in (("bspline", rc.RC_FILTER_BSPLINE, False), ("tf2d", rc.RC_FILTER_TRILINEAR, True),
                              ("bspline_tf2d", rc.RC_FILTER_BSPLINE, True)):
        if two_d:
            rc.rc_tf2d_set(ctx, tab2, TF2_GMAX)
        else:
            rc.rc_tf_set(ctx, synth.tf_table(w["K"]))
        P2 = rc.RenderParams(**{**P.__dict__, "filter": filt})
        st = rc.rc_render_views(ctx, vol, P2, cam_structs, outs, stats=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        for rep in range(3):
            ev[rep][0].record(stream)
            rc.rc_render_views(ctx, vol, P2, cam_structs, outs)
            ev[rep][1].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        launch_ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        n = len(cam_structs)
        bps = 256 if filt == rc.RC_FILTER_BSPLINE else BYTES_PER_SAMPLE
        achieved = st["evaluated_samples"] * bps / (launch_ms / 1e3) / 1e9
        mse = ((outs - ref_imgs) ** 2).mean(dim=(1, 2, 3))
        out[name] = {"ms_per_frame_median": launch_ms / n,
                     "gsamples_s": st["dense_samples"] / (launch_ms / 1e3) / 1e9,
                     "dense_samples": st["dense_samples"], "evaluated_samples": st["evaluated_samples"],
                     "bytes_per_evaluated_sample": bps, "achieved_gbs": achieved,
                     "frac_of_hbm": achieved / hbm_peak,
                     "psnr_db_min_vs_trilinear_1d": float((10 * torch.log10(1.0 / mse.clamp_min(1e-30))).min())}
    return out


def precision_form(rc, ctx, flush, stream, hbm_peak):
    """The precision configuration: 512x512x256 phantom, 2048^2 image, step
    0.25, shaded, 1024-entry table; FP32 storage (FP32 table) against FP16
    (offset-normalised) and uint16 storage with the FP16 table. One view; ms
    per frame, dense-equivalent Gsamples/s, evaluated samples, PSNR against the
    FP32 image. Also returns, for the error against the FP64 oracle (computed
    in the CPU-baseline leg), each form's colours at the 4096 seeded pixels of
    the 2048^2 frame and its full 512^2 frame."""
    import torch
    wp = synth.WORKLOADS["precision_512x512x256"]
    ph = synth.workload_phantom("precision_512x512x256")
    tf = synth.tf_table(wp["K"])
    cam = synth.orbit_camera(ph.dims, ph.spacing, wp["azimuths"][0], width=wp["width"], height=wp["height"])
    cs = synth.orbit_camera(ph.dims, ph.spacing, wp["azimuths"][0], width=wp["small_width"], height=wp["small_width"])
    pix = synth.sample_pixels(wp["width"], wp["height"], wp["n_rays"], seed=wp["ray_seed"])
    P = rc.RenderParams(step_vox=wp["step"], term=wp["term"], shade=wp["shade"], skip=True)
    img = torch.empty((wp["height"], wp["width"], 4), device="cuda")
    small = torch.empty((wp["small_width"], wp["small_width"], 4), device="cuda")
    ref = None
    capture = {"ph": ph, "tf": tf, "cam": cam, "cam_small": cs, "pix": pix, "w": wp, "images": {}}
    out = {"workload": "precision_512x512x256", "image": "2048x2048", "step_vox": wp["step"], "table_entries": wp["K"]}
    for name, storage, fp16 in (("f32", rc.RC_STORE_F32, False), ("f16", rc.RC_STORE_F16, True),
                                ("u16", rc.RC_STORE_U16, True)):
        vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, storage)
        rc.rc_volume_upload(ctx, vol, ph.vol)
        rc.rc_tf_set(ctx, tf, fp16)
        rc.rc_camera_set(ctx, cam)
        st = rc.rc_render(ctx, vol, P, img, stats=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        for e in ev:
            e[0].record(stream)
            rc.rc_render(ctx, vol, P, img)
            e[1].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        res = {"ms_per_frame": ms, "gsamples_s": st["dense_samples"] / (ms / 1e3) / 1e9,
               "dense_samples": st["dense_samples"], "evaluated_samples": st["evaluated_samples"]}
        if ref is None:
            ref = img.clone()
        else:
            mse = float(((img - ref) ** 2).mean())
            res["psnr_db_vs_f32"] = float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)
            res["speedup_vs_f32"] = out["f32"]["ms_per_frame"] / ms
        rc.rc_camera_set(ctx, cs)
        rc.rc_render(ctx, vol, P, small)
        torch.cuda.synchronize()
        capture["images"][name] = (img.view(-1, 4)[torch.from_numpy(pix).long().cuda()].cpu().numpy(),
                                   small.cpu().numpy())
        out[name] = res
        rc.rc_volume_destroy(ctx, vol)
    return out, capture


def precision_frames(rc, ctx, stream):
    """One 2048^2 frame of the precision workload per storage form (FP32 with
    the FP32 table, FP16 and uint16 with the FP16 table), each rendered twice
    (the second launch timed): exactly two march launches per form, in that
    order, for a profiler to capture."""
    import torch
    wp = synth.WORKLOADS["precision_512x512x256"]
    ph = synth.workload_phantom("precision_512x512x256")
    tf = synth.tf_table(wp["K"])
    cam = synth.orbit_camera(ph.dims, ph.spacing, wp["azimuths"][0], width=wp["width"], height=wp["height"])
    P = rc.RenderParams(step_vox=wp["step"], term=wp["term"], shade=wp["shade"], skip=True)
    img = torch.empty((wp["height"], wp["width"], 4), device="cuda")
    out = {}
    for name, storage, fp16 in (("f32", rc.RC_STORE_F32, False), ("f16", rc.RC_STORE_F16, True),
                                ("u16", rc.RC_STORE_U16, True)):
        vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, storage)
        rc.rc_volume_upload(ctx, vol, ph.vol)
        rc.rc_tf_set(ctx, tf, fp16)
        rc.rc_camera_set(ctx, cam)
        rc.rc_render(ctx, vol, P, img)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        rc.rc_render(ctx, vol, P, img)
        ev[1].record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms_per_frame": ev[0].elapsed_time(ev[1])}
        rc.rc_volume_destroy(ctx, vol)
    return out


def staged_form(rc, ctx, stream, flush, cams, reps=3):
    """The bench march (FP32, shaded, every view of `cams` in one launch)
    against its brick-staged variant (RC_MARCH_STAGED=1: each CTA stages the
    value+gradient brick its rays need next in shared memory): median launch
    time of each and whether the images are identical. With two views and
    one repetition it is the small case a profiler captures (two launches of
    each kernel, the first untimed)."""
    import torch
    w = synth.WORKLOADS[WORKLOAD]
    ph = synth.workload_phantom(WORKLOAD)
    vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, rc.RC_STORE_F32)
    rc.rc_volume_upload(ctx, vol, ph.vol)
    rc.rc_tf_set(ctx, synth.tf_table(w["K"]))
    cam_structs = [rc.make_camera(c) for c in cams]
    P = params(w)
    imgs = {}
    out = {"views": len(cams)}
    for name in ("cached", "staged"):
        if name == "staged":
            os.environ["RC_MARCH_STAGED"] = "1"
        img = torch.empty((len(cams), w["height"], w["width"], 4), device="cuda")
        rc.rc_render_views(ctx, vol, P, cam_structs, img)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            rc.rc_render_views(ctx, vol, P, cam_structs, img)
            b.record(stream)
            flush.zero_()
        rc.rc_context_sync(ctx)
        os.environ.pop("RC_MARCH_STAGED", None)
        out[name + "_ms_per_frame"] = statistics.median(x.elapsed_time(y) for x, y in ev) / len(cams)
        imgs[name] = img
    out["identical"] = bool(torch.equal(imgs["cached"], imgs["staged"]))
    out["staged_over_cached"] = out["staged_ms_per_frame"] / out["cached_ms_per_frame"]
    rc.rc_volume_destroy(ctx, vol)
    return out


def proposal_frames(rc, ctx, stream, cams, reps=2):
    """The learned-proposal render of the bench workload with a seeded
    (untrained) network: every view of `cams` in one launch pair (the camera-ray
    network kernel, then the importance march, 64 samples per ray, no
    fallback), reps times; median ms per frame. The small case a profiler
    captures."""
    import torch
    w = synth.WORKLOADS[WORKLOAD]
    ph = synth.workload_phantom(WORKLOAD)
    vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, rc.RC_STORE_F32)
    rc.rc_volume_upload(ctx, vol, ph.vol)
    rc.rc_tf_set(ctx, synth.tf_table(w["K"]))
    rc.rc_proposal_load(ctx, rc.pack_proposal_blob(synth.proposal_init_params(61)))
    cam_structs = [rc.make_camera(c) for c in cams]
    img = torch.empty((len(cams), w["height"], w["width"], 4), device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        rc.rc_render_proposal_views(ctx, vol, params(w), cam_structs, 64, 2.0, img)
        b.record(stream)
    rc.rc_context_sync(ctx)
    rc.rc_volume_destroy(ctx, vol)
    return {"views": len(cams), "ms_per_frame": statistics.median(x.elapsed_time(y) for x, y in ev) / len(cams)}


def oracle_errors(gpu, o):
    """Max-abs per channel of GPU colours against the oracle's (a ray whose
    stop decision is a termination tie takes the nearer branch) and the PSNR
    over the four channels (peak 1)."""
    g = gpu.reshape(-1, 4).astype(np.float64)
    a, b, tie = o["rgba"].reshape(-1, 4), o["alt"].reshape(-1, 4), o["tie"].reshape(-1)
    d1, d2 = np.abs(g - a).max(axis=1), np.abs(g - b).max(axis=1)
    use_b = tie & (d2 < d1)
    d = np.where(use_b, d2, d1)
    ref = np.where(use_b[:, None], b, a)
    mse = float(np.mean((g - ref) ** 2))
    return {"max_abs": float(d.max()), "psnr_db": float("inf") if mse == 0 else 10 * np.log10(1.0 / mse),
            "pixels": int(len(d)), "pixels_above_4e-3": int((d > 4e-3).sum()), "tie_rays": int(tie.sum())}


def precision_oracle_leg(cap, cores):
    """The FP64 oracle on the precision workload's original uint16 codes and
    FP32 table (total error of each form) on the machine's host cores: the 4096
    seeded pixels of the 2048^2 frame and the full 512^2 frame. Returns the
    per-image errors of every storage form and the oracle's own timing."""
    import oracle
    oracle.build()
    wp, ph, tf = cap["w"], cap["ph"], cap["tf"]
    kw = dict(step=wp["step"], term=wp["term"], shade=wp["shade"])
    t0 = time.perf_counter()
    o_rays = oracle.render(oracle.Scene(ph.vol, ph.spacing, tf, cap["cam"], **kw), pixels=cap["pix"], nthreads=cores)
    t1 = time.perf_counter()
    o_small = oracle.render(oracle.Scene(ph.vol, ph.spacing, tf, cap["cam_small"], **kw), nthreads=cores)
    t2 = time.perf_counter()
    res = {"oracle": "FP64, original uint16 codes and FP32 table (total error)", "tolerance": 4e-3}
    for name, (rays, small) in cap["images"].items():
        res[name] = {"rays_4096_of_2048sq": oracle_errors(rays, o_rays), "frame_512sq": oracle_errors(small, o_small)}
    samples = int(o_rays["nsamp"].sum()) + int(o_small["nsamp"].sum())
    res["oracle_time"] = {"rays_s": t1 - t0, "frame_512_s": t2 - t1, "cores": cores,
                          "gsamples_s": samples / (t2 - t0) / 1e9}
    return res


def batch_form(rc, ctx, vol, ph, P, cam_structs, flush, stream, n_extra=3):
    """Several volumes in one launch: the bench phantom and n_extra seeded
    phantoms of the learned-proposal family (same shape), every orbit view of
    each, against one multi-view launch per volume."""
    import torch
    wp = synth.WORKLOADS["proposal_256x256x180"]
    extra = synth.proposal_phantoms(wp["train_seeds"][:n_extra])
    vols = [vol]
    for v in extra:
        h = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, rc.RC_STORE_F32)
        rc.rc_volume_upload(ctx, h, v)
        vols.append(h)
    n = len(cam_structs)
    H, W = cam_structs[0].height, cam_structs[0].width
    out = torch.empty((len(vols), n, H, W, 4), device="cuda")
    st = rc.rc_render_batch(ctx, vols, P, cam_structs, out, stats=True)
    one = []
    batch = []
    for rep in range(3):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        rc.rc_render_batch(ctx, vols, P, cam_structs, out)
        e[1].record(stream)
        for i, h in enumerate(vols):
            rc.rc_render_views(ctx, h, P, cam_structs, out[i])
        e[2].record(stream)
        flush.zero_()
        batch.append(e)
    torch.cuda.synchronize()
    b_ms = statistics.median(a.elapsed_time(b) for a, b, c in batch)
    s_ms = statistics.median(b.elapsed_time(c) for a, b, c in batch)
    for h in vols[1:]:
        rc.rc_volume_destroy(ctx, h)
    frames = len(vols) * n
    return {"volumes": len(vols), "views_per_volume": n, "ms_per_frame_batch": b_ms / frames,
            "ms_per_frame_per_volume_launches": s_ms / frames,
            "gsamples_s_batch": st["dense_samples"] / (b_ms / 1e3) / 1e9}


def adjoint_form(rc, ctx, flush, stream):
    """Transfer-function gradient on the differentiable workload (128x128x96,
    8 views at 512^2, unshaded, step 0.5): time of rc_render_backward_views
    over the 8 views (one launch, gradient summed) per view against the
    forward rc_render_views of the same views, with the samples each pass
    marches (the backward recomputes the forward, then marches again)."""
    import torch
    wd = synth.WORKLOADS["diff_128x128x96"]
    ph = synth.workload_phantom("diff_128x128x96")
    vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, rc.RC_STORE_F32)
    rc.rc_volume_upload(ctx, vol, ph.vol)
    tf = torch.from_numpy(synth.noise_tf(wd["K"], wd["init_tf_seed"], alpha_max=0.1)).cuda()
    rc.rc_tf_set_device(ctx, tf)
    cams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=wd["width"], height=wd["height"])
            for az in wd["azimuths"]]
    P = rc.RenderParams(step_vox=wd["step"], term=wd["term"], shade=False, skip=False)
    img = torch.empty((wd["height"], wd["width"], 4), device="cuda")
    g = torch.randn(img.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    dtf = torch.empty_like(tf)
    dense = 0
    for cam in cams:
        rc.rc_camera_set(ctx, cam)
        dense += rc.rc_render(ctx, vol, P, img, stats=True)["dense_samples"]
    # every view in one launch: the forward render and the gradient summed
    # over the views (the loss of a table fit to the orbit)
    n = len(cams)
    cam_structs = [rc.make_camera(c) for c in cams]
    imgs = torch.empty((n, wd["height"], wd["width"], 4), device="cuda")
    G = torch.randn(imgs.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(0))

    def pair_ms(Pf, dt, reps):
        """Median forward, backward and backward-given-the-forward times per
        view over reps runs."""
        rc.rc_render_backward_views(ctx, vol, Pf, cam_structs, G, dt)    # builds what the form needs
        ev = []
        for rep in range(reps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            rc.rc_render_views(ctx, vol, Pf, cam_structs, imgs)
            e[1].record(stream)
            rc.rc_render_backward_views(ctx, vol, Pf, cam_structs, G, dt)
            e[2].record(stream)
            rc.rc_render_backward_views_with_forward(ctx, vol, Pf, cam_structs, imgs, G, dt)
            e[3].record(stream)
            ev.append(e)
            flush.zero_()
        torch.cuda.synchronize()
        return (statistics.median(a.elapsed_time(b) for a, b, c, d in ev) / n,
                statistics.median(b.elapsed_time(c) for a, b, c, d in ev) / n,
                statistics.median(c.elapsed_time(d) for a, b, c, d in ev) / n)

    f_ms, b_ms, bf_ms = pair_ms(P, dtf, 3)
    # the same with cubic B-spline reconstruction
    Pb = rc.RenderParams(step_vox=wd["step"], term=wd["term"], shade=False, skip=False, filter=rc.RC_FILTER_BSPLINE)
    fb_ms, bb_ms, bbf_ms = pair_ms(Pb, dtf, 3)
    # a 2-D table (the same rows, opacity rising with gradient magnitude):
    # the gradient scatters into four entries per sample in global memory
    M2 = 32
    tab2 = np.repeat(synth.noise_tf(wd["K"], wd["init_tf_seed"], alpha_max=0.1)[None], M2, axis=0)
    tab2[..., 3] *= np.linspace(0.4, 1.0, M2, dtype=np.float32)[:, None]
    rc.rc_tf2d_set(ctx, tab2, 1200.0)
    dtf2 = torch.empty((M2, wd["K"], 4), device="cuda")
    f2_ms, b2_ms, b2f_ms = pair_ms(P, dtf2, 3)
    rc.rc_volume_destroy(ctx, vol)
    per_view = dense / len(cams)
    return {"workload": "diff_128x128x96", "views": len(cams), "image": "512x512",
            "forward_ms_per_view": f_ms, "backward_ms_per_view": b_ms, "backward_over_forward": b_ms / f_ms,
            "backward_with_forward_ms_per_view": bf_ms, "backward_with_forward_over_forward": bf_ms / f_ms,
            "dense_samples_per_view": per_view,
            "backward_gsamples_s": 2 * per_view / (b_ms / 1e3) / 1e9,
            "bspline": {"forward_ms_per_view": fb_ms, "backward_ms_per_view": bb_ms,
                        "backward_over_forward": bb_ms / fb_ms, "backward_with_forward_ms_per_view": bbf_ms,
                        "backward_with_forward_over_forward": bbf_ms / fb_ms},
            "tf2d": {"table": f"{M2}x{wd['K']}", "forward_ms_per_view": f2_ms, "backward_ms_per_view": b2_ms,
                     "backward_over_forward": b2_ms / f2_ms, "backward_with_forward_ms_per_view": b2f_ms,
                     "backward_with_forward_over_forward": b2f_ms / f2_ms},
            "note": "exact skipping in the forward recompute, none in the gradient pass (an empty brick still has a gradient)"}


def proposal_form(rc, ctx, vol, ph, w, cams, P, outs, frame_ms, flush, stream, n_train):
    """Learned proposal on the bench workload: the network is trained on
    n_train seeded phantoms (never the bench phantom), then every view is
    rendered with 64 proposal samples per ray at several fallback thresholds
    and compared with the FP32 plain march (PSNR, time)."""
    import torch
    from paper_1211_5595_gb300 import proposal
    wp = synth.WORKLOADS["proposal_256x256x180"]
    t0 = time.perf_counter()
    vols = synth.proposal_phantoms(wp["train_seeds"][:n_train])
    train_vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, rc.RC_STORE_F32)
    rc.rc_proposal_load(ctx, rc.pack_proposal_blob(synth.proposal_init_params(61)))
    tcams = [synth.orbit_camera(ph.dims, ph.spacing, az, width=512, height=512) for az in wp["azimuths"][::3]]
    feats, tgts = [], []
    for i, v in enumerate(vols):
        rc.rc_volume_upload(ctx, train_vol, v)
        f, t = proposal.collect_rays(ctx, train_vol, tcams, P, 4096, seed=i)
        feats.append(f)
        tgts.append(t)
    rc.rc_volume_destroy(ctx, train_vol)
    F, T = torch.cat(feats), torch.cat(tgts)
    curve = proposal.train(ctx, F, T, epochs=30, batch=8192, lr=3e-3, seed=0)
    train_s = time.perf_counter() - t0
    del F, T, feats, tgts
    ref = outs
    n = len(cams)
    cam_structs = [rc.make_camera(c) for c in cams]
    imgs = torch.empty_like(outs)
    plain_frame_ms = statistics.median(frame_ms)      # the plain march, all views in one launch

    def measure(render, **rec):
        """Median time per frame of render() over 3 runs (every view in one
        call), PSNR of each view against the plain march, fallback rate."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        for rep in range(3):
            ev[rep][0].record(stream)
            render(False)
            ev[rep][1].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev) / n
        mse = ((imgs - ref) ** 2).mean(dim=(1, 2, 3)).double().cpu().numpy()
        psnrs = [float("inf") if m == 0 else 10 * np.log10(1.0 / m) for m in mse]
        st = render(True)
        finite = [p for p in psnrs if np.isfinite(p)]
        rec.update({"ms_per_frame_median": ms, "speedup_vs_f32": plain_frame_ms / ms,
                    "psnr_db_min": min(psnrs), "psnr_db_mean": float(np.mean(finite)) if finite else float("inf"),
                    "max_abs": float((imgs - ref).abs().max()),
                    "fallback_rate": st["fallback_rays"] / max(1, st["rays_hit"]),
                    "evaluated_samples": st["evaluated_samples"]})
        return rec

    def proposal(sampling, lam, nimp, eps):
        # network launch (range records or PDFs) + importance-march launch
        return lambda stats: rc.rc_render_proposal_sampled(ctx, vol, P, cam_structs, sampling, lam, nimp, eps, imgs,
                                                           stats=stats)

    def uniform(nimp):
        # no network: nimp samples at the centres of nimp equal segments of the chord
        return lambda stats: rc.rc_render_importance_views(ctx, vol, P, cam_structs, rc.RC_SAMPLING_INVCDF, 1.0,
                                                           None, None, nimp, 2.0, imgs, stats=stats)

    # fallback thresholds of the range reading at 64 samples per ray
    sweep = [measure(proposal(rc.RC_SAMPLING_RANGE, 0.0, 64, eps), sampling="range", nimp=64, eps=eps)
             for eps in (2.0, 0.02, 0.005, 0.0)]
    sweep += [measure(proposal(rc.RC_SAMPLING_INVCDF, 0.05, 64, eps), sampling="invcdf", lam=0.05, nimp=64, eps=eps)
              for eps in (0.02, 0.0)]
    # the readings of "few importance samples" at equal sample counts, no fallback
    readings = []
    for nimp in (16, 32, 64, 128):
        readings.append(measure(proposal(rc.RC_SAMPLING_RANGE, 0.0, nimp, 2.0), sampling="range", nimp=nimp))
        readings.append(measure(proposal(rc.RC_SAMPLING_INVCDF, 0.05, nimp, 2.0), sampling="invcdf", lam=0.05,
                                nimp=nimp))
        readings.append(measure(uniform(nimp), sampling="uniform_chord", nimp=nimp))
    ok = [r for r in sweep + readings if r["psnr_db_min"] >= 45.0]
    best = max(ok, key=lambda r: r["speedup_vs_f32"]) if ok else None
    return {"nimp": 64, "train_phantoms": n_train, "train_s": train_s, "views_per_launch": n,
            "plain_ms_per_frame": plain_frame_ms, "loss_first_last": [curve[0], curve[-1]], "sweep": sweep,
            "readings": readings,
            "readings_note": "eps 2 (no fallback): range = nimp equal segments of the range the network's PDF "
                             "marks; invcdf = stratified inverse CDF of 0.95 PDF + 0.05 uniform, midpoint "
                             "segments; uniform_chord = nimp equal segments of the whole chord (no network)",
            "speedup_at_psnr45": best["speedup_vs_f32"] if best else None,
            "config_at_psnr45": {k: best.get(k) for k in ("sampling", "nimp", "eps")} if best else None,
            "network": network_throughput(rc, ctx, stream)}


def network_throughput(rc, ctx, stream, n=1 << 20):
    """The tensor-core network alone on a feature matrix of n rays
    (rc_proposal_forward): algorithmic FLOPs (2 x 17,920 MACs per ray, the
    padded 8 outputs of the last layer not counted) and bytes (112 FP32
    features in, 33 FP32 outputs out per ray) per launch time."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    feat = torch.rand((n, 112), device="cuda", generator=g)
    out = torch.empty((n, 33), device="cuda")
    for _ in range(3):
        rc.rc_proposal_forward(ctx, feat, n, out)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for e in ev:
        e[0].record(stream)
        rc.rc_proposal_forward(ctx, feat, n, out)
        e[1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    flops = 2.0 * 17920 * n
    nbytes = (112 + 33) * 4 * n
    bf16 = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass
    # training gradient (rc_proposal_grad): forward, weight gradients of all
    # four layers and data gradients of layers 2-4, 46,592 MACs per ray, plus
    # the deterministic cross-CTA reduction
    tgt = torch.rand((n, 33), device="cuda", generator=g)
    grad = torch.empty(18152, device="cuda")
    loss = torch.empty(1, device="cuda")
    for _ in range(3):
        rc.rc_proposal_grad(ctx, feat, tgt, n, grad, loss)
    for e in ev:
        e[0].record(stream)
        rc.rc_proposal_grad(ctx, feat, tgt, n, grad, loss)
        e[1].record(stream)
    torch.cuda.synchronize()
    gms = statistics.median(a.elapsed_time(b) for a, b in ev)
    gflops = 2.0 * 46592 * n
    del tgt, grad, loss
    return {"rays": n, "ms": ms, "tflops_s": flops / (ms / 1e3) / 1e12, "gbs": nbytes / (ms / 1e3) / 1e9,
            "frac_of_bf16_peak": (flops / (ms / 1e3) / 1e12 / bf16) if bf16 else None,
            "note": "feature matrix in HBM: 580 B per ray against 35.8 kFLOP, so the launch is memory-bound",
            "grad_ms": gms, "grad_mrays_s": n / (gms / 1e3) / 1e6, "grad_tflops_s": gflops / (gms / 1e3) / 1e12,
            "grad_frac_of_bf16_peak": (gflops / (gms / 1e3) / 1e12 / bf16) if bf16 else None}


def run_reference(args, w, world, rank):
    """The oracle as the reference arm (host cores, bounded sample per step)."""
    if rank != 0:
        return 0
    ph = synth.workload_phantom(WORKLOAD)
    tf = synth.tf_table(w["K"])
    cams = cameras(ph, w)
    import oracle
    oracle.build()
    cores = oracle.default_threads()
    # every 64th image row of each view (16 full rows, 16384 rays): enough rays
    # per call that the oracle's per-call setup is amortised, and whole rows
    # keep neighbouring rays together as in a full frame
    rows = np.arange(w["height"] // 128, w["height"], w["height"] // 16)
    pix = (rows[:, None] * w["width"] + np.arange(w["width"])[None, :]).reshape(-1).astype(np.int32)
    per_view = len(pix)
    times, samples = [], 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s = 0
        for i, cam in enumerate(cams):
            sc = oracle.Scene(ph.vol, ph.spacing, tf, cam, step=w["step"], term=w["term"], shade=w["shade"])
            s += int(oracle.render(sc, pixels=pix, nthreads=cores)["nsamp"].sum())
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
            samples += s
    tot = sum(times)
    val = samples / tot / 1e9
    sample = f"{per_view} pixels (every 64th row) of each of the 36 views per step (FP64 oracle, all cores)"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gsamples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded head phantom)",
            "config": {"workload": WORKLOAD, "image": "1024x1024", "views": 36, "sample": sample},
            "cpu_baseline": {"value": val, "unit": "Gsamples/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--views", type=int, default=0, help="render only the first N orbit views (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16 / uint16 storage forms")
    ap.add_argument("--no-proposal", action="store_true", help="skip the learned-proposal form")
    ap.add_argument("--no-precision", action="store_true", help="skip the 512x512x256 precision form")
    ap.add_argument("--proposal-phantoms", type=int, default=8, help="training phantoms of the proposal form")
    ap.add_argument("--case", choices=["adjoint", "network", "precision", "staged", "proposal"], default=None,
                    help="run only the table-gradient form, the network throughput (forward and training "
                         "gradient, seeded initial network) or one 2048^2 frame of each precision form (FP32, "
                         "FP16, uint16 storage: two launches each, the first untimed) and print its JSON "
                         "(profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = synth.WORKLOADS[WORKLOAD]
    world, rank, local = setup_dist()
    if args.impl == "reference":
        return run_reference(args, w, world, rank)
    if world > 1:
        # the scaling line needs the main metric and e2e only: the forms
        # (identical on every rank) would only multiply host work per rank
        args.no_forms = args.no_proposal = args.no_precision = True

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1211_5595_gb300 import build as _b
    _b.build()
    import paper_1211_5595_gb300 as rc

    ph = synth.workload_phantom(WORKLOAD)
    tf = synth.tf_table(w["K"])
    cams = cameras(ph, w)
    if args.views:
        cams = cams[:args.views]
    nviews = len(cams)
    H, W = w["height"], w["width"]
    stream = torch.cuda.current_stream()
    ctx = rc.rc_context_create(local, stream.cuda_stream)
    if args.case:
        flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda", dtype=torch.float32)
        if args.case == "adjoint":
            out = adjoint_form(rc, ctx, flush, stream)
        elif args.case == "precision":
            out = precision_frames(rc, ctx, stream)
        elif args.case == "staged":
            out = staged_form(rc, ctx, stream, flush, cams)
        elif args.case == "proposal":
            out = proposal_frames(rc, ctx, stream, cams)
        else:
            rc.rc_proposal_load(ctx, rc.pack_proposal_blob(synth.proposal_init_params(61)))
            out = network_throughput(rc, ctx, stream)
        torch.cuda.synchronize()
        rc.rc_context_destroy(ctx)
        if rank == 0:
            print(json.dumps({"case": args.case, **out}))
        return 0
    vol = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, rc.RC_STORE_F32)
    codes_host = torch.from_numpy(ph.vol.view(np.int16).reshape(-1)).pin_memory()
    codes_dev = codes_host.to("cuda", non_blocking=True)
    tf_host = torch.from_numpy(tf).pin_memory()
    tf_dev = tf_host.to("cuda")
    rc.rc_volume_upload(ctx, vol, codes_dev)
    rc.rc_tf_set_device(ctx, tf_dev)
    P = params(w)
    outs = torch.empty((nviews, H, W, 4), device="cuda", dtype=torch.float32)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda", dtype=torch.float32)

    # dense-equivalent and evaluated samples of one orbit (deterministic)
    dense = evald = 0
    for v, cam in enumerate(cams):
        rc.rc_camera_set(ctx, cam)
        st = rc.rc_render(ctx, vol, P, outs[v], stats=True)
        dense += st["dense_samples"]
        evald += st["evaluated_samples"]

    cam_structs = [rc.make_camera(c) for c in cams]

    def step(events=None):
        rc.rc_volume_upload(ctx, vol, codes_dev)          # a1 re-layout + a2 min/max grid
        rc.rc_tf_set_device(ctx, tf_dev)                   # a3 occupancy for the table
        if events is not None:
            events[0].record(stream)
        rc.rc_render_views(ctx, vol, P, cam_structs, outs)   # a4-a11, every view in one launch
        if events is not None:
            events[1].record(stream)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        for s in range(args.steps):
            step_ev[s][0].record(stream)
            step(kern_ev[s])
            step_ev[s][1].record(stream)
            flush.zero_()                                   # L2 flush between steps, outside the events
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    fp32_imgs = outs.clone()                                # reference images of the other forms
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    launch_ms = [a.elapsed_time(b) for a, b in kern_ev]          # one launch renders every view
    frame_ms = [m / nviews for m in launch_ms]
    total_ms = max_over_ranks(sum(step_ms), world, "cuda")
    value = job_throughput(world, dense, args.steps, total_ms) / 1e9
    ms_per_step = total_ms / args.steps

    # end to end through the C-ABI with host buffers: pinned codes and table
    # in, every view's image out, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        img_host = torch.empty((nviews, H, W, 4), dtype=torch.float32).pin_memory()
        codes_np = codes_host.numpy().view(np.uint16)

        def e2e_step():
            # host codes in, host images out: the views are rendered in groups
            # whose device-to-host copies overlap the next group's march
            rc.rc_volume_upload(ctx, vol, codes_np)
            rc.rc_tf_set(ctx, tf)
            rc.rc_render_views_host(ctx, vol, P, cam_structs, img_host)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        # host-timed: three timed loops of the K steps, the median reported
        # (one loop alone moves by several percent with the host's load)
        # (the slowest rank's time of each loop, the ranks started together)
        runs, loop_steps = [], []
        # five timed loops, the median reported: a single step of a loop can
        # stall by 10-25 ms on a busy host; the garbage collector paused in
        # the loops, as timeit does; no clock sampler here: its queries go
        # through the same driver
        gc.collect()
        gc.disable()
        for _ in range(5):
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            ts = [t0]
            for _ in range(args.steps):
                e2e_step()                               # returns once the images are in host memory
                ts.append(time.perf_counter())
            el = max_over_ranks(ts[-1] - t0, world, "cuda")
            runs.append(world * dense * args.steps / el / 1e9)
            st_ms = [1e3 * (b - a) for a, b in zip(ts, ts[1:])]
            loop_steps.append({"median": statistics.median(st_ms), "min": min(st_ms), "max": max(st_ms)})
        gc.enable()
        e2e = {"value": statistics.median(runs), "unit": "Gsamples/s",
               "h2d_bytes_per_step": codes_host.numel() * 2 + tf.nbytes,
               "d2h_bytes_per_step": img_host.numel() * 4,
               "runs": runs, "run_step_ms": loop_steps,
               "timing": f"host clock over {args.steps} steps, median of 5 loops"}

    hbm_peak, peak_kind = peaks()
    # reduced-precision storage forms on the same workload: FP16 (normalised)
    # and raw uint16 volumes with the FP16 table, against the FP32 images
    forms = {}
    precision_capture = None
    if not args.no_forms:
        ref_imgs = fp32_imgs
        fp32_frame_ms = statistics.median(frame_ms)
        for name, storage in (("f16", rc.RC_STORE_F16), ("u16", rc.RC_STORE_U16)):
            v2 = rc.rc_volume_create(ctx, ph.dims, ph.spacing, synth.VMAX, storage)
            rc.rc_volume_upload(ctx, v2, codes_dev)
            rc.rc_tf_set_device(ctx, tf_dev, fp16=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
            for rep in range(3):
                ev[rep][0].record(stream)
                rc.rc_render_views(ctx, v2, P, cam_structs, outs)
                ev[rep][1].record(stream)
                flush.zero_()
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in ev) / nviews
            mse = ((outs - ref_imgs) ** 2).mean(dim=(1, 2, 3))
            psnr = float((10 * torch.log10(1.0 / mse.clamp_min(1e-30))).min())
            forms[name] = {"ms_per_frame_median": ms, "gsamples_s": dense / nviews / (ms / 1e3) / 1e9,
                           "speedup_vs_f32": fp32_frame_ms / ms, "psnr_db_min_vs_f32": psnr,
                           "max_abs_vs_f32": float((outs - ref_imgs).abs().max())}
            rc.rc_volume_destroy(ctx, v2)
        rc.rc_tf_set_device(ctx, tf_dev)
        forms.update(filter_forms(rc, ctx, vol, w, P, cam_structs, outs, fp32_imgs, flush, stream, hbm_peak))
        rc.rc_tf_set_device(ctx, tf_dev)
        forms["volume_batch"] = batch_form(rc, ctx, vol, ph, P, cam_structs, flush, stream)

    if not args.no_forms:
        forms["adjoint"] = adjoint_form(rc, ctx, flush, stream)
        if not args.no_precision:
            forms["precision"], precision_capture = precision_form(rc, ctx, flush, stream, hbm_peak)
        rc.rc_tf_set_device(ctx, tf_dev)

    if not args.no_proposal:
        forms["proposal"] = proposal_form(rc, ctx, vol, ph, w, cams, P, fp32_imgs, frame_ms, flush, stream,
                                          args.proposal_phantoms)

    launch_avg_s = statistics.mean(launch_ms) / 1e3
    achieved = evald * BYTES_PER_SAMPLE / launch_avg_s / 1e9
    counters = profiled_counters() if nviews == 36 else {}
    traffic = counters.get("dram_bytes_per_launch")
    # the memory level that serves the gathers: L1 (95% of the sectors hit
    # there), measured live with the L1 probe; beside it the DRAM and L2->L1
    # rates from the ncu counters of the same kernel, and the instruction issue
    # rate against 4 schedulers per SM x the SM count x the sampled clock
    l1_peak = l1_read_peak(stream)
    l2_peak = l2_read_peak(stream)
    clk = clocks.summary()
    sm_mhz = clk.get("sm_mhz") or 2070.0
    issue_peak = torch.cuda.get_device_properties(local).multi_processor_count * 4 * sm_mhz * 1e6
    dram = l2 = issue = None
    if traffic is not None:
        a = traffic / launch_avg_s / 1e9
        dram = {"achieved_gbs": a, "peak_gbs": hbm_peak, "frac": a / hbm_peak,
                "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch over the live launch time"}
    if "l2_to_l1_bytes_per_launch" in counters:
        a = counters["l2_to_l1_bytes_per_launch"] / launch_avg_s / 1e9
        l2 = {"achieved_gbs": a, "peak_gbs": l2_peak, "frac": a / l2_peak,
              "peak_kind": "measured in this run: rc_probe_read_l2, a 96 MB buffer read 40 times through L2"}
    if "warp_instructions_per_launch" in counters:
        a = counters["warp_instructions_per_launch"] / launch_avg_s
        issue = {"achieved_warp_inst_s": a, "peak_warp_inst_s": issue_peak, "frac": a / issue_peak,
                 "peak_kind": "4 issue slots per SM per clock x SMs x median SM clock under load"}
    # the bytes a frame cannot avoid: the volume's FP32 values read once and
    # the image written once (the brick grid and table are negligible), at
    # the measured HBM rate, against the measured frame time
    vol_bytes = 4 * int(np.prod(ph.dims))
    img_bytes = 16 * H * W
    floor_us = (vol_bytes + img_bytes) / (hbm_peak * 1e9) * 1e6
    floor = {"bytes_per_frame": vol_bytes + img_bytes, "volume_bytes": vol_bytes, "image_bytes": img_bytes,
             "us_per_frame_at_hbm_peak": floor_us,
             "frac_of_frame_time": floor_us / (1e3 * statistics.median(frame_ms))}
    line = {
        "metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded head phantom, Rician noise)",
        "config": {"workload": WORKLOAD, "volume": "256x256x180 u16 -> FP32 19^3 apron bricks + 17^3 value+gradient bricks", "image": "1024x1024",
                   "views": nviews, "step_vox": w["step"], "shading": "Blinn-Phong headlight",
                   "skip": "16^3 min/max brick grid + 4^3 sub-block mask (exact)", "term": w["term"],
                   "l2": "flushed between steps (256 MB write, outside the step events)",
                   "ms_per_frame_median": statistics.median(frame_ms),
                   "dense_samples_per_step": dense, "evaluated_samples_per_step": evald},
        "roofline": {"bound": "l1", "achieved": achieved, "peak": l1_peak, "unit": "GB/s",
                     "frac": achieved / l1_peak, "traffic": traffic,
                     "kernel": "composite_kernel<F32, shaded>, one launch per step for all views",
                     "model": f"{BYTES_PER_SAMPLE} B per evaluated sample (32 distinct FP32 voxels = 8 value+gradient float4) / mean launch time",
                     "peak_kind": "measured in this run: rc_probe_read_l1, coalesced 16-byte read-only loads of "
                                  "an L1-resident 32 KB buffer by 4 CTAs per SM",
                     "note": "95% of the gather sectors hit L1, so L1 is the memory level that serves the "
                             "algorithmic bytes; scattered 16-byte gathers use fewer bytes per L1 wavefront "
                             "than the probe's coalesced loads (ncu: L1 data pipe l1_data_pipe_frac), and "
                             "instruction issue (issue) is the co-limit",
                     "model_bytes_frac_of_hbm": achieved / hbm_peak,
                     "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json)",
                     "l1_data_pipe_frac": (counters["l1_data_pipe_pct"] / 100.0) if "l1_data_pipe_pct" in counters
                     else None,
                     "dram": dram, "l2": l2, "issue": issue,
                     "compulsory_floor": floor},
        "e2e": e2e,
        "forms": forms,
        # per step, this library's kernels (the ncu launch list): the volume
        # preparation (apron and value+gradient bricks, both trilinear grids),
        # the table's FP16 copy, the brick and the 4^3 sub-block occupancy
        # masks, the march of every view
        "gpu_launches": args.steps * 5,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, cores, desc = cpu_oracle_sample(ph, tf, w, cams, args.cpu_budget)
        v1, d1 = cpu_oracle_one_core(ph, tf, w, cams[0])
        line["cpu_baseline"] = {"value": val, "unit": "Gsamples/s", "cores": cores, "kind": "oracle", "sample": desc,
                                "cpu": cpu_model(), "one_core": {"value": v1, "sample": d1}}
        if precision_capture is not None:
            # the same oracle on the precision workload: each storage form's
            # error against the FP64 oracle, per image
            forms["precision"]["oracle_error"] = precision_oracle_leg(precision_capture, cores)
    rc.rc_volume_destroy(ctx, vol)
    rc.rc_context_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
