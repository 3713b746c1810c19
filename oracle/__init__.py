"""FP64 CPU oracle of the raycasting method (Adeshina et al., Sec. 4.1-4.2).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg are the only callers. The oracle shares no code with
the CUDA library (``paper_1211_5595_gb300``) and never imports it; the two meet
only in the seeded inputs of ``synth``.

``oracle.c`` holds the renderer, its transfer-function gradient, the opacity
profiles and the importance-sampled composite; ``mlp.py`` holds the FP64 proposal
network. Every function states the passage it follows in its own docstring or
comment.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

COMPOSITE, MIP, AVERAGE, XRAY, ISO, THRESHOLD = range(6)
TRILINEAR, BSPLINE = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FP contraction, so the FP32 ray
    specification rounds once per operation)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", "-o", _SO + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


class _Volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("sx", C.c_float), ("sy", C.c_float), ("sz", C.c_float),
                ("vmax", C.c_int32), ("value_mode", C.c_int32)]


class _TF(C.Structure):
    _fields_ = [("rgba", C.c_void_p), ("K", C.c_int32), ("fp16", C.c_int32), ("M", C.c_int32),
                ("gmax", C.c_float)]


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fovy_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("step_vox", C.c_float), ("term", C.c_float), ("shade", C.c_int32),
                ("ka", C.c_float), ("kd", C.c_float), ("ks", C.c_float),
                ("func", C.c_int32), ("iso", C.c_float), ("fp64_rays", C.c_int32),
                ("tie_band", C.c_float), ("filter", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.c_void_p
        L.orc_render.argtypes = [P, P, P, P, P, C.c_int64, P, P, P, P, P, C.c_int]
        L.orc_ray_samples.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_int, P, P]
        L.orc_ray_geometry.argtypes = [P, P, P, P, C.c_int, C.c_int, P]
        L.orc_render_grad.argtypes = [P, P, P, P, P, C.c_int64, P, P, P, C.c_int]
        L.orc_profiles.argtypes = [P, P, P, P, P, C.c_int64, P, P, C.c_int]
        L.orc_importance.argtypes = [P, P, P, P, P, C.c_int64, P, P, C.c_int, C.c_int, C.c_float, P, P, P, P, P,
                                     C.c_int]
        L.orc_importance_positions.argtypes = [P, P, P, P, C.c_int, C.c_int, P, P, C.c_int, C.c_int, C.c_float,
                                               P, P]
        L.orc_proposal_features.argtypes = [P, P, P, P, P, C.c_int64, P, P]
        L.orc_proposal_features.restype = C.c_int
        L.orc_brick_minmax.argtypes = [P, P, P]
        L.orc_brick_minmax_filter.argtypes = [P, C.c_int, P, P]
        L.orc_brick_minmax_filter.restype = None
        L.orc_occupancy.argtypes = [P, P, P, P, P]
        for f in ("orc_render", "orc_ray_samples", "orc_ray_geometry", "orc_render_grad",
                  "orc_profiles", "orc_importance", "orc_importance_positions"):
            getattr(L, f).restype = C.c_int
        L.orc_brick_minmax.restype = None
        L.orc_occupancy.restype = None
        _lib = L
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


class Scene:
    """Inputs of one render, marshalled once (keeps the arrays alive)."""

    def __init__(self, vol, spacing, tf, camera, *, step=0.5, term=0.99, shade=False,
                 ka=0.1, kd=0.7, ks=0.2, func=COMPOSITE, iso=0.0, fp64_rays=False,
                 tie_band=2e-5, vmax=4095, value_mode=0, tf_fp16=False, gmax=None,
                 filter=TRILINEAR):
        self.vol = np.ascontiguousarray(vol, dtype=np.uint16)
        assert self.vol.ndim == 3
        nz, ny, nx = self.vol.shape
        # tf: (K, 4) one-dimensional, or (M, K, 4) over (gradient magnitude, value)
        self.tf = np.ascontiguousarray(tf, dtype=np.float32)
        assert self.tf.ndim in (2, 3) and self.tf.shape[-1] == 4
        K = self.tf.shape[-2]
        M = self.tf.shape[0] if self.tf.ndim == 3 else 0
        if M:
            assert gmax is not None and gmax > 0
        self.v = _Volume(self.vol.ctypes.data, nx, ny, nz, *[float(s) for s in spacing],
                         int(vmax), int(value_mode))
        self.t = _TF(self.tf.ctypes.data, K, int(bool(tf_fp16)), M, float(gmax or 0.0))
        self.c = _Camera((C.c_float * 3)(*camera["eye"]), (C.c_float * 3)(*camera["target"]),
                         (C.c_float * 3)(*camera["up"]), float(camera["fovy_deg"]),
                         int(camera["width"]), int(camera["height"]))
        self.p = _Params(float(step), float(term), int(bool(shade)), float(ka), float(kd),
                         float(ks), int(func), float(iso), int(bool(fp64_rays)), float(tie_band),
                         int(filter))
        self.width = int(camera["width"])
        self.height = int(camera["height"])

    def refs(self):
        return C.byref(self.v), C.byref(self.t), C.byref(self.c), C.byref(self.p)

    def npix(self, pixels):
        return self.width * self.height if pixels is None else len(pixels)


def _pix(pixels):
    if pixels is None:
        return None, None
    arr = np.ascontiguousarray(pixels, dtype=np.int32)
    return arr, arr.ctypes.data


def render(scene: Scene, pixels=None, nthreads=None):
    """Render every pixel (row-major, y = 0 at the top) or the listed pixel
    indices y*W + x. Returns dict rgba (n, 4) premultiplied, alt (the other
    branch of the first termination tie), tie (bool), nsamp (samples
    composited up to termination) and nsamp_alt (the same on the other branch)."""
    n = scene.npix(pixels)
    rgba = np.zeros((n, 4)); alt = np.zeros((n, 4))
    tie = np.zeros(n, dtype=np.uint8); ns = np.zeros(n, dtype=np.int32)
    ns2 = np.zeros(n, dtype=np.int32)
    arr, ptr = _pix(pixels)
    rc = lib().orc_render(*scene.refs(), ptr, n, rgba.ctypes.data, alt.ctypes.data,
                          tie.ctypes.data, ns.ctypes.data, ns2.ctypes.data,
                          nthreads or default_threads())
    if rc:
        raise ValueError(f"oracle render failed ({rc})")
    if pixels is None:
        shp = (scene.height, scene.width)
        return dict(rgba=rgba.reshape(*shp, 4), alt=alt.reshape(*shp, 4),
                    tie=tie.reshape(shp).astype(bool), nsamp=ns.reshape(shp),
                    nsamp_alt=ns2.reshape(shp))
    return dict(rgba=rgba, alt=alt, tie=tie.astype(bool), nsamp=ns, nsamp_alt=ns2)


def ray_samples(scene: Scene, x, y, max_samples=100000):
    """Every sample of one ray without termination: structured columns t,
    px, py, pz, v, u, r, g, b, a, a_corr, col_r, col_g, col_b, gm (|grad f|,
    value units per mm) and gw (its 2-D table coordinate); gm and gw are 0
    unless shading or a 2-D table needs the gradient."""
    out = np.zeros((max_samples, 16))
    tot = C.c_int32(0)
    rc = lib().orc_ray_samples(*scene.refs(), int(x), int(y), max_samples, out.ctypes.data,
                               C.byref(tot))
    if rc:
        raise ValueError("oracle ray_samples failed")
    n = min(tot.value, max_samples)
    names = ("t", "px", "py", "pz", "v", "u", "r", "g", "b", "a", "a_corr", "col_r", "col_g", "col_b",
             "gm", "gw")
    return {k: out[:n, i].copy() for i, k in enumerate(names)}


def ray_geometry(scene: Scene, x, y):
    out = np.zeros(14)
    rc = lib().orc_ray_geometry(*scene.refs(), int(x), int(y), out.ctypes.data)
    if rc:
        raise ValueError("oracle ray_geometry failed")
    return dict(hit=bool(out[0]), tn=out[1], tf=out[2], ds=out[3], nsamp=int(out[4]),
                o=out[5:8].copy(), d=out[8:11].copy(), dir=out[11:14].copy())


def render_grad(scene: Scene, dimg, pixels=None, nthreads=None):
    """dL/dTF (FP64, the table's shape: K x 4, or M x K x 4 for a 2-D table)
    of the compositing function for the upstream image gradient dimg (per
    pixel RGBA); also returns the FP64 image."""
    n = scene.npix(pixels)
    g = np.ascontiguousarray(np.asarray(dimg, dtype=np.float64).reshape(n, 4))
    dtf = np.zeros(scene.tf.shape[:-1] + (4,)); rgba = np.zeros((n, 4))
    arr, ptr = _pix(pixels)
    rc = lib().orc_render_grad(*scene.refs(), ptr, n, g.ctypes.data, dtf.ctypes.data,
                               rgba.ctypes.data, nthreads or default_threads())
    if rc:
        raise ValueError("oracle render_grad failed")
    return dtf, rgba


def profiles(scene: Scene, pixels=None, nthreads=None):
    """32-bin opacity-weight profiles of the 512-sample march, and T_final."""
    n = scene.npix(pixels)
    bins = np.zeros((n, 32)); tfin = np.zeros(n)
    arr, ptr = _pix(pixels)
    rc = lib().orc_profiles(*scene.refs(), ptr, n, bins.ctypes.data, tfin.ctypes.data,
                            nthreads or default_threads())
    if rc:
        raise ValueError("oracle profiles failed")
    return bins, tfin


SAMPLING = {"range": 0, "invcdf": 1}


def _importance_inputs(scene, pdf, n, occ, sampling, lam):
    if sampling not in SAMPLING:
        raise ValueError(f"sampling {sampling!r}")
    p = None
    if pdf is not None:
        p = np.ascontiguousarray(np.asarray(pdf, dtype=np.float32).reshape(n, 32))
    if occ is None and sampling == "range":
        mn, mx = brick_minmax(scene.vol, vmax=scene.v.vmax, filter=scene.p.filter)
        occ = occupancy((scene.v.nx, scene.v.ny, scene.v.nz), scene.tf, mn, mx, vmax=scene.v.vmax,
                        value_mode=scene.v.value_mode, tf_fp16=bool(scene.t.fp16))
    o = None if occ is None else np.ascontiguousarray(occ, dtype=np.uint8)
    return p, o


def importance(scene: Scene, pdf, nimp=64, pixels=None, nthreads=None, occ=None, sampling="range", lam=0.05):
    """Composite of nimp samples per ray placed by the ray's 32-bin PDF.
    sampling "range": evenly spaced over the range from the first occupied bin
    to the bin where the PDF saturates (occ: cell-brick occupancy, computed
    from the scene when not given); "invcdf": stratified inverse CDF of the
    mixture (1 - lam) PDF + lam uniform, each sample standing for the stretch
    between the midpoints to its neighbours (pdf may be None for lam = 1).
    Returns rgba, alt (the other branch of a termination tie), tie, tfinal and
    nsamp, like render()."""
    n = scene.npix(pixels)
    p, o = _importance_inputs(scene, pdf, n, occ, sampling, lam)
    rgba = np.zeros((n, 4)); alt = np.zeros((n, 4)); tie = np.zeros(n, dtype=np.uint8)
    tfin = np.zeros(n); ns = np.zeros(n, dtype=np.int32)
    arr, ptr = _pix(pixels)
    rc = lib().orc_importance(*scene.refs(), ptr, n, None if p is None else p.ctypes.data,
                              None if o is None else o.ctypes.data, int(nimp), SAMPLING[sampling], float(lam),
                              rgba.ctypes.data, alt.ctypes.data, tie.ctypes.data, tfin.ctypes.data, ns.ctypes.data,
                              nthreads or default_threads())
    if rc:
        raise ValueError("oracle importance failed")
    return {"rgba": rgba, "alt": alt, "tie": tie.astype(bool), "tfinal": tfin, "nsamp": ns}


def importance_positions(scene: Scene, x, y, pdf, nimp=64, occ=None, sampling="range", lam=0.05):
    """Sample positions t (along the ray, mm) and the segment lengths of pixel
    (x, y)'s importance samples; empty arrays for a ray that misses."""
    p, o = _importance_inputs(scene, pdf, 1, occ, sampling, lam)
    t = np.zeros(nimp, dtype=np.float32); ln = np.zeros(nimp, dtype=np.float32)
    k = lib().orc_importance_positions(*scene.refs(), int(x), int(y), None if p is None else p.ctypes.data,
                                       None if o is None else o.ctypes.data, int(nimp), SAMPLING[sampling],
                                       float(lam), t.ctypes.data, ln.ctypes.data)
    if k < 0:
        raise ValueError("oracle importance_positions failed")
    return t[:k].astype(np.float64), ln[:k].astype(np.float64)


def brick_grid_shape(dims):
    nx, ny, nz = dims
    return ((nz - 1 + 15) // 16, (ny - 1 + 15) // 16, (nx - 1 + 15) // 16)


def brick_minmax(vol, vmax=4095, filter=TRILINEAR):
    """Per cell-brick min and max over the (clipped) voxel footprint of the
    filter: 17^3 voxels 16b..16b+16 for trilinear, 19^3 voxels 16b-1..16b+17
    for the cubic B-spline."""
    v = np.ascontiguousarray(vol, dtype=np.uint16)
    nz, ny, nx = v.shape
    shp = brick_grid_shape((nx, ny, nz))
    mn = np.zeros(shp, dtype=np.uint16); mx = np.zeros(shp, dtype=np.uint16)
    desc = _Volume(v.ctypes.data, nx, ny, nz, 1.0, 1.0, 1.0, int(vmax), 0)
    lib().orc_brick_minmax_filter(C.byref(desc), int(filter), mn.ctypes.data, mx.ctypes.data)
    return mn, mx


def occupancy(dims, tf, mn, mx, vmax=4095, value_mode=0, tf_fp16=False):
    """1 where a brick can hold a sample of non-zero opacity, else 0. tf is a
    (K, 4) table or an (M, K, 4) table over (gradient magnitude, value)."""
    nx, ny, nz = dims
    t = np.ascontiguousarray(tf, dtype=np.float32)
    M = t.shape[0] if t.ndim == 3 else 0
    mn = np.ascontiguousarray(mn, dtype=np.uint16); mx = np.ascontiguousarray(mx, dtype=np.uint16)
    occ = np.zeros(mn.shape, dtype=np.uint8)
    desc = _Volume(None, nx, ny, nz, 1.0, 1.0, 1.0, int(vmax), int(value_mode))
    tdesc = _TF(t.ctypes.data, t.shape[-2], int(bool(tf_fp16)), M, 1.0)
    lib().orc_occupancy(C.byref(desc), C.byref(tdesc), mn.ctypes.data, mx.ctypes.data,
                        occ.ctypes.data)
    return occ


def proposal_features(scene: Scene, occ, pixels=None):
    """The 112 features of the learned proposal per listed pixel (FP64)."""
    n = scene.npix(pixels)
    out = np.zeros((n, 112))
    o = np.ascontiguousarray(occ, dtype=np.uint8)
    arr, ptr = _pix(pixels)
    rc = lib().orc_proposal_features(*scene.refs(), ptr, n, o.ctypes.data, out.ctypes.data)
    if rc:
        raise ValueError("oracle proposal_features failed")
    return out
