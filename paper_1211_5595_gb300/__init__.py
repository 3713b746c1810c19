"""Python binding of librc.so, the GB300 direct-volume-rendering raycaster.

Argument marshalling only: every call goes straight to the same-named C entry
point of include/rc.h, and every step of the rendering runs in the library's
CUDA kernels. PyTorch supplies device memory (tensors) and streams. There is
no CPU fallback: when librc.so is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RC_DEBUG=1 in the environment loads the debug build (device index checks
# reported as RC_ERR_CUDA at the next synchronising call) instead
LIB_PATH = os.path.join(_HERE, "librc_debug.so" if os.environ.get("RC_DEBUG") == "1" else "librc.so")

RC_OK, RC_ERR_INVALID_ARG, RC_ERR_OOM, RC_ERR_CUDA, RC_ERR_STATE, RC_ERR_TIMEOUT, \
    RC_ERR_UNSUPPORTED, RC_ERR_FORMAT = range(8)
RC_STORE_F32, RC_STORE_F16, RC_STORE_U16 = range(3)
RC_FUNC_COMPOSITE, RC_FUNC_MIP, RC_FUNC_AVERAGE, RC_FUNC_XRAY, RC_FUNC_ISO, RC_FUNC_THRESHOLD = range(6)
RC_FILTER_TRILINEAR, RC_FILTER_BSPLINE = range(2)
RC_SAMPLING_RANGE, RC_SAMPLING_INVCDF = range(2)


class RCError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"[{status}] {message}")
        self.status = status


class rc_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fovy_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class rc_render_params(C.Structure):
    _fields_ = [("step_vox", C.c_float), ("term", C.c_float), ("shade", C.c_int32),
                ("ka", C.c_float), ("kd", C.c_float), ("ks", C.c_float), ("func", C.c_int32),
                ("iso", C.c_float), ("skip", C.c_int32), ("filter", C.c_int32)]


class rc_stats(C.Structure):
    _fields_ = [("dense_samples", C.c_uint64), ("evaluated_samples", C.c_uint64),
                ("rays_hit", C.c_uint64), ("rays_total", C.c_uint64), ("fallback_rays", C.c_uint64),
                ("device_ms", C.c_float)]


RC_PROPOSAL_BINS = 32
RC_PROPOSAL_FEATURES = 112
RC_PROPOSAL_OUTPUTS = 33
RC_PROPOSAL_PARAMS = 18152


# Every symbol include/rc.h declares, with its ctypes signature.
_P = C.c_void_p
_I = C.c_int
SIGNATURES = {
    "rc_status_string": (C.c_char_p, [_I]),
    "rc_last_error": (C.c_char_p, [_P]),
    "rc_context_create": (_I, [_I, _P, C.POINTER(_P)]),
    "rc_context_set_stream": (_I, [_P, _P]),
    "rc_context_sync": (_I, [_P]),
    "rc_context_destroy": (_I, [_P]),
    "rc_volume_create": (_I, [_P, _I, _I, _I, C.c_float, C.c_float, C.c_float, C.c_uint16, _I,
                              C.POINTER(_P)]),
    "rc_volume_upload": (_I, [_P, _P, C.c_size_t, _I]),
    "rc_volume_destroy": (_I, [_P]),
    "rc_volume_brick_dims": (_I, [_P, C.POINTER(C.c_int * 3)]),
    "rc_tf_set": (_I, [_P, _P, _I, _I]),
    "rc_tf_set_device": (_I, [_P, _P, _I, _I]),
    "rc_tf2d_set": (_I, [_P, _P, _I, _I, C.c_float, _I]),
    "rc_tf2d_set_device": (_I, [_P, _P, _I, _I, C.c_float, _I]),
    "rc_camera_set": (_I, [_P, C.POINTER(rc_camera)]),
    "rc_render": (_I, [_P, _P, C.POINTER(rc_render_params), _P, C.POINTER(rc_stats)]),
    "rc_render_views": (_I, [_P, _P, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I, _P,
                             C.POINTER(rc_stats)]),
    "rc_render_views_host": (_I, [_P, _P, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I, _I, _P,
                                  C.POINTER(rc_stats)]),
    "rc_render_backward": (_I, [_P, _P, C.POINTER(rc_render_params), _P, _P]),
    "rc_render_backward_noalloc": (_I, [_P, _P, C.POINTER(rc_render_params), _P, _P]),
    "rc_brick_grid_get": (_I, [_P, _P, _P, _P]),
    "rc_skip_mask_get": (_I, [_P, _P, _P]),
    "rc_brick_grid_get_filter": (_I, [_P, _P, _I, _P, _P]),
    "rc_skip_mask_get_filter": (_I, [_P, _P, _I, _P]),
    "rc_proposal_load": (_I, [_P, _P, C.c_size_t]),
    "rc_proposal_save": (_I, [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "rc_profiles_generate": (_I, [_P, _P, C.POINTER(rc_render_params), _P]),
    "rc_proposal_features": (_I, [_P, _P, C.POINTER(rc_render_params), _P]),
    "rc_proposal_forward": (_I, [_P, _P, C.c_int64, _P]),
    "rc_proposal_grad": (_I, [_P, _P, _P, C.c_int64, _P, _P]),
    "rc_proposal_train_step": (_I, [_P, _P, _P, C.c_int64, C.c_float, _P]),
    "rc_render_importance": (_I, [_P, _P, C.POINTER(rc_render_params), _P, _P, _I, C.c_float, _P, _P,
                                  C.POINTER(rc_stats)]),
    "rc_render_batch": (_I, [_P, _P, _I, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I, _P,
                             C.POINTER(rc_stats)]),
    "rc_render_backward_views": (_I, [_P, _P, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I, _P, _P]),
    "rc_render_backward_views_with_forward": (_I, [_P, _P, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I,
                                                   _P, _P, _P]),
    "rc_render_proposal": (_I, [_P, _P, C.POINTER(rc_render_params), _I, C.c_float, _P, _P, C.POINTER(rc_stats)]),
    "rc_render_proposal_views": (_I, [_P, _P, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I, _I, C.c_float,
                                      _P, _P, C.POINTER(rc_stats)]),
    "rc_render_importance_views": (_I, [_P, _P, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I, _I,
                                        C.c_float, _P, _P, _I, C.c_float, _P, _P, C.POINTER(rc_stats)]),
    "rc_render_proposal_sampled": (_I, [_P, _P, C.POINTER(rc_render_params), C.POINTER(rc_camera), _I, _I,
                                        C.c_float, _I, C.c_float, _P, _P, C.POINTER(rc_stats)]),
}

_lib = None


def lib():
    """The loaded librc.so; raises when the extension has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA extension missing: {LIB_PATH} (run paper_1211_5595_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, ctx=None, what=""):
    if status != RC_OK:
        msg = lib().rc_last_error(ctx)
        raise RCError(status, f"{what}: {msg.decode() if msg else lib().rc_status_string(status).decode()}")


def _ptr(x):
    """Device/host address of a torch tensor or numpy array (or an int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _default_stream(device):
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# same-named wrappers of the C entry points
# ---------------------------------------------------------------------------
def rc_status_string(status: int) -> str:
    return lib().rc_status_string(status).decode()


def rc_last_error(ctx=None) -> str:
    m = lib().rc_last_error(ctx)
    return m.decode() if m else ""


def rc_context_create(device: int = 0, stream=None):
    out = _P()
    s = _default_stream(device) if stream is None else stream
    _check(lib().rc_context_create(device, s, C.byref(out)), None, "rc_context_create")
    return out.value


def rc_context_sync(ctx):
    _check(lib().rc_context_sync(ctx), ctx, "rc_context_sync")


def rc_context_set_stream(ctx, stream):
    _check(lib().rc_context_set_stream(ctx, stream), ctx, "rc_context_set_stream")


def rc_context_destroy(ctx):
    _check(lib().rc_context_destroy(ctx), ctx, "rc_context_destroy")


def rc_volume_create(ctx, dims, spacing, vmax=4095, storage=RC_STORE_F32):
    out = _P()
    nx, ny, nz = (int(d) for d in dims)
    sx, sy, sz = (float(s) for s in spacing)
    _check(lib().rc_volume_create(ctx, nx, ny, nz, sx, sy, sz, int(vmax), int(storage), C.byref(out)),
           ctx, "rc_volume_create")
    return out.value


def rc_volume_upload(ctx, vol, src):
    """src: numpy uint16 array (host) or a CUDA tensor of 2-byte codes."""
    dev = hasattr(src, "is_cuda") and src.is_cuda
    if not dev:
        src = np.ascontiguousarray(src, dtype=np.uint16)
    n = src.numel() if dev else src.size
    _check(lib().rc_volume_upload(vol, _ptr(src), n, 1 if dev else 0), ctx, "rc_volume_upload")


def rc_volume_destroy(ctx, vol):
    _check(lib().rc_volume_destroy(vol), ctx, "rc_volume_destroy")


def rc_volume_brick_dims(vol):
    d = (C.c_int * 3)()
    _check(lib().rc_volume_brick_dims(vol, C.byref(d)), None, "rc_volume_brick_dims")
    return tuple(d)


def rc_tf_set(ctx, rgba, fp16=False):
    t = np.ascontiguousarray(rgba, dtype=np.float32)
    _check(lib().rc_tf_set(ctx, t.ctypes.data, t.shape[0], int(bool(fp16))), ctx, "rc_tf_set")


def rc_tf2d_set(ctx, rgba, gmax, fp16=False):
    """2-D table over (gradient magnitude, value): rgba of shape (n_grad, n_values, 4)."""
    t = np.ascontiguousarray(rgba, dtype=np.float32)
    if t.ndim != 3 or t.shape[2] != 4:
        raise ValueError("rc_tf2d_set: rgba must have shape (n_grad, n_values, 4)")
    _check(lib().rc_tf2d_set(ctx, t.ctypes.data, t.shape[1], t.shape[0], float(gmax), int(bool(fp16))), ctx,
           "rc_tf2d_set")


def rc_tf_set_device(ctx, rgba, fp16=False):
    _check(lib().rc_tf_set_device(ctx, _ptr(rgba), rgba.shape[0], int(bool(fp16))), ctx, "rc_tf_set_device")


def rc_tf2d_set_device(ctx, rgba, gmax, fp16=False):
    """2-D table from a CUDA float32 tensor of shape (n_grad, n_values, 4)."""
    if rgba.dim() != 3 or rgba.shape[2] != 4:
        raise ValueError("rc_tf2d_set_device: rgba must have shape (n_grad, n_values, 4)")
    _check(lib().rc_tf2d_set_device(ctx, _ptr(rgba), rgba.shape[1], rgba.shape[0], float(gmax), int(bool(fp16))),
           ctx, "rc_tf2d_set_device")


def make_camera(cam) -> rc_camera:
    return rc_camera((C.c_float * 3)(*cam["eye"]), (C.c_float * 3)(*cam["target"]),
                     (C.c_float * 3)(*cam["up"]), float(cam["fovy_deg"]), int(cam["width"]),
                     int(cam["height"]))


def rc_camera_set(ctx, cam):
    c = cam if isinstance(cam, rc_camera) else make_camera(cam)
    _check(lib().rc_camera_set(ctx, C.byref(c)), ctx, "rc_camera_set")


@dataclass
class RenderParams:
    step_vox: float = 0.5
    term: float = 0.99
    shade: bool = False
    ka: float = 0.1
    kd: float = 0.7
    ks: float = 0.2
    func: int = RC_FUNC_COMPOSITE
    iso: float = 0.0
    skip: bool = True
    filter: int = RC_FILTER_TRILINEAR

    def c(self) -> rc_render_params:
        return rc_render_params(self.step_vox, self.term, int(bool(self.shade)), self.ka, self.kd,
                                self.ks, int(self.func), self.iso, int(bool(self.skip)), int(self.filter))


def _params(p):
    if isinstance(p, rc_render_params):
        return p
    if isinstance(p, RenderParams):
        return p.c()
    return RenderParams(**p).c()


def rc_render(ctx, vol, params, out, stats=False):
    """Renders into out (CUDA float32 tensor H x W x 4). With stats=True the
    call synchronises and returns the sample counters."""
    p = _params(params)
    st = rc_stats() if stats else None
    _check(lib().rc_render(ctx, vol, C.byref(p), _ptr(out), C.byref(st) if st is not None else None),
           ctx, "rc_render")
    return _stats_dict(st)


def _stats_dict(st):
    if st is None:
        return None
    return dict(dense_samples=st.dense_samples, evaluated_samples=st.evaluated_samples,
                rays_hit=st.rays_hit, rays_total=st.rays_total, fallback_rays=st.fallback_rays,
                device_ms=st.device_ms)


def rc_render_views(ctx, vol, params, cams, out, stats=False):
    """Renders every camera in one launch into out (CUDA float32 tensor
    n x H x W x 4)."""
    p = _params(params)
    arr = (rc_camera * len(cams))(*[c if isinstance(c, rc_camera) else make_camera(c) for c in cams])
    st = rc_stats() if stats else None
    _check(lib().rc_render_views(ctx, vol, C.byref(p), arr, len(cams), _ptr(out),
                                 C.byref(st) if st is not None else None), ctx, "rc_render_views")
    return _stats_dict(st)


def rc_render_views_host(ctx, vol, params, cams, out, group=0, stats=False):
    """Renders every camera into out, a host float32 tensor n x H x W x 4
    (page-locked for the copies to overlap the rendering), in groups of
    `group` views (0: automatic); returns when the images are in out."""
    p = _params(params)
    arr = (rc_camera * len(cams))(*[c if isinstance(c, rc_camera) else make_camera(c) for c in cams])
    st = rc_stats() if stats else None
    _check(lib().rc_render_views_host(ctx, vol, C.byref(p), arr, len(cams), int(group), _ptr(out),
                                      C.byref(st) if st is not None else None), ctx, "rc_render_views_host")
    return _stats_dict(st)


def rc_render_batch(ctx, vols, params, cams, out, stats=False):
    """Every camera of every volume in one launch (out: CUDA float32
    nvols x nviews x H x W x 4)."""
    p = _params(params)
    varr = (C.c_void_p * len(vols))(*vols)
    arr = (rc_camera * len(cams))(*[c if isinstance(c, rc_camera) else make_camera(c) for c in cams])
    st = rc_stats() if stats else None
    _check(lib().rc_render_batch(ctx, varr, len(vols), C.byref(p), arr, len(cams), _ptr(out),
                                 C.byref(st) if st is not None else None), ctx, "rc_render_batch")
    return _stats_dict(st)


def rc_render_backward(ctx, vol, params, dimage, dtf):
    p = _params(params)
    _check(lib().rc_render_backward(ctx, vol, C.byref(p), _ptr(dimage), _ptr(dtf)), ctx,
           "rc_render_backward")


def rc_render_backward_views(ctx, vol, params, cams, dimages, dtf):
    """Table gradient summed over every camera's view (dimages: CUDA float32 n x H x W x 4)."""
    p = _params(params)
    arr = (rc_camera * len(cams))(*[c if isinstance(c, rc_camera) else make_camera(c) for c in cams])
    _check(lib().rc_render_backward_views(ctx, vol, C.byref(p), arr, len(cams), _ptr(dimages), _ptr(dtf)), ctx,
           "rc_render_backward_views")


def rc_render_backward_noalloc(ctx, vol, params, dimage, dtf):
    """rc_render_backward without any device allocation (static scratch,
    tables of at most 1024 entries); see include/rc.h."""
    p = _params(params)
    _check(lib().rc_render_backward_noalloc(ctx, vol, C.byref(p), _ptr(dimage), _ptr(dtf)), ctx,
           "rc_render_backward_noalloc")


def rc_brick_grid_get(ctx, vol, mn, mx):
    _check(lib().rc_brick_grid_get(ctx, vol, _ptr(mn), _ptr(mx)), ctx, "rc_brick_grid_get")


def rc_skip_mask_get(ctx, vol, occ):
    _check(lib().rc_skip_mask_get(ctx, vol, _ptr(occ)), ctx, "rc_skip_mask_get")


def rc_brick_grid_get_filter(ctx, vol, filter, mn, mx):
    _check(lib().rc_brick_grid_get_filter(ctx, vol, int(filter), _ptr(mn), _ptr(mx)), ctx,
           "rc_brick_grid_get_filter")


def rc_skip_mask_get_filter(ctx, vol, filter, occ):
    _check(lib().rc_skip_mask_get_filter(ctx, vol, int(filter), _ptr(occ)), ctx, "rc_skip_mask_get_filter")


# ---------------------------------------------------------------------------
# learned proposal
# ---------------------------------------------------------------------------
_BLOB_MAGIC = b"RCPROP01"


def pack_proposal_blob(params, m=None, v=None, adam_step=0) -> bytes:
    """The rc_proposal_load blob of include/rc.h (little-endian)."""
    import struct
    p = np.ascontiguousarray(params, dtype="<f4").reshape(-1)
    assert p.size == RC_PROPOSAL_PARAMS
    has_adam = m is not None
    head = _BLOB_MAGIC + struct.pack("<8IQ", 1, 112, 64, 3, 40, 33, RC_PROPOSAL_PARAMS, int(has_adam),
                                     int(adam_step))
    body = p.tobytes()
    if has_adam:
        body += np.ascontiguousarray(m, dtype="<f4").tobytes() + np.ascontiguousarray(v, dtype="<f4").tobytes()
    return head + body


def unpack_proposal_blob(blob: bytes) -> dict:
    import struct
    assert blob[:8] == _BLOB_MAGIC
    vals = struct.unpack("<8IQ", blob[8:48])
    n = vals[6]
    arr = np.frombuffer(blob[48:], dtype="<f4")
    out = dict(params=arr[:n].copy(), adam_step=vals[8])
    if vals[7]:
        out["m"] = arr[n:2 * n].copy()
        out["v"] = arr[2 * n:3 * n].copy()
    return out


def rc_proposal_load(ctx, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib().rc_proposal_load(ctx, buf, len(blob)), ctx, "rc_proposal_load")


def rc_proposal_save(ctx) -> bytes:
    n = C.c_size_t(0)
    _check(lib().rc_proposal_save(ctx, None, 0, C.byref(n)), ctx, "rc_proposal_save")
    buf = C.create_string_buffer(n.value)
    _check(lib().rc_proposal_save(ctx, buf, n.value, C.byref(n)), ctx, "rc_proposal_save")
    return buf.raw[:n.value]


def rc_profiles_generate(ctx, vol, params, out):
    p = _params(params)
    _check(lib().rc_profiles_generate(ctx, vol, C.byref(p), _ptr(out)), ctx, "rc_profiles_generate")


def rc_proposal_features(ctx, vol, params, out):
    p = _params(params)
    _check(lib().rc_proposal_features(ctx, vol, C.byref(p), _ptr(out)), ctx, "rc_proposal_features")


def rc_proposal_forward(ctx, features, n, out):
    _check(lib().rc_proposal_forward(ctx, _ptr(features), int(n), _ptr(out)), ctx, "rc_proposal_forward")


def rc_proposal_grad(ctx, features, targets, n, grad, loss=None):
    _check(lib().rc_proposal_grad(ctx, _ptr(features), _ptr(targets), int(n), _ptr(grad), _ptr(loss)), ctx,
           "rc_proposal_grad")


def rc_proposal_train_step(ctx, features, targets, n, lr, loss=None):
    _check(lib().rc_proposal_train_step(ctx, _ptr(features), _ptr(targets), int(n), float(lr), _ptr(loss)), ctx,
           "rc_proposal_train_step")


def rc_render_importance(ctx, vol, params, pdf, that, nimp, eps, out, fallback=None, stats=False):
    p = _params(params)
    st = rc_stats() if stats else None
    _check(lib().rc_render_importance(ctx, vol, C.byref(p), _ptr(pdf), _ptr(that), int(nimp), float(eps), _ptr(out),
                                      _ptr(fallback), C.byref(st) if st is not None else None), ctx,
           "rc_render_importance")
    return _stats_dict(st)


def rc_render_proposal(ctx, vol, params, nimp, eps, out, fallback=None, stats=False):
    p = _params(params)
    st = rc_stats() if stats else None
    _check(lib().rc_render_proposal(ctx, vol, C.byref(p), int(nimp), float(eps), _ptr(out), _ptr(fallback),
                                    C.byref(st) if st is not None else None), ctx, "rc_render_proposal")
    return _stats_dict(st)


def rc_render_proposal_views(ctx, vol, params, cams, nimp, eps, out, fallback=None, stats=False):
    """Learned-proposal render of every camera (out: CUDA float32 n x H x W x 4)."""
    p = _params(params)
    arr = (rc_camera * len(cams))(*[c if isinstance(c, rc_camera) else make_camera(c) for c in cams])
    st = rc_stats() if stats else None
    _check(lib().rc_render_proposal_views(ctx, vol, C.byref(p), arr, len(cams), int(nimp), float(eps), _ptr(out),
                                          _ptr(fallback), C.byref(st) if st is not None else None), ctx,
           "rc_render_proposal_views")
    return _stats_dict(st)


def _camera_array(cams):
    return (rc_camera * len(cams))(*[c if isinstance(c, rc_camera) else make_camera(c) for c in cams])


def rc_render_importance_views(ctx, vol, params, cams, sampling, lam, pdf, that, nimp, eps, out, fallback=None,
                               stats=False):
    """Importance-sampled render of every camera from given PDFs (pdf: CUDA
    float32 n x H x W x 32 or None for the uniform density, that: n x H x W or
    None for no fallback; out: n x H x W x 4); sampling RC_SAMPLING_*."""
    p = _params(params)
    st = rc_stats() if stats else None
    _check(lib().rc_render_importance_views(ctx, vol, C.byref(p), _camera_array(cams), len(cams), int(sampling),
                                            float(lam), _ptr(pdf), _ptr(that), int(nimp), float(eps), _ptr(out),
                                            _ptr(fallback), C.byref(st) if st is not None else None), ctx,
           "rc_render_importance_views")
    return _stats_dict(st)


def rc_render_proposal_sampled(ctx, vol, params, cams, sampling, lam, nimp, eps, out, fallback=None, stats=False):
    """Learned-proposal render of every camera with the chosen placement of
    the importance samples (RC_SAMPLING_*)."""
    p = _params(params)
    st = rc_stats() if stats else None
    _check(lib().rc_render_proposal_sampled(ctx, vol, C.byref(p), _camera_array(cams), len(cams), int(sampling),
                                            float(lam), int(nimp), float(eps), _ptr(out), _ptr(fallback),
                                            C.byref(st) if st is not None else None), ctx,
           "rc_render_proposal_sampled")
    return _stats_dict(st)


def rc_render_backward_views_with_forward(ctx, vol, params, cams, images, dimages, dtf):
    """rc_render_backward_views given the forward images of the same views
    (images: CUDA float32 n x H x W x 4, as rc_render_views wrote them): one
    march per ray instead of two."""
    p = _params(params)
    _check(lib().rc_render_backward_views_with_forward(ctx, vol, C.byref(p), _camera_array(cams), len(cams),
                                                       _ptr(images), _ptr(dimages), _ptr(dtf)), ctx,
           "rc_render_backward_views_with_forward")
