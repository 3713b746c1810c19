"""torch.autograd.Function over the library's render and its hand-written
adjoint: gradients of an image loss with respect to the transfer-function table
(Eq. 4-5 are differentiable in the table entries). Marshalling only: the
forward calls rc_render, the backward calls rc_render_backward_views_with_forward
with the forward's image (one march per ray instead of two).
"""
from __future__ import annotations

import torch

from . import rc_camera_set, rc_render, rc_render_backward_views_with_forward, rc_tf2d_set_device, rc_tf_set_device


def _set_table(handle, tf, gmax):
    if tf.dim() == 3:
        if gmax is None:
            raise ValueError("render_tf: a 2-D table needs gmax")
        rc_tf2d_set_device(handle, tf, gmax)
    else:
        rc_tf_set_device(handle, tf)


class RenderTF(torch.autograd.Function):
    """image = RenderTF.apply(tf, ctx, vol, params, camera, gmax)

    tf: CUDA float32 (K, 4), or (M, K, 4) for a 2-D (value x gradient
    magnitude) table with row spacing gmax, entries in [0, 1]; returns the
    (H, W, 4) premultiplied image. The context's table and camera are set
    from the arguments on every call.
    """

    @staticmethod
    def forward(fctx, tf, handle, vol, params, camera, gmax=None):
        tf = tf.detach().contiguous()
        _set_table(handle, tf, gmax)
        rc_camera_set(handle, camera)
        out = torch.empty((camera["height"], camera["width"], 4), device=tf.device, dtype=torch.float32)
        rc_render(handle, vol, params, out)
        fctx.handle, fctx.vol, fctx.params, fctx.camera, fctx.gmax = handle, vol, params, camera, gmax
        fctx.save_for_backward(tf, out)
        return out

    @staticmethod
    def backward(fctx, gout):
        tf, out = fctx.saved_tensors
        _set_table(fctx.handle, tf, fctx.gmax)
        dtf = torch.empty_like(tf)
        rc_render_backward_views_with_forward(fctx.handle, fctx.vol, fctx.params, [fctx.camera], out,
                                              gout.contiguous(), dtf)
        return dtf, None, None, None, None, None


def render_tf(tf, handle, vol, params, camera, gmax=None):
    return RenderTF.apply(tf, handle, vol, params, camera, gmax)
