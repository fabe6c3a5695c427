"""torch.autograd.Function over the library's forward and adjoint kernels.

``render(params, origin, dir, bg, ...)`` returns per ray (C_hat rgb, D_hat, opacity, sum of sigma) computed by
romap_fn_forward (sampling, hash encoding, MLP, volume rendering of Sec. V-B, Eq. 6); its backward is
romap_fn_backward (compositing adjoint, MLP input and weight gradients, hash-gradient scatter).  For short rays the
forward stores every sample's MLP activations and the backward reads them back (ROMAP_STORE_ACT); when rays get long
(more than ``STORE_MAX_SAMPLES`` samples per ray) the backward recomputes them instead, so memory does not grow with
the activations.  Only ``params`` (the object's hash table and MLP weights, FP32, laid out as romap_param_layout
describes) receives a gradient.  PyTorch provides device memory and streams; every computation runs in libromap's
kernels.
"""
import ctypes as C

import torch

from . import romap as R

# rays with at most this many samples keep their activations between forward and backward; longer ones recompute
STORE_MAX_SAMPLES = 256


class Context:
    """A romap context bound to torch's current stream (config from romap.make_config)."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.h = C.c_void_p()
        R.check(R.romap_init(C.byref(cfg), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(self.h)),
                "romap_init")
        self.layout = R.param_layout(cfg)

    def close(self):
        if self.h:
            R.check(R.romap_destroy(self.h), "romap_destroy")
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, origin, direction, bg, rctx, half, seed, step, jitter, occupancy, store_act):
        n = origin.shape[0]
        flags = (R.ROMAP_JITTER if jitter else 0) | (R.ROMAP_STORE_ACT if store_act else 0)
        ws_bytes = C.c_size_t()
        R.check(R.romap_fn_workspace_size(rctx.h, n, flags, C.byref(ws_bytes)), "romap_fn_workspace_size")
        ws = torch.empty(ws_bytes.value, dtype=torch.uint8, device=params.device)
        out = torch.empty(n, 6, dtype=torch.float32, device=params.device)
        halfa = (C.c_float * 3)(*half)
        R.check(R.romap_fn_forward(rctx.h, params.data_ptr(), halfa, seed, step, R.ptr(occupancy), origin.data_ptr(),
                                   direction.data_ptr(), bg.data_ptr(), n, flags, ws.data_ptr(), ws.numel(),
                                   out.data_ptr(), None), "romap_fn_forward")
        ctx.save_for_backward(params, origin, direction, bg, ws)
        ctx.rctx, ctx.half, ctx.seed, ctx.step, ctx.flags, ctx.occ = rctx, half, seed, step, flags, occupancy
        return out

    @staticmethod
    def backward(ctx, grad_out):
        params, origin, direction, bg, ws = ctx.saved_tensors
        grad = torch.zeros_like(params)
        g = grad_out.contiguous().to(torch.float32)
        halfa = (C.c_float * 3)(*ctx.half)
        R.check(R.romap_fn_backward(ctx.rctx.h, params.data_ptr(), halfa, ctx.seed, ctx.step, R.ptr(ctx.occ),
                                    origin.data_ptr(), direction.data_ptr(), bg.data_ptr(), origin.shape[0],
                                    ctx.flags, ws.data_ptr(), ws.numel(), g.data_ptr(), grad.data_ptr(), None),
                "romap_fn_backward")
        return grad, None, None, None, None, None, None, None, None, None, None


def render(params, origin, direction, bg, rctx, half=(0.5, 0.5, 0.5), seed=0, step=0, jitter=True, occupancy=None,
           recompute=None):
    """Differentiable render of object-frame rays (unit directions).  Returns [n, 6].  recompute: None picks by ray
    length (stored activations up to STORE_MAX_SAMPLES samples per ray), True / False force it."""
    for t in (params, origin, direction, bg):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("params, origin, direction and bg must be contiguous float32 CUDA tensors")
    if recompute is None:
        recompute = rctx.cfg.n_samples > STORE_MAX_SAMPLES
    return RenderFunction.apply(params, origin, direction, bg, rctx, tuple(half), int(seed), int(step), bool(jitter),
                                occupancy, not recompute)
