"""torch.autograd.Function over the library's forward and adjoint kernels.

``render(params, origin, dir, bg, ...)`` returns per ray (C_hat rgb, D_hat, opacity, sum of sigma) computed by
romap_fn_forward (sampling, hash encoding, MLP, volume rendering of Sec. V-B, Eq. 6); its backward is
romap_fn_backward (compositing adjoint, MLP input and weight gradients, hash-gradient scatter).  For short rays the
forward stores every sample's MLP activations and the backward reads them back (ROMAP_STORE_ACT); when rays get long
(more than ``STORE_MAX_SAMPLES`` samples per ray) the backward recomputes them instead, so memory does not grow with
the activations.  Only ``params`` (the object's hash table and MLP weights, FP32, laid out as romap_param_layout
describes) receives a gradient.  PyTorch provides device memory and streams; every computation runs in libromap's
kernels.

``step_loss(rctx, ids, params, step)`` is the front of the training step itself, in the context's precision (the
fused tcgen05 kernel for the mixed precisions): for every listed object it loads ``params[k]`` into the object,
draws the rays of training step ``step`` from the object's pool (Sec. V-A), and returns the total loss of Eq. 11 over
that batch together with its four terms; the backward hands back the gradient romap_forward_backward left in the
object's gradient buffer, scaled by the upstream gradient of the total.  The objects of the context serve as the
function's workspace: their parameters, Adam moments (reset to zero) and step counters are overwritten.
"""
import ctypes as C

import numpy as np

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


class StepLossFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rctx, ids, step, *params):
        n = len(ids)
        n_params = rctx.layout.n_params
        dev = params[0].device
        zeros = torch.zeros(n_params, dtype=torch.float32, device=dev)
        for oid, p in zip(ids, params):
            st = R.romap_state(p.data_ptr(), zeros.data_ptr(), zeros.data_ptr(), n_params, step - 1,
                               R.ROMAP_DEVICE_PTR)
            R.check(R.romap_set_state(rctx.h, oid, C.byref(st)), "romap_set_state")
        loss = np.zeros(5 * n, np.float32)
        R.check(R.romap_forward_backward(rctx.h, (C.c_int32 * n)(*ids), n, loss.ctypes.data),
                "romap_forward_backward")
        grads = []
        for oid in ids:
            g = torch.empty(n_params, dtype=torch.float32, device=dev)
            R.check(R.romap_get_grad(rctx.h, oid, g.data_ptr(), R.ROMAP_DEVICE_PTR), "romap_get_grad")
            grads.append(g)
        ctx.save_for_backward(*grads)
        out = torch.from_numpy(loss.reshape(n, 5)).to(dev)
        total, terms = out[:, 0].contiguous(), out[:, 1:].contiguous()
        ctx.mark_non_differentiable(terms)
        return total, terms

    @staticmethod
    def backward(ctx, grad_total, grad_terms):
        grads = ctx.saved_tensors
        return (None, None, None) + tuple(grad_total[k] * g for k, g in enumerate(grads))


def step_loss(rctx, ids, params, step):
    """Per-object total loss (Eq. 11) of training step ``step`` (1-based: the ray draw of the object's step-th
    training step) at the given parameters, differentiable in them.  rctx: a context with ``h`` (romap_ctx) and
    ``layout`` bound to torch's current stream; ids: distinct object ids of that context, each with rays in its pool;
    params: one contiguous FP32 CUDA tensor of n_params per object.  Returns (total [n], terms [n, 4]: the rgb, rr,
    depth and density sums divided by B, not differentiable)."""
    ids = tuple(int(i) for i in ids)
    params = tuple(params)
    if len(ids) != len(params) or not ids:
        raise ValueError("one parameter tensor per listed object is required")
    if len(set(ids)) != len(ids):
        raise ValueError("listed ids must be distinct")
    if step < 1:
        raise ValueError("step counts training steps from 1")
    for p in params:
        if not (p.is_cuda and p.dtype == torch.float32 and p.is_contiguous() and p.numel() == rctx.layout.n_params):
            raise ValueError("params must be contiguous float32 CUDA tensors of n_params elements")
    return StepLossFunction.apply(rctx, ids, int(step), *params)
