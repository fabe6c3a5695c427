"""Helpers shared by the GPU tests: paired oracle/CUDA configurations and a context wrapper over the C ABI."""
import ctypes as C

import numpy as np

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R

# Forward renders: FP32 vs FP64 within 1e-5 relative; gradients within 1e-4 of the largest entry.
FWD_RTOL, FWD_ATOL = 1e-5, 1e-6
GRAD_TOL = 1e-4


def paired_config(L=8, T=2 ** 12, n_min=16, growth=1.5, n_max=0, n_samples=32, rays_per_step=256, dir_dims=3,
                  bg_random=False, lambda1=0.5, lambda2=0.01, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15,
                  max_objects=64, precision=R.ROMAP_PREC_FP32, single_net=False, hidden_layers=1):
    oc = O.make_config(L=L, T=T, n_min=n_min, growth=growth, n_max=n_max, n_samples=n_samples,
                       rays_per_step=rays_per_step, dir_dims=dir_dims, bg_random=bg_random, lambda1=lambda1,
                       lambda2=lambda2, lr=lr, beta1=beta1, beta2=beta2, eps=eps, single_net=single_net,
                       hidden_layers=hidden_layers)
    rc = R.make_config(n_levels=L, log2_table_size=int(np.log2(T)), base_resolution=n_min, growth=growth,
                       max_resolution=n_max, n_samples=n_samples, rays_per_step=rays_per_step, dir_dims=dir_dims,
                       bg_random=bg_random, lambda1=lambda1, lambda2=lambda2, lr=lr, beta1=beta1, beta2=beta2,
                       eps=eps, max_objects=max_objects, precision=precision, single_net=single_net,
                       hidden_layers=hidden_layers)
    # the oracle takes the loss weights and Adam constants in FP64; feed it the FP32 values the GPU uses
    for name in ("lambda1", "lambda2", "lr", "beta1", "beta2", "eps"):
        setattr(oc, name, float(np.float32(getattr(oc, name))))
    return oc, rc


class Ctx:
    """A romap context on torch's current stream."""

    def __init__(self, rc):
        import torch
        self.torch = torch
        self.rc = rc
        self.h = C.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        R.check(R.romap_init(C.byref(rc), C.c_void_p(stream), C.byref(self.h)), "romap_init")
        self.layout = R.param_layout(rc)
        self.n_params = self.layout.n_params

    def close(self):
        if self.h:
            R.check(R.romap_destroy(self.h), "romap_destroy")
            self.h = C.c_void_p()

    def create(self, t=(0, 0, 0), yaw=0.0, half=(0.5, 0.5, 0.5), seed=0, rays_per_step=0):
        oid = C.c_int32()
        d = R.object_desc(t=t, yaw=yaw, half_size=half, seed=seed, rays_per_step=rays_per_step)
        R.check(R.romap_create_object(self.h, C.byref(d), C.byref(oid)), "romap_create_object")
        return oid.value

    def add_rays(self, oid, pool, flags=0):
        o = np.ascontiguousarray(pool["origin"], np.float32)
        d = np.ascontiguousarray(pool["dir"], np.float32)
        rgb = np.ascontiguousarray(pool["rgb"], np.float32)
        dep = None if pool.get("depth") is None else np.ascontiguousarray(pool["depth"], np.float32)
        cls = None if pool.get("cls") is None else np.ascontiguousarray(pool["cls"], np.uint8)
        rays = R.romap_rays(o.ctypes.data, d.ctypes.data, rgb.ctypes.data,
                            None if dep is None else dep.ctypes.data, None if cls is None else cls.ctypes.data)
        R.check(R.romap_add_rays(self.h, oid, C.byref(rays), o.size // 3, flags), "romap_add_rays")

    def ids(self, ids):
        return (C.c_int32 * len(ids))(*ids)

    def fwd_bwd(self, ids):
        loss = np.zeros(5 * len(ids), np.float32)
        R.check(R.romap_forward_backward(self.h, self.ids(ids), len(ids), loss.ctypes.data), "romap_forward_backward")
        return loss.reshape(len(ids), 5)

    def adam(self, ids):
        R.check(R.romap_adam_step(self.h, self.ids(ids), len(ids)), "romap_adam_step")

    def train(self, ids, n_steps=1, want_loss=True):
        loss = np.zeros(len(ids), np.float32)
        R.check(R.romap_train_step(self.h, self.ids(ids), len(ids), n_steps, loss.ctypes.data if want_loss else None),
                "romap_train_step")
        return loss

    def grad(self, oid):
        g = np.zeros(self.n_params, np.float32)
        R.check(R.romap_get_grad(self.h, oid, g.ctypes.data, 0), "romap_get_grad")
        return g

    def state(self, oid):
        p, m, v = (np.zeros(self.n_params, np.float32) for _ in range(3))
        st = R.romap_state(p.ctypes.data, m.ctypes.data, v.ctypes.data, self.n_params, 0, 0)
        R.check(R.romap_get_state(self.h, oid, C.byref(st)), "romap_get_state")
        return p, m, v, st.step

    def set_state(self, oid, p, m=None, v=None, step=0):
        p = np.ascontiguousarray(p, np.float32)
        m = np.zeros_like(p) if m is None else np.ascontiguousarray(m, np.float32)
        v = np.zeros_like(p) if v is None else np.ascontiguousarray(v, np.float32)
        st = R.romap_state(p.ctypes.data, m.ctypes.data, v.ctypes.data, self.n_params, step, 0)
        R.check(R.romap_set_state(self.h, oid, C.byref(st)), "romap_set_state")

    def last_batch(self, oid, B):
        idx = np.zeros(B, np.int64)
        bg = np.zeros((B, 3), np.float32)
        n = C.c_int64()
        R.check(R.romap_last_batch(self.h, oid, idx.ctypes.data, bg.ctypes.data, C.byref(n)), "romap_last_batch")
        assert n.value == B
        return idx, bg

    # functional API on torch device tensors
    def fn_forward(self, params, half, seed, step, o, d, bg, jitter=True, occ=None, want_samples=False,
                   store_act=False):
        torch = self.torch
        n = o.shape[0]
        ws_bytes = C.c_size_t()
        flags = (R.ROMAP_JITTER if jitter else 0) | (R.ROMAP_STORE_ACT if store_act else 0)
        R.check(R.romap_fn_workspace_size(self.h, n, flags, C.byref(ws_bytes)), "romap_fn_workspace_size")
        ws = torch.empty(ws_bytes.value + 256, dtype=torch.uint8, device="cuda")
        out = torch.empty(n, 6, dtype=torch.float32, device="cuda")
        samples = torch.empty(n, self.rc.n_samples, 6, device="cuda") if want_samples else None
        halfa = (C.c_float * 3)(*half)
        R.check(R.romap_fn_forward(self.h, params.data_ptr(), halfa, seed, step, R.ptr(occ), o.data_ptr(),
                                   d.data_ptr(), bg.data_ptr(), n, flags, ws.data_ptr(),
                                   ws.numel(), out.data_ptr(), R.ptr(samples)), "romap_fn_forward")
        return out, samples, ws

    def fn_backward(self, params, half, seed, step, o, d, bg, ws, grad_ray, jitter=True, occ=None, store_act=False):
        torch = self.torch
        n = o.shape[0]
        g = torch.zeros(self.n_params, dtype=torch.float32, device="cuda")
        ds = torch.empty(n, self.rc.n_samples, device="cuda")
        halfa = (C.c_float * 3)(*half)
        R.check(R.romap_fn_backward(self.h, params.data_ptr(), halfa, seed, step, R.ptr(occ), o.data_ptr(),
                                    d.data_ptr(), bg.data_ptr(), n,
                                    (R.ROMAP_JITTER if jitter else 0) | (R.ROMAP_STORE_ACT if store_act else 0),
                                    ws.data_ptr(), ws.numel(), grad_ray.data_ptr(), g.data_ptr(), ds.data_ptr()),
                "romap_fn_backward")
        return g, ds


def object_frame_pool(scene):
    """The oracle's object-frame copy of a synthetic scene's world-frame pool."""
    o, d = O.world_to_object(scene.pool["origin"], scene.pool["dir"], scene.t.astype(np.float32), scene.yaw)
    return dict(o=o.reshape(-1, 3), d=d.reshape(-1, 3), rgb=scene.pool["rgb"], depth=scene.pool["depth"],
                cls=scene.pool["cls"])


def assert_grad_close(g_gpu, g_ref, tol=GRAD_TOL, what="gradient"):
    g_ref = np.asarray(g_ref, np.float64)
    g_gpu = np.asarray(g_gpu, np.float64)
    scale = np.abs(g_ref).max()
    err = np.abs(g_gpu - g_ref)
    worst = (err / (scale + 1e-30)).max()
    assert np.all(err <= tol * scale + tol * np.abs(g_ref)), f"{what}: worst relative error {worst:.3e}"
    return worst
