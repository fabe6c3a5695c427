"""Asynchronous training steps: romap_train_step_async returns the same per-object losses as romap_train_step (copied
into page-locked host memory after the stream passes the call), romap_add_rays_multi with ROMAP_ASYNC_HOST builds the
same pools as without it, and a non-finite loss of an asynchronous step is reported by romap_check_device_status,
after which the context stays usable."""
import ctypes as C

import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, paired_config

pytestmark = pytest.mark.gpu
KEYS = ("origin", "dir", "rgb", "depth", "cls")


@pytest.fixture
def torch():
    import torch
    return torch


def _objects(ctx, scenes):
    ids = []
    for sc in scenes:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, half=tuple(sc.half), seed=sc.seed, rays_per_step=300)
        ctx.add_rays(oid, sc.pool)
        ids.append(oid)
    return ids


@pytest.mark.parametrize("precision", [R.ROMAP_PREC_FP32, R.ROMAP_PREC_MIXED_BF16])
def test_async_step_losses_match_sync(torch, precision):
    scenes = synth.multi_object_scene(3, seed0=31, n_frames=2, W=64, H=48, f=64.0)
    _, rc = paired_config(precision=precision, bg_random=True)
    a, b = Ctx(rc), Ctx(rc)
    try:
        ia, ib = _objects(a, scenes), _objects(b, scenes)
        out = torch.zeros(len(ib), dtype=torch.float32, pin_memory=True)
        for step in range(4):
            la = a.train(ia)
            R.check(R.romap_train_step_async(b.h, b.ids(ib), len(ib), 1, C.c_void_p(out.data_ptr())))
            torch.cuda.synchronize()
            lb = out.numpy().copy()
            # the first step sees identical inputs; later steps differ only by the order of atomic additions
            tol = 1e-6 if step == 0 else (1e-5 if precision == R.ROMAP_PREC_FP32 else 1e-3)
            assert np.allclose(lb, la, rtol=tol, atol=0), (step, la, lb)
        assert R.romap_check_device_status(b.h) == R.ROMAP_OK
        # several steps in one call: the losses are those of the last one
        R.check(R.romap_train_step_async(b.h, b.ids(ib), len(ib), 3, C.c_void_p(out.data_ptr())))
        la = a.train(ia, n_steps=3)
        torch.cuda.synchronize()
        assert np.allclose(out.numpy(), la, rtol=1e-2)
    finally:
        a.close()
        b.close()


def test_async_host_rays_build_the_same_pools(torch):
    scenes = synth.multi_object_scene(2, seed0=33, n_frames=2, W=64, H=48, f=64.0, depth_frac=0.3)
    _, rc = paired_config(rays_per_step=256)
    outs = []
    for flags in (0, R.ROMAP_ASYNC_HOST):
        ctx = Ctx(rc)
        try:
            ids = [ctx.create(t=tuple(sc.t), yaw=sc.yaw, half=tuple(sc.half), seed=sc.seed) for sc in scenes]
            parts = [{k: np.ascontiguousarray(sc.pool[k][:200]) for k in KEYS} for sc in scenes]
            pinned = {k: torch.from_numpy(np.concatenate([p[k] for p in parts])).pin_memory() for k in KEYS}
            rays = R.romap_rays(*(pinned[k].data_ptr() for k in KEYS))
            counts = (C.c_int64 * 2)(200, 200)
            R.check(R.romap_add_rays_multi(ctx.h, ctx.ids(ids), counts, 2, C.byref(rays), flags))
            torch.cuda.synchronize()  # the pinned arrays stay alive until here
            ctx.fwd_bwd(ids)
            per = []
            for i in ids:
                n = C.c_int64()
                R.check(R.romap_last_outputs(ctx.h, i, None, C.byref(n)))
                o = np.zeros(6 * n.value, np.float32)
                R.check(R.romap_last_outputs(ctx.h, i, o.ctypes.data, C.byref(n)))
                per.append(o)
            outs.append(per)
        finally:
            ctx.close()
    assert all(x.size > 0 and np.array_equal(x, y) for x, y in zip(*outs))


def test_async_nonfinite_loss_reported_by_status_check(torch):
    oc, rc = paired_config()
    ctx = Ctx(rc)
    try:
        sc = synth.config0_scene()
        oid = ctx.create(seed=0)
        dev = {k: torch.tensor(v, device="cuda") for k, v in sc.pool.items()}
        dev["rgb"][::7, 0] = float("nan")
        rays = R.romap_rays(*(dev[k].data_ptr() for k in KEYS))
        R.check(R.romap_add_rays(ctx.h, oid, R.C.byref(rays), sc.pool["cls"].size, R.ROMAP_DEVICE_PTR))
        out = torch.zeros(1, dtype=torch.float32, pin_memory=True)
        R.check(R.romap_train_step_async(ctx.h, ctx.ids([oid]), 1, 1, C.c_void_p(out.data_ptr())))
        assert R.romap_check_device_status(ctx.h) == R.ROMAP_ERR_NONFINITE
        assert not np.isfinite(out.numpy()).all()
        assert R.romap_check_device_status(ctx.h) == R.ROMAP_OK  # cleared
        ctx.add_rays(oid, sc.pool, flags=R.ROMAP_REPLACE)
        ctx.set_state(oid, O.init_params(oc, 0))
        R.check(R.romap_train_step_async(ctx.h, ctx.ids([oid]), 1, 1, C.c_void_p(out.data_ptr())))
        assert R.romap_check_device_status(ctx.h) == R.ROMAP_OK
        assert np.isfinite(out.numpy()).all()
    finally:
        ctx.close()
