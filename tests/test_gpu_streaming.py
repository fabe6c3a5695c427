"""Incremental training data (Eq. 5) and budgeted training: romap_observe appends rays and grants iterations only
when the view angle to the last used image exceeds the threshold; romap_train_budget trains the objects that owe
steps, drops each one when its steps are used, and stops at the time budget."""
import ctypes as C

import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, paired_config

pytestmark = pytest.mark.gpu


def _rays(pool, sel):
    arrs = {k: np.ascontiguousarray(pool[k][sel]) for k in ("origin", "dir", "rgb", "depth", "cls")}
    rays = R.romap_rays(arrs["origin"].ctypes.data, arrs["dir"].ctypes.data, arrs["rgb"].ctypes.data,
                        arrs["depth"].ctypes.data, arrs["cls"].ctypes.data)
    return rays, arrs


def _pool_size(ctx, oid):
    n = C.c_int64()
    R.check(R.romap_pool_size(ctx.h, oid, C.byref(n)))
    return n.value


def _pending(ctx, oid):
    n = C.c_int64()
    R.check(R.romap_pending(ctx.h, oid, C.byref(n)))
    return n.value


@pytest.mark.parametrize("precision", [R.ROMAP_PREC_FP32, R.ROMAP_PREC_MIXED_BF16])
def test_observe_follows_the_data_rule(precision):
    import torch  # noqa: F401

    oc, rc = paired_config(precision=precision)
    sc = synth.multi_object_scene(1, seed0=21, n_frames=1, W=64, H=48, f=64.0)[0]
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
        t_o = np.asarray(sc.t, np.float64)
        upd = C.c_int32()
        cams, decisions = [], []
        # cameras on a circle around the object: 0, 10, 20, 30, 40, 70 degrees
        for deg in (0.0, 10.0, 20.0, 30.0, 40.0, 70.0):
            th = np.deg2rad(deg)
            cam = t_o + 2.5 * np.array([np.cos(th), np.sin(th), 0.3])
            rays, keep = _rays(sc.pool, slice(0, 300))
            before = _pool_size(ctx, oid)
            R.check(R.romap_observe(ctx.h, oid, np.ascontiguousarray(cam).ctypes.data, 25.0, C.byref(rays), 300, 0,
                                    300, C.byref(upd)))
            last = next((c for c, d in zip(reversed(cams), reversed(decisions)) if d), None)
            want = O.should_update(last, cam, t_o, 25.0)
            assert bool(upd.value) == want
            assert _pool_size(ctx, oid) == before + (300 if want else 0)
            cams.append(cam)
            decisions.append(want)
        assert decisions == [True, False, False, True, False, True]
        assert _pending(ctx, oid) == 300 * sum(decisions)
    finally:
        ctx.close()


def test_budgeted_training_consumes_owed_steps():
    import torch  # noqa: F401

    oc, rc = paired_config(precision=R.ROMAP_PREC_MIXED_BF16, rays_per_step=512)
    scenes = synth.multi_object_scene(3, seed0=22, n_frames=2, W=64, H=48, f=64.0)
    ctx = Ctx(rc)
    try:
        ids = []
        for sc in scenes:
            oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
            ctx.add_rays(oid, sc.pool)
            ids.append(oid)
        owed = [5, 12, 40]
        for oid, k in zip(ids, owed):
            R.check(R.romap_set_pending(ctx.h, oid, k))
        arr = (C.c_int32 * 3)(*ids)
        steps, ms = C.c_int32(), C.c_float()
        loss = np.zeros(3, np.float32)
        R.check(R.romap_train_budget(ctx.h, arr, 3, 1e6, 8, C.byref(steps), C.byref(ms), loss.ctypes.data))
        assert steps.value == max(owed) and ms.value > 0
        assert all(_pending(ctx, oid) == 0 for oid in ids)
        assert [ctx.state(oid)[3] for oid in ids] == owed
        assert np.isfinite(loss).all()
        # nothing owed: nothing runs
        R.check(R.romap_train_budget(ctx.h, arr, 3, 1e6, 8, C.byref(steps), C.byref(ms), loss.ctypes.data))
        assert steps.value == 0 and np.isnan(loss).all()
        # a known composition and a budget of about 10 steps
        for oid in ids:
            R.check(R.romap_set_pending(ctx.h, oid, 1000))
        R.check(R.romap_train_budget(ctx.h, arr, 3, 3.0, 4, C.byref(steps), C.byref(ms), None))  # its step time
        assert steps.value >= 1
        per = ms.value / steps.value
        R.check(R.romap_train_budget(ctx.h, arr, 3, 0.0, 4, C.byref(steps), C.byref(ms), None))
        assert steps.value == 0
        R.check(R.romap_train_budget(ctx.h, arr, 3, 10.5 * per, 4, C.byref(steps), C.byref(ms), None))
        print(f"\nstep {per:.3f} ms; budget {10.5 * per:.3f} ms -> {steps.value} steps in {ms.value:.3f} ms")
        # about 10 full steps, then single-object steps fill what is left
        assert 5 <= steps.value <= 14 and ms.value <= 1.5 * 10.5 * per
    finally:
        ctx.close()
