"""Adam's exact skip of never-touched parameter chunks: parameters, moments and losses are bit-identical to dense
Adam over 20 culled training steps (deterministic FP32 mode, so that the gradients themselves are reproducible),
the skip really leaves untouched table regions alone, and a checkpoint loaded into a fresh context continues with
the same bits (the loaded moments mark the touched chunks)."""
import numpy as np
import pytest

from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, paired_config

pytestmark = pytest.mark.gpu


def _setup(ctx):
    scenes = synth.multi_object_scene(2, seed0=81, n_frames=2, W=80, H=60, f=80.0)
    ids = []
    for k, sc in enumerate(scenes):
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed, rays_per_step=400 + 300 * k)
        ctx.add_rays(oid, sc.pool)
        bits = synth.occupancy_bits(sc.shape, sc.half, dilate=1, p=0.0, seed=sc.seed)
        R.check(R.romap_set_occupancy(ctx.h, oid, np.ascontiguousarray(bits).ctypes.data, 0))
        ids.append(oid)
    return ids


def _config():
    _, rc = paired_config(L=16, T=2 ** 15, growth=0.0, n_max=512, n_samples=64, bg_random=True)
    rc.deterministic = 1
    return rc


def test_adam_skip_is_bit_identical_to_dense_adam():
    import torch  # noqa: F401

    rc = _config()
    res = []
    for skip in (1, 0):
        ctx = Ctx(rc)
        try:
            R.check(R.romap_set_adam_skip(ctx.h, skip))
            ids = _setup(ctx)
            p_init = [ctx.state(i)[0] for i in ids]
            losses = [ctx.train(ids) for _ in range(20)]
            res.append((np.array(losses), [ctx.state(i)[:3] for i in ids], p_init))
        finally:
            ctx.close()
    (la, sa, pinit), (lb, sb, _) = res
    assert np.array_equal(la, lb)
    for (pa, ma, va), (pb, mb, vb), p0 in zip(sa, sb, pinit):
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb) and np.array_equal(va, vb)
        # culled empty space: whole chunks never received a gradient, so they kept their initial values
        untouched = (ma == 0) & (va == 0)
        assert untouched.mean() > 0.05, untouched.mean()
        assert np.array_equal(pa[untouched], p0[untouched])


def test_checkpoint_marks_touched_chunks():
    import torch  # noqa: F401

    rc = _config()
    ctx = Ctx(rc)
    try:
        ids = _setup(ctx)
        for _ in range(6):
            ctx.train(ids)
        saved = [ctx.state(i) for i in ids]
        for _ in range(6):
            ctx.train(ids)
        want = [ctx.state(i)[:3] for i in ids]
    finally:
        ctx.close()
    ctx = Ctx(rc)
    try:
        ids = _setup(ctx)
        for oid, (p, m, v, step) in zip(ids, saved):
            ctx.set_state(oid, p, m, v, step)
        for _ in range(6):
            ctx.train(ids)
        got = [ctx.state(i)[:3] for i in ids]
    finally:
        ctx.close()
    for (pa, ma, va), (pb, mb, vb) in zip(want, got):
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb) and np.array_equal(va, vb)
