"""The deterministic FP32 mode (config field `deterministic`): gradients and loss sums accumulated in 64-bit fixed
point, so that the order in which the GPU's atomics land does not change a bit.

Two runs with the same inputs give bit-identical parameters, moments and losses; a batch of objects gives every
object the bits of its own separate launches; and the gradient still matches the FP64 oracle (Eq. 6-11 and their
adjoints) and the floating-point-atomic FP32 path within the FP32 tolerances."""
import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, assert_grad_close, object_frame_pool, paired_config

pytestmark = pytest.mark.gpu


def _scenes(n=3, seed0=61):
    scenes = synth.multi_object_scene(n, seed0=seed0, n_frames=2, W=80, H=60, f=80.0, depth_frac=0.1)
    occ = [synth.occupancy_bits(sc.shape, sc.half, dilate=2, p=0.05, seed=sc.seed) for sc in scenes]
    return scenes, occ


def _load(ctx, scenes, occ, rays=(300, 700, 1100)):
    ids = []
    for k, (sc, bits) in enumerate(zip(scenes, occ)):
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed, rays_per_step=rays[k % len(rays)])
        ctx.add_rays(oid, sc.pool)
        R.check(R.romap_set_occupancy(ctx.h, oid, np.ascontiguousarray(bits).ctypes.data, 0))
        ids.append(oid)
    return ids


def _config(**kw):
    oc, rc = paired_config(L=16, T=2 ** 14, growth=0.0, n_max=512, n_samples=64, bg_random=True, **kw)
    rc.deterministic = 1
    return oc, rc


def _run(rc, scenes, occ, steps, per_object=False):
    rc.per_object = 1 if per_object else 0
    ctx = Ctx(rc)
    try:
        ids = _load(ctx, scenes, occ)
        losses = [ctx.train(ids) for _ in range(steps)]
        return np.array(losses), [ctx.state(i)[:3] for i in ids]
    finally:
        ctx.close()


def test_deterministic_runs_are_bit_identical():
    import torch  # noqa: F401

    _, rc = _config()
    scenes, occ = _scenes()
    la, sa = _run(rc, scenes, occ, 8)
    lb, sb = _run(rc, scenes, occ, 8)
    assert np.array_equal(la, lb), (la, lb)
    for (pa, ma, va), (pb, mb, vb) in zip(sa, sb):
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb) and np.array_equal(va, vb)
    assert np.all(np.isfinite(la)) and la[-1].mean() < la[0].mean()


def test_deterministic_batch_equals_separate_launches():
    """One batched launch sequence for three uneven objects vs one launch sequence per object (per_object): the same
    bits for every object, its losses included."""
    import torch  # noqa: F401

    _, rc = _config()
    scenes, occ = _scenes()
    lb, sb = _run(rc, scenes, occ, 5)
    ls, ss = _run(rc, scenes, occ, 5, per_object=True)
    assert np.array_equal(lb, ls), (lb, ls)
    for k, ((pa, ma, va), (pb, mb, vb)) in enumerate(zip(sb, ss)):
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb) and np.array_equal(va, vb), k


def test_deterministic_gradient_matches_oracle_and_atomic_path():
    import torch  # noqa: F401

    oc, rc = _config(rays_per_step=1500)
    scenes, occ = _scenes(1, seed0=65)
    sc, bits = scenes[0], occ[0]
    pool = object_frame_pool(sc)
    assert len(np.unique(pool["cls"])) >= 2 and np.isfinite(pool["depth"]).any()
    grads, losses = [], []
    for det in (1, 0):
        rc.deterministic = det
        ctx = Ctx(rc)
        try:
            oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
            ctx.add_rays(oid, sc.pool)
            R.check(R.romap_set_occupancy(ctx.h, oid, np.ascontiguousarray(bits).ctypes.data, 0))
            losses.append(ctx.fwd_bwd([oid])[0])
            grads.append(ctx.grad(oid))
        finally:
            ctx.close()
    p0 = O.init_params(oc, sc.seed)
    ref = O.train_step(oc, sc.half.astype(np.float32), sc.seed, 1, pool, p0, p0 * 0, p0 * 0, occ=bits,
                       do_adam=False)
    assert np.allclose(losses[0], ref["loss"], rtol=1e-5, atol=1e-7), (losses[0], ref["loss"])
    nh = O.hash_param_count(oc)
    assert_grad_close(grads[0][:nh], ref["grad"][:nh], what="hash gradient (deterministic)")
    assert_grad_close(grads[0][nh:], ref["grad"][nh:], what="MLP gradient (deterministic)")
    # against the same step with floating-point atomics: both are FP32 sums of the same contributions
    assert np.allclose(losses[0], losses[1], rtol=1e-5, atol=1e-8)
    assert_grad_close(grads[0], grads[1], tol=1e-5, what="deterministic vs atomic FP32")
    assert np.array_equal(grads[0] != 0, grads[1] != 0)  # the same entries receive gradient


@pytest.mark.parametrize("per_object", [False, True])
def test_pipelined_steps_equal_single_steps(per_object):
    """n_steps > 1 in one call runs each step's sampling beside the previous step's Adam update (a second stream,
    captured as a fork in the step graphs).  In the deterministic mode the result is bit for bit that of the same
    number of one-step calls: parameters, moments, the step counter and the last step's losses, and so is a second
    pipelined call (graph replays) continuing from there."""
    import torch  # noqa: F401

    _, rc = _config()
    rc.per_object = 1 if per_object else 0
    scenes, occ = _scenes()
    out = []
    for pipelined in (False, True):
        ctx = Ctx(rc)
        try:
            ids = _load(ctx, scenes, occ)
            if pipelined:
                la = ctx.train(ids, n_steps=5)
                lb = ctx.train(ids, n_steps=5)
            else:
                la = [ctx.train(ids) for _ in range(5)][-1]
                lb = [ctx.train(ids) for _ in range(5)][-1]
            out.append((la, lb, [ctx.state(i) for i in ids]))
        finally:
            ctx.close()
    (la0, lb0, s0), (la1, lb1, s1) = out
    assert np.array_equal(la0, la1) and np.array_equal(lb0, lb1)
    for (p0, m0, v0, t0), (p1, m1, v1, t1) in zip(s0, s1):
        assert t0 == t1 == 10
        assert np.array_equal(p0, p1) and np.array_equal(m0, m1) and np.array_equal(v0, v1)


def test_pipelined_mixed_steps_train_like_single_steps():
    """The mixed-precision path pipelined the same way: its atomics make single runs differ in the last bits, so the
    parameters after a pipelined call and after one-step calls agree to the rounding of those sums."""
    import torch  # noqa: F401

    _, rc = _config(precision=R.ROMAP_PREC_MIXED_BF16)
    rc.deterministic = 0
    scenes, occ = _scenes()
    out = []
    for pipelined in (False, True):
        ctx = Ctx(rc)
        try:
            ids = _load(ctx, scenes, occ)
            if pipelined:
                losses = ctx.train(ids, n_steps=4)
            else:
                losses = [ctx.train(ids) for _ in range(4)][-1]
            out.append((losses, [ctx.state(i) for i in ids]))
        finally:
            ctx.close()
    (l0, s0), (l1, s1) = out
    assert np.allclose(l0, l1, rtol=1e-3)
    for (p0, _, _, t0), (p1, _, _, t1) in zip(s0, s1):
        assert t0 == t1 == 4
        assert np.abs(p0 - p1).max() <= 1e-3 * np.abs(p0).max()
