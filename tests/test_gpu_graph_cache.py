"""The training step's CUDA graphs are cached per batch composition: alternating single-object calls (the plain
per-object path) capture one graph per object in the first round and only replay afterwards, and give the same bits
as eager launches (deterministic FP32 mode) and as the per_object configuration."""
import ctypes as C

import numpy as np
import pytest

from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, paired_config

pytestmark = pytest.mark.gpu


def _config():
    _, rc = paired_config(L=8, T=2 ** 12, growth=1.5, n_samples=32, rays_per_step=500, bg_random=True)
    rc.deterministic = 1
    return rc


def _load(ctx, scenes):
    ids = []
    for k, sc in enumerate(scenes):
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed, rays_per_step=300 + 200 * k)
        ctx.add_rays(oid, sc.pool)
        ids.append(oid)
    return ids


def _stats(ctx):
    st = R.romap_stats()
    R.check(R.romap_get_stats(ctx.h, C.byref(st)))
    return st


def test_alternating_single_object_calls_replay_cached_graphs():
    import torch  # noqa: F401

    rc = _config()
    scenes = synth.multi_object_scene(3, seed0=91, n_frames=2, W=64, H=48, f=64.0)
    res = []
    for profiling in (0, 1):  # profiling launches eagerly
        ctx = Ctx(rc)
        try:
            R.check(R.romap_set_profiling(ctx.h, profiling))
            ids = _load(ctx, scenes)
            R.check(R.romap_reset_stats(ctx.h))
            losses = []
            for rnd in range(5):
                losses.append([ctx.train([i])[0] for i in ids])
                st = _stats(ctx)
                if not profiling:
                    assert st.graph_captures == 3, (rnd, st.graph_captures)
                    assert st.graph_replays == 3 * rnd, (rnd, st.graph_replays)
                else:
                    assert st.graph_captures == 0 and st.graph_replays == 0
            res.append((np.array(losses), [ctx.state(i)[:3] for i in ids]))
        finally:
            ctx.close()
    (la, sa), (lb, sb) = res
    assert np.array_equal(la, lb)
    for (pa, ma, va), (pb, mb, vb) in zip(sa, sb):
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb) and np.array_equal(va, vb)

    # per_object: one call trains every listed object with its own launch sequence, back to back
    rc.per_object = 1
    ctx = Ctx(rc)
    try:
        ids = _load(ctx, scenes)
        R.check(R.romap_reset_stats(ctx.h))
        lp = []
        for _ in range(5):
            lp.append(ctx.train(ids))
        st = _stats(ctx)
        assert st.graph_captures == 3 and st.graph_replays == 12
        assert np.array_equal(np.array(lp), la)
        for i, (pa, ma, va) in zip(ids, sa):
            p, m, v = ctx.state(i)[:3]
            assert np.array_equal(p, pa) and np.array_equal(m, ma) and np.array_equal(v, va)
        # n_steps > 1 in one call: each object's steps back to back, losses of each object's last step
        l2 = ctx.train(ids, n_steps=2)
        assert np.all(np.isfinite(l2)) and l2.shape == (3,)
    finally:
        ctx.close()


def test_batch_and_single_graphs_coexist():
    """The batched composition and a single-object composition alternate without re-capturing."""
    import torch  # noqa: F401

    rc = _config()
    scenes = synth.multi_object_scene(2, seed0=95, n_frames=2, W=64, H=48, f=64.0)
    ctx = Ctx(rc)
    try:
        ids = _load(ctx, scenes)
        R.check(R.romap_reset_stats(ctx.h))
        for _ in range(4):
            ctx.train(ids)
            ctx.train([ids[0]])
        st = _stats(ctx)
        assert st.graph_captures == 2 and st.graph_replays == 6
        n = C.c_int64()
        R.check(R.romap_last_outputs(ctx.h, ids[0], None, C.byref(n)))
        assert 0 < n.value <= 300  # the last step was the single-object one
        assert R.romap_last_outputs(ctx.h, ids[1], None, C.byref(n)) == R.ROMAP_ERR_BAD_STATE
    finally:
        ctx.close()
