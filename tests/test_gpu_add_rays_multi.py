"""romap_add_rays_multi (one keyframe's rays of several objects in one call) against romap_add_rays per object: the
pools it builds give bit-identical per-ray renders (Eq. 6 outputs of a step that uses each whole pool in order) for
host, page-locked host and device inputs, appends and replacements; argument, capacity and non-finite errors leave
every pool unchanged."""
import ctypes as C

import numpy as np
import pytest

from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, paired_config

pytestmark = pytest.mark.gpu
KEYS = ("origin", "dir", "rgb", "depth", "cls")


@pytest.fixture
def torch():
    import torch
    return torch


def _chunks(n_obj=3, sizes=((70, 50), (0, 90), (110, 0))):
    """Per object: its pose and two consecutive ray chunks of its synthetic pool."""
    scenes = synth.multi_object_scene(n_obj, seed0=11, n_frames=2, W=64, H=48, f=64.0, depth_frac=0.3,
                                      occluder_prob=1.0)
    out = []
    for sc, (a, b) in zip(scenes, sizes):
        p = {k: np.ascontiguousarray(sc.pool[k][: a + b]) for k in KEYS}
        out.append((sc, [{k: v[:a] for k, v in p.items()}, {k: v[a: a + b] for k, v in p.items()}]))
    return out


def _concat(parts):
    return {k: np.ascontiguousarray(np.concatenate([p[k] for p in parts])) for k in KEYS}


def _rays(arrs, ptr=lambda a: a.ctypes.data):
    """Ray struct of raw pointers into arrs: the caller keeps arrs referenced until the library has read them."""
    return R.romap_rays(*(ptr(arrs[k]) for k in KEYS))


def _outputs(ctx, ids):
    ctx.fwd_bwd(ids)
    outs = []
    for i in ids:
        n = C.c_int64()
        R.check(R.romap_last_outputs(ctx.h, i, None, C.byref(n)))
        o = np.zeros(6 * n.value, np.float32)
        R.check(R.romap_last_outputs(ctx.h, i, o.ctypes.data, C.byref(n)))
        outs.append(o)
    return outs


def _pool_sizes(ctx, ids):
    out = []
    for i in ids:
        n = C.c_int64()
        R.check(R.romap_pool_size(ctx.h, i, C.byref(n)))
        out.append(n.value)
    return out


def _make(objs):
    _, rc = paired_config(rays_per_step=256)
    ctx = Ctx(rc)
    ids = [ctx.create(t=tuple(sc.t), yaw=sc.yaw, half=tuple(sc.half), seed=sc.seed) for sc, _ in objs]
    return ctx, ids


@pytest.mark.parametrize("mode", ["host", "pinned", "device"])
def test_multi_append_matches_per_object(torch, mode):
    objs = _chunks()
    ref, rid = _make(objs)
    new, nid = _make(objs)
    try:
        for c in range(2):
            for i, (_, ch) in zip(rid, objs):
                if ch[c]["cls"].size:
                    ref.add_rays(i, ch[c])
            parts = [ch[c] for _, ch in objs]
            cat = _concat(parts)
            counts = (C.c_int64 * len(nid))(*[p["cls"].size for p in parts])
            flags = 0
            keep = cat
            if mode == "pinned":
                keep = {k: torch.from_numpy(v).pin_memory() for k, v in cat.items()}
                rays = _rays(keep, lambda t: t.data_ptr())
            elif mode == "device":
                keep = {k: torch.from_numpy(v).cuda() for k, v in cat.items()}
                rays = _rays(keep, lambda t: t.data_ptr())
                flags = R.ROMAP_DEVICE_PTR
            else:
                rays = _rays(cat)
            R.check(R.romap_add_rays_multi(new.h, new.ids(nid), counts, len(nid), C.byref(rays), flags))
            torch.cuda.synchronize()
        assert _pool_sizes(new, nid) == _pool_sizes(ref, rid) == [120, 90, 110]
        for a, b in zip(_outputs(ref, rid), _outputs(new, nid)):
            assert a.size > 0 and np.array_equal(a, b)
    finally:
        ref.close()
        new.close()


def test_multi_replace_and_object_frame(torch):
    objs = _chunks()
    ref, rid = _make(objs)
    new, nid = _make(objs)
    try:
        for i, (_, ch) in zip(rid, objs):
            ref.add_rays(i, _concat(ch))
        all_rays = _concat([_concat(ch) for _, ch in objs])  # referenced until the call has copied it
        R.check(R.romap_add_rays_multi(new.h, new.ids(nid), (C.c_int64 * 3)(*[120, 90, 110]), 3,
                                       C.byref(_rays(all_rays)), 0))
        # replace object 0's pool by its second chunk, empty object 2's (count 0), keep object 1 out of the call
        second = objs[0][1][1]
        ref.add_rays(rid[0], second, R.ROMAP_REPLACE)
        R.check(R.romap_add_rays(ref.h, rid[2], C.byref(_rays(second)), 0, R.ROMAP_REPLACE))
        R.check(R.romap_add_rays_multi(new.h, new.ids([nid[0], nid[2]]), (C.c_int64 * 2)(50, 0), 2,
                                       C.byref(_rays(second)), R.ROMAP_REPLACE))
        assert _pool_sizes(new, nid) == _pool_sizes(ref, rid) == [50, 90, 0]
        a, b = _outputs(ref, rid[:2]), _outputs(new, nid[:2])
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        # object-frame rays: the same arrays appended with ROMAP_OBJECT_FRAME by both calls
        third = objs[1][1][1]
        ref.add_rays(rid[1], third, R.ROMAP_OBJECT_FRAME)
        R.check(R.romap_add_rays_multi(new.h, new.ids([nid[1]]), (C.c_int64 * 1)(90), 1, C.byref(_rays(third)),
                                       R.ROMAP_OBJECT_FRAME))
        assert _pool_sizes(new, nid) == _pool_sizes(ref, rid) == [50, 180, 0]
        a, b = _outputs(ref, rid[:2]), _outputs(new, nid[:2])
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    finally:
        ref.close()
        new.close()


def test_multi_errors_leave_pools_unchanged(torch):
    objs = _chunks()
    ctx, ids = _make(objs)
    try:
        cat = _concat([ch[0] for _, ch in objs])
        counts = (C.c_int64 * 3)(70, 0, 110)
        R.check(R.romap_add_rays_multi(ctx.h, ctx.ids(ids), counts, 3, C.byref(_rays(cat)), 0))
        before = _pool_sizes(ctx, ids)
        dup = ctx.ids([ids[0], ids[0]])
        assert R.romap_add_rays_multi(ctx.h, dup, (C.c_int64 * 2)(1, 1), 2, C.byref(_rays(cat)), 0) == \
            R.ROMAP_ERR_INVALID_ARG
        assert R.romap_add_rays_multi(ctx.h, ctx.ids(ids), (C.c_int64 * 3)(70, -1, 110), 3, C.byref(_rays(cat)), 0) \
            == R.ROMAP_ERR_INVALID_ARG
        big = (C.c_int64 * 3)(70, 1 << 40, 110)
        assert R.romap_add_rays_multi(ctx.h, ctx.ids(ids), big, 3, C.byref(_rays(cat)), 0) == R.ROMAP_ERR_CAPACITY
        bad = {k: v.copy() for k, v in cat.items()}
        bad["rgb"][150, 1] = np.nan  # a ray of the third object
        assert R.romap_add_rays_multi(ctx.h, ctx.ids(ids), counts, 3, C.byref(_rays(bad)), 0) == \
            R.ROMAP_ERR_NONFINITE
        bad = {k: v.copy() for k, v in cat.items()}
        bad["cls"][3] = 7
        assert R.romap_add_rays_multi(ctx.h, ctx.ids(ids), counts, 3, C.byref(_rays(bad)), 0) == \
            R.ROMAP_ERR_INVALID_ARG
        assert _pool_sizes(ctx, ids) == before == [70, 0, 110]
    finally:
        ctx.close()
