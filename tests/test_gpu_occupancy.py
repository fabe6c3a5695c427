"""Occupancy update from the learned density (romap_update_occupancy) against the FP64 oracle: per-cell densities
within FP32 tolerance, bits identical away from the threshold, the moving maximum over two updates, and a training
step culled by the learned grid equal to the oracle's step with the same bits."""
import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, assert_grad_close, object_frame_pool, paired_config

pytestmark = pytest.mark.gpu


def _bits_of(d, thr):
    bits = np.zeros(4096, np.uint64)
    for i in np.nonzero(d > thr)[0]:
        bits[i >> 6] |= np.uint64(1) << np.uint64(i & 63)
    return bits


def _unpack(bits):
    return ((bits[:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)).astype(bool).reshape(-1)


def _random_model(oc, seed, scale):
    rng = np.random.default_rng(seed)
    p = O.init_params(oc, seed)
    nh = O.hash_param_count(oc)
    p[:nh] = rng.uniform(-scale, scale, nh)
    return p.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("L,T", [(8, 2 ** 12), (16, 2 ** 16)])
def test_update_matches_oracle(L, T):
    import torch  # noqa: F401

    oc, rc = paired_config(L=L, T=T, growth=0.0, n_max=256)
    half = np.array([0.45, 0.5, 0.35], np.float32)
    ctx = Ctx(rc)
    try:
        oid = ctx.create(half=tuple(half), seed=3)
        p1, p2 = _random_model(oc, 1, 2.0), _random_model(oc, 2, 2.0)
        thr, decay = 1.5, 0.9
        ctx.set_state(oid, p1)
        R.check(R.romap_update_occupancy(ctx.h, oid, decay, thr, 0))
        ctx.set_state(oid, p2)
        R.check(R.romap_update_occupancy(ctx.h, oid, decay, thr, 0))
        bits = np.zeros(4096, np.uint64)
        dens = np.zeros(64 ** 3, np.float32)
        R.check(R.romap_get_occupancy(ctx.h, oid, bits.ctypes.data, dens.ctypes.data))
        s1 = O.density_grid(oc, p1, half)
        s2 = O.density_grid(oc, p2, half)
        d1, _ = O.occupancy_update(s1, decay, thr, np.zeros_like(s1))
        d2, b2 = O.occupancy_update(s2, decay, thr, d1)
        rel = np.abs(dens - d2) / d2
        print(f"\nL={L}: density max rel err {rel.max():.2e}, occupied {(d2 > thr).mean():.3f} of the cells")
        assert rel.max() < 2e-5
        # bits: identical wherever the density is not within rounding of the threshold
        clear = np.abs(d2 - thr) > 1e-4 * thr
        assert np.array_equal(_unpack(bits)[clear], _unpack(b2)[clear])
        assert np.array_equal(bits, _bits_of(dens, thr))  # the kernel's own bits follow its own densities
        # ROMAP_REPLACE restarts the moving maximum
        R.check(R.romap_update_occupancy(ctx.h, oid, decay, thr, R.ROMAP_REPLACE))
        R.check(R.romap_get_occupancy(ctx.h, oid, None, dens.ctypes.data))
        assert np.max(np.abs(dens - s2) / s2) < 2e-5
    finally:
        ctx.close()


def test_training_step_culled_by_learned_grid():
    """The learned grid drives the sampler: the FP32 step with it equals the oracle's step with the same bits, and
    it keeps fewer live samples than the full box."""
    import torch  # noqa: F401

    oc, rc = paired_config(L=8, T=2 ** 12, growth=1.5, n_samples=64, rays_per_step=512, bg_random=True)
    sc = synth.multi_object_scene(1, seed0=12, n_frames=2, W=64, H=48, f=64.0)[0]
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
        ctx.add_rays(oid, sc.pool)
        p = _random_model(oc, 5, 3.0)
        ctx.set_state(oid, p)
        st = R.romap_stats()
        R.check(R.romap_reset_stats(ctx.h))
        ctx.fwd_bwd([oid])
        R.check(R.romap_get_stats(ctx.h, R.C.byref(st)))
        live_full = st.live_samples
        ctx.set_state(oid, p)
        R.check(R.romap_update_occupancy(ctx.h, oid, 0.0, 2.0, 0))
        bits = np.zeros(4096, np.uint64)
        R.check(R.romap_get_occupancy(ctx.h, oid, bits.ctypes.data, None))
        R.check(R.romap_reset_stats(ctx.h))
        loss = ctx.fwd_bwd([oid])[0]
        R.check(R.romap_get_stats(ctx.h, R.C.byref(st)))
        frac = _unpack(bits).mean()
        print(f"\nlearned grid keeps {frac:.3f} of the cells; live samples {st.live_samples} vs {live_full}")
        assert 0.02 < frac < 0.98 and st.live_samples < live_full
        ref = O.train_step(oc, sc.half.astype(np.float32), sc.seed, 1, object_frame_pool(sc), p, p * 0, p * 0,
                           occ=bits, do_adam=False)
        assert np.allclose(loss, ref["loss"], rtol=1e-5, atol=1e-8), (loss, ref["loss"])
        g = ctx.grad(oid)
        nh = O.hash_param_count(oc)
        assert_grad_close(g[:nh], ref["grad"][:nh], what="hash gradient")
        assert_grad_close(g[nh:], ref["grad"][nh:], what="MLP gradient")
    finally:
        ctx.close()


def test_occupancy_argument_errors():
    import torch  # noqa: F401

    oc, rc = paired_config()
    ctx = Ctx(rc)
    try:
        oid = ctx.create(seed=0)
        bits = np.zeros(4096, np.uint64)
        assert R.romap_get_occupancy(ctx.h, oid, bits.ctypes.data, None) == R.ROMAP_ERR_BAD_STATE
        for decay, thr, flags in ((-0.1, 1.0, 0), (1.5, 1.0, 0), (0.5, -1.0, 0), (0.5, float("nan"), 0),
                                  (0.5, float("inf"), 0), (0.5, 1.0, 0x100)):
            assert R.romap_update_occupancy(ctx.h, oid, decay, thr, flags) == R.ROMAP_ERR_INVALID_ARG
        assert R.romap_update_occupancy(ctx.h, 99, 0.5, 1.0, 0) != R.ROMAP_OK
        R.check(R.romap_update_occupancy(ctx.h, oid, 0.5, 1.0, 0))
        R.check(R.romap_get_occupancy(ctx.h, oid, bits.ctypes.data, None))
    finally:
        ctx.close()
