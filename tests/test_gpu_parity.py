"""CUDA path vs the CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import FWD_ATOL, FWD_RTOL, Ctx, assert_grad_close, object_frame_pool, paired_config

pytestmark = pytest.mark.gpu


@pytest.fixture
def torch():
    import torch
    return torch


def _rays_at_box(n, rng, half=0.5, miss_frac=0.1):
    o = np.zeros((n, 3)); d = np.zeros((n, 3))
    for r in range(n):
        az, el = rng.uniform(-np.pi, np.pi), rng.uniform(-0.6, 0.9)
        cam = rng.uniform(1.5, 3.0) * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        tgt = rng.uniform(-half, half, 3) * (3.0 if rng.uniform() < miss_frac else 0.9)
        dd = tgt - cam
        o[r], d[r] = cam, dd / np.linalg.norm(dd)
    return o.astype(np.float32), d.astype(np.float32)


# ---------------------------------------------------------------------------
# bit-exact stages
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 12345, (7 << 32) + 3])
def test_init_params_bit_exact(torch, seed):
    oc, rc = paired_config(L=16, T=2 ** 16, growth=0.0, n_max=512)
    ctx = Ctx(rc)
    try:
        oid = ctx.create(seed=seed)
        p, m, v, step = ctx.state(oid)
        ref = O.init_params(oc, seed).astype(np.float32)
        assert np.array_equal(p, ref)
        assert not m.any() and not v.any() and step == 0
    finally:
        ctx.close()


@pytest.mark.parametrize("N,use_occ", [(32, False), (64, False), (128, True), (1024, False)])
def test_sample_positions_bit_exact(torch, N, use_occ):
    oc, rc = paired_config(L=4, T=2 ** 10, growth=2.0, n_samples=N)
    rng = np.random.default_rng(N)
    n = 300 if N <= 128 else 40
    o, d = _rays_at_box(n, rng)
    half = np.array([0.5, 0.4, 0.3], np.float32)
    occ = None
    if use_occ:
        occ = synth.occupancy_bits(synth.Shape(kind="ellipsoid", axes=np.array([0.3, 0.25, 0.2])), half, dilate=1,
                                   p=0.05, seed=3)
    ctx = Ctx(rc)
    try:
        params = torch.tensor(O.init_params(oc, 4).astype(np.float32), device="cuda")
        to = lambda a: torch.tensor(a, device="cuda")
        occ_t = None if occ is None else torch.tensor(occ.view(np.int64), device="cuda")
        out, samples, _ = ctx.fn_forward(params, half, 99, 5, to(o), to(d), to(np.ones((n, 3), np.float32)),
                                         jitter=True, occ=occ_t, want_samples=True)
        smp = samples.cpu().numpy()
        n_live = 0
        for r in range(n):
            s = O.sample_ray(o[r], d[r], half, N, seed=99, step=5, slot=r, jitter=True, occ=occ)
            live = s["live"] & s["hit"]
            n_live += live.sum()
            got = smp[r]
            assert np.array_equal(got[live, 0], s["t"][live]), r
            assert np.array_equal(got[live, 1], s["delta"][live]), r
            assert np.array_equal(got[live, 2:5], s["x"][live]), r
            assert np.all(got[~live] == 0.0)
            assert np.all(got[live, 5] > 0.0)
        assert n_live > 0
    finally:
        ctx.close()


def test_world_to_object_transform_bit_exact(torch):
    """Rendering world-frame rays equals the functional forward on the oracle's object-frame copy of them (same
    midpoint samples and background), bit for bit: the device transform matches the oracle's FP32 transform."""
    oc, rc = paired_config()
    rng = np.random.default_rng(1)
    o_obj, d_obj = _rays_at_box(200, rng)
    t, yaw = np.array([0.7, -1.3, 0.25], np.float32), 0.83
    Rz = synth.yaw_matrix(yaw)
    o_w = (o_obj.astype(np.float64) @ Rz.T + t).astype(np.float32)
    d_w = (d_obj.astype(np.float64) @ Rz.T * 1.7).astype(np.float32)
    oo, do = O.world_to_object(o_w, d_w, t, yaw)
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(t), yaw=yaw, seed=3)
        bgv = (0.2, 0.3, 0.4)
        bg = (R.C.c_float * 3)(*bgv)
        rgb = np.zeros((200, 3), np.float32); dep = np.zeros(200, np.float32); op = np.zeros(200, np.float32)
        R.check(R.romap_render(ctx.h, oid, o_w.ctypes.data, d_w.ctypes.data, 200, bg, rgb.ctypes.data,
                               dep.ctypes.data, op.ctypes.data, 0), "romap_render")
        params = torch.tensor(ctx.state(oid)[0], device="cuda")
        to = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32).reshape(-1, 3), device="cuda")
        out, _, _ = ctx.fn_forward(params, (0.5, 0.5, 0.5), 3, 0, to(oo), to(do), to(np.tile(bgv, (200, 1))),
                                   jitter=False)
        out = out.cpu().numpy()
        assert np.array_equal(rgb, out[:, :3]) and np.array_equal(dep, out[:, 3]) and np.array_equal(op, out[:, 4])
        assert (op > 0).sum() > 100
    finally:
        ctx.close()


def test_ray_draw_and_background_bit_exact(torch):
    oc, rc = paired_config(L=4, T=2 ** 10, growth=2.0, n_samples=16, rays_per_step=512, bg_random=True)
    sc = synth.multi_object_scene(1, seed0=4, n_frames=2, W=64, H=48, f=64.0)[0]
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=77)
        ctx.add_rays(oid, sc.pool)
        n_pool = sc.pool["cls"].size
        assert n_pool > 512
        for step in (1, 2):
            ctx.fwd_bwd([oid])
            idx, bg = ctx.last_batch(oid, 512)
            ref_idx, ref_bg = O.draw_batch(oc, 77, step, n_pool)
            assert np.array_equal(idx, ref_idx)
            assert np.array_equal(bg, ref_bg.astype(np.float32))
            ctx.adam([oid])
    finally:
        ctx.close()


# ---------------------------------------------------------------------------
# forward renders and gradients of the functional API
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cfg_kw,N,n", [
    (dict(L=8, T=2 ** 12, growth=1.5), 32, 256),                     # plain-method configuration
    (dict(L=4, T=2 ** 10, growth=2.0), 16, 64),                      # differentiation-check configuration
    (dict(L=4, T=2 ** 10, growth=2.0), 1024, 16),                    # long rays
    (dict(L=16, T=2 ** 16, growth=0.0, n_max=512), 64, 128),         # multi-object configuration
])
def test_fn_forward_backward_parity(torch, cfg_kw, N, n):
    oc, rc = paired_config(n_samples=N, **cfg_kw)
    rng = np.random.default_rng(N + n)
    o, d = _rays_at_box(n, rng)
    bg = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    half = np.array([0.5, 0.5, 0.5], np.float32)
    p64 = O.init_params(oc, 11)
    nh = O.hash_param_count(oc)
    p64[:nh] = rng.uniform(-1, 1, nh)  # non-trivial features and densities
    p32 = p64.astype(np.float32)
    up = rng.normal(size=(n, 6)).astype(np.float32)
    ref = O.rays_loss_grad(oc, p32.astype(np.float64), half, 31, 9, o, d, bg=bg.astype(np.float64),
                           upstream=up.astype(np.float64), inv_B=1.0, want_samples=True)
    ctx = Ctx(rc)
    try:
        to = lambda a: torch.tensor(a, device="cuda")
        params = to(p32)
        out, _, ws = ctx.fn_forward(params, half, 31, 9, to(o), to(d), to(bg))
        got = out.cpu().numpy()
        assert np.allclose(got[:, :5], ref["ray"][:, :5], rtol=FWD_RTOL, atol=FWD_ATOL), \
            np.abs(got[:, :5] - ref["ray"][:, :5]).max()
        assert np.allclose(got[:, 5], ref["ray"][:, 5], rtol=FWD_RTOL, atol=FWD_ATOL * N)
        g, ds = ctx.fn_backward(params, half, 31, 9, to(o), to(d), to(bg), ws, to(up))
        g = g.cpu().numpy()
        assert_grad_close(g[:nh], ref["grad"][:nh], what="hash gradient")
        assert_grad_close(g[nh:], ref["grad"][nh:], what="MLP gradient")
        assert_grad_close(ds.cpu().numpy().reshape(-1), ref["samples"][:, :, 7].reshape(-1), what="dL/dsigma")
    finally:
        ctx.close()


# ---------------------------------------------------------------------------
# the training step
# ---------------------------------------------------------------------------
def _load_scene0(ctx):
    sc = synth.config0_scene()
    oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=0)
    ctx.add_rays(oid, sc.pool)
    return sc, oid


def test_train_step_parity_plain_config(torch):
    """Plain method, 1 object, one forward+backward+Adam step, seed 0."""
    oc, rc = paired_config()
    ctx = Ctx(rc)
    try:
        sc, oid = _load_scene0(ctx)
        pool = object_frame_pool(sc)
        p0 = O.init_params(oc, 0)
        ref = O.train_step(oc, sc.half.astype(np.float32), 0, 1, pool, p0, np.zeros_like(p0), np.zeros_like(p0))
        loss = ctx.fwd_bwd([oid])[0]
        assert np.allclose(loss, ref["loss"], rtol=1e-5, atol=1e-7), (loss, ref["loss"])
        g = ctx.grad(oid)
        nh = O.hash_param_count(oc)
        assert_grad_close(g[:nh], ref["grad"][:nh], what="hash gradient")
        assert_grad_close(g[nh:], ref["grad"][nh:], what="MLP gradient")
        ctx.adam([oid])
        p1, m1, v1, step = ctx.state(oid)
        assert step == 1
        # Adam applied by the oracle to the GPU's own gradient
        pa, ma, va = O.adam(p0.astype(np.float32).astype(np.float64), np.zeros_like(p0), np.zeros_like(p0),
                            g.astype(np.float64), 1, oc.lr, oc.beta1, oc.beta2, oc.eps)
        assert np.allclose(p1, pa, rtol=1e-6, atol=1e-7)
        assert np.allclose(m1, ma, rtol=1e-5, atol=1e-12) and np.allclose(v1, va, rtol=1e-5, atol=1e-20)
        # and the oracle's own step where the gradient is well above rounding
        big = np.abs(ref["grad"]) > 1e-3 * np.abs(ref["grad"]).max()
        assert np.allclose(p1[big], ref["params"][big], rtol=1e-6, atol=1e-6)
        assert not ctx.grad(oid).any()  # Adam zeroes the gradient
    finally:
        ctx.close()


def test_training_loss_decreases_plain_config(torch):
    oc, rc = paired_config()
    ctx = Ctx(rc)
    try:
        _, oid = _load_scene0(ctx)
        losses = [ctx.train([oid])[0] for _ in range(30)]
        assert losses[-1] < 0.3 * losses[0], losses
    finally:
        ctx.close()


def test_masked_losses_parity(torch):
    """Object, background (random colour + density loss), occluder and depth rays, posed object."""
    oc, rc = paired_config(L=8, T=2 ** 12, growth=1.5, n_samples=32, rays_per_step=2048, bg_random=True)
    sc = synth.multi_object_scene(1, seed0=5, n_frames=3, W=80, H=60, f=80.0, depth_frac=0.2, occluder_prob=1.0)[0]
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=5)
        ctx.add_rays(oid, sc.pool)
        pool = object_frame_pool(sc)
        assert len(np.unique(pool["cls"])) == 3 and np.isfinite(pool["depth"]).any()
        p0 = O.init_params(oc, 5)
        loss = ctx.fwd_bwd([oid])[0]
        ref = O.train_step(oc, sc.half.astype(np.float32), 5, 1, pool, p0, p0 * 0, p0 * 0, do_adam=False)
        assert np.allclose(loss, ref["loss"], rtol=1e-5, atol=1e-7), (loss, ref["loss"])
        g = ctx.grad(oid)
        nh = O.hash_param_count(oc)
        assert_grad_close(g[:nh], ref["grad"][:nh], what="hash gradient")
        assert_grad_close(g[nh:], ref["grad"][nh:], what="MLP gradient")
    finally:
        ctx.close()


def test_batched_objects_equal_separate_launches(torch):
    oc, rc = paired_config(L=8, T=2 ** 12, growth=1.5, n_samples=32, rays_per_step=700, bg_random=True)
    scenes = synth.multi_object_scene(4, seed0=11, n_frames=2, W=64, H=48, f=64.0)
    ctx = Ctx(rc)
    try:
        ids = []
        for sc in scenes:
            oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed, rays_per_step=300 + 150 * len(ids))
            ctx.add_rays(oid, sc.pool)
            ids.append(oid)
        lb = ctx.fwd_bwd(ids)
        gb = [ctx.grad(i) for i in ids]
        ctx2 = Ctx(rc)
        try:
            for k, sc in enumerate(scenes):
                oid = ctx2.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed, rays_per_step=300 + 150 * k)
                ctx2.add_rays(oid, sc.pool)
                ls = ctx2.fwd_bwd([oid])
                assert np.allclose(ls[0], lb[k], rtol=1e-5, atol=1e-8)  # FP32 atomic sums, any order
                assert_grad_close(ctx2.grad(oid), gb[k], tol=1e-5, what=f"object {k}")
        finally:
            ctx2.close()
    finally:
        ctx.close()


def test_checkpoint_roundtrip_continues_training(torch):
    oc, rc = paired_config()
    ctx = Ctx(rc)
    try:
        sc, oid = _load_scene0(ctx)
        ctx.train([oid], n_steps=3, want_loss=False)
        p, m, v, step = ctx.state(oid)
        assert step == 3
        a = ctx.train([oid], n_steps=2)
        oid2 = ctx.create(seed=0)
        ctx.add_rays(oid2, sc.pool)
        ctx.set_state(oid2, p, m, v, step)
        b = ctx.train([oid2], n_steps=2)
        assert np.allclose(a, b, rtol=1e-5)
        assert np.allclose(ctx.state(oid)[0], ctx.state(oid2)[0], rtol=1e-4, atol=1e-6)
    finally:
        ctx.close()


# ---------------------------------------------------------------------------
# failures are reported, not hidden (host-side injection only)
# ---------------------------------------------------------------------------
def test_errors_are_reported(torch):
    oc, rc = paired_config(max_objects=2)
    ctx = Ctx(rc)
    try:
        a = ctx.create(seed=1)
        b = ctx.create(seed=2)
        with pytest.raises(R.RomapError) as e:
            ctx.create(seed=3)
        assert e.value.status == R.ROMAP_ERR_CAPACITY
        with pytest.raises(R.RomapError) as e:
            ctx.train([a])                       # no rays yet
        assert e.value.status == R.ROMAP_ERR_BAD_STATE
        with pytest.raises(R.RomapError) as e:
            ctx.train([a, a])
        assert e.value.status == R.ROMAP_ERR_INVALID_ARG
        with pytest.raises(R.RomapError) as e:
            ctx.train([5])
        assert e.value.status == R.ROMAP_ERR_NOT_FOUND
        pool = dict(origin=np.zeros((4, 3)), dir=np.ones((4, 3)), rgb=np.zeros((4, 3)))
        pool["origin"][2, 1] = np.nan
        with pytest.raises(R.RomapError) as e:
            ctx.add_rays(a, pool)
        assert e.value.status == R.ROMAP_ERR_NONFINITE
        R.check(R.romap_destroy_object(ctx.h, b))
        with pytest.raises(R.RomapError) as e:
            ctx.grad(b)
        assert e.value.status == R.ROMAP_ERR_NOT_FOUND
    finally:
        ctx.close()


def test_allocation_failure_is_reported(torch):
    """A caller allocator that refuses: the library reports ROMAP_ERR_OOM and stays usable."""
    state = {"fail": False, "live": {}}

    def alloc(user, n):
        if state["fail"]:
            return None
        t = torch.empty(int(n), dtype=torch.uint8, device="cuda")
        state["live"][t.data_ptr()] = t
        return t.data_ptr()

    def dealloc(user, p):
        state["live"].pop(p, None)

    oc, rc = paired_config()
    rc.alloc, rc.dealloc = R.ALLOC_FN(alloc), R.DEALLOC_FN(dealloc)
    ctx = Ctx(rc)
    try:
        oid = ctx.create(seed=1)
        state["fail"] = True
        with pytest.raises(R.RomapError) as e:
            ctx.create(seed=2)
        assert e.value.status == R.ROMAP_ERR_OOM
        state["fail"] = False
        sc = synth.config0_scene()
        ctx.add_rays(oid, sc.pool)
        assert np.isfinite(ctx.train([oid])[0])
    finally:
        ctx.close()
    assert not state["live"]


@pytest.mark.parametrize("precision", [R.ROMAP_PREC_FP32, R.ROMAP_PREC_MIXED_BF16])
def test_graph_replay_matches_eager_launches(torch, precision):
    """romap_train_step replays a captured CUDA graph after its first step; with profiling on it launches eagerly.
    Both give the same losses step by step, and the same parameters after 6 steps."""
    oc, rc = paired_config(L=8, T=2 ** 12, growth=1.5, n_samples=32, rays_per_step=600, bg_random=True,
                           precision=precision)
    scenes = synth.multi_object_scene(3, seed0=31, n_frames=2, W=64, H=48, f=64.0)
    res = []
    for profiling in (0, 1):
        ctx = Ctx(rc)
        try:
            R.check(R.romap_set_profiling(ctx.h, profiling))
            ids = []
            for sc in scenes:
                oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
                ctx.add_rays(oid, sc.pool)
                ids.append(oid)
            losses = [ctx.train(ids) for _ in range(3)]
            losses.append(ctx.train(ids, n_steps=3))
            ctx.adam([ids[0]])  # another batch through the same buffers, then more graph replays
            losses.append(ctx.train(ids))
            res.append((np.array(losses), [ctx.state(i)[0] for i in ids]))
        finally:
            ctx.close()
    (la, pa), (lb, pb) = res
    assert np.allclose(la, lb, rtol=1e-4, atol=1e-7), (la, lb)
    # Adam moves a parameter whose gradient is within rounding of zero by about +-lr, and FP32 atomics sum in a
    # different order in every run: compare parameters as a whole, and entry by entry for almost all of them (runs
    # of this case have shown 0.7% of the entries flipped after 7 steps).
    for x, y in zip(pa, pb):
        assert np.linalg.norm(x - y) <= 1e-2 * np.linalg.norm(y)
        assert np.mean(np.isclose(x, y, rtol=1e-3, atol=1e-5)) > 0.985


def test_device_wait_timeout_is_reported_and_context_survives(torch):
    """A bounded device wait that nothing signals gives up and reports ROMAP_ERR_TIMEOUT; training continues."""
    oc, rc = paired_config(precision=R.ROMAP_PREC_MIXED_BF16)
    ctx = Ctx(rc)
    try:
        assert R.romap_selftest_wait_timeout(ctx.h, 1 << 14) == R.ROMAP_ERR_TIMEOUT
        assert "gave up" in R.last_error()
        sc = synth.config0_scene()
        oid = ctx.create(seed=0)
        ctx.add_rays(oid, sc.pool)
        assert np.isfinite(ctx.train([oid], n_steps=2)).all()
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", [R.ROMAP_PREC_FP32, R.ROMAP_PREC_MIXED_BF16])
def test_nonfinite_device_rays_reported_through_status_word(torch, precision):
    """Device-pointer rays skip the host-side finiteness check; a NaN target reaches the loss and the device status
    word turns it into ROMAP_ERR_NONFINITE; the context stays usable."""
    oc, rc = paired_config(precision=precision)
    ctx = Ctx(rc)
    try:
        sc = synth.config0_scene()
        oid = ctx.create(seed=0)
        dev = {k: torch.tensor(v, device="cuda") for k, v in sc.pool.items()}
        dev["rgb"][::7, 0] = float("nan")
        rays = R.romap_rays(dev["origin"].data_ptr(), dev["dir"].data_ptr(), dev["rgb"].data_ptr(),
                            dev["depth"].data_ptr(), dev["cls"].data_ptr())
        R.check(R.romap_add_rays(ctx.h, oid, R.C.byref(rays), sc.pool["cls"].size, R.ROMAP_DEVICE_PTR))
        with pytest.raises(R.RomapError) as e:
            ctx.train([oid])
        assert e.value.status == R.ROMAP_ERR_NONFINITE
        ctx.add_rays(oid, sc.pool, flags=R.ROMAP_REPLACE)
        ctx.set_state(oid, O.init_params(oc, 0))
        assert np.isfinite(ctx.train([oid])).all()
    finally:
        ctx.close()


def test_accuracy_mode_tightens_long_ray_renders(torch):
    """With the FP64 transmittance log-sum (accuracy_mode), 1024-sample renders of dense rays come closer to the FP64
    oracle than the FP32 scan does; both stay within the forward tolerance."""
    errs = {}
    n, N = 256, 1024
    rng = np.random.default_rng(77)
    o, d = _rays_at_box(n, rng)
    bg = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    half = np.array([0.5, 0.5, 0.5], np.float32)
    for acc in (0, 1):
        oc, rc = paired_config(L=4, T=2 ** 10, growth=2.0, n_samples=N)
        rc.accuracy_mode = acc
        p64 = O.init_params(oc, 12)
        nh = O.hash_param_count(oc)
        p64[:nh] = np.random.default_rng(5).uniform(-3, 3, nh)  # dense regions: long transmittance sums
        p32 = p64.astype(np.float32)
        ref = O.rays_loss_grad(oc, p32.astype(np.float64), half, 31, 9, o, d, bg=bg.astype(np.float64),
                               upstream=np.zeros((n, 6)), inv_B=1.0, want_grad=False)["ray"]
        ctx = Ctx(rc)
        try:
            to = lambda a: torch.tensor(a, device="cuda")
            out, _, _ = ctx.fn_forward(to(p32), half, 31, 9, to(o), to(d), to(bg))
            got = out.cpu().numpy().astype(np.float64)
        finally:
            ctx.close()
        errs[acc] = np.abs(got[:, :5] - ref[:, :5]).max()
        assert np.allclose(got[:, :5], ref[:, :5], rtol=FWD_RTOL, atol=FWD_ATOL)
    print(f"\n1024-sample renders, max abs error vs FP64: FP32 scan {errs[0]:.2e}, FP64 log-sum {errs[1]:.2e}")
    assert errs[1] <= errs[0]
