"""The torch.autograd.Function front of the training step (autograd.step_loss over romap_forward_backward), which
carries the fused tcgen05 kernel of the mixed precisions into torch's autograd.

* Deterministic FP32 mode (64-bit fixed-point sums, so that the order of the atomics changes no bit): the front's
  losses and gradients, weighted per object by the upstream gradient, equal bit for bit the library's own
  romap_forward_backward of the same step on an identically trained second context (three uneven objects in one
  batch, at step 4 after three library training steps).
* Mixed BF16 (the fused kernel): loss and gradient against the FP64 oracle's at the same step (the bars of the
  mixed-precision step test); a second call scales its gradient by its own upstream weight and nothing accumulates
  between calls.
* Training through the front with torch.optim.Adam (the paper's optimiser, Sec. V-B) follows the library's own
  training of the same object: the mean loss of the last ten of 40 steps within 5%, both far below the first step's.
"""
import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, object_frame_pool, paired_config

pytestmark = pytest.mark.gpu
MIXED = R.ROMAP_PREC_MIXED_BF16


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _cos(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))


def _det_objects(ctx, scenes, occ, rays=(300, 700, 1100)):
    ids = []
    for k, (sc, bits) in enumerate(zip(scenes, occ)):
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed, rays_per_step=rays[k])
        ctx.add_rays(oid, sc.pool)
        R.check(R.romap_set_occupancy(ctx.h, oid, np.ascontiguousarray(bits).ctypes.data, 0))
        ids.append(oid)
    return ids


def test_step_loss_equals_the_library_step_bit_for_bit():
    import torch

    from paper_2304_05735_gb300.autograd import step_loss

    _, rc = paired_config(L=16, T=2 ** 14, growth=0.0, n_max=512, n_samples=64, bg_random=True)
    rc.deterministic = 1
    scenes = synth.multi_object_scene(3, seed0=71, n_frames=2, W=80, H=60, f=80.0, depth_frac=0.1)
    occ = [synth.occupancy_bits(sc.shape, sc.half, dilate=2, p=0.05, seed=sc.seed) for sc in scenes]
    ref = Ctx(rc)
    try:
        ids = _det_objects(ref, scenes, occ)
        for _ in range(3):
            ref.train(ids)
        states = [ref.state(i) for i in ids]
        assert all(s[3] == 3 for s in states)
        loss_ref = ref.fwd_bwd(ids)  # step 4's draw at the parameters after three steps
        g_ref = [ref.grad(i) for i in ids]
    finally:
        ref.close()
    ctx = Ctx(rc)
    try:
        ids2 = _det_objects(ctx, scenes, occ)
        params = [torch.tensor(s[0], device="cuda", requires_grad=True) for s in states]
        total, terms = step_loss(ctx, ids2, params, step=4)
        w = torch.tensor([1.0, 2.5, -0.5], device="cuda")
        (w * total).sum().backward()
        torch.cuda.synchronize()
        assert np.array_equal(total.detach().cpu().numpy(), loss_ref[:, 0])
        assert np.array_equal(terms.cpu().numpy(), loss_ref[:, 1:])
        assert not terms.requires_grad
        for k, p in enumerate(params):
            assert np.array_equal(p.grad.cpu().numpy(), np.float32(w[k].item()) * g_ref[k]), k
    finally:
        ctx.close()


def test_step_loss_mixed_against_the_oracle_and_without_accumulation():
    import torch

    from paper_2304_05735_gb300.autograd import step_loss

    oc, rc = paired_config(precision=MIXED)
    sc = synth.config0_scene()
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
        ctx.add_rays(oid, sc.pool)
        p0 = O.init_params(oc, sc.seed)
        ref = O.train_step(oc, sc.half.astype(np.float32), sc.seed, 1, object_frame_pool(sc), p0, p0 * 0, p0 * 0,
                           do_adam=False)
        pa = torch.tensor(p0.astype(np.float32), device="cuda", requires_grad=True)
        total, _ = step_loss(ctx, [oid], [pa], step=1)
        total.sum().backward()
        pb = torch.tensor(p0.astype(np.float32), device="cuda", requires_grad=True)
        total_b, _ = step_loss(ctx, [oid], [pb], step=1)
        (3.0 * total_b).sum().backward()
        ga, gb = pa.grad.cpu().numpy(), pb.grad.cpu().numpy()
        nh = O.hash_param_count(oc)
        rel_loss = abs(total.item() - ref["loss"][0]) / abs(ref["loss"][0])
        rel_h, rel_m = _rel(ga[:nh], ref["grad"][:nh]), _rel(ga[nh:], ref["grad"][nh:])
        print(f"\nstep_loss (bf16) vs oracle: loss rel {rel_loss:.2e}, hash-grad rel L2 {rel_h:.2e}, "
              f"mlp-grad rel L2 {rel_m:.2e}; second call / 3 vs first: rel {_rel(gb / 3.0, ga):.2e}")
        assert rel_loss < 1e-3
        assert rel_h < 5e-2 and rel_m < 5e-2 and _cos(ga, ref["grad"]) > 0.998
        # the same step again: the upstream weight scales the gradient, and the first call's gradient is gone
        assert abs(total_b.item() - total.item()) <= 1e-6 * abs(total.item())
        assert _rel(gb / 3.0, ga) < 1e-4
    finally:
        ctx.close()


def test_training_through_step_loss_with_torch_adam_follows_the_library():
    import torch

    from paper_2304_05735_gb300.autograd import step_loss

    oc, rc = paired_config(precision=MIXED, bg_random=True)
    sc = synth.config0_scene()
    steps = 40
    lib = Ctx(rc)
    try:
        oid = lib.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
        lib.add_rays(oid, sc.pool)
        p0 = lib.state(oid)[0]
        lib_loss = np.array([lib.train([oid])[0] for _ in range(steps)], np.float64)
    finally:
        lib.close()
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
        ctx.add_rays(oid, sc.pool)
        p = torch.tensor(p0, device="cuda", requires_grad=True)
        opt = torch.optim.Adam([p], lr=rc.lr, betas=(rc.beta1, rc.beta2), eps=rc.eps)
        front = []
        for t in range(1, steps + 1):
            opt.zero_grad()
            total, _ = step_loss(ctx, [oid], [p], step=t)
            total.sum().backward()
            opt.step()
            front.append(total.item())
        front = np.array(front, np.float64)
    finally:
        ctx.close()
    a, b = front[-10:].mean(), lib_loss[-10:].mean()
    print(f"\nfirst-step loss {front[0]:.5e} (library {lib_loss[0]:.5e}); last ten: front {a:.5e}, library {b:.5e} "
          f"({100 * (a - b) / b:+.2f}%)")
    assert abs(front[0] - lib_loss[0]) <= 1e-3 * lib_loss[0]
    assert abs(a - b) <= 0.05 * b
    assert a < 0.5 * front[0] and b < 0.5 * lib_loss[0]
