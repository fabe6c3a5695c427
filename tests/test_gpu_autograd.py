"""The torch.autograd.Function over the library's adjoint kernels, against the FP64 oracle's analytic gradient and
against central finite differences of the FP64 oracle (differentiation-check configuration: L=4, F=2, T=2^10 so
that resolutions 16..128 force hash collisions; 64 rays x 16 samples; and 1024 samples per ray)."""
import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R

from _harness import assert_grad_close, paired_config

pytestmark = pytest.mark.gpu


def _rays(n, seed):
    rng = np.random.default_rng(seed)
    az, el = rng.uniform(-np.pi, np.pi, n), rng.uniform(-0.5, 0.8, n)
    cam = 2.2 * np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1)
    d = rng.uniform(-0.4, 0.4, (n, 3)) - cam
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return cam.astype(np.float32), d.astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32)


def _loss_torch(out, tgt, w_depth, torch):
    # photometric L2 + L1 depth + density sum, through torch ops on the kernel outputs
    return ((out[:, :3] - tgt) ** 2).sum() + w_depth * (out[:, 3] - 1.7).abs().sum() + 0.01 * out[:, 5].sum()


def _upstream_np(ray_out, tgt, w_depth):
    u = np.zeros((ray_out.shape[0], 6))
    u[:, :3] = 2 * (ray_out[:, :3] - tgt)
    u[:, 3] = w_depth * np.sign(ray_out[:, 3] - 1.7)
    u[:, 5] = 0.01
    return u


def _setup(N, n, rc_kw=None):
    oc, rc = paired_config(L=4, T=2 ** 10, growth=2.0, n_samples=N)
    rng = np.random.default_rng(N)
    p64 = O.init_params(oc, 3)
    nh = O.hash_param_count(oc)
    p64[:nh] = rng.uniform(-1, 1, nh)
    p32 = p64.astype(np.float32)
    o, d, bg = _rays(n, N)
    tgt = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    return oc, rc, rng, p32, o, d, bg, tgt, nh


def _gpu_grad(rc, p32, o, d, bg, tgt, half, recompute=None):
    import torch

    from paper_2304_05735_gb300.autograd import Context, render

    rctx = Context(rc)
    try:
        params = torch.tensor(p32, device="cuda", requires_grad=True)
        to = lambda a: torch.tensor(a, device="cuda")
        out = render(params, to(o), to(d), to(bg), rctx, half=half, seed=5, step=2, recompute=recompute)
        loss = _loss_torch(out, to(tgt), 0.5, torch)
        loss.backward()
        return out.detach().cpu().numpy(), params.grad.cpu().numpy().astype(np.float64)
    finally:
        rctx.close()


def _oracle_grad(oc, p32, half, o, d, bg, tgt, n):
    ref_fwd = O.rays_loss_grad(oc, p32.astype(np.float64), half, 5, 2, o, d, bg=bg.astype(np.float64),
                               upstream=np.zeros((n, 6)), inv_B=1.0, want_grad=False, want_samples=True)
    up = _upstream_np(ref_fwd["ray"][:, :6], tgt.astype(np.float64), 0.5)
    ref = O.rays_loss_grad(oc, p32.astype(np.float64), half, 5, 2, o, d, bg=bg.astype(np.float64), upstream=up,
                           inv_B=1.0)
    return ref_fwd, ref


def _rays_of_entries(oc, ref_fwd, half, n):
    """For every hash parameter, the rays whose live samples interpolate it (brute force over samples and levels)."""
    rays = {}
    S = ref_fwd["samples"]  # per sample: t, delta, x, y, z, live, sigma, dL/dsigma
    for r in range(n):
        for i in range(S.shape[1]):
            if not S[r, i, 5]:
                continue
            x = S[r, i, 2:5].astype(np.float32)
            for l in range(oc.L):
                idx, w = O.level_corners(oc, l, x, half)
                base = O.level_offset(oc, l)
                for k in range(8):
                    if w[k] != 0.0:
                        for f in range(2):
                            rays.setdefault(2 * (base + int(idx[k])) + f, set()).add(r)
    return rays


def test_autograd_every_parameter_vs_finite_differences():
    """Differentiation-check configuration (64 rays x 16 samples, L=4, T=2^10): the GPU backward against the
    oracle's analytic gradient for every parameter, and against central differences (h = 1e-4, FP64) of the oracle's
    loss for every touched hash entry and every MLP weight."""
    import multiprocessing as mp
    import os

    import _fd_worker

    N, n = 16, 64
    oc, rc, rng, p32, o, d, bg, tgt, nh = _setup(N, n)
    half = np.array([0.5, 0.5, 0.5], np.float32)
    out, g = _gpu_grad(rc, p32, o, d, bg, tgt, half)
    ref_fwd, ref = _oracle_grad(oc, p32, half, o, d, bg, tgt, n)
    assert np.allclose(out, ref_fwd["ray"][:, :6], rtol=1e-5, atol=1e-5 * N)
    assert_grad_close(g[:nh], ref["grad"][:nh], what="hash gradient")
    assert_grad_close(g[nh:], ref["grad"][nh:], what="MLP gradient")
    rays = _rays_of_entries(oc, ref_fwd, half, n)
    touched = np.nonzero(ref["grad"][:nh])[0]
    assert set(int(i) for i in touched) <= set(rays), "a touched entry that no sample interpolates"
    tasks = [(int(i), sorted(rays[int(i)])) for i in touched] + [(nh + j, None) for j in range(p32.size - nh)]
    scale = float(np.abs(ref["grad"]).max())
    kw = dict(L=4, T=2 ** 10, growth=2.0, n_samples=N)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4), initializer=_fd_worker.init,
                                      initargs=(kw, p32.astype(np.float64), half, 5, 2, o, d, bg, tgt, 0.5, 0.01, g,
                                                scale)) as pool:
        res = pool.map(_fd_worker.check, tasks, chunksize=16)
    bad = [(i, fd, g[i]) for i, ok, fd in res if not ok]
    print(f"\n{len(touched)} touched hash entries and {p32.size - nh} MLP weights checked by central differences; "
          f"{len(bad)} disagree")
    assert not bad, bad[:10]


def test_autograd_long_rays_vs_oracle_and_finite_differences():
    """1024 samples per ray (12 rays): the recomputing backward against the oracle's gradient and, on a sample of
    parameters, central differences of the oracle's loss."""
    N, n = 1024, 12
    oc, rc, rng, p32, o, d, bg, tgt, nh = _setup(N, n)
    half = np.array([0.5, 0.5, 0.5], np.float32)
    out, g = _gpu_grad(rc, p32, o, d, bg, tgt, half)
    ref_fwd, ref = _oracle_grad(oc, p32, half, o, d, bg, tgt, n)
    assert np.allclose(out, ref_fwd["ray"][:, :6], rtol=1e-5, atol=1e-5 * N)
    assert_grad_close(g[:nh], ref["grad"][:nh], what="hash gradient")
    assert_grad_close(g[nh:], ref["grad"][nh:], what="MLP gradient")

    def oracle_loss(p):
        r = O.rays_loss_grad(oc, p, half, 5, 2, o, d, bg=bg.astype(np.float64), upstream=np.zeros((n, 6)),
                             inv_B=1.0, want_grad=False)["ray"]
        return np.sum((r[:, :3] - tgt) ** 2) + 0.5 * np.abs(r[:, 3] - 1.7).sum() + 0.01 * r[:, 5].sum()

    touched = np.nonzero(ref["grad"][:nh])[0]
    idx = list(rng.choice(touched, min(25, touched.size), replace=False))
    idx += list(nh + rng.choice(p32.size - nh, 25, replace=False))
    base = p32.astype(np.float64)
    scale = np.abs(ref["grad"]).max()
    bad = 0
    for i in idx:
        ok = False
        for h in (1e-4, 1e-6):
            e = np.zeros_like(base)
            e[i] = h
            fd = (oracle_loss(base + e) - oracle_loss(base - e)) / (2 * h)
            if abs(fd - g[i]) <= 2e-4 * scale + 1e-3 * abs(fd):
                ok = True
                break
        bad += not ok
    assert bad == 0, f"{bad} of {len(idx)} parameters disagree with central differences"


@pytest.mark.parametrize("N,n", [(1024, 12), (16, 64)])
def test_stored_and_recomputed_activations_agree(N, n):
    """The backward that reads the forward's stored activations (ROMAP_STORE_ACT) and the one that recomputes them
    give the same outputs and the same gradient (to FP32 atomic-ordering noise), at 1024 samples per ray too."""
    oc, rc, rng, p32, o, d, bg, tgt, nh = _setup(N, n)
    half = np.array([0.5, 0.5, 0.5], np.float32)
    out_r, g_r = _gpu_grad(rc, p32, o, d, bg, tgt, half, recompute=True)
    out_s, g_s = _gpu_grad(rc, p32, o, d, bg, tgt, half, recompute=False)
    assert np.array_equal(out_r, out_s)
    assert np.count_nonzero(g_r) > 0.3 * g_r.size
    assert_grad_close(g_s, g_r, tol=1e-6, what="stored vs recomputed activations")
