"""Central differences of the FP64 oracle's loss for the GPU differentiation check, one parameter per task, run in
worker processes (started with spawn by the test).  The loss is a sum over rays, so a hash entry's difference is
evaluated on the rays whose samples touch the entry (each ray keeps its own RNG slot, hence its own jitter); an MLP
weight's difference is evaluated on all rays.

The loss matches tests/test_gpu_autograd.py: sum_r ||C_hat_r - tgt_r||^2 + w_depth |D_hat_r - 1.7| + w_sigma
sum_i sigma_ri (Eq. 6 outputs of the explicit rays)."""
import numpy as np

from oracle import romap_oracle as O

_S = {}


def init(cfg_kw, params, half, seed, step, o, d, bg, tgt, w_depth, w_sigma, g_gpu, scale):
    _S.update(cfg=O.make_config(**cfg_kw), p=np.asarray(params, np.float64), half=half, seed=seed, step=step, o=o,
              d=d, bg=np.asarray(bg, np.float64), tgt=np.asarray(tgt, np.float64), w_depth=w_depth,
              w_sigma=w_sigma, g=g_gpu, scale=scale)


def _loss(p, rays):
    S = _S
    if rays is None:
        r = O.rays_loss_grad(S["cfg"], p, S["half"], S["seed"], S["step"], S["o"], S["d"], bg=S["bg"],
                             upstream=np.zeros((S["o"].shape[0], 6)), inv_B=1.0, want_grad=False)["ray"]
        tgt = S["tgt"]
    else:
        outs = []
        for k in rays:
            outs.append(O.rays_loss_grad(S["cfg"], p, S["half"], S["seed"], S["step"], S["o"][k:k + 1],
                                         S["d"][k:k + 1], bg=S["bg"][k:k + 1], upstream=np.zeros((1, 6)), inv_B=1.0,
                                         slot0=int(k), want_grad=False)["ray"])
        r = np.concatenate(outs)
        tgt = S["tgt"][list(rays)]
    return (np.sum((r[:, :3] - tgt) ** 2) + S["w_depth"] * np.abs(r[:, 3] - 1.7).sum()
            + S["w_sigma"] * r[:, 5].sum())


def check(task):
    """task = (parameter index, ray list or None); returns (index, agrees, fd at h = 1e-4).  A parameter whose
    h = 1e-4 difference disagrees is re-checked at h = 1e-6 (a ReLU or |.| kink within 1e-4 of the point is the only
    legitimate cause)."""
    i, rays = task
    S = _S
    fd0 = None
    for h in (1e-4, 1e-6):
        e = np.zeros_like(S["p"])
        e[i] = h
        fd = (_loss(S["p"] + e, rays) - _loss(S["p"] - e, rays)) / (2 * h)
        fd0 = fd if fd0 is None else fd0
        if abs(fd - S["g"][i]) <= 2e-4 * S["scale"] + 1e-3 * abs(fd):
            return i, True, fd0
    return i, False, fd0
