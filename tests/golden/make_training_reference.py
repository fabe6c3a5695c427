"""Writes tests/golden/training_reference.json: two objects trained by the FP64 CPU oracle for 300 iterations (the
paper's iterations per data update, Sec. V-A-1) at the streaming model size (hash grid L=16, F=2, T=2^19,
resolutions 16..512; 4096 rays x 32 samples per iteration; random background colours), the reference that the GPU
paths' training of the same objects is compared with (tests/test_gpu_training_reference.py).

Per object: the total loss of every iteration, and the PSNR of the trained parameters on a fixed evaluation set (4096
of the pool's object rays evenly strided over it, midpoint samples, grey background, rendered by the oracle).  Only oracle/ and
the seeded scene generator are called.  Each object trains in its own process (about 25 minutes each).

    python tests/golden/make_training_reference.py
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

STEPS = int(os.environ.get("ROMAP_REF_STEPS", "300"))
N_OBJECTS = 2
SCENE = dict(seed0=900, n_frames=3, W=320, H=240, f=320.0)
CONFIG = dict(L=16, T=2 ** 19, n_min=16, growth=0.0, n_max=512, n_samples=32, rays_per_step=4096, bg_random=True)
EVAL_RAYS = 4096
EVAL_BG = 0.5


def scenes():
    from paper_2304_05735_gb300 import synth
    return synth.multi_object_scene(N_OBJECTS, **SCENE)


def object_pool(O, sc):
    o, d = O.world_to_object(sc.pool["origin"], sc.pool["dir"], sc.t.astype(np.float32), sc.yaw)
    return dict(o=o.reshape(-1, 3), d=d.reshape(-1, 3), rgb=sc.pool["rgb"], depth=sc.pool["depth"],
                cls=sc.pool["cls"])


def eval_rays(pool):
    """The evaluation set: EVAL_RAYS of the pool's object rays (class 0), evenly strided over the pool."""
    obj = np.nonzero(pool["cls"] == 0)[0]
    return obj[np.linspace(0, obj.size - 1, min(EVAL_RAYS, obj.size)).astype(np.int64)]


def eval_psnr(O, cfg, params, sc, pool):
    """PSNR of the parameters on the evaluation rays: the oracle's render (midpoint samples) over a grey background
    against the rays' target colours."""
    idx = eval_rays(pool)
    n = idx.size
    bg = np.full((n, 3), EVAL_BG, np.float64)
    out = O.rays_loss_grad(cfg, params, sc.half.astype(np.float32), sc.seed, 1, pool["o"][idx], pool["d"][idx],
                           bg=bg, upstream=np.zeros((n, 6)), inv_B=1.0, jitter=False, want_grad=False)["ray"]
    mse = float(((out[:, :3] - pool["rgb"][idx].astype(np.float64)) ** 2).mean())
    return -10.0 * np.log10(max(mse, 1e-12))


def train_one(k):
    from oracle import romap_oracle as O
    cfg = O.make_config(**CONFIG)
    # the GPU runs these constants in FP32; the oracle takes the FP32 values
    for name in ("lambda1", "lambda2", "lr", "beta1", "beta2", "eps"):
        setattr(cfg, name, float(np.float32(getattr(cfg, name))))
    sc = scenes()[k]
    pool = object_pool(O, sc)
    p = O.init_params(cfg, sc.seed)
    m, v = np.zeros_like(p), np.zeros_like(p)
    losses = []
    for step in range(1, STEPS + 1):
        r = O.train_step(cfg, sc.half.astype(np.float32), sc.seed, step, pool, p, m, v)
        p, m, v = r["params"], r["m"], r["v"]
        losses.append(float(r["loss"][0]))
    return dict(seed=int(sc.seed), pool_rays=int(pool["cls"].size), loss=losses,
                final_loss=float(np.mean(losses[-STEPS // 4:])), psnr=eval_psnr(O, cfg, p, sc, pool),
                psnr_init=eval_psnr(O, cfg, O.init_params(cfg, sc.seed), sc, pool))


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(N_OBJECTS) as pool:
        objs = pool.map(train_one, range(N_OBJECTS))
    out = dict(recipe=dict(steps=STEPS, scene=SCENE, config=CONFIG, eval_rays=EVAL_RAYS, eval_bg=EVAL_BG,
                           final_loss="mean total loss (Eq. 11) of the last steps / 4 iterations",
                           source="FP64 CPU oracle (oracle/romap_oracle.c), this script"),
               objects=objs)
    with open(os.path.join(HERE, "training_reference.json"), "w") as f:
        json.dump(out, f, indent=1)
    for o in objs:
        print(f"seed {o['seed']}: final loss {o['final_loss']:.5e}, PSNR {o['psnr']:.2f} dB "
              f"(initial {o['psnr_init']:.2f})")


if __name__ == "__main__":
    main()
