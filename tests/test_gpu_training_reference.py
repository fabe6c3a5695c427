"""Training against the FP64 oracle's: two objects at the streaming model size (hash grid L=16, F=2, T=2^19,
resolutions 16..512, 4096 rays x 32 samples per iteration, random background colours), trained for 300 iterations
(the paper's iterations per data update, Sec. V-A-1) by the GPU's FP32 path and by its mixed-precision path, against
the same objects trained by the oracle (tests/golden/training_reference.json, written by
tests/golden/make_training_reference.py, which calls only oracle/ and the scene generator).

Both sides draw the same rays, jitter and background colours at every iteration (the counter-based generator is
bit-exact), so the first iterations agree to the per-step parity bars; from there on training is chaotic (a change
of summation order alone moves a 500-step run's final loss by about 1%), so the trained objects are compared by what
training is for: the final loss (mean of the last 75 iterations) within 5% of the oracle-trained object's, and the
PSNR of the trained parameters, rendered by the oracle on the reference's evaluation rays, within 3 dB of the
oracle-trained parameters' PSNR (the measured spread between equally converged trainings)."""
import importlib.util
import json
import os

import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth

from _harness import Ctx, paired_config

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_training_reference",
                                               os.path.join(HERE, "golden", "make_training_reference.py"))
REFMOD = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(REFMOD)
REF_PATH = os.path.join(HERE, "golden", "training_reference.json")


@pytest.mark.parametrize("precision", [R.ROMAP_PREC_FP32, R.ROMAP_PREC_MIXED_BF16])
def test_training_matches_the_oracle_trained_objects(precision):
    import torch  # noqa: F401
    with open(REF_PATH) as f:
        reference = json.load(f)
    rec = reference["recipe"]
    steps = rec["steps"]
    c = rec["config"]
    oc, rc = paired_config(L=c["L"], T=c["T"], n_min=c["n_min"], growth=c["growth"], n_max=c["n_max"],
                           n_samples=c["n_samples"], rays_per_step=c["rays_per_step"], bg_random=c["bg_random"],
                           precision=precision)
    scenes = synth.multi_object_scene(len(reference["objects"]), **rec["scene"])
    ctx = Ctx(rc)
    results = []
    try:
        for sc, ref in zip(scenes, reference["objects"]):
            assert sc.seed == ref["seed"]
            oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=sc.seed)
            ctx.add_rays(oid, sc.pool)
            losses = np.array([ctx.train([oid])[0] for _ in range(steps)], np.float64)
            p = ctx.state(oid)[0].astype(np.float64)
            pool = REFMOD.object_pool(O, sc)
            psnr = REFMOD.eval_psnr(O, oc, p, sc, pool)
            final = float(losses[-steps // 4:].mean())
            rel1 = abs(losses[0] - ref["loss"][0]) / ref["loss"][0]
            relf = (final - ref["final_loss"]) / ref["final_loss"]
            print(f"\n[seed {sc.seed}, precision {precision}] step-1 loss rel {rel1:.2e}; final loss {final:.5e} vs "
                  f"oracle {ref['final_loss']:.5e} ({100 * relf:+.2f}%); PSNR {psnr:.2f} vs oracle {ref['psnr']:.2f} dB "
                  f"(untrained {ref['psnr_init']:.2f})")
            results.append((rel1, relf, psnr, ref))
    finally:
        ctx.close()
    for rel1, relf, psnr, ref in results:
        assert rel1 < (1e-5 if precision == R.ROMAP_PREC_FP32 else 1e-3)
        assert abs(relf) < 0.05
        # the evaluation MSE is dominated by a few silhouette rays: between trainings whose final losses agree to
        # 0.1-3%, the PSNR of the two objects was measured to move by up to 2.3 dB either way (GPU FP32 and mixed
        # against the oracle, and the GPU's own repeated runs); 3 dB bounds that spread
        assert abs(psnr - ref["psnr"]) < 3.0
        assert psnr > ref["psnr_init"] + 20.0  # training did its job
