"""The stored oracle-trained references (tests/golden/training_reference.json) against the oracle itself: the first
iteration's loss of each object, recomputed from the recipe, equals the stored one, and the stored curve is a
training curve (the last quarter's mean loss far below the first iteration's)."""
import importlib.util
import json
import os

import numpy as np

from oracle import romap_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _refmod():
    spec = importlib.util.spec_from_file_location("make_training_reference",
                                                  os.path.join(HERE, "golden", "make_training_reference.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_stored_reference_first_iteration_matches_the_oracle():
    M = _refmod()
    with open(os.path.join(HERE, "golden", "training_reference.json")) as f:
        ref = json.load(f)
    assert ref["recipe"]["steps"] == len(ref["objects"][0]["loss"]) == 300
    cfg = O.make_config(**ref["recipe"]["config"])
    for name in ("lambda1", "lambda2", "lr", "beta1", "beta2", "eps"):
        setattr(cfg, name, float(np.float32(getattr(cfg, name))))
    scenes = M.scenes()
    for sc, obj in zip(scenes, ref["objects"]):
        assert sc.seed == obj["seed"]
        pool = M.object_pool(O, sc)
        assert pool["cls"].size == obj["pool_rays"]
        p = O.init_params(cfg, sc.seed)
        r = O.train_step(cfg, sc.half.astype(np.float32), sc.seed, 1, pool, p, p * 0, p * 0, do_adam=False)
        assert abs(r["loss"][0] - obj["loss"][0]) <= 1e-12 * abs(obj["loss"][0])
        assert obj["final_loss"] == np.mean(obj["loss"][-75:])
        assert obj["final_loss"] < 1e-2 * obj["loss"][0]
        assert obj["psnr"] > obj["psnr_init"] + 20.0
