"""The bounds-checked build (libromap_checked.so, compiled with -DROMAP_CHECKED): the parity tests pass on it, and a
device index beyond an object's logical ray pool is caught and reported as ROMAP_ERR_BOUNDS while the context stays
usable.

The violation is made with romap_debug_set_pool_size: the object's pool size as the kernels see it shrinks below
its rays per step, so the next step's whole-pool ray draw indexes past the logical pool but stays inside the
allocated, filled pool (the unchecked build would only read those older rays; it is not run here).  Both tests run
in child processes that load the checked library (ROMAP_LIB=checked)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _env():
    env = dict(os.environ)
    env["ROMAP_LIB"] = "checked"
    return env


@pytest.fixture(scope="module")
def checked_lib():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "paper_2304_05735_gb300", "build.py"), "--checked"],
                       cwd=ROOT, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout.strip()


_VIOLATION = r'''
import ctypes as C, sys
import numpy as np, torch
sys.path.insert(0, "tests")
from paper_2304_05735_gb300 import romap as R
from paper_2304_05735_gb300 import synth
from _harness import Ctx, paired_config
flag = C.c_int32(-1)
R.check(R.romap_checked_build(C.byref(flag)))
assert flag.value == 1, "the checked library is not the one loaded"
torch.cuda.set_device(0)
sc = synth.config0_scene()
for prec in (R.ROMAP_PREC_FP32, R.ROMAP_PREC_MIXED_BF16):
    _, rc = paired_config(precision=prec)
    ctx = Ctx(rc)
    try:
        oid = ctx.create(t=tuple(sc.t), yaw=sc.yaw, seed=0)
        ctx.add_rays(oid, sc.pool)                     # 256 rays, rays per step 256: the whole pool, in order
        ctx.train([oid], n_steps=2)
        R.check(R.romap_debug_set_pool_size(ctx.h, oid, 100))
        loss = np.zeros(1, np.float32)
        st = R.romap_train_step(ctx.h, ctx.ids([oid]), 1, 1, loss.ctypes.data)
        assert st == R.ROMAP_ERR_BOUNDS, (prec, st, R.last_error())
        assert "bounds" in R.last_error()
        R.check(R.romap_debug_set_pool_size(ctx.h, oid, 256))
        out = ctx.train([oid], n_steps=2)              # the context stays usable
        assert np.all(np.isfinite(out))
    finally:
        ctx.close()
print("checked build: bounds violation reported")
'''


def test_checked_build_reports_index_beyond_logical_pool(checked_lib):
    r = subprocess.run([sys.executable, "-c", _VIOLATION], cwd=ROOT, env=_env(), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "violation reported" in r.stdout


def test_parity_tests_pass_on_checked_build(checked_lib):
    """The FP32 parity tests and the mixed-precision oracle and uneven-batch tests, run on the checked library: no
    check fires on valid inputs (a fired check fails the step with ROMAP_ERR_BOUNDS) and the results still match."""
    tests = ["tests/test_gpu_parity.py", "tests/test_gpu_mixed.py::test_mixed_step_vs_oracle",
             "tests/test_gpu_batched32.py::test_uneven_batch_with_occupancy_mixed", "tests/test_gpu_occupancy.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *tests],
                       cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
