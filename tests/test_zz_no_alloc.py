"""The forward entry point that allocates nothing (romap_fn_forward_noalloc) gives the same rays as the
workspace-based romap_fn_forward, call after call.

Callers that cannot allocate device memory where they render (a plugin whose host framework owns all device
memory, or a real-time loop that must not call cudaMalloc/cudaFree) use this entry point; its scratch is a static
array inside the library, shared by every call.  This file is collected last so that a stop at the first failure
has already run every other test; it passes alone in a fresh process as well.
"""
import ctypes as C
import sys
import os

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from _harness import FWD_ATOL, FWD_RTOL, Ctx, paired_config  # noqa: E402
from oracle import romap_oracle as O  # noqa: E402
from paper_2304_05735_gb300 import romap as R  # noqa: E402

pytestmark = pytest.mark.gpu


def _rays(n, seed):
    rng = np.random.default_rng(seed)
    az = rng.uniform(-np.pi, np.pi, n)
    el = rng.uniform(-0.5, 0.8, n)
    cam = 2.5 * np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1)
    d = rng.uniform(-0.45, 0.45, (n, 3)) - cam
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return cam.astype(np.float32), d.astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32)


def test_noalloc_forward_matches_workspace_forward_twice():
    import torch

    oc, rc = paired_config(L=8, T=2 ** 12, growth=1.5, n_samples=32)
    ctx = Ctx(rc)
    try:
        p = O.init_params(oc, 3)
        nh = O.hash_param_count(oc)
        p[:nh] = np.random.default_rng(0).uniform(-1, 1, nh)
        params = torch.tensor(p.astype(np.float32), device="cuda")
        half = (0.5, 0.45, 0.4)
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        # two calls on the caller's stream, then one on the legacy default stream (cuda_stream = NULL); the last
        # call is smaller than the first, so a stale scratch word from the first call would show
        for call, (n, seed, step, strm) in enumerate([(700, 1, 3, stream), (300, 2, 4, stream), (520, 3, 5, None)]):
            o, d, bg = (torch.tensor(a, device="cuda") for a in _rays(n, seed))
            ref, _, _ = ctx.fn_forward(params, half, 17, step, o, d, bg, jitter=True)
            torch.cuda.synchronize()
            out = torch.full((n, 6), float("nan"), device="cuda")
            torch.cuda.synchronize()
            R.check(R.romap_fn_forward_noalloc(C.byref(rc), strm, params.data_ptr(), (C.c_float * 3)(*half), 17,
                                               step, None, o.data_ptr(), d.data_ptr(), bg.data_ptr(), n,
                                               R.ROMAP_JITTER, out.data_ptr()), "romap_fn_forward_noalloc")
            torch.cuda.synchronize()
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(got)), call
            # the same kernels on the same inputs: the rays agree bit for bit (the forward has no atomics), which
            # also catches a carving or offset slip in the static scratch that a tolerance could hide
            assert np.allclose(got, want, rtol=FWD_RTOL, atol=FWD_ATOL), (call, np.abs(got - want).max())
            assert np.array_equal(got, want), (call, np.abs(got - want).max())
            assert (got[:, 4] > 0).sum() > n // 2
    finally:
        ctx.close()


def test_noalloc_forward_rejects_sizes_beyond_its_scratch():
    import torch

    _, rc = paired_config(L=8, T=2 ** 12, growth=1.5, n_samples=1024)
    x = torch.zeros(8, device="cuda")
    st = R.romap_fn_forward_noalloc(C.byref(rc), None, x.data_ptr(), (C.c_float * 3)(0.5, 0.5, 0.5), 0, 0, None,
                                    x.data_ptr(), x.data_ptr(), x.data_ptr(), 1 << 20, 0, x.data_ptr())
    assert st == R.ROMAP_ERR_CAPACITY
    assert "static scratch" in R.last_error() and "at most" in R.last_error()
    st = R.romap_fn_forward_noalloc(C.byref(rc), None, x.data_ptr(), (C.c_float * 3)(0.5, 0.5, 0.5), 0, 0, None,
                                    x.data_ptr(), x.data_ptr(), x.data_ptr(), (1 << 24) + 1, 0, x.data_ptr())
    assert st == R.ROMAP_ERR_INVALID_ARG and "2^24" in R.last_error()
