"""The C ABI library loads and exports every function include/romap.h declares; host-side argument checks and
the parameter layout work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import romap_oracle as O
from paper_2304_05735_gb300 import romap as R

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "romap.h")


def declared_functions():
    src = open(HEADER).read()
    return re.findall(r"^ROMAP_API\s+[\w\s\*]+?\b(romap_\w+)\s*\(", src, flags=re.M)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("romap_create_object", "romap_add_rays", "romap_train_step", "romap_render", "romap_init",
                     "romap_fn_forward", "romap_fn_backward", "romap_get_state", "romap_set_state"):
        assert required in names
    assert set(names) == set(R.SIGNATURES), set(names) ^ set(R.SIGNATURES)


def test_library_exports_every_declared_symbol():
    L = R.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings_and_null_arguments():
    assert R.status_string(R.ROMAP_OK) == "ok"
    assert R.status_string(R.ROMAP_ERR_NONFINITE) == "non-finite value"
    out = C.c_void_p()
    assert R.romap_init(None, None, C.byref(out)) == R.ROMAP_ERR_INVALID_ARG
    assert R.romap_destroy(None) == R.ROMAP_ERR_INVALID_ARG
    assert R.romap_create_object(None, None, None) == R.ROMAP_ERR_INVALID_ARG
    assert R.romap_train_step(None, None, 0, 1, None) == R.ROMAP_ERR_INVALID_ARG
    assert "ctx is NULL" in R.last_error()


@pytest.mark.parametrize("field,value,status", [
    ("n_levels", 0, R.ROMAP_ERR_INVALID_ARG), ("n_levels", 17, R.ROMAP_ERR_INVALID_ARG),
    ("n_features", 4, R.ROMAP_ERR_UNSUPPORTED), ("log2_table_size", 30, R.ROMAP_ERR_INVALID_ARG),
    ("hidden", 32, R.ROMAP_ERR_UNSUPPORTED), ("dir_dims", 2, R.ROMAP_ERR_INVALID_ARG),
    ("n_samples", 0, R.ROMAP_ERR_INVALID_ARG), ("n_samples", 2000, R.ROMAP_ERR_INVALID_ARG),
    ("lr", 0.0, R.ROMAP_ERR_INVALID_ARG), ("beta1", 1.0, R.ROMAP_ERR_INVALID_ARG),
    ("precision", 7, R.ROMAP_ERR_INVALID_ARG), ("max_objects", 0, R.ROMAP_ERR_INVALID_ARG),
    ("accuracy_mode", 2, R.ROMAP_ERR_INVALID_ARG), ("single_net", 2, R.ROMAP_ERR_INVALID_ARG),
    ("hidden_layers", 4, R.ROMAP_ERR_INVALID_ARG), ("hidden_layers", 2, R.ROMAP_ERR_UNSUPPORTED),
    ("reserved", 1, R.ROMAP_ERR_INVALID_ARG), ("deterministic", 2, R.ROMAP_ERR_INVALID_ARG),
    ("per_object", -1, R.ROMAP_ERR_INVALID_ARG),
])
def test_config_validation_is_host_side(field, value, status):
    cfg = R.make_config()
    setattr(cfg, field, value)
    lay = R.romap_layout()
    assert R.romap_param_layout(C.byref(cfg), C.byref(lay)) == status
    out = C.c_void_p()
    assert R.romap_init(C.byref(cfg), None, C.byref(out)) == status


def test_single_net_is_not_combined_with_fp8():
    cfg = R.make_config(precision=R.ROMAP_PREC_MIXED_FP8, single_net=True)
    lay = R.romap_layout()
    assert R.romap_param_layout(C.byref(cfg), C.byref(lay)) == R.ROMAP_ERR_UNSUPPORTED
    cfg = R.make_config(precision=R.ROMAP_PREC_MIXED_BF16, single_net=True)
    assert R.romap_param_layout(C.byref(cfg), C.byref(lay)) == R.ROMAP_OK


def test_deterministic_mode_is_fp32_only():
    lay = R.romap_layout()
    for prec in (R.ROMAP_PREC_MIXED_BF16, R.ROMAP_PREC_MIXED_FP16, R.ROMAP_PREC_MIXED_FP8):
        cfg = R.make_config(precision=prec, deterministic=True)
        assert R.romap_param_layout(C.byref(cfg), C.byref(lay)) == R.ROMAP_ERR_UNSUPPORTED
    cfg = R.make_config(deterministic=True, per_object=True)
    assert R.romap_param_layout(C.byref(cfg), C.byref(lay)) == R.ROMAP_OK


def test_allocator_hooks_must_come_in_pairs():
    cfg = R.make_config()
    cfg.alloc = R.ALLOC_FN(lambda u, n: None)
    lay = R.romap_layout()
    assert R.romap_param_layout(C.byref(cfg), C.byref(lay)) == R.ROMAP_ERR_INVALID_ARG


@pytest.mark.parametrize("kw,okw", [
    (dict(n_levels=8, log2_table_size=12, base_resolution=16, growth=1.5), dict(L=8, T=2 ** 12, growth=1.5)),
    (dict(n_levels=16, log2_table_size=16, base_resolution=16, growth=0.0, max_resolution=512),
     dict(L=16, T=2 ** 16, growth=0.0, n_max=512)),
    (dict(n_levels=4, log2_table_size=10, base_resolution=16, growth=2.0), dict(L=4, T=2 ** 10, growth=2.0)),
    (dict(n_levels=16, log2_table_size=19, base_resolution=16, growth=0.0, max_resolution=512, dir_dims=0),
     dict(L=16, T=2 ** 19, growth=0.0, n_max=512, dir_dims=0)),
    (dict(n_levels=8, log2_table_size=12, growth=1.5, dir_dims=0, single_net=True, hidden_layers=2),
     dict(L=8, T=2 ** 12, growth=1.5, dir_dims=0, single_net=True, hidden_layers=2)),
    (dict(n_levels=16, log2_table_size=16, growth=0.0, max_resolution=2048, dir_dims=0, single_net=True,
          hidden_layers=3),
     dict(L=16, T=2 ** 16, growth=0.0, n_max=2048, dir_dims=0, single_net=True, hidden_layers=3)),
])
def test_param_layout_matches_oracle(kw, okw):
    lay = R.param_layout(R.make_config(**kw))
    oc = O.make_config(**okw)
    assert lay.n_params == O.param_count(oc)
    assert lay.n_hash_params == O.hash_param_count(oc)
    for l in range(lay.n_levels):
        assert lay.resolution[l] == oc.res[l]
        assert lay.level_offset[l] == O.level_offset(oc, l)
        assert bool(lay.dense[l]) == O.level_is_dense(oc, l)
    assert lay.n_mlp_layers == 5 + (okw.get("hidden_layers", 1) - 1)
    for i in range(lay.n_mlp_layers):
        assert lay.mlp_offset[i] == O.hash_param_count(oc) + O.mlp_layer_offset(oc, i)
        assert lay.mlp_offset[i] + lay.mlp_rows[i] * lay.mlp_cols[i] == \
            (O.hash_param_count(oc) + O.mlp_layer_offset(oc, i + 1) if i + 1 < lay.n_mlp_layers else lay.n_params)


def test_init_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = C.c_void_p()
    cfg = R.make_config()
    assert R.romap_init(C.byref(cfg), None, C.byref(out)) == R.ROMAP_ERR_CUDA
    assert not out.value


def test_view_angle_matches_oracle():
    """Eq. 5 in the library (host code) against the oracle's FP64 restatement on random camera pairs."""
    import ctypes as C

    import numpy as np

    from oracle import romap_oracle as O

    rng = np.random.default_rng(11)
    out = C.c_double()
    for _ in range(500):
        o = rng.normal(size=3)
        a, b = o + rng.normal(size=3) * 2, o + rng.normal(size=3) * 2
        arr = [np.ascontiguousarray(x, np.float64) for x in (a, b, o)]
        assert R.romap_view_angle(*(x.ctypes.data for x in arr), C.byref(out)) == R.ROMAP_OK
        assert out.value == pytest.approx(O.view_angle_deg(a, b, o), abs=1e-6)
    z = np.zeros(3)
    assert R.romap_view_angle(z.ctypes.data, np.ones(3).ctypes.data, z.ctypes.data, C.byref(out)) == R.ROMAP_OK
    assert out.value == 180.0
    assert R.romap_view_angle(None, z.ctypes.data, z.ctypes.data, C.byref(out)) == R.ROMAP_ERR_INVALID_ARG


def test_step_loss_checks_its_arguments_on_the_host():
    """The autograd front of the training step refuses mismatched, duplicate or host tensors before any library
    call (the stand-in context has no library handle at all)."""
    torch = pytest.importorskip("torch")
    from paper_2304_05735_gb300.autograd import step_loss

    class Stub:
        h = None

        class layout:
            n_params = 8

    p = torch.zeros(8)
    with pytest.raises(ValueError):
        step_loss(Stub, [0, 1], [p], step=1)
    with pytest.raises(ValueError):
        step_loss(Stub, [0, 0], [p, p], step=1)
    with pytest.raises(ValueError):
        step_loss(Stub, [0], [p], step=0)
    with pytest.raises(ValueError):
        step_loss(Stub, [0], [p], step=1)  # a host tensor
