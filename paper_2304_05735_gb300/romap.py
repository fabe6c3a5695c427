"""ctypes binding of libromap (include/romap.h): same names, argument marshalling only.

Every computation of the training step runs in the CUDA kernels of
libromap.so.  There is no fallback: if the library is missing or cannot be
loaded, every call raises.  PyTorch is used by callers only for device
memory and streams; pass tensors' data_ptr() where the C ABI takes device
pointers.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libromap.so")
# ROMAP_LIB=checked loads the bounds-checked build (libromap_checked.so, see romap_checked_build in romap.h)
LIB_PATH_CHECKED = os.path.join(HERE, "libromap_checked.so")

ROMAP_OK = 0
ROMAP_ERR_INVALID_ARG = -1
ROMAP_ERR_NOT_FOUND = -2
ROMAP_ERR_OOM = -3
ROMAP_ERR_CAPACITY = -4
ROMAP_ERR_CUDA = -5
ROMAP_ERR_NONFINITE = -6
ROMAP_ERR_TIMEOUT = -7
ROMAP_ERR_BAD_STATE = -8
ROMAP_ERR_UNSUPPORTED = -9
ROMAP_ERR_BOUNDS = -10

ROMAP_DEVICE_PTR = 0x1
ROMAP_OBJECT_FRAME = 0x2
ROMAP_REPLACE = 0x4
ROMAP_JITTER = 0x8
ROMAP_ASYNC_HOST = 0x10
ROMAP_STORE_ACT = 0x20

ROMAP_CLS_OBJECT, ROMAP_CLS_BACKGROUND, ROMAP_CLS_OCCLUDER = 0, 1, 2
ROMAP_PREC_FP32, ROMAP_PREC_MIXED_BF16, ROMAP_PREC_MIXED_FP8, ROMAP_PREC_MIXED_FP16 = 0, 1, 2, 3

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
DEALLOC_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class romap_config(C.Structure):
    _fields_ = [
        ("n_levels", C.c_int32), ("n_features", C.c_int32), ("log2_table_size", C.c_int32),
        ("base_resolution", C.c_int32), ("growth", C.c_double), ("max_resolution", C.c_int32),
        ("hidden", C.c_int32), ("dir_dims", C.c_int32), ("n_samples", C.c_int32), ("rays_per_step", C.c_int32),
        ("lambda1", C.c_float), ("lambda2", C.c_float),
        ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
        ("bg_random", C.c_int32), ("bg_const", C.c_float * 3),
        ("precision", C.c_int32), ("max_objects", C.c_int32), ("max_rays_per_object", C.c_int64),
        ("accuracy_mode", C.c_int32), ("single_net", C.c_int32),
        ("hidden_layers", C.c_int32), ("deterministic", C.c_int32), ("per_object", C.c_int32),
        ("reserved", C.c_int32),
        ("alloc", ALLOC_FN), ("dealloc", DEALLOC_FN), ("alloc_user", C.c_void_p),
    ]


class romap_object_desc(C.Structure):
    _fields_ = [("t", C.c_float * 3), ("yaw", C.c_double), ("half_size", C.c_float * 3), ("seed", C.c_uint64),
                ("rays_per_step", C.c_int32)]


class romap_rays(C.Structure):
    _fields_ = [("origin", C.c_void_p), ("dir", C.c_void_p), ("rgb", C.c_void_p), ("depth", C.c_void_p),
                ("cls", C.c_void_p)]


class romap_layout(C.Structure):
    _fields_ = [("n_params", C.c_int64), ("n_hash_params", C.c_int64), ("n_levels", C.c_int32),
                ("resolution", C.c_int32 * 16), ("dense", C.c_int32 * 16), ("level_offset", C.c_int64 * 16),
                ("mlp_offset", C.c_int64 * 7), ("mlp_rows", C.c_int32 * 7), ("mlp_cols", C.c_int32 * 7),
                ("n_mlp_layers", C.c_int32)]


class romap_state(C.Structure):
    _fields_ = [("params", C.c_void_p), ("adam_m", C.c_void_p), ("adam_v", C.c_void_p), ("n_params", C.c_int64),
                ("step", C.c_int64), ("flags", C.c_uint32)]


class romap_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rays", C.c_int64), ("live_samples", C.c_int64),
                ("kernel_launches", C.c_int64), ("graph_captures", C.c_int64), ("graph_replays", C.c_int64)]


_vp, _i32, _i64, _u32, _u64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t
_P = C.POINTER
# name -> (restype, argtypes); the declaration order of include/romap.h
SIGNATURES = {
    "romap_init": (_i32, [_P(romap_config), _vp, _P(_vp)]),
    "romap_destroy": (_i32, [_vp]),
    "romap_status_string": (C.c_char_p, [_i32]),
    "romap_last_error": (_i32, [C.c_char_p, _sz]),
    "romap_param_layout": (_i32, [_P(romap_config), _P(romap_layout)]),
    "romap_create_object": (_i32, [_vp, _P(romap_object_desc), _P(_i32)]),
    "romap_destroy_object": (_i32, [_vp, _i32]),
    "romap_set_occupancy": (_i32, [_vp, _i32, _vp, _u32]),
    "romap_view_angle": (_i32, [_vp, _vp, _vp, _P(C.c_double)]),
    "romap_observe": (_i32, [_vp, _i32, _vp, C.c_float, _P(romap_rays), _i64, _u32, _i32, _P(_i32)]),
    "romap_pending": (_i32, [_vp, _i32, _P(_i64)]),
    "romap_set_pending": (_i32, [_vp, _i32, _i64]),
    "romap_train_budget": (_i32, [_vp, _vp, _i32, C.c_float, _i32, _P(_i32), _P(C.c_float), _vp]),
    "romap_density_lattice": (_i32, [_vp, _i32, _vp, _u32]),
    "romap_extract_mesh": (_i32, [_vp, _i32, C.c_float, _vp, _i64, _vp, _i64, _P(_i64), _P(_i64), _u32]),
    "romap_mc_case_table": (_i32, [_vp, _vp]),
    "romap_update_occupancy": (_i32, [_vp, _i32, C.c_float, C.c_float, _u32]),
    "romap_get_occupancy": (_i32, [_vp, _i32, _vp, _vp]),
    "romap_add_rays": (_i32, [_vp, _i32, _P(romap_rays), _i64, _u32]),
    "romap_add_rays_multi": (_i32, [_vp, _vp, _vp, _i32, _P(romap_rays), _u32]),
    "romap_train_step_async": (_i32, [_vp, _vp, _i32, _i32, _vp]),
    "romap_check_device_status": (_i32, [_vp]),
    "romap_pool_size": (_i32, [_vp, _i32, _P(_i64)]),
    "romap_train_step": (_i32, [_vp, _vp, _i32, _i32, _vp]),
    "romap_forward_backward": (_i32, [_vp, _vp, _i32, _vp]),
    "romap_adam_step": (_i32, [_vp, _vp, _i32]),
    "romap_get_grad": (_i32, [_vp, _i32, _vp, _u32]),
    "romap_last_batch": (_i32, [_vp, _i32, _vp, _vp, _P(_i64)]),
    "romap_last_outputs": (_i32, [_vp, _i32, _vp, _P(_i64)]),
    "romap_render": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _u32]),
    "romap_get_state": (_i32, [_vp, _i32, _P(romap_state)]),
    "romap_set_state": (_i32, [_vp, _i32, _P(romap_state)]),
    "romap_fn_workspace_size": (_i32, [_vp, _i64, _u32, _P(_sz)]),
    "romap_fn_forward": (_i32, [_vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _i64, _u32, _vp, _sz, _vp, _vp]),
    "romap_fn_backward": (_i32, [_vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _i64, _u32, _vp, _sz, _vp, _vp,
                                 _vp]),
    "romap_get_stats": (_i32, [_vp, _P(romap_stats)]),
    "romap_reset_stats": (_i32, [_vp]),
    "romap_fn_forward_noalloc": (_i32, [_P(romap_config), _vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _i64, _u32,
                                        _vp]),
    "romap_selftest_wait_timeout": (_i32, [_vp, _i32]),
    "romap_set_tile_kernel": (_i32, [_vp, _i32]),
    "romap_autotune_report": (_i32, [_vp, _P(_i32), _vp, _i32, C.c_char_p, _sz]),
    "romap_set_profiling": (_i32, [_vp, _i32]),
    "romap_set_adam_skip": (_i32, [_vp, _i32]),
    "romap_set_graphs": (_i32, [_vp, _i32]),
    "romap_checked_build": (_i32, [_P(_i32)]),
    "romap_debug_set_pool_size": (_i32, [_vp, _i32, _i64]),
    "romap_phase_times": (_i32, [_vp, _vp, _vp]),
    "romap_measure_request_rates": (_i32, [_vp, _vp]),
}
ROMAP_N_PHASES = 5
PHASES = ("sampling", "mlp_forward", "composite_loss_adjoint", "mlp_backward_scatter", "adam")

_lib = None


class RomapError(RuntimeError):
    def __init__(self, status, fn, msg):
        super().__init__(f"{fn} -> {status} ({status_string(status)}): {msg}")
        self.status = status


def lib():
    """Loads libromap.so, or libromap_checked.so when ROMAP_LIB=checked (building it first if it is absent and nvcc
    is available)."""
    global _lib
    if _lib is None:
        checked = os.environ.get("ROMAP_LIB", "") == "checked"
        path = LIB_PATH_CHECKED if checked else LIB_PATH
        if not os.path.exists(path):
            from . import build as _build
            _build.build(checked=checked)
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(s):
    return lib().romap_status_string(int(s)).decode()


def last_error():
    buf = C.create_string_buffer(1024)
    lib().romap_last_error(buf, 1024)
    return buf.value.decode()


def check(status, fn="romap"):
    if status != ROMAP_OK:
        raise RomapError(status, fn, last_error())
    return status


def _wrap(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    f.__doc__ = f"{name}: see include/romap.h"
    return f


for _name in SIGNATURES:
    globals()[_name] = _wrap(_name)


# ---------------------------------------------------------------------------
# small marshalling helpers
# ---------------------------------------------------------------------------
def make_config(n_levels=8, log2_table_size=12, base_resolution=16, growth=1.5, max_resolution=0, n_samples=32,
                rays_per_step=256, dir_dims=3, lambda1=0.5, lambda2=0.01, lr=1e-2, beta1=0.9, beta2=0.99,
                eps=1e-15, bg_random=False, bg_const=(1.0, 1.0, 1.0), precision=ROMAP_PREC_FP32, max_objects=64,
                max_rays_per_object=1 << 24, alloc=None, dealloc=None, accuracy_mode=0,
                single_net=False, hidden_layers=1, deterministic=False, per_object=False):
    c = romap_config()
    c.n_levels, c.n_features, c.log2_table_size = n_levels, 2, log2_table_size
    c.base_resolution, c.growth, c.max_resolution = base_resolution, growth, max_resolution
    c.hidden, c.dir_dims, c.n_samples, c.rays_per_step = 64, dir_dims, n_samples, rays_per_step
    c.lambda1, c.lambda2 = lambda1, lambda2
    c.lr, c.beta1, c.beta2, c.eps = lr, beta1, beta2, eps
    c.bg_random = 1 if bg_random else 0
    for k in range(3):
        c.bg_const[k] = bg_const[k]
    c.precision, c.max_objects, c.max_rays_per_object = precision, max_objects, max_rays_per_object
    c.accuracy_mode, c.single_net = int(accuracy_mode), 1 if single_net else 0
    c.hidden_layers, c.reserved = int(hidden_layers), 0
    c.deterministic, c.per_object = int(bool(deterministic)), int(bool(per_object))
    if alloc is not None:
        c.alloc, c.dealloc = ALLOC_FN(alloc), DEALLOC_FN(dealloc)
    return c


def object_desc(t=(0.0, 0.0, 0.0), yaw=0.0, half_size=(0.5, 0.5, 0.5), seed=0, rays_per_step=0):
    d = romap_object_desc()
    for k in range(3):
        d.t[k], d.half_size[k] = t[k], half_size[k]
    d.yaw, d.seed, d.rays_per_step = yaw, seed, rays_per_step
    return d


def param_layout(cfg):
    lay = romap_layout()
    check(romap_param_layout(C.byref(cfg), C.byref(lay)), "romap_param_layout")
    return lay


def ptr(x):
    """Address of a torch tensor or numpy array (or None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    assert x.flags["C_CONTIGUOUS"]
    return x.ctypes.data
