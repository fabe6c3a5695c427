"""ctypes wrapper of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and bench.py's CPU-baseline leg may import this
module.  It wraps oracle/romap_oracle.c (plain FP64 C, FP32 sampler stage),
which implements the per-object NeRF training step of RO-MAP (Sec. V, Eq.
6-11) and the multiresolution hash encoding it cites.  Parity of every
function is pinned in tests/test_oracle_pins.py against closed forms,
invariants, brute force and finite differences.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_LEVELS = 32
CLS_OBJECT, CLS_BACKGROUND, CLS_OCCLUDER = 0, 1, 2


class OracleConfig(C.Structure):
    _fields_ = [
        ("L", C.c_int32), ("F", C.c_int32), ("T", C.c_uint32),
        ("res", C.c_int32 * MAX_LEVELS),
        ("n_samples", C.c_int32), ("rays_per_step", C.c_int32),
        ("hidden", C.c_int32), ("geo", C.c_int32), ("dir_dims", C.c_int32),
        ("bg_random", C.c_int32),
        ("bg_const", C.c_double * 3),
        ("lambda1", C.c_double), ("lambda2", C.c_double),
        ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
        ("single_net", C.c_int32), ("hidden_layers", C.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        d, f, u32, u64, i32, i64 = C.c_double, C.c_float, C.c_uint32, C.c_uint64, C.c_int32, C.c_int64
        vp = C.c_void_p
        sig = {
            "oc_philox4x32_10": (None, [vp, vp, vp]),
            "oc_u01": (f, [u32]),
            "oc_level_resolutions": (C.c_int, [i32, d, d, d, vp]),
            "oc_level_is_dense": (C.c_int, [vp, C.c_int]),
            "oc_level_size": (u64, [vp, C.c_int]),
            "oc_level_offset": (u64, [vp, C.c_int]),
            "oc_hash_param_count": (u64, [vp]),
            "oc_mlp_layer_offset": (u64, [vp, C.c_int]),
            "oc_mlp_param_count": (u64, [vp]),
            "oc_param_count": (u64, [vp]),
            "oc_grid_index": (u32, [vp, C.c_int, u32, u32, u32]),
            "oc_init_params": (None, [vp, u64, vp]),
            "oc_world_to_object": (None, [i64, vp, vp, vp, d, vp, vp]),
            "oc_ray_aabb": (C.c_int, [vp, vp, vp, vp, vp]),
            "oc_occupied": (C.c_int, [vp, vp, vp]),
            "oc_sample_ray": (C.c_int, [vp, vp, vp, C.c_int, vp, u32, u32, C.c_int, vp, vp, vp, vp, vp, vp, vp]),
            "oc_level_corners": (None, [vp, C.c_int, vp, vp, vp, vp]),
            "oc_encode": (None, [vp, vp, vp, vp, vp]),
            "oc_mlp_forward": (None, [vp, vp, vp, vp, vp]),
            "oc_mlp_backward": (None, [vp, vp, vp, d, vp, vp, vp]),
            "oc_encode_backward": (None, [vp, vp, vp, vp, vp]),
            "oc_composite": (None, [C.c_int, vp, vp, vp, vp, vp, vp, vp]),
            "oc_composite_backward": (None, [C.c_int, vp, vp, vp, vp, vp, vp, d, d, vp, vp]),
            "oc_ray_loss": (d, [C.c_int, vp, d, vp, f, vp, d, d, d, vp, vp, vp, vp]),
            "oc_adam": (None, [i64, vp, vp, vp, vp, i64, d, d, d, d]),
            "oc_draw_batch": (i64, [vp, u64, u32, i64, vp, vp]),
            "oc_rays_loss_grad": (d, [vp, vp, vp, u64, u32, i64, C.c_int, vp, i64, vp, vp, vp, vp, vp, vp, vp, d,
                                      vp, vp, vp, vp]),
            "oc_train_step": (i64, [vp, vp, u64, u32, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int, vp, vp, vp,
                                    vp, vp, vp]),
            "oc_cell_centre": (None, [vp, C.c_int, C.c_int, C.c_int, vp]),
            "oc_density": (d, [vp, vp, vp, vp]),
            "oc_density_grid": (None, [vp, vp, vp, vp]),
            "oc_occupancy_update": (None, [i64, vp, d, d, vp, vp]),
            "oc_view_angle_deg": (d, [vp, vp, vp]),
            "oc_lattice_vertex": (None, [vp, C.c_int, C.c_int, C.c_int, vp]),
            "oc_density_lattice": (None, [vp, vp, vp, vp]),
            "oc_mesh_vertices": (i64, [vp, vp, d, vp, vp]),
            "oc_should_update": (C.c_int, [C.c_int, vp, vp, vp, d]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    """Pointer of a contiguous numpy array (or None)."""
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def level_resolutions(L, n_min, growth=0.0, n_max=0.0):
    res = np.zeros(MAX_LEVELS, np.int32)
    rc = lib().oc_level_resolutions(L, float(n_min), float(growth), float(n_max), _p(res))
    assert rc == 0
    return res[:L].copy()


def make_config(L=8, F=2, T=2 ** 12, n_min=16, growth=1.5, n_max=0.0, n_samples=32, rays_per_step=256,
                hidden=64, geo=15, dir_dims=3, bg_random=False, bg_const=(1.0, 1.0, 1.0), lambda1=0.5,
                lambda2=0.01, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15, single_net=False, hidden_layers=1):
    c = OracleConfig()
    c.L, c.F, c.T = L, F, T
    res = level_resolutions(L, n_min, growth, n_max)
    for i, r in enumerate(res):
        c.res[i] = int(r)
    c.n_samples, c.rays_per_step = n_samples, rays_per_step
    c.hidden, c.geo, c.dir_dims = hidden, geo, dir_dims
    c.bg_random = 1 if bg_random else 0
    for k in range(3):
        c.bg_const[k] = bg_const[k]
    c.lambda1, c.lambda2 = lambda1, lambda2
    c.lr, c.beta1, c.beta2, c.eps = lr, beta1, beta2, eps
    c.single_net = 1 if single_net else 0
    assert 1 <= hidden_layers <= 3 and (single_net or hidden_layers == 1)
    c.hidden_layers = int(hidden_layers)
    return c


def _cp(cfg):
    return C.addressof(cfg)


def philox(ctr, key):
    ctr = np.ascontiguousarray(ctr, np.uint32)
    key = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oc_philox4x32_10(_p(ctr), _p(key), _p(out))
    return out


def u01(x):
    return lib().oc_u01(int(x))


def param_count(cfg):
    return int(lib().oc_param_count(_cp(cfg)))


def hash_param_count(cfg):
    return int(lib().oc_hash_param_count(_cp(cfg)))


def mlp_layer_offset(cfg, layer):
    return int(lib().oc_mlp_layer_offset(_cp(cfg), layer))


def level_offset(cfg, l):
    return int(lib().oc_level_offset(_cp(cfg), l))


def level_size(cfg, l):
    return int(lib().oc_level_size(_cp(cfg), l))


def level_is_dense(cfg, l):
    return bool(lib().oc_level_is_dense(_cp(cfg), l))


def grid_index(cfg, l, cx, cy, cz):
    return int(lib().oc_grid_index(_cp(cfg), l, cx, cy, cz))


def init_params(cfg, seed):
    p = np.zeros(param_count(cfg), np.float64)
    lib().oc_init_params(_cp(cfg), seed, _p(p))
    return p


def world_to_object(o_w, d_w, t, yaw):
    o_w, d_w = _f32(o_w), _f32(d_w)
    n = o_w.size // 3
    o_o = np.zeros_like(o_w)
    d_o = np.zeros_like(d_w)
    t = _f32(t)
    lib().oc_world_to_object(n, _p(o_w), _p(d_w), _p(t), float(yaw), _p(o_o), _p(d_o))
    return o_o, d_o


def ray_aabb(o, d, half):
    o, d, half = _f32(o), _f32(d), _f32(half)
    tn = np.zeros(1, np.float32)
    tf = np.zeros(1, np.float32)
    hit = lib().oc_ray_aabb(_p(o), _p(d), _p(half), _p(tn), _p(tf))
    return bool(hit), float(tn[0]), float(tf[0])


def occupied(bits, x, half):
    x, half = _f32(x), _f32(half)
    bits = None if bits is None else np.ascontiguousarray(bits, np.uint64)
    return bool(lib().oc_occupied(_p(bits), _p(x), _p(half)))


def sample_ray(o, d, half, N, seed, step, slot, jitter=True, occ=None):
    o, d, half = _f32(o), _f32(d), _f32(half)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)
    t = np.zeros(N, np.float32)
    dl = np.zeros(N, np.float32)
    x = np.zeros(3 * N, np.float32)
    live = np.zeros(N, np.uint8)
    tn = np.zeros(1, np.float32)
    tf = np.zeros(1, np.float32)
    occ = None if occ is None else np.ascontiguousarray(occ, np.uint64)
    hit = lib().oc_sample_ray(_p(o), _p(d), _p(half), N, _p(key), step, slot, 1 if jitter else 0, _p(occ), _p(t),
                              _p(dl), _p(x), _p(live), _p(tn), _p(tf))
    return dict(hit=bool(hit), t=t, delta=dl, x=x.reshape(N, 3), live=live.astype(bool), t_near=float(tn[0]),
                t_far=float(tf[0]))


def level_corners(cfg, l, x, half):
    x, half = _f32(x), _f32(half)
    idx = np.zeros(8, np.uint32)
    w = np.zeros(8, np.float64)
    lib().oc_level_corners(_cp(cfg), l, _p(x), _p(half), _p(idx), _p(w))
    return idx, w


def encode(cfg, table, x, half):
    table = _f64(table)
    x, half = _f32(x), _f32(half)
    enc = np.zeros(cfg.L * cfg.F, np.float64)
    lib().oc_encode(_cp(cfg), _p(table), _p(x), _p(half), _p(enc))
    return enc


class _Act(C.Structure):
    _fields_ = [("enc", C.c_double * 64), ("h1", C.c_double * 128), ("hx", (C.c_double * 128) * 2),
                ("out", C.c_double * 32),
                ("cin", C.c_double * 34), ("h2", C.c_double * 128), ("h3", C.c_double * 128),
                ("logit", C.c_double * 3), ("rgb", C.c_double * 3), ("sigma", C.c_double)]


def mlp_forward(cfg, mlp, enc, direction):
    mlp, enc = _f64(mlp), _f64(enc)
    direction = _f32(direction)
    a = _Act()
    lib().oc_mlp_forward(_cp(cfg), _p(mlp), _p(enc), _p(direction), C.byref(a))
    H, G = cfg.hidden, cfg.geo
    return dict(h1=np.array(a.h1[:H]), out=np.array(a.out[:1 + G]), h2=np.array(a.h2[:H]),
                h3=np.array(a.h3[:H]), logit=np.array(a.logit[:]), rgb=np.array(a.rgb[:]), sigma=a.sigma,
                _act=a)


def mlp_backward(cfg, mlp, fwd, gsigma, grgb):
    mlp = _f64(mlp)
    grgb = _f64(grgb)
    gmlp = np.zeros(mlp.size, np.float64)
    genc = np.zeros(cfg.L * cfg.F, np.float64)
    lib().oc_mlp_backward(_cp(cfg), _p(mlp), C.byref(fwd["_act"]), float(gsigma), _p(grgb), _p(gmlp), _p(genc))
    return gmlp, genc


def encode_backward(cfg, x, half, genc, n_table):
    x, half, genc = _f32(x), _f32(half), _f64(genc)
    g = np.zeros(n_table, np.float64)
    lib().oc_encode_backward(_cp(cfg), _p(x), _p(half), _p(genc), _p(g))
    return g


def composite(sigma, delta, t, rgb, bg):
    sigma, delta, t, rgb, bg = _f64(sigma), _f64(delta), _f64(t), _f64(rgb), _f64(bg)
    n = sigma.size
    out = np.zeros(5, np.float64)
    w = np.zeros(max(n, 1), np.float64)
    lib().oc_composite(n, _p(sigma), _p(delta), _p(t), _p(rgb), _p(bg), _p(out), _p(w))
    return out, w[:n]


def composite_backward(sigma, delta, t, rgb, bg, gC, gD, gA):
    sigma, delta, t, rgb, bg, gC = _f64(sigma), _f64(delta), _f64(t), _f64(rgb), _f64(bg), _f64(gC)
    n = sigma.size
    gs = np.zeros(max(n, 1), np.float64)
    gc = np.zeros(max(3 * n, 1), np.float64)
    lib().oc_composite_backward(n, _p(sigma), _p(delta), _p(t), _p(rgb), _p(bg), _p(gC), float(gD), float(gA),
                                _p(gs), _p(gc))
    return gs[:n], gc[:3 * n].reshape(n, 3)


def adam(p, m, v, g, step, lr, beta1, beta2, eps):
    p, m, v, g = _f64(p).copy(), _f64(m).copy(), _f64(v).copy(), _f64(g)
    lib().oc_adam(p.size, _p(p), _p(m), _p(v), _p(g), step, lr, beta1, beta2, eps)
    return p, m, v


def draw_batch(cfg, seed, step, n_pool):
    cap = min(cfg.rays_per_step, n_pool)
    idx = np.zeros(max(cap, 1), np.int64)
    bg = np.zeros(3 * max(cap, 1), np.float64)
    B = lib().oc_draw_batch(_cp(cfg), seed, step, n_pool, _p(idx), _p(bg))
    return idx[:B], bg[:3 * B].reshape(B, 3)


def rays_loss_grad(cfg, params, half, seed, step, o, d, rgb=None, depth=None, cls=None, bg=None, upstream=None,
                   inv_B=None, slot0=0, jitter=True, occ=None, want_grad=True, want_samples=False):
    """Forward + loss (or upstream-weighted outputs) + backward over explicit object-frame rays."""
    params = _f64(params)
    o, d = _f32(o), _f32(d)
    n = o.size // 3
    rgb = _f32(np.zeros((n, 3)) if rgb is None else rgb)
    depth = _f32(np.full(n, np.nan) if depth is None else depth)
    cls = np.ascontiguousarray(np.zeros(n) if cls is None else cls, np.uint8)
    bg = _f64(np.ones((n, 3)) if bg is None else bg)
    up = None if upstream is None else _f64(upstream)
    if inv_B is None:
        inv_B = 1.0 / max(n, 1)
    grad = np.zeros(params.size, np.float64) if want_grad else None
    ray_out = np.zeros((n, 8), np.float64)
    sample_out = np.zeros((n, cfg.n_samples, 8), np.float64) if want_samples else None
    comps = np.zeros(4, np.float64)
    occ = None if occ is None else np.ascontiguousarray(occ, np.uint64)
    total = lib().oc_rays_loss_grad(_cp(cfg), _p(params), _p(_f32(half)), seed, step, slot0, 1 if jitter else 0,
                                    _p(occ), n, _p(o), _p(d), _p(rgb), _p(depth), _p(cls), _p(bg), _p(up),
                                    float(inv_B), _p(grad), _p(ray_out), _p(sample_out), _p(comps))
    return dict(total=total, grad=grad, ray=ray_out, samples=sample_out, comps=comps)


def train_step(cfg, half, seed, step, pool, params, m, v, occ=None, do_adam=True, want_rays=False,
               want_samples=False):
    """One step of one object.  pool: dict of object-frame SoA arrays o, d, rgb, depth, cls."""
    params, m, v = _f64(params).copy(), _f64(m).copy(), _f64(v).copy()
    o, d = _f32(pool["o"]), _f32(pool["d"])
    n_pool = o.size // 3
    rgb, depth = _f32(pool["rgb"]), _f32(pool["depth"])
    cls = np.ascontiguousarray(pool["cls"], np.uint8)
    B = min(cfg.rays_per_step, n_pool)
    grad = np.zeros(params.size, np.float64)
    loss = np.zeros(5, np.float64)
    pidx = np.zeros(B, np.int64)
    bg = np.zeros((B, 3), np.float64)
    ray_out = np.zeros((B, 8), np.float64) if want_rays else None
    sample_out = np.zeros((B, cfg.n_samples, 8), np.float64) if want_samples else None
    occ = None if occ is None else np.ascontiguousarray(occ, np.uint64)
    got = lib().oc_train_step(_cp(cfg), _p(_f32(half)), seed, step, _p(occ), n_pool, _p(o), _p(d), _p(rgb),
                              _p(depth), _p(cls), _p(params), _p(m), _p(v), 1 if do_adam else 0, _p(grad),
                              _p(loss), _p(pidx), _p(bg), _p(ray_out), _p(sample_out))
    assert got == B
    return dict(params=params, m=m, v=v, grad=grad, loss=loss, pool_idx=pidx, bg=bg, rays=ray_out,
                samples=sample_out)


def cell_centre(half, ix, iy, iz):
    """Centre of occupancy cell (ix, iy, iz) of the box [-half, half] (FP32, fixed order)."""
    x = np.zeros(3, np.float32)
    lib().oc_cell_centre(_p(_f32(half)), int(ix), int(iy), int(iz), _p(x))
    return x


def density(cfg, params, x, half):
    """sigma of the density net at one object-frame point."""
    return float(lib().oc_density(_cp(cfg), _p(_f64(params)), _p(_f32(x)), _p(_f32(half))))


def density_grid(cfg, params, half):
    """sigma at all 64^3 cell centres, index x + 64 y + 4096 z."""
    out = np.zeros(64 ** 3, np.float64)
    lib().oc_density_grid(_cp(cfg), _p(_f64(params)), _p(_f32(half)), _p(out))
    return out


def occupancy_update(sigma, decay, threshold, density_in):
    """density = max(decay * density, sigma); returns (density, 64-bit words of density > threshold)."""
    sigma = _f64(sigma)
    dens = _f64(density_in).copy()
    bits = np.zeros((sigma.size + 63) // 64, np.uint64)
    lib().oc_occupancy_update(sigma.size, _p(sigma), float(decay), float(threshold), _p(dens), _p(bits))
    return dens, bits


def view_angle_deg(t_m, t_n, t_o):
    """Eq. 5: angle between the object-to-camera vectors of the last updated and the current image, degrees."""
    return float(lib().oc_view_angle_deg(_p(_f64(t_m)), _p(_f64(t_n)), _p(_f64(t_o))))


def should_update(t_m, t_n, t_o, threshold_deg):
    """The data-update rule: True when t_m is None (no image yet) or the Eq. 5 angle exceeds the threshold."""
    if t_m is None:
        return bool(lib().oc_should_update(0, None, _p(_f64(t_n)), _p(_f64(t_o)), float(threshold_deg)))
    return bool(lib().oc_should_update(1, _p(_f64(t_m)), _p(_f64(t_n)), _p(_f64(t_o)), float(threshold_deg)))


def lattice_vertex(half, i, j, k):
    """Marching-cubes lattice vertex (i, j, k), 0..64 per axis, of the box [-half, half] (FP32, fixed order)."""
    x = np.zeros(3, np.float32)
    lib().oc_lattice_vertex(_p(_f32(half)), int(i), int(j), int(k), _p(x))
    return x


def density_lattice(cfg, params, half):
    """sigma at the 65^3 lattice vertices, index i + 65 j + 65^2 k."""
    out = np.zeros(65 ** 3, np.float64)
    lib().oc_density_lattice(_cp(cfg), _p(_f64(params)), _p(_f32(half)), _p(out))
    return out


def mesh_vertices(sigma, half, iso):
    """Edge-crossing vertices of the lattice densities: (edge codes 3 v + axis, positions [n, 3])."""
    sigma = _f64(sigma)
    n = int(lib().oc_mesh_vertices(_p(sigma), _p(_f32(half)), float(iso), None, None))
    codes = np.zeros(n, np.int64)
    pos = np.zeros((n, 3), np.float64)
    lib().oc_mesh_vertices(_p(sigma), _p(_f32(half)), float(iso), _p(codes), _p(pos))
    return codes, pos
